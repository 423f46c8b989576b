// Index persistence: the index is built once and queried many times (Methods, "Index
// Construction & Querying"), so a built device index can be written to a file and read back
// onto a device without rebuilding.
//
// File layout (native little-endian): a 128-byte header
//   "MTIDX\0\0\1" | u32 G, k, w, canonical, slot_shift, hk_db, flags | u64 total_bases, n_occ,
//   n_keys, slots, ref_words, occ_bytes | u64 check (FNV-1a of the preceding bytes) | zero pad
// then the arrays glen[G], gword[G], ref[ref_words], table[slots] (32 bytes a slot),
// occ[occ_bytes / 8], and the 8-byte trailer "MTIDXEND".
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

#include "internal.h"

namespace mt {
namespace {

constexpr char MAGIC[8] = {'M', 'T', 'I', 'D', 'X', 0, 0, 1};
constexpr char TRAILER[8] = {'M', 'T', 'I', 'D', 'X', 'E', 'N', 'D'};
constexpr size_t HEADER_BYTES = 128;
constexpr size_t STAGE_BYTES = 64ull << 20;

struct Header {
    char magic[8];
    uint32_t G, k, w, canonical, slot_shift, hk_db, flags;
    uint64_t total_bases, n_occ, n_keys, slots, ref_words, occ_bytes;
    uint64_t check;
};
static_assert(sizeof(Header) <= HEADER_BYTES, "header fits its block");

uint64_t fnv1a(const void *p, size_t n) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    uint64_t h = 0xcbf29ce484222325ull;
    for (size_t i = 0; i < n; i++) { h ^= b[i]; h *= 0x100000001b3ull; }
    return h;
}

struct File {
    FILE *f = nullptr;
    ~File() { if (f) fclose(f); }
};

struct Pinned {
    void *p = nullptr;
    ~Pinned() { if (p) cudaFreeHost(p); }
};

// device -> file through the pinned staging buffer
int write_dev(FILE *f, const void *dev, uint64_t bytes, void *stage, cudaStream_t s) {
    const char *d = static_cast<const char *>(dev);
    for (uint64_t o = 0; o < bytes; o += STAGE_BYTES) {
        const uint64_t n = std::min<uint64_t>(STAGE_BYTES, bytes - o);
        MT_CK(cudaMemcpyAsync(stage, d + o, n, cudaMemcpyDeviceToHost, s));
        MT_CK(cudaStreamSynchronize(s));
        if (fwrite(stage, 1, n, f) != n) return MT_EIO;
    }
    return MT_OK;
}

// file -> device through the pinned staging buffer
int read_dev(FILE *f, void *dev, uint64_t bytes, void *stage, cudaStream_t s) {
    char *d = static_cast<char *>(dev);
    for (uint64_t o = 0; o < bytes; o += STAGE_BYTES) {
        const uint64_t n = std::min<uint64_t>(STAGE_BYTES, bytes - o);
        if (fread(stage, 1, n, f) != n) return MT_EIO;
        MT_CK(cudaMemcpyAsync(d + o, stage, n, cudaMemcpyHostToDevice, s));
        MT_CK(cudaStreamSynchronize(s));
    }
    return MT_OK;
}

// The header's fields are consistent with an index this library can build.
bool header_ok(const Header &h) {
    if (memcmp(h.magic, MAGIC, 8) != 0) return false;
    if (h.check != fnv1a(&h, offsetof(Header, check))) return false;
    if (h.G == 0 || h.G > MT_MAX_GENOMES || h.k == 0 || h.k > MT_MAX_K || h.w == 0 || h.w > MT_MAX_W) return false;
    if (h.canonical > 1 || (h.flags & ~MT_INDEX_HPC) != 0 || h.slots == 0 || (h.slots & (h.slots - 1)) != 0) return false;
    uint32_t lg = 0;
    while ((1ull << lg) < h.slots) lg++;
    if (h.slot_shift != 64 - lg || h.n_keys > h.slots || h.n_keys > h.n_occ + 1) return false;
    if (h.ref_words != (h.total_bases >> 5) + h.G + 1) return false;
    if (h.occ_bytes != std::max<uint64_t>(1, h.n_occ) * 8) return false;
    return true;
}

}  // namespace
}  // namespace mt

using namespace mt;

extern "C" int mt_save_index(const mt_index *ix, const char *path, void *stream) {
    if (!ix || !path) return MT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Header h{};
    memcpy(h.magic, MAGIC, 8);
    h.G = ix->G; h.k = ix->k; h.w = ix->w; h.canonical = ix->canonical;
    h.slot_shift = ix->slot_shift; h.hk_db = ix->hk_db; h.flags = ix->hpc ? MT_INDEX_HPC : 0u;
    h.total_bases = ix->total_bases; h.n_occ = ix->n_occ; h.n_keys = ix->n_keys; h.slots = ix->slots;
    h.ref_words = ix->ref_words;
    h.occ_bytes = std::max<uint64_t>(1, ix->n_occ) * 8;
    h.check = fnv1a(&h, offsetof(Header, check));
    File file;
    file.f = fopen(path, "wb");
    if (!file.f) return MT_EIO;
    unsigned char block[HEADER_BYTES] = {0};
    memcpy(block, &h, sizeof(h));
    if (fwrite(block, 1, HEADER_BYTES, file.f) != HEADER_BYTES) return MT_EIO;
    if (fwrite(ix->h_glen.data(), 8, ix->G, file.f) != ix->G) return MT_EIO;
    Pinned stage;
    MT_CK(cudaMallocHost(&stage.p, STAGE_BYTES));
    int rc;
    if ((rc = write_dev(file.f, ix->d_gword, ix->G * 8ull, stage.p, s))) return rc;
    if ((rc = write_dev(file.f, ix->d_ref, ix->ref_words * 8, stage.p, s))) return rc;
    if ((rc = write_dev(file.f, ix->d_table, ix->slots * 32, stage.p, s))) return rc;
    if ((rc = write_dev(file.f, ix->d_occ, h.occ_bytes, stage.p, s))) return rc;
    if (fwrite(TRAILER, 1, 8, file.f) != 8) return MT_EIO;
    if (fflush(file.f) != 0) return MT_EIO;
    return MT_OK;
}

extern "C" int mt_load_index(const char *path, void *stream, mt_index **out) {
    if (!path || !out) return MT_EINVAL;
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    File file;
    file.f = fopen(path, "rb");
    if (!file.f) return MT_EIO;
    unsigned char block[HEADER_BYTES];
    if (fread(block, 1, HEADER_BYTES, file.f) != HEADER_BYTES) return MT_EIO;
    Header h;
    memcpy(&h, block, sizeof(h));
    if (!header_ok(h)) return MT_EIO;
    // the file must hold exactly the arrays the header announces
    const uint64_t body = h.G * 16ull + h.ref_words * 8 + h.slots * 32 + h.occ_bytes + 8;
    if (fseek(file.f, 0, SEEK_END) != 0) return MT_EIO;
    const long size = ftell(file.f);
    if (size < 0 || (uint64_t)size != HEADER_BYTES + body) return MT_EIO;
    if (fseek(file.f, (long)HEADER_BYTES, SEEK_SET) != 0) return MT_EIO;

    std::unique_ptr<mt_index, void (*)(mt_index *)> ix(new mt_index(), mt_free_index);
    ix->G = h.G; ix->k = h.k; ix->w = h.w; ix->canonical = h.canonical;
    ix->slot_shift = h.slot_shift; ix->hk_db = h.hk_db; ix->hpc = (h.flags & MT_INDEX_HPC) ? 1 : 0;
    ix->total_bases = h.total_bases; ix->n_occ = h.n_occ; ix->n_keys = h.n_keys; ix->slots = h.slots;
    ix->ref_words = h.ref_words;
    MT_CK(cudaGetDevice(&ix->device));
    ix->h_glen.resize(h.G);
    if (fread(ix->h_glen.data(), 8, h.G, file.f) != h.G) return MT_EIO;
    uint64_t sum = 0;
    for (uint64_t L : ix->h_glen) sum += L;
    if (sum != h.total_bases) return MT_EIO;
    MT_CK(cudaMalloc((void **)&ix->d_gword, h.G * 8ull));
    MT_CK(cudaMalloc((void **)&ix->d_glen, h.G * 8ull));
    MT_CK(cudaMalloc((void **)&ix->d_ref, h.ref_words * 8));
    MT_CK(cudaMalloc((void **)&ix->d_table, h.slots * 32));
    MT_CK(cudaMalloc((void **)&ix->d_occ, h.occ_bytes));
    MT_CK(cudaMemcpyAsync(ix->d_glen, ix->h_glen.data(), h.G * 8ull, cudaMemcpyHostToDevice, s));
    Pinned stage;
    MT_CK(cudaMallocHost(&stage.p, STAGE_BYTES));
    int rc;
    if ((rc = read_dev(file.f, ix->d_gword, h.G * 8ull, stage.p, s))) return rc;
    if ((rc = read_dev(file.f, ix->d_ref, h.ref_words * 8, stage.p, s))) return rc;
    if ((rc = read_dev(file.f, ix->d_table, h.slots * 32, stage.p, s))) return rc;
    if ((rc = read_dev(file.f, ix->d_occ, h.occ_bytes, stage.p, s))) return rc;
    char tr[8];
    if (fread(tr, 1, 8, file.f) != 8 || memcmp(tr, TRAILER, 8) != 0) return MT_EIO;
    if ((rc = build_key_filter(ix.get(), s))) return rc;   // derived data: rebuilt, not stored
    MT_CK(cudaStreamSynchronize(s));
    ix->device_bytes = ix->ref_words * 8 + h.G * 16ull + h.slots * 32 + h.occ_bytes + ix->filter_blocks * 8;
    *out = ix.release();
    return MT_OK;
}
