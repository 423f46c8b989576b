// Host-side definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace mt {

// NVTX ranges (host-side, shown by Nsight Systems and ncu's range filters; no cost without a
// tool attached): Trace covers one scope, StageTrace a sequence of stages in one scope.
struct Trace {
    explicit Trace(const char *name) { nvtxRangePushA(name); }
    ~Trace() { nvtxRangePop(); }
    Trace(const Trace &) = delete;
    Trace &operator=(const Trace &) = delete;
};
struct StageTrace {
    bool open = false;
    void next(const char *name) {
        if (open) nvtxRangePop();
        nvtxRangePushA(name);
        open = true;
    }
    ~StageTrace() {
        if (open) nvtxRangePop();
    }
};

void set_cuda_error(cudaError_t e, const char *what);
bool cuda_ok(cudaError_t e, const char *what);

#define MT_CK(call)                                     \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (!::mt::cuda_ok(e_, #call)) return MT_ECUDA; \
    } while (0)

int sm_count();
const char *last_cuda_error();

// Stream-ordered device allocation from the default memory pool (kept cached).
int dalloc(void **p, size_t bytes, cudaStream_t s);
// True when an injected allocation failure (mt_inject_alloc_failure) is due now; every
// allocation of the library's calls asks once.
bool alloc_fault();
void dfree(void *p, cudaStream_t s);

// Carves aligned sub-buffers out of one allocation.
struct Carver {
    size_t off = 0;
    template <typename T>
    size_t take(uint64_t count) {
        size_t o = (off + 255) & ~size_t(255);
        off = o + count * sizeof(T);
        return o;
    }
};

}  // namespace mt

struct mt_index {
    int device = 0;
    uint32_t G = 0, k = 0, w = 0, canonical = 0;
    uint64_t total_bases = 0, n_occ = 0, n_keys = 0, slots = 0;
    uint32_t slot_shift = 0;
    uint32_t hk_db = 0;          // diagonal bits of 32-bit match keys; 0 if they do not fit
    uint32_t hpc = 0;            // built over homopolymer-compressed genomes (containment only)
    uint64_t ref_words = 0;
    uint64_t *d_ref = nullptr, *d_gword = nullptr, *d_glen = nullptr, *d_occ = nullptr;
    ulonglong2 *d_table = nullptr;
    uint64_t *d_filter = nullptr;   // key filter, filter_blocks 64-bit blocks (derived from the table)
    uint64_t filter_blocks = 0;
    uint32_t filter_shift = 0;
    uint64_t device_bytes = 0;
    std::vector<uint64_t> h_glen;

    IndexView view() const {
        IndexView v;
        v.table = d_table;
        v.slot_mask = slots - 1;
        v.slot_shift = slot_shift;
        v.G = G;
        v.occ = d_occ;
        v.ref = d_ref;
        v.gword = d_gword;
        v.glen = d_glen;
        v.k = k; v.w = w; v.canonical = canonical; v.hk_db = hk_db;
        return v;
    }
};

// Kernel launch helpers implemented in the .cu files.
namespace mt {
// Device scratch of one mt_classify call with host buffers and a known longest read.
uint64_t classify_ws_bytes(const mt_index *ix, uint64_t n_bases, uint64_t n_reads,
                           const mt_classify_params *p, uint32_t maxn, bool host_io);
int launch_pack_seqs(const uint8_t *seq, const uint64_t *off, uint64_t n, uint64_t *words,
                     uint64_t total_words, uint32_t *err, cudaStream_t s);
// (Re)builds the index's key filter from its table (after a build or a load).
int build_key_filter(mt_index *ix, cudaStream_t s);
// Seed hits of several indexes (at most MULTI_MAX_INDEXES, so that a (minimizer, index) pair
// number divided by their count stays exact with a 32-bit multiply) of one (k, w, canonical,
// compression) in one pass over device reads; hits (device) gets the indexes' genome counters
// one after another.
constexpr uint32_t MULTI_MAX_INDEXES = 4096;
int contain_multi(const mt_index *const *batches, uint32_t n_batches, const uint8_t *reads, uint64_t n_bases,
                  const uint64_t *offsets, uint64_t n_reads, uint32_t max_occ, uint64_t *hits, cudaStream_t s);
// Per-read location lists of R genome shards (device, rank order) merged by rank and decided:
// taxon / nloc / locs (device, n_reads entries) and abundance (device, G).
int merge_decide(const mt_loc *lists, uint32_t R, const uint64_t *roff, uint64_t n_reads, uint32_t G,
                 const mt_classify_params *p, int32_t *taxon, uint8_t *nloc, mt_loc *locs, double *abundance,
                 cudaStream_t s);
// The argument checks of mt_classify's parameters (MT_OK or MT_EINVAL).
int check_classify_params(const mt_classify_params *p);
// keep[g] = (hits[g] * cont_den > max(hits) * cont_num), on the device
int launch_mask(const uint64_t *hits, uint32_t G, uint32_t cont_num, uint32_t cont_den, uint8_t *keep,
                cudaStream_t s);
}
