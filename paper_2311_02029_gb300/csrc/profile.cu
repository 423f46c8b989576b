// Taxonomic roll-up of a profile (Fig. 1, 3b; "Taxonomic Profile Generation"): the relative
// abundance of a taxon is the sum over the genomes below it. mt_profile_rollup is host code
// over host arrays; mt_profile_rollup_device runs on the device over the abundance vector a
// device classification left there (one thread per genome adds its abundance to every taxon
// on its path).
#include <algorithm>
#include <cstdint>
#include <vector>

#include "internal.h"

extern "C" int mt_profile_rollup(const double *abundance, uint32_t n_genomes, const uint32_t *genome_node,
                                 const int32_t *parent, uint32_t n_nodes, double *node_abundance) {
    if ((n_genomes && (!abundance || !genome_node)) || (n_nodes && (!parent || !node_abundance)))
        return MT_EINVAL;
    for (uint32_t v = 0; v < n_nodes; v++)
        if (parent[v] < -1 || parent[v] >= (int64_t)n_nodes) return MT_EINVAL;
    for (uint32_t g = 0; g < n_genomes; g++)
        if (genome_node[g] >= n_nodes) return MT_EINVAL;
    std::vector<double> acc(n_nodes, 0.0);
    for (uint32_t g = 0; g < n_genomes; g++) {
        int64_t v = genome_node[g];
        for (uint32_t depth = 0; v != -1; depth++) {
            if (depth >= n_nodes) return MT_EINVAL;     // the parent links hold a cycle
            acc[(size_t)v] += abundance[g];
            v = parent[v];
        }
    }
    for (uint32_t v = 0; v < n_nodes; v++) node_abundance[v] = acc[v];
    return MT_OK;
}

namespace {

// One thread per genome: its abundance is added to every taxon on its path to a root. A node
// out of range, or a path longer than the node count (a cycle), sets err.
__global__ void k_rollup(const double *a, uint32_t G, const uint32_t *genome_node, const int32_t *parent, uint32_t T,
                         double *out, uint32_t *err) {
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G; g += (uint64_t)gridDim.x * blockDim.x) {
        int64_t v = genome_node[g];
        const double x = a[g];
        for (uint32_t steps = 0; v != -1; steps++) {
            if (v < 0 || v >= (int64_t)T || steps >= T) {
                atomicOr(err, 1u);
                break;
            }
            atomicAdd(&out[v], x);
            v = parent[v];
        }
    }
}

}  // namespace

extern "C" int mt_profile_rollup_device(const double *abundance, uint32_t n_genomes, const uint32_t *genome_node,
                                        const int32_t *parent, uint32_t n_nodes, double *node_abundance,
                                        void *stream) {
    if ((n_genomes && (!abundance || !genome_node)) || (n_nodes && (!parent || !node_abundance)) ||
        (n_genomes && !n_nodes))
        return MT_EINVAL;
    mt::Trace trace("mt_profile_rollup_device");
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *err = nullptr;
    int rc = mt::dalloc((void **)&err, 4, s);
    if (rc) return rc;
    uint32_t h = 0;
    bool ok = mt::cuda_ok(cudaMemsetAsync(err, 0, 4, s), "rollup err") &&
              (!n_nodes || mt::cuda_ok(cudaMemsetAsync(node_abundance, 0, n_nodes * 8ull, s), "rollup out"));
    if (ok && n_genomes) {
        const unsigned blocks = (unsigned)std::min<uint64_t>((n_genomes + 255) / 256, (uint64_t)mt::sm_count() * 4);
        k_rollup<<<blocks, 256, 0, s>>>(abundance, n_genomes, genome_node, parent, n_nodes, node_abundance, err);
        ok = mt::cuda_ok(cudaGetLastError(), "k_rollup");
    }
    ok = ok && mt::cuda_ok(cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, s), "rollup err") &&
         mt::cuda_ok(cudaStreamSynchronize(s), "rollup");
    mt::dfree(err, s);
    if (!ok) return MT_ECUDA;
    return h ? MT_EINVAL : MT_OK;
}
