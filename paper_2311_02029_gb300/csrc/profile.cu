// Taxonomic roll-up of a profile (Fig. 1, 3b; "Taxonomic Profile Generation"): the relative
// abundance of a taxon is the sum over the genomes below it. Host code: the profile is one
// value per genome, produced by the last classification kernel.
#include <cstdint>
#include <vector>

#include "../../include/mt.h"

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
