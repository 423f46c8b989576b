"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle on the same
seeded inputs and compare element by element."""
import numpy as np

import oracle

FIELDS = ("genome", "seeds", "strand", "dist", "wstart")
ABUND_TOL = 1e-6     # absolute; every other output must match bit for bit


def oracle_params(prm: dict) -> dict:
    keys = ("max_occ", "e_abs", "e_permille", "min_seeds", "top_n", "cont_num", "cont_den", "abund_cutoff")
    p = oracle.params(**{k: prm[k] for k in keys if k in prm})
    p["eda_algo"] = (prm.get("eda_mode", 0) >> 4) & 15   # the library's mode: form | algorithm << 4
    return p


def as_np(x):
    if x is None:
        return None
    if type(x).__module__.startswith("torch"):
        return x.cpu().numpy()
    return x


def compare_classify(gpu: dict, ref: dict, idx=None, check_global=True):
    """Bit-exact per-read outputs (taxon, nloc, every location field) and containment
    counts; abundances within ABUND_TOL."""
    import paper_2311_02029_gb300 as mt
    taxon = as_np(gpu["taxon"])
    nloc = as_np(gpu["nloc"])
    locs = gpu["locs"]
    if locs is not None and type(locs).__module__.startswith("torch"):
        locs = mt.locs_from_device(locs)
    if idx is not None:
        taxon, nloc, locs = taxon[idx], nloc[idx], locs[idx]
    bad = np.flatnonzero(taxon != ref["taxon"])
    assert len(bad) == 0, "taxon differs at %d reads, first %s: gpu %s oracle %s" % (
        len(bad), bad[:5], taxon[bad[:5]], ref["taxon"][bad[:5]])
    assert np.array_equal(nloc, ref["nloc"]), "nloc differs"
    for f in FIELDS:
        d = np.flatnonzero((locs[f] != ref["locs"][f]).any(axis=1))
        assert len(d) == 0, "locs.%s differs at %d reads, first %d: gpu %s oracle %s" % (
            f, len(d), d[0], locs[d[0]], ref["locs"][d[0]])
    if check_global:
        gh = as_np(gpu["genome_hits"]).astype(np.uint64)
        assert np.array_equal(gh, ref["genome_hits"]), "genome hits differ"
        ab = as_np(gpu["abundance"])
        err = np.abs(ab - ref["abundance"]).max() if len(ab) else 0.0
        assert err <= ABUND_TOL, "abundance differs by %g" % err
