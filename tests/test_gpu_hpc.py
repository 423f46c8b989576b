"""GPU parity of containment alone (mt_containment) and of mapping under a given genome mask
(mt_classify_masked), with the paper's containment seeds: an index over homopolymer-compressed
genomes with k = 28, w = 18 (minimap2's -H). Hits and masks bit-exact against the oracle; reads
with homopolymer-length errors, long runs and reads that compress below k included."""
import numpy as np
import pytest

import gen
import oracle
from helpers import compare_classify, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mt():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2311_02029_gb300 import _build
    _build.build()
    import paper_2311_02029_gb300 as m
    oracle.build()
    return m


def _stretched_reads(rng, r, frac=0.5):
    """Some reads with every homopolymer run lengthened or shortened by one, plus reads made of
    long runs (which compress below k)."""
    out = []
    for i in range(r.n):
        s = r.seq[int(r.offsets[i]):int(r.offsets[i + 1])].tobytes()
        if rng.random() < frac:
            parts, j = [], 0
            while j < len(s):
                e = j
                while e < len(s) and s[e] == s[j]:
                    e += 1
                parts.append(s[j:j + 1] * max(1, (e - j) + int(rng.integers(-1, 2))))
                j = e
            s = b"".join(parts)[:1024]
        out.append(s)
    for L in (1, 5, 40, 300):
        out.append(b"".join(bytes([b"ACGT"[int(x)]]) * L for x in rng.integers(0, 4, 60))[:1024])
    seq = np.frombuffer(b"".join(out), np.uint8).copy()
    off = np.cumsum([0] + [len(x) for x in out]).astype(np.uint64)
    return seq, off


@pytest.fixture(scope="module")
def work(mt):
    c = gen.config(2, n_genomes=20, genome_len=100_000, n_reads=20_000)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    rng = np.random.default_rng(17)
    seq, off = _stretched_reads(rng, r)
    return c, g, seq, off


def test_containment_with_the_mapping_index(mt, work):
    c, g, seq, off = work
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    out = mt.containment(ix, seq, off, max_occ=1024, cont_num=1, cont_den=10)
    hits = oracle.count_hits(oix, seq, off, 1024)
    assert np.array_equal(out["genome_hits"], hits)
    assert np.array_equal(out["keep"], oracle.keep_mask(hits, 1, 10))


def test_compressed_containment_index(mt, work):
    import torch
    c, g, seq, off = work
    hix = mt.Index(g.seq, g.offsets, 28, 18, 1, hpc=True)
    ohix = oracle.Index(g.seq, g.offsets, 28, 18, 1, compressed=True)
    info = hix.info()
    assert info["flags"] == mt.MT_INDEX_HPC and info["n_occ"] == ohix.n_occ
    assert info["total_bases"] < int(g.offsets[-1])
    hits = oracle.count_hits(ohix, seq, off, 1024)
    assert hits.sum() > 0
    for cut in ((1, 10000), (1, 10), (1, 2)):
        out = mt.containment(hix, seq, off, max_occ=1024, cont_num=cut[0], cont_den=cut[1])
        assert np.array_equal(out["genome_hits"], hits)
        assert np.array_equal(out["keep"], oracle.keep_mask(hits, *cut))
    dev = mt.containment(hix, torch.from_numpy(seq).cuda(), torch.from_numpy(off.astype(np.int64)).cuda(),
                         max_occ=1024, cont_den=10)
    assert np.array_equal(dev["genome_hits"].cpu().numpy().view(np.uint64), hits)
    # a small max_occ filters repeated seeds the same way
    assert np.array_equal(mt.containment(hix, seq, off, max_occ=2)["genome_hits"], oracle.count_hits(ohix, seq, off, 2))


def test_mapping_under_the_compressed_containment_mask(mt, work):
    c, g, seq, off = work
    hix = mt.Index(g.seq, g.offsets, 28, 18, 1, hpc=True)
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    keep = mt.containment(hix, seq, off, cont_num=1, cont_den=4)["keep"]
    assert 0 < keep.sum() <= len(keep)
    prm = dict(e_abs=c["e_abs"], e_permille=0, min_seeds=3, top_n=3, max_occ=1024, abund_cutoff=1e-4)
    out = mt.classify_masked(ix, seq, off, keep, **prm)
    ref = oracle.classify(oix, seq, off, oracle_params(prm), threads=8, keep=keep)
    compare_classify(out, ref)
    with pytest.raises(mt.MtError):
        mt.classify(hix, seq[:300], off[:3], **prm)          # a containment index cannot map
