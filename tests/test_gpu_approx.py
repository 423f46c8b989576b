"""GPU parity of the pipeline's other edit-distance approximations (HD, Base Counting, q-gram,
SHD; Table 1) against the oracle: the EDA stage alone on batching pairs and on extreme shapes,
and whole classifications, in both execution forms."""
import numpy as np
import pytest

import gen
import oracle
from helpers import compare_classify, oracle_params
from test_gpu_eda import to_dev

pytestmark = pytest.mark.gpu

ALGOS = [("hamming", 0x10, 1), ("base_counting", 0x20, 2), ("qgram", 0x30, 3), ("shd", 0x40, 4)]


@pytest.fixture(scope="module")
def mt():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2311_02029_gb300 import _build
    _build.build()
    import paper_2311_02029_gb300 as m
    oracle.build()
    return m


@pytest.fixture(scope="module")
def batching(mt):
    pairs = gen.make_eda_pairs(gen.config(3), n_pairs=100_000, seed=91)
    return pairs, to_dev(pairs, mt)


@pytest.mark.parametrize("name,bits,algo", ALGOS)
def test_batch_matches_oracle(mt, batching, name, bits, algo):
    pairs, dev = batching
    ref = oracle.eda_batch(pairs, threads=8, algo=algo)
    for form in (0, 1):
        dist = mt.eda_batch(*dev, mode=bits | form).cpu().numpy()
        bad = np.flatnonzero(dist != ref)
        assert len(bad) == 0, "%s form %d: %d pairs differ, first %s gpu %s oracle %s" % (
            name, form, len(bad), bad[:5], dist[bad[:5]], ref[bad[:5]])
    assert (ref <= pairs.E.astype(np.int64) + 1).all() and (ref <= pairs.E).any()


def _extreme_pairs(seed):
    rng = np.random.default_rng(seed)
    reads, wins, Es = [], [], []
    for i in range(500):
        n = int(rng.choice([1, 2, 4, 5, 6, 31, 32, 33, 64, 65, 500, 1024]))
        E = int(rng.choice([0, 1, 2, 5, 31, 64, 127]))
        r = gen.ascii_of(rng.integers(0, 4, n, dtype=np.uint8))
        w = gen.ascii_of(rng.integers(0, 4, n + 2 * E, dtype=np.uint8))
        if i % 2:
            s = int(rng.integers(0, 2 * E + 1))
            w[s:s + n] = r
            for _ in range(int(rng.integers(0, 4))):
                j = s + int(rng.integers(0, n))
                w[j] = ord("A") if w[j] != ord("A") else ord("G")
        reads.append(r)
        wins.append(w)
        Es.append(E)
    return gen.EdaPairs(read_seq=np.concatenate(reads), read_off=np.cumsum([0] + [len(x) for x in reads]).astype(np.uint64),
                        win_seq=np.concatenate(wins), win_off=np.cumsum([0] + [len(x) for x in wins]).astype(np.uint64),
                        pair_read=np.arange(len(reads), dtype=np.uint32), E=np.array(Es, np.uint16),
                        planted=np.zeros(len(reads), np.uint16))


@pytest.mark.parametrize("name,bits,algo", ALGOS)
def test_batch_extreme_shapes(mt, name, bits, algo):
    """Reads of 1 to 1024 bases (shorter than q, block edges), E from 0 to 127."""
    pairs = _extreme_pairs(5 + algo)
    ref = oracle.eda_batch(pairs, algo=algo)
    for form in (0, 1):
        dist = mt.eda_batch(*to_dev(pairs, mt), mode=bits | form).cpu().numpy()
        assert np.array_equal(dist, ref), (name, form, np.flatnonzero(dist != ref)[:5])


@pytest.fixture(scope="module")
def tiny(mt):
    c = gen.config(1)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    return c, g, r, ix, oix


@pytest.fixture(scope="module")
def clade(mt):
    c = gen.config(2, n_genomes=20, genome_len=100_000, n_reads=20_000)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    return c, g, r, ix, oix


@pytest.mark.parametrize("name,bits,algo", ALGOS)
@pytest.mark.parametrize("work", ["tiny", "clade"])
def test_classification_matches_oracle(mt, request, work, name, bits, algo):
    """Whole classifications with each approximation, both forms; the clade workload's reads
    come from both strands, so reverse-complemented reads and windows at genome ends occur."""
    c, g, r, ix, oix = request.getfixturevalue(work)
    prm = dict(e_abs=c["e_abs"], e_permille=c["e_permille"], min_seeds=c["min_seeds"], top_n=3, max_occ=1024,
               cont_num=1, cont_den=10000, abund_cutoff=1e-4, eda_mode=bits)
    ref = oracle.classify(oix, r.seq, r.offsets, oracle_params(prm), threads=8)
    for form in (0, 1):
        out = mt.classify(ix, r.seq, r.offsets, **dict(prm, eda_mode=bits | form))
        compare_classify(out, ref)
    assert (ref["taxon"] >= 0).mean() > 0.5


def test_invalid_modes_are_rejected(mt, tiny):
    c, g, r, ix, oix = tiny
    for mode in (2, 0x50, 0x12):
        with pytest.raises(mt.MtError):
            mt.classify(ix, r.seq[:300], r.offsets[:3], eda_mode=mode)
