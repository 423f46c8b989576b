"""GPU parity of the edit-distance-approximation stage alone (mt_pack_seqs + mt_eda_batch)
against the oracle, in both execution forms."""
import numpy as np
import pytest

import gen
import oracle

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


def np_pack(seq: np.ndarray, off: np.ndarray) -> np.ndarray:
    """Reference of the documented packed layout: base j of sequence i at bits 2*(j%32) of
    word (off[i] >> 5) + i + j // 32, codes A0 C1 G2 T3."""
    code = np.zeros(256, np.uint64)
    for i, b in enumerate(b"ACGT"):
        code[b] = i
    n = len(off) - 1
    words = np.zeros(int(off[-1]) // 32 + n + 1, np.uint64)
    for i in range(n):
        s = seq[int(off[i]):int(off[i + 1])]
        base = int(off[i]) // 32 + i
        for j in range(0, len(s), 32):
            c = code[s[j:j + 32]]
            words[base + j // 32] = np.bitwise_or.reduce(c << (2 * np.arange(len(c), dtype=np.uint64)))
    return words


def to_dev(pairs, mt):
    import torch
    dev = "cuda"
    rs = torch.from_numpy(pairs.read_seq).to(dev)
    ro = torch.from_numpy(pairs.read_off.astype(np.int64)).to(dev)
    ws = torch.from_numpy(pairs.win_seq).to(dev)
    wo = torch.from_numpy(pairs.win_off.astype(np.int64)).to(dev)
    rw = mt.pack_seqs(rs, ro, mt.packed_words(pairs.read_off))
    ww = mt.pack_seqs(ws, wo, mt.packed_words(pairs.win_off))
    pr = torch.from_numpy(pairs.pair_read.astype(np.int32)).to(dev)
    E = torch.from_numpy(pairs.E.astype(np.int16)).to(dev)
    return rw, ro, ww, wo, pr, E


def test_pack_matches_layout(mt):
    import torch
    rng = np.random.default_rng(1)
    lens = rng.integers(0, 100, 300)
    off = np.zeros(301, np.uint64)
    off[1:] = np.cumsum(lens) + 7          # non-zero first offset
    off[0] = 7
    seq = gen.ascii_of(rng.integers(0, 4, int(off[-1]), dtype=np.uint8))
    words = mt.pack_seqs(torch.from_numpy(seq).cuda(), torch.from_numpy(off.astype(np.int64)).cuda(),
                         mt.packed_words(off))
    exp = np_pack(seq, off)
    got = words.cpu().numpy().view(np.uint64)
    # words before the first sequence are not part of the layout
    first = int(off[0]) // 32
    assert np.array_equal(got[first:], exp[first:])


def test_pack_rejects_bad_bases(mt):
    import torch
    seq = np.frombuffer(b"ACGTNACGT", np.uint8).copy()
    off = np.array([0, 9], np.int64)
    with pytest.raises(mt.MtError):
        mt.pack_seqs(torch.from_numpy(seq).cuda(), torch.from_numpy(off).cuda(), 2)


@pytest.mark.parametrize("mode", [0, 1])
def test_eda_batch_matches_oracle(mt, mode):
    """Reads of 100-250 bp, E in {2,4,6,10}% of n, 70% of windows within E planted edits."""
    pairs = gen.make_eda_pairs(gen.config(3), n_pairs=200_000, seed=77)
    dist = mt.eda_batch(*to_dev(pairs, mt), mode=mode).cpu().numpy()
    ref = oracle.eda_batch(pairs, threads=8)
    bad = np.flatnonzero(dist != ref)
    assert len(bad) == 0, "%d pairs differ, first %s gpu %s oracle %s" % (len(bad), bad[:5], dist[bad[:5]], ref[bad[:5]])
    assert 0.3 < (ref <= pairs.E).mean() < 0.95


def test_eda_batch_extreme_shapes(mt):
    """E = 0 and E = 127, reads of 1 and 1024 bases, in one call (several classes)."""
    rng = np.random.default_rng(3)
    reads, wins, pr, Es = [], [], [], []
    for i in range(600):
        n = int(rng.choice([1, 2, 31, 32, 33, 64, 500, 1024]))
        E = int(rng.choice([0, 1, 5, 31, 64, 127]))
        r = gen.ascii_of(rng.integers(0, 4, n, dtype=np.uint8))
        w = gen.ascii_of(rng.integers(0, 4, n + 2 * E, dtype=np.uint8))
        if i % 2:
            s = int(rng.integers(0, 2 * E + 1))
            w[s:s + n] = r
            if n > 4:
                w[s + n // 2] = ord("A") if r[n // 2] != ord("A") else ord("C")
        reads.append(r)
        wins.append(w)
        pr.append(i)
        Es.append(E)
    pairs = gen.EdaPairs(read_seq=np.concatenate(reads), read_off=np.cumsum([0] + [len(x) for x in reads]).astype(np.uint64),
                         win_seq=np.concatenate(wins), win_off=np.cumsum([0] + [len(x) for x in wins]).astype(np.uint64),
                         pair_read=np.array(pr, np.uint32), E=np.array(Es, np.uint16), planted=np.zeros(len(pr), np.uint16))
    ref = oracle.eda_batch(pairs)
    for mode in (0, 1):
        dist = mt.eda_batch(*to_dev(pairs, mt), mode=mode).cpu().numpy()
        assert np.array_equal(dist, ref), mode


def test_eda_batch_rejects_bad_pairs(mt):
    import torch
    pairs = gen.make_eda_pairs(gen.config(3), n_pairs=1000, seed=5)
    rw, ro, ww, wo, pr, E = to_dev(pairs, mt)
    E2 = E.clone()
    E2[10] += 1                      # window length no longer n + 2E
    with pytest.raises(mt.MtError):
        mt.eda_batch(rw, ro, ww, wo, pr, E2)
    E3 = E.clone()
    E3[3] = 200                      # above MT_MAX_E
    with pytest.raises(mt.MtError):
        mt.eda_batch(rw, ro, ww, wo, pr, E3)
    d = mt.eda_batch(rw, ro, ww, wo, pr, E)   # still usable
    assert d.numel() == 1000
    torch.cuda.synchronize()


def test_autotune_reports_keeps_and_does_not_change_results(mt):
    """mt_eda_batch_autotune times the batched kernel's shapes per edit-threshold class and keeps
    the fastest: the shapes it reports are valid, mt_eda_shape_for returns them afterwards, and
    the distances (tuned call, later untuned batched call, plain call) equal the oracle's, also
    with the extreme shapes (E = 0 and E = 127 in one call)."""
    pairs = gen.make_eda_pairs(gen.config(3), n_pairs=300_000, seed=91)
    dev = to_dev(pairs, mt)
    ref = oracle.eda_batch(pairs, threads=8)
    dist, shapes = mt.eda_batch_autotune(*dev)
    assert np.array_equal(dist.cpu().numpy(), ref)
    present = sorted({int(e).bit_length() - 1 if e >= 2 else 0 for e in np.unique(pairs.E)})
    for c in range(mt.EDA_CLASSES):
        sh = shapes[c]
        if c in present:
            assert sh["lanes_per_pair"] in (1, 2, 4, 8, 16, 32) and sh["tuned"] == 1
            assert sh["pairs_per_chunk"] in (32, 64, 128, 256) and sh["cta_threads"] in (128, 256, 512, 1024)
            assert sh["refill"] in (0, 1) and (sh["refill"] == 0 or sh["lanes_per_pair"] == 1)
        else:
            assert sh == {"lanes_per_pair": 0, "pairs_per_chunk": 0, "cta_threads": 0, "refill": 0, "tuned": 0}
    for e in np.unique(pairs.E):
        c = int(e).bit_length() - 1 if e >= 2 else 0
        got = mt.eda_shape_for(0, False, int(e))
        assert got == shapes[c]
    for mode in (mt.MT_EDA_BATCHED, mt.MT_EDA_PLAIN):
        assert np.array_equal(mt.eda_batch(*dev, mode=mode).cpu().numpy(), ref)


def test_classify_tunes_only_when_asked(mt):
    """mt_classify never times shapes (the kept shape stays the default); mt_classify_autotune
    tunes the batch's class, reports the shape it used, keeps it for later calls, and every
    call's outputs equal the oracle's."""
    from helpers import compare_classify, oracle_params
    c = gen.config(2, n_genomes=20, genome_len=100_000, n_reads=20_000)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    prm = dict(e_abs=31, e_permille=0, min_seeds=3, top_n=3, max_occ=1024)   # a class no other test tunes
    ref = oracle.classify(oix, r.seq, r.offsets, oracle_params(prm), threads=8)
    before = mt.eda_shape_for(0, True, 31)
    assert before["tuned"] == 0
    compare_classify(mt.classify(ix, r.seq, r.offsets, **prm), ref)
    assert mt.eda_shape_for(0, True, 31) == before
    out = mt.classify_autotune(ix, r.seq, r.offsets, **prm)
    compare_classify(out, ref)
    sh = out["eda_shape"]
    assert sh["tuned"] == 1 and sh["lanes_per_pair"] in (1, 2, 4, 8, 16, 32)
    kept = mt.eda_shape_for(0, True, 31)
    assert kept["tuned"] == 1 and kept["pairs_per_chunk"] == sh["pairs_per_chunk"] and kept["cta_threads"] == sh["cta_threads"]
    compare_classify(mt.classify(ix, r.seq, r.offsets, **prm), ref)
    ix.close()


def _all_class_pairs(seed):
    """Pairs of every edit-threshold class ([0,1] ... [64,127]) and lengths 1 to 1024, half of
    them within a few substitutions of a window offset."""
    rng = np.random.default_rng(seed)
    reads, wins, Es = [], [], []
    for i in range(700):
        n = int(rng.choice([1, 5, 32, 33, 150, 251, 1024]))
        E = int(rng.choice([0, 1, 2, 3, 4, 7, 8, 15, 16, 31, 32, 63, 64, 127]))
        r = gen.ascii_of(rng.integers(0, 4, n, dtype=np.uint8))
        w = gen.ascii_of(rng.integers(0, 4, n + 2 * E, dtype=np.uint8))
        if i % 2:
            s = int(rng.integers(0, 2 * E + 1))
            w[s:s + n] = r
            for _ in range(int(rng.integers(0, 5))):
                j = s + int(rng.integers(0, n))
                w[j] = ord("A") if w[j] != ord("A") else ord("T")
        reads.append(r)
        wins.append(w)
        Es.append(E)
    return gen.EdaPairs(read_seq=np.concatenate(reads), read_off=np.cumsum([0] + [len(x) for x in reads]).astype(np.uint64),
                        win_seq=np.concatenate(wins), win_off=np.cumsum([0] + [len(x) for x in wins]).astype(np.uint64),
                        pair_read=np.arange(len(reads), dtype=np.uint32), E=np.array(Es, np.uint16),
                        planted=np.zeros(len(reads), np.uint16))


CLASS_E = [0, 2, 4, 8, 16, 32, 64]          # one edit threshold of each class that can occur
ALGO_BITS = [(0x00, 0), (0x10, 1), (0x20, 2), (0x30, 3), (0x40, 4)]


def _shapes(bits):
    if bits == 0x30:                          # q-gram: a whole warp per pair
        lanes = [(32, 0)]
    else:
        lanes = [(G, 0) for G in (1, 2, 4, 8, 16, 32)] + ([(1, 1)] if bits == 0 else [])
    return [(G, ch, cta, rf) for G, rf in lanes for ch, cta in ((1, 32), (7, 96), (128, 256), (4096, 1024))]


@pytest.mark.parametrize("bits,algo", ALGO_BITS)
def test_every_kept_shape_gives_the_oracles_distances(mt, bits, algo):
    """mt_eda_set_shape: every valid shape (lanes per pair, refilled lanes, pairs per steal from
    1 to 4096, CTAs of 1 to 32 warps), each class of one call on a different shape (so a call
    mixes refilled and lockstep launches and widened groups), gives the oracle's distances;
    mt_eda_shape_for reports what was kept and lanes_per_pair = 0 brings the default back."""
    pairs = _all_class_pairs(40 + algo)
    dev = to_dev(pairs, mt)
    ref = oracle.eda_batch(pairs, threads=8, algo=algo)
    shapes = _shapes(bits)
    try:
        for i in range(len(shapes)):
            for c, e in enumerate(CLASS_E):
                mt.eda_set_shape(bits, False, e, *shapes[(i + c) % len(shapes)])
            got = mt.eda_shape_for(bits, False, CLASS_E[0])
            G, ch, cta, rf = shapes[i]
            assert got == {"lanes_per_pair": G, "pairs_per_chunk": ch, "cta_threads": cta, "refill": rf, "tuned": 1}
            dist = mt.eda_batch(*dev, mode=bits).cpu().numpy()
            bad = np.flatnonzero(dist != ref)
            assert len(bad) == 0, (shapes[i], bad[:5], dist[bad[:5]], ref[bad[:5]])
    finally:
        for e in CLASS_E:
            mt.eda_set_shape(bits, False, e, 0)
    assert all(mt.eda_shape_for(bits, False, e)["tuned"] == 0 for e in CLASS_E)
    assert np.array_equal(mt.eda_batch(*dev, mode=bits).cpu().numpy(), ref)


def test_classification_on_kept_shapes(mt):
    """A classification runs the shape kept for its class (refilled lanes, one-pair steals on
    one-warp CTAs, whole-warp groups) and its outputs equal the oracle's on every one."""
    from helpers import compare_classify, oracle_params
    c = gen.config(2, n_genomes=20, genome_len=100_000, n_reads=20_000)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    prm = dict(e_abs=12, e_permille=0, min_seeds=3, top_n=3, max_occ=1024)
    ref = oracle.classify(oix, r.seq, r.offsets, oracle_params(prm), threads=8)
    try:
        for shape in ((1, 64, 256, 1), (1, 1, 32, 0), (4, 4096, 1024, 0), (32, 7, 96, 0)):
            mt.eda_set_shape(0, True, 12, *shape)
            compare_classify(mt.classify(ix, r.seq, r.offsets, **prm), ref)
    finally:
        mt.eda_set_shape(0, True, 12, 0)
        ix.close()
    assert mt.eda_shape_for(0, True, 12)["tuned"] == 0
