"""GPU parity of the classification path (mt_build_index + mt_classify) against the oracle:
every per-read decision, location, seed count and distance bit-exact, genome hit counts
bit-exact, abundances within 1e-6 absolute."""
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


def _params(c, **kw):
    p = dict(e_abs=c["e_abs"], e_permille=c["e_permille"], min_seeds=c["min_seeds"], top_n=3, max_occ=1024,
             cont_num=1, cont_den=10000, abund_cutoff=1e-4)
    p.update(kw)
    return p


@pytest.fixture(scope="module")
def tiny(mt):
    c = gen.config(1)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    return c, g, r, ix, oix


@pytest.mark.parametrize("mode", [0, 1])
def test_tiny_workload_host_buffers(mt, tiny, mode):
    """8 x 50 kb genomes, k15 w10, 10,000 reads of 150 bp, E = 6, seed threshold 2."""
    c, g, r, ix, oix = tiny
    prm = _params(c)
    ref = oracle.classify(oix, r.seq, r.offsets, oracle_params(prm))
    out = mt.classify(ix, r.seq, r.offsets, eda_mode=mode, **prm)
    compare_classify(out, ref)
    assert out["stats"]["n_reads"] == r.n
    assert (ref["taxon"] >= 0).mean() > 0.85


def test_tiny_workload_device_buffers(mt, tiny):
    import torch
    c, g, r, ix, oix = tiny
    prm = _params(c)
    ref = oracle.classify(oix, r.seq, r.offsets, oracle_params(prm))
    out = mt.classify(ix, torch.from_numpy(r.seq).cuda(), torch.from_numpy(r.offsets.astype(np.int64)).cuda(), **prm)
    compare_classify(out, ref)


@pytest.mark.parametrize("shift", [0, 3])
def test_device_reads_mid_buffer(mt, tiny, shift):
    """A batch whose first read starts inside the device buffer, with the buffer at an aligned
    address (vector loads and prefetch) and at an odd one (byte loads)."""
    import torch
    c, g, r, ix, oix = tiny
    prm = _params(c)
    a, b = 1234, 5679
    seq = r.seq[int(r.offsets[a]):int(r.offsets[b])]
    ref = oracle.classify(oix, seq, r.offsets[a:b + 1] - r.offsets[a], oracle_params(prm))
    buf = torch.zeros(len(r.seq) + 16, dtype=torch.uint8, device="cuda")
    view = buf[shift:shift + len(r.seq)]
    view.copy_(torch.from_numpy(r.seq))
    assert (view.data_ptr() % 16 == 0) == (shift == 0)
    out = mt.classify(ix, view, torch.from_numpy(r.offsets[a:b + 1].astype(np.int64)).cuda(), **prm)
    compare_classify(out, ref)


def test_index_counts_match_oracle(mt, tiny):
    c, g, r, ix, oix = tiny
    info = ix.info()
    assert info["n_occ"] == oix.n_occ
    assert info["n_genomes"] == g.n and info["k"] == c["k"]


@pytest.fixture(scope="module")
def clade(mt):
    """A scaled-down medium workload: 4 clades x 10 genomes of 100 kb at 1-10% divergence,
    k21 w11 canonical, 20,000 reads of 150 bp on both strands, E = 8."""
    c = gen.config(2, n_genomes=40, genome_len=100_000, n_reads=20_000)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    return c, g, r, ix, oix


def test_clade_workload_general_window_path(mt):
    """The clade workload with w = 9: the seeding kernel's general window-minimum path (four
    windows a lane over keys in shared memory) instead of the block path it takes for w = 11."""
    c = gen.config(2, n_genomes=20, genome_len=100_000, n_reads=5_000, w=9)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    prm = _params(c)
    ref = oracle.classify(oix, r.seq, r.offsets, oracle_params(prm), threads=8)
    compare_classify(mt.classify(ix, r.seq, r.offsets, **prm), ref)


@pytest.mark.parametrize("long_genome", [False, True])
@pytest.mark.parametrize("w", [11, 9])
def test_more_genomes_than_shared_counters(mt, w, long_genome):
    """4,200 genomes of 2 kb (clades of 10): more genome counters than the seeding kernel keeps
    in shared memory, so counts and unique reads go to global memory; the block path (w = 11)
    and the general one (w = 9); 32-bit match keys, or 64-bit ones with one more genome of
    4.2 Mb (its diagonals and 4,201 genome ids do not fit 32 bits). Outputs equal the oracle's."""
    c = gen.config(2, n_genomes=4200, genome_len=2_000, clade_size=10, n_reads=4_000, seed=63, w=w)
    g = gen.make_genomes(c)
    if long_genome:
        rng = np.random.default_rng(64)
        extra = gen.ascii_of(rng.integers(0, 4, 4_200_000, dtype=np.uint8))
        g = gen.Genomes(seq=np.concatenate([g.seq, extra]),
                        offsets=np.append(g.offsets, g.offsets[-1] + np.uint64(len(extra))).astype(np.uint64),
                        clade=np.append(g.clade, g.clade.max() + 1).astype(np.int32))
    r = gen.make_reads(c, g)
    if long_genome:   # the first 300 reads: exact copies from the long genome, both strands
        off0 = int(g.offsets[-2])
        for i in range(300):
            p = off0 + int(rng.integers(0, len(extra) - 150))
            seg = g.seq[p:p + 150]
            r.seq[int(r.offsets[i]):int(r.offsets[i]) + 150] = gen.revcomp_ascii(seg) if i % 2 else seg
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    prm = _params(c)
    ref = oracle.classify(oix, r.seq, r.offsets, oracle_params(prm), threads=8)
    out = mt.classify(ix, r.seq, r.offsets, **prm)
    compare_classify(out, ref)
    assert (ref["taxon"] >= 0).mean() > 0.5 and ref["genome_hits"].astype(bool).sum() > 1000
    ix.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_clade_workload(mt, clade, mode):
    c, g, r, ix, oix = clade
    prm = _params(c)
    ref = oracle.classify(oix, r.seq, r.offsets, oracle_params(prm), threads=8)
    out = mt.classify(ix, r.seq, r.offsets, eda_mode=mode, **prm)
    compare_classify(out, ref)
    assert (ref["multi"][:, 0] >= 0).sum() > 0, "workload should contain multi-mapped reads"


@pytest.mark.parametrize("kw", [dict(top_n=1), dict(top_n=8, min_seeds=1), dict(e_abs=0, e_permille=100),
                                dict(max_occ=2), dict(cont_num=1, cont_den=50), dict(abund_cutoff=0.05),
                                dict(e_abs=0, e_permille=0)])
def test_clade_parameter_sweep(mt, clade, kw):
    c, g, r, ix, oix = clade
    prm = _params(c, **kw)
    n = 4000
    seq, off = r.seq[:int(r.offsets[n])], r.offsets[:n + 1]
    ref = oracle.classify(oix, seq, off, oracle_params(prm), threads=8)
    out = mt.classify(ix, seq, off, **prm)
    compare_classify(out, ref)


@pytest.mark.parametrize("kw", [(15, 10), (13, 7), (21, 11)])
def test_mixed_lengths_and_edges(mt, kw):
    """Reads of 1..1024 bases (below k+w-1, exactly MT_MAX_READ_LEN), reads overhanging genome
    ends on both strands, E from a per-mille threshold. w = 10 and 7 run the general
    window-minimum path; w = 11 the block path, whose passes cover 150 windows each, so reads
    above 160 bases carry the last window's selection from pass to pass."""
    k, w = kw
    rng = np.random.default_rng(5)
    gs = [gen.ascii_of(rng.integers(0, 4, L, dtype=np.uint8)) for L in (3000, 1500, 5000)]
    gseq = np.concatenate(gs)
    goff = np.cumsum([0] + [len(x) for x in gs]).astype(np.uint64)
    reads = []
    for i in range(400):
        gi = int(rng.integers(0, 3))
        L = int(rng.choice([1, 10, 29, 30, 31, 100, 150, 251, 513, 1024]))
        L = min(L, len(gs[gi]))
        kind = i % 4
        over = min(5, L // 4)
        if kind == 0:      # starts before the genome start
            s = np.concatenate([gen.ascii_of(rng.integers(0, 4, over, dtype=np.uint8)), gs[gi][:L - over]])
        elif kind == 1:    # runs past the genome end
            s = np.concatenate([gs[gi][len(gs[gi]) - (L - over):], gen.ascii_of(rng.integers(0, 4, over, dtype=np.uint8))])
        else:
            p = int(rng.integers(0, len(gs[gi]) - L + 1))
            s = gs[gi][p:p + L].copy()
        if i % 3 == 0:
            s = gen.revcomp_ascii(s)
        reads.append(s)
    rseq = np.concatenate(reads)
    roff = np.cumsum([0] + [len(x) for x in reads]).astype(np.uint64)
    ix = mt.Index(gseq, goff, k, w, 1)
    oix = oracle.Index(gseq, goff, k, w, 1)
    for prm in (dict(e_abs=0, e_permille=60, min_seeds=2), dict(e_abs=5, e_permille=0, min_seeds=1, top_n=5)):
        p = _params(dict(e_abs=0, e_permille=0, min_seeds=2), **prm)
        ref = oracle.classify(oix, rseq, roff, oracle_params(p))
        out = mt.classify(ix, rseq, roff, **p)
        compare_classify(out, ref)


def test_repeats_take_the_exact_slow_path(mt):
    """A genome made of a repeated unit gives reads with far more seed matches than fit in
    shared memory; they are re-mapped by the exact per-read slow path."""
    rng = np.random.default_rng(7)
    unit = gen.ascii_of(rng.integers(0, 4, 300, dtype=np.uint8))
    g0 = np.concatenate([unit] * 40)
    g1 = gen.ascii_of(rng.integers(0, 4, 20000, dtype=np.uint8))
    gseq = np.concatenate([g0, g1])
    goff = np.array([0, len(g0), len(g0) + len(g1)], np.uint64)
    reads = [g0[i * 37:i * 37 + 150] for i in range(40)] + [g1[i * 400:i * 400 + 150] for i in range(40)]
    rseq = np.concatenate(reads)
    roff = np.cumsum([0] + [len(x) for x in reads]).astype(np.uint64)
    ix = mt.Index(gseq, goff, 15, 10, 1)
    oix = oracle.Index(gseq, goff, 15, 10, 1)
    p = _params(dict(e_abs=6, e_permille=0, min_seeds=2), max_occ=64)
    ref = oracle.classify(oix, rseq, roff, oracle_params(p))
    out = mt.classify(ix, rseq, roff, **p)
    compare_classify(out, ref)
    assert out["stats"]["n_fallback"] >= 40


def test_masked_genomes_exhaust_stored_locations(mt):
    """Twelve genomes share one segment; only genome 0 also has a large unique part with
    many reads. With a 1/10 cutoff genomes 1..11 are dropped, so reads of the shared segment
    have 12 qualifying locations of which the eight stored ones hold only one kept genome:
    the exact slow path must find the rest."""
    rng = np.random.default_rng(11)
    X = gen.ascii_of(rng.integers(0, 4, 2000, dtype=np.uint8))
    Y = gen.ascii_of(rng.integers(0, 4, 60000, dtype=np.uint8))
    gs = [np.concatenate([X, Y])] + [np.concatenate([gen.ascii_of(rng.integers(0, 4, 500, dtype=np.uint8)), X])
                                      for _ in range(11)]
    gseq = np.concatenate(gs)
    goff = np.cumsum([0] + [len(x) for x in gs]).astype(np.uint64)
    reads = [Y[i * 200:i * 200 + 150] for i in range(250)] + [X[i * 100:i * 100 + 150] for i in range(15)]
    rseq = np.concatenate(reads)
    roff = np.cumsum([0] + [len(x) for x in reads]).astype(np.uint64)
    ix = mt.Index(gseq, goff, 15, 10, 0)
    oix = oracle.Index(gseq, goff, 15, 10, 0)
    p = _params(dict(e_abs=6, e_permille=0, min_seeds=2), cont_num=1, cont_den=10, top_n=3)
    ref = oracle.classify(oix, rseq, roff, oracle_params(p))
    assert ref["keep"].tolist() == [1] + [0] * 11
    out = mt.classify(ix, rseq, roff, **p)
    compare_classify(out, ref)
    assert out["stats"]["n_fallback"] >= 15


def test_plan_graph_replays_match_oracle(mt, clade):
    """A plan captured into a CUDA graph on its second call serves batches of different sizes
    (host and device buffers) with results identical to mt_classify and the oracle."""
    import torch
    c, g, r, ix, oix = clade
    prm = _params(c)
    plan = mt.Plan(ix, max_reads=8000, max_bases=8000 * 150, max_read_len=150, **prm)
    cuts = [(0, 5000), (5000, 5300), (7000, 15000), (100, 7100), (15000, 15001), (300, 300)]
    for i, (a, b) in enumerate(cuts):
        seq = r.seq[int(r.offsets[a]):int(r.offsets[b])]
        off = (r.offsets[a:b + 1] - r.offsets[a]).astype(np.uint64)
        ref = oracle.classify(oix, seq, off, oracle_params(prm), threads=8)
        if i % 2:
            out = plan.classify(torch.from_numpy(seq.copy()).cuda(), torch.from_numpy(off.astype(np.int64)).cuda())
        else:
            out = plan.classify(seq, off)
        compare_classify(out, ref)
        direct = mt.classify(ix, seq, off, **prm)
        assert np.array_equal(np.asarray(out["taxon"].cpu() if hasattr(out["taxon"], "cpu") else out["taxon"]),
                              direct["taxon"])
    with pytest.raises(mt.MtError):
        plan.classify(r.seq, r.offsets)            # above the capacity
    # inputs the kernels reject: a read above the plan's read length, offsets out of order
    longer = np.concatenate([r.seq[:300], r.seq[:1]])
    with pytest.raises(mt.MtError) as e:
        plan.classify(longer, np.array([0, 149, 301], np.uint64))
    assert e.value.status == mt.MT_EINVAL
    with pytest.raises(mt.MtError) as e:
        plan.classify(r.seq[:300], np.array([0, 200, 150, 300], np.uint64))
    assert e.value.status == mt.MT_EINVAL
    ok = plan.classify(r.seq[:300], np.array([0, 150, 300], np.uint64))   # still usable
    assert len(ok["taxon"]) == 2
    plan.close()


def test_invalid_inputs(mt, tiny):
    c, g, r, ix, oix = tiny
    prm = _params(c)
    bad = r.seq[:300].copy()
    bad[170] = ord("N")
    with pytest.raises(mt.MtError) as e:
        mt.classify(ix, bad, np.array([0, 150, 300], np.uint64), **prm)
    assert e.value.status == mt.MT_EINVAL
    long = np.frombuffer(b"ACGT" * 300, np.uint8)
    with pytest.raises(mt.MtError):
        mt.classify(ix, long, np.array([0, 1200], np.uint64), **prm)
    with pytest.raises(mt.MtError):
        mt.classify(ix, r.seq[:300], np.array([0, 200, 100], np.uint64), **prm)
    with pytest.raises(mt.MtError):
        mt.classify(ix, r.seq[:300], np.array([0, 150], np.uint64), **dict(prm, top_n=9))
    # the library is still usable afterwards
    out = mt.classify(ix, r.seq[:1500], r.offsets[:11], **prm)
    ref = oracle.classify(oix, r.seq[:1500], r.offsets[:11], oracle_params(prm))
    compare_classify(out, ref)


def test_empty_batch(mt, tiny):
    c, g, r, ix, oix = tiny
    out = mt.classify(ix, np.zeros(0, np.uint8), np.zeros(1, np.uint64), **_params(c))
    assert len(out["taxon"]) == 0
    assert out["genome_hits"].tolist() == [0] * g.n
    assert out["abundance"].tolist() == [0.0] * g.n


def test_host_batch_uploaded_in_chunks(mt):
    """A host batch above the 32 MB chunk size goes up in several chunks, each seeded as it
    lands: results equal the device-buffer call's, read for read, and the oracle's on a sample."""
    import torch
    c = gen.config(2, n_genomes=20, genome_len=100_000, n_reads=500_000)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    assert len(r.seq) > (64 << 20) // 2
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    prm = _params(c, e_permille=0)
    host = mt.classify(ix, r.seq, r.offsets, **prm)
    dev = mt.classify(ix, torch.from_numpy(r.seq).cuda(), torch.from_numpy(r.offsets.astype(np.int64)).cuda(), **prm)
    assert np.array_equal(host["taxon"], dev["taxon"].cpu().numpy())
    assert np.array_equal(host["nloc"], dev["nloc"].cpu().numpy())
    assert np.array_equal(host["locs"], mt.locs_from_device(dev["locs"]))
    assert np.array_equal(host["genome_hits"], dev["genome_hits"].cpu().numpy().view(np.uint64))
    # page-locked output buffers
    def pinned(shape, dtype):
        n = int(np.prod(shape)) * np.dtype(dtype).itemsize
        return torch.empty(n, dtype=torch.uint8).pin_memory().numpy().view(dtype).reshape(shape)
    pout = dict(taxon=pinned((r.n,), np.int32), nloc=pinned((r.n,), np.uint8), locs=pinned((r.n, 3), mt.LOC_DTYPE),
                genome_hits=pinned((g.n,), np.uint64), abundance=pinned((g.n,), np.float64))
    pres = mt.classify(ix, r.seq, r.offsets, out=pout, **prm)
    for k in ("taxon", "nloc", "locs", "genome_hits", "abundance"):
        assert np.array_equal(pres[k], host[k]), k
    # The chunks start uploading before the offsets are checked: offsets past the bytes from
    # the middle on, one decreasing offset and an end past the bytes are each refused, and the
    # next call is unaffected.
    bad = []
    for edit in ("past", "decreasing", "end"):
        off = r.offsets.copy()
        if edit == "past":
            off[300_000:] += np.uint64(10 ** 9)
        elif edit == "decreasing":
            off[250_000] = off[250_002] + np.uint64(1)
        else:
            off[-1] = np.uint64(len(r.seq) + 1)
        bad.append(off)
    for off in bad:
        with pytest.raises(mt.MtError) as e:
            mt.classify(ix, r.seq, off, **prm)
        assert e.value.status == mt.MT_EINVAL
    again = mt.classify(ix, r.seq, r.offsets, **prm)
    for k in ("taxon", "nloc", "locs", "genome_hits", "abundance"):
        assert np.array_equal(again[k], host[k]), k
    oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    ref = oracle.classify(oix, r.seq, r.offsets, oracle_params(prm), threads=16)
    compare_classify(host, ref)


def test_plan_with_chunked_uploads_matches_oracle(mt):
    """A plan of 300,000 reads uploads host batches in chunks of reads (2 here), each seeded as it lands,
    inside the captured graph: batches spanning several chunks, device batches through the
    same graph, and an offset at a chunk boundary past the bytes refused before any copy."""
    import torch
    c = gen.config(2, n_genomes=20, genome_len=100_000, n_reads=250_000, seed=97)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"], threads=8)
    prm = _params(c)
    plan = mt.Plan(ix, max_reads=300_000, max_bases=300_000 * 150, max_read_len=150, **prm)
    cuts = [(0, 250_000), (20_000, 120_000), (100_000, 170_001), (5, 5_005), (0, 250_000)]
    for i, (a, b) in enumerate(cuts):
        seq = r.seq[int(r.offsets[a]):int(r.offsets[b])]
        off = (r.offsets[a:b + 1] - r.offsets[a]).astype(np.uint64)
        ref = oracle.classify(oix, seq, off, oracle_params(prm), threads=16)
        if i == 1:
            out = plan.classify(torch.from_numpy(seq.copy()).cuda(), torch.from_numpy(off.astype(np.int64)).cuda())
        else:
            out = plan.classify(seq, off)
        compare_classify(out, ref)
    seq = r.seq[:int(r.offsets[200_000])]
    off = r.offsets[:200_001].copy()
    off[150_000:] += np.uint64(10 ** 9)          # reads past the bytes from the second chunk on
    with pytest.raises(mt.MtError) as e:
        plan.classify(seq, off)
    assert e.value.status == mt.MT_EINVAL
    ok = plan.classify(r.seq[:300], np.array([0, 150, 300], np.uint64))   # still usable
    assert len(ok["taxon"]) == 2
    plan.close()
