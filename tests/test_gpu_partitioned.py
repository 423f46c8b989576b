"""GPU parity of a query against a reference database cut into batches (mt_part_*,
mt_classify_partitioned): per-batch containment with each batch's own repeat filter, the
highest count of a genome held by several batches, the cutoff over the whole database, and
mapping against the subset index of the kept genomes. Every output bit-exact against the
oracle's partitioned pipeline (abundances within 1e-6); batches resident, or saved to files
and loaded one at a time; the paper's compressed containment seeds (k = 28, w = 18);
nothing kept; an empty read batch; refused calls."""
import numpy as np
import pytest

import gen
import oracle
from helpers import ABUND_TOL, as_np, compare_classify, oracle_params

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


def _work(n_genomes=20, genome_len=50_000, clade=5, n_reads=4_000, seed=31):
    c = gen.config(2, n_genomes=n_genomes, genome_len=genome_len, clade_size=clade, n_reads=n_reads, seed=seed)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    return c, g, r


def _parts_with_copies(mt, g, n_batches):
    """Consecutive-id batches, plus copies of a few genomes in other batches."""
    parts = mt.split_batches(g.offsets, n_batches)
    extra = {0: [g.n - 1], n_batches - 1: [0, 1]} if n_batches > 1 else {}
    return [np.concatenate([p, np.array(extra.get(b, []), np.uint32)]).astype(np.uint32) for b, p in enumerate(parts)]


def _batches(make, g, parts, k, w, can, hpc=False):
    out = []
    for ids in parts:
        seq, off = oracle.gather_genomes(g.seq, g.offsets, ids)
        out.append(make(seq, off, k, w, can, hpc))
    return out


def _prm(c, **kw):
    prm = dict(e_abs=c["e_abs"], e_permille=c["e_permille"], min_seeds=c["min_seeds"], top_n=3, max_occ=1024,
               cont_num=1, cont_den=10000, abund_cutoff=1e-4)
    prm.update(kw)
    return prm


@pytest.mark.parametrize("n_batches,max_occ,cont_den", [(4, 3, 10000), (5, 1024, 20), (1, 2, 10000)])
def test_one_call_matches_oracle(mt, n_batches, max_occ, cont_den):
    """Resident batches, host buffers. A small max_occ makes per-batch filtering differ from
    one index over all genomes (clade members share most minimizers)."""
    c, g, r = _work()
    parts = _parts_with_copies(mt, g, n_batches)
    k, w, can = c["k"], c["w"], c["canonical"]
    prm = _prm(c, max_occ=max_occ, cont_den=cont_den)
    gpu_b = _batches(lambda s, o, k, w, can, h: mt.Index(s, o, k, w, can), g, parts, k, w, can)
    got = mt.classify_partitioned(gpu_b, parts, g.seq, g.offsets, r.seq, r.offsets, k=k, w=w, canonical=can, **prm)
    ora_b = [(oracle.Index(*oracle.gather_genomes(g.seq, g.offsets, ids), k, w, can), ids) for ids in parts]
    ref = oracle.classify_partitioned(ora_b, g.n, g.seq, g.offsets, r.seq, r.offsets, oracle_params(prm), k, w, can,
                                      threads=8)
    compare_classify(got, ref)
    assert (ref["taxon"] >= 0).mean() > 0.5
    if cont_den == 20:
        assert 0 < int(ref["keep"].sum()) < g.n


def test_staged_query_with_batches_from_files(mt, tmp_path):
    """Device tensors; each database batch is saved, then loaded, queried and freed in turn
    (only one batch resident at a time); containment batches are the paper's compressed
    k = 28, w = 18 indexes, the subset index is k21 w11."""
    import torch
    c, g, r = _work(n_genomes=24, genome_len=40_000, clade=4, n_reads=5_000, seed=41)
    parts = _parts_with_copies(mt, g, 6)
    paths = []
    for b, ids in enumerate(parts):
        seq, off = oracle.gather_genomes(g.seq, g.offsets, ids)
        ix = mt.Index(seq, off, 28, 18, 1, hpc=True)
        paths.append(str(tmp_path / ("batch%02d.idx" % b)))
        ix.save(paths[-1])
        ix.close()
    prm = _prm(c, max_occ=2)
    dev = torch.device("cuda:0")
    reads = torch.from_numpy(r.seq).to(dev)
    offs = torch.from_numpy(r.offsets.astype(np.int64)).to(dev)
    q = mt.PartitionedQuery(g.n, reads, offs)
    for ids, path in zip(parts, paths):
        ix = mt.Index.load(path)
        q.contain(ix, ids, max_occ=prm["max_occ"])
        ix.close()
    sub = q.subset(prm["cont_num"], prm["cont_den"])
    kept = sub["kept"]
    sub_ix = mt.Index(*oracle.gather_genomes(g.seq, g.offsets, kept), c["k"], c["w"], c["canonical"]) if len(kept) else None
    got = q.classify(sub_ix, **prm)
    q.close()

    ora_b = [(oracle.Index(*oracle.gather_genomes(g.seq, g.offsets, ids), 28, 18, 1, compressed=True), ids)
             for ids in parts]
    ref = oracle.classify_partitioned(ora_b, g.n, g.seq, g.offsets, r.seq, r.offsets, oracle_params(prm), c["k"],
                                      c["w"], c["canonical"], threads=8)
    assert np.array_equal(as_np(sub["genome_hits"]).astype(np.uint64), ref["genome_hits"])
    assert np.array_equal(sub["keep"], ref["keep"]) and np.array_equal(kept, ref["kept"])
    compare_classify(got, ref, check_global=False)
    assert np.abs(as_np(got["abundance"]) - ref["abundance"]).max() <= ABUND_TOL


def test_mid_sized_database_in_25_batches(mt):
    """The paper's 25 database batches over a clade-structured reference of 200 genomes."""
    c, g, r = _work(n_genomes=200, genome_len=100_000, clade=10, n_reads=20_000, seed=51)
    parts = mt.split_batches(g.offsets, 25)
    k, w, can = c["k"], c["w"], c["canonical"]
    prm = _prm(c, max_occ=6)
    gpu_b = [mt.Index(*oracle.gather_genomes(g.seq, g.offsets, ids), k, w, can) for ids in parts]
    got = mt.classify_partitioned(gpu_b, parts, g.seq, g.offsets, r.seq, r.offsets, k=k, w=w, canonical=can, **prm)
    ora_b = [(oracle.Index(*oracle.gather_genomes(g.seq, g.offsets, ids), k, w, can, threads=8), ids) for ids in parts]
    ref = oracle.classify_partitioned(ora_b, g.n, g.seq, g.offsets, r.seq, r.offsets, oracle_params(prm), k, w, can,
                                      threads=16)
    compare_classify(got, ref)


@pytest.mark.parametrize("hpc,many", [(False, False), (True, False), (False, True)])
def test_one_pass_over_all_batches_equals_one_pass_each(mt, hpc, many):
    """mt_part_contain_batches (each read's minimizers found once, looked up in every batch)
    gives the counts of one mt_part_contain per batch, and the oracle's. ``many``: more genome
    counters than fit in shared memory (4,200 small genomes)."""
    import torch
    if many:
        c = gen.config(2, n_genomes=4200, genome_len=2_000, clade_size=10, n_reads=3_000, seed=61)
    else:
        c = gen.config(2, n_genomes=30, genome_len=40_000, clade_size=5, n_reads=6_000, seed=62)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    parts = _parts_with_copies(mt, g, 7)
    k, w = (28, 18) if hpc else (c["k"], c["w"])
    bs = [mt.Index(*oracle.gather_genomes(g.seq, g.offsets, ids), k, w, 1, hpc=hpc) for ids in parts]
    dev = torch.device("cuda:0")
    reads = torch.from_numpy(r.seq).to(dev)
    offs = torch.from_numpy(r.offsets.astype(np.int64)).to(dev)
    res = []
    for fused in (True, False):
        q = mt.PartitionedQuery(g.n, reads, offs)
        if fused:
            q.contain_batches(bs, parts, max_occ=3)
        else:
            for ix, ids in zip(bs, parts):
                q.contain(ix, ids, max_occ=3)
        res.append(as_np(q.subset(1, 10000)["genome_hits"]).astype(np.uint64))
        q.close()
    assert np.array_equal(res[0], res[1])
    ora_b = [(oracle.Index(*oracle.gather_genomes(g.seq, g.offsets, ids), k, w, 1, compressed=hpc), ids)
             for ids in parts]
    ref = oracle.partitioned_hits(ora_b, g.n, r.seq, r.offsets, 3, threads=8)
    assert np.array_equal(res[0], ref) and ref.sum() > 0
    # batches whose seeds differ cannot share one pass
    other = mt.Index(*oracle.gather_genomes(g.seq, g.offsets, parts[0]), k - 1, w, 1, hpc=hpc)
    q = mt.PartitionedQuery(g.n, reads, offs)
    with pytest.raises(mt.MtError):
        q.contain_batches([bs[1], other], [parts[1], parts[0]])
    q.close()


def test_subset_index_equals_index_over_gathered_genomes(mt):
    """mt_build_index_subset (bytes copied run by run from the set) answers like an index built
    from the gathered bytes: ids out of order, with gaps, a repeat and adjacent runs."""
    c, g, r = _work(n_genomes=20, genome_len=30_000, clade=5, n_reads=3_000, seed=71)
    ids = np.array([7, 8, 9, 2, 15, 3, 4, 19, 0, 9], np.uint32)
    a = mt.Index.subset(g.seq, g.offsets, ids, c["k"], c["w"], c["canonical"])
    b = mt.Index(*oracle.gather_genomes(g.seq, g.offsets, ids), c["k"], c["w"], c["canonical"])
    assert a.info() == b.info()
    prm = _prm(c)
    x = mt.classify(a, r.seq, r.offsets, **prm)
    y = mt.classify(b, r.seq, r.offsets, **prm)
    for k in ("taxon", "nloc", "genome_hits"):
        assert np.array_equal(x[k], y[k])
    assert np.array_equal(x["locs"], y["locs"]) and np.array_equal(x["abundance"], y["abundance"])


def test_nothing_kept_and_empty_batch(mt):
    c, g, _ = _work(n_genomes=10, genome_len=20_000, clade=5, n_reads=10)
    parts = mt.split_batches(g.offsets, 3)
    k, w, can = c["k"], c["w"], c["canonical"]
    gpu_b = [mt.Index(*oracle.gather_genomes(g.seq, g.offsets, ids), k, w, can) for ids in parts]
    rng = np.random.default_rng(5)
    rs = np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, 150 * 40)].copy()
    ro = np.arange(0, 150 * 41, 150, dtype=np.uint64)
    prm = _prm(c)
    got = mt.classify_partitioned(gpu_b, parts, g.seq, g.offsets, rs, ro, k=k, w=w, canonical=can, **prm)
    ora_b = [(oracle.Index(*oracle.gather_genomes(g.seq, g.offsets, ids), k, w, can), ids) for ids in parts]
    ref = oracle.classify_partitioned(ora_b, g.n, g.seq, g.offsets, rs, ro, oracle_params(prm), k, w, can)
    compare_classify(got, ref)
    if not ref["genome_hits"].any():
        assert (got["taxon"] == -1).all() and not got["abundance"].any()
    # no reads at all
    empty = mt.classify_partitioned(gpu_b, parts, g.seq, g.offsets, np.zeros(0, np.uint8), np.zeros(1, np.uint64),
                                    k=k, w=w, canonical=can, **prm)
    assert len(empty["taxon"]) == 0 and not empty["genome_hits"].any() and not empty["abundance"].any()


def test_refused_calls(mt):
    c, g, r = _work(n_genomes=10, genome_len=20_000, clade=5, n_reads=200)
    k, w, can = c["k"], c["w"], c["canonical"]
    ix = mt.Index(*oracle.gather_genomes(g.seq, g.offsets, [0, 1, 2]), k, w, can)
    q = mt.PartitionedQuery(g.n, r.seq, r.offsets)
    with pytest.raises(mt.MtError):
        q.classify(ix, **_prm(c))                   # before the cutoff
    with pytest.raises(mt.MtError):
        q.contain(ix, [0, 1, g.n])                  # a global id out of range
    q.contain(ix, [0, 1, 2])
    kept = q.subset(1, 10000)["kept"]
    assert set(kept.tolist()) <= {0, 1, 2} and len(kept) > 0
    wrong = mt.Index(*oracle.gather_genomes(g.seq, g.offsets, np.arange(3, 4 + len(kept))), k, w, can)
    with pytest.raises(mt.MtError):
        q.classify(wrong, **_prm(c))                # an index over another number of genomes
    one = mt.Index(*oracle.gather_genomes(g.seq, g.offsets, [3]), k, w, can)
    q.kept = np.array([3], np.uint32)
    with pytest.raises(mt.MtError):
        q.classify(one, **_prm(c))                  # not the kept list
    q.close()


def test_more_batches_than_one_counting_pass_holds(mt):
    """4,100 batches, more than the 4,096 indexes one counting pass takes: mt_part_contain_batches
    makes a second pass for the last four, whose counters follow the first pass's. Every batch
    holds one genome except the last, which also holds a copy of genome 7 (its count there is
    merged with batch 7's by the highest-count rule). The per-genome counts equal one
    mt_part_contain call per batch and the oracle's per-batch counts, on both sides of the
    boundary."""
    rng = np.random.default_rng(41)
    G, L, k, w = 4100, 400, 21, 11
    seq = gen.ascii_of(rng.integers(0, 4, G * L, dtype=np.uint8))
    off = np.arange(G + 1, dtype=np.uint64) * np.uint64(L)
    parts = [np.array([b], np.uint32) for b in range(G)]
    parts[-1] = np.array([G - 1, 7], np.uint32)
    # 1,220 reads of 100 bp: 300 from the genomes around the boundary, 20 from genome 7 (held by
    # two batches), the rest anywhere
    src = np.concatenate([rng.integers(4090, G, 300), np.full(20, 7), rng.integers(0, G, 900)])
    reads = []
    for gid in src:
        p = int(rng.integers(0, L - 100))
        r = seq[gid * L + p:gid * L + p + 100]
        reads.append(gen.revcomp_ascii(r) if rng.random() < 0.5 else r)
    r_seq = np.concatenate(reads)
    r_off = np.arange(len(reads) + 1, dtype=np.uint64) * np.uint64(100)
    dev = [mt.Index(*oracle.gather_genomes(seq, off, ids), k, w, 1) for ids in parts]
    try:
        q = mt.PartitionedQuery(G, r_seq, r_off)
        q.contain_batches(dev, parts, max_occ=1024)
        H = q.subset(1, 10000)["genome_hits"].astype(np.uint64)
        q.close()
        q = mt.PartitionedQuery(G, r_seq, r_off)
        for ix, ids in zip(dev, parts):
            q.contain(ix, ids, max_occ=1024)
        H1 = q.subset(1, 10000)["genome_hits"].astype(np.uint64)
        q.close()
    finally:
        for ix in dev:
            ix.close()
    ob = [(oracle.Index(*oracle.gather_genomes(seq, off, ids), k, w, 1), ids) for ids in parts]
    H2 = oracle.partitioned_hits(ob, G, r_seq, r_off, 1024, threads=8)
    assert np.array_equal(H, H2) and np.array_equal(H1, H2)
    assert H[4096:].sum() > 0 and H[4090:4096].sum() > 0 and H[7] > 0
