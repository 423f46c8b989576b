"""Pins of the oracle's partitioned-database pipeline (Methods, "Reference Database
Organisation and Index Construction & Querying"; Evaluation Methodology): special cases
that reduce to the pinned single-index pipeline, and per-batch seed counts against a brute
force enumeration written here."""
import numpy as np
import pytest

import gen
import oracle
from test_oracle_pins import _RC, _brute_db, _tiny_db, brute_minimizers


def _db(n_reads=400):
    c = gen.config(2, n_genomes=20, genome_len=20_000, clade_size=5, n_reads=n_reads, seed=77)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    return c, g, r


def _split(G, n_batches, seed):
    rng = np.random.default_rng(seed)
    perm = rng.permutation(G)
    return [np.sort(perm[i::n_batches]) if i % 2 == 0 else perm[i::n_batches]   # any id order
            for i in range(n_batches)]


def _batches(g, c, parts):
    out = []
    for ids in parts:
        seq, off = oracle.gather_genomes(g.seq, g.offsets, ids)
        out.append((oracle.Index(seq, off, c["k"], c["w"], c["canonical"]), np.asarray(ids)))
    return out


def _same(a, b):
    assert np.array_equal(a["genome_hits"], b["genome_hits"])
    assert np.array_equal(a["keep"], b["keep"])
    assert np.array_equal(a["taxon"], b["taxon"])
    assert np.array_equal(a["nloc"], b["nloc"])
    for f in ("genome", "seeds", "strand", "dist", "wstart"):
        assert np.array_equal(a["locs"][f], b["locs"][f]), f
    assert np.array_equal(a["U"], b["U"])
    assert np.abs(a["abundance"] - b["abundance"]).max() <= 1e-12


@pytest.mark.parametrize("n_batches,cont_den", [(1, 10000), (3, 10000), (4, 10)])
def test_no_repeat_filter_equals_single_index(oracle_lib, n_batches, cont_den):
    """When no key reaches the repeat filter, every batch sees the same occurrences of its
    genomes as one index over all of them, the highest count of a genome is its count, and
    the subset index holds exactly the kept genomes' occurrences: the partitioned pipeline
    must then equal the single-index one (containment mask + masked mapping)."""
    c, g, r = _db()
    p = oracle.params(max_occ=2048, e_abs=c["e_abs"], e_permille=0, min_seeds=c["min_seeds"], cont_den=cont_den)
    full = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    ref = oracle.classify(full, r.seq, r.offsets, p)
    got = oracle.classify_partitioned(_batches(g, c, _split(g.n, n_batches, 5 + n_batches)), g.n, g.seq,
                                      g.offsets, r.seq, r.offsets, p, c["k"], c["w"], c["canonical"])
    _same(got, ref)
    if cont_den == 10:   # the cutoff dropped some genomes: ids went through the subset and back
        assert 0 < int(ref["keep"].sum()) < g.n
    assert (ref["taxon"] >= 0).mean() > 0.5


def test_genome_in_several_batches_counts_once(oracle_lib):
    """A genome held by several batches keeps its highest count, not the sum: copies of
    genomes 2 and 7 in other batches leave every output unchanged."""
    c, g, r = _db(300)
    p = oracle.params(max_occ=2048, e_abs=c["e_abs"], e_permille=0, min_seeds=c["min_seeds"])
    parts = _split(g.n, 3, 9)
    base = oracle.classify_partitioned(_batches(g, c, parts), g.n, g.seq, g.offsets, r.seq, r.offsets, p,
                                       c["k"], c["w"], c["canonical"])
    dup = [np.concatenate([parts[0], [2, 7]]), np.concatenate([[7], parts[1]]), np.concatenate([parts[2], [2]])]
    got = oracle.classify_partitioned(_batches(g, c, dup), g.n, g.seq, g.offsets, r.seq, r.offsets, p,
                                      c["k"], c["w"], c["canonical"])
    _same(got, base)
    assert base["genome_hits"][2] > 0 and base["genome_hits"][7] > 0


@pytest.mark.parametrize("max_occ", [1, 2, 1024])
def test_repeat_filter_is_per_batch_brute_force(oracle_lib, max_occ):
    """Each batch filters keys by its own occurrence count (each batch is queried as its own
    index): per-genome counts from a brute-force enumeration over each batch's genomes."""
    rng = np.random.default_rng(23)
    k, w, can = 7, 5, 1
    gs, _, _ = _tiny_db(rng)          # genomes 0 and 1 share a segment; genome 2 has a repeat
    parts = [[0, 2], [1, 3]]
    reads = []
    for _ in range(40):
        gi = int(rng.integers(0, len(gs)))
        pos = int(rng.integers(0, len(gs[gi]) - 60))
        rd = gs[gi][pos:pos + 60]
        if rng.random() < 0.5:
            rd = rd[::-1].translate(_RC)
        reads.append(rd)
    reads.append(gs[0][120:180])      # inside the shared segment
    exp = np.zeros(len(gs), np.uint64)
    for ids in parts:
        db = _brute_db([gs[i] for i in ids], k, w, can)
        for rd in reads:
            for (_, code, _) in brute_minimizers(rd, k, w, can):
                occ = db.get(code, [])
                if len(occ) > max_occ:
                    continue
                for (l, _, _) in occ:
                    exp[ids[l]] += 1
    rs = np.frombuffer("".join(reads).encode(), np.uint8).copy()
    ro = np.cumsum([0] + [len(x) for x in reads]).astype(np.uint64)
    seq = np.frombuffer("".join(gs).encode(), np.uint8).copy()
    off = np.cumsum([0] + [len(x) for x in gs]).astype(np.uint64)
    batches = []
    for ids in parts:
        bs, bo = oracle.gather_genomes(seq, off, ids)
        batches.append((oracle.Index(bs, bo, k, w, can), np.array(ids)))
    got = oracle.partitioned_hits(batches, len(gs), rs, ro, max_occ)
    assert got.tolist() == exp.tolist()
    if max_occ == 1:   # the shared segment is filtered in one index but counted per batch
        whole = oracle.count_hits(oracle.Index(seq, off, k, w, can), rs, ro, max_occ)
        assert got[0] > whole[0] and got[1] > whole[1]


def test_nothing_kept(oracle_lib):
    """Reads that share no seed with the database: no genome is kept, no read maps."""
    c, g, _ = _db(10)
    rng = np.random.default_rng(3)
    rs = np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, 150 * 5)].copy()
    ro = np.arange(0, 151 * 5, 150, dtype=np.uint64)[:6]
    p = oracle.params(e_abs=8, e_permille=0, min_seeds=3)
    got = oracle.classify_partitioned(_batches(g, c, _split(g.n, 2, 1)), g.n, g.seq, g.offsets, rs, ro, p,
                                      c["k"], c["w"], c["canonical"])
    if got["genome_hits"].any():
        pytest.skip("a random read happened to share a seed")
    assert not got["keep"].any()
    assert (got["taxon"] == -1).all() and not got["nloc"].any() and (got["locs"]["genome"] == -1).all()
    assert not got["abundance"].any()


def test_gather_genomes_keeps_order(oracle_lib):
    seq = np.frombuffer(b"AAACCGTTTT", np.uint8)
    off = np.array([0, 3, 5, 6, 10], np.uint64)
    s, o = oracle.gather_genomes(seq, off, [3, 0])
    assert bytes(s) == b"TTTTAAA" and o.tolist() == [0, 4, 7]


# ---------------------------------------------------------------------------------------
# genome shards on separate devices: per-shard mapping, lists merged by the rank key
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("n_shards,max_occ,cont_den", [(1, 3, 10000), (2, 2048, 10000), (3, 2048, 10),
                                                       (4, 2048, 10000)])
def test_genome_shards_equal_single_index(oracle_lib, n_shards, max_occ, cont_den):
    """Disjoint genome shards, every shard seeing every read: when no key reaches the repeat
    filter (or with one shard) per-genome counts and locations are those of one index over all
    genomes, so the merged top_n and the decision must equal the single-index pipeline (whose
    decision the C oracle takes; the merge and decision here are separately written)."""
    c, g, r = _db()
    p = oracle.params(max_occ=max_occ, e_abs=c["e_abs"], e_permille=0, min_seeds=c["min_seeds"], cont_den=cont_den)
    full = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    ref = oracle.classify(full, r.seq, r.offsets, p)
    parts = [np.sort(x) for x in _split(g.n, n_shards, 13 + n_shards)]
    got = oracle.classify_genome_sharded(_batches(g, c, parts), g.n, r.seq, r.offsets, p)
    _same(got, ref)
    assert np.array_equal(got["multi"], ref["multi"])
    if n_shards > 1:
        assert (ref["taxon"] >= 0).mean() > 0.5


def test_merge_rank_order_hand_case(oracle_lib):
    """Two shards' lists of one read (E = 4): seeds first, then genome, strand, window start;
    the merged first three decide the read (distances 5 > E, 2, 2: best 2 in genomes 3 then 1)."""
    def L(g, seeds, strand, wstart, dist):
        x = np.zeros((), oracle.LOC_DTYPE)
        x["genome"], x["seeds"], x["strand"], x["wstart"], x["dist"] = g, seeds, strand, wstart, dist
        return x
    none = L(-1, 0, 0, 0, 0)
    # read 1: both best locations lie in genome 2 (two strands): unique, not multi-mapped
    a = np.array([[L(3, 9, 0, 100, 2), L(5, 4, 1, 7, 1), none],
                  [L(2, 6, 0, 10, 1), L(2, 6, 1, 400, 1), none]], oracle.LOC_DTYPE)
    b = np.array([[L(1, 9, 1, 50, 5), L(1, 4, 0, 900, 0), L(1, 4, 0, 800, 2)],
                  [none, none, none]], oracle.LOC_DTYPE)
    p = oracle.params(e_abs=4, e_permille=0, top_n=3)
    out = oracle.merge_and_decide([a, b], np.array([0, 100, 200], np.uint64), p, 6)
    assert out["locs"][0]["genome"].tolist() == [1, 3, 1]
    assert out["locs"][0]["wstart"].tolist() == [50, 100, 800]
    assert out["taxon"][0] == 3 and out["multi"][0].tolist() == [3, 1, -1]
    assert out["nloc"].tolist() == [3, 2]
    assert out["taxon"][1] == 2 and out["multi"][1].tolist() == [-1, -1, -1]
    assert out["U"].tolist() == [0, 0, 1, 0, 0, 0]
