"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test states what fixes the expected value: a published test vector, a hand-worked
example, a brute-force enumeration written independently here, a closed-form reduction or
a proven bound. None of them re-calls the oracle to produce its own expectation.
"""
import itertools
import os

import numpy as np
import pytest

import gen
import oracle

M64 = (1 << 64) - 1
HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------------------------------
# key mixer: SplitMix64 finaliser (Steele, Lea & Flood 2014)
# ---------------------------------------------------------------------------------------
def test_mix64_published_splitmix_sequence(oracle_lib):
    # SplitMix64 seeded with 0 advances its state by the golden gamma 0x9e3779b97f4a7c15 and
    # outputs the finaliser of the state; its published first outputs are these three.
    expect = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    s = 0
    for e in expect:
        s = (s + 0x9E3779B97F4A7C15) & M64
        assert oracle.mix64(s) == e


def _inv_xorshift(y, s):
    x = y
    for _ in range(64 // s + 1):
        x = y ^ (x >> s)
    return x & M64


def test_mix64_is_a_bijection(oracle_lib):
    # invert each step (xor-shift and odd multiply) and recover the input
    inv1 = pow(0xBF58476D1CE4E5B9, -1, 1 << 64)
    inv2 = pow(0x94D049BB133111EB, -1, 1 << 64)
    rng = np.random.default_rng(1)
    for x in [0, 1, 2, 3, (1 << 42) - 1] + [int(v) for v in rng.integers(0, 1 << 62, 200)]:
        y = oracle.mix64(x)
        z = _inv_xorshift(y, 31)
        z = (z * inv2) & M64
        z = _inv_xorshift(z, 27)
        z = (z * inv1) & M64
        z = _inv_xorshift(z, 30)
        assert z == x
    assert oracle.mix64(0) == 0


# ---------------------------------------------------------------------------------------
# minimizers: brute force over windows
# ---------------------------------------------------------------------------------------
def _py_mix(z):
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def test_python_mixer_matches_published_vectors():
    s, out = 0, []
    for _ in range(3):
        s = (s + 0x9E3779B97F4A7C15) & M64
        out.append(_py_mix(s))
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


_TR = str.maketrans("ACGT", "0123")
_RC = str.maketrans("ACGT", "TGCA")


def brute_minimizers(s: str, k: int, w: int, canonical: int):
    """Every window of w k-mers, its smallest key (leftmost on ties); the set of chosen
    positions. k-mer codes come from reading the k-mer as a base-4 numeral."""
    nk = len(s) - k + 1
    if nk < w or len(s) < k:
        return []
    info = []
    for i in range(nk):
        km = s[i:i + k]
        fwd = int(km.translate(_TR), 4)
        rc = int(km[::-1].translate(_RC).translate(_TR), 4)
        if canonical:
            code, st = (rc, 1) if rc < fwd else (fwd, 0)
        else:
            code, st = fwd, 0
        info.append((code, _py_mix(code), st))
    chosen = set()
    for j in range(nk - w + 1):
        chosen.add(min(range(j, j + w), key=lambda t: (info[t][1], t)))
    return [(i, info[i][0], info[i][2]) for i in sorted(chosen)]


@pytest.mark.parametrize("k,w,canonical", [(1, 2, 0), (3, 4, 1), (5, 3, 0), (15, 10, 0),
                                           (21, 11, 1), (7, 1, 1), (31, 5, 1), (4, 6, 1)])
def test_minimizers_match_brute_force(oracle_lib, k, w, canonical):
    rng = np.random.default_rng(k * 100 + w)
    for trial in range(12):
        n = int(rng.integers(max(1, k - 2), 160))
        alphabet = "ACGT" if trial % 3 else "AC"       # low-entropy sequences force ties
        s = "".join(rng.choice(list(alphabet), n))
        exp = brute_minimizers(s, k, w, canonical)
        code, key, pos, strand = oracle.minimizers(s, k, w, canonical)
        got = list(zip(pos.tolist(), code.tolist(), strand.tolist()))
        assert got == exp, (s, k, w, canonical)
        assert all(_py_mix(c) == int(kk) for c, kk in zip(code.tolist(), key))


def test_minimizers_hand_example(oracle_lib):
    # k = 1, w = 3, forward codes A=0 < others; mix64(0) = 0 is the smallest key, so every
    # window holding an A picks its leftmost A. "CCACCAC": windows 0-2, 1-3, 2-4 pick 2;
    # windows 3-5 and 4-6 pick 5.
    _, _, pos, _ = oracle.minimizers("CCACCAC", 1, 3, 0)
    assert pos.tolist() == [2, 5]
    # a sequence with fewer than w k-mers (n < k + w - 1) has none
    assert len(oracle.minimizers("ACGTACGTACGTACGTACGTACGT", 15, 11, 0)[0]) == 0
    assert len(oracle.minimizers("ACGTACGTACGTACGTACGTACGTA", 15, 11, 0)[0]) == 1


def test_minimizers_reject_bad_bases(oracle_lib):
    with pytest.raises(oracle.OracleError):
        oracle.minimizers("ACGTNACGT", 3, 2, 0)
    with pytest.raises(oracle.OracleError):
        oracle.minimizers("acgtacgt", 3, 2, 0)


# ---------------------------------------------------------------------------------------
# index, seed matches and containment counts: brute force over all genomes
# ---------------------------------------------------------------------------------------
def _tiny_db(rng, G=4, L=600, with_repeat=True):
    gs = ["".join(rng.choice(list("ACGT"), L)) for _ in range(G)]
    # shared segment between genomes 0 and 1, a low-complexity repeat in genome 2
    gs[1] = gs[1][:200] + gs[0][100:300] + gs[1][400:]
    if with_repeat:
        gs[2] = gs[2][:100] + "A" * 80 + gs[2][180:]
    seq = np.frombuffer("".join(gs).encode(), np.uint8).copy()
    off = np.cumsum([0] + [len(x) for x in gs]).astype(np.uint64)
    return gs, seq, off


def _brute_db(gs, k, w, canonical):
    db = {}
    for g, s in enumerate(gs):
        for (p, code, st) in brute_minimizers(s, k, w, canonical):
            db.setdefault(code, []).append((g, p, st))
    return db


@pytest.mark.parametrize("k,w,canonical", [(5, 4, 0), (7, 5, 1), (11, 3, 1)])
def test_index_lookup_matches_brute_force(oracle_lib, k, w, canonical):
    rng = np.random.default_rng(7 + k)
    gs, seq, off = _tiny_db(rng)
    ix = oracle.Index(seq, off, k, w, canonical)
    db = _brute_db(gs, k, w, canonical)
    assert ix.n_occ == sum(len(v) for v in db.values())
    for code, occ in db.items():
        g, p, st = ix.lookup(code)
        assert list(zip(g.tolist(), p.tolist(), st.tolist())) == sorted(occ)
    assert len(ix.lookup((1 << (2 * k)) - 1)[0]) == len(db.get((1 << (2 * k)) - 1, []))


@pytest.mark.parametrize("max_occ", [1, 3, 1024])
def test_count_hits_matches_brute_force(oracle_lib, max_occ):
    rng = np.random.default_rng(11)
    k, w, can = 7, 5, 1
    gs, seq, off = _tiny_db(rng)
    db = _brute_db(gs, k, w, can)
    reads = []
    for _ in range(40):
        g = int(rng.integers(0, len(gs)))
        p = int(rng.integers(0, len(gs[g]) - 60))
        r = gs[g][p:p + 60]
        if rng.random() < 0.5:
            r = r[::-1].translate(_RC)
        reads.append(r)
    reads.append("A" * 60)
    reads.append("ACGT" * 3)  # too short for any window
    exp = np.zeros(len(gs), np.uint64)
    for r in reads:
        for (_, code, _) in brute_minimizers(r, k, w, can):
            occ = db.get(code, [])
            if len(occ) > max_occ:
                continue
            for (g, _, _) in occ:
                exp[g] += 1
    rs = np.frombuffer("".join(reads).encode(), np.uint8).copy()
    ro = np.cumsum([0] + [len(r) for r in reads]).astype(np.uint64)
    ix = oracle.Index(seq, off, k, w, can)
    got = oracle.count_hits(ix, rs, ro, max_occ)
    assert got.tolist() == exp.tolist()


def test_keep_mask_hand_cases(oracle_lib):
    # normalised cutoff 1e-4 (Results, "Evaluation Methodology"), strictly above
    assert oracle.keep_mask(np.array([10000, 1, 2, 0], np.uint64), 1, 10000).tolist() == [1, 0, 1, 0]
    assert oracle.keep_mask(np.array([0, 0, 0], np.uint64), 1, 10000).tolist() == [0, 0, 0]
    assert oracle.keep_mask(np.array([4, 2, 3], np.uint64), 1, 2).tolist() == [1, 0, 1]
    big = np.array([2 ** 62, 2 ** 62 // 10000 + 1, 2 ** 62 // 10000], np.uint64)
    assert oracle.keep_mask(big, 1, 10000).tolist() == [1, 1, 0]


# ---------------------------------------------------------------------------------------
# SneakySnake: hand examples, closed-form reduction, exact restatement, bounds
# ---------------------------------------------------------------------------------------
def _golden_eda():
    rows = []
    with open(os.path.join(HERE, "golden", "eda_hand.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            E, r, W, d = line.split()
            rows.append((int(E), r, W, int(d)))
    return rows


def test_eda_hand_worked_examples(oracle_lib):
    rows = _golden_eda()
    assert len(rows) >= 8
    for E, r, W, d in rows:
        assert oracle.eda(r, W, E) == d, (E, r, W)


def _map(r, W, E, obst=None):
    n = len(r)
    M = np.zeros((2 * E + 1, n), bool)
    for di, d in enumerate(range(-E, E + 1)):
        for j in range(n):
            x = E + j + d
            M[di, j] = (obst is not None and obst[x]) or (r[j] != W[x])
    return M


def _greedy_by_dp(M, E):
    """Exact restatement: the least number of obstacles needed to cross the map when, from
    column c, one may follow any row's zero run for any length (possibly 0) and then must
    pay one obstacle to step over the next column -- minimised over all choices by DP."""
    rows, n = M.shape
    INF = 10 ** 9
    f = [INF] * (n + 2)
    f[n] = 0
    f[n + 1] = 0
    for c in range(n - 1, -1, -1):
        best = INF
        for d in range(rows):
            run = 0
            while c + run < n and not M[d, c + run]:
                run += 1
            for e in range(c, c + run + 1):
                best = min(best, 0 if e >= n else 1 + f[e + 1])
        f[c] = best
    return min(f[0], E + 1)


def _banded_ed(r, W, E, obst=None):
    """Edit distance of all of r against a substring of W with the alignment confined to
    diagonals d = j - i - E in [-E, E] (free start and end inside the band)."""
    n, m = len(r), len(W)
    INF = 10 ** 9
    D = [[INF] * (m + 1) for _ in range(n + 1)]
    for j in range(0, 2 * E + 1):
        D[0][j] = 0
    for i in range(0, n + 1):
        for j in range(0, m + 1):
            if not (0 <= j - i <= 2 * E):
                continue
            if i == 0:
                continue
            v = INF
            if j > 0 and D[i - 1][j - 1] < INF:
                mis = (obst is not None and obst[j - 1]) or r[i - 1] != W[j - 1]
                v = min(v, D[i - 1][j - 1] + int(mis))
            if D[i - 1][j] < INF:
                v = min(v, D[i - 1][j] + 1)          # read base not in the window
            if j > 0 and D[i][j - 1] < INF:
                v = min(v, D[i][j - 1] + 1)          # window base skipped
            D[i][j] = v
    return min(D[n][j] for j in range(n, min(m, n + 2 * E) + 1))


def _rand_pair(rng, n, E, alphabet="ACGT", edits=None):
    r = "".join(rng.choice(list(alphabet), n))
    W = list("".join(rng.choice(list(alphabet), n + 2 * E)))
    if edits is not None:
        # plant r near diagonal 0 with a few random edits
        body = list(r)
        for _ in range(edits):
            t = int(rng.integers(0, 3))
            p = int(rng.integers(0, len(body))) if body else 0
            if t == 0 and body:
                body[p] = rng.choice([b for b in alphabet if b != body[p]] or list(alphabet))
            elif t == 1:
                body.insert(p, rng.choice(list(alphabet)))
            elif body:
                del body[p]
        s = E + int(rng.integers(-E, E + 1)) if E else 0
        s = max(0, min(s, 2 * E))
        for i, b in enumerate(body):
            if s + i < len(W):
                W[s + i] = b
    return r, "".join(W)


def test_eda_E0_is_capped_hamming(oracle_lib):
    rng = np.random.default_rng(3)
    for _ in range(300):
        n = int(rng.integers(1, 40))
        r, W = _rand_pair(rng, n, 0, edits=int(rng.integers(0, 3)))
        ham = sum(a != b for a, b in zip(r, W))
        assert oracle.eda(r, W, 0) == min(ham, 1)


def test_eda_equals_exact_dp_restatement(oracle_lib):
    rng = np.random.default_rng(5)
    for trial in range(400):
        n = int(rng.integers(1, 24))
        E = int(rng.integers(0, 5))
        alpha = "ACGT" if trial % 2 else "AC"
        r, W = _rand_pair(rng, n, E, alpha, edits=int(rng.integers(0, E + 3)))
        obst = None
        if trial % 5 == 0:
            obst = np.zeros(n + 2 * E, bool)
            obst[: int(rng.integers(0, E + 1))] = True
            obst[len(obst) - int(rng.integers(0, E + 1)):] = True
        M = _map(r, W, E, obst)
        assert oracle.eda(r, W, E, obst) == _greedy_by_dp(M, E), (r, W, E)


def test_eda_bounds_no_false_reject(oracle_lib):
    """Upper bounds: Hamming distance on every diagonal, and the banded edit distance (so a
    pair whose band-restricted edit distance is <= E is never rejected). Lower bound: the
    number of columns where every diagonal is an obstacle."""
    rng = np.random.default_rng(9)
    for trial in range(500):
        n = int(rng.integers(1, 13))
        E = int(rng.integers(0, 4))
        alpha = "ACGT" if trial % 3 else "AG"
        r, W = _rand_pair(rng, n, E, alpha, edits=int(rng.integers(0, 2 * E + 2)))
        got = oracle.eda(r, W, E)
        M = _map(r, W, E)
        ham = min(int(M[d].sum()) for d in range(2 * E + 1))
        assert got <= min(ham, E + 1)
        assert got <= min(_banded_ed(r, W, E), E + 1)
        walls = int(M.all(axis=0).sum())
        assert got >= min(walls, E + 1)


def test_eda_exhaustive_tiny(oracle_lib):
    """All reads of length 4 over {A, C} against all windows of length 6 (E = 1)."""
    E = 1
    for r in itertools.product("AC", repeat=4):
        for W in itertools.product("AC", repeat=6):
            r_, W_ = "".join(r), "".join(W)
            got = oracle.eda(r_, W_, E)
            assert got == _greedy_by_dp(_map(r_, W_, E), E)
            assert got <= min(_banded_ed(r_, W_, E), E + 1)


def test_eda_substring_on_any_diagonal_is_zero(oracle_lib):
    rng = np.random.default_rng(13)
    for _ in range(200):
        n = int(rng.integers(1, 60))
        E = int(rng.integers(0, 8))
        r = "".join(rng.choice(list("ACGT"), n))
        W = list("".join(rng.choice(list("ACGT"), n + 2 * E)))
        s = int(rng.integers(0, 2 * E + 1))
        W[s:s + n] = list(r)
        assert oracle.eda(r, "".join(W), E) == 0


def test_eda_all_obstacles(oracle_lib):
    for n, E in [(1, 0), (5, 2), (10, 3), (3, 7)]:
        r = "A" * n
        W = "A" * (n + 2 * E)
        obst = np.ones(n + 2 * E, bool)
        assert oracle.eda(r, W, E, obst) == min(n, E + 1)


# ---------------------------------------------------------------------------------------
# mapping: planted truth and hand-computed profiles
# ---------------------------------------------------------------------------------------
def _rand_genomes(rng, lens):
    return ["".join(rng.choice(list("ACGT"), L)) for L in lens]


def _pack(strs):
    seq = np.frombuffer("".join(strs).encode(), np.uint8).copy()
    off = np.cumsum([0] + [len(s) for s in strs]).astype(np.uint64)
    return seq, off


def test_error_free_reads_map_to_source(oracle_lib):
    """An error-free read taken from a genome (either strand, canonical seeds) maps there at
    distance 0 with window start = source position - E, and every read minimizer is a seed
    match of that location (full windows of the read are windows of the genome)."""
    rng = np.random.default_rng(17)
    k, w, E = 15, 10, 5
    gs = _rand_genomes(rng, [3000, 2500, 4000])
    seq, off = _pack(gs)
    ix = oracle.Index(seq, off, k, w, 1)
    reads, truth = [], []
    for i in range(60):
        g = int(rng.integers(0, 3))
        n = int(rng.integers(80, 200))
        p = int(rng.integers(0, len(gs[g]) - n))
        s = gs[g][p:p + n]
        st = int(rng.random() < 0.5)
        reads.append(s[::-1].translate(_RC) if st else s)
        truth.append((g, p, st, n))
    rs, ro = _pack(reads)
    prm = oracle.params(e_abs=E, e_permille=0, min_seeds=2)
    res = oracle.classify(ix, rs, ro, prm)
    for i, (g, p, st, n) in enumerate(truth):
        nm = len(brute_minimizers(reads[i], k, w, 1))
        top = res["locs"][i, 0]
        assert res["taxon"][i] == g
        assert top["genome"] == g and top["strand"] == st and top["dist"] == 0
        assert top["wstart"] == p - E
        assert top["seeds"] == nm


def test_profile_hand_computed_unique_and_multi(oracle_lib):
    """g0 = X+A, g1 = X+B, g2 = C. Reads: 3 from C (unique g2), 1 from A (unique g0), 2 from
    the shared X (multi {g0, g1}). U = (1, 0, 3); each multi read adds U0/(U0+U1) = 1 to g0.
    Abundance = (1+2, 0, 3) / 6 = (0.5, 0, 0.5)."""
    rng = np.random.default_rng(19)
    X, A, B, C = _rand_genomes(rng, [2000, 1500, 1500, 3000])
    gs = [X + A, X + B, C]
    seq, off = _pack(gs)
    ix = oracle.Index(seq, off, 15, 10, 0)
    reads = [C[100:250], C[1000:1150], C[2500:2650], A[600:750], X[300:450], X[1200:1350]]
    rs, ro = _pack(reads)
    res = oracle.classify(ix, rs, ro, oracle.params(e_abs=6, e_permille=0, min_seeds=2))
    assert res["taxon"].tolist() == [2, 2, 2, 0, 0, 0]
    assert res["U"].tolist() == [1, 0, 3]
    assert res["multi"][4].tolist()[:2] == [0, 1] and res["multi"][5].tolist()[:2] == [0, 1]
    np.testing.assert_allclose(res["abundance"], [0.5, 0.0, 0.5], atol=1e-15)


def test_profile_split_and_cutoff_hand_cases(oracle_lib):
    # U = (1, 3), two multi reads over {0, 1}: M = 2*(1/4, 3/4) -> a = (1.5, 4.5)/6
    multi = np.array([[0, 1, -1], [0, 1, -1], [-1, -1, -1]], np.int32)
    a = oracle.abundance(np.array([1, 3], np.uint64), multi, 3, 1e-4)
    np.testing.assert_allclose(a, [0.25, 0.75], atol=1e-15)
    # U = (0, 0, 3), multi {0,1} twice with no unique support: 1/2 each -> (1, 1, 3)/5
    multi = np.array([[0, 1, -1], [0, 1, -1]], np.int32)
    a = oracle.abundance(np.array([0, 0, 3], np.uint64), multi, 3, 1e-4)
    np.testing.assert_allclose(a, [0.2, 0.2, 0.6], atol=1e-15)
    # the same with a 25% cutoff: 0.2 < 0.25 are dropped, the rest renormalised
    a = oracle.abundance(np.array([0, 0, 3], np.uint64), multi, 3, 0.25)
    np.testing.assert_allclose(a, [0.0, 0.0, 1.0], atol=1e-15)
    # nothing classified: all zeros
    a = oracle.abundance(np.zeros(4, np.uint64), np.full((3, 3), -1, np.int32), 3, 1e-4)
    assert a.tolist() == [0.0] * 4
    # exactly at the cutoff is kept ("below 0.01%" is dropped)
    U = np.array([9999, 1], np.uint64)
    a = oracle.abundance(U, np.full((1, 3), -1, np.int32), 3, 1e-4)
    np.testing.assert_allclose(a, [0.9999, 0.0001], atol=1e-15)


def test_containment_drops_low_genomes(oracle_lib):
    """With a 1/2 normalised cutoff, a genome hit by one read while another is hit by ten is
    dropped, so its read maps nowhere (stage 1 feeds stage 2)."""
    rng = np.random.default_rng(23)
    gs = _rand_genomes(rng, [5000, 5000])
    seq, off = _pack(gs)
    ix = oracle.Index(seq, off, 15, 10, 0)
    reads = [gs[0][i * 400:i * 400 + 150] for i in range(10)] + [gs[1][700:850]]
    rs, ro = _pack(reads)
    res = oracle.classify(ix, rs, ro, oracle.params(e_abs=6, e_permille=0, min_seeds=2,
                                                    cont_num=1, cont_den=2))
    assert res["keep"].tolist() == [1, 0]
    assert res["taxon"].tolist() == [0] * 10 + [-1]
    res = oracle.classify(ix, rs, ro, oracle.params(e_abs=6, e_permille=0, min_seeds=2))
    assert res["taxon"].tolist() == [0] * 10 + [1]


def test_invariants_on_tiny_workload(oracle_lib):
    c = gen.config(1, n_reads=3000)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    ix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    prm = oracle.params(e_abs=c["e_abs"], e_permille=0, min_seeds=c["min_seeds"])
    res = oracle.classify(ix, r.seq, r.offsets, prm)
    nl = res["nloc"]
    L = res["locs"]
    assert (nl <= 3).all()
    for i in range(r.n):
        s = L[i, :nl[i]]["seeds"]
        assert (s >= c["min_seeds"]).all() and (np.diff(s.astype(np.int64)) <= 0).all()
        assert (L[i, nl[i]:]["genome"] == -1).all()
        d = L[i, :nl[i]]["dist"]
        assert (d <= c["e_abs"] + 1).all()
        acc = d <= c["e_abs"]
        assert (res["taxon"][i] >= 0) == bool(acc.any())
    a = res["abundance"]
    assert abs(a.sum() - 1.0) < 1e-12 and (a >= 0).all()
    # planted truth: reads from a genome are classified to it almost always
    src = r.truth_genome >= 0
    assert (res["taxon"][src] == r.truth_genome[src]).mean() > 0.98
    assert (res["taxon"][~src] < 0).all()


def _brute_hits(read, gs, k, w, can):
    """Seed matches (g, rel, diag) of a read, by brute-force enumeration of every genome's
    minimizers; diag is the read start on the genome's forward strand."""
    db = _brute_db(gs, k, w, can)
    n = len(read)
    out = []
    for (rp, code, rst) in brute_minimizers(read, k, w, can):
        for (g, gp, gst) in db.get(code, []):
            rel = rst ^ gst
            out.append((g, rel, gp - (n - k - rp if rel else rp)))
    return out


def test_location_spans_exactly_E_diagonals(oracle_lib):
    """A read missing E genome bases in its middle has seed matches on diagonals p and
    p + E. A location takes every match with diag <= d0 + E, so all of them form ONE
    location whose seed count is the number of matches on those two diagonals."""
    rng = np.random.default_rng(29)
    k, w, E = 11, 5, 6
    gs = _rand_genomes(rng, [4000])
    seq, off = _pack(gs)
    ix = oracle.Index(seq, off, k, w, 0)
    for p in [500, 1500, 2500]:
        read = gs[0][p:p + 70] + gs[0][p + 70 + E:p + 150 + E]
        hits = _brute_hits(read, gs, k, w, 0)
        on = [h for h in hits if h[2] in (p, p + E)]
        assert any(h[2] == p for h in on) and any(h[2] == p + E for h in on)
        assert len(on) == len(hits)
        rs, ro = _pack([read])
        res = oracle.classify(ix, rs, ro, oracle.params(e_abs=E, e_permille=0, min_seeds=2))
        assert res["nloc"][0] == 1
        top = res["locs"][0, 0]
        assert top["seeds"] == len(on) and top["wstart"] == p - E


def test_window_outside_genome_is_obstacle(oracle_lib):
    """A read overhanging the genome start: the window bases before position 0 match
    nothing. The expected distance is the exact DP walk over a map built here from the
    genome with an explicit obstacle mask."""
    rng = np.random.default_rng(31)
    k, w, E = 11, 5, 6
    for trial in range(6):
        gs = _rand_genomes(rng, [3000])
        seq, off = _pack(gs)
        ix = oracle.Index(seq, off, k, w, 0)
        over = 2 + trial % 4
        pre = "".join(rng.choice(list("ACGT"), over))
        read = pre + gs[0][:150 - over]
        if trial % 2:   # overhang at the genome end instead
            read = gs[0][-(150 - over):] + pre
        rs, ro = _pack([read])
        res = oracle.classify(ix, rs, ro, oracle.params(e_abs=E, e_permille=0, min_seeds=2))
        top = res["locs"][0, 0]
        ws = int(top["wstart"])
        W, obst = [], []
        for x in range(len(read) + 2 * E):
            gp = ws + x
            inside = 0 <= gp < len(gs[0])
            W.append(gs[0][gp] if inside else "A")
            obst.append(not inside)
        assert any(obst)
        exp = _greedy_by_dp(_map(read, "".join(W), E, np.array(obst)), E)
        assert top["dist"] == exp
        # the overhanging bases cannot be matched: the read is not at distance 0
        assert exp >= 1


def test_window_does_not_run_into_the_next_genome(oracle_lib):
    """The read overhangs genome 0's end with exactly the first bases of genome 1; window
    bases past genome 0's last position are still obstacles (genomes are separate)."""
    rng = np.random.default_rng(37)
    k, w, E = 11, 5, 6
    for over in (1, 2, 3, 5):
        gs = _rand_genomes(rng, [3000, 3000])
        seq, off = _pack(gs)
        ix = oracle.Index(seq, off, k, w, 0)
        read = gs[0][-(150 - over):] + gs[1][:over]
        rs, ro = _pack([read])
        res = oracle.classify(ix, rs, ro, oracle.params(e_abs=E, e_permille=0, min_seeds=2))
        top = res["locs"][0, 0]
        assert top["genome"] == 0
        ws = int(top["wstart"])
        W = [gs[0][ws + x] if 0 <= ws + x < len(gs[0]) else "A" for x in range(len(read) + 2 * E)]
        obst = np.array([not (0 <= ws + x < len(gs[0])) for x in range(len(read) + 2 * E)])
        assert top["dist"] == _greedy_by_dp(_map(read, "".join(W), E, obst), E) >= 1


def test_threaded_index_build_is_identical(oracle_lib):
    """The threaded build used for large verification runs gives the single-threaded index."""
    c = gen.config(2, n_genomes=30, genome_len=20_000, n_reads=2000)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    a = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    b = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"], threads=5)
    assert a.n_occ == b.n_occ
    p = oracle.params(e_abs=8, e_permille=0, min_seeds=3)
    ra, rb = oracle.classify(a, r.seq, r.offsets, p), oracle.classify(b, r.seq, r.offsets, p)
    for key in ("taxon", "nloc", "genome_hits", "U"):
        assert np.array_equal(ra[key], rb[key])
    assert np.array_equal(ra["locs"], rb["locs"])
    for code in np.unique(oracle.minimizers(g.genome(3), c["k"], c["w"], 1)[0])[:200]:
        assert [x.tolist() for x in a.lookup(int(code))] == [x.tolist() for x in b.lookup(int(code))]


def test_rank_ties_break_by_strand_then_first_diagonal(oracle_lib):
    """Hand-worked ranking of equal-seed locations (Methods, "Empirically Determined
    Parameters": the top three locations by seed count). One genome holds an exact copy of
    the read S at p1, its reverse complement at p2 and S again at p3, with p1 < p2 < p3. With
    canonical seeds every read minimizer matches all three copies, so the three locations
    tie on seeds and on genome. Written by hand from the ranking reading (seeds descending,
    then genome, strand and first diagonal ascending), the order is (+, p1), (+, p3), (-, p2):
    strand before diagonal, both ascending. A second genome holding one forward copy ranks
    after every location of genome 0, whatever its strand."""
    rng = np.random.default_rng(41)
    k, w, E, n = 15, 10, 4, 150
    S = "".join(rng.choice(list("ACGT"), n))
    rcS = S[::-1].translate(_RC)
    f = _rand_genomes(rng, [300, 400, 500, 300, 350, 250])
    g0 = f[0] + S + f[1] + rcS + f[2] + S + f[3]
    p1 = len(f[0])
    p2 = p1 + n + len(f[1])
    p3 = p2 + n + len(f[2])
    g1 = f[4] + S + f[5]
    q1 = len(f[4])
    seq, off = _pack([g0, g1])
    ix = oracle.Index(seq, off, k, w, 1)
    nm = len(brute_minimizers(S, k, w, 1))
    assert nm >= 3
    rs, ro = _pack([S])
    res = oracle.classify(ix, rs, ro, oracle.params(e_abs=E, e_permille=0, min_seeds=2, top_n=3))
    got = [(int(L["genome"]), int(L["strand"]), int(L["wstart"]), int(L["seeds"]), int(L["dist"]))
           for L in res["locs"][0]]
    assert got == [(0, 0, p1 - E, nm, 0), (0, 0, p3 - E, nm, 0), (0, 1, p2 - E, nm, 0)]
    # with room for all four, genome 1's forward copy comes last
    res = oracle.classify(ix, rs, ro, oracle.params(e_abs=E, e_permille=0, min_seeds=2, top_n=4))
    assert [(int(L["genome"]), int(L["strand"]), int(L["wstart"])) for L in res["locs"][0]] == \
        [(0, 0, p1 - E), (0, 0, p3 - E), (0, 1, p2 - E), (1, 0, q1 - E)]
    # the reverse-complemented read: the rc copy is now the forward-strand location
    rs, ro = _pack([rcS])
    res = oracle.classify(ix, rs, ro, oracle.params(e_abs=E, e_permille=0, min_seeds=2, top_n=3))
    assert [(int(L["genome"]), int(L["strand"]), int(L["wstart"])) for L in res["locs"][0]] == \
        [(0, 0, p2 - E), (0, 1, p1 - E), (0, 1, p3 - E)]


def _brute_locations(read, db, k, w, can, E, min_seeds, top_n, max_occ):
    """Mapping locations of one read from a brute-force seed enumeration (db from
    _brute_db): matches of keys with more than max_occ occurrences skipped, then greedy
    diagonal bands per (genome, strand), at least min_seeds matches, ranked by seeds
    descending then genome, strand, first diagonal; (genome, strand, wstart, seeds)."""
    n = len(read)
    hits = []
    for (rp, code, rst) in brute_minimizers(read, k, w, can):
        occ = db.get(code, [])
        if len(occ) > max_occ:
            continue
        for (g, gp, gst) in occ:
            rel = rst ^ gst
            hits.append((g, rel, gp - (n - k - rp if rel else rp)))
    hits.sort()
    locs, i = [], 0
    while i < len(hits):
        g, rel, d0 = hits[i]
        j = i + 1
        while j < len(hits) and hits[j][0] == g and hits[j][1] == rel and hits[j][2] <= d0 + E:
            j += 1
        if j - i >= min_seeds:
            locs.append((-(j - i), g, rel, d0))
        i = j
    locs.sort()
    return [(g, rel, d0 - E, -s) for (s, g, rel, d0) in locs[:top_n]]


def test_mapping_repeat_filter_at_the_exact_occurrence_count(oracle_lib):
    """The repeat filter at mapping time (Methods, "Index Construction & Querying": minimap2
    skips over-represented minimizers; reading: a key with more than max_occ occurrences is
    skipped). A 120-base segment X sits in genomes 0, 1 and 2, so its minimizers occur three
    times; reads spanning X are mapped with max_occ = 3 (X's matches count: 3 is not more
    than 3) and with max_occ = 2 (they are skipped). Expected locations come from a
    brute-force enumeration of every genome's minimizers, with the filter applied here; the
    two settings give different expected locations, so the boundary decides the test."""
    rng = np.random.default_rng(43)
    k, w, can, E = 11, 5, 1, 5
    X = "".join(rng.choice(list("ACGT"), 120))
    f = _rand_genomes(rng, [400, 500, 300, 450, 350, 600, 900])
    gs = [f[0] + X + f[1], f[2] + X + f[3], f[4] + X[::-1].translate(_RC) + f[5], f[6]]
    seq, off = _pack(gs)
    ix = oracle.Index(seq, off, k, w, can)
    db = _brute_db(gs, k, w, can)
    x_codes = {code for (_, code, _) in brute_minimizers(X, k, w, can)}
    assert x_codes and all(len(db[c]) == 3 for c in x_codes)
    reads = []
    for t in range(12):
        a = int(rng.integers(len(f[0]) - 80, len(f[0]) + 40))
        r = gs[0][a:a + 150]
        reads.append(r[::-1].translate(_RC) if t % 2 else r)
    reads.append(X)
    rs, ro = _pack(reads)
    expect = {}
    for max_occ in (3, 2):
        prm = oracle.params(e_abs=E, e_permille=0, min_seeds=2, top_n=3, max_occ=max_occ)
        res = oracle.classify(ix, rs, ro, prm)
        # a genome is dropped only with no counted match at all (tiny batch, cutoff 1e-4)
        assert res["keep"].tolist()[:3] == ([1, 1, 1] if max_occ == 3 else [1, 0, 0])
        expect[max_occ] = []
        for i, r in enumerate(reads):
            exp = _brute_locations(r, db, k, w, can, E, 2, 3, max_occ)
            got = [(int(L["genome"]), int(L["strand"]), int(L["wstart"]), int(L["seeds"]))
                   for L in res["locs"][i][:res["nloc"][i]]]
            assert got == exp, (max_occ, i)
            expect[max_occ].append(exp)
    assert expect[3] != expect[2]
    # the read X itself: three locations at max_occ = 3, none at max_occ = 2
    assert len(expect[3][-1]) == 3 and expect[2][-1] == []
