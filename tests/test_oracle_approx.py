"""Pins of the oracle's other edit-distance approximations (HD, Base Counting, q-gram, SHD;
Table 1 and the Discussion of their cost), checked against what holds independently of the
oracle: hand-worked examples (tests/golden/approx_hand.txt), the textbook bounds
BC <= q-gram-type lower bounds <= Levenshtein(read, segment) <= HD (an independent dynamic
program here), Base Counting as the q = 1 case of the separately written q-gram function,
SneakySnake <= HD on the same diagonal, and identical pairs at 0."""
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ALGO = {"hd": 1, "bc": 2, "qgram": 3, "shd": 4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _hand_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "approx_hand.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            a, E, r, w, want = line.split()
            rows.append((a, int(E), r, w, int(want)))
    return rows


@pytest.mark.parametrize("row", _hand_rows(), ids=lambda r: "%s-%s-%s" % (r[0], r[2], r[3]))
def test_hand_examples(row):
    a, E, r, w, want = row
    obst = np.array([c == "N" for c in w])
    win = w.replace("N", "A")
    assert oracle.approx(r, win, E, ALGO[a], obstacles=obst if obst.any() else None) == want


def _lev(a, b):
    """Levenshtein distance; 'N' equals nothing."""
    prev = list(range(len(b) + 1))
    for i in range(1, len(a) + 1):
        cur = [i] + [0] * len(b)
        for j in range(1, len(b) + 1):
            sub = 0 if (a[i - 1] == b[j - 1] and b[j - 1] != "N") else 1
            cur[j] = min(prev[j] + 1, cur[j - 1] + 1, prev[j - 1] + sub)
        prev = cur
    return prev[-1]


def _mutate(rng, s, k):
    s = list(s)
    for _ in range(k):
        op = rng.integers(3)
        i = int(rng.integers(len(s) + 1))
        if op == 0 and i < len(s):
            s[i] = "ACGT"[(("ACGT".index(s[i])) + 1 + int(rng.integers(3))) % 4]
        elif op == 1:
            s.insert(i, "ACGT"[int(rng.integers(4))])
        elif op == 2 and i < len(s) and len(s) > 1:
            del s[i]
    return "".join(s)


def _pairs(seed, count):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        n = int(rng.integers(3, 40))
        E = int(rng.integers(0, 7))
        r = "".join("ACGT"[x] for x in rng.integers(0, 4, n))
        core = _mutate(rng, r, int(rng.integers(0, 6)))
        L = n + 2 * E
        pre = int(rng.integers(0, 2 * E + 1))
        w = "".join("ACGT"[x] for x in rng.integers(0, 4, L))
        w = (w[:pre] + core + w[pre + len(core):])[:L]
        w = w + "".join("ACGT"[x] for x in rng.integers(0, 4, L - len(w)))
        obst = rng.random(L) < (0.1 if rng.random() < 0.3 else 0.0)
        yield r, w, E, obst


def test_bounds_against_levenshtein_on_random_pairs():
    for r, w, E, obst in _pairs(7, 400):
        o = obst if obst.any() else None
        S = "".join("N" if obst[E + j] else w[E + j] for j in range(len(r)))
        lev = min(_lev(r, S), E + 1)
        hd = oracle.approx(r, w, E, 1, o)
        bc = oracle.approx(r, w, E, 2, o)
        qg = oracle.approx(r, w, E, 3, o)
        ham = min(sum(1 for j in range(len(r)) if S[j] == "N" or S[j] != r[j]), E + 1)
        assert hd == ham
        assert bc <= lev <= hd
        assert qg <= lev
        assert oracle.qgram_q(r, w, E, 1, o) == bc
        assert oracle.approx(r, w, E, 0, o) <= hd          # SneakySnake never exceeds HD
        assert 0 <= oracle.approx(r, w, E, 4, o) <= E + 1


def test_identical_segment_gives_zero():
    rng = np.random.default_rng(3)
    for _ in range(100):
        n = int(rng.integers(1, 60))
        E = int(rng.integers(0, 6))
        r = "".join("ACGT"[x] for x in rng.integers(0, 4, n))
        w = "".join("ACGT"[x] for x in rng.integers(0, 4, E)) + r + "".join("ACGT"[x] for x in rng.integers(0, 4, E))
        for a in (0, 1, 2, 3, 4):
            assert oracle.approx(r, w, E, a) == 0


def test_counts_ignore_order_but_hamming_does_not():
    # a rotation of the segment keeps base counts (BC 0) but not positions (HD > 0)
    r = "AACCGGTTAC"
    w = "GG" + r[3:] + r[:3] + "TT"
    assert oracle.approx(r, w, 2, 2) == 0
    assert oracle.approx(r, w, 2, 1) == 3


def test_unknown_algorithm_is_rejected():
    assert oracle.approx("ACGT", "ACGT", 0, 9) == 0xFFFFFFFF
