"""Pins of the oracle's homopolymer-compressed containment seeds (minimap2's -H in the paper's
containment index, k = 28, w = 18): hand-worked compressions, runs never joining across
sequences, idempotence, and the property the compression exists for: a read whose only
differences from its genome are homopolymer lengths gets the same compressed seed hits as the
exact read."""
import numpy as np
import pytest

import gen
import oracle


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _seqs(*xs):
    seq = np.frombuffer(b"".join(x.encode() for x in xs), np.uint8).copy()
    off = np.cumsum([0] + [len(x) for x in xs]).astype(np.uint64)
    return seq, off


def test_hand_worked_compression():
    seq, off = _seqs("AAACCGTTTA", "GGGG", "", "ACGT", "AA", "AT")
    out, o = oracle.hpc(seq, off)
    parts = [out[int(o[i]):int(o[i + 1])].tobytes().decode() for i in range(len(o) - 1)]
    assert parts == ["ACGTA", "G", "", "ACGT", "A", "AT"]     # "AA" then "AT": no joining


def test_idempotent_and_identity_without_runs():
    rng = np.random.default_rng(2)
    x = gen.ascii_of(rng.integers(0, 4, 5000, dtype=np.uint8))
    off = np.array([0, 1200, 1200, 5000], np.uint64)
    a, ao = oracle.hpc(x, off)
    b, bo = oracle.hpc(a, ao)
    assert np.array_equal(a, b) and np.array_equal(ao, bo)
    y = np.frombuffer(b"ACGTACGTCT" * 10, np.uint8).copy()
    c, co = oracle.hpc(y, np.array([0, 100], np.uint64))
    assert np.array_equal(c, y)


def _stretch(rng, s):
    """The same sequence with every homopolymer run lengthened or shortened (never removed)."""
    out = []
    i = 0
    while i < len(s):
        j = i
        while j < len(s) and s[j] == s[i]:
            j += 1
        L = max(1, (j - i) + int(rng.integers(-1, 3)))
        out.append(s[i:i + 1] * L)
        i = j
    return b"".join(out)


def test_homopolymer_length_errors_keep_compressed_hits():
    c = gen.config(1, n_genomes=4, genome_len=20_000)
    g = gen.make_genomes(c)
    ix = oracle.Index(g.seq, g.offsets, 28, 18, 1, compressed=True)
    plain = oracle.Index(g.seq, g.offsets, 28, 18, 1)
    rng = np.random.default_rng(5)
    reads, stretched = [], []
    for _ in range(60):
        gi = int(rng.integers(0, 4))
        a = int(g.offsets[gi]) + int(rng.integers(0, 20_000 - 200))
        r = g.seq[a:a + 200].tobytes()
        reads.append(r)
        stretched.append(_stretch(rng, r))
    s1, o1 = _seqs(*[x.decode() for x in reads])
    s2, o2 = _seqs(*[x.decode() for x in stretched])
    h1 = oracle.count_hits(ix, s1, o1, 1024)
    h2 = oracle.count_hits(ix, s2, o2, 1024)
    assert np.array_equal(h1, h2) and h1.sum() > 0
    # the uncompressed seeds do see the length changes
    assert not np.array_equal(oracle.count_hits(plain, s1, o1, 1024), oracle.count_hits(plain, s2, o2, 1024))
