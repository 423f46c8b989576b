"""Taxonomic roll-up and the CAMI / OPAL profile output (Fig. 1, 3b). The oracle's roll-up is
pinned by hand-worked trees and by the invariant that every root holds the sum of its
genomes; the library's roll-up (host code, no GPU) must equal it; the written profile is
parsed back."""
import io

import numpy as np
import pytest

import gen
import oracle


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def test_hand_worked_tree():
    # root 0 <- 1 <- {3 (g0), 4 (g1)};  root 0 <- 2 <- 5 (g2);  a second root 6 (g3 directly)
    parent = [-1, 0, 0, 1, 1, 2, -1]
    gnode = [3, 4, 5, 6]
    a = [0.5, 0.25, 0.125, 0.125]
    want = [0.875, 0.75, 0.125, 0.5, 0.25, 0.125, 0.125]
    assert np.array_equal(oracle.rollup(a, gnode, parent), want)


def test_two_genomes_on_one_leaf_and_empty_profile():
    parent = [-1, 0, 0]
    assert np.array_equal(oracle.rollup([0.3, 0.7], [1, 1], parent), [1.0, 1.0, 0.0])
    assert np.array_equal(oracle.rollup([0.0, 0.0], [1, 2], parent), [0.0, 0.0, 0.0])


def test_cycles_and_bad_nodes_are_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.rollup([1.0], [1], [1, 0])       # 0 <-> 1
    with pytest.raises(oracle.OracleError):
        oracle.rollup([1.0], [5], [-1])


@pytest.fixture(scope="module")
def mtlib():
    from paper_2311_02029_gb300 import _build
    _build.build()
    import paper_2311_02029_gb300 as m
    return m


def test_library_rollup_equals_oracle_on_the_clade_taxonomy(mtlib):
    c = gen.config(2, n_genomes=40, genome_len=1000)
    g = gen.make_genomes(c)
    t = gen.make_taxonomy(g)
    rng = np.random.default_rng(8)
    a = rng.dirichlet(np.ones(g.n))
    a[rng.random(g.n) < 0.3] = 0.0
    a /= a.sum()
    got = mtlib.profile_rollup(a, t.genome_node, t.parent)
    ref = oracle.rollup(a, t.genome_node, t.parent)
    assert np.abs(got - ref).max() <= 1e-15
    assert abs(got[0] - 1.0) < 1e-12
    with pytest.raises(mtlib.MtError):
        mtlib.profile_rollup([1.0], [1], [1, 0])


def test_cami_profile_round_trip(mtlib):
    c = gen.config(2, n_genomes=20, genome_len=1000)
    g = gen.make_genomes(c)
    t = gen.make_taxonomy(g)
    a = np.zeros(g.n)
    a[[0, 1, 13]] = [0.5, 0.3, 0.2]
    node = mtlib.profile_rollup(a, t.genome_node, t.parent)
    f = io.StringIO()
    mtlib.write_cami_profile(f, "sample_1", t, node)
    lines = f.getvalue().splitlines()
    assert lines[:3] == ["@SampleID:sample_1", "@Version:0.9.1", "@Ranks:superkingdom|genus|species"]
    head = lines.index("@@TAXID\tRANK\tTAXPATH\tTAXPATHSN\tPERCENTAGE")
    rows = [x.split("\t") for x in lines[head + 1:]]
    assert [r[1] for r in rows] == ["superkingdom", "genus", "genus", "species", "species", "species"]
    byname = {r[3].split("|")[-1]: float(r[4]) for r in rows}
    assert byname == {"Synthetica": 100.0, "Clade_0": 80.0, "Clade_1": 20.0,
                      "Genome_0": 50.0, "Genome_1": 30.0, "Genome_13": 20.0}
    g13 = [r for r in rows if r[3].endswith("Genome_13")][0]
    assert g13[2] == "%d|%d|%d" % (10 ** 6, 10 ** 6 + 2, 10 ** 6 + 1 + 2 + 13)
