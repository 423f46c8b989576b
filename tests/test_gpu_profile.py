"""GPU parity of the taxonomic roll-up on the device (mt_profile_rollup_device; Fig. 1, 3b;
"Taxonomic Profile Generation"): the abundance vector a device-buffer classification leaves on
the device is summed up the taxonomy without a host pass, and equals the oracle's roll-up of the
same vector (within 1e-12: only the order of additions differs); hand-worked trees; cycles and
out-of-range nodes refused."""
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


def _dev(x, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=dtype)).cuda()


def test_rollup_of_a_device_classification(mt):
    c = gen.config(2, n_genomes=40, genome_len=50_000, n_reads=20_000)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    tax = gen.make_taxonomy(g)
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    out = mt.classify(ix, _dev(r.seq, np.uint8), _dev(r.offsets, np.int64), e_abs=c["e_abs"], e_permille=0,
                      min_seeds=3, top_n=3, max_occ=1024)
    node = mt.profile_rollup_device(out["abundance"], _dev(tax.genome_node, np.int32), _dev(tax.parent, np.int32))
    a = out["abundance"].cpu().numpy()
    want = oracle.rollup(a, tax.genome_node, tax.parent)
    got = node.cpu().numpy()
    assert np.abs(got - want).max() <= 1e-12
    assert abs(got[0] - a.sum()) <= 1e-12 and got[0] > 0.99          # the root holds the whole profile
    assert np.abs(got - mt.profile_rollup(a, tax.genome_node, tax.parent)).max() <= 1e-12
    ix.close()


def test_rollup_hand_worked_and_refusals(mt):
    # root 0 <- 1 <- {3 (g0), 4 (g1)};  root 0 <- 2 <- 5 (g2);  a second root 6 (g3 directly)
    parent = [-1, 0, 0, 1, 1, 2, -1]
    a = [0.5, 0.25, 0.125, 0.125]
    got = mt.profile_rollup_device(_dev(a, np.float64), _dev([3, 4, 5, 6], np.int32), _dev(parent, np.int32))
    assert np.array_equal(got.cpu().numpy(), [0.875, 0.75, 0.125, 0.5, 0.25, 0.125, 0.125])
    with pytest.raises(mt.MtError):       # 0 <-> 1
        mt.profile_rollup_device(_dev([1.0], np.float64), _dev([1], np.int32), _dev([1, 0], np.int32))
    with pytest.raises(mt.MtError):       # genome on a node that does not exist
        mt.profile_rollup_device(_dev([1.0], np.float64), _dev([5], np.int32), _dev([-1], np.int32))
    with pytest.raises(mt.MtError):       # a parent out of range
        mt.profile_rollup_device(_dev([1.0], np.float64), _dev([0], np.int32), _dev([3], np.int32))
    # still usable
    got = mt.profile_rollup_device(_dev([0.3, 0.7], np.float64), _dev([1, 1], np.int32), _dev([-1, 0, 0], np.int32))
    assert np.array_equal(got.cpu().numpy(), [1.0, 1.0, 0.0])
