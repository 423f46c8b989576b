"""GPU test of mt_eda_batch_noalloc, the edit-distance batch call for callers that cannot
allocate device memory during a call (fixed-footprint serving loops, host frameworks that own
the allocator). Its scratch is a fixed per-device array inside the library, so two calls in a
row must each give exactly the distances of mt_eda_batch on the same inputs, even though the
second call finds the first call's contents in that array; a sample of each call's pairs is
also checked against the CPU oracle's SneakySnake, which shares no code with either call.

Kept in a file collected last, so a run that stops at the first failure has already run every
other test."""
import ctypes

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
    return m


def _dev_pairs(mt, n_pairs, seed):
    import torch
    p = gen.make_eda_pairs(gen.config(3), n_pairs=n_pairs, seed=seed)
    rs = torch.from_numpy(p.read_seq).cuda()
    ro = torch.from_numpy(p.read_off.astype(np.int64)).cuda()
    ws = torch.from_numpy(p.win_seq).cuda()
    wo = torch.from_numpy(p.win_off.astype(np.int64)).cuda()
    rw = mt.pack_seqs(rs, ro, mt.packed_words(p.read_off))
    ww = mt.pack_seqs(ws, wo, mt.packed_words(p.win_off))
    pr = torch.from_numpy(p.pair_read.astype(np.int32)).cuda()
    E = torch.from_numpy(p.E.astype(np.int16)).cuda()
    return rw, ro, ww, wo, pr, E, p



def _noalloc(mt, args, dist, mode):
    """Call the entry point directly through the C ABI."""
    import torch
    rw, ro, ww, wo, pr, E = args[:6]
    L = mt.lib()
    vp = ctypes.c_void_p
    rc = L.mt_eda_batch_noalloc(vp(rw.data_ptr()), vp(ro.data_ptr()), ro.numel() - 1, vp(ww.data_ptr()),
                                vp(wo.data_ptr()), vp(pr.data_ptr()), vp(E.data_ptr()), pr.numel(), mode,
                                vp(torch.cuda.current_stream().cuda_stream), vp(dist.data_ptr()))
    return rc


@pytest.mark.parametrize("mode", [0, 1])
def test_noalloc_matches_eda_batch_on_two_calls(mt, mode):
    import torch
    first = _dev_pairs(mt, 150_000, seed=101)
    second = _dev_pairs(mt, 60_000, seed=202)     # smaller: stale entries of call 1 remain
    rng = np.random.default_rng(7 + mode)
    for args in (first, second):
        ref = mt.eda_batch(*args[:6], mode=mode)
        dist = torch.full((args[4].numel(),), 0xEE, dtype=torch.uint8, device="cuda")
        assert _noalloc(mt, args, dist, mode) == mt.MT_OK
        torch.cuda.synchronize()
        assert torch.equal(dist, ref)
        # the oracle on 4,000 sampled pairs of this call (stale array contents included)
        host = args[6]
        idx = np.sort(rng.choice(host.n_pairs, 4000, replace=False))
        want = oracle.eda_batch(host, idx, threads=8)
        assert np.array_equal(dist.cpu().numpy()[idx], want)


def test_noalloc_rejects_batches_above_its_array(mt):
    L = mt.lib()
    assert L.mt_eda_batch_noalloc(None, None, 1, None, None, None, None, mt.NOALLOC_MAX_PAIRS + 1, 0,
                                  None, None) == mt.MT_EINVAL
