"""GPU tests of the continuous-batching request loop (mt_server_*): every request's result is
the same when it runs alone and when it runs in a mix of overlapping requests, admission by
the HBM budget, cancellation and bounded polling."""
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


@pytest.fixture(scope="module")
def work(mt):
    c = gen.config(2, n_genomes=20, genome_len=100_000, n_reads=30_000)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    prm = dict(e_abs=c["e_abs"], e_permille=0, min_seeds=3, top_n=3, max_occ=1024)
    return c, g, r, ix, prm


def _batch(r, a, b):
    seq = r.seq[int(r.offsets[a]):int(r.offsets[b])].copy()
    off = (r.offsets[a:b + 1] - r.offsets[a]).astype(np.uint64)
    return seq, off


def _same(out, ref):
    assert np.array_equal(out["taxon"], ref["taxon"])
    assert np.array_equal(out["nloc"], ref["nloc"])
    for f in ("genome", "seeds", "strand", "dist", "wstart"):
        assert np.array_equal(out["locs"][f], ref["locs"][f])
    assert np.array_equal(out["genome_hits"], ref["genome_hits"])
    assert np.abs(out["abundance"] - ref["abundance"]).max() <= 1e-6


def test_results_identical_alone_and_in_the_mix(mt, work):
    import torch
    c, g, r, ix, prm = work
    rng = np.random.default_rng(3)
    cuts = []
    for size in (1, 7, 250, 3000, 9000, 120, 5000, 1, 20000, 64, 800, 0):
        a = int(rng.integers(0, r.n - size + 1))
        cuts.append((a, a + size))
    batches = [_batch(r, a, b) for a, b in cuts]
    alone = [mt.classify(ix, s, o, **prm) for s, o in batches]
    free, _ = torch.cuda.mem_get_info()
    srv = mt.Server(ix, hbm_budget=free // 3, max_slots=3, **prm)
    ids = [srv.submit(s, o) for s, o in batches]          # all in flight together
    for rid, ref in zip(ids, alone):
        rc, lat, out = srv.poll(rid, 120_000)
        assert rc == mt.MT_OK and lat is not None and lat >= 0
        _same(out, ref)
    srv.close()
    # and against the oracle for two of them
    oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    for (s, o), out in ((batches[4], alone[4]), (batches[8], alone[8])):
        compare_classify(out, oracle.classify(oix, s, o, oracle_params(prm), threads=8))


def test_admission_by_budget(mt, work):
    c, g, r, ix, prm = work
    small = _batch(r, 0, 2000)
    big = _batch(r, 0, 30000)
    need_small = mt.workspace_bytes(ix, len(small[0]), 2000, 150, **prm)
    need_big = mt.workspace_bytes(ix, len(big[0]), 30000, 150, **prm)
    budget = need_small + need_small // 5                # too small for any slot plan
    assert need_big > budget
    srv = mt.Server(ix, hbm_budget=budget, max_slots=2, **prm)
    rid_big = srv.submit(*big)
    rid_small = srv.submit(*small)
    rc, _, _ = srv.poll(rid_big, 120_000)
    assert rc == mt.MT_ENOMEM
    rc, _, out = srv.poll(rid_small, 120_000)
    assert rc == mt.MT_OK
    _same(out, mt.classify(ix, *small, **prm))
    srv.close()


def test_cancel_and_bounded_poll(mt, work):
    c, g, r, ix, prm = work
    need = mt.workspace_bytes(ix, 30000 * 150, 30000, 150, **prm)
    srv = mt.Server(ix, hbm_budget=need + need // 2, max_slots=1, **prm)   # one at a time, no plan
    ids = [srv.submit(*_batch(r, 0, 30000)) for _ in range(4)]
    assert srv.cancel(ids[-1]) == mt.MT_OK
    rc, _, _ = srv.poll(ids[-1], 0)
    assert rc == mt.MT_ECANCELED
    for rid in ids[:-1]:
        rc, _, out = srv.poll(rid, 120_000)
        assert rc == mt.MT_OK
    assert srv.cancel(ids[0]) == mt.MT_EINVAL             # done, polled and released
    rc, _, _ = srv.poll(ids[0], 0)
    assert rc == mt.MT_EINVAL
    srv.close()


def test_server_releases_polled_requests(mt, work):
    """The server keeps no request once a poll has reported its final status: a submitted,
    finished and polled request's id is unknown afterwards, while an unpolled finished one still
    answers, and cancelling a finished unpolled request is refused as busy."""
    c, g, r, ix, prm = work
    need = mt.workspace_bytes(ix, 3000 * 150, 3000, 150, **prm)
    srv = mt.Server(ix, hbm_budget=4 * need, max_slots=1, **prm)
    a = srv.submit(*_batch(r, 0, 3000))
    b = srv.submit(*_batch(r, 3000, 6000))
    rc, _, _ = srv.poll(b, 120_000)
    assert rc == mt.MT_OK
    assert srv.cancel(a) == mt.MT_EBUSY    # one slot, first in first out: a finished before b
    rc, _, _ = srv.poll(a, 0)
    assert rc == mt.MT_OK
    for rid in (a, b):
        assert mt.lib().mt_server_poll(srv._h, rid, 0, None) == mt.MT_EINVAL
        assert srv.cancel(rid) == mt.MT_EINVAL
    srv.close()


def test_requests_into_reused_output_arrays(mt, work):
    """Caller-owned output arrays, larger than the batch and reused by later requests, hold each
    request's results exactly; arrays too small are refused before anything is queued."""
    import torch
    c, g, r, ix, prm = work
    free, _ = torch.cuda.mem_get_info()
    srv = mt.Server(ix, hbm_budget=free // 3, max_slots=2, **prm)
    cap, G = 6000, g.n
    buf = dict(taxon=np.full(cap, 7, np.int32), nloc=np.full(cap, 9, np.uint8),
               locs=np.zeros((cap, 3), mt.LOC_DTYPE), genome_hits=np.zeros(G, np.uint64),
               abundance=np.zeros(G, np.float64))
    for a, b in ((0, 5000), (7000, 7100), (100, 6100)):
        seq, off = _batch(r, a, b)
        ref = mt.classify(ix, seq, off, **prm)
        rid = srv.submit(seq, off, out=buf)
        rc, lat, out = srv.poll(rid, 60_000)
        assert rc == mt.MT_OK and len(out["taxon"]) == b - a
        _same(out, ref)
        assert out["taxon"].base is buf["taxon"] or np.shares_memory(out["taxon"], buf["taxon"])
    seq, off = _batch(r, 0, cap + 1)
    with pytest.raises(ValueError):
        srv.submit(seq, off, out=buf)
    srv.close()
