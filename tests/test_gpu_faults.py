"""Host-side fault injection (the paper has none; this is the serving side's failure handling).
The library's device allocations are made to fail one at a time with mt_inject_alloc_failure:
the failure is decided on the host before the allocation is requested, so no GPU faults. Every
call that meets the failure must return MT_ENOMEM, hold none of the stream-ordered pool's
memory afterwards, and leave the library usable: the next call gives exactly the results of an
undisturbed call, which are themselves checked against the CPU oracle."""
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
    c = gen.config(2, n_genomes=20, genome_len=100_000, n_reads=3000)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    prm = dict(e_abs=c["e_abs"], e_permille=0, min_seeds=3, top_n=3, max_occ=1024)
    ref = oracle.classify(oix, r.seq, r.offsets, oracle_params(prm), threads=8)
    compare_classify(mt.classify(ix, r.seq, r.offsets, **prm), ref)   # also tunes the EDA kernel
    return c, g, r, ix, prm, ref


def _sweep(mt, call, check, max_n=64):
    """Fails the n-th allocation of `call` for n = 0, 1, ... until the call makes fewer than n + 1
    allocations. Returns how many allocations failed (the call's allocation count)."""
    import torch
    L = mt.lib()
    for n in range(max_n):
        torch.cuda.synchronize()
        used0 = L.mt_pool_used_bytes()
        L.mt_inject_alloc_failure(n)
        try:
            out, rc = call(), mt.MT_OK
        except mt.MtError as e:
            out, rc = None, e.status
        finally:
            L.mt_inject_alloc_failure(-1)
        torch.cuda.synchronize()
        assert L.mt_pool_used_bytes() == used0, "the call kept pool memory after failing at allocation %d" % n
        if rc == mt.MT_OK:
            check(out)
            return n
        assert rc == mt.MT_ENOMEM, "allocation %d: status %d" % (n, rc)
        check(call())          # nothing injected: the library is usable and exact
    raise AssertionError("the call still failed after %d allocations" % max_n)


def test_classify_host_buffers(mt, work):
    c, g, r, ix, prm, ref = work
    assert _sweep(mt, lambda: mt.classify(ix, r.seq, r.offsets, **prm), lambda o: compare_classify(o, ref)) >= 3


def test_classify_device_buffers(mt, work):
    import torch
    c, g, r, ix, prm, ref = work
    d_reads = torch.from_numpy(r.seq).cuda()
    d_off = torch.from_numpy(r.offsets.astype(np.int64)).cuda()
    assert _sweep(mt, lambda: mt.classify(ix, d_reads, d_off, **prm), lambda o: compare_classify(o, ref)) >= 2


def test_containment(mt, work):
    c, g, r, ix, prm, ref = work

    def check(o):
        assert np.array_equal(o["genome_hits"].astype(np.uint64), ref["genome_hits"])
        assert np.array_equal(o["keep"], ref["keep"])
    assert _sweep(mt, lambda: mt.containment(ix, r.seq, r.offsets, cont_den=10000), check) >= 1


def test_plan_create_and_classify(mt, work):
    """A plan's workspace is its one device allocation: creating a plan fails cleanly, and a
    plan made afterwards classifies exactly (first call direct, then replayed from its graph)."""
    import torch
    c, g, r, ix, prm, ref = work
    free0, _ = torch.cuda.mem_get_info()
    n = int(r.n)

    def make():
        return mt.Plan(ix, max_reads=n, max_bases=int(r.offsets[-1]), max_read_len=int(r.lengths.max()), **prm)

    def check(pl):
        for _ in range(3):
            compare_classify(pl.classify(r.seq, r.offsets), ref)
        pl.close()
    assert _sweep(mt, make, check) >= 1
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < (64 << 20)      # no plan workspace left behind


def test_eda_batch(mt):
    import torch
    p = gen.make_eda_pairs(gen.config(3), n_pairs=20_000, seed=77)
    rs = torch.from_numpy(p.read_seq).cuda()
    ro = torch.from_numpy(p.read_off.astype(np.int64)).cuda()
    ws = torch.from_numpy(p.win_seq).cuda()
    wo = torch.from_numpy(p.win_off.astype(np.int64)).cuda()
    rw = mt.pack_seqs(rs, ro, mt.packed_words(p.read_off))
    ww = mt.pack_seqs(ws, wo, mt.packed_words(p.win_off))
    pr = torch.from_numpy(p.pair_read.astype(np.int32)).cuda()
    E = torch.from_numpy(p.E.astype(np.int16)).cuda()
    want = oracle.eda_batch(p, threads=8)

    def check(d):
        assert np.array_equal(d.cpu().numpy(), want)
    assert _sweep(mt, lambda: mt.eda_batch(rw, ro, ww, wo, pr, E), check) >= 1


def test_partitioned_query(mt, work):
    """Every mt_part_* step of a database cut into batches (create, one-pass containment of all
    batches, cutoff, mapping against the subset index). The subset index is built once, outside
    the injected window (its build is not one of these calls)."""
    c, g, r, ix, prm, ref = work
    pids = mt.split_batches(g.offsets, 4)
    pbs = [mt.Index.subset(g.seq, g.offsets, ids, c["k"], c["w"], c["canonical"]) for ids in pids]
    q0 = mt.PartitionedQuery(g.n, r.seq, r.offsets)
    q0.contain_batches(pbs, pids, max_occ=prm["max_occ"])
    kept = q0.subset(1, 10000)["kept"]
    six = mt.Index.subset(g.seq, g.offsets, kept, c["k"], c["w"], c["canonical"])
    ref_q = q0.classify(six, **prm)
    q0.close()

    def run():
        q = mt.PartitionedQuery(g.n, r.seq, r.offsets)
        try:
            q.contain_batches(pbs, pids, max_occ=prm["max_occ"])
            assert np.array_equal(q.subset(1, 10000)["kept"], kept)
            return q.classify(six, **prm)
        finally:
            q.close()

    def check(o):
        for key in ("taxon", "nloc", "abundance"):
            assert np.array_equal(o[key], ref_q[key])
        assert np.array_equal(o["locs"], ref_q["locs"])
    assert _sweep(mt, run, check) >= 3
    six.close()
    for b in pbs:
        b.close()


def test_server_request_after_a_failed_one(mt, work):
    """A request whose workspace allocation fails reports MT_ENOMEM when polled; the server
    keeps serving, and the next request is exact."""
    c, g, r, ix, prm, ref = work
    need = mt.workspace_bytes(ix, int(r.offsets[-1]), r.n, int(r.lengths.max()), **prm)
    srv = mt.Server(ix, hbm_budget=need + need // 2, max_slots=1, **prm)   # too small for plans
    L = mt.lib()
    L.mt_inject_alloc_failure(0)
    try:
        rid = srv.submit(r.seq, r.offsets)
        rc, _, _ = srv.poll(rid, 120_000)
    finally:
        L.mt_inject_alloc_failure(-1)
    assert rc == mt.MT_ENOMEM
    rid = srv.submit(r.seq, r.offsets)
    rc, _, out = srv.poll(rid, 120_000)
    assert rc == mt.MT_OK
    compare_classify(out, ref)
    srv.close()
