"""Full-size bit-exact verification: every read of the medium workload (10^7 reads of 150 bp,
200 x 2 Mb reference, the bench's configuration) through the batched call against the oracle
sharded over all host cores; and a stream of serving requests (Poisson 20 batches/s,
log-uniform 10^3-10^6 reads, drawn from the same reads) through the request loop, every
request against the oracle on its own batch."""
import os
import time

import numpy as np
import pytest

import gen
import oracle
from helpers import compare_classify, oracle_params

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

THREADS = max(1, len(os.sched_getaffinity(0)))


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
def medium(mt):
    c = gen.config(2)
    t0 = time.time()
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"], threads=THREADS)
    print("medium workload and both indexes %.1fs" % (time.time() - t0))
    prm = dict(e_abs=c["e_abs"], e_permille=c["e_permille"], min_seeds=c["min_seeds"], top_n=3, max_occ=1024,
               cont_num=1, cont_den=10000, abund_cutoff=1e-4)
    return c, g, r, ix, oix, prm


def test_every_read_of_the_medium_workload(mt, medium):
    import torch
    c, g, r, ix, oix, prm = medium
    assert r.n == 10_000_000
    out = mt.classify(ix, torch.from_numpy(r.seq).cuda(), torch.from_numpy(r.offsets.astype(np.int64)).cuda(), **prm)
    t0 = time.time()
    ref = oracle.classify(oix, r.seq, r.offsets, oracle_params(prm), threads=THREADS)
    print("oracle, %d threads: %.1fs" % (THREADS, time.time() - t0))
    compare_classify(out, ref)


def test_serving_request_stream(mt, medium):
    import torch
    c, g, r, ix, oix, prm = medium
    c4 = gen.config(4)
    t_arr, sizes = gen.make_arrivals(c4, n_batches=40)
    free, _ = torch.cuda.mem_get_info()
    srv = mt.Server(ix, hbm_budget=free // 3, max_slots=4, **prm)
    rng = np.random.default_rng(404)
    batches, ids = [], []
    t0 = time.perf_counter()
    for ta, sz in zip(t_arr, sizes):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        sz = int(min(sz, r.n))
        a = int(rng.integers(0, r.n - sz + 1))
        b0, b1 = int(r.offsets[a]), int(r.offsets[a + sz])
        seq = r.seq[b0:b1]
        off = (r.offsets[a:a + sz + 1] - np.uint64(b0)).astype(np.uint64)
        batches.append((seq, off))
        ids.append(srv.submit(seq, off))
    outs = []
    for rid in ids:
        rc, lat, out = srv.poll(rid, 600_000)
        assert rc == mt.MT_OK
        outs.append(out)
    srv.close()
    assert sum(len(o) - 1 for _, o in batches) == int(sizes.clip(max=r.n).sum())
    for (seq, off), out in zip(batches, outs):
        compare_classify(out, oracle.classify(oix, seq, off, oracle_params(prm), threads=THREADS))
