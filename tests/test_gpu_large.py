"""GPU parity on the large workload's full reference: 2,000 genomes x 3 Mb (200 clades x 10 at
1-15% divergence, 6 Gb), k21 w11 canonical, with a 10^6-read batch drawn as the workload
describes (60% 150 bp / 40% 250 bp, log-normal(0, 2) abundances, 1% / 0.1% errors, 10% random,
E = 5% of n). Every per-read output and genome count bit-exact, abundances within 1e-6, for
the direct batched call (device buffers) and for a graph-replayed plan."""
import os

import numpy as np
import pytest

import gen
import oracle
from helpers import compare_classify, oracle_params

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_large_reference_batch_matches_oracle():
    import time

    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2311_02029_gb300 import _build
    _build.build()
    import paper_2311_02029_gb300 as mt
    threads = max(1, len(os.sched_getaffinity(0)))
    c = gen.config(5)
    t0 = time.time()
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g, n_reads=1_000_000)
    print("data %.1fs" % (time.time() - t0))
    t0 = time.time()
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    print("gpu index %.1fs %s" % (time.time() - t0, ix.info()))
    t0 = time.time()
    oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"], threads=threads)
    print("oracle index %.1fs" % (time.time() - t0))
    assert ix.info()["n_occ"] == oix.n_occ
    prm = dict(e_abs=c["e_abs"], e_permille=c["e_permille"], min_seeds=c["min_seeds"], top_n=3, max_occ=1024,
               cont_num=1, cont_den=10000, abund_cutoff=1e-4)
    t0 = time.time()
    ref = oracle.classify(oix, r.seq, r.offsets, oracle_params(prm), threads=threads)
    print("oracle classify %.1fs" % (time.time() - t0))
    d_reads = torch.from_numpy(r.seq).cuda()
    d_off = torch.from_numpy(r.offsets.astype(np.int64)).cuda()
    out = mt.classify(ix, d_reads, d_off, **prm)
    compare_classify(out, ref)
    plan = mt.Plan(ix, max_reads=r.n, max_bases=len(r.seq), max_read_len=250, **prm)
    for _ in range(3):                      # direct, capture, replay
        outp = plan.classify(d_reads, d_off)
    compare_classify(outp, ref)
    plan.close()
    src = r.truth_genome >= 0
    assert (ref["taxon"][src] == r.truth_genome[src]).mean() > 0.8
