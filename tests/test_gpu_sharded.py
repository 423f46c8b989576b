"""GPU parity of one batch sharded over ranks (mt_classify_sharded). The ranks are emulated by
host threads on one GPU, each with its own CUDA stream, whose exchanges are summed on the host
(the threads wait on the host only, never in a kernel). Every shard's per-read outputs must
equal those of the unsharded call for the same reads, and genome hits and abundances must be
the whole batch's. The shards hold reads of different genomes, so a shard-local containment
cutoff, multi-read split or profile would give other answers; the test checks that the
shard-local counts and profiles do differ."""
import threading

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
    c = gen.config(2, n_genomes=20, genome_len=100_000, n_reads=24_000)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    # a cutoff that bites: genomes below a tenth of the top hit count are masked
    prm = dict(e_abs=c["e_abs"], e_permille=0, min_seeds=3, top_n=3, max_occ=1024, cont_num=1, cont_den=10)
    return c, g, r, ix, prm


class HostAllreduce:
    """Sums each exchange over `n` threads: every thread deposits its vector, all wait, each
    takes the sum (in shard order, so every thread gets the same doubles)."""

    def __init__(self, n):
        self.n = n
        self.bufs = [None] * n
        self.bar = threading.Barrier(n, timeout=120)
        self.kinds = [[] for _ in range(n)]

    def for_rank(self, i):
        def fn(kind, arr):
            self.kinds[i].append(kind)
            self.bufs[i] = arr.copy()
            self.bar.wait()
            tot = self.bufs[0].copy()
            for b in self.bufs[1:]:
                tot = tot + b
            self.bar.wait()
            arr[...] = tot
        return fn


def _subset(r, idx):
    return gen.subsample_reads(r, np.asarray(idx, dtype=np.int64))


def _run_shards(mt, ix, shards, prm):
    import torch
    n = len(shards)
    ar = HostAllreduce(n)
    res, err = [None] * n, [None] * n

    def worker(i):
        try:
            s = torch.cuda.Stream()
            res[i] = mt.classify_sharded(ix, shards[i].seq, shards[i].offsets, ar.for_rank(i),
                                         stream=s.cuda_stream, **prm)
        except Exception as e:   # noqa: BLE001
            err[i] = e
            ar.bar.abort()

    th = [threading.Thread(target=worker, args=(i,)) for i in range(n)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert all(e is None for e in err), err
    assert all(k == [mt.MT_XCHG_GENOME_HITS, mt.MT_XCHG_UNIQUE, mt.MT_XCHG_MULTI] for k in ar.kinds)
    return res


def _same_reads(out, ref, idx):
    assert np.array_equal(out["taxon"], ref["taxon"][idx])
    assert np.array_equal(out["nloc"], ref["nloc"][idx])
    for f in ("genome", "seeds", "strand", "dist", "wstart"):
        assert np.array_equal(out["locs"][f], ref["locs"][f][idx])


@pytest.mark.parametrize("layout", ["two", "three_one_empty"])
def test_sharded_batch_equals_whole_batch(mt, work, layout):
    c, g, r, ix, prm = work
    tg = r.truth_genome
    if layout == "two":       # shard 0: reads of genomes 0-5 and random reads; shard 1: the rest
        parts = [np.flatnonzero(tg < 6), np.flatnonzero(tg >= 6)]
    else:
        parts = [np.flatnonzero(tg < 3), np.array([], np.int64), np.flatnonzero(tg >= 3)]
    order = np.concatenate(parts)
    whole = _subset(r, order)
    ref = mt.classify(ix, whole.seq, whole.offsets, **prm)
    shards = [_subset(r, p) for p in parts]
    outs = _run_shards(mt, ix, shards, prm)
    start = 0
    for p, out in zip(parts, outs):
        idx = np.arange(start, start + len(p))
        start += len(p)
        _same_reads(out, ref, idx)
        assert np.array_equal(out["genome_hits"], ref["genome_hits"])
        assert np.abs(out["abundance"] - ref["abundance"]).max() <= 1e-12
    # the whole batch is also the oracle's
    merged = dict(taxon=np.concatenate([o["taxon"] for o in outs]), nloc=np.concatenate([o["nloc"] for o in outs]),
                  locs=np.concatenate([o["locs"] for o in outs]), genome_hits=outs[0]["genome_hits"],
                  abundance=outs[0]["abundance"])
    oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    compare_classify(merged, oracle.classify(oix, whole.seq, whole.offsets, oracle_params(prm), threads=8))
    # and shard-local stages would not have given it
    alone = [mt.classify(ix, sh.seq, sh.offsets, **prm) for sh in shards if sh.n]
    assert all(not np.array_equal(a["genome_hits"], ref["genome_hits"]) for a in alone)
    assert all(np.abs(a["abundance"] - ref["abundance"]).max() > 1e-3 for a in alone)


def test_failed_exchange_stops_the_call(mt, work):
    c, g, r, ix, prm = work
    sh = _subset(r, np.arange(100))

    def bad(kind, arr):
        raise RuntimeError("peer lost")

    with pytest.raises(mt.MtError) as e:
        mt.classify_sharded(ix, sh.seq, sh.offsets, bad, **prm)
    assert e.value.status == mt.MT_EXCHANGE
