"""GPU parity of one read batch against genome shards held by several ranks
(mt_classify_genome_sharded). The ranks are emulated by host threads on one GPU, each with
its own CUDA stream and its own shard index; exchanges (holders and hits summed, locations
gathered) run on the host, so threads only ever wait on the host, never in a kernel. Every
rank's outputs must equal the oracle's genome-sharded pipeline, and mt_classify over one
index of all genomes when no key reaches the repeat filter."""
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
    c = gen.config(2, n_genomes=24, genome_len=60_000, clade_size=4, n_reads=8_000, seed=91)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    return c, g, r


class HostExchange:
    """Host-side exchanges of `n` emulated ranks: element-wise sums and all-gathers in rank
    order. A rank whose exchange is made to fail breaks the barrier for the others."""

    def __init__(self, n, fail_rank=-1, timeout=120):
        self.n = n
        self.bufs = [None] * n
        self.bar = threading.Barrier(n, timeout=timeout)
        self.fail_rank = fail_rank

    def _swap(self, i, x):
        self.bufs[i] = x
        self.bar.wait()
        out = list(self.bufs)
        self.bar.wait()
        return out

    def allreduce(self, i):
        def fn(kind, arr):
            parts = self._swap(i, arr.copy())
            tot = parts[0].copy()
            for b in parts[1:]:
                tot = tot + b
            arr[...] = tot
        return fn

    def allgather(self, i):
        def fn(kind, send, recv):
            if i == self.fail_rank:
                self.bar.abort()
                raise RuntimeError("peer lost")
            parts = self._swap(i, send.copy())
            recv[...] = np.concatenate(parts) if len(send) else recv
        return fn


def _run(mt, g, c, parts, reads, offs, prm, fail_rank=-1, timeout=120):
    import torch
    n = len(parts)
    ex = HostExchange(n, fail_rank, timeout)
    shards = [mt.Index(*oracle.gather_genomes(g.seq, g.offsets, ids), c["k"], c["w"], c["canonical"]) for ids in parts]
    res, err = [None] * n, [None] * n

    def worker(i):
        try:
            s = torch.cuda.Stream()
            res[i] = mt.classify_genome_sharded(shards[i], parts[i], g.n, n, reads, offs, ex.allreduce(i),
                                                ex.allgather(i), stream=s.cuda_stream, **prm)
        except Exception as e:   # noqa: BLE001
            err[i] = e

    th = [threading.Thread(target=worker, args=(i,)) for i in range(n)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    return res, err


def _parts(G, n, seed):
    perm = np.random.default_rng(seed).permutation(G)
    return [np.sort(perm[i::n]).astype(np.uint32) for i in range(n)]


def _prm(c, **kw):
    prm = dict(e_abs=c["e_abs"], e_permille=0, min_seeds=3, top_n=3, max_occ=2048, cont_num=1, cont_den=10000)
    prm.update(kw)
    return prm


@pytest.mark.parametrize("n_ranks,cont_den", [(1, 10000), (3, 10000), (4, 2)])
def test_shards_equal_one_index_without_repeat_filter(mt, work, n_ranks, cont_den):
    c, g, r = work
    prm = _prm(c, cont_den=cont_den)
    res, err = _run(mt, g, c, _parts(g.n, n_ranks, n_ranks), r.seq, r.offsets, prm)
    assert err == [None] * n_ranks, err
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    one = mt.classify(ix, r.seq, r.offsets, **prm)
    full = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"], threads=8)
    ref = oracle.classify(full, r.seq, r.offsets, oracle_params(prm), threads=8)
    for out in res:
        compare_classify(out, ref)
        for k in ("taxon", "nloc", "genome_hits"):
            assert np.array_equal(out[k], one[k])
        assert np.array_equal(out["locs"], one["locs"])
    if cont_den == 2:   # the cutoff drops genomes: ranks map against part of their shards
        assert 0 < int(ref["keep"].sum()) < g.n


def test_shards_with_repeat_filter_match_oracle(mt, work):
    """max_occ 2: each rank filters by its own index, which one index would not; device reads."""
    import torch
    c, g, r = work
    prm = _prm(c, max_occ=2)
    parts = _parts(g.n, 4, 7)
    dev = torch.device("cuda:0")
    reads = torch.from_numpy(r.seq).to(dev)
    offs = torch.from_numpy(r.offsets.astype(np.int64)).to(dev)
    res, err = _run(mt, g, c, parts, reads, offs, prm)
    assert err == [None] * 4, err
    shards = [(oracle.Index(*oracle.gather_genomes(g.seq, g.offsets, ids), c["k"], c["w"], c["canonical"]), ids)
              for ids in parts]
    ref = oracle.classify_genome_sharded(shards, g.n, r.seq, r.offsets, oracle_params(prm), threads=8)
    for out in res:
        compare_classify(out, ref)
    one = oracle.classify(oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"]), r.seq, r.offsets,
                          oracle_params(prm), threads=8)
    assert not np.array_equal(one["genome_hits"], ref["genome_hits"])   # the filter did differ


def test_overlapping_shards_and_a_failed_exchange(mt, work):
    c, g, r = work
    parts = _parts(g.n, 3, 3)
    parts[1] = np.sort(np.concatenate([parts[1], parts[0][:1]])).astype(np.uint32)   # a genome held twice
    res, err = _run(mt, g, c, parts, r.seq, r.offsets, _prm(c))
    assert all(isinstance(e, mt.MtError) and e.status == mt.MT_EINVAL for e in err), err
    # ids not increasing: that rank refuses before its first exchange; the others' exchange
    # ends by its own time limit
    parts = _parts(g.n, 3, 3)
    parts[2] = parts[2][::-1].copy()
    _, err = _run(mt, g, c, parts, r.seq, r.offsets, _prm(c), timeout=5)
    assert isinstance(err[2], mt.MtError) and err[2].status == mt.MT_EINVAL
    assert all(isinstance(e, mt.MtError) and e.status == mt.MT_EXCHANGE for e in err[:2]), err
    res, err = _run(mt, g, c, _parts(g.n, 3, 3), r.seq, r.offsets, _prm(c), fail_rank=2)
    assert all(isinstance(e, mt.MtError) and e.status == mt.MT_EXCHANGE for e in err), err
