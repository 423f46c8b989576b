"""Multi-rank host logic of bench.py on CPU: two gloo ranks (world size 2, 127.0.0.1).

The path shards as independent batches, one per rank (replicas, weak scaling): no collective
sits on the data path. What runs across ranks is the timing contract: every rank reports its
own time, the job's time is the slowest rank's, and the job's throughput counts the units of
all ranks; only rank 0 prints, and the reference arm does no work on other ranks."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, local, w = bench.dist_env()
    my_ms = 10.0 + 5.0 * rank                   # rank 1 is the slow one
    ms = bench.max_over_ranks(my_ms, w, device="cpu")
    second = bench.max_over_ranks(100.0 - rank, w, device="cpu")   # a second reduction, same order
    rate = bench.job_rate(1000, w, ms)
    printed = None
    if rank != 0:
        # the reference arm returns at once on ranks other than 0 (no data, no output)
        import contextlib
        import io
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            bench.run_reference(type("A", (), dict(steps=1, warmup=3, ref_sample=10))())
        printed = buf.getvalue()
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump(dict(env=[r, local, w], ms=ms, second=second, rate=rate, printed=printed), f)


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    import torch.multiprocessing as tmp
    port = _free_port()
    tmp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    for r, x in enumerate(res):
        assert x["env"] == [r, r, 2]
        assert x["ms"] == 15.0                   # the slowest rank's time on every rank
        assert x["second"] == 100.0
        assert x["rate"] == pytest.approx(2 * 1000 / 0.015)
    assert res[1]["printed"] == ""


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_rate(10_000_000, 1, 31.6) == pytest.approx(1e7 / 0.0316)


def test_clock_samples_are_parsed_without_a_gpu(tmp_path):
    """The nvidia-smi sample parser: median SM clock, max clock, active throttle reasons."""
    sys.path.insert(0, ROOT)
    import bench
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1995, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbled line"]
    with open(c.path, "w") as f:
        f.write("\n".join(rows) + "\n")

    class Done:
        def terminate(self): pass
        def wait(self, timeout=None): return 0
    c.p = Done()
    c.f = open(os.devnull, "w")
    out = c.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]


def _xchg_main(rank, world, port, out_dir):
    """One rank of the sharded-batch exchange: the library's callback type wrapping the
    torch.distributed allreduce, called through its C function pointer as the library does."""
    import ctypes

    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import paper_2311_02029_gb300 as mt
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cb = mt.allreduce_callback(mt.dist_allreduce())
    fnptr = ctypes.cast(cb, ctypes.c_void_p).value
    call = mt.AllreduceFn(fnptr)
    hits = np.array([5, 0, 2 ** 40 + rank, 7 * rank], np.uint64)
    uniq = np.array([rank, 1, 0, 3], np.uint64)
    multi = np.array([0.25 * (rank + 1), 1e-17, 0.0, 2.5], np.float64)
    rcs = [call(None, mt.MT_XCHG_GENOME_HITS, hits.ctypes.data, len(hits)),
           call(None, mt.MT_XCHG_UNIQUE, uniq.ctypes.data, len(uniq)),
           call(None, mt.MT_XCHG_MULTI, multi.ctypes.data, len(multi))]
    empty = np.zeros(1, np.uint64)   # an index with no genomes still exchanges (count 0)
    rcs.append(call(None, mt.MT_XCHG_GENOME_HITS, empty.ctypes.data, 0))

    def broken(kind, arr):
        raise RuntimeError("peer lost")
    rcs.append(mt.allreduce_callback(broken)(None, mt.MT_XCHG_UNIQUE, uniq.ctypes.data, len(uniq)))
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "x%d.json" % rank), "w") as f:
        json.dump(dict(rcs=rcs, hits=[int(x) for x in hits], uniq=[int(x) for x in uniq],
                       multi=[float(x) for x in multi]), f)


def test_sharded_exchange_sums_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as tmp
    tmp.spawn(_xchg_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / ("x%d.json" % r))) for r in range(2)]
    for x in res:
        assert x["rcs"] == [0, 0, 0, 0, 1]
        assert x["hits"] == [10, 0, 2 ** 41 + 1, 7]
        assert x["uniq"] == [1, 2, 0, 6]
        assert x["multi"] == [0.75, 2e-17, 0.0, 5.0]


def _gather_main(rank, world, port, out_dir):
    """One rank of the genome-sharded exchange: the library's all-gather callback type wrapping
    torch.distributed, called through its C function pointer as the library does, with the
    holders sum that refuses overlapping shards."""
    import ctypes

    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import paper_2311_02029_gb300 as mt
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cb = mt.allgather_callback(mt.dist_allgather(), world)
    call = mt.AllgatherFn(ctypes.cast(cb, ctypes.c_void_p).value)
    locs = np.zeros(4, mt.LOC_DTYPE)          # this rank's per-read locations, 24 bytes each
    locs["genome"] = np.arange(4) + 100 * rank
    locs["wstart"] = -(rank + 1)
    locs["dist"] = rank + 3
    recv = np.zeros(4 * world, mt.LOC_DTYPE)
    rcs = [call(None, mt.MT_XCHG_LOCATIONS, locs.ctypes.data, locs.nbytes, recv.ctypes.data)]
    nothing = np.zeros(1, np.uint8)            # a batch with no reads still exchanges (0 bytes)
    rcs.append(call(None, mt.MT_XCHG_LOCATIONS, nothing.ctypes.data, 0, nothing.ctypes.data))
    hold = np.array([1, 0, 1, 0], np.uint64) if rank == 0 else np.array([0, 1, 1, 0], np.uint64)
    ar = mt.AllreduceFn(ctypes.cast(mt.allreduce_callback(mt.dist_allreduce()), ctypes.c_void_p).value)
    rcs.append(ar(None, mt.MT_XCHG_HOLDERS, hold.ctypes.data, len(hold)))

    def broken(kind, send, recv):
        raise RuntimeError("peer lost")
    rcs.append(mt.allgather_callback(broken, world)(None, mt.MT_XCHG_LOCATIONS, locs.ctypes.data, locs.nbytes,
                                                     recv.ctypes.data))
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "g%d.json" % rank), "w") as f:
        json.dump(dict(rcs=rcs, genome=recv["genome"].tolist(), wstart=recv["wstart"].tolist(),
                       dist=recv["dist"].tolist(), hold=[int(x) for x in hold]), f)


def test_genome_sharded_exchanges_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as tmp
    tmp.spawn(_gather_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / ("g%d.json" % r))) for r in range(2)]
    for x in res:
        assert x["rcs"] == [0, 0, 0, 1]
        assert x["genome"] == [0, 1, 2, 3, 100, 101, 102, 103]      # rank order
        assert x["wstart"] == [-1] * 4 + [-2] * 4
        assert x["dist"] == [3] * 4 + [4] * 4
        assert x["hold"] == [1, 1, 2, 0]                              # genome 2 held twice: refused


def test_seeding_counters_are_dropped_when_the_kernel_sources_change(monkeypatch):
    """The stored ncu counters of the seeding kernel (traffic and instructions per read) are
    reported only while the kernel's sources hash to the value stored with them."""
    sys.path.insert(0, ROOT)
    import bench
    good = dict(bench.SEED_PROFILE)
    monkeypatch.setattr(bench, "SEED_PROFILE", dict(good, source_sha256=bench.seed_source_sha256()))
    traffic, inst = bench.seed_profile()
    assert traffic == good["dram_bytes_per_read"] and inst == good["warp_inst_per_read"]
    monkeypatch.setattr(bench, "SEED_PROFILE", dict(good, source_sha256="0" * 64))
    assert bench.seed_profile() == (None, None)
