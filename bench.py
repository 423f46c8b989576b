#!/usr/bin/env python
"""Benchmark of the GB300 MetaTrinity hot path; prints ONE JSON line on rank 0.

A step is one mt_classify call over one batch of the medium workload (200 genomes x 2 Mb in
20 clades x 10 at 1-10% divergence, k21 w11 canonical, 10^7 reads of 150 bp, E = 8): packing,
minimizers, index lookups, containment counts, locations, SneakySnake on every candidate and
the abundance profile. Inputs are resident in HBM when the timed region starts (1.5 GB of
reads, larger than L2). `value` is reads/s of the batched form; the plain form, the
end-to-end form with host buffers, the edit-distance stage alone on the batching workload
(read-versus-window pairs), the serving workload (2,000 Poisson-arriving batches) and the
large workload (6 Gb reference, a 10^7-read sub-batch) are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402

METRIC = "reads/s and candidate pairs/s at 1 GB300 (batched vs plain, bit-exact); p50/p99"
# Counters of the seeding kernel (k_seed) from one ncu capture of the bench command, per read:
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) and warp instructions
# (smsp__inst_executed.sum). They hold only for the kernel source they were taken on: its
# files' SHA-256 is stored beside them, and the bench reports null for both whenever the
# current source differs (the kernel changed since the capture).
SEED_PROFILE = {"source_sha256": "409357c70a3ab6c9e5f48d8c1503dd4ede4b748268e137857c729d67da4570bc",
                "dram_bytes_per_read": (35609344512 + 1294191616) / 1e7,
                "warp_inst_per_read": 13003210652 / 1e7,
                "capture": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,smsp__inst_executed.sum,"
                           "gpu__time_duration.sum --clock-control none -k regex:k_seed -s 4 -c 1 (1 pass) on "
                           "python bench.py --steps 3 --warmup 3 --eda-pairs 0 --serve-seconds 0 --cpu-sample 0 "
                           "--part-batches 0 --large-reads 0 (the medium workload, 10^7 reads)"}
SEED_SOURCES = ("paper_2311_02029_gb300/csrc/classify.cu", "paper_2311_02029_gb300/csrc/common.cuh",
                "paper_2311_02029_gb300/csrc/internal.h", "include/mt.h")


def seed_source_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in SEED_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def seed_profile():
    """(dram bytes per read, warp instructions per read) of the committed capture, or
    (None, None) when the seeding kernel's sources have changed since it was taken."""
    if SEED_PROFILE["source_sha256"] != seed_source_sha256():
        return None, None
    return SEED_PROFILE["dram_bytes_per_read"], SEED_PROFILE["warp_inst_per_read"]


def workload_name(c: dict) -> str:
    """The medium workload's description for its actual genome and read counts."""
    return ("medium: %d genomes x 2 Mb (%d clades x 10, 1-10%% divergence), k21 w11 canonical, "
            "%.3g reads x 150 bp (both strands, 0.5%% subst + 0.05%% indel, 5%% random), E=8, min_seeds 3, top 3"
            % (c["n_genomes"], c["n_genomes"] // 10, c["n_reads"]))




def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest x over all ranks (for times: the slowest rank); x itself on one rank.
    Every rank must call it, in the same order."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank / (ms_max / 1000.0)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region (SM clock, max clock, throttle reasons)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.p = None
        # the raw samples, summarised into the JSON line (MT_CLOCKS_DIR keeps them elsewhere)
        self.path = os.path.join(os.environ.get("MT_CLOCKS_DIR", tempfile.gettempdir()),
                                 "mt_bench_clocks_%d_%d.csv" % (gpu, os.getpid()))

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def params(c, mode):
    return dict(e_abs=c["e_abs"], e_permille=c["e_permille"], min_seeds=c["min_seeds"], top_n=3, max_occ=1024,
                cont_num=1, cont_den=10000, abund_cutoff=1e-4, eda_mode=mode)


# ---------------------------------------------------------------------------------------------
# reference arm: the oracle, timed on host cores
# ---------------------------------------------------------------------------------------------
def run_reference(args):
    import oracle
    rank, _, world = dist_env()
    if rank != 0:
        return
    c = gen.config(2)
    t0 = time.time()
    g = gen.make_genomes(c)
    reads = gen.make_reads(c, g)
    log("[ref] data %.1fs" % (time.time() - t0))
    t0 = time.time()
    oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    log("[ref] oracle index %.1fs" % (time.time() - t0))
    p = oracle.params(**{k: v for k, v in params(c, 0).items() if k != "eda_mode"})
    S = args.ref_sample
    rng = np.random.default_rng(1234)
    times = []
    for step in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(reads.n, S, replace=False))
        sub = gen.subsample_reads(reads, idx)
        t = time.perf_counter()
        oracle.classify(oix, sub.seq, sub.offsets, p, threads=1)
        dt = time.perf_counter() - t
        if step >= args.warmup:
            times.append(dt)
    ms = 1000.0 * statistics.mean(times)
    v = S / (ms / 1000.0)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "reads/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": workload_name(c), "reads": c["n_reads"], "genomes": c["n_genomes"]},
            "cpu_baseline": {"value": v, "unit": "reads/s", "cores": 1, "kind": "oracle",
                             "sample": "%d random reads of the workload per step (containment over the sample)" % S},
            "e2e": {"value": v, "unit": "reads/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------------
def gather_ceiling(torch, n_idx=1 << 26, table_gib=4, reps=5):
    """Random-access ceiling of this GPU: 8-byte words gathered at uniformly random indices
    from a table far larger than L2 by the library gather (torch.index_select). The index
    reads and output writes are streaming and inside the timed region, so the rate is a
    slight underestimate. Returns G gathers/s."""
    table = torch.ones(table_gib << 27, dtype=torch.int64, device="cuda")
    gen_ = torch.Generator(device="cuda")
    gen_.manual_seed(99)
    idx = torch.randint(0, table.numel(), (n_idx,), device="cuda", generator=gen_)
    out = torch.empty(n_idx, dtype=torch.int64, device="cuda")
    for _ in range(2):
        torch.index_select(table, 0, idx, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        torch.index_select(table, 0, idx, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    del table, idx, out
    torch.cuda.empty_cache()
    return n_idx / (ms / 1000.0) / 1e9


def timed_steps(fn, steps, warmup, stream, torch):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    outs = []
    e0.record(stream)
    for _ in range(steps):
        outs.append(fn())
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, outs


def large_workload(mt, torch, n_reads, steps, warmup, hbm):
    """The large workload: 2,000 genomes x 3 Mb (6 Gb, one resident index) and a sub-batch of
    n_reads reads (60% 150 bp, 40% 250 bp, E = 5% of n), batched form, inputs in HBM."""
    c = gen.config(5)
    t0 = time.time()
    g = gen.make_genomes(c)
    reads = gen.make_reads(c, g, n_reads=n_reads)
    t_data = time.time() - t0
    t0 = time.time()
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    t_index = time.time() - t0
    info = ix.info()
    d_reads = torch.from_numpy(reads.seq).cuda()
    d_off = torch.from_numpy(reads.offsets.astype(np.int64)).cuda()
    stream = torch.cuda.current_stream()
    eda_shape = mt.classify_autotune(ix, d_reads, d_off, **params(c, mt.MT_EDA_BATCHED))["eda_shape"]
    ms, outs = timed_steps(lambda: mt.classify(ix, d_reads, d_off, **params(c, mt.MT_EDA_BATCHED)),
                           steps, warmup, stream, torch)
    st = {k: statistics.mean(o["stats"][k] for o in outs) for k in outs[0]["stats"]}
    n_bases = int(reads.offsets[-1])
    # the same batch through a preallocated plan replayed from its captured CUDA graph
    plan = mt.Plan(ix, max_reads=reads.n, max_bases=n_bases, max_read_len=int(reads.lengths.max()),
                   **params(c, mt.MT_EDA_BATCHED))
    ms_graph, gouts = timed_steps(lambda: plan.classify(d_reads, d_off), steps, warmup, stream, torch)
    graph_identical = (torch.equal(outs[-1]["taxon"], gouts[-1]["taxon"])
                       and torch.equal(outs[-1]["locs"], gouts[-1]["locs"])
                       and torch.equal(outs[-1]["genome_hits"], gouts[-1]["genome_hits"])
                       and bool((outs[-1]["abundance"] - gouts[-1]["abundance"]).abs().max().item() <= 1e-6))
    plan.close()
    del gouts
    seed_bytes = (n_bases + 2 * (n_bases / 32.0 + reads.n) * 8 + st["n_minimizers"] * (32 + 32)
                  + st["n_hits"] * 16 * 2)
    achieved = seed_bytes / (st["ms_seed"] / 1000.0) / 1e9
    out = {"workload": "large: 2000 genomes x 3 Mb (200 clades x 10, 1-15%% divergence, 6 Gb), k21 w11 canonical, "
                       "%d reads (60%% 150 bp, 40%% 250 bp), E = 5%% of n, min_seeds 3, top 3" % reads.n,
           "reads_per_s": reads.n / (ms / 1000.0), "ms_per_step": ms,
           "pairs_per_s": st["n_candidates"] / (ms / 1000.0),
           "graph": {"reads_per_s": reads.n / (ms_graph / 1000.0), "ms_per_step": ms_graph,
                     "identical": graph_identical,
                     "form": "batched persistent path, preallocated plan replayed from its captured CUDA graph"},
           "stage_ms": {k[3:]: st[k] for k in ("ms_seed", "ms_select", "ms_eda", "ms_profile", "ms_total")},
           "seed_roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                             "algorithmic_bytes_per_launch": seed_bytes},
           "classified_frac": float((outs[-1]["taxon"] >= 0).float().mean().item()),
           "eda_shape": eda_shape,
           "index": {"build_s": t_index, **info}, "data_s": t_data, "steps": steps, "warmup": warmup}
    del outs, d_reads, d_off
    ix.close()
    torch.cuda.empty_cache()
    return out


# the paper's other approximations (Table 1), measured beside SneakySnake
EDA_OTHERS = (("hamming", 0x10), ("base_counting", 0x20), ("qgram", 0x30), ("shd", 0x40))


def eda_stage(mt, torch, n_pairs, steps, warmup):
    c3 = gen.config(3)
    t0 = time.time()
    pairs = gen.make_eda_pairs(c3, n_pairs=n_pairs)
    log("[eda] %d pairs generated in %.1fs" % (pairs.n_pairs, time.time() - t0))
    dev = "cuda"
    rs = torch.from_numpy(pairs.read_seq).to(dev)
    ro = torch.from_numpy(pairs.read_off.astype(np.int64)).to(dev)
    rw = mt.pack_seqs(rs, ro, mt.packed_words(pairs.read_off))
    del rs
    ws = torch.from_numpy(pairs.win_seq).to(dev)
    wo = torch.from_numpy(pairs.win_off.astype(np.int64)).to(dev)
    ww = mt.pack_seqs(ws, wo, mt.packed_words(pairs.win_off))
    del ws
    pr = torch.from_numpy(pairs.pair_read.astype(np.int32)).to(dev)
    E = torch.from_numpy(pairs.E.astype(np.int16)).to(dev)
    stream = torch.cuda.current_stream()
    res = {}
    outs = {}
    _, shapes = mt.eda_batch_autotune(rw, ro, ww, wo, pr, E)
    for name, mode in (("batched", mt.MT_EDA_BATCHED), ("plain", mt.MT_EDA_PLAIN)):
        ms, o = timed_steps(lambda: mt.eda_batch(rw, ro, ww, wo, pr, E, mode=mode), steps, warmup, stream, torch)
        res[name] = pairs.n_pairs / (ms / 1000.0)
        res["ms_" + name] = ms
        outs[name] = o[-1]
    same = bool(torch.equal(outs["batched"], outs["plain"]))
    accepted = float((outs["batched"].cpu().numpy() <= pairs.E).mean())
    window_bytes = int(pairs.win_off[-1])
    # the other approximations on the same pairs, batched form
    others = {}
    for name, bits in EDA_OTHERS:
        mt.eda_batch_autotune(rw, ro, ww, wo, pr, E, mode=bits | mt.MT_EDA_BATCHED)
        ms, o = timed_steps(lambda: mt.eda_batch(rw, ro, ww, wo, pr, E, mode=bits | mt.MT_EDA_BATCHED), steps,
                            warmup, stream, torch)
        others[name] = {"pairs_per_s": pairs.n_pairs / (ms / 1000.0), "ms": ms,
                        "accepted_frac": float((o[-1].cpu().numpy() <= pairs.E).mean())}
    return {"workload": "batching: %d read-vs-window pairs, n~U[100,250], E in {2,4,6,10}%% of n, "
                        "geometric(6) candidates per read, %d reads" % (pairs.n_pairs, pairs.n_reads),
            "pairs_per_s_batched": res["batched"], "pairs_per_s_plain": res["plain"],
            "ms_batched": res["ms_batched"], "ms_plain": res["ms_plain"],
            "batched_over_plain": res["batched"] / res["plain"], "identical": same,
            "shapes_by_class": {"E %s" % rng: sh for rng, sh in zip(
                ("0-1", "2-3", "4-7", "8-15", "16-31", "32-63", "64-127", "128+"), shapes) if sh["lanes_per_pair"]},
            "accepted_frac": accepted, "window_bases": window_bytes, "other_approximations": others}


def serving_sample(mt, ix, reads, c, seconds, torch, pinned_seq=None):
    """Poisson arrivals at 20 batches/s, log-uniform 1k-1M reads per batch drawn from the
    medium workload's reads; p50/p99 of submit-to-result latency. pinned_seq: the reads' bytes
    in pinned host memory (the client's staging area); outputs then go to pinned arrays too."""
    c4 = gen.config(4)
    n_batches = max(1, int(seconds * c4["rate"]))
    t_arr, sizes = gen.make_arrivals(c4, n_batches=n_batches)
    free, total = torch.cuda.mem_get_info()
    budget = int(free * 0.5)
    srv = mt.Server(ix, budget, max_slots=4, **params(c, mt.MT_EDA_BATCHED))
    rng = np.random.default_rng(99)
    ids = []
    lat = []
    done_reads = 0
    pending = {}
    lock = threading.Lock()
    stop = [False]
    # output arrays for the largest batch, reused across requests (a client keeps its result
    # buffers; fresh arrays would fault in new pages for every request)
    top_n, G = 3, ix.n_genomes
    cap = int(min(c4["batch_max"], reads.n))
    free_outs = []

    def arr(shape, dtype):
        if pinned_seq is None:
            return np.zeros(shape, dtype)
        nb = int(np.prod(shape)) * np.dtype(dtype).itemsize
        return torch.empty(nb, dtype=torch.uint8).pin_memory().numpy().view(dtype).reshape(shape)

    def new_out():   # a request's buffers: its rebased offsets and its outputs
        return dict(off=arr((cap + 1,), np.uint64), taxon=arr((cap,), np.int32), nloc=arr((cap,), np.uint8),
                    locs=arr((cap, top_n), mt.LOC_DTYPE), genome_hits=arr((G,), np.uint64),
                    abundance=arr((G,), np.float64))
    src = reads.seq if pinned_seq is None else pinned_seq
    owner = {}

    def poller():
        nonlocal done_reads
        while True:
            with lock:
                items = list(pending.items())
            if not items and stop[0]:
                return
            for rid, n in items:
                rc, l, out = srv.poll(rid, 0)
                if rc in (mt.MT_EBUSY, mt.MT_ETIMEDOUT):
                    continue
                with lock:
                    del pending[rid]
                    free_outs.append(owner.pop(rid))
                if rc == mt.MT_OK:
                    lat.append(l)
                    done_reads += n
            time.sleep(0.0005)

    th = threading.Thread(target=poller)
    th.start()
    t0 = time.perf_counter()
    for ta, sz in zip(t_arr, sizes):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        sz = int(min(sz, reads.n))
        a = int(rng.integers(0, reads.n - sz + 1))
        b0, b1 = int(reads.offsets[a]), int(reads.offsets[a + sz])
        with lock:
            buf = free_outs.pop() if free_outs else new_out()
        off = buf["off"][:sz + 1]
        np.subtract(reads.offsets[a:a + sz + 1], np.uint64(b0), out=off, dtype=np.uint64)
        rid = srv.submit(src[b0:b1], off, out=buf)
        with lock:
            owner[rid] = buf
            pending[rid] = sz
        ids.append(rid)
    stop[0] = True
    th.join()
    wall = time.perf_counter() - t0
    srv.close()
    lat_ms = np.array(lat) * 1000.0
    return {"workload": "serving: medium-workload index resident; Poisson 20 batches/s, "
                        "log-uniform 1k-1M reads per batch; %d batches (%.0f s of arrivals); %s host buffers"
                        % (n_batches, t_arr[-1], "pageable" if pinned_seq is None else "pinned"),
            "reads_per_s": done_reads / wall, "p50_ms": float(np.percentile(lat_ms, 50)) if len(lat_ms) else None,
            "p99_ms": float(np.percentile(lat_ms, 99)) if len(lat_ms) else None, "completed": len(lat_ms),
            "offered_reads_per_s": float(sizes.sum() / max(t_arr[-1], 1e-9)), "hbm_budget_bytes": budget,
            "slots": 4}


def run_ours(args):
    import torch

    import paper_2311_02029_gb300 as mt
    from paper_2311_02029_gb300 import _build
    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    _build.build()
    mt.lib()

    c = gen.config(2, n_reads=args.reads, n_genomes=args.genomes)
    t0 = time.time()
    g = gen.make_genomes(c)
    reads = gen.make_reads(c, g, seed=c["seed"] + rank)
    log("[ours] data %.1fs" % (time.time() - t0))
    stream = torch.cuda.current_stream()
    t0 = time.time()
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    index_s = time.time() - t0
    info = ix.info()
    log("[ours] index %.1fs %s" % (index_s, info))

    d_reads = torch.from_numpy(reads.seq).cuda()
    d_off = torch.from_numpy(reads.offsets.astype(np.int64)).cuda()
    n_reads, n_bases = reads.n, int(reads.offsets[-1])

    def step(mode):
        return lambda: mt.classify(ix, d_reads, d_off, **params(c, mode))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # the approximation kernel's shape for this workload, timed once on the batch itself
    # (mt_classify never times anything on its own)
    if args.tune:
        eda_shape = mt.classify_autotune(ix, d_reads, d_off, **params(c, mt.MT_EDA_BATCHED))["eda_shape"]
    else:
        eda_shape = mt.eda_shape_for(mt.MT_EDA_BATCHED, True, c["e_abs"])
    # batched form (the headline); clocks sampled during its timed region
    for _ in range(args.warmup):
        step(mt.MT_EDA_BATCHED)()
    barrier()
    clk = Clocks(local)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    e0.record(stream)
    for _ in range(args.steps):
        out = step(mt.MT_EDA_BATCHED)()
        stats.append(out["stats"])
    e1.record(stream)
    barrier()
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    value = job_rate(n_reads, world, ms)
    batched_out = out

    # plain form on the same inputs: identical outputs required
    ms_plain, outs = timed_steps(step(mt.MT_EDA_PLAIN), args.steps, 1, stream, torch)
    ms_plain = max_over_ranks(ms_plain, world)
    plain_out = outs[-1]
    identical = (torch.equal(batched_out["taxon"], plain_out["taxon"])
                 and torch.equal(batched_out["locs"], plain_out["locs"])
                 and torch.equal(batched_out["genome_hits"], plain_out["genome_hits"])
                 and bool((batched_out["abundance"] - plain_out["abundance"]).abs().max().item() <= 1e-6))

    # batched form replayed from a captured CUDA graph (preallocated plan)
    plan = mt.Plan(ix, max_reads=n_reads, max_bases=n_bases, max_read_len=int(reads.lengths.max()),
                   **params(c, mt.MT_EDA_BATCHED))
    ms_graph, gouts = timed_steps(lambda: plan.classify(d_reads, d_off), args.steps, 3, stream, torch)
    ms_graph = max_over_ranks(ms_graph, world)
    graph_out = gouts[-1]
    graph_identical = (torch.equal(batched_out["taxon"], graph_out["taxon"])
                       and torch.equal(batched_out["locs"], graph_out["locs"])
                       and torch.equal(batched_out["genome_hits"], graph_out["genome_hits"])
                       and bool((batched_out["abundance"] - graph_out["abundance"]).abs().max().item() <= 1e-6))
    del gouts, graph_out

    # end to end: pinned host buffers, copies inside the timed region
    h_reads = torch.from_numpy(reads.seq).pin_memory()
    h_off = torch.from_numpy(reads.offsets.astype(np.int64)).pin_memory()
    top_n = 3
    G = g.n
    def pinned(shape, dtype):
        return torch.empty(int(np.prod(shape)) * np.dtype(dtype).itemsize, dtype=torch.uint8).pin_memory() \
            .numpy().view(dtype).reshape(shape)
    h_out = dict(taxon=pinned((n_reads,), np.int32), nloc=pinned((n_reads,), np.uint8),
                 locs=pinned((n_reads, top_n), mt.LOC_DTYPE), genome_hits=pinned((G,), np.uint64),
                 abundance=pinned((G,), np.float64))
    # the classification's result (the problem statement's per-read taxon and abundance vector,
    # with each read's location count and the per-genome hits); the per-read locations are an
    # extra 72 bytes a read, measured beside it
    h_res = dict(h_out, locs=None)
    e2e_ms, _ = timed_steps(lambda: mt.classify(ix, h_reads.numpy(), h_off.numpy().view(np.uint64),
                                                out=h_res, **params(c, mt.MT_EDA_BATCHED)),
                            max(1, args.steps // 2), 1, stream, torch)
    e2e_locs_ms, _ = timed_steps(lambda: mt.classify(ix, h_reads.numpy(), h_off.numpy().view(np.uint64),
                                                     out=h_out, **params(c, mt.MT_EDA_BATCHED)),
                                 max(1, args.steps // 2), 1, stream, torch)
    e2e_graph_ms, _ = timed_steps(lambda: plan.classify(h_reads.numpy(), h_off.numpy().view(np.uint64), out=h_out),
                                  max(1, args.steps // 2), 1, stream, torch)
    plan.close()
    e2e_ms = max_over_ranks(e2e_ms, world)
    e2e_locs_ms = max_over_ranks(e2e_locs_ms, world)
    e2e_graph_ms = max_over_ranks(e2e_graph_ms, world)
    h2d = n_bases + (n_reads + 1) * 8
    d2h = n_reads * (4 + 1) + G * 16
    d2h_locs = d2h + n_reads * 24 * top_n

    # whole classification with each other approximation (batched form, same inputs)
    approx = {}
    if rank == 0 and world == 1:
        for name, bits in EDA_OTHERS:
            prm = dict(params(c, mt.MT_EDA_BATCHED), eda_mode=bits | mt.MT_EDA_BATCHED)
            mt.classify_autotune(ix, d_reads, d_off, **prm)
            fn = lambda: mt.classify(ix, d_reads, d_off, **prm)  # noqa: E731
            ms_a, o = timed_steps(fn, max(1, args.steps // 2), 1, stream, torch)
            sa = o[-1]["stats"]
            approx[name] = {"reads_per_s": n_reads / (ms_a / 1000.0), "ms_per_step": ms_a, "ms_eda": sa["ms_eda"],
                            "classified_frac": float((o[-1]["taxon"] >= 0).float().mean().item())}
            del o

    # containment alone (stage 1), with this index and with the paper's containment seeds
    # (homopolymer-compressed genomes, k = 28, w = 18)
    contain = {}
    if rank == 0 and world == 1:
        hix = mt.Index(g.seq, g.offsets, 28, 18, 1, hpc=True)
        for name, cix in (("mapping_index_k21_w11", ix), ("hpc_index_k28_w18", hix)):
            fn = lambda: mt.containment(cix, d_reads, d_off, cont_den=10000)  # noqa: E731
            ms_c, _ = timed_steps(fn, max(1, args.steps // 2), 1, stream, torch)
            contain[name] = {"reads_per_s": n_reads / (ms_c / 1000.0), "ms_per_step": ms_c,
                             "index_bytes": cix.info()["device_bytes"]}
        hix.close()

    # a database cut into batches (the paper's 25): per batch a compressed k28 w18 containment
    # index; the cutoff over the database; the subset index (k21 w11) of the kept genomes built
    # per query; mapping against it. Every call synchronises, so host timers bracket the stages.
    part = {}
    if rank == 0 and world == 1 and args.part_batches > 0:
        t0 = time.time()
        pids = mt.split_batches(g.offsets, args.part_batches)
        pbs = [mt.Index.subset(g.seq, g.offsets, ids, 28, 18, 1, hpc=True) for ids in pids]
        pbuild = time.time() - t0
        prm = params(c, mt.MT_EDA_BATCHED)

        def part_step(one_pass=True):
            t = [time.perf_counter()]
            q = mt.PartitionedQuery(g.n, d_reads, d_off)
            if one_pass:    # each read's minimizers found once, looked up in every batch
                q.contain_batches(pbs, pids, max_occ=prm["max_occ"])
            else:
                for bix, ids in zip(pbs, pids):
                    q.contain(bix, ids, max_occ=prm["max_occ"])
            t.append(time.perf_counter())
            kept = q.subset(prm["cont_num"], prm["cont_den"])["kept"]
            six = mt.Index.subset(g.seq, g.offsets, kept, c["k"], c["w"], c["canonical"])
            t.append(time.perf_counter())
            o = q.classify(six, **prm)
            t.append(time.perf_counter())
            six.close()
            q.close()
            return np.diff(t) * 1000.0, o, len(kept)

        part_step()
        runs = [part_step() for _ in range(max(2, args.steps // 3))]
        ms_stage = np.mean([r[0] for r in runs], axis=0)
        ms_part = float(ms_stage.sum())
        per_batch = [part_step(False) for _ in range(2)]
        same = all(torch.equal(p[1]["taxon"], runs[-1][1]["taxon"]) and torch.equal(p[1]["locs"], runs[-1][1]["locs"])
                   for p in per_batch)
        ms_per_batch = float(np.mean([p[0][0] for p in per_batch]))
        part = {"workload": "medium reads against the medium reference cut into %d batches of consecutive genomes "
                            "(compressed k28 w18 containment index per batch, subset index k21 w11)" % len(pids),
                "reads_per_s": n_reads / (ms_part / 1000.0), "ms_per_step": ms_part,
                "ms_containment_all_batches": float(ms_stage[0]), "ms_cutoff_and_subset_index": float(ms_stage[1]),
                "ms_mapping": float(ms_stage[2]), "n_batches": len(pids), "n_kept": runs[-1][2],
                "ms_containment_one_pass_per_batch": ms_per_batch, "one_pass_identical": same,
                "batch_index_bytes": int(sum(b.info()["device_bytes"] for b in pbs)), "batch_build_s": pbuild,
                "classified_frac": float((runs[-1][1]["taxon"] >= 0).float().mean().item())}
        for b in pbs:
            b.close()
        del runs, per_batch
        log("[ours] partitioned %.1fs" % (time.time() - t0))

    # roofline of the dominant kernel (the seeding pass). Algorithmic bytes per launch, as the
    # seeding stage's per-read figure counts them (stage by stage through HBM): read bytes in,
    # packed reads written and read back, one 32-byte slot sector and one 32-byte occurrence
    # sector per lookup, every seed match written and read back as 16 bytes
    st = {k: statistics.mean(s[k] for s in stats) for k in stats[0]}
    seed_bytes = (n_bases
                  + 2 * (n_bases / 32.0 + n_reads) * 8
                  + st["n_minimizers"] * (32 + 32)
                  + st["n_hits"] * 16 * 2)
    # the bytes this fused kernel cannot avoid: matches stay in shared memory and up to three
    # occurrences sit in the slot itself
    design_bytes = (n_bases                          # read bytes in
                    + (n_bases / 32.0 + n_reads) * 8  # packed reads out
                    + st["n_minimizers"] * 32         # one 32-byte slot per lookup
                    + st["n_ext_occ"] * 8             # occurrences outside the slot
                    + n_reads * 4 + st["n_stored"] * 16)   # location counts and records out
    hbm, peak_kind = peaks()
    seed_requests = st["n_minimizers"] + st["n_ext_occ"] * 8 / 32.0
    gather_gps = gather_ceiling(torch)
    achieved = seed_bytes / (st["ms_seed"] / 1000.0) / 1e9
    # instruction issue: one warp instruction per cycle per scheduler, 4 schedulers per SM, at
    # the SM clock sampled during the timed region (the maximum clock when none was sampled)
    issue = None
    seed_dram_per_read, seed_inst_per_read = seed_profile()
    if seed_inst_per_read:
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
        peak_issue = sms * 4 * mhz * 1e6 / 1e9
        got_issue = seed_inst_per_read * n_reads / (st["ms_seed"] / 1000.0) / 1e9
        issue = {"achieved": got_issue, "peak": peak_issue, "unit": "G warp instructions/s",
                 "frac": got_issue / peak_issue, "warp_instructions_per_read": seed_inst_per_read,
                 "peak_kind": "%d SMs x 4 schedulers x 1 instruction/cycle x %.0f MHz (sampled SM clock)" % (sms, mhz)}
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": (seed_dram_per_read * n_reads if seed_dram_per_read else None),
                "traffic_capture": SEED_PROFILE["capture"] if seed_dram_per_read else None,
                "kernel": "k_seed",
                "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
                "algorithmic_bytes_per_launch": seed_bytes, "ms_per_launch": st["ms_seed"],
                "algorithmic_bytes_per_read": seed_bytes / n_reads,
                "fused_minimum": {"bytes_per_launch": design_bytes, "bytes_per_read": design_bytes / n_reads,
                                  "achieved": design_bytes / (st["ms_seed"] / 1000.0) / 1e9,
                                  "frac": design_bytes / (st["ms_seed"] / 1000.0) / 1e9 / hbm},
                "issue": issue,
                "random_access": {"achieved": seed_requests / (st["ms_seed"] / 1000.0) / 1e9,
                                  "peak": gather_gps, "unit": "G random requests/s",
                                  "frac": seed_requests / (st["ms_seed"] / 1000.0) / 1e9 / gather_gps,
                                  "requests_per_launch": seed_requests,
                                  "requests": "one 32-byte slot per lookup + occurrence-list bytes / 32",
                                  "peak_kind": "measured in this run: torch.index_select of 8-byte words at "
                                               "2^26 random indices over a 4 GiB table"},
                "stage_ms": {k[3:]: st[k] for k in ("ms_seed", "ms_select", "ms_eda", "ms_profile", "ms_total")}}

    line = {"metric": METRIC, "value": value, "unit": "reads/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic (seeded generator; the paper's CAMI reads "
                                                            "and NCBI database are not available)",
            "config": {"workload": workload_name(c), "reads": n_reads, "genomes": g.n, "reference_bases": int(g.offsets[-1]),
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (%.2f GB reads, %.2f GB index)" % (n_bases / 1e9, info["device_bytes"] / 1e9)},
            "pairs_per_s": st["n_candidates"] / (ms / 1000.0) * world,
            "plain": {"value": job_rate(n_reads, world, ms_plain), "ms_per_step": ms_plain, "identical": identical},
            "graph": {"value": job_rate(n_reads, world, ms_graph), "ms_per_step": ms_graph,
                      "identical": graph_identical,
                      "e2e_value": job_rate(n_reads, world, e2e_graph_ms), "e2e_ms_per_step": e2e_graph_ms},
            "roofline": roofline,
            "e2e": {"value": job_rate(n_reads, world, e2e_ms), "unit": "reads/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                    "result": "per-read taxon and location count, per-genome hits and abundances (pinned host arrays)",
                    "with_locations": {"value": job_rate(n_reads, world, e2e_locs_ms), "ms_per_step": e2e_locs_ms,
                                       "d2h_bytes_per_step": d2h_locs}},
            "clocks": clocks, "gpu_launches": int(st["n_launches"]) * args.steps,
            "eda_shape": eda_shape,
            "index": {"build_s": index_s, **info},
            "classified_frac": float((batched_out["taxon"] >= 0).float().mean().item()),
            "other_approximations": approx,
            "containment_only": contain,
            "partitioned_database": part,
            "counts_per_step": {k: st[k] for k in ("n_minimizers", "n_hits", "n_candidates", "n_accepted",
                                                   "n_multi", "n_fallback", "n_ext_occ", "n_stored")}}

    # the serving sample runs before the EDA-only leg, whose ~10 GB of generated host pairs
    # otherwise leave the host-side transfers of the request loop measurably slower
    if rank == 0 and world == 1 and args.serve_seconds > 0:
        t0 = time.time()
        line["serving"] = serving_sample(mt, ix, reads, c, args.serve_seconds, torch, h_reads.numpy())
        log("[ours] serving %.1fs" % (time.time() - t0))
    if rank == 0 and world == 1 and args.eda_pairs > 0:
        t0 = time.time()
        line["eda_stage"] = eda_stage(mt, torch, args.eda_pairs, max(1, args.steps // 2), 1)
        log("[ours] eda stage %.1fs" % (time.time() - t0))
        torch.cuda.empty_cache()
    if rank == 0 and world == 1 and args.large_reads > 0:
        t0 = time.time()
        line["large_workload"] = large_workload(mt, torch, args.large_reads, max(1, args.steps // 2), 3, hbm)
        log("[ours] large workload %.1fs" % (time.time() - t0))
    if rank == 0 and world == 1 and args.cpu_sample > 0:
        import oracle
        t0 = time.time()
        oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
        rng = np.random.default_rng(4321)
        idx = np.sort(rng.choice(reads.n, args.cpu_sample, replace=False))
        sub = gen.subsample_reads(reads, idx)
        p = oracle.params(**{k: v for k, v in params(c, 0).items() if k != "eda_mode"})
        t = time.perf_counter()
        oracle.classify(oix, sub.seq, sub.offsets, p, threads=1)
        dt = time.perf_counter() - t
        line["cpu_baseline"] = {"value": args.cpu_sample / dt, "unit": "reads/s", "cores": 1, "kind": "oracle",
                                "sample": "%d random reads of the workload, one thread, index prebuilt "
                                          "(host has %d cores)" % (args.cpu_sample, len(os.sched_getaffinity(0))),
                                "seconds": dt}
        log("[ours] cpu baseline %.1fs" % (time.time() - t0))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--reads", type=int, default=gen.CONFIGS[2]["n_reads"])
    ap.add_argument("--genomes", type=int, default=gen.CONFIGS[2]["n_genomes"],
                    help="genomes of the medium reference (clades of 10); fewer make a small profiling case")
    ap.add_argument("--eda-pairs", type=int, default=gen.CONFIGS[3]["n_pairs"])
    ap.add_argument("--serve-seconds", type=float, default=100.0,
                    help="seconds of serving arrivals (20 batches/s; 100 s = the workload's 2,000 batches)")
    ap.add_argument("--cpu-sample", type=int, default=200_000)
    ap.add_argument("--part-batches", type=int, default=25)
    ap.add_argument("--large-reads", type=int, default=10_000_000,
                    help="time the large workload (6 Gb reference) on a sub-batch of this many reads (0: skip)")
    ap.add_argument("--ref-sample", type=int, default=20_000)
    ap.add_argument("--tune", type=int, default=1,
                    help="1: time the approximation kernel's shapes once before the classification legs; "
                         "0: run the untuned default shape (for profiling: tuning under a profiler times noise)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
