"""Seeded generators for the five workloads (genomes, reads, EDA pairs, serving arrivals).

Everything is drawn with numpy's PCG64 from a fixed seed and vectorised over chunks, so
the paper-sized inputs (10^7 reads, 4x10^8 reference bases) are produced in seconds.

Bases are ASCII ``A C G T`` (uint8). Genomes and reads are returned as one concatenated
byte array plus a uint64 offsets array of length ``count + 1``.

The five configurations mirror the paper's workloads (short Illumina reads of 100-250 bp
against clade-structured microbial references, Results "Evaluation Methodology"; the CAMI
sets hold ~10^8 reads of 150 bp). The paper's own read sets and NCBI database are not
available, so these seeded stand-ins are used instead.
"""
from __future__ import annotations

import ctypes
import dataclasses
import hashlib
import math
import os
import subprocess
import threading

import numpy as np

ASCII = np.frombuffer(b"ACGT", dtype=np.uint8)
_COMP = np.zeros(256, dtype=np.uint8)
for _a, _b in zip(b"ACGT", b"TGCA"):
    _COMP[_a] = _b


_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LIB_LOCK = threading.Lock()


def _assemble_lib():
    """Compile (once) and load the window-assembly helper written in plain C."""
    global _LIB
    with _LIB_LOCK:
        if _LIB is None:
            src = os.path.join(_HERE, "_assemble.c")
            so = os.path.join(_HERE, "_assemble.so")
            cmd = ["gcc", "-O2", "-shared", "-fPIC"]
            with open(src, "rb") as f:
                want = hashlib.sha256(repr(cmd).encode() + f.read()).hexdigest()
            stamp = so + ".sha256"
            have = open(stamp).read().strip() if os.path.exists(stamp) else ""
            if not os.path.exists(so) or have != want:   # rebuilt on a content change, not on file times
                tmp = so + ".%d.tmp" % os.getpid()
                subprocess.check_call(cmd + ["-o", tmp, src])
                os.replace(tmp, so)
                with open(stamp + ".tmp", "w") as f:
                    f.write(want + "\n")
                os.replace(stamp + ".tmp", stamp)
            _LIB = ctypes.CDLL(so)
            _LIB.gen_assemble.restype = ctypes.c_int
        return _LIB


def build() -> None:
    """Compile the C helper ahead of time."""
    _assemble_lib()


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


def ascii_of(codes: np.ndarray) -> np.ndarray:
    """Map integer codes 0..3 to ASCII bases A, C, G, T."""
    return ASCII[codes]


def revcomp_ascii(seq: np.ndarray) -> np.ndarray:
    """Reverse complement of an ASCII ACGT array (used to draw reverse-strand reads)."""
    return _COMP[seq[::-1]]


@dataclasses.dataclass
class Genomes:
    seq: np.ndarray        # uint8 ASCII, all genomes concatenated
    offsets: np.ndarray    # uint64, n_genomes + 1
    clade: np.ndarray      # int32 clade id per genome

    @property
    def n(self) -> int:
        return len(self.offsets) - 1

    def genome(self, g: int) -> np.ndarray:
        return self.seq[self.offsets[g]:self.offsets[g + 1]]


@dataclasses.dataclass
class Reads:
    seq: np.ndarray        # uint8 ASCII, all reads concatenated
    offsets: np.ndarray    # uint64, n_reads + 1
    truth_genome: np.ndarray   # int32, -1 for random reads
    truth_pos: np.ndarray      # int64, forward-strand start of the source segment
    truth_strand: np.ndarray   # uint8, 1 = read is the reverse complement

    @property
    def n(self) -> int:
        return len(self.offsets) - 1

    @property
    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def read(self, i: int) -> np.ndarray:
        return self.seq[self.offsets[i]:self.offsets[i + 1]]


@dataclasses.dataclass
class EdaPairs:
    read_seq: np.ndarray   # uint8 ASCII reads, concatenated
    read_off: np.ndarray   # uint64, n_reads + 1
    win_seq: np.ndarray    # uint8 ASCII windows, concatenated
    win_off: np.ndarray    # uint64, n_pairs + 1
    pair_read: np.ndarray  # uint32 read index of each pair
    E: np.ndarray          # uint16 edit threshold of each pair
    planted: np.ndarray    # uint16 number of edits drawn for each pair (not a label)

    @property
    def n_pairs(self) -> int:
        return len(self.pair_read)

    @property
    def n_reads(self) -> int:
        return len(self.read_off) - 1


# --------------------------------------------------------------------------------------
# Workload definitions (sizes follow the paper's short-read setting: 150 bp CAMI reads,
# 100 bp TARA reads, clade-structured microbial references).
# --------------------------------------------------------------------------------------
CONFIGS = {
    1: dict(name="tiny: 8x50kb uniform, k15 w10, 10k x 150bp, E=6",
            n_genomes=8, genome_len=50_000, clade_size=1, gc=(0.5, 0.5), divergence=(0.0, 0.0),
            genome_seed=0, k=15, w=10, canonical=0, n_reads=10_000, read_lens=((150, 1.0),),
            abundance="uniform", p_sub=0.01, p_indel=0.001, p_random=0.10, both_strands=False,
            min_seeds=2, e_abs=6, e_permille=0, seed=1001),
    2: dict(name="medium: 200x2Mb (20 clades x 10), k21 w11 canonical, 10M x 150bp, E=8",
            n_genomes=200, genome_len=2_000_000, clade_size=10, gc=(0.30, 0.70),
            divergence=(0.01, 0.10), genome_seed=1002, k=21, w=11, canonical=1,
            n_reads=10_000_000, read_lens=((150, 1.0),), abundance="lognormal", sigma=1.5,
            p_sub=0.005, p_indel=0.0005, p_random=0.05, both_strands=True,
            min_seeds=3, e_abs=8, e_permille=0, seed=2002),
    3: dict(name="EDA batch: 5e7 pairs, n~U[100,250], E in {2,4,6,10}% of n",
            n_pairs=50_000_000, len_range=(100, 250), e_fracs=(0.02, 0.04, 0.06, 0.10),
            mean_cands=6, max_cands=200, frac_within=0.70, seed=3003),
    4: dict(name="serving: config-2 index, Poisson 20 batches/s, 1k-1M reads log-uniform",
            rate=20.0, batch_min=1_000, batch_max=1_000_000, n_batches=2000, seed=4004),
    5: dict(name="large: 2000x3Mb (200 clades x 10), k21 w11, 1e8 reads 60%150/40%250, E=5%",
            n_genomes=2000, genome_len=3_000_000, clade_size=10, gc=(0.30, 0.70),
            divergence=(0.01, 0.15), genome_seed=5005, k=21, w=11, canonical=1,
            n_reads=100_000_000, read_lens=((150, 0.6), (250, 0.4)), abundance="lognormal",
            sigma=2.0, p_sub=0.01, p_indel=0.001, p_random=0.10, both_strands=True,
            min_seeds=3, e_abs=0, e_permille=50, seed=5006),
}


def config(cfg_id: int, **overrides) -> dict:
    """Return a copy of workload ``cfg_id`` with optional overrides (e.g. n_reads=...)."""
    c = dict(CONFIGS[cfg_id])
    c.update(overrides)
    return c


# --------------------------------------------------------------------------------------
# Genomes
# --------------------------------------------------------------------------------------
def _draw_codes(rng: np.random.Generator, n: int, gc: float) -> np.ndarray:
    """i.i.d. bases with P(C)=P(G)=gc/2 and P(A)=P(T)=(1-gc)/2, as codes 0..3."""
    u = rng.random(n, dtype=np.float32)
    at = (1.0 - gc) / 2.0
    # cumulative thresholds for A, C, G, T
    t1, t2, t3 = at, at + gc / 2.0, at + gc
    out = np.full(n, 3, dtype=np.uint8)
    out[u < t3] = 2
    out[u < t2] = 1
    out[u < t1] = 0
    return out


def _substitute(rng: np.random.Generator, codes: np.ndarray, rate: float, gc: float) -> np.ndarray:
    """Substitute each base with probability ``rate``; the new base is drawn from the
    same GC composition, conditioned on differing from the old base."""
    out = codes.copy()
    idx = np.flatnonzero(rng.random(len(codes), dtype=np.float32) < rate)
    if len(idx) == 0:
        return out
    old = out[idx]
    new = _draw_codes(rng, len(idx), gc)
    for _ in range(8):
        same = new == old
        if not same.any():
            break
        new[same] = _draw_codes(rng, int(same.sum()), gc)
    same = new == old
    new[same] = (old[same] + rng.integers(1, 4, int(same.sum()), dtype=np.uint8)) % 4
    out[idx] = new
    return out


def make_genomes(c: dict) -> Genomes:
    """Clade-structured reference: ``n_genomes / clade_size`` clade roots with a per-clade
    GC content, members are substitution-mutated copies of the root (divergence drawn
    uniformly per member). ``clade_size == 1`` gives independent genomes. Clades are drawn on
    threads, each from its own child seed, so the result does not depend on the thread count."""
    G, L, cs = c["n_genomes"], c["genome_len"], c["clade_size"]
    n_clades = G // cs
    seq = np.empty(G * L, dtype=np.uint8)
    clade = np.repeat(np.arange(n_clades, dtype=np.int32), cs)

    def one(cl, rng):
        gc = float(rng.uniform(*c["gc"]))
        root = _draw_codes(rng, L, gc)
        for m in range(cs):
            g = cl * cs + m
            if cs == 1:
                member = root
            else:
                div = float(rng.uniform(*c["divergence"]))
                member = _substitute(rng, root, div, gc)
            seq[g * L:(g + 1) * L] = ASCII[member]

    _run_chunks(one, n_clades, c["genome_seed"])
    offsets = np.arange(G + 1, dtype=np.uint64) * np.uint64(L)
    return Genomes(seq=seq, offsets=offsets, clade=clade)


# --------------------------------------------------------------------------------------
# Reads
# --------------------------------------------------------------------------------------
def _abundance(rng: np.random.Generator, c: dict, G: int) -> np.ndarray:
    if c["abundance"] == "uniform":
        return np.full(G, 1.0 / G)
    w = rng.lognormal(mean=0.0, sigma=c["sigma"], size=G)
    return w / w.sum()


def _sample_segments(rng, gseq, goff, glen, src_g, n, p_sub, p_indel):
    """Draw ``len(src_g)`` forward-strand reads of length n from the given source genomes
    with per-base substitution / 1-bp insertion / 1-bp deletion errors. Error positions are
    drawn sparsely (a binomial count, then uniform positions). Returns (ASCII[m, n], start)."""
    m = len(src_g)
    src_g = src_g.astype(np.int64)
    n_ev = int(rng.binomial(m * n, p_indel)) if p_indel > 0 else 0
    ev_pos = rng.integers(0, m * n, n_ev)
    ev_ins = rng.random(n_ev) < 0.5
    rows_with = np.unique(ev_pos // n)
    span = np.full(m, n, dtype=np.int64)
    if len(rows_with):
        kr = np.searchsorted(rows_with, ev_pos // n)
        col = ev_pos % n
        ins = np.zeros((len(rows_with), n), dtype=bool)
        dele = np.zeros((len(rows_with), n), dtype=bool)
        ins[kr[ev_ins], col[ev_ins]] = True
        dele[kr[~ev_ins], col[~ev_ins]] = True
        dele &= ~ins
        adv = 1 + dele.astype(np.int64) - ins.astype(np.int64)
        span[rows_with] = adv.sum(axis=1)
    gl = glen[src_g].astype(np.int64)
    start = np.floor(rng.random(m) * (gl - span + 1)).astype(np.int64)
    gstart = goff[src_g].astype(np.int64) + start
    out = np.empty((m, n), dtype=np.uint8)
    plain = np.ones(m, dtype=bool)
    plain[rows_with] = False
    out[plain] = np.lib.stride_tricks.sliding_window_view(gseq, n)[gstart[plain]]
    if len(rows_with):
        ptr = np.cumsum(adv, axis=1) - adv           # source offset before each output base
        srcpos = np.minimum(start[rows_with, None] + ptr + dele, gl[rows_with, None] - 1)
        sub_rows = gseq[goff[src_g[rows_with]].astype(np.int64)[:, None] + srcpos]
        sub_rows[ins] = ASCII[rng.integers(0, 4, int(ins.sum()), dtype=np.uint8)]
        out[rows_with] = sub_rows
    n_sub = int(rng.binomial(m * n, p_sub)) if p_sub > 0 else 0
    if n_sub:
        pos = rng.integers(0, m * n, n_sub)
        flat = out.reshape(-1)
        codes = np.searchsorted(ASCII, flat[pos]).astype(np.uint8)
        flat[pos] = ASCII[(codes + rng.integers(1, 4, n_sub, dtype=np.uint8)) % 4]
    return out, start


def _threads() -> int:
    import os
    try:
        return max(1, min(16, len(os.sched_getaffinity(0))))
    except AttributeError:  # pragma: no cover
        return max(1, min(16, os.cpu_count() or 1))


def _run_chunks(fn, n_chunks: int, seed: int):
    """Run fn(chunk_index, rng) for every chunk in a thread pool; every chunk draws from its
    own child seed, so the output does not depend on the thread count."""
    from concurrent.futures import ThreadPoolExecutor
    seeds = np.random.SeedSequence(seed).spawn(n_chunks)
    with ThreadPoolExecutor(_threads()) as ex:
        list(ex.map(lambda i: fn(i, np.random.Generator(np.random.PCG64(seeds[i]))),
                    range(n_chunks)))


def make_reads(c: dict, genomes: Genomes, n_reads: int | None = None, seed: int | None = None,
               chunk: int = 1 << 17) -> Reads:
    """Reads drawn as the workload describes: a fraction of uniform-random (non-matching)
    reads, the rest sampled from genomes by (uniform or log-normal) abundance with
    substitution/indel errors and, where ``both_strands``, a 50/50 strand."""
    n_reads = c["n_reads"] if n_reads is None else n_reads
    seed = c["seed"] if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed))
    G = genomes.n
    goff = genomes.offsets.astype(np.int64)
    glen = np.diff(goff)
    ab = _abundance(rng, c, G)

    lens_vals = np.array([l for l, _ in c["read_lens"]], dtype=np.int64)
    lens_p = np.array([p for _, p in c["read_lens"]], dtype=np.float64)
    lens = lens_vals[rng.choice(len(lens_vals), size=n_reads, p=lens_p / lens_p.sum())]
    is_rand = rng.random(n_reads) < c["p_random"]
    n_src = int((~is_rand).sum())
    if c["abundance"] == "uniform":
        src_list = rng.integers(0, G, n_src)
    else:
        counts = rng.multinomial(n_src, ab)
        src_list = np.repeat(np.arange(G), counts)
        rng.shuffle(src_list)
    src_g = np.full(n_reads, -1, dtype=np.int32)
    src_g[~is_rand] = src_list
    strand = np.zeros(n_reads, dtype=np.uint8)
    if c["both_strands"]:
        strand[~is_rand] = (rng.random(n_src) < 0.5).astype(np.uint8)

    offsets = np.zeros(n_reads + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum(lens)
    seq = np.empty(int(offsets[-1]), dtype=np.uint8)
    pos = np.full(n_reads, -1, dtype=np.int64)
    n_chunks = (n_reads + chunk - 1) // chunk

    def one(ci, crng):
        lo, hi = ci * chunk, min(n_reads, (ci + 1) * chunk)
        base0 = int(offsets[lo])
        local = seq[base0:int(offsets[hi])]
        for L in np.unique(lens[lo:hi]):
            idx = lo + np.flatnonzero(lens[lo:hi] == L)
            out = np.empty((len(idx), L), dtype=np.uint8)
            r = is_rand[idx]
            if r.any():
                out[r] = ASCII[crng.integers(0, 4, (int(r.sum()), L), dtype=np.uint8)]
            nr = ~r
            if nr.any():
                seg, st = _sample_segments(crng, genomes.seq, goff, glen, src_g[idx[nr]], int(L),
                                           c["p_sub"], c["p_indel"])
                rc = strand[idx[nr]] == 1
                if rc.any():
                    seg[rc] = _COMP[seg[rc][:, ::-1]]
                out[nr] = seg
                pos[idx[nr]] = st
            if len(idx) == hi - lo:          # one length in this chunk: contiguous rows
                local[:] = out.reshape(-1)
            else:
                dst = (offsets[idx].astype(np.int64) - base0)[:, None] + np.arange(L)[None, :]
                local[dst.ravel()] = out.ravel()

    _run_chunks(one, n_chunks, seed + 1)
    return Reads(seq=seq, offsets=offsets, truth_genome=src_g, truth_pos=pos, truth_strand=strand)


def subsample_reads(reads: Reads, idx: np.ndarray) -> Reads:
    """A read set holding reads ``idx`` (in that order)."""
    idx = np.asarray(idx, dtype=np.int64)
    lens = (reads.offsets[idx + 1] - reads.offsets[idx]).astype(np.int64)
    off = np.zeros(len(idx) + 1, dtype=np.uint64)
    off[1:] = np.cumsum(lens)
    seq = np.empty(int(off[-1]), dtype=np.uint8)
    for L in np.unique(lens):
        sel = np.flatnonzero(lens == L)
        src = reads.offsets[idx[sel]].astype(np.int64)[:, None] + np.arange(L)[None, :]
        dst = off[sel].astype(np.int64)[:, None] + np.arange(L)[None, :]
        seq[dst.ravel()] = reads.seq[src.ravel()]
    return Reads(seq=seq, offsets=off, truth_genome=reads.truth_genome[idx],
                 truth_pos=reads.truth_pos[idx], truth_strand=reads.truth_strand[idx])


# --------------------------------------------------------------------------------------
# Read-versus-window pairs for the edit-distance-approximation stage alone
# --------------------------------------------------------------------------------------
def make_eda_pairs(c: dict, n_pairs: int | None = None, seed: int | None = None,
                   chunk: int = 1 << 18) -> EdaPairs:
    """Reads with n ~ U[len_range], a per-read count of candidate windows ~ geometric
    (mean ``mean_cands``, capped), and per pair E = floor(n * f) with f drawn from
    ``e_fracs``. Each window has length n + 2E and holds the read with a planted number of
    random edits (``frac_within`` of pairs draw <= E edits, the rest E+1..3E; substitution,
    insertion or deletion at uniform positions), between random flanks, shifted by up to
    E/2 from diagonal 0. The planted count is only a generator knob: which pairs pass is
    decided by the oracle."""
    n_pairs = c["n_pairs"] if n_pairs is None else n_pairs
    seed = c["seed"] if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = c["len_range"]
    counts = []
    tot = 0
    while tot < n_pairs:
        k = np.minimum(rng.geometric(1.0 / c["mean_cands"], size=max(1024, (n_pairs - tot) // 5)),
                       c["max_cands"])
        counts.append(k)
        tot += int(k.sum())
    counts = np.concatenate(counts)
    cs = np.cumsum(counts)
    n_reads = int(np.searchsorted(cs, n_pairs) + 1)
    counts = counts[:n_reads].copy()
    counts[-1] -= int(cs[n_reads - 1] - n_pairs)
    pair_read = np.repeat(np.arange(n_reads, dtype=np.uint32), counts)

    rlen = rng.integers(lo, hi + 1, n_reads).astype(np.int64)
    read_off = np.zeros(n_reads + 1, dtype=np.uint64)
    read_off[1:] = np.cumsum(rlen)
    read_seq = ASCII[rng.integers(0, 4, int(read_off[-1]), dtype=np.uint8)]

    fr = np.asarray(c["e_fracs"], dtype=np.float64)
    n_of_pair = rlen[pair_read]
    E = np.floor(n_of_pair * fr[rng.integers(0, len(fr), n_pairs)] + 1e-9).astype(np.int64)
    within = rng.random(n_pairs) < c["frac_within"]
    e_lo = np.where(within, 0, E + 1)
    e_hi = np.where(within, E, 3 * E)
    planted = (e_lo + np.floor(rng.random(n_pairs) * (e_hi - e_lo + 1))).astype(np.int64)

    shift = np.floor((rng.random(n_pairs) - 0.5) * (E + 1)).astype(np.int64)
    left = np.clip(E + shift, 0, 2 * E)
    wlen = n_of_pair + 2 * E
    win_off = np.zeros(n_pairs + 1, dtype=np.uint64)
    win_off[1:] = np.cumsum(wlen)
    win_seq = np.empty(int(win_off[-1]), dtype=np.uint8)
    lib = _assemble_lib()
    n_chunks = (n_pairs + chunk - 1) // chunk

    def one(ci, crng):
        a, b = ci * chunk, min(n_pairs, (ci + 1) * chunk)
        w0, w1 = int(win_off[a]), int(win_off[b])
        win_seq[w0:w1] = ASCII[crng.integers(0, 4, w1 - w0, dtype=np.uint8)]
        ne = planted[a:b]
        ev_off = np.zeros(b - a + 1, dtype=np.uint64)
        ev_off[1:] = np.cumsum(ne)
        tot = int(ev_off[-1])
        ev_pos = np.floor(crng.random(tot) * np.repeat(n_of_pair[a:b], ne)).astype(np.int32)
        ev_kind = crng.integers(0, 3, tot, dtype=np.uint8)
        ev_sub = crng.integers(1, 4, tot, dtype=np.uint8)
        woff = (win_off[a:b + 1] - np.uint64(w0)).astype(np.uint64)
        lib.gen_assemble(
            ctypes.c_uint64(b - a), _p(read_seq), _p(read_off), _p(pair_read[a:b]), _p(woff),
            _p(np.ascontiguousarray(wlen[a:b])), _p(np.ascontiguousarray(left[a:b])), _p(ev_off),
            _p(ev_pos), _p(ev_kind), _p(ev_sub), _p(win_seq[w0:w1]))

    _run_chunks(one, n_chunks, seed + 1)
    return EdaPairs(read_seq=read_seq, read_off=read_off, win_seq=win_seq, win_off=win_off,
                    pair_read=pair_read, E=E.astype(np.uint16), planted=planted.astype(np.uint16))


# --------------------------------------------------------------------------------------
# Serving arrivals
# --------------------------------------------------------------------------------------
def make_arrivals(c: dict, n_batches: int | None = None, seed: int | None = None):
    """Poisson arrival times (seconds) and log-uniform batch sizes (reads)."""
    n_batches = c["n_batches"] if n_batches is None else n_batches
    rng = np.random.Generator(np.random.PCG64(c["seed"] if seed is None else seed))
    gaps = rng.exponential(1.0 / c["rate"], n_batches)
    t = np.cumsum(gaps) - gaps[0]
    lo, hi = math.log10(c["batch_min"]), math.log10(c["batch_max"])
    sizes = np.round(10.0 ** rng.uniform(lo, hi, n_batches)).astype(np.int64)
    return t, sizes


# --------------------------------------------------------------------------------------
# Taxonomy (synthetic: the NCBI taxonomy is not available)
# --------------------------------------------------------------------------------------
@dataclasses.dataclass
class Taxonomy:
    parent: np.ndarray        # int32 per node, -1 for the root
    rank: list                # rank name per node
    name: list                # scientific name per node
    taxid: np.ndarray         # int64 identifier per node
    genome_node: np.ndarray   # uint32 leaf node of each genome
    ranks: tuple              # the ranks present, root first


def make_taxonomy(genomes: Genomes) -> Taxonomy:
    """A three-rank tree over the reference: one superkingdom, a genus per clade, a species per
    genome (clade members are the species of their clade's genus). Node 0 is the root, nodes
    1..C the clades, nodes C+1.. the genomes; taxids are 10^6 + node."""
    n_clades = int(genomes.clade.max()) + 1 if genomes.n else 0
    n = 1 + n_clades + genomes.n
    parent = np.empty(n, np.int32)
    parent[0] = -1
    parent[1:1 + n_clades] = 0
    parent[1 + n_clades:] = 1 + genomes.clade
    rank = ["superkingdom"] + ["genus"] * n_clades + ["species"] * genomes.n
    name = ["Synthetica"] + ["Clade_%d" % i for i in range(n_clades)] + ["Genome_%d" % g for g in range(genomes.n)]
    return Taxonomy(parent=parent, rank=rank, name=name, taxid=10 ** 6 + np.arange(n, dtype=np.int64),
                    genome_node=(1 + n_clades + np.arange(genomes.n)).astype(np.uint32),
                    ranks=("superkingdom", "genus", "species"))
