"""CPU oracle of the MetaTrinity hot path -- TEST INFRASTRUCTURE ONLY.

A plain single-threaded C implementation (``mt_oracle.c``) of seeding, containment
counting, location filtering, SneakySnake edit-distance approximation and abundance
estimation, written step by step from the paper (arXiv 2311.02029), plus this thin ctypes
wrapper. Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline and
reference legs may import it; the CUDA library never does, and shares no code with it.

Parity pins (tests/test_oracle_*.py): the SplitMix64 published output sequence, brute-force
window minima, brute-force seed enumeration per genome, a hand-worked SneakySnake example,
the E = 0 Hamming reduction, an exact dynamic-programming restatement of the greedy walk,
upper bounds by per-diagonal Hamming distance and by banded edit distance (no false
reject), a lower bound by all-obstacle columns, planted-truth mapping of error-free reads,
a location spanning exactly E diagonals, a hand-worked rank order of equal-seed locations
(strand, then first diagonal), brute-force mapping locations with the repeat filter at the
exact occurrence count, and hand-computed abundance splits; for a database cut into batches,
reduction to the single-index pipeline when no key reaches the repeat filter,
highest-not-summed counts of a genome held by several batches, and brute-force per-batch
repeat filtering; for genome shards on separate devices, reduction to the single-index
pipeline and a hand-worked merge by rank with a unique read whose best locations share one
genome. Every reading the oracle takes (mixer, leftmost-minimum tie, location clustering,
rank tie-breaks, repeat filter, window edges, multi-read split) has such a pin.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mt_oracle.c")
_SO = os.path.join(_HERE, "_mt_oracle.so")
_lib = None
_lock = threading.Lock()

LOC_DTYPE = np.dtype({"names": ["wstart", "genome", "seeds", "strand", "dist"],
                      "formats": [np.int64, np.int32, np.uint32, np.uint8, np.uint8],
                      "offsets": [0, 8, 12, 16, 17], "itemsize": 24})


_CMD = ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread"]


def build() -> str:
    """Compile the oracle with gcc (plain C, -O2, no machine-specific flags); rebuilt whenever
    the SHA-256 of the command and the source differs from the one it was built from."""
    with _lock:
        with open(_SRC, "rb") as f:
            want = hashlib.sha256(repr(_CMD).encode() + f.read()).hexdigest()
        stamp = _SO + ".sha256"
        have = open(stamp).read().strip() if os.path.exists(stamp) else ""
        if not os.path.exists(_SO) or have != want:
            tmp = _SO + ".%d.tmp" % os.getpid()
            subprocess.check_call(_CMD + ["-o", tmp, _SRC])
            os.replace(tmp, _SO)
            with open(stamp + ".tmp", "w") as f:
                f.write(want + "\n")
            os.replace(stamp + ".tmp", stamp)
    return _SO


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        u64, u32, vp, i64 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int64
        lib.or_mix64.restype = u64
        lib.or_mix64.argtypes = [u64]
        lib.or_minimizers.restype = i64
        lib.or_minimizers.argtypes = [vp, u64, u32, u32, u32, vp, vp, vp, vp]
        lib.or_build_index.restype = vp
        lib.or_build_index.argtypes = [vp, vp, u32, u32, u32, u32, ctypes.POINTER(ctypes.c_int)]
        lib.or_build_index_threads.restype = vp
        lib.or_build_index_threads.argtypes = [vp, vp, u32, u32, u32, u32, u32, ctypes.POINTER(ctypes.c_int)]
        lib.or_free_index.argtypes = [vp]
        lib.or_index_n_occ.restype = u64
        lib.or_index_n_occ.argtypes = [vp]
        lib.or_index_lookup.restype = u64
        lib.or_index_lookup.argtypes = [vp, u64, vp, u64]
        lib.or_count_hits.restype = ctypes.c_int
        lib.or_count_hits.argtypes = [vp, vp, vp, u64, u32, vp]
        lib.or_keep.argtypes = [vp, u32, u32, u32, vp]
        lib.or_eda_codes.restype = u32
        lib.or_eda_codes.argtypes = [vp, u32, vp, u32]
        lib.or_eda_ascii.restype = u32
        lib.or_eda_ascii.argtypes = [vp, u32, vp, u32]
        lib.or_eda_batch.restype = ctypes.c_int
        lib.or_eda_batch.argtypes = [vp, vp, vp, vp, vp, vp, u64, u32, vp]
        for fn in ("or_hd_codes", "or_bc_codes", "or_qgram_codes", "or_shd_codes"):
            getattr(lib, fn).restype = u32
            getattr(lib, fn).argtypes = [vp, u32, vp, u32]
        lib.or_qgram_q.restype = u32
        lib.or_qgram_q.argtypes = [vp, u32, vp, u32, u32]
        lib.or_hpc.argtypes = [vp, vp, u64, vp, vp]
        lib.or_rollup.restype = ctypes.c_int
        lib.or_rollup.argtypes = [vp, u32, vp, vp, u32, vp]
        lib.or_approx_codes.restype = u32
        lib.or_approx_codes.argtypes = [u32, vp, u32, vp, u32]
        lib.or_map_reads.restype = ctypes.c_int
        lib.or_map_reads.argtypes = [vp, vp, vp, u64, u32, u32, u32, u32, u32, u32, vp, vp, vp, vp,
                                     vp, vp]
        lib.or_abundance.argtypes = [vp, u32, vp, u64, u32, ctypes.c_double, vp]
        _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "arrays passed to the oracle must be contiguous"
    return ctypes.c_void_p(a.ctypes.data)


def _u8(seq) -> np.ndarray:
    if isinstance(seq, (bytes, bytearray, str)):
        seq = seq.encode() if isinstance(seq, str) else bytes(seq)
        return np.frombuffer(seq, dtype=np.uint8).copy()
    return np.ascontiguousarray(seq, dtype=np.uint8)


class OracleError(RuntimeError):
    pass


def mix64(z: int) -> int:
    return int(_L().or_mix64(ctypes.c_uint64(z & 0xFFFFFFFFFFFFFFFF)))


def minimizers(seq, k: int, w: int, canonical: int):
    """(code, key, pos, strand) arrays of the (w,k)-minimizers of an ASCII sequence."""
    s = _u8(seq)
    n = len(s)
    code = np.zeros(max(n, 1), np.uint64)
    key = np.zeros(max(n, 1), np.uint64)
    pos = np.zeros(max(n, 1), np.uint64)
    strand = np.zeros(max(n, 1), np.uint8)
    m = _L().or_minimizers(_p(s), n, k, w, canonical, _p(code), _p(key), _p(pos), _p(strand))
    if m < 0:
        raise OracleError("or_minimizers failed: %d" % m)
    return code[:m], key[:m], pos[:m].astype(np.int64), strand[:m]


class Index:
    """The oracle's reference index: all genome minimizers sorted by k-mer code."""

    def __init__(self, seq, offsets, k: int, w: int, canonical: int, threads: int = 1, compressed: bool = False):
        """``threads > 1`` builds the same index with the work split over host threads.
        ``compressed``: minimizers of the homopolymer-compressed genomes (a containment
        index; its positions are in compressed coordinates)."""
        self.hpc = bool(compressed)
        if self.hpc:
            seq, offsets = hpc(seq, offsets)
        self.seq = _u8(seq)
        self.offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        self.G = len(self.offsets) - 1
        self.k, self.w, self.canonical = k, w, canonical
        err = ctypes.c_int(0)
        if threads > 1:
            h = _L().or_build_index_threads(_p(self.seq), _p(self.offsets), self.G, k, w, canonical, threads,
                                            ctypes.byref(err))
        else:
            h = _L().or_build_index(_p(self.seq), _p(self.offsets), self.G, k, w, canonical,
                                    ctypes.byref(err))
        if not h:
            raise OracleError("or_build_index failed: %d" % err.value)
        self._h = ctypes.c_void_p(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.or_free_index(h)
            self._h = None

    @property
    def n_occ(self) -> int:
        return int(_L().or_index_n_occ(self._h))

    def lookup(self, code: int):
        n = int(_L().or_index_lookup(self._h, ctypes.c_uint64(code), None, 0))
        out = np.zeros(max(n, 1), np.uint64)
        _L().or_index_lookup(self._h, ctypes.c_uint64(code), _p(out), n)
        out = out[:n]
        return (out >> np.uint64(33)).astype(np.int64), ((out >> np.uint64(1)) & np.uint64(0xFFFFFFFF)).astype(np.int64), (out & np.uint64(1)).astype(np.uint8)


# eda_algo: 0 SneakySnake, 1 Hamming distance, 2 Base Counting, 3 q-gram (q = 5), 4 SHD
DEFAULT_PARAMS = dict(max_occ=1024, e_abs=0, e_permille=100, min_seeds=3, top_n=3,
                      cont_num=1, cont_den=10000, abund_cutoff=1e-4, eda_algo=0)
ALGOS = {"sneakysnake": 0, "hamming": 1, "base_counting": 2, "qgram": 3, "shd": 4}


def params(**kw) -> dict:
    p = dict(DEFAULT_PARAMS)
    p.update(kw)
    return p


def hpc(seq, offsets):
    """Homopolymer compression of a sequence set: each run of one base becomes one base."""
    s = _u8(seq)
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    n = len(off) - 1
    out = np.zeros(max(1, int(off[-1] - off[0])), np.uint8)
    out_off = np.zeros(n + 1, np.uint64)
    _L().or_hpc(_p(s), _p(off), n, _p(out), _p(out_off))
    return out[:int(out_off[-1])].copy(), out_off


def count_hits(ix: Index, reads_seq, reads_off, max_occ: int, hits: np.ndarray | None = None):
    """Seed hits per genome (containment); over compressed reads for a compressed index."""
    s = _u8(reads_seq)
    off = np.ascontiguousarray(reads_off, dtype=np.uint64)
    if getattr(ix, "hpc", False):
        s, off = hpc(s, off)
    if hits is None:
        hits = np.zeros(ix.G, np.uint64)
    rc = _L().or_count_hits(ix._h, _p(s), _p(off), len(off) - 1, max_occ, _p(hits))
    if rc != 0:
        raise OracleError("or_count_hits failed: %d" % rc)
    return hits


def keep_mask(hits: np.ndarray, num: int, den: int) -> np.ndarray:
    h = np.ascontiguousarray(hits, dtype=np.uint64)
    keep = np.zeros(len(h), np.uint8)
    _L().or_keep(_p(h), len(h), num, den, _p(keep))
    return keep


def map_reads(ix: Index, reads_seq, reads_off, p: dict, keep: np.ndarray):
    s = _u8(reads_seq)
    off = np.ascontiguousarray(reads_off, dtype=np.uint64)
    n = len(off) - 1
    tn = p["top_n"]
    taxon = np.zeros(n, np.int32)
    locs = np.zeros(n * tn, LOC_DTYPE)
    nloc = np.zeros(n, np.uint8)
    multi = np.zeros(n * tn, np.int32)
    U = np.zeros(ix.G, np.uint64)
    keep = np.ascontiguousarray(keep, dtype=np.uint8)
    rc = _L().or_map_reads(ix._h, _p(s), _p(off), n, p["max_occ"], p["e_abs"], p["e_permille"],
                           p["min_seeds"], tn, p.get("eda_algo", 0), _p(keep), _p(taxon), _p(locs), _p(nloc),
                           _p(multi), _p(U))
    if rc != 0:
        raise OracleError("or_map_reads failed: %d" % rc)
    return dict(taxon=taxon, locs=locs.reshape(n, tn), nloc=nloc, multi=multi.reshape(n, tn), U=U)


def abundance(U: np.ndarray, multi: np.ndarray, top_n: int, cutoff: float) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.uint64)
    m = np.ascontiguousarray(multi, dtype=np.int32).reshape(-1)
    a = np.zeros(len(U), np.float64)
    _L().or_abundance(_p(U), len(U), _p(m), len(m) // top_n, top_n, cutoff, _p(a))
    return a


def _shards(n: int, parts: int):
    parts = max(1, min(parts, n))
    b = np.linspace(0, n, parts + 1).astype(np.int64)
    return [(int(b[i]), int(b[i + 1])) for i in range(parts) if b[i + 1] > b[i]]


def _slice_reads(reads_seq, reads_off, a: int, b: int):
    off = np.ascontiguousarray(reads_off[a:b + 1], dtype=np.uint64)
    base = int(off[0])
    return reads_seq[base:int(off[-1])], off - np.uint64(base)


def classify(ix: Index, reads_seq, reads_off, p: dict, threads: int = 1, keep=None):
    """The whole batch: containment over all reads, the kept-genome mask, mapping and the
    per-read decision, then abundances. ``threads > 1`` shards the reads over host threads
    (the per-read results do not depend on the sharding; genome hits and unique counts are
    sums; the abundance step runs once over all reads). A given ``keep`` mask (e.g. from a
    separate containment index) replaces the batch's own containment mask."""
    s = _u8(reads_seq)
    off = np.ascontiguousarray(reads_off, dtype=np.uint64)
    n = len(off) - 1
    shards = _shards(n, threads) if n else []
    given = keep
    if threads <= 1 or len(shards) <= 1:
        hits = count_hits(ix, s, off, p["max_occ"])
        keep = keep_mask(hits, p["cont_num"], p["cont_den"]) if given is None else np.asarray(given, np.uint8)
        m = map_reads(ix, s, off, p, keep)
    else:
        with ThreadPoolExecutor(len(shards)) as ex:
            parts = list(ex.map(lambda ab: count_hits(ix, *_slice_reads(s, off, *ab), p["max_occ"]),
                                shards))
            hits = np.sum(parts, axis=0, dtype=np.uint64)
            keep = keep_mask(hits, p["cont_num"], p["cont_den"]) if given is None else np.asarray(given, np.uint8)
            ms = list(ex.map(lambda ab: map_reads(ix, *_slice_reads(s, off, *ab), p, keep), shards))
        m = dict(taxon=np.concatenate([x["taxon"] for x in ms]),
                 locs=np.concatenate([x["locs"] for x in ms]),
                 nloc=np.concatenate([x["nloc"] for x in ms]),
                 multi=np.concatenate([x["multi"] for x in ms]),
                 U=np.sum([x["U"] for x in ms], axis=0, dtype=np.uint64))
    a = abundance(m["U"], m["multi"], p["top_n"], p["abund_cutoff"])
    m.update(genome_hits=hits, keep=keep, abundance=a)
    return m


def gather_genomes(genomes_seq, genomes_off, ids):
    """The bytes and offsets of the genomes ``ids`` (in that order), concatenated."""
    seq = _u8(genomes_seq)
    off = np.asarray(genomes_off, dtype=np.uint64)
    ids = np.asarray(ids, dtype=np.int64)
    parts = [seq[int(off[g]):int(off[g + 1])] for g in ids]
    out_off = np.zeros(len(ids) + 1, np.uint64)
    out_off[1:] = np.cumsum([len(x) for x in parts]) if len(parts) else []
    return (np.concatenate(parts) if parts else np.zeros(0, np.uint8)), out_off


def partitioned_hits(batches, n_genomes: int, reads_seq, reads_off, max_occ: int, threads: int = 1):
    """Stage 1 over a database cut into batches (Methods, "Reference Database Organisation
    and Index Construction & Querying"): every batch is its own index, queried on its own,
    so its repeat filter counts occurrences within that batch only; its seed hits are counted
    per genome and mapped to global genome ids, and a genome held by several batches keeps
    its highest count. ``batches``: a list of (Index, global ids of its genomes)."""
    H = np.zeros(n_genomes, np.uint64)
    for ix, ids in batches:
        ids = np.asarray(ids, dtype=np.int64)
        h = count_hits_sharded(ix, reads_seq, reads_off, max_occ, threads)
        for l, g in enumerate(ids):
            H[g] = max(H[g], h[l])
    return H


def classify_partitioned(batches, n_genomes: int, genomes_seq, genomes_off, reads_seq, reads_off, p: dict,
                         k: int, w: int, canonical: int, threads: int = 1):
    """The pipeline over a partitioned database, in the paper's order (Fig. 1; Methods,
    "Reference Database Organisation and Index Construction & Querying"; Evaluation
    Methodology):
      1. seed hits per genome from every batch's own index, highest count per genome
         (``partitioned_hits``);
      2. the normalised cutoff over the whole database: keep g iff hits[g]/max > num/den;
      3. the subset database: a new (k, w) index over the kept genomes only, in global id
         order (``genomes_seq`` / ``genomes_off`` hold every genome, by global id);
      4. read mapping and profiling against the subset, all of whose genomes are kept;
         genome ids are reported as global ids.
    With nothing kept, no read maps and every abundance is 0."""
    s = _u8(reads_seq)
    off = np.ascontiguousarray(reads_off, dtype=np.uint64)
    n = len(off) - 1
    tn = p["top_n"]
    H = partitioned_hits(batches, n_genomes, s, off, p["max_occ"], threads)
    keep = keep_mask(H, p["cont_num"], p["cont_den"])
    kept = np.flatnonzero(keep)
    if len(kept) == 0:
        locs = np.zeros((n, tn), LOC_DTYPE)
        locs["genome"] = -1
        return dict(taxon=np.full(n, -1, np.int32), locs=locs, nloc=np.zeros(n, np.uint8),
                    multi=np.full((n, tn), -1, np.int32), U=np.zeros(n_genomes, np.uint64),
                    genome_hits=H, keep=keep, abundance=np.zeros(n_genomes), kept=kept)
    sub_seq, sub_off = gather_genomes(genomes_seq, genomes_off, kept)
    sub = Index(sub_seq, sub_off, k, w, canonical, threads=threads)
    m = classify(sub, s, off, p, threads=threads, keep=np.ones(len(kept), np.uint8))
    to_global = np.concatenate([kept.astype(np.int32), np.array([-1], np.int32)])
    taxon = to_global[m["taxon"]]          # -1 indexes the trailing -1
    locs = m["locs"].copy()
    locs["genome"] = to_global[locs["genome"]]
    multi = to_global[m["multi"]]
    U = np.zeros(n_genomes, np.uint64)
    U[kept] = m["U"]
    a = np.zeros(n_genomes, np.float64)
    a[kept] = m["abundance"]
    return dict(taxon=taxon, locs=locs, nloc=m["nloc"], multi=multi, U=U, genome_hits=H, keep=keep,
                abundance=a, kept=kept)


def _rank_key(L):
    """Rank of a location (Fig. 1, 2c; "Empirically Determined Parameters"): seeds descending,
    then genome, strand and window start ascending (one E per read, so the window start orders
    like the first diagonal)."""
    return (-int(L["seeds"]), int(L["genome"]), int(L["strand"]), int(L["wstart"]))


def merge_and_decide(loc_lists, reads_off, p: dict, n_genomes: int):
    """Per read, the location lists of several genome shards (each the shard's top_n with
    their distances, global genome ids) merged by the rank key and cut to top_n; then the
    decision and profile of a single index (reading of Fig. 1, 3a-b): accepted = distance <= E;
    taxon = genome of the first accepted location at the smallest distance; unique when one
    genome holds that distance, else multi-mapped over those genomes."""
    tn = p["top_n"]
    off = np.asarray(reads_off, dtype=np.uint64)
    n = len(off) - 1
    taxon = np.full(n, -1, np.int32)
    nloc = np.zeros(n, np.uint8)
    locs = np.zeros((n, tn), LOC_DTYPE)
    locs["genome"] = -1
    multi = np.full((n, tn), -1, np.int32)
    U = np.zeros(n_genomes, np.uint64)
    for r in range(n):
        ln = int(off[r + 1] - off[r])
        E = (ln * p["e_permille"]) // 1000 if p["e_permille"] else p["e_abs"]
        cand = [L for lst in loc_lists for L in lst[r] if L["genome"] >= 0]
        cand.sort(key=_rank_key)
        cand = cand[:tn]
        nloc[r] = len(cand)
        for t, L in enumerate(cand):
            locs[r, t] = L
        acc = [L for L in cand if int(L["dist"]) <= E]
        if not acc:
            continue
        best = min(int(L["dist"]) for L in acc)
        S = []
        for L in cand:
            if int(L["dist"]) == best and int(L["genome"]) not in S:
                S.append(int(L["genome"]))
        taxon[r] = S[0]
        if len(S) == 1:
            U[S[0]] += 1
        else:
            multi[r, :len(S)] = S
    a = abundance(U, multi, tn, p["abund_cutoff"])
    return dict(taxon=taxon, locs=locs, nloc=nloc, multi=multi, U=U, abundance=a)


def classify_genome_sharded(shards, n_genomes: int, reads_seq, reads_off, p: dict, threads: int = 1):
    """One read batch against a database whose genomes are split over several shards (one per
    device; disjoint global ids), every shard seeing every read: stage 1 counts each shard's
    genomes with its own index, the cutoff runs over all counts; each shard maps the reads
    against its kept genomes (its own index, masked); the shards' per-read location lists are
    merged by the rank key (``merge_and_decide``) and decided once. ``shards``: a list of
    (Index, global ids of its genomes), the ids increasing within a shard (a shard ranks ties
    between genomes by its own genome order, which then is the global one)."""
    for _, ids in shards:
        if np.any(np.diff(np.asarray(ids, dtype=np.int64)) <= 0):
            raise OracleError("genome ids of a shard must increase")
    s = _u8(reads_seq)
    off = np.ascontiguousarray(reads_off, dtype=np.uint64)
    H = np.zeros(n_genomes, np.uint64)
    for ix, ids in shards:
        H[np.asarray(ids, dtype=np.int64)] += count_hits_sharded(ix, s, off, p["max_occ"], threads)
    keep = keep_mask(H, p["cont_num"], p["cont_den"])
    lists = []
    for ix, ids in shards:
        ids = np.asarray(ids, dtype=np.int64)
        m = map_subset(ix, s, off, np.arange(len(off) - 1), p, keep[ids], threads)
        g = m["locs"]["genome"]
        m["locs"]["genome"] = np.where(g >= 0, ids[np.maximum(g, 0)], -1)
        lists.append(m["locs"])
    out = merge_and_decide(lists, off, p, n_genomes)
    out.update(genome_hits=H, keep=keep)
    return out


def map_subset(ix: Index, reads_seq, reads_off, idx, p: dict, keep: np.ndarray, threads: int = 1):
    """Per-read results for reads ``idx`` only, under a given kept-genome mask (used to
    check sampled reads of a large batch)."""
    idx = np.asarray(idx, dtype=np.int64)
    lens = (np.asarray(reads_off)[idx + 1] - np.asarray(reads_off)[idx]).astype(np.int64)
    off = np.zeros(len(idx) + 1, np.uint64)
    off[1:] = np.cumsum(lens)
    seq = np.concatenate([reads_seq[int(reads_off[i]):int(reads_off[i + 1])] for i in idx]) \
        if len(idx) else np.zeros(0, np.uint8)
    shards = _shards(len(idx), threads)
    if threads <= 1 or len(shards) <= 1:
        return map_reads(ix, seq, off, p, keep)
    with ThreadPoolExecutor(len(shards)) as ex:
        ms = list(ex.map(lambda ab: map_reads(ix, *_slice_reads(seq, off, *ab), p, keep), shards))
    return dict(taxon=np.concatenate([x["taxon"] for x in ms]),
                locs=np.concatenate([x["locs"] for x in ms]),
                nloc=np.concatenate([x["nloc"] for x in ms]),
                multi=np.concatenate([x["multi"] for x in ms]),
                U=np.sum([x["U"] for x in ms], axis=0, dtype=np.uint64))


def count_hits_sharded(ix: Index, reads_seq, reads_off, max_occ: int, threads: int = 1):
    s = _u8(reads_seq)
    off = np.ascontiguousarray(reads_off, dtype=np.uint64)
    shards = _shards(len(off) - 1, threads)
    if threads <= 1 or len(shards) <= 1:
        return count_hits(ix, s, off, max_occ)
    with ThreadPoolExecutor(len(shards)) as ex:
        parts = list(ex.map(lambda ab: count_hits(ix, *_slice_reads(s, off, *ab), max_occ), shards))
    return np.sum(parts, axis=0, dtype=np.uint64)


_CODE = np.full(256, 255, np.uint8)
for _i, _b in enumerate(b"ACGT"):
    _CODE[_b] = _i


def _codes_pair(read, window, E: int, obstacles=None):
    r = _CODE[_u8(read)]
    W = _CODE[_u8(window)].copy()
    if (r == 255).any() or (W == 255).any():
        raise OracleError("non-ACGT base")
    if len(W) != len(r) + 2 * E:
        raise OracleError("window length must be read length + 2E")
    if obstacles is not None:
        W[np.asarray(obstacles, dtype=bool)] = 4
    return np.ascontiguousarray(r), np.ascontiguousarray(W)


def approx(read, window, E: int, algo: int = 0, obstacles=None) -> int:
    """Approximation ``algo`` (see ALGOS) of one pair, as ``eda``."""
    r, W = _codes_pair(read, window, E, obstacles)
    return int(_L().or_approx_codes(algo, _p(r), len(r), _p(W), E))


def qgram_q(read, window, E: int, q: int, obstacles=None) -> int:
    """The q-gram estimate for any q in [1, 8] (the pipeline uses q = 5)."""
    r, W = _codes_pair(read, window, E, obstacles)
    return int(_L().or_qgram_q(_p(r), len(r), _p(W), E, q))


def eda(read, window, E: int, obstacles=None) -> int:
    """SneakySnake approximation of one pair. ``window`` has len(read) + 2E bases;
    ``obstacles`` (bool array over the window) marks bases outside the genome."""
    r, W = _codes_pair(read, window, E, obstacles)
    return int(_L().or_eda_codes(_p(r), len(r), _p(W), E))


def eda_batch(pairs, idx=None, threads: int = 1, algo: int = 0) -> np.ndarray:
    """Distances (approximation ``algo``) for a read-versus-window pair set
    (``gen.EdaPairs``), optionally only for the pairs ``idx``."""
    if idx is None:
        n = pairs.n_pairs
        win_seq, win_off = pairs.win_seq, pairs.win_off
        pr, E = pairs.pair_read, pairs.E
    else:
        idx = np.asarray(idx, dtype=np.int64)
        lens = (pairs.win_off[idx + 1] - pairs.win_off[idx]).astype(np.int64)
        win_off = np.zeros(len(idx) + 1, np.uint64)
        win_off[1:] = np.cumsum(lens)
        win_seq = np.concatenate([pairs.win_seq[int(pairs.win_off[i]):int(pairs.win_off[i + 1])]
                                  for i in idx]) if len(idx) else np.zeros(0, np.uint8)
        pr, E = pairs.pair_read[idx], pairs.E[idx]
        n = len(idx)
    pr = np.ascontiguousarray(pr, dtype=np.uint32)
    E = np.ascontiguousarray(E, dtype=np.uint16)
    dist = np.zeros(n, np.uint8)
    rs = np.ascontiguousarray(pairs.read_seq, dtype=np.uint8)
    ro = np.ascontiguousarray(pairs.read_off, dtype=np.uint64)

    def run(ab):
        a, b = ab
        wo = np.ascontiguousarray(win_off[a:b + 1] - win_off[a])
        ws = np.ascontiguousarray(win_seq[int(win_off[a]):int(win_off[b])])
        out = np.zeros(b - a, np.uint8)
        _L().or_eda_batch(_p(rs), _p(ro), _p(ws), _p(wo), _p(np.ascontiguousarray(pr[a:b])),
                          _p(np.ascontiguousarray(E[a:b])), b - a, algo, _p(out))
        dist[a:b] = out

    shards = _shards(n, threads) if n else []
    if threads <= 1 or len(shards) <= 1:
        for sh in shards:
            run(sh)
    else:
        with ThreadPoolExecutor(len(shards)) as ex:
            list(ex.map(run, shards))
    return dist


def rollup(abundance, genome_node, parent) -> np.ndarray:
    """Taxon abundances: each taxon sums the genomes in its subtree."""
    a = np.ascontiguousarray(abundance, dtype=np.float64)
    gn = np.ascontiguousarray(genome_node, dtype=np.uint32)
    par = np.ascontiguousarray(parent, dtype=np.int32)
    out = np.zeros(len(par), np.float64)
    rc = _L().or_rollup(_p(a), len(a), _p(gn), _p(par), len(par), _p(out))
    if rc != 0:
        raise OracleError("or_rollup failed: %d" % rc)
    return out
