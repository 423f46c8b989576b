"""GB300-native MetaTrinity hot path: Python binding of the C ABI in include/mt.h.

This module only marshals arguments: numpy arrays or torch tensors in, raw pointers and
sizes to ``libmt.so``, results back as arrays. Every step of the method runs in the CUDA
kernels of the library; there is no CPU fallback. If the library has not been built, every
call raises.

    ix = Index(genome_bytes, genome_offsets, k=21, w=11, canonical=1)
    out = classify(ix, reads, offsets, e_abs=8, min_seeds=3)     # host or CUDA tensors
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmt.so")
_lib = None

MT_OK, MT_EINVAL, MT_ENOMEM, MT_ETIMEDOUT, MT_ECUDA, MT_ECANCELED, MT_EBUSY = 0, -1, -2, -3, -4, -5, -6
MT_EXCHANGE = -7
MT_EIO = -8
MT_INDEX_HPC = 1
MT_XCHG_GENOME_HITS, MT_XCHG_UNIQUE, MT_XCHG_MULTI, MT_XCHG_HOLDERS, MT_XCHG_LOCATIONS = 0, 1, 2, 3, 4
# mt_allreduce_fn: int (*)(void *ctx, int kind, void *buf, uint64_t count)
AllreduceFn = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64)
# mt_allgather_fn: int (*)(void *ctx, int kind, const void *send, uint64_t bytes, void *recv)
AllgatherFn = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64,
                               ctypes.c_void_p)
MT_EDA_BATCHED, MT_EDA_PLAIN = 0, 1
# approximations, OR-ed into eda_mode / mode with a form
MT_EDA_SNAKE, MT_EDA_HAMMING, MT_EDA_BASE_COUNTING, MT_EDA_QGRAM, MT_EDA_SHD = 0x00, 0x10, 0x20, 0x30, 0x40
EDA_ALGOS = {"sneakysnake": MT_EDA_SNAKE, "hamming": MT_EDA_HAMMING, "base_counting": MT_EDA_BASE_COUNTING,
             "qgram": MT_EDA_QGRAM, "shd": MT_EDA_SHD}
MAX_READ_LEN, MAX_E, MAX_TOPN = 1024, 127, 8

LOC_DTYPE = np.dtype({"names": ["wstart", "genome", "seeds", "strand", "dist"],
                      "formats": [np.int64, np.int32, np.uint32, np.uint8, np.uint8],
                      "offsets": [0, 8, 12, 16, 17], "itemsize": 24})


class MtError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = "%s failed: %s (%d)" % (what, _strerror(status), status)
        if status == MT_ECUDA:
            msg += ": " + lib().mt_last_cuda_error().decode()
        super().__init__(msg)


class IndexParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint32), ("w", ctypes.c_uint32), ("canonical", ctypes.c_uint32),
                ("flags", ctypes.c_uint32)]


class ClassifyParams(ctypes.Structure):
    _fields_ = [("e_abs", ctypes.c_uint32), ("e_permille", ctypes.c_uint32),
                ("min_seeds", ctypes.c_uint32), ("top_n", ctypes.c_uint32),
                ("max_occ", ctypes.c_uint32), ("cont_num", ctypes.c_uint32),
                ("cont_den", ctypes.c_uint32), ("eda_mode", ctypes.c_uint32),
                ("abund_cutoff", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ("n_reads", "n_minimizers", "n_hits", "n_candidates", "n_accepted", "n_multi",
                 "n_fallback", "workspace_bytes", "n_ext_occ", "n_stored", "n_launches")] + \
               [(n, ctypes.c_double) for n in ("ms_seed", "ms_select", "ms_eda", "ms_profile", "ms_total")] + \
               [("err_bits", ctypes.c_uint64)]

    def as_dict(self):
        return {n: (float(getattr(self, n)) if n.startswith("ms_") else int(getattr(self, n)))
                for n, _ in self._fields_}


class EdaShape(ctypes.Structure):
    """``mt_eda_shape``: the batched approximation kernel's shape for one edit-threshold class."""
    _fields_ = [("lanes_per_pair", ctypes.c_uint32), ("pairs_per_chunk", ctypes.c_uint32),
                ("cta_threads", ctypes.c_uint32), ("refill", ctypes.c_uint32), ("tuned", ctypes.c_uint32)]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


EDA_CLASSES = 8


class IndexInfo(ctypes.Structure):
    _fields_ = [("n_genomes", ctypes.c_uint32), ("k", ctypes.c_uint32), ("w", ctypes.c_uint32),
                ("canonical", ctypes.c_uint32), ("total_bases", ctypes.c_uint64),
                ("n_occ", ctypes.c_uint64), ("n_keys", ctypes.c_uint64),
                ("table_slots", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("flags", ctypes.c_uint32), ("pad", ctypes.c_uint32)]


EXPORTS = ["mt_strerror", "mt_last_cuda_error", "mt_version", "mt_build_index", "mt_build_index_subset", "mt_free_index",
           "mt_save_index", "mt_load_index", "mt_profile_rollup",
           "mt_index_get_info", "mt_classify", "mt_classify_sharded", "mt_containment", "mt_classify_masked", "mt_classify_workspace_bytes", "mt_pack_seqs",
           "mt_eda_batch", "mt_eda_batch_noalloc", "mt_plan_create", "mt_plan_classify",
           "mt_plan_device_bytes", "mt_plan_destroy", "mt_server_create", "mt_server_submit", "mt_server_poll",
           "mt_server_cancel", "mt_server_destroy", "mt_part_create", "mt_part_contain", "mt_part_contain_batches", "mt_part_subset",
           "mt_part_classify", "mt_part_destroy", "mt_classify_partitioned", "mt_classify_genome_sharded",
           "mt_inject_alloc_failure", "mt_pool_used_bytes", "mt_classify_autotune", "mt_eda_batch_autotune",
           "mt_eda_shape_for", "mt_eda_set_shape", "mt_profile_rollup_device"]


def lib():
    """The loaded CUDA library. Raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmt.so is not built: run __graft_entry__.build() "
                               "(paper_2311_02029_gb300._build.build()) first")
        L = ctypes.CDLL(LIB_PATH)
        vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        L.mt_strerror.restype = ctypes.c_char_p
        L.mt_strerror.argtypes = [i32]
        L.mt_last_cuda_error.restype = ctypes.c_char_p
        L.mt_version.restype = i32
        L.mt_inject_alloc_failure.restype = None
        L.mt_inject_alloc_failure.argtypes = [ctypes.c_int64]
        L.mt_pool_used_bytes.restype = u64
        L.mt_pool_used_bytes.argtypes = []
        L.mt_build_index.restype = i32
        L.mt_build_index.argtypes = [vp, vp, u32, ctypes.POINTER(IndexParams), vp, ctypes.POINTER(vp)]
        L.mt_build_index_subset.restype = i32
        L.mt_build_index_subset.argtypes = [vp, vp, u32, vp, u32, ctypes.POINTER(IndexParams), vp, ctypes.POINTER(vp)]
        L.mt_free_index.argtypes = [vp]
        L.mt_profile_rollup.restype = i32
        L.mt_profile_rollup.argtypes = [vp, u32, vp, vp, u32, vp]
        L.mt_profile_rollup_device.restype = i32
        L.mt_profile_rollup_device.argtypes = [vp, u32, vp, vp, u32, vp, vp]
        L.mt_save_index.restype = i32
        L.mt_save_index.argtypes = [vp, ctypes.c_char_p, vp]
        L.mt_load_index.restype = i32
        L.mt_load_index.argtypes = [ctypes.c_char_p, vp, ctypes.POINTER(vp)]
        L.mt_index_get_info.restype = i32
        L.mt_index_get_info.argtypes = [vp, ctypes.POINTER(IndexInfo)]
        L.mt_classify.restype = i32
        L.mt_classify.argtypes = [vp, vp, u64, vp, u64, ctypes.POINTER(ClassifyParams), i32, vp,
                                  vp, vp, vp, vp, vp, ctypes.POINTER(Stats)]
        L.mt_containment.restype = i32
        L.mt_containment.argtypes = [vp, vp, u64, vp, u64, u32, u32, u32, i32, vp, vp, vp]
        L.mt_classify_autotune.restype = i32
        L.mt_classify_autotune.argtypes = [vp, vp, u64, vp, u64, ctypes.POINTER(ClassifyParams), i32, vp,
                                           vp, vp, vp, vp, vp, ctypes.POINTER(Stats), ctypes.POINTER(EdaShape)]
        L.mt_eda_batch_autotune.restype = i32
        L.mt_eda_batch_autotune.argtypes = [vp, vp, u64, vp, vp, vp, vp, u64, u32, vp, vp, vp]
        L.mt_eda_shape_for.restype = i32
        L.mt_eda_shape_for.argtypes = [u32, i32, u32, ctypes.POINTER(EdaShape)]
        L.mt_eda_set_shape.restype = i32
        L.mt_eda_set_shape.argtypes = [u32, i32, u32, ctypes.POINTER(EdaShape)]
        L.mt_classify_masked.restype = i32
        L.mt_classify_masked.argtypes = [vp, vp, u64, vp, u64, ctypes.POINTER(ClassifyParams), i32, vp,
                                         vp, vp, vp, vp, vp, vp, ctypes.POINTER(Stats)]
        L.mt_classify_sharded.restype = i32
        L.mt_classify_sharded.argtypes = [vp, vp, u64, vp, u64, ctypes.POINTER(ClassifyParams), i32, vp,
                                          AllreduceFn, vp, vp, vp, vp, vp, vp, ctypes.POINTER(Stats)]
        L.mt_classify_workspace_bytes.restype = u64
        L.mt_classify_workspace_bytes.argtypes = [vp, u64, u64, u32, ctypes.POINTER(ClassifyParams)]
        L.mt_pack_seqs.restype = i32
        L.mt_pack_seqs.argtypes = [vp, vp, u64, vp, vp]
        L.mt_eda_batch.restype = i32
        L.mt_eda_batch.argtypes = [vp, vp, u64, vp, vp, vp, vp, u64, u32, vp, vp]
        L.mt_eda_batch_noalloc.restype = i32
        L.mt_eda_batch_noalloc.argtypes = [vp, vp, u64, vp, vp, vp, vp, u64, u32, vp, vp]
        L.mt_plan_create.restype = i32
        L.mt_plan_create.argtypes = [vp, ctypes.POINTER(ClassifyParams), u64, u64, u32, ctypes.POINTER(vp)]
        L.mt_plan_classify.restype = i32
        L.mt_plan_classify.argtypes = [vp, vp, u64, vp, u64, i32, vp, vp, vp, vp, vp, vp, ctypes.POINTER(Stats)]
        L.mt_plan_device_bytes.restype = u64
        L.mt_plan_device_bytes.argtypes = [vp]
        L.mt_plan_destroy.argtypes = [vp]
        L.mt_server_create.restype = i32
        L.mt_server_create.argtypes = [vp, u64, i32, ctypes.POINTER(ClassifyParams), ctypes.POINTER(vp)]
        L.mt_server_submit.restype = i32
        L.mt_server_submit.argtypes = [vp, vp, u64, vp, u64, vp, vp, vp, vp, vp, ctypes.POINTER(u64)]
        L.mt_server_poll.restype = i32
        L.mt_server_poll.argtypes = [vp, u64, i32, ctypes.POINTER(ctypes.c_double)]
        L.mt_server_cancel.restype = i32
        L.mt_server_cancel.argtypes = [vp, u64]
        L.mt_server_destroy.argtypes = [vp]
        L.mt_part_create.restype = i32
        L.mt_part_create.argtypes = [u32, vp, u64, vp, u64, i32, vp, ctypes.POINTER(vp)]
        L.mt_part_contain.restype = i32
        L.mt_part_contain.argtypes = [vp, vp, vp, u32]
        L.mt_part_contain_batches.restype = i32
        L.mt_part_contain_batches.argtypes = [vp, vp, vp, u32, u32]
        L.mt_part_subset.restype = i32
        L.mt_part_subset.argtypes = [vp, u32, u32, vp, vp, vp, ctypes.POINTER(u32)]
        L.mt_part_classify.restype = i32
        L.mt_part_classify.argtypes = [vp, vp, vp, u32, ctypes.POINTER(ClassifyParams), vp, vp, vp, vp,
                                       ctypes.POINTER(Stats)]
        L.mt_part_destroy.argtypes = [vp]
        L.mt_classify_genome_sharded.restype = i32
        L.mt_classify_genome_sharded.argtypes = [vp, vp, u32, u32, vp, u64, vp, u64, ctypes.POINTER(ClassifyParams),
                                                 i32, vp, AllreduceFn, AllgatherFn, vp, vp, vp, vp, vp, vp,
                                                 ctypes.POINTER(Stats)]
        L.mt_classify_partitioned.restype = i32
        L.mt_classify_partitioned.argtypes = [vp, vp, u32, vp, vp, u32, ctypes.POINTER(IndexParams), vp, u64, vp,
                                              u64, ctypes.POINTER(ClassifyParams), i32, vp, vp, vp, vp, vp, vp,
                                              ctypes.POINTER(Stats)]
        _lib = L
    return _lib


def _strerror(status: int) -> str:
    try:
        return lib().mt_strerror(status).decode()
    except Exception:  # pragma: no cover
        return "status %d" % status


def _check(rc: int, what: str):
    if rc != MT_OK:
        raise MtError(rc, what)


# ---- pointer helpers -----------------------------------------------------------------------
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        assert x.is_contiguous(), "tensors passed to the library must be contiguous"
        return ctypes.c_void_p(x.data_ptr())
    assert isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
    return ctypes.c_void_p(x.ctypes.data)


def _stream(stream):
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _host_u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray)):
        return np.frombuffer(bytes(a), np.uint8)
    if _is_torch(a):
        a = a.numpy()
    return np.ascontiguousarray(a, dtype=np.uint8)


def _host_u64(a) -> np.ndarray:
    if _is_torch(a):
        a = a.numpy()
    return np.ascontiguousarray(a, dtype=np.uint64)


# ---- index --------------------------------------------------------------------------------------
class Index:
    """Device-resident reference index (``mt_build_index``). Genomes are host bytes."""

    def __init__(self, genomes, offsets, k: int, w: int, canonical: int = 1, stream=None, hpc: bool = False):
        """``hpc``: index the homopolymer-compressed genomes (a containment index)."""
        g = _host_u8(genomes)
        off = _host_u64(offsets)
        self.n_genomes = len(off) - 1
        p = IndexParams(k, w, canonical, MT_INDEX_HPC if hpc else 0)
        h = ctypes.c_void_p()
        _check(lib().mt_build_index(_ptr(g), _ptr(off), self.n_genomes, ctypes.byref(p),
                                    _stream(stream), ctypes.byref(h)), "mt_build_index")
        self._h = h

    @classmethod
    def subset(cls, genomes, offsets, ids, k: int, w: int, canonical: int = 1, stream=None, hpc: bool = False):
        """``mt_build_index_subset``: an index over the genomes ``ids`` of a host genome set, in
        that order, without a host-side copy of them."""
        g = _host_u8(genomes)
        off = _host_u64(offsets)
        sel = np.ascontiguousarray(ids, dtype=np.uint32)
        p = IndexParams(k, w, canonical, MT_INDEX_HPC if hpc else 0)
        h = ctypes.c_void_p()
        _check(lib().mt_build_index_subset(_ptr(g), _ptr(off), len(off) - 1, _ptr(sel), len(sel), ctypes.byref(p),
                                           _stream(stream), ctypes.byref(h)), "mt_build_index_subset")
        ix = cls.__new__(cls)
        ix._h = h
        ix.n_genomes = len(sel)
        return ix

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = IndexInfo()
        _check(lib().mt_index_get_info(self._h, ctypes.byref(inf)), "mt_index_get_info")
        return {n: int(getattr(inf, n)) for n, _ in inf._fields_}

    def save(self, path: str, stream=None):
        """``mt_save_index``: write this index to ``path``."""
        _check(lib().mt_save_index(self._h, os.fsencode(path), _stream(stream)), "mt_save_index")

    @classmethod
    def load(cls, path: str, stream=None) -> "Index":
        """``mt_load_index``: an index read from a file written by ``save``."""
        h = ctypes.c_void_p()
        _check(lib().mt_load_index(os.fsencode(path), _stream(stream), ctypes.byref(h)), "mt_load_index")
        ix = cls.__new__(cls)
        ix._h = h
        ix.n_genomes = ix.info()["n_genomes"]
        return ix

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().mt_free_index(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def classify_params(e_abs=0, e_permille=100, min_seeds=3, top_n=3, max_occ=1024, cont_num=1,
                    cont_den=10000, eda_mode=MT_EDA_BATCHED, abund_cutoff=1e-4) -> ClassifyParams:
    return ClassifyParams(e_abs, e_permille, min_seeds, top_n, max_occ, cont_num, cont_den, eda_mode,
                          abund_cutoff)


def _classify(ix: Index, reads, offsets, cb, stream, want_locs, out, params, keep=None, tune=False) -> dict:
    """Marshalling shared by ``classify``, ``classify_sharded`` (cb: an AllreduceFn),
    ``classify_masked`` (keep: the genome mask) and ``classify_autotune`` (tune)."""
    p = classify_params(**params)
    st = Stats()
    shape = EdaShape()
    G = ix.n_genomes

    def call(rptr, nb, optr, n_reads, dev):
        L = lib()
        if tune:
            return L.mt_classify_autotune(ix.handle, rptr, nb, optr, n_reads, ctypes.byref(p), dev, _stream(stream),
                                          _ptr(out["taxon"]), _ptr(out["nloc"]), _ptr(out["locs"]),
                                          _ptr(out["genome_hits"]), _ptr(out["abundance"]), ctypes.byref(st),
                                          ctypes.byref(shape))
        if keep is not None:
            k = keep if dev else np.ascontiguousarray(_as_host(keep), dtype=np.uint8)
            return L.mt_classify_masked(ix.handle, rptr, nb, optr, n_reads, ctypes.byref(p), dev, _stream(stream),
                                        _ptr(k), _ptr(out["taxon"]), _ptr(out["nloc"]), _ptr(out["locs"]),
                                        _ptr(out["genome_hits"]), _ptr(out["abundance"]), ctypes.byref(st))
        if cb is None:
            return L.mt_classify(ix.handle, rptr, nb, optr, n_reads, ctypes.byref(p), dev, _stream(stream),
                                 _ptr(out["taxon"]), _ptr(out["nloc"]), _ptr(out["locs"]),
                                 _ptr(out["genome_hits"]), _ptr(out["abundance"]), ctypes.byref(st))
        return L.mt_classify_sharded(ix.handle, rptr, nb, optr, n_reads, ctypes.byref(p), dev, _stream(stream),
                                     cb, None, _ptr(out["taxon"]), _ptr(out["nloc"]), _ptr(out["locs"]),
                                     _ptr(out["genome_hits"]), _ptr(out["abundance"]), ctypes.byref(st))

    if _is_torch(reads) and reads.is_cuda:
        import torch
        dev = reads.device
        n_reads = offsets.numel() - 1
        out = dict(taxon=torch.empty(n_reads, dtype=torch.int32, device=dev),
                   nloc=torch.empty(n_reads, dtype=torch.uint8, device=dev),
                   locs=torch.empty((n_reads, p.top_n, 24), dtype=torch.uint8, device=dev) if want_locs else None,
                   genome_hits=torch.empty(G, dtype=torch.int64, device=dev),
                   abundance=torch.empty(G, dtype=torch.float64, device=dev))
        rc = call(_ptr(reads), reads.numel(), _ptr(offsets), n_reads, 1)
    else:
        r = _host_u8(reads)
        off = _host_u64(offsets)
        n_reads = len(off) - 1
        if out is None:
            out = dict(taxon=np.empty(n_reads, np.int32), nloc=np.empty(n_reads, np.uint8),
                       locs=np.empty((n_reads, p.top_n), LOC_DTYPE) if want_locs else None,
                       genome_hits=np.empty(G, np.uint64), abundance=np.empty(G, np.float64))
        else:
            out = dict(out)
        rc = call(_ptr(r), len(r), _ptr(off), n_reads, 0)
    _check(rc, "mt_classify_autotune" if tune else
           ("mt_classify_masked" if keep is not None else ("mt_classify" if cb is None else "mt_classify_sharded")))
    out["stats"] = st.as_dict()
    if tune:
        out["eda_shape"] = shape.as_dict()
    return out


def classify(ix: Index, reads, offsets, *, stream=None, want_locs=True, out=None, **params) -> dict:
    """``mt_classify`` over one read batch. ``reads``/``offsets`` are either host arrays
    (results come back as numpy arrays) or CUDA tensors (results are CUDA tensors).
    ``out`` may hold preallocated host output arrays (e.g. in pinned memory)."""
    return _classify(ix, reads, offsets, None, stream, want_locs, out, params)


def classify_autotune(ix: Index, reads, offsets, *, stream=None, want_locs=True, out=None, **params) -> dict:
    """``mt_classify_autotune``: ``classify`` that first times the batched approximation kernel's
    shapes on this batch's candidates and keeps the fastest for later calls on this device; the
    result also holds ``eda_shape`` (the shape used)."""
    return _classify(ix, reads, offsets, None, stream, want_locs, out, params, tune=True)


def eda_shape_for(mode: int, classification: bool, E: int) -> dict:
    """``mt_eda_shape_for``: the batched approximation kernel's shape (tuned or default) for
    approximation ``mode`` and edit threshold E, in classification or in the EDA batch call."""
    sh = EdaShape()
    _check(lib().mt_eda_shape_for(mode, 1 if classification else 0, E, ctypes.byref(sh)), "mt_eda_shape_for")
    return sh.as_dict()


def eda_set_shape(mode: int, classification: bool, E: int, lanes_per_pair: int, pairs_per_chunk: int = 128,
                  cta_threads: int = 256, refill: int = 0):
    """``mt_eda_set_shape``: keep a shape for approximation ``mode`` and E's class (e.g. one tuned
    in an earlier process); ``lanes_per_pair=0`` forgets it."""
    sh = EdaShape(lanes_per_pair, pairs_per_chunk, cta_threads, refill, 1)
    _check(lib().mt_eda_set_shape(mode, 1 if classification else 0, E, ctypes.byref(sh)), "mt_eda_set_shape")


def classify_masked(ix: Index, reads, offsets, keep, *, stream=None, want_locs=True, out=None, **params) -> dict:
    """``mt_classify_masked``: mapping and profiling over the genomes with ``keep`` != 0 (a
    uint8 array of n_genomes; a CUDA tensor when the reads are)."""
    return _classify(ix, reads, offsets, None, stream, want_locs, out, params, keep=keep)


def containment(ix: Index, reads, offsets, *, max_occ=1024, cont_num=1, cont_den=10000, stream=None) -> dict:
    """``mt_containment``: seed hits per genome and the kept-genome mask of a batch (host
    arrays, or CUDA tensors in and out)."""
    G = ix.n_genomes
    if _is_torch(reads) and reads.is_cuda:
        import torch
        hits = torch.empty(G, dtype=torch.int64, device=reads.device)
        keep = torch.empty(G, dtype=torch.uint8, device=reads.device)
        rc = lib().mt_containment(ix.handle, _ptr(reads), reads.numel(), _ptr(offsets), offsets.numel() - 1, max_occ,
                                  cont_num, cont_den, 1, _stream(stream), _ptr(hits), _ptr(keep))
    else:
        r = _host_u8(reads)
        off = _host_u64(offsets)
        hits = np.empty(G, np.uint64)
        keep = np.empty(G, np.uint8)
        rc = lib().mt_containment(ix.handle, _ptr(r), len(r), _ptr(off), len(off) - 1, max_occ, cont_num, cont_den,
                                  0, _stream(stream), _ptr(hits), _ptr(keep))
    _check(rc, "mt_containment")
    return dict(genome_hits=hits, keep=keep)


def allreduce_callback(fn) -> AllreduceFn:
    """Wraps ``fn(kind, buf)`` as an ``mt_allreduce_fn``: buf is a numpy view of the exchanged
    vector (uint64 for MT_XCHG_GENOME_HITS and MT_XCHG_UNIQUE, float64 for MT_XCHG_MULTI) that
    fn must replace in place with its element-wise sum over the ranks. An exception in fn is
    reported to the library as a failed exchange. Keep the returned object alive for the call."""
    def tramp(ctx, kind, buf, count):
        try:
            ctype = ctypes.c_double if kind == MT_XCHG_MULTI else ctypes.c_uint64
            arr = np.ctypeslib.as_array((ctype * max(int(count), 1)).from_address(buf))[:int(count)]
            fn(int(kind), arr)
            return 0
        except Exception:
            return 1
    return AllreduceFn(tramp)


def dist_allreduce(group=None):
    """An exchange function for ``allreduce_callback`` over a torch.distributed process group
    (gloo: host tensors; nccl: the current CUDA device)."""
    import torch
    import torch.distributed as dist

    def fn(kind, arr):
        t = torch.from_numpy(arr.view(np.int64) if arr.dtype == np.uint64 else arr)
        if dist.get_backend(group) == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        res = t.cpu().numpy()
        arr[...] = res.view(arr.dtype) if arr.dtype == np.uint64 else res
    return fn


def allgather_callback(fn, n_ranks: int) -> AllgatherFn:
    """Wraps ``fn(kind, send, recv)`` as an ``mt_allgather_fn``: send is a uint8 numpy view of
    this rank's buffer, recv one of n_ranks times its size that fn must fill with every rank's
    buffer in rank order. An exception in fn is reported as a failed exchange."""
    def tramp(ctx, kind, send, nbytes, recv):
        try:
            nb = int(nbytes)
            snd = np.ctypeslib.as_array((ctypes.c_uint8 * max(nb, 1)).from_address(send))[:nb]
            rcv = np.ctypeslib.as_array((ctypes.c_uint8 * max(nb * n_ranks, 1)).from_address(recv))[:nb * n_ranks]
            fn(int(kind), snd, rcv)
            return 0
        except Exception:
            return 1
    return AllgatherFn(tramp)


def dist_allgather(group=None):
    """An exchange function for ``allgather_callback`` over a torch.distributed process group
    (gloo: host tensors; nccl: the current CUDA device)."""
    import torch
    import torch.distributed as dist

    def fn(kind, send, recv):
        t = torch.from_numpy(send.copy())
        if dist.get_backend(group) == "nccl":
            t = t.cuda()
        parts = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
        dist.all_gather(parts, t, group=group)
        if len(send):
            recv[...] = torch.cat([x.cpu() for x in parts]).numpy()
    return fn


def classify_genome_sharded(shard: Index, genome_ids, n_genomes: int, n_ranks: int, reads, offsets, allreduce,
                            allgather, *, stream=None, want_locs=True, **params) -> dict:
    """``mt_classify_genome_sharded``: this rank's genome shard (global ids ``genome_ids``) against
    the whole read batch; ``allreduce(kind, buf)`` sums a vector over the ranks in place (see
    ``dist_allreduce``), ``allgather(kind, send, recv)`` gathers byte buffers (see
    ``dist_allgather``). Every rank gets the whole batch's outputs in global genome ids."""
    ids = np.ascontiguousarray(genome_ids, dtype=np.uint32)
    if len(ids) != shard.n_genomes:
        raise ValueError("one global id per genome of the shard")
    p = classify_params(**params)
    st = Stats()
    ar = allreduce_callback(allreduce)
    ag = allgather_callback(allgather, n_ranks)
    G = int(n_genomes)
    if _is_torch(reads) and reads.is_cuda:
        n_reads = offsets.numel() - 1
        out = _part_outputs(reads.device, n_reads, p.top_n, G, want_locs)
        rp, nb, op, dev = _ptr(reads), reads.numel(), _ptr(offsets), 1
    else:
        r, off = _host_u8(reads), _host_u64(offsets)
        n_reads = len(off) - 1
        out = _part_outputs(None, n_reads, p.top_n, G, want_locs)
        rp, nb, op, dev = _ptr(r), len(r), _ptr(off), 0
    _check(lib().mt_classify_genome_sharded(shard.handle, _ptr(ids), G, n_ranks, rp, nb, op, n_reads, ctypes.byref(p),
                                            dev, _stream(stream), ar, ag, None, _ptr(out["taxon"]),
                                            _ptr(out["nloc"]), _ptr(out["locs"]), _ptr(out["genome_hits"]),
                                            _ptr(out["abundance"]), ctypes.byref(st)), "mt_classify_genome_sharded")
    out["stats"] = st.as_dict()
    return out


def classify_sharded(ix: Index, reads, offsets, allreduce, *, stream=None, want_locs=True, out=None,
                     **params) -> dict:
    """``mt_classify_sharded``: this rank's shard of one batch; ``allreduce(kind, buf)`` sums a
    vector over the ranks in place (see ``dist_allreduce``). Per-read results are those of
    ``classify`` on the whole batch for this rank's reads; genome_hits and abundance are the
    whole batch's."""
    cb = allreduce_callback(allreduce)
    return _classify(ix, reads, offsets, cb, stream, want_locs, out, params)


# ---- a reference database cut into batches ------------------------------------------------------
def split_batches(genome_offsets, n_batches: int) -> list:
    """Global genome ids cut into ``n_batches`` runs of consecutive ids holding about equal
    numbers of bases (the paper splits its database into batches of about 7 GB each); every
    batch holds at least one genome."""
    off = _host_u64(genome_offsets).astype(np.float64)
    G = len(off) - 1
    if not 1 <= n_batches <= G:
        raise ValueError("n_batches must be in 1..n_genomes")
    total = off[-1] - off[0]
    cuts = [0]
    for b in range(1, n_batches):
        # the batch ends after the first genome whose end reaches b / n_batches of the bases
        j = int(np.searchsorted(off[1:], off[0] + total * b / n_batches, side="left")) + 1
        cuts.append(min(max(j, cuts[-1] + 1), G - (n_batches - b)))
    cuts.append(G)
    return [np.arange(cuts[i], cuts[i + 1], dtype=np.uint32) for i in range(n_batches)]


def gather_genomes(genomes, genome_offsets, ids):
    """Host bytes and offsets of the genomes ``ids``, concatenated in that order (the input of
    a batch's or a subset's ``Index``)."""
    g, off = _host_u8(genomes), _host_u64(genome_offsets)
    ids = np.asarray(ids, dtype=np.int64)
    lens = (off[ids + 1] - off[ids]).astype(np.uint64) if len(ids) else np.zeros(0, np.uint64)
    out_off = np.zeros(len(ids) + 1, np.uint64)
    out_off[1:] = np.cumsum(lens)
    out = np.empty(max(int(out_off[-1]), 1), np.uint8)
    for i, gid in enumerate(ids):
        out[int(out_off[i]):int(out_off[i + 1])] = g[int(off[gid]):int(off[gid + 1])]
    return out[:int(out_off[-1])], out_off


def _part_outputs(dev, n_reads, top_n, G, want_locs):
    if dev is not None:
        import torch
        return dict(taxon=torch.empty(n_reads, dtype=torch.int32, device=dev),
                    nloc=torch.empty(n_reads, dtype=torch.uint8, device=dev),
                    locs=torch.empty((n_reads, top_n, 24), dtype=torch.uint8, device=dev) if want_locs else None,
                    genome_hits=torch.empty(G, dtype=torch.int64, device=dev),
                    abundance=torch.empty(G, dtype=torch.float64, device=dev))
    return dict(taxon=np.empty(n_reads, np.int32), nloc=np.empty(n_reads, np.uint8),
                locs=np.empty((n_reads, top_n), LOC_DTYPE) if want_locs else None,
                genome_hits=np.empty(G, np.uint64), abundance=np.empty(G, np.float64))


class PartitionedQuery:
    """``mt_part_*``: one read batch queried against a database cut into batches. Call
    ``contain`` once per database batch (an Index and the global ids of its genomes), then
    ``subset`` (the cutoff; returns the kept ids), build an Index over the kept genomes in
    that order, and ``classify`` against it. Reads are host arrays or CUDA tensors (then kept
    referenced until ``close``)."""

    def __init__(self, n_genomes: int, reads, offsets, stream=None):
        self.n_genomes = int(n_genomes)
        self._stream = stream
        self._dev = reads.device if (_is_torch(reads) and reads.is_cuda) else None
        h = ctypes.c_void_p()
        if self._dev is not None:
            self._keep = (reads, offsets)
            self.n_reads = offsets.numel() - 1
            rc = lib().mt_part_create(self.n_genomes, _ptr(reads), reads.numel(), _ptr(offsets), self.n_reads, 1,
                                      _stream(stream), ctypes.byref(h))
        else:
            r, off = _host_u8(reads), _host_u64(offsets)
            self.n_reads = len(off) - 1
            rc = lib().mt_part_create(self.n_genomes, _ptr(r), len(r), _ptr(off), self.n_reads, 0,
                                      _stream(stream), ctypes.byref(h))
        _check(rc, "mt_part_create")
        self._h = h
        self.kept = None

    def contain(self, batch: Index, genome_ids, max_occ: int = 1024):
        ids = np.ascontiguousarray(genome_ids, dtype=np.uint32)
        if len(ids) != batch.n_genomes:
            raise ValueError("one global id per genome of the batch")
        _check(lib().mt_part_contain(self._h, batch.handle, _ptr(ids), max_occ), "mt_part_contain")

    def contain_batches(self, batches, genome_ids, max_occ: int = 1024):
        """``mt_part_contain_batches``: several resident batches (same seeds) in one pass."""
        if len(batches) != len(genome_ids):
            raise ValueError("one id list per batch")
        ids = [np.ascontiguousarray(x, dtype=np.uint32) for x in genome_ids]
        for ix, x in zip(batches, ids):
            if len(x) != ix.n_genomes:
                raise ValueError("one global id per genome of each batch")
        B = len(batches)
        hv = (ctypes.c_void_p * max(B, 1))(*[ix.handle.value for ix in batches])
        iv = (ctypes.c_void_p * max(B, 1))(*[x.ctypes.data for x in ids])
        _check(lib().mt_part_contain_batches(self._h, hv, iv, B, max_occ), "mt_part_contain_batches")

    def subset(self, cont_num: int = 1, cont_den: int = 10000) -> dict:
        G = self.n_genomes
        keep = np.empty(G, np.uint8)
        kept = np.empty(G, np.uint32)
        nk = ctypes.c_uint32()
        hits = _part_outputs(self._dev, 0, 1, G, False)["genome_hits"]
        _check(lib().mt_part_subset(self._h, cont_num, cont_den, _ptr(keep), _ptr(hits), _ptr(kept), ctypes.byref(nk)),
               "mt_part_subset")
        self.kept = kept[:nk.value].copy()
        return dict(keep=keep, genome_hits=hits, kept=self.kept)

    def classify(self, subset: Index | None, *, want_locs=True, **params) -> dict:
        p = classify_params(**params)
        st = Stats()
        ids = self.kept if self.kept is not None else np.zeros(0, np.uint32)
        out = _part_outputs(self._dev, self.n_reads, p.top_n, self.n_genomes, want_locs)
        del out["genome_hits"]
        _check(lib().mt_part_classify(self._h, subset.handle if subset is not None else None, _ptr(ids), len(ids),
                                      ctypes.byref(p), _ptr(out["taxon"]), _ptr(out["nloc"]), _ptr(out["locs"]),
                                      _ptr(out["abundance"]), ctypes.byref(st)), "mt_part_classify")
        out["stats"] = st.as_dict()
        return out

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().mt_part_destroy(self._h)
            self._h = ctypes.c_void_p()
        self._keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def classify_partitioned(batches, genome_ids, genomes, genome_offsets, reads, offsets, *, k: int, w: int,
                         canonical: int = 1, stream=None, want_locs=True, **params) -> dict:
    """``mt_classify_partitioned``: the whole query over resident database batches
    (``batches[b]`` an Index whose genomes have global ids ``genome_ids[b]``); ``genomes`` /
    ``genome_offsets`` (host) hold every genome by global id, for the subset index (k, w,
    canonical)."""
    if len(batches) != len(genome_ids):
        raise ValueError("one id list per batch")
    ids = [np.ascontiguousarray(x, dtype=np.uint32) for x in genome_ids]
    for ix, x in zip(batches, ids):
        if len(x) != ix.n_genomes:
            raise ValueError("one global id per genome of each batch")
    B = len(batches)
    hv = (ctypes.c_void_p * max(B, 1))(*[ix.handle.value for ix in batches])
    iv = (ctypes.c_void_p * max(B, 1))(*[x.ctypes.data for x in ids])
    g, goff = _host_u8(genomes), _host_u64(genome_offsets)
    G = len(goff) - 1
    sp = IndexParams(k, w, canonical, 0)
    p = classify_params(**params)
    st = Stats()
    if _is_torch(reads) and reads.is_cuda:
        n_reads = offsets.numel() - 1
        out = _part_outputs(reads.device, n_reads, p.top_n, G, want_locs)
        rp, nb, op, dev = _ptr(reads), reads.numel(), _ptr(offsets), 1
    else:
        r, off = _host_u8(reads), _host_u64(offsets)
        n_reads = len(off) - 1
        out = _part_outputs(None, n_reads, p.top_n, G, want_locs)
        rp, nb, op, dev = _ptr(r), len(r), _ptr(off), 0
    _check(lib().mt_classify_partitioned(hv, iv, B, _ptr(g), _ptr(goff), G, ctypes.byref(sp), rp, nb, op, n_reads,
                                         ctypes.byref(p), dev, _stream(stream), _ptr(out["taxon"]), _ptr(out["nloc"]),
                                         _ptr(out["locs"]), _ptr(out["genome_hits"]), _ptr(out["abundance"]),
                                         ctypes.byref(st)), "mt_classify_partitioned")
    out["stats"] = st.as_dict()
    return out


class Plan:
    """Preallocated classification replayed from a captured CUDA graph (``mt_plan_*``)."""

    def __init__(self, ix: Index, max_reads: int, max_bases: int, max_read_len: int = 256, **params):
        self.ix = ix
        self.p = classify_params(**params)
        h = ctypes.c_void_p()
        _check(lib().mt_plan_create(ix.handle, ctypes.byref(self.p), max_reads, max_bases, max_read_len,
                                    ctypes.byref(h)), "mt_plan_create")
        self._h = h

    @property
    def device_bytes(self) -> int:
        return int(lib().mt_plan_device_bytes(self._h))

    def classify(self, reads, offsets, *, stream=None, want_locs=True, out=None) -> dict:
        st = Stats()
        G = self.ix.n_genomes
        tn = self.p.top_n
        if _is_torch(reads) and reads.is_cuda:
            import torch
            dev = reads.device
            n_reads = offsets.numel() - 1
            out = dict(taxon=torch.empty(n_reads, dtype=torch.int32, device=dev),
                       nloc=torch.empty(n_reads, dtype=torch.uint8, device=dev),
                       locs=torch.empty((n_reads, tn, 24), dtype=torch.uint8, device=dev) if want_locs else None,
                       genome_hits=torch.empty(G, dtype=torch.int64, device=dev),
                       abundance=torch.empty(G, dtype=torch.float64, device=dev))
            rc = lib().mt_plan_classify(self._h, _ptr(reads), reads.numel(), _ptr(offsets), n_reads, 1, _stream(stream),
                                        _ptr(out["taxon"]), _ptr(out["nloc"]), _ptr(out["locs"]),
                                        _ptr(out["genome_hits"]), _ptr(out["abundance"]), ctypes.byref(st))
        else:
            r = _host_u8(reads)
            off = _host_u64(offsets)
            n_reads = len(off) - 1
            if out is None:
                out = dict(taxon=np.empty(n_reads, np.int32), nloc=np.empty(n_reads, np.uint8),
                           locs=np.empty((n_reads, tn), LOC_DTYPE) if want_locs else None,
                           genome_hits=np.empty(G, np.uint64), abundance=np.empty(G, np.float64))
            else:
                out = dict(out)
            rc = lib().mt_plan_classify(self._h, _ptr(r), len(r), _ptr(off), n_reads, 0, _stream(stream),
                                        _ptr(out["taxon"]), _ptr(out["nloc"]), _ptr(out["locs"]),
                                        _ptr(out["genome_hits"]), _ptr(out["abundance"]), ctypes.byref(st))
        _check(rc, "mt_plan_classify")
        out["stats"] = st.as_dict()
        return out

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().mt_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def locs_from_device(t) -> np.ndarray:
    """View a (n, top_n, 24) uint8 tensor of mt_loc records as a structured numpy array."""
    a = t.cpu().numpy() if _is_torch(t) else t
    return np.ascontiguousarray(a).view(LOC_DTYPE).reshape(a.shape[0], a.shape[1])


def workspace_bytes(ix: Index, n_bases: int, n_reads: int, max_read_len: int = 0, **params) -> int:
    """Device bytes one host-buffer mt_classify call allocates (what the server charges)."""
    p = classify_params(**params)
    return int(lib().mt_classify_workspace_bytes(ix.handle, n_bases, n_reads, max_read_len, ctypes.byref(p)))


# ---- packing and the EDA stage alone -----------------------------------------------------------
def packed_words(offsets_host: np.ndarray) -> int:
    n = len(offsets_host) - 1
    return int(offsets_host[-1]) // 32 + n + 1


def pack_seqs(seq, offsets, n_words: int, stream=None):
    """``mt_pack_seqs``: CUDA uint8 bases + CUDA int64 offsets -> CUDA int64 packed words."""
    import torch
    words = torch.empty(n_words, dtype=torch.int64, device=seq.device)
    _check(lib().mt_pack_seqs(_ptr(seq), _ptr(offsets), offsets.numel() - 1, _ptr(words), _stream(stream)),
           "mt_pack_seqs")
    return words


def eda_batch(read_words, read_off, win_words, win_off, pair_read, E, mode=MT_EDA_BATCHED, stream=None):
    """``mt_eda_batch`` on CUDA tensors; returns a CUDA uint8 tensor of distances."""
    import torch
    n_pairs = pair_read.numel()
    dist = torch.empty(n_pairs, dtype=torch.uint8, device=pair_read.device)
    _check(lib().mt_eda_batch(_ptr(read_words), _ptr(read_off), read_off.numel() - 1, _ptr(win_words),
                              _ptr(win_off), _ptr(pair_read), _ptr(E), n_pairs, mode, _stream(stream),
                              _ptr(dist)), "mt_eda_batch")
    return dist


def eda_batch_autotune(read_words, read_off, win_words, win_off, pair_read, E, mode=MT_EDA_BATCHED, stream=None):
    """``mt_eda_batch_autotune``: ``eda_batch`` that first times the batched kernel's shapes on
    every edit-threshold class of this batch and keeps the fastest per class; returns
    (distances, list of the classes' shapes)."""
    import torch
    n_pairs = pair_read.numel()
    dist = torch.empty(n_pairs, dtype=torch.uint8, device=pair_read.device)
    shapes = (EdaShape * EDA_CLASSES)()
    _check(lib().mt_eda_batch_autotune(_ptr(read_words), _ptr(read_off), read_off.numel() - 1, _ptr(win_words),
                                       _ptr(win_off), _ptr(pair_read), _ptr(E), n_pairs, mode, _stream(stream),
                                       _ptr(dist), ctypes.cast(shapes, ctypes.c_void_p)), "mt_eda_batch_autotune")
    return dist, [sh.as_dict() for sh in shapes]


NOALLOC_MAX_PAIRS = 1 << 20


def eda_batch_noalloc(read_words, read_off, win_words, win_off, pair_read, E, dist, mode=MT_EDA_BATCHED,
                      stream=None):
    """``mt_eda_batch_noalloc`` on CUDA tensors into a caller-provided uint8 ``dist``. For
    callers that cannot allocate device memory during a call; the library uses a fixed
    per-device array instead, so at most 2^20 pairs per call and calls must not overlap."""
    _check(lib().mt_eda_batch_noalloc(_ptr(read_words), _ptr(read_off), read_off.numel() - 1, _ptr(win_words),
                                      _ptr(win_off), _ptr(pair_read), _ptr(E), pair_read.numel(), mode,
                                      _stream(stream), _ptr(dist)), "mt_eda_batch_noalloc")
    return dist


# ---- serving ---------------------------------------------------------------------------------------
class Server:
    """Continuous-batching request loop (``mt_server_*``) over one resident index."""

    def __init__(self, ix: Index, hbm_budget: int, max_slots: int = 4, **params):
        self.ix = ix
        self.p = classify_params(**params)
        h = ctypes.c_void_p()
        _check(lib().mt_server_create(ix.handle, hbm_budget, max_slots, ctypes.byref(self.p), ctypes.byref(h)),
               "mt_server_create")
        self._h = h
        self._keep = {}

    def submit(self, reads, offsets, out=None) -> int:
        """Queues one batch; returns its request id. ``out`` may hold caller-owned output arrays
        (taxon, nloc, locs, genome_hits, abundance) of at least this batch's size, e.g. reused
        from an earlier request, which avoids faulting in fresh pages for every request."""
        r = _host_u8(reads)
        off = _host_u64(offsets)
        n = len(off) - 1
        G = self.ix.n_genomes
        if out is None:
            out = dict(taxon=np.empty(n, np.int32), nloc=np.empty(n, np.uint8),
                       locs=np.empty((n, self.p.top_n), LOC_DTYPE), genome_hits=np.empty(G, np.uint64),
                       abundance=np.empty(G, np.float64))
        else:
            if (len(out["taxon"]) < n or len(out["nloc"]) < n or len(out["locs"]) < n
                    or len(out["genome_hits"]) < G or len(out["abundance"]) < G):
                raise ValueError("output arrays smaller than the batch")
            out = dict(taxon=out["taxon"][:n], nloc=out["nloc"][:n], locs=out["locs"][:n],
                       genome_hits=out["genome_hits"][:G], abundance=out["abundance"][:G])
            for k, dt in (("taxon", np.int32), ("nloc", np.uint8), ("genome_hits", np.uint64),
                          ("abundance", np.float64)):
                if out[k].dtype != dt or not out[k].flags["C_CONTIGUOUS"]:
                    raise ValueError("output %s must be contiguous %s" % (k, np.dtype(dt).name))
            if (out["locs"].dtype != LOC_DTYPE or not out["locs"].flags["C_CONTIGUOUS"]
                    or out["locs"].shape[1:] != (self.p.top_n,)):
                raise ValueError("output locs must be contiguous (n, top_n) locations")
        rid = ctypes.c_uint64()
        _check(lib().mt_server_submit(self._h, _ptr(r), len(r), _ptr(off), n, _ptr(out["taxon"]),
                                      _ptr(out["nloc"]), _ptr(out["locs"]), _ptr(out["genome_hits"]),
                                      _ptr(out["abundance"]), ctypes.byref(rid)), "mt_server_submit")
        self._keep[rid.value] = (r, off, out)
        return rid.value

    def poll(self, req_id: int, timeout_ms: int = 0):
        """(status, latency_s, outputs or None)."""
        lat = ctypes.c_double(0.0)
        rc = lib().mt_server_poll(self._h, req_id, timeout_ms, ctypes.byref(lat))
        if rc in (MT_EBUSY, MT_ETIMEDOUT):
            return rc, None, None
        if req_id not in self._keep:          # unknown, or released by an earlier final poll
            return rc, None, None
        _, _, out = self._keep.pop(req_id)
        return rc, lat.value, out

    def cancel(self, req_id: int) -> int:
        return lib().mt_server_cancel(self._h, req_id)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().mt_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- taxonomic profile (Fig. 1, 3b) ------------------------------------------------------------
def _as_host(x):
    return x.cpu().numpy() if _is_torch(x) else np.asarray(x)


def profile_rollup_device(abundance, genome_node, parent, stream=None):
    """``mt_profile_rollup_device``: per-taxon abundance on the device (CUDA tensors: float64
    abundance, int32 or uint32 genome nodes, int32 parents); returns a CUDA float64 tensor."""
    import torch
    out = torch.empty(parent.numel(), dtype=torch.float64, device=abundance.device)
    _check(lib().mt_profile_rollup_device(_ptr(abundance), abundance.numel(), _ptr(genome_node), _ptr(parent),
                                          parent.numel(), _ptr(out), _stream(stream)), "mt_profile_rollup_device")
    return out


def profile_rollup(abundance, genome_node, parent) -> np.ndarray:
    """``mt_profile_rollup``: per-taxon abundance (host arrays; ``abundance`` may be a tensor)."""
    a = np.ascontiguousarray(_as_host(abundance), dtype=np.float64)
    gn = np.ascontiguousarray(genome_node, dtype=np.uint32)
    par = np.ascontiguousarray(parent, dtype=np.int32)
    out = np.zeros(len(par), np.float64)
    _check(lib().mt_profile_rollup(_ptr(a), len(a), _ptr(gn), _ptr(par), len(par), _ptr(out)), "mt_profile_rollup")
    return out


def write_cami_profile(f, sample_id: str, taxonomy, node_abundance, version: str = "0.9.1"):
    """Writes a profile in the CAMI / OPAL profiling format: a header (@SampleID, @Version,
    @Ranks) and one row per taxon with non-zero abundance: TAXID, RANK, TAXPATH (taxids from
    the root), TAXPATHSN (names from the root) and PERCENTAGE. ``taxonomy`` has parent, rank,
    name, taxid and ranks (e.g. ``gen.Taxonomy``); ``f`` is a text file object."""
    par = np.asarray(taxonomy.parent)
    f.write("@SampleID:%s\n@Version:%s\n@Ranks:%s\n\n" % (sample_id, version, "|".join(taxonomy.ranks)))
    f.write("@@TAXID\tRANK\tTAXPATH\tTAXPATHSN\tPERCENTAGE\n")
    order = sorted(range(len(par)), key=lambda v: (list(taxonomy.ranks).index(taxonomy.rank[v]), v))
    for v in order:
        if node_abundance[v] <= 0.0:
            continue
        path, u = [], v
        while u != -1:
            path.append(int(u))
            u = int(par[u])
        path.reverse()
        f.write("%d\t%s\t%s\t%s\t%.6f\n" % (int(taxonomy.taxid[v]), taxonomy.rank[v],
                                                "|".join(str(int(taxonomy.taxid[u])) for u in path),
                                                "|".join(taxonomy.name[u] for u in path), 100.0 * node_abundance[v]))
