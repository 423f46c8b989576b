"""Host-side checks of the C ABI that need no GPU: the library loads, exports every entry
point declared in include/mt.h, and the binding's struct layouts match the header."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mtlib():
    from paper_2311_02029_gb300 import _build
    _build.build()
    import paper_2311_02029_gb300 as mt
    return mt


def _declared():
    src = open(os.path.join(ROOT, "include", "mt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mt_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("mt_build_index", "mt_classify", "mt_eda_batch", "mt_pack_seqs", "mt_server_create",
                 "mt_server_submit", "mt_server_poll", "mt_free_index"):
        assert must in names


def test_library_exports_every_declared_symbol(mtlib):
    L = mtlib.lib()
    for name in _declared():
        assert hasattr(L, name), "libmt.so does not export %s" % name
    assert sorted(mtlib.EXPORTS) == _declared()


def test_struct_layouts_match_header(mtlib):
    assert ctypes.sizeof(mtlib.IndexParams) == 16
    assert ctypes.sizeof(mtlib.ClassifyParams) == 40
    assert mtlib.LOC_DTYPE.itemsize == 24
    assert ctypes.sizeof(mtlib.Stats) == 136
    assert ctypes.sizeof(mtlib.IndexInfo) == 64
    assert ctypes.sizeof(mtlib.EdaShape) == 20


def test_status_strings_and_argument_checks_without_gpu(mtlib):
    L = mtlib.lib()
    assert L.mt_version() >= 1
    assert L.mt_strerror(0) == b"ok"
    assert L.mt_strerror(mtlib.MT_EINVAL)
    # argument validation happens before any CUDA call
    out = ctypes.c_void_p()
    p = mtlib.IndexParams(0, 10, 0, 0)          # k = 0 is out of range
    g = np.frombuffer(b"ACGT" * 10, np.uint8)
    off = np.array([0, 40], np.uint64)
    rc = L.mt_build_index(ctypes.c_void_p(g.ctypes.data), ctypes.c_void_p(off.ctypes.data), 1,
                          ctypes.byref(p), None, ctypes.byref(out))
    assert rc == mtlib.MT_EINVAL and not out.value
    p = mtlib.IndexParams(15, 65, 0, 0)         # w above MT_MAX_W
    assert L.mt_build_index(ctypes.c_void_p(g.ctypes.data), ctypes.c_void_p(off.ctypes.data), 1,
                            ctypes.byref(p), None, ctypes.byref(out)) == mtlib.MT_EINVAL
    assert L.mt_eda_batch(None, None, 0, None, None, None, None, 5, 7, None, None) == mtlib.MT_EINVAL
    assert L.mt_server_create(None, 1, 1, None, ctypes.byref(out)) == mtlib.MT_EINVAL
    cp = mtlib.classify_params()
    assert L.mt_classify_sharded(None, None, 0, None, 0, ctypes.byref(cp), 0, None, mtlib.AllreduceFn(), None,
                                 None, None, None, None, None, None) == mtlib.MT_EINVAL   # no allreduce
    assert L.mt_strerror(mtlib.MT_EXCHANGE) != L.mt_strerror(-99)


def test_partitioned_query_argument_checks_without_gpu(mtlib):
    L = mtlib.lib()
    out = ctypes.c_void_p()
    off = np.array([0, 4], np.uint64)
    r = np.frombuffer(b"ACGT", np.uint8)
    assert L.mt_part_create(0, ctypes.c_void_p(r.ctypes.data), 4, ctypes.c_void_p(off.ctypes.data), 1, 0, None,
                            ctypes.byref(out)) == mtlib.MT_EINVAL          # no genomes
    assert L.mt_part_create(3, None, 4, ctypes.c_void_p(off.ctypes.data), 1, 0, None,
                            ctypes.byref(out)) == mtlib.MT_EINVAL          # no reads buffer
    assert not out.value
    assert L.mt_part_contain(None, None, None, 16) == mtlib.MT_EINVAL
    assert L.mt_part_subset(None, 1, 10000, None, None, None, None) == mtlib.MT_EINVAL
    cp = mtlib.classify_params()
    assert L.mt_part_classify(None, None, None, 0, ctypes.byref(cp), None, None, None, None, None) == mtlib.MT_EINVAL
    L.mt_part_destroy(None)
    ids = np.zeros(1, np.uint32)
    assert L.mt_classify_genome_sharded(None, ctypes.c_void_p(ids.ctypes.data), 4, 2, ctypes.c_void_p(r.ctypes.data), 4,
                                        ctypes.c_void_p(off.ctypes.data), 1, ctypes.byref(cp), 0, None,
                                        mtlib.AllreduceFn(), mtlib.AllgatherFn(), None, None, None, None, None, None,
                                        None) == mtlib.MT_EINVAL   # no shard, no exchange functions
    g = np.frombuffer(b"ACGT" * 10, np.uint8)
    goff = np.array([0, 40], np.uint64)
    ip = mtlib.IndexParams(15, 10, 1, 0)
    bad = np.array([0, 1], np.uint32)                       # id 1 is not in a one-genome set
    assert L.mt_build_index_subset(ctypes.c_void_p(g.ctypes.data), ctypes.c_void_p(goff.ctypes.data), 1,
                                   ctypes.c_void_p(bad.ctypes.data), 2, ctypes.byref(ip), None,
                                   ctypes.byref(out)) == mtlib.MT_EINVAL
    assert L.mt_build_index_subset(ctypes.c_void_p(g.ctypes.data), ctypes.c_void_p(goff.ctypes.data), 1, None, 1,
                                   ctypes.byref(ip), None, ctypes.byref(out)) == mtlib.MT_EINVAL
    sp = mtlib.IndexParams(15, 10, 1, mtlib.MT_INDEX_HPC)   # a subset index must support mapping
    assert L.mt_classify_partitioned(None, None, 0, ctypes.c_void_p(g.ctypes.data), ctypes.c_void_p(goff.ctypes.data),
                                     1, ctypes.byref(sp), ctypes.c_void_p(r.ctypes.data), 4,
                                     ctypes.c_void_p(off.ctypes.data), 1, ctypes.byref(cp), 0, None, None, None,
                                     None, None, None, None) == mtlib.MT_EINVAL


@pytest.mark.parametrize("n_batches", [1, 2, 5, 25, 40])
def test_split_batches(mtlib, n_batches):
    """Consecutive ids, every genome once, no empty batch, about equal bases per batch."""
    rng = np.random.default_rng(n_batches)
    lens = rng.integers(1_000, 50_000, 40)
    off = np.concatenate([[7], 7 + np.cumsum(lens)]).astype(np.uint64)
    parts = mtlib.split_batches(off, n_batches)
    assert len(parts) == n_batches and all(len(x) > 0 for x in parts)
    assert np.array_equal(np.concatenate(parts), np.arange(40))
    sizes = [int(lens[x].sum()) for x in parts]
    if n_batches <= 5:   # each batch within one genome of its share
        assert max(sizes) - min(sizes) <= 2 * int(lens.max())
    with pytest.raises(ValueError):
        mtlib.split_batches(off, 41)


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2311_02029_gb300 as mt
    monkeypatch.setattr(mt, "_lib", None)
    monkeypatch.setattr(mt, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        mt.lib()


def test_load_index_refuses_non_index_files_without_gpu(mtlib, tmp_path):
    """The header and size checks run before any CUDA call."""
    L = mtlib.lib()
    out = ctypes.c_void_p()
    assert L.mt_load_index(str(tmp_path / "missing.idx").encode(), None, ctypes.byref(out)) == mtlib.MT_EIO
    p = tmp_path / "junk.idx"
    p.write_bytes(b"not an index" * 20)
    assert L.mt_load_index(str(p).encode(), None, ctypes.byref(out)) == mtlib.MT_EIO
    p.write_bytes(b"MTIDX\0\0\1" + bytes(200))        # right magic, bad check field
    assert L.mt_load_index(str(p).encode(), None, ctypes.byref(out)) == mtlib.MT_EIO
    assert not out.value
    assert L.mt_load_index(None, None, ctypes.byref(out)) == mtlib.MT_EINVAL


def test_gather_genomes_without_gpu(mtlib):
    """The binding's host gather of genome bytes (inputs of batch and subset indexes): ids in
    any order, repeats, empty genomes, no ids."""
    rng = np.random.default_rng(5)
    lens = rng.integers(0, 40, 12)
    lens[3] = 0
    seq = np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, int(lens.sum()))].copy()
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    for ids in ([5, 1, 3, 3, 11], [0], [], list(range(12))[::-1]):
        s, o = mtlib.gather_genomes(seq, off, ids)
        assert o.tolist() == [0] + np.cumsum([int(lens[i]) for i in ids]).tolist()
        exp = b"".join(seq[int(off[i]):int(off[i + 1])].tobytes() for i in ids)
        assert s.tobytes() == exp


def test_header_is_plain_c(mtlib, tmp_path):
    """include/mt.h compiles as strict C99 (the boundary takes no C++ or torch types) and links
    against libmt.so from a C program."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text('#include "mt.h"\n#include <stdio.h>\nint main(void) {\n'
                   '    mt_index *ix = 0;\n    printf("%d %s\\n", mt_version(), mt_strerror(MT_EINVAL));\n'
                   '    return mt_build_index(0, 0, 0, 0, 0, &ix) == MT_EINVAL && ix == 0 ? 0 : 1;\n}\n')
    exe = tmp_path / "use"
    libdir = os.path.dirname(mtlib.LIB_PATH)
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                        os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", libdir, "-lmt",
                        "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)   # argument checks only
    assert r.returncode == 0 and r.stdout.split()[0] == str(mtlib.lib().mt_version()), (r.stdout, r.stderr)


def test_every_entry_point_refuses_null_arguments_without_gpu(mtlib):
    """Missing or out-of-range arguments come back as MT_EINVAL (0 for the size query) from
    every entry point, before any device work; no call aborts the process."""
    L = mtlib.lib()
    E = mtlib.MT_EINVAL
    cp = mtlib.classify_params()
    st = mtlib.Stats()
    out = ctypes.c_void_p()
    d = ctypes.c_double()
    rid = ctypes.c_uint64()
    buf = np.zeros(64, np.uint64)
    p = ctypes.c_void_p(buf.ctypes.data)
    assert L.mt_classify(None, p, 8, p, 1, ctypes.byref(cp), 0, None, p, p, p, p, p, ctypes.byref(st)) == E
    assert L.mt_classify_masked(None, p, 8, p, 1, ctypes.byref(cp), 0, None, None, p, p, p, p, p,
                                ctypes.byref(st)) == E
    assert L.mt_containment(None, p, 8, p, 1, 16, 1, 10000, 0, None, p, p) == E
    assert L.mt_classify_workspace_bytes(None, 8, 1, 150, ctypes.byref(cp)) == 0
    assert L.mt_plan_create(None, ctypes.byref(cp), 10, 1000, 150, ctypes.byref(out)) == E and not out.value
    assert L.mt_plan_classify(None, p, 8, p, 1, 0, None, p, p, p, p, p, ctypes.byref(st)) == E
    assert L.mt_pack_seqs(None, p, 1, p, None) == E
    assert L.mt_eda_batch_noalloc(p, p, 1, p, p, p, p, 1, 99, None, p) == E            # no such form
    assert L.mt_eda_batch_noalloc(p, p, 1, p, p, p, p, 1 << 40, 0, None, p) == E       # too many pairs
    assert L.mt_save_index(None, b"/nonexistent/x.idx", None) == E
    assert L.mt_load_index(None, None, ctypes.byref(out)) == E
    assert L.mt_index_get_info(None, None) == E
    assert L.mt_server_submit(None, p, 8, p, 1, p, p, p, p, p, ctypes.byref(rid)) == E
    assert L.mt_server_poll(None, 1, 0, ctypes.byref(d)) == E
    assert L.mt_profile_rollup(None, 2, None, None, 0, None) == E
    assert L.mt_profile_rollup_device(None, 2, None, None, 0, None, None) == E
    sh = mtlib.EdaShape()
    assert L.mt_eda_shape_for(0x70, 0, 8, ctypes.byref(sh)) == E                     # no such approximation
    assert L.mt_eda_shape_for(0, 0, 200, ctypes.byref(sh)) == E                      # E above MT_MAX_E
    for bad in ((3, 128, 256, 0), (64, 128, 256, 0), (1, 0, 256, 0), (1, 128, 2048, 0),
                (1, 128, 100, 0), (2, 128, 256, 1), (1, 128, 256, 2)):
        assert L.mt_eda_set_shape(0, 0, 8, ctypes.byref(mtlib.EdaShape(*bad, 1))) == E, bad
    assert L.mt_eda_set_shape(0x30, 1, 8, ctypes.byref(mtlib.EdaShape(1, 128, 256, 0, 1))) == E   # q-gram: 32 lanes
    assert L.mt_eda_set_shape(0x10, 1, 8, ctypes.byref(mtlib.EdaShape(1, 128, 256, 1, 1))) == E   # refill: SneakySnake only
    assert L.mt_eda_set_shape(0, 0, 8, None) == E
    assert L.mt_eda_batch_autotune(p, p, 1, p, p, p, p, 1, 99, None, p, None) == E   # no such form
    assert L.mt_classify_autotune(None, p, 8, p, 1, ctypes.byref(cp), 0, None, p, p, p, p, p, ctypes.byref(st),
                                  ctypes.byref(sh)) == E
