"""GPU round trip of the index file (mt_save_index / mt_load_index): a loaded index answers
every query exactly as the one saved, and damaged files are refused."""
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


@pytest.mark.parametrize("cfg", [1, 2])
def test_saved_index_answers_like_the_original(mt, tmp_path, cfg):
    c = gen.config(cfg, n_genomes=20, genome_len=100_000, n_reads=10_000) if cfg == 2 else gen.config(1)
    g = gen.make_genomes(c)
    r = gen.make_reads(c, g)
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    path = str(tmp_path / "ref.idx")
    ix.save(path)
    iy = mt.Index.load(path)
    assert iy.info() == ix.info()
    prm = dict(e_abs=c["e_abs"], e_permille=c["e_permille"], min_seeds=c["min_seeds"], top_n=3, max_occ=1024,
               cont_num=1, cont_den=10000, abund_cutoff=1e-4)
    a = mt.classify(ix, r.seq, r.offsets, **prm)
    b = mt.classify(iy, r.seq, r.offsets, **prm)
    for k in ("taxon", "nloc", "genome_hits"):
        assert np.array_equal(a[k], b[k])
    assert np.array_equal(a["locs"], b["locs"])
    assert np.array_equal(a["abundance"], b["abundance"])
    oix = oracle.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    compare_classify(b, oracle.classify(oix, r.seq, r.offsets, oracle_params(prm), threads=8))
    iy.close()


def test_damaged_files_are_refused(mt, tmp_path):
    c = gen.config(1)
    g = gen.make_genomes(c)
    ix = mt.Index(g.seq, g.offsets, c["k"], c["w"], c["canonical"])
    path = tmp_path / "ref.idx"
    ix.save(str(path))
    data = path.read_bytes()
    for name, bad in (("truncated", data[:-9]), ("trailer", data[:-1] + b"X"),
                      ("header", data[:20] + bytes([data[20] ^ 1]) + data[21:]), ("longer", data + b"\0")):
        p = tmp_path / (name + ".idx")
        p.write_bytes(bad)
        with pytest.raises(mt.MtError) as e:
            mt.Index.load(str(p))
        assert e.value.status == mt.MT_EIO, name
