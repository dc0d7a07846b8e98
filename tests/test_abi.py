"""The C ABI library builds for sm_103a, loads without a GPU and exports
every entry point include/proxybdpt.h declares; host-side argument checks
reject bad calls before any device work."""

import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2503_23412_gb300 import build
    build.build()
    from paper_2503_23412_gb300 import native
    return native.lib()


def declared():
    src = open(os.path.join(ROOT, "include", "proxybdpt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pb_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("pb_create", "pb_destroy", "pb_scene_upload", "pb_tables_upload", "pb_render",
              "pb_film_readback", "pb_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    for n in declared():
        assert hasattr(L, n), n


def test_null_arguments_are_rejected_without_a_device(L):
    from paper_2503_23412_gb300 import native as N
    assert L.pb_create(None, 0, None) == N.PB_ERR_ARG
    assert L.pb_scene_upload(None, None) == N.PB_ERR_ARG
    assert L.pb_render(None, None, None) == N.PB_ERR_ARG
    assert L.pb_film_readback(None, None, 0) == N.PB_ERR_ARG
    assert L.pb_last_error(None) == b"null context"


def test_network_parameter_count_matches_the_layout(L):
    """W1 16x64 (its bias rides on the constant input), W2 64x64, b2, W3
    K_S x 64, b3, and a 4-d embedding per eye subspace."""
    for KS, KT in ((1, 1), (40, 12), (300, 64)):
        assert L.pb_mlp_nparams(KS, KT) == 16 * 64 + 64 * 64 + 64 + 64 * KS + KS + 4 * KT


def test_autotune_cache_text_round_trip(L, tmp_path):
    """The tuning cache is host state: loading keeps only valid lines (a batch
    of 1..64 iterations, an estimator schedule of 0 or 1), saving writes one
    line per key, and clearing empties it. No device is touched."""
    from paper_2503_23412_gb300 import native as N
    src = tmp_path / "in.txt"
    src.write_text("s256x256_d8 16 0 4.25\n"
                   "s64x64_d6 32 1 1.5\n"
                   "bad_batch 0 0 1.0\n"
                   "bad_batch2 65 1 1.0\n"
                   "bad_sched 8 2 1.0\n")
    N.autotune_cache_clear()
    N.autotune_cache_load(str(src))
    out = tmp_path / "out.txt"
    N.autotune_cache_save(str(out))
    rows = sorted(line.split() for line in out.read_text().splitlines())
    assert [r[:3] for r in rows] == [["s256x256_d8", "16", "0"], ["s64x64_d6", "32", "1"]]
    assert [float(r[3]) for r in rows] == [4.25, 1.5]
    N.autotune_cache_clear()
    N.autotune_cache_save(str(out))
    assert out.read_text() == ""
    with pytest.raises(N.PBError):
        N.autotune_cache_load(str(tmp_path / "missing.txt"))
