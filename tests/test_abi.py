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
