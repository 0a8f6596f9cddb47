"""CPU checks of the C-ABI library: it builds, loads, exports every symbol that
include/*.h declares, and its host-only helpers behave.  No compute calls."""
import ctypes
import glob
import os
import re

import pytest

from paper_2006_13714_gb300 import bm as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(?:int|void|size_t|const char\s*\*)\s+(bm_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("bm_create", "bm_match", "bm_submit", "bm_poll", "bm_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(B.build_ext.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("H,W,p,s,want", [
    (64, 64, 8, 1, (57, 57)), (512, 512, 8, 3, (169, 169)), (1024, 1024, 8, 3, (339, 339)),
    (321, 481, 7, 4, (79, 119)), (8, 8, 8, 5, (1, 1))])
def test_num_refs(H, W, p, s, want):
    assert B.bm_num_refs(H, W, p, s) == want


@pytest.mark.parametrize("args", [(8, 8, 9, 1), (8, 8, 0, 1), (8, 8, 2, 0), (0, 8, 1, 1)])
def test_num_refs_rejects(args):
    with pytest.raises(B.BMError) as e:
        B.bm_num_refs(*args)
    assert e.value.code == B.BM_ERR_INVALID


def test_create_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(B.BMError) as e:
        B.bm_create(0)
    assert e.value.code in (B.BM_ERR_CUDA, B.BM_ERR_INVALID)


def test_window_split_query():
    # small jobs split their windows (alone they leave SMs idle), large ones do not
    assert B.bm_window_split(64, 64, 1, B.BM_U8, 8, 21, 1, 16) == 4
    assert B.bm_window_split(2048, 2048, 1, B.BM_F32, 8, 39, 3, 16) == 1
    assert B.bm_window_split(64, 64, 1, B.BM_U8, 8, 22, 1, 16) == 0  # even window: invalid
    for args in [(96, 88, 1, B.BM_F32, 8, 39, 3, 16), (150, 133, 1, B.BM_F32, 7, 61, 4, 70),
                 (80, 72, 4, B.BM_U8, 8, 39, 3, 32), (8, 12, 1, B.BM_U8, 8, 7, 1, 5)]:
        assert B.bm_window_split(*args) in (1, 2, 4)


def test_workspace_bytes_query():
    # the context workspace holds at least the static path's buffers, plus
    # the window split's part lists when the job splits
    for args in [(96, 96, 1, B.BM_F32, 8, 39, 3, 16), (512, 512, 1, B.BM_F32, 8, 39, 3, 16),
                 (64, 64, 1, B.BM_U8, 8, 21, 1, 16)]:
        ws = B.bm_workspace_bytes(*args)
        assert ws >= B.bm_static_scratch_bytes(*args) - 256 > 0
    assert B.bm_workspace_bytes(160, 150, 4, B.BM_U8, 8, 127, 4, 128) == 0  # direct kernel
    # column parts (the staged tile fits only per part): 2 parts, their lists included
    assert B.bm_window_split(160, 150, 1, B.BM_U8, 8, 127, 4, 128) == 2
    assert B.bm_workspace_bytes(160, 150, 1, B.BM_U8, 8, 127, 4, 128) > 0
    assert B.bm_window_split(512, 512, 4, B.BM_F32, 8, 61, 3, 32) == 2
    assert B.bm_static_scratch_bytes(512, 512, 4, B.BM_F32, 8, 61, 3, 32) > \
        B.bm_static_scratch_bytes(512, 512, 4, B.BM_F32, 8, 61, 3, 16)
    assert B.bm_workspace_bytes(64, 64, 1, B.BM_U8, 8, 22, 1, 16) == 0      # invalid
