"""Host-side checks of the C ABI (no GPU needed): the in-tree library builds,
loads, exports every function that include/mvtsdf.h declares, the binding
declares the same set, and argument validation fails cleanly before any CUDA
work."""
import ctypes as C
import os
import re

import pytest

from paper_1511_07106_b300 import _abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mvtsdf.h")


def header_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mv_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _abi.lib()


def test_header_declares_the_paper_calls():
    fns = header_functions()
    for name in ("mv_create", "mv_destroy", "mv_add_volume", "mv_remove_volume", "mv_integrate",
                 "mv_raycast", "mv_swap_out", "mv_swap_in", "mv_read_volume", "mv_write_volume"):
        assert name in fns


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_binding_covers_header_exactly():
    assert sorted(_abi.declared_functions()) == header_functions()


def test_struct_sizes_match_header_layout():
    assert C.sizeof(_abi.mv_intrinsics) == 24
    assert C.sizeof(_abi.mv_config) == 28
    assert C.sizeof(_abi.mv_volume_desc) == 32
    assert C.sizeof(_abi.mv_stats) == 80


def test_version_and_defaults(lib):
    assert b"mvtsdf" in lib.mv_version()
    cfg = _abi.mv_config()
    assert lib.mv_config_default(C.byref(cfg)) == _abi.MV_OK
    assert cfg.trunc_voxels == 4.0 and cfg.w_max == 128.0 and cfg.ray_step == 1.0
    assert lib.mv_config_default(None) == _abi.MV_ERR_ARG


def test_argument_validation_without_gpu(lib):
    h = C.c_void_p()
    assert lib.mv_create(None, 0, None) == _abi.MV_ERR_ARG
    bad = _abi.mv_config()
    lib.mv_config_default(C.byref(bad))
    bad.ray_step = 2.0  # must be in (0, 1]
    assert lib.mv_create(C.byref(bad), 0, C.byref(h)) == _abi.MV_ERR_ARG
    bad.ray_step = 1.0
    bad.color_w_max = 300
    assert lib.mv_create(C.byref(bad), 0, C.byref(h)) == _abi.MV_ERR_ARG
    # null contexts are rejected, never dereferenced
    assert lib.mv_integrate(None, None, None, None, None, None) == _abi.MV_ERR_ARG
    assert lib.mv_raycast(None, None, None, None, None, None, None, None, None) == _abi.MV_ERR_ARG
    assert lib.mv_swap_out(None, 0, None) == _abi.MV_ERR_ARG
    assert lib.mv_destroy(None) == _abi.MV_OK
    assert lib.mv_last_error(None) == b"null context"


def test_create_without_device_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert lib.mv_create(None, 0, C.byref(h)) == _abi.MV_ERR_CUDA
    assert not h.value


def test_merge_calls_refuse_misaligned_buffers_before_any_launch(lib):
    """mv_pack_hits and mv_merge_hits check their buffers' alignment on the
    host before anything else: addresses off a 4-byte (maps) or 8-byte (keys)
    boundary come back as MV_ERR_ARG, never dereferenced."""
    word, odd, half = C.c_void_p(0x1000), C.c_void_p(0x1001), C.c_void_p(0x1004)
    keys = C.c_void_p(0x2000)
    assert lib.mv_pack_hits(odd, word, None, 0, 16, keys, None) == _abi.MV_ERR_ARG
    assert lib.mv_pack_hits(word, odd, None, 0, 16, keys, None) == _abi.MV_ERR_ARG
    assert lib.mv_pack_hits(word, word, None, 0, 16, half, None) == _abi.MV_ERR_ARG
    assert lib.mv_merge_hits(half, keys, 16, None, None, None, None, None, None) == _abi.MV_ERR_ARG
    assert lib.mv_merge_hits(keys, half, 16, None, None, None, None, None, None) == _abi.MV_ERR_ARG
    assert lib.mv_merge_hits(keys, keys, 16, None, None, odd, None, None, None) == _abi.MV_ERR_ARG
    assert lib.mv_merge_hits(keys, keys, 16, None, None, None, C.c_void_p(0x1002), None, None) == _abi.MV_ERR_ARG
