"""The C-ABI library builds, loads and exports every symbol include/adms.h declares (no GPU needed)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(adms_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2104_03989_gb300 import build

    return build.build()


def test_header_declares_the_step_calls():
    names = declared_symbols()
    for required in ("adms_render_reference", "adms_forward_loss", "adms_backward", "adms_optimizer_step",
                     "adms_ctx_create", "adms_job_create"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_2104_03989_gb300 import binding

    assert set(declared_symbols()) <= set(binding.SIGNATURES)
    binding.lib()  # loads without touching a GPU


@pytest.mark.parametrize("n_verts,n_tris,n_views,H,W", [
    (2**31 - 1, 1, 2**31 - 1, 16, 16),        # views x vertices x 16 B wraps a 64-bit size
    (3, 2**31 - 1, 2**31 - 1, 16, 16),        # views x triangles x 96 B wraps
    (3, 1 << 20, 100, 16, 16),                 # no wrap, far beyond the 32 MiB array
    (3, 1, 2**31 - 1, 16384, 16384),           # tiles of the views alone exceed it
])
def test_noalloc_refuses_oversized_requests_before_any_cuda_call(libpath, n_verts, n_tris, n_views, H, W):
    """adms_visibility_noalloc sizes its scratch with checked arithmetic before it
    touches CUDA, so requests whose size products overflow, or do not fit, are
    refused with ADMS_ERR_ARG on the host (here: a machine without a GPU; the
    pointers are never dereferenced)."""
    lib = ctypes.CDLL(libpath)
    f = lib.adms_visibility_noalloc
    P = ctypes.c_void_p
    f.argtypes = [P, ctypes.c_int32, P, ctypes.c_int32, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P]
    f.restype = ctypes.c_int
    dummy = P(16)
    assert f(dummy, n_verts, dummy, n_tris, dummy, n_views, H, W, dummy, None) == -1   # ADMS_ERR_ARG
