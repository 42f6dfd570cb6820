"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/mpgemm.h declares (no GPU needed: nothing is called that computes)."""
import ctypes
import os
import re

import pytest

from paper_1410_1599_gb300 import binding
from paper_1410_1599_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "mpgemm.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(mp[a-z_0-9]*)\s*\(", hdr, flags=re.M)
    return sorted(set(names))


def test_header_declarations_match_binding_list():
    assert _declared() == sorted(binding.EXPORTS)


def test_library_builds_and_exports_everything():
    path = libbuild.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_host_only_calls():
    lib = binding.load_library()
    assert lib.mp_version() == 100
    assert lib.mp_strerror(-3) == b"zero pivot: matrix is singular"
    assert lib.mp_set_odd_policy(7) == -1
    assert lib.mp_set_lu(0, 0, 64) == -1
    assert lib.mp_set_lu(128, 3, -1) == -1 and lib.mp_set_lu(128, 3, 0) == 0 and lib.mp_set_lu(128, 0, 64) == 0
    # cutoff 0: the library's choice, 64 up to 1024 bits and 32 above
    for p, c in ((512, 64), (1024, 64), (2048, 32)):
        assert lib.mpgemm_workspace_size(1000, 1000, 1000, p, 3, 0) == \
            lib.mpgemm_workspace_size(1000, 1000, 1000, p, 3, c) > 0
    assert lib.mp_set_lu_pivoting(2) == -1
    assert lib.mp_set_lu_pivoting(0) == 0 and lib.mp_set_lu_pivoting(1) == 0
    assert lib.mp_set_split_truncation(3) == -1
    assert lib.mp_set_split_truncation(0) == 0 and lib.mp_set_split_truncation(1) == 0
    # Simple and Block need no workspace; the recursion does
    assert lib.mpgemm_workspace_size(1024, 1024, 1024, 512, 0, 64) == 0
    assert lib.mpgemm_workspace_size(1024, 1024, 1024, 512, 3, 64) > 0
    assert lib.mpgemm_workspace_size(64, 64, 64, 512, 3, 64) == 0


def test_argument_errors_without_gpu():
    """Argument checks run on the host before any CUDA call."""
    lib = binding.load_library()
    bad = binding.MPMat(100000, 0, 2, 2, 2, 4, 1, 1, 1)      # precision out of range
    assert lib.mpgemm(2, 2, 2, 100000, 0, 64, ctypes.byref(bad), ctypes.byref(bad),
                      ctypes.byref(bad)) == -1
    A = binding.MPMat(128, 0, 2, 3, 3, 6, 4096, 8192, 12288)
    B = binding.MPMat(128, 0, 3, 2, 2, 6, 16384, 20480, 24576)
    Cm = binding.MPMat(128, 0, 2, 2, 1, 4, 32768, 36864, 40960)  # ld < cols
    assert lib.mpgemm(2, 3, 2, 128, 0, 64, ctypes.byref(A), ctypes.byref(B), ctypes.byref(Cm)) == -1
    Cm = binding.MPMat(128, 0, 2, 2, 2, 4, 4096, 8192, 12288)    # aliases A
    assert lib.mpgemm(2, 3, 2, 128, 0, 64, ctypes.byref(A), ctypes.byref(B), ctypes.byref(Cm)) == -1
    assert lib.mpgemm(2, 3, 2, 128, 9, 64, ctypes.byref(A), ctypes.byref(B), ctypes.byref(A)) == -1


def test_noalloc_limit_checked_on_the_host():
    """mpgemm_noalloc rejects a product whose recursion needs more than its
    static scratch before any CUDA call, and an empty product returns at
    once; the limit is the recursion's workspace size.  (Only paths that
    never reach the device are taken here: the pointers are placeholders.)"""
    lib = binding.load_library()
    limit = binding.NOALLOC_SCRATCH_BYTES
    p = 512
    for n in (256, 300, 512):
        assert lib.mpgemm_workspace_size(n, n, n, p, 3, 64) > limit
        A = binding.MPMat(p, 0, n, n, n, n * n, 1 << 20, 1 << 30, 1 << 31)
        B = binding.MPMat(p, 0, n, n, n, n * n, 1 << 32, 1 << 33, 1 << 34)
        Cm = binding.MPMat(p, 0, n, n, n, n * n, 1 << 35, 1 << 36, 1 << 37)
        assert lib.mpgemm_noalloc(n, n, n, p, 3, 64, ctypes.byref(A), ctypes.byref(B), ctypes.byref(Cm)) == -8
    assert lib.mpgemm_workspace_size(200, 200, 200, p, 3, 64) <= limit
    E = binding.MPMat(p, 0, 0, 5, 5, 0, 0, 0, 0)
    F = binding.MPMat(p, 0, 5, 4, 4, 20, 1 << 20, 1 << 30, 1 << 31)
    G = binding.MPMat(p, 0, 0, 4, 4, 0, 0, 0, 0)
    assert lib.mpgemm_noalloc(0, 5, 4, p, 3, 64, ctypes.byref(E), ctypes.byref(F), ctypes.byref(G)) == 0


def test_multi_rhs_solve_argument_errors_without_gpu():
    """mplu_solve checks its arguments on the host: precision, shapes (B and
    X n x nrhs), a missing pivot vector, X overlapping the factors or B; an
    empty system returns at once.  (Placeholder pointers: no path here
    reaches the device.)"""
    lib = binding.load_library()
    p, n, r = 256, 3, 2
    LU = binding.MPMat(p, 0, n, n, n, n * n, 4096, 8192, 12288)
    B = binding.MPMat(p, 0, n, r, r, n * r, 16384, 20480, 24576)
    X = binding.MPMat(p, 0, n, r, r, n * r, 32768, 36864, 40960)
    piv = ctypes.c_void_p(65536)
    ok = lambda *a: lib.mplu_solve(*a)
    bad_p = binding.MPMat(9000, 0, n, n, n, n * n, 4096, 8192, 12288)
    assert ok(n, 9000, ctypes.byref(bad_p), piv, ctypes.byref(B), ctypes.byref(X)) == -1
    Xs = binding.MPMat(p, 0, n, r + 1, r + 1, n * (r + 1), 32768, 36864, 40960)   # nrhs differs from B
    assert ok(n, p, ctypes.byref(LU), piv, ctypes.byref(B), ctypes.byref(Xs)) == -1
    assert ok(n, p, ctypes.byref(LU), None, ctypes.byref(B), ctypes.byref(X)) == -1
    Xa = binding.MPMat(p, 0, n, r, r, n * r, 16384, 20480, 24576)                  # X = B
    assert ok(n, p, ctypes.byref(LU), piv, ctypes.byref(B), ctypes.byref(Xa)) == -1
    E = binding.MPMat(p, 0, 0, 0, 0, 0, 0, 0, 0)
    assert ok(0, p, ctypes.byref(E), None, ctypes.byref(E), ctypes.byref(E)) == 0
