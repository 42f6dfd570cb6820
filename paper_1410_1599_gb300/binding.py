"""Thin ctypes binding of libmpgemm.so (include/mpgemm.h).

Argument marshalling only: every arithmetic step runs in the library's CUDA
kernels.  PyTorch provides device memory and streams.  There is no CPU
fallback: if the library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from .inputs import EXP_ZERO, HostMP, limbs_for

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libmpgemm.so")

SIMPLE, BLOCK, STRASSEN, WINOGRAD, EXACT, SPLIT = 0, 1, 2, 3, 4, 5
PEEL, MIXED = 0, 1
OP_ADD, OP_SUB, OP_MUL, OP_DIV = 0, 1, 2, 3

MP_OK = 0
ERRORS = {-1: "MP_ERR_ARG", -2: "MP_ERR_NOMEM", -3: "MP_ERR_SINGULAR", -4: "MP_ERR_TIMEOUT",
          -5: "MP_ERR_CUDA", -6: "MP_ERR_RANGE", -7: "MP_ERR_UNSUPPORTED", -8: "MP_ERR_SCRATCH"}
NOALLOC_SCRATCH_BYTES = 64 << 20

# every symbol include/mpgemm.h declares
EXPORTS = ["mp_set_stream", "mp_set_workspace", "mp_set_odd_policy", "mp_set_lu", "mp_set_lu_pivoting",
           "mp_set_split_truncation", "mp_split_fallbacks", "mp_set_leaf_tma",
           "mp_elementwise", "mp_convert", "mpgemm_workspace_size", "mpgemm",
           "mplu_workspace_size", "mplu", "mplu_solve", "mp_sync_status", "mp_singular_column",
           "mp_strerror", "mp_version", "mp_profile_enable", "mp_profile_read", "mp_wait_selftest",
           "mpgemm_noalloc", "mpgemm_batched", "mp_server_create", "mp_server_submit", "mp_server_cancel",
           "mp_server_poll", "mp_server_drain", "mp_server_stats", "mp_server_set_graphs",
           "mp_server_graph_stats", "mp_server_destroy"]

REQ_GEMM, REQ_LU_SOLVE = 0, 1
REQ_DONE, REQ_PENDING, REQ_RUNNING, REQ_CANCELLED, REQ_FAILED = 0, 1, 2, 3, 4

(K_LEAF, K_SIMPLE, K_OPERANDS, K_COMBINE, K_FIXUP, K_ELEMENTWISE, K_LU, K_SPLIT, K_SPLIT_AUX, K_EXACT,
 K_LU_TRSM, K_LU_UPDATE, K_LU_SOLVE, K_LEAF_TMA) = range(14)
K_NAMES = ["leaf_gemm", "simple_gemm", "operands", "combine", "fixup", "elementwise", "lu_panel",
           "split_slices", "split_aux", "exact_gemm", "lu_trsm", "lu_update", "lu_solve", "leaf_tma"]


class MPError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__("%s (%d)%s" % (ERRORS.get(code, "MP_ERR"), code, (": " + what) if what else ""))


class MPMat(C.Structure):
    _fields_ = [("prec", C.c_int32), ("reserved", C.c_int32), ("rows", C.c_int64),
                ("cols", C.c_int64), ("ld", C.c_int64), ("plane", C.c_int64),
                ("limb", C.c_void_p), ("exp", C.c_void_p), ("sign", C.c_void_p)]


class MPRequest(C.Structure):
    _fields_ = [("id", C.c_int64), ("kind", C.c_int32), ("prec", C.c_int32),
                ("m", C.c_int64), ("l", C.c_int64), ("n", C.c_int64),
                ("algo", C.c_int32), ("cutoff", C.c_int32), ("lu_panel", C.c_int32),
                ("reserved", C.c_int32),
                ("a_limb", C.c_void_p), ("a_exp", C.c_void_p), ("a_sign", C.c_void_p),
                ("b_limb", C.c_void_p), ("b_exp", C.c_void_p), ("b_sign", C.c_void_p),
                ("c_limb", C.c_void_p), ("c_exp", C.c_void_p), ("c_sign", C.c_void_p)]


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load libmpgemm.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError("libmpgemm.so is not built (run paper_1410_1599_gb300/build.py)")
            lib = C.CDLL(path)
            lib.mpgemm_workspace_size.restype = C.c_size_t
            lib.mpgemm_workspace_size.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_int32,
                                                  C.c_int32, C.c_int32]
            lib.mplu_workspace_size.restype = C.c_size_t
            lib.mplu_workspace_size.argtypes = [C.c_int64, C.c_int32]
            lib.mp_wait_selftest.argtypes = [C.c_int64]
            lib.mpgemm.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_int32, C.c_int32,
                                   C.c_int32, C.POINTER(MPMat), C.POINTER(MPMat), C.POINTER(MPMat)]
            lib.mpgemm_noalloc.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_int32, C.c_int32,
                                           C.c_int32, C.POINTER(MPMat), C.POINTER(MPMat),
                                           C.POINTER(MPMat)]
            lib.mplu.argtypes = [C.c_int64, C.c_int32, C.POINTER(MPMat), C.c_void_p,
                                 C.POINTER(MPMat), C.POINTER(MPMat)]
            lib.mplu_solve.argtypes = [C.c_int64, C.c_int32, C.POINTER(MPMat), C.c_void_p,
                                       C.POINTER(MPMat), C.POINTER(MPMat)]
            lib.mpgemm_batched.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_int32,
                                           C.c_int32, C.POINTER(MPMat), C.POINTER(MPMat),
                                           C.POINTER(MPMat)]
            lib.mp_elementwise.argtypes = [C.c_int, C.POINTER(MPMat), C.POINTER(MPMat),
                                           C.POINTER(MPMat)]
            lib.mp_convert.argtypes = [C.POINTER(MPMat), C.POINTER(MPMat)]
            lib.mp_set_stream.argtypes = [C.c_void_p]
            lib.mp_set_workspace.argtypes = [C.c_void_p, C.c_size_t]
            lib.mp_singular_column.restype = C.c_int64
            lib.mp_split_fallbacks.restype = C.c_int64
            lib.mp_strerror.restype = C.c_char_p
            lib.mp_server_create.restype = C.c_void_p
            lib.mp_server_create.argtypes = [C.c_size_t, C.c_int]
            lib.mp_server_submit.argtypes = [C.c_void_p, C.POINTER(MPRequest)]
            lib.mp_server_cancel.argtypes = [C.c_void_p, C.c_int64]
            lib.mp_server_poll.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
            lib.mp_server_drain.argtypes = [C.c_void_p]
            lib.mp_server_set_graphs.argtypes = [C.c_void_p, C.c_int]
            lib.mp_server_graph_stats.argtypes = [C.c_void_p, C.c_void_p]
            lib.mp_server_stats.argtypes = [C.c_void_p, C.c_void_p]
            lib.mp_server_destroy.argtypes = [C.c_void_p]
            lib.mp_profile_read.argtypes = [C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                            C.POINTER(C.c_double)]
            _lib = lib
    return _lib


def _check(rc: int, what: str = ""):
    if rc != MP_OK:
        raise MPError(rc, what)


class DeviceMP:
    """A rows x cols matrix of p-bit numbers in device memory (torch tensors):
    limb (L, rows, ld) int64 bit patterns, exp (rows, ld) int64, sign (rows, ld) int8."""

    def __init__(self, limb, exp, sign, p: int, rows: int, cols: int, ld: int | None = None,
                 plane: int | None = None, offset: int = 0):
        self.limb, self.exp, self.sign = limb, exp, sign
        self.p, self.rows, self.cols = p, rows, cols
        self.ld = cols if ld is None else ld
        self.plane = rows * self.ld if plane is None else plane
        self.offset = offset          # element offset of (0, 0) inside the arrays

    @staticmethod
    def empty(rows: int, cols: int, p: int, device="cuda"):
        import torch
        L = limbs_for(p)
        return DeviceMP(torch.empty((L, rows, cols), dtype=torch.int64, device=device),
                        torch.empty((rows, cols), dtype=torch.int64, device=device),
                        torch.empty((rows, cols), dtype=torch.int8, device=device), p, rows, cols)

    @staticmethod
    def from_host(M: HostMP, device="cuda"):
        import torch
        rows, cols = M.shape
        limb = torch.from_numpy(np.ascontiguousarray(M.limb).view(np.int64)).to(device)
        exp = torch.from_numpy(np.ascontiguousarray(M.exp)).to(device)
        sign = torch.from_numpy(np.ascontiguousarray(M.sign)).to(device)
        return DeviceMP(limb, exp, sign, M.p, rows, cols)

    def to_host(self) -> HostMP:
        L = limbs_for(self.p)
        limb = self.limb.reshape(-1).cpu().numpy().view(np.uint64)
        exp = self.exp.reshape(-1).cpu().numpy()
        sign = self.sign.reshape(-1).cpu().numpy()
        idx = self.offset + np.arange(self.rows)[:, None] * self.ld + np.arange(self.cols)[None, :]
        lm = np.stack([limb[k * self.plane + idx] for k in range(L)]) if L else \
            np.zeros((0, self.rows, self.cols), np.uint64)
        return HostMP(np.ascontiguousarray(lm), exp[idx].copy(), sign[idx].copy(), self.p)

    def view(self, r0: int, c0: int, rows: int, cols: int) -> "DeviceMP":
        return DeviceMP(self.limb, self.exp, self.sign, self.p, rows, cols, self.ld, self.plane,
                        self.offset + r0 * self.ld + c0)

    def struct(self) -> MPMat:
        return MPMat(self.p, 0, self.rows, self.cols, self.ld, self.plane,
                     self.limb.data_ptr() + 8 * self.offset, self.exp.data_ptr() + 8 * self.offset,
                     self.sign.data_ptr() + self.offset)

    def nbytes(self) -> int:
        return self.limb.numel() * 8 + self.exp.numel() * 8 + self.sign.numel()


# ------------------------------------------------------------------ settings
def set_stream(stream) -> None:
    """stream: a torch.cuda.Stream, a raw handle, or None (legacy default)."""
    h = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(load_library().mp_set_stream(C.c_void_p(h)))


def set_workspace(tensor=None) -> None:
    lib = load_library()
    if tensor is None:
        _check(lib.mp_set_workspace(None, 0))
    else:
        _check(lib.mp_set_workspace(C.c_void_p(tensor.data_ptr()), tensor.numel() * tensor.element_size()))


def set_odd_policy(policy: int) -> None:
    _check(load_library().mp_set_odd_policy(policy), "odd policy")


def set_lu(panel: int = 128, algo: int = SIMPLE, cutoff: int = 64) -> None:
    _check(load_library().mp_set_lu(panel, algo, cutoff), "lu settings")


def set_lu_pivoting(on: bool = True) -> None:
    _check(load_library().mp_set_lu_pivoting(1 if on else 0), "lu pivoting")


def set_split_truncation(on: bool = True) -> None:
    _check(load_library().mp_set_split_truncation(1 if on else 0), "split truncation")


def set_leaf_tma(on: bool = True) -> None:
    """Stage the Block kernel's tiles with TMA where the layout allows (default)."""
    _check(load_library().mp_set_leaf_tma(1 if on else 0), "leaf staging")


def split_fallbacks() -> int:
    """Outputs the truncated split form left to the exact kernel, as counted
    by the last sync_status()."""
    return load_library().mp_split_fallbacks()


def sync_status() -> int:
    return load_library().mp_sync_status()


def check_status(what: str = "") -> None:
    _check(sync_status(), what)


def version() -> int:
    return load_library().mp_version()


def wait_selftest(cycles: int) -> int:
    """Status of one bounded device wait on a barrier nothing completes
    (MP_ERR_TIMEOUT = -4 when the failure detection works)."""
    return load_library().mp_wait_selftest(cycles)


def profile_enable(on: bool = True) -> None:
    _check(load_library().mp_profile_enable(1 if on else 0))


def profile_read() -> dict:
    """{class name: (launches, milliseconds, work units)} since profile_enable."""
    lib = load_library()
    out = {}
    for k, name in enumerate(K_NAMES):
        n, ms, u = C.c_int64(), C.c_double(), C.c_double()
        _check(lib.mp_profile_read(k, C.byref(n), C.byref(ms), C.byref(u)))
        out[name] = (n.value, ms.value, u.value)
    return out


# ---------------------------------------------------------------- operations
def elementwise(op: int, X: DeviceMP, Y: DeviceMP, R: DeviceMP) -> None:
    x, y, r = X.struct(), Y.struct(), R.struct()
    _check(load_library().mp_elementwise(op, C.byref(x), C.byref(y), C.byref(r)), "elementwise")


def convert(X: DeviceMP, R: DeviceMP) -> None:
    x, r = X.struct(), R.struct()
    _check(load_library().mp_convert(C.byref(x), C.byref(r)), "convert")


def workspace_size(m: int, l: int, n: int, p: int, algo: int, cutoff: int) -> int:
    return load_library().mpgemm_workspace_size(m, l, n, p, algo, cutoff)


def mpgemm(A: DeviceMP, B: DeviceMP, C_: DeviceMP, algo: int = SIMPLE, cutoff: int = 64) -> None:
    a, b, c = A.struct(), B.struct(), C_.struct()
    _check(load_library().mpgemm(A.rows, A.cols, B.cols, A.p, algo, cutoff, C.byref(a),
                                 C.byref(b), C.byref(c)), "mpgemm")


def mpgemm_batched(batch: int, A: DeviceMP, B: DeviceMP, C_: DeviceMP, algo: int = BLOCK) -> None:
    """batch independent products on row-stacked operands (see include/mpgemm.h)."""
    m, l, n = A.rows // batch, A.cols, B.cols
    a, b, c = A.struct(), B.struct(), C_.struct()
    _check(load_library().mpgemm_batched(batch, m, l, n, A.p, algo, C.byref(a), C.byref(b),
                                         C.byref(c)), "mpgemm_batched")


def mpgemm_noalloc(A: DeviceMP, B: DeviceMP, C_: DeviceMP, algo: int = WINOGRAD,
                   cutoff: int = 64) -> None:
    """mpgemm with the recursion's temporaries in the library's static device
    scratch (no allocation); see include/mpgemm.h."""
    a, b, c = A.struct(), B.struct(), C_.struct()
    _check(load_library().mpgemm_noalloc(A.rows, A.cols, B.cols, A.p, algo, cutoff, C.byref(a),
                                         C.byref(b), C.byref(c)), "mpgemm_noalloc")


def mplu_solve(LU: DeviceMP, piv, B: DeviceMP, X: DeviceMP) -> None:
    """X = A^-1 B from the factors mplu left in LU (see include/mpgemm.h)."""
    a, b, x = LU.struct(), B.struct(), X.struct()
    _check(load_library().mplu_solve(LU.rows, LU.p, C.byref(a), C.c_void_p(piv.data_ptr()), C.byref(b),
                                      C.byref(x)), "mplu_solve")


def mplu(A: DeviceMP, piv, b: DeviceMP | None, x: DeviceMP | None) -> None:
    a = A.struct()
    bs = b.struct() if b is not None else None
    xs = x.struct() if x is not None else None
    _check(load_library().mplu(A.rows, A.p, C.byref(a), C.c_void_p(piv.data_ptr()),
                               C.byref(bs) if bs is not None else None,
                               C.byref(xs) if xs is not None else None), "mplu")


# ------------------------------------------------------------------ serving
def _host_arrays(M, pinned: bool):
    """Contiguous interchange arrays of a HostMP, and the objects owning their
    memory (page-locked torch tensors when pinned)."""
    arrs = [np.ascontiguousarray(M.limb, dtype=np.uint64), np.ascontiguousarray(M.exp, dtype=np.int64),
            np.ascontiguousarray(M.sign, dtype=np.int8)]
    if not pinned:
        return arrs, arrs
    import torch
    views, owners = [], []
    for a in arrs:
        t = torch.empty(a.shape, dtype=torch.int8 if a.dtype == np.int8 else torch.int64,
                        pin_memory=True)
        v = t.numpy().view(a.dtype)
        v[...] = a
        views.append(v)
        owners.append(t)
    return views, owners


class Server:
    """Continuous-batching request loop of the library (mp_server_*)."""

    def __init__(self, budget_bytes: int, slots: int = 8, pinned: bool = True, keep_outputs: bool = True):
        self.lib = load_library()
        self.h = self.lib.mp_server_create(C.c_size_t(budget_bytes), slots)
        if not self.h:
            raise MPError(-5, "mp_server_create")
        self.pinned = pinned
        self.keep_outputs = keep_outputs     # False: results keep status and latency only
        self.live = {}            # id -> buffers kept alive until completion
        self.results = {}         # id -> (status, latency_ms, output HostMP)

    def _prepare(self, rid, kind, prec, m, l, n, algo, cutoff, panel, A, B, out):
        """The request record and its host buffers (page-locked copies when
        pinned), ready for submit(): preparing costs a copy of the operands,
        submitting only queues the request."""
        a, ka = _host_arrays(A, self.pinned)
        b, kb = _host_arrays(B, self.pinned)
        o, ko = _host_arrays(out, self.pinned)
        ptr = lambda x: x.ctypes.data_as(C.c_void_p)
        r = MPRequest(rid, kind, prec, m, l, n, algo, cutoff, panel, 0,
                      ptr(a[0]), ptr(a[1]), ptr(a[2]), ptr(b[0]), ptr(b[1]), ptr(b[2]),
                      ptr(o[0]), ptr(o[1]), ptr(o[2]))
        return (rid, r, (a, b, o, prec, (ka, kb, ko)))

    def submit(self, prepared) -> int:
        rid, r, bufs = prepared
        self.live[rid] = bufs
        rc = self.lib.mp_server_submit(self.h, C.byref(r))
        if rc != MP_OK:
            del self.live[rid]
        return rc

    def prepare_gemm(self, rid, A, B, algo=BLOCK, cutoff=64):
        m, l = A.shape
        n = B.shape[1]
        out = HostMP.zeros(m, n, A.p)
        return self._prepare(rid, REQ_GEMM, A.p, m, l, n, algo, cutoff, 0, A, B, out)

    def prepare_lu(self, rid, A, b, algo=SIMPLE, cutoff=64, panel=128):
        n = A.shape[0]
        out = HostMP.zeros(n, 1, A.p)
        return self._prepare(rid, REQ_LU_SOLVE, A.p, n, n, 1, algo, cutoff, panel, A, b, out)

    def submit_gemm(self, rid, A, B, algo=BLOCK, cutoff=64):
        return self.submit(self.prepare_gemm(rid, A, B, algo, cutoff))

    def submit_lu(self, rid, A, b, algo=SIMPLE, cutoff=64, panel=128):
        return self.submit(self.prepare_lu(rid, A, b, algo, cutoff, panel))

    def cancel(self, rid) -> int:
        return self.lib.mp_server_cancel(self.h, rid)

    def poll(self, max_n: int = 4096):
        ids = np.zeros(max_n, np.int64)
        st = np.zeros(max_n, np.int32)
        ms = np.zeros(max_n, np.float64)
        k = self.lib.mp_server_poll(self.h, ids.ctypes.data_as(C.c_void_p), st.ctypes.data_as(C.c_void_p),
                                    ms.ctypes.data_as(C.c_void_p), max_n)
        done = []
        for i in range(k):
            rid = int(ids[i])
            bufs = self.live.pop(rid, None)
            out = None
            if bufs is not None and self.keep_outputs:
                o, prec = bufs[2], bufs[3]
                out = HostMP(o[0].copy(), o[1].copy(), o[2].copy(), prec)
            self.results[rid] = (int(st[i]), float(ms[i]), out)
            done.append(rid)
        return done

    def drain(self):
        _check(self.lib.mp_server_drain(self.h), "drain")
        self.poll()

    def stats(self) -> dict:
        out = np.zeros(8, np.int64)
        _check(self.lib.mp_server_stats(self.h, out.ctypes.data_as(C.c_void_p)))
        keys = ["submitted", "completed", "batches", "batched_requests", "peak_bytes", "budget",
                "running", "queued"]
        return dict(zip(keys, (int(x) for x in out)))

    def set_graphs(self, max_graphs: int) -> None:
        """Size of the server's CUDA-graph cache for repeated request shapes (0: off)."""
        _check(self.lib.mp_server_set_graphs(self.h, max_graphs), "set_graphs")

    def graph_stats(self) -> dict:
        out = np.zeros(4, np.int64)
        _check(self.lib.mp_server_graph_stats(self.h, out.ctypes.data_as(C.c_void_p)))
        return dict(zip(["captured", "replays", "cached", "cached_bytes"], (int(x) for x in out)))

    def close(self):
        if self.h:
            self.lib.mp_server_drain(self.h)
            self.poll()
            self.lib.mp_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
