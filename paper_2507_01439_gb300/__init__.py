"""Python binding of the GB300 TurboReg registration library.

Thin ctypes layer over ``libturboreg_gb300.so`` (C ABI in
``include/turboreg.h``): it only marshals arguments.  Every step of the
registration path runs in the library's CUDA kernels; there is no Python or
CPU fallback, and importing the library raises if it has not been built.

Inputs may be NumPy arrays (host memory, copied by the library) or CUDA
torch tensors (device memory, read in place).  PyTorch is used only for
device memory and streams.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libturboreg_gb300.so")

TURBOREG_MAX_N = 32768
TURBOREG_K1_MAX = 8192
TURBOREG_K2_MAX = 16

OK, ERR_INVALID_ARG, ERR_TOO_FEW, ERR_NONFINITE, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NO_HYPOTHESIS = range(8)
GRAPH_O2, GRAPH_SC2 = 0, 1
SCORE_IN, SCORE_MAE, SCORE_MSE = 0, 1, 2
PROPOSAL_PLAIN, PROPOSAL_LEARNED = 0, 1
FLAG_SC2_BITSET = 0x1
FLAG_STAGE_TIMES = 0x2
FLAG_NO_GRAPH = 0x4
FLAG_SC2_SINGLE_CTA = 0x8
FLAG_VERIFY_PTS32 = 0x10
FLAG_VERIFY_PTS128 = 0x20
FLAG_SC2_GEMM = 0x40
FLAG_DEBUG_STALL_COMPAT = 0x10000   # test hook: every compat block's wait expires (TIMEOUT)

(BUF_ADJ_BITS, BUF_ADJ_FP8, BUF_SC2, BUF_PIVOTS, BUF_CLIQUES, BUF_RT, BUF_INLIERS, BUF_ROWSCORE, BUF_DEGREE,
 BUF_FEATURES, BUF_PROB, BUF_SCORES) = range(1, 13)
SCORE_UNITS = 1 << 22   # BUF_SCORES units per theta (MAE) or theta^2 (MSE)

# symbols the library must export (declared in include/turboreg.h and include/turboreg_internal.h)
EXPORTED = (
    "turboreg_default_params", "turboreg_create", "turboreg_register", "turboreg_register_batched",
    "turboreg_destroy", "turboreg_status_string", "turboreg_debug_shape", "turboreg_debug_copy",
    "turboreg_debug_sc2_path",
    "turboreg_stage_times", "turboreg_stage_name", "turboreg_select_pivots_noalloc",
    "turboreg_set_proposal_model", "turboreg_features", "turboreg_mlp_create", "turboreg_mlp_destroy",
    "turboreg_mlp_get_params", "turboreg_mlp_set_params", "turboreg_mlp_get_state", "turboreg_mlp_set_state",
    "turboreg_mlp_forward", "turboreg_mlp_grad", "turboreg_mlp_train_step", "turboreg_score_transforms",
    "turboreg_kabsch_cliques", "turboreg_register_async", "turboreg_synchronize",
)
TURBOREG_MLP_PARAMS = 17217
TURBOREG_NOALLOC_MAX_N = 8192


class turboreg_params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_float), ("k1", ctypes.c_int32), ("k2", ctypes.c_int32),
                ("inlier_thresh", ctypes.c_float), ("graph_mode", ctypes.c_int32),
                ("proposal", ctypes.c_int32), ("kappa_fp64", ctypes.c_float), ("flags", ctypes.c_uint32),
                ("learned_min_inliers", ctypes.c_int32), ("scoring", ctypes.c_int32)]


class turboreg_result(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("clique", ctypes.c_int32 * 3),
                ("inlier_count", ctypes.c_int32), ("hypothesis", ctypes.c_int32),
                ("n_pivots", ctypes.c_int32), ("n_valid", ctypes.c_int32), ("used_fp64", ctypes.c_int32),
                ("used_fallback", ctypes.c_int32), ("status", ctypes.c_int32), ("score", ctypes.c_float)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load the CUDA library; raise if it is missing (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"TurboReg CUDA library not built: {path} is missing "
                           "(run __graft_entry__.build() or python -m paper_2507_01439_gb300.build)")
    lib = ctypes.CDLL(path)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.turboreg_default_params.argtypes = [ctypes.POINTER(turboreg_params), ctypes.c_float, i32, ctypes.c_float]
    lib.turboreg_default_params.restype = None
    lib.turboreg_create.argtypes = [ctypes.c_int, i32, i32, P, ctypes.POINTER(P)]
    lib.turboreg_create.restype = ctypes.c_int
    lib.turboreg_register.argtypes = [P, P, P, i32, ctypes.POINTER(turboreg_params),
                                      ctypes.POINTER(turboreg_result)]
    lib.turboreg_register.restype = ctypes.c_int
    lib.turboreg_register_batched.argtypes = [P, P, P, P, i32, ctypes.POINTER(turboreg_params), i32,
                                              ctypes.POINTER(turboreg_result)]
    lib.turboreg_register_batched.restype = ctypes.c_int
    lib.turboreg_register_async.argtypes = [P, P, P, i32, ctypes.POINTER(turboreg_params), P]
    lib.turboreg_register_async.restype = ctypes.c_int
    lib.turboreg_synchronize.argtypes = [P]
    lib.turboreg_synchronize.restype = ctypes.c_int
    lib.turboreg_destroy.argtypes = [P]
    lib.turboreg_destroy.restype = None
    lib.turboreg_status_string.argtypes = [ctypes.c_int]
    lib.turboreg_status_string.restype = ctypes.c_char_p
    lib.turboreg_debug_shape.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                         ctypes.POINTER(i32)]
    lib.turboreg_debug_shape.restype = ctypes.c_int
    lib.turboreg_debug_sc2_path.argtypes = [P, ctypes.POINTER(i32)]
    lib.turboreg_debug_sc2_path.restype = ctypes.c_int
    lib.turboreg_debug_copy.argtypes = [P, ctypes.c_int, P, i64]
    lib.turboreg_debug_copy.restype = i64
    lib.turboreg_stage_times.argtypes = [P, ctypes.POINTER(ctypes.c_float), i32]
    lib.turboreg_stage_times.restype = ctypes.c_int
    lib.turboreg_stage_name.argtypes = [i32]
    lib.turboreg_stage_name.restype = ctypes.c_char_p
    lib.turboreg_select_pivots_noalloc.argtypes = [P, i32, i32, i32, P, P, P]
    lib.turboreg_select_pivots_noalloc.restype = ctypes.c_int
    F = ctypes.POINTER(ctypes.c_float)
    lib.turboreg_score_transforms.argtypes = [P, P, P, i32, ctypes.POINTER(turboreg_params), P, i32, P, P]
    lib.turboreg_score_transforms.restype = ctypes.c_int
    lib.turboreg_kabsch_cliques.argtypes = [P, P, P, i32, ctypes.POINTER(turboreg_params), P, i32, i32, P, P]
    lib.turboreg_kabsch_cliques.restype = ctypes.c_int
    lib.turboreg_set_proposal_model.argtypes = [P, P]
    lib.turboreg_features.argtypes = [P, P, P, i32, ctypes.POINTER(turboreg_params), P]
    lib.turboreg_mlp_create.argtypes = [ctypes.c_int, i32, ctypes.c_uint64, P, ctypes.POINTER(P)]
    lib.turboreg_mlp_destroy.argtypes = [P]
    lib.turboreg_mlp_destroy.restype = None
    lib.turboreg_mlp_get_params.argtypes = [P, P]
    lib.turboreg_mlp_set_params.argtypes = [P, P]
    lib.turboreg_mlp_get_state.argtypes = [P, P, P, ctypes.POINTER(i32)]
    lib.turboreg_mlp_set_state.argtypes = [P, P, P, i32]
    lib.turboreg_mlp_forward.argtypes = [P, P, i32, P]
    lib.turboreg_mlp_grad.argtypes = [P, P, P, i32, P, F]
    lib.turboreg_mlp_train_step.argtypes = [P, P, P, i32, ctypes.c_float, F]
    for nm in ("turboreg_set_proposal_model", "turboreg_features", "turboreg_mlp_create", "turboreg_mlp_get_params",
               "turboreg_mlp_set_params", "turboreg_mlp_get_state", "turboreg_mlp_set_state",
               "turboreg_mlp_forward", "turboreg_mlp_grad", "turboreg_mlp_train_step"):
        getattr(lib, nm).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a):
    """Raw address of a NumPy array or a torch tensor (host or CUDA)."""
    if isinstance(a, np.ndarray):
        return ctypes.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError("expected a numpy array or a torch tensor")


def _check_points(a, n=None):
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or a.ndim != 2 or a.shape[1] != 3 or not a.flags.c_contiguous:
            raise ValueError("points must be C-contiguous float32 [N,3]")
    else:
        import torch
        if a.dtype != torch.float32 or a.dim() != 2 or a.shape[1] != 3 or not a.is_contiguous():
            raise ValueError("points must be contiguous float32 [N,3]")
    if n is not None and a.shape[0] != n:
        raise ValueError("src and dst must have the same number of rows")


def default_params(tau, k1, inlier_thresh, k2=2, kappa_fp64=100.0, flags=0, proposal=PROPOSAL_PLAIN,
                   learned_min_inliers=0, graph_mode=GRAPH_O2, scoring=SCORE_IN):
    p = turboreg_params()
    load_library().turboreg_default_params(ctypes.byref(p), float(tau), int(k1), float(inlier_thresh))
    p.k2 = int(k2)
    p.kappa_fp64 = float(kappa_fp64)
    p.flags = int(flags)
    p.proposal = int(proposal)
    p.learned_min_inliers = int(learned_min_inliers)
    p.graph_mode = int(graph_mode)
    p.scoring = int(scoring)
    return p


def score_values(units, inl, params, n):
    """Selection scores from the library's integer outputs: the inlier
    number (SCORE_IN), or the capped error sums (BUF_SCORES units) as means
    in metres (MAE) or square metres (MSE)."""
    if params.scoring == SCORE_IN:
        return np.asarray(inl, dtype=np.float64)
    th = float(np.float32(params.inlier_thresh))
    unit = th if params.scoring == SCORE_MAE else th * th
    return np.asarray(units, dtype=np.float64) * unit / (SCORE_UNITS * n)


def status_string(code: int) -> str:
    return load_library().turboreg_status_string(int(code)).decode()


@dataclass
class Result:
    status: int
    R: np.ndarray
    t: np.ndarray
    clique: tuple
    inlier_count: int
    hypothesis: int
    n_pivots: int
    n_valid: int
    used_fp64: int
    used_fallback: int
    score: float = 0.0

    @staticmethod
    def from_c(r: turboreg_result) -> "Result":
        return Result(int(r.status), np.array(r.R[:], dtype=np.float32).reshape(3, 3),
                      np.array(r.t[:], dtype=np.float32), tuple(r.clique[:]), int(r.inlier_count),
                      int(r.hypothesis), int(r.n_pivots), int(r.n_valid), int(r.used_fp64),
                      int(r.used_fallback), float(r.score))


class ResultSlots:
    """Page-locked host memory for `count` results of register_async (read
    them after TurboReg.synchronize())."""

    def __init__(self, count: int):
        import torch
        self.count = int(count)
        self._buf = torch.empty(self.count * ctypes.sizeof(turboreg_result), dtype=torch.uint8, pin_memory=True)

    def address(self, k: int):
        if not 0 <= k < self.count:
            raise IndexError(k)
        return ctypes.c_void_p(self._buf.data_ptr() + k * ctypes.sizeof(turboreg_result))

    def result(self, k: int) -> "Result":
        return Result.from_c(turboreg_result.from_address(self.address(k).value))


class TurboReg:
    """One library context (device workspace sized for max_n); not thread-safe."""

    def __init__(self, max_n=5000, max_batch=1, device=0, stream=None):
        self._lib = load_library()
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream) if stream else None
        rc = self._lib.turboreg_create(int(device), int(max_n), int(max_batch), st, ctypes.byref(h))
        if rc != OK:
            raise RuntimeError(f"turboreg_create failed: {status_string(rc)}")
        self.handle = h
        self.max_n = max_n

    def close(self):
        if getattr(self, "handle", None):
            self._lib.turboreg_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def register(self, src, dst, params: turboreg_params) -> Result:
        _check_points(src)
        _check_points(dst, src.shape[0])
        out = turboreg_result()
        self._lib.turboreg_register(self.handle, _ptr(src), _ptr(dst), int(src.shape[0]),
                                    ctypes.byref(params), ctypes.byref(out))
        return Result.from_c(out)

    def register_async(self, src, dst, params: turboreg_params, slots, k: int = 0) -> None:
        """Enqueue one registration on the context's stream without waiting;
        its result lands in slot k of `slots` (a ResultSlots) once
        synchronize() returns.  src, dst: CUDA tensors or page-locked host
        tensors, unchanged until then."""
        _check_points(src)
        _check_points(dst, src.shape[0])
        rc = self._lib.turboreg_register_async(self.handle, _ptr(src), _ptr(dst), int(src.shape[0]),
                                               ctypes.byref(params), slots.address(k))
        if rc != OK:
            raise RuntimeError(f"turboreg_register_async failed: {status_string(rc)}")

    def synchronize(self) -> None:
        rc = self._lib.turboreg_synchronize(self.handle)
        if rc != OK:
            raise RuntimeError(f"turboreg_synchronize failed: {status_string(rc)}")

    def register_batched(self, src_cat, dst_cat, offsets, params) -> list:
        _check_points(src_cat)
        _check_points(dst_cat, src_cat.shape[0])
        offs = np.ascontiguousarray(offsets, dtype=np.int64)
        num = offs.shape[0] - 1
        if isinstance(params, turboreg_params):
            parr, pc = (turboreg_params * 1)(params), 1
        else:
            parr, pc = (turboreg_params * len(params))(*params), len(params)
        out = (turboreg_result * num)()
        rc = self._lib.turboreg_register_batched(self.handle, _ptr(src_cat), _ptr(dst_cat),
                                                 ctypes.c_void_p(offs.ctypes.data), num, parr, pc, out)
        if rc != OK:
            raise RuntimeError(f"turboreg_register_batched failed: {status_string(rc)}")
        return [Result.from_c(out[b]) for b in range(num)]

    def marshal_batched(self, offsets, params):
        """Pre-built arguments of register_batched_raw: (offsets int64 array,
        ctypes params array, its count, ctypes result array)."""
        offs = np.ascontiguousarray(offsets, dtype=np.int64)
        num = offs.shape[0] - 1
        if isinstance(params, turboreg_params):
            parr, pc = (turboreg_params * 1)(params), 1
        else:
            parr, pc = (turboreg_params * len(params))(*params), len(params)
        return offs, parr, pc, (turboreg_result * num)()

    def register_batched_raw(self, src_cat, dst_cat, marshalled) -> int:
        """turboreg_register_batched on arguments prepared once by
        marshal_batched (no per-call conversion); returns the status code,
        results in marshalled[3]."""
        offs, parr, pc, out = marshalled
        return self._lib.turboreg_register_batched(self.handle, _ptr(src_cat), _ptr(dst_cat),
                                                   ctypes.c_void_p(offs.ctypes.data), offs.shape[0] - 1,
                                                   parr, pc, out)

    # ---- inspection (internal header) ----
    def shape(self):
        n, npad, npiv, nh = (ctypes.c_int32() for _ in range(4))
        rc = self._lib.turboreg_debug_shape(self.handle, ctypes.byref(n), ctypes.byref(npad),
                                            ctypes.byref(npiv), ctypes.byref(nh))
        if rc != OK:
            raise RuntimeError(status_string(rc))
        return n.value, npad.value, npiv.value, nh.value

    def sc2_path(self):
        """SC^2 path of the last registration: 1 CUDA-core bitset form, 2 tensor-core GEMM."""
        p = ctypes.c_int32()
        rc = self._lib.turboreg_debug_sc2_path(self.handle, ctypes.byref(p))
        if rc != OK:
            raise RuntimeError(status_string(rc))
        return p.value

    def buffer(self, which: int) -> np.ndarray:
        n, npad, npiv, nh = self.shape()
        spec = {
            BUF_ADJ_BITS: (np.uint32, (npad, npad // 32)),
            BUF_ADJ_FP8: (np.uint8, (npad, npad)),
            BUF_SC2: (np.uint16, (npad, npad)),
            BUF_PIVOTS: (np.int32, (npiv, 4)),
            BUF_CLIQUES: (np.int32, (nh, 4)),
            BUF_RT: (np.float32, (nh, 16)),
            BUF_INLIERS: (np.int32, (nh,)),
            BUF_ROWSCORE: (np.int32, (n,)),
            BUF_DEGREE: (np.int32, (n,)),
            BUF_FEATURES: (np.float32, (n, 8)),
            BUF_PROB: (np.float32, (n,)),
            BUF_SCORES: (np.uint64, (nh,)),
        }[which]
        arr = np.zeros(spec[1], dtype=spec[0])
        got = self._lib.turboreg_debug_copy(self.handle, int(which), ctypes.c_void_p(arr.ctypes.data),
                                            arr.nbytes)
        if got < 0:
            raise RuntimeError(status_string(-got))
        return arr

    def score_transforms(self, src, dst, params, rt):
        """Score transforms rt [m, 12] (R row-major, t) on one problem with the
        library's verification kernel: (inlier numbers int32 [m], selection
        scores float64 [m]: the inlier number, or the capped MAE / MSE)."""
        _check_points(src)
        _check_points(dst, src.shape[0])
        rt = np.ascontiguousarray(rt, dtype=np.float32).reshape(-1, 12)
        m = rt.shape[0]
        n = int(src.shape[0])
        inl = np.zeros(m, dtype=np.int32)
        units = np.zeros(m, dtype=np.uint64)
        rc = self._lib.turboreg_score_transforms(self.handle, _ptr(src), _ptr(dst), n, ctypes.byref(params),
                                                 ctypes.c_void_p(rt.ctypes.data), m,
                                                 ctypes.c_void_p(inl.ctypes.data),
                                                 ctypes.c_void_p(units.ctypes.data))
        if rc != OK:
            raise RuntimeError(f"turboreg_score_transforms failed: {status_string(rc)}")
        return inl, score_values(units, inl, params, n)

    def kabsch_cliques(self, src, dst, idx, params=None):
        """Kabsch of index tuples idx [m, k] (3 <= k <= 32): (rt float32 [m, 12]
        = R row-major then t, valid bool [m]).  k = 3 runs the registration
        path's closed form; k >= 4 runs Horn's method in FP64."""
        _check_points(src)
        _check_points(dst, src.shape[0])
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        if idx.ndim != 2:
            raise ValueError("idx must be [m, k]")
        m, k = idx.shape
        prm = params if params is not None else default_params(0.0, 1, 1.0)
        rt = np.zeros((m, 12), dtype=np.float32)
        valid = np.zeros(m, dtype=np.int32)
        rc = self._lib.turboreg_kabsch_cliques(self.handle, _ptr(src), _ptr(dst), int(src.shape[0]),
                                               ctypes.byref(prm), ctypes.c_void_p(idx.ctypes.data), k, m,
                                               ctypes.c_void_p(rt.ctypes.data), ctypes.c_void_p(valid.ctypes.data))
        if rc != OK:
            raise RuntimeError(f"turboreg_kabsch_cliques failed: {status_string(rc)}")
        return rt, valid.astype(bool)

    def set_proposal_model(self, params):
        w = np.ascontiguousarray(params, dtype=np.float32)
        if w.shape != (TURBOREG_MLP_PARAMS,):
            raise ValueError("proposal model needs TURBOREG_MLP_PARAMS float32 values")
        rc = self._lib.turboreg_set_proposal_model(self.handle, ctypes.c_void_p(w.ctypes.data))
        if rc != OK:
            raise RuntimeError(f"turboreg_set_proposal_model failed: {status_string(rc)}")

    def features(self, src, dst, params, out=None):
        """Proposal features [n, 8] (float32); `out` may be a CUDA tensor."""
        _check_points(src)
        _check_points(dst, src.shape[0])
        n = int(src.shape[0])
        if out is None:
            out = np.zeros((n, 8), dtype=np.float32)
        rc = self._lib.turboreg_features(self.handle, _ptr(src), _ptr(dst), n, ctypes.byref(params), _ptr(out))
        if rc != OK:
            raise RuntimeError(f"turboreg_features failed: {status_string(rc)}")
        return out

    def stage_times(self):
        buf = (ctypes.c_float * 16)()
        k = self._lib.turboreg_stage_times(self.handle, buf, 16)
        return {self._lib.turboreg_stage_name(i).decode(): float(buf[i]) for i in range(k)}


# ---- the C ABI under its own names (argument marshalling only) ----

def turboreg_create(device=0, max_n=5000, max_batch=1, stream=None) -> TurboReg:
    return TurboReg(max_n=max_n, max_batch=max_batch, device=device, stream=stream)


def turboreg_register(ctx: TurboReg, src, dst, params: turboreg_params) -> Result:
    return ctx.register(src, dst, params)


def turboreg_register_batched(ctx: TurboReg, src_cat, dst_cat, offsets, params) -> list:
    return ctx.register_batched(src_cat, dst_cat, offsets, params)


def turboreg_destroy(ctx: TurboReg) -> None:
    ctx.close()


def turboreg_select_pivots_noalloc(w_dev, n, ldw, k1, pivots_dev, n_pivots_dev, stream=None) -> int:
    """Pivot selection on a device weight matrix without any allocation (see
    include/turboreg_internal.h): w_dev uint16 [n, ldw] CUDA tensor, outputs
    pivots_dev int32 [k1, 4] and n_pivots_dev int32 [1] CUDA tensors."""
    st = ctypes.c_void_p(stream) if stream else None
    return load_library().turboreg_select_pivots_noalloc(_ptr(w_dev), int(n), int(ldw), int(k1),
                                                         _ptr(pivots_dev), _ptr(n_pivots_dev), st)


class MLPTrainer:
    """Device-side trainer of the proposal MLP (forward/backward/Adam kernels)."""

    def __init__(self, max_samples=65536, seed=0, device=0, stream=None):
        self._lib = load_library()
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream) if stream else None
        rc = self._lib.turboreg_mlp_create(int(device), int(max_samples), int(seed), st, ctypes.byref(h))
        if rc != OK:
            raise RuntimeError(f"turboreg_mlp_create failed: {status_string(rc)}")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self._lib.turboreg_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc, what):
        if rc != OK:
            raise RuntimeError(f"{what} failed: {status_string(rc)}")

    def get_params(self):
        w = np.zeros(TURBOREG_MLP_PARAMS, dtype=np.float32)
        self._chk(self._lib.turboreg_mlp_get_params(self.handle, ctypes.c_void_p(w.ctypes.data)), "get_params")
        return w

    def set_params(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        self._chk(self._lib.turboreg_mlp_set_params(self.handle, ctypes.c_void_p(w.ctypes.data)), "set_params")

    def get_state(self):
        m = np.zeros(TURBOREG_MLP_PARAMS, dtype=np.float32)
        v = np.zeros_like(m)
        st = ctypes.c_int32()
        self._chk(self._lib.turboreg_mlp_get_state(self.handle, ctypes.c_void_p(m.ctypes.data),
                                                   ctypes.c_void_p(v.ctypes.data), ctypes.byref(st)), "get_state")
        return m, v, int(st.value)

    def set_state(self, m, v, step):
        m = np.ascontiguousarray(m, dtype=np.float32)
        v = np.ascontiguousarray(v, dtype=np.float32)
        self._chk(self._lib.turboreg_mlp_set_state(self.handle, ctypes.c_void_p(m.ctypes.data),
                                                   ctypes.c_void_p(v.ctypes.data), int(step)), "set_state")

    def forward(self, feat_dev, prob_dev):
        self._chk(self._lib.turboreg_mlp_forward(self.handle, _ptr(feat_dev), int(feat_dev.shape[0]),
                                                 _ptr(prob_dev)), "forward")

    def grad(self, feat_dev, label_dev):
        g = np.zeros(TURBOREG_MLP_PARAMS, dtype=np.float32)
        loss = ctypes.c_float()
        self._chk(self._lib.turboreg_mlp_grad(self.handle, _ptr(feat_dev), _ptr(label_dev), int(feat_dev.shape[0]),
                                              ctypes.c_void_p(g.ctypes.data), ctypes.byref(loss)), "grad")
        return g, float(loss.value)

    def train_step(self, feat_dev, label_dev, lr, want_loss=False):
        loss = ctypes.c_float()
        self._chk(self._lib.turboreg_mlp_train_step(self.handle, _ptr(feat_dev), _ptr(label_dev),
                                                    int(feat_dev.shape[0]), float(lr),
                                                    ctypes.byref(loss) if want_loss else None), "train_step")
        return float(loss.value) if want_loss else None

    # checkpoint: flat binary with a header (magic, version, params, step, seed) + weights + Adam moments
    def save(self, path, seed=0):
        w = self.get_params()
        m, v, step = self.get_state()
        hdr = np.array([0x54524D4C, 1, TURBOREG_MLP_PARAMS, step, seed], dtype=np.int64)
        with open(path, "wb") as f:
            f.write(hdr.tobytes()); f.write(w.tobytes()); f.write(m.tobytes()); f.write(v.tobytes())

    def load(self, path):
        w, m, v, step = load_checkpoint(path)
        self.set_params(w)
        self.set_state(m, v, step)
        return step


def load_checkpoint(path):
    """(params, adam_m, adam_v, step) of a checkpoint written by MLPTrainer.save."""
    raw = open(path, "rb").read()
    hdr = np.frombuffer(raw[:40], dtype=np.int64)
    if hdr[0] != 0x54524D4C or hdr[2] != TURBOREG_MLP_PARAMS:
        raise ValueError(f"{path}: not a proposal-MLP checkpoint")
    P = TURBOREG_MLP_PARAMS
    body = np.frombuffer(raw[40:], dtype=np.float32)
    return body[:P].copy(), body[P:2 * P].copy(), body[2 * P:3 * P].copy(), int(hdr[3])
