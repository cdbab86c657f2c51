"""FP64 CPU oracle of the TurboReg registration path (ctypes wrapper).

TEST INFRASTRUCTURE.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never touches it, and the two share
no code.

The arithmetic lives in ``turboreg_oracle.c`` (plain C, double precision,
``-ffp-contract=off``); this module compiles it with gcc on first use and
wraps each stage for NumPy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "turboreg_oracle.c")
_HDR = os.path.join(_HERE, "turboreg_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (gcc, portable C)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = force or not os.path.exists(_LIB) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class OrcParams(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_float), ("k1", ctypes.c_int32), ("k2", ctypes.c_int32),
                ("theta", ctypes.c_float), ("near_band", ctypes.c_double),
                ("graph_mode", ctypes.c_int32), ("scoring", ctypes.c_int32)]


class OrcResult(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3),
                ("clique", ctypes.c_int32 * 3), ("inlier_count", ctypes.c_int32),
                ("hypothesis", ctypes.c_int32), ("n_pivots", ctypes.c_int32),
                ("n_valid", ctypes.c_int32), ("status", ctypes.c_int32),
                ("kappa", ctypes.c_double), ("score", ctypes.c_double)]

GRAPH_O2, GRAPH_SC2 = 0, 1
SCORE_IN, SCORE_MAE, SCORE_MSE = 0, 1, 2


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32 = ctypes.c_int32
        lib.orc_compat.argtypes = [P, P, i32, ctypes.c_float, P]
        lib.orc_sc2.argtypes = [P, i32, P]
        lib.orc_pivots.argtypes = [P, i32, i32, P, P, P]
        lib.orc_pivots.restype = i32
        lib.orc_cliques.argtypes = [P, i32, P, P, i32, i32, i32, P, P]
        lib.orc_kabsch.argtypes = [P, P, P, P, P]
        lib.orc_kabsch.restype = i32
        lib.orc_kabsch_n.argtypes = [P, P, i32, P, P, P]
        lib.orc_kabsch_n.restype = i32
        lib.orc_svd3.argtypes = [P, P, P, P]
        lib.orc_inliers.argtypes = [P, P, i32, P, P, ctypes.c_float, ctypes.c_double, P]
        lib.orc_inliers.restype = i32
        lib.orc_score.argtypes = [P, P, i32, P, P, ctypes.c_float, i32]
        lib.orc_score.restype = ctypes.c_double
        lib.orc_register.argtypes = [P, P, i32, ctypes.POINTER(OrcParams),
                                     ctypes.POINTER(OrcResult), P, P, P, P, P]
        lib.orc_register.restype = i32
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _pts(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    assert a.ndim == 2 and a.shape[1] == 3
    return a


def compat(x, y, tau) -> np.ndarray:
    """Eq. 1: uint8 [n,n] compatibility graph, zero diagonal."""
    x, y = _pts(x), _pts(y)
    n = x.shape[0]
    A = np.zeros((n, n), dtype=np.uint8)
    _load().orc_compat(_p(x), _p(y), n, float(np.float32(tau)), _p(A))
    return A


def sc2(A) -> np.ndarray:
    """Eq. 2: int32 [n,n] SC^2 graph of a 0/1 matrix."""
    A = np.ascontiguousarray(A, dtype=np.uint8)
    n = A.shape[0]
    S = np.zeros((n, n), dtype=np.int32)
    _load().orc_sc2(_p(A), n, _p(S))
    return S


def pivots(S, k1):
    """Eq. 4 on the O2Graph: (pi, pj, pw) int32 arrays of length |P|."""
    S = np.ascontiguousarray(S, dtype=np.int32)
    n = S.shape[0]
    pi = np.zeros(max(k1, 1), dtype=np.int32)
    pj = np.zeros_like(pi)
    pw = np.zeros_like(pi)
    m = _load().orc_pivots(_p(S), n, k1, _p(pi), _p(pj), _p(pw))
    if m < 0:
        raise MemoryError("oracle pivot selection failed to allocate")
    return pi[:m].copy(), pj[:m].copy(), pw[:m].copy()


def cliques(S, pi, pj, k2, graph_mode=GRAPH_O2):
    """Eq. 5-7: (cliques int32 [k2*|P|, 3], valid bool [k2*|P|]) in Alg. 2 order,
    searched on the O2Graph (graph_mode 0) or the undirected SC^2 graph (1)."""
    S = np.ascontiguousarray(S, dtype=np.int32)
    pi = np.ascontiguousarray(pi, dtype=np.int32)
    pj = np.ascontiguousarray(pj, dtype=np.int32)
    np_ = pi.shape[0]
    cl = np.zeros((max(np_ * k2, 1), 3), dtype=np.int32)
    va = np.zeros(max(np_ * k2, 1), dtype=np.uint8)
    _load().orc_cliques(_p(S), S.shape[0], _p(pi), _p(pj), np_, k2, int(graph_mode), _p(cl), _p(va))
    return cl[:np_ * k2].copy(), va[:np_ * k2].astype(bool)


def svd3(H):
    H = np.ascontiguousarray(H, dtype=np.float64)
    U = np.zeros((3, 3)); s = np.zeros(3); V = np.zeros((3, 3))
    _load().orc_svd3(_p(H), _p(U), _p(s), _p(V))
    return U, s, V


def kabsch(xs, ys):
    """Kabsch on 3 matches: (valid, R [3,3], t [3], kappa)."""
    xs = np.ascontiguousarray(xs, dtype=np.float64)
    ys = np.ascontiguousarray(ys, dtype=np.float64)
    R = np.zeros((3, 3)); t = np.zeros(3); k = np.zeros(1)
    ok = _load().orc_kabsch(_p(xs), _p(ys), _p(R), _p(t), _p(k))
    return bool(ok), R, t, float(k[0])


def kabsch_n(xs, ys):
    """Kabsch on m >= 3 matches: (valid, R [3,3], t [3], kappa)."""
    xs = np.ascontiguousarray(xs, dtype=np.float64)
    ys = np.ascontiguousarray(ys, dtype=np.float64)
    R = np.zeros((3, 3)); t = np.zeros(3); k = np.zeros(1)
    ok = _load().orc_kabsch_n(_p(xs), _p(ys), xs.shape[0], _p(R), _p(t), _p(k))
    return bool(ok), R, t, float(k[0])


def inliers(x, y, R, t, theta, band=0.0):
    """(inlier number, near-threshold count) of one hypothesis."""
    x, y = _pts(x), _pts(y)
    R = np.ascontiguousarray(R, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    near = np.zeros(1, dtype=np.int32)
    c = _load().orc_inliers(_p(x), _p(y), x.shape[0], _p(R), _p(t),
                            float(np.float32(theta)), float(band), _p(near))
    return int(c), int(near[0])


def score(x, y, R, t, theta, mode):
    """Selection score of one hypothesis: IN (mode 0), or the mean residual
    capped at theta (MAE, mode 1) / mean squared residual capped at theta^2
    (MSE, mode 2)."""
    x, y = _pts(x), _pts(y)
    R = np.ascontiguousarray(R, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    return float(_load().orc_score(_p(x), _p(y), x.shape[0], _p(R), _p(t),
                                   float(np.float32(theta)), int(mode)))


@dataclass
class OracleResult:
    status: int
    R: np.ndarray
    t: np.ndarray
    clique: tuple
    inlier_count: int
    hypothesis: int
    n_pivots: int
    n_valid: int
    kappa: float
    in_counts: np.ndarray      # int32 [k1*k2], -1 where no valid hypothesis
    near_counts: np.ndarray    # int32 [k1*k2]
    rt: np.ndarray             # float64 [k1*k2, 12]
    hyp_valid: np.ndarray      # bool [k1*k2]
    score: float = 0.0         # the winner's selection score
    scores: np.ndarray = None  # float64 [k1*k2], NaN where no valid hypothesis


def register(x, y, tau, k1, theta, k2=2, near_band=1e-5, graph_mode=GRAPH_O2,
             scoring=SCORE_IN) -> OracleResult:
    """The whole path (Eq. 1 -> Eq. 9) in FP64 on one host core."""
    x, y = _pts(x), _pts(y)
    n = x.shape[0]
    prm = OrcParams(float(np.float32(tau)), int(k1), int(k2),
                    float(np.float32(theta)), float(near_band), int(graph_mode), int(scoring))
    res = OrcResult()
    nh = max(int(k1) * int(k2), 1)
    inc = np.zeros(nh, dtype=np.int32)
    nec = np.zeros(nh, dtype=np.int32)
    rt = np.zeros((nh, 12), dtype=np.float64)
    hv = np.zeros(nh, dtype=np.uint8)
    sc = np.zeros(nh, dtype=np.float64)
    _load().orc_register(_p(x), _p(y), n, ctypes.byref(prm), ctypes.byref(res),
                         _p(inc), _p(nec), _p(rt), _p(hv), _p(sc))
    return OracleResult(
        status=int(res.status), R=np.array(res.R[:]).reshape(3, 3), t=np.array(res.t[:]),
        clique=tuple(res.clique[:]), inlier_count=int(res.inlier_count),
        hypothesis=int(res.hypothesis), n_pivots=int(res.n_pivots),
        n_valid=int(res.n_valid), kappa=float(res.kappa),
        in_counts=inc, near_counts=nec, rt=rt, hyp_valid=hv.astype(bool),
        score=float(res.score), scores=sc)
