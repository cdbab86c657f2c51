"""Autotuner of the batched registration form.

It picks, by measurement on the device at hand:

  tile shapes  the SC^2 GEMM form (2-CTA pair MMAs or independent
               128 x 256 CTAs) and the
               verification tile (128 hypotheses x 128 / 256 / 512 matches per
               block); every candidate gives the same results, only the time
               differs;
  K schedule   the pivot count K1 per problem class (compatibility threshold
               tau and a bucket of N): the smallest candidate K1 whose success
               rate on calibration problems equals the best candidate's, i.e.
               the cheapest K1 at equal success rate.

Calibration problems come from the caller with their ground truth (the
library has no generator of its own); success is rotation error < re_deg and
translation error < te_m, as in the paper's evaluation (Sec. 4.1).  The
result is a Schedule that turns (N, tau, theta) into turboreg_params, and can
be stored as JSON next to the caller's data.
"""
from __future__ import annotations

import json
import time
from dataclasses import asdict, dataclass, field

import numpy as np

from . import (FLAG_SC2_BITSET, FLAG_SC2_SINGLE_CTA, FLAG_VERIFY_PTS32, FLAG_VERIFY_PTS128, TurboReg,
               default_params)

TILE_CANDIDATES = {
    "sc2_pair+verify256": 0,
    "sc2_pair+verify128": FLAG_VERIFY_PTS32,
    "sc2_pair+verify512": FLAG_VERIFY_PTS128,
    "sc2_single+verify256": FLAG_SC2_SINGLE_CTA,
    "sc2_single+verify512": FLAG_SC2_SINGLE_CTA | FLAG_VERIFY_PTS128,
    "sc2_bitset+verify256": FLAG_SC2_BITSET,
}


@dataclass
class Calib:
    """One calibration problem: matches and ground truth."""
    x: np.ndarray            # float32 [n, 3]
    y: np.ndarray            # float32 [n, 3]
    R_gt: np.ndarray         # [3, 3]
    t_gt: np.ndarray         # [3]
    tau: float
    theta: float
    re_deg: float
    te_m: float


@dataclass
class Schedule:
    flags: int = 0                                   # tile-shape flags of every batched call
    tile: str = "sc2_pair+verify256"
    k1_rules: list = field(default_factory=list)     # [tau, n_max, k1], first match wins
    default_k1: int = 1000
    timings_ms: dict = field(default_factory=dict)   # per tile candidate
    success: dict = field(default_factory=dict)      # per class and K1 candidate

    def k1_for(self, n: int, tau: float) -> int:
        same = sorted((r for r in self.k1_rules
                       if abs(float(r[0]) - float(tau)) <= 1e-6 * max(1.0, abs(float(tau)))),
                      key=lambda r: r[1])
        for _, n_max, k1 in same:
            if n <= n_max:
                return int(k1)
        # larger than every calibrated bucket: the largest bucket's K1
        return int(same[-1][2]) if same else int(self.default_k1)

    def params(self, n: int, tau: float, theta: float, **kw):
        p = default_params(tau, self.k1_for(n, tau), theta, **kw)
        p.flags |= self.flags
        return p

    def to_json(self) -> str:
        return json.dumps(asdict(self), indent=1)

    @staticmethod
    def from_json(text: str) -> "Schedule":
        return Schedule(**json.loads(text))


def _success(res, prob: Calib) -> bool:
    if res.status != 0:
        return False
    c = (np.trace(np.asarray(prob.R_gt, np.float64).T @ res.R.astype(np.float64)) - 1.0) / 2.0
    re = float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))
    te = float(np.linalg.norm(res.t.astype(np.float64) - np.asarray(prob.t_gt, np.float64)))
    return re < prob.re_deg and te < prob.te_m


def _batch_arrays(problems):
    offs = np.cumsum([0] + [p.x.shape[0] for p in problems]).astype(np.int64)
    xs = np.ascontiguousarray(np.concatenate([p.x for p in problems]), dtype=np.float32)
    ys = np.ascontiguousarray(np.concatenate([p.y for p in problems]), dtype=np.float32)
    try:   # device-resident inputs keep host copies out of the timings
        import torch
        if torch.cuda.is_available():
            return torch.from_numpy(xs).cuda(), torch.from_numpy(ys).cuda(), offs
    except ImportError:
        pass
    return xs, ys, offs


def choose_k1(success_by_k1: dict) -> int:
    """Smallest K1 whose success count equals the best one (equal success rate)."""
    best = max(success_by_k1.values())
    return min(k for k, s in success_by_k1.items() if s >= best)


def class_key(tau: float, n: int, bucket_edges) -> tuple:
    for e in bucket_edges:
        if n <= e:
            return (float(tau), int(e))
    return (float(tau), int(bucket_edges[-1]))


def tune(ctx: TurboReg, problems, k1_candidates=(100, 250, 500, 1000, 2000),
         bucket_edges=(1500, 3000, 5000), tiles=None, reps=3, log=None) -> Schedule:
    """Measure tile shapes and K1 candidates on `problems` (list of Calib)."""
    tiles = TILE_CANDIDATES if tiles is None else tiles
    xs, ys, offs = _batch_arrays(problems)
    k_top = max(k1_candidates)

    def run(k1_of, flags):
        prm = []
        for p in problems:
            q = default_params(p.tau, k1_of(p), p.theta)
            q.flags |= flags
            prm.append(q)
        return ctx.register_batched(xs, ys, offs, prm)

    # 1. tile shapes at the largest K1 (the most verification work)
    timings = {}
    for name, fl in tiles.items():
        run(lambda p: k_top, fl)                      # capture the graph of this plan
        best = float("inf")
        for _ in range(reps):
            t0 = time.perf_counter()
            run(lambda p: k_top, fl)
            best = min(best, time.perf_counter() - t0)
        timings[name] = 1e3 * best
        if log:
            log(f"  tile {name}: {timings[name]:.2f} ms")
    tile = min(timings, key=timings.get)
    flags = tiles[tile]

    # 2. K1 schedule per (tau, N bucket): cheapest K1 at the best success rate
    succ = {}
    for k1 in sorted(k1_candidates):
        out = run(lambda p: k1, flags)
        for p, r in zip(problems, out):
            key = class_key(p.tau, p.x.shape[0], bucket_edges)
            succ.setdefault(key, {}).setdefault(k1, 0)
            succ[key][k1] += int(_success(r, p))
    rules = []
    for (tau, edge), by_k in sorted(succ.items()):
        k1 = choose_k1(by_k)
        rules.append([tau, edge, k1])
        if log:
            log(f"  tau {tau:g}, N <= {edge}: success {by_k} -> K1 = {k1}")
    return Schedule(flags=flags, tile=tile, k1_rules=rules, default_k1=k_top, timings_ms=timings,
                    success={f"{t:g}/{e}": {str(k): v for k, v in by_k.items()} for (t, e), by_k in succ.items()})
