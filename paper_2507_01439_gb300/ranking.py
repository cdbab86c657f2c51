"""Ranking-based registration recall of the hypotheses Pivot-Guided Search
produces (the ranking study of Table 6).

For one problem with a known ground truth (R_gt, t_gt) and known inlier
flags, the K1*K2 hypotheses of a register call are ranked by the selection
score (inlier number IN, larger first; capped MAE or MSE, smaller first;
ties to the lower hypothesis index h, as the selection itself) and:

  RR     the top-1 hypothesis is a successful registration
         (rotation error < re_deg and translation error < te_m, Sec. 4.1);
  TQRR   the top-1 hypothesis scores at least as well as the ground-truth
         transform under the same score;
  ICRR   the top-1 hypothesis's TurboClique consists of three inliers;
  TKRR@K at least one of the top-K hypotheses is a successful registration.

The hypotheses come from the library's stage buffers and the ground truth is
scored by the library's verification kernel (turboreg_score_transforms), so
every number here comes from the CUDA path; this module only ranks and counts.
"""
from __future__ import annotations

import numpy as np

from . import (BUF_CLIQUES, BUF_INLIERS, BUF_RT, BUF_SCORES, SCORE_IN, TurboReg, score_values)

KS = (2, 3, 5, 50)


def rotation_error_deg(R_gt, R) -> float:
    """arccos((tr(R_gt^T R) - 1) / 2) in degrees."""
    c = (np.trace(np.asarray(R_gt, dtype=np.float64).T @ np.asarray(R, dtype=np.float64)) - 1.0) / 2.0
    return float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))


def is_success(R, t, R_gt, t_gt, re_deg, te_m) -> bool:
    te = float(np.linalg.norm(np.asarray(t, dtype=np.float64) - np.asarray(t_gt, dtype=np.float64)))
    return rotation_error_deg(R_gt, R) < re_deg and te < te_m


def hypotheses(ctx: TurboReg, params) -> dict:
    """Hypotheses of the context's most recent register call: valid [m],
    R [m,3,3], t [m,3], cliques [m,3], inliers [m], score [m]."""
    RT = ctx.buffer(BUF_RT)
    C = ctx.buffer(BUF_CLIQUES)
    IN = ctx.buffer(BUF_INLIERS)
    units = ctx.buffer(BUF_SCORES)
    n = ctx.shape()[0]
    valid = (RT[:, 13].view(np.int32) & 1) != 0
    return {"valid": valid, "R": RT[:, :9].reshape(-1, 3, 3).astype(np.float64),
            "t": RT[:, 9:12].astype(np.float64), "cliques": C[:, :3].copy(), "inliers": IN.copy(),
            "score": score_values(units, IN, params, n)}


def rank(score, valid, scoring) -> np.ndarray:
    """Indices of the valid hypotheses, best first; ties go to the lower index."""
    h = np.flatnonzero(valid)
    key = -np.asarray(score)[h] if scoring == SCORE_IN else np.asarray(score)[h]
    return h[np.lexsort((h, key))]


def better_or_equal(a, b, scoring) -> bool:
    """Score a is at least as good as score b."""
    return a >= b if scoring == SCORE_IN else a <= b


def problem_record(hyp: dict, order, gt_score, scoring, R_gt, t_gt, inlier_flags, re_deg, te_m, ks=KS) -> dict:
    """RR / TQRR / ICRR / TKRR@K booleans of one problem (all False if it has no hypothesis)."""
    rec = {"RR": False, "TQRR": False, "ICRR": False}
    rec.update({f"TKRR@{k}": False for k in ks})
    if len(order) == 0:
        return rec
    ok = [is_success(hyp["R"][h], hyp["t"][h], R_gt, t_gt, re_deg, te_m) for h in order[:max(ks + (1,))]]
    top = int(order[0])
    rec["RR"] = bool(ok[0])
    rec["TQRR"] = bool(better_or_equal(hyp["score"][top], gt_score, scoring))
    rec["ICRR"] = bool(np.asarray(inlier_flags)[hyp["cliques"][top]].all())
    for k in ks:
        rec[f"TKRR@{k}"] = bool(any(ok[:k]))
    return rec


def summarize(records, ks=KS) -> dict:
    """Percentages over problems."""
    keys = ["RR", "TQRR", "ICRR"] + [f"TKRR@{k}" for k in ks]
    m = max(len(records), 1)
    return {k: 100.0 * sum(r[k] for r in records) / m for k in keys}


def evaluate(ctx: TurboReg, x, y, params, R_gt, t_gt, inlier_flags, re_deg, te_m, ks=KS) -> dict:
    """Register one problem and compute its ranking record."""
    res = ctx.register(x, y, params)
    if res.status != 0:
        return problem_record({}, [], 0.0, params.scoring, R_gt, t_gt, inlier_flags, re_deg, te_m, ks)
    hyp = hypotheses(ctx, params)
    order = rank(hyp["score"], hyp["valid"], params.scoring)
    if int(order[0]) != res.hypothesis:
        raise RuntimeError("ranking disagrees with the library's selection")
    gt = np.concatenate([np.asarray(R_gt, dtype=np.float32).ravel(), np.asarray(t_gt, dtype=np.float32)])
    _, gt_score = ctx.score_transforms(x, y, params, gt[None, :])
    return problem_record(hyp, order, float(gt_score[0]), params.scoring, R_gt, t_gt, inlier_flags,
                          re_deg, te_m, ks)
