"""Host logic of the ranking study (Table 6): ordering, the four recall
definitions and the percentages, on hand-made hypothesis tables."""
import numpy as np

from paper_2507_01439_gb300 import SCORE_IN, SCORE_MAE, SCORE_MSE
from paper_2507_01439_gb300 import ranking


def _rz(deg):
    a = np.radians(deg)
    return np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1.0]])


def test_rank_orders_by_score_then_index():
    valid = np.array([True, True, True, False, True])
    assert ranking.rank(np.array([5, 7, 7, 9, 7.0]), valid, SCORE_IN).tolist() == [1, 2, 4, 0]
    assert ranking.rank(np.array([0.2, 0.1, 0.1, 0.05, 0.3]), valid, SCORE_MSE).tolist() == [1, 2, 0, 4]
    assert ranking.rank(np.array([0.2, 0.1, 0.1, 0.05, 0.3]), valid, SCORE_MAE).tolist() == [1, 2, 0, 4]
    assert ranking.rank(np.zeros(3), np.zeros(3, bool), SCORE_IN).tolist() == []


def test_rotation_error_and_success():
    assert abs(ranking.rotation_error_deg(np.eye(3), _rz(30)) - 30.0) < 1e-9
    assert abs(ranking.rotation_error_deg(_rz(10), _rz(-20)) - 30.0) < 1e-9
    assert ranking.is_success(_rz(14), [0, 0, 0.29], np.eye(3), np.zeros(3), 15, 0.3)
    assert not ranking.is_success(_rz(15.5), [0, 0, 0], np.eye(3), np.zeros(3), 15, 0.3)
    assert not ranking.is_success(np.eye(3), [0.3, 0, 0], np.eye(3), np.zeros(3), 15, 0.3)


def _table():
    # four hypotheses: h0 wrong rotation, h1 right, h2 right but outlier clique, h3 invalid
    R = np.stack([_rz(40), _rz(1), _rz(2), np.eye(3)])
    t = np.zeros((4, 3))
    cliques = np.array([[0, 1, 2], [0, 1, 3], [0, 4, 5], [0, 0, 0]])
    return {"valid": np.array([True, True, True, False]), "R": R, "t": t, "cliques": cliques}


def test_problem_record_inlier_number():
    hyp = _table()
    hyp["score"] = np.array([30.0, 25.0, 25.0, 99.0])
    inl = np.array([1, 1, 1, 1, 0, 0], bool)
    order = ranking.rank(hyp["score"], hyp["valid"], SCORE_IN)
    assert order.tolist() == [0, 1, 2]
    rec = ranking.problem_record(hyp, order, 28.0, SCORE_IN, np.eye(3), np.zeros(3), inl, 15, 0.3, ks=(1, 2, 3))
    # top-1 is the wrong rotation with a higher IN than the ground truth
    assert rec == {"RR": False, "TQRR": True, "ICRR": True, "TKRR@1": False, "TKRR@2": True, "TKRR@3": True}
    rec = ranking.problem_record(hyp, order, 30.0, SCORE_IN, np.eye(3), np.zeros(3), inl, 15, 0.3, ks=(1,))
    assert rec["TQRR"]                       # equal counts as reaching the ground truth
    rec = ranking.problem_record(hyp, order, 31.0, SCORE_IN, np.eye(3), np.zeros(3), inl, 15, 0.3, ks=(1,))
    assert not rec["TQRR"]


def test_problem_record_capped_error():
    hyp = _table()
    hyp["score"] = np.array([0.004, 0.002, 0.001, 0.0])
    inl = np.array([1, 1, 1, 1, 0, 0], bool)
    order = ranking.rank(hyp["score"], hyp["valid"], SCORE_MSE)
    assert order.tolist() == [2, 1, 0]
    rec = ranking.problem_record(hyp, order, 0.0015, SCORE_MSE, np.eye(3), np.zeros(3), inl, 15, 0.3, ks=(1, 3))
    # top-1 (h2) registers correctly but its clique holds two outliers
    assert rec == {"RR": True, "TQRR": True, "ICRR": False, "TKRR@1": True, "TKRR@3": True}
    rec = ranking.problem_record(hyp, order, 0.0009, SCORE_MSE, np.eye(3), np.zeros(3), inl, 15, 0.3, ks=(1,))
    assert not rec["TQRR"]


def test_no_hypothesis_record_and_summary():
    rec = ranking.problem_record({}, [], 0.0, SCORE_IN, np.eye(3), np.zeros(3), np.ones(3, bool), 15, 0.3)
    assert not any(rec.values())
    recs = [{"RR": True, "TQRR": True, "ICRR": False, "TKRR@2": True},
            {"RR": False, "TQRR": True, "ICRR": False, "TKRR@2": True},
            {"RR": False, "TQRR": False, "ICRR": True, "TKRR@2": False},
            {"RR": True, "TQRR": True, "ICRR": True, "TKRR@2": True}]
    s = ranking.summarize(recs, ks=(2,))
    assert s == {"RR": 50.0, "TQRR": 75.0, "ICRR": 50.0, "TKRR@2": 75.0}
