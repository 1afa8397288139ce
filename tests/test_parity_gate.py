"""The tie gate of the step-size replay (host logic of the parity tests),
checked on the CPU with the oracle standing in for both sides: a decision
that differs at a genuine KL tie is accepted, one that differs anywhere else
fails, and the decisions implied by an accepted step are the ones the search
took."""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import workloads as W
from _parity import TIE_FP64, check_tie_replays, implied_decisions


@pytest.fixture(scope="module")
def run(ora):
    pb, op = W.c1_point2d(N=20, iters=5)
    op = replace(op, kl_eps=0.5)
    return pb, op, ora.plan(pb, op)


def test_implied_decisions_match_the_search(run):
    pb, op, st = run
    for k, l in enumerate(st.logs):
        tr = [(t["beta"], t["feasible"]) for t in st.trials if t["iter"] == k]
        assert implied_decisions(l["beta"], op.beta_max, op.max_bisect) == tr
    assert implied_decisions(0.0, 0.5, 3) == [(0.5, False), (0.25, False), (0.125, False), (0.0625, False)]


def test_a_decision_away_from_a_tie_fails(run):
    pb, op, st = run
    gb = np.array([l["beta"] for l in st.logs])
    bad = gb.copy()
    bad[2] = gb[2] + op.beta_max / 2 ** op.max_bisect      # one bisection leaf off
    ora = oracle.plan(pb, replace(op, replay_beta=bad))
    logs = [dict(l) for l in st.logs]
    with pytest.raises(AssertionError, match="no tie"):
        check_tie_replays(ora, bad, logs, op, TIE_FP64)


def test_a_decision_at_a_tie_is_accepted(ora):
    """Set eps to exactly the KL of the first trial (beta_max): the oracle then
    accepts beta_max, and a side that rejected it (rounding on the other side
    of eps) took a legitimate branch."""
    pb, op = W.c1_point2d(N=20, iters=3)
    op = replace(op, kl_eps=0.5)
    st = ora.plan(pb, op)
    kl0 = [t for t in st.trials if t["iter"] == 0][0]["kl"]
    op_t = replace(op, kl_eps=kl0)
    st_t = ora.plan(pb, op_t)
    assert st_t.logs[0]["beta"] == op.beta_max
    other = np.array([l["beta"] for l in st_t.logs])
    other[0] = op.beta_max * (1 - 2.0 ** -op.max_bisect)     # rejected beta_max, accepted every halving
    ora_r = oracle.plan(pb, replace(op_t, replay_beta=other))
    logs = [dict(kl=l["kl"]) for l in ora_r.logs]
    recs = check_tie_replays(ora_r, other, logs, op_t, TIE_FP64)
    assert recs and recs[0]["iter"] == 0 and recs[0]["trial"] == 0 and recs[0]["kl_gap"] < 1e-12
