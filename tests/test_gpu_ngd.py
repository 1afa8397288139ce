"""The natural-gradient update (Sec. 3.1(d); options.update = 1) on the GPU
against the oracle, whose NGD step is pinned on the CPU by a finite-
difference Fisher natural gradient and by its fixed points.  Thread and block
forms, every precision, a binding KL bound, the arm and Alg. 2."""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import workloads as W
from _parity import TOL_FP64_SMALL, TOL_MIXED, compare_plan, gpu_solve, rel_mu

pytestmark = pytest.mark.gpu

MIXED, FP64, MIXED_DF = 1, 0, 2
NGD = 1


@pytest.fixture(scope="module")
def pg():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA device"
    import paper_2411_03416_b300 as pg
    pg.lib()
    return pg


@pytest.mark.parametrize("tpb", [0, 64])
@pytest.mark.parametrize("prec,tol", [(FP64, TOL_FP64_SMALL), (MIXED, TOL_MIXED), (MIXED_DF, TOL_MIXED)])
def test_ngd_c1_point2d(pg, prec, tol, tpb):
    pb, op = W.c1_point2d()
    op = replace(op, update=NGD)
    res = gpu_solve([pb], [replace(op, plan_threads=tpb)], prec)[0]
    info, ora = compare_plan(pb, op, res, rtol_mu=tol["mu"], rtol_sigma=tol["sigma"],
                             max_replays=0 if prec == FP64 else None, prec=prec)
    assert len(res.logs) == op.iters
    # a different method from Thm 1's: the KL-proximal plan ends elsewhere
    prox = gpu_solve([pb], [replace(op, update=0, plan_threads=tpb)], prec)[0]
    assert rel_mu(prox.mu, res.mu) > 1e-6


@pytest.mark.parametrize("tpb", [0, 64])
def test_ngd_binding_kl_bound_fp64(pg, tpb):
    pb, op = W.c1_point2d(N=30, iters=8)
    op = replace(op, update=NGD, kl_eps=0.5)
    res = gpu_solve([pb], [replace(op, plan_threads=tpb)], FP64)[0]
    assert any(l["trials"] > 1 for l in res.logs)
    compare_plan(pb, op, res, rtol_mu=1e-9, rtol_sigma=1e-9, max_replays=0)


def test_ngd_no_obstacles_precision_recursion(pg):
    """psi = 0, unbounded KL: Lambda_k = K^-1 + (1-beta)^k (Lambda_0 - K^-1)."""
    pb, op = W.c1_point2d(N=20)
    pb = replace(pb, cost_kind=W.COST_NONE)
    beta, s, k = 0.4, 2.0, 6
    op = replace(op, update=NGD, kl_eps=float("inf"), beta_max=beta, iters=k, init_kind=1, init_scale=s)
    res = gpu_solve([pb], [op], FP64)[0]
    pr = oracle.prior(pb)
    want = pr.Kd + (1 - beta) ** k * (np.stack([s * np.eye(4)] * 21) - pr.Kd)
    assert np.linalg.norm(res.Ld - want) <= 1e-12 * np.linalg.norm(want)
    assert all(l["beta"] == beta and l["trials"] == 1 for l in res.logs)


@pytest.mark.parametrize("prec,tol", [(FP64, TOL_FP64_SMALL), (MIXED, TOL_MIXED)])
def test_ngd_arm_short(pg, prec, tol):
    pb, op = W.c3_arm(N=30, iters=8)
    op = replace(op, update=NGD)
    res = gpu_solve([pb], [op], prec)[0]
    compare_plan(pb, op, res, rtol_mu=tol["mu"], rtol_sigma=tol["sigma"], prec=prec)


@pytest.mark.parametrize("tpb", [0, 64])
def test_ngd_quadrotor_slr_fp64(pg, tpb):
    """Alg. 2 with the natural-gradient inner update."""
    pb, op = W.c4_quadrotor(N=40, iters=5, slr_iters=3)
    op = replace(op, update=NGD)
    res = gpu_solve([pb], [replace(op, plan_threads=tpb)], FP64)[0]
    compare_plan(pb, op, res, rtol_mu=3e-8, rtol_sigma=1e-6)
