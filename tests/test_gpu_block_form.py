"""The block (latency) form: one thread block per plan, block recursions by
cyclic reduction over time.  The same plans as the thread form, against the
oracle, at the sizes and edge cases where the reduction's level structure
changes (N a power of two, one more or one less, N = 1)."""
from dataclasses import replace

import numpy as np
import pytest

import workloads as W
from _parity import TOL_FP64_SMALL, TOL_MIXED, compare_plan, fp64_tol_from_conditioning, gpu_solve

pytestmark = pytest.mark.gpu

MIXED, FP64, MIXED_DF = 1, 0, 2


@pytest.fixture(scope="module")
def pg():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA device"
    import paper_2411_03416_b300 as pg
    pg.lib()
    return pg


def block(op, tpb=64):
    return replace(op, plan_threads=tpb)


@pytest.mark.parametrize("prec,tol", [(FP64, TOL_FP64_SMALL), (MIXED, TOL_MIXED), (MIXED_DF, TOL_MIXED)])
def test_c1_point2d_block_form(pg, prec, tol):
    pb, op = W.c1_point2d()
    res = gpu_solve([pb], [block(op)], prec)[0]
    compare_plan(pb, op, res, rtol_mu=tol["mu"], rtol_sigma=tol["sigma"], prec=prec)
    assert len(res.logs) == op.iters


@pytest.mark.parametrize("N", [1, 2, 3, 7, 8, 9, 31, 32, 33, 64, 100])
@pytest.mark.parametrize("tpb", [32, 128])
def test_reduction_levels_fp64(pg, N, tpb):
    """Every level structure of the cyclic reduction, including states with
    only a left neighbour, more threads than states and the reverse."""
    pb, op = W.c1_point2d(N=N, iters=4)
    op = replace(op, kl_eps=0.05 * (N + 1))       # binds: the bisection runs several trials
    res = gpu_solve([pb], [block(op, tpb)], FP64)[0]
    tol = fp64_tol_from_conditioning(pb)
    compare_plan(pb, op, res, rtol_mu=tol, rtol_sigma=tol)


@pytest.mark.parametrize("prec,tol", [(FP64, TOL_FP64_SMALL), (MIXED, TOL_MIXED), (MIXED_DF, TOL_MIXED)])
def test_c3_arm_block_form(pg, prec, tol):
    pb, op = W.c3_arm(N=30, iters=10)
    res = gpu_solve([pb], [block(op, 32)], prec)[0]
    compare_plan(pb, op, res, rtol_mu=tol["mu"], rtol_sigma=tol["sigma"], prec=prec)


def test_c4_quadrotor_slr_block_form_fp64(pg):
    """Alg. 2 with the SLR linearisation and the LTV prior spread over the block."""
    pb, op = W.c4_quadrotor(N=40, iters=5, slr_iters=3)
    res = gpu_solve([pb], [block(op)], FP64)[0]
    compare_plan(pb, op, res, rtol_mu=3e-8, rtol_sigma=1e-6)
    assert len(res.logs) == 15


@pytest.mark.parametrize("N", [40, 300])
def test_c4_quadrotor_first_linearisation_block_form_mixed(pg, N):
    pb, op = W.c4_quadrotor(N=N, iters=2, slr_iters=1)
    res = gpu_solve([pb], [block(op, 128)], MIXED)[0]
    compare_plan(pb, op, res, rtol_mu=TOL_MIXED["mu"], rtol_sigma=TOL_MIXED["sigma"])


@pytest.mark.parametrize("iters", [1, 2])
@pytest.mark.parametrize("prec,tol", [(FP64, dict(mu=1e-5, sigma=1e-5)), (MIXED, TOL_MIXED)])
def test_c2_dense_horizon_block_form_first_iterations(pg, prec, tol, iters):
    pb, op = W.c2_point2d_dense(iters=iters)
    res = gpu_solve([pb], [block(op, 128)], prec)[0]
    compare_plan(pb, op, res, rtol_mu=tol["mu"], rtol_sigma=tol["sigma"], prec=prec)


def test_block_form_matches_thread_form(pg):
    """Two elimination orders of the same SPD chains: FP64 results agree to
    rounding on a non-chaotic plan, with the same step sizes."""
    pb, op = W.c1_point2d(N=60, iters=12)
    a = gpu_solve([pb], [op], FP64)[0]
    b = gpu_solve([pb], [block(op, 64)], FP64)[0]
    assert [l["beta"] for l in a.logs] == [l["beta"] for l in b.logs]
    assert np.linalg.norm(a.mu - b.mu) <= 1e-10 * np.linalg.norm(a.mu)
    assert np.max(np.abs(a.Sd - b.Sd)) <= 1e-10 * np.max(np.abs(a.Sd))


@pytest.mark.parametrize("prec", [MIXED, FP64])
def test_block_form_batch_equals_alone(pg, prec):
    probs = [W.c1_point2d(request=r, N=N, iters=6) for r, N in enumerate([7, 50, 33, 1, 64])]
    pbs, ops = [p for p, _ in probs], [block(o) for _, o in probs]
    together = gpu_solve(pbs, ops, prec)
    for i in range(len(pbs)):
        alone = gpu_solve([pbs[i]], [ops[i]], prec)[0]
        np.testing.assert_array_equal(together[i].mu, alone.mu)
        np.testing.assert_array_equal(together[i].Sd, alone.Sd)


def test_c3_arm_full_size_block_form(pg):
    """The arm at its full size (N = 200, 25 iterations) in the block form the server uses for it."""
    pb, op = W.c3_arm()
    res = gpu_solve([pb], [block(op, 256)], MIXED)[0]
    compare_plan(pb, op, res, rtol_mu=TOL_MIXED["mu"], rtol_sigma=TOL_MIXED["sigma"])


def test_c2_full_plan_invariants_block_form(pg):
    """The whole 30-iteration N = 750 plan (chaotic in FP64, so checked by
    invariants, as for the thread form)."""
    pb, op = W.c2_point2d_dense()
    res = gpu_solve([pb], [block(op, 256)], MIXED)[0]
    assert len(res.logs) == op.iters
    assert np.all(np.isfinite(res.mu)) and np.all(np.isfinite(res.Sd))
    for S in res.Sd:
        np.linalg.cholesky(0.5 * (S + S.T))
    for l in res.logs:
        if l["beta"] > 0:
            assert l["kl"] <= op.kl_eps * (1 + 1e-12)
            k = l["beta"] / op.beta_max * 2 ** op.max_bisect
            assert abs(k - round(k)) < 1e-9
    assert res.logs[-1]["collision_cost"] < res.logs[0]["collision_cost"]


@pytest.mark.parametrize("N", [1, 2, 7, 8, 9, 33, 100])
@pytest.mark.parametrize("tpb", [32, 128])
def test_reduction_levels_double_float(pg, N, tpb):
    """The block form with double-float recursions over the level structures
    of the cyclic reduction (a binding KL bound runs several trials)."""
    pb, op = W.c1_point2d(N=N, iters=4)
    op = replace(op, kl_eps=0.05 * (N + 1))
    res = gpu_solve([pb], [block(op, tpb)], MIXED_DF)[0]
    compare_plan(pb, op, res, rtol_mu=TOL_MIXED["mu"], rtol_sigma=TOL_MIXED["sigma"], prec=MIXED_DF)


@pytest.mark.parametrize("n_make", ["point3d", "quadrotor"])
def test_double_float_block_form_other_dimensions(pg, n_make):
    """n = 6: the 3-D point robot and the first linearisation of Alg. 2."""
    if n_make == "point3d":
        pb, op = W.point3d(request=1, N=80)
    else:
        pb, op = W.c4_quadrotor(N=60, iters=3, slr_iters=1)
    res = gpu_solve([pb], [block(op, 64)], MIXED_DF)[0]
    compare_plan(pb, op, res, rtol_mu=TOL_MIXED["mu"], rtol_sigma=TOL_MIXED["sigma"], prec=MIXED_DF)


def test_double_float_block_form_equals_alone_in_a_batch(pg):
    probs = [W.c1_point2d(request=r, N=N, iters=6) for r, N in enumerate([7, 50, 33, 1])]
    pbs, ops = [p for p, _ in probs], [block(o, 64) for _, o in probs]
    together = gpu_solve(pbs, ops, MIXED_DF)
    for i in range(len(probs)):
        alone = gpu_solve([pbs[i]], [ops[i]], MIXED_DF)[0]
        np.testing.assert_array_equal(together[i].mu, alone.mu)
        np.testing.assert_array_equal(together[i].Sd, alone.Sd)


# ---- the warp-cooperative reduction (n >= 6: one warp per elimination)

@pytest.mark.parametrize("N", [1, 2, 3, 8, 9, 31, 32, 33, 100])
@pytest.mark.parametrize("tpb", [32, 256])
def test_warp_reduction_levels_point3d_fp64(pg, N, tpb):
    """n = 6 over every level structure of the reduction, with a binding KL
    bound (several trials an iteration), one warp and eight."""
    pb, op = W.point3d(request=2, N=N)
    op = replace(op, iters=4, kl_eps=0.05 * (N + 1))
    res = gpu_solve([pb], [block(op, tpb)], FP64)[0]
    tol = fp64_tol_from_conditioning(pb)
    compare_plan(pb, op, res, rtol_mu=tol, rtol_sigma=tol, max_replays=0)


@pytest.mark.parametrize("N", [1, 2, 7, 8, 9, 33])
@pytest.mark.parametrize("prec", [FP64, MIXED_DF])
def test_warp_reduction_levels_arm(pg, N, prec):
    """n = 14 (a 7-DOF arm) over level structures of the reduction."""
    pb, op = W.c3_arm(N=N, iters=4)
    res = gpu_solve([pb], [block(op, 128)], prec)[0]
    if prec == FP64:
        tol = max(TOL_FP64_SMALL["mu"], fp64_tol_from_conditioning(pb))
        compare_plan(pb, op, res, rtol_mu=tol, rtol_sigma=tol, max_replays=0)
    else:
        compare_plan(pb, op, res, rtol_mu=TOL_MIXED["mu"], rtol_sigma=TOL_MIXED["sigma"], prec=prec)


def test_c3_arm_full_size_block_form_double_float(pg):
    """The full-size arm plan (N = 200, 25 iterations) with double-float
    recursions, the form a single arm plan is served in for latency."""
    pb, op = W.c3_arm()
    res = gpu_solve([pb], [block(op, 256)], MIXED_DF)[0]
    compare_plan(pb, op, res, rtol_mu=TOL_MIXED["mu"], rtol_sigma=TOL_MIXED["sigma"], prec=MIXED_DF)


def test_warp_reduction_batch_equals_alone(pg):
    """Plans of different horizons in one launch give the results they give alone."""
    probs = [W.point3d(request=r, N=N) for r, N in enumerate([9, 40, 1, 33])]
    pbs = [p for p, _ in probs]
    ops = [block(replace(o, iters=5), 64) for _, o in probs]
    for prec in (FP64, MIXED_DF):
        together = gpu_solve(pbs, ops, prec)
        for i in range(len(pbs)):
            alone = gpu_solve([pbs[i]], [ops[i]], prec)[0]
            np.testing.assert_array_equal(together[i].mu, alone.mu)
            np.testing.assert_array_equal(together[i].Sd, alone.Sd)
