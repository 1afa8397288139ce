"""Helpers shared by the GPU parity tests: run the CUDA path and the oracle on
the same seeded problem and compare them.  The oracle never receives a value
computed by the CUDA path except a replayed step-size sequence (the bisection
decisions), which is the documented tie-breaking reading for near-equal KL."""
from dataclasses import replace

import numpy as np

import oracle

# Tolerances.  Mixed precision (FP32 quadrature): the mean to 1e-4 and the
# marginal covariances to 1e-3, relative.  All-FP64: 1e-9 where the problem's
# conditioning allows it; at N ~ 750 two FP64 implementations of the
# marginals already differ by ~1e-7 (the chain precision is ill-conditioned),
# so the FP64 bound there is derived from that measured floor.
TOL_MIXED = dict(mu=1e-4, sigma=1e-3)
TOL_FP64_SMALL = dict(mu=1e-9, sigma=1e-9)
TOL_FP64_DENSE = dict(mu=2e-6, sigma=2e-6)


def fp64_tol_from_conditioning(pb, floor=1e-9):
    """FP64 bound for two elimination orders of the same chain: 10 kappa u,
    with kappa the 2-norm condition number of the prior precision K^-1 (the
    initial Lambda) and u = 2^-53; never below `floor`.  For the C1 robot
    kappa is 9e5 at N = 50, 1.5e7 at N = 100 and 4.7e10 at N = 750."""
    pr = oracle.prior(pb)
    n, N = pb.n, pb.N
    D = n * (N + 1)
    M = np.zeros((D, D))
    for i in range(N + 1):
        M[i * n:(i + 1) * n, i * n:(i + 1) * n] = pr.Kd[i]
    for i in range(N):
        M[(i + 1) * n:(i + 2) * n, i * n:(i + 1) * n] = pr.Ko[i]
        M[i * n:(i + 1) * n, (i + 1) * n:(i + 2) * n] = pr.Ko[i].T
    return max(floor, 10.0 * np.linalg.cond(M) * 2.0 ** -53)


def rel_mu(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_sigma(a, b):
    num = np.linalg.norm(a - b, axis=(1, 2))
    den = np.linalg.norm(b, axis=(1, 2))
    return float(np.max(num / den))


def gpu_solve(problems, options, precision):
    import paper_2411_03416_b300 as pg
    return pg.solve(problems, options, precision)


def oracle_solve(pb, op):
    return oracle.solve(pb, op)


def compare_plan(pb, op, gres, *, rtol_mu, rtol_sigma, slr=False):
    """Compares one GPU plan with the oracle.  If the accepted step sizes
    differ (a bisection decision taken on the other side of a KL tie), the
    oracle is rerun with the GPU's step sequence."""
    ora = oracle_solve(pb, op)
    gb = np.array([l["beta"] for l in gres.logs])
    ob = np.array([l["beta"] for l in ora.logs])
    replayed = False
    if gb.shape != ob.shape or not np.array_equal(gb, ob):
        ora = oracle_solve(pb, replace(op, replay_beta=gb))
        replayed = True
    em = rel_mu(gres.mu, ora.mu)
    es = rel_sigma(gres.Sd, ora.Sd)
    info = dict(err_mu=em, err_sigma=es, replayed=replayed, n_iters=len(gb),
                max_abs_mu=float(np.max(np.abs(gres.mu - ora.mu))))
    assert em <= rtol_mu, info
    assert es <= rtol_sigma, info
    return info, ora
