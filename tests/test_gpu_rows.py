"""Per-row parity of the CUDA path with the oracle, through the C ABI's
single-phase entry points (pgvimp_batch_phase) on the same seeded inputs.

Rows: prior build, marginals, factor quadrature + gradients, one Thm 1 trial,
SLR linearisation.  The GPU reads only its own inputs; expected values come
from the oracle alone."""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import workloads as W
from _parity import rel_sigma

pytestmark = pytest.mark.gpu

MIXED, FP64 = 1, 0


@pytest.fixture(scope="module")
def pg():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA device"
    import paper_2411_03416_b300 as pg
    from paper_2411_03416_b300 import _lib
    pg.lib()
    return _lib


def _batch(L, pbs, ops, precision):
    b = L.Batch(pbs, ops, precision)
    b.upload()
    b.reset()
    return b


def _sync():
    import torch
    torch.cuda.synchronize()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


# ------------------------------------------------------------------- a0 prior

@pytest.mark.parametrize("N", [1, 12, 50, 750])
def test_prior_matches_oracle(pg, N):
    pb, op = W.c1_point2d(N=N)
    b = _batch(pg, [pb], [op], FP64)
    b.phase(pg.PHASE_PRIOR)
    _sync()
    n = pb.n
    pr = oracle.prior(pb)
    Kd = b.read(0, pg.BUF_KD, (N + 1, n, n))
    Ko = b.read(0, pg.BUF_KO, (N, n, n))
    bb = b.read(0, pg.BUF_B, (N + 1, n))
    assert rel(Kd, pr.Kd) < 1e-12 and rel(Ko, pr.Ko) < 1e-12
    assert rel(bb, pr.b) < 1e-11
    # the initial iterate: the straight line and Lambda_0 = K^-1
    np.testing.assert_allclose(b.read(0, pg.BUF_MU, (N + 1, n)), oracle.init_mean(pb), rtol=0, atol=1e-13)
    assert rel(b.read(0, pg.BUF_LD, (N + 1, n, n)), pr.Kd) < 1e-12
    b.close()


def test_prior_ltv_and_temperature(pg):
    rng = np.random.default_rng(4)
    pb, op = W.c1_point2d(N=9)
    A = np.stack([pb.A + 0.2 * rng.standard_normal((4, 4)) for _ in range(9)])
    a = 0.3 * rng.standard_normal((9, 4))
    pb = replace(pb, A=A, a=a, temperature=2.5)
    b = _batch(pg, [pb], [op], FP64)
    b.phase(pg.PHASE_PRIOR)
    _sync()
    pr = oracle.prior(pb)
    assert rel(b.read(0, pg.BUF_KD, (10, 4, 4)), pr.Kd) < 1e-12
    assert rel(b.read(0, pg.BUF_KO, (9, 4, 4)), pr.Ko) < 1e-12
    assert rel(b.read(0, pg.BUF_B, (10, 4)), pr.b) < 1e-11
    b.close()


# -------------------------------------------------------------- a1 marginals

def _rand_bt(rng, n, N, scale=1.0):
    D = n * (N + 1)
    Bm = np.zeros((D, D))
    for i in range(N + 1):
        Bm[i * n:(i + 1) * n, i * n:(i + 1) * n] = rng.standard_normal((n, n)) + 2 * np.eye(n)
        if i < N:
            Bm[i * n:(i + 1) * n, (i + 1) * n:(i + 2) * n] = rng.standard_normal((n, n))
    M = scale * (Bm.T @ Bm + np.eye(D))
    Ld = np.stack([M[i * n:(i + 1) * n, i * n:(i + 1) * n] for i in range(N + 1)])
    Lo = np.stack([M[(i + 1) * n:(i + 2) * n, i * n:(i + 1) * n] for i in range(N)])
    return Ld, Lo


@pytest.mark.parametrize("make,N", [(W.c1_point2d, 1), (W.c1_point2d, 37), (W.c3_arm, 11), (W.c4_quadrotor, 23)])
def test_marginals_match_oracle(pg, make, N):
    pb, op = make(N=N)
    rng = np.random.default_rng(N)
    b = _batch(pg, [pb], [op], FP64)
    b.phase(pg.PHASE_PRIOR)
    Ld, Lo = _rand_bt(rng, pb.n, N, scale=3.0)
    b.write(0, pg.BUF_LD, Ld)
    b.write(0, pg.BUF_LO, Lo)
    b.phase(pg.PHASE_MARGINALS)
    _sync()
    Sd, So, ld = oracle.marginals(Ld, Lo)
    gS = b.read(0, pg.BUF_SD, Sd.shape)
    gO = b.read(0, pg.BUF_SO, So.shape)
    sc = b.read(0, pg.BUF_SCAL, (24,))
    assert rel_sigma(gS, Sd) < 1e-10
    assert rel(gO, So) < 1e-10
    assert abs(sc[pg.S_LOGDET] - ld) < 1e-9 * max(1.0, abs(ld))
    assert sc[pg.S_STATUS] == 0
    b.close()


def test_marginals_dense_horizon_prior(pg):
    """N=750 prior precision: the marginals agree to the FP64 conditioning
    floor of this chain (~1e-7 between any two FP64 algorithms)."""
    pb, op = W.c2_point2d_dense()
    b = _batch(pg, [pb], [op], FP64)
    b.phase(pg.PHASE_PRIOR)
    _sync()
    pr = oracle.prior(pb)
    Sd, So, ld = oracle.marginals(pr.Kd, pr.Ko)
    gS = b.read(0, pg.BUF_SD, Sd.shape)
    sc = b.read(0, pg.BUF_SCAL, (24,))
    assert rel_sigma(gS, Sd) < 2e-6
    assert abs(sc[pg.S_LOGDET] - ld) < 1e-6
    b.close()


def test_marginals_not_pd_sets_status(pg):
    pb, op = W.c1_point2d(N=6)
    b = _batch(pg, [pb], [op], FP64)
    b.phase(pg.PHASE_PRIOR)
    Ld, Lo = _rand_bt(np.random.default_rng(0), 4, 6)
    Ld[3] -= 1e4 * np.eye(4)
    b.write(0, pg.BUF_LD, Ld)
    b.write(0, pg.BUF_LO, Lo)
    b.phase(pg.PHASE_MARGINALS)
    _sync()
    assert b.read(0, pg.BUF_SCAL, (24,))[pg.S_STATUS] == 2
    b.close()


# --------------------------------------------------------- a2-a4 quadrature

def _oracle_grads(pb, op, mu, Sd, per_factor=False):
    n = pb.n
    g, G, coll = np.zeros_like(mu), np.zeros_like(Sd), 0.0
    s0 = np.zeros(pb.N + 1)
    for i in range(pb.N + 1):
        S0, S1, S2 = oracle.quad_moments(pb, op, i, mu[i], Sd[i])
        g[i], G[i] = oracle.gradients(Sd[i], S0, S1, S2)
        coll += S0
        s0[i] = S0
    return (g, G, coll, s0) if per_factor else (g, G, coll)


CASES = [
    ("point2d_gh3", lambda: W.c1_point2d(N=40)),
    ("point2d_gh5", lambda: W.c2_point2d_dense(N=60)),
    ("arm_deg3", lambda: W.c3_arm(N=12)),
    ("quadrotor_gh3", lambda: W.c4_quadrotor(N=15)),
]


def _perturbed_state(pb, seed):
    """A mean/covariance with the hinge active: the straight line shifted a
    little and the prior marginals."""
    rng = np.random.default_rng(seed)
    mu = oracle.init_mean(pb) + 0.05 * rng.standard_normal((pb.N + 1, pb.n))
    pr = oracle.prior(pb)
    Sd, So, _ = oracle.marginals(pr.Kd + 0.0, pr.Ko)
    return mu, Sd, So


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_quadrature_and_gradients(pg, name, make, prec):
    pb, op = make()
    if pb.dyn_kind != 0:
        # the SLR model: use a fixed LTV-free problem for this row
        pb = replace(pb, dyn_kind=0, A=np.zeros((6, 6)))
    mu, Sd, So = _perturbed_state(pb, 1)
    b = _batch(pg, [pb], [op], prec)
    b.phase(pg.PHASE_PRIOR)
    b.write(0, pg.BUF_MU, mu)
    b.write(0, pg.BUF_SD, Sd)
    b.phase(pg.PHASE_QUAD)
    _sync()
    g_o, G_o, coll_o, s0_o = _oracle_grads(pb, op, mu, Sd, per_factor=True)
    g = b.read(0, pg.BUF_G1, g_o.shape)
    G = b.read(0, pg.BUF_G2, G_o.shape)
    coll = b.read(0, pg.BUF_SCAL, (24,))[pg.S_COLL]
    assert coll_o > 0, "the case must exercise the hinge"
    tol = 1e-9 if prec == FP64 else 3e-4
    assert abs(coll - coll_o) <= tol * abs(coll_o) + 1e-12
    assert rel(g, g_o) <= tol, (rel(g, g_o), name)
    assert rel(G, G_o) <= tol, (rel(G, G_o), name)
    # factor by factor, wherever the hinge is active: a wrong factor near the
    # start or goal, where psi is small, cannot hide in the whole-array norm
    active = np.nonzero(s0_o > 1e-6 * s0_o.max())[0]
    assert len(active) >= 2
    ftol = 1e-8 if prec == FP64 else 2e-3
    worst = []
    for i in active:
        eg = np.linalg.norm(g[i] - g_o[i]) / np.linalg.norm(g_o[i])
        eG = np.linalg.norm(G[i] - G_o[i]) / np.linalg.norm(G_o[i])
        worst.append((max(eg, eG), i))
        assert eg <= ftol and eG <= ftol, (name, i, s0_o[i], eg, eG)
    # in FP64, factors with no active sigma point are exactly zero on both sides
    if prec == FP64:
        inactive = np.nonzero(s0_o == 0.0)[0]
        assert np.all(g[inactive] == 0.0) and np.all(G[inactive] == 0.0), name
    b.close()


# ------------------------------------------------------------- a5 one trial

@pytest.mark.parametrize("beta", [0.5, 0.125, 1e-3])
@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_trial_matches_oracle(pg, beta, prec):
    pb, op = W.c1_point2d(N=30)
    b = _batch(pg, [pb], [op], prec)
    b.phase(pg.PHASE_PRIOR)
    b.phase(pg.PHASE_QUAD)
    b.phase(pg.PHASE_TRIAL, beta)
    _sync()
    pr = oracle.prior(pb)
    mu0 = oracle.init_mean(pb)
    Sd, So, ld = oracle.marginals(pr.Kd, pr.Ko)
    g, G, _ = _oracle_grads(pb, op, mu0, Sd)
    rc, t = oracle.trial(pb, beta, pr, mu0, pr.Kd, pr.Ko, ld, g, G)
    assert rc == 0
    sc = b.read(0, pg.BUF_SCAL, (24,))
    mu_t = b.read(0, pg.BUF_TMU, mu0.shape)
    Sd_t = b.read(0, pg.BUF_TSD, Sd.shape)
    So_t = b.read(0, pg.BUF_TSO, So.shape)
    tol = 1e-9 if prec == FP64 else 1e-4
    assert sc[pg.S_T_PD] == 1
    assert rel(mu_t, t["mu"]) < tol
    assert rel_sigma(Sd_t, t["Sd"]) < max(tol, 1e-9) * 10
    assert rel(So_t, t["So"]) < max(tol, 1e-9) * 10
    assert abs(sc[pg.S_T_LOGDET] - t["logdet"]) < 1e-8 * abs(t["logdet"])
    assert abs(sc[pg.S_T_KL] - t["kl"]) <= (1e-6 if prec == FP64 else 1e-3) * max(1.0, abs(t["kl"]))
    b.close()


# ------------------------------------------------------------------ a6 SLR

@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_slr_matches_oracle(pg, prec):
    pb, op = W.c4_quadrotor(N=20)
    b = _batch(pg, [pb], [op], prec)
    b.phase(pg.PHASE_PRIOR)          # SLR about the straight line with K0, then the prior
    _sync()
    xbar = oracle.init_mean(pb)
    Sbar = np.stack([pb.K0] * (pb.N + 1))
    A_o, a_o = oracle.slr(pb, op, xbar, Sbar)
    A = b.read(0, pg.BUF_ALTV, A_o.shape)
    a = b.read(0, pg.BUF_ALTVA, a_o.shape)
    tol = 1e-10 if prec == FP64 else 2e-5
    assert rel(A, A_o) < tol and rel(a, a_o) < tol
    # the prior of the linearised system
    pr = oracle.prior(pb, A_ltv=A_o, a_ltv=a_o)
    assert rel(b.read(0, pg.BUF_KD, pr.Kd.shape), pr.Kd) < (1e-11 if prec == FP64 else 1e-4)
    # around a non-trivial nominal (the current iterate)
    rng = np.random.default_rng(2)
    mu = xbar + 0.3 * rng.standard_normal(xbar.shape)
    Sd = np.stack([np.diag(rng.uniform(0.01, 0.2, 6)) for _ in range(pb.N + 1)])
    b.write(0, pg.BUF_MU, mu)
    b.write(0, pg.BUF_SD, Sd)
    b.phase(pg.PHASE_SLR)
    _sync()
    A_o, a_o = oracle.slr(pb, op, mu, Sd)
    assert rel(b.read(0, pg.BUF_ALTV, A_o.shape), A_o) < tol * 10
    assert rel(b.read(0, pg.BUF_ALTVA, a_o.shape), a_o) < tol * 10
    b.close()
