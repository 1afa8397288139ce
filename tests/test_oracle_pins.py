"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible mistake in the oracle (a dropped term,
a wrong sign or index, a transposed operand) fails it.  None of them needs a
GPU.
"""
import json
import math
import os
from dataclasses import replace

import numpy as np
import pytest
import scipy.linalg

import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def dense(Ld, Lo):
    N1, n = Ld.shape[0], Ld.shape[1]
    M = np.zeros((N1 * n, N1 * n))
    for i in range(N1):
        M[i * n:(i + 1) * n, i * n:(i + 1) * n] = Ld[i]
    for i in range(N1 - 1):
        M[(i + 1) * n:(i + 2) * n, i * n:(i + 1) * n] = Lo[i]
        M[i * n:(i + 1) * n, (i + 1) * n:(i + 2) * n] = Lo[i].T
    return M


def blocks(S, n):
    N1 = S.shape[0] // n
    Sd = np.stack([S[i * n:(i + 1) * n, i * n:(i + 1) * n] for i in range(N1)])
    So = np.stack([S[(i + 1) * n:(i + 2) * n, i * n:(i + 1) * n] for i in range(N1 - 1)])
    return Sd, So


def rand_bt_spd(rng, n, N, scale=1.0):
    """Random SPD block-tridiagonal matrix: B^T B + I with B block-bidiagonal."""
    D = n * (N + 1)
    Bm = np.zeros((D, D))
    for i in range(N + 1):
        Bm[i * n:(i + 1) * n, i * n:(i + 1) * n] = rng.standard_normal((n, n)) + 2 * np.eye(n)
        if i < N:
            Bm[i * n:(i + 1) * n, (i + 1) * n:(i + 2) * n] = rng.standard_normal((n, n))
    M = scale * (Bm.T @ Bm + np.eye(D))
    return blocks(M, n)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


# ------------------------------------------------------------- quadrature rules

def test_gh_rule_closed_forms(ora):
    g = json.load(open(os.path.join(GOLD, "gauss_hermite.json")))
    for p, r in g["rules"].items():
        x, w = ora.gh_rule(int(p))
        ex = [eval(s, {"sqrt": math.sqrt}) for s in r["nodes"]]
        ew = [eval(s, {"sqrt": math.sqrt}) for s in r["weights"]]
        np.testing.assert_allclose(x, ex, rtol=0, atol=1e-14)
        np.testing.assert_allclose(w, ew, rtol=1e-13, atol=0)


@pytest.mark.parametrize("p", range(1, 13))
def test_gh_rule_matches_library_and_sums_to_one(ora, p):
    x, w = ora.gh_rule(p)
    xl, wl = np.polynomial.hermite_e.hermegauss(p)
    np.testing.assert_allclose(x, xl, atol=1e-12)
    np.testing.assert_allclose(w, wl / math.sqrt(2 * math.pi), rtol=1e-10, atol=1e-15)
    assert abs(w.sum() - 1.0) < 1e-13


def _double_factorial(k):
    return 1 if k <= 0 else k * _double_factorial(k - 2)


@pytest.mark.parametrize("p", range(2, 10))
def test_gh_exact_to_degree_2p_minus_1(ora, p):
    x, w = ora.gh_rule(p)
    for k in range(0, 2 * p):
        exact = 0.0 if k % 2 else float(_double_factorial(k - 1))
        scale = max(1.0, exact, float(np.sum(np.abs(w * x ** k))))
        assert abs(np.sum(w * x ** k) - exact) <= 1e-13 * scale, (p, k)
    # negative pin: degree 2p is not integrated exactly
    assert abs(np.sum(w * x ** (2 * p)) - _double_factorial(2 * p - 1)) > 1e-6


def test_tensor_rule_per_dimension_degree(ora):
    n, p = 3, 3
    xi, Wt = ora.rule(n, W.RULE_GH, p)
    assert xi.shape == (p ** n, n)
    for a in range(6):
        for b in range(6):
            for c in (0, 2, 5):
                val = np.sum(Wt * xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c)
                ex = 1.0
                for k in (a, b, c):
                    ex *= 0.0 if k % 2 else _double_factorial(k - 1)
                assert abs(val - ex) < 1e-11 * max(1, ex)
    # lexicographic order, dimension 0 slowest
    x1, _ = ora.gh_rule(p)
    np.testing.assert_allclose(xi[1], [x1[0], x1[0], x1[1]], atol=1e-15)
    np.testing.assert_allclose(xi[p], [x1[0], x1[1], x1[0]], atol=1e-15)


def test_degree3_rule(ora):
    n = 5
    xi, Wt = ora.rule(n, W.RULE_DEG3, 0)
    assert xi.shape == (2 * n + 1, n)
    assert abs(Wt.sum() - 1) < 1e-15 and abs(Wt[0] - (1 - n / 3)) < 1e-15
    for i in range(n):
        assert abs(np.sum(Wt * xi[:, i])) < 1e-15
        assert abs(np.sum(Wt * xi[:, i] ** 3)) < 1e-14
        assert abs(np.sum(Wt * xi[:, i] ** 4) - 3.0) < 1e-13
        for j in range(n):
            assert abs(np.sum(Wt * xi[:, i] * xi[:, j]) - (i == j)) < 1e-14
            if i != j:
                assert abs(np.sum(Wt * xi[:, i] ** 2 * xi[:, j])) < 1e-14
                # deliberate negative pin: E[xi_i^2 xi_j^2] = 1 is not reproduced
                assert abs(np.sum(Wt * xi[:, i] ** 2 * xi[:, j] ** 2) - 0.0) < 1e-14


# ------------------------------------------------------------------------ prior

def test_expm_against_library(ora):
    rng = np.random.default_rng(0)
    for d in (1, 3, 8, 12):
        M = rng.standard_normal((d, d)) * 2.0
        np.testing.assert_allclose(ora.expm(M), scipy.linalg.expm(M), rtol=1e-12, atol=1e-12)
    Nil = np.zeros((4, 4)); Nil[:2, 2:] = np.eye(2) * 0.3
    E = np.eye(4); E[:2, 2:] = np.eye(2) * 0.3
    np.testing.assert_allclose(ora.expm(Nil), E, atol=1e-16)


def test_double_integrator_prior_closed_form(ora):
    g = json.load(open(os.path.join(GOLD, "double_integrator_prior.json")))
    pb, _ = W.c1_point2d()
    pb = replace(pb, cost_kind=W.COST_NONE)
    pr = ora.prior(pb)
    dt, Qc = pb.T / pb.N, 0.8
    Phi = np.block([[np.eye(2), dt * np.eye(2)], [np.zeros((2, 2)), np.eye(2)]])
    Q = np.kron(np.array([[dt ** 3 / 3, dt ** 2 / 2], [dt ** 2 / 2, dt]]), Qc * np.eye(2))
    Qi = np.kron(np.array([[12 / dt ** 3, -6 / dt ** 2], [-6 / dt ** 2, 4 / dt]]), np.eye(2) / Qc)
    assert abs(Qi[0, 0] - g["Qinv_pos_pos_value"]) < 1e-9
    assert abs(Qi[0, 0] - eval(g["Qinv_pos_pos"])) < 1e-9
    assert abs(Qi[0, 2] - eval(g["Qinv_pos_vel"])) < 1e-9 and abs(Qi[2, 2] - eval(g["Qinv_vel_vel"])) < 1e-9
    for i in range(pb.N):
        np.testing.assert_allclose(pr.Phi[i], Phi, atol=1e-14)
        np.testing.assert_allclose(pr.Q[i], Q, rtol=1e-12, atol=1e-17)
        np.testing.assert_allclose(pr.u[i], 0.0, atol=1e-16)
    K0i = np.linalg.inv(pb.K0)
    # assembled blocks: interior diag = Phi^T Qi Phi + Qi, off = -Qi Phi, ends add start/goal
    np.testing.assert_allclose(pr.Kd[0], Phi.T @ Qi @ Phi + K0i, rtol=1e-11, atol=1e-8)
    np.testing.assert_allclose(pr.Kd[7], Phi.T @ Qi @ Phi + Qi, rtol=1e-11, atol=1e-8)
    np.testing.assert_allclose(pr.Kd[pb.N], Qi + K0i, rtol=1e-11, atol=1e-8)
    np.testing.assert_allclose(pr.Ko[3], -Qi @ Phi, rtol=1e-11, atol=1e-8)
    np.testing.assert_allclose(pr.b[0], K0i @ pb.mu0, atol=1e-9)
    np.testing.assert_allclose(pr.b[pb.N], K0i @ pb.muN, rtol=1e-12)
    np.testing.assert_allclose(pr.b[1:pb.N], 0.0, atol=1e-9)
    # prior mean solves K^-1 mubar = b
    np.testing.assert_allclose(dense(pr.Kd, pr.Ko) @ pr.mubar.ravel(), pr.b.ravel(), rtol=1e-8, atol=1e-6)


def test_ou_and_constant_drift_offsets(ora):
    th, q, dt = 0.7, 0.3, 0.25
    pb = W.Problem(n=1, m=1, N=4, T=1.0, A=np.array([[-th]]), B=np.array([[1.0]]), Qc=np.array([[q]]),
                   mu0=np.zeros(1), K0=np.eye(1), muN=np.zeros(1), KN=np.eye(1))
    pr = ora.prior(pb)
    assert abs(pr.Phi[0, 0, 0] - math.exp(-th * dt)) < 1e-15
    assert abs(pr.Q[0, 0, 0] - q * (1 - math.exp(-2 * th * dt)) / (2 * th)) < 1e-15
    A, B = W.double_integrator(1)
    av = 1.7
    pb2 = W.Problem(n=2, m=1, N=5, T=1.0, A=A, B=B, Qc=np.eye(1), a=np.array([0.0, av]),
                    mu0=np.zeros(2), K0=np.eye(2), muN=np.zeros(2), KN=np.eye(2))
    pr2 = ora.prior(pb2)
    d2 = 0.2
    np.testing.assert_allclose(pr2.u[2], [0.5 * av * d2 ** 2, av * d2], rtol=1e-14)


def test_temperature_scales_prior(ora):
    pb, _ = W.c1_point2d(N=10)
    p1 = ora.prior(pb)
    p2 = ora.prior(replace(pb, temperature=4.0))
    np.testing.assert_allclose(p2.Kd, p1.Kd / 4.0, rtol=1e-15)
    np.testing.assert_allclose(p2.b, p1.b / 4.0, rtol=1e-15)
    np.testing.assert_allclose(p2.mubar, p1.mubar, rtol=1e-10, atol=1e-9)


# ---------------------------------------------------------------------- marginals

@pytest.mark.parametrize("n,N", [(4, 1), (4, 30), (6, 17), (14, 9), (2, 40)])
def test_gbp_marginals_equal_dense_inverse(ora, n, N):
    rng = np.random.default_rng(n * 100 + N)
    Ld, Lo = rand_bt_spd(rng, n, N)
    Sd, So, ld = ora.marginals(Ld, Lo)
    M = dense(Ld, Lo)
    Sdx, Sox = blocks(np.linalg.inv(M), n)
    assert rel(Sd, Sdx) < 1e-12 and rel(So, Sox) < 1e-12
    assert abs(ld - np.linalg.slogdet(M)[1]) < 1e-10 * abs(ld) + 1e-10


def test_gbp_marginals_of_prior(ora):
    pb, _ = W.c1_point2d(N=20)
    pr = ora.prior(pb)
    Sd, So, ld = ora.marginals(pr.Kd, pr.Ko)
    M = dense(pr.Kd, pr.Ko)
    Sdx, Sox = blocks(np.linalg.inv(M), 4)
    assert rel(Sd, Sdx) < 1e-10 and rel(So, Sox) < 1e-10
    assert abs(ld - np.linalg.slogdet(M)[1]) < 1e-9


def test_not_positive_definite_is_reported(ora):
    rng = np.random.default_rng(3)
    Ld, Lo = rand_bt_spd(rng, 4, 6)
    Ld[3] -= 1e4 * np.eye(4)
    with pytest.raises(ora.OracleError) as e:
        ora.marginals(Ld, Lo)
    assert e.value.rc == ora.ENOTPD


def test_block_solve_equals_dense(ora):
    rng = np.random.default_rng(5)
    Ld, Lo = rand_bt_spd(rng, 6, 12)
    r = rng.standard_normal((13, 6))
    x = ora.block_solve(Ld, Lo, r)
    np.testing.assert_allclose(x.ravel(), np.linalg.solve(dense(Ld, Lo), r.ravel()), rtol=1e-11, atol=1e-12)


# ------------------------------------------------------------- update and KL

def _dense_kl(mu1, L1, mu0, L0):
    """KL(N(mu1, L1^-1) || N(mu0, L0^-1)) from dense matrices."""
    S1 = np.linalg.inv(L1)
    d = mu1 - mu0
    D = len(mu1)
    return 0.5 * (np.trace(L0 @ S1) + d @ L0 @ d - D + np.linalg.slogdet(L1)[1] - np.linalg.slogdet(L0)[1])


def test_thm1_trial_equals_dense_solve(ora):
    rng = np.random.default_rng(11)
    pb, _ = W.c1_point2d(N=8)
    n, N = 4, 8
    pr = ora.prior(pb)
    Ld, Lo = rand_bt_spd(rng, n, N, scale=50.0)
    mu = rng.standard_normal((N + 1, n))
    _, _, ldk = ora.marginals(Ld, Lo)
    g = rng.standard_normal((N + 1, n))
    G = np.stack([0.5 * (A + A.T) for A in rng.standard_normal((N + 1, n, n))]) * 0.5
    beta = 0.37
    rc, t = ora.trial(pb, beta, pr, mu, Ld, Lo, ldk, g, G)
    assert rc == 0
    Kinv, Lk = dense(pr.Kd, pr.Ko), dense(Ld, Lo)
    Gd = scipy.linalg.block_diag(*G)
    mu_x = np.linalg.solve(Kinv + Lk / beta, -g.ravel() + pr.b.ravel() + Lk @ mu.ravel() / beta)
    Lam_x = beta / (beta + 1) * (2 * Gd + Kinv + Lk / beta)
    assert rel(t["mu"].ravel(), mu_x) < 1e-9
    assert rel(dense(t["Ld"], t["Lo"]), Lam_x) < 1e-13
    Sdx, Sox = blocks(np.linalg.inv(Lam_x), n)
    assert rel(t["Sd"], Sdx) < 1e-9 and rel(t["So"], Sox) < 1e-9
    kl_x = _dense_kl(mu_x, Lam_x, mu.ravel(), Lk)
    assert abs(t["kl"] - kl_x) < 1e-7 * max(1, abs(kl_x))
    assert t["kl"] >= 0


def test_kl_vanishes_for_tiny_step(ora):
    rng = np.random.default_rng(12)
    pb, _ = W.c1_point2d(N=6)
    pr = ora.prior(pb)
    Ld, Lo = rand_bt_spd(rng, 4, 6, scale=10.0)
    mu = rng.standard_normal((7, 4))
    _, _, ldk = ora.marginals(Ld, Lo)
    g = rng.standard_normal((7, 4))
    G = np.zeros((7, 4, 4))
    kls = []
    for beta in (1e-2, 1e-3, 1e-4):
        rc, t = ora.trial(pb, beta, pr, mu, Ld, Lo, ldk, g, G)
        assert rc == 0 and t["kl"] >= -1e-12
        kls.append(t["kl"])
    # KL(q_beta || q_k) = O(beta^2) as beta -> 0
    assert kls[1] < kls[0] / 50 and kls[2] < kls[1] / 50


def test_no_obstacles_closed_form_recursion(ora):
    pb, op = W.c1_point2d(N=15)
    pb = replace(pb, cost_kind=W.COST_NONE)
    pr = ora.prior(pb)
    beta, s = 0.5, 3.0
    op1 = replace(op, kl_eps=float("inf"), beta_max=beta, iters=7, init_kind=1, init_scale=s)
    st = ora.plan(pb, op1)
    Lam0 = np.stack([s * np.eye(4)] * 16)
    ex_d = pr.Kd + (beta + 1) ** -7 * (Lam0 - pr.Kd)
    ex_o = pr.Ko + (beta + 1) ** -7 * (0.0 - pr.Ko)
    assert rel(st.Ld, ex_d) < 1e-12 and rel(st.Lo, ex_o) < 1e-12
    assert all(l["beta"] == beta and l["trials"] == 1 for l in st.logs)
    # with Lambda_0 = K^-1 the mean contracts to the GP prior mean geometrically
    op2 = replace(op, kl_eps=float("inf"), beta_max=beta, iters=6)
    st2 = ora.plan(pb, op2)
    mu0 = ora.init_mean(pb)
    np.testing.assert_allclose(st2.mu - pr.mubar, (beta + 1) ** -6 * (mu0 - pr.mubar), rtol=1e-7, atol=1e-8)


def test_no_obstacles_fixed_point_is_gp_posterior(ora):
    pb, op = W.c1_point2d(N=10)
    pb = replace(pb, cost_kind=W.COST_NONE)
    pr = ora.prior(pb)
    st = ora.plan(pb, replace(op, kl_eps=float("inf"), iters=95))
    np.testing.assert_allclose(st.mu, pr.mubar, rtol=1e-12, atol=1e-11)
    K = np.linalg.inv(dense(pr.Kd, pr.Ko))
    Sdx, _ = blocks(K, 4)
    assert rel(st.Sd, Sdx) < 1e-11
    # the posterior conditioned on start and goal: end means pinned near mu0 / muN
    assert np.linalg.norm(st.mu[0] - pb.mu0) < 0.1 and np.linalg.norm(st.mu[-1] - pb.muN) < 0.1


def _quadratic_problem(N=9, seed=4):
    rng = np.random.default_rng(seed)
    pb, op = W.c1_point2d(N=N)
    n = 4
    Wm = []
    for _ in range(N + 1):
        A = rng.standard_normal((n, n))
        Wm.append(A @ A.T * 0.5 + 0.1 * np.eye(n))
    c = rng.standard_normal((N + 1, n)) * 3
    pb = replace(pb, cost_kind=W.COST_QUADRATIC, quad_c=c, quad_W=np.stack(Wm))
    return pb, op


def test_quadratic_cost_moments_closed_form(ora):
    pb, op = _quadratic_problem()
    rng = np.random.default_rng(9)
    for i in (0, 4):
        A = rng.standard_normal((4, 4))
        Sig = A @ A.T + 0.3 * np.eye(4)
        mu = rng.standard_normal(4)
        for p in (3, 4, 6):
            S0, S1, S2 = ora.quad_moments(pb, replace(op, gh_p=p), i, mu, Sig)
            Wi, ci = pb.quad_W[i], pb.quad_c[i]
            e = mu - ci
            assert abs(S0 - 0.5 * (np.trace(Wi @ Sig) + e @ Wi @ e)) < 1e-10 * abs(S0)
            np.testing.assert_allclose(S1, Sig @ Wi @ e, rtol=1e-10, atol=1e-10)
            g, G = ora.gradients(Sig, S0, S1, S2)
            np.testing.assert_allclose(g, Wi @ e, rtol=1e-9, atol=1e-10)
            np.testing.assert_allclose(2 * G, Wi, rtol=1e-9, atol=1e-10)


def test_quadratic_pseudo_obstacles_fixed_point(ora):
    pb, op = _quadratic_problem(N=7)
    pr = ora.prior(pb)
    beta = 0.5
    st = ora.plan(pb, replace(op, kl_eps=float("inf"), beta_max=beta, iters=95))
    Kinv = dense(pr.Kd, pr.Ko)
    Wd = scipy.linalg.block_diag(*pb.quad_W)
    Lstar = Kinv + Wd
    mustar = np.linalg.solve(Lstar, pr.b.ravel() + Wd @ pb.quad_c.ravel())
    assert rel(dense(st.Ld, st.Lo), Lstar) < 1e-12
    assert rel(st.mu.ravel(), mustar) < 1e-10
    # exact k-step precision recursion from Lambda_0 = K^-1
    st5 = ora.plan(pb, replace(op, kl_eps=float("inf"), beta_max=beta, iters=5))
    ex = Lstar + (beta + 1) ** -5 * (Kinv - Lstar)
    assert rel(dense(st5.Ld, st5.Lo), ex) < 1e-12


def test_bisection_accepts_beta_max_and_halves(ora):
    pb, op = W.c1_point2d(N=20, iters=3)
    st = ora.plan(pb, replace(op, kl_eps=float("inf")))
    assert all(l["beta"] == 0.5 and l["trials"] == 1 for l in st.logs)
    # a bound tight enough to bind: accepted beta is a dyadic fraction of beta_max
    st2 = ora.plan(pb, replace(op, kl_eps=0.05))
    for l in st2.logs:
        assert l["kl"] <= 0.05 + 1e-12
        assert l["trials"] in (1, 11)
        if l["trials"] == 11:
            k = l["beta"] / 0.5 * 1024
            assert abs(k - round(k)) < 1e-9 and l["beta"] < 0.5


def test_replay_beta(ora):
    pb, op = W.c1_point2d(N=20, iters=4)
    st = ora.plan(pb, op)
    betas = np.array([l["beta"] for l in st.logs])
    st2 = ora.plan(pb, replace(op, replay_beta=betas))
    np.testing.assert_array_equal(st2.mu, st.mu)
    assert not any(l["replayed"] for l in st2.logs)


# --------------------------------------------------------------- cost and SDF

def _affine_map(a, d, cell=0.125, n=64, origin=(-2.0, -2.0)):
    xs = origin[0] + cell * np.arange(n)
    ys = origin[1] + cell * np.arange(n)
    X, Y = np.meshgrid(xs, ys)
    return (a[0] * X + a[1] * Y + d).astype(np.float32)


def test_sdf_bilinear_nodes_affine_and_clamp(ora):
    pb, _ = W.c1_point2d(N=4)
    a, d = (0.5, -0.25), 0.75
    pb = replace(pb, sdf=_affine_map(a, d), sdf_origin=(-2.0, -2.0, 0.0), sdf_cell=0.125)
    rng = np.random.default_rng(1)
    for _ in range(50):
        p = rng.uniform(-1.9, 5.7, size=2)
        assert abs(ora.sdf(pb, p) - (a[0] * p[0] + a[1] * p[1] + d)) < 1e-12
    # outside the grid the coordinate is clamped to the border
    far = ora.sdf(pb, (100.0, 0.0))
    edge = ora.sdf(pb, (-2.0 + 0.125 * 63, 0.0))
    assert abs(far - edge) < 1e-12
    g = pb.sdf
    assert ora.sdf(pb, (-2.0 + 0.125 * 5, -2.0 + 0.125 * 7)) == float(g[7, 5])


def test_affine_sdf_hinge_is_quadratic(ora):
    """A half-plane SDF with a margin larger than any sigma-point distance:
    psi = sigma (k - a^T p)^2 is quadratic, so the moments have closed forms."""
    a, d, sig, eps = np.array([0.5, 0.25]), 0.5, 0.7, 40.0
    pb, op = W.c1_point2d(N=4)
    pb = replace(pb, sdf=_affine_map(a, d, n=128), sdf_origin=(-2.0, -2.0, 0.0), sdf_cell=0.125,
                 eps=eps, sigma_obs=sig)
    ta = np.zeros(4); ta[:2] = a
    k = eps - d
    rng = np.random.default_rng(2)
    A = rng.standard_normal((4, 4)) * 0.3
    Sig = A @ A.T + 0.05 * np.eye(4)
    mu = np.array([4.0, 5.0, 0.3, -0.2])
    S0, S1, S2 = ora.quad_moments(pb, replace(op, gh_p=3), 2, mu, Sig)
    r = k - ta @ mu
    assert abs(S0 - sig * (r * r + ta @ Sig @ ta)) < 1e-9 * S0
    g, G = ora.gradients(Sig, S0, S1, S2)
    np.testing.assert_allclose(g, -2 * sig * r * ta, rtol=1e-8, atol=1e-9)
    np.testing.assert_allclose(G, sig * np.outer(ta, ta), rtol=1e-8, atol=1e-9)
    # psi form 1 (h^2 / sigma^2)
    pb1 = replace(pb, psi_form=1)
    S0b, _, _ = ora.quad_moments(pb1, replace(op, gh_p=3), 2, mu, Sig)
    assert abs(S0b - S0 / sig ** 3) < 1e-9 * S0b


def test_hinge_inactive_gives_zero_and_factor_set(ora):
    pb, op = W.c1_point2d(N=4)
    pb = replace(pb, sdf=np.full((180, 180), 10.0, dtype=np.float32))
    S0, S1, S2 = ora.quad_moments(pb, op, 1, np.zeros(4), np.eye(4) * 0.01)
    assert S0 == 0.0 and not S1.any() and not S2.any()
    pb2 = replace(pb, sdf=np.full((180, 180), -1.0, dtype=np.float32), factor_set=1)
    assert ora.psi(pb2, 0, np.zeros(4)) == 0.0 and ora.psi(pb2, 4, np.zeros(4)) == 0.0
    assert abs(ora.psi(pb2, 2, np.zeros(4)) - 0.5 * 1.5 ** 2) < 1e-15


def _polar_integral(f, rmax):
    """Integral of f(x, y, rho) * rho over the disk of radius rmax around the
    obstacle centre, in polar coordinates (scipy's adaptive quadrature)."""
    from scipy import integrate
    return integrate.dblquad(lambda rho, th: f(th, rho) * rho, 0.0, 2 * math.pi, 0.0, rmax,
                             epsabs=1e-13, epsrel=1e-11)[0]


def test_disk_hinge_moments_match_independent_integral(ora):
    """Expected hinge cost of one disk obstacle (Sec. 4.2: E[psi] and E[psi (x - mu)]
    over a factor's marginal) against an independent integral.

    The hinge sigma * max(0, eps - sdf)^2 of a disk (centre c, radius r) is
    supported on |p - c| < r + eps, so E[psi] and its first moment are
    integrals of the exact disk SDF against the position marginal's density,
    evaluated here by scipy in polar coordinates around c.  The oracle takes
    the same expectations by its own route: a node-centred FP32 grid with
    bilinear lookups, a 20-point-per-dimension Gauss-Hermite tensor rule over
    all four state dimensions and sigma points from the lower Cholesky factor
    of a correlated covariance.  The hinge is only C^1 at the band's edge, so
    the rule converges slowly (0.3% at 12 points, 5e-5 at 20), and the 0.02 m
    grid adds an interpolation error of about cell^2 / (8 |p - c|); 3e-3
    covers both.  The obstacle and the mean sit off the diagonal, so a swapped
    grid axis (61% off), a wrong hinge sign, weight form or origin fails."""
    cx, cy, r, eps, sig = 1.3, 0.6, 0.9, 0.5, 0.7
    org, cell = (-2.0, -2.5), 0.02
    pb, op = W.c1_point2d(N=4)
    grid = W.sdf_grid_2d(300, 300, org, cell, disks=[(cx, cy, r)])
    pb = replace(pb, sdf=grid, sdf_origin=(org[0], org[1], 0.0), sdf_cell=cell, eps=eps, sigma_obs=sig)
    mu = np.array([2.55, 0.95, 0.4, -0.3])
    A = np.array([[0.30, 0.0, 0.0, 0.0], [0.12, 0.22, 0.0, 0.0], [0.05, -0.02, 0.3, 0.0], [0.01, 0.03, 0.04, 0.2]])
    Sig = A @ A.T
    P, m2 = Sig[:2, :2], mu[:2]
    Pi, norm = np.linalg.inv(P), 1.0 / (2 * math.pi * math.sqrt(np.linalg.det(P)))

    def weighted(k):
        def f(th, rho):
            d = np.array([cx + rho * math.cos(th), cy + rho * math.sin(th)]) - m2
            w = sig * (r + eps - rho) ** 2 * norm * math.exp(-0.5 * d @ Pi @ d)
            return w if k < 0 else w * d[k]
        return f

    E0 = _polar_integral(weighted(-1), r + eps)
    E1 = np.array([_polar_integral(weighted(k), r + eps) for k in (0, 1)])
    S0, S1, _ = ora.quad_moments(pb, replace(op, gh_p=20), 2, mu, Sig)
    assert abs(S0 - E0) <= 3e-3 * E0, (S0, E0)
    assert np.abs(S1[:2] - E1).max() <= 3e-3 * np.abs(E1).max(), (S1[:2], E1)


def test_sphere_hinge_expectation_matches_independent_integral(ora):
    """The trilinear 3-D path: E[psi] of one spherical obstacle for the 3-D point
    robot (n = 6) against scipy's integral of the exact sphere SDF in
    spherical coordinates around the centre.  The oracle runs a 10-point rule
    on all six dimensions (10^6 points) over a 0.025 m FP32 grid stored
    (z, y, x); it converges to 4e-5 here, and 2e-3 also covers the grid's
    interpolation error.  Centre and mean differ in every coordinate, so a
    permuted grid axis fails."""
    from scipy import integrate
    c, r, eps, sig = np.array([0.9, 0.5, 0.7]), 0.7, 0.4, 0.6
    org, cell = (-1.0, -1.2, -0.9), 0.025
    pb, op = W.point3d(N=4)
    xs, ys, zs = (org[k] + cell * np.arange(m) for k, m in enumerate((140, 120, 110)))
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    grid = (np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) - r).astype(np.float32)
    pb = replace(pb, sdf=grid, sdf_origin=org, sdf_cell=cell, eps=eps, sigma_obs=sig)
    mu = np.array([1.85, 0.95, 1.1, 0.2, -0.1, 0.3])
    rng = np.random.default_rng(3)
    A = np.tril(rng.uniform(-0.08, 0.08, (6, 6))) + np.diag([0.25, 0.2, 0.18, 0.2, 0.2, 0.2])
    Sig = A @ A.T
    P, m3 = Sig[:3, :3], mu[:3]
    Pi, norm = np.linalg.inv(P), 1.0 / ((2 * math.pi) ** 1.5 * math.sqrt(np.linalg.det(P)))

    def f(rho, th, ph):
        u = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        d = c + rho * u - m3
        return sig * (r + eps - rho) ** 2 * norm * math.exp(-0.5 * d @ Pi @ d) * rho * rho * math.sin(th)

    E0 = integrate.tplquad(f, 0.0, 2 * math.pi, 0.0, math.pi, 0.0, r + eps, epsabs=1e-11, epsrel=1e-8)[0]
    S0, _, _ = ora.quad_moments(pb, replace(op, gh_p=10), 2, mu, Sig)
    assert abs(S0 - E0) <= 2e-3 * E0, (S0, E0)


def test_arm_fk_invariants(ora):
    pb, _ = W.c3_arm(N=10)
    rng = np.random.default_rng(0)
    c0 = ora.arm_fk(pb, np.zeros(7))
    # base link spheres sit on the z axis at their fractions of d_0
    base = pb.sphere_link == 0
    np.testing.assert_allclose(c0[base, :2], 0.0, atol=1e-15)
    np.testing.assert_allclose(c0[base, 2], pb.sphere_off[base, 2], atol=1e-15)
    for _ in range(5):
        q = rng.uniform(-np.pi, np.pi, size=7)
        c = ora.arm_fk(pb, q)
        # rigid links: distances between spheres of one link do not depend on q
        for j in np.unique(pb.sphere_link):
            idx = np.nonzero(pb.sphere_link == j)[0]
            for u in idx:
                for v in idx:
                    assert abs(np.linalg.norm(c[u] - c[v]) - np.linalg.norm(c0[u] - c0[v])) < 1e-12
        # joint 0 rotates the whole arm about z
        q2 = q.copy(); q2[0] += 0.8
        c2 = ora.arm_fk(pb, q2)
        R = np.array([[np.cos(0.8), -np.sin(0.8), 0], [np.sin(0.8), np.cos(0.8), 0], [0, 0, 1]])
        np.testing.assert_allclose(c2, c @ R.T, atol=1e-12)
        # the last joint only spins the end link about its own axis: links < 6 unchanged
        q3 = q.copy(); q3[6] += 1.1
        c3 = ora.arm_fk(pb, q3)
        np.testing.assert_allclose(c3[pb.sphere_link < 6], c[pb.sphere_link < 6], atol=1e-14)


def test_planar_arm_cost_closed_form(ora):
    """Arm cost psi = sum_s sigma * max(0, eps + r_s - sdf(c_s))^2 on a special
    case with a textbook answer.  With every link twist, offset and joint
    offset zero, the DH chain is a planar arm: link j starts at
    P_j = sum_{k<j} l_k (cos th_k, sin th_k) with th_k = q_0 + ... + q_k, and a
    sphere fixed at (u, v, w) in link j's frame sits at
    P_j + u (cos th_j, sin th_j) + v (-sin th_j, cos th_j) + w e_z.  An affine
    SDF a.p + d is reproduced exactly by trilinear interpolation, so psi has a
    closed form up to the grid's FP32 rounding.  A wrong rotation order, a
    translation applied before its rotation, a dropped radius or a hinge sign
    fails it."""
    pb, _ = W.c3_arm(N=4)
    lengths = np.array([0.3, 0.25, 0.2, 0.15, 0.12, 0.1, 0.08])
    dh = np.zeros((7, 4))
    dh[:, 0] = lengths
    rng = np.random.default_rng(11)
    links = np.repeat(np.arange(7), 2).astype(np.int32)
    offs = np.stack([rng.uniform(0.0, 1.0, 14) * lengths[links], rng.uniform(-0.05, 0.05, 14),
                     rng.uniform(-0.05, 0.05, 14)], axis=1)
    radii = rng.uniform(0.05, 0.12, 14)
    a, d = np.array([0.6, -0.5, 0.3]), 0.25
    org, cell, shape = (-1.5, -1.5, -0.3), 0.05, (13, 61, 61)      # (z, y, x) nodes
    zs, ys, xs = (org[2 - k] + cell * np.arange(m) for k, m in enumerate(shape))
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    grid = (a[0] * X + a[1] * Y + a[2] * Z + d).astype(np.float32)
    eps, sig = 0.3, 3.0
    pb = replace(pb, dh=dh, sphere_link=links, sphere_off=offs, sphere_r=radii, sdf=grid,
                 sdf_origin=org, sdf_cell=cell, eps=eps, sigma_obs=sig)
    active = []
    for _ in range(6):
        q = rng.uniform(-1.2, 1.2, 7)
        th = np.cumsum(q)
        P = np.concatenate([[[0.0, 0.0]], np.cumsum(lengths[:, None] * np.stack([np.cos(th), np.sin(th)], 1), 0)])
        want = np.zeros((14, 3))
        for k, j in enumerate(links):
            u, v, w = offs[k]
            want[k, :2] = P[j] + u * np.array([np.cos(th[j]), np.sin(th[j])]) + v * np.array([-np.sin(th[j]),
                                                                                             np.cos(th[j])])
            want[k, 2] = w
        np.testing.assert_allclose(ora.arm_fk(pb, q), want, atol=1e-13)
        h = np.maximum(0.0, eps + radii - (want @ a + d))
        psi = sig * np.sum(h * h)
        active.append(np.count_nonzero(h))
        x = np.concatenate([q, rng.standard_normal(7)])
        assert abs(ora.psi(pb, 2, x) - psi) <= 1e-5 * max(psi, 1e-3), (ora.psi(pb, 2, x), psi)
    assert 0 < sum(active) < 6 * 14, active      # both sides of the hinge are exercised


# ------------------------------------------------------------------------- SLR

def test_slr_recovers_affine_drift(ora):
    rng = np.random.default_rng(8)
    n, N = 6, 5
    F = rng.standard_normal((n, n))
    c = rng.standard_normal(n)
    pb = W.Problem(n=n, m=n, N=N, T=1.0, A=np.zeros((n, n)), B=np.eye(n), Qc=np.eye(n), mu0=np.zeros(n),
                   K0=np.eye(n), muN=np.zeros(n), KN=np.eye(n), dyn_kind=W.DYN_AFFINE_TEST, dyn_F=F, dyn_c=c)
    xbar = rng.standard_normal((N + 1, n))
    Sb = []
    for _ in range(N + 1):
        A = rng.standard_normal((n, n))
        Sb.append(A @ A.T + 0.1 * np.eye(n))
    for rule, p in ((W.RULE_GH, 2), (W.RULE_GH, 3), (W.RULE_DEG3, 0)):
        Al, al = ora.slr(pb, W.Options(rule=rule, gh_p=p), xbar, np.stack(Sb))
        for i in range(N):
            np.testing.assert_allclose(Al[i], F, atol=1e-11)
            np.testing.assert_allclose(al[i], c, atol=1e-11)


def test_slr_small_covariance_is_jacobian(ora):
    pb, op = W.c4_quadrotor(N=3)
    x = np.array([1.0, 2.0, 0.3, 0.7, -0.4, 0.2])
    xbar = np.tile(x, (4, 1))
    Sbar = np.stack([np.eye(6) * 1e-10] * 4)
    Al, al = ora.slr(pb, op, xbar, Sbar)
    J = np.zeros((6, 6))
    h = 1e-6
    for j in range(6):
        e = np.zeros(6); e[j] = h
        J[:, j] = (ora.drift(pb, x + e) - ora.drift(pb, x - e)) / (2 * h)
    np.testing.assert_allclose(Al[0], J, atol=1e-6)
    np.testing.assert_allclose(al[0], ora.drift(pb, x) - J @ x, atol=1e-5)
    # hover attitude: d(vx_dot)/d(phi) = -g, d(vz_dot)/d(phi) = 0 at phi = 0
    x0 = np.zeros(6)
    Al0, _ = ora.slr(pb, op, np.tile(x0, (4, 1)), Sbar)
    assert abs(Al0[0][3, 2] + 9.81) < 1e-6 and abs(Al0[0][4, 2]) < 1e-6


def test_plan_slr_runs_and_logs(ora):
    pb, op = W.c4_quadrotor(N=20, iters=3, slr_iters=3)
    st = ora.plan_slr(pb, replace(op, gh_p=2))
    assert st.slr_norms.shape == (3,) and np.all(np.isfinite(st.slr_norms))
    assert len(st.logs) == 9
    assert np.all(np.isfinite(st.mu))


def test_monotone_total_cost_small_step(ora):
    """App. B / Sec. 7.3(a): with a small step the total cost (prior +
    collision - entropy) does not increase; violations are counted."""
    pb, op = W.c1_point2d(N=25, iters=12)
    st = ora.plan(pb, replace(op, beta_max=0.05, kl_eps=float("inf")))
    tot = [l["prior_cost"] + l["collision_cost"] - l["entropy"] for l in st.logs]
    ups = sum(1 for a, b in zip(tot, tot[1:]) if b > a + 1e-9 * abs(a))
    assert ups <= 2, tot


def test_two_phase_temperature_closed_form(ora):
    """psi = 0, unbounded KL (beta = beta_max every iteration), Lambda_0 = K^-1
    at T-hat = 1, then T-hat = 10 from iteration 5: the optimum at temperature
    T is N(mu*, T K), so Lambda stays K^-1 for five iterations and then
    contracts to K^-1 / 10 at rate 1/(beta+1):
        Lambda_{5+m} = K^-1/10 + (beta+1)^-m (K^-1 - K^-1/10)."""
    pb, op = W.c1_point2d(N=20, iters=40)
    pb = replace(pb, cost_kind=W.COST_NONE)
    op = replace(op, kl_eps=float("inf"), temperature_high=10.0, switch_iter=5)
    st = ora.plan(pb, op)
    pr = ora.prior(pb)
    r = (1.0 + op.beta_max) ** -(op.iters - 5)
    want_d = pr.Kd / 10.0 + r * (pr.Kd - pr.Kd / 10.0)
    want_o = pr.Ko / 10.0 + r * (pr.Ko - pr.Ko / 10.0)
    np.testing.assert_allclose(st.Ld, want_d, rtol=1e-9, atol=1e-9 * np.abs(pr.Kd).max())
    np.testing.assert_allclose(st.Lo, want_o, rtol=1e-9, atol=1e-9 * np.abs(pr.Kd).max())
    assert all(l["beta"] == op.beta_max for l in st.logs)
    # the mean converges to the GP posterior mean, which does not depend on T-hat
    assert np.linalg.norm(st.mu - pr.mubar) <= 1e-4 * np.linalg.norm(pr.mubar)
    # entropy rises once the temperature is high (covariances grow towards 10 K)
    assert st.logs[-1]["entropy"] > st.logs[4]["entropy"] + 0.5 * pb.n * (pb.N + 1) * np.log(5.0)


# ------------------------------------------------------------ Smolyak sparse grids (Lemma 1)

def _gauss_moment(a):
    """E[prod xi_j^a_j] under N(0, I): prod (a_j - 1)!! for even a_j, else 0."""
    out = 1.0
    for m in a:
        if m % 2:
            return 0.0
        out *= math.prod(range(m - 1, 0, -2)) if m > 1 else 1.0
    return out


@pytest.mark.parametrize("d,k", [(1, 4), (2, 2), (2, 3), (3, 3), (4, 4), (6, 3)])
def test_smolyak_exact_to_total_degree(ora, d, k):
    import itertools
    xi, Wt = ora.rule(d, W.RULE_SMOLYAK, k)
    assert abs(Wt.sum() - 1.0) < 1e-13
    for deg in range(2 * k):
        for alpha in itertools.combinations_with_replacement(range(d), deg):
            a = np.bincount(alpha, minlength=d)
            val = float(np.sum(Wt * np.prod(xi ** a, axis=1)))
            assert abs(val - _gauss_moment(a)) < 1e-12 * max(1.0, _gauss_moment(a)), (a, val)
    # not exact one degree higher: xi_0^(2k) has moment (2k-1)!!
    a = np.zeros(d, dtype=int)
    a[0] = 2 * k
    assert abs(float(np.sum(Wt * xi[:, 0] ** (2 * k))) - _gauss_moment(a)) > 1e-3


def test_smolyak_small_cases(ora):
    """d = 1 is the k-point Gauss-Hermite rule; level 2 in d dims is the
    origin (weight 1 - d) and +-e_j (1/2 each)."""
    xi, Wt = ora.rule(1, W.RULE_SMOLYAK, 4)
    x4, w4 = ora.gh_rule(4)
    order = np.argsort(xi[:, 0])
    np.testing.assert_allclose(xi[order, 0], np.sort(x4), atol=1e-14)
    np.testing.assert_allclose(Wt[order], w4[np.argsort(x4)], atol=1e-14)
    xi, Wt = ora.rule(3, W.RULE_SMOLYAK, 2)
    assert len(Wt) == 7
    k0 = np.where(np.all(xi == 0.0, axis=1))[0][0]
    assert abs(Wt[k0] - (1 - 3)) < 1e-14
    assert np.allclose(np.delete(Wt, k0), 0.5)


@pytest.mark.parametrize("n,dc,k", [(4, 2, 3), (6, 3, 3), (14, 7, 2), (14, 7, 3)])
def test_smolyak_reduces_to_the_cost_coordinates(ora, n, dc, k):
    """For f depending on the leading dc coordinates, the n-dimensional grid
    of level k gives the dc-dimensional grid's value, and a trailing second
    moment xi_b^2 f gives the level k-1 value (what the reduced GPU
    quadrature uses); odd trailing moments vanish."""
    rng = np.random.default_rng(7)
    c = rng.normal(size=dc)
    f = lambda X: np.cos(X[:, :dc] @ c) + 0.3 * np.sin(X[:, 0]) ** 2
    Xn, Wn = ora.rule(n, W.RULE_SMOLYAK, k)
    Xd, Wd = ora.rule(dc, W.RULE_SMOLYAK, k)
    Xe, We = ora.rule(dc, W.RULE_SMOLYAK, k - 1)
    full = np.sum(Wn * f(Xn))
    assert abs(full - np.sum(Wd * f(Xd))) < 1e-12
    b = n - 1
    assert abs(np.sum(Wn * Xn[:, b] ** 2 * f(Xn)) - np.sum(We * f(Xe))) < 1e-12
    assert abs(np.sum(Wn * Xn[:, b] * f(Xn))) < 1e-12
    assert abs(np.sum(Wn * Xn[:, b] * Xn[:, 0] * f(Xn))) < 1e-12


# -------------------------------------------------- arm: twists and offsets

def test_arm_fk_twist_and_offset_closed_form(ora):
    """The DH chain with non-zero twists and offsets against FK written out
    from the geometry, independently of the DH matrices.  Joint 1 (a = 0,
    twist +pi/2, offset d1) turns the arm's vertical plane about z: its
    horizontal direction is x1 = (c1, s1, 0), the up direction y1 = e_z, and
    joint 2's axis is z1 = (s1, -c1, 0).  Joint 2 (length a2, offset d2 along
    z1, joint offset th02) and joint 3 (length a3, twist +pi/2) move in that
    plane: x2 = cos(t2) x1 + sin(t2) y1, x3 = cos(t2+t3) x1 + sin(t2+t3) y1
    with t2 = q2 + th02.  After joint 3's twist its y axis is z1, so a sphere
    at (r, 0, 0) in link 4's frame sits at
        (0, 0, d1) + d2 z1 + a2 x2 + a3 x3 + r (cos q4 x3 + sin q4 z1).
    A twist with the wrong sign, an offset along the wrong axis or a twist
    applied before the link's own rotation fails it."""
    pb, _ = W.c3_arm(N=4)
    d1, a2, d2, a3, th02, r = 0.31, 0.42, 0.07, 0.27, 0.35, 0.13
    dh = np.array([[0.0, np.pi / 2, d1, 0.0],
                   [a2, 0.0, d2, th02],
                   [a3, np.pi / 2, 0.0, 0.0],
                   [0.0, 0.0, 0.0, 0.0]])
    pb = replace(pb, dh=dh, sphere_link=np.array([3, 1], dtype=np.int32),
                 sphere_off=np.array([[r, 0.0, 0.0], [0.0, 0.0, 0.0]]), sphere_r=np.array([0.05, 0.05]))
    rng = np.random.default_rng(21)
    for _ in range(8):
        q = rng.uniform(-np.pi, np.pi, 4)
        c1, s1 = np.cos(q[0]), np.sin(q[0])
        t2, t23 = q[1] + th02, q[1] + th02 + q[2]
        x1, y1, z1 = np.array([c1, s1, 0.0]), np.array([0.0, 0.0, 1.0]), np.array([s1, -c1, 0.0])
        x2 = np.cos(t2) * x1 + np.sin(t2) * y1
        x3 = np.cos(t23) * x1 + np.sin(t23) * y1
        want_end = np.array([0.0, 0.0, d1]) + d2 * z1 + a2 * x2 + a3 * x3 + r * (np.cos(q[3]) * x3
                                                                                 + np.sin(q[3]) * z1)
        # a sphere with zero offset on link 2 sits at the origin of link 1's frame after Tz(d1)
        want_base = np.array([0.0, 0.0, d1])
        c = ora.arm_fk(pb, q)
        np.testing.assert_allclose(c[0], want_end, atol=1e-13)
        np.testing.assert_allclose(c[1], want_base, atol=1e-13)


# ----------------------------------------------- natural-gradient update (NGD)

def _ngd_problem(seed=3):
    """n = 4, N = 1: one pair of states, quadratic pseudo-obstacles."""
    rng = np.random.default_rng(seed)
    pb, op = W.c1_point2d(N=1)
    pb = replace(pb, T=1.0, K0=0.5 * np.eye(4), KN=0.5 * np.eye(4))
    Wm = []
    for _ in range(2):
        A = rng.standard_normal((4, 4))
        Wm.append(A @ A.T * 0.3 + 0.2 * np.eye(4))
    c = rng.standard_normal((2, 4))
    pb = replace(pb, cost_kind=W.COST_QUADRATIC, quad_c=c, quad_W=np.stack(Wm))
    return pb, op


def test_ngd_step_is_the_fisher_natural_gradient_step(ora):
    """Sec. 3.1(d): the NGD step is delta theta = beta G(theta)^-1 grad L with
    the Fisher matrix G.  Here both G and the gradient come from central
    differences in the natural parameters eta = (Lambda mu, -Lambda/2) (the
    Fisher matrix as the Jacobian of the expectation parameters E[T(x)]), and
    the objective J = -L = E[psi] + KL(q || N(mu_bar, K)) + const is evaluated
    in closed form for quadratic costs.  The oracle's step must equal
    eta - beta G^-1 grad_eta J.  A missing factor 2 on G, a wrong sign or the
    step taken on the mean without the new precision fails it."""
    pb, op = _ngd_problem()
    n, D = 4, 8
    pr = ora.prior(pb)
    Kinv = dense(pr.Kd, pr.Ko)
    mubar = pr.mubar.ravel()
    rng = np.random.default_rng(5)
    A = rng.standard_normal((D, D))
    Lam_k = A @ A.T / D + 1.5 * np.eye(D)
    mu_k = rng.standard_normal(D)
    Wd = scipy.linalg.block_diag(*pb.quad_W)
    cvec = pb.quad_c.ravel()
    iu = np.triu_indices(D)

    def unpack(v):
        E2 = np.zeros((D, D))
        E2[iu] = v[D:]
        E2 = E2 + np.triu(E2, 1).T
        Lam = -2.0 * E2
        Sig = np.linalg.inv(Lam)
        return Sig @ v[:D], Sig, Lam

    def pack(mu, Lam):
        E2 = -0.5 * Lam
        return np.concatenate([Lam @ mu, E2[iu]])

    def J(v):
        mu, Sig, Lam = unpack(v)
        e = mu - cvec
        epsi = 0.5 * (np.trace(Wd @ Sig) + e @ Wd @ e)
        dp = mu - mubar
        prior = 0.5 * (np.trace(Kinv @ Sig) + dp @ Kinv @ dp)
        return epsi + prior - 0.5 * np.linalg.slogdet(Sig)[1]

    def m(v):
        mu, Sig, _ = unpack(v)
        S2 = Sig + np.outer(mu, mu)
        w = np.where(iu[0] == iu[1], 1.0, 2.0)       # tr(E2 x x^T) counts off-diagonals twice
        return np.concatenate([mu, w * S2[iu]])

    v0 = pack(mu_k, Lam_k)
    h = 1e-5
    P = v0.size
    grad = np.zeros(P)
    F = np.zeros((P, P))
    for j in range(P):
        dv = np.zeros(P)
        dv[j] = h
        grad[j] = (J(v0 + dv) - J(v0 - dv)) / (2 * h)
        F[:, j] = (m(v0 + dv) - m(v0 - dv)) / (2 * h)
    beta = 0.3
    v1 = v0 - beta * np.linalg.solve(F, grad)
    mu_x, _, Lam_x = unpack(v1)

    Ld, Lo = blocks(Lam_k, n)
    Sd, _, ldk = ora.marginals(Ld, Lo)
    g, G = np.zeros((2, n)), np.zeros((2, n, n))
    for i in range(2):
        S0, S1, S2 = ora.quad_moments(pb, op, i, mu_k[i * n:(i + 1) * n], Sd[i])
        g[i], G[i] = ora.gradients(Sd[i], S0, S1, S2)
    rc, t = ora.trial(pb, beta, pr, mu_k.reshape(2, n), Ld, Lo, ldk, g, G, update=ora.UPDATE_NGD)
    assert rc == 0
    assert rel(dense(t["Ld"], t["Lo"]), Lam_x) < 1e-7
    assert rel(t["mu"].ravel(), mu_x) < 1e-7
    # the KL-proximal step at the same beta is a different point (same fixed point, other path)
    rc, tp = ora.trial(pb, beta, pr, mu_k.reshape(2, n), Ld, Lo, ldk, g, G)
    assert rel(dense(tp["Ld"], tp["Lo"]), Lam_x) > 1e-3


def test_ngd_no_obstacles_closed_form(ora):
    """psi = 0, unbounded KL, fixed beta: Lambda_k = K^-1 + (1-beta)^k
    (Lambda_0 - K^-1); from Lambda_0 = K^-1 the mean contracts to the GP
    prior mean by (1-beta) per iteration."""
    pb, op = W.c1_point2d(N=12)
    pb = replace(pb, cost_kind=W.COST_NONE)
    pr = ora.prior(pb)
    beta, s = 0.4, 2.0
    st = ora.plan(pb, replace(op, update=1, kl_eps=float("inf"), beta_max=beta, iters=6, init_kind=1,
                              init_scale=s))
    Lam0 = np.stack([s * np.eye(4)] * 13)
    assert rel(st.Ld, pr.Kd + (1 - beta) ** 6 * (Lam0 - pr.Kd)) < 1e-12
    assert rel(st.Lo, pr.Ko + (1 - beta) ** 6 * (0.0 - pr.Ko)) < 1e-12
    st2 = ora.plan(pb, replace(op, update=1, kl_eps=float("inf"), beta_max=beta, iters=5))
    mu0 = ora.init_mean(pb)
    np.testing.assert_allclose(st2.mu - pr.mubar, (1 - beta) ** 5 * (mu0 - pr.mubar), rtol=1e-7, atol=1e-8)


def test_ngd_quadratic_pseudo_obstacles_fixed_point(ora):
    """The NGD iteration has the same fixed point as Thm 1's: precision
    K^-1 + blockdiag(W) and mean (K^-1 + W)^-1 (b + W c); its precision
    contracts at rate (1 - beta)."""
    pb, op = _quadratic_problem(N=7)
    pr = ora.prior(pb)
    Kinv = dense(pr.Kd, pr.Ko)
    Wd = scipy.linalg.block_diag(*pb.quad_W)
    Lstar = Kinv + Wd
    mustar = np.linalg.solve(Lstar, pr.b.ravel() + Wd @ pb.quad_c.ravel())
    beta = 0.5
    st = ora.plan(pb, replace(op, update=1, kl_eps=float("inf"), beta_max=beta, iters=80))
    assert rel(dense(st.Ld, st.Lo), Lstar) < 1e-12
    assert rel(st.mu.ravel(), mustar) < 1e-10
    st4 = ora.plan(pb, replace(op, update=1, kl_eps=float("inf"), beta_max=beta, iters=4))
    assert rel(dense(st4.Ld, st4.Lo), Lstar + (1 - beta) ** 4 * (Kinv - Lstar)) < 1e-12


# ------------------------------------------- step-size search records and replay

def test_search_records_follow_the_bisection(ora):
    """Every trial of the step-size search is recorded; the accepted step is
    the largest feasible trial, and the trials walk the dyadic bisection."""
    pb, op = W.c1_point2d(N=20, iters=4)
    op = replace(op, kl_eps=0.5)
    st = ora.plan(pb, op)
    for k, l in enumerate(st.logs):
        tr = [t for t in st.trials if t["iter"] == k]
        assert len(tr) == l["trials"]
        assert tr[0]["beta"] == op.beta_max
        feas = [t["beta"] for t in tr if t["feasible"]]
        assert l["beta"] == (max(feas) if feas else 0.0)
        lo, hi = 0.0, op.beta_max
        for t in tr[1:]:
            assert t["beta"] == 0.5 * (lo + hi)
            lo, hi = (t["beta"], hi) if t["feasible"] else (lo, t["beta"])
            assert t["feasible"] == (t["pd"] and t["kl"] <= op.kl_eps)
        assert l["beta_own"] == l["beta"] and not l["replayed"]
        assert l["pd_margin"] == min(abs(t["rel_pivot"]) for t in tr)


def test_replay_records_the_own_search(ora):
    """In replay mode the oracle still searches on its own (beta_own) and
    takes the given step, recording its KL without enforcing it."""
    pb, op = W.c1_point2d(N=20, iters=4)
    op = replace(op, kl_eps=0.5)
    st = ora.plan(pb, op)
    betas = np.array([l["beta"] for l in st.logs])
    forced = betas.copy()
    forced[1] = betas[1] * 2          # a step the bound rejects
    st2 = ora.plan(pb, replace(op, replay_beta=forced))
    assert not st2.logs[0]["replayed"] and st2.logs[1]["replayed"]
    assert st2.logs[1]["beta"] == forced[1] and st2.logs[1]["beta_own"] == betas[1]
    assert st2.logs[1]["kl"] > op.kl_eps      # recorded, not enforced
    np.testing.assert_array_equal(st2.logs[0]["beta"], betas[0])
