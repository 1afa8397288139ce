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


# Tie margins of the step-size search (App. C).  A GPU plan may take a
# different bisection branch than the oracle only at a trial where the two
# sides' arithmetic straddles a decision boundary: |KL - eps| / eps below
# TIE_KL, or the smallest relative pivot of Lambda'(beta) below TIE_PD in
# magnitude.  FP32 quadrature perturbs g and G by ~1e-6 relative (25-point
# sums of FP32 bilinear lookups), which moves a KL near eps by about as much;
# in FP64 both sides agree to ~1e-12 on small problems.
TIE_MIXED = dict(kl=1e-5, pd=1e-5)
TIE_FP64 = dict(kl=1e-9, pd=1e-10)


_KAPPA = {}


def prior_condition(pb):
    """2-norm condition number of the prior precision K^-1 (cached per
    problem shape)."""
    key = (pb.n, pb.N, pb.T, pb.dyn_kind, np.asarray(pb.Qc).tobytes(), np.asarray(pb.K0).tobytes(),
           np.asarray(pb.KN).tobytes(), np.asarray(pb.A).tobytes())
    if key not in _KAPPA:
        pr = oracle.prior(pb)
        n, N = pb.n, pb.N
        D = n * (N + 1)
        M = np.zeros((D, D))
        for i in range(N + 1):
            M[i * n:(i + 1) * n, i * n:(i + 1) * n] = pr.Kd[i]
        for i in range(N):
            M[(i + 1) * n:(i + 2) * n, i * n:(i + 1) * n] = pr.Ko[i]
            M[i * n:(i + 1) * n, (i + 1) * n:(i + 2) * n] = pr.Ko[i].T
        _KAPPA[key] = float(np.linalg.cond(M))
    return _KAPPA[key]


def tie_from_conditioning(pb, prec):
    """Tie margins for a precision form: the fixed margins above, or ten times
    kappa(K^-1) times the unit roundoff of the recursions (2^-53 in FP64,
    2^-48 in double-float) where that is larger -- the size by which two
    correct eliminations of the chain can differ.  For the 750-step robot
    (kappa 4.7e10) this is 1.7e-3 in double-float and 5.2e-5 in FP64."""
    base = TIE_FP64 if prec == 0 else TIE_MIXED
    u = 2.0 ** -48 if prec == 2 else 2.0 ** -53
    floor = 10.0 * prior_condition(pb) * u
    return dict(kl=max(base["kl"], floor), pd=max(base["pd"], floor))


def gpu_solve(problems, options, precision):
    import paper_2411_03416_b300 as pg
    return pg.solve(problems, options, precision)


def oracle_solve(pb, op):
    return oracle.solve(pb, op)


def implied_decisions(beta, beta_max, max_bisect):
    """The trials (beta_t, feasible_t) of the App. C search that end at the
    accepted step `beta`: beta_max first; if it is infeasible, max_bisect
    halvings of [0, beta_max], each keeping the feasible side.  The accepted
    step is the final lower end, so trial t was feasible exactly when
    beta >= its midpoint (all values are dyadic, exact in FP64)."""
    if beta == beta_max:
        return [(beta_max, True)]
    out = [(beta_max, False)]
    lo, hi = 0.0, beta_max
    for _ in range(max_bisect):
        mid = 0.5 * (lo + hi)
        f = beta >= mid
        out.append((mid, f))
        lo, hi = (mid, hi) if f else (lo, mid)
    assert lo == beta, f"step {beta} is not a result of the bisection of [0, {beta_max}]"
    return out


def check_tie_replays(ora, gbetas, glogs, op, tie):
    """`ora` is the oracle run that replays the GPU's steps (running its own
    search at every iteration from the replayed iterate).  At every iteration
    where the GPU's step differs from the oracle's own, walk both searches to
    the first trial they decide differently; that trial must be a tie
    (|KL - eps| / eps < tie["kl"], or |relative pivot| < tie["pd"]).  The
    oracle's KL at the GPU's accepted step must also be within the KL margin of
    the bound.  Returns one record per replayed decision."""
    eps = op.kl_eps
    out = []
    for k, l in enumerate(ora.logs):
        if not l["replayed"]:
            continue
        trials = [t for t in ora.trials if t["iter"] == k]
        dec = implied_decisions(gbetas[k], op.beta_max, op.max_bisect)
        flip = None
        for j, (bt, feas) in enumerate(dec):
            assert j < len(trials) and trials[j]["beta"] == bt, (k, j, bt)
            if trials[j]["feasible"] != feas:
                flip = (j, trials[j])
                break
        assert flip is not None, f"iteration {k}: steps differ but every trial decided alike"
        j, t = flip
        kl_gap = abs(t["kl"] - eps) / eps if (t["pd"] and np.isfinite(eps) and eps > 0) else np.inf
        pd_gap = abs(t["rel_pivot"]) if np.isfinite(t["rel_pivot"]) else np.inf
        rec = dict(iter=k, trial=j, beta_gpu=float(gbetas[k]), beta_oracle=l["beta_own"], kl_gap=kl_gap,
                   pd_gap=pd_gap)
        assert kl_gap < tie["kl"] or pd_gap < tie["pd"], \
            f"iteration {k}: GPU step {gbetas[k]} vs oracle {l['beta_own']} decided apart at trial {j} " \
            f"(beta {t['beta']}) with no tie: {rec}"
        if gbetas[k] > 0 and np.isfinite(eps) and eps > 0:
            assert l["kl"] <= eps * (1 + tie["kl"]), (k, l["kl"], eps)
            assert abs(glogs[k]["kl"] - l["kl"]) <= tie["kl"] * eps, (k, glogs[k]["kl"], l["kl"])
        out.append(rec)
    return out


def compare_plan(pb, op, gres, *, rtol_mu, rtol_sigma, tie=None, prec=None, max_replays=None, slr=False):
    """Compares one GPU plan with the oracle.  If the accepted step sizes
    differ, the oracle is rerun replaying the GPU's steps, and every decision
    that differs must be a tie of the step-size search (check_tie_replays).
    `tie` defaults to tie_from_conditioning(pb, prec) when the precision form
    is given, else to TIE_MIXED for mixed-precision tolerances and TIE_FP64
    otherwise; `max_replays` bounds the replayed decisions."""
    if tie is None:
        if prec is not None:
            tie = tie_from_conditioning(pb, prec)
        else:
            tie = TIE_MIXED if rtol_mu >= 1e-6 else TIE_FP64
    ora = oracle_solve(pb, op)
    gb = np.array([l["beta"] for l in gres.logs])
    ob = np.array([l["beta"] for l in ora.logs])
    replays = []
    if gb.shape != ob.shape or not np.array_equal(gb, ob):
        assert gb.shape == ob.shape, (gb.shape, ob.shape)
        ora = oracle_solve(pb, replace(op, replay_beta=gb))
        replays = check_tie_replays(ora, gb, gres.logs, op, tie)
    em = rel_mu(gres.mu, ora.mu)
    es = rel_sigma(gres.Sd, ora.Sd)
    # element by element: no state's mean may be off by more than the
    # tolerance times the trajectory's largest coordinate
    ea = float(np.max(np.abs(gres.mu - ora.mu)) / np.max(np.abs(ora.mu)))
    info = dict(err_mu=em, err_sigma=es, err_mu_maxabs=ea, replays=len(replays), replay_records=replays,
                n_iters=len(gb), max_abs_mu=float(np.max(np.abs(gres.mu - ora.mu))))
    assert em <= rtol_mu, info
    assert ea <= rtol_mu, info
    assert es <= rtol_sigma, info
    if max_replays is not None:
        assert len(replays) <= max_replays, info
    return info, ora
