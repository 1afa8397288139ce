"""ctypes binding of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It never imports the CUDA binding and shares no
code with it; problems arrive as :class:`workloads.Problem` objects.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pgvimp_oracle.c")
_HDR = os.path.join(_HERE, "pgvimp_oracle.h")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

OK, EINVAL, ENOTPD, ENOMEM = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc -O2 into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = (not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC),
                                                                         os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("n", C.c_int), ("m", C.c_int), ("N", C.c_int), ("T", C.c_double),
        ("A", C.c_void_p), ("A_per_step", C.c_int),
        ("a", C.c_void_p), ("a_per_step", C.c_int),
        ("B", C.c_void_p), ("Qc", C.c_void_p),
        ("mu0", C.c_void_p), ("K0", C.c_void_p), ("muN", C.c_void_p), ("KN", C.c_void_p),
        ("cost_kind", C.c_int), ("psi_form", C.c_int), ("factor_set", C.c_int),
        ("eps", C.c_double), ("sigma_obs", C.c_double), ("temperature", C.c_double),
        ("sdf_nx", C.c_int), ("sdf_ny", C.c_int), ("sdf_nz", C.c_int),
        ("sdf_origin", C.c_double * 3), ("sdf_cell", C.c_double), ("sdf", C.c_void_p),
        ("arm_dof", C.c_int), ("dh", C.c_void_p), ("n_spheres", C.c_int),
        ("sphere_link", C.c_void_p), ("sphere_off", C.c_void_p), ("sphere_r", C.c_void_p),
        ("quad_c", C.c_void_p), ("quad_W", C.c_void_p),
        ("dyn_kind", C.c_int), ("dyn_params", C.c_double * 4),
        ("dyn_F", C.c_void_p), ("dyn_c", C.c_void_p),
    ]


class _Options(C.Structure):
    _fields_ = [
        ("rule", C.c_int), ("gh_p", C.c_int), ("beta_max", C.c_double), ("kl_eps", C.c_double),
        ("max_bisect", C.c_int), ("iters", C.c_int), ("slr_iters", C.c_int),
        ("init_kind", C.c_int), ("init_scale", C.c_double), ("replay_beta", C.c_void_p),
        ("temperature_high", C.c_double), ("switch_iter", C.c_int),
        ("update", C.c_int), ("trials_out", C.c_void_p), ("trials_cap", C.c_int), ("trials_n", C.c_void_p),
    ]


class _IterLog(C.Structure):
    _fields_ = [
        ("beta", C.c_double), ("kl", C.c_double), ("kl_margin", C.c_double),
        ("prior_cost", C.c_double), ("collision_cost", C.c_double), ("entropy", C.c_double),
        ("trials", C.c_int), ("accepted", C.c_int),
        ("beta_own", C.c_double), ("pd_margin", C.c_double), ("replayed", C.c_int), ("pad", C.c_int),
    ]


class _TrialRec(C.Structure):
    _fields_ = [
        ("iter", C.c_int), ("pd", C.c_int), ("feasible", C.c_int), ("pad", C.c_int),
        ("beta", C.c_double), ("kl", C.c_double), ("rel_pivot", C.c_double),
    ]


UPDATE_PROX, UPDATE_NGD = 0, 1


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.ora_psi.restype = C.c_double
        _lib.ora_sdf.restype = C.c_double
    return _lib


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class _Marshal:
    """Keeps the numpy buffers alive for as long as the ctypes struct is used."""

    def __init__(self, pb, op=None):
        self.keep = []
        s = _Problem()
        s.n, s.m, s.N, s.T = pb.n, pb.m, pb.N, pb.T
        A = self._k(_f64(pb.A))
        s.A, s.A_per_step = _ptr(A), int(A.ndim == 3)
        if pb.a is not None:
            a = self._k(_f64(pb.a))
            s.a, s.a_per_step = _ptr(a), int(a.ndim == 2)
        s.B, s.Qc = _ptr(self._k(_f64(pb.B))), _ptr(self._k(_f64(pb.Qc)))
        s.mu0, s.K0 = _ptr(self._k(_f64(pb.mu0))), _ptr(self._k(_f64(pb.K0)))
        s.muN, s.KN = _ptr(self._k(_f64(pb.muN))), _ptr(self._k(_f64(pb.KN)))
        s.cost_kind, s.psi_form, s.factor_set = pb.cost_kind, pb.psi_form, pb.factor_set
        s.eps, s.sigma_obs, s.temperature = pb.eps, pb.sigma_obs, pb.temperature
        if pb.sdf is not None:
            g = self._k(np.ascontiguousarray(pb.sdf, dtype=np.float32))
            if g.ndim == 2:
                s.sdf_ny, s.sdf_nx, s.sdf_nz = g.shape[0], g.shape[1], 1
            else:
                s.sdf_nz, s.sdf_ny, s.sdf_nx = g.shape
            s.sdf = _ptr(g)
        for d in range(3):
            s.sdf_origin[d] = pb.sdf_origin[d]
        s.sdf_cell = pb.sdf_cell
        if pb.dh is not None:
            s.arm_dof = pb.dh.shape[0]
            s.dh = _ptr(self._k(_f64(pb.dh)))
            s.n_spheres = len(pb.sphere_r)
            s.sphere_link = _ptr(self._k(np.ascontiguousarray(pb.sphere_link, dtype=np.int32)))
            s.sphere_off = _ptr(self._k(_f64(pb.sphere_off)))
            s.sphere_r = _ptr(self._k(_f64(pb.sphere_r)))
        if pb.quad_c is not None:
            s.quad_c = _ptr(self._k(_f64(pb.quad_c)))
            s.quad_W = _ptr(self._k(_f64(pb.quad_W)))
        s.dyn_kind = pb.dyn_kind
        for d in range(4):
            s.dyn_params[d] = pb.dyn_params[d]
        if pb.dyn_F is not None:
            s.dyn_F = _ptr(self._k(_f64(pb.dyn_F)))
        if pb.dyn_c is not None:
            s.dyn_c = _ptr(self._k(_f64(pb.dyn_c)))
        self.pb = s
        self.op = None
        if op is not None:
            o = _Options()
            o.rule, o.gh_p, o.beta_max, o.kl_eps = op.rule, op.gh_p, op.beta_max, op.kl_eps
            o.max_bisect, o.iters, o.slr_iters = op.max_bisect, op.iters, op.slr_iters
            o.init_kind, o.init_scale = op.init_kind, op.init_scale
            o.temperature_high = getattr(op, "temperature_high", 0.0)
            o.switch_iter = getattr(op, "switch_iter", 0)
            o.update = getattr(op, "update", UPDATE_PROX)
            if op.replay_beta is not None:
                o.replay_beta = _ptr(self._k(_f64(op.replay_beta)))
            # every trial of the own step-size search is recorded
            total = max(op.iters, 1) * max(getattr(op, "slr_iters", 0), 1)
            self.trial_recs = (_TrialRec * (total * (op.max_bisect + 1)))()
            self.trial_n = C.c_int(0)
            o.trials_out = C.cast(self.trial_recs, C.c_void_p)
            o.trials_cap = len(self.trial_recs)
            o.trials_n = C.cast(C.pointer(self.trial_n), C.c_void_p)
            self.op = o

    def trials(self):
        return [dict(iter=t.iter, pd=bool(t.pd), feasible=bool(t.feasible), beta=t.beta, kl=t.kl,
                     rel_pivot=t.rel_pivot) for t in self.trial_recs[:self.trial_n.value]]

    def _k(self, a):
        self.keep.append(a)
        return a


def _check(rc, what):
    if rc != OK:
        raise OracleError(rc, what)


class OracleError(RuntimeError):
    def __init__(self, rc, what):
        super().__init__(f"oracle {what} failed with status {rc}")
        self.rc = rc


# ----------------------------------------------------------------- dense / rules

def expm(M):
    M = _f64(M)
    d = M.shape[0]
    E = np.zeros_like(M)
    _check(lib().ora_expm(d, _ptr(M), _ptr(E)), "expm")
    return E


def gh_rule(p):
    x, w = np.zeros(p), np.zeros(p)
    _check(lib().ora_gh_rule(p, _ptr(x), _ptr(w)), "gh_rule")
    return x, w


def rule(n, kind, p):
    P = lib().ora_rule_size(n, kind, p)
    xi, W = np.zeros((P, n)), np.zeros(P)
    _check(lib().ora_rule(n, kind, p, _ptr(xi), _ptr(W)), "rule")
    return xi, W


# ---------------------------------------------------------------------- prior

@dataclass
class Prior:
    Kd: np.ndarray
    Ko: np.ndarray
    b: np.ndarray
    Phi: np.ndarray
    Q: np.ndarray
    u: np.ndarray
    mubar: np.ndarray


def prior(pb, A_ltv=None, a_ltv=None) -> Prior:
    m = _Marshal(pb)
    n, N = pb.n, pb.N
    Kd, Ko, b = np.zeros((N + 1, n, n)), np.zeros((N, n, n)), np.zeros((N + 1, n))
    Phi, Q, u = np.zeros((N, n, n)), np.zeros((N, n, n)), np.zeros((N, n))
    Al = None if A_ltv is None else _f64(A_ltv)
    al = None if a_ltv is None else _f64(a_ltv)
    _check(lib().ora_prior(C.byref(m.pb), _ptr(Al), _ptr(al), _ptr(Kd), _ptr(Ko), _ptr(b),
                           _ptr(Phi), _ptr(Q), _ptr(u)), "prior")
    mubar = np.zeros((N + 1, n))
    _check(lib().ora_prior_mean(C.byref(m.pb), _ptr(Kd), _ptr(Ko), _ptr(b), _ptr(mubar)), "prior_mean")
    return Prior(Kd, Ko, b, Phi, Q, u, mubar)


def init_mean(pb):
    m = _Marshal(pb)
    mu = np.zeros((pb.N + 1, pb.n))
    lib().ora_init_mean(C.byref(m.pb), _ptr(mu))
    return mu


# ------------------------------------------------------------------ marginals

def marginals(Ld, Lo):
    """GBP marginals of a block-tridiagonal precision: (Sd, So, logdet)."""
    Ld, Lo = _f64(Ld), _f64(Lo)
    N1, n = Ld.shape[0], Ld.shape[1]
    Sd, So = np.zeros_like(Ld), np.zeros((max(N1 - 1, 0), n, n))
    ld = C.c_double(0.0)
    _check(lib().ora_marginals(n, N1 - 1, _ptr(Ld), _ptr(Lo), _ptr(Sd), _ptr(So), C.byref(ld)), "marginals")
    return Sd, So, ld.value


def marginals_pivot(Ld, Lo):
    """(status, smallest relative pivot) of the forward elimination of a
    block-tridiagonal precision (status ENOTPD: not positive definite)."""
    Ld, Lo = _f64(Ld), _f64(Lo)
    N1, n = Ld.shape[0], Ld.shape[1]
    Sd, So = np.zeros_like(Ld), np.zeros((max(N1 - 1, 0), n, n))
    ld, piv = C.c_double(0.0), C.c_double(0.0)
    rc = lib().ora_marginals_pivot(n, N1 - 1, _ptr(Ld), _ptr(Lo), _ptr(Sd), _ptr(So), C.byref(ld), C.byref(piv))
    return rc, piv.value


def block_solve(Md, Mo, r):
    Md, Mo, r = _f64(Md), _f64(Mo), _f64(r)
    x = np.zeros_like(r)
    _check(lib().ora_block_solve(Md.shape[1], Md.shape[0] - 1, _ptr(Md), _ptr(Mo), _ptr(r), _ptr(x)),
           "block_solve")
    return x


# -------------------------------------------------------------- cost / moments

def sdf(pb, pos):
    m = _Marshal(pb)
    p = _f64(np.resize(np.asarray(pos, dtype=float), 3))
    return lib().ora_sdf(C.byref(m.pb), _ptr(p))


def arm_fk(pb, q):
    m = _Marshal(pb)
    q = _f64(q)
    c = np.zeros((len(pb.sphere_r), 3))
    _check(lib().ora_arm_fk(C.byref(m.pb), _ptr(q), _ptr(c)), "arm_fk")
    return c


def psi(pb, i, x):
    m = _Marshal(pb)
    x = _f64(x)
    return lib().ora_psi(C.byref(m.pb), i, _ptr(x))


def quad_moments(pb, op, i, mu_i, Sig_ii):
    m = _Marshal(pb, op)
    mu_i, Sig_ii = _f64(mu_i), _f64(Sig_ii)
    n = pb.n
    S0 = C.c_double(0.0)
    S1, S2 = np.zeros(n), np.zeros((n, n))
    _check(lib().ora_quad_moments(C.byref(m.pb), C.byref(m.op), i, _ptr(mu_i), _ptr(Sig_ii),
                                  C.byref(S0), _ptr(S1), _ptr(S2)), "quad_moments")
    return S0.value, S1, S2


def gradients(Sig_ii, S0, S1, S2):
    Sig_ii, S1, S2 = _f64(Sig_ii), _f64(S1), _f64(S2)
    n = Sig_ii.shape[0]
    g, G = np.zeros(n), np.zeros((n, n))
    _check(lib().ora_gradients(n, _ptr(Sig_ii), C.c_double(S0), _ptr(S1), _ptr(S2), _ptr(g), _ptr(G)),
           "gradients")
    return g, G


# ---------------------------------------------------------------- update / plan

@dataclass
class State:
    mu: np.ndarray
    Ld: np.ndarray
    Lo: np.ndarray
    Sd: np.ndarray
    So: np.ndarray
    logs: list
    slr_norms: Optional[np.ndarray] = None
    trials: Optional[list] = None     # every trial of the own step-size searches


def _logs_to_list(arr):
    return [dict(beta=l.beta, kl=l.kl, kl_margin=l.kl_margin, prior_cost=l.prior_cost,
                 collision_cost=l.collision_cost, entropy=l.entropy, trials=l.trials,
                 accepted=l.accepted, beta_own=l.beta_own, pd_margin=l.pd_margin,
                 replayed=bool(l.replayed)) for l in arr]


def trial(pb, beta, pr: Prior, mu, Ld, Lo, logdet_k, g, G, update: int = UPDATE_PROX):
    """One trial step (Thm 1, or the natural-gradient step with update=1)."""
    m = _Marshal(pb)
    n, N = pb.n, pb.N
    mu, Ld, Lo, g, G = _f64(mu), _f64(Ld), _f64(Lo), _f64(g), _f64(G)
    mun, Ldn, Lon = np.zeros_like(mu), np.zeros_like(Ld), np.zeros_like(Lo)
    Sdn, Son = np.zeros_like(Ld), np.zeros_like(Lo)
    ld, kl, piv = C.c_double(0.0), C.c_double(0.0), C.c_double(0.0)
    rc = lib().ora_trial_ex(C.byref(m.pb), update, C.c_double(beta), _ptr(pr.Kd), _ptr(pr.Ko), _ptr(pr.b),
                            _ptr(mu), _ptr(Ld), _ptr(Lo), C.c_double(logdet_k), _ptr(g), _ptr(G), _ptr(mun),
                            _ptr(Ldn), _ptr(Lon), _ptr(Sdn), _ptr(Son), C.byref(ld), C.byref(kl), C.byref(piv))
    return rc, dict(mu=mun, Ld=Ldn, Lo=Lon, Sd=Sdn, So=Son, logdet=ld.value, kl=kl.value, rel_pivot=piv.value)


def plan(pb, op, state: Optional[State] = None) -> State:
    """Alg. 1 for op.iters iterations from the default initial iterate (or
    from `state`, warm)."""
    m = _Marshal(pb, op)
    n, N = pb.n, pb.N
    if state is None:
        mu, Ld, Lo = np.zeros((N + 1, n)), np.zeros((N + 1, n, n)), np.zeros((N, n, n))
        init = 1
    else:
        mu, Ld, Lo = _f64(state.mu).copy(), _f64(state.Ld).copy(), _f64(state.Lo).copy()
        init = 0
    Sd, So = np.zeros((N + 1, n, n)), np.zeros((N, n, n))
    logs = (_IterLog * max(op.iters, 1))()
    _check(lib().ora_plan(C.byref(m.pb), C.byref(m.op), init, _ptr(mu), _ptr(Ld), _ptr(Lo), _ptr(Sd),
                          _ptr(So), logs), "plan")
    return State(mu, Ld, Lo, Sd, So, _logs_to_list(logs[:op.iters]), trials=m.trials())


def drift(pb, x):
    m = _Marshal(pb)
    x = _f64(x)
    f = np.zeros(pb.n)
    _check(lib().ora_drift(C.byref(m.pb), _ptr(x), _ptr(f)), "drift")
    return f


def slr(pb, op, xbar, Sbar):
    m = _Marshal(pb, op)
    n, N = pb.n, pb.N
    xbar, Sbar = _f64(xbar), _f64(Sbar)
    A, a = np.zeros((N, n, n)), np.zeros((N, n))
    _check(lib().ora_slr(C.byref(m.pb), C.byref(m.op), _ptr(xbar), _ptr(Sbar), _ptr(A), _ptr(a)), "slr")
    return A, a


def plan_slr(pb, op) -> State:
    """Alg. 2: op.slr_iters linearisations, each followed by op.iters
    proximal iterations."""
    m = _Marshal(pb, op)
    n, N = pb.n, pb.N
    mu, Ld, Lo = np.zeros((N + 1, n)), np.zeros((N + 1, n, n)), np.zeros((N, n, n))
    Sd, So = np.zeros((N + 1, n, n)), np.zeros((N, n, n))
    total = max(op.iters * op.slr_iters, 1)
    logs = (_IterLog * total)()
    norms = np.zeros(max(op.slr_iters, 1))
    _check(lib().ora_plan_slr(C.byref(m.pb), C.byref(m.op), _ptr(mu), _ptr(Ld), _ptr(Lo), _ptr(Sd),
                              _ptr(So), logs, _ptr(norms)), "plan_slr")
    return State(mu, Ld, Lo, Sd, So, _logs_to_list(logs[:op.iters * op.slr_iters]), norms[:op.slr_iters],
                 trials=m.trials())


def solve(pb, op) -> State:
    """Alg. 2 when the problem has a nonlinear drift, else Alg. 1."""
    if pb.dyn_kind != 0 and op.slr_iters > 0:
        return plan_slr(pb, op)
    return plan(pb, op)
