"""Seeded synthetic inputs for the P-GVIMP planner (arXiv 2411.03416).

This module is shared by the oracle, the CUDA binding's tests and the
benchmark.  It holds no arithmetic of the method itself: it only draws maps,
robot models, start/goal Gaussians and options, and evaluates the exact signed
distance of the drawn shapes on the grid nodes (the SDF is an input of the
method, Sec. 4.1).

The paper's own maps, WAM/PR2 kinematics and seeds are not available; these
generators stand in for its workloads with the paper's shapes (dense horizons,
2-D point robot, 7-DOF arm, planar quadrotor; Sec. 7).  Seeds follow
``seed = 1_000_000 * config + request_index`` with numpy's PCG64.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

import numpy as np

COST_NONE, COST_POINT2D, COST_POINT3D, COST_ARM, COST_QUADRATIC = 0, 1, 2, 3, 4
DYN_LINEAR, DYN_PLANAR_QUAD, DYN_AFFINE_TEST = 0, 1, 2
RULE_GH, RULE_DEG3, RULE_SMOLYAK = 0, 1, 2


@dataclass
class Problem:
    """One planning problem.  Matrices are float64, row-major; the state is
    x = [q; qdot] (n = 2*nq)."""
    n: int
    m: int
    N: int
    T: float
    A: np.ndarray                      # (n,n) LTI or (N,n,n) LTV
    B: np.ndarray                      # (n,m)
    Qc: np.ndarray                     # (m,m)
    mu0: np.ndarray
    K0: np.ndarray
    muN: np.ndarray
    KN: np.ndarray
    a: Optional[np.ndarray] = None     # None, (n,) or (N,n)
    cost_kind: int = COST_NONE
    psi_form: int = 0                  # 0: sigma_obs*h^2, 1: h^2/sigma_obs^2
    factor_set: int = 0                # 0: states 0..N, 1: states 1..N-1
    eps: float = 0.0
    sigma_obs: float = 1.0
    temperature: float = 1.0
    sdf: Optional[np.ndarray] = None   # float32 (ny,nx) or (nz,ny,nx)
    sdf_origin: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    sdf_cell: float = 1.0
    dh: Optional[np.ndarray] = None            # (dof,4): a, alpha, d, theta0
    sphere_link: Optional[np.ndarray] = None   # (S,) int32
    sphere_off: Optional[np.ndarray] = None    # (S,3)
    sphere_r: Optional[np.ndarray] = None      # (S,)
    quad_c: Optional[np.ndarray] = None        # (N+1,n)
    quad_W: Optional[np.ndarray] = None        # (N+1,n,n)
    dyn_kind: int = DYN_LINEAR
    dyn_params: Tuple[float, float, float, float] = (0.0, 0.0, 0.0, 0.0)
    dyn_F: Optional[np.ndarray] = None
    dyn_c: Optional[np.ndarray] = None
    name: str = ""

    @property
    def nq(self) -> int:
        return self.n // 2


@dataclass
class Options:
    rule: int = RULE_GH
    gh_p: int = 3
    beta_max: float = 0.5
    kl_eps: float = float("inf")
    max_bisect: int = 10
    iters: int = 20
    slr_iters: int = 0
    init_kind: int = 0
    init_scale: float = 1.0
    replay_beta: Optional[np.ndarray] = None
    plan_threads: int = 0   # execution form of the CUDA path (0: thread per plan; 32..256: block per plan)
    temperature_high: float = 0.0   # two-phase temperature: T-hat from switch_iter on (0: one phase)
    switch_iter: int = 0
    update: int = 0         # 0: KL-proximal step (Thm 1); 1: natural-gradient step (Sec. 3.1(d))


def rng_for(config: int, request: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(1_000_000 * config + request))


# ----------------------------------------------------------------- models

def double_integrator(nq: int):
    """A = [[0, I],[0, 0]], B = [0; I] (Sec. 7.1)."""
    n = 2 * nq
    A = np.zeros((n, n))
    A[:nq, nq:] = np.eye(nq)
    B = np.zeros((n, nq))
    B[nq:, :] = np.eye(nq)
    return A, B


def point_problem(nq: int, N: int, T: float, start, goal, Qc: float, cov: float) -> Problem:
    A, B = double_integrator(nq)
    n = 2 * nq
    mu0 = np.zeros(n)
    mu0[:nq] = start
    muN = np.zeros(n)
    muN[:nq] = goal
    return Problem(n=n, m=nq, N=N, T=float(T), A=A, B=B, Qc=Qc * np.eye(nq), mu0=mu0,
                   K0=cov * np.eye(n), muN=muN, KN=cov * np.eye(n))


# ------------------------------------------------------------------- maps

def _disk_sdf(px, py, cx, cy, r):
    return np.hypot(px - cx, py - cy) - r


def _box_sdf(P, c, h):
    """Exact signed distance of an axis-aligned box (any dimension)."""
    q = np.abs(P - c) - h
    outside = np.linalg.norm(np.maximum(q, 0.0), axis=-1)
    inside = np.minimum(np.max(q, axis=-1), 0.0)
    return outside + inside


def sdf_grid_2d(nx, ny, origin, cell, disks=(), boxes=()):
    xs = origin[0] + cell * np.arange(nx)
    ys = origin[1] + cell * np.arange(ny)
    X, Y = np.meshgrid(xs, ys)                     # (ny, nx)
    d = np.full((ny, nx), np.inf)
    for (cx, cy, r) in disks:
        d = np.minimum(d, _disk_sdf(X, Y, cx, cy, r))
    P = np.stack([X, Y], axis=-1)
    for (c, h) in boxes:
        d = np.minimum(d, _box_sdf(P, np.asarray(c), np.asarray(h)))
    if not np.isfinite(d).all():
        d = np.full((ny, nx), 100.0)
    return d.astype(np.float32)


def sdf_grid_3d(n3, origin, cell, boxes=()):
    nx, ny, nz = n3
    xs = origin[0] + cell * np.arange(nx)
    ys = origin[1] + cell * np.arange(ny)
    zs = origin[2] + cell * np.arange(nz)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")   # (nz, ny, nx)
    P = np.stack([X, Y, Z], axis=-1)
    d = np.full((nz, ny, nx), np.inf)
    for (c, h) in boxes:
        d = np.minimum(d, _box_sdf(P, np.asarray(c), np.asarray(h)))
    if not np.isfinite(d).all():
        d = np.full((nz, ny, nx), 100.0)
    return d.astype(np.float32)


def _shape_clear(kind, params, pts, margin):
    for p in pts:
        p = np.asarray(p, dtype=float)
        if kind == "disk":
            cx, cy, r = params
            if np.hypot(p[0] - cx, p[1] - cy) - r < margin:
                return False
        else:
            c, h = params
            if _box_sdf(p[None, :], np.asarray(c), np.asarray(h))[0] < margin:
                return False
    return True


def random_shapes_2d(rng, count, box_frac, region, rad, half, keep_clear, margin):
    """Disks with radius U(rad) and axis-aligned boxes with half-sides U(half),
    centres U(region); a shape is redrawn if it comes within `margin` of any
    point in keep_clear."""
    disks, boxes = [], []
    (x0, x1), (y0, y1) = region
    while len(disks) + len(boxes) < count:
        is_box = rng.random() < box_frac
        c = (rng.uniform(x0, x1), rng.uniform(y0, y1))
        if is_box:
            h = (rng.uniform(*half), rng.uniform(*half))
            if _shape_clear("box", (c, h), keep_clear, margin):
                boxes.append((c, h))
        else:
            r = rng.uniform(*rad)
            if _shape_clear("disk", (c[0], c[1], r), keep_clear, margin):
                disks.append((c[0], c[1], r))
    return disks, boxes


# ---------------------------------------------------------------- configs

def c1_point2d(request: int = 0, N: int = 50, iters: int = 20, config: int = 1) -> Tuple[Problem, Options]:
    """Small plain case: 2-D point robot, double integrator, N=50 over T=5 s,
    Qc=0.8 I2, start (0,0,0,0), goal (17,14,0,0), covariance 0.01 I4;
    180x180 SDF at 0.1 m from 6 disks r~U(0.8,2.0); eps=0.5, sigma_obs=0.5;
    GH 3 points per dim; 20 iterations, beta_max 0.5."""
    rng = rng_for(config, request)
    start, goal, eps = (0.0, 0.0), (17.0, 14.0), 0.5
    pb = point_problem(2, N, 5.0, start, goal, 0.8, 0.01)
    disks, boxes = random_shapes_2d(rng, 6, 0.0, ((1.0, 16.0), (1.0, 13.0)), (0.8, 2.0), (0.5, 1.5),
                                    [start, goal], eps + 0.5)
    origin = (-0.5, -0.5, 0.0)
    pb.sdf = sdf_grid_2d(180, 180, origin, 0.1, disks, boxes)
    pb.sdf_origin, pb.sdf_cell = origin, 0.1
    pb.cost_kind, pb.eps, pb.sigma_obs = COST_POINT2D, eps, 0.5
    pb.name = f"point2d_N{N}"
    op = Options(rule=RULE_GH, gh_p=3, beta_max=0.5, kl_eps=0.1 * (N + 1), max_bisect=10, iters=iters)
    return pb, op


def c2_point2d_dense(request: int = 0, N: int = 750, iters: int = 30, config: int = 2) -> Tuple[Problem, Options]:
    """Dense horizon: the 2-D point robot with N=750, a 500x500 SDF at 0.05 m
    from 25 disks and axis-aligned boxes (half/half), GH 5 points per dim,
    30 iterations."""
    rng = rng_for(config, request)
    start, goal, eps = (0.0, 0.0), (17.0, 14.0), 0.5
    pb = point_problem(2, N, 5.0, start, goal, 0.8, 0.01)
    disks, boxes = random_shapes_2d(rng, 25, 0.5, ((1.0, 16.0), (1.0, 13.0)), (0.8, 2.0), (0.5, 1.5),
                                    [start, goal], eps + 0.5)
    origin = (-4.0, -4.0, 0.0)
    pb.sdf = sdf_grid_2d(500, 500, origin, 0.05, disks, boxes)
    pb.sdf_origin, pb.sdf_cell = origin, 0.05
    pb.cost_kind, pb.eps, pb.sigma_obs = COST_POINT2D, eps, 0.5
    pb.name = f"point2d_dense_N{N}"
    op = Options(rule=RULE_GH, gh_p=5, beta_max=0.5, kl_eps=0.1 * (N + 1), max_bisect=10, iters=iters)
    return pb, op


# A synthetic 7-revolute arm (standard DH rows: a, alpha, d, theta0).  Link
# lengths and twists are this project's own choice (the WAM/PR2 parameters are
# not available); the chain reaches about 1.26 m.
ARM_DH = np.array([
    [0.0, -np.pi / 2, 0.34, 0.0],
    [0.0, np.pi / 2, 0.0, 0.0],
    [0.0, np.pi / 2, 0.40, 0.0],
    [0.0, -np.pi / 2, 0.0, 0.0],
    [0.0, -np.pi / 2, 0.39, 0.0],
    [0.0, np.pi / 2, 0.0, 0.0],
    [0.0, 0.0, 0.13, 0.0],
])
# Spheres per link carrying length (links 0, 2, 4, 6): 5 + 6 + 6 + 3 = 20, at
# evenly spaced fractions of the segment from the joint to the next origin.
_ARM_SPHERES = [(0, 5), (2, 6), (4, 6), (6, 3)]


def arm_model(rng):
    links, offs = [], []
    for (j, count) in _ARM_SPHERES:
        d = ARM_DH[j, 2]
        for k in range(count):
            t = (k + 0.5) / count
            links.append(j)
            offs.append((0.0, 0.0, t * d))
    radii = rng.uniform(0.05, 0.12, size=len(links))
    return ARM_DH.copy(), np.array(links, dtype=np.int32), np.array(offs, dtype=float), radii


def _fk_points(dh, links, offs, q):
    """Sphere centres of the arm at joint vector q (input preparation only:
    used to keep the drawn boxes clear of the start and goal poses)."""
    T = np.eye(4)
    out = np.zeros((len(links), 3))
    for j in range(dh.shape[0]):
        a, al, d, th0 = dh[j]
        th = q[j] + th0
        c, s = np.cos(th), np.sin(th)
        Rz = np.array([[c, -s, 0, 0], [s, c, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1.0]])
        R = T @ Rz
        for k in np.nonzero(links == j)[0]:
            out[k] = (R @ np.append(offs[k], 1.0))[:3]
        ca, sa = np.cos(al), np.sin(al)
        Tz = np.eye(4); Tz[2, 3] = d
        Tx = np.eye(4); Tx[0, 3] = a
        Rx = np.array([[1, 0, 0, 0], [0, ca, -sa, 0], [0, sa, ca, 0], [0, 0, 0, 1.0]])
        T = R @ Tz @ Tx @ Rx
    return out


def c3_arm(request: int = 0, N: int = 200, iters: int = 25, config: int = 3) -> Tuple[Problem, Options]:
    """7-DOF serial arm in 3-D: double integrator per joint (n=14), N=200,
    T=2 s, Qc=0.8 I7; 20 spheres r~U(0.05,0.12); 128^3 SDF at 0.02 m from 12
    boxes (half-sides U(0.05,0.25)) kept clear of the start and goal poses;
    sigma_obs=20, eps_sdf=0.1; degree-3 rule; 25 iterations."""
    rng = rng_for(config, request)
    dh, links, offs, radii = arm_model(rng)
    q0 = rng.uniform(-1.0, 1.0, size=7)
    qN = rng.uniform(-1.0, 1.0, size=7)
    pb = point_problem(7, N, 2.0, q0, qN, 0.8, 0.01)
    origin = (-1.28, -1.28, -0.3)
    pose_pts = np.concatenate([_fk_points(dh, links, offs, q0), _fk_points(dh, links, offs, qN)])
    pose_r = np.concatenate([radii, radii])
    boxes = []
    while len(boxes) < 12:
        c = np.array([rng.uniform(-1.0, 1.0), rng.uniform(-1.0, 1.0), rng.uniform(0.0, 1.4)])
        h = rng.uniform(0.05, 0.25, size=3)
        dist = _box_sdf(pose_pts, c, h)
        if np.all(dist > pose_r + 0.05):
            boxes.append((c, h))
    pb.sdf = sdf_grid_3d((128, 128, 128), origin, 0.02, boxes)
    pb.sdf_origin, pb.sdf_cell = origin, 0.02
    pb.cost_kind, pb.eps, pb.sigma_obs = COST_ARM, 0.1, 20.0
    pb.dh, pb.sphere_link, pb.sphere_off, pb.sphere_r = dh, links, offs, radii
    pb.name = f"arm7_N{N}"
    op = Options(rule=RULE_DEG3, gh_p=3, beta_max=0.5, kl_eps=0.1 * (N + 1), max_bisect=10, iters=iters)
    return pb, op


def point3d(request: int = 0, N: int = 50, iters: int = 20, config: int = 6) -> Tuple[Problem, Options]:
    """3-D point robot (the middle column of the paper's point-robot tables):
    double integrator in 3-D (n=6), N=50 over T=5 s, Qc=0.8 I3, start
    (0,0,0), goal (9,8,4), covariance 0.01 I6; 110x100x60 SDF at 0.1 m from
    10 boxes (half-sides U(0.3,1.0)) kept clear of start and goal; eps=0.5,
    sigma_obs=0.5; GH 3 points per dim (27 distinct points on the three
    position coordinates); 20 iterations."""
    rng = rng_for(config, request)
    start, goal, eps = (0.0, 0.0, 0.0), (9.0, 8.0, 4.0), 0.5
    pb = point_problem(3, N, 5.0, start, goal, 0.8, 0.01)
    ends = np.array([start, goal])
    boxes = []
    while len(boxes) < 10:
        c = np.array([rng.uniform(1.0, 9.0), rng.uniform(1.0, 8.0), rng.uniform(0.5, 4.5)])
        h = rng.uniform(0.3, 1.0, size=3)
        if np.all(_box_sdf(ends, c, h) > eps + 0.5):
            boxes.append((c, h))
    origin = (-1.0, -1.0, -1.0)
    pb.sdf = sdf_grid_3d((110, 100, 60), origin, 0.1, boxes)
    pb.sdf_origin, pb.sdf_cell = origin, 0.1
    pb.cost_kind, pb.eps, pb.sigma_obs = COST_POINT3D, eps, 0.5
    pb.name = f"point3d_N{N}"
    op = Options(rule=RULE_GH, gh_p=3, beta_max=0.5, kl_eps=0.1 * (N + 1), max_bisect=10, iters=iters)
    return pb, op


def c4_quadrotor(request: int = 0, N: int = 300, iters: int = 15, slr_iters: int = 10,
                 config: int = 4) -> Tuple[Problem, Options]:
    """Planar quadrotor (eq. planar_quad; state (x, z, phi, vx, vz, phidot)),
    prior drift with u = 0, process noise 0.05 I6 (B = I6), N=300, T=5 s;
    400x400 SDF at 0.05 m from 15 disks r~U(0.8,2.0); eps=1.5,
    sigma_obs=6.0; GH 3 points per dim on all 6 dims; 10 SLR x 15 iterations."""
    rng = rng_for(config, request)
    start, goal, eps = (0.0, 0.0, 0.0), (16.0, 16.0, 0.0), 1.5
    n = 6
    mu0 = np.zeros(n); mu0[:3] = start
    muN = np.zeros(n); muN[:3] = goal
    pb = Problem(n=n, m=n, N=N, T=5.0, A=np.zeros((n, n)), B=np.eye(n), Qc=0.05 * np.eye(n),
                 mu0=mu0, K0=0.01 * np.eye(n), muN=muN, KN=0.01 * np.eye(n))
    disks, _ = random_shapes_2d(rng, 15, 0.0, ((1.0, 15.0), (1.0, 15.0)), (0.8, 2.0), (0.5, 1.5),
                                [start[:2], goal[:2]], eps + 0.5)
    origin = (-2.0, -2.0, 0.0)
    pb.sdf = sdf_grid_2d(400, 400, origin, 0.05, disks, ())
    pb.sdf_origin, pb.sdf_cell = origin, 0.05
    pb.cost_kind, pb.eps, pb.sigma_obs = COST_POINT2D, eps, 6.0
    pb.dyn_kind, pb.dyn_params = DYN_PLANAR_QUAD, (1.0, 0.25, 1.0, 9.81)
    pb.name = f"quadrotor_N{N}"
    op = Options(rule=RULE_GH, gh_p=3, beta_max=0.5, kl_eps=0.1 * (N + 1), max_bisect=10,
                 iters=iters, slr_iters=slr_iters)
    return pb, op


@dataclass
class Request:
    index: int
    arrival_s: float
    kind: str
    problem: Problem
    options: Options


def c5_mix(count: int = 512, rate_hz: float = 2000.0, config: int = 5) -> List[Request]:
    """Serving mix: `count` requests with Exp(1/rate) inter-arrival times;
    50% point robot (N ~ U{50..1000}), 30% quadrotor SLR (N ~ U{100..500}),
    20% 7-DOF arm (N ~ U{100..300}); each request has its own seeded map."""
    rng = rng_for(config, 0)
    gaps = rng.exponential(1.0 / rate_hz, size=count)
    arrivals = np.cumsum(gaps) - gaps[0]
    kinds = rng.choice(3, size=count, p=[0.5, 0.3, 0.2])
    out = []
    for r in range(count):
        k = int(kinds[r])
        if k == 0:
            N = int(rng.integers(50, 1001))
            pb, op = c1_point2d(request=r + 1, N=N, config=config)
            kind = "point2d"
        elif k == 1:
            N = int(rng.integers(100, 501))
            pb, op = c4_quadrotor(request=r + 1, N=N, config=config)
            kind = "quadrotor"
        else:
            N = int(rng.integers(100, 301))
            pb, op = c3_arm(request=r + 1, N=N, config=config)
            kind = "arm"
        out.append(Request(r, float(arrivals[r]), kind, pb, op))
    return out


def tiny_point2d(N: int = 12, request: int = 0, iters: int = 4, gh_p: int = 3) -> Tuple[Problem, Options]:
    """A small 2-D case for tests: the C1 map and robot with a short horizon."""
    pb, op = c1_point2d(request=request, N=N, iters=iters)
    op = replace(op, gh_p=gh_p, kl_eps=0.1 * (N + 1))
    pb.name = f"tiny_point2d_N{N}"
    return pb, op
