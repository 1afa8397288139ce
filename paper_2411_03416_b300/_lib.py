"""Thin ctypes binding of libpgvimp.so (the C ABI in include/pgvimp.h).

Argument marshalling only: every step of the planner runs in the library's
CUDA kernels.  PyTorch provides device memory (the batch arena) and streams.
There is no CPU fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("PGVIMP_LIB") or os.path.join(_HERE, "_build", "libpgvimp.so")

OK, EINVAL, ENOMEM, ENOTPD, ECUDA, ETIMEOUT, EBUSY, ENOTFINITE, ENOTREADY = range(9)
PREC_PLAIN_FP64, PREC_MIXED, PREC_MIXED_DF = 0, 1, 2
UPDATE_PROX, UPDATE_NGD = 0, 1
PHASE_PRIOR, PHASE_MARGINALS, PHASE_QUAD, PHASE_TRIAL, PHASE_SLR = range(5)
(BUF_MU, BUF_LD, BUF_LO, BUF_SD, BUF_SO, BUF_KD, BUF_KO, BUF_B, BUF_G1, BUF_G2, BUF_TMU, BUF_TSD, BUF_TSO,
 BUF_ALTV, BUF_ALTVA, BUF_SCAL) = range(16)
# slots of the per-plan scalar buffer
S_LOGDET, S_T_LOGDET, S_T_KL, S_T_PD, S_COLL, S_K, S_KIN, S_J, S_INIT, S_CUR, S_PRIOR, S_T_PRIOR, S_STATUS, \
    S_T_DELTA, S_T_TRACE = range(15)

EXPORTED = [
    "pgvimp_batch_arena_bytes", "pgvimp_batch_create", "pgvimp_batch_upload", "pgvimp_batch_reset",
    "pgvimp_batch_run", "pgvimp_batch_download", "pgvimp_batch_download_results", "pgvimp_batch_result",
    "pgvimp_batch_io_bytes",
    "pgvimp_batch_destroy", "pgvimp_batch_phase", "pgvimp_batch_read", "pgvimp_batch_write",
    "pgvimp_create", "pgvimp_step", "pgvimp_plan", "pgvimp_get", "pgvimp_destroy", "pgvimp_last_error",
    "pgvimp_version", "pgvimp_abi_sizes", "pgvimp_marginals_noalloc",
    "pgvimp_server_create", "pgvimp_submit", "pgvimp_poll", "pgvimp_server_stats", "pgvimp_server_destroy",
]


class PgvimpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"pgvimp status {status}: {msg}")
        self.status = status


class Problem(C.Structure):
    _fields_ = [
        ("n", C.c_int), ("m", C.c_int), ("N", C.c_int), ("T", C.c_double),
        ("A", C.c_void_p), ("A_per_step", C.c_int), ("a", C.c_void_p), ("a_per_step", C.c_int),
        ("B", C.c_void_p), ("Qc", C.c_void_p), ("mu0", C.c_void_p), ("K0", C.c_void_p),
        ("muN", C.c_void_p), ("KN", C.c_void_p),
        ("cost_kind", C.c_int), ("psi_form", C.c_int), ("factor_set", C.c_int),
        ("eps", C.c_double), ("sigma_obs", C.c_double), ("temperature", C.c_double),
        ("sdf_nx", C.c_int), ("sdf_ny", C.c_int), ("sdf_nz", C.c_int),
        ("sdf_origin", C.c_double * 3), ("sdf_cell", C.c_double), ("sdf", C.c_void_p),
        ("arm_dof", C.c_int), ("arm_dh", C.c_void_p), ("n_spheres", C.c_int),
        ("sphere_link", C.c_void_p), ("sphere_off", C.c_void_p), ("sphere_r", C.c_void_p),
        ("dyn_kind", C.c_int), ("dyn_params", C.c_double * 4),
    ]


class Options(C.Structure):
    _fields_ = [
        ("rule", C.c_int), ("gh_p", C.c_int), ("beta_max", C.c_double), ("kl_eps", C.c_double),
        ("max_bisect", C.c_int), ("iters", C.c_int), ("slr_iters", C.c_int), ("init_kind", C.c_int),
        ("init_scale", C.c_double), ("plan_threads", C.c_int), ("temperature_high", C.c_double),
        ("switch_iter", C.c_int), ("update", C.c_int),
    ]


class StepInfo(C.Structure):
    _fields_ = [
        ("beta", C.c_double), ("kl", C.c_double), ("kl_margin", C.c_double),
        ("prior_cost", C.c_double), ("collision_cost", C.c_double), ("entropy", C.c_double),
        ("trials", C.c_int), ("iter", C.c_int),
    ]


class ServerConfig(C.Structure):
    _fields_ = [
        ("hbm_budget_bytes", C.c_size_t), ("host_staging_bytes", C.c_size_t), ("precision", C.c_int),
        ("plan_threads", C.c_int), ("max_inflight", C.c_int), ("max_batch", C.c_int),
        ("batch_window_ms", C.c_double),
    ]


class RequestInfo(C.Structure):
    _fields_ = [
        ("status", C.c_int), ("n", C.c_int), ("N", C.c_int), ("n_logs", C.c_int), ("batch_size", C.c_int),
        ("submit_ms", C.c_double), ("start_ms", C.c_double), ("done_ms", C.c_double), ("last", StepInfo),
    ]


class ServerStats(C.Structure):
    _fields_ = [
        ("queued", C.c_int), ("inflight", C.c_int), ("batches", C.c_uint64), ("plans", C.c_uint64),
        ("dev_used", C.c_size_t), ("host_used", C.c_size_t), ("now_ms", C.c_double),
        ("host_launch_ms", C.c_double), ("host_collect_ms", C.c_double),
        ("graph_launches", C.c_uint64), ("graph_instantiations", C.c_uint64),
    ]


_lib = None


def lib():
    """Loads libpgvimp.so (building it first if it is missing and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        from . import build as _build
        _build.build()
    L = C.CDLL(LIB_PATH)
    for name in EXPORTED:
        getattr(L, name)  # raises AttributeError if a declared symbol is missing
    L.pgvimp_last_error.restype = C.c_char_p
    L.pgvimp_last_error.argtypes = [C.c_void_p]
    L.pgvimp_batch_create.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_size_t,
                                      C.POINTER(C.c_void_p)]
    L.pgvimp_batch_arena_bytes.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_size_t)]
    for nm in ("pgvimp_batch_upload", "pgvimp_batch_reset", "pgvimp_batch_download", "pgvimp_batch_download_results"):
        getattr(L, nm).argtypes = [C.c_void_p, C.c_void_p]
    L.pgvimp_batch_run.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
    L.pgvimp_batch_phase.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_void_p]
    L.pgvimp_batch_result.argtypes = [C.c_void_p, C.c_int] + [C.c_void_p] * 6 + [C.c_int, C.POINTER(C.c_int)]
    L.pgvimp_batch_io_bytes.argtypes = [C.c_void_p, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t),
                                        C.POINTER(C.c_size_t)]
    L.pgvimp_batch_destroy.argtypes = [C.c_void_p]
    L.pgvimp_batch_read.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_size_t]
    L.pgvimp_batch_write.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_size_t]
    L.pgvimp_create.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]
    L.pgvimp_step.argtypes = [C.c_void_p, C.c_void_p]
    L.pgvimp_plan.argtypes = [C.c_void_p, C.c_int]
    L.pgvimp_get.argtypes = [C.c_void_p] + [C.c_void_p] * 4
    L.pgvimp_destroy.argtypes = [C.c_void_p]
    L.pgvimp_version.argtypes = [C.c_char_p, C.c_size_t]
    L.pgvimp_marginals_noalloc.argtypes = [C.c_int, C.c_int] + [C.c_void_p] * 6
    L.pgvimp_server_create.argtypes = [C.c_void_p, C.POINTER(C.c_void_p)]
    L.pgvimp_submit.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_uint64)]
    L.pgvimp_poll.argtypes = [C.c_void_p, C.c_uint64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    L.pgvimp_server_stats.argtypes = [C.c_void_p, C.c_void_p]
    L.pgvimp_server_destroy.argtypes = [C.c_void_p]
    _lib = L
    return L


def _check(st: int):
    if st != OK:
        raise PgvimpError(st, lib().pgvimp_last_error(None).decode(errors="replace"))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class _Keep:
    def __init__(self):
        self.refs = []

    def __call__(self, a):
        self.refs.append(a)
        return a


def marshal_problem(pb, keep: _Keep) -> Problem:
    """workloads.Problem -> pgvimp_problem (host pointers kept alive by `keep`)."""
    s = Problem()
    s.n, s.m, s.N, s.T = pb.n, pb.m, pb.N, pb.T
    A = keep(_f64(pb.A))
    s.A, s.A_per_step = _p(A), int(A.ndim == 3)
    if pb.a is not None:
        a = keep(_f64(pb.a))
        s.a, s.a_per_step = _p(a), int(a.ndim == 2)
    s.B, s.Qc = _p(keep(_f64(pb.B))), _p(keep(_f64(pb.Qc)))
    s.mu0, s.K0 = _p(keep(_f64(pb.mu0))), _p(keep(_f64(pb.K0)))
    s.muN, s.KN = _p(keep(_f64(pb.muN))), _p(keep(_f64(pb.KN)))
    s.cost_kind, s.psi_form, s.factor_set = pb.cost_kind, pb.psi_form, pb.factor_set
    s.eps, s.sigma_obs, s.temperature = pb.eps, pb.sigma_obs, pb.temperature
    if pb.sdf is not None:
        g = keep(np.ascontiguousarray(pb.sdf, dtype=np.float32))
        if g.ndim == 2:
            s.sdf_ny, s.sdf_nx, s.sdf_nz = g.shape[0], g.shape[1], 1
        else:
            s.sdf_nz, s.sdf_ny, s.sdf_nx = g.shape
        s.sdf = _p(g)
    for d in range(3):
        s.sdf_origin[d] = pb.sdf_origin[d]
    s.sdf_cell = pb.sdf_cell
    if pb.dh is not None:
        s.arm_dof = pb.dh.shape[0]
        s.arm_dh = _p(keep(_f64(pb.dh)))
        s.n_spheres = len(pb.sphere_r)
        s.sphere_link = _p(keep(np.ascontiguousarray(pb.sphere_link, dtype=np.int32)))
        s.sphere_off = _p(keep(_f64(pb.sphere_off)))
        s.sphere_r = _p(keep(_f64(pb.sphere_r)))
    s.dyn_kind = pb.dyn_kind
    for d in range(4):
        s.dyn_params[d] = pb.dyn_params[d]
    return s


def marshal_options(op) -> Options:
    o = Options()
    o.rule, o.gh_p, o.beta_max, o.kl_eps = op.rule, op.gh_p, op.beta_max, op.kl_eps
    o.max_bisect, o.iters, o.slr_iters = op.max_bisect, op.iters, op.slr_iters
    o.init_kind, o.init_scale = op.init_kind, op.init_scale
    o.plan_threads = getattr(op, "plan_threads", 0)
    o.temperature_high = getattr(op, "temperature_high", 0.0)
    o.switch_iter = getattr(op, "switch_iter", 0)
    o.update = getattr(op, "update", 0)
    return o


def _stream_handle(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


@dataclass
class PlanResult:
    mu: np.ndarray
    Sd: np.ndarray
    So: Optional[np.ndarray]
    Ld: Optional[np.ndarray]
    Lo: Optional[np.ndarray]
    logs: List[dict]


def _log_dicts(arr, k):
    return [dict(beta=l.beta, kl=l.kl, kl_margin=l.kl_margin, prior_cost=l.prior_cost,
                 collision_cost=l.collision_cost, entropy=l.entropy, trials=l.trials, iter=l.iter)
            for l in arr[:k]]


class Batch:
    """A device-resident batch of plans (pgvimp_batch_*).  The arena is a
    PyTorch CUDA tensor unless `torch_arena` is False."""

    def __init__(self, problems: Sequence, options: Sequence, precision: int = PREC_MIXED,
                 torch_arena: bool = True):
        L = lib()
        if len(problems) != len(options):
            raise ValueError("one options object per problem")
        self.problems = list(problems)
        keep = _Keep()
        cnt = len(problems)
        parr = (Problem * cnt)(*[marshal_problem(p, keep) for p in problems])
        oarr = (Options * cnt)(*[marshal_options(o) for o in options])
        self.precision = precision
        nbytes = C.c_size_t(0)
        _check(L.pgvimp_batch_arena_bytes(cnt, C.cast(parr, C.c_void_p), C.cast(oarr, C.c_void_p), precision,
                                          C.byref(nbytes)))
        self.arena_bytes = nbytes.value
        self._arena_t = None
        arena_ptr = None
        if torch_arena:
            import torch
            self._arena_t = torch.empty(self.arena_bytes + 256, dtype=torch.uint8, device="cuda")
            base = self._arena_t.data_ptr()
            arena_ptr = (base + 255) & ~255
        h = C.c_void_p()
        _check(L.pgvimp_batch_create(cnt, C.cast(parr, C.c_void_p), C.cast(oarr, C.c_void_p), precision,
                                     arena_ptr, self.arena_bytes if torch_arena else 0, C.byref(h)))
        self.h = h
        self.count = cnt
        self.log_cap = max(o.iters * (max(o.slr_iters, 1) if p.dyn_kind != 0 else 1)
                           for p, o in zip(problems, options))

    def upload(self, stream=None):
        _check(lib().pgvimp_batch_upload(self.h, _stream_handle(stream)))

    def reset(self, stream=None):
        _check(lib().pgvimp_batch_reset(self.h, _stream_handle(stream)))

    def run(self, iters: int = 0, stream=None):
        _check(lib().pgvimp_batch_run(self.h, iters, _stream_handle(stream)))

    def phase(self, phase: int, arg: float = 0.0, stream=None):
        _check(lib().pgvimp_batch_phase(self.h, phase, C.c_double(arg), _stream_handle(stream)))

    def download(self, stream=None):
        _check(lib().pgvimp_batch_download(self.h, _stream_handle(stream)))

    def download_results(self, stream=None):
        _check(lib().pgvimp_batch_download_results(self.h, _stream_handle(stream)))

    def io_bytes(self):
        """(host-to-device bytes per upload, device-to-host bytes per full
        download, device-to-host bytes per results-only download)"""
        a, b, c = C.c_size_t(0), C.c_size_t(0), C.c_size_t(0)
        _check(lib().pgvimp_batch_io_bytes(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def status(self, i: int) -> int:
        """Per-plan status slot from the last download (0: ok)."""
        return int(self.read(i, BUF_SCAL, (24,))[S_STATUS])

    def result(self, i: int, full: bool = True) -> PlanResult:
        pb = self.problems[i]
        n, N = pb.n, pb.N
        mu, Sd = np.zeros((N + 1, n)), np.zeros((N + 1, n, n))
        So = np.zeros((N, n, n)) if full else None
        Ld = np.zeros((N + 1, n, n)) if full else None
        Lo = np.zeros((N, n, n)) if full else None
        logs = (StepInfo * max(self.log_cap, 1))()
        nl = C.c_int(0)
        _check(lib().pgvimp_batch_result(self.h, i, _p(mu), _p(Sd), _p(So), _p(Ld), _p(Lo),
                                         C.cast(logs, C.c_void_p), self.log_cap, C.byref(nl)))
        return PlanResult(mu, Sd, So, Ld, Lo, _log_dicts(logs, nl.value))

    def read(self, i: int, buf: int, shape) -> np.ndarray:
        out = np.zeros(shape)
        _check(lib().pgvimp_batch_read(self.h, i, buf, _p(out), out.size))
        return out

    def write(self, i: int, buf: int, arr):
        a = _f64(arr)
        _check(lib().pgvimp_batch_write(self.h, i, buf, _p(a), a.size))

    def close(self):
        if getattr(self, "h", None):
            lib().pgvimp_batch_destroy(self.h)
            self.h = None
        self._arena_t = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """The single-plan calls (pgvimp_create / step / plan / get / destroy)."""

    def __init__(self, problem, options, precision: int = PREC_MIXED):
        keep = _Keep()
        self._p = marshal_problem(problem, keep)
        self._o = marshal_options(options)
        self.problem = problem
        h = C.c_void_p()
        _check(lib().pgvimp_create(C.byref(self._p), C.byref(self._o), precision, C.byref(h)))
        self.h = h

    def step(self) -> dict:
        info = StepInfo()
        _check(lib().pgvimp_step(self.h, C.byref(info)))
        return _log_dicts([info], 1)[0]

    def plan(self, iters: int = 0):
        _check(lib().pgvimp_plan(self.h, iters))

    def get(self):
        n, N = self.problem.n, self.problem.N
        mu, Sd = np.zeros((N + 1, n)), np.zeros((N + 1, n, n))
        Ld, Lo = np.zeros((N + 1, n, n)), np.zeros((N, n, n))
        _check(lib().pgvimp_get(self.h, _p(mu), _p(Sd), _p(Ld), _p(Lo)))
        return mu, Sd, Ld, Lo

    def close(self):
        if getattr(self, "h", None):
            lib().pgvimp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The serving calls (pgvimp_server_create / submit / poll / destroy):
    continuous batching of independent plan requests on one GPU."""

    def __init__(self, hbm_budget_bytes: int, precision: int = PREC_MIXED, plan_threads: int = 64,
                 max_inflight: int = 32, max_batch: int = 16, batch_window_ms: float = 2.0,
                 host_staging_bytes: int = 0):
        cfg = ServerConfig(hbm_budget_bytes, host_staging_bytes, precision, plan_threads, max_inflight, max_batch,
                           batch_window_ms)
        h = C.c_void_p()
        _check(lib().pgvimp_server_create(C.byref(cfg), C.byref(h)))
        self.h = h
        self._sizes = {}

    @staticmethod
    def prepare(problem, options):
        """Marshals a request once (so that a timed submit only crosses the C ABI)."""
        keep = _Keep()
        return (marshal_problem(problem, keep), marshal_options(options), keep, (problem.n, problem.N))

    def submit(self, problem, options=None) -> int:
        """Queues a request: (problem, options), or a tuple from prepare()."""
        p, o, keep, size = problem if options is None else self.prepare(problem, options)
        rid = C.c_uint64(0)
        _check(lib().pgvimp_submit(self.h, C.byref(p), C.byref(o), C.byref(rid)))
        self._sizes[rid.value] = size
        return rid.value

    def poll(self, rid: int, timeout_ms: int = -1):
        """(mu, Sigma_ii, info) once the request is done; None if it is not
        finished within timeout_ms; raises PgvimpError if the plan failed."""
        n, N = self._sizes[rid]
        mu, Sd = np.zeros((N + 1, n)), np.zeros((N + 1, n, n))
        info = RequestInfo()
        st = lib().pgvimp_poll(self.h, rid, timeout_ms, _p(mu), _p(Sd), C.byref(info))
        if st == ENOTREADY:
            return None
        del self._sizes[rid]
        _check(st)
        d = {k: getattr(info, k) for k in ("status", "n", "N", "n_logs", "batch_size", "submit_ms", "start_ms",
                                           "done_ms")}
        d["last"] = _log_dicts([info.last], 1)[0]
        return mu, Sd, d

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib().pgvimp_server_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().pgvimp_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def marginals_noalloc(n: int, N: int, Ld, Lo, Sd, So, logdet, stream=None):
    """pgvimp_marginals_noalloc on CUDA tensors (float64, contiguous): block
    marginals of (Ld, Lo) into (Sd, So) and log det into `logdet` (1 element),
    with no device allocation by the library."""
    _check(lib().pgvimp_marginals_noalloc(n, N, C.c_void_p(Ld.data_ptr()), C.c_void_p(Lo.data_ptr()),
                                          C.c_void_p(Sd.data_ptr()), C.c_void_p(So.data_ptr()),
                                          C.c_void_p(logdet.data_ptr()), _stream_handle(stream)))


def version() -> str:
    buf = C.create_string_buffer(256)
    _check(lib().pgvimp_version(buf, 256))
    return buf.value.decode()


def solve(problems, options, precision: int = PREC_MIXED, stream=None) -> List[PlanResult]:
    """Plans every problem (one batch, all on the device) and returns results."""
    import torch
    b = Batch(problems, options, precision)
    b.upload(stream)
    b.reset(stream)
    b.run(0, stream)
    b.download(stream)
    torch.cuda.synchronize()
    out = [b.result(i) for i in range(b.count)]
    b.close()
    return out
