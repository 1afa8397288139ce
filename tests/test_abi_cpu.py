"""The C ABI library loads without a GPU, exports every symbol that
include/pgvimp.h declares, agrees with the binding on struct layouts, and
rejects bad problems at validation (no compute calls, no device needed)."""
import ctypes as C
import os
import re
from dataclasses import replace

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pg():
    import paper_2411_03416_b300 as pg
    pg.lib()
    return pg


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "pgvimp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pgvimp_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(pg):
    L = pg.lib()
    names = declared_symbols()
    assert len(names) >= 20
    for name in names:
        assert hasattr(L, name), name
    from paper_2411_03416_b300 import _lib
    assert set(_lib.EXPORTED) == set(names)


def test_struct_sizes_match_binding(pg):
    from paper_2411_03416_b300 import _lib
    a, b, c = C.c_size_t(), C.c_size_t(), C.c_size_t()
    assert pg.lib().pgvimp_abi_sizes(C.byref(a), C.byref(b), C.byref(c)) == 0
    assert a.value == C.sizeof(_lib.Problem)
    assert b.value == C.sizeof(_lib.Options)
    assert c.value == C.sizeof(_lib.StepInfo)


def _arena_status(pg, pb, op, precision=1):
    from paper_2411_03416_b300 import _lib
    keep = _lib._Keep()
    p = _lib.marshal_problem(pb, keep)
    o = _lib.marshal_options(op)
    nb = C.c_size_t()
    st = pg.lib().pgvimp_batch_arena_bytes(1, C.byref(p), C.byref(o), precision, C.byref(nb))
    return st, nb.value, pg.lib().pgvimp_last_error(None).decode()


def test_validation_accepts_the_configs(pg):
    for make in (W.c1_point2d, W.c3_arm):
        pb, op = make(N=20)
        st, nb, msg = _arena_status(pg, pb, op)
        assert st == 0, msg
        assert nb > 0
    pb, op = W.c4_quadrotor(N=20)
    assert _arena_status(pg, pb, op)[0] == 0


def test_validation_rejects_bad_inputs(pg):
    from paper_2411_03416_b300 import _lib
    pb, op = W.c1_point2d(N=10)
    cases = [
        (replace(pb, n=5), op, _lib.EINVAL),
        (replace(pb, N=0), op, _lib.EINVAL),
        (replace(pb, T=-1.0), op, _lib.EINVAL),
        (replace(pb, K0=-np.eye(4)), op, _lib.ENOTPD),
        (replace(pb, Qc=np.array([[1.0, 2.0], [0.0, 1.0]])), op, _lib.ENOTPD),
        (replace(pb, mu0=np.array([np.nan, 0, 0, 0])), op, _lib.ENOTFINITE),
        (pb, replace(op, gh_p=1), _lib.EINVAL),
        (pb, replace(op, beta_max=0.0), _lib.EINVAL),
        (pb, replace(op, max_bisect=100), _lib.EINVAL),
        (replace(pb, sdf=np.full((1, 1), 1.0, dtype=np.float32)), op, _lib.EINVAL),
    ]
    for p, o, want in cases:
        st, _, msg = _arena_status(pg, p, o)
        assert st == want, (want, st, msg)
        assert msg
    bad_sdf = pb.sdf.copy()
    bad_sdf[3, 3] = np.inf
    assert _arena_status(pg, replace(pb, sdf=bad_sdf), op)[0] == _lib.ENOTFINITE
    assert _arena_status(pg, pb, op, precision=7)[0] == _lib.EINVAL


def test_plans_sharing_a_map_store_it_once(pg):
    """Plans that pass the same grid share one device copy of it; distinct
    grids with equal contents are still stored separately."""
    from paper_2411_03416_b300 import _lib
    pb, op = W.c1_point2d()
    keep = _lib._Keep()

    def arena(probs):
        parr = (_lib.Problem * len(probs))(*[_lib.marshal_problem(p, keep) for p in probs])
        oarr = (_lib.Options * len(probs))(*[_lib.marshal_options(op) for _ in probs])
        nb = C.c_size_t(0)
        assert pg.lib().pgvimp_batch_arena_bytes(len(probs), C.cast(parr, C.c_void_p), C.cast(oarr, C.c_void_p),
                                                 1, C.byref(nb)) == 0
        return nb.value

    grid = pb.sdf.nbytes
    shared = arena([pb, replace(pb, muN=pb.muN + 0.1)])
    separate = arena([pb, replace(pb, sdf=np.array(pb.sdf, copy=True))])
    assert separate - shared >= grid


def test_plan_threads_validation(pg):
    """The thread form (1), the lane form (16, n = 4 only), the default (0) and
    the block form with 32..256 threads in multiples of 32; one value per batch."""
    from paper_2411_03416_b300 import _lib
    pb, op = W.c1_point2d()
    for bad in (-1, 2, 8, 48, 288, 512):
        assert _arena_status(pg, pb, replace(op, plan_threads=bad))[0] == _lib.EINVAL
    for good in (0, 1, 16, 32, 64, 256):
        assert _arena_status(pg, pb, replace(op, plan_threads=good))[0] == 0
    pq, oq = W.c4_quadrotor(N=20)
    assert _arena_status(pg, pq, replace(oq, plan_threads=16))[0] == _lib.EINVAL
    keep = _lib._Keep()
    parr = (_lib.Problem * 2)(*[_lib.marshal_problem(pb, keep) for _ in range(2)])
    oarr = (_lib.Options * 2)(_lib.marshal_options(op), _lib.marshal_options(replace(op, plan_threads=16)))
    nb = C.c_size_t(0)
    st = pg.lib().pgvimp_batch_arena_bytes(2, C.cast(parr, C.c_void_p), C.cast(oarr, C.c_void_p), 1, C.byref(nb))
    assert st == _lib.EINVAL
    # the block form runs every precision, double-float recursions included
    assert _arena_status(pg, pb, replace(op, plan_threads=64), precision=2)[0] == 0


def test_update_validation(pg):
    """The update is Thm 1's (0) or the natural-gradient step (1), which
    needs beta_max <= 1."""
    from paper_2411_03416_b300 import _lib
    pb, op = W.c1_point2d()
    assert _arena_status(pg, pb, replace(op, update=1))[0] == 0
    assert _arena_status(pg, pb, replace(op, update=2))[0] == _lib.EINVAL
    assert _arena_status(pg, pb, replace(op, update=-1))[0] == _lib.EINVAL
    assert _arena_status(pg, pb, replace(op, update=1, beta_max=1.5))[0] == _lib.EINVAL
    assert _arena_status(pg, pb, replace(op, update=0, beta_max=1.5))[0] == 0


def test_temperature_schedule_validation(pg):
    from paper_2411_03416_b300 import _lib
    pb, op = W.c1_point2d()
    assert _arena_status(pg, pb, replace(op, temperature_high=10.0, switch_iter=5))[0] == 0
    assert _arena_status(pg, pb, replace(op, temperature_high=-1.0, switch_iter=5))[0] == _lib.EINVAL
    assert _arena_status(pg, pb, replace(op, temperature_high=float("inf"), switch_iter=5))[0] == _lib.EINVAL
    assert _arena_status(pg, pb, replace(op, temperature_high=10.0, switch_iter=-2))[0] == _lib.EINVAL


def test_smolyak_validation(pg):
    from paper_2411_03416_b300 import _lib
    pb, op = W.c1_point2d()
    assert _arena_status(pg, pb, replace(op, rule=W.RULE_SMOLYAK, gh_p=3))[0] == 0
    assert _arena_status(pg, pb, replace(op, rule=W.RULE_SMOLYAK, gh_p=1))[0] == _lib.EINVAL
    assert _arena_status(pg, pb, replace(op, rule=7))[0] == _lib.EINVAL
    arm, aop = W.c3_arm(N=20)
    assert _arena_status(pg, arm, replace(aop, rule=W.RULE_SMOLYAK, gh_p=3))[0] == 0
    assert _arena_status(pg, arm, replace(aop, rule=W.RULE_SMOLYAK, gh_p=10))[0] == _lib.EINVAL   # too large
