"""The serving calls: continuous batching of independent requests.  Each
result must be the same alone and in the mix (the plan a request gets does not
depend on what shares its batch), match the oracle, and admission control must
hold under a budget that fits only a few plans at once."""
import time
from dataclasses import replace

import numpy as np
import pytest

import workloads as W
from _parity import TOL_MIXED, compare_plan, gpu_solve

pytestmark = pytest.mark.gpu

MIXED, FP64, MIXED_DF = 1, 0, 2


@pytest.fixture(scope="module")
def pg():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA device"
    import paper_2411_03416_b300 as pg
    pg.lib()
    return pg


def _mix():
    """A small mix of the three request kinds (point robot, quadrotor SLR, arm)."""
    reqs = []
    for r, N in enumerate([40, 75, 20, 60]):
        reqs.append(W.c1_point2d(request=r, N=N, iters=8))
    reqs.append(W.c4_quadrotor(request=0, N=30, iters=4, slr_iters=2))
    reqs.append(W.c4_quadrotor(request=1, N=45, iters=4, slr_iters=2))
    reqs.append(W.c3_arm(request=0, N=25, iters=5))
    return reqs


@pytest.mark.parametrize("prec,tpb", [(MIXED, 64), (MIXED_DF, 0), (MIXED, 0), (FP64, 32), (MIXED_DF, 64)])
def test_server_results_equal_alone(pg, prec, tpb):
    """Every batch is launched as one captured CUDA graph; each result equals
    the same plan run alone."""
    reqs = _mix()
    srv = pg.Server(2 << 30, precision=prec, plan_threads=tpb, max_inflight=4, max_batch=8, batch_window_ms=5.0)
    ids = [srv.submit(pb, op) for pb, op in reqs]
    out = [srv.poll(i, timeout_ms=120_000) for i in ids]
    stats = srv.stats()
    srv.close()
    assert all(o is not None for o in out)
    assert stats["plans"] == len(reqs)
    assert stats["graph_launches"] == stats["batches"] and stats["graph_instantiations"] >= 1
    for (pb, op), (mu, Sd, info) in zip(reqs, out):
        alone = gpu_solve([pb], [replace(op, plan_threads=tpb)], prec)[0]
        np.testing.assert_array_equal(mu, alone.mu)
        np.testing.assert_array_equal(Sd, alone.Sd)
        assert info["status"] == 0 and info["n_logs"] == op.iters * max(1, op.slr_iters)
        assert info["submit_ms"] <= info["start_ms"] <= info["done_ms"]


def test_server_matches_oracle(pg):
    pb, op = W.c1_point2d(N=50, iters=10)
    srv = pg.Server(1 << 30, precision=MIXED, plan_threads=64)
    mu, Sd, info = srv.poll(srv.submit(pb, op))
    srv.close()

    class R:  # the shape compare_plan expects
        pass
    r = R()
    r.mu, r.Sd = mu, Sd
    alone = gpu_solve([pb], [replace(op, plan_threads=64)], MIXED)[0]
    r.logs = alone.logs
    compare_plan(pb, op, r, rtol_mu=TOL_MIXED["mu"], rtol_sigma=TOL_MIXED["sigma"])


def test_admission_under_a_tight_budget(pg):
    """A budget that holds about two of these plans: all requests still
    finish, in more batches than the window alone would form."""
    from paper_2411_03416_b300 import _lib as L
    reqs = [W.c1_point2d(request=r, N=200, iters=4) for r in range(8)]
    one = L.Batch([reqs[0][0]], [replace(reqs[0][1], plan_threads=64)], MIXED, torch_arena=False)
    need = one.arena_bytes
    one.close()
    srv = pg.Server(int(2.5 * need), precision=MIXED, plan_threads=64, max_inflight=8, max_batch=8,
                    batch_window_ms=20.0, host_staging_bytes=64 << 20)
    ids = [srv.submit(pb, op) for pb, op in reqs]
    out = [srv.poll(i, timeout_ms=120_000) for i in ids]
    stats = srv.stats()
    srv.close()
    assert all(o is not None for o in out)
    assert stats["batches"] >= 4               # never more than two plans' memory at once
    assert max(o[2]["batch_size"] for o in out) <= 2


def test_poll_not_ready_and_errors(pg):
    from paper_2411_03416_b300 import _lib as L
    pb, op = W.c2_point2d_dense(iters=30)
    srv = pg.Server(1 << 30, precision=FP64, plan_threads=0, max_inflight=1, max_batch=1, batch_window_ms=0.0)
    rid = srv.submit(pb, op)
    assert srv.poll(rid, timeout_ms=0) is None          # a 30-iteration N = 750 plan takes far longer
    with pytest.raises(L.PgvimpError) as e:
        srv.submit(replace(pb, K0=-np.eye(4)), op)       # validated at submit
    assert e.value.status == L.ENOTPD
    with pytest.raises(L.PgvimpError) as e:
        srv.submit(pb, replace(op, gh_p=1))
    assert e.value.status == L.EINVAL
    small = pg.Server(1 << 20, precision=MIXED)
    with pytest.raises(L.PgvimpError) as e:
        small.submit(pb, op)                              # larger than the whole pool
    assert e.value.status == L.ENOMEM
    small.close()
    with pytest.raises(L.PgvimpError) as e:
        L._check(L.lib().pgvimp_poll(srv.h, 987654, 0, None, None, None))
    assert e.value.status == L.EINVAL
    t = time.time()
    assert srv.poll(rid, timeout_ms=600_000) is not None
    assert time.time() - t < 600
    srv.close()
