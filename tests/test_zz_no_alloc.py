"""The allocation-free marginals entry point (pgvimp_marginals_noalloc).

It serves callers that cannot allocate device memory (for example while
their stream is captured into a CUDA graph, or under a fixed memory budget):
its scratch is a fixed device array inside the library.  Its results must
equal those of the allocating path, PGVIMP_PHASE_MARGINALS on a batch, on two
calls in a row (the second call reuses the shared scratch left by the first).
This file is collected last so that a failure here comes after every other
test has run."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _spd_chain(rng, n, N, scale):
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


def _reference(L, pb, op, Ld, Lo):
    """The allocating entry point: a batch's marginals phase."""
    import torch
    b = L.Batch([pb], [op], L.PREC_PLAIN_FP64)
    b.upload()
    b.reset()
    b.phase(L.PHASE_PRIOR)
    b.write(0, L.BUF_LD, Ld)
    b.write(0, L.BUF_LO, Lo)
    b.phase(L.PHASE_MARGINALS)
    torch.cuda.synchronize()
    Sd = b.read(0, L.BUF_SD, Ld.shape)
    So = b.read(0, L.BUF_SO, Lo.shape)
    ld = b.read(0, L.BUF_SCAL, (24,))[L.S_LOGDET]
    b.close()
    return Sd, So, ld


@pytest.mark.parametrize("make,N", [(W.c1_point2d, 50), (W.c3_arm, 20)])
def test_noalloc_marginals_match_allocating_path_twice(make, N):
    import torch
    assert torch.cuda.is_available()
    from paper_2411_03416_b300 import _lib as L
    pb, op = make(N=N)
    n = pb.n
    rng = np.random.default_rng(1234 + n)
    Sd_t = torch.empty((N + 1, n, n), dtype=torch.float64, device="cuda")
    So_t = torch.empty((N, n, n), dtype=torch.float64, device="cuda")
    ld_t = torch.empty(1, dtype=torch.float64, device="cuda")
    for call, scale in enumerate((1.0, 7.5)):
        Ld, Lo = _spd_chain(rng, n, N, scale)
        Sd_r, So_r, ld_r = _reference(L, pb, op, Ld, Lo)
        Ld_t = torch.from_numpy(Ld).cuda()
        Lo_t = torch.from_numpy(Lo).cuda()
        L.marginals_noalloc(n, N, Ld_t, Lo_t, Sd_t, So_t, ld_t)
        torch.cuda.synchronize()
        Sd, So, ld = Sd_t.cpu().numpy(), So_t.cpu().numpy(), float(ld_t.item())
        np.testing.assert_allclose(Sd, Sd_r, rtol=1e-12, atol=1e-14 * np.abs(Sd_r).max(), err_msg=f"call {call}")
        np.testing.assert_allclose(So, So_r, rtol=1e-12, atol=1e-14 * np.abs(So_r).max(), err_msg=f"call {call}")
        assert abs(ld - ld_r) <= 1e-12 * abs(ld_r), (call, ld, ld_r)


def test_noalloc_rejects_sizes_beyond_the_fixed_scratch():
    import torch
    from paper_2411_03416_b300 import _lib as L
    t = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(L.PgvimpError) as e:
        L.marginals_noalloc(4, 20164, t, t, t, t, t)
    assert e.value.status == L.EINVAL and "limit" in str(e.value)
    with pytest.raises(L.PgvimpError) as e:
        L.marginals_noalloc(5, 10, t, t, t, t, t)
    assert e.value.status == L.EINVAL
