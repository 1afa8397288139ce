"""The allocation-free marginals entry point (pgvimp_marginals_noalloc).

It serves callers that cannot allocate device memory (for example while
their stream is captured into a CUDA graph, or under a fixed memory budget):
its scratch is a fixed device array inside the library.  Its results must
equal those of the allocating path, PGVIMP_PHASE_MARGINALS on a batch, on two
calls in a row (the second call reuses the shared scratch left by the first),
and the oracle's belief-propagation marginals.  This file is collected last
so that a failure here comes after every other test has run."""
import numpy as np
import pytest

import oracle
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
        # and the oracle (literal GBP messages), element by element
        Sd_o, So_o, ld_o = oracle.marginals(Ld, Lo)
        np.testing.assert_allclose(Sd, Sd_o, rtol=1e-10, atol=1e-12 * np.abs(Sd_o).max(), err_msg=f"call {call}")
        np.testing.assert_allclose(So, So_o, rtol=1e-10, atol=1e-12 * np.abs(So_o).max(), err_msg=f"call {call}")
        assert abs(ld - ld_o) <= 1e-10 * abs(ld_o), (call, ld, ld_o)


def _spd_chain_blocks(rng, n, N, scale):
    """B^T B + I for a random block-bidiagonal B, assembled block by block
    (large N without the dense matrix)."""
    Bd = rng.standard_normal((N + 1, n, n)) + 2 * np.eye(n)
    Bu = rng.standard_normal((N, n, n))        # block (i, i+1)
    Ld = np.einsum("iab,iac->ibc", Bd, Bd) + np.eye(n)
    Ld[1:] += np.einsum("iab,iac->ibc", Bu, Bu)
    Lo = np.einsum("iab,iac->ibc", Bu, Bd[:-1])  # (B^T B)_{i+1,i} = B_{i,i+1}^T B_{i,i}
    return scale * Ld, scale * Lo


def test_noalloc_at_the_largest_accepted_size():
    """n = 4 with N = 20163, the largest horizon the fixed 4 MiB scratch
    holds, is accepted and matches the oracle; N = 20164 is rejected."""
    import torch
    from paper_2411_03416_b300 import _lib as L
    n, N = 4, 20163
    rng = np.random.default_rng(77)
    Ld, Lo = _spd_chain_blocks(rng, n, N, 2.0)
    Sd_t = torch.empty((N + 1, n, n), dtype=torch.float64, device="cuda")
    So_t = torch.empty((N, n, n), dtype=torch.float64, device="cuda")
    ld_t = torch.empty(1, dtype=torch.float64, device="cuda")
    L.marginals_noalloc(n, N, torch.from_numpy(Ld).cuda(), torch.from_numpy(Lo).cuda(), Sd_t, So_t, ld_t)
    torch.cuda.synchronize()
    Sd_o, So_o, ld_o = oracle.marginals(Ld, Lo)
    np.testing.assert_allclose(Sd_t.cpu().numpy(), Sd_o, rtol=1e-10, atol=1e-12 * np.abs(Sd_o).max())
    np.testing.assert_allclose(So_t.cpu().numpy(), So_o, rtol=1e-10, atol=1e-12 * np.abs(So_o).max())
    assert abs(float(ld_t.item()) - ld_o) <= 1e-10 * abs(ld_o)
    t = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(L.PgvimpError) as e:
        L.marginals_noalloc(n, N + 1, t, t, t, t, t)
    assert e.value.status == L.EINVAL


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
