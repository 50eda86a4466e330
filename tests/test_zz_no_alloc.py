"""mg_solve_batch_noalloc: the batched solve for callers that cannot allocate device
memory (its workspace is a fixed array inside the library). It must give the same
results as mg_solve_batch, call after call, although every call reuses the array
and finds the previous call's data in it. This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import paper_1607_03252_gb300 as mg
from paper_1607_03252_gb300.workloads import random_coefficient, random_rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(cfg, k, u, f=None):
    B, n = k.shape[0], k.shape[1]
    stats = (mg.MgStats * B)()
    st = mg.lib().mg_solve_batch_noalloc(ctypes.byref(cfg), B, n, ctypes.c_void_p(k.data_ptr()),
                                         ctypes.c_void_p(f.data_ptr() if f is not None else 0),
                                         ctypes.c_void_p(u.data_ptr()), stats,
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, np.array([s.cycles for s in stats]), np.array([s.rel_res for s in stats])


@pytest.mark.parametrize("prec", [mg.MLMC_PREC_F64, mg.MLMC_PREC_MIXED])
def test_noalloc_matches_allocating_solve_twice(prec):
    cfg = mg.mg_cfg(2, 2, 1e-10, 100, prec)
    cases = [(17, 3, 11), (33, 2, 12)]  # two calls in a row with different sizes
    for n, B, seed in cases:
        k = torch.from_numpy(np.stack([random_coefficient(n, seed + s, 1.0) for s in range(B)])).cuda()
        f = torch.from_numpy(np.stack([random_rhs(n, seed + 50 + s) for s in range(B)])).cuda()
        u_ref = torch.zeros_like(k)
        cyc_ref, rel_ref, st_ref = mg.mg_solve_batch(cfg, k, u_ref, f)
        u = torch.zeros_like(k)  # the same (zero) initial guess as the allocating solve
        st, cyc, rel = _noalloc(cfg, k, u, f)
        torch.cuda.synchronize()
        assert st == mg.MLMC_OK == st_ref
        assert np.array_equal(cyc, cyc_ref)
        np.testing.assert_allclose(rel, rel_ref, rtol=1e-12, atol=0)
        ur, un = u_ref.cpu().numpy(), u.cpu().numpy()
        assert np.abs(un - ur).max() <= 1e-12 * np.abs(ur).max()


def test_noalloc_rejects_sizes_beyond_its_workspace():
    cfg = mg.mg_cfg()
    k = torch.ones((2, 65, 65, 65), dtype=torch.float64, device="cuda")
    u = torch.zeros_like(k)
    st, _, _ = _noalloc(cfg, k, u)
    assert st == mg.MLMC_ERR_INVALID
    msg = mg.lib().mlmc_last_error_string().decode()
    assert "workspace" in msg and "bytes" in msg
    assert torch.count_nonzero(u).item() == 0
