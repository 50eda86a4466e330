"""Failure paths, made to happen without faulting the GPU:

  - an expired bounded wait inside a kernel: the TMA bulk-copy smoother's mbarrier
    waits get a budget of 0 SM clocks (mlmc_set_wait_budget), so they give up at the
    first plane whose copy has not landed; the kernel drains its copies, returns, and
    the solve reports MLMC_ERR_TIMEOUT; with the budget restored the same context
    solves again, bit for bit as before;
  - a device allocation that fails: injected on the host (mlmc_inject_alloc_failure),
    reported as MLMC_ERR_OOM by the level call and by the service's batch, with the
    partially allocated batch released; afterwards everything runs again;
  - a request withdrawn from the service queue (mlmc_cancel) and a wait that must time out;
  - a wait of the tcgen05 field kernel on an mbarrier that nothing arrives on (injected on the
    host, mlmc_inject_wait_failure): NaN in the blocks' nodes, MLMC_ERR_TIMEOUT, and the
    context usable afterwards.
"""
import time

import numpy as np
import pytest

import paper_1607_03252_gb300 as mg
from paper_1607_03252_gb300.workloads import RUN_SEED, random_coefficient, random_rhs, sample_ids

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELD = dict(run_seed=RUN_SEED, sigma2=1.0, ell=0.3, M=64)


@pytest.fixture
def restore_controls():
    yield
    mg.set_wait_budget(2_000_000_000)
    mg.inject_alloc_failure(-1)
    mg.inject_wait_failure(0)


def _solve(k, f, smoother, cycles=3):
    u = torch.zeros_like(k)
    cyc, rel, st = mg.mg_solve_batch(mg.mg_cfg(2, 2, 0.0, cycles, mg.MLMC_PREC_F64, smoother), k, u, f)
    torch.cuda.synchronize()
    return u.cpu().numpy(), rel


@pytest.mark.parametrize("smoother", [mg.MLMC_SMOOTH_BULK_32x8, mg.MLMC_SMOOTH_BULK_64x8])
def test_expired_kernel_wait_reports_timeout_and_context_survives(restore_controls, smoother):
    n, B = 65, 2
    k = torch.from_numpy(np.stack([random_coefficient(n, 40 + s, 1.0) for s in range(B)])).cuda()
    f = torch.from_numpy(np.stack([random_rhs(n, 50 + s) for s in range(B)])).cuda()
    ref, rel_ref = _solve(k, f, mg.MLMC_SMOOTH_TWO_PASS)
    prev = mg.set_wait_budget(0)
    assert prev == 2_000_000_000
    with pytest.raises(mg.MlmcError) as e:
        _solve(k, f, smoother)
    assert e.value.status == mg.MLMC_ERR_TIMEOUT
    mg.set_wait_budget(prev)
    u, rel = _solve(k, f, smoother)
    assert np.array_equal(u, ref) and np.array_equal(rel, rel_ref)


def test_wait_budget_argument_checked():
    with pytest.raises(mg.MlmcError) as e:
        mg.set_wait_budget(-1)
    assert e.value.status == mg.MLMC_ERR_INVALID


@pytest.mark.parametrize("after", [0, 2, 5])
def test_injected_allocation_failure_reports_oom(restore_controls, after):
    cfg = mg.make_mlmc_cfg(FIELD["run_seed"], FIELD["sigma2"], FIELD["ell"], FIELD["M"], n0=17, rtol=1e-10)
    first = int(sample_ids(1, 0, 1)[0])
    _, Y_ref, _, _ = mg.mlmc_level_estimate(cfg, 1, first, 4)
    mg.inject_alloc_failure(after)  # the level batch needs more than 5 device allocations
    with pytest.raises(mg.MlmcError) as e:
        mg.mlmc_level_estimate(cfg, 1, first, 4)
    assert e.value.status == mg.MLMC_ERR_OOM
    assert "injected" in mg.lib().mlmc_last_error_string().decode()
    mg.inject_alloc_failure(-1)
    _, Y, _, _ = mg.mlmc_level_estimate(cfg, 1, first, 4)
    assert np.array_equal(Y, Y_ref)


def _svc(**kw):
    args = dict(n0=17, max_level=2, max_batch=8, workers=1, batch_wait_ms=1.0)
    args.update(kw)
    return mg.Service(mg.field_cfg(**FIELD), mg.mg_cfg(rtol=1e-10), **args)


def test_service_batch_with_failed_allocation(restore_controls):
    sid = int(sample_ids(1, 3, 1)[0])
    with _svc() as svc:
        mg.inject_alloc_failure(0)
        st, r = svc.wait(svc.submit(1, sid))
        assert st == mg.MLMC_OK and r.status == mg.MLMC_ERR_OOM
        mg.inject_alloc_failure(-1)
        st, r2 = svc.wait(svc.submit(1, sid))
        assert r2.status == mg.MLMC_OK
        assert svc.report().bytes_in_use == 0
    cfg = mg.make_mlmc_cfg(FIELD["run_seed"], FIELD["sigma2"], FIELD["ell"], FIELD["M"], n0=17, rtol=1e-10)
    _, Y, _, _ = mg.mlmc_level_estimate(cfg, 1, sid, 1)
    assert r2.Y == Y[0]


def test_service_cancel_queued_request():
    ids = [int(sample_ids(1, i, 1)[0]) for i in range(3)]
    # one worker that waits 300 ms for batch-mates: the requests stay queued meanwhile
    with _svc(batch_wait_ms=300.0) as svc:
        t = [svc.submit(1, sid) for sid in ids]
        assert svc.cancel(t[1]) == mg.MLMC_OK
        st, r = svc.wait(t[1], timeout_ms=10.0)  # delivered at once, not after the batch
        assert st == mg.MLMC_OK and r.status == mg.MLMC_ERR_CANCELLED
        with pytest.raises(mg.MlmcError) as e:
            svc.cancel(t[1])  # delivered: unknown now
        assert e.value.status == mg.MLMC_ERR_NOT_FOUND
        res = [svc.wait(t[i])[1] for i in (0, 2)]
        assert all(x.status == mg.MLMC_OK for x in res)
        rep = svc.report()
        assert rep.cancelled == 1 and rep.completed == 2 and rep.pending == 0
        # a finished request can no longer be withdrawn
        t3 = svc.submit(0, int(sample_ids(0, 9, 1)[0]))
        deadline = time.monotonic() + 60.0
        while svc.report().completed < 3 and time.monotonic() < deadline:
            time.sleep(0.001)
        assert svc.cancel(t3) == mg.MLMC_ERR_BUSY
        assert svc.wait(t3)[1].status == mg.MLMC_OK


def test_service_wait_times_out_behind_a_pending_batch():
    with _svc(batch_wait_ms=200.0) as svc:
        t = svc.submit(2, int(sample_ids(2, 0, 1)[0]))
        st, r = svc.wait(t, timeout_ms=0.001)  # the batch starts 200 ms after the submission
        assert st == mg.MLMC_ERR_TIMEOUT and r.status == mg.MLMC_PENDING
        st, r = svc.wait(t)
        assert st == mg.MLMC_OK and r.status == mg.MLMC_OK


def test_expired_field_wait_reports_timeout_and_context_survives(restore_controls):
    """The tensor-core field (tcgen05 from 65^3) bounds its mbarrier waits. With the failure
    injected on the host (its issuing thread also waits on an mbarrier nothing arrives on) and
    a short budget, the wait runs out: the blocks drain their copies and products, write NaN,
    free their tensor memory, and mlmc_field_eval reports MLMC_ERR_TIMEOUT. The injection is
    used up; the same context then gives the field again, bit for bit."""
    n, B = 65, 2
    fc = mg.field_cfg(**FIELD)
    ids = sample_ids(2, 11, B)
    ref = torch.empty((B, n, n, n), dtype=torch.float64, device="cuda")
    mg.mlmc_field_eval(fc, ids, ref)
    prev = mg.set_wait_budget(100_000)
    mg.inject_wait_failure(1)
    k = torch.zeros_like(ref)
    with pytest.raises(mg.MlmcError) as e:
        mg.mlmc_field_eval(fc, ids, k)
    assert e.value.status == mg.MLMC_ERR_TIMEOUT
    assert torch.isnan(k[..., : n - 1]).all()  # the tcgen05 volume; the face x = n - 1 is another kernel's
    mg.set_wait_budget(prev)
    k2 = torch.empty_like(ref)
    mg.mlmc_field_eval(fc, ids, k2)
    assert torch.equal(k2, ref)
    with pytest.raises(mg.MlmcError):
        mg.inject_wait_failure(-1)
