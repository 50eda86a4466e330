"""GPU tests of the continuous-batching solve service: results equal the batch call's
bit for bit (alone and in a mixed stream of levels), backpressure, timeouts."""
import time

import numpy as np
import pytest

import paper_1607_03252_gb300 as mg
from paper_1607_03252_gb300.workloads import RUN_SEED, sample_ids

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELD = dict(run_seed=RUN_SEED, sigma2=1.0, ell=0.3, M=64)


def _svc(**kw):
    args = dict(n0=17, max_level=2, max_batch=8, workers=2, batch_wait_ms=1.0)
    args.update(kw)
    return mg.Service(mg.field_cfg(**FIELD), mg.mg_cfg(rtol=1e-10), **args)


def _reference(level, ids):
    cfg = mg.make_mlmc_cfg(FIELD["run_seed"], FIELD["sigma2"], FIELD["ell"], FIELD["M"], n0=17, rtol=1e-10,
                           max_batch=3)
    out = []
    for sid in ids:  # one id per call: each sample alone
        _, Y, Qf, Qc = mg.mlmc_level_estimate(cfg, level, int(sid), 1)
        out.append((Y[0], Qf[0], Qc[0]))
    return out


def test_service_results_equal_alone_and_in_mix():
    rng = np.random.default_rng(5)
    reqs = [(int(l), int(sample_ids(int(l), int(i), 1)[0])) for l, i in zip(rng.integers(0, 3, 40), rng.integers(0, 10, 40))]
    with _svc() as svc:
        tickets = [svc.submit(l, sid) for l, sid in reqs]
        results = [svc.wait(t)[1] for t in tickets]
        rep = svc.report()
    assert rep.completed == len(reqs) and rep.pending == 0
    for (l, sid), r in zip(reqs, results):
        assert r.status == mg.MLMC_OK and r.level == l and r.sample_id == sid
        (Y, Qf, Qc), = _reference(l, [sid])
        assert r.Y == Y and r.Qf == Qf and r.Qc == Qc  # bitwise: the batch does not change a sample
        assert r.t_submit <= r.t_start <= r.t_done


def test_service_single_request_alone():
    sid = int(sample_ids(2, 3, 1)[0])
    with _svc(workers=1) as svc:
        st, r = svc.wait(svc.submit(2, sid))
    (Y, Qf, Qc), = _reference(2, [sid])
    assert r.Y == Y


def test_service_backpressure_and_errors():
    with _svc(queue_capacity=4, workers=1, batch_wait_ms=50.0) as svc:
        tickets = [svc.submit(2, int(sample_ids(2, i, 1)[0])) for i in range(12)]
        assert any(t is None for t in tickets)  # MLMC_ERR_BUSY once 4 are pending
        with pytest.raises(mg.MlmcError):
            svc.submit(7, 1)  # level outside 0..max_level
        with pytest.raises(mg.MlmcError):
            svc.poll(123456789)  # unknown ticket
        live = [t for t in tickets if t is not None]
        # the worker waits 50 ms for batch-mates before it starts: still pending after 1 us
        st, r = svc.wait(live[-1], timeout_ms=0.001)
        assert st == mg.MLMC_ERR_TIMEOUT
        for t in live:
            st, r = svc.wait(t)
            assert r.status == mg.MLMC_OK
        assert svc.report().rejected >= 1


def test_service_admission_budget_limits_batches():
    # a budget that holds about one level-2 sample at a time: batches shrink, results stay equal
    per = 80 << 20
    with _svc(hbm_budget_bytes=per, max_batch=8) as svc:
        ids = [int(sample_ids(2, i, 1)[0]) for i in range(6)]
        res = [svc.wait(svc.submit(2, sid))[1] for sid in ids]
        assert svc.report().bytes_in_use == 0
    ref = _reference(2, ids)
    assert all(r.Y == y for r, (y, _, _) in zip(res, ref))
