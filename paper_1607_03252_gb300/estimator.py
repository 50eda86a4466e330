"""Adaptive MLMC estimator (Algorithm 2) -- a ctypes wrapper of mlmc_adaptive_* in the library.

Every decision of the algorithm (sample sizes by Eq. 15, the bias test of Eq. 14, the
online rate fits, level growth, the lane plan of a round) is made in libmlmc_gb300.so;
this class marshals the configuration, optionally hands the library a Python sampler in
place of its GPU level pipeline, and keeps the per-round log and JSON checkpoints.

Sample ids of level l are (l << 48) | i for i = 0, 1, ... in order, so a run restored
from `state()` continues with exactly the ids an uninterrupted run would use and ends
with the same records.
"""
from __future__ import annotations

import ctypes
import json
import math

from . import _capi as mg


class MLMCEstimator:
    def __init__(self, run_seed, sigma2, ell, M, levels, N_init, eps, theta=0.5, n0=17, nu=(2, 2), rtol=1e-10,
                 precision=mg.MLMC_PREC_F64, accel=mg.MLMC_ACCEL_NONE, smoother=mg.MLMC_SMOOTH_AUTO,
                 max_batch=0, max_cycles=300, stream=None, cost_model="measured", streams=None, max_level=None,
                 alpha=None, alpha0=2.0 / 3.0, alpha_floor=0.1, cov=mg.MLMC_COV_GAUSS, sampler=None):
        """levels must be 0..L0. sampler (optional): f(level, first_index, count) -> (N, mean,
        M2) replaces the GPU level pipeline (e.g. a host model of the level differences)."""
        if cost_model not in ("measured", "nodes"):
            raise ValueError("cost_model must be 'measured' or 'nodes'")
        levels = list(levels)
        if levels != list(range(len(levels))):
            raise ValueError("levels must be 0..L0")
        if isinstance(N_init, int):
            N_init = [N_init] * len(levels)
        if len(N_init) != len(levels):
            raise ValueError("N_init needs one count per level")
        if max_level is not None and (len(levels) < 2 or max_level < levels[-1]):
            raise ValueError("level growth starts from levels 0..L (L >= 1) with L <= max_level")
        self.params = dict(cost_model=cost_model, run_seed=int(run_seed), sigma2=float(sigma2), ell=float(ell), M=int(M),
                           levels=levels, N_init=[int(x) for x in N_init], eps=float(eps), theta=float(theta),
                           n0=int(n0), nu=list(nu), rtol=float(rtol), precision=int(precision), accel=int(accel),
                           smoother=int(smoother), max_batch=int(max_batch), max_cycles=int(max_cycles),
                           max_level=None if max_level is None else int(max_level),
                           alpha=None if alpha is None else float(alpha), alpha0=float(alpha0),
                           alpha_floor=float(alpha_floor), cov=int(cov))
        self.stream = stream
        self.streams = list(streams) if streams else [stream]
        self.log = []
        self._sampler_py = sampler
        self._sampler_c = None
        self._h = None
        self._make_handle()

    # -- handle -------------------------------------------------------------------------
    def _make_handle(self):
        p = self.params
        c = mg.AdaptiveCfg()
        c.level = mg.make_mlmc_cfg(p["run_seed"], p["sigma2"], p["ell"], p["M"], n0=p["n0"], nu1=p["nu"][0],
                                   nu2=p["nu"][1], rtol=p["rtol"], max_cycles=p["max_cycles"],
                                   precision=p["precision"], max_batch=p["max_batch"], stream=self.stream,
                                   smoother=p["smoother"], accel=p["accel"], cov=p["cov"])
        c.L0 = len(p["levels"]) - 1
        c.max_level = c.L0 if p["max_level"] is None else p["max_level"]
        for l, n in enumerate(p["N_init"]):
            c.N_init[l] = n
        for l in range(len(p["N_init"]), min(c.max_level + 1, mg.MLMC_MAX_LEVELS)):
            c.N_init[l] = p["N_init"][-1]  # grown levels start at the last pilot count
        c.eps, c.theta = p["eps"], p["theta"]
        c.cost_model = mg.MLMC_COST_NODES if p["cost_model"] == "nodes" else mg.MLMC_COST_MEASURED
        c.alpha = p["alpha"] if p["alpha"] is not None else 0.0
        c.alpha0, c.alpha_floor = p["alpha0"], p["alpha_floor"]
        c.lanes = len(self.streams)
        for k, st in enumerate(self.streams):
            c.lane_streams[k] = st.cuda_stream if st is not None else None
        self._cfg = c
        h = mg.lib().mlmc_adaptive_create(ctypes.byref(c))
        if not h:
            raise mg.MlmcError(mg.MLMC_ERR_INVALID, "mlmc_adaptive_create", mg.lib().mlmc_last_error_string().decode())
        self._h = h
        if self._sampler_py is not None:
            f = self._sampler_py

            def cb(user, level, first, count, N, mean, M2):
                try:
                    n, m, m2 = f(int(level), int(first), int(count))
                except Exception:
                    return mg.MLMC_ERR_INVALID
                N[0], mean[0], M2[0] = float(n), float(m), float(m2)
                return mg.MLMC_OK

            self._sampler_c = mg.LEVEL_SAMPLER(cb)
            mg._check(mg.lib().mlmc_adaptive_set_sampler(self._h, self._sampler_c, None), "mlmc_adaptive_set_sampler")

    def __del__(self):
        try:
            if self._h:
                mg.lib().mlmc_adaptive_destroy(self._h)
                self._h = None
        except Exception:
            pass

    def _summary(self):
        s = mg.AdaptiveSummary()
        mg._check(mg.lib().mlmc_adaptive_result(self._h, ctypes.byref(s)), "mlmc_adaptive_result")
        return s

    def _state(self):
        st = mg.AdaptiveState()
        mg._check(mg.lib().mlmc_adaptive_get_state(self._h, ctypes.byref(st)), "mlmc_adaptive_get_state")
        return st

    # -- views ---------------------------------------------------------------------------
    @property
    def levels(self):
        return list(range(self._state().L + 1))

    @property
    def have(self):
        st = self._state()
        return [int(st.have[l]) for l in range(st.L + 1)]

    @property
    def records(self):
        st = self._state()
        return [(st.N[l], st.mean[l], st.M2[l]) for l in range(st.L + 1)]

    @property
    def rounds(self):
        return self._state().rounds

    # -- state ---------------------------------------------------------------------------
    def state(self) -> dict:
        st = self._state()
        fields = {k: (list(getattr(st, k)) if not isinstance(getattr(st, k), int) else getattr(st, k))
                  for k, _ in mg.AdaptiveState._fields_}
        return {"params": self.params, "state": fields, "log": self.log}

    def checkpoint(self, path):
        with open(path, "w") as fh:
            json.dump(self.state(), fh)

    @classmethod
    def from_state(cls, state, stream=None, streams=None, sampler=None):
        p = state["params"]
        est = cls(p["run_seed"], p["sigma2"], p["ell"], p["M"], p["levels"], p["N_init"], p["eps"], p["theta"],
                  p["n0"], tuple(p["nu"]), p["rtol"], p["precision"], p["accel"], p["smoother"], p["max_batch"],
                  p["max_cycles"], stream, p["cost_model"], streams=streams, max_level=p["max_level"],
                  alpha=p["alpha"], alpha0=p["alpha0"], alpha_floor=p["alpha_floor"], cov=p["cov"], sampler=sampler)
        st = mg.AdaptiveState()
        for k, _ in mg.AdaptiveState._fields_:
            v = state["state"][k]
            if isinstance(v, list):
                arr = getattr(st, k)
                for i, x in enumerate(v):
                    arr[i] = x
            else:
                setattr(st, k, v)
        mg._check(mg.lib().mlmc_adaptive_set_state(est._h, ctypes.byref(st)), "mlmc_adaptive_set_state")
        est.log = list(state.get("log", []))
        return est

    @classmethod
    def restore(cls, path, stream=None, streams=None, sampler=None):
        with open(path) as fh:
            return cls.from_state(json.load(fh), stream, streams, sampler)

    # -- computation ---------------------------------------------------------------------
    def step(self) -> bool:
        """One round of Algorithm 2 (in the library); returns True when neither N_l nor L
        changed."""
        fin = ctypes.c_int()
        mg._check(mg.lib().mlmc_adaptive_step(self._h, ctypes.byref(fin)), "mlmc_adaptive_step")
        n = mg.lib().mlmc_adaptive_log_count(self._h)
        e = mg.AdaptiveRound()
        mg._check(mg.lib().mlmc_adaptive_log_get(self._h, n - 1, ctypes.byref(e)), "mlmc_adaptive_log_get")
        nl = e.L + 1
        self.log.append({"round": e.round, "levels": list(range(nl)), "have": list(e.have[:nl]),
                         "N_next": list(e.N_next[:nl]), "alpha": e.alpha, "bias": e.bias, "grow": bool(e.grow)})
        return bool(fin.value)

    def run(self, max_rounds=50):
        for _ in range(max_rounds):
            if self.step():
                break
        return self.result()

    def rates(self):
        """(alpha as the bias test uses it, beta, gamma); None where no fit exists."""
        s = self._summary()
        nan = lambda x: None if math.isnan(x) else x
        return s.alpha, nan(s.beta), nan(s.gamma)

    def result(self) -> dict:
        s = self._summary()
        nl = s.L + 1
        return {"Q_hat": s.Q_hat, "level_means": list(s.mean[:nl]), "level_vars": list(s.var[:nl]),
                "N": [int(x) for x in s.N[:nl]], "levels": list(range(nl)), "L": s.L,
                "sampling_var": s.sampling_var, "eps_s2": s.eps_s2,
                "cost_per_sample_s": [s.seconds[l] / max(int(s.N[l]), 1) for l in range(nl)],
                "rounds": s.rounds, "alpha": s.alpha, "beta": None if math.isnan(s.beta) else s.beta,
                "gamma": None if math.isnan(s.gamma) else s.gamma, "bias": s.bias, "bias_ok": bool(s.bias_ok)}
