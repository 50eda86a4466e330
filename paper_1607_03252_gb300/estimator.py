"""Adaptive MLMC estimator (Algorithm 2) on the GPU library, with checkpoint / resume.

Each round computes the missing samples of every level (Algorithm 2, step 2.a) through
`mlmc_level_estimate`, folds their (N, mean, M2) records into the level's running record
(Chan's merge, Sec. 2.3's Y-hat_l and s_l^2), estimates the cost per sample C_l (measured
wall time, or the deterministic node-count model), and sizes
N_l by Eq. 15 for eps_s^2 = theta eps^2 (Eq. 6); it stops when no level needs more samples
(step 4). Sample ids of level l are sample_id(l, 0), sample_id(l, 1), ... in order, so a
run restored from `state()` continues with exactly the ids an uninterrupted run would use
and ends with the same records. With several `streams`, the levels of a round run
concurrently (one host thread and one stream per lane, levels assigned longest first by
their node count); a level's records do not depend on that.

With `max_level` set, the number of levels adapts too (Algorithm 2, step 3): after each
round the bias estimate of Eq. 14, |Y-hat_L| / (8^alpha - 1), is compared with eps_b
(Eq. 6), and while it is larger and L < max_level the next level joins with N_init samples.
alpha is given, or fitted online from the level means l >= 1 (least squares of
log_8 |Y-hat_l| against l, M_l ~ 8^l; `alpha0` until two such levels exist, never below
`alpha_floor`). The rates beta (variances) and gamma (costs) of Eq. 12 are fitted the same
way and reported.
"""
from __future__ import annotations

import json
import math
import threading
import time

from . import _capi as mg
from .stats import chan_merge, eps_split, fit_rate, sample_sizes
from .workloads import sample_id


class MLMCEstimator:
    def __init__(self, run_seed, sigma2, ell, M, levels, N_init, eps, theta=0.5, n0=17, nu=(2, 2), rtol=1e-10,
                 precision=mg.MLMC_PREC_F64, accel=mg.MLMC_ACCEL_NONE, smoother=mg.MLMC_SMOOTH_AUTO,
                 max_batch=0, max_cycles=300, stream=None, cost_model="measured", streams=None, max_level=None,
                 alpha=None, alpha0=2.0 / 3.0, alpha_floor=0.1, cov=mg.MLMC_COV_GAUSS):
        if cost_model not in ("measured", "nodes"):
            raise ValueError("cost_model must be 'measured' or 'nodes'")
        levels = list(levels)
        if isinstance(N_init, int):
            N_init = [N_init] * len(levels)
        if len(N_init) != len(levels):
            raise ValueError("N_init needs one count per level")
        if max_level is not None and (levels != list(range(len(levels))) or len(levels) < 2 or max_level < levels[-1]):
            raise ValueError("level growth starts from levels 0..L (L >= 1) with L <= max_level")
        self.params = dict(cost_model=cost_model, run_seed=int(run_seed), sigma2=float(sigma2), ell=float(ell), M=int(M),
                           levels=levels, N_init=list(N_init), eps=float(eps), theta=float(theta), n0=int(n0),
                           nu=list(nu), rtol=float(rtol), precision=int(precision), accel=int(accel),
                           smoother=int(smoother), max_batch=int(max_batch), max_cycles=int(max_cycles),
                           max_level=None if max_level is None else int(max_level),
                           alpha=None if alpha is None else float(alpha), alpha0=float(alpha0),
                           alpha_floor=float(alpha_floor), cov=int(cov))
        self.stream = stream
        self.streams = list(streams) if streams else [stream]
        self.levels = list(levels)
        L = len(self.levels)
        self.have = [0] * L
        self.records = [(0.0, 0.0, 0.0)] * L
        self.seconds = [0.0] * L
        self.target = list(self.params["N_init"])
        self.rounds = 0
        self.log = []

    # -- state ------------------------------------------------------------------------
    def state(self) -> dict:
        return {"params": self.params, "levels": self.levels, "have": self.have,
                "records": [list(r) for r in self.records],
                "seconds": self.seconds, "target": self.target, "rounds": self.rounds, "log": self.log}

    def checkpoint(self, path):
        with open(path, "w") as fh:
            json.dump(self.state(), fh)

    @classmethod
    def from_state(cls, state, stream=None):
        p = state["params"]
        est = cls(p["run_seed"], p["sigma2"], p["ell"], p["M"], p["levels"], p["N_init"], p["eps"], p["theta"],
                  p["n0"], tuple(p["nu"]), p["rtol"], p["precision"], p["accel"], p["smoother"], p["max_batch"],
                  p["max_cycles"], stream, p.get("cost_model", "measured"), max_level=p.get("max_level"),
                  alpha=p.get("alpha"), alpha0=p.get("alpha0", 2.0 / 3.0), alpha_floor=p.get("alpha_floor", 0.1),
                  cov=p.get("cov", mg.MLMC_COV_GAUSS))
        est.levels = list(state.get("levels", p["levels"]))
        est.have = list(state["have"])
        est.records = [tuple(r) for r in state["records"]]
        est.seconds = list(state["seconds"])
        est.target = list(state["target"])
        est.rounds = int(state["rounds"])
        est.log = list(state["log"])
        return est

    @classmethod
    def restore(cls, path, stream=None):
        with open(path) as fh:
            return cls.from_state(json.load(fh), stream)

    # -- computation --------------------------------------------------------------------
    def _cfg(self, stream=None):
        p = self.params
        return mg.make_mlmc_cfg(p["run_seed"], p["sigma2"], p["ell"], p["M"], n0=p["n0"], nu1=p["nu"][0],
                                nu2=p["nu"][1], rtol=p["rtol"], max_cycles=p["max_cycles"], precision=p["precision"],
                                max_batch=p["max_batch"], stream=stream if stream is not None else self.stream,
                                smoother=p["smoother"], accel=p["accel"], cov=p["cov"])

    def add_samples(self, i, count, stream=None):
        """Computes samples have[i] .. have[i] + count - 1 of level levels[i]."""
        if count <= 0:
            return
        level = self.levels[i]
        t = time.perf_counter()
        st, _, _, _ = mg.mlmc_level_estimate(self._cfg(stream), level, sample_id(level, self.have[i]), count,
                                             want_samples=False)
        self.seconds[i] += time.perf_counter() - t
        self.records[i] = chan_merge([self.records[i], (float(st.N), st.mean, st.M2)])
        self.have[i] += count

    def variances(self):
        return [r[2] / (r[0] - 1.0) if r[0] > 1 else 0.0 for r in self.records]

    def costs(self):
        """C_l: measured seconds per sample, or the model cost n_l^3 + n_{l-1}^3 (nodes of
        the fine and coarse grid, deterministic)."""
        if self.params["cost_model"] == "nodes":
            n0 = self.params["n0"]
            out = []
            for l in self.levels:
                nf = (n0 - 1) * 2 ** l + 1
                nc = (n0 - 1) * 2 ** (l - 1) + 1 if l > 0 else 0
                out.append(float(nf ** 3 + nc ** 3))
            return out
        return [self.seconds[i] / self.have[i] for i in range(len(self.have))]

    def _node_cost(self, i):
        n0, l = self.params["n0"], self.levels[i]
        nf = (n0 - 1) * 2 ** l + 1
        nc = (n0 - 1) * 2 ** (l - 1) + 1 if l > 0 else 0
        return float(nf ** 3 + nc ** 3)

    def _add_round(self):
        todo = [(i, self.target[i] - self.have[i]) for i in range(len(self.have)) if self.target[i] > self.have[i]]
        if len(self.streams) <= 1 or len(todo) <= 1:
            for i, c in todo:
                self.add_samples(i, c, self.streams[0])
            return
        loads = [0.0] * len(self.streams)
        lanes = [[] for _ in self.streams]
        for i, c in sorted(todo, key=lambda t: -t[1] * self._node_cost(t[0])):
            k = min(range(len(lanes)), key=lambda j: loads[j])
            lanes[k].append((i, c))
            loads[k] += c * self._node_cost(i)
        errors = []

        def run(k):
            try:
                for i, c in lanes[k]:
                    self.add_samples(i, c, self.streams[k])
            except BaseException as e:  # re-raised on the calling thread
                errors.append(e)

        threads = [threading.Thread(target=run, args=(k,)) for k in range(1, len(lanes)) if lanes[k]]
        for t in threads:
            t.start()
        run(0)
        for t in threads:
            t.join()
        if errors:
            raise errors[0]

    def rates(self):
        """(alpha, beta, gamma) of Eqs. 12 and 14 fitted over the levels l >= 1 with
        samples (None where fewer than two such levels exist); alpha as the bias test
        uses it (given, else fitted, else alpha0; at least alpha_floor)."""
        p = self.params
        idx = [i for i, l in enumerate(self.levels) if l >= 1 and self.have[i] > 0]
        ls = [self.levels[i] for i in idx]
        V, C = self.variances(), self.costs() if self.have and min(self.have) > 0 else None
        fit_a = fit_rate(ls, [self.records[i][1] for i in idx])
        beta = fit_rate(ls, [V[i] for i in idx]) if all(V[i] > 0 for i in idx) else None
        gamma = None
        if C is not None and all(C[i] > 0 for i in idx):
            g = fit_rate(ls, [C[i] for i in idx])
            gamma = -g if g is not None else None
        if p["alpha"] is not None:
            alpha = p["alpha"]
        else:
            alpha = max(fit_a if fit_a is not None else p["alpha0"], p["alpha_floor"])
        return alpha, beta, gamma

    def bias_estimate(self):
        """|Y-hat_L| / (8^alpha - 1) (Eq. 14)."""
        alpha = self.rates()[0]
        return abs(self.records[-1][1]) / (8.0 ** alpha - 1.0)

    def step(self) -> bool:
        """One round of Algorithm 2; returns True when neither N_l nor L changes."""
        p = self.params
        self.rounds += 1
        self._add_round()
        V = self.variances()
        C = self.costs()
        eps_s, eps_b = eps_split(p["eps"], p["theta"])
        need = sample_sizes([max(v, 1e-30) for v in V], C, eps_s)
        grow = False
        entry = {"round": self.rounds, "levels": list(self.levels), "have": list(self.have), "N_next": need}
        if p["max_level"] is not None:
            bias = self.bias_estimate()
            grow = bias > eps_b and self.levels[-1] < p["max_level"]
            entry.update(alpha=self.rates()[0], bias=bias, grow=grow)
        self.log.append(entry)
        if not grow and all(nn <= h for nn, h in zip(need, self.have)):
            return True
        self.target = [max(a, b) for a, b in zip(self.target, need)]
        if grow:
            self.levels.append(self.levels[-1] + 1)
            self.have.append(0)
            self.records.append((0.0, 0.0, 0.0))
            self.seconds.append(0.0)
            self.target.append(p["N_init"][-1])
        return False

    def run(self, max_rounds=50):
        for _ in range(max_rounds):
            if self.step():
                break
        return self.result()

    def result(self) -> dict:
        V = self.variances()
        means = [r[1] for r in self.records]
        eps_s, eps_b = eps_split(self.params["eps"], self.params["theta"])
        alpha, beta, gamma = self.rates()
        bias = abs(means[-1]) / (8.0 ** alpha - 1.0)
        return {"Q_hat": math.fsum(means), "level_means": means, "level_vars": V, "N": list(self.have),
                "levels": list(self.levels), "L": self.levels[-1],
                "sampling_var": math.fsum(v / max(h, 1) for v, h in zip(V, self.have)), "eps_s2": eps_s ** 2,
                "cost_per_sample_s": [self.seconds[i] / max(self.have[i], 1) for i in range(len(self.have))],
                "rounds": self.rounds, "alpha": alpha, "beta": beta, "gamma": gamma, "bias": bias,
                "bias_ok": bias <= eps_b}
