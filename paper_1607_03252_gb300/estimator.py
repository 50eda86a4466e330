"""Adaptive MLMC estimator (Algorithm 2 with a fixed number of levels) on the GPU
library, with checkpoint / resume.

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
"""
from __future__ import annotations

import json
import math
import threading
import time

from . import _capi as mg
from .stats import chan_merge, eps_split, sample_sizes
from .workloads import sample_id


class MLMCEstimator:
    def __init__(self, run_seed, sigma2, ell, M, levels, N_init, eps, theta=0.5, n0=17, nu=(2, 2), rtol=1e-10,
                 precision=mg.MLMC_PREC_F64, accel=mg.MLMC_ACCEL_NONE, smoother=mg.MLMC_SMOOTH_AUTO,
                 max_batch=0, max_cycles=300, stream=None, cost_model="measured", streams=None):
        if cost_model not in ("measured", "nodes"):
            raise ValueError("cost_model must be 'measured' or 'nodes'")
        self.params = dict(cost_model=cost_model, run_seed=int(run_seed), sigma2=float(sigma2), ell=float(ell), M=int(M),
                           levels=list(levels), N_init=list(N_init), eps=float(eps), theta=float(theta), n0=int(n0),
                           nu=list(nu), rtol=float(rtol), precision=int(precision), accel=int(accel),
                           smoother=int(smoother), max_batch=int(max_batch), max_cycles=int(max_cycles))
        self.stream = stream
        self.streams = list(streams) if streams else [stream]
        L = len(self.params["levels"])
        self.have = [0] * L
        self.records = [(0.0, 0.0, 0.0)] * L
        self.seconds = [0.0] * L
        self.target = list(self.params["N_init"])
        self.rounds = 0
        self.log = []

    # -- state ------------------------------------------------------------------------
    def state(self) -> dict:
        return {"params": self.params, "have": self.have, "records": [list(r) for r in self.records],
                "seconds": self.seconds, "target": self.target, "rounds": self.rounds, "log": self.log}

    def checkpoint(self, path):
        with open(path, "w") as fh:
            json.dump(self.state(), fh)

    @classmethod
    def from_state(cls, state, stream=None):
        p = state["params"]
        est = cls(p["run_seed"], p["sigma2"], p["ell"], p["M"], p["levels"], p["N_init"], p["eps"], p["theta"],
                  p["n0"], tuple(p["nu"]), p["rtol"], p["precision"], p["accel"], p["smoother"], p["max_batch"],
                  p["max_cycles"], stream, p.get("cost_model", "measured"))
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
                                smoother=p["smoother"],
                                accel=p["accel"])

    def add_samples(self, i, count, stream=None):
        """Computes samples have[i] .. have[i] + count - 1 of level levels[i]."""
        if count <= 0:
            return
        level = self.params["levels"][i]
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
            for l in self.params["levels"]:
                nf = (n0 - 1) * 2 ** l + 1
                nc = (n0 - 1) * 2 ** (l - 1) + 1 if l > 0 else 0
                out.append(float(nf ** 3 + nc ** 3))
            return out
        return [self.seconds[i] / self.have[i] for i in range(len(self.have))]

    def _node_cost(self, i):
        n0, l = self.params["n0"], self.params["levels"][i]
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

    def step(self) -> bool:
        """One round of Algorithm 2; returns True when no level needs more samples."""
        self.rounds += 1
        self._add_round()
        V = self.variances()
        C = self.costs()
        eps_s, _ = eps_split(self.params["eps"], self.params["theta"])
        need = sample_sizes([max(v, 1e-30) for v in V], C, eps_s)
        self.log.append({"round": self.rounds, "have": list(self.have), "N_next": need})
        if all(nn <= h for nn, h in zip(need, self.have)):
            return True
        self.target = [max(a, b) for a, b in zip(self.target, need)]
        return False

    def run(self, max_rounds=50):
        for _ in range(max_rounds):
            if self.step():
                break
        return self.result()

    def result(self) -> dict:
        V = self.variances()
        means = [r[1] for r in self.records]
        eps_s, _ = eps_split(self.params["eps"], self.params["theta"])
        return {"Q_hat": math.fsum(means), "level_means": means, "level_vars": V, "N": list(self.have),
                "sampling_var": math.fsum(v / max(h, 1) for v, h in zip(V, self.have)), "eps_s2": eps_s ** 2,
                "cost_per_sample_s": [self.seconds[i] / max(self.have[i], 1) for i in range(len(self.have))],
                "rounds": self.rounds}
