"""Writes tests/golden/workload_sizes.json: the FP64 oracle's values for one sample of the
two largest workload levels, for the GPU parity test at full size.

  - the mixed-precision 5-level workload's finest level (level 4: 257^3 fine, 129^3 coarse;
    sigma^2 = 2, ell = 0.1, M = 256), realisation id sample_id(4, 0);
  - the large adaptive workload's finest level (level 5: 513^3 fine, 257^3 coarse;
    sigma^2 = 1, ell = 0.05, M = 1024), realisation id sample_id(5, 0).

Both solves of each pair run the oracle's V(2,2) cycle (Sec. 2.2, Eq. 8: Y = Q_l - Q_{l-1} on
one realisation) to a relative residual just above the FP64 rounding floor of the grid:
1e-11 at 257^3 (the oracle's residual stalls near 7e-12 there on this field, 1.7e-12 at
129^3) and 1e-10 at 513^3. Only the oracle is called; nothing here comes from the CUDA
path. Run from the repository root:

    python tests/golden/make_workload_golden.py

(about 25 minutes on 8 cores; the oracle's independent plane loops use all OpenMP threads).
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1607_03252_gb300.workloads import RUN_SEED, level_n, sample_id  # noqa: E402

CASES = [
    dict(name="mixed5_level4", level=4, sigma2=2.0, ell=0.1, M=256, rtol=1e-11),
    dict(name="adaptive6_level5", level=5, sigma2=1.0, ell=0.05, M=1024, rtol=1e-10),
]
MAX_CYCLES = 400


def main():
    out = {"script": "tests/golden/make_workload_golden.py", "run_seed": RUN_SEED, "cycle": "V(2,2)", "cases": []}
    for c in CASES:
        sid = sample_id(c["level"], 0)
        cfg = oracle.make_cfg(RUN_SEED, c["sigma2"], c["ell"], c["M"], rtol=c["rtol"], max_cycles=MAX_CYCLES)
        t = time.perf_counter()
        st, qf, qc, cf, cc = oracle.sample(cfg, level_n(c["level"]), level_n(c["level"] - 1), sid)
        if st != 0:
            raise SystemExit("oracle status %d for %s" % (st, c["name"]))
        rec = dict(c, sample_id=sid, n_fine=level_n(c["level"]), n_coarse=level_n(c["level"] - 1), Qf=qf, Qc=qc,
                   Y=qf - qc, cycles_fine=cf, cycles_coarse=cc, oracle_seconds=round(time.perf_counter() - t, 1))
        print(json.dumps(rec), flush=True)
        out["cases"].append(rec)
    with open(os.path.join(ROOT, "tests", "golden", "workload_sizes.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
