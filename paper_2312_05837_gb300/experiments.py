"""The pruning experiment of Sec. IV-B (Table 1) on the GPU path: for
1000-spin 6-regular instances of the uniform, Gaussian and binary families,
domain selection with pruning (PDS: ising_solve) and without (DS:
ising_select_domain on the full instance); reports the pruning rate eta, the
solve times and chi_hat of both, and the gain Delta chi_hat = chi_hat_PDS -
chi_hat_DS (means and standard deviations over the trials). With
--converge each run stops by the Sec. IV-B rule (at most --steps steps) and
the iterations to convergence are reported, as in the table; otherwise each
run takes a fixed --steps steps.

    python -m paper_2312_05837_gb300.experiments table1 --trials 1000 --converge --steps 1000
"""

from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def table1_trial(ctx, inst, restarts: int, steps: int, seed: int, converge: bool = False) -> dict:
    """One instance: eta from the pruning, then PDS and DS with the same
    seed; energies are those of full spin vectors on the full instance. With
    the convergence rule, `iters` is the mean stopping step of the DS run's
    restarts (steps for a restart that never stops)."""
    import numpy as np
    from paper_2312_05837_gb300 import api
    from paper_2312_05837_gb300.metrics import chi_hat
    pr = api.prune(ctx, inst)
    eta = pr.eta
    pr.close()
    t0 = time.perf_counter()
    pds = api.solve(ctx, inst, restarts=restarts, steps=steps, seed=seed, converge=converge)
    t1 = time.perf_counter()
    s = api.Session(ctx, inst, restarts=restarts, steps=steps, seed=seed, converge=converge)
    s.run(steps)
    s.finish()
    ds = s.result()
    t2 = time.perf_counter()
    conv = s.convergence()
    s.close()
    iters = float(np.where(conv > 0, conv, steps).mean()) if converge else float(steps)
    c_pds = chi_hat(inst, pds["best_energy"])
    c_ds = chi_hat(inst, ds["best_energy"])
    return {"eta": eta, "T_pds": t1 - t0, "T_ds": t2 - t1, "chi_pds": c_pds, "chi_ds": c_ds,
            "d_chi": c_pds - c_ds, "E_pds": pds["best_energy"], "E_ds": ds["best_energy"],
            "iters": iters, "steps_run_ds": ds["steps_done"], "steps_run_pds": pds["steps_done"],
            "spins_pds": pds["best_spins"], "spins_ds": ds["best_spins"]}


def table1(ctx, dist: str, trials: int, restarts: int = 1, steps: int = 100,
           seed0: int = 0, converge: bool = False) -> dict:
    import numpy as np
    import synth
    rows = []
    for k in range(trials):
        inst = synth.table1_instance(dist, seed0 + k)
        r = table1_trial(ctx, inst, restarts, steps, seed=seed0 + k, converge=converge)
        rows.append({key: v for key, v in r.items() if not key.startswith("spins")})
    out = {"family": dist, "trials": trials, "restarts": restarts, "steps": steps,
           "converge": converge}
    for key in ["eta", "iters", "T_ds", "chi_ds", "T_pds", "chi_pds", "d_chi", "steps_run_ds",
                "steps_run_pds"]:
        v = np.array([r[key] for r in rows])
        out[key] = [float(v.mean()), float(v.std())]
    return out


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("experiment", choices=["table1"])
    ap.add_argument("--trials", type=int, default=1000)
    ap.add_argument("--restarts", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--families", default="uniform,gaussian,binary")
    ap.add_argument("--converge", action="store_true", help="stop each run by the Sec. IV-B rule")
    a = ap.parse_args()
    from paper_2312_05837_gb300 import api
    ctx = api.Context(0)
    for fam in a.families.split(","):
        print(json.dumps(table1(ctx, fam, a.trials, a.restarts, a.steps, converge=a.converge)),
              flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
