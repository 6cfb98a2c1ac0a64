"""Runs a domain-selection session on a named synthetic workload with the
step kernels timed launch by launch (ISING_DS_PROFILE) — the driver used for
the ncu captures summarised under profiles/.

    python -m paper_2312_05837_gb300.profile_step er2000 --restarts 1024 --steps 30
"""

from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--restarts", type=int, default=1024)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--precision", default="auto")
    ap.add_argument("--trace", action="store_true", help="print the per-CTA role timeline")
    ap.add_argument("--resident-trace", action="store_true",
                    help="label the timeline with the resident form's slots")
    a = ap.parse_args()
    import numpy as np
    import synth
    from paper_2312_05837_gb300 import api
    inst = synth.workload(a.workload, 0)
    ctx = api.Context(0)
    s = api.Session(ctx, inst, restarts=a.restarts, steps=a.steps, seed=1,
                    precision=a.precision, profile=True)
    s.run(a.steps)
    r = s.result()
    print(f"{a.workload} n={inst.n} B={a.restarts} steps={a.steps} path={r['path']} "
          f"precision={r['precision']} step kernel {1e3 * r['kernel_ms'] / max(r['kernel_launches'], 1):.2f} us/launch")
    if a.trace:
        tr = s.trace().astype(np.int64)
        if tr.size:
            rel = (tr - tr[:, 0].min()) / 1e3
            names = (["step_start", "tma_last", "mma_last", "tracked", "epi_acc", "epi_done",
                      "ctl_done", "barrier"] if a.resident_trace else
                     ["start", "tma_first", "tma_last", "mma_first", "mma_last", "epi_acc",
                      "epi_done", "end"])
            for k, nm in enumerate(names):
                print(f"  {nm:10s} median {np.median(rel[:, k]):8.2f} us  max {rel[:, k].max():8.2f} us")
    s.close()
    ctx.close()


if __name__ == "__main__":
    main()
