"""Writes table7_oracle.json: the FP64 oracle's cycle counts for Sec. 6, Table 7 (V-cycle plus the
ray correction as a stand-alone solver, kh = 0.3125, centre source, relres 1e-7 from x = 0) for
HLM-V, SL-V and HYB-V at k = 20, 40, 80, 160, with the relative residual after every cycle, the solution on a
lattice of sampled nodes (every n/8-th node in each direction), and the paper's printed counts
beside them.

Everything computed here comes from ``oracle/`` alone (``helmholtz_matrix``, ``build_hierarchy``,
``ray_setup``, ``cycle_solve``) on the seeded inputs of ``paper_table7_workloads``; the benchmark
and the GPU tests read the file and never run this script (the k = 160 column takes about a minute
of oracle set-up per variant).

Usage: python tests/golden/make_table7_oracle.py
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as o  # noqa: E402
from paper_1312_2880_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(HERE, "table7_oracle.json")


def main():
    out = {"source": "Sec. 6, Table 7 (paper counts); oracle.cycle_solve with oracle.ray_setup (ours)",
           "tol": 1e-7, "columns": [], "paper": {v: list(c) for v, c in I.PAPER_TABLE7_CYCLES.items()}, "oracle": {}}
    for col, wl in I.paper_table7_workloads():
        A = o.helmholtz_matrix(wl.n, wl.kfield)
        t0 = time.time()
        ray = o.ray_setup(A, wl.n, wl.k_ref)
        out["columns"].append({"column": col, "k": wl.k_ref, "n": wl.n, "m": ray.m,
                               "ray_unknowns": int(ray.Ac.shape[0])})
        for variant in ("hlm", "sl", "hyb"):
            H = o.build_hierarchy(wl.n, wl.kfield, wl.k_ref, variant)
            res = o.cycle_solve(A, wl.rhs.ravel(), H, ray, tol=wl.tol, maxc=60)
            x = res.x.reshape(wl.n + 1, wl.n + 1)
            step = wl.n // 8
            samples = [[i, j, float(f"{x[j, i].real:.15e}"), float(f"{x[j, i].imag:.15e}")]
                       for j in range(0, wl.n + 1, step) for i in range(0, wl.n + 1, step)]
            out["oracle"].setdefault(variant, []).append({"cycles": res.cycles, "status": res.status,
                                                          "history": [float(f"{h:.12e}") for h in res.history],
                                                          "max_abs_x": float(np.abs(res.x).max()),
                                                          "sampled": samples})
            print(col, variant, res.cycles, res.status, f"{time.time() - t0:.1f}s", flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
