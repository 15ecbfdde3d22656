"""Writes grf_n4096_k1000_oracle.json: the FP64 oracle's own solve of the n = 4096, k = 1000
random-field workload (k (1 + 0.3 g), centre source 1/h^2, HYB-V, 10 levels, Bi-CGSTAB to relres
1e-6, Sec. 5-6), sampled on a coarse lattice of nodes.

The oracle needs hours for this solve on one host core, so the sampled solution is stored once and
read by the GPU tests and the benchmark (which compare against it; they never run this script).
Everything written here comes from ``oracle/`` alone: the workload's inputs from the seeded
generators, the solution from ``oracle.build_hierarchy`` / ``oracle.vcycle`` / ``oracle.bicgstab``.

Usage: python tests/golden/make_grf4096_oracle.py [--save-x PATH.npy]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as o  # noqa: E402
from paper_1312_2880_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(HERE, "grf_n4096_k1000_oracle.json")
STRIDE = 128  # lattice of sampled nodes: every STRIDE-th node in each direction
WINDOW = 4  # plus the (2 WINDOW + 1)^2 nodes around the source


def sample_nodes(n: int):
    """The sampled nodes (i, j): the lattice, then the window around the centre source."""
    nodes = [(i, j) for j in range(0, n + 1, STRIDE) for i in range(0, n + 1, STRIDE)]
    c = n // 2
    nodes += [(i, j) for j in range(c - WINDOW, c + WINDOW + 1) for i in range(c - WINDOW, c + WINDOW + 1)
              if (i % STRIDE, j % STRIDE) != (0, 0)]
    return nodes


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--save-x", default=None, help="also save the whole solution (complex128 .npy)")
    ap.add_argument("--maxit", type=int, default=3000)
    args = ap.parse_args()
    wl = I.grf_n4096()
    n = wl.n
    t0 = time.time()
    A = o.helmholtz_matrix(n, wl.kfield)
    H = o.build_hierarchy(n, wl.kfield, wl.k_ref, wl.variant, wl.levels)
    t_setup = time.time() - t0
    b = wl.rhs.ravel()
    t0 = time.time()
    res = o.bicgstab(A, b, lambda v: o.vcycle(H, v), tol=wl.tol, maxit=args.maxit)
    t_solve = time.time() - t0
    x = res.x.reshape(n + 1, n + 1)
    if args.save_x:
        np.save(args.save_x, x)
    amax = int(np.argmax(np.abs(x)))
    out = {
        "workload": wl.name, "n": n, "k": wl.k_ref, "levels": wl.levels, "variant": wl.variant, "tol": wl.tol,
        "schedule": [[lv.n, lv.relax_op, lv.smoother, lv.resid_op] for lv in H.levels],
        "iterations": res.iterations, "status": res.status, "true_relres": res.true_relres,
        "history_len": len(res.history), "max_abs_x": float(np.abs(x).max()),
        "argmax_node": [amax % (n + 1), amax // (n + 1)], "norm2_x": float(np.linalg.norm(x)),
        "setup_s": round(t_setup, 1), "solve_s": round(t_solve, 1),
        "sampled": [[i, j, float(x[j, i].real), float(x[j, i].imag)] for i, j in sample_nodes(n)],
    }
    with open(OUT, "w") as fh:
        json.dump(out, fh)
    print(json.dumps({k: v for k, v in out.items() if k != "sampled"}))


if __name__ == "__main__":
    main()
