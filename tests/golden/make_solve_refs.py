"""Writes tests/golden/solve_refs.json: MBAR free energies computed by the
CPU oracle alone, for problems whose oracle solve takes too long to repeat
inside the GPU tests (minutes for the K = 500 alchemical case).

Every input is drawn by the seeded generators of
paper_2609_03541_b300/workloads.py from the (kind, sizes, seed) stored next
to the result, so the GPU test rebuilds the same u_kn. The stored f is the
unique MBAR root (gauge f_0 = 0; Eq. 1 at its unbinned fixed point, Sec. II)
as oracle.solve_mbar defines it; each entry also records the smallest
eigenvalue of the oracle's gauge-reduced Hessian there (how poorly the
states overlap, which sets how far rounding in a gradient moves the root).

Run from the repository root:  python tests/golden/make_solve_refs.py
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2609_03541_b300 import workloads as W  # noqa: E402

# (name, kind, generator arguments); the batched workload's problem types
# (harmonic d = 3 and umbrella windows, K from 4 to 256) and the default
# benchmark's shapes at a reduced sample count
CASES = [
    ("umbrella_K4_s0", "umbrella", dict(K=4, N_k=4299, seed=0)),
    ("umbrella_K4_s1", "umbrella", dict(K=4, N_k=4299, seed=1)),
    ("umbrella_K4_s2", "umbrella", dict(K=4, N_k=4299, seed=2)),
    ("umbrella_K4_s4", "umbrella", dict(K=4, N_k=4299, seed=4)),
    ("umbrella_K4_s7", "umbrella", dict(K=4, N_k=4299, seed=7)),
    ("umbrella_K9", "umbrella", dict(K=9, N_k=1500, seed=9)),
    ("umbrella_K17", "umbrella", dict(K=17, N_k=800, seed=17)),
    ("umbrella_K64", "umbrella", dict(K=64, N_k=300, seed=64)),
    ("umbrella_K256", "umbrella", dict(K=256, N_k=100, seed=256)),
    ("harmonic_K4", "harmonic", dict(K=4, N_k=3000, seed=4)),
    ("harmonic_K33", "harmonic", dict(K=33, N_k=600, seed=33)),
    ("harmonic_K130", "harmonic", dict(K=130, N_k=150, seed=130)),
    ("harmonic_K256", "harmonic", dict(K=256, N_k=100, seed=256)),
    ("alchemical_K500", "alchemical", dict(K=500, N_k=20, seed=6)),
    ("tempering_K50", "parallel_tempering", dict(K=50, N_k=2000, seed=3)),
]


def make(kind: str, args: dict) -> W.Problem:
    if kind == "umbrella":
        return W.umbrella(grid_points=1 << 13, **args)
    if kind == "harmonic":
        return W.harmonic(d=3, **args)
    if kind == "alchemical":
        return W.alchemical(**args)
    if kind == "parallel_tempering":
        return W.parallel_tempering(**args)
    raise ValueError(kind)


def main() -> None:
    out = {
        "citation": "Eq. 1 at its unbinned fixed point (Sec. II: the limit of one sample per bin is UWHAM = MBAR, "
                    "which BU-MBAR reaches at the end of Algorithm 1 and its derivative-based finish); gauge f_0 = 0. "
                    "Values from oracle.solve_mbar on inputs rebuilt from workloads.py by (kind, args).",
        "cases": [],
    }
    for name, kind, args in CASES:
        p = make(kind, args)
        t0 = time.time()
        f = O.solve_mbar(p.u_kn, p.N_k)
        lam = float(np.linalg.eigvalsh(O.mbar_hessian(p.u_kn, f, p.N_k)[1:, 1:]).min())
        gmax = float(np.max(np.abs(O.mbar_gradient(p.u_kn, f, p.N_k))))
        out["cases"].append(dict(name=name, kind=kind, args=args, f=[float(x) for x in f], lambda_min=lam,
                                 max_abs_gradient=gmax))
        print(f"{name}: {time.time() - t0:.1f} s, lambda_min {lam:.3g}, max|g| {gmax:.2e}", flush=True)
    with open(os.path.join(HERE, "solve_refs.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
