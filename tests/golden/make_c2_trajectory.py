"""Writes c2_trajectory.json: the FP64 oracle's first time steps of the
100x100x10 workload (seeded layered lognormal permeability, 5-spot, 10-day
steps from the initial state, the schedule's controls and BHP limits), at
sampled cells.

    python tests/golden/make_c2_trajectory.py

Runs only the oracle (oracle.model.run, Newton to a scaled residual of 1e-10
with a direct sparse solve) on the seeded inputs of scenarios/; nothing here
comes from the CUDA path.  The cells: 400 seeded ones over the whole grid,
every cell within 4 cells of a corner injector column (where saturation and
polymer move first) and the 3x3 columns around the producer.  Each step
records the accepted sub-steps, the wells' switched flags, P, S, C at the
cells, every bottom-hole pressure and the max-norm of each field (the scale
of the 1e-6 comparison).  Takes about an hour and a half on one host core
(the first step alone needs 11 Newton iterations with a 100,000-cell direct
solve each).
"""

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import model as M  # noqa: E402
from scenarios import generate as G  # noqa: E402

N_STEPS = 3
OUT = os.path.join(HERE, "c2_trajectory.json")


def sample_cells(sc):
    nx, ny, nz = sc["nx"], sc["ny"], sc["nz"]
    rng = np.random.default_rng(2002)
    cells = set(int(c) for c in rng.choice(nx * ny * nz, 400, replace=False))
    for (i0, j0) in [(0, 0), (nx - 4, 0), (0, ny - 4), (nx - 4, ny - 4)]:
        for k in range(nz):
            for j in range(j0, j0 + 4):
                for i in range(i0, i0 + 4):
                    cells.add(i + nx * (j + ny * k))
    for k in range(nz):
        for j in range(ny // 2 - 1, ny // 2 + 2):
            for i in range(nx // 2 - 1, nx // 2 + 2):
                cells.add(i + nx * (j + ny * k))
    return sorted(cells)


def main():
    sc = G.scenario_c2()
    cells = sample_cells(sc)
    idx = np.asarray(cells)
    steps = []

    def record(st, x, h):
        n = st.n
        P, S, C = x[0:3 * n:3], x[1:3 * n:3], x[2:3 * n:3]
        steps.append({"t_days": h["t"] / G.DAY, "substeps_days": [d / G.DAY for d in h["substeps"]],
                      "newton": h["newton"], "cuts": h["cuts"], "switched": [bool(s) for s in h["switched"]],
                      "P": [float(v) for v in P[idx]], "S": [float(v) for v in S[idx]],
                      "C": [float(v) for v in C[idx]], "Pb": [float(v) for v in x[3 * n:]],
                      "max_abs": {"P": float(np.abs(P).max()), "S": float(np.abs(S).max()),
                                  "C": float(np.abs(C).max())}})
        print("step %d: t = %g d, %d Newton iterations, %d cuts" % (len(steps), h["t"] / G.DAY, h["newton"],
                                                                    h["cuts"]), flush=True)

    M.run(sc, n_steps=N_STEPS, callback=record)
    out = {"_source": "oracle.model.run on scenarios.generate.scenario_c2() (seed 2), written by "
                      "tests/golden/make_c2_trajectory.py; Newton tolerance 1e-10 (scaled residual)",
           "scenario": "scenario_c2", "newton_tol": 1e-10, "n_steps": N_STEPS, "cells": cells, "steps": steps}
    with open(OUT, "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print("wrote", OUT)


if __name__ == "__main__":
    main()
