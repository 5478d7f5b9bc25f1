"""Write the sampled FP64-oracle reference of the full-size 3D sphere run.

The 200 x 100 x 100 shock-on-a-sphere workload (inflow beta_x = 0.5,
tau = 0.8, 5000 steps) costs the oracle about 1e10 cell updates, too long for
a test, so this script runs it once and stores the macroscopic fields at
sampled cells (seeded random fluid cells plus the x centre line through the
sphere) together with the oracle's run statistics.  It calls only ``oracle``
and ``workloads``; the oracle is bit-reproducible across platforms (binary64,
no contraction, sqrt only), so the stored values are what the oracle gives
anywhere.

    python tests/golden/make_sphere_golden.py [steps] [out.json]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def sample_cells(w, nrand=400, seed=11):
    rng = np.random.default_rng(seed)
    fluid = np.flatnonzero(w.solid.reshape(-1) == 0)
    pick = np.sort(rng.choice(fluid, size=nrand, replace=False))
    line = np.array([(50 * w.ny + 50) * w.nx + x for x in range(w.nx)])
    line = line[w.solid.reshape(-1)[line] == 0]
    return np.unique(np.concatenate([pick, line]))


def main():
    steps = int(sys.argv[1]) if len(sys.argv) > 1 else 5000
    out = sys.argv[2] if len(sys.argv) > 2 else os.path.join(os.path.dirname(__file__), f"sphere_fp64_{steps}.json")
    w = W.sphere_3d(steps=steps)
    p = oracle.Params(**w.params())
    st = oracle.init(p, w.n, w.eps, w.beta, w.solid)
    stats = oracle.Stats()
    t0 = time.time()
    oracle.run(p, st, steps, solid=w.solid, stats=stats)
    dt = time.time() - t0
    n, e, b, bad = oracle.macro(p, st, w.solid)
    cells = sample_cells(w)
    rec = {
        "_what": "FP64 oracle, sphere_3d workload (200x100x100, tau 0.8, beta_in 0.5, interior eps 1, n 0.3), "
                 "macroscopic fields at sampled cells after the given number of steps",
        "steps": steps,
        "oracle_seconds": dt,
        "oracle_threads": oracle.get_threads(),
        "stats": dict(n_unphysical=stats.n_unphysical, first_bad=stats.first_bad,
                      n_nonpositive_eq=stats.n_nonpositive_eq, macro_unphysical=bad),
        "cells": cells.tolist(),
        "n": n.reshape(-1)[cells].tolist(),
        "eps": e.reshape(-1)[cells].tolist(),
        "beta": [b[a].reshape(-1)[cells].tolist() for a in range(3)],
        "max_abs_beta": float(np.nanmax(np.abs(b))),
    }
    with open(out, "w") as fh:
        json.dump(rec, fh)
    print(f"wrote {out}: {len(cells)} cells, {dt:.0f} s, stats {rec['stats']}")


if __name__ == "__main__":
    main()
