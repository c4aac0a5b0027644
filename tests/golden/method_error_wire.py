"""Method error of P-AIM (O2) against the direct definition (O1) on the benchmark's wire geometry.

Writes ``method_error_wire.json`` beside this file.  Calls only the oracle (and ``meshgen``
for the seeded input), never the CUDA path.

Workload: the 1D-periodic protruding wire of the benchmark (period 100 nm along z, radius
20 nm, 8 seeded bumps, shear 0.15, seed 0) at 1/64 of its node count, with the benchmark's
grid scaled by 1/4 per axis (128 x 128 x 256 -> 32 x 32 x 64), so that the number of nodes
per grid cell, which sets the P-AIM error, is the benchmark's.  O1 is evaluated at a seeded
subsample of unknowns and their adjacency neighbours (the gradient of Eq. 14d at a sampled
unknown needs the potential on its 1-ring).

Reported, each as a relative L2 error over the sampled unknowns (all three components):
  * O2 against O1 with the same near-element radius: the error of the BAIM steps alone
    (grid, stencil and box-near precorrection of Sec. 3.2), for near_boxes 1..4, at the
    scaled grid and at a grid twice as fine, for the random m of the parity tests and the
    vortex m of the benchmark;
  * O2 with near_elem_factor 0 (touching elements only) and 1 (elements whose centroid lies
    within one mean edge: the "tetrahedron size" radius of Sec. 3.2) against O1 with factor
    2, the closest to the continuous potential that this study computes;
  * precorrection entries per row for each setting (they set the bytes of BAIM step 4).

Run:  python tests/golden/method_error_wire.py  [--nodes N] [--samples S]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import meshgen                                   # noqa: E402
from oracle.direct import potential_direct       # noqa: E402
from oracle.problem import OracleProblem         # noqa: E402
from oracle.topology import pair_nodes           # noqa: E402

WIRE = dict(L=100e-9, R=20e-9, seed=0)
BENCH_NODES, BENCH_GRID = 1_000_000, (128, 128, 256)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nodes", type=int, default=BENCH_NODES // 64)
    ap.add_argument("--samples", type=int, default=300)
    ap.add_argument("--out", default=os.path.join(HERE, "method_error_wire.json"))
    a = ap.parse_args()
    scale = round((BENCH_NODES / a.nodes) ** (1 / 3))
    grid = tuple(n // scale for n in BENCH_GRID)
    fine = tuple(2 * n for n in grid)
    t0 = time.time()
    mesh = meshgen.wire_cell(L=WIRE["L"], R=WIRE["R"], target_nodes=a.nodes, seed=WIRE["seed"])
    lca, roots = pair_nodes(mesh.xyz, mesh.periods)
    Np = int(roots.size)
    rng = np.random.default_rng(2)
    sample = np.sort(rng.choice(Np, size=min(a.samples, Np), replace=False))
    touch = np.isin(lca[mesh.tets], sample).any(axis=1)
    obs = np.unique(lca[mesh.tets[touch]])
    where = np.searchsorted(obs, sample)

    def problem(**kw):
        return OracleProblem(mesh.xyz, mesh.tets, mesh.periods, Ms=8e5, A=1.3e-11, alpha=0.02,
                             observers=obs, **kw)

    base = problem()
    ms = {"random": meshgen.m_random(Np, seed=3), "vortex": meshgen.m_vortex(base.pos_f, core=5e-9)}
    q = np.stack([base.charges(m) for m in ms.values()], 1)
    # O1 point-charge lattice sums at the observers, shared by every near-element radius
    u_pt = potential_direct(base.pos_f, q, base.periods, None, obs, eta=base.eta)
    t_o1 = time.time() - t0

    def h_at_samples(ob, u_obs):
        u = np.zeros(Np)
        u[obs] = u_obs
        return ob.h_ms_from_potential(u)[sample]

    out = {"workload": "wire-1d-periodic-protruding", "nodes": int(mesh.xyz.shape[0]), "unknowns": Np,
           "grid": list(grid), "fine_grid": list(fine), "bench_nodes": BENCH_NODES, "bench_grid": list(BENCH_GRID),
           "samples": int(sample.size), "observers": int(obs.size), "p": 3, "o1": {}, "o2": []}
    H1 = {}
    for f in (0.0, 1.0, 2.0):
        ob = base if f == 0.0 else problem(near_elem_factor=f)
        for i, (name, m) in enumerate(ms.items()):
            H1[(f, name)] = h_at_samples(ob, u_pt[:, i] + ob.EM(m)[obs])
    for name in ms:
        out["o1"][name] = {"factor0_vs_factor2": rel(H1[(0.0, name)], H1[(2.0, name)]),
                           "factor1_vs_factor2": rel(H1[(1.0, name)], H1[(2.0, name)])}
    for g in (grid, fine):
        for f in (0.0, 1.0):
            for nb in (1, 2, 3, 4):
                ob = problem(grid=g, p=3, near_boxes=nb, near_elem_factor=f)
                rec = {"grid": list(g), "near_boxes": nb, "near_elem_factor": f,
                       "precorrection_entries_per_row": float(ob.C.nnz / obs.size)}
                for name, m in ms.items():
                    H2 = ob.h_ms(m, "paim")[sample]
                    rec[f"{name}_vs_O1_same_factor"] = rel(H2, H1[(f, name)])
                    rec[f"{name}_vs_O1_factor2"] = rel(H2, H1[(2.0, name)])
                out["o2"].append(rec)
                print(json.dumps(rec), flush=True)
    out["o1_seconds"] = round(t_o1, 1)
    out["total_seconds"] = round(time.time() - t0, 1)
    with open(a.out, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out["o1"]))


if __name__ == "__main__":
    main()
