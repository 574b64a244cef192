"""Write tests/golden/fullsize_bounds.json: the oracle's bounds for the full-size workloads.

Calls only oracle/ (and the seeded input generators in microstructures/):
  * cube3d_N41        3D cube cell N = 41^3 (double grid 81^3), contrast 100: O2 (matrix
                      DFTs + CG), tol 1e-10;
  * spheres3d_N113    3D cell with 16 random balls (seed 0), volume fraction 0.3, contrast
                      1000, N = 113^3 (double grid 225^3): O3 (library FFTs + the same CG),
                      tol 1e-8 (O3 = O2 is pinned by tests/test_oracle_o3_pins.py);
  * rects2d_seed{2,6,5,10}  cells of the 256-cell random-rectangle batch with N = 113 (seeds
                      2, 6) and N = 203 (seeds 5, 10): O2, tol 1e-10.
With the CG residual r below tol ||E||, the energy error of a side is r.C^{-1}r <=
tol^2 / lambda_min(C), lambda_min >= a_min (primal) or 1/a_max (dual), so these tolerances
put every stored bound within 1e-10 relative of the exact Galerkin bound.

Usage: python tests/golden/make_fullsize_goldens.py [--only NAME ...] [--workers K]
Entries are merged into the existing file, so long entries can be made one at a time.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "fullsize_bounds.json")


def entries():
    import microstructures as ms
    e = {
        "cube3d_N41": (lambda: ms.cube_inclusion_3d(), "O2", 1e-10,
                       "3D cube cell N=41^3 (double grid 81^3), side 0.5, a = 1 / 100"),
        "spheres3d_N113": (lambda: ms.random_spheres_3d(0, N=113), "O3", 1e-8,
                           "3D cell, 16 random balls (seed 0), volume fraction 0.3, contrast 1000, "
                           "N=113^3 (double grid 225^3)"),
    }
    for s in (2, 6, 5, 10):
        e[f"rects2d_seed{s}"] = (lambda s=s: ms.random_rectangles_2d(s), "O2", 1e-10,
                                 f"random-rectangle cell of the 256-cell batch, seed {s}")
    return e


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", nargs="*", default=None)
    ap.add_argument("--workers", type=int, default=None)
    args = ap.parse_args()
    from oracle import fftcg, matfree
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name, (make, which, tol, desc) in entries().items():
        if args.only and name not in args.only:
            continue
        p = make()
        t = time.time()
        if which == "O2":
            out = matfree.matfree_bounds(p, tol=tol)
            out["history_primal"] = out["history_dual"] = None
        else:
            out = fftcg.fft_bounds(p, tol=tol, workers=args.workers,
                                   log=lambda m: print(f"  {name}: {m} ({time.time() - t:.0f} s)", flush=True))
        data[name] = {"workload": desc, "oracle": which, "tol": tol, "N": [int(n) for n in p.N],
                      "upper": out["upper"].tolist(), "lower": out["lower"].tolist(),
                      "iters_primal": [int(i) for i in out["iters_primal"]],
                      "iters_dual": [int(i) for i in out["iters_dual"]], "seconds": round(time.time() - t, 1)}
        if out["history_primal"] is not None:
            # CG iterations each solve needed to reach a relative residual of 1e-4 (the same
            # CG run, read off its residual history)
            data[name]["iters_to_1e-4"] = [[next(i for i, r in enumerate(h) if r <= 1e-4) for h in out[k]]
                                           for k in ("history_primal", "history_dual")]
        print(name, json.dumps(data[name]), flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
            f.write("\n")


if __name__ == "__main__":
    main()
