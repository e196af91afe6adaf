"""Count study in the manner of the paper's Sec. 4 on 25 x 25 stand-ins.

The paper compares the source orders by the number of propagations needed
to fill the array and reports relative differences Delta_r(X) = (P_X -
P_method) / P_X against the naive and the spiral orders (Sec. 4, table of
relative differences), on three 25 x 25 images that are not available here.
This script runs the oracle (``oracle.fill``, B = 1 as in the paper,
8-connected) on seeded stand-ins of the same kind and size:

* "bumps": a few smooth Gaussian bumps with light noise (``synth.blobs``);
* "hairpin bend": a dark serpentine corridor (``synth.corridor``);
* "random": i.i.d. grey levels (``synth.uniform_random``).

It writes ``count_study.json`` beside itself: mean propagations per order
over five seeds, the relative differences, and the filling-rate curve of
seed 0. Nothing here touches the CUDA library. Run from the repository
root:

    python tests/golden/count_study.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2007_16076_gb300 import synth  # noqa: E402

ORDERS = ("naive", "spiral", "repulsion", "extrema", "minfill")
IMAGES = {
    "bumps": lambda s: synth.blobs(25, 25, 4, 4.0, 10.0, seed=s),
    "hairpin bend": lambda s: synth.corridor(25, 25, seed=s),
    "random": lambda s: synth.uniform_random(25, 25, 1, 255, seed=s),
}
SEEDS = range(5)


def main():
    N = 25 * 25
    A = N * (N - 1) // 2
    out = {"cite": "Sec. 4, table of relative differences (naive and spiral references)",
           "conn": 8, "B": 1, "seeds": list(SEEDS), "images": {}}
    for name, make in IMAGES.items():
        props = {o: [] for o in ORDERS}
        curves = {}
        for s in SEEDS:
            img = make(s)
            for o in ORDERS:
                r = oracle.fill(img, o, B=1, seed=s, conn=8)
                props[o].append(r.propagations)
                if s == 0:
                    tau = np.cumsum(r.round_new) / A
                    curves[o] = [round(float(t), 4) for t in tau[::10]]
        mean = {o: float(np.mean(v)) for o, v in props.items()}
        dr_naive = {o: round(100.0 * (mean["naive"] - mean[o]) / mean["naive"], 1) for o in ORDERS[1:]}
        dr_spiral = {o: round(100.0 * (mean["spiral"] - mean[o]) / mean["spiral"], 1) for o in ORDERS[2:]}
        out["images"][name] = {"mean_propagations": mean, "delta_r_naive_percent": dr_naive,
                               "delta_r_spiral_percent": dr_spiral,
                               "tau_every_10_propagations_seed0": curves}
        print(name, mean, dr_naive, dr_spiral, flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "count_study.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
