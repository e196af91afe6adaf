"""The paper's Sec. 4 count study, reproduced by the CUDA path.

``tests/golden/count_study.json`` holds the oracle's results on the 25 x 25
stand-ins of the paper's three test images (five seeds, B = 1 as in the
paper, 8-connected): the mean number of propagations each order needs and
the filling-rate curve of seed 0. The GPU path must give the same numbers
for every image and order: the same means (every seed's count equal), the
same curve, and the Dijkstra array.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2007_16076_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "count_study.json")
IMAGES = {
    "bumps": lambda s: synth.blobs(25, 25, 4, 4.0, 10.0, seed=s),
    "hairpin bend": lambda s: synth.corridor(25, 25, seed=s),
    "random": lambda s: synth.uniform_random(25, 25, 1, 255, seed=s),
}


@pytest.fixture(scope="module")
def gp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2007_16076_gb300 as g
    g.load()
    return g


@pytest.mark.parametrize("image", list(IMAGES))
def test_count_study_on_gpu(gp, image):
    gold = json.load(open(GOLDEN))
    rec = gold["images"][image]
    N = 25 * 25
    A = N * (N - 1) // 2
    for order, mean in rec["mean_propagations"].items():
        props = []
        for s in gold["seeds"]:
            img = IMAGES[image](s)
            with gp.Image(img, conn=gold["conn"], B=gold["B"], seed=s) as im:
                D, st = im.all_pairs(order, want_log=True)
            props.append(st["propagations"])
            if s == 0:
                tau = np.cumsum(st["round_new"].astype(np.float64)) / A
                curve = [round(float(t), 4) for t in tau[::10]]
                assert curve == rec["tau_every_10_propagations_seed0"][order], order
                assert np.array_equal(gp.as_uint32(D), oracle.apsp(img, conn=gold["conn"]))
        assert float(np.mean(props)) == mean, order
    # the relative differences follow from the means
    m = rec["mean_propagations"]
    for o, v in rec["delta_r_naive_percent"].items():
        assert round(100.0 * (m["naive"] - m[o]) / m["naive"], 1) == v
