"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values
printed in the paper, closed forms, hand-worked counts, brute force on tiny
graphs, an independent Floyd-Warshall, a plain BFS, and invariants of the
distance and of the method.
"""
import itertools
import json
import os
from collections import deque

import numpy as np
import pytest

import oracle
from paper_2007_16076_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U = oracle.UNREACH


def _nbrs(H, W, conn, p, free=None):
    r, c = divmod(p, W)
    out = []
    for dr in (-1, 0, 1):
        for dc in (-1, 0, 1):
            if dr == 0 and dc == 0:
                continue
            if conn == 4 and dr != 0 and dc != 0:
                continue
            rr, cc = r + dr, c + dc
            if 0 <= rr < H and 0 <= cc < W:
                q = rr * W + cc
                if free is None or (free[p] and free[q]):
                    out.append(q)
    return out


# --------------------------------------------------------------------------
# Sec. 2: distances
# --------------------------------------------------------------------------

def test_property1_printed_example():
    """Sec. 2, eq. 'chasles': 8 = 20 - 12 on a geodesic path A, C, D."""
    g = json.load(open(os.path.join(GOLDEN, "property1_example.json")))
    img = np.array(g["image"], dtype=np.uint8)
    dA = oracle.sssp(img, g["A"], conn=g["conn"])
    dC = oracle.sssp(img, g["C"], conn=g["conn"])
    assert dA[g["C"]] == g["d_AC"]
    assert dA[g["D"]] == g["d_AD"]
    assert dC[g["D"]] == g["d_CD"]
    assert dA[g["D"]] - dA[g["C"]] == dC[g["D"]]


def _brute_force(img, conn):
    """Minimum over all simple paths, by exhaustive enumeration."""
    H, W = img.shape
    N = H * W
    f = img.reshape(-1).astype(np.int64)
    D = np.full((N, N), U, dtype=np.uint64)
    for s in range(N):
        D[s, s] = 0
        stack = [(s, 0, 1 << s)]
        while stack:
            v, cost, seen = stack.pop()
            for q in _nbrs(H, W, conn, v):
                if seen >> q & 1:
                    continue
                c2 = cost + int(f[v] + f[q] + 1)
                if c2 < D[s, q]:
                    D[s, q] = c2
                stack.append((q, c2, seen | (1 << q)))
    return D.astype(np.uint32)


@pytest.mark.parametrize("shape", [(2, 2), (2, 3), (3, 3)])
@pytest.mark.parametrize("conn", [4, 8])
def test_brute_force_paths(shape, conn):
    """Eqs. 'temps'/'distance': the infimum over paths of summed weights."""
    rng = np.random.default_rng(7 + shape[0] * 10 + shape[1] + conn)
    for _ in range(3):
        img = rng.integers(0, 256, size=shape).astype(np.uint8)
        assert np.array_equal(oracle.apsp(img, conn=conn), _brute_force(img, conn))


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("shape", [(1, 7), (5, 1), (4, 6), (7, 7), (8, 5)])
def test_floyd_warshall(shape, conn):
    rng = np.random.default_rng(shape[0] * 100 + shape[1] + conn)
    img = rng.integers(0, 256, size=shape).astype(np.uint8)
    assert np.array_equal(oracle.apsp(img, conn=conn), oracle.floyd(img, conn=conn))


@pytest.mark.parametrize("conn", [4, 8])
def test_floyd_warshall_mask(conn):
    rng = np.random.default_rng(conn)
    mask = (rng.random((7, 8)) > 0.35).astype(np.uint8)
    img = np.zeros((7, 8), dtype=np.uint8)
    a = oracle.apsp(img, conn=conn, kind="mask", mask=mask)
    b = oracle.floyd(img, conn=conn, kind="mask", mask=mask)
    assert np.array_equal(a, b)


def _brute_force_l1(img, conn):
    """Minimum over all simple paths of the L1 weights |f(p) - f(q)| + 1."""
    H, W = img.shape
    N = H * W
    f = img.reshape(-1).astype(np.int64)
    D = np.full((N, N), U, dtype=np.uint64)
    for s in range(N):
        D[s, s] = 0
        stack = [(s, 0, 1 << s)]
        while stack:
            v, cost, seen = stack.pop()
            for q in _nbrs(H, W, conn, v):
                if seen >> q & 1:
                    continue
                c2 = cost + int(abs(f[v] - f[q]) + 1)
                if c2 < D[s, q]:
                    D[s, q] = c2
                stack.append((q, c2, seen | (1 << q)))
    return D.astype(np.uint32)


@pytest.mark.parametrize("shape", [(2, 2), (2, 3), (3, 3)])
@pytest.mark.parametrize("conn", [4, 8])
def test_l1_brute_force_paths(shape, conn):
    """Sec. 2, pseudo-metric L1 (eq. 'distance abs difference') with +1 per
    edge, summed along paths (eq. 'temps') and minimised (eq. 'distance')."""
    rng = np.random.default_rng(11 + shape[0] * 10 + shape[1] + conn)
    for _ in range(3):
        img = rng.integers(0, 256, size=shape).astype(np.uint8)
        assert np.array_equal(oracle.apsp(img, conn=conn, kind="l1"), _brute_force_l1(img, conn))


# --------------------------------------------------------------------------
# Multichannel images (Sec. 2: values in T^L), sum pseudo-metric over the
# channels: w(p,q) = sum_l (f_l(p) + f_l(q)) + 1
# --------------------------------------------------------------------------

def _brute_force_channels(ch, conn):
    """Minimum over all simple paths of the channel-summed weights, each
    weight added up channel by channel."""
    L, H, W = ch.shape
    N = H * W
    f = ch.reshape(L, -1).astype(np.int64)
    D = np.full((N, N), U, dtype=np.uint64)
    for s in range(N):
        D[s, s] = 0
        stack = [(s, 0, 1 << s)]
        while stack:
            v, cost, seen = stack.pop()
            for q in _nbrs(H, W, conn, v):
                if seen >> q & 1:
                    continue
                c2 = cost + 1 + sum(int(f[l, v] + f[l, q]) for l in range(L))
                if c2 < D[s, q]:
                    D[s, q] = c2
                stack.append((q, c2, seen | (1 << q)))
    return D.astype(np.uint32)


@pytest.mark.parametrize("shape", [(2, 3), (3, 3)])
@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("L", [2, 3])
def test_channels_brute_force_paths(shape, conn, L):
    rng = np.random.default_rng(17 + shape[0] * 10 + shape[1] + conn + L)
    for _ in range(2):
        ch = rng.integers(0, 256, size=(L,) + shape).astype(np.uint8)
        assert np.array_equal(oracle.apsp(ch, conn=conn, kind="sum"), _brute_force_channels(ch, conn))


@pytest.mark.parametrize("conn", [4, 8])
def test_channels_one_channel_is_grey(conn):
    """With one channel the channel sum is the grey sum pseudo-metric."""
    img = synth.blobs(13, 17, 3, 3.0, 55.0, seed=conn)
    assert np.array_equal(oracle.apsp(img[None], conn=conn, kind="sum"), oracle.apsp(img, conn=conn))


@pytest.mark.parametrize("conn", [4, 8])
def test_channels_constant_closed_form(conn):
    """Constant channels c_l: every edge costs 2 sum(c) + 1, so d is that
    times the chessboard (8) or city-block (4) step count."""
    c = np.array([3, 0, 250, 17], dtype=np.uint8)
    H, W = 6, 9
    ch = np.broadcast_to(c[:, None, None], (4, H, W)).copy()
    D = oracle.apsp(ch, conn=conn, kind="sum")
    r, col = np.divmod(np.arange(H * W), W)
    dr = np.abs(r[:, None] - r[None, :])
    dc = np.abs(col[:, None] - col[None, :])
    steps = np.maximum(dr, dc) if conn == 8 else dr + dc
    assert np.array_equal(D, (2 * int(c.sum()) + 1) * steps)


@pytest.mark.parametrize("W", [2, 9, 31])
def test_channels_one_row_closed_form(W):
    """1 x W (eq. 'distance geo somme' over the channel sums F): d(i,j) =
    F(i) + F(j) + 2 sum_{i<k<j} F(k) + |j - i|."""
    rng = np.random.default_rng(W)
    ch = rng.integers(0, 256, size=(3, 1, W)).astype(np.uint8)
    F = ch.astype(np.int64).sum(axis=0)[0]
    D = oracle.apsp(ch, conn=8, kind="sum")
    for i in range(W):
        for j in range(W):
            lo, hi = min(i, j), max(i, j)
            want = 0 if i == j else F[i] + F[j] + 2 * F[lo + 1:hi].sum() + (hi - lo)
            assert D[i, j] == want


def test_channels_floyd_warshall_and_fill():
    rng = np.random.default_rng(5)
    ch = rng.integers(0, 256, size=(5, 7, 8)).astype(np.uint8)
    D = oracle.apsp(ch, conn=8, kind="sum")
    assert np.array_equal(D, oracle.floyd(ch, conn=8, kind="sum"))
    r = oracle.fill(ch, "minfill", B=3, conn=8, kind="sum", want_D=True)
    assert np.array_equal(r.D, D)
    assert r.new_pairs == 56 * 55 // 2


@pytest.mark.parametrize("W", [1, 2, 9, 40])
def test_l1_one_row_closed_form(W):
    """L1 on a 1xW image: the path is unique, so d(i,j) is the total variation
    of f between i and j plus one per step."""
    rng = np.random.default_rng(100 + W)
    f = rng.integers(0, 256, size=W).astype(np.int64)
    D = oracle.apsp(f.astype(np.uint8).reshape(1, W), conn=4, kind="l1")
    for i in range(W):
        for j in range(W):
            lo, hi = min(i, j), max(i, j)
            assert D[i, j] == np.abs(np.diff(f[lo:hi + 1])).sum() + (hi - lo)


@pytest.mark.parametrize("conn", [4, 8])
def test_l1_constant_image_and_floyd_warshall(conn):
    """L1 on a constant image costs one per step (city-block or chessboard);
    on a random image it agrees with Floyd-Warshall."""
    H, W = 5, 7
    D = oracle.apsp(np.full((H, W), 90, dtype=np.uint8), conn=conn, kind="l1")
    rr, cc = np.divmod(np.arange(H * W), W)
    dr = np.abs(rr[:, None] - rr[None, :])
    dc = np.abs(cc[:, None] - cc[None, :])
    assert np.array_equal(D.astype(np.int64), dr + dc if conn == 4 else np.maximum(dr, dc))
    img = np.random.default_rng(conn).integers(0, 256, size=(6, 7)).astype(np.uint8)
    assert np.array_equal(oracle.apsp(img, conn=conn, kind="l1"), oracle.floyd(img, conn=conn, kind="l1"))


@pytest.mark.parametrize("order", ["naive", "minfill"])
def test_l1_fill_invariants(order):
    """The method is indifferent to the pseudo-metric: with L1 weights the
    Property-1 array equals the Dijkstra array and every pair is filled."""
    img = synth.blobs(9, 11, 3, 2.5, 55.0, seed=4)
    r = oracle.fill(img, order, B=3, conn=8, kind="l1", want_D=True)
    assert np.array_equal(r.D, oracle.apsp(img, conn=8, kind="l1"))
    assert r.new_pairs == 99 * 98 // 2


@pytest.mark.parametrize("W", [1, 2, 9, 40])
def test_one_row_closed_form(W):
    """Eq. 'distance geo somme' with the +1 per edge: on a 1xW image the path
    is unique and d(i,j) = f(i) + f(j) + 2*sum_{i<k<j} f(k) + |j - i|."""
    rng = np.random.default_rng(W)
    f = rng.integers(0, 256, size=W).astype(np.int64)
    img = f.astype(np.uint8).reshape(1, W)
    D = oracle.apsp(img, conn=8)
    for i in range(W):
        for j in range(W):
            lo, hi = min(i, j), max(i, j)
            exp = 0 if i == j else f[lo] + f[hi] + 2 * f[lo + 1:hi].sum() + (hi - lo)
            assert D[i, j] == exp


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("c", [0, 1, 77, 255])
def test_constant_image_closed_form(conn, c):
    """Constant grey level c: every edge costs 2c+1, so d = (2c+1) times the
    city-block (4-neighbourhood) or chessboard (8-neighbourhood) step count."""
    H, W = 6, 9
    img = np.full((H, W), c, dtype=np.uint8)
    D = oracle.apsp(img, conn=conn)
    rr, cc = np.divmod(np.arange(H * W), W)
    dr = np.abs(rr[:, None] - rr[None, :])
    dc = np.abs(cc[:, None] - cc[None, :])
    steps = dr + dc if conn == 4 else np.maximum(dr, dc)
    assert np.array_equal(D.astype(np.int64), (2 * c + 1) * steps)


@pytest.mark.parametrize("conn", [4, 8])
def test_mask_is_twice_bfs_hops(conn):
    """Mask variant: w = 2 between free pixels, so d = 2 x (BFS hop count)
    inside a component and unreachable across components and obstacles."""
    m = synth.disk_mask(20, 23, 0.4, 2, 4, seed=3)
    H, W = m.shape
    N = H * W
    free = m.reshape(-1).astype(bool)
    D = oracle.apsp(np.zeros_like(m), conn=conn, kind="mask", mask=m)
    for s in range(0, N, 7):
        hop = np.full(N, -1)
        if free[s]:
            hop[s] = 0
            dq = deque([s])
            while dq:
                v = dq.popleft()
                for q in _nbrs(H, W, conn, v, free):
                    if hop[q] < 0:
                        hop[q] = hop[v] + 1
                        dq.append(q)
        exp = np.where(hop >= 0, 2 * hop, U).astype(np.uint32)
        exp[s] = 0
        assert np.array_equal(D[s], exp)


@pytest.mark.parametrize("conn", [4, 8])
def test_distance_invariants(conn):
    """Symmetry (the neighbour relation is symmetric, Sec. 2), zero diagonal,
    triangle inequality, and d(p,q) = w(p,q) for neighbours (a detour through
    any pixel x adds 2 f(x) + 1 >= 1)."""
    img = synth.blobs(12, 13, 3, 2.5, 55.0, seed=1)
    H, W = img.shape
    N = H * W
    D = oracle.apsp(img, conn=conn).astype(np.int64)
    assert np.array_equal(D, D.T)
    assert np.all(np.diag(D) == 0)
    f = img.reshape(-1).astype(np.int64)
    for p in range(N):
        for q in _nbrs(H, W, conn, p):
            assert D[p, q] == f[p] + f[q] + 1
    tri = D[:, :, None] <= D[:, None, :] + D.T[None, :, :]  # d(i,j) <= d(i,k)+d(k,j)
    assert tri.all()


def test_multi_source_is_min_of_rows():
    img = synth.blobs(10, 11, 3, 2.0, 55.0, seed=4)
    src = [0, 17, 93]
    ms = oracle.msssp(img, src, conn=8)
    R = oracle.rows(img, src, conn=8)
    assert np.array_equal(ms, R.min(axis=0))


# --------------------------------------------------------------------------
# Sec. 2: geodesic tree
# --------------------------------------------------------------------------

@pytest.mark.parametrize("conn", [4, 8])
def test_parents_against_floyd(conn):
    """The canonical tree: each reached b != s points to its smallest-index
    neighbour q with d(s,q) + w(q,b) = d(s,b), distances from Floyd-Warshall.
    Following parents reaches s with strictly decreasing distance."""
    rng = np.random.default_rng(11)
    img = rng.integers(0, 40, size=(6, 7)).astype(np.uint8)
    H, W = img.shape
    N = H * W
    F = oracle.floyd(img, conn=conn).astype(np.int64)
    f = img.reshape(-1).astype(np.int64)
    for s in range(N):
        par = oracle.parents(img, F[s].astype(np.uint32), s, conn=conn)
        assert par[s] == -1
        for b in range(N):
            if b == s:
                continue
            tight = [q for q in _nbrs(H, W, conn, b) if F[s, q] + f[q] + f[b] + 1 == F[s, b]]
            assert par[b] == min(tight)
            x, steps = b, 0
            while x != s:
                assert F[s, par[x]] < F[s, x]
                x = par[x]
                steps += 1
                assert steps <= N


def test_one_row_tree_is_the_path():
    img = np.array([[3, 9, 2, 2, 7, 1]], dtype=np.uint8)
    d = oracle.sssp(img, 2, conn=4)
    par = oracle.parents(img, d, 2, conn=4)
    assert list(par) == [1, 2, -1, 2, 3, 4]


# --------------------------------------------------------------------------
# Sec. 3: orders
# --------------------------------------------------------------------------

def test_spiral_frames_structure():
    """Sec. 3.1: concentric one-pixel frames, outermost first; each frame is
    a permutation of its pixels."""
    H, W = 7, 10
    seq = oracle.spiral_sequence(H, W, seed=123)
    assert sorted(seq.tolist()) == list(range(H * W))
    r, c = np.divmod(seq, W)
    frame = np.minimum(np.minimum(r, c), np.minimum(H - 1 - r, W - 1 - c))
    assert np.all(np.diff(frame) >= 0)
    assert (frame == 0).sum() == 2 * (H + W) - 4
    # different seeds draw different orders within a frame
    assert not np.array_equal(seq, oracle.spiral_sequence(H, W, seed=124))


def test_spiral_draws_are_uniform():
    """Sec. 3.1: within a frame, the source is drawn uniformly at random.
    Over many seeds the first source of a 1 x 8 frame is spread evenly."""
    counts = np.zeros(8)
    for seed in range(4000):
        counts[oracle.spiral_sequence(1, 8, seed)[0]] += 1
    exp = 4000 / 8
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 24.3  # chi-square, 7 dof, p = 0.001


def _ring(H, W, k):
    """Frame k as a turn of the spiral: its pixels clockwise from (k, k)."""
    r0, r1, c0, c1 = k, H - 1 - k, k, W - 1 - k
    out = [(r0, c) for c in range(c0, c1 + 1)]
    if r1 > r0:
        out += [(r, c1) for r in range(r0 + 1, r1 + 1)]
        if c1 > c0:
            out += [(r1, c) for c in range(c1 - 1, c0 - 1, -1)]
            out += [(r, c0) for r in range(r1 - 1, r0, -1)]
    return [r * W + c for r, c in out], (r1 > r0 and c1 > c0)


def test_repulsion_keeps_sources_apart_on_a_turn():
    """Algorithm "spiral method with repulsion" (h = 3): the first sources
    come from the outermost turn, and each takes its two neighbours on each
    side out of the draw, so sources drawn in one pass over a turn are at
    least three ring steps apart. On a 25 x 25 image the outer turn has 96
    points; the first 8 draws (at most 40 points removed, no turn point
    filled yet but the sources) all belong to the first pass."""
    img = synth.blobs(25, 25, 4, 3.0, 55.0, seed=3)
    ring, cyclic = _ring(25, 25, 0)
    assert cyclic and len(ring) == 96
    pos = {p: i for i, p in enumerate(ring)}
    for seed in range(5):
        r = oracle.fill(img, "repulsion", B=1, conn=8, seed=seed)
        first = [int(x) for x in r.sources[:8]]
        assert all(p in pos for p in first)
        for a in range(8):
            for b in range(a):
                dd = abs(pos[first[a]] - pos[first[b]])
                assert min(dd, 96 - dd) >= 3
        # without repulsion (spiral), some seed puts two early sources close
    close = 0
    for seed in range(20):
        sp = [int(x) for x in oracle.fill(img, "spiral", B=1, conn=8, seed=seed).sources[:8]]
        for a in range(8):
            for b in range(a):
                dd = abs(pos[sp[a]] - pos[sp[b]])
                close += min(dd, 96 - dd) < 3
    assert close > 0


def test_repulsion_open_line_and_batches():
    """A single row is an open turn (no wrap-around): on 1 x 11 the first
    pass takes sources at least three apart along the row; with B sources
    per round each round draws them one after the other from the state at
    the round's start, and the result is a valid fill."""
    img = synth.uniform_random(1, 11, 1, 255, seed=2)
    for seed in range(10):
        r = oracle.fill(img, "repulsion", B=3, conn=8, seed=seed)
        first = sorted(int(x) for x in r.sources[:3])
        assert first[1] - first[0] >= 3 and first[2] - first[1] >= 3
        assert r.new_pairs == 11 * 10 // 2


def test_repulsion_first_draw_is_uniform():
    """The first source is drawn uniformly from the outermost turn (here the
    20 points of a 6 x 6 frame)."""
    img = np.full((6, 6), 7, dtype=np.uint8)
    ring, _ = _ring(6, 6, 0)
    counts = {p: 0 for p in ring}
    n = 2000
    for seed in range(n):
        counts[int(oracle.fill(img, "repulsion", B=1, conn=4, seed=seed).sources[0])] += 1
    exp = n / 20
    chi2 = sum((c - exp) ** 2 / exp for c in counts.values())
    assert chi2 < 43.8  # chi-square, 19 dof, p = 0.001


def test_extrema_constant_square():
    """Sec. 3.3 on a constant image: the centroid is the pixel farthest from
    the edges (the centre), and Ext starts at the corners."""
    img = np.full((5, 5), 10, dtype=np.uint8)
    ex = oracle.extrema(img, conn=8)
    assert ex.centroids.tolist() == [12]
    assert ex.e[12] == 2 * 21
    corners = {0, 4, 20, 24}
    first4 = set(int(np.argwhere(ex.rank == k)[0, 0]) for k in range(4))
    assert first4 <= set(range(25)) and len(first4) == 4
    assert all(ex.g[p] == 2 * 21 for p in first4)  # chessboard 2 from the centre
    assert corners <= {p for p in range(25) if ex.g[p] == 2 * 21}
    # 4x4: four inner pixels tie; the smallest index wins
    ex4 = oracle.extrema(np.full((4, 4), 3, dtype=np.uint8), conn=8)
    assert ex4.centroids.tolist() == [5]


def test_extrema_one_row():
    ex = oracle.extrema(np.array([[4, 4, 9, 1, 0, 7]], dtype=np.uint8), conn=8)
    assert ex.centroids.tolist() == [0]
    assert ex.rank[5] == 0 and ex.rank[0] == 5


# --------------------------------------------------------------------------
# The method's counts
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLDEN, "hand_counts.json")))["cases"],
                         ids=lambda c: c["name"])
def test_hand_counts(case):
    img = np.array(case["image"], dtype=np.uint8)
    seed = case.get("seed", 0)
    if "sequence" in case:
        # the frame sequence the derivation starts from (pinned on its own by
        # the frame-structure and uniformity tests of the spiral order)
        assert oracle.spiral_sequence(*img.shape, seed).tolist() == case["sequence"]
    if "draws_raw" in case:
        # the draws the derivation reduces: SplitMix64 from the handle's seed
        assert [str(x) for x in _splitmix64(seed, len(case["draws_raw"]))] == case["draws_raw"]
    r = oracle.fill(img, case["order"], B=case["B"], seed=seed, conn=case["conn"], want_D=True)
    for k in ("propagations", "prepass_propagations", "distance_ops", "new_pairs", "rounds"):
        assert getattr(r, k) == case[k], k
    assert r.sources.tolist() == case["sources"]
    if "round_new" in case:
        assert r.round_new.tolist() == case["round_new"]
    assert np.array_equal(r.D, oracle.apsp(img, conn=case["conn"]))


def _splitmix64(seed, n):
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) from its published
    definition: state += 0x9E3779B97F4A7C15, then two xor-shift-multiply
    steps and a final xor-shift."""
    m = (1 << 64) - 1
    s, out = seed & m, []
    for _ in range(n):
        s = (s + 0x9E3779B97F4A7C15) & m
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_published_vector():
    """The first outputs of SplitMix64 from state 0, as published with the
    generator, so that the draws listed in the hand counts are its outputs."""
    assert _splitmix64(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


@pytest.mark.parametrize("W", [2, 5, 31])
def test_one_row_minfill_single_propagation(W):
    """On a path graph the greatest extremum is an end, and its tree relates
    every pair: one propagation, ops = sum of depths = W(W-1)/2."""
    rng = np.random.default_rng(W)
    img = rng.integers(0, 256, size=(1, W)).astype(np.uint8)
    r = oracle.fill(img, "minfill", B=1, conn=8)
    assert r.propagations == 1 and r.prepass_propagations == 2
    assert r.distance_ops == W * (W - 1) // 2
    assert r.new_pairs == W * (W - 1) // 2


@pytest.mark.parametrize("order", ["naive", "spiral", "repulsion", "extrema", "minfill"])
@pytest.mark.parametrize("B", [1, 3, 8])
@pytest.mark.parametrize("conn", [4, 8])
def test_fill_invariants(order, B, conn):
    """Sec. 2: every pair is filled exactly once (sum of new pairs = A,
    eq. 'A'), the array filled by Property 1 equals the Dijkstra array, and
    every point ends filled (tau = 1)."""
    img = synth.blobs(11, 12, 3, 2.5, 55.0, seed=B + conn)
    N = img.size
    r = oracle.fill(img, order, B=B, seed=5, conn=conn, want_D=True)
    assert r.new_pairs == (N * N - N) // 2
    assert r.round_new.sum() == r.new_pairs
    assert np.array_equal(r.D, oracle.apsp(img, conn=conn))
    assert r.propagations <= N
    assert len(set(r.sources.tolist())) == r.propagations
    # every round but the last takes B sources (all selected points end filled)
    assert r.rounds == -(-r.propagations // B)


@pytest.mark.parametrize("order", ["naive", "spiral", "repulsion", "extrema", "minfill"])
def test_fill_mask_invariants(order):
    """Mask variant: pairs in different components are filled at the start
    with 'unreachable'; the trees fill exactly the same-component pairs."""
    m = synth.disk_mask(14, 15, 0.4, 2, 3, seed=2)
    img = np.zeros_like(m)
    r = oracle.fill(img, order, B=4, conn=8, kind="mask", mask=m, want_D=True)
    N = m.size
    D = oracle.apsp(img, conn=8, kind="mask", mask=m)
    assert np.array_equal(r.D, D)
    same = (D != U) & ~np.eye(N, dtype=bool)
    assert r.new_pairs == same.sum() // 2
    assert r.prefilled_pairs + r.new_pairs == (N * N - N) // 2
    assert r.components >= 2


def test_naive_full_row_count():
    """Naive without the tree (Sec. 1): N propagations, one row each."""
    img = synth.blobs(6, 7, 2, 2.0, 55.0, seed=0)
    R = oracle.rows(img, np.arange(img.size), conn=8)
    assert R.shape == (img.size, img.size)
    assert np.array_equal(R, oracle.apsp(img, conn=8))


def test_published_ranking_on_bumps_standins():
    """Sec. 4 / Table 'comparaison': on structured ('bumps') images the
    filling-rate method needs fewer propagations than the spiral and naive
    orders. Checked qualitatively on seeded 25x25 blob stand-ins (the paper's
    images are not available)."""
    wins = 0
    for seed in range(4):
        img = synth.blobs(25, 25, 6, 3.0, 30.0, seed=seed)
        img = np.maximum(img, 1)  # grey levels 1-255 as in the paper
        mf = oracle.fill(img, "minfill", B=1, conn=8).propagations + 2
        sp = oracle.fill(img, "spiral", B=1, seed=seed, conn=8).propagations
        nv = oracle.fill(img, "naive", B=1, conn=8).propagations
        wins += (mf < sp) and (mf < nv)
    assert wins >= 3
