"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Distances are integers, so every comparison is bit-exact. Counts
(propagations, distance operations, new pairs, rounds) and the order of the
selected sources must equal the oracle's simulation of the same order.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_2007_16076_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def gp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2007_16076_gb300 as g
    g.load()
    return g


def _u32(t):
    return t.detach().cpu().numpy().view(np.uint32)


# --------------------------------------------------------------------------
# gapsp_rows: single-source propagations
# --------------------------------------------------------------------------

ROW_SHAPES = [(1, 1), (1, 9), (13, 1), (2, 2), (7, 13), (31, 33), (33, 45), (64, 64),
              (100, 37), (37, 100), (128, 128), (129, 130), (200, 256)]


@pytest.mark.parametrize("shape", ROW_SHAPES, ids=lambda s: f"{s[0]}x{s[1]}")
@pytest.mark.parametrize("conn", [4, 8])
def test_rows_grey(gp, shape, conn):
    H, W = shape
    img = synth.blobs(H, W, max(1, H * W // 300), max(1.5, (H + W) / 16), 55.0, seed=H * 7 + W)
    N = H * W
    rng = np.random.default_rng(H + W)
    src = np.unique(np.concatenate([[0, N - 1, N // 2], rng.integers(0, N, size=min(N, 24))]))
    src = src.astype(np.int32)
    with gp.Image(img, conn=conn) as im:
        out = _u32(im.rows(src))
    ref = oracle.rows(img, src, conn=conn)
    assert np.array_equal(out, ref)


@pytest.mark.parametrize("shape", [(5, 5), (40, 33), (128, 128), (256, 256)], ids=lambda s: f"{s[0]}x{s[1]}")
@pytest.mark.parametrize("conn", [4, 8])
def test_rows_mask(gp, shape, conn):
    H, W = shape
    m = synth.disk_mask(H, W, 0.4, 3 if H > 20 else 1, 12 if H > 20 else 2, seed=H + conn)
    N = H * W
    rng = np.random.default_rng(N)
    src = rng.integers(0, N, size=min(N, 20)).astype(np.int32)  # obstacles included
    with gp.Image(None, conn=conn, kind="mask", mask=m) as im:
        out = _u32(im.rows(src))
    ref = oracle.rows(np.zeros_like(m), src, conn=conn, kind="mask", mask=m)
    assert np.array_equal(out, ref)


@pytest.mark.parametrize("shape", [(1, 9), (7, 13), (33, 45), (128, 128), (100, 37)], ids=lambda s: f"{s[0]}x{s[1]}")
@pytest.mark.parametrize("conn", [4, 8])
def test_rows_l1(gp, shape, conn):
    """The L1 pseudo-metric (Sec. 2): w = |f(p) - f(q)| + 1."""
    H, W = shape
    img = synth.blobs(H, W, max(1, H * W // 300), max(1.5, (H + W) / 16), 55.0, seed=H * 5 + W)
    N = H * W
    rng = np.random.default_rng(N + conn)
    src = np.unique(np.concatenate([[0, N - 1], rng.integers(0, N, size=min(N, 20))])).astype(np.int32)
    with gp.Image(img, conn=conn, kind="l1") as im:
        out = _u32(im.rows(src))
    assert np.array_equal(out, oracle.rows(img, src, conn=conn, kind="l1"))


@pytest.mark.parametrize("order", ["naive", "spiral", "repulsion", "extrema", "minfill"])
@pytest.mark.parametrize("conn", [4, 8])
def test_all_pairs_l1(gp, order, conn):
    img = synth.blobs(17, 23, 3, 2.5, 55.0, seed=conn)
    _check_fill(gp, img, order, 5, conn, kind="l1")


def test_rows_structured_images(gp):
    """Winding corridors and step edges need many sweeps; uniform noise and
    constant images are the other extremes."""
    imgs = [synth.corridor(64, 64, seed=1), synth.corridor(25, 25, seed=2),
            synth.uniform_random(50, 70, 1, 255, seed=3), np.full((40, 40), 9, np.uint8),
            synth.blobs_with_steps(96, 96, 16, 8.0, 20, 100.0, 40.0, seed=4)]
    for img in imgs:
        N = img.size
        src = np.array([0, N - 1, N // 3, (2 * N) // 3], dtype=np.int32)
        for conn in (4, 8):
            with gp.Image(img, conn=conn) as im:
                out = _u32(im.rows(src))
            assert np.array_equal(out, oracle.rows(img, src, conn=conn))


def test_rows_host_buffers(gp):
    img = synth.blobs(30, 40, 4, 3.0, 55.0, seed=9)
    src = np.array([3, 500, 1199], dtype=np.int32)
    out = np.zeros((3, img.size), dtype=np.uint32)
    with gp.Image(img, conn=8) as im:
        im.rows(src, out=out)
    assert np.array_equal(out, oracle.rows(img, src, conn=8))


def test_rows_many_sources_full_array(gp):
    """All N sources (the naive method of Sec. 1) in one call."""
    img = synth.blobs(32, 32, 8, 4.0, 55.0, seed=0)
    N = img.size
    with gp.Image(img, conn=4) as im:
        out = _u32(im.rows(np.arange(N, dtype=np.int32)))
    assert np.array_equal(out, oracle.apsp(img, conn=4))


def test_rows_invalid_source(gp):
    img = synth.blobs(8, 8, 2, 2.0, 55.0, seed=1)
    with gp.Image(img, conn=8) as im:
        with pytest.raises(gp.GapspError) as e:
            im.rows(np.array([0, 64], dtype=np.int32))
        assert e.value.code == 1
        with pytest.raises(gp.GapspError):
            im.rows(np.array([-1], dtype=np.int32))
        out = im.rows(np.zeros(0, dtype=np.int32))
        assert out.numel() == 0


# --------------------------------------------------------------------------
# gapsp_all_pairs: the method
# --------------------------------------------------------------------------

def _check_fill(gp, img, order, B, conn, kind="grey", mask=None, seed=0):
    with gp.Image(img, conn=conn, kind=kind, mask=mask, B=B, seed=seed) as im:
        D, st = im.all_pairs(order, want_log=True)
    D = _u32(D)
    ref = oracle.fill(img if img is not None else np.zeros_like(mask), order, B=B, seed=seed,
                      conn=conn, kind=kind, mask=mask)
    Dref = oracle.apsp(img if img is not None else np.zeros_like(mask), conn=conn, kind=kind, mask=mask)
    assert np.array_equal(D, Dref)
    for k in ("propagations", "prepass_propagations", "distance_ops", "new_pairs", "rounds"):
        assert st[k] == getattr(ref, k), k
    assert np.array_equal(st["round_new"], ref.round_new)
    if B == 1:
        assert np.array_equal(st["sources"], ref.sources)
    else:  # order inside a round is by key for minfill, by sequence otherwise
        assert np.array_equal(st["sources"], ref.sources)
    return st


@pytest.mark.parametrize("order", ["naive", "spiral", "repulsion", "extrema", "minfill"])
def test_all_pairs_plain_32(gp, order):
    """32x32 blobs, 4-connected, B = 1: the paper's sequential loop."""
    w = synth.plain_32(0)
    _check_fill(gp, w.img, order, 1, 4)


@pytest.mark.parametrize("order", ["naive", "spiral", "repulsion", "extrema", "minfill"])
@pytest.mark.parametrize("B", [2, 5, 32])
@pytest.mark.parametrize("shape,conn", [((17, 23), 8), ((24, 9), 4), ((1, 40), 8)])
def test_all_pairs_batched(gp, order, B, shape, conn):
    img = synth.blobs(shape[0], shape[1], 3, 2.5, 55.0, seed=B + conn)
    _check_fill(gp, img, order, B, conn, seed=B)


@pytest.mark.parametrize("order", ["naive", "spiral", "repulsion", "extrema", "minfill"])
@pytest.mark.parametrize("conn", [4, 8])
def test_all_pairs_mask(gp, order, conn):
    m = synth.disk_mask(26, 31, 0.4, 2, 4, seed=conn)
    st = _check_fill(gp, None, order, 4, conn, kind="mask", mask=m)
    ref = oracle.fill(np.zeros_like(m), order, B=4, conn=conn, kind="mask", mask=m)
    assert st["prefilled_pairs"] == ref.prefilled_pairs


def test_all_pairs_degenerate(gp):
    for img in (np.array([[7]], np.uint8), np.array([[1, 2]], np.uint8),
                np.full((3, 1), 4, np.uint8)):
        for order in ("naive", "spiral", "repulsion", "extrema", "minfill"):
            _check_fill(gp, img, order, 1, 8)


def test_all_pairs_host_array(gp):
    img = synth.blobs(20, 21, 3, 2.5, 55.0, seed=5)
    N = img.size
    D = np.zeros((N, N), dtype=np.uint32)
    with gp.Image(img, conn=8, B=8) as im:
        im.all_pairs("minfill", out=D)
    assert np.array_equal(D, oracle.apsp(img, conn=8))


def test_all_pairs_repeat_and_orders_share_handle(gp):
    """D is the same for every order and B; a handle can be reused."""
    img = synth.blobs(19, 22, 3, 2.5, 55.0, seed=6)
    ref = oracle.apsp(img, conn=8)
    with gp.Image(img, conn=8, B=3) as im:
        for order in ("minfill", "naive", "extrema", "spiral", "minfill"):
            D, _ = im.all_pairs(order)
            assert np.array_equal(_u32(D), ref)


@pytest.mark.parametrize("order", ["minfill", "naive", "spiral", "extrema", "repulsion"])
@pytest.mark.parametrize("lookahead", [-1, 1, 5, 0])
def test_lookahead_changes_nothing(gp, order, lookahead):
    """Rows computed ahead of their round (any candidate count, or none)
    leave D, the counts, the per-round new pairs and the source order as the
    oracle's simulation has them."""
    img = synth.blobs(37, 29, 5, 3.0, 55.0, seed=8)
    with gp.Image(img, conn=8, B=6, lookahead=lookahead) as im:
        D, st = im.all_pairs(order, want_log=True)
    ref = oracle.fill(img, order, B=6, conn=8)
    assert np.array_equal(_u32(D), oracle.apsp(img, conn=8))
    for k in ("propagations", "prepass_propagations", "distance_ops", "new_pairs", "rounds"):
        assert st[k] == getattr(ref, k), k
    assert np.array_equal(st["round_new"], ref.round_new)
    assert np.array_equal(st["sources"], ref.sources)
    if lookahead < 0 or order == "repulsion":  # random draws: nothing to foresee
        assert st["lookahead_propagations"] == 0
    else:
        assert st["lookahead_propagations"] > 0


@pytest.mark.parametrize("shape,conn,kind,prop_blocks", [
    ((37, 29), 8, "grey", 0),   # odd width: one value at a time
    ((32, 40), 8, "grey", 0),   # width a multiple of 4: 16-byte loads
    ((40, 32), 4, "l1", 0),
    ((33, 36), 8, "mask", 0),   # obstacles: neither helpers nor bounds through them
    ((48, 48), 8, "grey", 2),   # row strips on a cluster of two blocks
    ((64, 24), 4, "grey", 4),
])
@pytest.mark.parametrize("warm", [0, -1])
def test_warm_start_changes_nothing(gp, shape, conn, kind, prop_blocks, warm):
    """Propagations started from the complete rows of filled neighbours (or
    from the source alone) give the oracle's D, counts and source order."""
    H, W = shape
    img = synth.blobs(H, W, 5, 3.0, 55.0, seed=H + W)
    mask = synth.disk_mask(H, W, 0.3, 2, 4, seed=5) if kind == "mask" else None
    with gp.Image(img, conn=conn, kind=kind, mask=mask, B=5, warm_start=warm,
                  prop_blocks=prop_blocks) as im:
        D, st = im.all_pairs("minfill", want_log=True)
    ref = oracle.fill(img, "minfill", B=5, conn=conn, kind=kind, mask=mask)
    assert np.array_equal(_u32(D), oracle.apsp(img, conn=conn, kind=kind, mask=mask))
    for k in ("propagations", "prepass_propagations", "distance_ops", "new_pairs", "rounds"):
        assert st[k] == getattr(ref, k), k
    assert np.array_equal(st["sources"], ref.sources)


def test_warm_start_sweeps_fewer_lines(gp):
    """The warm start is taken: with it the propagations process fewer lines."""
    img = synth.blobs(64, 64, 8, 4.0, 55.0, seed=3)
    lines = {}
    for warm in (0, -1):
        with gp.Image(img, conn=8, B=16, warm_start=warm) as im:
            _, st = im.all_pairs("minfill")
        lines[warm] = st["lines"] / (st["propagations"] + st["lookahead_propagations"])
    assert lines[0] < 0.8 * lines[-1], lines


def test_lookahead_rejects_bad_counts(gp):
    img = synth.blobs(8, 8, 2, 2.0, 55.0, seed=1)
    for bad in (-2, 1025):
        with pytest.raises(gp.GapspError) as e:
            gp.Image(img, conn=8, B=4, lookahead=bad)
        assert e.value.code == 1


def test_misaligned_device_arrays_rejected(gp):
    """Rows of D move 16 bytes at a time: a device array that does not start
    on a 16-byte boundary is refused before any launch, and left alone."""
    import torch
    img = synth.blobs(8, 8, 2, 2.0, 55.0, seed=1)
    N = 64
    buf = torch.full((N * N + 4,), 7, dtype=torch.int32, device="cuda")
    with gp.Image(img, conn=8, B=4) as im:
        with pytest.raises(gp.GapspError) as e:
            im.all_pairs("minfill", out=buf[1:1 + N * N].view(N, N))
        assert e.value.code == 1
        with pytest.raises(gp.GapspError) as e:
            im.rows(np.array([0, 5], dtype=np.int32), out=buf[1:1 + 2 * N].view(2, N))
        assert e.value.code == 1
        with pytest.raises(gp.GapspError) as e:
            gp.rows_noalloc(torch.from_numpy(img).cuda(), np.array([3], dtype=np.int32),
                            buf[2:2 + N].view(1, N))
        assert e.value.code == 1
    torch.cuda.synchronize()
    assert bool((buf == 7).all())


def test_budget_rejected_before_allocation(gp):
    img = synth.blobs(64, 64, 4, 4.0, 55.0, seed=1)
    with gp.Image(img, conn=8, B=32, mem_budget=1 << 20) as im:
        with pytest.raises(gp.GapspError) as e:
            im.all_pairs("minfill")
        assert e.value.code == 3


# --------------------------------------------------------------------------
# Full-size workload: 128x128, 8-connected, B = 32
# --------------------------------------------------------------------------

@pytest.mark.parametrize("order", ["minfill", "naive", "spiral", "extrema", "repulsion"])
def test_full_size_blobs128(gp, order):
    """The benchmark's workload in the benchmark's launch configuration:
    counts, per-round new pairs and the selected sources against the
    oracle's stored simulation; sampled rows of D against Dijkstra; the
    whole array against invariants that hold at any size."""
    import torch
    path = os.path.join(GOLDEN, "counts_blobs128.json")
    if not os.path.exists(path):
        pytest.skip("counts fixture not generated")
    gold_all = json.load(open(path))["orders"]
    if order not in gold_all:
        pytest.skip(f"{order} counts not generated")
    gold = gold_all[order]
    w = synth.batched_128(0)
    with gp.Image(w.img, conn=w.conn, B=w.B, seed=0) as im:
        D, st = im.all_pairs(order, want_log=True)
    for k in ("propagations", "prepass_propagations", "distance_ops", "new_pairs", "rounds"):
        assert st[k] == gold[k], k
    assert [int(x) for x in st["round_new"]] == gold["round_new"]
    assert hashlib.sha256(st["sources"].astype("<i4").tobytes()).hexdigest() == gold["sources_sha256"]
    N = w.N
    rng = np.random.default_rng(1)
    rows = np.unique(np.concatenate([[0, N - 1], rng.integers(0, N, size=40)])).astype(np.int32)
    Dr = _u32(D[torch.from_numpy(rows).long().cuda()])
    assert np.array_equal(Dr, oracle.rows(w.img, rows, conn=w.conn))
    Dc = _u32(D[:, torch.from_numpy(rows).long().cuda()]).T
    assert np.array_equal(Dc, oracle.rows(w.img, rows, conn=w.conn))
    # symmetry and zero diagonal of the whole array, on the device
    assert bool((D == D.T).all())
    assert bool((torch.diagonal(D) == 0).all())
    assert int((D.view(torch.int32) < 0).sum()) == 0  # no unreachable pair on a grey image


# --------------------------------------------------------------------------
# Just above 16384 pixels: the larger images' code paths (eight-strip tree
# clusters with their own depth sums, selection without the key cache,
# one value per lane where the width is not a multiple of 4)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("fill_rows", [0, -1, -2, -3, 1, 8])
@pytest.mark.parametrize("shape,conn,kind", [((29, 31), 8, "grey"), ((40, 24), 4, "mask"), ((136, 121), 8, "grey")])
def test_fill_variants(gp, shape, conn, kind, fill_rows):
    """The tree fill with the marks claimed in global memory (fill_rows 0,
    the default) and staged in shared memory (1 or 8 rows per block): the
    whole array against Dijkstra and the counts against the oracle."""
    H, W = shape
    if kind == "mask":
        mask = synth.disk_mask(H, W, 0.4, 2, 4, seed=H)
        img = np.zeros((H, W), dtype=np.uint8)
    else:
        mask = None
        img = synth.scaled_blobs(H, W, conn, seed=W).img
    with gp.Image(None if mask is not None else img, conn=conn, kind=kind, mask=mask, B=32,
                  fill_rows=fill_rows) as im:
        D, st = im.all_pairs("minfill")
    assert np.array_equal(_u32(D), oracle.apsp(img, conn=conn, kind=kind, mask=mask))
    if H * W <= 4096:
        ref = oracle.fill(img, "minfill", B=32, conn=conn, kind=kind, mask=mask)
        for k in ("propagations", "distance_ops", "new_pairs", "rounds"):
            assert st[k] == getattr(ref, k), k


@pytest.mark.parametrize("order", ["minfill", "extrema"])
def test_counts_blobs136x121(gp, order):
    """136x121 (N = 16456), 8-connected, B = 32: counts, per-round new pairs
    and the selected sources against the oracle's stored simulation, and the
    whole array against Dijkstra from every pixel."""
    path = os.path.join(GOLDEN, "counts_blobs136x121.json")
    if not os.path.exists(path):
        pytest.skip("counts fixture not generated")
    gold_all = json.load(open(path))["orders"]
    if order not in gold_all:
        pytest.skip(f"{order} counts not generated")
    gold = gold_all[order]
    w = synth.scaled_blobs(136, 121, 8, seed=0, B=32)
    with gp.Image(w.img, conn=w.conn, B=w.B, seed=0) as im:
        D, st = im.all_pairs(order, want_log=True)
    for k in ("propagations", "prepass_propagations", "distance_ops", "new_pairs", "rounds"):
        assert st[k] == gold[k], k
    assert [int(x) for x in st["round_new"]] == gold["round_new"]
    assert hashlib.sha256(st["sources"].astype("<i4").tobytes()).hexdigest() == gold["sources_sha256"]
    assert np.array_equal(_u32(D), oracle.apsp(w.img, conn=w.conn))


# --------------------------------------------------------------------------
# Full-size 256x256 workloads (17.2 GB array on the device)
# --------------------------------------------------------------------------

def _with_B(w, B):
    w.B = B
    return w


@pytest.mark.parametrize("name,factory,order,fill_rows", [("steps256", synth.steps_256, o, 0) for o in
                                                         ("minfill", "naive", "spiral", "extrema", "repulsion")] +
                         [("mask256", synth.mask_256, "minfill", 0),
                          ("steps256_B256", lambda seed: _with_B(synth.steps_256(seed), 256), "minfill", 0),
                          ("steps256_B256", lambda seed: _with_B(synth.steps_256(seed), 256), "minfill", -2),
                          ("steps256_B512", lambda seed: _with_B(synth.steps_256(seed), 512), "minfill", -2)])
def test_full_size_256(gp, name, factory, order, fill_rows):
    """256x256, 8-connected, B = 32 (every order; and the obstacle mask),
    B = 256 with the default fill and with the one-sided first round, and
    B = 512 (one round covers every pair): the counts against the oracle's stored
    simulation, sampled rows and columns of D against Dijkstra, and the
    whole array certified."""
    import torch
    path = os.path.join(GOLDEN, f"counts_{name}.json")
    if not os.path.exists(path):
        pytest.skip("counts fixture not generated")
    gold_all = json.load(open(path))["orders"]
    if order not in gold_all:
        pytest.skip(f"{order} counts not generated")
    gold = gold_all[order]
    w = factory(0)
    N = w.N
    img = w.img if w.kind == "grey" else None
    D = torch.empty((N, N), dtype=torch.int32, device="cuda")
    with gp.Image(img, conn=w.conn, kind=w.kind, mask=w.mask, B=w.B, seed=0, fill_rows=fill_rows) as im:
        _, st = im.all_pairs(order, out=D, want_log=True)
    for k in ("propagations", "prepass_propagations", "distance_ops", "new_pairs", "rounds"):
        assert st[k] == gold[k], k
    assert [int(x) for x in st["round_new"]] == gold["round_new"]
    assert hashlib.sha256(st["sources"].astype("<i4").tobytes()).hexdigest() == gold["sources_sha256"]
    rng = np.random.default_rng(2)
    rows = np.unique(np.concatenate([[0, N - 1], rng.integers(0, N, size=24)])).astype(np.int32)
    ref = oracle.rows(w.img, rows, conn=w.conn, kind=w.kind, mask=w.mask)
    idx = torch.from_numpy(rows).long().cuda()
    assert np.array_equal(_u32(D[idx]), ref)
    assert np.array_equal(_u32(D[:, idx]).T, ref)
    # the whole array, certified on the device: every entry satisfies the
    # distance equations, which only the exact distances do
    with gp.Image(img, conn=w.conn, kind=w.kind, mask=w.mask) as im:
        assert im.certify(D) == 0
    del D
    torch.cuda.empty_cache()


# --------------------------------------------------------------------------
# Batched form: many images of uneven sizes side by side
# --------------------------------------------------------------------------

@pytest.mark.parametrize("fill_rows", [0, -1, -2, -3])
def test_all_pairs_batch_equals_alone(gp, fill_rows):
    """Each image of a batch gets the array and counts it gets alone
    (images of uneven sizes, 4- and 8-connected, one mask; every fill variant
    that walks the marks in global memory, the one-sided first round's mirror
    pass captured too)."""
    rng = np.random.default_rng(4)
    specs = []
    for k in range(6):
        H, W = int(rng.integers(5, 30)), int(rng.integers(5, 30))
        specs.append((synth.blobs(H, W, 3, 2.5, 55.0, seed=k), None, 4 if k % 2 else 8))
    specs.append((None, synth.disk_mask(21, 26, 0.4, 2, 3, seed=9), 8))
    ims = [gp.Image(img, conn=c, kind="grey" if m is None else "mask", mask=m, B=4, fill_rows=fill_rows)
           for img, m, c in specs]
    try:
        outs, stats = gp.all_pairs_batch(ims, "minfill")
        for (img, m, c), D, st in zip(specs, outs, stats):
            base = img if m is None else np.zeros_like(m)
            kind = "grey" if m is None else "mask"
            assert np.array_equal(_u32(D), oracle.apsp(base, conn=c, kind=kind, mask=m))
            ref = oracle.fill(base, "minfill", B=4, conn=c, kind=kind, mask=m)
            for key in ("propagations", "distance_ops", "new_pairs", "rounds"):
                assert st[key] == getattr(ref, key), key
    finally:
        for im in ims:
            im.close()


@pytest.mark.parametrize("order", ["minfill", "naive", "spiral", "extrema", "repulsion"])
def test_batch_graph_every_order(gp, order):
    """The batch runs as one CUDA graph over all images: twelve images of
    uneven sizes (one 136 x 121, above the small-image paths), each equal to
    its fill alone; the handles work normally afterwards."""
    rng = np.random.default_rng(7)
    specs = [(int(rng.integers(6, 48)), int(rng.integers(6, 48)), 4 if k % 3 == 0 else 8) for k in range(11)]
    specs.append((136, 121, 8))
    imgs = [synth.scaled_blobs(H, W, c, seed=k).img for k, (H, W, c) in enumerate(specs)]
    ims = [gp.Image(img, conn=c, B=16 if k % 2 else 32, seed=k) for k, (img, (H, W, c)) in
           enumerate(zip(imgs, specs))]
    try:
        outs, stats = gp.all_pairs_batch(ims, order)
        for im, img, (H, W, c), D, st in zip(ims, imgs, specs, outs, stats):
            alone, sa = im.all_pairs(order)
            assert np.array_equal(_u32(D), _u32(alone))
            for key in ("propagations", "distance_ops", "new_pairs", "rounds"):
                assert st[key] == sa[key], key
            if H * W <= 1024:
                assert np.array_equal(_u32(D), oracle.apsp(img, conn=c))
        # a second batch on the same handles gives the same again
        outs2, stats2 = gp.all_pairs_batch(ims, order)
        for D, D2, st, st2 in zip(outs, outs2, stats, stats2):
            assert np.array_equal(_u32(D), _u32(D2))
            assert st["propagations"] == st2["propagations"]
    finally:
        for im in ims:
            im.close()


def test_tune_picks_a_candidate_and_caches(gp, tmp_path):
    """The autotuner returns one of its candidates, and the result of a fill
    with the tuned options is the same array; a second call reads the
    cache instead of measuring again."""
    img = synth.scaled_blobs(40, 44, 8, seed=3).img
    cache = tmp_path / "tune.txt"
    t = gp.tune(img, conn=8, cache=cache)
    assert t["B"] in (16, 32, 64, 128, 256, 512, 1024) and t["lookahead"] in (0, -1) and t["fill_rows"] in (0, 8, -1, -2, -3)
    assert t["ms"] > 0
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith("gapsp-tune-2 40 44 8 0 2 ")
    t2 = gp.tune(img, conn=8, cache=cache)
    keys = ("B", "lookahead", "fill_rows")
    assert {k: t2[k] for k in keys} == {k: t[k] for k in keys} and abs(t2["ms"] - t["ms"]) < 1e-3
    assert len(cache.read_text().splitlines()) == 1
    with gp.Image(img, conn=8, B=t["B"], lookahead=t["lookahead"], fill_rows=t["fill_rows"]) as im:
        D, _ = im.all_pairs("minfill")
    assert np.array_equal(_u32(D), oracle.apsp(img, conn=8))


# --------------------------------------------------------------------------
# Multichannel images: the sum pseudo-metric over L channels (16-bit levels)
# --------------------------------------------------------------------------

def _channels(L, H, W, seed):
    return np.stack([synth.blobs(H, W, max(1, H * W // 300), max(1.5, (H + W) / 16), 55.0, seed=seed + l)
                     for l in range(L)])


@pytest.mark.parametrize("shape,L", [((7, 13), 2), ((64, 64), 3), ((129, 130), 8), ((256, 256), 5)],
                         ids=lambda x: str(x))
@pytest.mark.parametrize("conn", [4, 8])
def test_rows_channels(gp, shape, L, conn):
    H, W = shape
    ch = _channels(L, H, W, seed=H + W)
    N = H * W
    rng = np.random.default_rng(N)
    src = np.unique(np.concatenate([[0, N - 1], rng.integers(0, N, size=12)])).astype(np.int32)
    with gp.Image(ch, conn=conn, kind="sum") as im:
        out = _u32(im.rows(src))
    assert np.array_equal(out, oracle.rows(ch, src, conn=conn, kind="sum"))


@pytest.mark.parametrize("order", ["naive", "spiral", "repulsion", "extrema", "minfill"])
@pytest.mark.parametrize("conn", [4, 8])
def test_all_pairs_channels(gp, order, conn):
    ch = _channels(3, 19, 23, seed=conn)
    with gp.Image(ch, conn=conn, kind="sum", B=5, seed=3) as im:
        D, st = im.all_pairs(order, want_log=True)
    assert np.array_equal(_u32(D), oracle.apsp(ch, conn=conn, kind="sum"))
    ref = oracle.fill(ch, order, B=5, seed=3, conn=conn, kind="sum")
    for k in ("propagations", "prepass_propagations", "distance_ops", "new_pairs", "rounds"):
        assert st[k] == getattr(ref, k), k
    assert st["sources"].tolist() == ref.sources.tolist()


def test_channels_whole_array_136x121(gp):
    """Above 16384 pixels (eight-strip trees, 16-bit levels staged there too)."""
    ch = _channels(4, 136, 121, seed=9)
    with gp.Image(ch, conn=8, kind="sum", B=32) as im:
        D, _ = im.all_pairs("minfill")
    assert np.array_equal(_u32(D), oracle.apsp(ch, conn=8, kind="sum"))


def test_channels_largest_levels(gp):
    """32 channels at 255 (F = 8160, the largest distances the kernels take):
    constant image, so d = (2 * 8160 + 1) x chessboard steps; and 33
    channels are refused."""
    H, W = 64, 256
    ch = np.full((32, H, W), 255, dtype=np.uint8)
    src = np.array([0, W - 1, H * W - 1, (H // 2) * W + 7], dtype=np.int32)
    with gp.Image(ch, conn=8, kind="sum") as im:
        out = _u32(im.rows(src))
    r, c = np.divmod(np.arange(H * W), W)
    for k, s in enumerate(src):
        steps = np.maximum(np.abs(r - s // W), np.abs(c - s % W))
        assert np.array_equal(out[k], (2 * 8160 + 1) * steps)
    with pytest.raises(gp.GapspError) as e:
        gp.Image(np.zeros((33, 8, 8), np.uint8), conn=8, kind="sum")
    assert e.value.code == 1


# --------------------------------------------------------------------------
# Certificate of a result (gapsp_certify, opts.checked)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["grey", "mask", "l1", "sum"])
@pytest.mark.parametrize("conn", [4, 8])
def test_certify_detects_wrong_entries(gp, kind, conn):
    """Exact arrays and rows certify with no violation; one entry made too
    large or too small, or a wrong unreachable marker, is caught."""
    import torch
    H, W = 23, 19
    mask = synth.disk_mask(H, W, 0.3, 1, 3, seed=conn) if kind == "mask" else None
    if kind == "sum":
        img = _channels(3, H, W, seed=conn)
    else:
        img = synth.blobs(H, W, 3, 3.0, 55.0, seed=conn)
    with gp.Image(None if kind == "mask" else img, conn=conn, kind=kind, mask=mask, B=8, checked=1) as im:
        D, _ = im.all_pairs("minfill")  # checked: certified before it returns
        assert im.certify(D) == 0
        src = np.array([0, 7, 100, H * W - 1], dtype=np.int32)
        R = im.rows(src)
        assert im.certify(R, src) == 0
        N = H * W
        free = np.arange(N) if mask is None else np.flatnonzero(mask.reshape(-1))
        p = int(free[3])
        Dh = _u32(D)
        joined = np.flatnonzero((Dh[p] != 0xFFFFFFFF) & (np.arange(N) != p))
        q = int(joined[-1])  # a pixel a path joins to p
        for delta in (1, -1):
            E = D.clone()
            E[p, q] = int(Dh[p, q]) + delta
            assert im.certify(E) >= 1
        E = D.clone()
        E[p, q] = -1  # UNREACH where a path exists
        assert im.certify(E) >= 1
        E = R.clone()
        E[1, 7] = 3  # the source's own entry
        assert im.certify(E, src) >= 1
