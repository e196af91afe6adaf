"""gapsp_rows_noalloc against gapsp_rows.

The no-allocation entry point serves callers that cannot allocate device
memory when they call (an engine that owns the device through its own fixed
pool, code where an allocation would stall the device). It must give exactly
the rows of the regular entry point, call after call, although every call
reuses the same fixed scratch array. Distances are integers: the comparison
is bit-exact.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2007_16076_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2007_16076_gb300 as gp
    gp.load()
    return gp, torch


def _cases():
    return [
        ("grey-8", synth.blobs(64, 64, 6, 4.0, 55.0, seed=11), None, 8),
        ("grey-4", synth.blobs(37, 50, 4, 3.0, 55.0, seed=12), None, 4),
        ("mask-8", None, synth.disk_mask(40, 45, 0.4, 2, 5, seed=13), 8),
        ("l1-8", synth.blobs(33, 41, 4, 3.0, 55.0, seed=14), None, 8),
        # a map too large for one block's shared memory: row strips on a cluster
        ("grey-8-256", synth.blobs(256, 256, 64, 16.0, 40.0, seed=15), None, 8),
    ]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_noalloc_matches_rows_twice(env, case):
    gp, torch = env
    name, img, mask, conn = case
    kind = "mask" if mask is not None else ("l1" if name.startswith("l1") else "grey")
    plane = img if mask is None else mask
    H, W = plane.shape
    N = H * W
    dev_img = torch.from_numpy(np.ascontiguousarray(plane)).cuda()
    with gp.Image(img if mask is None else None, conn=conn, kind=kind, mask=mask) as im:
        for call, seed in enumerate((1, 2)):
            rng = np.random.default_rng(seed)
            src = rng.integers(0, N, size=40 + 9 * call).astype(np.int32)
            ref = gp.as_uint32(im.rows(src))
            out = torch.full((len(src), N), 7, dtype=torch.int32, device="cuda")
            srcs = torch.from_numpy(src).cuda() if call == 0 else src  # device, then host sources
            gp.rows_noalloc(dev_img, srcs, out, conn=conn, kind=kind)
            torch.cuda.synchronize()
            assert np.array_equal(gp.as_uint32(out), ref), f"call {call}"


def test_noalloc_rejects_beyond_limits(env):
    gp, torch = env
    img = synth.blobs(16, 16, 2, 2.0, 55.0, seed=3)
    dev_img = torch.from_numpy(img).cuda()
    K = gp.NOALLOC_MAX_SOURCES + 1
    src = torch.zeros(K, dtype=torch.int32, device="cuda")
    out = torch.empty((1, 256), dtype=torch.int32, device="cuda")
    with pytest.raises(gp.GapspError) as e:
        rc = gp.load().gapsp_rows_noalloc(ctypes.c_void_p(dev_img.data_ptr()), 16, 16, 8, 0,
                                          ctypes.c_void_p(src.data_ptr()), K,
                                          ctypes.c_void_p(out.data_ptr()), None)
        if rc != 0:
            raise gp.GapspError(rc, "gapsp_rows_noalloc")
    assert e.value.code == 1
    # a source outside the image is rejected and nothing is written
    out = torch.full((2, 256), 5, dtype=torch.int32, device="cuda")
    with pytest.raises(gp.GapspError) as e:
        gp.rows_noalloc(dev_img, np.array([3, 256], dtype=np.int32), out)
    assert e.value.code == 1
    assert bool((out == 5).all())


@pytest.mark.parametrize("K", [1, 305, 4096])
def test_noalloc_source_counts(env, K):
    """One source, the count past which the kernel runs one warp per sweep
    direction (more than two sources per multiprocessor), and the maximum;
    on a side stream."""
    gp, torch = env
    img = synth.blobs(20, 24, 3, 3.0, 55.0, seed=16)
    N = img.size
    src = (np.arange(K, dtype=np.int64) * 7 + 3) % N
    dev_img = torch.from_numpy(img).cuda()
    s = torch.cuda.Stream()
    with gp.Image(img, conn=8) as im:
        ref = gp.as_uint32(im.rows(src.astype(np.int32)))
    for call in range(2):
        out = torch.full((K, N), 9, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        # int64 host sources are converted, not read as pairs of int32 words
        gp.rows_noalloc(dev_img, src, out, conn=8, stream=s)
        s.synchronize()
        assert np.array_equal(gp.as_uint32(out), ref), f"call {call}"


def test_noalloc_rejects_bad_buffers(env):
    gp, torch = env
    img = synth.blobs(16, 16, 2, 2.0, 55.0, seed=3)
    dev_img = torch.from_numpy(img).cuda()
    src = np.array([1, 2, 3], dtype=np.int32)
    # an output too small for K rows
    with pytest.raises(ValueError):
        gp.rows_noalloc(dev_img, src, torch.empty((2, 256), dtype=torch.int32, device="cuda"))
    # a host image or output, and device sources of the wrong type
    with pytest.raises(ValueError):
        gp.rows_noalloc(torch.from_numpy(img), src, torch.empty((3, 256), dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        gp.rows_noalloc(dev_img, src, torch.empty((3, 256), dtype=torch.int32))
    with pytest.raises(ValueError):
        gp.rows_noalloc(dev_img, torch.from_numpy(src.astype(np.int64)).cuda(),
                        torch.empty((3, 256), dtype=torch.int32, device="cuda"))
    # the C entry point itself refuses an output that is not device memory
    host_out = np.zeros((3, 256), dtype=np.uint32)
    rc = gp.load().gapsp_rows_noalloc(ctypes.c_void_p(dev_img.data_ptr()), 16, 16, 8, 0,
                                      ctypes.c_void_p(src.ctypes.data), 3,
                                      ctypes.c_void_p(host_out.ctypes.data), None)
    assert rc == 1
    assert not host_out.any()
