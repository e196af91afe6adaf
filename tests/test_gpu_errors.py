"""Error paths on the GPU, made to happen without faulting anything.

- the sweep limit of a propagation (opts.max_sweep_rounds) runs out on the
  device: the kernel stops, sets a status bit and the call returns
  GAPSP_E_NOT_CONVERGED;
- the round limit of the all-pairs loop (opts.max_rounds) runs out:
  GAPSP_E_TIMEOUT;
- gapsp_cancel from another thread: GAPSP_E_CANCELLED;
- a host-side allocation failure injected by gapsp_debug_fail_alloc:
  GAPSP_E_NOMEM, with nothing leaked.
While one handle fails, another handle's fill runs on its own stream in a
second thread and must give the oracle's array. After each error the handle
must still work.
"""
import threading

import numpy as np
import pytest

import oracle
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


def _u32(t):
    return t.detach().cpu().numpy().view(np.uint32)


class Bystander:
    """A second handle filling a 48x40 image on its own stream in a thread."""

    def __init__(self, gp, torch, order="naive"):
        self.img = synth.blobs(48, 40, 4, 4.0, 55.0, seed=21)
        self.gp, self.torch, self.order = gp, torch, order
        self.stream = torch.cuda.Stream()
        self.err = None
        self.D = None

    def _run(self):
        try:
            with self.torch.cuda.stream(self.stream):
                with self.gp.Image(self.img, conn=8, B=1, stream=self.stream) as im:
                    for _ in range(3):
                        self.D, _ = im.all_pairs(self.order)
                self.stream.synchronize()
        except Exception as e:  # reported by check()
            self.err = e

    def __enter__(self):
        self.t = threading.Thread(target=self._run)
        self.t.start()
        return self

    def __exit__(self, *exc):
        self.t.join()

    def check(self):
        assert self.err is None, self.err
        assert np.array_equal(_u32(self.D), oracle.apsp(self.img, conn=8))


def test_sweep_limit_not_converged(env):
    gp, torch = env
    img = synth.blobs(40, 36, 4, 4.0, 55.0, seed=5)
    src = np.array([0, 700, 1439], dtype=np.int32)
    with Bystander(gp, torch) as by:
        with gp.Image(img, conn=8, B=4, max_sweep_rounds=1) as im:
            with pytest.raises(gp.GapspError) as e:
                im.rows(src)
            assert e.value.code == 5
            with pytest.raises(gp.GapspError) as e:
                im.all_pairs("minfill")
            assert e.value.code == 5
        # a handle with the default limit on the same image is exact
        with gp.Image(img, conn=8, B=4) as im:
            assert np.array_equal(_u32(im.rows(src)), oracle.rows(img, src, conn=8))
    by.check()


def test_round_limit_timeout(env):
    gp, torch = env
    img = synth.blobs(30, 30, 4, 4.0, 55.0, seed=6)
    with Bystander(gp, torch, order="minfill") as by:
        with gp.Image(img, conn=8, B=1, max_rounds=3) as im:
            with pytest.raises(gp.GapspError) as e:
                im.all_pairs("naive")
            assert e.value.code == 6
            # the same handle, same limit, on a 1 x 5 image's worth of rounds: the
            # limit is checked per chunk of 8 rounds, so a fill of <= 8 rounds passes
        with gp.Image(img[:1, :5], conn=8, B=1, max_rounds=3) as im:
            D, st = im.all_pairs("minfill")
            assert st["rounds"] <= 8
            assert np.array_equal(_u32(D), oracle.apsp(img[:1, :5], conn=8))
    by.check()


def test_cancel(env):
    gp, torch = env
    img = synth.batched_128(0).img
    im = gp.Image(img, conn=8, B=1, lookahead=-1)
    out = {}

    def run():
        try:
            im.all_pairs("naive")
            out["rc"] = 0
        except gp.GapspError as e:
            out["rc"] = e.code

    try:
        t = threading.Thread(target=run)
        t.start()
        import time
        time.sleep(0.2)  # a B = 1 naive fill of 16384 pixels runs for seconds
        im.cancel()
        t.join()
        assert out["rc"] == 7
        # the handle still works, and a cancel with no call running has no effect
        im.cancel()
        small = gp.Image(img[:20, :24], conn=8, B=4)
        D, _ = small.all_pairs("minfill")
        small.close()
        assert np.array_equal(_u32(D), oracle.apsp(img[:20, :24], conn=8))
    finally:
        im.close()


def test_alloc_failure_nomem_nothing_leaked(env):
    gp, torch = env
    img = synth.blobs(24, 28, 3, 3.0, 55.0, seed=8)
    ref = oracle.apsp(img, conn=8)
    D = torch.empty((img.size, img.size), dtype=torch.int32, device="cuda")
    live0 = gp.debug_fail_alloc(-1)
    seen_nomem = 0
    try:
        for k in list(range(0, 48, 3)) + [1000]:
            with gp.Image(img, conn=8, B=4) as im:
                live1 = gp.debug_fail_alloc(k)
                try:
                    im.all_pairs("minfill", out=D)
                    ok = True
                except gp.GapspError as e:
                    assert e.code == 2, e
                    ok = False
                    seen_nomem += 1
                    # the failed call freed what it had allocated
                    assert gp.debug_fail_alloc(-1) == live1
                gp.debug_fail_alloc(-1)
                # the handle recovers: the next call allocates what is missing
                D.fill_(0)
                im.all_pairs("minfill", out=D)
                assert np.array_equal(_u32(D), ref), f"after failing allocation {k}"
            assert gp.debug_fail_alloc(-1) == live0
            if ok:
                break
        # a failure inside gapsp_create leaves no handle and no allocation behind
        for k in range(0, 6):
            gp.debug_fail_alloc(k)
            with pytest.raises(gp.GapspError) as e:
                gp.Image(img, conn=8)
            assert e.value.code == 2
            assert gp.debug_fail_alloc(-1) == live0
    finally:
        gp.debug_fail_alloc(-1)
    assert seen_nomem >= 3
