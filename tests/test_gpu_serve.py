"""The request server (gapsp_server_*): results in the mix equal results alone.

Requests of different kinds and sizes run side by side on the GPU (rows
queries and all-pairs fills of several images, orders and pseudo-metrics,
some submitted while others are running). Every result must be bit-identical
to the same request run alone through gapsp_all_pairs / gapsp_rows, and the
small ones also to the CPU oracle. Admission: a request above the whole
budget is rejected, and a tight budget makes requests wait their turn
without ever holding more than the budget.
"""
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


def _mix(seed=0):
    """(kind, image, mask, conn, img_kind, order, sources) of a request mix."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(14):
        if k % 3 == 0:
            s = int(rng.integers(64, 129))
            img = synth.scaled_blobs(s, s, 8, seed=100 + k).img
            src = rng.integers(0, s * s, size=int(rng.integers(1, 300))).astype(np.int32)
            out.append(("rows", img, None, 8, "grey", "minfill", src))
        else:
            H, W = int(rng.integers(12, 56)), int(rng.integers(12, 56))
            order = ["minfill", "naive", "spiral", "extrema", "repulsion"][k % 5]
            if k == 4:
                m = synth.disk_mask(H, W, 0.4, 2, 4, seed=k)
                out.append(("all", np.zeros((H, W), np.uint8), m, 8, "mask", order, None))
            elif k == 5:
                out.append(("all", synth.blobs(H, W, 3, 3.0, 55.0, seed=k), None, 8, "l1", order, None))
            else:
                out.append(("all", synth.blobs(H, W, 3, 3.0, 55.0, seed=k), None, 4 if k % 2 else 8,
                            "grey", order, None))
    return out


def _alone(gp, req):
    kind, img, mask, conn, ik, order, src = req
    with gp.Image(None if ik == "mask" else img, conn=conn, kind=ik, mask=mask, B=32) as im:
        if kind == "rows":
            return _u32(im.rows(src)), None
        D, st = im.all_pairs(order)
        return _u32(D), st


def _submit(srv, torch, req):
    kind, img, mask, conn, ik, order, src = req
    N = img.size
    if kind == "rows":
        out = torch.full((len(src), N), 3, dtype=torch.int32, device="cuda")
        rid = srv.submit_rows(img, src, conn=conn, kind=ik, mask=mask, out=out)
    else:
        out = torch.full((N, N), 3, dtype=torch.int32, device="cuda")
        rid = srv.submit_all_pairs(img, conn=conn, order=order, kind=ik, mask=mask, out=out)
    return rid, out


def test_results_in_the_mix_equal_alone(env):
    gp, torch = env
    reqs = _mix(0)
    torch.cuda.synchronize()
    with gp.Server(mem_budget=8 << 30, slots=6, B=32) as srv:
        first = [_submit(srv, torch, r) for r in reqs[:8]]
        # more requests while the first ones are on the GPU
        srv.wait(first[0][0])
        later = [_submit(srv, torch, r) for r in reqs[8:]]
        subs = first + later
        res = [srv.wait(rid, timeout_ms=120000) for rid, _ in subs]
        for r in res:
            assert r["done"] and r["status"] == 0, r
        got = [_u32(out) for _, out in subs]
        for (rid, _), r in zip(subs, res):
            srv.release(rid)
        st = srv.stats()
    assert st["admitted"] == len(reqs) and st["rejected"] == 0 and st["failed"] == 0
    assert st["bytes_in_use"] == 0
    for req, g, r in zip(reqs, got, res):
        ref, rst = _alone(gp, req)
        assert np.array_equal(g, ref), req[0]
        if rst is not None:
            assert r["propagations"] == rst["propagations"] and r["rounds"] == rst["rounds"]
        kind, img, mask, conn, ik, order, src = req
        if kind == "all" and img.size <= 900:
            assert np.array_equal(g, oracle.apsp(img, conn=conn, kind=ik, mask=mask))


def test_admission_by_footprint(env):
    gp, torch = env
    imgs = [synth.blobs(40, 40, 4, 4.0, 55.0, seed=k) for k in range(6)]
    ref = _alone(gp, ("all", imgs[0], None, 8, "grey", "minfill", None))[0]
    # one 40x40 fill holds its 10 MB result plus a few MB of state: a 40 MB
    # budget admits a few at a time; 1200 rows of a 256x256 image (315 MB)
    # are above it
    budget = 40 << 20
    with gp.Server(mem_budget=budget, slots=8) as srv:
        big = synth.blobs(256, 256, 8, 8.0, 55.0, seed=1)
        with pytest.raises(gp.GapspError) as e:
            srv.submit_rows(big, np.arange(1200, dtype=np.int32))
        assert e.value.code == 3
        ids = [srv.submit_all_pairs(im) for im in imgs]
        # results count against the budget until released: read the first
        # one, then release each result as it completes
        first = srv.wait(ids[0], timeout_ms=60000)
        assert first["status"] == 0 and first["ptr"] and first["result_bytes"] == ref.nbytes
        host = np.empty(ref.shape, dtype=np.uint32)
        srv.read(ids[0], host)  # a server-owned result, read back through the C ABI
        assert np.array_equal(host, ref)
        res = {ids[0]: first}
        srv.release(ids[0])
        import time
        t_end = time.time() + 60
        while len(res) < len(ids) and time.time() < t_end:
            for r in srv.poll():
                if r["id"] not in res:
                    res[r["id"]] = r
                    srv.release(r["id"])
            time.sleep(0.001)
        res = [res[i] for i in ids]
        st = srv.stats()
        assert all(r["status"] == 0 for r in res)
        assert st["peak_bytes"] <= budget and st["rejected"] == 1
        # the queue held requests back: no more than budget // footprint ran
        # at once, so later admissions came after completions
        cap = budget // res[0]["footprint"]
        assert cap < len(ids)
        admits = sorted(r["t_admit_ms"] for r in res)
        dones = sorted(r["t_done_ms"] for r in res)
        assert admits[cap] >= dones[0]
        assert srv.stats()["bytes_in_use"] == 0
