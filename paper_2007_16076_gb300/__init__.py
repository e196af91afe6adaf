"""Python binding of libgapsp (all pairs of geodesic distances on one GPU).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libgapsp.so`` behind the C ABI of ``include/gapsp.h``. There is
no CPU fallback; if the library cannot be loaded the calls raise.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA). Output
arrays default to CUDA tensors of dtype int32 holding the uint32 bit
patterns; :func:`as_uint32` views them as numpy uint32.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

UNREACH = 0xFFFFFFFF
ORDERS = {"naive": 0, "spiral": 1, "minfill": 2, "extrema": 3, "repulsion": 4}
KINDS = {"grey": 0, "mask": 1, "l1": 2, "sum": 3}
KERNELS = ("select", "propagate", "tree", "lookahead", "fill", "init", "prepass", "depths", "recount", "mirror")
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "memory budget exceeded",
          4: "CUDA runtime error", 5: "propagation did not converge", 6: "round limit exceeded",
          7: "cancelled", 8: "result failed its certificate"}

_lib = None


class GapspError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        detail = ""
        if code in (2, 4) and _lib is not None:
            d = _lib.gapsp_last_error_detail()
            detail = f" [{d.decode(errors='replace')}]" if d else ""
        super().__init__(f"{where}: {STATUS.get(code, code)} (status {code}){detail}")


class Opts(ctypes.Structure):
    _fields_ = [("conn", ctypes.c_int), ("kind", ctypes.c_int), ("B", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("mem_budget", ctypes.c_size_t),
                ("sweep_phases", ctypes.c_int), ("fill_rows", ctypes.c_int), ("checked", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("prop_blocks", ctypes.c_int),
                ("lookahead", ctypes.c_int), ("warm_start", ctypes.c_int),
                ("max_sweep_rounds", ctypes.c_int), ("max_rounds", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("propagations", ctypes.c_uint64), ("prepass_propagations", ctypes.c_uint64),
                ("distance_ops", ctypes.c_uint64), ("new_pairs", ctypes.c_uint64),
                ("rounds", ctypes.c_uint64), ("prefilled_pairs", ctypes.c_uint64),
                ("ms_total", ctypes.c_double),
                ("round_new", ctypes.POINTER(ctypes.c_uint64)), ("round_new_cap", ctypes.c_uint64),
                ("sources", ctypes.POINTER(ctypes.c_int32)), ("sources_cap", ctypes.c_uint64),
                ("sweeps", ctypes.c_uint64), ("lines", ctypes.c_uint64),
                ("lookahead_propagations", ctypes.c_uint64), ("lookahead_hits", ctypes.c_uint64)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("img", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("H", ctypes.c_int), ("W", ctypes.c_int), ("conn", ctypes.c_int),
                ("img_kind", ctypes.c_int), ("order", ctypes.c_int), ("sources", ctypes.c_void_p),
                ("K", ctypes.c_int), ("out", ctypes.c_void_p)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_size_t), ("slots", ctypes.c_int), ("B", ctypes.c_int),
                ("lookahead", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("done", ctypes.c_int), ("status", ctypes.c_int),
                ("result", ctypes.c_void_p), ("result_bytes", ctypes.c_size_t),
                ("footprint", ctypes.c_size_t), ("t_submit_ms", ctypes.c_double),
                ("t_admit_ms", ctypes.c_double), ("t_done_ms", ctypes.c_double),
                ("propagations", ctypes.c_uint64), ("rounds", ctypes.c_uint64)]


class ServerCounts(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("bytes_in_use", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t),
                ("budget", ctypes.c_size_t)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libgapsp.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libgapsp.so is not built; run paper_2007_16076_gb300._build.build()")
    lib = ctypes.CDLL(_build.LIB)
    P = ctypes.c_void_p
    lib.gapsp_default_opts.argtypes = [ctypes.POINTER(Opts)]
    lib.gapsp_create.argtypes = [P, ctypes.c_int, ctypes.c_int, P, ctypes.POINTER(Opts),
                                 ctypes.POINTER(P)]
    lib.gapsp_create.restype = ctypes.c_int
    lib.gapsp_create_channels.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Opts),
                                          ctypes.POINTER(P)]
    lib.gapsp_create_channels.restype = ctypes.c_int
    lib.gapsp_all_pairs.argtypes = [P, ctypes.c_int, P, ctypes.POINTER(Stats)]
    lib.gapsp_all_pairs.restype = ctypes.c_int
    lib.gapsp_rows.argtypes = [P, P, ctypes.c_int, P]
    lib.gapsp_rows.restype = ctypes.c_int
    lib.gapsp_destroy.argtypes = [P]
    lib.gapsp_destroy.restype = None
    lib.gapsp_strerror.argtypes = [ctypes.c_int]
    lib.gapsp_strerror.restype = ctypes.c_char_p
    lib.gapsp_kernel_launches.argtypes = [P]
    lib.gapsp_kernel_launches.restype = ctypes.c_uint64
    lib.gapsp_profile_enable.argtypes = [P, ctypes.c_int]
    lib.gapsp_profile_enable.restype = ctypes.c_int
    lib.gapsp_profile_read.argtypes = [P, P, P]
    lib.gapsp_profile_read.restype = ctypes.c_int
    lib.gapsp_profile_trace.argtypes = [P, P, P, P, P, ctypes.c_uint64, P]
    lib.gapsp_profile_trace.restype = ctypes.c_int
    lib.gapsp_all_pairs_batch.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P]
    lib.gapsp_all_pairs_batch.restype = ctypes.c_int
    lib.gapsp_rows_noalloc.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       P, ctypes.c_int, P, P]
    lib.gapsp_rows_noalloc.restype = ctypes.c_int
    lib.gapsp_server_default_opts.argtypes = [ctypes.POINTER(ServerOpts)]
    lib.gapsp_server_default_opts.restype = None
    lib.gapsp_server_create.argtypes = [ctypes.POINTER(ServerOpts), ctypes.POINTER(P)]
    lib.gapsp_server_create.restype = ctypes.c_int
    lib.gapsp_server_submit.argtypes = [P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    lib.gapsp_server_submit.restype = ctypes.c_int
    lib.gapsp_server_wait.argtypes = [P, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(Result)]
    lib.gapsp_server_wait.restype = ctypes.c_int
    lib.gapsp_server_poll.argtypes = [P, ctypes.POINTER(Result), ctypes.c_int]
    lib.gapsp_server_poll.restype = ctypes.c_int
    lib.gapsp_server_read.argtypes = [P, ctypes.c_uint64, P, ctypes.c_size_t]
    lib.gapsp_server_read.restype = ctypes.c_int
    lib.gapsp_server_release.argtypes = [P, ctypes.c_uint64]
    lib.gapsp_server_release.restype = ctypes.c_int
    lib.gapsp_server_stats.argtypes = [P, ctypes.POINTER(ServerCounts)]
    lib.gapsp_server_stats.restype = ctypes.c_int
    lib.gapsp_server_destroy.argtypes = [P]
    lib.gapsp_server_destroy.restype = None
    lib.gapsp_tune.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Opts), ctypes.c_int,
                               ctypes.c_char_p, ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_double)]
    lib.gapsp_tune.restype = ctypes.c_int
    lib.gapsp_last_error_detail.argtypes = []
    lib.gapsp_last_error_detail.restype = ctypes.c_char_p
    lib.gapsp_certify.argtypes = [P, P, P, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]
    lib.gapsp_certify.restype = ctypes.c_int
    lib.gapsp_cancel.argtypes = [P]
    lib.gapsp_cancel.restype = ctypes.c_int
    lib.gapsp_debug_fail_alloc.argtypes = [ctypes.c_int]
    lib.gapsp_debug_fail_alloc.restype = ctypes.c_longlong
    _lib = lib
    return lib


def _ptr(x):
    """Raw address of a numpy array or torch tensor (host or device)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    raise TypeError(f"unsupported array type {type(x)}")


def as_uint32(x) -> np.ndarray:
    """Host numpy uint32 view/copy of an int32/uint32 array or tensor."""
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.asarray(x).view(np.uint32)


def _torch_stream(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def all_pairs_batch(images, order: str = "minfill", outs=None):
    """gapsp_all_pairs_batch: fills the arrays of several images at once.

    `images` is a list of :class:`Image` handles; `outs` (optional) one
    N_i x N_i array per image (CUDA tensors by default). Returns (outs, stats
    list); every result equals that of ``Image.all_pairs`` alone.
    """
    lib = load()
    n = len(images)
    if outs is None:
        import torch
        outs = [torch.empty((im.N, im.N), dtype=torch.int32, device="cuda") for im in images]
    hs = (ctypes.c_void_p * max(n, 1))(*[im._h for im in images])
    ds = (ctypes.c_void_p * max(n, 1))(*[_ptr(o) for o in outs])
    sts = (Stats * max(n, 1))()
    rc = lib.gapsp_all_pairs_batch(hs, n, ORDERS[order], ds, sts)
    if rc != 0:
        raise GapspError(rc, "gapsp_all_pairs_batch")
    stats = [{"propagations": sts[i].propagations, "prepass_propagations": sts[i].prepass_propagations,
              "distance_ops": sts[i].distance_ops, "new_pairs": sts[i].new_pairs,
              "rounds": sts[i].rounds, "ms_total": sts[i].ms_total} for i in range(n)]
    return outs, stats


NOALLOC_MAX_SOURCES = 4096


def tune(img, conn: int = 8, kind: str = "grey", mask=None, order: str = "minfill", cache=None) -> dict:
    """gapsp_tune: the fastest B, lookahead and fill variant for this image's
    fill, measured on the GPU (or read from the text cache `cache`).
    Returns the keyword arguments for :class:`Image` and the time (ms)."""
    lib = load()
    a = None if kind == "mask" else np.ascontiguousarray(img, dtype=np.uint8)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    H, W = (m if kind == "mask" else a).shape
    o = Opts()
    lib.gapsp_default_opts(ctypes.byref(o))
    o.conn, o.kind = conn, KINDS[kind]
    best = Opts()
    ms = ctypes.c_double()
    rc = lib.gapsp_tune(_ptr(a), _ptr(m), H, W, ctypes.byref(o), ORDERS[order],
                        None if cache is None else str(cache).encode(), ctypes.byref(best), ctypes.byref(ms))
    if rc != 0:
        raise GapspError(rc, "gapsp_tune")
    return {"B": best.B, "lookahead": best.lookahead, "fill_rows": best.fill_rows, "ms": ms.value}


def debug_fail_alloc(n: int) -> int:
    """Host-side fault injection (gapsp_debug_fail_alloc): the library's
    allocation after n more successful ones fails; n < 0 turns it off.
    Returns the number of allocations the library holds."""
    return int(load().gapsp_debug_fail_alloc(int(n)))


def rows_noalloc(img, sources, out, conn: int = 8, kind: str = "grey", stream=None):
    """gapsp_rows_noalloc: rows d(sources[k], .) into `out` with no allocation.

    `img` (uint8, H x W; free flags for the mask kind) and `out` (K x N,
    int32 or uint32) must be contiguous CUDA tensors the caller owns;
    `sources` is a host array (converted to int32) or a CUDA int32 tensor.
    For callers that cannot allocate device memory at call time; calls share
    one fixed scratch array, so order them on one stream.
    """
    lib = load()
    if not (hasattr(img, "is_cuda") and img.is_cuda and img.dim() == 2 and
            str(img.dtype) == "torch.uint8" and img.is_contiguous()):
        raise ValueError("img must be a contiguous 2-D CUDA uint8 tensor")
    H, W = int(img.shape[0]), int(img.shape[1])
    if hasattr(sources, "data_ptr"):
        if not sources.is_cuda or str(sources.dtype) != "torch.int32" or not sources.is_contiguous():
            raise ValueError("a tensor of sources must be a contiguous CUDA int32 tensor")
        src = sources
        K = int(src.numel())
    else:
        src = np.ascontiguousarray(np.asarray(sources).reshape(-1))
        if src.size and (src.min() < np.iinfo(np.int32).min or src.max() > np.iinfo(np.int32).max):
            raise ValueError("source index out of the int32 range")
        src = src.astype(np.int32)
        K = int(src.size)
    if not (hasattr(out, "is_cuda") and out.is_cuda and str(out.dtype) in ("torch.int32", "torch.uint32")
            and out.is_contiguous()):
        raise ValueError("out must be a contiguous CUDA int32 (or uint32) tensor")
    if int(out.numel()) < K * H * W:
        raise ValueError(f"out holds {int(out.numel())} entries, {K * H * W} needed")
    rc = lib.gapsp_rows_noalloc(_ptr(img), H, W, conn, KINDS[kind], _ptr(src), K, _ptr(out),
                                _torch_stream(stream))
    if rc != 0:
        raise GapspError(rc, "gapsp_rows_noalloc")
    return out


class Image:
    """A handle on one image (gapsp_create / gapsp_destroy).

    kind "grey", "l1": img is H x W grey levels; "mask": mask is H x W free
    flags; "sum": img is L x H x W, a multichannel image whose channels' sum
    pseudo-metric weighs the edges (gapsp_create_channels)."""

    def __init__(self, img, conn: int = 8, kind: str = "grey", mask=None, B: int = 32,
                 seed: int = 0, mem_budget: int = 0, stream=None, sweep_phases: int = 0,
                 fill_rows: int = 0, prop_blocks: int = 0, lookahead: int = 0,
                 warm_start: int = 0, max_sweep_rounds: int = 0, max_rounds: int = 0,
                 checked: int = 0):
        lib = load()
        self._lib = lib
        self._h = ctypes.c_void_p()
        if kind == "sum":
            img_a = img if hasattr(img, "data_ptr") else np.ascontiguousarray(img, dtype=np.uint8)
            if len(img_a.shape) != 3:
                raise ValueError("the sum kind takes an L x H x W image")
            L, H, W = (int(x) for x in img_a.shape)
        elif kind != "mask":
            img_a = img if hasattr(img, "data_ptr") else np.ascontiguousarray(img, dtype=np.uint8)
            H, W = int(img_a.shape[0]), int(img_a.shape[1])
        else:
            img_a = None
            if mask is None:
                raise ValueError("mask kind needs a mask")
            H, W = int(mask.shape[0]), int(mask.shape[1])
        mask_a = None
        if mask is not None:
            mask_a = mask if hasattr(mask, "data_ptr") else np.ascontiguousarray(mask, dtype=np.uint8)
        o = Opts()
        lib.gapsp_default_opts(ctypes.byref(o))
        o.conn, o.kind, o.B = conn, KINDS[kind], B
        o.seed = seed & (2 ** 64 - 1)
        o.mem_budget = mem_budget
        o.sweep_phases = sweep_phases
        o.fill_rows = fill_rows
        o.prop_blocks = prop_blocks
        o.lookahead = lookahead
        o.warm_start = warm_start
        o.max_sweep_rounds = max_sweep_rounds
        o.max_rounds = max_rounds
        o.checked = checked
        o.stream = _torch_stream(stream)
        self.H, self.W, self.N, self.conn, self.kind, self.B = H, W, H * W, conn, kind, B
        if kind == "sum":
            rc = lib.gapsp_create_channels(_ptr(img_a), L, H, W, ctypes.byref(o), ctypes.byref(self._h))
        else:
            rc = lib.gapsp_create(_ptr(img_a), H, W, _ptr(mask_a), ctypes.byref(o), ctypes.byref(self._h))
        if rc != 0:
            self._h = ctypes.c_void_p()
            raise GapspError(rc, "gapsp_create")

    def close(self):
        if self._h:
            self._lib.gapsp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def certify(self, D, sources=None) -> int:
        """gapsp_certify: the number of entries of D (CUDA, K x N; row k =
        d(sources[k], .), or rows 0.. when sources is None) that break the
        distance equations; 0 proves the rows exact."""
        K = int(D.shape[0])
        src = None
        if sources is not None:
            src = sources if hasattr(sources, "data_ptr") else np.ascontiguousarray(sources, dtype=np.int32)
        bad = ctypes.c_uint64()
        rc = self._lib.gapsp_certify(self._h, _ptr(D), _ptr(src), K, ctypes.byref(bad))
        if rc != 0:
            raise GapspError(rc, "gapsp_certify")
        return int(bad.value)

    def cancel(self):
        """Asks the all-pairs call running on this handle in another thread to
        stop (gapsp_cancel); that call then raises with status 7."""
        rc = self._lib.gapsp_cancel(self._h)
        if rc != 0:
            raise GapspError(rc, "gapsp_cancel")

    @property
    def kernel_launches(self) -> int:
        return int(self._lib.gapsp_kernel_launches(self._h))

    def profile(self, enable: bool = True):
        """Turns per-kernel event timing on or off (gapsp_profile_enable)."""
        rc = self._lib.gapsp_profile_enable(self._h, int(enable))
        if rc != 0:
            raise GapspError(rc, "gapsp_profile_enable")

    def profile_read(self) -> dict:
        """Per-kernel {name: (ms, launches)} since the last read."""
        ms = np.zeros(len(KERNELS), dtype=np.float64)
        n = np.zeros(len(KERNELS), dtype=np.uint64)
        rc = self._lib.gapsp_profile_read(self._h, _ptr(ms), _ptr(n))
        if rc != 0:
            raise GapspError(rc, "gapsp_profile_read")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNELS)}

    def profile_trace(self, cap: int = 1 << 16):
        """Per-launch (kernel name, ms) in launch order, since the last read."""
        ms = np.zeros(len(KERNELS), dtype=np.float64)
        n = np.zeros(len(KERNELS), dtype=np.uint64)
        kind = np.zeros(cap, dtype=np.int32)
        dur = np.zeros(cap, dtype=np.float32)
        cnt = np.zeros(1, dtype=np.uint64)
        rc = self._lib.gapsp_profile_trace(self._h, _ptr(ms), _ptr(n), _ptr(kind), _ptr(dur),
                                           cap, _ptr(cnt))
        if rc != 0:
            raise GapspError(rc, "gapsp_profile_trace")
        m = min(int(cnt[0]), cap)
        return [(KERNELS[int(kind[i])], float(dur[i])) for i in range(m)]

    def all_pairs(self, order: str = "minfill", out=None, want_log: bool = False):
        """Fills the N x N array (gapsp_all_pairs). Returns (D, stats dict)."""
        N = self.N
        if out is None:
            import torch
            out = torch.empty((N, N), dtype=torch.int32, device="cuda")
        st = Stats()
        rn = sl = None
        if want_log:
            rn = np.zeros(N + 1, dtype=np.uint64)
            sl = np.zeros(N + 1, dtype=np.int32)
            st.round_new = rn.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
            st.round_new_cap = len(rn)
            st.sources = sl.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            st.sources_cap = len(sl)
        rc = self._lib.gapsp_all_pairs(self._h, ORDERS[order], _ptr(out), ctypes.byref(st))
        if rc != 0:
            raise GapspError(rc, "gapsp_all_pairs")
        stats = {"propagations": st.propagations, "prepass_propagations": st.prepass_propagations,
                 "distance_ops": st.distance_ops, "new_pairs": st.new_pairs, "rounds": st.rounds,
                 "prefilled_pairs": st.prefilled_pairs, "ms_total": st.ms_total,
                 "sweeps": st.sweeps, "lines": st.lines,
                 "lookahead_propagations": st.lookahead_propagations,
                 "lookahead_hits": st.lookahead_hits}
        if want_log:
            stats["round_new"] = rn[:st.rounds].copy()
            stats["sources"] = sl[:st.propagations].copy()
        return out, stats

    def rows(self, sources, out=None):
        """out[k] = d(sources[k], .) (gapsp_rows)."""
        if hasattr(sources, "data_ptr"):
            if str(sources.dtype) != "torch.int32":
                raise ValueError("a tensor of sources must hold int32")
            src = sources
            K = int(src.numel())
        else:
            src = np.ascontiguousarray(sources, dtype=np.int32)
            K = int(src.size)
        if out is None:
            import torch
            out = torch.empty((K, self.N), dtype=torch.int32, device="cuda")
        rc = self._lib.gapsp_rows(self._h, _ptr(src), K, _ptr(out))
        if rc != 0:
            raise GapspError(rc, "gapsp_rows")
        return out


def _result_dict(r: Result) -> dict:
    return {"id": int(r.id), "done": bool(r.done), "status": int(r.status), "ptr": r.result or 0,
            "result_bytes": int(r.result_bytes), "footprint": int(r.footprint),
            "t_submit_ms": r.t_submit_ms, "t_admit_ms": r.t_admit_ms, "t_done_ms": r.t_done_ms,
            "latency_ms": r.t_done_ms - r.t_submit_ms, "propagations": int(r.propagations),
            "rounds": int(r.rounds)}


class Server:
    """A request loop with continuous batching (gapsp_server_*).

    Requests are queued by :meth:`submit_all_pairs` / :meth:`submit_rows`
    (inputs are copied) and run side by side on the GPU as slots and memory
    free up; :meth:`wait` / :meth:`poll` report them and :meth:`release`
    frees a result. ``out`` may be a caller-owned CUDA tensor (int32, N x N
    or K x N) that receives the result; otherwise the server owns it.
    """

    def __init__(self, mem_budget: int = 0, slots: int = 0, B: int = 0, lookahead: int = 0):
        lib = load()
        self._lib = lib
        o = ServerOpts()
        lib.gapsp_server_default_opts(ctypes.byref(o))
        if mem_budget:
            o.mem_budget = mem_budget
        if slots:
            o.slots = slots
        if B:
            o.B = B
        o.lookahead = lookahead
        self._s = ctypes.c_void_p()
        rc = lib.gapsp_server_create(ctypes.byref(o), ctypes.byref(self._s))
        if rc != 0:
            raise GapspError(rc, "gapsp_server_create")

    def _submit(self, kind, img, conn, img_kind, mask, order, sources, out):
        q = Request()
        q.kind = kind
        q.conn = conn
        q.img_kind = KINDS[img_kind]
        q.order = ORDERS[order]
        keep = []
        if img_kind == "mask":
            m = np.ascontiguousarray(mask, dtype=np.uint8)
            keep.append(m)
            q.mask = m.ctypes.data
            q.H, q.W = m.shape
        else:
            a = np.ascontiguousarray(img, dtype=np.uint8)
            keep.append(a)
            q.img = a.ctypes.data
            q.H, q.W = a.shape
        if sources is not None:
            src = np.ascontiguousarray(np.asarray(sources).reshape(-1)).astype(np.int32)
            keep.append(src)
            q.sources = src.ctypes.data
            q.K = int(src.size)
        if out is not None:
            q.out = _ptr(out).value
        rid = ctypes.c_uint64()
        rc = self._lib.gapsp_server_submit(self._s, ctypes.byref(q), ctypes.byref(rid))
        if rc != 0:
            raise GapspError(rc, "gapsp_server_submit")
        return int(rid.value)

    def submit_all_pairs(self, img, conn: int = 8, order: str = "minfill", kind: str = "grey",
                         mask=None, out=None) -> int:
        return self._submit(0, img, conn, kind, mask, order, None, out)

    def submit_rows(self, img, sources, conn: int = 8, kind: str = "grey", mask=None, out=None) -> int:
        return self._submit(1, img, conn, kind, mask, "minfill", sources, out)

    def wait(self, rid: int, timeout_ms: int = -1) -> dict:
        r = Result()
        rc = self._lib.gapsp_server_wait(self._s, rid, timeout_ms, ctypes.byref(r))
        if rc != 0:
            raise GapspError(rc, "gapsp_server_wait")
        return _result_dict(r)

    def poll(self, cap: int = 256) -> list:
        buf = (Result * cap)()
        n = self._lib.gapsp_server_poll(self._s, buf, cap)
        return [_result_dict(buf[i]) for i in range(n)]

    def read(self, rid: int, dst):
        """Copies a finished request's result into dst (numpy array or tensor)."""
        nbytes = dst.nbytes if isinstance(dst, np.ndarray) else dst.numel() * dst.element_size()
        rc = self._lib.gapsp_server_read(self._s, rid, _ptr(dst), nbytes)
        if rc != 0:
            raise GapspError(rc, "gapsp_server_read")
        return dst

    def release(self, rid: int):
        rc = self._lib.gapsp_server_release(self._s, rid)
        if rc != 0:
            raise GapspError(rc, "gapsp_server_release")

    def stats(self) -> dict:
        c = ServerCounts()
        rc = self._lib.gapsp_server_stats(self._s, ctypes.byref(c))
        if rc != 0:
            raise GapspError(rc, "gapsp_server_stats")
        return {k: int(getattr(c, k)) for k, _ in ServerCounts._fields_}

    def close(self):
        if self._s:
            self._lib.gapsp_server_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
