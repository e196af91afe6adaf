"""CPU oracle for all pairs of geodesic distances (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. The CUDA library never calls it, and the two
share no code: the C source next to this file is compiled on its own by
:func:`build` with the host C compiler.

Each wrapper names the passage of Noyel, Angulo & Jeulin, "Fast computation
of all pairs of geodesic distances", that the C function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gapsp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

UNREACH = 0xFFFFFFFF
UNSET = 0xFFFFFFFE
ORDERS = {"naive": 0, "spiral": 1, "minfill": 2, "extrema": 3, "repulsion": 4}


def build(force: bool = False) -> str:
    """Compile the oracle into ``liboracle.so`` beside its source."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                               "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i = ctypes.c_int
        lib.or_sssp.argtypes = [P, P, i, i, i, i, i, P]
        lib.or_msssp.argtypes = [P, P, i, i, i, i, P, i, P]
        lib.or_rows.argtypes = [P, P, i, i, i, i, P, i, P, i]
        lib.or_floyd.argtypes = [P, P, i, i, i, i, P]
        lib.or_parents.argtypes = [P, P, i, i, i, i, P, i, P]
        lib.or_spiral_sequence.argtypes = [P, i, i, i, ctypes.c_uint64, P]
        lib.or_spiral_sequence.restype = i
        lib.or_extrema.argtypes = [P, P, i, i, i, i, P, P, P, P]
        lib.or_extrema.restype = i
        lib.or_fill.argtypes = [P, P, i, i, i, i, i, i, ctypes.c_uint64, P, P, P, P]
        lib.or_fill.restype = i
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


KINDS = {"grey": 0, "mask": 1, "l1": 2, "sum": 3}


def _prep(img, mask, kind):
    """Image, mask, sizes and the oracle's kind code. For kind "sum" the
    image is L x H x W (a multichannel image, Sec. 2: values in T^L) and the
    code carries L: 3 | (L << 8)."""
    k = KINDS[kind] if isinstance(kind, str) else int(kind)
    img = np.ascontiguousarray(img, dtype=np.uint8)
    if k == 3:
        if img.ndim != 3:
            raise ValueError("the sum kind takes an L x H x W image")
        L, H, W = img.shape
        return img, None, H, W, 3 | (L << 8)
    H, W = img.shape
    m = None
    if k == 1:
        if mask is None:
            raise ValueError("mask kind needs a mask")
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        if m.shape != img.shape:
            raise ValueError("mask shape differs from image shape")
    return img, m, H, W, k


def sssp(img, s, conn=8, kind="grey", mask=None) -> np.ndarray:
    """Geodesic distance row d(s, .) (Sec. 2, eqs. "temps"/"distance")."""
    img, m, H, W, k = _prep(img, mask, kind)
    out = np.empty(H * W, dtype=np.uint32)
    _load().or_sssp(_ptr(img), _ptr(m), H, W, conn, k, int(s), _ptr(out))
    return out


def msssp(img, sources, conn=8, kind="grey", mask=None) -> np.ndarray:
    """Distance to the nearest of several sources (all start at 0)."""
    img, m, H, W, k = _prep(img, mask, kind)
    src = np.ascontiguousarray(sources, dtype=np.int32)
    out = np.empty(H * W, dtype=np.uint32)
    _load().or_msssp(_ptr(img), _ptr(m), H, W, conn, k, _ptr(src), len(src), _ptr(out))
    return out


def rows(img, sources=None, conn=8, kind="grey", mask=None, threads=None) -> np.ndarray:
    """Rows d(s, .) for the given sources, or the full N x N array.

    One propagation per source: the naive method (Sec. 1).
    """
    img, m, H, W, k = _prep(img, mask, kind)
    N = H * W
    threads = threads or os.cpu_count() or 1
    if sources is None:
        out = np.empty((N, N), dtype=np.uint32)
        _load().or_rows(_ptr(img), _ptr(m), H, W, conn, k, None, 0, _ptr(out), threads)
    else:
        src = np.ascontiguousarray(sources, dtype=np.int32)
        out = np.empty((len(src), N), dtype=np.uint32)
        _load().or_rows(_ptr(img), _ptr(m), H, W, conn, k, _ptr(src), len(src),
                        _ptr(out), threads)
    return out


def apsp(img, conn=8, kind="grey", mask=None, threads=None) -> np.ndarray:
    """Full N x N geodesic distance array by Dijkstra from every pixel."""
    return rows(img, None, conn, kind, mask, threads)


def floyd(img, conn=8, kind="grey", mask=None) -> np.ndarray:
    """Full array by Floyd-Warshall (tiny images only)."""
    img, m, H, W, k = _prep(img, mask, kind)
    N = H * W
    if N > 400:
        raise ValueError("Floyd-Warshall oracle is for tiny images")
    out = np.empty((N, N), dtype=np.uint32)
    _load().or_floyd(_ptr(img), _ptr(m), H, W, conn, k, _ptr(out))
    return out


def parents(img, drow, s, conn=8, kind="grey", mask=None) -> np.ndarray:
    """Canonical geodesic tree of source s (Sec. 2, "geodesic tree")."""
    img, m, H, W, k = _prep(img, mask, kind)
    d = np.ascontiguousarray(drow, dtype=np.uint32)
    out = np.empty(H * W, dtype=np.int32)
    _load().or_parents(_ptr(img), _ptr(m), H, W, conn, k, _ptr(d), int(s), _ptr(out))
    return out


def spiral_sequence(H, W, seed, kind="grey", mask=None) -> np.ndarray:
    """Frame-by-frame shuffled pixel sequence (Sec. 3.1, spiral method)."""
    k = KINDS[kind] if isinstance(kind, str) else int(kind)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    out = np.empty(H * W, dtype=np.int32)
    n = _load().or_spiral_sequence(_ptr(m), k, H, W, ctypes.c_uint64(seed & (2**64 - 1)),
                                   _ptr(out))
    return out[:n].copy()


@dataclass
class Extrema:
    e: np.ndarray          # distance from the boundary vertices
    g: np.ndarray          # distance from the centroid(s)
    centroids: np.ndarray  # one per component
    rank: np.ndarray       # position in the decreasing extrema list Ext


def extrema(img, conn=8, kind="grey", mask=None) -> Extrema:
    """Geodesic centroid and extrema list (Sec. 3.3)."""
    img, m, H, W, k = _prep(img, mask, kind)
    N = H * W
    e = np.empty(N, dtype=np.uint32)
    g = np.empty(N, dtype=np.uint32)
    cen = np.empty(N, dtype=np.int32)
    rank = np.empty(N, dtype=np.int32)
    nc = _load().or_extrema(_ptr(img), _ptr(m), H, W, conn, k, _ptr(e), _ptr(g),
                            _ptr(cen), _ptr(rank))
    return Extrema(e, g, cen[:nc].copy(), rank)


@dataclass
class FillResult:
    propagations: int
    prepass_propagations: int
    distance_ops: int
    new_pairs: int
    rounds: int
    prefilled_pairs: int
    components: int
    sources: np.ndarray
    round_new: np.ndarray
    D: np.ndarray | None

    def counts(self) -> dict:
        return {"propagations": self.propagations,
                "prepass_propagations": self.prepass_propagations,
                "distance_ops": self.distance_ops,
                "new_pairs": self.new_pairs,
                "rounds": self.rounds}


def fill(img, order="minfill", B=1, seed=0, conn=8, kind="grey", mask=None,
         want_D=False) -> FillResult:
    """Simulate the method: fill D from geodesic trees in a source order.

    Sec. 3: naive (raster), spiral (Algorithm "spiral method"), geodesic
    extrema (Algorithm "geodesic extrema method") and minimum filling rate
    (Algorithm "method based on the filling rate"); B sources are chosen per
    round from the state at the round's start.
    """
    img, m, H, W, k = _prep(img, mask, kind)
    N = H * W
    stats = np.zeros(8, dtype=np.uint64)
    seq = np.full(N, -1, dtype=np.int32)
    rnew = np.zeros(N, dtype=np.uint64)
    D = np.empty((N, N), dtype=np.uint32) if want_D else None
    rc = _load().or_fill(_ptr(img), _ptr(m), H, W, conn, k, ORDERS[order], int(B),
                         ctypes.c_uint64(seed & (2**64 - 1)), _ptr(stats), _ptr(seq),
                         _ptr(rnew), _ptr(D))
    if rc != 0:
        raise RuntimeError("oracle fill did not terminate")
    P = int(stats[0])
    R = int(stats[4])
    return FillResult(P, int(stats[1]), int(stats[2]), int(stats[3]), R, int(stats[5]),
                      int(stats[6]), seq[:P].copy(), rnew[:R].copy(), D)
