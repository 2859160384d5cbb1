"""FP64 CPU oracle of the Fast Bilateral Solver.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference arm are the only callers.  The CUDA
library never loads it and shares no code with it.

``fbs_oracle.c`` holds the arithmetic (plain loops, FP64, in the order of
the paper's equations and algorithms); this module only marshals numpy
arrays through ctypes and compiles the C file on first use.

Parity status per function (what pins each one is in ``tests/test_oracle_pins.py``):
  keys, grid, bistochastize, splat, diag, apply_A, flat_init, pcg,
  pcg_single, pyramid, hierarchical (preconditioner and initialisation),
  slice, solve, solve_robust, backward, lowrank_factors, solve_lowrank,
  domain_transform --
  all pinned (closed forms, brute force, dense linear algebra, invariants,
  finite differences).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fbs_oracle.c")
_SO = os.path.join(_HERE, "_build", "libfbs_oracle.so")
_lock = threading.Lock()
_form_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_D = ctypes.c_double


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            L.fbso_keys.argtypes = [_P, _I64, _I64, _D, _D, _D, _P]
            L.fbso_keys.restype = _I
            L.fbso_grid.argtypes = [_P, _I64, _P, _P, _P, _P]
            L.fbso_grid.restype = _I64
            L.fbso_bistochastize.argtypes = [_I64, _P, _P, _I, _P]
            L.fbso_bistochastize.restype = _I
            L.fbso_splat.argtypes = [_I64, _I64, _I, _P, _P, _P, _P, _P]
            L.fbso_splat.restype = _I
            L.fbso_diag.argtypes = [_I64, _P, _P, _P, _P, _D, _P, _P]
            L.fbso_diag.restype = None
            L.fbso_apply_A.argtypes = [_I64, _P, _P, _P, _D, _P, _P]
            L.fbso_apply_A.restype = None
            L.fbso_flat_init.argtypes = [_I64, _P, _P, _P]
            L.fbso_flat_init.restype = None
            L.fbso_pcg.argtypes = [_I64, _P, _P, _P, _P, _D, _P, _P, _I]
            L.fbso_pcg.restype = _I
            L.fbso_pcg_single.argtypes = [_I64, _P, _P, _P, _P, _D, _P, _P, _I]
            L.fbso_pcg_single.restype = _I
            L.fbso_set_pcg_form.argtypes = [_I]
            L.fbso_set_pcg_form.restype = None
            L.fbso_pyramid.argtypes = [_I64, _P, _I, _P, _P, _I64]
            L.fbso_pyramid.restype = _I
            L.fbso_set_hierarchical.argtypes = [_I, _I, _P, _P, _D, _D, _D, _D]
            L.fbso_set_hierarchical.restype = None
            L.fbso_hier_precond.argtypes = [_P, _P, _P]
            L.fbso_hier_precond.restype = _I
            L.fbso_hier_init.argtypes = [_P, _P, _P]
            L.fbso_hier_init.restype = _I
            L.fbso_domain_transform.argtypes = [_I64, _I64, _I, _P, _D, _D, _I, _P]
            L.fbso_domain_transform.restype = _I
            L.fbso_slice.argtypes = [_I64, _I64, _I, _P, _P, _P]
            L.fbso_slice.restype = None
            L.fbso_solve.argtypes = [_I64, _I64, _I, _P, _P, _P, _P, _P, _P, _D, _I, _P, _P]
            L.fbso_solve.restype = _I
            L.fbso_solve_robust.argtypes = [_I64, _I64, _P, _P, _P, _P, _P, _P, _D, _D, _I, _I,
                                            _P, _P]
            L.fbso_solve_robust.restype = _I
            L.fbso_backward.argtypes = [_I64, _I64, _I, _P, _P, _P, _P, _P, _P, _D, _I, _P, _P,
                                        _P, _P]
            L.fbso_backward.restype = _I
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class OracleError(RuntimeError):
    pass


def _check(st):
    if st:
        raise OracleError({1: "invalid argument", 2: "key field out of range",
                           3: "out of memory"}.get(int(st), f"status {st}"))


FIELD_SHIFT = {"x": 36, "y": 48, "l": 24, "u": 12, "v": 0}


def keys(yuv, sigma_xy, sigma_l, sigma_uv) -> np.ndarray:
    """Packed 5-D keys (uint64, row-major pixels) of a planar 3 x H x W YUV image."""
    yuv = _c(yuv, np.float32)
    _, h, w = yuv.shape
    out = np.empty(h * w, dtype=np.uint64)
    _check(lib().fbso_keys(_ptr(yuv), h, w, float(sigma_xy), float(sigma_l), float(sigma_uv),
                           _ptr(out)))
    return out


def grid(k: np.ndarray):
    """Distinct sorted keys, pixel -> vertex map, counts m = S 1 and +-1 neighbour table."""
    k = _c(k, np.uint64)
    n = k.size
    vkey = np.empty(max(n, 1), np.uint64)
    vid = np.empty(max(n, 1), np.uint32)
    m = np.empty(max(n, 1), np.uint32)
    nbr = np.empty((max(n, 1), 10), np.int32)
    V = lib().fbso_grid(_ptr(k), n, _ptr(vkey), _ptr(vid), _ptr(m), _ptr(nbr))
    if V < 0:
        _check(-V)
    return vkey[:V].copy(), vid[:n].copy(), m[:V].copy(), nbr[:V].copy()


def bistochastize(m, nbr, iters) -> np.ndarray:
    m = _c(m, np.uint32)
    nbr = _c(nbr, np.int32)
    n = np.empty(max(m.size, 1), np.float64)
    _check(lib().fbso_bistochastize(m.size, _ptr(m), _ptr(nbr), int(iters), _ptr(n)))
    return n[:m.size]


def splat(vid, t, c, V):
    vid = _c(vid, np.uint32)
    t = _c(t, np.float32)
    c = _c(c, np.float32)
    C = t.shape[0]
    N = vid.size
    b = np.empty((C, V), np.float64)
    sc = np.empty(V, np.float64)
    _check(lib().fbso_splat(N, V, C, _ptr(vid), _ptr(t), _ptr(c), _ptr(b), _ptr(sc)))
    return b, sc


def diag(m, nbr, n, sc, lam):
    m = _c(m, np.uint32); nbr = _c(nbr, np.int32); n = _c(n, np.float64); sc = _c(sc, np.float64)
    a = np.empty(m.size, np.float64)
    minv = np.empty(m.size, np.float64)
    lib().fbso_diag(m.size, _ptr(m), _ptr(nbr), _ptr(n), _ptr(sc), float(lam), _ptr(a), _ptr(minv))
    return a, minv


def apply_A(nbr, n, a, lam, z):
    nbr = _c(nbr, np.int32); n = _c(n, np.float64); a = _c(a, np.float64); z = _c(z, np.float64)
    out = np.empty_like(z)
    lib().fbso_apply_A(z.size, _ptr(nbr), _ptr(n), _ptr(a), float(lam), _ptr(z), _ptr(out))
    return out


def flat_init(b, sc):
    b = _c(b, np.float64); sc = _c(sc, np.float64)
    y = np.empty_like(b)
    lib().fbso_flat_init(b.size, _ptr(b), _ptr(sc), _ptr(y))
    return y


def pcg(nbr, n, a, minv, lam, b, y0, iters):
    nbr = _c(nbr, np.int32); n = _c(n, np.float64); a = _c(a, np.float64)
    minv = _c(minv, np.float64); b = _c(b, np.float64)
    y = np.array(y0, dtype=np.float64, copy=True, order="C")
    _check(lib().fbso_pcg(b.size, _ptr(nbr), _ptr(n), _ptr(a), _ptr(minv), float(lam), _ptr(b),
                          _ptr(y), int(iters)))
    return y


def pcg_single(nbr, n, a, minv, lam, b, y0, iters):
    """The single-reduction form of the same PCG (one global reduction per
    iteration); equal iterates to ``pcg`` in exact arithmetic."""
    nbr = _c(nbr, np.int32); n = _c(n, np.float64); a = _c(a, np.float64)
    minv = _c(minv, np.float64); b = _c(b, np.float64)
    y = np.array(y0, dtype=np.float64, copy=True, order="C")
    _check(lib().fbso_pcg_single(b.size, _ptr(nbr), _ptr(n), _ptr(a), _ptr(minv), float(lam),
                                 _ptr(b), _ptr(y), int(iters)))
    return y


PCG_FORMS = {"standard": 0, "single": 1}


class pcg_form:
    """``with oracle.pcg_form("single"): ...`` -- the solves inside use the
    single-reduction PCG; the standard form is restored afterwards."""

    def __init__(self, form: str):
        self.form = PCG_FORMS[form]

    def __enter__(self):
        L = lib()
        _form_lock.acquire()
        L.fbso_set_pcg_form(self.form)
        return self

    def __exit__(self, *exc):
        lib().fbso_set_pcg_form(0)
        _form_lock.release()


MAX_LEVELS = 64


def pyramid(vkey):
    """Bilateral-space pyramid of a grid's vertex keys: (sizes, parent), with
    sizes[k] the vertex count of level k (level 0 = the grid, the last level
    one vertex) and parent the concatenated parent indices of levels
    0..K-2."""
    vkey = _c(vkey, np.uint64)
    V = vkey.size
    sizes = np.zeros(MAX_LEVELS, np.int64)
    # first pass: level sizes only; second: the parents, into an exact buffer
    K = lib().fbso_pyramid(V, _ptr(vkey), MAX_LEVELS, _ptr(sizes), None, 0)
    if K < 0:
        raise OracleError(f"fbso_pyramid failed ({-K})")
    n_par = int(sizes[:K - 1].sum())
    parent = np.zeros(max(n_par, 1), np.int32)
    K2 = lib().fbso_pyramid(V, _ptr(vkey), MAX_LEVELS, _ptr(sizes), _ptr(parent), n_par)
    if K2 != K:
        raise OracleError(f"fbso_pyramid failed ({-K2})")
    return sizes[:K].copy(), parent[:n_par].copy()


class hierarchical:
    """``with oracle.hierarchical(grid): ...`` -- the solves inside use the
    hierarchical preconditioner and initialisation of Sec. 4 on the grid's
    bilateral-space pyramid; Jacobi and the flat initialisation afterwards."""

    def __init__(self, g, prec=(2.0, 5.0), init=(4.0, 0.0)):
        self.sizes, self.parent = pyramid(g.vkey)
        self.prec, self.init_ab = prec, init

    def __enter__(self):
        L = lib()
        _form_lock.acquire()
        L.fbso_set_hierarchical(1, len(self.sizes), _ptr(self.sizes), _ptr(self.parent),
                                self.prec[0], self.prec[1], self.init_ab[0], self.init_ab[1])
        return self

    def __exit__(self, *exc):
        lib().fbso_set_hierarchical(0, 0, None, None, 0.0, 0.0, 0.0, 0.0)
        _form_lock.release()

    def precond(self, a, r):
        """M_hier^-1 r for diag(A) = a (inside the context)."""
        a = _c(a, np.float64); r = _c(r, np.float64)
        s = np.empty_like(r)
        _check(lib().fbso_hier_precond(_ptr(a), _ptr(r), _ptr(s)))
        return s

    def init(self, b, sc):
        """The hierarchical initialisation of b with weights sc (inside the context)."""
        b = _c(b, np.float64); sc = _c(sc, np.float64)
        y = np.empty_like(b)
        _check(lib().fbso_hier_init(_ptr(b), _ptr(sc), _ptr(y)))
        return y


def slice_(vid, y):
    vid = _c(vid, np.uint32)
    y = _c(np.atleast_2d(y), np.float64)
    C, V = y.shape
    x = np.empty((C, vid.size), np.float64)
    lib().fbso_slice(vid.size, V, C, _ptr(vid), _ptr(y), _ptr(x))
    return x


@dataclasses.dataclass
class Grid:
    """Everything the oracle derives from one reference image."""
    height: int
    width: int
    keys: np.ndarray
    vkey: np.ndarray
    vid: np.ndarray
    m: np.ndarray
    nbr: np.ndarray
    n: Optional[np.ndarray] = None

    @property
    def V(self) -> int:
        return int(self.vkey.size)

    @property
    def N(self) -> int:
        return int(self.vid.size)


def build_grid(yuv, sigma_xy, sigma_l, sigma_uv, bistoch_iters: Optional[int] = 2) -> Grid:
    k = keys(yuv, sigma_xy, sigma_l, sigma_uv)
    vkey, vid, m, nbr = grid(k)
    g = Grid(int(yuv.shape[1]), int(yuv.shape[2]), k, vkey, vid, m, nbr)
    if bistoch_iters is not None:
        g.n = bistochastize(m, nbr, bistoch_iters)
    return g


def solve(g: Grid, t, c, lam, pcg_iters):
    """Forward solve; returns (y C x V, x C x N) in FP64."""
    t = _c(t, np.float32).reshape(-1, g.N)
    c = _c(c, np.float32).reshape(g.N)
    C = t.shape[0]
    y = np.empty((C, g.V), np.float64)
    x = np.empty((C, g.N), np.float64)
    _check(lib().fbso_solve(g.N, g.V, C, _ptr(g.vid), _ptr(g.m), _ptr(g.nbr), _ptr(g.n), _ptr(t),
                            _ptr(c), float(lam), int(pcg_iters), _ptr(y), _ptr(x)))
    return y, x


def solve_robust(g: Grid, t, c_init, lam, sigma_gm, irls_iters, pcg_iters):
    """Geman-McClure robust solve (one channel); returns (y 1 x V, x 1 x N)."""
    t = _c(t, np.float32).reshape(g.N)
    c = _c(c_init, np.float32).reshape(g.N)
    y = np.empty((1, g.V), np.float64)
    x = np.empty((1, g.N), np.float64)
    _check(lib().fbso_solve_robust(g.N, g.V, _ptr(g.vid), _ptr(g.m), _ptr(g.nbr), _ptr(g.n),
                                   _ptr(t), _ptr(c), float(lam), float(sigma_gm), int(irls_iters),
                                   int(pcg_iters), _ptr(y), _ptr(x)))
    return y, x


def backward(g: Grid, t, c, lam, pcg_iters, yhat, dx):
    """Gradients (dL/dt C x N, dL/dc N) of the solve given dL/dx (C x N) and yhat (C x V)."""
    t = _c(t, np.float32).reshape(-1, g.N)
    c = _c(c, np.float32).reshape(g.N)
    C = t.shape[0]
    yhat = _c(yhat, np.float64).reshape(C, g.V)
    dx = _c(dx, np.float64).reshape(C, g.N)
    dt = np.empty((C, g.N), np.float64)
    dc = np.empty(g.N, np.float64)
    _check(lib().fbso_backward(g.N, g.V, C, _ptr(g.vid), _ptr(g.m), _ptr(g.nbr), _ptr(g.n),
                               _ptr(t), _ptr(c), float(lam), int(pcg_iters), _ptr(yhat), _ptr(dx),
                               _ptr(dt), _ptr(dc)))
    return dt, dc


def lowrank_factors(B, eps):
    """The reduction of a wide right-hand side (supplement, multiple output
    channels): B (V x C) = Q R P^T by a column-pivoted QR (LAPACK's
    Businger-Golub pivoting, the library step); R' = R P^T; row masses
    m_i = |R'_i|^2; rows ranked by mass (stable); the fewest leading rows
    whose mass reaches (1 - eps) of the total are kept.  Returns
    (Q~ V x t, R~ t x C, t); t = 0 when B = 0.  (The printed cut-off reads
    "largest t with sum_{i<t} m_i <= (1 - eps) sum m_i", which can keep
    nothing; the reading here keeps enough rows that the dropped mass is at
    most eps of the total, the stated intent.)"""
    import scipy.linalg
    B = np.asarray(B, np.float64)
    V, C = B.shape
    Q, R, piv = scipy.linalg.qr(B, mode="economic", pivoting=True)
    Rp = np.empty_like(R)
    Rp[:, piv] = R                       # R P^T: columns back in input order
    mass = (Rp ** 2).sum(axis=1)
    total = float(mass.sum())
    if total <= 0.0:
        return Q[:, :0], Rp[:0], 0
    order = np.argsort(-mass, kind="stable")
    csum = np.cumsum(mass[order])
    t = min(int(np.searchsorted(csum, (1.0 - eps) * total, side="left")) + 1, len(order))
    keep = order[:t]
    return Q[:, keep], Rp[keep, :], t


def solve_lowrank(g: Grid, t, c, lam, pcg_iters, eps):
    """Forward solve of a wide target through the low-rank reduction:
    B = S(c o t) (Eq. 7's b, one column per channel), B ~ Q~ R~
    (``lowrank_factors``), Y~ = A^-1 Q~ by Jacobi-PCG from the flat
    initialisation per column (the same solve as every channel of
    ``solve``), Y = Y~ R~, x = S^T Y.  Returns (y C x V, x C x N, t)."""
    t = _c(t, np.float32).reshape(-1, g.N)
    c = _c(c, np.float32).reshape(g.N)
    C = t.shape[0]
    b, sc = splat(g.vid, t, c, g.V)
    Qt, Rt, r = lowrank_factors(b.T, eps)
    a, minv = diag(g.m, g.nbr, g.n, sc, lam)
    y = np.zeros((C, g.V), np.float64)
    for q in range(r):
        bq = np.ascontiguousarray(Qt[:, q])
        yq = pcg(g.nbr, g.n, a, minv, lam, bq, flat_init(bq, sc), pcg_iters)
        y += np.outer(Rt[q], yq)
    return y, slice_(g.vid, y), r


def domain_transform(guide, x, sigma_s, sigma_r, iters=3):
    """The domain transform post-filter (recursive formulation of Gastal
    and Oliveira 2011, as the paper's Sec. 5 applies it to the solver's
    output): guide 3 x H x W, x C x H x W; returns the filtered x (FP64)."""
    guide = _c(guide, np.float32)
    H, W = guide.shape[1], guide.shape[2]
    x = np.array(x, dtype=np.float64, copy=True, order="C").reshape(-1, H, W)
    _check(lib().fbso_domain_transform(H, W, x.shape[0], _ptr(guide), float(sigma_s),
                                       float(sigma_r), int(iters), _ptr(x)))
    return x


def run_instance(inst, bistoch_iters=2, pcg_iters=25):
    """Grid + bistochastisation + forward solve of one synthetic instance."""
    g = build_grid(inst.yuv, inst.sigma_xy, inst.sigma_l, inst.sigma_uv, bistoch_iters)
    y, x = solve(g, inst.t, inst.c, inst.lam, pcg_iters)
    return g, y, x
