"""Python binding of libfbs (include/fbs.h): argument marshalling only.

Every step of the solver runs in the CUDA kernels of libfbs.so; this module
passes device pointers (torch CUDA tensors), sizes and the current CUDA
stream through ctypes.  There is no CPU fallback: if the library is not
built or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import List, Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfbs.so")

FBS_OK = 0
STATUS_NAMES = {0: "FBS_OK", 1: "FBS_ERR_ARG", 2: "FBS_ERR_RANGE", 3: "FBS_ERR_OOM",
                4: "FBS_ERR_CUDA", 5: "FBS_ERR_TIMEOUT", 6: "FBS_ERR_NONFINITE",
                7: "FBS_ERR_STATE"}

# every symbol include/fbs.h declares
EXPORTED = ["fbs_grid_build", "fbs_bistochastize", "fbs_solve", "fbs_solve_robust",
            "fbs_solve_backward", "fbs_grid_info", "fbs_grid_export", "fbs_grid_sync",
            "fbs_grid_destroy", "fbs_status_string", "fbs_profile_enable", "fbs_profile_read",
            "fbs_set_option", "fbs_solve_static", "fbs_autotune", "fbs_solve_lowrank",
            "fbs_domain_transform", "fbs_pyramid_export"]

OPT_VECTOR_PRECISION, OPT_PCG_LAUNCH, OPT_INJECT_BARRIER_TIMEOUT, OPT_PCG_FORM = 1, 2, 3, 4
OPT_PHASE_BLOCKS, OPT_PRECONDITIONER, OPT_TUNE_SINGLE_SOLVE = 5, 6, 7
PRECOND_JACOBI, PRECOND_HIERARCHICAL = 0, 1
VECTORS_AUTO, VECTORS_FP32, VECTORS_COMPENSATED = 0, 1, 2
PCG_AUTO, PCG_PERSISTENT, PCG_PER_PHASE = 0, 1, 2
PCG_FORM_STANDARD, PCG_FORM_SINGLE = 0, 1


class FbsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        name = STATUS_NAMES.get(self.status, str(status))
        msg = _lib.fbs_status_string(self.status).decode() if _lib is not None else name
        super().__init__(f"{where}: {name} ({msg})")


class ImageDesc(ctypes.Structure):
    _fields_ = [("yuv", ctypes.c_void_p), ("height", ctypes.c_int), ("width", ctypes.c_int),
                ("sigma_xy", ctypes.c_float), ("sigma_l", ctypes.c_float),
                ("sigma_uv", ctypes.c_float)]


class ProblemDesc(ctypes.Structure):
    _fields_ = [("t", ctypes.c_void_p), ("c", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("y", ctypes.c_void_p), ("channels", ctypes.c_int), ("lambda_", ctypes.c_float)]


_lib = None
_lock = threading.Lock()


def load(path: Optional[str] = None):
    """Load libfbs.so (built by ``paper_1511_03296_gb300.build``); raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libfbs.so is not built ({p}); run "
                               "`python -m paper_1511_03296_gb300.build` first")
        L = ctypes.CDLL(p)
        P, I, F, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_int64
        L.fbs_grid_build.argtypes = [ctypes.POINTER(ImageDesc), I, P, ctypes.POINTER(P)]
        L.fbs_bistochastize.argtypes = [P, I, P]
        L.fbs_solve.argtypes = [P, ctypes.POINTER(ProblemDesc), I, P]
        L.fbs_solve_robust.argtypes = [P, ctypes.POINTER(ProblemDesc), F, I, I, P]
        L.fbs_solve_lowrank.argtypes = [P, ctypes.POINTER(ProblemDesc), I, ctypes.c_double,
                                        ctypes.POINTER(I), P]
        L.fbs_domain_transform.argtypes = [P, I, I, P, I, F, F, I, P]
        L.fbs_pyramid_export.argtypes = [P, I, I, P, ctypes.POINTER(I), ctypes.POINTER(I64), P, P,
                                         P]
        L.fbs_solve_backward.argtypes = [P, ctypes.POINTER(ProblemDesc), ctypes.POINTER(P),
                                         ctypes.POINTER(P), ctypes.POINTER(P), I, P]
        L.fbs_grid_info.argtypes = [P, I, ctypes.POINTER(I64), ctypes.POINTER(I64)]
        L.fbs_grid_export.argtypes = [P, I, P, P, P, P, P, P]
        L.fbs_grid_sync.argtypes = [P, P]
        L.fbs_set_option.argtypes = [P, I, I]
        L.fbs_solve_static.argtypes = [P, ctypes.POINTER(ProblemDesc), I, P]
        L.fbs_grid_destroy.argtypes = [P, P]
        L.fbs_status_string.argtypes = [I]
        L.fbs_status_string.restype = ctypes.c_char_p
        L.fbs_profile_enable.argtypes = [I]
        L.fbs_profile_read.argtypes = [ctypes.POINTER(I), ctypes.POINTER(ctypes.c_char_p),
                                       ctypes.POINTER(I64), ctypes.POINTER(ctypes.c_double)]
        for name in EXPORTED:
            if name != "fbs_status_string":
                getattr(L, name).restype = I
        _lib = L
        return L


def _check(st, where):
    if st != FBS_OK:
        raise FbsError(st, where)


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, name, dtype=None):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


class Grid:
    """A bilateral grid handle (one or more reference images)."""

    def __init__(self, handle, n_images, shapes):
        self._h = handle
        self.n_images = n_images
        self.shapes = shapes           # [(H, W)]
        self.vertex_counts = []
        self.vertex_offsets = []
        for k in range(n_images):
            nv, off = ctypes.c_int64(), ctypes.c_int64()
            _check(load().fbs_grid_info(self._h, k, ctypes.byref(nv), ctypes.byref(off)),
                   "fbs_grid_info")
            self.vertex_counts.append(nv.value)
            self.vertex_offsets.append(off.value)

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("grid destroyed")
        return self._h

    def destroy(self, stream=None):
        if self._h is not None:
            _check(load().fbs_grid_destroy(self._h, _stream_ptr(stream)), "fbs_grid_destroy")
            self._h = None

    def __del__(self):
        try:
            if self._h is not None and _lib is not None:
                _lib.fbs_grid_destroy(self._h, None)
        except Exception:
            pass


def grid_build(yuv: Sequence, sigma_xy, sigma_l, sigma_uv, stream=None) -> Grid:
    """Build the grid of a list of planar 3 x H x W float32 CUDA images."""
    import torch
    n = len(yuv)
    descs = (ImageDesc * n)()
    sig = [sigma_xy, sigma_l, sigma_uv]
    sig = [s if isinstance(s, (list, tuple)) else [s] * n for s in sig]
    shapes = []
    for k, im in enumerate(yuv):
        if im.dim() != 3 or im.shape[0] != 3:
            raise ValueError("yuv images must be 3 x H x W")
        descs[k] = ImageDesc(_dev_ptr(im, f"yuv[{k}]", torch.float32), int(im.shape[1]),
                             int(im.shape[2]), float(sig[0][k]), float(sig[1][k]),
                             float(sig[2][k]))
        shapes.append((int(im.shape[1]), int(im.shape[2])))
    h = ctypes.c_void_p()
    _check(load().fbs_grid_build(descs, n, _stream_ptr(stream), ctypes.byref(h)),
           "fbs_grid_build")
    return Grid(h, n, shapes)


def bistochastize(grid: Grid, iters: int = 2, stream=None) -> None:
    _check(load().fbs_bistochastize(grid.handle, int(iters), _stream_ptr(stream)),
           "fbs_bistochastize")


def _problems(grid, t, c, lam, x, y):
    import torch
    n = grid.n_images
    if len(t) != n or len(c) != n:
        raise ValueError("one target and one confidence per image")
    lam = lam if isinstance(lam, (list, tuple)) else [lam] * n
    x = x if x is not None else [None] * n
    y = y if y is not None else [None] * n
    probs = (ProblemDesc * n)()
    for k in range(n):
        H, W = grid.shapes[k]
        if t[k].dim() != 3 or tuple(t[k].shape[1:]) != (H, W):
            raise ValueError(f"t[{k}] must be C x {H} x {W}")
        C = int(t[k].shape[0])
        if tuple(c[k].shape) != (H, W):
            raise ValueError(f"c[{k}] must be {H} x {W}")
        if x[k] is not None and tuple(x[k].shape) != (C, H, W):
            raise ValueError(f"x[{k}] must be {C} x {H} x {W}")
        if y[k] is not None and tuple(y[k].shape) != (C, grid.vertex_counts[k]):
            raise ValueError(f"y[{k}] must be {C} x {grid.vertex_counts[k]}")
        probs[k] = ProblemDesc(_dev_ptr(t[k], f"t[{k}]", torch.float32),
                               _dev_ptr(c[k], f"c[{k}]", torch.float32),
                               _dev_ptr(x[k], f"x[{k}]", torch.float32),
                               _dev_ptr(y[k], f"y[{k}]", torch.float32), C, float(lam[k]))
    return probs


class _TuneResult(ctypes.Structure):
    _fields_ = [("pcg_launch", ctypes.c_int), ("pcg_form", ctypes.c_int),
                ("phase_blocks", ctypes.c_int), ("solve_ms", ctypes.c_float),
                ("candidates", ctypes.c_int)]


def tuning_key(grid: Grid, t: List, device_name: Optional[str] = None) -> str:
    """The autotuner cache's key of a problem: the GPU's name and the
    problem's shape class -- the image count and the total vertex count
    (each in powers of two) and the widest padded channel row."""
    import math
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name(t[0].device)
    n = grid.n_images
    v = max(1, sum(grid.vertex_counts))
    cmax = max(int(tt.shape[0]) for tt in t)
    row = cmax if cmax <= 2 else (cmax + 3) // 4 * 4
    return (f"{device_name}|images~2^{math.ceil(math.log2(n)) if n > 1 else 0}"
            f"|vertices~2^{round(math.log2(v))}|row={row}")


def _cache_read(path: str) -> dict:
    import json
    try:
        with open(path) as f:
            d = json.load(f)
        return d.get("entries", {}) if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def _cache_write(path: str, key: str, tuning: dict) -> None:
    import json
    entries = _cache_read(path)
    entries[key] = {k: tuning[k] for k in ("pcg_launch", "pcg_form", "phase_blocks", "solve_ms")}
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump({"format": "fbs autotune cache 1", "entries": entries}, f, indent=1,
                  sort_keys=True)
    os.replace(tmp, path)


def autotune(grid: Grid, t: List, c: List, lam, pcg_iters: int = 25, x: Optional[List] = None,
             y: Optional[List] = None, stream=None, cache: Optional[str] = None,
             single_solve: bool = False) -> dict:
    """fbs_autotune: times the PCG launch configurations on this problem, leaves
    the fastest set on the grid and returns it (the outputs hold its result).
    The same settings can be applied to another grid of the same shape with
    ``apply_tuning``.

    cache: a JSON file of earlier choices keyed by ``tuning_key`` (GPU name
    and shape class).  On a hit the stored choice is set on the grid and one
    solve fills the outputs, with no timing ("cached": True in the result);
    on a miss the problem is tuned and the choice stored.

    single_solve: time each configuration as the first solve on a grid
    (OPT_TUNE_SINGLE_SOLVE), for callers that build a new grid per solve;
    otherwise repeated solves on the grid (graph replay) are timed."""
    key = None
    if cache is not None:
        key = tuning_key(grid, t) + ("|single-solve" if single_solve else "|repeated")
    if cache is not None:
        hit = _cache_read(cache).get(key)
        if hit is not None:
            apply_tuning(grid, hit)
            solve(grid, t, c, lam, pcg_iters, x=x, y=y, stream=stream)
            return dict(hit, candidates=0, cached=True, key=key)
    probs = _problems(grid, t, c, lam, x, y)
    r = _TuneResult()
    set_option(grid, OPT_TUNE_SINGLE_SOLVE, 1 if single_solve else 0)
    _check(load().fbs_autotune(grid.handle, probs, int(pcg_iters), _stream_ptr(stream),
                               ctypes.byref(r)), "fbs_autotune")
    out = {"pcg_launch": r.pcg_launch, "pcg_form": r.pcg_form, "phase_blocks": r.phase_blocks,
           "solve_ms": r.solve_ms, "candidates": r.candidates}
    if cache is not None:
        _cache_write(cache, key, out)
        out.update(cached=False, key=key)
    return out


def apply_tuning(grid: Grid, tuning: dict) -> None:
    """Sets an autotune result's options on a grid."""
    set_option(grid, OPT_PCG_LAUNCH, tuning["pcg_launch"])
    set_option(grid, OPT_PCG_FORM, tuning["pcg_form"])
    set_option(grid, OPT_PHASE_BLOCKS, tuning["phase_blocks"])


def solve(grid: Grid, t: List, c: List, lam, pcg_iters: int = 25, x: Optional[List] = None,
          y: Optional[List] = None, stream=None) -> None:
    """Forward solve; writes x (C x H x W) and/or y (C x V) per image."""
    probs = _problems(grid, t, c, lam, x, y)
    _check(load().fbs_solve(grid.handle, probs, int(pcg_iters), _stream_ptr(stream)), "fbs_solve")


def solve_static(grid: Grid, t: List, c: List, lam, pcg_iters: int = 25,
                 x: Optional[List] = None, y: Optional[List] = None, stream=None) -> None:
    """fbs_solve without any device allocation: the solver's scratch lives in
    a fixed 64 MiB array inside the library (for callers that cannot
    allocate; calls must not overlap on the GPU -- see include/fbs.h)."""
    probs = _problems(grid, t, c, lam, x, y)
    _check(load().fbs_solve_static(grid.handle, probs, int(pcg_iters), _stream_ptr(stream)),
           "fbs_solve_static")


def solve_lowrank(grid: Grid, t: List, c: List, lam, pcg_iters: int = 25, eps: float = 0.01,
                  x: Optional[List] = None, stream=None) -> List[int]:
    """fbs_solve_lowrank: a wide target solved through the low-rank
    reduction of B = S(c o t) (column-pivoted QR, rows kept by mass down to
    a residual fraction eps); writes x (C x H x W) per image and returns the
    rank each image was solved at.  Synchronises the stream."""
    probs = _problems(grid, t, c, lam, x, None)
    ranks = (ctypes.c_int * grid.n_images)()
    _check(load().fbs_solve_lowrank(grid.handle, probs, int(pcg_iters), float(eps), ranks,
                                    _stream_ptr(stream)), "fbs_solve_lowrank")
    return list(ranks)


def pyramid_export(grid: Grid, image: int = 0, stream=None) -> list:
    """The bilateral-space pyramid of one image, level by level: a list of
    dicts {keys, parent, count} (numpy arrays), level 0 first; built on the
    GPU first if no hierarchical solve has built it."""
    import numpy as np
    L = load()
    levels, n = ctypes.c_int(0), ctypes.c_int64(0)
    _check(L.fbs_pyramid_export(grid.handle, int(image), 0, _stream_ptr(stream),
                                ctypes.byref(levels), ctypes.byref(n), None, None, None),
           "fbs_pyramid_export")
    out = []
    for k in range(levels.value):
        _check(L.fbs_pyramid_export(grid.handle, int(image), k, _stream_ptr(stream), None,
                                    ctypes.byref(n), None, None, None), "fbs_pyramid_export")
        keys = np.empty(n.value, np.uint64)
        parent = np.empty(n.value, np.int32)
        count = np.empty(n.value, np.float32)
        _check(L.fbs_pyramid_export(grid.handle, int(image), k, _stream_ptr(stream), None,
                                    ctypes.byref(n), keys.ctypes.data, parent.ctypes.data,
                                    count.ctypes.data), "fbs_pyramid_export")
        out.append({"keys": keys, "parent": parent, "count": count})
    return out


def domain_transform(guide, x, sigma_s: float, sigma_r: float, iterations: int = 3,
                     stream=None) -> None:
    """fbs_domain_transform: edge-aware recursive filtering of x (C x H x W,
    in place) guided by a 3 x H x W image -- the post-filter the paper runs
    on the solver's output."""
    import torch
    if guide.dim() != 3 or guide.shape[0] != 3:
        raise ValueError("guide must be 3 x H x W")
    H, W = int(guide.shape[1]), int(guide.shape[2])
    if x.dim() == 2:
        x = x.unsqueeze(0)
    if x.dim() != 3 or tuple(x.shape[1:]) != (H, W):
        raise ValueError("x must be C x H x W with the guide's H and W")
    _check(load().fbs_domain_transform(_dev_ptr(guide, "guide", torch.float32), H, W,
                                       _dev_ptr(x, "x", torch.float32), int(x.shape[0]),
                                       float(sigma_s), float(sigma_r), int(iterations),
                                       _stream_ptr(stream)), "fbs_domain_transform")


def solve_robust(grid: Grid, t: List, c: List, lam, sigma_gm: float, irls_iters: int = 10,
                 pcg_iters: int = 25, x: Optional[List] = None, y: Optional[List] = None,
                 stream=None) -> None:
    probs = _problems(grid, t, c, lam, x, y)
    _check(load().fbs_solve_robust(grid.handle, probs, float(sigma_gm), int(irls_iters),
                                   int(pcg_iters), _stream_ptr(stream)), "fbs_solve_robust")


def solve_backward(grid: Grid, t: List, c: List, lam, yhat: List, dL_dx: List, dL_dt: List,
                   dL_dc: List, pcg_iters: int = 25, stream=None) -> None:
    import torch
    probs = _problems(grid, t, c, lam, None, yhat)
    n = grid.n_images
    P = ctypes.c_void_p
    dx = (P * n)(*[_dev_ptr(g, "dL_dx", torch.float32) for g in dL_dx])
    dt = (P * n)(*[_dev_ptr(g, "dL_dt", torch.float32) for g in dL_dt])
    dc = (P * n)(*[_dev_ptr(g, "dL_dc", torch.float32) for g in dL_dc])
    _check(load().fbs_solve_backward(grid.handle, probs, dx, dt, dc, int(pcg_iters),
                                     _stream_ptr(stream)), "fbs_solve_backward")


def set_option(grid: Grid, option: int, value: int) -> None:
    """OPT_VECTOR_PRECISION: VECTORS_AUTO / VECTORS_FP32 / VECTORS_COMPENSATED;
    OPT_PCG_LAUNCH: PCG_AUTO / PCG_PERSISTENT / PCG_PER_PHASE; OPT_PCG_FORM:
    PCG_FORM_STANDARD / PCG_FORM_SINGLE; OPT_PHASE_BLOCKS: 1, 2, 4;
    OPT_PRECONDITIONER: PRECOND_JACOBI / PRECOND_HIERARCHICAL (see
    include/fbs.h)."""
    _check(load().fbs_set_option(grid.handle, int(option), int(value)), "fbs_set_option")


def set_vector_precision(grid: Grid, precision: int) -> None:
    set_option(grid, OPT_VECTOR_PRECISION, precision)


def grid_info(grid: Grid, image: int):
    nv, off = ctypes.c_int64(), ctypes.c_int64()
    _check(load().fbs_grid_info(grid.handle, int(image), ctypes.byref(nv), ctypes.byref(off)),
           "fbs_grid_info")
    return nv.value, off.value


def grid_export(grid: Grid, image: int, with_n: bool = True, stream=None):
    """Host copies (numpy) of one image's keys, vid, counts, nbr and n."""
    import numpy as np
    V, _ = grid_info(grid, image)
    H, W = grid.shapes[image]
    keys = np.empty(V, np.uint64)
    vid = np.empty(H * W, np.uint32)
    m = np.empty(V, np.uint32)
    nbr = np.empty((V, 10), np.int32)
    n = np.empty(V, np.float64) if with_n else None
    _check(load().fbs_grid_export(grid.handle, int(image), _stream_ptr(stream),
                                  keys.ctypes.data, vid.ctypes.data, m.ctypes.data,
                                  nbr.ctypes.data, n.ctypes.data if with_n else None),
           "fbs_grid_export")
    return keys, vid, m, nbr, n


def grid_sync(grid: Grid, stream=None) -> None:
    _check(load().fbs_grid_sync(grid.handle, _stream_ptr(stream)), "fbs_grid_sync")


def grid_destroy(grid: Grid, stream=None) -> None:
    grid.destroy(stream)


def profile_enable(level: int = 1) -> None:
    """0 = off, 1 = every kernel family, 2 = multi-launch regions."""
    _check(load().fbs_profile_enable(int(level)), "fbs_profile_enable")


def profile_read():
    """{family: (launches, total_ms)} of the kernels launched since profile_enable."""
    L = load()
    cnt = ctypes.c_int(64)
    names = (ctypes.c_char_p * 64)()
    launches = (ctypes.c_int64 * 64)()
    ms = (ctypes.c_double * 64)()
    _check(L.fbs_profile_read(ctypes.byref(cnt), names, launches, ms), "fbs_profile_read")
    return {names[i].decode(): (launches[i], ms[i]) for i in range(min(cnt.value, 64))}


# ------------------------------------------------------------- autograd ---

def _forward_batch(grid, ts, cs, lam, pcg_iters):
    """One fbs_solve over every image of the grid; returns (xs, ys)."""
    import torch
    ts = [t.contiguous() for t in ts]
    cs = [c.contiguous() for c in cs]
    xs = [torch.empty_like(t) for t in ts]
    ys = [torch.empty((int(t.shape[0]), grid.vertex_counts[k]), device=t.device,
                      dtype=torch.float32) for k, t in enumerate(ts)]
    solve(grid, ts, cs, lam, pcg_iters, x=xs, y=ys)
    return ts, cs, xs, ys


def _backward_batch(grid, ts, cs, ys, gxs, lam, pcg_iters):
    """One fbs_solve_backward over every image of the grid; an output that
    took no part in the loss (gradient None) contributes zeros."""
    import torch
    gxs = [torch.zeros_like(t) if g is None else g.contiguous() for g, t in zip(gxs, ts)]
    dts = [torch.empty_like(t) for t in ts]
    dcs = [torch.empty_like(c) for c in cs]
    solve_backward(grid, ts, cs, lam, ys, gxs, dts, dcs, pcg_iters)
    return dts, dcs


def _autograd_functions():
    import torch

    class BilateralSolve(torch.autograd.Function):
        """x = solve(t, c) on a prebuilt, bistochastised grid of ONE image:
        ``BilateralSolve.apply(t, c, grid, lam, pcg_iters)``.

        forward saves only the bilateral-space solution y (C x V), as Sec. 3
        notes; backward runs a second PCG with the same A (fbs_solve_backward)
        to produce dL/dt and dL/dc."""

        @staticmethod
        def forward(ctx, t, c, grid, lam, pcg_iters):
            if grid.n_images != 1:
                raise ValueError("BilateralSolve takes a one-image grid; use "
                                 "BilateralSolveBatch (bilateral_solve with lists) for a batch")
            ts, cs, xs, ys = _forward_batch(grid, [t], [c], lam, pcg_iters)
            ctx.save_for_backward(ts[0], cs[0], ys[0])
            ctx.grid, ctx.lam, ctx.iters = grid, lam, pcg_iters
            return xs[0]

        @staticmethod
        def backward(ctx, gx):
            t, c, y = ctx.saved_tensors
            dts, dcs = _backward_batch(ctx.grid, [t], [c], [y], [gx], ctx.lam, ctx.iters)
            return dts[0], dcs[0], None, None, None

    class BilateralSolveBatch(torch.autograd.Function):
        """Every image of a batched grid in one forward launch sequence and one
        backward: ``BilateralSolveBatch.apply(grid, lam, pcg_iters, t_0, ..,
        t_{n-1}, c_0, .., c_{n-1})`` returns (x_0, .., x_{n-1}).  lam is one
        value or one per image.  forward saves the targets, confidences and
        the solutions y_k only; backward is one fbs_solve_backward call for
        the whole batch."""

        @staticmethod
        def forward(ctx, grid, lam, pcg_iters, *tc):
            n = grid.n_images
            if len(tc) != 2 * n:
                raise ValueError(f"expected {n} targets and {n} confidences")
            ts, cs, xs, ys = _forward_batch(grid, tc[:n], tc[n:], lam, pcg_iters)
            ctx.save_for_backward(*ts, *cs, *ys)
            ctx.grid, ctx.lam, ctx.iters, ctx.n = grid, lam, pcg_iters, n
            return tuple(xs)

        @staticmethod
        def backward(ctx, *gxs):
            n = ctx.n
            saved = ctx.saved_tensors
            ts, cs, ys = saved[:n], saved[n:2 * n], saved[2 * n:]
            dts, dcs = _backward_batch(ctx.grid, ts, cs, ys, gxs, ctx.lam, ctx.iters)
            return (None, None, None, *dts, *dcs)

    return BilateralSolve, BilateralSolveBatch


_FUNCS = None


def _functions():
    global _FUNCS
    if _FUNCS is None:
        _FUNCS = _autograd_functions()
    return _FUNCS


def bilateral_solve(t, c, grid: Grid, lam, pcg_iters: int = 25):
    """Differentiable solve.  t, c tensors: one image (BilateralSolve), x
    returned.  t, c lists with one entry per image of the grid: the whole
    batch (BilateralSolveBatch), a list of x returned."""
    if isinstance(t, (list, tuple)):
        if not isinstance(c, (list, tuple)) or len(t) != len(c):
            raise ValueError("lists of targets and confidences of equal length")
        return list(_functions()[1].apply(grid, lam, pcg_iters, *t, *c))
    return _functions()[0].apply(t, c, grid, lam, pcg_iters)


def __getattr__(name):
    # fbs.BilateralSolve / fbs.BilateralSolveBatch (torch.autograd.Function
    # classes), built on first access so that importing the binding does not
    # import torch
    if name == "BilateralSolve":
        return _functions()[0]
    if name == "BilateralSolveBatch":
        return _functions()[1]
    raise AttributeError(f"module {__name__!r} has no attribute {name!r}")
