"""Independent dense constructions used to pin the oracle on tiny images.

Nothing here calls the oracle: keys are quantised with exact rational
arithmetic, vertices come from ``numpy.unique``, neighbours from an O(V^2)
field-by-field search, and S, Bbar, A, W-hat are assembled as dense
matrices straight from the equations of Sec. 2 and the supplement.
"""
from fractions import Fraction

import numpy as np

SHIFT = {"x": 36, "y": 48, "l": 24, "u": 12, "v": 0}
DIMS = ("x", "y", "l", "u", "v")


def exact_round_half_up(p: float, sigma: float) -> int:
    """floor(p / sigma + 1/2) in exact rational arithmetic."""
    q = Fraction(p) / Fraction(sigma) + Fraction(1, 2)
    return q.numerator // q.denominator


def exact_keys(yuv, sxy, sl, suv):
    """Packed keys via exact rationals (slow; tiny images only)."""
    _, h, w = yuv.shape
    out = np.empty(h * w, dtype=np.uint64)
    for r in range(h):
        for col in range(w):
            f = {"x": exact_round_half_up(col, sxy), "y": exact_round_half_up(r, sxy),
                 "l": exact_round_half_up(float(yuv[0, r, col]), sl),
                 "u": exact_round_half_up(float(yuv[1, r, col]), suv),
                 "v": exact_round_half_up(float(yuv[2, r, col]), suv)}
            k = 0
            for d in DIMS:
                assert 0 <= f[d] <= 4095
                k |= f[d] << SHIFT[d]
            out[r * w + col] = k
    return out


def fields(vkey):
    vkey = np.asarray(vkey, dtype=np.uint64)
    return np.stack([((vkey >> np.uint64(SHIFT[d])) & np.uint64(4095)).astype(np.int64)
                     for d in DIMS], axis=1)


def brute_neighbours(vkey):
    """nbr[v][2d+s] by comparing every pair of vertices field by field."""
    F = fields(vkey)
    V = F.shape[0]
    nbr = -np.ones((V, 10), dtype=np.int64)
    for v in range(V):
        diff = F - F[v]
        nz = (diff != 0).sum(axis=1)
        for u in np.nonzero(nz == 1)[0]:
            d = int(np.nonzero(diff[u])[0][0])
            s = int(diff[u, d])
            if s == -1:
                nbr[v, 2 * d] = u
            elif s == 1:
                nbr[v, 2 * d + 1] = u
    return nbr


def dense_S(vid, V):
    N = len(vid)
    S = np.zeros((V, N))
    S[np.asarray(vid, dtype=np.int64), np.arange(N)] = 1.0
    return S


def dense_Bbar(nbr):
    """Bbar = sum over dims of the [1, 2, 1] stencil = 10 I + adjacency."""
    V = nbr.shape[0]
    B = 10.0 * np.eye(V)
    for v in range(V):
        for k in range(10):
            u = nbr[v, k]
            if u >= 0:
                B[v, u] += 1.0
    return B


def dense_A(m, n, Bbar, sc, lam):
    """A = lambda (D_m - D_n Bbar D_n) + diag(S c)  (Eq. (6))."""
    Dn = np.diag(n)
    return lam * (np.diag(np.asarray(m, float)) - Dn @ Bbar @ Dn) + np.diag(sc)


def dense_What(S, m, n, Bbar):
    """W-hat = S^T D_m^-1 D_n Bbar D_n D_m^-1 S  (Eq. (4))."""
    Dl = np.diag(np.asarray(n, float) / np.asarray(m, float))
    return S.T @ Dl @ Bbar @ Dl @ S
