"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test compares the oracle with an independent construction (exact
rationals, numpy.unique, brute force, dense linear algebra, closed forms,
invariants, finite differences), so that a dropped term, a wrong sign or
index or a transposed operand in ``oracle/fbs_oracle.c`` fails one of them.
"""
import json
import os
import types

import numpy as np
import pytest

import oracle
from paper_1511_03296_gb300 import synth
from tests import dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny(seed=11, h=20, w=28, sig=(6.0, 24.0, 24.0), lam=4.0, C=2, npoly=3):
    return synth.make_tiny(seed, h, w, npoly, C, sig, lam)


def pack(fields):
    k = 0
    for d, f in zip(dense.DIMS, fields):
        k |= int(f) << dense.SHIFT[d]
    return k


# ---------------------------------------------------------------- keys ----

@pytest.mark.parametrize("name", ["keys_2x3.json", "grid_1x5.json"])
def test_keys_golden(name):
    g = json.load(open(os.path.join(GOLDEN, name)))
    h, w = g["height"], g["width"]
    yuv = np.stack([np.array(g[p], np.float32).reshape(h, w) for p in "luv"])
    k = oracle.keys(yuv, g["sigma_xy"], g["sigma_l"], g["sigma_uv"])
    if "fields" in g:
        assert [int(x) for x in k] == [pack(f) for f in g["fields"]]
    vkey, vid, m, nbr = oracle.grid(k)
    assert vid.tolist() == g["vid"]
    assert m.tolist() == g["m"]
    if "vkey_fields" in g:
        assert [int(x) for x in vkey] == [pack(f) for f in g["vkey_fields"]]
    if "nbr" in g:
        assert nbr.tolist() == g["nbr"]


def test_keys_exact_rational():
    inst = tiny(seed=3, h=12, w=17, sig=(3.0, 5.0, 7.0))
    # plant exact ties (k + 1/2) sigma and their float32 neighbours
    yuv = inst.yuv.copy()
    ties = np.array([2.5, 7.5, 12.5, 17.5], np.float32)
    yuv[0, 0, :4] = ties * 5.0
    yuv[0, 1, :4] = np.nextafter(ties * 5.0, np.float32(0))
    yuv[1, 2, :4] = ties * 7.0
    yuv[2, 3, :4] = np.nextafter(ties * 7.0, np.float32(1e9))
    got = oracle.keys(yuv, 3.0, 5.0, 7.0)
    want = dense.exact_keys(yuv, 3.0, 5.0, 7.0)
    assert np.array_equal(got, want)


def test_keys_non_integer_sigma():
    inst = tiny(seed=4, h=9, w=13)
    yuv = inst.yuv
    for sig in [(1.7, 2.3, 3.1), (0.75, 0.5, 1.25)]:
        assert np.array_equal(oracle.keys(yuv, *sig), dense.exact_keys(yuv, *sig))


@pytest.mark.parametrize("bad", [-3.0, np.nan, 4095.5 * 4.0 + 1.0])
def test_keys_out_of_range(bad):
    yuv = np.full((3, 2, 2), 10.0, np.float32)
    yuv[1, 1, 1] = bad
    with pytest.raises(oracle.OracleError):
        oracle.keys(yuv, 2.0, 4.0, 4.0)


def test_keys_field_max_is_inclusive():
    yuv = np.full((3, 1, 1), 0.0, np.float32)
    yuv[0] = 4095.0 * 4.0 + 1.99     # rounds to 4095, still in range
    k = oracle.keys(yuv, 1.0, 4.0, 4.0)
    assert int(k[0]) >> 24 & 4095 == 4095


# ---------------------------------------------------------------- grid ----

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_grid_matches_unique_and_brute_force(seed):
    inst = tiny(seed=seed, h=24, w=32, sig=(4.0, 8.0, 8.0))
    k = oracle.keys(inst.yuv, inst.sigma_xy, inst.sigma_l, inst.sigma_uv)
    vkey, vid, m, nbr = oracle.grid(k)
    u, inv, cnt = np.unique(k, return_inverse=True, return_counts=True)
    assert np.array_equal(vkey, u)
    assert np.array_equal(vid, inv.astype(np.uint32))
    assert np.array_equal(m, cnt.astype(np.uint32))
    assert np.array_equal(nbr, dense.brute_neighbours(vkey))
    assert (nbr >= 0).any(), "test image should have some neighbours"


def test_grid_no_wrap_at_field_edges():
    # v field 0 next to a vertex whose u is one less and v = 4095: not a neighbour
    yuv = np.zeros((3, 1, 2), np.float32)
    yuv[:, 0, 0] = (0.0, 5.0, 0.0)
    yuv[:, 0, 1] = (0.0, 4.0, 4095.0)
    k = oracle.keys(yuv, 100.0, 1.0, 1.0)
    vkey, vid, m, nbr = oracle.grid(k)
    assert int(vkey[1]) - int(vkey[0]) == 1  # adjacent packed keys
    assert (nbr == -1).all()


def test_SSt_is_Dm():
    inst = tiny(seed=5)
    g = oracle.build_grid(inst.yuv, inst.sigma_xy, inst.sigma_l, inst.sigma_uv, 2)
    S = dense.dense_S(g.vid, g.V)
    assert np.array_equal(S @ S.T, np.diag(g.m.astype(float)))   # supplement Eq. (5)
    assert int(g.m.sum()) == g.N


# ---------------------------------------------------- bistochastisation ----

def _grid(seed=6, **kw):
    inst = tiny(seed=seed, **kw)
    g = oracle.build_grid(inst.yuv, inst.sigma_xy, inst.sigma_l, inst.sigma_uv, None)
    return inst, g


def test_bistoch_one_sweep_closed_form():
    _, g = _grid()
    B = dense.dense_Bbar(dense.brute_neighbours(g.vkey))
    n1 = oracle.bistochastize(g.m, g.nbr, 1)
    # from n = 1: n <- sqrt(m / (Bbar 1))   (Alg. 1)
    assert np.allclose(n1, np.sqrt(g.m / (B @ np.ones(g.V))), rtol=1e-15, atol=0)
    n2 = oracle.bistochastize(g.m, g.nbr, 2)
    assert np.allclose(n2, np.sqrt(n1 * g.m / (B @ n1)), rtol=1e-14, atol=0)


def test_bistoch_zero_sweeps_is_ones():
    _, g = _grid()
    assert np.array_equal(oracle.bistochastize(g.m, g.nbr, 0), np.ones(g.V))


def test_bistoch_fixed_point_row_sums():
    _, g = _grid()
    B = dense.dense_Bbar(dense.brute_neighbours(g.vkey))
    res = []
    for it in (1, 4, 16, 64, 4000):
        n = oracle.bistochastize(g.m, g.nbr, it)
        res.append(np.linalg.norm(n * (B @ n) - g.m) / np.linalg.norm(g.m))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(res, res[1:])), res
    assert res[-1] < 1e-10
    # at the fixed point the bistochastised W-hat has unit row sums
    n = oracle.bistochastize(g.m, g.nbr, 4000)
    S = dense.dense_S(g.vid, g.V)
    W = dense.dense_What(S, g.m, n, B)
    assert np.allclose(W.sum(axis=1), 1.0, atol=1e-9)


# ------------------------------------------------------------ problem A, b -

def _problem(seed=7, iters=2, lam=4.0, C=2, **kw):
    inst = tiny(seed=seed, lam=lam, C=C, **kw)
    g = oracle.build_grid(inst.yuv, inst.sigma_xy, inst.sigma_l, inst.sigma_uv, iters)
    nb = dense.brute_neighbours(g.vkey)
    B = dense.dense_Bbar(nb)
    S = dense.dense_S(g.vid, g.V)
    c = inst.c.reshape(-1).astype(np.float64)
    t = inst.t.reshape(inst.channels, -1).astype(np.float64)
    sc = S @ c
    A = dense.dense_A(g.m, g.n, B, sc, lam)
    b = (S @ (c[None] * t).T).T
    return inst, g, S, B, A, b, sc


def test_splat_and_diag_match_dense():
    inst, g, S, B, A, b, sc = _problem()
    ob, osc = oracle.splat(g.vid, inst.t.reshape(inst.channels, -1), inst.c.reshape(-1), g.V)
    assert np.allclose(ob, b, rtol=1e-13, atol=1e-10)
    assert np.allclose(osc, sc, rtol=1e-13, atol=1e-12)
    a, minv = oracle.diag(g.m, g.nbr, g.n, osc, inst.lam)
    assert np.allclose(a, np.diag(A), rtol=1e-12, atol=1e-9 * inst.lam)
    assert np.allclose(minv, np.where(a > 0, 1.0 / a, 0.0))


def test_apply_A_matches_dense_and_is_symmetric():
    inst, g, S, B, A, b, sc = _problem()
    a, _ = oracle.diag(g.m, g.nbr, g.n, sc, inst.lam)
    cols = np.stack([oracle.apply_A(g.nbr, g.n, a, inst.lam, e) for e in np.eye(g.V)], axis=1)
    assert np.allclose(cols, A, rtol=1e-12, atol=1e-9 * inst.lam)
    assert np.array_equal(cols, cols.T)


@pytest.mark.parametrize("iters", [1, 4000])
def test_A_is_spd(iters):
    inst, g, S, B, A, b, sc = _problem(iters=iters)
    np.linalg.cholesky(A)     # raises if not SPD
    assert np.linalg.eigvalsh(A).min() > 0


def test_A_min_eigenvalue_two_sweeps_reported():
    # PSD is not guaranteed at an intermediate sweep count; record what it is
    inst, g, S, B, A, b, sc = _problem(iters=2)
    lam_min = np.linalg.eigvalsh(A).min()
    assert np.isfinite(lam_min)


def test_bilateral_loss_equals_pixel_loss():
    # supplement Eq. (9) (pixel space) equals 2 x Eq. (16) (bilateral space) under x = S^T y
    inst, g, S, B, A, b, sc = _problem(iters=3)
    c = inst.c.reshape(-1).astype(np.float64)
    t = inst.t.reshape(inst.channels, -1).astype(np.float64)[0]
    W = dense.dense_What(S, g.m, g.n, B)
    ob, osc = oracle.splat(g.vid, inst.t.reshape(inst.channels, -1), inst.c.reshape(-1), g.V)
    a, _ = oracle.diag(g.m, g.nbr, g.n, osc, inst.lam)
    rng = np.random.default_rng(0)
    for _ in range(3):
        y = rng.normal(size=g.V) * 50
        x = S.T @ y
        pix = x @ (inst.lam * (np.eye(g.N) - W) + np.diag(c)) @ x - 2 * (c * t) @ x + (c * t) @ t
        Ay = oracle.apply_A(g.nbr, g.n, a, inst.lam, y)
        bil = 0.5 * y @ Ay - ob[0] @ y + 0.5 * (c * t) @ t
        assert np.isclose(pix, 2 * bil, rtol=1e-10, atol=1e-6)


# ----------------------------------------------------------------- solve --

def test_lambda_zero_gives_weighted_mean():
    inst = tiny(seed=8, lam=0.0, C=2)
    g = oracle.build_grid(inst.yuv, inst.sigma_xy, inst.sigma_l, inst.sigma_uv, 2)
    y, x = oracle.solve(g, inst.t, inst.c, 0.0, 25)
    c = inst.c.reshape(-1).astype(np.float64)
    for ch in range(inst.channels):
        t = inst.t[ch].reshape(-1).astype(np.float64)
        num = np.bincount(g.vid, weights=c * t, minlength=g.V)
        den = np.bincount(g.vid, weights=c, minlength=g.V)
        want = np.where(den > 0, num / np.where(den > 0, den, 1), 0.0)
        assert np.allclose(y[ch], want, rtol=1e-14, atol=1e-12)


def test_zero_confidence_vertex_stays_zero():
    inst = tiny(seed=9, lam=0.0, C=1)
    c = inst.c.copy()
    c[:, :] = 0.0
    g = oracle.build_grid(inst.yuv, inst.sigma_xy, inst.sigma_l, inst.sigma_uv, 2)
    y, x = oracle.solve(g, inst.t, c, 0.0, 25)
    assert np.array_equal(y, np.zeros_like(y))


def test_constant_target_is_preserved():
    inst = tiny(seed=10, lam=128.0, C=1)
    t = np.full_like(inst.t, 77.25)
    c = np.full_like(inst.c, 0.5)
    g = oracle.build_grid(inst.yuv, inst.sigma_xy, inst.sigma_l, inst.sigma_uv, 4000)
    y, x = oracle.solve(g, t, c, 128.0, 25)
    assert np.allclose(x, 77.25, rtol=1e-10, atol=0)


def test_pcg_converged_matches_dense_solve():
    inst, g, S, B, A, b, sc = _problem(iters=2, lam=16.0)
    y, _ = oracle.solve(g, inst.t, inst.c, inst.lam, 600)
    ystar = np.linalg.solve(A, b.T).T
    assert np.allclose(y, ystar, rtol=1e-9, atol=1e-9 * np.abs(ystar).max())


def test_pcg_energy_error_decreases():
    inst, g, S, B, A, b, sc = _problem(iters=1, lam=16.0, C=1)
    a, minv = oracle.diag(g.m, g.nbr, g.n, sc, inst.lam)
    y0 = oracle.flat_init(b[0], sc)
    ystar = np.linalg.solve(A, b[0])
    errs = []
    for k in range(0, 30):
        yk = oracle.pcg(g.nbr, g.n, a, minv, inst.lam, b[0], y0, k)
        e = yk - ystar
        errs.append(e @ A @ e)
    assert all(e1 <= e0 * (1 + 1e-9) + 1e-18 for e0, e1 in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-6 * errs[0]


def test_pcg_matches_textbook_on_dense_matrix():
    # Jacobi PCG written against the dense A with numpy (Shewchuk B3 / Alg. 2)
    inst, g, S, B, A, b, sc = _problem(iters=2, lam=16.0, C=1)
    a, minv = oracle.diag(g.m, g.nbr, g.n, sc, inst.lam)
    y0 = oracle.flat_init(b[0], sc)
    Minv = np.diag(np.where(np.diag(A) > 0, 1.0 / np.diag(A), 0.0))
    yk, r = y0.copy(), b[0] - A @ y0
    d = Minv @ r
    delta = r @ d
    for _ in range(7):
        q = A @ d
        alpha = delta / (d @ q)
        yk = yk + alpha * d
        r = r - alpha * q
        s = Minv @ r
        delta, delta_old = r @ s, delta
        d = s + (delta / delta_old) * d
    got = oracle.pcg(g.nbr, g.n, a, minv, inst.lam, b[0], y0, 7)
    assert np.allclose(got, yk, rtol=1e-9, atol=1e-9 * np.abs(yk).max())


def test_slice_is_adjoint_of_splat():
    inst, g, S, B, A, b, sc = _problem(C=1)
    rng = np.random.default_rng(1)
    y = rng.normal(size=(1, g.V))
    gvec = rng.normal(size=(1, g.N)).astype(np.float32)
    x = oracle.slice_(g.vid, y)
    assert np.allclose(x, (S.T @ y[0])[None])
    Sg, _ = oracle.splat(g.vid, gvec, np.ones(g.N, np.float32), g.V)
    assert np.isclose((x * gvec).sum(), (y * Sg).sum(), rtol=1e-12)


# ------------------------------------------------------------ robust -------

def test_gm_weight_is_rho_prime_over_e():
    s = 1.3
    e = np.linspace(-6, 6, 41)
    e = e[e != 0]
    rho = lambda z: z * z / (s * s + z * z)
    h = 1e-6
    drho = (rho(e + h) - rho(e - h)) / (2 * h)
    w = 2 * s * s / (s * s + e * e) ** 2
    assert np.allclose(drho / e, w, rtol=1e-6)


def test_robust_first_iteration_is_plain_solve_and_loop_reweights():
    inst = tiny(seed=12, C=1, lam=2.0)
    g = oracle.build_grid(inst.yuv, inst.sigma_xy, inst.sigma_l, inst.sigma_uv, 2)
    y1, x1 = oracle.solve_robust(g, inst.t, inst.c, inst.lam, 3.0, 1, 25)
    yp, xp = oracle.solve(g, inst.t, inst.c, inst.lam, 25)
    assert np.array_equal(y1, yp)
    e = x1[0] - inst.t.reshape(-1)
    w = 2 * 9.0 / (9.0 + e * e) ** 2
    # second IRLS solve == plain solve with c = w(e); compare through float32 weights
    y2, _ = oracle.solve_robust(g, inst.t, inst.c, inst.lam, 3.0, 2, 25)
    y2p, _ = oracle.solve(g, inst.t, w.astype(np.float32), inst.lam, 25)
    assert np.allclose(y2, y2p, rtol=1e-5, atol=1e-4)


def test_robust_objective_decreases():
    # with exact inner solves IRLS is majorise-minimise for
    # F(x) = lambda x^T (I - W) x + 2 sum rho(x - t)
    inst = tiny(seed=13, h=16, w=20, C=1, lam=1.0, sig=(5.0, 30.0, 30.0))
    t = inst.t.copy()
    t[0, 3, 4] = 250.0
    t[0, 10, 12] = 0.0
    g = oracle.build_grid(inst.yuv, inst.sigma_xy, inst.sigma_l, inst.sigma_uv, 4000)
    S = dense.dense_S(g.vid, g.V)
    W = dense.dense_What(S, g.m, g.n, dense.dense_Bbar(dense.brute_neighbours(g.vkey)))
    s = 4.0
    F = []
    for it in range(2, 7):
        _, x = oracle.solve_robust(g, t, inst.c, inst.lam, s, it, 3000)
        e = x[0] - t.reshape(-1)
        F.append(inst.lam * x[0] @ (np.eye(g.N) - W) @ x[0] + 2 * np.sum(e * e / (s * s + e * e)))
    assert all(f1 <= f0 + 1e-7 * abs(f0) for f0, f1 in zip(F, F[1:])), F


# ------------------------------------------------------------- backward ----

def _seg_crop():
    rng = np.random.Generator(np.random.PCG64(5))
    inst = synth.segmentation_instance(rng, 48, 64, 21, (8.0, 4.0, 3.0), 128.0, blob_sigma=6.0)
    return synth.crop(inst, 8, 16, 24, 32)


def _dense_forward(g, t, c, lam):
    C = t.shape[0]
    b, sc = oracle.splat(g.vid, t.reshape(C, -1), c.reshape(-1), g.V)
    a, _ = oracle.diag(g.m, g.nbr, g.n, sc, lam)
    A = np.stack([oracle.apply_A(g.nbr, g.n, a, lam, e) for e in np.eye(g.V)], axis=1)
    y = np.linalg.solve(A, b.T).T
    return y, y[:, g.vid]


def test_backward_matches_finite_differences():
    inst = _seg_crop()
    g = oracle.build_grid(inst.yuv, inst.sigma_xy, inst.sigma_l, inst.sigma_uv, 2)
    C = inst.channels
    label = inst.label.reshape(C, -1).astype(np.float64)
    t64 = inst.t.reshape(C, -1).astype(np.float64)
    c64 = inst.c.reshape(-1).astype(np.float64)

    def loss(t, c):
        # the forward in FP64 end to end (the oracle's splat takes float32, so
        # assemble b and S c here from the dense S built independently)
        S = dense.dense_S(g.vid, g.V)
        sc = S @ c
        b = (S @ (c[None] * t).T).T
        a, _ = oracle.diag(g.m, g.nbr, g.n, sc, inst.lam)
        A = np.stack([oracle.apply_A(g.nbr, g.n, a, inst.lam, e) for e in np.eye(g.V)], axis=1)
        y = np.linalg.solve(A, b.T).T
        x = y[:, g.vid]
        return np.mean((x - label) ** 2), y, x

    L0, y, x = loss(t64, c64)
    dx = 2.0 * (x - label) / x.size
    dt, dc = oracle.backward(g, inst.t, inst.c, inst.lam, 400, y, dx)
    rng = np.random.default_rng(2)
    for _ in range(6):
        ch, i = int(rng.integers(C)), int(rng.integers(g.N))
        h = 1e-4
        tp, tm = t64.copy(), t64.copy()
        tp[ch, i] += h
        tm[ch, i] -= h
        fd = (loss(tp, c64)[0] - loss(tm, c64)[0]) / (2 * h)
        assert np.isclose(dt[ch, i], fd, rtol=1e-5, atol=1e-12), (ch, i, dt[ch, i], fd)
    for _ in range(6):
        i = int(rng.integers(g.N))
        h = 1e-5
        cp, cm = c64.copy(), c64.copy()
        cp[i] += h
        cm[i] -= h
        fd = (loss(t64, cp)[0] - loss(t64, cm)[0]) / (2 * h)
        assert np.isclose(dc[i], fd, rtol=1e-5, atol=1e-12), (i, dc[i], fd)


# ---- single-reduction PCG (Chronopoulos-Gear form of the same iteration) ----

def test_pcg_single_equals_standard_iterates():
    # the two forms produce the same iterates in exact arithmetic; compare
    # every iteration count against the pinned standard form
    inst, g, S, B, A, b, sc = _problem(iters=2, lam=16.0, C=1)
    a, minv = oracle.diag(g.m, g.nbr, g.n, sc, inst.lam)
    y0 = oracle.flat_init(b[0], sc)
    for k in range(0, 16):
        ys = oracle.pcg(g.nbr, g.n, a, minv, inst.lam, b[0], y0, k)
        y1 = oracle.pcg_single(g.nbr, g.n, a, minv, inst.lam, b[0], y0, k)
        assert np.allclose(y1, ys, rtol=1e-9, atol=1e-9 * np.abs(ys).max()), k


def _pcg_zform_dense(A, minv, b, y0, iters):
    """Jacobi PCG with the recurrence the GPU's FP32 phase 1 uses from the
    second iteration: d = z + beta d_old is linear in z = M^-1 r, so
    A d = A z + beta (A d_old); the product A d itself is formed only in
    iteration 0.  Written here from that identity on a dense A, with the
    oracle's guards (alpha = 0 unless d^T A d > 0 and rho != 0; beta = 0 when
    rho = 0)."""
    y = y0.copy()
    r = b - A @ y
    z = minv * r
    rho = r @ z
    d = z.copy()
    q = A @ d
    for it in range(iters):
        if it > 0:
            d = z + beta * d
            q = A @ z + beta * q
        dq = d @ q
        alpha = rho / dq if (dq > 0.0 and rho != 0.0) else 0.0
        y = y + alpha * d
        r = r - alpha * q
        z = minv * r
        rho_next = r @ z
        beta = rho_next / rho if rho != 0.0 else 0.0
        rho = rho_next
    return y


def test_pcg_zform_recurrence_equals_standard_iterates():
    # A d = A z + beta A d_old: the z form's iterates equal the standard
    # form's (the oracle's) at every iteration count in exact arithmetic
    inst, g, S, B, A, b, sc = _problem(iters=2, lam=16.0, C=1)
    a, minv = oracle.diag(g.m, g.nbr, g.n, sc, inst.lam)
    y0 = oracle.flat_init(b[0], sc)
    for k in range(0, 16):
        ys = oracle.pcg(g.nbr, g.n, a, minv, inst.lam, b[0], y0, k)
        yz = _pcg_zform_dense(A, minv, b[0], y0, k)
        assert np.allclose(yz, ys, rtol=1e-9, atol=1e-9 * np.abs(ys).max()), k


def test_pcg_single_converged_matches_dense_solve():
    inst, g, S, B, A, b, sc = _problem(iters=2, lam=16.0)
    with oracle.pcg_form("single"):
        y, _ = oracle.solve(g, inst.t, inst.c, inst.lam, 600)
    ystar = np.linalg.solve(A, b.T).T
    assert np.allclose(y, ystar, rtol=1e-9, atol=1e-9 * np.abs(ystar).max())


def test_pcg_single_zero_right_hand_side_stays_zero():
    inst, g, S, B, A, b, sc = _problem(iters=2, lam=16.0, C=1)
    a, minv = oracle.diag(g.m, g.nbr, g.n, sc, inst.lam)
    z = np.zeros_like(b[0])
    y = oracle.pcg_single(g.nbr, g.n, a, minv, inst.lam, z, z, 25)
    assert np.all(y == 0.0)


def test_pcg_form_context_restores_standard():
    inst, g, S, B, A, b, sc = _problem(iters=2, lam=16.0, C=1)
    y_std, _ = oracle.solve(g, inst.t, inst.c, inst.lam, 5)
    with oracle.pcg_form("single"):
        y_one, _ = oracle.solve(g, inst.t, inst.c, inst.lam, 5)
    y_again, _ = oracle.solve(g, inst.t, inst.c, inst.lam, 5)
    assert np.array_equal(y_std, y_again)
    assert np.allclose(y_one, y_std, rtol=1e-9, atol=1e-9 * np.abs(y_std).max())


# ---- bilateral-space pyramid and the hierarchical preconditioner (Sec. 4) ----

def _halve(keys):
    out = np.zeros_like(keys)
    for shift in (48, 36, 24, 12, 0):
        out |= ((keys >> np.uint64(shift)) & np.uint64(4095)) >> np.uint64(1) << np.uint64(shift)
    return out


@pytest.mark.parametrize("h,w,sig", [(40, 56, (8.0, 4.0, 3.0)),
                                     # sparse: levels shrink by less than half, so
                                     # the parents outnumber twice the vertices
                                     (30, 400, (1.0, 4.0, 3.0))])
def test_pyramid_matches_brute_force(h, w, sig):
    inst = synth.make_tiny(60, h, w, 5, 1, sig)
    g = oracle.build_grid(inst.yuv, inst.sigma_xy, inst.sigma_l, inst.sigma_uv, 2)
    sizes, parent = oracle.pyramid(g.vkey)
    if sig[0] == 1.0:
        assert parent.size > 2 * g.V
    keys, off = g.vkey.astype(np.uint64), 0
    for k in range(len(sizes) - 1):
        assert keys.size == sizes[k]
        h = _halve(keys)
        up = np.unique(h)
        assert np.array_equal(parent[off:off + keys.size], np.searchsorted(up, h))
        off += keys.size
        keys = up
    assert sizes[-1] == 1 and keys.size == 1


def _hier_problem(seed=61, h=24, w=32, C=1):
    inst = synth.make_tiny(seed, h, w, 4, C)
    g = oracle.build_grid(inst.yuv, inst.sigma_xy, inst.sigma_l, inst.sigma_uv, 2)
    b, sc = oracle.splat(g.vid, inst.t, inst.c, g.V)
    a, minv = oracle.diag(g.m, g.nbr, g.n, sc, inst.lam)
    return inst, g, b, sc, a, minv


def test_hier_preconditioner_is_symmetric_positive_definite():
    inst, g, b, sc, a, minv = _hier_problem()
    with oracle.hierarchical(g) as H:
        M = np.stack([H.precond(a, e) for e in np.eye(g.V)], axis=1)
    assert np.allclose(M, M.T, rtol=1e-12, atol=1e-14 * np.abs(M).max())
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_hier_preconditioner_degenerates_to_jacobi():
    # coarse levels weighted by alpha^-(beta + k): with beta large only the
    # finest level (Jacobi) remains
    inst, g, b, sc, a, minv = _hier_problem()
    r = np.random.default_rng(1).normal(size=g.V)
    with oracle.hierarchical(g, prec=(2.0, 80.0), init=(4.0, 80.0)) as H:
        s = H.precond(a, r)
        y = H.init(b[0], sc)
    assert np.allclose(s, minv * r, rtol=1e-12, atol=0)
    assert np.allclose(y, oracle.flat_init(b[0], sc), rtol=1e-12, atol=0)


def test_hier_init_keeps_a_target_proportional_to_confidence():
    # b = kappa S c: numerator and denominator of the push-pull differ by kappa
    inst, g, b, sc, a, minv = _hier_problem()
    with oracle.hierarchical(g) as H:
        y = H.init(37.5 * sc, sc)
    assert np.allclose(y[sc > 0], 37.5, rtol=1e-12, atol=0)


def test_hier_pcg_converged_matches_dense_solve():
    inst, g, S, B, A, b, sc = _problem(iters=2, lam=16.0)
    with oracle.hierarchical(g):
        y, _ = oracle.solve(g, inst.t, inst.c, inst.lam, 400)
    ystar = np.linalg.solve(A, b.T).T
    assert np.allclose(y, ystar, rtol=1e-9, atol=1e-9 * np.abs(ystar).max())


def test_hier_converges_faster_than_jacobi():
    # the paper's claim (Sec. 4, figure on preconditioning and initialisation):
    # at equal iteration counts the hierarchical preconditioner and
    # initialisation leave a smaller objective gap than Jacobi with the flat
    # initialisation
    sig, lam = (8.0, 4.0, 3.0), 128.0
    inst = synth.make_tiny(70, 120, 160, 10, 1, sig, lam)
    g = oracle.build_grid(inst.yuv, *sig, 2)
    b, sc = oracle.splat(g.vid, inst.t, inst.c, g.V)
    a, minv = oracle.diag(g.m, g.nbr, g.n, sc, lam)

    def loss(y):
        return 0.5 * y @ oracle.apply_A(g.nbr, g.n, a, lam, y) - b[0] @ y

    f_star = loss(oracle.solve(g, inst.t, inst.c, lam, 2000)[0][0])
    for k in (10, 25):
        yj, _ = oracle.solve(g, inst.t, inst.c, lam, k)
        with oracle.hierarchical(g):
            yh, _ = oracle.solve(g, inst.t, inst.c, lam, k)
        assert loss(yh[0]) - f_star < 0.5 * (loss(yj[0]) - f_star), k


# ---- low-rank reduction of a wide target (supplement, multiple output channels) ----

def test_lowrank_rank_rule_closed_form():
    # orthogonal columns of norms 3, 0, 4, 1: the pivoted QR takes them in the
    # order 4, 3, 1 with a diagonal R, so the row masses are 16, 9, 1, 0 of a
    # total 26; the kept rows are the fewest whose mass reaches (1 - eps) 26
    rng = np.random.default_rng(0)
    U, _ = np.linalg.qr(rng.standard_normal((50, 4)))
    B = U * np.array([3.0, 0.0, 4.0, 1.0])
    for eps, t_exp in ((0.5, 1), (0.1, 2), (0.05, 2), (0.01, 3), (1e-9, 3)):
        Qt, Rt, t = oracle.lowrank_factors(B, eps)
        assert t == t_exp, (eps, t)
        # Q~ R~ keeps exactly the kept columns of B
        kept = np.argsort(-np.array([9.0, 0.0, 16.0, 1.0]), kind="stable")[:t]
        expect = np.zeros_like(B)
        expect[:, kept] = B[:, kept]
        assert np.allclose(Qt @ Rt, expect, atol=1e-12)


def test_lowrank_factors_invariants():
    # Q~ orthonormal; the dropped mass is at most eps of |B|_F^2; one row
    # fewer would drop more (t is minimal)
    rng = np.random.default_rng(1)
    B = rng.standard_normal((400, 9)) @ np.diag(2.0 ** -np.arange(9)) @ rng.standard_normal((9, 9))
    total = (B ** 2).sum()
    for eps in (0.2, 0.01, 1e-4):
        Qt, Rt, t = oracle.lowrank_factors(B, eps)
        assert np.allclose(Qt.T @ Qt, np.eye(t), atol=1e-12)
        assert ((B - Qt @ Rt) ** 2).sum() <= eps * total * (1 + 1e-9)
        if t > 1:
            assert ((B - Qt[:, :t - 1] @ Rt[:t - 1]) ** 2).sum() > eps * total


def test_lowrank_exact_rank_converged_equals_full_solve():
    # a 5-channel target of rank 2 (pixel-level combinations of two channels):
    # B = S(c o T) has rank 2, the reduction keeps 2 columns for any small
    # eps, and converged solves agree, as A^-1 B = (A^-1 Q~) R~ exactly
    inst = synth.make_tiny(71, 40, 56, 5, 2)
    t1, t2 = inst.t[0].astype(np.float64), inst.t[1].astype(np.float64)
    T = np.stack([t1, t2, t1 + t2, 0.0 * t1, 2.0 * t1 - t2]).astype(np.float32)
    g = oracle.build_grid(inst.yuv, inst.sigma_xy, inst.sigma_l, inst.sigma_uv, 2)
    y, x, t = oracle.solve_lowrank(g, T, inst.c, inst.lam, 600, 1e-9)
    assert t == 2
    yf, xf = oracle.solve(g, T, inst.c, inst.lam, 600)
    assert np.linalg.norm(x - xf) <= 1e-8 * np.linalg.norm(xf)
    assert np.abs(x[3]).max() == 0.0 or np.abs(x[3]).max() <= 1e-10 * np.abs(xf).max()


def test_lowrank_zero_target():
    inst = synth.make_tiny(72, 24, 32, 3, 3)
    g = oracle.build_grid(inst.yuv, inst.sigma_xy, inst.sigma_l, inst.sigma_uv, 2)
    y, x, t = oracle.solve_lowrank(g, np.zeros_like(inst.t), inst.c, inst.lam, 25, 0.01)
    assert t == 0 and not x.any() and not y.any()


def test_lowrank_tiny_eps_equals_full_solve_at_any_iteration_count_for_one_channel():
    # one channel: Q~ = b / |b| and R~ = |b|, and PCG is homogeneous of
    # degree 1 in b, so the reduced solve equals the plain one at every
    # iteration count
    inst = synth.make_tiny(73, 40, 56, 5, 1)
    g = oracle.build_grid(inst.yuv, inst.sigma_xy, inst.sigma_l, inst.sigma_uv, 2)
    for it in (0, 3, 25):
        _, x, t = oracle.solve_lowrank(g, inst.t, inst.c, inst.lam, it, 0.01)
        _, xf = oracle.solve(g, inst.t, inst.c, inst.lam, it)
        assert t == 1
        assert np.linalg.norm(x - xf) <= 1e-12 * np.linalg.norm(xf)


# ---- domain transform post-filter (Sec. 5; Gastal and Oliveira 2011, recursive form) ----

def test_domain_transform_keeps_constants():
    rng = np.random.default_rng(2)
    guide = rng.uniform(0, 255, size=(3, 17, 23)).astype(np.float32)
    x = np.full((2, 17, 23), 3.25)
    out = oracle.domain_transform(guide, x, 16.0, 32.0, 3)
    assert np.allclose(out, 3.25, rtol=0, atol=1e-12)


def test_domain_transform_impulse_response_closed_form():
    # one iteration on a single row of a flat guide (every step of length 1):
    # the forward then backward recursive filter of feedback a has the
    # two-sided impulse response (1 - a) / (1 + a) a^|n| away from the ends
    L, sig = 401, 4.0
    guide = np.zeros((3, 1, L), np.float32)
    x = np.zeros((1, 1, L))
    x[0, 0, L // 2] = 1.0
    out = oracle.domain_transform(guide, x, sig, 10.0, 1)[0, 0]
    a = np.exp(-np.sqrt(2.0) / sig)
    n = np.arange(L) - L // 2
    assert np.allclose(out, (1 - a) / (1 + a) * a ** np.abs(n), rtol=1e-12, atol=1e-15)


def test_domain_transform_stops_at_an_edge():
    # a hard edge in the guide and a tiny range bandwidth: nothing crosses it,
    # so each side is filtered as an image of its own
    rng = np.random.default_rng(3)
    H, W, k = 12, 30, 14
    guide = np.zeros((3, H, W), np.float32)
    guide[:, :, k + 1:] = 255.0
    x = rng.standard_normal((2, H, W))
    out = oracle.domain_transform(guide, x, 8.0, 1e-6, 3)
    left = oracle.domain_transform(guide[:, :, :k + 1], x[:, :, :k + 1], 8.0, 1e-6, 3)
    right = oracle.domain_transform(guide[:, :, k + 1:], x[:, :, k + 1:], 8.0, 1e-6, 3)
    assert np.allclose(out[:, :, :k + 1], left, rtol=0, atol=1e-12)
    assert np.allclose(out[:, :, k + 1:], right, rtol=0, atol=1e-12)
    assert not np.allclose(out, x)


# ---- hierarchical preconditioner and initialisation, hand-computed (Sec. 4) ----

def _hand_pyramid():
    # five vertices along x (x = 0, 1, 2, 3 and a second colour at x = 3):
    # halving x gives level 1 = {x=0: vertices 0, 1; x=1: vertices 2, 3, 4},
    # halving again gives the single top vertex, so P(1) = (1,1,1,1,1 | 2, 3 | 5)
    sh = {"x": 36, "y": 48, "l": 24, "u": 12, "v": 0}

    def key(**f):
        return sum(int(v) << sh[k] for k, v in f.items())

    vkey = np.array([key(x=0), key(x=1), key(x=2), key(x=3), key(x=3, l=1)], np.uint64)
    return types.SimpleNamespace(vkey=vkey)


def test_hand_pyramid_levels():
    sizes, parent = oracle.pyramid(_hand_pyramid().vkey)
    assert sizes.tolist() == [5, 2, 1]
    assert parent.tolist() == [0, 0, 1, 1, 1, 0, 0]


def test_hier_preconditioner_hand_computed():
    # M_hier^-1 = P^T(z_weight o P(1) o P(.) / P(diag A)) with (alpha, beta) =
    # (2, 5): z_weight = 1, 2^-6, 2^-7 on levels 0, 1, 2.  With diag(A) =
    # (1, 2, 3, 4, 5): P(diag A) = (3, 12) on level 1 and 15 on level 2, so
    # the level scalings are 1/a_v; 2^-6 * 2/3 = 1/96 and 2^-6 * 3/12 = 1/256;
    # 2^-7 * 5/15 = 1/384.  Dropping P(1), or weighting by alpha^-(beta k),
    # changes every coarse entry.
    a = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    expect = np.diag(1.0 / a)
    expect[:2, :2] += 1.0 / 96.0
    expect[2:, 2:] += 1.0 / 256.0
    expect += 1.0 / 384.0
    with oracle.hierarchical(_hand_pyramid(), prec=(2.0, 5.0)) as H:
        M = np.stack([H.precond(a, e) for e in np.eye(5)], axis=1)
    assert np.allclose(M, expect, rtol=1e-14, atol=0)


def test_hier_init_hand_computed():
    # y_hier = P^T(z_weight o P(b) / P(1)) / P^T(z_weight o P(Sc) / P(1)) with
    # (alpha, beta) = (4, 0): z_weight = 1, 1/4, 1/16.  b = (3, 0, 2, 5, 0),
    # Sc = (1, 0, 2, 1, 0):
    #   numerator   level 1: (3/2, 7/3)/4 = (3/8, 7/12); level 2: (10/5)/16 = 1/8
    #               -> (7/2, 1/2, 65/24, 137/24, 17/24)
    #   denominator level 1: (1/2, 3/3)/4 = (1/8, 1/4); level 2: (4/5)/16 = 1/20
    #               -> (47/40, 7/40, 23/10, 13/10, 3/10)
    b = np.array([3.0, 0.0, 2.0, 5.0, 0.0])
    sc = np.array([1.0, 0.0, 2.0, 1.0, 0.0])
    expect = np.array([140 / 47, 20 / 7, 325 / 276, 685 / 156, 85 / 36])
    with oracle.hierarchical(_hand_pyramid(), init=(4.0, 0.0)) as H:
        y = H.init(b, sc)
    assert np.allclose(y, expect, rtol=1e-14, atol=0)


# ---- domain transform: the iterations' sigma schedule (Gastal and Oliveira) ----

def _dt_three_samples(a):
    # one iteration on a 3-sample line with a flat guide (every step has
    # length 1, weight a): the forward pass is lower triangular, the backward
    # pass upper triangular, written out by hand from the recursion
    fwd = np.array([[1.0, 0.0, 0.0],
                    [a, 1.0 - a, 0.0],
                    [a * a, a * (1.0 - a), 1.0 - a]])
    bwd = np.array([[1.0 - a, a * (1.0 - a), a * a],
                    [0.0, 1.0 - a, a],
                    [0.0, 0.0, 1.0]])
    return bwd @ fwd


@pytest.mark.parametrize("iters", [2, 3])
def test_domain_transform_sigma_schedule(iters):
    # The cascade's per-iteration sigmas halve from one iteration to the next,
    # starting large, and their squares add up to sigma_s^2: for 2 iterations
    # (2, 1) sigma_s / sqrt(5), for 3 (4, 2, 1) sigma_s / sqrt(21).  On a
    # 3-sample line the iterations do not commute (the ends), so the order is
    # checked too; a reversed schedule moves the result by ~0.1.
    sig_s = 3.0
    sig = {2: [2 / 5 ** 0.5, 1 / 5 ** 0.5],
           3: [4 / 21 ** 0.5, 2 / 21 ** 0.5, 1 / 21 ** 0.5]}[iters]
    x = np.array([1.0, -2.0, 5.0])
    expect = x.copy()
    for s in sig:
        expect = _dt_three_samples(np.exp(-np.sqrt(2.0) / (s * sig_s))) @ expect
    guide = np.zeros((3, 1, 3), np.float32)
    out = oracle.domain_transform(guide, x.reshape(1, 1, 3), sig_s, 10.0, iters)[0, 0]
    assert np.allclose(out, expect, rtol=1e-14, atol=1e-15)
