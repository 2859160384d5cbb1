"""Write robust_sensitivity.json: how far the FP64 robust solve (supplement
Alg. 3) moves when the state carried between its IRLS iterations is rounded
to float32, as any implementation with FP32 vectors must store it.

Calls only the oracle.  For the 1400 x 1000 robust workload (sigma = 4,
lambda = 0.25, sigma_gm = 1, 25 PCG iterations per solve) it records, for
each IRLS count k = 1..10, the rel-L2 distance between the plain FP64 loop
and the same loop with
  - the solution y of every solve rounded to float32 ("y"), or
  - the right-hand side b = S(c o t) of every solve rounded to float32 ("b"),
  - every quantity an FP32-vector implementation keeps in float32 rounded
    to float32 at every IRLS step: the weights, b, the diagonal of A and
    M^-1, the bistochastisation vector n and the solution y ("store32"),
  - the same with each value moved instead by a seeded uniform amount
    within half a float32 ulp, three seeds ("store32_draws"): other
    representation errors of the same size, as another implementation's
    rounding would make.
For the last two it records the sliced output x = S^T y too ("_x").  The
GPU parity test of the robust solver takes as its tolerance the largest of
the store32 deviations (of y for y, of x for x).

    python tests/golden/make_robust_sensitivity.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1511_03296_gb300 import synth  # noqa: E402

F32 = lambda a: np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


def f32_moved(seed):
    """A float32-sized representation error of another pattern: each value
    moved by a seeded uniform amount within half a float32 ulp of it (the
    error round-to-nearest makes, drawn independently)."""
    rng = np.random.default_rng(seed)

    def r(a):
        a = np.asarray(a, np.float64)
        ulp = np.spacing(np.abs(a).astype(np.float32)).astype(np.float64)
        return a + ulp * rng.uniform(-0.5, 0.5, a.shape)
    return r


def irls(g, t, c0, lam, sigma_gm, iters, pcg_iters, round_y=False, round_b=False, store=None):
    """Alg. 3 assembled from oracle steps; returns y after each IRLS iteration.
    store: a rounding function applied to everything kept in float32."""
    s2 = sigma_gm * sigma_gm
    c = c0.astype(np.float64)
    n = g.n if store is None else store(g.n)
    out = []
    for _ in range(iters):
        sc = np.bincount(g.vid, weights=c, minlength=g.V)
        b = np.bincount(g.vid, weights=c * t, minlength=g.V)
        if round_b:
            b = F32(b)
        a, minv = oracle.diag(g.m, g.nbr, n, sc, lam)
        if store is not None:
            b, a, minv = store(b), store(a), store(minv)
        y = oracle.pcg(g.nbr, n, a, minv, lam, b, oracle.flat_init(b, sc), pcg_iters)
        if round_y:
            y = F32(y)
        if store is not None:
            y = store(y)
        out.append(y)
        e = y[g.vid] - t
        c = 2.0 * s2 / (s2 + e * e) ** 2
        if store is not None:
            c = store(c)
    return out


def main():
    wl = synth.robust_1400x1000()
    inst = wl.instances[0]
    g = oracle.build_grid(inst.yuv, inst.sigma_xy, inst.sigma_l, inst.sigma_uv, wl.bistoch_iters)
    t = inst.t.reshape(-1).astype(np.float64)
    c0 = inst.c.reshape(-1)
    ref = irls(g, t, c0, inst.lam, wl.sigma_gm, wl.irls_iters, wl.pcg_iters)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    res = {"_cite": "supplement Sec. 3, Alg. 3 (robust bilateral solver); written by "
                    "tests/golden/make_robust_sensitivity.py from the oracle only",
           "workload": wl.name, "sigma_gm": wl.sigma_gm, "pcg_iters": wl.pcg_iters}
    for key, kw in (("y", {"round_y": True}), ("b", {"round_b": True}), ("store32", {"store": F32})):
        pert = irls(g, t, c0, inst.lam, wl.sigma_gm, wl.irls_iters, wl.pcg_iters, **kw)
        res[key] = [rel(p, r) for p, r in zip(pert, ref)]
        if key == "store32":            # the sliced output x = S^T y as well
            res["store32_x"] = [rel(p[g.vid], r[g.vid]) for p, r in zip(pert, ref)]
    res["store32_draws"], res["store32_draws_x"] = [], []
    for seed in (1, 2, 3):
        pert = irls(g, t, c0, inst.lam, wl.sigma_gm, wl.irls_iters, wl.pcg_iters,
                    store=f32_moved(seed))
        res["store32_draws"].append([rel(p, r) for p, r in zip(pert, ref)])
        res["store32_draws_x"].append([rel(p[g.vid], r[g.vid]) for p, r in zip(pert, ref)])
    # cross-check: the assembled loop reproduces the oracle's own robust solve
    oy, _ = oracle.solve_robust(g, inst.t, inst.c, inst.lam, wl.sigma_gm, wl.irls_iters,
                                wl.pcg_iters)
    res["assembled_vs_oracle"] = rel(ref[-1], oy[0])
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "robust_sensitivity.json")
    with open(path, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
