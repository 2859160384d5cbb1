"""Helpers shared by the GPU tests: run the CUDA path through the C ABI
binding and the oracle on the same seeded inputs."""
import numpy as np

import oracle

REL_L2_TOL = 1e-5     # rel-L2 bound on y and x at equal iteration counts


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


PCG_LAUNCH = {"mode": 0}    # fbs.PCG_AUTO; tests may switch to PCG_PERSISTENT / PCG_PER_PHASE
PCG_FORM = {"form": 0}      # fbs.PCG_FORM_STANDARD; tests may switch to PCG_FORM_SINGLE
PRECOND = {"kind": 0}       # fbs.PRECOND_JACOBI; tests may switch to PRECOND_HIERARCHICAL


def gpu_grid(insts, bistoch_iters=2):
    from paper_1511_03296_gb300 import fbs
    yuv = [to_dev(i.yuv) for i in insts]
    g = fbs.grid_build(yuv, [i.sigma_xy for i in insts], [i.sigma_l for i in insts],
                       [i.sigma_uv for i in insts])
    fbs.set_option(g, fbs.OPT_PCG_LAUNCH, PCG_LAUNCH["mode"])
    fbs.set_option(g, fbs.OPT_PCG_FORM, PCG_FORM["form"])
    fbs.set_option(g, fbs.OPT_PRECONDITIONER, PRECOND["kind"])
    if bistoch_iters:
        fbs.bistochastize(g, bistoch_iters)
    return g


def gpu_solve(g, insts, pcg_iters=25):
    import torch
    from paper_1511_03296_gb300 import fbs
    t = [to_dev(i.t) for i in insts]
    c = [to_dev(i.c) for i in insts]
    x = [torch.empty_like(tt) for tt in t]
    y = [torch.empty((i.channels, g.vertex_counts[k]), device="cuda")
         for k, i in enumerate(insts)]
    fbs.solve(g, t, c, [i.lam for i in insts], pcg_iters, x=x, y=y)
    fbs.grid_sync(g)
    return [xx.cpu().numpy() for xx in x], [yy.cpu().numpy() for yy in y]


def oracle_grid(inst, bistoch_iters=2):
    return oracle.build_grid(inst.yuv, inst.sigma_xy, inst.sigma_l, inst.sigma_uv, bistoch_iters)


def assert_grid_bit_exact(g, k, og, with_n=True):
    from paper_1511_03296_gb300 import fbs
    keys, vid, m, nbr, n = fbs.grid_export(g, k, with_n=with_n)
    assert keys.shape == og.vkey.shape, (keys.shape, og.vkey.shape)
    assert np.array_equal(keys, og.vkey)
    assert np.array_equal(vid, og.vid)
    assert np.array_equal(m, og.m)
    assert np.array_equal(nbr, og.nbr)
    if with_n:
        assert np.array_equal(n.view(np.uint64), og.n.view(np.uint64)), \
            f"n differs in {(n != og.n).sum()} of {n.size} entries"
