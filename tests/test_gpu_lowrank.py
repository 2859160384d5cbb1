"""Parity of the low-rank reduction of a wide target (supplement, multiple
output channels: column-pivoted QR of B = S(c o t), rows kept by mass) on
the GPU with the oracle's ``solve_lowrank``: the rank chosen per image is
equal (an integer decided in FP64 on both sides, from inputs whose mass
spectrum has no near-tie at the cut-off) and x is within rel-L2 1e-5 at
equal iteration counts.  The GPU takes R from the pivoted Cholesky
factorisation of B^T B, the oracle from LAPACK's pivoted Householder QR:
the same R up to row signs, and x does not depend on those signs."""
import numpy as np
import pytest

from paper_1511_03296_gb300 import synth
from tests.gpu_util import REL_L2_TOL, gpu_grid, oracle_grid, rel_l2, to_dev

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1511_03296_gb300 import build, fbs
    build.build()
    fbs.load()
    assert torch.cuda.is_available()


def _scene(seed, h, w, n_present):
    rng = np.random.Generator(np.random.PCG64(seed))
    return synth.segmentation_instance(rng, h, w, 21, (8.0, 4.0, 3.0), 128.0, n_present=n_present)


def _gpu_lowrank(insts, iters, eps):
    import torch
    from paper_1511_03296_gb300 import fbs
    g = gpu_grid(insts, 2)
    t = [to_dev(i.t) for i in insts]
    c = [to_dev(i.c) for i in insts]
    x = [torch.empty_like(tt) for tt in t]
    ranks = fbs.solve_lowrank(g, t, c, [i.lam for i in insts], iters, eps, x=x)
    fbs.grid_sync(g)
    return ranks, [xx.cpu().numpy() for xx in x]


def _check(insts, iters=25, eps=0.01, expect_ranks=None):
    ranks, xs = _gpu_lowrank(insts, iters, eps)
    for k, inst in enumerate(insts):
        og = oracle_grid(inst, 2)
        _, ox, r = oracle.solve_lowrank(og, inst.t, inst.c, inst.lam, iters, eps)
        assert ranks[k] == r, (k, ranks[k], r)
        if expect_ranks is not None:
            assert r == expect_ranks[k]
        C = inst.t.shape[0]
        if r == 0:
            assert not xs[k].any()
        else:
            e = rel_l2(xs[k].reshape(C, -1), ox)
            assert e <= REL_L2_TOL, (k, e)
    return ranks


@pytest.mark.parametrize("eps", [0.1, 0.01, 1e-5])
@pytest.mark.parametrize("iters", [0, 5, 25])
def test_lowrank_scene(eps, iters):
    _check([_scene(1, 96, 128, 3)], iters, eps)


def test_lowrank_batch_of_mixed_images():
    zero = synth.make_tiny(5, 33, 47, 3, 4)
    zero.t[:] = 0.0
    insts = [_scene(2, 120, 160, 2), _scene(3, 77, 201, 6), synth.make_tiny(4, 50, 70, 4, 1),
             zero, synth.make_tiny(6, 64, 48, 5, 3), _scene(7, 9, 300, 4)]
    ranks = _check(insts, 25, 0.01)
    assert ranks[3] == 0 and ranks[2] == 1


def test_lowrank_exact_rank_target():
    inst = synth.make_tiny(71, 40, 56, 5, 2)
    t1, t2 = inst.t[0].astype(np.float64), inst.t[1].astype(np.float64)
    inst.t = np.stack([t1, t2, t1 + t2, 0.0 * t1, 2.0 * t1 - t2]).astype(np.float32)
    _check([inst], 25, 1e-6, expect_ranks=[2])


def test_lowrank_sixty_four_channels():
    # the widest target (64 channels, the Gram blocks' largest stride), of
    # rank 3: pixel-level combinations of three channels
    inst = synth.make_tiny(74, 48, 64, 5, 3)
    rng = np.random.default_rng(4)
    mix = rng.standard_normal((64, 3))
    mix[10:20] = 0.0
    inst.t = np.einsum("kc,chw->khw", mix, inst.t.astype(np.float64)).astype(np.float32)
    _check([inst], 25, 1e-6, expect_ranks=[3])


def test_lowrank_full_size_scenes_sampled():
    w = synth.segmentation_scenes_16(n_images=4)
    ranks = _check(w.instances, 25, 0.01)
    print("ranks of four 640x480 scenes (21 channels):", ranks)
    assert all(1 <= r <= 6 for r in ranks)


def test_lowrank_deterministic():
    insts = [_scene(8, 120, 160, 4)]
    a = _gpu_lowrank(insts, 25, 0.01)
    b = _gpu_lowrank(insts, 25, 0.01)
    assert a[0] == b[0] and np.array_equal(a[1][0], b[1][0])


def test_lowrank_argument_errors():
    import torch
    from paper_1511_03296_gb300 import fbs
    inst = _scene(9, 24, 32, 2)
    g = gpu_grid([inst], 2)
    t, c = to_dev(inst.t), to_dev(inst.c)
    x = torch.empty_like(t)
    for eps in (0.0, 1.0, -0.5, float("nan")):
        with pytest.raises(fbs.FbsError):
            fbs.solve_lowrank(g, [t], [c], [128.0], 25, eps, x=[x])
