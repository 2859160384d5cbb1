"""Parity of the domain transform post-filter (Sec. 5; Gastal and Oliveira
2011, recursive formulation) on the GPU with the oracle: rel-L2 <= 1e-5.
The GPU runs each row as a parallel scan of affine maps and each column as
a sequential walk in FP32; the oracle walks every line in FP64."""
import numpy as np
import pytest

from paper_1511_03296_gb300 import synth
from tests.gpu_util import REL_L2_TOL, rel_l2, to_dev

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1511_03296_gb300 import build, fbs
    build.build()
    fbs.load()
    assert torch.cuda.is_available()


def _case(seed, H, W, C):
    rng = np.random.Generator(np.random.PCG64(seed))
    rgb, _, _ = synth.polygon_scene(rng, H, W, 6)
    guide = np.ascontiguousarray(np.moveaxis(rgb.astype(np.float32), -1, 0))
    x = rng.uniform(0.0, 100.0, size=(C, H, W)).astype(np.float32)
    return guide, x


def _check(guide, x, sigma_s, sigma_r, iters, tol=REL_L2_TOL):
    from paper_1511_03296_gb300 import fbs
    xd = to_dev(x)
    fbs.domain_transform(to_dev(guide), xd, sigma_s, sigma_r, iters)
    got = xd.cpu().numpy()
    ref = oracle.domain_transform(guide, x, sigma_s, sigma_r, iters)
    e = rel_l2(got, ref)
    assert e <= tol, e
    return e


@pytest.mark.parametrize("H,W,C", [(64, 48, 1), (97, 131, 3), (1, 300, 2), (300, 1, 2),
                                   (5, 257, 1), (40, 2000, 1)])
@pytest.mark.parametrize("iters", [1, 3])
def test_dt_shapes(H, W, C, iters):
    guide, x = _case(H * 7 + W, H, W, C)
    _check(guide, x, 32.0, 64.0, iters)


@pytest.mark.parametrize("sigma_s,sigma_r", [(4.0, 8.0), (60.0, 300.0), (8.0, 1e-3)])
def test_dt_bandwidths(sigma_s, sigma_r):
    guide, x = _case(11, 120, 160, 2)
    _check(guide, x, sigma_s, sigma_r, 3)


def test_dt_full_hd_after_a_solve():
    # the paper's use: the solver's output post-filtered with the reference as guide
    import torch
    from paper_1511_03296_gb300 import fbs
    inst = synth.plain_1080p().instances[0]
    g = fbs.grid_build([to_dev(inst.yuv)], inst.sigma_xy, inst.sigma_l, inst.sigma_uv)
    fbs.bistochastize(g, 2)
    x = torch.empty_like(to_dev(inst.t))
    fbs.solve(g, [to_dev(inst.t)], [to_dev(inst.c)], inst.lam, 25, x=[x])
    fbs.grid_sync(g)
    xs = x.cpu().numpy()
    e = _check(inst.yuv, xs, 32.0, 64.0, 3)
    print("1080p domain transform rel-L2:", e)


def test_dt_many_channels_and_determinism():
    from paper_1511_03296_gb300 import fbs
    guide, x = _case(12, 60, 80, 21)
    _check(guide, x, 16.0, 32.0, 3)
    a, b = to_dev(x), to_dev(x)
    fbs.domain_transform(to_dev(guide), a, 16.0, 32.0, 3)
    fbs.domain_transform(to_dev(guide), b, 16.0, 32.0, 3)
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())


def test_dt_widest_row():
    # 28000 pixels: the row kernel's largest shared-memory staging (231 KB)
    guide, x = _case(14, 3, 28000, 1)
    _check(guide, x, 32.0, 64.0, 2)


def test_dt_argument_errors():
    from paper_1511_03296_gb300 import fbs
    guide, x = _case(13, 8, 8, 1)
    g, xd = to_dev(guide), to_dev(x)
    for args in ((0.0, 1.0, 3), (1.0, 0.0, 3), (1.0, 1.0, 0), (1.0, 1.0, 17),
                 (float("nan"), 1.0, 3)):
        with pytest.raises(fbs.FbsError):
            fbs.domain_transform(g, xd, *args)
