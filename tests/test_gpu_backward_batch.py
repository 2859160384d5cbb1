"""Backward pass (Sec. 3) on batches of images, through the C ABI and
through the autograd Functions, against the FP64 oracle.

The forward solution y-hat enters the gradient of the confidence through
t - S^T y-hat, which cancels where the solve reproduces the target, so an
FP32 rounding of y-hat is amplified there.  Each comparison below therefore
hands the oracle the same y-hat (and the same dL/dx) that the GPU used, so
that it checks the backward operation alone at the stated bar; the forward
x is checked on its own at the same bar."""
import numpy as np
import pytest

import oracle
from paper_1511_03296_gb300 import synth
from tests import dense
from tests.gpu_util import REL_L2_TOL, gpu_grid, oracle_grid, rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_1511_03296_gb300 import build, fbs
    build.build()
    fbs.load()
    assert torch.cuda.is_available()


def _mixed_batch():
    """Uneven sizes and channel counts: segmentation crops of 21 channels,
    a one-channel depth image and a 5-channel target."""
    rng = np.random.Generator(np.random.PCG64(40))
    seg = synth.segmentation_instance(rng, 96, 128, 21, (8.0, 4.0, 3.0), 128.0, blob_sigma=8.0)
    return [
        synth.crop(seg, 8, 16, 24, 32),
        synth.make_tiny(41, 75, 61, 5, 1, (8.0, 4.0, 3.0), 32.0),
        synth.crop(seg, 0, 0, 96, 128),
        synth.make_tiny(42, 33, 90, 4, 5, (16.0, 8.0, 8.0), 128.0),
    ]


def _gpu_forward(g, insts, iters):
    import torch
    from paper_1511_03296_gb300 import fbs
    t = [to_dev(i.t) for i in insts]
    c = [to_dev(i.c) for i in insts]
    x = [torch.empty_like(tt) for tt in t]
    y = [torch.empty((i.channels, g.vertex_counts[k]), device="cuda")
         for k, i in enumerate(insts)]
    fbs.solve(g, t, c, [i.lam for i in insts], iters, x=x, y=y)
    return t, c, x, y


def test_solve_backward_mixed_batch():
    # one fbs_solve_backward call for four images of different sizes and
    # channel counts; every image's dL/dt and dL/dc against the oracle
    import torch
    from paper_1511_03296_gb300 import fbs
    insts = _mixed_batch()
    g = gpu_grid(insts, 2)
    rng = np.random.default_rng(9)
    yh, dx, ogs = [], [], []
    for inst in insts:
        og = oracle_grid(inst, 2)
        oy, _ = oracle.solve(og, inst.t, inst.c, inst.lam, 25)
        ogs.append(og)
        yh.append(oy.astype(np.float32))
        dx.append(rng.normal(size=inst.t.shape).astype(np.float32))
    t = [to_dev(i.t) for i in insts]
    c = [to_dev(i.c) for i in insts]
    dt = [torch.empty_like(tt) for tt in t]
    dc = [torch.empty_like(cc) for cc in c]
    fbs.solve_backward(g, t, c, [i.lam for i in insts], [to_dev(v) for v in yh],
                       [to_dev(v) for v in dx], dt, dc, 25)
    fbs.grid_sync(g)
    for k, inst in enumerate(insts):
        C = inst.channels
        odt, odc = oracle.backward(ogs[k], inst.t, inst.c, inst.lam, 25,
                                   yh[k].astype(np.float64), dx[k].reshape(C, -1))
        e_t = rel_l2(dt[k].cpu().numpy().reshape(C, -1), odt)
        e_c = rel_l2(dc[k].cpu().numpy().reshape(-1), odc)
        assert e_t <= REL_L2_TOL and e_c <= REL_L2_TOL, (k, e_t, e_c)


def test_batched_backward_equals_images_alone():
    # batching changes no result: each image's gradients from the batched
    # call are bitwise those of a call on its own grid
    import torch
    from paper_1511_03296_gb300 import fbs
    insts = _mixed_batch()
    g = gpu_grid(insts, 2)
    t, c, _, y = _gpu_forward(g, insts, 25)
    rng = np.random.default_rng(10)
    dx = [to_dev(rng.normal(size=i.t.shape).astype(np.float32)) for i in insts]
    dt = [torch.empty_like(tt) for tt in t]
    dc = [torch.empty_like(cc) for cc in c]
    fbs.solve_backward(g, t, c, [i.lam for i in insts], y, dx, dt, dc, 25)
    fbs.grid_sync(g)
    for k, inst in enumerate(insts):
        g1 = gpu_grid([inst], 2)
        dt1, dc1 = torch.empty_like(t[k]), torch.empty_like(c[k])
        fbs.solve_backward(g1, [t[k]], [c[k]], inst.lam, [y[k]], [dx[k]], [dt1], [dc1], 25)
        fbs.grid_sync(g1)
        assert torch.equal(dt1, dt[k]) and torch.equal(dc1, dc[k]), k


def _check_autograd_batch(insts, iters, sample=None):
    """Forward and backward through BilateralSolveBatch with an MSE loss; x
    per image against the oracle, then the gradients against the oracle's
    backward given the GPU's own y-hat and dL/dx."""
    import torch
    from paper_1511_03296_gb300 import fbs
    g = gpu_grid(insts, 2)
    t = [to_dev(i.t).requires_grad_(True) for i in insts]
    c = [to_dev(i.c).requires_grad_(True) for i in insts]
    labels = [to_dev(i.label.astype(np.float32)) for i in insts]
    xs = fbs.bilateral_solve(t, c, g, [i.lam for i in insts], iters)
    n_total = sum(x.numel() for x in xs)
    loss = sum(((x - lab) ** 2).sum() for x, lab in zip(xs, labels)) / n_total
    loss.backward()
    # the saved y-hat: a second forward on the same inputs is bitwise equal
    _, _, x2, yh = _gpu_forward(g, insts, iters)
    fbs.grid_sync(g)
    errs = []
    for k in (range(len(insts)) if sample is None else sample):
        inst = insts[k]
        C = inst.channels
        assert torch.equal(x2[k], xs[k].detach())
        assert torch.isfinite(t[k].grad).all() and torch.isfinite(c[k].grad).all()
        og = oracle_grid(inst, 2)
        _, ox = oracle.solve(og, inst.t, inst.c, inst.lam, iters)
        e_x = rel_l2(xs[k].detach().cpu().numpy().reshape(C, -1), ox)
        dx = (2.0 * (xs[k].detach() - labels[k]) / n_total).cpu().numpy().reshape(C, -1)
        odt, odc = oracle.backward(og, inst.t, inst.c, inst.lam, iters,
                                   yh[k].cpu().numpy().astype(np.float64),
                                   dx.astype(np.float64))
        e_t = rel_l2(t[k].grad.cpu().numpy().reshape(C, -1), odt)
        e_c = rel_l2(c[k].grad.cpu().numpy().reshape(-1), odc)
        errs.append((e_x, e_t, e_c))
        assert e_x <= REL_L2_TOL and e_t <= REL_L2_TOL and e_c <= REL_L2_TOL, (k, e_x, e_t, e_c)
    return errs


def _with_labels(insts, seed):
    rng = np.random.default_rng(seed)
    for inst in insts:
        if getattr(inst, "label", None) is None:
            inst.label = rng.random(inst.t.shape).astype(np.float32)
    return insts


def test_autograd_batch_mixed():
    _check_autograd_batch(_with_labels(_mixed_batch(), 11), 25)


def test_autograd_batch_segmentation_16x640x480():
    # the segmentation workload in full: 16 images of 640 x 480 with 21
    # channels through BilateralSolveBatch; three images compared with the
    # oracle (each takes seconds on the host), all sixteen checked finite
    insts = synth.segmentation_16().instances
    errs = _check_autograd_batch(insts, 25, sample=(0, 7, 15))
    print("16 x 640x480 x 21 autograd rel-L2 (x, dt, dc) on images 0, 7, 15:", errs)


def test_autograd_gradient_matches_finite_differences():
    # the 32 x 24 crop with 21 channels: the Function's gradient, with solves
    # run to convergence, against FP64 central differences of the loss built
    # from a dense direct solve (independent of both implementations)
    import torch
    from paper_1511_03296_gb300 import fbs
    rng = np.random.Generator(np.random.PCG64(5))
    seg = synth.segmentation_instance(rng, 48, 64, 21, (8.0, 4.0, 3.0), 128.0, blob_sigma=6.0)
    inst = synth.crop(seg, 8, 16, 24, 32)
    C = inst.channels
    g = gpu_grid([inst], 2)
    t = to_dev(inst.t).requires_grad_(True)
    c = to_dev(inst.c).requires_grad_(True)
    label = inst.label.reshape(C, -1).astype(np.float64)
    x = fbs.bilateral_solve(t, c, g, inst.lam, 400)
    loss = ((x - to_dev(inst.label.astype(np.float32))) ** 2).mean()
    loss.backward()
    gt = t.grad.cpu().numpy().reshape(C, -1).astype(np.float64)
    gc = c.grad.cpu().numpy().reshape(-1).astype(np.float64)

    og = oracle_grid(inst, 2)
    S = dense.dense_S(og.vid, og.V)
    t64 = inst.t.reshape(C, -1).astype(np.float64)
    c64 = inst.c.reshape(-1).astype(np.float64)

    def dense_loss(tt, cc):
        sc = S @ cc
        b = (S @ (cc[None] * tt).T).T
        a, _ = oracle.diag(og.m, og.nbr, og.n, sc, inst.lam)
        A = np.stack([oracle.apply_A(og.nbr, og.n, a, inst.lam, e) for e in np.eye(og.V)], 1)
        y = np.linalg.solve(A, b.T).T
        return np.mean((y[:, og.vid] - label) ** 2)

    pick = np.random.default_rng(3)
    fd_t, gpu_t, fd_c, gpu_c = [], [], [], []
    for _ in range(8):
        ch, i = int(pick.integers(C)), int(pick.integers(og.N))
        tp, tm = t64.copy(), t64.copy()
        tp[ch, i] += 1e-4
        tm[ch, i] -= 1e-4
        fd_t.append((dense_loss(tp, c64) - dense_loss(tm, c64)) / 2e-4)
        gpu_t.append(gt[ch, i])
    for _ in range(8):
        i = int(pick.integers(og.N))
        cp, cm = c64.copy(), c64.copy()
        cp[i] += 1e-5
        cm[i] -= 1e-5
        fd_c.append((dense_loss(t64, cp) - dense_loss(t64, cm)) / 2e-5)
        gpu_c.append(gc[i])
    e_t, e_c = rel_l2(gpu_t, fd_t), rel_l2(gpu_c, fd_c)
    print("autograd vs FP64 central differences rel-L2 (dt, dc):", e_t, e_c)
    assert e_t <= REL_L2_TOL and e_c <= REL_L2_TOL, (e_t, e_c)
