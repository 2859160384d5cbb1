"""Thousands of PCG iterations with FP32 vectors stay finite and end at the
oracle's converged solution (rel-L2 1e-5 on y and x), for every launch style
and both PCG forms, with Jacobi and the hierarchical preconditioner.  The two
images are the ones of the 64-image batched workload whose y turned NaN after
3000 iterations before the CG scalars froze a stalled channel: once
r^T M^-1 r has fallen to 2^-96 of its first value the FP32 recursive residual
is far below anything y resolves, and past that point it shrank into the
subnormal range, where beta overflowed."""
import functools

import numpy as np
import pytest

from paper_1511_03296_gb300 import synth
from tests.gpu_util import (PCG_FORM, PCG_LAUNCH, PRECOND, REL_L2_TOL, gpu_grid, gpu_solve,
                            oracle_grid, rel_l2)

import oracle

pytestmark = pytest.mark.gpu

LONG = 3000
CONVERGED = 400      # the oracle (FP64) is converged to rounding by then on both images


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1511_03296_gb300 import build, fbs
    build.build()
    fbs.load()
    assert torch.cuda.is_available()


@functools.lru_cache(maxsize=None)
def _batched_image(k):
    return synth.batched_64().instances[k]


@functools.lru_cache(maxsize=None)
def _oracle_converged(k, hier):
    inst = _batched_image(k)
    og = oracle_grid(inst, 2)
    if hier:
        with oracle.hierarchical(og):
            return oracle.solve(og, inst.t, inst.c, inst.lam, CONVERGED)
    return oracle.solve(og, inst.t, inst.c, inst.lam, CONVERGED)


@pytest.mark.parametrize("k,hier,launch,form", [
    (56, False, "auto", "standard"),
    (35, True, "auto", "standard"),
    (35, False, "persistent", "standard"),
    (35, False, "per_phase", "standard"),
    (35, False, "auto", "single"),
])
def test_long_run_stays_finite_and_converged(k, hier, launch, form):
    from paper_1511_03296_gb300 import fbs
    inst = _batched_image(k)
    saved = dict(PCG_LAUNCH), dict(PCG_FORM), dict(PRECOND)
    PCG_LAUNCH["mode"] = {"auto": fbs.PCG_AUTO, "persistent": fbs.PCG_PERSISTENT,
                          "per_phase": fbs.PCG_PER_PHASE}[launch]
    PCG_FORM["form"] = fbs.PCG_FORM_SINGLE if form == "single" else fbs.PCG_FORM_STANDARD
    PRECOND["kind"] = fbs.PRECOND_HIERARCHICAL if hier else fbs.PRECOND_JACOBI
    try:
        g = gpu_grid([inst], 2)
        xs, ys = gpu_solve(g, [inst], LONG)
    finally:
        PCG_LAUNCH.update(saved[0]); PCG_FORM.update(saved[1]); PRECOND.update(saved[2])
    assert np.isfinite(ys[0]).all() and np.isfinite(xs[0]).all()
    oy, ox = _oracle_converged(k, hier)
    ey, ex = rel_l2(ys[0], oy), rel_l2(xs[0].reshape(inst.channels, -1), ox)
    assert ey <= REL_L2_TOL and ex <= REL_L2_TOL, (ey, ex)
