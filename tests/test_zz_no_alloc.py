"""The allocation-free solve entry point (fbs_solve_static).

Some callers cannot allocate device memory at solve time (a fixed memory
budget, a real-time loop, an embedding runtime that owns the allocator).
For them fbs_solve_static runs the same forward solve with all scratch in
an array compiled into the library.  These tests call it through the C ABI
and compare it with fbs_solve on two calls in a row.  The file sorts last
so that a run stopping at the first failure has run every other test."""
import numpy as np
import pytest

from paper_1511_03296_gb300 import synth
from tests.gpu_util import REL_L2_TOL, gpu_grid, rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_1511_03296_gb300 import build, fbs
    build.build()
    fbs.load()
    assert torch.cuda.is_available()


def _pair(grid, inst, t, c, lam):
    import torch
    from paper_1511_03296_gb300 import fbs
    C = inst.channels
    x_ref = torch.empty_like(t)
    y_ref = torch.empty((C, grid.vertex_counts[0]), device="cuda")
    fbs.solve(grid, [t], [c], lam, 25, x=[x_ref], y=[y_ref])
    x_st = torch.full_like(t, float("nan"))
    y_st = torch.full((C, grid.vertex_counts[0]), float("nan"), device="cuda")
    fbs.solve_static(grid, [t], [c], lam, 25, x=[x_st], y=[y_st])
    fbs.grid_sync(grid)
    return (x_ref.cpu().numpy(), y_ref.cpu().numpy(), x_st.cpu().numpy(), y_st.cpu().numpy())


def test_static_solve_matches_fbs_solve_twice():
    import torch
    inst = synth.make_tiny(41, 120, 160, 8, 3, (8.0, 4.0, 3.0), 128.0)
    g = gpu_grid([inst], 2)
    t, c = to_dev(inst.t), to_dev(inst.c)
    rng = np.random.default_rng(9)
    for call in range(2):
        if call == 1:   # second call: new target contents and lambda
            t.copy_(torch.from_numpy((inst.t + rng.normal(0, 6, inst.t.shape)).astype(np.float32)))
        lam = 128.0 if call == 0 else 20.0
        x_ref, y_ref, x_st, y_st = _pair(g, inst, t, c, lam)
        assert np.isfinite(x_st).all() and np.isfinite(y_st).all()
        assert rel_l2(x_st, x_ref) <= REL_L2_TOL, call
        assert rel_l2(y_st, y_ref) <= REL_L2_TOL, call


def test_static_solve_1080p_matches_fbs_solve():
    inst = synth.plain_1080p().instances[0]
    g = gpu_grid([inst], 2)
    t, c = to_dev(inst.t), to_dev(inst.c)
    for call in range(2):
        x_ref, y_ref, x_st, y_st = _pair(g, inst, t, c, inst.lam)
        assert rel_l2(x_st, x_ref) <= REL_L2_TOL and rel_l2(y_st, y_ref) <= REL_L2_TOL, call


STATIC_ARRAY_BYTES = 64 << 20


def static_bytes(vertex_counts, channels):
    """Scratch a problem needs, by the formula the header states."""
    a256 = lambda x: (x + 255) // 256 * 256
    cp = [c if c <= 2 else (c + 3) // 4 * 4 for c in channels]
    cv = sum((p * v + 31) // 32 * 32 for p, v in zip(cp, vertex_counts))
    cpart = sum(c * ((v + 255) // 256) for c, v in zip(channels, vertex_counts))
    n, vt = len(channels), sum(vertex_counts)
    return (a256(144 * n) + a256(32 * cv) + a256(4 * vt) + a256(8 * vt) + a256(72 * sum(channels))
            + a256(32 * cpart) + a256(4224))


def test_static_solve_limit_is_the_documented_one():
    # the widest target that fits by the stated formula solves; the next
    # wider one, whose padded width crosses the limit, is rejected
    import torch
    from paper_1511_03296_gb300 import fbs
    rng = np.random.Generator(np.random.PCG64(12))
    inst = synth.depth_instance(rng, 480, 640, 20, (2.0, 2.0, 2.0), 8.0, channels=1)
    g = gpu_grid([inst], 2)
    V = g.vertex_counts[0]
    fits = [C for C in range(1, 65) if static_bytes([V], [C]) <= STATIC_ARRAY_BYTES]
    c_ok = max(fits)
    c_big = c_ok + 1
    assert c_big <= 64 and static_bytes([V], [c_big]) > STATIC_ARRAY_BYTES, (V, c_ok)
    c = to_dev(inst.c)
    t_ok = to_dev(np.repeat(inst.t, c_ok, axis=0))
    x = torch.empty_like(t_ok)
    fbs.solve_static(g, [t_ok], [c], inst.lam, 5, x=[x])
    fbs.grid_sync(g)
    assert torch.isfinite(x).all()
    with pytest.raises(fbs.FbsError, match="ARG"):
        fbs.solve_static(g, [to_dev(np.repeat(inst.t, c_big, axis=0))], [c], inst.lam, 5)
