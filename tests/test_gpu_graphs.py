"""CUDA graphs around the solver: the library's own replay of captured
segments and a solve captured by the caller (torch.cuda.graph) keep
parity with the oracle when the inputs change between replays, with the
Jacobi and with the hierarchical preconditioner (whose pyramid must exist
before the caller's capture: a first solve outside it builds the pyramid
and sizes the workspace)."""
import contextlib

import numpy as np
import pytest

from paper_1511_03296_gb300 import synth
from tests.gpu_util import PRECOND, REL_L2_TOL, gpu_grid, oracle_grid, rel_l2, to_dev

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1511_03296_gb300 import build, fbs
    build.build()
    fbs.load()
    assert torch.cuda.is_available()


def _oracle_x(og, t, c, lam, hier):
    ctx = oracle.hierarchical(og) if hier else contextlib.nullcontext()
    with ctx:
        return oracle.solve(og, t, c, lam, 25)[1]


@pytest.fixture(params=[False, True], ids=["jacobi", "hierarchical"])
def hier(request):
    from paper_1511_03296_gb300 import fbs
    PRECOND["kind"] = fbs.PRECOND_HIERARCHICAL if request.param else fbs.PRECOND_JACOBI
    yield request.param
    PRECOND["kind"] = fbs.PRECOND_JACOBI


def test_library_graph_replay_with_new_inputs(hier):
    import torch
    from paper_1511_03296_gb300 import fbs
    inst = synth.make_tiny(41, 80, 100, 6, 2)
    g = gpu_grid([inst], 2)
    t, c = to_dev(inst.t), to_dev(inst.c)
    x = torch.empty_like(t)
    og = oracle_grid(inst, 2)
    rng = np.random.default_rng(5)
    for k in range(4):
        tk = (inst.t + rng.normal(0, 5, inst.t.shape)).astype(np.float32)
        t.copy_(torch.from_numpy(tk))
        fbs.solve(g, [t], [c], inst.lam, 25, x=[x])
        fbs.grid_sync(g)
        assert rel_l2(x.cpu().numpy().reshape(2, -1), _oracle_x(og, tk, inst.c, inst.lam, hier)) \
            <= REL_L2_TOL, k


def test_solve_captured_by_the_caller(hier):
    import torch
    from paper_1511_03296_gb300 import fbs
    inst = synth.make_tiny(42, 72, 96, 6, 3)
    g = gpu_grid([inst], 2)
    t, c = to_dev(inst.t), to_dev(inst.c)
    x = torch.empty_like(t)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        fbs.solve(g, [t], [c], inst.lam, 25, x=[x])     # sizes the workspace, builds the pyramid
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        fbs.solve(g, [t], [c], inst.lam, 25, x=[x])
    og = oracle_grid(inst, 2)
    rng = np.random.default_rng(6)
    for k in range(3):
        tk = (inst.t + rng.normal(0, 5, inst.t.shape)).astype(np.float32)
        t.copy_(torch.from_numpy(tk))
        x.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert rel_l2(x.cpu().numpy().reshape(3, -1), _oracle_x(og, tk, inst.c, inst.lam, hier)) \
            <= REL_L2_TOL, k
