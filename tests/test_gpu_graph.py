"""The V-cycle replayed from a captured CUDA graph (contexts on a capturable
stream) gives bitwise the results and launch counts of direct launches
(contexts on the legacy default stream, which cannot be captured)."""
import numpy as np
import pytest
import torch

import paper_2104_01636_b300 as vd
from paper_2104_01636_b300 import inputs as I
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _run(case, solver, stream, nsteps):
    st = [dev(a) for a in case.state()]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        with vd.VofContext(case.grid, case.phys, solver, stream=stream) as C:
            reps = [C.step(*st, case.dt, s) for s in range(nsteps)]
            n = C.launch_count()
    torch.cuda.synchronize()
    return [host(t) for t in st], reps, n


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_matches_direct_launches(prec):
    case = I.rising_swarm(64, 48, 64, nbub=5, d_cells=10, seed=91, steps=3)
    sv = vd.c_solver(prec, rtol=1e-9, max_iter=300)
    direct, rd, nd = _run(case, sv, torch.cuda.default_stream(), 3)
    graph, rg, ng = _run(case, sv, torch.cuda.Stream(), 3)
    for a, b in zip(direct, graph):
        assert np.array_equal(a, b)
    assert [r["iters"] for r in rd] == [r["iters"] for r in rg]
    assert nd == ng
