"""The request server: a request's result does not depend on what else was
running (bitwise equal to the same request run alone through a context),
admission is FIFO within the memory budget, and requests that can never fit
are rejected at submission."""
import numpy as np
import pytest

import paper_2104_01636_b300 as vd
from paper_2104_01636_b300 import inputs as I
from gpu_util import ctx, dev, host

pytestmark = pytest.mark.gpu


def _swarm(nx, ny, nz, nbub, seed):
    return I.rising_swarm(nx, ny, nz, nbub=nbub, d_cells=8, seed=seed, steps=3)


def _state_copy(case):
    return [np.array(a, dtype=np.float64, order="C", copy=True) for a in case.state()]


def _alone_steps(case, solver_kw, n):
    """The same request through a context on device tensors."""
    st = [dev(a) for a in case.state()]
    with ctx(case, **solver_kw) as C:
        for s in range(n):
            C.step(*st, case.dt, s)
    return [host(t) for t in st]


def _alone_solve(g, ph, solver_kw, alpha, b):
    p = dev(np.zeros_like(b))
    with ctx(g, ph, **solver_kw) as C:
        C.pressure_solve(dev(alpha), dev(b), p)
    return host(p)


def _solve_case(dims, seed):
    g = I.Grid(*dims)
    c = I.place_spheres(g, 2, 8 * g.h, seed, wall_gap=g.h)
    a = I.sphere_alpha(g, c, 4 * g.h)
    b = np.random.default_rng(seed).normal(size=g.shapes()[0])
    return g, I.Phys(), a, b - b.mean()


@pytest.mark.parametrize("prec", [0, 1])
def test_mix_equals_alone(prec):
    kw = dict(precision=prec, rtol=1e-9, max_iter=300)
    steps = [(_swarm(32, 32, 48, 3, 11), 3), (_swarm(24, 40, 64, 4, 12), 2),
             (_swarm(40, 24, 32, 2, 13), 3)]
    solves = [_solve_case((37, 21, 30), 5), _solve_case((48, 40, 64), 6)]
    budget = 4 << 30
    with vd.VofServer(budget, max_concurrent=4) as S:
        ids, outs = [], []
        for case, n in steps:
            st = _state_copy(case)
            ids.append(S.submit_step(case.grid, case.phys, vd.c_solver(**kw), st, n, case.dt))
            outs.append(st)
        for g, ph, a, b in solves:
            p = np.zeros_like(b)
            ids.append(S.submit_solve(g, ph, vd.c_solver(**kw), a.copy(), b.copy(), p))
            outs.append(p)
        res = [S.wait(i) for i in ids]
    for r in res:
        assert r["status"] == "VOF_OK", r
        assert r["state"] == 2
        assert r["t_submit"] <= r["t_admit"] <= r["t_finish"]
    for (case, n), out in zip(steps, outs):
        ref = _alone_steps(case, kw, n)
        for got, want in zip(out, ref):
            assert np.array_equal(got, want)
    for (g, ph, a, b), out in zip(solves, outs[len(steps):]):
        assert np.array_equal(out, _alone_solve(g, ph, kw, a, b))


def test_fifo_admission_within_budget():
    """A budget that holds one request at a time serialises them in arrival
    order; every request still finishes."""
    kw = dict(precision=1, rtol=1e-8, max_iter=300)
    cases = [_solve_case((32, 32, 32), s) for s in range(4)]
    need = vd.workspace_bytes(cases[0][0], vd.c_solver(**kw)) + 3 * 8 * 32 ** 3
    with vd.VofServer(int(need * 1.5), max_concurrent=4) as S:
        ids = [S.submit_solve(g, ph, vd.c_solver(**kw), a, b, np.zeros_like(b))
               for g, ph, a, b in cases]
        res = [S.wait(i) for i in ids]
    assert all(r["status"] == "VOF_OK" for r in res)
    for r0, r1 in zip(res, res[1:]):
        assert r1["t_admit"] >= r0["t_finish"] - 1e-6  # no overlap: one fits at a time
        assert r1["t_admit"] >= r0["t_admit"]


def test_oversize_request_rejected():
    g, ph, a, b = _solve_case((32, 32, 32), 1)
    with vd.VofServer(1 << 20, max_concurrent=2) as S:
        with pytest.raises(vd.VofError) as e:
            S.submit_solve(g, ph, vd.c_solver(), a, b, np.zeros_like(b))
        assert e.value.name == "VOF_ERR_ADMISSION"


def test_failed_request_reports_status():
    """A step whose CFL number exceeds one finishes with VOF_ERR_CFL; the
    server keeps serving the next request."""
    case = _swarm(32, 32, 48, 3, 21)
    kw = dict(precision=1, rtol=1e-8, max_iter=300)
    with vd.VofServer(2 << 30, max_concurrent=2) as S:
        bad = S.submit_step(case.grid, case.phys, vd.c_solver(**kw), _state_copy(case), 1,
                            case.dt * 1e4)
        good = S.submit_step(case.grid, case.phys, vd.c_solver(**kw), _state_copy(case), 1,
                             case.dt)
        rb, rg = S.wait(bad), S.wait(good)
    assert rb["status"] == "VOF_ERR_CFL"
    assert rg["status"] == "VOF_OK"
