"""Error behaviour of the C ABI on a GPU: host-detected conditions, and a
bounded device wait that runs out (no kernel is driven into a fault or a
hang)."""
import ctypes

import numpy as np
import pytest

import paper_2104_01636_b300 as vd
from paper_2104_01636_b300 import inputs as I
from gpu_util import ctx, dev

pytestmark = pytest.mark.gpu


def test_cfl_violation_is_rejected_before_launch():
    g = I.Grid(16, 16, 16)
    cs, us, vs, ws = g.shapes()
    a = dev(np.ones(cs))
    with ctx(g, I.Phys()) as C:
        with pytest.raises(vd.VofError) as e:
            C.vof_advect(a, dev(np.zeros(us)), dev(np.zeros(vs)), dev(np.full(ws, 1.0)),
                         2.0 * g.h, 0)
        assert e.value.name == "VOF_ERR_CFL"
        assert "Courant" in str(e.value)


def test_null_pointer_and_bad_args():
    g = I.Grid(16, 16, 16)
    lib = vd.load()
    with ctx(g, I.Phys()) as C:
        assert lib.ssf_force(C._ctx, None, None, None, None, None) == 1
        assert b"NULL" in lib.vof_last_error(C._ctx)
        cs, us, vs, ws = g.shapes()
        with pytest.raises(vd.VofError) as e:
            C.step(dev(np.ones(cs)), dev(np.zeros(cs)), dev(np.zeros(cs)), dev(np.zeros(cs)),
                   dev(np.zeros(us)), dev(np.zeros(vs)), dev(np.zeros(ws)), dev(np.zeros(cs)),
                   -1.0, 0)
        assert e.value.name == "VOF_ERR_ARG"


def test_admission_budget():
    g = I.Grid(64, 64, 64)
    with pytest.raises(vd.VofError) as e:
        vd.VofContext(g, I.Phys(), budget_bytes=1 << 20)
    assert e.value.name == "VOF_ERR_ADMISSION"


def test_not_converged_keeps_last_iterate():
    g = I.Grid(32, 32, 32)
    a = I.sphere_alpha(g, np.array([[16 * g.h] * 3]), 6 * g.h)
    b = np.random.default_rng(3).normal(size=g.shapes()[0])
    with ctx(g, I.Phys(), rtol=1e-14, max_iter=1) as C:
        p = dev(np.zeros_like(b))
        with pytest.raises(vd.VofError) as e:
            C.pressure_solve(dev(a), dev(b), p)
        assert e.value.name == "VOF_ERR_NOT_CONVERGED"
        assert e.value.report["iters"] >= 1
        assert np.isfinite(p.cpu().numpy()).all() and p.abs().max().item() > 0


def test_periodic_walls_unsupported_in_solve():
    g = I.Grid(16, 16, 16, per_x=1)
    cs = g.shapes()[0]
    with ctx(g, I.Phys()) as C:
        with pytest.raises(vd.VofError) as e:
            C.pressure_solve(dev(np.ones(cs)), dev(np.zeros(cs)), dev(np.zeros(cs)))
        assert e.value.name == "VOF_ERR_UNSUPPORTED"


def test_bounded_wait_times_out_and_context_stays_usable():
    """A bounded device wait that runs out (a barrier nothing completes) sets
    the device error flag and becomes VOF_ERR_TIMEOUT, without a fault or a
    hang; the same context then steps normally."""
    case = I.rising_swarm(32, 32, 32, nbub=1, d_cells=8, seed=101, steps=1)
    with vd.VofContext(case.grid, case.phys, vd.c_solver(vd.PREC_MIXED_FP32, rtol=1e-9)) as C:
        with pytest.raises(vd.VofError) as ei:
            C.diag_wait_timeout()
        assert ei.value.name == "VOF_ERR_TIMEOUT"
        T = [dev(a) for a in case.state()]
        rep = C.step(*T, case.dt, 0)
        assert rep["res"] <= 1e-9
