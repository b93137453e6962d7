"""The allocation-free operator entry point, vof_apply_operator_noalloc.

It serves callers that cannot call cudaMalloc (hosts that own all device
memory in their own arena, allocation-free loops), so it takes no context and
keeps its face coefficients in one fixed device array that every call
reuses. These checks call it through the C ABI and compare it with the
context-based vof_apply_operator (bitwise: the same kernels) and with the
FP64 CPU oracle's operator (element-wise), for several calls in a row on
different grids (so the shared array is reused with stale contents from the
previous call), and check that a grid too large for the array, or one that
vof_create would refuse, is refused before any launch.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2104_01636_b300 as vd
from paper_2104_01636_b300 import inputs as I
from gpu_util import ctx, dev, host, rel_max

pytestmark = pytest.mark.gpu


def _entry():
    fn = vd.load().vof_apply_operator_noalloc
    fn.argtypes = [ctypes.POINTER(vd.CGrid), ctypes.POINTER(vd.CPhys), ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def _inputs(g, seed):
    centres = I.place_spheres(g, 2, 8 * g.h, seed, wall_gap=g.h)
    a = I.sphere_alpha(g, centres, 4 * g.h)
    x = np.random.default_rng(seed).normal(size=g.shapes()[0])
    return a, x


def test_noalloc_operator_matches_context_operator_call_after_call():
    import torch
    fn = _entry()
    ph = I.Phys()
    stream = torch.cuda.current_stream().cuda_stream
    for g, seed in [(I.Grid(37, 21, 30), 11), (I.Grid(48, 40, 64), 12), (I.Grid(20, 36, 18), 13)]:
        a, x = _inputs(g, seed)
        with ctx(g, ph) as C:
            y_ref = dev(np.zeros_like(x))
            C.vof_apply_operator(dev(a), dev(x), y_ref)
            torch.cuda.synchronize()
        A, X = dev(a), dev(x)
        for _ in range(2):  # two calls in a row on the same inputs
            Y = dev(np.full_like(x, np.nan))
            st = fn(ctypes.byref(vd.c_grid(g)), ctypes.byref(vd.c_phys(ph)), A.data_ptr(),
                    X.data_ptr(), Y.data_ptr(), stream)
            assert st == 0
            torch.cuda.synchronize()
            assert np.array_equal(host(Y), host(y_ref))
        bx, by, bz = oracle.beta(g, ph, a)
        assert rel_max(host(Y), oracle.apply_A(g, bx, by, bz, x)) <= 1e-12


def test_noalloc_operator_rejects_grids_beyond_its_scratch():
    import torch
    fn = _entry()
    g = I.Grid(128, 128, 128)  # about 6.3M faces > VOF_NOALLOC_MAX_FACES
    assert (g.nx + 1) * g.ny * g.nz * 3 > (3 << 20)
    Y = torch.zeros(4, device="cuda", dtype=torch.float64)
    st = fn(ctypes.byref(vd.c_grid(g)), ctypes.byref(vd.c_phys(I.Phys())), Y.data_ptr(),
            Y.data_ptr(), Y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert vd.STATUS[st] == "VOF_ERR_ADMISSION"
    torch.cuda.synchronize()
    assert torch.all(Y == 0).item()


@pytest.mark.parametrize("bad", [dict(nz=3), dict(nz=31), dict(h=float("inf")), dict(h=0.0)])
def test_noalloc_operator_checks_grids_as_vof_create_does(bad):
    import torch
    fn = _entry()
    kw = dict(nx=16, ny=12, nz=16, h=2.5e-4)
    kw.update(bad)
    g = I.Grid(**kw)
    Y = torch.zeros(4, device="cuda", dtype=torch.float64)
    st = fn(ctypes.byref(vd.c_grid(g)), ctypes.byref(vd.c_phys(I.Phys())), Y.data_ptr(),
            Y.data_ptr(), Y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert vd.STATUS[st] == "VOF_ERR_ARG"
    torch.cuda.synchronize()
    assert torch.all(Y == 0).item()
