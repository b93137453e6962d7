"""Python binding of libvofduct.so, the sm_103a projection-step library.

Argument marshalling only: every step of the time step runs in the CUDA
kernels behind the C ABI of include/vof.h. Fields are torch float64 CUDA
tensors (contiguous) shaped like the arrays of `paper_2104_01636_b300.inputs`:
cells (nz, ny, nx), x-faces (nz, ny, nx+1), y-faces (nz, ny+1, nx), z-faces
(nz, ny, nx). Velocities come as cell-centred (uc, vc, wc) and face (u, v, w)
fields. Calls run on the context's stream (the current torch stream at
creation unless one is given).

There is no CPU fallback: a missing library or device raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libvofduct.so")

STATUS = {0: "VOF_OK", 1: "VOF_ERR_ARG", 2: "VOF_ERR_OOM", 3: "VOF_ERR_CUDA",
          4: "VOF_ERR_NOT_CONVERGED", 5: "VOF_ERR_NONFINITE", 6: "VOF_ERR_CFL",
          7: "VOF_ERR_TIMEOUT", 8: "VOF_ERR_ADMISSION", 9: "VOF_ERR_UNSUPPORTED"}
PREC_FP64, PREC_MIXED_FP32 = 0, 1


class VofError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str = "", report=None):
        self.status = status
        self.name = STATUS.get(status, str(status))
        self.report = report
        super().__init__(f"{where}: {self.name}{': ' + msg if msg else ''}")


class CGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_double), ("periodic_x", ctypes.c_int), ("periodic_y", ctypes.c_int)]


class CPhys(ctypes.Structure):
    _fields_ = [("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double),
                ("mu_l", ctypes.c_double), ("mu_g", ctypes.c_double),
                ("sigma", ctypes.c_double), ("g_z", ctypes.c_double),
                ("rho0", ctypes.c_double), ("dpdz", ctypes.c_double),
                ("conv_scheme", ctypes.c_int), ("kappa_mode", ctypes.c_int),
                ("kappa_exact", ctypes.c_double)]


class CSolver(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("rtol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int),
                ("mg_omega", ctypes.c_double), ("coarse_iters", ctypes.c_int),
                ("coarse_tol", ctypes.c_double), ("mg_interp", ctypes.c_int),
                ("mg_coarsen", ctypes.c_int), ("mg_cycle", ctypes.c_int),
                ("mg_w_depth", ctypes.c_int), ("graph", ctypes.c_int),
                ("nu_fine", ctypes.c_int), ("ssf_solves", ctypes.c_int),
                ("mg_tail", ctypes.c_int), ("mg_tune", ctypes.c_int)]


class CReport(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("refinements", ctypes.c_int),
                ("res0", ctypes.c_double), ("res", ctypes.c_double),
                ("b_mean", ctypes.c_double), ("vol_before", ctypes.c_double),
                ("vol_after", ctypes.c_double), ("vol_clipped", ctypes.c_double),
                ("max_div", ctypes.c_double), ("max_u", ctypes.c_double),
                ("hf_fallbacks", ctypes.c_longlong), ("ms", ctypes.c_float * 8)]

    def as_dict(self) -> dict:
        d = {n: getattr(self, n) for n, _ in self._fields_ if n != "ms"}
        d["ms"] = list(self.ms)
        return d


REQ_STEP, REQ_SOLVE = 0, 1
_DP = ctypes.POINTER(ctypes.c_double)


class CRequest(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("grid", CGrid), ("phys", CPhys), ("solver", CSolver),
                ("n_steps", ctypes.c_int), ("dt", ctypes.c_double), ("step0", ctypes.c_longlong),
                ("alpha", _DP), ("uc", _DP), ("vc", _DP), ("wc", _DP), ("u", _DP), ("v", _DP),
                ("w", _DP), ("p", _DP), ("b", _DP)]


class CResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("state", ctypes.c_int), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_finish", ctypes.c_double), ("report", CReport)]

    def as_dict(self) -> dict:
        return {"status": STATUS.get(self.status, self.status), "state": self.state,
                "t_submit": self.t_submit, "t_admit": self.t_admit, "t_finish": self.t_finish,
                "report": self.report.as_dict()}


_lib = None
_VP = ctypes.c_void_p
_D = ctypes.c_double


def load() -> ctypes.CDLL:
    """Load libvofduct.so (built in-tree); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2104_01636_b300.build` (nvcc, sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    sig = {
        "vof_workspace_bytes": [P(CGrid), P(CSolver), P(ctypes.c_size_t)],
        "vof_create": [P(CGrid), P(CPhys), P(CSolver), ctypes.c_size_t, _VP, P(_VP)],
        "vof_destroy": [_VP],
        "vof_advect": [_VP, _VP, _VP, _VP, _VP, _D, ctypes.c_longlong, _VP, _VP, _VP,
                       P(CReport)],
        "ssf_force": [_VP, _VP, _VP, _VP, _VP, _VP],
        "pressure_solve": [_VP, _VP, _VP, _VP, P(CReport)],
        "vof_apply_operator": [_VP, _VP, _VP, _VP],
        "vof_predict": [_VP] * 12 + [_D],
        "project": [_VP] * 12 + [_D, P(CReport)],
        "step": [_VP] * 9 + [_D, ctypes.c_longlong, P(CReport)],
        "vof_step_host": [_VP] * 9 + [_D, ctypes.c_longlong, P(CReport)],
        "vof_host_join": [_VP],
        "vof_diag_wait_timeout": [_VP],
        "vof_set_timing": [_VP, ctypes.c_int],
        "vof_launch_count": [_VP, ctypes.POINTER(ctypes.c_longlong)],
        "vof_mg_shape": [_VP, ctypes.c_int, P(ctypes.c_int)],
        "vof_mg_set_shape": [_VP, ctypes.c_int, P(ctypes.c_int)],
        "vof_kernel_times": [_VP, P(ctypes.c_char_p), P(_D), P(ctypes.c_longlong), ctypes.c_int,
                             P(ctypes.c_int)],
        "vof_server_create": [ctypes.c_size_t, ctypes.c_int, P(_VP)],
        "vof_submit": [_VP, P(CRequest), P(ctypes.c_ulonglong)],
        "vof_poll": [_VP, ctypes.c_ulonglong, P(CResult)],
        "vof_wait": [_VP, ctypes.c_ulonglong, P(CResult)],
        "vof_server_destroy": [_VP],
        "vof_ensemble_create": [P(CGrid), P(CPhys), ctypes.c_int, P(CSolver), ctypes.c_int,
                                ctypes.c_int, P(_VP)],
        "vof_ensemble_step": [_VP, P(_VP), P(_D), ctypes.c_longlong, P(ctypes.c_int), P(CReport)],
        "vof_ensemble_destroy": [_VP],
        "vof_ensemble_create_mode": [P(CGrid), P(CPhys), ctypes.c_int, P(CSolver), ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, P(_VP)],
        "vof_ensemble_batched": [_VP, P(ctypes.c_int)],
        "vof_ensemble_launch_count": [_VP, P(ctypes.c_longlong)],
        "vof_ensemble_phase_ms": [_VP, P(_D)],
        "vof_ensemble_graph_steps": [_VP, P(ctypes.c_longlong)],
        "vof_ensemble_mg_shape": [_VP, ctypes.c_int, P(ctypes.c_int)],
        "vof_stats_create": [P(CGrid), P(_VP)],
        "vof_stats_accumulate": [_VP, _VP, _VP, _VP, _VP, _VP],
        "vof_stats_read": [_VP, P(_D), P(ctypes.c_longlong)],
        "vof_stats_reset": [_VP],
        "vof_stats_destroy": [_VP],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.vof_last_error.argtypes = [_VP]
    lib.vof_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def c_grid(g) -> CGrid:
    return CGrid(int(g.nx), int(g.ny), int(g.nz), float(g.h), int(getattr(g, "per_x", 0)),
                 int(getattr(g, "per_y", 0)))


def c_phys(p) -> CPhys:
    return CPhys(p.rho_l, p.rho_g, p.mu_l, p.mu_g, p.sigma, p.g_z, p.rho0, p.dpdz,
                 int(p.conv_scheme), int(p.kappa_mode), float(p.kappa_exact))


COARSEN_FACE_MEAN, COARSEN_DENSITY_MEAN = 0, 1
CYCLE_W, CYCLE_V = 0, 1
GRAPH_AUTO, GRAPH_OFF, GRAPH_CYCLE = 0, 1, 2
TAIL_LAUNCHES, TAIL_CLUSTER = 0, 1
TUNE_AUTO, TUNE_OFF = 0, 1


def c_solver(precision=PREC_FP64, rtol=1e-10, max_iter=200, nu_pre=2, nu_post=2, mg_omega=0.0,
             coarse_iters=0, coarse_tol=0.0, mg_interp=0, mg_coarsen=COARSEN_FACE_MEAN,
             mg_cycle=CYCLE_W, mg_w_depth=0, graph=GRAPH_AUTO, nu_fine=0,
             ssf_solves=1, mg_tail=0, mg_tune=TUNE_AUTO) -> CSolver:
    return CSolver(int(precision), float(rtol), int(max_iter), int(nu_pre), int(nu_post),
                   float(mg_omega), int(coarse_iters), float(coarse_tol), int(mg_interp),
                   int(mg_coarsen), int(mg_cycle), int(mg_w_depth), int(graph), int(nu_fine),
                   int(ssf_solves), int(mg_tail), int(mg_tune))


def workspace_bytes(grid, solver: CSolver | None = None) -> int:
    out = ctypes.c_size_t(0)
    g = c_grid(grid)
    s = solver or c_solver()
    st = load().vof_workspace_bytes(ctypes.byref(g), ctypes.byref(s), ctypes.byref(out))
    if st:
        raise VofError(st, "vof_workspace_bytes")
    return int(out.value)


class VofContext:
    """One library context (workspace on the current CUDA device)."""

    def __init__(self, grid, phys, solver: CSolver | None = None, budget_bytes: int = 0,
                 stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.lib = load()
        self.grid = grid
        self.shapes = ((grid.nz, grid.ny, grid.nx), (grid.nz, grid.ny, grid.nx + 1),
                       (grid.nz, grid.ny + 1, grid.nx), (grid.nz, grid.ny, grid.nx))
        self._g, self._p = c_grid(grid), c_phys(phys)
        self._s = solver or c_solver()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self._ctx = _VP()
        st = self.lib.vof_create(ctypes.byref(self._g), ctypes.byref(self._p),
                                 ctypes.byref(self._s), ctypes.c_size_t(budget_bytes),
                                 _VP(stream.cuda_stream), ctypes.byref(self._ctx))
        if st:
            raise VofError(st, "vof_create")

    # -- helpers -------------------------------------------------------------
    def _chk(self, st: int, where: str, rep: CReport | None = None):
        if st:
            msg = self.lib.vof_last_error(self._ctx)
            raise VofError(st, where, msg.decode() if msg else "",
                           rep.as_dict() if rep is not None else None)

    def _ptr(self, t, kind: int, name: str):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
                and t.is_contiguous()):
            raise TypeError(f"{name}: need a contiguous float64 CUDA tensor")
        if tuple(t.shape) != self.shapes[kind]:
            raise ValueError(f"{name}: shape {tuple(t.shape)} != {self.shapes[kind]}")
        return _VP(t.data_ptr())

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            self.lib.vof_destroy(self._ctx)
            self._ctx = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- entry points (same names as the C ABI) --------------------------------
    def vof_advect(self, alpha, u, v, w, dt: float, step_index: int, fluxes=None,
                   report: bool = True):
        """fluxes: optional (fx, fy, fz) face tensors receiving the liquid fluxes."""
        rep = CReport()
        fl = ([self._ptr(f, k + 1, n) for k, (f, n) in enumerate(zip(fluxes, ("fx", "fy", "fz")))]
              if fluxes is not None else [None, None, None])
        st = self.lib.vof_advect(self._ctx, self._ptr(alpha, 0, "alpha"), self._ptr(u, 1, "u"),
                                 self._ptr(v, 2, "v"), self._ptr(w, 3, "w"), float(dt),
                                 int(step_index), *fl, ctypes.byref(rep) if report else None)
        self._chk(st, "vof_advect", rep)
        return rep.as_dict() if report else None

    def ssf_force(self, alpha, kappa, sx, sy, sz):
        st = self.lib.ssf_force(self._ctx, self._ptr(alpha, 0, "alpha"), self._ptr(kappa, 0, "kappa"),
                                self._ptr(sx, 1, "sx"), self._ptr(sy, 2, "sy"), self._ptr(sz, 3, "sz"))
        self._chk(st, "ssf_force")

    def pressure_solve(self, alpha, b, p, report: bool = True):
        rep = CReport()
        st = self.lib.pressure_solve(self._ctx, self._ptr(alpha, 0, "alpha"), self._ptr(b, 0, "b"),
                                     self._ptr(p, 0, "p"), ctypes.byref(rep) if report else None)
        self._chk(st, "pressure_solve", rep)
        return rep.as_dict() if report else None

    def vof_apply_operator(self, alpha, x, y):
        st = self.lib.vof_apply_operator(self._ctx, self._ptr(alpha, 0, "alpha"),
                                         self._ptr(x, 0, "x"), self._ptr(y, 0, "y"))
        self._chk(st, "vof_apply_operator")

    def vof_predict(self, alpha_n, alpha_np1, uc, vc, wc, u, v, w, fx, fy, fz, dt: float):
        st = self.lib.vof_predict(self._ctx, self._ptr(alpha_n, 0, "alpha_n"),
                                  self._ptr(alpha_np1, 0, "alpha_np1"), self._ptr(uc, 0, "uc"),
                                  self._ptr(vc, 0, "vc"), self._ptr(wc, 0, "wc"),
                                  self._ptr(u, 1, "u"), self._ptr(v, 2, "v"), self._ptr(w, 3, "w"),
                                  self._ptr(fx, 1, "fx"), self._ptr(fy, 2, "fy"),
                                  self._ptr(fz, 3, "fz"), float(dt))
        self._chk(st, "vof_predict")

    def project(self, alpha, uc, vc, wc, u, v, w, p, sx, sy, sz, dt: float, report: bool = True):
        rep = CReport()
        st = self.lib.project(self._ctx, self._ptr(alpha, 0, "alpha"), self._ptr(uc, 0, "uc"),
                              self._ptr(vc, 0, "vc"), self._ptr(wc, 0, "wc"), self._ptr(u, 1, "u"),
                              self._ptr(v, 2, "v"), self._ptr(w, 3, "w"), self._ptr(p, 0, "p"),
                              self._ptr(sx, 1, "sx"), self._ptr(sy, 2, "sy"), self._ptr(sz, 3, "sz"),
                              float(dt), ctypes.byref(rep) if report else None)
        self._chk(st, "project", rep)
        return rep.as_dict() if report else None

    def step(self, alpha, uc, vc, wc, u, v, w, p, dt: float, step_index: int,
             report: bool = True):
        rep = CReport()
        st = self.lib.step(self._ctx, self._ptr(alpha, 0, "alpha"), self._ptr(uc, 0, "uc"),
                           self._ptr(vc, 0, "vc"), self._ptr(wc, 0, "wc"), self._ptr(u, 1, "u"),
                           self._ptr(v, 2, "v"), self._ptr(w, 3, "w"), self._ptr(p, 0, "p"),
                           float(dt), int(step_index), ctypes.byref(rep) if report else None)
        self._chk(st, "step", rep)
        return rep.as_dict() if report else None

    def _hptr(self, t, kind: int, name: str):
        import torch
        if not (isinstance(t, torch.Tensor) and t.device.type == "cpu"
                and t.dtype == torch.float64 and t.is_contiguous()):
            raise TypeError(f"{name}: need a contiguous float64 host tensor")
        if tuple(t.shape) != self.shapes[kind]:
            raise ValueError(f"{name}: shape {tuple(t.shape)} != {self.shapes[kind]}")
        return _VP(t.data_ptr())

    def step_host(self, alpha, uc, vc, wc, u, v, w, p, dt: float, step_index: int,
                  report: bool = True):
        """One step on host tensors (pinned for overlapped copies). With a
        report the tensors hold the new state on return; without, after
        host_join() and a synchronisation of the context stream."""
        rep = CReport()
        st = self.lib.vof_step_host(
            self._ctx, self._hptr(alpha, 0, "alpha"), self._hptr(uc, 0, "uc"),
            self._hptr(vc, 0, "vc"), self._hptr(wc, 0, "wc"), self._hptr(u, 1, "u"),
            self._hptr(v, 2, "v"), self._hptr(w, 3, "w"), self._hptr(p, 0, "p"), float(dt),
            int(step_index), ctypes.byref(rep) if report else None)
        self._chk(st, "vof_step_host", rep)
        return rep.as_dict() if report else None

    def host_join(self):
        """Order the copies of earlier step_host calls before later work on
        the context stream."""
        self._chk(self.lib.vof_host_join(self._ctx), "vof_host_join")

    def diag_wait_timeout(self):
        """Runs the bounded-wait failure path once (raises VofError
        VOF_ERR_TIMEOUT); the context stays usable."""
        self._chk(self.lib.vof_diag_wait_timeout(self._ctx), "vof_diag_wait_timeout")

    def launch_count(self) -> int:
        n = ctypes.c_longlong(0)
        self._chk(self.lib.vof_launch_count(self._ctx, ctypes.byref(n)), "vof_launch_count")
        return int(n.value)

    def mg_shape(self, level: int):
        """Launch shape of a coarse level's colour passes: (z planes per
        thread of a tiled pass or 0, threads of a 1-D block or 0, threads of
        a 1-D block of the restriction from it or 0, timed)."""
        sh = (ctypes.c_int * 4)()
        self._chk(self.lib.vof_mg_shape(self._ctx, int(level), sh), "vof_mg_shape")
        return (sh[0], sh[1], sh[2], bool(sh[3]))

    def set_mg_shape(self, level: int, planes: int, block: int, restrict_block: int):
        """Sets a coarse level's launch shape (the first three values of
        mg_shape); before the first solve."""
        sh = (ctypes.c_int * 3)(int(planes), int(block), int(restrict_block))
        self._chk(self.lib.vof_mg_set_shape(self._ctx, int(level), sh), "vof_mg_set_shape")

    def set_timing(self, on: bool):
        self._chk(self.lib.vof_set_timing(self._ctx, int(bool(on))), "vof_set_timing")

    def kernel_times(self) -> dict:
        cap = 32
        names = (ctypes.c_char_p * cap)()
        ms = (ctypes.c_double * cap)()
        n_l = (ctypes.c_longlong * cap)()
        n = ctypes.c_int(0)
        self._chk(self.lib.vof_kernel_times(self._ctx, names, ms, n_l, cap, ctypes.byref(n)),
                  "vof_kernel_times")
        return {names[i].decode(): (ms[i], int(n_l[i])) for i in range(n.value)}


class VofServer:
    """Continuous-batching server of independent cases on the current device.

    Requests carry numpy float64 host arrays (C order, the shapes above);
    the server reads them when the request starts and writes the results
    back into the same arrays when it finishes. The binding keeps each
    request's arrays alive until its result has been collected.
    """

    def __init__(self, budget_bytes: int, max_concurrent: int = 4):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        torch.cuda.init()
        self.lib = load()
        self._srv = _VP()
        st = self.lib.vof_server_create(ctypes.c_size_t(int(budget_bytes)), int(max_concurrent),
                                        ctypes.byref(self._srv))
        if st:
            raise VofError(st, "vof_server_create")
        self._keep = {}

    @staticmethod
    def _arr(a, shape, name):
        import numpy as np
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
                and a.flags.writeable):
            raise TypeError(f"{name}: need a writeable C-contiguous float64 numpy array")
        if tuple(a.shape) != tuple(shape):
            raise ValueError(f"{name}: shape {tuple(a.shape)} != {tuple(shape)}")
        return a.ctypes.data_as(_DP)

    def _submit(self, rq: CRequest, keep) -> int:
        rid = ctypes.c_ulonglong(0)
        st = self.lib.vof_submit(self._srv, ctypes.byref(rq), ctypes.byref(rid))
        if st:
            raise VofError(st, "vof_submit")
        self._keep[rid.value] = (rq, keep)
        return int(rid.value)

    def submit_step(self, grid, phys, solver, state, n_steps: int, dt: float, step0: int = 0) -> int:
        """state: the eight arrays (alpha, uc, vc, wc, u, v, w, p), advanced in place."""
        cs = (grid.nz, grid.ny, grid.nx)
        shapes = (cs, cs, cs, cs, (grid.nz, grid.ny, grid.nx + 1), (grid.nz, grid.ny + 1, grid.nx),
                  cs, cs)
        names = ("alpha", "uc", "vc", "wc", "u", "v", "w", "p")
        ptrs = [self._arr(a, sh, n) for a, sh, n in zip(state, shapes, names)]
        rq = CRequest(REQ_STEP, c_grid(grid), c_phys(phys), solver or c_solver(), int(n_steps),
                      float(dt), int(step0), *ptrs, None)
        return self._submit(rq, tuple(state))

    def submit_solve(self, grid, phys, solver, alpha, b, p) -> int:
        """One pressure solve; p holds the initial guess and receives the solution."""
        cs = (grid.nz, grid.ny, grid.nx)
        pa, pb, pp = self._arr(alpha, cs, "alpha"), self._arr(b, cs, "b"), self._arr(p, cs, "p")
        rq = CRequest(REQ_SOLVE, c_grid(grid), c_phys(phys), solver or c_solver(), 0, 0.0, 0,
                      pa, None, None, None, None, None, None, pp, pb)
        return self._submit(rq, (alpha, b, p))

    def poll(self, rid: int) -> dict:
        res = CResult()
        st = self.lib.vof_poll(self._srv, ctypes.c_ulonglong(rid), ctypes.byref(res))
        if st:
            raise VofError(st, "vof_poll")
        if res.state == 2:
            self._keep.pop(rid, None)
        return res.as_dict()

    def wait(self, rid: int) -> dict:
        res = CResult()
        st = self.lib.vof_wait(self._srv, ctypes.c_ulonglong(rid), ctypes.byref(res))
        if st:
            raise VofError(st, "vof_wait")
        self._keep.pop(rid, None)
        return res.as_dict()

    def close(self):
        if getattr(self, "_srv", None) and self._srv.value:
            self.lib.vof_server_destroy(self._srv)
            self._srv = _VP()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class VofEnsemble:
    """n independent cases of one grid advanced together by one step per call
    (fields: per case the eight device tensors of `VofContext.step`)."""

    AUTO, STREAMS, BATCHED = 0, 1, 2

    def __init__(self, grid, phys_list, solver: CSolver | None = None, n_streams: int = 8,
                 mode: int = 0):
        """mode: AUTO (batched solves where the solver allows them, else
        streams), STREAMS or BATCHED (vof_ensemble_create_mode)."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        torch.cuda.init()
        self.lib = load()
        self.grid = grid
        self.n = len(phys_list)
        self._phys = (CPhys * self.n)(*[c_phys(p) for p in phys_list])
        self._g = c_grid(grid)
        self._s = solver or c_solver()
        self._e = _VP()
        st = self.lib.vof_ensemble_create_mode(ctypes.byref(self._g), self._phys, self.n,
                                               ctypes.byref(self._s), self.n, int(n_streams),
                                               int(mode), ctypes.byref(self._e))
        if st:
            raise VofError(st, "vof_ensemble_create_mode")
        b = ctypes.c_int(0)
        self.lib.vof_ensemble_batched(self._e, ctypes.byref(b))
        self.batched = bool(b.value)
        cs = (grid.nz, grid.ny, grid.nx)
        self.shapes = (cs, cs, cs, cs, (grid.nz, grid.ny, grid.nx + 1),
                       (grid.nz, grid.ny + 1, grid.nx), cs, cs)

    def phase_ms(self):
        """ms so far (before the solves, the batched solve, after it): host
        time for host-driven steps, the device timer for graph steps."""
        ms = (_D * 3)()
        self.lib.vof_ensemble_phase_ms(self._e, ms)
        return tuple(ms)

    def launch_count(self) -> int:
        n = ctypes.c_longlong(0)
        self.lib.vof_ensemble_launch_count(self._e, ctypes.byref(n))
        return int(n.value)

    def graph_steps(self) -> int:
        """Steps so far that ran as one CUDA graph launch."""
        n = ctypes.c_longlong(0)
        self.lib.vof_ensemble_graph_steps(self._e, ctypes.byref(n))
        return int(n.value)

    def mg_shape(self, level: int):
        """Ctx.mg_shape of the batched solve's launches."""
        sh = (ctypes.c_int * 4)()
        st = self.lib.vof_ensemble_mg_shape(self._e, int(level), sh)
        if st != 0:
            raise VofError(st, "vof_ensemble_mg_shape")
        return (sh[0], sh[1], sh[2], bool(sh[3]))

    def step(self, fields, dts, step_index: int, reports: bool = False):
        """fields: list (one per case) of the eight CUDA float64 tensors."""
        import torch
        if len(fields) != self.n or len(dts) != self.n:
            raise ValueError("one field set and one dt per case")
        ptrs = (_VP * (8 * self.n))()
        for c, fs in enumerate(fields):
            for q, (t, sh) in enumerate(zip(fs, self.shapes)):
                if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
                        and t.is_contiguous() and tuple(t.shape) == sh):
                    raise TypeError(f"case {c} field {q}: need a contiguous float64 CUDA tensor {sh}")
                ptrs[8 * c + q] = t.data_ptr()
        dt = (_D * self.n)(*[float(x) for x in dts])
        status = (ctypes.c_int * self.n)()
        reps = (CReport * self.n)() if reports else None
        torch.cuda.current_stream().synchronize()  # inputs written on torch's stream are ready
        st = self.lib.vof_ensemble_step(self._e, ptrs, dt, int(step_index), status, reps)
        if st:
            raise VofError(st, "vof_ensemble_step", f"case statuses {list(status)}")
        return [r.as_dict() for r in reps] if reports else None

    def close(self):
        if getattr(self, "_e", None) and self._e.value:
            self.lib.vof_ensemble_destroy(self._e)
            self._e = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


NSTAT = 20
STAT_NAMES = ("phi", "u", "v", "w", "uu", "vv", "ww", "uv", "uw", "vw")


class VofStats:
    """Running z- and time-sums of the duct statistics on the device
    (`vof_stats_*`); `means()` turns them into profiles over the cross-section."""

    def __init__(self, grid):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        torch.cuda.init()
        self.lib = load()
        self.grid = grid
        self._g = c_grid(grid)
        self._s = _VP()
        st = self.lib.vof_stats_create(ctypes.byref(self._g), ctypes.byref(self._s))
        if st:
            raise VofError(st, "vof_stats_create")

    def accumulate(self, alpha, uc, vc, wc, stream=None):
        import torch
        shape = (self.grid.nz, self.grid.ny, self.grid.nx)
        for t in (alpha, uc, vc, wc):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
                    and t.is_contiguous() and tuple(t.shape) == shape):
                raise TypeError(f"need contiguous float64 CUDA tensors of shape {shape}")
        s = stream if stream is not None else torch.cuda.current_stream()
        st = self.lib.vof_stats_accumulate(self._s, alpha.data_ptr(), uc.data_ptr(), vc.data_ptr(),
                                           wc.data_ptr(), _VP(s.cuda_stream))
        if st:
            raise VofError(st, "vof_stats_accumulate")

    def sums(self):
        import numpy as np
        out = np.zeros((NSTAT, self.grid.ny, self.grid.nx))
        n = ctypes.c_longlong(0)
        st = self.lib.vof_stats_read(self._s, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     ctypes.byref(n))
        if st:
            raise VofError(st, "vof_stats_read")
        return out, int(n.value)

    def means(self):
        """Mixture means of phi, u, v, w and the second moments; the liquid
        means (alpha-weighted, prefixed 'l_'); and the Reynolds stresses
        ('rs_uu' = <uu> - <u><u>, ...), each a (ny, nx) array."""
        import numpy as np
        S, n = self.sums()
        if n == 0:
            raise ValueError("no samples")
        N = n * self.grid.nz
        out = {name: S[q] / N for q, name in enumerate(STAT_NAMES)}
        wa = np.where(S[10] > 0, S[10], 1.0)
        for q, name in enumerate(STAT_NAMES[1:], start=1):
            out["l_" + name] = S[10 + q] / wa
        for p in ("l_", ""):
            for a, b in (("u", "u"), ("v", "v"), ("w", "w"), ("u", "v"), ("u", "w"), ("v", "w")):
                out[p + "rs_" + a + b] = out[p + a + b] - out[p + a] * out[p + b]
        out["samples"] = n
        return out

    def reset(self):
        st = self.lib.vof_stats_reset(self._s)
        if st:
            raise VofError(st, "vof_stats_reset")

    def close(self):
        if getattr(self, "_s", None) and self._s.value:
            self.lib.vof_stats_destroy(self._s)
            self._s = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def fold_quadrants(profile, parity_x: int = 1, parity_y: int = 1):
    """Average a (ny, nx) cross-section profile over the duct's four
    quadrants (mirror symmetry about both centre lines). parity_x/_y = -1
    for a quantity odd under the mirror in x/y (u under x-mirror, v under
    y-mirror, uv under either, ...)."""
    import numpy as np
    p = np.asarray(profile)
    return 0.25 * (p + parity_x * p[:, ::-1] + parity_y * p[::-1, :] +
                   parity_x * parity_y * p[::-1, ::-1])
