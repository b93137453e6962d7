"""Helpers for the GPU parity tests (device copies, contexts, norms)."""
import numpy as np

import paper_2104_01636_b300 as vd


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def ctx(case_or_grid, phys=None, rtol=1e-12, max_iter=400, precision=0, **kw):
    g = case_or_grid.grid if phys is None else case_or_grid
    p = case_or_grid.phys if phys is None else phys
    return vd.VofContext(g, p, vd.c_solver(precision, rtol=rtol, max_iter=max_iter, **kw))


def rel_l2(a, b):
    a = np.concatenate([np.ravel(x) for x in a]) if isinstance(a, (list, tuple)) else np.ravel(a)
    b = np.concatenate([np.ravel(x) for x in b]) if isinstance(b, (list, tuple)) else np.ravel(b)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def rel_max(a, b):
    den = np.max(np.abs(b))
    return np.max(np.abs(a - b)) / (den if den > 0 else 1.0)
