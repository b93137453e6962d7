"""FP64 CPU oracle for the duct statistics (Section 4: profiles averaged over
the streamwise direction and time, for the mixture and for the liquid).

TEST INFRASTRUCTURE ONLY: imported by the test suite, never by the CUDA
library or its binding. The definitions are written out directly: for each
cross-section column, sums over z of the gas fraction phi = 1 - alpha, the
cell velocities, their pairwise products, and the same quantities weighted
by alpha (liquid-phase averages are alpha-weighted sums over the sum of
alpha).
"""
from __future__ import annotations

import numpy as np

NAMES = ("phi", "u", "v", "w", "uu", "vv", "ww", "uv", "uw", "vw")


def column_sums(alpha, uc, vc, wc):
    """(20, ny, nx): rows 0-9 sum_z of phi, u, v, w, uu, vv, ww, uv, uw, vw;
    row 10 sum_z alpha; rows 11-19 sum_z alpha times u ... vw."""
    a, u, v, w = (np.asarray(x, dtype=np.float64) for x in (alpha, uc, vc, wc))
    m = [1.0 - a, u, v, w, u * u, v * v, w * w, u * v, u * w, v * w]
    out = [x.sum(axis=0) for x in m]
    out.append(a.sum(axis=0))
    out += [(a * x).sum(axis=0) for x in m[1:]]
    return np.stack(out)


def means(sums, samples: int, nz: int):
    """Mixture means, alpha-weighted liquid means ('l_') and Reynolds
    stresses ('rs_', 'l_rs_') from accumulated column sums."""
    N = samples * nz
    out = {n: sums[q] / N for q, n in enumerate(NAMES)}
    wa = np.where(sums[10] > 0, sums[10], 1.0)
    for q, n in enumerate(NAMES[1:], start=1):
        out["l_" + n] = sums[10 + q] / wa
    for p in ("l_", ""):
        for a, b in (("u", "u"), ("v", "v"), ("w", "w"), ("u", "v"), ("u", "w"), ("v", "w")):
            out[p + "rs_" + a + b] = out[p + a + b] - out[p + a] * out[p + b]
    return out
