"""Device statistics against the oracle's column sums over several samples."""
import numpy as np
import pytest

import paper_2104_01636_b300 as vd
from oracle import stats as S
from paper_2104_01636_b300 import inputs as I
from gpu_util import dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims", [(37, 21, 30), (64, 48, 16)])
def test_stats_match_oracle(dims):
    g = I.Grid(*dims)
    rng = np.random.default_rng(5)
    ref = np.zeros((S.NAMES.__len__() * 2, g.ny, g.nx))
    with vd.VofStats(g) as st:
        for _ in range(3):
            a = rng.uniform(size=g.shapes()[0])
            u, v, w = (rng.normal(size=g.shapes()[0]) for _ in range(3))
            st.accumulate(dev(a), dev(u), dev(v), dev(w))
            ref += S.column_sums(a, u, v, w)
        got, n = st.sums()
        m = st.means()
    assert n == 3
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    mo = S.means(ref, 3, g.nz)
    for k in ("phi", "w", "rs_uw", "l_u", "l_rs_ww"):
        assert np.allclose(m[k], mo[k], rtol=1e-10, atol=1e-12)
