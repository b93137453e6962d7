"""The ensemble: every case's result is bitwise that of the same case stepped
alone; a case that fails reports its own status."""
import numpy as np
import pytest

import paper_2104_01636_b300 as vd
from paper_2104_01636_b300 import inputs as I
from gpu_util import ctx, dev, host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,streams", [(1, 2), (0, 3), (1, 1)])
def test_ensemble_equals_solo(prec, streams):
    cases = I.ensemble_cases(3, dims=(32, 32, 48), seed=77)
    kw = dict(precision=prec, rtol=1e-9, max_iter=300)
    fields = [[dev(a) for a in c.state()] for c in cases]
    with vd.VofEnsemble(cases[0].grid, [c.phys for c in cases], vd.c_solver(**kw),
                        n_streams=streams) as E:
        for s in range(3):
            reps = E.step(fields, [c.dt for c in cases], s, reports=True)
            assert all(r["res"] <= 1e-9 for r in reps)
    for c, fs in zip(cases, fields):
        solo = [dev(a) for a in c.state()]
        with ctx(c, **kw) as C:
            for s in range(3):
                C.step(*solo, c.dt, s)
        for a, b in zip(fs, solo):
            assert np.array_equal(host(a), host(b))


def test_ensemble_reports_failing_case():
    cases = I.ensemble_cases(2, dims=(32, 32, 48), seed=78)
    fields = [[dev(a) for a in c.state()] for c in cases]
    with vd.VofEnsemble(cases[0].grid, [c.phys for c in cases], vd.c_solver(1, rtol=1e-8),
                        n_streams=2) as E:
        with pytest.raises(vd.VofError) as e:
            E.step(fields, [cases[0].dt, cases[1].dt * 1e4], 0)
        assert e.value.name == "VOF_ERR_CFL"
        assert "[0, 6]" in str(e.value)
