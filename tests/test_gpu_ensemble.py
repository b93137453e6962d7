"""The ensemble: every case's result is bitwise that of the same case stepped
alone, with the cases' pressure solves batched into shared launches (the
whole step one CUDA graph launch, or its loops driven from the host) or with
the cases overlapped on streams; a case that fails reports its own status."""
import numpy as np
import pytest

import paper_2104_01636_b300 as vd
from paper_2104_01636_b300 import inputs as I
from gpu_util import ctx, dev, host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,streams,mode,batched,graph", [
    (1, 2, vd.VofEnsemble.AUTO, True, vd.GRAPH_AUTO),
    (0, 3, vd.VofEnsemble.AUTO, False, vd.GRAPH_AUTO),
    (1, 1, vd.VofEnsemble.STREAMS, False, vd.GRAPH_AUTO),
    (1, 3, vd.VofEnsemble.BATCHED, True, vd.GRAPH_AUTO),
    (1, 3, vd.VofEnsemble.BATCHED, True, vd.GRAPH_CYCLE)])
def test_ensemble_equals_solo(prec, streams, mode, batched, graph):
    """Three steps (both sweep orders, so both captured step graphs)."""
    cases = I.ensemble_cases(3, dims=(32, 32, 48), seed=77)
    kw = dict(precision=prec, rtol=1e-9, max_iter=300, graph=graph)
    fields = [[dev(a) for a in c.state()] for c in cases]
    with vd.VofEnsemble(cases[0].grid, [c.phys for c in cases], vd.c_solver(**kw),
                        n_streams=streams, mode=mode) as E:
        assert E.batched == batched
        for s in range(3):
            reps = E.step(fields, [c.dt for c in cases], s, reports=True)
            assert all(r["res"] <= 1e-9 for r in reps)
        assert E.graph_steps() == (3 if batched and graph == vd.GRAPH_AUTO else 0)
    for c, fs in zip(cases, fields):
        solo = [dev(a) for a in c.state()]
        with ctx(c, **kw) as C:
            for s in range(3):
                C.step(*solo, c.dt, s)
        for a, b in zip(fs, solo):
            assert np.array_equal(host(a), host(b))


def test_batched_ensemble_of_many_cases_equals_solo():
    """Eight cases with different bubbles (so their solves take different
    numbers of iterations and the batch switches finished cases off) and
    reports; each case bitwise equal to its solo run, iteration counts
    equal to the solo solve's."""
    cases = I.ensemble_cases(8, dims=(48, 48, 96), seed=2109)
    kw = dict(precision=1, rtol=1e-8, max_iter=500)
    fields = [[dev(a) for a in c.state()] for c in cases]
    with vd.VofEnsemble(cases[0].grid, [c.phys for c in cases], vd.c_solver(**kw),
                        n_streams=4, mode=vd.VofEnsemble.BATCHED) as E:
        assert E.batched
        reps = [E.step(fields, [c.dt for c in cases], s, reports=True) for s in range(2)]
        assert E.graph_steps() == 2
    iters = set()
    for k, (c, fs) in enumerate(zip(cases, fields)):
        solo = [dev(a) for a in c.state()]
        with ctx(c, **kw) as C:
            solo_reps = [C.step(*solo, c.dt, s) for s in range(2)]
        for a, b in zip(fs, solo):
            assert np.array_equal(host(a), host(b))
        for s in range(2):
            assert reps[s][k]["iters"] == solo_reps[s]["iters"]
            assert reps[s][k]["res"] == solo_reps[s]["res"]
            assert reps[s][k]["max_div"] == solo_reps[s]["max_div"]
            iters.add(reps[s][k]["iters"])
    assert len(iters) > 1  # the cases did not all take the same number of iterations


def test_step_graph_in_four_case_groups_equals_solo():
    """Sixteen cases run as four groups of four, each group with its own
    batched solve and the groups' parts before their solves pipelined; every
    case bitwise equal to its solo run over both sweep orders."""
    cases = I.ensemble_cases(16, dims=(32, 32, 48), seed=81)
    kw = dict(precision=1, rtol=1e-9, max_iter=300)
    fields = [[dev(a) for a in c.state()] for c in cases]
    with vd.VofEnsemble(cases[0].grid, [c.phys for c in cases], vd.c_solver(**kw),
                        n_streams=3, mode=vd.VofEnsemble.BATCHED) as E:
        reps = [E.step(fields, [c.dt for c in cases], s, reports=True) for s in range(2)]
        assert E.graph_steps() == 2
    for k, (c, fs) in enumerate(zip(cases, fields)):
        solo = [dev(a) for a in c.state()]
        with ctx(c, **kw) as C:
            solo_reps = [C.step(*solo, c.dt, s) for s in range(2)]
        for a, b in zip(fs, solo):
            assert np.array_equal(host(a), host(b))
        for s in range(2):
            assert reps[s][k]["iters"] == solo_reps[s]["iters"]


def test_step_graph_recaptured_for_new_time_steps_and_fields():
    """The step graph is captured for the field pointers, the time steps and
    the sweep order: a new dt and new field tensors are captured again, and
    each case stays bitwise equal to its solo run with the same dt."""
    cases = I.ensemble_cases(3, dims=(32, 32, 48), seed=79)
    kw = dict(precision=1, rtol=1e-9, max_iter=300)
    fields = [[dev(a) for a in c.state()] for c in cases]
    dts = [[c.dt for c in cases], [c.dt for c in cases], [0.8 * c.dt for c in cases],
           [0.8 * c.dt for c in cases]]
    with vd.VofEnsemble(cases[0].grid, [c.phys for c in cases], vd.c_solver(**kw),
                        n_streams=2, mode=vd.VofEnsemble.BATCHED) as E:
        for s in range(4):
            if s == 3:
                fields = [[t.clone() for t in f] for f in fields]
            E.step(fields, dts[s], s)
        assert E.graph_steps() == 4
    for k, (c, fs) in enumerate(zip(cases, fields)):
        solo = [dev(a) for a in c.state()]
        with ctx(c, **kw) as C:
            for s in range(4):
                C.step(*solo, dts[s][k], s)
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
        # the step graph's CFL test failed, so the step ran host-driven
        assert E.graph_steps() == 0
