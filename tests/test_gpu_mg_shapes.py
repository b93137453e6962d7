"""Launch shapes of the coarse multigrid levels' colour passes and narrow
restrictions: timed when a context is created (mg_tune), reported, and
settable; every shape gives the same bits, because the passes are pointwise
and round the same way under every thread mapping."""
import numpy as np
import pytest

import paper_2104_01636_b300 as vd
from paper_2104_01636_b300 import inputs as I
from gpu_util import ctx, dev, host

pytestmark = pytest.mark.gpu

# 128^3: level 1 (64^3 = 2^18 cells) runs tiled passes on FP16 coefficient
# copies in the mixed cycle, levels 2 and 3 (32^3, 16^3) run 1-D blocks,
# level 4 (8^3) is solved densely
CASE = dict(nx=128, ny=128, nz=128, nbub=6, d_cells=12, seed=2113)


def _run(case, steps, kw, shapes=None):
    fields = [dev(a) for a in case.state()]
    with ctx(case, **kw) as C:
        got = [C.mg_shape(l) for l in (1, 2, 3)]
        if shapes:
            for l, sh in shapes.items():
                C.set_mg_shape(l, *sh)
        reps = [C.step(*fields, case.dt, s) for s in range(steps)]
        after = [C.mg_shape(l) for l in (1, 2, 3)]
    return [host(t) for t in fields], reps, got, after


@pytest.mark.parametrize("prec", [1, 0])
def test_timed_and_set_shapes_give_the_same_bits(prec):
    case = I.rising_swarm(**CASE)
    kw = dict(precision=prec, rtol=1e-9, max_iter=300)
    ref, ref_reps, off, _ = _run(case, 2, dict(kw, mg_tune=vd.TUNE_OFF))
    # built in: a quarter of the level's z chunk on the tiled level, 256-thread blocks
    assert off[0][0] > 0 and off[0][1:] == (0, 0, False)
    assert off[1][:2] == (0, 256) and off[2][:2] == (0, 256)
    assert not off[1][3] and not off[2][3]
    # the 1-D restriction exists on the mixed path (FP32 coefficients) only
    assert (off[1][2], off[2][2]) == ((256, 256) if prec == 1 else (0, 0))

    got, reps, tuned, _ = _run(case, 2, kw)
    assert all(t[3] for t in tuned)
    assert tuned[0][1] == 0 and tuned[1][0] == 0 and tuned[2][0] == 0
    assert tuned[1][1] in (64, 128, 256, 512) and tuned[2][1] in (64, 128, 256, 512)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    assert [r["iters"] for r in reps] == [r["iters"] for r in ref_reps]

    # shapes outside the timed candidates, set by hand
    rb = (lambda b: b if prec == 1 else 0)
    for shapes in ({1: (1, 0, 0), 2: (0, 32, rb(1024)), 3: (0, 1024, rb(32))},
                   {1: (64, 0, 0), 2: (0, 96, rb(160)), 3: (0, 480, rb(64))},
                   {1: (3, 0, 0), 2: (0, 512, rb(128)), 3: (0, 64, rb(96))}):
        got, _, _, after = _run(case, 2, dict(kw, mg_tune=vd.TUNE_OFF), shapes)
        assert [a[:3] for a in after] == [shapes[l] for l in (1, 2, 3)]
        assert not any(a[3] for a in after)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)


def test_set_shape_rejects_bad_values():
    case = I.rising_swarm(**CASE)
    with ctx(case, precision=1, rtol=1e-9, mg_tune=vd.TUNE_OFF) as C:
        before = [C.mg_shape(l) for l in (1, 2, 3)]
        bad = [(0, (4, 0, 0)),          # the finest level: the fused sweep
               (4, (0, 256, 256)),      # the coarsest: solved densely
               (1, (0, 256, 0)),        # a tiled level takes planes, not a block
               (1, (65, 0, 0)),         # more planes than the level has
               (2, (2, 0, 256)),        # a 1-D level takes no planes
               (2, (0, 48, 256)),       # not a multiple of 32
               (2, (0, 2048, 256)),     # above 1024
               (3, (0, 256, 0))]        # its restriction is 1-D as well
        for level, sh in bad:
            with pytest.raises(vd.VofError) as e:
                C.set_mg_shape(level, *sh)
            assert e.value.name == "VOF_ERR_ARG"
        assert [C.mg_shape(l) for l in (1, 2, 3)] == before


def test_ensemble_batched_shapes_are_timed():
    """The batched solve's shapes are timed for the launches of all its
    cases at once; the cases stay bitwise equal to their solo runs (the
    equality tests of the ensemble run with the timed shapes)."""
    cases = I.ensemble_cases(8, dims=(32, 32, 48), seed=83)
    kw = dict(precision=1, rtol=1e-9, max_iter=300)
    fields = [[dev(a) for a in c.state()] for c in cases]
    with vd.VofEnsemble(cases[0].grid, [c.phys for c in cases], vd.c_solver(**kw),
                        n_streams=2, mode=vd.VofEnsemble.BATCHED) as E:
        sh = E.mg_shape(1)  # 16 x 16 x 24 per case: 1-D blocks
        assert sh[0] == 0 and sh[1] in (64, 128, 256, 512) and sh[3]
        E.step(fields, [c.dt for c in cases], 0)
    for c, fs in zip(cases, fields):
        solo = [dev(a) for a in c.state()]
        with ctx(c, mg_tune=vd.TUNE_OFF, **kw) as C:
            C.step(*solo, c.dt, 0)
        for a, b in zip(fs, solo):
            assert np.array_equal(host(a), host(b))
