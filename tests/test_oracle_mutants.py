"""The viscous and face-curvature pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a flipped
sign, a stencil at the wrong cell or in the wrong direction, a wrong ghost
sign, a face average replaced by one cell, a fallback branch miswired),
builds that copy, and requires at least one of the pins named for it to
fail. The oracle itself is not changed; the planted copy lives in a
temporary folder for the duration of the test only.
"""
import os
import shutil
import subprocess

import pytest

import oracle
import test_oracle_face_curvature as FK
import test_oracle_viscous as VI


def _viscous_pins():
    return [VI.test_interior_quadratic_fields_give_lap_plus_grad_div,
            *[(lambda w=w: VI.test_no_slip_ghosts_exact_for_fields_odd_about_the_wall(w))
              for w in ("x0", "x1", "y0", "y1")],
            *[(lambda c=c: VI.test_no_slip_ghosts_exact_in_the_corners(c))
              for c in ((0, 0), (1, 0), (0, 1), (1, 1))],
            VI.test_viscous_fluxes_telescope_for_any_viscosity_field,
            VI.test_two_fluid_shear_layer_with_uniform_traction_is_in_equilibrium]


def _face_pins():
    return [FK.test_face_value_with_two_valid_cells_is_their_mean_curvature,
            FK.test_face_curvature_branches_on_a_capped_cylinder]


MUTANTS = {
    "transpose term with the wrong sign":
        ("s += sg * muf * (dq + dt_);", "s += sg * muf * (dq - dt_);", _viscous_pins),
    "tangential difference of the neighbour taken at the cell itself":
        ("VC(g, U[d], ni + e[0], nj + e[1], nk + e[2])", "VC(g, U[d], i + e[0], j + e[1], k + e[2])",
         _viscous_pins),
    "tangential difference along the face normal":
        ("e[comp] = 1;", "e[d] = 1;", _viscous_pins),
    "no sign change of the ghost across the y walls":
        ("if (j < 0) { j = 0; s = -s; }", "if (j < 0) { j = 0; }", _viscous_pins),
    "face viscosity of one cell":
        ("const double muf = 0.5 * (MUC(g, p, a, i, j, k) + MUC(g, p, a, ni, nj, nk));",
         "const double muf = MUC(g, p, a, i, j, k);", _viscous_pins),
    "face value from one valid cell only":
        ("return 0.5 * (kappa[cL] + kappa[cR]);", "return kappa[cL];", _face_pins),
    "one-valid branch returning the other cell":
        ("if (valid[cR]) return kappa[cR];", "if (valid[cR]) return kappa[cL];", _face_pins),
    "block mean over all 18 cells":
        ("return cnt ? s / cnt : 0.0;", "return cnt ? s / 18.0 : 0.0;", _face_pins),
    "block oriented across the face":
        ("x[dir] += side; x[t1] += p; x[t2] += q;", "x[t1] += side; x[dir] += p; x[t2] += q;",
         _face_pins),
    "fallbacks not counted":
        ("(*fallbacks)++;", "", _face_pins),
    "invalid cells averaged in the block":
        ("if (valid[c]) { s += kappa[c]; ++cnt; }", "{ s += kappa[c]; ++cnt; }", _face_pins),
}


@pytest.fixture(scope="module")
def sources():
    here = os.path.dirname(os.path.abspath(oracle.__file__))
    with open(os.path.join(here, "vof_oracle.c")) as f:
        return f.read(), os.path.join(here, "vof_oracle.h")


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_fails_a_pin(name, sources, tmp_path, monkeypatch):
    src, hdr = sources
    old, new, pins = MUTANTS[name]
    assert src.count(old) == 1, f"anchor of '{name}' not unique in the oracle source"
    shutil.copy(hdr, tmp_path / "vof_oracle.h")
    (tmp_path / "vof_oracle.c").write_text(src.replace(old, new))
    so = str(tmp_path / "libmutant.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                    "-fno-fast-math", "-o", so, str(tmp_path / "vof_oracle.c"), "-lm"], check=True)
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(oracle, "build", lambda force=False: so)
    failed = 0
    for pin in pins():
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed >= 1, f"no pin caught the planted mistake '{name}'"
