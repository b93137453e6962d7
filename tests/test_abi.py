"""The C-ABI library: builds for sm_103a, loads without a GPU, exports every
entry point its header declares, and sizes/validates workspaces on the host."""
import ctypes
import os
import re

import pytest

import paper_2104_01636_b300 as vd
from paper_2104_01636_b300 import build as vbuild
from paper_2104_01636_b300.inputs import Grid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:vof_status|const\s+char\s*\*)\s+(\w+)\s*\(", src, flags=re.M)
    return names


def test_library_builds_and_exports_every_declared_symbol():
    vbuild.build()
    lib = vd.load()
    names = declared_functions()
    assert len(names) >= 13
    for n in ["vof_advect", "ssf_force", "pressure_solve", "project", "step", "vof_create"]:
        assert n in names
    for n in names:
        assert hasattr(lib, n), n
    raw = ctypes.CDLL(vd.LIB_PATH)
    for n in names:
        getattr(raw, n)


def test_workspace_bytes_on_host():
    b64 = vd.workspace_bytes(Grid(64, 64, 64))
    b128 = vd.workspace_bytes(Grid(128, 128, 128))
    assert 150 * 64 ** 3 < b64 < 450 * 64 ** 3
    # fields scale with the cell count; the dense coarsest-level inverse does not
    assert 7 < b128 / b64 < 8.5
    big = vd.workspace_bytes(Grid(224, 224, 640))
    assert big < 16e9  # the paper-shaped duct fits comfortably in one B300


@pytest.mark.parametrize("dims", [(1, 8, 8), (8, 8, 3), (8, 8, 7), (8, 8, 2)])
def test_invalid_grids_rejected(dims):
    with pytest.raises(vd.VofError) as e:
        vd.workspace_bytes(Grid(*dims))
    assert e.value.name == "VOF_ERR_ARG"


def test_binding_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of the C structs have the header's sizes and offsets."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    checks = {
        "vof_grid": (vd.CGrid, ["nx", "h", "periodic_y"]),
        "vof_phys": (vd.CPhys, ["rho_l", "conv_scheme", "kappa_exact"]),
        "vof_solver": (vd.CSolver, ["precision", "rtol", "mg_omega", "coarse_tol", "mg_interp",
                                    "mg_coarsen", "mg_cycle", "mg_w_depth", "graph",
                                    "nu_fine", "ssf_solves", "mg_tail", "mg_tune"]),
        "vof_report": (vd.CReport, ["iters", "res0", "hf_fallbacks", "ms"]),
        "vof_request": (vd.CRequest, ["kind", "grid", "phys", "solver", "n_steps", "dt", "step0",
                                      "alpha", "p", "b"]),
        "vof_result": (vd.CResult, ["status", "t_submit", "report"]),
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "vof.h"', "int main(void){"]
    for cname, (_, fields) in checks.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        cname, f, val = line.split()
        got[(cname, f)] = int(val)
    for cname, (cls, fields) in checks.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for f in fields:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_binding_constants_match_header(tmp_path):
    """The binding's enum and status constants have the header's values."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    consts = {
        "VOF_PREC_FP64": vd.PREC_FP64, "VOF_PREC_MIXED_FP32": vd.PREC_MIXED_FP32,
        "VOF_COARSEN_FACE_MEAN": vd.COARSEN_FACE_MEAN,
        "VOF_COARSEN_DENSITY_MEAN": vd.COARSEN_DENSITY_MEAN,
        "VOF_CYCLE_W": vd.CYCLE_W, "VOF_CYCLE_V": vd.CYCLE_V,
        "VOF_GRAPH_AUTO": vd.GRAPH_AUTO, "VOF_GRAPH_OFF": vd.GRAPH_OFF,
        "VOF_GRAPH_CYCLE": vd.GRAPH_CYCLE,
        "VOF_TAIL_LAUNCHES": vd.TAIL_LAUNCHES, "VOF_TAIL_CLUSTER": vd.TAIL_CLUSTER,
        "VOF_TUNE_AUTO": vd.TUNE_AUTO, "VOF_TUNE_OFF": vd.TUNE_OFF,
        "VOF_REQ_STEP": vd.REQ_STEP, "VOF_REQ_SOLVE": vd.REQ_SOLVE,
        "VOF_ENSEMBLE_AUTO": vd.VofEnsemble.AUTO, "VOF_ENSEMBLE_STREAMS": vd.VofEnsemble.STREAMS,
        "VOF_ENSEMBLE_BATCHED": vd.VofEnsemble.BATCHED,
    }
    consts.update({name: code for code, name in vd.STATUS.items()})
    lines = ['#include <stdio.h>', '#include "vof.h"', "int main(void){"]
    lines += [f'printf("{n} %d\\n", (int)({n}));' for n in consts]
    lines.append("return 0;}")
    src = tmp_path / "consts.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = dict((n, int(v)) for n, v in (line.split() for line in out.splitlines()))
    assert got == consts


def test_library_binds_its_own_symbols():
    """glibc exports a legacy function named step; the library is linked
    -Bsymbolic so that its internal calls reach its own definitions."""
    import shutil
    import subprocess
    vbuild.build()
    if shutil.which("readelf") is None:
        pytest.skip("readelf not available")
    out = subprocess.run(["readelf", "-d", vd.LIB_PATH], check=True, capture_output=True,
                         text=True).stdout
    assert "SYMBOLIC" in out
    assert hasattr(vd.load(), "vof_step")
