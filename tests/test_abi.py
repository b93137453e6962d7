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
