"""The duct driver: a run interrupted by a checkpoint and resumed equals the
uninterrupted run bit for bit; statistics are sampled; a laden restart
inserts bubbles into an unladen field."""
import json
import os

import numpy as np
import pytest

from paper_2104_01636_b300 import checkpoint as ck
from paper_2104_01636_b300 import run

pytestmark = pytest.mark.gpu

SMALL = ["--nx", "32", "--ny", "32", "--nz", "48", "--bubbles", "4", "--rtol", "1e-9"]


def test_resume_equals_uninterrupted(tmp_path):
    a, b, c = (str(tmp_path / n) for n in "abc")
    run.main(SMALL + ["--steps", "6", "--out", a, "--stats-every", "2"])
    run.main(SMALL + ["--steps", "3", "--out", b])
    run.main(SMALL + ["--steps", "3", "--out", c, "--resume", os.path.join(b, "ckpt.bin")])
    ha, xa = ck.load(os.path.join(a, "ckpt.bin"))
    hc, xc = ck.load(os.path.join(c, "ckpt.bin"))
    assert ha["step_index"] == hc["step_index"] == 6
    for p, q in zip(xa, xc):
        assert np.array_equal(p, q)
    s = json.load(open(os.path.join(a, "summary.json")))
    assert s["stats_samples"] == 3
    sums = np.load(os.path.join(a, "stats_sums.npy"))
    assert sums.shape == (20, 32, 32) and np.all(np.isfinite(sums))


def test_laden_restart_inserts_bubbles(tmp_path):
    u, l = str(tmp_path / "u"), str(tmp_path / "l")
    run.main(SMALL + ["--unladen", "--steps", "2", "--out", u])
    hu, xu = ck.load(os.path.join(u, "ckpt.bin"))
    assert xu[0].min() > 1.0 - 1e-12  # liquid everywhere, to round-off
    run.main(SMALL + ["--steps", "2", "--out", l, "--resume", os.path.join(u, "ckpt.bin"),
                      "--insert-bubbles", "3"])
    hl, xl = ck.load(os.path.join(l, "ckpt.bin"))
    assert xl[0].min() < 0.5 and hl["step_index"] == 4
