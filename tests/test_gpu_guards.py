"""Guard canaries around the caller's fields: every field lives in the middle
of a larger device buffer whose margins hold a NaN with a distinctive bit
pattern. After whole steps (FP64 and mixed, the density-staged finest level
and the face-array one) the margins keep their bits (no write outside a
field), the results hold no NaN (no read of a margin reached them), and the
results are bitwise those of unpadded fields."""
import numpy as np
import pytest
import torch

import paper_2104_01636_b300 as vd
from paper_2104_01636_b300 import inputs as I
from gpu_util import dev, host

pytestmark = pytest.mark.gpu

GUARD = 8192  # doubles on either side of a field
CANARY = np.array([0x7FF8DEADBEEF1234], dtype=np.uint64).view(np.float64)[0]


def _guarded(a):
    n = a.size
    big = torch.full((n + 2 * GUARD,), float("nan"), dtype=torch.float64, device="cuda")
    big.view(torch.int64).fill_(int(np.array([CANARY]).view(np.int64)[0]))
    big[GUARD:GUARD + n] = torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()
    return big, big[GUARD:GUARD + n].view(a.shape)


def _steps(case, sv, fields, steps):
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        with vd.VofContext(case.grid, case.phys, sv, stream=stream) as C:
            for s in range(steps):
                C.step(*fields, case.dt, s)
            stream.synchronize()


@pytest.mark.parametrize("dims", [(40, 32, 48), (36, 28, 24)])
@pytest.mark.parametrize("prec", [vd.PREC_FP64, vd.PREC_MIXED_FP32])
def test_fields_untouched_outside(dims, prec):
    case = I.rising_swarm(*dims, nbub=3, d_cells=8, seed=102, steps=2)
    sv = vd.c_solver(prec, rtol=1e-9, max_iter=300)
    plain = [dev(a) for a in case.state()]
    _steps(case, sv, plain, 2)
    bigs, views = zip(*[_guarded(a) for a in case.state()])
    _steps(case, sv, list(views), 2)
    canary = int(np.array([CANARY]).view(np.int64)[0])
    for big, view, ref in zip(bigs, views, plain):
        bits = big.view(torch.int64)
        assert bool((bits[:GUARD] == canary).all()) and bool((bits[-GUARD:] == canary).all())
        got = host(view)
        assert not np.isnan(got).any()
        assert np.array_equal(got, host(ref))
