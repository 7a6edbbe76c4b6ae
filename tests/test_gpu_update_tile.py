"""GPU: the x/p update tile (kw_set_update_tile) and its autotuner.

The tile (4, 8 or 16 shifts per block item) only decides which block updates
which (shift, element) pair of Eq. 23-24, so every tile, and the timed pick,
gives the same x bit for bit, in every form and with FP32 shift storage; the
pick is one of the three; a batch with a forced tile equals the default.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2001_08707_gb300 import komega as kw
from paper_2001_08707_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2001_08707_gb300 import build

    build.build()


@pytest.mark.parametrize("form", ["f64", "df64", "df64+x32", "c32"])
def test_every_tile_gives_the_same_x(form):
    p = w.anderson_small(L=9, K=37, delta=0.1, tol=1e-9)   # K not a multiple of any tile
    prec = form.split("+")[0]
    xs, tiles = {}, {}
    for ts in (0, 4, 8, 16):
        s = kw.Solver(prec, tol=p.tol)
        s.set_csr(p.H.rowptr, p.H.col, p.H.val)
        s.set_shift_storage(form.endswith("x32"))
        s.set_update_tile(ts)
        r = s.solve(p.b, p.z, full=True)
        assert r.status == "KW_OK"
        xs[ts] = r.x.cpu().numpy()
        tiles[ts] = s.update_tile()
    assert tiles[4] == 4 and tiles[8] == 8 and tiles[16] == 16 and tiles[0] in (4, 8, 16)
    for ts in (4, 8, 16):
        np.testing.assert_array_equal(xs[ts], xs[0])


def test_batch_with_forced_tile_equals_default():
    probs = w.anderson_batch(n=3, L_range=(6, 9), K_range=(5, 40))
    problems = [{"H": q.H, "b": q.b, "z": q.z, "tol": q.tol, "full": True} for q in probs]
    out = []
    for ts in (0, 16):
        s = kw.Solver("df64", tol=1e-8)
        s.set_update_tile(ts)
        out.append(s.solve_batched(problems))
    for a, b in zip(*out):
        assert a.status == b.status == "KW_OK"
        np.testing.assert_array_equal(a.x.cpu().numpy(), b.x.cpu().numpy())


def test_update_tile_argument():
    s = kw.Solver("df64")
    for bad in (1, 2, 3, 32, -1):
        assert s._lib.kw_set_update_tile(s._ctx, bad) == kw.KW_ERR_ARG
    assert s.update_tile() == 0
