"""CPU pins for the oracle's recalculation at new shifts (oracle/recalc.py, Sec. 3.3 (iv)).

* Without seed switching the seed sequence does not depend on the other shifts,
  so shifts replayed from the log of a run must equal, bit for bit, the same
  shifts carried inside a combined run (when they freeze before the run ends).
* With seed switching: replayed projections agree with the dense definition
  P (z I - H)^{-1} b within the residual bound ||a|| res / dist(z, spec).
* Replaying the run's own shifts reproduces its projections and freeze points.
* Large |z|: b^T x matches the moment expansion 1/z + b^T H b/z^2 + b^T H^2 b/z^3.
* A truncated log replays exactly the run stopped at that iteration.
* Planted mistakes in the replay (no switch rescale, shifted w index, sign of
  c) are rejected by the dense pin.
"""
import sys
import types

import numpy as np
import pytest

import oracle.recalc as orc_mod
from oracle import shifted_cocg as oc
from paper_2001_08707_gb300 import workloads as w


def _anderson(L=8, seed=3, nleft=3):
    H = w.anderson_3d(L, 2.0, seed=seed)
    Hs = H.to_scipy()
    b = w.gaussian_unit(H.m, seed + 2)
    left = np.stack([w.gaussian_unit(H.m, seed + 3 + i) for i in range(nleft)])
    return Hs, b, left


def _dense_proj(Hs, b, left, z):
    Hd = Hs.toarray()
    M = b.size
    X = np.stack([np.linalg.solve(zk * np.eye(M) - Hd, b) for zk in z])
    ev = np.linalg.eigvalsh(Hd)
    dist = np.array([np.abs(zk - ev).min() for zk in z])
    return X @ np.vstack([b, left]).T, dist


def test_replay_equals_combined_run_without_switching():
    Hs, b, left = _anderson()
    zA = np.concatenate([[0.01 + 0.05j], w.shiftk_grid(-8, 8, 32, 0.05)])   # seed near the band centre
    zB = w.shiftk_grid(-8, 8, 20, 0.2) + 0.1
    r = oc.shifted_cocg(Hs, b, zA, left=left, tol=1e-10, full=False, seed_switch=False, log=True)
    rab = oc.shifted_cocg(Hs, b, np.concatenate([zA, zB]), left=left, tol=1e-10, full=False, seed_switch=False)
    assert r.status == oc.STATUS_OK and rab.iters == r.iters
    rc = orc_mod.recalc(r.log, zB)
    assert rc.converged
    np.testing.assert_array_equal(rc.conv_iter, rab.conv_iter[zA.size:])
    assert np.abs(rc.proj - rab.proj[zA.size:]).max() <= 1e-14 * np.abs(rab.proj).max()


@pytest.mark.parametrize("delta", [0.05, 0.2])
def test_replay_matches_dense_definition_with_switching(delta):
    Hs, b, left = _anderson()
    zA = w.shiftk_grid(-8, 8, 32, delta)
    zB = zA + 0.25 + 0.01j          # midpoints, slightly further from the axis
    r = oc.shifted_cocg(Hs, b, zA, left=left, tol=1e-10, full=False, log=True)
    assert r.status == oc.STATUS_OK and r.n_seed_switch > 0
    rc = orc_mod.recalc(r.log, zB)
    # a shift that was not in the run need not freeze within it; the bound
    # below uses its last residual estimate either way
    assert np.all(rc.final_res <= 1e-6)
    ref, dist = _dense_proj(Hs, b, left, zB)
    norms = np.linalg.norm(np.vstack([b, left]), axis=1)
    bound = 2.0 * rc.final_res[:, None] * norms[None, :] / dist[:, None] + 1e-13
    assert np.all(np.abs(rc.proj - ref) <= bound)


def test_replay_of_own_shifts_reproduces_run():
    Hs, b, left = _anderson(L=7, seed=8)
    z = w.shiftk_grid(-8, 8, 48, 0.05)
    r = oc.shifted_cocg(Hs, b, z, left=left, tol=1e-10, full=False, log=True)
    rc = orc_mod.recalc(r.log, z)
    np.testing.assert_array_equal(rc.conv_iter, r.conv_iter)
    assert np.abs(rc.proj - r.proj).max() <= 1e-12 * np.abs(r.proj).max()


def test_large_shift_moment_expansion():
    Hs, b, left = _anderson(L=6, seed=11)
    z = np.array([1e3j, -1e3j, 1e3 + 1e3j])
    r = oc.shifted_cocg(Hs, b, w.shiftk_grid(-8, 8, 16, 0.1), left=left, tol=1e-12, full=False, log=True)
    rc = orc_mod.recalc(r.log, z)
    hb = Hs @ b
    m1, m2 = b @ hb, hb @ hb
    series = 1 / z + m1 / z ** 2 + m2 / z ** 3
    hnorm = np.abs(Hs).sum(axis=1).max()                 # ||H||_inf bounds the spectral radius
    assert np.all(np.abs(rc.proj[:, 0] - series) <= 2 * hnorm ** 3 / np.abs(z) ** 4 + 1e-15)


@pytest.mark.parametrize("n", [0, 1, 7, 40])
def test_truncated_log_replays_stopped_run(n):
    Hs, b, left = _anderson(L=6, seed=4)
    z = w.shiftk_grid(-8, 8, 24, 0.05)
    r = oc.shifted_cocg(Hs, b, z, left=left, tol=1e-10, full=False, log=True)
    rn = oc.shifted_cocg(Hs, b, z, left=left, tol=1e-10, full=False, maxiter=n)
    lg = r.log
    cut = oc.KrylovLog(zs=lg.zs[:n], alpha=lg.alpha[:n], c=lg.c[:n], beta=lg.beta[:n], nu=lg.nu[:n],
                       pj1=lg.pj1[:n], pj0=lg.pj0[:n], w=lg.w[:n], w0=lg.w0, thresh=lg.thresh)
    rc = orc_mod.recalc(cut, z)
    assert not rc.converged
    np.testing.assert_array_equal(rc.conv_iter, rn.conv_iter)
    assert np.abs(rc.proj - rn.proj).max() <= 1e-12 * max(np.abs(rn.proj).max(), 1e-300)


# ---------------------------------------------------------------- planted mistakes
SRC = open(orc_mod.__file__).read()
MUTATIONS = {
    "no_switch_rescale": ("            pi[active] = pi[active] / log.pj1[n]\n"
                          "            pi_old[active] = pi_old[active] / log.pj0[n]\n",
                          "            pass\n"),
    "w_index": ("U[k] = log.w[n][None, :]", "U[k] = log.w[max(n - 1, 0)][None, :]"),
    "c_sign": ("* pi[k] - c * pi_old[k]", "* pi[k] + c * pi_old[k]"),
    "seed_shift": ("(z[k] - log.zs[n])", "(z[k] - log.zs[0])"),
}


def _mutant(name):
    old, new = MUTATIONS[name]
    assert SRC.count(old) == 1, name
    mod = types.ModuleType("recalc_mutant_" + name)
    sys.modules[mod.__name__] = mod
    try:
        exec(compile(SRC.replace(old, new), mod.__name__, "exec"), mod.__dict__)
    finally:
        del sys.modules[mod.__name__]
    return mod


def _dense_pin_passes(mod):
    Hs, b, left = _anderson(L=6, seed=9)
    zA = w.shiftk_grid(-8, 8, 24, 0.05)
    zB = zA + 0.3 + 0.15j          # midpoints further from the axis: they freeze within the run
    r = oc.shifted_cocg(Hs, b, zA, left=left, tol=1e-10, full=False, log=True)
    with np.errstate(all="ignore"):
        rc = mod.recalc(r.log, zB)
    ref, dist = _dense_proj(Hs, b, left, zB)
    norms = np.linalg.norm(np.vstack([b, left]), axis=1)
    bound = 2.0 * rc.final_res[:, None] * norms[None, :] / dist[:, None] + 1e-13
    return bool(rc.converged and np.all(np.isfinite(rc.proj)) and np.all(rc.final_res <= 1e-9)
                and np.all(np.abs(rc.proj - ref) <= bound))


def test_dense_pin_accepts_the_oracle():
    assert _dense_pin_passes(orc_mod)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_dense_pin_rejects_planted_mistake(name):
    assert not _dense_pin_passes(_mutant(name))
