"""CPU reproduction of the FP32-vector stall at small delta.

The FP32-vector form stores the seed vectors r and q in complex FP32 while every
scalar stays FP64.  A copy of the oracle in which q and r_{n+1} are rounded to
complex FP32 after each step (FP64 arithmetic otherwise; the real oracle is not
modified) shows the same behaviour on the Heisenberg chain N=14 at delta=0.01:
the seed switches keep the seed at the slowest mid-spectrum shift, where the
unconjugated rho = r^T r cancels (|r^T r| / ||r||^2 near 1e-4), so FP32 storage
leaves rho with few correct digits and the seed residual stalls; shifts stay
unconverged at 1.5x the FP64 iteration count and the spectrum error sits far
above 1e-6.  At delta=0.05 the same emulation converges with a small spectrum
error.  This is the reason the FP32 storage is applied to the shifted x/p
(kw_set_shift_storage) and not to the seed recurrence.
"""
import sys
import types

import numpy as np

import oracle.shifted_cocg as oc_mod
from paper_2001_08707_gb300 import workloads as w

SRC = open(oc_mod.__file__).read()
ROUND = ".astype(np.complex64).astype(np.complex128)"


def _fp32_storage_oracle():
    src = SRC
    for old in ("q = z[s] * r - _matvec(H, r)", "r_new = (1.0 + c) * r - alpha * q - c * r_old"):
        assert src.count(old) == 1, old
        lhs, rhs = old.split(" = ", 1)
        src = src.replace(old, f"{lhs} = ({rhs}){ROUND}")
    mod = types.ModuleType("oracle_fp32_storage")
    sys.modules["oracle_fp32_storage"] = mod
    try:
        exec(compile(src, "<oracle_fp32_storage>", "exec"), mod.__dict__)
    finally:
        del sys.modules["oracle_fp32_storage"]
    return mod


def _spectrum(proj):
    return -np.imag(proj[:, 0]) / np.pi


def test_fp32_seed_storage_stalls_at_delta_0_01():
    p = w.heisenberg_projected(N=14, K=96, delta=0.01, tol=1e-10)
    Hs = p.H.to_scipy()
    ref = oc_mod.shifted_cocg(Hs, p.b, p.z, tol=p.tol, full=False)
    assert ref.status == oc_mod.STATUS_OK
    emu = _fp32_storage_oracle()
    cap = int(1.5 * ref.iters)
    r32 = emu.shifted_cocg(Hs, p.b, p.z, tol=p.tol, full=False, maxiter=cap)
    unconverged = int(np.sum(r32.conv_iter < 0))
    err = np.abs(_spectrum(r32.proj) - _spectrum(ref.proj)).max() / np.abs(_spectrum(ref.proj)).max()
    print(f"FP64 {ref.iters} iterations; FP32 storage: {unconverged} of {p.z.size} shifts unconverged "
          f"after {r32.iters}, spectrum error {err:.1e}")
    assert r32.status != oc_mod.STATUS_OK and unconverged > 0
    assert err > 1e-6


def test_fp32_seed_storage_converges_at_delta_0_05():
    p = w.heisenberg_projected(N=12, K=48, delta=0.05, tol=1e-6)
    Hs = p.H.to_scipy()
    ref = oc_mod.shifted_cocg(Hs, p.b, p.z, tol=1e-10, full=False)
    r32 = _fp32_storage_oracle().shifted_cocg(Hs, p.b, p.z, tol=p.tol, full=False, maxiter=4 * ref.iters)
    assert r32.status == oc_mod.STATUS_OK
    err = np.abs(_spectrum(r32.proj) - _spectrum(ref.proj)).max() / np.abs(_spectrum(ref.proj)).max()
    assert err < 1e-5
