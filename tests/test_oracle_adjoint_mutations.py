"""The adjoint oracle's pins must catch plausible mistakes.

Each case plants one mistake into a copy of oracle/adjoint.py (a conjugated
bilinear form, a lost sign or 1/pi, the wrong solution in the a != b form, a
missing residual weight in the loss gradient, the left vector's solve replaced
by b's), loads the copy as a module of its own and checks that the pins
reject it: the derivatives against the explicit inverse, -(1/pi) Im b^T G H_m G b
and a^T G H_m G b, and the loss gradient against its definition
sum_k (A_k - A*_k) dA_k/dtheta.  The real oracle is never modified.
"""
import sys
import types

import numpy as np
import pytest

import oracle.adjoint as oa_mod
from paper_2001_08707_gb300 import workloads as w

SRC = open(oa_mod.__file__).read()

MUTATIONS = {
    "conjugated_form": ("dA[:, m] = -np.imag(np.sum(X * HX, axis=1)) / np.pi",
                        "dA[:, m] = -np.imag(np.sum(np.conj(X) * HX, axis=1)) / np.pi"),
    "lost_sign": ("dA[:, m] = -np.imag(np.sum(X * HX, axis=1)) / np.pi",
                  "dA[:, m] = np.imag(np.sum(X * HX, axis=1)) / np.pi"),
    "lost_pi": ("dA[:, m] = -np.imag(np.sum(X * HX, axis=1)) / np.pi",
                "dA[:, m] = -np.imag(np.sum(X * HX, axis=1))"),
    "unweighted_loss_gradient": ("return A, 0.5 * float(res @ res), dA.T @ res, dA",
                                 "return A, 0.5 * float(res @ res), dA.sum(axis=0), dA"),
    "x_for_y": ("dG[:, m] = np.sum(Y * HX, axis=1)", "dG[:, m] = np.sum(X * HX, axis=1)"),
    "left_solve_with_b": ("Y = X if a is b else shifted_cocg(H, a, z, tol=tol, full=True, maxiter=maxiter).x",
                          "Y = X if a is b else shifted_cocg(H, b, z, tol=tol, full=True, maxiter=maxiter).x"),
    "green_conjugated": ("G = np.sum(X * a[None, :], axis=1)", "G = np.sum(np.conj(X) * a[None, :], axis=1)"),
}


def _exec_module(modname, source):
    mod = types.ModuleType(modname)
    sys.modules[modname] = mod
    try:
        exec(compile(source, f"<{modname}>", "exec"), mod.__dict__)
    finally:
        del sys.modules[modname]
    return mod


def _pins_pass(mod):
    j = w.j1j2_chain(8, 1.0, 0.4, 0.2, seed=3)
    terms = [t.to_scipy() for t in j.terms]
    M = j.terms[0].m
    b = w.gaussian_unit(M, 3)
    a = w.gaussian_unit(M, 4, w.STREAM_LEFT)
    z = w.shiftk_grid(-3.0, 2.0, 6, 0.2)
    rng = np.random.default_rng(1)
    target = rng.normal(0.0, 0.1, z.size)
    A, _, grad, dA = mod.spectrum_and_gradient(terms, j.theta, b, z, target, tol=1e-13)
    H = mod.assemble(terms, j.theta).toarray()
    Gs = [np.linalg.inv(zk * np.eye(M) - H) for zk in z]
    for k in range(z.size):
        for m, Hm in enumerate(terms):
            ref = -np.imag(b @ Gs[k] @ Hm.toarray() @ Gs[k] @ b) / np.pi
            if abs(dA[k, m] - ref) > 1e-9 * (1 + abs(ref)):
                return False
    A_ref = np.array([-np.imag(b @ G @ b) / np.pi for G in Gs])
    if np.abs(A - A_ref).max() > 1e-9:
        return False
    if np.abs(grad - dA.T @ (A_ref - target)).max() > 1e-9 * (1 + np.abs(grad).max()):
        return False
    G_ab, dG = mod.green_and_gradient(terms, j.theta, a, b, z, tol=1e-13)
    for k in range(z.size):
        if abs(G_ab[k] - a @ Gs[k] @ b) > 1e-9:
            return False
        for m, Hm in enumerate(terms):
            ref = a @ Gs[k] @ Hm.toarray() @ Gs[k] @ b
            if abs(dG[k, m] - ref) > 1e-9 * (1 + abs(ref)):
                return False
    return True


def test_pins_accept_the_oracle():
    assert _pins_pass(_exec_module("oracle_adjoint_copy", SRC))


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_reject_planted_mistake(name):
    old, new = MUTATIONS[name]
    assert SRC.count(old) == 1, name
    assert not _pins_pass(_exec_module(f"oracle_adjoint_mutant_{name}", SRC.replace(old, new)))
