"""GPU checks of the hand-written adjoint (kw_bilinear + GreenSpectrum).

d A_k / d theta_t = -(1/pi) Im(x_k^T H_t x_k) (from dG/dtheta = G H_t G,
G^T = G).  Checked against numpy bilinear forms, the oracle gradient (reduced
size) and central differences of the GPU's own forward solves (full size:
J1-J2 chain N=20, M=184,756, 22 parameters, K=256 shifts at delta=0.05)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import adjoint as oa
from paper_2001_08707_gb300 import adjoint
from paper_2001_08707_gb300 import komega as kw
from paper_2001_08707_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2001_08707_gb300 import build

    build.build()


def test_bilinear_matches_numpy():
    j = w.j1j2_chain(10, 1.0, 0.4, 0.2, seed=2)
    m = j.terms[0].m
    rng = np.random.default_rng(3)
    K = 13                                       # not a multiple of the shift tile
    X = rng.standard_normal((K, m)) + 1j * rng.standard_normal((K, m))
    Y = rng.standard_normal((K, m)) + 1j * rng.standard_normal((K, m))
    s = kw.Solver("f64")
    ts = adjoint.TermSet(j.terms)
    Xd, Yd = torch.as_tensor(X, device="cuda"), torch.as_tensor(Y, device="cuda")
    for y_is_x in (True, False):
        out = s.bilinear(ts.device_terms, Xd, None if y_is_x else Yd)
        YY = X if y_is_x else Y
        ref = np.stack([np.sum(YY * (t.to_scipy() @ X.T).T, axis=1) for t in j.terms], axis=1)
        np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def _problem(N, K, seed=w.SEED_BASE + 3):
    j = w.j1j2_chain(N, 1.0, 0.4, 0.2, seed=seed)
    lo, hi = w.chain_bounds(j.assemble())
    z = w.shiftk_grid(lo - 0.5, hi + 0.5, K, 0.05)
    b = w.gaussian_unit(j.terms[0].m, seed)
    rng = np.random.default_rng([seed, w.STREAM_PERTURB])
    theta_star = j.theta + rng.normal(0.0, 0.05, j.theta.size)
    return j, z, b, theta_star


@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_gradient_matches_oracle(prec):
    j, z, b, theta_star = _problem(12, 32)
    terms = [t.to_scipy() for t in j.terms]
    target = oa.spectrum(terms, theta_star, b, z, tol=1e-12)[0]
    A_o, loss_o, grad_o, _ = oa.spectrum_and_gradient(terms, j.theta, b, z, target, tol=1e-12)
    model = adjoint.GreenSpectrum(j.terms, b, z, prec=prec, tol=1e-12)
    theta = torch.tensor(j.theta, dtype=torch.float64, requires_grad=True)
    A = model(theta)
    loss = 0.5 * torch.sum((A - torch.as_tensor(target)) ** 2)
    loss.backward()
    np.testing.assert_allclose(A.detach().numpy(), A_o, rtol=0, atol=1e-10 * np.abs(A_o).max())
    g = theta.grad.numpy()
    assert np.abs(g - grad_o).max() <= 1e-8 * np.abs(grad_o).max(), (g, grad_o)


def test_gradcheck_tiny_chain():
    """torch.autograd.gradcheck of the spectrum A(theta) (every output, every
    parameter) on a J1-J2 chain N=8 (M=70, 10 parameters), 6 shifts: the
    hand-written backward against torch's central differences of the forward
    solves (converged to 1e-13, so the difference noise is ~1e-13/eps)."""
    j, z, b, _ = _problem(8, 6)
    model = adjoint.GreenSpectrum(j.terms, b, z, prec="f64", tol=1e-13)
    theta = torch.tensor(j.theta, dtype=torch.float64, requires_grad=True)
    assert torch.autograd.gradcheck(lambda th: model(th), (theta,), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_fullsize_gradient_vs_central_differences():
    """J1-J2 N=20 with 22 parameters, K=256 shifts: adjoint gradient of the
    quadratic spectrum loss against central differences (step 1e-5) of the GPU's
    own forward solves for J1, J2 and two site fields."""
    j, z, b, theta_star = _problem(20, 256)
    assert j.terms[0].m == 184756 and len(j.terms) == 22
    model = adjoint.GreenSpectrum(j.terms, b, z, prec="df64", tol=1e-12)
    target = model.solve(theta_star)[0]
    theta = torch.tensor(j.theta, dtype=torch.float64, requires_grad=True)
    A = model(theta)
    loss = 0.5 * torch.sum((A - torch.as_tensor(target)) ** 2)
    loss.backward()
    g = theta.grad.numpy()
    h = 1e-5
    for t in (0, 1, 2, 11):
        e = np.zeros(j.theta.size)
        e[t] = h
        lp = 0.5 * np.sum((model.solve(j.theta + e)[0] - target) ** 2)
        lm = 0.5 * np.sum((model.solve(j.theta - e)[0] - target) ** 2)
        fd = (lp - lm) / (2 * h)
        print(f"param {t}: adjoint {g[t]:.10e} central difference {fd:.10e}")
        assert abs(fd - g[t]) <= 1e-5 * abs(g[t]) + 1e-9


def test_bilinear_c64_matches_numpy():
    """kw_bilinear_c64: complex FP32 X and Y widened to FP64, FP64 sums."""
    j = w.j1j2_chain(10, 1.0, 0.4, 0.2, seed=2)
    m = j.terms[0].m
    rng = np.random.default_rng(4)
    K = 11
    X = (rng.standard_normal((K, m)) + 1j * rng.standard_normal((K, m))).astype(np.complex64)
    Y = (rng.standard_normal((K, m)) + 1j * rng.standard_normal((K, m))).astype(np.complex64)
    s = kw.Solver("f64")
    ts = adjoint.TermSet(j.terms)
    Xd, Yd = torch.as_tensor(X, device="cuda"), torch.as_tensor(Y, device="cuda")
    X64, Y64 = X.astype(np.complex128), Y.astype(np.complex128)
    for y_is_x in (True, False):
        out = s.bilinear(ts.device_terms, Xd, None if y_is_x else Yd)
        YY = X64 if y_is_x else Y64
        ref = np.stack([np.sum(YY * (t.to_scipy() @ X64.T).T, axis=1) for t in j.terms], axis=1)
        np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    with pytest.raises(ValueError):
        s.bilinear(ts.device_terms, Xd, Yd.to(torch.complex128))


@pytest.mark.parametrize("form", ["f64", "df64", "df64+x32"])
def test_green_a_ne_b_gradient_matches_oracle(form):
    """d(a^T G b)/dtheta for a left vector a different from b (second solve with
    rhs a) against the oracle's two solves, through a real loss on the complex
    G_ab.  With FP32 shift storage the stored x_k, y_k carry FP32 error, so the
    gradient is compared at 1e-5 (the values still come from the FP64-class
    recurrences)."""
    j, z, b, theta_star = _problem(12, 24)
    terms = [t.to_scipy() for t in j.terms]
    a = w.gaussian_unit(j.terms[0].m, 13, w.STREAM_LEFT)
    G_star, _ = oa.green_and_gradient(terms, theta_star, a, b, z, tol=1e-12)
    G_o, dG_o = oa.green_and_gradient(terms, j.theta, a, b, z, tol=1e-12)
    grad_o = np.real(np.conj(2 * (G_o - G_star)) @ dG_o)     # L = sum |G - G*|^2
    prec = form.split("+")[0]
    model = adjoint.GreenBilinear(j.terms, b, z, a=a, prec=prec, tol=1e-12, shift_fp32=form.endswith("x32"))
    theta = torch.tensor(j.theta, dtype=torch.float64, requires_grad=True)
    G = model(theta)
    loss = torch.sum(torch.abs(G - torch.as_tensor(G_star)) ** 2)
    loss.backward()
    np.testing.assert_allclose(G.detach().numpy(), G_o, rtol=0, atol=1e-10 * np.abs(G_o).max())
    g = theta.grad.numpy()
    tol = 1e-5 if form.endswith("x32") else 1e-8
    print(f"{form}: max gradient error {np.abs(g - grad_o).max() / np.abs(grad_o).max():.2e}")
    assert np.abs(g - grad_o).max() <= tol * np.abs(grad_o).max(), (g, grad_o)


def test_green_a_ne_b_gradcheck_tiny():
    """gradcheck of the complex outputs G_ab(theta) (a != b) on N=8, 5 shifts."""
    j, z, b, _ = _problem(8, 5)
    a = w.gaussian_unit(j.terms[0].m, 17, w.STREAM_LEFT)
    model = adjoint.GreenBilinear(j.terms, b, z, a=a, prec="f64", tol=1e-13)
    theta = torch.tensor(j.theta, dtype=torch.float64, requires_grad=True)
    assert torch.autograd.gradcheck(lambda th: model(th), (theta,), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_spectrum_gradient_with_fp32_shift_storage():
    """GreenSpectrum with FP32 x/p storage: the spectrum keeps the FP64-class
    agreement (projected recurrences), the gradient agrees at FP32 level."""
    j, z, b, theta_star = _problem(12, 32)
    terms = [t.to_scipy() for t in j.terms]
    target = oa.spectrum(terms, theta_star, b, z, tol=1e-12)[0]
    A_o, _, grad_o, _ = oa.spectrum_and_gradient(terms, j.theta, b, z, target, tol=1e-12)
    model = adjoint.GreenSpectrum(j.terms, b, z, prec="df64", tol=1e-12, shift_fp32=True)
    theta = torch.tensor(j.theta, dtype=torch.float64, requires_grad=True)
    A = model(theta)
    loss = 0.5 * torch.sum((A - torch.as_tensor(target)) ** 2)
    loss.backward()
    np.testing.assert_allclose(A.detach().numpy(), A_o, rtol=0, atol=1e-10 * np.abs(A_o).max())
    g = theta.grad.numpy()
    print(f"max gradient error {np.abs(g - grad_o).max() / np.abs(grad_o).max():.2e}")
    assert np.abs(g - grad_o).max() <= 1e-5 * np.abs(grad_o).max()


def _csr_dev(A):
    A = A.tocsr()
    return (torch.as_tensor(A.indptr.astype(np.int64), device="cuda"),
            torch.as_tensor(A.indices.astype(np.int32), device="cuda"),
            torch.as_tensor(A.data.astype(np.float64), device="cuda"))


@pytest.mark.parametrize("dtype", [np.complex128, np.complex64])
def test_bilinear_diagonal_path_edge_terms(dtype):
    """kw_bilinear finds the terms whose rows hold at most one entry, on the
    diagonal, and sums up to 16 of them in one pass over X and Y.  Mixed here:
    19 diagonal terms (two groups) with empty rows, a term with one entry off
    the diagonal, a term with a diagonal entry stored twice in one row, an
    empty term (nnz 0) and a general term, at a ragged shift count; against
    numpy's y_k^T H_t x_k, with Y = X and Y given."""
    sp = pytest.importorskip("scipy.sparse")
    rng = np.random.default_rng(8)
    m, K = 1031, 19
    terms = []
    for t in range(19):
        dvals = rng.standard_normal(m)
        dvals[rng.random(m) < 0.2] = 0.0
        terms.append(sp.diags(dvals).tocsr())
        terms[-1].eliminate_zeros()                     # some rows empty
    off = sp.diags(rng.standard_normal(m)).tolil()
    off[5, 9] = 0.75                                   # one entry off the diagonal
    terms.insert(3, off.tocsr())
    dup = sp.diags(rng.standard_normal(m)).tocsr()
    r0 = dup.indptr[7]
    dup = sp.csr_matrix((np.insert(dup.data, r0, 0.5), np.insert(dup.indices, r0, 7),
                         np.concatenate([dup.indptr[:8], dup.indptr[8:] + 1])), shape=(m, m))
    assert dup.indptr[8] - dup.indptr[7] == 2 and not dup.has_canonical_format
    terms.insert(11, dup)                              # (7, 7) stored twice
    terms.append(sp.csr_matrix((m, m)))                # empty
    terms.append(sp.random(m, m, density=0.01, random_state=3, format="csr"))
    X = (rng.standard_normal((K, m)) + 1j * rng.standard_normal((K, m))).astype(dtype)
    Y = (rng.standard_normal((K, m)) + 1j * rng.standard_normal((K, m))).astype(dtype)
    Xd, Yd = torch.as_tensor(X, device="cuda"), torch.as_tensor(Y, device="cuda")
    dev = [_csr_dev(A) for A in terms]
    s = kw.Solver("f64")
    X64, Y64 = X.astype(np.complex128), Y.astype(np.complex128)
    for y_is_x in (True, False):
        out = s.bilinear(dev, Xd, None if y_is_x else Yd)
        YY = X64 if y_is_x else Y64
        ref = np.stack([np.sum(YY * (A @ X64.T).T, axis=1) for A in terms], axis=1)
        np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
