"""GPU: the device-side iteration loop (kw_options.use_graph).

With use_graph the iterations run as the body of a CUDA graph WHILE node that
repeats until the device stop flag is raised; without it the host enqueues
them in chunks and polls the flag.  The kernels, their launch shapes and their
order are the same, so every output must agree bit for bit with the host loop:
in all three forms, projected and full, with seed switches, at an iteration
cap that is not a multiple of the chunk, after a resume, when the captured
graph is reused or recaptured, and for batched solves.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import shifted_cocg as oc
from paper_2001_08707_gb300 import komega as kw
from paper_2001_08707_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2001_08707_gb300 import build

    build.build()


def _problem(L=8, K=36):
    H = w.anderson_3d(L, 3.0, seed=11)
    b = w.gaussian_unit(H.m, 12)
    left = np.stack([w.gaussian_unit(H.m, 13 + i) for i in range(2)])
    z = w.shiftk_grid(-8, 8, K, 0.03)
    return H, b, left, z


def _solve(s, H, b, left, z, full):
    s.set_csr(H.rowptr, H.col, H.val)
    r = s.solve(b, z, left=left, full=full, check=False)
    ci, fr = s.shift_status(z.size)
    x = None if r.x is None else r.x.cpu().numpy()
    return r, ci, fr, x


def _same(a, b):
    ra, rb = a[0], b[0]
    assert (ra.iters, ra.status, ra.n_seed_switch, ra.updates, ra.seed) == \
        (rb.iters, rb.status, rb.n_seed_switch, rb.updates, rb.seed)
    np.testing.assert_array_equal(ra.proj, rb.proj)
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2], b[2])
    if a[3] is not None:
        np.testing.assert_array_equal(a[3], b[3])


@pytest.mark.parametrize("full", [False, True])
@pytest.mark.parametrize("prec", ["f64", "df64", "c32"])
@pytest.mark.parametrize("graph", [1, 6, 2])
def test_device_loop_matches_host_loop_bitwise(prec, full, graph):
    H, b, left, z = _problem()
    a = _solve(kw.Solver(prec, tol=1e-9, maxiter=3000, use_graph=0), H, b, left, z, full)
    g = _solve(kw.Solver(prec, tol=1e-9, maxiter=3000, use_graph=graph), H, b, left, z, full)
    assert a[0].n_seed_switch > 5
    _same(a, g)


def test_device_loop_parity_with_oracle():
    H, b, left, z = _problem(6, 20)
    s = kw.Solver("f64", tol=1e-10, use_graph=1)
    r, _, _, x = _solve(s, H, b, left, z, True)
    ref = oc.shifted_cocg(H.to_scipy(), b, z, left=left, tol=1e-10, full=True)
    # about 420 iterations on a 216-row matrix: far past the loss of orthogonality,
    # where the convergence delay depends on the rounding of every step (a change of
    # FMA contraction in the FP64 scalars moves it by tens of iterations), so the
    # count agrees within 5%; the error bound below is the parity check
    assert r.status == "KW_OK" and abs(r.iters - ref.iters) <= max(2, ref.iters // 20)
    # both stop within tol of the exact solution: |x - x*| <= tol ||b|| / dist(z, spectrum) each
    err = np.abs(x - ref.x).max(axis=1) * np.abs(z.imag)
    assert err.max() < 4e-10, err.max()


@pytest.mark.parametrize("maxiter", [37, 40, 1])
def test_iteration_cap_inside_a_trip(maxiter):
    H, b, left, z = _problem()
    a = _solve(kw.Solver("df64", tol=1e-12, maxiter=maxiter, use_graph=0), H, b, left, z, True)
    g = _solve(kw.Solver("df64", tol=1e-12, maxiter=maxiter, use_graph=1), H, b, left, z, True)
    assert g[0].status == "KW_NOT_CONVERGED" and g[0].iters == maxiter
    _same(a, g)


def test_resume_in_the_device_loop():
    H, b, left, z = _problem()
    whole = _solve(kw.Solver("f64", tol=1e-9, maxiter=3000, use_graph=1), H, b, left, z, False)
    s = kw.Solver("f64", tol=1e-9, maxiter=101, use_graph=1)
    s.set_csr(H.rowptr, H.col, H.val)
    first = s.solve(b, z, left=left, check=False)
    assert first.status == "KW_NOT_CONVERGED" and first.iters == 101   # odd: the resumed loop starts on parity 1
    r = s.resume(5000)
    assert r.iters == whole[0].iters
    np.testing.assert_array_equal(r.proj, whole[0].proj)


def test_graph_reuse_and_recapture():
    """One context: the same solve twice (the graph is relaunched), then other
    shift counts and modes (recaptured), then the first again; each equals a
    fresh context's result."""
    H, b, left, z = _problem()
    _, _, _, z2 = _problem(K=13)
    s = kw.Solver("df64", tol=1e-9, maxiter=3000, use_graph=1)
    runs = [(z, False), (z, False), (z2, False), (z2, True), (z, False)]
    for zz, full in runs:
        got = _solve(s, H, b, left, zz, full)
        ref = _solve(kw.Solver("df64", tol=1e-9, maxiter=3000, use_graph=0), H, b, left, zz, full)
        _same(got, ref)


def test_launch_count_of_the_device_loop():
    """The launch counter covers the loop's trips: (K2, K1, K3 per iteration +
    the condition per trip), so it grows with the iterations run."""
    H, b, left, z = _problem()
    s = kw.Solver("f64", tol=1e-9, maxiter=3000, use_graph=4)
    s.set_csr(H.rowptr, H.col, H.val)
    r = s.solve(b, z, left=left)
    trips = -(-r.iters // 4)
    n = s.stats()["launches"]
    assert 5 + trips * (4 * 3 + 1) <= n <= 5 + (trips + 2) * (4 * 3 + 1)


def test_timing_and_callback_use_the_host_loop():
    H, b, left, z = _problem()
    ref = _solve(kw.Solver("f64", tol=1e-9, maxiter=3000, use_graph=0), H, b, left, z, False)
    s = kw.Solver("f64", tol=1e-9, maxiter=3000, use_graph=1)
    s.set_kernel_timing(1)
    got = _solve(s, H, b, left, z, False)
    _same(got, ref)
    assert s.stats()["timed_iters"] > 0
    Hd = torch.as_tensor(H.to_scipy().toarray(), device="cuda").to(torch.complex128)

    def mv(r, q):
        q.copy_(Hd @ r)

    s2 = kw.Solver("f64", tol=1e-9, maxiter=3000, use_graph=1)
    s2.set_matvec(mv, H.m)
    r = s2.solve(b, z, left=left, check=False)
    assert abs(r.iters - ref[0].iters) <= 2 + ref[0].iters // 50   # dense product: other rounding
    np.testing.assert_allclose(r.proj, ref[0].proj, rtol=0, atol=1e-6 * np.abs(ref[0].proj).max())


def test_batched_device_loop_matches_host_loop():
    probs = w.anderson_batch(n=5, L_range=(4, 7), K_range=(5, 40), seed=78)
    batch = [{"H": p.H, "b": p.b, "z": p.z, "tol": p.tol, "full": i % 2 == 0} for i, p in enumerate(probs)]
    out = {}
    for graph in (0, 1):
        s = kw.Solver("df64", tol=1e-8, maxiter=4000, use_graph=graph)
        out[graph] = s.solve_batched(batch)
    for a, g in zip(out[0], out[1]):
        assert (a.iters, a.n_seed_switch, a.status) == (g.iters, g.n_seed_switch, g.status)
        np.testing.assert_array_equal(a.proj, g.proj)
        if a.x is not None:
            np.testing.assert_array_equal(a.x.cpu().numpy(), g.x.cpu().numpy())
