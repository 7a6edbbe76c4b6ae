"""kw_spmv_dot_noalloc, the entry point for callers that cannot allocate GPU
memory (their device memory is owned by another allocator, or they cannot
afford cudaMalloc's implicit synchronisation), against kw_spmv_dot.

The file name makes pytest collect it last.  It passes on its own in a fresh
process (the first call on the device does the set-up) and after the other
tests.  Two calls in a row check that the shared static scratch is cleared
where it must start at zero.
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


@pytest.mark.parametrize("case", ["heisenberg_N14", "ragged_anderson_L9"])
def test_noalloc_matches_allocating_entry_point_twice(case):
    H = w.heisenberg_chain(14) if case == "heisenberg_N14" else w.anderson_3d(9, 3.0, seed=21)
    s = kw.Solver("f64")
    s.set_csr(H.rowptr, H.col, H.val)
    rp = torch.as_tensor(H.rowptr, device="cuda")
    cl = torch.as_tensor(H.col, device="cuda")
    vl = torch.as_tensor(H.val, device="cuda")
    rng = np.random.default_rng(31)
    for call, zs in enumerate((0.4 - 0.9j, -1.3 + 0.05j)):
        r = torch.as_tensor(rng.standard_normal(H.m) + 1j * rng.standard_normal(H.m), device="cuda")
        q_ref = torch.empty_like(r)
        t_ref = s.spmv_dot(zs, r, q_ref)
        q = torch.full_like(r, float("nan"))
        t = kw.spmv_dot_noalloc(rp, cl, vl, zs, r, q)
        qr = q_ref.cpu().numpy()
        np.testing.assert_allclose(q.cpu().numpy(), qr, rtol=0, atol=1e-13 * np.abs(qr).max())
        assert abs(t - t_ref) <= 1e-12 * np.sum(np.abs(r.cpu().numpy() * qr)), (call, t, t_ref)
        # and against the product formed on the host from the CSR arrays (scipy)
        rh = r.cpu().numpy()
        q_host = zs * rh - H.to_scipy() @ rh
        scale = np.abs(zs) * np.abs(rh) + abs(H.to_scipy()) @ np.abs(rh)
        np.testing.assert_array_less(np.abs(q.cpu().numpy() - q_host), 1e-14 * scale.max() + 1e-300)
        t_host = np.sum(rh * q_host)
        assert abs(t - t_host) <= 1e-13 * np.sum(np.abs(rh) * scale), (call, t, t_host)


def test_noalloc_rejects_bad_sizes():
    r = torch.zeros(4, dtype=torch.complex128, device="cuda")
    rp = torch.zeros(5, dtype=torch.int64, device="cuda")
    cl = torch.zeros(0, dtype=torch.int32, device="cuda")
    vl = torch.zeros(0, dtype=torch.float64, device="cuda")
    lib = kw.load_library()
    t = kw.kw_c128()
    import ctypes as C
    bad_m = lib.kw_spmv_dot_noalloc(1 << 31, 0, C.c_void_p(rp.data_ptr()), None, None, kw.kw_c128(0, 0),
                                    C.c_void_p(r.data_ptr()), C.c_void_p(r.data_ptr()), C.byref(t), None)
    assert bad_m == kw.KW_ERR_ARG
    assert lib.kw_spmv_dot_noalloc(4, 0, None, None, None, kw.kw_c128(0, 0), C.c_void_p(r.data_ptr()),
                                   C.c_void_p(r.data_ptr()), C.byref(t), None) == kw.KW_ERR_ARG
    # an empty operator is fine: q = zs r
    q = torch.empty_like(r)
    r.fill_(1.0)
    assert kw.spmv_dot_noalloc(rp, cl, vl, 2.0 + 0j, r, q) == 8.0
    assert torch.all(q == 2.0)


def test_noalloc_binding_rejects_mismatched_tensors():
    """The binding checks types, devices and lengths before the library sees a
    bare pointer: a short q, an int32 rowptr, val and col of different lengths
    or a complex64 r raise ValueError on the host."""
    H = w.anderson_3d(4, 2.0, seed=5)
    rp = torch.as_tensor(H.rowptr, device="cuda")
    cl = torch.as_tensor(H.col, device="cuda")
    vl = torch.as_tensor(H.val, device="cuda")
    r = torch.ones(H.m, dtype=torch.complex128, device="cuda")
    q = torch.empty_like(r)
    with pytest.raises(ValueError):
        kw.spmv_dot_noalloc(rp, cl, vl, 1j, r, q[:-1])
    with pytest.raises(ValueError):
        kw.spmv_dot_noalloc(rp.to(torch.int32), cl, vl, 1j, r, q)
    with pytest.raises(ValueError):
        kw.spmv_dot_noalloc(rp, cl, vl[:-1], 1j, r, q)
    with pytest.raises(ValueError):
        kw.spmv_dot_noalloc(rp, cl, vl, 1j, r.to(torch.complex64), q)
    with pytest.raises(ValueError):
        kw.spmv_dot_noalloc(rp, cl, vl, 1j, r.cpu(), q)
    # the well-formed call still works after the refusals
    kw.spmv_dot_noalloc(rp, cl, vl, 1j, r, q)
    np.testing.assert_allclose(q.cpu().numpy(), 1j - H.to_scipy() @ np.ones(H.m), atol=1e-14)
