"""fosb_getrf_static -- the LU entry point that allocates no device memory -- against
the allocating entry point (fosb_factor + fosb_solve) on the same matrices.

Callers that cannot allocate (hosts whose own allocator owns the device memory, or that
forbid allocation after start-up) factor in place with fosb_getrf_static; its factors
must give the same solutions as fosb_factor's, at the tolerance of the other parity
tests (1e-8 for complex128, 1e-4 for complex64), on two calls in a row that share the
static scratch array.  Collected last so a failure here stops a -x run only after all
other tests ran."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_01457_gb300 as mod

    mod.build.build()
    L = mod.lib()
    L.fosb_getrf_static.restype = ctypes.c_int
    return mod


def _lu_solve_host(lu, piv, b):
    """Solve with packed factors (unit-lower L below the diagonal, U on and above) and
    LAPACK-order row interchanges, on the host."""
    from scipy.linalg import solve_triangular

    x = b.copy()
    for i, p in enumerate(piv):
        if p != i:
            x[[i, p]] = x[[p, i]]
    y = solve_triangular(lu, x, lower=True, unit_diagonal=True)
    return solve_triangular(lu, y, lower=False)


def _static_factor(F, A, prec):
    n = A.shape[0]
    piv = torch.full((n,), -1, dtype=torch.int32, device=A.device)
    st = F.lib().fosb_getrf_static(ctypes.c_void_p(A.data_ptr()), ctypes.c_int64(n), ctypes.c_int64(A.stride(0)),
                                   ctypes.c_int(prec), ctypes.c_void_p(piv.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, F.lib().fosb_last_error().decode()
    return A, piv.cpu().numpy()


def _matrices(F):
    import fosb_synth as S

    sm = S.icosphere(2)
    m = F.mesh_create(sm.verts, sm.tris, sm.vnormals)
    Z = torch.zeros((m.n_edges, m.n_edges), dtype=torch.complex128, device="cuda")
    F.assemble_efie(m, 3.0, Z)
    rng = np.random.default_rng(11)
    R = rng.standard_normal((300, 300)) + 1j * rng.standard_normal((300, 300))  # ragged: 4 panels + 44
    return [Z, torch.tensor(R, dtype=torch.complex128, device="cuda")]


@pytest.mark.parametrize("prec_name,tol", [("FP64", 1e-8), ("FP32", 1e-4)])
def test_static_lu_matches_allocating_entry_point(F, prec_name, tol):
    prec = getattr(F, prec_name)
    dt = torch.complex128 if prec == F.FP64 else torch.complex64
    rng = np.random.default_rng(5)
    for call, A0 in enumerate(_matrices(F) * 2):  # two calls in a row on each matrix
        A = A0.to(dt)
        n = A.shape[0]
        bh = rng.standard_normal((n, 2)) + 1j * rng.standard_normal((n, 2))
        b = torch.tensor(bh, dtype=dt, device="cuda")
        lu_ref = F.factor(A.clone(), prec=prec)
        x_ref = torch.zeros_like(b)
        F.solve(lu_ref, b, x_ref)
        x_ref = x_ref.cpu().numpy().astype(np.complex128)
        lu, piv = _static_factor(F, A.clone(), prec)
        assert piv.min() >= 0 and np.all(piv >= np.arange(n)) and piv.max() < n
        x = _lu_solve_host(lu.cpu().numpy().astype(np.complex128), piv, bh)
        assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < tol, call


def test_static_lu_rejects_sizes_beyond_its_scratch(F):
    A = torch.zeros((2, 2), dtype=torch.complex128, device="cuda")
    piv = torch.zeros(2, dtype=torch.int32, device="cuda")
    # the limit: min(SM count, 256) panel CTAs of at most 2048 rows (311,296 on 152 SMs)
    n_max = min(torch.cuda.get_device_properties(0).multi_processor_count, 256) * 2048
    for n in (n_max + 1, 524288 + 1):
        st = F.lib().fosb_getrf_static(ctypes.c_void_p(A.data_ptr()), ctypes.c_int64(n), ctypes.c_int64(n),
                                       ctypes.c_int(F.FP64), ctypes.c_void_p(piv.data_ptr()), None)
        assert st == F.FOSB_ERR_INVALID_ARG
        assert f"exceeds the limit {n_max}".encode() in F.lib().fosb_last_error()
