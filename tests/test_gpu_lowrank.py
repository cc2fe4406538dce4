"""Low-rank right-hand side on the GPU (Section VI, further work (ii)) against the oracle.

* fosb_kernel_lowrank with every pivot taken reproduces the kernel matrix (R^T R against
  the oracle's cov_kernel at 1e-12 of sigma^2) and, on vertices perturbed so that no two
  diagonal entries of a Schur complement tie, takes the oracle's pivots: the factor rows
  equal the oracle's pivoted_cholesky columns.
* With a tolerance over two meshes the reported trace error is the trace of
  K - R^T R formed by the oracle from the returned factor, below tol trace(K), at the
  oracle's rank.
* The low-rank CT far-field covariance and pseudo-covariance (levels 0..2, MIXED) equal the
  oracle's full ct_farfield_covariance at 1e-8 when the tolerance drops nothing of
  consequence (1e-14), and the full GPU path at 1e-9.
* At tol = 1e-3 the difference to the full covariance is positive and within
  err * sum_blocks ||G_l1||_2 ||G_l2||_F (G_l = A_l Z_l^{-1} B_l from the oracle)."""
import numpy as np
import pytest

import fosb_synth as S
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_01457_gb300 as mod

    mod.build.build()
    O.build()
    return mod


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _perturbed(level, seed):
    sm = S.icosphere(level)
    rng = np.random.default_rng(seed)
    return sm.verts + 0.01 * rng.standard_normal(sm.verts.shape), sm.tris


def test_full_factor_reproduces_kernel_and_oracle_pivots(F):
    v, t = _perturbed(1, 4)
    m = F.mesh_create(v, t)
    sig, ell = 0.7, 0.3
    R, rank, err, offs = F.kernel_lowrank([m], F.COV_MATERN32, sig, ell, tol=0.0, device=DEV)
    K = O.cov_kernel(v, v, "matern32", sig, ell)
    Rh = R.cpu().numpy()
    assert rank == v.shape[0] and offs == [0]
    assert np.abs(Rh.T @ Rh - K).max() < 1e-12 * sig**2
    L, piv, err_o = O.pivoted_cholesky(K, tol=0.0)
    assert L.shape[1] == rank
    assert np.abs(Rh.T - L).max() < 1e-10 * sig
    assert abs(err - err_o) < 1e-12 * np.trace(K)


def test_two_mesh_factor_meets_tolerance_at_oracle_rank(F):
    (v1, t1), (v2, t2) = _perturbed(1, 6), _perturbed(2, 7)
    m1, m2 = F.mesh_create(v1, t1), F.mesh_create(v2, t2)
    sig, ell, tol = 0.2, 0.5, 1e-6
    R, rank, err, offs = F.kernel_lowrank([m1, m2], F.COV_GAUSS, sig, ell, tol=tol, device=DEV)
    X = np.vstack([v1, v2])
    K = O.cov_kernel(X, X, "gauss", sig, ell)
    Rh = R.cpu().numpy()
    assert offs == [0, v1.shape[0]]
    assert err <= tol * np.trace(K)
    assert abs(err - np.trace(K - Rh.T @ Rh)) < 1e-9 * np.trace(K)
    L, _, err_o = O.pivoted_cholesky(K, tol=tol)
    assert rank == L.shape[1]
    # the cross-mesh block is the product of the two meshes' columns
    K12 = Rh[:, :v1.shape[0]].T @ Rh[:, v1.shape[0]:]
    assert np.abs(K12 - K[:v1.shape[0], v1.shape[0]:]).max() <= err * (1 + 1e-8) + 1e-15


@pytest.fixture(scope="module")
def ct_case(F):
    k, sig, ell = 1.5, 0.3, 0.6
    dirs = S.hplane_directions(7)
    meshes = [S.icosphere(l + 1) for l in range(3)]
    lev = {l: O.nominal_level(O.from_synth(sm), k, [0, 0, 1], [1, 0, 0], dirs) for l, sm in enumerate(meshes)}
    return k, sig, ell, dirs, meshes, lev


def _run(F, ct_case, tol):
    from paper_2308_01457_gb300.ct import FOSBProblem

    k, sig, ell, dirs, meshes, _ = ct_case
    prob = FOSBProblem(meshes, k, (0, 0, 1), (1, 0, 0), dirs, 0, 2, F.COV_GAUSS, sig, ell, prec=F.MIXED,
                       arith=F.ASM_FF, pseudo=True, lowrank_tol=tol).setup()
    _, cov, pcov = (x.cpu().numpy() for x in prob.run())
    out = (cov, pcov, getattr(prob, "rank", None), getattr(prob, "trace_err", None))
    prob.release()
    return out


def test_lowrank_ct_covariance_matches_oracle(F, ct_case):
    k, sig, ell, dirs, meshes, lev = ct_case
    cov, pcov, rank, err = _run(F, ct_case, 1e-14)
    cov_o = O.ct_farfield_covariance(lev, 0, 2, "gauss", sig, ell)
    pcov_o = O.ct_farfield_covariance(lev, 0, 2, "gauss", sig, ell, pseudo=True)
    assert rank < 42 + 162 + 642
    assert _rel(cov, cov_o) < 1e-8
    assert _rel(pcov, pcov_o) < 1e-8
    cov_f, pcov_f, _, _ = _run(F, ct_case, None)
    assert _rel(cov, cov_f) < 1e-9 and _rel(pcov, pcov_f) < 1e-9


def test_lowrank_truncation_error_within_bound(F, ct_case):
    k, sig, ell, dirs, meshes, lev = ct_case
    cov, _, rank, err = _run(F, ct_case, 1e-3)
    cov_f, _, _, _ = _run(F, ct_case, None)
    G = {l: lv.A @ np.linalg.solve(lv.Z, lv.B) for l, lv in lev.items()}
    bound = 0.0
    for (l1, l2), _ in O.ct_hermitian_blocks(0, 2):
        b = np.linalg.norm(G[l1], 2) * np.linalg.norm(G[l2], "fro")
        bound += 2 * b if l1 != l2 else b
    diff = np.linalg.norm(cov - cov_f)
    assert 0 < diff <= err * bound * 1.01, (diff, err * bound)
    assert rank <= 70


def test_lowrank_arguments_are_checked(F):
    m = F.mesh_create(*_perturbed(1, 1))
    with pytest.raises(F.FosbError) as ei:
        F.kernel_lowrank([m], F.COV_GAUSS, 1.0, -1.0, tol=1e-6, device=DEV)
    assert ei.value.status == F.FOSB_ERR_INVALID_ARG
    with pytest.raises(F.FosbError) as ei:
        F.kernel_lowrank([m], F.COV_GAUSS, 1.0, 0.5, tol=-1.0, device=DEV)
    assert ei.value.status == F.FOSB_ERR_INVALID_ARG


def test_lowrank_fp32_path_matches_oracle_at_fp32_accuracy(F):
    """complex64 factors without refinement: the low-rank covariance (complex64 Y) agrees
    with the oracle's full covariance at the FP32 path's 1e-4."""
    from paper_2308_01457_gb300.ct import FOSBProblem

    k, sig, ell = 1.5, 0.3, 0.6
    dirs = S.hplane_directions(7)
    meshes = [S.icosphere(l + 1) for l in range(2)]
    prob = FOSBProblem(meshes, k, (0, 0, 1), (1, 0, 0), dirs, 0, 1, F.COV_GAUSS, sig, ell, prec=F.FP32,
                       arith=F.ASM_FP32, lowrank_tol=1e-12).setup()
    _, cov = prob.run()
    assert cov.dtype == torch.complex64
    lev = {l: O.nominal_level(O.from_synth(sm), k, [0, 0, 1], [1, 0, 0], dirs) for l, sm in enumerate(meshes)}
    cov_o = O.ct_farfield_covariance(lev, 0, 1, "gauss", sig, ell)
    assert _rel(cov.cpu().numpy().astype(np.complex128), cov_o) < 1e-4
    prob.release()
