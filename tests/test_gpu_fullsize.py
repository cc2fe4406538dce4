"""Parity at the full size of the mixed-precision sphere workload (icospheres of 80 ..
20480 triangles, N up to 30720, k = 4, float-float assembly, complex64 tensor-core LU
with FP64-class refinement), in the launch configuration the benchmark times.

The oracle cannot assemble or factor N = 30720 in seconds, so this file checks what it
can compute one by one, plus identities that hold at any size:
  * sampled Z entries (random, diagonal and touching pairs) against the oracle's per-entry
    assembly, and the whole plane-wave RHS;
  * the refined solve's normwise backward error, from an independent complex128 product;
  * the covariance block (4, 0) through its definition Z1 Sigma Z2^H = B1 K12 B2^H
    (Sections III and IV-A), with B from the oracle's SD right-hand side at the solutions
    certified above and K from the oracle's kernel;
  * the mean far field and the far-field block A1 Sigma A2^H against the oracle's A.
"""
import math

import numpy as np
import pytest

import fosb_synth as S
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
C128 = torch.complex128

# the mixed-precision sphere workload: levels 0..4 (icosphere s = l + 1), k a = 4,
# Gaussian sigma = 0.005, l = 0.3, 181 H-plane directions, d = +z, p = x
LEVELS = [0, 1, 2, 3, 4]
K_WAVE, SIGMA, ELL, N_DIR = 4.0, 0.005, 0.3, 181


@pytest.fixture(scope="module")
def run():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_01457_gb300 as F
    from paper_2308_01457_gb300.ct import FOSBProblem

    F.build.build()
    O.build()
    meshes = [S.icosphere(l + 1) for l in LEVELS]
    dirs = S.hplane_directions(N_DIR)
    prob = FOSBProblem(meshes, K_WAVE, (0, 0, 1), (1, 0, 0), dirs, 0, 4, F.COV_GAUSS, SIGMA, ELL,
                       prec=F.MIXED, arith=F.ASM_FF).setup()
    Fmean, cov = prob.run()
    torch.cuda.synchronize()
    yield F, prob, meshes, dirs, Fmean, cov
    prob.release()


def test_fullsize_z_samples_and_rhs(run):
    F, prob, meshes, dirs, _, _ = run
    st = prob.levels[4]
    om = O.from_synth(meshes[4])
    N = om.n_edges
    assert N == 30720 and st.Z.shape == (N, N)
    rng = np.random.default_rng(1457)
    rows = [rng.integers(0, N, 192)]
    cols = [rng.integers(0, N, 192)]
    d = rng.integers(0, N, 32)
    rows.append(d)
    cols.append(d)
    # touching pairs: every edge of T+ and T- of sampled edges (identical, edge and vertex classes)
    for e in rng.integers(0, N, 16):
        for t in om.edge_tris[e]:
            for n in om.tri_edge[t]:
                rows.append(np.array([e]))
                cols.append(np.array([n]))
    r = np.concatenate(rows).astype(np.int64)
    c = np.concatenate(cols).astype(np.int64)
    zo = O.z_entries(om, K_WAVE, r, c)
    zg = st.Z[torch.as_tensor(r, device=DEV), torch.as_tensor(c, device=DEV)].cpu().numpy()
    scale = np.abs(zo).max()
    assert np.abs(zg - zo).max() <= 1e-12 * scale
    bo = O.rhs_planewave(om, K_WAVE, [0, 0, 1], [1, 0, 0])
    assert np.abs(st.b.cpu().numpy() - bo).max() <= 1e-12 * np.abs(bo).max()


def test_fullsize_refined_solve_backward_error(run):
    F, prob, _, _, _, _ = run
    for l in LEVELS:
        st = prob.levels[l]
        N = st.Z.shape[0]
        r = st.b - st.Z @ st.u
        zn = st.Z.abs().sum(dim=1).max().item()
        berr = r.abs().max().item() / (zn * st.u.abs().max().item() + st.b.abs().max().item())
        tol = max(64.0, 8.0 * math.sqrt(N)) * 2.0**-52
        assert berr <= 2.0 * tol, (l, berr, tol)
        assert st.berr <= tol


def test_fullsize_covariance_block_identity(run):
    F, prob, meshes, dirs, _, _ = run
    a, c = prob.levels[4], prob.levels[0]
    N1, N2 = a.mesh.n_edges, c.mesh.n_edges
    Sig = torch.zeros((N1, N2), dtype=C128, device=DEV)
    F.covariance(a.mesh, a.lu, a.u, c.mesh, c.lu, c.u, K_WAVE, Sig, F.COV_GAUSS, SIGMA, ELL)
    om1, om2 = O.from_synth(meshes[4]), O.from_synth(meshes[0])
    B1 = O.sd_rhs(om1, K_WAVE, a.u.cpu().numpy()[:, 0], dense=False)
    B2 = O.sd_rhs(om2, K_WAVE, c.u.cpu().numpy()[:, 0])
    K12 = O.cov_kernel(om1.verts, om2.verts, "gauss", SIGMA, ELL)
    C = B1 @ (K12 @ B2.conj().T)
    lhs = ((a.Z @ Sig) @ c.Z.conj().T).cpu().numpy()
    scale = ((a.Z.abs() @ Sig.abs()) @ c.Z.abs().T).cpu().numpy()
    err = np.linalg.norm(lhs - C) / np.linalg.norm(scale)
    assert err < 1e-11, err
    assert np.linalg.norm(C) > 0.0

    # far-field block A1 Sigma A2^H against the oracle's far-field matrices
    nd3 = 3 * dirs.shape[0]
    out = torch.zeros((nd3, nd3), dtype=C128, device=DEV)
    F.farfield_moments(a.mesh, K_WAVE, dirs, Sig, out, m2=c.mesh, prec=F.MIXED)
    A1, A2 = O.farfield_matrix(om1, K_WAVE, dirs), O.farfield_matrix(om2, K_WAVE, dirs)
    ref = A1 @ Sig.cpu().numpy() @ A2.conj().T
    assert np.linalg.norm(out.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-10


def test_fullsize_mean_farfield_and_ct_covariance_shape(run):
    F, prob, meshes, dirs, Fmean, cov = run
    om = O.from_synth(meshes[4])
    ref = O.farfield_matrix(om, K_WAVE, dirs) @ prob.levels[4].u.cpu().numpy()
    assert np.linalg.norm(Fmean.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-12
    cv = cov.cpu().numpy()
    assert np.all(np.isfinite(cv))
    # the CT sum of Hermitian-mirrored blocks is Hermitian
    assert np.linalg.norm(cv - cv.conj().T) <= 1e-12 * np.linalg.norm(cv)
