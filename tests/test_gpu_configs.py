"""Parity cases for the other workloads of the method, each at its own size:
  * plain FP64: unit icosphere of 320 triangles (N = 480), k = 1, full tensor covariance
    480 x 480 (Gaussian, std 0.01, l = 0.5), far-field and RCS moments at 181 angles;
  * batched: seeded ellipsoids (semi-axes U[0.5, 1.5], k U[1, 6]) with 16 Fibonacci
    incident directions each, complex64 factors with FP64 refinement;
  * differentiation: monostatic RCS gradient at 8 angles of the 5120-triangle sphere
    (N = 7680), k = 3;
  * largest: torus R = 1, r = 0.35 over 5 nested grids (N up to 30720), k = 10,
    Matern-3/2 (std 0.002, l = 0.2), combination technique L0 = 1, L = 5, 361 angles.
Where the oracle cannot solve the full size in seconds, sampled entries and identities
that hold at any size are checked instead."""
import math

import numpy as np
import pytest

import fosb_synth as S
import oracle as O
from oracle import mie

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
C128 = torch.complex128


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


def test_plain_fp64_full_tensor_and_rcs_moments(F):
    sm = S.icosphere(2)
    k, sig, ell = 1.0, 0.01, 0.5
    xh = S.hplane_directions(181)
    m = F.mesh_create(sm.verts, sm.tris, sm.vnormals)
    N = m.n_edges
    assert N == 480
    Z = torch.zeros((N, N), dtype=C128, device=DEV)
    b = torch.zeros((N, 1), dtype=C128, device=DEV)
    F.assemble_efie(m, k, Z, inc=F.incidence((0, 0, 1), (1, 0, 0)), b=b, arith=F.ASM_FP64, prec=F.FP64)
    lu = F.factor(Z, prec=F.FP64)
    u = torch.zeros_like(b)
    F.solve(lu, b, u)
    Sig = torch.zeros((N, N), dtype=C128, device=DEV)
    PSig = torch.zeros((N, N), dtype=C128, device=DEV)
    F.covariance(m, lu, u, m, lu, u, k, Sig, F.COV_GAUSS, sig, ell)
    F.covariance(m, lu, u, m, lu, u, k, PSig, F.COV_GAUSS, sig, ell, pseudo=True)
    nd3 = 3 * xh.shape[0]
    Fm = torch.zeros((nd3, 1), dtype=C128, device=DEV)
    cov = torch.zeros((nd3, nd3), dtype=C128, device=DEV)
    pcov = torch.zeros((nd3, nd3), dtype=C128, device=DEV)
    F.farfield_moments(m, k, xh, u, Fm)
    F.farfield_moments(m, k, xh, Sig, cov, m2=m)
    F.farfield_moments(m, k, xh, PSig, pcov, m2=m, pseudo=True)

    om = O.from_synth(sm)
    lev = O.nominal_level(om, k, [0, 0, 1], [1, 0, 0], xh)
    K = O.cov_kernel(om.verts, om.verts, "gauss", sig, ell)
    So = O.covariance(lev.Z, lev.B, lev.Z, lev.B, K)
    Po = O.covariance(lev.Z, lev.B, lev.Z, lev.B, K, pseudo=True)
    assert _rel(Sig.cpu().numpy(), So) < 1e-8
    assert _rel(PSig.cpu().numpy(), Po) < 1e-8
    Fo = lev.A @ lev.u
    covo, pcovo = lev.A @ So @ lev.A.conj().T, lev.A @ Po @ lev.A.T
    assert _rel(Fm.cpu().numpy()[:, 0], Fo) < 1e-8
    assert _rel(cov.cpu().numpy(), covo) < 1e-8
    assert _rel(pcov.cpu().numpy(), pcovo) < 1e-8
    # RCS mean (dB) and its delta-method variance from the GPU moments
    f = Fm.cpu().numpy()[:, 0].reshape(-1, 3)
    var = O.rcs_variance_db(f, cov.cpu().numpy(), pcov.cpu().numpy())
    var_o = O.rcs_variance_db(Fo.reshape(-1, 3), covo, pcovo)
    assert np.all(var >= 0.0) and _rel(var, var_o) < 1e-7
    assert np.abs(O.rcs_db(f) - O.rcs_db(Fo.reshape(-1, 3))).max() < 1e-8
    # the library's RCS moments (fosb_rcs_moments) against the oracle's, from the oracle's moments
    nd = xh.shape[0]
    r_db = torch.zeros(nd, dtype=torch.float64, device=DEV)
    v_db = torch.zeros(nd, dtype=torch.float64, device=DEV)
    v_f = torch.zeros(3 * nd, dtype=torch.float64, device=DEV)
    F.rcs_moments(nd, Fm, cov, pcov, rcs_db=r_db, var_db=v_db, var_f=v_f)
    rcs_o = O.rcs_db(Fo.reshape(-1, 3))
    assert np.abs(r_db.cpu().numpy() - rcs_o).max() < 1e-8 * np.abs(rcs_o).max()
    assert _rel(v_db.cpu().numpy(), var_o) < 1e-8
    assert _rel(v_f.cpu().numpy(), np.diag(covo).real) < 1e-8
    F.rcs_moments(nd, Fm, rcs_db=r_db, convention=1)  # the printed 4 pi |F|^2: + 10 log10((4 pi)^2)
    assert np.abs(r_db.cpu().numpy() - rcs_o - 20 * math.log10(4 * math.pi)).max() < 1e-10
    # the mean field against the Mie series (discretisation error at 320 triangles)
    assert _rel(f, mie.farfield(k, 1.0, xh)) < 0.06


def test_batched_ellipsoids_mixed_solves(F):
    table = S.batched_ellipsoid_table()
    picked = [(i, row) for i, row in enumerate(table) if row[2] in (2, 3)][:4]
    assert len(picked) == 4
    d = S.fibonacci_directions(16)
    p = np.asarray(S.polarisation_for(d)).reshape(-1, 3)
    for i, (ax, k, lvl) in picked:
        sm = S.ellipsoid(lvl, tuple(ax))
        m = F.mesh_create(sm.verts, sm.tris, sm.vnormals)
        N = m.n_edges
        inc = F.incidence(d, p)
        Z = torch.zeros((N, N), dtype=C128, device=DEV)
        B = torch.zeros((N, 16), dtype=C128, device=DEV)
        F.assemble_efie(m, k, Z, inc=inc, b=B, arith=F.ASM_FF, prec=F.MIXED)
        lu = F.factor(Z, prec=F.MIXED)
        X = torch.zeros_like(B)
        _, iters, berr = F.solve(lu, B, X)
        om = O.from_synth(sm)
        Zo = O.assemble_z(om, k)
        Xo = O.solve(Zo, O.rhs_planewave(om, k, d, p))
        Xg = X.cpu().numpy()
        for c in range(16):
            assert _rel(Xg[:, c], Xo[:, c]) < 1e-8, (i, c)
        assert berr <= max(64.0, 8.0 * math.sqrt(N)) * 2.0**-52


def test_differentiation_fullsize_matches_finite_differences(F):
    """Adjoint gradient at N = 7680 against central differences of the GPU's own FP64 RCS
    (h = 1e-5) at sampled vertex coordinates: a property of any correct gradient."""
    sm = S.icosphere(4)
    k = 3.0
    d, p, _ = S.monostatic_directions(8)
    w = np.random.default_rng(4).standard_normal(len(d))

    def rcs(verts, prec, grad=None):
        m = F.mesh_create(verts, sm.tris, sm.vnormals)
        N = m.n_edges
        inc = F.incidence(d, p)
        Z = torch.zeros((N, N), dtype=C128, device=DEV)
        B = torch.zeros((N, len(d)), dtype=C128, device=DEV)
        F.assemble_efie(m, k, Z, inc=inc, b=B, arith=F.ASM_FP64, prec=prec)
        lu = F.factor(Z, prec=prec)
        U = torch.zeros_like(B)
        F.solve(lu, B, U)
        return F.rcs_monostatic(m, k, inc, U, lu=lu, weights=w, grad=grad)

    grad = torch.zeros((sm.nv, 3), dtype=torch.float64, device=DEV)
    sig0 = rcs(sm.verts, F.MIXED, grad)
    assert sm.tris.shape[0] == 5120 and np.all(sig0 > 0)
    g = grad.cpu().numpy()
    rng = np.random.default_rng(7)
    coords = [(int(v), int(c)) for v, c in zip(rng.choice(sm.nv, 6, replace=False), rng.integers(0, 3, 6))]
    h = 1e-5
    g_fd, g_ad = [], []
    for v, c in coords:
        vp, vm = sm.verts.copy(), sm.verts.copy()
        vp[v, c] += h
        vm[v, c] -= h
        g_fd.append(float(w @ (rcs(vp, F.FP64) - rcs(vm, F.FP64))) / (2 * h))
        g_ad.append(g[v, c])
    g_fd, g_ad = np.array(g_fd), np.array(g_ad)
    assert np.linalg.norm(g_ad - g_fd) <= 1e-4 * np.linalg.norm(g_fd), (g_ad, g_fd)


@pytest.fixture(scope="module")
def torus_run(F):
    from paper_2308_01457_gb300.ct import FOSBProblem

    meshes = S.torus_hierarchy([1, 2, 3, 4, 5])
    dirs = S.zplane_directions(361)
    prob = FOSBProblem(meshes, 10.0, (1, 0, 0), (0, 0, 1), dirs, 1, 5, F.COV_MATERN32, 0.002, 0.2,
                       prec=F.MIXED, arith=F.ASM_FF, pseudo=True).setup()
    Fm, cov, pcov = prob.run()
    torch.cuda.synchronize()
    yield prob, meshes, dirs, Fm, cov, pcov
    prob.release()


def test_torus_fullsize_samples_and_identities(F, torus_run):
    prob, meshes, dirs, Fm, cov, pcov = torus_run
    k = 10.0
    fine = prob.levels[5]
    om = O.from_synth(meshes[4])
    N = om.n_edges
    assert N == 30720
    rng = np.random.default_rng(10)
    rows = list(rng.integers(0, N, 128))
    cols = list(rng.integers(0, N, 128))
    for e in rng.integers(0, N, 12):
        for t in om.edge_tris[e]:
            for n in om.tri_edge[t]:
                rows.append(e)
                cols.append(n)
    r, c = np.array(rows, np.int64), np.array(cols, np.int64)
    zo = O.z_entries(om, k, r, c)
    zg = fine.Z[torch.as_tensor(r, device=DEV), torch.as_tensor(c, device=DEV)].cpu().numpy()
    assert np.abs(zg - zo).max() <= 1e-12 * np.abs(zo).max()
    bo = O.rhs_planewave(om, k, [1, 0, 0], [0, 0, 1])
    assert np.abs(fine.b.cpu().numpy() - bo).max() <= 1e-12 * np.abs(bo).max()
    for l, st in prob.levels.items():
        assert st.berr <= max(64.0, 8.0 * math.sqrt(st.Z.shape[0])) * 2.0**-52, (l, st.berr)
    # mean far field at 361 angles against the oracle's far-field matrix
    A = O.farfield_matrix(om, k, dirs)
    ref = A @ fine.u.cpu().numpy()
    assert _rel(Fm.cpu().numpy(), ref) < 1e-12
    # CT moments: Hermitian covariance, complex-symmetric pseudo-covariance, RCS variance >= 0
    cv, pv = cov.cpu().numpy(), pcov.cpu().numpy()
    assert np.linalg.norm(cv - cv.conj().T) <= 1e-12 * np.linalg.norm(cv)
    assert np.linalg.norm(pv - pv.T) <= 1e-12 * np.linalg.norm(pv)
    var = O.rcs_variance_db(Fm.cpu().numpy()[:, 0].reshape(-1, 3), cv, pv)
    assert np.all(np.isfinite(var))
    # the library's RCS moments on the same GPU moments (361 directions, 30720 unknowns)
    nd = dirs.shape[0]
    r_db = torch.zeros(nd, dtype=torch.float64, device=DEV)
    v_db = torch.zeros(nd, dtype=torch.float64, device=DEV)
    F.rcs_moments(nd, Fm, cov, pcov, rcs_db=r_db, var_db=v_db)
    assert _rel(v_db.cpu().numpy(), var) < 1e-12
    rcs_o = O.rcs_db(Fm.cpu().numpy()[:, 0].reshape(-1, 3))
    assert np.abs(r_db.cpu().numpy() - rcs_o).max() < 1e-12 * np.abs(rcs_o).max()
    # the duplicated endpoint of the 361 directions: F(0) = F(2 pi)
    f = Fm.cpu().numpy()[:, 0].reshape(-1, 3)
    assert np.abs(f[0] - f[-1]).max() <= 1e-12 * np.abs(f).max()


def test_torus_covariance_block_identity(F, torus_run):
    """Block (5, 1) of the torus hierarchy: Z5 Sigma Z1^H = B5 K51 B1^H with the Matern
    kernel, B from the oracle's SD right-hand side at the certified GPU solutions."""
    prob, meshes, dirs, _, _, _ = torus_run
    k = 10.0
    a, c = prob.levels[5], prob.levels[1]
    Sig = torch.zeros((a.mesh.n_edges, c.mesh.n_edges), dtype=C128, device=DEV)
    F.covariance(a.mesh, a.lu, a.u, c.mesh, c.lu, c.u, k, Sig, F.COV_MATERN32, 0.002, 0.2)
    om1, om2 = O.from_synth(meshes[4]), O.from_synth(meshes[0])
    B1 = O.sd_rhs(om1, k, a.u.cpu().numpy()[:, 0], dense=False)
    B2 = O.sd_rhs(om2, k, c.u.cpu().numpy()[:, 0])
    K = O.cov_kernel(om1.verts, om2.verts, "matern32", 0.002, 0.2)
    C = B1 @ (K @ B2.conj().T)
    lhs = ((a.Z @ Sig) @ c.Z.conj().T).cpu().numpy()
    scale = ((a.Z.abs() @ Sig.abs()) @ c.Z.abs().T).cpu().numpy()
    assert np.linalg.norm(lhs - C) / np.linalg.norm(scale) < 1e-11
