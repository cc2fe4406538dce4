"""GPU parity: every CUDA step through the C ABI against the FP64 oracle on the same
seeded meshes.  Tolerances: Z and b entrywise relative to max|Z| (resp. max|b|) at
1e-12 in FP64 (rounding only: same quadrature), 1e-5 in FP32; currents, far fields
and covariances normwise at 1e-8 for FP64 and MIXED (refined), 1e-4 for FP32."""
import math

import numpy as np
import pytest

import fosb_synth as S
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global F
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_01457_gb300 as mod

    mod.build.build()
    F = mod
    O.build()
    yield


DEV = "cuda:0"
C128, C64 = torch.complex128, torch.complex64


def _mesh(sm):
    return F.mesh_create(sm.verts, sm.tris, sm.vnormals), O.from_synth(sm)


MESHES = {
    "ico1": lambda: S.icosphere(1),
    "ico2": lambda: S.icosphere(2),
    "torus20x8": lambda: S.torus(20, 8),
    "ellipsoid2": lambda: S.ellipsoid(2, (0.6, 1.3, 0.9)),
}


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name", list(MESHES))
def test_mesh_tables_match_oracle(name):
    sm = MESHES[name]()
    m, om = _mesh(sm)
    e, et = m.edges()
    assert np.array_equal(e, om.edges) and np.array_equal(et, om.edge_tris)
    assert m.n_edges == om.n_edges == 3 * sm.nt // 2


@pytest.mark.parametrize("name,k", [("ico1", 1.0), ("ico2", 4.0), ("torus20x8", 3.0), ("ellipsoid2", 2.5)])
def test_assembly_fp64_matches_oracle(name, k):
    sm = MESHES[name]()
    m, om = _mesh(sm)
    N = m.n_edges
    Z = torch.zeros((N, N), dtype=C128, device=DEV)
    inc = F.incidence([[0, 0, 1], [0.6, 0.0, 0.8]], [[1, 0, 0], [0, 1j, 0]])
    b = torch.zeros((N, 2), dtype=C128, device=DEV)
    F.assemble_efie(m, k, Z, inc=inc, b=b)
    Zo = O.assemble_z(om, k)
    bo = O.rhs_planewave(om, k, inc[:, :3], inc[:, 3:6] + 1j * inc[:, 6:9])
    Zg = Z.cpu().numpy()
    assert np.abs(Zg - Zo).max() <= 1e-12 * np.abs(Zo).max()
    assert np.abs(b.cpu().numpy() - bo).max() <= 1e-12 * np.abs(bo).max()
    assert np.abs(Zg - Zg.T).max() <= 1e-12 * np.abs(Zo).max()


@pytest.mark.parametrize("name,k", [("ico1", 1.0), ("ico2", 4.0), ("torus20x8", 3.0), ("ellipsoid2", 2.5)])
def test_assembly_float_float_matches_oracle(name, k):
    """Float-float regular pairs (FP32 pipe) reach FP64-class accuracy: 1e-12 of max|Z|."""
    sm = MESHES[name]()
    m, om = _mesh(sm)
    N = m.n_edges
    Z = torch.zeros((N, N), dtype=C128, device=DEV)
    F.assemble_efie(m, k, Z, arith=F.ASM_FF)
    Zo = O.assemble_z(om, k)
    err = np.abs(Z.cpu().numpy() - Zo).max() / np.abs(Zo).max()
    assert err <= 1e-12, err


def test_float_float_solution_matches_oracle():
    sm = S.icosphere(3)
    k = 4.0
    m, om = _mesh(sm)
    N = m.n_edges
    Z = torch.zeros((N, N), dtype=C128, device=DEV)
    b = torch.zeros((N, 1), dtype=C128, device=DEV)
    F.assemble_efie(m, k, Z, inc=F.incidence([0, 0, 1], [1, 0, 0]), b=b, arith=F.ASM_FF)
    lu = F.factor(Z, prec=F.MIXED)
    u = torch.zeros_like(b)
    F.solve(lu, b, u)
    Zo = O.assemble_z(om, k)
    uo = O.solve(Zo, O.rhs_planewave(om, k, [0, 0, 1], [1, 0, 0]))
    assert _rel(u.cpu().numpy(), uo) < 1e-8


def test_float_float_phase_range_is_checked():
    sm = S.icosphere(1)
    m = F.mesh_create(sm.verts, sm.tris)
    Z = torch.zeros((m.n_edges, m.n_edges), dtype=C128, device=DEV)
    with pytest.raises(F.FosbError) as ei:
        F.assemble_efie(m, 30.0, Z, arith=F.ASM_FF)  # k * diameter = 60 > 48
    assert ei.value.status == F.FOSB_ERR_INVALID_ARG


def test_assembly_fp32_matches_oracle():
    sm = S.icosphere(2)
    m, om = _mesh(sm)
    N = m.n_edges
    Z = torch.zeros((N, N), dtype=C64, device=DEV)
    F.assemble_efie(m, 2.0, Z, prec=F.FP32)
    Zo = O.assemble_z(om, 2.0)
    assert np.abs(Z.cpu().numpy() - Zo).max() <= 2e-5 * np.abs(Zo).max()


def test_assembly_leading_dimension_and_nss():
    sm = S.icosphere(1)
    m, om = _mesh(sm)
    N = m.n_edges
    big = torch.full((N, N + 7), 7.0 + 0j, dtype=C128, device=DEV)
    F.assemble_efie(m, 1.5, big[:, :N], n_ss=4)
    Zo = O.assemble_z(om, 1.5, n_ss=4)
    assert np.abs(big[:, :N].cpu().numpy() - Zo).max() <= 1e-12 * np.abs(Zo).max()
    assert torch.all(big[:, N:] == 7.0)


def _nominal(sm, k, prec, d=(0, 0, 1), p=(1, 0, 0)):
    m, om = _mesh(sm)
    N = m.n_edges
    dt = C64 if prec == F.FP32 else C128
    Z = torch.zeros((N, N), dtype=dt, device=DEV)
    b = torch.zeros((N, 1), dtype=dt, device=DEV)
    F.assemble_efie(m, k, Z, inc=F.incidence(d, p), b=b, prec=prec)
    lu = F.factor(Z, prec=prec)
    u = torch.zeros_like(b)
    _, iters, berr = F.solve(lu, b, u)
    return m, om, Z, b, lu, u, iters, berr


@pytest.mark.parametrize("prec,tol", [("FP64", 1e-8), ("MIXED", 1e-8), ("FP32", 1e-4)])
@pytest.mark.parametrize("lvl", [1, 2, 3])
def test_solve_matches_oracle(prec, tol, lvl):
    sm = S.icosphere(lvl)
    k = 2.0
    m, om, Z, b, lu, u, iters, berr = _nominal(sm, k, getattr(F, prec))
    Zo = O.assemble_z(om, k)
    uo = O.solve(Zo, O.rhs_planewave(om, k, [0, 0, 1], [1, 0, 0]))
    assert _rel(u.cpu().numpy().astype(np.complex128), uo) < tol
    if prec == "MIXED":
        assert iters >= 1 and berr < 1e-13


def test_solve_multiple_rhs_and_ragged_sizes():
    """Sizes that do not fill the 64-wide panels and tiles (N = 3 nu nv for a torus)."""
    sm = S.torus(14, 6)  # N = 252: 3 full panels + a ragged 60
    k = 1.7
    m, om = _mesh(sm)
    N = m.n_edges
    Z = torch.zeros((N, N), dtype=C128, device=DEV)
    F.assemble_efie(m, k, Z)
    rng = np.random.default_rng(3)
    Bh = rng.standard_normal((N, 11)) + 1j * rng.standard_normal((N, 11))
    B = torch.tensor(Bh, dtype=C128, device=DEV)
    Zo = O.assemble_z(om, k)
    Xo = np.linalg.solve(Zo, Bh)
    for prec in (F.FP64, F.MIXED):
        lu = F.factor(Z, prec=prec)
        X = torch.zeros_like(B)
        F.solve(lu, B, X)
        assert _rel(X.cpu().numpy(), Xo) < 1e-8
    # in place
    lu = F.factor(Z, prec=F.MIXED)
    B2 = B.clone()
    F.solve(lu, B2)
    assert _rel(B2.cpu().numpy(), Xo) < 1e-8


@pytest.mark.parametrize("n", [600, 700, 1030])
def test_complex64_lu_spans_column_blocks_and_ragged_panels(n):
    """The complex64 LU works in 256-column blocks of four 64-column panels with one
    K = 256 trailing update per block: n = 600, 700, 1030 leave a last block of 88, 188
    and 6 columns (ragged panels) and ragged 128-row tiles.  A row-permuted, diagonally
    dominant matrix forces a pivot on every column; a plain complex Gaussian matrix
    pivots freely.  MIXED solves agree with LAPACK at 1e-10; FP32 (complex64 factors,
    no refinement) at 1e-4."""
    rng = np.random.default_rng(n)
    G = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(2 * n)
    Ap = (G + 2.0 * np.eye(n))[rng.permutation(n)]
    Bh = rng.standard_normal((n, 5)) + 1j * rng.standard_normal((n, 5))
    for Ah in (Ap, G * math.sqrt(n)):
        Xo = np.linalg.solve(Ah, Bh)
        A = torch.tensor(Ah, dtype=C128, device=DEV)
        B = torch.tensor(Bh, dtype=C128, device=DEV)
        X = torch.zeros_like(B)
        F.solve(F.factor(A, prec=F.MIXED), B, X)
        assert _rel(X.cpu().numpy(), Xo) < 1e-10
        if Ah is Ap:
            A32, B32 = A.to(C64), B.to(C64)
            X32 = torch.zeros_like(B32)
            F.solve(F.factor(A32, prec=F.FP32), B32, X32)
            assert _rel(X32.cpu().numpy().astype(np.complex128), Xo) < 1e-4


def test_solve_many_rhs_ragged_digit_residual():
    """More than 8 right-hand sides at N >= 256 put the refinement residuals on the
    digit-split tensor-core product. N = 336 (torus 14 x 8) leaves a ragged 80-row tile
    and a last 64-wide k chunk of one 16-wide step; 37 columns leave a ragged column tile."""
    sm = S.torus(14, 8)
    k = 1.7
    m, om = _mesh(sm)
    N = m.n_edges
    assert N == 336
    Z = torch.zeros((N, N), dtype=C128, device=DEV)
    F.assemble_efie(m, k, Z)
    rng = np.random.default_rng(7)
    # columns of very different scales: the digits take one exponent per column
    Bh = (rng.standard_normal((N, 37)) + 1j * rng.standard_normal((N, 37))) * 10.0 ** rng.uniform(-6, 6, 37)
    B = torch.tensor(Bh, dtype=C128, device=DEV)
    Xo = np.linalg.solve(O.assemble_z(om, k), Bh)
    lu = F.factor(Z, prec=F.MIXED)
    X = torch.zeros_like(B)
    _, iters, berr = F.solve(lu, B, X)
    Xg = X.cpu().numpy()
    for c in range(37):
        assert _rel(Xg[:, c], Xo[:, c]) < 1e-8, c
    assert berr <= max(64.0, 8.0 * math.sqrt(N)) * 2.0**-52
    # the FP64 residual of the returned solution, from an independent complex128 product
    R = B - Z @ X
    zn = Z.abs().sum(dim=1).max().item()
    for c in range(37):
        be = R[:, c].abs().max().item() / (zn * X[:, c].abs().max().item() + B[:, c].abs().max().item())
        assert be <= 2.0 * max(64.0, 8.0 * math.sqrt(N)) * 2.0**-52, (c, be)


@pytest.mark.parametrize("prec,tol", [("FP64", 1e-8), ("MIXED", 1e-8), ("FP32", 1e-4)])
def test_farfield_mean_matches_oracle(prec, tol):
    sm = S.icosphere(2)
    k = 2.0
    m, om, Z, b, lu, u, _, _ = _nominal(sm, k, getattr(F, prec))
    xh = S.hplane_directions(181)
    out = torch.zeros((3 * 181, 1), dtype=u.dtype, device=DEV)
    F.farfield_moments(m, k, xh, u, out)
    Zo = O.assemble_z(om, k)
    uo = O.solve(Zo, O.rhs_planewave(om, k, [0, 0, 1], [1, 0, 0]))
    Fo = O.farfield_matrix(om, k, xh) @ uo
    assert _rel(out.cpu().numpy().astype(np.complex128), Fo) < tol


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
@pytest.mark.parametrize("pair,kind,pseudo", [((1, 1), "gauss", False), ((2, 1), "matern32", False),
                                              ((1, 2), "gauss", False), ((2, 1), "gauss", True)])
def test_covariance_block_matches_oracle(prec, pair, kind, pseudo):
    k = 2.0
    P = getattr(F, prec)
    lv = {}
    for l in set(pair):
        sm = S.icosphere(l)
        m, om, Z, b, lu, u, _, _ = _nominal(sm, k, P)
        Zo = O.assemble_z(om, k)
        uo = O.solve(Zo, O.rhs_planewave(om, k, [0, 0, 1], [1, 0, 0]))[:, 0]
        lv[l] = (m, om, Z, lu, u, Zo, O.sd_rhs(om, k, uo))
    a, c = lv[pair[0]], lv[pair[1]]
    Sig = torch.zeros((a[0].n_edges, c[0].n_edges), dtype=C128, device=DEV)
    kk = F.COV_GAUSS if kind == "gauss" else F.COV_MATERN32
    F.covariance(a[0], a[3], a[4], c[0], c[3], c[4], k, Sig, kk, 0.01, 0.5, pseudo=pseudo)
    K = O.cov_kernel(a[1].verts, c[1].verts, kind, 0.01, 0.5)
    So = O.covariance(a[5], a[6], c[5], c[6], K, pseudo=pseudo)
    assert _rel(Sig.cpu().numpy(), So) < 1e-8


def test_ct_farfield_covariance_matches_oracle():
    """Combination technique L0 = 0, L = 2 over icospheres 1..3: signed sum of
    A_l1 Sigma A_l2^H with the Hermitian mirror, accumulated on the device."""
    k = 1.5
    xh = S.hplane_directions(13)
    nd3 = 3 * xh.shape[0]
    gl, ol = {}, {}
    for l in (0, 1, 2):
        sm = S.icosphere(l + 1)
        m, om, Z, b, lu, u, _, _ = _nominal(sm, k, F.MIXED)
        gl[l] = (m, lu, u)
        ol[l] = O.nominal_level(om, k, [0, 0, 1], [1, 0, 0], xh)
    out = torch.zeros((nd3, nd3), dtype=C128, device=DEV)
    first = True
    for (l1, l2), sgn in O.ct_hermitian_blocks(0, 2):
        a, c = gl[l1], gl[l2]
        Sig = torch.zeros((a[0].n_edges, c[0].n_edges), dtype=C128, device=DEV)
        F.covariance(a[0], a[1], a[2], c[0], c[1], c[2], k, Sig, F.COV_GAUSS, 1.0, 0.6)
        F.farfield_moments(a[0], k, xh, Sig, out, m2=c[0], weight=float(sgn), mirror=(l1 != l2), accumulate=not first)
        first = False
    ref = O.ct_farfield_covariance(ol, 0, 2, "gauss", 1.0, 0.6)
    assert _rel(out.cpu().numpy(), ref) < 1e-8


def test_errors_are_reported():
    sm = S.icosphere(1)
    bad = sm.tris.copy()
    bad[0, 1], bad[0, 2] = bad[0, 2], bad[0, 1]  # flip one triangle: inconsistent orientation
    with pytest.raises(F.FosbError) as ei:
        F.mesh_create(sm.verts, bad)
    assert ei.value.status == F.FOSB_ERR_MESH
    m = F.mesh_create(sm.verts, sm.tris)
    Z = torch.zeros((m.n_edges, m.n_edges), dtype=C128, device=DEV)
    with pytest.raises(F.FosbError) as ei:
        F.assemble_efie(m, -1.0, Z)
    assert ei.value.status == F.FOSB_ERR_INVALID_ARG
    Zs = torch.zeros((4, 4), dtype=C128, device=DEV)
    with pytest.raises(F.FosbError) as ei:
        F.factor(Zs, prec=F.FP64)
    assert ei.value.status == F.FOSB_ERR_SINGULAR
