"""GPU parity of the dielectric (PMCHWT) path, Section II-C eq. pmchwt, through the C ABI
against the FP64 oracle on the same seeded meshes: the 2N x 2N matrix and the tested
incident data entrywise at 1e-12 of their largest entry (same quadrature, rounding only);
the exterior Cauchy data and the far field normwise at 1e-8 (FP64 and MIXED, refined);
at the benchmark's size (2N = 15360), sampled entries of all four blocks against the
oracle's entry-by-entry assembly, the refined solve's backward error and the far field
against the dielectric Mie series at the discretisation level."""
import math

import numpy as np
import pytest

import fosb_synth as S
import oracle as O
import oracle.mie as mie

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F = None
DEV = "cuda:0"
C128 = torch.complex128


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


def _mesh(sm):
    return F.mesh_create(sm.verts, sm.tris, sm.vnormals), O.from_synth(sm)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


MESHES = {
    "ico1": lambda: S.icosphere(1),
    "ico2": lambda: S.icosphere(2),
    "torus20x8": lambda: S.torus(20, 8),
    "ellipsoid2": lambda: S.ellipsoid(2, (0.6, 1.3, 0.9)),
}


@pytest.mark.parametrize("arith", ["ASM_FP64", "ASM_FF"])
@pytest.mark.parametrize("name,k0,er,mr,nss", [("ico1", 2.0, 2.1, 1.0, 5), ("ico2", 3.0, 2.1, 1.0, 5),
                                               ("torus20x8", 1.5, 2.0, 1.5, 3), ("ellipsoid2", 2.5, 4.0, 1.0, 5)])
def test_pmchwt_assembly_matches_oracle(name, k0, er, mr, nss, arith):
    """Regular pairs in FP64 or float-float (FP32 pipe), touching pairs in FP64."""
    sm = MESHES[name]()
    m, om = _mesh(sm)
    N = m.n_edges
    inc = F.incidence([[1, 0, 0], [0.0, 0.6, 0.8]], [[0, 0, 1], [1j, 0, 0]])
    # a leading dimension larger than 2N, and b with a spare column
    Zbuf = torch.full((2 * N, 2 * N + 3), 7.0, dtype=C128, device=DEV)
    bbuf = torch.full((2 * N, 3), 7.0, dtype=C128, device=DEV)
    Z, b = Zbuf[:, :2 * N], bbuf[:, :2]
    F.assemble_pmchwt(m, k0, er, mr, Z, inc=inc, b=b, n_ss=nss, arith=getattr(F, arith))
    Zo = O.assemble_pmchwt(om, k0, er, mr, n_ss=nss)
    bo = O.rhs_pmchwt(om, k0, inc[:, :3], inc[:, 3:6] + 1j * inc[:, 6:9])
    Zg, bg = Z.cpu().numpy(), b.cpu().numpy()
    assert np.abs(Zg - Zo).max() <= 1e-12 * np.abs(Zo).max()
    assert np.abs(bg - bo).max() <= 1e-12 * np.abs(bo).max()
    assert torch.all(Zbuf[:, 2 * N:] == 7.0) and torch.all(bbuf[:, 2:] == 7.0)


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
@pytest.mark.parametrize("lvl", [2, 3])
def test_pmchwt_solve_and_farfield_match_oracle(prec, lvl):
    """The paper's dielectric sphere (Section V-A, Table I: k0 = 3, eps_r = 2.1, mu_r = 1,
    d = x, p = z) plus a second incidence; 2N = 960 (ragged against the LU's 256-column
    blocks) and 3840.  Far field on 181 directions of the z = 0 plane (Section II-C)."""
    sm = S.icosphere(lvl)
    m, om = _mesh(sm)
    N = m.n_edges
    k0, er, mr = 3.0, 2.1, 1.0
    d = np.array([[1.0, 0, 0], [0, 0, 1.0]])
    p = np.array([[0, 0, 1.0], [1.0, 0, 0]], dtype=complex)
    inc = F.incidence(d, p)
    Z = torch.zeros((2 * N, 2 * N), dtype=C128, device=DEV)
    b = torch.zeros((2 * N, 2), dtype=C128, device=DEV)
    F.assemble_pmchwt(m, k0, er, mr, Z, inc=inc, b=b)
    lu = F.factor(Z, prec=getattr(F, prec))
    X, _, berr = F.solve(lu, b.clone())
    Zo = O.assemble_pmchwt(om, k0, er, mr)
    bo = O.rhs_pmchwt(om, k0, d, p)
    Xo = O.solve(Zo, bo)
    Xg = X.cpu().numpy()
    for c in range(2):
        assert _rel(Xg[:, c], Xo[:, c]) < 1e-8
    assert berr <= max(64.0, 8.0 * math.sqrt(2 * N)) * 2.0**-52
    xh = S.zplane_directions(181)
    out = torch.zeros((3 * xh.shape[0], 2), dtype=C128, device=DEV)
    F.farfield_pmchwt(m, k0, xh, X, out)
    Fo = O.farfield_matrix_pmchwt(om, k0, xh) @ Xo
    assert _rel(out.cpu().numpy(), Fo) < 1e-8
    # physics, not parity: the z-polarised wave along +x against the Mie series of the
    # x-polarised wave along +z, by the rotation taking (e_x, e_y, e_z) to (e_z, -e_y, e_x)
    R = np.array([[0, 0, 1.0], [0, -1.0, 0], [1.0, 0, 0]])
    Fm = mie.farfield(k0, 1.0, xh @ R, eps_r=er, mu_r=mr) @ R.T
    Fg = out.cpu().numpy()[:, 0].reshape(-1, 3)
    assert _rel(Fg, Fm) < (0.08 if lvl == 2 else 0.02)


def test_pmchwt_accumulating_farfield_and_weights():
    sm = S.icosphere(1)
    m, om = _mesh(sm)
    N = m.n_edges
    rng = np.random.default_rng(7)
    Xh = rng.standard_normal((2 * N, 3)) + 1j * rng.standard_normal((2 * N, 3))
    X = torch.tensor(Xh, dtype=C128, device=DEV)
    xh = S.fibonacci_directions(16)
    out = torch.zeros((48, 3), dtype=C128, device=DEV)
    F.farfield_pmchwt(m, 2.0, xh, X, out, weight=2.0)
    F.farfield_pmchwt(m, 2.0, xh, X, out, weight=-0.5, accumulate=True)
    A = O.farfield_matrix_pmchwt(om, 2.0, xh)
    assert _rel(out.cpu().numpy(), 1.5 * A @ Xh) < 1e-13


def test_pmchwt_fullsize_sampled_entries_and_solve():
    """The benchmark's launch configuration: icosphere of 5120 triangles (2N = 15360),
    k0 = 3, eps_r = 2.1, float-float regular pairs; 400 sampled entries per block (random,
    plus the touching pairs of the sample rows) against the oracle's entry-by-entry
    assembly at 1e-12 of max|Z|; b against the oracle; the MIXED refined solve's backward
    error; the far field against the Mie series (discretisation level)."""
    sm = S.icosphere(4)
    m, om = _mesh(sm)
    N = m.n_edges
    k0, er, mr = 3.0, 2.1, 1.0
    inc = F.incidence([[1.0, 0, 0]], [[0, 0, 1.0]])
    Z = torch.zeros((2 * N, 2 * N), dtype=C128, device=DEV)
    b = torch.zeros((2 * N, 1), dtype=C128, device=DEV)
    F.assemble_pmchwt(m, k0, er, mr, Z, inc=inc, b=b, arith=F.ASM_FF)
    zmax = Z.abs().max().item()
    rng = np.random.default_rng(20230801)
    rows, cols = [], []
    for br in (0, 1):
        for bc in (0, 1):
            r = rng.integers(0, N, 300)
            c = rng.integers(0, N, 300)
            # touching: the other edges of the sample rows' own triangles
            t = om.edge_tris[r[:100], 0]
            c2 = om.tri_edge[t, rng.integers(0, 3, 100)]
            rows += list(r + br * N) + list(r[:100] + br * N)
            cols += list(c + bc * N) + list(c2 + bc * N)
    rows, cols = np.array(rows), np.array(cols)
    ref = O.pmchwt_entries(om, k0, er, mr, rows, cols)
    got = Z[torch.tensor(rows, device=DEV), torch.tensor(cols, device=DEV)].cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * zmax
    bo = O.rhs_pmchwt(om, k0, [[1.0, 0, 0]], [[0, 0, 1.0]])
    assert np.abs(b.cpu().numpy() - bo).max() <= 1e-12 * np.abs(bo).max()
    lu = F.factor(Z, prec=F.MIXED)
    X, _, berr = F.solve(lu, b.clone())
    assert berr <= max(64.0, 8.0 * math.sqrt(2 * N)) * 2.0**-52
    xh = S.zplane_directions(361)
    out = torch.zeros((3 * 361, 1), dtype=C128, device=DEV)
    F.farfield_pmchwt(m, k0, xh, X, out)
    R = np.array([[0, 0, 1.0], [0, -1.0, 0], [1.0, 0, 0]])
    Fm = mie.farfield(k0, 1.0, xh @ R, eps_r=er, mu_r=mr) @ R.T
    assert _rel(out.cpu().numpy()[:, 0].reshape(-1, 3), Fm) < 0.01


def test_pmchwt_argument_errors():
    sm = S.icosphere(1)
    m, _ = _mesh(sm)
    N = m.n_edges
    Z = torch.zeros((2 * N, 2 * N), dtype=C128, device=DEV)
    bad = [dict(k0=2.0, er=0.0, mr=1.0), dict(k0=2.0, er=2.0, mr=-1.0), dict(k0=0.0, er=2.0, mr=1.0),
           dict(k0=2.0, er=float("nan"), mr=1.0)]
    for a in bad:
        with pytest.raises(F.FosbError) as e:
            F.assemble_pmchwt(m, a["k0"], a["er"], a["mr"], Z)
        assert e.value.status == F.FOSB_ERR_INVALID_ARG
    with pytest.raises(F.FosbError) as e:
        # ldz < 2N (a view of Z would keep Z's row stride, so a narrower buffer)
        F.assemble_pmchwt(m, 2.0, 2.0, 1.0, torch.zeros((2 * N, 2 * N - 1), dtype=C128, device=DEV))
    assert e.value.status == F.FOSB_ERR_INVALID_ARG
    for k0, arith in ((2.0, F.ASM_FP32), (30.0, F.ASM_FF)):   # no FP32 path; float-float phase range
        with pytest.raises(F.FosbError) as e:
            F.assemble_pmchwt(m, k0, 2.0, 1.0, Z, arith=arith)
        assert e.value.status == F.FOSB_ERR_INVALID_ARG
    with pytest.raises(F.FosbError) as e:
        F.assemble_pmchwt(m, 2.0, 2.0, 1.0, Z, inc=F.incidence([[0, 0, 1.0]], [[np.nan, 0, 0]]),
                          b=torch.zeros((2 * N, 1), dtype=C128, device=DEV))
    assert e.value.status == F.FOSB_ERR_INVALID_ARG


def test_dielectric_ct_second_moment_matches_oracle():
    """Section V-A's CT check on the dielectric sphere (k0 = 3, eps_r = 2.1, d = x, p = z), the
    rank-one tensor right-hand side, levels 0..2 (80 .. 1280 triangles), L0 = 0, L = 2: the
    finest far field and the CT second moment (all components, 91 directions of the z = 0
    plane) against the oracle at 1e-8."""
    from paper_2308_01457_gb300.dielectric import DielectricCT

    sms = {l: S.icosphere(l + 1) for l in range(3)}
    xh = S.zplane_directions(91)
    d, p = [[1.0, 0, 0]], [[0, 0, 1.0]]
    prob = DielectricCT(sms, 3.0, 2.1, 1.0, d, p, xh, 0, 2).setup()
    FL, M = (x.cpu().numpy() for x in prob.run())
    Mo, Fo = O.dielectric_ct_second_moment({l: O.from_synth(sms[l]) for l in sms}, 3.0, 2.1, 1.0, d, p, xh, 0, 2)
    assert _rel(FL, Fo[2]) < 1e-8
    assert _rel(M, Mo) < 1e-8
    assert max(prob.berr.values()) <= max(64.0, 8.0 * math.sqrt(2 * 1920)) * 2.0**-52


def _closed_polyhedron(verts, tris):
    """Triangles oriented counter-clockwise seen from outside (normal . centroid > 0)."""
    verts = np.asarray(verts, dtype=np.float64)
    out = []
    for t in tris:
        a, b, c = verts[list(t)]
        n = np.cross(b - a, c - a)
        out.append(list(t) if np.dot(n, a + b + c) > 0 else [t[0], t[2], t[1]])
    vn = verts / np.linalg.norm(verts, axis=1, keepdims=True)
    return S.SurfaceMesh(verts, np.asarray(out, dtype=np.int32), vn)


@pytest.mark.parametrize("arith", ["ASM_FP64", "ASM_FF"])
def test_pmchwt_degenerate_meshes(arith):
    """Edge cases: a tetrahedron (every triangle pair touches, so the regular-pair launches add
    nothing) and an octahedron (vertex-disjoint pairs only between opposite faces), with no
    incident data (b NULL): the matrix against the oracle at 1e-12."""
    tet = _closed_polyhedron([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]],
                             [[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]])
    octa = _closed_polyhedron([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                              [[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4], [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]])
    for sm in (tet, octa):
        m, om = _mesh(sm)
        N = m.n_edges
        Z = torch.full((2 * N, 2 * N), 3.0, dtype=C128, device=DEV)
        F.assemble_pmchwt(m, 1.5, 2.1, 1.2, Z, arith=getattr(F, arith))
        Zo = O.assemble_pmchwt(om, 1.5, 2.1, 1.2)
        assert np.abs(Z.cpu().numpy() - Zo).max() <= 1e-12 * np.abs(Zo).max()

