"""GPU adjoint shape gradient (fosb_rcs_monostatic with grad, and the FosbRCS autograd
function) against the oracle's forward-mode derivatives of the same discrete RCS.
Tolerance 1e-8 relative (FP64 kernels, refined solves)."""
import numpy as np
import pytest

import fosb_synth as S
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_01457_gb300 as mod

    mod.build.build()
    O.build()
    return mod


def _solve(F, sm, k, d, p):
    m = F.mesh_create(sm.verts, sm.tris, sm.vnormals)
    inc = F.incidence(d, p)
    N, n = m.n_edges, inc.shape[0]
    Z = torch.zeros((N, N), dtype=torch.complex128, device="cuda")
    b = torch.zeros((N, n), dtype=torch.complex128, device="cuda")
    F.assemble_efie(m, k, Z, inc=inc, b=b)
    lu = F.factor(Z, prec=F.MIXED)
    U = torch.zeros_like(b)
    F.solve(lu, b, U)
    return m, inc, Z, lu, U


@pytest.mark.parametrize("lvl,ncoord", [(1, 60), (2, 18)])
def test_adjoint_gradient_matches_oracle(F, lvl, ncoord):
    sm = S.icosphere(lvl)
    k = 3.0
    d, p, _ = S.monostatic_directions(8)
    m, inc, Z, lu, U = _solve(F, sm, k, d, p)
    rng = np.random.default_rng(lvl)
    w = rng.standard_normal(len(d))
    grad = torch.zeros((sm.nv, 3), dtype=torch.float64, device="cuda")
    sig = F.rcs_monostatic(m, k, inc, U, lu=lu, weights=w, grad=grad)
    sel = rng.choice(sm.nv * 3, size=ncoord, replace=False)
    coords = [(int(s // 3), int(s % 3)) for s in sel]
    sig_o, J = O.rcs_monostatic_jacobian(O.from_synth(sm), k, d, p, coords)
    assert np.abs(sig - sig_o).max() <= 1e-9 * np.abs(sig_o).max()
    g = grad.cpu().numpy().reshape(-1)[sel]
    go = w @ J
    assert np.linalg.norm(g - go) <= 1e-8 * np.linalg.norm(go), (g[:5], go[:5])


def test_autograd_function_backward(F):
    from paper_2308_01457_gb300.autograd import FosbRCS

    sm = S.icosphere(1)
    k = 2.0
    d, p, _ = S.monostatic_directions(8)
    verts = torch.tensor(sm.verts, dtype=torch.float64, requires_grad=True)
    sig_db = FosbRCS.apply(verts, sm.tris, k, d, p, True)
    wts = torch.linspace(-1.0, 1.0, len(d), dtype=torch.float64)
    (sig_db * wts).sum().backward()
    coords = [(v, c) for v in range(0, sm.nv, 3) for c in range(3)]
    sig_o, J = O.rcs_monostatic_jacobian(O.from_synth(sm), k, d, p, coords)
    assert np.abs(sig_db.detach().numpy() - 10 * np.log10(sig_o)).max() < 1e-8
    # d(10 log10 sigma) = 10/ln10 dsigma/sigma
    go = (wts.numpy() * 10.0 / np.log(10.0) / sig_o) @ J
    g = np.array([verts.grad[v, c].item() for v, c in coords])
    assert np.linalg.norm(g - go) <= 1e-8 * np.linalg.norm(go)


def test_adjoint_gradient_against_fosb_shape_derivative(F):
    """The adjoint gradient (the exact derivative of the discrete RCS) projected on the
    vertex normals, against the FOSB shape-derivative path of Section III:
    d sigma_i / d xi_p = 2 Re(conj(F_i) . A_i Z^{-1} B_i e_p) / (4 pi), with B the shape-
    derivative right-hand side for v_n = psi_p (n_p . n_T).  One differentiates the discrete
    surface and the other the continuous one, so they agree only to discretisation error:
    the gap must fall under refinement (about 5.7x per level here), not reach 1e-8."""
    k = 2.0
    d, p, _ = S.monostatic_directions(8)
    w = np.random.default_rng(4).standard_normal(len(d))
    gaps = []
    for lvl in (1, 2, 3):
        sm = S.icosphere(lvl)
        m = F.mesh_create(sm.verts, sm.tris, sm.vnormals)
        N = m.n_edges
        inc = F.incidence(d, p)
        Z = torch.zeros((N, N), dtype=torch.complex128, device="cuda")
        B = torch.zeros((N, len(d)), dtype=torch.complex128, device="cuda")
        F.assemble_efie(m, k, Z, inc=inc, b=B)
        lu = F.factor(Z, prec=F.FP64)
        U = torch.zeros_like(B)
        F.solve(lu, B, U)
        grad = torch.zeros((sm.nv, 3), dtype=torch.float64, device="cuda")
        F.rcs_monostatic(m, k, inc, U, lu=lu, weights=w, grad=grad)
        gn = np.sum(grad.cpu().numpy() * sm.vnormals, axis=1)
        om = O.from_synth(sm)
        Zo = O.assemble_z(om, k)
        Uo = O.solve(Zo, O.rhs_planewave(om, k, d, p))
        h = np.zeros(om.nv)
        for i in range(len(d)):
            A = O.farfield_matrix(om, k, -d[i][None])
            Fi = A @ Uo[:, i]
            dF = A @ np.linalg.solve(Zo, O.sd_rhs(om, k, Uo[:, i]))
            h += w[i] * 2.0 * np.real(np.conj(Fi) @ dF) / (4.0 * np.pi)
        gaps.append(np.linalg.norm(gn - h) / np.linalg.norm(h))
    assert gaps[0] / gaps[1] > 3.0 and gaps[1] / gaps[2] > 3.0, gaps
    assert gaps[2] < 0.01, gaps
