"""GMRES-based iterative refinement (the Krylov part of the solver stack): where plain
refinement with complex64 factors stalls because kappa(Z) u_32 is not small, the refined
solve still reaches FP64 backward error by solving each correction equation with GMRES
preconditioned by the same factors."""
import math

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


def _ill_conditioned(n, kappa, seed=5):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    W, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    s = np.logspace(0.0, -math.log10(kappa), n)
    A = (U * s) @ W.conj().T
    x = rng.standard_normal((n, 2)) + 1j * rng.standard_normal((n, 2))
    return A, A @ x


def test_gmres_ir_converges_where_refinement_stalls(F):
    n, kappa = 700, 3e7  # ragged size; kappa u_32 ~ 2: plain refinement cannot contract
    A, b = _ill_conditioned(n, kappa)
    Ad = torch.tensor(A, dtype=torch.complex128, device=DEV)
    bd = torch.tensor(b, dtype=torch.complex128, device=DEV)
    lu = F.factor(Ad, prec=F.MIXED)
    x = torch.zeros_like(bd)
    with pytest.raises(F.FosbError) as e:
        F.solve(lu, bd, x, solver=F.REFINE_IR)
    assert e.value.status == F.FOSB_ERR_NOT_CONVERGED
    x = torch.zeros_like(bd)
    _, iters, berr = F.solve(lu, bd, x)  # default: refinement, then GMRES-IR
    xh = x.cpu().numpy()
    tol = max(64.0, 8.0 * math.sqrt(n)) * 2.0**-52
    assert berr <= tol and iters > 10
    # an independent complex128 backward error, and LAPACK's solution to kappa * eps
    r = b - A @ xh
    be = np.abs(r).max(axis=0) / (np.abs(A).sum(axis=1).max() * np.abs(xh).max(axis=0) + np.abs(b).max(axis=0))
    assert be.max() <= 2.0 * tol, be  # the stopping rule's bound (x2 for a different summation order)
    xl = np.linalg.solve(A, b)
    assert np.linalg.norm(xh - xl) / np.linalg.norm(xl) < 100 * kappa * 2.0**-52


def test_gmres_ir_solution_matches_oracle(F):
    sm = S.icosphere(3)
    k = 3.0
    m = F.mesh_create(sm.verts, sm.tris, sm.vnormals)
    N = m.n_edges
    d = S.fibonacci_directions(3)
    p = np.asarray(S.polarisation_for(d)).reshape(-1, 3)
    Z = torch.zeros((N, N), dtype=torch.complex128, device=DEV)
    B = torch.zeros((N, 3), dtype=torch.complex128, device=DEV)
    F.assemble_efie(m, k, Z, inc=F.incidence(d, p), b=B, arith=F.ASM_FF, prec=F.MIXED)
    lu = F.factor(Z, prec=F.MIXED)
    X = torch.zeros_like(B)
    _, iters, berr = F.solve(lu, B, X, solver=F.REFINE_GMRES)
    assert iters > 0 and berr <= max(64.0, 8.0 * math.sqrt(N)) * 2.0**-52
    om = O.from_synth(sm)
    Xo = O.solve(O.assemble_z(om, k), O.rhs_planewave(om, k, d, p))
    Xg = X.cpu().numpy()
    for c in range(3):
        assert np.linalg.norm(Xg[:, c] - Xo[:, c]) / np.linalg.norm(Xo[:, c]) < 1e-8
