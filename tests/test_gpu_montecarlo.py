"""Monte Carlo over random shapes on the GPU (Section V-C): sample surfaces
x_p + t xi_p n_p with xi = L z (fosb_field_samples), batched assembly and solves, sample
far-field moments (fosb_mc_moments).

* On the same standard normal draws, the GPU estimator and the oracle's (numpy Cholesky,
  LAPACK solve per sample surface) are the same computation: mean, covariance and
  pseudo-covariance agree at 1e-8.
* Against the first-order covariance (the FOSB result), the Monte Carlo covariance agrees
  within discretisation and sampling error, as the oracle's own Monte Carlo does."""
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


def test_field_samples_match_the_oracle_factor(F):
    sm = S.icosphere(2)
    m = F.mesh_create(sm.verts, sm.tris, sm.vnormals)
    z = S.gaussian_field_samples(5, m.nv, seed=3)
    xi = F.field_samples(m, z, F.COV_MATERN32, 0.3, 0.4)
    K = O.cov_kernel(sm.verts, sm.verts, "matern32", 0.3, 0.4) + 1e-12 * 0.09 * np.eye(m.nv)
    assert np.abs(xi - z @ np.linalg.cholesky(K).T).max() < 1e-12 * np.abs(xi).max()


def test_monte_carlo_matches_oracle_on_the_same_draws(F):
    from paper_2308_01457_gb300.montecarlo import MonteCarloProblem

    sm = S.icosphere(2)
    k, sig, ell, t = 2.0, 1.0, 0.5, 1e-3
    xh = S.hplane_directions(19)
    z = S.gaussian_field_samples(40, sm.verts.shape[0], seed=11)
    mc = MonteCarloProblem(sm, k, (0, 0, 1), (1, 0, 0), xh, z, F.COV_GAUSS, sig, ell, t, chunk=16).setup()
    F0, mean, cov, pcov = (x.cpu().numpy() for x in mc.run())
    F0o, Fso, covo, pcovo = O.monte_carlo(O.from_synth(sm), k, [0, 0, 1], [1, 0, 0], xh, "gauss", sig, ell, t, z)
    assert _rel(F0, F0o) < 1e-8
    assert _rel(mean, Fso.mean(axis=0)) < 1e-8
    # (F_s - F_0)/t amplifies the solves' rounding by 1/t: still far inside 1e-8
    assert _rel(cov, covo) < 1e-8 and _rel(pcov, pcovo) < 1e-8


def test_monte_carlo_approaches_first_order_covariance(F):
    from paper_2308_01457_gb300.montecarlo import MonteCarloProblem

    sm = S.icosphere(1)
    k, sig, ell, t = 2.0, 1.0, 0.5, 1e-3
    xh = S.hplane_directions(7)
    z = S.gaussian_field_samples(400, sm.verts.shape[0], seed=7)
    mc = MonteCarloProblem(sm, k, (0, 0, 1), (1, 0, 0), xh, z, F.COV_GAUSS, sig, ell, t).setup()
    F0, _, cov_mc, _ = (x.cpu().numpy() for x in mc.run())
    m = mc.base
    N = m.n_edges
    Z = torch.zeros((N, N), dtype=torch.complex128, device=DEV)
    b = torch.zeros((N, 1), dtype=torch.complex128, device=DEV)
    F.assemble_efie(m, k, Z, inc=F.incidence((0, 0, 1), (1, 0, 0)), b=b)
    lu = F.factor(Z, prec=F.MIXED)
    u = torch.zeros_like(b)
    F.solve(lu, b, u)
    Sig = torch.zeros((N, N), dtype=torch.complex128, device=DEV)
    F.covariance(m, lu, u, m, lu, u, k, Sig, F.COV_GAUSS, sig, ell)
    cov = torch.zeros((21, 21), dtype=torch.complex128, device=DEV)
    F.farfield_moments(m, k, xh, Sig, cov, m2=m)
    cov = cov.cpu().numpy()
    var_rel = np.linalg.norm(np.diag(cov_mc).real - np.diag(cov).real) / np.linalg.norm(np.diag(cov).real)
    assert var_rel < 0.35, var_rel
    assert _rel(cov_mc, cov) < 0.4


def test_dielectric_monte_carlo_matches_oracle_on_the_same_draws(F):
    """A dielectric sphere (eps_r = 2.1): every sample surface solved by the PMCHWT system in
    float-float assembly and MIXED solves, against the oracle's LAPACK solves on the same draws."""
    from paper_2308_01457_gb300.montecarlo import MonteCarloProblem

    sm = S.icosphere(2)
    k, er, sig, ell, t = 2.0, 2.1, 1.0, 0.5, 1e-3
    xh = S.hplane_directions(19)
    z = S.gaussian_field_samples(8, sm.verts.shape[0], seed=13)
    mc = MonteCarloProblem(sm, k, (0, 0, 1), (1, 0, 0), xh, z, F.COV_GAUSS, sig, ell, t, chunk=3,
                           eps_r=er).setup()
    F0, mean, cov, pcov = (x.cpu().numpy() for x in mc.run())
    F0o, Fso, covo, pcovo = O.monte_carlo_dielectric(O.from_synth(sm), k, er, 1.0, [0, 0, 1], [1, 0, 0], xh, "gauss",
                                                     sig, ell, t, z)
    assert _rel(F0, F0o) < 1e-8
    assert _rel(mean, Fso.mean(axis=0)) < 1e-8
    assert _rel(cov, covo) < 1e-8 and _rel(pcov, pcovo) < 1e-8
