"""Pins of the oracle's covariance kernel and RCS moments by routes that do not share
their formulas.

* ``cov_kernel`` (the second moment M^2[v_n] of the normal velocity, Section III, sampled
  at the mesh vertices): Bochner's theorem writes a stationary kernel as the average of
  cos(w . (x - y)) over its spectral measure.  The Gaussian sigma^2 exp(-r^2/(2 l^2)) has
  w ~ N(0, I / l^2); the Matern-3/2 kernel has the Student-t spectral measure with 3
  degrees of freedom, w = (z / l) sqrt(3 / u) with z ~ N(0, I) and u ~ chi^2_3.  A seeded
  Monte Carlo average over w is compared with the oracle within its sampling bound, plus
  literal values at r = 0, l/2 and l.
* ``rcs_variance_db`` (the delta-method variance of RCS_dB, eq. RCS with the pseudo-
  covariance): for F' = G xi with real xi ~ N(0, K) the linearisation of RCS_dB(F + F')
  is c^T xi, whose variance is exactly c^T K c.  The gradient c is taken by central
  differences of ``rcs_db`` in xi-space, so neither the 1/2, the pseudo-covariance term
  nor the conjugates of the delta-method formula enter the expected value.  A Monte
  Carlo over xi of the nonlinear RCS_dB checks the same at small amplitude.
* ``rcs_db`` (sigma = |F|^2 / (4 pi), Section II-C): the PEC sphere's Mie backscatter
  against the textbook Rayleigh (9 pi a^2 (ka)^4) and optical (pi a^2) limits.
"""
import math

import numpy as np
import pytest

import fosb_synth as S
import oracle as O
import oracle.mie as mie


def _pairs(seed=3, n=40):
    """Vertex pairs of the 320-triangle unit icosphere with chordal distances spread
    over [0, 2] (r = 0 included)."""
    v = S.icosphere(2).verts
    rng = np.random.default_rng(seed)
    p = rng.integers(0, v.shape[0], n)
    q = rng.integers(0, v.shape[0], n)
    q[0] = p[0]
    return v[p], v[q]


def _spectral_average(x1, x2, sample_w, m_total=2_000_000, chunk=200_000, seed=0):
    """Monte Carlo mean of cos(w . (x1_i - x2_i)) over w drawn by sample_w(rng, m)."""
    rng = np.random.default_rng(seed)
    r = (x1 - x2).T  # 3 x P
    acc = np.zeros(r.shape[1])
    for _ in range(m_total // chunk):
        w = sample_w(rng, chunk)
        acc += np.cos(w @ r).sum(axis=0)
    return acc / m_total


@pytest.mark.parametrize("ell,sigma", [(0.5, 1.0), (0.3, 0.005)])
def test_gaussian_kernel_matches_its_spectral_measure(ell, sigma):
    x1, x2 = _pairs()
    mc = _spectral_average(x1, x2, lambda rng, m: rng.standard_normal((m, 3)) / ell)
    K = np.array([O.cov_kernel(a[None], b[None], "gauss", sigma, ell)[0, 0] for a, b in zip(x1, x2)])
    # each cos term has variance <= 1/2: 6 standard errors of the mean
    assert np.abs(K / sigma**2 - mc).max() < 6 * math.sqrt(0.5 / 2_000_000)
    assert np.ptp(np.linalg.norm(x1 - x2, axis=1)) > 1.5  # the pairs span the kernel's range


@pytest.mark.parametrize("ell,sigma", [(0.5, 1.0), (0.2, 0.002)])
def test_matern32_kernel_matches_its_spectral_measure(ell, sigma):
    x1, x2 = _pairs(seed=4)

    def student_t3(rng, m):
        z = rng.standard_normal((m, 3))
        u = rng.chisquare(3, m)
        return z / ell * np.sqrt(3.0 / u)[:, None]

    mc = _spectral_average(x1, x2, student_t3, seed=1)
    K = np.array([O.cov_kernel(a[None], b[None], "matern32", sigma, ell)[0, 0] for a, b in zip(x1, x2)])
    assert np.abs(K / sigma**2 - mc).max() < 6 * math.sqrt(0.5 / 2_000_000)


def test_kernel_literal_values():
    """K(0) = sigma^2; Gaussian e^{-1/8}, e^{-1/2} and Matern (1 + sqrt3/2) e^{-sqrt3/2},
    (1 + sqrt3) e^{-sqrt3} at r = l/2 and r = l (decimals evaluated to 25 digits)."""
    sig, ell = 0.7, 0.4
    x0 = np.zeros((1, 3))
    pts = np.array([[0.0, 0.0, 0.0], [0.0, ell / 2, 0.0], [ell, 0.0, 0.0]])
    g = O.cov_kernel(x0, pts, "gauss", sig, ell)[0] / sig**2
    m = O.cov_kernel(x0, pts, "matern32", sig, ell)[0] / sig**2
    np.testing.assert_allclose(g, [1.0, 0.8824969025845954, 0.6065306597126334], rtol=1e-14)
    np.testing.assert_allclose(m, [1.0, 0.7848876539574507, 0.4833577245965077], rtol=1e-14)
    assert O.cov_kernel(x0, x0, "gauss", sig, ell)[0, 0] == pytest.approx(sig**2, rel=1e-15)


def _moment_problem(seed, n_dir=5, V=12):
    """A random complex far field F (n_dir x 3), a random linear map G (3 n_dir x V) and a
    random SPD K: F' = G xi with xi ~ N(0, K) has E[F'F'^H] = G K G^H, E[F'F'^T] = G K G^T."""
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((n_dir, 3)) + 1j * rng.standard_normal((n_dir, 3))
    G = rng.standard_normal((3 * n_dir, V)) + 1j * rng.standard_normal((3 * n_dir, V))
    R = rng.standard_normal((V, V))
    K = R @ R.T + 0.1 * np.eye(V)
    return F, G, K


def test_rcs_variance_is_the_exact_variance_of_the_linearised_rcs():
    for seed in range(4):
        F, G, K = _moment_problem(seed)
        n_dir, V = F.shape[0], K.shape[0]
        got = O.rcs_variance_db(F, G @ K @ G.conj().T, G @ K @ G.T)
        h = 1e-5
        c = np.zeros((n_dir, V))
        for p in range(V):
            dF = G[:, p].reshape(n_dir, 3)
            c[:, p] = (O.rcs_db(F + h * dF) - O.rcs_db(F - h * dF)) / (2 * h)
        want = np.einsum("dp,pq,dq->d", c, K, c)
        np.testing.assert_allclose(got, want, rtol=1e-7)


def test_rcs_variance_matches_monte_carlo_of_the_nonlinear_rcs():
    """Sample variance of RCS_dB(F + t G xi) / t^2 at small t: the delta method within the
    sampling error (M = 40000: about 1.5% one standard error)."""
    F, G, K = _moment_problem(7)
    n_dir, V = F.shape[0], K.shape[0]
    pred = O.rcs_variance_db(F, G @ K @ G.conj().T, G @ K @ G.T)
    rng = np.random.default_rng(8)
    L = np.linalg.cholesky(K)
    M, t = 40000, 1e-4
    xi = rng.standard_normal((M, V)) @ L.T
    Fp = F[None] + t * (xi @ G.T).reshape(M, n_dir, 3)
    mc = np.var(O.rcs_db(Fp), axis=0) / t**2
    assert np.abs(mc / pred - 1).max() < 0.06, (mc, pred)


def test_rcs_db_rayleigh_and_optical_limits():
    """Mie backscatter of a PEC sphere in dB against 10 log10 of the textbook limits."""
    a = 1.0
    for k in (0.01, 0.02):
        F = mie.farfield(k, a, np.array([[0.0, 0.0, -1.0]]))
        assert O.rcs_db(F)[0] == pytest.approx(10 * math.log10(9 * math.pi * a**2 * (k * a) ** 4), abs=0.01)
    F = mie.farfield(60.0, a, np.array([[0.0, 0.0, -1.0]]))
    assert O.rcs_db(F)[0] == pytest.approx(10 * math.log10(math.pi * a**2), abs=0.25)
    # a single complex component is |F_c|^2 / (4 pi) in dB
    assert O.rcs_db(np.array([2.0 + 0j]))[0] == pytest.approx(10 * math.log10(1 / math.pi), rel=1e-14)
