"""Sphere Mie series: the closed-form scattered far field the paper checks its
sphere experiment against (Section V-A, "MIE series"), for the PEC sphere and for
the homogeneous dielectric sphere of the PMCHWT problem.

TEST INFRASTRUCTURE ONLY (part of the oracle's pins).

Conventions: time factor exp(-i w t) (Section II-A), incident field x_hat exp(ikz).
With psi_n(x) = x j_n(x), xi_n(x) = x h_n^(1)(x), the PEC limit of the Lorenz-Mie
coefficients is a_n = psi_n'(x)/xi_n'(x), b_n = psi_n(x)/xi_n(x) (x = ka).  The
scattered field behaves as E_s ~ exp(ikr)/(-ikr) [cos(phi) S2 e_theta - sin(phi) S1 e_phi]
with S1 = sum (2n+1)/(n(n+1)) (a_n pi_n + b_n tau_n), S2 = sum (2n+1)/(n(n+1)) (a_n tau_n + b_n pi_n),
and the far field of Section II-C (E_s ~ exp(ik|x|)/(4 pi |x|) F) is F = (4 pi i / k) [...].
For a dielectric sphere (relative index m = sqrt(eps_r mu_r), relative permeability mu_r)
the coefficients are Bohren and Huffman's (Absorption and Scattering of Light by Small
Particles, eq. 4.53):
  a_n = [m^2 j_n(mx) psi_n'(x) - mu_r j_n(x) psi_n'(mx)] / [m^2 j_n(mx) xi_n'(x) - mu_r h_n(x) psi_n'(mx)],
  b_n = [mu_r j_n(mx) psi_n'(x) - j_n(x) psi_n'(mx)] / [mu_r j_n(mx) xi_n'(x) - h_n(x) psi_n'(mx)],
which tend to the PEC coefficients as m grows.
The Bessel functions are scipy.special's (a library primitive).
"""
from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def coefficients(x: float, nmax: int | None = None):
    if nmax is None:
        nmax = int(np.ceil(x + 4.05 * x ** (1.0 / 3.0) + 10))
    n = np.arange(1, nmax + 1)
    jn = spherical_jn(n, x)
    yn = spherical_yn(n, x)
    jnp = spherical_jn(n, x, derivative=True)
    ynp = spherical_yn(n, x, derivative=True)
    hn = jn + 1j * yn
    hnp = jnp + 1j * ynp
    psi = x * jn
    dpsi = jn + x * jnp
    xi = x * hn
    dxi = hn + x * hnp
    a = dpsi / dxi
    b = psi / xi
    return n, a, b


def coefficients_dielectric(x: float, eps_r: float, mu_r: float, nmax: int | None = None):
    m = np.sqrt(eps_r * mu_r)
    if nmax is None:  # the series converges once n passes the outer size parameter x
        nmax = int(np.ceil(x + 4.05 * x ** (1.0 / 3.0) + 10))
    n = np.arange(1, nmax + 1)
    mx = m * x
    jx, yx = spherical_jn(n, x), spherical_yn(n, x)
    djx, dyx = spherical_jn(n, x, derivative=True), spherical_yn(n, x, derivative=True)
    jm, djm = spherical_jn(n, mx), spherical_jn(n, mx, derivative=True)
    hx = jx + 1j * yx
    dpsi_x = jx + x * djx                  # psi_n'(x)
    dxi_x = hx + x * (djx + 1j * dyx)      # xi_n'(x)
    dpsi_m = jm + mx * djm                 # psi_n'(mx)
    a = (m * m * jm * dpsi_x - mu_r * jx * dpsi_m) / (m * m * jm * dxi_x - mu_r * hx * dpsi_m)
    b = (mu_r * jm * dpsi_x - jx * dpsi_m) / (mu_r * jm * dxi_x - hx * dpsi_m)
    return n, a, b


def angular(n_max: int, mu: np.ndarray):
    """pi_n = P_n^1(mu)/sin(theta), tau_n = dP_n^1/dtheta by the upward recurrences
    pi_n = ((2n-1) mu pi_{n-1} - n pi_{n-2})/(n-1), tau_n = n mu pi_n - (n+1) pi_{n-1}."""
    mu = np.asarray(mu, dtype=np.float64)
    pi = np.zeros((n_max + 1,) + mu.shape)
    tau = np.zeros_like(pi)
    pi[1] = 1.0
    tau[1] = mu
    for n in range(2, n_max + 1):
        pi[n] = ((2 * n - 1) * mu * pi[n - 1] - n * pi[n - 2]) / (n - 1)
        tau[n] = n * mu * pi[n] - (n + 1) * pi[n - 1]
    return pi[1:], tau[1:]


def amplitudes(ka: float, theta: np.ndarray, coef=None):
    n, a, b = coefficients(ka) if coef is None else coef
    pi, tau = angular(n[-1], np.cos(theta))
    c = ((2 * n + 1) / (n * (n + 1)))[:, None]
    S1 = np.sum(c * (a[:, None] * pi + b[:, None] * tau), axis=0)
    S2 = np.sum(c * (a[:, None] * tau + b[:, None] * pi), axis=0)
    return S1, S2


def farfield(k: float, radius: float, xhat: np.ndarray, eps_r: float | None = None, mu_r: float = 1.0) -> np.ndarray:
    """F(xh) (n_dir x 3, complex) for the unit-amplitude x-polarised wave along +z, PEC
    sphere (eps_r None) or dielectric sphere (eps_r, mu_r relative to the outside)."""
    xhat = np.atleast_2d(xhat)
    theta = np.arccos(np.clip(xhat[:, 2], -1.0, 1.0))
    phi = np.arctan2(xhat[:, 1], xhat[:, 0])
    coef = None if eps_r is None else coefficients_dielectric(k * radius, eps_r, mu_r)
    S1, S2 = amplitudes(k * radius, theta, coef)
    e_th = np.stack([np.cos(theta) * np.cos(phi), np.cos(theta) * np.sin(phi), -np.sin(theta)], axis=1)
    e_ph = np.stack([-np.sin(phi), np.cos(phi), np.zeros_like(phi)], axis=1)
    amp = (np.cos(phi) * S2)[:, None] * e_th - (np.sin(phi) * S1)[:, None] * e_ph
    return (4j * np.pi / k) * amp


def cross_sections(k: float, radius: float, eps_r: float | None = None, mu_r: float = 1.0):
    """(sigma_ext, sigma_sca) from the optical theorem and the coefficient sum."""
    n, a, b = coefficients(k * radius) if eps_r is None else coefficients_dielectric(k * radius, eps_r, mu_r)
    ext = (2 * np.pi / k**2) * np.sum((2 * n + 1) * (a + b).real)
    sca = (2 * np.pi / k**2) * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    return ext, sca
