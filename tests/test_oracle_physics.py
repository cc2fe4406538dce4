"""Pins of the oracle's method-level results against what the paper and the
mathematics fix: the Mie series (with its own optical-theorem and Rayleigh checks),
O(h^2) convergence (Section V-A), central finite differences of the discrete far
field for the shape derivative (Section III), the first-order t-scaling (Section V-B),
Monte Carlo for the covariance (Section V-C), and the combination-technique
bookkeeping against the printed Fichera and kite numbers (Sections IV-B, V-C, V-D)."""
import math
import os

import numpy as np
import pytest

import fosb_synth as S
import oracle as O
import oracle.mie as mie

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line:
            key, *vals = line.split()
            rows.setdefault(key, []).append([float(v) for v in vals])
    return rows


# ---------------------------------------------------------------- Mie series
def test_mie_optical_theorem():
    for ka in (0.3, 1.0, 4.0, 10.0):
        ext, sca = mie.cross_sections(ka, 1.0)
        assert abs(ext - sca) < 1e-10 * sca


def test_mie_rayleigh_backscatter():
    """Small PEC sphere: sigma_back -> 9 pi a^2 (ka)^4 (textbook Rayleigh limit)."""
    a, k = 1.0, 0.01
    F = mie.farfield(k, a, np.array([[0.0, 0.0, -1.0]]))
    sigma = np.sum(np.abs(F) ** 2) / (4 * np.pi)
    assert abs(sigma / (9 * np.pi * a**2 * (k * a) ** 4) - 1) < 1e-3


def test_mie_optical_limit_backscatter():
    """Large PEC sphere: sigma_back -> pi a^2 (geometric-optics limit)."""
    F = mie.farfield(60.0, 1.0, np.array([[0.0, 0.0, -1.0]]))
    sigma = np.sum(np.abs(F) ** 2) / (4 * np.pi)
    assert abs(sigma / np.pi - 1) < 0.05


def test_oracle_converges_to_mie_at_second_order(oracle_mod):
    """Far field of the Galerkin solution vs Mie: O(h^2) (Section V-A)."""
    xh = S.hplane_directions(37)
    Fm = mie.farfield(1.0, 1.0, xh)
    errs = []
    for lvl in (1, 2, 3):
        m = O.from_synth(S.icosphere(lvl))
        Z = O.assemble_z(m, 1.0)
        u = O.solve(Z, O.rhs_planewave(m, 1.0, [0, 0, 1], [1, 0, 0])[:, 0])
        F = (O.farfield_matrix(m, 1.0, xh) @ u).reshape(-1, 3)
        errs.append(np.linalg.norm(F - Fm) / np.linalg.norm(Fm))
    assert errs[-1] < 0.01, errs
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


# ---------------------------------------------------------------- shape derivative
def _far(verts, sm, k, xh, d=(0, 0, 1), p=(1, 0, 0)):
    m = O.RWGMesh(verts, sm.tris, sm.vnormals)
    Z = O.assemble_z(m, k)
    u = O.solve(Z, O.rhs_planewave(m, k, d, p)[:, 0])
    return O.farfield_matrix(m, k, xh) @ u, m, Z, u


def test_shape_derivative_matches_finite_differences(oracle_mod):
    """A Z^{-1} B xi vs central FD of the discrete far field under x_p -> x_p + h xi_p n_p:
    the gap is discretisation error (continuous vs discrete derivative) and falls like h^2."""
    xh = S.hplane_directions(19)
    k = 2.0
    gaps = []
    for lvl in (1, 2):
        sm = S.icosphere(lvl)
        xi = np.sin(2 * sm.verts[:, 0]) + sm.verts[:, 1] * sm.verts[:, 2]
        F0, m, Z, u = _far(sm.verts, sm, k, xh)
        dF = O.farfield_matrix(m, k, xh) @ np.linalg.solve(Z, O.sd_rhs(m, k, u) @ xi)
        h = 1e-4
        Fp = _far(sm.verts + h * xi[:, None] * sm.vnormals, sm, k, xh)[0]
        Fn = _far(sm.verts - h * xi[:, None] * sm.vnormals, sm, k, xh)[0]
        fd = (Fp - Fn) / (2 * h)
        gaps.append(np.linalg.norm(fd - dF) / np.linalg.norm(fd))
    assert gaps[1] < 0.05, gaps
    assert gaps[0] / gaps[1] > 3.0, gaps


def test_first_order_t_scaling(oracle_mod):
    """ZOA error |F_t - F| is O(t) and FOA error |F_t - F - t F'| is O(t^2) (Section V-B),
    for the deterministic normal perturbation xi_p = z_p^2 on the 480-edge sphere."""
    xh = S.hplane_directions(19)
    k = 2.0
    sm = S.icosphere(2)
    xi = sm.verts[:, 2] ** 2
    F0, m, Z, u = _far(sm.verts, sm, k, xh)
    dF = O.farfield_matrix(m, k, xh) @ np.linalg.solve(Z, O.sd_rhs(m, k, u) @ xi)
    ts = [0.02, 0.01, 0.005]
    zoa, foa = [], []
    for t in ts:
        Ft = _far(sm.verts + t * xi[:, None] * sm.vnormals, sm, k, xh)[0]
        zoa.append(np.linalg.norm(Ft - F0))
        foa.append(np.linalg.norm(Ft - F0 - t * dF))
    # ZOA halves with t; FOA shrinks faster than ZOA (second order up to the
    # discretisation floor of the continuous shape derivative)
    assert 1.8 < zoa[0] / zoa[1] < 2.2 and 1.8 < zoa[1] / zoa[2] < 2.2
    assert all(f < 0.2 * z for f, z in zip(foa, zoa)), (foa, zoa)


# ---------------------------------------------------------------- covariance
def test_covariance_identities(oracle_mod):
    """Sigma = Z1^{-1} B1 K B2^H Z2^{-H}: Hermitian PSD on the diagonal block, the mirror
    identity Sigma_{21} = Sigma_{12}^H, and the per-mode expansion with K = R R^T."""
    k = 2.0
    lv = {}
    xh = S.hplane_directions(7)
    for l, lvl in ((0, 1), (1, 2)):
        lv[l] = O.nominal_level(O.from_synth(S.icosphere(lvl)), k, [0, 0, 1], [1, 0, 0], xh)
    K11 = O.cov_kernel(lv[0].mesh.verts, lv[0].mesh.verts, "gauss", 0.01, 0.5)
    S11 = O.covariance(lv[0].Z, lv[0].B, lv[0].Z, lv[0].B, K11)
    assert np.abs(S11 - S11.conj().T).max() < 1e-12 * np.abs(S11).max()
    assert np.linalg.eigvalsh(0.5 * (S11 + S11.conj().T)).min() > -1e-10 * np.abs(S11).max()
    K10 = O.cov_kernel(lv[1].mesh.verts, lv[0].mesh.verts, "matern32", 0.01, 0.5)
    S10 = O.covariance(lv[1].Z, lv[1].B, lv[0].Z, lv[0].B, K10)
    S01 = O.covariance(lv[0].Z, lv[0].B, lv[1].Z, lv[1].B, K10.T)
    assert np.abs(S01 - S10.conj().T).max() < 1e-12 * np.abs(S10).max()
    # per-mode route: K = R R^T (eigen-decomposition), Sigma = sum_q y1_q y1_q^H
    w, V = np.linalg.eigh(K11)
    R = V * np.sqrt(np.maximum(w, 0))
    Y = np.linalg.solve(lv[0].Z, lv[0].B @ R)
    assert np.abs(Y @ Y.conj().T - S11).max() < 1e-9 * np.abs(S11).max()


def test_monte_carlo_matches_first_order_covariance(oracle_mod):
    """Perturbed-mesh Monte Carlo (Section V-C, oracle.monte_carlo) on the 120-edge sphere,
    xi ~ N(0, K), t xi n_p displacements: the sample covariance of (F_t - F)/t approaches
    A Sigma A^H within discretisation (about 15% at this level, see the FD pin) and sampling
    error, and the sample variance of RCS_dB over the sample surfaces approaches the delta method."""
    xh = S.hplane_directions(7)
    k, sigma, ell = 2.0, 1.0, 0.5
    sm = S.icosphere(1)
    F0, m, Z, u = _far(sm.verts, sm, k, xh)
    A = O.farfield_matrix(m, k, xh)
    B = O.sd_rhs(m, k, u)
    K = O.cov_kernel(m.verts, m.verts, "gauss", sigma, ell)
    cov = A @ O.covariance(Z, B, Z, B, K) @ A.conj().T
    M, t = 400, 1e-3
    F0m, Fs, mc, mc_p = O.monte_carlo(m, k, [0, 0, 1], [1, 0, 0], xh, "gauss", sigma, ell, t,
                                      S.gaussian_field_samples(M, m.nv, seed=7))
    assert np.abs(F0m - F0).max() <= 1e-14 * np.abs(F0).max()
    var_rel = np.linalg.norm(np.diag(mc).real - np.diag(cov).real) / np.linalg.norm(np.diag(cov).real)
    assert var_rel < 0.35, var_rel
    full_rel = np.linalg.norm(mc - cov) / np.linalg.norm(cov)
    assert full_rel < 0.4, full_rel
    # RCS_dB of the perturbed meshes: its sample variance / t^2 against the delta method on
    # the first-order covariance and pseudo-covariance (the paper's MC-vs-FOSB comparison)
    pcov = A @ O.covariance(Z, B, Z, B, K, pseudo=True) @ A.T
    pred = O.rcs_variance_db(F0.reshape(-1, 3), cov, pcov)
    rcs = O.rcs_db(Fs.reshape(M, -1, 3))
    ratio = np.var(rcs, axis=0) / t**2 / pred
    assert np.abs(np.median(ratio) - 1) < 0.25 and np.abs(ratio - 1).max() < 0.6, ratio


# ---------------------------------------------------------------- combination technique
def test_ct_index_sets():
    lp, lm = O.ct_index_sets(0, 4)
    assert lp == [(0, 4), (1, 3), (2, 2), (3, 1), (4, 0)]
    assert lm == [(0, 3), (1, 2), (2, 1), (3, 0)]
    herm = O.ct_hermitian_blocks(0, 4)
    assert herm == [((2, 2), 1), ((3, 1), 1), ((4, 0), 1), ((2, 1), -1), ((3, 0), -1)]
    assert O.ct_index_sets(2, 2) == ([(2, 2)], [])


def test_ct_dofs_fichera_and_kite():
    g = _read_golden("fichera_ct.txt")
    N = dict(enumerate(int(v) for v in g["N"][0]))
    printed = {(int(a), int(b)): v for a, b, v in g["block"]}
    for (a, b), v in printed.items():
        exact = N[a] * N[b]
        if (a, b) == (1, 0):
            assert abs(exact - 2.14e5) < 1e3  # the printed 2.10e5 is a typo of 2.14e5
        else:
            assert abs(exact - v) <= 0.005e5
    total, mx = O.ct_dofs(N, 0, 2, hermitian=True)
    full = N[2] ** 2
    assert abs(full - g["full"][0][2]) / full < 0.03
    # the paper's 5.87 uses the printed rounded values; the exact efficiency is 6.02
    eff_printed = g["full"][0][2] / sum(printed.values())
    assert abs(eff_printed - g["efficiency"][0][0]) < 0.01
    assert abs(full / total - 6.017) < 1e-3
    kite = _read_golden("kite_ct.txt")
    NL = kite["N_L"][0][0]
    assert abs(NL**2 - kite["N_L_squared"][0][0]) / NL**2 < 0.002
    assert abs(NL**2 / kite["N_hat"][0][0] - kite["efficiency_total"][0][0]) < 0.01
    assert abs(NL**2 / kite["N_hat_max"][0][0] - kite["efficiency_max"][0][0]) < 0.01


def test_ct_single_level_is_full_tensor(oracle_mod):
    """With L0 = L the combination technique is the full tensor A Sigma A^H."""
    xh = S.hplane_directions(7)
    lev = {1: O.nominal_level(O.from_synth(S.icosphere(1)), 2.0, [0, 0, 1], [1, 0, 0], xh)}
    ct = O.ct_farfield_covariance(lev, 1, 1, "gauss", 0.01, 0.5)
    a = lev[1]
    K = O.cov_kernel(a.mesh.verts, a.mesh.verts, "gauss", 0.01, 0.5)
    full = a.A @ O.covariance(a.Z, a.B, a.Z, a.B, K) @ a.A.conj().T
    assert np.abs(ct - full).max() < 1e-14 * np.abs(full).max()


def test_ct_converges_to_full_tensor(oracle_mod):
    """CT far-field covariance over levels {0,1,2} approaches the finest full tensor
    (Section V-A, Fig. 3(d)): closer than the coarsest level alone."""
    xh = S.hplane_directions(7)
    k = 1.5
    lev = {l: O.nominal_level(O.from_synth(S.icosphere(l + 1)), k, [0, 0, 1], [1, 0, 0], xh) for l in (0, 1, 2)}
    ct = O.ct_farfield_covariance(lev, 0, 2, "gauss", 1.0, 0.6)
    full2 = O.ct_farfield_covariance(lev, 2, 2, "gauss", 1.0, 0.6)
    full0 = O.ct_farfield_covariance(lev, 0, 0, "gauss", 1.0, 0.6)
    e_ct = np.linalg.norm(ct - full2) / np.linalg.norm(full2)
    e_0 = np.linalg.norm(full0 - full2) / np.linalg.norm(full2)
    assert e_ct < 0.5 * e_0, (e_ct, e_0)
