"""Pins of the oracle's dielectric (PMCHWT) path, Section II-C eq. pmchwt, against what
the mathematics fixes rather than against the oracle itself:

  * the dielectric-sphere Mie series (Section V-A), itself pinned by the optical
    theorem of a lossless sphere, the Rayleigh limit of a small sphere, the vanishing
    of every coefficient for a sphere of the outside medium, and its PEC limit;
  * second-order convergence of the Galerkin far field to that series, for eps_r != 1
    (the paper's sphere parameters) and for mu_r != 1 (which alone exercises the
    eta scaling of A^_1);
  * the transparent scatterer (eps_r = mu_r = 1): the exact solution is the incident
    Cauchy data and the scattered far field must vanish under refinement (the
    Calderon identity A_0 xi_inc = xi_inc / 2 of an interior field);
  * the MFIO point formula against the curl of the vector potential taken by central
    differences, and the symmetry of the MFIO Galerkin matrix in the x-pairing.
A dropped term, a wrong sign, a transposed cross product or a misplaced eta fails one
of them."""
import math

import numpy as np
import pytest

import fosb_synth as S
import oracle as O
import oracle.mie as mie


# ---------------------------------------------------------------- dielectric Mie series
def test_dielectric_mie_optical_theorem():
    """Lossless sphere: extinction (optical theorem) = scattering (coefficient sum)."""
    for ka, er, mr in ((0.3, 2.1, 1.0), (2.0, 2.1, 1.0), (3.0, 1.9, 1.0), (1.5, 2.0, 1.5), (6.0, 4.0, 1.0)):
        ext, sca = mie.cross_sections(ka, 1.0, eps_r=er, mu_r=mr)
        assert abs(ext - sca) < 1e-10 * sca, (ka, er, mr, ext, sca)


def test_dielectric_mie_rayleigh_limit():
    """Small dielectric sphere: the induced dipole p = 4 pi eps0 a^3 (eps_r - 1)/(eps_r + 2) E0
    radiates F = 4 pi k^2 a^3 (eps_r - 1)/(eps_r + 2) (xh x p) x xh (textbook Rayleigh limit)."""
    k, a, er = 0.01, 1.0, 2.1
    xh = S.hplane_directions(7)
    F = mie.farfield(k, a, xh, eps_r=er)
    p = np.array([1.0, 0.0, 0.0])
    expect = 4 * np.pi * k**2 * a**3 * (er - 1) / (er + 2) * np.cross(np.cross(xh, p), xh)
    assert np.linalg.norm(F - expect) < 1e-3 * np.linalg.norm(expect)


def test_dielectric_mie_special_cases():
    """A sphere of the outside medium scatters nothing; a very dense one tends to the PEC
    sphere, with a gap of order 1/m = 1/sqrt(eps_r) (the skin term of the tangential field)."""
    _, a, b = mie.coefficients_dielectric(2.0, 1.0, 1.0)
    assert np.max(np.abs(a)) < 1e-14 and np.max(np.abs(b)) < 1e-14
    xh = S.hplane_directions(19)
    Fp = mie.farfield(2.0, 1.0, xh)
    gap = [np.linalg.norm(mie.farfield(2.0, 1.0, xh, eps_r=e) - Fp) / np.linalg.norm(Fp) for e in (1e4, 1e6)]
    assert gap[1] < 1e-2 and 5.0 < gap[0] / gap[1] < 20.0, gap


# ---------------------------------------------------------------- PMCHWT Galerkin solution
def _rel_err(lvl, k0, er, mr, xh, Fm, ref=None):
    m = O.from_synth(S.icosphere(lvl))
    _, _, _, F = O.dielectric_farfield(m, k0, er, mr, [0, 0, 1], [1, 0, 0], xh)
    return np.linalg.norm(F - Fm) / np.linalg.norm(Fm if ref is None else ref)


def test_pmchwt_converges_to_mie_at_second_order(oracle_mod):
    """Far field of the PMCHWT Galerkin solution vs the dielectric Mie series: O(h^2)
    (Section V-A, the paper's unit-sphere check; eps_r = 2.1, mu_r = 1 as in Table I)."""
    xh = S.hplane_directions(37)
    k0, er = 2.0, 2.1
    Fm = mie.farfield(k0, 1.0, xh, eps_r=er)
    errs = [_rel_err(lvl, k0, er, 1.0, xh, Fm) for lvl in (1, 2, 3)]
    assert errs[-1] < 0.015, errs
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


def test_pmchwt_magnetic_contrast_converges_to_mie(oracle_mod):
    """mu_r != 1: eta = sqrt(mu_r/eps_r) scales the interior EFIO blocks of A^_1; a
    misplaced eta (or 1/eta) leaves an O(1) gap that does not fall with h."""
    xh = S.hplane_directions(37)
    k0, er, mr = 1.5, 2.0, 1.5
    Fm = mie.farfield(k0, 1.0, xh, eps_r=er, mu_r=mr)
    errs = [_rel_err(lvl, k0, er, mr, xh, Fm) for lvl in (1, 2)]
    assert errs[-1] < 0.05, errs
    assert errs[0] / errs[1] > 3.5, errs


def test_pmchwt_transparent_scatterer(oracle_mod):
    """eps_r = mu_r = 1: the interior is the outside medium, the exact exterior Cauchy data
    are the incident field's, and the scattered far field vanishes as h -> 0."""
    xh = S.hplane_directions(37)
    k0 = 2.0
    ref = mie.farfield(k0, 1.0, xh, eps_r=2.1)   # scale of a genuine dielectric's far field
    zero = np.zeros_like(ref)
    errs = [_rel_err(lvl, k0, 1.0, 1.0, xh, zero, ref) for lvl in (1, 2)]
    assert errs[-1] < 1e-3, errs
    assert errs[0] / errs[1] > 4.0, errs


def test_pmchwt_block_structure(oracle_mod):
    """The 2N x 2N matrix is [[K0 + K1, T0 + eta T1], [-T0 - T1/eta, K0 + K1]] with the
    oracle's own EFIO and MFIO matrices (the assembly's bookkeeping, not its quadrature)."""
    m = O.from_synth(S.icosphere(1))
    k0, er, mr = 2.0, 2.1, 1.3
    k1, eta = O.dielectric_wavenumbers(k0, er, mr)
    assert abs(k1 - k0 * math.sqrt(er * mr)) < 1e-15 and abs(eta - math.sqrt(mr / er)) < 1e-15
    Z = O.assemble_pmchwt(m, k0, er, mr)
    T0, T1 = O.assemble_z(m, k0), O.assemble_z(m, k1)
    K0, K1 = O.assemble_mfio(m, k0), O.assemble_mfio(m, k1)
    N = m.n_edges
    s = np.abs(Z).max()
    assert np.abs(Z[:N, :N] - (K0 + K1)).max() < 1e-14 * s
    assert np.abs(Z[N:, N:] - (K0 + K1)).max() < 1e-14 * s
    assert np.abs(Z[:N, N:] - (T0 + eta * T1)).max() < 1e-14 * s
    assert np.abs(Z[N:, :N] - (-T0 - T1 / eta)).max() < 1e-14 * s


# ---------------------------------------------------------------- MFIO quadrature
def _curl_fd_block(m: O.RWGMesh, k: float, t1: int, t2: int, h: float = 1e-5):
    """-int f_i(x) . curl_x A_j(x) with A_j(x) = int G(x, y) f_j(y) dy by the 6-point rule in y,
    the curl by central differences in x (numpy only)."""
    qb, qw = O.triangle_rule6()
    V = m.verts
    def tri_pts(t):
        P = V[m.tris[t]]
        return qb @ P, qw * m.tri_area[t], P

    def rwg(t, i, x):
        s = m.tri_sign[t, i]
        L = m.edge_len[m.tri_edge[t, i]]
        return s * L / (2 * m.tri_area[t]) * (x - V[m.tris[t, i]])

    ys, wy, _ = tri_pts(t2)

    def pot(x, j):
        r = np.linalg.norm(x[None, :] - ys, axis=1)
        G = np.exp(1j * k * r) / (4 * np.pi * r)
        return np.sum((wy * G)[:, None] * rwg(t2, j, ys), axis=0)

    xs, wx, _ = tri_pts(t1)
    out = np.zeros((3, 3), dtype=np.complex128)
    E = np.eye(3) * h
    for x, w in zip(xs, wx):
        for j in range(3):
            dA = [(pot(x + E[c], j) - pot(x - E[c], j)) / (2 * h) for c in range(3)]  # dA[c] = d A / d x_c
            curl = np.array([dA[1][2] - dA[2][1], dA[2][0] - dA[0][2], dA[0][1] - dA[1][0]])
            for i in range(3):
                out[i, j] += -w * np.dot(rwg(t1, i, x), curl)
    return out


def test_mfio_point_formula_against_curl_by_differences(oracle_mod):
    """The MFIO kernel (x - y).(f_n(y) x f_m(x)) G'(r)/r equals -f_m . curl of the EFIO's
    vector potential: checked on vertex-disjoint pairs near and far, at two wavenumbers."""
    m = O.from_synth(S.icosphere(1))
    tris = m.tris
    t1 = 0
    far = [t for t in range(m.nt) if not set(tris[t]) & set(tris[t1])]
    c = m.verts[tris].mean(axis=1)
    d = np.linalg.norm(c - c[t1], axis=1)
    near = min(far, key=lambda t: d[t])
    opposite = max(far, key=lambda t: d[t])
    for k in (1.0, 4.0):
        for t2 in (near, opposite):
            K = O.mfio_block(m, k, t1, t2)
            ref = _curl_fd_block(m, k, t1, t2)
            assert np.abs(K - ref).max() < 1e-7 * np.abs(ref).max(), (k, t2, np.abs(K - ref).max())


def test_mfio_symmetric(oracle_mod):
    """<K f_n, f_m>_x = <K f_m, f_n>_x: exchanging the two integration variables maps the
    kernel onto itself.  Checked on the sphere and on a ragged torus."""
    for sm in (S.icosphere(1), S.torus(7, 3)):
        m = O.from_synth(sm)
        K = O.assemble_mfio(m, 2.5)
        assert np.abs(K - K.T).max() < 1e-13 * np.abs(K).max()


def test_mfio_identical_pairs_vanish(oracle_mod):
    """On one flat triangle x - y lies in the plane and f_n x f_m is normal to it: the
    Sauter-Schwab sum over an identical pair is zero to rounding."""
    m = O.from_synth(S.icosphere(1))
    k = 3.0
    ref = np.abs(O.mfio_block(m, k, 0, 1)).max() + np.abs(O.mfio_block(m, k, 0, 5)).max()
    for t in (0, 7, 33):
        assert np.abs(O.mfio_block(m, k, t, t)).max() < 1e-14 * ref


def test_dielectric_monte_carlo_is_first_order_in_t(oracle_mod):
    """The dielectric Monte Carlo (Section V-C) on fixed draws: its scaled deviations
    D_s = (F_s - F0)/t tend to the linearised response G xi_s (G by central differences of
    the PMCHWT far field along each draw, step 1e-4) at first order in t, so halving t
    halves the gap; the sample covariance is Hermitian and positive semi-definite."""
    sm = S.icosphere(1)
    m = O.from_synth(sm)
    k0, er, mr = 2.0, 2.1, 1.0
    xh = S.hplane_directions(7)
    d, p = [0, 0, 1], [1, 0, 0]
    z = S.gaussian_field_samples(3, m.nv, seed=11)
    sig, ell = 0.05, 0.5
    K = O.cov_kernel(m.verts, m.verts, "gauss", sig, ell) + 1e-12 * sig**2 * np.eye(m.nv)
    xi = z @ np.linalg.cholesky(K).T

    def far(v):
        return O.dielectric_farfield(O.RWGMesh(v, m.tris, m.vnormals), k0, er, mr, d, p, xh)[3].reshape(-1)

    h = 1e-4
    lin = np.stack([(far(m.verts + h * x[:, None] * m.vnormals) - far(m.verts - h * x[:, None] * m.vnormals)) / (2 * h)
                    for x in xi])
    gaps = []
    for t in (0.02, 0.01):
        F0, Fs, cov, pcov = O.monte_carlo_dielectric(m, k0, er, mr, d, p, xh, "gauss", sig, ell, t, z)
        D = (Fs - F0[None]) / t
        gaps.append(np.linalg.norm(D - lin) / np.linalg.norm(lin))
        assert np.abs(cov - cov.conj().T).max() < 1e-12 * np.abs(cov).max()
        assert np.linalg.eigvalsh(0.5 * (cov + cov.conj().T)).min() > -1e-10 * np.abs(cov).max()
        assert np.abs(pcov - pcov.T).max() < 1e-12 * np.abs(pcov).max()
    assert gaps[0] < 0.05, gaps
    assert 1.6 < gaps[0] / gaps[1] < 2.4, gaps


def test_dielectric_ct_second_moment_converges_like_the_full_tensor(oracle_mod):
    """Section V-A: the dielectric unit sphere (k0 = 3, eps_r = 2.1, d = x, p = z) with the
    rank-one tensor right-hand side f (x) f, whose exact second moment is xi (x) xi: the CT
    second moment of the far field's z component converges to the Mie series' F_z (x) conj F_z
    at the full tensor's rate (within a factor 2 of its error), and L0 = L is the full tensor."""
    k0, er = 3.0, 2.1
    xh = S.zplane_directions(91)
    R = np.array([[0, 0, 1.0], [0, -1.0, 0], [1.0, 0, 0]])
    Fz = (mie.farfield(k0, 1.0, xh @ R, eps_r=er) @ R.T)[:, 2]
    Mex = np.outer(Fz, Fz.conj())
    meshes = {l: O.from_synth(S.icosphere(l + 1)) for l in range(3)}
    M, F = O.dielectric_ct_second_moment(meshes, k0, er, 1.0, [[1.0, 0, 0]], [[0, 0, 1.0]], xh, 0, 2)
    zz = np.arange(2, 3 * len(xh), 3)
    ct = lambda L0, L: O.ct_second_moment_rank1(F, L0, L)[np.ix_(zz, zz)] if (L0, L) != (0, 2) else M[np.ix_(zz, zz)]
    err = lambda A: np.linalg.norm(A - Mex) / np.linalg.norm(Mex)
    full = {L: np.outer(F[L], F[L].conj())[np.ix_(zz, zz)] for L in range(3)}
    assert np.abs(ct(2, 2) - full[2]).max() == 0.0
    e_ct = [err(ct(0, L)) for L in (1, 2)]
    assert e_ct[0] / e_ct[1] > 2.5, e_ct
    assert e_ct[1] < 2.0 * err(full[2]), (e_ct, err(full[2]))
    assert np.abs(M - M.conj().T).max() < 1e-14 * np.abs(M).max()


def test_pmchwt_discrete_reciprocity(oracle_mod):
    """Reciprocity of the scattering amplitude, p2 . F(-d2; d1, p1) = p1 . F(-d1; d2, p2), holds
    for the discrete PMCHWT solution to rounding (on an ellipsoid, two oblique waves,
    mu_r != 1).  It fixes the conventions of the incident data (the d x p block) and of the
    far field of (j, m), which the Mie pins see only through a symmetric sphere."""
    m = O.from_synth(S.ellipsoid(1, (0.6, 1.3, 0.9)))
    k0, er, mr = 2.0, 2.1, 1.3
    d1 = np.array([0.3, 0.4, math.sqrt(0.75)])
    d1 /= np.linalg.norm(d1)
    d2 = np.array([-0.5, 0.7, 0.2])
    d2 /= np.linalg.norm(d2)
    p1 = np.cross(d1, [0, 0, 1.0])
    p1 /= np.linalg.norm(p1)
    p2 = np.cross(d2, [1.0, 0, 0])
    p2 /= np.linalg.norm(p2)
    Z = O.assemble_pmchwt(m, k0, er, mr)
    b = O.rhs_pmchwt(m, k0, np.stack([d1, d2]), np.stack([p1, p2]).astype(complex))
    x = O.solve(Z, b)
    A = O.farfield_matrix_pmchwt(m, k0, np.stack([-d2, -d1]))
    a, c = p2 @ (A[0:3] @ x[:, 0]), p1 @ (A[3:6] @ x[:, 1])
    assert abs(a - c) < 1e-12 * abs(a), (a, c)


def test_pmchwt_entry_sampler_matches_the_assembled_matrix(oracle_mod):
    """The entry-by-entry sampler that the full-size GPU test compares against gives the
    assembled matrix's entries in all four blocks, touching and regular pairs alike."""
    m = O.from_synth(S.torus(7, 3))
    k0, er, mr = 2.0, 2.1, 1.3
    Z = O.assemble_pmchwt(m, k0, er, mr)
    n2 = 2 * m.n_edges
    rng = np.random.default_rng(5)
    r, c = rng.integers(0, n2, 200), rng.integers(0, n2, 200)
    r = np.concatenate([r, np.arange(n2)])      # the diagonals: identical-pair entries
    c = np.concatenate([c, np.arange(n2)])
    e = O.pmchwt_entries(m, k0, er, mr, r, c)
    assert np.abs(e - Z[r, c]).max() < 1e-14 * np.abs(Z).max()
