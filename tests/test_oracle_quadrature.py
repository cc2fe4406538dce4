"""Pins of the oracle's quadrature against closed forms and independent integrals.

The triangle rule and Gauss-Legendre rule must integrate polynomials exactly; the
Sauter-Schwab regularised rule must reproduce exact integrals of polynomial kernels
(this pins every map and Jacobian factor) and converge to an independently computed
1/|x-y| integral (analytic potential of a uniform triangle, Wilton et al. 1984, plus
an adaptive outer rule)."""
import ctypes
import math

import numpy as np
import pytest

import oracle as O

IDENT, EDGE, VERTEX = 3, 2, 1


def _ss(P, Q, kind, n, kernel):
    gx, gw = O.gauss_legendre01(n)
    lib = O._load()
    P = np.ascontiguousarray(P, dtype=np.float64)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    return lib.orc_ss_integral(O._p(P), O._p(Q), ctypes.c_int(kind), O._p(gx), O._p(gw), ctypes.c_int(n),
                               ctypes.c_int(kernel))


def _area(T):
    return 0.5 * np.linalg.norm(np.cross(T[1] - T[0], T[2] - T[0]))


# non-coplanar touching configurations (shared vertex/edge listed first)
T_ID = np.array([[0.1, -0.2, 0.0], [1.1, 0.05, 0.1], [0.35, 0.9, -0.2]])
E_P = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.4, 0.8, 0.1]])
E_Q = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.6, -0.7, 0.35]])
V_P = np.array([[0.0, 0.0, 0.0], [1.0, 0.2, 0.1], [0.3, 0.9, 0.0]])
V_Q = np.array([[0.0, 0.0, 0.0], [-0.8, 0.3, 0.4], [-0.4, -0.9, 0.2]])
CASES = [(T_ID, T_ID, IDENT), (E_P, E_Q, EDGE), (V_P, V_Q, VERTEX)]


def test_triangle_rule_exact_to_degree_4():
    """int_T lambda1^a lambda2^b lambda3^c dA / |T| = 2 a! b! c! / (a+b+c+2)!  (a+b+c <= 4)."""
    bary, w = O.triangle_rule6()
    assert abs(w.sum() - 1.0) < 1e-15
    for a in range(5):
        for b in range(5 - a):
            for c in range(5 - a - b):
                approx = np.sum(w * bary[:, 0] ** a * bary[:, 1] ** b * bary[:, 2] ** c)
                exact = 2.0 * math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 2)
                assert abs(approx - exact) < 1e-15, (a, b, c)
    # and it is not exact at degree 5 for every monomial (it is a degree-4 rule)
    approx = np.sum(w * bary[:, 0] ** 5)
    assert abs(approx - 2.0 * math.factorial(5) / math.factorial(7)) > 1e-6


def test_gauss_legendre_exact():
    x, w = O.gauss_legendre01(5)
    for p in range(10):
        assert abs(np.sum(w * x**p) - 1.0 / (p + 1)) < 1e-15


@pytest.mark.parametrize("P,Q,kind", CASES)
def test_sauter_schwab_polynomial_kernels_exact(P, Q, kind):
    """Constant kernel gives |T1| |T2|; x.y gives (|T1| c1).(|T2| c2) (centroids c)."""
    for n in (3, 5):
        one = _ss(P, Q, kind, n, 0)
        assert abs(one - _area(P) * _area(Q)) < 1e-14
        xy = _ss(P, Q, kind, n, 2)
        exact = np.dot(_area(P) * P.mean(0), _area(Q) * Q.mean(0))
        assert abs(xy - exact) < 1e-13 * max(1.0, abs(exact))


def _potential(T, x):
    """int_T 1/|x - y| dy for points x (M x 3): the closed form for a uniform flat
    triangle (Wilton, Rao, Glisson et al., IEEE TAP 1984)."""
    n = np.cross(T[1] - T[0], T[2] - T[0])
    n /= np.linalg.norm(n)
    d = (x - T[0]) @ n
    rho = x - d[:, None] * n[None, :]
    total = np.zeros(x.shape[0])
    for i in range(3):
        a, b = T[i], T[(i + 1) % 3]
        lh = (b - a) / np.linalg.norm(b - a)
        uh = np.cross(lh, n)
        lp = (b - rho) @ lh
        lm = (a - rho) @ lh
        P0 = (a - rho) @ uh  # signed distance to the edge line (outward positive)
        Rp = np.sqrt(np.sum((b - rho) ** 2, 1) + d**2)
        Rm = np.sqrt(np.sum((a - rho) ** 2, 1) + d**2)
        R0sq = P0**2 + d**2
        ad = np.abs(d)
        with np.errstate(divide="ignore", invalid="ignore"):
            logt = np.where(np.abs(P0) > 1e-15, P0 * np.log((Rp + lp) / (Rm + lm)), 0.0)
            at = np.arctan2(P0 * lp, R0sq + ad * Rp) - np.arctan2(P0 * lm, R0sq + ad * Rm)
        total += logt - ad * at
    return total


def _adaptive_outer(T, f, tol=1e-12, depth=14):
    """Adaptive integration of f over triangle T (degree-4 rule vs its 4-way split)."""
    bary, w = O.triangle_rule6()

    def rule(tri):  # tri: K x 3 x 3
        pts = np.einsum("qa,kad->kqd", bary, tri)
        vals = f(pts.reshape(-1, 3)).reshape(tri.shape[0], -1)
        area = 0.5 * np.linalg.norm(np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]), axis=1)
        return area * (vals @ w)

    def split(tri):
        a, b, c = tri[:, 0], tri[:, 1], tri[:, 2]
        ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
        return np.stack([np.stack(t, 1) for t in ((a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca))], 1).reshape(-1, 3, 3)

    tris = T[None]
    coarse = rule(tris)
    total = 0.0
    for _ in range(depth):
        kids = split(tris)
        fine = rule(kids).reshape(-1, 4).sum(1)
        done = np.abs(fine - coarse) < tol
        total += fine[done].sum()
        if done.all():
            return total
        tris = kids.reshape(-1, 4, 3, 3)[~done].reshape(-1, 3, 3)
        coarse = rule(tris)
    return total + coarse.sum()


@pytest.mark.parametrize("P,Q,kind", CASES)
def test_sauter_schwab_one_over_r(P, Q, kind):
    """Sauter-Schwab integral of 1/|x-y| converges (n_ss = 4..10) to the value from the
    analytic inner potential and an adaptive outer rule; n_ss = 5 is within 1e-5."""
    ref = _adaptive_outer(P, lambda x: _potential(Q, x))
    vals = [_ss(P, Q, kind, n, 1) for n in (4, 5, 7, 10)]
    errs = [abs(v - ref) / abs(ref) for v in vals]
    assert errs[-1] < 1e-8, errs
    assert errs[1] < 1e-5, errs
    assert errs[-1] < errs[0]


def test_z_complex_symmetric(oracle_mod):
    import fosb_synth as S

    m = O.from_synth(S.icosphere(1))
    Z = O.assemble_z(m, 2.5)
    assert np.abs(Z - Z.T).max() <= 1e-13 * np.abs(Z).max()
    # sampled entries agree with the dense assembly
    rng = np.random.default_rng(0)
    r, c = rng.integers(0, m.n_edges, 40), rng.integers(0, m.n_edges, 40)
    e = O.z_entries(m, 2.5, r, c)
    assert np.abs(e - Z[r, c]).max() <= 1e-14 * np.abs(Z).max()


def test_rwg_divergence_integrates_to_zero(oracle_mod):
    """Each RWG function is divergence-free in total: (l/A+) A+ - (l/A-) A- = 0, and the
    T+/T- signs follow the edge orientation rule."""
    import fosb_synth as S

    m = O.from_synth(S.icosphere(2))
    tot = np.zeros(m.n_edges)
    for t in range(m.nt):
        for i in range(3):
            e = m.tri_edge[t, i]
            tot[e] += m.tri_sign[t, i] * m.edge_len[e]
    assert np.abs(tot).max() < 1e-15
    assert np.all(m.tri_sign[m.edge_tris[:, 0], :].max(1) > 0)
