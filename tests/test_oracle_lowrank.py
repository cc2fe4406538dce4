"""Pins of the oracle's pivoted Cholesky factorisation and of the low-rank combination-
technique covariance built on it (the low-rank right-hand side of Section VI), by routes
that do not share their arithmetic:

* with every pivot taken, the factor is LAPACK's Cholesky factor of the pivot-permuted
  matrix (numpy.linalg.cholesky);
* a Gram matrix of rank 5 stops at exactly 5 columns and is reproduced;
* every pivot is the largest diagonal entry of the Schur complement of the earlier pivots,
  and the reported error is that complement's trace, both formed independently with
  numpy.linalg.solve;
* the trace of the remainder equals trace(K) - ||L||_F^2;
* the low-rank CT covariance equals the full one when nothing is dropped, and otherwise
  differs from it by at most err * sum over blocks of ||G_l1||_2 ||G_l2||_F with
  G_l = A_l Z_l^{-1} B_l (the dropped part K - R R^T is positive semi-definite with trace
  err, so its spectral norm is at most err)."""
import numpy as np
import pytest

import fosb_synth as S
import oracle as O


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    return A @ A.T + n * np.eye(n)


def test_full_pivoting_is_lapack_cholesky_of_the_permuted_matrix():
    K = _spd(30, 1)
    L, piv, err = O.pivoted_cholesky(K)
    assert L.shape == (30, 30) and sorted(piv.tolist()) == list(range(30))
    Lp = L[piv]  # rows in pivot order: lower triangular
    assert np.abs(np.triu(Lp, 1)).max() == 0.0
    ref = np.linalg.cholesky(K[np.ix_(piv, piv)])
    assert np.abs(Lp - ref).max() < 1e-12 * np.abs(ref).max()
    assert abs(err) < 1e-10 * np.trace(K)


def test_exact_low_rank_stops_at_its_rank():
    rng = np.random.default_rng(2)
    G = rng.standard_normal((40, 5))
    K = G @ G.T
    L, piv, err = O.pivoted_cholesky(K, tol=1e-13)
    assert L.shape[1] == 5
    assert np.abs(L @ L.T - K).max() < 1e-12 * np.abs(K).max()
    assert err <= 1e-13 * np.trace(K)


def test_pivots_are_schur_complement_argmax_and_error_is_its_trace():
    X = S.icosphere(1).verts
    rng = np.random.default_rng(5)
    X = X + 0.01 * rng.standard_normal(X.shape)  # break the sphere's symmetric ties
    K = O.cov_kernel(X, X, "matern32", 1.3, 0.7)
    for m in (1, 4, 9, 17):
        L, piv, err = O.pivoted_cholesky(K, max_rank=m)
        assert len(piv) == m
        P = piv[:m - 1]
        if m > 1:
            Sc = K - K[:, P] @ np.linalg.solve(K[np.ix_(P, P)], K[P, :])
        else:
            Sc = K.copy()
        dS = np.diag(Sc).copy()
        dS[P] = -np.inf
        assert int(np.argmax(dS)) == piv[m - 1]
        Sm = K - K[:, piv] @ np.linalg.solve(K[np.ix_(piv, piv)], K[piv, :])
        rest = np.setdiff1d(np.arange(K.shape[0]), piv)
        assert abs(err - np.trace(Sm[np.ix_(rest, rest)])) < 1e-10 * np.trace(K)
        assert abs(err - (np.trace(K) - (L * L).sum())) < 1e-10 * np.trace(K)


def test_tolerance_is_met_and_rank_grows_as_it_shrinks():
    X = S.icosphere(2).verts
    K = O.cov_kernel(X, X, "gauss", 0.2, 0.5)
    ranks = []
    for tol in (1e-2, 1e-4, 1e-6, 1e-8):
        L, _, err = O.pivoted_cholesky(K, tol=tol)
        assert err <= tol * np.trace(K)
        E = K - L @ L.T
        assert np.abs(E).max() <= err * (1 + 1e-8) + 1e-15  # |E_ij| <= max diag(E) <= trace(E)
        ranks.append(L.shape[1])
    assert ranks == sorted(ranks) and ranks[0] < ranks[-1] <= K.shape[0]


@pytest.fixture(scope="module")
def levels(oracle_mod):
    xh = S.hplane_directions(7)
    return {l: O.nominal_level(O.from_synth(S.icosphere(l + 1)), 1.5, [0, 0, 1], [1, 0, 0], xh) for l in (0, 1, 2)}


def test_lowrank_ct_covariance_without_truncation_is_the_full_one(levels):
    for pseudo in (False, True):
        full = O.ct_farfield_covariance(levels, 0, 2, "gauss", 0.3, 0.6, pseudo=pseudo)
        lr, rank, err = O.ct_farfield_covariance_lowrank(levels, 0, 2, "gauss", 0.3, 0.6, tol=1e-15, pseudo=pseudo)
        assert rank < 42 + 162 + 642
        assert np.abs(lr - full).max() < 1e-9 * np.abs(full).max()


def test_lowrank_ct_covariance_error_bound(levels):
    full = O.ct_farfield_covariance(levels, 0, 2, "gauss", 0.3, 0.6)
    lr, rank, err = O.ct_farfield_covariance_lowrank(levels, 0, 2, "gauss", 0.3, 0.6, tol=1e-3)
    G = {l: lv.A @ np.linalg.solve(lv.Z, lv.B) for l, lv in levels.items()}
    bound = 0.0
    for (l1, l2), _ in O.ct_hermitian_blocks(0, 2):
        b = np.linalg.norm(G[l1], 2) * np.linalg.norm(G[l2], "fro")
        bound += 2 * b if l1 != l2 else b
    diff = np.linalg.norm(lr - full)
    assert 0 < diff <= err * bound, (diff, err * bound)
