"""Pins of the oracle's shape derivatives (forward-mode differentiation of the discrete
quadrature): the differentiated code reproduces the oracle's Z, and its derivatives of
the monostatic RCS agree with central finite differences of the oracle itself."""
import numpy as np

import fosb_synth as S
import oracle as O


def test_dual_quadrature_value_is_the_oracle_z(oracle_mod):
    sm = S.icosphere(1)
    m = O.from_synth(sm)
    for k in (0.7, 3.0):
        Z = O.assemble_z(m, k)
        assert np.abs(O.grad_value_z(m, k) - Z).max() <= 1e-13 * np.abs(Z).max()


def test_rcs_jacobian_matches_central_differences(oracle_mod):
    sm = S.icosphere(1)
    m = O.from_synth(sm)
    k = 3.0
    d, p, _ = S.monostatic_directions(8)
    d, p = d[::3], p[::3]
    rng = np.random.default_rng(1)
    coords = [(int(v), int(c)) for v, c in zip(rng.integers(0, sm.nv, 5), rng.integers(0, 3, 5))]
    sigma, J = O.rcs_monostatic_jacobian(m, k, d, p, coords)
    h = 1e-5
    for col, (pv, c) in enumerate(coords):
        vals = []
        for delta in (h, -h):
            V = sm.verts.copy()
            V[pv, c] += delta
            vals.append(O.rcs_monostatic_jacobian(O.RWGMesh(V, sm.tris, sm.vnormals), k, d, p, [])[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert np.abs(J[:, col] - fd).max() <= 1e-6 * np.abs(fd).max() + 1e-12, (col, J[:, col], fd)
    assert np.all(sigma > 0)


def test_translation_invariance_of_the_gradient(oracle_mod):
    """Moving every vertex by the same vector changes sigma only through the phase of the
    incident wave, which cancels in the monostatic |F|^2: the x-, y- and z-sums of the
    gradient vanish."""
    sm = S.icosphere(1)
    m = O.from_synth(sm)
    d, p, _ = S.monostatic_directions(2)
    coords = [(v, c) for v in range(sm.nv) for c in range(3)]
    sigma, J = O.rcs_monostatic_jacobian(m, 2.0, d, p, coords)
    G = J.reshape(len(d), sm.nv, 3)
    tot = G.sum(axis=1)
    assert np.abs(tot).max() <= 1e-9 * np.abs(G).max()
