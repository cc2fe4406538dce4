"""Parity at the benchmark's own physics against the FP64 oracle.

* The mixed-precision sphere workload one level below the benchmark's finest: icosphere
  levels 0..3 (N = 120 .. 7680), k = 4, d = +z, p = x, 181 H-plane angles, Gaussian
  covariance sigma = 0.005, l = 0.3, combination technique L0 = 0, L = 3 (Section IV-B,
  eq. CTsubsystem; Section V-A).  The mean far field, the CT far-field covariance and
  pseudo-covariance, and the RCS moments are compared element-wise with the oracle's
  ct_farfield_covariance (LAPACK at N = 7680) at 1e-8 -- the same kernels and launch
  configuration as the benchmark step, whose finest level the oracle cannot solve in
  seconds.
* Two level-4 scatterers (N = 7680) of the 64-entry batched ellipsoid table, 16
  Fibonacci incident directions each: every solution column at 1e-8."""
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


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_sphere_ka4_ct_levels_0_to_3_match_oracle(F):
    from paper_2308_01457_gb300.ct import FOSBProblem

    k, sig, ell = 4.0, 0.005, 0.3
    dirs = S.hplane_directions(181)
    meshes = [S.icosphere(l + 1) for l in range(4)]
    prob = FOSBProblem(meshes, k, (0, 0, 1), (1, 0, 0), dirs, 0, 3, F.COV_GAUSS, sig, ell, prec=F.MIXED,
                       arith=F.ASM_FF, pseudo=True).setup()
    Fm, cov, pcov = (t.cpu().numpy() for t in prob.run())
    rcs_db, var_db = prob.rcs_db.cpu().numpy(), prob.var_db.cpu().numpy()
    assert prob.levels[3].mesh.n_edges == 7680

    lev = {l: O.nominal_level(O.from_synth(sm), k, [0, 0, 1], [1, 0, 0], dirs) for l, sm in enumerate(meshes)}
    Fo = lev[3].A @ lev[3].u
    cov_o = O.ct_farfield_covariance(lev, 0, 3, "gauss", sig, ell)
    pcov_o = O.ct_farfield_covariance(lev, 0, 3, "gauss", sig, ell, pseudo=True)
    assert _rel(Fm[:, 0], Fo) < 1e-8
    assert _rel(cov, cov_o) < 1e-8
    assert _rel(pcov, pcov_o) < 1e-8
    assert np.abs(rcs_db - O.rcs_db(Fo.reshape(-1, 3))).max() < 1e-8 * np.abs(O.rcs_db(Fo.reshape(-1, 3))).max()
    assert _rel(var_db, O.rcs_variance_db(Fo.reshape(-1, 3), cov_o, pcov_o)) < 1e-8
    prob.release()


def test_level_overlap_gives_the_sequential_result(F):
    """The coarse levels on a side stream beside the finest level's assembly (the default)
    give the sequential step's result (only the order of the FP64 atomics may differ)."""
    from paper_2308_01457_gb300.ct import FOSBProblem

    k, sig, ell = 4.0, 0.005, 0.3
    dirs = S.hplane_directions(31)
    meshes = [S.icosphere(l + 1) for l in range(3)]
    outs = []
    for overlap in (True, False):
        prob = FOSBProblem(meshes, k, (0, 0, 1), (1, 0, 0), dirs, 0, 2, F.COV_GAUSS, sig, ell, prec=F.MIXED,
                           arith=F.ASM_FF, pseudo=True, overlap=overlap).setup()
        for _ in range(2):  # the second step reuses the buffers of the first
            res = [t.cpu().numpy() for t in prob.run()]
            prob.release()
        outs.append(res)
    for a, b in zip(*outs):
        assert _rel(a, b) < 1e-12


def test_batched_level4_ellipsoids_match_oracle(F):
    table = S.batched_ellipsoid_table()
    picked = [(i, row) for i, row in enumerate(table) if row[2] == 4][:2]
    d = S.fibonacci_directions(16)
    p = np.asarray(S.polarisation_for(d)).reshape(-1, 3)
    for i, (ax, k, lvl) in picked:
        sm = S.ellipsoid(lvl, tuple(ax))
        m = F.mesh_create(sm.verts, sm.tris, sm.vnormals)
        N = m.n_edges
        assert N == 7680
        inc = F.incidence(d, p)
        Z = torch.zeros((N, N), dtype=torch.complex128, device=DEV)
        B = torch.zeros((N, 16), dtype=torch.complex128, device=DEV)
        F.assemble_efie(m, k, Z, inc=inc, b=B, arith=F.ASM_FF, prec=F.MIXED)
        lu = F.factor(Z, prec=F.MIXED)
        X = torch.zeros_like(B)
        _, iters, berr = F.solve(lu, B, X)
        om = O.from_synth(sm)
        Xo = O.solve(O.assemble_z(om, k), O.rhs_planewave(om, k, d, p))
        Xg = X.cpu().numpy()
        for c in range(16):
            assert _rel(Xg[:, c], Xo[:, c]) < 1e-8, (i, c)
        assert berr <= max(64.0, 8.0 * math.sqrt(N)) * 2.0**-52
