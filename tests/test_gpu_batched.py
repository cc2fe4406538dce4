"""Batched scatterers: the persistent batched assembly against the per-mesh assembly, and
the batched factor + refined solve of the 64-ellipsoid table (semi-axes U[0.5, 1.5], k
U[1, 6], N in {480, 1920, 7680}, 16 Fibonacci incident directions each) against the FP64
oracle at 1e-8 -- every scatterer, every direction."""
import ctypes
import math

import numpy as np
import pytest

import fosb_synth as S
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
C128 = torch.complex128


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


def _small_batch():
    """Uneven sizes and shapes: ellipsoids of levels 1-3, a torus, an icosphere."""
    rng = np.random.default_rng(3)
    meshes = [S.ellipsoid(lvl, tuple(rng.uniform(0.5, 1.5, 3))) for lvl in (1, 3, 2, 1, 2)]
    meshes += [S.torus(14, 6), S.icosphere(2)]
    ks = list(rng.uniform(1.0, 6.0, len(meshes)))
    return meshes, ks


@pytest.mark.parametrize("arith", ["ASM_FF", "ASM_FP64"])
def test_batched_assembly_matches_per_mesh(F, arith):
    meshes, ks = _small_batch()
    a = getattr(F, arith)
    hs = [F.mesh_create(m.verts, m.tris, m.vnormals) for m in meshes]
    d = S.fibonacci_directions(5)
    p = np.asarray(S.polarisation_for(d)).reshape(-1, 3)
    incs = [F.incidence(d[: 1 + i % 5], p[: 1 + i % 5]) for i in range(len(hs))]
    incs[3] = None  # an item without right-hand sides
    Zs = [torch.full((h.n_edges, h.n_edges + 3), 7.0, dtype=C128, device=DEV)[:, : h.n_edges] for h in hs]  # ld > N
    Bs = [None if inc is None else torch.full((h.n_edges, inc.shape[0]), 7.0, dtype=C128, device=DEV)
          for h, inc in zip(hs, incs)]
    tun = F.assemble_efie_batched(hs, ks, Zs, incs, Bs, arith=a, tune=True)
    if a == F.ASM_FF:
        assert tun.warps in (4, 8) and tun.tuned_ms > 0.0
    tun2 = F.assemble_efie_batched(hs, ks, Zs, incs, Bs, arith=a, tune=True)  # cached: same shape, no re-tuning
    assert (tun2.warps, tun2.ctas_per_sm) == (tun.warps, tun.ctas_per_sm)
    for h, k, Z, inc, B in zip(hs, ks, Zs, incs, Bs):
        Zr = torch.zeros((h.n_edges, h.n_edges), dtype=C128, device=DEV)
        Br = None if inc is None else torch.zeros((h.n_edges, inc.shape[0]), dtype=C128, device=DEV)
        F.assemble_efie(h, k, Zr, inc=inc, b=Br, arith=a, prec=F.MIXED)
        zr = Zr.cpu().numpy()
        # the same quadrature; only the order of the atomic additions differs
        assert np.abs(Z.cpu().numpy() - zr).max() <= 1e-13 * np.abs(zr).max()
        if B is not None:
            br = Br.cpu().numpy()
            assert np.abs(B.cpu().numpy() - br).max() <= 1e-13 * np.abs(br).max()


def test_batched_64_ellipsoids_match_oracle(F):
    from paper_2308_01457_gb300.batched import BatchedProblem

    table = S.batched_ellipsoid_table()
    assert len(table) == 64
    meshes = [S.ellipsoid(lvl, tuple(ax)) for ax, _, lvl in table]
    ks = [k for _, k, _ in table]
    d = S.fibonacci_directions(16)
    p = np.asarray(S.polarisation_for(d)).reshape(-1, 3)
    prob = BatchedProblem(meshes, ks, d, p).setup()
    prob.run(tune=True)
    torch.cuda.synchronize()
    sizes = sorted({h.n_edges for h in prob.handles})
    assert sizes == [480, 1920, 7680]
    assert all(st == 0 for st in prob.status)
    for i, (sm, k) in enumerate(zip(meshes, ks)):
        N = prob.handles[i].n_edges
        assert prob.berr[i] <= max(64.0, 8.0 * math.sqrt(N)) * 2.0**-52, (i, prob.berr[i])
        om = O.from_synth(sm)
        Xo = O.solve(O.assemble_z(om, k), O.rhs_planewave(om, k, d, p))
        Xg = prob.X[i].cpu().numpy()
        for c in range(16):
            assert _rel(Xg[:, c], Xo[:, c]) < 1e-8, (i, c)


def test_batched_solve_reports_item_errors(F):
    """A singular item among good ones: the call reports FOSB_ERR_SINGULAR for it and solves
    the others."""
    meshes, ks = _small_batch()
    hs = [F.mesh_create(m.verts, m.tris, m.vnormals) for m in meshes[:3]]
    inc = F.incidence([0, 0, 1], [1, 0, 0])
    Zs, Bs = [], []
    for h, k in zip(hs, ks):
        Z = torch.zeros((h.n_edges, h.n_edges), dtype=C128, device=DEV)
        B = torch.zeros((h.n_edges, 1), dtype=C128, device=DEV)
        F.assemble_efie(h, k, Z, inc=inc, b=B, arith=F.ASM_FF, prec=F.MIXED)
        Zs.append(Z)
        Bs.append(B)
    Zs[1] = torch.zeros_like(Zs[1])  # exactly singular
    Xs = [torch.zeros_like(b) for b in Bs]
    n = len(Zs)
    st = (ctypes.c_int * n)()
    status = F.lib().fosb_solve_batched(ctypes.c_int64(n), F._ptr_array(Zs), F._i64_array([z.shape[0] for z in Zs]),
                                        F._i64_array([z.shape[0] for z in Zs]), F._ptr_array(Bs),
                                        F._i64_array([1] * n), F._i64_array([1] * n), F._ptr_array(Xs),
                                        F._i64_array([1] * n), ctypes.c_int(F.MIXED), None, ctypes.c_int(2), None, st,
                                        None)
    assert status == F.FOSB_ERR_SINGULAR and list(st) == [0, F.FOSB_ERR_SINGULAR, 0]
    for i in (0, 2):
        x = Xs[i]
        r = (Bs[i] - Zs[i] @ x).abs().max().item() / (Zs[i].abs().sum(1).max().item() * x.abs().max().item())
        assert r < 1e-13
