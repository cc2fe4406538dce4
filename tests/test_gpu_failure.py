"""Failure detection on the GPU without a fault: the bounded device waits are made to run
out by a tiny poll limit (fosb_debug_set_wait_limit), and the refinement is made to stall
by allowing it no step.  Each case checks the status the host reads, then that the
context still works (a normal factorisation and solve after the limit is restored)."""
import ctypes

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


def _system(F, lvl=3, k=2.0):
    sm = S.icosphere(lvl)
    m = F.mesh_create(sm.verts, sm.tris, sm.vnormals)
    N = m.n_edges
    Z = torch.zeros((N, N), dtype=torch.complex128, device=DEV)
    b = torch.zeros((N, 1), dtype=torch.complex128, device=DEV)
    F.assemble_efie(m, k, Z, inc=F.incidence((0, 0, 1), (1, 0, 0)), b=b)
    return sm, m, Z, b


def _healthy(F, Z, b, prec):
    lu = F.factor(Z, prec=prec)
    x = torch.zeros_like(b)
    _, _, berr = F.solve(lu, b, x)
    r = (b - Z @ x).abs().max().item() / (Z.abs().sum(1).max().item() * x.abs().max().item())
    assert r < 1e-13, r


def test_panel_grid_barrier_time_out_is_reported(F):
    """FP64 factorisation (cooperative panel, one grid barrier per column) and the
    no-allocation LU, with waits that give up after one poll: FOSB_ERR_TIMEOUT."""
    _, _, Z, b = _system(F, lvl=3)
    try:
        F.debug_set_wait_limit(1)
        with pytest.raises(F.FosbError) as e:
            F.factor(Z, prec=F.FP64)
        assert e.value.status == F.FOSB_ERR_TIMEOUT
        A = Z.clone()
        piv = torch.zeros(A.shape[0], dtype=torch.int32, device=DEV)
        st = F.lib().fosb_getrf_static(ctypes.c_void_p(A.data_ptr()), ctypes.c_int64(A.shape[0]),
                                       ctypes.c_int64(A.shape[0]), ctypes.c_int(F.FP64),
                                       ctypes.c_void_p(piv.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == F.FOSB_ERR_TIMEOUT
    finally:
        F.debug_set_wait_limit(0)
    _healthy(F, Z, b, F.FP64)


def test_sweep_flag_time_out_is_reported(F):
    """MIXED solve: the streaming triangular sweeps wait on per-block flags; with a
    one-poll limit the solve reports FOSB_ERR_TIMEOUT."""
    _, _, Z, b = _system(F, lvl=3)
    lu = F.factor(Z, prec=F.MIXED)
    x = torch.zeros_like(b)
    try:
        F.debug_set_wait_limit(1)
        with pytest.raises(F.FosbError) as e:
            F.solve(lu, b, x)
        assert e.value.status == F.FOSB_ERR_TIMEOUT
    finally:
        F.debug_set_wait_limit(0)
    del lu
    _healthy(F, Z, b, F.MIXED)


def test_stalled_refinement_reports_not_converged_with_best_iterate(F):
    """No refinement step allowed: the complex64 first iterate is written and the call
    returns FOSB_ERR_NOT_CONVERGED."""
    sm, _, Z, b = _system(F, lvl=2)
    lu = F.factor(Z, prec=F.MIXED)
    x = torch.zeros_like(b)
    with pytest.raises(F.FosbError) as e:
        F.solve(lu, b, x, max_iters=0)
    assert e.value.status == F.FOSB_ERR_NOT_CONVERGED
    om = O.from_synth(sm)
    xo = O.solve(O.assemble_z(om, 2.0), O.rhs_planewave(om, 2.0, [0, 0, 1], [1, 0, 0]))
    rel = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert 1e-12 < rel < 1e-4, rel  # complex64 accuracy: written, not refined
    _, iters, berr = F.solve(lu, b, x)  # the same handle then refines normally
    assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) < 1e-8
