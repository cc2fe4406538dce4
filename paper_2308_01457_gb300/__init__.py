"""Python binding of the GB300 FOSB/EFIE library (``libfosb.so``, C ABI in include/fosb.h).

Argument marshalling only: every step runs in the CUDA kernels behind the C ABI.
Device buffers are torch CUDA tensors (used for memory and streams); host inputs are
numpy arrays.  If the shared library is missing or cannot be loaded, every call
raises -- there is no CPU fallback.

The call names mirror the C ABI (fosb_mesh_create -> mesh_create, ...).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

FOSB_OK, FOSB_ERR_INVALID_ARG, FOSB_ERR_MESH, FOSB_ERR_SINGULAR, FOSB_ERR_NOT_CONVERGED, FOSB_ERR_OOM, \
    FOSB_ERR_CUDA, FOSB_ERR_TIMEOUT = range(8)
FP64, MIXED, FP32 = 0, 1, 2
REFINE_AUTO, REFINE_IR, REFINE_GMRES = 0, 1, 2
ASM_FP64, ASM_FF, ASM_FP32 = 0, 1, 2
COV_GAUSS, COV_MATERN32 = 0, 1
_STATUS = {0: "OK", 1: "INVALID_ARG", 2: "MESH", 3: "SINGULAR", 4: "NOT_CONVERGED", 5: "OOM", 6: "CUDA", 7: "TIMEOUT"}

_lib = None


class FosbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"FOSB_ERR_{_STATUS.get(status, status)}: {msg}")
        self.status = status


class QuadOpts(ctypes.Structure):
    _fields_ = [("n_ss", ctypes.c_int), ("arith", ctypes.c_int)]


class RefineOpts(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int), ("tol", ctypes.c_double), ("solver", ctypes.c_int)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("backward_error", ctypes.c_double)]


class BatchTuning(ctypes.Structure):
    _fields_ = [("warps", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("tuned_ms", ctypes.c_double)]


class CovKernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("sigma", ctypes.c_double), ("ell", ctypes.c_double)]


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libfosb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libfosb.so not built ({path}); run __graft_entry__.build() or "
                               "python -m paper_2308_01457_gb300.build")
        L = ctypes.CDLL(path)
        L.fosb_last_error.restype = ctypes.c_char_p
        L.fosb_version.restype = ctypes.c_char_p
        L.fosb_kernel_launches.restype = ctypes.c_uint64
        for name in ("fosb_mesh_create", "fosb_mesh_info", "fosb_mesh_edges", "fosb_mesh_destroy",
                     "fosb_assemble_efie", "fosb_factor", "fosb_solve", "fosb_lu_info", "fosb_lu_destroy",
                     "fosb_covariance", "fosb_farfield_moments", "fosb_rcs_monostatic",
                     "fosb_getrf_static", "fosb_profile_enable", "fosb_profile_read", "fosb_rcs_moments",
                     "fosb_debug_set_wait_limit", "fosb_peak_microbench", "fosb_assemble_efie_batched",
                     "fosb_solve_batched", "fosb_field_samples", "fosb_mesh_perturb", "fosb_mc_moments",
                     "fosb_zgemm_fp64class", "fosb_kernel_lowrank", "fosb_covariance_lowrank",
                     "fosb_lowrank_combine", "fosb_assemble_pmchwt", "fosb_farfield_pmchwt"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status: int):
    if status != FOSB_OK:
        raise FosbError(status, lib().fosb_last_error().decode())


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _stream(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ld(t) -> int:
    """Leading dimension (row stride, in elements) of a row-major 2-D tensor."""
    if t.dim() == 1:
        return 1
    if t.stride(1) != 1:
        raise ValueError("tensor rows must be contiguous")
    return t.stride(0)


def _prec_of(t) -> int:
    import torch

    return FP32 if t.dtype == torch.complex64 else FP64


class Mesh:
    """Handle of fosb_mesh_create (RWG tables on the device)."""

    @classmethod
    def _from_handle(cls, h):
        self = cls.__new__(cls)
        self.handle = h
        nv, nt, ne, ntouch = (ctypes.c_int64() for _ in range(4))
        _check(lib().fosb_mesh_info(h, ctypes.byref(nv), ctypes.byref(nt), ctypes.byref(ne), ctypes.byref(ntouch)))
        self.nv, self.nt, self.n_edges, self.n_touching = nv.value, nt.value, ne.value, ntouch.value
        return self

    def __init__(self, verts, tris, vnormals=None):
        v = _np(verts, np.float64)
        t = _np(tris, np.int32)
        vn = None if vnormals is None else _np(vnormals, np.float64)
        h = ctypes.c_void_p()
        _check(lib().fosb_mesh_create(v.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(v.shape[0]),
                                      t.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(t.shape[0]),
                                      None if vn is None else vn.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)))
        self.handle = h
        nv, nt, ne, ntouch = (ctypes.c_int64() for _ in range(4))
        _check(lib().fosb_mesh_info(h, ctypes.byref(nv), ctypes.byref(nt), ctypes.byref(ne), ctypes.byref(ntouch)))
        self.nv, self.nt, self.n_edges, self.n_touching = nv.value, nt.value, ne.value, ntouch.value

    def edges(self):
        e = np.zeros((self.n_edges, 2), np.int32)
        et = np.zeros((self.n_edges, 2), np.int32)
        _check(lib().fosb_mesh_edges(self.handle, e.ctypes.data_as(ctypes.c_void_p), et.ctypes.data_as(ctypes.c_void_p)))
        return e, et

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.fosb_mesh_destroy(self.handle)
            self.handle = None


def mesh_create(verts, tris, vnormals=None) -> Mesh:
    return Mesh(verts, tris, vnormals)


def incidence(d, p) -> np.ndarray:
    """Plane waves p exp(ik d.x) packed as rows d(3), Re p(3), Im p(3)."""
    d = np.atleast_2d(np.asarray(d, np.float64))
    p = np.atleast_2d(np.asarray(p, np.complex128))
    return np.ascontiguousarray(np.concatenate([d, p.real, p.imag], axis=1))


def assemble_efie(mesh: Mesh, k: float, Z, inc=None, b=None, n_ss: int = 5, arith: int = ASM_FP64,
                  prec: int | None = None, stream=None):
    """fosb_assemble_efie: writes Z (N x N) and, if inc is given, b (N x n_inc)."""
    prec = _prec_of(Z) if prec is None else prec
    opts = QuadOpts(n_ss, arith)
    inc_a = None if inc is None else _np(inc, np.float64).reshape(-1, 9)
    n_inc = 0 if inc_a is None else inc_a.shape[0]
    _check(lib().fosb_assemble_efie(mesh.handle, ctypes.c_double(k), ctypes.byref(opts), ctypes.c_int(prec), _ptr(Z),
                                    ctypes.c_int64(_ld(Z)),
                                    None if inc_a is None else inc_a.ctypes.data_as(ctypes.c_void_p),
                                    ctypes.c_int64(n_inc), None if b is None else _ptr(b),
                                    ctypes.c_int64(_ld(b) if b is not None else 0), _stream(stream)))


class LU:
    """Handle of fosb_factor (owns the factors; MIXED keeps a reference to Z)."""

    def __init__(self, handle, n, prec, zref):
        self.handle, self.n, self.prec, self._zref = handle, n, prec, zref

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.fosb_lu_destroy(self.handle)
            self.handle = None


def factor(Z, prec: int | None = None, stream=None) -> LU:
    prec = _prec_of(Z) if prec is None else prec
    h = ctypes.c_void_p()
    _check(lib().fosb_factor(_ptr(Z), ctypes.c_int64(Z.shape[0]), ctypes.c_int64(_ld(Z)), ctypes.c_int(prec),
                             ctypes.byref(h), _stream(stream)))
    return LU(h, Z.shape[0], prec, Z)


def solve(lu: LU, B, X=None, max_iters: int = 10, tol: float = 0.0, solver: int = REFINE_AUTO, stream=None):
    """fosb_solve: X = Z^{-1} B (in place when X is None).  Returns (X, iters, backward_error).
    solver: REFINE_AUTO (refinement, GMRES-IR where it stalls), REFINE_IR, REFINE_GMRES."""
    X = B if X is None else X
    nrhs = 1 if B.dim() == 1 else B.shape[1]
    st = SolveStats()
    ro = RefineOpts(max_iters, tol, solver)
    _check(lib().fosb_solve(lu.handle, ctypes.c_char(b"N"), _ptr(B), ctypes.c_int64(nrhs),
                            ctypes.c_int64(1 if B.dim() == 1 else _ld(B)), _ptr(X), ctypes.c_int64(1 if X.dim() == 1 else _ld(X)),
                            ctypes.byref(ro), ctypes.byref(st), _stream(stream)))
    return X, st.iters, st.backward_error


def covariance(m1: Mesh, lu1: LU, u1, m2: Mesh, lu2: LU, u2, k: float, Sigma, kind: int = COV_GAUSS,
               sigma: float = 1.0, ell: float = 1.0, pseudo: bool = False, max_iters: int = 10,
               tol: float = 0.0, stream=None):
    """fosb_covariance: Sigma (N1 x N2) with Z1 Sigma Z2^H = B1 K12 B2^H (or the pseudo form)."""
    ker = CovKernel(kind, sigma, ell)
    ro = RefineOpts(max_iters, tol)
    _check(lib().fosb_covariance(m1.handle, lu1.handle, _ptr(u1), m2.handle, lu2.handle, _ptr(u2), ctypes.c_double(k),
                                 ctypes.byref(ker), ctypes.c_int(int(pseudo)), _ptr(Sigma), ctypes.c_int64(_ld(Sigma)),
                                 ctypes.byref(ro), _stream(stream)))
    return Sigma


def kernel_lowrank(meshes, kind: int = COV_GAUSS, sigma: float = 1.0, ell: float = 1.0, tol: float = 1e-10,
                   max_rank: int | None = None, device="cuda:0", stream=None):
    """fosb_kernel_lowrank: pivoted Cholesky K ~ R^T R of the covariance kernel over the
    vertices of `meshes` stacked in order.  Returns (R (rank x V float64, device; the
    columns of mesh i are R[:, off_i:off_i + nv_i]), rank, trace error, offsets)."""
    import torch

    meshes = list(meshes)
    V = sum(m.nv for m in meshes)
    max_rank = V if max_rank is None else min(int(max_rank), V)
    R = torch.zeros((max_rank, V), dtype=torch.float64, device=device)
    arr = (ctypes.c_void_p * len(meshes))(*[m.handle.value if isinstance(m.handle, ctypes.c_void_p) else m.handle
                                            for m in meshes])
    rank, err = ctypes.c_int64(), ctypes.c_double()
    _check(lib().fosb_kernel_lowrank(arr, ctypes.c_int64(len(meshes)), ctypes.byref(CovKernel(kind, sigma, ell)),
                                     ctypes.c_double(tol), ctypes.c_int64(max_rank), _ptr(R), ctypes.c_int64(V),
                                     ctypes.byref(rank), ctypes.byref(err), _stream(stream)))
    offs, o = [], 0
    for m in meshes:
        offs.append(o)
        o += m.nv
    return R[:rank.value], rank.value, err.value, offs


def covariance_lowrank(mesh: Mesh, lu: LU, u, k: float, R, dirs, Y=None, max_iters: int = 10, tol: float = 0.0,
                       stream=None):
    """fosb_covariance_lowrank: Y = A Z^{-1} B R^T (3 n_dir x r) for one level; R is the
    level's columns of the kernel factor (r x V_l view of kernel_lowrank's R)."""
    import torch

    d = _np(dirs, np.float64).reshape(-1, 3)
    r = R.shape[0]
    if Y is None:
        dt = torch.complex64 if lu.prec == FP32 else torch.complex128
        Y = torch.empty((3 * d.shape[0], r), dtype=dt, device=R.device)
    ro = RefineOpts(max_iters, tol)
    _check(lib().fosb_covariance_lowrank(mesh.handle, lu.handle, _ptr(u), ctypes.c_double(k), _ptr(R),
                                         ctypes.c_int64(R.stride(0)), ctypes.c_int64(r),
                                         d.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(d.shape[0]),
                                         ctypes.byref(ro), _ptr(Y), ctypes.c_int64(_ld(Y)), _stream(stream)))
    return Y


def lowrank_combine(Y1, Y2, out, weight: float = 1.0, mirror: bool = False, pseudo: bool = False,
                    accumulate: bool = False, prec: int | None = None, stream=None):
    """fosb_lowrank_combine: out (+)= weight (Y1 op(Y2) [+ its op]), op = ^H or ^T (pseudo)."""
    prec = _prec_of(Y1) if prec is None else prec
    _check(lib().fosb_lowrank_combine(ctypes.c_int64(Y1.shape[0]), ctypes.c_int64(Y1.shape[1]), _ptr(Y1),
                                      ctypes.c_int64(_ld(Y1)), _ptr(Y2), ctypes.c_int64(_ld(Y2)),
                                      ctypes.c_double(weight), ctypes.c_int(int(mirror)), ctypes.c_int(int(pseudo)),
                                      ctypes.c_int(prec), _ptr(out), ctypes.c_int64(_ld(out)),
                                      ctypes.c_int(int(accumulate)), _stream(stream)))
    return out


def farfield_moments(m1: Mesh, k: float, dirs, X, out, m2: Mesh | None = None, weight: float = 1.0,
                     mirror: bool = False, pseudo: bool = False, accumulate: bool = False, prec: int | None = None,
                     stream=None):
    """fosb_farfield_moments.  Mean mode (m2 None): out = w A1 X.  Covariance mode:
    out = w A1 X A2^H (+ its ^H if mirror; ^T variants if pseudo)."""
    d = _np(dirs, np.float64).reshape(-1, 3)
    prec = _prec_of(X) if prec is None else prec
    ncols = 1 if X.dim() == 1 else X.shape[1]
    _check(lib().fosb_farfield_moments(m1.handle, None if m2 is None else m2.handle, ctypes.c_double(k),
                                       d.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(d.shape[0]), _ptr(X),
                                       ctypes.c_int64(1 if X.dim() == 1 else _ld(X)), ctypes.c_int64(ncols),
                                       ctypes.c_double(weight), ctypes.c_int(int(mirror)), ctypes.c_int(int(pseudo)),
                                       ctypes.c_int(prec), _ptr(out), ctypes.c_int64(1 if out.dim() == 1 else _ld(out)),
                                       ctypes.c_int(int(accumulate)), _stream(stream)))
    return out


def assemble_pmchwt(mesh: Mesh, k0: float, eps_r: float, mu_r: float, Z, inc=None, b=None, n_ss: int = 5,
                    arith: int = ASM_FP64, stream=None):
    """fosb_assemble_pmchwt: the dielectric scatterer's PMCHWT matrix Z (2N x 2N complex128)
    and, if inc is given, the tested incident Cauchy data b (2N x n_inc); regular pairs in
    FP64 (ASM_FP64) or float-float (ASM_FF)."""
    import torch

    if Z.dtype != torch.complex128 or (b is not None and b.dtype != torch.complex128):
        raise ValueError("assemble_pmchwt: Z and b must be complex128")
    opts = QuadOpts(n_ss, arith)
    inc_a = None if inc is None else _np(inc, np.float64).reshape(-1, 9)
    n_inc = 0 if inc_a is None else inc_a.shape[0]
    _check(lib().fosb_assemble_pmchwt(mesh.handle, ctypes.c_double(k0), ctypes.c_double(eps_r), ctypes.c_double(mu_r),
                                      ctypes.byref(opts), _ptr(Z), ctypes.c_int64(_ld(Z)),
                                      None if inc_a is None else inc_a.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.c_int64(n_inc), None if b is None else _ptr(b),
                                      ctypes.c_int64(_ld(b) if b is not None else 0), _stream(stream)))


def farfield_pmchwt(mesh: Mesh, k0: float, dirs, X, out, weight: float = 1.0, accumulate: bool = False, stream=None):
    """fosb_farfield_pmchwt: out (3 n_dir x ncols) = w A X for exterior Cauchy data X (2N x ncols)."""
    import torch

    if X.dtype != torch.complex128 or out.dtype != torch.complex128:
        raise ValueError("farfield_pmchwt: X and out must be complex128")
    d = _np(dirs, np.float64).reshape(-1, 3)
    ncols = 1 if X.dim() == 1 else X.shape[1]
    _check(lib().fosb_farfield_pmchwt(mesh.handle, ctypes.c_double(k0), d.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.c_int64(d.shape[0]), _ptr(X), ctypes.c_int64(1 if X.dim() == 1 else _ld(X)),
                                      ctypes.c_int64(ncols), ctypes.c_double(weight), _ptr(out),
                                      ctypes.c_int64(1 if out.dim() == 1 else _ld(out)), ctypes.c_int(int(accumulate)),
                                      _stream(stream)))
    return out


def rcs_monostatic(mesh: Mesh, k: float, inc, U, lu: LU | None = None, weights=None, grad=None, n_ss: int = 5,
                   db: bool = False, stream=None):
    """fosb_rcs_monostatic: q_i = sigma_i = |F(-d_i)|^2/(4 pi), or RCS_dB_i with db=True (numpy, n),
    for solved currents U (N x n); with `grad` (device V x 3 float64) also sum_i weights_i dq_i/dX."""
    inc_a = _np(inc, np.float64).reshape(-1, 9)
    n = inc_a.shape[0]
    sig = np.zeros(n)
    w = None if weights is None else _np(weights, np.float64)
    opts = QuadOpts(n_ss, ASM_FP64)
    _check(lib().fosb_rcs_monostatic(mesh.handle, None if lu is None else lu.handle, ctypes.c_double(k),
                                     ctypes.byref(opts), inc_a.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(n),
                                     _ptr(U), ctypes.c_int64(_ld(U)),
                                     None if w is None else w.ctypes.data_as(ctypes.c_void_p), ctypes.c_int(int(db)),
                                     sig.ctypes.data_as(ctypes.c_void_p), None if grad is None else _ptr(grad),
                                     _stream(stream)))
    return sig


def rcs_moments(n_dir: int, F, cov=None, pcov=None, rcs_db=None, var_db=None, var_f=None, incf: int | None = None,
                convention: int = 0, prec: int | None = None, stream=None):
    """fosb_rcs_moments: per direction, RCS_dB of the mean far field F (3 n_dir complex; a
    column of a mean-mode output), the delta-method variance of RCS_dB from the covariance
    and pseudo-covariance blocks, and the variance of each far-field component.  Outputs are
    device float64 tensors (rcs_db, var_db: n_dir; var_f: 3 n_dir); any may be None."""
    prec = _prec_of(F) if prec is None else prec
    if incf is None:
        incf = 1 if F.dim() == 1 else _ld(F)
    _check(lib().fosb_rcs_moments(ctypes.c_int64(n_dir), _ptr(F), ctypes.c_int64(incf),
                                  None if cov is None else _ptr(cov), ctypes.c_int64(0 if cov is None else _ld(cov)),
                                  None if pcov is None else _ptr(pcov), ctypes.c_int64(0 if pcov is None else _ld(pcov)),
                                  ctypes.c_int(prec), ctypes.c_int(convention),
                                  None if rcs_db is None else _ptr(rcs_db), None if var_db is None else _ptr(var_db),
                                  None if var_f is None else _ptr(var_f), _stream(stream)))
    return rcs_db, var_db, var_f


def debug_set_wait_limit(polls: int):
    """fosb_debug_set_wait_limit: poll limit of the bounded panel-barrier and sweep-flag
    waits on the current device (polls <= 0 restores the default)."""
    _check(lib().fosb_debug_set_wait_limit(ctypes.c_int64(polls)))


def peak_microbench(kind: str) -> float:
    """fosb_peak_microbench: measured TFLOP/s of 'fp32' or 'fp64' FMA, or of back-to-back
    tcgen05 'tf32' or 'bf16' MMAs (M = 128, N = 256), on the current device."""
    out = ctypes.c_double()
    _check(lib().fosb_peak_microbench(ctypes.c_int(["fp32", "fp64", "tf32", "bf16"].index(kind)), ctypes.byref(out)))
    return out.value


def _ptr_array(ts):
    return (ctypes.c_void_p * len(ts))(*[None if t is None else t.data_ptr() for t in ts])


def _i64_array(vals):
    return (ctypes.c_int64 * len(vals))(*[int(v) for v in vals])


def assemble_efie_batched(meshes, ks, Zs, incs=None, bs=None, n_ss: int = 5, arith: int = ASM_FF, tune: bool = True,
                          stream=None) -> BatchTuning:
    """fosb_assemble_efie_batched: Z_i (and b_i for incs[i]) for every scatterer, regular pairs
    of all of them in one persistent launch.  Returns the tile shape used."""
    n = len(meshes)
    opts = QuadOpts(n_ss, arith)
    handles = (ctypes.c_void_p * n)(*[m.handle.value for m in meshes])
    kk = (ctypes.c_double * n)(*[float(k) for k in ks])
    inc_np = [None if incs is None or incs[i] is None else _np(incs[i], np.float64).reshape(-1, 9) for i in range(n)]
    inc_ptrs = (ctypes.c_void_p * n)(*[None if a is None else a.ctypes.data for a in inc_np])
    n_inc = _i64_array([0 if a is None else a.shape[0] for a in inc_np])
    b_list = [None] * n if bs is None else list(bs)
    tun = BatchTuning()
    _check(lib().fosb_assemble_efie_batched(ctypes.c_int64(n), handles, kk, ctypes.byref(opts), _ptr_array(Zs),
                                            _i64_array([_ld(z) for z in Zs]), inc_ptrs, n_inc, _ptr_array(b_list),
                                            _i64_array([0 if b is None else _ld(b) for b in b_list]),
                                            ctypes.c_int(int(tune)), ctypes.byref(tun), _stream(stream)))
    return tun


def solve_batched(Zs, Bs, Xs, prec: int = MIXED, workers: int = 4, max_iters: int = 10, tol: float = 0.0,
                  stream=None):
    """fosb_solve_batched: X_i = Z_i^{-1} B_i for every item (worker threads take the items
    largest first).  Returns (iters, backward_error, status) lists."""
    n = len(Zs)
    ro = RefineOpts(max_iters, tol)
    stats = (SolveStats * n)()
    st = (ctypes.c_int * n)()
    status = lib().fosb_solve_batched(ctypes.c_int64(n), _ptr_array(Zs), _i64_array([z.shape[0] for z in Zs]),
                                      _i64_array([_ld(z) for z in Zs]), _ptr_array(Bs),
                                      _i64_array([1 if b.dim() == 1 else b.shape[1] for b in Bs]),
                                      _i64_array([_ld(b) for b in Bs]), _ptr_array(Xs),
                                      _i64_array([_ld(x) for x in Xs]), ctypes.c_int(prec), ctypes.byref(ro),
                                      ctypes.c_int(workers), stats, st, _stream(stream))
    _check(status)
    return [s.iters for s in stats], [s.backward_error for s in stats], list(st)


def field_samples(mesh: Mesh, z, kind: int = COV_GAUSS, sigma: float = 1.0, ell: float = 1.0):
    """fosb_field_samples: xi (nsamp x nv, numpy) = L z with L L^T the vertex covariance."""
    zz = _np(z, np.float64)
    xi = np.zeros_like(zz)
    ker = CovKernel(kind, sigma, ell)
    _check(lib().fosb_field_samples(mesh.handle, ctypes.byref(ker), ctypes.c_int64(zz.shape[0]),
                                    zz.ctypes.data_as(ctypes.c_void_p), xi.ctypes.data_as(ctypes.c_void_p)))
    return xi


def mesh_perturb(base: Mesh, xi, t: float) -> Mesh:
    """fosb_mesh_perturb: the surface x_p + t xi_p n_p of base as a new mesh."""
    x = _np(xi, np.float64)
    h = ctypes.c_void_p()
    _check(lib().fosb_mesh_perturb(base.handle, x.ctypes.data_as(ctypes.c_void_p), ctypes.c_double(t),
                                   ctypes.byref(h)))
    return Mesh._from_handle(h)


def mc_moments(Fs, F0, t: float, mean=None, cov=None, pcov=None, stream=None):
    """fosb_mc_moments: sample mean of the columns of Fs and covariance / pseudo-covariance
    of (F_s - F0)/t, into the given device tensors."""
    _check(lib().fosb_mc_moments(ctypes.c_int64(Fs.shape[0]), ctypes.c_int64(Fs.shape[1]), _ptr(Fs),
                                 ctypes.c_int64(_ld(Fs)), _ptr(F0), ctypes.c_double(t),
                                 None if mean is None else _ptr(mean), None if cov is None else _ptr(cov),
                                 ctypes.c_int64(0 if cov is None else _ld(cov)), None if pcov is None else _ptr(pcov),
                                 ctypes.c_int64(0 if pcov is None else _ld(pcov)), _stream(stream)))
    return mean, cov, pcov


def zgemm_fp64class(A, B, C, method: int = 0, stream=None):
    """fosb_zgemm_fp64class: C = A B (complex128) with FP64-class accuracy, by exact digit
    splitting on the bf16 tensor cores (method 0) or float-float on the FP32 pipe (1)."""
    _check(lib().fosb_zgemm_fp64class(ctypes.c_int64(A.shape[0]), ctypes.c_int64(B.shape[1]), ctypes.c_int64(A.shape[1]),
                                      _ptr(A), ctypes.c_int64(_ld(A)), _ptr(B), ctypes.c_int64(_ld(B)), _ptr(C),
                                      ctypes.c_int64(_ld(C)), ctypes.c_int(method), _stream(stream)))
    return C
