"""FP64 CPU oracle of the FOSB hot path (PEC EFIE, RWG, combination technique).

TEST INFRASTRUCTURE ONLY: the slow, plain reference the CUDA library is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg import it; the library never does, and the two share no code.  The
seeded mesh generators of ``fosb_synth`` feed both sides.

Every function states the passage of the paper it follows.  Quadrature loops live in
``efie_oracle.cpp`` (plain C++, one point pair at a time); the dense linear algebra
uses numpy/LAPACK as a library primitive (``numpy.linalg.solve``).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C++ quadrature core with g++ (OpenMP over test triangles)."""
    srcs = [os.path.join(_HERE, "efie_oracle.cpp"), os.path.join(_HERE, "efie_oracle_grad.cpp")]
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or any(os.path.getmtime(_SO) < os.path.getmtime(s) for s in srcs):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared"] + srcs + ["-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.orc_ss_integral.restype = ctypes.c_double
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def n_threads() -> int:
    return len(os.sched_getaffinity(0))


# ---------------------------------------------------------------------------
# Quadrature rules
# ---------------------------------------------------------------------------
def triangle_rule6():
    """Symmetric 6-point degree-4 triangle rule (Dunavant 1985), in closed form.

    Nodes (a, a, 1-2a) and (b, b, 1-2b) with
      a = (8 - sqrt10 + sqrt(38 - 44 sqrt(2/5)))/18,  b = (8 - sqrt10 - sqrt(38 - 44 sqrt(2/5)))/18,
    weights (620 +- sqrt(213125 - 53320 sqrt10))/3720 (normalised to sum 1)."""
    s10 = math.sqrt(10.0)
    r = math.sqrt(38.0 - 44.0 * math.sqrt(0.4))
    a = (8.0 - s10 + r) / 18.0
    b = (8.0 - s10 - r) / 18.0
    q = math.sqrt(213125.0 - 53320.0 * s10)
    wa = (620.0 + q) / 3720.0
    wb = (620.0 - q) / 3720.0
    bary = np.array(
        [[1 - 2 * a, a, a], [a, 1 - 2 * a, a], [a, a, 1 - 2 * a],
         [1 - 2 * b, b, b], [b, 1 - 2 * b, b], [b, b, 1 - 2 * b]], dtype=np.float64)
    w = np.array([wa, wa, wa, wb, wb, wb], dtype=np.float64)
    return bary, w


def gauss_legendre01(n: int):
    """n-point Gauss-Legendre rule on [0, 1] (numpy's leggauss, mapped)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


# ---------------------------------------------------------------------------
# RWG tables (Section IV: lowest-order div-conforming elements on flat triangles)
# ---------------------------------------------------------------------------
@dataclass
class RWGMesh:
    """Edges numbered in lexicographic order of their vertex pair (a < b).  Local edge i
    of a triangle is the one opposite its local vertex i; the triangle is T+ of the edge
    when the edge runs a -> b in the triangle's counter-clockwise order (sign +1), T-
    otherwise (sign -1)."""

    verts: np.ndarray
    tris: np.ndarray
    vnormals: np.ndarray
    edges: np.ndarray = field(init=False)      # N x 2 (a < b)
    edge_len: np.ndarray = field(init=False)   # N
    edge_tris: np.ndarray = field(init=False)  # N x 2 (T+, T-)
    tri_edge: np.ndarray = field(init=False)   # T x 3
    tri_sign: np.ndarray = field(init=False)   # T x 3

    def __post_init__(self):
        self.verts = np.ascontiguousarray(self.verts, dtype=np.float64)
        self.tris = np.ascontiguousarray(self.tris, dtype=np.int32)
        T = self.tris.shape[0]
        keys = {}
        for t in range(T):
            for i in range(3):
                u, v = int(self.tris[t, (i + 1) % 3]), int(self.tris[t, (i + 2) % 3])
                keys.setdefault((min(u, v), max(u, v)), []).append((t, i, +1.0 if u < v else -1.0))
        order = sorted(keys)
        N = len(order)
        self.edges = np.array(order, dtype=np.int32).reshape(N, 2)
        self.edge_len = np.linalg.norm(self.verts[self.edges[:, 1]] - self.verts[self.edges[:, 0]], axis=1)
        self.edge_tris = np.zeros((N, 2), dtype=np.int32)
        self.tri_edge = np.zeros((T, 3), dtype=np.int32)
        self.tri_sign = np.zeros((T, 3), dtype=np.float64)
        for m, key in enumerate(order):
            occ = keys[key]
            if len(occ) != 2 or occ[0][2] == occ[1][2]:
                raise ValueError(f"edge {key} is not shared by two consistently oriented triangles")
            for t, i, s in occ:
                self.tri_edge[t, i] = m
                self.tri_sign[t, i] = s
                self.edge_tris[m, 0 if s > 0 else 1] = t
        a = self.verts[self.tris[:, 0]]
        self.tri_area = 0.5 * np.linalg.norm(np.cross(self.verts[self.tris[:, 1]] - a, self.verts[self.tris[:, 2]] - a), axis=1)

    @property
    def n_edges(self) -> int:
        return int(self.edges.shape[0])

    @property
    def nv(self) -> int:
        return int(self.verts.shape[0])

    @property
    def nt(self) -> int:
        return int(self.tris.shape[0])

    def _args(self):
        return (_p(self.verts), _p(self.tris), ctypes.c_int64(self.nt), _p(self.tri_edge), _p(self.tri_sign),
                _p(self.edge_len))


def from_synth(m) -> RWGMesh:
    return RWGMesh(m.verts, m.tris, m.vnormals)


# ---------------------------------------------------------------------------
# EFIE matrix, right-hand side, far field (Sections II-B, II-C, IV-A)
# ---------------------------------------------------------------------------
def assemble_z(mesh: RWGMesh, k: float, n_ss: int = 5, threads: int | None = None) -> np.ndarray:
    """Dense Galerkin matrix Z (N x N complex128) of the EFIO, Section IV-A (Z_L u_L = b_L)."""
    qb, qw = triangle_rule6()
    gx, gw = gauss_legendre01(n_ss)
    N = mesh.n_edges
    Z = np.zeros((N, N), dtype=np.complex128)
    _load().orc_assemble_z(*mesh._args(), ctypes.c_int64(N), ctypes.c_double(k), _p(qb), _p(qw), ctypes.c_int(6),
                           _p(gx), _p(gw), ctypes.c_int(n_ss), _p(Z), ctypes.c_int(threads or n_threads()))
    return Z


def z_entries(mesh: RWGMesh, k: float, rows, cols, n_ss: int = 5, threads: int | None = None) -> np.ndarray:
    """Selected entries Z[rows[e], cols[e]] computed one by one (for large-N parity samples)."""
    qb, qw = triangle_rule6()
    gx, gw = gauss_legendre01(n_ss)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    out = np.zeros(rows.shape[0], dtype=np.complex128)
    _load().orc_z_entries(*mesh._args(), _p(mesh.edge_tris), ctypes.c_double(k), _p(qb), _p(qw), ctypes.c_int(6),
                          _p(gx), _p(gw), ctypes.c_int(n_ss), _p(rows), _p(cols), ctypes.c_int64(rows.shape[0]),
                          _p(out), ctypes.c_int(threads or n_threads()))
    return out


def incidence(d, p):
    """Pack plane waves E_inc = p exp(ik d.x) (Section V) as rows d(3), Re p(3), Im p(3)."""
    d = np.atleast_2d(np.asarray(d, dtype=np.float64))
    p = np.atleast_2d(np.asarray(p, dtype=np.complex128))
    return np.ascontiguousarray(np.concatenate([d, p.real, p.imag], axis=1))


def rhs_planewave(mesh: RWGMesh, k: float, d, p) -> np.ndarray:
    """b_m = <gamma_D E_inc, f_m>_x = -int E_inc . f_m  (N x n_inc), Sections II-C and IV-A."""
    inc = incidence(d, p)
    qb, qw = triangle_rule6()
    b = np.zeros((mesh.n_edges, inc.shape[0]), dtype=np.complex128)
    _load().orc_rhs(*mesh._args(), ctypes.c_int64(mesh.n_edges), ctypes.c_double(k), _p(qb), _p(qw), ctypes.c_int(6),
                    _p(inc), ctypes.c_int64(inc.shape[0]), _p(b))
    return b


def farfield_matrix(mesh: RWGMesh, k: float, xhat) -> np.ndarray:
    """A (3 n_dir x N): F(xh_d)_c = sum_n A[3d + c, n] u_n, from E_sc = -E_k j and the
    far-field expansion E_sc ~ exp(ik|x|)/(4 pi |x|) F (Section II-C)."""
    xhat = np.ascontiguousarray(np.atleast_2d(xhat), dtype=np.float64)
    qb, qw = triangle_rule6()
    A = np.zeros((3 * xhat.shape[0], mesh.n_edges), dtype=np.complex128)
    _load().orc_farfield_matrix(*mesh._args(), ctypes.c_int64(mesh.n_edges), ctypes.c_double(k), _p(qb), _p(qw),
                                ctypes.c_int(6), _p(xhat), ctypes.c_int64(xhat.shape[0]), _p(A))
    return A


def solve(Z: np.ndarray, b: np.ndarray) -> np.ndarray:
    """u = Z^{-1} b (Section IV-A, eq. linear_system), LAPACK partial-pivot LU."""
    return np.linalg.solve(Z, b)


def rcs_db(F: np.ndarray) -> np.ndarray:
    """RCS in dB of a far-field vector or component: sigma = 4 pi |E_sc|^2 r^2 = |F|^2/(4 pi)
    with E_sc ~ exp(ik r)/(4 pi r) F and |p| = 1 (Section II-C, eq. RCS read with the
    far-field normalisation of the expansion)."""
    F = np.asarray(F)
    mag2 = np.sum(np.abs(F) ** 2, axis=-1) if F.ndim >= 1 and F.shape[-1] == 3 else np.abs(F) ** 2
    return 10.0 * np.log10(mag2 / (4.0 * np.pi))


# ---------------------------------------------------------------------------
# Dielectric scatterer: the PMCHWT system (Section II-C eq. pmchwt)
# ---------------------------------------------------------------------------
def dielectric_wavenumbers(k0: float, eps_r: float, mu_r: float):
    """k1 = k0 sqrt(eps_r mu_r) inside and eta = sqrt(mu_r/eps_r) (Section II-A,
    eq. relativeParameters; k_i = omega sqrt(mu_i eps_i))."""
    return k0 * math.sqrt(eps_r * mu_r), math.sqrt(mu_r / eps_r)


def assemble_mfio(mesh: RWGMesh, k: float, n_ss: int = 5, threads: int | None = None) -> np.ndarray:
    """<K_k f_n, f_m>_x (N x N): the MFIO K_k = {gamma_D H_k} of Section II-B tested with
    the x-pairing, -int int (x - y).(f_n(y) x f_m(x)) exp(ikr)(ikr - 1)/(4 pi r^3)."""
    qb, qw = triangle_rule6()
    gx, gw = gauss_legendre01(n_ss)
    N = mesh.n_edges
    K = np.zeros((N, N), dtype=np.complex128)
    _load().orc_assemble_mfio(*mesh._args(), ctypes.c_int64(N), ctypes.c_double(k), _p(qb), _p(qw), ctypes.c_int(6),
                              _p(gx), _p(gw), ctypes.c_int(n_ss), _p(K), ctypes.c_int(threads or n_threads()))
    return K


def mfio_block(mesh: RWGMesh, k: float, t1: int, t2: int, n_ss: int = 5) -> np.ndarray:
    """3 x 3 MFIO block of the triangle pair (t1 test, t2 trial), local edges in order."""
    qb, qw = triangle_rule6()
    gx, gw = gauss_legendre01(n_ss)
    out = np.zeros((3, 3), dtype=np.complex128)
    _load().orc_mfio_block(*mesh._args(), ctypes.c_double(k), _p(qb), _p(qw), ctypes.c_int(6), _p(gx), _p(gw),
                           ctypes.c_int(n_ss), ctypes.c_int64(t1), ctypes.c_int64(t2), _p(out))
    return out


def assemble_pmchwt(mesh: RWGMesh, k0: float, eps_r: float, mu_r: float, n_ss: int = 5,
                    threads: int | None = None) -> np.ndarray:
    """Galerkin matrix (2N x 2N) of A_0 + A^_1 (Section II-C eq. pmchwt; A_k and the scaled
    A^_k of eq. BOmultitraceA) for the exterior Cauchy data (j, m) = (gamma_D^c E, gamma_N^c E):
      [[K_0 + K_1, T_0 + eta T_1], [-T_0 - T_1/eta, K_0 + K_1]]."""
    k1, eta = dielectric_wavenumbers(k0, eps_r, mu_r)
    qb, qw = triangle_rule6()
    gx, gw = gauss_legendre01(n_ss)
    N = mesh.n_edges
    Z = np.zeros((2 * N, 2 * N), dtype=np.complex128)
    _load().orc_assemble_pmchwt(*mesh._args(), ctypes.c_int64(N), ctypes.c_double(k0), ctypes.c_double(k1),
                                ctypes.c_double(eta), _p(qb), _p(qw), ctypes.c_int(6), _p(gx), _p(gw),
                                ctypes.c_int(n_ss), _p(Z), ctypes.c_int(threads or n_threads()))
    return Z


def pmchwt_entries(mesh: RWGMesh, k0: float, eps_r: float, mu_r: float, rows, cols, n_ss: int = 5,
                   threads: int | None = None) -> np.ndarray:
    """Selected entries of assemble_pmchwt's matrix, computed one by one (large-N samples)."""
    k1, eta = dielectric_wavenumbers(k0, eps_r, mu_r)
    qb, qw = triangle_rule6()
    gx, gw = gauss_legendre01(n_ss)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    out = np.zeros(rows.shape[0], dtype=np.complex128)
    _load().orc_pmchwt_entries(*mesh._args(), _p(mesh.edge_tris), ctypes.c_int64(mesh.n_edges), ctypes.c_double(k0),
                               ctypes.c_double(k1), ctypes.c_double(eta), _p(qb), _p(qw), ctypes.c_int(6), _p(gx),
                               _p(gw), ctypes.c_int(n_ss), _p(rows), _p(cols), ctypes.c_int64(rows.shape[0]), _p(out),
                               ctypes.c_int(threads or n_threads()))
    return out


def rhs_pmchwt(mesh: RWGMesh, k0: float, d, p) -> np.ndarray:
    """Tested incident Cauchy data (2N x n_inc): <gamma_D E_inc, f_m>_x = -int E_inc . f_m on
    top and <gamma_N E_inc, f_m>_x = -int (curl E_inc/(ik0)) . f_m below; for
    E_inc = p exp(ik0 d.x), curl E_inc/(ik0) = (d x p) exp(ik0 d.x) (Section V eq. incidentNumexp)."""
    d = np.atleast_2d(np.asarray(d, dtype=np.float64))
    p = np.atleast_2d(np.asarray(p, dtype=np.complex128))
    return np.vstack([rhs_planewave(mesh, k0, d, p), rhs_planewave(mesh, k0, d, np.cross(d, p))])


def farfield_matrix_pmchwt(mesh: RWGMesh, k0: float, xhat) -> np.ndarray:
    """A (3 n_dir x 2N): F(xh) = -ik0 [xh x sum j_n v_n + (I - xh xh^T) sum m_n v_n],
    v_n = int f_n exp(-ik0 xh.y), from E_sc = -E_k0 m - H_k0 j outside (Section II-C)."""
    xhat = np.ascontiguousarray(np.atleast_2d(xhat), dtype=np.float64)
    qb, qw = triangle_rule6()
    A = np.zeros((3 * xhat.shape[0], 2 * mesh.n_edges), dtype=np.complex128)
    _load().orc_farfield_matrix_pmchwt(*mesh._args(), ctypes.c_int64(mesh.n_edges), ctypes.c_double(k0), _p(qb),
                                       _p(qw), ctypes.c_int(6), _p(xhat), ctypes.c_int64(xhat.shape[0]), _p(A))
    return A


def dielectric_farfield(mesh: RWGMesh, k0: float, eps_r: float, mu_r: float, d, p, xhat, n_ss: int = 5):
    """Assemble, solve (LAPACK) and map the PMCHWT problem: returns (Z, b, x, F (n_dir x 3))."""
    Z = assemble_pmchwt(mesh, k0, eps_r, mu_r, n_ss)
    b = rhs_pmchwt(mesh, k0, d, p)
    x = solve(Z, b)
    F = (farfield_matrix_pmchwt(mesh, k0, xhat) @ x[:, 0]).reshape(-1, 3)
    return Z, b, x, F


# ---------------------------------------------------------------------------
# Shape derivative, covariance, combination technique (Sections III and IV)
# ---------------------------------------------------------------------------
def triangle_normals(mesh: RWGMesh) -> np.ndarray:
    a = mesh.verts[mesh.tris[:, 0]]
    n = np.cross(mesh.verts[mesh.tris[:, 1]] - a, mesh.verts[mesh.tris[:, 2]] - a)
    return n / np.linalg.norm(n, axis=1, keepdims=True)


def sd_rhs(mesh: RWGMesh, k: float, u: np.ndarray, vnormals=None, dense: bool = True):
    """B (N x V): the shape-derivative right-hand side g = B xi of Section III (PEC),
    for the normal perturbation v_n = sum_p xi_p psi_p (n_p . n_T), in weak form
      B_mp = - sum_n u_n int psi_p nu_{p,T} [ik f_m.f_n + 1/(ik) div f_m div f_n]."""
    vn = np.ascontiguousarray(mesh.vnormals if vnormals is None else vnormals, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.complex128).reshape(-1)
    qb, qw = triangle_rule6()
    vals = np.zeros((mesh.nt, 3, 3), dtype=np.complex128)
    _load().orc_sd_rhs(*mesh._args(), ctypes.c_double(k), _p(qb), _p(qw), ctypes.c_int(6), _p(vn), _p(u), _p(vals))
    rows = np.repeat(mesh.tri_edge[:, :, None], 3, axis=2).ravel()
    cols = np.repeat(mesh.tris[:, None, :], 3, axis=1).ravel()
    import scipy.sparse as sp
    B = sp.coo_matrix((vals.ravel(), (rows, cols)), shape=(mesh.n_edges, mesh.nv)).tocsr()
    return B.toarray() if dense else B


def cov_kernel(x1: np.ndarray, x2: np.ndarray, kind: str, sigma: float, ell: float) -> np.ndarray:
    """K_pq = sigma^2 rho(|x_p - x_q|): Gaussian rho = exp(-r^2/(2 l^2)) or Matern-3/2
    rho = (1 + sqrt3 r/l) exp(-sqrt3 r/l), chordal distance: the second moment
    M^2[v_n] of the random normal velocity (Section III) expanded at the mesh vertices."""
    r = np.sqrt(np.maximum(((x1[:, None, :] - x2[None, :, :]) ** 2).sum(-1), 0.0))
    if kind == "gauss":
        return sigma**2 * np.exp(-(r**2) / (2 * ell**2))
    if kind == "matern32":
        s = math.sqrt(3.0) * r / ell
        return sigma**2 * (1.0 + s) * np.exp(-s)
    raise ValueError(kind)


def covariance(Z1, B1, Z2, B2, K12, pseudo: bool = False) -> np.ndarray:
    """Sigma_{l1,l2} solving (Z_l1 (x) conj Z_l2) Sigma = C_{l1,l2} (Sections IV-A/B,
    eqs. linear_system2 and CTsubsystem), i.e. Z1 Sigma Z2^H = C with C = B1 K12 B2^H
    (= E[g1 g2^H] for g = B xi).  pseudo=True gives Z1 S Z2^T = B1 K12 B2^T."""
    C = B1 @ K12 @ (B2.T if pseudo else B2.conj().T)
    Y = np.linalg.solve(Z1, C)                      # Z1^{-1} C
    Z2x = Z2 if pseudo else Z2.conj()
    return np.linalg.solve(Z2x, Y.T).T              # Y Z2^{-H}  (resp. Y Z2^{-T})


def ct_index_sets(L0: int, L: int):
    """Lambda_+ = {l1 + l2 = L + L0}, Lambda_- = {l1 + l2 = L + L0 - 1}, with
    L0 <= l1, l2 <= L (Section IV-B)."""
    lp = [(l1, L + L0 - l1) for l1 in range(L0, L + 1) if L0 <= L + L0 - l1 <= L]
    lm = [(l1, L + L0 - 1 - l1) for l1 in range(L0, L + 1) if L0 <= L + L0 - 1 - l1 <= L]
    return lp, lm


def ct_hermitian_blocks(L0: int, L: int):
    """Blocks with l1 >= l2 and their signs (+1 on Lambda_+, -1 on Lambda_-): the
    Hermitian reduction Sigma_{l2,l1} = Sigma_{l1,l2}^H of Section IV-B."""
    lp, lm = ct_index_sets(L0, L)
    return [(b, +1) for b in lp if b[0] >= b[1]] + [(b, -1) for b in lm if b[0] >= b[1]]


def ct_dofs(N, L0: int, L: int, hermitian: bool = False):
    """N_hat_L = sum over Lambda of N_l1 N_l2 and N_hat_L^max (eq. efficiency, Section IV-B).
    N maps level -> number of dofs."""
    lp, lm = ct_index_sets(L0, L)
    blocks = lp + lm
    if hermitian:
        blocks = [b for b in blocks if b[0] >= b[1]]
    sizes = [N[a] * N[b] for a, b in blocks]
    return sum(sizes), max(sizes)


@dataclass
class Level:
    mesh: RWGMesh
    Z: np.ndarray
    u: np.ndarray
    A: np.ndarray
    B: np.ndarray


def nominal_level(mesh: RWGMesh, k: float, d, p, xhat, n_ss: int = 5) -> Level:
    """Assemble, solve and map one level: Z_l, u_l = Z_l^{-1} b_l, A_l, B_l(u_l)."""
    Z = assemble_z(mesh, k, n_ss)
    b = rhs_planewave(mesh, k, d, p)[:, 0]
    u = solve(Z, b)
    A = farfield_matrix(mesh, k, xhat)
    B = sd_rhs(mesh, k, u)
    return Level(mesh, Z, u, A, B)


def ct_farfield_covariance(levels: dict, L0: int, L: int, kernel: str, sigma: float, ell: float,
                           pseudo: bool = False) -> np.ndarray:
    """Far-field covariance of the combination technique (Section IV-B):
      Cov_hat = sum_{Lambda_+} A_l1 Sigma_{l1,l2} A_l2^H - sum_{Lambda_-} (same),
    computed for l1 >= l2 and mirrored (M + M^H) when l1 != l2.  pseudo=True gives the
    pseudo-covariance sum A_l1 S_{l1,l2} A_l2^T (mirrored with the transpose)."""
    out = None
    for (l1, l2), sgn in ct_hermitian_blocks(L0, L):
        a, b = levels[l1], levels[l2]
        K = cov_kernel(a.mesh.verts, b.mesh.verts, kernel, sigma, ell)
        S = covariance(a.Z, a.B, b.Z, b.B, K, pseudo)
        M = a.A @ S @ (b.A.T if pseudo else b.A.conj().T)
        if l1 != l2:
            M = M + (M.T if pseudo else M.conj().T)
        out = sgn * M if out is None else out + sgn * M
    return out


def pivoted_cholesky(K: np.ndarray, tol: float = 0.0, max_rank: int | None = None):
    """Pivoted (greedy) Cholesky factorisation K ~ L L^T of a symmetric positive
    semi-definite matrix: the low-rank factorisation of the tensor equations' right-hand
    side that Section VI names as further work (Harbrecht, Peters and Schneider 2012).
    With P the pivots chosen so far, the remainder is the Schur complement
    S = K - L L^T; each step takes the largest remaining diagonal entry of S (ties to the
    lowest index) as the next pivot p, appends the column S[:, p] / sqrt(S[p, p]), and
    the steps stop once trace(S) <= tol * trace(K), no positive diagonal entry is left,
    or max_rank columns exist.  Returns (L (n x m), pivots (m), trace(S))."""
    n = K.shape[0]
    max_rank = n if max_rank is None else min(int(max_rank), n)
    d = np.array(np.diag(K), dtype=float)
    trace = d.sum()
    used = np.zeros(n, dtype=bool)
    L = np.zeros((n, max_rank))
    piv = []
    err = trace
    m = 0
    while m < max_rank:
        cand = np.where(used, -np.inf, d)
        p = int(np.argmax(cand))
        if err <= tol * trace or not (cand[p] > 0.0):
            break
        lpp = math.sqrt(d[p])
        col = (K[:, p] - L[:, :m] @ L[p, :m]) / lpp   # column p of the Schur complement / sqrt(pivot)
        col[used] = 0.0
        col[p] = lpp
        L[:, m] = col
        d = d - col * col
        used[p] = True
        d[p] = 0.0
        piv.append(p)
        m += 1
        err = np.where(used, 0.0, np.maximum(d, 0.0)).sum()
    return L[:, :m], np.array(piv, dtype=np.int64), float(err)


def ct_farfield_covariance_lowrank(levels: dict, L0: int, L: int, kernel: str, sigma: float, ell: float,
                                   tol: float, max_rank: int | None = None, pseudo: bool = False):
    """The combination-technique far-field covariance (Section IV-B) with the covariance
    kernel replaced by its pivoted-Cholesky factor over the vertices of all levels
    L0..L stacked in level order, K ~ R R^T (Section VI): K_{l1,l2} ~ R_l1 R_l2^T, so
    Sigma_{l1,l2} ~ (Z_l1^{-1} B_l1 R_l1)(Z_l2^{-1} B_l2 R_l2)^H and, with
    Y_l = A_l Z_l^{-1} B_l R_l, each block's far-field term is Y_l1 Y_l2^H (Y_l1 Y_l2^T for
    the pseudo-covariance), mirrored when l1 != l2.  Returns (Cov, rank, trace error)."""
    lv = list(range(L0, L + 1))
    X = np.vstack([levels[l].mesh.verts for l in lv])
    R, _, err = pivoted_cholesky(cov_kernel(X, X, kernel, sigma, ell), tol, max_rank)
    Y, off = {}, 0
    for l in lv:
        a = levels[l]
        V = a.mesh.verts.shape[0]
        Y[l] = a.A @ np.linalg.solve(a.Z, a.B @ R[off:off + V])
        off += V
    out = None
    for (l1, l2), sgn in ct_hermitian_blocks(L0, L):
        M = Y[l1] @ (Y[l2].T if pseudo else Y[l2].conj().T)
        if l1 != l2:
            M = M + (M.T if pseudo else M.conj().T)
        out = sgn * M if out is None else out + sgn * M
    return out, R.shape[1], err


def rcs_variance_db(F: np.ndarray, cov: np.ndarray, pcov: np.ndarray) -> np.ndarray:
    """Delta-method variance of RCS_dB = 10 log10(|F|^2/(4 pi)) at each direction:
    Var = (20/ln 10)^2 Var[Re(conj F . F')]/|F|^4 with Var[Re z] = (E|z|^2 + Re E[z^2])/2,
    E|z|^2 = F^H-weighted covariance, E[z^2] from the pseudo-covariance.
    F: n_dir x 3; cov, pcov: (3 n_dir) x (3 n_dir)."""
    n = F.shape[0]
    out = np.zeros(n)
    for d in range(n):
        f = F[d]
        C = cov[3 * d:3 * d + 3, 3 * d:3 * d + 3]
        P = pcov[3 * d:3 * d + 3, 3 * d:3 * d + 3]
        ez2 = np.conj(f) @ C @ f             # E[z conj z], z = conj(f) . F'
        ezz = np.conj(f) @ P @ np.conj(f)    # E[z z]
        var_re = 0.5 * (ez2.real + ezz.real)
        out[d] = (20.0 / math.log(10.0)) ** 2 * var_re / np.sum(np.abs(f) ** 2) ** 2
    return out


def monte_carlo(mesh: RWGMesh, k: float, d, p, xhat, kind: str, sigma: float, ell: float, t: float, z):
    """Monte Carlo estimator of the far-field statistics (Section V-C): sample surfaces
    x_p + t xi_p n_p with xi = L z, L L^T = K + 1e-12 sigma^2 I (numpy Cholesky; z: nsamp x nv
    standard normal draws), each assembled and solved with LAPACK.  Returns (F0, the samples
    F_s (S x 3 n_dir), (1/S) sum D D^H, (1/S) sum D D^T) with D_s = (F_s - F0)/t."""
    K = cov_kernel(mesh.verts, mesh.verts, kind, sigma, ell) + 1e-12 * sigma**2 * np.eye(mesh.nv)
    xi = np.asarray(z, dtype=np.float64) @ np.linalg.cholesky(K).T

    def far(verts):
        m = RWGMesh(verts, mesh.tris, mesh.vnormals)
        u = solve(assemble_z(m, k), rhs_planewave(m, k, d, p)[:, 0])
        return farfield_matrix(m, k, xhat) @ u

    F0 = far(mesh.verts)
    Fs = np.stack([far(mesh.verts + t * x[:, None] * mesh.vnormals) for x in xi])
    D = (Fs - F0[None]) / t
    S = Fs.shape[0]
    return F0, Fs, D.T @ D.conj() / S, D.T @ D / S


def ct_second_moment_rank1(F: dict, L0: int, L: int) -> np.ndarray:
    """Combination-technique second moment of a rank-one tensor right-hand side (Section V-A):
    with M^2[f] = f (x) f the block system (Z_l1 (x) conj Z_l2) Sigma = f_l1 f_l2^H is solved by
    Sigma_{l1,l2} = x_l1 x_l2^H, whose far field is F_l1 F_l2^H; the CT sums it with signs over
    Lambda_+/- (Section IV-B), l1 >= l2 with the mirror.  F maps level -> far field vector."""
    out = None
    for (l1, l2), sgn in ct_hermitian_blocks(L0, L):
        M = np.outer(F[l1], np.conj(F[l2]))
        if l1 != l2:
            M = M + M.conj().T
        out = sgn * M if out is None else out + sgn * M
    return out


def dielectric_ct_second_moment(meshes: dict, k0: float, eps_r: float, mu_r: float, d, p, xhat, L0: int, L: int):
    """Section V-A's check of the CT on the dielectric sphere: every level's PMCHWT far field
    (dielectric_farfield, one plane wave) and the CT second moment of the rank-one right-hand
    side.  meshes maps level -> RWGMesh.  Returns (second moment (3 n_dir)^2, {level: F_l})."""
    F = {l: dielectric_farfield(meshes[l], k0, eps_r, mu_r, d, p, xhat)[3].reshape(-1) for l in range(L0, L + 1)}
    return ct_second_moment_rank1(F, L0, L), F


def monte_carlo_dielectric(mesh: RWGMesh, k0: float, eps_r: float, mu_r: float, d, p, xhat, kind: str,
                           sigma: float, ell: float, t: float, z):
    """The Monte Carlo estimator of Section V-C for a dielectric scatterer: the sample surfaces
    of monte_carlo (xi = L z, L L^T = K + 1e-12 sigma^2 I), each solved by the PMCHWT system
    (dielectric_farfield: assembly, LAPACK solve, far field of the exterior Cauchy data).
    Returns (F0, F_s (S x 3 n_dir), (1/S) sum D D^H, (1/S) sum D D^T), D_s = (F_s - F0)/t."""
    K = cov_kernel(mesh.verts, mesh.verts, kind, sigma, ell) + 1e-12 * sigma**2 * np.eye(mesh.nv)
    xi = np.asarray(z, dtype=np.float64) @ np.linalg.cholesky(K).T

    def far(verts):
        m = RWGMesh(verts, mesh.tris, mesh.vnormals)
        return dielectric_farfield(m, k0, eps_r, mu_r, d, p, xhat)[3].reshape(-1)

    F0 = far(mesh.verts)
    Fs = np.stack([far(mesh.verts + t * x[:, None] * mesh.vnormals) for x in xi])
    D = (Fs - F0[None]) / t
    S = Fs.shape[0]
    return F0, Fs, D.T @ D.conj() / S, D.T @ D / S


# ---------------------------------------------------------------------------
# Shape derivatives of the discrete quantities (forward mode, efie_oracle_grad.cpp)
# ---------------------------------------------------------------------------
def grad_value_z(mesh: RWGMesh, k: float, n_ss: int = 5) -> np.ndarray:
    """Z assembled from the value parts of the dual-number pair blocks (pins that the
    differentiated quadrature is the oracle's quadrature)."""
    qb, qw = triangle_rule6()
    gx, gw = gauss_legendre01(n_ss)
    N = mesh.n_edges
    Z = np.zeros((N, N), dtype=np.complex128)
    _load().orc_grad_value_z(_p(mesh.verts), _p(mesh.tris), ctypes.c_int64(mesh.nt), _p(mesh.tri_edge),
                             _p(mesh.tri_sign), ctypes.c_int64(N), ctypes.c_double(k), _p(qb), _p(qw),
                             ctypes.c_int(6), _p(gx), _p(gw), ctypes.c_int(n_ss), _p(Z))
    return Z


def rcs_monostatic_jacobian(mesh: RWGMesh, k: float, d, p, coords, n_ss: int = 5):
    """Monostatic RCS sigma_i = |F_i|^2/(4 pi), F_i = A(xh_i) u_i with xh_i = -d_i,
    u_i = Z^{-1} b_i (Sections II-C and IV-A), and its exact derivatives with respect to
    the vertex coordinates coords = [(p, c), ...] by forward-mode differentiation of the
    discrete quadrature:  d sigma_i = 2 Re(conj(F_i) . (dA_i u_i + A_i du_i))/(4 pi),
    du_i = Z^{-1}(db_i - dZ u_i).  Returns (sigma (n), J (n x len(coords)))."""
    inc = incidence(d, p)
    n = inc.shape[0]
    qb, qw = triangle_rule6()
    gx, gw = gauss_legendre01(n_ss)
    N = mesh.n_edges
    Z = assemble_z(mesh, k, n_ss)
    B = rhs_planewave(mesh, k, inc[:, :3], inc[:, 3:6] + 1j * inc[:, 6:9])
    U = np.ascontiguousarray(solve(Z, B))
    xh = np.ascontiguousarray(-inc[:, :3])
    A = farfield_matrix(mesh, k, xh)
    F = np.stack([A[3 * i:3 * i + 3] @ U[:, i] for i in range(n)])
    sigma = np.sum(np.abs(F) ** 2, axis=1) / (4 * np.pi)
    lib = _load()
    args = (_p(mesh.verts), _p(mesh.tris), ctypes.c_int64(mesh.nt), _p(mesh.tri_edge), _p(mesh.tri_sign),
            ctypes.c_int64(N), ctypes.c_double(k))
    J = np.zeros((n, len(coords)))
    for col, (pv, c) in enumerate(coords):
        dZU = np.zeros((N, n), dtype=np.complex128)
        for i in range(n):
            ui = np.ascontiguousarray(U[:, i])
            out = np.zeros(N, dtype=np.complex128)
            lib.orc_grad_dz_u(*args, _p(qb), _p(qw), ctypes.c_int(6), _p(gx), _p(gw), ctypes.c_int(n_ss),
                              ctypes.c_int32(pv), ctypes.c_int(c), _p(ui), _p(out))
            dZU[:, i] = out
        dB = np.zeros((N, n), dtype=np.complex128)
        lib.orc_grad_db(*args, _p(qb), _p(qw), ctypes.c_int(6), ctypes.c_int32(pv), ctypes.c_int(c), _p(inc),
                        ctypes.c_int64(n), _p(dB))
        dAU = np.zeros((3 * n, n), dtype=np.complex128)
        lib.orc_grad_da_u(*args, _p(qb), _p(qw), ctypes.c_int(6), ctypes.c_int32(pv), ctypes.c_int(c), _p(xh),
                          ctypes.c_int64(n), _p(U), ctypes.c_int64(n), _p(dAU))
        dU = np.linalg.solve(Z, dB - dZU)
        for i in range(n):
            dF = dAU[3 * i:3 * i + 3, i] + A[3 * i:3 * i + 3] @ dU[:, i]
            J[i, col] = 2.0 * np.real(np.vdot(F[i], dF)) / (4 * np.pi)
    return sigma, J
