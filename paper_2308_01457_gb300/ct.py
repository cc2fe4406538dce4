"""Combination-technique driver of the FOSB second moment (Section IV-B) on one GPU.

The index sets Lambda_+/- and the Hermitian reduction are host bookkeeping; every
numerical step runs through the C ABI (assembly, factorisation, refined solves,
covariance blocks, far-field moments).
"""
from __future__ import annotations

import threading
from dataclasses import dataclass, field

import numpy as np

from . import (ASM_FP64, COV_GAUSS, FP32, MIXED, assemble_efie, covariance, covariance_lowrank, factor,
               farfield_moments, incidence, kernel_lowrank, lowrank_combine, mesh_create, rcs_moments, solve)


def index_sets(L0: int, L: int):
    """Lambda_+ = {(l1, l2): l1 + l2 = L + L0}, Lambda_- = {l1 + l2 = L + L0 - 1}, both
    restricted to L0 <= l1, l2 <= L."""
    plus = [(a, L + L0 - a) for a in range(L0, L + 1) if L0 <= L + L0 - a <= L]
    minus = [(a, L + L0 - 1 - a) for a in range(L0, L + 1) if L0 <= L + L0 - 1 - a <= L]
    return plus, minus


def hermitian_blocks(L0: int, L: int):
    """The blocks actually solved: l1 >= l2 on Lambda_+ (sign +1) and Lambda_- (sign -1);
    Sigma_{l2,l1} = Sigma_{l1,l2}^H supplies the rest (Section IV-B)."""
    plus, minus = index_sets(L0, L)
    return [(b, 1) for b in plus if b[0] >= b[1]] + [(b, -1) for b in minus if b[0] >= b[1]]


def dofs(n_of_level, L0: int, L: int):
    """(N_hat_L, N_hat_L^max) of eq. efficiency for the full index set Lambda."""
    plus, minus = index_sets(L0, L)
    sizes = [n_of_level[a] * n_of_level[b] for a, b in plus + minus]
    return sum(sizes), max(sizes)


@dataclass
class LevelState:
    mesh: object
    Z: object
    b: object
    u: object = None
    lu: object = None
    iters: int = 0
    berr: float = 0.0


@dataclass
class FOSBProblem:
    """One FOSB run: meshes of levels L0..L (meshes[i] is level L0 + i), wavenumber k,
    one plane wave (d, p), observation directions, covariance kernel of the normal
    perturbation."""

    meshes: list
    k: float
    d: tuple
    p: tuple
    dirs: np.ndarray
    L0: int
    L: int
    kernel: int = COV_GAUSS
    sigma: float = 1.0
    ell: float = 1.0
    prec: int = MIXED
    arith: int = ASM_FP64
    n_ss: int = 5
    pseudo: bool = False
    # low-rank right-hand side (Section VI): None solves every CT block with fosb_covariance;
    # a tolerance factors the kernel over all levels' vertices by pivoted Cholesky to that
    # relative trace error and forms each block as Y_l1 Y_l2^H (fosb_covariance_lowrank)
    lowrank_tol: float | None = None
    max_rank: int | None = None
    # run the coarser levels' assembly, factorisation and solve on a high-priority side stream
    # while the finest level's assembly runs, then the CT blocks without the finest level (in a
    # host thread, on the same side stream) while it factors and solves: the levels and those
    # blocks are independent of the finest level until the signed sum
    overlap: bool = True
    levels: dict = field(default_factory=dict)

    def setup(self, device="cuda:0"):
        """fosb_mesh_create for every level and device buffers for Z and b (A1)."""
        import torch

        dt = torch.complex64 if self.prec == FP32 else torch.complex128
        for i, sm in enumerate(self.meshes):
            l = self.L0 + i
            m = mesh_create(sm.verts, sm.tris, sm.vnormals)
            N = m.n_edges
            self.levels[l] = LevelState(m, torch.empty((N, N), dtype=dt, device=device),
                                        torch.empty((N, 1), dtype=dt, device=device))
        self.inc = incidence(self.d, self.p)
        return self

    def nominal(self, l: int, timers=None):
        """A2-A6 for one level: assembly, factorisation, refined solve.  timers: optional
        dict name -> list of (start, end) CUDA events recorded on the current stream."""
        self.assemble(l, timers)
        self.factor_solve(l, timers)

    @staticmethod
    def _ev(timers, name, l):
        import torch

        if timers is None:
            return None
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        timers.setdefault(f"{name}_l{l}", []).append((a, b))
        a.record()
        return b

    def assemble(self, l: int, timers=None):
        """A2-A4 for one level (enqueued on the current stream)."""
        st = self.levels[l]
        e = self._ev(timers, "assemble", l)
        assemble_efie(st.mesh, self.k, st.Z, inc=self.inc, b=st.b, n_ss=self.n_ss, arith=self.arith, prec=self.prec)
        if e is not None:
            e.record()

    def factor_solve(self, l: int, timers=None):
        """A5-A6 for one level: factorisation and refined solve (both synchronise the stream)."""
        import torch

        st = self.levels[l]
        ev = lambda name: self._ev(timers, name, l)
        e = ev("factor")
        st.lu = factor(st.Z, prec=self.prec)
        if e is not None:
            e.record()
        if st.u is None:
            st.u = torch.empty_like(st.b)
        e = ev("solve")
        _, st.iters, st.berr = solve(st.lu, st.b, st.u)
        if e is not None:
            e.record()
        return st

    def run(self, timers=None):
        """Full step: nominal solves on all levels, the mean far field on level L, the CT
        far-field covariance (and pseudo-covariance if requested) and the RCS moments
        (self.rcs_db, self.var_f, and self.var_db with the pseudo-covariance).  Returns
        device tensors (F_mean (3 n_dir x 1), Cov (3 n_dir x 3 n_dir)[, PCov])."""
        import torch

        nd3 = 3 * self.dirs.shape[0]
        dt = self.levels[self.L].Z.dtype
        dev = self.levels[self.L].Z.device
        lv = sorted(self.levels)
        fine = self.levels[self.L]
        cov = torch.empty((nd3, nd3), dtype=dt, device=dev)
        pcov = torch.empty((nd3, nd3), dtype=dt, device=dev) if self.pseudo else None
        blocks = hermitian_blocks(self.L0, self.L)
        early = []  # CT blocks computed beside the finest level's factorisation
        if self.overlap and len(lv) > 1:
            main = torch.cuda.current_stream()
            if getattr(self, "_side", None) is None:
                self._side = torch.cuda.Stream(device=dev, priority=-5)  # clamped to the highest priority
            side = self._side
            side.wait_stream(main)  # the coarse Z, b and the outputs may still be used by earlier work on main
            self.assemble(lv[-1], timers)
            with torch.cuda.stream(side):
                for l in lv[:-1]:
                    self.nominal(l, timers)
            worker, err = None, []
            if self.lowrank_tol is None:
                # the blocks without the finest level need none of its results: a host thread
                # computes them on the side stream while this one factors and solves level L
                early = [b for b in blocks if self.L not in b[0]]

                def coarse():
                    try:
                        torch.cuda.set_device(dev)
                        with torch.cuda.stream(side):
                            self._full_blocks(cov, pcov, early, first=True)
                    except BaseException as e:  # re-raised by the caller after the join
                        err.append(e)

                if early:
                    cov.record_stream(side)
                    if pcov is not None:
                        pcov.record_stream(side)
                    worker = threading.Thread(target=coarse, name="fosb-ct-coarse-blocks")
                    worker.start()
            try:
                self.factor_solve(lv[-1], timers)
            finally:
                if worker is not None:
                    worker.join()
            if err:
                raise err[0]
            main.wait_stream(side)
        else:
            for l in lv:
                self.nominal(l, timers)
        if timers is not None:
            cov_start = torch.cuda.Event(enable_timing=True)
            cov_start.record()
        F = torch.empty((nd3, 1), dtype=dt, device=dev)
        farfield_moments(fine.mesh, self.k, self.dirs, fine.u, F, prec=self.prec)
        if self.lowrank_tol is not None:
            self._lowrank_blocks(cov, pcov)
        else:
            self._full_blocks(cov, pcov, [b for b in blocks if b not in early], first=not early)
        # A11: RCS_dB of the mean field and the variance of every far-field component; with the
        # pseudo-covariance also the delta-method variance of RCS_dB (device float64 tensors)
        n_dir = self.dirs.shape[0]
        self.rcs_db = torch.empty(n_dir, dtype=torch.float64, device=dev)
        self.var_f = torch.empty(nd3, dtype=torch.float64, device=dev)
        self.var_db = torch.empty(n_dir, dtype=torch.float64, device=dev) if pcov is not None else None
        rcs_moments(n_dir, F, cov, pcov, rcs_db=self.rcs_db, var_db=self.var_db, var_f=self.var_f, prec=self.prec)
        if timers is not None:
            cov_end = torch.cuda.Event(enable_timing=True)
            cov_end.record()
            timers.setdefault("covariance_ct", []).append((cov_start, cov_end))
        return (F, cov) if pcov is None else (F, cov, pcov)

    def _full_blocks(self, cov, pcov, blocks, first=True):
        """CT sum over `blocks` ((l1, l2), sign) of the Hermitian blocks, each Sigma_{l1,l2}
        from fosb_covariance and projected by fosb_farfield_moments (mirrored when l1 != l2);
        first: the first block overwrites the outputs, the others add to them."""
        import torch

        for (l1, l2), sgn in blocks:
            a, c = self.levels[l1], self.levels[l2]
            for pseudo, out in ((False, cov), (True, pcov)):
                if out is None:
                    continue
                Sig = torch.empty((a.mesh.n_edges, c.mesh.n_edges), dtype=cov.dtype, device=cov.device)
                covariance(a.mesh, a.lu, a.u, c.mesh, c.lu, c.u, self.k, Sig, self.kernel, self.sigma, self.ell,
                           pseudo=pseudo)
                farfield_moments(a.mesh, self.k, self.dirs, Sig, out, m2=c.mesh, weight=float(sgn), mirror=(l1 != l2),
                                 prec=self.prec, pseudo=pseudo, accumulate=not first)
            first = False

    def _lowrank_blocks(self, cov, pcov):
        """CT sum with the kernel factor K ~ R^T R over the vertices of levels L0..L:
        Y_l = A_l Z_l^{-1} B_l R_l^T once per level, then Y_l1 Y_l2^H (and Y_l1 Y_l2^T for the
        pseudo-covariance) per block.  Sets self.rank and self.trace_err."""
        lv = list(range(self.L0, self.L + 1))
        dev = self.levels[self.L].Z.device
        R, self.rank, self.trace_err, offs = kernel_lowrank([self.levels[l].mesh for l in lv], self.kernel, self.sigma,
                                                            self.ell, self.lowrank_tol, self.max_rank, device=dev)
        Y = {}
        for l, off in zip(lv, offs):
            st = self.levels[l]
            Y[l] = covariance_lowrank(st.mesh, st.lu, st.u, self.k, R[:, off:off + st.mesh.nv], self.dirs)
        first = True
        for (l1, l2), sgn in hermitian_blocks(self.L0, self.L):
            for pseudo, out in ((False, cov), (True, pcov)):
                if out is not None:
                    lowrank_combine(Y[l1], Y[l2], out, weight=float(sgn), mirror=(l1 != l2), pseudo=pseudo,
                                    accumulate=not first, prec=self.prec)
            first = False

    def release(self):
        for st in self.levels.values():
            st.lu = None
