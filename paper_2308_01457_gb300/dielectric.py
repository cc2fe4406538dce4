"""Dielectric scatterer over a mesh hierarchy: every level's PMCHWT solve (Section II-C eq.
pmchwt) and the combination-technique second moment of the paper's convergence check on
the dielectric unit sphere (Section V-A): with the rank-one tensor right-hand side
M^2[f] = f (x) f, the block system (Z_l1 (x) conj Z_l2) Sigma_{l1,l2} = f_l1 f_l2^H is solved by
Sigma_{l1,l2} = x_l1 x_l2^H, so its far-field block is F_l1 F_l2^H, and the CT sums the blocks
over Lambda_+/- (Section IV-B), l1 >= l2 with the mirror.  Sequence of C-ABI calls only:
fosb_assemble_pmchwt, fosb_factor, fosb_solve, fosb_farfield_pmchwt, fosb_lowrank_combine."""
from __future__ import annotations

import numpy as np

from . import (ASM_FF, MIXED, assemble_pmchwt, factor, farfield_pmchwt, incidence, lowrank_combine, mesh_create,
               solve)
from .ct import hermitian_blocks


class DielectricCT:
    """meshes: level -> object with verts, tris, vnormals (levels L0..L); one plane wave (d, p);
    observation directions dirs (n_dir x 3)."""

    def __init__(self, meshes: dict, k0: float, eps_r: float, mu_r: float, d, p, dirs, L0: int, L: int,
                 arith: int = ASM_FF, prec: int = MIXED, device: str = "cuda:0"):
        self.src, self.k0, self.eps_r, self.mu_r = meshes, k0, eps_r, mu_r
        self.inc = incidence(d, p)
        self.dirs = np.ascontiguousarray(dirs, dtype=np.float64)
        self.L0, self.L, self.arith, self.prec, self.device = L0, L, arith, prec, device
        self.berr = {}

    def setup(self):
        self.meshes = {l: mesh_create(self.src[l].verts, self.src[l].tris, self.src[l].vnormals)
                       for l in range(self.L0, self.L + 1)}
        return self

    def farfield(self, l):
        """Level l's PMCHWT solve; returns its far field (3 n_dir x 1 device tensor)."""
        import torch

        m = self.meshes[l]
        n2 = 2 * m.n_edges
        c128 = torch.complex128
        Z = torch.empty((n2, n2), dtype=c128, device=self.device)
        b = torch.empty((n2, 1), dtype=c128, device=self.device)
        assemble_pmchwt(m, self.k0, self.eps_r, self.mu_r, Z, inc=self.inc, b=b, arith=self.arith)
        lu = factor(Z, prec=self.prec)
        _, _, self.berr[l] = solve(lu, b)
        del lu, Z
        F = torch.empty((3 * self.dirs.shape[0], 1), dtype=c128, device=self.device)
        farfield_pmchwt(m, self.k0, self.dirs, b, F)
        return F

    def run(self):
        """Returns (the finest level's far field F_L (3 n_dir), the CT second moment (3 n_dir)^2)."""
        import torch

        F = {l: self.farfield(l) for l in range(self.L0, self.L + 1)}
        nd3 = 3 * self.dirs.shape[0]
        M = torch.empty((nd3, nd3), dtype=torch.complex128, device=self.device)
        for i, ((l1, l2), sgn) in enumerate(hermitian_blocks(self.L0, self.L)):
            lowrank_combine(F[l1], F[l2], M, weight=float(sgn), mirror=l1 != l2, accumulate=i > 0)
        return F[self.L][:, 0], M
