"""Monte Carlo over random normal perturbations of one scatterer (the paper's reference
estimator, Section V-C) on the GPU: sample surfaces x_p + t xi_p n_p with xi ~ N(0, K) from
the caller's standard normal draws, all samples assembled together (one persistent launch
per chunk), factored and solved by the batched scheduler, their far fields formed, and the
sample mean, covariance and pseudo-covariance of (F_s - F_0)/t computed on the device --
all through the C ABI."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import (ASM_FF, COV_GAUSS, MIXED, assemble_efie, assemble_efie_batched, factor, farfield_moments,
               field_samples, incidence, mc_moments, mesh_create, mesh_perturb, solve, solve_batched)


@dataclass
class MonteCarloProblem:
    """mesh: object with verts, tris, vnormals; one plane wave (d, p); observation directions
    dirs (n_dir x 3); covariance kernel of the normal velocity; amplitude t; z: nsamp x nv
    standard normal draws (the random numbers of the estimator)."""

    mesh: object
    k: float
    d: tuple
    p: tuple
    dirs: np.ndarray
    z: np.ndarray
    kernel: int = COV_GAUSS
    sigma: float = 1.0
    ell: float = 1.0
    t: float = 1.0
    chunk: int = 128
    workers: int = 8
    prec: int = MIXED
    arith: int = ASM_FF

    def setup(self, device="cuda:0"):
        self.device = device
        self.base = mesh_create(self.mesh.verts, self.mesh.tris, self.mesh.vnormals)
        self.xi = field_samples(self.base, self.z, self.kernel, self.sigma, self.ell)
        self.inc = incidence(self.d, self.p)
        return self

    def run(self):
        """Returns device tensors (F0 (3 n_dir), mean (3 n_dir), cov, pcov (3 n_dir x 3 n_dir))."""
        import torch

        dev, c128 = self.device, torch.complex128
        nsamp, n3 = self.z.shape[0], 3 * self.dirs.shape[0]
        N = self.base.n_edges
        Z0 = torch.empty((N, N), dtype=c128, device=dev)
        b0 = torch.empty((N, 1), dtype=c128, device=dev)
        assemble_efie(self.base, self.k, Z0, inc=self.inc, b=b0, arith=self.arith, prec=self.prec)
        lu = factor(Z0, prec=self.prec)
        u0 = torch.empty_like(b0)
        solve(lu, b0, u0)
        del lu
        F0 = torch.empty((n3, 1), dtype=c128, device=dev)
        farfield_moments(self.base, self.k, self.dirs, u0, F0, prec=self.prec)
        Fs = torch.empty((n3, nsamp), dtype=c128, device=dev)
        for c0 in range(0, nsamp, self.chunk):
            ids = range(c0, min(nsamp, c0 + self.chunk))
            hs = [mesh_perturb(self.base, self.xi[s], self.t) for s in ids]
            Zs = [torch.empty((N, N), dtype=c128, device=dev) for _ in hs]
            Bs = [torch.empty((N, 1), dtype=c128, device=dev) for _ in hs]
            assemble_efie_batched(hs, [self.k] * len(hs), Zs, [self.inc] * len(hs), Bs, arith=self.arith)
            solve_batched(Zs, Bs, Bs, prec=self.prec, workers=self.workers)
            for j, s in enumerate(ids):
                farfield_moments(hs[j], self.k, self.dirs, Bs[j], Fs[:, s:s + 1], prec=self.prec)
            del Zs, Bs, hs
        mean = torch.empty(n3, dtype=c128, device=dev)
        cov = torch.empty((n3, n3), dtype=c128, device=dev)
        pcov = torch.empty((n3, n3), dtype=c128, device=dev)
        mc_moments(Fs, F0, self.t, mean, cov, pcov)
        return F0[:, 0], mean, cov, pcov
