"""Monte Carlo over random normal perturbations of one scatterer (the paper's reference
estimator, Section V-C) on the GPU: sample surfaces x_p + t xi_p n_p with xi ~ N(0, K) from
the caller's standard normal draws, all samples assembled together (one persistent launch
per chunk), factored and solved by the batched scheduler, their far fields formed, and the
sample mean, covariance and pseudo-covariance of (F_s - F_0)/t computed on the device --
all through the C ABI.  With eps_r given the scatterer is dielectric: every surface is
solved by the PMCHWT system (fosb_assemble_pmchwt, the batched factorisation and solves of
the 2N x 2N systems, fosb_farfield_pmchwt)."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import (ASM_FF, COV_GAUSS, MIXED, assemble_efie, assemble_efie_batched, assemble_pmchwt, factor,
               farfield_moments, farfield_pmchwt, field_samples, incidence, mc_moments, mesh_create, mesh_perturb,
               solve, solve_batched)


@dataclass
class MonteCarloProblem:
    """mesh: object with verts, tris, vnormals; one plane wave (d, p); observation directions
    dirs (n_dir x 3); covariance kernel of the normal velocity; amplitude t; z: nsamp x nv
    standard normal draws (the random numbers of the estimator); eps_r, mu_r: relative
    permittivity and permeability of a dielectric scatterer (eps_r None: perfect conductor)."""

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
    eps_r: float | None = None
    mu_r: float = 1.0

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
        de = self.eps_r is not None
        N = self.base.n_edges * (2 if de else 1)

        def assemble(m, Z, b):
            if de:
                assemble_pmchwt(m, self.k, self.eps_r, self.mu_r, Z, inc=self.inc, b=b, arith=self.arith)
            else:
                assemble_efie(m, self.k, Z, inc=self.inc, b=b, arith=self.arith, prec=self.prec)

        def far(m, X, out):
            if de:
                farfield_pmchwt(m, self.k, self.dirs, X, out)
            else:
                farfield_moments(m, self.k, self.dirs, X, out, prec=self.prec)

        Z0 = torch.empty((N, N), dtype=c128, device=dev)
        b0 = torch.empty((N, 1), dtype=c128, device=dev)
        assemble(self.base, Z0, b0)
        lu = factor(Z0, prec=self.prec)
        u0 = torch.empty_like(b0)
        solve(lu, b0, u0)
        del lu
        F0 = torch.empty((n3, 1), dtype=c128, device=dev)
        far(self.base, u0, F0)
        Fs = torch.empty((n3, nsamp), dtype=c128, device=dev)
        for c0 in range(0, nsamp, self.chunk):
            ids = range(c0, min(nsamp, c0 + self.chunk))
            hs = [mesh_perturb(self.base, self.xi[s], self.t) for s in ids]
            Zs = [torch.empty((N, N), dtype=c128, device=dev) for _ in hs]
            Bs = [torch.empty((N, 1), dtype=c128, device=dev) for _ in hs]
            if de:
                for j in range(len(hs)):
                    assemble(hs[j], Zs[j], Bs[j])
            else:
                assemble_efie_batched(hs, [self.k] * len(hs), Zs, [self.inc] * len(hs), Bs, arith=self.arith)
            solve_batched(Zs, Bs, Bs, prec=self.prec, workers=self.workers)
            for j, s in enumerate(ids):
                far(hs[j], Bs[j], Fs[:, s:s + 1])
            del Zs, Bs, hs
        mean = torch.empty(n3, dtype=c128, device=dev)
        cov = torch.empty((n3, n3), dtype=c128, device=dev)
        pcov = torch.empty((n3, n3), dtype=c128, device=dev)
        mc_moments(Fs, F0, self.t, mean, cov, pcov)
        return F0[:, 0], mean, cov, pcov
