"""Batched scatterers on one GPU: many independent EFIE systems of uneven size, each with
several plane waves, assembled together (one persistent launch for all regular pairs) and
factored and solved together (a worker pool over streams, largest first), all through the
C ABI.  The paper processes its independent sub-systems concurrently (Section V-D)."""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import ASM_FF, MIXED, assemble_efie_batched, incidence, mesh_create, solve_batched


@dataclass
class BatchedProblem:
    """meshes[i] (objects with verts, tris, vnormals), wavenumbers ks[i], and the plane waves
    (directions d, polarisations p) shared by every scatterer."""

    meshes: list
    ks: list
    d: np.ndarray
    p: np.ndarray
    prec: int = MIXED
    arith: int = ASM_FF
    workers: int = 4
    handles: list = field(default_factory=list)

    def setup(self, device="cuda:0"):
        import torch

        self.inc = incidence(self.d, self.p)
        n_inc = self.inc.shape[0]
        self.handles = [mesh_create(sm.verts, sm.tris, sm.vnormals) for sm in self.meshes]
        self.Z = [torch.empty((h.n_edges, h.n_edges), dtype=torch.complex128, device=device) for h in self.handles]
        self.B = [torch.empty((h.n_edges, n_inc), dtype=torch.complex128, device=device) for h in self.handles]
        self.X = [torch.empty_like(b) for b in self.B]
        return self

    def assemble(self, tune: bool = True):
        self.tuning = assemble_efie_batched(self.handles, self.ks, self.Z, [self.inc] * len(self.handles), self.B,
                                            arith=self.arith, tune=tune)
        return self.tuning

    def solve(self):
        self.iters, self.berr, self.status = solve_batched(self.Z, self.B, self.X, prec=self.prec,
                                                           workers=self.workers)
        return self.X

    def run(self, tune: bool = True):
        self.assemble(tune)
        return self.solve()

    @property
    def entries(self) -> int:
        return sum(h.n_edges ** 2 for h in self.handles)
