"""torch.autograd.Function for monostatic RCS with respect to the mesh vertices.

forward: EFIE assembly, mixed-precision LU with FP64 refinement and the solves for the
given plane waves, then sigma_i = |F(-d_i)|^2 / (4 pi) -- all through the C ABI.
backward: the hand-written adjoint (fosb_rcs_monostatic with weights = grad_output):
lambda = Z^{-1} A^T c, then reverse-mode kernels over the triangle pairs and triangles.
The factorisation is kept from forward to backward (it is reused for the adjoint solve).
"""
from __future__ import annotations

import numpy as np
import torch

from . import MIXED, assemble_efie, factor, incidence, mesh_create, rcs_monostatic, solve


class FosbRCS(torch.autograd.Function):
    """sigma = FosbRCS.apply(verts, tris, k, d, p, db): verts (V x 3, float64, any device)
    -> sigma (n, float64 on verts.device); db=True returns RCS_dB = 10 log10(sigma) (the
    conversion and its chain rule run in the library)."""

    @staticmethod
    def forward(ctx, verts, tris, k, d, p, db=False):
        v = verts.detach().to("cpu", torch.float64).numpy()
        t = np.asarray(tris, np.int32)
        mesh = mesh_create(v, t)
        inc = incidence(d, p)
        n = inc.shape[0]
        N = mesh.n_edges
        dev = torch.device("cuda", torch.cuda.current_device())
        Z = torch.empty((N, N), dtype=torch.complex128, device=dev)
        b = torch.empty((N, n), dtype=torch.complex128, device=dev)
        assemble_efie(mesh, k, Z, inc=inc, b=b)
        lu = factor(Z, prec=MIXED)
        U = torch.empty_like(b)
        solve(lu, b, U)
        out = rcs_monostatic(mesh, k, inc, U, db=bool(db))
        ctx.state = (mesh, lu, Z, U, inc, k, bool(db), verts.device)
        return torch.tensor(out, dtype=torch.float64, device=verts.device)

    @staticmethod
    def backward(ctx, grad_out):
        mesh, lu, Z, U, inc, k, db, vdev = ctx.state
        g = grad_out.detach().to("cpu", torch.float64).numpy()
        grad = torch.zeros((mesh.nv, 3), dtype=torch.float64, device=Z.device)
        rcs_monostatic(mesh, k, inc, U, lu=lu, weights=g, grad=grad, db=db)
        return grad.to(vdev), None, None, None, None, None
