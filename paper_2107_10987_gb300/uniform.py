"""RK3 time stepping of a uniform octree level through the C ABI (plumbing only).

A uniform level of nbx x nby x nbz sub-grids (sub-grid s = (kz*nby + ky)*nbx
+ kx) with periodic or outflow boundaries: two state buffers used in turn
(the first stage of a step writes the other buffer), the work buffers of
hydro_step, an optional static gravitational field, and optionally the step
captured once into a CUDA graph.  Every step of the method runs in the
library's kernels; this class only owns buffers and orders calls.
"""
from __future__ import annotations

import numpy as np
import torch

from . import hydro as H


class UniformRun:
    def __init__(self, ctx, U, origin, h, nb, bc: int = H.HYDRO_BC_OUTFLOW, g=None, cfl: float = 0.4,
                 device="cuda", fused: bool = False):
        """U: [n][F][N][N][N] interiors or [n][F][S][S][S] padded states (array
        or tensor; N the context's sub-grid edge, 8 or 16, S = N + 6); origin
        [n][3]; h scalar or [n]; nb = (nbx, nby, nbz) or an int; g: optional
        [n][3][N][N][N] gravitational acceleration; fused:
        each time step as one persistent launch (mixed precision; the ghost
        layers of the state buffers are then not maintained)."""
        self.ctx = ctx
        self.nb = (nb, nb, nb) if isinstance(nb, int) else tuple(nb)
        U = torch.as_tensor(U)
        n = U.shape[0]
        assert n == self.nb[0] * self.nb[1] * self.nb[2]
        self.N = N = getattr(ctx, "N", 8)  # the sub-grids' edge (8 or 16)
        Sp = N + 6
        a = torch.zeros((n, 10, Sp, Sp, Sp), dtype=torch.float64, device=device)
        self.bufs = (a, torch.zeros_like(a))
        self.origin = torch.as_tensor(np.asarray(origin, dtype=np.float64)).to(device).contiguous()
        self.h = torch.as_tensor(np.broadcast_to(np.asarray(h, dtype=np.float64), (n,)).copy()).to(device)
        self.g = torch.as_tensor(g).to(device).contiguous() if g is not None else None
        if U.shape[-1] == N:
            H.hydro_scatter_interior(ctx, H.make_batch(a, self.origin, self.h), U.to(device).contiguous())
        else:
            a.copy_(U)
        self.dU = torch.empty((n, 10, N, N, N), dtype=torch.float64, device=device)
        self.am = torch.empty(n, dtype=torch.float64, device=device)
        self.dt = torch.empty(1, dtype=torch.float64, device=device)
        self.sums_buf = torch.empty(11, dtype=torch.float64, device=device)
        self.desc = H.make_rk3_desc(self.bufs[0], self.bufs[1], self.origin, self.h, self.nb, bc, self.dU, self.am,
                                    self.dt, cfl, g=self.g, fused=fused)
        self.batches = (H.make_batch(self.bufs[0], self.origin, self.h, self.g),
                        H.make_batch(self.bufs[1], self.origin, self.h, self.g))
        self.parity = 0
        self.graph = None
        self.n = n

    @property
    def U(self):
        return self.bufs[self.parity]

    def step(self, use_graph: bool = False):
        """One RK3 step (asynchronous); dt from the first stage's amax."""
        if use_graph:
            if self.graph is None:
                assert self.parity == 0, "capture starts from the first buffer"
                self.graph = H.hydro_rk3_graph_create(self.ctx, self.desc)
            H.hydro_rk3_graph_launch(self.graph)
        else:
            H.hydro_rk3_step(self.ctx, self.desc, self.parity)
        self.parity ^= 1

    def last_dt(self) -> float:
        """dt of the last step (synchronises)."""
        return self.dt.item()

    def sums(self) -> np.ndarray:
        """sum U h^3 per field and the angular momentum about +z (synchronises)."""
        H.hydro_conserved_sums(self.ctx, self.batches[self.parity], self.sums_buf)
        return self.sums_buf.cpu().numpy()

    def interior(self) -> torch.Tensor:
        """The current interiors, [n][F][N][N][N] (a new tensor)."""
        out = torch.empty((self.n, 10, self.N, self.N, self.N), dtype=torch.float64, device=self.U.device)
        H.hydro_gather_interior(self.ctx, self.batches[self.parity], out)
        return out

    def close(self):
        if self.graph is not None:
            H.hydro_rk3_graph_destroy(self.graph)
            self.graph = None
