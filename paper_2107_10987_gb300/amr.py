"""Host-side description of an adaptive octree for the C ABI (plumbing only).

For every level l of the mesh a dense table over the (2^l)^3 sub-grid
positions holds the index of the leaf at that position (>= 0), -1 where the
position is refined into finer leaves, or -2 where it lies inside a coarser
leaf.  The ghost fill and the coarse-fine flux correction kernels look leaves
up in these tables.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import hydro as H


class AMRDesc(C.Structure):
    _fields_ = [("lmin", C.c_int), ("lmax", C.c_int), ("table", C.c_void_p), ("leaf_level", C.c_void_p),
                ("leaf_ijk", C.c_void_p), ("bc", C.c_int), ("order", C.c_void_p)]


def build_tables(level: np.ndarray, ijk: np.ndarray):
    """Concatenated per-level tables (int32), level l at offset
    sum_{m<l} 8^m (m from lmin), index ((k * 2^l) + j) * 2^l + i."""
    level = np.asarray(level)
    ijk = np.asarray(ijk)
    lmin, lmax = int(level.min()), int(level.max())
    tabs = {l: np.full((2 ** l,) * 3, -2, dtype=np.int32) for l in range(lmin, lmax + 1)}
    for s, (l, (i, j, k)) in enumerate(zip(level.tolist(), ijk.tolist())):
        tabs[l][k, j, i] = s
        # coarser levels: the ancestors are refined
        for lc in range(lmin, l):
            sh = l - lc
            tabs[lc][k >> sh, j >> sh, i >> sh] = -1
    # consistency: every position is a leaf, refined, or inside a coarser leaf
    flat = np.concatenate([tabs[l].ravel() for l in range(lmin, lmax + 1)])
    return lmin, lmax, flat


def morton_order(level: np.ndarray, ijk: np.ndarray) -> np.ndarray:
    """The leaves along the Z-order (Morton) curve of their first cells at the
    finest level: a permutation of 0 .. n-1 that keeps spatial neighbours
    close, for the kernels' processing order (int32)."""
    level = np.asarray(level, dtype=np.int64)
    ijk = np.asarray(ijk, dtype=np.int64)
    lmax = int(level.max())
    p = ijk << (lmax - level)[:, None]
    key = np.zeros(len(level), dtype=np.int64)
    for b in range(lmax + 1):
        for d in range(3):
            key |= ((p[:, d] >> b) & 1) << (3 * b + d)
    return np.argsort(key, kind="stable").astype(np.int32)


class AMRMesh:
    """Device copy of the tables and leaf coordinates of a mesh, and the order
    in which the kernels take the leaves (order="morton": along the Z-order
    curve, None: index order; results are the same either way)."""

    def __init__(self, level, ijk, bc: int = H.HYDRO_BC_OUTFLOW, device="cuda", order="morton"):
        self.level = np.asarray(level, dtype=np.int32)
        self.ijk = np.ascontiguousarray(ijk, dtype=np.int32)
        self.lmin, self.lmax, flat = build_tables(self.level, self.ijk)
        self.table = torch.tensor(flat, device=device)
        self.leaf_level = torch.tensor(self.level, device=device)
        self.leaf_ijk = torch.tensor(self.ijk.reshape(-1), device=device)
        self.bc = bc
        self.order = (torch.tensor(morton_order(self.level, self.ijk), device=device) if order == "morton"
                      else None)
        self.desc = AMRDesc(self.lmin, self.lmax, self.table.data_ptr(), self.leaf_level.data_ptr(),
                            self.leaf_ijk.data_ptr(), bc,
                            self.order.data_ptr() if self.order is not None else None)


class AMRRun:
    """RK3 time stepping of a batch of AMR leaves through the C ABI: two state
    buffers (ping-pong), the work buffers, and optionally a captured graph."""

    def __init__(self, ctx, U, level, ijk, bc: int = H.HYDRO_BC_OUTFLOW, cfl: float = 0.4, device="cuda",
                 order="morton", g=None):
        from . import workloads as W
        self.ctx = ctx
        self.mesh = AMRMesh(level, ijk, bc, device, order)
        N = getattr(ctx, "N", 8)  # the leaves' edge (8 or 16)
        o, h = W.amr_geometry(level, ijk, N)
        n = len(level)
        self.origin = torch.tensor(o, device=device)
        self.h = torch.tensor(h, device=device)
        Sp = N + 6
        self.bufs = (torch.as_tensor(U, device=device).clone(), torch.zeros((n, 10, Sp, Sp, Sp), dtype=torch.float64,
                                                                            device=device))
        self.dU = torch.empty((n, 10, N, N, N), dtype=torch.float64, device=device)
        self.am = torch.empty(n, dtype=torch.float64, device=device)
        self.dt = torch.empty(1, dtype=torch.float64, device=device)
        self.faces = torch.empty((n, 6, 13, N, N), dtype=torch.float64, device=device)
        # g: optional gravitational acceleration [n][3][N][N][N] at the cell centres
        self.g = torch.as_tensor(g, device=device) if g is not None else None
        self.desc = H.make_rk3_desc(self.bufs[0], self.bufs[1], self.origin, self.h, None, bc, self.dU, self.am,
                                    self.dt, cfl, g=self.g, mesh=self.mesh, face_flux=self.faces)
        self.parity = 0
        self.graph = None
        self.t = 0.0

    @property
    def U(self):
        return self.bufs[self.parity]

    def step(self, use_graph: bool = False):
        """One RK3 step (asynchronous); the state then lives in self.U."""
        if use_graph:
            if self.graph is None:
                assert self.parity == 0, "capture starts from buffer a"
                self.graph = H.hydro_rk3_graph_create(self.ctx, self.desc)
            H.hydro_rk3_graph_launch(self.graph)
        else:
            H.hydro_rk3_step(self.ctx, self.desc, self.parity)
        self.parity ^= 1

    def close(self):
        if self.graph is not None:
            H.hydro_rk3_graph_destroy(self.graph)
            self.graph = None
