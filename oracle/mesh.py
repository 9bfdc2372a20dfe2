"""Cartesian spectral-element mesh, global numbering and the packed skeleton.

Global nodes form the grid (mx p + 1) x (my p + 1) x (mz p + 1), numbered
gx + Nx (gy + Ny gz).  Element (ex, ey, ez) owns local node (a, b, c) at global
(ex p + a, ey p + b, ez p + c); R_e^T of Sec. 3 is this index map.  Nodes on the
domain boundary carry homogeneous Dirichlet values and are excluded from the
unknowns.

The skeleton (element-boundary nodes) is packed entity by entity, in the order
declared in include/sem.h:

  x-faces (f, ey, ez)   (mx+1) my mz   local (j, k), j fastest, n^2 values
  y-faces (ex, f, ez)   mx (my+1) mz   local (i, k), i fastest
  z-faces (ex, ey, f)   mx my (mz+1)   local (i, j), i fastest
  x-edges (ex, vy, vz)  mx (my+1)(mz+1)  local i, n values
  y-edges (vx, ey, vz)  (mx+1) my (mz+1) local j
  z-edges (vx, vy, ez)  (mx+1)(my+1) mz  local k
  vertices (vx, vy, vz) (mx+1)(my+1)(mz+1)

with n = p - 1, local indices 1..n, and the first entity index fastest within
each block.  This module writes that layout out independently of the library.

Test infrastructure only.
"""
from __future__ import annotations

from dataclasses import dataclass
from functools import cached_property

import numpy as np

from .gll import gll


@dataclass(eq=False)
class Mesh:
    p: int
    hx: np.ndarray
    hy: np.ndarray
    hz: np.ndarray

    def __post_init__(self):
        self.hx = np.asarray(self.hx, float)
        self.hy = np.asarray(self.hy, float)
        self.hz = np.asarray(self.hz, float)
        self.mx, self.my, self.mz = len(self.hx), len(self.hy), len(self.hz)
        self.n = self.p - 1
        self.Nx = self.mx * self.p + 1
        self.Ny = self.my * self.p + 1
        self.Nz = self.mz * self.p + 1

    @property
    def n_elements(self):
        return self.mx * self.my * self.mz

    @property
    def n_global(self):
        return self.Nx * self.Ny * self.Nz

    def gid(self, gx, gy, gz):
        return np.asarray(gx) + self.Nx * (np.asarray(gy) + self.Ny * np.asarray(gz))

    # ----- coordinates -------------------------------------------------------
    def axis_coords(self, h):
        """Global node coordinates along one axis (element offsets + mapped GLL)."""
        xi, _ = gll(self.p)
        X0 = np.concatenate(([0.0], np.cumsum(h)[:-1]))
        pts = np.empty(len(h) * self.p + 1)
        for e, (x0, he) in enumerate(zip(X0, h)):
            pts[e * self.p: e * self.p + self.p + 1] = x0 + 0.5 * he * (xi + 1.0)
        pts[-1] = float(np.sum(h))
        return pts

    def coords(self):
        """(X, Y, Z) arrays of shape (Nz, Ny, Nx)."""
        x = self.axis_coords(self.hx)
        y = self.axis_coords(self.hy)
        z = self.axis_coords(self.hz)
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        return X, Y, Z

    # ----- element maps ------------------------------------------------------
    def elements(self):
        """Iterate (e, ex, ey, ez) with e = ex + mx (ey + my ez)."""
        e = 0
        for ez in range(self.mz):
            for ey in range(self.my):
                for ex in range(self.mx):
                    yield e, ex, ey, ez
                    e += 1

    def widths(self, ex, ey, ez):
        return (self.hx[ex], self.hy[ey], self.hz[ez])

    @cached_property
    def elem_widths(self):
        """(n_e, 3) widths in element order."""
        out = np.empty((self.n_elements, 3))
        for e, ex, ey, ez in self.elements():
            out[e] = self.widths(ex, ey, ez)
        return out

    @cached_property
    def local_to_global(self):
        """(n_e, (p+1)^3) global node index of each element's local node."""
        q = self.p + 1
        c, b, a = np.meshgrid(np.arange(q), np.arange(q), np.arange(q), indexing="ij")
        a, b, c = a.ravel(), b.ravel(), c.ravel()
        out = np.empty((self.n_elements, q ** 3), dtype=np.int64)
        for e, ex, ey, ez in self.elements():
            out[e] = self.gid(ex * self.p + a, ey * self.p + b, ez * self.p + c)
        return out

    @cached_property
    def free_mask(self):
        """True at global nodes that are not on the domain boundary."""
        gz, gy, gx = np.meshgrid(np.arange(self.Nz), np.arange(self.Ny),
                                 np.arange(self.Nx), indexing="ij")
        m = ((gx > 0) & (gx < self.Nx - 1) & (gy > 0) & (gy < self.Ny - 1)
             & (gz > 0) & (gz < self.Nz - 1))
        return m.ravel()

    @cached_property
    def skeleton_mask(self):
        """True at global nodes on some element boundary."""
        gz, gy, gx = np.meshgrid(np.arange(self.Nz), np.arange(self.Ny),
                                 np.arange(self.Nx), indexing="ij")
        p = self.p
        return ((gx % p == 0) | (gy % p == 0) | (gz % p == 0)).ravel()

    # ----- packed skeleton ---------------------------------------------------
    @cached_property
    def block_counts(self):
        mx, my, mz = self.mx, self.my, self.mz
        return dict(
            xface=(mx + 1) * my * mz, yface=mx * (my + 1) * mz, zface=mx * my * (mz + 1),
            xedge=mx * (my + 1) * (mz + 1), yedge=(mx + 1) * my * (mz + 1),
            zedge=(mx + 1) * (my + 1) * mz, vertex=(mx + 1) * (my + 1) * (mz + 1))

    @cached_property
    def n_skeleton(self):
        c = self.block_counts
        n = self.n
        return (n * n * (c["xface"] + c["yface"] + c["zface"])
                + n * (c["xedge"] + c["yedge"] + c["zedge"]) + c["vertex"])

    @cached_property
    def pack_map(self):
        """Global node index of every packed skeleton entry (length N_B)."""
        p, n = self.p, self.n
        mx, my, mz = self.mx, self.my, self.mz
        out = []
        loc = np.arange(1, n + 1)
        # x-faces: entity (f, ey, ez), values (j, k) with j fastest
        K2, J2 = np.meshgrid(loc, loc, indexing="ij")
        J2, K2 = J2.ravel(), K2.ravel()
        for ez in range(mz):
            for ey in range(my):
                for f in range(mx + 1):
                    out.append(self.gid(f * p + 0 * J2, ey * p + J2, ez * p + K2))
        # y-faces: entity (ex, f, ez), values (i, k) with i fastest
        I2, K2b = J2, K2
        for ez in range(mz):
            for f in range(my + 1):
                for ex in range(mx):
                    out.append(self.gid(ex * p + I2, f * p + 0 * I2, ez * p + K2b))
        # z-faces: entity (ex, ey, f), values (i, j) with i fastest
        for f in range(mz + 1):
            for ey in range(my):
                for ex in range(mx):
                    out.append(self.gid(ex * p + I2, ey * p + K2b, f * p + 0 * I2))
        # x-edges (ex, vy, vz)
        for vz in range(mz + 1):
            for vy in range(my + 1):
                for ex in range(mx):
                    out.append(self.gid(ex * p + loc, vy * p + 0 * loc, vz * p + 0 * loc))
        # y-edges (vx, ey, vz)
        for vz in range(mz + 1):
            for ey in range(my):
                for vx in range(mx + 1):
                    out.append(self.gid(vx * p + 0 * loc, ey * p + loc, vz * p + 0 * loc))
        # z-edges (vx, vy, ez)
        for ez in range(mz):
            for vy in range(my + 1):
                for vx in range(mx + 1):
                    out.append(self.gid(vx * p + 0 * loc, vy * p + 0 * loc, ez * p + loc))
        # vertices
        for vz in range(mz + 1):
            for vy in range(my + 1):
                for vx in range(mx + 1):
                    out.append(np.array([self.gid(vx * p, vy * p, vz * p)]))
        pm = np.concatenate(out).astype(np.int64)
        assert len(pm) == self.n_skeleton
        return pm

    @cached_property
    def skeleton_free(self):
        """True at packed skeleton entries that are unknowns (not Dirichlet)."""
        return self.free_mask[self.pack_map]

    def pack(self, u_full):
        return np.asarray(u_full).ravel()[self.pack_map]

    def unpack(self, uB):
        out = np.zeros(self.n_global)
        out[self.pack_map] = uB
        return out

    @cached_property
    def skeleton_slot(self):
        """Packed index of each global skeleton node (-1 elsewhere)."""
        s = -np.ones(self.n_global, dtype=np.int64)
        s[self.pack_map] = np.arange(self.n_skeleton)
        return s

    def entity_blocks(self):
        """List of index arrays into the packed vector, one per entity
        (face, edge or vertex), in packed order."""
        n = self.n
        c = self.block_counts
        blocks = []
        off = 0
        for kind, size in (("xface", n * n), ("yface", n * n), ("zface", n * n),
                           ("xedge", n), ("yedge", n), ("zedge", n), ("vertex", 1)):
            for _ in range(c[kind]):
                blocks.append((kind, np.arange(off, off + size)))
                off += size
        return blocks
