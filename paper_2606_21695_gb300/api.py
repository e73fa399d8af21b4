"""Convenience constructors over the C ABI (marshalling only).

``make_problem`` builds a mesh and problem for a synthetic workload: node
coordinates come from the library (``hz_mesh_node_coords``), the wave speed
and source are evaluated there by the seeded generators in ``workloads``.
"""

from __future__ import annotations

import numpy as np

from . import _binding as B


class Case:
    """A mesh + problem pair with its host-side inputs (owns both handles)."""

    def __init__(self, wl, device=0, fields=True):
        self.wl = wl
        self.mesh = B.hz_mesh_create(*wl.box, wl.nx, wl.ny, wl.P, wl.sub_nx, wl.sub_ny)
        self.n = B.hz_mesh_num_nodes(self.mesh)
        xy = B.hz_mesh_node_coords(self.mesh)
        NX, NY = wl.nx * wl.P + 1, wl.ny * wl.P + 1
        self.gx = xy[:NX, 0].copy()
        self.gy = xy[::NX, 1].copy()
        self.pr = B.hz_problem_create(self.mesh, device)
        self.c = self.f = self.g = None
        self.X = self.Y = None
        if getattr(wl, "warp", 0.0) > 0.0:  # curved quadrilaterals: node positions from the workload
            self.X, self.Y = wl.node_xy(self.gx, self.gy)
            B.hz_problem_set(self.pr, B.HZ_NODE_COORDS, np.stack([self.X.ravel(), self.Y.ravel()], axis=1).ravel())
        if fields:
            if self.X is not None:
                self.c = wl.speed_at(self.X, self.Y)
                self.f = wl.source_at(self.X, self.Y)
            else:
                self.c = wl.speed(self.gx, self.gy)
                self.f = wl.source(self.gx, self.gy)
            self.g = wl.boundary()
            B.hz_problem_set(self.pr, B.HZ_WAVE_SPEED, self.c.ravel())
            B.hz_problem_set(self.pr, B.HZ_OMEGA, np.array([wl.omega]))
            B.hz_problem_set(self.pr, B.HZ_SOURCE, self.f.ravel())
            B.hz_problem_set(self.pr, B.HZ_BOUNDARY, boundary_vector(self.g))

    def close(self):
        if self.pr is not None:
            B.hz_problem_destroy(self.pr)
            self.pr = None
        if self.mesh is not None:
            B.hz_mesh_destroy(self.mesh)
            self.mesh = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def boundary_vector(g):
    """Concatenate per-edge boundary data in the C ABI order S, E, N, W."""
    return np.concatenate([np.asarray(g[k], complex).ravel() for k in ("S", "E", "N", "W")])
