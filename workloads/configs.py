"""The five synthetic workloads (seeded), described by their parameters.

Each ``Workload`` carries the mesh parameters and returns nodal wave speed and
source for caller-supplied 1D node coordinate vectors ``gx`` (NX,) and ``gy``
(NY,) of the structured mesh (node (I, J) sits at (gx[I], gy[J])).  No solver
arithmetic lives here.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import fields


@dataclass
class Workload:
    name: str
    box: tuple
    nx: int
    ny: int
    P: int
    sub_nx: int
    sub_ny: int
    omega: float
    speed_kind: str  # "const", "channel", "random"
    src_center: tuple
    src_width: float
    speed_seed: int = 3
    corr_len: float = 0.05
    extra: dict = field(default_factory=dict)

    @property
    def num_nodes(self):
        return (self.nx * self.P + 1) * (self.ny * self.P + 1)

    @property
    def L(self):
        return (self.nx // self.sub_nx) * (self.ny // self.sub_ny)

    def grid(self, gx, gy):
        return np.meshgrid(np.asarray(gx, float), np.asarray(gy, float))

    def speed(self, gx, gy):
        X, Y = self.grid(gx, gy)
        if self.speed_kind == "const":
            return np.ones_like(X)
        if self.speed_kind == "channel":
            # channel geometry is defined on the unit square; map the box onto it
            x0, x1, y0, y1 = self.box
            return fields.y_channel_speed((X - x0) / (x1 - x0), (Y - y0) / (y1 - y0))
        if self.speed_kind == "random":
            return fields.random_speed(gx, gy, self.corr_len, self.speed_seed)
        raise ValueError(self.speed_kind)

    def source(self, gx, gy):
        X, Y = self.grid(gx, gy)
        return fields.gaussian_source(X, Y, self.src_center, self.src_width).astype(complex)

    # ---- meshes of curved quadrilaterals (extra["warp"] = amplitude > 0)
    @property
    def warp(self):
        return float(self.extra.get("warp", 0.0))

    def node_xy(self, gx, gy):
        """Physical node positions (NY, NX): the Cartesian grid, warped when
        the workload is a curved-quadrilateral mesh."""
        X, Y = self.grid(gx, gy)
        if self.warp > 0.0:
            X, Y = fields.warp_nodes(X, Y, self.box, self.warp)
        return X, Y

    def speed_at(self, X, Y):
        """Wave speed at arbitrary node positions (const and channel kinds)."""
        if self.speed_kind == "const":
            return np.ones_like(X)
        if self.speed_kind == "channel":
            x0, x1, y0, y1 = self.box
            return fields.y_channel_speed((X - x0) / (x1 - x0), (Y - y0) / (y1 - y0))
        raise ValueError(f"speed kind {self.speed_kind!r} is defined on the Cartesian grid only")

    def source_at(self, X, Y):
        return fields.gaussian_source(X, Y, self.src_center, self.src_width).astype(complex)

    def boundary(self):
        """Outer boundary data g: zero (first-order absorbing boundary)."""
        NX, NY = self.nx * self.P + 1, self.ny * self.P + 1
        return {"S": np.zeros(NX, complex), "E": np.zeros(NY, complex),
                "N": np.zeros(NX, complex), "W": np.zeros(NY, complex)}

    def dof_per_sweep(self, nt, m_wh):
        """Subdomain node updates of one sweep: L * n_l * (N_t - 1) * m_wh."""
        nl = (self.sub_nx * self.P + 1) * (self.sub_ny * self.P + 1)
        return self.L * nl * (nt - 1) * m_wh


def config1():
    """32x32 quads, P=2 (4225 nodes), 4x4 subdomains of 8x8, c=1, w=10,
    Gaussian source (width 0.02) at (0.3, 0.6), g=0, FP64."""
    return Workload("cfg1_32x32_p2_sub8", (0.0, 1.0, 0.0, 1.0), 32, 32, 2, 8, 8, 10.0, "const", (0.3, 0.6), 0.02)


def config2():
    """256x256 quads, P=3, 32x32 subdomains of 8x8 (625 nodes each), Y channel
    of width 0.08 at c=1/3 in c=1; w = 64 pi gives 8 node spacings per slow
    wavelength (node spacing 1/768); off-centre source in the stem.  The
    source width (0.003) resolves the slow wavelength (0.0104)."""
    return Workload("cfg2_256x256_p3_sub8_ychannel", (0.0, 1.0, 0.0, 1.0), 256, 256, 3, 8, 8, 64.0 * math.pi,
                    "channel", (0.52, 0.22), 0.003)


def config3():
    """1024x1024 quads on [-1,1]^2, P=4, 32x32 subdomains of 32x32 elements
    (16641 nodes each), c = 1 + 0.5 g (g: Gaussian random field, correlation
    length 0.05, clipped to [-1.5,1.5]), w for 10 node spacings per wavelength
    at c=1 (spacing 1/2048): w = 2 pi 204.8."""
    return Workload("cfg3_1024x1024_p4_sub32_random", (-1.0, 1.0, -1.0, 1.0), 1024, 1024, 4, 32, 32,
                    2.0 * math.pi * 204.8, "random", (0.3, -0.2), 0.001)


def config4(n_problems=64, seed0=4):
    """Batch of independent problems: meshes 64^2..512^2, P 2..5, subdomains
    4^2..32^2 elements (s <= n/4), w log-uniform in [5, 80], random-field or
    channel speed (50/50), source uniform in [0.2, 0.8]^2."""
    out = []
    for i in range(n_problems):
        rng = np.random.default_rng(seed0 + i)
        n = int(rng.choice([64, 128, 256, 512]))
        P = int(rng.choice([2, 3, 4, 5]))
        s = int(rng.choice([s for s in (4, 8, 16, 32) if s <= n // 4]))
        w = float(math.exp(rng.uniform(math.log(5.0), math.log(80.0))))
        kind = "random" if rng.uniform() < 0.5 else "channel"
        ctr = tuple(rng.uniform(0.2, 0.8, 2))
        cmin = 0.25 if kind == "random" else 1.0 / 3.0
        width = min(0.02, 0.25 * 2.0 * math.pi * cmin / w)
        out.append(Workload(f"cfg4_{i:02d}_n{n}_p{P}_s{s}", (0.0, 1.0, 0.0, 1.0), n, n, P, s, s, w, kind,
                            ctr, width, speed_seed=1000 + i))
    return out


def config5_arrivals(n_requests=2000, rate=200.0, seed=5, group_prob=0.2, group_size=8):
    """Poisson arrival stream: (arrival_time_s, workload, n_sources) tuples
    drawn from the config-4 sampler; with probability group_prob a request is
    a group of group_size sources sharing mesh, speed and frequency."""
    rng = np.random.default_rng(seed)
    pool = config4(64, seed0=500)
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += rng.exponential(1.0 / rate)
        wl = pool[int(rng.integers(len(pool)))]
        k = group_size if rng.uniform() < group_prob else 1
        out.append((t, wl, k))
    return out


def config2m(amp=0.03):
    """config2 on curved quadrilaterals: the same element grid with its
    interior nodes moved by fields.warp_nodes (amplitude 3% of the box), so
    every element is a different curved quad; boundary nodes stay on the
    square.  Exercises the element-form (metric) stiffness of Sec. 4."""
    w = config2()
    return Workload("cfg2m_256x256_p3_sub8_ychannel_warp3", w.box, w.nx, w.ny, w.P, w.sub_nx, w.sub_ny, w.omega,
                    w.speed_kind, w.src_center, w.src_width, w.speed_seed, w.corr_len, extra={"warp": amp})


def mapped(w: Workload, amp: float, name=None):
    """The same workload on a warped (curved-quadrilateral) node grid."""
    extra = dict(w.extra)
    extra["warp"] = amp
    return Workload(name or f"{w.name}_warp", w.box, w.nx, w.ny, w.P, w.sub_nx, w.sub_ny, w.omega, w.speed_kind,
                    w.src_center, w.src_width, w.speed_seed, w.corr_len, extra=extra)


def scaled(w: Workload, nx: int, ny: int, sub_nx: Optional[int] = None, sub_ny: Optional[int] = None, name=None):
    """Same physics on a smaller mesh (parity cases the oracle finishes
    quickly); omega and fields are unchanged."""
    return Workload(name or f"{w.name}_scaled{nx}x{ny}", w.box, nx, ny, w.P, sub_nx or w.sub_nx, sub_ny or w.sub_ny,
                    w.omega, w.speed_kind, w.src_center, w.src_width, w.speed_seed, w.corr_len, extra=dict(w.extra))
