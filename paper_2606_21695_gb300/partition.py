"""Distribution of subdomains over ranks (one GPU each) and the exchange of
transmission data across cut interfaces.

The DD sweep partitions naturally (Sec. 8 of the paper: only interface data
crosses between GPUs).  Ranks own rectangular blocks of the S_x x S_y
subdomain grid.  In one sweep every rank solves its own subdomains; the
lambda values a subdomain writes for a neighbour owned by another rank are
packed, sent point-to-point, and unpacked into that rank's lambda vector.
The outer Krylov iteration needs one all-reduce of its dot products per
Arnoldi step.

This module is host-side index logic only (plans and packing of lambda
vectors in the layout of include/hz.h: [L][4 edges W,E,S,N][NE] complex).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

W, E, S, N = 0, 1, 2, 3
OPP = (E, W, N, S)


def process_grid(R, Sx, Sy):
    """px x py = R ranks, chosen to make blocks as square as possible."""
    best = None
    for px in range(1, R + 1):
        if R % px:
            continue
        py = R // px
        if px > Sx or py > Sy:
            continue
        cost = abs(Sx / px - Sy / py)
        if best is None or cost < best[0]:
            best = (cost, px, py)
    if best is None:
        raise ValueError("more ranks than subdomains")
    return best[1], best[2]


def _splits(n, k):
    base, rem = divmod(n, k)
    edges = [0]
    for i in range(k):
        edges.append(edges[-1] + base + (1 if i < rem else 0))
    return edges


@dataclass
class Partition:
    Sx: int
    Sy: int
    R: int

    def __post_init__(self):
        self.px, self.py = process_grid(self.R, self.Sx, self.Sy)
        self.xe = _splits(self.Sx, self.px)
        self.ye = _splits(self.Sy, self.py)
        self.owner = np.empty(self.Sx * self.Sy, dtype=int)
        for l in range(self.Sx * self.Sy):
            sx, sy = l % self.Sx, l // self.Sx
            bx = max(i for i in range(self.px) if self.xe[i] <= sx)
            by = max(i for i in range(self.py) if self.ye[i] <= sy)
            self.owner[l] = by * self.px + bx

    def subdomains(self, rank):
        return np.nonzero(self.owner == rank)[0]

    def neighbour(self, l, e):
        sx, sy = l % self.Sx, l // self.Sx
        if e == W:
            return l - 1 if sx > 0 else -1
        if e == E:
            return l + 1 if sx < self.Sx - 1 else -1
        if e == S:
            return l - self.Sx if sy > 0 else -1
        return l + self.Sx if sy < self.Sy - 1 else -1

    def send_plan(self, rank):
        """{dest rank: [(l, e)]}: edge e of own subdomain l faces a subdomain of
        dest; the sweep writes lambda slot (neighbour, OPP[e]) for it."""
        plan = {}
        for l in self.subdomains(rank):
            for e in range(4):
                r = self.neighbour(l, e)
                if r >= 0 and self.owner[r] != rank:
                    plan.setdefault(int(self.owner[r]), []).append((int(r), OPP[e]))
        return plan

    def recv_plan(self, rank):
        """{source rank: [(l, e)]}: slots of own subdomains written by source."""
        plan = {}
        for l in self.subdomains(rank):
            for e in range(4):
                r = self.neighbour(l, e)
                if r >= 0 and self.owner[r] != rank:
                    plan.setdefault(int(self.owner[r]), []).append((int(l), e))
        # order both sides identically: by the writer's (neighbour, edge) enumeration
        for src, items in plan.items():
            order = {s: k for k, s in enumerate(self.send_plan(src)[rank])}
            plan[src] = sorted(items, key=lambda s: order[s])
        return plan


def pack(lam, slots):
    """lam: (L, 4, NE) complex -> contiguous buffer of the listed slots."""
    return np.ascontiguousarray(np.stack([lam[l, e] for l, e in slots]))


def unpack(lam, slots, buf):
    for k, (l, e) in enumerate(slots):
        lam[l, e] = buf[k]
