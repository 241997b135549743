"""Seeded synthetic agent populations and dynamics (the simulation harness).

This module produces the agent states that both the CUDA path and the oracle
consume.  It holds none of the exchange method's arithmetic (no classification,
serialization or codec); it only plays the part of the agent operations that
run between two aura updates: spherical cells that move, grow, divide and die.

The paper's benchmark simulations (cell clustering, cell proliferation,
epidemiology, oncology; Sec. 3.1) and their parameters are not available, so
the workloads below are synthetic stand-ins with the same kind of agent record
(id, position, diameter, volume, adherence, density).

A state is a dict of 1-D tensors of equal length on one device:
  id (int64, non-negative, read as uint64 by the library), x, y, z, diameter,
  volume, adherence, density (float64), and for drifting workloads vx, vy, vz.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

FIELDS = ("id", "x", "y", "z", "diameter", "volume", "adherence", "density")


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n0: int
    lo: tuple
    hi: tuple
    grid: tuple
    w: float
    iterations: int
    layout: str = "uniform"        # "uniform" or "blobs"
    p_move: float = 0.3
    step_sigma: float = 0.5
    p_grow: float = 0.0
    grow_factor: float = 1.01
    p_divide: float = 0.0
    p_die: float = 0.0
    persistent: bool = False       # velocity = 0.8 v + 0.2 N(0, sigma) + drift
    n_blobs: int = 32
    seed: int = 0
    boundary: str = "closed"       # "closed" (clamp) or "toroidal" (wrap)
    wrap_axes: int = 7             # axis bit mask that wraps when toroidal

    @property
    def n_boxes(self) -> int:
        return self.grid[0] * self.grid[1] * self.grid[2]

    @property
    def n_pairs(self) -> int:
        return self.n_boxes * 27

    @property
    def periodic(self) -> int:
        """Axis bit mask of toroidal axes, as the library's grid takes it."""
        return self.wrap_axes if self.boundary == "toroidal" else 0


def _cube(side):
    return (0.0, 0.0, 0.0), (float(side),) * 3


WORKLOADS = {
    # 4,096 agents in a 100^3 cube, 2x2x1 boxes, aura 30, 10 iterations, moves only.
    "uniform_4k": Workload("uniform_4k", 4096, *_cube(100), (2, 2, 1), 30.0, 10,
                           seed=0x7E7A0001),
    # 1M agents in a 1000^3 cube, 4x4x4 boxes, 50 iterations, move/grow/divide/die.
    "uniform_1m": Workload("uniform_1m", 1 << 20, *_cube(1000), (4, 4, 4), 30.0, 50,
                           p_grow=0.1, p_divide=0.005, p_die=0.002, seed=0x7E7A0002),
    # 16M agents from 32 Gaussian blobs in a 4000^3 cube (box sizes differ ~10x).
    "blobs_16m": Workload("blobs_16m", 16 << 20, *_cube(4000), (4, 4, 4), 30.0, 50,
                          layout="blobs", p_grow=0.1, p_divide=0.005, p_die=0.002,
                          seed=0x7E7A0003),
    # 100M agents in an 8000^3 cube, 8x8x8 boxes, 20 iterations, 1% divide, 1% die.
    "uniform_100m": Workload("uniform_100m", 100_000_000, *_cube(8000), (8, 8, 8), 30.0, 20,
                             p_grow=0.1, p_divide=0.01, p_die=0.01, seed=0x7E7A0004),
    # 16M blob agents with persistent motion in a smooth drift field.
    "drift_16m": Workload("drift_16m", 16 << 20, *_cube(4000), (4, 4, 4), 30.0, 220,
                          layout="blobs", p_move=1.0, persistent=True, seed=0x7E7A0005),
    # the 1M workload on a toroidal domain (every axis wraps)
    "torus_1m": Workload("torus_1m", 1 << 20, *_cube(1000), (4, 4, 4), 30.0, 50,
                         p_grow=0.1, p_divide=0.005, p_die=0.002, boundary="toroidal",
                         seed=0x7E7A0006),
}


def scaled(wl: Workload, n0: int, iterations: int | None = None, **kw) -> Workload:
    """The same workload with fewer agents (box count and cube unchanged)."""
    return dataclasses.replace(wl, n0=n0, iterations=iterations or wl.iterations, **kw)


def _clamp(v: torch.Tensor, lo: float, hi: float) -> torch.Tensor:
    # closed boundary: keep positions inside [lo, nextafter(hi, lo)]
    top = torch.nextafter(torch.tensor(hi, dtype=torch.float64),
                          torch.tensor(lo, dtype=torch.float64)).item()
    return v.clamp_(lo, top)


def _wrap(v: torch.Tensor, lo: float, hi: float) -> torch.Tensor:
    # toroidal boundary: lo + (v - lo) mod (hi - lo); a remainder that rounds
    # up to the full period is kept just below hi
    v = lo + torch.remainder(v - lo, hi - lo)
    return _clamp(v, lo, hi)


class Generator:
    """Seeded population + dynamics.  Deterministic for a (workload, device)."""

    def __init__(self, wl: Workload, device="cpu", seed: int | None = None):
        self.wl = wl
        self.device = torch.device(device)
        self.seed = wl.seed if seed is None else seed
        self.g = torch.Generator(device=self.device)
        self.g.manual_seed(self.seed)
        self.next_id = wl.n0
        per = wl.periodic
        self._bounds = [(_wrap if per >> a & 1 else _clamp) for a in range(3)]

    # -- random helpers on the workload's device --
    def _rand(self, n):
        return torch.rand(n, generator=self.g, device=self.device, dtype=torch.float64)

    def _randn(self, n):
        return torch.randn(n, generator=self.g, device=self.device, dtype=torch.float64)

    def initial(self) -> dict:
        wl, n = self.wl, self.wl.n0
        pos = []
        if wl.layout == "uniform":
            for a in range(3):
                pos.append(wl.lo[a] + (wl.hi[a] - wl.lo[a]) * self._rand(n))
        else:
            rng = np.random.default_rng(self.seed)
            sig = rng.uniform(20.0, 200.0, wl.n_blobs)
            wts = rng.dirichlet(np.full(wl.n_blobs, 0.5))
            ctr = rng.uniform(np.array(wl.lo), np.array(wl.hi), (wl.n_blobs, 3))
            blob = torch.multinomial(torch.tensor(wts, dtype=torch.float64, device=self.device),
                                     n, replacement=True, generator=self.g)
            sig_t = torch.tensor(sig, dtype=torch.float64, device=self.device)[blob]
            ctr_t = torch.tensor(ctr, dtype=torch.float64, device=self.device)[blob]
            for a in range(3):
                pos.append(ctr_t[:, a] + sig_t * self._randn(n))
        for a in range(3):
            pos[a] = self._bounds[a](pos[a], wl.lo[a], wl.hi[a])
        d = 8.0 + 4.0 * self._rand(n)
        st = dict(id=torch.arange(n, dtype=torch.int64, device=self.device),
                  x=pos[0], y=pos[1], z=pos[2], diameter=d,
                  volume=(math.pi / 6.0) * d * d * d,
                  adherence=0.3 + 0.4 * self._rand(n),
                  density=torch.ones(n, dtype=torch.float64, device=self.device))
        if wl.persistent:
            for k in ("vx", "vy", "vz"):
                st[k] = torch.zeros(n, dtype=torch.float64, device=self.device)
        return st

    def step(self, st: dict) -> dict:
        """One iteration of agent operations: move, grow, divide, die."""
        wl = self.wl
        st = {k: v.clone() for k, v in st.items()}
        n = st["x"].shape[0]
        axes = ("x", "y", "z")
        if wl.persistent:
            drift = (torch.sin(st["y"] / 500.0), torch.cos(st["z"] / 500.0),
                     torch.sin(st["x"] / 500.0))
            for a, k in enumerate(axes):
                vk = "v" + k
                st[vk] = 0.8 * st[vk] + 0.2 * wl.step_sigma * self._randn(n) + 0.5 * drift[a]
                st[k] = self._bounds[a](st[k] + st[vk], wl.lo[a], wl.hi[a])
        elif wl.p_move > 0:
            mv = self._rand(n) < wl.p_move
            for a, k in enumerate(axes):
                step = wl.step_sigma * self._randn(n)
                st[k] = self._bounds[a](torch.where(mv, st[k] + step, st[k]),
                                          wl.lo[a], wl.hi[a])
        if wl.p_grow > 0:
            gr = self._rand(n) < wl.p_grow
            d = torch.where(gr, st["diameter"] * wl.grow_factor, st["diameter"])
            st["diameter"] = d
            st["volume"] = torch.where(gr, (math.pi / 6.0) * d * d * d, st["volume"])
        if wl.p_divide > 0:
            dv = torch.nonzero(self._rand(n) < wl.p_divide).flatten()
            k = dv.numel()
            if k:
                d_old = st["diameter"][dv]
                d = d_old * 2.0 ** (-1.0 / 3.0)
                u = torch.stack([self._randn(k) for _ in range(3)], 1)
                u = u / u.norm(dim=1, keepdim=True).clamp_min(1e-300)
                child = {f: st[f][dv].clone() for f in st}
                for a, ax in enumerate(axes):
                    child[ax] = self._bounds[a](st[ax][dv] + 0.5 * d_old * u[:, a],
                                                  wl.lo[a], wl.hi[a])
                st["diameter"][dv] = d
                st["volume"][dv] = (math.pi / 6.0) * d * d * d
                child["diameter"] = d.clone()
                child["volume"] = (math.pi / 6.0) * d * d * d
                child["id"] = torch.arange(self.next_id, self.next_id + k, dtype=torch.int64,
                                           device=self.device)
                self.next_id += k
                st = {f: torch.cat([st[f], child[f]]) for f in st}
        if wl.p_die > 0:
            n = st["x"].shape[0]
            keep = self._rand(n) >= wl.p_die
            st = {f: v[keep] for f, v in st.items()}
        return st

    def series(self, iterations: int | None = None):
        """Yield the states of iterations 0, 1, ... (iteration 0 is the initial state)."""
        st = self.initial()
        yield st
        for _ in range((iterations or self.wl.iterations) - 1):
            st = self.step(st)
            yield st


def to_numpy(st: dict) -> dict:
    out = {}
    for k, v in st.items():
        a = v.detach().cpu().numpy()
        out[k] = a.view(np.uint64) if k == "id" else a
    return out
