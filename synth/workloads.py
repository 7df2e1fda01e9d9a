"""Named workloads (particle count, mesh, box, cosmology, codes, schedule).

pm64   : 64^3 particles, 128^3 mesh, 100 Mpc/h, EdS, P ~ k^-2, x1v2,
         10 steps uniform in a from 0.02 to 0.1.
pm256  : 256^3 particles, 512^3 mesh, 300 Mpc/h, flat LCDM (0.3, h 0.7,
         sigma8 0.8) with BBKS, x1v1, 50 steps from z = 49 to z = 0.
pm128o : the 128^3-particle / 256^3-mesh version of pm256 with the same seed
         (the size the oracle runs for the pm256 comparison).
pm512  : 512^3 particles, 1024^3 mesh, 600 Mpc/h, same LCDM, code widths varied.
All use a coarse cell of 4 fine cells and two fine cells per particle spacing.
"""
import dataclasses
from dataclasses import dataclass

import numpy as np

from .ics import einstein_de_sitter, lcdm_bbks, zeldovich


@dataclass(frozen=True)
class Workload:
    name: str
    n_part_side: int
    n_fine: int
    box: float
    cosmo_kind: str
    x_bytes: int
    v_bytes: int
    a_init: float
    a_final: float
    n_steps: int
    seed: int
    ratio: int = 4
    sigma8: float = 0.8

    @property
    def n_particles(self):
        return self.n_part_side ** 3

    def cosmology(self):
        return einstein_de_sitter(self.sigma8) if self.cosmo_kind == "eds" else lcdm_bbks(sigma8=self.sigma8)

    def omega(self):
        c = self.cosmology()
        return c.omega_m, c.omega_l, c.h


WORKLOADS = {
    "pm64": Workload("pm64", 64, 128, 100.0, "eds", 1, 2, 0.02, 0.1, 10, 1712001),
    "pm256": Workload("pm256", 256, 512, 300.0, "lcdm", 1, 1, 0.02, 1.0, 50, 1712002),
    "pm128o": Workload("pm128o", 128, 256, 300.0, "lcdm", 1, 1, 0.02, 1.0, 50, 1712002),
    "pm512": Workload("pm512", 512, 1024, 600.0, "lcdm", 1, 1, 0.02, 1.0, 50, 1712003),
}


def ensemble_c4(n=64, seed=1712004):
    """An ensemble of uneven realisations: particles per side drawn from
    {32, 48, 64, 96, 128}, mesh twice that, box uniform in [50, 400] Mpc/h,
    sigma8 uniform in [0.7, 0.9], flat LCDM BBKS, x1v1, 30 steps uniform in a
    from z = 49 to z = 0, IC seeds 0 .. n-1."""
    rng = np.random.default_rng(seed)
    sides = rng.choice([32, 48, 64, 96, 128], size=n)
    boxes = rng.uniform(50.0, 400.0, size=n)
    s8 = rng.uniform(0.7, 0.9, size=n)
    return [Workload(f"c4_{i}", int(sides[i]), 2 * int(sides[i]), float(boxes[i]), "lcdm", 1, 1, 0.02, 1.0, 30, i,
                     sigma8=float(s8[i])) for i in range(n)]


@dataclass(frozen=True)
class Request:
    """One simulation request of the serving stream."""
    arrival: float               # seconds after the stream starts
    workload: Workload


def serving_c5(n=40, rate=20.0, seed=1712005):
    """A Poisson-arrival stream of simulation requests (mean `rate` per
    second): particles per side drawn from {64, 96, 128, 192, 256} (mesh
    twice that; 2^a 3^b sides), box 300 Mpc/h x side / 256 (the 256^3
    workload's resolution), sigma8 uniform in [0.7, 0.9], flat LCDM BBKS,
    x1v1, a step count uniform in 10 .. 60 with the 256^3 workload's step
    Delta a = 0.0196 from z = 49 (a_final = min(1, 0.02 + 0.0196 n)), IC
    seed per request."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    sides = rng.choice([64, 96, 128, 192, 256], size=n)
    s8 = rng.uniform(0.7, 0.9, size=n)
    steps = rng.integers(10, 61, size=n)
    out = []
    for i in range(n):
        ns = int(sides[i])
        a_final = min(1.0, 0.02 + 0.0196 * int(steps[i]))
        out.append(Request(float(t[i]), Workload(f"c5_{i}", ns, 2 * ns, 300.0 * ns / 256, "lcdm", 1, 1, 0.02,
                                                 a_final, int(steps[i]), 2000 + i, sigma8=float(s8[i]))))
    return out


def rescaled_ics(ic, factor):
    """The same Zel'dovich realisation with its amplitude (sigma8) times
    `factor`: displacements from the Lagrangian lattice, momenta and the
    velocity scale are linear in the amplitude."""
    nf = ic.n_fine
    ng = round(len(ic.ids) ** (1.0 / 3.0))
    s = nf / ng
    i = ic.ids.astype(np.int64)
    q = np.stack([(i % ng) * s + 0.5, ((i // ng) % ng) * s + 0.5, (i // (ng * ng)) * s + 0.5])
    d = ic.pos.astype(np.float64) - q
    d -= nf * np.round(d / nf)
    pos = np.mod(q + factor * d, float(nf)).astype(np.float32)
    pos[pos >= np.float32(nf)] = 0.0
    vel = (ic.vel.astype(np.float64) * factor).astype(np.float32)
    return dataclasses.replace(ic, pos=pos, vel=vel, sigma_1d=ic.sigma_1d * factor)


def uniform_schedule(a_init, a_final, n_steps):
    """Scale factors a_0 .. a_n, uniform in a."""
    return np.linspace(a_init, a_final, n_steps + 1)


def make_ics(w, n_part_side=None, n_fine=None, seed=None):
    """Zel'dovich ICs for workload `w` (optionally at another resolution)."""
    nps = n_part_side or w.n_part_side
    nf = n_fine or (w.n_fine if n_part_side is None else 2 * nps)
    return zeldovich(nps, nf, w.box, w.cosmology(), w.a_init, seed if seed is not None else w.seed, w.ratio)
