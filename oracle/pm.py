"""The compressed particle store and one PM step, FP64 (Sections 2.1-2.3).

Store = {rho_c (counts), v_c, chi_d, nu_d, I_P} plus the codec scale sigma
(Section 2.3.1's checkpoint, with sigma added because decoding needs it).

One step, KD order (reading of the (DKKD)^n splitting of Section 2.3.3:
positions live at a_n, momenta at a_{n-1/2}; the first step kicks half a
step from the momenta's epoch):
  1. decode positions (Eq. x) and velocities (Eq. v);
  2. CIC density -> Poisson -> FD4 force -> CIC gather (mesh.py);
  3. kick v += F * int da/(a^2 E) over [a_{n-1/2}, a_{n+1/2}] and store the
     kicked velocity as a code relative to the same v_c (Fig. update_vp);
  4. measure sigma^2 = <(v - v_c)^2> from the kicked velocities and scale it
     by the momentum growth ratio g(a_{n+1}) / g(a_n) for the next store
     (Section 2.2, last paragraph), snapped to 1/16 octave;
  5. drift x += v * int da/(a^3 E) over [a_n, a_{n+1}] inside the old cell
     (Fig. update_xp);
  6. rebuild the cell-ordered store from the drifted particles: counts, new
     v_c, chi (Eq. chi) and nu relative to the new v_c (Eq. nu), ordered by
     new cell and, within a cell, by old storage index (encode_drifted).

The codes are integers decided by floating point; the oracle takes those
decisions on the same FP32 values the CUDA path stores (the kicked momentum,
the drifted offset inside the cell, v - v_c), and does the rest in FP64.
"""
from dataclasses import dataclass, field, replace

import numpy as np

from . import codec, cosmo, layout, mesh

VEL_FIX = 2.0 ** 24          # fixed-point quantum of the v_c averages


@dataclass(frozen=True)
class Params:
    n_fine: int
    n_particles: int
    ratio: int = 4
    x_bytes: int = 1
    v_bytes: int = 1
    box: float = 100.0
    omega_m: float = 1.0
    omega_l: float = 0.0
    deconv_power: int = 2
    brick: int = 0

    @property
    def n_coarse(self):
        return self.n_fine // self.ratio

    @property
    def brick_side(self):
        return self.brick or layout.auto_brick(self.n_coarse)

    @property
    def mass(self):
        """Particle mass in units of the mean density per fine cell."""
        return self.n_fine ** 3 / self.n_particles


@dataclass
class Store:
    params: Params
    counts: np.ndarray            # int64 [N_c^3], storage order
    vc: np.ndarray                # float32 [3][N_c^3], storage order
    chi: np.ndarray               # int64 [3][N]
    nu: np.ndarray                # int64 [3][N]
    ids: np.ndarray               # uint32 [N]
    sigma: float                  # per-dimension codec scale
    a: float                      # epoch of the positions
    a_p: float                    # epoch of the momenta
    extra: dict = field(default_factory=dict)

    def cells(self):
        """(cx, cy, cz) of every stored particle, from the counts."""
        P = self.params
        return layout.cell_coords(layout.particle_cells(self.counts), P.n_coarse, P.brick_side)


def f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def fma_f32(a, b, c):
    """fl32(a * b + c) with a single rounding, for FP32 a, b, c: the drifted
    offset u + p * dc of Fig. update_xp as an FP32 value (reading: the
    position code is decided on that FP32 value, rounded once).

    a * b is exact in FP64 (two 24-bit significands).  The sum with c is
    s + e exactly, s = fl64(a b + c) and e its rounding error (Knuth's
    TwoSum); s is then rounded to odd (moved one FP64 ulp toward e when e is
    non-zero and s is even), after which rounding to FP32 gives the correctly
    rounded value: rounding to odd at 53 bits followed by rounding to nearest
    at 24 <= 53 - 2 bits is a single rounding (Boldo & Melquiond, 2008).
    A plain FP64 add followed by an FP32 conversion rounds twice and can
    land one FP32 ulp away on a tie.
    """
    a = np.asarray(a, np.float32).astype(np.float64)
    b = np.asarray(b, np.float32).astype(np.float64)
    c = np.asarray(c, np.float32).astype(np.float64)
    prod = a * b
    s = prod + c
    bv = s - prod
    e = (prod - (s - bv)) + (c - bv)
    even = (np.asarray(s).view(np.int64) & 1) == 0
    odd = np.where((e != 0) & even, np.nextafter(s, np.where(e > 0, np.inf, -np.inf)), s)
    return np.asarray(odd, np.float64).astype(np.float32)


def cell_mean_velocity(key, vel32, n_cells):
    """v_c of each cell: mean of its particles' FP32 velocities (Eq. deltav).

    Reading: the mean is taken in fixed point -- each velocity rounded to a
    multiple of 2^-24 (half to even), summed exactly, divided by the count in
    FP64 and rounded to FP32 -- so any summation order gives the same value.
    Empty cells get 0.
    """
    key = np.asarray(key, dtype=np.int64)
    cnt = np.bincount(key, minlength=n_cells)
    out = np.zeros((3, n_cells), dtype=np.float32)
    for d in range(3):
        q = np.rint(np.asarray(vel32[d], dtype=np.float32).astype(np.float64) * VEL_FIX).astype(np.int64)
        s = np.zeros(n_cells, dtype=np.int64)
        np.add.at(s, key, q)
        with np.errstate(invalid="ignore", divide="ignore"):
            m = (s.astype(np.float64) / cnt) * (1.0 / VEL_FIX)
        out[d] = np.where(cnt > 0, m, 0.0).astype(np.float32)
    return out


def _build(P, cell3, chi3, vel32, ids, sigma, a, a_p):
    """Common tail of encode / encode_drifted: order, counts, v_c, nu."""
    nc, b = P.n_coarse, P.brick_side
    key = layout.storage_index(cell3[0], cell3[1], cell3[2], nc, b)
    order = layout.stable_order(key)
    counts = np.bincount(key, minlength=nc ** 3).astype(np.int64)
    vc = cell_mean_velocity(key, vel32, nc ** 3)
    # v - v_c is the FP32 difference the stored codes are decided on
    nu = np.stack([codec.vel_encode((np.asarray(vel32[d], np.float32) - vc[d][key]).astype(np.float32),
                                    sigma, P.v_bytes)
                   for d in range(3)])
    ids = np.asarray(ids, dtype=np.uint32) if ids is not None else np.arange(len(key), dtype=np.uint32)
    return Store(P, counts, vc, chi3[:, order], nu[:, order], ids[order], sigma, a, a_p)


def measured_sigma(vel32, vc_of_particle):
    """sqrt(<(v - v_c)^2>) over particles and the three dimensions (FP64)."""
    d = np.asarray(vel32, np.float64) - np.asarray(vc_of_particle, np.float64)
    return float(np.sqrt(np.mean(d * d)))


def encode(P, pos, vel, ids=None, a=0.02, sigma=0.0, snap=True):
    """Float particles -> compressed store (the second pass of Fig. fig.ic).

    pos: [3][N] fine-cell coordinates, vel: [3][N] momenta (FP32 values).
    Cell = floor(pos / R) (periodic), chi by Eq. chi, v_c by cell_mean_velocity,
    nu by Eq. nu relative to v_c.  Order: by cell, then by input index.
    sigma <= 0 means: measure it from the particles, as the per-step update does.
    The scale is snapped to 2^(m/16) unless `snap` is False (a scale that is
    already snapped elsewhere is then used as given).
    """
    pos = np.asarray(pos, dtype=np.float32)
    vel = np.asarray(vel, dtype=np.float32)
    nc = P.n_coarse
    cell3, chi3 = [], []
    for d in range(3):
        c, ch = codec.pos_encode(pos[d].astype(np.float64) / P.ratio, P.x_bytes)
        cell3.append(np.mod(c, nc))
        chi3.append(ch)
    cell3, chi3 = np.stack(cell3), np.stack(chi3)
    if sigma <= 0:
        key = layout.storage_index(cell3[0], cell3[1], cell3[2], nc, P.brick_side)
        vc = cell_mean_velocity(key, vel, nc ** 3)
        sigma = measured_sigma(vel, vc[:, key])
    if snap:
        sigma = codec.snap_sigma(sigma)
    return _build(P, cell3, chi3, vel, ids, sigma, a, a)


def encode_drifted(P, cell_old, u_new, p32, ids, sigma, a, a_p):
    """Rebuild the store from drifted particles (Fig. update_xp, both loops).

    cell_old: [3][N] old coarse cell, u_new: [3][N] FP32 drifted offset in
    coarse units relative to the old cell, p32: [3][N] FP32 momenta.  The new
    cell is cell_old + floor(u_new) (periodic) and chi follows Eq. chi; the
    input order is the old storage order, so the stable sort keeps particles
    of one new cell in old-index order.
    """
    u = np.asarray(u_new, dtype=np.float32).astype(np.float64)
    nc = P.n_coarse
    cell3, chi3 = [], []
    for d in range(3):
        shift, ch = codec.pos_encode(u[d], P.x_bytes)
        if np.any(np.abs(shift) > 1):
            raise ValueError("a particle drifted more than one coarse cell")
        cell3.append(np.mod(np.asarray(cell_old[d]) + shift, nc))
        chi3.append(ch)
    return _build(P, np.stack(cell3), np.stack(chi3), p32, ids, sigma, a, a_p)


def decode(store):
    """Store -> (pos [3][N] fine units FP64, vel [3][N] FP64, ids) in storage order."""
    P = store.params
    cells = store.cells()
    key = layout.particle_cells(store.counts)
    pos = np.stack([P.ratio * codec.pos_decode(cells[d], store.chi[d], P.x_bytes) for d in range(3)])
    vel = np.stack([codec.vel_decode(store.nu[d], store.vc[d][key], store.sigma, P.v_bytes) for d in range(3)])
    return pos, vel, store.ids.copy()


def density(store):
    pos, _, _ = decode(store)
    return mesh.cic_deposit(pos, store.params.n_fine, store.params.mass)


def kick_drift(P, u, vc_old, nu, sigma, force, kf, dc):
    """Steps 3 and 5 of `step` for the given particles ([3][n] arrays): the
    decoded momentum (Eq. v) kicked by force * kf and stored as an FP32
    value, re-coded against the same v_c (Eq. nu, Fig. update_vp) and
    decoded again; then the in-cell offset u (coarse units) drifted by that
    momentum times dc, as the FP32 value of one rounding (Fig. update_xp).
    Returns (p2, u_new), both FP32."""
    v = np.stack([codec.vel_decode(nu[d], vc_old[d], sigma, P.v_bytes) for d in range(3)])
    p1 = f32(v + force * kf)
    nu1 = np.stack([codec.vel_encode((p1[d] - vc_old[d]).astype(np.float32), sigma, P.v_bytes)
                    for d in range(3)])
    p2 = f32(np.stack([codec.vel_decode(nu1[d], vc_old[d], sigma, P.v_bytes) for d in range(3)]))
    u_new = fma_f32(p2, np.broadcast_to(np.float32(dc), p2.shape), np.asarray(u, np.float32))
    return p2, u_new


def step(store, a_from, a_to, keep_drifted=False):
    """One KD step of the compressed store (module docstring, steps 1-6)."""
    P = store.params
    if abs(a_from - store.a) > 1e-12 * max(1.0, abs(a_from)):
        raise ValueError("a_from must equal the store's epoch")
    om, ol = P.omega_m, P.omega_l
    cells = store.cells()
    key = layout.particle_cells(store.counts)
    nb = 2 ** (8 * P.x_bytes)
    # 1-2: positions, density, force
    u = np.stack([(store.chi[d].astype(np.float64) + nb // 2 + 0.5) / nb for d in range(3)])
    pos = np.stack([P.ratio * (cells[d] + u[d]) for d in range(3)])
    rho = mesh.cic_deposit(pos, P.n_fine, P.mass)
    force = mesh.force_at(pos, rho, om, P.deconv_power)
    # 3, 5: kick, re-quantised relative to the same v_c; drift
    a_mid = 0.5 * (a_from + a_to)
    kf = cosmo.kick_factor(store.a_p, a_mid, om, ol)
    dc = np.float32(cosmo.drift_factor(a_from, a_to, om, ol) / P.ratio)
    vc_old = store.vc[:, key]
    p2, u_new = kick_drift(P, u, vc_old, store.nu, store.sigma, force, kf, dc)
    # 4: codec scale for the new store
    ratio = cosmo.momentum_growth(a_to, om, ol) / cosmo.momentum_growth(a_from, om, ol)
    sigma_new = codec.snap_sigma(measured_sigma(p2, vc_old) * ratio)
    # 6: rebuild
    out = encode_drifted(P, cells, u_new, p2, store.ids, sigma_new, a_to, a_mid)
    if keep_drifted:
        out.extra.update(cell_old=np.stack(cells), u_new=u_new, p=p2, rho=rho,
                         force=force, sigma_meas_ratio=ratio)
    return out


def run(store, schedule, keep_last_drifted=False):
    """Apply `step` over consecutive scale factors of `schedule`."""
    for i in range(len(schedule) - 1):
        last = keep_last_drifted and i == len(schedule) - 2
        store = step(store, float(schedule[i]), float(schedule[i + 1]), keep_drifted=last)
    return store


def power_spectrum(store, n_bins):
    """P(k) of the store's particles on its fine mesh (Section 3.2)."""
    P = store.params
    pos, _, _ = decode(store)
    return mesh.power_spectrum(pos, P.n_fine, P.mass, P.box, n_bins)


# ---------------------------------------------------------------- uncompressed FP64 mode
@dataclass
class Exact:
    """Plain FP64 particles (no codec), same PM force and KD splitting."""
    params: Params
    pos: np.ndarray
    vel: np.ndarray
    a: float
    a_p: float


def exact_from(P, pos, vel, a):
    return Exact(P, np.asarray(pos, np.float64).copy(), np.asarray(vel, np.float64).copy(), a, a)


def exact_step(st, a_from, a_to):
    P = st.params
    om, ol = P.omega_m, P.omega_l
    rho = mesh.cic_deposit(st.pos, P.n_fine, P.mass)
    force = mesh.force_at(st.pos, rho, om, P.deconv_power)
    a_mid = 0.5 * (a_from + a_to)
    vel = st.vel + force * cosmo.kick_factor(st.a_p, a_mid, om, ol)
    pos = np.mod(st.pos + vel * cosmo.drift_factor(a_from, a_to, om, ol), P.n_fine)
    return replace(st, pos=pos, vel=vel, a=a_to, a_p=a_mid)


def exact_run(st, schedule):
    for i in range(len(schedule) - 1):
        st = exact_step(st, float(schedule[i]), float(schedule[i + 1]))
    return st
