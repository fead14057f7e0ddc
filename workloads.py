"""Seeded synthetic inputs for the Lienard-Wiechert field grid and the Lorentz-oscillator runs.

This module only draws and lays out inputs: positions, axes, prescribed trajectories and
parameters.  It holds none of the method's arithmetic (no retarded time, no field, no
equation of motion), so that both the CUDA path and the CPU oracle can take their inputs from
here without sharing any of the computation.

Shapes follow the paper's workloads (arXiv 2107.12437):
  * Sec. 4.1 / Listing 1: point charges with predefined trajectories on a planar grid;
  * Sec. 4.2 / Listing 2: Lorentz oscillators with charges +-e, electron masses, dt = 1e-18 s.
All arrays are float64 numpy arrays in SI units.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# CODATA 2018 (exact SI values for c and e)
C = 299792458.0
E_CHARGE = 1.602176634e-19
M_E = 9.1093837015e-31
EPS0 = 8.8541878128e-12

SEED_CFG2 = 2107
SEED_CFG4 = 12437
SEED_CFG5 = 210712437
SEED_ADJ = 1243721


@dataclasses.dataclass
class Charges:
    """Point charges with sampled trajectories: sample k at time t0 + k dt."""

    q: np.ndarray  # [M]
    pos: np.ndarray  # [M][S][3]
    vel: np.ndarray  # [M][S][3]
    acc: np.ndarray  # [M][S][3]
    t0: float
    dt: float
    static_before: int = 0

    @property
    def M(self) -> int:
        return int(self.q.shape[0])

    @property
    def S(self) -> int:
        return int(self.pos.shape[1])


@dataclasses.dataclass
class Dipoles:
    """Dipole sources: moment d(t) along a fixed unit axis, samples at t0 + n dt."""

    origin: np.ndarray  # [N][3]
    axis: np.ndarray  # [N][3]
    q: np.ndarray  # [N]
    m1: np.ndarray  # [N] mass of the positive charge
    m2: np.ndarray  # [N] mass of the negative charge
    d: np.ndarray  # [N][S]
    d_dot: np.ndarray  # [N][S]
    d_ddot: np.ndarray  # [N][S]
    t0: float
    dt: float

    @property
    def N(self) -> int:
        return int(self.origin.shape[0])

    @property
    def S(self) -> int:
        return int(self.d.shape[1])


@dataclasses.dataclass
class LOConfig:
    """A batch of B independent Lorentz-oscillator configurations of N dipoles each."""

    origin: np.ndarray  # [B][N][3]
    axis: np.ndarray  # [B][N][3]
    q: np.ndarray  # [B][N]
    m1: np.ndarray  # [B][N]
    m2: np.ndarray  # [B][N]
    omega0: np.ndarray  # [B][N]
    d0: np.ndarray  # [B][N] initial moment along the axis
    dt: float
    n_steps: int
    first_index: int

    @property
    def B(self) -> int:
        return int(self.origin.shape[0])

    @property
    def N(self) -> int:
        return int(self.origin.shape[1])


def unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


# ----------------------------------------------------------------------------------------------
# Field-grid workloads
# ----------------------------------------------------------------------------------------------
def plane_grid(x: np.ndarray, y: np.ndarray, z: float) -> np.ndarray:
    """Points [len(x)*len(y)][3], x the slow index (numpy meshgrid 'ij' order)."""
    X, Y = np.meshgrid(x, y, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], axis=1).astype(np.float64)


def orbit_pair(dt: float = 1e-18, t_end: float = 10e-15, radius: float = 1e-9, beta: float = 0.1):
    """Static +e at the origin and -e on a circle of the given radius in the z = 0 plane.

    Angular speed beta c / radius; position, velocity and acceleration sampled exactly.
    """
    S = int(round(t_end / dt)) + 1
    t = np.arange(S) * dt
    w = beta * C / radius
    pos = np.zeros((2, S, 3))
    vel = np.zeros((2, S, 3))
    acc = np.zeros((2, S, 3))
    pos[1, :, 0] = radius * np.cos(w * t)
    pos[1, :, 1] = radius * np.sin(w * t)
    vel[1, :, 0] = -radius * w * np.sin(w * t)
    vel[1, :, 1] = radius * w * np.cos(w * t)
    acc[1, :, 0] = -radius * w * w * np.cos(w * t)
    acc[1, :, 1] = -radius * w * w * np.sin(w * t)
    q = np.array([E_CHARGE, -E_CHARGE])
    return Charges(q=q, pos=pos, vel=vel, acc=acc, t0=0.0, dt=dt, static_before=1)


def cfg1(n_grid: int = 101):
    """Two charges (static +e at the origin, -e on a 1 nm orbit at 0.1 c), grid +-50 nm, t = 10 fs."""
    ch = orbit_pair()
    g = np.linspace(-50e-9, 50e-9, n_grid)
    points = plane_grid(g, g, 0.0)
    times = np.array([10e-15])
    return ch, points, times


def sinusoidal_dipoles(origin, axis, omega0, amp, dt, t_end, q=E_CHARGE):
    """Dipoles whose charge separation is amp*sin(omega0 t) along the axis: d = q amp sin(omega0 t)."""
    N = origin.shape[0]
    S = int(round(t_end / dt)) + 1
    t = np.arange(S) * dt
    s = amp * np.sin(omega0 * t)
    sd = amp * omega0 * np.cos(omega0 * t)
    sdd = -amp * omega0 * omega0 * np.sin(omega0 * t)
    ones = np.ones((N, 1))
    return Dipoles(
        origin=np.ascontiguousarray(origin, dtype=np.float64),
        axis=np.ascontiguousarray(axis, dtype=np.float64),
        q=np.full(N, q),
        m1=np.full(N, M_E),
        m2=np.full(N, M_E),
        d=q * ones * s[None, :],
        d_dot=q * ones * sd[None, :],
        d_ddot=q * ones * sdd[None, :],
        t0=0.0,
        dt=dt,
    )


def cfg2(n_grid: int = 2048, n_frames: int = 16, n_dipoles: int = 64, t_end: float = 15e-15):
    """64 oscillating dipoles (128 charges +-e) in a 1 um cube, 2048^2 plane grid at z = 0.5 um, 16 frames."""
    rng = np.random.default_rng(SEED_CFG2)
    origin = rng.uniform(0.0, 1e-6, size=(n_dipoles, 3))
    axis = unit_vectors(rng, n_dipoles)
    omega0 = 2 * math.pi * 200e12
    dp = sinusoidal_dipoles(origin, axis, omega0, 1e-11, 1e-18, t_end)
    g = np.linspace(0.0, 1e-6, n_grid)
    times = 10e-15 + np.arange(n_frames) * (5e-15 / 16)
    return dp, g, 0.5e-6, times


def dipoles_as_charges(dp: Dipoles) -> Charges:
    """The same sinusoidal sources written as independent charges +q at R + s/2 u, -q at R - s/2 u.

    Valid for the equal-mass sinusoidal sources built by sinusoidal_dipoles (the separation s is
    d/q and each charge sits s/2 from the origin); used to feed the generic-charge path.
    """
    N, S = dp.N, dp.S
    s = dp.d / dp.q[:, None]
    sd = dp.d_dot / dp.q[:, None]
    sdd = dp.d_ddot / dp.q[:, None]
    pos = np.zeros((2 * N, S, 3))
    vel = np.zeros((2 * N, S, 3))
    acc = np.zeros((2 * N, S, 3))
    q = np.zeros(2 * N)
    for j in range(N):
        u = dp.axis[j]
        for k, sign in ((2 * j, 1.0), (2 * j + 1, -1.0)):
            pos[k] = dp.origin[j][None, :] + sign * 0.5 * s[j][:, None] * u[None, :]
            vel[k] = sign * 0.5 * sd[j][:, None] * u[None, :]
            acc[k] = sign * 0.5 * sdd[j][:, None] * u[None, :]
            q[k] = sign * dp.q[j]
    return Charges(q=q, pos=pos, vel=vel, acc=acc, t0=dp.t0, dt=dp.dt, static_before=1)


# ----------------------------------------------------------------------------------------------
# Lorentz-oscillator workloads
# ----------------------------------------------------------------------------------------------
def lo_batch(origins, axes, omega0, r_dip0, dt, n_steps, first_index, q=E_CHARGE, m=M_E) -> LOConfig:
    origins = np.asarray(origins, dtype=np.float64)
    axes = np.asarray(axes, dtype=np.float64)
    B, N = origins.shape[:2]
    om = np.broadcast_to(np.asarray(omega0, dtype=np.float64), (B, N)).copy()
    return LOConfig(
        origin=origins.copy(),
        axis=axes.copy(),
        q=np.full((B, N), q),
        m1=np.full((B, N), m),
        m2=np.full((B, N), m),
        omega0=om,
        d0=np.full((B, N), q * r_dip0),
        dt=dt,
        n_steps=n_steps,
        first_index=first_index,
    )


def cfg3(B: int = 256, n_steps: int = 40000, orientation: str = "s"):
    """Two in-phase LOs (moments along x) at B separations log-spaced 1 nm .. 1 um.

    orientation 's': separation along y (transverse); 'p': separation along x (longitudinal).
    """
    sep = np.logspace(-9, -6, B)
    origins = np.zeros((B, 2, 3))
    k = 1 if orientation == "s" else 0
    origins[:, 1, k] = sep
    axes = np.zeros((B, 2, 3))
    axes[:, :, 0] = 1.0
    cfg = lo_batch(origins, axes, 2 * math.pi * 200e12, 1e-11, 1e-18, n_steps, 10000)
    return cfg, sep


def listing2(n_steps: int = 40000):
    """Two s dipoles of the paper's listing: axis y, 80 nm apart along x, 2 pi 100 THz, r_dip 1 nm."""
    origins = np.array([[[0.0, 0.0, 0.0], [80e-9, 0.0, 0.0]]])
    axes = np.array([[[0.0, 1.0, 0.0], [0.0, 1.0, 0.0]]])
    return lo_batch(origins, axes, 2 * math.pi * 100e12, 1e-9, 1e-18, n_steps, 10000)


def cfg4(N: int = 256, n_steps: int = 20000):
    """N LOs on a ring of radius 200 nm, moments along z, omega0 jittered +-1% (seeded)."""
    rng = np.random.default_rng(SEED_CFG4)
    ang = 2 * math.pi * np.arange(N) / N
    origins = np.stack([200e-9 * np.cos(ang), 200e-9 * np.sin(ang), np.zeros(N)], axis=1)[None]
    axes = np.zeros((1, N, 3))
    axes[..., 2] = 1.0
    om = 2 * math.pi * 200e12 * (1.0 + rng.uniform(-0.01, 0.01, size=(1, N)))
    return lo_batch(origins, axes, om, 1e-11, 1e-18, n_steps, 10000)


def cfg5(N: int = 4096, n_steps: int = 20000, side: float = 600e-9, min_spacing: float = 5e-9,
         seed: int = SEED_CFG5):
    """N LOs at seeded random positions in a cube with a minimum spacing, random axes."""
    rng = np.random.default_rng(seed)
    pts = np.empty((0, 3))
    cell = min_spacing
    grid = {}
    out = []
    while len(out) < N:
        cand = rng.uniform(0.0, side, size=(4096, 3))
        for p in cand:
            key = tuple((p // cell).astype(int))
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        for qidx in grid.get((key[0] + dx, key[1] + dy, key[2] + dz), ()):
                            if np.sum((out[qidx] - p) ** 2) < min_spacing * min_spacing:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                grid.setdefault(key, []).append(len(out))
                out.append(p)
                if len(out) == N:
                    break
    pts = np.array(out)[None]
    axes = unit_vectors(rng, N)[None]
    return lo_batch(pts, axes, 2 * math.pi * 200e12, 1e-11, 1e-18, n_steps, 10000)


def adjoint_cluster(B: int = 2, N: int = 3, n_steps: int = 3000, spacing: float = 6e-9, seed: int = SEED_ADJ,
                    margin: float = 0.08, charge: float = 1.0, first_index: int = 0) -> LOConfig:
    """B clusters of N LOs (random axes, omega0 = 2 pi 200 THz +-1%, r_dip0 = 10 pm) for gradient
    checks.  Pair distances are drawn so that no retarded time sits within `margin` steps of a
    history sample at the whole- or half-step stage times: a centre-to-centre delay tau (steps)
    with frac(tau) and frac(tau + 1/2) both farther than `margin` from an integer.  The charges
    move by at most r_dip0/(c dt) = 0.033 steps, so finite-difference steps of the inputs do not
    cross the kinks of the piecewise-linear history.  charge scales q (in units of e; the
    radiative decay rate grows as q^2), first_index is the first fitted step."""
    rng = np.random.default_rng(seed)
    dt = 1e-18
    L = C * dt
    origins = np.zeros((B, N, 3))
    for b in range(B):
        while True:
            pts = rng.uniform(0.0, spacing * N ** (1 / 3) * 1.5, size=(N, 3))
            dist = np.linalg.norm(pts[:, None] - pts[None], axis=-1)[np.triu_indices(N, 1)]
            if N > 1 and dist.min() < spacing:
                continue
            f = np.mod(dist / L, 0.5)
            if np.all((f > margin) & (f < 0.5 - margin)):
                break
        origins[b] = pts
    axes = unit_vectors(rng, B * N).reshape(B, N, 3)
    om = 2 * math.pi * 200e12 * (1.0 + rng.uniform(-0.01, 0.01, size=(B, N)))
    return lo_batch(origins, axes, om, 1e-11, dt, n_steps, first_index, q=charge * E_CHARGE)


def population_pair(n_steps: int = 2_100_000, dt: float = 1e-17, r_dip: float = 1e-11, sep: float = 80e-9):
    """Two s dipoles (moments along y, separated along x by 80 nm), q = 20 e, m1 = m2 = m_e,
    omega0 = 2 pi 200 THz; dipole a starts with moment q r_dip, dipole b at rest with none."""
    origins = np.array([[[0.0, 0.0, 0.0], [sep, 0.0, 0.0]]])
    axes = np.array([[[0.0, 1.0, 0.0], [0.0, 1.0, 0.0]]])
    cfg = lo_batch(origins, axes, 2 * math.pi * 200e12, r_dip, dt, n_steps, 0, q=20 * E_CHARGE)
    cfg.d0[0, 1] = 0.0
    return cfg


def oscillating_origins(cfg: LOConfig, amp, Omega, direction=(1.0, 0.0, 0.0), n_steps=None):
    """Origin trajectories R(t) = R0 + amp (cos(Omega t) - 1) u for every dipole (moving dipoles,
    Sec. 4.3: an origin oscillating along x as in the paper's listing, shifted so that R(0) = R0),
    sampled at the half steps t = h dt / 2, h = 0 .. 2 n_steps: (pos, vel, acc)
    [B][N][2 n_steps + 1][3].  amp may be an array [B][N] (0 for fixed dipoles)."""
    n_steps = cfg.n_steps if n_steps is None else n_steps
    B, N = cfg.B, cfg.N
    amp = np.broadcast_to(np.asarray(amp, dtype=np.float64), (B, N))
    u = np.asarray(direction, dtype=np.float64)
    u = u / np.linalg.norm(u)
    t = np.arange(2 * n_steps + 1) * (cfg.dt / 2)
    c, s = np.cos(Omega * t), np.sin(Omega * t)
    pos = cfg.origin[:, :, None, :] + amp[:, :, None, None] * (c - 1.0)[None, None, :, None] * u
    vel = -amp[:, :, None, None] * Omega * s[None, None, :, None] * u
    acc = -amp[:, :, None, None] * Omega ** 2 * c[None, None, :, None] * u
    return pos, vel, np.ascontiguousarray(acc)


def param_charges(seed: int = 41):
    """A mixed set of point charges on analytic trajectories (stationary, oscillating, circular,
    accelerating; par layout of pc_fields_param) within a few nm of the origin, speeds up to 0.5 c,
    and random observation points 5-60 nm away."""
    rng = np.random.default_rng(seed)
    kind, q, par = [], [], []

    def unit():
        v = rng.standard_normal(3)
        return v / np.linalg.norm(v)

    for k in range(12):
        kd = k % 4
        p = np.zeros(12)
        p[:3] = rng.uniform(-3e-9, 3e-9, 3)
        if kd == 1:
            p[3:6] = unit()
            p[6], p[7], p[8] = rng.uniform(0.2e-9, 1e-9), rng.uniform(1e15, 5e16), rng.uniform(0, 2 * math.pi)
            p[7] = min(p[7], 0.5 * C / p[6])
        elif kd == 2:
            e1 = unit()
            e2 = np.cross(e1, unit())
            e2 /= np.linalg.norm(e2)
            p[3:6], p[6:9] = e1, e2
            p[9] = rng.uniform(0.5e-9, 2e-9)
            p[10] = rng.uniform(0.05, 0.4) * C / p[9]
            p[11] = rng.uniform(0, 2 * math.pi)
        elif kd == 3:
            p[3:6] = rng.uniform(-0.1, 0.1, 3) * C
            p[6:9] = rng.uniform(-1, 1, 3) * 1e22
            p[9] = rng.uniform(-5e-15, 5e-15)
        kind.append(kd)
        q.append(E_CHARGE * (1 if k % 3 else -1) * (1 + k % 2))
        par.append(p)
    d = rng.standard_normal((256, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pts = d * rng.uniform(5e-9, 60e-9, size=(256, 1))
    return np.array(kind, dtype=np.int32), np.array(q), np.array(par), pts


def kink_free_points(cfg: LOConfig, times, n: int = 8, r_min: float = 15e-9, r_max: float = 60e-9,
                     margin: float = 0.08, seed: int = 77):
    """n observation points around configuration 0 of cfg whose retarded times from every dipole
    centre, at every one of `times`, sit at least `margin` samples from a history sample (so
    finite-difference steps of the inputs do not cross the kinks of the piecewise-linear history)."""
    rng = np.random.default_rng(seed)
    L = C * cfg.dt
    centre = cfg.origin[0].mean(axis=0)
    out = []
    while len(out) < n:
        d = rng.standard_normal(3)
        p = centre + d / np.linalg.norm(d) * rng.uniform(r_min, r_max)
        ok = True
        for t in times:
            x = t / cfg.dt - np.linalg.norm(cfg.origin[0] - p, axis=1) / L
            f = x - np.floor(x)
            if np.any((f < margin) | (f > 1 - margin)):
                ok = False
                break
        if ok:
            out.append(p)
    return np.array(out)
