"""Pins of the oracle's binary128 field sum (oracle.fields_x) against closed forms (no GPU).

fields_x repeats the float64 oracle's steps (bisection on the retarded time, linear interpolation of
the history, Jackson's form of Eqs. V, A, E, B, superposition over charges) with every intermediate
in binary128.  It serves as the reference where a dipole's +-q charges cancel by R/s, which costs the
float64 evaluation that many digits.  The pins:
  * agreement with the float64 oracle where nothing cancels (point charges of config 1);
  * a charge in uniform motion against the Heaviside-Feynman field (the retarded-time solve and the
    velocity terms);
  * a static dipole on its axis and broadside, whose fields have closed forms free of cancellation,
    at R/s up to 5e5 -- where the float64 oracle visibly loses digits and fields_x must not;
  * a dipole whose charges separate at constant speed (each in uniform motion) against the sum of
    two Heaviside-Feynman fields evaluated in 40-digit arithmetic (mpmath).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import theory as th

K_E = 1.0 / (4.0 * math.pi * W.EPS0)


def _rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    if a.ndim >= 2 and a.shape[-1] == 3:
        return float(np.max(np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)))
    return float(np.max(np.abs(a - b) / np.abs(b)))


def test_fields_x_matches_float64_where_nothing_cancels():
    ch, pts, times = W.cfg1(n_grid=21)
    a = oracle.fields_x(pts, times, charges=ch, r_excl=1e-15)
    b = oracle.fields(pts, times, charges=ch, r_excl=1e-15)
    assert a["status"] == oracle.OK and b["status"] == oracle.OK
    assert np.array_equal(a["mask"], b["mask"])
    m = ~b["mask"].astype(bool)
    # two point charges 1 nm apart seen from 5 nm and beyond.  The float64 oracle rounds each term at
    # its own size (scale_charge: for B that is |E| / c, since B = n x E / c of a nearly radial E is a
    # small cross product), and its interpolation fraction (t' / dt ~ 1e4 samples) carries ~1e-12
    # sample, which moves the orbiting charge's acceleration (turning by 0.03 rad per sample) by ~3e-14
    # of itself: the two agree to 1e-12 of that scale
    for k in ("E", "B", "phi", "A"):
        num = np.abs(a[k] - b[k]) if a[k].ndim == 2 else np.linalg.norm(a[k] - b[k], axis=-1)
        assert float(np.max(num[m] / b["scale_charge"][k][m])) < 1e-12, k


@pytest.mark.parametrize("beta", [0.1, 0.5, 0.9])
def test_fields_x_uniform_motion(beta):
    dt = 1e-18
    S = 3001
    t = np.arange(S) * dt
    v = beta * W.C * np.array([0.0, 0.6, 0.8])
    r0 = np.array([0.0, -20e-9, 3e-9])
    pos = (r0[None, :] + t[:, None] * v[None, :])[None]
    ch = W.Charges(q=np.array([-W.E_CHARGE]), pos=pos, vel=np.broadcast_to(v, pos.shape).copy(),
                   acc=np.zeros_like(pos), t0=0.0, dt=dt)
    T = 2500 * dt
    rng = np.random.default_rng(3)
    pts = r0 + T * v + rng.uniform(-60e-9, 60e-9, size=(20, 3))
    out = oracle.fields_x(pts, [T], charges=ch)
    assert out["status"] == oracle.OK
    E, B, phi, A = th.uniform_motion(-W.E_CHARGE, r0 + v * T, v, pts)
    # the closed form is float64 (~1e-15); the sampled positions are rounded float64 values
    assert _rel(out["E"][0], E) < 1e-13
    assert _rel(out["B"][0], B) < 1e-13
    assert _rel(out["A"][0], A) < 1e-13
    assert _rel(out["phi"][0], phi) < 1e-13


def _single_dipole(d_samples, dd_samples, dt, axis, q=W.E_CHARGE):
    S = d_samples.shape[0]
    return W.Dipoles(origin=np.zeros((1, 3)), axis=np.asarray(axis, dtype=np.float64)[None, :], q=np.array([q]),
                     m1=np.array([W.M_E]), m2=np.array([W.M_E]), d=d_samples[None, :].copy(),
                     d_dot=dd_samples[None, :].copy(), d_ddot=np.zeros((1, S)), t0=0.0, dt=dt)


def test_fields_x_static_dipole_axis_and_broadside():
    # charges +-e at +-s/2 along z, at rest; on the axis E_z = k q 2 R s / (R^2 - s^2/4)^2 and
    # phi = k q s / (R^2 - s^2/4); broadside E = -k q s / (R^2 + s^2/4)^(3/2) z and phi = 0
    s = 1e-11
    q = W.E_CHARGE
    S = 12
    dp = _single_dipole(np.full(S, q * s), np.zeros(S), 1e-18, [0.0, 0.0, 1.0])
    R = np.geomspace(5e-8, 5e-6, 9)
    axis_pts = np.stack([np.zeros_like(R), np.zeros_like(R), R], axis=1)
    ang = np.linspace(0.1, 6.0, R.size)
    side_pts = np.stack([R * np.cos(ang), R * np.sin(ang), np.zeros_like(R)], axis=1)
    t = [10 * 1e-18]  # every retarded time falls in the static pre-history: the charges rest there
    ax = oracle.fields_x(axis_pts, t, dipoles=dp)
    sd = oracle.fields_x(side_pts, t, dipoles=dp)
    ax64 = oracle.fields(axis_pts, t, dipoles=dp)
    assert ax["status"] == oracle.OK and sd["status"] == oracle.OK
    Ez = K_E * q * 2 * R * s / (R * R - s * s / 4) ** 2
    phi_ax = K_E * q * s / (R * R - s * s / 4)
    Eside = -K_E * q * s / (R * R + s * s / 4) ** 1.5
    E_ax = np.stack([np.zeros_like(R), np.zeros_like(R), Ez], axis=1)
    E_sd = np.stack([np.zeros_like(R), np.zeros_like(R), Eside], axis=1)
    assert _rel(ax["E"][0], E_ax) < 1e-14
    assert _rel(ax["phi"][0], phi_ax) < 1e-14
    assert _rel(sd["E"][0], E_sd) < 1e-14
    # broadside the two potentials cancel exactly: what is left is below binary128 rounding of one
    assert np.all(np.abs(sd["phi"][0]) <= 1e-28 * K_E * q / R)
    # static: no magnetic field or vector potential
    assert np.all(ax["A"] == 0.0) and np.all(sd["A"] == 0.0)
    assert np.all(np.linalg.norm(ax["B"][0], axis=1) <= 1e-28 * np.abs(Ez) / W.C)
    # the float64 oracle loses ~log10(R/s) digits here, which the pin must be able to tell apart
    assert _rel(ax64["phi"][0], phi_ax) > 1e-13


def test_fields_x_separating_charges_mpmath():
    # d(t) = d0 + d1 t: each charge moves at constant speed +-d1/(2q) along the axis (linear history,
    # exact under linear interpolation), so each field is the Heaviside-Feynman field of its present
    # position; the +-e sum cancels by R/s ~ 1e5 and is formed in 40-digit arithmetic
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    q = W.E_CHARGE
    dt = 1e-18
    S = 6001
    tt = np.arange(S) * dt
    d0, d1 = q * 1e-11, q * 6e3  # separation 1e-11 m growing at 6 km/s
    axis = np.array([0.6, 0.0, 0.8])
    dp = _single_dipole(d0 + d1 * tt, np.full(S, d1), dt, axis)
    T = 5000 * dt
    rng = np.random.default_rng(8)
    dirs = rng.normal(size=(12, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    pts = dirs * np.geomspace(1e-7, 1e-6, 12)[:, None]
    out = oracle.fields_x(pts, [T], dipoles=dp)
    assert out["status"] == oracle.OK

    def hf(qc, r_now, v, r):
        c = mp.mpf(W.C)
        Rv = [r[i] - r_now[i] for i in range(3)]
        R = mp.sqrt(sum(x * x for x in Rv))
        vv = sum(x * x for x in v)
        b2 = vv / (c * c)
        cos_th = sum(Rv[i] * v[i] for i in range(3)) / (R * mp.sqrt(vv))
        den = 1 - b2 * (1 - cos_th * cos_th)
        k = qc / (4 * mp.pi * mp.mpf(W.EPS0))
        E = [k * (1 - b2) * Rv[i] / (R ** 3 * den ** mp.mpf(1.5)) for i in range(3)]
        B = [(v[(i + 1) % 3] * E[(i + 2) % 3] - v[(i + 2) % 3] * E[(i + 1) % 3]) / (c * c) for i in range(3)]
        phi = k / (R * mp.sqrt(den))
        A = [v[i] * phi / (c * c) for i in range(3)]
        return E, B, phi, A

    d_now = mp.mpf(d0) + mp.mpf(d1) * mp.mpf(T)
    ax = [mp.mpf(x) for x in axis]
    half = d_now / (2 * mp.mpf(q))
    vh = mp.mpf(d1) / (2 * mp.mpf(q))
    for p in range(pts.shape[0]):
        r = [mp.mpf(x) for x in pts[p]]
        Ep, Bp, php, Ap = hf(mp.mpf(q), [half * a for a in ax], [vh * a for a in ax], r)
        Em, Bm, phm, Am = hf(-mp.mpf(q), [-half * a for a in ax], [-vh * a for a in ax], r)
        E = np.array([float(Ep[i] + Em[i]) for i in range(3)])
        B = np.array([float(Bp[i] + Bm[i]) for i in range(3)])
        A = np.array([float(Ap[i] + Am[i]) for i in range(3)])
        phi = float(php + phm)
        assert np.linalg.norm(out["E"][0, p] - E) <= 1e-14 * np.linalg.norm(E), p
        assert np.linalg.norm(out["B"][0, p] - B) <= 1e-14 * np.linalg.norm(B), p
        assert np.linalg.norm(out["A"][0, p] - A) <= 1e-14 * np.linalg.norm(A), p
        assert abs(out["phi"][0, p] - phi) <= 1e-14 * abs(phi), p
