"""Pins of the FP64 oracle against what the paper and the physics fix (no GPU).

Every test here checks the oracle against something other than itself: values the paper prints,
textbook closed forms, brute force on tiny inputs, or invariants.  Each is chosen so that a dropped
term, a flipped sign, a swapped index or operand in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import fit, theory as th

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.linalg.norm(np.atleast_2d(a - b), axis=-1) / np.linalg.norm(np.atleast_2d(b), axis=-1)))


# ------------------------------------------------------------------------------------------------
# Green's-function theory (App. A) against the numbers the paper prints
# ------------------------------------------------------------------------------------------------
def test_theory_listing2_values():
    d12, g12 = th.s_dipole_theory(80e-9, 2 * math.pi * 100e12)
    assert round(d12, 3) == GOLDEN["listing2_delta12_th"]["value"]
    assert round(g12, 3) == GOLDEN["listing2_gamma12_th"]["value"]


def test_theory_fft_figure_shift():
    d12, _ = th.s_dipole_theory(80e-9, 2 * math.pi * 200e12)
    assert round(d12, 2) == GOLDEN["fft_delta12_th"]["value"]


def test_gamma0_values():
    # printed to the shown digits: 19.791 MHz and 7.916 GHz (rates in 1/s)
    g = th.gamma0(W.E_CHARGE, W.M_E / 2, 2 * math.pi * 200e12)
    assert round(g / 1e6, 3) == round(GOLDEN["gamma0_e_200THz"]["value"] / 1e6, 3)
    g20 = th.gamma0(20 * W.E_CHARGE, W.M_E / 2, 2 * math.pi * 200e12)
    assert round(g20 / 1e9, 3) == round(GOLDEN["gamma0_20e_200THz"]["value"] / 1e9, 3)


def test_gamma0_tls_equals_lo_rate():
    # Eq. f with f = 1 (q^2/m = 2 w0 d0^2 / hbar) maps the LO rate onto Eq. SE0
    w0 = 2 * math.pi * 200e12
    q, m = W.E_CHARGE, W.M_E / 2
    d0 = math.sqrt(q * q * th.HBAR / (2 * m * w0))
    assert abs(th.gamma0_tls(w0, d0) / th.gamma0(q, m, w0) - 1) < 1e-13


def test_green_self_term_reduces_to_gamma0():
    # Im G(R -> 0) = k^3/(6 pi): the pair rate tends to gamma0 (gamma_12 -> gamma_0) at small R
    # (k R = 1e-3: the deviation (kR)^2/5 and the cancellation error eps/(kR)^3 are both ~1e-7)
    w0 = 2 * math.pi * 200e12
    sep = 1e-3 * th.C / w0
    _, g12 = th.s_dipole_theory(sep, w0)
    assert abs(g12 - 1.0) < 1e-6
    _, g12p = th.p_dipole_theory(sep, w0)
    assert abs(g12p - 1.0) < 1e-6


def test_exact_pole_reduces_to_markov_theory():
    # where |delta|/w0 << 1 the exact classical pole and App. A agree to first order
    w0 = 2 * math.pi * 100e12
    g0 = th.gamma0(W.E_CHARGE, W.M_E / 2, w0)
    for sep in (80e-9, 300e-9):
        _, dl, g = th.exact_pair_pole([sep, 0, 0], [0, 1, 0], w0, W.E_CHARGE, W.M_E / 2)
        d12, g12 = th.s_dipole_theory(sep, w0)
        assert abs(dl / g0 - d12) < 1e-4 * max(1.0, abs(d12))
        assert abs(g / g0 - (1 + g12)) < 1e-4
    # antisymmetric mode decays at gamma0 - gamma12 (Eq. gamma_super_sub)
    _, dlm, gm = th.exact_pair_pole([80e-9, 0, 0], [0, 1, 0], w0, W.E_CHARGE, W.M_E / 2, in_phase=False)
    d12, g12 = th.s_dipole_theory(80e-9, w0)
    assert abs(gm / g0 - (1 - g12)) < 1e-4
    assert abs(dlm / g0 + d12) < 1e-4 * abs(d12)


# ------------------------------------------------------------------------------------------------
# Retarded time (Eq. ret_t)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("beta", [0.1, 0.5, 0.9])
def test_retarded_delay_uniform_motion(beta):
    dt = 1e-18
    S = 2001
    t = np.arange(S) * dt
    v = np.array([beta * W.C * 0.6, beta * W.C * 0.8, 0.0])
    r0 = np.array([1e-9, -2e-9, 0.5e-9])
    pos = (r0[None, :] + t[:, None] * v[None, :])[None]
    ch = W.Charges(q=np.array([W.E_CHARGE]), pos=pos, vel=np.broadcast_to(v, pos.shape).copy(),
                   acc=np.zeros_like(pos), t0=0.0, dt=dt)
    rng = np.random.default_rng(1)
    pts = rng.uniform(-100e-9, 100e-9, size=(20, 3))
    T = 1800 * dt
    exact = th.uniform_delay(r0, v, T, pts)
    for p, e in zip(pts, exact):
        tau, st = oracle.retarded_delay(0, T, p, charges=ch)
        assert st == oracle.OK
        assert abs(tau - e) <= 1e-13 * e


def test_retarded_delay_brute_force_tiny():
    # random slow piecewise-linear trajectories: scan g(tau) = c tau - |r - r_s(t - tau)| densely,
    # check that it changes sign exactly once and that bisection lands inside that cell
    rng = np.random.default_rng(7)
    dt = 1e-18
    for trial in range(12):
        S = int(rng.integers(8, 50))
        steps = rng.normal(size=(S, 3))
        steps *= (0.7 * W.C * dt) / np.linalg.norm(steps, axis=1, keepdims=True) * rng.uniform(0.05, 1.0, (S, 1))
        pos = np.cumsum(steps, axis=0)[None]
        ch = W.Charges(q=np.array([1.0]), pos=pos, vel=np.zeros_like(pos), acc=np.zeros_like(pos), t0=0.0, dt=dt)
        t = (S - 1) * dt
        r = pos[0, -1] + rng.normal(size=3) * 0.2 * W.C * dt * S * 0.3
        tau, st = oracle.retarded_delay(0, t, r, charges=ch)
        if st != oracle.OK:
            # the root would precede the first sample: confirm by brute force that g(t - t0) < 0
            assert st == oracle.ERR_HISTORY
            g_end = W.C * t - np.linalg.norm(r - pos[0, 0])
            assert g_end < 0
            continue
        taus = np.linspace(0.0, t, 20001)
        x = (t - taus) / dt
        k = np.minimum(np.floor(x).astype(int), S - 2)
        thv = x - k
        ps = pos[0, k] + thv[:, None] * (pos[0, k + 1] - pos[0, k])
        g = W.C * taus - np.linalg.norm(r[None, :] - ps, axis=1)
        sc = np.nonzero(np.diff(np.sign(g)) != 0)[0]
        assert len(sc) == 1
        assert taus[sc[0]] - 1e-30 <= tau <= taus[sc[0] + 1] + 1e-30


def test_history_error_without_static_extension():
    ch, pts, times = W.cfg1()
    ch.static_before = 0
    # at t = 0.1 fs the retarded time of a point 50 nm away precedes the first sample
    out = oracle.fields(pts[:5], [1e-16], charges=ch)
    assert out["status"] == oracle.ERR_HISTORY
    ch.static_before = 1
    out = oracle.fields(pts[:5], [1e-16], charges=ch)
    assert out["status"] == oracle.OK


# ------------------------------------------------------------------------------------------------
# Fields: static, uniform motion, Jackson vs Griffiths, Hertzian dipole, Larmor
# ------------------------------------------------------------------------------------------------
def test_static_charges_x1_geometry():
    # Listing 1: +-e at (+-10 nm, 0, 0), grid +-50 nm, t = 0 (history held static)
    S = 3
    pos = np.zeros((2, S, 3))
    pos[0, :, 0] = 10e-9
    pos[1, :, 0] = -10e-9
    ch = W.Charges(q=np.array([W.E_CHARGE, -W.E_CHARGE]), pos=pos, vel=np.zeros_like(pos), acc=np.zeros_like(pos),
                   t0=0.0, dt=1e-18, static_before=1)
    g = np.linspace(-50e-9, 50e-9, 41)
    pts = W.plane_grid(g, g, 0.0)
    out = oracle.fields(pts, [2e-18], charges=ch, r_excl=1e-15)
    assert out["status"] == oracle.OK
    m = out["mask"][0].astype(bool)
    assert m.sum() == 2  # (+-10 nm, 0, 0) are on the grid
    E1, p1 = th.coulomb_static(W.E_CHARGE, [10e-9, 0, 0], pts[~m])
    E2, p2 = th.coulomb_static(-W.E_CHARGE, [-10e-9, 0, 0], pts[~m])
    assert rel(out["E"][0][~m], E1 + E2) < 1e-13
    assert np.max(np.abs(out["phi"][0][~m] - (p1 + p2)) / (np.abs(p1) + np.abs(p2))) < 1e-14
    # B = n x E / c of a static charge vanishes up to rounding; A vanishes exactly (v = 0)
    Bn = np.linalg.norm(out["B"][0][~m], axis=1)
    En = np.linalg.norm(out["E"][0][~m], axis=1)
    assert np.all(Bn <= 1e-15 * En / W.C)
    assert np.all(out["A"] == 0.0)


@pytest.mark.parametrize("beta", [0.1, 0.5, 0.9])
def test_uniform_motion_heaviside_feynman(beta):
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
    pts = r0 + T * v + rng.uniform(-60e-9, 60e-9, size=(50, 3))
    out = oracle.fields(pts, [T], charges=ch)
    assert out["status"] == oracle.OK
    E, B, phi, A = th.uniform_motion(-W.E_CHARGE, r0 + v * T, v, pts)
    assert rel(out["E"][0], E) < 1e-12
    assert rel(out["B"][0], B) < 1e-12
    assert rel(out["A"][0], A) < 1e-12
    assert np.max(np.abs(out["phi"][0] - phi) / np.abs(phi)) < 1e-12
    # radiation field of an unaccelerated charge is exactly zero
    out_r = oracle.fields(pts, [T], charges=ch, kind=oracle.RADIATION)
    assert np.all(out_r["E"] == 0.0)


def test_jackson_equals_griffiths_and_potential_identities():
    rng = np.random.default_rng(11)
    for _ in range(200):
        aR = rng.normal(size=3) * 10 ** rng.uniform(-10, -6)
        v = rng.normal(size=3)
        v *= rng.uniform(0.0, 0.95) * W.C / np.linalg.norm(v)
        acc = rng.normal(size=3) * 10 ** rng.uniform(18, 26)
        q = W.E_CHARGE
        Ec, Er, phi, A = oracle.lw_jackson(q, aR, v, acc)
        Eg, Bg = oracle.lw_griffiths(q, aR, v, acc)
        assert rel(Ec + Er, Eg) < 1e-12
        # A = v phi / c^2 (reading of Eq. A)
        assert rel(A, v * phi / W.C ** 2) < 1e-14
        # B = n x E / c is perpendicular to E and to n
        n = aR / np.linalg.norm(aR)
        assert abs(np.dot(Bg, Eg)) <= 1e-12 * np.linalg.norm(Bg) * np.linalg.norm(Eg)
        # radiation field is transverse: n . E_rad = 0
        assert abs(np.dot(n, Er)) <= 1e-12 * np.linalg.norm(Er)


def test_hertzian_dipole_app_e():
    # Sec. 4.1: oscillating dipole, omega0 = 7e16 rad/s, d0 = 4 e 1e-9 C m, from two charges
    # q = 1e5 e separated by 4e-14 m (reading of the garbled separation), along x; E and B on the z axis
    w = 7e16
    q = 1e5 * W.E_CHARGE
    sep = 4e-14
    lam = 2 * math.pi * W.C / w
    dt = 2e-21
    zs = np.array([0.05, 0.1, 0.3, 0.7, 1.0, 1.6, 2.5]) * lam
    t_eval = 3.0 * lam / W.C + 0.37e-16
    S = int(t_eval / dt) + 3
    tt = np.arange(S) * dt
    d = q * sep * np.cos(w * tt)
    dp = W.Dipoles(origin=np.zeros((1, 3)), axis=np.array([[1.0, 0.0, 0.0]]), q=np.array([q]),
                   m1=np.array([1.0]), m2=np.array([1.0]), d=d[None], d_dot=(-q * sep * w * np.sin(w * tt))[None],
                   d_ddot=(-q * sep * w * w * np.cos(w * tt))[None], t0=0.0, dt=dt)
    pts = np.stack([np.zeros_like(zs), np.zeros_like(zs), zs], axis=1)
    out = oracle.fields(pts, [t_eval], dipoles=dp)
    assert out["status"] == oracle.OK
    E_th, B_th = th.hertzian_dipole([q * sep, 0, 0], w, pts, t_eval)
    errE = np.linalg.norm(out["E"][0] - E_th, axis=1) / np.linalg.norm(E_th, axis=1)
    errB = np.linalg.norm(out["B"][0] - B_th, axis=1) / np.linalg.norm(B_th, axis=1)
    # the physical dipole departs from the ideal one as (sep/z)^2 and through interpolation (w dt)^2/8
    assert np.all(errE < GOLDEN["hertzian_rel_error_bound"]["value"])
    assert np.all(errB < GOLDEN["hertzian_rel_error_bound"]["value"])
    # dropping either term of Eq. E breaks the agreement by many orders
    out_c = oracle.fields(pts, [t_eval], dipoles=dp, kind=oracle.COULOMB)
    assert np.max(np.linalg.norm(out_c["E"][0] - E_th, axis=1) / np.linalg.norm(E_th, axis=1)) > 1e-2


def _flux_average(ch, r_sphere, times, n_theta=48):
    """Time-averaged outward flux of E_rad x B_rad / mu0 through a sphere around the origin."""
    x, wq = np.polynomial.legendre.leggauss(n_theta)
    pts = np.stack([r_sphere * np.sqrt(1 - x * x), np.zeros_like(x), r_sphere * x], axis=1)
    out = oracle.fields(pts, times, charges=ch, kind=oracle.RADIATION)
    assert out["status"] == oracle.OK
    S = np.cross(out["E"], out["B"]) / th.MU0
    Sr = np.sum(S * (pts / r_sphere)[None], axis=2)
    flux = 2 * math.pi * r_sphere ** 2 * np.sum(Sr * wq[None, :], axis=1)
    return float(np.mean(flux))


def test_larmor_power_linear_oscillation():
    # charge oscillating along z with beta_max = 0.01: radiated power averaged over a period equals
    # the period average of Lienard's q^2 gamma^6 a^2 / (6 pi eps0 c^3) (-> Larmor as beta -> 0)
    w = 1e15
    x0 = 0.01 * W.C / w
    r_s = 3e-3
    Tp = 2 * math.pi / w
    dt = 1e-19
    # the retarded times of the sphere lie in [0, Tp] up to x0/c: sample [-Tp, 2 Tp]
    t_start = -Tp
    n_t = 32
    times = r_s / W.C + np.arange(n_t) * Tp / n_t
    S = int(3 * Tp / dt) + 3
    tt = t_start + np.arange(S) * dt
    pos = np.zeros((1, S, 3))
    vel = np.zeros((1, S, 3))
    acc = np.zeros((1, S, 3))
    pos[0, :, 2] = x0 * np.cos(w * tt)
    vel[0, :, 2] = -x0 * w * np.sin(w * tt)
    acc[0, :, 2] = -x0 * w * w * np.cos(w * tt)
    ch = W.Charges(q=np.array([W.E_CHARGE]), pos=pos, vel=vel, acc=acc, t0=t_start, dt=dt)
    P_flux = _flux_average(ch, r_s, times)
    tq = np.arange(4096) * Tp / 4096
    a2 = (x0 * w * w * np.cos(w * tq)) ** 2
    g6 = (1.0 / (1.0 - (x0 * w * np.sin(w * tq) / W.C) ** 2)) ** 3
    P_lienard = float(np.mean(th.larmor_power(W.E_CHARGE, a2 * g6)))
    P_larmor = th.larmor_power(W.E_CHARGE, 0.5 * (x0 * w * w) ** 2)
    assert abs(P_flux / P_lienard - 1) < 1e-5
    assert abs(P_flux / P_larmor - 1) < 2e-4  # O(beta^2) relativistic correction


def test_lienard_power_circular_orbit():
    # cfg1's orbiting charge (beta = 0.1): constant radiated power q^2 gamma^4 a^2 / (6 pi eps0 c^3)
    radius = 1e-9
    beta = 0.1
    w = beta * W.C / radius
    r_s = 2e-4
    Tp = 2 * math.pi / w
    dt = 1e-19
    t_start = -Tp
    times = r_s / W.C + np.arange(8) * Tp / 8
    S = int(3 * Tp / dt) + 3
    tt = t_start + np.arange(S) * dt
    pos = np.zeros((1, S, 3))
    vel = np.zeros((1, S, 3))
    acc = np.zeros((1, S, 3))
    pos[0, :, 0], pos[0, :, 1] = radius * np.cos(w * tt), radius * np.sin(w * tt)
    vel[0, :, 0], vel[0, :, 1] = -radius * w * np.sin(w * tt), radius * w * np.cos(w * tt)
    acc[0, :, 0], acc[0, :, 1] = -radius * w * w * np.cos(w * tt), -radius * w * w * np.sin(w * tt)
    ch = W.Charges(q=np.array([W.E_CHARGE]), pos=pos, vel=vel, acc=acc, t0=t_start, dt=dt)
    # the radiation pattern is not axisymmetric about z: integrate in azimuth as well
    x, wq = np.polynomial.legendre.leggauss(32)
    n_ph = 32
    phis = np.arange(n_ph) * 2 * math.pi / n_ph
    st = np.sqrt(1 - x * x)
    pts = np.concatenate([np.stack([r_s * st * math.cos(p), r_s * st * math.sin(p), r_s * x], axis=1) for p in phis])
    wts = np.concatenate([wq * (2 * math.pi / n_ph) for _ in phis])
    out = oracle.fields(pts, times, charges=ch, kind=oracle.RADIATION)
    assert out["status"] == oracle.OK
    S_ = np.cross(out["E"], out["B"]) / th.MU0
    Sr = np.sum(S_ * (pts / r_s)[None], axis=2)
    flux = r_s ** 2 * np.sum(Sr * wts[None, :], axis=1)
    P = th.lienard_power_circular(W.E_CHARGE, beta * W.C, beta * W.C * w)
    assert np.max(np.abs(flux / P - 1)) < 1e-4


def test_dipole_charges_follow_centre_of_mass():
    # a static dipole with unequal masses is two static charges whose centre of mass is the origin
    # (Sec. 2.3: R = (m1 r1 + m2 r2)/(m1 + m2)) and whose separation r1 - r2 is d/q along the axis
    q = W.E_CHARGE
    m1, m2 = 3.0 * W.M_E, W.M_E
    Rc = np.array([1e-9, 2e-9, -1e-9])
    u = np.array([0.0, 0.6, 0.8])
    rdip = 0.7e-9
    S = 4
    dp = W.Dipoles(origin=Rc[None], axis=u[None], q=np.array([q]), m1=np.array([m1]), m2=np.array([m2]),
                   d=np.full((1, S), q * rdip), d_dot=np.zeros((1, S)), d_ddot=np.zeros((1, S)), t0=0.0, dt=1e-18)
    # solve m1 r1 + m2 r2 = (m1 + m2) Rc and r1 - r2 = rdip u for r1, r2
    Mx = np.array([[m1, m2], [1.0, -1.0]])
    sol = np.linalg.solve(Mx, np.stack([(m1 + m2) * Rc, rdip * u]))
    r1, r2 = sol[0], sol[1]
    rng = np.random.default_rng(5)
    pts = Rc + rng.uniform(-5e-9, 5e-9, size=(30, 3))
    out = oracle.fields(pts, [2e-18], dipoles=dp)
    E1, p1 = th.coulomb_static(q, r1, pts)
    E2, p2 = th.coulomb_static(-q, r2, pts)
    assert rel(out["E"][0], E1 + E2) < 1e-12


# ------------------------------------------------------------------------------------------------
# Lorentz-oscillator run (Algorithm 1)
# ------------------------------------------------------------------------------------------------
def _isolated_cfg(dt, n_steps):
    cfg = W.lo_batch([[[0.0, 0.0, 0.0]]], [[[1.0, 0.0, 0.0]]], 2 * math.pi * 200e12, 1e-11, dt, n_steps, 0)
    return cfg


def test_isolated_lo_closed_form_and_rk4_order():
    errs = []
    for dt in (2e-17, 1e-17):
        n = int(round(2e-14 / dt))
        cfg = _isolated_cfg(dt, n)
        out = oracle.dipoles_run(cfg)
        assert out["status"] == oracle.OK
        t = np.arange(n + 1) * dt
        g0 = th.gamma0(W.E_CHARGE, W.M_E / 2, cfg.omega0[0, 0])
        d_ex, _ = th.isolated_lo(t, cfg.d0[0, 0], cfg.omega0[0, 0], g0)
        errs.append(np.max(np.abs(out["d"][0] - d_ex)) / cfg.d0[0, 0])
    # fourth order: halving dt divides the error by ~16
    assert 12.0 < errs[0] / errs[1] < 20.0
    assert errs[1] < 1e-7


def test_isolated_lo_energy_decays_at_gamma0():
    dt = 1e-18
    cfg = _isolated_cfg(dt, 20000)
    out = oracle.dipoles_run(cfg)
    g0 = th.gamma0(W.E_CHARGE, W.M_E / 2, cfg.omega0[0, 0])
    e = out["energy"][0]
    # energy averaged over whole periods decays as exp(-gamma0 t) (Sec. 2.3; Larmor, Sec. 2.4)
    per = int(round(2 * math.pi / cfg.omega0[0, 0] / dt))
    e1 = np.mean(e[0:per])
    e2 = np.mean(e[3 * per:4 * per])
    rate = -math.log(e2 / e1) / (3 * per * dt)
    assert abs(rate / g0 - 1) < 1e-3
    # energy at t = 0 (Eq. dipoleE): m w0^2 d0^2 / (2 q^2)
    m = W.M_E / 2
    assert abs(e[0] - m * cfg.omega0[0, 0] ** 2 * cfg.d0[0, 0] ** 2 / (2 * W.E_CHARGE ** 2)) <= 1e-15 * e[0]


def test_listing2_coupled_dipoles():
    cfg = W.listing2()
    out = oracle.dipoles_run(cfg)
    assert out["status"] == oracle.OK
    m = W.M_E / 2
    ke = m * out["d_dot"][0] ** 2 / (2 * W.E_CHARGE ** 2)
    f = fit.ke_fit(ke, cfg.dt, cfg.first_index)
    g0 = th.gamma0(W.E_CHARGE, m, cfg.omega0[0, 0])
    d12 = (f["omega"] - cfg.omega0[0, 0]) / g0
    gp = f["gamma"] / g0
    # the paper prints 156.919 and 1.997; its stated accuracy is 0.2 %
    assert round(d12, 3) == GOLDEN["listing2_delta12_sim"]["value"]
    assert abs(gp / GOLDEN["listing2_gamma_plus_sim"]["value"] - 1) < GOLDEN["sweep_rel_error_bound"]["value"]
    # both dipoles are identical by symmetry
    assert np.max(np.abs(out["d"][0] - out["d"][1])) <= 1e-12 * cfg.d0[0, 0]


def test_p_dipoles_against_exact_pole():
    # p dipoles (moments along the separation) at 100 nm, 2 pi 200 THz: simulation vs exact pole and App. A
    w0 = 2 * math.pi * 200e12
    origins = np.array([[[0.0, 0.0, 0.0], [100e-9, 0.0, 0.0]]])
    axes = np.array([[[1.0, 0.0, 0.0], [1.0, 0.0, 0.0]]])
    cfg = W.lo_batch(origins, axes, w0, 1e-11, 1e-18, 30000, 10000)
    out = oracle.dipoles_run(cfg)
    assert out["status"] == oracle.OK
    m = W.M_E / 2
    ke = m * out["d_dot"][0] ** 2 / (2 * W.E_CHARGE ** 2)
    f = fit.ke_fit(ke, cfg.dt, cfg.first_index)
    g0 = th.gamma0(W.E_CHARGE, m, w0)
    _, dl, g = th.exact_pair_pole([100e-9, 0, 0], [1, 0, 0], w0, W.E_CHARGE, m)
    d12, g12 = th.p_dipole_theory(100e-9, w0)
    assert abs((f["omega"] - w0) / dl - 1) < 2e-3
    assert abs(f["gamma"] / g - 1) < 2e-3
    assert abs((f["omega"] - w0) / g0 / d12 - 1) < 2e-3
    assert abs(f["gamma"] / g0 / (1 + g12) - 1) < 2e-3


def test_causality_and_velocity_guards():
    # Sec. 3.2: dt must be below the light crossing time between dipoles
    origins = np.array([[[0.0, 0.0, 0.0], [0.2e-9, 0.0, 0.0]]])
    axes = np.array([[[0.0, 1.0, 0.0], [0.0, 1.0, 0.0]]])
    cfg = W.lo_batch(origins, axes, 2 * math.pi * 200e12, 1e-12, 1e-18, 10, 0)
    assert oracle.dipoles_run(cfg)["status"] == oracle.ERR_CAUSALITY
    # Sec. 3.2: a charge faster than max_vel (default c/100) stops the run
    cfg = _isolated_cfg(1e-18, 2000)
    cfg.d0[:] = W.E_CHARGE * 1e-8  # amplitude 10 nm at 200 THz: peak charge speed ~6e6 m/s > c/100
    assert oracle.dipoles_run(cfg)["status"] == oracle.ERR_VELOCITY


def test_ed_stage_reading_matches_paper_frozen_does_not():
    # reading of Algorithm 1: E_d evaluated at each RK4 stage time (default) reproduces the
    # printed gamma+ = 1.997 within 0.2 %; holding E_d at its value at t for all stages does not
    cfg = W.listing2()
    m = W.M_E / 2
    res = []
    for mode in (0, 1):
        out = oracle.dipoles_run(cfg, ed_mode=mode)
        assert out["status"] == oracle.OK
        ke = m * out["d_dot"][0] ** 2 / (2 * W.E_CHARGE ** 2)
        res.append(fit.ke_fit(ke, cfg.dt, cfg.first_index))
    g0 = th.gamma0(W.E_CHARGE, m, cfg.omega0[0, 0])
    gp = GOLDEN["listing2_gamma_plus_sim"]["value"]
    assert abs(res[0]["gamma"] / g0 / gp - 1) < GOLDEN["sweep_rel_error_bound"]["value"]
    assert abs(res[1]["gamma"] / g0 / gp - 1) > 0.02


# ------------------------------------------------------------------------------------------------
# Kinetic-energy fit (Eq. KE)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("gamma", [0.0, 2e7, 3e10])
def test_fit_recovers_synthetic_parameters(gamma):
    dt = 1e-18
    w = 2 * math.pi * 200e12 * (1 + 3.1e-7)
    t = np.arange(40000) * dt
    A, ph = 2.5e-21, 0.4
    ke = A * np.exp(-gamma * t) * np.sin(w * t + ph) ** 2
    f = fit.ke_fit(ke, dt, 10000)
    assert abs(f["omega"] / w - 1) < 1e-9
    assert abs(f["gamma"] - gamma) < 1e-6 * max(gamma, 2e7)


def test_scale_outputs_bound_the_superposition():
    # the magnitude sums are upper bounds of the superposed fields (triangle inequality), the source
    # sums lie between them, and for a lone charge all of them equal the field itself
    dp, g, z, times = W.cfg2(n_dipoles=64)
    pts = W.plane_grid(g[::256], g[::256], z)
    out = oracle.fields(pts, times[:1], dipoles=dp)
    for k in ("E", "B", "phi", "A"):
        f = np.abs(out[k][0]) if k == "phi" else np.linalg.norm(out[k][0], axis=-1)
        sc, ss = out["scale_charge"][k][0], out["scale_source"][k][0]
        assert np.all(f <= ss * (1 + 1e-12)) and np.all(ss <= sc * (1 + 1e-12))
    # a dipole's two fields cancel: the charge sum exceeds the source sum by ~R/s
    assert np.median(out["scale_charge"]["E"][0] / out["scale_source"]["E"][0]) > 1e3
    ch, pts1, _ = W.cfg1(n_grid=11)
    ch1 = W.Charges(q=ch.q[1:], pos=ch.pos[1:], vel=ch.vel[1:], acc=ch.acc[1:], t0=ch.t0, dt=ch.dt, static_before=1)
    o1 = oracle.fields(pts1, [1e-14], charges=ch1)
    En = np.linalg.norm(o1["E"][0], axis=-1)
    assert np.allclose(o1["scale_source"]["E"][0], En, rtol=1e-15)
    # the per-term rounding scale adds the magnitudes of the Coulomb and radiation parts
    oc = oracle.fields(pts1, [1e-14], charges=ch1, kind=oracle.COULOMB)
    orad = oracle.fields(pts1, [1e-14], charges=ch1, kind=oracle.RADIATION)
    ecr = np.linalg.norm(oc["E"][0], axis=-1) + np.linalg.norm(orad["E"][0], axis=-1)
    assert np.allclose(o1["scale_charge"]["E"][0], ecr, rtol=1e-14)


def test_populations_solve_the_density_matrix_equations():
    # Eq. DM in the dressed basis, integrated numerically from rho_aa(0) = 1: rho_++ = rho_-- =
    # rho_+- = rho_-+ = 1/2 (|+-> = (|e_a g_b> +- |g_a e_b>)/sqrt 2), and
    # rho_aa = <sigma_a^+ sigma_a^-> = (rho_++ + rho_-- + rho_+- + rho_-+)/2,
    # rho_bb = (rho_++ + rho_-- - rho_+- - rho_-+)/2
    from scipy.integrate import solve_ivp

    g0, g12, d12 = 1.0, 0.83, 7.3

    def rhs(t, y):
        pp, mm, pm_re, pm_im = y
        pm = pm_re + 1j * pm_im
        dpm = -(g0 + 2j * d12) * pm
        return [-(g0 + g12) * pp, -(g0 - g12) * mm, dpm.real, dpm.imag]

    ts = np.linspace(0.0, 3.0, 61)
    sol = solve_ivp(rhs, (0.0, 3.0), [0.5, 0.5, 0.5, 0.0], t_eval=ts, rtol=1e-12, atol=1e-14)
    pp, mm, pm_re = sol.y[0], sol.y[1], sol.y[2]
    raa_num = 0.5 * (pp + mm + 2.0 * pm_re)
    rbb_num = 0.5 * (pp + mm - 2.0 * pm_re)
    raa, rbb = th.populations(ts, g0, g12, d12)
    assert np.max(np.abs(raa - raa_num)) < 1e-9
    assert np.max(np.abs(rbb - rbb_num)) < 1e-9
    assert raa[0] == pytest.approx(1.0) and rbb[0] == pytest.approx(0.0, abs=1e-15)
    # the limit of very small separations, gamma12 -> gamma0 (App. A)
    raa0, _ = th.populations(ts, g0, g0, d12)
    assert np.allclose(raa0, 0.25 * (1 + np.exp(-2 * g0 * ts) + 2 * np.cos(2 * d12 * ts) * np.exp(-g0 * ts)))


def _moving_cfg(n_steps=600):
    # two s dipoles 20 nm apart; dipole 0's origin oscillates along x (0.1 nm, 2 pi 20 THz: up to
    # 1.3e4 m/s), dipole 1 rests
    origins = np.array([[[0.0, 0.0, 0.0], [20e-9, 0.0, 0.0]]])
    axes = np.array([[[0.0, 1.0, 0.0], [0.0, 1.0, 0.0]]])
    cfg = W.lo_batch(origins, axes, 2 * math.pi * 200e12, 1e-11, 1e-18, n_steps, 0, q=10 * W.E_CHARGE)
    motion = W.oscillating_origins(cfg, np.array([[1e-10, 0.0]]), 2 * math.pi * 20e12)
    return cfg, motion


def test_moving_dipoles_without_motion_match_fixed_run():
    cfg, _ = _moving_cfg(300)
    still = W.oscillating_origins(cfg, 0.0, 1.0)
    a = oracle.dipoles_run(cfg)
    b = oracle.dipoles_run(cfg, motion=still)
    assert a["status"] == oracle.OK and b["status"] == oracle.OK
    for k in ("d", "d_dot", "d_ddot", "Ed"):
        assert np.array_equal(a[k], b[k]), k


def test_moving_dipole_driving_field_equals_point_charge_field():
    # the driving field of the moving run at whole steps against the generic point-charge path
    # (pinned on its own) fed with the same dipole's two charges written out as sampled trajectories
    cfg, motion = _moving_cfg(600)
    r = oracle.dipoles_run(cfg, motion=motion)
    assert r["status"] == oracle.OK
    pos, vel, acc = motion
    S = cfg.n_steps + 1
    # source the moving dipole and receiver the fixed one, then the reverse
    for src, rcv in ((0, 1), (1, 0)):
        m1, m2, q = cfg.m1[0, src], cfg.m2[0, src], cfg.q[0, src]
        u = cfg.axis[0, src]
        P, V, A = pos[0, src, ::2], vel[0, src, ::2], acc[0, src, ::2]
        cp, cv, ca = [], [], []
        for w in (m2 / (m1 + m2), -m1 / (m1 + m2)):
            cp.append(P + (w * r["d"][src] / q)[:, None] * u)
            cv.append(V + (w * r["d_dot"][src] / q)[:, None] * u)
            ca.append(A + (w * r["d_ddot"][src] / q)[:, None] * u)
        ch = W.Charges(q=np.array([q, -q]), pos=np.stack(cp), vel=np.stack(cv), acc=np.stack(ca), t0=0.0,
                       dt=cfg.dt, static_before=1)
        for n in (50, 301, 600):
            pt = pos[0, rcv, 2 * n][None]
            f = oracle.fields(pt, [n * cfg.dt], charges=ch)
            assert f["status"] == oracle.OK
            ed = float(f["E"][0, 0] @ cfg.axis[0, rcv])
            assert abs(ed - r["Ed"][rcv, n]) <= 1e-12 * abs(ed), (src, n, ed, r["Ed"][rcv, n])


# ---- point charges on analytic trajectories ----

def _par(*vals):
    p = np.zeros(12)
    flat = np.concatenate([np.atleast_1d(np.asarray(v, dtype=np.float64)) for v in vals])
    p[:flat.size] = flat
    return p


@pytest.mark.parametrize("beta", [0.1, 0.5, 0.9])
def test_param_uniform_motion_heaviside_feynman(beta):
    v = beta * W.C * np.array([0.0, 0.6, 0.8])
    r0 = np.array([0.0, -20e-9, 3e-9])
    T = 2.5e-15
    rng = np.random.default_rng(3)
    pts = r0 + T * v + rng.uniform(-60e-9, 60e-9, size=(50, 3))
    # accelerating kind with zero acceleration, clock started at t = 0
    out = oracle.fields_param(pts, [T], [3], [-W.E_CHARGE], [_par(r0, v, [0, 0, 0], 0.0)])
    assert out["status"] == oracle.OK
    E, B, phi, A = th.uniform_motion(-W.E_CHARGE, r0 + v * T, v, pts)
    assert rel(out["E"][0], E) < 1e-12
    assert rel(out["B"][0], B) < 1e-12
    assert np.max(np.abs(out["phi"][0] - phi) / np.abs(phi)) < 1e-12
    assert rel(out["A"][0], A) < 1e-12


def test_param_stationary_is_coulomb():
    pts = np.random.default_rng(4).uniform(-5e-9, 5e-9, size=(30, 3))
    out = oracle.fields_param(pts, [1e-15], [0], [W.E_CHARGE], [_par([1e-9, -2e-9, 0.5e-9])])
    E, phi = th.coulomb_static(W.E_CHARGE, [1e-9, -2e-9, 0.5e-9], pts)
    assert rel(out["E"][0], E) < 1e-13
    assert np.max(np.abs(out["phi"][0] - phi) / np.abs(phi)) < 1e-14


def test_param_oscillating_pair_is_hertzian_dipole():
    # Sec. 4.1 / App. E: +-q oscillating in antiphase, amplitude sep/2 each, d = q sep cos(w t);
    # no sampling, so only the (sep/z)^2 departure of the physical dipole remains
    w = 7e16
    q = 1e5 * W.E_CHARGE
    sep = 4e-14
    lam = 2 * math.pi * W.C / w
    zs = np.array([0.05, 0.1, 0.3, 0.7, 1.0, 1.6, 2.5]) * lam
    t_eval = 3.0 * lam / W.C + 0.37e-16
    pts = np.stack([np.zeros_like(zs), np.zeros_like(zs), zs], axis=1)
    ux = [1.0, 0.0, 0.0]
    pars = [_par([0, 0, 0], ux, sep / 2, w, 0.0), _par([0, 0, 0], ux, -sep / 2, w, 0.0)]
    out = oracle.fields_param(pts, [t_eval], [1, 1], [q, -q], pars)
    assert out["status"] == oracle.OK
    E_th, B_th = th.hertzian_dipole([q * sep, 0, 0], w, pts, t_eval)
    errE = np.linalg.norm(out["E"][0] - E_th, axis=1) / np.linalg.norm(E_th, axis=1)
    errB = np.linalg.norm(out["B"][0] - B_th, axis=1) / np.linalg.norm(B_th, axis=1)
    assert np.all(errE < 1e-9) and np.all(errB < 1e-9)


def test_param_circular_orbit_lienard_power():
    radius, beta = 1e-9, 0.1
    w = beta * W.C / radius
    r_s = 2e-4
    Tp = 2 * math.pi / w
    times = r_s / W.C + np.arange(8) * Tp / 8
    x, wq = np.polynomial.legendre.leggauss(32)
    n_ph = 32
    phis = np.arange(n_ph) * 2 * math.pi / n_ph
    st = np.sqrt(1 - x * x)
    pts = np.concatenate([np.stack([r_s * st * math.cos(p), r_s * st * math.sin(p), r_s * x], axis=1) for p in phis])
    wts = np.concatenate([wq * (2 * math.pi / n_ph) for _ in phis])
    par = _par([0, 0, 0], [1, 0, 0], [0, 1, 0], radius, w, 0.0)
    out = oracle.fields_param(pts, times, [2], [W.E_CHARGE], [par], fkind=oracle.RADIATION)
    assert out["status"] == oracle.OK
    S_ = np.cross(out["E"], out["B"]) / th.MU0
    flux = r_s ** 2 * np.sum(np.sum(S_ * (pts / r_s)[None], axis=2) * wts[None, :], axis=1)
    P = th.lienard_power_circular(W.E_CHARGE, beta * W.C, beta * W.C * w)
    assert np.max(np.abs(flux / P - 1)) < 1e-4
    # at the orbit's centre the retarded time is exactly t - radius / c
    c0 = oracle.fields_param(np.zeros((1, 3)), [times[0]], [2], [W.E_CHARGE], [par])
    tp = times[0] - radius / W.C
    p = radius * np.array([math.cos(w * tp), math.sin(w * tp), 0.0])
    v = radius * w * np.array([-math.sin(w * tp), math.cos(w * tp), 0.0])
    a = -w * w * p
    Ec, Er, _, _ = oracle.lw_jackson(W.E_CHARGE, -p, v, a)
    assert rel(c0["E"][0], (Ec + Er)[None]) < 1e-12
