"""Closed forms that pin the oracle (test infrastructure only; FP64 numpy).

Each function states the passage or the textbook result it writes out.
"""
from __future__ import annotations

import math

import numpy as np

C = 299792458.0
EPS0 = 8.8541878128e-12
MU0 = 1.0 / (EPS0 * C * C)
HBAR = 1.054571817e-34
K_E = 1.0 / (4.0 * math.pi * EPS0)


# ---------------------------------------------------------------------------------------------
# Lorentz oscillator constants (Sec. 2.3)
# ---------------------------------------------------------------------------------------------
def effective_mass(m1, m2):
    """Eq. eff_mass."""
    return m1 * m2 / (m1 + m2)


def gamma0(q, m, omega0):
    """Free-space energy decay rate of a Lorentz oscillator, Sec. 2.3: q^2 w0^2 / (6 pi eps0 c^3 m)."""
    return q * q * omega0 * omega0 / (6.0 * math.pi * EPS0 * C ** 3 * m)


def gamma0_tls(omega0, d0):
    """Eq. SE0 / App. C: w0^3 d0^2 / (3 pi eps0 hbar c^3)."""
    return omega0 ** 3 * d0 * d0 / (3.0 * math.pi * EPS0 * HBAR * C ** 3)


def isolated_lo(t, d0, omega0, g0):
    """Undriven LO d'' + g0 d' + w0^2 d = 0, d(0) = d0, d'(0) = 0 (Eq. LO_equation with E_d = 0)."""
    wd = math.sqrt(omega0 * omega0 - 0.25 * g0 * g0)
    e = np.exp(-0.5 * g0 * t)
    d = d0 * e * (np.cos(wd * t) + (0.5 * g0 / wd) * np.sin(wd * t))
    dd = d0 * e * (-(omega0 * omega0 / wd) * np.sin(wd * t))
    return d, dd


# ---------------------------------------------------------------------------------------------
# Green's function rates (App. A)
# ---------------------------------------------------------------------------------------------
def green_hom(Rvec, k):
    """Free-space dyadic Green's function of App. A for R != 0, complex k allowed.

    Reading: the mu0 in the second line of G_hom is dropped, so that Im G(R -> 0) = k^3/(6 pi) I and
    Eq. qed_gamma_ab reduces to Eq. SE0 (App. C).
    """
    Rvec = np.asarray(Rvec, dtype=np.float64)
    R = float(np.linalg.norm(Rvec))
    kR = k * R
    pref = k * k * np.exp(1j * kR) / (4.0 * math.pi * R)
    a = 1.0 + (1j * kR - 1.0) / (kR * kR)
    b = (3.0 - 3.0j * kR - kR * kR) / (kR * kR)
    RR = np.outer(Rvec, Rvec) / (R * R)
    return pref * (a * np.eye(3) + b * RR)


def pair_rates(Rvec, p_hat, omega0):
    """(delta_12 / gamma0, gamma_12 / gamma0) of two identical dipoles along p_hat, Eqs. qed_gamma_ab, qed_delta.

    gamma_12 = 2 d.Im G.d / (eps0 hbar), delta_12 = -d.Re G.d / (eps0 hbar), gamma0 from Eq. SE0 with the
    same d; the ratio is independent of |d| and hbar.
    """
    k = omega0 / C
    p = np.asarray(p_hat, dtype=np.float64)
    p = p / np.linalg.norm(p)
    d0 = 1e-29  # any moment; it cancels in the ratios
    d = d0 * p
    G = green_hom(Rvec, k)
    g12 = 2.0 * (d @ G.imag @ d) / (EPS0 * HBAR)
    dl12 = -(d @ G.real @ d) / (EPS0 * HBAR)
    g0 = gamma0_tls(omega0, d0)
    return dl12 / g0, g12 / g0


def s_dipole_theory(sep, omega0):
    """Transverse pair: moments perpendicular to the separation."""
    return pair_rates([sep, 0.0, 0.0], [0.0, 1.0, 0.0], omega0)


def p_dipole_theory(sep, omega0):
    """Longitudinal pair: moments along the separation."""
    return pair_rates([sep, 0.0, 0.0], [1.0, 0.0, 0.0], omega0)


def exact_pair_pole(Rvec, p_hat, omega0, q, m, in_phase=True):
    """Complex frequency of the symmetric (+) or antisymmetric (-) mode of two identical LOs.

    From Eq. LO_equation with a harmonic moment d e^{-i w t}; the partner's field at the origin is
    G(R, w/c) d / eps0 (App. A with App. E's time convention), so
        w^2 + i g0 w - w0^2 +- (q^2 / (m eps0)) p.G(R, w/c).p = 0.
    Solved by complex Newton from the first-order (Markov) estimate.  Returns (omega complex,
    delta = Re w - w0, gamma = -2 Im w) with delta and gamma in s^-1.
    """
    g0 = gamma0(q, m, omega0)
    p = np.asarray(p_hat, dtype=np.float64)
    p = p / np.linalg.norm(p)
    sgn = 1.0 if in_phase else -1.0
    coup = q * q / (m * EPS0)

    def F(w):
        G = green_hom(Rvec, w / C)
        return w * w + 1j * g0 * w - omega0 * omega0 + sgn * coup * (p @ G @ p)

    w = omega0 - 0.5j * g0 - sgn * coup * (p @ green_hom(Rvec, omega0 / C) @ p) / (2.0 * omega0)
    for _ in range(100):
        h = abs(w) * 1e-7
        dF = (F(w + h) - F(w - h)) / (2.0 * h)
        step = F(w) / dF
        w = w - step
        if abs(step) < 1e-15 * abs(w):
            break
    return w, w.real - omega0, -2.0 * w.imag


# ---------------------------------------------------------------------------------------------
# Textbook fields used as pins
# ---------------------------------------------------------------------------------------------
def coulomb_static(q, r_charge, points):
    """Static charge: E = q R_hat / (4 pi eps0 R^2), phi = q / (4 pi eps0 R), B = A = 0."""
    R = np.asarray(points) - np.asarray(r_charge)[None, :]
    d = np.linalg.norm(R, axis=1)
    E = K_E * q * R / d[:, None] ** 3
    phi = K_E * q / d
    return E, phi


def uniform_motion(q, r_now, v, points):
    """Charge in uniform motion (Heaviside-Feynman / Griffiths Ch. 10), from its PRESENT position r_now.

    E = q (1 - b^2) R / (4 pi eps0 R^3 (1 - b^2 sin^2 th)^{3/2}), phi = q / (4 pi eps0 R sqrt(1 - b^2 sin^2 th)),
    B = v x E / c^2, A = v phi / c^2.
    """
    v = np.asarray(v, dtype=np.float64)
    Rv = np.asarray(points) - np.asarray(r_now)[None, :]
    R = np.linalg.norm(Rv, axis=1)
    b2 = float(v @ v) / (C * C)
    vn = math.sqrt(float(v @ v))
    cos_th = (Rv @ v) / (R * vn)
    sin2 = 1.0 - cos_th * cos_th
    den = (1.0 - b2 * sin2)
    E = K_E * q * (1.0 - b2) * Rv / (R[:, None] ** 3 * den[:, None] ** 1.5)
    B = np.cross(np.broadcast_to(v, E.shape), E) / (C * C)
    phi = K_E * q / (R * np.sqrt(den))
    A = v[None, :] * phi[:, None] / (C * C)
    return E, B, phi, A


def uniform_delay(r0, v, t, points):
    """Exact delay of a charge at r0 + v t seen from points at time t: |D + v tau| = c tau, D = r - r0 - v t."""
    v = np.asarray(v, dtype=np.float64)
    D = np.asarray(points) - (np.asarray(r0) + v * t)[None, :]
    Dv = D @ v
    D2 = np.sum(D * D, axis=1)
    a = C * C - float(v @ v)
    return (Dv + np.sqrt(Dv * Dv + a * D2)) / a


def hertzian_dipole(d0_vec, omega, points, t):
    """Ideal oscillating dipole d = d0 e^{-i w t} at the origin (App. E); real parts of E and B."""
    k = omega / C
    r = np.asarray(points, dtype=np.float64)
    rn = np.linalg.norm(r, axis=1)
    rh = r / rn[:, None]
    d = np.asarray(d0_vec, dtype=np.complex128)[None, :] * np.exp(-1j * omega * t)
    ph = np.exp(1j * k * rn)[:, None]
    rxd = np.cross(rh, d)
    term1 = k * k * np.cross(rxd, rh) * ph / rn[:, None]
    rd = np.sum(rh * d, axis=1)[:, None]
    term2 = (3.0 * rd * rh - d) * (1.0 / rn ** 3 - 1j * k / rn ** 2)[:, None] * ph
    E = K_E * (term1 + term2)
    B = MU0 / (4.0 * math.pi) * C * k * k * rxd * ph / rn[:, None] * (1.0 - 1.0 / (1j * k * rn))[:, None]
    return E.real, B.real


def larmor_power(q, a2):
    """Larmor formula, Sec. 2.4: P = q^2 a^2 / (6 pi eps0 c^3)."""
    return q * q * a2 / (6.0 * math.pi * EPS0 * C ** 3)


def lienard_power_circular(q, speed, accel):
    """Lienard's generalisation for v perpendicular to a: P = q^2 gamma^4 a^2 / (6 pi eps0 c^3)."""
    g2 = 1.0 / (1.0 - (speed / C) ** 2)
    return q * q * g2 * g2 * accel * accel / (6.0 * math.pi * EPS0 * C ** 3)


def populations(t, gamma0, gamma12, delta12):
    """Excited-state populations (rho_aa, rho_bb) of two identical coupled dipoles, dipole a
    excited at t = 0 (App. A, Eqs. rho_aa and rho_bb): a quarter of the sum of the superradiant
    and subradiant decays, plus (a) or minus (b) their beating 2 cos(2 delta12 t) exp(-gamma0 t)."""
    t = np.asarray(t, dtype=np.float64)
    slow = np.exp(-(gamma0 - gamma12) * t)
    fast = np.exp(-(gamma0 + gamma12) * t)
    beat = 2.0 * np.cos(2.0 * delta12 * t) * np.exp(-gamma0 * t)
    return 0.25 * (slow + fast + beat), 0.25 * (slow + fast - beat)


def normalized_energy(energy):
    """n_e(t) = E(t) / max E over both dipoles (Eq. ne_energy), energy [N][S]."""
    e = np.asarray(energy, dtype=np.float64)
    return e / np.max(e)
