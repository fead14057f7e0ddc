"""Kinetic-energy fit of Eq. KE (Sec. 2.4) -- oracle side, test infrastructure only.

KE(t) = A exp(-gamma t) sin^2(omega t + phi) is fitted to the samples from first_index on
(Sec. 3.4 / Listing 2 use the values after the first 10 000 steps).  The fit is a
Levenberg-Marquardt least-squares problem (SciPy's MINPACK 'lm', as the paper's SciPy curve fit)
with an analytic Jacobian, time centred on the first fitted sample and scaled parameters
(A/A_g, gamma T, (omega - omega_g) T, phi), T the fitted time span.

Initial guess: omega_g from the spacing of the refined KE minima (zeros of sin^2), phi_g from the
first minimum, gamma_g from a straight-line fit of ln KE at its maxima, A_g from the largest sample.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import least_squares


def _refined_extrema(y, dt, kind):
    i = np.arange(1, y.size - 1)
    if kind == "min":
        sel = i[(y[i] <= y[i - 1]) & (y[i] < y[i + 1])]
    else:
        sel = i[(y[i] >= y[i - 1]) & (y[i] > y[i + 1])]
    den = y[sel - 1] - 2.0 * y[sel] + y[sel + 1]
    off = np.where(den != 0.0, 0.5 * (y[sel - 1] - y[sel + 1]) / np.where(den != 0.0, den, 1.0), 0.0)
    return (sel + off) * dt, sel


def initial_guess(y, dt):
    tmin, _ = _refined_extrema(y, dt, "min")
    tmax, imax = _refined_extrema(y, dt, "max")
    if tmin.size >= 2:
        w = math.pi * (tmin.size - 1) / (tmin[-1] - tmin[0])
        phi = (-w * tmin[0]) % math.pi
    else:
        raise ValueError("fewer than two kinetic-energy minima in the fitted window")
    if imax.size >= 2:
        slope = np.polyfit(tmax, np.log(y[imax]), 1)[0]
        g = max(-slope, 0.0)
    else:
        g = 0.0
    A = float(np.max(y)) * math.exp(g * float(tmax[np.argmax(y[imax])] if imax.size else 0.0))
    return A, g, w, phi


def ke_fit(ke, dt, first_index):
    """Fit Eq. KE to ke[first_index:] sampled every dt; returns dict(A, gamma, omega, phi, rms)."""
    y = np.asarray(ke, dtype=np.float64)[first_index:]
    tau = np.arange(y.size) * dt
    T = tau[-1]
    A_g, g_g, w_g, phi_g = initial_guess(y, dt)

    def unpack(x):
        return A_g * x[0], x[1] / T, w_g + x[2] / T, x[3]

    def res(x):
        A, g, w, ph = unpack(x)
        return (A * np.exp(-g * tau) * np.sin(w * tau + ph) ** 2 - y) / A_g

    def jac(x):
        A, g, w, ph = unpack(x)
        env = np.exp(-g * tau)
        s = np.sin(w * tau + ph)
        co = np.cos(w * tau + ph)
        J = np.empty((tau.size, 4))
        J[:, 0] = env * s * s
        J[:, 1] = -tau * A * env * s * s / T / A_g
        J[:, 2] = 2.0 * A * env * s * co * tau / T / A_g
        J[:, 3] = 2.0 * A * env * s * co / A_g
        return J

    x0 = np.array([1.0, g_g * T, 0.0, phi_g])
    sol = least_squares(res, x0, jac=jac, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=4000)
    A, g, w, ph = unpack(sol.x)
    rms = float(np.sqrt(np.mean(sol.fun ** 2)))
    return dict(A=A, gamma=g, omega=w, phi=ph, rms=rms, nfev=int(sol.nfev))
