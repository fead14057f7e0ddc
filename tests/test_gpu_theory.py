"""Decay rate and frequency shift of two coupled Lorentz oscillators from the GPU run, across all 256
separations of the batched-pairs workload (1 nm .. 1 um), for s dipoles (moments perpendicular to the
separation) and p dipoles (moments along it), against theory (Sec. 4.2 and App. A).

Each configuration starts in phase, which excites the symmetric mode only; the Eq. KE fit of a
dipole's kinetic energy gives its frequency omega and energy decay rate gamma, so that
delta_12 = omega - omega0 and gamma_+ = gamma.  Two references:
  * the exact classical pole of the pair, w^2 + i g0 w - w0^2 + (q^2 / m eps0) p.G(R, w/c).p = 0
    (oracle/theory.py), valid at every separation;
  * the Markov (Green's-function) rates of App. A, valid only where |delta_12| / omega0 << 1
    (here below 1e-4, from ~13 nm on).
Bounds (the paper's 0.2 %):
  * delta_12 within 0.2 % of the exact pole at every separation (or within 1e-5 gamma0 where the p
    shift crosses zero near 670 nm);
  * gamma_+ within 0.2 % of the exact pole from 3 nm on.  Below 3 nm the fit cannot resolve it: the
    energy decays by only gamma_+ T ~ 1e-6 over the 30 000-step window, while the shift is 4e5 .. 2.5e7
    gamma0 and the discrete model's own coupling error (linear interpolation of the partner's history
    at a retarded time 3.3 .. 10 samples back, ~(omega dt)^2 / 8 = 2e-7 relative in phase) modulates the
    envelope at that level; the oracle's own run gives fitted rates off by up to 0.5 % (s) and 22 %
    (p) at the separations tried, the GPU fits at some p separations below 1.5 nm go negative.  This
    is the workload's resolution, not the GPU (whose fits match the oracle's, test_gpu_dipoles.py);
    there the error is only recorded (bench.py, pair_theory).
"""
import numpy as np
import pytest

import paper_2107_12437_gb300 as pc
import workloads as W
from oracle import theory as th

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = pc.Context(0)
    yield c
    c.close()


def sweep(ctx, orientation, prec, near_f64=0.0):
    cfg, sep = W.cfg3(B=256, n_steps=40000, orientation=orientation)
    out = pc.pc_dipoles_run(ctx, pc.lo_config_to_device(cfg), cfg.dt, cfg.n_steps, fit=True,
                            first_index=cfg.first_index, precision=prec, near_f64=near_f64, want_energy=False)
    w0 = float(cfg.omega0[0, 0])
    m = W.M_E / 2
    g0 = th.gamma0(W.E_CHARGE, m, w0)
    d_fit = (out["omega"].cpu().numpy() - w0) / g0  # [B][2]
    g_fit = out["gamma"].cpu().numpy() / g0
    d_ex, g_ex, d_mk, g_mk = (np.zeros(cfg.B) for _ in range(4))
    for b, R in enumerate(sep):
        vec = [0.0, R, 0.0] if orientation == "s" else [R, 0.0, 0.0]
        _, dl, g = th.exact_pair_pole(vec, [1.0, 0.0, 0.0], w0, W.E_CHARGE, m)
        d_ex[b], g_ex[b] = dl / g0, g / g0
        d12, g12 = th.pair_rates(vec, [1.0, 0.0, 0.0], w0)
        d_mk[b], g_mk[b] = d12, 1.0 + g12
    return sep, w0 / g0, d_fit, g_fit, d_ex, g_ex, d_mk, g_mk


@pytest.mark.parametrize("orientation", ["s", "p"])
@pytest.mark.parametrize("prec,near", [(pc.PC_F64, 0.0), (pc.PC_MIXED, 10e-9)])
def test_pair_rates_against_theory(ctx, orientation, prec, near):
    sep, w0_g0, d_fit, g_fit, d_ex, g_ex, d_mk, g_mk = sweep(ctx, orientation, prec, near)
    far = sep >= 3e-9
    # both oscillators of a configuration see the same mode (below 3 nm the fitted decay rate is
    # discretisation-limited and the two fits differ by up to ~1e-3 of gamma0)
    assert np.allclose(d_fit[:, 0], d_fit[:, 1], rtol=1e-6, atol=1e-6)
    assert np.allclose(g_fit[far, 0], g_fit[far, 1], rtol=1e-4, atol=1e-4)
    df, gf = d_fit[:, 0], g_fit[:, 0]
    err_d = np.abs(df - d_ex)
    assert np.all((err_d <= 2e-3 * np.abs(d_ex)) | (err_d <= 1e-5)), np.max(err_d / np.abs(d_ex))
    rel_g = np.abs(gf - g_ex) / g_ex
    assert np.all(rel_g[far] <= 2e-3), float(rel_g[far].max())
    assert np.all(np.isfinite(gf[~far]))  # below 3 nm only recorded (see the module docstring)
    # App. A where the Markov approximation holds
    markov = np.abs(d_ex) / w0_g0 < 1e-4
    assert markov.sum() > 150
    err_dm = np.abs(df - d_mk)
    assert np.all(((err_dm <= 2e-3 * np.abs(d_mk)) | (err_dm <= 1e-4))[markov])
    assert np.all((np.abs(gf - g_mk) / g_mk)[markov] <= 2e-3)
    print(f"{orientation} prec={prec} near={near}: max |d-d_ex|/|d_ex| = {np.max(err_d / np.abs(d_ex)):.2e}, "
          f"max gamma rel err >= 3 nm {rel_g[far].max():.2e}, < 3 nm {rel_g[~far].max():.2e}")
