"""Population dynamics of two coupled dipoles, one initially excited (App. A, Eqs. rho_aa and
rho_bb; Sec. 4.2 population figure): the normalized energies of the CUDA oscillator run (Eq.
ne_energy) against the closed forms, and the run against the FP64 oracle over its first steps."""
import math

import numpy as np
import pytest

import oracle
import paper_2107_12437_gb300 as pc
import workloads as W
from oracle import theory as th

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = pc.Context(0)
    yield c
    c.close()


def _rates(cfg):
    q, m, w0 = cfg.q[0, 0], W.M_E / 2, cfg.omega0[0, 0]
    g0 = th.gamma0(q, m, w0)
    # exact classical poles of the symmetric and antisymmetric modes
    _, dp, gp = th.exact_pair_pole([80e-9, 0, 0], [0, 1, 0], w0, q, m, in_phase=True)
    _, dm, gm = th.exact_pair_pole([80e-9, 0, 0], [0, 1, 0], w0, q, m, in_phase=False)
    return g0, 0.5 * (gp + gm), 0.5 * (gp - gm), 0.5 * (dp - dm)


@pytest.mark.parametrize("prec", [pc.PC_F64, pc.PC_MIXED])
def test_population_beating_matches_closed_form(ctx, prec):
    # one beating period pi / delta12 (2.1e6 steps of 10 as)
    cfg = W.population_pair()
    out = pc.pc_dipoles_run(ctx, pc.lo_config_to_device(cfg), cfg.dt, cfg.n_steps, precision=prec)
    e = out["energy"][0].cpu().numpy()
    ne = th.normalized_energy(e)
    g0, gbar, g12, d12 = _rates(cfg)
    idx = np.arange(0, cfg.n_steps + 1, 5000)
    t = idx * cfg.dt
    raa, rbb = th.populations(t, gbar, g12, d12)
    assert np.max(np.abs(ne[0, idx] - raa)) < 2e-3
    assert np.max(np.abs(ne[1, idx] - rbb)) < 2e-3
    # the Markov rates of App. A describe the same beating to their own accuracy (delta12 / omega0 ~ 1e-4)
    d12m, g12m = th.s_dipole_theory(80e-9, cfg.omega0[0, 0])
    raa_m, _ = th.populations(t, g0, g12m * g0, d12m * g0)
    assert np.max(np.abs(ne[0, idx] - raa_m)) < 1e-2
    # energy moves from a to b and back: b peaks near half a beating period
    assert ne[1, idx].max() > 0.4


def test_population_run_matches_oracle(ctx):
    cfg = W.population_pair(n_steps=20000)
    ref = oracle.dipoles_run(cfg)
    assert ref["status"] == oracle.OK
    out = pc.pc_dipoles_run(ctx, pc.lo_config_to_device(cfg), cfg.dt, cfg.n_steps, precision=pc.PC_F64)
    for k in ("d", "d_dot", "energy"):
        g = out[k][0].cpu().numpy()
        assert np.max(np.abs(g - ref[k])) <= 1e-10 * np.max(np.abs(ref[k])), k
