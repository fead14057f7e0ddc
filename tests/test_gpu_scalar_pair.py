"""The float64 driving field of fixed origins (scalar form) against the general vector form (GPU).

With fixed origins, pc_dipoles_run and pc_dipoles_adjoint evaluate a source's charges in scalar
form: every vector of the pair lies in the plane of rho = R_i - R_j and the source axis, so the
retarded-time quadratic, the interpolation and p_i . E (and their reverse) need only |rho|^2,
rho.p_j, rho.p_i and p_j.p_i.  The moving-origin entry points evaluate the same Eqs. in the general
form: each charge's position, velocity and acceleration as 3-vectors, the quadratic of solve_f64,
Griffiths' E as vectors.  With origins that do not move (amplitude 0) the two compute the same
quantities, so the histories agree to float64 rounding, and so do the adjoint gradients; the
fixed-origin gradient equals the sum of the moving run's origin-sample gradients (every sample of
the origin is R_0).  Both the persistent path (pairs) and the grid path (96 dipoles) are covered.
"""
import numpy as np
import pytest
import torch

import paper_2107_12437_gb300 as pc
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = pc.Context(0)
    yield c
    c.close()


def _cases():
    cfg3, _ = W.cfg3(B=256, n_steps=3000)
    pairs = W.lo_batch(cfg3.origin[::32], cfg3.axis[::32], 2 * np.pi * 200e12, 1e-11, cfg3.dt, 3000, 0)
    cloud = W.cfg5(N=96, n_steps=400, side=150e-9, min_spacing=5e-9, seed=7)
    return {"pairs": pairs, "cloud": cloud}


def _rel(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("name", ["pairs", "cloud"])
def test_scalar_form_matches_vector_form(ctx, name):
    cfg = _cases()[name]
    n = cfg.n_steps
    lod = pc.lo_config_to_device(cfg, "cuda")
    motion = tuple(torch.from_numpy(np.ascontiguousarray(x)).to("cuda")
                   for x in W.oscillating_origins(cfg, 0.0, 2 * np.pi * 20e12, n_steps=n))
    fixed = pc.pc_dipoles_run(ctx, lod, cfg.dt, n, precision=pc.PC_F64)
    moving = pc.pc_dipoles_run_moving(ctx, lod, motion, cfg.dt, n)
    for k in ("d", "d_dot", "d_ddot", "energy"):
        assert _rel(fixed[k], moving[k]) <= 1e-12, (k, _rel(fixed[k], moving[k]))
    w = torch.ones((cfg.B, cfg.N), dtype=torch.float64, device="cuda")
    g_origin, g_omega0, g_d0 = pc.pc_dipoles_adjoint(ctx, lod, cfg.dt, n, w)
    _, m_omega0, m_d0, m_pos, _, _ = pc.pc_dipoles_adjoint_moving(ctx, lod, motion, cfg.dt, n, w)
    assert _rel(g_omega0, m_omega0) <= 1e-9
    assert _rel(g_d0, m_d0) <= 1e-9
    assert _rel(g_origin, m_pos.sum(dim=2)) <= 1e-9
