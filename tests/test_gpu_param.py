"""Point charges on analytic trajectories: pc_fields_param (CUDA, float64, through the C ABI)
against the FP64 oracle, which brackets the retarded time by bisection on the same trajectories."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2107_12437_gb300 as pc
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = pc.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("fkind", [pc.PC_TOTAL, pc.PC_COULOMB, pc.PC_RADIATION])
def test_param_fields_match_oracle(ctx, fkind):
    kind, q, par, pts = W.param_charges()
    times = [0.0, 3.3e-15, 1.7e-14]
    out = pc.pc_fields_param(ctx, kind, q, par, torch.tensor(pts, device="cuda"), times, field_kind=fkind)
    ref = oracle.fields_param(pts, times, kind, q, par, fkind=fkind)
    assert ref["status"] == oracle.OK
    # superposition scale: per-charge magnitudes summed (the scale at which any float64 sum rounds),
    # plus the conditioning of Eq. ret_t in float64: t' = t - tau carries the rounding of t, so two
    # correct evaluations differ by up to |dF_c/dt'| times a few units in the last place of t (one
    # unit moves B of the fastest orbiting charge here by 8.7e-13 of itself at t = 17 fs); dF_c/dt'
    # is taken as the central difference of the oracle in t (dt'/dt = 1/(1 - n.beta) = O(1))
    sc = {k: np.zeros(ref[k].shape[:2]) for k in ("E", "B", "A")}
    sc_phi = np.zeros(ref["phi"].shape)
    h = 1e-21
    tl = [t + h for t in times]
    tm = [t - h for t in times]
    ulps = 4.0 * np.spacing(np.abs(np.array(times)) + 1e-15)[:, None]
    for c in range(len(kind)):
        sl = slice(c, c + 1)
        r1 = oracle.fields_param(pts, times, kind[sl], q[sl], par[sl], fkind=fkind)
        rp = oracle.fields_param(pts, tl, kind[sl], q[sl], par[sl], fkind=fkind)
        rm = oracle.fields_param(pts, tm, kind[sl], q[sl], par[sl], fkind=fkind)
        for k in sc:
            sc[k] += 1e-12 * np.linalg.norm(r1[k], axis=-1)
            sc[k] += np.linalg.norm(rp[k] - rm[k], axis=-1) / (2 * h) * ulps
        sc_phi += 1e-12 * np.abs(r1["phi"]) + np.abs(rp["phi"] - rm["phi"]) / (2 * h) * ulps
    for k in ("E", "B", "A"):
        d = np.linalg.norm(out[k].cpu().numpy() - ref[k], axis=-1)
        assert np.all(d <= sc[k] + 1e-300), k
    assert np.all(np.abs(out["phi"].cpu().numpy() - ref["phi"]) <= sc_phi)
    assert not out["mask"].any()


def test_param_removes_interpolation_error(ctx):
    # the same oscillating charge as a sampled history (pc_fields, linear interpolation, Sec. 3.1)
    # differs from the analytic trajectory by O((w dt)^2); the analytic path matches the oracle
    w, amp = 2e16, 1e-9
    q = W.E_CHARGE
    par = np.zeros((1, 12))
    par[0, 3:6] = [0.0, 0.0, 1.0]
    par[0, 6], par[0, 7] = amp, w
    dt = 2e-19
    S = 40001
    tt = np.arange(S) * dt
    pos = np.zeros((1, S, 3))
    vel = np.zeros((1, S, 3))
    acc = np.zeros((1, S, 3))
    pos[0, :, 2] = amp * np.cos(w * tt)
    vel[0, :, 2] = -amp * w * np.sin(w * tt)
    acc[0, :, 2] = -amp * w * w * np.cos(w * tt)
    ch = W.Charges(q=np.array([q]), pos=pos, vel=vel, acc=acc, t0=0.0, dt=dt, static_before=1)
    pts = np.random.default_rng(2).uniform(-500e-9, 500e-9, size=(64, 3))
    t = 6e-15
    exact = oracle.fields_param(pts, [t], [1], [q], par)
    a = pc.pc_fields_param(ctx, [1], [q], par, torch.tensor(pts, device="cuda"), [t])
    s = pc.pc_fields(ctx, charges=pc.charges_to_device(ch), points=torch.tensor(pts, device="cuda"), times=[t],
                     precision=pc.PC_F64)
    ea = np.linalg.norm(a["E"].cpu().numpy() - exact["E"], axis=-1) / np.linalg.norm(exact["E"], axis=-1)
    es = np.linalg.norm(s["E"].cpu().numpy() - exact["E"], axis=-1) / np.linalg.norm(exact["E"], axis=-1)
    assert ea.max() < 1e-12
    assert es.max() > 1e3 * ea.max()  # interpolation error of the sampled history


def test_param_many_frames_and_empty(ctx):
    kind, q, par, pts = W.param_charges()
    times = list(np.linspace(0.0, 2e-14, 37))  # more frames than one launch takes
    out = pc.pc_fields_param(ctx, kind, q, par, torch.tensor(pts[:40], device="cuda"), times)
    ref = oracle.fields_param(pts[:40], times, kind, q, par)
    err = np.linalg.norm(out["E"].cpu().numpy() - ref["E"], axis=-1) / np.linalg.norm(ref["E"], axis=-1)
    assert err.max() < 1e-9
    empty = pc.pc_fields_param(ctx, kind, q, par, torch.zeros((0, 3), dtype=torch.float64, device="cuda"), times)
    assert empty["E"].shape == (37, 0, 3)
    with pytest.raises(pc.PcError):
        pc.pc_fields_param(ctx, [7], [1.0], np.zeros((1, 12)), torch.tensor(pts[:4], device="cuda"), [0.0])
