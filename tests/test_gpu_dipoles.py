"""Parity of pc_dipoles_run and pc_ke_fit (CUDA, through the C ABI) with the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2107_12437_gb300 as pc
import workloads as W
from oracle import fit, theory as th

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = pc.Context(0)
    yield c
    c.close()


def hist_err(gpu, ref):
    g = gpu.cpu().numpy() if isinstance(gpu, torch.Tensor) else gpu
    return float(np.max(np.abs(g - ref)) / np.max(np.abs(ref)))


# history tolerance (relative to the largest value) and fit tolerances per precision
HIST_TOL = {pc.PC_F64: 1e-10, pc.PC_MIXED: 1e-5}
OMEGA_TOL = {pc.PC_F64: 1e-11, pc.PC_MIXED: 1e-9}
GAMMA_TOL = {pc.PC_F64: 1e-5, pc.PC_MIXED: 1e-3}  # in units of gamma0


@pytest.fixture(scope="module")
def listing2_ref():
    cfg = W.listing2()
    ref = oracle.dipoles_run(cfg)
    assert ref["status"] == oracle.OK
    return cfg, ref


@pytest.mark.parametrize("prec", [pc.PC_F64, pc.PC_MIXED])
def test_listing2_history_and_fit(ctx, listing2_ref, prec):
    cfg, ref = listing2_ref
    out = pc.pc_dipoles_run(ctx, pc.lo_config_to_device(cfg), cfg.dt, cfg.n_steps, fit=True,
                            first_index=cfg.first_index, want_Ed=True, precision=prec)
    for k in ("d", "d_dot", "d_ddot", "energy", "Ed"):
        assert hist_err(out[k][0], ref[k]) < HIST_TOL[prec], k
    m = W.M_E / 2
    g0 = th.gamma0(W.E_CHARGE, m, cfg.omega0[0, 0])
    for i in range(2):
        ke = m * ref["d_dot"][i] ** 2 / (2 * W.E_CHARGE ** 2)
        f = fit.ke_fit(ke, cfg.dt, cfg.first_index)
        w = float(out["omega"][0, i])
        g = float(out["gamma"][0, i])
        assert abs(w - f["omega"]) / f["omega"] < OMEGA_TOL[prec]
        assert abs(g - f["gamma"]) / g0 < GAMMA_TOL[prec]
        # the paper prints delta_12 = 156.919 gamma0 for this listing
        assert round((w - cfg.omega0[0, 0]) / g0, 3) == 156.919


@pytest.fixture(scope="module")
def cfg3_sub():
    # eight separations of config 3 (1 nm .. 1 um), 12 000 steps
    cfg, sep = W.cfg3(B=256, n_steps=12000)
    sel = np.array([0, 30, 70, 110, 150, 190, 230, 255])
    sub = W.lo_batch(cfg.origin[sel], cfg.axis[sel], cfg.omega0[0, 0], 1e-11, cfg.dt, cfg.n_steps, 4000)
    refs = [oracle.dipoles_run(sub, b=b) for b in range(len(sel))]
    assert all(r["status"] == oracle.OK for r in refs)
    return sub, refs


@pytest.mark.parametrize("prec", [pc.PC_F64, pc.PC_MIXED])
def test_cfg3_subset_batched(ctx, cfg3_sub, prec):
    # all eight configurations advance in one launch (one CTA each, causal blocks of K <= 16 steps)
    sub, refs = cfg3_sub
    out = pc.pc_dipoles_run(ctx, pc.lo_config_to_device(sub), sub.dt, sub.n_steps, precision=prec)
    for b, ref in enumerate(refs):
        for k in ("d", "d_dot", "energy"):
            assert hist_err(out[k][b], ref[k]) < HIST_TOL[prec], (b, k)


def test_isolated_lo_matches_closed_form(ctx):
    # one dipole alone: E_d = 0 and d(t) is the damped oscillator of Eq. LO_equation
    dt = 1e-17
    cfg = W.lo_batch([[[0.0, 0.0, 0.0]]], [[[0.0, 0.0, 1.0]]], 2 * math.pi * 200e12, 1e-11, dt, 2000, 0)
    out = pc.pc_dipoles_run(ctx, pc.lo_config_to_device(cfg), dt, cfg.n_steps)
    t = np.arange(cfg.n_steps + 1) * dt
    g0 = th.gamma0(W.E_CHARGE, W.M_E / 2, cfg.omega0[0, 0])
    d_ex, _ = th.isolated_lo(t, cfg.d0[0, 0], cfg.omega0[0, 0], g0)
    assert hist_err(out["d"][0, 0], d_ex) < 1e-7


def test_causality_and_velocity_errors(ctx):
    origins = np.array([[[0.0, 0.0, 0.0], [0.2e-9, 0.0, 0.0]]])
    axes = np.array([[[0.0, 1.0, 0.0], [0.0, 1.0, 0.0]]])
    cfg = W.lo_batch(origins, axes, 2 * math.pi * 200e12, 1e-12, 1e-18, 10, 0)
    with pytest.raises(pc.PcError) as ei:
        pc.pc_dipoles_run(ctx, pc.lo_config_to_device(cfg), cfg.dt, cfg.n_steps)
    assert ei.value.status == pc.capi.PC_ERR_CAUSALITY
    cfg = W.lo_batch([[[0.0, 0.0, 0.0]]], [[[1.0, 0.0, 0.0]]], 2 * math.pi * 200e12, 1e-8, 1e-18, 2000, 0)
    with pytest.raises(pc.PcError) as ei:
        pc.pc_dipoles_run(ctx, pc.lo_config_to_device(cfg), cfg.dt, cfg.n_steps)
    assert ei.value.status == pc.capi.PC_ERR_VELOCITY


@pytest.mark.parametrize("prec", [pc.PC_F64, pc.PC_MIXED])
@pytest.mark.parametrize("N", [2, 80])
def test_zero_steps_and_argument_errors(ctx, prec, N):
    # n_steps = 0 (the one-CTA and the grid path): the history is the initial state alone, d0 at
    # rest, with its energy m w0^2 d0^2 / (2 q^2) (Eq. dipoleE); malformed calls are argument errors
    cfg = W.cfg5(N=N, n_steps=0, side=150e-9, min_spacing=8e-9, seed=3)
    dp = pc.lo_config_to_device(cfg)
    out = pc.pc_dipoles_run(ctx, dp, cfg.dt, 0, precision=prec)
    m = cfg.m1 * cfg.m2 / (cfg.m1 + cfg.m2)
    e0 = m * cfg.omega0 ** 2 * cfg.d0 ** 2 / (2 * cfg.q ** 2)
    assert out["d"].shape == (1, N, 1)
    assert np.array_equal(out["d"][..., 0].cpu().numpy(), cfg.d0)
    assert not out["d_dot"].any() and not out["d_ddot"].any()
    assert np.allclose(out["energy"][..., 0].cpu().numpy(), e0, rtol=1e-14, atol=0)
    for kw in (dict(ed_mode=2), dict(fit=True, first_index=0)):
        with pytest.raises(pc.PcError) as ei:
            pc.pc_dipoles_run(ctx, dp, cfg.dt, 4, precision=prec, **kw)
        assert ei.value.status == pc.capi.PC_ERR_ARG
    with pytest.raises(pc.PcError) as ei:
        pc.pc_dipoles_run(ctx, dp, -cfg.dt, 4, precision=prec)
    assert ei.value.status == pc.capi.PC_ERR_ARG
    if prec == pc.PC_MIXED:
        # 32-bit sample indices of the mixed drive: a run of 2^30 steps or more is an argument
        # error before anything is touched (the output arrays here are short)
        import ctypes

        buf = [torch.empty((1, N, 1), dtype=torch.float64, device="cuda") for _ in range(3)]
        d = pc.capi.PcDipoles(B=1, N=N, origin=pc.capi._ptr(dp.origin), axis=pc.capi._ptr(dp.axis),
                              q=pc.capi._ptr(dp.q), m1=pc.capi._ptr(dp.m1), m2=pc.capi._ptr(dp.m2),
                              omega0=pc.capi._ptr(dp.omega0), d0=pc.capi._ptr(dp.d0))
        opts = pc.capi.PcRunOpts(v_max=0.0, ed_mode=0, fit=0, first_index=0, precision=pc.PC_MIXED)
        ro = pc.capi.PcRunOut(d=pc.capi._ptr(buf[0]), d_dot=pc.capi._ptr(buf[1]), d_ddot=pc.capi._ptr(buf[2]))
        st = ctx.lib.pc_dipoles_run(ctx.handle, ctypes.byref(d), float(cfg.dt), 1 << 30, ctypes.byref(opts),
                                    ctypes.byref(ro), None)
        assert st == pc.capi.PC_ERR_ARG


@pytest.mark.parametrize("gamma", [0.0, 2e7, 3e10])
def test_ke_fit_synthetic(ctx, gamma):
    dt = 1e-18
    w = 2 * math.pi * 200e12 * (1 + 3.1e-7)
    t = np.arange(40000) * dt
    ke = 2.5e-21 * np.exp(-gamma * t) * np.sin(w * t + 0.4) ** 2
    f = fit.ke_fit(ke, dt, 10000)
    g, om, a, p = pc.pc_ke_fit(ctx, torch.as_tensor(ke[None], device="cuda"), dt, 10000)
    assert abs(float(om[0]) / w - 1) < 1e-10
    assert abs(float(g[0]) - gamma) < 1e-6 * max(gamma, 2e7)
    assert abs(float(om[0]) - f["omega"]) / w < 1e-11


@pytest.mark.parametrize("prec,near", [(pc.PC_F64, 0.0), (pc.PC_MIXED, 10e-9), (pc.PC_MIXED, 0.0)])
def test_cfg3_full_size_sampled(ctx, prec, near):
    # the launch the benchmark times: all 256 separations x 40 000 steps in one launch with the
    # Eq. KE fit; sampled separations (1 nm, 1.9 nm, 16 nm, 1 um) against the oracle run one by one.
    # The mixed drive alone resolves the decay rate of pairs closer than ~6 nm only to
    # 1e-3..0.7 gamma0 (their radiative coupling is ~(kR)^3 below the near field, under float32
    # rounding): its fitted gamma and omega are checked from 10 nm on, and with sources within
    # 10 nm summed in float64 (near_f64) at every separation
    cfg, sep = W.cfg3(B=256, n_steps=40000)
    out = pc.pc_dipoles_run(ctx, pc.lo_config_to_device(cfg), cfg.dt, cfg.n_steps, fit=True,
                            first_index=cfg.first_index, precision=prec, near_f64=near)
    m = W.M_E / 2
    g0 = th.gamma0(W.E_CHARGE, m, cfg.omega0[0, 0])
    for b in (0, 24, 100, 255):
        ref = oracle.dipoles_run(cfg, b=b)
        assert ref["status"] == oracle.OK
        for k in ("d", "d_dot", "energy"):
            assert hist_err(out[k][b], ref[k]) < HIST_TOL[prec], (b, k)
        for i in range(cfg.N):
            ke = m * ref["d_dot"][i] ** 2 / (2 * W.E_CHARGE ** 2)
            f = fit.ke_fit(ke, cfg.dt, cfg.first_index)
            if prec == pc.PC_F64 or near > 0 or float(np.ravel(sep)[b]) >= 10e-9:
                assert abs(float(out["omega"][b, i]) - f["omega"]) / f["omega"] < OMEGA_TOL[prec], (b, i)
                assert abs(float(out["gamma"][b, i]) - f["gamma"]) / g0 < GAMMA_TOL[prec], (b, i)
            else:
                # the shift itself is still resolved to 1e-6 of its size (0.16 omega0 at 1 nm)
                assert abs(float(out["omega"][b, i]) - f["omega"]) < 1e-6 * abs(f["omega"] - cfg.omega0[b, i])
    with pytest.raises(pc.PcError):
        pc.pc_dipoles_run(ctx, pc.lo_config_to_device(cfg), cfg.dt, 8, precision=prec, near_f64=-1e-9)


@pytest.mark.parametrize("prec", [pc.PC_F64, pc.PC_MIXED])
def test_cloud_full_size_first_block(ctx, prec):
    # the 4096-oscillator cloud in the benchmark's launch configuration: over its first causal
    # block (16 steps, below the 5 nm / (c dt) = 16.7-sample minimum delay) every retarded time
    # falls before t = 0, so each driving field is that of the other dipoles resting at d0 (Sec.
    # 3.2), which the oracle evaluates receiver by receiver; sampled receivers at steps 0, 8, 16
    cfg = W.cfg5(n_steps=32)
    out = pc.pc_dipoles_run(ctx, pc.lo_config_to_device(cfg), cfg.dt, cfg.n_steps, want_Ed=True, precision=prec)
    tol = {pc.PC_F64: 1e-10, pc.PC_MIXED: 1e-5}[prec]
    steps = np.array([0, 8, 16])
    for i in (0, 1234, 2900, 4095):
        others = np.arange(cfg.N) != i
        n = int(others.sum())
        dps = W.Dipoles(origin=cfg.origin[0, others], axis=cfg.axis[0, others], q=cfg.q[0, others],
                        m1=cfg.m1[0, others], m2=cfg.m2[0, others], d=np.repeat(cfg.d0[0, others, None], 2, axis=1),
                        d_dot=np.zeros((n, 2)), d_ddot=np.zeros((n, 2)), t0=0.0, dt=cfg.dt)
        ref = oracle.fields(cfg.origin[0, i][None], steps * cfg.dt, dipoles=dps)
        assert ref["status"] == oracle.OK
        ed = ref["E"][:, 0, :] @ cfg.axis[0, i]
        scale = ref["scale_source"]["E"][:, 0]
        got = out["Ed"][0, i, steps].cpu().numpy()
        assert np.all(np.abs(got - ed) <= tol * scale), (i, got, ed)
        assert np.all(np.abs(ed) > 1e-3 * scale)  # a field that does not cancel away


@pytest.mark.parametrize("prec,near", [(pc.PC_F64, 0.0), (pc.PC_MIXED, 0.0), (pc.PC_MIXED, 12e-9)])
def test_cloud_grid_path(ctx, prec, near):
    # 96 oscillators in a 150 nm cube (5 nm minimum spacing, random axes): above the size that runs
    # as one CTA per configuration, so the run takes the grid-wide drive / RK4 launches; with near
    # sources (within 12 nm) in float64
    cfg = W.cfg5(N=96, n_steps=240, side=150e-9, min_spacing=5e-9, seed=7)
    ref = oracle.dipoles_run(cfg)
    assert ref["status"] == oracle.OK
    out = pc.pc_dipoles_run(ctx, pc.lo_config_to_device(cfg), cfg.dt, cfg.n_steps, precision=prec, want_Ed=True,
                            near_f64=near)
    for k in ("d", "d_dot", "Ed"):
        assert hist_err(out[k][0], ref[k]) < HIST_TOL[prec], k


@pytest.mark.parametrize("prec", [pc.PC_F64, pc.PC_MIXED])
def test_grid_path_host_loop_matches_graph(ctx, prec, monkeypatch):
    # the causal-block loop launched from the host (one drive and one RK4 launch per block) runs the
    # same kernels in the same order as the device-side graph loop: identical results, also when
    # the last block is shorter than the others
    cfg = W.cfg5(N=96, n_steps=203, side=150e-9, min_spacing=5e-9, seed=7)
    dp = pc.lo_config_to_device(cfg)
    g = pc.pc_dipoles_run(ctx, dp, cfg.dt, cfg.n_steps, precision=prec, want_Ed=True)
    monkeypatch.setenv("PYCHARGE_GB300_HOST_LOOP", "1")
    h = pc.pc_dipoles_run(ctx, dp, cfg.dt, cfg.n_steps, precision=prec, want_Ed=True)
    for k in ("d", "d_dot", "d_ddot", "energy", "Ed"):
        assert torch.equal(g[k], h[k]), k


@pytest.mark.parametrize("prec", [pc.PC_F64, pc.PC_MIXED])
def test_frozen_field_reading_and_unequal_masses(ctx, prec):
    # E_d held at its value at t over each step (the alternative reading of Algorithm 1) and
    # dipoles with unequal charge masses, against the oracle with the same reading
    origins = np.array([[[0.0, 0.0, 0.0], [30e-9, 0.0, 0.0], [0.0, 22e-9, 9e-9]]])
    axes = np.array([[[0.0, 1.0, 0.0], [0.6, 0.8, 0.0], [0.0, 0.0, 1.0]]])
    cfg = W.lo_batch(origins, axes, 2 * math.pi * 200e12, 1e-11, 1e-18, 6000, 0, q=5 * W.E_CHARGE)
    cfg.m1[0] = W.M_E * np.array([1.0, 3.0, 1836.0])
    cfg.m2[0] = W.M_E * np.array([1.0, 0.7, 1.0])
    ref = oracle.dipoles_run(cfg, ed_mode=1)
    assert ref["status"] == oracle.OK
    out = pc.pc_dipoles_run(ctx, pc.lo_config_to_device(cfg), cfg.dt, cfg.n_steps, ed_mode=1, want_Ed=True,
                            precision=prec)
    for k in ("d", "d_dot", "d_ddot", "energy", "Ed"):
        assert hist_err(out[k][0], ref[k]) < HIST_TOL[prec], k


@pytest.mark.parametrize("prec", [pc.PC_F64, pc.PC_MIXED])
def test_cloud_full_size_past_static_block(ctx, prec):
    # The 4096-oscillator cloud in the benchmark's launch configuration (grid path: source slices per
    # receiver, the per-pair tables, the graph-captured block loop) run for 200 steps, far past the
    # first causal block: from step ~17 on the nearest sources' retarded times fall inside the run,
    # and by step 200 every source within 60 nm of a receiver is seen moving.  For sampled receivers
    # the oracle evaluates the driving field (p_i . E at the origin, every other dipole's two charges,
    # retarded time by bisection, Jackson's form) on the GPU run's own d, d', d'' history at steps
    # 20 .. 200; Ed must match within 1e-10 (float64) or 1e-5 (mixed) of the source scale
    # sum_j |E_j|, and the sample must see the sources move (Ed away from the static field).
    cfg = W.cfg5(n_steps=200)
    out = pc.pc_dipoles_run(ctx, pc.lo_config_to_device(cfg), cfg.dt, cfg.n_steps, want_Ed=True, precision=prec)
    tol = {pc.PC_F64: 1e-10, pc.PC_MIXED: 1e-5}[prec]
    hist = {k: out[k][0].cpu().numpy() for k in ("d", "d_dot", "d_ddot", "Ed")}
    org = cfg.origin[0]
    sq = np.sum(org * org, axis=1)
    d2 = sq[:, None] + sq[None, :] - 2.0 * (org @ org.T)
    np.fill_diagonal(d2, np.inf)
    nn = np.sqrt(np.maximum(d2.min(axis=1), 0.0))
    rng = np.random.default_rng(77)
    recv = np.unique(np.r_[np.argsort(nn)[:6], rng.choice(cfg.N, 6, replace=False)])
    steps = np.array([20, 40, 80, 120, 160, 200])
    moved = 0
    for i in recv:
        others = np.arange(cfg.N) != i
        sub = dict(origin=org[others], axis=cfg.axis[0, others], q=cfg.q[0, others], m1=cfg.m1[0, others],
                   m2=cfg.m2[0, others], t0=0.0, dt=cfg.dt)
        dps = W.Dipoles(d=hist["d"][others], d_dot=hist["d_dot"][others], d_ddot=hist["d_ddot"][others], **sub)
        ref = oracle.fields(org[i][None], steps * cfg.dt, dipoles=dps)
        assert ref["status"] == oracle.OK
        ed = ref["E"][:, 0, :] @ cfg.axis[0, i]
        scale = ref["scale_source"]["E"][:, 0]
        got = hist["Ed"][i, steps]
        assert np.all(np.abs(got - ed) <= tol * scale), (i, got, ed)
        # the same sources at rest (their pre-history): the run must have moved away from it
        n = int(others.sum())
        still = W.Dipoles(d=np.repeat(cfg.d0[0, others, None], 2, axis=1), d_dot=np.zeros((n, 2)),
                          d_ddot=np.zeros((n, 2)), **sub)
        st = oracle.fields(org[i][None], [steps[-1] * cfg.dt], dipoles=still)
        moved += int(abs(ed[-1] - st["E"][0, 0] @ cfg.axis[0, i]) > 1e-3 * scale[-1])
    assert moved >= len(recv) // 2


def test_cloud_mixed_against_f64():
    # Config 5 in both precisions (the mixed path against the all-float64 GPU path).
    # (1) The 4096-oscillator cloud over its first 1000 steps: total-energy trace within 1e-10 of its
    #     largest value, moment histories d, d' within 1e-7 of each dipole's peak.
    # (2) A cloud of the same density (1024 oscillators in a 378 nm cube, 5 nm minimum spacing) over
    #     6000 steps with the Eq. KE fit from step 1000: fitted omega within 1e-9 relative and gamma
    #     within 2e-3 gamma0 per dipole (at 5 nm spacing the energies beat rather than decay: the
    #     comparison is of the same fit applied to both runs).
    ctx = pc.Context(0)
    cfg = W.cfg5(n_steps=1000)
    lod = pc.lo_config_to_device(cfg)
    o = {p: pc.pc_dipoles_run(ctx, lod, cfg.dt, cfg.n_steps, precision=p) for p in (pc.PC_MIXED, pc.PC_F64)}
    m, f = o[pc.PC_MIXED], o[pc.PC_F64]
    et_m, et_f = m["energy"][0].sum(0), f["energy"][0].sum(0)
    assert float((et_m - et_f).abs().max() / et_f.abs().max()) < 1e-10
    for k in ("d", "d_dot"):
        err = ((m[k][0] - f[k][0]).abs().amax(-1) / f[k][0].abs().amax(-1)).max()
        assert float(err) < 1e-7, k
    del o, m, f
    cfg = W.cfg5(N=1024, side=378e-9, n_steps=6000)
    cfg.first_index = 1000
    lod = pc.lo_config_to_device(cfg)
    o = {p: pc.pc_dipoles_run(ctx, lod, cfg.dt, cfg.n_steps, precision=p, fit=True, first_index=cfg.first_index,
                              want_energy=False) for p in (pc.PC_MIXED, pc.PC_F64)}
    mass = cfg.m1[0] * cfg.m2[0] / (cfg.m1[0] + cfg.m2[0])
    g0 = th.gamma0(cfg.q[0], mass, cfg.omega0[0])
    gm, gf = o[pc.PC_MIXED]["gamma"][0].cpu().numpy(), o[pc.PC_F64]["gamma"][0].cpu().numpy()
    wm, wf = o[pc.PC_MIXED]["omega"][0].cpu().numpy(), o[pc.PC_F64]["omega"][0].cpu().numpy()
    assert np.all(np.isfinite(gf)) and np.all(np.isfinite(wf))
    assert float(np.max(np.abs(wm - wf) / wf)) < 1e-9
    assert float(np.max(np.abs(gm - gf) / g0)) < 2e-3
    ctx.close()


@pytest.mark.parametrize("prec", [pc.PC_F64, pc.PC_MIXED])
def test_run_tuner_and_slice_counts_keep_parity(ctx, prec):
    # the grid path's launch shape (source slices per receiver) chosen by the tuner, and every shape
    # set by hand, against the oracle on 96 oscillators; the shapes differ only in the order the
    # driving-field sum adds its terms
    cfg = W.cfg5(N=96, n_steps=240, side=150e-9, min_spacing=5e-9, seed=7)
    ref = oracle.dipoles_run(cfg)
    assert ref["status"] == oracle.OK
    lod = pc.lo_config_to_device(cfg)
    try:
        chosen = pc.pc_autotune_run(ctx, lod, cfg.dt, probe_steps=32, precision=prec)
        assert chosen in (1, 2, 4, 8, 12)
        outs = {}
        for sl in (0, 1, 2, 4, 12):
            pc.pc_set_run_tiling(ctx, sl)
            outs[sl] = pc.pc_dipoles_run(ctx, lod, cfg.dt, cfg.n_steps, precision=prec, want_Ed=True)
            for k in ("d", "d_dot", "Ed"):
                assert hist_err(outs[sl][k][0], ref[k]) < HIST_TOL[prec], (sl, k)
        for sl in (1, 2, 4, 12):
            err = float(((outs[sl]["d"] - outs[0]["d"]).abs().amax(-1) / outs[0]["d"].abs().amax(-1)).max())
            assert err < {pc.PC_F64: 1e-12, pc.PC_MIXED: 1e-6}[prec], (sl, err)
        # one CTA per configuration: nothing to tune
        small = W.cfg5(N=40, n_steps=40, side=120e-9, min_spacing=5e-9, seed=3)
        assert pc.pc_autotune_run(ctx, pc.lo_config_to_device(small), small.dt, precision=prec) == 1
        with pytest.raises(pc.PcError):
            pc.pc_set_run_tiling(ctx, 65)
    finally:
        pc.pc_set_run_tiling(ctx, 0)


def test_near_sources_match_float64():
    # separations up to 10 nm with the near sources (within 10 nm) in float64: every source of a pair
    # is near, so the mixed run's driving field is the float64 one and the run follows the float64
    # run to its rounding (moment histories within 1e-11 of their peaks, fitted omega within 1e-12
    # and gamma within 1e-5 gamma0 -- where float32 alone is off by up to 0.7 gamma0)
    ctx = pc.Context(0)
    cfg, sep = W.cfg3(B=256, n_steps=40000)
    sel = np.nonzero(sep < 9.9e-9)[0]  # clear of the 10 nm bound, which float32 distances blur
    sub = W.lo_batch(cfg.origin[sel], cfg.axis[sel], cfg.omega0[sel], 1e-11, cfg.dt, cfg.n_steps, cfg.first_index)
    assert sub.B >= 80
    lod = pc.lo_config_to_device(sub)
    kw = dict(fit=True, first_index=sub.first_index, want_energy=False)
    f = pc.pc_dipoles_run(ctx, lod, sub.dt, sub.n_steps, precision=pc.PC_F64, **kw)
    m = pc.pc_dipoles_run(ctx, lod, sub.dt, sub.n_steps, precision=pc.PC_MIXED, near_f64=10e-9, **kw)
    for k in ("d", "d_dot"):
        err = float(((m[k] - f[k]).abs().amax(-1) / f[k].abs().amax(-1)).max())
        assert err < 1e-11, (k, err)
    g0 = th.gamma0(W.E_CHARGE, W.M_E / 2, float(cfg.omega0[0, 0]))
    assert float(((m["omega"] - f["omega"]).abs() / f["omega"]).max()) < 1e-12
    assert float((m["gamma"] - f["gamma"]).abs().max()) / g0 < 1e-5
    ctx.close()
