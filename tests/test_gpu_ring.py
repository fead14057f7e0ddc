"""The oscillator run's history store, run states and the checkpointed adjoint (GPU, through the C ABI).

Without the full d, d', d'' outputs the run keeps its history in a ring of the context holding only
the samples a causal block can still reach (the largest delay between two dipoles plus a margin), so
its memory does not grow with the number of steps (Algorithm 1 reads the history back at retarded
times only).  A run state (the last samples and E_d at one step) resumes a run exactly; the adjoint
keeps such a state every K steps and recomputes each segment in its reverse sweep.  Checked here:
  * ring and full stores give bit-identical histories, driving fields and fits (persistent and grid
    paths, both precisions); the ring's memory is the same for 2 000 and 200 000 steps;
  * a run resumed from its state at a multiple of the causal block equals the uninterrupted run bit
    for bit, and to rounding elsewhere; foreign states are argument errors;
  * the checkpointed adjoint's gradients equal the whole-history adjoint's (energy and rate losses).
"""
import numpy as np
import pytest
import torch

import paper_2107_12437_gb300 as pc
import workloads as W
from paper_2107_12437_gb300 import capi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = pc.Context(0)
    yield c
    c.close()


def _cfgs():
    cfg3, _ = W.cfg3(B=256, n_steps=8000)
    # every 16th separation, 8 000 steps, the Eq. KE fit from step 1 000 (three kinetic-energy minima)
    sub = W.lo_batch(cfg3.origin[::16], cfg3.axis[::16], 2 * np.pi * 200e12, 1e-11, cfg3.dt, 8000, 1000)
    cloud = W.cfg5(N=96, n_steps=300, side=150e-9, min_spacing=5e-9, seed=7)
    cloud.first_index = 0
    return {"pairs": sub, "cloud": cloud}


@pytest.mark.parametrize("which", ["pairs", "cloud"])
@pytest.mark.parametrize("prec", [pc.PC_F64, pc.PC_MIXED])
def test_ring_store_matches_full_history(ctx, which, prec):
    cfg = _cfgs()[which]
    lod = pc.lo_config_to_device(cfg)
    fit = which == "pairs"
    kw = dict(precision=prec, want_Ed=True, fit=fit, first_index=cfg.first_index)
    full = pc.pc_dipoles_run(ctx, lod, cfg.dt, cfg.n_steps, **kw)
    ring = pc.pc_dipoles_run(ctx, lod, cfg.dt, cfg.n_steps, want_history=False, **kw)
    assert "d" not in ring
    for k in ("Ed",) + (("gamma", "omega") if fit else ()):
        assert torch.equal(full[k], ring[k]), k
    assert float((full["energy"] - ring["energy"]).abs().max() / full["energy"].abs().max()) < 1e-15
    # only some history outputs: the run still keeps its own ring and writes those
    B, N, S = full["d"].shape
    part = {"d": torch.empty((B, N, S), dtype=torch.float64, device="cuda")}
    pc.pc_dipoles_run(ctx, lod, cfg.dt, cfg.n_steps, precision=prec, out=part)
    assert torch.equal(part["d"], full["d"])


def test_ring_memory_does_not_grow_with_steps():
    # the population pair (80 nm apart: the ring holds 64 samples per dipole) over 2 000 and 200 000
    # steps, energies only, each in a fresh context: the device memory the run takes is the same
    cfg = W.population_pair(n_steps=200_000)
    used = []
    for n in (2000, 200_000):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        c = pc.Context(0)
        lod = pc.lo_config_to_device(cfg)
        out = pc.pc_dipoles_run(c, lod, cfg.dt, n, want_history=False, want_energy=False)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        used.append(free0 - free1 - sum(v.numel() * v.element_size() for v in out.values()))
        del out, lod
        c.close()
    assert abs(used[1] - used[0]) <= 4 << 20, used


@pytest.mark.parametrize("prec", [pc.PC_F64, pc.PC_MIXED])
def test_resume_matches_uninterrupted_run(ctx, prec):
    # grid path (96 oscillators, causal blocks of 16 steps): split at step 160 (a block boundary,
    # bit-identical) and at step 100 (inside a block: equal to rounding)
    cfg = _cfgs()["cloud"]
    lod = pc.lo_config_to_device(cfg)
    n = cfg.n_steps
    ref = pc.pc_dipoles_run(ctx, lod, cfg.dt, n, precision=prec, want_Ed=True)
    size = pc.pc_dipoles_state_size(ctx, lod, cfg.dt)
    for split, exact in ((160, True), (100, False)):
        state = torch.zeros(size, dtype=torch.float64, device="cuda")
        a = pc.pc_dipoles_run(ctx, lod, cfg.dt, split, precision=prec, want_Ed=True, state_out=state)
        b = pc.pc_dipoles_run(ctx, lod, cfg.dt, n - split, precision=prec, want_Ed=True, state_in=state)
        assert int(state[1]) == split
        for k in ("d", "d_dot", "d_ddot", "Ed", "energy"):
            got = torch.cat([a[k], b[k][..., 1:]], dim=-1)
            err = float(((got - ref[k]).abs().amax(-1) / ref[k].abs().amax(-1)).max())
            if k == "energy" and exact:
                # formed per step in the resumed run, after the run in the uninterrupted one
                assert err < 1e-15, (k, split, err)
            elif exact:
                assert torch.equal(a[k][..., -1], b[k][..., 0]), k
                assert torch.equal(got, ref[k]), (k, split)
            else:
                # inside a block the stage fields are summed in another order: float32 rounding of
                # the mixed drive, float64 rounding of the other (E_d, a sum over sources that partly
                # cancel, relative to its own largest value)
                tol = {pc.PC_F64: 1e-12, pc.PC_MIXED: 1e-6}[prec] * (1e3 if k == "Ed" else 1.0)
                assert err < tol, (k, split, err)
    # the persistent path (pairs, a block length per configuration) resumed to rounding
    cfg = _cfgs()["pairs"]
    lod = pc.lo_config_to_device(cfg)
    ref = pc.pc_dipoles_run(ctx, lod, cfg.dt, cfg.n_steps, precision=prec)
    state = torch.zeros(pc.pc_dipoles_state_size(ctx, lod, cfg.dt), dtype=torch.float64, device="cuda")
    a = pc.pc_dipoles_run(ctx, lod, cfg.dt, 4800, precision=prec, state_out=state)
    b = pc.pc_dipoles_run(ctx, lod, cfg.dt, cfg.n_steps - 4800, precision=prec, state_in=state)
    got = torch.cat([a["d"], b["d"][..., 1:]], dim=-1)
    err = float(((got - ref["d"]).abs().amax(-1) / ref["d"].abs().amax(-1)).max())
    assert err < {pc.PC_F64: 1e-12, pc.PC_MIXED: 1e-6}[prec], err


def test_foreign_states_are_argument_errors(ctx):
    cfg = _cfgs()["cloud"]
    lod = pc.lo_config_to_device(cfg)
    size = pc.pc_dipoles_state_size(ctx, lod, cfg.dt)
    state = torch.zeros(size, dtype=torch.float64, device="cuda")
    with pytest.raises(pc.PcError) as ei:  # never written: no header
        pc.pc_dipoles_run(ctx, lod, cfg.dt, 10, state_in=state)
    assert ei.value.status == capi.PC_ERR_ARG
    pc.pc_dipoles_run(ctx, lod, cfg.dt, 32, state_out=state)
    other = W.cfg5(N=80, n_steps=40, side=150e-9, min_spacing=5e-9, seed=9)
    with pytest.raises(pc.PcError) as ei:  # another number of dipoles
        pc.pc_dipoles_run(ctx, pc.lo_config_to_device(other), other.dt, 10, state_in=state)
    assert ei.value.status == capi.PC_ERR_ARG


@pytest.mark.parametrize("prec", [pc.PC_F64, pc.PC_MIXED])
def test_checkpointed_adjoint_matches_whole_history(ctx, prec):
    # gradients of sum E(T): the 256-oscillator ring over 2 400 steps and small clusters over 3 000,
    # with the state kept every 1 000 steps (rounded up to whole causal blocks) and every 77
    for cfg in (W.cfg4(n_steps=2400), W.adjoint_cluster(B=2, N=3, n_steps=3000)):
        lod = pc.lo_config_to_device(cfg)
        w = torch.ones((cfg.B, cfg.N), dtype=torch.float64, device="cuda")
        ref = pc.pc_dipoles_adjoint(ctx, lod, cfg.dt, cfg.n_steps, w, precision=prec)
        for ce in (1000, 77):
            got = pc.pc_dipoles_adjoint(ctx, lod, cfg.dt, cfg.n_steps, w, precision=prec, checkpoint_every=ce)
            for r, g_ in zip(ref, got):
                assert float((g_ - r).abs().max()) <= 1e-12 * float(r.abs().max()), ce


def test_checkpointed_rates_adjoint_matches_whole_history(ctx):
    cfg = W.adjoint_cluster(B=2, N=2, n_steps=12000, charge=20.0, first_index=2000)
    lod = pc.lo_config_to_device(cfg)
    wg = torch.ones((cfg.B, cfg.N), dtype=torch.float64, device="cuda")
    ref = pc.pc_dipoles_rates_adjoint(ctx, lod, cfg.dt, cfg.n_steps, cfg.first_index, dL_dgamma=wg)
    got = pc.pc_dipoles_rates_adjoint(ctx, lod, cfg.dt, cfg.n_steps, cfg.first_index, dL_dgamma=wg,
                                      checkpoint_every=1500)
    for r, g_ in zip(ref, got):
        assert float((g_ - r).abs().max()) <= 1e-12 * float(r.abs().max())
    # a field loss or moving origins read the whole history: no checkpointing there
    with pytest.raises(pc.PcError) as ei:
        capi_opts_field_loss(ctx, lod, cfg)
    assert ei.value.status == capi.PC_ERR_ARG


def capi_opts_field_loss(ctx, lod, cfg):
    import ctypes

    P, T = 4, 1
    pts = torch.zeros((P, 3), dtype=torch.float64, device="cuda") + 1e-7
    cE = torch.ones((cfg.B, T, P, 3), dtype=torch.float64, device="cuda")
    g = [torch.empty(s, dtype=torch.float64, device="cuda") for s in ((cfg.B, cfg.N, 3), (cfg.B, cfg.N),
                                                                       (cfg.B, cfg.N))]
    opts = capi.PcRunOpts(ed_mode=0, precision=pc.PC_F64, checkpoint_every=100)
    grads = capi.PcDipoleGrads(origin=capi._ptr(g[0]), omega0=capi._ptr(g[1]), d0=capi._ptr(g[2]))
    tarr = (ctypes.c_double * T)(1e-15)
    st = ctx.lib.pc_dipoles_fields_adjoint(ctx.handle, ctypes.byref(capi._dipoles(lod)), float(cfg.dt), 200,
                                           ctypes.byref(opts), capi._ptr(pts), P, tarr, T,
                                           ctypes.byref(capi._out_struct({"E": cE})), ctypes.byref(grads), None)
    capi._check(st, "pc_dipoles_fields_adjoint")
