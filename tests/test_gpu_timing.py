"""Launch timing of the oscillator run (pc_set_run_timing / pc_get_run_timing; GPU, through the C ABI).

A timed run launches the grid path's causal-block loop from the host with CUDA events around every
drive and RK4 launch (the untimed run replays it as one CUDA graph), and the persistent path with
one event pair around its single launch.  Checked here: the timed runs give the untimed runs'
results bit for bit; the counters count one drive and one RK4 launch per causal block (the ring of
256 oscillators, 4.9 nm apart: blocks of 16 steps) and one launch per persistent call, with positive
times; enabling clears the counters, disabling keeps them readable; bad arguments are refused.
"""
import ctypes

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


def _run(ctx, cfg, prec, n_steps):
    lod = pc.lo_config_to_device(cfg, "cuda")
    out = pc.pc_dipoles_run(ctx, lod, cfg.dt, n_steps, precision=prec, want_Ed=True)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("prec", [pc.PC_MIXED, pc.PC_F64])
def test_grid_path_timed_equals_untimed(ctx, prec):
    cfg = W.cfg4(n_steps=200)
    ref = _run(ctx, cfg, prec, 200)
    pc.pc_set_run_timing(ctx, 1)
    got = _run(ctx, cfg, prec, 200)
    t = pc.pc_get_run_timing(ctx)
    pc.pc_set_run_timing(ctx, 0)
    for k in ("d", "d_dot", "d_ddot", "energy", "Ed"):
        assert torch.equal(got[k], ref[k]), k
    # 200 steps in causal blocks of 16: 12 whole blocks and one of 8
    assert t["drive_launches"] == 13 and t["rk4_launches"] == 13
    assert t["drive_ms"] > 0.0 and t["rk4_ms"] > 0.0
    assert t["run_launches"] == 0 and t["run_ms"] == 0.0
    # disabled: the counters stay readable and do not move
    _run(ctx, cfg, prec, 64)
    assert pc.pc_get_run_timing(ctx) == t


def test_persistent_path_timed_equals_untimed(ctx):
    cfg3, _ = W.cfg3(B=256, n_steps=600)
    sub = W.lo_batch(cfg3.origin[::32], cfg3.axis[::32], 2 * np.pi * 200e12, 1e-11, cfg3.dt, 600, 100)
    ref = _run(ctx, sub, pc.PC_MIXED, 600)
    pc.pc_set_run_timing(ctx, 1)
    got = _run(ctx, sub, pc.PC_MIXED, 600)
    got2 = _run(ctx, sub, pc.PC_MIXED, 600)
    t = pc.pc_get_run_timing(ctx)
    for k in ("d", "energy", "Ed"):
        assert torch.equal(got[k], ref[k]) and torch.equal(got2[k], ref[k]), k
    assert t["run_launches"] == 2 and t["run_ms"] > 0.0
    assert t["drive_launches"] == 0 and t["rk4_launches"] == 0
    # enabling again clears the counters
    pc.pc_set_run_timing(ctx, 1)
    assert pc.pc_get_run_timing(ctx) == {"drive_launches": 0, "drive_ms": 0.0, "rk4_launches": 0, "rk4_ms": 0.0,
                                         "run_launches": 0, "run_ms": 0.0}
    pc.pc_set_run_timing(ctx, 0)


def test_timing_arguments(ctx):
    lib = capi.load()
    assert lib.pc_set_run_timing(ctx.handle, 2) == capi.PC_ERR_ARG
    assert lib.pc_set_run_timing(None, 1) == capi.PC_ERR_ARG
    assert lib.pc_get_run_timing(ctx.handle, None) == capi.PC_ERR_ARG
    t = capi.PcRunTiming()
    assert lib.pc_get_run_timing(None, ctypes.byref(t)) == capi.PC_ERR_ARG
