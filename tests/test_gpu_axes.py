"""Dipole axes must be unit vectors (GPU, through the C ABI).

A dipole's charges move along its axis (Eqs. r_1, r_2), and the pair algebra of both precisions,
the float64 scalar form of the driving field included, uses p . p = 1.  An axis whose squared norm
is more than 1e-10 from 1 is an argument error of every entry point that takes dipoles: the
oscillator run (persistent and grid paths) and the field sums (both precisions, the
allocation-free one too).  Axes normalised in float64 pass.
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


def _run_status(ctx, cfg, n_steps=32, prec=pc.PC_F64):
    lod = pc.lo_config_to_device(cfg, "cuda")
    try:
        pc.pc_dipoles_run(ctx, lod, cfg.dt, n_steps, precision=prec)
        return capi.PC_OK
    except pc.PcError as e:
        return e.status


@pytest.mark.parametrize("N", [2, 96])
@pytest.mark.parametrize("prec", [pc.PC_F64, pc.PC_MIXED])
def test_run_rejects_non_unit_axis(ctx, N, prec):
    if N == 2:
        cfg, _ = W.cfg3(B=4, n_steps=32)
    else:
        cfg = W.cfg5(N=96, n_steps=32, side=150e-9, min_spacing=5e-9, seed=7)
    assert _run_status(ctx, cfg, prec=prec) == capi.PC_OK
    cfg.axis[0, 1] *= 1.001
    assert _run_status(ctx, cfg, prec=prec) == capi.PC_ERR_ARG
    # the context stays usable: the next valid call succeeds
    cfg.axis[0, 1] /= np.linalg.norm(cfg.axis[0, 1])
    assert _run_status(ctx, cfg, prec=prec) == capi.PC_OK


@pytest.mark.parametrize("prec", [pc.PC_F64, pc.PC_MIXED])
def test_fields_reject_non_unit_axis(ctx, prec):
    dp, g, z, times = W.cfg2()
    pts = torch.as_tensor(W.plane_grid(g[::256], g[::256], z), device="cuda")
    dpd = pc.dipoles_to_device(dp)
    pc.pc_fields(ctx, dipoles=dpd, points=pts, times=[float(times[0])], precision=prec)
    bad = dp.axis.copy()
    bad[3] *= 0.999
    dpd.axis = torch.as_tensor(bad, device="cuda")
    with pytest.raises(pc.PcError) as ei:
        pc.pc_fields(ctx, dipoles=dpd, points=pts, times=[float(times[0])], precision=prec)
    assert ei.value.status == capi.PC_ERR_ARG
    if prec == pc.PC_MIXED:
        with pytest.raises(pc.PcError) as ei:
            capi.pc_fields_noalloc(dipoles=dpd, points=pts, times=[float(times[0])])
        assert ei.value.status == capi.PC_ERR_ARG
