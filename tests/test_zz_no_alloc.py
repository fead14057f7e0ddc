"""pc_fields_noalloc: the allocation-free variant of the mixed-precision field sum.

Some callers cannot allocate device memory (a framework that owns the whole device pool, a
latency-critical loop that must not call cudaMalloc); this entry point keeps its scratch in a static
device array instead of a context.  Checked through the C ABI against pc_fields (PC_MIXED) on the
same inputs, on two calls in a row with different sources, so that the second call must not see
anything the first one left in the shared array.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2107_12437_gb300 as pc
import workloads as W
from paper_2107_12437_gb300 import capi

pytestmark = pytest.mark.gpu

MIX_TOL = 1e-5  # the mixed-path tolerance of the parity tests


def _sub_dipoles(dp, sel):
    return W.Dipoles(origin=dp.origin[sel], axis=dp.axis[sel], q=dp.q[sel], m1=dp.m1[sel], m2=dp.m2[sel],
                     d=dp.d[sel], d_dot=dp.d_dot[sel], d_ddot=dp.d_ddot[sel], t0=dp.t0, dt=dp.dt)


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    num = np.abs(a - b) if a.ndim == 2 else np.linalg.norm(a - b, axis=-1)
    den = np.abs(b) if b.ndim == 2 else np.linalg.norm(b, axis=-1)
    return float(np.max(num / np.maximum(den, 1e-300)))


def test_noalloc_matches_pc_fields_twice():
    ctx = pc.Context(0)
    dp, g, z, times = W.cfg2()
    rng = np.random.default_rng(4)
    pts = W.plane_grid(g[rng.choice(2048, 37, replace=False)], g[rng.choice(2048, 29, replace=False)], z)
    ptd = torch.as_tensor(pts, device="cuda")
    calls = [(_sub_dipoles(dp, np.arange(0, 40)), [times[0], times[9]]),
             (_sub_dipoles(dp, np.arange(24, 64)), [times[5]])]
    for srcs, tsel in calls:
        dpd = pc.dipoles_to_device(srcs)
        ref = pc.pc_fields(ctx, dipoles=dpd, points=ptd, times=tsel, precision=pc.PC_MIXED)
        out = capi.alloc_field_out(ptd.shape[0], len(tsel), pc.PC_MIXED, "cuda")
        capi.pc_fields_noalloc(dipoles=dpd, points=ptd, times=tsel, out=out)
        torch.cuda.synchronize()
        assert torch.equal(out["mask"], ref["mask"])
        for k in ("E", "B", "phi", "A"):
            assert _rel(out[k], ref[k]) <= MIX_TOL, k
    ctx.close()


def test_noalloc_rejects_sources_beyond_its_scratch():
    dp, g, z, times = W.cfg2()
    # 64 dipoles x 20 000 samples need 20.5 MB of mirrors, above the 16 MiB static array
    n = 20000
    big = W.Dipoles(origin=dp.origin, axis=dp.axis, q=dp.q, m1=dp.m1, m2=dp.m2,
                    d=np.zeros((64, n)), d_dot=np.zeros((64, n)), d_ddot=np.zeros((64, n)), t0=0.0, dt=dp.dt)
    ptd = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(pc.PcError) as ei:
        capi.pc_fields_noalloc(dipoles=pc.dipoles_to_device(big), points=ptd, times=[1e-14])
    assert ei.value.status == capi.PC_ERR_ARG


def test_noalloc_point_charges_and_dipoles_many_frames():
    # point charges (the orbiting pair: their mirrors and reference positions sit after the
    # dipoles' in the static array) together with 32 dipoles, at 33 times (two launches of at most
    # 32 frames); against pc_fields (PC_MIXED) everywhere and against the oracle on a few points
    ctx = pc.Context(0)
    ch, _, _ = W.cfg1()
    dp, _, _, _ = W.cfg2()
    srcs = _sub_dipoles(dp, np.arange(32))
    g = np.linspace(-60e-9, 60e-9, 23)
    pts = np.concatenate([W.plane_grid(g, g[::3], 2e-9), W.plane_grid(g[::2] + 5e-7, g[::4] + 4e-7, 5e-7)])
    ptd = torch.as_tensor(pts, device="cuda")
    times = [float(t) for t in np.linspace(8.0e-15, 9.9e-15, 33)]
    chd, dpd = pc.charges_to_device(ch), pc.dipoles_to_device(srcs)
    ref = pc.pc_fields(ctx, charges=chd, dipoles=dpd, points=ptd, times=times, precision=pc.PC_MIXED)
    for _ in range(2):
        out = capi.alloc_field_out(ptd.shape[0], len(times), pc.PC_MIXED, "cuda")
        for v in out.values():
            v.fill_(7)
        capi.pc_fields_noalloc(charges=chd, dipoles=dpd, points=ptd, times=times, out=out)
        torch.cuda.synchronize()
        assert torch.equal(out["mask"], ref["mask"])
        for k in ("E", "B", "phi", "A"):
            assert _rel(out[k], ref[k]) <= MIX_TOL, k
    # the oracle on every 17th point at the first and the last frame: the mixed-path metric,
    # |dF| <= 1e-5 of the sum over sources of |F_j| (B at that sum of |E_j| / c)
    sel = np.arange(0, pts.shape[0], 17)
    fr = [0, 32]
    orc = oracle.fields(pts[sel], [times[f] for f in fr], charges=ch, dipoles=srcs)
    assert orc["status"] == oracle.OK
    for k in ("E", "B", "phi", "A"):
        got = out[k][fr][:, sel].double().cpu().numpy()
        num = np.abs(got - orc[k]) if got.ndim == 2 else np.linalg.norm(got - orc[k], axis=-1)
        scale = orc["scale_source"]["E"] / W.C if k == "B" else orc["scale_source"][k]
        assert float(np.max(num / scale)) <= MIX_TOL, k
    ctx.close()


def test_noalloc_rejects_outputs_and_points_it_cannot_use():
    dp, g, z, times = W.cfg2()
    dpd = pc.dipoles_to_device(_sub_dipoles(dp, np.arange(4)))
    ptd = torch.zeros((5, 3), dtype=torch.float64, device="cuda")
    # a float64 output or one of the wrong length is refused before the call
    bad = capi.alloc_field_out(5, 1, pc.PC_MIXED, "cuda")
    bad["E"] = torch.empty((1, 5, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        capi.pc_fields_noalloc(dipoles=dpd, points=ptd, times=[float(times[0])], out=bad)
    short = capi.alloc_field_out(4, 1, pc.PC_MIXED, "cuda")
    with pytest.raises(ValueError):
        capi.pc_fields_noalloc(dipoles=dpd, points=ptd, times=[float(times[0])], out=short)
    # points in host memory are an argument error of the C entry point itself
    import ctypes

    hpts = torch.zeros((5, 3), dtype=torch.float64)
    out = capi.alloc_field_out(5, 1, pc.PC_MIXED, "cuda")
    tarr = (ctypes.c_double * 1)(float(times[0]))
    st = capi.load().pc_fields_noalloc(None, ctypes.byref(capi._dipoles_struct(dpd)),
                                       ctypes.c_void_p(hpts.data_ptr()), 5, tarr, 1, pc.PC_TOTAL, 0.0,
                                       ctypes.byref(capi._out_struct(out)), None)
    assert st == capi.PC_ERR_ARG
