"""Moving dipoles (Sec. 4.3): pc_dipoles_run_moving (CUDA, float64 and mixed, through the C ABI)
against the FP64 oracle with the same half-step origin trajectories."""
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


def _dev(motion):
    return tuple(torch.tensor(np.ascontiguousarray(x), device="cuda") for x in motion)


def _err(g, ref):
    g = g.cpu().numpy()
    return float(np.max(np.abs(g - ref)) / np.max(np.abs(ref)))


def test_moving_pair_matches_oracle(ctx):
    origins = np.array([[[0.0, 0.0, 0.0], [20e-9, 0.0, 0.0]], [[0.0, 0.0, 0.0], [0.0, 35e-9, 0.0]]])
    axes = np.array([[[0.0, 1.0, 0.0], [0.0, 1.0, 0.0]], [[1.0, 0.0, 0.0], [1.0, 0.0, 0.0]]])
    cfg = W.lo_batch(origins, axes, 2 * math.pi * 200e12, 1e-11, 1e-18, 4000, 0, q=10 * W.E_CHARGE)
    motion = W.oscillating_origins(cfg, np.array([[1e-10, 0.0], [2e-10, 5e-11]]), 2 * math.pi * 20e12)
    out = pc.pc_dipoles_run_moving(ctx, pc.lo_config_to_device(cfg), _dev(motion), cfg.dt, cfg.n_steps, want_Ed=True)
    for b in range(cfg.B):
        ref = oracle.dipoles_run(cfg, b=b, motion=motion)
        assert ref["status"] == oracle.OK
        for k in ("d", "d_dot", "d_ddot", "energy", "Ed"):
            assert _err(out[k][b], ref[k]) < 1e-10, (b, k)
    # the motion changes the run: without it the histories differ
    still = pc.pc_dipoles_run(ctx, pc.lo_config_to_device(cfg), cfg.dt, cfg.n_steps, precision=pc.PC_F64)
    assert _err(still["d"][0], out["d"][0].cpu().numpy()) > 1e-8


def test_moving_cloud_grid_path_matches_oracle(ctx):
    # more than 64 dipoles: the grid-wide drive and graph loop with moving origins
    cfg = W.cfg5(N=80, n_steps=160, side=200e-9, min_spacing=12e-9, seed=W.SEED_CFG5 + 3)
    rng = np.random.default_rng(5)
    motion = W.oscillating_origins(cfg, rng.uniform(0.0, 2e-10, size=(1, 80)), 2 * math.pi * 30e12,
                                   direction=(1.0, 1.0, 0.0))
    out = pc.pc_dipoles_run_moving(ctx, pc.lo_config_to_device(cfg), _dev(motion), cfg.dt, cfg.n_steps, want_Ed=True)
    ref = oracle.dipoles_run(cfg, motion=motion)
    assert ref["status"] == oracle.OK
    for k in ("d", "d_dot", "Ed"):
        assert _err(out[k][0], ref[k]) < 1e-10, k


def _pair_case():
    origins = np.array([[[0.0, 0.0, 0.0], [20e-9, 0.0, 0.0]], [[0.0, 0.0, 0.0], [0.0, 35e-9, 0.0]]])
    axes = np.array([[[0.0, 1.0, 0.0], [0.0, 1.0, 0.0]], [[1.0, 0.0, 0.0], [1.0, 0.0, 0.0]]])
    cfg = W.lo_batch(origins, axes, 2 * math.pi * 200e12, 1e-11, 1e-18, 4000, 0, q=10 * W.E_CHARGE)
    motion = W.oscillating_origins(cfg, np.array([[1e-10, 0.0], [2e-10, 5e-11]]), 2 * math.pi * 20e12)
    return cfg, motion


def test_moving_mixed_pair_matches_oracle(ctx):
    # the mixed drive with moving origins (the float32 pair in difference form with the origin's
    # motion, one persistent CTA per configuration): histories and driving fields within 1e-5 of the
    # oracle's; and not the float64 run's to rounding, so the float32 pairs did run
    cfg, motion = _pair_case()
    dp = pc.lo_config_to_device(cfg)
    mx = pc.pc_dipoles_run_moving(ctx, dp, _dev(motion), cfg.dt, cfg.n_steps, want_Ed=True, precision=pc.PC_MIXED)
    f64 = pc.pc_dipoles_run_moving(ctx, dp, _dev(motion), cfg.dt, cfg.n_steps, want_Ed=True)
    for b in range(cfg.B):
        ref = oracle.dipoles_run(cfg, b=b, motion=motion)
        assert ref["status"] == oracle.OK
        for k in ("d", "d_dot", "d_ddot", "energy", "Ed"):
            assert _err(mx[k][b], ref[k]) < 1e-5, (b, k, _err(mx[k][b], ref[k]))
        assert _err(mx["Ed"][b], f64["Ed"][b].cpu().numpy()) > 1e-12


def test_moving_mixed_cloud_grid_path_matches_oracle(ctx):
    # 80 dipoles: the grid-wide mixed drive with moving origins
    cfg = W.cfg5(N=80, n_steps=400, side=200e-9, min_spacing=12e-9, seed=W.SEED_CFG5 + 3)
    rng = np.random.default_rng(5)
    motion = W.oscillating_origins(cfg, rng.uniform(0.0, 2e-10, size=(1, 80)), 2 * math.pi * 30e12,
                                   direction=(1.0, 1.0, 0.0))
    out = pc.pc_dipoles_run_moving(ctx, pc.lo_config_to_device(cfg), _dev(motion), cfg.dt, cfg.n_steps, want_Ed=True,
                                   precision=pc.PC_MIXED)
    ref = oracle.dipoles_run(cfg, motion=motion)
    assert ref["status"] == oracle.OK
    for k in ("d", "d_dot", "Ed"):
        assert _err(out[k][0], ref[k]) < 1e-5, (k, _err(out[k][0], ref[k]))


def test_moving_mixed_all_near_is_the_float64_run(ctx):
    # near_f64 beyond every distance: each source takes the float64 pair, so the mixed run is the
    # float64 run up to the order of the float64 sums
    cfg, motion = _pair_case()
    dp = pc.lo_config_to_device(cfg)
    mx = pc.pc_dipoles_run_moving(ctx, dp, _dev(motion), cfg.dt, cfg.n_steps, want_Ed=True, precision=pc.PC_MIXED,
                                  near_f64=1e-6)
    f64 = pc.pc_dipoles_run_moving(ctx, dp, _dev(motion), cfg.dt, cfg.n_steps, want_Ed=True)
    for k in ("d", "d_dot", "Ed"):
        assert _err(mx[k], f64[k].cpu().numpy()) < 1e-12, k


def _weights(cfg, seed=5):
    rng = np.random.default_rng(seed)
    e0 = 0.5 * (W.M_E / 2) * float(cfg.omega0.mean()) ** 2 * (1e-11) ** 2
    return rng.uniform(0.5, 1.5, size=(cfg.B, cfg.N)) / e0


def test_moving_adjoint_without_motion_matches_static(ctx):
    # origins that stay put: the gradient of a rigid shift of a dipole's whole trajectory (the sum
    # over its position samples) is the static adjoint's origin gradient, and omega0, d0 agree
    cfg = W.adjoint_cluster(B=2, N=3, n_steps=2000)
    motion = W.oscillating_origins(cfg, 0.0, 1e13)
    w = torch.tensor(_weights(cfg), device="cuda")
    dp = pc.lo_config_to_device(cfg)
    st = pc.pc_dipoles_adjoint(ctx, dp, cfg.dt, cfg.n_steps, w)
    mv = pc.pc_dipoles_adjoint_moving(ctx, dp, _dev(motion), cfg.dt, cfg.n_steps, w)
    assert not mv[0].any()
    shift = mv[3].sum(dim=2)
    assert float((shift - st[0]).abs().max() / st[0].abs().max()) < 1e-9
    for a, b in ((st[1], mv[1]), (st[2], mv[2])):
        assert float((a - b).abs().max() / a.abs().max()) < 1e-12
    for gv in mv[4:]:
        assert torch.isfinite(gv).all() and gv.abs().max() > 0


def test_moving_adjoint_vs_finite_differences(ctx):
    # gradients of sum w E(T) of a moving run against central differences of the GPU forward:
    # omega0 and d0 of every dipole; rigid shifts of each dipole's trajectory; and shifts of its
    # position, velocity and acceleration samples inside one time window
    cfg = W.adjoint_cluster(B=1, N=3, n_steps=2000)
    motion = W.oscillating_origins(cfg, np.array([[1e-10, 0.0, 5e-11]]), 2 * math.pi * 20e12,
                                   direction=(1.0, 0.5, 0.0))
    wn = _weights(cfg)
    w = torch.tensor(wn, device="cuda")
    g = pc.pc_dipoles_adjoint_moving(ctx, pc.lo_config_to_device(cfg), _dev(motion), cfg.dt, cfg.n_steps, w)
    g = [x.cpu().numpy() for x in g]

    def loss(c, m):
        out = pc.pc_dipoles_run_moving(ctx, pc.lo_config_to_device(c), _dev(m), c.dt, c.n_steps)
        return float((out["energy"][:, :, -1].cpu().numpy() * wn).sum())

    import copy

    def check(adj, fd, tol):
        adj, fd = np.asarray(adj), np.asarray(fd)
        scale = np.max(np.abs(fd))
        assert scale > 0
        assert np.max(np.abs(adj - fd)) / scale < tol, (adj, fd)

    for name, rel in (("omega0", 1e-6), ("d0", 1e-6)):
        fd = []
        for i in range(cfg.N):
            h = rel * float(getattr(cfg, name)[0, i])
            cp, cm = copy.deepcopy(cfg), copy.deepcopy(cfg)
            getattr(cp, name)[0, i] += h
            getattr(cm, name)[0, i] -= h
            fd.append((loss(cp, motion) - loss(cm, motion)) / (2 * h))
        check(g[1 if name == "omega0" else 2][0], fd, 1e-5)
    win = slice(1200, 1601)
    L0 = loss(cfg, motion)
    for arr, gi, h, sl in ((0, 3, 6e-13, slice(None)), (0, 3, 6e-13, win), (1, 4, None, win), (2, 5, None, win)):
        adj, fd = [], []
        if h is None:
            # velocity and acceleration samples: a step that moves the loss by ~1e-7 of itself, far
            # above its rounding and still in the linear range
            h = 1e-7 * abs(L0) / max(abs(g[gi][0, i, sl, c].sum()) for i in range(cfg.N) for c in range(3))
        for i in range(cfg.N):
            for c in range(3):
                mp = [x.copy() for x in motion]
                mm = [x.copy() for x in motion]
                mp[arr][0, i, sl, c] += h
                mm[arr][0, i, sl, c] -= h
                fd.append((loss(cfg, mp) - loss(cfg, mm)) / (2 * h))
                adj.append(g[gi][0, i, sl, c].sum())
        check(adj, fd, 1e-4)


def test_moving_adjoint_mixed_forward(ctx):
    # the forward with the mixed driving field (moving pairs in float32), the reverse in float64:
    # its gradients agree with the float64 forward's to within 1e-5 of each group's largest entry
    # (measured: 1.1e-6 on the ring's position samples over 2000 steps, 1e-9 for omega0, d0), ten
    # times inside the 1e-4 agreement with finite differences the adjoint is held to; the cluster
    # takes the one-CTA path, the ring of 256 oscillators the grid path
    cases = [(W.adjoint_cluster(B=2, N=3, n_steps=2000), 1e-10, 2 * math.pi * 20e12, (1.0, 0.5, 0.0)),
             (W.cfg4(n_steps=400), 1e-10, 2 * math.pi * 20e12, (1.0, 0.0, 0.0))]
    for cfg, amp, Om, direction in cases:
        motion = _dev(W.oscillating_origins(cfg, amp, Om, direction=direction))
        w = torch.tensor(_weights(cfg) if cfg.N < 10 else np.ones((cfg.B, cfg.N)), device="cuda")
        dp = pc.lo_config_to_device(cfg)
        g64 = pc.pc_dipoles_adjoint_moving(ctx, dp, motion, cfg.dt, cfg.n_steps, w)
        gmx = pc.pc_dipoles_adjoint_moving(ctx, dp, motion, cfg.dt, cfg.n_steps, w, precision=pc.PC_MIXED)
        for a, b in zip(g64[1:], gmx[1:]):
            scale = float(a.abs().max())
            assert scale > 0
            assert float((a - b).abs().max()) / scale < 1e-5


def test_fast_origin_matches_oracle(ctx):
    # an origin accelerating from rest toward its partner, to 2 % of c after 3000 steps: over the
    # 117-sample delay it moves by up to ~2 samples, so the retarded segment of the origin lies
    # samples away from the first guess taken at the block start; both precisions against the
    # oracle (histories within 1e-10 and 1e-5), and the mixed run's float32 pairs did run
    origins = np.array([[[0.0, 0.0, 0.0], [35e-9, 0.0, 0.0]]])
    axes = np.array([[[0.0, 1.0, 0.0], [0.0, 0.6, 0.8]]])
    n = 3000
    cfg = W.lo_batch(origins, axes, 2 * math.pi * 200e12, 1e-11, 1e-18, n, 0, q=10 * W.E_CHARGE)
    a0 = 0.02 * W.C / (n * cfg.dt)
    t = np.arange(2 * n + 1) * (cfg.dt / 2)
    u = np.array([1.0, 0.0, 0.0])
    pos = np.repeat(cfg.origin[:, :, None, :], 2 * n + 1, axis=2)
    vel, acc = np.zeros_like(pos), np.zeros_like(pos)
    pos[0, 0] += 0.5 * a0 * (t ** 2)[:, None] * u
    vel[0, 0] = a0 * t[:, None] * u
    acc[0, 0] = a0 * u
    motion = (pos, vel, acc)
    ref = oracle.dipoles_run(cfg, motion=motion)
    assert ref["status"] == oracle.OK
    dp = pc.lo_config_to_device(cfg)
    f64 = pc.pc_dipoles_run_moving(ctx, dp, _dev(motion), cfg.dt, n, want_Ed=True)
    mx = pc.pc_dipoles_run_moving(ctx, dp, _dev(motion), cfg.dt, n, want_Ed=True, precision=pc.PC_MIXED)
    for k in ("d", "d_dot", "Ed"):
        assert _err(f64[k][0], ref[k]) < 1e-10, (k, _err(f64[k][0], ref[k]))
        assert _err(mx[k][0], ref[k]) < 1e-5, (k, _err(mx[k][0], ref[k]))
    assert _err(mx["Ed"][0], f64["Ed"][0].cpu().numpy()) > 1e-12
