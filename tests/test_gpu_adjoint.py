"""Gradients of the float64 oscillator run (pc_dipoles_adjoint, CUDA through the C ABI) against
central finite differences of the GPU forward and of the FP64 oracle."""
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


def _loss_gpu(ctx, cfg, w):
    dp = pc.lo_config_to_device(cfg)
    out = pc.pc_dipoles_run(ctx, dp, cfg.dt, cfg.n_steps, precision=pc.PC_F64)
    return float((out["energy"][:, :, -1].cpu().numpy() * w).sum())


def _loss_oracle(cfg, w):
    tot = 0.0
    for b in range(cfg.B):
        r = oracle.dipoles_run(cfg, b=b)
        assert r["status"] == oracle.OK
        tot += float((r["energy"][:, -1] * w[b]).sum())
    return tot


def _perturbed(cfg, name, idx, h):
    import copy

    c = copy.deepcopy(cfg)
    getattr(c, name)[idx] += h
    return c


def _steps(cfg):
    # origins: 1e-4 of the smallest spacing (far from the history kinks, see adjoint_cluster);
    # omega0 and d0: 1e-6 relative
    return {"origin": 6e-13, "omega0": 1e-6 * float(cfg.omega0.mean()), "d0": 1e-6 * float(cfg.d0.mean())}


def _adjoint(ctx, cfg, w):
    dp = pc.lo_config_to_device(cfg)
    g = pc.pc_dipoles_adjoint(ctx, dp, cfg.dt, cfg.n_steps, torch.tensor(w, device="cuda"))
    return {k: v.cpu().numpy() for k, v in zip(("origin", "omega0", "d0"), g)}


def _check(g_adj, g_fd, tol):
    scale = np.max(np.abs(g_fd))
    assert scale > 0
    err = np.max(np.abs(g_adj - g_fd)) / scale
    assert err < tol, (err, g_adj, g_fd)


def _weights(cfg, seed=5):
    rng = np.random.default_rng(seed)
    e0 = 0.5 * (W.M_E / 2) * float(cfg.omega0.mean()) ** 2 * (1e-11) ** 2
    return rng.uniform(0.5, 1.5, size=(cfg.B, cfg.N)) / e0


def test_adjoint_vs_gpu_finite_differences(ctx):
    cfg = W.adjoint_cluster(B=2, N=3, n_steps=3000)
    w = _weights(cfg)
    g = _adjoint(ctx, cfg, w)
    hs = _steps(cfg)
    for name in ("origin", "omega0", "d0"):
        arr = getattr(cfg, name)
        fd = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            h = hs[name]
            lp = _loss_gpu(ctx, _perturbed(cfg, name, idx, h), w)
            lm = _loss_gpu(ctx, _perturbed(cfg, name, idx, -h), w)
            fd[idx] = (lp - lm) / (2 * h)
        _check(g[name], fd, 1e-5 if name != "origin" else 1e-4)


def test_adjoint_vs_oracle_finite_differences(ctx):
    cfg = W.adjoint_cluster(B=1, N=3, n_steps=1200, seed=W.SEED_ADJ + 1)
    w = _weights(cfg, seed=6)
    g = _adjoint(ctx, cfg, w)
    hs = _steps(cfg)
    for name in ("origin", "omega0", "d0"):
        arr = getattr(cfg, name)
        fd = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            h = hs[name]
            fd[idx] = (_loss_oracle(_perturbed(cfg, name, idx, h), w) -
                       _loss_oracle(_perturbed(cfg, name, idx, -h), w)) / (2 * h)
        _check(g[name], fd, 1e-5 if name != "origin" else 1e-4)


def test_isolated_dipole_gradient_closed_form(ctx):
    # a single LO decays freely: E(T) from the RK4 recurrence alone; d0 enters linearly in d(T),
    # so dE(T)/dd0 = 2 E(T)/d0 exactly
    cfg = W.adjoint_cluster(B=1, N=1, n_steps=500)
    w = np.ones((1, 1))
    g = _adjoint(ctx, cfg, w)
    out = pc.pc_dipoles_run(ctx, pc.lo_config_to_device(cfg), cfg.dt, cfg.n_steps, precision=pc.PC_F64)
    E = float(out["energy"][0, 0, -1])
    assert abs(g["d0"][0, 0] - 2 * E / cfg.d0[0, 0]) <= 1e-12 * abs(2 * E / cfg.d0[0, 0])
    assert np.all(g["origin"] == 0.0)


def test_autograd_wrapper(ctx):
    cfg = W.adjoint_cluster(B=1, N=3, n_steps=800)
    dp = pc.lo_config_to_device(cfg)
    dp.origin.requires_grad_(True)
    dp.omega0.requires_grad_(True)
    dp.d0.requires_grad_(True)
    w = torch.tensor(_weights(cfg), device="cuda")
    loss = (pc.final_energy(ctx, dp, cfg.dt, cfg.n_steps) * w).sum()
    loss.backward()
    g = _adjoint(ctx, cfg, w.cpu().numpy())
    assert np.array_equal(dp.origin.grad.cpu().numpy(), g["origin"]) or \
        np.allclose(dp.origin.grad.cpu().numpy(), g["origin"], rtol=1e-12, atol=0)
    assert np.allclose(dp.d0.grad.cpu().numpy(), g["d0"], rtol=1e-12, atol=0)


def test_adjoint_argument_errors(ctx):
    cfg = W.adjoint_cluster(B=1, N=2, n_steps=50)
    dp = pc.lo_config_to_device(cfg)
    w = torch.ones((1, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(pc.PcError):
        pc.pc_dipoles_adjoint(ctx, dp, cfg.dt, 0, w)
    with pytest.raises(pc.PcError):
        pc.pc_dipoles_adjoint(ctx, dp, -1.0, 50, w)
