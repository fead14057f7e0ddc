"""Benchmark of the Lienard-Wiechert field-grid hot path on GB300 (one JSON line on stdout).

Step = one pc_fields_plane call on the field-grid workload: 64 oscillating dipoles (128 charges),
2048 x 2048 plane at z = 0.5 um, 16 frames, mixed precision (float64 delays per tile, float32
pair algebra), i.e. 16 * 2048^2 * 128 = 8.59e9 retarded Lienard-Wiechert pair evaluations.
`value` = pair evaluations per second over all ranks, inputs resident in HBM.

Also reported on the same line: the plain float64 GPU path on a bounded sample of the same
workload, the batched two-oscillator run (256 separations x 40 000 RK4 steps + fit) in
dipole-steps/s, the end-to-end number through the C ABI with host buffers, the rooflines of the
field kernel and of the cloud's drive kernel, clocks sampled during the timed region and the FP64
CPU oracle on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --profile fields_mixed_small|fields_mixed2_small|fields_f64_small|lo_small|lo_f64_small|
                            ring_small|cloud_small|cloud_late|ring_moving_small|adj_small
                                                     (one small run for ncu)
Multi-GPU (torchrun, one rank per GPU): every rank evaluates its own copy of the workload
(independent problems, no data-path collective), so scaling is weak.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "LW pair evals/s & dipole-steps/s at 1 GB300, mixed vs plain FP64 GPU path"
# Algorithmic floating-point operations of one retarded pair evaluation (point, charge, time) of the
# plain per-charge method: the retarded time as the root of a quadratic on one linear history
# segment, linear interpolation of the charge's state there, and Griffiths' form of the
# Lienard-Wiechert E, B, phi, A added to the sums.  An add, subtract, multiply, divide, square root or
# reciprocal (square root) counts 1 flop; a dot product of 3-vectors 5; a fused multiply-add 2.
FLOP_TALLY = {
    "retarded time (quadratic on one segment)": {
        "a = r - p_k, D = p_k+1 - p_k, T = u - k": 7,
        "A = (c dt)^2 - D.D": 6,
        "B = a.D - (c dt)^2 T": 7,
        "C = (c dt)^2 T^2 - a.a": 8,
        "B^2 - A C": 3,
        "square root": 1,
        "root C / (sqrt - B)": 2,
    },
    "interpolation at the root": {
        "position p_k + th D": 6,
        "velocity v_k + th (v_k+1 - v_k)": 9,
        "acceleration a_k + th (a_k+1 - a_k)": 9,
        "separation r - p": 3,
    },
    "Lienard-Wiechert fields (Griffiths)": {
        "R^2, 1/R, R": 7,
        "n = a / R": 3,
        "u = c n - v": 6,
        "R u = c R - a.v": 7,
        "1 / (R u)": 1,
        "f = k q R / (R u)^3": 4,
        "g = f (c^2 - v.v)": 7,
        "velocity field g u": 3,
        "a.acc": 5,
        "radiation field f (u (a.acc) - acc (R u))": 15,
        "E +=": 3,
        "B += n x E / c": 15,
        "phi += k q c / (R u)": 2,
        "A += (phi / c^2) v": 7,
    },
}
FLOPS_PER_PAIR = sum(sum(v.values()) for v in FLOP_TALLY.values())
# The same for one charge's contribution to an oscillator's driving field at one stage time: the
# retarded time and interpolation as above, Griffiths' E alone, and its projection on the receiver's
# axis added to the sum.
DRIVE_FLOP_TALLY = {
    "retarded time (quadratic on one segment)": FLOP_TALLY["retarded time (quadratic on one segment)"],
    "interpolation at the root": FLOP_TALLY["interpolation at the root"],
    "Lienard-Wiechert E (Griffiths)": {k: v for k, v in FLOP_TALLY["Lienard-Wiechert fields (Griffiths)"].items()
                                       if not k.startswith(("E +=", "B +=", "phi +=", "A +="))},
    "projection": {"p_i . E": 5, "sum +=": 1},
}
DRIVE_FLOPS_PER_PAIR = sum(sum(v.values()) for v in DRIVE_FLOP_TALLY.values())
FP32_LANES_PER_SM = 128  # compute capability 10.x: 128 float32 FMA lanes per SM


def kernel_source_hash():
    """sha256 over the sources of the mixed field kernels (pc_fields.cu and the headers it includes)."""
    import hashlib

    h = hashlib.sha256()
    for f in ("pc_fields.cu", "pc_lw_f32.cuh", "pc_lw_f32x2.cuh", "pc_lw_f64.cuh"):
        with open(os.path.join(ROOT, "paper_2107_12437_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest value of a per-rank scalar over all ranks (the slowest rank sets the job time)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, seconds_per_rank, world, dist=None, device="cpu"):
    """Whole-job throughput of `world` replicas that each process units_per_rank: the total units
    over the slowest rank's time (weak scaling, no data-path collective)."""
    return world * units_per_rank / max_over_ranks(seconds_per_rank, dist, device)


def gpu_local_cpus(dev):
    """The host CPUs attached to the GPU's PCI device (sysfs local_cpulist), or None."""
    import torch

    try:
        pr = torch.cuda.get_device_properties(dev)
        path = "/sys/bus/pci/devices/%04x:%02x:%02x.0/local_cpulist" % (pr.pci_domain_id, pr.pci_bus_id,
                                                                       pr.pci_device_id)
        cpus = set()
        for part in open(path).read().strip().split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        return cpus & set(os.sched_getaffinity(0)) or None
    except Exception:
        return None


def max_sm_clock_mhz(gpu_index):
    """The GPU's maximum SM clock (MHz) as nvidia-smi reports it (clocks.max.sm), or None."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=30)
        return float(out.stdout.strip().splitlines()[0])
    except Exception:
        return None


def rank_info():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


# ------------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# CPU oracle legs
# ------------------------------------------------------------------------------------------------
def oracle_sample(n_side=720, threads=0):
    """The FP64 oracle on one frame of a strided n_side x n_side sub-grid of the field-grid workload."""
    import oracle

    dp, g, z, times = W.cfg2()
    idx = np.linspace(0, 2047, n_side).astype(int)
    pts = W.plane_grid(g[idx], g[idx], z)
    threads = threads or len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    r = oracle.fields(pts, times[:1], dipoles=dp, nthreads=threads)
    sec = time.perf_counter() - t0
    assert r["status"] == oracle.OK
    pairs = pts.shape[0] * 2 * dp.N
    return dict(value=pairs / sec, unit="LW pair evals/s", cores=threads, kind="oracle",
                sample=f"1 frame x {n_side}x{n_side} strided points of the 2048^2 grid x 128 charges "
                       f"({pairs:.3g} pair evals, {sec:.2f} s wall)")


def oracle_lo_sample(threads=0, n_sep=12):
    """The FP64 oracle on n_sep separations of the batched run (two coupled oscillators each) over
    all 40 000 steps, one configuration after another."""
    import oracle

    cfg, _ = W.cfg3(B=256, n_steps=40000)
    bs = np.linspace(0, cfg.B - 1, n_sep).astype(int)
    t0 = time.perf_counter()
    for b in bs:
        r = oracle.dipoles_run(cfg, b=int(b), nthreads=threads or 1)
        assert r["status"] == oracle.OK
    sec = time.perf_counter() - t0
    return dict(value=n_sep * 2 * cfg.n_steps / sec, unit="dipole-steps/s", cores=threads or 1, kind="oracle",
                sample=f"{n_sep} of the 256 separations (2 oscillators each) x 40000 steps ({sec:.1f} s wall)")


def oracle_cloud_sample(threads=0):
    """The FP64 oracle on the 4096-oscillator cloud for one RK4 step (4096 dipole-steps), all host
    cores (the receivers split across threads)."""
    import oracle

    threads = threads or len(os.sched_getaffinity(0))
    cfg = W.cfg5(n_steps=1)
    t0 = time.perf_counter()
    r = oracle.dipoles_run(cfg, n_steps=1, nthreads=threads)
    sec = time.perf_counter() - t0
    assert r["status"] == oracle.OK
    return dict(value=cfg.N / sec, unit="dipole-steps/s", cores=threads, kind="oracle",
                sample=f"4096-oscillator cloud, 1 of its 20000 steps ({sec:.1f} s wall)")


def compare_cloud(pc, ctx, dev, n_steps):
    """The 4096-oscillator cloud (600 nm cube, 5 nm minimum spacing, random axes) over n_steps in
    both precisions with the Eq. KE fit: run times, and the mixed path's total-energy trace,
    moment histories and fitted gamma, omega against the all-float64 GPU path."""
    import torch

    cfg = W.cfg5(n_steps=n_steps)
    lod = pc.lo_config_to_device(cfg, dev)
    s = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res, outs = {"workload": f"cloud: 4096 oscillators in a 600 nm cube, {n_steps} RK4 steps, fit from step "
                             f"{cfg.first_index}"}, {}
    for name, prec in (("mixed", pc.PC_MIXED), ("f64", pc.PC_F64)):
        pc.pc_dipoles_run(ctx, lod, cfg.dt, 64, precision=prec)
        torch.cuda.synchronize()
        e0.record(s)
        o = pc.pc_dipoles_run(ctx, lod, cfg.dt, n_steps, precision=prec, fit=True, first_index=cfg.first_index)
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res[name] = {"ms": ms, "dipole_steps_per_s": cfg.N * n_steps / (ms * 1e-3)}
        outs[name] = {k: o[k][0] for k in ("d", "d_dot", "energy", "gamma", "omega")}
        del o
    m, f = outs["mixed"], outs["f64"]
    et_m, et_f = m["energy"].sum(0), f["energy"].sum(0)
    mass = cfg.m1[0] * cfg.m2[0] / (cfg.m1[0] + cfg.m2[0])
    g0 = torch.as_tensor(cfg.q[0] ** 2 * cfg.omega0[0] ** 2 / (6 * math.pi * W.EPS0 * W.C ** 3 * mass), device=dev)
    w0 = torch.as_tensor(cfg.omega0[0], device=dev)
    res["mixed_over_f64"] = res["f64"]["ms"] / res["mixed"]["ms"]
    res["energy_trace_max_rel_err"] = float((et_m - et_f).abs().max() / et_f.abs().max())
    for k in ("d", "d_dot"):
        res[k + "_max_err_rel_to_peak"] = float(((m[k] - f[k]).abs().amax(-1) / f[k].abs().amax(-1)).max())
    res["gamma_max_abs_err_over_gamma0"] = float(((m["gamma"] - f["gamma"]).abs() / g0).max())
    res["omega_max_rel_err"] = float(((m["omega"] - f["omega"]).abs() / w0).max())
    res["gamma_over_gamma0_f64_range"] = [float((f["gamma"] / g0).min()), float((f["gamma"] / g0).max())]
    res["delta_omega_over_gamma0_f64_range"] = [float(((f["omega"] - w0) / g0).min()),
                                                 float(((f["omega"] - w0) / g0).max())]
    return res


def field_errors(out_mixed, out_f64, dp, g, z, times, n_per_frame=64):
    """Per-output errors of both GPU paths on a strided sample of the whole step (n_per_frame
    points in each of the 16 frames) against the binary128 oracle: plain relative error |dF| / |F|
    (max, 99th percentile, fraction above the target: 1e-10 float64, 1e-5 mixed) and, for the mixed
    path, the error over the source scale sum_j |F_j| (from the float64 oracle)."""
    import oracle

    oracle.build()
    rng = np.random.default_rng(2107)
    nfr = len(times)
    idx = np.stack([rng.choice(g.size * g.size, n_per_frame, replace=False) for _ in range(nfr)])
    step = float(g[1] - g[0])
    res = {"sample": f"{n_per_frame} random points in each of the {nfr} frames of the 2048^2 grid",
           "reference": "oracle in binary128 (fields_x)"}
    acc = {p: {k: [] for k in ("E", "B", "phi", "A")} for p in ("f64", "mixed")}
    srcs = {k: [] for k in ("E", "B", "phi", "A")}
    for f in range(nfr):
        pts = np.stack([(idx[f] // g.size) * step, (idx[f] % g.size) * step, np.full(n_per_frame, z)], axis=1)
        ref = oracle.fields_x(pts, [times[f]], dipoles=dp)
        r64 = oracle.fields(pts, [times[f]], dipoles=dp)
        for k in ("E", "B", "phi", "A"):
            den = np.abs(ref[k][0]) if ref[k].ndim == 2 else np.linalg.norm(ref[k][0], axis=-1)
            for p, o in (("f64", out_f64), ("mixed", out_mixed)):
                got = o[k][f, idx[f]].double().cpu().numpy()
                num = np.abs(got - ref[k][0]) if got.ndim == 1 else np.linalg.norm(got - ref[k][0], axis=-1)
                acc[p][k].append(np.stack([num, den], axis=1))
            srcs[k].append(r64["scale_source"]["E"][0] / W.C if k == "B" else r64["scale_source"][k][0])
    for p, tol in (("f64", 1e-10), ("mixed", 1e-5)):
        res[p] = {}
        for k in ("E", "B", "phi", "A"):
            a = np.concatenate(acc[p][k])
            rel = a[:, 0] / a[:, 1]
            e = {"plain_max": float(rel.max()), "plain_p99": float(np.percentile(rel, 99)),
                 "plain_frac_above_target": float(np.mean(rel > tol))}
            if p == "mixed":
                sc = np.concatenate(srcs[k])
                e["source_scale_max"] = float(np.max(a[:, 0] / sc))
            res[p][k] = e
    return res


def pair_theory(pc, ctx, dev):
    """The batched pairs (256 separations, 40 000 steps, Eq. KE fit) for s and p dipoles, float64 and
    mixed with near sources in float64: fitted delta_12 and gamma_+ against the exact classical pole
    of the pair (oracle/theory.py), the largest relative errors per separation range."""
    from oracle import theory as th

    res = {"reference": "exact classical pole w^2 + i g0 w - w0^2 + (q^2/m eps0) p.G(R, w/c).p = 0"}
    bands = [(1e-9, 3e-9), (3e-9, 10e-9), (10e-9, 100e-9), (100e-9, 1.01e-6)]
    for orient in ("s", "p"):
        cfg, sep = W.cfg3(B=256, n_steps=40000, orientation=orient)
        w0 = float(cfg.omega0[0, 0])
        m = W.M_E / 2
        g0 = th.gamma0(W.E_CHARGE, m, w0)
        d_ex, g_ex = np.zeros(cfg.B), np.zeros(cfg.B)
        for b, R in enumerate(sep):
            vec = [0.0, R, 0.0] if orient == "s" else [R, 0.0, 0.0]
            _, dl, g = th.exact_pair_pole(vec, [1.0, 0.0, 0.0], w0, W.E_CHARGE, m)
            d_ex[b], g_ex[b] = dl / g0, g / g0
        for name, prec, near in (("f64", pc.PC_F64, 0.0), ("mixed_near_f64", pc.PC_MIXED, 10e-9)):
            out = pc.pc_dipoles_run(ctx, pc.lo_config_to_device(cfg, dev), cfg.dt, cfg.n_steps, fit=True,
                                    first_index=cfg.first_index, precision=prec, near_f64=near, want_energy=False)
            df = (out["omega"][:, 0].cpu().numpy() - w0) / g0
            gf = out["gamma"][:, 0].cpu().numpy() / g0
            rd = np.abs(df - d_ex) / np.maximum(np.abs(d_ex), 1e-30)
            rg = np.abs(gf - g_ex) / g_ex
            res[f"{orient}_{name}"] = {
                f"{lo * 1e9:g}-{hi * 1e9:g} nm": {"delta_max_rel_err": float(rd[(sep >= lo) & (sep < hi)].max()),
                                                 "gamma_max_rel_err": float(rg[(sep >= lo) & (sep < hi)].max())}
                for lo, hi in bands}
    return res


def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    threads = len(os.sched_getaffinity(0))
    for _ in range(args.warmup):
        oracle_sample(n_side=64, threads=threads)
    vals, secs = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle_sample(n_side=96, threads=threads)
        secs.append(time.perf_counter() - t0)
        vals.append(r["value"])
    value = sum(96 * 96 * 128 for _ in secs) / sum(secs)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "LW pair evals/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / len(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "field grid: 64 oscillating dipoles (128 charges), 2048^2 plane, 16 frames; each "
                               "reference step evaluates a bounded sample: 1 frame x 96x96 strided points",
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "LW pair evals/s", "cores": threads, "kind": "oracle",
                         "sample": "1 frame x 96x96 strided points x 128 charges per step"},
        "e2e": {"value": value, "unit": "LW pair evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
# GPU legs
# ------------------------------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--profile", default=None,
                    choices=["fields_mixed_small", "fields_mixed2_small", "fields_f64_small", "lo_small",
                             "lo_f64_small", "ring_small", "cloud_small", "cloud_late", "ring_moving_small",
                             "adj_small"])
    ap.add_argument("--no-extra", action="store_true", help="skip the float64, oscillator and CPU legs")
    ap.add_argument("--compare-cloud", type=int, default=0, metavar="STEPS",
                    help="run the 4096-oscillator cloud for STEPS steps in both precisions and compare them")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch

    import paper_2107_12437_gb300 as pc

    rank, world, local = rank_info()
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    ctx = pc.Context(dev.index)
    dp, g, z, times = W.cfg2()
    step = float(g[1] - g[0])
    dpd = pc.dipoles_to_device(dp, dev)
    NU = NV = 2048
    T = len(times)
    pairs_per_step = NU * NV * T * 2 * dp.N

    if args.profile:
        if args.profile in ("fields_mixed_small", "fields_mixed2_small"):
            # 512 rows of the grid, frames 5 and 11; one point per thread (16 x 16 tiles) or two
            pc.pc_set_plane_tiling(ctx, *((16, 16) if args.profile == "fields_mixed_small" else (32, 16)))
            pc.pc_fields_plane(ctx, dipoles=dpd, origin=(0.0, 0.0, z), eu=(step, 0, 0), ev=(0, step, 0), nu=512,
                               nv=2048, times=[float(times[5]), float(times[11])], precision=pc.PC_MIXED)
        elif args.profile == "fields_f64_small":
            pc.pc_fields_plane(ctx, dipoles=dpd, origin=(0.0, 0.0, z), eu=(step, 0, 0), ev=(0, step, 0), nu=64,
                               nv=2048, times=list(times[:1]), precision=pc.PC_F64)
        elif args.profile in ("lo_small", "lo_f64_small"):
            # batched pairs, mixed or float64: one persistent launch over 2000 steps
            cfg, _ = W.cfg3(B=256, n_steps=2000)
            prec = pc.PC_MIXED if args.profile == "lo_small" else pc.PC_F64
            pc.pc_dipoles_run(ctx, pc.lo_config_to_device(cfg, dev), cfg.dt, cfg.n_steps, precision=prec)
        elif args.profile == "cloud_late":
            # the cloud past its static pre-history: 4000 steps (graph loop), the state kept, then 32
            # steps resumed from it with the block loop launched from the host; only the resumed run
            # lies inside the profiler's range (ncu --profile-from-start off)
            cfg = W.cfg5(n_steps=4000)
            lod = pc.lo_config_to_device(cfg, dev)
            pc.pc_set_run_tiling(ctx, 16)  # the slice count the tuner picks for the cloud
            st = torch.empty(pc.pc_dipoles_state_size(ctx, lod, cfg.dt), dtype=torch.float64, device=dev)
            pc.pc_dipoles_run(ctx, lod, cfg.dt, 4000, precision=pc.PC_MIXED, want_history=False, want_energy=False,
                              state_out=st)
            torch.cuda.synchronize()
            os.environ["PYCHARGE_GB300_HOST_LOOP"] = "1"
            torch.cuda.profiler.start()
            pc.pc_dipoles_run(ctx, lod, cfg.dt, 32, precision=pc.PC_MIXED, want_history=False, want_energy=False,
                              state_in=st)
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
        elif args.profile in ("ring_small", "cloud_small"):
            # grid path, mixed, block loop launched from the host so that the profiler sees every
            # launch: the 256-oscillator ring over 200 steps (13 causal blocks), or the 4096-oscillator
            # cloud over 64 steps (4 blocks)
            os.environ["PYCHARGE_GB300_HOST_LOOP"] = "1"
            cfg = W.cfg4(n_steps=200) if args.profile == "ring_small" else W.cfg5(n_steps=64)
            pc.pc_dipoles_run(ctx, pc.lo_config_to_device(cfg, dev), cfg.dt, cfg.n_steps, precision=pc.PC_MIXED)
        elif args.profile == "ring_moving_small":
            # the ring with moving origins (1e-10 m along x at 20 THz), mixed, 1600 steps (100 causal
            # blocks of 16), block loop launched from the host; from block 84 on (step 1344) every
            # source is past its static pre-history, past the ring's largest delay of 1 334 samples
            os.environ["PYCHARGE_GB300_HOST_LOOP"] = "1"
            cfg = W.cfg4(n_steps=1600)
            mot = tuple(torch.from_numpy(x).to(dev) for x in W.oscillating_origins(cfg, 1e-10, 2 * math.pi * 20e12))
            pc.pc_dipoles_run_moving(ctx, pc.lo_config_to_device(cfg, dev), mot, cfg.dt, cfg.n_steps,
                                     precision=pc.PC_MIXED)
        else:
            # adjoint of the ring's float64 run over 2000 steps (past the ring's largest delay, 1 334
            # samples, so that the last blocks, reversed first, see no source in its static
            # pre-history)
            cfg = W.cfg4(n_steps=2000)
            w = torch.ones((1, cfg.N), dtype=torch.float64, device=dev)
            pc.pc_dipoles_adjoint(ctx, pc.lo_config_to_device(cfg, dev), cfg.dt, cfg.n_steps, w)
        torch.cuda.synchronize()
        return 0

    if args.compare_cloud:
        print(json.dumps(compare_cloud(pc, ctx, dev, args.compare_cloud)), flush=True)
        ctx.close()
        return 0

    out = pc.capi.alloc_field_out(NU * NV, T, pc.PC_MIXED, dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2

    def step_fn():
        pc.pc_fields_plane(ctx, dipoles=dpd, origin=(0.0, 0.0, z), eu=(step, 0, 0), ev=(0, step, 0), nu=NU, nv=NV,
                           times=list(times), precision=pc.PC_MIXED, out=out)

    # plan: the tile shape of the mixed plane kernel, tuned on this workload before the timed steps
    tile_rows, tile_cols, tile_stage = pc.pc_autotune_plane(ctx, dipoles=dpd, origin=(0.0, 0.0, z), eu=(step, 0, 0),
                                                ev=(0, step, 0), nu=NU, nv=NV, times=list(times), out=out)
    for _ in range(args.warmup):
        step_fn()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(dev.index) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for e0, e1 in evs:
            flush.fill_(1.0)  # between steps: evict L2 (outside the timed events)
            e0.record(s)
            step_fn()
            e1.record(s)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    total_ms = max_over_ranks(sum(ms), dist, dev)
    value = whole_job_rate(pairs_per_step * args.steps, total_ms * 1e-3, world)
    # dominant kernel: fields_mixed_kernel, its average launch over the timed steps (each step's
    # events also hold the float32 mirror preparation, < 0.1 % of the step)
    kernel_ms = sum(ms) / len(ms)
    avg_ms = total_ms / args.steps

    # ---- end to end through the C ABI with host buffers ----
    # the page-locked buffers are placed (first touch) on the memory of the CPUs attached to the
    # GPU: run on those CPUs while allocating and copying, as a caller would
    cpus_all = set(os.sched_getaffinity(0))
    cpus_gpu = gpu_local_cpus(dev)
    if cpus_gpu:
        os.sched_setaffinity(0, cpus_gpu)
    host_in = {k: getattr(dp, k).copy() for k in ("origin", "axis", "q", "m1", "m2", "d", "d_dot", "d_ddot")}
    pin_in = {k: torch.from_numpy(v).pin_memory() for k, v in host_in.items()}
    pin_out = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in out.items()}
    for v in pin_out.values():
        v.zero_()  # first touch by the bound thread
    h2d = sum(v.numel() * v.element_size() for v in pin_in.values())
    d2h = sum(v.numel() * v.element_size() for v in out.values())

    def e2e_step():
        # host inputs to the device, then the library's host-output entry point: the outputs are
        # page-locked, so the kernels store the fields into host memory as they compute them
        dev_in = {k: v.to(dev, non_blocking=True) for k, v in pin_in.items()}
        from types import SimpleNamespace

        dps = SimpleNamespace(t0=dp.t0, dt=dp.dt, **dev_in)
        pc.pc_fields_plane_to_host(ctx, dipoles=dps, origin=(0.0, 0.0, z), eu=(step, 0, 0), ev=(0, step, 0), nu=NU,
                                   nv=NV, times=list(times), precision=pc.PC_MIXED, out=pin_out)
        torch.cuda.current_stream(dev).synchronize()

    e2e_step()
    n_e2e = max(2, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        e2e_step()
    e2e_sec = (time.perf_counter() - t0) / n_e2e
    e2e_value = whole_job_rate(pairs_per_step, e2e_sec, world, dist, dev)
    os.sched_setaffinity(0, cpus_all)
    del pin_out, pin_in

    # ---- roofline of the field kernel (float32 ALU) ----
    # peak = SMs x float32 FMA lanes x 2 flop x maximum SM clock, the SM count and the clock read
    # from this device; the measured FMA rate (dependent-chain kernels) is reported beside it
    fp32_fma, fp64_fma = pc.pc_alu_peaks(ctx)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = max_sm_clock_mhz(dev.index)
    clk_basis = "maximum SM clock from nvidia-smi"
    if not sm_max:
        sm_max, clk_basis = 2070.0, "maximum SM clock of the GB300 data sheet (nvidia-smi unavailable)"
    peak_tflops = 2.0 * n_sm * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12
    achieved = FLOPS_PER_PAIR * pairs_per_step / (kernel_ms * 1e-3) / 1e12
    # DRAM bytes of one full launch, scaled from an ncu capture of a smaller case; valid only while
    # the kernel sources are the ones that capture was taken of
    traffic = None
    prof = os.path.join(ROOT, "profiles", "fields_mixed_traffic.json")
    if os.path.exists(prof):
        try:
            rec = json.load(open(prof))
            if rec.get("source_sha256") == kernel_source_hash():
                traffic = rec.get("bytes_per_full_launch")
        except Exception:
            traffic = None

    line = {
        "metric": METRIC, "value": value, "unit": "LW pair evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": avg_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64 (mixed)", "data": "synthetic",
        "config": {"workload": "field grid: 64 oscillating dipoles (128 charges +-e, 1e-11 m sin(w0 t), "
                               "w0 = 2 pi 200 THz, origins in a 1 um cube, seed 2107), 2048x2048 plane at "
                               "z = 0.5 um, 16 frames t = 10 fs + f 5/16 fs, mixed precision, float32 outputs",
                   "pairs_per_step": pairs_per_step, "parallelism": f"replicas x{world}",
                   "tile": f"{tile_rows} x {tile_cols} points, {tile_rows * tile_cols // 256} per thread, "
                           f"{tile_stage} sources per shared-memory stage (autotuned)",
                   "l2": "flushed between steps (256 MB write); outputs 2.7 GB > L2"},
        # per step: the dipole-axis check, the float32 mirror of the histories, the field kernel
        # (all 16 frames in one launch)
        "gpu_launches": 3 * args.steps,
        "clocks": clk.summary(),
        "e2e": {"value": e2e_value, "unit": "LW pair evals/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "host_cpus": f"{len(cpus_gpu)} GPU-local" if cpus_gpu else "unbound"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": traffic,
                     "kernel": "fields_mixed2_kernel" if tile_rows * tile_cols > 256 else "fields_mixed_kernel",
                     "flops_per_pair": FLOPS_PER_PAIR,
                     "flops_per_pair_basis": "itemized tally of the per-charge method (bench.FLOP_TALLY)",
                     "peak_basis": f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {sm_max:.0f} MHz "
                                   f"({clk_basis})",
                     "measured_fp32_fma_per_s": fp32_fma, "measured_fp64_fma_per_s": fp64_fma,
                     "frac_of_measured_fp32_fma": achieved * 1e12 / (2.0 * fp32_fma)},
    }

    if not args.no_extra:
        # the plain float64 GPU path on the whole step (2048 x 2048 plane, 16 frames): one untimed
        # call, then one timed
        out64 = pc.capi.alloc_field_out(NU * NV, T, pc.PC_F64, dev)

        def f64_step():
            pc.pc_fields_plane(ctx, dipoles=dpd, origin=(0.0, 0.0, z), eu=(step, 0, 0), ev=(0, step, 0), nu=NU,
                               nv=NV, times=list(times), precision=pc.PC_F64, out=out64)

        f64_step()
        torch.cuda.synchronize()
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        f64_step()
        e1.record(s)
        torch.cuda.synchronize()
        f64_ms = e0.elapsed_time(e1)
        f64_value = pairs_per_step / (f64_ms * 1e-3)
        line["fp64_path"] = {"value": f64_value, "unit": "LW pair evals/s", "ms": f64_ms,
                             "sample": "the whole step (2048 x 2048 x 16 frames), float64 path",
                             "mixed_over_fp64": value / world / f64_value,
                             "roofline": {"bound": "alu", "achieved": FLOPS_PER_PAIR * f64_value / 1e12,
                                          "peak": 2.0 * fp64_fma / 1e12, "unit": "TFLOP/s",
                                          "frac": FLOPS_PER_PAIR * f64_value / (2.0 * fp64_fma),
                                          "peak_basis": "measured float64 FMA rate (pc_alu_peaks)"}}
        if rank == 0:
            line["errors"] = field_errors(out, out64, dp, g, z, times)
        del out64
        # oscillator runs: dipole-steps per second (float64 RK4 state; driving field per precision)
        def lo_time(cfg, n_steps, prec, fit, near_f64=0.0):
            lod = pc.lo_config_to_device(cfg, dev)
            pc.pc_dipoles_run(ctx, lod, cfg.dt, min(n_steps, 64), precision=prec, near_f64=near_f64)
            torch.cuda.synchronize()
            e0.record(s)
            pc.pc_dipoles_run(ctx, lod, cfg.dt, n_steps, precision=prec, fit=fit, first_index=cfg.first_index,
                              near_f64=near_f64)
            e1.record(s)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            return {"value": cfg.B * cfg.N * n_steps / (ms * 1e-3), "unit": "dipole-steps/s", "ms": ms}

        cfg3, _ = W.cfg3(B=256, n_steps=40000)
        ds = {}
        for name, prec in (("mixed", pc.PC_MIXED), ("f64", pc.PC_F64)):
            r = lo_time(cfg3, cfg3.n_steps, prec, False)
            r["workload"] = ("batched pairs: 256 separations (1 nm .. 1 um) x 2 oscillators x 40000 RK4 steps, "
                             "one launch")
            ds["pairs_" + name] = r
        r = lo_time(cfg3, cfg3.n_steps, pc.PC_MIXED, False, near_f64=10e-9)
        r["workload"] = ("the same, mixed with the sources within 10 nm summed in float64 (decay rates of the "
                         "closest pairs resolved)")
        ds["pairs_mixed_near_f64"] = r
        # latency floor of the batch: its slowest configuration (1 nm, causal blocks of 3 steps,
        # 13 334 blocks) run alone; the batch's time per block against that chain's
        one = W.lo_batch(cfg3.origin[:1], cfg3.axis[:1], cfg3.omega0[:1], 1e-11, cfg3.dt, cfg3.n_steps,
                         cfg3.first_index)
        nblk = -(-cfg3.n_steps // 3)
        for name, prec in (("mixed", pc.PC_MIXED), ("f64", pc.PC_F64)):
            r1 = lo_time(one, one.n_steps, prec, False)
            ds["pairs_latency_" + name] = {
                "closest_alone_ms": r1["ms"], "us_per_block_alone": 1e3 * r1["ms"] / nblk,
                "us_per_block_batch": 1e3 * ds["pairs_" + name]["ms"] / nblk,
                "batch_over_floor": ds["pairs_" + name]["ms"] / r1["ms"],
                "workload": "the 1 nm configuration alone: 13334 causal blocks of 3 steps, one CTA"}
        if rank == 0:
            line["pair_theory"] = pair_theory(pc, ctx, dev)
        # the Eq. KE fit of all 512 kinetic-energy series of that run (30 001 samples each)
        lod = pc.lo_config_to_device(cfg3, dev)
        out3 = pc.pc_dipoles_run(ctx, lod, cfg3.dt, cfg3.n_steps, precision=pc.PC_MIXED)
        m3 = lod.m1 * lod.m2 / (lod.m1 + lod.m2)
        ke = (m3[..., None] * out3["d_dot"] ** 2 / (2 * lod.q[..., None] ** 2)).reshape(cfg3.B * cfg3.N, -1)
        pc.pc_ke_fit(ctx, ke, cfg3.dt, cfg3.first_index)
        torch.cuda.synchronize()
        e0.record(s)
        pc.pc_ke_fit(ctx, ke, cfg3.dt, cfg3.first_index)
        e1.record(s)
        torch.cuda.synchronize()
        ds["ke_fit"] = {"value": cfg3.B * cfg3.N / (e0.elapsed_time(e1) * 1e-3), "unit": "series/s",
                        "ms": e0.elapsed_time(e1), "workload": "512 kinetic-energy series x 30001 samples"}
        del out3, ke
        # ring of 256 oscillators (200 nm radius, omega0 +-1 %), 20 000 steps: forward in both
        # precisions, and the float64 adjoint of sum E(T) (forward repeated inside, then reverse)
        cfg4 = W.cfg4()
        for name, prec in (("mixed", pc.PC_MIXED), ("f64", pc.PC_F64)):
            # the grid path's launch shape tuned on this workload first (source slices per receiver)
            sl = pc.pc_autotune_run(ctx, pc.lo_config_to_device(cfg4, dev), cfg4.dt, probe_steps=256, precision=prec)
            r = lo_time(cfg4, cfg4.n_steps, prec, False)
            r["workload"] = "ring: 256 oscillators on a 200 nm ring x 20000 RK4 steps"
            r["source_slices"] = sl
            ds["ring_" + name] = r
        pc.pc_set_run_tiling(ctx, 0)
        lod4 = pc.lo_config_to_device(cfg4, dev)
        w4 = torch.ones((1, cfg4.N), dtype=torch.float64, device=dev)
        pc.pc_dipoles_adjoint(ctx, lod4, cfg4.dt, 64, w4)
        torch.cuda.synchronize()
        e0.record(s)
        pc.pc_dipoles_adjoint(ctx, lod4, cfg4.dt, cfg4.n_steps, w4)
        e1.record(s)
        torch.cuda.synchronize()
        ms4 = e0.elapsed_time(e1)
        ds["ring_adjoint_f64"] = {"value": cfg4.N * cfg4.n_steps / (ms4 * 1e-3), "unit": "dipole-steps/s", "ms": ms4,
                                  "workload": "gradients of sum E(T) w.r.t. 768 origin coordinates, 256 omega0, "
                                              "256 d0 of the 256-oscillator ring, 20000 steps (forward + reverse)"}
        # the same gradients with the run's state kept every 1000 steps and each segment recomputed
        # in the reverse sweep (memory: the states plus one segment, not the whole history)
        pc.pc_dipoles_adjoint(ctx, lod4, cfg4.dt, 64, w4, checkpoint_every=1000)
        torch.cuda.synchronize()
        e0.record(s)
        pc.pc_dipoles_adjoint(ctx, lod4, cfg4.dt, cfg4.n_steps, w4, checkpoint_every=1000)
        e1.record(s)
        torch.cuda.synchronize()
        ms4c = e0.elapsed_time(e1)
        ds["ring_adjoint_f64_checkpointed"] = {
            "value": cfg4.N * cfg4.n_steps / (ms4c * 1e-3), "unit": "dipole-steps/s", "ms": ms4c,
            "workload": "the same gradients, the run's state kept every 1000 steps (1008: whole causal blocks), "
                        "each segment recomputed in the reverse sweep"}
        pc.pc_dipoles_adjoint(ctx, lod4, cfg4.dt, 64, w4, precision=pc.PC_MIXED)
        torch.cuda.synchronize()
        e0.record(s)
        pc.pc_dipoles_adjoint(ctx, lod4, cfg4.dt, cfg4.n_steps, w4, precision=pc.PC_MIXED)
        e1.record(s)
        torch.cuda.synchronize()
        ms4m = e0.elapsed_time(e1)
        ds["ring_adjoint_mixed_forward"] = {"value": cfg4.N * cfg4.n_steps / (ms4m * 1e-3), "unit": "dipole-steps/s",
                                            "ms": ms4m, "workload": "the same gradients with the forward run's "
                                                                    "driving field mixed, the reverse float64"}
        cfg5 = W.cfg5()
        sl = pc.pc_autotune_run(ctx, pc.lo_config_to_device(cfg5, dev), cfg5.dt, probe_steps=64, precision=pc.PC_MIXED)
        r = lo_time(cfg5, cfg5.n_steps, pc.PC_MIXED, False)
        r["workload"] = "cloud: 4096 oscillators in a 600 nm cube x 20000 RK4 steps (1250 causal blocks of 16 steps)"
        r["source_slices"] = sl
        ds["cloud_mixed"] = r
        # the cloud's dominant kernel, the grid-path drive, against the float32 roofline: 4000 steps to
        # a state (past the static pre-history of most pairs), then 100 causal blocks resumed from it
        # with every launch timed by the library (pc_set_run_timing: CUDA events on the run's stream)
        lod5 = pc.lo_config_to_device(cfg5, dev)
        st5 = torch.empty(pc.pc_dipoles_state_size(ctx, lod5, cfg5.dt), dtype=torch.float64, device=dev)
        pc.pc_dipoles_run(ctx, lod5, cfg5.dt, 4000, precision=pc.PC_MIXED, want_history=False, want_energy=False,
                          state_out=st5)
        pc.pc_set_run_timing(ctx, 1)
        pc.pc_dipoles_run(ctx, lod5, cfg5.dt, 1600, precision=pc.PC_MIXED, want_history=False, want_energy=False,
                          state_in=st5)
        tm = pc.pc_get_run_timing(ctx)
        pc.pc_set_run_timing(ctx, 0)
        del st5
        drive_ms = tm["drive_ms"] / max(tm["drive_launches"], 1)
        drive_pairs = 2 * cfg5.B * cfg5.N * (cfg5.N - 1) * 32  # charge pairs x stage times per block
        drive_tf = DRIVE_FLOPS_PER_PAIR * drive_pairs / (drive_ms * 1e-3) / 1e12
        line["roofline_drive"] = {
            "kernel": "lo_drive_kernel (mixed, grid path)", "bound": "alu", "achieved": drive_tf,
            "peak": peak_tflops, "unit": "TFLOP/s", "frac": drive_tf / peak_tflops,
            "frac_of_measured_fp32_fma": drive_tf / (2.0 * fp32_fma / 1e12),
            "flops_per_pair": DRIVE_FLOPS_PER_PAIR, "flops_per_pair_basis": "bench.DRIVE_FLOP_TALLY",
            "launch_ms": drive_ms, "launches": tm["drive_launches"], "rk4_launch_ms": tm["rk4_ms"] / max(tm["rk4_launches"], 1),
            "charge_pair_evals_per_launch": drive_pairs, "source_slices": sl,
            "workload": "cloud (4096 oscillators), blocks 250-349 (steps 4000-5599) resumed from a state, 16 steps "
                        "(32 stage times) per launch; launch times from CUDA events on the run's stream"}
        # the all-float64 GPU path on the same cloud over its first 1000 steps (the whole run takes
        # ~7 minutes in float64), and the mixed path over the same steps for a like-for-like factor
        cfg5s = W.cfg5(n_steps=1000)
        for name, prec in (("mixed", pc.PC_MIXED), ("f64", pc.PC_F64)):
            r = lo_time(cfg5s, cfg5s.n_steps, prec, False)
            r["workload"] = "cloud: 4096 oscillators in a 600 nm cube x the first 1000 RK4 steps"
            ds["cloud_1000_" + name] = r
        ds["cloud_1000_mixed_over_f64"] = ds["cloud_1000_f64"]["ms"] / ds["cloud_1000_mixed"]["ms"]
        pc.pc_set_run_tiling(ctx, 0)

        def timed(fn):
            fn()
            torch.cuda.synchronize()
            e0.record(s)
            fn()
            e1.record(s)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)

        # gradients of the fitted decay rates (Eq. KE fit) of the batched pairs: forward, fit, fit
        # adjoint and reverse sweep, float64
        lod3 = pc.lo_config_to_device(cfg3, dev)
        wg3 = torch.ones((cfg3.B, cfg3.N), dtype=torch.float64, device=dev)
        ms = timed(lambda: pc.pc_dipoles_rates_adjoint(ctx, lod3, cfg3.dt, cfg3.n_steps, cfg3.first_index,
                                                       dL_dgamma=wg3))
        ds["pairs_rates_adjoint_f64"] = {
            "value": cfg3.B * cfg3.N * cfg3.n_steps / (ms * 1e-3), "unit": "dipole-steps/s", "ms": ms,
            "workload": "gradients of sum gamma of the 256 x 2 batched pairs (40000 steps) w.r.t. origins, "
                        "omega0, d0 (forward + fit + reverse)"}
        # moving dipoles (Sec. 4.3): the ring with every origin oscillating along x (1 A, 20 THz)
        cfg4m = W.cfg4(n_steps=4000)
        mot = tuple(torch.from_numpy(x).to(dev)
                    for x in W.oscillating_origins(cfg4m, 1e-10, 2 * math.pi * 20e12))
        lod4m = pc.lo_config_to_device(cfg4m, dev)
        ms = timed(lambda: pc.pc_dipoles_run_moving(ctx, lod4m, mot, cfg4m.dt, cfg4m.n_steps))
        ds["ring_moving_f64"] = {"value": cfg4m.N * cfg4m.n_steps / (ms * 1e-3), "unit": "dipole-steps/s", "ms": ms,
                                 "workload": "ring of 256 oscillators, origins oscillating along x "
                                             "(1e-10 m, 20 THz), 4000 RK4 steps, float64"}
        ms = timed(lambda: pc.pc_dipoles_run_moving(ctx, lod4m, mot, cfg4m.dt, cfg4m.n_steps, precision=pc.PC_MIXED))
        om = pc.pc_dipoles_run_moving(ctx, lod4m, mot, cfg4m.dt, cfg4m.n_steps, precision=pc.PC_MIXED)
        of = pc.pc_dipoles_run_moving(ctx, lod4m, mot, cfg4m.dt, cfg4m.n_steps)
        ds["ring_moving_mixed"] = {
            "value": cfg4m.N * cfg4m.n_steps / (ms * 1e-3), "unit": "dipole-steps/s", "ms": ms,
            "max_rel_d_vs_f64": float((om["d"] - of["d"]).abs().max() / of["d"].abs().max()),
            "workload": "the same, mixed (sources whose retarded times precede sample 1 in float64)"}
        del mot, om, of
        # population dynamics (App. A): one excited and one unexcited dipole, q = 20 e, 80 nm,
        # one beating period (2.1e6 steps of 10 as)
        cfgp = W.population_pair()
        lodp = pc.lo_config_to_device(cfgp, dev)
        for name, prec in (("mixed", pc.PC_MIXED), ("f64", pc.PC_F64)):
            ms = timed(lambda: pc.pc_dipoles_run(ctx, lodp, cfgp.dt, cfgp.n_steps, precision=prec))
            ds["populations_" + name] = {"value": cfgp.B * cfgp.N * cfgp.n_steps / (ms * 1e-3),
                                         "unit": "dipole-steps/s", "ms": ms,
                                         "workload": "two dipoles, 80 nm, q = 20 e, 2.1e6 RK4 steps of 10 as"}
        line["dipole_steps"] = ds
        # charges on analytic trajectories (no history samples): the orbiting pair (static +e, -e on
        # a 1 nm circle at 0.1 c) on a 2048 x 2048 grid over +-50 nm, 4 frames, float64
        ng = 2048
        gx = torch.linspace(-50e-9, 50e-9, ng, dtype=torch.float64, device=dev)
        pts = torch.stack([gx[:, None].expand(ng, ng), gx[None, :].expand(ng, ng),
                           torch.zeros((ng, ng), dtype=torch.float64, device=dev)], dim=-1).reshape(-1, 3)
        par = np.zeros((2, 12))
        par[1, 3], par[1, 7], par[1, 9], par[1, 10] = 1.0, 1.0, 1e-9, 0.1 * W.C / 1e-9
        kinds = [pc.PC_TRAJ_STATIONARY, pc.PC_TRAJ_CIRCULAR]
        tp = [10e-15 + f * 50e-18 for f in range(4)]
        pout = pc.capi.alloc_field_out(ng * ng, len(tp), pc.PC_F64, dev)
        ms = timed(lambda: pc.pc_fields_param(ctx, kinds, [W.E_CHARGE, -W.E_CHARGE], par, pts, tp, out=pout))
        line["param_fields_f64"] = {"value": ng * ng * len(tp) * 2 / (ms * 1e-3), "unit": "LW pair evals/s",
                                    "ms": ms, "workload": "static +e and -e on a 1 nm circle at 0.1 c, analytic "
                                                          "trajectories, 2048 x 2048 grid over +-50 nm, 4 frames"}
        del pout, pts
        if rank == 0:
            import oracle

            oracle.build()
            line["cpu_baseline"] = oracle_sample()
            line["cpu_baseline_lo"] = oracle_lo_sample()
            line["cpu_baseline_cloud"] = oracle_cloud_sample()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
