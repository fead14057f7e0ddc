"""ctypes binding of libpycharge_gb300.so (include/pycharge_gb300.h); argument marshalling only.

Every computation happens in the CUDA library.  Sources and outputs are torch CUDA tensors (the
library only sees their device pointers and the current CUDA stream).  If the library cannot be
loaded the import fails: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from types import SimpleNamespace

import torch

from . import build as _build

PC_OK, PC_ERR_ARG, PC_ERR_CUDA, PC_ERR_HISTORY, PC_ERR_VELOCITY, PC_ERR_CAUSALITY, PC_ERR_NOCONV, PC_ERR_TIMEOUT = range(8)
PC_TOTAL, PC_COULOMB, PC_RADIATION = 0, 1, 2
PC_F64, PC_MIXED = 0, 1

STATUS_NAMES = {
    PC_OK: "PC_OK", PC_ERR_ARG: "PC_ERR_ARG", PC_ERR_CUDA: "PC_ERR_CUDA", PC_ERR_HISTORY: "PC_ERR_HISTORY",
    PC_ERR_VELOCITY: "PC_ERR_VELOCITY", PC_ERR_CAUSALITY: "PC_ERR_CAUSALITY", PC_ERR_NOCONV: "PC_ERR_NOCONV",
    PC_ERR_TIMEOUT: "PC_ERR_TIMEOUT",
}

_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_f64 = ctypes.c_double


class PcCharges(ctypes.Structure):
    _fields_ = [("M", _i32), ("S", _i64), ("t0", _f64), ("dt", _f64), ("q", _vp), ("pos", _vp), ("vel", _vp),
                ("acc", _vp), ("static_before", _i32)]


class PcDipoleSources(ctypes.Structure):
    _fields_ = [("N", _i32), ("S", _i64), ("t0", _f64), ("dt", _f64), ("origin", _vp), ("axis", _vp), ("q", _vp),
                ("m1", _vp), ("m2", _vp), ("d", _vp), ("d_dot", _vp), ("d_ddot", _vp)]


class PcFieldOut(ctypes.Structure):
    _fields_ = [("E", _vp), ("B", _vp), ("phi", _vp), ("A", _vp), ("mask", _vp)]


class PcPlane(ctypes.Structure):
    _fields_ = [("origin", _f64 * 3), ("eu", _f64 * 3), ("ev", _f64 * 3), ("nu", _i64), ("nv", _i64)]


class PcDipoles(ctypes.Structure):
    _fields_ = [("B", _i32), ("N", _i32), ("origin", _vp), ("axis", _vp), ("q", _vp), ("m1", _vp), ("m2", _vp),
                ("omega0", _vp), ("d0", _vp)]


class PcRunOpts(ctypes.Structure):
    _fields_ = [("v_max", _f64), ("ed_mode", _i32), ("fit", _i32), ("first_index", _i64), ("precision", _i32),
                ("near_f64", _f64), ("state_in", _vp), ("state_out", _vp), ("checkpoint_every", _i64)]


class PcRunOut(ctypes.Structure):
    _fields_ = [("d", _vp), ("d_dot", _vp), ("d_ddot", _vp), ("energy", _vp), ("Ed", _vp), ("gamma", _vp),
                ("omega", _vp)]


class PcParamCharges(ctypes.Structure):
    _fields_ = [("M", _i32), ("kind", _vp), ("q", _vp), ("par", _vp)]


PC_TRAJ_STATIONARY, PC_TRAJ_OSCILLATING, PC_TRAJ_CIRCULAR, PC_TRAJ_ACCELERATING = 0, 1, 2, 3


class PcDipoleMotion(ctypes.Structure):
    _fields_ = [("pos", _vp), ("vel", _vp), ("acc", _vp)]


class PcPlaneTiling(ctypes.Structure):
    _fields_ = [("tile_rows", _i32), ("tile_cols", _i32), ("sources_per_stage", _i32)]


class PcRunTiming(ctypes.Structure):
    _fields_ = [("drive_launches", _i64), ("drive_ms", _f64), ("rk4_launches", _i64), ("rk4_ms", _f64),
                ("run_launches", _i64), ("run_ms", _f64)]


class PcDipoleGrads(ctypes.Structure):
    _fields_ = [("origin", _vp), ("omega0", _vp), ("d0", _vp)]


# every entry point of include/pycharge_gb300.h with its argument types
SIGNATURES = {
    "pc_ctx_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int]),
    "pc_ctx_destroy": (ctypes.c_int, [_vp]),
    "pc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "pc_fields": (ctypes.c_int, [_vp, ctypes.POINTER(PcCharges), ctypes.POINTER(PcDipoleSources), _vp, _i64,
                                 ctypes.POINTER(_f64), _i32, _i32, _i32, _f64, ctypes.POINTER(PcFieldOut), _vp]),
    "pc_fields_plane": (ctypes.c_int, [_vp, ctypes.POINTER(PcCharges), ctypes.POINTER(PcDipoleSources),
                                       ctypes.POINTER(PcPlane), ctypes.POINTER(_f64), _i32, _i32, _i32, _f64,
                                       ctypes.POINTER(PcFieldOut), _vp]),
    "pc_dipoles_run": (ctypes.c_int, [_vp, ctypes.POINTER(PcDipoles), _f64, _i64, ctypes.POINTER(PcRunOpts),
                                      ctypes.POINTER(PcRunOut), _vp]),
    "pc_dipoles_state_size": (ctypes.c_int, [_vp, ctypes.POINTER(PcDipoles), _f64, ctypes.POINTER(_i64), _vp]),
    "pc_autotune_run": (ctypes.c_int, [_vp, ctypes.POINTER(PcDipoles), _f64, _i64, ctypes.POINTER(PcRunOpts),
                                       ctypes.POINTER(_i32), _vp]),
    "pc_set_run_tiling": (ctypes.c_int, [_vp, _i32]),
    "pc_set_run_timing": (ctypes.c_int, [_vp, _i32]),
    "pc_get_run_timing": (ctypes.c_int, [_vp, _vp]),
    "pc_fields_to_host": (ctypes.c_int, [_vp, ctypes.POINTER(PcCharges), ctypes.POINTER(PcDipoleSources), _vp, _i64,
                                         ctypes.POINTER(_f64), _i32, _i32, _i32, _f64, ctypes.POINTER(PcFieldOut),
                                         _vp]),
    "pc_fields_plane_to_host": (ctypes.c_int, [_vp, ctypes.POINTER(PcCharges), ctypes.POINTER(PcDipoleSources),
                                               ctypes.POINTER(PcPlane), ctypes.POINTER(_f64), _i32, _i32, _i32, _f64,
                                               ctypes.POINTER(PcFieldOut), _vp]),
    "pc_autotune_plane": (ctypes.c_int, [_vp, ctypes.POINTER(PcCharges), ctypes.POINTER(PcDipoleSources),
                                         ctypes.POINTER(PcPlane), ctypes.POINTER(_f64), _i32, _i32, _f64,
                                         ctypes.POINTER(PcFieldOut), ctypes.POINTER(PcPlaneTiling), _vp]),
    "pc_set_plane_tiling": (ctypes.c_int, [_vp, ctypes.POINTER(PcPlaneTiling)]),
    "pc_fields_param": (ctypes.c_int, [_vp, ctypes.POINTER(PcParamCharges), _vp, _i64, ctypes.POINTER(_f64), _i32,
                                       _i32, _f64, ctypes.POINTER(PcFieldOut), _vp]),
    "pc_dipoles_run_moving": (ctypes.c_int, [_vp, ctypes.POINTER(PcDipoles), ctypes.POINTER(PcDipoleMotion), _f64,
                                             _i64, ctypes.POINTER(PcRunOpts), ctypes.POINTER(PcRunOut), _vp]),
    "pc_dipoles_adjoint_moving": (ctypes.c_int, [_vp, ctypes.POINTER(PcDipoles), ctypes.POINTER(PcDipoleMotion),
                                                 _f64, _i64, ctypes.POINTER(PcRunOpts), _vp,
                                                 ctypes.POINTER(PcDipoleGrads), ctypes.POINTER(PcDipoleMotion), _vp]),
    "pc_dipoles_adjoint": (ctypes.c_int, [_vp, ctypes.POINTER(PcDipoles), _f64, _i64, ctypes.POINTER(PcRunOpts),
                                          _vp, ctypes.POINTER(PcDipoleGrads), _vp]),
    "pc_dipoles_rates_adjoint": (ctypes.c_int, [_vp, ctypes.POINTER(PcDipoles), _f64, _i64,
                                                ctypes.POINTER(PcRunOpts), _vp, _vp, _vp, _vp,
                                                ctypes.POINTER(PcDipoleGrads), _vp]),
    "pc_dipoles_fields_adjoint": (ctypes.c_int, [_vp, ctypes.POINTER(PcDipoles), _f64, _i64,
                                                 ctypes.POINTER(PcRunOpts), _vp, _i64, ctypes.POINTER(_f64), _i32,
                                                 ctypes.POINTER(PcFieldOut), ctypes.POINTER(PcDipoleGrads), _vp]),
    "pc_ke_fit": (ctypes.c_int, [_vp, _vp, _i32, _i64, _f64, _i64, _vp, _vp, _vp, _vp, _vp]),
    "pc_alu_peaks": (ctypes.c_int, [_vp, ctypes.POINTER(_f64), ctypes.POINTER(_f64), _vp]),
    "pc_fields_noalloc": (ctypes.c_int, [ctypes.POINTER(PcCharges), ctypes.POINTER(PcDipoleSources), _vp, _i64,
                                         ctypes.POINTER(_f64), _i32, _i32, _f64, ctypes.POINTER(PcFieldOut), _vp]),
}

_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load the shared library (building it first if asked); raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libpycharge_gb300.so not found at {path}; run paper_2107_12437_gb300/build.py")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class PcError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = load().pc_status_string(status).decode()
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({msg})")


def _check(st: int, where: str):
    if st != PC_OK:
        raise PcError(st, where)


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """pc_ctx on one device."""

    def __init__(self, device: int = 0):
        self.lib = load()
        self.device = device
        h = _vp()
        _check(self.lib.pc_ctx_create(ctypes.byref(h), device), "pc_ctx_create")
        self.handle = h

    def close(self):
        if self.handle:
            self.lib.pc_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _dev(x, device):
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=torch.float64).contiguous()
    return torch.as_tensor(x, dtype=torch.float64, device=device).contiguous()


def charges_to_device(ch, device="cuda"):
    """Copy a host description of point charges (fields q, pos, vel, acc, t0, dt, static_before)."""
    return SimpleNamespace(q=_dev(ch.q, device), pos=_dev(ch.pos, device), vel=_dev(ch.vel, device),
                           acc=_dev(ch.acc, device), t0=float(ch.t0), dt=float(ch.dt),
                           static_before=int(getattr(ch, "static_before", 0)))


def dipoles_to_device(dp, device="cuda"):
    """Copy a host description of dipole sources (origin, axis, q, m1, m2, d, d_dot, d_ddot, t0, dt)."""
    return SimpleNamespace(origin=_dev(dp.origin, device), axis=_dev(dp.axis, device), q=_dev(dp.q, device),
                           m1=_dev(dp.m1, device), m2=_dev(dp.m2, device), d=_dev(dp.d, device),
                           d_dot=_dev(dp.d_dot, device), d_ddot=_dev(dp.d_ddot, device), t0=float(dp.t0),
                           dt=float(dp.dt))


def _charges_struct(ch):
    if ch is None:
        return None
    return PcCharges(M=int(ch.q.shape[0]), S=int(ch.pos.shape[1]), t0=ch.t0, dt=ch.dt, q=_ptr(ch.q),
                     pos=_ptr(ch.pos), vel=_ptr(ch.vel), acc=_ptr(ch.acc), static_before=int(ch.static_before))


def _dipoles_struct(dp):
    if dp is None:
        return None
    return PcDipoleSources(N=int(dp.origin.shape[0]), S=int(dp.d.shape[1]), t0=dp.t0, dt=dp.dt,
                           origin=_ptr(dp.origin), axis=_ptr(dp.axis), q=_ptr(dp.q), m1=_ptr(dp.m1), m2=_ptr(dp.m2),
                           d=_ptr(dp.d), d_dot=_ptr(dp.d_dot), d_ddot=_ptr(dp.d_ddot))


def alloc_field_out(P, T, precision, device="cuda", which=("E", "B", "phi", "A", "mask")):
    dt = torch.float64 if precision == PC_F64 else torch.float32
    o = {}
    if "E" in which:
        o["E"] = torch.empty((T, P, 3), dtype=dt, device=device)
    if "B" in which:
        o["B"] = torch.empty((T, P, 3), dtype=dt, device=device)
    if "phi" in which:
        o["phi"] = torch.empty((T, P), dtype=dt, device=device)
    if "A" in which:
        o["A"] = torch.empty((T, P, 3), dtype=dt, device=device)
    if "mask" in which:
        o["mask"] = torch.empty((T, P), dtype=torch.uint8, device=device)
    return o


def _hptr(t):
    if t is None:
        return None
    assert not t.is_cuda and t.is_contiguous(), "host outputs must be contiguous CPU tensors"
    return ctypes.c_void_p(t.data_ptr())


def _host_out_struct(o):
    return PcFieldOut(E=_hptr(o.get("E")), B=_hptr(o.get("B")), phi=_hptr(o.get("phi")), A=_hptr(o.get("A")),
                      mask=_hptr(o.get("mask")))


def _out_struct(o):
    return PcFieldOut(E=_ptr(o.get("E")), B=_ptr(o.get("B")), phi=_ptr(o.get("phi")), A=_ptr(o.get("A")),
                      mask=_ptr(o.get("mask")))


def pc_fields(ctx, charges=None, dipoles=None, points=None, times=(0.0,), kind=PC_TOTAL, precision=PC_F64,
              r_excl=0.0, out=None, stream=None):
    """pc_fields: points is a [P][3] float64 CUDA tensor; returns the dict of output tensors."""
    P = int(points.shape[0])
    T = len(times)
    o = alloc_field_out(P, T, precision, points.device) if out is None else out
    tarr = (_f64 * T)(*[float(t) for t in times])
    chs = _charges_struct(charges)
    dps = _dipoles_struct(dipoles)
    st = ctx.lib.pc_fields(ctx.handle, ctypes.byref(chs) if chs else None, ctypes.byref(dps) if dps else None,
                           _ptr(points), P, tarr, T, kind, precision, float(r_excl), ctypes.byref(_out_struct(o)),
                           _stream(stream))
    _check(st, "pc_fields")
    return o


def pc_fields_plane(ctx, charges=None, dipoles=None, origin=(0, 0, 0), eu=(1, 0, 0), ev=(0, 1, 0), nu=1, nv=1,
                    times=(0.0,), kind=PC_TOTAL, precision=PC_F64, r_excl=0.0, out=None, stream=None,
                    device="cuda"):
    """pc_fields_plane: point (iu, iv) = origin + iu eu + iv ev, output index iu*nv + iv."""
    T = len(times)
    o = alloc_field_out(nu * nv, T, precision, device) if out is None else out
    pl = PcPlane(origin=(_f64 * 3)(*origin), eu=(_f64 * 3)(*eu), ev=(_f64 * 3)(*ev), nu=nu, nv=nv)
    tarr = (_f64 * T)(*[float(t) for t in times])
    chs = _charges_struct(charges)
    dps = _dipoles_struct(dipoles)
    st = ctx.lib.pc_fields_plane(ctx.handle, ctypes.byref(chs) if chs else None, ctypes.byref(dps) if dps else None,
                                 ctypes.byref(pl), tarr, T, kind, precision, float(r_excl),
                                 ctypes.byref(_out_struct(o)), _stream(stream))
    _check(st, "pc_fields_plane")
    return o


def pc_autotune_plane(ctx, charges=None, dipoles=None, origin=(0, 0, 0), eu=(1, 0, 0), ev=(0, 1, 0), nu=1, nv=1,
                      times=(0.0,), kind=PC_TOTAL, r_excl=0.0, out=None, stream=None, device="cuda"):
    """pc_autotune_plane: times the tile shapes on this mixed plane workload, keeps the fastest in
    the context and returns it as (rows, columns, sources per stage)."""
    T = len(times)
    o = alloc_field_out(nu * nv, T, PC_MIXED, device) if out is None else out
    pl = PcPlane(origin=(_f64 * 3)(*origin), eu=(_f64 * 3)(*eu), ev=(_f64 * 3)(*ev), nu=nu, nv=nv)
    tarr = (_f64 * T)(*[float(t) for t in times])
    chs = _charges_struct(charges)
    dps = _dipoles_struct(dipoles)
    t = PcPlaneTiling()
    st = ctx.lib.pc_autotune_plane(ctx.handle, ctypes.byref(chs) if chs else None, ctypes.byref(dps) if dps else None,
                                   ctypes.byref(pl), tarr, T, kind, float(r_excl), ctypes.byref(_out_struct(o)),
                                   ctypes.byref(t), _stream(stream))
    _check(st, "pc_autotune_plane")
    return t.tile_rows, t.tile_cols, t.sources_per_stage


def pc_set_plane_tiling(ctx, tile_rows, tile_cols, sources_per_stage=64):
    """pc_set_plane_tiling: the mixed plane tile shape (256 points, or 512 with two per thread) and
    the sources per shared-memory stage (32 or 64)."""
    t = PcPlaneTiling(tile_rows=int(tile_rows), tile_cols=int(tile_cols), sources_per_stage=int(sources_per_stage))
    _check(ctx.lib.pc_set_plane_tiling(ctx.handle, ctypes.byref(t)), "pc_set_plane_tiling")


def alloc_host_field_out(P, T, precision, which=("E", "B", "phi", "A", "mask"), pinned=True):
    """Host outputs for pc_fields_plane_to_host / pc_fields_to_host: page-locked (the kernels store
    into them directly) or, with pinned=False, pageable (filled by chunked copies)."""
    dt = torch.float64 if precision == PC_F64 else torch.float32
    shapes = {"E": (T, P, 3), "B": (T, P, 3), "phi": (T, P), "A": (T, P, 3), "mask": (T, P)}
    return {k: torch.empty(shapes[k], dtype=torch.uint8 if k == "mask" else dt, pin_memory=pinned) for k in which}


def pc_fields_to_host(ctx, charges=None, dipoles=None, points=None, times=(0.0,), kind=PC_TOTAL, precision=PC_F64,
                      r_excl=0.0, out=None, stream=None):
    """pc_fields_to_host: points [P][3] float64 CUDA tensor, outputs host tensors (page-locked by
    default)."""
    P = int(points.shape[0])
    T = len(times)
    o = alloc_host_field_out(P, T, precision) if out is None else out
    tarr = (_f64 * T)(*[float(t) for t in times])
    chs = _charges_struct(charges)
    dps = _dipoles_struct(dipoles)
    st = ctx.lib.pc_fields_to_host(ctx.handle, ctypes.byref(chs) if chs else None,
                                   ctypes.byref(dps) if dps else None, _ptr(points), P, tarr, T, kind, precision,
                                   float(r_excl), ctypes.byref(_host_out_struct(o)), _stream(stream))
    _check(st, "pc_fields_to_host")
    return o


def pc_fields_plane_to_host(ctx, charges=None, dipoles=None, origin=(0, 0, 0), eu=(1, 0, 0), ev=(0, 1, 0), nu=1,
                            nv=1, times=(0.0,), kind=PC_TOTAL, precision=PC_F64, r_excl=0.0, out=None, stream=None):
    """pc_fields_plane_to_host: sources on the device, outputs host tensors (page-locked by default)."""
    T = len(times)
    o = alloc_host_field_out(nu * nv, T, precision) if out is None else out
    pl = PcPlane(origin=(_f64 * 3)(*origin), eu=(_f64 * 3)(*eu), ev=(_f64 * 3)(*ev), nu=nu, nv=nv)
    tarr = (_f64 * T)(*[float(t) for t in times])
    chs = _charges_struct(charges)
    dps = _dipoles_struct(dipoles)
    st = ctx.lib.pc_fields_plane_to_host(ctx.handle, ctypes.byref(chs) if chs else None,
                                         ctypes.byref(dps) if dps else None, ctypes.byref(pl), tarr, T, kind,
                                         precision, float(r_excl), ctypes.byref(_host_out_struct(o)),
                                         _stream(stream))
    _check(st, "pc_fields_plane_to_host")
    return o


def pc_fields_param(ctx, kind, q, par, points, times=(0.0,), field_kind=PC_TOTAL, r_excl=0.0, out=None, stream=None):
    """pc_fields_param: charges on analytic trajectories (kind [M] int32, q [M], par [M][12]);
    returns float64 E, B, A [T][P][3], phi [T][P], mask [T][P]."""
    dev = points.device if isinstance(points, torch.Tensor) else torch.device("cuda")
    kd = torch.as_tensor(kind, dtype=torch.int32, device=dev).contiguous()
    qq = torch.as_tensor(q, dtype=torch.float64, device=dev).contiguous()
    pr = torch.as_tensor(par, dtype=torch.float64, device=dev).reshape(-1, 12).contiguous()
    pts = torch.as_tensor(points, dtype=torch.float64, device=dev).reshape(-1, 3).contiguous()
    P, T = int(pts.shape[0]), len(times)
    if out is None:
        out = alloc_field_out(P, T, PC_F64, dev)
    ch = PcParamCharges(M=int(kd.numel()), kind=_ptr(kd), q=_ptr(qq), par=_ptr(pr))
    tarr = (_f64 * T)(*[float(t) for t in times])
    st = ctx.lib.pc_fields_param(ctx.handle, ctypes.byref(ch), _ptr(pts), P, tarr, T, int(field_kind), float(r_excl),
                                 ctypes.byref(_out_struct(out)), _stream(stream))
    _check(st, "pc_fields_param")
    return out


def lo_config_to_device(cfg, device="cuda"):
    """Copy a host LO configuration batch (origin, axis, q, m1, m2, omega0, d0 with leading [B][N])."""
    return SimpleNamespace(origin=_dev(cfg.origin, device), axis=_dev(cfg.axis, device), q=_dev(cfg.q, device),
                           m1=_dev(cfg.m1, device), m2=_dev(cfg.m2, device), omega0=_dev(cfg.omega0, device),
                           d0=_dev(cfg.d0, device))


def _dipoles(dp):
    return PcDipoles(B=int(dp.origin.shape[0]), N=int(dp.origin.shape[1]), origin=_ptr(dp.origin), axis=_ptr(dp.axis),
                     q=_ptr(dp.q), m1=_ptr(dp.m1), m2=_ptr(dp.m2), omega0=_ptr(dp.omega0), d0=_ptr(dp.d0))


def pc_autotune_run(ctx, dp, dt, probe_steps=64, precision=PC_F64, near_f64=0.0, v_max=0.0, stream=None):
    """pc_autotune_run: times the grid path's source-slice counts on this configuration and keeps
    the fastest in the context; returns it (1 for configurations that run as one CTA each)."""
    opts = PcRunOpts(v_max=float(v_max), ed_mode=0, fit=0, first_index=0, precision=int(precision),
                     near_f64=float(near_f64))
    c = _i32(0)
    _check(ctx.lib.pc_autotune_run(ctx.handle, ctypes.byref(_dipoles(dp)), float(dt), int(probe_steps),
                                   ctypes.byref(opts), ctypes.byref(c), _stream(stream)), "pc_autotune_run")
    return int(c.value)


def pc_set_run_tiling(ctx, source_slices):
    """pc_set_run_tiling: source slices per receiver of the grid path (0: the heuristic)."""
    _check(ctx.lib.pc_set_run_tiling(ctx.handle, int(source_slices)), "pc_set_run_tiling")


def pc_set_run_timing(ctx, enable):
    """pc_set_run_timing: 1 clears the launch-time counters and times later oscillator runs (their
    grid-path block loop then launched from the host); 0 turns it off."""
    _check(ctx.lib.pc_set_run_timing(ctx.handle, int(bool(enable))), "pc_set_run_timing")


def pc_get_run_timing(ctx):
    """pc_get_run_timing: the counters since the last enable, as a dict."""
    t = PcRunTiming()
    _check(ctx.lib.pc_get_run_timing(ctx.handle, ctypes.byref(t)), "pc_get_run_timing")
    return {k: getattr(t, k) for k, _ in PcRunTiming._fields_}


def pc_dipoles_state_size(ctx, dp, dt, stream=None):
    """pc_dipoles_state_size: the number of float64 values of a run state of these dipoles."""
    n = _i64(0)
    _check(ctx.lib.pc_dipoles_state_size(ctx.handle, ctypes.byref(_dipoles(dp)), float(dt), ctypes.byref(n),
                                         _stream(stream)), "pc_dipoles_state_size")
    return int(n.value)


def pc_dipoles_run(ctx, dp, dt, n_steps, v_max=0.0, ed_mode=0, fit=False, first_index=0, precision=PC_F64,
                   want_energy=True, want_Ed=False, out=None, near_f64=0.0, want_history=True, state_in=None,
                   state_out=None, stream=None):
    """pc_dipoles_run: dp holds [B][N] / [B][N][3] CUDA tensors; returns the dict of outputs.

    want_history=False leaves out d, d_dot, d_ddot (the run then keeps its history in a ring of the
    context, memory independent of n_steps).  state_in / state_out: float64 CUDA tensors of
    pc_dipoles_state_size values (resume from / save the state at the last step)."""
    B, N = int(dp.origin.shape[0]), int(dp.origin.shape[1])
    S = int(n_steps) + 1
    dev = dp.origin.device
    if out is None:
        out = {}
        if want_history:
            out.update(d=torch.empty((B, N, S), dtype=torch.float64, device=dev),
                       d_dot=torch.empty((B, N, S), dtype=torch.float64, device=dev),
                       d_ddot=torch.empty((B, N, S), dtype=torch.float64, device=dev))
        if want_energy:
            out["energy"] = torch.empty((B, N, S), dtype=torch.float64, device=dev)
        if want_Ed:
            out["Ed"] = torch.empty((B, N, S), dtype=torch.float64, device=dev)
        if fit:
            out["gamma"] = torch.empty((B, N), dtype=torch.float64, device=dev)
            out["omega"] = torch.empty((B, N), dtype=torch.float64, device=dev)
    d = _dipoles(dp)
    opts = PcRunOpts(v_max=float(v_max), ed_mode=int(ed_mode), fit=int(bool(fit)), first_index=int(first_index),
                     precision=int(precision), near_f64=float(near_f64), state_in=_ptr(state_in),
                     state_out=_ptr(state_out))
    ro = PcRunOut(d=_ptr(out.get("d")), d_dot=_ptr(out.get("d_dot")), d_ddot=_ptr(out.get("d_ddot")),
                  energy=_ptr(out.get("energy")), Ed=_ptr(out.get("Ed")), gamma=_ptr(out.get("gamma")),
                  omega=_ptr(out.get("omega")))
    st = ctx.lib.pc_dipoles_run(ctx.handle, ctypes.byref(d), float(dt), int(n_steps), ctypes.byref(opts),
                                ctypes.byref(ro), _stream(stream))
    _check(st, "pc_dipoles_run")
    return out


def pc_dipoles_adjoint(ctx, dp, dt, n_steps, dL_dEnergyFinal, v_max=0.0, precision=PC_F64, checkpoint_every=0,
                       stream=None):
    """pc_dipoles_adjoint: gradients of sum w E(T) (w = dL_dEnergyFinal, [B][N] CUDA float64) with
    respect to the origins, omega0 and d0; returns (g_origin [B][N][3], g_omega0 [B][N], g_d0 [B][N]).
    precision selects the forward run's driving field (the reverse is float64); checkpoint_every > 0
    keeps the run's state every that many steps and recomputes each segment in the reverse sweep."""
    B, N = int(dp.origin.shape[0]), int(dp.origin.shape[1])
    dev = dp.origin.device
    w = dL_dEnergyFinal.to(device=dev, dtype=torch.float64).contiguous()
    g_origin = torch.empty((B, N, 3), dtype=torch.float64, device=dev)
    g_omega0 = torch.empty((B, N), dtype=torch.float64, device=dev)
    g_d0 = torch.empty((B, N), dtype=torch.float64, device=dev)
    d = PcDipoles(B=B, N=N, origin=_ptr(dp.origin), axis=_ptr(dp.axis), q=_ptr(dp.q), m1=_ptr(dp.m1),
                  m2=_ptr(dp.m2), omega0=_ptr(dp.omega0), d0=_ptr(dp.d0))
    opts = PcRunOpts(v_max=float(v_max), ed_mode=0, fit=0, first_index=0, precision=int(precision),
                     checkpoint_every=int(checkpoint_every))
    g = PcDipoleGrads(origin=_ptr(g_origin), omega0=_ptr(g_omega0), d0=_ptr(g_d0))
    st = ctx.lib.pc_dipoles_adjoint(ctx.handle, ctypes.byref(d), float(dt), int(n_steps), ctypes.byref(opts),
                                    _ptr(w), ctypes.byref(g), _stream(stream))
    _check(st, "pc_dipoles_adjoint")
    return g_origin, g_omega0, g_d0


def pc_dipoles_rates_adjoint(ctx, dp, dt, n_steps, first_index, dL_dgamma=None, dL_domega=None, v_max=0.0,
                             checkpoint_every=0, stream=None):
    """pc_dipoles_rates_adjoint: gradients of sum(dL_dgamma gamma + dL_domega omega) of the Eq. KE
    fit; returns (gamma, omega, g_origin, g_omega0, g_d0)."""
    B, N = int(dp.origin.shape[0]), int(dp.origin.shape[1])
    dev = dp.origin.device

    def cot(x):
        return None if x is None else x.to(device=dev, dtype=torch.float64).contiguous()

    wg, ww = cot(dL_dgamma), cot(dL_domega)
    gamma = torch.empty((B, N), dtype=torch.float64, device=dev)
    omega = torch.empty((B, N), dtype=torch.float64, device=dev)
    g_origin = torch.empty((B, N, 3), dtype=torch.float64, device=dev)
    g_omega0 = torch.empty((B, N), dtype=torch.float64, device=dev)
    g_d0 = torch.empty((B, N), dtype=torch.float64, device=dev)
    d = PcDipoles(B=B, N=N, origin=_ptr(dp.origin), axis=_ptr(dp.axis), q=_ptr(dp.q), m1=_ptr(dp.m1),
                  m2=_ptr(dp.m2), omega0=_ptr(dp.omega0), d0=_ptr(dp.d0))
    opts = PcRunOpts(v_max=float(v_max), ed_mode=0, fit=1, first_index=int(first_index), precision=PC_F64,
                     checkpoint_every=int(checkpoint_every))
    g = PcDipoleGrads(origin=_ptr(g_origin), omega0=_ptr(g_omega0), d0=_ptr(g_d0))
    st = ctx.lib.pc_dipoles_rates_adjoint(ctx.handle, ctypes.byref(d), float(dt), int(n_steps), ctypes.byref(opts),
                                          _ptr(wg), _ptr(ww), _ptr(gamma), _ptr(omega), ctypes.byref(g),
                                          _stream(stream))
    _check(st, "pc_dipoles_rates_adjoint")
    return gamma, omega, g_origin, g_omega0, g_d0


def pc_dipoles_fields_adjoint(ctx, dp, dt, n_steps, points, times, cE=None, cB=None, cphi=None, cA=None, v_max=0.0,
                              precision=PC_F64, stream=None):
    """pc_dipoles_fields_adjoint: gradients of sum <c, field> of the oscillators' own fields at the
    points and times; cotangents [B][T][P][3] / [B][T][P] CUDA float64 (any may be None).
    Returns (g_origin, g_omega0, g_d0)."""
    B, N = int(dp.origin.shape[0]), int(dp.origin.shape[1])
    dev = dp.origin.device
    pts = torch.as_tensor(points, dtype=torch.float64, device=dev).reshape(-1, 3).contiguous()
    P, T = int(pts.shape[0]), len(times)

    def c(x):
        return None if x is None else torch.as_tensor(x, dtype=torch.float64, device=dev).contiguous()

    cot = {k: c(v) for k, v in (("E", cE), ("B", cB), ("phi", cphi), ("A", cA))}
    g_origin = torch.empty((B, N, 3), dtype=torch.float64, device=dev)
    g_omega0 = torch.empty((B, N), dtype=torch.float64, device=dev)
    g_d0 = torch.empty((B, N), dtype=torch.float64, device=dev)
    d = PcDipoles(B=B, N=N, origin=_ptr(dp.origin), axis=_ptr(dp.axis), q=_ptr(dp.q), m1=_ptr(dp.m1),
                  m2=_ptr(dp.m2), omega0=_ptr(dp.omega0), d0=_ptr(dp.d0))
    opts = PcRunOpts(v_max=float(v_max), ed_mode=0, fit=0, first_index=0, precision=int(precision))
    g = PcDipoleGrads(origin=_ptr(g_origin), omega0=_ptr(g_omega0), d0=_ptr(g_d0))
    tarr = (_f64 * T)(*[float(t) for t in times])
    st = ctx.lib.pc_dipoles_fields_adjoint(ctx.handle, ctypes.byref(d), float(dt), int(n_steps), ctypes.byref(opts),
                                           _ptr(pts), P, tarr, T, ctypes.byref(_out_struct(cot)), ctypes.byref(g),
                                           _stream(stream))
    _check(st, "pc_dipoles_fields_adjoint")
    return g_origin, g_omega0, g_d0


class FittedRates(torch.autograd.Function):
    """(gamma, omega) [B][N] of the Eq. KE fit after the float64 run, differentiable in
    (origin, omega0, d0); the backward pass is pc_dipoles_rates_adjoint."""

    @staticmethod
    def forward(fctx, origin, omega0, d0, rest, ctx, dt, n_steps, first_index, v_max):
        dp = SimpleNamespace(origin=origin.contiguous(), omega0=omega0.contiguous(), d0=d0.contiguous(),
                             axis=rest.axis, q=rest.q, m1=rest.m1, m2=rest.m2)
        out = pc_dipoles_run(ctx, dp, dt, n_steps, v_max=v_max, precision=PC_F64, fit=True, first_index=first_index,
                             want_energy=False)
        fctx.dp, fctx.pc, fctx.args = dp, ctx, (dt, n_steps, first_index, v_max)
        return out["gamma"], out["omega"]

    @staticmethod
    def backward(fctx, grad_gamma, grad_omega):
        dt, n_steps, first_index, v_max = fctx.args
        _, _, go, gw, gd = pc_dipoles_rates_adjoint(fctx.pc, fctx.dp, dt, n_steps, first_index, grad_gamma,
                                                    grad_omega, v_max=v_max)
        return go, gw, gd, None, None, None, None, None, None


def fitted_rates(ctx, dp, dt, n_steps, first_index, v_max=0.0):
    """Differentiable (gamma, omega) of the Eq. KE fit of pc_dipoles_run in float64."""
    return FittedRates.apply(dp.origin, dp.omega0, dp.d0, dp, ctx, float(dt), int(n_steps), int(first_index),
                             float(v_max))


class FinalEnergy(torch.autograd.Function):
    """E(T) [B][N] of the float64 oscillator run as a differentiable function of (origin, omega0, d0);
    the backward pass is pc_dipoles_adjoint.  Other configuration tensors are held fixed."""

    @staticmethod
    def forward(fctx, origin, omega0, d0, rest, ctx, dt, n_steps, v_max):
        dp = SimpleNamespace(origin=origin.contiguous(), omega0=omega0.contiguous(), d0=d0.contiguous(),
                             axis=rest.axis, q=rest.q, m1=rest.m1, m2=rest.m2)
        out = pc_dipoles_run(ctx, dp, dt, n_steps, v_max=v_max, precision=PC_F64, want_energy=True)
        fctx.dp, fctx.pc, fctx.dt, fctx.n_steps, fctx.v_max = dp, ctx, dt, n_steps, v_max
        return out["energy"][:, :, -1].clone()

    @staticmethod
    def backward(fctx, grad_E):
        go, gw, gd = pc_dipoles_adjoint(fctx.pc, fctx.dp, fctx.dt, fctx.n_steps, grad_E, v_max=fctx.v_max)
        return go, gw, gd, None, None, None, None, None


def final_energy(ctx, dp, dt, n_steps, v_max=0.0):
    """Differentiable E(T) [B][N] (Eq. dipoleE at the last step) of pc_dipoles_run in float64."""
    return FinalEnergy.apply(dp.origin, dp.omega0, dp.d0, dp, ctx, float(dt), int(n_steps), float(v_max))


def pc_dipoles_run_moving(ctx, dp, motion, dt, n_steps, v_max=0.0, ed_mode=0, fit=False, first_index=0,
                          want_energy=True, want_Ed=False, precision=PC_F64, near_f64=0.0, stream=None):
    """pc_dipoles_run_moving: motion = (pos, vel, acc) CUDA float64 tensors [B][N][2 n_steps + 1][3];
    precision PC_F64 or PC_MIXED (near_f64: sources closer than this many metres in float64)."""
    B, N = int(dp.origin.shape[0]), int(dp.origin.shape[1])
    S = int(n_steps) + 1
    dev = dp.origin.device
    out = dict(d=torch.empty((B, N, S), dtype=torch.float64, device=dev),
               d_dot=torch.empty((B, N, S), dtype=torch.float64, device=dev),
               d_ddot=torch.empty((B, N, S), dtype=torch.float64, device=dev))
    if want_energy:
        out["energy"] = torch.empty((B, N, S), dtype=torch.float64, device=dev)
    if want_Ed:
        out["Ed"] = torch.empty((B, N, S), dtype=torch.float64, device=dev)
    if fit:
        out["gamma"] = torch.empty((B, N), dtype=torch.float64, device=dev)
        out["omega"] = torch.empty((B, N), dtype=torch.float64, device=dev)
    pos, vel, acc = (x.to(device=dev, dtype=torch.float64).contiguous() for x in motion)
    for x in (pos, vel, acc):
        if tuple(x.shape) != (B, N, 2 * S - 1, 3):
            raise ValueError("motion arrays must be [B][N][2 n_steps + 1][3]")
    d = PcDipoles(B=B, N=N, origin=_ptr(dp.origin), axis=_ptr(dp.axis), q=_ptr(dp.q), m1=_ptr(dp.m1),
                  m2=_ptr(dp.m2), omega0=_ptr(dp.omega0), d0=_ptr(dp.d0))
    mo = PcDipoleMotion(pos=_ptr(pos), vel=_ptr(vel), acc=_ptr(acc))
    opts = PcRunOpts(v_max=float(v_max), ed_mode=int(ed_mode), fit=int(bool(fit)), first_index=int(first_index),
                     precision=int(precision), near_f64=float(near_f64))
    ro = PcRunOut(d=_ptr(out["d"]), d_dot=_ptr(out["d_dot"]), d_ddot=_ptr(out["d_ddot"]),
                  energy=_ptr(out.get("energy")), Ed=_ptr(out.get("Ed")), gamma=_ptr(out.get("gamma")),
                  omega=_ptr(out.get("omega")))
    st = ctx.lib.pc_dipoles_run_moving(ctx.handle, ctypes.byref(d), ctypes.byref(mo), float(dt), int(n_steps),
                                       ctypes.byref(opts), ctypes.byref(ro), _stream(stream))
    _check(st, "pc_dipoles_run_moving")
    return out


def pc_dipoles_adjoint_moving(ctx, dp, motion, dt, n_steps, dL_dEnergyFinal, v_max=0.0, precision=PC_F64,
                              stream=None):
    """pc_dipoles_adjoint_moving: gradients of sum w E(T) of a moving run (motion = (pos, vel, acc)
    CUDA float64 [B][N][2 n_steps + 1][3]; precision: the forward's driving field, the reverse is
    float64); returns (g_origin (zeros), g_omega0, g_d0, g_pos, g_vel, g_acc)."""
    B, N = int(dp.origin.shape[0]), int(dp.origin.shape[1])
    dev = dp.origin.device
    H = 2 * int(n_steps) + 1
    pos, vel, acc = (x.to(device=dev, dtype=torch.float64).contiguous() for x in motion)
    for x in (pos, vel, acc):
        if tuple(x.shape) != (B, N, H, 3):
            raise ValueError("motion arrays must be [B][N][2 n_steps + 1][3]")
    w = dL_dEnergyFinal.to(device=dev, dtype=torch.float64).contiguous()
    g_origin = torch.empty((B, N, 3), dtype=torch.float64, device=dev)
    g_omega0 = torch.empty((B, N), dtype=torch.float64, device=dev)
    g_d0 = torch.empty((B, N), dtype=torch.float64, device=dev)
    gm = [torch.empty((B, N, H, 3), dtype=torch.float64, device=dev) for _ in range(3)]
    d = PcDipoles(B=B, N=N, origin=_ptr(dp.origin), axis=_ptr(dp.axis), q=_ptr(dp.q), m1=_ptr(dp.m1),
                  m2=_ptr(dp.m2), omega0=_ptr(dp.omega0), d0=_ptr(dp.d0))
    mo = PcDipoleMotion(pos=_ptr(pos), vel=_ptr(vel), acc=_ptr(acc))
    opts = PcRunOpts(v_max=float(v_max), ed_mode=0, fit=0, first_index=0, precision=int(precision))
    g = PcDipoleGrads(origin=_ptr(g_origin), omega0=_ptr(g_omega0), d0=_ptr(g_d0))
    gmo = PcDipoleMotion(pos=_ptr(gm[0]), vel=_ptr(gm[1]), acc=_ptr(gm[2]))
    st = ctx.lib.pc_dipoles_adjoint_moving(ctx.handle, ctypes.byref(d), ctypes.byref(mo), float(dt), int(n_steps),
                                           ctypes.byref(opts), _ptr(w), ctypes.byref(g), ctypes.byref(gmo),
                                           _stream(stream))
    _check(st, "pc_dipoles_adjoint_moving")
    return (g_origin, g_omega0, g_d0, *gm)


def pc_ke_fit(ctx, ke, dt, first_index, stream=None):
    """pc_ke_fit on a [K][S] float64 CUDA tensor; returns (gamma, omega, amp, phase) tensors [K]."""
    K, S = int(ke.shape[0]), int(ke.shape[1])
    dev = ke.device
    g = torch.empty(K, dtype=torch.float64, device=dev)
    w = torch.empty(K, dtype=torch.float64, device=dev)
    a = torch.empty(K, dtype=torch.float64, device=dev)
    p = torch.empty(K, dtype=torch.float64, device=dev)
    st = ctx.lib.pc_ke_fit(ctx.handle, _ptr(ke), K, S, float(dt), int(first_index), _ptr(g), _ptr(w), _ptr(a),
                           _ptr(p), _stream(stream))
    _check(st, "pc_ke_fit")
    return g, w, a, p


def pc_alu_peaks(ctx, stream=None):
    """(fp32 FMA/s, fp64 FMA/s) measured on the context's device."""
    a, b = _f64(0.0), _f64(0.0)
    _check(ctx.lib.pc_alu_peaks(ctx.handle, ctypes.byref(a), ctypes.byref(b), _stream(stream)), "pc_alu_peaks")
    return a.value, b.value


def _check_noalloc_out(o, P, T, device):
    """The caller's outputs of pc_fields_noalloc: float32 [T][P][3] / [T][P], uint8 mask [T][P],
    contiguous, on the points' device."""
    shapes = {"E": (T, P, 3), "B": (T, P, 3), "phi": (T, P), "A": (T, P, 3), "mask": (T, P)}
    for k, t in o.items():
        if k not in shapes or t is None:
            continue
        want = torch.uint8 if k == "mask" else torch.float32
        if t.dtype != want or tuple(t.shape) != shapes[k] or not t.is_contiguous() or t.device != device:
            raise ValueError(f"pc_fields_noalloc: output {k} must be a contiguous {want} tensor of shape "
                             f"{shapes[k]} on {device}")


def pc_fields_noalloc(charges=None, dipoles=None, points=None, times=(0.0,), kind=PC_TOTAL, r_excl=0.0, out=None,
                      stream=None):
    """pc_fields_noalloc on the points' device: mixed precision, no allocation inside the library.

    `out` (float32 tensors, see alloc_field_out) should be allocated by the caller ahead of time.
    Every source tensor must sit on the points' device.
    """
    lib = load()
    dev = points.device
    if dev.type != "cuda":
        raise ValueError("pc_fields_noalloc: points must be a CUDA tensor")
    for src in (charges, dipoles):
        if src is None:
            continue
        for name, t in vars(src).items():
            if isinstance(t, torch.Tensor) and t.device != dev:
                raise ValueError(f"pc_fields_noalloc: source tensor {name} is on {t.device}, points on {dev}")
    P = int(points.shape[0])
    T = len(times)
    with torch.cuda.device(dev):
        o = alloc_field_out(P, T, PC_MIXED, dev) if out is None else out
        _check_noalloc_out(o, P, T, dev)
        tarr = (_f64 * T)(*[float(t) for t in times])
        chs = _charges_struct(charges)
        dps = _dipoles_struct(dipoles)
        st = lib.pc_fields_noalloc(ctypes.byref(chs) if chs else None, ctypes.byref(dps) if dps else None,
                                   _ptr(points), P, tarr, T, kind, float(r_excl), ctypes.byref(_out_struct(o)),
                                   _stream(stream))
    _check(st, "pc_fields_noalloc")
    return o
