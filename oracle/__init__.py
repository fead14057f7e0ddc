"""FP64 CPU oracle for the PyCharge hot path (arXiv 2107.12437) -- test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may import this
package.  It shares no code with the CUDA library (paper_2107_12437_gb300); both take their inputs
from workloads.py, which holds no method arithmetic.

  * pc_oracle.c     retarded-time bisection, Lienard-Wiechert fields (Jackson and Griffiths forms),
                    superposition, dipole charges, Lorentz-oscillator run (Algorithm 1, RK4); the
                    field sum once more in binary128 (fields_x) for points where dipoles cancel
  * theory.py       closed forms used as pins: Coulomb, uniform motion, Hertzian dipole, Larmor,
                    free-space Green's function rates (App. A), exact classical pole
  * fit.py          Levenberg-Marquardt fit of the kinetic energy to Eq. KE

Every function is FP64 except fields_x (binary128 throughout).  Parity pins live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_SRC = os.path.join(_HERE, "pc_oracle.c")

OK, ERR_ARG, ERR_HISTORY, ERR_VELOCITY, ERR_CAUSALITY, ERR_NOCONV = 0, 1, 2, 3, 4, 5
TOTAL, COULOMB, RADIATION = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile pc_oracle.c with gcc (plain -O2, no fast-math) into oracle/_build/liborc.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_P = ctypes.POINTER(ctypes.c_double)


class _Sources(ctypes.Structure):
    _fields_ = [
        ("M", ctypes.c_int32), ("S", ctypes.c_int64), ("t0", ctypes.c_double), ("dt", ctypes.c_double),
        ("q", _P), ("pos", _P), ("vel", _P), ("acc", _P), ("static_before", ctypes.c_int32),
        ("N", ctypes.c_int32), ("Sd", ctypes.c_int64), ("t0d", ctypes.c_double), ("dtd", ctypes.c_double),
        ("origin", _P), ("axis", _P), ("qd", _P), ("m1", _P), ("m2", _P),
        ("d", _P), ("d_dot", _P), ("d_ddot", _P), ("last_valid", ctypes.c_int64),
        ("org_pos", _P), ("org_vel", _P), ("org_acc", _P),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.orc_sources_size.restype = ctypes.c_int64
        assert _lib.orc_sources_size() == ctypes.sizeof(_Sources), "oracle struct layout mismatch"
        _lib.orc_fields.restype = ctypes.c_int
        _lib.orc_fields_x.restype = ctypes.c_int
        _lib.orc_retarded_delay.restype = ctypes.c_int
        _lib.orc_dipoles_run.restype = ctypes.c_int
        _lib.orc_dipoles_run_moving.restype = ctypes.c_int
        _lib.orc_fields_param.restype = ctypes.c_int
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_P) if a is not None else None


class _Keep:
    """Holds contiguous float64 copies alive while C reads them."""

    def __init__(self):
        self.arrs = []

    def __call__(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        self.arrs.append(a)
        return a


def _sources(charges=None, dipoles=None, keep=None, last_valid=-1):
    s = _Sources()
    s.last_valid = last_valid
    if charges is not None:
        s.M = charges.M
        s.S = charges.S
        s.t0, s.dt = charges.t0, charges.dt
        s.q = _ptr(keep(charges.q))
        s.pos = _ptr(keep(charges.pos))
        s.vel = _ptr(keep(charges.vel))
        s.acc = _ptr(keep(charges.acc))
        s.static_before = int(charges.static_before)
    if dipoles is not None:
        s.N = dipoles.N
        s.Sd = dipoles.S
        s.t0d, s.dtd = dipoles.t0, dipoles.dt
        s.origin = _ptr(keep(dipoles.origin))
        s.axis = _ptr(keep(dipoles.axis))
        s.qd = _ptr(keep(dipoles.q))
        s.m1 = _ptr(keep(dipoles.m1))
        s.m2 = _ptr(keep(dipoles.m2))
        s.d = _ptr(keep(dipoles.d))
        s.d_dot = _ptr(keep(dipoles.d_dot))
        s.d_ddot = _ptr(keep(dipoles.d_ddot))
    return s


def fields(points, times, charges=None, dipoles=None, kind=TOTAL, r_excl=0.0, nthreads=0):
    """E, B, A [T][P][3], phi [T][P], mask [T][P] and the oracle status (Sec. 2.2, Sec. 3.2)."""
    keep = _Keep()
    s = _sources(charges, dipoles, keep)
    pts = keep(np.asarray(points).reshape(-1, 3))
    tms = keep(np.atleast_1d(times))
    P, T = pts.shape[0], tms.shape[0]
    E = np.zeros((T, P, 3))
    B = np.zeros((T, P, 3))
    A = np.zeros((T, P, 3))
    phi = np.zeros((T, P))
    mask = np.zeros((T, P), dtype=np.uint8)
    scale = np.zeros((T, P, 8))
    st = lib().orc_fields(ctypes.byref(s), _ptr(pts), ctypes.c_int64(P), _ptr(tms), ctypes.c_int32(T),
                          ctypes.c_int32(kind), ctypes.c_double(r_excl), _ptr(E), _ptr(B), _ptr(phi), _ptr(A),
                          mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _ptr(scale), ctypes.c_int32(nthreads))
    # scale_charge: per-term magnitude sums over charges (E and B: |E_Coul| + |E_rad| of each term, B in
    # units of E/c); scale_source: |E|, |B|, |phi|, |A| summed over sources (a dipole's two charges
    # summed first).  They tell how strongly the superposition cancels.
    return dict(E=E, B=B, A=A, phi=phi, mask=mask, status=st,
                scale_charge=dict(E=scale[..., 0], B=scale[..., 1], phi=scale[..., 2], A=scale[..., 3]),
                scale_source=dict(E=scale[..., 4], B=scale[..., 5], phi=scale[..., 6], A=scale[..., 7]))


def fields_x(points, times, charges=None, dipoles=None, kind=TOTAL, r_excl=0.0, nthreads=0):
    """fields() with every intermediate in binary128 (orc_fields_x): E, B, A [T][P][3], phi [T][P],
    mask [T][P] and the status.  The +-q pair of a dipole no longer costs digits, so these are the
    fields of the discrete history to float64 rounding.  Fixed dipole origins only."""
    keep = _Keep()
    s = _sources(charges, dipoles, keep)
    pts = keep(np.asarray(points).reshape(-1, 3))
    tms = keep(np.atleast_1d(times))
    P, T = pts.shape[0], tms.shape[0]
    E = np.zeros((T, P, 3))
    B = np.zeros((T, P, 3))
    A = np.zeros((T, P, 3))
    phi = np.zeros((T, P))
    mask = np.zeros((T, P), dtype=np.uint8)
    st = lib().orc_fields_x(ctypes.byref(s), _ptr(pts), ctypes.c_int64(P), _ptr(tms), ctypes.c_int32(T),
                            ctypes.c_int32(kind), ctypes.c_double(r_excl), _ptr(E), _ptr(B), _ptr(phi), _ptr(A),
                            mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), ctypes.c_int32(nthreads))
    return dict(E=E, B=B, A=A, phi=phi, mask=mask, status=st)


def retarded_delay(c, t, r, charges=None, dipoles=None):
    """Delay t - t' of charge c seen from r at time t (Eq. ret_t) and the oracle status."""
    keep = _Keep()
    s = _sources(charges, dipoles, keep)
    rr = keep(np.asarray(r, dtype=np.float64))
    tau = ctypes.c_double(0.0)
    st = lib().orc_retarded_delay(ctypes.byref(s), ctypes.c_int(c), ctypes.c_double(t), _ptr(rr), ctypes.byref(tau))
    return tau.value, st


def lw_jackson(q, aR, v, acc):
    """Coulomb E, radiation E, phi, A of one charge (Eqs. V, A, E, ECoulomb, Eradiation)."""
    keep = _Keep()
    a, vv, ac = keep(aR), keep(v), keep(acc)
    Ec, Er, A = np.zeros(3), np.zeros(3), np.zeros(3)
    phi = ctypes.c_double(0.0)
    lib().orc_lw_jackson(ctypes.c_double(q), _ptr(a), _ptr(vv), _ptr(ac), _ptr(Ec), _ptr(Er), ctypes.byref(phi),
                         _ptr(A))
    return Ec, Er, phi.value, A


def lw_griffiths(q, aR, v, acc):
    """E and B of one charge in Griffiths' notation (cross-check of lw_jackson)."""
    keep = _Keep()
    a, vv, ac = keep(aR), keep(v), keep(acc)
    E, B = np.zeros(3), np.zeros(3)
    lib().orc_lw_griffiths(ctypes.c_double(q), _ptr(a), _ptr(vv), _ptr(ac), _ptr(E), _ptr(B))
    return E, B


def dipoles_run(cfg, b=0, n_steps=None, ed_mode=0, v_max=None, nthreads=0, motion=None):
    """Algorithm 1 for configuration b of a workloads.LOConfig.

    motion: optional (pos, vel, acc) [B][N][2 n_steps + 1][3] origin trajectories at the half steps
    (moving dipoles, Sec. 4.3).  Returns dict d, d_dot, d_ddot, energy, Ed [N][n_steps+1] and status.
    """
    from workloads import C as _c

    n_steps = cfg.n_steps if n_steps is None else n_steps
    v_max = _c / 100.0 if v_max is None else v_max
    keep = _Keep()
    N = cfg.N
    S = n_steps + 1
    d = np.zeros((N, S))
    dd = np.zeros((N, S))
    ddd = np.zeros((N, S))
    en = np.zeros((N, S))
    Ed = np.zeros((N, S))
    mo = [None, None, None]
    if motion is not None:
        H = 2 * n_steps + 1
        mo = [keep(np.asarray(x)[b, :, :H]) for x in motion]
    st = lib().orc_dipoles_run_moving(
        ctypes.c_int32(N), _ptr(keep(cfg.origin[b])), _ptr(keep(cfg.axis[b])), _ptr(keep(cfg.q[b])),
        _ptr(keep(cfg.m1[b])), _ptr(keep(cfg.m2[b])), _ptr(keep(cfg.omega0[b])), _ptr(keep(cfg.d0[b])),
        _ptr(mo[0]), _ptr(mo[1]), _ptr(mo[2]),
        ctypes.c_double(cfg.dt), ctypes.c_int64(n_steps), ctypes.c_double(v_max), ctypes.c_int32(ed_mode),
        _ptr(d), _ptr(dd), _ptr(ddd), _ptr(en), _ptr(Ed), ctypes.c_int32(nthreads))
    return dict(d=d, d_dot=dd, d_ddot=ddd, energy=en, Ed=Ed, status=st)


def fields_param(points, times, kind, q, par, fkind=TOTAL, r_excl=0.0, nthreads=0):
    """E, B, A [T][P][3], phi [T][P], mask [T][P] of point charges on analytic trajectories
    (kind [M] in 0..3, q [M], par [M][12]; the layouts are those of orc_fields_param)."""
    keep = _Keep()
    pts = keep(np.asarray(points).reshape(-1, 3))
    tms = keep(np.atleast_1d(times))
    P, T = pts.shape[0], tms.shape[0]
    kd = np.ascontiguousarray(kind, dtype=np.int32)
    qq = keep(q)
    pr = keep(np.asarray(par).reshape(-1, 12))
    E = np.zeros((T, P, 3))
    B = np.zeros((T, P, 3))
    A = np.zeros((T, P, 3))
    phi = np.zeros((T, P))
    mask = np.zeros((T, P), dtype=np.uint8)
    st = lib().orc_fields_param(
        ctypes.c_int32(kd.size), kd.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _ptr(qq), _ptr(pr), _ptr(pts),
        ctypes.c_int64(P), _ptr(tms), ctypes.c_int32(T), ctypes.c_int32(fkind), ctypes.c_double(r_excl), _ptr(E),
        _ptr(B), _ptr(phi), _ptr(A), mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), ctypes.c_int32(nthreads))
    return dict(E=E, B=B, A=A, phi=phi, mask=mask, status=st)
