// Fields of point charges on analytic trajectories (float64): the retarded time is solved on the
// exact trajectory r(t) (Eq. ret_t) by a bracketed Newton iteration, and the Lienard-Wiechert
// fields (Eqs. V, A, E, B) use the exact velocity and acceleration, so no history interpolation
// enters.  The trajectories are those of the paper's predefined charges (Sec. 2.2, Sec. 3.1):
// stationary, oscillating along a line, orbiting on a circle, and linearly accelerating.
#include <string.h>

#include "pc_internal.cuh"
#include "pc_lw_f64.cuh"

namespace pc {

constexpr int kParamMaxT = 32;

struct ParamLaunch {
  int32_t M;
  const int32_t *kind;
  const double *q, *par;
  const double *pts;
  int64_t P;
  int32_t T;
  int64_t frame0;
  double times[kParamMaxT];
  double r_excl;
  pc_field_out out;
  int *status;
};

// position, velocity and acceleration of a parametric charge at time t (layouts in the header)
__device__ __forceinline__ void param_state(int kind, const double *p, double t, double r[3], double v[3],
                                            double a[3]) {
  if (kind == PC_TRAJ_OSCILLATING) {
    double sn, cs;
    sincos(p[7] * t + p[8], &sn, &cs);
    const double amp = p[6], w = p[7];
    for (int i = 0; i < 3; ++i) {
      r[i] = p[i] + amp * cs * p[3 + i];
      v[i] = -amp * w * sn * p[3 + i];
      a[i] = -amp * w * w * cs * p[3 + i];
    }
  } else if (kind == PC_TRAJ_CIRCULAR) {
    double sn, cs;
    sincos(p[10] * t + p[11], &sn, &cs);
    const double rad = p[9], w = p[10];
    for (int i = 0; i < 3; ++i) {
      const double e = cs * p[3 + i] + sn * p[6 + i];
      r[i] = p[i] + rad * e;
      v[i] = rad * w * (-sn * p[3 + i] + cs * p[6 + i]);
      a[i] = -rad * w * w * e;
    }
  } else if (kind == PC_TRAJ_ACCELERATING) {
    const double s = t - p[9];
    const bool on = s >= 0.0;
    for (int i = 0; i < 3; ++i) {
      r[i] = p[i] + p[3 + i] * s + (on ? 0.5 * p[6 + i] * s * s : 0.0);
      v[i] = p[3 + i] + (on ? p[6 + i] * s : 0.0);
      a[i] = on ? p[6 + i] : 0.0;
    }
  } else {  // stationary
    for (int i = 0; i < 3; ++i) {
      r[i] = p[i];
      v[i] = 0.0;
      a[i] = 0.0;
    }
  }
}

// Root of g(t') = c (t - t') - |r - r(t')| (decreasing while the charge is slower than light) by
// Newton steps with g'(t') = -c + n.v inside a bracket [lo, hi] (g(lo) >= 0 >= g(hi)); a step that
// leaves the bracket is replaced by the false-position point of the bracket (bisection if that
// rounds onto an end).  First guess: the retarded time of a charge that keeps its velocity at t
// (exact for uniform motion).  Converged when the Newton step is below 1e-15 (|t| + |t - t'|), a
// few units in the last place (g itself is only known to rounding, and a tighter test would chase
// that noise); that last step is then taken, so the root is exact to rounding.  Returns the root
// and the state there.
__device__ int param_retarded(int kind, const double *p, double t, const double r[3], double *tp, double rc[3],
                              double v[3], double a[3]) {
  constexpr double kTol = 1e-15;
  param_state(kind, p, t, rc, v, a);
  const double D[3] = {r[0] - rc[0], r[1] - rc[1], r[2] - rc[2]};
  const double R0 = sqrt(dot3(D, D));
  // c^2 tau^2 = |D + v tau|^2: (c^2 - v^2) tau^2 - 2 (D.v) tau - R0^2 = 0, the positive root in
  // the form without cancellation
  const double Dv = dot3(D, v), c2v2 = kC * kC - dot3(v, v);
  double tau = R0 / kC;
  if (c2v2 > 0.0) {
    const double sq = sqrt(Dv * Dv + c2v2 * R0 * R0);
    tau = Dv >= 0.0 ? (Dv + sq) / c2v2 : (R0 * R0) / (sq - Dv);
  }
  double x = t - tau;
  param_state(kind, p, x, rc, v, a);
  double E[3] = {r[0] - rc[0], r[1] - rc[1], r[2] - rc[2]};
  double R = sqrt(dot3(E, E));
  double g = kC * (t - x) - R;
  double lo = x, hi = t, glo = g, ghi = -R0;
  if (g < 0.0) {
    hi = x;
    ghi = g;
    if (R > 0.0) {
      const double step = g / (-kC + dot3(E, v) / R);
      if (fabs(step) <= kTol * (fabs(t) + fabs(t - x))) {
        // the guess is within one small Newton step of the root
        *tp = x - step;
        param_state(kind, p, *tp, rc, v, a);
        return 0;
      }
    }
    // the root lies further back: double the look-back until g >= 0
    double span = fmax(2.0 * tau, R0 / kC) + 1e-30;
    bool found = false;
    for (int it = 0; it < 64; ++it) {
      x = t - span;
      param_state(kind, p, x, rc, v, a);
      for (int i = 0; i < 3; ++i) E[i] = r[i] - rc[i];
      R = sqrt(dot3(E, E));
      g = kC * (t - x) - R;
      if (g >= 0.0) {
        found = true;
        break;
      }
      hi = x;
      ghi = g;
      span *= 2.0;
    }
    if (!found) return PC_ERR_NOCONV;
    lo = x;
    glo = g;
  }
  for (int it = 0;; ++it) {
    if (g >= 0.0) {
      lo = x;
      glo = g;
    } else {
      hi = x;
      ghi = g;
    }
    if (!(R > 0.0)) break;  // the point sits on the charge at x (masked by the field sum)
    const double step = g / (-kC + dot3(E, v) / R);
    const double tol = kTol * (fabs(t) + fabs(t - x)) + 1e-300;
    if (fabs(step) <= tol) {
      x -= step;
      param_state(kind, p, x, rc, v, a);
      break;
    }
    if (!(hi - lo > tol)) break;
    if (it == 100) return PC_ERR_NOCONV;
    double xn = x - step;
    if (!(xn > lo && xn < hi)) {
      xn = lo + (hi - lo) * (glo / (glo - ghi));
      if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    }
    x = xn;
    param_state(kind, p, x, rc, v, a);
    for (int i = 0; i < 3; ++i) E[i] = r[i] - rc[i];
    R = sqrt(dot3(E, E));
    g = kC * (t - x) - R;
  }
  *tp = x;
  return 0;
}

template <int KIND>
__global__ void __launch_bounds__(128) fields_param_kernel(const ParamLaunch L) {
  const int64_t pi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  if (pi >= L.P || f >= L.T) return;
  const double r[3] = {L.pts[3 * pi], L.pts[3 * pi + 1], L.pts[3 * pi + 2]};
  const double t = L.times[f];
  double E[3] = {0, 0, 0}, B[3] = {0, 0, 0}, A[3] = {0, 0, 0}, phi = 0.0;
  uint8_t mask = 0;
  for (int c = 0; c < L.M; ++c) {
    const int kd = __ldg(L.kind + c);
    if (kd < PC_TRAJ_STATIONARY || kd > PC_TRAJ_ACCELERATING) {
      set_status(L.status, PC_ERR_ARG);
      return;
    }
    const double *p = L.par + 12 * c;
    double tp, rc[3], v[3], a[3];
    const int e = param_retarded(kd, p, t, r, &tp, rc, v, a);
    if (e) {
      set_status(L.status, e);
      return;
    }
    const double av[3] = {r[0] - rc[0], r[1] - rc[1], r[2] - rc[2]};
    lw_add_f64<KIND>(__ldg(L.q + c), av, v, a, L.r_excl, E, B, &phi, A, &mask);
  }
  const int64_t o = (L.frame0 + f) * L.P + pi;
  if (L.out.E)
    for (int i = 0; i < 3; ++i) ((double *)L.out.E)[3 * o + i] = E[i];
  if (L.out.B)
    for (int i = 0; i < 3; ++i) ((double *)L.out.B)[3 * o + i] = B[i];
  if (L.out.A)
    for (int i = 0; i < 3; ++i) ((double *)L.out.A)[3 * o + i] = A[i];
  if (L.out.phi) ((double *)L.out.phi)[o] = phi;
  if (L.out.mask) L.out.mask[o] = mask;
}

}  // namespace pc

extern "C" pc_status pc_fields_param(pc_ctx *ctx, const pc_param_charges *ch, const double *points, int64_t P,
                                     const double *times, int32_t T, int32_t kind, double r_excl,
                                     const pc_field_out *out, void *stream) {
  if (!ctx || !ch || !out || !times || T < 1 || P < 0 || ch->M < 1) return PC_ERR_ARG;
  if (!ch->kind || !ch->q || !ch->par) return PC_ERR_ARG;
  if (kind < PC_TOTAL || kind > PC_RADIATION || !(r_excl >= 0.0)) return PC_ERR_ARG;
  for (int i = 0; i < T; ++i)
    if (!isfinite(times[i])) return PC_ERR_ARG;
  if (P == 0) return PC_OK;
  if (!points) return PC_ERR_ARG;
  pc::DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  pc_status bs = pc::begin_call(ctx, st);
  if (bs != PC_OK) return bs;
  pc::ParamLaunch L;
  memset(&L, 0, sizeof(L));
  L.M = ch->M;
  L.kind = ch->kind;
  L.q = ch->q;
  L.par = ch->par;
  L.pts = points;
  L.P = P;
  L.r_excl = r_excl;
  L.out = *out;
  L.status = ctx->d_status;
  for (int32_t f0 = 0; f0 < T; f0 += pc::kParamMaxT) {
    L.T = T - f0 < pc::kParamMaxT ? T - f0 : pc::kParamMaxT;
    L.frame0 = f0;
    for (int i = 0; i < L.T; ++i) L.times[i] = times[f0 + i];
    const dim3 grid((unsigned)((P + 127) / 128), (unsigned)L.T);
    if (kind == PC_TOTAL) pc::fields_param_kernel<PC_TOTAL><<<grid, 128, 0, st>>>(L);
    else if (kind == PC_COULOMB) pc::fields_param_kernel<PC_COULOMB><<<grid, 128, 0, st>>>(L);
    else pc::fields_param_kernel<PC_RADIATION><<<grid, 128, 0, st>>>(L);
  }
  return pc::end_call(ctx, st);
}
