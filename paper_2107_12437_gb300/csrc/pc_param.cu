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

// Root of g(t') = c (t - t') - |r - r(t')| (decreasing while the charge is slower than light):
// a bracket [lo, t] with g(lo) >= 0 by doubling the look-back, then Newton steps with
// g'(t') = -c + n.v, any step that leaves the bracket replaced by bisection.
__device__ int param_retarded(int kind, const double *p, double t, const double r[3], double *tp) {
  double rc[3], v[3], a[3];
  param_state(kind, p, t, rc, v, a);
  double D[3] = {r[0] - rc[0], r[1] - rc[1], r[2] - rc[2]};
  double span = sqrt(dot3(D, D)) / kC;
  double lo = t - span, hi = t;
  bool found = false;
  for (int it = 0; it < 64; ++it) {
    param_state(kind, p, lo, rc, v, a);
    const double E[3] = {r[0] - rc[0], r[1] - rc[1], r[2] - rc[2]};
    if (kC * (t - lo) - sqrt(dot3(E, E)) >= 0.0) {
      found = true;
      break;
    }
    span = 2.0 * span + 1e-30;
    lo = t - span;
  }
  if (!found) return PC_ERR_NOCONV;
  double x = lo;
  for (int it = 0; it < 100; ++it) {
    param_state(kind, p, x, rc, v, a);
    const double E[3] = {r[0] - rc[0], r[1] - rc[1], r[2] - rc[2]};
    const double R = sqrt(dot3(E, E));
    const double g = kC * (t - x) - R;
    if (g >= 0.0) lo = x;
    else hi = x;
    const double dg = -kC + dot3(E, v) / R;
    double xn = x - g / dg;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    const double tol = 2e-16 * (fabs(t) + fabs(t - x)) + 1e-300;
    if (fabs(xn - x) <= tol || !(hi - lo > tol)) {
      *tp = xn;
      return 0;
    }
    x = xn;
  }
  return PC_ERR_NOCONV;
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
    double tp;
    const int e = param_retarded(kd, p, t, r, &tp);
    if (e) {
      set_status(L.status, e);
      return;
    }
    double rc[3], v[3], a[3];
    param_state(kd, p, tp, rc, v, a);
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
