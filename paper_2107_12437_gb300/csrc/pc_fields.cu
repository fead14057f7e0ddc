// Retarded Lienard-Wiechert field sum (arXiv 2107.12437, Sec. 2.1-2.2) on sm_103a.
//
// Two paths:
//   PC_F64   one thread per (point, time); every charge's retarded time is found by solving, on one
//            segment of its piecewise-linear history, the quadratic c^2 (t - t')^2 = |r - r_s(t')|^2
//            (Eq. ret_t with linear interpolation, Sec. 3.1), moving to the segment the root points
//            to until it lies inside; fields from Griffiths' form of Eqs. E, B, V, A in float64, a
//            dipole's two charges together in the difference form of the mixed path (below).
//   PC_MIXED a CTA owns a tile of points.  Per (tile, source) the float64 distance from the tile's
//            anchor point to the source reference gives the integer part of the retarded sample
//            index; per (point, source) everything else runs in float32 on offsets (lengths in
//            units of c*dt, so a delay in samples equals a distance).  The two charges of a dipole
//            are evaluated together in difference form: the net field q[E(x+) - E(x-)] is built
//            from differences of the scalar coefficients of the Lienard-Wiechert field that carry
//            no cancellation, so the s/R loss of the +-q pair (s = charge separation) does not
//            appear.  Contributions are summed in groups of 32 (the two-point kernel: 16) and the
//            group sums are added with Kahan compensation.
#include <stdio.h>

#include <algorithm>
#include <type_traits>

#include "pc_internal.cuh"
#include "pc_lw_f32.cuh"
#include "pc_lw_f32x2.cuh"
#include "pc_lw_f64.cuh"

namespace pc {

constexpr int kMaxT = 32;        // times per launch (the host splits longer lists)
constexpr int kMixThreads = 256; // points per CTA in the mixed path
constexpr int kChunk = 64;       // sources staged in shared memory at a time (the largest stage)
// per-chunk bit mask of the pairs that left the fast path: 32 or 64 sources per stage
template <int CH>
struct SlowMask {
  using T = typename std::conditional<(CH <= 32), unsigned, unsigned long long>::type;
  static __device__ __forceinline__ T bit(int j) { return (T)1 << j; }
  static __device__ __forceinline__ int first(T m) {
    if constexpr (CH <= 32) return __ffs((int)m) - 1;
    else return __ffsll((long long)m) - 1;
  }
};
// a dipole closer than kNearL c*dt to a point whose near field there cancels by more than kCancel
// (dipole_cancellation) is summed in float64 instead
constexpr float kNearL = 400.f;
constexpr float kCancel = 6.f;

struct Points {
  const double *list;  // [P][3] or null for a plane
  double o[3], eu[3], ev[3];
  int64_t nu, nv;
  int64_t P;
};

__device__ __forceinline__ void point_at(const Points &pd, int64_t p, double r[3]) {
  if (pd.list) {
    r[0] = pd.list[3 * p];
    r[1] = pd.list[3 * p + 1];
    r[2] = pd.list[3 * p + 2];
  } else {
    double iu = (double)(p / pd.nv), iv = (double)(p % pd.nv);
    r[0] = pd.o[0] + iu * pd.eu[0] + iv * pd.ev[0];
    r[1] = pd.o[1] + iu * pd.eu[1] + iv * pd.ev[1];
    r[2] = pd.o[2] + iu * pd.eu[2] + iv * pd.ev[2];
  }
}

struct Sources {
  // point charges
  int32_t M;
  int64_t S;
  double t0, dt;
  const double *q, *pos, *vel, *acc;
  int32_t static_before;
  // dipoles
  int32_t N;
  int64_t Sd;
  double t0d, dtd;
  const double *origin, *axis, *qd, *m1, *m2, *d, *dd, *ddd;
};

struct Outs {
  void *E, *B, *phi, *A;
  uint8_t *mask;
};

struct Launch {
  Points pts;
  Sources src;
  Outs out;
  int32_t T;            // times in this launch
  int64_t frame0;       // output frame of times[0]
  double times[kMaxT];
  double r_excl;
  int *status;
  // mixed path: float32 mirrors and per-charge references
  const float4 *Hd;     // [N][Sd] (d/(qL), d'/(qc), d'' dt/(qc), 0)
  const float4 *Hc;     // [M][S][3]: offset/L, v/c, a dt/c
  const double *cref;   // [M][3] reference position (sample 0)
  int32_t tile_shift;   // plane tiles of (256 >> tile_shift) rows x (1 << tile_shift) columns
  // mixed path, set on the host: each frame's time in dipole samples, 1/(c dt) of the dipole
  // history, and per dipole two float4 records (axis x, y, z, q/e), (m2/(m1+m2), m1/(m1+m2), 0, 0)
  double uf[kMaxT];
  float uf_hi[kMaxT], uf_lo[kMaxT];  // the same as float-float
  double iLd;
  float eu_L[3], ev_L[3];            // plane steps in units of c dt (dipole history)
  const float4 *srcf;
  float unit[4];                     // SI units of the float32 sums of E, B, phi, A
  // loop constants of the dipole sum, read from the parameter bank rather than held in registers:
  // r_excl in units of c dt, that plus 1.5 (the fast path's distance bound), and the number of
  // interior segments S - 3 (fast segments 1 <= j <= S - 3)
  float rex, rex_fast;
  unsigned jlim;
  // point charges: each frame's time in their samples, 1/(c dt) of their history, and the scales
  // of their float32 terms to the output unit (E, phi)
  double ufc[kMaxT];
  double iLc;
  float sE, sP;
};

// the float32 outputs' units: E in k_e e / L^2, B in k_e e / (L^2 c), phi in k_e e / L,
// A in k_e e / (L c), L = c dt of the dipoles (of the point charges when there are no dipoles)
__host__ inline void set_units(Launch &L) {
  const double Lref = (L.src.N > 0) ? kC * L.src.dtd : kC * L.src.dt;
  if (L.src.N > 0) {
    L.rex = (float)(L.r_excl * L.iLd);
    L.rex_fast = L.rex + 1.5f;
    L.jlim = L.src.Sd > 3 ? (unsigned)(L.src.Sd - 3) : 0u;
  }
  const double kE2 = kKe * kE / (Lref * Lref), kP = kKe * kE / Lref;
  L.unit[0] = (float)kE2;
  L.unit[1] = (float)(kE2 / kC);
  L.unit[2] = (float)kP;
  L.unit[3] = (float)(kP / kC);
  if (L.src.M > 0) {
    const double Lch = kC * L.src.dt;
    L.iLc = 1.0 / Lch;
    L.sE = (float)((Lref / Lch) * (Lref / Lch));
    L.sP = (float)(Lref / Lch);
  }
}

// the frames of one launch: their times and, for the dipoles, the times in samples
__host__ inline void set_frames(Launch &L, const double *times, int32_t f0, int32_t n) {
  L.T = n;
  L.frame0 = f0;
  for (int i = 0; i < n; ++i) {
    L.times[i] = times[f0 + i];
    L.uf[i] = L.src.N > 0 ? (times[f0 + i] - L.src.t0d) / L.src.dtd : 0.0;
    L.ufc[i] = L.src.M > 0 ? (times[f0 + i] - L.src.t0) / L.src.dt : 0.0;
    L.uf_hi[i] = (float)L.uf[i];
    L.uf_lo[i] = (float)(L.uf[i] - (double)L.uf_hi[i]);
  }
}

// ================================================================================================
// float64 path
// ================================================================================================
template <int KIND>
__global__ void __launch_bounds__(128) fields_f64_kernel(const Launch L) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int f = blockIdx.y;
  if (p >= L.pts.P || f >= L.T) return;
  double r[3];
  point_at(L.pts, p, r);
  const double t = L.times[f];
  double E[3] = {0, 0, 0}, B[3] = {0, 0, 0}, A[3] = {0, 0, 0}, phi = 0.0;
  uint8_t mask = 0;
  int err = 0;
  const Sources &s = L.src;
  // ---- point charges ----
  if (s.M > 0) {
    const double u = (t - s.t0) / s.dt, cdt = kC * s.dt;
    for (int c = 0; c < s.M && !err; ++c) {
      TrajF64 tr;
      tr.dipole = false;
      tr.pos = s.pos + (size_t)c * s.S * 3;
      tr.vel = s.vel + (size_t)c * s.S * 3;
      tr.acc = s.acc + (size_t)c * s.S * 3;
      int64_t kr = (int64_t)floor(u);
      kr = kr < 0 ? 0 : (kr > s.S - 1 ? s.S - 1 : kr);
      double pr[3];
      tr.p(kr, pr);
      double dv[3] = {r[0] - pr[0], r[1] - pr[1], r[2] - pr[2]};
      double tau0 = sqrt(dot3(dv, dv)) * L.iLc;
      int64_t k;
      double th;
      err = solve_f64(tr, s.S, s.static_before, r, u, cdt, (int64_t)floor(u - tau0), &k, &th);
      if (err) break;
      double p0[3], v[3], a[3];
      if (k < 0) {
        tr.p(0, p0);
        v[0] = v[1] = v[2] = 0.0;
        a[0] = a[1] = a[2] = 0.0;
      } else {
        double p1[3], v1[3], a1[3];
        tr.p(k, p0);
        tr.p(k + 1, p1);
        tr.va(k, v, a);
        tr.va(k + 1, v1, a1);
        for (int i = 0; i < 3; ++i) {
          p0[i] += th * (p1[i] - p0[i]);
          v[i] += th * (v1[i] - v[i]);
          a[i] += th * (a1[i] - a[i]);
        }
      }
      double av[3] = {r[0] - p0[0], r[1] - p0[1], r[2] - p0[2]};
      lw_add_f64<KIND>(s.q[c], av, v, a, L.r_excl, E, B, &phi, A, &mask);
    }
  }
  // ---- dipoles: the two charges of each (Eqs. r_1, r_2) in difference form ----
  // Each charge's retarded time is the exact root on its own history segment (offsets from the
  // dipole centre in units of c dt, times in samples); the net field q [F(x+) - F(x-)] is formed
  // from differences of the Lienard-Wiechert coefficients (pc_lw_f32.cuh, dipole_pair), so the
  // R/s cancellation of the +-q pair costs no digits.
  if (s.N > 0 && !err) {
    const double u = (t - s.t0d) / s.dtd, iLd = L.iLd;
    const double rex = L.r_excl * iLd;
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int j = 0; j < s.N && !err; ++j) {
      const double q = s.qd[j], m1 = s.m1[j], m2 = s.m2[j];
      const double rx = (r[0] - s.origin[3 * j]) * iLd, ry = (r[1] - s.origin[3 * j + 1]) * iLd,
                   rz = (r[2] - s.origin[3 * j + 2]) * iLd;
      const double rn = sqrt(rx * rx + ry * ry + rz * rz);
      const double px = s.axis[3 * j], py = s.axis[3 * j + 1], pz = s.axis[3 * j + 2];
      const double rp = rx * px + ry * py + rz * pz;
      const double x = u - rn;
      const double fl = floor(x);
      HistF64 H;
      H.d = s.d + (size_t)j * s.Sd;
      H.dd = s.dd + (size_t)j * s.Sd;
      H.ddd = s.ddd + (size_t)j * s.Sd;
      const double iq = 1.0 / q, imm = 1.0 / (m1 + m2);
      H.sx = iq * iLd;
      H.sv = iq * (1.0 / kC);
      H.sa = iq * (s.dtd / kC);
      double Xp, Vp, Ap, dp, Xm, Vm, Am, dm;
      const double mup = m2 * imm, mum = m1 * imm;
      err = dip_pair_exact<double, HistF64>(H, (int)s.Sd, (int)fl, x - fl, rn, rp, mup, mum, Xp, Vp, Ap, dp, Xm, Vm,
                                           Am, dm, 1e-9);
      if (err) break;
      dipole_pair<KIND, double>(rx, ry, rz, rn, px, py, pz, rp, mup, mum, q * (1.0 / kE), Xp, Vp, Ap, dp, Xm, Vm, Am,
                                dm, rex, acc, mask);
    }
    // units of the difference form: E in k_e e / L^2, B in k_e e / (L^2 c), phi in k_e e / L,
    // A in k_e e / (L c), L = c dt of the dipole history
    const double uP = kKe * kE * iLd, uE = uP * iLd;
    for (int i = 0; i < 3; ++i) {
      E[i] += uE * acc[i];
      B[i] += uE * (1.0 / kC) * acc[3 + i];
      A[i] += uP * (1.0 / kC) * acc[7 + i];
    }
    phi += uP * acc[6];
  }
  if (err) {
    set_status(L.status, err);
    return;
  }
  const int64_t o = (L.frame0 + f) * L.pts.P + p;
  if (L.out.E) {
    double *e = (double *)L.out.E + 3 * o;
    e[0] = E[0];
    e[1] = E[1];
    e[2] = E[2];
  }
  if (L.out.B) {
    double *b = (double *)L.out.B + 3 * o;
    b[0] = B[0];
    b[1] = B[1];
    b[2] = B[2];
  }
  if (L.out.phi) ((double *)L.out.phi)[o] = phi;
  if (L.out.A) {
    double *a = (double *)L.out.A + 3 * o;
    a[0] = A[0];
    a[1] = A[1];
    a[2] = A[2];
  }
  if (L.out.mask) L.out.mask[o] = mask;
}

// ================================================================================================
// mixed path
// ================================================================================================
__global__ void prep_dipoles_f32(const Sources s, float4 *H, float4 *srcf) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t n = (int64_t)s.N * s.Sd;
  if (i >= n) return;
  int j = (int)(i / s.Sd);
  const double q = s.qd[j];
  const double Lc = kC * s.dtd;
  H[i] = make_float4((float)(s.d[i] / (q * Lc)), (float)(s.dd[i] / (q * kC)), (float)(s.ddd[i] * s.dtd / (q * kC)),
                     0.f);
  if (i % s.Sd == 0) {
    const double m1 = s.m1[j], m2 = s.m2[j];
    srcf[4 * j] = make_float4((float)s.axis[3 * j], (float)s.axis[3 * j + 1], (float)s.axis[3 * j + 2], (float)(q / kE));
    srcf[4 * j + 1] = make_float4((float)(m2 / (m1 + m2)), (float)(m1 / (m1 + m2)), 0.f, 0.f);
    float hi[3], lo[3];
    for (int c = 0; c < 3; ++c) {
      const double x = s.origin[3 * j + c] / Lc;
      hi[c] = (float)x;
      lo[c] = (float)(x - (double)hi[c]);
    }
    srcf[4 * j + 2] = make_float4(hi[0], hi[1], hi[2], 0.f);
    srcf[4 * j + 3] = make_float4(lo[0], lo[1], lo[2], 0.f);
  }
}

__global__ void prep_charges_f32(const Sources s, float4 *H, double *cref) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t n = (int64_t)s.M * s.S;
  if (i >= n) return;
  int c = (int)(i / s.S);
  const double *p0 = s.pos + (size_t)c * s.S * 3;
  const double Lc = kC * s.dt;
  const double *p = s.pos + 3 * i, *v = s.vel + 3 * i, *a = s.acc + 3 * i;
  H[3 * i + 0] = make_float4((float)((p[0] - p0[0]) / Lc), (float)((p[1] - p0[1]) / Lc), (float)((p[2] - p0[2]) / Lc),
                             0.f);
  H[3 * i + 1] = make_float4((float)(v[0] / kC), (float)(v[1] / kC), (float)(v[2] / kC), 0.f);
  H[3 * i + 2] = make_float4((float)(a[0] * s.dt / kC), (float)(a[1] * s.dt / kC), (float)(a[2] * s.dt / kC), 0.f);
  if (i % s.S == 0) {
    cref[3 * c] = p0[0];
    cref[3 * c + 1] = p0[1];
    cref[3 * c + 2] = p0[2];
  }
}

// ---- float-float arithmetic (error-free transformations with fma) for list-mode delays ----
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = ff_two_sum(a.hi, b.hi);
  float lo = s.lo + a.lo + b.lo;
  return ff_two_sum(s.hi, lo);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return ff_two_sum(p, e);
}
__device__ __forceinline__ ff ff_sqrt(ff a) {
  float s0 = sqrtf(a.hi);
  if (!(s0 > 0.f)) return {0.f, 0.f};
  float r = fmaf(-s0, s0, a.hi) + a.lo;  // a - s0^2
  return ff_two_sum(s0, r / (2.f * s0));
}
__device__ __forceinline__ ff ff_from_double(double x) {
  float hi = (float)x;
  return {hi, (float)(x - (double)hi)};
}

// Both charges of dipole j in float64, added to the float32 accumulators in their units.  Used for
// points within kNearL of the dipole, where the float32 difference form loses accuracy: there the
// sampled position X and velocity V at the retarded time combine as X + R V, which nearly vanishes
// whenever the dipole's instantaneous moment crosses zero.  Exact per-charge roots (no segment
// extension), the same difference form in double.
template <int KIND>
__device__ __noinline__ int near_dipole_f64(const Sources &s, int j, const double r[3], double u, double Ld,
                                               double r_excl, float *part, uint8_t *mask) {
  const double q = s.qd[j], m1 = s.m1[j], m2 = s.m2[j];
  const double rx = (r[0] - s.origin[3 * j]) / Ld, ry = (r[1] - s.origin[3 * j + 1]) / Ld,
               rz = (r[2] - s.origin[3 * j + 2]) / Ld;
  const double rn = sqrt(rx * rx + ry * ry + rz * rz);
  const double px = s.axis[3 * j], py = s.axis[3 * j + 1], pz = s.axis[3 * j + 2];
  const double rp = rx * px + ry * py + rz * pz;
  const double x = u - rn;
  const double fl = floor(x);
  HistF64 H;
  H.d = s.d + (size_t)j * s.Sd;
  H.dd = s.dd + (size_t)j * s.Sd;
  H.ddd = s.ddd + (size_t)j * s.Sd;
  H.sx = 1.0 / (q * Ld);
  H.sv = 1.0 / (q * kC);
  H.sa = s.dtd / (q * kC);
  double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  const int e = dipole_net<KIND, double, HistF64>(H, (int)s.Sd, (int)fl, x - fl, rx, ry, rz, rn, px, py, pz, rp,
                                                  m2 / (m1 + m2), m1 / (m1 + m2), q / kE, r_excl / Ld, true, acc,
                                                  *mask);
  if (e) return e;
#pragma unroll
  for (int i = 0; i < 10; ++i) part[i] += (float)acc[i];
  return 0;
}

// A dipole pair the inner loop could not take on its fast path (a charge offset beyond the shared
// segment, a point close to a charge, or an ill-conditioned near field): exact float32 roots of
// both charges, then the float32 difference form, or the float64 near path where the near field
// cancels.  Kept out of line so that the inner loop makes no calls.
template <int KIND>
__device__ __noinline__ int slow_dipole(const Sources &s, int j, const float4 *hist, int S, int kb, float xc, float rx,
                                        float ry, float rz, float rn, float4 ax, float mup, float mum, float rex,
                                        const double r[3], double u, double Ld, double r_excl, float *part,
                                        uint8_t *mask) {
  const float rp = rx * ax.x + ry * ax.y + rz * ax.z;
  const HistF32 H{hist};
  float Xp, Vp, Ap, dp, Xm, Vm, Am, dm;
  const int e = dipole_states<float, HistF32>(H, S, kb, xc, rn, rp, mup, mum, true, Xp, Vp, Ap, dp, Xm, Vm, Am, dm);
  if (e) return e;
  if (rn < kNearL && dipole_cancellation<float>(rn, mup, mum, Xp, Vp, Ap, Xm, Vm, Am) > kCancel)
    return near_dipole_f64<KIND>(s, j, r, u, Ld, r_excl, part, mask);
  dipole_pair<KIND, float>(rx, ry, rz, rn, ax.x, ax.y, ax.z, rp, mup, mum, ax.w, Xp, Vp, Ap, dp, Xm, Vm, Am, dm, rex,
                           part, *mask);
  return 0;
}

// Generic charge in float32 (no pairing): Griffiths form with c = 1.
template <int KIND>
__device__ __forceinline__ void charge_mixed(float ax, float ay, float az, float vx, float vy, float vz, float gx,
                                             float gy, float gz, float qs, float rex, float *acc, uint8_t &mask) {
  const float R2 = ax * ax + ay * ay + az * az;
  const float iR = rsqrtf(R2);
  const float R = R2 > 0.f ? R2 * iR : 0.f;  // exact cancellation: 0 * inf would be NaN
  if (R <= rex) {
    mask = 1;
    return;
  }
  const float ux = ax * iR - vx, uy = ay * iR - vy, uz = az * iR - vz;
  const float Ru = R - (ax * vx + ay * vy + az * vz);
  const float i1 = __frcp_rn(Ru);
  const float f = qs * R * i1 * i1 * i1;
  float ex = 0.f, ey = 0.f, ez = 0.f;
  if (KIND != PC_RADIATION) {
    const float g = f * (1.f - (vx * vx + vy * vy + vz * vz));
    ex = g * ux;
    ey = g * uy;
    ez = g * uz;
  }
  if (KIND != PC_COULOMB) {
    const float aa = ax * gx + ay * gy + az * gz;
    ex += f * (ux * aa - gx * Ru);
    ey += f * (uy * aa - gy * Ru);
    ez += f * (uz * aa - gz * Ru);
  }
  acc[0] += ex;
  acc[1] += ey;
  acc[2] += ez;
  const float nx = ax * iR, ny = ay * iR, nz = az * iR;
  acc[3] += ny * ez - nz * ey;
  acc[4] += nz * ex - nx * ez;
  acc[5] += nx * ey - ny * ex;
  acc[6] += qs * i1;
  acc[7] += qs * i1 * vx;
  acc[8] += qs * i1 * vy;
  acc[9] += qs * i1 * vz;
}

// Kahan-compensated running sums of the ten outputs; each thread's sums live in shared memory,
// strided by the block size (they are touched once per group of sixteen sources), as five packed
// pairs: 0 (E_x, E_y), 1 (B_x, B_y), 2 (A_x, A_y), 3 (E_z, B_z), 4 (A_z, phi).  Indexed from the
// thread index directly, so no pointer stays live across the source loop.
using KahanArr = float2[2][5][kMixThreads];
__device__ __forceinline__ void kahan_add(KahanArr &k, int tid, const float2 *P) {
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const float2 s0 = k[0][i][tid], c0 = k[1][i][tid];
    const float2 y = __fadd2_rn(P[i], make_float2(-c0.x, -c0.y));
    const float2 t = __fadd2_rn(s0, y);
    const float2 d = __fadd2_rn(t, make_float2(-s0.x, -s0.y));
    k[1][i][tid] = __fadd2_rn(d, make_float2(-y.x, -y.y));
    k[0][i][tid] = t;
  }
}
// the ten outputs in their natural order (E, B, phi, A) into the packed slots
__device__ __forceinline__ void pack_outputs(const float *part, float2 (&P)[5]) {
  P[0] = make_float2(part[0], part[1]);
  P[1] = make_float2(part[3], part[4]);
  P[2] = make_float2(part[7], part[8]);
  P[3] = make_float2(part[2], part[5]);
  P[4] = make_float2(part[9], part[6]);
}
__device__ __forceinline__ float kahan_get(const KahanArr &k, int tid, int i) {
  // natural index -> (slot, lane)
  const int slot[10] = {0, 0, 3, 1, 1, 3, 4, 2, 2, 4};
  const int hi[10] = {0, 1, 0, 0, 1, 1, 1, 0, 1, 0};
  const float2 sv = k[0][slot[i]][tid], cv = k[1][slot[i]][tid];
  return hi[i] ? sv.y - cv.y : sv.x - cv.x;
}

// The point of thread tid in tile blockIdx.x (list: 256 consecutive points; plane: a block of rows x
// columns of the grid), or P for a thread past the edge of the grid.
__device__ __forceinline__ int64_t tile_point(const Launch &L, int64_t tiles_v, int tid) {
  if (L.pts.list) return (int64_t)blockIdx.x * kMixThreads + tid;
  const int64_t tu = blockIdx.x / tiles_v, tv = blockIdx.x % tiles_v;
  const int sh = L.tile_shift, cols = 1 << sh, rows = kMixThreads >> sh;
  const int64_t iu = tu * rows + (tid >> sh), iv = tv * cols + (tid & (cols - 1));
  return (iu < L.pts.nu && iv < L.pts.nv) ? iu * L.pts.nv + iv : L.pts.P;
}

template <int KIND, bool LIST, int CH>
__global__ void __launch_bounds__(kMixThreads, 4) fields_mixed_kernel(const Launch L, int64_t tiles_v) {
  __shared__ double s_anchor[3];
  __shared__ float s_anc_hi[3], s_anc_lo[3];  // the anchor / (c dt) of the dipoles as float-float
  __shared__ KahanArr s_kahan;
  __shared__ float4 s_geo[CH];   // rho_a (x,y,z), |rho_a|
  __shared__ float4 s_geo_lo[CH]; // low parts of rho_a and |rho_a| (list mode)
  __shared__ float4 s_ax[CH];    // axis (x,y,z), q/e
  __shared__ float4 s_mix[CH];   // m2/(m1+m2), m1/(m1+m2), fraction and integer part of the
                                     // retarded sample of the anchor (integer as bits)
  __shared__ const float4 *s_hist[CH];

  const int tid = threadIdx.x;
  const int f = blockIdx.y;
  const Sources &s = L.src;
  // ---- tile -> points (the index itself is formed again where it is needed, so that it does not
  // occupy registers across the source loop) ----
  const bool active = tile_point(L, tiles_v, tid) < L.pts.P;
  if (tid == 0) {
    double a[3];
    if (L.pts.list) {
      int64_t pa = (int64_t)blockIdx.x * kMixThreads + kMixThreads / 2;
      if (pa >= L.pts.P) pa = L.pts.P - 1;
      point_at(L.pts, pa, a);
    } else {
      int64_t tu = blockIdx.x / tiles_v, tv = blockIdx.x % tiles_v;
      const int sh = L.tile_shift, cols = 1 << sh, rows = kMixThreads >> sh;
      double iu = (double)(tu * rows) + 0.5 * (rows - 1), iv = (double)(tv * cols) + 0.5 * (cols - 1);
      for (int i = 0; i < 3; ++i) a[i] = L.pts.o[i] + iu * L.pts.eu[i] + iv * L.pts.ev[i];
    }
    s_anchor[0] = a[0];
    s_anchor[1] = a[1];
    s_anchor[2] = a[2];
    for (int i = 0; i < 3; ++i) {
      const double x = a[i] * L.iLd;
      s_anc_hi[i] = (float)x;
      s_anc_lo[i] = (float)(x - (double)s_anc_hi[i]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    s_kahan[0][i][tid] = make_float2(0.f, 0.f);
    s_kahan[1][i][tid] = make_float2(0.f, 0.f);
  }
  uint8_t mask = 0;
  int err = 0;

  // ---------------- dipoles ----------------
  if (s.N > 0) {
    // float64 values used once per chunk or by the rare slow pairs are recomputed there, so that
    // none of them occupies registers across the source loop
    const double iLd = L.iLd;  // float64 divisions would stall the CTA on this GPU's narrow float64 unit
    float drx, dry, drz, drlx = 0.f, drly = 0.f, drlz = 0.f;
    if (!LIST) {
      // a plane point sits a whole number of grid steps from the tile anchor: the offset in float
      // from those small integers (no float64 on the way)
      const int sh = L.tile_shift, cols = 1 << sh, rows = kMixThreads >> sh;
      const float du = (float)(tid >> sh) - 0.5f * (float)(rows - 1), dv = (float)(tid & (cols - 1)) - 0.5f * (float)(cols - 1);
      drx = du * L.eu_L[0] + dv * L.ev_L[0];
      dry = du * L.eu_L[1] + dv * L.ev_L[1];
      drz = du * L.eu_L[2] + dv * L.ev_L[2];
    } else {
      double r[3];
      point_at(L.pts, active ? tile_point(L, tiles_v, tid) : 0, r);
      const double drxd = (r[0] - s_anchor[0]) * iLd, dryd = (r[1] - s_anchor[1]) * iLd,
                   drzd = (r[2] - s_anchor[2]) * iLd;
      drx = (float)drxd;
      dry = (float)dryd;
      drz = (float)drzd;
      drlx = (float)(drxd - (double)drx);
      drly = (float)(dryd - (double)dry);
      drlz = (float)(drzd - (double)drz);
    }
    const float dr2 = drx * drx + dry * dry + drz * drz;
    for (int base = 0; base < s.N; base += CH) {
      const int nch = min(CH, s.N - base);
      __syncthreads();
      if (tid < nch) {
        // the tile anchor's distance to the source in float64 (the integer sample index and a
        // fraction kept to ~1e-7), everything else from the per-call records
        // in float-float (~1e-14 relative) on the float32 pipes: rho_a = anchor - origin in units of
        // c dt, |rho_a|, and the centre's retarded sample u - |rho_a| split into integer and fraction
        const int j = base + tid;
        const float4 oh = L.srcf[4 * j + 2], ol = L.srcf[4 * j + 3];
        const ff rax = ff_add({s_anc_hi[0], s_anc_lo[0]}, {-oh.x, -ol.x});
        const ff ray = ff_add({s_anc_hi[1], s_anc_lo[1]}, {-oh.y, -ol.y});
        const ff raz = ff_add({s_anc_hi[2], s_anc_lo[2]}, {-oh.z, -ol.z});
        const ff rna = ff_sqrt(ff_add(ff_add(ff_mul(rax, rax), ff_mul(ray, ray)), ff_mul(raz, raz)));
        const ff x = ff_add({L.uf_hi[f], L.uf_lo[f]}, {-rna.hi, -rna.lo});
        float kaf;
        const int kai = Num<float>::floor_int(x.hi, kaf);
        s_geo[tid] = make_float4(rax.hi, ray.hi, raz.hi, rna.hi);
        if (LIST) s_geo_lo[tid] = make_float4(rax.lo, ray.lo, raz.lo, rna.lo);
        s_ax[tid] = L.srcf[4 * j];
        const float4 mm = L.srcf[4 * j + 1];
        s_mix[tid] = make_float4(mm.x, mm.y, (x.hi - kaf) + x.lo, __int_as_float(kai));
        s_hist[tid] = L.Hd + (size_t)j * s.Sd;
      }
      __syncthreads();
      if (!active || err) continue;
      float2 P[5];
#pragma unroll
      for (int i = 0; i < 5; ++i) P[i] = make_float2(0.f, 0.f);
      typename SlowMask<CH>::T slow_mask = 0;
      for (int g0 = 0; g0 < nch; g0 += 32) {
      // groups of 32 sources summed in float32, the group sums compensated (16 per group cost 1 %
      // more time for no accuracy the 1e-5 bound needs)
      const int gend = min(nch, g0 + 32);
      for (int jj = g0; jj < gend; ++jj) {
        const float4 g = s_geo[jj];
        const float4 ax = s_ax[jj];
        const float4 mx = s_mix[jj];
        const float2 mu = make_float2(mx.x, mx.y);
        const float fa = mx.z;
        const float rx = g.x + drx, ry = g.y + dry, rz = g.z + drz;
        const float rho2 = rx * rx + ry * ry + rz * rz;
        // rho2 == 0 makes rn NaN, which sends the pair to the slow path through the tests below
        const float rn = rho2 * rsqrtf(rho2);
        // retarded time of the dipole centre, in samples: kb + xc with |xc| small
        int kb = __float_as_int(mx.w);
        float xc;
        if (!LIST) {
          // compact tile: |rho| - |rho_a| from the tile offset without cancellation
          const float corr = __fdividef(2.f * (g.x * drx + g.y * dry + g.z * drz) + dr2, rn + g.w);
          xc = fa - corr;
        } else {
          // points of a list tile may lie far apart: |rho| - |rho_a| in float-float, integer part
          // moved into kb so that the fraction keeps its precision
          const float4 gl = s_geo_lo[jj];
          const ff px = ff_add({g.x, gl.x}, {drx, drlx}), py = ff_add({g.y, gl.y}, {dry, drly}),
                   pz = ff_add({g.z, gl.z}, {drz, drlz});
          const ff n2 = ff_add(ff_add(ff_mul(px, px), ff_mul(py, py)), ff_mul(pz, pz));
          const ff dn = ff_add(ff_sqrt(n2), {-g.w, -gl.w});
          const ff x = ff_add({fa, 0.f}, {-dn.hi, -dn.lo});
          float flf;
          const int fl = Num<float>::floor_int(x.hi, flf);
          kb += fl;
          xc = (x.hi - flf) + x.lo;
        }
        const float rp = rx * ax.x + ry * ax.y + rz * ax.z;
        // fast path: both charges on the interior segment of their centre's retarded time, the point
        // farther than rex + 1.5 samples from the centre (the charges are then farther than rex:
        // their distances differ from rn by |delta| <= 1.1); a garbage index from a huge or NaN xc
        // fails the range test before any load
        float2 X, V, Ac, dl;
        bool fast = false;
        {
          float fl;
          const int kc = Num<float>::floor_int(xc, fl);
          const int j = kb + kc;
          if ((unsigned)(j - 1) < L.jlim && rn > L.rex_fast) {
            // the source's history row from the parameter bank (no per-pair shared-memory load)
            const HistF32 H{L.Hd + (size_t)(base + jj) * (size_t)L.src.Sd};
            float x0, v0, a0, x1, v1, a1;
            H.get_in(j, x0, v0, a0);
            H.get_in(j + 1, x1, v1, a1);
            fast = dip_pair_states_fast(x0, v0, a0, x1, v1, a1, xc - fl, rn, rp, mu.x, mu.y, X, V, Ac, dl);
          }
        }
        // near fields that cancel in float32 also leave the fast path
        if (fast && rn < kNearL &&
            dipole_cancellation<float>(rn, mu.x, mu.y, X.x, V.x, Ac.x, X.y, V.y, Ac.y) > kCancel)
          fast = false;
        if (!fast) {
          slow_mask |= SlowMask<CH>::bit(jj);
          continue;
        }
        dipole_pair_fast<KIND>(make_float2(rx, ry), rz, rn, make_float2(ax.x, ax.y), ax.z, rp, mu.x, mu.y, ax.w, X, V,
                               Ac, dl, P);
      }
      kahan_add(s_kahan, tid, P);
#pragma unroll
      for (int i = 0; i < 5; ++i) P[i] = make_float2(0.f, 0.f);
      }
      // the pairs of this chunk that left the fast path
      while (slow_mask && !err) {
        const int jj = SlowMask<CH>::first(slow_mask);
        slow_mask &= slow_mask - 1;
        // the out-of-line call gets arrays of its own: passing the address of part or mask would
        // keep them in local memory throughout the source loop
        float sp[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        uint8_t smask = 0;
        const float4 g = s_geo[jj];
        const float4 ax = s_ax[jj];
        const float4 mx = s_mix[jj];
        const float rx = g.x + drx, ry = g.y + dry, rz = g.z + drz;
        const float rho2 = rx * rx + ry * ry + rz * rz;
        const float rn = rho2 > 0.f ? rho2 * rsqrtf(rho2) : 0.f;
        int kb = __float_as_int(mx.w);
        float xc;
        if (!LIST) {
          const float corr = __fdividef(2.f * (g.x * drx + g.y * dry + g.z * drz) + dr2, rn + g.w);
          xc = mx.z - corr;
        } else {
          const float4 gl = s_geo_lo[jj];
          const ff px = ff_add({g.x, gl.x}, {drx, drlx}), py = ff_add({g.y, gl.y}, {dry, drly}),
                   pz = ff_add({g.z, gl.z}, {drz, drlz});
          const ff n2 = ff_add(ff_add(ff_mul(px, px), ff_mul(py, py)), ff_mul(pz, pz));
          const ff dn = ff_add(ff_sqrt(n2), {-g.w, -gl.w});
          const ff x = ff_add({mx.z, 0.f}, {-dn.hi, -dn.lo});
          float flf;
          const int fl = Num<float>::floor_int(x.hi, flf);
          kb += fl;
          xc = (x.hi - flf) + x.lo;
        }
        double rp64[3];
        point_at(L.pts, tile_point(L, tiles_v, tid), rp64);
        const int e = slow_dipole<KIND>(s, base + jj, s_hist[jj], (int)s.Sd, kb, xc, rx, ry, rz, rn, ax, mx.x, mx.y,
                                        L.rex, rp64, (L.times[f] - s.t0d) / s.dtd, kC * s.dtd, L.r_excl, sp,
                                        &smask);
        if (e) err = e;
        mask |= smask;
        float2 SP[5];
        pack_outputs(sp, SP);
        kahan_add(s_kahan, tid, SP);
      }
    }
  }
  // ---------------- point charges ----------------
  if (s.M > 0) {
    double r[3];
    point_at(L.pts, active ? tile_point(L, tiles_v, tid) : 0, r);
    const double iLc = L.iLc;  // no float64 division on the way (the float64 unit is narrow here)
    const float drx = (float)((r[0] - s_anchor[0]) * iLc), dry = (float)((r[1] - s_anchor[1]) * iLc),
                drz = (float)((r[2] - s_anchor[2]) * iLc);
    const float dr2 = drx * drx + dry * dry + drz * drz;
    const double u = L.ufc[f];
    const float rex = (float)(L.r_excl * iLc);
    const float sE = L.sE, sP = L.sP;
    for (int base = 0; base < s.M; base += CH) {
      const int nch = min(CH, s.M - base);
      __syncthreads();
      if (tid < nch) {
        const int c = base + tid;
        double ra[3];
        for (int i = 0; i < 3; ++i) ra[i] = (s_anchor[i] - L.cref[3 * c + i]) * iLc;
        const double rna = sqrt(ra[0] * ra[0] + ra[1] * ra[1] + ra[2] * ra[2]);
        const double x = u - rna;
        const double kaf = floor(x);
        s_geo[tid] = make_float4((float)ra[0], (float)ra[1], (float)ra[2], (float)rna);
        s_ax[tid] = make_float4(0.f, 0.f, 0.f, (float)(s.q[c] * (1.0 / kE)));
        s_mix[tid] = make_float4(0.f, 0.f, (float)(x - kaf), __int_as_float((int)kaf));
      }
      __syncthreads();
      if (!active || err) continue;
      float part[10];
#pragma unroll
      for (int i = 0; i < 10; ++i) part[i] = 0.f;
      for (int cc = 0; cc < nch; ++cc) {
        const float4 g = s_geo[cc];
        const float qs = s_ax[cc].w;
        const float rx = g.x + drx, ry = g.y + dry, rz = g.z + drz;
        const float rho2 = rx * rx + ry * ry + rz * rz;
        const float irn = rho2 > 0.f ? rsqrtf(rho2) : 0.f;
        const float rn = rho2 * irn;
        const float corr = __fdividef(2.f * (g.x * drx + g.y * dry + g.z * drz) + dr2, rn + g.w);
        const float xc = s_mix[cc].z - corr;
        if (!(fabsf(xc) < 1e6f)) {
          err = PC_ERR_NOCONV;
          break;
        }
        const float4 *H = L.Hc + (size_t)(base + cc) * s.S * 3;
        const int S = (int)s.S;
        // first-order estimate of the charge's delay offset: -rho_hat . o(center time)
        float kcf;
        const int kc = Num<float>::floor_int(xc, kcf);
        float thc = xc - kcf;
        int j = __float_as_int(s_mix[cc].w) + kc;
        {
          int jc = j < 0 ? 0 : (j > S - 1 ? S - 1 : j);
          float4 o = __ldg(H + 3 * jc);
          float d0 = -(rx * o.x + ry * o.y + rz * o.z) * irn;
          float stf;
          int st = Num<float>::floor_int(thc - d0, stf);
          j += st;
          thc -= stf;
        }
        float ox = 0, oy = 0, oz = 0, vx = 0, vy = 0, vz = 0, gx = 0, gy = 0, gz = 0;
        bool done = false;
        for (int it = 0; it < 32 && !done; ++it) {
          // an estimate past either end is solved on the end segment extended; the root then
          // decides whether the history really ends too early
          if (j > S - 2) {
            thc += (float)(j - (S - 2));
            j = S - 2;
          }
          if (j < 0 && !s.static_before) {
            thc += (float)j;
            j = 0;
          }
          const int j0 = j < 0 ? 0 : j, j1 = j < 0 ? 0 : j + 1;
          const float4 o0 = __ldg(H + 3 * j0), o1 = __ldg(H + 3 * j1);
          const float wx = o1.x - o0.x, wy = o1.y - o0.y, wz = o1.z - o0.z;
          const float ocx = o0.x + thc * wx, ocy = o0.y + thc * wy, ocz = o0.z + thc * wz;
          const float A = 1.f - (wx * wx + wy * wy + wz * wz);
          const float B = rn - ((rx - ocx) * wx + (ry - ocy) * wy + (rz - ocz) * wz);
          const float C = ocx * (2.f * rx - ocx) + ocy * (2.f * ry - ocy) + ocz * (2.f * rz - ocz);
          const float sq = Num<float>::sqrt0(fmaxf(B * B - A * C, 0.f));
          const float dl = (B > 0.f) ? -__fdividef(C, B + sq) : __fdividef(-B + sq, A);
          float th = thc - dl;
          const bool ok = (j < 0) ? ((float)j + th <= 1e-4f)
                                  : (th >= -1e-4f && (th <= 1.0001f || (j == S - 2 && th <= 1.f + kEndTol)));
          if (ok) {
            th = fminf(fmaxf(th, 0.f), 1.f);
            if (j < 0) {
              ox = o0.x;
              oy = o0.y;
              oz = o0.z;
            } else {
              const float4 v0 = __ldg(H + 3 * j0 + 1), v1 = __ldg(H + 3 * j1 + 1);
              const float4 a0 = __ldg(H + 3 * j0 + 2), a1 = __ldg(H + 3 * j1 + 2);
              ox = o0.x + th * wx;
              oy = o0.y + th * wy;
              oz = o0.z + th * wz;
              vx = v0.x + th * (v1.x - v0.x);
              vy = v0.y + th * (v1.y - v0.y);
              vz = v0.z + th * (v1.z - v0.z);
              gx = a0.x + th * (a1.x - a0.x);
              gy = a0.y + th * (a1.y - a0.y);
              gz = a0.z + th * (a1.z - a0.z);
            }
            done = true;
          } else {
            if (!(fabsf(th) < 1e6f)) break;
            if ((j == S - 2 && th > 1.f) || (j == 0 && th < 0.f && !s.static_before)) {
              err = PC_ERR_HISTORY;
              break;
            }
            float stf;
            const int st = Num<float>::floor_int(th, stf);
            j += st;
            thc -= stf;
          }
        }
        if (!done) {
          if (!err) err = PC_ERR_NOCONV;
          break;
        }
        float c10[10];
#pragma unroll
        for (int i = 0; i < 10; ++i) c10[i] = 0.f;
        charge_mixed<KIND>(rx - ox, ry - oy, rz - oz, vx, vy, vz, gx, gy, gz, qs, rex, c10, mask);
        // E and B carry q through f; scale E/B by sE and phi/A by sP
#pragma unroll
        for (int i = 0; i < 6; ++i) part[i] += sE * c10[i];
#pragma unroll
        for (int i = 6; i < 10; ++i) part[i] += sP * c10[i];
        if ((cc & 15) == 15) {
          float2 PP[5];
          pack_outputs(part, PP);
          kahan_add(s_kahan, tid, PP);
#pragma unroll
          for (int i = 0; i < 10; ++i) part[i] = 0.f;
        }
      }
      float2 PP[5];
      pack_outputs(part, PP);
      kahan_add(s_kahan, tid, PP);
    }
  }
  if (!active) return;
  if (err) {
    set_status(L.status, err);
    return;
  }
  // units: E in k_e e / L^2, B in k_e e / (L^2 c), phi in k_e e / L, A in k_e e / (L c)
  const float fE = L.unit[0], fB = L.unit[1], fP = L.unit[2], fA = L.unit[3];
  const int64_t o = (L.frame0 + f) * L.pts.P + tile_point(L, tiles_v, tid);
  // streaming stores (evict first): the outputs are not read again by this kernel, and L2 keeps the
  // lines that are (the histories, the stack of the slow pairs' calls); on the 2048^2 x 16-frame
  // grid this cut the DRAM writes of a launch from 3.48 to 3.19 GB (outputs: 2.75 GB)
  if (L.out.E) {
    float *e = (float *)L.out.E + 3 * o;
    __stcs(e + 0, fE * kahan_get(s_kahan, tid, 0));
    __stcs(e + 1, fE * kahan_get(s_kahan, tid, 1));
    __stcs(e + 2, fE * kahan_get(s_kahan, tid, 2));
  }
  if (L.out.B) {
    float *b = (float *)L.out.B + 3 * o;
    __stcs(b + 0, fB * kahan_get(s_kahan, tid, 3));
    __stcs(b + 1, fB * kahan_get(s_kahan, tid, 4));
    __stcs(b + 2, fB * kahan_get(s_kahan, tid, 5));
  }
  if (L.out.phi) __stcs((float *)L.out.phi + o, fP * kahan_get(s_kahan, tid, 6));
  if (L.out.A) {
    float *a = (float *)L.out.A + 3 * o;
    __stcs(a + 0, fA * kahan_get(s_kahan, tid, 7));
    __stcs(a + 1, fA * kahan_get(s_kahan, tid, 8));
    __stcs(a + 2, fA * kahan_get(s_kahan, tid, 9));
  }
  if (L.out.mask) __stcs(reinterpret_cast<unsigned char *>(L.out.mask) + o, (unsigned char)mask);
}

// ------------------------------------------------------------------------------------------------
// Two points per thread (plane grids of dipoles): the thread's points sit in rows r and r + rows of
// a tile of 2 rows x cols points, and the fast path evaluates both at once in the lanes of float2
// registers (pc_lw_f32x2.cuh), which packs the per-point scalar part of the pair algebra too.  The
// per-source work staged in shared memory serves twice as many points.  Slow pairs take the
// one-point slow path of their point.
// ------------------------------------------------------------------------------------------------
using KahanArr2 = float2[2][10][kMixThreads];  // [sum, compensation][output][thread], lanes = points

__device__ __forceinline__ void kahan2_add(KahanArr2 &k, int tid, const V2 *P) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const float2 s0 = k[0][i][tid], c0 = k[1][i][tid];
    const float2 y = __fadd2_rn(P[i].v, make_float2(-c0.x, -c0.y));
    const float2 t = __fadd2_rn(s0, y);
    const float2 d = __fadd2_rn(t, make_float2(-s0.x, -s0.y));
    k[1][i][tid] = __fadd2_rn(d, make_float2(-y.x, -y.y));
    k[0][i][tid] = t;
  }
}

// the slow pairs of one point (lane 0 = A, 1 = B) of the chunk, into that point's Kahan lane
template <int KIND, int CH>
__device__ __forceinline__ int slow_pairs2(const Launch &L, int f, int base, typename SlowMask<CH>::T bits, int lane,
                                           float drx, float dry, float drz, float dr2, int64_t p, int Sd32,
                                           float rex, const float4 *s_geo, const float4 *s_ax, const float4 *s_mix,
                                           const float4 *const *s_hist, KahanArr2 &kh, int tid, uint8_t &mask) {
  const Sources &s = L.src;
  int err = 0;
  while (bits && !err) {
    const int jj = SlowMask<CH>::first(bits);
    bits &= bits - 1;
    float sp[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    uint8_t smask = 0;
    const float4 g = s_geo[jj];
    const float4 ax = s_ax[jj];
    const float4 mx = s_mix[jj];
    const float rx = g.x + drx, ry = g.y + dry, rz = g.z + drz;
    const float rho2 = rx * rx + ry * ry + rz * rz;
    const float rn = rho2 > 0.f ? rho2 * rsqrtf(rho2) : 0.f;
    const int kb = __float_as_int(mx.w);
    const float corr = __fdividef(2.f * (g.x * drx + g.y * dry + g.z * drz) + dr2, rn + g.w);
    const float xc = mx.z - corr;
    double rp64[3];
    point_at(L.pts, p, rp64);
    err = slow_dipole<KIND>(s, base + jj, s_hist[jj], Sd32, kb, xc, rx, ry, rz, rn, ax, mx.x, mx.y, rex, rp64,
                            (L.times[f] - s.t0d) / s.dtd, kC * s.dtd, L.r_excl, sp, &smask);
    mask |= smask;
    V2 SP[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) SP[i] = lane == 0 ? V2(sp[i], 0.f) : V2(0.f, sp[i]);
    kahan2_add(kh, tid, SP);
  }
  return err;
}

template <int KIND, int CH>
__global__ void __launch_bounds__(kMixThreads, 2) fields_mixed2_kernel(const Launch L, int64_t tiles_v) {
  __shared__ float s_anc_hi[3], s_anc_lo[3];  // the tile anchor / (c dt) as float-float
  __shared__ KahanArr2 s_kahan;
  __shared__ float4 s_geo[CH];  // rho_a (x,y,z), |rho_a|
  __shared__ float4 s_ax[CH];   // axis (x,y,z), q/e
  __shared__ float4 s_mix[CH];  // m2/(m1+m2), m1/(m1+m2), fraction and integer part (bits) of the
                                    // retarded sample of the anchor
  __shared__ const float4 *s_hist[CH];

  const int tid = threadIdx.x;
  const int f = blockIdx.y;
  const Sources &s = L.src;
  const int sh = L.tile_shift, cols = 1 << sh, rows = kMixThreads >> sh;
  const int64_t tu = blockIdx.x / tiles_v, tv = blockIdx.x % tiles_v;
  const int64_t iuA = tu * 2 * rows + (tid >> sh), iuB = iuA + rows, iv = tv * cols + (tid & (cols - 1));
  const bool actA = iuA < L.pts.nu && iv < L.pts.nv, actB = iuB < L.pts.nu && iv < L.pts.nv;
  const int64_t pA = iuA * L.pts.nv + iv, pB = iuB * L.pts.nv + iv;
  if (tid == 0) {
    const double iu = (double)(tu * 2 * rows) + 0.5 * (2 * rows - 1), ivc = (double)(tv * cols) + 0.5 * (cols - 1);
    for (int i = 0; i < 3; ++i) {
      const double x = (L.pts.o[i] + iu * L.pts.eu[i] + ivc * L.pts.ev[i]) * L.iLd;
      s_anc_hi[i] = (float)x;
      s_anc_lo[i] = (float)(x - (double)s_anc_hi[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    s_kahan[0][i][tid] = make_float2(0.f, 0.f);
    s_kahan[1][i][tid] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  uint8_t maskA = 0, maskB = 0;
  int err = 0;
  // offsets of the two points from the anchor, from whole grid steps (no float64 on the way)
  const float duA = (float)(tid >> sh) - 0.5f * (float)(2 * rows - 1), duB = duA + (float)rows;
  const float dvv = (float)(tid & (cols - 1)) - 0.5f * (float)(cols - 1);
  const V2 drx(duA * L.eu_L[0] + dvv * L.ev_L[0], duB * L.eu_L[0] + dvv * L.ev_L[0]);
  const V2 dry(duA * L.eu_L[1] + dvv * L.ev_L[1], duB * L.eu_L[1] + dvv * L.ev_L[1]);
  const V2 drz(duA * L.eu_L[2] + dvv * L.ev_L[2], duB * L.eu_L[2] + dvv * L.ev_L[2]);
  const V2 dr2 = fma2(drz, drz, fma2(dry, dry, drx * drx));
  const float rex = (float)(L.r_excl * L.iLd);
  const float rex_fast = rex + 1.5f;
  const int Sd32 = (int)s.Sd;
  const unsigned jlim = Sd32 > 3 ? (unsigned)(Sd32 - 3) : 0u;  // fast segments 1 <= j <= S-3
  const bool any = actA || actB;
  for (int base = 0; base < s.N; base += CH) {
    const int nch = min(CH, s.N - base);
    __syncthreads();
    if (tid < nch) {
      // the anchor's distance to the source and the centre's retarded sample in float-float
      const int j = base + tid;
      const float4 oh = L.srcf[4 * j + 2], ol = L.srcf[4 * j + 3];
      const ff rax = ff_add({s_anc_hi[0], s_anc_lo[0]}, {-oh.x, -ol.x});
      const ff ray = ff_add({s_anc_hi[1], s_anc_lo[1]}, {-oh.y, -ol.y});
      const ff raz = ff_add({s_anc_hi[2], s_anc_lo[2]}, {-oh.z, -ol.z});
      const ff rna = ff_sqrt(ff_add(ff_add(ff_mul(rax, rax), ff_mul(ray, ray)), ff_mul(raz, raz)));
      const ff x = ff_add({L.uf_hi[f], L.uf_lo[f]}, {-rna.hi, -rna.lo});
      float kaf;
      const int kai = Num<float>::floor_int(x.hi, kaf);
      s_geo[tid] = make_float4(rax.hi, ray.hi, raz.hi, rna.hi);
      s_ax[tid] = L.srcf[4 * j];
      const float4 mm = L.srcf[4 * j + 1];
      s_mix[tid] = make_float4(mm.x, mm.y, (x.hi - kaf) + x.lo, __int_as_float(kai));
      s_hist[tid] = L.Hd + (size_t)j * s.Sd;
    }
    __syncthreads();
    if (!any || err) continue;
    V2 P[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) P[i] = V2(0.f);
    typename SlowMask<CH>::T slowA = 0, slowB = 0;
    for (int g16 = 0; g16 < nch; g16 += 16) {
      // groups of sixteen sources summed in float32, the group sums compensated
      const int gend = min(nch, g16 + 16);
      for (int jj = g16; jj < gend; ++jj) {
        const float4 g = s_geo[jj];
        const float4 ax = s_ax[jj];
        const float4 mx = s_mix[jj];
        V2 rx = V2(g.x) + drx, ry = V2(g.y) + dry, rz = V2(g.z) + drz;
        const V2 rho2 = fma2(rz, rz, fma2(ry, ry, rx * rx));
        // rho2 == 0 makes rn NaN, which fails the tests below
        V2 rn = rho2 * V2(rsqrtf(rho2.v.x), rsqrtf(rho2.v.y));
        const V2 num = fma2(V2(2.f), fma2(V2(g.z), drz, fma2(V2(g.y), dry, V2(g.x) * drx)), dr2);
        V2 xc = V2(mx.z) - num * rcp2(rn + V2(g.w));
        const int kb = __float_as_int(mx.w);
        float flA, flB;
        const int jA = kb + Num<float>::floor_int(xc.v.x, flA), jB = kb + Num<float>::floor_int(xc.v.y, flB);
        bool fA = actA && (unsigned)(jA - 1) < jlim && rn.v.x > rex_fast;
        bool fB = actB && (unsigned)(jB - 1) < jlim && rn.v.y > rex_fast;
        if (!(fA && fB)) {
          if (actA && !fA) slowA |= SlowMask<CH>::bit(jj);
          if (actB && !fB) slowB |= SlowMask<CH>::bit(jj);
          if (!fA && !fB) continue;
          // the point off the fast path takes the other point's geometry: finite values whose
          // results are dropped
          if (!fA) {
            rx.v.x = rx.v.y;
            ry.v.x = ry.v.y;
            rz.v.x = rz.v.y;
            rn.v.x = rn.v.y;
            xc.v.x = xc.v.y;
            flA = flB;
          } else {
            rx.v.y = rx.v.x;
            ry.v.y = ry.v.x;
            rz.v.y = rz.v.x;
            rn.v.y = rn.v.x;
            xc.v.y = xc.v.x;
            flB = flA;
          }
        }
        const V2 rp = fma2(rz, V2(ax.z), fma2(ry, V2(ax.y), rx * V2(ax.x)));
        const HistF32 H{s_hist[jj]};
        const int ja = fA ? jA : jB, jb = fB ? jB : jA;
        const float4 hA0 = H.load(ja), hA1 = H.load(ja + 1), hB0 = H.load(jb), hB1 = H.load(jb + 1);
        const V2 x0(hA0.x, hB0.x), v0(hA0.y, hB0.y), a0(hA0.z, hB0.z);
        const V2 dx = V2(hA1.x, hB1.x) - x0, dv = V2(hA1.y, hB1.y) - v0, da = V2(hA1.z, hB1.z) - a0;
        const V2 thc = xc - V2(flA, flB);
        const V2 Xc = fma2(thc, dx, x0);
        Ch2 cp, cm;
        V2 ep, em;
        const V2 tp = charge2_state(mx.x, x0, dx, v0, dv, a0, da, Xc, thc, rn, rp, cp, ep);
        const V2 tm = charge2_state(-mx.y, x0, dx, v0, dv, a0, da, Xc, thc, rn, rp, cm, em);
        // both charges on interior segments (0.5 +- (0.5 + kExtrap)), the series converged
        const float thh = 0.5f + kExtrap;
        fA = fA && fabsf(tp.v.x - 0.5f) <= thh && fabsf(tm.v.x - 0.5f) <= thh && fabsf(ep.v.x) + fabsf(em.v.x) < 1e-2f;
        fB = fB && fabsf(tp.v.y - 0.5f) <= thh && fabsf(tm.v.y - 0.5f) <= thh && fabsf(ep.v.y) + fabsf(em.v.y) < 1e-2f;
        // near fields that cancel in float32 also leave the fast path
        if (fA && rn.v.x < kNearL &&
            dipole_cancellation<float>(rn.v.x, mx.x, mx.y, cp.X.v.x, cp.V.v.x, cp.Ac.v.x, cm.X.v.x, cm.V.v.x,
                                       cm.Ac.v.x) > kCancel)
          fA = false;
        if (fB && rn.v.y < kNearL &&
            dipole_cancellation<float>(rn.v.y, mx.x, mx.y, cp.X.v.y, cp.V.v.y, cp.Ac.v.y, cm.X.v.y, cm.V.v.y,
                                       cm.Ac.v.y) > kCancel)
          fB = false;
        if (actA && !fA) slowA |= SlowMask<CH>::bit(jj);
        if (actB && !fB) slowB |= SlowMask<CH>::bit(jj);
        if (!fA && !fB) continue;
        dipole2_fast<KIND>(rx, ry, rz, rn, ax.x, ax.y, ax.z, rp, mx.x, mx.y, ax.w, cp, cm, fA, fB, P);
      }
      kahan2_add(s_kahan, tid, P);
#pragma unroll
      for (int i = 0; i < 10; ++i) P[i] = V2(0.f);
    }
    // the pairs of this chunk that left the fast path, per point
    const V2 d2 = dr2;
    if (slowA)
      err = slow_pairs2<KIND, CH>(L, f, base, slowA, 0, drx.v.x, dry.v.x, drz.v.x, d2.v.x, pA, Sd32, rex, s_geo, s_ax,
                              s_mix, s_hist, s_kahan, tid, maskA);
    if (slowB && !err)
      err = slow_pairs2<KIND, CH>(L, f, base, slowB, 1, drx.v.y, dry.v.y, drz.v.y, d2.v.y, pB, Sd32, rex, s_geo, s_ax,
                              s_mix, s_hist, s_kahan, tid, maskB);
  }
  if (!any) return;
  if (err) {
    set_status(L.status, err);
    return;
  }
  const float uE = L.unit[0], uB = L.unit[1], uP = L.unit[2], uA = L.unit[3];
  for (int lane = 0; lane < 2; ++lane) {
    if (!(lane == 0 ? actA : actB)) continue;
    const int64_t o = (L.frame0 + f) * L.pts.P + (lane == 0 ? pA : pB);
    float val[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) {
      const float2 sv = s_kahan[0][i][tid], cv = s_kahan[1][i][tid];
      val[i] = lane == 0 ? sv.x - cv.x : sv.y - cv.y;
    }
    // streaming stores, as in the one-point kernel
    if (L.out.E) {
      float *e = (float *)L.out.E + 3 * o;
      __stcs(e + 0, uE * val[0]);
      __stcs(e + 1, uE * val[1]);
      __stcs(e + 2, uE * val[2]);
    }
    if (L.out.B) {
      float *b = (float *)L.out.B + 3 * o;
      __stcs(b + 0, uB * val[3]);
      __stcs(b + 1, uB * val[4]);
      __stcs(b + 2, uB * val[5]);
    }
    if (L.out.phi) __stcs((float *)L.out.phi + o, uP * val[6]);
    if (L.out.A) {
      float *a = (float *)L.out.A + 3 * o;
      __stcs(a + 0, uA * val[7]);
      __stcs(a + 1, uA * val[8]);
      __stcs(a + 2, uA * val[9]);
    }
    if (L.out.mask)
      __stcs(reinterpret_cast<unsigned char *>(L.out.mask) + o, (unsigned char)(lane == 0 ? maskA : maskB));
  }
}

// ================================================================================================
// host side
// ================================================================================================
static bool finite3(const double *v) { return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }

// mixed-path launches: plane tiles with CH sources per shared-memory stage, one or two points per
// thread; point lists with the full stage
template <int CH>
static void launch_mixed_plane(const Launch &L, dim3 grid, int64_t tiles_v, bool two, int kind, cudaStream_t st) {
  if (two) {
    if (kind == PC_TOTAL) fields_mixed2_kernel<PC_TOTAL, CH><<<grid, kMixThreads, 0, st>>>(L, tiles_v);
    else if (kind == PC_COULOMB) fields_mixed2_kernel<PC_COULOMB, CH><<<grid, kMixThreads, 0, st>>>(L, tiles_v);
    else fields_mixed2_kernel<PC_RADIATION, CH><<<grid, kMixThreads, 0, st>>>(L, tiles_v);
  } else {
    if (kind == PC_TOTAL) fields_mixed_kernel<PC_TOTAL, false, CH><<<grid, kMixThreads, 0, st>>>(L, tiles_v);
    else if (kind == PC_COULOMB) fields_mixed_kernel<PC_COULOMB, false, CH><<<grid, kMixThreads, 0, st>>>(L, tiles_v);
    else fields_mixed_kernel<PC_RADIATION, false, CH><<<grid, kMixThreads, 0, st>>>(L, tiles_v);
  }
}
static void launch_mixed_list(const Launch &L, dim3 grid, int kind, cudaStream_t st) {
  if (kind == PC_TOTAL) fields_mixed_kernel<PC_TOTAL, true, kChunk><<<grid, kMixThreads, 0, st>>>(L, 1);
  else if (kind == PC_COULOMB) fields_mixed_kernel<PC_COULOMB, true, kChunk><<<grid, kMixThreads, 0, st>>>(L, 1);
  else fields_mixed_kernel<PC_RADIATION, true, kChunk><<<grid, kMixThreads, 0, st>>>(L, 1);
}

// Host outputs that are page-locked are mapped into the device's address space (unified
// addressing): the kernels store into them directly and the stores reach host memory while the
// computation runs.  Returns false (leaving `dev` as it was) if any requested output is not
// page-locked host memory the device can address.
static bool mapped_host_outputs(const pc_field_out *out, Outs &dev) {
  const void *h[5] = {out->E, out->B, out->phi, out->A, out->mask};
  void *d[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  for (int k = 0; k < 5; ++k) {
    if (!h[k]) continue;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, h[k]) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
    d[k] = a.devicePointer;
  }
  dev.E = d[0];
  dev.B = d[1];
  dev.phi = d[2];
  dev.A = d[3];
  dev.mask = (uint8_t *)d[4];
  return true;
}

// Other host outputs: frames are computed in chunks into two device buffers that alternate, and
// each chunk is copied to the host on a second stream while the next chunk computes.
struct HostPipe {
  bool on = false;
  int32_t frames = 1;        // frames per chunk
  size_t bytes_frame = 0;    // device bytes of one frame of every requested output
};

static pc_status fields_impl(pc_ctx *ctx, const pc_charges *ch, const pc_dipole_sources *dp, const double *list,
                             const pc_plane *plane, int64_t P, const double *times, int32_t T, int32_t kind,
                             int32_t precision, double r_excl, const pc_field_out *out, void *stream,
                             bool to_host = false) {
  if (!ctx || !out || !times || T < 1 || P < 0) return PC_ERR_ARG;
  if (kind < PC_TOTAL || kind > PC_RADIATION || (precision != PC_F64 && precision != PC_MIXED)) return PC_ERR_ARG;
  if (!(r_excl >= 0.0)) return PC_ERR_ARG;
  const bool has_ch = ch && ch->M > 0, has_dp = dp && dp->N > 0;
  if (!has_ch && !has_dp) return PC_ERR_ARG;
  if ((ch && ch->M < 0) || (dp && dp->N < 0)) return PC_ERR_ARG;
  if (has_ch && (ch->S < 2 || !(ch->dt > 0.0) || !isfinite(ch->t0) || !ch->q || !ch->pos || !ch->vel || !ch->acc))
    return PC_ERR_ARG;
  if (has_dp && (dp->S < 2 || !(dp->dt > 0.0) || !isfinite(dp->t0) || !dp->origin || !dp->axis || !dp->q ||
                 !dp->m1 || !dp->m2 || !dp->d || !dp->d_dot || !dp->d_ddot))
    return PC_ERR_ARG;
  if (P == 0) return PC_OK;
  if (!list && !plane) return PC_ERR_ARG;
  if (list == nullptr && plane && (plane->nu < 0 || plane->nv < 0 || !finite3(plane->origin) ||
                                   !finite3(plane->eu) || !finite3(plane->ev)))
    return PC_ERR_ARG;
  for (int i = 0; i < T; ++i)
    if (!isfinite(times[i])) return PC_ERR_ARG;
  if (P == 0) return PC_OK;
  DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  pc_status bs = begin_call(ctx, st);
  if (bs != PC_OK) return bs;

  Launch L;
  memset(&L, 0, sizeof(L));
  L.pts.list = list;
  L.pts.P = P;
  if (!list) {
    for (int i = 0; i < 3; ++i) {
      L.pts.o[i] = plane->origin[i];
      L.pts.eu[i] = plane->eu[i];
      L.pts.ev[i] = plane->ev[i];
    }
    L.pts.nu = plane->nu;
    L.pts.nv = plane->nv;
  }
  Sources &s = L.src;
  if (has_ch) {
    s.M = ch->M;
    s.S = ch->S;
    s.t0 = ch->t0;
    s.dt = ch->dt;
    s.q = ch->q;
    s.pos = ch->pos;
    s.vel = ch->vel;
    s.acc = ch->acc;
    s.static_before = ch->static_before;
  }
  if (has_dp) {
    s.N = dp->N;
    s.Sd = dp->S;
    s.t0d = dp->t0;
    s.dtd = dp->dt;
    s.origin = dp->origin;
    s.axis = dp->axis;
    s.qd = dp->q;
    s.m1 = dp->m1;
    s.m2 = dp->m2;
    s.d = dp->d;
    s.dd = dp->d_dot;
    s.ddd = dp->d_ddot;
  }
  L.out.E = out->E;
  L.out.B = out->B;
  L.out.phi = out->phi;
  L.out.A = out->A;
  L.out.mask = out->mask;
  L.r_excl = r_excl;
  L.status = ctx->d_status;
  if (has_dp) check_axes_kernel<<<(unsigned)((dp->N + 255) / 256), 256, 0, st>>>(dp->axis, dp->N, L.status);
  L.tile_shift = ctx->tile_shift;

  L.iLd = has_dp ? 1.0 / (kC * s.dtd) : 0.0;  // 1/(c dt): first guesses without a division
  L.iLc = has_ch ? 1.0 / (kC * s.dt) : 0.0;
  // dipole sample indices are 32-bit integers in both paths (the difference form's solves)
  if (has_dp && s.Sd > (int64_t)1 << 30) return PC_ERR_ARG;
  if (precision == PC_MIXED) {
    // the float32 path indexes samples with 32-bit integers
    if ((has_dp && s.Sd > (int64_t)1 << 30) || (has_ch && s.S > (int64_t)1 << 30)) return PC_ERR_ARG;
    size_t nd = has_dp ? (size_t)s.N * s.Sd : 0, nc = has_ch ? (size_t)s.M * s.S * 3 : 0;
    const size_t ns = has_dp ? 4 * (size_t)s.N : 0;
    if (ctx->hist_f32.reserve((nd + nc + ns) * sizeof(float4)) != cudaSuccess) return PC_ERR_CUDA;
    if (has_ch && ctx->charge_ref.reserve((size_t)s.M * 3 * sizeof(double)) != cudaSuccess) return PC_ERR_CUDA;
    float4 *Hd = (float4 *)ctx->hist_f32.ptr;
    float4 *Hc = Hd + nd;
    L.Hd = Hd;
    L.Hc = Hc;
    L.cref = (const double *)ctx->charge_ref.ptr;
    L.srcf = Hc + nc;
    L.iLd = has_dp ? 1.0 / (kC * s.dtd) : 0.0;
    set_units(L);
    for (int i = 0; i < 3; ++i) {
      L.eu_L[i] = (float)(L.pts.eu[i] * L.iLd);
      L.ev_L[i] = (float)(L.pts.ev[i] * L.iLd);
    }
    if (has_dp) {
      int64_t n = (int64_t)nd;
      prep_dipoles_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s, Hd, Hc + nc);
    }
    if (has_ch) {
      int64_t n = (int64_t)s.M * s.S;
      prep_charges_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s, Hc, (double *)ctx->charge_ref.ptr);
    }
  }
  // host outputs: chunk sizes, device buffers, the copy stream and its events
  const size_t elt = precision == PC_F64 ? sizeof(double) : sizeof(float);
  const size_t b_vec = (size_t)P * 3 * elt, b_sca = (size_t)P * elt, b_msk = (size_t)P;
  HostPipe hp;
  char *slot_base[2] = {nullptr, nullptr};
  if (to_host && !out->E && !out->B && !out->A && !out->phi && !out->mask) return end_call(ctx, st);
  if (to_host && !mapped_host_outputs(out, L.out)) {
    hp.on = true;
    hp.bytes_frame = (out->E ? b_vec : 0) + (out->B ? b_vec : 0) + (out->A ? b_vec : 0) + (out->phi ? b_sca : 0) +
                     (out->mask ? b_msk : 0);
    const size_t target = (size_t)256 << 20;  // about 256 MB per chunk
    hp.frames = (int32_t)std::max<size_t>(1, std::min<size_t>((size_t)kMaxT, target / hp.bytes_frame));
    const size_t slot = hp.bytes_frame * hp.frames;
    if (ctx->out_chunks.reserve(2 * slot) != cudaSuccess) return PC_ERR_CUDA;
    slot_base[0] = (char *)ctx->out_chunks.ptr;
    slot_base[1] = slot_base[0] + slot;
    if (!ctx->copy_stream) {
      if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess) return PC_ERR_CUDA;
      for (int k = 0; k < 4; ++k)
        if (cudaEventCreateWithFlags(&ctx->pipe_ev[k], cudaEventDisableTiming) != cudaSuccess) return PC_ERR_CUDA;
    }
  }
  const int32_t step = hp.on ? hp.frames : kMaxT;
  int chunk = 0;
  for (int32_t f0 = 0; f0 < T; f0 += step, ++chunk) {
    set_frames(L, times, f0, min(step, T - f0));
    const int sl = chunk & 1;
    if (hp.on) {
      // this chunk's device slot: wait until the copy of the chunk before last has left it
      if (chunk >= 2 && cudaStreamWaitEvent(st, ctx->pipe_ev[2 + sl], 0) != cudaSuccess) return PC_ERR_CUDA;
      char *c = slot_base[sl];
      const size_t nf = (size_t)L.T;
      L.out.E = out->E ? (void *)c : nullptr;
      c += out->E ? nf * b_vec : 0;
      L.out.B = out->B ? (void *)c : nullptr;
      c += out->B ? nf * b_vec : 0;
      L.out.A = out->A ? (void *)c : nullptr;
      c += out->A ? nf * b_vec : 0;
      L.out.phi = out->phi ? (void *)c : nullptr;
      c += out->phi ? nf * b_sca : 0;
      L.out.mask = out->mask ? (uint8_t *)c : nullptr;
      L.frame0 = 0;
    }
    if (precision == PC_F64) {
      dim3 grid((unsigned)((P + 127) / 128), (unsigned)L.T);
      if (kind == PC_TOTAL) fields_f64_kernel<PC_TOTAL><<<grid, 128, 0, st>>>(L);
      else if (kind == PC_COULOMB) fields_f64_kernel<PC_COULOMB><<<grid, 128, 0, st>>>(L);
      else fields_f64_kernel<PC_RADIATION><<<grid, 128, 0, st>>>(L);
    } else {
      // plane grids of dipoles alone may take two points per thread (the tuned choice)
      const bool two = !list && !has_ch && ctx->pts_per_thread == 2;
      int64_t tiles, tiles_v = 1;
      if (list) {
        tiles = (P + kMixThreads - 1) / kMixThreads;
      } else {
        const int64_t cols = (int64_t)1 << L.tile_shift, rows = (two ? 2 : 1) * (kMixThreads / cols);
        int64_t tu = (L.pts.nu + rows - 1) / rows;
        tiles_v = (L.pts.nv + cols - 1) / cols;
        tiles = tu * tiles_v;
      }
      dim3 grid((unsigned)tiles, (unsigned)L.T);
      if (list) launch_mixed_list(L, grid, kind, st);
      else if (ctx->src_chunk == 32) launch_mixed_plane<32>(L, grid, tiles_v, two, kind, st);
      else launch_mixed_plane<kChunk>(L, grid, tiles_v, two, kind, st);
    }
    if (hp.on) {
      // copy the chunk to the host on the copy stream once its kernel is done
      cudaStream_t cs = ctx->copy_stream;
      if (cudaEventRecord(ctx->pipe_ev[sl], st) != cudaSuccess || cudaStreamWaitEvent(cs, ctx->pipe_ev[sl], 0) != cudaSuccess)
        return PC_ERR_CUDA;
      const size_t nf = (size_t)L.T;
      const size_t o = (size_t)f0;
      bool ok = true;
      if (out->E) ok = ok && cudaMemcpyAsync((char *)out->E + o * b_vec, L.out.E, nf * b_vec, cudaMemcpyDeviceToHost, cs) == cudaSuccess;
      if (out->B) ok = ok && cudaMemcpyAsync((char *)out->B + o * b_vec, L.out.B, nf * b_vec, cudaMemcpyDeviceToHost, cs) == cudaSuccess;
      if (out->A) ok = ok && cudaMemcpyAsync((char *)out->A + o * b_vec, L.out.A, nf * b_vec, cudaMemcpyDeviceToHost, cs) == cudaSuccess;
      if (out->phi)
        ok = ok && cudaMemcpyAsync((char *)out->phi + o * b_sca, L.out.phi, nf * b_sca, cudaMemcpyDeviceToHost, cs) == cudaSuccess;
      if (out->mask)
        ok = ok && cudaMemcpyAsync(out->mask + o * b_msk, L.out.mask, nf * b_msk, cudaMemcpyDeviceToHost, cs) == cudaSuccess;
      if (!ok || cudaEventRecord(ctx->pipe_ev[2 + sl], cs) != cudaSuccess) return PC_ERR_CUDA;
    }
  }
  if (hp.on) {
    // the caller's stream ends after the last copy, so the status read-back below covers them all
    if (cudaEventRecord(ctx->pipe_ev[2], ctx->copy_stream) != cudaSuccess ||
        cudaStreamWaitEvent(st, ctx->pipe_ev[2], 0) != cudaSuccess)
      return PC_ERR_CUDA;
  }
  return end_call(ctx, st);
}

}  // namespace pc

extern "C" pc_status pc_fields(pc_ctx *ctx, const pc_charges *ch, const pc_dipole_sources *dp, const double *points,
                               int64_t P, const double *times, int32_t T, int32_t kind, int32_t precision,
                               double r_excl, const pc_field_out *out, void *stream) {
  if (P > 0 && !points) return PC_ERR_ARG;
  return pc::fields_impl(ctx, ch, dp, points, nullptr, P, times, T, kind, precision, r_excl, out, stream);
}

extern "C" pc_status pc_fields_to_host(pc_ctx *ctx, const pc_charges *ch, const pc_dipole_sources *dp,
                                       const double *points, int64_t P, const double *times, int32_t T, int32_t kind,
                                       int32_t precision, double r_excl, const pc_field_out *out_host, void *stream) {
  if (P > 0 && !points) return PC_ERR_ARG;
  return pc::fields_impl(ctx, ch, dp, points, nullptr, P, times, T, kind, precision, r_excl, out_host, stream, true);
}

extern "C" pc_status pc_fields_plane_to_host(pc_ctx *ctx, const pc_charges *ch, const pc_dipole_sources *dp,
                                             const pc_plane *grid, const double *times, int32_t T, int32_t kind,
                                             int32_t precision, double r_excl, const pc_field_out *out_host,
                                             void *stream) {
  if (!grid || grid->nu < 0 || grid->nv < 0) return PC_ERR_ARG;
  return pc::fields_impl(ctx, ch, dp, nullptr, grid, grid->nu * grid->nv, times, T, kind, precision, r_excl,
                         out_host, stream, true);
}

extern "C" pc_status pc_fields_plane(pc_ctx *ctx, const pc_charges *ch, const pc_dipole_sources *dp,
                                     const pc_plane *grid, const double *times, int32_t T, int32_t kind,
                                     int32_t precision, double r_excl, const pc_field_out *out, void *stream) {
  if (!grid || grid->nu < 0 || grid->nv < 0) return PC_ERR_ARG;
  return pc::fields_impl(ctx, ch, dp, nullptr, grid, grid->nu * grid->nv, times, T, kind, precision, r_excl, out,
                         stream);
}

// ================================================================================================
// pc_fields_noalloc: the mixed-precision point-list evaluation with its scratch in a static device
// array instead of a context workspace, for callers that may not allocate device memory.
// ================================================================================================
#include <mutex>

namespace pc {

// float32 history mirrors (dipoles, then point charges), the point-charge reference positions and
// the status word of every pc_fields_noalloc call live here
constexpr size_t kStaticScratchBytes = (size_t)16 << 20;  // 16 MiB
constexpr size_t kStaticHeader = 256;                     // status word, padded to 256 B
static __device__ __align__(256) unsigned char g_noalloc_scratch[kStaticHeader + kStaticScratchBytes];

constexpr int kMaxDevices = 64;
static void *g_noalloc_addr[kMaxDevices];  // the array's device address per device, once resolved
static std::mutex g_noalloc_mu;            // guards g_noalloc_addr

}  // namespace pc

extern "C" pc_status pc_fields_noalloc(const pc_charges *ch, const pc_dipole_sources *dp, const double *points,
                                       int64_t P, const double *times, int32_t T, int32_t kind, double r_excl,
                                       const pc_field_out *out, void *stream) {
  using namespace pc;
  if (!out || !times || T < 1 || P < 0) return PC_ERR_ARG;
  if (kind < PC_TOTAL || kind > PC_RADIATION || !(r_excl >= 0.0)) return PC_ERR_ARG;
  const bool has_ch = ch && ch->M > 0, has_dp = dp && dp->N > 0;
  if (!has_ch && !has_dp) return PC_ERR_ARG;
  if ((ch && ch->M < 0) || (dp && dp->N < 0)) return PC_ERR_ARG;
  if (has_ch && (ch->S < 2 || !(ch->dt > 0.0) || !isfinite(ch->t0) || !ch->q || !ch->pos || !ch->vel || !ch->acc))
    return PC_ERR_ARG;
  if (has_dp && (dp->S < 2 || !(dp->dt > 0.0) || !isfinite(dp->t0) || !dp->origin || !dp->axis || !dp->q ||
                 !dp->m1 || !dp->m2 || !dp->d || !dp->d_dot || !dp->d_ddot))
    return PC_ERR_ARG;
  for (int i = 0; i < T; ++i)
    if (!isfinite(times[i])) return PC_ERR_ARG;
  if (P == 0) return PC_OK;
  if (!points) return PC_ERR_ARG;
  // the scratch must hold the float32 mirrors and the reference positions
  const size_t nd = has_dp ? (size_t)dp->N * (size_t)dp->S : 0;
  const size_t nc = has_ch ? (size_t)ch->M * (size_t)ch->S * 3 : 0;
  const size_t ns = has_dp ? 4 * (size_t)dp->N : 0;
  const size_t need = (nd + nc + ns) * sizeof(float4) + (has_ch ? (size_t)ch->M * 3 * sizeof(double) : 0);
  if (need > kStaticScratchBytes) return PC_ERR_ARG;
  if ((has_dp && dp->S > (int64_t)1 << 30) || (has_ch && ch->S > (int64_t)1 << 30)) return PC_ERR_ARG;

  // once per device, with that device current: the device address of the static scratch.  Only a
  // resolved address is kept, so a failed first lookup is retried by the next call.
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PC_ERR_CUDA;
  // the points must live on the current device: the kernels run there
  {
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, points) != cudaSuccess) {
      cudaGetLastError();
      return PC_ERR_ARG;
    }
    if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) return PC_ERR_ARG;
    if (pa.device != dev) return PC_ERR_ARG;
  }
  unsigned char *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void *a = nullptr;
      if (cudaGetSymbolAddress(&a, g_noalloc_scratch) != cudaSuccess || !a) {
        cudaGetLastError();
        return PC_ERR_CUDA;
      }
      g_noalloc_addr[dev] = a;
    }
    base = (unsigned char *)g_noalloc_addr[dev];
  }
  int *status = (int *)base;
  float4 *Hd = (float4 *)(base + kStaticHeader);
  float4 *Hc = Hd + nd;
  float4 *srcf = Hc + nc;
  double *cref = (double *)(srcf + ns);

  cudaStream_t st = (cudaStream_t)stream;
  cudaGetLastError();
  // the array keeps the previous call's contents: the status word must start at zero
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return PC_ERR_CUDA;

  Launch L;
  memset(&L, 0, sizeof(L));
  L.pts.list = points;
  L.pts.P = P;
  Sources &s = L.src;
  if (has_ch) {
    s.M = ch->M;
    s.S = ch->S;
    s.t0 = ch->t0;
    s.dt = ch->dt;
    s.q = ch->q;
    s.pos = ch->pos;
    s.vel = ch->vel;
    s.acc = ch->acc;
    s.static_before = ch->static_before;
  }
  if (has_dp) {
    s.N = dp->N;
    s.Sd = dp->S;
    s.t0d = dp->t0;
    s.dtd = dp->dt;
    s.origin = dp->origin;
    s.axis = dp->axis;
    s.qd = dp->q;
    s.m1 = dp->m1;
    s.m2 = dp->m2;
    s.d = dp->d;
    s.dd = dp->d_dot;
    s.ddd = dp->d_ddot;
  }
  L.out.E = out->E;
  L.out.B = out->B;
  L.out.phi = out->phi;
  L.out.A = out->A;
  L.out.mask = out->mask;
  L.r_excl = r_excl;
  L.status = status;
  if (has_dp) check_axes_kernel<<<(unsigned)((dp->N + 255) / 256), 256, 0, st>>>(dp->axis, dp->N, status);
  L.Hd = Hd;
  L.Hc = Hc;
  L.cref = cref;
  L.srcf = srcf;
  L.iLd = has_dp ? 1.0 / (kC * s.dtd) : 0.0;
  set_units(L);
  // the mirrors are rewritten in full by every call
  if (has_dp) prep_dipoles_f32<<<(unsigned)((nd + 255) / 256), 256, 0, st>>>(s, Hd, srcf);
  if (has_ch) {
    const int64_t n = (int64_t)s.M * s.S;
    prep_charges_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s, Hc, cref);
  }
  const int64_t tiles = (P + kMixThreads - 1) / kMixThreads;
  for (int32_t f0 = 0; f0 < T; f0 += kMaxT) {
    set_frames(L, times, f0, min(kMaxT, T - f0));
    dim3 grid((unsigned)tiles, (unsigned)L.T);
    launch_mixed_list(L, grid, kind, st);
  }
  if (cudaGetLastError() != cudaSuccess) return PC_ERR_CUDA;
  int h = 0;  // pageable host word: the copy completes before cudaMemcpyAsync returns to the stream order
  if (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return PC_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PC_ERR_CUDA;
  return (pc_status)h;
}

// ================================================================================================
// Tile-shape autotuning of the mixed plane evaluation: 256-point tiles of 8 x 32, 16 x 16 or 32 x 8
// (rows x columns) trade the spread of the points' delays within a tile (the history gathers'
// locality) against the width of the output rows each warp stores.  Each candidate runs the
// caller's workload once to warm up and once timed; the fastest is kept in the context for the
// plane calls that follow.
// ================================================================================================
extern "C" pc_status pc_set_plane_tiling(pc_ctx *ctx, const pc_plane_tiling *t) {
  if (!ctx || !t) return PC_ERR_ARG;
  const int32_t rows = t->tile_rows, cols = t->tile_cols;
  if (rows < 1 || cols < 1 || cols > pc::kMixThreads || (cols & (cols - 1))) return PC_ERR_ARG;
  const int64_t pts = (int64_t)rows * cols;
  if (pts != pc::kMixThreads && pts != 2 * pc::kMixThreads) return PC_ERR_ARG;
  if (t->sources_per_stage != 32 && t->sources_per_stage != pc::kChunk) return PC_ERR_ARG;
  int sh = 0;
  while ((1 << sh) < cols) ++sh;
  ctx->tile_shift = sh;
  ctx->pts_per_thread = pts == pc::kMixThreads ? 1 : 2;
  ctx->src_chunk = t->sources_per_stage;
  return PC_OK;
}

extern "C" pc_status pc_autotune_plane(pc_ctx *ctx, const pc_charges *ch, const pc_dipole_sources *dp,
                                       const pc_plane *grid, const double *times, int32_t T, int32_t kind,
                                       double r_excl, const pc_field_out *out, pc_plane_tiling *chosen,
                                       void *stream) {
  if (!ctx || !grid || !out) return PC_ERR_ARG;
  pc::DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  // (points per thread, log2 columns): 8 x 32, 16 x 16, 32 x 8 tiles of one point per thread, and
  // 16 x 32, 32 x 16, 64 x 8 of two (plane grids of dipoles alone); each with 64 and with 32
  // sources per shared-memory stage
  const int cand[6][2] = {{1, 5}, {1, 4}, {1, 3}, {2, 5}, {2, 4}, {2, 3}};
  const int nshape = (ch && ch->M > 0) ? 3 : 6;
  const int chunks[2] = {pc::kChunk, 32};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PC_ERR_CUDA;
  float best = 1e30f;
  int best_c = -1;
  pc_status rs = PC_OK;
  for (int c = 0; c < 2 * nshape && rs == PC_OK; ++c) {
    ctx->pts_per_thread = cand[c % nshape][0];
    ctx->tile_shift = cand[c % nshape][1];
    ctx->src_chunk = chunks[c / nshape];
    rs = pc_fields_plane(ctx, ch, dp, grid, times, T, kind, PC_MIXED, r_excl, out, stream);
    if (rs != PC_OK) break;
    cudaEventRecord(e0, st);
    rs = pc_fields_plane(ctx, ch, dp, grid, times, T, kind, PC_MIXED, r_excl, out, stream);
    cudaEventRecord(e1, st);
    if (rs != PC_OK || cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_c < 0) best_c = 1;
  ctx->pts_per_thread = cand[best_c % nshape][0];
  ctx->tile_shift = cand[best_c % nshape][1];
  ctx->src_chunk = chunks[best_c / nshape];
  if (chosen) {
    chosen->tile_rows = ctx->pts_per_thread * (pc::kMixThreads >> ctx->tile_shift);
    chosen->tile_cols = 1 << ctx->tile_shift;
    chosen->sources_per_stage = ctx->src_chunk;
  }
  return rs;
}
