// Lorentz-oscillator run (Algorithm 1 of arXiv 2107.12437) and the kinetic-energy fit (Eq. KE).
//
// pc_dipoles_run: one persistent CTA per configuration.  Time advances in causal blocks of K steps:
// with R_min the smallest distance between a receiving dipole's origin and another dipole's
// charges, every field needed by the RK4 stages of steps n0 .. n0+K-1 (times n0 + 1/2, n0 + 1, ...,
// n0 + K, in steps) has its retarded time at or before n0 when K c dt <= R_min, so all 2K stage
// fields of all receivers are independent and are computed together (phase A); then each receiver
// advances K RK4 steps (Eq. LO_equation) and appends d, d', d'' to the history (phase B).
// Phase A: one warp per receiver; lane = (stage, source slot); each lane sums its sources for its
// stage (float32 pair difference form, or float64 per charge) and the slots are reduced in shared
// memory.  The caller's history arrays are the trajectory store; the mixed path also keeps a
// float32 mirror of it.
// pc_ke_fit: one CTA per series; Levenberg-Marquardt with block reductions.
#include <stdio.h>

#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <vector>

#include "pc_internal.cuh"
#include "pc_lw_f32.cuh"
#include "pc_lw_f64.cuh"
#include "pc_adjoint.cuh"

namespace pc {

constexpr int kRunWarps = 8;   // receivers advanced concurrently by one CTA
constexpr int kMaxBlock = 16;  // steps per causal block (2K <= 32 stages, one per lane)
constexpr int kSmallN = 64;    // configurations up to this size run as one persistent CTA each
constexpr int kMaxSplit = 64;  // source slices per receiver on the grid path

struct RunArgs {
  int B, N;
  const double *origin, *axis, *q, *m1, *m2, *omega0, *d0;
  double dt;
  int64_t n_begin;    // the call's first step (absolute: 0, or the step of the state it resumes from)
  int64_t n_steps;    // the call's last step (absolute): steps n_begin .. n_steps - 1 are advanced
  double v_max;
  int ed_mode;
  // history store: sample n of dipole bi at bi * hs + (n & wm); wm = -1 when the store holds every
  // sample at its index (the caller's full outputs), W - 1 for a ring of W slots (a power of two at
  // least the deepest retarded reach of a causal block)
  double *d, *dd, *ddd;
  float4 *H32;        // the float32 mirror of the store (mixed path), same slots
  int64_t hs, wm;
  // outputs [B][N][So], So = n_steps - n_begin + 1, sample n at index n - n_begin (null: not wanted;
  // the store's own rows when it is the caller's full outputs)
  double *od, *odd, *oddd, *energy, *Ed;
  int energy_loop;    // energies written per step (no full history to take them from afterwards)
  // kinetic energies m d'^2 / (2 q^2) (and d') for the fit, per step from relative step ke_first,
  // [B][N][So - ke_first] (null: taken from the full history after the run)
  double *ke, *kdd;
  int64_t ke_first, ke_len;  // absolute first step and row length of ke / kdd
  // resume (null: a fresh run at rest with moment d0 for t <= 0): the state at step n_begin, see
  // state layout below; state_out receives the state at step n_steps (or null)
  const double *state_in;
  double *state_out;
  int64_t state_D;    // samples of history a state keeps before its step
  double *Es;         // scratch [B][N][2*kMaxBlock+1] stage fields
  int *status;
  // tables built once per run (mixed path): per-dipole float records, per-pair centre delays
  float *dipf;        // [B][N][kDipF]: origin/L as hi+lo (6), axis (3), m2/(m1+m2), m1/(m1+m2), q/e
  int2 *delay;        // [B][N][N]: |R_i - R_j| / (c dt) = x + y, x integer, y the fraction (float bits)
  // [B][N][N] (mixed path): rho = (R_i - R_j) / (c dt) as (|rho|, rho . p_j, rho . p_i, p_j . p_i)
  float4 *pgeo;
  // [B][3]: closest distance of two origins (over the run for moving ones), largest origin speed
  // and largest distance of two origins, as the bits of non-negative doubles (ordered like the
  // values under integer min / max)
  unsigned long long *rstat;
  int *kblock;        // [B] causal block length per configuration
  int *reach;         // [B] deepest retarded reach of a block behind its start (samples): the state depth
  double *Ehalf;      // [B][N][So - 1] E_d at t_n + dt/2 (kept for the adjoint), or null
  // grid path: sources split into nsplit slices whose partial stage fields Epart
  // [nsplit][B][N][2*kMaxBlock+1] are summed in slice order; blk = {block start, block length}
  double *Epart;
  int nsplit;
  int64_t *blk;
  // moving dipoles (float64 path): origin position, velocity, acceleration at the half steps,
  // [B][N][2 n_steps + 1][3], or null for fixed origins
  const double *org_pos, *org_vel, *org_acc;
  // their float32 mirror for the mixed drive, [B][N][2 n_steps + 1][3] float4 per half-step
  // sample: (P_hi, V_x), (P_lo, V_y), (V_z, A): the position in units of c dt as hi + lo parts,
  // the velocity in units of c, the acceleration in units of c / dt; or null
  float4 *omf;
  // moving origins: each origin's largest distance from its first sample over the run, [B][N]
  double *odisp;
  // per dipole: the RK4 step as an affine map y' = M y + c1 e1 + c2 e2 + c4 e4, as
  // [B][N][kTab]: M^1 .. M^kMaxBlock (row-major 2x2 each), then c1, c2, c4
  double *rk4tab;
  double e_unit;  // k_e e / (c dt)^2: the float32 driving field's unit (V/m)
  float near_L;   // mixed drive: sources whose centre is closer than this (units of c dt) go float64
};

// State of a run at step s (pc_run_opts.state_in / state_out), float64 on the device:
//   [0] kStateMagic, [1] s, [2] D, [3] B N;  [4 .. 4 + B N) E_d(s) of each dipole;
//   then [B][N][D + 1][3]: d, d', d'' of samples s - D .. s (oldest first; samples before 0 are the
//   rest state d0, 0, 0).  D covers every sample a causal block starting at s can reach.
constexpr double kStateMagic = 20547.0625;
__host__ __device__ inline int64_t state_doubles(int64_t nbn, int64_t D) { return 4 + nbn + 3 * nbn * (D + 1); }

// then the dipole's constants, so that no block recomputes them (float64 divisions are costly on
// this GPU): gamma0, omega0^2, q^2/m, the largest charge-speed factor, 1/(q L), 1/(q c), dt/(q c),
// m/(2 q^2), and the charges' signed offsets per unit moment m2/((m1+m2) q), -m1/((m1+m2) q)
constexpr int kTabC = 4 * 16 + 6;
constexpr int kTab = kTabC + 11;

constexpr int kDipF = 12;

__device__ __forceinline__ size_t bidx(const RunArgs &a, int b, int i) { return (size_t)b * a.N + i; }

// double -> float rounded to nearest (ties away from zero) from the bits, on the integer units: the
// conversion instruction issues to this GPU's narrow float64 unit, the bottleneck of the per-step
// path of small configurations.  Magnitudes below the float range flush to zero, above it go to
// infinity (the scaled history values stay far from both).
__device__ __forceinline__ float dbl2flt(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  if (e <= 0) return __int_as_float((int)sign);
  if (e >= 255) return __int_as_float((int)(sign | 0x7f800000u));
  const unsigned m = (unsigned)((b >> 29) & 0x7fffffu), r = (unsigned)((b >> 28) & 1u);
  return __int_as_float((int)((sign | ((unsigned)e << 23) | m) + r));
}

// One RK4 step of d'' + g0 d' + w2 d = qm E (Eq. LO_equation) on y = (d, d') with stage fields
// e1 (t), e2 (t + dt/2, both middle stages) and e4 (t + dt).
__device__ __forceinline__ void rk4_step(double y0, double y1, double e1, double e2, double e4, double g0, double w2,
                                         double qm, double dt, double &n0, double &n1) {
  const double k1a = y1, k1b = -g0 * y1 - w2 * y0 + qm * e1;
  const double y0b = y0 + 0.5 * dt * k1a, y1b = y1 + 0.5 * dt * k1b;
  const double k2a = y1b, k2b = -g0 * y1b - w2 * y0b + qm * e2;
  const double y0c = y0 + 0.5 * dt * k2a, y1c = y1 + 0.5 * dt * k2b;
  const double k3a = y1c, k3b = -g0 * y1c - w2 * y0c + qm * e2;
  const double y0d = y0 + dt * k3a, y1d = y1 + dt * k3b;
  const double k4a = y1d, k4b = -g0 * y1d - w2 * y0d + qm * e4;
  n0 = y0 + dt / 6.0 * (k1a + 2.0 * k2a + 2.0 * k3a + k4a);
  n1 = y1 + dt / 6.0 * (k1b + 2.0 * k2b + 2.0 * k3b + k4b);
}

// The step is linear in (y, e1, e2, e4): its matrix M and stage responses c1, c2, c4 are the step
// applied to unit inputs; the table holds M^1 .. M^16 for the block scan.
__device__ void rk4_table(const RunArgs &a, size_t bi) {
  const double m1 = a.m1[bi], m2 = a.m2[bi], q = a.q[bi], w0 = a.omega0[bi];
  const double m = m1 * m2 / (m1 + m2);
  const double g0 = q * q * w0 * w0 / (6.0 * kPi * kEps0 * kC * kC * kC * m);
  const double qm = q * q / m, w2 = w0 * w0, dt = a.dt;
  double M[4], c[6];
  rk4_step(1.0, 0.0, 0.0, 0.0, 0.0, g0, w2, qm, dt, M[0], M[2]);
  rk4_step(0.0, 1.0, 0.0, 0.0, 0.0, g0, w2, qm, dt, M[1], M[3]);
  rk4_step(0.0, 0.0, 1.0, 0.0, 0.0, g0, w2, qm, dt, c[0], c[1]);
  rk4_step(0.0, 0.0, 0.0, 1.0, 0.0, g0, w2, qm, dt, c[2], c[3]);
  rk4_step(0.0, 0.0, 0.0, 0.0, 1.0, g0, w2, qm, dt, c[4], c[5]);
  double *T = a.rk4tab + bi * kTab;
  double P[4] = {M[0], M[1], M[2], M[3]};
  for (int j = 0; j < 16; ++j) {
    for (int e = 0; e < 4; ++e) T[4 * j + e] = P[e];
    const double Q[4] = {M[0] * P[0] + M[1] * P[2], M[0] * P[1] + M[1] * P[3], M[2] * P[0] + M[3] * P[2],
                         M[2] * P[1] + M[3] * P[3]};
    for (int e = 0; e < 4; ++e) P[e] = Q[e];
  }
  for (int e = 0; e < 6; ++e) T[64 + e] = c[e];
  const double L = kC * dt;
  T[kTabC + 0] = g0;
  T[kTabC + 1] = w2;
  T[kTabC + 2] = qm;
  T[kTabC + 3] = fmax(m1, m2) / (m1 + m2) / q;
  T[kTabC + 4] = 1.0 / (q * L);
  T[kTabC + 5] = 1.0 / (q * kC);
  T[kTabC + 6] = dt / (q * kC);
  T[kTabC + 7] = m / (2.0 * q * q);
  T[kTabC + 8] = m2 / (m1 + m2) / q;
  T[kTabC + 9] = -m1 / (m1 + m2) / q;
  T[kTabC + 10] = a.v_max / T[kTabC + 3];  // the largest |d'| the velocity guard allows
}

// The kb steps of a causal block at once, one lane per step: with every stage field of the block
// known, y_{k+1} = M^(k+1) y_0 + sum_{m <= k} M^(k-m) b_m, b_m = c1 e1_m + c2 e2_m + c4 e4_m, an
// inclusive scan over the lanes (log2 kb shuffle rounds) instead of kb dependent steps.  Called by
// all 32 lanes of a warp; appends d, d', d'' (and the float32 mirror, energy, E_d, the half-step
// fields) to the history exactly as the stepwise form.
// Es: the receiver's stage-field row (global, or shared in the persistent kernel); ys: null (the
// block's starting state read from the history store), or the state (d, d') carried in shared
// memory from the previous block, which the block's last lane updates; Tsh / fsc: null, or the
// receiver's table row and the float32 mirror's three scales held in shared memory (the persistent
// kernel: the chain of a block then waits on no global load of constants).
// HWCVT: the float32 mirror converted by the hardware conversion (round to nearest even) instead
// of dbl2flt: on the persistent path a block's chain waits on these conversions, while the grid
// path keeps the float64 unit for its drive
template <bool MIXED, bool HWCVT = false>
__device__ void rk4_block_warp(const RunArgs &a, int b, int i, int64_t n0, int kb, int *stop, double *Es,
                               double *ys = nullptr, const double *Tsh = nullptr, const float *fsc = nullptr) {
  const int lane = threadIdx.x & 31;
  const int64_t So = a.n_steps - a.n_begin + 1;
  const size_t bi = bidx(a, b, i);
  const double *T = Tsh ? Tsh : a.rk4tab + bi * kTab;
  const double g0 = T[kTabC + 0], w2 = T[kTabC + 1], qm = T[kTabC + 2];
  const size_t row = bi * (size_t)a.hs;
  const double y0 = ys ? ys[0] : a.d[row + (n0 & a.wm)], y1 = ys ? ys[1] : a.dd[row + (n0 & a.wm)];
  double vx = 0.0, vy = 0.0, e2 = 0.0, e4 = 0.0;
  if (lane < kb) {
    const double e1 = Es[2 * lane];
    e2 = Es[2 * lane + 1];
    e4 = Es[2 * lane + 2];
    const double f2 = (a.ed_mode == 1) ? e1 : e2, f4 = (a.ed_mode == 1) ? e1 : e4;
    vx = T[64] * e1 + T[66] * f2 + T[68] * f4;
    vy = T[65] * e1 + T[67] * f2 + T[69] * f4;
  }
  for (int off = 1; off < kb; off <<= 1) {
    const double ox = __shfl_up_sync(0xffffffffu, vx, off), oy = __shfl_up_sync(0xffffffffu, vy, off);
    if (lane >= off) {
      const double *P = T + 4 * (off - 1);  // M^off
      vx = fma(P[1], oy, fma(P[0], ox, vx));  // two dependent float64 steps, not three
      vy = fma(P[3], oy, fma(P[2], ox, vy));
    }
  }
  int bad = 0;
  if (lane < kb) {
    const double *P = T + 4 * lane;  // M^(lane+1)
    const double yn0 = fma(P[0], y0, fma(P[1], y1, vx));
    const double yn1 = fma(P[2], y0, fma(P[3], y1, vy));
    const int64_t n = n0 + lane;
    const double ydd = qm * e4 - g0 * yn1 - w2 * yn0;
    const size_t sl = row + ((n + 1) & a.wm);
    a.d[sl] = yn0;
    a.dd[sl] = yn1;
    a.ddd[sl] = ydd;
    if (MIXED)
      // the float32 mirror scaled in float32 (one rounding more than scaling in float64: below the
      // mirror's own rounding budget), the values converted on the integer units
      a.H32[sl] = HWCVT ? make_float4(__double2float_rn(yn0) * fsc[0], __double2float_rn(yn1) * fsc[1],
                                      __double2float_rn(ydd) * fsc[2], 0.f)
                        : make_float4(dbl2flt(yn0) * (fsc ? fsc[0] : dbl2flt(T[kTabC + 4])),
                                      dbl2flt(yn1) * (fsc ? fsc[1] : dbl2flt(T[kTabC + 5])),
                                      dbl2flt(ydd) * (fsc ? fsc[2] : dbl2flt(T[kTabC + 6])), 0.f);
    const size_t o = bi * So + (size_t)(n + 1 - a.n_begin);
    if (a.od) a.od[o] = yn0;
    if (a.odd) a.odd[o] = yn1;
    if (a.oddd) a.oddd[o] = ydd;
    if (a.Ed) a.Ed[o] = e4;
    if (a.Ehalf) a.Ehalf[bi * (So - 1) + (size_t)(n - a.n_begin)] = e2;
    if (a.energy_loop) a.energy[o] = T[kTabC + 7] * (w2 * yn0 * yn0 + yn1 * yn1);
    if (a.ke && n + 1 >= a.ke_first && n + 1 < a.ke_first + a.ke_len) {
      const size_t kk = bi * (size_t)a.ke_len + (size_t)(n + 1 - a.ke_first);
      a.ke[kk] = T[kTabC + 7] * yn1 * yn1;
      if (a.kdd) a.kdd[kk] = yn1;
    }
    bad = fabs(yn1) > T[kTabC + 10];
    if (ys && lane == kb - 1) {
      ys[0] = yn0;
      ys[1] = yn1;
    }
  }
  if (__any_sync(0xffffffffu, bad)) {
    if (lane == 0) set_status(a.status, PC_ERR_VELOCITY);
    *stop = 1;
  }
  __syncwarp();
  if (lane == 0) Es[0] = Es[2 * kb];
  __syncwarp();
}

// pair_drive_f64 for fixed origins in scalar form.  Every vector of the pair lies in the plane of
// rho = R_i - R_j and the source's unit axis p_j: a charge sits at R_j + s p_j (s = w d), moves
// with v = s' p_j and accelerates with s'' p_j, so the quadratic of the retarded time on a segment
// and the Lienard-Wiechert field projected on p_i need only |rho|^2, rho.p_j, rho.p_i and p_j.p_i.
// The same steps as solve_f64 (the root on the segment of the centre's retarded time, other
// segments searched the same way) and lw_E_f64 (Griffiths' E with u = c n - v), on the same
// samples, with a third fewer float64 instructions: the float64 unit, one per SM on this GPU, sets
// the pace of this path.  Returns false, leaving *out, where the general form must decide (the
// static pre-history, the end of the history, no root).
// The retarded sample of a charge at offset s = w d along its axis, fixed origins, in scalar form
// (rr = |rho|^2, ra = rho.p_j): the root th on segment k of the quadratic of solve_f64, starting from
// segment kg, with s0 = w d_k and ds = w d_(k+1) - s0.  False where the general form must decide
// (before the first sample, past the last, no root).
__device__ __forceinline__ bool scalar_root(const double *dh, int64_t wm, double w, double rr, double ra, double u,
                                            double cdt2, int64_t nv, int64_t kg, int64_t *k_out, double *th_out,
                                            double *s0_out, double *ds_out) {
  int64_t k = kg < 0 ? 0 : kg;
  if (k > nv - 1) k = nv - 1;
  for (int it = 0; it < 96; ++it) {
    const double s0 = w * dh[k & wm];
    const double ds = w * dh[(k + 1) & wm] - s0;
    const double T = u - (double)k;
    const double A = cdt2 - ds * ds;
    const double B = ds * (ra - s0) - cdt2 * T;
    const double C = cdt2 * T * T - (rr - s0 * (2.0 * ra - s0));
    const double sq = sqrt(fmax(B * B - A * C, 0.0));
    double t;
    if (B <= 0.0) {
      const double den = -B + sq;
      t = (den > 0.0) ? C / den : T;
    } else {
      t = (-B - sq) / A;
    }
    if (!(t == t)) return false;
    if (t >= -1e-12 && t <= 1.0 + 1e-12) {
      const double th = fmin(fmax(t, 0.0), 1.0);
      if (k == 0 && th == 0.0) return false;  // exactly at the first sample: the general form
      *k_out = k;
      *th_out = th;
      *s0_out = s0;
      *ds_out = ds;
      return true;
    }
    if (t < 0.0) {
      if (k == 0) return false;  // before the first sample
      const double st = floor(t);
      k += (st < -1e15) ? -k : (int64_t)st;
      if (k < 0) k = 0;
    } else {
      if (k == nv - 1) return false;
      const double st = floor(t);
      k += (st > 1e15) ? nv : (int64_t)st;
      if (k > nv - 1) k = nv - 1;
    }
  }
  return false;
}

__device__ bool pair_drive_f64_scalar(const RunArgs &a, int b, int i, int j, double u, int64_t nv, int64_t kg,
                                      int sg0, int sg1, double *out) {
  const double cdt = kC * a.dt, cdt2 = cdt * cdt;
  const size_t bi = bidx(a, b, i), bj = bidx(a, b, j);
  const double *Ri = a.origin + 3 * bi, *Rj = a.origin + 3 * bj;
  const double *pi = a.axis + 3 * bi, *pj = a.axis + 3 * bj;
  const double rho[3] = {Ri[0] - Rj[0], Ri[1] - Rj[1], Ri[2] - Rj[2]};
  const double rr = dot3(rho, rho), ra = dot3(rho, pj), rp = dot3(rho, pi), ap = dot3(pj, pi);
  const double *Tj = a.rk4tab + bj * kTab;
  const double q = a.q[bj];
  const double *dh = a.d + bj * a.hs, *ddh = a.dd + bj * a.hs, *dddh = a.ddd + bj * a.hs;
  const int64_t wm = a.wm;
  const double c = kC;
  double acc = 0.0;
  for (int sg = sg0; sg < sg1; ++sg) {
    const double w = Tj[kTabC + 8 + sg];
    int64_t k;
    double th, s0, ds;
    if (!scalar_root(dh, wm, w, rr, ra, u, cdt2, nv, kg, &k, &th, &s0, &ds)) return false;
    const double sv0 = w * ddh[k & wm], sa0 = w * dddh[k & wm];
    const double s = s0 + th * ds;
    const double sv = sv0 + th * (w * ddh[(k + 1) & wm] - sv0);
    const double sa = sa0 + th * (w * dddh[(k + 1) & wm] - sa0);
    // a = rho - s p_j: a.a, a.p_j, a.p_i
    const double aj = ra - s, aiv = rp - s * ap;
    const double R2 = rr - s * (2.0 * ra - s);
    const double iR = rsqrt(R2);
    const double R = R2 * iR;
    const double Ru = c * R - sv * aj;  // R c - a . v
    const double iRu = 1.0 / Ru;
    const double f = kKe * (sg == 0 ? q : -q) * R * iRu * iRu * iRu;
    const double g = f * (c * c - sv * sv);
    const double pu = c * iR * aiv - sv * ap;  // p_i . u
    acc += g * pu + f * (pu * (sa * aj) - sa * ap * Ru);
  }
  *out = acc;
  return true;
}

// Contribution of dipole j to the driving field of receiver i at time u (steps), history 0..nv.
// float64: charge by charge (Eqs. r_1, r_2, E), charges sg0 .. sg1 - 1 (0 = +q, 1 = -q); returns
// p_i . E.
__device__ double pair_drive_f64(const RunArgs &a, int b, int i, int j, double u, int64_t nv, int64_t kg_fixed,
                                 int *err, int sg0 = 0, int sg1 = 2) {
  // (a centre whose retarded sample precedes the history: its charges are in the static
  // pre-history, which the general form takes directly)
  if (!a.org_pos && nv > 0 && kg_fixed >= 0) {
    double v;
    if (pair_drive_f64_scalar(a, b, i, j, u, nv, kg_fixed, sg0, sg1, &v)) return v;
  }
  const double cdt = kC * a.dt;
  const size_t bi = bidx(a, b, i), bj = bidx(a, b, j);
  // receiver at its origin; a moving origin at the stage time (half-step index 2u; moving runs start
  // at step 0 and keep every sample, so the index is absolute)
  const int64_t H = 2 * a.n_steps + 1;
  const int64_t hh = (int64_t)llrint(2.0 * u);
  const double *Ri = a.org_pos ? a.org_pos + (bi * H + hh) * 3 : a.origin + 3 * bi;
  const double *pi = a.axis + 3 * bi;
  TrajF64 tr;
  tr.dipole = true;
  tr.d = a.d + bj * a.hs;
  tr.dd = a.dd + bj * a.hs;
  tr.ddd = a.ddd + bj * a.hs;
  tr.wm = a.wm;
  for (int k = 0; k < 3; ++k) {
    tr.R[k] = a.origin[3 * bj + k];
    tr.ax[k] = a.axis[3 * bj + k];
  }
  if (a.org_pos) {
    tr.Rp = a.org_pos + bj * H * 3;
    tr.Rv = a.org_vel + bj * H * 3;
    tr.Ra = a.org_acc + bj * H * 3;
    for (int k = 0; k < 3; ++k) tr.R[k] = tr.Rp[6 * nv + k];  // the source now, for the first guess
  }
  const double q = a.q[bj];
  const double *Tj = a.rk4tab + bj * kTab;
  // first guess of the retarded sample: the centre delay (from the pair table for fixed origins)
  int64_t kg = kg_fixed;
  if (a.org_pos) {
    double dv[3] = {Ri[0] - tr.R[0], Ri[1] - tr.R[1], Ri[2] - tr.R[2]};
    kg = (int64_t)floor(u - sqrt(dot3(dv, dv)) / cdt);
  }
  double E[3] = {0.0, 0.0, 0.0};
  for (int sg = sg0; sg < sg1; ++sg) {
    tr.w = Tj[kTabC + 8 + sg];
    double p0[3], v[3] = {0, 0, 0}, ac[3] = {0, 0, 0};
    if (nv == 0) {
      // only the static pre-history exists: the root must precede t = 0
      tr.p(0, p0);
      double av[3] = {Ri[0] - p0[0], Ri[1] - p0[1], Ri[2] - p0[2]};
      if (u * cdt - sqrt(dot3(av, av)) > 0.0) {
        *err = PC_ERR_CAUSALITY;
        return 0.0;
      }
    } else {
      int64_t k;
      double th;
      int e = solve_f64(tr, nv + 1, 1, Ri, u, cdt, kg, &k, &th);
      if (e) {
        *err = (e == PC_ERR_HISTORY) ? PC_ERR_CAUSALITY : e;
        return 0.0;
      }
      if (k < 0 || (k == 0 && th == 0.0)) {
        tr.p(0, p0);
      } else {
        double p1[3], v1[3], a1[3];
        tr.p(k, p0);
        tr.p(k + 1, p1);
        tr.va(k, v, ac);
        tr.va(k + 1, v1, a1);
        for (int c = 0; c < 3; ++c) {
          p0[c] += th * (p1[c] - p0[c]);
          v[c] += th * (v1[c] - v[c]);
          ac[c] += th * (a1[c] - ac[c]);
        }
      }
    }
    double av[3] = {Ri[0] - p0[0], Ri[1] - p0[1], Ri[2] - p0[2]};
    lw_E_f64(sg == 0 ? q : -q, av, v, ac, E);
  }
  return dot3(pi, E);
}

// float32: the dipole pair in difference form from the float32 mirror; returns p_i . E in units
// of k_e e / (c dt)^2.  kb + xc is the retarded time of dipole j's centre.
// RING: the store is a ring (slot j & wm); otherwise it holds every sample at its index and the mask
// folds away at compile time (the mixed drive issues every instruction it executes)
template <bool RING>
__device__ float pair_drive_f32(const RunArgs &a, int b, int i, int j, int kb, float xc, const float4 g, int nvalid,
                                int *err) {
  const size_t bi = bidx(a, b, i), bj = bidx(a, b, j);
  const float *fj = a.dipf + bj * kDipF;
  // pair geometry from the table (fixed origins); the source's charge split and charge
  const float rn = g.x, rp = g.y, rpi = g.z, ppi = g.w;
  const float4 cj = *reinterpret_cast<const float4 *>(fj + 8);  // (p_z, mu+, mu-, q/e)
  const HistF32Ring H{a.H32 + bj * (size_t)a.hs, RING ? (int)a.wm : -1};
  // fast path: both charges on the segment of the centre's retarded time (packed solve), then only
  // the driving-field projection p_i . E of the pair
  {
    float fl;
    const int kc = Num<float>::floor_int(xc, fl);
    const int k = kb + kc;
    if (k < -1) {
      // the centre's retarded time lies a sample or more before t = 0; when both charges' offsets
      // (at most |s| samples) keep them there too, they rest at their first position with no
      // velocity or acceleration (Sec. 3.2), and their distances are exact without a solve:
      // R_c = |rho - s_c p|, delta_c = R_c - rn = s_c (s_c - 2 rp) / (R_c + rn)
      float x0, v0, a0;
      H.get_in(0, x0, v0, a0);
      const float sp = cj.y * x0, sm = -cj.z * x0;
      if ((float)kb + xc + fmaxf(fabsf(sp), fabsf(sm)) < -0.01f) {
        const float Rp = sqrtf(fmaxf(rn * rn + sp * (sp - 2.f * rp), 0.f));
        const float Rm = sqrtf(fmaxf(rn * rn + sm * (sm - 2.f * rp), 0.f));
        const float2 dl = make_float2(__fdividef(sp * (sp - 2.f * rp), Rp + rn), __fdividef(sm * (sm - 2.f * rp), Rm + rn));
        const float2 zero = make_float2(0.f, 0.f);
        if (Rp > 0.f && Rm > 0.f)
          return dipole_drive_fast(rn, rp, cj.y, cj.z, cj.w, make_float2(x0, x0), zero, zero, dl, rpi, ppi);
      }
    }
    if (k >= 0 && k <= nvalid - 2) {
      float x0, v0, a0, x1, v1, a1;
      H.get_in(k, x0, v0, a0);
      H.get_in(k + 1, x1, v1, a1);
      // the first segment may not be extended backwards, the last one only by kEndTol
      const float lo = (k == 0) ? 0.f : -kExtrap, hi = 1.f + ((k == nvalid - 2) ? kEndTol : kExtrap);
      float2 X, V, Ac, dl;
      if (dip_pair_states_fast(x0, v0, a0, x1, v1, a1, xc - fl, rn, rp, cj.y, cj.z, X, V, Ac, dl, 0.5f * (lo + hi),
                               0.5f * (hi - lo)))
        return dipole_drive_fast(rn, rp, cj.y, cj.z, cj.w, X, V, Ac, dl, rpi, ppi);
    }
  }
  // general case: the geometry again from the float records (origin offsets from hi + lo parts: the
  // hi difference of nearby origins is exact)
  const float *fi = a.dipf + bi * kDipF;
  const float rx = (fi[0] - fj[0]) + (fi[3] - fj[3]);
  const float ry = (fi[1] - fj[1]) + (fi[4] - fj[4]);
  const float rz = (fi[2] - fj[2]) + (fi[5] - fj[5]);
  const float rn2 = sqrtf(rx * rx + ry * ry + rz * rz);
  const float px = fj[6], py = fj[7], pz = fj[8];
  const float rp2 = rx * px + ry * py + rz * pz;
  float acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  uint8_t mk = 0;
  const int e = dipole_net<PC_TOTAL, float, HistF32Ring>(H, nvalid, kb, xc, rx, ry, rz, rn2, px, py, pz, rp2, cj.y, cj.z,
                                                     cj.w, 0.f, false, acc, mk);
  if (e) {
    *err = (e == PC_ERR_HISTORY) ? PC_ERR_CAUSALITY : e;
    return 0.f;
  }
  return acc[0] * fi[6] + acc[1] * fi[7] + acc[2] * fi[8];
}

// A source whose charges both still rest at their first position at their retarded times (a
// sample or more before t = 0, Sec. 3.2): their distances in closed form without a solve, then the
// driving-field projection, as in pair_drive_f32.  x0: the first sample's X; false where the
// closed form does not apply.
__device__ __forceinline__ bool static_pair_drive(float x0, const float4 cj, int kb, float xc, const float4 geo,
                                                  float &v) {
  const float rn = geo.x, rp = geo.y;
  const float sp = cj.y * x0, sm = -cj.z * x0;
  if (!((float)kb + xc + fmaxf(fabsf(sp), fabsf(sm)) < -0.01f)) return false;
  const float Rp = sqrtf(fmaxf(rn * rn + sp * (sp - 2.f * rp), 0.f));
  const float Rm = sqrtf(fmaxf(rn * rn + sm * (sm - 2.f * rp), 0.f));
  const float2 dl = make_float2(__fdividef(sp * (sp - 2.f * rp), Rp + rn), __fdividef(sm * (sm - 2.f * rp), Rm + rn));
  const float2 zero = make_float2(0.f, 0.f);
  if (!(Rp > 0.f && Rm > 0.f)) return false;
  v = dipole_drive_fast(rn, rp, cj.y, cj.z, cj.w, make_float2(x0, x0), zero, zero, dl, geo.z, geo.w);
  return true;
}

__device__ __forceinline__ float dot3f(float ax, float ay, float az, float bx, float by, float bz) {
  return fmaf(az, bz, fmaf(ay, by, ax * bx));
}

// Moving origins, mixed precision (Sec. 4.3 with Eqs. r_1, r_2, E): p_i . E of source j's two charges
// at the receiver's origin at half-step hh (time u = n0 + stage_f, history samples 0..n0 known), in
// the units of dipole_drive_fast.  Each charge sits at the origin plus its offset along the axis;
// within one history segment k both move linearly, the origin by W per sample.  Steps:
//  1. the origin's own retarded time k + t_o: |rho_k - t_o W| = T - t_o with rho_k = R_i(u) - P_j(k),
//     T = u - k (the root of that quadratic near T - |rho_k|; while t_o leaves [0, 1], k moves to
//     the segment it points at, at most three segments tried); rn = T - t_o, rho_o = rho_k - t_o W;
//  2. each charge's retarded time k + t_o - delta_c relative to it: with b = rho_o - s_c p_j and the
//     charge's velocity per sample m = W + w_c p_j, A delta^2 + 2 B delta + C = 0 where A = 1 - m.m,
//     B = rn - b.m, C = s_c (2 rho_o.p_j - s_c) (the fixed-origin quadratic with the origin's motion
//     added), solved as a series in A C / B^2 so that delta_c keeps its own precision;
//  3. E per charge in Griffiths' form E = (G / Ru^3) a - (G R / Ru^3) v - (R / Ru^2) acc with
//     a = rho_o + delta_c W - s_c p_j, v = V + s_c' p_j, acc = A + s_c'' p_j, Ru = R - a.v,
//     G = 1 - v.v + a.acc, R = rn + delta_c; the difference of the two charges' fields from the
//     differences of their inputs (da = dR W - ds p_j, dv = -dR dV + ds' p_j, ...), every product
//     differenced as d(f g) = df g+ + f- dg, so that the +-q cancellation costs no digits.
// A source still wholly in the static pre-history is the fixed dipole at its first position
// (static_pair_drive).  Returns false where neither applies (a retarded time on segment 0 or past the
// newest sample, a charge more than kExtrap samples off the origin's segment, a near source with
// near_f64 set); the caller then takes the float64 pair.
__device__ bool pair_drive_mov_f32(const RunArgs &a, int b, int i, int j, int n0, int hh, float stage_f, float &out) {
  const size_t bi = bidx(a, b, i), bj = bidx(a, b, j);
  const int64_t H = 2 * a.n_steps + 1;
  const float4 *Oi = a.omf + ((size_t)bi * H + hh) * 3;
  const float4 *Oj = a.omf + (size_t)bj * H * 3;  // sample k at Oj + 6 k (half-step index 2 k)
  const float4 ri0 = Oi[0], ri1 = Oi[1];
  const float *fi = a.dipf + bi * kDipF, *fj = a.dipf + bj * kDipF;
  // 1. the origin's retarded time: first guess from the origin at the block start
  int k;
  {
    const float4 p0 = Oj[6 * (size_t)n0], p1 = Oj[6 * (size_t)n0 + 1];
    const float rx = (ri0.x - p0.x) + (ri1.x - p1.x), ry = (ri0.y - p0.y) + (ri1.y - p1.y),
                rz = (ri0.z - p0.z) + (ri1.z - p1.z);
    float fl;
    k = n0 + Num<float>::floor_int(stage_f - sqrtf(dot3f(rx, ry, rz, rx, ry, rz)), fl);
  }
  if (k < 1) {
    // the static pre-history: before t = 0 the origin rests at its first sample and the charges at
    // their first offsets (Sec. 3.2), so a source whose two charges both have retarded times there is
    // a fixed dipole at rho_0 = R_i(u) - P_j(0): the fixed-origin form, no solve
    const float4 p0 = Oj[0], p1 = Oj[1];
    const float rx = (ri0.x - p0.x) + (ri1.x - p1.x), ry = (ri0.y - p0.y) + (ri1.y - p1.y),
                rz = (ri0.z - p0.z) + (ri1.z - p1.z);
    const float rn0 = sqrtf(dot3f(rx, ry, rz, rx, ry, rz));
    const float xu = ((float)n0 - rn0) + stage_f;  // the origin's retarded time if it precedes t = 0
    if (xu < 0.f) {
      if (a.near_L > 0.f && rn0 < a.near_L) return false;
      const float4 cj = *reinterpret_cast<const float4 *>(fj + 8);  // (p_z, mu+, mu-, q/e)
      const float4 geo = make_float4(rn0, dot3f(rx, ry, rz, fj[6], fj[7], cj.x), dot3f(rx, ry, rz, fi[6], fi[7], fi[8]),
                                     dot3f(fj[6], fj[7], cj.x, fi[6], fi[7], fi[8]));
      if (static_pair_drive(a.H32[bj * (size_t)a.hs].x, cj, 0, xu, geo, out)) return true;
    }
    return false;
  }
  float to = -1.f, T = 0.f, rkx = 0.f, rky = 0.f, rkz = 0.f, Wx = 0.f, Wy = 0.f, Wz = 0.f;
  for (int it = 0; it < 3; ++it) {
    if (k < 1 || k > n0 - 1) return false;
    const float4 *Pk = Oj + 6 * (size_t)k;
    const float4 a0 = Pk[0], a1 = Pk[1], b0 = Pk[6], b1 = Pk[7];
    rkx = (ri0.x - a0.x) + (ri1.x - a1.x);
    rky = (ri0.y - a0.y) + (ri1.y - a1.y);
    rkz = (ri0.z - a0.z) + (ri1.z - a1.z);
    Wx = (b0.x - a0.x) + (b1.x - a1.x);
    Wy = (b0.y - a0.y) + (b1.y - a1.y);
    Wz = (b0.z - a0.z) + (b1.z - a1.z);
    T = (float)(n0 - k) + stage_f;
    const float rk = sqrtf(dot3f(rkx, rky, rkz, rkx, rky, rkz));
    const float Ao = 1.f - dot3f(Wx, Wy, Wz, Wx, Wy, Wz);
    const float Bo = T - dot3f(rkx, rky, rkz, Wx, Wy, Wz);
    const float Co = (T - rk) * (T + rk);
    to = Co / (Bo + sqrtf(fmaxf(Bo * Bo - Ao * Co, 0.f)));
    if (!(to == to)) return false;
    if (to >= 0.f && to <= 1.f) break;
    // the segment the root on this one's linear extension falls in (one or more samples away)
    k += (int)fmaxf(-64.f, fminf(64.f, floorf(to)));
  }
  if (!(to >= 0.f && to <= 1.f)) return false;
  const float rn = T - to;
  if (a.near_L > 0.f && rn < a.near_L) return false;
  const float rox = rkx - to * Wx, roy = rky - to * Wy, roz = rkz - to * Wz;
  const float pjx = fj[6], pjy = fj[7], pjz = fj[8], mup = fj[9], mum = fj[10], qs = fj[11];
  const float pix = fi[6], piy = fi[7], piz = fi[8];
  const float rp = dot3f(rox, roy, roz, pjx, pjy, pjz), rW = dot3f(rox, roy, roz, Wx, Wy, Wz);
  const float Wp = dot3f(Wx, Wy, Wz, pjx, pjy, pjz), W2 = dot3f(Wx, Wy, Wz, Wx, Wy, Wz);
  // 2. the two charges' retarded times relative to the origin's (+ charge in .x, - charge in .y)
  const HistF32Ring Hj{a.H32 + bj * (size_t)a.hs, -1};
  float x0, v0, a0, x1, v1, a1;
  Hj.get_in(k, x0, v0, a0);
  Hj.get_in(k + 1, x1, v1, a1);
  const float dx = x1 - x0, dvm = v1 - v0, dam = a1 - a0;
  const float Xc = x0 + to * dx;
  const float2 mu = make_float2(mup, -mum);
  float2 dl, th;
  float epsum = 0.f;
  {
    const float sc[2] = {mu.x * Xc, mu.y * Xc}, w[2] = {mu.x * dx, mu.y * dx};
    float dlc[2], thc[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float A = 1.f - (W2 + w[c] * (2.f * Wp + w[c]));
      const float B = rn - (rW + w[c] * rp - sc[c] * (Wp + w[c]));
      const float C = sc[c] * (2.f * rp - sc[c]);
      const float r = __fdividef(1.f, B);
      const float Cr = C * r;
      const float h = 0.5f * Cr;
      const float eps = A * Cr * r;
      const float ndl = fmaf(h, eps * fmaf(eps, 0.125f, 0.25f), h);  // -delta_c
      dlc[c] = -ndl;
      thc[c] = to + ndl;
      epsum += fabsf(eps);
    }
    dl = make_float2(dlc[0], dlc[1]);
    th = make_float2(thc[0], thc[1]);
  }
  // the last segment may be extended only by kEndTol (no sample beyond n0)
  const float lo = -kExtrap, hi = 1.f + ((k == n0 - 1) ? kEndTol : kExtrap);
  if (!(th.x >= lo && th.x <= hi && th.y >= lo && th.y <= hi && epsum < 1e-2f)) return false;
  // 3. the charges' states at their retarded times
  const float Xp = x0 + th.x * dx, Xm = x0 + th.y * dx;
  const float Sp = v0 + th.x * dvm, Sm = v0 + th.y * dvm;
  const float Lp = a0 + th.x * dam, Lm = a0 + th.y * dam;
  const float sm = mu.y * Xm, sdm = mu.y * Sm, sam = mu.y * Lm;
  const float ds = mup * Xp + mum * Xm, dsd = mup * Sp + mum * Sm, dsa = mup * Lp + mum * Lm;
  const float dR = dl.x - dl.y;
  const float Rm = rn + dl.y, Rp = rn + dl.x;
  // the origin's velocity and acceleration on segment k (the - charge's time) and their slopes
  const float4 *Pk = Oj + 6 * (size_t)k;
  const float4 c00 = Pk[0], c01 = Pk[1], c02 = Pk[2], c10 = Pk[6], c11 = Pk[7], c12 = Pk[8];
  const float dVx = c10.w - c00.w, dVy = c11.w - c01.w, dVz = c12.x - c02.x;
  const float dAx = c12.y - c02.y, dAy = c12.z - c02.z, dAz = c12.w - c02.w;
  const float vmx = fmaf(th.y, dVx, c00.w) + sdm * pjx, vmy = fmaf(th.y, dVy, c01.w) + sdm * pjy,
              vmz = fmaf(th.y, dVz, c02.x) + sdm * pjz;
  const float gmx = fmaf(th.y, dAx, c02.y) + sam * pjx, gmy = fmaf(th.y, dAy, c02.z) + sam * pjy,
              gmz = fmaf(th.y, dAz, c02.w) + sam * pjz;
  const float amx = rox + dl.y * Wx - sm * pjx, amy = roy + dl.y * Wy - sm * pjy, amz = roz + dl.y * Wz - sm * pjz;
  // differences (+ minus -) of position, velocity and acceleration
  const float Dax = dR * Wx - ds * pjx, Day = dR * Wy - ds * pjy, Daz = dR * Wz - ds * pjz;
  const float Dvx = dsd * pjx - dR * dVx, Dvy = dsd * pjy - dR * dVy, Dvz = dsd * pjz - dR * dVz;
  const float Dgx = dsa * pjx - dR * dAx, Dgy = dsa * pjy - dR * dAy, Dgz = dsa * pjz - dR * dAz;
  const float apx = amx + Dax, apy = amy + Day, apz = amz + Daz;
  const float vpx = vmx + Dvx, vpy = vmy + Dvy, vpz = vmz + Dvz;
  const float gpx = gmx + Dgx, gpy = gmy + Dgy, gpz = gmz + Dgz;
  // R_u and G of the - charge and their differences
  const float Rum = Rm - dot3f(amx, amy, amz, vmx, vmy, vmz);
  const float dRu = dR - (dot3f(Dax, Day, Daz, vpx, vpy, vpz) + dot3f(amx, amy, amz, Dvx, Dvy, Dvz));
  const float Rup = Rum + dRu;
  const float Gm = 1.f - dot3f(vmx, vmy, vmz, vmx, vmy, vmz) + dot3f(amx, amy, amz, gmx, gmy, gmz);
  const float dG = dot3f(Dax, Day, Daz, gpx, gpy, gpz) + dot3f(amx, amy, amz, Dgx, Dgy, Dgz) -
                   dot3f(Dvx, Dvy, Dvz, vpx + vmx, vpy + vmy, vpz + vmz);
  const float ip = __fdividef(1.f, Rup), im = __fdividef(1.f, Rum);
  const float di = -dRu * ip * im;
  const float di2 = di * (ip + im);
  const float di3 = di * (ip * ip + ip * im + im * im);
  const float ip2 = ip * ip, ip3 = ip2 * ip, im2 = im * im, im3 = im2 * im;
  // coefficients of a, v, acc: C = G / Ru^3, K = G R / Ru^3, L = R / Ru^2 (- charge and differences)
  const float Cm = Gm * im3, dC = dG * ip3 + Gm * di3;
  const float GRm = Gm * Rm, dGR = dG * Rp + Gm * dR;
  const float Km = GRm * im3, dK = dGR * ip3 + GRm * di3;
  const float Lm_ = Rm * im2, dL = dR * ip2 + Rm * di2;
  const float pE = dC * dot3f(apx, apy, apz, pix, piy, piz) + Cm * dot3f(Dax, Day, Daz, pix, piy, piz) -
                   dK * dot3f(vpx, vpy, vpz, pix, piy, piz) - Km * dot3f(Dvx, Dvy, Dvz, pix, piy, piz) -
                   dL * dot3f(gpx, gpy, gpz, pix, piy, piz) - Lm_ * dot3f(Dgx, Dgy, Dgz, pix, piy, piz);
  out = qs * pE;
  return true;
}

// The grid path's float32 source loop (sources j = j_lo + m, step slots): the pair-table rows, the
// sources' records and history rows are reached by 32-bit indices and a pointer that advances with
// j (no 64-bit products per source), and pair_drive_f32's fast path and static pre-history are
// written out here; every other case (the general solve) goes to pair_drive_f32 itself, which then
// takes the same steps as for the plain loop.  Groups of 32 sources are summed in float32, the
// group sums added with Kahan compensation into (accf, comp).
template <bool RING>
__device__ __forceinline__ void drive_sources_grid(const RunArgs &a, int b, int i, int64_t n0, float stage_f, int m,
                                                   int slots, int j_lo, int j_hi, float &accf, float &comp,
                                                   int *err) {
  const size_t row = (size_t)bidx(a, b, i) * a.N;
  const size_t b0 = bidx(a, b, 0);
  const int2 *pd = a.delay + row;
  const float4 *pg = a.pgeo + row;
  const float4 *pc = reinterpret_cast<const float4 *>(a.dipf + b0 * kDipF) + 2;  // (p_z, mu+, mu-, q/e)
  const size_t hstep = (size_t)slots * (size_t)a.hs;
  const int mask = RING ? (int)a.wm : -1;
  const int n0i = (int)n0, nvalid = n0i + 1;
  for (int j0 = j_lo + m; j0 < j_hi; j0 += 32 * slots) {
    const int jend = min(j_hi, j0 + 32 * slots);
    float grp = 0.f;
    const float4 *hj = a.H32 + (b0 + (size_t)j0) * (size_t)a.hs;
    for (int j = j0; j < jend; j += slots, hj += hstep) {
      if (j == i) continue;
      const int2 dl = pd[j];
      const float4 geo = pg[j];
      const float xs = stage_f - __int_as_float(dl.y);
      float flf;
      const int fl = Num<float>::floor_int(xs, flf);
      const int k = n0i - dl.x + fl;
      const float xc = xs - flf;
      if (k >= 0 && k <= nvalid - 2) {
        const float4 cj = pc[j * (kDipF / 4)];
        const float4 h0 = hj[k & mask], h1 = hj[(k + 1) & mask];
        const float lo = (k == 0) ? 0.f : -kExtrap, hi = 1.f + ((k == nvalid - 2) ? kEndTol : kExtrap);
        float2 X, V, Ac, dlt;
        if (dip_pair_states_fast(h0.x, h0.y, h0.z, h1.x, h1.y, h1.z, xc, geo.x, geo.y, cj.y, cj.z, X, V, Ac, dlt,
                                 0.5f * (lo + hi), 0.5f * (hi - lo))) {
          grp += dipole_drive_fast(geo.x, geo.y, cj.y, cj.z, cj.w, X, V, Ac, dlt, geo.z, geo.w);
          continue;
        }
      } else if (k < -1) {
        float v;
        if (static_pair_drive(hj[0].x, pc[j * (kDipF / 4)], k, xc, geo, v)) {
          grp += v;
          continue;
        }
      }
      grp += pair_drive_f32<RING>(a, b, i, j, k, xc, geo, nvalid, err);
    }
    const float y = grp - comp;
    const float t = accf + y;
    comp = (t - accf) - y;
    accf = t;
  }
}

// Phase A for one receiver (one warp): stage fields E_d(n0 + (s+1)/2), s < ns, into Es[1 + s];
// ns == 0 evaluates E_d(n0) into Es[0].  History samples 0..n0 are known.  GROUPS: the float32
// sources through drive_sources_grid (the grid path, whose warps loop over many sources; in the
// persistent kernel a lane has one or two, and the group loop only raises its registers).
// MOV: moving origins in the mixed drive (pair_drive_mov_f32, the float64 pair where it declines).
template <bool MIXED, bool NEAR = false, bool RING = true, bool GROUPS = false, bool MOV = false>
__device__ void drive_phase(const RunArgs &a, int b, int i, int64_t n0, int ns, double *sh /* [32] */, int *err,
                            int j_lo, int j_hi, double *dst_row, int sgsel = -1) {
  const int lane = threadIdx.x & 31;
  const int nst = ns > 0 ? ns : 1;
  const int slots = 32 / nst;
  const int s = lane % nst, m = lane / nst;
  const double stage = ns > 0 ? 0.5 * (s + 1) : 0.0;  // the float64 drive's
  // float(s + 1) from the bits (exact below 2^23): conversion instructions issue to the narrow
  // float64 unit
  const float stage_f = ns > 0 ? 0.5f * (__int_as_float(0x4B000000 | (s + 1)) - 8388608.f) : 0.f;
  double accd = 0.0;
  float accf = 0.f, comp = 0.f;
  // fewer float64 sources than half the slots (small configurations): the two charges of each
  // take two slots, which halves the serial float64 chain of a slot
  // (sgsel = 0 or 1: only that charge of every float64 source, the other taken by another warp)
  const bool split = sgsel < 0 && (!MIXED || NEAR) && 2 * (j_hi - j_lo) <= slots;
  // source j's charges sg0 .. sg1 - 1
  auto source = [&](int j, int sg0, int sg1) {
    if (j == i) return;
    if constexpr (MIXED && MOV) {
      // the receiver at its origin of the stage time: half-step index 2 n0 + s + 1 (2 n0 for ns = 0)
      float v;
      if (pair_drive_mov_f32(a, b, i, j, (int)n0, 2 * (int)n0 + (ns > 0 ? s + 1 : 0), stage_f, v)) {
        const float y = v - comp;
        const float t = accf + y;
        comp = (t - accf) - y;
        accf = t;
      } else {
        // (the float64 pair takes its first guess from the moving origins)
        accd += pair_drive_f64(a, b, i, j, (double)n0 + stage, n0, 0, err, 0, 2);
      }
      return;
    }
    if (MIXED) {
      // retarded time of j's centre: n0 + stage - |R_i - R_j| / (c dt), split in integer + fraction
      const size_t ij = (size_t)bidx(a, b, i) * a.N + j;
      const int2 dl = a.delay[ij];
      const float4 geo = a.pgeo[ij];
      const float xs = stage_f - __int_as_float(dl.y);
      float flf;
      const int fl = Num<float>::floor_int(xs, flf);
      if (NEAR && geo.x < a.near_L) {
        // a near source whose radiative coupling float32 cannot resolve: the float64 pair
        accd += pair_drive_f64(a, b, i, j, (double)n0 + stage, n0, (int)n0 - dl.x + fl, err, sg0, sg1);
        return;
      }
      if (sg0 == 1) return;  // the float32 pair takes both charges at once
      const float v = pair_drive_f32<RING>(a, b, i, j, (int)n0 - dl.x + fl, xs - flf, geo, (int)n0 + 1, err);
      // Kahan sum over sources
      const float y = v - comp;
      const float t = accf + y;
      comp = (t - accf) - y;
      accf = t;
    } else {
      // first guess: the sample of the centre's retarded time, n0 + stage - delay
      const int2 dl = a.delay[(size_t)bidx(a, b, i) * a.N + j];
      const int kg = (int)n0 - dl.x + Num<float>::floor_int(stage_f - __int_as_float(dl.y));
      accd += pair_drive_f64(a, b, i, j, (double)n0 + stage, n0, kg, err, sg0, sg1);
    }
  };
  if (m < slots) {
    if constexpr (MIXED && !NEAR && !MOV && GROUPS) {
      drive_sources_grid<RING>(a, b, i, n0, stage_f, m, slots, j_lo, j_hi, accf, comp, err);
    } else if constexpr (MIXED && !NEAR) {
      for (int j = j_lo + m; j < j_hi; j += slots) source(j, 0, 2);
    } else {
      // one loop, so that the float64 pair is inlined once
      const int nh = split ? 2 * (j_hi - j_lo) : j_hi - j_lo;
      for (int h = m; h < nh; h += slots) {
        const int sg0 = split ? h & 1 : (sgsel < 0 ? 0 : sgsel);
        source(j_lo + (split ? h >> 1 : h), sg0, (split || sgsel >= 0) ? sg0 + 1 : 2);
      }
    }
  }
  if (MIXED && !NEAR && !MOV) {
    // the slots' float32 sums added in float32, one conversion per stage (conversions and float64
    // arithmetic issue to the narrow float64 unit)
    float *shf = reinterpret_cast<float *>(sh);
    shf[lane] = (m < slots) ? accf : 0.f;
    __syncwarp();
    if (lane < nst) {
      float t = 0.f;
      for (int mm = 0; mm < slots; ++mm) t += shf[mm * nst + lane];
      dst_row[ns > 0 ? 1 + lane : 0] = (double)t * a.e_unit;
    }
  } else {
    double mine = MIXED ? (double)accf * a.e_unit + accd : accd;
    sh[lane] = (m < slots) ? mine : 0.0;
    __syncwarp();
    if (lane < nst) {
      double t = 0.0;
      for (int mm = 0; mm < slots; ++mm) t += sh[mm * nst + lane];
      dst_row[ns > 0 ? 1 + lane : 0] = t;
    }
  }
  __syncwarp();
}

// NEAR: the mixed drive sums its near sources in float64 (near_f64 > 0), a separate instantiation
// so that the float32 source loop of the default one keeps its registers.  At most two CTAs share
// an SM here (one per configuration), so the register bound is one CTA's: held to the 80 of the
// compiler's default choice the time loop spilled and ran 7 % slower.
template <bool MIXED, bool NEAR = false, bool RING = true, bool MOV = false>
__global__ void __launch_bounds__(kRunWarps * 32, 1) lo_run_kernel(const RunArgs a) {
  const int b = blockIdx.x;
  const int N = a.N;
  const int64_t So = a.n_steps - a.n_begin + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double sh[kRunWarps][32];
  // the stage fields of the block and each receiver's state (d, d') at the block's start stay in
  // shared memory (the phases hand them over within the CTA, not through global memory); the
  // float64 drive's second-charge partial fields (2 N <= kRunWarps) beside them
  __shared__ double s_Es[kSmallN][2 * kMaxBlock + 1];
  __shared__ double s_ys[kSmallN][2];
  __shared__ double s_Ep[kRunWarps / 2][2 * kMaxBlock + 1];
  __shared__ float s_fsc[kSmallN][3];
  extern __shared__ double s_tab[];  // [N][kTab]: the configuration's RK4 tables (dynamic)
  __shared__ int s_stop, s_K;
  if (threadIdx.x == 0) {
    s_K = a.kblock[b];
    s_stop = 0;
  }
  {
    const double *gT = a.rk4tab + bidx(a, b, 0) * kTab;  // the configuration's rows are contiguous
    for (int t = threadIdx.x; t < N * kTab; t += blockDim.x) s_tab[t] = gT[t];
    for (int t = threadIdx.x; t < 3 * N; t += blockDim.x) s_fsc[t / 3][t % 3] = dbl2flt(gT[(t / 3) * kTab + kTabC + 4 + t % 3]);
  }
  // (the first sample and, when resuming, the earlier ones are in the store: lo_first_kernel)
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const size_t sl = bidx(a, b, i) * (size_t)a.hs + (a.n_begin & a.wm);
    s_ys[i][0] = a.d[sl];
    s_ys[i][1] = a.dd[sl];
    if (a.state_in) s_Es[i][0] = a.Es[bidx(a, b, i) * (2 * kMaxBlock + 1)];
  }
  __syncthreads();
  const int K = s_K;
  // ---- E_d at the first step: the resumed state's, or that of the static configuration ----
  for (int i = warp; i < N; i += kRunWarps) {
    if (!a.state_in) {
      int err = 0;
      drive_phase<MIXED, NEAR, RING, false, MOV>(a, b, i, a.n_begin, 0, sh[warp], &err, 0, N, s_Es[i]);
      if (err) {
        set_status(a.status, err);
        s_stop = 1;
      }
    }
    __syncwarp();
    if (lane == 0 && a.Ed) a.Ed[bidx(a, b, i) * So] = s_Es[i][0];
  }
  __syncthreads();
  for (int64_t n0 = a.n_begin; n0 < a.n_steps; n0 += K) {
    if (s_stop) break;
    const int kb = (int)min((int64_t)K, a.n_steps - n0);
    // phase A: all stage fields of the block.  A float64 drive whose lanes are all taken while
    // warps are idle (2 N <= kRunWarps < 2 N * 32 / (2 kb)) gives each charge of the sources its own
    // warp: warp 2i + h sums charge h of receiver i's sources, h = 1 into Epart, added after (not
    // in the mixed instantiations, whose registers it would raise)
    const int nst = 2 * kb;
    const bool xsplit = !MIXED && 2 * N <= kRunWarps && 2 * N > 32 / nst;
    for (int w = warp; w < (xsplit ? 2 * N : N); w += kRunWarps) {
      int err = 0;
      drive_phase<MIXED, NEAR, RING, false, MOV>(a, b, xsplit ? w >> 1 : w, n0, nst, sh[warp], &err, 0, N,
                                     (xsplit && (w & 1)) ? s_Ep[w >> 1] : s_Es[xsplit ? w >> 1 : w],
                                     xsplit ? w & 1 : -1);
      if (err) {
        set_status(a.status, err);
        s_stop = 1;
      }
    }
    __syncthreads();
    if (s_stop) break;
    if (xsplit) {
      for (int t = threadIdx.x; t < N * nst; t += blockDim.x) s_Es[t / nst][1 + t % nst] += s_Ep[t / nst][1 + t % nst];
      __syncthreads();
    }
    // phase B: the kb RK4 steps of each receiver, one warp per receiver, one lane per step
    for (int i = warp; i < N; i += kRunWarps) {
      int stop = 0;
      rk4_block_warp<MIXED, true>(a, b, i, n0, kb, &stop, s_Es[i], s_ys[i], s_tab + (size_t)i * kTab, s_fsc[i]);
      if (stop && lane == 0) s_stop = 1;
    }
    __syncthreads();
  }
  // E_d at the last step for a state saved after the run (lo_save_kernel)
  for (int i = threadIdx.x; i < N; i += blockDim.x) a.Es[bidx(a, b, i) * (2 * kMaxBlock + 1)] = s_Es[i][0];
}

// The first sample of the call (step n_begin) into the store and the outputs: at rest with moment d0
// (Sec. 3.2) for a fresh run; for a resumed one, the state's samples n_begin - D .. n_begin into the
// store's slots and its E_d(n_begin) into the stage fields.  Grid-stride over the dipoles; runs after
// lo_tables_kernel (the mirror's scales).
template <bool MIXED>
__global__ void lo_first_kernel(const RunArgs a) {
  const int64_t nbn = (int64_t)a.B * a.N;
  const int64_t So = a.n_steps - a.n_begin + 1;
  const double L = kC * a.dt;
  for (int64_t bi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; bi < nbn; bi += (int64_t)gridDim.x * blockDim.x) {
    const double *T = a.rk4tab + bi * kTab;
    const size_t row = (size_t)bi * a.hs;
    if (!a.state_in) {
      const size_t sl = row + (a.n_begin & a.wm);
      a.d[sl] = a.d0[bi];
      a.dd[sl] = 0.0;
      a.ddd[sl] = 0.0;
      if (MIXED) a.H32[sl] = make_float4((float)(a.d0[bi] / (a.q[bi] * L)), 0.f, 0.f, 0.f);
    } else {
      const int64_t D = (int64_t)a.state_in[2];
      const double *smp = a.state_in + 4 + nbn + (size_t)bi * (D + 1) * 3;
      for (int64_t t = 0; t <= D; ++t) {
        const int64_t k = a.n_begin - D + t;
        if (k < 0) continue;
        const size_t sl = row + (k & a.wm);
        const double x = smp[3 * t], v = smp[3 * t + 1], ac = smp[3 * t + 2];
        a.d[sl] = x;
        a.dd[sl] = v;
        a.ddd[sl] = ac;
        if (MIXED)
          a.H32[sl] = (k == 0) ? make_float4((float)(x / (a.q[bi] * L)), 0.f, 0.f, 0.f)
                               : make_float4(dbl2flt(x) * dbl2flt(T[kTabC + 4]), dbl2flt(v) * dbl2flt(T[kTabC + 5]),
                                             dbl2flt(ac) * dbl2flt(T[kTabC + 6]), 0.f);
      }
      a.Es[bi * (2 * kMaxBlock + 1)] = a.state_in[4 + bi];
    }
    const size_t sl = row + (a.n_begin & a.wm);
    const double x = a.d[sl], v = a.dd[sl], ac = a.ddd[sl];
    const size_t o = (size_t)bi * So;
    if (a.od) a.od[o] = x;
    if (a.odd) a.odd[o] = v;
    if (a.oddd) a.oddd[o] = ac;
    if (a.energy) a.energy[o] = T[kTabC + 7] * (T[kTabC + 1] * x * x + v * v);
    if (a.ke && a.n_begin >= a.ke_first && a.n_begin < a.ke_first + a.ke_len) {
      const size_t kk = (size_t)bi * a.ke_len + (size_t)(a.n_begin - a.ke_first);
      a.ke[kk] = T[kTabC + 7] * v * v;
      if (a.kdd) a.kdd[kk] = v;
    }
  }
}

// The state at step n_steps (the call's last) from the store and the stage fields: see the state
// layout above.  Grid-stride over the dipoles and their samples.
__global__ void lo_save_kernel(const RunArgs a, int64_t D) {
  const int64_t nbn = (int64_t)a.B * a.N;
  double *st = a.state_out;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st[0] = kStateMagic;
    st[1] = (double)a.n_steps;
    st[2] = (double)D;
    st[3] = (double)nbn;
  }
  const int64_t tot = nbn * (D + 1);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t bi = idx / (D + 1), t = idx % (D + 1);
    const int64_t k = a.n_steps - D + t;
    double *o = st + 4 + nbn + 3 * idx;
    if (k < 0) {
      o[0] = a.d0[bi];
      o[1] = 0.0;
      o[2] = 0.0;
    } else {
      const size_t sl = (size_t)bi * a.hs + (k & a.wm);
      o[0] = a.d[sl];
      o[1] = a.dd[sl];
      o[2] = a.ddd[sl];
    }
    if (t == 0) st[4 + bi] = a.Es[bi * (2 * kMaxBlock + 1)];
  }
}

// Per-run tables: float records of every dipole, centre-to-centre delays of every pair, and the
// causal block length of every configuration (the smallest distance between an origin and another
// dipole's charges, which sit up to |r_dip| from their origin; three times the initial amplitude
// is allowed for).  One CTA per configuration.
__global__ void lo_tables_kernel(const RunArgs a) {
  const int b = blockIdx.x;
  const int N = a.N;
  const double L = kC * a.dt;
  __shared__ double s_smax[256];
  double smax = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const size_t bi = bidx(a, b, i);
    float *f = a.dipf + bi * kDipF;
    {
      const double *ax = a.axis + 3 * bi;
      if (!(fabs(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2] - 1.0) <= kAxisTol)) set_status(a.status, PC_ERR_ARG);
    }
    for (int c = 0; c < 3; ++c) {
      const double x = a.origin[3 * bi + c] / L;
      const float hi = (float)x;
      f[c] = hi;
      f[3 + c] = (float)(x - (double)hi);
      f[6 + c] = (float)a.axis[3 * bi + c];
    }
    rk4_table(a, bi);
    const double m1 = a.m1[bi], m2 = a.m2[bi];
    f[9] = (float)(m2 / (m1 + m2));
    f[10] = (float)(m1 / (m1 + m2));
    f[11] = (float)(a.q[bi] / kE);
    smax = fmax(smax, fabs(a.d0[bi] / a.q[bi]));
  }
  s_smax[threadIdx.x] = smax;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int t = 1; t < blockDim.x; ++t) smax = fmax(smax, s_smax[t]);
    const double rmin = __longlong_as_double((long long)a.rstat[3 * b]);
    const double vmax = __longlong_as_double((long long)a.rstat[3 * b + 1]);
    const double rmax = __longlong_as_double((long long)a.rstat[3 * b + 2]);
    // within a block of K steps a source origin moves at most vmax K dt closer
    const double kk = floor((rmin - 3.0 * smax) / (L * (1.0 + vmax / kC)));
    a.kblock[b] = (int)fmax(1.0, fmin((double)kMaxBlock, kk));
    // the oldest sample a block's retarded times reach, behind the block's start: the largest
    // centre delay, the charges' offsets (three times the initial amplitude) and a few samples of
    // the solves' search
    a.reach[b] = (int)fmin(ceil(rmax / L) + ceil(3.0 * smax / L) + 8.0, 1073741824.0);
  }
}

// The float32 mirror of moving origins for the mixed drive (RunArgs::omf), once per run,
// grid-stride over the [B][N][2 n_steps + 1] half-step samples.
__global__ void lo_origin_mirror_kernel(const RunArgs a) {
  const int64_t H = 2 * a.n_steps + 1, n = (int64_t)a.B * a.N * H;
  const double iL = 1.0 / (kC * a.dt), ic = 1.0 / kC, adt = a.dt / kC;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double *p = a.org_pos + 3 * t, *v = a.org_vel + 3 * t, *ac = a.org_acc + 3 * t;
    float hi[3], lo[3];
    for (int c = 0; c < 3; ++c) {
      const double x = p[c] * iL;
      hi[c] = (float)x;
      lo[c] = (float)(x - (double)hi[c]);
    }
    float4 *o = a.omf + 3 * t;
    o[0] = make_float4(hi[0], hi[1], hi[2], (float)(v[0] * ic));
    o[1] = make_float4(lo[0], lo[1], lo[2], (float)(v[1] * ic));
    o[2] = make_float4((float)(v[2] * ic), (float)(ac[0] * adt), (float)(ac[1] * adt), (float)(ac[2] * adt));
  }
}

// Moving origins: each origin's largest distance from its first sample over the run (RunArgs::odisp),
// one thread per dipole.
__global__ void lo_origin_disp_kernel(const RunArgs a) {
  const int64_t H = 2 * a.n_steps + 1, nbn = (int64_t)a.B * a.N;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nbn; t += (int64_t)gridDim.x * blockDim.x) {
    const double *p = a.org_pos + t * H * 3;
    double d2 = 0.0;
    for (int64_t h = 1; h < H; ++h) {
      const double ex = p[3 * h] - p[0], ey = p[3 * h + 1] - p[1], ez = p[3 * h + 2] - p[2];
      d2 = fmax(d2, ex * ex + ey * ey + ez * ez);
    }
    a.odisp[t] = sqrt(d2);
  }
}

// Moving origins, after lo_pairs_kernel: the exact closest approach over the run of every pair
// i < j whose distance can fall to the configuration's bound in a.rstat (|R_i(0) - R_j(0)| - D_i
// - D_j <= bound: the triangle inequality bounds it from below); the pair that attains the minimum
// is one of them, so the minimum over these scans is the closest approach of the configuration.
// Grid: x over pairs, y over configurations.
__global__ void __launch_bounds__(256) lo_closest_kernel(const RunArgs a) {
  const int N = a.N;
  const int64_t NN = (int64_t)N * N;
  const int64_t H = 2 * a.n_steps + 1;
  for (int b = blockIdx.y; b < a.B; b += gridDim.y) {
    const double bound = __longlong_as_double((long long)a.rstat[3 * b]);
    for (int64_t ij = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ij < NN;
         ij += (int64_t)gridDim.x * blockDim.x) {
      const int i = (int)(ij / N), j = (int)(ij % N);
      if (i >= j) continue;
      const size_t bi = bidx(a, b, i), bj = bidx(a, b, j);
      const double *Ri = a.origin + 3 * bi, *Rj = a.origin + 3 * bj;
      const double dx = Ri[0] - Rj[0], dy = Ri[1] - Rj[1], dz = Ri[2] - Rj[2];
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      if (r - a.odisp[bi] - a.odisp[bj] > bound * (1.0 + 1e-12)) continue;
      // squared distances, one square root
      double r2min = r * r;
      for (int64_t h = 0; h < H; ++h) {
        const double *pi_ = a.org_pos + (bi * H + h) * 3, *pj_ = a.org_pos + (bj * H + h) * 3;
        const double ex = pi_[0] - pj_[0], ey = pi_[1] - pj_[1], ez = pi_[2] - pj_[2];
        r2min = fmin(r2min, ex * ex + ey * ey + ez * ez);
      }
      atomicMin(a.rstat + 3 * b, (unsigned long long)__double_as_longlong(sqrt(r2min)));
    }
  }
}

// Presets a.rstat to (a large distance, 0, 0): 0x7f7f... is about 1.4e306 as a double.
__global__ void lo_rstat_init_kernel(const RunArgs a) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.B) return;
  a.rstat[3 * b] = 0x7f7f7f7f7f7f7f7full;
  a.rstat[3 * b + 1] = 0ull;
  a.rstat[3 * b + 2] = 0ull;
}

// Per pair (i, j) of a configuration: the centre delay |R_i - R_j| / (c dt) (the first guess of
// the retarded-time solves; its integer part capped at 2^30, beyond every history), the float32
// pair geometry of the mixed drive, and the configuration's closest origin distance (over the run
// for moving origins) and largest origin speed, for the causal block length.  Grid: x over pair
// blocks, y over configurations.
__global__ void __launch_bounds__(256) lo_pairs_kernel(const RunArgs a) {
  __shared__ double s_r[256], s_v[256], s_x[256];
  const int N = a.N;
  const int64_t NN = (int64_t)N * N;
  const double L = kC * a.dt;
  const int64_t H = 2 * a.n_steps + 1;
  for (int b = blockIdx.y; b < a.B; b += gridDim.y) {
    double rmin = 1e300, vmax = 0.0, rmax = 0.0;
    for (int64_t ij = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ij < NN;
         ij += (int64_t)gridDim.x * blockDim.x) {
      const int i = (int)(ij / N), j = (int)(ij % N);
      const size_t bi = bidx(a, b, i), bj = bidx(a, b, j);
      const double *Ri = a.origin + 3 * bi, *Rj = a.origin + 3 * bj;
      const double dx = Ri[0] - Rj[0], dy = Ri[1] - Rj[1], dz = Ri[2] - Rj[2];
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      if (i != j) {
        rmin = fmin(rmin, r);
        rmax = fmax(rmax, r);
        // moving origins: r + D_i + D_j bounds the pair's distance from above at every time, so
        // their minimum bounds the closest approach; lo_closest_kernel then scans the pairs that
        // can reach below it
        if (a.org_pos) rmin = fmin(rmin, r + a.odisp[bi] + a.odisp[bj]);
      } else if (a.org_pos) {
        double v2max = 0.0;
        for (int64_t h = 0; h < H; ++h) {
          const double *vi = a.org_vel + (bi * H + h) * 3;
          v2max = fmax(v2max, vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]);
        }
        vmax = fmax(vmax, sqrt(v2max));
      }
      const double x = r / L;
      const double fl = floor(x);
      a.delay[bi * N + j] = make_int2((int)fmin(fl, 1073741824.0), __float_as_int((float)(x - fl)));
      if (a.pgeo) {
        const double *pi_ = a.axis + 3 * bi, *pj_ = a.axis + 3 * bj;
        const double rx = dx / L, ry = dy / L, rz = dz / L;
        a.pgeo[bi * N + j] =
            make_float4((float)x, (float)(rx * pj_[0] + ry * pj_[1] + rz * pj_[2]),
                        (float)(rx * pi_[0] + ry * pi_[1] + rz * pi_[2]),
                        (float)(pj_[0] * pi_[0] + pj_[1] * pi_[1] + pj_[2] * pi_[2]));
      }
    }
    s_r[threadIdx.x] = rmin;
    s_v[threadIdx.x] = vmax;
    s_x[threadIdx.x] = rmax;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) {
        s_r[threadIdx.x] = fmin(s_r[threadIdx.x], s_r[threadIdx.x + w]);
        s_v[threadIdx.x] = fmax(s_v[threadIdx.x], s_v[threadIdx.x + w]);
        s_x[threadIdx.x] = fmax(s_x[threadIdx.x], s_x[threadIdx.x + w]);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      atomicMin(a.rstat + 3 * b, (unsigned long long)__double_as_longlong(s_r[0]));
      atomicMax(a.rstat + 3 * b + 1, (unsigned long long)__double_as_longlong(s_v[0]));
      atomicMax(a.rstat + 3 * b + 2, (unsigned long long)__double_as_longlong(s_x[0]));
    }
    __syncthreads();
  }
}

// Grid-wide phases for large configurations: history sample 0, stage fields (one warp per
// receiver and source slice) and RK4 (one thread per receiver), one launch each per causal block;
// the block loop runs inside one CUDA graph (a device-side while loop).
// Grid path: the block cursor starts at the call's first step.
__global__ void lo_init_kernel(const RunArgs a, int K) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.blk[0] = a.n_begin;
    a.blk[1] = K;
  }
}

// Grid path, phase A: one warp per (receiver, source slice).  ns < 0 takes the block from the
// device cursor a.blk (graph replay); ns == 0 evaluates E_d(0).
template <bool MIXED, bool NEAR = false, bool RING = true, bool MOV = false>
__global__ void __launch_bounds__(kRunWarps * 32) lo_drive_kernel(const RunArgs a, int64_t n0, int ns) {
  __shared__ double sh[kRunWarps][32];
  if (*((volatile int *)a.status)) return;  // an earlier block failed
  if (ns < 0) {
    n0 = a.blk[0];
    if (n0 >= a.n_steps) return;
    ns = 2 * (int)min(a.blk[1], a.n_steps - n0);
  }
  const int warp = threadIdx.x >> 5;
  const int b = blockIdx.y;
  const int i = blockIdx.x * kRunWarps + warp;
  if (i >= a.N) return;
  const int z = blockIdx.z;
  const int chunk = (a.N + a.nsplit - 1) / a.nsplit;
  const int j_lo = min(a.N, z * chunk), j_hi = min(a.N, j_lo + chunk);
  double *dst = a.nsplit > 1 ? a.Epart + (size_t)z * a.B * a.N * (2 * kMaxBlock + 1) : a.Es;
  int err = 0;
  drive_phase<MIXED, NEAR, RING, true, MOV>(a, b, i, n0, ns, sh[warp], &err, j_lo, j_hi,
                                       dst + bidx(a, b, i) * (2 * kMaxBlock + 1));
  if (err) set_status(a.status, err);
}

// Sum of the slices' partial stage fields (fixed order) into Es[lo..hi].
__device__ __forceinline__ void sum_slices(const RunArgs &a, size_t bi, int lo, int hi) {
  if (a.nsplit <= 1) return;
  const size_t stride = (size_t)a.B * a.N * (2 * kMaxBlock + 1);
  const double *src = a.Epart + bi * (2 * kMaxBlock + 1);
  for (int k = lo; k <= hi; ++k) {
    double t = 0.0;
    for (int z = 0; z < a.nsplit; ++z) t += src[z * stride + k];
    a.Es[bi * (2 * kMaxBlock + 1) + k] = t;
  }
}

// E_d at the first step: slice sums (a fresh run; a resumed one has it from its state) and the first
// driving-field sample.
__global__ void lo_start_kernel(const RunArgs a) {
  const int64_t bi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (bi >= (int64_t)a.B * a.N) return;
  if (!a.state_in) sum_slices(a, bi, 0, 0);
  if (a.Ed) a.Ed[bi * (a.n_steps - a.n_begin + 1)] = a.Es[bi * (2 * kMaxBlock + 1)];
}

template <bool MIXED>
__global__ void lo_rk4_kernel(const RunArgs a, int64_t n0, int kb) {
  if (*((volatile int *)a.status)) return;
  if (kb < 0) {
    n0 = a.blk[0];
    if (n0 >= a.n_steps) return;
    kb = (int)min(a.blk[1], a.n_steps - n0);
  }
  // one warp per receiver
  const int64_t bi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (bi >= (int64_t)a.B * a.N) return;
  const int lane = threadIdx.x & 31;
  if (a.nsplit > 1 && lane < 2 * kb) sum_slices(a, bi, 1 + lane, 1 + lane);
  __syncwarp();
  int stop = 0;
  rk4_block_warp<MIXED>(a, (int)(bi / a.N), (int)(bi % a.N), n0, kb, &stop, a.Es + bi * (2 * kMaxBlock + 1));
}

// Advances the device cursor by one block and sets the loop condition of the graph.
__global__ void lo_advance_kernel(const RunArgs a, cudaGraphConditionalHandle loop) {
  const int64_t n0 = a.blk[0] + a.blk[1];
  a.blk[0] = n0;
  cudaGraphSetConditional(loop, (n0 < a.n_steps && *((volatile int *)a.status) == 0) ? 1u : 0u);
}

// ------------------------------------------------------------------------------------------------
// kinetic-energy series for the fit
// ------------------------------------------------------------------------------------------------
// Eq. dipoleE of every history sample, E = m (w0^2 d^2 + d'^2) / (2 q^2), after the run (off the
// per-block path of the time loop)
// (full store only: hs = n_steps + 1, n_begin = 0)
__global__ void energy_kernel(const RunArgs a) {
  const int64_t S = a.n_steps + 1;
  const int64_t n = (int64_t)a.B * a.N * S;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const double *T = a.rk4tab + (idx / S) * kTab;
    const double x = a.d[idx], v = a.dd[idx];
    a.energy[idx] = T[kTabC + 7] * (T[kTabC + 1] * x * x + v * v);
  }
}

// kinetic energies m d'^2 / (2 q^2) of the full store (the same expression as the per-step ones of
// rk4_block_warp, so that both stores give the fit the same series)
__global__ void ke_series_kernel(const RunArgs a, double *ke) {
  const int64_t S = a.n_steps + 1;
  const int64_t n = (int64_t)a.B * a.N * S;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const double *T = a.rk4tab + (idx / S) * kTab;
    const double v = a.dd[idx];
    ke[idx] = T[kTabC + 7] * v * v;
  }
}

// ------------------------------------------------------------------------------------------------
// Levenberg-Marquardt fit of KE = A exp(-gamma t) sin^2(omega t + phi)  (Eq. KE)
// ------------------------------------------------------------------------------------------------
constexpr int kFitThreads = 256;

template <int NV>
__device__ void block_sum(double (&v)[NV], double *sh /* [NV][kFitThreads/32] */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[k * (kFitThreads / 32) + wid] = x;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = (lane < kFitThreads / 32) ? sh[k * (kFitThreads / 32) + lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) sh[k * (kFitThreads / 32)] = x;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = sh[k * (kFitThreads / 32)];
  __syncthreads();
}

struct FitArgs {
  const double *ke;
  int K;
  int64_t S;
  double dt;
  int64_t first;
  double *gamma, *omega, *amp, *phase;
  int *status;
};

// residual/Jacobian pass.  mode 0: cost only; mode 1: cost, J^T J (10), J^T r (4).
// Each thread takes a contiguous chunk of samples; sin, cos and exp of the model are evaluated
// exactly at the chunk start and advanced by rotation and multiplication by the one-sample factors
// (float64; the chunk is ~1e2 samples, so the recurrence adds ~1e-14 relative).
__device__ void fit_pass(const double *y, int64_t n, double dt, double T, double Ag, double wg, const double x[4],
                         int mode, double out[15]) {
  for (int k = 0; k < 15; ++k) out[k] = 0.0;
  const double A = Ag * x[0], g = x[1] / T, w = wg + x[2] / T, ph = x[3];
  const int64_t chunk = (n + kFitThreads - 1) / kFitThreads;
  const int64_t i0 = (int64_t)threadIdx.x * chunk, i1 = min(n, i0 + chunk);
  if (i0 >= i1) return;
  double s, c, cw, sw;
  sincos(w * ((double)i0 * dt) + ph, &s, &c);
  sincos(w * dt, &sw, &cw);
  double env = exp(-g * ((double)i0 * dt));
  const double e1 = exp(-g * dt);
  const double iA = 1.0 / Ag, iT = 1.0 / T;
  for (int64_t i = i0; i < i1; ++i) {
    const double tau = (double)i * dt;
    const double ss = s * s;
    const double model = A * env * ss;
    const double r = (model - y[i]) * iA;
    out[0] += r * r;
    if (mode) {
      double J[4];
      J[0] = env * ss;
      J[1] = -tau * model * iT * iA;
      J[3] = 2.0 * A * env * s * c * iA;
      J[2] = J[3] * tau * iT;
      int idx = 1;
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = p; q < 4; ++q) out[idx++] += J[p] * J[q];
#pragma unroll
      for (int p = 0; p < 4; ++p) out[11 + p] += J[p] * r;
    }
    // advance the phase by w dt and the envelope by exp(-g dt)
    const double s1 = s * cw + c * sw;
    c = c * cw - s * sw;
    s = s1;
    env *= e1;
  }
}

// Full-Hessian pass in the fit's scaled parameters x (A = A_g x0, gamma = x1 / T,
// omega = omega_g + x2 / T, phi = x3; residuals r = (model - y) / A_g): out[0] = sum r^2,
// out[1..10] = H = sum (J J^T + r d2r/dx2) (upper triangle, row-major), out[11..14] = J^T r.
__device__ void fit_newton_pass(const double *y, int64_t n, double dt, double T, double Ag, double wg,
                                const double x[4], double out[15]) {
  for (int k = 0; k < 15; ++k) out[k] = 0.0;
  const double A = Ag * x[0], g = x[1] / T, w = wg + x[2] / T, ph = x[3];
  const double iA = 1.0 / Ag, iT = 1.0 / T;
  const int64_t chunk = (n + kFitThreads - 1) / kFitThreads;
  const int64_t i0 = (int64_t)threadIdx.x * chunk, i1 = min(n, i0 + chunk);
  if (i0 >= i1) return;
  double s, c, cw, sw;
  sincos(w * ((double)i0 * dt) + ph, &s, &c);
  sincos(w * dt, &sw, &cw);
  double en = exp(-g * ((double)i0 * dt));
  const double e1 = exp(-g * dt);
  for (int64_t i = i0; i < i1; ++i) {
    const double u = (double)i * dt * iT;  // tau / T
    const double ss = s * s, s2 = 2.0 * s * c, c2 = c * c - s * s;
    const double mA = A * en * iA;
    const double r = (A * en * ss - y[i]) * iA;
    double J[4], D[10];
    J[0] = en * ss;
    J[1] = -u * mA * ss;
    J[3] = mA * s2;
    J[2] = J[3] * u;
    D[0] = 0.0;
    D[1] = -u * en * ss;
    D[2] = en * s2 * u;
    D[3] = en * s2;
    D[4] = mA * ss * u * u;
    D[5] = -mA * s2 * u * u;
    D[6] = -mA * s2 * u;
    D[7] = 2.0 * mA * c2 * u * u;
    D[8] = 2.0 * mA * c2 * u;
    D[9] = 2.0 * mA * c2;
    out[0] += r * r;
    int idx = 0;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = p; q < 4; ++q, ++idx) out[1 + idx] += J[p] * J[q] + r * D[idx];
#pragma unroll
    for (int p = 0; p < 4; ++p) out[11 + p] += J[p] * r;
    const double s1 = s * cw + c * sw;
    c = c * cw - s * sw;
    s = s1;
    en *= e1;
  }
}

// Solves M z = rhs (4x4, M given as the upper triangle h[10] of a symmetric matrix) by Gaussian
// elimination with partial pivoting; returns false for a singular matrix.
__device__ bool solve4_sym(const double *h, const double *rhs_in, double *z) {
  double M[4][4], rhs[4];
  int idx = 0;
  for (int p = 0; p < 4; ++p)
    for (int q = p; q < 4; ++q, ++idx) M[p][q] = M[q][p] = h[idx];
  for (int p = 0; p < 4; ++p) rhs[p] = rhs_in[p];
  for (int cc = 0; cc < 4; ++cc) {
    int best = cc;
    for (int r = cc + 1; r < 4; ++r)
      if (fabs(M[r][cc]) > fabs(M[best][cc])) best = r;
    if (best != cc) {
      for (int q = 0; q < 4; ++q) {
        const double t = M[cc][q];
        M[cc][q] = M[best][q];
        M[best][q] = t;
      }
      const double t = rhs[cc];
      rhs[cc] = rhs[best];
      rhs[best] = t;
    }
    if (!(fabs(M[cc][cc]) > 0.0)) return false;
    for (int r = cc + 1; r < 4; ++r) {
      const double f = M[r][cc] / M[cc][cc];
      for (int q = cc; q < 4; ++q) M[r][q] -= f * M[cc][q];
      rhs[r] -= f * rhs[cc];
    }
  }
  for (int cc = 3; cc >= 0; --cc) {
    double t = rhs[cc];
    for (int q = cc + 1; q < 4; ++q) t -= M[cc][q] * z[q];
    z[cc] = t / M[cc][cc];
  }
  return true;
}

__global__ void __launch_bounds__(kFitThreads) ke_fit_kernel(const FitArgs fa) {
  __shared__ double sh[16 * (kFitThreads / 32)];
  __shared__ double s_x[4], s_xt[4], s_par[4];
  __shared__ int s_flag;
  const int k = blockIdx.x;
  const double *y = fa.ke + (size_t)k * fa.S + fa.first;
  const int64_t n = fa.S - fa.first;
  const double dt = fa.dt;
  // ---- initial guess: refined minima (zeros of sin^2) and maxima of the series ----
  double v[12];
  for (int q = 0; q < 12; ++q) v[q] = 0.0;
  // v: 0 count_min, 1 first_min_idx(min), 2 t_first, 3 last_min_idx(max), 4 t_last,
  //    5 cnt_max, 6 St, 7 Stt, 8 Sl, 9 Stl, 10 ymax, 11 t_at_ymax
  double first_idx = 1e300, last_idx = -1.0, t_first = 0.0, t_last = 0.0, ymax = -1.0, t_ymax = 0.0;
  const int64_t chunk = (n + kFitThreads - 1) / kFitThreads;
  const int64_t i0 = max((int64_t)1, (int64_t)threadIdx.x * chunk), i1 = min(n - 1, (int64_t)(threadIdx.x + 1) * chunk);
  for (int64_t i = i0; i < i1; ++i) {
    const double ym = y[i - 1], y0 = y[i], yp = y[i + 1];
    const double den = ym - 2.0 * y0 + yp;
    const double off = (den != 0.0) ? 0.5 * (ym - yp) / den : 0.0;
    const double tr = ((double)i + off) * dt;
    if (y0 <= ym && y0 < yp) {
      v[0] += 1.0;
      if ((double)i < first_idx) {
        first_idx = (double)i;
        t_first = tr;
      }
      if ((double)i > last_idx) {
        last_idx = (double)i;
        t_last = tr;
      }
    }
    if (y0 >= ym && y0 > yp) {
      const double l = log(y0);
      v[5] += 1.0;
      v[6] += tr;
      v[7] += tr * tr;
      v[8] += l;
      v[9] += tr * l;
      if (y0 > ymax) {
        ymax = y0;
        t_ymax = tr;
      }
    }
  }
  double cnt[8] = {v[0], v[5], v[6], v[7], v[8], v[9], 0.0, 0.0};
  block_sum<8>(cnt, sh);
  // min/max reductions through shared memory (first/last minimum, largest maximum)
  __shared__ double s_first[kFitThreads], s_tf[kFitThreads], s_last[kFitThreads], s_tl[kFitThreads],
      s_ym[kFitThreads], s_ty[kFitThreads];
  s_first[threadIdx.x] = first_idx;
  s_tf[threadIdx.x] = t_first;
  s_last[threadIdx.x] = last_idx;
  s_tl[threadIdx.x] = t_last;
  s_ym[threadIdx.x] = ymax;
  s_ty[threadIdx.x] = t_ymax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double fi = 1e300, tf = 0, li = -1, tl = 0, ym = -1, ty = 0;
    for (int q = 0; q < kFitThreads; ++q) {
      if (s_first[q] < fi) {
        fi = s_first[q];
        tf = s_tf[q];
      }
      if (s_last[q] > li) {
        li = s_last[q];
        tl = s_tl[q];
      }
      if (s_ym[q] > ym) {
        ym = s_ym[q];
        ty = s_ty[q];
      }
    }
    s_flag = 0;
    const double cmin = cnt[0];
    if (cmin < 2.0 || !(tl > tf)) {
      s_flag = 1;
    } else {
      const double wgs = kPi * (cmin - 1.0) / (tl - tf);
      double ph = -wgs * tf;
      ph = ph - kPi * floor(ph / kPi);
      double g = 0.0;
      const double cm = cnt[1];
      if (cm >= 2.0) {
        const double slope = (cm * cnt[5] - cnt[2] * cnt[4]) / (cm * cnt[3] - cnt[2] * cnt[2]);
        g = fmax(-slope, 0.0);
      }
      const double T = (double)(n - 1) * dt;
      s_par[0] = ym * exp(g * ty);  // A_g
      s_par[1] = wgs;               // omega_g
      s_par[2] = T;
      s_x[0] = 1.0;
      s_x[1] = g * T;
      s_x[2] = 0.0;
      s_x[3] = ph;
    }
  }
  __syncthreads();
  if (s_flag) {
    if (threadIdx.x == 0) set_status(fa.status, PC_ERR_NOCONV);
    return;
  }
  const double Ag = s_par[0], wg = s_par[1], T = s_par[2];
  double lam = 1e-3;
  double cost = 0.0;
  for (int it = 0; it < 400; ++it) {
    double x[4] = {s_x[0], s_x[1], s_x[2], s_x[3]};
    double acc[15];
    fit_pass(y, n, dt, T, Ag, wg, x, 1, acc);
    double a15[16];
    for (int q = 0; q < 15; ++q) a15[q] = acc[q];
    a15[15] = 0.0;
    block_sum<16>(a15, sh);
    cost = a15[0];
    // damped normal equations (J^T J + lam diag(J^T J)) dx = -J^T r, solved on thread 0
    bool stop = false;
    for (int tries = 0; tries < 30; ++tries) {
      if (threadIdx.x == 0) {
        double M[4][4], rhs[4];
        int idx = 1;
        for (int p = 0; p < 4; ++p)
          for (int q = p; q < 4; ++q) {
            M[p][q] = M[q][p] = a15[idx++];
          }
        for (int p = 0; p < 4; ++p) {
          M[p][p] *= (1.0 + lam);
          rhs[p] = -a15[11 + p];
        }
        // Gaussian elimination with partial pivoting
        int piv[4] = {0, 1, 2, 3};
        for (int c = 0; c < 4; ++c) {
          int best = c;
          for (int r = c + 1; r < 4; ++r)
            if (fabs(M[r][c]) > fabs(M[best][c])) best = r;
          if (best != c) {
            for (int q = 0; q < 4; ++q) {
              double tmp = M[c][q];
              M[c][q] = M[best][q];
              M[best][q] = tmp;
            }
            double tmp = rhs[c];
            rhs[c] = rhs[best];
            rhs[best] = tmp;
            int ti = piv[c];
            piv[c] = piv[best];
            piv[best] = ti;
          }
          for (int r = c + 1; r < 4; ++r) {
            double f = M[r][c] / M[c][c];
            for (int q = c; q < 4; ++q) M[r][q] -= f * M[c][q];
            rhs[r] -= f * rhs[c];
          }
        }
        double dx[4];
        for (int c = 3; c >= 0; --c) {
          double s = rhs[c];
          for (int q = c + 1; q < 4; ++q) s -= M[c][q] * dx[q];
          dx[c] = s / M[c][c];
        }
        for (int p = 0; p < 4; ++p) s_xt[p] = s_x[p] + dx[p];
        double dn = 0.0, xn = 0.0;
        for (int p = 0; p < 4; ++p) {
          dn += dx[p] * dx[p];
          xn += s_x[p] * s_x[p];
        }
        s_flag = (dn <= 1e-30 * (xn + 1e-30)) ? 2 : 0;
      }
      __syncthreads();
      double xt[4] = {s_xt[0], s_xt[1], s_xt[2], s_xt[3]};
      double c1[15];
      fit_pass(y, n, dt, T, Ag, wg, xt, 0, c1);
      double cc[1] = {c1[0]};
      block_sum<1>(cc, sh);
      const bool conv = (s_flag == 2);
      __syncthreads();
      if (cc[0] < cost && cc[0] == cc[0]) {
        if (threadIdx.x == 0)
          for (int p = 0; p < 4; ++p) s_x[p] = s_xt[p];
        lam = fmax(lam * 0.3, 1e-12);
        stop = conv || (cost - cc[0] <= 1e-15 * cost);
        __syncthreads();
        break;
      }
      lam *= 4.0;
      if (conv || lam > 1e16) {
        stop = true;
        break;
      }
    }
    __syncthreads();
    if (stop) break;
  }
  // Newton steps with the full Hessian polish the optimum where LM slows down (the decay rate is
  // weakly determined when gamma T is small): the gradient of the cost then vanishes to rounding,
  // as the implicit-function derivative of the fit assumes
  for (int it = 0; it < 2; ++it) {
    double x[4] = {s_x[0], s_x[1], s_x[2], s_x[3]};
    double hp[15];
    fit_newton_pass(y, n, dt, T, Ag, wg, x, hp);
    double h16[16];
    for (int q = 0; q < 15; ++q) h16[q] = hp[q];
    h16[15] = 0.0;
    block_sum<16>(h16, sh);
    if (threadIdx.x == 0) {
      const double rhs[4] = {-h16[11], -h16[12], -h16[13], -h16[14]};
      double dx[4];
      s_flag = solve4_sym(h16 + 1, rhs, dx) ? 0 : 1;
      for (int p = 0; p < 4; ++p) s_xt[p] = s_flag ? s_x[p] : s_x[p] + dx[p];
    }
    __syncthreads();
    double xt[4] = {s_xt[0], s_xt[1], s_xt[2], s_xt[3]};
    double c1[15];
    fit_pass(y, n, dt, T, Ag, wg, xt, 0, c1);
    double cc[1] = {c1[0]};
    block_sum<1>(cc, sh);
    if (threadIdx.x == 0 && !s_flag && cc[0] <= h16[0] * (1.0 + 1e-12) && cc[0] == cc[0])
      for (int p = 0; p < 4; ++p) s_x[p] = s_xt[p];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double A = Ag * s_x[0], g = s_x[1] / T, w = wg + s_x[2] / T, ph = s_x[3];
    if (fa.gamma) fa.gamma[k] = g;
    if (fa.omega) fa.omega[k] = w;
    if (fa.amp) fa.amp[k] = A;
    if (fa.phase) fa.phase[k] = ph;
  }
}

static pc_status launch_fit(pc_ctx *ctx, const double *ke, int K, int64_t S, double dt, int64_t first, double *gamma,
                            double *omega, double *amp, double *phase, cudaStream_t st) {
  FitArgs fa;
  fa.ke = ke;
  fa.K = K;
  fa.S = S;
  fa.dt = dt;
  fa.first = first;
  fa.gamma = gamma;
  fa.omega = omega;
  fa.amp = amp;
  fa.phase = phase;
  fa.status = ctx->d_status;
  ke_fit_kernel<<<K, kFitThreads, 0, st>>>(fa);
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

// Adjoint of the Eq. KE fit through its optimum (implicit-function theorem).  With the fit's scaled
// parameters x = (A/A_g, gamma T, (omega - omega_g) T, phi) and scaled residuals r_n = (m_n - y_n)/A_g,
// the optimum solves g(x, y) = sum_n r_n dr_n/dx = 0, so dx/dy_n = H^-1 J_n / A_g with
// H = sum_n (J_n J_n^T + r_n d2r_n/dx2) the full Hessian of the least-squares cost.  For a loss
// with cotangents (dL/dgamma, dL/domega), dL/dy_n = z . J_n / A_g with z = H^-1 (0, dL/dgamma / T,
// dL/domega / T, 0).  The kinetic energy y_n = m d'_n^2 / (2 q^2) (n >= first) then passes
// dL/dd'_n = dL/dy_n m d'_n / q^2 into the history adjoint of sample n.
struct FitAdjArgs {
  const double *ke;            // [K][S] the fitted series
  int K;
  int64_t S, first;
  double dt;
  const double *gamma, *omega, *amp, *phase;  // the optimum, physical units
  const double *dL_dgamma, *dL_domega;        // [K]
  const double *dd, *m1, *m2, *q;             // forward d' ([K][S] like ke) and the dipoles' constants
  double *seed;                               // [K][S - first] out: the cotangent of d'_n, n >= first
  int *status;
};

__global__ void __launch_bounds__(kFitThreads) ke_fit_adjoint_kernel(const FitAdjArgs fa) {
  __shared__ double sh[16 * (kFitThreads / 32)];
  __shared__ double s_z[4];
  __shared__ int s_bad;
  const int k = blockIdx.x;
  const double *y = fa.ke + (size_t)k * fa.S + fa.first;
  const int64_t n = fa.S - fa.first;
  const double dt = fa.dt, T = (double)(n - 1) * dt;
  const double A = fa.amp[k], g = fa.gamma[k], w = fa.omega[k], ph = fa.phase[k];
  // scaled about the optimum itself: A_g = A, omega_g = omega, so x = (1, gamma T, 0, phi)
  const double Ag = A, iA = 1.0 / Ag, iT = 1.0 / T;
  const double x[4] = {1.0, g * T, 0.0, ph};
  double hp[15];
  fit_newton_pass(y, n, dt, T, Ag, w, x, hp);
  double h16[16];
  for (int q = 0; q < 15; ++q) h16[q] = hp[q];
  h16[15] = 0.0;
  block_sum<16>(h16, sh);
  if (threadIdx.x == 0) {
    const double rhs[4] = {0.0, fa.dL_dgamma ? fa.dL_dgamma[k] * iT : 0.0, fa.dL_domega ? fa.dL_domega[k] * iT : 0.0,
                           0.0};
    double z[4];
    s_bad = solve4_sym(h16 + 1, rhs, z) ? 0 : 1;
    for (int p = 0; p < 4; ++p) s_z[p] = s_bad ? 0.0 : z[p];
    if (s_bad) set_status(fa.status, PC_ERR_NOCONV);
  }
  __syncthreads();
  if (s_bad) return;
  const double z0 = s_z[0], z1 = s_z[1], z2 = s_z[2], z3 = s_z[3];
  const double m = fa.m1[k] * fa.m2[k] / (fa.m1[k] + fa.m2[k]), qq = fa.q[k];
  const double kv = m / (qq * qq);
  const double *ddk = fa.dd + (size_t)k * fa.S + fa.first;
  double *sk = fa.seed + (size_t)k * (fa.S - fa.first);
  // dL/dy_n = z . J_n / A_g, into the adjoint of d'_n
  const int64_t chunk = (n + kFitThreads - 1) / kFitThreads;
  const int64_t i0 = (int64_t)threadIdx.x * chunk, i1 = min(n, i0 + chunk);
  if (i0 >= i1) return;
  double sn, cs, cw, sw;
  sincos(w * ((double)i0 * dt) + ph, &sn, &cs);
  sincos(w * dt, &sw, &cw);
  double en = exp(-g * ((double)i0 * dt));
  const double e1 = exp(-g * dt);
  for (int64_t i = i0; i < i1; ++i) {
    const double u = (double)i * dt * iT;
    const double ss = sn * sn, s2 = 2.0 * sn * cs;
    const double mA = A * en * iA;
    const double J0 = en * ss, J1 = -u * mA * ss, J3 = mA * s2, J2 = J3 * u;
    const double dy = (z0 * J0 + z1 * J1 + z2 * J2 + z3 * J3) * iA;
    sk[i] = dy * kv * ddk[i];
    const double s1 = sn * cw + cs * sw;
    cs = cs * cw - sn * sw;
    sn = s1;
    en *= e1;
  }
}

}  // namespace pc

extern "C" pc_status pc_ke_fit(pc_ctx *ctx, const double *ke, int32_t K, int64_t S, double dt, int64_t first_index,
                               double *gamma, double *omega, double *amp, double *phase, void *stream) {
  if (!ctx || !ke || K < 1 || S < 8 || !(dt > 0.0) || first_index < 0 || S - first_index < 8) return PC_ERR_ARG;
  if (!gamma || !omega) return PC_ERR_ARG;
  pc::DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  pc_status bs = pc::begin_call(ctx, st);
  if (bs != PC_OK) return bs;
  pc_status ls = pc::launch_fit(ctx, ke, K, S, dt, first_index, gamma, omega, amp, phase, st);
  if (ls != PC_OK) return ls;
  return pc::end_call(ctx, st);
}

namespace pc {
// The instantiation of the drive for a run: float64, or mixed with or without near float64 sources,
// the mixed ones specialised for a full-history store (no slot mask)
static void *drive_kernel_for(const RunArgs &a, bool mixed) {
  if (!mixed) return (void *)lo_drive_kernel<false>;
  if (a.org_pos) return (void *)lo_drive_kernel<true, false, false, true>;  // moving runs keep every sample
  const bool ring = a.wm >= 0;
  if (a.near_L > 0.f)
    return ring ? (void *)lo_drive_kernel<true, true, true> : (void *)lo_drive_kernel<true, true, false>;
  return ring ? (void *)lo_drive_kernel<true, false, true> : (void *)lo_drive_kernel<true, false, false>;
}
static void *run_kernel_for(const RunArgs &a, bool mixed) {
  if (!mixed) return (void *)lo_run_kernel<false>;
  if (a.org_pos) return (void *)lo_run_kernel<true, false, false, true>;
  const bool ring = a.wm >= 0;
  if (a.near_L > 0.f)
    return ring ? (void *)lo_run_kernel<true, true, true> : (void *)lo_run_kernel<true, true, false>;
  return ring ? (void *)lo_run_kernel<true, false, true> : (void *)lo_run_kernel<true, false, false>;
}
static cudaError_t launch_run_args(void *fn, dim3 grid, dim3 block, const RunArgs &a, cudaStream_t st,
                                   size_t smem = 0) {
  RunArgs aa = a;
  void *args[] = {&aa};
  if (smem > 0) {
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaLaunchKernel(fn, grid, block, args, smem, st);
}
static cudaError_t launch_drive(void *fn, dim3 grid, const RunArgs &a, int64_t n0, int ns, cudaStream_t st) {
  RunArgs aa = a;
  void *args[] = {&aa, &n0, &ns};
  return cudaLaunchKernel(fn, grid, dim3(kRunWarps * 32), args, 0, st);
}

// The causal-block loop of the grid path as one CUDA graph: a while node whose body is
// drive -> RK4 -> advance.  The advance kernel moves the device cursor a.blk by one block and
// clears the loop condition after the last block or after an error, so the loop ends after at
// most ceil(n_steps / K) passes.  The graph is kept in the context until its next use (every
// entry point has synchronised its stream by then) or until the context is destroyed.
static pc_status launch_block_loop(pc_ctx *ctx, const RunArgs &a, bool mixed, dim3 dgrid, unsigned rgrid,
                                   cudaStream_t st) {
  if (ctx->loop_exec) {
    cudaGraphExecDestroy(ctx->loop_exec);
    ctx->loop_exec = nullptr;
  }
  if (ctx->loop_graph) {
    cudaGraphDestroy(ctx->loop_graph);
    ctx->loop_graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return PC_ERR_CUDA;
  ctx->loop_graph = g;
  cudaGraphConditionalHandle loop;
  if (cudaGraphConditionalHandleCreate(&loop, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) return PC_ERR_CUDA;
  // zero-initialised storage: the struct's union has no default constructor
  alignas(cudaGraphNodeParams) unsigned char cp_mem[sizeof(cudaGraphNodeParams)] = {};
  cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cp_mem);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = loop;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cn;
  if (cudaGraphAddNode(&cn, g, nullptr, nullptr, 0, &cp) != cudaSuccess) return PC_ERR_CUDA;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  RunArgs args = a;
  int64_t from_cursor = -1;
  int from_cursor_i = -1;
  void *drive_args[] = {&args, &from_cursor, &from_cursor_i};
  void *rk4_args[] = {&args, &from_cursor, &from_cursor_i};
  void *adv_args[] = {&args, &loop};
  cudaKernelNodeParams kp;
  memset(&kp, 0, sizeof(kp));
  cudaGraphNode_t n1, n2, n3;
  kp.func = drive_kernel_for(a, mixed);
  kp.gridDim = dgrid;
  kp.blockDim = dim3(kRunWarps * 32);
  kp.kernelParams = drive_args;
  if (cudaGraphAddKernelNode(&n1, body, nullptr, 0, &kp) != cudaSuccess) return PC_ERR_CUDA;
  kp.func = mixed ? (void *)lo_rk4_kernel<true> : (void *)lo_rk4_kernel<false>;
  kp.gridDim = dim3((unsigned)(((size_t)a.B * a.N * 32 + 127) / 128));  // one warp per receiver
  kp.blockDim = dim3(128);
  kp.kernelParams = rk4_args;
  if (cudaGraphAddKernelNode(&n2, body, &n1, 1, &kp) != cudaSuccess) return PC_ERR_CUDA;
  kp.func = (void *)lo_advance_kernel;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(1);
  kp.kernelParams = adv_args;
  if (cudaGraphAddKernelNode(&n3, body, &n2, 1, &kp) != cudaSuccess) return PC_ERR_CUDA;
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) return PC_ERR_CUDA;
  ctx->loop_exec = ex;
  return cudaGraphLaunch(ex, st) == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

// Timed grid path: the events of nev / 3 blocks (drive start, RK4 start, RK4 end) into the context's
// sums, after the last of them has completed.
static pc_status read_block_times(pc_ctx *ctx, int nev) {
  if (nev < 3) return PC_OK;
  if (cudaEventSynchronize(ctx->tev[nev - 1]) != cudaSuccess) return PC_ERR_CUDA;
  for (int e = 0; e + 2 < nev; e += 3) {
    float d = 0.f, r = 0.f;
    if (cudaEventElapsedTime(&d, ctx->tev[e], ctx->tev[e + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&r, ctx->tev[e + 1], ctx->tev[e + 2]) != cudaSuccess)
      return PC_ERR_CUDA;
    ctx->timing.drive_ms += d;
    ctx->timing.drive_launches += 1;
    ctx->timing.rk4_ms += r;
    ctx->timing.rk4_launches += 1;
  }
  return PC_OK;
}

// Internal knobs of run_impl beyond pc_run_opts (the adjoint's and the state-size query's).
struct RunPlan {
  double *Ehalf = nullptr;                  // [B][N][n_steps] E_d at the half steps, or null
  int *k_out = nullptr;                     // the shortest causal block over the batch
  const pc_dipole_motion *motion = nullptr;
  const int2 **delay_out = nullptr;         // the pair delay table (valid until the context's next run)
  const double **rk4tab_out = nullptr;      // the per-dipole tables (idem)
  // a history store supplied by the caller of run_impl, [B][N][shs] with sample n at slot n & swm
  // (null: the caller's full outputs, or a ring of the context)
  double *sd = nullptr, *sdd = nullptr, *sddd = nullptr;
  int64_t shs = 0, swm = -1;
  // per-step kinetic energies and d' over absolute steps [ke_first, ke_first + ke_len), or null
  double *ke = nullptr, *kdd = nullptr;
  int64_t ke_first = 0, ke_len = 0;
  int64_t *reach_out = nullptr;             // the state depth D of this geometry
  bool tables_only = false;                 // stop after the tables (the state-size query)
};

static int64_t pow2_at_least(int64_t x) {
  int64_t w = 1;
  while (w < x) w <<= 1;
  return w;
}

// Forward run (Algorithm 1) over steps n_begin .. n_begin + n_steps, n_begin = 0 or the step of the
// resumed state.  The history the retarded fields read is kept in one of three stores: the caller's
// full d, d', d'' outputs (all three given, no resume), a store supplied through the plan (the
// adjoint's segment ring), or a ring of the context of W = 2^k >= D + 16 + 2 slots per dipole, D the
// deepest retarded reach of a causal block (largest origin distance / (c dt) plus the charges'
// offsets and a margin): memory O(B N D) whatever the number of steps.
static pc_status run_impl(pc_ctx *ctx, const pc_dipoles *dp, double dt, int64_t n_steps, const pc_run_opts *opts,
                          const pc_run_out *out, cudaStream_t st, const RunPlan &pl = RunPlan()) {
  if (!ctx || !dp || !opts || !out) return PC_ERR_ARG;
  if (dp->B < 1 || dp->N < 1 || !(dt > 0.0) || n_steps < 0) return PC_ERR_ARG;
  if (!dp->origin || !dp->axis || !dp->q || !dp->m1 || !dp->m2 || !dp->omega0 || !dp->d0) return PC_ERR_ARG;
  if (opts->ed_mode != 0 && opts->ed_mode != 1) return PC_ERR_ARG;
  if (opts->precision != PC_F64 && opts->precision != PC_MIXED) return PC_ERR_ARG;
  if (!(opts->near_f64 >= 0.0) || !std::isfinite(opts->near_f64)) return PC_ERR_ARG;
  if (opts->fit && (!out->gamma || !out->omega || opts->first_index < 0 || n_steps + 1 - opts->first_index < 8))
    return PC_ERR_ARG;
  const pc_dipole_motion *motion = pl.motion;
  const size_t nbn = (size_t)dp->B * dp->N;
  const bool mixed = opts->precision == PC_MIXED;
  if (motion && (!motion->pos || !motion->vel || !motion->acc)) return PC_ERR_ARG;
  if (dp->N > pc::kSmallN && dp->B > 65535) return PC_ERR_ARG;  // grid path: configurations on grid y
  // the resumed state's step (and a check of its header)
  int64_t n_begin = 0, D_in = 0;
  if (opts->state_in) {
    if (motion) return PC_ERR_ARG;  // moving origins run from t = 0 with every sample kept
    double hdr[4];
    if (cudaMemcpyAsync(hdr, opts->state_in, sizeof(hdr), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return PC_ERR_CUDA;
    if (hdr[0] != kStateMagic || hdr[3] != (double)nbn || !(hdr[1] >= 0.0) || hdr[1] != std::floor(hdr[1]) ||
        !(hdr[2] >= 1.0) || hdr[1] > 9.0e15)
      return PC_ERR_ARG;
    n_begin = (int64_t)hdr[1];
    D_in = (int64_t)hdr[2];
  }
  const int64_t So = n_steps + 1;
  const int64_t n_end = n_begin + n_steps;
  if (mixed && n_end + 1 > ((int64_t)1 << 30)) return PC_ERR_ARG;  // 32-bit sample indices
  const bool full_store = !pl.sd && !opts->state_in && out->d && out->d_dot && out->d_ddot;
  if (motion && !full_store) return PC_ERR_ARG;
  // ---- phase 1: per-run tables (pair delays and geometry, dipole records, RK4 powers, block
  // lengths, reach) in the run scratch ----
  auto al = [](size_t n) { return (n + 255) & ~(size_t)255; };
  const bool grid = dp->N > pc::kSmallN;
  const size_t es_bytes = al(nbn * (2 * pc::kMaxBlock + 1) * sizeof(double));
  const size_t f_bytes = al(nbn * pc::kDipF * sizeof(float));
  const size_t dl_bytes = al(nbn * dp->N * sizeof(int2));
  const size_t geo_bytes = mixed ? al(nbn * dp->N * sizeof(float4)) : 0;
  const size_t rs_bytes = al(3 * (size_t)dp->B * sizeof(unsigned long long));
  const size_t k_bytes = al(2 * (size_t)dp->B * sizeof(int));
  const size_t part_bytes = grid ? al((size_t)pc::kMaxSplit * es_bytes) : es_bytes;
  const size_t blk_bytes = al(2 * sizeof(int64_t));
  const size_t tab_bytes = al(nbn * pc::kTab * sizeof(double));
  const size_t f_off = es_bytes, dl_off = f_off + f_bytes, k_off = dl_off + dl_bytes;
  const size_t part_off = k_off + k_bytes, blk_off = part_off + part_bytes, tab_off = blk_off + blk_bytes;
  const size_t geo_off = tab_off + tab_bytes, rs_off = geo_off + geo_bytes;
  const size_t od_off = rs_off + rs_bytes, od_bytes = motion ? al(nbn * sizeof(double)) : 0;
  if (ctx->run_scratch.reserve(od_off + od_bytes) != cudaSuccess) return PC_ERR_CUDA;
  char *scr = (char *)ctx->run_scratch.ptr;
  pc::RunArgs a;
  memset(&a, 0, sizeof(a));
  a.B = dp->B;
  a.N = dp->N;
  a.origin = dp->origin;
  a.axis = dp->axis;
  a.q = dp->q;
  a.m1 = dp->m1;
  a.m2 = dp->m2;
  a.omega0 = dp->omega0;
  a.d0 = dp->d0;
  a.dt = dt;
  a.n_begin = n_begin;
  a.n_steps = n_end;
  a.v_max = opts->v_max > 0.0 ? opts->v_max : pc::kC / 100.0;
  a.ed_mode = opts->ed_mode;
  a.Es = (double *)scr;
  a.dipf = (float *)(scr + f_off);
  a.delay = (int2 *)(scr + dl_off);
  a.kblock = (int *)(scr + k_off);
  a.reach = a.kblock + dp->B;
  a.pgeo = mixed ? (float4 *)(scr + geo_off) : nullptr;
  a.rstat = (unsigned long long *)(scr + rs_off);
  a.Ehalf = pl.Ehalf;
  a.Epart = (double *)(scr + part_off);
  a.nsplit = 1;
  a.blk = nullptr;
  a.rk4tab = (double *)(scr + tab_off);
  a.e_unit = pc::kKe * pc::kE / ((pc::kC * dt) * (pc::kC * dt));
  a.near_L = mixed ? (float)(opts->near_f64 / (pc::kC * dt)) : 0.f;
  a.org_pos = motion ? motion->pos : nullptr;
  a.org_vel = motion ? motion->vel : nullptr;
  a.org_acc = motion ? motion->acc : nullptr;
  a.odisp = motion ? (double *)(scr + od_off) : nullptr;
  a.status = ctx->d_status;
  if (pl.delay_out) *pl.delay_out = a.delay;
  if (pl.rk4tab_out) *pl.rk4tab_out = a.rk4tab;
  {
    // pair tables and the per-configuration distance / speed extremes, then the per-dipole tables
    const int64_t NN = (int64_t)dp->N * dp->N;
    const unsigned gx = (unsigned)std::min<int64_t>((NN + 255) / 256, 2048);
    const unsigned gy = (unsigned)std::min(dp->B, 65535);
    pc::lo_rstat_init_kernel<<<(dp->B + 255) / 256, 256, 0, st>>>(a);
    if (motion) pc::lo_origin_disp_kernel<<<(unsigned)std::min<size_t>((nbn + 127) / 128, 4096), 128, 0, st>>>(a);
    pc::lo_pairs_kernel<<<dim3(gx, gy), 256, 0, st>>>(a);
    if (motion) pc::lo_closest_kernel<<<dim3(gx, gy), 256, 0, st>>>(a);
  }
  pc::lo_tables_kernel<<<dp->B, 256, 0, st>>>(a);
  // block lengths and reaches back on the host, and the status of the tables (unit axes)
  std::vector<int> kr(2 * (size_t)dp->B + 1);
  if (cudaMemcpyAsync(kr.data(), a.kblock, 2 * (size_t)dp->B * sizeof(int), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(kr.data() + 2 * (size_t)dp->B, a.status, sizeof(int), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PC_ERR_CUDA;
  if (kr[2 * (size_t)dp->B] == PC_ERR_ARG) return PC_ERR_ARG;
  int K = pc::kMaxBlock;
  int64_t D = 1;
  for (int b = 0; b < dp->B; ++b) {
    K = std::min(K, kr[b]);
    D = std::max<int64_t>(D, kr[dp->B + b]);
  }
  if (pl.k_out) *pl.k_out = K;
  if (pl.reach_out) *pl.reach_out = D;
  if (pl.tables_only) return PC_OK;
  if (opts->state_in && D_in < D) return PC_ERR_ARG;  // a state of another geometry
  // ---- phase 2: the history store, its mirror and the per-step fit inputs ----
  const int64_t W = pow2_at_least(D + pc::kMaxBlock + 2);
  int64_t hs, wm;
  if (full_store) {
    hs = So;
    wm = -1;
  } else if (pl.sd) {
    hs = pl.shs;
    wm = pl.swm;
    if (wm >= 0 && wm + 1 < W) return PC_ERR_ARG;
  } else {
    hs = W;
    wm = W - 1;
  }
  const bool own_ring = !full_store && !pl.sd;
  const size_t ring_b = own_ring ? al(nbn * (size_t)hs * sizeof(double)) : 0;
  const size_t h_bytes = mixed ? al(nbn * (size_t)hs * sizeof(float4)) : 0;
  // the fit's kinetic energies: after the run from the full store, or per step into their own rows
  const int64_t first = opts->fit ? opts->first_index : 0;
  const size_t ke_b = opts->fit ? al(nbn * (size_t)(full_store ? So : So - first) * sizeof(double)) : 0;
  // moving origins in the mixed drive: their float32 mirror (three float4 per half-step sample)
  const size_t om_b = (motion && mixed) ? al(nbn * (size_t)(2 * n_end + 1) * 3 * sizeof(float4)) : 0;
  if (ctx->run_store.reserve(3 * ring_b + h_bytes + ke_b + om_b) != cudaSuccess) return PC_ERR_CUDA;
  char *sto = (char *)ctx->run_store.ptr;
  a.hs = hs;
  a.wm = wm;
  if (full_store) {
    a.d = out->d;
    a.dd = out->d_dot;
    a.ddd = out->d_ddot;
  } else if (pl.sd) {
    a.d = pl.sd;
    a.dd = pl.sdd;
    a.ddd = pl.sddd;
  } else {
    a.d = (double *)sto;
    a.dd = (double *)(sto + ring_b);
    a.ddd = (double *)(sto + 2 * ring_b);
  }
  if (!full_store) {
    a.od = out->d;
    a.odd = out->d_dot;
    a.oddd = out->d_ddot;
  }
  a.H32 = mixed ? (float4 *)(sto + 3 * ring_b) : nullptr;
  a.energy = out->energy;
  a.energy_loop = (out->energy && !full_store) ? 1 : 0;
  a.Ed = out->Ed;
  double *ke_fit = opts->fit ? (double *)(sto + 3 * ring_b + h_bytes) : nullptr;
  a.omf = om_b ? (float4 *)(sto + 3 * ring_b + h_bytes + ke_b) : nullptr;
  if (a.omf) pc::lo_origin_mirror_kernel<<<ctx->num_sms * 4, 256, 0, st>>>(a);
  if (pl.ke) {
    a.ke = pl.ke;
    a.kdd = pl.kdd;
    a.ke_first = pl.ke_first;
    a.ke_len = pl.ke_len;
  } else if (opts->fit && !full_store) {
    a.ke = ke_fit;
    a.ke_first = n_begin + first;
    a.ke_len = So - first;
  }
  a.state_in = opts->state_in;
  a.state_out = opts->state_out;
  a.state_D = D;
  const unsigned rgrid = (unsigned)((nbn + 127) / 128);
  if (mixed) pc::lo_first_kernel<true><<<rgrid, 128, 0, st>>>(a);
  else pc::lo_first_kernel<false><<<rgrid, 128, 0, st>>>(a);
  const bool timed = ctx->run_timing != 0;
  if (dp->N <= pc::kSmallN) {
    // small configurations: one persistent CTA each, the time loop inside
    if (timed) cudaEventRecord(ctx->tev[0], st);
    // (dynamic shared memory: the configuration's RK4 tables, N x kTab doubles, 41 KB at N = 64)
    if (pc::launch_run_args(pc::run_kernel_for(a, mixed), dim3(dp->B), dim3(pc::kRunWarps * 32), a, st,
                            (size_t)dp->N * pc::kTab * sizeof(double)) != cudaSuccess)
      return PC_ERR_CUDA;
    if (timed) {
      cudaEventRecord(ctx->tev[1], st);
      float ms = 0.f;
      if (cudaEventSynchronize(ctx->tev[1]) != cudaSuccess ||
          cudaEventElapsedTime(&ms, ctx->tev[0], ctx->tev[1]) != cudaSuccess)
        return PC_ERR_CUDA;
      ctx->timing.run_ms += ms;
      ctx->timing.run_launches += 1;
    }
  } else {
    // large configurations: grid-wide phases, one drive and one RK4 launch per causal block of the
    // shortest block length over the batch; sources split so that about two resident warps per SM
    // slot are in flight
    const int64_t target = (int64_t)ctx->num_sms * 64;
    int nsplit = (int)std::min<int64_t>(std::max<int64_t>(1, (target + (int64_t)nbn - 1) / (int64_t)nbn),
                                        std::max(1, dp->N / 8));
    if (ctx->run_slices > 0) {
      nsplit = std::min(ctx->run_slices, std::max(1, dp->N / 8));  // set or tuned
    } else if (motion && mixed) {
      // the moving mixed drive holds about twice the registers of the fixed one (two CTAs per SM
      // instead of four): as many slices as fill two whole waves of its CTAs
      int occ = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pc::drive_kernel_for(a, mixed), pc::kRunWarps * 32, 0) !=
              cudaSuccess ||
          occ < 1)
        occ = 1;
      const int64_t per_slice = (int64_t)((dp->N + pc::kRunWarps - 1) / pc::kRunWarps) * dp->B;  // CTAs
      nsplit = (int)std::min<int64_t>(std::max<int64_t>(1, 2 * (int64_t)ctx->num_sms * occ / per_slice),
                                      std::max(1, dp->N / 8));
    }
    nsplit = std::min(nsplit, kMaxSplit);
    a.nsplit = nsplit;
    a.Epart = nsplit > 1 ? (double *)(scr + part_off) : nullptr;
    a.blk = (int64_t *)(scr + blk_off);
    const dim3 dgrid((unsigned)((dp->N + pc::kRunWarps - 1) / pc::kRunWarps), (unsigned)dp->B, (unsigned)nsplit);
    pc::lo_init_kernel<<<1, 32, 0, st>>>(a, K);
    void *drive = pc::drive_kernel_for(a, mixed);
    if (!opts->state_in && pc::launch_drive(drive, dgrid, a, n_begin, 0, st) != cudaSuccess) return PC_ERR_CUDA;
    pc::lo_start_kernel<<<rgrid, 128, 0, st>>>(a);
    if (n_steps > 0) {
      // the block loop runs as one graph with a device-side while node; the host-driven loop (one
      // drive and one RK4 launch per block, same kernels and order) serves where that node is not
      // available, and on request through PYCHARGE_GB300_HOST_LOOP=1 (profilers that do not
      // descend into conditional graph nodes see every launch)
      // (and always when the launches are timed, pc_set_run_timing: an event pair around each)
      const char *hl = getenv("PYCHARGE_GB300_HOST_LOOP");
      pc_status gs = (timed || (hl && hl[0] == '1')) ? PC_ERR_CUDA
                                                     : pc::launch_block_loop(ctx, a, mixed, dgrid, rgrid, st);
      if (gs != PC_OK) {
        cudaGetLastError();
        int nev = 0;
        for (int64_t n0 = n_begin; n0 < n_end; n0 += K) {
          const int kb = (int)std::min<int64_t>(K, n_end - n0);
          if (timed) cudaEventRecord(ctx->tev[nev++], st);
          pc::launch_drive(drive, dgrid, a, n0, 2 * kb, st);
          if (timed) cudaEventRecord(ctx->tev[nev++], st);
          const unsigned wgrid = (unsigned)((nbn * 32 + 127) / 128);
          if (mixed) pc::lo_rk4_kernel<true><<<wgrid, 128, 0, st>>>(a, n0, kb);
          else pc::lo_rk4_kernel<false><<<wgrid, 128, 0, st>>>(a, n0, kb);
          if (timed) {
            cudaEventRecord(ctx->tev[nev++], st);
            if (nev + 3 > 3 * 64 || n0 + K >= n_end) {
              if (pc::read_block_times(ctx, nev) != PC_OK) return PC_ERR_CUDA;
              nev = 0;
            }
          }
        }
        if (cudaGetLastError() != cudaSuccess) return PC_ERR_CUDA;
      }
    }
  }
  if (opts->state_out) pc::lo_save_kernel<<<ctx->num_sms * 4, 256, 0, st>>>(a, D);
  if (a.energy && !a.energy_loop) pc::energy_kernel<<<ctx->num_sms * 4, 256, 0, st>>>(a);
  if (opts->fit) {
    if (full_store) pc::ke_series_kernel<<<ctx->num_sms * 4, 256, 0, st>>>(a, ke_fit);
    pc_status ls = pc::launch_fit(ctx, ke_fit, (int)nbn, full_store ? So : So - first, dt,
                                  full_store ? first : 0, out->gamma, out->omega, nullptr, nullptr, st);
    if (ls != PC_OK) return ls;
  }
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}
}  // namespace pc

extern "C" pc_status pc_dipoles_run_moving(pc_ctx *ctx, const pc_dipoles *dp, const pc_dipole_motion *motion,
                                           double dt, int64_t n_steps, const pc_run_opts *opts, const pc_run_out *out,
                                           void *stream) {
  if (!ctx || !motion) return PC_ERR_ARG;
  pc::DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  pc_status bs = pc::begin_call(ctx, st);
  if (bs != PC_OK) return bs;
  pc::RunPlan pl;
  pl.motion = motion;
  pc_status rs = pc::run_impl(ctx, dp, dt, n_steps, opts, out, st, pl);
  if (rs != PC_OK) return rs;
  return pc::end_call(ctx, st);
}

extern "C" pc_status pc_dipoles_state_size(pc_ctx *ctx, const pc_dipoles *dp, double dt, int64_t *n_doubles,
                                           void *stream) {
  if (!ctx || !n_doubles) return PC_ERR_ARG;
  pc::DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  pc_status bs = pc::begin_call(ctx, st);
  if (bs != PC_OK) return bs;
  pc_run_opts o;
  memset(&o, 0, sizeof(o));
  pc_run_out none;
  memset(&none, 0, sizeof(none));
  pc::RunPlan pl;
  int64_t D = 0;
  pl.reach_out = &D;
  pl.tables_only = true;
  pc_status rs = pc::run_impl(ctx, dp, dt, 0, &o, &none, st, pl);
  if (rs != PC_OK) return rs;
  *n_doubles = pc::state_doubles((int64_t)dp->B * dp->N, D);
  return pc::end_call(ctx, st);
}

extern "C" pc_status pc_set_run_tiling(pc_ctx *ctx, int32_t source_slices) {
  if (!ctx || source_slices < 0 || source_slices > pc::kMaxSplit) return PC_ERR_ARG;
  ctx->run_slices = source_slices;
  return PC_OK;
}

extern "C" pc_status pc_set_run_timing(pc_ctx *ctx, int32_t enable) {
  if (!ctx || (enable != 0 && enable != 1)) return PC_ERR_ARG;
  pc::DeviceGuard g(ctx->device);
  if (enable && !ctx->tev[0]) {
    // all the events or none
    for (cudaEvent_t &e : ctx->tev) {
      if (cudaEventCreate(&e) != cudaSuccess) {
        e = nullptr;
        for (cudaEvent_t &f : ctx->tev) {
          if (f) cudaEventDestroy(f);
          f = nullptr;
        }
        return PC_ERR_CUDA;
      }
    }
  }
  ctx->run_timing = enable;
  if (enable) ctx->timing = pc_run_timing{};  // disabling keeps the counters readable
  return PC_OK;
}

extern "C" pc_status pc_get_run_timing(pc_ctx *ctx, pc_run_timing *out) {
  if (!ctx || !out) return PC_ERR_ARG;
  *out = ctx->timing;
  return PC_OK;
}

// Autotuning of the grid path's launch shape: each candidate number of source slices per receiver
// (powers of two up to 64 and N / 8, and the occupancy heuristic's own choice) runs the caller's
// configuration for probe_steps steps once to warm up and once timed; the fastest is kept in the
// context.  Configurations that run as one CTA each have nothing to tune.
extern "C" pc_status pc_autotune_run(pc_ctx *ctx, const pc_dipoles *dp, double dt, int64_t probe_steps,
                                     const pc_run_opts *opts, int32_t *chosen, void *stream) {
  if (!ctx || !dp || !opts || probe_steps < 1 || opts->fit || opts->state_in || opts->state_out) return PC_ERR_ARG;
  pc::DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (dp->N <= pc::kSmallN) {
    ctx->run_slices = 0;
    if (chosen) *chosen = 1;
    return PC_OK;
  }
  const int hi = std::min(pc::kMaxSplit, std::max(1, dp->N / 8));
  const int64_t nbn = (int64_t)dp->B * dp->N;
  const int heur = (int)std::min<int64_t>(
      std::min<int64_t>(std::max<int64_t>(1, ((int64_t)ctx->num_sms * 64 + nbn - 1) / nbn), hi), pc::kMaxSplit);
  std::vector<int> cand;
  for (int c = 1; c <= hi; c *= 2) cand.push_back(c);
  if (std::find(cand.begin(), cand.end(), heur) == cand.end()) cand.push_back(heur);
  if (std::find(cand.begin(), cand.end(), hi) == cand.end()) cand.push_back(hi);
  pc_run_out none;
  memset(&none, 0, sizeof(none));
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PC_ERR_CUDA;
  float best = 1e30f;
  int best_c = heur;
  pc_status rs = PC_OK;
  for (int c : cand) {
    ctx->run_slices = c;
    rs = pc_dipoles_run(ctx, dp, dt, probe_steps, opts, &none, stream);
    if (rs != PC_OK) break;
    cudaEventRecord(e0, st);
    rs = pc_dipoles_run(ctx, dp, dt, probe_steps, opts, &none, stream);
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
  ctx->run_slices = best_c;
  if (chosen) *chosen = best_c;
  return rs;
}

extern "C" pc_status pc_dipoles_run(pc_ctx *ctx, const pc_dipoles *dp, double dt, int64_t n_steps,
                                    const pc_run_opts *opts, const pc_run_out *out, void *stream) {
  if (!ctx) return PC_ERR_ARG;
  pc::DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  pc_status bs = pc::begin_call(ctx, st);
  if (bs != PC_OK) return bs;
  pc_status rs = pc::run_impl(ctx, dp, dt, n_steps, opts, out, st);
  if (rs != PC_OK) return rs;
  return pc::end_call(ctx, st);
}

// ================================================================================================
// Adjoint of the oscillator run (float64): gradients of L = sum_i w_i E_i(T) (Eq. dipoleE at the
// final step) with respect to the dipole origins, omega0 and the initial moments.
//
// The forward run keeps its whole history (it is the trajectory store the retarded fields read)
// and its half-step driving fields, so the reverse sweep recomputes nothing but the pair geometry.
// Reverse sweep over the causal blocks, last block first:
//   (1) per receiver, the reverse of its K RK4 steps: the adjoint of its state, of omega0 and of
//       the 2K stage driving fields of the block; the adjoint of each history sample (d, d', d'')
//       is complete by then, since only stages of later blocks read it;
//   (2) per source dipole (one CTA), the reverse of the retarded Lienard-Wiechert field of its two
//       charges at every receiver and stage of the block: adjoints of the source's history samples
//       (accumulated in a shared-memory window), of both origins, and of the retarded time itself
//       through the implicit-function theorem on c^2 (t - t')^2 = |r - r_s(t')|^2 (Eq. ret_t).
// ================================================================================================
namespace pc {

struct AdjArgs {
  RunArgs f;           // forward arguments; f.d/dd/ddd (store slots), f.Ed/Ehalf (steps f.n_begin ..
                       // f.n_steps) hold the forward history the reverse reads
  const double *wE;    // [B][N] dL / dE_i(T)
  double *mu;          // [B][N][f.hs][3] adjoints of the history samples (d, d', d''), sample n at
                       // slot n & f.wm; a slot is cleared once its sample's adjoint is consumed
  // the fitted rates' cotangent on d' over absolute steps [seed_first, seed_first + seed_len), or null
  const double *dseed;
  int64_t seed_first, seed_len;
  double *lam;         // [B][N][2] adjoint of the state (d, d') at the current step
  double *carry;       // [B][N] adjoint of E_d at the current block start (from its first RK4 stage)
  double *Ebar;        // [B][N][2*kMaxBlock+1] adjoints of the block's stage fields
  double *w0bar;       // [B][N]
  double *tau;         // [B][N][2] smallest and largest delay (steps) from a source to its receivers
  double *wts;         // [B][N][2] offsets of the charges per unit moment, m2/((m1+m2) q), -m1/((m1+m2) q)
  const int2 *delay;   // [B][N][N] centre delays of the forward run (first guesses of the solves)
  // moving origins (f.org_pos set): gradients of the origin samples, [B][N][2 n_steps + 1][3] each
  // (null: not wanted), and per dipole the largest origin displacement from its first sample (samples)
  double *gpos, *gvel, *gacc;
  double *disp;
  double *g_origin, *g_omega0, *g_d0;
  int64_t margin;      // samples of slack around the retarded window (charge offsets)
};

__global__ void adj_init_kernel(const AdjArgs A) {
  const RunArgs &a = A.f;
  const double L = kC * a.dt;
  for (int64_t bi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; bi < (int64_t)a.B * a.N;
       bi += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(bi / a.N), i = (int)(bi % a.N);
    const double m1 = a.m1[bi], m2 = a.m2[bi], q = a.q[bi], w0 = a.omega0[bi];
    const double m = m1 * m2 / (m1 + m2);
    const size_t sN = (size_t)bi * a.hs + (a.n_steps & a.wm);
    const double dN = a.d[sN], vN = a.dd[sN];
    const double w = A.wE ? A.wE[bi] : 0.0;
    A.wts[2 * bi] = m2 / (m1 + m2) / q;
    A.wts[2 * bi + 1] = -m1 / (m1 + m2) / q;
    double dmax = 0.0;
    if (a.org_pos) {
      const int64_t H = 2 * a.n_steps + 1;
      const double *P0 = a.org_pos + bi * H * 3;
      for (int64_t h = 1; h < H; ++h) {
        const double *Ph = P0 + 3 * h;
        const double ex = Ph[0] - P0[0], ey = Ph[1] - P0[1], ez = Ph[2] - P0[2];
        dmax = fmax(dmax, sqrt(ex * ex + ey * ey + ez * ez));
      }
    }
    A.disp[bi] = dmax / L;
    // E = m (w0^2 d^2 + d'^2) / (2 q^2)
    A.lam[2 * bi] = w * m * w0 * w0 * dN / (q * q);
    A.lam[2 * bi + 1] = w * m * vN / (q * q);
    A.w0bar[bi] = w * m * w0 * dN * dN / (q * q);
    A.carry[bi] = 0.0;
    for (int c = 0; c < 3; ++c) A.g_origin[3 * bi + c] = 0.0;
    double tmin = 1e300, tmax = 0.0;
    for (int jj = 0; jj < a.N; ++jj) {
      if (jj == i) continue;
      const size_t bj = bidx(a, b, jj);
      const double dx = a.origin[3 * bi] - a.origin[3 * bj], dy = a.origin[3 * bi + 1] - a.origin[3 * bj + 1],
                   dz = a.origin[3 * bi + 2] - a.origin[3 * bj + 2];
      const double t = sqrt(dx * dx + dy * dy + dz * dz) / L;
      tmin = fmin(tmin, t);
      tmax = fmax(tmax, t);
    }
    A.tau[2 * bi] = tmin;
    A.tau[2 * bi + 1] = tmax;
  }
}

// (1) reverse RK4 of steps n0 + kb - 1 .. n0 for one receiver; writes the stage-field adjoints of
// the block to Ebar[1 .. 2 kb] (stage s at time n0 + s/2).
__global__ void adj_rk4_kernel(const AdjArgs A, int64_t n0, int kb) {
  const RunArgs &a = A.f;
  const int64_t bi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (bi >= (int64_t)a.B * a.N) return;
  const int64_t So = a.n_steps - a.n_begin + 1;
  const size_t row = (size_t)bi * a.hs;
  const double m1 = a.m1[bi], m2 = a.m2[bi], q = a.q[bi], w0 = a.omega0[bi];
  const double m = m1 * m2 / (m1 + m2);
  const double g0 = q * q * w0 * w0 / (6.0 * kPi * kEps0 * kC * kC * kC * m);
  const double qm = q * q / m;
  const double dt = a.dt, h = 0.5 * dt;
  double l0 = A.lam[2 * bi], l1 = A.lam[2 * bi + 1];
  double carry = A.carry[bi];
  double w0b = 0.0;
  double *Eb = A.Ebar + bi * (2 * kMaxBlock + 1);
  for (int k = kb - 1; k >= 0; --k) {
    const int64_t n = n0 + k;
    // history sample n+1 = (d, d', d'') with d'' = qm E(n+1) - g0 d' - w0^2 d; its adjoint is
    // complete (only later blocks read the sample) and is consumed here, its slot cleared for reuse
    double *mu1 = A.mu + (row + ((n + 1) & a.wm)) * 3;
    const double m0 = mu1[0], m2v = mu1[2];
    double m1v = mu1[1];
    if (A.dseed && n + 1 >= A.seed_first && n + 1 < A.seed_first + A.seed_len)
      m1v += A.dseed[(size_t)bi * A.seed_len + (size_t)(n + 1 - A.seed_first)];
    mu1[0] = 0.0;
    mu1[1] = 0.0;
    mu1[2] = 0.0;
    const size_t sN = row + ((n + 1) & a.wm), s0 = row + (n & a.wm);
    const double yN0 = a.d[sN], yN1 = a.dd[sN];
    l0 += m0 - w0 * w0 * m2v;
    l1 += m1v - g0 * m2v;
    double e4b = carry + qm * m2v;
    double g0b = -yN1 * m2v, w2b = -yN0 * m2v;
    // forward stages of step n
    const double y0 = a.d[s0], y1 = a.dd[s0];
    const size_t o = (size_t)bi * So + (size_t)(n - a.n_begin);
    const double e1 = a.Ed[o], e2 = a.Ehalf[(size_t)bi * (So - 1) + (size_t)(n - a.n_begin)], e4 = a.Ed[o + 1];
    const double k1a = y1, k1b = -g0 * y1 - w0 * w0 * y0 + qm * e1;
    const double y0b = y0 + h * k1a, y1b = y1 + h * k1b;
    const double k2a = y1b, k2b = -g0 * y1b - w0 * w0 * y0b + qm * e2;
    const double y0c = y0 + h * k2a, y1c = y1 + h * k2b;
    const double k3a = y1c, k3b = -g0 * y1c - w0 * w0 * y0c + qm * e2;
    const double y0d = y0 + dt * k3a, y1d = y1 + dt * k3b;
    (void)e4;
    // reverse of y_{n+1} = y_n + dt/6 (k1 + 2 k2 + 2 k3 + k4)
    double y0bar = l0, y1bar = l1;
    double k1ab = dt / 6.0 * l0, k2ab = dt / 3.0 * l0, k3ab = dt / 3.0 * l0, k4ab = dt / 6.0 * l0;
    double k1bb = dt / 6.0 * l1, k2bb = dt / 3.0 * l1, k3bb = dt / 3.0 * l1, k4bb = dt / 6.0 * l1;
    double e2b = 0.0, e1b = 0.0;
    // k4 = f(y_d, e4)
    double y1db = k4ab - g0 * k4bb, y0db = -w0 * w0 * k4bb;
    e4b += qm * k4bb;
    g0b += -y1d * k4bb;
    w2b += -y0d * k4bb;
    y0bar += y0db;
    k3ab += dt * y0db;
    y1bar += y1db;
    k3bb += dt * y1db;
    // k3 = f(y_c, e2)
    double y1cb = k3ab - g0 * k3bb, y0cb = -w0 * w0 * k3bb;
    e2b += qm * k3bb;
    g0b += -y1c * k3bb;
    w2b += -y0c * k3bb;
    y0bar += y0cb;
    k2ab += h * y0cb;
    y1bar += y1cb;
    k2bb += h * y1cb;
    // k2 = f(y_b, e2)
    double y1bb = k2ab - g0 * k2bb, y0bb = -w0 * w0 * k2bb;
    e2b += qm * k2bb;
    g0b += -y1b * k2bb;
    w2b += -y0b * k2bb;
    y0bar += y0bb;
    k1ab += h * y0bb;
    y1bar += y1bb;
    k1bb += h * y1bb;
    // k1 = f(y_n, e1)
    y1bar += k1ab - g0 * k1bb;
    y0bar += -w0 * w0 * k1bb;
    e1b += qm * k1bb;
    g0b += -y1 * k1bb;
    w2b += -y0 * k1bb;
    // g0 = q^2 w0^2 / (6 pi eps0 c^3 m), w2 = w0^2
    w0b += g0b * 2.0 * g0 / w0 + w2b * 2.0 * w0;
    Eb[2 * k + 2] = e4b;
    Eb[2 * k + 1] = e2b;
    carry = e1b;
    l0 = y0bar;
    l1 = y1bar;
  }
  A.lam[2 * bi] = l0;
  A.lam[2 * bi + 1] = l1;
  A.carry[bi] = carry;
  A.w0bar[bi] += w0b;
}

// Reverse of the driving-field contribution F = p_i . E of dipole j's two charges at receiver i
// and time u (steps, history 0..nv).  eb = dL/dF.  Adds to the history adjoints of j (window
// win[0..W) for samples wlo..), to the receiver's and the source's origin adjoints.
template <bool MOV>
__device__ int pair_rev_f64(const AdjArgs &A, int b, int i, int j, double u, int64_t nv, double eb, double *win,
                            int64_t wlo, int W, double Rib[3], double Rjb[3]) {
  const RunArgs &a = A.f;
  const double cdt = kC * a.dt;
  const size_t bi = bidx(a, b, i), bj = bidx(a, b, j);
  const double *Ri = a.origin + 3 * bi;
  const double *pi = a.axis + 3 * bi;
  TrajF64 tr;
  tr.dipole = true;
  tr.d = a.d + bj * a.hs;
  tr.dd = a.dd + bj * a.hs;
  tr.ddd = a.ddd + bj * a.hs;
  tr.wm = a.wm;
  double pj[3];
  for (int c = 0; c < 3; ++c) {
    tr.R[c] = a.origin[3 * bj + c];
    tr.ax[c] = a.axis[3 * bj + c];
    pj[c] = tr.ax[c];
  }
  const double q = a.q[bj];
  // moving origins: the receiver at its origin of the stage time (half-step index 2u), the source
  // charges on the interpolated origin history; their adjoints go to the origin samples
  constexpr bool mov = MOV;  // moving origins (a.org_pos set, every sample kept): a separate instantiation
  const int64_t H = 2 * a.n_steps + 1;
  const int64_t hh = mov ? (int64_t)llrint(2.0 * u) : 0;
  int64_t kg;
  if (mov) {
    Ri = a.org_pos + (bi * H + hh) * 3;
    tr.Rp = a.org_pos + bj * H * 3;
    tr.Rv = a.org_vel + bj * H * 3;
    tr.Ra = a.org_acc + bj * H * 3;
    for (int c = 0; c < 3; ++c) tr.R[c] = tr.Rp[6 * nv + c];  // the source now, for the first guess
    const double dv[3] = {Ri[0] - tr.R[0], Ri[1] - tr.R[1], Ri[2] - tr.R[2]};
    kg = (int64_t)floor(u - sqrt(dot3(dv, dv)) / cdt);
  } else {
    // first guess: the sample of the centre's retarded time, u - delay (u - nv is a half-integer)
    const int2 dl = A.delay[bi * a.N + j];
    kg = nv - dl.x + Num<float>::floor_int((float)(u - (double)nv) - __int_as_float(dl.y));
  }
  const double Eb[3] = {eb * pi[0], eb * pi[1], eb * pi[2]};
  // fixed origins: the pair's scalars (rho = R_i - R_j; |p_j| = 1) for the scalar form below
  double rho[3] = {0.0, 0.0, 0.0}, rr = 0.0, ra = 0.0, rp = 0.0, apj = 0.0;
  if (!mov) {
    for (int c = 0; c < 3; ++c) rho[c] = Ri[c] - tr.R[c];
    rr = dot3(rho, rho);
    ra = dot3(rho, pj);
    rp = dot3(rho, pi);
    apj = dot3(pj, pi);
  }
  for (int sg = 0; sg < 2; ++sg) {
    const double w = A.wts[2 * bj + sg];
    tr.w = w;
    const double qc = sg == 0 ? q : -q;
    if (!mov && nv > 0 && kg >= 0) {
      // scalar form (the reverse of pair_drive_f64_scalar): F = p_i . E depends on the charge only
      // through R = |a|, a.p_j, a.p_i (a = rho - s p_j) and s', s''; the adjoint of a is assembled
      // from theirs, the history adjoints take those of s, s', s'' and of the retarded time
      int64_t k;
      double th, s0, ds;
      if (scalar_root(tr.d, a.wm, w, rr, ra, u, cdt * cdt, nv, kg, &k, &th, &s0, &ds)) {
        const int64_t k0 = k & a.wm, k1 = (k + 1) & a.wm;
        const double Dd = tr.d[k1] - tr.d[k0], Dv = tr.dd[k1] - tr.dd[k0], Da = tr.ddd[k1] - tr.ddd[k0];
        const double sv0 = w * tr.dd[k0], sa0 = w * tr.ddd[k0];
        const double sp = s0 + th * ds;
        const double sv = sv0 + th * (w * tr.dd[k1] - sv0);
        const double sa = sa0 + th * (w * tr.ddd[k1] - sa0);
        const double c = kC;
        const double aj = ra - sp, ai = rp - sp * apj;
        const double R2 = rr - sp * (2.0 * ra - sp);
        const double iR = rsqrt(R2), R = R2 * iR;
        const double Ru = c * R - sv * aj;
        const double iRu = 1.0 / Ru;
        const double f = kKe * qc * R * iRu * iRu * iRu;
        const double pu = c * ai * iR - sv * apj;
        const double Wf = c * c - sv * sv + sa * aj;
        // reverse of F = f (Wf pu - Ru sa p_i.p_j)
        const double fb = eb * (Wf * pu - Ru * sa * apj);
        const double Wb = eb * f * pu, pub = eb * f * Wf;
        double Rub = -eb * f * sa * apj;
        const double sab = -eb * f * Ru * apj + aj * Wb;
        double svb = -2.0 * sv * Wb - pub * apj;
        double ajb = sa * Wb;
        const double aib = pub * c * iR;
        double Rb = -pub * c * ai * iR * iR + fb * f * iR;
        Rub += -3.0 * fb * f * iRu;
        Rb += c * Rub;
        svb += -Rub * aj;
        ajb += -Rub * sv;
        double av[3];
        for (int cc = 0; cc < 3; ++cc) {
          av[cc] = rho[cc] - sp * pj[cc];
          const double abc = Rb * iR * av[cc] + ajb * pj[cc] + aib * pi[cc];
          Rib[cc] += abc;
          Rjb[cc] -= abc;
        }
        const double pb_p = -(Rb * iR * aj + ajb + aib * apj);  // -ab . p_j
        if (k < wlo || k + 1 >= wlo + W) return PC_ERR_NOCONV;
        const double Db = w * pb_p, Vb = w * svb, Ab = w * sab;
        const double thb = Db * Dd + Vb * Dv + Ab * Da;
        const double Gth = -2.0 * cdt * cdt * (u - (double)k - th) + 2.0 * w * Dd * aj;
        const double sfac = -thb / Gth;
        for (int cc = 0; cc < 3; ++cc) {
          Rib[cc] += sfac * (-2.0 * av[cc]);
          Rjb[cc] += sfac * (2.0 * av[cc]);
        }
        const double dbar = Db + sfac * 2.0 * aj * w;
        double *w0p = win + 3 * (k - wlo), *w1p = w0p + 3;
        atomicAdd(&w0p[0], (1.0 - th) * dbar);
        atomicAdd(&w0p[1], (1.0 - th) * Vb);
        atomicAdd(&w0p[2], (1.0 - th) * Ab);
        atomicAdd(&w1p[0], th * dbar);
        atomicAdd(&w1p[1], th * Vb);
        atomicAdd(&w1p[2], th * Ab);
        continue;
      }
    }
    int64_t k = -1;
    double th = 0.0;
    bool stat = true;
    if (nv > 0) {
      const int e = solve_f64(tr, nv + 1, 1, Ri, u, cdt, kg, &k, &th);
      if (e) return e;
      stat = (k < 0 || (k == 0 && th == 0.0));
    }
    double p[3], vel[3] = {0, 0, 0}, acc[3] = {0, 0, 0};
    double Dd = 0, Dv = 0, Da = 0;
    if (stat) {
      tr.p(0, p);
    } else {
      double p1[3], v1[3], a1[3];
      tr.p(k, p);
      tr.p(k + 1, p1);
      tr.va(k, vel, acc);
      tr.va(k + 1, v1, a1);
      Dd = tr.dk(k + 1) - tr.dk(k);
      Dv = tr.ddk(k + 1) - tr.ddk(k);
      Da = tr.dddk(k + 1) - tr.dddk(k);
      for (int c = 0; c < 3; ++c) {
        p[c] += th * (p1[c] - p[c]);
        vel[c] += th * (v1[c] - vel[c]);
        acc[c] += th * (a1[c] - acc[c]);
      }
    }
    const double av[3] = {Ri[0] - p[0], Ri[1] - p[1], Ri[2] - p[2]};
    double ab[3] = {0, 0, 0}, vb[3] = {0, 0, 0}, accb[3] = {0, 0, 0};
    lw_E_f64_rev(qc, av, vel, acc, Eb, ab, vb, accb);
    // a = r - p: receiver origin gets ab, the source position gets -ab
    double *gr = mov && A.gpos ? A.gpos + (bi * H + hh) * 3 : nullptr;  // receiver's origin sample
    for (int c = 0; c < 3; ++c) {
      if (mov) {
        if (gr) atomicAdd(gr + c, ab[c]);
      } else {
        Rib[c] += ab[c];
        Rjb[c] -= ab[c];
      }
    }
    const double pb_p = -dot3(ab, pj);  // adjoint of the charge offset along the axis
    if (stat) {
      // position R_j + w d[0] p_j: only d[0] (window slot of sample 0) and the first origin sample
      if (wlo != 0) return PC_ERR_NOCONV;
      atomicAdd(&win[0], w * pb_p);
      if (mov && A.gpos)
        for (int c = 0; c < 3; ++c) atomicAdd(A.gpos + bj * H * 3 + c, -ab[c]);
      continue;
    }
    if (k < wlo || k + 1 >= wlo + W) return PC_ERR_NOCONV;
    const double Db = w * pb_p, Vb = w * dot3(vb, pj), Ab = w * dot3(accb, pj);
    double *w0p = win + 3 * (k - wlo), *w1p = w0p + 3;
    // the fraction th depends on the inputs through G(th) = cdt^2 (u - k - th)^2 - |r - p(th)|^2 = 0
    double thb = Db * Dd + Vb * Dv + Ab * Da;
    const double ap = dot3(av, pj);
    double Gth = -2.0 * cdt * cdt * (u - (double)k - th) + 2.0 * w * Dd * ap;
    double dRp[3] = {0, 0, 0};
    if (mov) {
      // the origin's interpolated position, velocity and acceleration move with th too
      const double *P0 = tr.Rp + 6 * k, *V0 = tr.Rv + 6 * k, *A0 = tr.Ra + 6 * k;
      for (int c = 0; c < 3; ++c) {
        dRp[c] = P0[6 + c] - P0[c];
        thb += -ab[c] * dRp[c] + vb[c] * (V0[6 + c] - V0[c]) + accb[c] * (A0[6 + c] - A0[c]);
      }
      Gth += 2.0 * dot3(av, dRp);
    }
    const double sfac = -thb / Gth;
    if (mov) {
      // origin samples 2k and 2k + 2 carry the source's position (with the retarded-time term),
      // velocity and acceleration adjoints with weights 1 - th and th; the receiver's sample the
      // retarded-time term of r
      const size_t o0 = (bj * H + 2 * k) * 3, o1 = o0 + 6;
      for (int c = 0; c < 3; ++c) {
        const double pbv = -ab[c] + sfac * 2.0 * av[c];
        if (A.gpos) {
          atomicAdd(A.gpos + o0 + c, (1.0 - th) * pbv);
          atomicAdd(A.gpos + o1 + c, th * pbv);
          atomicAdd(gr + c, sfac * (-2.0 * av[c]));
        }
        if (A.gvel) {
          atomicAdd(A.gvel + o0 + c, (1.0 - th) * vb[c]);
          atomicAdd(A.gvel + o1 + c, th * vb[c]);
        }
        if (A.gacc) {
          atomicAdd(A.gacc + o0 + c, (1.0 - th) * accb[c]);
          atomicAdd(A.gacc + o1 + c, th * accb[c]);
        }
      }
    } else {
      for (int c = 0; c < 3; ++c) {
        Rib[c] += sfac * (-2.0 * av[c]);
        Rjb[c] += sfac * (2.0 * av[c]);
      }
    }
    const double dbar = Db + sfac * 2.0 * ap * w;
    atomicAdd(&w0p[0], (1.0 - th) * dbar);
    atomicAdd(&w0p[1], (1.0 - th) * Vb);
    atomicAdd(&w0p[2], (1.0 - th) * Ab);
    atomicAdd(&w1p[0], th * dbar);
    atomicAdd(&w1p[1], th * Vb);
    atomicAdd(&w1p[2], th * Ab);
  }
  return 0;
}

// (2) one CTA per (source j, configuration b): reverse of the block's stage fields at every
// receiver.  ns == 0 handles the field at t = 0 with the adjoint left in `carry`.  The source
// samples the block's retarded times reach lie in [n0 + 1/2 - tau_max - margin,
// n0 + ns/2 - tau_min + margin]; their adjoints are gathered in a shared-memory window.
template <bool MOV>
__global__ void __launch_bounds__(128, 4) adj_field_kernel(const AdjArgs A, int64_t n0, int ns, int wmax) {
  extern __shared__ double win[];  // [wmax][3]
  __shared__ double s_rj[3][128];
  const RunArgs &a = A.f;
  const int j = blockIdx.x, b = blockIdx.y;
  const size_t bj = bidx(a, b, j);
  int64_t wlo = 0, whi = 0;
  if (ns > 0) {
    const double lo = (double)n0 + 0.5 - A.tau[2 * bj + 1] - (double)A.margin;
    const double hi = (double)n0 + 0.5 * ns - A.tau[2 * bj] + (double)A.margin + 1.0;
    wlo = (int64_t)fmax(0.0, floor(lo));
    whi = (int64_t)fmin((double)n0, ceil(hi));
    if (whi < wlo) whi = wlo;
  }
  const int W = (int)(whi - wlo + 1);
  if (W > wmax) {
    if (threadIdx.x == 0) set_status(a.status, PC_ERR_NOCONV);
    return;
  }
  for (int t = threadIdx.x; t < 3 * W; t += blockDim.x) win[t] = 0.0;
  __syncthreads();
  double Rjb[3] = {0, 0, 0};
  int err = 0;
  const int nst = ns > 0 ? ns : 1;
  if (a.N >= (int)blockDim.x) {
    // many receivers: one thread per receiver, its stages in order, its origin adjoint in registers
    for (int i = threadIdx.x; i < a.N && !err; i += blockDim.x) {
      if (i == j) continue;
      const size_t bi = bidx(a, b, i);
      double Rib[3] = {0, 0, 0};
      for (int s = 1; s <= nst && !err; ++s) {
        const double eb = ns > 0 ? A.Ebar[bi * (2 * kMaxBlock + 1) + s] : A.carry[bi];
        if (eb == 0.0) continue;
        const double u = ns > 0 ? (double)n0 + 0.5 * s : 0.0;
        err = pair_rev_f64<MOV>(A, b, i, j, u, n0, eb, win, wlo, W, Rib, Rjb);
      }
      for (int c = 0; c < 3; ++c)
        if (Rib[c] != 0.0) atomicAdd(&A.g_origin[3 * bi + c], Rib[c]);
    }
  } else {
    // few receivers: each warp takes 32 / nst receivers at a time, one lane per (receiver, stage),
    // and a receiver's origin adjoint is summed over its stages in shared memory (fixed order)
    // before one atomic per component
    __shared__ double s_rib[4][32][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int slots = 32 / nst;
    const int m = lane / nst, s = 1 + lane % nst;
    for (int i0 = 0; i0 < a.N; i0 += 4 * slots) {
      const int i = i0 + warp * slots + m;
      double Rib[3] = {0, 0, 0};
      if (m < slots && i < a.N && i != j && !err) {
        const size_t bi = bidx(a, b, i);
        const double eb = ns > 0 ? A.Ebar[bi * (2 * kMaxBlock + 1) + s] : A.carry[bi];
        if (eb != 0.0) {
          const double u = ns > 0 ? (double)n0 + 0.5 * s : 0.0;
          err = pair_rev_f64<MOV>(A, b, i, j, u, n0, eb, win, wlo, W, Rib, Rjb);
        }
      }
      for (int c = 0; c < 3; ++c) s_rib[warp][lane][c] = Rib[c];
      __syncwarp();
      if (m < slots && s == 1 && i < a.N) {
        for (int c = 0; c < 3; ++c) {
          double t = 0.0;
          for (int q = 0; q < nst; ++q) t += s_rib[warp][lane + q][c];
          if (t != 0.0) atomicAdd(&A.g_origin[3 * bidx(a, b, i) + c], t);
        }
      }
      __syncwarp();
    }
  }
  if (err) set_status(a.status, err);
  for (int c = 0; c < 3; ++c) s_rj[c][threadIdx.x] = Rjb[c];
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int k = 0; k < (int)blockDim.x; ++k) t += s_rj[threadIdx.x][k];
    atomicAdd(&A.g_origin[3 * bj + threadIdx.x], t);
  }
  // the window into the source's history adjoints (this CTA owns source j during the launch)
  for (int t = threadIdx.x; t < 3 * W; t += blockDim.x)
    A.mu[(bj * a.hs + ((wlo + t / 3) & a.wm)) * 3 + t % 3] += win[t];
}

// Field-loss seed of the adjoint: L = sum over configurations b, frames f and points p of
// <cE, E> + <cB, B> + cphi phi + <cA, A> of the configuration's dipoles at the points (Sec. 2.2,
// Eqs. E, B, V, A on the run's own history).  One CTA per (source dipole, frame, configuration)
// reverses the field of the source's two charges at every point: the adjoints of its history
// samples collect in a shared-memory window spanning the points' retarded times (then added to
// the global history adjoints by atomics, several frames hitting the same samples), the adjoint of
// its origin by a block sum, and the retarded time is differentiated through its defining equation.
struct FieldSeed {
  const double *pts;   // [P][3]
  int64_t P;
  int32_t T;
  const double *times;  // device [T]
  const double *cE, *cB, *cphi, *cA;  // [B][T][P][3] / [B][T][P], any may be null
};

__device__ int field_rev_charge(const AdjArgs &A, const TrajF64 &tr, double qc, const double r[3], double u,
                                int64_t kg, const double *cE, const double *cB, double cphi, const double *cA,
                                double *win, int64_t wlo, int W, double Rjb[3]) {
  const RunArgs &a = A.f;
  const int64_t S = a.n_steps + 1;
  const double cdt = kC * a.dt;
  int64_t k = -1;
  double th = 0.0;
  const int e = solve_f64(tr, S, 1, r, u, cdt, kg, &k, &th);
  if (e) return e;
  const bool stat = k < 0;
  double p[3], vel[3] = {0, 0, 0}, acc[3] = {0, 0, 0};
  double Dd = 0, Dv = 0, Da = 0;
  if (stat) {
    tr.p(0, p);
  } else {
    double p1[3], v1[3], a1[3];
    tr.p(k, p);
    tr.p(k + 1, p1);
    tr.va(k, vel, acc);
    tr.va(k + 1, v1, a1);
    Dd = tr.dk(k + 1) - tr.dk(k);
    Dv = tr.ddk(k + 1) - tr.ddk(k);
    Da = tr.dddk(k + 1) - tr.dddk(k);
    for (int c = 0; c < 3; ++c) {
      p[c] += th * (p1[c] - p[c]);
      vel[c] += th * (v1[c] - vel[c]);
      acc[c] += th * (a1[c] - acc[c]);
    }
  }
  const double av[3] = {r[0] - p[0], r[1] - p[1], r[2] - p[2]};
  double ab[3] = {0, 0, 0}, vb[3] = {0, 0, 0}, accb[3] = {0, 0, 0};
  lw_full_f64_rev(qc, av, vel, acc, cE, cB, cphi, cA, ab, vb, accb);
  for (int c = 0; c < 3; ++c) Rjb[c] -= ab[c];  // a = r - p, p = R_j + w d axis
  const double w = tr.w;
  const double pb_p = -dot3(ab, tr.ax);
  if (stat) {
    if (wlo != 0) return PC_ERR_NOCONV;
    atomicAdd(&win[0], w * pb_p);
    return 0;
  }
  if (k < wlo || k + 1 >= wlo + W) return PC_ERR_NOCONV;
  const double Db = w * pb_p, Vb = w * dot3(vb, tr.ax), Ab = w * dot3(accb, tr.ax);
  const double thb = Db * Dd + Vb * Dv + Ab * Da;
  const double ap = dot3(av, tr.ax);
  const double Gth = -2.0 * cdt * cdt * (u - (double)k - th) + 2.0 * w * Dd * ap;
  const double sfac = -thb / Gth;
  for (int c = 0; c < 3; ++c) Rjb[c] += sfac * 2.0 * av[c];
  const double dbar = Db + sfac * 2.0 * ap * w;
  double *w0p = win + 3 * (k - wlo), *w1p = w0p + 3;
  atomicAdd(&w0p[0], (1.0 - th) * dbar);
  atomicAdd(&w0p[1], (1.0 - th) * Vb);
  atomicAdd(&w0p[2], (1.0 - th) * Ab);
  atomicAdd(&w1p[0], th * dbar);
  atomicAdd(&w1p[1], th * Vb);
  atomicAdd(&w1p[2], th * Ab);
  return 0;
}

__global__ void __launch_bounds__(128) fields_adj_kernel(const AdjArgs A, const FieldSeed F, int wmax) {
  extern __shared__ double win[];  // [wmax][3]
  __shared__ double s_red[3][128];
  __shared__ double s_lo[128], s_hi[128];
  const RunArgs &a = A.f;
  const int j = blockIdx.x, f = blockIdx.y, b = blockIdx.z;
  const size_t bj = bidx(a, b, j);
  const int64_t S = a.n_steps + 1;
  const double L = kC * a.dt;
  const double t = F.times[f];
  const double u = t / a.dt;
  TrajF64 tr;
  tr.dipole = true;
  tr.d = a.d + bj * a.hs;  // (the field-loss seed runs on the full store: hs = S, wm = -1)
  tr.dd = a.dd + bj * a.hs;
  tr.ddd = a.ddd + bj * a.hs;
  tr.wm = a.wm;
  for (int c = 0; c < 3; ++c) {
    tr.R[c] = a.origin[3 * bj + c];
    tr.ax[c] = a.axis[3 * bj + c];
  }
  // retarded-sample window of the points
  double lo = 1e300, hi = -1e300;
  for (int64_t p = threadIdx.x; p < F.P; p += blockDim.x) {
    const double dx = F.pts[3 * p] - tr.R[0], dy = F.pts[3 * p + 1] - tr.R[1], dz = F.pts[3 * p + 2] - tr.R[2];
    const double dist = sqrt(dx * dx + dy * dy + dz * dz) / L;
    lo = fmin(lo, dist);
    hi = fmax(hi, dist);
  }
  s_lo[threadIdx.x] = lo;
  s_hi[threadIdx.x] = hi;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)blockDim.x; ++q) {
      lo = fmin(lo, s_lo[q]);
      hi = fmax(hi, s_hi[q]);
    }
    s_lo[0] = lo;
    s_hi[0] = hi;
  }
  __syncthreads();
  const int64_t wlo = (int64_t)fmax(0.0, floor(u - s_hi[0] - (double)A.margin));
  int64_t whi = (int64_t)fmin((double)(S - 1), ceil(u - s_lo[0] + (double)A.margin) + 1.0);
  if (whi < wlo) whi = wlo;
  const int W = (int)(whi - wlo + 1);
  if (W > wmax) {
    if (threadIdx.x == 0) set_status(a.status, PC_ERR_NOCONV);
    return;
  }
  for (int q = threadIdx.x; q < 3 * W; q += blockDim.x) win[q] = 0.0;
  __syncthreads();
  const double q = a.q[bj], m1 = a.m1[bj], m2 = a.m2[bj];
  double Rjb[3] = {0, 0, 0};
  int err = 0;
  const size_t base = ((size_t)b * F.T + f) * (size_t)F.P;
  for (int64_t p = threadIdx.x; p < F.P && !err; p += blockDim.x) {
    const double r[3] = {F.pts[3 * p], F.pts[3 * p + 1], F.pts[3 * p + 2]};
    const double *cE = F.cE ? F.cE + 3 * (base + p) : nullptr;
    const double *cB = F.cB ? F.cB + 3 * (base + p) : nullptr;
    const double *cA = F.cA ? F.cA + 3 * (base + p) : nullptr;
    const double cphi = F.cphi ? F.cphi[base + p] : 0.0;
    const double dv[3] = {r[0] - tr.R[0], r[1] - tr.R[1], r[2] - tr.R[2]};
    const int64_t kg = (int64_t)floor(u - sqrt(dot3(dv, dv)) / L);
    for (int sg = 0; sg < 2 && !err; ++sg) {
      tr.w = (sg == 0) ? m2 / (m1 + m2) / q : -m1 / (m1 + m2) / q;
      err = field_rev_charge(A, tr, sg == 0 ? q : -q, r, u, kg, cE, cB, cphi, cA, win, wlo, W, Rjb);
    }
  }
  if (err) set_status(a.status, err);
  for (int c = 0; c < 3; ++c) s_red[c][threadIdx.x] = Rjb[c];
  __syncthreads();
  if (threadIdx.x < 3) {
    double tt = 0.0;
    for (int q2 = 0; q2 < (int)blockDim.x; ++q2) tt += s_red[threadIdx.x][q2];
    atomicAdd(&A.g_origin[3 * bj + threadIdx.x], tt);
  }
  for (int q2 = threadIdx.x; q2 < 3 * W; q2 += blockDim.x)
    if (win[q2] != 0.0) atomicAdd(&A.mu[(bj * a.hs + wlo) * 3 + q2], win[q2]);
}

__global__ void adj_final_kernel(const AdjArgs A) {
  const RunArgs &a = A.f;
  for (int64_t bi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; bi < (int64_t)a.B * a.N;
       bi += (int64_t)gridDim.x * blockDim.x) {
    // y_0 = (d0, 0) and the history before and at t = 0 sits at d0
    A.g_d0[bi] = A.lam[2 * bi] + A.mu[((size_t)bi * a.hs + (0 & a.wm)) * 3];
    A.g_omega0[bi] = A.w0bar[bi];
  }
}

}  // namespace pc

namespace pc {
// Reverse mode of the float64 run for L = sum w E(T) (wE, or null) plus, when rates is set,
// sum (dL/dgamma gamma + dL/domega omega) of the Eq. KE fit from first_index on.
static pc_status adjoint_core(pc_ctx *ctx, const pc_dipoles *dp, double dt, int64_t n_steps, const pc_run_opts *opts,
                              const double *wE, bool rates, const double *dL_dgamma, const double *dL_domega,
                              double *gamma_out, double *omega_out, const pc_dipole_grads *g, cudaStream_t st,
                              const FieldSeed *fseed = nullptr, const pc_dipole_motion *motion = nullptr,
                              const pc_dipole_motion_grads *gm = nullptr) {
  if (!dp || !opts || !g || !g->origin || !g->omega0 || !g->d0) return PC_ERR_ARG;
  // moving origins: the energy loss (the forward in either precision, as below)
  if (motion && (rates || fseed || !motion->pos || !motion->vel || !motion->acc)) return PC_ERR_ARG;
  // the forward may run its driving field in either precision (the reverse is float64 throughout);
  // the fitted rates' adjoint keeps the float64 forward
  if (opts->ed_mode != 0 || n_steps < 1) return PC_ERR_ARG;
  if (opts->precision != PC_F64 && (rates || opts->precision != PC_MIXED)) return PC_ERR_ARG;
  if (dp->B < 1 || dp->N < 1 || !(dt > 0.0)) return PC_ERR_ARG;
  if (rates && (opts->first_index < 0 || n_steps + 1 - opts->first_index < 8)) return PC_ERR_ARG;
  if (opts->state_in || opts->state_out || opts->checkpoint_every < 0) return PC_ERR_ARG;
  // checkpointing: the energy and rate losses of fixed origins (a field loss or moving origins read
  // the whole history)
  const int64_t Cask = opts->checkpoint_every;
  if (Cask > 0 && (fseed || motion)) return PC_ERR_ARG;
  const int64_t S = n_steps + 1;
  const size_t nbn = (size_t)dp->B * dp->N;
  auto al = [](size_t n) { return (n + 255) & ~(size_t)255; };
  pc_run_opts fo = *opts;
  fo.fit = 0;
  fo.checkpoint_every = 0;
  const int64_t first = rates ? opts->first_index : 0;
  const int64_t flen = S - first;  // the fit window's samples
  // ---- geometry: causal block length K and state depth D (tables only) ----
  int K = 1;
  int64_t D = 1;
  {
    pc_run_out none;
    memset(&none, 0, sizeof(none));
    RunPlan pl;
    pl.k_out = &K;
    pl.reach_out = &D;
    pl.tables_only = true;
    pc_status rs = run_impl(ctx, dp, dt, 0, &fo, &none, st, pl);
    if (rs != PC_OK) return rs;
  }
  // segment length: a multiple of K, so that the recomputed segments' causal blocks are the ones of
  // the uninterrupted run (bit-identical histories)
  const int64_t C = Cask > 0 ? ((Cask + K - 1) / K) * K : S;
  const int64_t nseg = Cask > 0 ? (n_steps + C - 1) / C : 1;
  const int64_t st_len = state_doubles((int64_t)nbn, D);
  // ---- scratch: history store, E_d at the whole and half steps of a segment, history adjoints,
  // small per-dipole arrays, the fit's inputs and its cotangent, the checkpoint states ----
  const int64_t Sg = Cask > 0 ? std::min(C, n_steps) + 1 : S;   // samples of a segment's outputs
  const int64_t Wg = Cask > 0 ? pow2_at_least(D + C + kMaxBlock + 2) : S;  // store rows
  const size_t hist = al(nbn * (size_t)Wg * sizeof(double));
  const size_t edb = al(nbn * (size_t)Sg * sizeof(double));
  const size_t half = al(nbn * (size_t)(Sg - 1) * sizeof(double));
  const size_t mu_b = al(nbn * (size_t)Wg * 3 * sizeof(double));
  const size_t small = al(nbn * (2 + 1 + (2 * kMaxBlock + 1) + 1 + 2 + 2 + 1) * sizeof(double));
  const size_t fit_b = rates ? 3 * al(nbn * (size_t)flen * sizeof(double)) + al(4 * nbn * sizeof(double)) : 0;
  const size_t ck_b = Cask > 0 ? al((size_t)std::max<int64_t>(nseg - 1, 0) * st_len * sizeof(double)) : 0;
  if (ctx->adj_scratch.reserve(3 * hist + edb + half + mu_b + small + fit_b + ck_b) != cudaSuccess) return PC_ERR_CUDA;
  char *p = (char *)ctx->adj_scratch.ptr;
  double *d = (double *)p, *dd = (double *)(p + hist), *ddd = (double *)(p + 2 * hist);
  double *Ed = (double *)(p + 3 * hist);
  double *Eh = (double *)(p + 3 * hist + edb);
  double *mu = (double *)(p + 3 * hist + edb + half);
  double *sm = (double *)(p + 3 * hist + edb + half + mu_b);
  char *fp_ = p + 3 * hist + edb + half + mu_b + small;
  double *ke = rates ? (double *)fp_ : nullptr;                             // [nbn][flen]
  double *kdd = rates ? (double *)(fp_ + al(nbn * (size_t)flen * 8)) : nullptr;  // d' over the window
  double *dseed = rates ? (double *)(fp_ + 2 * al(nbn * (size_t)flen * 8)) : nullptr;
  double *fpar = rates ? (double *)(fp_ + 3 * al(nbn * (size_t)flen * 8)) : nullptr;  // gamma, omega, amp, phase
  double *ck = Cask > 0 ? (double *)(fp_ + fit_b) : nullptr;  // state at step c C: ck + (c - 1) st_len
  const int2 *delay = nullptr;
  const double *tab = nullptr;
  // ---- forward ----
  if (Cask == 0) {
    // the whole history and the half-step fields, in the adjoint's scratch
    pc_run_out fw;
    memset(&fw, 0, sizeof(fw));
    fw.d = d;
    fw.d_dot = dd;
    fw.d_ddot = ddd;
    fw.Ed = Ed;
    RunPlan pl;
    pl.Ehalf = Eh;
    pl.motion = motion;
    pl.delay_out = &delay;
    pl.rk4tab_out = &tab;
    if (rates) {
      pl.ke = ke;
      pl.kdd = kdd;
      pl.ke_first = first;
      pl.ke_len = flen;
    }
    pc_status rs = run_impl(ctx, dp, dt, n_steps, &fo, &fw, st, pl);
    if (rs != PC_OK) return rs;
  } else {
    // segment by segment in a ring of the context, keeping the state at every segment boundary
    // (and the fit window's kinetic energies and d')
    for (int64_t c = 0; c < nseg; ++c) {
      const int64_t n0 = c * C, len = std::min(C, n_steps - n0);
      pc_run_opts so = fo;
      so.state_in = c > 0 ? ck + (c - 1) * st_len : nullptr;
      so.state_out = c + 1 < nseg ? ck + c * st_len : nullptr;
      pc_run_out none;
      memset(&none, 0, sizeof(none));
      RunPlan pl;
      if (rates) {
        pl.ke = ke;
        pl.kdd = kdd;
        pl.ke_first = first;
        pl.ke_len = flen;
      }
      pc_status rs = run_impl(ctx, dp, dt, len, &so, &none, st, pl);
      if (rs != PC_OK) return rs;
    }
  }
  const size_t hs = (size_t)(2 * n_steps + 1) * 3 * sizeof(double);
  if (motion && gm)
    for (double *gp : {gm->pos, gm->vel, gm->acc})
      if (gp && cudaMemsetAsync(gp, 0, nbn * hs, st) != cudaSuccess) return PC_ERR_CUDA;
  AdjArgs A;
  memset(&A, 0, sizeof(A));
  RunArgs &a = A.f;
  a.B = dp->B;
  a.N = dp->N;
  a.origin = dp->origin;
  a.axis = dp->axis;
  a.q = dp->q;
  a.m1 = dp->m1;
  a.m2 = dp->m2;
  a.omega0 = dp->omega0;
  a.d0 = dp->d0;
  a.dt = dt;
  a.n_begin = 0;
  a.n_steps = n_steps;
  a.d = d;
  a.dd = dd;
  a.ddd = ddd;
  a.hs = Wg;
  a.wm = Cask > 0 ? Wg - 1 : -1;
  a.Ed = Ed;
  a.Ehalf = Eh;
  a.rk4tab = const_cast<double *>(tab);
  a.nsplit = 1;
  a.status = ctx->d_status;
  A.wE = wE;
  A.mu = mu;
  A.lam = sm;
  A.carry = sm + 2 * nbn;
  A.Ebar = sm + 3 * nbn;
  A.w0bar = sm + (3 + 2 * kMaxBlock + 1) * nbn;
  A.tau = A.w0bar + nbn;
  A.wts = A.tau + 2 * nbn;
  A.disp = A.wts + 2 * nbn;
  A.delay = delay;
  if (motion) {
    a.org_pos = motion->pos;
    a.org_vel = motion->vel;
    a.org_acc = motion->acc;
    if (gm) {
      A.gpos = gm->pos;
      A.gvel = gm->vel;
      A.gacc = gm->acc;
    }
  }
  A.g_origin = g->origin;
  A.g_omega0 = g->omega0;
  A.g_d0 = g->d0;
  if (cudaMemsetAsync(mu, 0, nbn * (size_t)Wg * 3 * sizeof(double), st) != cudaSuccess) return PC_ERR_CUDA;
  if (rates) {
    // the fit of the forward run's kinetic energies, then its adjoint: a cotangent on every d'
    // sample of the window, added to that sample's adjoint when the reverse sweep consumes it
    if (cudaMemsetAsync(dseed, 0, nbn * (size_t)flen * sizeof(double), st) != cudaSuccess) return PC_ERR_CUDA;
    double *fg = fpar, *fw_ = fpar + nbn, *fa_ = fpar + 2 * nbn, *fph = fpar + 3 * nbn;
    pc_status ls = launch_fit(ctx, ke, (int)nbn, flen, dt, 0, fg, fw_, fa_, fph, st);
    if (ls != PC_OK) return ls;
    FitAdjArgs fj;
    fj.ke = ke;
    fj.K = (int)nbn;
    fj.S = flen;
    fj.first = 0;
    fj.dt = dt;
    fj.gamma = fg;
    fj.omega = fw_;
    fj.amp = fa_;
    fj.phase = fph;
    fj.dL_dgamma = dL_dgamma;
    fj.dL_domega = dL_domega;
    fj.dd = kdd;
    fj.m1 = dp->m1;
    fj.m2 = dp->m2;
    fj.q = dp->q;
    fj.seed = dseed;
    fj.status = ctx->d_status;
    ke_fit_adjoint_kernel<<<(unsigned)nbn, kFitThreads, 0, st>>>(fj);
    A.dseed = dseed;
    A.seed_first = first;
    A.seed_len = flen;
    if (gamma_out && cudaMemcpyAsync(gamma_out, fg, nbn * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return PC_ERR_CUDA;
    if (omega_out && cudaMemcpyAsync(omega_out, fw_, nbn * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return PC_ERR_CUDA;
  }
  const unsigned rgrid = (unsigned)((nbn + 127) / 128);
  // recompute segment c into the segment store (its E_d at the whole and half steps with it), and
  // point the reverse's arguments at it
  auto recompute = [&](int64_t c) -> pc_status {
    const int64_t n0 = c * C, len = std::min(C, n_steps - n0);
    pc_run_opts so = fo;
    so.state_in = c > 0 ? ck + (c - 1) * st_len : nullptr;
    pc_run_out ro;
    memset(&ro, 0, sizeof(ro));
    ro.Ed = Ed;
    RunPlan pl;
    pl.Ehalf = Eh;
    pl.sd = d;
    pl.sdd = dd;
    pl.sddd = ddd;
    pl.shs = Wg;
    pl.swm = Wg - 1;
    pl.delay_out = &delay;
    pl.rk4tab_out = &tab;
    pc_status rs = run_impl(ctx, dp, dt, len, &so, &ro, st, pl);
    if (rs != PC_OK) return rs;
    a.n_begin = n0;
    a.n_steps = n0 + len;
    a.rk4tab = const_cast<double *>(tab);
    A.delay = delay;
    return PC_OK;
  };
  if (Cask > 0) {
    pc_status rs = recompute(nseg - 1);
    if (rs != PC_OK) return rs;
  }
  adj_init_kernel<<<rgrid, 128, 0, st>>>(A);
  // margin for charge offsets: three times the largest initial |r_dip|, in samples, plus one
  std::vector<double> hq(nbn), hd0(nbn), htau(2 * nbn), hdisp(nbn);
  if (cudaMemcpyAsync(hq.data(), dp->q, nbn * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(hd0.data(), dp->d0, nbn * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(htau.data(), A.tau, 2 * nbn * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(hdisp.data(), A.disp, nbn * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PC_ERR_CUDA;
  double smax = 0.0, spread = 0.0;
  for (size_t k = 0; k < nbn; ++k) {
    smax = std::max(smax, std::fabs(hd0[k] / hq[k]));
    if (htau[2 * k] <= htau[2 * k + 1]) spread = std::max(spread, htau[2 * k + 1] - htau[2 * k]);
  }
  // moving origins: delays drift by up to the two origins' displacements
  double dmax = 0.0;
  for (double v : hdisp) dmax = std::max(dmax, v);
  A.margin = (int64_t)std::ceil(3.0 * smax / (kC * dt) + 2.0 * dmax) + 2;
  const int wmax = (int)std::max(1.0, std::min<double>(std::ceil(spread) + K + 2.0 * A.margin + 6.0, (double)S));
  const size_t smem = (size_t)wmax * 3 * sizeof(double);
  if (smem > 200 * 1024) return PC_ERR_ARG;  // source windows beyond shared memory
  const bool mov = motion != nullptr;
  if (cudaFuncSetAttribute(mov ? adj_field_kernel<true> : adj_field_kernel<false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return PC_ERR_CUDA;
  if (fseed && fseed->P > 0) {
    // the field loss seeds the history adjoints and the origin gradients before the sweep; its
    // window spans the points' delays from each source, at most 8 500 samples
    const int fw = 8500;
    const size_t fsm = (size_t)fw * 3 * sizeof(double);
    if (cudaFuncSetAttribute(fields_adj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm) != cudaSuccess)
      return PC_ERR_CUDA;
    fields_adj_kernel<<<dim3((unsigned)dp->N, (unsigned)fseed->T, (unsigned)dp->B), 128, fsm, st>>>(A, *fseed, fw);
  }
  const dim3 fgrid((unsigned)dp->N, (unsigned)dp->B);
  // reverse sweep over the causal blocks, last first (segment by segment when checkpointing)
  for (int64_t c = nseg - 1; c >= 0; --c) {
    if (Cask > 0 && c < nseg - 1) {
      pc_status rs = recompute(c);
      if (rs != PC_OK) return rs;
    }
    const int64_t s0 = c * C, s1 = std::min(n_steps, s0 + C);
    const int64_t nblocks = (s1 - s0 + K - 1) / K;
    for (int64_t bk = nblocks - 1; bk >= 0; --bk) {
      const int64_t n0 = s0 + bk * K;
      const int kb = (int)std::min((int64_t)K, s1 - n0);
      adj_rk4_kernel<<<rgrid, 128, 0, st>>>(A, n0, kb);
      if (mov) adj_field_kernel<true><<<fgrid, 128, smem, st>>>(A, n0, 2 * kb, wmax);
      else adj_field_kernel<false><<<fgrid, 128, smem, st>>>(A, n0, 2 * kb, wmax);
    }
  }
  // the driving field at t = 0 (static configuration) and the final gradients
  if (mov) adj_field_kernel<true><<<fgrid, 128, smem, st>>>(A, 0, 0, wmax);
  else adj_field_kernel<false><<<fgrid, 128, smem, st>>>(A, 0, 0, wmax);
  adj_final_kernel<<<rgrid, 128, 0, st>>>(A);
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}
}  // namespace pc

extern "C" pc_status pc_dipoles_adjoint(pc_ctx *ctx, const pc_dipoles *dp, double dt, int64_t n_steps,
                                        const pc_run_opts *opts, const double *dL_dEnergyFinal,
                                        const pc_dipole_grads *g, void *stream) {
  if (!ctx || !dL_dEnergyFinal) return PC_ERR_ARG;
  pc::DeviceGuard gd(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  pc_status bs = pc::begin_call(ctx, st);
  if (bs != PC_OK) return bs;
  pc_status rs = pc::adjoint_core(ctx, dp, dt, n_steps, opts, dL_dEnergyFinal, false, nullptr, nullptr, nullptr,
                                  nullptr, g, st);
  if (rs != PC_OK) return rs;
  return pc::end_call(ctx, st);
}

extern "C" pc_status pc_dipoles_adjoint_moving(pc_ctx *ctx, const pc_dipoles *dp, const pc_dipole_motion *motion,
                                               double dt, int64_t n_steps, const pc_run_opts *opts,
                                               const double *dL_dEnergyFinal, const pc_dipole_grads *g,
                                               const pc_dipole_motion_grads *gm, void *stream) {
  if (!ctx || !motion || !dL_dEnergyFinal) return PC_ERR_ARG;
  pc::DeviceGuard gd(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  pc_status bs = pc::begin_call(ctx, st);
  if (bs != PC_OK) return bs;
  pc_status rs = pc::adjoint_core(ctx, dp, dt, n_steps, opts, dL_dEnergyFinal, false, nullptr, nullptr, nullptr,
                                  nullptr, g, st, nullptr, motion, gm);
  if (rs != PC_OK) return rs;
  return pc::end_call(ctx, st);
}

extern "C" pc_status pc_dipoles_rates_adjoint(pc_ctx *ctx, const pc_dipoles *dp, double dt, int64_t n_steps,
                                              const pc_run_opts *opts, const double *dL_dgamma,
                                              const double *dL_domega, double *gamma, double *omega,
                                              const pc_dipole_grads *g, void *stream) {
  if (!ctx || (!dL_dgamma && !dL_domega)) return PC_ERR_ARG;
  pc::DeviceGuard gd(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  pc_status bs = pc::begin_call(ctx, st);
  if (bs != PC_OK) return bs;
  pc_status rs = pc::adjoint_core(ctx, dp, dt, n_steps, opts, nullptr, true, dL_dgamma, dL_domega, gamma, omega, g,
                                  st);
  if (rs != PC_OK) return rs;
  return pc::end_call(ctx, st);
}

extern "C" pc_status pc_dipoles_fields_adjoint(pc_ctx *ctx, const pc_dipoles *dp, double dt, int64_t n_steps,
                                               const pc_run_opts *opts, const double *points, int64_t P,
                                               const double *times, int32_t T, const pc_field_out *cot,
                                               const pc_dipole_grads *g, void *stream) {
  if (!ctx || !cot || !times || T < 1 || P < 0 || (P > 0 && !points)) return PC_ERR_ARG;
  if (cot->mask) return PC_ERR_ARG;  // the mask has no cotangent
  for (int i = 0; i < T; ++i)
    if (!isfinite(times[i]) || times[i] < 0.0) return PC_ERR_ARG;
  pc::DeviceGuard gd(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  pc_status bs = pc::begin_call(ctx, st);
  if (bs != PC_OK) return bs;
  // the frame times on the device (context scratch of the field outputs)
  if (ctx->out_chunks.reserve((size_t)T * sizeof(double)) != cudaSuccess) return PC_ERR_CUDA;
  double *tdev = (double *)ctx->out_chunks.ptr;
  if (cudaMemcpyAsync(tdev, times, (size_t)T * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return PC_ERR_CUDA;
  pc::FieldSeed fs;
  fs.pts = points;
  fs.P = P;
  fs.T = T;
  fs.times = tdev;
  fs.cE = (const double *)cot->E;
  fs.cB = (const double *)cot->B;
  fs.cphi = (const double *)cot->phi;
  fs.cA = (const double *)cot->A;
  pc_status rs = pc::adjoint_core(ctx, dp, dt, n_steps, opts, nullptr, false, nullptr, nullptr, nullptr, nullptr, g,
                                  st, &fs);
  if (rs != PC_OK) return rs;
  return pc::end_call(ctx, st);
}
