// float64 device helpers shared by the field sum and the oscillator run: the per-segment
// retarded-time solve (Eq. ret_t on a piecewise-linear history) and the Lienard-Wiechert field of
// one charge in Griffiths' form (Eqs. E, B, V, A).
#pragma once
#include "pc_internal.cuh"

namespace pc {

__device__ __forceinline__ double dot3(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// position of source charge `c` at sample k (generic charge, or dipole charge sigma*mu along axis)
struct TrajF64 {
  const double *pos;  // generic: [S][3]
  const double *vel, *acc;
  const double *d, *dd, *ddd;  // dipole: sample k at row slot (k & wm)
  int64_t wm = -1;             // -1: the row holds every sample at its index; W - 1: a ring of W slots
  double R[3], ax[3], w;       // dipole: origin, axis, signed weight / q
  bool dipole;
  __device__ __forceinline__ double dk(int64_t k) const { return d[k & wm]; }
  __device__ __forceinline__ double ddk(int64_t k) const { return dd[k & wm]; }
  __device__ __forceinline__ double dddk(int64_t k) const { return ddd[k & wm]; }
  // moving dipole origin (or null): position, velocity, acceleration at the half steps, [2 S - 1][3];
  // the history holds the whole steps (half-step index 2k)
  const double *Rp = nullptr, *Rv = nullptr, *Ra = nullptr;
  __device__ void p(int64_t k, double o[3]) const {
    if (!dipole) {
      o[0] = pos[3 * k];
      o[1] = pos[3 * k + 1];
      o[2] = pos[3 * k + 2];
    } else {
      double s = w * dk(k);
      const double *c = Rp ? Rp + 6 * k : R;
      o[0] = c[0] + s * ax[0];
      o[1] = c[1] + s * ax[1];
      o[2] = c[2] + s * ax[2];
    }
  }
  __device__ void va(int64_t k, double v[3], double a[3]) const {
    if (!dipole) {
      for (int i = 0; i < 3; ++i) {
        v[i] = vel[3 * k + i];
        a[i] = acc[3 * k + i];
      }
    } else {
      double sv = w * ddk(k), sa = w * dddk(k);
      for (int i = 0; i < 3; ++i) {
        v[i] = (Rv ? Rv[6 * k + i] : 0.0) + sv * ax[i];
        a[i] = (Ra ? Ra[6 * k + i] : 0.0) + sa * ax[i];
      }
    }
  }
};

// Retarded sample segment k and fraction th of one charge.  u = (t - t0)/dt, cdt = c dt.
// Returns 0, or an error code.  k = -1 marks the static state before the first sample.
__device__ inline int solve_f64(const TrajF64 &tr, int64_t S, int static_before, const double r[3], double u, double cdt,
                         int64_t k, int64_t *k_out, double *th_out) {
  const double cdt2 = cdt * cdt;
  if (k < 0) k = 0;
  if (k > S - 2) k = S - 2;
  for (int it = 0; it < 96; ++it) {
    double p0[3], p1[3];
    tr.p(k, p0);
    tr.p(k + 1, p1);
    double a[3] = {r[0] - p0[0], r[1] - p0[1], r[2] - p0[2]};
    double D[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
    double T = u - (double)k;
    double A = cdt2 - dot3(D, D);
    double B = dot3(a, D) - cdt2 * T;
    double C = cdt2 * T * T - dot3(a, a);
    double disc = fmax(B * B - A * C, 0.0);
    double sq = sqrt(disc);
    double th;
    if (B <= 0.0) {
      double den = -B + sq;
      th = (den > 0.0) ? C / den : T;
    } else {
      th = (-B - sq) / A;
    }
    if (!(th == th)) return PC_ERR_NOCONV;
    if (th >= -1e-12 && th <= 1.0 + 1e-12) {
      *k_out = k;
      *th_out = fmin(fmax(th, 0.0), 1.0);
      return 0;
    }
    if (th < 0.0) {
      if (k == 0) {
        // g(t') = c (t - t') - |r - r_s(t')| decreases in t': g(t0) < 0 puts the root before the
        // first sample (static extension or error); otherwise rounding put it at t0 itself
        double g0 = cdt * u - sqrt(dot3(a, a));
        if (g0 < 0.0) {
          if (!static_before) return PC_ERR_HISTORY;
          *k_out = -1;
          *th_out = 0.0;
        } else {
          *k_out = 0;
          *th_out = 0.0;
        }
        return 0;
      }
      double st = floor(th);
      int64_t step = (st < -1e15) ? -k : (int64_t)st;
      k = k + step;
      if (k < 0) k = 0;
    } else {
      if (k == S - 2) return PC_ERR_HISTORY;
      double st = floor(th);
      int64_t step = (st > 1e15) ? S : (int64_t)st;
      k = k + step;
      if (k > S - 2) k = S - 2;
    }
  }
  return PC_ERR_NOCONV;
}

template <int KIND>
__device__ __forceinline__ void lw_add_f64(double q, const double a[3], const double v[3], const double acc[3],
                                           double r_excl, double E[3], double B[3], double *phi, double A[3],
                                           uint8_t *mask) {
  const double c = kC;
  // 1/R and R from one reciprocal square root (float64 division and square root are long
  // sequences on this GPU's narrow float64 unit)
  const double R2 = dot3(a, a);
  const double iR = rsqrt(R2);
  const double R = R2 * iR;
  if (!(R > r_excl)) {
    *mask = 1;
    return;
  }
  double n[3] = {a[0] * iR, a[1] * iR, a[2] * iR};
  double u[3] = {c * n[0] - v[0], c * n[1] - v[1], c * n[2] - v[2]};
  double Ru = c * R - dot3(a, v);
  double iRu = 1.0 / Ru;
  double f = kKe * q * R * iRu * iRu * iRu;
  double e[3] = {0.0, 0.0, 0.0};
  if (KIND != PC_RADIATION) {
    double g = f * (c * c - dot3(v, v));
    e[0] = g * u[0];
    e[1] = g * u[1];
    e[2] = g * u[2];
  }
  if (KIND != PC_COULOMB) {
    // a x (u x acc) = u (a.acc) - acc (a.u)
    double aa = dot3(a, acc);
    e[0] += f * (u[0] * aa - acc[0] * Ru);
    e[1] += f * (u[1] * aa - acc[1] * Ru);
    e[2] += f * (u[2] * aa - acc[2] * Ru);
  }
  E[0] += e[0];
  E[1] += e[1];
  E[2] += e[2];
  const double ic = 1.0 / c;
  B[0] += (n[1] * e[2] - n[2] * e[1]) * ic;
  B[1] += (n[2] * e[0] - n[0] * e[2]) * ic;
  B[2] += (n[0] * e[1] - n[1] * e[0]) * ic;
  double ph = kKe * q * c * iRu;
  *phi += ph;
  double av = ph * ic * ic;
  A[0] += av * v[0];
  A[1] += av * v[1];
  A[2] += av * v[2];
}

}  // namespace pc

namespace pc {

// Electric field only (total), float64: used for the oscillator driving field.
__device__ __forceinline__ void lw_E_f64(double q, const double a[3], const double v[3], const double acc[3],
                                         double E[3]) {
  const double c = kC;
  const double R2 = dot3(a, a);
  const double iR = rsqrt(R2);
  const double R = R2 * iR;
  double u[3] = {c * a[0] * iR - v[0], c * a[1] * iR - v[1], c * a[2] * iR - v[2]};
  double Ru = c * R - dot3(a, v);
  double iRu = 1.0 / Ru;
  double f = kKe * q * R * iRu * iRu * iRu;
  double g = f * (c * c - dot3(v, v));
  double aa = dot3(a, acc);
  E[0] += g * u[0] + f * (u[0] * aa - acc[0] * Ru);
  E[1] += g * u[1] + f * (u[1] * aa - acc[1] * Ru);
  E[2] += g * u[2] + f * (u[2] * aa - acc[2] * Ru);
}

}  // namespace pc
