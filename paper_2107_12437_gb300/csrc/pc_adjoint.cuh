// Reverse-mode helpers of the oscillator adjoint: the adjoint of the float64 Lienard-Wiechert field
// of one charge (Eq. E in Griffiths' form) with respect to its geometric inputs.
#pragma once
#include "pc_lw_f64.cuh"

namespace pc {

// Reverse of lw_E_f64 for one charge: given the adjoint Eb of its field E (Griffiths' form,
// E = f [(c^2 - v.v + a.acc) u - R_u acc], u = c a/R - v, R_u = c R - a.v, f = k_e q R / R_u^3),
// adds the adjoints of its inputs a (point minus retarded position), v and acc.
__device__ __forceinline__ void lw_E_f64_rev(double q, const double a[3], const double v[3], const double acc[3],
                                             const double Eb[3], double ab[3], double vb[3], double accb[3]) {
  const double c = kC;
  const double R = sqrt(dot3(a, a));
  const double iR = 1.0 / R;
  const double u[3] = {c * a[0] * iR - v[0], c * a[1] * iR - v[1], c * a[2] * iR - v[2]};
  const double Ru = c * R - dot3(a, v);
  const double iRu = 1.0 / Ru;
  const double f = kKe * q * R * iRu * iRu * iRu;
  const double aa = dot3(a, acc);
  const double W = c * c - dot3(v, v) + aa;
  // E_k = f (W u_k - Ru acc_k)
  const double Eu = dot3(Eb, u), Eacc = dot3(Eb, acc);
  const double fb = W * Eu - Ru * Eacc;
  const double Wb = f * Eu;
  const double ub[3] = {f * W * Eb[0], f * W * Eb[1], f * W * Eb[2]};
  double Rub = -f * Eacc;
  for (int k = 0; k < 3; ++k) accb[k] += -f * Ru * Eb[k];
  // W = c^2 - v.v + a.acc
  for (int k = 0; k < 3; ++k) {
    accb[k] += Wb * a[k];
    ab[k] += Wb * acc[k];
    vb[k] += -2.0 * Wb * v[k];
  }
  // f = k_e q R Ru^-3
  double Rb = fb * f * iR;
  Rub += -3.0 * fb * f * iRu;
  // Ru = c R - a.v
  Rb += c * Rub;
  for (int k = 0; k < 3; ++k) {
    ab[k] += -Rub * v[k];
    vb[k] += -Rub * a[k];
  }
  // u = c a / R - v
  const double ua = dot3(ub, a);
  for (int k = 0; k < 3; ++k) {
    ab[k] += c * ub[k] * iR;
    vb[k] += -ub[k];
  }
  Rb += -c * ua * iR * iR;
  // R = |a|
  for (int k = 0; k < 3; ++k) ab[k] += Rb * a[k] * iR;
}

}  // namespace pc
