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
  const double R2 = dot3(a, a);
  const double iR = rsqrt(R2);  // 1/R and R from one reciprocal square root
  const double R = R2 * iR;
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

namespace pc {

// Reverse of lw_add_f64<PC_TOTAL> for one charge: given the cotangents of the charge's E, B, phi
// and A (Eqs. E, B, V, A in the Griffiths form of lw_add_f64: E = f [W u - R_u acc] with
// W = c^2 - v.v + a.acc, u = c n - v, R_u = c R - a.v, f = k_e q R / R_u^3; B = n x E / c;
// phi = k_e q c / R_u; A = phi v / c^2), adds the adjoints of a (point minus retarded position), v
// and acc.  Eb, Bb, Ab may be null (zero cotangent).
__device__ inline void lw_full_f64_rev(double q, const double a[3], const double v[3], const double acc[3],
                                       const double *Eb, const double *Bb, double phib, const double *Ab, double ab[3],
                                       double vb[3], double accb[3]) {
  const double c = kC;
  const double R2 = dot3(a, a);
  const double iR = rsqrt(R2);  // 1/R and R from one reciprocal square root
  const double R = R2 * iR;
  const double n[3] = {a[0] * iR, a[1] * iR, a[2] * iR};
  const double u[3] = {c * n[0] - v[0], c * n[1] - v[1], c * n[2] - v[2]};
  const double Ru = c * R - dot3(a, v);
  const double iRu = 1.0 / Ru;
  const double f = kKe * q * R * iRu * iRu * iRu;
  const double W = c * c - dot3(v, v) + dot3(a, acc);
  const double e[3] = {f * (W * u[0] - Ru * acc[0]), f * (W * u[1] - Ru * acc[1]), f * (W * u[2] - Ru * acc[2])};
  const double ph = kKe * q * c * iRu;
  // A = ph v / c^2 and phi = ph
  double phb = phib;
  if (Ab) {
    phb += dot3(Ab, v) / (c * c);
    for (int k = 0; k < 3; ++k) vb[k] += ph / (c * c) * Ab[k];
  }
  double iRub = phb * kKe * q * c;
  // B = (n x e) / c: e_bar += (B_bar / c) x n, n_bar += e x (B_bar / c)
  double eb[3] = {0.0, 0.0, 0.0}, nb[3] = {0.0, 0.0, 0.0};
  if (Eb)
    for (int k = 0; k < 3; ++k) eb[k] = Eb[k];
  if (Bb) {
    const double y[3] = {Bb[0] / c, Bb[1] / c, Bb[2] / c};
    eb[0] += y[1] * n[2] - y[2] * n[1];
    eb[1] += y[2] * n[0] - y[0] * n[2];
    eb[2] += y[0] * n[1] - y[1] * n[0];
    nb[0] += e[1] * y[2] - e[2] * y[1];
    nb[1] += e[2] * y[0] - e[0] * y[2];
    nb[2] += e[0] * y[1] - e[1] * y[0];
  }
  // e = f (W u - Ru acc)
  const double eu = dot3(eb, u), eacc = dot3(eb, acc);
  const double fb = W * eu - Ru * eacc;
  const double Wb = f * eu;
  double ub[3] = {f * W * eb[0], f * W * eb[1], f * W * eb[2]};
  double Rub = -f * eacc;
  for (int k = 0; k < 3; ++k) accb[k] += -f * Ru * eb[k];
  // W = c^2 - v.v + a.acc
  for (int k = 0; k < 3; ++k) {
    vb[k] += -2.0 * Wb * v[k];
    ab[k] += Wb * acc[k];
    accb[k] += Wb * a[k];
  }
  // f = k_e q R iRu^3
  double Rb = fb * f * iR;
  iRub += fb * 3.0 * f / iRu;
  // iRu = 1 / Ru
  Rub += -iRub * iRu * iRu;
  // Ru = c R - a.v
  Rb += c * Rub;
  for (int k = 0; k < 3; ++k) {
    ab[k] += -Rub * v[k];
    vb[k] += -Rub * a[k];
  }
  // u = c n - v
  for (int k = 0; k < 3; ++k) {
    nb[k] += c * ub[k];
    vb[k] += -ub[k];
  }
  // n = a iR
  const double iRb = dot3(nb, a);
  for (int k = 0; k < 3; ++k) ab[k] += iR * nb[k];
  Rb += -iRb * iR * iR;
  // R = |a|
  for (int k = 0; k < 3; ++k) ab[k] += Rb * a[k] * iR;
}

}  // namespace pc
