// float32 device helpers shared by the field sum and the oscillator run: the retarded state of
// one dipole charge from the float32 history mirror (Eq. ret_t on a linear segment, solved as a
// quadratic in offsets from the dipole centre) and the net field of a dipole's two charges in
// difference form (Eqs. E, B, V, A in Griffiths' form with v and a along the dipole axis).
// Lengths in units of c*dt, times in samples, velocities in units of c.
#pragma once
#include "pc_internal.cuh"

namespace pc {

// a root up to this many samples past the last sample is taken at the last sample
constexpr float kEndTol = 1e-3f;

__device__ __forceinline__ float fsqrt_approx(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }

// Sample j of a dipole history; before the first sample the dipole rests with moment d[0].
// Sample indices are 32-bit in the float32 path: conversions to 64-bit integers run on the
// float64 unit, which is the narrowest pipe of this GPU.
__device__ __forceinline__ float4 dip_sample(const float4 *H, int j) {
  if (j >= 0) return __ldg(H + j);
  float4 h0 = __ldg(H);
  return make_float4(h0.x, 0.f, 0.f, 0.f);
}

// Retarded state of one dipole charge at offset smu*X along the axis from the dipole centre.
//   kb + xc: retarded time of the centre, in samples (xc small)
//   rn = |rho|, rp = rho . axis (units of c dt)
// Out: X, V, Ac interpolated at the charge's own retarded time; delta = its distance minus rn.
__device__ __forceinline__ int dip_charge_solve(const float4 *H, int S, int kb, float xc, float rn, float rp,
                                                float smu, float &X, float &V, float &Ac, float &delta) {
  if (!(fabsf(xc) < 1e8f)) return PC_ERR_NOCONV;
  int kc = __float2int_rd(xc);
  float thc = xc - (float)kc;
  int j = kb + kc;
  // first-order estimate of the charge's delay offset picks its segment
  {
    float4 h = dip_sample(H, j < S ? j : S - 1);
    float d0 = (rn > 0.f) ? -smu * h.x * __fdividef(rp, rn) : 0.f;
    int st = __float2int_rd(thc - d0);
    j += st;
    thc -= (float)st;
  }
  for (int it = 0; it < 6; ++it) {
    if (j > S - 2) {
      // past the end: solve on the last segment extended; a root up to kEndTol past the last
      // sample is clamped to it, a later one is a history error
      thc += (float)(j - (S - 2));
      j = S - 2;
    }
    float4 h0 = dip_sample(H, j), h1 = dip_sample(H, j + 1);
    if (j < 0) h1 = h0;  // static segment
    float dx = h1.x - h0.x;
    float sc = smu * (h0.x + thc * dx);
    float w = smu * dx;
    float A = 1.f - w * w;
    float B = rn - w * (rp - sc);
    float C = sc * (2.f * rp - sc);
    float sq = fsqrt_approx(fmaxf(B * B - A * C, 0.f));
    float dl = (B > 0.f) ? -__fdividef(C, B + sq) : __fdividef(-B + sq, A);
    float th = thc - dl;
    bool ok = (j < 0) ? ((float)j + th <= 1e-4f)
                      : (th >= -1e-4f && (th <= 1.0001f || (j == S - 2 && th <= 1.f + kEndTol)));
    if (ok) {
      th = fminf(fmaxf(th, 0.f), 1.f);
      X = h0.x + th * dx;
      V = h0.y + th * (h1.y - h0.y);
      Ac = h0.z + th * (h1.z - h0.z);
      delta = dl;
      return 0;
    }
    if (!(fabsf(th) < 1e8f)) return PC_ERR_NOCONV;
    if (j == S - 2 && th > 1.f) return PC_ERR_HISTORY;
    int st = __float2int_rd(th);
    j += st;
    thc -= (float)st;
  }
  return PC_ERR_NOCONV;
}

template <int KIND>
__device__ __forceinline__ void dipole_pair_mixed(float rx, float ry, float rz, float rn, float px, float py, float pz,
                                                  float rp, float mup, float mum, float qs, float Xp, float Vp,
                                                  float Ap, float dp, float Xm, float Vm, float Am, float dm,
                                                  float rex, float *acc, uint8_t &mask) {
  // charge 1 = positive (offset +mup X), charge 0 = negative (offset -mum X)
  const float s1 = mup * Xp, s0 = -mum * Xm, ds = mup * Xp + mum * Xm;
  const float v1 = mup * Vp, v0 = -mum * Vm, dv = mup * Vp + mum * Vm;
  const float a1 = mup * Ap, a0 = -mum * Am, da = mup * Ap + mum * Am;
  const float R0 = rn + dm, dR = dp - dm, R1 = R0 + dR;
  if (R0 <= rex || R1 <= rex) {
    mask = 1;
    // one charge coincides with the point: add the other one alone
    const bool use1 = R1 > rex;
    if (!(R0 > rex) && !use1) return;
    const float s = use1 ? s1 : s0, v = use1 ? v1 : v0, al = use1 ? a1 : a0, R = use1 ? R1 : R0;
    const float sign = use1 ? qs : -qs;
    const float ap = rp - s;
    const float Ru = R - v * ap;
    const float i1 = __frcp_rn(Ru);
    const float i2 = i1 * i1, i3 = i2 * i1;
    float G = 0.f, Q = 0.f;
    if (KIND != PC_RADIATION) G += 1.f - v * v;
    if (KIND != PC_COULOMB) {
      G += al * ap;
      Q = al;
    }
    const float Ca = G * i3;
    const float Cp = -R * v * G * i3 - Q * R * i2;
    const float Bc = -v * G * i3 - Q * i2;
    const float ax_ = rx - s * px, ay_ = ry - s * py, az_ = rz - s * pz;
    acc[0] += sign * (Ca * ax_ + Cp * px);
    acc[1] += sign * (Ca * ay_ + Cp * py);
    acc[2] += sign * (Ca * az_ + Cp * pz);
    const float cx = ry * pz - rz * py, cy = rz * px - rx * pz, cz = rx * py - ry * px;
    acc[3] += sign * Bc * cx;
    acc[4] += sign * Bc * cy;
    acc[5] += sign * Bc * cz;
    acc[6] += sign * i1;
    const float va = sign * v * i1;
    acc[7] += va * px;
    acc[8] += va * py;
    acc[9] += va * pz;
    return;
  }
  const float ap0 = rp - s0, ap1 = rp - s1, dap = -ds;
  const float Ru0 = R0 - v0 * ap0;
  const float dRu = dR - (dv * ap1 + v0 * dap);
  const float Ru1 = Ru0 + dRu;
  const float i0 = __frcp_rn(Ru0), i1 = __frcp_rn(Ru1);
  const float di = -dRu * i0 * i1;
  const float i02 = i0 * i0, i12 = i1 * i1;
  const float i03 = i02 * i0, i13 = i12 * i1;
  const float di2 = di * (i0 + i1);
  const float di3 = di * (i12 + i1 * i0 + i02);
  float G0 = 0.f, dG = 0.f;
  if (KIND != PC_RADIATION) {
    G0 += 1.f - v0 * v0;
    dG += -dv * (v1 + v0);
  }
  if (KIND != PC_COULOMB) {
    G0 += a0 * ap0;
    dG += da * ap1 + a0 * dap;
  }
  const float G1 = G0 + dG;
  const float Ca0 = G0 * i03, Ca1 = G1 * i13;
  const float dCa = dG * i13 + G0 * di3;
  // C_p = -R v G i^3 - alpha R i^2 ; B coefficient C_p / R = -v G i^3 - alpha i^2
  const float P0 = R0 * v0 * G0;
  const float dP = dR * v1 * G1 + R0 * (dv * G1 + v0 * dG);
  float dCp = -(dP * i13 + P0 * di3);
  const float dvG = dv * G1 + v0 * dG;
  float dBc = -(dvG * i13 + v0 * G0 * di3);
  if (KIND != PC_COULOMB) {
    const float Q0 = a0 * R0, dQ = da * R1 + a0 * dR;
    dCp -= dQ * i12 + Q0 * di2;
    dBc -= da * i12 + a0 * di2;
  }
  const float ep = dCp - (Ca1 * s1 - Ca0 * s0);
  acc[0] += qs * (dCa * rx + ep * px);
  acc[1] += qs * (dCa * ry + ep * py);
  acc[2] += qs * (dCa * rz + ep * pz);
  const float cx = ry * pz - rz * py, cy = rz * px - rx * pz, cz = rx * py - ry * px;
  acc[3] += qs * dBc * cx;
  acc[4] += qs * dBc * cy;
  acc[5] += qs * dBc * cz;
  acc[6] += qs * di;
  const float dA = qs * (dv * i1 + v0 * di);
  acc[7] += dA * px;
  acc[8] += dA * py;
  acc[9] += dA * pz;
}

}  // namespace pc
