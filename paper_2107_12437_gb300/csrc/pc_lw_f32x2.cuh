// The float32 fast path of the dipole pair algebra (pc_lw_f32.cuh: dip_pair_states_fast,
// dipole_pair_fast) for two field points at once: point A in the x lane and point B in the y lane
// of every float2, so that the parts of the algebra that are scalar per point (the differences
// between a dipole's two charges that carry the cancellation, Sec. 2.3 dipoles seen from afar)
// also run as packed FFMA2 / FMUL2 / FADD2 instructions.  Same equations, same units and the same
// rounding per point as the one-point path, up to the order of the packed operations.
#pragma once
#include "pc_lw_f32.cuh"

namespace pc {

struct V2 {
  float2 v;
  __device__ __forceinline__ V2() {}
  __device__ __forceinline__ V2(float2 a) : v(a) {}
  __device__ __forceinline__ V2(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ explicit V2(float a) : v(make_float2(a, a)) {}
};
__device__ __forceinline__ V2 operator+(V2 a, V2 b) { return V2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ V2 operator-(V2 a) { return V2(-a.v.x, -a.v.y); }
__device__ __forceinline__ V2 operator-(V2 a, V2 b) { return V2(__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y))); }
__device__ __forceinline__ V2 operator*(V2 a, V2 b) { return V2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ V2 fma2(V2 a, V2 b, V2 c) { return V2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ V2 rcp2(V2 a) { return V2(__fdividef(1.f, a.v.x), __fdividef(1.f, a.v.y)); }

// Retarded state of one charge of the dipole (offset smu X along the axis; smu = mu+ or -mu-) at
// both points: the series root of dip_pair_states_fast on the segment [x0, x0 + dx] of the
// centre's retarded time, fraction thc.  Returns the charge's fraction on the segment; eps is the
// series parameter (the root is kept only for |eps_+| + |eps_-| < 1e-2).
struct Ch2 {
  V2 X, V, Ac, dl;  // offset / velocity / acceleration factors at the root, delta = R - rn
};
__device__ __forceinline__ V2 charge2_state(float smu, V2 x0, V2 dx, V2 v0, V2 dv, V2 a0, V2 da, V2 Xc, V2 thc,
                                            V2 rn, V2 rp, Ch2 &c, V2 &eps) {
  const V2 S(smu);
  const V2 sc = S * Xc, w = S * dx;
  const V2 A = fma2(-w, w, V2(1.f));          // 1 - w^2
  const V2 B = fma2(-w, rp - sc, rn);          // rn - w (rp - sc)
  const V2 C = sc * fma2(V2(2.f), rp, -sc);    // sc (2 rp - sc)
  const V2 r = rcp2(B);
  const V2 Cr = C * r;
  const V2 h = Cr * V2(0.5f);
  eps = A * Cr * r;
  const V2 ndl = fma2(h, eps * fma2(eps, V2(0.125f), V2(0.25f)), h);  // -delta
  const V2 th = thc + ndl;
  c.X = fma2(th, dx, x0);
  c.V = fma2(th, dv, v0);
  c.Ac = fma2(th, da, a0);
  c.dl = -ndl;
  return th;
}

// Net field of the dipole's two charges (charge + = P, charge - = M) at both points, added to
// acc[10] = (E_x, E_y, E_z, B_x, B_y, B_z, phi, A_x, A_y, A_z), each a float2 over the points; the
// algebra of dipole_pair_fast.  ok = (1 or 0, 1 or 0) keeps or drops each point's contribution
// (the coefficients of a dropped point are replaced by 0 before they multiply anything, so a
// non-finite intermediate of that point cannot reach the sums).
template <int KIND>
__device__ __forceinline__ void dipole2_fast(V2 rx, V2 ry, V2 rz, V2 rn, float px, float py, float pz, V2 rp,
                                             float mup, float mum, float qs, const Ch2 &P, const Ch2 &M, bool okA,
                                             bool okB, V2 (&acc)[10]) {
  const V2 mp(mup), mm(mum);
  const V2 s1 = mp * P.X, s0 = -(mm * M.X);
  const V2 v1 = mp * P.V, v0 = -(mm * M.V);
  const V2 a1 = mp * P.Ac, a0 = -(mm * M.Ac);
  const V2 ds = fma2(mp, P.X, mm * M.X), dv = fma2(mp, P.V, mm * M.V), da = fma2(mp, P.Ac, mm * M.Ac);
  const V2 R1 = rn + P.dl, R0 = rn + M.dl;
  const V2 dR = P.dl - M.dl;
  const V2 ap1 = rp - s1, ap0 = rp - s0;
  const V2 Ru1 = fma2(-v1, ap1, R1), Ru0 = fma2(-v0, ap0, R0);
  const V2 dRu = dR - fma2(dv, ap1, -(v0 * ds));
  const V2 i1 = rcp2(Ru1), i0 = rcp2(Ru0);
  const V2 i21 = i1 * i1, i20 = i0 * i0;
  const V2 i31 = i21 * i1, i30 = i20 * i0;
  const V2 di = -(dRu * i0 * i1);
  const V2 di2 = di * (i1 + i0);
  const V2 di3 = di * fma2(i1, i0, i21 + i20);
  V2 G0(0.f), dG(0.f);
  if (KIND != PC_RADIATION) {
    G0 = fma2(-v0, v0, V2(1.f));
    dG = -(dv * (v1 + v0));
  }
  if (KIND != PC_COULOMB) {
    G0 = fma2(a0, ap0, G0);
    dG = fma2(da, ap1, fma2(-a0, ds, dG));
  }
  const V2 G1 = G0 + dG;
  const V2 Ca1 = G1 * i31, Ca0 = G0 * i30;
  const V2 dCa = fma2(dG, i31, G0 * di3);
  const V2 P0 = R0 * v0 * G0;
  const V2 dvG = fma2(dv, G1, v0 * dG);
  const V2 dP = fma2(dR * v1, G1, R0 * dvG);
  V2 dCp = -fma2(dP, i31, P0 * di3);
  V2 dBc = -fma2(dvG, i31, v0 * G0 * di3);
  if (KIND != PC_COULOMB) {
    const V2 Q0 = a0 * R0, dQ = fma2(da, R1, a0 * dR);
    dCp = dCp - fma2(dQ, i21, Q0 * di2);
    dBc = dBc - fma2(da, i21, a0 * di2);
  }
  const V2 ep = dCp - fma2(Ca1, s1, -(Ca0 * s0));
  const V2 Q(qs);
  V2 cE = Q * dCa, cP = Q * ep, cB = Q * dBc, cA = Q * fma2(dv, i1, v0 * di), cF = Q * di;
  if (!(okA && okB)) {
    cE = V2(okA ? cE.v.x : 0.f, okB ? cE.v.y : 0.f);
    cP = V2(okA ? cP.v.x : 0.f, okB ? cP.v.y : 0.f);
    cB = V2(okA ? cB.v.x : 0.f, okB ? cB.v.y : 0.f);
    cA = V2(okA ? cA.v.x : 0.f, okB ? cA.v.y : 0.f);
    cF = V2(okA ? cF.v.x : 0.f, okB ? cF.v.y : 0.f);
  }
  const V2 X(px), Y(py), Z(pz);
  const V2 cx = fma2(ry, Z, -(rz * Y)), cy = fma2(rz, X, -(rx * Z)), cz = fma2(rx, Y, -(ry * X));
  acc[0] = fma2(cP, X, fma2(cE, rx, acc[0]));
  acc[1] = fma2(cP, Y, fma2(cE, ry, acc[1]));
  acc[2] = fma2(cP, Z, fma2(cE, rz, acc[2]));
  acc[3] = fma2(cB, cx, acc[3]);
  acc[4] = fma2(cB, cy, acc[4]);
  acc[5] = fma2(cB, cz, acc[5]);
  acc[6] = acc[6] + cF;
  acc[7] = fma2(cA, X, acc[7]);
  acc[8] = fma2(cA, Y, acc[8]);
  acc[9] = fma2(cA, Z, acc[9]);
}

}  // namespace pc
