// Device helpers for the net field of a dipole's two charges in difference form, shared by the
// field sum and the oscillator run, instantiated in float (the mixed path) and in double (pairs
// near a dipole).  Eq. ret_t on a linear history segment is a quadratic in the offset of a charge
// from its dipole centre; the Lienard-Wiechert fields (Eqs. E, B, V, A, Griffiths' form with v and
// a along the dipole axis) are written with scalar coefficients whose +/- differences carry no
// cancellation.  Lengths in units of c*dt, times in samples, velocities in units of c.
#pragma once
#include "pc_internal.cuh"

namespace pc {

// a root up to this many samples past the last sample is taken at the last sample
constexpr float kEndTol = 1e-3f;
// both charges are evaluated on their centre's segment, extended linearly, when their own
// retarded times lie within this many samples of it (the extension error is second order)
constexpr float kExtrap = 0.1f;

template <typename T>
struct Num;
template <>
struct Num<float> {
  static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.f, x); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
  static __device__ __forceinline__ float sqrt0(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
  // floor(x) as an integer and as a float, for |x| < 2^22, without conversion instructions (on this
  // GPU float<->int conversions issue to the float64 unit): adding 1.5 * 2^23 rounds x to an integer
  // held in the low mantissa bits.
  static __device__ __forceinline__ int floor_int(float x, float &fl) {
    const float magic = 12582912.f;
    const float y = x + magic;
    float r = y - magic;
    int i = __float_as_int(y) - 0x4B400000;
    if (r > x) {
      r -= 1.f;
      i -= 1;
    }
    fl = r;
    return i;
  }
  static __device__ __forceinline__ int floor_int(float x) {
    float fl;
    return floor_int(x, fl);
  }
};
template <>
struct Num<double> {
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double sqrt0(double x) { return x > 0.0 ? sqrt(x) : 0.0; }
  static __device__ __forceinline__ int floor_int(double x) { return (int)floor(x); }
  static __device__ __forceinline__ int floor_int(double x, double &fl) {
    fl = floor(x);
    return (int)fl;
  }
};

// Dipole history samples (X = d/(qL), V = d'/(qc), A = d'' dt/(qc)); before the first sample the
// dipole rests at X[0].  Sample indices are 32-bit: conversions to 64-bit integers run on the
// float64 unit, the narrowest pipe of this GPU.
// READ_ONLY: the history does not change while the kernel runs, so loads may use the read-only
// data cache; the oscillator run appends to the history it reads and uses coherent loads.
template <bool READ_ONLY>
struct HistF32T {
  const float4 *H;
  __device__ __forceinline__ float4 load(int j) const { return READ_ONLY ? __ldg(H + j) : H[j]; }
  __device__ __forceinline__ void get(int j, float &x, float &v, float &a) const {
    float4 h = load(j >= 0 ? j : 0);
    x = h.x;
    v = j >= 0 ? h.y : 0.f;
    a = j >= 0 ? h.z : 0.f;
  }
  // sample j >= 0 known to exist
  __device__ __forceinline__ void get_in(int j, float &x, float &v, float &a) const {
    float4 h = load(j);
    x = h.x;
    v = h.y;
    a = h.z;
  }
};
using HistF32 = HistF32T<true>;
using HistF32RW = HistF32T<false>;
// The oscillator run's float32 mirror: sample j at slot (j & mask) of the dipole's row (mask = -1:
// every sample at its index; W - 1: a ring of W slots holding the samples a block can reach).
// Coherent loads: the run appends to the rows it reads.
struct HistF32Ring {
  const float4 *H;
  int mask;
  __device__ __forceinline__ void get(int j, float &x, float &v, float &a) const {
    float4 h = H[(j >= 0 ? j : 0) & mask];
    x = h.x;
    v = j >= 0 ? h.y : 0.f;
    a = j >= 0 ? h.z : 0.f;
  }
  __device__ __forceinline__ void get_in(int j, float &x, float &v, float &a) const {
    float4 h = H[j & mask];
    x = h.x;
    v = h.y;
    a = h.z;
  }
};
struct HistF64 {
  const double *d, *dd, *ddd;
  double sx, sv, sa;  // 1/(qL), 1/(qc), dt/(qc)
  __device__ __forceinline__ void get(int j, double &x, double &v, double &a) const {
    const int k = j >= 0 ? j : 0;
    x = d[k] * sx;
    v = j >= 0 ? dd[k] * sv : 0.0;
    a = j >= 0 ? ddd[k] * sa : 0.0;
  }
  __device__ __forceinline__ void get_in(int j, double &x, double &v, double &a) const { get(j, x, v, a); }
};

// Retarded state of one dipole charge at offset smu*X along the axis from the dipole centre, found
// exactly on the piecewise-linear history.
//   kb + xc: retarded time of the centre, in samples (xc small)
//   rn = |rho|, rp = rho . axis
// Out: X, V, Ac at the charge's own retarded time; delta = its distance minus rn.
// end_tol: a root up to this many samples past the last sample is taken at the last sample.
template <typename T, typename Hist>
__device__ __forceinline__ int dip_charge_solve(const Hist &H, int S, int kb, T xc, T rn, T rp, T smu, T &X, T &V,
                                                T &Ac, T &delta, T end_tol = T(kEndTol)) {
  if (!(fabs(xc) < T(1e6))) return PC_ERR_NOCONV;
  T fl;
  int kc = Num<T>::floor_int(xc, fl);
  T thc = xc - fl;
  int j = kb + kc;
  // first-order estimate of the charge's delay offset picks its segment
  {
    T hx, hv, ha;
    H.get(j < S ? j : S - 1, hx, hv, ha);
    T d0 = (rn > T(0)) ? -smu * hx * Num<T>::div(rp, rn) : T(0);
    T fs;
    int st = Num<T>::floor_int(thc - d0, fs);
    j += st;
    thc -= fs;
  }
  for (int it = 0; it < 6; ++it) {
    if (j > S - 2) {
      // past the end: solve on the last segment extended; a root up to kEndTol past the last
      // sample is clamped to it, a later one is a history error
      if (j - (S - 2) > 1000) return PC_ERR_HISTORY;
      thc += (T)(j - (S - 2));
      j = S - 2;
    }
    T x0, v0, a0, x1, v1, a1;
    H.get(j, x0, v0, a0);
    if (j < 0) {  // static segment
      x1 = x0;
      v1 = v0;
      a1 = a0;
    } else {
      H.get(j + 1, x1, v1, a1);
    }
    const T dx = x1 - x0;
    const T sc = smu * (x0 + thc * dx);
    const T w = smu * dx;
    const T A = T(1) - w * w;
    const T B = rn - w * (rp - sc);
    const T C = sc * (T(2) * rp - sc);
    const T sq = Num<T>::sqrt0(fmax(B * B - A * C, T(0)));
    const T dl = (B > T(0)) ? -Num<T>::div(C, B + sq) : Num<T>::div(-B + sq, A);
    T th = thc - dl;
    // a root this far outside the segment is taken at its end (the neighbouring segment's value
    // there differs by that fraction of a sample times the history's second difference); float32
    // roots carry ~1e-6 sample of rounding, float64 ones ~1e-12
    const T edge = sizeof(T) == sizeof(float) ? T(1e-4) : T(1e-12);
    const bool ok = (j < 0) ? ((T)j + th <= edge)
                            : (th >= -edge && (th <= T(1) + edge || (j == S - 2 && th <= T(1) + end_tol)) &&
                               (j < S - 2 || th <= T(1) + end_tol));
    if (ok) {
      th = fmin(fmax(th, T(0)), T(1));
      X = x0 + th * dx;
      V = v0 + th * (v1 - v0);
      Ac = a0 + th * (a1 - a0);
      delta = dl;
      return 0;
    }
    if (!(fabs(th) < T(1e6))) return PC_ERR_NOCONV;
    if (j == S - 2 && th > T(1)) return PC_ERR_HISTORY;
    T fs;
    int st = Num<T>::floor_int(th, fs);
    j += st;
    thc -= fs;
  }
  return PC_ERR_NOCONV;
}

// Both charges of a dipole from their centre's segment j (samples x0.. at j, x1.. at j+1, the
// centre at fraction thc), the segment extended linearly when a charge's retarded time falls just
// outside it.  Returns false when an offset exceeds kExtrap samples; the caller then solves each
// charge with dip_charge_solve.
// first/last: segment j is the first (0) or the last (S-2) of the history, whose ends may not be
// extended (the history is static before sample 0 and unknown after the last sample).
template <typename T>
__device__ __forceinline__ bool dip_pair_states(T x0, T v0, T a0, T x1, T v1, T a1, T thc, T rn, T rp, T mup, T mum,
                                                bool first, bool last, T &Xp, T &Vp, T &Ap, T &dp, T &Xm, T &Vm,
                                                T &Am, T &dm) {
  const T dx = x1 - x0, dv = v1 - v0, da = a1 - a0;
  const T Xc = x0 + thc * dx;
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const T smu = c == 0 ? mup : -mum;
    const T sc = smu * Xc, w = smu * dx;
    const T A = T(1) - w * w;
    const T B = rn - w * (rp - sc);
    const T C = sc * (T(2) * rp - sc);
    T dl;
    if constexpr (sizeof(T) == sizeof(float)) {
      // away from the charge |A C| << B^2 and the smaller root -C / (B + sqrt(B^2 - A C)) is
      // -(C / 2B) (1 + eps/4 + eps^2/8 + O(eps^3)), eps = A C / B^2: below 1e-7 relative for
      // |eps| < 1e-2; other pairs take the exact per-charge solve
      const T r = Num<T>::rcp(B);
      const T h = T(0.5) * C * r;
      const T eps = A * C * r * r;
      dl = -(h + h * eps * (T(0.25) + T(0.125) * eps));
      ok = ok && B > T(0) && fabs(eps) < T(1e-2);
    } else {
      const T sq = Num<T>::sqrt0(fmax(B * B - A * C, T(0)));
      dl = (B > T(0)) ? -Num<T>::div(C, B + sq) : Num<T>::div(-B + sq, A);
    }
    const T th = thc - dl;
    ok = ok && th >= (first ? T(0) : T(-kExtrap)) && th <= T(1) + (last ? T(kEndTol) : T(kExtrap));
    const T X = x0 + th * dx, V = v0 + th * dv, Ac = a0 + th * da;
    if (c == 0) {
      Xp = X;
      Vp = V;
      Ap = Ac;
      dp = dl;
    } else {
      Xm = X;
      Vm = V;
      Am = Ac;
      dm = dl;
    }
  }
  return ok;
}

// Fast form of dip_pair_states for the float32 inner loop: segment j interior to the history
// (1 <= j <= S-3, checked by the caller), the series root only, and one combined test.  Returns
// false when a charge's root leaves [-kExtrap, 1 + kExtrap] of the segment or the series does not
// apply (|eps| >= 1e-2, which also covers B <= 0: B is positive unless the point lies within about
// 1e-3 sample of the dipole centre, where |eps| is large); NaN inputs fail the tests as well.
// The two charges run side by side in the lanes of float2 operations (packed FFMA2/FMUL2/FADD2:
// one instruction issue for both charges).
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
// th_mid, th_half: the roots must lie within th_mid +- th_half of the segment (the field kernel's
// interior segments: 0.5 +- (0.5 + kExtrap)).  The tests are written so that a NaN fails them.
__device__ __forceinline__ bool dip_pair_states_fast(float x0, float v0, float a0, float x1, float v1, float a1,
                                                     float thc, float rn, float rp, float mup, float mum, float2 &X,
                                                     float2 &V, float2 &Ac, float2 &dl, float th_mid = 0.5f,
                                                     float th_half = 0.5f + kExtrap) {
  const float dx = x1 - x0, dv = v1 - v0, da = a1 - a0;
  const float Xc = x0 + thc * dx;
  const float2 smu = make_float2(mup, -mum);  // (positive charge, negative charge)
  const float2 sc = __fmul2_rn(smu, f2(Xc));
  const float2 w = __fmul2_rn(smu, f2(dx));
  const float2 nw = make_float2(-w.x, -w.y), nsc = make_float2(-sc.x, -sc.y);
  const float2 A = __ffma2_rn(nw, w, f2(1.f));                       // 1 - w^2
  const float2 B = __ffma2_rn(nw, __fadd2_rn(f2(rp), nsc), f2(rn));  // rn - w (rp - sc)
  const float2 C = __fmul2_rn(sc, __ffma2_rn(f2(2.f), f2(rp), nsc));  // sc (2 rp - sc)
  const float2 r = make_float2(__fdividef(1.f, B.x), __fdividef(1.f, B.y));
  const float2 Cr = __fmul2_rn(C, r);
  const float2 h = __fmul2_rn(Cr, f2(0.5f));
  const float2 eps = __fmul2_rn(__fmul2_rn(A, Cr), r);
  const float2 poly = __ffma2_rn(eps, f2(0.125f), f2(0.25f));
  const float2 ndl = __ffma2_rn(h, __fmul2_rn(eps, poly), h);  // -delta
  const float2 th = __fadd2_rn(f2(thc), ndl);
  X = __ffma2_rn(th, f2(dx), f2(x0));
  V = __ffma2_rn(th, f2(dv), f2(v0));
  Ac = __ffma2_rn(th, f2(da), f2(a0));
  dl = make_float2(-ndl.x, -ndl.y);
  const float2 td = __fadd2_rn(th, f2(-th_mid));
  return fabsf(td.x) <= th_half && fabsf(td.y) <= th_half && fabsf(eps.x) + fabsf(eps.y) < 1e-2f;
}

// The driving-field part of dipole_pair_fast: p_i . E of the pair, given r . p_i (rpi) and
// p_j . p_i (ppi), in the units of dipole_pair (E = C_a a + C_p p_j summed over the two charges).
__device__ __forceinline__ float dipole_drive_fast(float rn, float rp, float mup, float mum, float qs, float2 X,
                                                   float2 V, float2 Ac, float2 dl, float rpi, float ppi) {
  const float2 mu2 = make_float2(mup, -mum);
  const float2 s = __fmul2_rn(mu2, X);
  const float2 v = __fmul2_rn(mu2, V);
  const float2 al = __fmul2_rn(mu2, Ac);
  const float ds = mup * X.x + mum * X.y, dv = mup * V.x + mum * V.y, da = mup * Ac.x + mum * Ac.y;
  const float2 R = __fadd2_rn(f2(rn), dl);
  const float dR = dl.x - dl.y;
  const float2 ap = __fadd2_rn(f2(rp), make_float2(-s.x, -s.y));
  const float2 Ru = __ffma2_rn(make_float2(-v.x, -v.y), ap, R);
  const float dRu = dR - (dv * ap.x - v.y * ds);
  const float2 i = make_float2(__fdividef(1.f, Ru.x), __fdividef(1.f, Ru.y));
  const float2 i2 = __fmul2_rn(i, i);
  const float2 i3 = __fmul2_rn(i2, i);
  const float di = -dRu * i.y * i.x;
  const float di2 = di * (i.x + i.y);
  const float di3 = di * (i2.x + i.x * i.y + i2.y);
  const float v0 = v.y, a0 = al.y, R0 = R.y;
  const float G0 = 1.f - v0 * v0 + a0 * ap.y;
  const float dG = -dv * (v.x + v0) + da * ap.x - a0 * ds;
  const float G1 = G0 + dG;
  const float2 Ca = __fmul2_rn(make_float2(G1, G0), i3);
  const float dCa = dG * i3.x + G0 * di3;
  const float P0 = R0 * v0 * G0;
  const float dP = dR * v.x * G1 + R0 * (dv * G1 + v0 * dG);
  const float Q0 = a0 * R0, dQ = da * R.x + a0 * dR;
  const float dCp = -(dP * i3.x + P0 * di3) - (dQ * i2.x + Q0 * di2);
  const float2 Cs = __fmul2_rn(Ca, s);
  const float ep = dCp - (Cs.x - Cs.y);
  return qs * (dCa * rpi + ep * ppi);
}

// dipole_pair (CHECK_REX = false) for the float32 fast path with both charges in float2 lanes,
// (positive, negative), and the ten outputs in five packed accumulators:
//   P[0] = (E_x, E_y), P[1] = (B_x, B_y), P[2] = (A_x, A_y), P[3] = (E_z, B_z), P[4] = (A_z, phi).
// Same algebra and units as dipole_pair.
template <int KIND>
__device__ __forceinline__ void dipole_pair_fast(float2 rxy, float rz, float rn, float2 pxy, float pz, float rp,
                                                 float mup, float mum, float qs, float2 X, float2 V, float2 Ac,
                                                 float2 dl, float2 (&P)[5]) {
  const float2 mu2 = make_float2(mup, -mum);
  const float2 s = __fmul2_rn(mu2, X);   // (s1, s0): charge offsets along the axis
  const float2 v = __fmul2_rn(mu2, V);   // (v1, v0)
  const float2 al = __fmul2_rn(mu2, Ac);  // (a1, a0)
  // the separations of the two charges' offsets, velocities and accelerations: differences of the
  // products above (mup X.x - (-mum X.y)), one add each
  const float ds = s.x - s.y, dv = v.x - v.y, da = al.x - al.y;
  const float2 R = __fadd2_rn(f2(rn), dl);  // (R1, R0)
  const float dR = dl.x - dl.y;
  const float2 ap = __fadd2_rn(f2(rp), make_float2(-s.x, -s.y));  // (ap1, ap0)
  const float2 Ru = __ffma2_rn(make_float2(-v.x, -v.y), ap, R);   // (Ru1, Ru0)
  const float dRu = dR - (dv * ap.x - v.y * ds);
  const float2 i = make_float2(__fdividef(1.f, Ru.x), __fdividef(1.f, Ru.y));  // (i1, i0)
  const float2 i2 = __fmul2_rn(i, i);
  const float2 i3 = __fmul2_rn(i2, i);
  const float ixy = i.x * i.y;  // formed once for di and di3
  const float di = -dRu * ixy;
  const float di2 = di * (i.x + i.y);
  const float di3 = di * (i2.x + ixy + i2.y);
  const float v0 = v.y, a0 = al.y, ap0 = ap.y, R0 = R.y;
  float G0 = 0.f, dG = 0.f;
  if (KIND != PC_RADIATION) {
    G0 += 1.f - v0 * v0;
    dG += -dv * (v.x + v0);
  }
  if (KIND != PC_COULOMB) {
    G0 += a0 * ap0;
    dG += da * ap.x - a0 * ds;
  }
  const float G1 = G0 + dG;
  const float2 Ca = __fmul2_rn(make_float2(G1, G0), i3);  // (Ca1, Ca0)
  const float dCa = dG * i3.x + G0 * di3;
  const float vG0 = v0 * G0;  // formed once for P0 and dBc
  const float P0 = R0 * vG0;
  const float dvG = dv * G1 + v0 * dG;
  const float dP = dR * v.x * G1 + R0 * dvG;
  float dCp = -(dP * i3.x + P0 * di3);
  float dBc = -(dvG * i3.x + vG0 * di3);
  if (KIND != PC_COULOMB) {
    const float Q0 = a0 * R0, dQ = da * R.x + a0 * dR;
    dCp -= dQ * i2.x + Q0 * di2;
    dBc -= da * i2.x + a0 * di2;
  }
  const float2 Cs = __fmul2_rn(Ca, s);
  const float ep = dCp - (Cs.x - Cs.y);
  const float cE = qs * dCa, cP = qs * ep, cB = qs * dBc;
  const float cx = rxy.y * pz - rz * pxy.y, cy = rz * pxy.x - rxy.x * pz, cz = rxy.x * pxy.y - rxy.y * pxy.x;
  const float dA = qs * (dv * i.x + v0 * di);
  P[0] = __ffma2_rn(f2(cE), rxy, P[0]);
  P[0] = __ffma2_rn(f2(cP), pxy, P[0]);
  P[1] = __ffma2_rn(f2(cB), make_float2(cx, cy), P[1]);
  P[2] = __ffma2_rn(f2(dA), pxy, P[2]);
  P[3] = __ffma2_rn(make_float2(cE, cB), make_float2(rz, cz), P[3]);
  P[3].x = fmaf(cP, pz, P[3].x);
  P[4] = __ffma2_rn(make_float2(dA, qs), make_float2(pz, di), P[4]);
}

// Net field q [F(x+) - F(x-)] of a dipole's two charges, added to acc[10] = (E, B, phi, A), in
// units of k_e e / L^2 (E), k_e e / (L^2 c) (B), k_e e / L (phi), k_e e / (L c) (A), qs = q / e.
// Per charge: E = C_a a + C_p p, B = (C_p / R) (rho x p), phi = 1/R_u, A = v p / R_u with
// a = rho - s p, R_u = R - v a.p, G = 1 - v^2 + alpha a.p, C_a = G / R_u^3,
// C_p = -R v G / R_u^3 - alpha R / R_u^2; the differences of C_a, C_p, C_p / R, 1/R_u and v/R_u
// are formed from the differences of their inputs (dR = delta+ - delta-, ds, dv, dalpha).
// CHECK_REX = false: the caller guarantees both charges farther than rex from the point.
template <int KIND, typename T, bool CHECK_REX = true>
__device__ __forceinline__ void dipole_pair(T rx, T ry, T rz, T rn, T px, T py, T pz, T rp, T mup, T mum, T qs, T Xp,
                                            T Vp, T Ap, T dp, T Xm, T Vm, T Am, T dm, T rex, T *acc,
                                            uint8_t &mask) {
  // charge 1 = positive (offset +mup X), charge 0 = negative (offset -mum X)
  const T s1 = mup * Xp, s0 = -mum * Xm, ds = mup * Xp + mum * Xm;
  const T v1 = mup * Vp, v0 = -mum * Vm, dv = mup * Vp + mum * Vm;
  const T a1 = mup * Ap, a0 = -mum * Am, da = mup * Ap + mum * Am;
  const T R0 = rn + dm, dR = dp - dm, R1 = R0 + dR;
  if (CHECK_REX && (R0 <= rex || R1 <= rex)) {
    mask = 1;
    // one charge coincides with the point: add the other one alone
    const bool use1 = R1 > rex;
    if (!(R0 > rex) && !use1) return;
    const T s = use1 ? s1 : s0, v = use1 ? v1 : v0, al = use1 ? a1 : a0, R = use1 ? R1 : R0;
    const T sign = use1 ? qs : -qs;
    const T ap = rp - s;
    const T Ru = R - v * ap;
    const T i1 = Num<T>::rcp(Ru);
    const T i2 = i1 * i1, i3 = i2 * i1;
    T G = T(0), Q = T(0);
    if (KIND != PC_RADIATION) G += T(1) - v * v;
    if (KIND != PC_COULOMB) {
      G += al * ap;
      Q = al;
    }
    const T Ca = G * i3;
    const T Cp = -R * v * G * i3 - Q * R * i2;
    const T Bc = -v * G * i3 - Q * i2;
    const T ax_ = rx - s * px, ay_ = ry - s * py, az_ = rz - s * pz;
    acc[0] += sign * (Ca * ax_ + Cp * px);
    acc[1] += sign * (Ca * ay_ + Cp * py);
    acc[2] += sign * (Ca * az_ + Cp * pz);
    const T cx = ry * pz - rz * py, cy = rz * px - rx * pz, cz = rx * py - ry * px;
    acc[3] += sign * Bc * cx;
    acc[4] += sign * Bc * cy;
    acc[5] += sign * Bc * cz;
    acc[6] += sign * i1;
    const T va = sign * v * i1;
    acc[7] += va * px;
    acc[8] += va * py;
    acc[9] += va * pz;
    return;
  }
  const T ap0 = rp - s0, ap1 = rp - s1, dap = -ds;
  const T Ru0 = R0 - v0 * ap0;
  const T dRu = dR - (dv * ap1 + v0 * dap);
  const T Ru1 = Ru0 + dRu;
  const T i0 = Num<T>::rcp(Ru0), i1 = Num<T>::rcp(Ru1);
  const T di = -dRu * i0 * i1;
  const T i02 = i0 * i0, i12 = i1 * i1;
  const T i03 = i02 * i0, i13 = i12 * i1;
  const T di2 = di * (i0 + i1);
  const T di3 = di * (i12 + i1 * i0 + i02);
  T G0 = T(0), dG = T(0);
  if (KIND != PC_RADIATION) {
    G0 += T(1) - v0 * v0;
    dG += -dv * (v1 + v0);
  }
  if (KIND != PC_COULOMB) {
    G0 += a0 * ap0;
    dG += da * ap1 + a0 * dap;
  }
  const T G1 = G0 + dG;
  const T Ca0 = G0 * i03, Ca1 = G1 * i13;
  const T dCa = dG * i13 + G0 * di3;
  // C_p = -R v G i^3 - alpha R i^2 ; B coefficient C_p / R = -v G i^3 - alpha i^2
  const T P0 = R0 * v0 * G0;
  const T dP = dR * v1 * G1 + R0 * (dv * G1 + v0 * dG);
  T dCp = -(dP * i13 + P0 * di3);
  const T dvG = dv * G1 + v0 * dG;
  T dBc = -(dvG * i13 + v0 * G0 * di3);
  if (KIND != PC_COULOMB) {
    const T Q0 = a0 * R0, dQ = da * R1 + a0 * dR;
    dCp -= dQ * i12 + Q0 * di2;
    dBc -= da * i12 + a0 * di2;
  }
  const T ep = dCp - (Ca1 * s1 - Ca0 * s0);
  acc[0] += qs * (dCa * rx + ep * px);
  acc[1] += qs * (dCa * ry + ep * py);
  acc[2] += qs * (dCa * rz + ep * pz);
  const T cx = ry * pz - rz * py, cy = rz * px - rx * pz, cz = rx * py - ry * px;
  acc[3] += qs * dBc * cx;
  acc[4] += qs * dBc * cy;
  acc[5] += qs * dBc * cz;
  acc[6] += qs * di;
  const T dA = qs * (dv * i1 + v0 * di);
  acc[7] += dA * px;
  acc[8] += dA * py;
  acc[9] += dA * pz;
}

// Exact per-charge roots of both charges, kept out of line: it only runs for large charge offsets
// (or near pairs), and inlining it would cost the common path registers.
template <typename T, typename Hist>
__device__ __noinline__ int dip_pair_exact(const Hist &H, int S, int kb, T xc, T rn, T rp, T mup, T mum, T &Xp, T &Vp,
                                           T &Ap, T &dp, T &Xm, T &Vm, T &Am, T &dm, T end_tol = T(kEndTol)) {
  const int e1 = dip_charge_solve<T>(H, S, kb, xc, rn, rp, mup, Xp, Vp, Ap, dp, end_tol);
  const int e2 = dip_charge_solve<T>(H, S, kb, xc, rn, rp, -mum, Xm, Vm, Am, dm, end_tol);
  return e1 ? e1 : e2;
}

// Retarded states of both charges of a dipole: their centre's segment extended when possible,
// exact per-charge roots otherwise (or when `exact`).  Returns 0 or an error code.
template <typename T, typename Hist>
__device__ __forceinline__ int dipole_states(const Hist &H, int S, int kb, T xc, T rn, T rp, T mup, T mum, bool exact,
                                             T &Xp, T &Vp, T &Ap, T &dp, T &Xm, T &Vm, T &Am, T &dm) {
  bool done = false;
  if (!exact && fabs(xc) < T(1e6)) {
    T fl;
    const int kc = Num<T>::floor_int(xc, fl);
    const T thc = xc - fl;
    const int j = kb + kc;
    if (j >= 0 && j <= S - 2) {
      T x0, v0, a0, x1, v1, a1;
      H.get_in(j, x0, v0, a0);
      H.get_in(j + 1, x1, v1, a1);
      done = dip_pair_states<T>(x0, v0, a0, x1, v1, a1, thc, rn, rp, mup, mum, j == 0, j == S - 2, Xp, Vp, Ap, dp,
                                Xm, Vm, Am, dm);
    }
  }
  if (!done) return dip_pair_exact<T, Hist>(H, S, kb, xc, rn, rp, mup, mum, Xp, Vp, Ap, dp, Xm, Vm, Am, dm);
  return 0;
}

// Cancellation ratio of a dipole's near field: its float32 evaluation works with terms of the size
// of the moment at the retarded time and its rate and acceleration, (|ds| + R |dv| + R^2 |da|),
// while the near field follows the moment at the present time, ds + R dv + R^2 da / 2, which
// passes through zero.  The ratio bounds the loss of relative accuracy of the difference form.
template <typename T>
__device__ __forceinline__ T dipole_cancellation(T rn, T mup, T mum, T Xp, T Vp, T Ap, T Xm, T Vm, T Am) {
  const T ds = mup * Xp + mum * Xm, dv = mup * Vp + mum * Vm, da = mup * Ap + mum * Am;
  const T num = fabs(ds) + rn * fabs(dv) + rn * rn * fabs(da);
  const T den = fabs(ds + rn * dv + T(0.5) * rn * rn * da);
  return Num<T>::div(num, fmax(den, T(1e-30) * num + T(1e-38)));
}

// Net field of a dipole pair in T precision: retarded states then the difference form.
template <int KIND, typename T, typename Hist>
__device__ __forceinline__ int dipole_net(const Hist &H, int S, int kb, T xc, T rx, T ry, T rz, T rn, T px, T py, T pz,
                                          T rp, T mup, T mum, T qs, T rex, bool exact, T *acc, uint8_t &mask) {
  T Xp, Vp, Ap, dp, Xm, Vm, Am, dm;
  const int e = dipole_states<T, Hist>(H, S, kb, xc, rn, rp, mup, mum, exact, Xp, Vp, Ap, dp, Xm, Vm, Am, dm);
  if (e) return e;
  dipole_pair<KIND, T>(rx, ry, rz, rn, px, py, pz, rp, mup, mum, qs, Xp, Vp, Ap, dp, Xm, Vm, Am, dm, rex, acc, mask);
  return 0;
}

}  // namespace pc
