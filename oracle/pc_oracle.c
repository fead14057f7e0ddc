/*
 * FP64 CPU oracle for the Lienard-Wiechert hot path of PyCharge (arXiv 2107.12437).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py may load this file.  It shares no code, header, table or
 * constant generator with the CUDA library; it is plain, slow and literal on purpose.
 *
 * What it computes, and where the paper defines it:
 *   - retarded time t' = t - R(t')/c  (Sec. 2.1, Eq. ret_t), solved here by plain bisection on the
 *     delay tau = t - t' (the paper uses a secant method; both converge to the unique root of the
 *     same piecewise-linear trajectory, Sec. 3.1: discrete histories are linearly interpolated);
 *   - Lienard-Wiechert potentials and fields in Jackson's notation (Sec. 2.1, Eqs. V, A, E, B and
 *     the Coulomb / radiation split Eqs. ECoulomb, Eradiation).  Reading of Eq. A: the printed
 *     mu0 q/(4 pi) [beta/(kappa R)] lacks a factor c; we use A = mu0 q c beta / (4 pi kappa R),
 *     which equals (v/c^2) Phi.  A second, independent evaluation in Griffiths' notation
 *     (footnote to Sec. 2.1) is exposed for a consistency check;
 *   - superposition over all charges (Sec. 2.2);
 *   - dipole charges from the dipole moment (Sec. 2.3, Eqs. eff_mass, r_1, r_2), static for t <= 0
 *     (Sec. 3.2);
 *   - the same field sum with every intermediate in binary128 (orc_fields_x), the reference for
 *     points where the +-q charges of dipoles cancel by many digits;
 *   - the Lorentz-oscillator run of Algorithm 1 with the equation of motion Eq. LO_equation,
 *     RK4 in time, driving field E_d = p . E at the dipole origin from all other dipoles (Sec. 2.3,
 *     Sec. 3.2), energy Eq. dipoleE, velocity guard (Sec. 3.2, default c/100).
 *
 * Units: SI throughout, all arithmetic in double precision.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA 2018 exact / recommended values */
#define ORC_C 299792458.0
#define ORC_EPS0 8.8541878128e-12
#define ORC_PI 3.14159265358979323846

/* oracle status codes (independent of the library's codes) */
enum {
  ORC_OK = 0,
  ORC_ERR_ARG = 1,
  ORC_ERR_HISTORY = 2,   /* retarded time before the first sample (no static extension) or after the last */
  ORC_ERR_VELOCITY = 3,  /* a dipole charge exceeded v_max */
  ORC_ERR_CAUSALITY = 4, /* a stage time needs history that is not computed yet */
  ORC_ERR_NOCONV = 5
};

/* field kinds (Sec. 3.2: calculate_E/B select total, Coulomb or radiation) */
enum { ORC_TOTAL = 0, ORC_COULOMB = 1, ORC_RADIATION = 2 };

typedef struct {
  /* point charges with sampled trajectories: sample k is at time t0 + k dt */
  int32_t M;
  int64_t S;
  double t0, dt;
  const double *q;             /* [M] */
  const double *pos, *vel, *acc; /* [M][S][3] */
  int32_t static_before;       /* 1: at rest at sample 0 for t < t0; 0: error */
  /* dipoles (Lorentz oscillators): moment history along a fixed unit axis */
  int32_t N;
  int64_t Sd;                  /* samples per dipole */
  double t0d, dtd;
  const double *origin;        /* [N][3] centre of mass R */
  const double *axis;          /* [N][3] unit polarisation axis */
  const double *qd, *m1, *m2;  /* [N] charge magnitude and the two masses */
  const double *d, *d_dot, *d_ddot; /* [N][Sd] moment along axis, C m, and its derivatives */
  int64_t last_valid;          /* dipole samples 0..last_valid are known; -1 = all */
  /* moving dipoles (Sec. 4.3): origin position, velocity and acceleration at the half steps
   * t0d + h dtd / 2, h = 0 .. 2 Sd - 2, [N][2 Sd - 1][3]; NULL for fixed origins */
  const double *org_pos, *org_vel, *org_acc;
} orc_sources;

static inline double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void cross3(const double *a, const double *b, double *o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

int orc_n_charges(const orc_sources *s) { return s->M + 2 * s->N; }

/*
 * State (charge, position, velocity, acceleration) of charge c at time tp.
 * Charges 0..M-1 are the sampled ones; charge M + 2j is the positive charge of dipole j (Eq. r_1),
 * M + 2j + 1 its negative charge (Eq. r_2).  Between samples every quantity is linearly
 * interpolated (Sec. 3.1).
 */
static int charge_state(const orc_sources *s, int c, double tp, double *qc, double p[3], double v[3], double a[3]) {
  if (c < s->M) {
    const double *P = s->pos + (int64_t)c * s->S * 3;
    const double *V = s->vel + (int64_t)c * s->S * 3;
    const double *A = s->acc + (int64_t)c * s->S * 3;
    *qc = s->q[c];
    double x = (tp - s->t0) / s->dt;
    /* the edge times t0 and t0 + (S-1) dt are rounded doubles: snap within 1e-9 step of an edge */
    if (x < 0.0 && x > -1e-9) x = 0.0;
    if (x > (double)(s->S - 1) && x < (double)(s->S - 1) + 1e-9) x = (double)(s->S - 1);
    if (x < 0.0) {
      if (!s->static_before) return ORC_ERR_HISTORY;
      for (int i = 0; i < 3; ++i) { p[i] = P[i]; v[i] = 0.0; a[i] = 0.0; }
      return ORC_OK;
    }
    int64_t k = (int64_t)floor(x);
    if (k >= s->S - 1) {
      if (x > (double)(s->S - 1)) return ORC_ERR_HISTORY;
      k = s->S - 2; /* exactly at the last sample */
    }
    double th = x - (double)k;
    for (int i = 0; i < 3; ++i) {
      p[i] = P[k * 3 + i] + th * (P[(k + 1) * 3 + i] - P[k * 3 + i]);
      v[i] = V[k * 3 + i] + th * (V[(k + 1) * 3 + i] - V[k * 3 + i]);
      a[i] = A[k * 3 + i] + th * (A[(k + 1) * 3 + i] - A[k * 3 + i]);
    }
    return ORC_OK;
  }
  int j = (c - s->M) / 2;
  int neg = (c - s->M) % 2;
  double m1 = s->m1[j], m2 = s->m2[j], q = s->qd[j];
  const double *u = s->axis + 3 * j;
  const double *R = s->origin + 3 * j;
  double dd, dv, da;
  double x = (tp - s->t0d) / s->dtd;
  const double *D = s->d + (int64_t)j * s->Sd;
  const double *DV = s->d_dot + (int64_t)j * s->Sd;
  const double *DA = s->d_ddot + (int64_t)j * s->Sd;
  /* a moving origin: the history holds the whole-step samples (even half-step indices), linearly
   * interpolated like every other history (Sec. 3.1); at rest at its first position for t <= t0 */
  double Rm[3] = {R[0], R[1], R[2]}, Rv[3] = {0.0, 0.0, 0.0}, Ra[3] = {0.0, 0.0, 0.0};
  const int64_t H = 2 * s->Sd - 1;
  if (s->org_pos) {
    const double *OP = s->org_pos + (int64_t)j * H * 3;
    for (int i = 0; i < 3; ++i) Rm[i] = OP[i];
  }
  if (x <= 0.0) {
    /* stationary dipole moment for t <= t0 (Sec. 3.2) */
    dd = D[0]; dv = 0.0; da = 0.0;
  } else {
    int64_t last = (s->last_valid >= 0) ? s->last_valid : (s->Sd - 1);
    if (x > (double)last && x < (double)last + 1e-9) x = (double)last;
    int64_t k = (int64_t)floor(x);
    if (k >= last) {
      if (x > (double)last) return (s->last_valid >= 0) ? ORC_ERR_CAUSALITY : ORC_ERR_HISTORY;
      k = last - 1;
    }
    double th = x - (double)k;
    dd = D[k] + th * (D[k + 1] - D[k]);
    dv = DV[k] + th * (DV[k + 1] - DV[k]);
    da = DA[k] + th * (DA[k + 1] - DA[k]);
    if (s->org_pos) {
      const double *OP = s->org_pos + ((int64_t)j * H + 2 * k) * 3;
      const double *OV = s->org_vel + ((int64_t)j * H + 2 * k) * 3;
      const double *OA = s->org_acc + ((int64_t)j * H + 2 * k) * 3;
      for (int i = 0; i < 3; ++i) {
        Rm[i] = OP[i] + th * (OP[6 + i] - OP[i]);
        Rv[i] = OV[i] + th * (OV[6 + i] - OV[i]);
        Ra[i] = OA[i] + th * (OA[6 + i] - OA[i]);
      }
    }
  }
  /* r_dip = d / q along the axis; r_1 = R + m2/(m1+m2) r_dip, r_2 = R - m1/(m1+m2) r_dip */
  double w = neg ? -m1 / (m1 + m2) : m2 / (m1 + m2);
  *qc = neg ? -q : q;
  for (int i = 0; i < 3; ++i) {
    p[i] = Rm[i] + w * (dd / q) * u[i];
    v[i] = Rv[i] + w * (dv / q) * u[i];
    a[i] = Ra[i] + w * (da / q) * u[i];
  }
  return ORC_OK;
}

/*
 * Retarded time t' of charge c seen from r at time t: the root of
 * g(t') = c (t - t') - |r - r_c(t')|  (Eq. ret_t).  g(t) <= 0 and g is strictly decreasing in t' while
 * the charge is slower than light, so plain bisection on a bracket [t'_lo, t'_hi] with
 * g(t'_lo) >= 0 >= g(t'_hi) converges to the unique root; it stops when the bracket cannot shrink.
 * The bracket is kept inside the stored history: before the first sample a charge either rests at
 * its first position (static extension) or the call fails with ORC_ERR_HISTORY; a root after the
 * last known sample fails with ORC_ERR_HISTORY, or ORC_ERR_CAUSALITY during a dipole run.
 */
static double g_at(const orc_sources *s, int c, double t, const double r[3], double tp, int *st) {
  double qc, p[3], v[3], a[3];
  *st = charge_state(s, c, tp, &qc, p, v, a);
  double D[3] = {r[0] - p[0], r[1] - p[1], r[2] - p[2]};
  return ORC_C * (t - tp) - sqrt(dot3(D, D));
}

int orc_retarded_time(const orc_sources *s, int c, double t, const double r[3], double *tp_out) {
  int st;
  int sampled = (c < s->M);
  double t_first = sampled ? s->t0 : s->t0d;
  double t_last;
  if (sampled) t_last = s->t0 + (double)(s->S - 1) * s->dt;
  else t_last = s->t0d + (double)((s->last_valid >= 0) ? s->last_valid : (s->Sd - 1)) * s->dtd;
  int err_late = (!sampled && s->last_valid >= 0) ? ORC_ERR_CAUSALITY : ORC_ERR_HISTORY;
  double hi = (t < t_last) ? t : t_last;
  double lo;
  if (sampled && !s->static_before) {
    lo = t_first;
    if (lo > hi) return ORC_ERR_HISTORY;
    double g = g_at(s, c, t, r, lo, &st);
    if (st) return st;
    if (g < 0.0) return ORC_ERR_HISTORY;   /* the root precedes the first sample */
  } else {
    /* before the first sample the charge rests at its first position */
    double qc, p[3], v[3], a[3];
    st = charge_state(s, c, (t < t_first) ? t : t_first, &qc, p, v, a);
    if (st) return st;
    double D[3] = {r[0] - p[0], r[1] - p[1], r[2] - p[2]};
    lo = t - sqrt(dot3(D, D)) / ORC_C * (1.0 + 1e-12) - 1e-30;
    if (lo > t_first) lo = t_first;
    if (lo > hi) lo = hi;
  }
  if (hi < t) {
    double g = g_at(s, c, t, r, hi, &st);
    if (st) return st;
    if (g > 0.0) return err_late;           /* the root lies after the last known sample */
    if (g == 0.0) { *tp_out = hi; return ORC_OK; }
  }
  for (int it = 0; it < 4000; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    double g = g_at(s, c, t, r, mid, &st);
    if (st) return st;
    if (g >= 0.0) lo = mid; else hi = mid;
  }
  *tp_out = 0.5 * (lo + hi);
  return ORC_OK;
}

int orc_retarded_delay(const orc_sources *s, int c, double t, const double r[3], double *tau_out) {
  double tp;
  int st = orc_retarded_time(s, c, t, r, &tp);
  if (st) return st;
  *tau_out = t - tp;
  return ORC_OK;
}

/*
 * Lienard-Wiechert fields and potentials of one charge, Jackson's notation (Eqs. V, A, E, B).
 * aR = r - r_p(t'), v and acc at t'.  Outputs are added into Ec (Coulomb E), Er (radiation E),
 * phi and A.
 */
static void lw_jackson(double q, const double aR[3], const double v[3], const double acc[3], double Ec[3],
                       double Er[3], double *phi, double A[3]) {
  double R = sqrt(dot3(aR, aR));
  double n[3] = {aR[0] / R, aR[1] / R, aR[2] / R};
  double beta[3] = {v[0] / ORC_C, v[1] / ORC_C, v[2] / ORC_C};
  double bdot[3] = {acc[0] / ORC_C, acc[1] / ORC_C, acc[2] / ORC_C};
  double kappa = 1.0 - dot3(n, beta);
  double b2 = dot3(beta, beta);
  double k = q / (4.0 * ORC_PI * ORC_EPS0);
  double nb[3] = {n[0] - beta[0], n[1] - beta[1], n[2] - beta[2]};
  double k3 = kappa * kappa * kappa;
  /* Coulomb term: (n - beta)(1 - beta^2) / (kappa^3 R^2) */
  for (int i = 0; i < 3; ++i) Ec[i] = k * nb[i] * (1.0 - b2) / (k3 * R * R);
  /* radiation term: n x ((n - beta) x beta_dot) / (c kappa^3 R) */
  double w[3], nw[3];
  cross3(nb, bdot, w);
  cross3(n, w, nw);
  for (int i = 0; i < 3; ++i) Er[i] = k * nw[i] / (ORC_C * k3 * R);
  *phi = k / (kappa * R);
  double mu0 = 1.0 / (ORC_EPS0 * ORC_C * ORC_C);
  for (int i = 0; i < 3; ++i) A[i] = mu0 * q * ORC_C / (4.0 * ORC_PI) * beta[i] / (kappa * R);
}

/*
 * The same field in Griffiths' notation: E = q/(4 pi eps0) R/(aR.u)^3 [(c^2 - v^2) u + aR x (u x acc)],
 * u = c n - v.  Used only to cross-check lw_jackson.
 */
void orc_lw_griffiths(double q, const double aR[3], const double v[3], const double acc[3], double E[3],
                      double B[3]) {
  double R = sqrt(dot3(aR, aR));
  double u[3];
  for (int i = 0; i < 3; ++i) u[i] = ORC_C * aR[i] / R - v[i];
  double Ru = dot3(aR, u);
  double f = q / (4.0 * ORC_PI * ORC_EPS0) * R / (Ru * Ru * Ru);
  double c2v2 = ORC_C * ORC_C - dot3(v, v);
  double ua[3], rua[3];
  cross3(u, acc, ua);
  cross3(aR, ua, rua);
  for (int i = 0; i < 3; ++i) E[i] = f * (c2v2 * u[i] + rua[i]);
  double n[3] = {aR[0] / R, aR[1] / R, aR[2] / R};
  double nE[3];
  cross3(n, E, nE);
  for (int i = 0; i < 3; ++i) B[i] = nE[i] / ORC_C;
}

void orc_lw_jackson(double q, const double aR[3], const double v[3], const double acc[3], double Ec[3], double Er[3],
                    double *phi, double A[3]) {
  lw_jackson(q, aR, v, acc, Ec, Er, phi, A);
}

/*
 * Fields at one point r and time t, summed over all charges except those of dipole `exclude`
 * (-1: none).  A charge closer than r_excl at its retarded position contributes nothing and sets
 * *mask.  Outputs are overwritten.
 */
static int fields_at(const orc_sources *s, const double r[3], double t, int kind, double r_excl, int exclude,
                     double E[3], double B[3], double *phi, double A[3], uint8_t *mask, double *scale) {
  int nc = orc_n_charges(s);
  for (int i = 0; i < 3; ++i) { E[i] = 0.0; B[i] = 0.0; A[i] = 0.0; }
  *phi = 0.0;
  *mask = 0;
  /* scale (optional, 8 values): sums over charges of |E_Coul,c| + |E_rad,c|, the same over c,
     |phi_c| and |A_c|; then |E|, |B|, |phi|, |A| summed over sources, a dipole's two charges
     counting as one source.  They measure how much the superposition cancels; they do not enter
     E, B, phi, A. */
  double src[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0}; /* running field of the current dipole: E, B, phi, A */
  if (scale) for (int i = 0; i < 8; ++i) scale[i] = 0.0;
  for (int c = 0; c < nc; ++c) {
    if (exclude >= 0 && c >= s->M && (c - s->M) / 2 == exclude) continue;
    double tp;
    int st = orc_retarded_time(s, c, t, r, &tp);
    if (st) return st;
    double qc, p[3], v[3], a[3];
    st = charge_state(s, c, tp, &qc, p, v, a);
    if (st) return st;
    double aR[3] = {r[0] - p[0], r[1] - p[1], r[2] - p[2]};
    double R = sqrt(dot3(aR, aR));
    if (R <= r_excl) {
      *mask = 1;
      if (scale && c >= s->M && (c - s->M) % 2 == 1) {
        scale[4] += sqrt(src[0] * src[0] + src[1] * src[1] + src[2] * src[2]);
        scale[5] += sqrt(src[3] * src[3] + src[4] * src[4] + src[5] * src[5]);
        scale[6] += fabs(src[6]);
        scale[7] += sqrt(src[7] * src[7] + src[8] * src[8] + src[9] * src[9]);
        for (int i = 0; i < 10; ++i) src[i] = 0.0;
      }
      continue;
    }
    double Ec[3], Er[3], ph, Ac[3];
    lw_jackson(qc, aR, v, a, Ec, Er, &ph, Ac);
    double Ek[3];
    for (int i = 0; i < 3; ++i)
      Ek[i] = (kind == ORC_COULOMB) ? Ec[i] : (kind == ORC_RADIATION) ? Er[i] : Ec[i] + Er[i];
    double n[3] = {aR[0] / R, aR[1] / R, aR[2] / R}, nE[3];
    cross3(n, Ek, nE);
    for (int i = 0; i < 3; ++i) {
      E[i] += Ek[i];
      B[i] += nE[i] / ORC_C; /* Eq. B */
      A[i] += Ac[i];
    }
    *phi += ph;
    if (scale) {
      /* E of a term is built from its Coulomb and radiation parts, and B = n x E / c of a nearly
         radial E is a small cross product: both round at (|E_Coul| + |E_rad|) of the term */
      double ecr = sqrt(dot3(Ec, Ec)) + sqrt(dot3(Er, Er));
      scale[0] += ecr;
      scale[1] += ecr / ORC_C;
      scale[2] += fabs(ph);
      scale[3] += sqrt(dot3(Ac, Ac));
      int dip = (c >= s->M);
      for (int i = 0; i < 3; ++i) { src[i] += Ek[i]; src[3 + i] += nE[i] / ORC_C; src[7 + i] += Ac[i]; }
      src[6] += ph;
      /* close the source after a point charge, or after the second charge of a dipole */
      if (!dip || ((c - s->M) % 2 == 1)) {
        scale[4] += sqrt(src[0] * src[0] + src[1] * src[1] + src[2] * src[2]);
        scale[5] += sqrt(src[3] * src[3] + src[4] * src[4] + src[5] * src[5]);
        scale[6] += fabs(src[6]);
        scale[7] += sqrt(src[7] * src[7] + src[8] * src[8] + src[9] * src[9]);
        for (int i = 0; i < 10; ++i) src[i] = 0.0;
      }
    }
  }
  return ORC_OK;
}

/*
 * Fields on P points at T times: E, B, A [T][P][3], phi [T][P], mask [T][P] (Sec. 2.2, Sec. 3.2).
 * scale (or NULL): [T][P][8] magnitude sums of the superposed terms, see fields_at.
 */
int orc_fields(const orc_sources *s, const double *points, int64_t P, const double *times, int32_t T, int32_t kind,
               double r_excl, double *E, double *B, double *phi, double *A, uint8_t *mask, double *scale,
               int32_t nthreads) {
  if (kind < 0 || kind > 2 || P < 0 || T < 0) return ORC_ERR_ARG;
  int status = ORC_OK;
  int64_t total = P * (int64_t)T;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
#endif
  for (int64_t idx = 0; idx < total; ++idx) {
    int64_t f = idx / P, pidx = idx % P;
    int st = fields_at(s, points + 3 * pidx, times[f], kind, r_excl, -1, E + 3 * idx, B + 3 * idx, phi + idx,
                       A + 3 * idx, mask + idx, scale ? scale + 8 * idx : NULL);
    if (st) {
#ifdef _OPENMP
#pragma omp critical
#endif
      if (status == ORC_OK) status = st;
    }
  }
  (void)nthreads;
  return status;
}

/*
 * Point charges on analytic trajectories r(t) (Sec. 2.2 and Sec. 3.1: the predefined trajectories
 * of the paper's stationary, oscillating, orbiting and linearly accelerating charges), with exact
 * velocity and acceleration.  par[12] per charge:
 *   0 stationary:   r0[3]
 *   1 oscillating:  r0[3], u[3] (unit), A, w, phi:        r = r0 + A cos(w t + phi) u
 *   2 circular:     c[3], e1[3], e2[3] (orthonormal), a, w, phi:  r = c + a (cos(w t + phi) e1 + sin(w t + phi) e2)
 *   3 accelerating: r0[3], v0[3], acc[3], ta:              r = r0 + v0 s + acc s^2 / 2 for s = t - ta >= 0,
 *                                                          r0 + v0 s before (uniform motion)
 */
static void param_state(int kind, const double *p, double t, double r[3], double v[3], double a[3]) {
  for (int i = 0; i < 3; ++i) { r[i] = p[i]; v[i] = 0.0; a[i] = 0.0; }
  if (kind == 1) {
    double ph = p[7] * t + p[8];
    for (int i = 0; i < 3; ++i) {
      r[i] = p[i] + p[6] * cos(ph) * p[3 + i];
      v[i] = -p[6] * p[7] * sin(ph) * p[3 + i];
      a[i] = -p[6] * p[7] * p[7] * cos(ph) * p[3 + i];
    }
  } else if (kind == 2) {
    double ph = p[10] * t + p[11], rad = p[9], w = p[10];
    for (int i = 0; i < 3; ++i) {
      r[i] = p[i] + rad * (cos(ph) * p[3 + i] + sin(ph) * p[6 + i]);
      v[i] = rad * w * (-sin(ph) * p[3 + i] + cos(ph) * p[6 + i]);
      a[i] = -rad * w * w * (cos(ph) * p[3 + i] + sin(ph) * p[6 + i]);
    }
  } else if (kind == 3) {
    double sdt = t - p[9];
    int on = sdt >= 0.0;
    for (int i = 0; i < 3; ++i) {
      r[i] = p[i] + p[3 + i] * sdt + (on ? 0.5 * p[6 + i] * sdt * sdt : 0.0);
      v[i] = p[3 + i] + (on ? p[6 + i] * sdt : 0.0);
      a[i] = on ? p[6 + i] : 0.0;
    }
  }
}

/* retarded time of a parametric charge: bisection on g(t') = c (t - t') - |r - r(t')| (Eq. ret_t),
   the lower end pushed back until g >= 0 */
static int param_retarded_time(int kind, const double *p, double t, const double r[3], double *tp_out) {
  double rc[3], v[3], a[3];
  param_state(kind, p, t, rc, v, a);
  double D[3] = {r[0] - rc[0], r[1] - rc[1], r[2] - rc[2]};
  double hi = t, lo = t - sqrt(dot3(D, D)) / ORC_C;
  double span = t - lo + 1e-30;
  for (int it = 0;; ++it) {
    param_state(kind, p, lo, rc, v, a);
    double E[3] = {r[0] - rc[0], r[1] - rc[1], r[2] - rc[2]};
    if (ORC_C * (t - lo) - sqrt(dot3(E, E)) >= 0.0) break;
    if (it >= 200) return ORC_ERR_NOCONV;
    span *= 2.0;
    lo = t - span;
  }
  for (int it = 0; it < 4000; ++it) {
    double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    param_state(kind, p, mid, rc, v, a);
    double E[3] = {r[0] - rc[0], r[1] - rc[1], r[2] - rc[2]};
    if (ORC_C * (t - mid) - sqrt(dot3(E, E)) >= 0.0) lo = mid;
    else hi = mid;
  }
  *tp_out = 0.5 * (lo + hi);
  return ORC_OK;
}

int orc_fields_param(int32_t M, const int32_t *kind, const double *q, const double *par, const double *points,
                     int64_t P, const double *times, int32_t T, int32_t fkind, double r_excl, double *E, double *B,
                     double *phi, double *A, uint8_t *mask, int32_t nthreads) {
  if (fkind < 0 || fkind > 2 || P < 0 || T < 0 || M < 0) return ORC_ERR_ARG;
  for (int c = 0; c < M; ++c)
    if (kind[c] < 0 || kind[c] > 3) return ORC_ERR_ARG;
  int status = ORC_OK;
  int64_t total = P * (int64_t)T;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
#endif
  for (int64_t idx = 0; idx < total; ++idx) {
    int64_t f = idx / P, pidx = idx % P;
    const double *r = points + 3 * pidx;
    double t = times[f];
    double *e = E + 3 * idx, *b = B + 3 * idx, *aa = A + 3 * idx;
    for (int i = 0; i < 3; ++i) { e[i] = 0.0; b[i] = 0.0; aa[i] = 0.0; }
    phi[idx] = 0.0;
    mask[idx] = 0;
    for (int c = 0; c < M; ++c) {
      double tp;
      int st = param_retarded_time(kind[c], par + 12 * c, t, r, &tp);
      if (st) {
#ifdef _OPENMP
#pragma omp critical
#endif
        if (status == ORC_OK) status = st;
        break;
      }
      double pc_[3], v[3], ac[3];
      param_state(kind[c], par + 12 * c, tp, pc_, v, ac);
      double aR[3] = {r[0] - pc_[0], r[1] - pc_[1], r[2] - pc_[2]};
      double R = sqrt(dot3(aR, aR));
      if (R <= r_excl) { mask[idx] = 1; continue; }
      double Ec[3], Er[3], ph, Ac[3];
      lw_jackson(q[c], aR, v, ac, Ec, Er, &ph, Ac);
      double Ek[3], n[3] = {aR[0] / R, aR[1] / R, aR[2] / R}, nE[3];
      for (int i = 0; i < 3; ++i)
        Ek[i] = (fkind == ORC_COULOMB) ? Ec[i] : (fkind == ORC_RADIATION) ? Er[i] : Ec[i] + Er[i];
      cross3(n, Ek, nE);
      for (int i = 0; i < 3; ++i) { e[i] += Ek[i]; b[i] += nE[i] / ORC_C; aa[i] += Ac[i]; }
      phi[idx] += ph;
    }
  }
  (void)nthreads;
  return status;
}

/*
 * Lorentz-oscillator run, Algorithm 1, for one configuration of N dipoles.
 *
 * Dipole i: origin R_i, unit axis p_i, charges +-q_i with masses m1_i (positive) and m2_i
 * (negative), natural frequency omega0_i, initial moment d0_i along p_i (d = q r_dip, Sec. 2.3).
 * Equation of motion (Eq. LO_equation) projected on p_i:
 *     d'' + gamma0 d' + omega0^2 d = (q^2/m) E_d(t),  gamma0 = q^2 omega0^2 / (6 pi eps0 c^3 m),
 *     m = m1 m2 / (m1 + m2)  (Eq. eff_mass),
 * E_d = p_i . E(R_i, t) summed over every other dipole's two charges (Sec. 3.2).
 * RK4 on y = (d, d'); with ed_mode == 0 E_d is evaluated at each RK4 stage time t, t + dt/2, t + dt,
 * with ed_mode == 1 it is held at its value at t for all stages.
 * History: d, d', d'' at t_n = n dt; the dipoles are stationary for t <= 0 (d = d0, d' = d'' = 0).
 * After each step d''_{n+1} is taken from the equation of motion at t_{n+1}.
 * Energy (Eq. dipoleE): m omega0^2 d^2 / (2 q^2) + m d'^2 / (2 q^2).
 * The run stops with ORC_ERR_VELOCITY if a charge exceeds v_max (Sec. 3.2).
 *
 * Outputs d, dd, ddd, energy, Ed: [N][n_steps + 1] (Ed may be NULL).
 */
int orc_dipoles_run_moving(int32_t N, const double *origin, const double *axis, const double *q, const double *m1,
                           const double *m2, const double *omega0, const double *d0, const double *org_pos,
                           const double *org_vel, const double *org_acc, double dt, int64_t n_steps, double v_max,
                           int32_t ed_mode, double *d, double *dd, double *ddd, double *energy, double *Ed,
                           int32_t nthreads);

int orc_dipoles_run(int32_t N, const double *origin, const double *axis, const double *q, const double *m1,
                    const double *m2, const double *omega0, const double *d0, double dt, int64_t n_steps,
                    double v_max, int32_t ed_mode, double *d, double *dd, double *ddd, double *energy, double *Ed,
                    int32_t nthreads) {
  return orc_dipoles_run_moving(N, origin, axis, q, m1, m2, omega0, d0, NULL, NULL, NULL, dt, n_steps, v_max, ed_mode,
                                d, dd, ddd, energy, Ed, nthreads);
}

/*
 * Moving dipoles (Sec. 4.3): the origin of dipole i follows a prescribed trajectory, given at the
 * half steps (org_pos/org_vel/org_acc [N][2 n_steps + 1][3], NULL for fixed origins).  The driving
 * field of each RK4 stage is taken at the origin's position at that stage's time (half-step
 * index 2n, 2n + 1, 2n + 2); the sources' retarded positions follow the whole-step history.
 */
int orc_dipoles_run_moving(int32_t N, const double *origin, const double *axis, const double *q, const double *m1,
                           const double *m2, const double *omega0, const double *d0, const double *org_pos,
                           const double *org_vel, const double *org_acc, double dt, int64_t n_steps, double v_max,
                           int32_t ed_mode, double *d, double *dd, double *ddd, double *energy, double *Ed,
                           int32_t nthreads) {
  if (N <= 0 || n_steps < 0 || !(dt > 0.0)) return ORC_ERR_ARG;
  if (org_pos && (!org_vel || !org_acc)) return ORC_ERR_ARG;
  int64_t S = n_steps + 1;
  const int64_t Hn = 2 * S - 1;
  orc_sources s;
  memset(&s, 0, sizeof(s));
  s.N = N; s.Sd = S; s.t0d = 0.0; s.dtd = dt;
  s.origin = origin; s.axis = axis; s.qd = q; s.m1 = m1; s.m2 = m2;
  s.d = d; s.d_dot = dd; s.d_ddot = ddd;
  s.org_pos = org_pos; s.org_vel = org_vel; s.org_acc = org_acc;
  double *ed_now = (double *)calloc((size_t)N, sizeof(double));
  double *ed_half = (double *)calloc((size_t)N, sizeof(double));
  double *ed_next = (double *)calloc((size_t)N, sizeof(double));
  if (!ed_now || !ed_half || !ed_next) { free(ed_now); free(ed_half); free(ed_next); return ORC_ERR_ARG; }
  for (int i = 0; i < N; ++i) {
    d[(int64_t)i * S] = d0[i];
    dd[(int64_t)i * S] = 0.0;
    ddd[(int64_t)i * S] = 0.0;
  }
  int status = ORC_OK;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#endif
  for (int64_t n = 0; n < n_steps && status == ORC_OK; ++n) {
    s.last_valid = n;
    double t = n * dt;
    int st_loop = ORC_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (int i = 0; i < N; ++i) {
      double E[3], B[3], ph, A[3];
      uint8_t mk;
      int st = ORC_OK;
      const double *p = axis + 3 * i;
      /* receiver position at the half steps 2n, 2n + 1, 2n + 2 */
      const double *r0 = org_pos ? org_pos + ((int64_t)i * Hn + 2 * n) * 3 : origin + 3 * i;
      const double *r1 = org_pos ? r0 + 3 : r0;
      const double *r2 = org_pos ? r0 + 6 : r0;
      if (n == 0) {
        st = fields_at(&s, r0, t, ORC_TOTAL, 0.0, i, E, B, &ph, A, &mk, NULL);
        ed_now[i] = dot3(p, E);
        if (Ed) Ed[(int64_t)i * S] = ed_now[i];
      }
      if (!st) {
        st = fields_at(&s, r1, t + 0.5 * dt, ORC_TOTAL, 0.0, i, E, B, &ph, A, &mk, NULL);
        ed_half[i] = dot3(p, E);
      }
      if (!st) {
        st = fields_at(&s, r2, t + dt, ORC_TOTAL, 0.0, i, E, B, &ph, A, &mk, NULL);
        ed_next[i] = dot3(p, E);
      }
      if (st) {
#ifdef _OPENMP
#pragma omp critical
#endif
        if (st_loop == ORC_OK) st_loop = st;
      }
    }
    if (st_loop) { status = st_loop; break; }
    for (int i = 0; i < N; ++i) {
      double m = m1[i] * m2[i] / (m1[i] + m2[i]);
      double w0 = omega0[i];
      double g0 = q[i] * q[i] * w0 * w0 / (6.0 * ORC_PI * ORC_EPS0 * ORC_C * ORC_C * ORC_C * m);
      double qm = q[i] * q[i] / m;
      double e1 = ed_now[i];
      double e2 = (ed_mode == 1) ? ed_now[i] : ed_half[i];
      double e4 = (ed_mode == 1) ? ed_now[i] : ed_next[i];
      double y0 = d[(int64_t)i * S + n], y1 = dd[(int64_t)i * S + n];
      /* f(t, d, d') = (d', -gamma0 d' - omega0^2 d + (q^2/m) E_d(t)) */
      double k1a = y1, k1b = -g0 * y1 - w0 * w0 * y0 + qm * e1;
      double k2a = y1 + 0.5 * dt * k1b, k2b = -g0 * (y1 + 0.5 * dt * k1b) - w0 * w0 * (y0 + 0.5 * dt * k1a) + qm * e2;
      double k3a = y1 + 0.5 * dt * k2b, k3b = -g0 * (y1 + 0.5 * dt * k2b) - w0 * w0 * (y0 + 0.5 * dt * k2a) + qm * e2;
      double k4a = y1 + dt * k3b, k4b = -g0 * (y1 + dt * k3b) - w0 * w0 * (y0 + dt * k3a) + qm * e4;
      double yn0 = y0 + dt / 6.0 * (k1a + 2.0 * k2a + 2.0 * k3a + k4a);
      double yn1 = y1 + dt / 6.0 * (k1b + 2.0 * k2b + 2.0 * k3b + k4b);
      d[(int64_t)i * S + n + 1] = yn0;
      dd[(int64_t)i * S + n + 1] = yn1;
      /* d'' at the step end from the equation of motion (field at t_{n+1}) */
      ddd[(int64_t)i * S + n + 1] = qm * ed_next[i] - g0 * yn1 - w0 * w0 * yn0;
      if (Ed) Ed[(int64_t)i * S + n + 1] = ed_next[i];
      double vmax_charge = fabs(yn1) / q[i] * ((m1[i] > m2[i] ? m1[i] : m2[i]) / (m1[i] + m2[i]));
      if (vmax_charge > v_max) status = ORC_ERR_VELOCITY;
      ed_now[i] = ed_next[i];
    }
  }
  for (int i = 0; i < N; ++i) {
    double m = m1[i] * m2[i] / (m1[i] + m2[i]);
    for (int64_t n = 0; n < S; ++n) {
      double x = d[(int64_t)i * S + n], xv = dd[(int64_t)i * S + n];
      energy[(int64_t)i * S + n] = m * omega0[i] * omega0[i] * x * x / (2.0 * q[i] * q[i]) + m * xv * xv / (2.0 * q[i] * q[i]);
    }
  }
  free(ed_now); free(ed_half); free(ed_next);
  return status;
}

/*
 * ---------------------------------------------------------------------------------------------
 * Extended precision: the same retarded-time bisection, linear interpolation of the history
 * (Sec. 3.1), Jackson form (Eqs. V, A, E, B) and superposition (Sec. 2.2) as fields_at, with every
 * intermediate in IEEE binary128 (113-bit significand; libgcc's software arithmetic on both the
 * x86-64 and the aarch64 build).  The inputs are the same float64 samples, read exactly; the sums
 * are rounded to float64 only at the end.  A dipole's two charges cancel by R/s in the sum (up to
 * 1e7 near a dipole whose moment crosses zero), which costs the float64 evaluation that many
 * digits; here the loss leaves ~1e-27 relative, so the result is the field of the discrete
 * history to float64 rounding.  Fixed origins only.
 * ---------------------------------------------------------------------------------------------
 */
typedef _Float128 xreal;

/* square root: float64 estimate, then two Newton steps (each doubles the correct bits: 53 -> 106
 * -> beyond the 113 of the format) */
static xreal xsqrt(xreal a) {
  if (!(a > 0)) return 0;
  xreal x = (xreal)sqrt((double)a);
  x = 0.5 * (x + a / x);
  x = 0.5 * (x + a / x);
  return x;
}

static xreal xdot3(const xreal *a, const xreal *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void xcross3(const xreal *a, const xreal *b, xreal *o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

/* charge_state in binary128: linear interpolation between the float64 samples (Sec. 3.1), dipole
 * charges at R +- w (d/q) p (Eqs. r_1, r_2), at rest before the first sample (Sec. 3.2) */
static int xcharge_state(const orc_sources *s, int c, xreal tp, xreal *qc, xreal p[3], xreal v[3], xreal a[3]) {
  if (c < s->M) {
    const double *P = s->pos + (int64_t)c * s->S * 3;
    const double *V = s->vel + (int64_t)c * s->S * 3;
    const double *A = s->acc + (int64_t)c * s->S * 3;
    *qc = s->q[c];
    xreal x = (tp - (xreal)s->t0) / (xreal)s->dt;
    if (x < 0 && x > -1e-9) x = 0;
    if (x > (xreal)(s->S - 1) && x < (xreal)(s->S - 1) + (xreal)1e-9) x = (xreal)(s->S - 1);
    if (x < 0) {
      if (!s->static_before) return ORC_ERR_HISTORY;
      for (int i = 0; i < 3; ++i) { p[i] = P[i]; v[i] = 0; a[i] = 0; }
      return ORC_OK;
    }
    int64_t k = (int64_t)x;
    if (k >= s->S - 1) {
      if (x > (xreal)(s->S - 1)) return ORC_ERR_HISTORY;
      k = s->S - 2;
    }
    xreal th = x - (xreal)k;
    for (int i = 0; i < 3; ++i) {
      p[i] = (xreal)P[k * 3 + i] + th * ((xreal)P[(k + 1) * 3 + i] - (xreal)P[k * 3 + i]);
      v[i] = (xreal)V[k * 3 + i] + th * ((xreal)V[(k + 1) * 3 + i] - (xreal)V[k * 3 + i]);
      a[i] = (xreal)A[k * 3 + i] + th * ((xreal)A[(k + 1) * 3 + i] - (xreal)A[k * 3 + i]);
    }
    return ORC_OK;
  }
  int j = (c - s->M) / 2;
  int neg = (c - s->M) % 2;
  xreal m1 = s->m1[j], m2 = s->m2[j], q = s->qd[j];
  const double *u = s->axis + 3 * j;
  const double *R = s->origin + 3 * j;
  const double *D = s->d + (int64_t)j * s->Sd;
  const double *DV = s->d_dot + (int64_t)j * s->Sd;
  const double *DA = s->d_ddot + (int64_t)j * s->Sd;
  xreal dd, dv, da;
  xreal x = (tp - (xreal)s->t0d) / (xreal)s->dtd;
  if (x <= 0) {
    dd = D[0]; dv = 0; da = 0;
  } else {
    int64_t last = s->Sd - 1;
    if (x > (xreal)last && x < (xreal)last + (xreal)1e-9) x = (xreal)last;
    int64_t k = (int64_t)x;
    if (k >= last) {
      if (x > (xreal)last) return ORC_ERR_HISTORY;
      k = last - 1;
    }
    xreal th = x - (xreal)k;
    dd = (xreal)D[k] + th * ((xreal)D[k + 1] - (xreal)D[k]);
    dv = (xreal)DV[k] + th * ((xreal)DV[k + 1] - (xreal)DV[k]);
    da = (xreal)DA[k] + th * ((xreal)DA[k + 1] - (xreal)DA[k]);
  }
  xreal w = neg ? -m1 / (m1 + m2) : m2 / (m1 + m2);
  *qc = neg ? -q : q;
  for (int i = 0; i < 3; ++i) {
    p[i] = (xreal)R[i] + w * (dd / q) * (xreal)u[i];
    v[i] = w * (dv / q) * (xreal)u[i];
    a[i] = w * (da / q) * (xreal)u[i];
  }
  return ORC_OK;
}

static xreal xg_at(const orc_sources *s, int c, xreal t, const xreal r[3], xreal tp, int *st) {
  xreal qc, p[3], v[3], a[3];
  *st = xcharge_state(s, c, tp, &qc, p, v, a);
  xreal D[3] = {r[0] - p[0], r[1] - p[1], r[2] - p[2]};
  return (xreal)ORC_C * (t - tp) - xsqrt(xdot3(D, D));
}

/* bisection of g(t') = c (t - t') - |r - r_c(t')| (Eq. ret_t) as orc_retarded_time, to the
 * resolution of binary128 */
static int xretarded_time(const orc_sources *s, int c, xreal t, const xreal r[3], xreal *tp_out) {
  int st;
  int sampled = (c < s->M);
  xreal t_first = sampled ? s->t0 : s->t0d;
  xreal t_last = sampled ? (xreal)s->t0 + (xreal)(s->S - 1) * (xreal)s->dt
                         : (xreal)s->t0d + (xreal)(s->Sd - 1) * (xreal)s->dtd;
  xreal hi = (t < t_last) ? t : t_last;
  xreal lo;
  if (sampled && !s->static_before) {
    lo = t_first;
    if (lo > hi) return ORC_ERR_HISTORY;
    xreal g = xg_at(s, c, t, r, lo, &st);
    if (st) return st;
    if (g < 0) return ORC_ERR_HISTORY;
  } else {
    xreal qc, p[3], v[3], a[3];
    st = xcharge_state(s, c, (t < t_first) ? t : t_first, &qc, p, v, a);
    if (st) return st;
    xreal D[3] = {r[0] - p[0], r[1] - p[1], r[2] - p[2]};
    lo = t - xsqrt(xdot3(D, D)) / (xreal)ORC_C * ((xreal)1 + (xreal)1e-12) - (xreal)1e-30;
    if (lo > t_first) lo = t_first;
    if (lo > hi) lo = hi;
  }
  if (hi < t) {
    xreal g = xg_at(s, c, t, r, hi, &st);
    if (st) return st;
    if (g > 0) return ORC_ERR_HISTORY;
    if (g == 0) { *tp_out = hi; return ORC_OK; }
  }
  for (int it = 0; it < 16000; ++it) {
    xreal mid = (xreal)0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    xreal g = xg_at(s, c, t, r, mid, &st);
    if (st) return st;
    if (g >= 0) lo = mid; else hi = mid;
  }
  *tp_out = (xreal)0.5 * (lo + hi);
  return ORC_OK;
}

/* lw_jackson in binary128 (Eqs. V, A, E, ECoulomb, Eradiation; A read as (v/c^2) phi) */
static void xlw_jackson(xreal q, const xreal aR[3], const xreal v[3], const xreal acc[3], xreal Ec[3], xreal Er[3],
                        xreal *phi, xreal A[3]) {
  const xreal c = ORC_C, eps0 = ORC_EPS0, pi = ORC_PI;
  xreal R = xsqrt(xdot3(aR, aR));
  xreal n[3] = {aR[0] / R, aR[1] / R, aR[2] / R};
  xreal beta[3] = {v[0] / c, v[1] / c, v[2] / c};
  xreal bdot[3] = {acc[0] / c, acc[1] / c, acc[2] / c};
  xreal kappa = 1 - xdot3(n, beta);
  xreal b2 = xdot3(beta, beta);
  xreal k = q / (4 * pi * eps0);
  xreal nb[3] = {n[0] - beta[0], n[1] - beta[1], n[2] - beta[2]};
  xreal k3 = kappa * kappa * kappa;
  for (int i = 0; i < 3; ++i) Ec[i] = k * nb[i] * (1 - b2) / (k3 * R * R);
  xreal w[3], nw[3];
  xcross3(nb, bdot, w);
  xcross3(n, w, nw);
  for (int i = 0; i < 3; ++i) Er[i] = k * nw[i] / (c * k3 * R);
  *phi = k / (kappa * R);
  xreal mu0 = 1 / (eps0 * c * c);
  for (int i = 0; i < 3; ++i) A[i] = mu0 * q * c / (4 * pi) * beta[i] / (kappa * R);
}

/*
 * Fields on P points at T times as orc_fields (outputs rounded to float64), every step in binary128.
 * Charges closer than r_excl at their retarded position are skipped and masked.
 */
int orc_fields_x(const orc_sources *s, const double *points, int64_t P, const double *times, int32_t T, int32_t kind,
                 double r_excl, double *E, double *B, double *phi, double *A, uint8_t *mask, int32_t nthreads) {
  if (kind < 0 || kind > 2 || P < 0 || T < 0 || s->org_pos || s->last_valid >= 0) return ORC_ERR_ARG;
  int status = ORC_OK;
  int64_t total = P * (int64_t)T;
  int nc = orc_n_charges(s);
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int64_t idx = 0; idx < total; ++idx) {
    int64_t f = idx / P, pidx = idx % P;
    const xreal r[3] = {points[3 * pidx], points[3 * pidx + 1], points[3 * pidx + 2]};
    const xreal t = times[f];
    xreal e[3] = {0, 0, 0}, b[3] = {0, 0, 0}, aa[3] = {0, 0, 0}, ph = 0;
    uint8_t mk = 0;
    int st = ORC_OK;
    for (int c = 0; c < nc && !st; ++c) {
      xreal tp;
      st = xretarded_time(s, c, t, r, &tp);
      if (st) break;
      xreal qc, p[3], v[3], ac[3];
      st = xcharge_state(s, c, tp, &qc, p, v, ac);
      if (st) break;
      xreal aR[3] = {r[0] - p[0], r[1] - p[1], r[2] - p[2]};
      xreal R = xsqrt(xdot3(aR, aR));
      if (R <= (xreal)r_excl) { mk = 1; continue; }
      xreal Ec[3], Er[3], phc, Ac[3], Ek[3], nE[3];
      xlw_jackson(qc, aR, v, ac, Ec, Er, &phc, Ac);
      for (int i = 0; i < 3; ++i)
        Ek[i] = (kind == ORC_COULOMB) ? Ec[i] : (kind == ORC_RADIATION) ? Er[i] : Ec[i] + Er[i];
      xreal n[3] = {aR[0] / R, aR[1] / R, aR[2] / R};
      xcross3(n, Ek, nE);
      for (int i = 0; i < 3; ++i) { e[i] += Ek[i]; b[i] += nE[i] / (xreal)ORC_C; aa[i] += Ac[i]; }
      ph += phc;
    }
    for (int i = 0; i < 3; ++i) {
      E[3 * idx + i] = (double)e[i];
      B[3 * idx + i] = (double)b[i];
      A[3 * idx + i] = (double)aa[i];
    }
    phi[idx] = (double)ph;
    mask[idx] = mk;
    if (st) {
#ifdef _OPENMP
#pragma omp critical
#endif
      if (status == ORC_OK) status = st;
    }
  }
  (void)nthreads;
  return status;
}

/* sizeof check for the Python binding */
int64_t orc_sources_size(void) { return (int64_t)sizeof(orc_sources); }
