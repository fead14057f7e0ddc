// Lorentz-oscillator run (Algorithm 1 of arXiv 2107.12437) and the kinetic-energy fit (Eq. KE).
//
// pc_dipoles_run: one CTA per configuration; its threads own dipoles.  Every step each thread
// evaluates the driving field of its dipoles at the two new RK4 stage times t + dt/2 and t + dt
// (the field at t is the previous step's t + dt value) from the stored history of every other
// dipole of the configuration, advances (d, d') by RK4 (Eq. LO_equation) and appends d, d', d''
// to the history; a CTA barrier separates steps.  The history arrays are the caller's outputs.
// pc_ke_fit: one CTA per series; Levenberg-Marquardt with block reductions.
#include <stdio.h>

#include "pc_internal.cuh"
#include "pc_lw_f64.cuh"

namespace pc {

struct RunArgs {
  int B, N;
  const double *origin, *axis, *q, *m1, *m2, *omega0, *d0;
  double dt;
  int64_t n_steps;
  double v_max;
  int ed_mode;
  double *d, *dd, *ddd, *energy, *Ed;
  double *ed_now;  // scratch [B][N]
  int *status;
};

// Driving field of dipole i of configuration b at time u (in steps), history samples 0..n_valid.
__device__ double drive_f64(const RunArgs &a, int b, int i, double u, int64_t n_valid, int *err) {
  const int N = a.N;
  const int64_t S = a.n_steps + 1;
  const double cdt = kC * a.dt;
  const double *Ri = a.origin + 3 * ((size_t)b * N + i);
  const double *pi = a.axis + 3 * ((size_t)b * N + i);
  double E[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < N; ++j) {
    if (j == i) continue;
    const size_t bj = (size_t)b * N + j;
    TrajF64 tr;
    tr.dipole = true;
    tr.d = a.d + bj * S;
    tr.dd = a.dd + bj * S;
    tr.ddd = a.ddd + bj * S;
    for (int k = 0; k < 3; ++k) {
      tr.R[k] = a.origin[3 * bj + k];
      tr.ax[k] = a.axis[3 * bj + k];
    }
    const double q = a.q[bj], m1 = a.m1[bj], m2 = a.m2[bj];
    double dv[3] = {Ri[0] - tr.R[0], Ri[1] - tr.R[1], Ri[2] - tr.R[2]};
    const double tau0 = sqrt(dot3(dv, dv)) / cdt;
    const int64_t kg = (int64_t)floor(u - tau0);
    for (int sg = 0; sg < 2; ++sg) {
      tr.w = (sg == 0) ? m2 / (m1 + m2) / q : -m1 / (m1 + m2) / q;
      double p0[3], v[3] = {0, 0, 0}, ac[3] = {0, 0, 0};
      if (n_valid == 0) {
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
        int e = solve_f64(tr, n_valid + 1, 1, Ri, u, cdt, kg, &k, &th);
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
  }
  return dot3(pi, E);
}

__global__ void __launch_bounds__(256) lo_run_f64_kernel(const RunArgs a) {
  const int b = blockIdx.x;
  const int N = a.N;
  const int64_t S = a.n_steps + 1;
  __shared__ int s_stop;
  if (threadIdx.x == 0) s_stop = 0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const size_t bi = (size_t)b * N + i;
    a.d[bi * S] = a.d0[bi];
    a.dd[bi * S] = 0.0;
    a.ddd[bi * S] = 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    int err = 0;
    const size_t bi = (size_t)b * N + i;
    double e0 = drive_f64(a, b, i, 0.0, 0, &err);
    if (err) {
      set_status(a.status, err);
      s_stop = 1;
    }
    a.ed_now[bi] = e0;
    if (a.Ed) a.Ed[bi * S] = e0;
    if (a.energy) {
      const double m = a.m1[bi] * a.m2[bi] / (a.m1[bi] + a.m2[bi]);
      const double w0 = a.omega0[bi], q = a.q[bi], x = a.d0[bi];
      a.energy[bi * S] = m * w0 * w0 * x * x / (2.0 * q * q);
    }
  }
  __syncthreads();
  for (int64_t n = 0; n < a.n_steps; ++n) {
    if (s_stop) break;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      int err = 0;
      const size_t bi = (size_t)b * N + i;
      const double e1 = a.ed_now[bi];
      double e2 = 0.0, e4 = 0.0;
      e2 = drive_f64(a, b, i, (double)n + 0.5, n, &err);
      if (!err) e4 = drive_f64(a, b, i, (double)n + 1.0, n, &err);
      if (err) {
        set_status(a.status, err);
        s_stop = 1;
        continue;
      }
      const double m1 = a.m1[bi], m2 = a.m2[bi], q = a.q[bi], w0 = a.omega0[bi];
      const double m = m1 * m2 / (m1 + m2);
      const double g0 = q * q * w0 * w0 / (6.0 * kPi * kEps0 * kC * kC * kC * m);
      const double qm = q * q / m;
      const double dt = a.dt;
      const double f2 = (a.ed_mode == 1) ? e1 : e2;
      const double f4 = (a.ed_mode == 1) ? e1 : e4;
      const double y0 = a.d[bi * S + n], y1 = a.dd[bi * S + n];
      // RK4 on (d, d') with d'' = -gamma0 d' - omega0^2 d + (q^2/m) E_d(t)
      const double k1a = y1, k1b = -g0 * y1 - w0 * w0 * y0 + qm * e1;
      const double y0b = y0 + 0.5 * dt * k1a, y1b = y1 + 0.5 * dt * k1b;
      const double k2a = y1b, k2b = -g0 * y1b - w0 * w0 * y0b + qm * f2;
      const double y0c = y0 + 0.5 * dt * k2a, y1c = y1 + 0.5 * dt * k2b;
      const double k3a = y1c, k3b = -g0 * y1c - w0 * w0 * y0c + qm * f2;
      const double y0d = y0 + dt * k3a, y1d = y1 + dt * k3b;
      const double k4a = y1d, k4b = -g0 * y1d - w0 * w0 * y0d + qm * f4;
      const double yn0 = y0 + dt / 6.0 * (k1a + 2.0 * k2a + 2.0 * k3a + k4a);
      const double yn1 = y1 + dt / 6.0 * (k1b + 2.0 * k2b + 2.0 * k3b + k4b);
      a.d[bi * S + n + 1] = yn0;
      a.dd[bi * S + n + 1] = yn1;
      a.ddd[bi * S + n + 1] = qm * e4 - g0 * yn1 - w0 * w0 * yn0;
      if (a.Ed) a.Ed[bi * S + n + 1] = e4;
      if (a.energy) a.energy[bi * S + n + 1] = m * (w0 * w0 * yn0 * yn0 + yn1 * yn1) / (2.0 * q * q);
      a.ed_now[bi] = e4;
      const double vch = fabs(yn1) / q * (fmax(m1, m2) / (m1 + m2));
      if (vch > a.v_max) {
        set_status(a.status, PC_ERR_VELOCITY);
        s_stop = 1;
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------------
// kinetic-energy series for the fit
// ------------------------------------------------------------------------------------------------
__global__ void ke_series_kernel(const RunArgs a, double *ke) {
  const int64_t S = a.n_steps + 1;
  const int64_t n = (int64_t)a.B * a.N * S;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t bi = idx / S;
    const double m = a.m1[bi] * a.m2[bi] / (a.m1[bi] + a.m2[bi]);
    const double q = a.q[bi], v = a.dd[idx];
    ke[idx] = m * v * v / (2.0 * q * q);
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

// residual/Jacobian pass.  mode 0: cost only; mode 1: cost, J^T J (10), J^T r (4)
__device__ void fit_pass(const double *y, int64_t n, double dt, double T, double Ag, double wg, const double x[4],
                         int mode, double out[15]) {
  for (int k = 0; k < 15; ++k) out[k] = 0.0;
  const double A = Ag * x[0], g = x[1] / T, w = wg + x[2] / T, ph = x[3];
  const int64_t chunk = (n + kFitThreads - 1) / kFitThreads;
  const int64_t i0 = (int64_t)threadIdx.x * chunk, i1 = min(n, i0 + chunk);
  for (int64_t i = i0; i < i1; ++i) {
    const double tau = (double)i * dt;
    double s, c;
    sincos(w * tau + ph, &s, &c);
    const double env = exp(-g * tau);
    const double model = A * env * s * s;
    const double r = (model - y[i]) / Ag;
    out[0] += r * r;
    if (mode) {
      double J[4];
      J[0] = env * s * s;
      J[1] = -tau * A * env * s * s / T / Ag;
      J[2] = 2.0 * A * env * s * c * tau / T / Ag;
      J[3] = 2.0 * A * env * s * c / Ag;
      int idx = 1;
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = p; q < 4; ++q) out[idx++] += J[p] * J[q];
#pragma unroll
      for (int p = 0; p < 4; ++p) out[11 + p] += J[p] * r;
    }
  }
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

extern "C" pc_status pc_dipoles_run(pc_ctx *ctx, const pc_dipoles *dp, double dt, int64_t n_steps,
                                    const pc_run_opts *opts, const pc_run_out *out, void *stream) {
  if (!ctx || !dp || !opts || !out) return PC_ERR_ARG;
  if (dp->B < 1 || dp->N < 1 || !(dt > 0.0) || n_steps < 0) return PC_ERR_ARG;
  if (!dp->origin || !dp->axis || !dp->q || !dp->m1 || !dp->m2 || !dp->omega0 || !dp->d0) return PC_ERR_ARG;
  if (!out->d || !out->d_dot || !out->d_ddot) return PC_ERR_ARG;
  if (opts->ed_mode != 0 && opts->ed_mode != 1) return PC_ERR_ARG;
  if (opts->precision != PC_F64 && opts->precision != PC_MIXED) return PC_ERR_ARG;
  if (opts->fit && (!out->gamma || !out->omega || opts->first_index < 0 || n_steps + 1 - opts->first_index < 8))
    return PC_ERR_ARG;
  pc::DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  pc_status bs = pc::begin_call(ctx, st);
  if (bs != PC_OK) return bs;
  const int64_t S = n_steps + 1;
  const size_t nbn = (size_t)dp->B * dp->N;
  size_t scratch = nbn * sizeof(double);
  if (opts->fit) scratch += nbn * S * sizeof(double);
  if (ctx->run_scratch.reserve(scratch) != cudaSuccess) return PC_ERR_CUDA;
  pc::RunArgs a;
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
  a.n_steps = n_steps;
  a.v_max = opts->v_max > 0.0 ? opts->v_max : pc::kC / 100.0;
  a.ed_mode = opts->ed_mode;
  a.d = out->d;
  a.dd = out->d_dot;
  a.ddd = out->d_ddot;
  a.energy = out->energy;
  a.Ed = out->Ed;
  a.ed_now = (double *)ctx->run_scratch.ptr;
  a.status = ctx->d_status;
  int threads = dp->N >= 256 ? 256 : ((dp->N + 31) / 32) * 32;
  pc::lo_run_f64_kernel<<<dp->B, threads, 0, st>>>(a);
  if (opts->fit) {
    double *ke = a.ed_now + nbn;
    pc::ke_series_kernel<<<ctx->num_sms * 4, 256, 0, st>>>(a, ke);
    pc_status ls = pc::launch_fit(ctx, ke, (int)nbn, S, dt, opts->first_index, out->gamma, out->omega, nullptr,
                                  nullptr, st);
    if (ls != PC_OK) return ls;
  }
  return pc::end_call(ctx, st);
}
