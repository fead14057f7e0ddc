// Internal declarations shared by the translation units of libpycharge_gb300.so.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pycharge_gb300.h"

namespace pc {

// CODATA 2018 (c and e exact)
constexpr double kC = 299792458.0;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kPi = 3.14159265358979323846;
constexpr double kKe = 1.0 / (4.0 * kPi * kEps0);  // 1/(4 pi eps0)
constexpr double kE = 1.602176634e-19;

// Device status word: the first error code wins.
__device__ __forceinline__ void set_status(int *st, int code) {
  if (*((volatile int *)st) == 0) atomicCAS(st, 0, code);
}

// Grow-only device buffer owned by the context.
struct Buf {
  void *ptr = nullptr;
  size_t bytes = 0;
  cudaError_t reserve(size_t n) {
    if (n <= bytes) return cudaSuccess;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&ptr, n);
    if (e == cudaSuccess) bytes = n;
    return e;
  }
  void release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
  }
};

}  // namespace pc

struct pc_ctx {
  int device = 0;
  int *d_status = nullptr;   // device status word
  int *h_status = nullptr;   // pinned host copy
  pc::Buf hist_f32;          // float32 mirrors of source histories (mixed path)
  pc::Buf charge_ref;        // per-charge float64 reference positions
  pc::Buf run_scratch;       // LO-run scratch (tables, stage fields)
  pc::Buf run_store;         // LO-run history ring, its float32 mirror, per-step fit inputs
  pc::Buf adj_scratch;       // adjoint: forward history, history adjoints
  cudaGraph_t loop_graph = nullptr;     // causal-block loop of the last grid-path run
  cudaGraphExec_t loop_exec = nullptr;
  int tile_shift = 4;                   // mixed plane tiles: (256 >> shift) rows x (1 << shift) columns
  int pts_per_thread = 1;               // mixed plane grids of dipoles: 1, or 2 (tiles twice as tall)
  int src_chunk = 64;                   // mixed plane tiles: sources per shared-memory stage (32 or 64)
  int run_slices = 0;                   // oscillator grid path: source slices per receiver (0: heuristic)
  int run_timing = 0;                   // oscillator run: record launch times (pc_set_run_timing)
  pc_run_timing timing = {};            // their sums since the last enable
  cudaEvent_t tev[3 * 64 + 2] = {};     // events of up to 64 timed blocks (or one persistent launch)
  pc::Buf out_chunks;                   // field outputs bound for the host: two alternating chunks
  cudaStream_t copy_stream = nullptr;   // their device-to-host copies
  cudaEvent_t pipe_ev[4] = {nullptr, nullptr, nullptr, nullptr};  // chunk computed (2), chunk copied (2)
  int num_sms = 0;
};

namespace pc {

// Switch to the context's device for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// Reset the status word, to be called at the start of an entry point.
pc_status begin_call(pc_ctx *ctx, cudaStream_t s);
// Read the status word back (synchronises the stream) and merge a launch error.
pc_status end_call(pc_ctx *ctx, cudaStream_t s);

// Dipole axes are unit vectors (a dipole's charges move along its axis; the pair algebra of both
// paths uses p . p = 1): an axis whose squared norm is more than kAxisTol from 1 sets PC_ERR_ARG.
constexpr double kAxisTol = 1e-10;
__global__ void check_axes_kernel(const double *axis, int64_t n, int *status);

}  // namespace pc
