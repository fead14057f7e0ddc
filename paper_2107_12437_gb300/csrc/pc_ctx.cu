// Context lifetime, status handling and the ALU peak probe.
#include <stdio.h>

#include "pc_internal.cuh"

namespace pc {

pc_status begin_call(pc_ctx *ctx, cudaStream_t s) {
  cudaGetLastError();  // clear a stale launch error of an unrelated caller
  if (cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s) != cudaSuccess) return PC_ERR_CUDA;
  return PC_OK;
}

pc_status end_call(pc_ctx *ctx, cudaStream_t s) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return PC_ERR_CUDA;
  if (cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PC_ERR_CUDA;
  return (pc_status)(*ctx->h_status);
}

__global__ void check_axes_kernel(const double *axis, int64_t n, int *status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = axis[3 * i], y = axis[3 * i + 1], z = axis[3 * i + 2];
  if (!(fabs(x * x + y * y + z * z - 1.0) <= kAxisTol)) set_status(status, PC_ERR_ARG);
}

}  // namespace pc

extern "C" pc_status pc_ctx_create(pc_ctx **out, int device) {
  if (!out) return PC_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return PC_ERR_ARG;
  pc::DeviceGuard g(device);
  pc_ctx *c = new pc_ctx();
  c->device = device;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&c->h_status, sizeof(int)) != cudaSuccess) {
    pc_ctx_destroy(c);
    return PC_ERR_CUDA;
  }
  cudaMemset(c->d_status, 0, sizeof(int));
  *c->h_status = 0;
  *out = c;
  return PC_OK;
}

extern "C" pc_status pc_ctx_destroy(pc_ctx *ctx) {
  if (!ctx) return PC_ERR_ARG;
  pc::DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  ctx->hist_f32.release();
  ctx->charge_ref.release();
  ctx->run_scratch.release();
  ctx->run_store.release();
  ctx->adj_scratch.release();
  if (ctx->loop_exec) cudaGraphExecDestroy(ctx->loop_exec);
  if (ctx->loop_graph) cudaGraphDestroy(ctx->loop_graph);
  ctx->out_chunks.release();
  for (int k = 0; k < 4; ++k)
    if (ctx->pipe_ev[k]) cudaEventDestroy(ctx->pipe_ev[k]);
  for (cudaEvent_t e : ctx->tev)
    if (e) cudaEventDestroy(e);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  delete ctx;
  return PC_OK;
}

extern "C" const char *pc_status_string(pc_status s) {
  switch (s) {
    case PC_OK: return "ok";
    case PC_ERR_ARG: return "invalid argument";
    case PC_ERR_CUDA: return "CUDA runtime error";
    case PC_ERR_HISTORY: return "retarded time outside the stored trajectory samples";
    case PC_ERR_VELOCITY: return "dipole charge exceeded the maximum velocity";
    case PC_ERR_CAUSALITY: return "time step exceeds a light-crossing time between dipoles";
    case PC_ERR_NOCONV: return "solver did not converge";
    case PC_ERR_TIMEOUT: return "reserved (no call returns it)";
  }
  return "unknown status";
}

// ------------------------------------------------------------------------------------------------
// ALU peak probe: independent FMA chains per thread, enough warps to fill every SM.
// ------------------------------------------------------------------------------------------------
template <typename T, int CH>
__global__ void fma_chains(T *out, int iters, T a, T b) {
  T x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
#pragma unroll
      for (int c = 0; c < CH; ++c) x[c] = x[c] * a + b;
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

extern "C" pc_status pc_alu_peaks(pc_ctx *ctx, double *fp32_fma_per_s, double *fp64_fma_per_s, void *stream) {
  if (!ctx || !fp32_fma_per_s || !fp64_fma_per_s) return PC_ERR_ARG;
  pc::DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int threads = 512, blocks = ctx->num_sms * 4;
  double *buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * threads * blocks) != cudaSuccess) return PC_ERR_CUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.f;
  const int it32 = 2048, it64 = 64;
  fma_chains<float, 8><<<blocks, threads, 0, s>>>((float *)buf, 8, 1.0001f, 0.5f);
  cudaEventRecord(e0, s);
  fma_chains<float, 8><<<blocks, threads, 0, s>>>((float *)buf, it32, 1.0001f, 0.5f);
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  *fp32_fma_per_s = (double)blocks * threads * it32 * 16 * 8 / (ms * 1e-3);
  fma_chains<double, 8><<<blocks, threads, 0, s>>>(buf, 2, 1.0001, 0.5);
  cudaEventRecord(e0, s);
  fma_chains<double, 8><<<blocks, threads, 0, s>>>(buf, it64, 1.0001, 0.5);
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  *fp64_fma_per_s = (double)blocks * threads * it64 * 16 * 8 / (ms * 1e-3);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaError_t e = cudaGetLastError();
  cudaFree(buf);
  return e == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}
