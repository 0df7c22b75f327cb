// Measurement probes (declared in include/dmpc.h; the paper has no counterpart): the two
// denominators the benchmark reports the fused kernel against.
//
//  * dmpc_probe_fp32_peak: FP32 FMA throughput of the whole device (every SM, eight
//    independent FMA chains per thread), the ALU roof of the fused kernel.
//  * dmpc_probe_pcg_floor: the latency of one iteration of the single-warp PCG inner loop of
//    the fused kernel (Algorithm 4: two block-tridiagonal products, two warp reductions,
//    alpha, beta and the vector updates; nx = 4, two knots per lane, register blocks), run by
//    one warp alone for a fixed number of iterations.  A PCG solve cannot finish faster than
//    its iteration count times this floor, so it is the latency roof of a launch whose time is
//    the serial PCG chain of its slowest OCP.
// Both run synchronously on the current device and time themselves with CUDA events.
#include <cuda_runtime.h>

#include "../../include/dmpc.h"
#include "fused.cuh"

namespace dmpc {

constexpr int kPeakChains = 8;

__global__ void __launch_bounds__(1024) probe_fma_kernel(float* sink, int iters, float m, float a) {
  float v[kPeakChains];
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) v[j] = (float)(threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) v[j] = fmaf(v[j], m, a);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) s += v[j];
  if (s == -1.2345f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

// One warp runs `iters` iterations of the FP32 PCG loop body of stage_pcg_warp<nx = 4, 2 knots
// per lane> on a synthetic SPD block-tridiagonal system (diagonal blocks 4 I + 0.1 J, off-diagonal
// 0.1 I; preconditioner blocks the diagonal inverse).  Writes the iterations executed.
__global__ void __launch_bounds__(32) probe_pcg_kernel(int iters, int* done, float* sink) {
  constexpr int NX = 4, KPL = 2;
  const int ln = threadIdx.x & 31;
  float Dk[KPL][NX * NX], Ok[KPL][NX * NX], Pdk[KPL][NX * NX], Pok[KPL][NX * NX];
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int a = 0; a < NX; ++a)
#pragma unroll
      for (int b = 0; b < NX; ++b) {
        const int k = ln * KPL + j;
        Dk[j][a * NX + b] = (a == b ? 4.f : 0.f) + 0.1f;
        Ok[j][a * NX + b] = (k > 0 && a == b) ? 0.1f : 0.f;
        Pdk[j][a * NX + b] = (a == b) ? 0.25f : 0.f;
        Pok[j][a * NX + b] = 0.f;
      }
  float r[KPL][NX], z[KPL][NX], p[KPL][NX], y[KPL][NX], dl[KPL][NX];
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int i = 0; i < NX; ++i) { r[j][i] = 1.f + 0.01f * (float)((ln * 7 + j * 3 + i) % 11); dl[j][i] = 0.f; }
  warp_btmv<NX, KPL>(Pdk, Pok, r, z, ln);
  float e1[1] = {0.f};
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int i = 0; i < NX; ++i) { p[j][i] = z[j][i]; e1[0] = fmaf(r[j][i], z[j][i], e1[0]); }
  warp_sum(e1);
  float eta = e1[0];
  int it = 0;
  for (; it < iters; ++it) {
    warp_btmv<NX, KPL>(Dk, Ok, p, y, ln);
    float v[1] = {0.f};
#pragma unroll
    for (int j = 0; j < KPL; ++j)
#pragma unroll
      for (int i = 0; i < NX; ++i) v[0] = fmaf(p[j][i], y[j][i], v[0]);
    warp_sum(v);
    if (!(v[0] > 0.f) || !isfinite(v[0])) break;
    const float alpha = __fdividef(eta, v[0]);
#pragma unroll
    for (int j = 0; j < KPL; ++j)
#pragma unroll
      for (int i = 0; i < NX; ++i) { dl[j][i] = fmaf(alpha, p[j][i], dl[j][i]); r[j][i] = fmaf(-alpha, y[j][i], r[j][i]); }
    warp_btmv<NX, KPL>(Pdk, Pok, r, z, ln);
    float e2[1] = {0.f};
#pragma unroll
    for (int j = 0; j < KPL; ++j)
#pragma unroll
      for (int i = 0; i < NX; ++i) e2[0] = fmaf(r[j][i], z[j][i], e2[0]);
    warp_sum(e2);
    const float eta_new = e2[0];
    if (!(eta_new > 0.f) || !isfinite(eta_new)) { ++it; break; }
    const float beta = __fdividef(eta_new, eta);
    eta = eta_new;
#pragma unroll
    for (int j = 0; j < KPL; ++j)
#pragma unroll
      for (int i = 0; i < NX; ++i) p[j][i] = fmaf(beta, p[j][i], z[j][i]);
    // keep the residual away from underflow: restart the direction from the current residual
    // when it has shrunk (a data-dependent branch like the loop's own convergence tests)
    if (eta < 1e-20f) {
#pragma unroll
      for (int j = 0; j < KPL; ++j)
#pragma unroll
        for (int i = 0; i < NX; ++i) { r[j][i] = 1.f; p[j][i] = 0.25f; }
      eta = 0.25f * 64.f * NX;
    }
  }
  if (ln == 0) *done = it;
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int i = 0; i < NX; ++i) s += dl[j][i];
  if (s == -1.2345f) sink[ln] = s;
}

}  // namespace dmpc

using namespace dmpc;

extern "C" dmpc_err dmpc_probe_fp32_peak(double* tflops_out, double* ms_out) {
  if (!tflops_out) return DMPC_E_ARG;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DMPC_E_CUDA;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DMPC_E_CUDA;
  const int threads = 1024, blocks = 2 * n_sm, iters = 1 << 16;
  float* sink = nullptr;  // the probe's one allocation: it runs outside any solve
  if (cudaMalloc(&sink, sizeof(float) * threads * blocks) != cudaSuccess) return DMPC_E_OOM;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) { cudaFree(sink); return DMPC_E_CUDA; }
  probe_fma_kernel<<<blocks, threads>>>(sink, iters / 16, 0.9999f, 1e-4f);  // warm-up
  float best = 1e30f;
  for (int rep = 0; rep < 5; ++rep) {
    cudaEventRecord(e0);
    probe_fma_kernel<<<blocks, threads>>>(sink, iters, 0.9999f, 1e-4f);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = ms < best ? ms : best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (cudaGetLastError() != cudaSuccess || best > 1e29f) return DMPC_E_CUDA;
  const double flops = 2.0 * kPeakChains * (double)iters * threads * blocks;
  *tflops_out = flops / (best * 1e-3) / 1e12;
  if (ms_out) *ms_out = best;
  return DMPC_OK;
}

extern "C" dmpc_err dmpc_probe_pcg_floor(int iters, double* us_per_iter_out) {
  if (!us_per_iter_out || iters < 1 || iters > (1 << 24)) return DMPC_E_ARG;
  int* d_done = nullptr;  // the probe's allocations: it runs outside any solve
  float* sink = nullptr;
  if (cudaMalloc(&d_done, sizeof(int)) != cudaSuccess) return DMPC_E_OOM;
  if (cudaMalloc(&sink, sizeof(float) * 32) != cudaSuccess) { cudaFree(d_done); return DMPC_E_OOM; }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaFree(d_done);
    cudaFree(sink);
    return DMPC_E_CUDA;
  }
  probe_pcg_kernel<<<1, 32>>>(iters / 8 + 1, d_done, sink);  // warm-up
  float best = 1e30f;
  int done = 0;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    probe_pcg_kernel<<<1, 32>>>(iters, d_done, sink);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = ms < best ? ms : best;
  }
  cudaError_t e = cudaMemcpy(&done, d_done, sizeof(int), cudaMemcpyDeviceToHost);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d_done);
  cudaFree(sink);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess || done < 1) return DMPC_E_CUDA;
  *us_per_iter_out = best * 1e3 / done;
  return DMPC_OK;
}
