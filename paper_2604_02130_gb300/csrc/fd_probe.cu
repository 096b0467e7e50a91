// fd_probe.cu -- FP64 FMA throughput probe (the roofline denominator of the FP64 pipe).
//
// Every thread runs 8 independent chains of dependent DFMAs; the result is written so the
// compiler cannot drop the work.  GFLOP/s = 2 * grid * threads * iters * 8 / time.
#include "fd_fp64.cuh"
#include "fd_kernels.h"

namespace fd {

__global__ void k_fp64_probe(int iters, double* sink) {
  double a0 = threadIdx.x * 1e-9, a1 = a0 + 1e-10, a2 = a0 + 2e-10, a3 = a0 + 3e-10;
  double a4 = a0 + 4e-10, a5 = a0 + 5e-10, a6 = a0 + 6e-10, a7 = a0 + 7e-10;
  const double m = 0.9999999, c = 1e-12;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
      a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
    }
  }
  double s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == 12345.678) sink[threadIdx.x] = s;  // practically never; keeps the chains live
}

cudaError_t run_fp64_probe(int grid, int threads, int iters, double* out, cudaStream_t stream) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double* sink = nullptr;
  cudaError_t err = cudaMalloc(&sink, sizeof(double) * threads);
  if (err != cudaSuccess) return err;
  k_fp64_probe<<<grid, threads, 0, stream>>>(iters / 8 + 1, sink);  // warm-up
  cudaEventRecord(e0, stream);
  k_fp64_probe<<<grid, threads, 0, stream>>>(iters, sink);
  cudaEventRecord(e1, stream);
  err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaFree(sink);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return err;
  double flops = 2.0 * grid * threads * (double)iters * 16.0 * 8.0;
  *out = flops / (ms * 1e-3) / 1e9;
  return cudaGetLastError();
}

// Issue cost of FP64 instructions, from inside one CTA: cycles per DFMA of one warp running one
// dependent chain with `lanes` active lanes (1 or 32), and with `warps` warps each running eight
// independent chains (the SM's shared FP64 throughput).  out[0] = cycles per instruction.
__global__ void k_fp64_issue(int lanes, int chains8, int iters, long long* out, double* sink) {
  const int lane = threadIdx.x & 31;
  double a0 = 1.0 + lane * 1e-9, a1 = a0 + 1e-10, a2 = a0 + 2e-10, a3 = a0 + 3e-10;
  double a4 = a0 + 4e-10, a5 = a0 + 5e-10, a6 = a0 + 6e-10, a7 = a0 + 7e-10;
  const double m = 0.999999999, c = 1e-12;
  __syncthreads();
  const long long t0 = clock64();
  if (lane < lanes) {
    if (!chains8) {
      for (int i = 0; i < iters; ++i) a0 = fma(a0, m, c);
    } else {
      for (int i = 0; i < iters; ++i) {
        a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
        a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
      }
    }
  }
  __syncwarp();
  const long long t1 = clock64();
  if (threadIdx.x == 0) out[0] = t1 - t0;
  const double s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == 42.0) sink[lane] = s;
}

cudaError_t run_fp64_issue(double* out3) {
  long long* d_out = nullptr;
  double* sink = nullptr;
  cudaError_t e = cudaMalloc(&d_out, sizeof(long long));
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&sink, 32 * sizeof(double));
  if (e != cudaSuccess) {
    cudaFree(d_out);
    return e;
  }
  const int iters = 4096;
  struct Case { int threads, lanes, chains8; } cases[3] = {{32, 1, 0}, {32, 32, 0}, {256, 32, 1}};
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    k_fp64_issue<<<1, cases[i].threads>>>(cases[i].lanes, cases[i].chains8, 64, d_out, sink);
    k_fp64_issue<<<1, cases[i].threads>>>(cases[i].lanes, cases[i].chains8, iters, d_out, sink);
    long long cyc = 0;
    e = cudaMemcpy(&cyc, d_out, sizeof(cyc), cudaMemcpyDeviceToHost);
    out3[i] = (double)cyc / ((double)iters * (cases[i].chains8 ? 8 : 1));
  }
  cudaFree(d_out);
  cudaFree(sink);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

// Self-check of the hand-written FP64 refinements used by the QR and LU steps (rcp64, rsqrt64,
// sqrt64 and reflector_math), each beside CUDA's correctly rounded IEEE operations on the same
// argument: out[16 i + k] for argument i --
//   0 rcp64(x)   1 __drcp_rn(x)   2 rsqrt64(x)   3 __drcp_rn(__dsqrt_rn(x))   4 sqrt64(x)
//   5 __dsqrt_rn(x)   6, 7 alpha   8, 9 1/c   10 tau   11 zero flag  of reflector_math(x + i y, z)
//   12..15 zero.
__global__ void k_refine_check(const double* x, const double* y, const double* z, int n,
                               double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = x[i];
  double* o = out + 16 * (size_t)i;
  o[0] = rcp64(a);
  o[1] = __drcp_rn(a);
  o[2] = rsqrt64(a);
  o[3] = __drcp_rn(__dsqrt_rn(a));
  o[4] = sqrt64(a);
  o[5] = __dsqrt_rn(a);
  const Refl r = reflector_math(cx(a, y[i]), z[i]);
  o[6] = r.alpha.re;
  o[7] = r.alpha.im;
  o[8] = r.cinv.re;
  o[9] = r.cinv.im;
  o[10] = r.tau;
  o[11] = r.zero ? 1.0 : 0.0;
  for (int k = 12; k < 16; ++k) o[k] = 0.0;
}

cudaError_t run_refine_check(const double* x, const double* y, const double* z, int n,
                             double* out, cudaStream_t stream) {
  if (n > 0) k_refine_check<<<(n + 127) / 128, 128, 0, stream>>>(x, y, z, n, out);
  return cudaGetLastError();
}

}  // namespace fd
