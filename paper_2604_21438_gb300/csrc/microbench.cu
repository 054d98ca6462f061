// microbench.cu -- FMA-throughput microbenchmarks used as measured ALU
// denominators of the roofline (FP64 and FP32 vector pipes), and device
// checks of the solver's FP32 math functions and of its integer FP32 <-> FP64
// conversions against CUDA's.  Each FMA thread
// runs 8 independent chains in registers; one launch covers every SM several
// times over.  Not part of the solver.
#include <cuda_runtime.h>
#include <cstdint>
#include "li_device.cuh"

template <typename T>
__global__ void __launch_bounds__(256) fma_chain(T *out, int iters, T a, T b) {
  T x0 = T(threadIdx.x) * T(1e-3), x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
  T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
      x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
  }
  T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == T(-1.2345)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never true; keeps the chains live
}

template <typename T>
static int run(int iters, int blocks_per_sm, double *flops_per_s, float *ms_out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  const int grid = sms * blocks_per_sm, tpb = 256;
  T *out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * grid * tpb) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_chain<T><<<grid, tpb>>>(out, iters / 4 + 1, T(0.999999), T(1e-7));   // warm-up
  cudaEventRecord(e0);
  fma_chain<T><<<grid, tpb>>>(out, iters, T(0.999999), T(1e-7));
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return 1;
  const double flops = 2.0 * 8.0 * 16.0 * double(iters) * double(grid) * double(tpb);
  *flops_per_s = flops / (double(ms) * 1e-3);
  *ms_out = ms;
  return 0;
}

extern "C" int sfbench_fma_fp64(int iters, double *flops_per_s, float *ms) {
  return run<double>(iters, 8, flops_per_s, ms);
}
extern "C" int sfbench_fma_fp32(int iters, double *flops_per_s, float *ms) {
  return run<float>(iters, 8, flops_per_s, ms);
}

// fn: 0 exp, 1 log, 2 rcp, 3 sqrt.  ours[i] = the solver's M<float> function
// of x[i], ref[i] = CUDA's expf / logf / 1.0f / x / sqrtf.  Host buffers.
// sfbench_rcp64_check: ours[i] = M<double>::rcp(x[i]), ref[i] = 1.0 / x[i].
__global__ void math_check(int fn, int n, const float *x, float *ours, float *ref) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = x[i];
  typedef sfc::M<float> m;
  float a = 0.f, b = 0.f;
  if (fn == 0) { a = m::exp(v); b = expf(v); }
  else if (fn == 1) { a = m::log(v); b = logf(v); }
  else if (fn == 2) { a = m::rcp(v); b = 1.0f / v; }
  else { a = m::sqrt(v); b = sqrtf(v); }
  ours[i] = a;
  ref[i] = b;
}

extern "C" int sfbench_math_check(int fn, int n, const float *x, float *ours, float *ref) {
  if (n <= 0 || fn < 0 || fn > 3 || !x || !ours || !ref) return 1;
  float *d = nullptr;
  if (cudaMalloc(&d, sizeof(float) * 3 * (size_t)n) != cudaSuccess) return 1;
  int rc = 0;
  if (cudaMemcpy(d, x, sizeof(float) * n, cudaMemcpyHostToDevice) != cudaSuccess) rc = 1;
  if (!rc) {
    math_check<<<(n + 255) / 256, 256>>>(fn, n, d, d + n, d + 2 * (size_t)n);
    if (cudaGetLastError() != cudaSuccess) rc = 1;
  }
  if (!rc && cudaMemcpy(ours, d + n, sizeof(float) * n, cudaMemcpyDeviceToHost) != cudaSuccess) rc = 1;
  if (!rc && cudaMemcpy(ref, d + 2 * (size_t)n, sizeof(float) * n, cudaMemcpyDeviceToHost) != cudaSuccess) rc = 1;
  cudaFree(d);
  return rc;
}

// The mixed path's integer conversions against the hardware ones: f2d_ours[i]
// = f2d_int(xf[i]) (FIN: f2d_fin), f2d_ref[i] = (double)xf[i]; d2f_ours[i] =
// d2f_int(xd[i]) (FIN: d2f_fin), d2f_ref[i] = __double2float_rn(xd[i]).  Host
// buffers of n elements each.
template <bool FIN>
__global__ void conv_check(int n, const float *xf, double *f2d_ours, double *f2d_ref, const double *xd,
                           float *d2f_ours, float *d2f_ref) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  f2d_ours[i] = FIN ? sfc::f2d_fin(xf[i]) : sfc::f2d_int(xf[i]);
  f2d_ref[i] = (double)xf[i];
  d2f_ours[i] = FIN ? sfc::d2f_fin(xd[i]) : sfc::d2f_int(xd[i]);
  d2f_ref[i] = __double2float_rn(xd[i]);
}

namespace {
int conv_check_run(bool fin, int n, const float *xf, double *f2d_ours, double *f2d_ref, const double *xd,
                   float *d2f_ours, float *d2f_ref) {
  if (n <= 0 || !xf || !f2d_ours || !f2d_ref || !xd || !d2f_ours || !d2f_ref) return 1;
  const size_t N = (size_t)n;
  char *d = nullptr;
  const size_t bytes = N * (sizeof(float) * 3 + sizeof(double) * 3);
  if (cudaMalloc(&d, bytes) != cudaSuccess) return 1;
  double *dxd = (double *)d, *dfo = dxd + N, *dfr = dfo + N;
  float *dxf = (float *)(dfr + N), *ddo = dxf + N, *ddr = ddo + N;
  int rc = 0;
  if (cudaMemcpy(dxf, xf, sizeof(float) * N, cudaMemcpyHostToDevice) != cudaSuccess) rc = 1;
  if (!rc && cudaMemcpy(dxd, xd, sizeof(double) * N, cudaMemcpyHostToDevice) != cudaSuccess) rc = 1;
  if (!rc) {
    if (fin)
      conv_check<true><<<(n + 255) / 256, 256>>>(n, dxf, dfo, dfr, dxd, ddo, ddr);
    else
      conv_check<false><<<(n + 255) / 256, 256>>>(n, dxf, dfo, dfr, dxd, ddo, ddr);
    if (cudaGetLastError() != cudaSuccess) rc = 1;
  }
  if (!rc && cudaMemcpy(f2d_ours, dfo, sizeof(double) * N, cudaMemcpyDeviceToHost) != cudaSuccess) rc = 1;
  if (!rc && cudaMemcpy(f2d_ref, dfr, sizeof(double) * N, cudaMemcpyDeviceToHost) != cudaSuccess) rc = 1;
  if (!rc && cudaMemcpy(d2f_ours, ddo, sizeof(float) * N, cudaMemcpyDeviceToHost) != cudaSuccess) rc = 1;
  if (!rc && cudaMemcpy(d2f_ref, ddr, sizeof(float) * N, cudaMemcpyDeviceToHost) != cudaSuccess) rc = 1;
  cudaFree(d);
  return rc;
}
}  // namespace

extern "C" int sfbench_conv_check(int n, const float *xf, double *f2d_ours, double *f2d_ref, const double *xd,
                                  float *d2f_ours, float *d2f_ref) {
  return conv_check_run(false, n, xf, f2d_ours, f2d_ref, xd, d2f_ours, d2f_ref);
}

extern "C" int sfbench_conv_check_fin(int n, const float *xf, double *f2d_ours, double *f2d_ref, const double *xd,
                                      float *d2f_ours, float *d2f_ref) {
  return conv_check_run(true, n, xf, f2d_ours, f2d_ref, xd, d2f_ours, d2f_ref);
}

__global__ void rcp64_check(int n, const double *x, double *ours, double *ref) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  ours[i] = sfc::M<double>::rcp(x[i]);
  ref[i] = 1.0 / x[i];
}

extern "C" int sfbench_rcp64_check(int n, const double *x, double *ours, double *ref) {
  if (n <= 0 || !x || !ours || !ref) return 1;
  double *d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * 3 * (size_t)n) != cudaSuccess) return 1;
  int rc = 0;
  if (cudaMemcpy(d, x, sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess) rc = 1;
  if (!rc) {
    rcp64_check<<<(n + 255) / 256, 256>>>(n, d, d + n, d + 2 * (size_t)n);
    if (cudaGetLastError() != cudaSuccess) rc = 1;
  }
  if (!rc && cudaMemcpy(ours, d + n, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess) rc = 1;
  if (!rc && cudaMemcpy(ref, d + 2 * (size_t)n, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess) rc = 1;
  cudaFree(d);
  return rc;
}
