// Measured throughput of the double-float multiply-add that the pair and
// rotation kernels are built from (df_fma of sl_df64.cuh): the compute roof
// of FP64-accurate arithmetic on the FP32 pipes of the current device.
//
// Every thread runs SL_PROBE_CHAINS independent chains a <- a b + c (the
// chains give each warp enough independent instructions to fill the FP32
// pipes), with |b| < 1 so the values stay finite; the grid is 4 blocks of
// 256 threads per SM.  Each multiply-add counts as 2 flop.
#include "sl_internal.cuh"
#include "sl_df64.cuh"
#include "sl_tc.cuh"

namespace {

constexpr int SL_PROBE_CHAINS = 8;
constexpr int SL_PROBE_THREADS = 256;

// Written only when a result equals an improbable value, so the compiler
// keeps the work without the kernel needing an output buffer.
__device__ float2 g_probe_sink;

__global__ void __launch_bounds__(SL_PROBE_THREADS) k_df_fma_rate(float2 bc0, float2 bc1, int iters) {
  const df b = df_make(bc0.x, bc0.y), c = df_make(bc1.x, bc1.y);
  df a[SL_PROBE_CHAINS];
#pragma unroll
  for (int j = 0; j < SL_PROBE_CHAINS; ++j) a[j] = df_make(1e-3f * (float)threadIdx.x + (float)j, 0.0f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < SL_PROBE_CHAINS; ++j) a[j] = df_fma(a[j], b, c);
  }
  df s = a[0];
#pragma unroll
  for (int j = 1; j < SL_PROBE_CHAINS; ++j) s = df_add(s, a[j]);
  if (s.hi == 12345.0f) g_probe_sink = make_float2(s.hi, s.lo);
}

// The bounded wait of the tensor-core kernels (mbar_wait_ns) on a barrier
// of count 1: completed by one arrival (arrive = 1) or by nothing.
__device__ int g_wait_status;
__global__ void k_bounded_wait(unsigned long long limit_ns, int arrive) {
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t b = smem_u32(&bar);
  if (threadIdx.x == 0) mbar_init(b, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (arrive) mbar_arrive(b);
    g_wait_status = mbar_wait_ns(b, 0, limit_ns) ? SL_OK : SL_ERR_TIMEOUT;
  }
}

// y = f(x) through the double-float functions: x to df (48 bits), the
// function, back to FP64.
__global__ void k_df_eval(int fn, const double* x, double* y, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const df a = df_from_double(x[k]);
  df r;
  if (fn == SL_DF_EXP) r = df_exp(a);
  else if (fn == SL_DF_RSQRT) r = df_rsqrt(a);
  else r = df_sqrt(a);
  y[k] = df_to_double(r);
}

}  // namespace

extern "C" int sl_check_bounded_wait(int64_t limit_ns, int32_t arrive, int32_t* status) {
  if (!status || limit_ns < 0 || limit_ns > 2000000000LL) return SL_ERR_ARG;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return SL_ERR_CUDA;
  int rc = SL_OK;
  int v = SL_ERR_CUDA;
  k_bounded_wait<<<1, 32, 0, st>>>((unsigned long long)limit_ns, arrive ? 1 : 0);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess ||
      cudaMemcpyFromSymbol(&v, g_wait_status, sizeof(int)) != cudaSuccess)
    rc = SL_ERR_CUDA;
  cudaStreamDestroy(st);
  if (rc == SL_OK) *status = v;
  return rc;
}

extern "C" int sl_df_eval(int32_t fn, const double* x, double* y, int64_t n, void* cuda_stream) {
  if (fn < SL_DF_EXP || fn > SL_DF_SQRT || n < 0 || (n > 0 && (!x || !y))) return SL_ERR_ARG;
  if (n == 0) return SL_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int64_t blocks = (n + 255) / 256;
  if (blocks > 0x7fffffffLL) return SL_ERR_ARG;
  k_df_eval<<<(unsigned)blocks, 256, 0, st>>>(fn, x, y, n);
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}

extern "C" int sl_df_fma_rate(int32_t iters, double* flop_per_s, double* ms) {
  if (!flop_per_s || iters < 1 || iters > (1 << 20)) return SL_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return SL_ERR_CUDA;
  const int blocks = 4 * sms;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = SL_ERR_CUDA;
  float best = 0.0f;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return SL_ERR_CUDA;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    const float2 b = make_float2(0.99999988f, 1.3e-9f), c = make_float2(0.25f, -2.1e-10f);
    rc = SL_OK;
    // one warm-up launch, then the best of three timed launches
    for (int rep = 0; rep < 4 && rc == SL_OK; ++rep) {
      cudaEventRecord(e0, st);
      k_df_fma_rate<<<blocks, SL_PROBE_THREADS, 0, st>>>(b, c, iters);
      cudaEventRecord(e1, st);
      float t = 0.0f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess ||
          cudaGetLastError() != cudaSuccess)
        rc = SL_ERR_CUDA;
      else if (rep > 0 && (best == 0.0f || t < best))
        best = t;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (rc != SL_OK || !(best > 0.0f)) return rc != SL_OK ? rc : SL_ERR_CUDA;
  const double fmas = (double)blocks * SL_PROBE_THREADS * (double)iters * SL_PROBE_CHAINS;
  *flop_per_s = 2.0 * fmas / (best * 1e-3);
  if (ms) *ms = best;
  return SL_OK;
}
