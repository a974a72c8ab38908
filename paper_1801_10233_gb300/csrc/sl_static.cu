// Allocation-free magnetisation of a caller's spin array.
//
// For callers that cannot allocate device memory themselves: code running
// where cudaMalloc is unavailable or forbidden (inside another library's
// allocator hooks, a plugin that only receives device pointers, or a process
// that must not grow its device footprint after start-up).  The entry point
// sl_magnetization_static below needs no context and no workspace: the block
// partial sums of its reduction live in a file-scope device array of fixed
// size that every GPU loading this library holds until the process exits.
#include <mutex>

#include "sl_internal.cuh"

namespace {

constexpr int kStaticBlock = 256;
constexpr int kStaticMaxAtoms = 1 << 21;                       // 2,097,152 spins
constexpr int kStaticMaxBlocks = kStaticMaxAtoms / kStaticBlock;  // 8,192 partials

// One partial (Mx, My, Mz, pad) per block: 8,192 x 32 B = 256 KB per device.
static __device__ __align__(256) double g_static_partials[kStaticMaxBlocks * 4];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_partials_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code may not use the symbol itself as a pointer).
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SL_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_partials) != cudaSuccess || !p) {
      cudaGetLastError();
      return SL_ERR_CUDA;
    }
    g_partials_addr[dev] = (double*)p;
  }
  *out = g_partials_addr[dev];
  return SL_OK;
}

// Pass 1: each block sums its 256 spins in a fixed tree order and writes its
// partial (every block writes its slot, so nothing has to start at zero).
__global__ void k_mag_partials(const double* __restrict__ s, int n, double* part) {
  __shared__ double sh[3][kStaticBlock];
  int i = blockIdx.x * kStaticBlock + threadIdx.x;
  double x = 0.0, y = 0.0, z = 0.0;
  if (i < n) { x = s[3 * (size_t)i]; y = s[3 * (size_t)i + 1]; z = s[3 * (size_t)i + 2]; }
  sh[0][threadIdx.x] = x; sh[1][threadIdx.x] = y; sh[2][threadIdx.x] = z;
  __syncthreads();
  for (int w = kStaticBlock / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) part[4 * (size_t)blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

// Pass 2: one thread per component sums the partials in block order.
__global__ void k_mag_final(const double* part, int nblk, int n, double* out) {
  __shared__ double m[3];
  int c = threadIdx.x;
  if (c < 3) {
    double acc = 0.0;
    for (int b = 0; b < nblk; ++b) acc += part[4 * (size_t)b + c];
    m[c] = acc / (double)n;
  }
  __syncthreads();
  if (c < 3) out[c] = m[c];
  if (c == 0) out[3] = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
}

}  // namespace

extern "C" int sl_magnetization_static(const double* s, int32_t n_atoms, double* out, void* cuda_stream) {
  if (!s || !out || n_atoms < 1) return SL_ERR_ARG;
  if (n_atoms > kStaticMaxAtoms) return SL_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the scratch address is the current device's: a stream of another device
  // is a caller error, reported before any launch
  int cur = 0, sdev = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return SL_ERR_CUDA;
  if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) {
    cudaGetLastError();
    return SL_ERR_ARG;
  }
  if (sdev != cur) return SL_ERR_ARG;
  double* part = nullptr;
  int e = scratch_address(&part);
  if (e) return e;
  int nblk = (n_atoms + kStaticBlock - 1) / kStaticBlock;
  k_mag_partials<<<nblk, kStaticBlock, 0, st>>>(s, n_atoms, part);
  k_mag_final<<<1, 32, 0, st>>>(part, nblk, n_atoms, out);
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}
