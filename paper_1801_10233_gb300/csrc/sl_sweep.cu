// The colour passes of the plain Hamiltonian (and the exchange-only
// asynchronous-gather pass): tile shapes 0-9 (sl_sweep.cuh).
#include "sl_sweep.cuh"

namespace {

template <bool SO>
void launch_half_op_shapes(const SlDev& d, cudaStream_t st, int subpass0) {
  switch (d.tune_sweep % 5) {
    case 1: launch_half_op_t<32, 256, SO>(d, st, subpass0); break;
    case 2: launch_half_op_t<16, 128, SO>(d, st, subpass0); break;
    case 3: launch_half_op_t<16, 128, SO, 1024>(d, st, subpass0); break;
    case 4: launch_half_op_t<8, 128, SO>(d, st, subpass0); break;
    default: launch_half_op_t<32, 192, SO>(d, st, subpass0); break;
  }
}

// Allow the sweep's dynamic shared memory (above the 48 KB default).
template <bool SO>
bool prepare_sweep() {
  bool ok = true;
  ok &= cudaFuncSetAttribute(k_sweep_pass<32, 192, SO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sweep_smem_bytes(true, 12 * 32, true, true)) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_sweep_pass<32, 256, SO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sweep_smem_bytes(true, 12 * 32, true, true)) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_sweep_pass<16, 128, SO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sweep_smem_bytes(true, 12 * 16, true, true)) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_sweep_pass<16, 128, SO, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sweep_smem_bytes(true, 12 * 16, true, true)) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_sweep_pass<8, 128, SO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sweep_smem_bytes(true, 12 * 8, true, true)) == cudaSuccess;
  return ok;
}

template <int SPB, int THREADS, int MAXA>
bool prepare_async() {
  return cudaFuncSetAttribute(k_sweep_async<SPB, THREADS, MAXA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sweep_async_smem(true, MAXA)) == cudaSuccess;
}

}  // namespace

int sl_prepare_sweep_plain() {
  const bool ok = prepare_sweep<false>() && prepare_async<16, 128, 128>() && prepare_async<8, 64, 64>() &&
                  prepare_async<32, 256, 256>() && prepare_async<8, 96, 96>() && prepare_async<4, 64, 48>();
  return ok ? SL_OK : SL_ERR_CUDA;
}

// Tile shapes: variants 0-4 are the pipelined pass k_sweep_pass (sectors per
// block 32, 32, 16, 16, 8 x 192, 256, 128, 128, 128 threads; variant 3 with
// registers for 1,024 threads per SM, the others 768); variants 5-9 the
// asynchronous-gather pass k_sweep_async (16, 8, 32, 8, 4 sectors x 128, 64,
// 256, 96, 64 threads, up to 128, 64, 256, 96, 48 atoms per block in shared
// memory).
void sl_launch_half_op_plain(const SlDev& d, cudaStream_t st, int subpass0) {
  switch (d.tune_sweep) {
    case 5: launch_half_op_async_t<16, 128, 128>(d, st, subpass0); break;
    case 6: launch_half_op_async_t<8, 64, 64>(d, st, subpass0); break;
    case 7: launch_half_op_async_t<32, 256, 256>(d, st, subpass0); break;
    case 8: launch_half_op_async_t<8, 96, 96>(d, st, subpass0); break;
    case 9: launch_half_op_async_t<4, 64, 48>(d, st, subpass0); break;
    default: launch_half_op_shapes<false>(d, st, subpass0); break;
  }
}
