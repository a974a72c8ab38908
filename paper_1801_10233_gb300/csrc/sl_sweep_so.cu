// The colour passes with the spin-orbit terms (anisotropy, Neel, DMI): the
// pipelined pass in tile shapes 0-4; shapes 5-9 run as 0-4 (sl_sweep.cuh).
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
}  // namespace

int sl_prepare_sweep_so() { return prepare_sweep<true>() ? SL_OK : SL_ERR_CUDA; }

void sl_launch_half_op_so(const SlDev& d, cudaStream_t st, int subpass0) {
  launch_half_op_shapes<true>(d, st, subpass0);
}
