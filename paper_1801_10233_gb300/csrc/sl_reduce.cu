// Observables: energies (Eq. sl_hamiltonian, each unordered pair once),
// magnetisation M = (1/N) sum_i s_i, and the sums behind T_L
// (Eq. lattice_temperature) and T_S (Eq. spin_temperature).
//
// Deterministic: per-block partials in a fixed tree order, then one thread
// per quantity sums the block partials in block order.
#include "sl_internal.cuh"
#include "sl_df64.cuh"

namespace {

constexpr int NQ = 10;  // Ek, Em, Ex, Ez, Mx, My, Mz, TSnum, TSden, nonfinite

__global__ void k_obs(SlDev d) {
  __shared__ double sh[NQ][SL_BLOCK];
  double q[NQ];
#pragma unroll
  for (int c = 0; c < NQ; ++c) q[c] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n; i += gridDim.x * blockDim.x) {
    double4_32a v = d.v[i], si = d.s[i], ri = d.r[i];
    q[0] += 0.5 * d.mass * (v.x * v.x + v.y * v.y + v.z * v.z) / SL_FTOA;
    double em = 0.0;
    int nm = d.mn[i];
    for (int k = 0; k < nm; ++k) {
      int j = d.mj[(size_t)k * d.n + i];
      double3 dd = sl_min_image(d, ri, d.r[j]);
      double r2 = dd.x * dd.x + dd.y * dd.y + dd.z * dd.z;
      if (r2 < d.m_rc2) {
        double e = exp(-d.m_alpha * (sqrt(r2) - d.m_r0));
        em += d.m_D0 * (e * e - 2.0 * e) - d.m_vshift;
      }
    }
    q[1] += 0.5 * em;
    double hx = d.zee[0], hy = d.zee[1], hz = d.zee[2];
    double ex = 0.0;
    int ne = d.exn[i];
    for (int k = 0; k < ne; ++k) {
      const size_t e = (size_t)k * d.n + i;
      const float2 J2 = d.exJ[e];
      double J = double_from_float(J2.x) + double_from_float(J2.y);
      double4_32a sj = d.s[d.exj[e]];
      ex += J * (si.x * sj.x + si.y * sj.y + si.z * sj.z);
      hx = fma(J, sj.x, hx); hy = fma(J, sj.y, hy); hz = fma(J, sj.z, hz);
    }
    q[2] -= 0.5 * ex;
    q[3] -= d.zee[0] * si.x + d.zee[1] * si.y + d.zee[2] * si.z;
    q[4] += si.x; q[5] += si.y; q[6] += si.z;
    const double ih = 1.0 / SL_HBAR;
    double wx = hx * ih, wy = hy * ih, wz = hz * ih;
    double cx = si.y * wz - si.z * wy, cy = si.z * wx - si.x * wz, cz = si.x * wy - si.y * wx;
    q[7] += cx * cx + cy * cy + cz * cz;
    q[8] += si.x * wx + si.y * wy + si.z * wz;
    double t = v.x + v.y + v.z + si.x + si.y + si.z + ri.x + ri.y + ri.z;
    if (!(t - t == 0.0)) q[9] += 1.0;
  }
#pragma unroll
  for (int c = 0; c < NQ; ++c) sh[c][threadIdx.x] = q[c];
  __syncthreads();
  for (int w = SL_BLOCK / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < NQ; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < NQ) d.part[(size_t)blockIdx.x * 16 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_obs_final(SlDev d, int nblk) {
  int c = threadIdx.x;
  if (c >= NQ) return;
  double acc = 0.0;
  for (int b = 0; b < nblk; ++b) acc += d.part[(size_t)b * 16 + c];
  d.ctrl->red[c] = acc;
  if (c == 9 && acc > 0.0) sl_set_error(d.ctrl, SL_ERR_NONFINITE);
}

}  // namespace

int sl_launch_observables(const SlDev& d, cudaStream_t st) {
  int g = (d.n + SL_BLOCK - 1) / SL_BLOCK;
  if (g > d.nblk_red) g = d.nblk_red;
  if (g < 1) g = 1;
  k_obs<<<g, SL_BLOCK, 0, st>>>(d);
  k_obs_final<<<1, 32, 0, st>>>(d, g);
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}
