// Observables: energies (Eq. sl_hamiltonian, each unordered pair once),
// magnetisation M = (1/N) sum_i s_i, and the sums behind T_L
// (Eq. lattice_temperature) and T_S (Eq. spin_temperature), per replica.
//
// Deterministic: every atom writes its terms to its caller-order slot; one
// block per replica then sums its contiguous range in a fixed order.
#include "sl_internal.cuh"
#include "sl_df64.cuh"
#include "sl_pair.cuh"

namespace {

constexpr int RED_THREADS = 256;

__global__ void k_obs_atoms(SlDev d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  const SlRep& R = d.reps[d.arep[i]];
  const double4_32a v = d.v[i], si = d.s[i], ri = d.r[i];
  double q[SL_NOBS];
  q[0] = 0.5 * d.mass * (v.x * v.x + v.y * v.y + v.z * v.z) / SL_FTOA;
  double em = 0.0;
  const int nm = (d.ham == SL_HAM_LEARNED && d.ctrl->ml_use) ? 0 : d.mn[i];
  double rho = 0.0;
  for (int k = 0; k < nm; ++k) {
    const int j = d.mj[(size_t)k * d.n + i];
    const double3 dd = sl_min_image(R, ri, d.r[j]);
    const double r2 = dd.x * dd.x + dd.y * dd.y + dd.z * dd.z;
    if (d.mech & SL_MECH_TAB) {
      // tabulated form: phi(r) and rho(r) inside the Morse cutoff
      if (r2 < d.m_rc2) {
        const double r = sqrt(r2);
        em += tab_value_d(d, SL_TAB_PHI, r);
        rho += tab_value_d(d, SL_TAB_RHO, r);
      }
      continue;
    }
    if (r2 < d.m_rc2) {
      const double e = exp(-d.m_alpha * (sqrt(r2) - d.m_r0));
      em += d.m_D0 * (e * e - 2.0 * e) - d.m_vshift;
    }
    if ((d.mech & SL_MECH_EAM) && r2 < d.em_d * d.em_d) {
      const double x = sqrt(r2) - d.em_d;
      rho += x * x + d.em_beta * x * x * x / d.em_d;
    }
  }
  q[1] = 0.5 * em;
  // embedding energy, one per atom: F(rho_i) = -A sqrt(rho_i), or the table's
  if (d.mech & SL_MECH_TAB) q[1] += tab_value_d(d, SL_TAB_F, rho);
  else if (d.mech & SL_MECH_EAM) q[1] += rho > 0.0 ? -d.em_A * sqrt(rho) : 0.0;
  double hx = d.zee[0], hy = d.zee[1], hz = d.zee[2];
  double ex = 0.0;
  const bool learned = d.ham == SL_HAM_LEARNED && d.ctrl->ml_use;
  if (learned) {
    // the network's energy E_i (lattice + exchange together) and field -dE/ds_i
    const float4 b = d.ml_B[i];
    q[1] = (double)d.ml_e[i];
    hx += b.x; hy += b.y; hz += b.z;
  }
  const int ne = learned ? 0 : d.exn[i];
  double eso = 0.0;
  for (int k = 0; k < ne; ++k) {
    const size_t e = (size_t)k * d.n + i;
    const float2 J2 = d.exJ[e];
    const double J = double_from_float(J2.x) + double_from_float(J2.y);
    const double4_32a sj = d.s[d.exj[e]];
    ex += J * (si.x * sj.x + si.y * sj.y + si.z * sj.z);
    if (d.mech & SL_MECH_GROUND) q[1] += 0.5 * J;   // + J(r) per unordered pair
    hx = fma(J, sj.x, hx); hy = fma(J, sj.y, hy); hz = fma(J, sj.z, hz);
    if (d.exso) {
      so_field_d(d, e, sj, hx, hy, hz);
      eso += so_pair_energy_d(d, e, si, sj);
    }
  }
  q[2] = -0.5 * ex;
  q[10] = 0.5 * eso;
  if (d.so & SL_SO_ANISO) {
    const double sn = si.x * d.an_n[0] + si.y * d.an_n[1] + si.z * d.an_n[2];
    q[10] -= d.an_K * sn * sn;
    hx += 2.0 * d.an_K * sn * d.an_n[0]; hy += 2.0 * d.an_K * sn * d.an_n[1]; hz += 2.0 * d.an_K * sn * d.an_n[2];
  }
  q[3] = -(d.zee[0] * si.x + d.zee[1] * si.y + d.zee[2] * si.z);
  q[4] = si.x; q[5] = si.y; q[6] = si.z;
  const double ih = 1.0 / SL_HBAR;
  const double wx = hx * ih, wy = hy * ih, wz = hz * ih;
  const double cx = si.y * wz - si.z * wy, cy = si.z * wx - si.x * wz, cz = si.x * wy - si.y * wx;
  q[7] = cx * cx + cy * cy + cz * cz;
  q[8] = si.x * wx + si.y * wy + si.z * wz;
  const double t = v.x + v.y + v.z + si.x + si.y + si.z + ri.x + ri.y + ri.z;
  q[9] = (t - t == 0.0) ? 0.0 : 1.0;
  double* out = d.obs_atom + (size_t)d.perm[i] * SL_NOBS;
#pragma unroll
  for (int c = 0; c < SL_NOBS; ++c) out[c] = q[c];
}

// One block per replica: fixed-order strided sums, then a fixed tree.
__global__ void k_obs_reps(SlDev d) {
  __shared__ double sh[SL_NOBS][RED_THREADS];
  const SlRep& R = d.reps[blockIdx.x];
  double q[SL_NOBS];
#pragma unroll
  for (int c = 0; c < SL_NOBS; ++c) q[c] = 0.0;
  for (int k = threadIdx.x; k < R.natoms; k += RED_THREADS) {
    const double* a = d.obs_atom + (size_t)(R.atom0 + k) * SL_NOBS;
#pragma unroll
    for (int c = 0; c < SL_NOBS; ++c) q[c] += a[c];
  }
#pragma unroll
  for (int c = 0; c < SL_NOBS; ++c) sh[c][threadIdx.x] = q[c];
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < SL_NOBS; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < SL_NOBS) {
    d.obs_rep[(size_t)blockIdx.x * SL_NOBS + threadIdx.x] = sh[threadIdx.x][0];
    if (threadIdx.x == 9 && sh[9][0] > 0.0) sl_set_error(d.ctrl, SL_ERR_NONFINITE);
  }
}

}  // namespace

int sl_launch_observables(const SlDev& d, cudaStream_t st) {
  k_obs_atoms<<<(d.n + SL_BLOCK - 1) / SL_BLOCK, SL_BLOCK, 0, st>>>(d);
  k_obs_reps<<<d.nrep, RED_THREADS, 0, st>>>(d);
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}
