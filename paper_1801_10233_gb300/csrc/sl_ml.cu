// Learned per-atom Hamiltonian: descriptors, the network on the tensor cores,
// forces and fields from the hand-written backward pass, the learned colour
// sweep, and training (forward-over-reverse parameter gradients, Adam).
// The paper has no learned model; the model is defined in include/sl.h.
//
// Layouts (sector-sorted atoms):
//   ml_x  [n][48] float   normalised descriptor x_i = (D_i - mean) * inv_std
//   ml_G  [n][16] float4  G_i[3k+m] = dE_i/dD_i[3k+m] as (m=0, m=1, m=2, 0) per k
//   ml_pq [max_m][n] float2 (P_ij, Q_ij) per Morse-list entry (0 beyond the cutoff)
#include <cuda_bf16.h>

#include "sl_internal.cuh"
#include "sl_df64.cuh"
#include "sl_pair.cuh"
#include "sl_tc.cuh"

namespace {

inline int grid_for(int n) { return (n + SL_BLOCK - 1) / SL_BLOCK; }

constexpr int NF = SL_ML_NF, NH = SL_ML_NH, NK = 16;
constexpr int TILE = SL_ML_ATOMS_PER_TILE;        // atoms per MMA tile (M = 128)

// Weight tiles, bfloat16, K-major canonical layout (sl_tc.cuh):
//   W1  : N = 64 hidden units x K = 48 features   (layer 1, x W1^T)
//   W2  : N = 64 x K = 64                         (layer 2, h1 W2^T)
//   W2T : N = 64 x K = 64, W2T[i][o] = W2[o][i]    (backward, g2 W2)
//   W1T : N = 48 x K = 64, W1T[f][o] = W1[o][f]    (backward, g1 W1)
constexpr int T_W1 = 0, T_W2 = T_W1 + 64 * 48 * 2, T_W2T = T_W2 + 64 * 64 * 2, T_W1T = T_W2T + 64 * 64 * 2;
constexpr int T_BYTES = T_W1T + 48 * 64 * 2;
static_assert(T_BYTES == SL_ML_TILE_BYTES, "tile size");
// Activation operand: 3 bfloat16 pieces of a 128 x K (K <= 64) matrix.
constexpr int PIECE = TILE * 64 * 2;
constexpr int ABUF = 3 * PIECE;
constexpr int GUARD = 16384;   // slack after the operands inside the allocation

__device__ __forceinline__ float ml_sig(float z) { return 1.0f / (1.0f + expf(-z)); }
__device__ __forceinline__ float ml_silu(float z) { return z * ml_sig(z); }
__device__ __forceinline__ float ml_dsilu(float z) { float q = ml_sig(z); return q * (1.0f + z * (1.0f - q)); }
__device__ __forceinline__ float ml_d2silu(float z) {
  float q = ml_sig(z);
  return q * (1.0f - q) * (2.0f + z * (1.0f - 2.0f * q));
}

// Gaussian centres 0.4 k (nearest floats).
__constant__ float kMu[NK] = {0.0f, 0.4f, 0.8f, 1.2f, 1.6f, 2.0f, 2.4f, 2.8f,
                              3.2f, 3.6f, 4.0f, 4.4f, 4.8f, 5.2f, 5.6f, 6.0f};

// Cutoff function fc(r) = (1 + cos(pi r/6))/2 and its derivative.
__device__ __forceinline__ void ml_cut(float r, float& fc, float& dfc) {
  float sp, cp;
  sincospif(r * (1.0f / 6.0f), &sp, &cp);
  fc = 0.5f * (1.0f + cp);
  dfc = -0.5f * (3.14159265358979f / 6.0f) * sp;
}
// g_k(r) = exp(-(r - mu_k)^2 / (2 0.4^2)) fc(r); 1/(2 0.4^2) = 3.125, 1/0.4^2 = 6.25.
__device__ __forceinline__ float ml_gauss(float r, int k) {
  float dq = r - kMu[k];
  return expf(-3.125f * dq * dq);
}

// Pair separation (float) from the exact split positions.
__device__ __forceinline__ float3 ml_sep(const box3& B, const p3& a, const p3& b) {
  df3 dd = pair_sep(B, a, b);
  return make_float3(dd.x.hi + dd.x.lo, dd.y.hi + dd.y.lo, dd.z.hi + dd.z.lo);
}
__device__ __forceinline__ float3 spin_f(const SlDev& d, int j) {
  float4 h = d.sdf[2 * (size_t)j];
  return make_float3(h.x, h.y, h.z);
}

// Three bfloat16 pieces hi + mid + lo of a float (each residual is exact).
__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(x);
  float r1 = x - __bfloat162float(a);
  b = __float2bfloat16_rn(r1);
  float r2 = r1 - __bfloat162float(b);
  c = __float2bfloat16_rn(r2);
}

// Row `row` (K values) of the three-piece activation operand at abuf.
__device__ __forceinline__ void store_row3(uint8_t* abuf, int row, const float* v, int K) {
  for (int c = 0; c < K / 8; ++c) {
    __align__(16) __nv_bfloat16 p0[8], p1[8], p2[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) split3(v[8 * c + e], p0[e], p1[e], p2[e]);
    const uint32_t off = kmajor_off(row, 8 * c, K);
    *(uint4*)(abuf + off) = *(const uint4*)p0;
    *(uint4*)(abuf + PIECE + off) = *(const uint4*)p1;
    *(uint4*)(abuf + 2 * PIECE + off) = *(const uint4*)p2;
  }
}
// Value of element (row, k) of a three-piece operand.
__device__ __forceinline__ float load3(const uint8_t* abuf, int row, int k, int K) {
  const uint32_t off = kmajor_off(row, k, K);
  return __bfloat162float(*(const __nv_bfloat16*)(abuf + off)) +
         __bfloat162float(*(const __nv_bfloat16*)(abuf + PIECE + off)) +
         __bfloat162float(*(const __nv_bfloat16*)(abuf + 2 * PIECE + off));
}

// Issue D (+)= sum over pieces of A_p B^T for one layer (thread 0 only).
__device__ __forceinline__ void issue_layer(uint32_t d_tmem, uint32_t a_base, uint32_t b_base, int K, int N,
                                            int accumulate) {
  const uint32_t idesc = idesc_bf16_f32(128, N);
  const uint32_t sbo = (uint32_t)K * 16u;
  int first = !accumulate;
  for (int p = 0; p < 3; ++p)
    for (int ks = 0; ks < K / 16; ++ks) {
      uint64_t a = smem_desc(a_base + p * PIECE + ks * 256, 128, sbo);
      uint64_t b = smem_desc(b_base + ks * 256, 128, sbo);
      mma_bf16(d_tmem, a, b, idesc, first ? 0u : 1u);
      first = 0;
    }
}

// ---------------------------------------------------------------------------
// Weight tiles and epilogue constants from the float32 master parameters.
// ---------------------------------------------------------------------------
__global__ void k_ml_prep(SlDev d) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  uint8_t* T = (uint8_t*)d.ml_tiles;
  const float* P = d.ml_par;
  if (t < 64 * 48) {
    const int o = t / 48, f = t % 48;
    const __nv_bfloat16 w = __float2bfloat16_rn(P[SL_ML_OFF_W1 + t]);
    *(__nv_bfloat16*)(T + T_W1 + kmajor_off(o, f, 48)) = w;
    *(__nv_bfloat16*)(T + T_W1T + kmajor_off(f, o, 64)) = w;
  }
  if (t < 64 * 64) {
    const int o = t / 64, i = t % 64;
    const __nv_bfloat16 w = __float2bfloat16_rn(P[SL_ML_OFF_W2 + t]);
    *(__nv_bfloat16*)(T + T_W2 + kmajor_off(o, i, 64)) = w;
    *(__nv_bfloat16*)(T + T_W2T + kmajor_off(i, o, 64)) = w;
  }
  if (t < 64) {
    d.ml_fc[SL_MLC_B1 + t] = P[SL_ML_OFF_B1 + t];
    d.ml_fc[SL_MLC_B2 + t] = P[SL_ML_OFF_B2 + t];
    d.ml_fc[SL_MLC_W3 + t] = __bfloat162float(__float2bfloat16_rn(P[SL_ML_OFF_W3 + t]));
  }
  if (t == 0) d.ml_fc[SL_MLC_B3] = P[SL_ML_OFF_B3];
  if (t < 4 * 48) d.ml_fc[SL_MLC_MEAN + t] = d.ml_norm[t];
}

// ---------------------------------------------------------------------------
// Descriptors and the range gate.  raw (optional, [n][48] float, sorted) and
// draw (optional, [n][48] double, caller order) receive the raw D.
// ---------------------------------------------------------------------------
__global__ void k_ml_desc(SlDev d, int count_gate, float* raw, double* draw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  const p3 pi = load_pos(d, i);
  const box3 B = load_box(d, d.reps[__ldg(d.arep + i)]);
  const float3 si = spin_f(d, i);
  float D[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) D[f] = 0.0f;
  const int nm = d.mn[i];
  for (int k = 0; k < nm; ++k) {
    const int j = __ldg(d.mj + (size_t)k * d.n + i);
    const float3 dd = ml_sep(B, pi, load_pos(d, j));
    const float r2 = dd.x * dd.x + dd.y * dd.y + dd.z * dd.z;
    if (!(r2 < 36.0f)) continue;
    const float r = sqrtf(r2);
    const float3 sj = spin_f(d, j);
    const float c = si.x * sj.x + si.y * sj.y + si.z * sj.z;
    float fc, dfc;
    ml_cut(r, fc, dfc);
#pragma unroll
    for (int q = 0; q < NK; ++q) {
      const float g = ml_gauss(r, q) * fc;
      D[3 * q] += g;
      D[3 * q + 1] = fmaf(g, c, D[3 * q + 1]);
      D[3 * q + 2] = fmaf(g * c, c, D[3 * q + 2]);
    }
  }
  const float* C = d.ml_fc;
  int bad = 0;
  float x[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    if (!(D[f] >= __ldg(C + SL_MLC_LO + f) && D[f] <= __ldg(C + SL_MLC_HI + f))) bad = 1;
    x[f] = (D[f] - __ldg(C + SL_MLC_MEAN + f)) * __ldg(C + SL_MLC_ISTD + f);
  }
  float4* xo = (float4*)(d.ml_x + (size_t)i * NF);
#pragma unroll
  for (int u = 0; u < NF / 4; ++u) xo[u] = make_float4(x[4 * u], x[4 * u + 1], x[4 * u + 2], x[4 * u + 3]);
  if (raw) {
    float4* ro = (float4*)(raw + (size_t)i * NF);
#pragma unroll
    for (int u = 0; u < NF / 4; ++u) ro[u] = make_float4(D[4 * u], D[4 * u + 1], D[4 * u + 2], D[4 * u + 3]);
  }
  if (draw) {
    double* o = draw + (size_t)d.perm[i] * NF;
#pragma unroll
    for (int f = 0; f < NF; ++f) o[f] = (double)D[f];
  }
  if (count_gate && bad) atomicAdd(&d.ctrl->ml_bad, 1);
}

__global__ void k_ml_gate(SlDev d) {
  SlCtrl* c = d.ctrl;
  c->ml_bad_last = c->ml_bad;
  c->ml_use = c->ml_bad == 0;
  if (c->ml_bad) c->ml_trips += 1;
  c->ml_bad = 0;
}

// ---------------------------------------------------------------------------
// Network forward and backward for 128 atoms per block on the tensor cores.
//   layer 1: a1 = x W1^T         (TMEM columns   0..63)
//   layer 2: a2 = h1 W2^T        (TMEM columns  64..127), h1 = silu(a1 + b1)
//   back 1 : q1 = g2 W2          (TMEM columns 128..191), g2 = w3 silu'(a2 + b2)
//   back 2 : gx = g1 W1          (TMEM columns 192..239), g1 = q1 silu'(a1 + b1)
// E_i = w3 . silu(a2 + b2) + b3 and G_i = gx * inv_std.  Thread t owns atom
// (row, TMEM lane) t; warp w reads lanes 32 w .. 32 w + 31.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128, 1) k_ml_mlp(SlDev d, int force) {
  if (!force && !d.ctrl->ml_use) return;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  uint8_t* tiles = smem;
  uint8_t* abuf = smem + T_BYTES;
  const int t = threadIdx.x, warp = t >> 5;
  const int a = blockIdx.x * TILE + t;
  const bool live = a < d.n;
  for (int k = t; k < T_BYTES / 16; k += TILE) ((uint4*)tiles)[k] = d.ml_tiles[k];
  if (warp == 0) tmem_alloc(smem_u32(&tbase), 256);
  if (t == 0) mbar_init(smem_u32(&bar), 1);
  {
    float x[NF];
    const float4* xi = (const float4*)(d.ml_x + (size_t)a * NF);
#pragma unroll
    for (int u = 0; u < NF / 4; ++u) {
      float4 v = live ? xi[u] : make_float4(0.f, 0.f, 0.f, 0.f);
      x[4 * u] = v.x; x[4 * u + 1] = v.y; x[4 * u + 2] = v.z; x[4 * u + 3] = v.w;
    }
    store_row3(abuf, t, x, NF);
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = tbase;
  const uint32_t lane_base = tm + ((uint32_t)(warp * 32) << 16);
  const uint32_t bar_a = smem_u32(&bar);
  const uint32_t a_s = smem_u32(abuf), t_s = smem_u32(tiles);
  const float* C = d.ml_fc;
  int ok = 1;
  uint32_t phase = 0;

  // layer 1
  if (t == 0) { issue_layer(tm + 0, a_s, t_s + T_W1, 48, 64, 0); mma_commit(bar_a); }
  ok &= mbar_wait(bar_a, phase); phase ^= 1;
  tc_fence_after();
  {
    float h[64];
    for (int c = 0; c < 4; ++c) {
      float v[16];
      tmem_ld16(lane_base + 0 + 16 * c, v);
#pragma unroll
      for (int e = 0; e < 16; ++e) h[16 * c + e] = ml_silu(v[e] + __ldg(C + SL_MLC_B1 + 16 * c + e));
    }
    store_row3(abuf, t, h, 64);
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // layer 2
  if (t == 0) { issue_layer(tm + 64, a_s, t_s + T_W2, 64, 64, 0); mma_commit(bar_a); }
  ok &= mbar_wait(bar_a, phase); phase ^= 1;
  tc_fence_after();
  {
    float g2[64];
    float e = 0.0f;
    for (int c = 0; c < 4; ++c) {
      float v[16];
      tmem_ld16(lane_base + 64 + 16 * c, v);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int o = 16 * c + k;
        const float z = v[k] + __ldg(C + SL_MLC_B2 + o);
        const float w3 = __ldg(C + SL_MLC_W3 + o);
        e = fmaf(w3, ml_silu(z), e);
        g2[o] = w3 * ml_dsilu(z);
      }
    }
    if (live) d.ml_e[a] = e + __ldg(C + SL_MLC_B3);
    store_row3(abuf, t, g2, 64);
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // backward through layer 2: q1 = g2 W2
  if (t == 0) { issue_layer(tm + 128, a_s, t_s + T_W2T, 64, 64, 0); mma_commit(bar_a); }
  ok &= mbar_wait(bar_a, phase); phase ^= 1;
  tc_fence_after();
  {
    float g1[64];
    for (int c = 0; c < 4; ++c) {
      float q[16], z[16];
      tmem_ld16(lane_base + 128 + 16 * c, q);
      tmem_ld16(lane_base + 0 + 16 * c, z);
#pragma unroll
      for (int k = 0; k < 16; ++k) g1[16 * c + k] = q[k] * ml_dsilu(z[k] + __ldg(C + SL_MLC_B1 + 16 * c + k));
    }
    store_row3(abuf, t, g1, 64);
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // backward through layer 1: gx = g1 W1
  if (t == 0) { issue_layer(tm + 192, a_s, t_s + T_W1T, 64, 48, 0); mma_commit(bar_a); }
  ok &= mbar_wait(bar_a, phase); phase ^= 1;
  tc_fence_after();
  {
    float gx[NF];
    for (int c = 0; c < 3; ++c) tmem_ld16(lane_base + 192 + 16 * c, gx + 16 * c);
    if (live) {
      float4* Go = (float4*)(d.ml_G + (size_t)a * 4 * NK);
#pragma unroll
      for (int q = 0; q < NK; ++q)
        Go[q] = make_float4(gx[3 * q] * __ldg(C + SL_MLC_ISTD + 3 * q),
                            gx[3 * q + 1] * __ldg(C + SL_MLC_ISTD + 3 * q + 1),
                            gx[3 * q + 2] * __ldg(C + SL_MLC_ISTD + 3 * q + 2), 0.0f);
    }
  }
  if (!ok && t == 0) sl_set_error(d.ctrl, SL_ERR_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, 256);
}

// ---------------------------------------------------------------------------
// Pair terms of the backward pass, per atom i over its neighbours j < 6 A:
//   phi_ij = sum_k [(G_i+G_j)[3k] + (G_i+G_j)[3k+1] c + (G_i+G_j)[3k+2] c^2] g_k'(r)
//   F_i    = sum_j phi_ij (r_j - r_i)/r                           (= -dE/dr_i)
//   P_ij   = sum_k (G_i+G_j)[3k+1] g_k(r),  Q_ij = sum_k (G_i+G_j)[3k+2] g_k(r)
//   B_i    = -sum_j (P_ij + 2 Q_ij c) s_j                         (= -dE/ds_i)
// with c = s_i.s_j.  fmode bit 0: F into the integrator's FP64 forces, bit 1:
// closing half-kick, bit 2: F into ml_gF (training scratch), bit 3: average
// (P, Q) with the table's previous entries (the predicted end of a half-op).  Fout, Bout
// (optional, caller order [n][3] double) receive F and B.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_ml_pair(SlDev d, int fmode, int force, double* Fout, double* Bout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  if (!force && !d.ctrl->ml_use) return;
  const p3 pi = load_pos(d, i);
  const box3 B = load_box(d, d.reps[__ldg(d.arep + i)]);
  const float3 si = spin_f(d, i);
  float Gi[NF];
  {
    const float4* g = (const float4*)(d.ml_G + (size_t)i * 4 * NK);
#pragma unroll
    for (int q = 0; q < NK; ++q) {
      float4 v = g[q];
      Gi[3 * q] = v.x; Gi[3 * q + 1] = v.y; Gi[3 * q + 2] = v.z;
    }
  }
  float fx = 0.f, fy = 0.f, fz = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
  const int nm = d.mn[i];
  const size_t n = (size_t)d.n;
  for (int k = 0; k < nm; ++k) {
    const size_t e = (size_t)k * n + i;
    const int j = __ldg(d.mj + e);
    const float3 dd = ml_sep(B, pi, load_pos(d, j));
    const float r2 = dd.x * dd.x + dd.y * dd.y + dd.z * dd.z;
    if (!(r2 < 36.0f)) { if (!(fmode & 8)) d.ml_pq[e] = make_float2(0.f, 0.f); continue; }
    const float r = sqrtf(r2), ir = 1.0f / r;
    const float3 sj = spin_f(d, j);
    const float c = si.x * sj.x + si.y * sj.y + si.z * sj.z;
    float fc, dfc;
    ml_cut(r, fc, dfc);
    const float4* Gj = (const float4*)(d.ml_G + (size_t)j * 4 * NK);
    float phi = 0.f, P = 0.f, Q = 0.f;
#pragma unroll
    for (int q = 0; q < NK; ++q) {
      const float dq = r - kMu[q];
      const float ex = expf(-3.125f * dq * dq);
      const float g = ex * fc;
      const float dg = ex * fmaf(-6.25f * dq, fc, dfc);
      const float4 gj = __ldg(Gj + q);
      const float s0 = Gi[3 * q] + gj.x, s1 = Gi[3 * q + 1] + gj.y, s2 = Gi[3 * q + 2] + gj.z;
      phi = fmaf(fmaf(fmaf(s2, c, s1), c, s0), dg, phi);
      P = fmaf(s1, g, P);
      Q = fmaf(s2, g, Q);
    }
    const float pr = phi * ir;
    fx = fmaf(pr, dd.x, fx); fy = fmaf(pr, dd.y, fy); fz = fmaf(pr, dd.z, fz);
    const float psi = fmaf(2.0f * Q, c, P);
    bx = fmaf(-psi, sj.x, bx); by = fmaf(-psi, sj.y, by); bz = fmaf(-psi, sj.z, bz);
    if (fmode & 8) {
      const float2 o = d.ml_pq[e];
      d.ml_pq[e] = make_float2(0.5f * (o.x + P), 0.5f * (o.y + Q));
    } else {
      d.ml_pq[e] = make_float2(P, Q);
    }
  }
  d.ml_B[i] = make_float4(bx, by, bz, 0.f);
  if (fmode & 1) {
    d.F[i] = make_double4_32a(fx, fy, fz, 0.0);
    if (fmode & 2) {
      const double cc = 0.5 * d.dt * d.acc;
      double4_32a v = d.v[i];
      v.x = fma(cc, (double)fx, v.x); v.y = fma(cc, (double)fy, v.y); v.z = fma(cc, (double)fz, v.z);
      if (d.any_lattice_bath) v = lattice_bath(d, i, v, 5);
      d.v[i] = v;
    }
  }
  if (fmode & 4) d.ml_gF[i] = make_float4(fx, fy, fz, 0.f);
  const size_t id = (size_t)d.perm[i];
  if (Fout) { Fout[3 * id] = fx; Fout[3 * id + 1] = fy; Fout[3 * id + 2] = fz; }
  if (Bout) { Bout[3 * id] = bx; Bout[3 * id + 1] = by; Bout[3 * id + 2] = bz; }
}

// ---------------------------------------------------------------------------
// One colour pass of a learned spin sweep.
//
// With the network in effect, the field of spin i is
//   B_i(s) = -p_i - 2 M_i s,  p_i = sum_j P_ij s_j,  M_i = sum_j Q_ij s_j s_j^T,
// and each single-spin factor rotates s_i exactly about omega at the
// rotation's midpoint m = u/|u|, u = s_i + (tau/2) omega(s_i) x s_i (float32,
// second order in the angle), omega(m) = (mu_s mu_B H + B_i(m))/hbar.
// Block b takes LS_SPB consecutive sectors of the colour:
//   phase 1 (8 lanes per atom, over its list): p_i and M_i from the
//           neighbours whose spins do not change before spin i turns (other
//           sectors, and later spins of its own sector in this pass's order),
//           the atom's float32 spin, and its entries for the earlier spins of
//           its sector (local index, P, Q) staged in shared memory;
//   phase 2 (one lane per sector, sequential): add those entries with the
//           updated spins, form B_i(m), and rotate the float32 copy that
//           later spins of the sector see;
//   phase 3 (one thread per atom): the double-float rotation of the FP64
//           spin about omega(m), added once.
// Blocks whose atoms or same-sector lists do not fit run every sector from
// global memory instead (one lane per sector).  With the gate closed the
// field is the analytic one, sum_j J_ij s_j over the exchange list
// (double-float), on the same per-lane path.  `predictor` = 1 runs only with
// the network in effect (the predictor sweep of the half-op).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int LS_SPB = 2;          // sectors per block
constexpr int LS_THREADS = 128;
constexpr int LS_MAXA = 96;        // atoms staged per block
constexpr int LS_MAXIN = 48;       // same-sector entries staged per atom
constexpr size_t LS_SMEM = (size_t)LS_MAXIN * LS_MAXA * (sizeof(float2) + sizeof(short)) +
                           (size_t)LS_MAXA * (3 + 9 + 3) * sizeof(float) + (size_t)LS_MAXA * sizeof(int);

// The network's part of the field at spin s: -(p + 2 M s), float32.
__device__ __forceinline__ float3 ml_field_f(const float* p, const float* M, float3 s) {
  return make_float3(-p[0] - 2.0f * (M[0] * s.x + M[3] * s.y + M[4] * s.z),
                     -p[1] - 2.0f * (M[3] * s.x + M[1] * s.y + M[5] * s.z),
                     -p[2] - 2.0f * (M[4] * s.x + M[5] * s.y + M[2] * s.z));
}

__device__ __forceinline__ void pm_add(float* p, float* M, float P, float Q, float3 sj) {
  p[0] = fmaf(P, sj.x, p[0]); p[1] = fmaf(P, sj.y, p[1]); p[2] = fmaf(P, sj.z, p[2]);
  const float qx = Q * sj.x, qy = Q * sj.y;
  M[0] = fmaf(qx, sj.x, M[0]); M[1] = fmaf(qy, sj.y, M[1]); M[2] = fmaf(Q * sj.z, sj.z, M[2]);
  M[3] = fmaf(qx, sj.y, M[3]); M[4] = fmaf(qx, sj.z, M[4]); M[5] = fmaf(qy, sj.z, M[5]);
}

// The network's field at the rotation's midpoint, from p, M and the float32 spin.
__device__ __forceinline__ float3 ml_mid_field(const SlDev& d, const float* p, const float* M, float3 s0, float tau) {
  const float ih = (float)(1.0 / SL_HBAR);
  const float3 b0 = ml_field_f(p, M, s0);
  const float w0x = ((float)d.zee[0] + b0.x) * ih, w0y = ((float)d.zee[1] + b0.y) * ih,
              w0z = ((float)d.zee[2] + b0.z) * ih;
  const float ht = 0.5f * tau;
  const float mx = fmaf(ht, w0y * s0.z - w0z * s0.y, s0.x);
  const float my = fmaf(ht, w0z * s0.x - w0x * s0.z, s0.y);
  const float mz = fmaf(ht, w0x * s0.y - w0y * s0.x, s0.z);
  const float mi = rsqrtf(mx * mx + my * my + mz * mz);
  return ml_field_f(p, M, make_float3(mx * mi, my * mi, mz * mi));
}

// omega = (mu_s mu_B H + b)/hbar with the Zeeman term and 1/hbar in double-float.
__device__ __forceinline__ df3 ml_omega_df(const SlDev& d, float3 b) {
  const df ih = F2(d.inv_hbar_f);
  df3 w;
  w.x = df_mul(df_add_f(F2(d.zee_f[0]), b.x), ih);
  w.y = df_mul(df_add_f(F2(d.zee_f[1]), b.y), ih);
  w.z = df_mul(df_add_f(F2(d.zee_f[2]), b.z), ih);
  return w;
}

// Float32 rotation of s about w by |w| tau (the copy later spins of a sector see).
__device__ __forceinline__ float3 rot_f(float3 w, float3 s, float tau) {
  const float u = (w.x * w.x + w.y * w.y + w.z * w.z) * tau * tau;
  float A, B;
  if (u < 1e-2f) {
    A = fmaf(u, fmaf(u, 1.0f / 120.0f, -1.0f / 6.0f), 1.0f);        // sin(t)/t
    B = fmaf(u, fmaf(u, 1.0f / 720.0f, -1.0f / 24.0f), 0.5f);       // (1 - cos t)/t^2
  } else {
    const float th = sqrtf(u);
    const float hs = sinf(0.5f * th);
    A = sinf(th) / th;
    B = 2.0f * hs * hs / u;
  }
  const float ws = w.x * s.x + w.y * s.y + w.z * s.z;
  const float cx = w.y * s.z - w.z * s.y, cy = w.z * s.x - w.x * s.z, cz = w.x * s.y - w.y * s.x;
  const float tA = tau * A, t2B = tau * tau * B * ws, uB = u * B;
  return make_float3(s.x - uB * s.x + tA * cx + t2B * w.x, s.y - uB * s.y + tA * cy + t2B * w.y,
                     s.z - uB * s.z + tA * cz + t2B * w.z);
}

__device__ __forceinline__ void apply_rotation(const SlDev& d, int i, const df3& w, df tau, int cayley) {
  const float4 h = d.sdf[2 * (size_t)i], l = d.sdf[2 * (size_t)i + 1];
  df3 s;
  s.x = df_make(h.x, l.x); s.y = df_make(h.y, l.y); s.z = df_make(h.z, l.z);
  const df3 inc = rot_increment(w, s, tau, cayley);
  double4_32a sd = d.s[i];
  sd.x += df_to_double(inc.x);
  sd.y += df_to_double(inc.y);
  sd.z += df_to_double(inc.z);
  d.s[i] = sd;
  store_spin_split(d, i, sd);
}

// Per-lane sequential update of one sector from global memory (fallback and
// analytic paths).
__device__ void ml_sector_global(const SlDev& d, int a0, int a1, int backward, int use, df tau) {
  const size_t n = (size_t)d.n;
  for (int t = 0; t < a1 - a0; ++t) {
    const int i = backward ? a1 - 1 - t : a0 + t;
    df3 w;
    if (use) {
      float p[3] = {0.f, 0.f, 0.f}, M[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const int nm = d.mn[i];
      for (int k = 0; k < nm; ++k) {
        const size_t e = (size_t)k * n + i;
        const float2 pq = __ldg(d.ml_pq + e);
        if (pq.x == 0.0f && pq.y == 0.0f) continue;
        const int j = __ldg(d.mj + e);
        const float4 sj = d.sdf[2 * (size_t)j];
        pm_add(p, M, pq.x, pq.y, make_float3(sj.x, sj.y, sj.z));
      }
      const float4 h = d.sdf[2 * (size_t)i];
      w = ml_omega_df(d, ml_mid_field(d, p, M, make_float3(h.x, h.y, h.z), tau.hi));
    } else {
      float xh = 0.f, xl = 0.f, yh = 0.f, yl = 0.f, zh = 0.f, zl = 0.f;
      const int ne = d.exn[i];
      for (int k = 0; k < ne; ++k) {
        const size_t e = (size_t)k * n + i;
        const df J = F2(__ldg(d.exJ + e));
        const int j = __ldg(d.exj + e);
        const float4 jh = d.sdf[2 * (size_t)j], jl = d.sdf[2 * (size_t)j + 1];
        acc_prod(xh, xl, J, df_make(jh.x, jl.x));
        acc_prod(yh, yl, J, df_make(jh.y, jl.y));
        acc_prod(zh, zl, J, df_make(jh.z, jl.z));
      }
      const df ih = F2(d.inv_hbar_f);
      w.x = df_mul(df_add(F2(d.zee_f[0]), acc_done(xh, xl)), ih);
      w.y = df_mul(df_add(F2(d.zee_f[1]), acc_done(yh, yl)), ih);
      w.z = df_mul(df_add(F2(d.zee_f[2]), acc_done(zh, zl)), ih);
    }
    apply_rotation(d, i, w, tau, !use && d.rotation == SL_ROT_CAYLEY);
  }
}

__global__ void __launch_bounds__(LS_THREADS) k_ml_sweep(SlDev d, int colour, int backward, int predictor) {
  extern __shared__ __align__(16) uint8_t lsm[];
  float2* inpq = (float2*)lsm;                                   // [LS_MAXIN][LS_MAXA]
  short* inj = (short*)(inpq + LS_MAXIN * LS_MAXA);              // [LS_MAXIN][LS_MAXA]
  float* sS = (float*)(inj + LS_MAXIN * LS_MAXA);                // [3][LS_MAXA] current float32 spins
  float* acc = sS + 3 * LS_MAXA;                                 // [9][LS_MAXA] p (3), M (6)
  float* bm = acc + 9 * LS_MAXA;                                 // [3][LS_MAXA] field at the midpoint
  int* nin = (int*)(bm + 3 * LS_MAXA);                           // [LS_MAXA]
  __shared__ int bounds[LS_SPB + 1];
  __shared__ int overflow;
  const int use = d.ctrl->ml_use;
  if (predictor && !use) return;
  const int sec0 = blockIdx.x * LS_SPB;
  if (sec0 >= d.s8) return;
  const int nsec = min(LS_SPB, d.s8 - sec0);
  const int q0 = colour * d.s8 + sec0;
  if (threadIdx.x <= nsec) bounds[threadIdx.x] = d.sec_start[q0 + threadIdx.x];
  if (threadIdx.x == 0) overflow = 0;
  __syncthreads();
  const int A0 = bounds[0], na = bounds[nsec] - A0;
  const df tau = F2(d.tau_f);
  const size_t n = (size_t)d.n;
  int staged = use && na <= LS_MAXA;
  if (staged) {
    // phase 1: groups of 8 lanes, one atom per group, the lanes over its list
    const int lane = threadIdx.x & 31, g8 = lane >> 3, l8 = lane & 7;
    const unsigned gmask = 0xFFu << (8 * g8);
    for (int t0 = (threadIdx.x >> 5) * 4; t0 < na; t0 += LS_THREADS / 8) {
      const int t = t0 + g8;
      const bool act = t < na;
      const int i = act ? A0 + t : A0;
      int lo = 0, hi = 0;
      for (int q = 0; q < nsec; ++q)
        if (i >= bounds[q] && i < bounds[q + 1]) { lo = bounds[q]; hi = bounds[q + 1]; }
      // same-sector spins later in this pass's order still hold their pass-start
      // values when spin i turns: only the earlier ones go to phase 2
      if (backward) lo = i + 1; else hi = i;
      if (act && l8 < 3) {
        const float4 sv = d.sdf[2 * (size_t)i];
        sS[l8 * LS_MAXA + t] = l8 == 0 ? sv.x : (l8 == 1 ? sv.y : sv.z);
      }
      float p[3] = {0.f, 0.f, 0.f}, M[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      int cnt = 0;
      const int nm = act ? d.mn[i] : 0;
      const int nmax = max(nm, __shfl_xor_sync(0xffffffffu, nm, 8));
      const int nall = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, 16));
      for (int k0 = 0; k0 < nall; k0 += 32) {
        // four entries per lane per round, loads issued together
        float2 pq[4];
        int jj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = k0 + 8 * u + l8;
          pq[u] = make_float2(0.f, 0.f);
          jj[u] = -1;
          if (k < nm) {
            const size_t e = (size_t)k * n + i;
            pq[u] = __ldg(d.ml_pq + e);
            jj[u] = __ldg(d.mj + e);
          }
        }
        float4 sj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool live = pq[u].x != 0.0f || pq[u].y != 0.0f;
          const bool ext = live && !(jj[u] >= lo && jj[u] < hi);
          sj[u] = ext ? d.sdf[2 * (size_t)jj[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool live = pq[u].x != 0.0f || pq[u].y != 0.0f;
          const bool internal = live && jj[u] >= lo && jj[u] < hi;
          if (live && !internal) pm_add(p, M, pq[u].x, pq[u].y, make_float3(sj[u].x, sj[u].y, sj[u].z));
          const unsigned mask = __ballot_sync(0xffffffffu, internal) & gmask;
          const int pos = cnt + __popc(mask & ((1u << lane) - 1u));
          if (internal && pos < LS_MAXIN) {
            inpq[pos * LS_MAXA + t] = pq[u];
            inj[pos * LS_MAXA + t] = (short)(jj[u] - A0);
          }
          cnt += __popc(mask);
        }
      }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) p[c] += __shfl_xor_sync(0xffffffffu, p[c], o);
#pragma unroll
        for (int c = 0; c < 6; ++c) M[c] += __shfl_xor_sync(0xffffffffu, M[c], o);
      }
      if (act && l8 == 0) {
        if (cnt > LS_MAXIN) overflow = 1;
        nin[t] = cnt;
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c * LS_MAXA + t] = p[c];
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[(3 + c) * LS_MAXA + t] = M[c];
      }
    }
    __syncthreads();
    staged = !overflow;
  }
  if (!staged) {
    // every sector of the block from global memory, one lane each
    if (threadIdx.x < nsec) ml_sector_global(d, bounds[threadIdx.x], bounds[threadIdx.x + 1], backward, use, tau);
    return;
  }
  // phase 2
  if (threadIdx.x < nsec) {
    const int lo = bounds[threadIdx.x] - A0, hi = bounds[threadIdx.x + 1] - A0;
    const float ih = (float)(1.0 / SL_HBAR);
    for (int u = 0; u < hi - lo; ++u) {
      const int t = backward ? hi - 1 - u : lo + u;
      float p[3], M[6];
#pragma unroll
      for (int c = 0; c < 3; ++c) p[c] = acc[c * LS_MAXA + t];
#pragma unroll
      for (int c = 0; c < 6; ++c) M[c] = acc[(3 + c) * LS_MAXA + t];
      const int cnt = nin[t];
#pragma unroll 4
      for (int e = 0; e < cnt; ++e) {
        const float2 pq = inpq[e * LS_MAXA + t];
        const int jl = inj[e * LS_MAXA + t];
        pm_add(p, M, pq.x, pq.y, make_float3(sS[jl], sS[LS_MAXA + jl], sS[2 * LS_MAXA + jl]));
      }
      const float3 s0 = make_float3(sS[t], sS[LS_MAXA + t], sS[2 * LS_MAXA + t]);
      const float3 b = ml_mid_field(d, p, M, s0, tau.hi);
      bm[t] = b.x; bm[LS_MAXA + t] = b.y; bm[2 * LS_MAXA + t] = b.z;
      const float3 w = make_float3(((float)d.zee[0] + b.x) * ih, ((float)d.zee[1] + b.y) * ih,
                                   ((float)d.zee[2] + b.z) * ih);
      const float3 s1 = rot_f(w, s0, tau.hi);
      sS[t] = s1.x; sS[LS_MAXA + t] = s1.y; sS[2 * LS_MAXA + t] = s1.z;
    }
  }
  __syncthreads();
  // phase 3
  for (int t = threadIdx.x; t < na; t += LS_THREADS)
    apply_rotation(d, A0 + t, ml_omega_df(d, make_float3(bm[t], bm[LS_MAXA + t], bm[2 * LS_MAXA + t])), tau, 0);
}

// Spins at the start of a learned half-op, kept for the corrector sweep.
__global__ void k_ml_save_spins(SlDev d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n || !d.ctrl->ml_use) return;
  d.ts[i] = d.s[i];
}
__global__ void k_ml_restore_spins(SlDev d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n || !d.ctrl->ml_use) return;
  const double4_32a s = d.ts[i];
  d.s[i] = s;
  store_spin_split(d, i, s);
}

// ---------------------------------------------------------------------------
// Per-replica energy sum_i E_i in a fixed order (via caller-order slots).
// ---------------------------------------------------------------------------
__global__ void k_ml_e_caller(SlDev d, double* slot) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  slot[d.perm[i]] = (double)d.ml_e[i];
}

constexpr int RT = 256;
__device__ __forceinline__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = RT / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void k_ml_erep(SlDev d, const double* slot) {
  __shared__ double sh[RT];
  const SlRep& R = d.reps[blockIdx.x];
  double s = 0.0;
  for (int k = threadIdx.x; k < R.natoms; k += RT) s += slot[R.atom0 + k];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) d.ml_erep[blockIdx.x] = s;
}

// Mean, standard deviation, minimum, maximum of each raw descriptor feature
// (one block per feature, fixed order).
__global__ void k_ml_dstats(SlDev d, const float* raw, double* out) {
  __shared__ double sh[RT];
  const int f = blockIdx.x;
  double s = 0.0, s2 = 0.0, lo = 1e300, hi = -1e300;
  for (int i = threadIdx.x; i < d.n; i += RT) {
    const double v = raw[(size_t)i * NF + f];
    s += v; s2 += v * v;
    lo = fmin(lo, v); hi = fmax(hi, v);
  }
  s = block_sum(s, sh);
  s2 = block_sum(s2, sh);
  sh[threadIdx.x] = lo;
  __syncthreads();
  for (int w = RT / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  lo = sh[0];
  __syncthreads();
  sh[threadIdx.x] = hi;
  __syncthreads();
  for (int w = RT / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  hi = sh[0];
  if (threadIdx.x == 0) {
    const double m = s / d.n;
    out[f] = m;
    out[NF + f] = sqrt(fmax(s2 / d.n - m * m, 0.0));
    out[2 * NF + f] = lo;
    out[3 * NF + f] = hi;
  }
}

// ---------------------------------------------------------------------------
// Training.
// ---------------------------------------------------------------------------
// Upstream gradients from caller-order device arrays (any may be NULL).
__global__ void k_ml_upstream(SlDev d, const double* gE, const double* gF, const double* gB) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  const size_t id = (size_t)d.perm[i];
  d.ml_alpha[i] = gE ? gE[d.arep[i]] : 0.0;
  d.ml_gF[i] = gF ? make_float4((float)gF[3 * id], (float)gF[3 * id + 1], (float)gF[3 * id + 2], 0.f)
                  : make_float4(0.f, 0.f, 0.f, 0.f);
  d.ml_gB[i] = gB ? make_float4((float)gB[3 * id], (float)gB[3 * id + 1], (float)gB[3 * id + 2], 0.f)
                  : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Per-atom loss terms and the upstream gradients of F and B
// (F in ml_gF and B in ml_B on entry, from k_ml_pair with fmode 4).
__global__ void k_ml_loss_atoms(SlDev d, const double* F_ref, const double* B_ref, double wF, double wW) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  const size_t id = (size_t)d.perm[i];
  const float4 Fp = d.ml_gF[i], Bp = d.ml_B[i];
  const double4_32a s = d.s[i];
  const double dF[3] = {Fp.x - F_ref[3 * id], Fp.y - F_ref[3 * id + 1], Fp.z - F_ref[3 * id + 2]};
  double dB[3] = {Bp.x - B_ref[3 * id], Bp.y - B_ref[3 * id + 1], Bp.z - B_ref[3 * id + 2]};
  const double sb = s.x * dB[0] + s.y * dB[1] + s.z * dB[2];
  dB[0] -= sb * s.x; dB[1] -= sb * s.y; dB[2] -= sb * s.z;
  const double ih2 = 1.0 / (SL_HBAR * SL_HBAR);
  d.ml_lossat[2 * id] = dF[0] * dF[0] + dF[1] * dF[1] + dF[2] * dF[2];
  d.ml_lossat[2 * id + 1] = (dB[0] * dB[0] + dB[1] * dB[1] + dB[2] * dB[2]) * ih2;
  const double cf = 2.0 * wF / d.n, cw = 2.0 * wW * ih2 / d.n;
  d.ml_gF[i] = make_float4((float)(cf * dF[0]), (float)(cf * dF[1]), (float)(cf * dF[2]), 0.f);
  d.ml_gB[i] = make_float4((float)(cw * dB[0]), (float)(cw * dB[1]), (float)(cw * dB[2]), 0.f);
}

// Loss totals; ml_erep (sum E_i per replica on entry) becomes dL/dE_r.
__global__ void k_ml_loss_reduce(SlDev d, const double* E_ref, double wE, double wF, double wW) {
  __shared__ double sh[RT];
  double lf = 0.0, lw = 0.0;
  for (int k = threadIdx.x; k < d.n; k += RT) { lf += d.ml_lossat[2 * k]; lw += d.ml_lossat[2 * k + 1]; }
  lf = block_sum(lf, sh);
  lw = block_sum(lw, sh);
  double le = 0.0;
  for (int r = threadIdx.x; r < d.nrep; r += RT) {
    const double N = d.reps[r].natoms;
    const double dE = (d.ml_erep[r] - E_ref[r]) / N;
    le += dE * dE;
  }
  le = block_sum(le, sh);
  for (int r = threadIdx.x; r < d.nrep; r += RT) {
    const double N = d.reps[r].natoms;
    const double dE = (d.ml_erep[r] - E_ref[r]) / N;
    d.ml_erep[r] = 2.0 * wE * dE / (N * d.nrep);
  }
  if (threadIdx.x == 0) {
    const double LE = wE * le / d.nrep, LF = wF * lf / d.n, LW = wW * lw / d.n;
    d.ml_loss[0] = LE + LF + LW;
    d.ml_loss[1] = LE; d.ml_loss[2] = LF; d.ml_loss[3] = LW;
  }
}

__global__ void k_ml_alpha(SlDev d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  d.ml_alpha[i] = d.ml_erep[d.arep[i]];
}

// Adjoint of G (at fixed r, s): Gbar_a[f] such that
//   sum_i gF_i.F_i + sum_i gB_i.B_i = sum_a Gbar_a . G_a,
//   Gbar_a[3k+m] = sum_j g_k'(r) c^m e_aj.(gF_a - gF_j) - sum_j m g_k(r) c^(m-1) (s_j.gB_a + s_a.gB_j);
// stored as the tangent direction u_a = Gbar_a * inv_std.
__global__ void __launch_bounds__(128) k_ml_gbar(SlDev d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  const p3 pi = load_pos(d, i);
  const box3 B = load_box(d, d.reps[__ldg(d.arep + i)]);
  const float3 si = spin_f(d, i);
  const float4 gFi = d.ml_gF[i], gBi = d.ml_gB[i];
  float Gb[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) Gb[f] = 0.f;
  const int nm = d.mn[i];
  for (int k = 0; k < nm; ++k) {
    const int j = __ldg(d.mj + (size_t)k * d.n + i);
    const float3 dd = ml_sep(B, pi, load_pos(d, j));
    const float r2 = dd.x * dd.x + dd.y * dd.y + dd.z * dd.z;
    if (!(r2 < 36.0f)) continue;
    const float r = sqrtf(r2), ir = 1.0f / r;
    const float3 sj = spin_f(d, j);
    const float c = si.x * sj.x + si.y * sj.y + si.z * sj.z;
    const float4 gFj = d.ml_gF[j], gBj = d.ml_gB[j];
    const float fe = ir * (dd.x * (gFi.x - gFj.x) + dd.y * (gFi.y - gFj.y) + dd.z * (gFi.z - gFj.z));
    const float be = -(sj.x * gBi.x + sj.y * gBi.y + sj.z * gBi.z + si.x * gBj.x + si.y * gBj.y + si.z * gBj.z);
    float fc, dfc;
    ml_cut(r, fc, dfc);
#pragma unroll
    for (int q = 0; q < NK; ++q) {
      const float dq = r - kMu[q];
      const float ex = expf(-3.125f * dq * dq);
      const float g = ex * fc;
      const float dg = ex * fmaf(-6.25f * dq, fc, dfc);
      const float a0 = dg * fe;
      Gb[3 * q] += a0;
      Gb[3 * q + 1] += fmaf(a0, c, g * be);
      Gb[3 * q + 2] += fmaf(a0 * c, c, 2.0f * g * c * be);
    }
  }
  float4* uo = (float4*)(d.ml_u + (size_t)i * NF);
  const float* C = d.ml_fc;
#pragma unroll
  for (int u = 0; u < NF / 4; ++u)
    uo[u] = make_float4(Gb[4 * u] * __ldg(C + SL_MLC_ISTD + 4 * u), Gb[4 * u + 1] * __ldg(C + SL_MLC_ISTD + 4 * u + 1),
                        Gb[4 * u + 2] * __ldg(C + SL_MLC_ISTD + 4 * u + 2),
                        Gb[4 * u + 3] * __ldg(C + SL_MLC_ISTD + 4 * u + 3));
}

// Parameter gradient of  alpha_a E_a(x_a) + u_a . dE_a/dx_a  summed over the
// block's 128 atoms (forward pass, its tangent along u, reverse mode through
// both), written to ml_gpart[block].  TMEM columns: a1 0..63, t1 64..127,
// a2 128..191, t2 192..255, then (reused) h1bar 128..191, p1bar 192..255.
// Shared memory: weight tiles, two three-piece operands X and U, and a
// float32 stage for the weight-gradient products.
constexpr int TR_STAGE = 2 * TILE * 64 * 4;
constexpr size_t TR_SMEM = T_BYTES + 2 * ABUF + TR_STAGE + GUARD;

__global__ void __launch_bounds__(128, 1) k_ml_train_mlp(SlDev d) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  __shared__ float red[4][64 + 64 + 64 + 1];     // per-warp partial sums of w3bar, b2bar, b1bar, b3bar
  uint8_t* tiles = smem;
  uint8_t* bx = smem + T_BYTES;
  uint8_t* bu = bx + ABUF;
  float* stage = (float*)(bu + ABUF);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int a = blockIdx.x * TILE + t;
  const bool live = a < d.n;
  for (int k = t; k < T_BYTES / 16; k += TILE) ((uint4*)tiles)[k] = d.ml_tiles[k];
  if (warp == 0) tmem_alloc(smem_u32(&tbase), 256);
  if (t == 0) mbar_init(smem_u32(&bar), 1);
  {
    float x[NF];
    const float4* xi = (const float4*)(d.ml_x + (size_t)a * NF);
#pragma unroll
    for (int u = 0; u < NF / 4; ++u) {
      float4 v = live ? xi[u] : make_float4(0.f, 0.f, 0.f, 0.f);
      x[4 * u] = v.x; x[4 * u + 1] = v.y; x[4 * u + 2] = v.z; x[4 * u + 3] = v.w;
    }
    store_row3(bx, t, x, NF);
    const float4* ui = (const float4*)(d.ml_u + (size_t)a * NF);
#pragma unroll
    for (int u = 0; u < NF / 4; ++u) {
      float4 v = live ? ui[u] : make_float4(0.f, 0.f, 0.f, 0.f);
      x[4 * u] = v.x; x[4 * u + 1] = v.y; x[4 * u + 2] = v.z; x[4 * u + 3] = v.w;
    }
    store_row3(bu, t, x, NF);
  }
  const float alpha = live ? (float)d.ml_alpha[a] : 0.0f;
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = tbase;
  const uint32_t lb = tm + ((uint32_t)(warp * 32) << 16);
  const uint32_t bar_a = smem_u32(&bar);
  const uint32_t x_s = smem_u32(bx), u_s = smem_u32(bu), t_s = smem_u32(tiles);
  const float* C = d.ml_fc;
  int ok = 1;
  uint32_t phase = 0;
  float* sh1 = stage;                  // [128][64] h1
  float* sp1 = stage + TILE * 64;      // [128][64] p1

  // layer 1 and its tangent
  if (t == 0) {
    issue_layer(tm + 0, x_s, t_s + T_W1, 48, 64, 0);
    issue_layer(tm + 64, u_s, t_s + T_W1, 48, 64, 0);
    mma_commit(bar_a);
  }
  ok &= mbar_wait(bar_a, phase); phase ^= 1;
  tc_fence_after();
  {
    float h[64], p[64];
    for (int c = 0; c < 4; ++c) {
      float z[16], tv[16];
      tmem_ld16(lb + 0 + 16 * c, z);
      tmem_ld16(lb + 64 + 16 * c, tv);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float zz = z[k] + __ldg(C + SL_MLC_B1 + 16 * c + k);
        h[16 * c + k] = ml_silu(zz);
        p[16 * c + k] = ml_dsilu(zz) * tv[k];
      }
    }
    store_row3(bx, t, h, 64);
    store_row3(bu, t, p, 64);
    for (int k = 0; k < 64; ++k) { sh1[t * 64 + k] = h[k]; sp1[t * 64 + k] = p[k]; }
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // layer 2 and its tangent
  if (t == 0) {
    issue_layer(tm + 128, x_s, t_s + T_W2, 64, 64, 0);
    issue_layer(tm + 192, u_s, t_s + T_W2, 64, 64, 0);
    mma_commit(bar_a);
  }
  ok &= mbar_wait(bar_a, phase); phase ^= 1;
  tc_fence_after();
  {
    float zb[64], tb[64];
    for (int c = 0; c < 4; ++c) {
      float z[16], tv[16];
      tmem_ld16(lb + 128 + 16 * c, z);
      tmem_ld16(lb + 192 + 16 * c, tv);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int o = 16 * c + k;
        const float zz = z[k] + __ldg(C + SL_MLC_B2 + o);
        const float w3 = __ldg(C + SL_MLC_W3 + o);
        const float s1 = ml_dsilu(zz), s2 = ml_d2silu(zz);
        const float h2 = ml_silu(zz), p2 = s1 * tv[k];
        // dJ/dw3 = alpha h2 + p2; dJ/db2 = zbar2
        const float gw3 = warp_sum(alpha * h2 + p2);
        tb[o] = s1 * w3;
        zb[o] = s1 * alpha * w3 + s2 * tv[k] * w3;
        const float gb2 = warp_sum(zb[o]);
        if (lane == 0) { red[warp][o] = gw3; red[warp][64 + o] = gb2; }
      }
    }
    const float gb3 = warp_sum(alpha);
    if (lane == 0) red[warp][192] = gb3;
    store_row3(bx, t, zb, 64);
    store_row3(bu, t, tb, 64);
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // reverse through layer 2 (both streams): h1bar = zbar2 W2, p1bar = tbar2 W2
  if (t == 0) {
    issue_layer(tm + 128, x_s, t_s + T_W2T, 64, 64, 0);
    issue_layer(tm + 192, u_s, t_s + T_W2T, 64, 64, 0);
    mma_commit(bar_a);
  }
  // W2bar[o][i] = sum_a zbar2[a][o] h1[a][i] + tbar2[a][o] p1[a][i] while the MMAs run
  // (they only read X and U).  Thread t: rows o0..o0+3, columns i0..i0+7.
  float w2acc[4][8];
  {
    const int o0 = (t >> 3) * 4, i0 = (t & 7) * 8;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) w2acc[r][c] = 0.f;
    for (int at = 0; at < TILE; ++at) {
      float zr[4], tr[4], hh[8], pp[8];
#pragma unroll
      for (int r = 0; r < 4; ++r) { zr[r] = load3(bx, at, o0 + r, 64); tr[r] = load3(bu, at, o0 + r, 64); }
#pragma unroll
      for (int c = 0; c < 8; ++c) { hh[c] = sh1[at * 64 + i0 + c]; pp[c] = sp1[at * 64 + i0 + c]; }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) w2acc[r][c] = fmaf(zr[r], hh[c], fmaf(tr[r], pp[c], w2acc[r][c]));
    }
  }
  ok &= mbar_wait(bar_a, phase); phase ^= 1;
  tc_fence_after();
  __syncthreads();   // everyone is done with the stage before it is overwritten
  float* szb1 = stage;                 // [128][64] zbar1
  float* stb1 = stage + TILE * 64;     // [128][64] tbar1
  {
    for (int c = 0; c < 4; ++c) {
      float hb[16], pb[16], z[16], tv[16];
      tmem_ld16(lb + 128 + 16 * c, hb);
      tmem_ld16(lb + 192 + 16 * c, pb);
      tmem_ld16(lb + 0 + 16 * c, z);
      tmem_ld16(lb + 64 + 16 * c, tv);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int i = 16 * c + k;
        const float zz = z[k] + __ldg(C + SL_MLC_B1 + i);
        const float s1 = ml_dsilu(zz), s2 = ml_d2silu(zz);
        const float tb1 = s1 * pb[k];
        const float zb1 = s1 * hb[k] + s2 * tv[k] * pb[k];
        szb1[t * 64 + i] = zb1;
        stb1[t * 64 + i] = tb1;
        const float gb1 = warp_sum(zb1);
        if (lane == 0) red[warp][128 + i] = gb1;
      }
    }
  }
  // X and U are free now: restage x and u as float32 [128][48] each
  float* sx = (float*)bx;
  float* su = (float*)bu;
  {
    const float4* xi = (const float4*)(d.ml_x + (size_t)a * NF);
    const float4* ui = (const float4*)(d.ml_u + (size_t)a * NF);
#pragma unroll
    for (int u = 0; u < NF / 4; ++u) {
      float4 v = live ? xi[u] : make_float4(0.f, 0.f, 0.f, 0.f);
      float4 w = live ? ui[u] : make_float4(0.f, 0.f, 0.f, 0.f);
      *(float4*)(sx + t * NF + 4 * u) = v;
      *(float4*)(su + t * NF + 4 * u) = w;
    }
  }
  __syncthreads();
  // W1bar[o][f] = sum_a zbar1[a][o] x[a][f] + tbar1[a][o] u[a][f]:
  // thread t: rows o0..o0+3, columns f0..f0+5
  float w1acc[4][6];
  {
    const int o0 = (t >> 3) * 4, f0 = (t & 7) * 6;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 6; ++c) w1acc[r][c] = 0.f;
    for (int at = 0; at < TILE; ++at) {
      float zr[4], tr[4], xx[6], uu[6];
#pragma unroll
      for (int r = 0; r < 4; ++r) { zr[r] = szb1[at * 64 + o0 + r]; tr[r] = stb1[at * 64 + o0 + r]; }
#pragma unroll
      for (int c = 0; c < 6; ++c) { xx[c] = sx[at * NF + f0 + c]; uu[c] = su[at * NF + f0 + c]; }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) w1acc[r][c] = fmaf(zr[r], xx[c], fmaf(tr[r], uu[c], w1acc[r][c]));
    }
  }
  // write this block's partial gradient
  float* gp = d.ml_gpart + (size_t)blockIdx.x * SL_ML_NPARAM;
  {
    const int o0 = (t >> 3) * 4, f0 = (t & 7) * 6, i0 = (t & 7) * 8;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
      for (int c = 0; c < 6; ++c) gp[SL_ML_OFF_W1 + (o0 + r) * NF + f0 + c] = w1acc[r][c];
#pragma unroll
      for (int c = 0; c < 8; ++c) gp[SL_ML_OFF_W2 + (o0 + r) * NH + i0 + c] = w2acc[r][c];
    }
  }
  __syncthreads();
  if (t < 64) {
    gp[SL_ML_OFF_W3 + t] = red[0][t] + red[1][t] + red[2][t] + red[3][t];
    gp[SL_ML_OFF_B2 + t] = red[0][64 + t] + red[1][64 + t] + red[2][64 + t] + red[3][64 + t];
    gp[SL_ML_OFF_B1 + t] = red[0][128 + t] + red[1][128 + t] + red[2][128 + t] + red[3][128 + t];
  }
  if (t == 0) gp[SL_ML_OFF_B3] = red[0][192] + red[1][192] + red[2][192] + red[3][192];
  if (!ok && t == 0) sl_set_error(d.ctrl, SL_ERR_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, 256);
}

// Sum of the per-block partial gradients, in block order, in FP64.
__global__ void k_ml_grad_reduce(SlDev d, int nblk, double* out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= SL_ML_NPARAM) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += (double)d.ml_gpart[(size_t)b * SL_ML_NPARAM + p];
  d.ml_grad[p] = s;
  if (out) out[p] = s;
}

// Adam (Kingma and Ba, 2015, Algorithm 1) on the float32 master parameters,
// FP64 moments; t is the 1-based step.
__global__ void k_ml_adam(SlDev d, double lr, double b1, double b2, double eps, double c1, double c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= SL_ML_NPARAM) return;
  const double g = d.ml_grad[p];
  const double m = b1 * d.ml_m1[p] + (1.0 - b1) * g;
  const double v = b2 * d.ml_m2[p] + (1.0 - b2) * g * g;
  d.ml_m1[p] = m;
  d.ml_m2[p] = v;
  const double mh = m / c1, vh = v / c2;
  d.ml_par[p] = (float)((double)d.ml_par[p] - lr * mh / (sqrt(vh) + eps));
}

constexpr size_t MLP_SMEM = T_BYTES + ABUF + GUARD;

}  // namespace

int sl_ml_prepare_kernels() {
  if (cudaFuncSetAttribute(k_ml_mlp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_SMEM) != cudaSuccess)
    return SL_ERR_CUDA;
  if (cudaFuncSetAttribute(k_ml_train_mlp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TR_SMEM) != cudaSuccess)
    return SL_ERR_CUDA;
  if (cudaFuncSetAttribute(k_ml_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LS_SMEM) != cudaSuccess)
    return SL_ERR_CUDA;
  return SL_OK;
}

static inline int ntiles(const SlDev& d) { return (d.n + TILE - 1) / TILE; }

int sl_ml_launch_prep(const SlDev& d, cudaStream_t st) {
  k_ml_prep<<<(64 * 64 + 127) / 128, 128, 0, st>>>(d);
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}

int sl_ml_launch_point(const SlDev& d, cudaStream_t st, int fmode) {
  const int gn = grid_for(d.n);
  k_ml_desc<<<gn, SL_BLOCK, 0, st>>>(d, 1, nullptr, nullptr);
  k_ml_gate<<<1, 1, 0, st>>>(d);
  k_ml_mlp<<<ntiles(d), TILE, MLP_SMEM, st>>>(d, 0);
  k_ml_pair<<<gn, SL_BLOCK, 0, st>>>(d, fmode, 0, nullptr, nullptr);
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}

int sl_ml_launch_half_op(const SlDev& d, cudaStream_t st) {
  const int g = (d.s8 + LS_SPB - 1) / LS_SPB;
  const int gn = grid_for(d.n);
  auto sweep = [&](int predictor) {
    for (int p = 0; p < 16; ++p) {
      const int colour = p < 8 ? p : 15 - p;
      k_ml_sweep<<<g, LS_THREADS, LS_SMEM, st>>>(d, colour, p >= 8, predictor);
    }
  };
  // predictor with the start's (P, Q); (P, Q) at the predicted end averaged in;
  // corrector from the start spins (a closed gate skips all but the last sweep)
  k_ml_save_spins<<<gn, SL_BLOCK, 0, st>>>(d);
  sweep(1);
  k_ml_desc<<<gn, SL_BLOCK, 0, st>>>(d, 0, nullptr, nullptr);
  k_ml_mlp<<<ntiles(d), TILE, MLP_SMEM, st>>>(d, 0);
  k_ml_pair<<<gn, SL_BLOCK, 0, st>>>(d, 8, 0, nullptr, nullptr);
  k_ml_restore_spins<<<gn, SL_BLOCK, 0, st>>>(d);
  sweep(0);
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}

// Network at the current state with the gate ignored; per-replica E into
// d.ml_erep; optional caller-order outputs.
int sl_ml_launch_eval(const SlDev& d, cudaStream_t st, double* F, double* B, double* D) {
  const int gn = grid_for(d.n);
  k_ml_desc<<<gn, SL_BLOCK, 0, st>>>(d, 0, nullptr, D);
  k_ml_mlp<<<ntiles(d), TILE, MLP_SMEM, st>>>(d, 1);
  k_ml_pair<<<gn, SL_BLOCK, 0, st>>>(d, 4, 1, F, B);
  k_ml_e_caller<<<gn, SL_BLOCK, 0, st>>>(d, d.stage);
  k_ml_erep<<<d.nrep, RT, 0, st>>>(d, d.stage);
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}

int sl_ml_launch_dstats(const SlDev& d, cudaStream_t st, double* out_dev) {
  const int gn = grid_for(d.n);
  k_ml_desc<<<gn, SL_BLOCK, 0, st>>>(d, 0, d.ml_u, nullptr);
  k_ml_dstats<<<NF, RT, 0, st>>>(d, d.ml_u, out_dev);
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}

// Parameter gradient for caller-given upstream gradients into d.ml_grad
// (the network must have been evaluated at the current state).
int sl_ml_launch_vjp(const SlDev& d, cudaStream_t st, const double* gE, const double* gF, const double* gB) {
  const int gn = grid_for(d.n);
  k_ml_upstream<<<gn, SL_BLOCK, 0, st>>>(d, gE, gF, gB);
  k_ml_gbar<<<gn, SL_BLOCK, 0, st>>>(d);
  k_ml_train_mlp<<<ntiles(d), TILE, TR_SMEM, st>>>(d);
  k_ml_grad_reduce<<<(SL_ML_NPARAM + 127) / 128, 128, 0, st>>>(d, ntiles(d), nullptr);
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}

int sl_ml_launch_train(const SlDev& d, cudaStream_t st, const double* E_ref, const double* F_ref,
                       const double* B_ref, const double w[3], double lr, double b1, double b2, double eps,
                       long long t) {
  const int gn = grid_for(d.n);
  int e = sl_ml_launch_eval(d, st, nullptr, nullptr, nullptr);
  if (e) return e;
  k_ml_loss_atoms<<<gn, SL_BLOCK, 0, st>>>(d, F_ref, B_ref, w[1], w[2]);
  k_ml_loss_reduce<<<1, RT, 0, st>>>(d, E_ref, w[0], w[1], w[2]);
  k_ml_alpha<<<gn, SL_BLOCK, 0, st>>>(d);
  k_ml_gbar<<<gn, SL_BLOCK, 0, st>>>(d);
  k_ml_train_mlp<<<ntiles(d), TILE, TR_SMEM, st>>>(d);
  k_ml_grad_reduce<<<(SL_ML_NPARAM + 127) / 128, 128, 0, st>>>(d, ntiles(d), nullptr);
  const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  k_ml_adam<<<(SL_ML_NPARAM + 127) / 128, 128, 0, st>>>(d, lr, b1, b2, eps, c1, c2);
  return sl_ml_launch_prep(d, st);
}
