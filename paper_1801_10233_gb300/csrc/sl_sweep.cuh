// The spin half-op of the timestep (Eq. spin_ST_sectoring, Sec. 5.1): 8
// colour passes forward then 8 backward, the two passes of colour 7 in the
// middle as one launch; each pass turns every sector of one colour
// concurrently and the spins inside a sector in their sequential order
// (in-sector dependency levels).  Two families of pass kernels, the
// pipelined pass (k_sweep_pass) and the asynchronous-gather pass
// (k_sweep_async), in the tile shapes the autotuner chooses from; the rest
// of the step is in sl_step.cu.  The kernels are templates in an anonymous
// namespace: sl_sweep.cu instantiates the plain Hamiltonian's shapes,
// sl_sweep_so.cu those with the spin-orbit terms, so that the build
// compiles the two beside each other.
#pragma once
#include <algorithm>

#include "sl_internal.cuh"
#include "sl_df64.cuh"
#include "sl_pair.cuh"

namespace {

// ---------------------------------------------------------------------------
// One colour pass.  Block b takes SW_SPB consecutive sectors of the colour
// (their atoms are contiguous in the sorted order):
//   phase 1 (all warps, parallel over atoms): the exchange field from atoms
//           outside the atom's own sector -- either in full, or as the
//           partial field precomputed during the previous pass plus the
//           previous pass's colour group of the atom's exchange list -- the
//           noise of the spin bath, the atom's same-sector list (local
//           index, J) in a shared-memory pool, and its dependency levels;
//   phase 2 (warp 0): the block's spins level by level (one lane per spin
//           of a level; a spin's same-sector neighbours before it in the
//           sweep order are of lower levels), each adding the field of its
//           sector's spins to the external one, forming omega and rotating
//           -- shared memory only.  This is the sequential in-sector order's
//           result: spins of one level share no list edge.  A block whose
//           levels go beyond SW_LMAX runs one lane per sector in order.
//           Meanwhile warps 1.. precompute, for block b's sectors of the
//           next colour in the sweep, the external field of every
//           neighbour not of this pass's colour (those spins are final for
//           this pass: two contiguous ranges of the colour-grouped list);
//   phase 3 (all warps, parallel over atoms): add each increment to the
//           FP64 spin once and refresh its float split.
// Blocks with more than SW_MAXA atoms use workspace scratch and read their
// lists from global memory.
// ---------------------------------------------------------------------------
// Tile shapes (sectors per block SPB <= 32, threads per block): the
// variants the autotuner chooses from (sl_autotune), variant 0 the default.
// A block stages up to 12 atoms per sector in shared memory.
constexpr int SW_MAXIN = 6;    // same-sector staging entries per atom slot (a block's atoms share
                               // SW_MAXIN x SW_MAXA; an atom whose entries do not fit reads them
                               // from global memory)
constexpr int SW_BATCH = 2;    // external neighbours gathered per batch
// In-sector dependency levels handled per block: SW_LMAX per direction (a
// block with a deeper sector runs its sectors' chains one spin at a time).
// Shared words: starts [2][SW_LMAX + 1], cursors [2][SW_LMAX], the staged
// same-sector entries, the deep-block flag, 4 spare.
constexpr int SW_LMAX = 32;
constexpr int SW_LWORDS = 2 * (SW_LMAX + 1) + 2 * SW_LMAX + 6;

// Dynamic shared memory of one block with up to maxa atoms: H, S (and E
// with noise) as float2 [3 maxa], same-sector lists J [SW_MAXIN maxa]
// float2, local index [SW_MAXIN maxa] short, counts [maxa] int.
// A fused pass (one colour forward then backward) also keeps the external
// field X [3 maxa] and, with noise, the second pass's noise [3 maxa].
size_t sweep_smem_bytes(bool noise, int maxa, bool fused = false, bool levels = false) {
  return (size_t)(noise ? 3 : 2) * 3 * maxa * sizeof(float2) + (size_t)SW_MAXIN * maxa * sizeof(float2) +
         (size_t)SW_MAXIN * maxa * sizeof(short) + (size_t)maxa * sizeof(int) +
         (levels ? SW_LWORDS * sizeof(int) + 2 * (size_t)maxa * sizeof(short) : 0) +
         (fused ? (size_t)(noise ? 2 : 1) * 3 * maxa * sizeof(float2) : 0);
}

// (h, l) += sum of J_ij s_j (with SO: the field of the exchange, Neel and DMI
// terms of the pair) over entries [k0, k1) of atom i's exchange list.
template <bool SO>
__device__ __forceinline__ void ext_field(const SlDev& d, int i, int k0, int k1, float& hx, float& lx, float& hy,
                                          float& ly, float& hz, float& lz) {
  const size_t n = (size_t)d.n;
  for (int kb = k0; kb < k1; kb += SW_BATCH) {
    int jj[SW_BATCH];
    float2 JJ[SW_BATCH];
    float4 vh[SW_BATCH], vl[SW_BATCH];
#pragma unroll
    for (int q = 0; q < SW_BATCH; ++q) {
      if (kb + q < k1) {
        const size_t e = (size_t)(kb + q) * n + i;
        jj[q] = __ldg(d.exj + e);
        if (!SO) JJ[q] = __ldg(d.exJ + e);
      }
    }
#pragma unroll
    for (int q = 0; q < SW_BATCH; ++q)
      if (kb + q < k1) load_sdf(d.sdf, jj[q], vh[q], vl[q]);
#pragma unroll
    for (int q = 0; q < SW_BATCH; ++q) {
      if (kb + q < k1) {
        if constexpr (SO) {
          const SoEntry so = load_so(d, (size_t)(kb + q) * n + i);
          df3 sj;
          sj.x = df_make(vh[q].x, vl[q].x); sj.y = df_make(vh[q].y, vl[q].y); sj.z = df_make(vh[q].z, vl[q].z);
          so_field_acc(so, sj, hx, lx, hy, ly, hz, lz);
        } else {
          const df J = F2(JJ[q]);
          acc_prod(hx, lx, J, df_make(vh[q].x, vl[q].x));
          acc_prod(hy, ly, J, df_make(vh[q].y, vl[q].y));
          acc_prod(hz, lz, J, df_make(vh[q].z, vl[q].z));
        }
      }
    }
  }
}

// Programmatic dependent launch: each colour pass loads what the previous
// pass does not write (lists, levels, its own spins, noise) before it waits
// for that pass's results (pdl_wait), and lets the next pass's blocks be
// scheduled only after that wait (pdl_trigger): the pass before the previous
// one, which turned the next pass's colour in the fused sweep order 6, 7, 6,
// is then complete, so the next pass's early loads see its results.  Both
// are no-ops for a launch without the programmatic dependency.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Start of colour c's group among atom i's other-sector entries (c = 8: the end).
__device__ __forceinline__ int group_start(uint2 g, int c, int ne) {
  if (c >= 8) return ne;
  const unsigned w = c < 4 ? g.x : g.y;
  return (int)((w >> (8 * (c & 3))) & 0xFFu);
}

// One single-spin factor e^{L_si tau} of a colour pass, for the atom i of
// the block's atoms starting at a0: add the field of the spins of its own
// sector (their current values) to its external field Fx, form omega and
// rotate.  Reads and writes the block's staged buffers (S: spins, H:
// increments); `second` marks the fused pass's second chain, whose increment
// adds to the first one's and which draws the second noise (E2).
template <bool SO>
__device__ __forceinline__ void sweep_rotate(const SlDev& d, int i, int a0, bool fits, bool second,
                                             const float2* Fx, float2* H, float2* S, const float2* E,
                                             const float2* E2, const int* sh_in, const short* sh_iu,
                                             const float2* sh_ij, bool bath, bool noise) {
  const df tau = F2(d.tau_f);
  const size_t n = (size_t)d.n;
  const df ih = F2(d.inv_hbar_f);
  const int t = i - a0;
  const float2 f0 = Fx[3 * t], f1 = Fx[3 * t + 1], f2 = Fx[3 * t + 2];
  float hx = f0.x, lx = f0.y, hy = f1.x, ly = f1.y, hz = f2.x, lz = f2.y;
  float gx = 0.0f, kx = 0.0f, gy = 0.0f, ky = 0.0f, gz = 0.0f, kz = 0.0f;
  // sh_in[t] packs the same-sector count (low byte) and 1 + the first staged
  // entry (0: the atom's entries are read from global memory)
  const int pk = fits ? sh_in[t] : 0;
  const int ni = fits ? (pk & 0xFF) : d.exin[i];
  const int sb = (pk >> 8) - 1;
  if constexpr (SO) {
    // one accumulator, entries in list order (the same for every tile shape)
    for (int k = 0; k < ni; ++k) {
      const size_t e = (size_t)k * n + i;
      const int u = __ldg(d.exj + e) - a0;
      const SoEntry so = load_so(d, e);
      df3 sj;
      sj.x = F2(S[3 * u]); sj.y = F2(S[3 * u + 1]); sj.z = F2(S[3 * u + 2]);
      so_field_acc(so, sj, hx, lx, hy, ly, hz, lz);
    }
  } else {
    // the same-sector entries in pairs (two interleaved accumulators), from
    // shared memory where staged; the order is the same whatever is staged,
    // so every tile shape gives the same bits
    auto entry = [&](int k, int& u, df& J) {
      if (sb >= 0) {
        u = sh_iu[sb + k];
        J = F2(sh_ij[sb + k]);
      } else {
        const size_t e = (size_t)k * n + i;
        u = d.exj[e] - a0;
        J = F2(d.exJ[e]);
      }
    };
    int k = 0;
    for (; k + 1 < ni; k += 2) {
      int u0, u1;
      df J0, J1;
      entry(k, u0, J0);
      entry(k + 1, u1, J1);
      acc_prod(hx, lx, J0, F2(S[3 * u0]));
      acc_prod(gx, kx, J1, F2(S[3 * u1]));
      acc_prod(hy, ly, J0, F2(S[3 * u0 + 1]));
      acc_prod(gy, ky, J1, F2(S[3 * u1 + 1]));
      acc_prod(hz, lz, J0, F2(S[3 * u0 + 2]));
      acc_prod(gz, kz, J1, F2(S[3 * u1 + 2]));
    }
    if (k < ni) {
      int u0;
      df J0;
      entry(k, u0, J0);
      acc_prod(hx, lx, J0, F2(S[3 * u0]));
      acc_prod(hy, ly, J0, F2(S[3 * u0 + 1]));
      acc_prod(hz, lz, J0, F2(S[3 * u0 + 2]));
    }
  }
  // the two running sums (each kept normalised by acc_prod) combined with
  // the sloppy sum: they are partial fields, not nearly opposite ones, and
  // this sits on the dependent chain of the in-sector rotations
  df3 w;
  w.x = df_mul(df_add_sloppy(df_make(hx, lx), df_make(gx, kx)), ih);
  w.y = df_mul(df_add_sloppy(df_make(hy, ly), df_make(gy, ky)), ih);
  w.z = df_mul(df_add_sloppy(df_make(hz, lz), df_make(gz, kz)), ih);
  df3 s;
  s.x = F2(S[3 * t]); s.y = F2(S[3 * t + 1]); s.z = F2(S[3 * t + 2]);
  // uniaxial anisotropy: exact half turns about n before and after the
  // turn under the rest of omega; inc_a collects the first one's increment
  const bool aniso = SO && (d.so & SL_SO_ANISO);
  const int cayley = d.rotation == SL_ROT_CAYLEY;
  df3 inc_a;
  inc_a.x = inc_a.y = inc_a.z = df_f(0.0f);
  if (aniso) {
    inc_a = aniso_increment(d, s, F2(bath ? d.an_cl_f : d.an_c_f), df_scale(tau, 0.5f), cayley);
    s.x = df_add(s.x, inc_a.x); s.y = df_add(s.y, inc_a.y); s.z = df_add(s.z, inc_a.z);
  }
  if (bath) {
    // Eq. sLLG as ds/dt = Om x s, Om = (w + eta + lambda s x w) / (1 + lambda^2);
    // the damping term takes the whole omega, anisotropy included
    df3 wt = w;
    if (aniso) {
      const df3 a = aniso_vec(d, s, F2(d.an_c_f));
      wt.x = df_add(wt.x, a.x); wt.y = df_add(wt.y, a.y); wt.z = df_add(wt.z, a.z);
    }
    df3 sxw = cross3(s, wt);
    const df lam = F2(d.lam_f), inv = F2(d.inv1pl2_f);
    if (noise) {
      const float2* Ed = second ? E2 : E;
      w.x = df_add(w.x, F2(Ed[3 * t]));
      w.y = df_add(w.y, F2(Ed[3 * t + 1]));
      w.z = df_add(w.z, F2(Ed[3 * t + 2]));
    }
    w.x = df_mul(df_add(w.x, df_mul(lam, sxw.x)), inv);
    w.y = df_mul(df_add(w.y, df_mul(lam, sxw.y)), inv);
    w.z = df_mul(df_add(w.z, df_mul(lam, sxw.z)), inv);
  }
  df3 inc = rot_increment(w, s, tau, cayley);
  if (aniso) {
    s.x = df_add(s.x, inc.x); s.y = df_add(s.y, inc.y); s.z = df_add(s.z, inc.z);
    const df3 i2 = aniso_increment(d, s, F2(bath ? d.an_cl_f : d.an_c_f), df_scale(tau, 0.5f), cayley);
    s.x = df_add(s.x, i2.x); s.y = df_add(s.y, i2.y); s.z = df_add(s.z, i2.z);
    inc.x = df_add(df_add(inc_a.x, inc.x), i2.x);
    inc.y = df_add(df_add(inc_a.y, inc.y), i2.y);
    inc.z = df_add(df_add(inc_a.z, inc.z), i2.z);
    S[3 * t] = D2(s.x); S[3 * t + 1] = D2(s.y); S[3 * t + 2] = D2(s.z);
  } else {
    // the turned spin for the later same-sector neighbours (the FP64 state
    // takes the increment itself): |inc| is of order theta, so the sloppy
    // sum's error stays below 2^-47 of a unit component
    S[3 * t] = D2(df_add_sloppy(s.x, inc.x));
    S[3 * t + 1] = D2(df_add_sloppy(s.y, inc.y));
    S[3 * t + 2] = D2(df_add_sloppy(s.z, inc.z));
  }
  if (second) {   // the fused pass's second chain: total increment
    H[3 * t] = D2(df_add(F2(H[3 * t]), inc.x));
    H[3 * t + 1] = D2(df_add(F2(H[3 * t + 1]), inc.y));
    H[3 * t + 2] = D2(df_add(F2(H[3 * t + 2]), inc.z));
  } else {
    H[3 * t] = D2(inc.x);
    H[3 * t + 1] = D2(inc.y);
    H[3 * t + 2] = D2(inc.z);
  }
}

// Phase 2 of a colour pass for one sector q (one lane): every spin in order
// (ascending atom id forward, descending backward; both, one after the
// other, in the fused pass).
template <bool SO>
__device__ __forceinline__ void sweep_chain(const SlDev& d, int q, int a0, bool fits, bool both, int backward,
                                            const float2* Fx, float2* H, float2* S, const float2* E,
                                            const float2* E2, const int* sh_in, const short* sh_iu,
                                            const float2* sh_ij, bool bath, bool noise) {
  const int sa = d.sec_start[q], sb = d.sec_start[q + 1];
  const int m = sb - sa;
  for (int dir = 0; dir < (both ? 2 : 1); ++dir)
    for (int c = 0; c < m; ++c) {
      const int i = (both ? dir : backward) ? sb - 1 - c : sa + c;
      sweep_rotate<SO>(d, i, a0, fits, both && dir, Fx, H, S, E, E2, sh_in, sh_iu, sh_ij, bath, noise);
    }
}

// SW_RES: threads per SM the register budget is cut for (768: 80 registers;
// 1024: 64, no spills for the plain instance).
template <int SW_SPB, int SW_THREADS, bool SO, int SW_RES = 768>
__global__ void __launch_bounds__(SW_THREADS, SW_RES / SW_THREADS)
k_sweep_pass(SlDev d, int colour, int backward, int subpass, int prev_colour, int next_colour, int pin, int pout) {
  constexpr int SW_MAXA = 12 * SW_SPB;
  extern __shared__ float2 smem[];
  const bool noise = d.any_noise != 0;
  const bool bath = d.lambda != 0.0 || noise;
  float2* sh_h = smem;
  float2* sh_s = sh_h + 3 * SW_MAXA;
  float2* sh_e = sh_s + 3 * SW_MAXA;
  float2* sh_ij = sh_e + (noise ? 3 * SW_MAXA : 0);
  short* sh_iu = (short*)(sh_ij + SW_MAXIN * SW_MAXA);
  int* sh_in = (int*)(sh_iu + SW_MAXIN * SW_MAXA);
  // backward = 2: the fused pass, this colour forward then backward with the
  // same external field (no other colour turns in between), noise of
  // sub-passes `subpass` and `subpass + 1`
  const bool both = backward == 2;
  // level starts (forward, backward), cursors, then the atoms sorted by level
  int* sh_lc = sh_in + SW_MAXA;
  short* sh_ll = (short*)(sh_lc + SW_LWORDS);
  float2* sh_x = (float2*)(sh_ll + 2 * SW_MAXA);
  float2* sh_e2 = sh_x + 3 * SW_MAXA;

  const int s8 = d.s8;
  const int q0 = colour * s8 + blockIdx.x * SW_SPB;
  const int q1 = min(q0 + SW_SPB, (colour + 1) * s8);
  const int a0 = d.sec_start[q0], a1 = d.sec_start[q1];
  const int na = a1 - a0;
  const bool fits = na <= SW_MAXA;
  float2* H = fits ? sh_h : d.hbuf + 3 * (size_t)a0;
  float2* S = fits ? sh_s : d.sbuf + 3 * (size_t)a0;
  float2* E = fits ? sh_e : d.ebuf + 3 * (size_t)a0;
  float2* X = fits ? sh_x : d.xbuf + 3 * (size_t)a0;     // fused pass only
  float2* E2 = fits ? sh_e2 : d.ebuf2 + 3 * (size_t)a0;  // fused pass with noise only
  float2* Fx = both ? X : H;                              // where phase 1 puts the external field
  const long long step = d.ctrl->step;
  const df tau = F2(d.tau_f);
  const size_t n = (size_t)d.n;
  const float2* P = pin >= 0 ? d.hpart[pin] : nullptr;
  for (int w = threadIdx.x; w < SW_LWORDS; w += blockDim.x) sh_lc[w] = 0;
  __syncthreads();

  // phase 1, before the previous pass's results: levels, own spins,
  // same-sector lists, noise
  for (int t = threadIdx.x; t < na; t += blockDim.x) {
    const int i = a0 + t;
    if (fits) {
      // level counts, stored one place up for the exclusive scan; a level
      // beyond SW_LMAX marks the block deep
      const unsigned lv = __ldg(d.lvl + i);
      const int lf = (int)(lv & 0xFFu), lb = (int)(lv >> 8);
      if (lf < SW_LMAX && lb < SW_LMAX) {
        atomicAdd(sh_lc + lf + 1, 1);
        atomicAdd(sh_lc + SW_LMAX + 1 + lb + 1, 1);
      } else {
        sh_lc[SW_LWORDS - 1] = 1;
      }
    }
    float4 s4h, s4l;
    load_sdf(d.sdf, i, s4h, s4l);
    const int ni = __ldg(d.exin + i);
    if (fits) {
      // all of the atom's same-sector entries go to the block's staging pool
      // when they fit (read-only loads: free to run ahead of the stores)
      int sb = -1;
      if (!SO && ni > 0) {
        sb = atomicAdd(sh_lc + SW_LWORDS - 2, ni);
        if (sb + ni > SW_MAXIN * SW_MAXA) sb = -1;
      }
      if (sb >= 0) {
#pragma unroll 4
        for (int k = 0; k < ni; ++k) {
          const size_t e = (size_t)k * n + i;
          sh_iu[sb + k] = (short)(__ldg(d.exj + e) - a0);
          sh_ij[sb + k] = __ldg(d.exJ + e);
        }
      }
      sh_in[t] = ni | ((sb + 1) << 8);
    }
    S[3 * t] = make_float2(s4h.x, s4l.x);
    S[3 * t + 1] = make_float2(s4h.y, s4l.y);
    S[3 * t + 2] = make_float2(s4h.z, s4l.z);
    if (noise) {
      // eta ~ N(0, 2 D_S / |tau|), D_S = lambda (1 + lambda^2) k_B T / hbar;
      // counter (atom id within its replica, step, sub-pass, replica)
      const SlRep& R = d.reps[__ldg(d.arep + i)];
      for (int h = 0; h < (both ? 2 : 1); ++h) {
        df3 g;
        g.x = g.y = g.z = df_f(0.0f);
        df sig = df_f(0.0f);
        if (R.temperature > 0.0) {
          g = gauss3_df(d.seed, R.replica, step, subpass + h, d.perm[i] - R.atom0);
          sig = F2(R.noise_sig);
        }
        float2* Eh = h ? E2 : E;
        Eh[3 * t] = D2(df_mul(sig, g.x));
        Eh[3 * t + 1] = D2(df_mul(sig, g.y));
        Eh[3 * t + 2] = D2(df_mul(sig, g.z));
      }
    }
  }
  pdl_wait();
  pdl_trigger();

  // phase 1, the external field: the partial field of every other colour
  // plus the colour the previous pass turned (the first pass: all of it)
  for (int t = threadIdx.x; t < na; t += blockDim.x) {
    const int i = a0 + t;
    const int ne = __ldg(d.exn + i);
    float hx, lx, hy, ly, hz, lz;
    if (P) {
      const float2 p0 = __ldcg(P + 3 * (size_t)i), p1 = __ldcg(P + 3 * (size_t)i + 1),
                   p2 = __ldcg(P + 3 * (size_t)i + 2);
      hx = p0.x; lx = p0.y; hy = p1.x; ly = p1.y; hz = p2.x; lz = p2.y;
      const uint2 g = __ldg(d.exc + i);
      ext_field<SO>(d, i, group_start(g, prev_colour, ne), group_start(g, prev_colour + 1, ne), hx, lx, hy, ly, hz,
                    lz);
    } else {
      hx = d.zee_f[0].x; lx = d.zee_f[0].y;
      hy = d.zee_f[1].x; ly = d.zee_f[1].y;
      hz = d.zee_f[2].x; lz = d.zee_f[2].y;
      ext_field<SO>(d, i, __ldg(d.exin + i), ne, hx, lx, hy, ly, hz, lz);
    }
    Fx[3 * t] = D2(acc_done(hx, lx));
    Fx[3 * t + 1] = D2(acc_done(hy, ly));
    Fx[3 * t + 2] = D2(acc_done(hz, lz));
  }
  __syncthreads();

  if (threadIdx.x < 32) {
    // phase 2 (warp 0)
    const int lane = threadIdx.x;
    if (fits && sh_lc[SW_LWORDS - 1] == 0) {
      // the block's spins level by level: spins of one level have no list
      // edge between them, and every same-sector neighbour they read is final
      // (lower level) or untouched (higher level), as in the sequential order
      int* st = sh_lc;                               // [2][SW_LMAX + 1]
      int* cur = sh_lc + 2 * (SW_LMAX + 1);          // [2][SW_LMAX]
      for (int h = 0; h < 2; ++h) {
        int* c = st + h * (SW_LMAX + 1);
        int v = c[lane + 1];                         // count of level `lane`
        for (int o = 1; o < 32; o <<= 1) {
          const int u = __shfl_up_sync(0xffffffffu, v, o);
          if (lane >= o) v += u;
        }
        c[lane + 1] = v;                             // starts of levels 1 .. 32 (level 0 starts at 0)
      }
      __syncwarp();
      for (int h = 0; h < 2; ++h) cur[h * SW_LMAX + lane] = st[h * (SW_LMAX + 1) + lane];
      __syncwarp();
      for (int t = lane; t < na; t += 32) {
        const unsigned lv = __ldg(d.lvl + a0 + t);
        sh_ll[atomicAdd(cur + (lv & 0xFFu), 1)] = (short)t;
        sh_ll[SW_MAXA + atomicAdd(cur + SW_LMAX + (lv >> 8), 1)] = (short)t;
      }
      __syncwarp();
      for (int dir = 0; dir < (both ? 2 : 1); ++dir) {
        const int h = (both ? dir : backward) ? 1 : 0;
        const int* c = st + h * (SW_LMAX + 1);
        const short* list = sh_ll + h * SW_MAXA;
        for (int lev = 0; lev < SW_LMAX && c[lev] < na; ++lev) {
          for (int x = c[lev] + lane; x < c[lev + 1]; x += 32)
            sweep_rotate<SO>(d, a0 + list[x], a0, fits, both && dir, Fx, H, S, E, E2, sh_in, sh_iu, sh_ij, bath,
                             noise);
          __syncwarp();
        }
      }
    } else {
      const int q = q0 + lane;
      if (q < q1)
        sweep_chain<SO>(d, q, a0, fits, both, backward, Fx, H, S, E, E2, sh_in, sh_iu, sh_ij, bath, noise);
    }
  } else if (pout >= 0) {
    // precompute the next pass's partial external field (all neighbours not
    // of this pass's colour) for block b's sectors of the next colour
    const int nq0 = next_colour * s8 + blockIdx.x * SW_SPB;
    const int nq1 = min(nq0 + SW_SPB, (next_colour + 1) * s8);
    const int n0 = d.sec_start[nq0], n1 = d.sec_start[nq1];
    float2* Q = d.hpart[pout];
    for (int t = threadIdx.x - 32; t < n1 - n0; t += blockDim.x - 32) {
      const int i = n0 + t;
      float hx = d.zee_f[0].x, lx = d.zee_f[0].y;
      float hy = d.zee_f[1].x, ly = d.zee_f[1].y;
      float hz = d.zee_f[2].x, lz = d.zee_f[2].y;
      // every other-sector neighbour not of this pass's colour: two ranges
      const int ne = __ldg(d.exn + i);
      const uint2 g = __ldg(d.exc + i);
      ext_field<SO>(d, i, __ldg(d.exin + i), group_start(g, colour, ne), hx, lx, hy, ly, hz, lz);
      ext_field<SO>(d, i, group_start(g, colour + 1, ne), ne, hx, lx, hy, ly, hz, lz);
      Q[3 * (size_t)i] = make_float2(hx, lx);
      Q[3 * (size_t)i + 1] = make_float2(hy, ly);
      Q[3 * (size_t)i + 2] = make_float2(hz, lz);
    }
  }
  __syncthreads();

  // phase 3
  for (int t = threadIdx.x; t < na; t += blockDim.x) {
    const int i = a0 + t;
    double4_32a s = d.s[i];
    s.x += df_to_double(F2(H[3 * t]));
    s.y += df_to_double(F2(H[3 * t + 1]));
    s.z += df_to_double(F2(H[3 * t + 2]));
    d.s[i] = s;
    store_spin_split(d, i, s);
  }
}

// ---------------------------------------------------------------------------
// Colour pass with asynchronous gathers (the plain exchange Hamiltonian, with
// or without the spin bath).  The external field of a pass's spins comes from
// the spins of other sectors, which no block of the pass changes; a block
// therefore copies, for each of its atoms, every other-sector neighbour's spin
// (hi and lo halves) and J_ij into a shared-memory pool with cp.async before
// it sums anything, so all of a block's gathers are in flight at once instead
// of a few per thread.  Slots are handed out per atom from a shared counter;
// entries beyond the pool are read from global memory when summed.  The sum
// is the Zeeman term plus the other-sector entries in list order, the same
// for every tile shape.  Phases 2 and 3 are those of k_sweep_pass.
// ---------------------------------------------------------------------------
constexpr int SW_SLOTS_PER_ATOM = 8;      // pool slots (other-sector entries) per atom a block can hold
constexpr int SW_JSPEC = 16;              // list rows whose indices load with the counts

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(a), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Pool bytes of a block for maxa atoms: hi and lo float4 and J float2 per
// slot, the slot counter and the largest levels.
size_t sweep_pool_bytes(int maxa) {
  return (size_t)SW_SLOTS_PER_ATOM * maxa * (2 * sizeof(float4) + sizeof(float2)) + 16;
}

template <int SW_SPB, int SW_THREADS, int SW_MAXA>
__global__ void __launch_bounds__(SW_THREADS, 768 / SW_THREADS)
k_sweep_async(SlDev d, int colour, int backward, int subpass, int prev_colour) {
  constexpr int SLOTS = SW_SLOTS_PER_ATOM * SW_MAXA;
  extern __shared__ float4 smem4[];
  float4* ph = smem4;                                   // [SLOTS] neighbour spins, hi halves
  float4* pl = ph + SLOTS;                              // [SLOTS] lo halves
  float2* pJ = reinterpret_cast<float2*>(pl + SLOTS);   // [SLOTS] J_ij
  int* used = reinterpret_cast<int*>(pJ + SLOTS);       // pool slots, largest levels, staged entries
  float2* sh_h = reinterpret_cast<float2*>(used + 4);
  const bool noise = d.any_noise != 0;
  const bool bath = d.lambda != 0.0 || noise;
  float2* sh_s = sh_h + 3 * SW_MAXA;
  float2* sh_e = sh_s + 3 * SW_MAXA;
  float2* sh_ij = sh_e + (noise ? 3 * SW_MAXA : 0);
  short* sh_iu = (short*)(sh_ij + SW_MAXIN * SW_MAXA);
  int* sh_in = (int*)(sh_iu + SW_MAXIN * SW_MAXA);
  const bool both = backward == 2;
  float2* sh_x = (float2*)(sh_in + SW_MAXA);
  float2* sh_e2 = sh_x + 3 * SW_MAXA;
  int* sh_base = (int*)(sh_e2 + (noise ? 3 * SW_MAXA : 0));   // [SW_MAXA] first slot of each atom
  unsigned short* sh_lv = (unsigned short*)(sh_base + SW_MAXA); // [SW_MAXA] levels

  const int s8 = d.s8;
  const int q0 = colour * s8 + blockIdx.x * SW_SPB;
  const int q1 = min(q0 + SW_SPB, (colour + 1) * s8);
  const int a0 = d.sec_start[q0], a1 = d.sec_start[q1];
  const int na = a1 - a0;
  const bool fits = na <= SW_MAXA;
  float2* H = fits ? sh_h : d.hbuf + 3 * (size_t)a0;
  float2* S = fits ? sh_s : d.sbuf + 3 * (size_t)a0;
  float2* E = fits ? sh_e : d.ebuf + 3 * (size_t)a0;
  float2* X = fits ? sh_x : d.xbuf + 3 * (size_t)a0;
  float2* E2 = fits ? sh_e2 : d.ebuf2 + 3 * (size_t)a0;
  float2* Fx = both ? X : H;
  const long long step = d.ctrl->step;
  const size_t n = (size_t)d.n;
  const int jspec = min(SW_JSPEC, d.max_ex);
  if (threadIdx.x == 0) { used[0] = 0; used[1] = 0; used[2] = 0; used[3] = 0; }
  __syncthreads();

  // phase 1a: the counts and the first SW_JSPEC neighbour indices in one
  // round (rows beyond the count are read but not used), then asynchronous
  // copies of every other-sector neighbour's spin and J into the pool and of
  // the staged same-sector J values; meanwhile the atom's own spin, levels
  // and noise
  for (int t = threadIdx.x; t < na; t += blockDim.x) {
    const int i = a0 + t;
    int jj[SW_JSPEC];
#pragma unroll
    for (int q = 0; q < SW_JSPEC; ++q)
      if (q < jspec) jj[q] = __ldg(d.exj + (size_t)q * n + i);
    const int ni = __ldg(d.exin + i), ne = __ldg(d.exn + i);
    const unsigned lv = __ldg(d.lvl + i);
    const int cnt = fits ? ne - ni : 0;           // a block beyond SW_MAXA atoms reads global memory
    const int base = cnt > 0 ? atomicAdd(used, cnt) : SLOTS;
    const int nslot = max(0, min(cnt, SLOTS - base));
    pdl_wait();                                   // the neighbours' spins are the previous pass's results
#pragma unroll
    for (int q = 0; q < SW_JSPEC; ++q) {
      const int k = q - ni;                       // pool entry of list row q
      if (q < jspec && k >= 0 && k < nslot) {
        cp_async16(ph + base + k, d.sdf + 2 * (size_t)jj[q]);
        cp_async16(pl + base + k, d.sdf + 2 * (size_t)jj[q] + 1);
        cp_async8(pJ + base + k, d.exJ + (size_t)q * n + i);
      }
    }
    for (int q = jspec; q < ni + nslot; ++q) {    // rows beyond the speculative ones
      const int k = q - ni;
      if (k < 0) continue;
      const int j = __ldg(d.exj + (size_t)q * n + i);
      cp_async16(ph + base + k, d.sdf + 2 * (size_t)j);
      cp_async16(pl + base + k, d.sdf + 2 * (size_t)j + 1);
      cp_async8(pJ + base + k, d.exJ + (size_t)q * n + i);
    }
    if (fits) {
      // all of the atom's same-sector entries to the staging pool when they fit
      int sb = -1;
      if (ni > 0) {
        sb = atomicAdd(used + 3, ni);
        if (sb + ni > SW_MAXIN * SW_MAXA) sb = -1;
      }
      if (sb >= 0) {
#pragma unroll
        for (int q = 0; q < SW_JSPEC; ++q)
          if (q < ni && q < jspec) {
            sh_iu[sb + q] = (short)(jj[q] - a0);
            cp_async8(sh_ij + sb + q, d.exJ + (size_t)q * n + i);
          }
        for (int q = jspec; q < ni; ++q) {
          sh_iu[sb + q] = (short)(__ldg(d.exj + (size_t)q * n + i) - a0);
          cp_async8(sh_ij + sb + q, d.exJ + (size_t)q * n + i);
        }
      }
      sh_in[t] = ni | ((sb + 1) << 8);
      sh_base[t] = base;
      sh_lv[t] = (unsigned short)lv;
    }
    atomicMax(used + 1, (int)(lv & 0xFFu));
    atomicMax(used + 2, (int)(lv >> 8));
    float4 s4h, s4l;
    load_sdf(d.sdf, i, s4h, s4l);
    S[3 * t] = make_float2(s4h.x, s4l.x);
    S[3 * t + 1] = make_float2(s4h.y, s4l.y);
    S[3 * t + 2] = make_float2(s4h.z, s4l.z);
    if (noise) {
      // eta ~ N(0, 2 D_S / |tau|) per component; counter (atom id within its
      // replica, step, sub-pass, replica)
      const SlRep& R = d.reps[__ldg(d.arep + i)];
      for (int h = 0; h < (both ? 2 : 1); ++h) {
        df3 g;
        g.x = g.y = g.z = df_f(0.0f);
        df sig = df_f(0.0f);
        if (R.temperature > 0.0) {
          g = gauss3_df(d.seed, R.replica, step, subpass + h, d.perm[i] - R.atom0);
          sig = F2(R.noise_sig);
        }
        float2* Eh = h ? E2 : E;
        Eh[3 * t] = D2(df_mul(sig, g.x));
        Eh[3 * t + 1] = D2(df_mul(sig, g.y));
        Eh[3 * t + 2] = D2(df_mul(sig, g.z));
      }
    }
  }
  pdl_wait();                                     // (threads without an atom)
  pdl_trigger();
  cp_async_wait_all();

  // phase 1b: each thread sums the external field of the atoms whose copies
  // it issued (complete after its own wait).  The order is the pipelined
  // pass's, so that every tile shape gives the same bits: the Zeeman term,
  // the other-sector entries not of the previous pass's colour in list
  // order, then that colour's group (the first pass: all in list order).
  for (int t = threadIdx.x; t < na; t += blockDim.x) {
    const int i = a0 + t;
    const int ni = fits ? (sh_in[t] & 0xFF) : __ldg(d.exin + i), ne = __ldg(d.exn + i);
    const int base = fits ? sh_base[t] : SLOTS;
    int g0 = ne, g1 = ne;                        // the previous colour's group
    if (prev_colour >= 0) {
      const uint2 g = __ldg(d.exc + i);
      g0 = group_start(g, prev_colour, ne);
      g1 = group_start(g, prev_colour + 1, ne);
    }
    float hx = d.zee_f[0].x, lx = d.zee_f[0].y;
    float hy = d.zee_f[1].x, ly = d.zee_f[1].y;
    float hz = d.zee_f[2].x, lz = d.zee_f[2].y;
    auto add = [&](int k) {
      const int slot = base + (k - ni);
      float4 vh, vl;
      df J;
      if (slot < SLOTS) {
        vh = ph[slot]; vl = pl[slot]; J = F2(pJ[slot]);
      } else {
        const size_t e = (size_t)k * n + i;
        const int j = __ldg(d.exj + e);
        load_sdf(d.sdf, j, vh, vl);
        J = F2(__ldg(d.exJ + e));
      }
      acc_prod(hx, lx, J, df_make(vh.x, vl.x));
      acc_prod(hy, ly, J, df_make(vh.y, vl.y));
      acc_prod(hz, lz, J, df_make(vh.z, vl.z));
    };
    for (int k = ni; k < g0; ++k) add(k);
    for (int k = g1; k < ne; ++k) add(k);
    for (int k = g0; k < g1; ++k) add(k);
    Fx[3 * t] = D2(acc_done(hx, lx));
    Fx[3 * t + 1] = D2(acc_done(hy, ly));
    Fx[3 * t + 2] = D2(acc_done(hz, lz));
  }
  __syncthreads();

  // phase 2: the in-sector sweeps level by level (all threads): the spins of
  // one level have no list edge between them, and every same-sector
  // neighbour they read is final (lower level) or untouched (higher level),
  // as in the sequential order
  const int mf = used[1], mb = used[2];
  const int nlev = both ? mf + mb + 2 : (backward ? mb + 1 : mf + 1);
  for (int L = 0; L < nlev; ++L) {
    const bool second = both && L > mf;
    const bool bw = both ? second : backward != 0;
    const int lev = second ? L - mf - 1 : L;
    for (int t = threadIdx.x; t < na; t += blockDim.x) {
      const unsigned lv = fits ? sh_lv[t] : __ldg(d.lvl + a0 + t);
      if ((int)(bw ? lv >> 8 : lv & 0xFFu) == lev)
        sweep_rotate<false>(d, a0 + t, a0, fits, second, Fx, H, S, E, E2, sh_in, sh_iu, sh_ij, bath, noise);
    }
    __syncthreads();
  }

  // phase 3: one FP64 add per component, then the float split
  for (int t = threadIdx.x; t < na; t += blockDim.x) {
    const int i = a0 + t;
    double4_32a sv = d.s[i];
    sv.x += df_to_double(F2(H[3 * t]));
    sv.y += df_to_double(F2(H[3 * t + 1]));
    sv.z += df_to_double(F2(H[3 * t + 2]));
    d.s[i] = sv;
    store_spin_split(d, i, sv);
  }
}

// The passes of a spin half-op: colours 0..6 forward, colour 7 forward then
// backward in one fused pass (nothing of another colour turns between the
// two), colours 6..0 backward.  Pass p reads the partial field written by
// pass p - 1 (none for p = 0) and precomputes the next pass's.
// Launch with programmatic stream serialization (pdl = true): the kernel may
// start while the previous one finishes; it waits for it with
// griddepcontrol.wait.  The first pass of a half-op is launched plainly: the
// kernel before it may be the last pass of the other half-op, which turns the
// same colour (spin-only dynamics), or any kernel of the step.
template <typename... KArgs, typename... Args>
void launch_pdl(bool pdl, void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
                Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

template <int SPB, int THREADS, bool SO, int RES = 768>
void launch_half_op_t(const SlDev& d, cudaStream_t st, int subpass0) {
  int g = (d.s8 + SPB - 1) / SPB;
  const bool noise = d.any_noise != 0;
  int col[SL_SWEEP_PASSES], bwd[SL_SWEEP_PASSES];
  for (int p = 0; p < 7; ++p) { col[p] = p; bwd[p] = 0; col[14 - p] = p; bwd[14 - p] = 1; }
  col[7] = 7; bwd[7] = 2;
  for (int p = 0; p < SL_SWEEP_PASSES; ++p) {
    const int prev = p > 0 ? col[p - 1] : -1;
    const int next = p < SL_SWEEP_PASSES - 1 ? col[p + 1] : -1;
    const int pin = p > 0 ? (p - 1) & 1 : -1;
    const int pout = p < SL_SWEEP_PASSES - 1 ? p & 1 : -1;
    const size_t sm = sweep_smem_bytes(noise, 12 * SPB, bwd[p] == 2, true);
    launch_pdl(p > 0, k_sweep_pass<SPB, THREADS, SO, RES>, g, THREADS, sm, st, d, col[p], bwd[p],
               subpass0 + (bwd[p] == 1), prev, next, pin, pout);
  }
}

// Shared memory of the asynchronous-gather pass: the pool, the staged
// buffers of the fused layout, the per-atom slot bases and levels.
size_t sweep_async_smem(bool noise, int maxa) {
  return sweep_pool_bytes(maxa) + sweep_smem_bytes(noise, maxa, true) + (size_t)maxa * (sizeof(int) + 2) + 16;
}

template <int SPB, int THREADS, int MAXA>
void launch_half_op_async_t(const SlDev& d, cudaStream_t st, int subpass0) {
  const int g = (d.s8 + SPB - 1) / SPB;
  const size_t sm = sweep_async_smem(d.any_noise != 0, MAXA);
  for (int p = 0; p < SL_SWEEP_PASSES; ++p) {
    const int col = p < 7 ? p : (p == 7 ? 7 : 14 - p);
    const int bwd = p < 7 ? 0 : (p == 7 ? 2 : 1);
    const int prev = p == 0 ? -1 : (p - 1 < 7 ? p - 1 : (p - 1 == 7 ? 7 : 14 - (p - 1)));
    launch_pdl(p > 0, k_sweep_async<SPB, THREADS, MAXA>, g, THREADS, sm, st, d, col, bwd, subpass0 + (bwd == 1), prev);
  }
}

}  // namespace
