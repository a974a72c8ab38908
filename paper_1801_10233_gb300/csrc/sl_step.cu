// One timestep of Eq. general_ST_decomposition (Sec. 3, arXiv 1801.10233):
//   half-kick, spin half-op, drift (+ rebuild check, exchange table),
//   spin half-op, forces + half-kick.
// The spin half-op e^{Ls dt/2} is 8 colour passes forward then 8 backward
// (Eq. spin_ST_sectoring, Sec. 5.1); each pass updates every sector of one
// colour concurrently, the spins inside a sector one after another.  The two
// passes of colour 7 in the middle run as one launch.
//
// The FP64 state (r, v, s, F) is authoritative.  Pair and rotation arithmetic
// runs in double-float on the FP32 pipes (sl_df64.cuh) from copies of r (64-bit
// fixed point, exact differences) and s (float pairs), and each result is
// added to the FP64 state once per atom.
#include <algorithm>

#include "sl_internal.cuh"
#include "sl_df64.cuh"
#include "sl_pair.cuh"

namespace {

inline int grid_for(int n) { return (n + SL_BLOCK - 1) / SL_BLOCK; }

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

__global__ void k_kick(SlDev d, double h) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.n) return;
  double c = h * d.acc;
  double4_32a v = d.v[k], F = d.F[k];
  if (d.any_lattice_bath) v = lattice_bath(d, k, v, 4);
  v.x = fma(c, F.x, v.x); v.y = fma(c, F.y, v.y); v.z = fma(c, F.z, v.z);
  d.v[k] = v;
}

// r += dt v, the fixed-point copy of r, the largest displacement since the
// last rebuild (float, from the exact fixed-point difference) and a
// finiteness check on the bits: the only FP64 arithmetic is the drift itself.
__global__ void k_drift(SlDev d) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  float m = 0.0f;
  if (k < d.n) {
    double4_32a r = d.r[k];
    const double4_32a v = d.v[k];
    r.x = fma(d.dt, v.x, r.x); r.y = fma(d.dt, v.y, r.y); r.z = fma(d.dt, v.z, r.z);
    d.r[k] = r;
    const SlFix x = fx_pos(r);
    d.rx[k] = x;
    m = fx_dist2(x, d.rbx[k]);
    if (!finite3(r) || !(m == m)) sl_set_error(d.ctrl, SL_ERR_NONFINITE);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0f)
    atomicMax(&d.ctrl->maxdisp2_bits, (unsigned long long)__double_as_longlong((double)m));
}

// Decide whether this step re-sectors (displacement trigger or schedule).
__global__ void k_decide(SlDev d) {
  SlCtrl* c = d.ctrl;
  double md2 = __longlong_as_double((long long)c->maxdisp2_bits);
  int need;
  if (d.rebuild_every > 0) {
    need = ((c->step + 1) % d.rebuild_every) == 0;
    if (!need && md2 > d.half_skin2) sl_set_error(c, SL_ERR_SKIN);
  } else {
    need = md2 > d.half_skin2;
  }
  c->need_rebuild = need;
  c->maxdisp2_bits = 0ull;
}

// Exchange coefficients at the current positions (recomputed after every
// drift, Sec. 3): J_ij = 4 alpha x (1 - gamma x) e^{-x}, x = r_ij^2/delta^2
// (Eq. BSfunction), zero beyond the cutoff.
// Embedding density: (h, l) += f(r) = x^2 (1 + (beta/d) x), x = r - d, for r^2 < d^2.
__device__ __forceinline__ void eam_f_acc(const SlDev& d, df r2, float& h, float& l) {
  if (!df_lt(r2, F2(d.em_d2_f))) return;
  const df x = df_sub(df_mul(r2, df_rsqrt(r2)), F2(d.em_d_f));
  acc_prod(h, l, df_sqr(x), df_add_f(df_mul(F2(d.em_bd_f), x), 1.0f));
}

// F'(rho_i) = -(A/2)/sqrt(rho_i) (0 at rho = 0) into the per-atom table.
__device__ __forceinline__ void eam_store_fp(const SlDev& d, int i, float h, float l) {
  const df rho = acc_done(h, l);
  const df fp = rho.hi > 0.0f ? df_neg(df_mul(F2(d.em_hA_f), df_rsqrt(rho))) : df_f(0.0f);
  d.em_fp[i] = D2(fp);
}

// SO: also the spin-orbit tables (g1, d, e); DENS: also the embedding density
// (when its cutoff d is within the exchange cutoff, the exchange entries hold
// every pair it needs).  The plain instance carries none of that code.
template <bool SO, bool DENS>
__global__ void k_jtable(SlDev d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  if (d.ham == SL_HAM_LEARNED && d.ctrl->ml_use) return;   // the network is in effect here
  const p3 pi = load_pos(d, i);
  const box3 B = load_box(d, d.reps[__ldg(d.arep + i)]);
  const int ne = d.exn[i];
  const size_t n = (size_t)d.n;
  const df ix = F2(d.ex_ix_f), a4 = F2(d.ex_4a_f), g = F2(d.ex_g_f), a8 = F2(d.ex_8ad2_f);
  const df rc2 = F2(d.ex_rc2_f);
  float rh = 0.0f, rl = 0.0f;   // embedding density
  for (int k = 0; k < ne; ++k) {
    const size_t e = (size_t)k * n + i;
    const int j = __ldg(d.exj + e);
    const df3 dd = pair_sep(B, pi, load_pos(d, j));
    const df r2 = sep_r2(dd);
    if (DENS) eam_f_acc(d, r2, rh, rl);
    df J = df_f(0.0f), dJr = df_f(0.0f);
    const bool in = df_lt(r2, rc2);
    if (in) {
      const df x = df_mul(r2, ix);
      const df ex = df_exp(df_neg(x));
      const df gx = df_mul(g, x);
      J = df_mul(df_mul(a4, x), df_mul(df_add_f(df_neg(gx), 1.0f), ex));
      // J'(r)/r = 8 alpha/delta^2 e^{-x} (1 - x (1 + 2 g - g x)) for the forces
      const df poly = df_add_f(df_neg(df_mul(x, df_add_f(df_sub(df_scale(g, 2.0f), gx), 1.0f))), 1.0f);
      dJr = df_mul(df_mul(a8, ex), poly);
    }
    d.exJ[e] = D2(J);
    d.exdJ[e] = D2(dJr);
    if (SO && d.exso) {
      // g1(r), d(r) and e = (r_j - r_i)/r of the spin-orbit pair terms
      const size_t P = (size_t)d.max_ex * n;
      df g1 = df_f(0.0f), dm = df_f(0.0f), fpr;
      df3 u;
      u.x = u.y = u.z = df_f(0.0f);
      if (in) {
        const df rinv = df_rsqrt(r2);
        u.x = df_mul(dd.x, rinv); u.y = df_mul(dd.y, rinv); u.z = df_mul(dd.z, rinv);
        if (d.so & SL_SO_NEEL) bs_eval(d.ne_bs, r2, g1, fpr);
        if (d.so & SL_SO_DMI) bs_eval(d.dm_bs, r2, dm, fpr);
      }
      d.exso[e] = D2(g1);
      d.exso[P + e] = D2(dm);
      d.exso[2 * P + e] = D2(u.x);
      d.exso[3 * P + e] = D2(u.y);
      d.exso[4 * P + e] = D2(u.z);
    }
  }
  if (DENS) eam_store_fp(d, i, rh, rl);
}

// Embedding density rho_i = sum_j f(r_ij) over the Morse list (r < d) and
// F'(rho_i), at the current positions, when d lies beyond the exchange cutoff
// (otherwise k_jtable computes it): recomputed after every drift, read by
// the force kernel for both atoms of a pair.
__global__ void k_density(SlDev d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  const p3 pi = load_pos(d, i);
  const box3 B = load_box(d, d.reps[__ldg(d.arep + i)]);
  const int nm = d.mn[i];
  if (d.mech & SL_MECH_TAB) {
    // tabulated form: rho_i = sum_j rho(r_ij) over r < morse_rc, then F'(rho_i)
    const df rc2 = F2(d.m_rc2_f);
    const float rc2_hi = rc2.hi * 1.0001f;
    df rho = df_f(0.0f);
    for (int k = 0; k < nm; ++k) {
      const int j = __ldg(d.mj + (size_t)k * d.n + i);
      const p3 pj = load_pos(d, j);
      const pre3 q = pair_pre(B, pi, pj);
      if (q.r2 > rc2_hi) continue;
      const df3 dd = pair_sep_k(B, pi, pj, q);
      float a = 0.0f, b = 0.0f;
      acc_prod(a, b, dd.x, dd.x);
      acc_prod(a, b, dd.y, dd.y);
      acc_prod(a, b, dd.z, dd.z);
      const df r2 = acc_done(a, b);
      if (!df_lt(r2, rc2)) continue;
      rho = df_add(rho, tab_value_df(d, SL_TAB_RHO, df_mul(r2, df_rsqrt(r2)), nullptr));
    }
    df fp;
    tab_value_df(d, SL_TAB_F, rho, &fp);
    d.em_fp[i] = D2(fp);
    return;
  }
  const float d2_hi = F2(d.em_d2_f).hi * 1.0001f;
  float h = 0.0f, l = 0.0f;
  for (int k = 0; k < nm; ++k) {
    const int j = __ldg(d.mj + (size_t)k * d.n + i);
    const p3 pj = load_pos(d, j);
    const pre3 q = pair_pre(B, pi, pj);
    if (q.r2 > d2_hi) continue;
    const df3 dd = pair_sep_k(B, pi, pj, q);
    float a = 0.0f, b = 0.0f;
    acc_prod(a, b, dd.x, dd.x);
    acc_prod(a, b, dd.y, dd.y);
    acc_prod(a, b, dd.z, dd.z);
    eam_f_acc(d, acc_done(a, b), h, l);
  }
  eam_store_fp(d, i, h, l);
}

// (F'(rho_i) + F'(rho_j)) f'(r)/r of the embedding term, f'(r) = x (2 + 3 (beta/d) x).
__device__ __forceinline__ df eam_coeff(const SlDev& d, df r2, df rinv, df fpij) {
  const df x = df_sub(df_mul(r2, rinv), F2(d.em_d_f));
  const df fpr = df_mul(x, df_add_f(df_mul(df_mul_f(F2(d.em_bd_f), 3.0f), x), 2.0f));
  return df_mul(fpij, df_mul(fpr, rinv));
}

// Forces at the current state, Eq. p_advance written as -dH/dr_i:
//   F_i = sum_j [V'(r) - J'(r) (s_i.s_j)] (r_j - r_i)/r
// with V'(r)/r = 2 a D0 e (1 - e)/r, e = exp(-a (r - r0)) (Morse, r < morse_rc)
// and J'(r)/r = 8 alpha/delta^2 e^{-x} (1 - 2 gamma x - x + gamma x^2),
// x = r^2/delta^2 (Eq. BSfunction, r < ex_rc), read from the exchange table
// that k_jtable filled at the same positions.  Loops over the Morse list;
// stored in FP64, then optionally v += (dt/2) F / m (the closing half-kick).
__device__ __forceinline__ df morse_coeff(df r2, df na, df r0, df c2, df& rinv) {
  rinv = df_rsqrt(r2);
  const df r = df_mul(r2, rinv);
  const df e = df_exp(df_mul(na, df_add_sloppy(r, df_neg(r0))));   // r carries an error of 2^-48 r already
  return df_mul(df_mul(c2, rinv), df_mul(e, df_add_f(df_neg(e), 1.0f)));   // V'(r)/r
}

// phi'(r)/r + (F'(rho_i) + F'(rho_j)) rho'(r)/r of the tabulated form.
__device__ __forceinline__ df tab_coeff(const SlDev& d, df r2, df fpij) {
  const df rinv = df_rsqrt(r2);
  const df r = df_mul(r2, rinv);
  const df c = df_add(tab_slope_df(d, SL_TAB_PHI, r), df_mul(fpij, tab_slope_df(d, SL_TAB_RHO, r)));
  return df_mul(c, rinv);
}

// MECH: also the embedding term (closed or tabulated form) and the
// ground-state subtraction.
// The plain instance is held to 64 registers (8 blocks of 128 per SM): with
// its neighbour pipeline it would take 77 and run 5 % slower at 6 blocks.
template <bool SO, bool MECH>
__global__ void __launch_bounds__(256, SO || MECH ? 2 : 4) k_force(SlDev d, int kick) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  if (d.ham == SL_HAM_LEARNED && d.ctrl->ml_use) return;   // the network is in effect here
  const p3 pi = load_pos(d, i);
  const box3 B = load_box(d, d.reps[__ldg(d.arep + i)]);
  const df3 si = load_spin(d, i);
  float fxh = 0.0f, fxl = 0.0f, fyh = 0.0f, fyl = 0.0f, fzh = 0.0f, fzl = 0.0f;
  const int nm = d.mn[i], ne = d.exn[i];
  const df na = F2(d.m_nalpha_f), r0 = F2(d.m_r0_f), c2 = F2(d.m_c2_f), rc2 = F2(d.m_rc2_f);
  const df xrc2 = F2(d.ex_rc2_f);
  const float rc2_hi = rc2.hi * 1.0001f;
  const bool eam = MECH && (d.mech & SL_MECH_EAM);
  const bool tab = MECH && (d.mech & SL_MECH_TAB);   // tabulated pair term and embedding replace Morse + FS
  const df ed2 = F2(d.em_d2_f);
  const df fpi = eam ? F2(__ldg(d.em_fp + i)) : df_f(0.0f);
  // neighbour ids two entries ahead and positions one ahead in each of the
  // three loops, so that the gathers overlap the arithmetic of the entry before
  const int mc = d.mnc[i];
  const size_t n = (size_t)d.n;
  const int* MJ = d.mj + i;
  int j1 = nm > 0 ? __ldg(MJ) : i, j2 = nm > 1 ? __ldg(MJ + n) : i;
  p3 p1 = load_pos(d, j1);
  auto advance = [&](int k, int kend) {
    j1 = j2;
    if (k + 2 < nm) j2 = __ldg(MJ + (size_t)(k + 2) * n);
    if (k + 1 < kend) p1 = load_pos(d, j1);
  };
  // entries 0..ne-1: exchange neighbours (also inside the Morse cutoff)
  for (int k = 0; k < ne; ++k) {
    const int j = j1;
    const p3 pj = p1;
    advance(k, nm);
    const df3 dd = pair_sep(B, pi, pj);
    const df r2 = sep_r2(dd);
    df rinv;
    df c = df_f(0.0f);
    if (tab) {
      if (df_lt(r2, rc2)) c = tab_coeff(d, r2, df_add(fpi, F2(__ldg(d.em_fp + j))));
    } else {
      c = df_lt(r2, rc2) ? morse_coeff(r2, na, r0, c2, rinv) : df_f(0.0f);
      if (eam && df_lt(r2, ed2)) c = df_add(c, eam_coeff(d, r2, rinv, df_add(fpi, F2(__ldg(d.em_fp + j)))));
    }
    if (df_lt(r2, xrc2)) {
      // J'(r)/r from the exchange table (same positions, same entry order)
      const df dJr = F2(__ldg(d.exdJ + (size_t)k * d.n + i));
      const df3 sj = load_spin(d, j);
      const df sij = dot3(si, sj);
      c = df_sub(c, df_mul(dJr, sij));
      if (MECH && (d.mech & SL_MECH_GROUND)) c = df_add(c, dJr);   // + J(r): -dJr (s_i.s_j - 1)
      if (SO && (d.so & (SL_SO_NEEL | SL_SO_DMI))) {
        // Neel, U = -g1 Q, Q = (e.s_i)(e.s_j) - s_i.s_j/3 (A = e.s_j, B = e.s_i):
        //   F_i = -g1' Q e - (g1/r) (A s_i + B s_j - 2 A B e);
        // DMI, W = d e.X, X = s_i x s_j: F_i = d' (e.X) e + (d/r) (X - e (e.X)).
        // With e = dd/r, the terms along e collect on dd (f' e = (f'/r) dd).
        const df ri = df_rsqrt(r2);
        df3 u;
        u.x = df_mul(dd.x, ri); u.y = df_mul(dd.y, ri); u.z = df_mul(dd.z, ri);
        df ci = df_f(0.0f), cj = df_f(0.0f), dr = df_f(0.0f);
        df3 X;
        X.x = X.y = X.z = df_f(0.0f);
        if (d.so & SL_SO_NEEL) {
          df g1, g1pr;
          bs_eval(d.ne_bs, r2, g1, g1pr);
          const df A = dot3(u, sj), Bv = dot3(u, si);
          const df AB = df_mul(A, Bv);
          const df Q = df_sub(AB, df_mul(sij, df_make(SL_INV_ODD3_HI, SL_INV_ODD3_LO)));
          const df gr = df_mul(g1, ri);
          c = df_sub(c, df_mul(g1pr, Q));
          c = df_add(c, df_mul(df_scale(df_mul(gr, ri), 2.0f), AB));
          ci = df_neg(df_mul(gr, A));
          cj = df_neg(df_mul(gr, Bv));
        }
        if (d.so & SL_SO_DMI) {
          df dm, dmpr;
          bs_eval(d.dm_bs, r2, dm, dmpr);
          X = cross3(si, sj);
          const df eX = dot3(u, X);
          dr = df_mul(dm, ri);
          c = df_add(c, df_mul(eX, df_sub(dmpr, df_mul(dr, ri))));
        }
        acc_prod(fxh, fxl, ci, si.x); acc_prod(fxh, fxl, cj, sj.x); acc_prod(fxh, fxl, dr, X.x);
        acc_prod(fyh, fyl, ci, si.y); acc_prod(fyh, fyl, cj, sj.y); acc_prod(fyh, fyl, dr, X.y);
        acc_prod(fzh, fzl, ci, si.z); acc_prod(fzh, fzl, cj, sj.z); acc_prod(fzh, fzl, dr, X.z);
      }
    }
    acc_prod(fxh, fxl, c, dd.x);
    acc_prod(fyh, fyl, c, dd.y);
    acc_prod(fzh, fzl, c, dd.z);
  }
  // entries ne..mc-1: Morse only, inside the cutoff until the next rebuild
  for (int k = ne; k < mc; ++k) {
    const int j = j1;
    const p3 pj = p1;
    advance(k, nm);
    const df3 dd = pair_sep(B, pi, pj);
    const df r2 = sep_r2(dd);
    df rinv;
    df c;
    if (tab) {
      c = tab_coeff(d, r2, df_add(fpi, F2(__ldg(d.em_fp + j))));
    } else {
      c = morse_coeff(r2, na, r0, c2, rinv);
      if (eam && df_lt(r2, ed2)) c = df_add(c, eam_coeff(d, r2, rinv, df_add(fpi, F2(__ldg(d.em_fp + j)))));
    }
    acc_prod(fxh, fxl, c, dd.x);
    acc_prod(fyh, fyl, c, dd.y);
    acc_prod(fzh, fzl, c, dd.z);
  }
  // entries mc..nm-1: Morse only, possibly outside the cutoff
  for (int k = mc; k < nm; ++k) {
    const int j = j1;
    const p3 pj = p1;
    advance(k, nm);
    // float pre-check: pairs clearly outside the cutoff skip the exact separation
    const pre3 q = pair_pre(B, pi, pj);
    if (q.r2 > rc2_hi) continue;
    const df3 dd = pair_sep_k(B, pi, pj, q);
    const df r2 = sep_r2(dd);
    if (!df_lt(r2, rc2)) continue;
    df rinv;
    df c;
    if (tab) {
      c = tab_coeff(d, r2, df_add(fpi, F2(__ldg(d.em_fp + j))));
    } else {
      c = morse_coeff(r2, na, r0, c2, rinv);
      if (eam && df_lt(r2, ed2)) c = df_add(c, eam_coeff(d, r2, rinv, df_add(fpi, F2(__ldg(d.em_fp + j)))));
    }
    acc_prod(fxh, fxl, c, dd.x);
    acc_prod(fyh, fyl, c, dd.y);
    acc_prod(fzh, fzl, c, dd.z);
  }
  const double fx = df_to_double(acc_done(fxh, fxl));
  const double fy = df_to_double(acc_done(fyh, fyl));
  const double fz = df_to_double(acc_done(fzh, fzl));
  d.F[i] = make_double4_32a(fx, fy, fz, 0.0);
  if (kick) {
    double c = 0.5 * d.dt * d.acc;
    double4_32a v = d.v[i];
    v.x = fma(c, fx, v.x); v.y = fma(c, fy, v.y); v.z = fma(c, fz, v.z);
    if (d.any_lattice_bath) v = lattice_bath(d, i, v, 5);
    d.v[i] = v;
  }
}

__global__ void k_end_step(SlDev d) { d.ctrl->step += 1; }

void launch_jtable(const SlDev& d, int grid, int block, cudaStream_t st, bool dens) {
  if (d.so && dens) k_jtable<true, true><<<grid, block, 0, st>>>(d);
  else if (d.so) k_jtable<true, false><<<grid, block, 0, st>>>(d);
  else if (dens) k_jtable<false, true><<<grid, block, 0, st>>>(d);
  else k_jtable<false, false><<<grid, block, 0, st>>>(d);
}

void launch_force(const SlDev& d, int grid, int block, cudaStream_t st, int kick) {
  if (d.so && d.mech) k_force<true, true><<<grid, block, 0, st>>>(d, kick);
  else if (d.so) k_force<true, false><<<grid, block, 0, st>>>(d, kick);
  else if (d.mech) k_force<false, true><<<grid, block, 0, st>>>(d, kick);
  else k_force<false, false><<<grid, block, 0, st>>>(d, kick);
}

// The per-step tables at the current positions: J (and the spin-orbit
// tables), then the embedding density.  Returns the kernels launched.
int launch_tables(const SlDev& d, int grid, int block, cudaStream_t st) {
  const bool eam = (d.mech & SL_MECH_EAM) != 0;
  launch_jtable(d, grid, block, st, eam && d.em_fused);
  if (eam && !d.em_fused) {
    k_density<<<grid, block, 0, st>>>(d);
    return 2;
  }
  return 1;
}

// The passes of a spin half-op: colours 0..6 forward, colour 7 forward then
// backward in one fused pass (nothing of another colour turns between the
// two), colours 6..0 backward.  Pass p reads the partial field written by
// pass p - 1 (none for p = 0) and precomputes the next pass's.
constexpr int SL_SWEEP_PASSES = 15;
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

template <bool SO>
void launch_half_op_so(const SlDev& d, cudaStream_t st, int subpass0) {
  switch (d.tune_sweep % 5) {
    case 1: launch_half_op_t<32, 256, SO>(d, st, subpass0); break;
    case 2: launch_half_op_t<16, 128, SO>(d, st, subpass0); break;
    case 3: launch_half_op_t<16, 128, SO, 1024>(d, st, subpass0); break;
    case 4: launch_half_op_t<8, 128, SO>(d, st, subpass0); break;
    default: launch_half_op_t<32, 192, SO>(d, st, subpass0); break;
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

// Tile shapes: variants 0-4 are the pipelined pass k_sweep_pass (sectors per
// block 32, 32, 16, 16, 8 x 192, 256, 128, 128, 128 threads; variant 3 with
// registers for 1,024 threads per SM, the others 768), for every
// Hamiltonian; variants 5-9 the asynchronous-gather pass k_sweep_async of the
// plain Hamiltonian (16, 8, 32, 8, 4 sectors x 128, 64, 256, 96, 64 threads,
// up to 128, 64, 256, 96, 48 atoms per block in shared memory); with the
// spin-orbit terms variants 5-9 run as 0-4.
void launch_half_op(const SlDev& d, cudaStream_t st, int subpass0) {
  if (d.so) {
    launch_half_op_so<true>(d, st, subpass0);
    return;
  }
  switch (d.tune_sweep) {
    case 5: launch_half_op_async_t<16, 128, 128>(d, st, subpass0); break;
    case 6: launch_half_op_async_t<8, 64, 64>(d, st, subpass0); break;
    case 7: launch_half_op_async_t<32, 256, 256>(d, st, subpass0); break;
    case 8: launch_half_op_async_t<8, 96, 96>(d, st, subpass0); break;
    case 9: launch_half_op_async_t<4, 64, 48>(d, st, subpass0); break;
    default: launch_half_op_so<false>(d, st, subpass0); break;
  }
}

// threads per block of the per-atom kernels (autotuned)
inline int tb(const SlDev& d) { return d.tune_block > 0 ? d.tune_block : SL_BLOCK; }
inline int grid_tb(const SlDev& d) { return (d.n + tb(d) - 1) / tb(d); }

// omega of every atom in caller order (device out [n][3]), FP64.
__global__ void k_omega_all(SlDev d, double* out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.n) return;
  double hx = d.zee[0], hy = d.zee[1], hz = d.zee[2];
  if (d.ham == SL_HAM_LEARNED && d.ctrl->ml_use) {
    // -(1/hbar) dH/ds of the network (exact gradient at the current state)
    const float4 b = d.ml_B[k];
    const double ih = 1.0 / SL_HBAR;
    size_t id = (size_t)d.perm[k];
    out[3 * id] = (hx + b.x) * ih; out[3 * id + 1] = (hy + b.y) * ih; out[3 * id + 2] = (hz + b.z) * ih;
    return;
  }
  for (int q = 0; q < d.exn[k]; ++q) {
    const size_t e = (size_t)q * d.n + k;
    float2 J2 = d.exJ[e];
    double J = double_from_float(J2.x) + double_from_float(J2.y);
    double4_32a sj = d.s[d.exj[e]];
    hx = fma(J, sj.x, hx); hy = fma(J, sj.y, hy); hz = fma(J, sj.z, hz);
    if (d.exso) so_field_d(d, e, sj, hx, hy, hz);
  }
  if (d.so & SL_SO_ANISO) {
    const double4_32a si = d.s[k];
    const double c = 2.0 * d.an_K * (si.x * d.an_n[0] + si.y * d.an_n[1] + si.z * d.an_n[2]);
    hx += c * d.an_n[0]; hy += c * d.an_n[1]; hz += c * d.an_n[2];
  }
  const double ih = 1.0 / SL_HBAR;
  size_t id = (size_t)d.perm[k];
  out[3 * id] = hx * ih; out[3 * id + 1] = hy * ih; out[3 * id + 2] = hz * ih;
}

// Split copies of r and s for every atom (after init, set_state, or a
// rebuild when `only_if_rebuild` is set).
__global__ void k_split_all(SlDev d, int only_if_rebuild) {
  if (only_if_rebuild && !d.ctrl->need_rebuild) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < d.n; k += gridDim.x * blockDim.x) {
    store_pos_split(d, k, d.r[k]);
    store_spin_split(d, k, d.s[k]);
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

template <int SPB, int THREADS, int MAXA>
bool prepare_async() {
  return cudaFuncSetAttribute(k_sweep_async<SPB, THREADS, MAXA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sweep_async_smem(true, MAXA)) == cudaSuccess;
}

int sl_prepare_kernels() {
  const bool ok = prepare_sweep<false>() && prepare_sweep<true>() && prepare_async<16, 128, 128>() &&
                  prepare_async<8, 64, 64>() && prepare_async<32, 256, 256>() && prepare_async<8, 96, 96>() &&
                  prepare_async<4, 64, 48>();
  return ok ? SL_OK : SL_ERR_CUDA;
}

int sl_launch_split(const SlDev& d, cudaStream_t st, int only_if_rebuild) {
  const int g = only_if_rebuild && d.rb_cap > 0 ? std::min(grid_for(d.n), d.rb_cap) : grid_for(d.n);
  k_split_all<<<g, SL_BLOCK, 0, st>>>(d, only_if_rebuild);
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}

// Exchange table and forces at the current state (after init/rebuild/set_state).
int sl_launch_pairs_and_forces(const SlDev& d, cudaStream_t st, int kick) {
  launch_tables(d, grid_tb(d), tb(d), st);
  launch_force(d, grid_tb(d), tb(d), st, kick);
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}

// One step with the learned Hamiltonian: the network is evaluated after the
// first half-op (and drift) and after the second; each evaluation point
// either uses the network or, if the gate closed, the analytic kernels.
static int launch_step_learned(const SlDev& d, cudaStream_t st, SlPhaseMark mark, void* user, int* kernels) {
  int gn = grid_for(d.n);
  const int lat = !d.fix_lattice;
  int nk = 0;
  auto phase = [&](int ph, int end) { if (mark) mark(user, ph, end, st); };
  if (lat) {
    phase(SL_PHASE_KICK, 0);
    k_kick<<<gn, SL_BLOCK, 0, st>>>(d, 0.5 * d.dt);
    phase(SL_PHASE_KICK, 1);
    nk += 1;
  }
  phase(SL_PHASE_SPIN1, 0);
  int e = sl_ml_launch_half_op(d, st);
  phase(SL_PHASE_SPIN1, 1);
  nk += 16;
  if (lat) {
    phase(SL_PHASE_DRIFT, 0);
    k_drift<<<gn, SL_BLOCK, 0, st>>>(d);
    k_decide<<<1, 1, 0, st>>>(d);
    if (!e) e = sl_launch_rebuild(d, st);
    phase(SL_PHASE_DRIFT, 1);
    nk += 2 + SL_REBUILD_KERNELS;
  }
  phase(SL_PHASE_JTABLE, 0);
  if (!e) e = sl_ml_launch_point(d, st, 0);
  k_jtable<false, false><<<gn, SL_BLOCK, 0, st>>>(d);
  phase(SL_PHASE_JTABLE, 1);
  nk += 5;
  phase(SL_PHASE_SPIN2, 0);
  if (!e) e = sl_ml_launch_half_op(d, st);
  phase(SL_PHASE_SPIN2, 1);
  nk += 16;
  phase(SL_PHASE_FORCE, 0);
  if (!e) e = sl_ml_launch_point(d, st, lat ? 3 : 0);
  k_jtable<false, false><<<gn, SL_BLOCK, 0, st>>>(d);
  nk += 5;
  if (lat) {
    k_force<false, false><<<gn, SL_BLOCK, 0, st>>>(d, 1);
    nk += 1;
  }
  phase(SL_PHASE_FORCE, 1);
  k_end_step<<<1, 1, 0, st>>>(d);
  nk += 1;
  if (kernels) *kernels = nk;
  if (e) return e;
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}

int sl_launch_step(const SlDev& d, cudaStream_t st, SlPhaseMark mark, void* user, int* kernels) {
  if (d.ham == SL_HAM_LEARNED) return launch_step_learned(d, st, mark, user, kernels);
  const int lat = !d.fix_lattice;
  int nk = 0;
  auto phase = [&](int ph, int end) { if (mark) mark(user, ph, end, st); };
  if (lat) {
    phase(SL_PHASE_KICK, 0);
    k_kick<<<grid_tb(d), tb(d), 0, st>>>(d, 0.5 * d.dt);
    phase(SL_PHASE_KICK, 1);
    nk += 1;
  }
  phase(SL_PHASE_SPIN1, 0);
  launch_half_op(d, st, 0);
  phase(SL_PHASE_SPIN1, 1);
  nk += SL_SWEEP_PASSES;
  if (lat) {
    phase(SL_PHASE_DRIFT, 0);
    k_drift<<<grid_tb(d), tb(d), 0, st>>>(d);
    k_decide<<<1, 1, 0, st>>>(d);
    int e = sl_launch_rebuild(d, st);
    if (e) return e;
    phase(SL_PHASE_DRIFT, 1);
    phase(SL_PHASE_JTABLE, 0);
    const int ntab = launch_tables(d, grid_tb(d), tb(d), st);
    phase(SL_PHASE_JTABLE, 1);
    nk += 2 + SL_REBUILD_KERNELS + ntab;
  }
  phase(SL_PHASE_SPIN2, 0);
  launch_half_op(d, st, 2);
  phase(SL_PHASE_SPIN2, 1);
  nk += SL_SWEEP_PASSES;
  if (lat) {
    phase(SL_PHASE_FORCE, 0);
    launch_force(d, grid_tb(d), tb(d), st, 1);
    phase(SL_PHASE_FORCE, 1);
    nk += 1;
  }
  k_end_step<<<1, 1, 0, st>>>(d);
  nk += 1;
  if (kernels) *kernels = nk;
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}

int sl_launch_omega_all(const SlDev& d, double* out, cudaStream_t st) {
  k_omega_all<<<grid_for(d.n), SL_BLOCK, 0, st>>>(d, out);
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}
