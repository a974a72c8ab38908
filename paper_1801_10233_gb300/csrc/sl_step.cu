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

}  // namespace

int sl_prepare_kernels() {
  return sl_prepare_sweep_plain() == SL_OK && sl_prepare_sweep_so() == SL_OK ? SL_OK : SL_ERR_CUDA;
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
  sl_launch_half_op(d, st, 0);
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
  sl_launch_half_op(d, st, 2);
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
