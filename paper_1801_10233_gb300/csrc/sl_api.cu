// C ABI of libsl: context lifecycle, workspace layout, state transfer and
// the per-step launch sequence (captured once into a CUDA graph).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "sl_internal.cuh"
#include "sl_df64.cuh"
#include "sl_pair.cuh"

struct sl_ctx {
  sl_params p;              // fields shared by every replica (replica 0's copy)
  int nrep;
  std::vector<SlRep> reps;  // host copy of the replica table
  SlDev d;
  cudaStream_t stream;
  cudaStream_t cap;         // private stream for graph capture
  cudaGraphExec_t graph;
  int graph_ok;
  int device;
  int sticky;
  int kernels_per_step;
  // optional per-phase event timing
  int timing;
  std::vector<cudaEvent_t> ev_pool;      // events owned by the context
  std::vector<int> ev_phase;             // phase of each recorded (begin, end) pair
  size_t ev_used;
  double phase_ms[SL_NPHASE];
  long long phase_n[SL_NPHASE];
  // learned Hamiltonian
  void* ws_base;            // the caller's workspace (all device state of the context)
  size_t ws_bytes;
  std::vector<double> lat_gamma, lat_temp;   // per-replica lattice bath (for sl_set_dt)
  int ml_ready;             // a model has been set
  int eam_ready;            // the tables of the tabulated embedded-atom form have been set
  int ml_stale;             // parameters changed since the last evaluation point
  long long ml_t;           // Adam steps taken
};

namespace {

inline int grid_for(int n) { return (n + SL_BLOCK - 1) / SL_BLOCK; }

struct DeviceGuard {
  int old = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&old) == cudaSuccess && old != dev) cudaSetDevice(dev);
    else old = -1;
  }
  ~DeviceGuard() { if (old >= 0) cudaSetDevice(old); }
};

// Sector grid of Sec. 5.1: the largest even count per edge with sector edge
// >= (exchange cutoff + skin)(1 + SL_SECTOR_MARGIN) (the network's cutoff +
// skin for the learned Hamiltonian, whose spins interact up to that
// distance).  The margin keeps two atoms of same-colour sectors more than
// the list radius apart by more than a float distance test can misjudge.
int sector_grid(const sl_params* p, int n[3], double e[3]) {
  double reach = p->ex_rc_A;
  if (p->hamiltonian == SL_HAM_LEARNED && SL_ML_RC > reach) reach = SL_ML_RC;
  double w = (reach + p->skin_A) * (1.0 + SL_SECTOR_MARGIN);
  for (int a = 0; a < 3; ++a) {
    int k = (int)std::floor(p->box[a] / w);
    if (k % 2) k -= 1;
    if (k < 2) return SL_ERR_BOX;
    n[a] = k;
    e[a] = p->box[a] / (double)k;
  }
  return SL_OK;
}

int validate(const sl_params* p) {
  if (!p) return SL_ERR_ARG;
  if (p->n_atoms < 1 || !(p->mass_amu > 0.0) || !(p->skin_A >= 0.0)) return SL_ERR_ARG;
  if (!(p->ex_rc_A > 0.0) || !(p->morse_rc_A > 0.0) || !(p->ex_delta_A > 0.0)) return SL_ERR_ARG;
  if (!(p->morse_rc_A >= p->ex_rc_A)) return SL_ERR_ARG;   // Morse list holds the exchange list
  if (p->rotation != SL_ROT_RODRIGUES && p->rotation != SL_ROT_CAYLEY) return SL_ERR_ARG;
  if (p->rebuild_every < 0 || p->max_ex_neighbors < 0 || p->max_morse_neighbors < 0) return SL_ERR_ARG;
  if (p->max_ex_neighbors > SL_MAX_EX_CAP) return SL_ERR_ARG;
  if (!(p->lambda >= 0.0) || !(p->temperature_K >= 0.0)) return SL_ERR_ARG;
  if (!(p->lattice_gamma_ps >= 0.0) || !(p->lattice_temperature_K >= 0.0)) return SL_ERR_ARG;
  if (!std::isfinite(p->dt_ps)) return SL_ERR_ARG;
  if (p->hamiltonian != SL_HAM_ANALYTIC && p->hamiltonian != SL_HAM_LEARNED) return SL_ERR_ARG;
  if (p->hamiltonian == SL_HAM_LEARNED && (!(p->morse_rc_A >= SL_ML_RC) || p->lambda != 0.0 ||
                                           p->temperature_K != 0.0 || p->rotation != SL_ROT_RODRIGUES))
    return SL_ERR_ARG;
  // spin-orbit terms: finite, a unit anisotropy axis, positive ranges; analytic Hamiltonian only
  const bool so = p->aniso_K_eV != 0.0 || p->neel_alpha_eV != 0.0 || p->dmi_alpha_eV != 0.0;
  if (!std::isfinite(p->aniso_K_eV) || !std::isfinite(p->neel_alpha_eV) || !std::isfinite(p->dmi_alpha_eV) ||
      !std::isfinite(p->neel_gamma) || !std::isfinite(p->dmi_gamma))
    return SL_ERR_ARG;
  if (so && p->hamiltonian != SL_HAM_ANALYTIC) return SL_ERR_ARG;
  if (p->aniso_K_eV != 0.0) {
    const double* a = p->aniso_axis;
    if (!(std::fabs(a[0] * a[0] + a[1] * a[1] + a[2] * a[2] - 1.0) <= 1e-12)) return SL_ERR_ARG;
  }
  if (p->neel_alpha_eV != 0.0 && !(p->neel_delta_A > 0.0)) return SL_ERR_ARG;
  if (p->dmi_alpha_eV != 0.0 && !(p->dmi_delta_A > 0.0)) return SL_ERR_ARG;
  // every exponential the pair kernels take inside a cutoff stays within the
  // double-float exp's accurate range: e^{-r^2/delta^2} for r < ex_rc
  // (Eq. BSfunction, also the Neel and DMI ranges) and e^{-a (r - r0)} for
  // 0 < r < morse_rc (also the fallback of the learned Hamiltonian)
  auto sq = [](double x) { return x * x; };
  if (!(sq(p->ex_rc_A / p->ex_delta_A) <= SL_DF_EXP_XMAX)) return SL_ERR_ARG;
  if (p->neel_alpha_eV != 0.0 && !(sq(p->ex_rc_A / p->neel_delta_A) <= SL_DF_EXP_XMAX)) return SL_ERR_ARG;
  if (p->dmi_alpha_eV != 0.0 && !(sq(p->ex_rc_A / p->dmi_delta_A) <= SL_DF_EXP_XMAX)) return SL_ERR_ARG;
  if (!(std::fabs(p->morse_alpha_invA) * std::fmax(std::fabs(p->morse_rc_A - p->morse_r0_A),
                                                   std::fabs(p->morse_r0_A)) <= SL_DF_EXP_XMAX))
    return SL_ERR_ARG;
  // embedding term and ground-state subtraction: analytic Hamiltonian only
  if (!std::isfinite(p->eam_A_eV) || !std::isfinite(p->eam_beta)) return SL_ERR_ARG;
  if (p->subtract_ground_exchange != 0 && p->subtract_ground_exchange != 1) return SL_ERR_ARG;
  if ((p->eam_A_eV != 0.0 || p->subtract_ground_exchange) && p->hamiltonian != SL_HAM_ANALYTIC) return SL_ERR_ARG;
  if (p->eam_A_eV != 0.0 && !(p->eam_d_A > 0.0 && p->eam_d_A <= p->morse_rc_A)) return SL_ERR_ARG;
  if (p->eam_tabulated != 0 && p->eam_tabulated != 1) return SL_ERR_ARG;
  if (p->eam_tabulated && (p->hamiltonian != SL_HAM_ANALYTIC || p->eam_A_eV != 0.0)) return SL_ERR_ARG;
  double rc = (p->morse_rc_A > p->ex_rc_A ? p->morse_rc_A : p->ex_rc_A) + p->skin_A;
  for (int a = 0; a < 3; ++a)
    if (!(p->box[a] >= 2.0 * rc) || !(p->box[a] < SL_FX_MAX_BOX)) return SL_ERR_BOX;
  int n[3]; double e[3];
  return sector_grid(p, n, e);
}

// Replicas of a batch may differ in n_atoms, box, temperature_K and replica;
// every other field must match replica 0.
int validate_batch(const sl_params* p, int nrep) {
  if (!p || nrep < 1) return SL_ERR_ARG;
  long long total = 0;
  for (int r = 0; r < nrep; ++r) {
    int e = validate(p + r);
    if (e) return e;
    total += p[r].n_atoms;
    const sl_params& a = p[0];
    const sl_params& b = p[r];
    bool same = a.rotation == b.rotation && a.fix_lattice == b.fix_lattice && a.rebuild_every == b.rebuild_every &&
                a.morse_shift_energy == b.morse_shift_energy && a.max_ex_neighbors == b.max_ex_neighbors &&
                a.max_morse_neighbors == b.max_morse_neighbors && a.mass_amu == b.mass_amu &&
                a.mu_s_muB == b.mu_s_muB && a.dt_ps == b.dt_ps && a.ex_alpha_eV == b.ex_alpha_eV &&
                a.ex_gamma == b.ex_gamma && a.ex_delta_A == b.ex_delta_A && a.ex_rc_A == b.ex_rc_A &&
                a.morse_D0_eV == b.morse_D0_eV && a.morse_alpha_invA == b.morse_alpha_invA &&
                a.morse_r0_A == b.morse_r0_A && a.morse_rc_A == b.morse_rc_A && a.skin_A == b.skin_A &&
                a.lambda == b.lambda && a.seed == b.seed && a.hamiltonian == b.hamiltonian &&
                a.aniso_K_eV == b.aniso_K_eV && a.neel_alpha_eV == b.neel_alpha_eV &&
                a.neel_gamma == b.neel_gamma && a.neel_delta_A == b.neel_delta_A &&
                a.dmi_alpha_eV == b.dmi_alpha_eV && a.dmi_gamma == b.dmi_gamma && a.dmi_delta_A == b.dmi_delta_A &&
                a.eam_A_eV == b.eam_A_eV && a.eam_d_A == b.eam_d_A && a.eam_beta == b.eam_beta &&
                a.subtract_ground_exchange == b.subtract_ground_exchange && a.eam_tabulated == b.eam_tabulated;
    for (int c = 0; c < 3; ++c) same = same && a.H_tesla[c] == b.H_tesla[c] && a.aniso_axis[c] == b.aniso_axis[c];
    if (!same) return SL_ERR_ARG;
  }
  if (total > 0x7fffffffLL) return SL_ERR_ARG;
  return SL_OK;
}

struct Layout {
  size_t off = 0;
  template <class T>
  size_t take(size_t count) {
    size_t o = (off + 255) & ~size_t(255);
    off = o + count * sizeof(T);
    return o;
  }
};

// x = hi + lo with hi = float(x), lo = float(x - hi): the double-float form of
// an FP64 scalar (host side).
float2 split_f2(double x) {
  float hi = (float)x;
  float lo = (float)(x - (double)hi);
  return make_float2(hi, lo);
}


// Double-float constants that depend on dt or H.
void fill_df_constants(SlDev& d) {
  for (int a = 0; a < 3; ++a) d.zee_f[a] = split_f2(d.zee[a]);
  d.tau_f = split_f2(0.25 * d.dt);
}

// Noise amplitude of each replica's spin bath for the current dt: each
// single-spin factor over tau = dt/4 draws eta ~ N(0, 2 D_S / |tau|) per
// component, D_S = lambda (1 + lambda^2) k_B T / hbar.
void fill_noise(std::vector<SlRep>& reps, const sl_params* ps, double dt) {
  for (size_t r = 0; r < reps.size(); ++r) {
    SlRep& R = reps[r];
    const double lambda = ps[0].lambda;
    double DS = lambda * (1.0 + lambda * lambda) * SL_KB * R.temperature / SL_HBAR;
    R.noise_sig = R.temperature > 0.0 && dt != 0.0 ? split_f2(std::sqrt(2.0 * DS / std::fabs(0.25 * dt)))
                                                   : make_float2(0.0f, 0.0f);
    // lattice bath (Eq. p_advance_T) over |dt|/2: exact Ornstein-Uhlenbeck flow
    const double g = ps[r].lattice_gamma_ps, T = ps[r].lattice_temperature_K;
    R.lat_c1 = g > 0.0 ? std::exp(-g * 0.5 * std::fabs(dt)) : 1.0;
    R.lat_sig = g > 0.0 && T > 0.0 ? std::sqrt((1.0 - R.lat_c1 * R.lat_c1) * SL_KB * T * SL_FTOA / ps[r].mass_amu)
                                   : 0.0;
  }
}

// Fill d's scalars, the replica table and (if base != NULL) d's pointers;
// returns the workspace bytes needed.

size_t plan(const sl_params* ps, int nrep, SlDev& d, std::vector<SlRep>& reps, char* base) {
  std::memset(&d, 0, sizeof(d));
  const sl_params* p = ps;
  reps.assign(nrep, SlRep());
  double reach = (p->morse_rc_A > p->ex_rc_A ? p->morse_rc_A : p->ex_rc_A) + p->skin_A;
  int atom0 = 0, sec8 = 0, noise = 0;
  const int fx = SL_FX_BITS;   // fixed-point positions X = rint(r 2^48)
  for (int r = 0; r < nrep; ++r) {
    SlRep& R = reps[r];
    std::memset(&R, 0, sizeof(R));
    int ns[3]; double e[3];
    sector_grid(ps + r, ns, e);
    R.nx = ns[0]; R.ny = ns[1]; R.nz = ns[2];
    R.s8 = ns[0] * ns[1] * ns[2] / 8;
    int* mm[3] = {&R.mx, &R.my, &R.mz};
    for (int a = 0; a < 3; ++a) {
      R.box[a] = ps[r].box[a];
      R.inv_box[a] = 1.0 / ps[r].box[a];
      R.edge[a] = e[a];
      *mm[a] = (int)std::ceil(reach / e[a]);
      R.boxX[a] = std::llrint(std::ldexp(ps[r].box[a], fx));
      R.halfX[a] = R.boxX[a] / 2;
    }
    R.sec8_off = sec8;
    R.atom0 = atom0;
    R.natoms = ps[r].n_atoms;
    R.replica = ps[r].replica;
    R.temperature = ps[r].temperature_K;
    if (R.temperature > 0.0) noise = 1;
    sec8 += R.s8;
    atom0 += R.natoms;
  }
  const int n = atom0;
  d.n = n;
  d.nrep = nrep;
  d.s8 = sec8;
  d.nsec = 8 * sec8;
  d.any_noise = noise;
  d.max_ex = p->max_ex_neighbors ? p->max_ex_neighbors : 24;
  d.max_m = p->max_morse_neighbors ? p->max_morse_neighbors : 128;
  if (d.max_m <= d.max_ex) d.max_m = d.max_ex + 1;
  d.rotation = p->rotation;
  d.fix_lattice = p->fix_lattice;
  d.rebuild_every = p->rebuild_every;
  d.morse_shift = p->morse_shift_energy;
  d.dt = p->dt_ps;
  for (int a = 0; a < 3; ++a) d.zee[a] = p->mu_s_muB * SL_MUB * p->H_tesla[a];
  d.mass = p->mass_amu;
  d.acc = SL_FTOA / p->mass_amu;
  d.ex_alpha = p->ex_alpha_eV; d.ex_gamma = p->ex_gamma; d.ex_delta = p->ex_delta_A;
  d.ex_rc2 = p->ex_rc_A * p->ex_rc_A;
  d.m_D0 = p->morse_D0_eV; d.m_alpha = p->morse_alpha_invA; d.m_r0 = p->morse_r0_A;
  d.m_rc2 = p->morse_rc_A * p->morse_rc_A;
  {
    double ec = std::exp(-p->morse_alpha_invA * (p->morse_rc_A - p->morse_r0_A));
    d.m_vshift = p->morse_shift_energy ? p->morse_D0_eV * (ec * ec - 2.0 * ec) : 0.0;
  }
  d.list_ex2 = (p->ex_rc_A + p->skin_A) * (p->ex_rc_A + p->skin_A);
  d.list_m2 = (p->morse_rc_A + p->skin_A) * (p->morse_rc_A + p->skin_A);
  d.fx_s40 = std::ldexp(1.0f, 40 - fx);
  d.fx_s20 = std::ldexp(1.0f, 20 - fx);
  d.fx_s0 = std::ldexp(1.0f, -fx);
  d.sure_m2 = p->morse_rc_A > p->skin_A ? (p->morse_rc_A - p->skin_A) * (p->morse_rc_A - p->skin_A) : 0.0;
  d.half_skin2 = 0.25 * p->skin_A * p->skin_A;
  d.lambda = p->lambda;
  d.seed = p->seed;
  d.ham = p->hamiltonian;
  d.inv_hbar_f = split_f2(1.0 / SL_HBAR);
  d.m_nalpha_f = split_f2(-p->morse_alpha_invA);
  d.m_r0_f = split_f2(p->morse_r0_A);
  d.m_c2_f = split_f2(2.0 * p->morse_alpha_invA * p->morse_D0_eV);
  d.m_rc2_f = split_f2(d.m_rc2);
  d.ex_ix_f = split_f2(1.0 / (p->ex_delta_A * p->ex_delta_A));
  d.ex_4a_f = split_f2(4.0 * p->ex_alpha_eV);
  d.ex_g_f = split_f2(p->ex_gamma);
  d.ex_8ad2_f = split_f2(8.0 * p->ex_alpha_eV / (p->ex_delta_A * p->ex_delta_A));
  d.ex_rc2_f = split_f2(d.ex_rc2);
  d.lam_f = split_f2(p->lambda);
  d.inv1pl2_f = split_f2(1.0 / (1.0 + p->lambda * p->lambda));
  // spin-orbit terms
  d.so = (p->aniso_K_eV != 0.0 ? SL_SO_ANISO : 0) | (p->neel_alpha_eV != 0.0 ? SL_SO_NEEL : 0) |
         (p->dmi_alpha_eV != 0.0 ? SL_SO_DMI : 0);
  d.an_K = p->aniso_K_eV;
  for (int a = 0; a < 3; ++a) {
    d.an_n[a] = p->aniso_axis[a];
    d.an_n_f[a] = split_f2(p->aniso_axis[a]);
  }
  d.an_c_f = split_f2(2.0 * p->aniso_K_eV / SL_HBAR);
  d.an_cl_f = split_f2(2.0 * p->aniso_K_eV / SL_HBAR / (1.0 + p->lambda * p->lambda));
  // embedding term and ground-state subtraction
  d.mech = (p->eam_A_eV != 0.0 ? SL_MECH_EAM : 0) | (p->subtract_ground_exchange ? SL_MECH_GROUND : 0) |
           (p->eam_tabulated ? SL_MECH_EAM | SL_MECH_TAB : 0);
  d.em_fused = p->eam_A_eV != 0.0 && p->eam_d_A <= p->ex_rc_A;
  d.em_A = p->eam_A_eV;
  d.em_d = p->eam_A_eV != 0.0 ? p->eam_d_A : 1.0;
  d.em_beta = p->eam_beta;
  d.em_d_f = split_f2(d.em_d);
  d.em_d2_f = split_f2(d.em_d * d.em_d);
  d.em_bd_f = split_f2(p->eam_beta / d.em_d);
  d.em_hA_f = split_f2(0.5 * p->eam_A_eV);
  {
    const double nd = p->neel_alpha_eV != 0.0 ? p->neel_delta_A : 1.0;
    const double dd = p->dmi_alpha_eV != 0.0 ? p->dmi_delta_A : 1.0;
    d.ne_bs = {split_f2(1.0 / (nd * nd)), split_f2(4.0 * p->neel_alpha_eV), split_f2(p->neel_gamma),
               split_f2(8.0 * p->neel_alpha_eV / (nd * nd))};
    d.dm_bs = {split_f2(1.0 / (dd * dd)), split_f2(4.0 * p->dmi_alpha_eV), split_f2(p->dmi_gamma),
               split_f2(8.0 * p->dmi_alpha_eV / (dd * dd))};
  }
  fill_df_constants(d);
  fill_noise(reps, ps, p->dt_ps);
  for (int r = 0; r < nrep; ++r)
    if (ps[r].lattice_gamma_ps > 0.0) d.any_lattice_bath = 1;

  Layout L;
  size_t nn = (size_t)n;
  size_t o_r = L.take<double4_32a>(nn), o_v = L.take<double4_32a>(nn), o_s = L.take<double4_32a>(nn);
  size_t o_F = L.take<double4_32a>(nn), o_rb = L.take<SlFix>(nn);
  size_t o_tr = L.take<double4_32a>(nn), o_tv = L.take<double4_32a>(nn), o_ts = L.take<double4_32a>(nn);
  size_t o_tF = L.take<double4_32a>(nn);
  size_t o_perm = L.take<int>(nn), o_rank = L.take<int>(nn), o_secq = L.take<int>(nn);
  size_t o_tsecq = L.take<int>(nn), o_tperm = L.take<int>(nn), o_src = L.take<int>(nn);
  size_t o_arep = L.take<int>(nn), o_tarep = L.take<int>(nn);
  size_t o_cnt = L.take<int>(d.nsec), o_start = L.take<int>(d.nsec + 1), o_fill = L.take<int>(d.nsec);
  size_t o_exj = L.take<int>(nn * d.max_ex), o_exn = L.take<int>(nn), o_exin = L.take<int>(nn);
  size_t o_exc = L.take<uint2>(nn), o_lvl = L.take<unsigned short>(nn);
  size_t o_exJ = L.take<float2>(nn * d.max_ex), o_exdJ = L.take<float2>(nn * d.max_ex);
  const bool so_pairs = d.so != 0;   // the spin-orbit sweep reads the tables whenever a term is on
  size_t o_exso = so_pairs ? L.take<float2>(5 * nn * d.max_ex) : 0;
  const bool eam = (d.mech & SL_MECH_EAM) != 0;
  size_t o_emfp = eam ? L.take<float2>(nn) : 0;
  // spline coefficients of the tabulated form, room for the largest tables
  const bool tab = (d.mech & SL_MECH_TAB) != 0;
  const size_t tint = (size_t)SL_EAM_MAX_POINTS - 1;
  size_t o_tabd[3] = {0, 0, 0}, o_tabf[3] = {0, 0, 0};
  if (tab)
    for (int t = 0; t < 3; ++t) { o_tabd[t] = L.take<double>(4 * tint); o_tabf[t] = L.take<float4>(2 * tint); }
  size_t o_rx = L.take<SlFix>(nn);
  size_t o_sdf = L.take<float4>(2 * nn);
  size_t o_hb = L.take<float2>(3 * nn), o_sb = L.take<float2>(3 * nn), o_eb = L.take<float2>(3 * nn);
  size_t o_xb = L.take<float2>(3 * nn), o_eb2 = L.take<float2>(3 * nn);
  size_t o_p0 = L.take<float2>(3 * nn), o_p1 = L.take<float2>(3 * nn);
  size_t o_mj = L.take<int>(nn * d.max_m), o_mn = L.take<int>(nn), o_mnc = L.take<int>(nn);
  size_t o_oa = L.take<double>(nn * SL_NOBS), o_or = L.take<double>((size_t)nrep * SL_NOBS);
  size_t o_reps = L.take<SlRep>((size_t)nrep);
  size_t o_stage = L.take<double>(nn * 9);
  size_t o_ctrl = L.take<SlCtrl>(1);
  const bool ml = p->hamiltonian == SL_HAM_LEARNED;
  const size_t ntile = (nn + SL_ML_ATOMS_PER_TILE - 1) / SL_ML_ATOMS_PER_TILE;
  size_t o_mpar = 0, o_mnorm = 0, o_mtiles = 0, o_mfc = 0, o_mx = 0, o_mG = 0, o_me = 0, o_mB = 0, o_mpq = 0;
  size_t o_mu = 0, o_mgF = 0, o_mgB = 0, o_malpha = 0, o_mgpart = 0, o_mgrad = 0, o_mm1 = 0, o_mm2 = 0;
  size_t o_merep = 0, o_mlossat = 0, o_mloss = 0;
  if (ml) {
    o_mpar = L.take<float>(SL_ML_NPARAM); o_mnorm = L.take<float>(SL_ML_NNORM);
    o_mtiles = L.take<uint4>(SL_ML_TILE_BYTES / 16); o_mfc = L.take<float>(SL_MLC_SIZE);
    o_mx = L.take<float>(nn * SL_ML_NF); o_mG = L.take<float>(nn * 64); o_me = L.take<float>(nn);
    o_mB = L.take<float4>(nn); o_mpq = L.take<float2>(nn * d.max_m);
    o_mu = L.take<float>(nn * SL_ML_NF); o_mgF = L.take<float4>(nn); o_mgB = L.take<float4>(nn);
    o_malpha = L.take<double>(nn); o_mgpart = L.take<float>(ntile * SL_ML_NPARAM);
    o_mgrad = L.take<double>(SL_ML_NPARAM); o_mm1 = L.take<double>(SL_ML_NPARAM);
    o_mm2 = L.take<double>(SL_ML_NPARAM); o_merep = L.take<double>((size_t)nrep);
    o_mlossat = L.take<double>(2 * nn); o_mloss = L.take<double>(4);
  }
  if (base && ml) {
    d.ml_par = (float*)(base + o_mpar); d.ml_norm = (float*)(base + o_mnorm);
    d.ml_tiles = (uint4*)(base + o_mtiles); d.ml_fc = (float*)(base + o_mfc);
    d.ml_x = (float*)(base + o_mx); d.ml_G = (float*)(base + o_mG); d.ml_e = (float*)(base + o_me);
    d.ml_B = (float4*)(base + o_mB); d.ml_pq = (float2*)(base + o_mpq);
    d.ml_u = (float*)(base + o_mu); d.ml_gF = (float4*)(base + o_mgF); d.ml_gB = (float4*)(base + o_mgB);
    d.ml_alpha = (double*)(base + o_malpha); d.ml_gpart = (float*)(base + o_mgpart);
    d.ml_grad = (double*)(base + o_mgrad); d.ml_m1 = (double*)(base + o_mm1); d.ml_m2 = (double*)(base + o_mm2);
    d.ml_erep = (double*)(base + o_merep); d.ml_lossat = (double*)(base + o_mlossat);
    d.ml_loss = (double*)(base + o_mloss);
  }
  if (base) {
    d.r = (double4_32a*)(base + o_r); d.v = (double4_32a*)(base + o_v); d.s = (double4_32a*)(base + o_s);
    d.F = (double4_32a*)(base + o_F); d.rbx = (SlFix*)(base + o_rb);
    d.tr = (double4_32a*)(base + o_tr); d.tv = (double4_32a*)(base + o_tv); d.ts = (double4_32a*)(base + o_ts);
    d.tF = (double4_32a*)(base + o_tF);
    d.perm = (int*)(base + o_perm); d.rank = (int*)(base + o_rank); d.secq = (int*)(base + o_secq);
    d.tsecq = (int*)(base + o_tsecq); d.tperm = (int*)(base + o_tperm); d.src = (int*)(base + o_src);
    d.arep = (int*)(base + o_arep); d.tarep = (int*)(base + o_tarep);
    d.sec_count = (int*)(base + o_cnt); d.sec_start = (int*)(base + o_start); d.sec_fill = (int*)(base + o_fill);
    d.exj = (int*)(base + o_exj); d.exn = (int*)(base + o_exn); d.exin = (int*)(base + o_exin);
    d.lvl = (unsigned short*)(base + o_lvl);
    d.exc = (uint2*)(base + o_exc);
    d.exJ = (float2*)(base + o_exJ); d.exdJ = (float2*)(base + o_exdJ);
    d.exso = so_pairs ? (float2*)(base + o_exso) : nullptr;
    d.em_fp = eam ? (float2*)(base + o_emfp) : nullptr;
    for (int t = 0; t < 3; ++t) {
      d.tab_d[t] = tab ? (double*)(base + o_tabd[t]) : nullptr;
      d.tab_f[t] = tab ? (float4*)(base + o_tabf[t]) : nullptr;
      d.tab_n[t] = 0;
    }
    d.rx = (SlFix*)(base + o_rx);
    d.sdf = (float4*)(base + o_sdf);
    d.hbuf = (float2*)(base + o_hb); d.sbuf = (float2*)(base + o_sb); d.ebuf = (float2*)(base + o_eb);
    d.xbuf = (float2*)(base + o_xb); d.ebuf2 = (float2*)(base + o_eb2);
    d.hpart[0] = (float2*)(base + o_p0); d.hpart[1] = (float2*)(base + o_p1);
    d.mj = (int*)(base + o_mj); d.mn = (int*)(base + o_mn); d.mnc = (int*)(base + o_mnc);
    d.obs_atom = (double*)(base + o_oa); d.obs_rep = (double*)(base + o_or);
    d.reps = (const SlRep*)(base + o_reps);
    d.stage = (double*)(base + o_stage);
    d.ctrl = (SlCtrl*)(base + o_ctrl);
  }
  return L.off;
}

__global__ void k_load(SlDev d, const double* r, const double* v, const double* s, int identity) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.n) return;
  if (identity) {
    d.perm[k] = k;
    d.rank[k] = k;
    int lo = 0, hi = d.nrep - 1;   // replica whose caller range holds k
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (d.reps[mid].atom0 <= k) lo = mid; else hi = mid - 1;
    }
    d.arep[k] = lo;
  }
  size_t id = (size_t)d.perm[k];
  if (r) d.r[k] = make_double4_32a(r[3 * id], r[3 * id + 1], r[3 * id + 2], 0.0);
  if (v) d.v[k] = make_double4_32a(v[3 * id], v[3 * id + 1], v[3 * id + 2], 0.0);
  if (s) d.s[k] = make_double4_32a(s[3 * id], s[3 * id + 1], s[3 * id + 2], 0.0);
}

__global__ void k_store(SlDev d, const double4_32a* src, double* out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.n) return;
  size_t id = (size_t)d.perm[k];
  double4_32a x = src[k];
  out[3 * id] = x.x; out[3 * id + 1] = x.y; out[3 * id + 2] = x.z;
}

// Unit spins (|1 - |s|| <= 1e-12) and finite state.
__global__ void k_check(SlDev d) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.n) return;
  double4_32a s = d.s[k], r = d.r[k], v = d.v[k];
  double t = r.x + r.y + r.z + v.x + v.y + v.z + s.x + s.y + s.z;
  if (!(t - t == 0.0)) { sl_set_error(d.ctrl, SL_ERR_NONFINITE); return; }
  double nn = sqrt(s.x * s.x + s.y * s.y + s.z * s.z);
  if (!(fabs(nn - 1.0) <= 1e-12)) sl_set_error(d.ctrl, SL_ERR_SPIN_NORM);
}

// Flag a rebuild if any atom is more than skin/2 from its build position.
__global__ void k_disp_flag(SlDev d) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.n) return;
  const float m = fx_dist2(fx_pos(d.r[k]), d.rbx[k]);
  if ((double)m > d.half_skin2) d.ctrl->need_rebuild = 1;
}

int cuda_err(sl_ctx* c) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { if (!c->sticky) c->sticky = SL_ERR_CUDA; return SL_ERR_CUDA; }
  return SL_OK;
}

// Synchronise and fold the device status into the sticky host error.
int sync_status(sl_ctx* c) {
  int st = 0;
  if (cudaMemcpyAsync(&st, &c->d.ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    if (!c->sticky) c->sticky = SL_ERR_CUDA;
    return c->sticky;
  }
  if (st && !c->sticky) c->sticky = st;
  return c->sticky;
}

void drop_graph(sl_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  c->graph_ok = 0;
}

// Capture one step's launch sequence into a graph on a private stream.
int build_graph(sl_ctx* c) {
  drop_graph(c);
  if (!c->cap && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) return SL_ERR_CUDA;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SL_ERR_CUDA;
  int e = sl_launch_step(c->d, c->cap, nullptr, nullptr, &c->kernels_per_step);
  cudaError_t ce = cudaStreamEndCapture(c->cap, &g);
  if (e || ce != cudaSuccess || !g) { if (g) cudaGraphDestroy(g); cudaGetLastError(); return SL_ERR_CUDA; }
  cudaError_t ie = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) { c->graph = nullptr; cudaGetLastError(); return SL_ERR_CUDA; }
  c->graph_ok = 1;
  return SL_OK;
}

// Record a timing event at a phase boundary on the phase's stream (the pool
// grows as needed).
void mark_phase(void* user, int phase, int end, cudaStream_t st) {
  sl_ctx* c = (sl_ctx*)user;
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) return;
    c->ev_pool.push_back(ev);
  }
  cudaEventRecord(c->ev_pool[c->ev_used], st);
  if (!end) c->ev_phase.push_back(phase);
  c->ev_used += 1;
}

// Fold recorded event pairs into the per-phase totals (synchronises).
int fold_timing(sl_ctx* c) {
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SL_ERR_CUDA;
  for (size_t k = 0; k + 1 < c->ev_used && k / 2 < c->ev_phase.size(); k += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev_pool[k], c->ev_pool[k + 1]) == cudaSuccess) {
      int ph = c->ev_phase[k / 2];
      c->phase_ms[ph] += ms;
      c->phase_n[ph] += 1;
    }
  }
  c->ev_used = 0;
  c->ev_phase.clear();
  return SL_OK;
}

// Exchange table + forces at the current state; rebuild first if flagged.
// With the learned Hamiltonian (once a model is set) this is an evaluation
// point: the analytic kernels only run where the gate closes.
int refresh(sl_ctx* c) {
  int e = sl_launch_rebuild(c->d, c->stream);
  if (!e && c->d.ham == SL_HAM_LEARNED && c->ml_ready) e = sl_ml_launch_point(c->d, c->stream, 1);
  if (!e) e = sl_launch_pairs_and_forces(c->d, c->stream, 0);
  if (!e) c->ml_stale = 0;
  return e ? e : cuda_err(c);
}

// Re-evaluate after the parameters changed (training) before state-dependent use.
int ml_fresh(sl_ctx* c) {
  if (c->d.ham != SL_HAM_LEARNED || !c->ml_stale) return SL_OK;
  return refresh(c);
}

}  // namespace

extern "C" {

int sl_workspace_bytes_batch(const sl_params* params, int32_t n_replicas, size_t* bytes) {
  if (!bytes) return SL_ERR_ARG;
  int e = validate_batch(params, n_replicas);
  if (e) return e;
  SlDev d;
  std::vector<SlRep> reps;
  *bytes = plan(params, n_replicas, d, reps, nullptr);
  return SL_OK;
}

int sl_workspace_bytes(const sl_params* params, size_t* bytes) {
  return sl_workspace_bytes_batch(params, 1, bytes);
}

int sl_sector_grid(const sl_params* params, int32_t nsec[3], double edge[3]) {
  if (!nsec || !edge) return SL_ERR_ARG;
  int e = validate(params);
  if (e) return e;
  int n[3];
  double w[3];
  e = sector_grid(params, n, w);
  if (e) return e;
  for (int a = 0; a < 3; ++a) { nsec[a] = n[a]; edge[a] = w[a]; }
  return SL_OK;
}

int sl_init_batch(const sl_params* params, int32_t n_replicas, const double* r, const double* v,
                  const double* s, void* workspace, size_t workspace_bytes, void* cuda_stream, sl_ctx** out) {
  if (!out) return SL_ERR_ARG;
  *out = nullptr;
  int e = validate_batch(params, n_replicas);
  if (e) return e;
  if (!r || !v || !s) return SL_ERR_ARG;
  SlDev d;
  std::vector<SlRep> reps;
  size_t need = plan(params, n_replicas, d, reps, nullptr);
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255)) return SL_ERR_WORKSPACE;
  sl_ctx* c = new (std::nothrow) sl_ctx();
  if (!c) return SL_ERR_ARG;
  c->p = params[0];
  c->nrep = n_replicas;
  c->ws_base = workspace;
  c->ws_bytes = need;
  for (int r = 0; r < n_replicas; ++r) {
    c->lat_gamma.push_back(params[r].lattice_gamma_ps);
    c->lat_temp.push_back(params[r].lattice_temperature_K);
  }
  plan(params, n_replicas, c->d, c->reps, (char*)workspace);
  c->stream = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return SL_ERR_CUDA; }
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c;
    return SL_ERR_CUDA;
  }
  c->d.rb_cap = 8 * nsm;
  if (sl_prepare_kernels() != SL_OK || (c->d.ham == SL_HAM_LEARNED && sl_ml_prepare_kernels() != SL_OK)) {
    sl_destroy(c);
    return SL_ERR_CUDA;
  }
  cudaMemsetAsync(c->d.ctrl, 0, sizeof(SlCtrl), c->stream);
  cudaMemcpyAsync((void*)c->d.reps, c->reps.data(), sizeof(SlRep) * n_replicas, cudaMemcpyHostToDevice,
                  c->stream);
  k_load<<<grid_for(c->d.n), SL_BLOCK, 0, c->stream>>>(c->d, r, v, s, 1);
  k_check<<<grid_for(c->d.n), SL_BLOCK, 0, c->stream>>>(c->d);
  sl_launch_force_rebuild_flag(c->d, c->stream);
  e = refresh(c);
  int st = sync_status(c);
  if (e || st) { sl_destroy(c); return e ? e : st; }
  *out = c;
  return SL_OK;
}

int sl_init(const sl_params* params, const double* r, const double* v, const double* s,
            void* workspace, size_t workspace_bytes, void* cuda_stream, sl_ctx** out) {
  return sl_init_batch(params, 1, r, v, s, workspace, workspace_bytes, cuda_stream, out);
}

int sl_batch_size(sl_ctx* c) { return c ? c->nrep : SL_ERR_ARG; }

int sl_build_neighbors(sl_ctx* c) {
  if (!c) return SL_ERR_ARG;
  if (c->sticky) return c->sticky;
  DeviceGuard g(c->device);
  sl_launch_force_rebuild_flag(c->d, c->stream);
  return refresh(c);
}

int sl_step(sl_ctx* c, int32_t n_steps) {
  if (!c || n_steps < 0) return SL_ERR_ARG;
  if (c->sticky) return c->sticky;
  if (c->d.ham == SL_HAM_LEARNED && !c->ml_ready) return SL_ERR_ARG;
  if ((c->d.mech & SL_MECH_TAB) && !c->eam_ready) return SL_ERR_ARG;
  DeviceGuard g(c->device);
  if (int e = ml_fresh(c)) return e;
  if (c->timing) {
    // direct launches with an event pair around each phase
    for (int k = 0; k < n_steps; ++k) {
      int e = sl_launch_step(c->d, c->stream, mark_phase, c, &c->kernels_per_step);
      if (e) { c->sticky = e; return e; }
      if (c->ev_used > 4096 && fold_timing(c)) return cuda_err(c);
    }
    return cuda_err(c);
  }
  if (!c->graph_ok && n_steps > 0) build_graph(c);
  for (int k = 0; k < n_steps; ++k) {
    if (c->graph_ok) {
      if (cudaGraphLaunch(c->graph, c->stream) != cudaSuccess) return cuda_err(c);
    } else {
      int e = sl_launch_step(c->d, c->stream, nullptr, nullptr, &c->kernels_per_step);
      if (e) { c->sticky = e; return e; }
    }
  }
  return cuda_err(c);
}

int sl_set_timing(sl_ctx* c, int32_t enable) {
  if (!c) return SL_ERR_ARG;
  DeviceGuard g(c->device);
  if (c->ev_used && fold_timing(c)) return cuda_err(c);
  c->timing = enable ? 1 : 0;
  for (int k = 0; k < SL_NPHASE; ++k) { c->phase_ms[k] = 0.0; c->phase_n[k] = 0; }
  return c->sticky;
}

int sl_get_timing(sl_ctx* c, double ms[8], int64_t count[8]) {
  if (!c || !ms || !count) return SL_ERR_ARG;
  DeviceGuard g(c->device);
  if (c->ev_used && fold_timing(c)) return cuda_err(c);
  for (int k = 0; k < 8; ++k) {
    ms[k] = k < SL_NPHASE ? c->phase_ms[k] : 0.0;
    count[k] = k < SL_NPHASE ? c->phase_n[k] : 0;
  }
  return c->sticky;
}

int sl_set_dt(sl_ctx* c, double dt) {
  if (!c || !std::isfinite(dt)) return SL_ERR_ARG;
  DeviceGuard g(c->device);
  c->p.dt_ps = dt;
  c->d.dt = dt;
  fill_df_constants(c->d);
  if (c->d.any_noise || c->d.any_lattice_bath) {
    std::vector<sl_params> ps(c->nrep, c->p);
    for (int r = 0; r < c->nrep; ++r) {
      ps[r].lattice_gamma_ps = c->lat_gamma[r];
      ps[r].lattice_temperature_K = c->lat_temp[r];
      ps[r].mass_amu = c->p.mass_amu;
    }
    fill_noise(c->reps, ps.data(), dt);
    if (cudaMemcpyAsync((void*)c->d.reps, c->reps.data(), sizeof(SlRep) * c->nrep, cudaMemcpyHostToDevice,
                        c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return cuda_err(c);
  }
  drop_graph(c);
  return c->sticky;
}

// Natural cubic spline through (k h, y_k), k = 0 .. n-1: the knot second
// derivatives M solve M_{k-1} + 4 M_k + M_{k+1} = 6 (y_{k+1} - 2 y_k + y_{k-1})/h^2
// with M_0 = M_{n-1} = 0 (Thomas algorithm); interval k is then
// y_k + u [(y_{k+1} - y_k) - h^2 (2 M_k + M_{k+1})/6] + u^2 h^2 M_k/2
// + u^3 h^2 (M_{k+1} - M_k)/6, u = x/h - k.  coef: [n-1][4].
static void natural_spline(int n, double h, const double* y, std::vector<double>& coef) {
  std::vector<double> M(n, 0.0), piv(n, 0.0), rhs(n, 0.0);
  for (int k = 1; k + 1 < n; ++k) {
    const double b = 4.0 - (k > 1 ? 1.0 / piv[k - 1] : 0.0);
    piv[k] = b;
    rhs[k] = 6.0 * (y[k + 1] - 2.0 * y[k] + y[k - 1]) / (h * h) - (k > 1 ? rhs[k - 1] / piv[k - 1] : 0.0);
  }
  for (int k = n - 2; k >= 1; --k) M[k] = (rhs[k] - M[k + 1]) / piv[k];
  coef.assign((size_t)(n - 1) * 4, 0.0);
  const double h2 = h * h;
  for (int k = 0; k + 1 < n; ++k) {
    coef[4 * k] = y[k];
    coef[4 * k + 1] = (y[k + 1] - y[k]) - h2 * (2.0 * M[k] + M[k + 1]) / 6.0;
    coef[4 * k + 2] = h2 * M[k] / 2.0;
    coef[4 * k + 3] = h2 * (M[k + 1] - M[k]) / 6.0;
  }
}

int sl_set_eam_tables(sl_ctx* c, const sl_eam_tables* t) {
  if (!c || !t || !(c->d.mech & SL_MECH_TAB)) return SL_ERR_ARG;
  if (!t->F || !t->rho || !t->phi) return SL_ERR_ARG;
  if (t->nrho < 2 || t->nr < 2 || t->nrho > SL_EAM_MAX_POINTS || t->nr > SL_EAM_MAX_POINTS) return SL_ERR_ARG;
  if (!(t->drho > 0.0) || !(t->dr > 0.0) || !std::isfinite(t->drho) || !std::isfinite(t->dr)) return SL_ERR_ARG;
  if (!((t->nr - 1) * t->dr >= c->p.morse_rc_A)) return SL_ERR_ARG;
  for (int k = 0; k < t->nrho; ++k) if (!std::isfinite(t->F[k])) return SL_ERR_ARG;
  for (int k = 0; k < t->nr; ++k) if (!std::isfinite(t->rho[k]) || !std::isfinite(t->phi[k])) return SL_ERR_ARG;
  if (c->sticky) return c->sticky;
  DeviceGuard g(c->device);
  const int n[3] = {t->nrho, t->nr, t->nr};
  const double h[3] = {t->drho, t->dr, t->dr};
  const double* y[3] = {t->F, t->rho, t->phi};
  for (int q = 0; q < 3; ++q) {
    std::vector<double> coef;
    natural_spline(n[q], h[q], y[q], coef);
    std::vector<float4> cf((size_t)(n[q] - 1) * 2);
    for (int k = 0; k + 1 < n[q]; ++k) {
      const float2 a = split_f2(coef[4 * k]), b = split_f2(coef[4 * k + 1]);
      const float2 e = split_f2(coef[4 * k + 2]), f = split_f2(coef[4 * k + 3]);
      cf[2 * k] = make_float4(a.x, a.y, b.x, b.y);
      cf[2 * k + 1] = make_float4(e.x, e.y, f.x, f.y);
    }
    if (cudaMemcpyAsync(c->d.tab_d[q], coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice,
                        c->stream) != cudaSuccess ||
        cudaMemcpyAsync(c->d.tab_f[q], cf.data(), cf.size() * sizeof(float4), cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return cuda_err(c);
    c->d.tab_n[q] = n[q];
    c->d.tab_ih[q] = 1.0 / h[q];
    c->d.tab_ih_f[q] = split_f2(1.0 / h[q]);
  }
  c->eam_ready = 1;
  drop_graph(c);
  // densities and forces of the current state with the new potential
  int e = sl_launch_pairs_and_forces(c->d, c->stream, 0);
  if (e) return e;
  return sync_status(c);
}

int sl_set_field(sl_ctx* c, const double H[3]) {
  if (!c || !H) return SL_ERR_ARG;
  for (int a = 0; a < 3; ++a) {
    c->p.H_tesla[a] = H[a];
    c->d.zee[a] = c->p.mu_s_muB * SL_MUB * H[a];
  }
  fill_df_constants(c->d);
  drop_graph(c);
  return c->sticky;
}

// Per-replica sums of the observable terms, host [nrep][SL_NOBS].
static int observe(sl_ctx* c, std::vector<double>& red) {
  if (c->sticky) return c->sticky;
  DeviceGuard g(c->device);
  if (int e = ml_fresh(c)) return e;
  int e = sl_launch_observables(c->d, c->stream);
  if (e) return e;
  red.assign((size_t)c->nrep * SL_NOBS, 0.0);
  if (cudaMemcpyAsync(red.data(), c->d.obs_rep, red.size() * sizeof(double), cudaMemcpyDeviceToHost,
                      c->stream) != cudaSuccess)
    return cuda_err(c);
  return sync_status(c);
}

static void energy_of(const double* q, long long n, double out[8]) {
  out[0] = q[0]; out[1] = q[1]; out[2] = q[2]; out[3] = q[3];
  out[4] = q[0] + q[1] + q[2] + q[3] + q[10];
  out[5] = n > 0 ? 2.0 * q[0] / (3.0 * (double)n * SL_KB) : 0.0;
  out[6] = q[8] != 0.0 ? SL_HBAR / (2.0 * SL_KB) * q[7] / q[8] : 0.0;
  out[7] = q[10];
}

static void magnetization_of(const double* q, long long n, double out[4]) {
  double inv = n > 0 ? 1.0 / (double)n : 0.0;
  out[0] = q[4] * inv; out[1] = q[5] * inv; out[2] = q[6] * inv;
  out[3] = std::sqrt(out[0] * out[0] + out[1] * out[1] + out[2] * out[2]);
}

int sl_energy_batch(sl_ctx* c, double* out) {
  if (!c || !out) return SL_ERR_ARG;
  std::vector<double> red;
  int e = observe(c, red);
  if (e) return e;
  for (int r = 0; r < c->nrep; ++r) energy_of(&red[(size_t)r * SL_NOBS], c->reps[r].natoms, out + 8 * r);
  return SL_OK;
}

int sl_magnetization_batch(sl_ctx* c, double* out) {
  if (!c || !out) return SL_ERR_ARG;
  std::vector<double> red;
  int e = observe(c, red);
  if (e) return e;
  for (int r = 0; r < c->nrep; ++r) magnetization_of(&red[(size_t)r * SL_NOBS], c->reps[r].natoms, out + 4 * r);
  return SL_OK;
}

int sl_energy(sl_ctx* c, double out[8]) {
  if (!c || !out) return SL_ERR_ARG;
  std::vector<double> red;
  int e = observe(c, red);
  if (e) return e;
  double q[SL_NOBS] = {0};
  for (int r = 0; r < c->nrep; ++r)
    for (int k = 0; k < SL_NOBS; ++k) q[k] += red[(size_t)r * SL_NOBS + k];
  energy_of(q, c->d.n, out);
  return SL_OK;
}

int sl_magnetization(sl_ctx* c, double out[4]) {
  if (!c || !out) return SL_ERR_ARG;
  std::vector<double> red;
  int e = observe(c, red);
  if (e) return e;
  double q[SL_NOBS] = {0};
  for (int r = 0; r < c->nrep; ++r)
    for (int k = 0; k < SL_NOBS; ++k) q[k] += red[(size_t)r * SL_NOBS + k];
  magnetization_of(q, c->d.n, out);
  return SL_OK;
}

int sl_get_state(sl_ctx* c, double* r, double* v, double* s) {
  if (!c) return SL_ERR_ARG;
  if (c->sticky) return c->sticky;
  DeviceGuard g(c->device);
  int gn = grid_for(c->d.n);
  if (r) k_store<<<gn, SL_BLOCK, 0, c->stream>>>(c->d, c->d.r, r);
  if (v) k_store<<<gn, SL_BLOCK, 0, c->stream>>>(c->d, c->d.v, v);
  if (s) k_store<<<gn, SL_BLOCK, 0, c->stream>>>(c->d, c->d.s, s);
  return cuda_err(c);
}

int sl_set_state(sl_ctx* c, const double* r, const double* v, const double* s) {
  if (!c || !r || !v || !s) return SL_ERR_ARG;
  if (c->sticky) return c->sticky;
  DeviceGuard g(c->device);
  int gn = grid_for(c->d.n);
  k_load<<<gn, SL_BLOCK, 0, c->stream>>>(c->d, r, v, s, 0);
  k_check<<<gn, SL_BLOCK, 0, c->stream>>>(c->d);
  sl_launch_split(c->d, c->stream, 0);
  k_disp_flag<<<gn, SL_BLOCK, 0, c->stream>>>(c->d);
  return refresh(c);
}

int sl_get_state_host(sl_ctx* c, double* r, double* v, double* s) {
  if (!c) return SL_ERR_ARG;
  if (c->sticky) return c->sticky;
  DeviceGuard g(c->device);
  size_t n3 = (size_t)c->d.n * 3;
  double* st[3] = {c->d.stage, c->d.stage + n3, c->d.stage + 2 * n3};
  int e = sl_get_state(c, r ? st[0] : nullptr, v ? st[1] : nullptr, s ? st[2] : nullptr);
  if (e) return e;
  double* hs[3] = {r, v, s};
  for (int a = 0; a < 3; ++a)
    if (hs[a] && cudaMemcpyAsync(hs[a], st[a], n3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
      return cuda_err(c);
  return sync_status(c);
}

int sl_set_state_host(sl_ctx* c, const double* r, const double* v, const double* s) {
  if (!c || !r || !v || !s) return SL_ERR_ARG;
  if (c->sticky) return c->sticky;
  DeviceGuard g(c->device);
  size_t n3 = (size_t)c->d.n * 3;
  double* st[3] = {c->d.stage, c->d.stage + n3, c->d.stage + 2 * n3};
  const double* hs[3] = {r, v, s};
  for (int a = 0; a < 3; ++a)
    if (cudaMemcpyAsync(st[a], hs[a], n3 * sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
      return cuda_err(c);
  int e = sl_set_state(c, st[0], st[1], st[2]);
  if (e) return e;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_err(c);
  return SL_OK;
}

int sl_get_forces(sl_ctx* c, double* F) {
  if (!c || !F) return SL_ERR_ARG;
  if (c->sticky) return c->sticky;
  DeviceGuard g(c->device);
  if (int e = ml_fresh(c)) return e;
  k_store<<<grid_for(c->d.n), SL_BLOCK, 0, c->stream>>>(c->d, c->d.F, F);
  return cuda_err(c);
}

int sl_get_omega(sl_ctx* c, double* w) {
  if (!c || !w) return SL_ERR_ARG;
  if (c->sticky) return c->sticky;
  DeviceGuard g(c->device);
  if (int e = ml_fresh(c)) return e;
  int e = sl_launch_omega_all(c->d, w, c->stream);
  return e ? e : cuda_err(c);
}

int sl_get_order(sl_ctx* c, int32_t* order_dev, int32_t colour_start[9], int32_t nsec[3]) {
  if (!c) return SL_ERR_ARG;
  if (c->sticky) return c->sticky;
  DeviceGuard g(c->device);
  if (order_dev &&
      cudaMemcpyAsync(order_dev, c->d.perm, sizeof(int) * c->d.n, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
    return cuda_err(c);
  if (colour_start)
    for (int k = 0; k <= 8; ++k)
      if (cudaMemcpyAsync(colour_start + k, c->d.sec_start + k * c->d.s8, sizeof(int), cudaMemcpyDeviceToHost,
                          c->stream) != cudaSuccess)
        return cuda_err(c);
  if (nsec) { nsec[0] = c->reps[0].nx; nsec[1] = c->reps[0].ny; nsec[2] = c->reps[0].nz; }
  return sync_status(c);
}

int sl_counters(sl_ctx* c, int64_t out[8]) {
  if (!c || !out) return SL_ERR_ARG;
  DeviceGuard g(c->device);
  SlCtrl h;
  if (cudaMemcpyAsync(&h, c->d.ctrl, sizeof(SlCtrl), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return cuda_err(c);
  out[0] = h.step; out[1] = h.rebuilds; out[2] = h.max_ex_seen; out[3] = h.max_m_seen;
  out[4] = c->kernels_per_step; out[5] = c->graph_ok; out[6] = 0; out[7] = 0;
  if (h.status && !c->sticky) c->sticky = h.status;
  return c->sticky;
}

// ---------------------------------------------------------------------------
// Autotuner of the launch shapes
// ---------------------------------------------------------------------------
int sl_autotune(sl_ctx* c, void* scratch, size_t scratch_bytes, int32_t steps, int64_t out[8]) {
  if (!c || !scratch || !out || steps < 1) return SL_ERR_ARG;
  if (c->sticky) return c->sticky;
  if (scratch_bytes < c->ws_bytes) return SL_ERR_WORKSPACE;
  if (c->d.ham == SL_HAM_LEARNED && !c->ml_ready) return SL_ERR_ARG;
  if ((c->d.mech & SL_MECH_TAB) && !c->eam_ready) return SL_ERR_ARG;
  DeviceGuard g(c->device);
  if (int e = ml_fresh(c)) return e;
  cudaStream_t st = c->stream;
  if (cudaMemcpyAsync(scratch, c->ws_base, c->ws_bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return cuda_err(c);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_err(c);
  }
  const int blocks[3] = {64, 128, 256};
  // the learned step has its own sweep kernel: only the block size applies
  // (with the spin-orbit terms variants 5-9 repeat 0-4)
  const int nvar = c->d.ham == SL_HAM_LEARNED ? 1 : (c->d.so ? 5 : SL_SWEEP_VARIANTS);
  const int keep_sweep = c->d.tune_sweep, keep_block = c->d.tune_block;
  double best = 1e300, base = 0.0;
  int best_v = 0, best_b = SL_BLOCK, tried = 0, err = SL_OK;
  for (int v = 0; v < nvar && !err; ++v)
    for (int bi = 0; bi < 3 && !err; ++bi) {
      c->d.tune_sweep = v;
      c->d.tune_block = blocks[bi];
      int kp = 0;
      err = sl_launch_step(c->d, st, nullptr, nullptr, &kp);      // warm-up
      cudaEventRecord(e0, st);
      for (int k = 0; k < steps && !err; ++k) err = sl_launch_step(c->d, st, nullptr, nullptr, &kp);
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (!err && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        err = SL_ERR_CUDA;
      // every candidate starts from the same state
      if (cudaMemcpyAsync(c->ws_base, scratch, c->ws_bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        err = SL_ERR_CUDA;
      if (err) break;
      const double per = (double)ms / steps;
      if (v == 0 && blocks[bi] == SL_BLOCK) base = per;
      if (per < best) { best = per; best_v = v; best_b = blocks[bi]; }
      ++tried;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaStreamSynchronize(st) != cudaSuccess) err = SL_ERR_CUDA;
  if (err) {
    c->d.tune_sweep = keep_sweep;
    c->d.tune_block = keep_block;
    if (!c->sticky) c->sticky = err;
    return err;
  }
  c->d.tune_sweep = best_v;
  c->d.tune_block = best_b;
  drop_graph(c);
  out[0] = best_v;
  out[1] = best_b;
  out[2] = (int64_t)(best * 1e6);
  out[3] = (int64_t)(base * 1e6);
  out[4] = tried;
  out[5] = kSlSweepSPB[best_v];
  out[6] = 0;
  out[7] = 0;
  return sync_status(c);
}

int sl_set_launch_shape(sl_ctx* c, int32_t sweep_variant, int32_t block) {
  if (!c || sweep_variant < 0 || sweep_variant >= SL_SWEEP_VARIANTS) return SL_ERR_ARG;
  if (block != 64 && block != 128 && block != 256) return SL_ERR_ARG;
  c->d.tune_sweep = sweep_variant;
  c->d.tune_block = block;
  drop_graph(c);
  return c->sticky;
}

// ---------------------------------------------------------------------------
// Learned Hamiltonian
// ---------------------------------------------------------------------------
static int ml_check(sl_ctx* c, bool need_model) {
  if (!c) return SL_ERR_ARG;
  if (c->d.ham != SL_HAM_LEARNED) return SL_ERR_ARG;
  if (need_model && !c->ml_ready) return SL_ERR_ARG;
  return c->sticky;
}

int sl_ml_set_model(sl_ctx* c, const float* params, const float* norm) {
  if (!params || !norm) return SL_ERR_ARG;
  if (int e = ml_check(c, false)) return e;
  DeviceGuard g(c->device);
  const SlDev& d = c->d;
  if (cudaMemcpyAsync(d.ml_par, params, sizeof(float) * SL_ML_NPARAM, cudaMemcpyDefault, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(d.ml_norm, norm, sizeof(float) * SL_ML_NNORM, cudaMemcpyDefault, c->stream) != cudaSuccess ||
      cudaMemsetAsync(d.ml_m1, 0, sizeof(double) * SL_ML_NPARAM, c->stream) != cudaSuccess ||
      cudaMemsetAsync(d.ml_m2, 0, sizeof(double) * SL_ML_NPARAM, c->stream) != cudaSuccess)
    return cuda_err(c);
  c->ml_t = 0;
  int e = sl_ml_launch_prep(d, c->stream);
  if (e) return e;
  c->ml_ready = 1;
  drop_graph(c);
  return refresh(c);
}

int sl_ml_get_model(sl_ctx* c, float* params) {
  if (!params) return SL_ERR_ARG;
  if (int e = ml_check(c, true)) return e;
  DeviceGuard g(c->device);
  if (cudaMemcpyAsync(params, c->d.ml_par, sizeof(float) * SL_ML_NPARAM, cudaMemcpyDefault, c->stream) !=
      cudaSuccess)
    return cuda_err(c);
  return c->sticky;
}

int sl_ml_eval(sl_ctx* c, double* e_rep, double* F, double* B, double* D) {
  if (int e = ml_check(c, true)) return e;
  DeviceGuard g(c->device);
  int e = sl_ml_launch_eval(c->d, c->stream, F, B, D);
  if (e) return e;
  if (e_rep) {
    if (cudaMemcpyAsync(e_rep, c->d.ml_erep, sizeof(double) * c->nrep, cudaMemcpyDeviceToHost, c->stream) !=
        cudaSuccess)
      return cuda_err(c);
    return sync_status(c);
  }
  return cuda_err(c);
}

int sl_ml_descriptor_stats(sl_ctx* c, double* out) {
  if (!out) return SL_ERR_ARG;
  if (int e = ml_check(c, false)) return e;
  DeviceGuard g(c->device);
  // the gradient buffer (SL_ML_NPARAM doubles) serves as device scratch
  int e = sl_ml_launch_dstats(c->d, c->stream, c->d.ml_grad);
  if (e) return e;
  if (cudaMemcpyAsync(out, c->d.ml_grad, sizeof(double) * 4 * SL_ML_NF, cudaMemcpyDeviceToHost, c->stream) !=
      cudaSuccess)
    return cuda_err(c);
  return sync_status(c);
}

int sl_ml_gate(sl_ctx* c, int64_t out[4]) {
  if (!out) return SL_ERR_ARG;
  if (int e = ml_check(c, false)) return e;
  DeviceGuard g(c->device);
  if (int e = ml_fresh(c)) return e;
  SlCtrl h;
  if (cudaMemcpyAsync(&h, c->d.ctrl, sizeof(SlCtrl), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return cuda_err(c);
  out[0] = h.ml_bad_last; out[1] = h.ml_use; out[2] = h.ml_trips; out[3] = 0;
  if (h.status && !c->sticky) c->sticky = h.status;
  return c->sticky;
}

int sl_ml_vjp(sl_ctx* c, const double* gE, const double* gF, const double* gB, double* grad) {
  if (!grad) return SL_ERR_ARG;
  if (int e = ml_check(c, true)) return e;
  DeviceGuard g(c->device);
  int e = sl_ml_launch_eval(c->d, c->stream, nullptr, nullptr, nullptr);
  if (!e) e = sl_ml_launch_vjp(c->d, c->stream, gE, gF, gB);
  if (e) return e;
  if (cudaMemcpyAsync(grad, c->d.ml_grad, sizeof(double) * SL_ML_NPARAM, cudaMemcpyDeviceToDevice, c->stream) !=
      cudaSuccess)
    return cuda_err(c);
  return cuda_err(c);
}

int sl_ml_train_step(sl_ctx* c, const double* E_ref, const double* F_ref, const double* B_ref, const double w[3],
                     double lr, double beta1, double beta2, double eps, double* loss) {
  if (!E_ref || !F_ref || !B_ref || !w) return SL_ERR_ARG;
  if (!(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
    return SL_ERR_ARG;
  if (int e = ml_check(c, true)) return e;
  DeviceGuard g(c->device);
  c->ml_t += 1;
  int e = sl_ml_launch_train(c->d, c->stream, E_ref, F_ref, B_ref, w, lr, beta1, beta2, eps, c->ml_t);
  if (e) return e;
  c->ml_stale = 1;
  if (loss) {
    if (cudaMemcpyAsync(loss, c->d.ml_loss, sizeof(double) * 4, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
      return cuda_err(c);
    return sync_status(c);
  }
  return cuda_err(c);
}

int sl_status(sl_ctx* c) {
  if (!c) return SL_ERR_ARG;
  DeviceGuard g(c->device);
  return sync_status(c);
}

const char* sl_strerror(int code) {
  switch (code) {
    case SL_OK: return "ok";
    case SL_ERR_ARG: return "invalid argument";
    case SL_ERR_CUDA: return "CUDA runtime error";
    case SL_ERR_BOX: return "box smaller than twice the cutoff plus skin, or fewer than 2 sectors per edge";
    case SL_ERR_SPIN_NORM: return "input spin is not a unit vector";
    case SL_ERR_SKIN: return "an atom moved more than half the skin without a scheduled rebuild";
    case SL_ERR_TIMEOUT: return "an in-kernel wait exceeded its iteration budget";
    case SL_ERR_NONFINITE: return "non-finite value in the state";
    case SL_ERR_WORKSPACE: return "workspace missing, too small or not 256-byte aligned";
    case SL_ERR_NBR_OVERFLOW: return "neighbour list capacity exceeded";
    default: return "unknown error";
  }
}

void sl_destroy(sl_ctx* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  drop_graph(c);
  if (c->cap) cudaStreamDestroy(c->cap);
  for (cudaEvent_t ev : c->ev_pool) cudaEventDestroy(ev);
  delete c;
}

}  // extern "C"
