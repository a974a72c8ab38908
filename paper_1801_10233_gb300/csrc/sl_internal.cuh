// Internal device-side layout and helpers of libsl (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sl.h"

// Physical constants in the metal unit set (A, ps, eV, amu, K, T).
#define SL_HBAR 6.582119569e-4    // eV ps / rad
#define SL_KB 8.617333262e-5      // eV / K
#define SL_MUB 5.7883818060e-5    // eV / T
#define SL_FTOA 9648.533212       // (eV/A)/amu -> A/ps^2

#define SL_BLOCK 128
// Sectors per block of the colour-pass tile shapes (threads: 192, 256, 128, 128, 128).
// Variants 0-4: the pipelined pass; 5-9: the asynchronous-gather pass of the
// plain Hamiltonian (run as 0-4 with the spin-orbit terms).
static const int kSlSweepSPB[SL_SWEEP_VARIANTS] = {32, 32, 16, 16, 8, 16, 8, 32, 8, 4};
#define SL_MAX_EX_CAP 64   // largest accepted max_ex_neighbors
// Fixed-point positions X = rint(r 2^48), one scale for every context so a
// replica's trajectory does not depend on the batch it is in: positions
// below 16 A are rounded by at most 2^-49 A (above, FP64 is coarser), and
// |X| < 2^61 for positions within one box length of boxes below SL_FX_MAX_BOX.
#define SL_FX_BITS 48
#define SL_FX_MAX_BOX 4096.0  // box edges below 2^(60 - SL_FX_BITS) A
// Largest |x| whose double-float exp(x) keeps its 4e-14 accuracy (the
// reduction x = n ln2/64 + r is exact for |n| < 1024); parameter sets whose
// exponentials reach beyond it inside a cutoff are rejected on the host.
#define SL_DF_EXP_XMAX 11.0
// Sector edges exceed the sector reach (cutoff + skin) by at least this
// relative margin, so that a float distance test at the reach never lists a
// pair from two sectors of one colour.
#define SL_SECTOR_MARGIN 1e-6

// Control block in device memory: sticky status, rebuild flag, counters.
struct SlCtrl {
  int32_t status;           // first device error (0 = OK)
  int32_t need_rebuild;     // 1 while a rebuild is pending this step
  long long step;           // completed steps
  unsigned long long maxdisp2_bits;  // max |r - r_build|^2 since the last drift check
  int32_t rebuilds;
  int32_t max_ex_seen;
  int32_t max_m_seen;
  int32_t pad;
  // learned Hamiltonian: range gate of the current evaluation point
  int32_t ml_bad;           // atoms counted out of range by the descriptor kernel
  int32_t ml_use;           // 1: this evaluation point uses the network
  int32_t ml_trips;         // evaluation points handed to the analytic Hamiltonian
  int32_t ml_bad_last;      // ml_bad of the last evaluation point
};

// One system of a batch: its box, sector grid, atom range and spin bath.
struct SlRep {
  double box[3], inv_box[3], edge[3];
  long long boxX[3], halfX[3];   // box and half box in fixed point (units 2^-F A)
  int nx, ny, nz;           // sectors per edge (even, >= 2)
  int s8;                   // sectors per colour
  int mx, my, mz;           // sector layers searched for Morse neighbours
  int sec8_off;             // this replica's first rank inside each colour block
  int atom0, natoms;        // atom range in caller order
  int replica;              // Philox counter word of the spin noise
  double temperature;       // spin bath temperature (K)
  float2 noise_sig;         // sqrt(2 D_S / |dt/4|) as (hi, lo), D_S = lambda (1 + lambda^2) k_B T / hbar
  double lat_c1, lat_sig;   // lattice bath over dt/2: v <- c1 v + sig xi (c1 = 1, sig = 0: none)
};

// Spin-orbit term bits of SlDev::so.
enum { SL_SO_ANISO = 1, SL_SO_NEEL = 2, SL_SO_DMI = 4 };
// Mechanical-potential bits of SlDev::mech: embedding term, ground-state
// subtraction, tabulated form (pair term and embedding from splines; set with
// SL_MECH_EAM).
enum { SL_MECH_EAM = 1, SL_MECH_GROUND = 2, SL_MECH_TAB = 4 };
// Tables of the tabulated embedded-atom potential.
enum { SL_TAB_F = 0, SL_TAB_RHO = 1, SL_TAB_PHI = 2 };

// Double-float constants of one f(r) = 4 alpha x (1 - gamma x) e^{-x},
// x = r^2/delta^2 (Eq. BSfunction): 1/delta^2, 4 alpha, gamma, 8 alpha/delta^2.
struct SlBsF {
  float2 ix, a4, g, a8d2;
};

// A position in fixed point (units 2^-F A), one 32-byte load.
struct __align__(32) SlFix {
  long long x, y, z, w;
};

// Everything a kernel needs, passed by value.  Scalars used by the
// double-float kernels are given as (hi, lo) float pairs split on the host.
// Sector ranks are global and colour-major: rank = colour * s8 + sec8_off of
// the replica + rank of the sector within its colour, so one colour pass
// covers the sectors of every replica.
struct SlDev {
  int n;                    // atoms of all replicas
  int nrep;
  int nsec, s8;             // sectors, sectors per colour (all replicas)
  int max_ex, max_m;
  int rotation, fix_lattice, rebuild_every, morse_shift;
  double dt;
  double zee[3];            // mu_s mu_B H (eV)
  double acc;               // FTOA / m
  double mass;
  double ex_alpha, ex_gamma, ex_delta, ex_rc2;
  double m_D0, m_alpha, m_r0, m_rc2, m_vshift;
  double list_ex2, list_m2; // (cutoff + skin)^2
  float fx_s40, fx_s20, fx_s0;   // 2^(40-F), 2^(20-F), 2^-F
  double sure_m2;           // (morse_rc - skin)^2 (0 if skin >= morse_rc)
  double half_skin2;
  double lambda;
  int any_noise;            // some replica has a bath temperature
  int any_lattice_bath;     // some replica has a lattice bath
  uint64_t seed;
  int ham;                  // SL_HAM_ANALYTIC or SL_HAM_LEARNED
  int tune_sweep;           // colour-pass tile shape variant (0 .. SL_SWEEP_VARIANTS-1)
  int tune_block;           // threads per block of the per-atom kernels (0: SL_BLOCK)
  int rb_cap;               // most blocks of a rebuild kernel (grid-stride loops)

  // double-float constants (hi, lo)
  float2 zee_f[3], inv_hbar_f, tau_f;        // tau = dt/4
  float2 m_nalpha_f, m_r0_f, m_c2_f, m_rc2_f; // -a, r0, 2 a D0, rc^2
  float2 ex_ix_f, ex_4a_f, ex_g_f, ex_8ad2_f, ex_rc2_f;  // 1/delta^2, 4 alpha, gamma, 8 alpha/delta^2, rc^2
  float2 lam_f, inv1pl2_f;                   // lambda, 1/(1 + lambda^2)

  // spin-orbit terms (App. A.2): so = SL_SO_ANISO | SL_SO_NEEL | SL_SO_DMI bits
  int so;
  double an_K, an_n[3];                       // -K sum_i (s_i.n)^2
  float2 an_c_f, an_cl_f, an_n_f[3];          // 2K/hbar, 2K/(hbar (1 + lambda^2)), n
  SlBsF ne_bs, dm_bs;                         // double-float constants of g1 and d

  // mechanical potential beyond the Morse pairs (App. B): mech = SL_MECH_EAM |
  // SL_MECH_GROUND bits; F(rho) = -A sqrt(rho), f(r) = (r - d)^2 + beta (r - d)^3 / d
  int mech;
  int em_fused;                               // d <= ex_rc: the density comes from the exchange entries
  double em_A, em_d, em_beta;
  float2 em_d_f, em_d2_f, em_bd_f, em_hA_f;   // d, d^2, beta/d, A/2
  // tabulated form (SL_MECH_TAB): natural cubic splines of F(rho), rho(r),
  // phi(r); interval k holds c0..c3 of c0 + u (c1 + u (c2 + u c3)), u = x/h - k,
  // in FP64 (tab_d, [n-1][4]) and as double-float pairs (tab_f, [n-1][2]:
  // (c0, c1), (c2, c3)); tab_n = 0 until the tables are set
  int tab_n[3];
  double tab_ih[3];                            // 1/h
  float2 tab_ih_f[3];
  double* tab_d[3];
  float4* tab_f[3];

  const SlRep* reps;        // [nrep]
  int* arep;                // replica of each sorted atom
  int* tarep;               // rebuild scratch

  // state, sector-sorted (FP64, authoritative)
  double4_32a *r, *v, *s, *F;
  SlFix *rbx;               // positions at the last rebuild, fixed point
  // copies for the pair and double-float kernels
  SlFix *rx;                // r in fixed point, rint(r 2^48)
  float4 *sdf;              // s = hi + lo to ~48 bits: sdf[2i] = hi, sdf[2i+1] = lo
  // rebuild scratch
  double4_32a *tr, *tv, *ts, *tF;
  int *perm, *rank, *secq, *tsecq, *tperm, *src;
  int *sec_count, *sec_start, *sec_fill;
  // neighbour lists
  int *exj, *exn, *exin;    // [max_ex][n] neighbour-major (same-sector entries first), counts
  uint2 *exc;               // [n] start of each colour's group of the other entries, one byte per colour
  // [n] dependency level of each atom inside its sector's sweep: low byte
  // forward, high byte backward (0 for an atom no earlier same-sector list
  // neighbour precedes, else 1 + the largest level of those neighbours)
  unsigned short *lvl;
  float2 *exJ;              // [max_ex][n] J_ij (hi, lo) at current r
  float2 *exdJ;             // [max_ex][n] J'(r_ij)/r_ij (hi, lo) at current r, for the forces
  // [5][max_ex][n] g1, d, e_x, e_y, e_z (hi, lo) at current r, e = (r_j - r_i)/r;
  // zero beyond ex_rc (NULL when so == 0)
  float2 *exso;
  // [n] F'(rho_i) (hi, lo) at current r, sorted order (NULL unless mech has SL_MECH_EAM)
  float2 *em_fp;
  int *mj, *mn;             // [max_m][n] neighbour-major, counts
  int *mnc;                 // [n] end of the entries certain to be inside morse_rc until the next rebuild
  // sweep scratch for blocks whose atoms exceed shared memory: [3 n] each
  float2 *hbuf, *sbuf, *ebuf;
  float2 *xbuf, *ebuf2;     // the fused pass's external field and second noise
  // partial external fields precomputed for the next colour pass (ping-pong)
  float2 *hpart[2];         // [3 n] each
  // per-atom observables in caller order [n][SL_NOBS], per-replica sums
  double *obs_atom, *obs_rep;   // [nrep][SL_NOBS]
  // staging for host copies, [n][3] doubles x 3
  double *stage;
  SlCtrl *ctrl;

  // learned Hamiltonian (NULL unless ham == SL_HAM_LEARNED)
  float *ml_par;            // [SL_ML_NPARAM] float32 master parameters
  float *ml_norm;           // [SL_ML_NNORM] mean, inv_std, gate lo, gate hi
  uint4 *ml_tiles;          // bfloat16 weight tiles in the MMA's shared-memory layout
  float *ml_fc;             // epilogue constants (SL_MLC_* offsets)
  float *ml_x;              // [n][48] normalised descriptors
  float *ml_G;              // [n][48] dE_i/dD_i
  float *ml_e;              // [n] E_i
  float4 *ml_B;             // [n] -dE/ds_i
  float2 *ml_pq;            // [max_m][n] frozen field coefficients (P, Q)
  float *ml_u;              // [n][48] tangent direction / descriptor scratch
  float4 *ml_gF, *ml_gB;    // [n] upstream gradients of F and B (sorted order)
  double *ml_alpha;         // [n] upstream gradient of E_i (its replica's)
  float *ml_gpart;          // [tiles][SL_ML_NPARAM] per-tile parameter gradients
  double *ml_grad;          // [SL_ML_NPARAM]
  double *ml_m1, *ml_m2;    // Adam moments
  double *ml_erep;          // [nrep] sum of E_i per replica
  double *ml_lossat;        // [n][2] per-atom loss terms
  double *ml_loss;          // [4]
};

// Offsets into ml_fc (floats): b1[64], b2[64], w3[64] (bfloat16 values), b3,
// then mean, inv_std, lo, hi [48] each.
#define SL_MLC_B1 0
#define SL_MLC_B2 64
#define SL_MLC_W3 128
#define SL_MLC_B3 192
#define SL_MLC_MEAN 256
#define SL_MLC_ISTD 304
#define SL_MLC_LO 352
#define SL_MLC_HI 400
#define SL_MLC_SIZE 448
// Bytes of the bfloat16 weight tiles: W1 [64 x 48], W2 [64 x 64], W2^T [64 x 64], W1^T [48 x 64].
#define SL_ML_TILE_BYTES (2 * (64 * 48 + 64 * 64 + 64 * 64 + 48 * 64))
#define SL_ML_ATOMS_PER_TILE 128

#define SL_NOBS 11  // Ek, Em, Ex, Ez, Mx, My, Mz, TS numerator, TS denominator, non-finite flag, E_spin_orbit

__device__ __forceinline__ void sl_set_error(SlCtrl* c, int code) { atomicCAS(&c->status, 0, code); }

// Minimum-image separation of a and b (b - a) in the replica's box.
__device__ __forceinline__ double3 sl_min_image(const SlRep& R, double4_32a a, double4_32a b) {
  double x = b.x - a.x, y = b.y - a.y, z = b.z - a.z;
  x -= R.box[0] * rint(x * R.inv_box[0]);
  y -= R.box[1] * rint(y * R.inv_box[1]);
  z -= R.box[2] * rint(z * R.inv_box[2]);
  return make_double3(x, y, z);
}

// Wrap one coordinate into [0, L] with explicitly rounded operations, so the
// result is the IEEE value of x - L * floor(x / L) (no contraction).
__device__ __forceinline__ double sl_wrap(double x, double L) {
  return __dsub_rn(x, __dmul_rn(L, floor(__ddiv_rn(x, L))));
}

__device__ __forceinline__ int sl_sector_coord(double xw, double e, int n) {
  int k = (int)floor(__ddiv_rn(xw, e));
  return k < 0 ? 0 : (k >= n ? n - 1 : k);
}

// Global sector rank: colours 0..7 in order; inside a colour, replicas in
// order; inside a replica, sectors by ascending linear index sx + nx (sy + ny sz).
__device__ __forceinline__ int sl_sector_rank(const SlDev& d, const SlRep& R, int sx, int sy, int sz) {
  int c = (sx & 1) + 2 * (sy & 1) + 4 * (sz & 1);
  int hx = sx >> 1, hy = sy >> 1, hz = sz >> 1;
  return c * d.s8 + R.sec8_off + hx + (R.nx >> 1) * (hy + (R.ny >> 1) * hz);
}

__device__ __forceinline__ void sl_sector_coords(const SlDev& d, const SlRep& R, int q, int& sx, int& sy, int& sz) {
  int c = q / d.s8, rem = q - c * d.s8 - R.sec8_off;
  int hxn = R.nx >> 1, hyn = R.ny >> 1;
  int hx = rem % hxn, hy = (rem / hxn) % hyn, hz = rem / (hxn * hyn);
  sx = 2 * hx + (c & 1);
  sy = 2 * hy + ((c >> 1) & 1);
  sz = 2 * hz + ((c >> 2) & 1);
}

// Launch helpers implemented in the .cu files.
int sl_launch_rebuild(const SlDev& d, cudaStream_t st);
int sl_launch_pairs_and_forces(const SlDev& d, cudaStream_t st, int kick);
int sl_launch_split(const SlDev& d, cudaStream_t st, int only_if_rebuild);
int sl_prepare_kernels();
// The spin half-op: its 15 colour passes in the context's tile shape, noise
// sub-passes from subpass0 (sl_sweep.cu for the plain Hamiltonian,
// sl_sweep_so.cu with the spin-orbit terms); the pass kernels'
// shared-memory limits.
#define SL_SWEEP_PASSES 15
void sl_launch_half_op_plain(const SlDev& d, cudaStream_t st, int subpass0);
void sl_launch_half_op_so(const SlDev& d, cudaStream_t st, int subpass0);
int sl_prepare_sweep_plain();
int sl_prepare_sweep_so();
inline void sl_launch_half_op(const SlDev& d, cudaStream_t st, int subpass0) {
  if (d.so) sl_launch_half_op_so(d, st, subpass0);
  else sl_launch_half_op_plain(d, st, subpass0);
}
// Phases of one step, for optional event timing.
enum { SL_PHASE_KICK = 0, SL_PHASE_SPIN1 = 1, SL_PHASE_DRIFT = 2, SL_PHASE_JTABLE = 3, SL_PHASE_SPIN2 = 4,
       SL_PHASE_FORCE = 5, SL_NPHASE = 6 };
#define SL_REBUILD_KERNELS 11
typedef void (*SlPhaseMark)(void* user, int phase, int end, cudaStream_t st);
int sl_launch_step(const SlDev& d, cudaStream_t st, SlPhaseMark mark, void* user, int* kernels);
int sl_launch_observables(const SlDev& d, cudaStream_t st);
int sl_launch_force_rebuild_flag(const SlDev& d, cudaStream_t st);
int sl_launch_omega_all(const SlDev& d, double* out, cudaStream_t st);
// Learned Hamiltonian (sl_ml.cu).
// Evaluation point: descriptors + gate, network, pair terms; fmode 0: only
// the field table, 1: also forces into F, 3: forces and the closing half-kick.
// With force = 1 the gate is ignored and left unchanged.
int sl_ml_launch_point(const SlDev& d, cudaStream_t st, int fmode);
int sl_ml_launch_half_op(const SlDev& d, cudaStream_t st);
int sl_ml_launch_prep(const SlDev& d, cudaStream_t st);
int sl_ml_launch_eval(const SlDev& d, cudaStream_t st, double* F, double* B, double* D);
int sl_ml_launch_dstats(const SlDev& d, cudaStream_t st, double* out_dev);
int sl_ml_launch_vjp(const SlDev& d, cudaStream_t st, const double* gE, const double* gF, const double* gB);
int sl_ml_launch_train(const SlDev& d, cudaStream_t st, const double* E_ref, const double* F_ref,
                       const double* B_ref, const double w[3], double lr, double b1, double b2, double eps,
                       long long t);
int sl_ml_prepare_kernels();
