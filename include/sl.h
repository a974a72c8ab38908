/*
 * libsl: coupled spin-lattice dynamics on one GPU (sm_103a), C ABI.
 *
 * The method is the symplectic Suzuki-Trotter integrator of
 * Tranchida, Plimpton, Thibaudeau, Thompson (arXiv 1801.10233):
 *
 *   one step = e^{Lp dt/2} e^{Ls dt/2} e^{Lr dt} e^{Ls dt/2} e^{Lp dt/2}
 *              (Eq. general_ST_decomposition, Sec. 3)
 *
 * where e^{Ls dt/2} sweeps the spins forward then backward with dt/4 per
 * single-spin factor (Eq. spin_ST_decomposition, Sec. 3), in the sectored
 * order of Eq. spin_ST_sectoring (Sec. 5.1): atoms are binned into sectors at
 * least (exchange cutoff + skin) wide, an even number per box edge, and each
 * sector gets one of 8 colours from the parities of its sector coordinates.
 * Same-colour sectors never interact, so a colour pass updates all of them at
 * once while the spins inside a sector go one after another (ascending atom
 * id forward, descending backward).
 *
 * Hamiltonian (Eq. s_hamiltonian and Eq. sl_hamiltonian, Sec. 2):
 *   H = -mu_s mu_B sum_i H.s_i - sum_{i<j} J(r_ij) s_i.s_j
 *       + sum_i p_i^2 / 2m + sum_{i<j} V(r_ij)
 * J(r) = 4 alpha (r/delta)^2 (1 - gamma (r/delta)^2) exp(-(r/delta)^2) for
 * r < ex_rc (Eq. BSfunction, App. A.1); V(r) = D0 (e^{-2a(r-r0)} -
 * 2 e^{-a(r-r0)}) for r < morse_rc.  omega_i = -(1/hbar) dH/ds_i and
 * ds_i/dt = omega_i x s_i (Eq. s_advance); the force is -dH/dr_i including
 * the magneto-elastic term -J'(r) (s_i.s_j) e_ij (Eq. p_advance).
 *
 * Units: Angstrom, ps, eV, amu, K, Tesla.  State arrays are FP64.
 *
 * Conventions for every entry point:
 *  - Pointers documented as "device" must be device memory of the current
 *    CUDA device; "host" pointers are host memory (pinned for best speed).
 *  - Position, velocity and spin arrays are [n_atoms][3] doubles (x,y,z per
 *    atom) in the caller's atom order.  The library never frees or retains
 *    caller memory beyond the call, except the workspace given to sl_init,
 *    which it uses until sl_destroy.
 *  - All work is ordered on the CUDA stream given to sl_init.  Only
 *    sl_init, sl_energy, sl_magnetization, sl_status, sl_counters and the
 *    *_host copies block the calling thread.
 *  - Return values are SL_OK (0) or a negative SL_ERR_* code.  Errors raised
 *    on the device (timeout, skin violation, list overflow, bad spin norm) are
 *    sticky: once set, every later call returns that code until sl_destroy.
 *    The library never aborts the process.
 */
#ifndef SL_H
#define SL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SL_OK = 0,
  SL_ERR_ARG = -1,          /* invalid argument or parameter */
  SL_ERR_CUDA = -2,         /* a CUDA runtime call failed */
  SL_ERR_BOX = -3,          /* box < 2 (cutoff + skin), < 2 sectors per edge, or an edge >= 4096 A */
  SL_ERR_SPIN_NORM = -4,    /* an input spin is not unit length (|1 - |s|| > 1e-12) */
  SL_ERR_SKIN = -5,         /* an atom moved > skin/2 with no rebuild scheduled */
  SL_ERR_TIMEOUT = -6,      /* an in-kernel wait ran out of its iteration budget */
  SL_ERR_NONFINITE = -7,    /* a NaN or Inf entered the state */
  SL_ERR_WORKSPACE = -8,    /* workspace missing, too small or misaligned */
  SL_ERR_NBR_OVERFLOW = -9  /* more neighbours than max_*_neighbors */
};

enum { SL_ROT_RODRIGUES = 0, SL_ROT_CAYLEY = 1 };
enum { SL_HAM_ANALYTIC = 0, SL_HAM_LEARNED = 1 };

/* Parameters of one system.  Zero-initialise and fill every field. */
typedef struct sl_params {
  int32_t n_atoms;
  int32_t rotation;            /* SL_ROT_RODRIGUES: exact rotation by |omega| tau;
                                  SL_ROT_CAYLEY: the Cayley-type propagator of Sec. 3 */
  int32_t fix_lattice;         /* 1: positions/velocities frozen, spin dynamics only */
  int32_t rebuild_every;       /* 0: rebuild sectors and lists when an atom moved more
                                  than skin/2; K > 0: every K steps (SL_ERR_SKIN if the
                                  skin is exceeded in between) */
  int32_t morse_shift_energy;  /* 1: report V(r) - V(rc) per pair (forces unchanged) */
  int32_t max_ex_neighbors;    /* exchange list capacity per atom (0: 24) */
  int32_t max_morse_neighbors; /* Morse list capacity per atom (0: 128); the list
                                  holds the exchange neighbours first, so values not
                                  above max_ex_neighbors are raised to it + 1 */
  int32_t hamiltonian;         /* SL_HAM_ANALYTIC (0) or SL_HAM_LEARNED (1), see below */
  double box[3];               /* orthorhombic periodic box edges */
  double mass_amu;
  double mu_s_muB;             /* magnetic moment, units of mu_B */
  double H_tesla[3];           /* applied field */
  double dt_ps;                /* timestep (may be negative: time reversal) */
  double ex_alpha_eV, ex_gamma, ex_delta_A, ex_rc_A;            /* Eq. BSfunction */
  double morse_D0_eV, morse_alpha_invA, morse_r0_A, morse_rc_A;
  double skin_A;               /* Verlet skin, also widens the sectors */
  double lambda;               /* transverse damping of Eq. sLLG (0: none) */
  double temperature_K;        /* spin bath temperature (0: no noise) */
  uint64_t seed;               /* Philox4x32-10 key for the spin and lattice noise */
  int32_t replica;             /* replica index, part of the noise counter */
  int32_t reserved1;
  double lattice_gamma_ps;     /* lattice bath damping rate gamma_L/m of Eq. p_advance_T
                                  (Sec. 4.2), 1/ps (0: NVE lattice) */
  double lattice_temperature_K;/* lattice bath temperature (noise D_L = 2 m gamma_L/m k_B T,
                                  the Einstein relation); the bath is the exact
                                  Ornstein-Uhlenbeck flow of the velocities over dt/2 at
                                  both ends of the step (before the first half-kick, after
                                  the closing one), noise counter sub-passes 4 and 5 */
  /* Spin-orbit terms (App. A.2), analytic Hamiltonian only; zero turns each off.
   * Uniaxial anisotropy H_an = -K sum_i (s_i.n)^2 with n a unit vector (|n| = 1
   * within 1e-12, else SL_ERR_ARG).  Its precession vector (2K/hbar)(s_i.n) n
   * keeps s_i.n fixed, so each single-spin factor turns s_i half its time about
   * n alone, then the whole time about the rest of omega_i, then the other
   * half about n: a symmetric split whose pieces are exact flows.
   * Neel pseudo-dipolar pair term -g1(r) ((e.s_i)(e.s_j) - s_i.s_j/3) and
   * Dzyaloshinskii-Moriya term d(r) e.(s_i x s_j), e = (r_j - r_i)/r, each
   * unordered pair within ex_rc_A once; g1 and d take the form of
   * Eq. BSfunction with their own (alpha, gamma, delta). */
  double aniso_K_eV;
  double aniso_axis[3];
  double neel_alpha_eV, neel_gamma, neel_delta_A;
  double dmi_alpha_eV, dmi_gamma, dmi_delta_A;
  /* Mechanical potential beyond the Morse pairs (App. B), analytic Hamiltonian
   * only; zero turns each off.  Embedding term sum_i F(rho_i) of the embedded-atom
   * method in the Finnis-Sinclair form: F(rho) = -eam_A_eV sqrt(rho) (0 at
   * rho = 0), rho_i = sum_j f(r_ij), f(r) = (r - d)^2 + beta (r - d)^3 / d for
   * r < d = eam_d_A (0 < d <= morse_rc_A, else SL_ERR_ARG), 0 beyond.  With
   * subtract_ground_exchange = 1 the collinear magnetic ground state is taken
   * out of the mechanical energy (Eq. app:mech1): + J(r_ij) per unordered pair,
   * so the exchange adds neither energy nor force to a collinear state.  Both
   * are reported in E_morse (the mechanical energy) by sl_energy. */
  double eam_A_eV, eam_d_A, eam_beta;
  int32_t subtract_ground_exchange;
  /* 1: the mechanical potential is the tabulated embedded-atom form of App. B
   * instead of the Morse pairs (and eam_A_eV must be 0): pair term phi(r) and
   * embedding F(rho_i), rho_i = sum_j rho(r_ij), over r < morse_rc_A, each a
   * natural cubic spline through a table on a uniform grid given by
   * sl_set_eam_tables (sl_step returns SL_ERR_ARG until then; the forces of
   * sl_init have no mechanical part).  Analytic Hamiltonian only; the
   * exchange and the ground-state subtraction combine with it as above. */
  int32_t eam_tabulated;
} sl_params;

typedef struct sl_ctx sl_ctx;  /* opaque, owned by the library */

/* Bytes of device workspace sl_init needs for these parameters.
 * Errors: SL_ERR_ARG (NULL pointer, n_atoms < 1, non-positive mass,
 * morse_rc_A < ex_rc_A, max_ex_neighbors above 64),
 * SL_ERR_BOX (box too small for the cutoffs or for 2 sectors per edge, or an
 * edge of 4096 A or more: positions are held in 64-bit fixed point too). */
int sl_workspace_bytes(const sl_params* params, size_t* bytes);

/* Sector grid of the sectored sweep (Sec. 5.1) for these parameters, on the
 * host (no device call): nsec (host, 3) sectors per edge, the largest even
 * counts whose edges edge (host, 3, A) exceed the spin reach (ex_rc_A, or
 * the learned model's 6 A cutoff, plus skin_A) by a relative margin of 1e-6.
 * Sectors of one colour are then more than the reach apart while no atom has
 * moved more than skin/2, so their spins never interact within a pass.
 * Errors: those of sl_workspace_bytes. */
int sl_sector_grid(const sl_params* params, int32_t nsec[3], double edge[3]);

/* Create a context: copies r, v, s (device, [n][3] doubles, caller order)
 * into the library's sector-sorted layout inside `workspace` (device,
 * >= sl_workspace_bytes, 256-byte aligned, owned by the caller and kept
 * alive until sl_destroy), wraps positions into the box, assigns sectors,
 * builds neighbour lists and the exchange table and computes the forces
 * F(r0, s0).  `cuda_stream` is a cudaStream_t (NULL: legacy default stream).
 * Blocks until done; on error *out is NULL and nothing is retained.
 * Errors: SL_ERR_ARG, SL_ERR_BOX, SL_ERR_WORKSPACE, SL_ERR_SPIN_NORM,
 * SL_ERR_NONFINITE, SL_ERR_NBR_OVERFLOW, SL_ERR_CUDA. */
int sl_init(const sl_params* params, const double* r, const double* v, const double* s,
            void* workspace, size_t workspace_bytes, void* cuda_stream, sl_ctx** out);

/* Batches: n_replicas independent systems advanced together, for instance
 * replicas of different sizes at different bath temperatures.  params[k]
 * describes replica k; replicas may differ in n_atoms, box, temperature_K,
 * lattice_gamma_ps, lattice_temperature_K and replica (the noise counter
 * word), and every other field must equal params[0]'s (SL_ERR_ARG otherwise).  r, v, s (device) hold all replicas'
 * atoms back to back in replica order, [sum n_atoms][3] doubles.  Each colour
 * pass of a step covers the sectors of every replica, so one step advances
 * the whole batch.  sl_workspace_bytes and sl_init are the n_replicas = 1
 * cases.  Replica k's trajectory is bitwise the one it has alone. */
int sl_workspace_bytes_batch(const sl_params* params, int32_t n_replicas, size_t* bytes);
int sl_init_batch(const sl_params* params, int32_t n_replicas, const double* r, const double* v,
                  const double* s, void* workspace, size_t workspace_bytes, void* cuda_stream, sl_ctx** out);

/* Number of replicas in the context (SL_ERR_ARG for NULL). */
int sl_batch_size(sl_ctx* ctx);

/* Per-replica observables: out (host) [n_replicas][8] as sl_energy, and
 * [n_replicas][4] as sl_magnetization.  Synchronise. */
int sl_energy_batch(sl_ctx* ctx, double* out);
int sl_magnetization_batch(sl_ctx* ctx, double* out);

/* Re-assign sectors and rebuild both neighbour lists, the exchange table
 * (J and J' at the current positions, Sec. 3) and the forces now, whatever
 * the displacement.  Stream-ordered. */
int sl_build_neighbors(sl_ctx* ctx);

/* Advance n_steps timesteps of Eq. general_ST_decomposition.  Stream-ordered;
 * device-side errors surface at the next synchronising call. */
int sl_step(sl_ctx* ctx, int32_t n_steps);

/* Change dt (negative runs the dynamics backwards) or the applied field. */
int sl_set_dt(sl_ctx* ctx, double dt_ps);
int sl_set_field(sl_ctx* ctx, const double H_tesla[3]);

/* Tables of the tabulated embedded-atom potential (App. B; contexts created
 * with eam_tabulated = 1), in the uniform-grid form such potentials are
 * distributed in: F at rho = k drho (k = 0 .. nrho-1, eV), rho(r) and phi(r)
 * (eV) at r = k dr (k = 0 .. nr-1), the r grid reaching at least morse_rc_A.
 * Each function is the natural cubic spline through its table (zero second
 * derivative at both ends; F is extended past its last point by its last
 * cubic).  The arrays are host memory, read during the call.
 * The library solves for the splines in FP64, keeps their coefficients in its
 * workspace (FP64 for the energies, double-float for the force and density
 * kernels), and recomputes the densities and forces at the current state.
 * Applies to every replica of a batch.  Synchronises.
 * Errors: SL_ERR_ARG (context without eam_tabulated, NULL arrays, fewer than
 * 2 or more than SL_EAM_MAX_POINTS points, non-positive spacing, an r grid
 * short of morse_rc_A, non-finite values), SL_ERR_CUDA. */
#define SL_EAM_MAX_POINTS 16384
typedef struct sl_eam_tables {
  int32_t nrho, nr;
  double drho, dr;
  const double* F;     /* [nrho] */
  const double* rho;   /* [nr] */
  const double* phi;   /* [nr] */
} sl_eam_tables;
int sl_set_eam_tables(sl_ctx* ctx, const sl_eam_tables* tables);

/* out[8] (host) = E_kin, E_morse (the mechanical energy: Morse, embedding and
 * ground-state subtraction), E_exchange, E_zeeman, E_total (eV),
 * T_L (Eq. lattice_temperature, K), T_S (Eq. spin_temperature, K), E_spin_orbit
 * (anisotropy + Neel + DMI, eV; part of E_total).
 * Pair energies count each unordered pair once.  For a batch: energies summed
 * over the replicas, temperatures over all atoms.  Synchronises. */
int sl_energy(sl_ctx* ctx, double out[8]);

/* out[4] (host) = Mx, My, Mz, |M| with M = (1/N) sum_i s_i (all atoms of a
 * batch).  Synchronises. */
int sl_magnetization(sl_ctx* ctx, double out[4]);

/* Copy the state out in caller atom order (device pointers, [n][3]; any of
 * them may be NULL).  Positions are wrapped into the box at every rebuild. */
int sl_get_state(sl_ctx* ctx, double* r, double* v, double* s);

/* Replace the state (device pointers, [n][3], caller order).  Sectors and
 * lists are rebuilt if an atom moved more than skin/2 from where the lists
 * were built; the exchange table and forces are recomputed.  Spins must be
 * unit length (SL_ERR_SPIN_NORM otherwise, sticky). */
int sl_set_state(sl_ctx* ctx, const double* r, const double* v, const double* s);

/* As sl_get_state / sl_set_state with HOST pointers: the copies run through
 * a staging area in the workspace.  sl_get_state_host blocks until the data
 * has arrived; sl_set_state_host blocks until the host buffers may be reused. */
int sl_get_state_host(sl_ctx* ctx, double* r, double* v, double* s);
int sl_set_state_host(sl_ctx* ctx, const double* r, const double* v, const double* s);

/* Forces F (eV/A) and precession vectors omega (rad/ps, no noise) of the
 * current state, device pointers [n][3], caller order. */
int sl_get_forces(sl_ctx* ctx, double* F);
int sl_get_omega(sl_ctx* ctx, double* omega);

/* Sweep order: order_dev[k] (device, n int32) = caller index of the k-th
 * atom of the sweep; colour_start[9] (host) = first sweep position of each
 * colour; nsec[3] (host) = sectors per box edge (of replica 0).  In a batch
 * the order is colour-major across replicas.  Synchronises. */
int sl_get_order(sl_ctx* ctx, int32_t* order_dev, int32_t colour_start[9], int32_t nsec[3]);

/* out[8] (host) = steps done, rebuilds done, largest exchange-list length
 * seen, largest Morse-list length seen, kernel launches per step, 1 if steps
 * run as a captured CUDA graph, 0, 0.  Synchronises. */
int sl_counters(sl_ctx* ctx, int64_t out[8]);

/* Per-phase timing.  With enable = 1, sl_step launches each step's kernels
 * directly (no graph) and records a CUDA event pair on the context's stream
 * around each phase: 0 half-kick, 1 first spin half-op (15 colour passes),
 * 2 drift + rebuild check (+ rebuild), 3 exchange table, 4 second spin
 * half-op, 5 forces (Morse + magneto-elastic) + closing half-kick.
 * sl_get_timing synchronises and returns ms[k] = total milliseconds and
 * count[k] = timed launches of phase k since timing was enabled (entries 6,
 * 7 are 0).  sl_set_timing resets the totals. */
int sl_set_timing(sl_ctx* ctx, int32_t enable);
int sl_get_timing(sl_ctx* ctx, double ms[8], int64_t count[8]);

/* Launch-shape autotuner.  The colour pass comes in SL_SWEEP_VARIANTS tile
 * shapes (sectors per block x threads per block): variants 0-4 a pipelined
 * pass whose spare warps gather the next pass's field while warp 0 turns the
 * in-sector spins (32x192 (variant 0, the default), 32x256, 16x128, 16x128 with
 * registers for 1,024 resident threads per SM, 8x128), variants 5-9 (plain Hamiltonian; with the spin-orbit terms they
 * run as 0-4) a pass that copies every neighbour's spin into shared memory
 * asynchronously first (16x128, 8x64, 32x256, 8x96, 4x64); and the
 * per-atom kernels (kick, drift, exchange table, forces) take 64, 128 (the
 * default) or 256 threads per block.  The shape changes only how the work is
 * grouped into blocks, never the arithmetic of a spin or an atom: results are
 * bitwise the same for every shape.
 * sl_autotune times `steps` timesteps (after one warm-up step) of every
 * combination on the context's own state, restoring the whole workspace from
 * `scratch` (device, >= the workspace's bytes, owned by the caller) before
 * each candidate and at the end, so the state afterwards is bitwise the state
 * before; then it keeps the fastest shape.  With the learned Hamiltonian only
 * the block size is tuned.  out (host, 8): chosen variant, chosen block, its
 * ns per step, the default shape's ns per step, candidates timed, sectors per
 * block of the chosen variant, 0, 0.  Synchronises.
 * Errors: SL_ERR_ARG, SL_ERR_WORKSPACE (scratch too small), SL_ERR_CUDA.
 * sl_set_launch_shape sets a shape directly (SL_ERR_ARG for unknown ones). */
#define SL_SWEEP_VARIANTS 10
int sl_autotune(sl_ctx* ctx, void* scratch, size_t scratch_bytes, int32_t steps, int64_t out[8]);
int sl_set_launch_shape(sl_ctx* ctx, int32_t sweep_variant, int32_t block);

/* Magnetisation of a caller's spin array without a context and without any
 * allocation, for callers that cannot call cudaMalloc (code running inside
 * another allocator's hooks, plugins handed device pointers only, processes
 * whose device footprint is fixed after start-up).  The paper has no
 * counterpart: this is a service entry point of this library.
 *   s        device, [n_atoms][3] doubles (caller order, not modified)
 *   n_atoms  1 .. 2,097,152; larger counts return SL_ERR_ARG before any launch
 *   out      device, 4 doubles: Mx, My, Mz, |M| with M = (1/N) sum_i s_i
 * The block partial sums live in a 256 KB file-scope device array that every
 * GPU loading libsl holds until the process exits; every block writes its own
 * slot, so no part of it has to start at zero.  All calls on a device share
 * that array: calls that overlap on the GPU (concurrent streams, or threads
 * using different streams) race and may return wrong results.  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress,
 * done once per device, with that device current); make that first call
 * before any stream capture.  The address is kept for the life of the
 * process: do not call this after cudaDeviceReset on that device.
 * cuda_stream must belong to the current device (SL_ERR_ARG otherwise,
 * before any launch).  Stream-ordered on cuda_stream; no host sync.
 * Errors: SL_ERR_ARG, SL_ERR_CUDA. */
int sl_magnetization_static(const double* s, int32_t n_atoms, double* out, void* cuda_stream);

/* Measured throughput of the library's double-float multiply-add (the
 * FP64-accurate a*b + c on the FP32 pipes that the pair and rotation kernels
 * are built from) on the current device: the compute roof those kernels are
 * compared with.  The paper has no counterpart: this is a measurement
 * service of the library.  Runs 4 blocks of 256 threads per SM, each thread
 * `iters` (1 .. 2^20) rounds of 8 independent multiply-adds, on a private
 * stream: one warm-up launch, then the best of three timed with CUDA events.
 *   flop_per_s (host) 2 flop per multiply-add / best launch time
 *   ms         (host, may be NULL) that launch's duration
 * Synchronises.  Errors: SL_ERR_ARG, SL_ERR_CUDA. */
int sl_df_fma_rate(int32_t iters, double* flop_per_s, double* ms);

/* The double-float functions of the pair and rotation kernels, evaluated on
 * the device for a check of their accuracy against FP64 (a measurement
 * service of the library; the paper has none): y[k] = f(x[k]) with x[k]
 * rounded to a double-float (~48 bits), f computed in double-float and the
 * result widened back to FP64.
 *   fn   SL_DF_EXP (exp x, used for x in [-12, 6]), SL_DF_RSQRT (1/sqrt x,
 *        x > 0) or SL_DF_SQRT (sqrt x, x >= 0)
 *   x, y device pointers to n doubles (caller-owned; y may not alias x)
 * Stream-ordered on cuda_stream; no host sync.  Errors: SL_ERR_ARG (fn, n
 * or pointers), SL_ERR_CUDA. */
#define SL_DF_EXP 0
#define SL_DF_RSQRT 1
#define SL_DF_SQRT 2
int sl_df_eval(int32_t fn, const double* x, double* y, int64_t n, void* cuda_stream);

/* Check of the library's bounded in-kernel wait (the one the tensor-core
 * kernels use for their MMA completion), on the current device: one thread
 * waits on a shared-memory barrier of count 1 for at most limit_ns
 * nanoseconds (0 .. 2e9) of the GPU's global timer; with arrive = 1 it first
 * arrives itself, so the wait completes, with arrive = 0 nothing ever does.
 * *status (host) receives SL_OK or SL_ERR_TIMEOUT, the code such a wait
 * leaves in a context's sticky status.  The paper has no counterpart: this
 * lets a caller confirm that a wait which never completes ends with an
 * error status, leaving the GPU usable, instead of hanging it.
 * Synchronises.  Errors: SL_ERR_ARG, SL_ERR_CUDA. */
int sl_check_bounded_wait(int64_t limit_ns, int32_t arrive, int32_t* status);

/* ------------------------------------------------------------------------
 * Learned per-atom Hamiltonian.  The paper has no learned model: this is an
 * extension of the library in which a small network stands in for the Morse
 * + exchange energy, so that the same integrator runs on it.
 *
 * Descriptor of atom i over its neighbours j with r_ij < SL_ML_RC:
 *   D_i[3k+m] = sum_j g_k(r_ij) (s_i.s_j)^m,  k = 0..15, m = 0, 1, 2,
 *   g_k(r) = exp(-(r - 0.4k)^2 / (2 * 0.4^2)) (1 + cos(pi r/SL_ML_RC))/2.
 * Network: x = (D - mean) * inv_std,
 *   E_i = w3 . silu(W2 silu(W1 x + b1) + b2) + b3,   silu(z) = z/(1+e^-z);
 * W1, W2, w3 are used rounded to bfloat16 (nearest even), biases as float.
 * E = sum_i E_i replaces the Morse + exchange terms; the Zeeman and kinetic
 * terms are unchanged.  Forces -dE/dr and fields -dE/ds come from the
 * hand-written backward pass (chain rule through D_i and every D_j).
 *
 * The network's GEMMs run on the tensor cores with bfloat16 operands and
 * float32 accumulation; activations are passed as three bfloat16 pieces
 * (hi + mid + lo) so that the products carry float32 precision.
 *
 * Parameters (float32, device): one vector of SL_ML_NPARAM floats, W1[64][48]
 * (row = hidden unit), b1[64], W2[64][64], b2[64], w3[64], b3, at the
 * SL_ML_OFF_* offsets.  Normalisation (float32, device): SL_ML_NNORM floats,
 * mean[48], inv_std[48], gate lo[48], gate hi[48].
 *
 * Dynamics with hamiltonian = SL_HAM_LEARNED: sectors are at least
 * SL_ML_RC + skin wide (the network couples spins up to SL_ML_RC apart) and
 * morse_rc_A must be >= SL_ML_RC (the Morse list is the descriptor list).
 * Each evaluation point (after the drift; with the forces) evaluates the
 * network at the current state.  If any atom's descriptor lies outside
 * [gate lo, gate hi], that point hands over to the analytic Hamiltonian: the
 * following spin half-op and/or forces use Morse + Bethe-Slater instead.
 * A learned spin half-op is time symmetric: a predictor sweep with the field
 * coefficients (P, Q) of the per-atom gradients G_i = dE_i/dD_i at the
 * half-op's start, the coefficients at the predicted end averaged with the
 * start's, and the corrector sweep from the start spins with the averages.
 * Each single-spin factor rotates s_i exactly about omega at the rotation's
 * midpoint m (found by a trial rotation about omega(s_i)), where
 *   omega(s) = (mu_s mu_B H - sum_j (P_ij + 2 Q_ij s.s_j) s_j) / hbar,
 *   P_ij = sum_k (G_i+G_j)[3k+1] g_k(r_ij),  Q_ij = sum_k (G_i+G_j)[3k+2] g_k(r_ij),
 * with the current neighbour spins.  The spin bath (lambda, temperature_K),
 * the Cayley propagator, the spin-orbit terms, the embedding term and the
 * ground-state subtraction are not available in this mode (SL_ERR_ARG).
 * ------------------------------------------------------------------------ */
#define SL_ML_NF 48
#define SL_ML_NH 64
#define SL_ML_RC 6.0
#define SL_ML_OFF_W1 0
#define SL_ML_OFF_B1 3072
#define SL_ML_OFF_W2 3136
#define SL_ML_OFF_B2 7232
#define SL_ML_OFF_W3 7296
#define SL_ML_OFF_B3 7360
#define SL_ML_NPARAM 7361
#define SL_ML_NNORM 192

/* Install a model (device float32 vectors, copied into the workspace) and
 * evaluate it at the current state (forces, fields, gate).  The context must
 * have been created with hamiltonian = SL_HAM_LEARNED (SL_ERR_ARG otherwise).
 * sl_step and the sl_ml_* calls below return SL_ERR_ARG until a model is set.
 * The optimiser state of sl_ml_train_step is reset.  Stream-ordered. */
int sl_ml_set_model(sl_ctx* ctx, const float* params, const float* norm);

/* Copy the current float32 parameters (after training) to params (device,
 * SL_ML_NPARAM floats).  Stream-ordered. */
int sl_ml_get_model(sl_ctx* ctx, float* params);

/* Evaluate the network at the current state, gate ignored.  Outputs, any may
 * be NULL: e_rep (host, [n_replicas]) sum_i E_i per replica; F and B (device,
 * [n][3] doubles, caller order) = -dE/dr (eV/A) and -dE/ds (eV); D (device,
 * [n][48] doubles, caller order) the raw descriptors.  Synchronises when
 * e_rep is given. */
int sl_ml_eval(sl_ctx* ctx, double* e_rep, double* F, double* B, double* D);

/* Statistics of the raw descriptors of the current state over all atoms:
 * out (host, [4][48]) = mean, standard deviation, minimum, maximum per
 * feature, summed in a fixed order.  Synchronises. */
int sl_ml_descriptor_stats(sl_ctx* ctx, double* out);

/* out[4] (host) = atoms outside the gate range at the last evaluation point,
 * 1 if the network was in use there, evaluation points handed to the analytic
 * Hamiltonian so far, 0.  Synchronises. */
int sl_ml_gate(sl_ctx* ctx, int64_t out[4]);

/* Parameter gradient of  sum_r gE[r] E_r + sum_i gF_i . F_i + sum_i gB_i . B_i
 * at the current state (E_r = sum of E_i over replica r; F, B as in
 * sl_ml_eval): the vector-Jacobian product behind both the energy and its
 * derivatives (forward-over-reverse through the network).  gE (device,
 * [n_replicas] doubles), gF, gB (device, [n][3] doubles, caller order) may be
 * NULL (zero).  grad (device, SL_ML_NPARAM doubles) is overwritten.
 * Stream-ordered; the sum over atoms is in a fixed order. */
int sl_ml_vjp(sl_ctx* ctx, const double* gE, const double* gF, const double* gB, double* grad);

/* One training step on the frames currently loaded (one replica per frame):
 *   L = w[0] mean_r (dE_r/N_r)^2 + w[1] (1/N) sum_i |dF_i|^2
 *       + w[2] (1/N) sum_i |(1 - s_i s_i^T) dB_i / hbar|^2,
 * d = network - reference, then one Adam update (Kingma and Ba, 2015) of the
 * float32 parameters with learning rate lr and moments beta1, beta2, eps
 * (moments kept in the workspace in FP64).  E_ref (device, [n_replicas]),
 * F_ref, B_ref (device, [n][3], caller order): reference potential energy
 * (Morse + exchange), forces and field -dE/ds (no Zeeman term).  loss (host,
 * 4 doubles: L and its three terms at the parameters before the update) may
 * be NULL; when given the call synchronises.  The gate is ignored. */
int sl_ml_train_step(sl_ctx* ctx, const double* E_ref, const double* F_ref, const double* B_ref,
                     const double w[3], double lr, double beta1, double beta2, double eps, double* loss);

/* Sticky device error word (SL_OK or SL_ERR_*).  Synchronises. */
int sl_status(sl_ctx* ctx);

/* Static description of an error code (never NULL). */
const char* sl_strerror(int code);

/* Release the context (not the caller's workspace).  Synchronises. */
void sl_destroy(sl_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SL_H */
