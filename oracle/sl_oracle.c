/*
 * Plain FP64 CPU oracle for the coupled spin-lattice timestep of
 * Tranchida, Plimpton, Thibaudeau, Thompson (arXiv 1801.10233).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA library is checked against.  It shares no code,
 * header, table or constant generator with the CUDA path; only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark load it.
 *
 * What it computes, in the paper's order:
 *   Hamiltonian   H = -mu_s mu_B sum_i H.s_i - sum_{i<j} J(r_ij) s_i.s_j
 *                     + sum_i p_i^2/2m + sum_{i<j} V(r_ij)
 *                 (Eq. s_hamiltonian and Eq. sl_hamiltonian, Sec. 2; every
 *                 unordered pair counted once), J(r) the Bethe-Slater form of
 *                 Eq. BSfunction (App. A.1), V(r) a Morse pair potential.
 *   Precession    omega_i = -(1/hbar) dH/ds_i                 (Sec. 2.1)
 *   EOM           dr/dt = p/m, dp/dt = -dH/dr, ds/dt = omega x s
 *                 (Eqs. r_advance, p_advance, s_advance, Sec. 2.2)
 *   Step          e^{Lp dt/2} e^{Ls dt/2} e^{Lr dt} e^{Ls dt/2} e^{Lp dt/2}
 *                 (Eq. general_ST_decomposition, Sec. 3)
 *   Spin half-op  prod_{k=1..N} e^{Ls_k dt/4} prod_{k=N..1} e^{Ls_k dt/4}
 *                 with omega_k recomputed right before each single-spin
 *                 update (Eq. spin_ST_decomposition, Sec. 3), the spins
 *                 numbered by (colour, sector, atom id) as in the sectored
 *                 form Eq. spin_ST_sectoring (Sec. 5.1).
 *   Single spin   exact rotation of s about omega by |omega| tau (default) or
 *                 the Cayley-type propagator printed in Sec. 3 (mode 1).
 *   Thermostat    stochastic precession vector of Eq. sLLG (Sec. 4.1) with
 *                 noise variance 2 D_S / tau per component; lattice bath of
 *                 Eq. p_advance_T (Sec. 4.2): friction -(gamma_L/m) p and a
 *                 white-noise force of strength D_L = 2 m (gamma_L/m) k_B T
 *                 (Einstein relation), integrated as the exact
 *                 Ornstein-Uhlenbeck flow over dt/2 at both ends of the step
 *                 (O B S R S B O).
 *   Spin-orbit    (App. A.2) uniaxial anisotropy -K (s.n)^2, Neel
 *                 pseudo-dipolar -g1(r)((e.s_i)(e.s_j) - s_i.s_j/3) and DMI
 *                 d(r) e_ij.(s_i x s_j) per unordered pair inside the exchange
 *                 cutoff, g1 and d of the form of Eq. BSfunction; the
 *                 anisotropy makes omega_i depend on s_i, so each
 *                 single-spin factor is split symmetrically: an exact half
 *                 turn under the anisotropy alone (it keeps s.n), the turn
 *                 under the rest of omega, another anisotropy half turn.
 *   Embedding     (Sec. 2, Eq. app:mech1) optional Finnis-Sinclair term
 *                 sum_i -A sqrt(rho_i), rho_i = sum_j f(r_ij), and optional
 *                 subtraction of the collinear exchange ground state; or
 *                 (App. B) the tabulated embedded-atom potential: pair term
 *                 phi(r) in place of Morse and embedding F(rho_i), rho_i =
 *                 sum_j rho(r_ij), all three from tables on uniform grids
 *                 through natural cubic splines (sl_eam_tab.c).
 *   Observables   kinetic, Morse, exchange, Zeeman energies; T_L
 *                 (Eq. lattice_temperature), T_S (Eq. spin_temperature),
 *                 magnetisation M = (1/N) sum_i s_i.
 *
 * Learned Hamiltonian mode (hamiltonian = 1; no counterpart in the paper):
 * the Morse + exchange energy is replaced by the per-atom network of
 * sl_learned.c.  Each evaluation point (the start of each spin half-op, the
 * force computation) evaluates the network at the current state; if any
 * atom's descriptor lies outside the model's trained range, that point uses
 * the analytic Hamiltonian instead.  A learned spin half-op is time
 * symmetric:
 *   1. P, Q from the per-atom gradients G at the half-op's start;
 *   2. predictor: the palindromic sweep with those P, Q;
 *   3. P, Q from G at the predicted end state; average them with step 1's;
 *   4. corrector: the sweep again from the start spins with the averages.
 * Each single-spin factor of a sweep rotates s_i exactly about omega_i taken
 * at the rotation's midpoint, omega(s) = (mu_s mu_B H - sum_j (P_ij + 2 Q_ij
 * s.s_j) s_j)/hbar with the current neighbour spins: the midpoint is
 * estimated as m = u/|u|, u = s_i + (tau/2) omega(s_i) x s_i (to second
 * order in the angle, as the rule needs), then s_i rotates about omega(m).
 * (Holding G, or omega during a rotation, fixed at the start of the step
 * makes the energy error first order in dt; the symmetric forms make it
 * second order.)  Sectors are at least the model's 6 A cutoff + skin wide
 * so that same-colour spins still do not interact.
 *
 * Pair lists are rebuilt from scratch at the exact cutoffs whenever the
 * positions change (brute force, or a plain cell list that the tests check
 * against brute force); there is no Verlet skin here.  The skin only enters
 * through the sector assignment, which is redone when an atom has moved more
 * than skin/2 since the last assignment (or on a fixed schedule), because the
 * colour order of the sweep depends on it.
 *
 * Threads (orc_set_threads, default 1): the sweep can turn the sectors of
 * one colour side by side, since they are further apart than every cutoff
 * while no atom has moved more than skin/2 (Sec. 5.1); the pair search, the
 * pair tables and the forces are sums per atom.  Each is split over OpenMP
 * threads without changing any operation or its order, so every thread
 * count gives the serial result bit for bit.  After a skin error the sweep
 * runs serially.
 *
 * Compiled with -ffp-contract=off so that every a*b+c rounds twice, as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "orc_learned.h"
#include "orc_eam_tab.h"

/* Physical constants in the paper's "metal" unit set (A, ps, eV, amu, K, T). */
#define ORC_HBAR 6.582119569e-4   /* eV ps / rad (Sec. 2.1 prints 1e3 too small) */
#define ORC_KB 8.617333262e-5     /* eV / K */
#define ORC_MUB 5.7883818060e-5   /* eV / T */
#define ORC_FTOA 9648.533212      /* (eV/A)/amu -> A/ps^2 */

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_BOX = -3, ORC_ERR_SPIN_NORM = -4,
       ORC_ERR_SKIN = -5, ORC_ERR_OOM = -8 };

typedef struct {
  int32_t n_atoms;
  int32_t rotation;      /* 0 exact (Rodrigues) rotation, 1 Cayley propagator of Sec. 3 */
  int32_t fix_lattice;   /* 1: positions and velocities frozen, spins only */
  int32_t rebuild_every; /* 0: re-sector when max displacement > skin/2; K>0: every K steps */
  int32_t morse_shift;   /* 1: report V(r)-V(rc) in the energy (dynamics unchanged) */
  int32_t brute_force;   /* 1: O(N^2) pair search instead of the cell list */
  double box[3];
  double mass;           /* amu */
  double mu_s;           /* magnetic moment in units of mu_B */
  double H[3];           /* applied field, T */
  double dt;             /* ps */
  double ex_alpha, ex_gamma, ex_delta, ex_rc;   /* Eq. BSfunction */
  double m_D0, m_alpha, m_r0, m_rc;             /* Morse */
  double skin;
  double lambda;         /* transverse damping of Eq. sLLG (0: none) */
  double temperature;    /* spin bath temperature, K (0: no noise) */
  uint64_t seed;
  int32_t replica;
  int32_t hamiltonian;   /* 0 analytic (Morse + Bethe-Slater), 1 learned */
  double lat_gamma;      /* lattice damping rate gamma_L/m of Eq. p_advance_T, 1/ps (0: none) */
  double lat_temperature;/* lattice bath temperature, K */
  /* spin-orbit terms of App. A.2 (all 0: none); g1 and d have the form of
   * Eq. BSfunction and the exchange cutoff */
  double an_K;           /* uniaxial anisotropy K, eV: H_an = -K sum_i (s_i.n)^2 */
  double an_axis[3];     /* unit axis n */
  double neel_alpha, neel_gamma, neel_delta;   /* g1(r): H = -sum_{i<j} g1 ((e.s_i)(e.s_j) - s_i.s_j/3) */
  double dmi_alpha, dmi_gamma, dmi_delta;      /* d(r): H = sum_{i<j} d e_ij.(s_i x s_j), D_ij = d e_ij */
  /* mechanical potential beyond the Morse pairs (App. B; 0: off): an
   * embedding term sum_i F(rho_i), F(rho) = -A sqrt(rho), rho_i = sum_j f(r_ij),
   * f(r) = (r - d)^2 + beta (r - d)^3 / d for r < d (Finnis-Sinclair form), and
   * with ground_sub = 1 the collinear magnetic ground state taken out of the
   * mechanical energy (Eq. app:mech1): + sum_{i<j} J(r_ij) */
  double eam_A, eam_d, eam_beta;
  int32_t ground_sub;
  /* 1: the mechanical potential is the tabulated embedded-atom form of
   * App. B instead of Morse (+ the Finnis-Sinclair term): pair term phi(r),
   * embedding F(rho_i), rho_i = sum_j rho(r_ij), r < m_rc, each from a table on
   * a uniform grid interpolated by a natural cubic spline (orc_set_eam_tables;
   * eam_A must be 0) */
  int32_t eam_tab;
} orc_params;

typedef struct {
  int n;
  int *off;    /* CSR offsets, n+1 */
  int *j;      /* neighbour ids, ascending within each row */
  int cap;
} orc_list;

typedef struct {
  orc_params p;
  int n;
  double *r, *v, *s, *F;   /* [n][3], indexed by atom id */
  double *rb;              /* positions at the last sector assignment */
  int nsec[3];
  double edge[3];
  int *sector;             /* linear sector index per atom */
  int *colour;             /* colour 0..7 per atom */
  int *order;              /* atom ids in sweep order: colour, sector, id */
  int colour_start[9];
  int *run;                /* starts of the sectors' runs in the sweep order, nrun + 1 */
  int nrun;
  int colour_run[9];       /* first run of each colour */
  int threads;             /* > 1: same-colour sectors, atoms and rows split over OpenMP threads */
  orc_list ex, mo;         /* exchange pairs (r < ex_rc), Morse pairs (r < m_rc) */
  double *exJ, *exdJ;      /* J(r_ij), J'(r_ij) per exchange list entry */
  double *exG1, *exDm;     /* g1(r_ij), d(r_ij) per exchange list entry */
  double *exE;             /* e_ij = (r_j - r_i)/r per exchange list entry, [3] */
  long step;               /* completed steps */
  int err;
  int rebuilds;
  orc_eam_tabs tabs;       /* tables of the tabulated embedded-atom potential */
  /* observation points inside a step (orc_set_hook): after each colour's
   * pass of a sweep (event 0, arg = colour) and after the drift (event 1);
   * the decomposition tests exchange halo data there */
  void (*hook)(void* user, int event, int arg);
  void* hook_user;
  /* learned Hamiltonian */
  orc_ml_model* ml;        /* NULL until orc_ml_set_model */
  orc_list mll;            /* pairs with r < ML_RC */
  double *mlP, *mlQ;       /* field coefficients per mll entry (frozen per half-op) */
  int use_ml;              /* the current evaluation point uses the network */
  int gate_bad;            /* out-of-range atoms at the last evaluation point */
  int gate_trips;          /* evaluation points handed to the analytic Hamiltonian */
} orc_state;

/* ------------------------------------------------------------------ */
/* Counter-based generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11).              */
/* ------------------------------------------------------------------ */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
  uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
  uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t n0 = hi1 ^ c[1] ^ k[0];
  uint32_t n2 = hi0 ^ c[3] ^ k[1];
  c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
    philox_round(c, k);
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Three standard normal deviates for (seed, replica, step, sub-pass, atom):
 * Box-Muller on the four 32-bit words, u = (x + 1/2) / 2^32 in (0,1). */
void orc_gauss3(uint64_t seed, int replica, long step, int subpass, int atom, double g[3]) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {(uint32_t)atom, (uint32_t)step, (uint32_t)subpass, (uint32_t)replica};
  uint32_t x[4];
  orc_philox4x32_10(ctr, key, x);
  const double two32 = 4294967296.0;
  const double twopi = 6.283185307179586476925286766559;
  double u0 = ((double)x[0] + 0.5) / two32, u1 = ((double)x[1] + 0.5) / two32;
  double u2 = ((double)x[2] + 0.5) / two32, u3 = ((double)x[3] + 0.5) / two32;
  double ra = sqrt(-2.0 * log(u0)), rb = sqrt(-2.0 * log(u2));
  g[0] = ra * cos(twopi * u1);
  g[1] = ra * sin(twopi * u1);
  g[2] = rb * cos(twopi * u3);
}

/* ------------------------------------------------------------------ */
/* Pair functions                                                      */
/* ------------------------------------------------------------------ */

/* Bethe-Slater exchange, Eq. BSfunction (App. A.1), without the cutoff step. */
static double bs_f(double alpha, double gamma, double delta, double r) {
  double x = (r / delta) * (r / delta);
  return 4.0 * alpha * x * (1.0 - gamma * x) * exp(-x);
}
/* d/dr of the same expression. */
static double bs_df(double alpha, double gamma, double delta, double r) {
  double x = (r / delta) * (r / delta);
  double dxdr = 2.0 * r / (delta * delta);
  /* d/dx [x (1 - g x) e^{-x}] = e^{-x} (1 - 2 g x - x + g x^2) */
  return 4.0 * alpha * exp(-x) * (1.0 - 2.0 * gamma * x - x + gamma * x * x) * dxdr;
}
static double bs_J(const orc_params* p, double r) { return bs_f(p->ex_alpha, p->ex_gamma, p->ex_delta, r); }
static double bs_dJ(const orc_params* p, double r) { return bs_df(p->ex_alpha, p->ex_gamma, p->ex_delta, r); }
static int has_neel(const orc_params* p) { return p->neel_alpha != 0.0; }
static int has_dmi(const orc_params* p) { return p->dmi_alpha != 0.0; }
/* Morse pair energy V(r) = D0 (e^{-2a(r-r0)} - 2 e^{-a(r-r0)}). */
static double morse_V(const orc_params* p, double r) {
  double e = exp(-p->m_alpha * (r - p->m_r0));
  return p->m_D0 * (e * e - 2.0 * e);
}
/* dV/dr. */
static double morse_dV(const orc_params* p, double r) {
  double e = exp(-p->m_alpha * (r - p->m_r0));
  return p->m_D0 * (-2.0 * p->m_alpha * e * e + 2.0 * p->m_alpha * e);
}
/* Embedding term: density contribution f(r), f'(r) (r < d), F(rho), F'(rho). */
static double eam_f(const orc_params* p, double r) {
  double x = r - p->eam_d;
  return r < p->eam_d ? x * x + p->eam_beta * x * x * x / p->eam_d : 0.0;
}
static double eam_df(const orc_params* p, double r) {
  double x = r - p->eam_d;
  return r < p->eam_d ? 2.0 * x + 3.0 * p->eam_beta * x * x / p->eam_d : 0.0;
}
static double eam_F(const orc_params* p, double rho) { return rho > 0.0 ? -p->eam_A * sqrt(rho) : 0.0; }
static double eam_dF(const orc_params* p, double rho) { return rho > 0.0 ? -0.5 * p->eam_A / sqrt(rho) : 0.0; }

/* The mechanical potential in either form (r < m_rc): pair term V(r) and
 * dV/dr -- Morse, or phi(r) from its table -- and embedding F(rho) with the
 * density contribution f(r) -- Finnis-Sinclair, or F(rho) and rho(r) from
 * their tables.  Tables that are not set yet (T NULL or not ready) count as
 * zero functions. */
static int tab_on(const orc_params* p, const orc_eam_tabs* T) { return p->eam_tab && T && T->ready; }
static int has_embed(const orc_params* p) { return p->eam_A != 0.0 || p->eam_tab; }
static double mech_V(const orc_params* p, const orc_eam_tabs* T, double r, double* dVdr) {
  if (p->eam_tab) {
    if (!tab_on(p, T)) { if (dVdr) *dVdr = 0.0; return 0.0; }
    return orc_spline_value(&T->phi, r, dVdr);
  }
  if (dVdr) *dVdr = morse_dV(p, r);
  return morse_V(p, r);
}
static double embed_f(const orc_params* p, const orc_eam_tabs* T, double r, double* dfdr) {
  if (p->eam_tab) {
    if (!tab_on(p, T)) { if (dfdr) *dfdr = 0.0; return 0.0; }
    return orc_spline_value(&T->rho, r, dfdr);
  }
  if (dfdr) *dfdr = eam_df(p, r);
  return eam_f(p, r);
}
static double embed_F(const orc_params* p, const orc_eam_tabs* T, double rho, double* dFdrho) {
  if (p->eam_tab) {
    if (!tab_on(p, T)) { if (dFdrho) *dFdrho = 0.0; return 0.0; }
    return orc_spline_value(&T->F, rho, dFdrho);
  }
  if (dFdrho) *dFdrho = eam_dF(p, rho);
  return eam_F(p, rho);
}
/* The energy shift of each pair term: V(m_rc) with morse_shift (Morse only). */
static double pair_shift(const orc_params* p) { return p->morse_shift && !p->eam_tab ? morse_V(p, p->m_rc) : 0.0; }

/* Minimum-image separation d = r_j - r_i. */
static void min_image(const orc_state* st, int i, int j, double d[3]) {
  for (int a = 0; a < 3; ++a) {
    double L = st->p.box[a];
    double x = st->r[3 * j + a] - st->r[3 * i + a];
    d[a] = x - L * nearbyint(x / L);
  }
}

static double wrap1(double x, double L) { return x - L * floor(x / L); }

/* ------------------------------------------------------------------ */
/* Pair search at an exact cutoff                                      */
/* ------------------------------------------------------------------ */
static int cmp_int(const void* a, const void* b) {
  int x = *(const int*)a, y = *(const int*)b;
  return (x > y) - (x < y);
}

static int list_push(orc_list* L, int* cnt, int j) {
  if (*cnt >= L->cap) {
    int nc = L->cap ? 2 * L->cap : 1024;
    int* nj = (int*)realloc(L->j, (size_t)nc * sizeof(int));
    if (!nj) return ORC_ERR_OOM;
    L->j = nj; L->cap = nc;
  }
  L->j[(*cnt)++] = j;
  return ORC_OK;
}

static int list_reserve(orc_list* L, int need) {
  if (need <= L->cap) return ORC_OK;
  int nc = L->cap ? L->cap : 1024;
  while (nc < need) nc *= 2;
  int* nj = (int*)realloc(L->j, (size_t)nc * sizeof(int));
  if (!nj) return ORC_ERR_OOM;
  L->j = nj; L->cap = nc;
  return ORC_OK;
}

typedef struct {
  int nx, ny, nz;
  const int *head, *next, *cellof;   /* chained cell lists, cell of each atom */
} cell_grid;

/* Row i of the list from the 27 cells around atom i: with pop given, only a
 * bound (the atoms in those cells); else the number of j != i within the
 * cutoff, written to out (sorted by j) when out is not NULL. */
static int cell_row(const orc_state* st, const cell_grid* g, int i, double rc2, const int* pop, int* out) {
  int m = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int x = (g->cellof[3 * i] + dx + g->nx) % g->nx;
        int y = (g->cellof[3 * i + 1] + dy + g->ny) % g->ny;
        int z = (g->cellof[3 * i + 2] + dz + g->nz) % g->nz;
        int c = x + g->nx * (y + g->ny * z);
        if (pop) { m += pop[c]; continue; }
        for (int j = g->head[c]; j >= 0; j = g->next[j]) {
          if (j == i) continue;
          double d[3];
          min_image(st, i, j, d);
          if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < rc2) {
            if (out) out[m] = j;
            m += 1;
          }
        }
      }
  if (out) qsort(out, (size_t)m, sizeof(int), cmp_int);
  return m;
}

/* All j != i with |min_image(r_j - r_i)| < rc, rows sorted by j. */
static int build_list(orc_state* st, double rc, orc_list* L) {
  int n = st->n;
  double rc2 = rc * rc;
  if (!L->off) { L->off = (int*)malloc((size_t)(n + 1) * sizeof(int)); if (!L->off) return ORC_ERR_OOM; }
  int cnt = 0;
  int nc[3];
  int use_cells = !st->p.brute_force;
  for (int a = 0; a < 3; ++a) {
    nc[a] = (int)floor(st->p.box[a] / rc);
    if (nc[a] < 3) use_cells = 0;
  }
  if (!use_cells) {
    for (int i = 0; i < n; ++i) {
      L->off[i] = cnt;
      for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        double d[3];
        min_image(st, i, j, d);
        if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < rc2)
          if (list_push(L, &cnt, j)) return ORC_ERR_OOM;
      }
    }
    L->off[n] = cnt;
    return ORC_OK;
  }
  /* cell list: cell edge >= rc, at least 3 cells per dimension */
  int ncell = nc[0] * nc[1] * nc[2];
  int* head = (int*)malloc((size_t)ncell * sizeof(int));
  int* pop = (int*)calloc((size_t)ncell, sizeof(int));
  int* next = (int*)malloc((size_t)n * sizeof(int));
  int* cellof = (int*)malloc((size_t)n * 3 * sizeof(int));
  if (!head || !pop || !next || !cellof) { free(head); free(pop); free(next); free(cellof); return ORC_ERR_OOM; }
  for (int c = 0; c < ncell; ++c) head[c] = -1;
  for (int i = n - 1; i >= 0; --i) {
    int cc[3];
    for (int a = 0; a < 3; ++a) {
      double L_ = st->p.box[a];
      int k = (int)floor(wrap1(st->r[3 * i + a], L_) / (L_ / nc[a]));
      if (k < 0) k = 0;
      if (k >= nc[a]) k = nc[a] - 1;
      cc[a] = k;
      cellof[3 * i + a] = k;
    }
    int c = cc[0] + nc[0] * (cc[1] + nc[1] * cc[2]);
    next[i] = head[c];
    head[c] = i;
    pop[c] += 1;
  }
  const cell_grid g = {nc[0], nc[1], nc[2], head, next, cellof};
  int e = ORC_OK;
  if (st->threads <= 1) {
    for (int i = 0; i < n; ++i) {
      L->off[i] = cnt;
      if (list_reserve(L, cnt + cell_row(st, &g, i, rc2, pop, NULL))) { e = ORC_ERR_OOM; break; }
      cnt += cell_row(st, &g, i, rc2, NULL, L->j + cnt);
    }
  } else {
    /* the same rows, counted in one parallel pass and written in a second */
    int nt = st->threads;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 256)
    for (int i = 0; i < n; ++i) L->off[i + 1] = cell_row(st, &g, i, rc2, NULL, NULL);
    L->off[0] = 0;
    for (int i = 0; i < n; ++i) L->off[i + 1] += L->off[i];
    cnt = L->off[n];
    if (list_reserve(L, cnt)) e = ORC_ERR_OOM;
    if (!e) {
#pragma omp parallel for num_threads(nt) schedule(dynamic, 256)
      for (int i = 0; i < n; ++i) cell_row(st, &g, i, rc2, NULL, L->j + L->off[i]);
    }
  }
  L->off[n] = cnt;
  free(head); free(pop); free(next); free(cellof);
  return e;
}

/* Pair lists and the exchange coefficients at the current positions
 * (J is recomputed after every drift, Sec. 3). */
static int refresh_pairs(orc_state* st) {
  int e = build_list(st, st->p.ex_rc, &st->ex);
  if (e) return e;
  e = build_list(st, st->p.m_rc, &st->mo);
  if (e) return e;
  if (st->p.hamiltonian == 1) {
    e = build_list(st, ML_RC, &st->mll);
    if (e) return e;
  }
  int np = st->ex.off[st->n];
  free(st->exJ); free(st->exdJ); free(st->exG1); free(st->exDm); free(st->exE);
  st->exJ = (double*)malloc((size_t)(np ? np : 1) * sizeof(double));
  st->exdJ = (double*)malloc((size_t)(np ? np : 1) * sizeof(double));
  st->exG1 = (double*)malloc((size_t)(np ? np : 1) * sizeof(double));
  st->exDm = (double*)malloc((size_t)(np ? np : 1) * sizeof(double));
  st->exE = (double*)malloc((size_t)(np ? np : 1) * 3 * sizeof(double));
  if (!st->exJ || !st->exdJ || !st->exG1 || !st->exDm || !st->exE) return ORC_ERR_OOM;
  int nt = st->threads > 1 ? st->threads : 1;
#pragma omp parallel for num_threads(nt) schedule(static) if (nt > 1)
  for (int i = 0; i < st->n; ++i)
    for (int k = st->ex.off[i]; k < st->ex.off[i + 1]; ++k) {
      double d[3];
      min_image(st, i, st->ex.j[k], d);
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      st->exJ[k] = bs_J(&st->p, r);
      st->exdJ[k] = bs_dJ(&st->p, r);
      st->exG1[k] = has_neel(&st->p) ? bs_f(st->p.neel_alpha, st->p.neel_gamma, st->p.neel_delta, r) : 0.0;
      st->exDm[k] = has_dmi(&st->p) ? bs_f(st->p.dmi_alpha, st->p.dmi_gamma, st->p.dmi_delta, r) : 0.0;
      for (int a = 0; a < 3; ++a) st->exE[3 * k + a] = d[a] / r;
    }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Sector assignment (Sec. 5.1) and the sweep order                   */
/* ------------------------------------------------------------------ */
/* The largest even number of sectors per edge whose edge exceeds the reach
 * of a spin's interactions plus the skin, by a relative margin of 1e-6: atoms
 * of two sectors of one colour stay further apart than the reach while none
 * has moved more than skin/2, with room to spare for a list built from
 * rounded distances. */
static int sector_grid(const orc_params* p, int nsec[3], double edge[3]) {
  double reach = p->ex_rc;
  if (p->hamiltonian == 1 && ML_RC > reach) reach = ML_RC;
  double w = (reach + p->skin) * (1.0 + 1e-6);
  for (int a = 0; a < 3; ++a) {
    int n = (int)floor(p->box[a] / w);
    if (n % 2) n -= 1;
    if (n < 2) return ORC_ERR_BOX;
    nsec[a] = n;
    edge[a] = p->box[a] / (double)n;
  }
  return ORC_OK;
}

typedef struct { int colour, sector, id; } orc_key;
static int cmp_key(const void* a, const void* b) {
  const orc_key* x = (const orc_key*)a; const orc_key* y = (const orc_key*)b;
  if (x->colour != y->colour) return x->colour < y->colour ? -1 : 1;
  if (x->sector != y->sector) return x->sector < y->sector ? -1 : 1;
  return (x->id > y->id) - (x->id < y->id);
}

/* Wrap positions into the box, assign each atom to its sector and colour,
 * order the atoms by (colour, sector, id), remember the positions. */
static int assign_sectors(orc_state* st) {
  int n = st->n;
  orc_key* keys = (orc_key*)malloc((size_t)(n ? n : 1) * sizeof(orc_key));
  if (!keys) return ORC_ERR_OOM;
  for (int i = 0; i < n; ++i) {
    int sx[3];
    for (int a = 0; a < 3; ++a) {
      double x = wrap1(st->r[3 * i + a], st->p.box[a]);
      st->r[3 * i + a] = x;
      int k = (int)floor(x / st->edge[a]);
      if (k < 0) k = 0;
      if (k >= st->nsec[a]) k = st->nsec[a] - 1;
      sx[a] = k;
    }
    st->sector[i] = sx[0] + st->nsec[0] * (sx[1] + st->nsec[1] * sx[2]);
    st->colour[i] = (sx[0] & 1) + 2 * (sx[1] & 1) + 4 * (sx[2] & 1);
    keys[i].colour = st->colour[i];
    keys[i].sector = st->sector[i];
    keys[i].id = i;
  }
  qsort(keys, (size_t)n, sizeof(orc_key), cmp_key);
  for (int c = 0; c <= 8; ++c) st->colour_start[c] = n;
  for (int k = n - 1; k >= 0; --k) {
    st->order[k] = keys[k].id;
    st->colour_start[keys[k].colour] = k;
  }
  for (int c = 7; c >= 0; --c)
    if (st->colour_start[c] > st->colour_start[c + 1]) st->colour_start[c] = st->colour_start[c + 1];
  /* the sweep order holds each sector as one run of consecutive entries */
  st->nrun = 0;
  for (int c = 0; c < 8; ++c) {
    st->colour_run[c] = st->nrun;
    for (int k = st->colour_start[c]; k < st->colour_start[c + 1]; ++k)
      if (k == st->colour_start[c] || st->sector[st->order[k]] != st->sector[st->order[k - 1]])
        st->run[st->nrun++] = k;
  }
  st->colour_run[8] = st->nrun;
  st->run[st->nrun] = n;
  memcpy(st->rb, st->r, (size_t)n * 3 * sizeof(double));
  free(keys);
  st->rebuilds += 1;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Precession vector and single-spin propagators                      */
/* ------------------------------------------------------------------ */

/* The part of omega_i that does not depend on s_i itself:
 * (1/hbar) (mu_s mu_B H + sum_j [J_ij s_j + g1 ((e.s_j) e - s_j/3) + d e x s_j]). */
static void omega_fixed(const orc_state* st, int i, double w[3]) {
  double zf = st->p.mu_s * ORC_MUB;
  double h[3] = {zf * st->p.H[0], zf * st->p.H[1], zf * st->p.H[2]};
  for (int k = st->ex.off[i]; k < st->ex.off[i + 1]; ++k) {
    const double* sj = st->s + 3 * st->ex.j[k];
    h[0] += st->exJ[k] * sj[0];
    h[1] += st->exJ[k] * sj[1];
    h[2] += st->exJ[k] * sj[2];
    const double* e = st->exE + 3 * k;
    if (has_neel(&st->p)) {
      double g = st->exG1[k], es = e[0] * sj[0] + e[1] * sj[1] + e[2] * sj[2];
      for (int a = 0; a < 3; ++a) h[a] += g * (es * e[a] - sj[a] / 3.0);
    }
    if (has_dmi(&st->p)) {
      double dm = st->exDm[k];
      h[0] += dm * (e[1] * sj[2] - e[2] * sj[1]);
      h[1] += dm * (e[2] * sj[0] - e[0] * sj[2]);
      h[2] += dm * (e[0] * sj[1] - e[1] * sj[0]);
    }
  }
  w[0] = h[0] / ORC_HBAR; w[1] = h[1] / ORC_HBAR; w[2] = h[2] / ORC_HBAR;
}

/* Uniaxial anisotropy part of omega at spin s: (2K/hbar) (s.n) n. */
static void omega_aniso(const orc_params* p, const double* s, double w[3]) {
  double c = 2.0 * p->an_K / ORC_HBAR * (s[0] * p->an_axis[0] + s[1] * p->an_axis[1] + s[2] * p->an_axis[2]);
  w[0] = c * p->an_axis[0]; w[1] = c * p->an_axis[1]; w[2] = c * p->an_axis[2];
}

/* omega_i = -(1/hbar) dH/ds_i at the current state. */
static void omega_of(const orc_state* st, int i, double w[3]) {
  omega_fixed(st, i, w);
  if (st->p.an_K != 0.0) {
    double a[3];
    omega_aniso(&st->p, st->s + 3 * i, a);
    w[0] += a[0]; w[1] += a[1]; w[2] += a[2];
  }
}

/* Learned-mode precession vector from the frozen pair coefficients:
 * omega_i = (mu_s mu_B H - sum_j (P_ij + 2 Q_ij s_i.s_j) s_j) / hbar. */
static void omega_ml_at(const orc_state* st, int i, const double* si, double w[3]) {
  double zf = st->p.mu_s * ORC_MUB;
  double h[3] = {zf * st->p.H[0], zf * st->p.H[1], zf * st->p.H[2]};
  for (int k = st->mll.off[i]; k < st->mll.off[i + 1]; ++k) {
    const double* sj = st->s + 3 * st->mll.j[k];
    double c = si[0] * sj[0] + si[1] * sj[1] + si[2] * sj[2];
    double psi = st->mlP[k] + 2.0 * st->mlQ[k] * c;
    h[0] -= psi * sj[0];
    h[1] -= psi * sj[1];
    h[2] -= psi * sj[2];
  }
  w[0] = h[0] / ORC_HBAR; w[1] = h[1] / ORC_HBAR; w[2] = h[2] / ORC_HBAR;
}

static void cross(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

/* s rotated exactly about w by |w| tau (Rodrigues), into out. */
static void rodrigues(const double w[3], const double* s, double tau, double out[3]) {
  double wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  double th = wn * tau;
  if (wn == 0.0 || th == 0.0) { out[0] = s[0]; out[1] = s[1]; out[2] = s[2]; return; }
  double nv[3] = {w[0] / wn, w[1] / wn, w[2] / wn};
  double c = cos(th), sn = sin(th), h = sin(0.5 * th);
  double omc = 2.0 * h * h;
  double nxs[3];
  cross(nv, s, nxs);
  double ns = nv[0] * s[0] + nv[1] * s[1] + nv[2] * s[2];
  for (int a = 0; a < 3; ++a) out[a] = s[a] * c + nxs[a] * sn + nv[a] * ns * omc;
}

/* Learned single-spin factor: exact rotation about omega at the midpoint. */
static void rotate_ml(orc_state* st, int i, double tau) {
  double* s = st->s + 3 * i;
  double w[3], wxs[3], m[3];
  omega_ml_at(st, i, s, w);
  cross(w, s, wxs);
  for (int a = 0; a < 3; ++a) m[a] = s[a] + 0.5 * tau * wxs[a];
  double mn = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
  for (int a = 0; a < 3; ++a) m[a] /= mn;
  omega_ml_at(st, i, m, w);
  double out[3];
  rodrigues(w, s, tau, out);
  s[0] = out[0]; s[1] = out[1]; s[2] = out[2];
}

/* s turned about w over time tau with the configured propagator: the exact
 * rotation by |w| tau (Rodrigues) or the Cayley-type form of Sec. 3. */
static void turn(const orc_params* p, const double w[3], double* s, double tau) {
  double out[3];
  if (p->rotation == 0) {
    rodrigues(w, s, tau, out);
  } else {
    double wxs[3];
    cross(w, s, wxs);
    double w2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double ws = w[0] * s[0] + w[1] * s[1] + w[2] * s[2];
    double q = tau * tau / 4.0;
    double den = 1.0 + q * w2;
    for (int a = 0; a < 3; ++a) out[a] = (s[a] + tau * wxs[a] + q * (2.0 * w[a] * ws - w2 * s[a])) / den;
  }
  s[0] = out[0]; s[1] = out[1]; s[2] = out[2];
}

/* Update spin i over time tau (one factor e^{L_si tau} of Eq. spin_ST_decomposition).
 * With uniaxial anisotropy the factor is itself split symmetrically: half a
 * turn under the anisotropy alone, a full turn under the field of the
 * neighbours and H, another anisotropy half turn.  The anisotropy precession
 * vector (2K/hbar)(s.n) n keeps s.n fixed, so each half turn is the exact
 * flow of that term and is undone exactly by the reversed step. */
static void rotate(orc_state* st, int i, double tau, int subpass) {
  if (st->use_ml) { rotate_ml(st, i, tau); return; }
  const orc_params* p = &st->p;
  double* s = st->s + 3 * i;
  int langevin = p->lambda != 0.0 || p->temperature != 0.0;
  double lam = p->lambda, den = 1.0 + lam * lam;
  double a[3];
  if (p->an_K != 0.0) {
    omega_aniso(p, s, a);
    if (langevin) for (int q = 0; q < 3; ++q) a[q] /= den;
    turn(p, a, s, 0.5 * tau);
  }
  double w[3];
  omega_fixed(st, i, w);
  if (langevin) {
    /* Eq. sLLG written as ds/dt = Om x s with
     * Om = (omega + eta + lambda s x omega) / (1 + lambda^2);
     * eta ~ N(0, 2 D_S / |tau|) per component, D_S = lambda (1+lambda^2) k_B T / hbar.
     * The damping term takes the whole omega, anisotropy included. */
    double eta[3] = {0, 0, 0};
    if (p->temperature > 0.0) {
      double g[3];
      orc_gauss3(p->seed, p->replica, st->step, subpass, i, g);
      double DS = lam * (1.0 + lam * lam) * ORC_KB * p->temperature / ORC_HBAR;
      double sig = sqrt(2.0 * DS / fabs(tau));
      eta[0] = sig * g[0]; eta[1] = sig * g[1]; eta[2] = sig * g[2];
    }
    double wt[3] = {w[0], w[1], w[2]};
    if (p->an_K != 0.0) {
      omega_aniso(p, s, a);
      for (int q = 0; q < 3; ++q) wt[q] += a[q];
    }
    double sxw[3];
    cross(s, wt, sxw);
    for (int q = 0; q < 3; ++q) w[q] = (w[q] + eta[q] + lam * sxw[q]) / den;
  }
  turn(p, w, s, tau);
  if (p->an_K != 0.0) {
    omega_aniso(p, s, a);
    if (langevin) for (int q = 0; q < 3; ++q) a[q] /= den;
    turn(p, a, s, 0.5 * tau);
  }
}

/* One evaluation point of the learned Hamiltonian at the current state:
 * sets use_ml (gate), the frozen field coefficients and, if F is given, the
 * learned forces.  Returns an error code. */
static int ml_point(orc_state* st, double* F) {
  st->use_ml = 0;
  if (st->p.hamiltonian != 1) return ORC_OK;
  if (!st->ml) return ORC_ERR_ARG;
  int np = st->mll.off[st->n];
  free(st->mlP); free(st->mlQ);
  st->mlP = (double*)malloc((size_t)(np ? np : 1) * sizeof(double));
  st->mlQ = (double*)malloc((size_t)(np ? np : 1) * sizeof(double));
  if (!st->mlP || !st->mlQ) return ORC_ERR_OOM;
  int bad = orc_ml_frame(st->n, st->r, st->s, st->p.box, st->mll.off, st->mll.j, st->ml, NULL, NULL, NULL, F,
                         NULL, st->mlP, st->mlQ);
  if (bad < 0) return ORC_ERR_OOM;
  st->gate_bad = bad;
  st->use_ml = bad == 0;
  if (bad) st->gate_trips += 1;
  return ORC_OK;
}

/* The palindromic sweep: forward over the sweep order with h/2 per spin, then backward. */
static void call_hook(orc_state* st, int event, int arg) {
  if (st->hook) st->hook(st->hook_user, event, arg);
}

static void sweep(orc_state* st, double h, int subpass0) {
  if (st->threads <= 1 || st->err != ORC_OK) {
    /* the order is colour-major: colour c's atoms are entries
     * colour_start[c] .. colour_start[c+1]-1, forward then backward */
    for (int c = 0; c < 8; ++c) {
      for (int k = st->colour_start[c]; k < st->colour_start[c + 1]; ++k) rotate(st, st->order[k], 0.5 * h, subpass0);
      call_hook(st, 0, c);
    }
    for (int c = 7; c >= 0; --c) {
      for (int k = st->colour_start[c + 1] - 1; k >= st->colour_start[c]; --k)
        rotate(st, st->order[k], 0.5 * h, subpass0 + 1);
      call_hook(st, 0, c);
    }
    return;
  }
  /* The same order with the sectors of one colour side by side: while every
   * atom stays within skin/2 of where the sectors were assigned, atoms of two
   * sectors of one colour are further apart than every cutoff (Sec. 5.1), so
   * no rotation reads a spin that another sector of its colour turns. */
  int nt = st->threads;
  for (int c = 0; c < 8; ++c) {
#pragma omp parallel for num_threads(nt) schedule(dynamic, 16)
    for (int q = st->colour_run[c]; q < st->colour_run[c + 1]; ++q)
      for (int k = st->run[q]; k < st->run[q + 1]; ++k) rotate(st, st->order[k], 0.5 * h, subpass0);
    call_hook(st, 0, c);
  }
  for (int c = 7; c >= 0; --c) {
#pragma omp parallel for num_threads(nt) schedule(dynamic, 16)
    for (int q = st->colour_run[c]; q < st->colour_run[c + 1]; ++q)
      for (int k = st->run[q + 1] - 1; k >= st->run[q]; --k) rotate(st, st->order[k], 0.5 * h, subpass0 + 1);
    call_hook(st, 0, c);
  }
}

/* e^{L_s h}.  Learned Hamiltonian: predictor sweep, field coefficients at the
 * predicted end averaged with the start's, corrector sweep from the start. */
static void spin_half_op(orc_state* st, double h, int subpass0) {
  if (st->p.hamiltonian != 1) { sweep(st, h, subpass0); return; }
  int e = ml_point(st, NULL);
  if (e) { if (st->err == ORC_OK) st->err = e; return; }
  if (!st->use_ml) { sweep(st, h, subpass0); return; }
  int n = st->n, np = st->mll.off[n];
  double* P0 = (double*)malloc((size_t)(np ? np : 1) * sizeof(double));
  double* Q0 = (double*)malloc((size_t)(np ? np : 1) * sizeof(double));
  double* s0 = (double*)malloc((size_t)(n ? n : 1) * 3 * sizeof(double));
  if (!P0 || !Q0 || !s0) { free(P0); free(Q0); free(s0); if (st->err == ORC_OK) st->err = ORC_ERR_OOM; return; }
  memcpy(P0, st->mlP, (size_t)np * sizeof(double));
  memcpy(Q0, st->mlQ, (size_t)np * sizeof(double));
  memcpy(s0, st->s, (size_t)n * 3 * sizeof(double));
  sweep(st, h, subpass0);                                   /* predictor */
  double* P1 = st->mlP;
  double* Q1 = st->mlQ;
  st->mlP = NULL; st->mlQ = NULL;
  free(P1); free(Q1);
  int use = st->use_ml;
  int gb = st->gate_bad, gt = st->gate_trips;
  e = ml_point(st, NULL);                                   /* G at the predicted end (gate ignored) */
  st->use_ml = use; st->gate_bad = gb; st->gate_trips = gt;
  if (e) { if (st->err == ORC_OK) st->err = e; free(P0); free(Q0); free(s0); return; }
  for (int k = 0; k < np; ++k) {
    st->mlP[k] = 0.5 * (P0[k] + st->mlP[k]);
    st->mlQ[k] = 0.5 * (Q0[k] + st->mlQ[k]);
  }
  memcpy(st->s, s0, (size_t)n * 3 * sizeof(double));
  sweep(st, h, subpass0);                                   /* corrector */
  free(P0); free(Q0); free(s0);
}

/* ------------------------------------------------------------------ */
/* Forces (Eq. p_advance derived from the energy)                     */
/* ------------------------------------------------------------------ */
/* Embedding density of atom i from the Morse list (eam_d <= m_rc). */
static double eam_rho(const orc_state* st, int i) {
  double rho = 0.0;
  for (int k = st->mo.off[i]; k < st->mo.off[i + 1]; ++k) {
    double d[3];
    min_image(st, i, st->mo.j[k], d);
    rho += embed_f(&st->p, &st->tabs, sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]), NULL);
  }
  return rho;
}

static void compute_forces(orc_state* st) {
  int n = st->n;
  if (st->p.hamiltonian == 1 && st->ml) {
    double* F = (double*)malloc((size_t)(n ? n : 1) * 3 * sizeof(double));
    int e = F ? ml_point(st, F) : ORC_ERR_OOM;
    if (e) {
      if (st->err == ORC_OK) st->err = e;
    } else if (st->use_ml) {
      memcpy(st->F, F, (size_t)n * 3 * sizeof(double));
      free(F);
      return;
    }
    free(F);
  }
  memset(st->F, 0, (size_t)n * 3 * sizeof(double));
  int nt = st->threads > 1 ? st->threads : 1;   /* each atom's sum is its own: any split gives the same F */
#pragma omp parallel for num_threads(nt) schedule(static) if (nt > 1)
  for (int i = 0; i < n; ++i) {
    double* f = st->F + 3 * i;
    for (int k = st->mo.off[i]; k < st->mo.off[i + 1]; ++k) {
      double d[3];
      min_image(st, i, st->mo.j[k], d);
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      double dv;
      mech_V(&st->p, &st->tabs, r, &dv);
      double c = dv / r;                        /* F_i += V'(r) (r_j - r_i)/r */
      f[0] += c * d[0]; f[1] += c * d[1]; f[2] += c * d[2];
    }
    const double* si = st->s + 3 * i;
    for (int k = st->ex.off[i]; k < st->ex.off[i + 1]; ++k) {
      int j = st->ex.j[k];
      double d[3];
      min_image(st, i, j, d);
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      const double* sj = st->s + 3 * j;
      double sij = si[0] * sj[0] + si[1] * sj[1] + si[2] * sj[2];
      /* F_i -= J'(r) s_i.s_j (r_j - r_i)/r; the ground-state subtraction
       * + J(r) adds J'(r) (r_j - r_i)/r */
      double c = -st->exdJ[k] * (st->p.ground_sub ? sij - 1.0 : sij) / r;
      f[0] += c * d[0]; f[1] += c * d[1]; f[2] += c * d[2];
      const double* e = st->exE + 3 * k;
      if (has_neel(&st->p)) {
        /* U = -g1(r) Q, Q = (e.s_i)(e.s_j) - s_i.s_j/3; de/dr_i = -(1 - e e^T)/r:
         * F_i = -g1' Q e - (g1/r) (dQ/de - e (e.dQ/de)), dQ/de = (e.s_j) s_i + (e.s_i) s_j */
        double g = st->exG1[k], gp = bs_df(st->p.neel_alpha, st->p.neel_gamma, st->p.neel_delta, r);
        double a = e[0] * sj[0] + e[1] * sj[1] + e[2] * sj[2];
        double b = e[0] * si[0] + e[1] * si[1] + e[2] * si[2];
        double Q = a * b - sij / 3.0;
        for (int q = 0; q < 3; ++q) {
          double dq = a * si[q] + b * sj[q];
          f[q] += -gp * Q * e[q] - g / r * (dq - e[q] * 2.0 * a * b);
        }
      }
      if (has_dmi(&st->p)) {
        /* W = d(r) e.X, X = s_i x s_j: F_i = d' (e.X) e + (d/r) (X - e (e.X)) */
        double dm = st->exDm[k], dp = bs_df(st->p.dmi_alpha, st->p.dmi_gamma, st->p.dmi_delta, r);
        double X[3];
        cross(si, sj, X);
        double eX = e[0] * X[0] + e[1] * X[1] + e[2] * X[2];
        for (int q = 0; q < 3; ++q) f[q] += dp * eX * e[q] + dm / r * (X[q] - e[q] * eX);
      }
    }
  }
  if (has_embed(&st->p)) {
    /* E = sum_i F(rho_i): F_i = sum_j (F'(rho_i) + F'(rho_j)) f'(r) (r_j - r_i)/r */
    double* dF = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!dF) { if (st->err == ORC_OK) st->err = ORC_ERR_OOM; return; }
#pragma omp parallel for num_threads(nt) schedule(static) if (nt > 1)
    for (int i = 0; i < n; ++i) embed_F(&st->p, &st->tabs, eam_rho(st, i), dF + i);
#pragma omp parallel for num_threads(nt) schedule(static) if (nt > 1)
    for (int i = 0; i < n; ++i) {
      double* f = st->F + 3 * i;
      for (int k = st->mo.off[i]; k < st->mo.off[i + 1]; ++k) {
        int j = st->mo.j[k];
        double d[3];
        min_image(st, i, j, d);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double df;
        embed_f(&st->p, &st->tabs, r, &df);
        double c = (dF[i] + dF[j]) * df / r;
        f[0] += c * d[0]; f[1] += c * d[1]; f[2] += c * d[2];
      }
    }
    free(dF);
  }
}

static void kick(orc_state* st, double h) {
  double c = h * ORC_FTOA / st->p.mass;
  for (int k = 0; k < 3 * st->n; ++k) st->v[k] += c * st->F[k];
}

/* Exact flow of the lattice bath over time |h| (Eq. p_advance_T without the
 * conservative force): v <- v e^{-g|h|} + sqrt((1 - e^{-2g|h|}) k_B T/m) xi,
 * xi ~ N(0, 1) per component from Philox (seed; atom, step, subpass, replica). */
static void lattice_bath(orc_state* st, double h, int subpass) {
  double g = st->p.lat_gamma;
  if (!(g > 0.0)) return;
  double c1 = exp(-g * fabs(h));
  double sig = sqrt((1.0 - c1 * c1) * ORC_KB * st->p.lat_temperature * ORC_FTOA / st->p.mass);
  for (int i = 0; i < st->n; ++i) {
    double xi[3] = {0.0, 0.0, 0.0};
    if (st->p.lat_temperature > 0.0) orc_gauss3(st->p.seed, st->p.replica, st->step, subpass, i, xi);
    for (int a = 0; a < 3; ++a) st->v[3 * i + a] = c1 * st->v[3 * i + a] + sig * xi[a];
  }
}

static double max_disp2(const orc_state* st) {
  double m = 0.0;
  for (int i = 0; i < st->n; ++i) {
    double d0 = st->r[3 * i] - st->rb[3 * i];
    double d1 = st->r[3 * i + 1] - st->rb[3 * i + 1];
    double d2 = st->r[3 * i + 2] - st->rb[3 * i + 2];
    double q = d0 * d0 + d1 * d1 + d2 * d2;
    if (q > m) m = q;
  }
  return m;
}

/* ------------------------------------------------------------------ */
/* Public interface                                                    */
/* ------------------------------------------------------------------ */
void orc_destroy(orc_state* st) {
  if (!st) return;
  free(st->r); free(st->v); free(st->s); free(st->F); free(st->rb);
  free(st->sector); free(st->colour); free(st->order); free(st->run);
  free(st->ex.off); free(st->ex.j); free(st->mo.off); free(st->mo.j);
  free(st->exJ); free(st->exdJ); free(st->exG1); free(st->exDm); free(st->exE);
  free(st->ml); free(st->mll.off); free(st->mll.j); free(st->mlP); free(st->mlQ);
  orc_spline_free(&st->tabs.F); orc_spline_free(&st->tabs.rho); orc_spline_free(&st->tabs.phi);
  free(st);
}

int orc_params_size(void) { return (int)sizeof(orc_params); }

static int set_threads(orc_state* st, int threads) {
#ifdef _OPENMP
  st->threads = threads > 1 ? threads : 1;
#else
  (void)threads;
  st->threads = 1;
#endif
  return st->threads;
}

/* r, v, s: [n][3] in atom-id order; threads as for orc_set_threads (the
 * initial lists and forces use them too).  Returns NULL and sets *err on
 * failure. */
orc_state* orc_create_threads(const orc_params* p, const double* r, const double* v, const double* s, int threads,
                              int* err) {
  *err = ORC_OK;
  if (!p || p->n_atoms < 0 || p->mass <= 0.0 || p->hamiltonian < 0 || p->hamiltonian > 1 ||
      (p->hamiltonian == 1 && p->rotation != 0) || !(p->lat_gamma >= 0.0) || !(p->lat_temperature >= 0.0) ||
      (p->an_K != 0.0 && !(fabs(p->an_axis[0] * p->an_axis[0] + p->an_axis[1] * p->an_axis[1] +
                                p->an_axis[2] * p->an_axis[2] - 1.0) <= 1e-12)) ||
      (p->eam_A != 0.0 && !(p->eam_d > 0.0 && p->eam_d <= p->m_rc)) ||
      ((p->eam_A != 0.0 || p->ground_sub || p->eam_tab) && p->hamiltonian != 0) ||
      (p->eam_tab != 0 && p->eam_tab != 1) || (p->eam_tab && p->eam_A != 0.0)) {
    *err = ORC_ERR_ARG;
    return NULL;
  }
  double reach = p->m_rc > p->ex_rc ? p->m_rc : p->ex_rc;
  if (p->hamiltonian == 1 && ML_RC > reach) reach = ML_RC;
  double need = 2.0 * (reach + p->skin);
  for (int a = 0; a < 3; ++a)
    if (!(p->box[a] >= need)) { *err = ORC_ERR_BOX; return NULL; }
  orc_state* st = (orc_state*)calloc(1, sizeof(orc_state));
  if (!st) { *err = ORC_ERR_OOM; return NULL; }
  st->p = *p;
  int n = p->n_atoms;
  st->n = n;
  size_t b3 = (size_t)(n ? n : 1) * 3 * sizeof(double);
  st->r = (double*)malloc(b3); st->v = (double*)malloc(b3); st->s = (double*)malloc(b3);
  st->F = (double*)malloc(b3); st->rb = (double*)malloc(b3);
  st->sector = (int*)malloc((size_t)(n ? n : 1) * sizeof(int));
  st->colour = (int*)malloc((size_t)(n ? n : 1) * sizeof(int));
  st->order = (int*)malloc((size_t)(n ? n : 1) * sizeof(int));
  st->run = (int*)malloc((size_t)(n + 1) * sizeof(int));
  set_threads(st, threads);
  if (!st->r || !st->v || !st->s || !st->F || !st->rb || !st->sector || !st->colour || !st->order || !st->run) {
    orc_destroy(st); *err = ORC_ERR_OOM; return NULL;
  }
  memcpy(st->r, r, (size_t)n * 3 * sizeof(double));
  memcpy(st->v, v, (size_t)n * 3 * sizeof(double));
  memcpy(st->s, s, (size_t)n * 3 * sizeof(double));
  for (int i = 0; i < n; ++i) {
    const double* si = s + 3 * i;
    double nn = sqrt(si[0] * si[0] + si[1] * si[1] + si[2] * si[2]);
    if (!(fabs(nn - 1.0) <= 1e-12)) { orc_destroy(st); *err = ORC_ERR_SPIN_NORM; return NULL; }
  }
  int e = sector_grid(p, st->nsec, st->edge);
  if (!e) e = assign_sectors(st);
  if (!e) e = refresh_pairs(st);
  if (e) { orc_destroy(st); *err = e; return NULL; }
  compute_forces(st);
  return st;
}

orc_state* orc_create(const orc_params* p, const double* r, const double* v, const double* s, int* err) {
  return orc_create_threads(p, r, v, s, 1, err);
}

/* Install the learned model (float params[ML_NPARAM], norm[ML_NNORM]) and
 * recompute the forces with it.  Only for hamiltonian = 1. */
int orc_ml_set_model(orc_state* st, const float* params, const float* norm) {
  if (st->p.hamiltonian != 1) return ORC_ERR_ARG;
  if (!st->ml) st->ml = (orc_ml_model*)malloc(sizeof(orc_ml_model));
  if (!st->ml) return ORC_ERR_OOM;
  orc_ml_load(params, norm, st->ml);
  compute_forces(st);
  return st->err;
}

/* Out-of-range atoms at the last learned evaluation point, and the number
 * of points handed to the analytic Hamiltonian so far. */
void orc_ml_gate(const orc_state* st, int out[2]) {
  out[0] = st->gate_bad;
  out[1] = st->gate_trips;
}

/* One or more timesteps of Eq. general_ST_decomposition. */
int orc_step(orc_state* st, int nsteps) {
  if (st->p.hamiltonian == 1 && !st->ml) return ORC_ERR_ARG;
  if (st->p.eam_tab && !st->tabs.ready) return ORC_ERR_ARG;
  for (int it = 0; it < nsteps; ++it) {
    double dt = st->p.dt;
    int lat = !st->p.fix_lattice;
    if (lat) {
      lattice_bath(st, 0.5 * dt, 4);
      kick(st, 0.5 * dt);
    }
    spin_half_op(st, 0.5 * dt, 0);
    if (lat) {
      for (int k = 0; k < 3 * st->n; ++k) st->r[k] += dt * st->v[k];
      call_hook(st, 1, 0);
      double h = 0.5 * st->p.skin;
      double md2 = max_disp2(st);
      int resector;
      if (st->p.rebuild_every > 0) {
        resector = ((st->step + 1) % st->p.rebuild_every) == 0;
        if (!resector && md2 > h * h && st->err == ORC_OK) st->err = ORC_ERR_SKIN;
      } else {
        resector = md2 > h * h;
      }
      if (resector) {
        int e = assign_sectors(st);
        if (e) return e;
      }
      int e = refresh_pairs(st);
      if (e) return e;
    }
    spin_half_op(st, 0.5 * dt, 2);
    if (lat) {
      compute_forces(st);
      kick(st, 0.5 * dt);
      lattice_bath(st, 0.5 * dt, 5);
    }
    st->step += 1;
  }
  return st->err;
}

void orc_set_dt(orc_state* st, double dt) { st->p.dt = dt; }

/* Observation points (see orc_state.hook); NULL removes them. */
void orc_set_hook(orc_state* st, void (*fn)(void* user, int event, int arg), void* user) {
  st->hook = fn;
  st->hook_user = user;
}

/* Overwrite positions and/or spins (NULL: keep) of m atoms given by id. */
void orc_set_atoms(orc_state* st, int m, const int* ids, const double* r, const double* s) {
  for (int q = 0; q < m; ++q) {
    int i = ids[q];
    if (i < 0 || i >= st->n) continue;
    for (int a = 0; a < 3; ++a) {
      if (r) st->r[3 * i + a] = r[3 * q + a];
      if (s) st->s[3 * i + a] = s[3 * q + a];
    }
  }
}

void orc_get_state(const orc_state* st, double* r, double* v, double* s) {
  size_t b = (size_t)st->n * 3 * sizeof(double);
  if (r) memcpy(r, st->r, b);
  if (v) memcpy(v, st->v, b);
  if (s) memcpy(s, st->s, b);
}

void orc_get_forces(const orc_state* st, double* F) {
  memcpy(F, st->F, (size_t)st->n * 3 * sizeof(double));
}

/* Learned energy per atom and field B = -dE/ds at the current state (exact
 * gradient, nothing frozen).  Returns 1 if the network is in effect there
 * (model set, every descriptor in range), 0 otherwise, -1 on failure. */
static int ml_current(const orc_state* st, double* e_atom, double* B) {
  if (st->p.hamiltonian != 1 || !st->ml) return 0;
  int bad = orc_ml_frame(st->n, st->r, st->s, st->p.box, st->mll.off, st->mll.j, st->ml, e_atom, NULL, NULL, NULL,
                         B, NULL, NULL);
  if (bad < 0) return -1;
  return bad == 0;
}

/* omega_i of the current state, [n][3], rad/ps (no noise, no damping):
 * -(1/hbar) dH/ds_i of the Hamiltonian in effect. */
void orc_get_omega(const orc_state* st, double* w) {
  int n = st->n;
  double* B = (double*)malloc((size_t)(n ? n : 1) * 3 * sizeof(double));
  if (B && ml_current(st, NULL, B) == 1) {
    double zf = st->p.mu_s * ORC_MUB;
    for (int i = 0; i < n; ++i)
      for (int a = 0; a < 3; ++a) w[3 * i + a] = (B[3 * i + a] + zf * st->p.H[a]) / ORC_HBAR;
    free(B);
    return;
  }
  free(B);
  for (int i = 0; i < n; ++i) omega_of(st, i, w + 3 * i);
}

/* Sweep order, colour boundaries, per-atom sector and colour, sector grid. */
void orc_get_order(const orc_state* st, int* order, int* colour_start, int* sector, int* colour, int* nsec) {
  if (order) memcpy(order, st->order, (size_t)st->n * sizeof(int));
  if (colour_start) memcpy(colour_start, st->colour_start, 9 * sizeof(int));
  if (sector) memcpy(sector, st->sector, (size_t)st->n * sizeof(int));
  if (colour) memcpy(colour, st->colour, (size_t)st->n * sizeof(int));
  if (nsec) { nsec[0] = st->nsec[0]; nsec[1] = st->nsec[1]; nsec[2] = st->nsec[2]; }
}

long orc_get_step(const orc_state* st) { return st->step; }
int orc_get_rebuilds(const orc_state* st) { return st->rebuilds; }

/* Threads for the sweep, the pair search, the pair tables and the forces
 * (default 1).  Every split gives results bit-identical to one thread.
 * Returns the number used: 1 when built without OpenMP. */
int orc_set_threads(orc_state* st, int threads) { return set_threads(st, threads); }
int orc_get_error(const orc_state* st) { return st->err; }
int orc_count_pairs(const orc_state* st, int which) {
  return which == 0 ? st->ex.off[st->n] : st->mo.off[st->n];
}

/* out[0..7] = E_kin, E_morse, E_exch, E_zeeman, E_total (eV), T_L, T_S (K),
 * E_spin-orbit (anisotropy + Neel + DMI, eV; included in E_total).
 * Where the learned Hamiltonian is in effect, out[1] is its energy sum_i E_i
 * (lattice + exchange together) and out[2] = 0. */
void orc_energy(const orc_state* st, double out[8]) {
  int n = st->n;
  double ek = 0.0, em = 0.0, ex = 0.0, ez = 0.0;
  double* eat = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
  double* B = (double*)malloc((size_t)(n ? n : 1) * 3 * sizeof(double));
  int learned = (eat && B) ? ml_current(st, eat, B) == 1 : 0;
  for (int i = 0; i < n; ++i) {
    const double* v = st->v + 3 * i;
    ek += 0.5 * st->p.mass * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / ORC_FTOA;
  }
  double vshift = pair_shift(&st->p);
  if (learned) {
    for (int i = 0; i < n; ++i) em += eat[i];
  } else {
  for (int i = 0; i < n; ++i)
    for (int k = st->mo.off[i]; k < st->mo.off[i + 1]; ++k) {
      int j = st->mo.j[k];
      if (j <= i) continue;
      double d[3];
      min_image(st, i, j, d);
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      em += mech_V(&st->p, &st->tabs, r, NULL) - vshift;
    }
  for (int i = 0; i < n; ++i)
    for (int k = st->ex.off[i]; k < st->ex.off[i + 1]; ++k) {
      int j = st->ex.j[k];
      if (j <= i) continue;
      const double* si = st->s + 3 * i;
      const double* sj = st->s + 3 * j;
      ex -= st->exJ[k] * (si[0] * sj[0] + si[1] * sj[1] + si[2] * sj[2]);
      if (st->p.ground_sub) em += st->exJ[k];
    }
  if (has_embed(&st->p))
    for (int i = 0; i < n; ++i) em += embed_F(&st->p, &st->tabs, eam_rho(st, i), NULL);
  }
  double zf = st->p.mu_s * ORC_MUB;
  for (int i = 0; i < n; ++i) {
    const double* si = st->s + 3 * i;
    ez -= zf * (st->p.H[0] * si[0] + st->p.H[1] * si[1] + st->p.H[2] * si[2]);
  }
  /* spin-orbit terms: anisotropy per site, Neel and DMI per unordered pair */
  double eo = 0.0;
  if (!learned) {
    for (int i = 0; i < n; ++i) {
      const double* si = st->s + 3 * i;
      double sn = si[0] * st->p.an_axis[0] + si[1] * st->p.an_axis[1] + si[2] * st->p.an_axis[2];
      eo -= st->p.an_K * sn * sn;
      for (int k = st->ex.off[i]; k < st->ex.off[i + 1]; ++k) {
        int j = st->ex.j[k];
        if (j <= i) continue;
        const double* sj = st->s + 3 * j;
        const double* e = st->exE + 3 * k;
        double sij = si[0] * sj[0] + si[1] * sj[1] + si[2] * sj[2];
        if (has_neel(&st->p)) {
          double a = e[0] * sj[0] + e[1] * sj[1] + e[2] * sj[2], b = e[0] * si[0] + e[1] * si[1] + e[2] * si[2];
          eo -= st->exG1[k] * (a * b - sij / 3.0);
        }
        if (has_dmi(&st->p)) {
          double X[3];
          cross(si, sj, X);
          eo += st->exDm[k] * (e[0] * X[0] + e[1] * X[1] + e[2] * X[2]);
        }
      }
    }
  }
  double num = 0.0, den = 0.0;
  for (int i = 0; i < n; ++i) {
    double w[3], c[3];
    if (learned) {
      for (int a = 0; a < 3; ++a) w[a] = (B[3 * i + a] + zf * st->p.H[a]) / ORC_HBAR;
    } else {
      omega_of(st, i, w);
    }
    const double* si = st->s + 3 * i;
    cross(si, w, c);
    num += c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    den += si[0] * w[0] + si[1] * w[1] + si[2] * w[2];
  }
  out[0] = ek; out[1] = em; out[2] = ex; out[3] = ez;
  out[4] = ek + em + ex + ez + eo;
  out[5] = n > 0 ? 2.0 * ek / (3.0 * n * ORC_KB) : 0.0;
  out[6] = den != 0.0 ? ORC_HBAR / (2.0 * ORC_KB) * num / den : 0.0;
  out[7] = eo;
  free(eat); free(B);
}

/* out = Mx, My, Mz, |M| with M = (1/N) sum_i s_i. */
void orc_magnetization(const orc_state* st, double out[4]) {
  double m[3] = {0, 0, 0};
  for (int i = 0; i < st->n; ++i)
    for (int a = 0; a < 3; ++a) m[a] += st->s[3 * i + a];
  double inv = st->n > 0 ? 1.0 / st->n : 0.0;
  out[0] = m[0] * inv; out[1] = m[1] * inv; out[2] = m[2] * inv;
  out[3] = sqrt(out[0] * out[0] + out[1] * out[1] + out[2] * out[2]);
}

/* Energy of arbitrary (r, s) without building a state: used by the
 * finite-difference tests.  Same definitions as orc_energy (potential part
 * only: out[1..3]).  Brute-force pairs. */
static int potential_energy(const orc_params* p, const orc_eam_tabs* T, const double* r, const double* s,
                            double out[5]) {
  orc_params q = *p;
  q.brute_force = 1;
  int n = q.n_atoms;
  double em = 0.0, ex = 0.0, ez = 0.0, eo = 0.0;
  double vshift = pair_shift(&q);
  double* rho = (double*)calloc((size_t)(n ? n : 1), sizeof(double));
  if (!rho) return ORC_ERR_OOM;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double d[3];
      for (int a = 0; a < 3; ++a) {
        double x = r[3 * j + a] - r[3 * i + a];
        d[a] = x - q.box[a] * nearbyint(x / q.box[a]);
      }
      double rr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      if (rr < q.m_rc) em += mech_V(&q, T, rr, NULL) - vshift;
      if (rr < q.m_rc && has_embed(&q)) {
        rho[i] += embed_f(&q, T, rr, NULL);
        rho[j] += embed_f(&q, T, rr, NULL);
      }
      if (rr < q.ex_rc) {
        const double* si = s + 3 * i;
        const double* sj = s + 3 * j;
        double sij = si[0] * sj[0] + si[1] * sj[1] + si[2] * sj[2];
        ex -= bs_J(&q, rr) * sij;
        if (q.ground_sub) em += bs_J(&q, rr);
        double e[3] = {d[0] / rr, d[1] / rr, d[2] / rr};
        if (has_neel(&q)) {
          double a = e[0] * sj[0] + e[1] * sj[1] + e[2] * sj[2], b = e[0] * si[0] + e[1] * si[1] + e[2] * si[2];
          eo -= bs_f(q.neel_alpha, q.neel_gamma, q.neel_delta, rr) * (a * b - sij / 3.0);
        }
        if (has_dmi(&q)) {
          double X[3] = {si[1] * sj[2] - si[2] * sj[1], si[2] * sj[0] - si[0] * sj[2], si[0] * sj[1] - si[1] * sj[0]};
          eo += bs_f(q.dmi_alpha, q.dmi_gamma, q.dmi_delta, rr) * (e[0] * X[0] + e[1] * X[1] + e[2] * X[2]);
        }
      }
    }
  double zf = q.mu_s * ORC_MUB;
  for (int i = 0; i < n; ++i) {
    ez -= zf * (q.H[0] * s[3 * i] + q.H[1] * s[3 * i + 1] + q.H[2] * s[3 * i + 2]);
    double sn = s[3 * i] * q.an_axis[0] + s[3 * i + 1] * q.an_axis[1] + s[3 * i + 2] * q.an_axis[2];
    eo -= q.an_K * sn * sn;
  }
  if (has_embed(&q))
    for (int i = 0; i < n; ++i) em += embed_F(&q, T, rho[i], NULL);
  free(rho);
  out[0] = em; out[1] = ex; out[2] = ez; out[3] = em + ex + ez + eo; out[4] = eo;
  return ORC_OK;
}

int orc_potential_energy(const orc_params* p, const double* r, const double* s, double out[5]) {
  return potential_energy(p, NULL, r, s, out);
}

/* The same with a state's parameters and tables (tabulated embedded-atom
 * potential), for arbitrary positions and spins of its n atoms. */
int orc_potential_energy_state(const orc_state* st, const double* r, const double* s, double out[5]) {
  return potential_energy(&st->p, &st->tabs, r, s, out);
}

/* Tables of the tabulated embedded-atom potential (App. B): F on the grid
 * rho = k drho (nrho points), rho(r) and phi(r) on r = k dr (nr points, the
 * grid reaching m_rc); natural cubic splines through them.  Recomputes the
 * forces. */
int orc_set_eam_tables(orc_state* st, int nrho, double drho, const double* F, int nr, double dr, const double* rho,
                       const double* phi) {
  if (!st->p.eam_tab || nrho < 2 || nr < 2 || !(drho > 0.0) || !(dr > 0.0) || !((nr - 1) * dr >= st->p.m_rc))
    return ORC_ERR_ARG;
  orc_eam_tabs T;
  T.ready = 0;
  int e = orc_spline_build(&T.F, nrho, drho, F);
  if (!e) e = orc_spline_build(&T.rho, nr, dr, rho);
  if (!e) e = orc_spline_build(&T.phi, nr, dr, phi);
  if (e) {
    orc_spline_free(&T.F); orc_spline_free(&T.rho); orc_spline_free(&T.phi);
    return e == -8 ? ORC_ERR_OOM : ORC_ERR_ARG;
  }
  orc_spline_free(&st->tabs.F); orc_spline_free(&st->tabs.rho); orc_spline_free(&st->tabs.phi);
  st->tabs = T;
  st->tabs.ready = 1;
  compute_forces(st);
  return st->err;
}
