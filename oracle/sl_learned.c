/*
 * Plain FP64 CPU oracle of the learned per-atom Hamiltonian.
 *
 * TEST INFRASTRUCTURE ONLY.  The paper has no learned model: this is the
 * definition the CUDA kernels are checked against, written as plainly as the
 * definition reads.  Its gradients are pinned by finite differences of its
 * own energy and loss (parity with the paper is unpinned: there is nothing in
 * the paper to pin it to).
 *
 * Model (one atom i, neighbours j with r_ij < rc = 6 A):
 *   D_i[3k+m] = sum_j g_k(r_ij) (s_i.s_j)^m,      k = 0..15, m = 0, 1, 2
 *   g_k(r)    = exp(-(r - 0.4 k)^2 / (2 0.4^2)) fc(r),  fc(r) = (1 + cos(pi r/rc))/2
 *   x_i       = (D_i - mean) * inv_std
 *   E_i       = w3 . silu(W2 silu(W1 x_i + b1) + b2) + b3,  silu(z) = z/(1+e^-z)
 *   E         = sum_i E_i        (stands in for the Morse + exchange energy)
 * W1, W2 and w3 take their values rounded to bfloat16 (round to nearest,
 * ties to even, on the float32 bit pattern); biases and the normalisation
 * are float32 values.  Forces F_i = -dE/dr_i and field B_i = -dE/ds_i by the
 * chain rule through both D_i and the neighbours' D_j.
 *
 * Compiled with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "orc_learned.h"

#define ML_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* bfloat16: the upper 16 bits of a float32, rounded to nearest even   */
/* ------------------------------------------------------------------ */
static double bf16_value(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return (double)x;  /* inf / nan unchanged */
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7FFFu + lsb;
  u &= 0xFFFF0000u;
  float y;
  memcpy(&y, &u, 4);
  return (double)y;
}

double orc_bf16_value(float x) { return bf16_value(x); }

void orc_ml_load(const float* params, const float* norm, orc_ml_model* m) {
  for (int o = 0; o < ML_NH; ++o)
    for (int i = 0; i < ML_NF; ++i) m->W1[o][i] = bf16_value(params[ML_OFF_W1 + o * ML_NF + i]);
  for (int o = 0; o < ML_NH; ++o)
    for (int i = 0; i < ML_NH; ++i) m->W2[o][i] = bf16_value(params[ML_OFF_W2 + o * ML_NH + i]);
  for (int o = 0; o < ML_NH; ++o) {
    m->b1[o] = params[ML_OFF_B1 + o];
    m->b2[o] = params[ML_OFF_B2 + o];
    m->w3[o] = bf16_value(params[ML_OFF_W3 + o]);
  }
  m->b3 = params[ML_OFF_B3];
  for (int f = 0; f < ML_NF; ++f) {
    m->mean[f] = norm[f];
    m->istd[f] = norm[ML_NF + f];
    m->lo[f] = norm[2 * ML_NF + f];
    m->hi[f] = norm[3 * ML_NF + f];
  }
}

/* ------------------------------------------------------------------ */
/* Radial basis and activation                                         */
/* ------------------------------------------------------------------ */
static void basis(double r, double g[ML_NK], double dg[ML_NK]) {
  double a = ML_PI * r / ML_RC;
  double fc = 0.5 * (1.0 + cos(a));
  double dfc = -0.5 * (ML_PI / ML_RC) * sin(a);
  double s2 = ML_SIGMA * ML_SIGMA;
  for (int k = 0; k < ML_NK; ++k) {
    double d = r - ML_DMU * k;
    double e = exp(-d * d / (2.0 * s2));
    g[k] = e * fc;
    if (dg) dg[k] = e * (-d / s2) * fc + e * dfc;
  }
}

static double sigm(double z) { return 1.0 / (1.0 + exp(-z)); }
static double silu(double z) { return z * sigm(z); }
static double dsilu(double z) { double q = sigm(z); return q * (1.0 + z * (1.0 - q)); }
static double d2silu(double z) { double q = sigm(z); return q * (1.0 - q) * (2.0 + z * (1.0 - 2.0 * q)); }

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void sep(const double* r, const double box[3], int i, int j, double d[3]) {
  for (int a = 0; a < 3; ++a) {
    double x = r[3 * j + a] - r[3 * i + a];
    d[a] = x - box[a] * nearbyint(x / box[a]);
  }
}

/* ------------------------------------------------------------------ */
/* Per-atom network                                                    */
/* ------------------------------------------------------------------ */
typedef struct {
  double z1[ML_NH], h1[ML_NH], z2[ML_NH], h2[ML_NH];
} act_t;

static double net_forward(const orc_ml_model* m, const double x[ML_NF], act_t* A) {
  for (int o = 0; o < ML_NH; ++o) {
    double a = 0.0;
    for (int i = 0; i < ML_NF; ++i) a += m->W1[o][i] * x[i];
    A->z1[o] = a + m->b1[o];
    A->h1[o] = silu(A->z1[o]);
  }
  double e = 0.0;
  for (int o = 0; o < ML_NH; ++o) {
    double a = 0.0;
    for (int i = 0; i < ML_NH; ++i) a += m->W2[o][i] * A->h1[i];
    A->z2[o] = a + m->b2[o];
    A->h2[o] = silu(A->z2[o]);
    e += m->w3[o] * A->h2[o];
  }
  return e + m->b3;
}

/* dE_i/dx_i */
static void net_backward(const orc_ml_model* m, const act_t* A, double gx[ML_NF]) {
  double g2[ML_NH], g1[ML_NH];
  for (int o = 0; o < ML_NH; ++o) g2[o] = m->w3[o] * dsilu(A->z2[o]);
  for (int i = 0; i < ML_NH; ++i) {
    double a = 0.0;
    for (int o = 0; o < ML_NH; ++o) a += m->W2[o][i] * g2[o];
    g1[i] = a * dsilu(A->z1[i]);
  }
  for (int f = 0; f < ML_NF; ++f) {
    double a = 0.0;
    for (int o = 0; o < ML_NH; ++o) a += m->W1[o][f] * g1[o];
    gx[f] = a;
  }
}

/* Gradient, with respect to the parameters, of  alpha E_i(x) + u . dE_i/dx
 * (the second term is the directional derivative of E_i along u), added to
 * grad[ML_NPARAM].  Forward pass, its tangent along u, then reverse mode
 * through both. */
static void net_param_grad(const orc_ml_model* m, const double x[ML_NF], const double u[ML_NF], double alpha,
                           double* grad) {
  double z1[ML_NH], h1[ML_NH], t1[ML_NH], p1[ML_NH];
  double z2[ML_NH], h2[ML_NH], t2[ML_NH], p2[ML_NH];
  for (int o = 0; o < ML_NH; ++o) {
    double a = 0.0, t = 0.0;
    for (int i = 0; i < ML_NF; ++i) { a += m->W1[o][i] * x[i]; t += m->W1[o][i] * u[i]; }
    z1[o] = a + m->b1[o];
    h1[o] = silu(z1[o]);
    t1[o] = t;
    p1[o] = dsilu(z1[o]) * t;
  }
  for (int o = 0; o < ML_NH; ++o) {
    double a = 0.0, t = 0.0;
    for (int i = 0; i < ML_NH; ++i) { a += m->W2[o][i] * h1[i]; t += m->W2[o][i] * p1[i]; }
    z2[o] = a + m->b2[o];
    h2[o] = silu(z2[o]);
    t2[o] = t;
    p2[o] = dsilu(z2[o]) * t;
  }
  /* output layer: J = alpha (w3.h2 + b3) + w3.p2 */
  double zb2[ML_NH], tb2[ML_NH];
  for (int o = 0; o < ML_NH; ++o) {
    grad[ML_OFF_W3 + o] += alpha * h2[o] + p2[o];
    double hb = alpha * m->w3[o], pb = m->w3[o];
    tb2[o] = dsilu(z2[o]) * pb;
    zb2[o] = dsilu(z2[o]) * hb + d2silu(z2[o]) * t2[o] * pb;
    grad[ML_OFF_B2 + o] += zb2[o];
    for (int i = 0; i < ML_NH; ++i) grad[ML_OFF_W2 + o * ML_NH + i] += zb2[o] * h1[i] + tb2[o] * p1[i];
  }
  grad[ML_OFF_B3] += alpha;
  for (int i = 0; i < ML_NH; ++i) {
    double hb = 0.0, pb = 0.0;
    for (int o = 0; o < ML_NH; ++o) { hb += m->W2[o][i] * zb2[o]; pb += m->W2[o][i] * tb2[o]; }
    double tb1 = dsilu(z1[i]) * pb;
    double zb1 = dsilu(z1[i]) * hb + d2silu(z1[i]) * t1[i] * pb;
    grad[ML_OFF_B1 + i] += zb1;
    for (int f = 0; f < ML_NF; ++f) grad[ML_OFF_W1 + i * ML_NF + f] += zb1 * x[f] + tb1 * u[f];
  }
}

/* ------------------------------------------------------------------ */
/* Descriptors, energy and gradients of one frame                      */
/* ------------------------------------------------------------------ */
static void descriptor(int i, const double* r, const double* s, const double box[3], const int* off, const int* jl,
                       double D[ML_NF]) {
  memset(D, 0, ML_NF * sizeof(double));
  for (int k = off[i]; k < off[i + 1]; ++k) {
    int j = jl[k];
    double d[3], g[ML_NK];
    sep(r, box, i, j, d);
    double rr = sqrt(dot3(d, d));
    if (!(rr < ML_RC)) continue;
    double c = dot3(s + 3 * i, s + 3 * j);
    basis(rr, g, NULL);
    for (int q = 0; q < ML_NK; ++q) {
      D[3 * q] += g[q];
      D[3 * q + 1] += g[q] * c;
      D[3 * q + 2] += g[q] * c * c;
    }
  }
}

static void normalise(const orc_ml_model* m, const double D[ML_NF], double x[ML_NF]) {
  for (int f = 0; f < ML_NF; ++f) x[f] = (D[f] - m->mean[f]) * m->istd[f];
}

int orc_ml_frame(int n, const double* r, const double* s, const double box[3], const int* off, const int* jl,
                 const orc_ml_model* m, double* e_atom, double* Dout, double* Gout, double* F, double* B, double* P,
                 double* Q) {
  double* D = (double*)malloc((size_t)(n ? n : 1) * ML_NF * sizeof(double));
  double* G = (double*)malloc((size_t)(n ? n : 1) * ML_NF * sizeof(double));
  if (!D || !G) { free(D); free(G); return -1; }
  int out_of_range = 0;
  for (int i = 0; i < n; ++i) {
    double* Di = D + (size_t)i * ML_NF;
    descriptor(i, r, s, box, off, jl, Di);
    int bad = 0;
    for (int f = 0; f < ML_NF; ++f)
      if (!(Di[f] >= m->lo[f] && Di[f] <= m->hi[f])) bad = 1;
    out_of_range += bad;
    double x[ML_NF], gx[ML_NF];
    act_t A;
    normalise(m, Di, x);
    double e = net_forward(m, x, &A);
    if (e_atom) e_atom[i] = e;
    net_backward(m, &A, gx);
    for (int f = 0; f < ML_NF; ++f) G[(size_t)i * ML_NF + f] = gx[f] * m->istd[f];   /* dE_i/dD_i */
  }
  /* pair terms: dE/dr_ij = phi_ij, field coefficients P_ij, Q_ij */
  for (int i = 0; i < n; ++i) {
    double f3[3] = {0, 0, 0}, b3[3] = {0, 0, 0};
    const double* si = s + 3 * i;
    for (int k = off[i]; k < off[i + 1]; ++k) {
      int j = jl[k];
      double d[3], g[ML_NK], dg[ML_NK];
      sep(r, box, i, j, d);
      double rr = sqrt(dot3(d, d));
      if (!(rr < ML_RC)) {
        if (P) P[k] = 0.0;
        if (Q) Q[k] = 0.0;
        continue;
      }
      const double* sj = s + 3 * j;
      double c = dot3(si, sj);
      basis(rr, g, dg);
      const double* Gi = G + (size_t)i * ML_NF;
      const double* Gj = G + (size_t)j * ML_NF;
      double phi = 0.0, pp = 0.0, qq = 0.0;
      for (int q = 0; q < ML_NK; ++q) {
        double s0 = Gi[3 * q] + Gj[3 * q];
        double s1 = Gi[3 * q + 1] + Gj[3 * q + 1];
        double s2 = Gi[3 * q + 2] + Gj[3 * q + 2];
        phi += (s0 + s1 * c + s2 * c * c) * dg[q];
        pp += s1 * g[q];
        qq += s2 * g[q];
      }
      /* F_i = -dE/dr_i = sum_j phi_ij e_ij, e_ij = (r_j - r_i)/r */
      for (int a = 0; a < 3; ++a) f3[a] += phi * d[a] / rr;
      /* B_i = -dE/ds_i = -sum_j (P_ij + 2 Q_ij c_ij) s_j */
      double psi = pp + 2.0 * qq * c;
      for (int a = 0; a < 3; ++a) b3[a] -= psi * sj[a];
      if (P) P[k] = pp;
      if (Q) Q[k] = qq;
    }
    if (F) for (int a = 0; a < 3; ++a) F[3 * i + a] = f3[a];
    if (B) for (int a = 0; a < 3; ++a) B[3 * i + a] = b3[a];
  }
  if (Dout) memcpy(Dout, D, (size_t)n * ML_NF * sizeof(double));
  if (Gout) memcpy(Gout, G, (size_t)n * ML_NF * sizeof(double));
  free(D); free(G);
  return out_of_range;
}

/* ------------------------------------------------------------------ */
/* Standalone entry points (brute-force pair list)                     */
/* ------------------------------------------------------------------ */
static int pairs_brute(int n, const double* r, const double box[3], int** off_out, int** jl_out) {
  int* off = (int*)malloc((size_t)(n + 1) * sizeof(int));
  int cap = 1024, cnt = 0;
  int* jl = (int*)malloc((size_t)cap * sizeof(int));
  if (!off || !jl) { free(off); free(jl); return -1; }
  for (int i = 0; i < n; ++i) {
    off[i] = cnt;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double d[3];
      sep(r, box, i, j, d);
      if (dot3(d, d) < ML_RC * ML_RC) {
        if (cnt == cap) {
          cap *= 2;
          int* nj = (int*)realloc(jl, (size_t)cap * sizeof(int));
          if (!nj) { free(off); free(jl); return -1; }
          jl = nj;
        }
        jl[cnt++] = j;
      }
    }
  }
  off[n] = cnt;
  *off_out = off;
  *jl_out = jl;
  return 0;
}

/* Learned energy and its gradients for one periodic frame.  r, s: [n][3];
 * outputs (any may be NULL): e_atom[n], D[n][48], G[n][48], F[n][3] (eV/A),
 * B[n][3] = -dE/ds (eV).  Returns the out-of-range atom count, or -1. */
int orc_ml_eval(int n, const double* r, const double* s, const double box[3], const float* params,
                const float* norm, double* e_atom, double* D, double* G, double* F, double* B) {
  orc_ml_model* m = (orc_ml_model*)malloc(sizeof(orc_ml_model));
  int *off = NULL, *jl = NULL;
  if (!m || pairs_brute(n, r, box, &off, &jl)) { free(m); return -1; }
  orc_ml_load(params, norm, m);
  int bad = orc_ml_frame(n, r, s, box, off, jl, m, e_atom, D, G, F, B, NULL, NULL);
  free(m); free(off); free(jl);
  return bad;
}

/* Adjoint of G: Gbar_a[f] such that sum_i gF_i.F_i + sum_i gB_i.B_i
 * = sum_a sum_f Gbar_a[f] G_a[f] at fixed positions and spins. */
static void g_adjoint(int n, const double* r, const double* s, const double box[3], const int* off, const int* jl,
                      const double* gF, const double* gB, double* Gbar) {
  memset(Gbar, 0, (size_t)n * ML_NF * sizeof(double));
  for (int a = 0; a < n; ++a) {
    double* Ga = Gbar + (size_t)a * ML_NF;
    const double* sa = s + 3 * a;
    for (int k = off[a]; k < off[a + 1]; ++k) {
      int j = jl[k];
      double d[3], g[ML_NK], dg[ML_NK];
      sep(r, box, a, j, d);
      double rr = sqrt(dot3(d, d));
      if (!(rr < ML_RC)) continue;
      const double* sj = s + 3 * j;
      double c = dot3(sa, sj);
      basis(rr, g, dg);
      /* F terms: phi_aj e_aj . gF_a from F_a, and phi_ja e_ja . gF_j from F_j, e_ja = -e_aj */
      double fe = 0.0;
      if (gF)
        for (int q = 0; q < 3; ++q) fe += d[q] / rr * (gF[3 * a + q] - gF[3 * j + q]);
      /* B terms: -psi_aj s_j . gB_a from B_a, and -psi_ja s_a . gB_j from B_j */
      double be = 0.0;
      if (gB) be = -(dot3(sj, gB + 3 * a) + dot3(sa, gB + 3 * j));
      for (int q = 0; q < ML_NK; ++q) {
        Ga[3 * q] += dg[q] * fe;
        Ga[3 * q + 1] += dg[q] * c * fe + g[q] * be;
        Ga[3 * q + 2] += dg[q] * c * c * fe + 2.0 * g[q] * c * be;
      }
    }
  }
}

/* Parameter gradient of  gE E + sum_i gF_i.F_i + sum_i gB_i.B_i  for one
 * frame (gF, gB may be NULL), added to grad[ML_NPARAM]. */
static int frame_param_grad(int n, const double* r, const double* s, const double box[3], const int* off,
                            const int* jl, const orc_ml_model* m, double gE, const double* gF, const double* gB,
                            double* grad) {
  double* D = (double*)malloc((size_t)(n ? n : 1) * ML_NF * sizeof(double));
  double* Gbar = (double*)malloc((size_t)(n ? n : 1) * ML_NF * sizeof(double));
  if (!D || !Gbar) { free(D); free(Gbar); return -1; }
  for (int i = 0; i < n; ++i) descriptor(i, r, s, box, off, jl, D + (size_t)i * ML_NF);
  g_adjoint(n, r, s, box, off, jl, gF, gB, Gbar);
  for (int i = 0; i < n; ++i) {
    double x[ML_NF], u[ML_NF];
    normalise(m, D + (size_t)i * ML_NF, x);
    /* G = inv_std * dE/dx, so Gbar . G = (Gbar * inv_std) . dE/dx */
    for (int f = 0; f < ML_NF; ++f) u[f] = Gbar[(size_t)i * ML_NF + f] * m->istd[f];
    net_param_grad(m, x, u, gE, grad);
  }
  free(D); free(Gbar);
  return 0;
}

int orc_ml_vjp(int n, const double* r, const double* s, const double box[3], const float* params, const float* norm,
               double gE, const double* gF, const double* gB, double* grad) {
  orc_ml_model* m = (orc_ml_model*)malloc(sizeof(orc_ml_model));
  int *off = NULL, *jl = NULL;
  if (!m || pairs_brute(n, r, box, &off, &jl)) { free(m); return -1; }
  orc_ml_load(params, norm, m);
  memset(grad, 0, ML_NPARAM * sizeof(double));
  int e = frame_param_grad(n, r, s, box, off, jl, m, gE, gF, gB, grad);
  free(m); free(off); free(jl);
  return e;
}

/* Training loss over a batch of frames and its parameter gradient.
 *   L = wE mean_f (dE_f/N_f)^2 + wF (1/Ntot) sum_i |dF_i|^2
 *       + wW (1/Ntot) sum_i |P_i dB_i / hbar|^2
 * with d = learned - reference, P_i = 1 - s_i s_i^T (only the part of the
 * precession vector omega = B/hbar normal to s_i moves the spin).
 * Frames are concatenated: n_of[f] atoms each, boxes[3 f..3 f+2].
 * out[0..3] = L and its three terms.  grad (may be NULL) gets dL/dparams. */
int orc_ml_loss(int nframes, const int* n_of, const double* r, const double* s, const double* boxes,
                const double* E_ref, const double* F_ref, const double* B_ref, const double w[3], double hbar,
                const float* params, const float* norm, double out[4], double* grad) {
  orc_ml_model* m = (orc_ml_model*)malloc(sizeof(orc_ml_model));
  if (!m) return -1;
  orc_ml_load(params, norm, m);
  long ntot = 0;
  for (int f = 0; f < nframes; ++f) ntot += n_of[f];
  double le = 0.0, lf = 0.0, lw = 0.0;
  if (grad) memset(grad, 0, ML_NPARAM * sizeof(double));
  long a0 = 0;
  int rc = 0;
  for (int f = 0; f < nframes && !rc; ++f) {
    int n = n_of[f];
    const double* rf = r + 3 * a0;
    const double* sf = s + 3 * a0;
    int *off = NULL, *jl = NULL;
    double* e = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
    double* F = (double*)malloc((size_t)(n ? n : 1) * 3 * sizeof(double));
    double* B = (double*)malloc((size_t)(n ? n : 1) * 3 * sizeof(double));
    double* gF = (double*)malloc((size_t)(n ? n : 1) * 3 * sizeof(double));
    double* gB = (double*)malloc((size_t)(n ? n : 1) * 3 * sizeof(double));
    if (!e || !F || !B || !gF || !gB || pairs_brute(n, rf, boxes + 3 * f, &off, &jl)) {
      rc = -1;
    } else {
      orc_ml_frame(n, rf, sf, boxes + 3 * f, off, jl, m, e, NULL, NULL, F, B, NULL, NULL);
      double E = 0.0;
      for (int i = 0; i < n; ++i) E += e[i];
      double dE = (E - E_ref[f]) / n;
      le += w[0] * dE * dE / nframes;
      double gE = 2.0 * w[0] * dE / ((double)n * nframes);
      for (int i = 0; i < n; ++i) {
        const double* si = sf + 3 * i;
        double dF[3], dB[3];
        for (int q = 0; q < 3; ++q) {
          dF[q] = F[3 * i + q] - F_ref[3 * (a0 + i) + q];
          dB[q] = B[3 * i + q] - B_ref[3 * (a0 + i) + q];
        }
        double sb = dot3(si, dB);
        double pb[3];
        for (int q = 0; q < 3; ++q) pb[q] = dB[q] - sb * si[q];
        lf += w[1] * dot3(dF, dF) / ntot;
        lw += w[2] * dot3(pb, pb) / (hbar * hbar * ntot);
        for (int q = 0; q < 3; ++q) {
          gF[3 * i + q] = 2.0 * w[1] * dF[q] / ntot;
          gB[3 * i + q] = 2.0 * w[2] * pb[q] / (hbar * hbar * ntot);
        }
      }
      if (grad) rc = frame_param_grad(n, rf, sf, boxes + 3 * f, off, jl, m, gE, gF, gB, grad);
    }
    free(e); free(F); free(B); free(gF); free(gB); free(off); free(jl);
    a0 += n;
  }
  free(m);
  out[0] = le + lf + lw;
  out[1] = le; out[2] = lf; out[3] = lw;
  return rc;
}

/* One Adam update (Kingma and Ba, ICLR 2015, Algorithm 1) of the float32
 * master parameters: t is the 1-based step count. */
void orc_ml_adam(int np, float* params, const double* grad, double* mom1, double* mom2, int t, double lr,
                 double beta1, double beta2, double eps) {
  double c1 = 1.0 - pow(beta1, t), c2 = 1.0 - pow(beta2, t);
  for (int i = 0; i < np; ++i) {
    mom1[i] = beta1 * mom1[i] + (1.0 - beta1) * grad[i];
    mom2[i] = beta2 * mom2[i] + (1.0 - beta2) * grad[i] * grad[i];
    double mh = mom1[i] / c1, vh = mom2[i] / c2;
    params[i] = (float)((double)params[i] - lr * mh / (sqrt(vh) + eps));
  }
}

/* ------------------------------------------------------------------ */
/* Sampled atoms of a large frame, one by one                          */
/* ------------------------------------------------------------------ */
/* Neighbours of atom a with r < ML_RC, by a scan over all n atoms. */
static int scan_neighbours(int n, const double* r, const double box[3], int a, int* out, int cap) {
  int cnt = 0;
  for (int j = 0; j < n; ++j) {
    if (j == a) continue;
    double d[3];
    sep(r, box, a, j, d);
    if (dot3(d, d) < ML_RC * ML_RC) {
      if (cnt < cap) out[cnt] = j;
      ++cnt;
    }
  }
  return cnt;
}

/* D and G of atom a from a scanned neighbour list. */
static void atom_DG(int n, const double* r, const double* s, const double box[3], const orc_ml_model* m, int a,
                    double D[ML_NF], double G[ML_NF], double* e) {
  int nb[512];
  int cnt = scan_neighbours(n, r, box, a, nb, 512);
  int off[2] = {0, cnt < 512 ? cnt : 512};
  /* descriptor() indexes off[i], off[i+1] with i = the atom: use a local list */
  memset(D, 0, ML_NF * sizeof(double));
  for (int k = 0; k < off[1]; ++k) {
    int j = nb[k];
    double d[3], g[ML_NK];
    sep(r, box, a, j, d);
    double rr = sqrt(dot3(d, d));
    if (!(rr < ML_RC)) continue;
    double c = dot3(s + 3 * a, s + 3 * j);
    basis(rr, g, NULL);
    for (int q = 0; q < ML_NK; ++q) {
      D[3 * q] += g[q];
      D[3 * q + 1] += g[q] * c;
      D[3 * q + 2] += g[q] * c * c;
    }
  }
  double x[ML_NF], gx[ML_NF];
  act_t A;
  normalise(m, D, x);
  double ea = net_forward(m, x, &A);
  if (e) *e = ea;
  net_backward(m, &A, gx);
  for (int f = 0; f < ML_NF; ++f) G[f] = gx[f] * m->istd[f];
}

/* For each sampled atom idx[q]: E_i, F_i (eV/A), B_i = -dE/ds_i (eV) and
 * D_i, computed from scratch (every neighbourhood by a scan over all atoms).
 * Returns -1 if an atom has more than 511 neighbours, else 0. */
int orc_ml_eval_sample(int n, const double* r, const double* s, const double box[3], const float* params,
                       const float* norm, int nsample, const int* idx, double* e_out, double* F_out,
                       double* B_out, double* D_out) {
  orc_ml_model* m = (orc_ml_model*)malloc(sizeof(orc_ml_model));
  if (!m) return -1;
  orc_ml_load(params, norm, m);
  int rc = 0;
  for (int q = 0; q < nsample && !rc; ++q) {
    int i = idx[q];
    int nb[512];
    int cnt = scan_neighbours(n, r, box, i, nb, 512);
    if (cnt > 511) { rc = -1; break; }
    double Di[ML_NF], Gi[ML_NF], Dj[ML_NF], Gj[ML_NF], ei;
    atom_DG(n, r, s, box, m, i, Di, Gi, &ei);
    double f3[3] = {0, 0, 0}, b3[3] = {0, 0, 0};
    const double* si = s + 3 * i;
    for (int k = 0; k < cnt; ++k) {
      int j = nb[k];
      double d[3], g[ML_NK], dg[ML_NK];
      sep(r, box, i, j, d);
      double rr = sqrt(dot3(d, d));
      atom_DG(n, r, s, box, m, j, Dj, Gj, NULL);
      const double* sj = s + 3 * j;
      double c = dot3(si, sj);
      basis(rr, g, dg);
      double phi = 0.0, pp = 0.0, qq = 0.0;
      for (int t = 0; t < ML_NK; ++t) {
        double s0 = Gi[3 * t] + Gj[3 * t], s1 = Gi[3 * t + 1] + Gj[3 * t + 1], s2 = Gi[3 * t + 2] + Gj[3 * t + 2];
        phi += (s0 + s1 * c + s2 * c * c) * dg[t];
        pp += s1 * g[t];
        qq += s2 * g[t];
      }
      for (int a = 0; a < 3; ++a) f3[a] += phi * d[a] / rr;
      double psi = pp + 2.0 * qq * c;
      for (int a = 0; a < 3; ++a) b3[a] -= psi * sj[a];
    }
    if (e_out) e_out[q] = ei;
    for (int a = 0; a < 3; ++a) {
      if (F_out) F_out[3 * q + a] = f3[a];
      if (B_out) B_out[3 * q + a] = b3[a];
    }
    if (D_out) memcpy(D_out + (size_t)q * ML_NF, Di, ML_NF * sizeof(double));
  }
  free(m);
  return rc;
}
