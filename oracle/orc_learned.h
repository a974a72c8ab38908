/*
 * Learned per-atom Hamiltonian of the CPU oracle (TEST INFRASTRUCTURE ONLY).
 * Shared between the two oracle translation units; nothing outside oracle/
 * includes it.
 */
#ifndef ORC_LEARNED_H
#define ORC_LEARNED_H

#define ML_NK 16            /* radial Gaussians */
#define ML_NM 3             /* powers of s_i.s_j: 0, 1, 2 */
#define ML_NF 48            /* features, index f = 3 k + m */
#define ML_NH 64            /* hidden width of both layers */
#define ML_RC 6.0           /* descriptor cutoff, A */
#define ML_DMU 0.4          /* spacing of the Gaussian centres, A */
#define ML_SIGMA 0.4        /* Gaussian width, A */

/* Flat parameter vector (float): W1[64][48], b1[64], W2[64][64], b2[64], w3[64], b3. */
#define ML_OFF_W1 0
#define ML_OFF_B1 (ML_OFF_W1 + ML_NH * ML_NF)
#define ML_OFF_W2 (ML_OFF_B1 + ML_NH)
#define ML_OFF_B2 (ML_OFF_W2 + ML_NH * ML_NH)
#define ML_OFF_W3 (ML_OFF_B2 + ML_NH)
#define ML_OFF_B3 (ML_OFF_W3 + ML_NH)
#define ML_NPARAM (ML_OFF_B3 + 1)
/* Normalisation vector (float): mean[48], inv_std[48], gate lo[48], gate hi[48]. */
#define ML_NNORM (4 * ML_NF)

typedef struct {
  double W1[ML_NH][ML_NF], b1[ML_NH], W2[ML_NH][ML_NH], b2[ML_NH], w3[ML_NH], b3;
  double mean[ML_NF], istd[ML_NF], lo[ML_NF], hi[ML_NF];
} orc_ml_model;

void orc_ml_load(const float* params, const float* norm, orc_ml_model* m);

/* Energy, forces F = -dE/dr, field B = -dE/ds of the learned model over a
 * full pair list (CSR: off[n+1], jl; every ordered pair with r < ML_RC).
 * Also returns D (n x 48), G = dE_i/dD_i (n x 48), per-atom E and the pair
 * coefficients P, Q of the field (one per list entry).  Any output may be NULL.
 * Returns the number of atoms whose descriptor lies outside the gate range. */
int orc_ml_frame(int n, const double* r, const double* s, const double box[3], const int* off, const int* jl,
                 const orc_ml_model* m, double* e_atom, double* D, double* G, double* F, double* B, double* P,
                 double* Q);

#endif
