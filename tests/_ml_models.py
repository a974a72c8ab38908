"""Shared helpers of the learned-Hamiltonian tests: seeded models and a
normalisation fitted to a frame's own descriptors (computed by the oracle)."""
import numpy as np

import oracle
from oracle import ML_NF, ML_NH, ML_NNORM, ML_OFF_B1, ML_OFF_B2, ML_OFF_B3, ML_OFF_W1, ML_OFF_W3
from paper_1801_10233_gb300 import inputs

BIG = np.float32(3e38)


def open_norm():
    n = np.zeros(ML_NNORM, np.float32)
    n[ML_NF:2 * ML_NF] = 1.0
    n[2 * ML_NF:3 * ML_NF] = -BIG
    n[3 * ML_NF:] = BIG
    return n


def fitted_norm(r, s, box):
    """mean / inv_std of the frame's own descriptors, gate wide open."""
    D = oracle.ml_eval(r, s, box, inputs.ml_init_params(1), open_norm())["D"]
    n = open_norm()
    n[:ML_NF] = D.mean(0)
    n[ML_NF:2 * ML_NF] = 1.0 / (D.std(0) + 1e-3)
    return n


def model(seed=3):
    p = inputs.ml_init_params(seed, e0=-4.0)
    rng = np.random.default_rng(seed)
    p[ML_OFF_B1:ML_OFF_B1 + ML_NH] = rng.normal(0, 0.3, ML_NH)
    p[ML_OFF_B2:ML_OFF_B2 + ML_NH] = rng.normal(0, 0.3, ML_NH)
    p[ML_OFF_W3:ML_OFF_W3 + ML_NH] *= 10.0
    return p


def spin_free(par):
    """Zero the weights of the s.s features: the energy no longer depends on the spins."""
    q = par.copy()
    W1 = q[ML_OFF_W1:ML_OFF_B1].reshape(ML_NH, ML_NF)
    W1[:, 1::3] = 0.0
    W1[:, 2::3] = 0.0
    return q
