"""Pins of the oracle's learned per-atom Hamiltonian (CPU only).

The paper has no learned model, so nothing here comes from it: the model is
pinned to closed forms of its definition (a dimer's descriptor), to library
routines (torch's Linear/SiLU/autograd, torch's bfloat16 rounding), to
finite differences of its own energy and loss, to invariances of the energy
(translation, cubic symmetry, global spin rotation, momentum, spin torque)
and, inside the integrator, to exact Larmor precession, time reversal and
the analytic path when the range gate refuses the network.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import ML_NF, ML_NH, ML_NNORM, ML_NPARAM, ML_OFF_B1, ML_OFF_B2, ML_OFF_B3, ML_OFF_W1, ML_OFF_W2, \
    ML_OFF_W3, HBAR
from paper_1801_10233_gb300 import inputs

from _ml_models import BIG, fitted_norm, model, open_norm, spin_free  # noqa: E402


def frame(ncells=5, seed=7, sigma=0.05):
    p, r, v, s = inputs.bcc_fe_system(ncells, seed, T=300.0, sigma=sigma, spins="uniform")
    return p, r, v, s


@pytest.fixture(scope="module")
def sys5():
    p, r, v, s = frame()
    box = np.array(p["box"])
    norm = fitted_norm(r, s, box)
    return p, r, v, s, box, norm


# ---------------------------------------------------------------------------
# Descriptor: closed forms
# ---------------------------------------------------------------------------
def test_dimer_descriptor_closed_form():
    box = np.array([20.0, 20.0, 20.0])
    r = np.array([[0.0, 0.0, 0.0], [2.4, 0.0, 0.0]])
    s = np.array([[1.0, 0.0, 0.0], [0.5, math.sqrt(3.0) / 2.0, 0.0]])
    D = oracle.ml_eval(r, s, box, model(), open_norm())["D"]
    fc = (3.0 + math.sqrt(5.0)) / 8.0          # (1 + cos(2 pi/5))/2, cos(2 pi/5) = (sqrt5 - 1)/4
    c = 0.5
    for k, val in [(6, fc), (5, math.exp(-0.5) * fc), (7, math.exp(-0.5) * fc), (4, math.exp(-2.0) * fc),
                   (0, math.exp(-18.0) * fc)]:
        for m in range(3):
            assert D[0, 3 * k + m] == pytest.approx(val * c ** m, rel=1e-14, abs=1e-300)
    assert np.array_equal(D[0], D[1])


def test_descriptor_vanishes_smoothly_at_cutoff():
    box = np.array([20.0, 20.0, 20.0])
    s = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
    eps = 1e-6
    D_in = oracle.ml_eval(np.array([[0, 0, 0], [6.0 - eps, 0, 0]], float), s, box, model(), open_norm())["D"]
    D_out = oracle.ml_eval(np.array([[0, 0, 0], [6.0 + eps, 0, 0]], float), s, box, model(), open_norm())["D"]
    assert np.all(D_out == 0.0)
    # fc(6 - eps) = (1 - cos(pi eps/6))/2 ~ (pi eps/6)^2/4; the k = 15 Gaussian is centred at 6 A
    assert D_in[0, 45] == pytest.approx((math.pi * eps / 6.0) ** 2 / 4.0, rel=1e-6)


# ---------------------------------------------------------------------------
# Network: library routines
# ---------------------------------------------------------------------------
def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = rng.normal(0, 1, 2000).astype(np.float32)
    # exact ties: a bf16 value plus half its ulp
    base = rng.normal(0, 1, 200).astype(np.float32)
    ties = (base.view(np.uint32) & 0xFFFF0000) | 0x8000
    x = np.concatenate([x, ties.astype(np.uint32).view(np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([oracle.bf16_value(float(v)) for v in x])
    assert np.array_equal(got, ref)


def test_network_matches_torch(sys5):
    torch = pytest.importorskip("torch")
    p, r, v, s, box, norm = sys5
    par = model()
    out = oracle.ml_eval(r, s, box, par, norm)
    pt = torch.from_numpy(par.astype(np.float32))
    bf = lambda a: a.to(torch.bfloat16).to(torch.float64)
    W1 = bf(pt[ML_OFF_W1:ML_OFF_B1].reshape(ML_NH, ML_NF))
    b1 = pt[ML_OFF_B1:ML_OFF_W2].double()
    W2 = bf(pt[ML_OFF_W2:ML_OFF_B2].reshape(ML_NH, ML_NH))
    b2 = pt[ML_OFF_B2:ML_OFF_W3].double()
    w3 = bf(pt[ML_OFF_W3:ML_OFF_B3].reshape(1, ML_NH))
    b3 = pt[ML_OFF_B3:].double()
    mean = torch.from_numpy(norm[:ML_NF]).double()
    istd = torch.from_numpy(norm[ML_NF:2 * ML_NF]).double()
    x = ((torch.from_numpy(out["D"]) - mean) * istd).requires_grad_(True)
    F = torch.nn.functional
    e = F.linear(F.silu(F.linear(F.silu(F.linear(x, W1, b1)), W2, b2)), w3, b3).squeeze(1)
    (gx,) = torch.autograd.grad(e.sum(), x)
    np.testing.assert_allclose(out["e_atom"], e.detach().numpy(), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(out["G"], (gx * istd).numpy(), rtol=1e-11, atol=1e-12)


# ---------------------------------------------------------------------------
# Gradients: finite differences of the oracle's own energy
# ---------------------------------------------------------------------------
def energy(r, s, box, par, norm):
    return oracle.ml_eval(r, s, box, par, norm)["e_atom"].sum()


def test_forces_are_minus_gradient(sys5):
    p, r, v, s, box, norm = sys5
    par = model()
    F = oracle.ml_eval(r, s, box, par, norm)["F"]
    h = 1e-5
    for a in (0, 17, 101, 249):
        for q in range(3):
            rp = r.copy(); rp[a, q] += h
            rm = r.copy(); rm[a, q] -= h
            fd = -(energy(rp, s, box, par, norm) - energy(rm, s, box, par, norm)) / (2 * h)
            assert fd == pytest.approx(F[a, q], abs=2e-7 * max(1.0, abs(F).max()))


def test_field_is_minus_spin_gradient(sys5):
    p, r, v, s, box, norm = sys5
    par = model()
    B = oracle.ml_eval(r, s, box, par, norm)["B"]
    h = 1e-5
    for a in (3, 50, 200):
        for q in range(3):
            sp = s.copy(); sp[a, q] += h
            sm = s.copy(); sm[a, q] -= h
            fd = -(energy(r, sp, box, par, norm) - energy(r, sm, box, par, norm)) / (2 * h)
            assert fd == pytest.approx(B[a, q], abs=2e-7 * max(1.0, abs(B).max()))


def test_invariances(sys5):
    p, r, v, s, box, norm = sys5
    par = model()
    o = oracle.ml_eval(r, s, box, par, norm)
    E = o["e_atom"].sum()
    # translation
    t = oracle.ml_eval(r + np.array([0.37, -1.1, 2.9]), s, box, par, norm)
    assert t["e_atom"].sum() == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(t["F"], o["F"], atol=1e-11)
    # 90 degree rotation about z of the cubic box (positions), spins untouched
    rr = np.stack([box[1] - r[:, 1], r[:, 0], r[:, 2]], axis=1)
    q = oracle.ml_eval(rr, s, box, par, norm)
    assert q["e_atom"].sum() == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(q["F"], np.stack([-o["F"][:, 1], o["F"][:, 0], o["F"][:, 2]], 1), atol=1e-11)
    # global spin rotation
    ang = 0.83
    R = np.array([[1, 0, 0], [0, math.cos(ang), -math.sin(ang)], [0, math.sin(ang), math.cos(ang)]])
    g = oracle.ml_eval(r, s @ R.T, box, par, norm)
    assert g["e_atom"].sum() == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(g["B"], o["B"] @ R.T, atol=1e-11)
    # momentum and spin torque: sum_i F_i = 0, sum_i s_i x B_i = 0
    assert np.abs(o["F"].sum(0)).max() < 1e-11 * max(1.0, np.abs(o["F"]).max()) * len(r)
    assert np.abs(np.cross(s, o["B"]).sum(0)).max() < 1e-11 * max(1.0, np.abs(o["B"]).max()) * len(r)


# ---------------------------------------------------------------------------
# Parameter gradients (forward-over-reverse) against finite differences
# ---------------------------------------------------------------------------
PROBE = [ML_OFF_W1 + 2 * ML_NF + 7, ML_OFF_W1 + 10 * ML_NF + 40, ML_OFF_W1 + 63 * ML_NF + 1,
         ML_OFF_B1 + 3, ML_OFF_W2 + 4 * ML_NH + 9, ML_OFF_W2 + 60 * ML_NH + 33, ML_OFF_B2 + 5,
         ML_OFF_W3 + 11, ML_OFF_B3]


def probe_fd(fun, par, idx, h=2.0 ** -14):
    """Central difference at a point where par[idx] = 0; +-h is exact in
    bfloat16 and float32, so the used weight moves by exactly h."""
    pp = par.copy(); pp[idx] = h
    pm = par.copy(); pm[idx] = -h
    return (fun(pp) - fun(pm)) / (2 * h)


def test_vjp_matches_finite_differences(sys5):
    p, r, v, s, box, norm = sys5
    par = model()
    par[PROBE] = 0.0
    rng = np.random.default_rng(11)
    gE = 0.7
    gF = rng.normal(0, 1, r.shape)
    gB = rng.normal(0, 1, r.shape)

    def S(pv):
        o = oracle.ml_eval(r, s, box, pv, norm)
        return gE * o["e_atom"].sum() + (gF * o["F"]).sum() + (gB * o["B"]).sum()

    grad = oracle.ml_vjp(r, s, box, par, norm, gE, gF, gB)
    scale = np.abs(grad).max()
    for idx in PROBE:
        assert probe_fd(S, par, idx) == pytest.approx(grad[idx], abs=1e-6 * scale)


def labelled_frames():
    frames, E_ref, F_ref, B_ref = [], [], [], []
    for cells, seed in [((5, 5, 5), 21), ((5, 5, 6), 22)]:
        p, r, v, s = inputs.bcc_fe_system(cells, seed, T=600.0, sigma=0.05, spins="uniform")
        o = oracle.Oracle(p, r, v, s)
        e = o.energy()
        zee = p["mu_s_muB"] * 5.7883818060e-5 * np.array(p["H_tesla"])
        frames.append((r, s, np.array(p["box"])))
        E_ref.append(e[1] + e[2])
        F_ref.append(o.forces())
        B_ref.append(o.omega() * HBAR - zee)
    return frames, np.array(E_ref), np.concatenate(F_ref), np.concatenate(B_ref)


def test_loss_gradient_matches_finite_differences():
    frames, E_ref, F_ref, B_ref = labelled_frames()
    norm = fitted_norm(*frames[0])
    par = model()
    par[PROBE] = 0.0
    w = [1.0, 0.5, 2e-6]
    out, grad = oracle.ml_loss(frames, E_ref, F_ref, B_ref, w, par, norm)
    assert out[0] == pytest.approx(out[1:].sum(), rel=1e-14)
    scale = np.abs(grad).max()
    for idx in PROBE:
        fd = probe_fd(lambda pv: oracle.ml_loss(frames, E_ref, F_ref, B_ref, w, pv, norm, False)[0][0], par, idx)
        assert fd == pytest.approx(grad[idx], abs=1e-6 * scale)


def test_loss_terms_special_cases(sys5):
    p, r, v, s, box, norm = sys5
    par = model()
    o = oracle.ml_eval(r, s, box, par, norm)
    n = len(r)
    E = o["e_atom"].sum()
    fr = [(r, s, box)]
    # energy term: reference off by delta per atom
    out, _ = oracle.ml_loss(fr, [E - 0.03 * n], o["F"], o["B"], [1, 0, 0], par, norm, False)
    assert out[0] == pytest.approx(0.03 ** 2, rel=1e-10)
    # force term: constant offset c on every atom
    c = np.array([0.1, -0.2, 0.05])
    out, _ = oracle.ml_loss(fr, [E], o["F"] + c, o["B"], [0, 1, 0], par, norm, False)
    assert out[0] == pytest.approx((c ** 2).sum(), rel=1e-12)
    # field term: a radial offset does not count, a tangential one of size tau does
    out, _ = oracle.ml_loss(fr, [E], o["F"], o["B"] + 0.3 * s, [0, 0, 1], par, norm, False)
    assert out[0] == pytest.approx(0.0, abs=1e-20)
    t = np.cross(s, np.array([0.0, 0.0, 1.0]))
    t = 0.01 * t / np.linalg.norm(t, axis=1, keepdims=True)
    out, _ = oracle.ml_loss(fr, [E], o["F"], o["B"] + t, [0, 0, 1], par, norm, False)
    assert out[0] == pytest.approx(0.01 ** 2 / HBAR ** 2, rel=1e-10)


def test_adam_first_steps_closed_form():
    rng = np.random.default_rng(5)
    par = rng.normal(0, 1, 100).astype(np.float32)
    g = rng.normal(0, 1, 100)
    m = np.zeros(100); v = np.zeros(100)
    p0 = par.copy()
    lr, eps = 1e-3, 1e-8
    oracle.ml_adam(par, g, m, v, 1, lr, eps=eps)
    # bias-corrected moments of a constant gradient are g and g^2
    np.testing.assert_allclose(par, (p0 - lr * g / (np.abs(g) + eps)).astype(np.float32), rtol=0, atol=1e-7)
    p1 = par.copy()
    oracle.ml_adam(par, g, m, v, 2, lr, eps=eps)
    np.testing.assert_allclose(par, (p1 - lr * g / (np.abs(g) + eps)).astype(np.float32), rtol=0, atol=1e-7)


# ---------------------------------------------------------------------------
# Learned integrator
# ---------------------------------------------------------------------------
def learned_oracle(par, norm, seed=31, ncells=5, **kw):
    p, r, v, s = inputs.bcc_fe_system(ncells, seed, T=300.0, sigma=0.05, spins="uniform", hamiltonian=1, **kw)
    o = oracle.Oracle(p, r, v, s)
    o.set_model(par, norm)
    return o, p, r, v, s


def test_learned_spin_free_model_gives_exact_larmor(sys5):
    *_, norm = sys5
    o, p, r, v, s = learned_oracle(spin_free(model()), norm)
    nsteps = 20
    o.step(nsteps)
    _, _, s1 = o.state()
    wz = p["mu_s_muB"] * 5.7883818060e-5 * p["H_tesla"][2] / HBAR
    th = wz * p["dt_ps"] * nsteps
    Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    np.testing.assert_allclose(s1, s @ Rz.T, atol=1e-13)
    assert o.gate() == (0, 0)


def test_learned_time_reversal_spin_free(sys5):
    *_, norm = sys5
    o, p, r, v, s = learned_oracle(spin_free(model()), norm, rebuild_every=5)
    o.step(10)
    o.set_dt(-p["dt_ps"])
    o.step(10)
    r1, v1, s1 = o.state()
    L = np.array(p["box"])
    dr = r1 - r
    dr -= L * np.round(dr / L)
    assert np.abs(dr).max() < 1e-10
    assert np.abs(s1 - s).max() < 1e-10


def test_learned_invariants(sys5):
    *_, norm = sys5
    o, p, r, v, s = learned_oracle(model(), norm)
    P0 = v.sum(0)
    o.step(30)
    r1, v1, s1 = o.state()
    assert np.abs(np.linalg.norm(s1, axis=1) - 1.0).max() < 1e-14
    assert np.abs(v1.sum(0) - P0).max() < 1e-10
    assert np.abs(s1 - s).max() > 1e-6          # the spins did move
    assert o.gate()[1] == 0


def test_learned_energy_and_omega_are_the_network(sys5):
    *_, norm = sys5
    par = model()
    o, p, r, v, s = learned_oracle(par, norm)
    ref = oracle.ml_eval(r, s, np.array(p["box"]), par, norm)
    e = o.energy()
    assert e[1] == pytest.approx(ref["e_atom"].sum(), rel=1e-13)
    assert e[2] == 0.0
    zee = p["mu_s_muB"] * 5.7883818060e-5 * np.array(p["H_tesla"])
    _, _, sw = o.state()
    order = np.argsort(np.arange(len(r)))  # ids unchanged by the oracle
    np.testing.assert_allclose(o.omega(), (ref["B"] + zee) / HBAR, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(o.forces(), ref["F"], rtol=1e-12, atol=1e-12)


def test_gate_hands_back_to_analytic_hamiltonian(sys5):
    *_, norm = sys5
    closed = norm.copy()
    closed[2 * ML_NF:] = 0.0            # lo = hi = 0: every descriptor out of range
    kw = dict(rebuild_every=5)
    o, p, r, v, s = learned_oracle(model(), closed, ncells=7, **kw)
    o.step(7)
    # analytic run with the same 2 x 2 x 2 sector grid: exchange cutoff + skin = 6 + 0.3
    pa = dict(p)
    pa["hamiltonian"] = 0
    pa["skin_A"] = 6.0 + 0.3 - p["ex_rc_A"]
    a = oracle.Oracle(pa, r, v, s)
    a.step(7)
    assert o.order()["nsec"].tolist() == a.order()["nsec"].tolist() == [2, 2, 2]
    for x, y in zip(o.state(), a.state()):
        assert np.array_equal(x, y)
    bad, trips = o.gate()
    assert bad == len(r) and trips == 1 + 3 * 7


def test_learned_spin_energy_error_is_second_order_in_dt(sys5):
    """The symmetric learned half-op (predictor-corrector G, midpoint omega)
    has an energy error O(dt^2): halving dt quarters the energy excursion over
    a fixed time (the frozen-G or frozen-omega forms are first order)."""
    *_, norm = sys5
    par = inputs.ml_init_params(21, e0=-4.0)
    dev = []
    for dt in (2e-4, 1e-4):
        o, p, r, v, s = learned_oracle(par, norm, fix_lattice=1, dt_ps=dt)
        n = len(r)
        e0 = o.energy()[4]
        steps = int(round(0.006 / dt))
        ex = 0.0
        for k in range(4):
            o.step(steps // 4)
            ex = max(ex, abs(o.energy()[4] - e0) / n)
        dev.append(ex)
    assert dev[0] / dev[1] > 3.0, dev


def test_sampled_evaluation_equals_full_evaluation(sys5):
    p, r, v, s, box, norm = sys5
    par = model()
    full = oracle.ml_eval(r, s, box, par, norm)
    idx = [0, 17, 101, 249]
    smp = oracle.ml_eval_sample(r, s, box, par, norm, idx)
    for k in ("e_atom", "F", "B", "D"):
        np.testing.assert_allclose(smp[k], full[k][idx], rtol=1e-13, atol=1e-13)
