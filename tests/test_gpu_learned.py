"""GPU parity of the learned per-atom Hamiltonian against the FP64 oracle.

Tolerances follow from the arithmetic of the CUDA path: descriptors, pair
terms and field sums in float32 (unit roundoff u = 2^-24 ~ 6e-8) over at most
~90 neighbours and 16 Gaussians, the network's products on the tensor cores
with bfloat16 weights (exact: the oracle uses the same bfloat16 values) and
activations split into three bfloat16 pieces (24 bits, float32 precision),
float32 accumulation over K <= 64.  Every float32 result is then within
about 100 u ~ 6e-6 of its scale (the largest magnitude of that quantity);
the checks allow 1e-4 of the scale.  The state stays FP64 and the rotation
double-float, so trajectories differ only through those field and force
errors (bounds per test).
"""
import numpy as np
import pytest

import oracle
from oracle import HBAR, ML_NF, ML_NPARAM
from paper_1801_10233_gb300 import inputs

from _ml_models import fitted_norm, model, open_norm, spin_free

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-4


def close(a, b, rel=REL, what=""):
    a = np.asarray(a.cpu() if hasattr(a, "cpu") else a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = max(np.abs(b).max(), 1e-30)
    err = np.abs(a - b).max()
    assert err <= rel * scale, f"{what}: max err {err:.3e} > {rel:.1e} x scale {scale:.3e}"
    return err / scale


def system(cells=7, seed=41, T=300.0, spins="uniform", **kw):
    p, r, v, s = inputs.bcc_fe_system(cells, seed, T=T, sigma=0.05, spins=spins, hamiltonian=1, **kw)
    return p, r, v, s


@pytest.fixture(scope="module")
def lib():
    from paper_1801_10233_gb300 import learned
    return learned


@pytest.fixture(scope="module")
def frame7():
    p, r, v, s = system()
    norm = fitted_norm(r, s, np.array(p["box"]))
    return p, r, v, s, norm


def test_eval_matches_oracle(lib, frame7):
    p, r, v, s, norm = frame7
    par = model()
    sysm = lib.learned_system(p, r, v, s, norm, par)
    e, F, B, D = sysm.ml_eval(want_D=True)
    ref = oracle.ml_eval(r, s, np.array(p["box"]), par, norm)
    close(D, ref["D"], what="descriptors")
    assert abs(e[0] - ref["e_atom"].sum()) <= REL * np.abs(ref["e_atom"]).max() * len(r)
    close(F, ref["F"], what="forces")
    close(B, ref["B"], what="fields")
    # the integrator's forces and omega are the network's
    close(sysm.forces(), ref["F"], what="integrator forces")
    zee = lib.zeeman_field(p)
    close(sysm.omega(), (ref["B"] + zee) / HBAR, what="omega")
    en = sysm.energy()
    assert en[2] == 0.0
    assert en[1] == pytest.approx(ref["e_atom"].sum(), abs=REL * np.abs(ref["e_atom"]).max() * len(r))
    assert sysm.ml_gate() == (0, 1, 0)


def test_eval_batch_of_uneven_frames(lib):
    plist, rs, ss, refs = [], [], [], []
    for k, cells in enumerate([(7, 7, 7), (7, 7, 8), (8, 7, 7)]):
        p, r, v, s = system(cells, seed=50 + k)
        plist.append(p); rs.append(r); ss.append(s)
    norm = fitted_norm(rs[0], ss[0], np.array(plist[0]["box"]))
    par = model(5)
    r = np.concatenate(rs); s = np.concatenate(ss)
    sysm = lib.learned_system(plist, r, np.zeros_like(r), s, norm, par)
    e, F, B, _ = sysm.ml_eval()
    a0 = 0
    for k, p in enumerate(plist):
        n = p["n_atoms"]
        ref = oracle.ml_eval(rs[k], ss[k], np.array(p["box"]), par, norm)
        assert e[k] == pytest.approx(ref["e_atom"].sum(), abs=REL * np.abs(ref["e_atom"]).max() * n)
        close(F[a0:a0 + n], ref["F"], what=f"forces {k}")
        close(B[a0:a0 + n], ref["B"], what=f"fields {k}")
        a0 += n


def test_vjp_matches_oracle(lib, frame7):
    p, r, v, s, norm = frame7
    par = model(7)
    sysm = lib.learned_system(p, r, v, s, norm, par)
    rng = np.random.default_rng(3)
    gE = np.array([0.7]); gF = rng.normal(0, 1, r.shape); gB = rng.normal(0, 1, r.shape)
    g = sysm.ml_vjp(gE, gF, gB).cpu().numpy()
    ref = oracle.ml_vjp(r, s, np.array(p["box"]), par, norm, gE[0], gF, gB)
    close(g, ref, what="parameter gradient")
    # energy-only and force-only parts separately
    close(sysm.ml_vjp(gE=gE).cpu().numpy(), oracle.ml_vjp(r, s, np.array(p["box"]), par, norm, gE[0]),
          what="dE/dparams")
    close(sysm.ml_vjp(gF=gF).cpu().numpy(), oracle.ml_vjp(r, s, np.array(p["box"]), par, norm, 0.0, gF),
          what="d(gF.F)/dparams")


def labelled(plist, rs, vs, ss):
    E, F, B = [], [], []
    for p, r, v, s in zip(plist, rs, vs, ss):
        pa = dict(p, hamiltonian=0)
        o = oracle.Oracle(pa, r, v, s)
        e = o.energy()
        E.append(e[1] + e[2])
        F.append(o.forces())
        B.append(o.omega() * HBAR - p["mu_s_muB"] * 5.7883818060e-5 * np.array(p["H_tesla"]))
    return np.array(E), np.concatenate(F), np.concatenate(B)


def test_train_step_matches_oracle(lib):
    plist, rs, vs, ss = [], [], [], []
    for k, cells in enumerate([(7, 7, 7), (7, 8, 7)]):
        p, r, v, s = system(cells, seed=60 + k, T=600.0)
        plist.append(p); rs.append(r); vs.append(v); ss.append(s)
    E, F, B = labelled(plist, rs, vs, ss)
    norm = fitted_norm(rs[0], ss[0], np.array(plist[0]["box"]))
    par = model(9)
    r = np.concatenate(rs); s = np.concatenate(ss)
    sysm = lib.learned_system(plist, r, np.zeros_like(r), s, norm, par)
    w = [1.0, 0.5, 2e-6]
    lr = 1e-3
    loss = sysm.ml_train_step(E, F, B, w, lr)
    frames = [(rs[k], ss[k], np.array(plist[k]["box"])) for k in range(2)]
    out, grad = oracle.ml_loss(frames, E, F, B, w, par, norm)
    np.testing.assert_allclose(loss, out, rtol=1e-4)
    # one Adam step from zero moments moves each parameter by lr g/(|g| + eps) ~ +-lr
    ref = par.copy()
    oracle.ml_adam(ref, grad, np.zeros(ML_NPARAM), np.zeros(ML_NPARAM), 1, lr)
    got = sysm.ml_get_model().cpu().numpy()
    settled = np.abs(grad) > 1e-3 * np.abs(grad).max()     # sign of g is certain there
    assert np.abs(got - ref)[settled].max() <= 1e-6
    assert np.abs(got - ref).max() <= 2.0 * lr + 1e-6


def test_learned_dynamics_matches_oracle(lib, frame7):
    p, r, v, s, norm = frame7
    pp = dict(p, rebuild_every=5)
    par = model(11)
    sysm = lib.learned_system(pp, r, v, s, norm, par)
    o = oracle.Oracle(pp, r, v, s)
    o.set_model(par, norm)
    nsteps = 10
    sysm.step(nsteps)
    o.step(nsteps)
    rg, vg, sg = (x.cpu().numpy() for x in sysm.state())
    ro, vo, so = o.state()
    L = np.array(p["box"])
    dr = rg - ro
    dr -= L * np.round(dr / L)
    # field errors <= 1e-4 |omega| -> rotation angle errors <= 1e-4 |omega| dt/4 per update (4 updates
    # per step, each from a predictor and a corrector sweep: 2 x 40 for 10 steps);
    # force errors <= 1e-4 |F| -> velocity and position errors from 10 kicks and drifts
    wmax = np.abs(o.omega()).max()
    Fmax = np.abs(o.forces()).max()
    acc = 9648.533212 / p["mass_amu"]
    dt = p["dt_ps"]
    assert np.abs(sg - so).max() <= 80 * REL * wmax * dt / 4
    assert np.abs(vg - vo).max() <= nsteps * REL * Fmax * acc * dt
    assert np.abs(dr).max() <= nsteps ** 2 * REL * Fmax * acc * dt ** 2
    eg = sysm.energy(); eo = o.energy()
    assert eg[1] == pytest.approx(eo[1], abs=REL * abs(eo[1]))
    assert sysm.ml_gate()[2] == 0 and o.gate()[1] == 0


def test_spin_free_model_gives_exact_larmor(lib, frame7):
    p, r, v, s, norm = frame7
    sysm = lib.learned_system(p, r, v, s, norm, spin_free(model()))
    nsteps = 20
    sysm.step(nsteps)
    s1 = sysm.state()[2].cpu().numpy()
    wz = p["mu_s_muB"] * 5.7883818060e-5 * p["H_tesla"][2] / HBAR
    th = wz * p["dt_ps"] * nsteps
    Rz = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    np.testing.assert_allclose(s1, s @ Rz.T, atol=1e-13)


def test_closed_gate_runs_the_analytic_hamiltonian(lib):
    p, r, v, s = system(7, seed=71)
    p = dict(p, rebuild_every=5)
    norm = fitted_norm(r, s, np.array(p["box"]))
    closed = norm.copy()
    closed[2 * ML_NF:] = 0.0
    par = model()
    sysm = lib.learned_system(p, r, v, s, closed, par)
    o = oracle.Oracle(p, r, v, s)
    o.set_model(par, closed)
    sysm.step(7)
    o.step(7)
    for a, b in zip(sysm.state(), o.state()):
        a = a.cpu().numpy()
        assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(b).max())
    bad, use, trips = sysm.ml_gate()
    assert bad == len(r) and use == 0 and trips == 1 + 2 * 7
    assert o.gate()[0] == len(r)


def test_learned_invariants(lib, frame7):
    # output weights at their initial (physical) scale: precession angles per
    # update of a few 1e-3 rad, as for the analytic Hamiltonian, so the
    # double-float rotation keeps |s| = 1 to 1e-14 over 800 updates
    p, r, v, s, norm = frame7
    par = inputs.ml_init_params(13, e0=-4.0)
    par[lib._lib.SL_ML_OFF_W3:lib._lib.SL_ML_OFF_B3] *= 0.2
    sysm = lib.learned_system(p, r, v, s, norm, par)
    assert np.abs(sysm.omega().cpu().numpy()).max() * p["dt_ps"] / 4 < 0.02
    P0 = v.sum(0)
    sysm.step(200)
    r1, v1, s1 = (x.cpu().numpy() for x in sysm.state())
    assert np.abs(np.linalg.norm(s1, axis=1) - 1.0).max() < 1e-14
    # float32 pair forces are antisymmetric to rounding: sum_i F_i ~ N u |F|
    Fmax = np.abs(sysm.forces().cpu().numpy()).max()
    acc = 9648.533212 / p["mass_amu"]
    assert np.abs(v1.sum(0) - P0).max() <= 200 * p["dt_ps"] * acc * len(r) * 1e-6 * Fmax
    assert sysm.counters()["graph"]


def test_autograd_functions(lib, frame7):
    p, r, v, s, norm = frame7
    par = model(17)
    sysm = lib.learned_system(p, r, v, s, norm, par)
    rt = torch.tensor(r, device="cuda", requires_grad=True)
    st = torch.tensor(s, device="cuda", requires_grad=True)
    pt = torch.tensor(par, device="cuda", requires_grad=True)
    E = lib.LearnedEnergy.apply(rt, st, pt, sysm)
    gr, gs, gp = torch.autograd.grad(E.sum(), [rt, st, pt])
    ref = oracle.ml_eval(r, s, np.array(p["box"]), par, norm)
    close(-gr, ref["F"], what="dE/dr = -F")
    close(-gs, ref["B"], what="dE/ds = -B")
    close(gp, oracle.ml_vjp(r, s, np.array(p["box"]), par, norm, 1.0), what="dE/dparams")
    # a loss on forces and fields, differentiated through LearnedForces
    pt2 = torch.tensor(par, device="cuda", requires_grad=True)
    E2, F2, B2 = lib.LearnedForces.apply(pt2, sysm)
    rng = np.random.default_rng(1)
    gF = torch.tensor(rng.normal(0, 1, r.shape), device="cuda")
    gB = torch.tensor(rng.normal(0, 1, r.shape), device="cuda")
    L = 0.3 * E2.sum() + (gF * F2).sum() + (gB * B2).sum()
    (g2,) = torch.autograd.grad(L, [pt2])
    close(g2, oracle.ml_vjp(r, s, np.array(p["box"]), par, norm, 0.3, gF.cpu().numpy(), gB.cpu().numpy()),
          what="d(loss)/dparams")


def test_training_reduces_loss(lib):
    plist, rs, vs, ss = [], [], [], []
    for k in range(4):
        p, r, v, s = system((7, 7, 7), seed=80 + k, T=100.0 + 300.0 * k)
        plist.append(p); rs.append(r); vs.append(v); ss.append(s)
    E, F, B = labelled(plist, rs, vs, ss)
    r = np.concatenate(rs); s = np.concatenate(ss)
    stats_sys = lib.learned_system(plist, r, np.zeros_like(r), s, open_norm(), model())
    norm = lib.normalisation(stats_sys.ml_descriptor_stats())
    sysm = lib.learned_system(plist, r, np.zeros_like(r), s, norm, inputs.ml_init_params(3, e0=float(E.mean() / 686)))
    w = [1.0, 1.0, 1e-6]
    losses = [sysm.ml_train_step(E, F, B, w, 2e-3) for _ in range(60)]
    assert losses[-1][0] < 0.5 * losses[0][0]


def test_learned_dynamics_staged_sweep_matches_oracle(lib):
    """10^3 cells: sectors small enough for the shared-memory sweep path."""
    p, r, v, s = system(10, seed=43, rebuild_every=5)
    norm = fitted_norm(r, s, np.array(p["box"]))
    par = inputs.ml_init_params(23, e0=-4.0)
    sysm = lib.learned_system(p, r, v, s, norm, par)
    o = oracle.Oracle(p, r, v, s)
    o.set_model(par, norm)
    nsteps = 6
    sysm.step(nsteps)
    o.step(nsteps)
    rg, vg, sg = (x.cpu().numpy() for x in sysm.state())
    ro, vo, so = o.state()
    L = np.array(p["box"])
    dr = rg - ro
    dr -= L * np.round(dr / L)
    wmax = np.abs(o.omega()).max()
    Fmax = np.abs(o.forces()).max()
    acc = 9648.533212 / p["mass_amu"]
    dt = p["dt_ps"]
    assert np.abs(sg - so).max() <= 8 * nsteps * REL * wmax * dt / 4
    assert np.abs(vg - vo).max() <= nsteps * REL * Fmax * acc * dt
    assert np.abs(dr).max() <= nsteps ** 2 * REL * Fmax * acc * dt ** 2


def test_learned_spin_energy_error_is_second_order(lib):
    p, r, v, s = system(10, seed=44, fix_lattice=1)
    norm = fitted_norm(r, s, np.array(p["box"]))
    par = inputs.ml_init_params(21, e0=-4.0)
    dev = []
    for dt in (2e-4, 1e-4):
        sysm = lib.learned_system(dict(p, dt_ps=dt), r, v, s, norm, par)
        e0 = sysm.energy()[4]
        steps = int(round(0.006 / dt))
        ex = 0.0
        for k in range(4):
            sysm.step(steps // 4)
            ex = max(ex, abs(sysm.energy()[4] - e0) / len(r))
        dev.append(ex)
        sysm.close()
    assert dev[0] / dev[1] > 3.0, dev


@pytest.mark.parametrize("name", ["fe_bcc_40x40x40_nve", "fe_bcc_100x100x100_nve"])
def test_full_size_sampled_atoms_match_oracle(lib, name):
    """The learned workloads at full size, in the benchmark's configuration:
    descriptors, forces and fields of sampled atoms against the oracle's
    atom-by-atom evaluation."""
    p, r, v, s = inputs.workload(name)
    box = np.array(p["box"])
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(p["n_atoms"], 6, replace=False))
    # normalisation from a cheap 6^3-cell frame of the same recipe
    p6, r6, v6, s6 = inputs.bcc_fe_system(6, 9, T=300.0, spins="uniform")
    norm = fitted_norm(r6, s6, np.array(p6["box"]))
    par = inputs.ml_init_params(31, e0=-4.0)
    sysm = lib.learned_system(lib.learned_params(p), r, v, s, norm, par)
    e, F, B, D = sysm.ml_eval(want_D=True)
    ref = oracle.ml_eval_sample(r, s, box, par, norm, idx)
    Fg, Bg, Dg = F.cpu().numpy()[idx], B.cpu().numpy()[idx], D.cpu().numpy()[idx]
    close(Dg, ref["D"], what="descriptors")
    close(Fg, ref["F"], what="forces")
    close(Bg, ref["B"], what="fields")
    sysm.step(2)
    assert sysm.ml_gate()[2] == 0
    sysm.close()
