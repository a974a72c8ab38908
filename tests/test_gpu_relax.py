"""Two-thermostat relaxation (Sec. 4.2): with only the spins coupled to a
bath the lattice heats up through the spin-lattice coupling; with only the
lattice coupled, near-collinear spins (isotropic exchange) stay cold over
the run.  The thermostatted part stays near the bath temperature."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_one_bath_at_a_time():
    from paper_1801_10233_gb300 import relax
    # lambda = 0.05 so that a 1 ps preparation brings the uniformly random
    # spins down to the bath temperature (at 0.01 it takes ~2 ps)
    out = relax.run(cells=6, T=300.0, ps=1.0, dt=5e-4, every=200, prep_ps=1.0, lam=0.05)
    a, b = out["spin_bath"], out["lattice_bath"]
    assert a["T_L"][0] == 0.0 and a["T_L"][-1] > 1.0          # lattice warmed by the spins
    assert 150.0 < sum(a["T_S"]) / len(a["T_S"]) < 450.0      # spins held near the bath
    assert b["T_S"][-1] < 0.1 * 300.0                          # spins stay cold (no torque at collinearity)
    assert 150.0 < sum(b["T_L"][1:]) / len(b["T_L"][1:]) < 450.0
