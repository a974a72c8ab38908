"""Order independence of the sectored sweep (Sec. 5.1, Sec. 5.2).

A different sector grid changes the order in which spins turn, so the two
runs are two different symmetric splittings of the same flow: both second
order, so their states differ by O(dt^2) (halving dt divides the difference
by 4), and the energy and |M| agree to that order.  A sweep that is not a
palindrome, or an update order that mixes colours, makes each scheme first
order and the ratio 2."""
import numpy as np

import oracle
from paper_1801_10233_gb300 import inputs

T_END = 0.01   # ps: no atom moves skin/2, so neither run re-sectors


def _run(skin, dt):
    p, r, v, s = inputs.bcc_fe_system(8, 51, T=300.0, sigma=0.02, spins="uniform", skin_A=skin, dt_ps=dt)
    o = oracle.Oracle(p, r, v, s, threads=4)
    assert o.step(int(round(T_END / dt))) == 0
    assert o.rebuilds == 1
    return o


def test_other_sector_grid_agrees_to_second_order():
    gaps = []
    for dt in (2e-4, 1e-4, 5e-5):
        a, b = _run(0.3, dt), _run(1.5, dt)
        assert list(a.order()["nsec"]) == [6, 6, 6] and list(b.order()["nsec"]) == [4, 4, 4]
        (ra, _, sa), (rb, _, sb) = a.state(), b.state()
        n = ra.shape[0]
        # energy: conserved by both to far below the splitting gap
        assert abs(a.energy()[4] - b.energy()[4]) / n < 1e-12
        gaps.append((np.abs(sa - sb).max(), np.abs(ra - rb).max(),
                     abs(a.magnetization()[3] - b.magnetization()[3])))
    gaps = np.array(gaps)
    assert gaps[1, 0] < 1e-5          # the orders differ, but only at the splitting error
    assert gaps[1, 0] > 1e-8          # ... which is there: the grids really order the spins differently
    for k in range(3):
        for q in range(2):
            ratio = gaps[q, k] / gaps[q + 1, k]
            assert 3.5 < ratio < 4.5, (k, q, ratio)
