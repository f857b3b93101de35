"""Pins of the oracle's wider limiter family (limiter table of Sect. 3.1.1):
superbee, woodward, mcbeta and albada beside minmod, vanleer and koren.

The limiter function phi(r) is measured from the oracle's own reconstruction
and checked against the published definitions' values at sample ratios
(tests/golden/limiter_phi.txt), against Sweby's second-order TVD region
(minmod <= phi <= superbee), for symmetry phi(r)/r = phi(1/r), exactness on
linear data, boundedness, and the order of the table.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SYMMETRIC = ["minmod", "vanleer", "superbee", "woodward", "mcbeta", "albada", "venk"]
ALL = SYMMETRIC + ["koren"]


def _phi(orc, lim, r):
    # cells (w_{i-1}, w_i, w_{i+1}) = (-r, 0, 1): dm = r, dp = 1, so the left
    # state at i+1/2 is phi(r)/2
    wl_, _ = orc.reconstruct(lim, np.array([-r, 0.0, 1.0]))
    return 2.0 * wl_[1]


def _golden_phi():
    rows = {}
    rs = None
    for line in open(os.path.join(GOLDEN, "limiter_phi.txt")):
        if line.startswith("# r:"):
            rs = [float(x) for x in line[4:].split()]
            continue
        line = line.split("#")[0].split()
        if line:
            rows[line[0]] = [float(x) for x in line[1:]]
    return rs, rows


def test_phi_matches_published_values(orc):
    rs, rows = _golden_phi()
    for lim, vals in rows.items():
        for r, want in zip(rs, vals):
            assert abs(_phi(orc, lim, r) - want) < 1e-14, (lim, r, want)


def test_second_order_tvd_region(orc):
    # Sweby: second-order TVD limiters lie between minmod and superbee
    for r in np.linspace(0.02, 6.0, 300):
        lo, hi = _phi(orc, "minmod", r), _phi(orc, "superbee", r)
        for lim in ("vanleer", "woodward", "mcbeta", "albada", "venk"):
            p = _phi(orc, lim, r)
            assert lo - 1e-15 <= p <= hi + 1e-15, (lim, r, p, lo, hi)
            assert p <= min(2 * r, 2) + 1e-15  # TVD bound


@pytest.mark.parametrize("lim", SYMMETRIC)
def test_symmetric_limiters(orc, lim):
    for r in (0.1, 0.3, 0.7, 1.3, 2.5, 7.0):
        assert abs(_phi(orc, lim, r) / r - _phi(orc, lim, 1 / r)) < 1e-14, (lim, r)


@pytest.mark.parametrize("lim", ALL)
def test_exact_on_linear_and_bounded(orc, lim):
    x = np.arange(12.0)
    w = 0.3 + 0.7 * x
    wl_, wr_ = orc.reconstruct(lim, w)
    np.testing.assert_allclose(wl_[1:-1], w[1:-1] + 0.35, rtol=0, atol=1e-14)
    np.testing.assert_allclose(wr_[1:-1], w[1:-1] - 0.35, rtol=0, atol=1e-14)
    rng = np.random.Generator(np.random.PCG64(17))
    w = rng.uniform(-1, 1, 300)
    wl_, wr_ = orc.reconstruct(lim, w)
    for i in range(1, 299):
        assert min(w[i], w[i + 1]) - 1e-15 <= wl_[i] <= max(w[i], w[i + 1]) + 1e-15
        assert min(w[i], w[i - 1]) - 1e-15 <= wr_[i] <= max(w[i], w[i - 1]) + 1e-15
        if (w[i] - w[i - 1]) * (w[i + 1] - w[i]) <= 0:
            assert wl_[i] == w[i] and wr_[i] == w[i]
    # mirror: reversing the data swaps the two face states
    wl2, wr2 = orc.reconstruct(lim, w[::-1].copy())
    np.testing.assert_allclose(wl2[1:-1], wr_[::-1][1:-1], rtol=0, atol=1e-15)


def _cp_err(orc, lim, n):
    import math
    from paper_2303_03026_gb300 import workloads as wl
    from util import rel_l1
    W = wl.cp_alfven(n, limiter=lim)
    U, t, ns, st = orc.mesh_for(W, 8).run(W.U, 1 / math.sqrt(2))
    assert st == 0
    _, _, _, Ue = wl.cp_alfven_exact(n, 1 / math.sqrt(2))
    return rel_l1(U[7], Ue[7])


@pytest.mark.parametrize("lim", ["woodward", "mcbeta", "albada", "venk"])
def test_new_limiters_second_order_on_cp_wave(orc, lim):
    import math
    e32, e64 = _cp_err(orc, lim, 32), _cp_err(orc, lim, 64)
    assert math.log2(e32 / e64) > 1.5, (lim, e32, e64)


def test_superbee_overcompresses_smooth_wave(orc):
    # superbee, the upper edge of the TVD region, steepens smooth extrema
    # (sine waves turn into square waves): it still converges, but slower and
    # with a larger error than vanleer on the smooth Alfven wave
    import math
    e32, e64 = _cp_err(orc, "superbee", 32), _cp_err(orc, "superbee", 64)
    assert 0.4 < math.log2(e32 / e64) < 1.5, (e32, e64)
    assert e64 > 1.3 * _cp_err(orc, "vanleer", 64)
