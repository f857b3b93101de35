"""Pins of the oracle's bootstrapping (fix_small_values, Sect. 7.4): the replace
and average methods on planted small cells, checked by brute force on the
primitives of the neighbouring cells, plus invariants (B and psi untouched,
other cells untouched, identity when nothing is small) and a near-vacuum run
that fails without the fix and completes with it.
"""
import numpy as np
import pytest

from paper_2303_03026_gb300 import workloads as wl

SD, SP = 1e-6, 1e-4


def _case():
    W = wl.cp_alfven(32)
    W.cfg.small_density, W.cfg.small_pressure = SD, SP
    return W


def _plant_negative_pressure(orc, W, b, c):
    g = W.instances[0].gamma
    u = W.U[:, b, c].copy()
    w = orc.cons_to_prim(g, u)
    w[4] = -0.05
    W.U[:, b, c] = orc.prim_to_cons(g, w)


def _block_at(W, L, i, j):
    for b, r in enumerate(W.block_meta):
        if r[1] == L and r[2] == i and r[3] == j:
            return b
    raise KeyError((L, i, j))


def _face_neighbours(W, b, c):
    """(block, cell) of the same-level face neighbours of cell c of block b
    (periodic unit square, single level)."""
    nx = W.cfg.block_nx[0]
    nbx = W.instances[0].base_blocks[0]
    L, bi, bj = W.block_meta[b][1], W.block_meta[b][2], W.block_meta[b][3]
    i, j = c % nx, c // nx
    out = []
    for d in range(2):
        for s in (-1, 1):
            gi, gj = bi * nx + i, bj * nx + j
            if d == 0:
                gi = (gi + s) % (nbx * nx)
            else:
                gj = (gj + s) % (nbx * nx)
            nb = _block_at(W, L, gi // nx, gj // nx)
            out.append((nb, (gj % nx) * nx + gi % nx))
    return out


def test_identity_when_nothing_is_small(orc):
    W = _case()
    m = orc.mesh_for(W)
    for method in ("replace", "average"):
        U, n = m.fix_small(W.U, method)
        assert n == 0 and np.array_equal(U, W.U)


def test_replace_floors_pressure_keeps_rho_v_b(orc):
    W = _case()
    _plant_negative_pressure(orc, W, 0, 5 * 16 + 5)
    m = orc.mesh_for(W)
    U, n = m.fix_small(W.U, "replace")
    assert n == 1
    g = W.instances[0].gamma
    w0 = orc.cons_to_prim(g, W.U[:, 0, 85])
    w1 = orc.cons_to_prim(g, U[:, 0, 85])
    assert abs(w1[4] - SP) < 1e-12 * SP
    np.testing.assert_allclose(w1[:4], w0[:4], rtol=1e-14)
    assert np.array_equal(U[5:, 0, 85], W.U[5:, 0, 85])  # B, psi untouched
    mask = np.ones(U.shape[1:], bool)
    mask[0, 85] = False
    assert np.array_equal(U[:, mask], W.U[:, mask])


def test_replace_non_positive_density(orc):
    W = _case()
    W.U[0, 1, 3] = -1e-3
    m = orc.mesh_for(W)
    U, n = m.fix_small(W.U, "replace")
    assert n == 1
    w = orc.cons_to_prim(W.instances[0].gamma, U[:, 1, 3])
    assert w[0] == SD and np.all(w[1:4] == 0.0) and abs(w[4] - SP) < 1e-12 * SP


@pytest.mark.parametrize("cell", [5 * 16 + 5, 7 * 16 + 15, 0])
def test_average_is_mean_of_face_neighbours(orc, cell):
    # interior cell, a cell on the +x block edge, a corner cell (periodic wrap)
    W = _case()
    _plant_negative_pressure(orc, W, 0, cell)
    m = orc.mesh_for(W)
    U, n = m.fix_small(W.U, "average")
    assert n == 1
    g = W.instances[0].gamma
    nbrs = [orc.cons_to_prim(g, W.U[:, b, c]) for b, c in _face_neighbours(W, 0, cell)]
    mean = np.mean(np.array(nbrs)[:, :5], axis=0)
    w = orc.cons_to_prim(g, U[:, 0, cell])
    np.testing.assert_allclose(w[:5], mean, rtol=1e-13)
    assert np.array_equal(U[5:, 0, cell], W.U[5:, 0, cell])


def test_average_skips_small_neighbours(orc):
    W = _case()
    a, b = 5 * 16 + 5, 5 * 16 + 6  # two x-neighbours, both small
    _plant_negative_pressure(orc, W, 0, a)
    _plant_negative_pressure(orc, W, 0, b)
    m = orc.mesh_for(W)
    U, n = m.fix_small(W.U, "average")
    assert n == 2
    g = W.instances[0].gamma
    nbrs = [orc.cons_to_prim(g, W.U[:, bb, c]) for bb, c in _face_neighbours(W, 0, a)
            if (bb, c) != (0, b)]
    assert len(nbrs) == 3
    w = orc.cons_to_prim(g, U[:, 0, a])
    np.testing.assert_allclose(w[:5], np.mean(np.array(nbrs)[:, :5], axis=0), rtol=1e-13)


def _vacuum_run(orc, fix):
    # double rarefaction at Mach ~ 7 (two streams leaving the centre): the
    # centre empties and the scheme produces negative pressures there
    W = wl.riemann_1d((1.0, -5.0, 0, 0, 0.4, 0, 0), (1.0, 5.0, 0, 0, 0.4, 0, 0), n=200,
                      gamma=1.4, bx=0.0, t_end=0.1, flux="hll", time="ssprk3")
    W.cfg.small_density, W.cfg.small_pressure = 1e-8, 1e-8
    W.cfg.fix_small_values = fix
    m = orc.mesh_for(W)
    return m.run(W.U, 0.1)


def test_vacuum_run_needs_the_fix(orc):
    U, t, ns, st = _vacuum_run(orc, "off")
    assert st == 4  # small values reported, run stopped
    for method in ("replace", "average"):
        U, t, ns, st = _vacuum_run(orc, method)
        assert st == 0 and abs(t[0] - 0.1) < 1e-14, (method, st, t)
        w = np.array([orc.cons_to_prim(1.4, U[:, 0, c]) for c in range(U.shape[2])])
        assert w[:, 0].min() >= 1e-8 and w[:, 4].min() >= 1e-8
        # mirror symmetry of the problem survives the fix
        np.testing.assert_allclose(w[:, 0], w[::-1, 0], rtol=1e-9, atol=1e-12)
