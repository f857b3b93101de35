"""Pins of the oracle's refluxing (conservative flux correction at coarse-fine
faces): a periodic AMR mesh conserves every conserved variable to round-off
with it and visibly does not without it (so a wrong sign, a wrong fine-flux
index or a missing second-output correction fails here); it is a bitwise no-op
on a single level and keeps a uniform flow uniform.
"""
import numpy as np
import pytest

from paper_2303_03026_gb300 import workloads as wl


def _drift(orc, W, steps):
    m = orc.mesh_for(W, 8)
    s0 = m.sums(W.U)
    U, t, ns, st = m.run(W.U, 1e30, maxsteps=steps)
    assert st == 0 and ns == steps
    s1 = m.sums(U)
    # per variable, floored by the mean magnitude of the whole state (momentum
    # starts at zero in the blast)
    scale = np.maximum(np.abs(s0), np.abs(W.U).reshape(9, -1).mean(axis=1)[None, :])
    scale = np.maximum(scale, np.abs(s0).max())
    return (np.abs(s1 - s0) / scale)[:, :8].max()


@pytest.mark.parametrize("time", ["ssprk3", "ssprk54"])
def test_reflux_conserves_on_amr_2d(orc, time):
    W = wl.small_amr_2d()
    W.cfg.time = time
    W.cfg.reflux = True
    assert _drift(orc, W, 6) < 2e-14
    W.cfg.reflux = False
    assert _drift(orc, W, 6) > 1e-9  # level changes without refluxing leak


def _advected_3d(orc):
    # the 3D three-level mesh with a density wave advected across its level
    # changes (uniform velocity and pressure, B along the flow)
    W = wl.c4_blast_amr(base=4, levels=3, bnx=4, shell=(0.2, 0.26), precision="fp64")
    g = W.instances[0].gamma
    for b in range(W.U.shape[1]):
        X, Y, Z = wl.cell_centres(W.cfg, W.instances[0], W.block_meta[b])
        rho = (1.0 + 0.3 * np.sin(2 * np.pi * (X + Y + Z))).ravel()
        for c in range(W.U.shape[2]):
            w = np.array([rho[c], 0.5, 0.3, 0.2, 1.0, 0.5, 0.3, 0.2, 0.0])
            W.U[:, b, c] = orc.prim_to_cons(g, w)
    return W


def test_reflux_conserves_on_amr_3d(orc):
    W = _advected_3d(orc)
    W.cfg.reflux = True
    assert _drift(orc, W, 3) < 2e-14
    W.cfg.reflux = False
    assert _drift(orc, W, 3) > 1e-9


def test_reflux_noop_on_single_level(orc):
    W = wl.cp_alfven(32)
    U0, *_ = orc.mesh_for(W).run(W.U, 1e30, maxsteps=2)
    W.cfg.reflux = True
    U1, *_ = orc.mesh_for(W).run(W.U, 1e30, maxsteps=2)
    assert np.array_equal(U0, U1)


def test_reflux_keeps_free_stream(orc):
    W = wl.small_amr_2d(field="uniform")
    W.cfg.reflux = True
    m = orc.mesh_for(W)
    dt, ch = m.cfl(W.U)
    out, st = m.stage(0, dt, ch, W.U, W.U)
    out, st = m.stage(0, dt, ch, W.U, W.U)  # a full-mesh stage refluxes
    assert np.abs(out - W.U).max() < 1e-14 * np.abs(W.U).max()
