"""Pins of per-level scheme choice (Sect. 3: flux scheme and reconstruction may
differ between AMR levels): every face of a block is computed with its level's
scheme, so each level's blocks must equal, bit for bit, the same stage run with
that level's scheme everywhere; overrides equal to the global choice change
nothing; with refluxing the mixed-scheme mesh still conserves to round-off."""
import numpy as np

from paper_2303_03026_gb300 import workloads as wl


def _stage(orc, W):
    m = orc.mesh_for(W)
    dt, ch = m.cfl(W.U)
    out, st = m.stage(0, dt, ch, W.U, W.U)
    assert st == 0
    return out


def test_each_level_uses_its_scheme(orc):
    W = wl.small_amr_2d()
    levels = W.block_meta[:, 1]
    assert len(set(levels)) >= 2
    W.cfg.level_flux = {1: "hll", 2: "tvdlf"}
    W.cfg.level_limiter = {1: "minmod", 2: "woodward"}
    mixed = _stage(orc, W)
    for L, flux, lim in ((0, "hlld", "vanleer"), (1, "hll", "minmod"), (2, "tvdlf", "woodward")):
        Wr = wl.small_amr_2d()
        Wr.cfg.flux, Wr.cfg.limiter = flux, lim
        ref = _stage(orc, Wr)
        sel = levels == L
        if sel.any():
            assert np.array_equal(mixed[:, sel], ref[:, sel]), L


def test_overrides_equal_to_global_change_nothing(orc):
    W = wl.small_amr_2d()
    base = _stage(orc, W)
    W.cfg.level_flux = {L: W.cfg.flux for L in range(4)}
    W.cfg.level_limiter = {L: W.cfg.limiter for L in range(4)}
    assert np.array_equal(_stage(orc, W), base)


def test_mixed_schemes_conserve_with_reflux(orc):
    W = wl.small_amr_2d()
    W.cfg.level_flux = {2: "hll"}
    W.cfg.reflux = True
    m = orc.mesh_for(W, 4)
    s0 = m.sums(W.U)
    U, t, ns, st = m.run(W.U, 1e30, maxsteps=5)
    assert st == 0
    drift = (np.abs(m.sums(U) - s0) / np.maximum(np.abs(s0), np.abs(s0).max()))[:, :8].max()
    assert drift < 2e-14
