"""Pins of the regridding oracle (oracle/regrid.py) against facts that do not
come from it: the estimator's closed form at a density jump (inside a block and
across a block face, with the sum over directions in the denominator), its
scale invariance and zero on uniform data; the plan's identity, split and
merge counts and 2:1 balance and tiling checked by brute force on random
flags; and the transfer's exact conservation, exactness on linear data and
split-then-merge identity.  The library's host plan (amrvac_regrid_plan)
is compared with the oracle's here too: it needs no GPU.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import regrid as rg
from paper_2303_03026_gb300 import workloads as wl


def _case(ndim, base, bnx, meta, prim, bc="outflow"):
    cfg = wl.Config(ndim=ndim, block_nx=tuple(bnx), flux="hll", limiter="minmod", time="ssprk2",
                    precision="fp64", glm=True, bc=((bc, bc),) * 3)
    inst = wl.Instance(base_blocks=tuple(base), gamma=5.0 / 3.0)
    U = wl._fill_from_function(cfg, [inst], meta, prim)
    return wl.Workload("regrid_case", cfg, [inst], np.ascontiguousarray(meta, np.int32), U)


def _rho_prim(fn):
    def prim(inst, x, y, z):
        rho = fn(x, y, z)
        zero = np.zeros_like(x)
        return wl.conserved_from_primitive(inst.gamma, rho, zero, zero, zero, 1.0 + zero,
                                           0.5 + zero, zero, zero)
    return prim


def _est(orc, W):
    return rg.estimator(orc.mesh_for(W), W.U, W.cfg)


# ----------------------------------------------------------------- estimator
def test_estimator_jump_inside_block_1d(orc):
    # rho = 1 left of x = 0.45, 2 right of it; 4 blocks of 10 cells: the jump
    # lies inside block 1 (between cells 17 and 18).  At the cell left of the jump
    # (p, c, m) = (2, 1, 1): E = 1 / (1 + 0.01 * 5); at the cell right of it
    # (2, 2, 1): E = 1 / (1 + 0.01 * 7); every other cell is flat.
    W = _case(1, (4, 1, 1), (10, 1, 1), wl.uniform_meta((4, 1, 1)),
              _rho_prim(lambda x, y, z: np.where(x < 0.45, 1.0, 2.0)))
    E = _est(orc, W)
    assert E[1] == pytest.approx(1.0 / 1.05, rel=1e-15)
    assert E[0] == 0.0 and E[2] == 0.0 and E[3] == 0.0


def test_estimator_jump_across_block_face_2d(orc):
    # the jump on the face between blocks (x = 0.5): each side sees the other
    # only through its ghost values.  Low side, last cell (p, c, m) = (2, 1, 1):
    # x term 1 / (1 + 0.01 * 5)^2; the flat y direction adds (0.01 * 4)^2 to
    # the denominator.  High side, first cell (2, 2, 1): 1 / (1 + 0.01 * 7)^2
    # and (0.01 * 8)^2 from y.
    W = _case(2, (2, 2, 1), (8, 8, 1), wl.uniform_meta((2, 2, 1)),
              _rho_prim(lambda x, y, z: np.where(x < 0.5, 1.0, 2.0)))
    E = _est(orc, W)
    lo = 1.0 / np.sqrt(1.05 ** 2 + 0.04 ** 2)
    hi = 1.0 / np.sqrt(1.07 ** 2 + 0.08 ** 2)
    for b, r in enumerate(W.block_meta):
        assert E[b] == pytest.approx(lo if r[2] == 0 else hi, rel=1e-14), (b, E)


def _prim_case(rho_fn, vx_fn, p_fn):
    def prim(inst, x, y, z):
        zero = np.zeros_like(x)
        return wl.conserved_from_primitive(inst.gamma, rho_fn(x), vx_fn(x), zero, zero,
                                           p_fn(x), 0.5 + zero, zero, zero)
    return _case(2, (2, 2, 1), (8, 8, 1), wl.uniform_meta((2, 2, 1)), prim)


def test_estimator_weighted_primitives(orc):
    step = lambda lo, hi: (lambda x: np.where(x < 0.5, lo, hi))  # noqa: E731
    lo = 1.0 / np.sqrt(1.05 ** 2 + 0.04 ** 2)
    hi = 1.0 / np.sqrt(1.07 ** 2 + 0.08 ** 2)
    # a pressure jump at the block face under uniform density: the pressure
    # weight sees the closed form of the density case, the density weight 0
    W = _prim_case(lambda x: 1.0 + 0 * x, lambda x: 0 * x, step(1.0, 2.0))
    wp = np.zeros(9)
    wp[4] = 1.0
    E = rg.estimator(orc.mesh_for(W), W.U, W.cfg, weights=wp)
    for b, r in enumerate(W.block_meta):
        assert E[b] == pytest.approx(lo if r[2] == 0 else hi, rel=1e-13)
    assert np.all(_est(orc, W) == 0.0)
    wmix = np.zeros(9)
    wmix[0] = wmix[4] = 0.5
    np.testing.assert_allclose(rg.estimator(orc.mesh_for(W), W.U, W.cfg, weights=wmix),
                               0.5 * E, rtol=1e-15)
    # uniform momentum across a density jump: the velocity (a derived
    # quantity) jumps 1 -> 0.5.  Low side, last cell (p, c, m) = (0.5, 1, 1):
    # 0.5 / sqrt((0.5 + 0.01 * 3.5)^2 + (0.01 * 4)^2); the momentum is flat
    W = _prim_case(step(1.0, 2.0), step(1.0, 0.5), lambda x: 1.0 + 0 * x)
    wv = np.zeros(9)
    wv[1] = 1.0
    E = rg.estimator(orc.mesh_for(W), W.U, W.cfg, weights=wv)
    want_lo = 0.5 / np.sqrt(0.535 ** 2 + 0.04 ** 2)
    assert E[0] == pytest.approx(want_lo, rel=1e-13)
    assert np.all(W.U[1] == 1.0)


def test_estimator_zero_on_uniform_and_scale_invariant(orc):
    W = _case(2, (2, 2, 1), (8, 8, 1), wl.uniform_meta((2, 2, 1)),
              _rho_prim(lambda x, y, z: 1.3 + 0 * x), bc="periodic")
    assert np.all(_est(orc, W) == 0.0)
    W = wl.small_amr_2d()
    E1 = _est(orc, W)
    W.U[0] *= 7.0
    E2 = _est(orc, W)
    assert E1.max() > 1e-3
    # invariant in exact arithmetic; the second difference of smooth data
    # cancels, so the rounding is absolute (relative to rho), not relative to E
    np.testing.assert_allclose(E2, E1, rtol=0, atol=1e-13)


def test_flags_thresholds_and_levels():
    meta = np.array([[0, 0, 0, 0, 0], [0, 1, 0, 0, 0], [0, 2, 0, 0, 0], [0, 2, 1, 0, 0],
                     [0, 0, 1, 0, 0], [0, 1, 1, 0, 0]])
    E = np.array([0.5, 0.5, 0.01, 0.3, 0.001, 0.025])
    f = rg.flags(E, meta, 0.2, 0.125, 2)
    # level 0 never coarsens; level 2 = max_level never refines; 0.025 is not
    # below 0.125 * 0.2
    assert f.tolist() == [1, 1, -1, 0, 0, 0]


# ----------------------------------------------------------------------- plan
def _check_mesh(cfg, inst, meta):
    """Brute force on the finest grid: the leaves tile the domain once, and
    fine cells adjacent across faces, edges or corners (periodic wrap, none
    across outflow edges) belong to leaves at most one level apart."""
    fine = int(max(r[1] for r in meta))
    N = [inst.base_blocks[d] << fine if d < cfg.ndim else 1 for d in range(3)]
    lev = np.full(N[::-1], -1, np.int32)
    for r in meta:
        L = int(r[1])
        s = 1 << (fine - L)
        lo = [int(r[2 + d]) * s if d < cfg.ndim else 0 for d in range(3)]
        hi = [lo[d] + (s if d < cfg.ndim else 1) for d in range(3)]
        box = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        assert np.all(lev[box] == -1), "overlap"
        lev[box] = L
    assert np.all(lev >= 0), "hole"
    rng = [(-1, 0, 1) if d < cfg.ndim else (0,) for d in range(3)]
    for sh in itertools.product(*rng):
        if sh == (0, 0, 0):
            continue
        nb = lev
        for d in range(cfg.ndim):
            if sh[d] == 0:
                continue
            ax = 2 - d
            if cfg.bc[d][0] == "periodic":
                nb = np.roll(nb, sh[d], axis=ax)
            else:
                pad = [(0, 0)] * 3
                pad[ax] = (1, 1)
                sl = [slice(None)] * 3
                nb = np.pad(nb, pad, mode="edge")
                sl[ax] = slice(1 - sh[d], 1 - sh[d] + N[d])
                nb = nb[tuple(sl)]
        assert np.abs(lev - nb).max() <= 1, sh


def test_plan_identity_and_counts():
    W = wl.small_amr_2d()
    inst = W.instances[0]
    nb = W.nblocks
    same = rg.plan(W.cfg, W.instances, W.block_meta, np.zeros(nb, np.int32))
    assert np.array_equal(same, np.array(sorted(map(tuple, W.block_meta), key=rg.block_order),
                                         np.int32))
    # split one level-1 block whose neighbours are all level >= 1: +3 blocks
    f = np.zeros(nb, np.int32)
    b = [i for i, r in enumerate(W.block_meta) if r[1] == 1][0]
    f[b] = 1
    new = rg.plan(W.cfg, W.instances, W.block_meta, f)
    _check_mesh(W.cfg, inst, new)
    assert len(new) >= nb + 3
    # uniform level-1 mesh with every family flagged: back to the base mesh
    base = wl.uniform_meta((3, 2, 1))
    ones = rg.plan(W.cfg, [wl.Instance(base_blocks=(3, 2, 1))], base,
                   np.ones(len(base), np.int32))
    assert len(ones) == 4 * len(base) and np.all(ones[:, 1] == 1)
    back = rg.plan(W.cfg, [wl.Instance(base_blocks=(3, 2, 1))], ones,
                   -np.ones(len(ones), np.int32))
    assert np.array_equal(back, np.array(sorted(map(tuple, base), key=rg.block_order), np.int32))
    # one sibling not asking: that family stays
    f = -np.ones(len(ones), np.int32)
    f[0] = 0
    part = rg.plan(W.cfg, [wl.Instance(base_blocks=(3, 2, 1))], ones, f)
    assert len(part) == len(base) - 1 + 4


def test_plan_split_closure_2to1():
    # a level-1 patch next to level-0 blocks: splitting a level-1 block on the
    # patch edge forces its level-0 neighbours to split
    W = wl.small_amr_2d(base=(4, 4, 1), maxlevel=1)
    inst = W.instances[0]
    lev1 = [i for i, r in enumerate(W.block_meta) if r[1] == 1]
    f = np.zeros(W.nblocks, np.int32)
    f[lev1] = 1
    new = rg.plan(W.cfg, W.instances, W.block_meta, f)
    _check_mesh(W.cfg, inst, new)
    assert new[:, 1].max() == 2
    assert sum(1 for r in new if r[1] == 1) > 0
    n0_before = sum(1 for r in W.block_meta if r[1] == 0)
    n0_after = sum(1 for r in new if r[1] == 0)
    assert n0_after < n0_before  # the closure split level-0 leaves


def test_plan_merge_blocked_by_2to1():
    # a level-2 patch inside level 1: merging the level-1 family that touches
    # it would put level 0 next to level 2, so it is refused
    W = wl.small_amr_2d(base=(8, 8, 1), maxlevel=2)
    f = np.where(W.block_meta[:, 1] == 1, -1, 0).astype(np.int32)
    new = rg.plan(W.cfg, W.instances, W.block_meta, f)
    _check_mesh(W.cfg, W.instances[0], new)
    assert len(new) < W.nblocks            # free families merged
    assert np.any(new[:, 1] == 1)          # those next to level 2 stayed


@pytest.mark.parametrize("seed", range(6))
def test_plan_random_flags_valid(seed):
    rng = np.random.Generator(np.random.PCG64(100 + seed))
    if seed % 2 == 0:
        W = wl.small_amr_2d(base=(3, 4, 1), maxlevel=2, periodic=seed % 4 == 0)
    else:
        W = wl.c4_blast_amr(base=2, levels=3, bnx=4, shell=(0.2, 0.26))
    meta = W.block_meta
    for _ in range(2):
        f = rng.integers(-1, 2, len(meta)).astype(np.int32)
        f[(meta[:, 1] == 0) & (f == -1)] = 0
        f[(meta[:, 1] >= 3) & (f == 1)] = 0
        meta = rg.plan(W.cfg, W.instances, meta, f)
        _check_mesh(W.cfg, W.instances[0], meta)


def test_library_plan_matches_oracle():
    from paper_2303_03026_gb300 import amrvac, build
    build.build()
    rng = np.random.Generator(np.random.PCG64(7))
    for W in (wl.small_amr_2d(base=(3, 4, 1), maxlevel=2),
              wl.small_amr_2d(periodic=False),
              wl.c5_instances(count=5, nmin=32, nmax=96, precision="fp64"),
              wl.c4_blast_amr(base=2, levels=3, bnx=4, shell=(0.2, 0.26)),
              _case(1, (5, 1, 1), (8, 1, 1), wl.uniform_meta((5, 1, 1)),
                    _rho_prim(lambda x, y, z: 1 + x))):
        meta = W.block_meta
        for _ in range(3):
            f = rng.integers(-1, 2, len(meta)).astype(np.int8)
            f[(meta[:, 1] == 0) & (f == -1)] = 0
            got = amrvac.regrid_plan(W.cfg, W.instances, meta, f)
            ref = rg.plan(W.cfg, W.instances, meta, f.astype(np.int32))
            assert np.array_equal(got, ref)
            meta = ref


def test_library_plan_rejects_bad_input():
    import ctypes as C
    from paper_2303_03026_gb300 import amrvac, build
    build.build()
    W = wl.small_amr_2d()
    L = amrvac.load()
    c = amrvac.make_config(W.cfg)
    inst = amrvac.make_instances(W.instances)
    meta = np.ascontiguousarray(W.block_meta, np.int32)
    n = C.c_int32(0)
    out = np.zeros((4, 5), np.int32)

    def call(flags, cap, m=meta):
        fl = np.ascontiguousarray(flags, np.int8)
        return L.amrvac_regrid_plan(C.byref(c), 1, inst, m.shape[0], m.ctypes.data,
                                    fl.ctypes.data, cap, out.ctypes.data, C.byref(n))

    z = np.zeros(len(meta), np.int8)
    assert call(z, 4) == 1 and n.value == len(meta)  # capacity too small: size reported
    bad = z.copy()
    bad[0] = 2
    assert call(bad, 4) == 1
    hole = np.ascontiguousarray(meta[1:])
    assert call(z[1:], 4, hole) == 1


# ------------------------------------------------------------------- transfer
def _integral(W_cfg, inst, meta, U):
    # exactly rounded sums (cell volumes are powers of two here)
    vol = np.array([np.prod(wl.cell_size(W_cfg, inst, int(r[1]))[:W_cfg.ndim]) for r in meta])
    return np.array([math.fsum((U[v] * vol[:, None]).ravel()) for v in range(9)])


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_transfer_conserves(orc, which):
    rng = np.random.Generator(np.random.PCG64(11))
    if which == "2d":
        W = wl.small_amr_2d()
    else:
        W = wl.c4_blast_amr(base=2, levels=3, bnx=4, shell=(0.2, 0.26), precision="fp64")
    inst = W.instances[0]
    f = rng.integers(-1, 2, W.nblocks).astype(np.int32)
    f[(W.block_meta[:, 1] == 0) & (f == -1)] = 0
    new = rg.plan(W.cfg, W.instances, W.block_meta, f)
    assert len(new) != W.nblocks
    Un = rg.transfer(W.cfg, W.instances, W.block_meta, W.U, orc.mesh_for(W), new)
    s0 = _integral(W.cfg, inst, W.block_meta, W.U)
    s1 = _integral(W.cfg, inst, new, Un)
    scale = np.abs(W.U).reshape(9, -1).max(axis=1)
    assert np.all(np.abs(s1 - s0) <= 4e-15 * scale)
    # merged and split blocks both present
    olds = set(map(tuple, W.block_meta))
    kinds = {("copy" if tuple(r) in olds else "new") for r in new}
    assert kinds == {"copy", "new"}


def test_transfer_exact_on_linear_data(orc):
    # linear conserved data: every split child whose parent cell is away from
    # the outflow boundary gets the linear function at its own centre
    W = wl.small_amr_2d(field="linear", periodic=False)
    f = np.ones(W.nblocks, np.int32)
    f[W.block_meta[:, 1] == 2] = 0
    new = rg.plan(W.cfg, W.instances, W.block_meta, f)
    Un = rg.transfer(W.cfg, W.instances, W.block_meta, W.U, orc.mesh_for(W), new)
    inst = W.instances[0]
    exact = wl._fill_from_function(W.cfg, W.instances, new,
                                   lambda i, x, y, z: np.stack(
                                       [1.0 + 0.1 * x + 0.05 * y, 0.1 * x, 0.2 * y, 0 * x,
                                        2.0 + 0.3 * x - 0.1 * y, 0.5 + 0 * x, 0.2 * x, 0.1 * y,
                                        0.01 * x]))
    checked = 0
    for b, r in enumerate(new):
        X, Y, _ = wl.cell_centres(W.cfg, inst, r)
        h = wl.cell_size(W.cfg, inst, int(r[1]))
        # away from the outflow edges, where zero-gradient ghosts flatten the
        # slopes of parents and of coarse ghost stencils
        m = 8
        inner = ((X > m * h[0]) & (X < 1 - m * h[0]) & (Y > m * h[1]) &
                 (Y < 1 - m * h[1])).ravel()
        err = np.abs(Un[:, b, inner] - exact[:, b, inner]).max() if inner.any() else 0.0
        assert err < 1e-14, (b, r, err)
        checked += inner.sum()
    assert checked > 1000


def test_split_then_merge_is_identity(orc):
    W = wl.small_amr_2d()
    f = np.ones(W.nblocks, np.int32)
    f[W.block_meta[:, 1] == 2] = 0
    mid = rg.plan(W.cfg, W.instances, W.block_meta, f)
    Um = rg.transfer(W.cfg, W.instances, W.block_meta, W.U, orc.mesh_for(W), mid)
    split = {tuple(r) for r in W.block_meta} - {tuple(r) for r in mid}
    back_f = np.array([-1 if (r[0], r[1] - 1, r[2] >> 1, r[3] >> 1, r[4] >> 1) in split else 0
                       for r in mid], np.int32)
    Wm = wl.Workload("mid", W.cfg, W.instances, mid, Um)
    back = rg.plan(W.cfg, W.instances, mid, back_f)
    Ub = rg.transfer(W.cfg, W.instances, mid, Um, orc.mesh_for(Wm), back)
    ref = {tuple(r): b for b, r in enumerate(W.block_meta)}
    scale = np.abs(W.U).max()
    merged = 0
    for b, r in enumerate(back):
        if tuple(r) in ref:
            assert np.abs(Ub[:, b] - W.U[:, ref[tuple(r)]]).max() <= 4e-15 * scale
            merged += tuple(r) in split
    assert merged >= 8


def test_library_plan_level_limit():
    # a 1D chain refined towards x = 0 through all 16 levels: splitting a
    # level-15 block is refused, splitting the coarser ones is not
    from paper_2303_03026_gb300 import amrvac, build
    build.build()
    meta = wl.amr_meta(1, (2, 1, 1), 15, lambda L, i, j, k: i == 0, periodic=False)
    cfg = wl.Config(ndim=1, block_nx=(8, 1, 1), bc=(("outflow", "outflow"),) * 3)
    inst = [wl.Instance(base_blocks=(2, 1, 1))]
    assert meta[:, 1].max() == 15
    f = np.where(meta[:, 1] == 15, 1, 0).astype(np.int8)
    with pytest.raises(amrvac.AmrvacError):
        amrvac.regrid_plan(cfg, inst, meta, f)
    f = np.where(meta[:, 1] == 14, 1, 0).astype(np.int8)
    got = amrvac.regrid_plan(cfg, inst, meta, f)
    assert np.array_equal(got, rg.plan(cfg, inst, meta, f.astype(np.int32)))
    _check_mesh(cfg, inst[0], got)


def test_library_plan_at_full_3d_size():
    # the 3D AMR blast mesh of the benchmark (18,304 blocks over 4 levels) with
    # random flags: the library's plan equals the oracle's and is a 2:1-balanced
    # tiling of the domain
    from paper_2303_03026_gb300 import amrvac, build
    build.build()
    W = wl.c4_blast_amr(base=6, precision="fp32")
    rng = np.random.Generator(np.random.PCG64(3))
    f = rng.integers(-1, 2, W.nblocks).astype(np.int8)
    f[(W.block_meta[:, 1] == 0) & (f == -1)] = 0
    got = amrvac.regrid_plan(W.cfg, W.instances, W.block_meta, f)
    assert np.array_equal(got, rg.plan(W.cfg, W.instances, W.block_meta, f.astype(np.int32)))
    _check_mesh(W.cfg, W.instances[0], got)
    assert len(got) > W.nblocks
