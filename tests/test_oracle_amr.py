"""Pins of the oracle's block mesh and AMR ghost values.

* same-level ghosts against brute-force indexing of one global periodic array;
* restriction and prolongation reproduce a linear field exactly (the minmod
  slopes of linear data are the exact slopes, the mean of the children of a
  linear field is the parent's centre value);
* symmetric data on a symmetric AMR mesh stays symmetric (x <-> y).
"""
import math

import numpy as np
import pytest

from paper_2303_03026_gb300 import workloads as wl


def _ghost_centres(W, b):
    """Centres (x, y, z) of the padded box of block b, shaped like the padding."""
    cfg = W.cfg
    inst = W.instances[int(W.block_meta[b, 0])]
    L = int(W.block_meta[b, 1])
    dx = wl.cell_size(cfg, inst, L)
    axes = []
    for d in range(3):
        if d >= cfg.ndim:
            axes.append(np.zeros(1))
            continue
        nx = cfg.block_nx[d]
        i0 = int(W.block_meta[b, 2 + d]) * nx
        idx = np.arange(-2, nx + 2) + i0
        axes.append(inst.xmin[d] + (idx + 0.5) * dx[d])
    z, y, x = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return x, y, z


def _face_mask(W):
    nx = [W.cfg.block_nx[d] if d < W.cfg.ndim else 1 for d in range(3)]
    g = [2 if d < W.cfg.ndim else 0 for d in range(3)]
    k, j, i = np.meshgrid(np.arange(-g[2], nx[2] + g[2]), np.arange(-g[1], nx[1] + g[1]),
                          np.arange(-g[0], nx[0] + g[0]), indexing="ij")
    out = ((i < 0) | (i >= nx[0])).astype(int) + ((j < 0) | (j >= nx[1])) + \
        ((k < 0) | (k >= nx[2]))
    return out == 1


def test_same_level_ghosts_brute_force(orc):
    # 2D periodic 4x3 blocks of 8x8, random data: ghosts index a global array
    rng = np.random.Generator(np.random.PCG64(21))
    cfg = wl.Config(ndim=2, block_nx=(8, 8, 1))
    inst = wl.Instance(base_blocks=(4, 3, 1))
    meta = wl.uniform_meta((4, 3, 1))
    G = rng.standard_normal((9, 24, 32))  # [var][y][x]
    U = np.zeros((9, 12, 64))
    for b, (_, _, bi, bj, _) in enumerate(meta):
        U[:, b] = G[:, bj * 8:(bj + 1) * 8, bi * 8:(bi + 1) * 8].reshape(9, 64)
    m = orc.Mesh(cfg, [inst], meta)
    P = m.fill_ghosts(U).reshape(9, 12, 12, 12)
    mask = _face_mask(wl.Workload("x", cfg, [inst], meta, U))[0]
    for b, (_, _, bi, bj, _) in enumerate(meta):
        ys = (np.arange(-2, 10) + bj * 8) % 24
        xs = (np.arange(-2, 10) + bi * 8) % 32
        ref = G[:, ys][:, :, xs]
        np.testing.assert_array_equal(P[:, b][:, mask], ref[:, mask])
    # outflow: ghosts copy the nearest in-domain cell of the same row
    cfg.bc = (("outflow", "outflow"),) * 3
    m = orc.Mesh(cfg, [inst], meta)
    P = m.fill_ghosts(U).reshape(9, 12, 12, 12)
    for b, (_, _, bi, bj, _) in enumerate(meta):
        ys = np.clip(np.arange(-2, 10) + bj * 8, 0, 23)
        xs = np.clip(np.arange(-2, 10) + bi * 8, 0, 31)
        ref = G[:, ys][:, :, xs]
        np.testing.assert_array_equal(P[:, b][:, mask], ref[:, mask])


@pytest.mark.parametrize("ndim", [2, 3])
def test_amr_ghosts_exact_for_linear_field(orc, ndim):
    if ndim == 2:
        W = wl.small_amr_2d(field="linear", periodic=False)
        lin = lambda x, y, z: np.stack([1.0 + 0.1 * x + 0.05 * y, 0.1 * x, 0.2 * y, 0 * x,
                                        2.0 + 0.3 * x - 0.1 * y, 0.5 + 0 * x, 0.2 * x,
                                        0.1 * y, 0.01 * x])
    else:
        W = wl.c4_blast_amr(base=4, levels=3, bnx=4, shell=(0.2, 0.26))
        W.cfg.bc = (("outflow", "outflow"),) * 3
        lin = lambda x, y, z: np.stack([1 + 0.2 * x - 0.1 * y + 0.3 * z, x, y, z,
                                        3 + x + y + z, 0.5 * z, -0.2 * x, 0.1 * y, 0 * x])
        for b in range(W.nblocks):
            x, y, z = wl.cell_centres(W.cfg, W.instances[0], W.block_meta[b])
            W.U[:, b] = lin(x, y, z).reshape(9, -1)
    levels = W.block_meta[:, 1]
    assert levels.min() < levels.max()  # a real multi-level mesh
    m = orc.mesh_for(W)
    P = m.fill_ghosts(W.U)
    mask = _face_mask(W).ravel()
    hc = 1.0 / (W.instances[0].base_blocks[0] * W.cfg.block_nx[0])  # coarsest cell
    checked = 0
    for b in range(W.nblocks):
        x, y, z = _ghost_centres(W, b)
        inside = np.ones(x.shape, bool)
        for c, d in ((x, 0), (y, 1), (z, 2)):
            if d < W.cfg.ndim:
                inside &= (c > 3.5 * hc) & (c < 1 - 3.5 * hc)
        sel = mask & inside.ravel()
        ref = lin(x, y, z).reshape(9, -1)
        np.testing.assert_allclose(P[:, b][:, sel], ref[:, sel], rtol=0, atol=1e-13)
        checked += sel.sum()
    assert checked > 100


def test_blast_xy_mirror_symmetry(orc):
    # blast with B0 along (1,1,0) on a mesh symmetric under x <-> y: the state
    # after one SSPRK3 step is symmetric to round-off
    W = wl.c4_blast_amr(base=4, levels=3, bnx=4, shell=(0.2, 0.26), precision="fp64")
    m = orc.mesh_for(W, 8)
    U, t, ns, st = m.run(W.U, 1.0, maxsteps=1)
    assert ns == 1 and st == 0
    key = {tuple(r[1:]): b for b, r in enumerate(W.block_meta)}
    n = 4
    worst = 0.0
    for b, r in enumerate(W.block_meta):
        L, i, j, k = (int(v) for v in r[1:])
        bm = key[(L, j, i, k)]
        A = U[:, b].reshape(9, n, n, n)
        B = U[:, bm].reshape(9, n, n, n).transpose(0, 1, 3, 2)  # swap x, y cells
        # swap the x and y vector components
        B = B[[0, 2, 1, 3, 4, 6, 5, 7, 8]]
        scale = np.abs(U).reshape(9, -1).max(axis=1)[:, None, None, None]
        worst = max(worst, float((np.abs(A - B) / np.maximum(scale, 1e-300)).max()))
    assert worst < 1e-12, worst
