"""Oracle of dynamic regridding (block AMR, Sect. 1 and 3: blocks are refined
and coarsened automatically on chosen plasma quantities).

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): plain numpy loops over
blocks and cells, no code shared with the GPU library.

The paper names the capability (automatic (de)refinement on weighted,
user-chosen plasma quantities, Sect. 1 and 3) but prints no criterion or
operator.  This restates the published methods below, with these readings of
the paper where it is silent:
  * estimator (Loehner 1987, the normalised second derivative, per direction):
      E_i(q) = sqrt( sum_d (q_{i+1} - 2 q_i + q_{i-1})^2 /
                     sum_d (|q_{i+1} - q_i| + |q_i - q_{i-1}|
                            + eps (|q_{i+1}| + 2 |q_i| + |q_{i-1}|))^2 )
    with eps = 0.01, summed over the primitive quantities q the caller
    weights (the paper's weighted, user-chosen quantities; default the
    density alone), neighbours across block faces from the conserved ghost
    values of the level (same operators as the update); a block's estimator
    is the maximum over its cells;
  * flags: refine when E > refine_threshold (and the level is below
    max_level), coarsen when E < derefine_ratio * refine_threshold (level > 0);
  * plan: refined blocks, then every block closer than one block (faces, edges,
    corners) to a block two levels finer is refined too until the mesh is 2:1
    balanced; a family of 2^d sibling leaves is coarsened only when all of
    them ask for it, none is refined, and the parent would stay 2:1 balanced,
    families tried in (instance, level, k, j, i) order of the parent and one
    level per regrid (a deterministic order: the paper gives none); the new
    list is sorted by (instance, level, k, j, i);
  * transfer: a block kept is copied; a refined block's children get the
    coarse value plus minmod-limited slopes times +-1/4 (the slopes from the
    block's own neighbours at its level, ghost values across its faces); a
    coarsened family's parent gets the mean of the children.  Every variable's
    integral is conserved exactly (up to rounding).
"""
from __future__ import annotations

import numpy as np

EPS = 0.01


def _nx(cfg):
    return [cfg.block_nx[d] if d < cfg.ndim else 1 for d in range(3)]


def _padded_block(m, Up, b, cfg):
    """Conserved values of block b with its ghost layers from the oracle's ghost
    fill (m.ng per active face; edges/corners unused)."""
    nx = _nx(cfg)
    g = [m.ng if d < cfg.ndim else 0 for d in range(3)]
    P = [nx[d] + 2 * g[d] for d in range(3)]
    return Up[:, b, :].reshape(9, P[2], P[1], P[0]), g


def _primitive(Pb, gamma):
    """Primitive (rho, v, p, B, psi) of conserved cells (ideal MHD, magnetic
    pressure B^2/2), numpy over whole arrays."""
    rho = Pb[0]
    with np.errstate(all="ignore"):  # unused zero edge/corner ghosts
        v = Pb[1:4] / rho
        ke = 0.5 * (Pb[1] * Pb[1] + Pb[2] * Pb[2] + Pb[3] * Pb[3]) / rho
    me = 0.5 * (Pb[5] * Pb[5] + Pb[6] * Pb[6] + Pb[7] * Pb[7])
    p = (gamma - 1.0) * (Pb[4] - ke - me)
    return np.concatenate([rho[None], v, p[None], Pb[5:9]])


def estimator(orc_mesh, U, cfg, weights=None):
    """Per-block maximum over cells of the weighted sum of Loehner estimators
    of the primitive variables (weights[9] over rho, v_x, v_y, v_z, p, B_x, B_y,
    B_z, psi; default the density alone).  A variable whose denominator
    vanishes (flat and zero) contributes 0."""
    w = np.zeros(9)
    if weights is None:
        w[0] = 1.0
    else:
        w[:] = weights
    Up = orc_mesh.fill_ghosts(U)
    nb = U.shape[1]
    nx = _nx(cfg)
    out = np.zeros(nb)
    for b in range(nb):
        Pb, g = _padded_block(orc_mesh, Up, b, cfg)
        if np.any(w[1:] != 0):
            Wb = _primitive(Pb, orc_mesh.instances[int(orc_mesh.meta[b][0])].gamma)
        else:
            Wb = Pb  # density only: the conserved density is the primitive one
        E = np.zeros((nx[2], nx[1], nx[0]))
        for var in range(9):
            if w[var] == 0:
                continue
            q = Wb[var]
            num = np.zeros((nx[2], nx[1], nx[0]))
            den = np.zeros_like(num)
            for d in range(cfg.ndim):
                sl = [slice(g[2], g[2] + nx[2]), slice(g[1], g[1] + nx[1]),
                      slice(g[0], g[0] + nx[0])]
                ax = 2 - d
                c = q[tuple(sl)]
                slp = list(sl)
                slp[ax] = slice(sl[ax].start + 1, sl[ax].stop + 1)
                slm = list(sl)
                slm[ax] = slice(sl[ax].start - 1, sl[ax].stop - 1)
                p, mm = q[tuple(slp)], q[tuple(slm)]
                num += (p - 2 * c + mm) ** 2
                den += (np.abs(p - c) + np.abs(c - mm) +
                        EPS * (np.abs(p) + 2 * np.abs(c) + np.abs(mm))) ** 2
            with np.errstate(all="ignore"):
                r = np.where(den > 0, num / den, 0.0)
            E += w[var] * np.sqrt(r)
        out[b] = E.max()
    return out


def flags(E, meta, refine_threshold, derefine_ratio, max_level):
    f = np.zeros(len(E), np.int32)
    for b, e in enumerate(E):
        L = meta[b][1]
        if e > refine_threshold and L < max_level:
            f[b] = 1
        elif e < derefine_ratio * refine_threshold and L > 0:
            f[b] = -1
    return f


def block_order(key):
    """Sort key of a block (instance, level, i, j, k): instance, level, then
    k, j, i (the last index fastest, like cells in a block)."""
    q, L, i, j, k = key
    return (q, L, k, j, i)


def plan(cfg, instances, meta, fl):
    """New block list (sorted by instance, level, k, j, i) from the flags."""
    nd = cfg.ndim
    leaves = {tuple(int(v) for v in r): b for b, r in enumerate(meta)}

    def nblk(q, L, d):
        return instances[q].base_blocks[d] << L if d < nd else 1

    def periodic(d):
        return cfg.bc[d][0] == "periodic"

    def neighbours(q, L, i, j, k):
        rng = [(-1, 0, 1) if d < nd else (0,) for d in range(3)]
        for dz in rng[2]:
            for dy in rng[1]:
                for dx in rng[0]:
                    if dx == dy == dz == 0:
                        continue
                    p = [i + dx, j + dy, k + dz]
                    ok = True
                    for d in range(nd):
                        n = nblk(q, L, d)
                        if p[d] < 0 or p[d] >= n:
                            if periodic(d):
                                p[d] %= n
                            else:
                                ok = False
                    if ok:
                        yield tuple(p)

    def leaf_covering(q, L, p):
        # the leaf at level <= L covering the level-L position p, or None
        # when finer leaves cover it
        pp = list(p)
        for LL in range(L, -1, -1):
            key = (q, LL, pp[0], pp[1], pp[2])
            if key in cur:
                return key
            pp = [v >> 1 for v in pp]
        return None

    cur = dict(leaves)  # current leaf set: key -> anything
    refine = {tuple(int(v) for v in meta[b]) for b in range(len(meta)) if fl[b] == 1}
    # 2:1 after refinement: a refined block's neighbours one level coarser must
    # refine too (their children would touch level L+1 otherwise)
    changed = True
    while changed:
        changed = False
        for key in list(refine):
            q, L, i, j, k = key
            for p in neighbours(q, L, i, j, k):
                lc = leaf_covering(q, L, p)
                if lc is not None and lc[1] < L and lc not in refine:
                    refine.add(lc)
                    changed = True
    new = set()
    for key in cur:
        if key in refine:
            q, L, i, j, k = key
            for oz in range(2 if nd > 2 else 1):
                for oy in range(2 if nd > 1 else 1):
                    for ox in range(2):
                        new.add((q, L + 1, 2 * i + ox, 2 * j + oy if nd > 1 else 0,
                                 2 * k + oz if nd > 2 else 0))
        else:
            new.add(key)
    # coarsening: complete families of leaves asking for it
    want = {tuple(int(v) for v in meta[b]) for b in range(len(meta)) if fl[b] == -1}
    parents = {}
    for key in want:
        if key in refine or key[1] == 0:
            continue
        q, L, i, j, k = key
        parents.setdefault((q, L - 1, i >> 1, j >> 1, k >> 1), []).append(key)
    nchild = 2 ** nd
    newset = set(new)

    def covering_in(s, q, L, p):
        pp = list(p)
        for LL in range(L, -1, -1):
            if (q, LL, pp[0], pp[1], pp[2]) in s:
                return LL
            pp = [v >> 1 for v in pp]
        return None

    def finest_near(s, q, L, i, j, k):
        # deepest leaf level among the positions around parent (q, L, i, j, k)
        best = L
        for p in neighbours(q, L, i, j, k):
            lev = covering_in(s, q, L, p)
            if lev is None:  # finer leaves there: look one level deeper
                for oz in range(2 if nd > 2 else 1):
                    for oy in range(2 if nd > 1 else 1):
                        for ox in range(2):
                            c = (2 * p[0] + ox, 2 * p[1] + oy if nd > 1 else 0,
                                 2 * p[2] + oz if nd > 2 else 0)
                            l2 = covering_in(s, q, L + 1, c)
                            best = max(best, L + 2 if l2 is None else l2)
            else:
                best = max(best, lev)
        return best

    for par in sorted(parents, key=block_order):
        kids = parents[par]
        if len(kids) != nchild or any(c not in newset for c in kids):
            continue
        trial = (newset - set(kids)) | {par}
        q, L, i, j, k = par
        if finest_near(trial, q, L, i, j, k) <= L + 1:
            newset = trial
    return np.array(sorted(newset, key=block_order), np.int32)


def transfer(cfg, instances, old_meta, Uold, orc_mesh, new_meta, only=None):
    """State of the new mesh from the old one (copy / prolongation / restriction).
    ``only``: indices of the new blocks to compute (the others stay 0)."""
    nd = cfg.ndim
    nx = _nx(cfg)
    ncell = nx[0] * nx[1] * nx[2]
    old = {tuple(int(v) for v in r): b for b, r in enumerate(old_meta)}
    Up = orc_mesh.fill_ghosts(Uold)
    out = np.zeros((9, len(new_meta), ncell))
    for nb, r in enumerate(new_meta):
        if only is not None and nb not in only:
            continue
        key = tuple(int(v) for v in r)
        q, L, i, j, k = key
        if key in old:
            out[:, nb] = Uold[:, old[key]]
            continue
        pkey = (q, L - 1, i >> 1, j >> 1, k >> 1)
        if pkey in old:
            # refined: prolongation from the parent's cells and slopes
            Pb, g = _padded_block(orc_mesh, Up, old[pkey], cfg)
            off = [(i & 1) * nx[0] // 2, (j & 1) * nx[1] // 2 if nd > 1 else 0,
                   (k & 1) * nx[2] // 2 if nd > 2 else 0]
            for c in range(ncell):
                ci = [c % nx[0], (c // nx[0]) % nx[1], c // (nx[0] * nx[1])]
                pc = [off[d] + ci[d] // 2 if d < nd else 0 for d in range(3)]
                val = Pb[:, g[2] + pc[2], g[1] + pc[1], g[0] + pc[0]].copy()
                base = val.copy()
                for d in range(nd):
                    idx_p = [g[2] + pc[2], g[1] + pc[1], g[0] + pc[0]]
                    idx_m = list(idx_p)
                    idx_p[2 - d] += 1
                    idx_m[2 - d] -= 1
                    up, um = Pb[:, idx_p[0], idx_p[1], idx_p[2]], Pb[:, idx_m[0], idx_m[1], idx_m[2]]
                    a, bb = base - um, up - base
                    slope = np.where(a * bb > 0, np.where(a > 0, np.minimum(a, bb), np.maximum(a, bb)), 0.0)
                    w = 0.25 if ci[d] % 2 == 1 else -0.25
                    val = val + w * slope
                out[:, nb, c] = val
            continue
        # coarsened: mean of the 2^d children
        acc = np.zeros((9, ncell))
        n = 0
        for oz in range(2 if nd > 2 else 1):
            for oy in range(2 if nd > 1 else 1):
                for ox in range(2):
                    ck = (q, L + 1, 2 * i + ox, 2 * j + oy if nd > 1 else 0, 2 * k + oz if nd > 2 else 0)
                    cb = old[ck]
                    for c in range(ncell):
                        ci = [c % nx[0], (c // nx[0]) % nx[1], c // (nx[0] * nx[1])]
                        # child cell ci covers parent cell (off + ci // 2)
                        pc = [(ox * nx[0] + ci[0]) // 2, (oy * nx[1] + ci[1]) // 2 if nd > 1 else 0,
                              (oz * nx[2] + ci[2]) // 2 if nd > 2 else 0]
                        pcell = (pc[2] * nx[1] + pc[1]) * nx[0] + pc[0]
                        acc[:, pcell] += Uold[:, cb, c]
                    n += 1
        out[:, nb] = acc / (2 ** nd)
    return out
