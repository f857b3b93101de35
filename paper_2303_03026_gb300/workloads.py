"""Seeded synthetic inputs for the ideal-MHD block update.

This module only builds inputs: block lists (the mesh), per-instance domain
descriptions and initial conserved states.  It contains none of the update's
arithmetic (no reconstruction, Riemann flux, stage update or time step).  Both
the CUDA path and the CPU oracle are fed from here, so that the two sides see
identical bits.

Conserved state layout everywhere: ``U[var, block, cell]`` with the nine
variables (rho, m_x, m_y, m_z, e, B_x, B_y, B_z, psi) and cells ordered
x-fastest inside a block.  Magnetic field units make the magnetic pressure
B^2/2, so the total energy density of an initial state is
e = p/(gamma-1) + rho v^2/2 + B^2/2 (the definition of the conserved energy
in the ideal-MHD system the paper evolves, Sect. 2 and Sect. 3).

Workloads (stand-ins for the paper's 2D/3D MHD runs, whose data files are not
public inputs; all seeds fixed):

* ``c1_riemann``     1D, 512 cells, one block, outflow, seeded MHD shock tube.
* ``c2_orszag_tang`` 2D Orszag-Tang vortex, 1024^2 in 16^2 blocks, periodic.
* ``cp_alfven``      2D circularly polarised Alfven wave (exact solution),
                     the smooth convergence test of Sect. 3 (via Porth 2014).
* ``c3_turbulence``  3D 256^3 random-phase solenoidal Mach-1 flow, beta 0.01.
* ``c4_blast_amr``   3D block-AMR (4 levels, ratio 2) around a blast shell.
* ``c5_instances``   256 independent uneven 2D problems (64^2 .. 512^2).
* ``shu_osher``      1D Shu-Osher IC printed in Sect. 3.1.1 (B = 0).
"""
from __future__ import annotations

import math
from collections import deque
from dataclasses import dataclass, field

import numpy as np

NVAR = 9
RHO, MX, MY, MZ, EN, BX, BY, BZ, PSI = range(NVAR)
VAR_NAMES = ("rho", "m_x", "m_y", "m_z", "e", "B_x", "B_y", "B_z", "psi")

# option values shared by the C ABI (include/amrvac.h) and the oracle
FLUX = {"hll": 0, "hlld": 1, "tvdlf": 2, "hllc": 3}
LIMITER = {"minmod": 0, "vanleer": 1, "koren": 2, "superbee": 3, "woodward": 4, "mcbeta": 5,
           "albada": 6, "mp5": 7, "weno5": 8, "wenoz5": 9, "cada3": 10, "wenozp5": 11,
           "venk": 12}
TIME = {"ssprk2": 0, "ssprk3": 1, "ssprk43": 2, "ssprk54": 3}
PRECISION = {"fp64": 0, "fp32": 1}
BC = {"periodic": 0, "outflow": 1, "symmetric": 2}
FIX = {"off": 0, "replace": 1, "average": 2}


@dataclass
class Config:
    """Scheme options; names follow the paper's option strings (Sect. 3)."""

    ndim: int = 2
    block_nx: tuple = (16, 16, 1)
    flux: str = "hlld"
    limiter: str = "vanleer"
    time: str = "ssprk3"
    precision: str = "fp64"
    glm: bool = True
    glm_alpha: float = 0.5
    courant: float = 0.8
    bc: tuple = (("periodic", "periodic"),) * 3
    small_density: float = 0.0
    small_pressure: float = 0.0
    check_small_values: bool = True
    fix_small_values: str = "off"   # "off", "replace" or "average" (Sect. 7.4)
    reflux: bool = False            # conservative flux correction at level changes
    level_flux: dict = None         # {level: flux} overrides per AMR level (Sect. 3)
    level_limiter: dict = None      # {level: limiter} overrides per AMR level


@dataclass
class Instance:
    xmin: tuple = (0.0, 0.0, 0.0)
    xmax: tuple = (1.0, 1.0, 1.0)
    base_blocks: tuple = (1, 1, 1)
    gamma: float = 5.0 / 3.0
    t0: float = 0.0
    t_end: float = 1e30


@dataclass
class Workload:
    name: str
    cfg: Config
    instances: list
    block_meta: np.ndarray          # int32 [nblocks, 5] = (instance, level, i, j, k)
    U: np.ndarray                   # float64 [NVAR, nblocks, ncell]
    info: dict = field(default_factory=dict)

    @property
    def nblocks(self) -> int:
        return int(self.block_meta.shape[0])

    @property
    def ncell(self) -> int:
        nx = self.cfg.block_nx
        return int(nx[0] * nx[1] * nx[2])

    def interior_cells(self) -> int:
        return self.nblocks * self.ncell


# ----------------------------------------------------------------------------
# geometry helpers (pure indexing)
# ----------------------------------------------------------------------------

def uniform_meta(base_blocks, instance=0):
    """Block list of one instance covered by its level-0 blocks, x fastest."""
    bx, by, bz = base_blocks
    k, j, i = np.meshgrid(np.arange(bz), np.arange(by), np.arange(bx), indexing="ij")
    n = bx * by * bz
    meta = np.zeros((n, 5), np.int32)
    meta[:, 0] = instance
    meta[:, 1] = 0
    meta[:, 2] = i.ravel()
    meta[:, 3] = j.ravel()
    meta[:, 4] = k.ravel()
    return meta


def cell_centres(cfg: Config, inst: Instance, meta_row):
    """Cell-centre coordinates (x, y, z) of one block, each shaped [nz, ny, nx]."""
    _, level, bi, bj, bk = (int(v) for v in meta_row)
    out = []
    for d, b in enumerate((bi, bj, bk)):
        nx = cfg.block_nx[d]
        if d >= cfg.ndim:
            out.append(np.zeros(nx))
            continue
        ncell_dom = inst.base_blocks[d] * nx * (1 << level)
        dx = (inst.xmax[d] - inst.xmin[d]) / ncell_dom
        idx = b * nx + np.arange(nx)
        out.append(inst.xmin[d] + (idx + 0.5) * dx)
    z, y, x = np.meshgrid(out[2], out[1], out[0], indexing="ij")
    return x, y, z


def cell_size(cfg: Config, inst: Instance, level: int):
    dx = []
    for d in range(3):
        if d >= cfg.ndim:
            dx.append(1.0)
        else:
            n = inst.base_blocks[d] * cfg.block_nx[d] * (1 << level)
            dx.append((inst.xmax[d] - inst.xmin[d]) / n)
    return dx


def conserved_from_primitive(gamma, rho, vx, vy, vz, p, bx, by, bz, psi=None):
    """Initial-state conserved variables from a primitive description."""
    if psi is None:
        psi = np.zeros_like(rho)
    e = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) \
        + 0.5 * (bx * bx + by * by + bz * bz)
    return np.stack([rho, rho * vx, rho * vy, rho * vz, e, bx, by, bz, psi])


def _fill_from_function(cfg, instances, meta, prim_fn):
    nb = meta.shape[0]
    ncell = cfg.block_nx[0] * cfg.block_nx[1] * cfg.block_nx[2]
    U = np.zeros((NVAR, nb, ncell))
    for b in range(nb):
        inst = instances[int(meta[b, 0])]
        x, y, z = cell_centres(cfg, inst, meta[b])
        U[:, b, :] = prim_fn(inst, x, y, z).reshape(NVAR, -1)
    return U


# ----------------------------------------------------------------------------
# C1: 1D seeded MHD Riemann problem
# ----------------------------------------------------------------------------

def c1_riemann(seed: int = 1, n: int = 512, precision: str = "fp64") -> Workload:
    """1D, one block of n cells on [0,1], interface at 0.5, outflow, gamma 5/3.

    rho_L,R and p_L,R ~ U[0.1,1], v = 0, B_x = 0.75, B_y,L/R ~ U[-1,1], B_z = 0.
    HLL + vanleer, SSPRK2 at Courant 0.8, to t = 0.1.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    rl, rr = rng.uniform(0.1, 1.0, 2)
    pl, pr = rng.uniform(0.1, 1.0, 2)
    byl, byr = rng.uniform(-1.0, 1.0, 2)
    cfg = Config(ndim=1, block_nx=(n, 1, 1), flux="hll", limiter="vanleer",
                 time="ssprk2", precision=precision, glm=False, courant=0.8,
                 bc=(("outflow", "outflow"),) * 3)
    inst = Instance(xmin=(0.0, 0.0, 0.0), xmax=(1.0, 1.0, 1.0), base_blocks=(1, 1, 1),
                    gamma=5.0 / 3.0, t0=0.0, t_end=0.1)
    meta = uniform_meta((1, 1, 1))

    def prim(inst, x, y, z):
        left = x < 0.5
        rho = np.where(left, rl, rr)
        p = np.where(left, pl, pr)
        by = np.where(left, byl, byr)
        zero = np.zeros_like(x)
        return conserved_from_primitive(inst.gamma, rho, zero, zero, zero, p,
                                        0.75 + zero, by, zero)

    U = _fill_from_function(cfg, [inst], meta, prim)
    return Workload("c1_riemann", cfg, [inst], meta, U,
                    {"seed": seed, "left": (rl, pl, byl), "right": (rr, pr, byr)})


def riemann_1d(left, right, n=512, gamma=5.0 / 3.0, bx=0.75, t_end=0.1, x0=0.5,
               flux="hll", limiter="vanleer", time="ssprk2", nblocks=1,
               xmin=0.0, xmax=1.0) -> Workload:
    """General 1D Riemann problem; left/right = (rho, vx, vy, vz, p, by, bz)."""
    nxb = n // nblocks
    cfg = Config(ndim=1, block_nx=(nxb, 1, 1), flux=flux, limiter=limiter, time=time,
                 precision="fp64", glm=False, bc=(("outflow", "outflow"),) * 3)
    inst = Instance(xmin=(xmin, 0, 0), xmax=(xmax, 1, 1), base_blocks=(nblocks, 1, 1),
                    gamma=gamma, t_end=t_end)
    meta = uniform_meta((nblocks, 1, 1))

    def prim(inst, x, y, z):
        L = x < x0
        st = [np.where(L, a, b) for a, b in zip(left, right)]
        rho, vx, vy, vz, p, by, bz = st
        return conserved_from_primitive(gamma, rho, vx, vy, vz, p, bx + 0 * x, by, bz)

    U = _fill_from_function(cfg, [inst], meta, prim)
    return Workload("riemann_1d", cfg, [inst], meta, U)


def shu_osher(n: int = 256, nblocks: int = 1, t_end: float = 1.8) -> Workload:
    """Shu-Osher shock/entropy-wave IC of Sect. 3.1.1 with B = 0 (gamma 1.4)."""
    nxb = n // nblocks
    cfg = Config(ndim=1, block_nx=(nxb, 1, 1), flux="hll", limiter="vanleer",
                 time="ssprk3", precision="fp64", glm=False,
                 bc=(("outflow", "outflow"),) * 3)
    inst = Instance(xmin=(-4.5, 0, 0), xmax=(4.5, 1, 1), base_blocks=(nblocks, 1, 1),
                    gamma=1.4, t_end=t_end)
    meta = uniform_meta((nblocks, 1, 1))

    def prim(inst, x, y, z):
        L = x < -4.0
        rho = np.where(L, 3.857143, 1.0 + 0.2 * np.sin(5.0 * x))
        vx = np.where(L, 2.629369, 0.0)
        p = np.where(L, 10.33333, 1.0)
        zero = np.zeros_like(x)
        return conserved_from_primitive(1.4, rho, vx, zero, zero, p, zero, zero, zero)

    U = _fill_from_function(cfg, [inst], meta, prim)
    return Workload("shu_osher", cfg, [inst], meta, U)


# ----------------------------------------------------------------------------
# C2: Orszag-Tang; CP Alfven wave
# ----------------------------------------------------------------------------

def c2_orszag_tang(n: int = 1024, bnx: int = 16, precision: str = "fp64",
                   flux="hlld", limiter="koren") -> Workload:
    """2D Orszag-Tang vortex on the periodic unit square, gamma 5/3, GLM on."""
    nb = n // bnx
    cfg = Config(ndim=2, block_nx=(bnx, bnx, 1), flux=flux, limiter=limiter,
                 time="ssprk3", precision=precision, glm=True, courant=0.8)
    inst = Instance(base_blocks=(nb, nb, 1), gamma=5.0 / 3.0)
    meta = uniform_meta((nb, nb, 1))
    r0 = 25.0 / (36.0 * math.pi)
    p0 = 5.0 / (12.0 * math.pi)
    b0 = 1.0 / math.sqrt(4.0 * math.pi)

    def prim(inst, x, y, z):
        tp = 2.0 * math.pi
        zero = np.zeros_like(x)
        return conserved_from_primitive(inst.gamma, r0 + zero, -np.sin(tp * y), np.sin(tp * x),
                                        zero, p0 + zero, -b0 * np.sin(tp * y),
                                        b0 * np.sin(2 * tp * x), zero)

    U = _fill_from_function(cfg, [inst], meta, prim)
    return Workload("c2_orszag_tang", cfg, [inst], meta, U, {"n": n})


CP_RHO, CP_P, CP_BPAR, CP_AMP = 1.0, 0.1, 1.0, 0.1


def cp_alfven_exact(n: int, t: float, bnx: int = 16, gamma: float = 5.0 / 3.0):
    """Exact cell averages of the 2D circularly polarised Alfven wave at time t.

    The wave vector is 2*pi*(1,1) on the periodic unit square, so the
    wavelength is 1/sqrt(2).  rho = 1, p = 0.1, B_par = 1 along n = (1,1)/sqrt2,
    B_perp = A sin(phi) along t = (-1,1)/sqrt2, B_z = A cos(phi) with A = 0.1,
    and v_perp = B_perp/sqrt(rho), v_z = B_z/sqrt(rho): an exact nonlinear
    Alfven wave travelling towards -n at v_A = B_par/sqrt(rho) = 1, i.e.
    phi = 2 pi (x + y) + 2 pi sqrt(2) t.  Cell averages use the exact factor
    (sin(pi h)/(pi h))^2 of a square cell of side h.  |B|^2, |v|^2 are constant,
    so e is constant and exact.
    """
    nb = n // bnx
    cfg = Config(ndim=2, block_nx=(bnx, bnx, 1))
    inst = Instance(base_blocks=(nb, nb, 1), gamma=gamma)
    meta = uniform_meta((nb, nb, 1))
    h = 1.0 / n
    fac = (math.sin(math.pi * h) / (math.pi * h)) ** 2
    s2 = 1.0 / math.sqrt(2.0)
    sq = math.sqrt(CP_RHO)

    def cons(inst, x, y, z):
        ph = 2 * math.pi * (x + y) + 2 * math.pi * math.sqrt(2.0) * t
        sn = CP_AMP * np.sin(ph) * fac
        cs = CP_AMP * np.cos(ph) * fac
        bpar = CP_BPAR
        bx = s2 * bpar - s2 * sn
        by = s2 * bpar + s2 * sn
        bz = cs
        vx = -s2 * sn / sq
        vy = s2 * sn / sq
        vz = cs / sq
        rho = CP_RHO + 0 * x
        e = CP_P / (gamma - 1.0) + 0.5 * CP_RHO * CP_AMP ** 2 / CP_RHO \
            + 0.5 * (bpar ** 2 + CP_AMP ** 2) + 0 * x
        return np.stack([rho, rho * vx, rho * vy, rho * vz, e, bx, by, bz, 0 * x])

    U = _fill_from_function(cfg, [inst], meta, cons)
    return cfg, inst, meta, U


def cp_alfven(n: int = 64, bnx: int = 16, limiter: str = "vanleer", flux: str = "hlld",
              precision: str = "fp64", glm: bool = True) -> Workload:
    cfg0, inst, meta, U = cp_alfven_exact(n, 0.0, bnx)
    cfg = Config(ndim=2, block_nx=(bnx, bnx, 1), flux=flux, limiter=limiter, time="ssprk3",
                 precision=precision, glm=glm, courant=0.8)
    inst.t_end = 1.0 / math.sqrt(2.0)
    return Workload("cp_alfven", cfg, [inst], meta, U, {"n": n})


# ----------------------------------------------------------------------------
# C3: 3D Mach-1 solenoidal turbulence at beta 0.01
# ----------------------------------------------------------------------------

def solenoidal_velocity(n: int, seed: int, kmin: int = 1, kmax: int = 16) -> np.ndarray:
    """Random-phase solenoidal field on an n^3 periodic grid, |v_k| ~ k^-2.

    Shell spectrum E(k) ~ k^2 |v_k|^2 ~ k^-2 for integer |k| in [kmin, kmax];
    projected so k . v_k = 0; rescaled to unit rms.  Returns [3, n, n, n]
    indexed [comp, z, y, x].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    k1 = np.fft.fftfreq(n, 1.0 / n)
    kz, ky, kx = np.meshgrid(k1, k1, k1[: n // 2 + 1], indexing="ij")
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    shell = (kk >= kmin - 0.5) & (kk < kmax + 0.5)
    amp = np.where(shell, np.where(kk > 0, kk, 1.0) ** -2.0, 0.0)
    vh = []
    for _ in range(3):
        ph = rng.uniform(0, 2 * math.pi, kk.shape)
        g = rng.standard_normal(kk.shape)
        vh.append(amp * g * np.exp(1j * ph))
    vh = np.stack(vh)
    kvec = np.stack([kx, ky, kz])
    k2 = np.where(kk > 0, kk * kk, 1.0)
    dot = (kvec * vh).sum(0)
    vh = vh - kvec * dot / k2
    v = np.stack([np.fft.irfftn(vh[c], s=(n, n, n), axes=(0, 1, 2)) for c in range(3)])
    rms = math.sqrt(float((v * v).sum(0).mean()))
    return v / rms


def c3_turbulence(n: int = 256, bnx: int = 16, seed: int = 3, precision: str = "fp32",
                  beta: float = 0.01, flux="hlld", limiter="vanleer",
                  mach: float = 1.0) -> Workload:
    """3D periodic box, rho = 1, p = 1/gamma (c_s = 1), rms velocity ``mach``
    (Mach 1 by default), uniform B0 along z with plasma beta 2p/B0^2 = beta,
    psi = 0."""
    gamma = 5.0 / 3.0
    nb = n // bnx
    cfg = Config(ndim=3, block_nx=(bnx, bnx, bnx), flux=flux, limiter=limiter,
                 time="ssprk3", precision=precision, glm=True, courant=0.8)
    inst = Instance(base_blocks=(nb, nb, nb), gamma=gamma)
    meta = uniform_meta((nb, nb, nb))
    v = solenoidal_velocity(n, seed, 1, min(16, n // 4)) * mach
    p0 = 1.0 / gamma
    b0 = math.sqrt(2.0 * p0 / beta)
    # scatter the global fields into blocks ([var][block][cell])
    ncell = bnx ** 3
    U = np.empty((NVAR, meta.shape[0], ncell))
    vb = v.reshape(3, nb, bnx, nb, bnx, nb, bnx).transpose(0, 1, 3, 5, 2, 4, 6)
    vb = vb.reshape(3, nb * nb * nb, ncell)  # block order k, j, i (i fastest) matches uniform_meta
    one = np.ones((meta.shape[0], ncell))
    zero = np.zeros_like(one)
    U[:] = conserved_from_primitive(gamma, one, vb[0], vb[1], vb[2], p0 * one, zero, zero,
                                    b0 * one)
    return Workload("c3_turbulence", cfg, [inst], meta, U,
                    {"seed": seed, "beta": beta, "B0": b0, "mach": mach})


# ----------------------------------------------------------------------------
# C4: 3D block-AMR blast
# ----------------------------------------------------------------------------

def _box_shell_hit(lo, hi, c, r0, r1):
    """True if the axis-aligned box [lo, hi] meets the shell r0 <= |x-c| <= r1."""
    near = 0.0
    far = 0.0
    for d in range(3):
        a, b = lo[d] - c[d], hi[d] - c[d]
        if a > 0:
            near += a * a
        elif b < 0:
            near += b * b
        far += max(a * a, b * b)
    return near <= r1 * r1 and far >= r0 * r0


def balanced_tree(ndim, base, maxlevel, refine_fn, periodic=True):
    """Leaves of a block tree refined by ``refine_fn(level, idx)`` and then graded
    so that leaves touching across faces, edges or corners differ by at most one
    level (full 2:1 balance, with periodic wrap).  Returns a sorted list of
    (level, i, j, k)."""
    leaves = set()
    for k in range(base[2]):
        for j in range(base[1]):
            for i in range(base[0]):
                leaves.add((0, i, j, k))

    def children(L, i, j, k):
        out = []
        for oz in range(2 if ndim > 2 else 1):
            for oy in range(2 if ndim > 1 else 1):
                for ox in range(2):
                    out.append((L + 1, 2 * i + ox, 2 * j + oy, 2 * k + oz))
        return out

    changed = True
    while changed:
        changed = False
        for leaf in sorted(leaves):
            if leaf[0] < maxlevel and refine_fn(*leaf):
                leaves.discard(leaf)
                leaves.update(children(*leaf))
                changed = True

    def covering(L, i, j, k):
        # wrap to domain at level L, then walk up until a leaf is found
        n = [base[d] << L for d in range(3)]
        p = [i, j, k]
        for d in range(3):
            if d >= ndim:
                p[d] = 0
            elif periodic:
                p[d] %= n[d]
            elif not 0 <= p[d] < n[d]:
                return None
        while L >= 0:
            if (L, *p) in leaves:
                return (L, *p)
            L -= 1
            p = [q // 2 for q in p]
        return None

    rng3 = [(-1, 0, 1) if d < ndim else (0,) for d in range(3)]
    dirs = [(dx, dy, dz) for dz in rng3[2] for dy in rng3[1] for dx in rng3[0]
            if (dx, dy, dz) != (0, 0, 0)]
    queue = deque(sorted(leaves, reverse=True))
    while queue:
        leaf = queue.popleft()
        if leaf not in leaves:
            continue
        L, i, j, k = leaf
        if L < 2:
            continue
        for dx, dy, dz in dirs:
            c = covering(L, i + dx, j + dy, k + dz)
            if c is not None and c[0] < L - 1:
                leaves.discard(c)
                ch = children(*c)
                leaves.update(ch)
                queue.extend(ch)
                queue.append(leaf)
                break
    return sorted(leaves)


def c4_blast_amr(base: int = 7, levels: int = 4, seed: int = 4, precision: str = "fp32",
                 flux="hlld", limiter="vanleer", bnx: int = 16,
                 shell=(0.2, 0.3), order: str = "level") -> Workload:
    """3D periodic unit cube, blocks of bnx^3, ``levels`` levels (ratio 2).

    Refinement flags: a block is refined while it intersects the shell
    0.2 <= r <= 0.3 about the centre, down to the finest level; the tree is then
    graded to full 2:1 balance.  The flags are geometric, so the seed only
    fixes the block storage order when ``order == "shuffled"``.
    Blast: p = 100 for r < 0.1 else 1; rho = 1; v = 0; B0 = (1,1,0)/sqrt(2).
    """
    maxlevel = levels - 1
    c = (0.5, 0.5, 0.5)
    basev = (base, base, base)

    def refine(L, i, j, k):
        h = 1.0 / (base << L)
        lo = (i * h, j * h, k * h)
        hi = ((i + 1) * h, (j + 1) * h, (k + 1) * h)
        return _box_shell_hit(lo, hi, c, shell[0], shell[1])

    leaves = balanced_tree(3, basev, maxlevel, refine)
    meta = np.zeros((len(leaves), 5), np.int32)
    for b, (L, i, j, k) in enumerate(leaves):
        meta[b] = (0, L, i, j, k)
    if order == "shuffled":
        rng = np.random.Generator(np.random.PCG64(seed))
        meta = meta[rng.permutation(meta.shape[0])]
    cfg = Config(ndim=3, block_nx=(bnx, bnx, bnx), flux=flux, limiter=limiter,
                 time="ssprk3", precision=precision, glm=True, courant=0.8)
    inst = Instance(base_blocks=basev, gamma=5.0 / 3.0)
    s = 1.0 / math.sqrt(2.0)

    def prim(inst, x, y, z):
        r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
        p = np.where(r < 0.1, 100.0, 1.0)
        zero = np.zeros_like(x)
        return conserved_from_primitive(inst.gamma, 1.0 + zero, zero, zero, zero, p,
                                        s + zero, s + zero, zero)

    U = _fill_from_function(cfg, [inst], meta, prim)
    counts = np.bincount(meta[:, 1], minlength=levels)
    return Workload("c4_blast_amr", cfg, [inst], meta, U,
                    {"base": base, "levels": levels, "blocks_per_level": counts.tolist()})


def amr_meta(ndim, base, maxlevel, refine_fn, periodic=True, instance=0):
    leaves = balanced_tree(ndim, base, maxlevel, refine_fn, periodic)
    meta = np.zeros((len(leaves), 5), np.int32)
    for b, (L, i, j, k) in enumerate(leaves):
        meta[b] = (instance, L, i, j, k)
    return meta


# ----------------------------------------------------------------------------
# C5: batched uneven 2D instances
# ----------------------------------------------------------------------------

def _modes(rng, nmodes, kmax=3):
    out = []
    for _ in range(nmodes):
        kx, ky = (int(v) for v in rng.integers(-kmax, kmax + 1, 2))
        if kx == 0 and ky == 0:
            kx = 1
        out.append((kx, ky, float(rng.uniform(-1, 1)), float(rng.uniform(0, 2 * math.pi))))
    return out


def _eval_modes(modes, x, y):
    """Sum of a sin(2 pi (kx x + ky y) + ph), divided by the mode count (|f| <= 1)."""
    f = np.zeros_like(x)
    for kx, ky, a, ph in modes:
        f = f + a * np.sin(2 * math.pi * (kx * x + ky * y) + ph)
    return f / len(modes)


def c5_instances(count: int = 256, seed: int = 5, precision: str = "fp32",
                 nmin: int = 64, nmax: int = 512, bnx: int = 16,
                 flux="hlld", limiter="vanleer") -> Workload:
    """``count`` independent periodic unit squares, N log-uniform in [nmin, nmax]
    rounded to a multiple of bnx, gamma in {5/3, 1.4}; smooth random data with
    at most 4 Fourier modes per field: rho, p in [0.5, 1.5], |v| <= 0.5,
    B = curl(A_z z) + B_z z from a random A_z (divergence-free in the continuum)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = []
    for _ in range(count):
        N = int(bnx * round(math.exp(rng.uniform(math.log(nmin), math.log(nmax))) / bnx))
        sizes.append(max(bnx, N))
    gammas = [5.0 / 3.0 if rng.uniform() < 0.5 else 1.4 for _ in range(count)]
    fields = [[_modes(rng, int(rng.integers(1, 5))) for _ in range(6)] for _ in range(count)]
    bz0 = [float(rng.uniform(-0.5, 0.5)) for _ in range(count)]
    instances = []
    metas = []
    for q in range(count):
        nb = sizes[q] // bnx
        instances.append(Instance(base_blocks=(nb, nb, 1), gamma=gammas[q]))
        metas.append(uniform_meta((nb, nb, 1), q))
    meta = np.concatenate(metas)
    cfg = Config(ndim=2, block_nx=(bnx, bnx, 1), flux=flux, limiter=limiter,
                 time="ssprk3", precision=precision, glm=True, courant=0.8)
    ncell = bnx * bnx
    U = np.zeros((NVAR, meta.shape[0], ncell))
    vmax = 0.5 / math.sqrt(3.0)
    for b in range(meta.shape[0]):
        q = int(meta[b, 0])
        inst = instances[q]
        x, y, _ = cell_centres(cfg, inst, meta[b])
        fm = fields[q]
        rho = 1.0 + 0.5 * _eval_modes(fm[0], x, y)
        p = 1.0 + 0.5 * _eval_modes(fm[1], x, y)
        vx = vmax * _eval_modes(fm[2], x, y)
        vy = vmax * _eval_modes(fm[3], x, y)
        vz = vmax * _eval_modes(fm[4], x, y)
        # B = (dA/dy, -dA/dx) for A_z = 0.05 * sum a sin(2 pi (kx x + ky y) + ph) / n
        bx = np.zeros_like(x)
        by = np.zeros_like(x)
        for kx, ky, a, ph in fm[5]:
            c = 0.05 * a * 2 * math.pi * np.cos(2 * math.pi * (kx * x + ky * y) + ph) / len(fm[5])
            bx = bx + c * ky
            by = by - c * kx
        bz = bz0[q] + 0 * x
        U[:, b, :] = conserved_from_primitive(inst.gamma, rho, vx, vy, vz, p, bx, by,
                                              bz).reshape(NVAR, -1)
    return Workload("c5_instances", cfg, instances, meta, U,
                    {"seed": seed, "sizes": sizes, "gammas": gammas})


def small_amr_2d(seed: int = 7, base=(4, 4, 1), maxlevel: int = 2, bnx: int = 8,
                 field: str = "smooth", periodic=True, flux="hlld", limiter="vanleer",
                 precision="fp64") -> Workload:
    """Small 2D three-level mesh refined around a seeded point (tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cx, cy = rng.uniform(0.3, 0.7, 2)
    radius = (0.3, 0.12)

    def refine(L, i, j, k):
        h = 1.0 / (base[0] << L)
        xc, yc = (i + 0.5) * h, (j + 0.5) * h
        return L < maxlevel and math.hypot(xc - cx, yc - cy) < radius[min(L, 1)]

    meta = amr_meta(2, base, maxlevel, refine, periodic)
    bc = (("periodic", "periodic"),) * 3 if periodic else (("outflow", "outflow"),) * 3
    cfg = Config(ndim=2, block_nx=(bnx, bnx, 1), flux=flux, limiter=limiter, time="ssprk3",
                 precision=precision, glm=True, bc=bc)
    inst = Instance(base_blocks=base, gamma=5.0 / 3.0)

    def prim(inst, x, y, z):
        tp = 2 * math.pi
        zero = np.zeros_like(x)
        if field == "uniform":
            return conserved_from_primitive(inst.gamma, 1.0 + zero, 0.3 + zero, -0.2 + zero,
                                            0.1 + zero, 0.8 + zero, 0.5 + zero, 0.4 + zero,
                                            -0.3 + zero)
        if field == "linear":
            # linear conserved data (exact prolongation where slopes agree)
            return np.stack([1.0 + 0.1 * x + 0.05 * y, 0.1 * x, 0.2 * y, 0 * x,
                             2.0 + 0.3 * x - 0.1 * y, 0.5 + 0 * x, 0.2 * x, 0.1 * y,
                             0.01 * x])
        rho = 1.0 + 0.2 * np.sin(tp * x) * np.cos(tp * y)
        vx = 0.3 * np.sin(tp * y)
        vy = -0.2 * np.sin(tp * x)
        p = 0.7 + 0.1 * np.cos(tp * (x + y))
        bx = 0.4 + 0.1 * np.sin(tp * y)
        by = 0.3 + 0.1 * np.sin(tp * x)
        psi = 0.01 * np.sin(tp * x)
        return conserved_from_primitive(inst.gamma, rho, vx, vy, 0.05 + zero, p, bx, by,
                                        0.2 + zero, psi)

    U = _fill_from_function(cfg, [inst], meta, prim)
    return Workload("small_amr_2d", cfg, [inst], meta, U)
