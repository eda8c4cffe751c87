"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module only *generates* inputs: meshes (vertex coordinates, cell vertex
lists in tensor-product order, subdomain ids, tagged boundary faces), per-cell
mu^{-1} fields and the named workload configurations.  It contains none of the
method's arithmetic (no basis functions, element matrices, assembly or
solvers), so neither side of a parity test can lean on the other through it.

Random numbers come from splitmix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out below from its
published definition; every stream is derived from (master seed, purpose).

Boundary tags: 0 = impedance (Gamma^inf), 1 = Dirichlet (Gamma^inc),
2 = natural (no boundary term; used only by the plane-wave test geometry).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASTER_SEED = 20210525
MASK64 = (1 << 64) - 1

TAG_IMPEDANCE = 0
TAG_DIRICHLET = 1
TAG_NATURAL = 2


# --------------------------------------------------------------------------
# splitmix64
# --------------------------------------------------------------------------
def _splitmix64_next(state: int) -> tuple[int, int]:
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


def _splitmix64_array(seed: int, n: int) -> np.ndarray:
    """n successive splitmix64 outputs from `seed` (vectorised, uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & MASK64) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def stream_seed(*keys) -> int:
    """Derive a 64-bit stream seed from the master seed and any str/int keys."""
    state = MASTER_SEED
    for k in keys:
        if isinstance(k, str):
            for ch in k.encode():
                state, out = _splitmix64_next(state ^ ch)
                state = out
        else:
            state, out = _splitmix64_next(state ^ (int(k) & MASK64))
            state = out
    return state


class Rng:
    """splitmix64 stream: uniforms in [0,1) with 53 random bits."""

    def __init__(self, *keys):
        self.seed = stream_seed(*keys)
        self.count = 0

    def u64(self, n: int) -> np.ndarray:
        out = _splitmix64_array((self.seed + self.count * 0x9E3779B97F4A7C15) & MASK64, n)
        self.count += n
        return out

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def integers(self, n: int, lo: int, hi_inclusive: int) -> np.ndarray:
        span = hi_inclusive - lo + 1
        return lo + (self.u64(n) % np.uint64(span)).astype(np.int64)

    def normal(self, n: int) -> np.ndarray:
        """Box-Muller on pairs of uniforms."""
        m = (n + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        u1 = np.where(u1 <= 0.0, 1e-300, u1)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2 * math.pi * u2), r * np.sin(2 * math.pi * u2)])
        return z[:n]

    def permutation(self, n: int) -> np.ndarray:
        return np.argsort(self.u64(n), kind="stable")


# --------------------------------------------------------------------------
# Meshes
# --------------------------------------------------------------------------
@dataclass
class Mesh:
    dim: int
    coords: np.ndarray          # float64 [n_vert, dim]
    cells: np.ndarray           # int64 [n_cell, 4|8], tensor-product vertex order
    cell_sub: np.ndarray        # int32 [n_cell]
    bfaces: np.ndarray          # int64 [n_bface, 2|4] vertex ids
    btag: np.ndarray            # uint8 [n_bface]
    shape: tuple = field(default=())   # (nx, ny[, nz]) cells, for reference only
    n_sub: int = 1

    @property
    def n_vert(self):
        return self.coords.shape[0]

    @property
    def n_cell(self):
        return self.cells.shape[0]


# The 8 symmetries of the square acting on tensor-order corner listings
# (v0,v1,v2,v3) = (00,10,01,11): each row is a valid re-listing of one cell.
_SQUARE_SYMS = np.array([
    [0, 1, 2, 3], [1, 0, 3, 2], [2, 3, 0, 1], [3, 2, 1, 0],
    [0, 2, 1, 3], [2, 0, 3, 1], [1, 3, 0, 2], [3, 1, 2, 0],
], dtype=np.int64)


def _cube_syms() -> np.ndarray:
    """48 re-listings of a hex's tensor-order corners (axis perms x flips)."""
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        for flips in itertools.product((0, 1), repeat=3):
            row = []
            for v in range(8):
                bits = [(v >> a) & 1 for a in range(3)]
                # new local corner v has local coords bits; its position along
                # original axis perm[a] is bits[a] xor flips[a]
                orig = [0, 0, 0]
                for a in range(3):
                    orig[perm[a]] = bits[a] ^ flips[a]
                row.append(orig[0] + 2 * orig[1] + 4 * orig[2])
            out.append(row)
    return np.array(out, dtype=np.int64)


_CUBE_SYMS = _cube_syms()


def structured_mesh_2d(nx: int, ny: int, sx: int = 1, sy: int = 1, *,
                       bc: str = "config", relabel: bool = False,
                       rotate_cells: bool = False, seed_key: str = "mesh2d",
                       lx: float = 1.0, ly: float = 1.0) -> Mesh:
    """nx x ny quads on [0,lx]x[0,ly], split into sx x sy blocks of subdomains.

    bc="config":     Dirichlet on x=0, impedance on the other three sides.
    bc="planewave":  Dirichlet on x=0, y=0, y=ly; impedance on x=lx.
    bc="impedance":  impedance on all four sides.
    relabel:         random permutation of global vertex ids.
    rotate_cells:    each cell listed in a random one of its 8 tensor orders.
    """
    assert 1 <= sx <= nx and 1 <= sy <= ny
    rng = Rng(seed_key, nx, ny, sx, sy)
    I, J = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    coords = np.stack([I.ravel() * (lx / nx), J.ravel() * (ly / ny)], 1).astype(np.float64)
    vid = lambda i, j: j * (nx + 1) + i
    ci, cj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ci = ci.ravel(); cj = cj.ravel()
    cells = np.stack([vid(ci, cj), vid(ci + 1, cj), vid(ci, cj + 1), vid(ci + 1, cj + 1)], 1).astype(np.int64)
    # balanced blocks: cell column ci is in block floor(ci * sx / nx) (equal
    # blocks when sx divides nx, otherwise sizes differ by at most one cell)
    cell_sub = ((cj * sy // ny) * sx + (ci * sx // nx)).astype(np.int32)

    faces, tags = [], []
    def side(pairs, tag):
        for p in pairs:
            faces.append(p); tags.append(tag)
    left = [(vid(0, j), vid(0, j + 1)) for j in range(ny)]
    right = [(vid(nx, j), vid(nx, j + 1)) for j in range(ny)]
    bottom = [(vid(i, 0), vid(i + 1, 0)) for i in range(nx)]
    top = [(vid(i, ny), vid(i + 1, ny)) for i in range(nx)]
    if bc == "config":
        side(left, TAG_DIRICHLET); side(right, TAG_IMPEDANCE); side(bottom, TAG_IMPEDANCE); side(top, TAG_IMPEDANCE)
    elif bc == "planewave":
        side(left, TAG_DIRICHLET); side(right, TAG_IMPEDANCE); side(bottom, TAG_DIRICHLET); side(top, TAG_DIRICHLET)
    elif bc == "impedance":
        side(left, TAG_IMPEDANCE); side(right, TAG_IMPEDANCE); side(bottom, TAG_IMPEDANCE); side(top, TAG_IMPEDANCE)
    else:
        raise ValueError(bc)
    bfaces = np.array(faces, dtype=np.int64)
    btag = np.array(tags, dtype=np.uint8)

    if rotate_cells:
        pick = rng.integers(cells.shape[0], 0, 7)
        cells = np.take_along_axis(cells, _SQUARE_SYMS[pick], axis=1)
    if relabel:
        perm = rng.permutation(coords.shape[0])       # new id of old vertex v is perm[v]
        new_coords = np.empty_like(coords)
        new_coords[perm] = coords
        coords = new_coords
        cells = perm[cells]
        bfaces = perm[bfaces]
    # boundary faces listed in a random vertex order when relabelled
    return Mesh(2, coords, cells, cell_sub, bfaces, btag, (nx, ny), sx * sy)


def structured_mesh_3d(n: int, s: int = 1, *, bc: str = "config", relabel: bool = False,
                       rotate_cells: bool = False, seed_key: str = "mesh3d") -> Mesh:
    """n^3 hexes on the unit cube, s^3 cube subdomains.

    bc="config":    Dirichlet on x=0, impedance on the other five faces.
    bc="planewave": Dirichlet on x=0, y=0, y=1; natural on z=0, z=1;
                    impedance on x=1 (a y-polarised plane wave along +x is
                    then exactly one-dimensional).
    """
    assert n % s == 0
    rng = Rng(seed_key, n, s)
    h = 1.0 / n
    r = np.arange(n + 1)
    K, J, I = np.meshgrid(r, r, r, indexing="ij")
    coords = np.stack([I.ravel() * h, J.ravel() * h, K.ravel() * h], 1).astype(np.float64)
    vid = lambda i, j, k: (k * (n + 1) + j) * (n + 1) + i
    c = np.arange(n)
    ck, cj, ci = np.meshgrid(c, c, c, indexing="ij")
    ci = ci.ravel(); cj = cj.ravel(); ck = ck.ravel()
    cells = np.stack([vid(ci + (v & 1), cj + ((v >> 1) & 1), ck + ((v >> 2) & 1)) for v in range(8)], 1).astype(np.int64)
    b = n // s
    cell_sub = (((ck // b) * s + (cj // b)) * s + (ci // b)).astype(np.int32)

    faces, tags = [], []
    a, bb = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    a = a.ravel(); bb = bb.ravel()

    def quad(fn):
        return np.stack([fn(a, bb, 0, 0), fn(a, bb, 1, 0), fn(a, bb, 0, 1), fn(a, bb, 1, 1)], 1)

    fx0 = quad(lambda p, q, dp, dq: vid(0, p + dp, q + dq))
    fx1 = quad(lambda p, q, dp, dq: vid(n, p + dp, q + dq))
    fy0 = quad(lambda p, q, dp, dq: vid(p + dp, 0, q + dq))
    fy1 = quad(lambda p, q, dp, dq: vid(p + dp, n, q + dq))
    fz0 = quad(lambda p, q, dp, dq: vid(p + dp, q + dq, 0))
    fz1 = quad(lambda p, q, dp, dq: vid(p + dp, q + dq, n))
    if bc == "config":
        plan = [(fx0, TAG_DIRICHLET), (fx1, TAG_IMPEDANCE), (fy0, TAG_IMPEDANCE), (fy1, TAG_IMPEDANCE),
                (fz0, TAG_IMPEDANCE), (fz1, TAG_IMPEDANCE)]
    elif bc == "planewave":
        plan = [(fx0, TAG_DIRICHLET), (fx1, TAG_IMPEDANCE), (fy0, TAG_DIRICHLET), (fy1, TAG_DIRICHLET),
                (fz0, TAG_NATURAL), (fz1, TAG_NATURAL)]
    else:
        raise ValueError(bc)
    for f, t in plan:
        faces.append(f); tags.append(np.full(f.shape[0], t, np.uint8))
    bfaces = np.concatenate(faces).astype(np.int64)
    btag = np.concatenate(tags)
    if rotate_cells:
        pick = rng.integers(cells.shape[0], 0, 47)
        cells = np.take_along_axis(cells, _CUBE_SYMS[pick], axis=1)
    if relabel:
        perm = rng.permutation(coords.shape[0])
        new_coords = np.empty_like(coords)
        new_coords[perm] = coords
        coords = new_coords
        cells = perm[cells]
        bfaces = perm[bfaces]
    return Mesh(3, coords, cells, cell_sub, bfaces, btag, (n, n, n), s ** 3)


# --------------------------------------------------------------------------
# mu^{-1} fields
# --------------------------------------------------------------------------
def mu_inv_blocks_2d(nx: int, ny: int, block: int, lo: float, hi: float, key: str) -> np.ndarray:
    """Piecewise-constant mu^{-1} on block x block cell tiles, U[lo,hi] per tile."""
    bx, by = nx // block, ny // block
    vals = Rng(key, nx, ny, block).uniform(bx * by, lo, hi).reshape(by, bx)
    ci, cj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    return vals[cj.ravel() // block, ci.ravel() // block].astype(np.float64)


def mu_inv_lognormal(n_cell: int, sigma: float, key) -> np.ndarray:
    return np.exp(sigma * Rng("lognormal", key).normal(n_cell))


def mu_inv_smooth_3d(n: int, amp: float, sigma_cells: float, key: str) -> np.ndarray:
    """exp(amp*g): g = white noise per cell, separable Gaussian filter (sigma in
    cells, truncated at 4 sigma, reflecting boundaries), standardised."""
    w = Rng(key, n).normal(n ** 3).reshape(n, n, n)      # [k, j, i]
    rad = int(math.ceil(4 * sigma_cells))
    t = np.arange(-rad, rad + 1)
    ker = np.exp(-0.5 * (t / sigma_cells) ** 2)
    ker /= ker.sum()
    g = w
    for ax in range(3):
        g = np.apply_along_axis(lambda v: np.convolve(np.pad(v, rad, mode="symmetric"), ker, mode="valid"), ax, g)
    g = (g - g.mean()) / g.std()
    return np.exp(amp * g).ravel().astype(np.float64)


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------
@dataclass
class Problem:
    name: str
    mesh: Mesh
    order: int
    mu_inv: np.ndarray
    omega: float
    kappa: float
    pol: np.ndarray       # complex [dim]: E_inc(x) = pol * exp(-i omega dir.x)
    direction: np.ndarray  # real unit [dim]
    eps: np.ndarray | None = None   # relative permittivity per cell (None: 1 everywhere)


def plane_wave_y(dim: int):
    pol = np.zeros(dim, np.complex128); pol[1] = 1.0
    d = np.zeros(dim); d[0] = 1.0
    return pol, d


def square_problem(n: int, s: int, order: int, omega: float, *, kappa: float = 1.0,
                   mu_inv=None, bc: str = "config", relabel=False, rotate_cells=False,
                   name: str = "square") -> Problem:
    mesh = structured_mesh_2d(n, n, s, s, bc=bc, relabel=relabel, rotate_cells=rotate_cells)
    if mu_inv is None:
        mu_inv = np.ones(mesh.n_cell)
    pol, d = plane_wave_y(2)
    return Problem(name, mesh, order, np.asarray(mu_inv, np.float64), float(omega), float(kappa), pol, d)


def cube_problem(n: int, s: int, omega: float, *, kappa: float = 1.0, mu_inv=None,
                 bc: str = "config", relabel=False, rotate_cells=False, name="cube") -> Problem:
    mesh = structured_mesh_3d(n, s, bc=bc, relabel=relabel, rotate_cells=rotate_cells)
    if mu_inv is None:
        mu_inv = np.ones(mesh.n_cell)
    pol, d = plane_wave_y(3)
    return Problem(name, mesh, 1, np.asarray(mu_inv, np.float64), float(omega), float(kappa), pol, d)


def block_benchmark(n: int, s: int, order: int, omega: float, *, n_core: float = 1.516,
                    name: str = "block") -> Problem:
    """The block benchmark of the paper's Example 1 (Section 4) as far as it is
    described: the unit square with a centre block of refractive index
    n_core = 1.516 in air (n = 1).  The block's size is not given; here it is
    the centre square [0.25, 0.75]^2.  eps = n^2 per cell, mu^{-1} = 1,
    Dirichlet x = 0 with E_inc = (0, exp(-i omega x)), impedance elsewhere,
    n x n quads in s x s subdomains."""
    P = square_problem(n, s, order, omega, name=name)
    X = P.mesh.coords[P.mesh.cells].mean(1)
    inside = np.all((X > 0.25) & (X < 0.75), axis=1)
    P.eps = np.where(inside, n_core ** 2, 1.0).astype(np.float64)
    return P


def config(name: str) -> Problem:
    """The named workloads.

    square32_p1:   32x32 quads, order 1, 2x2 subdomains, omega=4pi, mu^{-1}=1.
    square256_p2:  256x256 quads, order 2, 8x8 subdomains, omega=40pi,
                   mu^{-1} piecewise constant on 16x16-cell tiles, U[0.5,2].
    square64_p2:   64x64 quads, order 2, 2x2 subdomains of 32x32 cells (the
                   subdomain of square256_p2: 8,320 free DOFs), omega=10pi
                   (the same omega*h as square256_p2), mu^{-1} on 16x16-cell
                   tiles, U[0.5,2].
    cube64_p1:     64^3 hexes, order 1, 4^3 subdomains, omega=16pi, mu^{-1}=1.
    cube48_adj:    48^3 hexes, order 1, 3^3 subdomains, omega=12pi,
                   mu^{-1}=exp(0.3 g), g smoothed white noise (sigma 3 cells).
    """
    if name == "square32_p1":
        return square_problem(32, 2, 1, 4 * math.pi, name=name)
    if name == "square256_p2":
        mu = mu_inv_blocks_2d(256, 256, 16, 0.5, 2.0, "square256_p2/mu")
        return square_problem(256, 8, 2, 40 * math.pi, mu_inv=mu, name=name)
    if name == "square64_p2":
        mu = mu_inv_blocks_2d(64, 64, 16, 0.5, 2.0, "square64_p2/mu")
        return square_problem(64, 2, 2, 10 * math.pi, mu_inv=mu, name=name)
    if name == "cube64_p1":
        return cube_problem(64, 4, 16 * math.pi, name=name)
    if name == "cube48_adj":
        mu = mu_inv_smooth_3d(48, 0.3, 3.0, "cube48_adj/mu")
        return cube_problem(48, 3, 12 * math.pi, mu_inv=mu, name=name)
    raise KeyError(name)


def batch_problems(count: int = 512, key: str = "batch512"):
    """Independent 2D order-1 problems: side U{16..128}, omega U[2pi,32pi],
    kappa=1, mu^{-1} lognormal(0,0.3), s=ceil(n/32) subdomains per side
    (balanced, possibly unequal blocks)."""
    rng = Rng(key)
    sides = rng.integers(count, 16, 128)
    omegas = rng.uniform(count, 2 * math.pi, 32 * math.pi)
    probs = []
    for p in range(count):
        n = int(sides[p])
        s = int(math.ceil(n / 32))
        mesh = structured_mesh_2d(n, n, s, s)
        mu = mu_inv_lognormal(mesh.n_cell, 0.3, f"{key}/{p}")
        pol, d = plane_wave_y(2)
        probs.append(Problem(f"{key}[{p}]", mesh, 1, mu, float(omegas[p]), 1.0, pol, d))
    return probs
