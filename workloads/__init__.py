"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module produces *inputs only*: vertex coordinates and cell-to-vertex connectivity of
jittered triangle / tetrahedron meshes, and cell averages of prescribed initial (or exact)
primitive fields. It contains none of the finite-volume method's arithmetic (no geometry
of the scheme, no stencils, no least squares, no reconstruction, no fluxes); both the
oracle and the CUDA library receive these arrays and do all of that themselves.

Randomness comes from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), written out here with numpy uint64 arithmetic so the streams are
identical on every machine and numpy version.

Workloads (sizes of the paper's experiments, Sec. 3):
  * density_wave_2d  : periodic unit square, rho = 1 + 0.2 sin(2 pi (x+y)), u = v = 1, p = 1
                       (Sec. 3.1.1, the order test).
  * shock_tube_2d    : [0,1]x[0,0.25], Sod states split at x = 0.5 (Sec. 3.2).
  * density_wave_3d  : periodic unit cube, rho = 1 + 0.2 sin(2 pi (x+y+z)), u = v = w = 1, p = 1.
  * quadrants_batch  : 64 periodic-construction triangle meshes of log-uniform side, each a
                       four-quadrant Riemann problem with random states.
  * blast_3d         : unit cube, p = 10 inside r < 0.2 around the centre, 0.1 outside (Sec. 3.8
                       analogue).
"""
from __future__ import annotations

import concurrent.futures
import math
import os
from dataclasses import dataclass, field

import numpy as np

GAMMA = 1.4
_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


# ----------------------------------------------------------------------------------------------
# SplitMix64 stream
# ----------------------------------------------------------------------------------------------
class SplitMix64:
    """Counter-based SplitMix64: value i of the stream is mix(seed + (i+1) * golden_gamma)."""

    GOLDEN = np.uint64(0x9E3779B97F4A7C15)

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            k = np.arange(1, n + 1, dtype=np.uint64)
            z = self.state + k * self.GOLDEN
            self.state = self.state + np.uint64(n) * self.GOLDEN
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """n doubles uniform in [lo, hi): top 53 bits scaled by 2^-53."""
        u = (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def bits(self, n: int) -> np.ndarray:
        return (self.next_u64(n) >> np.uint64(63)).astype(np.int64)


# ----------------------------------------------------------------------------------------------
# Meshes
# ----------------------------------------------------------------------------------------------
@dataclass
class Mesh:
    dim: int
    xyz: np.ndarray          # [nverts, dim] float64
    cells: np.ndarray        # [ncells, dim+1] int32, vertex ids (orientation not normalised)
    period: np.ndarray       # [dim] float64; 0 in a direction that is not periodic
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def ncells(self) -> int:
        return int(self.cells.shape[0])

    @property
    def nverts(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def periodic(self) -> bool:
        return bool(np.any(self.period > 0))


def tri_mesh(nx: int, ny: int, lx: float = 1.0, ly: float = 1.0, periodic: bool = True,
             jitter: float = 0.1, seed: int = 0, name: str = "") -> Mesh:
    """nx*ny squares, each split into two triangles along a diagonal drawn from the seed.

    Vertices strictly inside the domain are moved uniformly by +-jitter*h in each coordinate;
    vertices on x in {0, lx} or y in {0, ly} stay on the lattice. Periodic meshes store each
    lattice vertex once (index (i mod nx, j mod ny)); ``period`` gives the box lengths.
    """
    hx, hy = lx / nx, ly / ny
    rng = SplitMix64(seed)
    vx = nx if periodic else nx + 1
    vy = ny if periodic else ny + 1
    ii, jj = np.meshgrid(np.arange(vx), np.arange(vy), indexing="ij")
    ii = ii.ravel()
    jj = jj.ravel()
    xyz = np.stack([ii * hx, jj * hy], axis=1).astype(np.float64)
    interior = (ii > 0) & (ii < nx) & (jj > 0) & (jj < ny)
    d = rng.uniform(2 * xyz.shape[0], -1.0, 1.0).reshape(-1, 2)
    xyz[interior, 0] += jitter * hx * d[interior, 0]
    xyz[interior, 1] += jitter * hy * d[interior, 1]

    def vid(i, j):
        if periodic:
            return (i % nx) * vy + (j % ny)
        return i * vy + j

    si, sj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    si = si.ravel()
    sj = sj.ravel()
    v00, v10, v11, v01 = vid(si, sj), vid(si + 1, sj), vid(si + 1, sj + 1), vid(si, sj + 1)
    diag = rng.bits(si.size)
    t0 = np.where(diag[:, None] == 0, np.stack([v00, v10, v11], 1), np.stack([v00, v10, v01], 1))
    t1 = np.where(diag[:, None] == 0, np.stack([v00, v11, v01], 1), np.stack([v10, v11, v01], 1))
    cells = np.empty((2 * si.size, 3), dtype=np.int32)
    cells[0::2] = t0
    cells[1::2] = t1
    period = np.array([lx, ly] if periodic else [0.0, 0.0])
    return Mesh(2, xyz, cells, period, name=name or f"tri{nx}x{ny}",
                meta=dict(nx=nx, ny=ny, lx=lx, ly=ly, jitter=jitter, seed=seed))


_KUHN_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def tet_mesh(n: int, length: float = 1.0, periodic: bool = True, jitter: float = 0.08,
             seed: int = 0, name: str = "") -> Mesh:
    """n^3 cubes, each split into the 6 Kuhn tetrahedra along its (0,0,0)-(1,1,1) diagonal.

    All cubes use the same diagonal, so the split is conforming. Vertices strictly inside the
    box are jittered by +-jitter*h per coordinate.
    """
    h = length / n
    rng = SplitMix64(seed)
    nv1 = n if periodic else n + 1
    ii, jj, kk = np.meshgrid(np.arange(nv1), np.arange(nv1), np.arange(nv1), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    xyz = np.stack([ii * h, jj * h, kk * h], axis=1).astype(np.float64)
    interior = (ii > 0) & (ii < n) & (jj > 0) & (jj < n) & (kk > 0) & (kk < n)
    d = rng.uniform(3 * xyz.shape[0], -1.0, 1.0).reshape(-1, 3)
    xyz[interior] += jitter * h * d[interior]

    def vid(i, j, k):
        if periodic:
            return ((i % n) * nv1 + (j % n)) * nv1 + (k % n)
        return (i * nv1 + j) * nv1 + k

    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    base = np.stack([ci.ravel(), cj.ravel(), ck.ravel()], axis=1)
    cells = np.empty((base.shape[0] * 6, 4), dtype=np.int32)
    for t, perm in enumerate(_KUHN_PERMS):
        p = base.copy()
        verts = [vid(p[:, 0], p[:, 1], p[:, 2])]
        for ax in perm:
            p[:, ax] += 1
            verts.append(vid(p[:, 0], p[:, 1], p[:, 2]))
        cells[t::6] = np.stack(verts, axis=1)
    period = np.full(3, length if periodic else 0.0)
    return Mesh(3, xyz, cells, period, name=name or f"tet{n}",
                meta=dict(n=n, length=length, jitter=jitter, seed=seed))


# ----------------------------------------------------------------------------------------------
# Cell averages of prescribed fields (input data, not part of the scheme)
# ----------------------------------------------------------------------------------------------
def _simplex_rule(dim: int, n: int):
    """Collapsed (Duffy) Gauss-Legendre rule on the unit simplex: barycentric points, weights
    summing to 1. Exact for polynomials of degree 2n - dim."""
    g, w = np.polynomial.legendre.leggauss(n)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    if dim == 2:
        u, v = np.meshgrid(g, g, indexing="ij")
        wu, wv = np.meshgrid(w, w, indexing="ij")
        x = u
        y = v * (1.0 - u)
        wt = wu * wv * (1.0 - u) * 2.0
        lam = np.stack([1 - x - y, x, y], axis=-1).reshape(-1, 3)
    else:
        u, v, s = np.meshgrid(g, g, g, indexing="ij")
        wu, wv, ws = np.meshgrid(w, w, w, indexing="ij")
        x = u
        y = v * (1.0 - u)
        z = s * (1.0 - u) * (1.0 - v)
        wt = wu * wv * ws * (1.0 - u) ** 2 * (1.0 - v) * 6.0
        lam = np.stack([1 - x - y - z, x, y, z], axis=-1).reshape(-1, 4)
    return lam, wt.reshape(-1)


def unwrapped_cell_vertices(mesh: Mesh) -> np.ndarray:
    """[ncells, dim+1, dim] vertex coordinates, periodic images moved next to vertex 0."""
    v = mesh.xyz[mesh.cells]                      # [nc, d+1, d]
    if mesh.periodic:
        per = np.where(mesh.period > 0, mesh.period, np.inf)
        dv = v - v[:, :1, :]
        shift = np.where(np.isfinite(per), np.round(dv / np.where(np.isfinite(per), per, 1.0)), 0.0)
        v = v - shift * np.where(np.isfinite(per), per, 0.0)
    return v


def cell_volumes(mesh: Mesh) -> np.ndarray:
    """|V_i| of each simplex (used only to weight test error norms)."""
    v = unwrapped_cell_vertices(mesh)
    J = v[:, 1:, :] - v[:, :1, :]
    return np.abs(np.linalg.det(J)) / math.factorial(mesh.dim)


def cell_centroids(mesh: Mesh) -> np.ndarray:
    return unwrapped_cell_vertices(mesh).mean(axis=1)


def primitive_to_conserved(prim: np.ndarray, gamma: float = GAMMA) -> np.ndarray:
    """prim [..., d+2] = (rho, u, v[, w], p) -> (rho, rho u, rho v[, rho w], E)."""
    rho = prim[..., 0]
    vel = prim[..., 1:-1]
    p = prim[..., -1]
    out = np.empty_like(prim)
    out[..., 0] = rho
    out[..., 1:-1] = rho[..., None] * vel
    out[..., -1] = p / (gamma - 1.0) + 0.5 * rho * np.sum(vel * vel, axis=-1)
    return out


def cell_average(mesh: Mesh, prim_fn, n_rule: int = 8, gamma: float = GAMMA,
                 chunk: int = 1 << 16) -> np.ndarray:
    """Cell averages of the conserved variables of ``prim_fn(x) -> prim`` ([npts, dim] ->
    [npts, d+2]). Returns [nv, ncells] (variable-major, the layout the library takes)."""
    lam, wt = _simplex_rule(mesh.dim, n_rule)
    nq = wt.size
    nv = mesh.dim + 2
    out = np.empty((nv, mesh.ncells))

    def one(c0):
        sub = Mesh(mesh.dim, mesh.xyz, mesh.cells[c0:c0 + chunk], mesh.period)
        v = unwrapped_cell_vertices(sub)                       # [nc, d+1, d]
        nc = v.shape[0]
        pts = np.matmul(lam, v)                                # [nc, nq, d]
        prim = np.ascontiguousarray(prim_fn(pts.reshape(-1, mesh.dim)).T)   # [nv, nc*nq]
        rho, vel, p = prim[0], prim[1:-1], prim[-1]
        cons = np.empty_like(prim)
        cons[0] = rho
        cons[1:-1] = rho * vel
        cons[-1] = p / (gamma - 1.0) + 0.5 * rho * np.sum(vel * vel, axis=0)
        out[:, c0:c0 + nc] = cons.reshape(nv, nc, nq) @ wt

    # chunks are independent (numpy releases the interpreter lock inside these operations)
    starts = range(0, mesh.ncells, chunk)
    if len(starts) > 1:
        with concurrent.futures.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
            list(ex.map(one, starts))
    else:
        for c0 in starts:
            one(c0)
    return out


# ----------------------------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    mesh: Mesh
    U0: np.ndarray                 # [nv, ncells] conserved cell averages
    params: dict                   # scheme parameters the workload is defined with
    exact: object = None           # callable(t) -> [nv, ncells] exact cell averages, or None


def _wave_prim(dim, t):
    def f(x):
        s = x.sum(axis=1) - dim * t
        prim = np.ones((x.shape[0], dim + 2))
        prim[:, 0] = 1.0 + 0.2 * np.sin(2.0 * np.pi * s)
        return prim
    return f


def density_wave_2d(n: int = 32, seed: int = 0, jitter: float = 0.1) -> Workload:
    """Periodic unit square, 2 n^2 triangles; exact solution rho = 1 + 0.2 sin(2 pi (x+y-2t))."""
    mesh = tri_mesh(n, n, 1.0, 1.0, periodic=True, jitter=jitter, seed=seed)
    return Workload(f"density_wave_2d_n{n}", mesh, cell_average(mesh, _wave_prim(2, 0.0)),
                    dict(dim=2, degree=2, cfl=0.5),
                    exact=lambda t, m=mesh: cell_average(m, _wave_prim(2, t)))


def density_wave_3d(n: int = 32, seed: int = 0, jitter: float = 0.08) -> Workload:
    mesh = tet_mesh(n, 1.0, periodic=True, jitter=jitter, seed=seed)
    return Workload(f"density_wave_3d_n{n}", mesh, cell_average(mesh, _wave_prim(3, 0.0), n_rule=5),
                    dict(dim=3, degree=2, cfl=0.5),
                    exact=lambda t, m=mesh: cell_average(m, _wave_prim(3, t), n_rule=5))


def shock_tube_2d(nx: int = 512, ny: int = 128, seed: int = 0, jitter: float = 0.1) -> Workload:
    """Sod states on [0,1]x[0,0.25]: (1,0,0,1) for x < 0.5, (0.125,0,0,0.1) otherwise."""
    mesh = tri_mesh(nx, ny, 1.0, 0.25 * ny / 128 if False else 0.25, periodic=False,
                    jitter=jitter, seed=seed)

    def f(x):
        left = x[:, 0] < 0.5
        prim = np.zeros((x.shape[0], 4))
        prim[:, 0] = np.where(left, 1.0, 0.125)
        prim[:, 3] = np.where(left, 1.0, 0.1)
        return prim
    return Workload(f"shock_tube_2d_{nx}x{ny}", mesh, cell_average(mesh, f, n_rule=6),
                    dict(dim=2, cfl=0.4))


def triple_point_2d(nx: int = 500, ny: int = 215, seed: int = 0, jitter: float = 0.1) -> Workload:
    """The single-material triple point problem (Sec. 3.4) on [0,7]x[0,3] with walls all round:
    (1,0,0,1) for x <= 1, (0.125,0,0,0.1) for x > 1 and y > 1.5, (1,0,0,0.1) for x > 1 and
    y <= 1.5. 500 x 215 squares give 215000 triangles (the paper's mesh: 214770, h ~ 1/67).
    The paper states no ratio of specific heats for it: gamma = 1.4."""
    mesh = tri_mesh(nx, ny, 7.0, 3.0, periodic=False, jitter=jitter, seed=seed)

    def f(x):
        left = x[:, 0] <= 1.0
        top = x[:, 1] > 1.5
        prim = np.zeros((x.shape[0], 4))
        prim[:, 0] = np.where(left, 1.0, np.where(top, 0.125, 1.0))
        prim[:, 3] = np.where(left, 1.0, 0.1)
        return prim
    return Workload(f"triple_point_2d_{nx}x{ny}", mesh, cell_average(mesh, f, n_rule=6),
                    dict(dim=2, cfl=0.4, boundary="wall"))


# Double Mach reflection (Sec. 3.3): a Mach-10 shock at 60 degrees from x = 1/6 on the bottom wall.
DMR_PRE = (1.4, 0.0, 0.0, 1.0)
# post-shock state: rho and velocity as printed (8.25 (cos 30, -sin 30)); the pressure from the
# Rankine-Hugoniot condition of the Mach-10 shock into DMR_PRE, (2 gamma M^2 - (gamma - 1)) / (gamma + 1)
# = 116.5 (the paper prints 116.8333, which that shock does not produce)
DMR_POST = (8.0, 8.25 * np.cos(np.pi / 6), -8.25 * np.sin(np.pi / 6), 116.5)


def dmr_2d(ny: int = 20, seed: int = 0, jitter: float = 0.1) -> Workload:
    """[0,4]x[0,1], 4 ny x ny squares -> 8 ny^2 triangles (ny = 215: 369800, ny = 299: 715208, the
    paper's 369604 and 714138), post-shock state where y >= sqrt(3) (x - 1/6), pre-shock elsewhere;
    boundaries from dmr_boundary()."""
    mesh = tri_mesh(4 * ny, ny, 4.0, 1.0, periodic=False, jitter=jitter, seed=seed)

    def f(x):
        post = x[:, 1] >= np.sqrt(3.0) * (x[:, 0] - 1.0 / 6.0)
        return np.where(post[:, None], np.array(DMR_POST), np.array(DMR_PRE))
    return Workload(f"dmr_2d_{4 * ny}x{ny}", mesh, cell_average(mesh, f, n_rule=6), dict(dim=2, cfl=0.4))


def dmr_boundary():
    """(regions, states) of the double Mach reflection: boundary faces by the box their midpoint
    lies in -- left x = 0 and bottom x < 1/6 the post-shock state (kind 2), bottom x >= 1/6 a
    reflective wall (kind 1), top y = 1 the moving shock (kind 3: post-shock left of the line
    x = 1/6 + (y + 20 t) / sqrt(3), pre-shock right of it), right x = 4 transmissive (kind 0, the
    default) -- and the states (A = post-shock, B = pre-shock, conserved) with the line's xs0, sy, vs."""
    eps = 1e-9
    regions = [((-1.0, -1.0), (eps, 2.0), 2),
               ((-1.0, -1.0), (1.0 / 6.0, eps), 2),
               ((1.0 / 6.0, -1.0), (5.0, eps), 1),
               ((-1.0, 1.0 - eps), (5.0, 2.0), 3)]
    A = primitive_to_conserved(np.array([DMR_POST]))[0]
    B = primitive_to_conserved(np.array([DMR_PRE]))[0]
    return regions, (A, B, 1.0 / 6.0, 1.0 / np.sqrt(3.0), 20.0 / np.sqrt(3.0))


def quadrant_states(seed: int, k: int) -> np.ndarray:
    """Per-quadrant primitive states of batch member k: rho, p ~ U[0.1,2], u, v ~ U[-1,1]."""
    rng = SplitMix64(seed * 1000003 + 7919 * (k + 1))
    rho = rng.uniform(4, 0.1, 2.0)
    u = rng.uniform(4, -1.0, 1.0)
    v = rng.uniform(4, -1.0, 1.0)
    p = rng.uniform(4, 0.1, 2.0)
    return np.stack([rho, u, v, p], axis=1)


def quadrants_batch(n_meshes: int = 64, seed: int = 0, nmin: int = 16, nmax: int = 256,
                    jitter: float = 0.1, periodic: bool = False) -> list[Workload]:
    """Batch of independent four-quadrant Riemann problems on triangle meshes of side N_k,
    N_k = round(exp(U[ln nmin, ln nmax])) drawn from the seed."""
    rng = SplitMix64(seed)
    sides = np.rint(np.exp(rng.uniform(n_meshes, math.log(nmin), math.log(nmax)))).astype(int)
    out = []
    for k, n in enumerate(sides):
        mesh = tri_mesh(int(n), int(n), 1.0, 1.0, periodic=periodic, jitter=jitter,
                        seed=seed * 7777 + k)
        st = quadrant_states(seed, k)

        def f(x, st=st):
            q = (x[:, 0] >= 0.5).astype(int) + 2 * (x[:, 1] >= 0.5).astype(int)
            return st[q]
        out.append(Workload(f"quadrant_{k}_n{n}", mesh, cell_average(mesh, f, n_rule=4),
                            dict(dim=2, degree=2, cfl=0.4)))
    return out


def blast_3d(n: int = 96, seed: int = 0, jitter: float = 0.08) -> Workload:
    """Unit cube: rho = 1, u = 0, p = 10 for |x - c| < 0.2, 0.1 elsewhere; transmissive."""
    mesh = tet_mesh(n, 1.0, periodic=False, jitter=jitter, seed=seed)

    def f(x):
        r = np.linalg.norm(x - 0.5, axis=1)
        prim = np.zeros((x.shape[0], 5))
        prim[:, 0] = 1.0
        prim[:, 4] = np.where(r < 0.2, 10.0, 0.1)
        return prim
    return Workload(f"blast_3d_n{n}", mesh, cell_average(mesh, f, n_rule=3),
                    dict(dim=3, degree=3, cfl=0.3))


def uniform_state(mesh: Mesh, prim) -> np.ndarray:
    prim = np.asarray(prim, dtype=np.float64)
    cons = primitive_to_conserved(prim[None, :])[0]
    return np.repeat(cons[:, None], mesh.ncells, axis=1)
