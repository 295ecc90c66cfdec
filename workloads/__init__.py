"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only generates inputs: counter-based random numbers (splitmix64),
point sets, Delaunay meshes, the finite-volume Poisson matrix those meshes
define, right-hand sides and random initial network parameters.  It holds none
of the solver's arithmetic (no coarsening, smoothing, V-cycle or network
evaluation), so both sides of every parity check can consume it.

Sign convention: every matrix produced here is the symmetric positive
(semi-)definite form of the Poisson operator (positive diagonal, non-positive
off-diagonals), i.e. minus the negative semi-definite operator of Sec. 2.1.

Workload recipes (all seeded; sizes follow the paper's workloads, the paper's
own datasets are not available and these stand in for them):

* ``poisson5(m)``: 5-point finite-difference Laplacian, unscaled stencil
  (4, -1, -1, -1, -1), Dirichlet boundary eliminated, n = m*m.
* ``fv_mesh(kind, n_points, seed)``: vertex-centred finite volumes on a
  Delaunay triangulation of the unit square.  Edge coupling
  w_ij = (cot a + cot b)/2 over the one or two triangles sharing edge ij
  (the Voronoi-dual two-point flux); couplings that come out non-positive
  (obtuse pairs) are clipped to zero and counted.  Dirichlet on x = 1
  (those nodes eliminated, their couplings kept on the diagonal), Neumann
  elsewhere.  Point-set kinds:
    - "uniform": stratified jittered points, uniform density;
    - "graded":  x-density proportional to (10 - 9x) (10:1 toward x = 0);
    - "band":    graded points plus a horizontal band of anisotropic
                 lattice rows centred on y = 0.5, cell aspect ratio growing
                 geometrically (row height x1.1 per row) from
                 ``max_aspect`` at the centre toward 1, the band kept
                 inside 0.45 <= y <= 0.55.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "CSR", "splitmix64", "uniform01", "uniform_pm1", "poisson5", "fv_mesh",
    "rhs_uniform", "rhs_zero_mean", "gcin_init_params", "c2_matrix",
    "c3_batch", "c4_matrix", "GCIN_PARAM_SIZES", "gcin_param_sizes", "poisson5_body", "structured_batch",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


@dataclass
class CSR:
    """Square or rectangular CSR matrix: int32 row_ptr/col, float64 val."""
    n_rows: int
    n_cols: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n_rows, self.n_cols))
        rows = np.repeat(np.arange(self.n_rows), np.diff(self.row_ptr))
        np.add.at(d, (rows, self.col), self.val)
        return d


# ----------------------------------------------------------------------------
# counter-based random numbers
# ----------------------------------------------------------------------------
def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset+1 .. offset+n of the splitmix64 sequence started at seed."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of splitmix64."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in [-1, 1)."""
    return 2.0 * uniform01(seed, n, offset) - 1.0


def _sub_seed(seed: int, tag: int) -> int:
    return int(splitmix64(seed * 1000003 + tag, 1)[0])


# ----------------------------------------------------------------------------
# structured 5-point Laplacian (64x64 is the small parity case)
# ----------------------------------------------------------------------------
def poisson5(m: int) -> CSR:
    """5-point Laplacian on an m x m interior grid, Dirichlet eliminated."""
    n = m * m
    rows, cols, vals = [], [], []
    idx = np.arange(n).reshape(m, m)
    for di, dj, v in ((0, 0, 4.0), (-1, 0, -1.0), (1, 0, -1.0), (0, -1, -1.0), (0, 1, -1.0)):
        i0, i1 = max(0, -di), m - max(0, di)
        j0, j1 = max(0, -dj), m - max(0, dj)
        src = idx[i0:i1, j0:j1].ravel()
        dst = idx[i0 + di:i1 + di, j0 + dj:j1 + dj].ravel()
        rows.append(src)
        cols.append(dst)
        vals.append(np.full(src.size, v))
    return _coo_to_csr(n, n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def poisson7(m: int, body_ratio: float = 1.0, radius: float = 0.2) -> CSR:
    """7-point finite-volume Laplacian on an m x m x m interior grid of the unit
    cube, Dirichlet eliminated (a Cartesian 3D stand-in).  Cells inside a
    centred sphere of the given radius carry conductivity body_ratio (1 = the
    plain Laplacian; small values mimic an immersed solid); face coefficients
    are harmonic means of the two cells, boundary faces use the cell's own."""
    n = m ** 3
    h = 1.0 / (m + 1)
    g = (np.arange(m) + 1) * h
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    cond = np.where((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2 < radius ** 2, body_ratio, 1.0)
    idx = np.arange(n).reshape(m, m, m)
    rows, cols, vals = [], [], []
    diag = np.zeros((m, m, m))
    for axis in range(3):
        for side in (-1, 1):
            nb = np.roll(cond, -side, axis=axis)
            face = 2.0 * cond * nb / (cond + nb)
            edge = [slice(None)] * 3
            edge[axis] = slice(m - 1, m) if side == 1 else slice(0, 1)
            face[tuple(edge)] = cond[tuple(edge)]          # Dirichlet face
            diag += face
            inner = [slice(None)] * 3
            inner[axis] = slice(0, m - 1) if side == 1 else slice(1, m)
            inner = tuple(inner)
            src = idx[inner].ravel()
            dst = np.roll(idx, -side, axis=axis)[inner].ravel()
            rows.append(src)
            cols.append(dst)
            vals.append(-face[inner].ravel())
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    return _coo_to_csr(n, n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def poisson5_body(m: int, body_ratio: float = 1.0, radius: float = 0.2, center=(0.5, 0.5)) -> CSR:
    """5-point finite-volume Laplacian on an m x m interior grid of the unit
    square, Dirichlet eliminated, with cells inside a disk (radius, center)
    of conductivity body_ratio; face coefficients are harmonic means of the two
    cells, boundary faces use the cell's own (the 2D analogue of poisson7)."""
    n = m * m
    h = 1.0 / (m + 1)
    g = (np.arange(m) + 1) * h
    X, Y = np.meshgrid(g, g, indexing="ij")
    cond = np.where((X - center[0]) ** 2 + (Y - center[1]) ** 2 < radius ** 2, body_ratio, 1.0)
    idx = np.arange(n).reshape(m, m)
    rows, cols, vals = [], [], []
    diag = np.zeros((m, m))
    for axis in range(2):
        for side in (-1, 1):
            nb = np.roll(cond, -side, axis=axis)
            face = 2.0 * cond * nb / (cond + nb)
            edge = [slice(None)] * 2
            edge[axis] = slice(m - 1, m) if side == 1 else slice(0, 1)
            face[tuple(edge)] = cond[tuple(edge)]          # Dirichlet face
            diag += face
            inner = [slice(None)] * 2
            inner[axis] = slice(0, m - 1) if side == 1 else slice(1, m)
            inner = tuple(inner)
            rows.append(idx[inner].ravel())
            cols.append(np.roll(idx, -side, axis=axis)[inner].ravel())
            vals.append(-face[inner].ravel())
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    return _coo_to_csr(n, n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def structured_batch(n_meshes: int, seed: int = 0) -> list:
    """Cartesian training set for the structured-mesh networks: alternating 2D
    grids (m in 16..64, poisson5_body) and 3D grids (m in 8..16, poisson7),
    each with an immersed body of conductivity 10^-U[0, 3] and radius
    U[0.1, 0.3] (2D disks off-centre by up to 0.15)."""
    out = []
    for k in range(n_meshes):
        u = uniform01(_sub_seed(seed, 9000 + k), 5)
        ratio = 10.0 ** (-3.0 * u[1])
        radius = 0.1 + 0.2 * u[2]
        if k % 2 == 0:
            m = 16 + int(48 * u[0])
            out.append(poisson5_body(m, ratio, radius, (0.35 + 0.3 * u[3], 0.35 + 0.3 * u[4])))
        else:
            m = 8 + int(8 * u[0])
            out.append(poisson7(m, ratio, radius))
    return out


def _coo_to_csr(nr, nc, r, c, v) -> CSR:
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    row_ptr = np.zeros(nr + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return CSR(nr, nc, row_ptr.astype(np.int32), c.astype(np.int32), v.astype(np.float64))


# ----------------------------------------------------------------------------
# point sets
# ----------------------------------------------------------------------------
def _graded_x(u: np.ndarray) -> np.ndarray:
    """Inverse CDF of the density (10 - 9x)/5.5 on [0, 1]."""
    return (10.0 - np.sqrt(100.0 - 99.0 * u)) / 9.0


def _stratified(n: int, seed: int, graded: bool) -> np.ndarray:
    """About n jittered stratified points strictly inside the unit square."""
    ny = max(2, int(round(np.sqrt(n))))
    nx = max(2, int(round(n / ny)))
    gx, gy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    gx, gy = gx.ravel().astype(np.float64), gy.ravel().astype(np.float64)
    j = uniform_pm1(_sub_seed(seed, 1), 2 * gx.size).reshape(2, -1)
    u = (gx + 0.5 + 0.35 * j[0]) / nx
    v = (gy + 0.5 + 0.35 * j[1]) / ny
    x = _graded_x(u) if graded else u
    return np.stack([x, v], axis=1)


def _boundary_points(per_side: int, graded: bool) -> tuple[np.ndarray, np.ndarray]:
    """Points on the square's boundary; returns (points, on_dirichlet_side)."""
    t = np.arange(per_side, dtype=np.float64) / per_side
    xs = _graded_x(t) if graded else t
    bottom = np.stack([xs, np.zeros_like(t)], 1)               # (x, 0), x in [0,1)
    right = np.stack([np.ones_like(t), t], 1)                   # (1, y), y in [0,1)
    top = np.stack([_graded_x(1.0 - t) if graded else 1.0 - t, np.ones_like(t)], 1)  # (x, 1), x in (0,1]
    left = np.stack([np.zeros_like(t), 1.0 - t], 1)             # (0, y), y in (0,1]
    pts = np.concatenate([bottom, right, top, left])
    dir_mask = np.isclose(pts[:, 0], 1.0)
    return pts, dir_mask


def _band_rows(max_aspect: float, h: float) -> np.ndarray:
    """y offsets (from 0.5) of anisotropic lattice rows, aspect 1 -> max_aspect."""
    hy = h / max_aspect
    ys, y = [0.0], 0.0
    while hy < h and y + hy < 0.05:
        y += hy
        ys.append(y)
        hy *= 1.1
    ys = np.array(ys)
    return np.concatenate([-ys[:0:-1], ys])


def fv_points(kind: str, n_points: int, seed: int, max_aspect: float = 1000.0):
    """Point set of the requested kind and its Dirichlet mask."""
    graded = kind in ("graded", "band")
    per_side = max(8, int(round(np.sqrt(n_points))))
    bnd, bnd_dir = _boundary_points(per_side, graded)
    n_int = max(16, n_points - bnd.shape[0])
    if kind == "band":
        h = 1.0 / per_side
        rows = _band_rows(max_aspect, h)
        half = rows.max() + 0.5 * h
        n_cols = per_side
        cu = (np.arange(n_cols) + 0.5) / n_cols
        cx = _graded_x(cu)
        BX, BY = np.meshgrid(cx, 0.5 + rows, indexing="ij")
        # jitter of 1% of the local row spacing breaks cocircular quadruples
        gaps = np.diff(rows)
        dy = np.minimum(np.concatenate([[gaps[0]], gaps]), np.concatenate([gaps, [gaps[-1]]]))
        DY = np.broadcast_to(dy[None, :], BX.shape).ravel()
        jit = uniform_pm1(_sub_seed(seed, 2), 2 * BX.size).reshape(2, -1)
        band = np.stack([BX.ravel() + 0.01 * DY * jit[0], BY.ravel() + 0.01 * DY * jit[1]], 1)
        n_iso = max(16, n_int - band.shape[0])
        iso = _stratified(int(n_iso / (1.0 - 2 * half)), seed, True)
        iso = iso[np.abs(iso[:, 1] - 0.5) > half + 0.35 * h]
        interior = np.concatenate([iso, band])
    else:
        interior = _stratified(n_int, seed, graded)
    pts = np.concatenate([bnd, interior])
    dmask = np.concatenate([bnd_dir, np.zeros(interior.shape[0], dtype=bool)])
    return pts, dmask


# ----------------------------------------------------------------------------
# vertex-centred finite-volume assembly on a Delaunay triangulation
# ----------------------------------------------------------------------------
def delaunay_fv(points: np.ndarray, dirichlet: np.ndarray, drop=None):
    """Assemble the SPD FV Laplacian; returns (CSR, stats dict).

    drop(centroids) -> bool mask removes triangles outside the domain (e.g.
    inside an airfoil, whose surface is then a Neumann boundary)."""
    from scipy.spatial import Delaunay

    tri = Delaunay(points).simplices.astype(np.int64)
    if drop is not None:
        tri = tri[~drop(points[tri].mean(axis=1))]
    n_all = points.shape[0]
    ea, eb, ew = [], [], []
    for k in range(3):
        p0 = tri[:, k]
        pa = tri[:, (k + 1) % 3]
        pb = tri[:, (k + 2) % 3]
        e1 = points[pa] - points[p0]
        e2 = points[pb] - points[p0]
        cross = np.abs(e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
        dot = e1[:, 0] * e2[:, 0] + e1[:, 1] * e2[:, 1]
        ok = cross > 1e-300
        cot = np.where(ok, dot / np.where(ok, cross, 1.0), 0.0)
        ea.append(np.minimum(pa, pb))
        eb.append(np.maximum(pa, pb))
        ew.append(0.5 * cot)
    ea, eb, ew = np.concatenate(ea), np.concatenate(eb), np.concatenate(ew)
    key = ea * n_all + eb
    uk, inv = np.unique(key, return_inverse=True)
    w = np.bincount(inv, weights=ew)
    ia, ib = uk // n_all, uk % n_all
    n_clipped = int(np.count_nonzero(w <= 0.0))
    wmax_node = np.zeros(n_all)
    np.maximum.at(wmax_node, ia, np.maximum(w, 0))
    np.maximum.at(wmax_node, ib, np.maximum(w, 0))
    keep = w > 1e-12 * np.maximum(wmax_node[ia], wmax_node[ib])
    ia, ib, w = ia[keep], ib[keep], w[keep]
    diag = np.zeros(n_all)
    np.add.at(diag, ia, w)
    np.add.at(diag, ib, w)
    live = ~dirichlet
    if drop is not None:   # points left without a kept triangle or coupling are not unknowns
        live &= diag > 0.0
    newid = -np.ones(n_all, dtype=np.int64)
    newid[live] = np.arange(int(live.sum()))
    both = live[ia] & live[ib]
    ra, rb, rw = newid[ia[both]], newid[ib[both]], w[both]
    n = int(live.sum())
    rows = np.concatenate([ra, rb, np.arange(n)])
    cols = np.concatenate([rb, ra, np.arange(n)])
    vals = np.concatenate([-rw, -rw, diag[live]])
    A = _coo_to_csr(n, n, rows, cols, vals)
    stats = {"n_points": n_all, "n_triangles": int(tri.shape[0]), "n_clipped": n_clipped,
             "n_dirichlet": int(dirichlet.sum()), "n": n, "nnz": A.nnz, "live": live}
    return A, stats


def fv_mesh(kind: str, n_points: int, seed: int, max_aspect: float = 1000.0):
    pts, dmask = fv_points(kind, n_points, seed, max_aspect)
    return delaunay_fv(pts, dmask)


# ----------------------------------------------------------------------------
# the named workloads
# ----------------------------------------------------------------------------
def c2_matrix(seed: int = 0) -> CSR:
    """50k-point graded (10:1) Delaunay FV Laplacian."""
    return fv_mesh("graded", 50_000, seed)[0]


def c3_batch(n_meshes: int = 64, seed: int = 0, n_min: int = 2000, n_max: int = 20000):
    """Training batch: meshes of uneven size cycling uniform/graded/band kinds."""
    kinds = ("uniform", "graded", "band")
    sizes = n_min + (splitmix64(_sub_seed(seed, 7), n_meshes) % np.uint64(n_max - n_min + 1)).astype(np.int64)
    out = []
    for m in range(n_meshes):
        kind = kinds[m % 3]
        out.append(fv_mesh(kind, int(sizes[m]), seed * 1000 + m, max_aspect=100.0)[0])
    return out


_C4_CACHE: dict = {}


def renumber_rcm(A: CSR) -> CSR:
    """The same matrix with its unknowns renumbered by reverse Cuthill-McKee
    (scipy's, on the symmetric pattern): the locality order finite-volume
    codes give their cells, so that a row's couplings lie within a few
    thousand rows of it."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import reverse_cuthill_mckee

    M = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n_rows, A.n_cols))
    p = reverse_cuthill_mckee(M, symmetric_mode=True)
    Mp = M[p][:, p].tocsr()
    Mp.sort_indices()
    return CSR(A.n_rows, A.n_cols, Mp.indptr.astype(np.int32), Mp.indices.astype(np.int32),
               Mp.data.astype(np.float64))


def c4_matrix(seed: int = 0, n_points: int = 2_500_000) -> CSR:
    """2.5M-point graded mesh with an anisotropic band (aspect up to 1000),
    its cells numbered by reverse Cuthill-McKee (the generator's own order
    puts the band and the boundary points at the ends).  Kept for the life of
    the process (its triangulation takes ~40 s); callers must not modify the
    returned arrays."""
    key = (seed, n_points)
    if key not in _C4_CACHE:
        _C4_CACHE[key] = renumber_rcm(fv_mesh("band", n_points, seed, max_aspect=1000.0)[0])
    return _C4_CACHE[key]


# ----------------------------------------------------------------------------
# airfoil sequence: NACA m4 12 in a circular farfield
# ----------------------------------------------------------------------------
def _naca(x, m, p=0.4, t=0.12):
    """Camber line, its slope and the half thickness of a NACA 4-digit section
    with a closed trailing edge (last thickness coefficient -0.1036)."""
    yt = 5 * t * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x ** 2 + 0.2843 * x ** 3 - 0.1036 * x ** 4)
    if m == 0.0:
        return np.zeros_like(x), np.zeros_like(x), yt
    front = x < p
    yc = np.where(front, m / p ** 2 * (2 * p * x - x ** 2), m / (1 - p) ** 2 * ((1 - 2 * p) + 2 * p * x - x ** 2))
    dyc = np.where(front, 2 * m / p ** 2 * (p - x), 2 * m / (1 - p) ** 2 * (p - x))
    return yc, dyc, yt


def naca_points(seed: int, n_surface: int = 1000, n_far: int = 200_000, r_far: float = 20.0,
                h1: float = 1e-5, growth: float = 1.1):
    """Points of an airfoil mesh: cosine-spaced surface points, wall-normal
    layers (first height h1 chords, growth 1.1, until a layer is as tall as
    the local surface spacing), then points uniform in angle and in log r out
    to a farfield circle of radius r_far (Dirichlet).  Camber m ~ U[0, 0.04]
    by seed, p = 0.4, thickness 12 %.  Returns (points, dirichlet mask, m)."""
    m = 0.04 * float(uniform01(_sub_seed(seed, 51), 1)[0])
    half = n_surface // 2
    beta = np.linspace(0.0, np.pi, half + 1)
    xs = 0.5 * (1.0 - np.cos(beta))
    yc, dyc, yt = _naca(xs, m)
    th = np.arctan(dyc)
    up = np.stack([xs - yt * np.sin(th), yc + yt * np.cos(th)], 1)
    lo = np.stack([xs + yt * np.sin(th), yc - yt * np.cos(th)], 1)
    surf = np.concatenate([up, lo[1:-1][::-1]])              # closed loop, leading edge at index 0
    nxt, prv = np.roll(surf, -1, 0), np.roll(surf, 1, 0)
    tang = nxt - prv
    normal = np.stack([tang[:, 1], -tang[:, 0]], 1)
    normal /= np.linalg.norm(normal, axis=1, keepdims=True)
    # orient outward: away from the section's centroid line
    cx = surf - np.array([0.5, 0.0])
    sign = np.sign(np.sum(normal * cx, axis=1))
    sign[sign == 0] = 1.0
    normal *= sign[:, None]
    ds = 0.5 * np.linalg.norm(tang, axis=1)                  # local surface spacing
    layers, h, dist = [surf], h1, 0.0
    while True:
        dist += h
        live = h < ds
        if not live.any() or dist > 0.5:
            break
        layers.append((surf + dist * normal)[live])
        h *= growth
    inner = np.concatenate(layers)
    r0 = 0.5 + dist + 0.1
    u = uniform01(_sub_seed(seed, 52), n_far)
    v = uniform01(_sub_seed(seed, 53), n_far)
    r = r0 * np.exp(u * np.log(r_far / r0))
    ang = 2 * np.pi * v
    far = np.stack([0.5 + r * np.cos(ang), r * np.sin(ang)], 1)
    n_ring = 2000
    a = 2 * np.pi * np.arange(n_ring) / n_ring
    ring = np.stack([0.5 + r_far * np.cos(a), r_far * np.sin(a)], 1)
    pts = np.concatenate([inner, far[r < r_far * 0.999], ring])
    dmask = np.zeros(len(pts), dtype=bool)
    dmask[-n_ring:] = True
    return pts, dmask, m


def c5_problem(seed: int = 0, n_rhs: int = 50, **kw):
    """Airfoil pressure sequence (C5): the FV Laplacian of naca_points, with
    the wall (inside of the section) removed, and n_rhs right-hand sides
    f_t = f_{t-1} + 0.05 g_t, f_0 = g_0, each g a zero-mean sum of 16 Fourier
    modes with wave numbers 1..3 over the farfield diameter.
    Returns (A, list of f_t, camber m)."""
    pts, dmask, m = naca_points(seed, **kw)

    def inside(c):
        x = c[:, 0]
        ok = (x > 0.0) & (x < 1.0)
        xc = np.clip(x, 0.0, 1.0)
        yc, _, yt = _naca(xc, m)
        return ok & (np.abs(c[:, 1] - yc) < yt)

    A, st = delaunay_fv(pts, dmask, drop=inside)
    xy = pts[st["live"]]
    L = 40.0
    seqs, f = [], None
    for t in range(n_rhs):
        s = _sub_seed(seed, 1000 + t)
        kx = np.floor(1 + 3 * uniform01(_sub_seed(s, 1), 16))
        ky = np.floor(1 + 3 * uniform01(_sub_seed(s, 2), 16))
        ph = 2 * np.pi * uniform01(_sub_seed(s, 3), 16)
        amp = uniform_pm1(_sub_seed(s, 4), 16)
        g = np.zeros(len(xy))
        for k in range(16):
            g += amp[k] * np.sin(2 * np.pi * (kx[k] * xy[:, 0] + ky[k] * xy[:, 1]) / L + ph[k])
        g -= g.mean()
        f = g if f is None else f + 0.05 * g
        seqs.append(f.copy())
    return A, seqs, m


def rhs_uniform(seed: int, n: int) -> np.ndarray:
    """b ~ U[-1, 1)."""
    return uniform_pm1(_sub_seed(seed, 11), n)


def rhs_zero_mean(seed: int, n: int) -> np.ndarray:
    """b = xi - mean(xi), xi ~ U[-1, 1)."""
    xi = uniform_pm1(_sub_seed(seed, 13), n)
    return xi - xi.mean()


# ----------------------------------------------------------------------------
# random initial network parameters
# ----------------------------------------------------------------------------
# (size, fan_in) of each parameter tensor in flat order.  The order is the
# parameter-vector interface of the coefficient network of GCIN width H
# (64, or 32 for the cheaper network): conv linears (weight [in][out] then
# bias) for 4 layers, instance-norm affine (gamma, beta) for 4 layers,
# per-layer readout linears 2H->32, layer norm (gamma, beta), head linears
# 128->128, 128->64, 64->5.  fan_in = 0 marks gamma (init 1) and -1 marks
# beta (init 0).
def gcin_param_sizes(hidden: int = 64):
    H = hidden
    return ([(2 * H, 2), (H, 2)]
            + [(H * H, H), (H, H)] * 3
            + [(H, 0), (H, -1)] * 4
            + [(2 * H * 32, 2 * H), (32, 2 * H)] * 4
            + [(128, 0), (128, -1)]
            + [(128 * 128, 128), (128, 128), (128 * 64, 128), (64, 128), (64 * 5, 64), (5, 64)])


GCIN_PARAM_SIZES = gcin_param_sizes(64)


def gcin_init_params(seed: int, last_bias=(2.0 / 3.0, 0.0, 0.0, 0.0, 0.0), last_scale: float = 0.1,
                     hidden: int = 64) -> np.ndarray:
    """Flat float64 parameter vector: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights.

    The last layer's weights are scaled by ``last_scale`` and its bias set to
    ``last_bias`` so that an untrained network starts near weighted Jacobi.
    """
    parts = []
    for t, (size, fan_in) in enumerate(gcin_param_sizes(hidden)):
        if fan_in == 0:
            parts.append(np.ones(size))
        elif fan_in == -1:
            parts.append(np.zeros(size))
        else:
            parts.append(uniform_pm1(_sub_seed(seed, 100 + t), size) / np.sqrt(fan_in))
    parts[-2] = parts[-2] * last_scale
    parts[-1] = np.asarray(last_bias, dtype=np.float64).copy()
    return np.concatenate(parts)
