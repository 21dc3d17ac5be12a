"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the method (no kernel, no transform, no
sum over cell pairs): it only turns a shape into the boundary cell list that
``bem_plan`` takes (grid index, boundary measure w, outward normal) and
evaluates analytic harmonic fields and random densities on it.

Discretisation of a shape (Section 3: the boundary S lies *within* a uniform
grid that encloses it; Section 4: the grid over the unit square with n nodes
per side):
  * grid spacing h = 1/n, node k at (k + 1/2) h, cell k = [k h, (k+1) h)
    (half-open floor rule, so every boundary point belongs to exactly one cell);
  * a boundary cell is a grid cell that contains a positive length (2D) or
    area (3D) of S;
  * w_j is that in-cell length/area (the boundary measure the cell carries);
  * p_j is the sample of S inside the cell closest to the in-cell centroid of
    S, and the analytic outward normal n_j and the data u, q are evaluated
    there.
Seeds: numpy PCG64 with seed = 180900845 + config index unless given.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 180900845


@dataclasses.dataclass
class Boundary:
    """Boundary cell list on an n^dim grid over the unit square/cube."""

    dim: int
    n: int
    cell: np.ndarray      # (nb, dim) int32 grid indices, axis 0 = x
    w: np.ndarray         # (nb,) boundary measure carried by each cell
    normal: np.ndarray    # (nb, dim) unit outward normals at p
    point: np.ndarray     # (nb, dim) boundary point p_j inside the cell
    param: np.ndarray     # (nb,) or (nb, 2) curve/surface parameter of p_j

    @property
    def nb(self) -> int:
        return int(self.cell.shape[0])

    @property
    def h(self) -> float:
        return 1.0 / self.n


# ----------------------------------------------------------------- 2D curves --

def star_curve(r0=0.3, eps=0.3, k=5, centre=(0.5, 0.5)):
    """r(theta) = r0 (1 + eps cos(k theta)) about ``centre`` (counter-clockwise)."""
    cx, cy = centre

    def f(t):
        r = r0 * (1.0 + eps * np.cos(k * t))
        dr = -r0 * eps * k * np.sin(k * t)
        c, s = np.cos(t), np.sin(t)
        p = np.stack([cx + r * c, cy + r * s], axis=-1)
        dp = np.stack([dr * c - r * s, dr * s + r * c], axis=-1)
        return p, dp

    return f


def circle_curve(radius=0.35, centre=(0.5, 0.5)):
    return star_curve(r0=radius, eps=0.0, k=0, centre=centre)


def random_star_curve(rng: np.random.Generator, r0=0.3, kmin=2, kmax=6, amax=0.05, centre=(0.5, 0.5)):
    """r(theta) = r0 (1 + sum_k a_k cos(k theta + phi_k)), a_k ~ U(0, amax)."""
    ks = np.arange(kmin, kmax + 1)
    a = rng.uniform(0.0, amax, size=ks.size)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=ks.size)
    cx, cy = centre

    def f(t):
        t = np.asarray(t)
        arg = ks[None, :] * t[..., None] + phi[None, :]
        r = r0 * (1.0 + np.sum(a * np.cos(arg), axis=-1))
        dr = -r0 * np.sum(a * ks * np.sin(arg), axis=-1)
        c, s = np.cos(t), np.sin(t)
        p = np.stack([cx + r * c, cy + r * s], axis=-1)
        dp = np.stack([dr * c - r * s, dr * s + r * c], axis=-1)
        return p, dp

    f.coeffs = (ks, a, phi)
    return f


def curve_boundary(n: int, curve, samples_per_cell: int = 64) -> Boundary:
    """Boundary cells of a closed counter-clockwise curve on an n x n grid.

    Cells are returned in the order the curve first enters them (arclength
    order starting at theta = 0)."""
    h = 1.0 / n
    tc = (np.arange(4096) + 0.5) * (2 * math.pi / 4096)
    _, dpc = curve(tc)
    length = float(np.sum(np.hypot(dpc[:, 0], dpc[:, 1])) * (2 * math.pi / 4096))
    m = int(math.ceil(samples_per_cell * length / h))
    dt = 2.0 * math.pi / m
    t = (np.arange(m) + 0.5) * dt
    p, dp = curve(t)
    speed = np.hypot(dp[:, 0], dp[:, 1])
    ds = speed * dt
    g = np.floor(p / h).astype(np.int64)
    if g.min() < 0 or g.max() >= n:
        raise ValueError("curve leaves the unit square")
    key = g[:, 1] * n + g[:, 0]
    uniq, first, inv = np.unique(key, return_index=True, return_inverse=True)
    nb = uniq.size
    w = np.bincount(inv, weights=ds, minlength=nb)
    cen = np.stack([np.bincount(inv, weights=p[:, a] * ds, minlength=nb) for a in range(2)], axis=-1) / w[:, None]
    dist = np.hypot(p[:, 0] - cen[inv, 0], p[:, 1] - cen[inv, 1])
    order = np.lexsort((dist, inv))
    pick = order[np.searchsorted(inv[order], np.arange(nb))]
    tj = t[pick]
    pj, dpj = curve(tj)
    sp = np.hypot(dpj[:, 0], dpj[:, 1])
    nrm = np.stack([dpj[:, 1] / sp, -dpj[:, 0] / sp], axis=-1)
    cells = np.stack([uniq % n, uniq // n], axis=-1)
    arc = np.argsort(first, kind="stable")
    return Boundary(2, n, cells[arc].astype(np.int32), w[arc], nrm[arc], pj[arc], tj[arc])


def circle_boundary(n: int = 128, radius: float = 0.35, samples_per_cell: int = 64) -> Boundary:
    return curve_boundary(n, circle_curve(radius), samples_per_cell)


def star_boundary(n: int = 4096, samples_per_cell: int = 64) -> Boundary:
    return curve_boundary(n, star_curve(0.3, 0.3, 5), samples_per_cell)


def square_boundary(n: int) -> Boundary:
    """The paper's Section 4 example: grid-aligned square whose sides run through
    node rows/columns n/4 and 3n/4 (nodes lie exactly on S, w = h)."""
    lo, hi = n // 4, (3 * n) // 4
    cells, nrm = [], []
    for gx in range(lo, hi + 1):
        for gy in range(lo, hi + 1):
            if gx in (lo, hi) or gy in (lo, hi):
                nx = (-1.0 if gx == lo else 1.0 if gx == hi else 0.0)
                ny = (-1.0 if gy == lo else 1.0 if gy == hi else 0.0)
                nn = math.hypot(nx, ny)
                cells.append((gx, gy))
                nrm.append((nx / nn, ny / nn))
    cells = np.array(cells, dtype=np.int32)
    h = 1.0 / n
    w = np.full(len(cells), h)
    pts = (cells + 0.5) * h
    return Boundary(2, n, cells, w, np.array(nrm), pts, np.zeros(len(cells)))


def full_plane_boundary(n: int, rng: np.random.Generator) -> Boundary:
    """Every cell of the n x n grid (the half-space special case of Eq. 9:
    the boundary fills the whole parameter space).  Random unit normals."""
    gx, gy = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    cells = np.stack([gx.ravel(), gy.ravel()], axis=-1).astype(np.int32)
    ang = rng.uniform(0, 2 * math.pi, size=cells.shape[0])
    nrm = np.stack([np.cos(ang), np.sin(ang)], axis=-1)
    w = rng.uniform(0.5, 1.5, size=cells.shape[0]) / n
    return Boundary(2, n, cells, w, nrm, (cells + 0.5) / n, np.zeros(cells.shape[0]))


def random_cells(n: int, nb: int, rng: np.random.Generator, dim: int = 2) -> Boundary:
    """nb distinct random cells with random weights and unit normals (a
    boundary-free stress input for parity: any cell set is a valid operand)."""
    total = n ** dim
    nb = min(nb, total)
    flat = rng.choice(total, size=nb, replace=False)
    cells = np.stack([(flat // n ** a) % n for a in range(dim)], axis=-1).astype(np.int32)
    v = rng.normal(size=(nb, dim))
    nrm = v / np.linalg.norm(v, axis=1, keepdims=True)
    w = rng.uniform(0.5, 1.5, size=nb) / n ** (dim - 1)
    return Boundary(dim, n, cells, w, nrm, (cells + 0.5) / n, np.zeros(nb))


# ---------------------------------------------------------------- 3D surfaces --

def ellipsoid_boundary(n: int = 256, axes=(0.4, 0.3, 0.2), centre=(0.5, 0.5, 0.5),
                       samples_per_cell: int = 6) -> Boundary:
    """Boundary cells of an ellipsoid on an n^3 grid.  The surface is sampled
    on a (theta, phi) grid fine enough that neighbouring samples are at most
    h / samples_per_cell apart; w_j = in-cell area (sum of the samples' area
    elements), normal = analytic at the in-cell sample closest to the in-cell
    centroid.  Cells are returned sorted by (theta, phi) of their first sample."""
    a, b, c = axes
    h = 1.0 / n
    amax = max(axes)
    d = h / samples_per_cell / amax
    nt = int(math.ceil(math.pi / d))
    npf = int(math.ceil(2 * math.pi / d))
    cells_acc = {}
    th = (np.arange(nt) + 0.5) * (math.pi / nt)
    dth = math.pi / nt
    dph = 2 * math.pi / npf
    keys_all, area_all, pts_all, par_all = [], [], [], []
    chunk = max(1, 2_000_000 // npf)
    ph = (np.arange(npf) + 0.5) * dph
    for i0 in range(0, nt, chunk):
        t = th[i0:i0 + chunk][:, None]
        st, ct = np.sin(t), np.cos(t)
        cp, sp = np.cos(ph)[None, :], np.sin(ph)[None, :]
        x = centre[0] + a * st * cp
        y = centre[1] + b * st * sp
        z = centre[2] + c * ct * np.ones_like(cp)
        # |p_theta x p_phi|
        nx, ny, nz = b * c * st * st * cp, a * c * st * st * sp, a * b * st * ct * np.ones_like(cp)
        dA = np.sqrt(nx * nx + ny * ny + nz * nz) * dth * dph
        P = np.stack([x, y, z], axis=-1).reshape(-1, 3)
        g = np.floor(P / h).astype(np.int64)
        keys_all.append((g[:, 2] * n + g[:, 1]) * n + g[:, 0])
        area_all.append(dA.reshape(-1))
        pts_all.append(P)
        par_all.append(np.stack([np.broadcast_to(t, x.shape), np.broadcast_to(ph[None, :], x.shape)],
                                axis=-1).reshape(-1, 2))
    key = np.concatenate(keys_all)
    dA = np.concatenate(area_all)
    P = np.concatenate(pts_all)
    par = np.concatenate(par_all)
    uniq, first, inv = np.unique(key, return_index=True, return_inverse=True)
    nb = uniq.size
    w = np.bincount(inv, weights=dA, minlength=nb)
    cen = np.stack([np.bincount(inv, weights=P[:, k] * dA, minlength=nb) for k in range(3)], axis=-1) / w[:, None]
    dist = np.linalg.norm(P - cen[inv], axis=1)
    order = np.lexsort((dist, inv))
    pick = order[np.searchsorted(inv[order], np.arange(nb))]
    pj = P[pick]
    grad = np.stack([(pj[:, 0] - centre[0]) / a ** 2, (pj[:, 1] - centre[1]) / b ** 2,
                     (pj[:, 2] - centre[2]) / c ** 2], axis=-1)
    nrm = grad / np.linalg.norm(grad, axis=1, keepdims=True)
    cells = np.stack([uniq % n, (uniq // n) % n, uniq // (n * n)], axis=-1).astype(np.int32)
    arc = np.argsort(first, kind="stable")
    return Boundary(3, n, cells[arc], w[arc], nrm[arc], pj[arc], par[pick][arc])


def cube_boundary(n: int = 128, lo: int = None, hi: int = None) -> Boundary:
    """Cube whose faces run through the node planes lo and hi (default n/4
    and 3n/4: side 0.5 for the unit box): every grid cell whose node lies on
    the surface.  Face cells carry w = h^2; cells on an edge carry the two
    half-cells h^2/2 + h^2/2 and an averaged normal; corner cells carry
    3 (h/2)^2 and the averaged normal of the three faces."""
    lo = n // 4 if lo is None else lo
    hi = (3 * n) // 4 if hi is None else hi
    h = 1.0 / n
    rng = np.arange(lo, hi + 1)
    gx, gy, gz = np.meshgrid(rng, rng, rng, indexing="ij")
    g = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=-1)
    on = (g == lo) | (g == hi)
    keep = on.any(axis=1)
    g, on = g[keep], on[keep]
    nrm = np.where(g == hi, 1.0, 0.0) - np.where(g == lo, 1.0, 0.0)
    k = on.sum(axis=1)
    w = np.where(k == 1, h * h, np.where(k == 2, h * h, 0.75 * h * h))
    nrm = nrm / np.linalg.norm(nrm, axis=1, keepdims=True)
    order = np.lexsort((g[:, 0], g[:, 1], g[:, 2]))
    g = g[order].astype(np.int32)
    return Boundary(3, n, g, w[order], nrm[order], (g + 0.5) * h, k[order].astype(np.float64))


# ------------------------------------------------------------ analytic fields --

@dataclasses.dataclass
class PanelBoundary:
    """A closed curve as nb straight panels (accuracy mode): panel j runs from
    vertex j to vertex j + 1 (cyclic), vertices on the curve, equally spaced in
    arclength, counter-clockwise (outward normal = tangent turned clockwise).
    ``param`` is the curve parameter of each panel's first vertex."""

    n: int
    panels: np.ndarray    # (nb, 4): A.x, A.y, B.x, B.y
    param: np.ndarray     # (nb,)

    @property
    def nb(self) -> int:
        return int(self.panels.shape[0])

    @property
    def h(self) -> float:
        return 1.0 / self.n

    @property
    def mid(self) -> np.ndarray:
        return 0.5 * (self.panels[:, 0:2] + self.panels[:, 2:4])

    @property
    def length(self) -> np.ndarray:
        d = self.panels[:, 2:4] - self.panels[:, 0:2]
        return np.hypot(d[:, 0], d[:, 1])

    @property
    def normal(self) -> np.ndarray:
        d = self.panels[:, 2:4] - self.panels[:, 0:2]
        d = d / np.hypot(d[:, 0], d[:, 1])[:, None]
        return np.stack([d[:, 1], -d[:, 0]], axis=1)


def curve_panels(n: int, curve, panels_per_h: float = 1.0, samples: int = 1 << 16) -> PanelBoundary:
    """Flat panels of length about h / panels_per_h on a closed curve; the
    vertices are placed at equal arclength (the curve's length from a fine
    trapezoid sum, inverted by linear interpolation)."""
    t = np.linspace(0.0, 2.0 * math.pi, samples + 1)
    _, dp = curve(t)
    sp = np.hypot(dp[:, 0], dp[:, 1])
    s = np.concatenate([[0.0], np.cumsum(0.5 * (sp[1:] + sp[:-1]) * np.diff(t))])
    nb = max(3, int(math.ceil(s[-1] * n * panels_per_h)))
    tv = np.interp(np.arange(nb) * (s[-1] / nb), s, t)
    v, _ = curve(tv)
    if v.min() <= 0.0 or v.max() >= 1.0:
        raise ValueError("curve leaves the unit square")
    panels = np.concatenate([v, np.roll(v, -1, axis=0)], axis=1)
    return PanelBoundary(n, panels, tv)


def panel_data(b: PanelBoundary, field):
    """(u, q) of an analytic field at the panel midpoints, q = n . grad u."""
    u, g = field(b.mid)
    return u, np.sum(g * b.normal, axis=-1)


def field_x2y2(p):
    """u = x^2 - y^2 and its gradient (harmonic)."""
    x, y = p[..., 0], p[..., 1]
    return x * x - y * y, np.stack([2 * x, -2 * y], axis=-1)


def field_expcos(p):
    """u = e^x cos y and its gradient (harmonic)."""
    x, y = p[..., 0], p[..., 1]
    e = np.exp(x)
    return e * np.cos(y), np.stack([e * np.cos(y), -e * np.sin(y)], axis=-1)


def field_xy_z(p):
    """u = x y + z and its gradient (harmonic, 3D)."""
    x, y, z = p[..., 0], p[..., 1], p[..., 2]
    return x * y + z, np.stack([y, x, np.ones_like(z)], axis=-1)


def boundary_data(b: Boundary, field):
    """(u, q) of an analytic field at the boundary points, q = n . grad u."""
    u, g = field(b.point)
    return u, np.sum(g * b.normal, axis=-1)


def mixed_bc_theta(b: Boundary) -> np.ndarray:
    """Dirichlet (0) for curve parameter theta < pi, Neumann (1) elsewhere."""
    return (np.asarray(b.param) >= math.pi).astype(np.uint8)


def random_density(nb: int, rng: np.random.Generator, ncomp: int = 1) -> np.ndarray:
    x = rng.standard_normal(size=(nb, ncomp) if ncomp > 1 else nb)
    return x


def rng_for(config_index: int, offset: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + config_index + offset))
