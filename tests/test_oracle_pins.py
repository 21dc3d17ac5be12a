"""Pins of the CPU oracle to facts outside itself (no GPU).

Each test ties one part of the oracle to something the paper or the
mathematics fixes: closed-form cell averages against numerical quadrature,
Green's identity (Eq. 4 with c = 1 inside, 0 outside) with spectrally accurate
quadrature, Somigliana's identity (Eq. 8) for rigid and linear elastic fields,
the half-space special case (Eq. 9: a boundary filling the whole grid is a
plain 2D convolution, checked with scipy's convolution), and the dense LU
solve.  A dropped term, a wrong sign, a transposed offset (source minus
target instead of target minus source) or a wrong prefactor in any kernel
fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy import integrate, signal

from paper_1809_00845_gb300 import inputs as I


# ------------------------------------------------------ singular-cell constants

def test_L2_closed_form_matches_quadrature(oracle_mod):
    # mean of ln r over [-1/2, 1/2]^2 = 4 * integral over [0, 1/2]^2
    val, err = integrate.dblquad(lambda y, x: 0.5 * math.log(x * x + y * y), 0.0, 0.5, 0.0, 0.5,
                                 epsabs=1e-13, epsrel=1e-13)
    assert abs(4.0 * val - oracle_mod.L2()) < 1e-10
    assert abs(oracle_mod.L2() - (-1.0611754268825244)) < 1e-15


def test_C3_closed_form_matches_quadrature(oracle_mod):
    # integral of 1/r over the unit cube = 8 * integral over [0, 1/2]^3; the
    # z-integral is done in closed form (asinh), the rest numerically.
    f = lambda y, x: math.asinh(0.5 / math.hypot(x, y)) if (x > 0 or y > 0) else 0.0
    val, err = integrate.dblquad(f, 0.0, 0.5, 0.0, 0.5, epsabs=1e-13, epsrel=1e-13)
    assert abs(8.0 * val - oracle_mod.C3()) < 1e-9


@pytest.mark.parametrize("h", [1.0 / 8, 1.0 / 128, 1.0 / 4096])
def test_2d_singular_cell_is_cell_average(oracle_mod, h):
    # average of -ln r / (2 pi) over the h-square centred at the node
    val, _ = integrate.dblquad(lambda y, x: -0.25 * math.log(x * x + y * y) / math.pi, 0.0, h / 2, 0.0, h / 2,
                               epsabs=1e-14, epsrel=1e-12)
    avg = 4.0 * val / (h * h)
    assert abs(_lap2d_U0(oracle_mod, h) - avg) < 1e-10


def _lap2d_U0(oracle_mod, h):
    return oracle_mod._load().bo_lap2d_U(0.0, 0.0, h)


@pytest.mark.parametrize("h", [1.0 / 16, 1.0 / 256])
def test_3d_singular_cell_is_cell_average(oracle_mod, h):
    f = lambda y, x: math.asinh((h / 2) / math.hypot(x, y)) / (4 * math.pi) if (x > 0 or y > 0) else 0.0
    val, _ = integrate.dblquad(f, 0.0, h / 2, 0.0, h / 2, epsabs=1e-14, epsrel=1e-12)
    avg = 8.0 * val / h ** 3
    assert abs(oracle_mod._load().bo_lap3d_U(0.0, 0.0, 0.0, h) - avg) < 1e-9 * avg


def test_kelvin_singular_cell_is_cell_average(oracle_mod):
    nu, mu, h = 0.3, 1.0, 1.0 / 64
    # average of Eq. 7 over the cube, by quadrature in spherical-safe form:
    # <d_x^2 / r^3> over the cube via tplquad on [0, h/2]^3 (8-fold symmetry).
    g = lambda z, y, x: (x * x) / (x * x + y * y + z * z) ** 1.5
    inv_r = lambda z, y, x: 1.0 / math.sqrt(x * x + y * y + z * z)
    opts = dict(epsabs=1e-10, epsrel=1e-8)
    gxx = 8 * integrate.tplquad(g, 0, h / 2, 0, h / 2, 0, h / 2, **opts)[0] / h ** 3
    ir = 8 * integrate.tplquad(inv_r, 0, h / 2, 0, h / 2, 0, h / 2, **opts)[0] / h ** 3
    expect = ((3 - 4 * nu) * ir + gxx) / (16 * math.pi * mu * (1 - nu))
    # the singular block through the matrix assembly of a one-cell boundary
    A = oracle_mod.matrix("kelvin3d", 0, np.zeros((1, 3), np.int32), h, np.ones(1), np.array([[1.0, 0, 0]]), nu, mu)
    assert np.allclose(np.diag(A), expect, rtol=1e-6)
    assert np.allclose(A - np.diag(np.diag(A)), 0.0)


# ------------------------------------------------------------ Green's identity

def _circle_quadrature(m, R, c):
    t = 2 * math.pi * np.arange(m) / m
    p = np.stack([c[0] + R * np.cos(t), c[1] + R * np.sin(t)], axis=-1)
    n = np.stack([np.cos(t), np.sin(t)], axis=-1)
    ds = np.full(m, 2 * math.pi * R / m)
    return p, n, ds


@pytest.mark.parametrize("field", [I.field_x2y2, I.field_expcos])
def test_green_identity_2d(oracle_mod, field):
    """Eq. 4/Eq. 15 with the oracle's kernels: sum U q + sum Q.n u = c u(x0),
    c = 1 inside, 0 outside (trapezoidal rule is spectral for a smooth periodic
    integrand)."""
    R, c = 0.3, (0.5, 0.5)
    p, n, ds = _circle_quadrature(600, R, c)
    u, g = field(p)
    q = np.sum(g * n, axis=-1)
    for x0, inside in [((0.5, 0.5), 1), ((0.62, 0.41), 1), ((0.35, 0.7), 1), ((0.95, 0.5), 0), ((0.1, 0.1), 0)]:
        acc = 0.0
        for k in range(p.shape[0]):
            d = [x0[0] - p[k, 0], x0[1] - p[k, 1]]
            acc += oracle_mod.kernel_point("laplace2d", 0, d) * q[k] * ds[k]
            acc += oracle_mod.kernel_point("laplace2d", 1, d, n[k]) * u[k] * ds[k]
        u0 = field(np.array(x0))[0]
        assert abs(acc - inside * u0) < 1e-10, (x0, acc, u0)


def _sphere_quadrature(nt, nphi, R, c):
    xg, wg = np.polynomial.legendre.leggauss(nt)  # cos(theta)
    phi = 2 * math.pi * np.arange(nphi) / nphi
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    n = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=-1).reshape(-1, 3)
    p = np.asarray(c)[None, :] + R * n
    dA = (R * R * wg[:, None] * np.full_like(ph, 2 * math.pi / nphi)).reshape(-1)
    return p, n, dA


def test_green_identity_3d(oracle_mod):
    R, c = 0.3, (0.5, 0.5, 0.5)
    p, n, dA = _sphere_quadrature(40, 80, R, c)
    u, g = I.field_xy_z(p)
    q = np.sum(g * n, axis=-1)
    for x0, inside in [((0.5, 0.5, 0.5), 1), ((0.6, 0.45, 0.4), 1), ((0.9, 0.5, 0.5), 0)]:
        acc = 0.0
        for k in range(p.shape[0]):
            d = np.asarray(x0) - p[k]
            acc += oracle_mod.kernel_point("laplace3d", 0, d) * q[k] * dA[k]
            acc += oracle_mod.kernel_point("laplace3d", 1, d, n[k]) * u[k] * dA[k]
        u0 = I.field_xy_z(np.array(x0))[0]
        assert abs(acc - inside * u0) < 1e-9, (x0, acc, u0)


# -------------------------------------------------------- Somigliana identity

@pytest.mark.parametrize("kind", ["rigid", "diag", "general"])
def test_somigliana_kelvin(oracle_mod, kind):
    """Eq. 8 at interior points: u(x0) = int U t dS - int T u dS for an
    elastic field with constant stress (linear displacement, Hooke's law with
    lambda = 2 mu nu / (1 - 2 nu)), t = sigma n.  Rigid translation has t = 0."""
    nu, mu = 0.3, 1.0
    lam = 2 * mu * nu / (1 - 2 * nu)
    rng = np.random.default_rng(7)
    if kind == "rigid":
        G, u0 = np.zeros((3, 3)), np.array([0.3, -0.2, 0.5])
    elif kind == "diag":
        G, u0 = np.diag([0.01, -0.003, 0.002]), np.zeros(3)
    else:
        G, u0 = rng.normal(size=(3, 3)) * 0.01, rng.normal(size=3) * 0.1
    eps = 0.5 * (G + G.T)
    sig = lam * np.trace(eps) * np.eye(3) + 2 * mu * eps
    if kind == "diag":
        assert np.allclose(np.diag(sig), [0.0335, 0.0075, 0.0175])
    R, c = 0.3, np.array([0.5, 0.5, 0.5])
    p, n, dA = _sphere_quadrature(40, 80, R, c)
    u = u0[None, :] + p @ G.T
    t = n @ sig.T
    for x0 in [np.array([0.5, 0.5, 0.5]), np.array([0.58, 0.44, 0.61])]:
        acc = np.zeros(3)
        for k in range(p.shape[0]):
            d = x0 - p[k]
            acc += oracle_mod.kernel_point("kelvin3d", 0, d, None, nu, mu) @ t[k] * dA[k]
            acc -= oracle_mod.kernel_point("kelvin3d", 1, d, n[k], nu, mu) @ u[k] * dA[k]
        expect = u0 + G @ x0
        assert np.allclose(acc, expect, atol=1e-9), (acc, expect)


# ------------------------------------------- half-space case (Eq. 9) structure

@pytest.mark.parametrize("layer", [0, 1])
def test_full_plane_is_plain_convolution(oracle_mod, layer):
    """When the boundary fills the whole n x n grid, the direct sum is the 2D
    linear convolution of the kernel table with the weighted density (Eq. 9)."""
    n = 12
    rng = np.random.default_rng(3)
    b = I.full_plane_boundary(n, rng)
    h = b.h
    x = rng.standard_normal(b.nb)
    out = oracle_mod.apply("laplace2d", layer, b.cell, h, b.w, b.normal, x)
    # densities on the grid image[gy, gx]
    offs = np.arange(-(n - 1), n)
    if layer == 0:
        img = np.zeros((n, n))
        img[b.cell[:, 1], b.cell[:, 0]] = b.w * x
        K = np.array([[_k2(oracle_mod, 0, dx * h, dy * h, h) for dx in offs] for dy in offs])
        conv = signal.convolve2d(img, K, mode="full")[n - 1:2 * n - 1, n - 1:2 * n - 1]
    else:
        conv = 0.0
        for a in range(2):
            img = np.zeros((n, n))
            img[b.cell[:, 1], b.cell[:, 0]] = b.w * b.normal[:, a] * x
            K = np.array([[_k2q(oracle_mod, a, dx * h, dy * h) for dx in offs] for dy in offs])
            conv = conv + signal.convolve2d(img, K, mode="full")[n - 1:2 * n - 1, n - 1:2 * n - 1]
    ref = conv[b.cell[:, 1], b.cell[:, 0]]
    assert np.allclose(out, ref, rtol=1e-12, atol=1e-12)


def _k2(o, layer, dx, dy, h):
    return o._load().bo_lap2d_U(dx, dy, h)


def _k2q(o, a, dx, dy):
    return o._load().bo_lap2d_Q(a, dx, dy)


# ------------------------------------------------------------ dense LU solve

def test_dense_lu_solves_mixed_system(oracle_mod):
    b = I.circle_boundary(16, 0.3)
    u, q = I.boundary_data(b, I.field_x2y2)
    bc = I.mixed_bc_theta(b)
    A, rhs = oracle_mod.system("laplace2d", b.cell, b.h, b.w, b.normal, bc, u, q)
    x = oracle_mod.solve_lu(A, rhs)
    assert np.linalg.norm(A @ x - rhs) <= 1e-12 * np.linalg.norm(rhs)
    # the matrix-free direct-sum form of the same system agrees with the dense one
    y = oracle_mod.system_apply("laplace2d", b.cell, b.h, b.w, b.normal, bc, x)
    assert np.allclose(y, A @ x, rtol=1e-12, atol=1e-13)
    r2 = oracle_mod.system_rhs("laplace2d", b.cell, b.h, b.w, b.normal, bc, u, q)
    assert np.allclose(r2, rhs, rtol=1e-12, atol=1e-13)
    # brute-force Gaussian elimination (no pivoting library) on the same system
    M = np.concatenate([A, rhs[:, None]], axis=1).copy()
    m = M.shape[0]
    for col in range(m):
        piv = col + int(np.argmax(np.abs(M[col:, col])))
        M[[col, piv]] = M[[piv, col]]
        M[col + 1:] -= np.outer(M[col + 1:, col] / M[col, col], M[col])
    xb = np.zeros(m)
    for r in range(m - 1, -1, -1):
        xb[r] = (M[r, -1] - M[r, r + 1:m] @ xb[r + 1:]) / M[r, r]
    assert np.allclose(xb, x, rtol=1e-9, atol=1e-12)


def test_rows_slice_matches_full(oracle_mod):
    rng = np.random.default_rng(11)
    b = I.random_cells(16, 40, rng, dim=3)
    x = rng.standard_normal((b.nb, 3))
    full = oracle_mod.apply("kelvin3d", 1, b.cell, b.h, b.w, b.normal, x)
    part = oracle_mod.apply("kelvin3d", 1, b.cell, b.h, b.w, b.normal, x, rows=(5, 7))
    assert np.array_equal(full[5:12], part)


@pytest.mark.parametrize("kernel", ["laplace2d", "laplace3d", "kelvin3d"])
def test_split_system_is_the_unsplit_equation(oracle_mod, kernel):
    """The boundary-condition split against the equation it splits: for any
    data (u, q) and any split, A x - b with x = q on Dirichlet and u on
    Neumann entries equals the residual of the BIE as the paper writes it,
    S q + D u - c u for Laplace (Eq. 15, Eq. 4) and U t - T u - c u for Navier
    (Eq. 8), with the direct-sum operators."""
    rng = np.random.default_rng(17)
    dim = 2 if kernel == "laplace2d" else 3
    b = I.random_cells(16, 30, rng, dim=dim)
    nc = 3 if kernel == "kelvin3d" else 1
    u = rng.standard_normal(b.nb * nc)
    q = rng.standard_normal(b.nb * nc)
    c = 0.5
    args = (b.cell, b.h, b.w, b.normal)
    Sq = oracle_mod.apply(kernel, 0, *args, q).reshape(-1)
    Du = oracle_mod.apply(kernel, 1, *args, u).reshape(-1)
    residual = Sq + (Du if kernel != "kelvin3d" else -Du) - c * u
    for trial in range(3):
        bc = (rng.uniform(size=b.nb * nc) < 0.5).astype(np.uint8)
        x = np.where(bc == 0, q, u)
        A, rhs = oracle_mod.system(kernel, *args, bc, u, q, c=c)
        assert np.allclose(A @ x - rhs, residual, rtol=1e-12, atol=1e-12)
        y = oracle_mod.system_apply(kernel, *args, bc, x, c=c) - oracle_mod.system_rhs(kernel, *args, bc, u, q, c=c)
        assert np.allclose(y, residual, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("kernel", ["laplace2d", "laplace3d", "kelvin3d"])
def test_right_hand_side_is_the_complementary_split_applied_to_the_data(oracle_mod, kernel):
    """The reading behind the one-apply right-hand side of the GPU solves: with
    data d (u on the Dirichlet entries, q on the Neumann entries), the known
    terms b of the split equation are minus the split operator of the
    complementary mask applied to d, since swapping the mask swaps which layer
    each entry feeds and moves the c u term onto the Dirichlet entries
    (Eq. 15 with the BC split; Eq. 8 for Navier)."""
    rng = np.random.default_rng(23)
    dim = 2 if kernel == "laplace2d" else 3
    b = I.random_cells(16, 30, rng, dim=dim)
    nc = 3 if kernel == "kelvin3d" else 1
    args = (b.cell, b.h, b.w, b.normal)
    for trial in range(3):
        u = rng.standard_normal(b.nb * nc)
        q = rng.standard_normal(b.nb * nc)
        bc = (rng.uniform(size=b.nb * nc) < 0.5).astype(np.uint8)
        c = 0.5 if trial else 0.25
        d = np.where(bc == 0, u, q)
        rhs = oracle_mod.system_rhs(kernel, *args, bc, u, q, c=c)
        comp = oracle_mod.system_apply(kernel, *args, 1 - bc, d, c=c)
        assert np.allclose(-comp, rhs, rtol=1e-12, atol=1e-12 * np.abs(rhs).max())


def _double_layer_at_targets(oracle_mod, kernel, b, targets, u):
    """The oracle's assembled double layer of the constant density u, read at
    extra zero-weight target cells (they add no source)."""
    dim = b.dim
    cell = np.concatenate([b.cell, np.asarray(targets, np.int32)])
    w = np.concatenate([b.w, np.zeros(len(targets))])
    nrm = np.concatenate([b.normal, np.tile(np.eye(dim)[0], (len(targets), 1))])
    x = np.tile(u, cell.shape[0])
    return oracle_mod.apply(kernel, 1, cell, b.h, w, nrm, x, rows=(b.nb, len(targets)))


@pytest.mark.parametrize("kernel", ["laplace2d", "laplace3d", "kelvin3d"])
def test_discrete_double_layer_of_a_constant(oracle_mod, kernel):
    """The constant-density invariant through the assembled discrete operator
    (cells, weights = in-cell boundary measure, outward normals, d = target
    minus source): at targets away from the boundary the double layer of u = 1
    is 1 inside and 0 outside (Eq. 4 with q = 0: c = 1 inside, 0 outside), and
    the Kelvin traction operator applied to a rigid translation u0 gives -u0
    inside and 0 outside (Eq. 8 with t = 0).  Measured within 9e-5 (2D, n = 256)
    and 1e-3 (3D, n = 64)."""
    if kernel == "laplace2d":
        n = 256
        b = I.circle_boundary(n, 0.35)
        targets = [[n // 2, n // 2], [n // 2 + n // 10, n // 2 - n // 12], [n // 16, n // 16], [n - 3, n // 2]]
        tol = 5e-4
    else:
        n = 64
        b = I.ellipsoid_boundary(n)
        targets = [[n // 2, n // 2, n // 2], [n // 2 + n // 10, n // 2, n // 2 - n // 20], [2, 2, 2],
                   [n - 2, n // 2, n // 2]]
        tol = 4e-3
    inside = np.array([1.0, 1.0, 0.0, 0.0])
    if kernel == "kelvin3d":
        u0 = np.array([0.3, -0.2, 0.5])
        got = _double_layer_at_targets(oracle_mod, kernel, b, targets, u0)
        assert np.allclose(got, -inside[:, None] * u0[None, :], atol=tol), got
    else:
        got = _double_layer_at_targets(oracle_mod, kernel, b, targets, np.ones(1))
        assert np.allclose(got, inside, atol=tol), got


def test_paper_square_dirichlet_solve_approaches_the_analytic_flux(oracle_mod):
    """The paper's own geometry (Section 4, Fig. 3): a grid-aligned square
    whose sides run through node rows, so the nodes lie on S and w = h.  The
    grid-node solve of the Dirichlet problem u = x^2 - y^2 (A = S, b = u/2 - D u,
    Eq. 15) approaches the analytic flux away from the corners, slowly (the
    corner cells carry averaged normals and the flux jumps there): measured
    5.2e-2, 4.0e-2, 2.7e-2 at n = 64, 128, 256."""
    errs = []
    for n in (64, 128, 256):
        b = I.square_boundary(n)
        u, q = I.boundary_data(b, I.field_x2y2)
        bc = np.zeros(b.nb, np.uint8)
        A, rhs = oracle_mod.system("laplace2d", b.cell, b.h, b.w, b.normal, bc, u, q)
        x = oracle_mod.solve_lu(A, rhs)
        p = b.point
        lo, hi = p.min(axis=0), p.max(axis=0)
        side = hi[0] - lo[0]
        near = np.minimum(np.abs(p - lo), np.abs(p - hi)) < 0.1 * side
        away = ~(near[:, 0] & near[:, 1])
        errs.append(np.linalg.norm((x - q)[away]) / np.linalg.norm(q[away]))
    assert errs[2] < 3.5e-2 and errs[2] < errs[1] < errs[0], errs
