"""Pins of the accuracy-mode oracle (CPU): the flat-panel collocation BEM (O2)
and its grid-accelerated approximation, each checked against something other
than itself -- adaptive quadrature, Gauss's law for the double layer,
convergence to analytic harmonic fields, polynomial reproduction of the
stencils, and the all-near limit."""
import math

import numpy as np
import pytest

from oracle import panel_oracle as PO
from paper_1809_00845_gb300 import inputs as I


def _quad(f, a, b):
    integrate = pytest.importorskip("scipy.integrate")
    return integrate.quad(f, a, b, limit=200, epsabs=1e-15, epsrel=1e-13)[0]


def test_panel_integrals_match_adaptive_quadrature():
    rng = np.random.default_rng(5)
    for _ in range(12):
        A = rng.uniform(0.2, 0.8, 2)
        ang = rng.uniform(0, 2 * math.pi)
        L = rng.uniform(0.001, 0.05)
        B = A + L * np.array([math.cos(ang), math.sin(ang)])
        panel = np.concatenate([A, B])[None, :]
        t = (B - A) / L
        n = np.array([t[1], -t[0]])
        for x in (A + 0.3 * (B - A) + 0.7 * L * n, A - 0.2 * L * n + 1.5 * L * t, A + 2.0 * (B - A),
                  A + 0.5 * (B - A)):
            def y(s):
                return A + s * t
            s_ref = _quad(lambda s: -math.log(np.linalg.norm(x - y(s))) / (2 * math.pi), 0, L) if \
                np.linalg.norm(x - (A + 0.5 * (B - A))) > 1e-12 else \
                2 * _quad(lambda s: -math.log(s) / (2 * math.pi), 0, L / 2)
            d_ref = _quad(lambda s: -np.dot(x - y(s), n) / (2 * math.pi * np.dot(x - y(s), x - y(s))), 0, L) \
                if abs(np.dot(x - A, n)) > 1e-12 else 0.0
            s_val = PO.panel_single(x[None, :], panel)[0, 0]
            d_val = PO.panel_double(x[None, :], panel)[0, 0]
            assert abs(s_val - s_ref) <= 1e-12 * max(1.0, abs(s_ref)), (s_val, s_ref)
            assert abs(d_val - d_ref) <= 1e-12, (d_val, d_ref)
    # the self term of a panel at its midpoint: (L / 2 pi) (1 - ln(L / 2))
    panel = np.array([[0.3, 0.4, 0.31, 0.405]])
    L = math.hypot(0.01, 0.005)
    assert abs(PO.panel_single(PO.panel_geometry(panel)[0], panel)[0, 0]
               - L / (2 * math.pi) * (1 - math.log(L / 2))) < 1e-15


@pytest.mark.parametrize("curve", [I.circle_curve(0.35), I.star_curve(0.3, 0.3, 5)])
def test_gauss_law_double_layer_of_one_is_one_half(curve):
    """On a closed polygon the exact double layer of u = 1 is 1/2 at every
    panel midpoint (the subtended angles of all panels add to pi)."""
    b = I.curve_panels(64, curve)
    _, D = PO.o2_matrices(b.panels)
    assert np.max(np.abs(D.sum(axis=1) - 0.5)) < 1e-12


def test_o2_converges_to_the_analytic_flux_on_the_circle():
    """Dirichlet u = x^2 - y^2 on the circle r = 0.35: the flat-panel BEM's flux
    error falls about 4x per halving of h, and so does the interior potential
    error of the representation formula."""
    errs, ierrs = [], []
    xi = np.array([[0.5, 0.5], [0.6, 0.45], [0.4, 0.62]])
    for n in (32, 64, 128):
        b = I.curve_panels(n, I.circle_curve(0.35))
        u, q = I.panel_data(b, I.field_x2y2)
        bc = np.zeros(b.nb, np.uint8)
        S, D = PO.o2_matrices(b.panels)
        x = np.linalg.solve(PO.system(S, D, bc), PO.rhs(S, D, bc, u, np.zeros_like(q)))
        errs.append(np.linalg.norm(x - q) / np.linalg.norm(q))
        ue, _ = I.field_x2y2(xi)
        ierrs.append(np.max(np.abs(PO.interior_potential(xi, b.panels, x, u) - ue)))
    assert errs[0] < 2e-3 and errs[2] < 1e-4
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3
    assert ierrs[2] < ierrs[0] / 8


@pytest.mark.parametrize("order", [2, 3])
def test_stencils_reproduce_polynomials(order):
    """Interpolation weights reproduce every polynomial x^a y^b with a, b <= p
    (and its gradient); the projected panel moments reproduce int phi ds and
    -int n . grad phi ds for polynomials of degree <= p."""
    rng = np.random.default_rng(order)
    n = 64
    h = 1.0 / n
    b = I.curve_panels(n, I.star_curve(0.3, 0.3, 5))
    m, L, t, nrm = PO.panel_geometry(b.panels)
    idx, W, G = PO.stencils(m, h, order)
    xk = (idx + 0.5) * h
    for a in range(order + 1):
        for c in range(order + 1):
            phi = xk[..., 0] ** a * xk[..., 1] ** c
            assert np.allclose(np.sum(W * phi, axis=1), m[:, 0] ** a * m[:, 1] ** c, rtol=0, atol=1e-13)
            gx = (a * m[:, 0] ** max(a - 1, 0) if a else 0 * m[:, 0]) * m[:, 1] ** c
            gy = m[:, 0] ** a * (c * m[:, 1] ** max(c - 1, 0) if c else 0 * m[:, 1])
            assert np.allclose(np.sum(G[..., 0] * phi, axis=1), gx, atol=1e-11)
            assert np.allclose(np.sum(G[..., 1] * phi, axis=1), gy, atol=1e-11)
    idx2, PS, PD = PO.projection_weights(b.panels, h, order)
    assert np.array_equal(idx, idx2)
    xk = (idx + 0.5) * h
    for j in rng.choice(b.nb, 6, replace=False):
        A, B = b.panels[j, 0:2], b.panels[j, 2:4]
        for a in range(order + 1):
            for c in range(order + 1 - a):
                def phi(p):
                    return p[0] ** a * p[1] ** c

                def dphi(p):
                    return np.array([a * p[0] ** max(a - 1, 0) * p[1] ** c if a else 0.0,
                                     c * p[0] ** a * p[1] ** max(c - 1, 0) if c else 0.0])
                ref = _quad(lambda s: phi(A + s * t[j]), 0, L[j])
                dref = -_quad(lambda s: float(np.dot(nrm[j], dphi(A + s * t[j]))), 0, L[j])
                got = float(np.sum(PS[j] * xk[j, :, 0] ** a * xk[j, :, 1] ** c))
                dgot = float(np.sum(PD[j] * xk[j, :, 0] ** a * xk[j, :, 1] ** c))
                assert abs(got - ref) <= 1e-13 + 1e-11 * abs(ref)
                assert abs(dgot - dref) <= 1e-11 + 1e-9 * abs(dref)


def test_accelerated_equals_o2_when_every_pair_is_near():
    b = I.curve_panels(32, I.star_curve(0.3, 0.3, 5))
    S, D = PO.o2_matrices(b.panels)
    Sa, Da = PO.accelerated_matrices(b.panels, b.h, 3, 10 ** 6)
    assert np.array_equal(Sa, S)
    assert np.max(np.abs(Da - D)) < 1e-13  # the row-sum term is 1/2 - (D 1)_i, zero by Gauss's law


def test_accelerated_error_falls_with_stencil_order_and_radius():
    """Flux error of the accelerated Dirichlet solve against O2's own solution
    (star, n = 128): smaller for a larger near radius and a higher order, and
    already below 1e-2 at order 2, R = 2; without the row-sum term it is
    several times larger."""
    b = I.curve_panels(128, I.star_curve(0.3, 0.3, 5))
    u, q = I.panel_data(b, I.field_x2y2)
    bc = np.zeros(b.nb, np.uint8)
    S, D = PO.o2_matrices(b.panels)
    xe = np.linalg.solve(PO.system(S, D, bc), PO.rhs(S, D, bc, u, np.zeros_like(q)))
    errs = {}
    for order, R in ((2, 2), (3, 3), (3, 5)):
        Sa, Da = PO.accelerated_matrices(b.panels, b.h, order, R)
        x = np.linalg.solve(PO.system(Sa, Da, bc), PO.rhs(Sa, Da, bc, u, np.zeros_like(q)))
        errs[(order, R)] = np.linalg.norm(x - xe) / np.linalg.norm(xe)
        if (order, R) == (3, 3):
            Dn = Da - np.diag(np.diag(Da) - np.diag(D))  # drop the row-sum term
            xn = np.linalg.solve(PO.system(Sa, Dn, bc), PO.rhs(Sa, Dn, bc, u, np.zeros_like(q)))
            assert np.linalg.norm(xn - xe) / np.linalg.norm(xe) > 3 * errs[(3, 3)]
    assert errs[(2, 2)] < 1e-2
    assert errs[(3, 3)] < errs[(2, 2)] and errs[(3, 5)] < errs[(3, 3)]


@pytest.mark.parametrize("curve", [I.circle_curve(0.35), I.star_curve(0.3, 0.3, 5)])
def test_curve_panels_close_the_curve_with_equal_arclength_and_outward_normals(curve):
    """The accuracy mode's input recipe: the panels form a closed polygon whose
    vertices lie on the curve at (nearly) equal arclength spacing, about h
    long, numbered counter-clockwise so that the normals point outward."""
    n = 256
    b = I.curve_panels(n, curve)
    P = b.panels
    assert np.array_equal(P[:, 2:4], np.roll(P[:, 0:2], -1, axis=0))  # closed, consecutive
    L = b.length
    assert abs(L.mean() * n - 1.0) < 0.05 and L.std() / L.mean() < 0.05
    # vertices on the curve
    pv, _ = curve(b.param)
    assert np.max(np.abs(pv - P[:, 0:2])) < 1e-12
    # outward: the normal points away from the centre for these star-shaped curves
    out = np.sum(b.normal * (b.mid - 0.5), axis=1)
    assert np.all(out > 0)
    # the polygon's length approaches the curve's (chords of length ~h)
    t = np.linspace(0, 2 * np.pi, 200001)
    _, dp = curve(t)
    length = np.trapezoid(np.hypot(dp[:, 0], dp[:, 1]), t)
    assert 0 < length - L.sum() < 1e-4 * length


@pytest.mark.parametrize("layer", ["single", "double", "system"])
def test_row_wise_accelerated_operator_equals_the_dense_one(layer):
    """The row-wise form (used on grids too large for dense matrices) agrees
    with the dense accelerated matrices on every row."""
    rng = np.random.default_rng(3)
    b = I.curve_panels(64, I.star_curve(0.3, 0.3, 5))
    x = rng.standard_normal(b.nb)
    bc = (rng.uniform(size=b.nb) < 0.5).astype(np.uint8)
    S, D = PO.accelerated_matrices(b.panels, b.h, 3, 3)
    M = {"single": S, "double": D, "system": PO.system(S, D, bc)}[layer]
    rows = np.arange(0, b.nb, 7)
    got = PO.accelerated_rows(b.panels, b.h, 3, 3, x, rows, layer, bc)
    ref = (M @ x)[rows]
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("h", [1.0 / 64, 1.0 / 4096])
def test_grid_kernel_self_term_is_the_cell_average(h):
    """The node-to-node kernel of the accelerated operator: the point value
    -ln(h |dk|) / (2 pi) off the diagonal, and on it the mean of -ln r / (2 pi)
    over the h-square centred at the node (adaptive quadrature)."""
    val = 4.0 * _dblquad(lambda y, x: -0.25 * math.log(x * x + y * y) / math.pi, 0.0, h / 2, 0.0, h / 2) / (h * h)
    dk = np.array([[0, 0], [1, 0], [3, -4], [-7, 2]])
    G = PO.grid_kernel(dk, h)
    assert abs(G[0] - val) < 1e-10 * abs(val)
    r = h * np.hypot(dk[1:, 0], dk[1:, 1])
    assert np.allclose(G[1:], -np.log(r) / (2 * math.pi), rtol=1e-15, atol=0)


def _dblquad(f, a, b, c, d):
    integrate = pytest.importorskip("scipy.integrate")
    return integrate.dblquad(f, a, b, c, d, epsabs=1e-15, epsrel=1e-13)[0]


@pytest.mark.parametrize("conditions", ["dirichlet", "mixed"])
def test_o2_solve_on_the_star_reaches_the_analytic_field(conditions):
    """u = e^x cos y on the star (its mean on the curve is not zero, so the
    double layer of the known data matters): the O2 solve of the
    boundary-condition split returns the analytic flux on Dirichlet panels and
    potential on Neumann panels (theta >= pi), with an error that falls about
    3x per halving of h (measured 8.7e-3 / 2.7e-3 Dirichlet, 5.8e-3 / 1.9e-3
    mixed at n = 64 / 128)."""
    errs = []
    for n in (64, 128):
        b = I.curve_panels(n, I.star_curve(0.3, 0.3, 5))
        u, q = I.panel_data(b, I.field_expcos)
        bc = np.zeros(b.nb, np.uint8) if conditions == "dirichlet" else (np.asarray(b.param) >= np.pi).astype(np.uint8)
        S, D = PO.o2_matrices(b.panels)
        x = np.linalg.solve(PO.system(S, D, bc), PO.rhs(S, D, bc, u, q))
        truth = np.where(bc == 0, q, u)
        errs.append(np.linalg.norm(x - truth) / np.linalg.norm(truth))
    assert errs[1] < 5e-3 and errs[1] < errs[0] / 2.5, errs
