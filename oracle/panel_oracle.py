"""Accuracy-mode oracle: flat-panel collocation BEM and its grid-accelerated
(precorrected-FFT) approximation, 2D Laplace, FP64 numpy.

TEST INFRASTRUCTURE ONLY: the tests and ``__graft_entry__.smoke()`` are the
only callers.  The product path never imports this module, and this module
imports nothing from the product package.

Why it exists.  The paper's operator (Section 4, Eq. 15-16) puts sources and
targets on grid nodes; on a curved boundary that discretisation does not
converge.  The accuracy mode keeps the paper's convolution on the grid (the
same spectra, the same FFT path) but moves the unknowns onto the boundary
itself, the way the precorrected-FFT method does (Phillips and White, IEEE
TCAD 16(10), 1997): sources are projected onto small stencils of grid nodes,
the grid convolution carries the far field, the potential is interpolated
back to the boundary, and near pairs are replaced by exact integrals.

Definitions (every function below follows them literally)
----------------------------------------------------------
Boundary: nb straight panels; panel j runs from A_j to B_j, length L_j, unit
tangent t_j = (B_j - A_j) / L_j, normal n_j = (t_j.y, -t_j.x) (outward for
counter-clockwise curves), collocation point m_j = (A_j + B_j) / 2.
Kernel U(r) = -ln r / (2 pi) (Section 3, the 2D Laplace fundamental
solution).  Operators with the paper's signs (Eq. 15: c u = S q + D u):
    (S q)_i = sum_j q_j  int_{panel j} U(|m_i - y|) ds_y
    (D u)_i = sum_j u_j  int_{panel j} -(m_i - y).n_j / (2 pi |m_i - y|^2) ds_y
(constant values per panel).  c = 1/2 at every collocation point (the
midpoint of a flat panel is a smooth boundary point).

Stencils.  Grid node k = (kx, ky) sits at ((kx + 1/2) h, (ky + 1/2) h) as in
the paper's grid (Section 4).  A point m has grid coordinates
u = m / h - 1/2; its stencil of order p has (p + 1)^2 nodes: per axis the
nodes a - 1 .. a + p - 1 around the anchor a = floor(u + 1/2) (p = 2) or
floor(u) (p = 3), with tensor-product Lagrange weights L_k(m).

O2 (the exact-geometry reference).  Every entry is the exact panel integral
(closed forms, panel_single / panel_double): the flat-panel collocation BEM,
which converges like h^2 on smooth curves.

Accelerated operator (what the GPU accuracy mode computes).  A pair (i, j)
is *near* when the anchors of m_i and m_j differ by at most R along both
axes; near entries are exact (as O2).  Far entries go through the grid:
    S_ij = sum_k sum_l L_k(m_i) U_grid(x_k - x_l) PS_lj
    D_ij = sum_k sum_l L_k(m_i) U_grid(x_k - x_l) PD_lj
with the panel projected onto the stencil of its midpoint by its moments,
    PS_lj = int_{panel j} L_l(y) ds_y,   PD_lj = -int_{panel j} n_j . grad L_l(y) ds_y,
(Gauss-Legendre with p + 1 points along the panel: exact, the integrands are
polynomials of degree <= 2p in the arclength), so that the grid charges
carry every moment of the panel up to the stencil's order (the
precorrected-FFT projection), and the potential interpolated at m_i from the
stencil of m_i.  U_grid(x_k - x_l) = U(|x_k - x_l|) for k != l and the cell
average -(ln h + L2) / (2 pi) for k = l (the paper-form table; with R >= p
the stencils of a far pair share no node, so that value never enters a far
entry).  Finally the double layer gets a diagonal term so that its rows sum to
1/2: on a closed curve Gauss's law gives (D 1)_i = 1/2 exactly at every
collocation point (c = 1/2 for u = 1, q = 0), O2 satisfies it to rounding,
and restoring it in the accelerated operator turns its far-field error into
one acting on u_j - u_i, which vanishes for smooth data as h -> 0 (without
it the first-kind Dirichlet solve amplifies that error in proportion to n).
"""
from __future__ import annotations

import math

import numpy as np

L2_CONST = math.pi / 4 - 1.5 - 0.5 * math.log(2.0)


# ------------------------------------------------------------------ geometry

def panel_geometry(panels):
    """panels (nb, 4): A.x, A.y, B.x, B.y -> midpoints, lengths, tangents, normals."""
    P = np.asarray(panels, dtype=np.float64)
    A, B = P[:, 0:2], P[:, 2:4]
    d = B - A
    L = np.hypot(d[:, 0], d[:, 1])
    t = d / L[:, None]
    nrm = np.stack([t[:, 1], -t[:, 0]], axis=1)
    return 0.5 * (A + B), L, t, nrm


def _local(x, A, t, nrm):
    """Coordinates of targets x (m, 2) in every panel's frame: s0 along the
    tangent from A, eta along the normal."""
    dx = x[:, None, :] - A[None, :, :]
    s0 = dx[..., 0] * t[None, :, 0] + dx[..., 1] * t[None, :, 1]
    eta = dx[..., 0] * nrm[None, :, 0] + dx[..., 1] * nrm[None, :, 1]
    return s0, eta


def panel_single(x, panels):
    """int_{panel j} U(|x_i - y|) ds_y for targets x (m, 2): closed form of
    int ln sqrt(u^2 + eta^2) du = u ln sqrt(u^2 + eta^2) - u + eta atan(u / eta)."""
    A = np.asarray(panels, np.float64)[:, 0:2]
    _, L, t, nrm = panel_geometry(panels)
    s0, eta = _local(np.asarray(x, np.float64), A, t, nrm)
    tiny = 1e-11 * L[None, :]  # on the panel's line (rounding of the frame)
    eta = np.where(np.abs(eta) < tiny, 0.0, eta)

    def F(u):
        r2 = u * u + eta * eta
        with np.errstate(divide="ignore", invalid="ignore"):
            lg = np.where(r2 > 0, 0.5 * u * np.log(np.where(r2 > 0, r2, 1.0)), 0.0)
            at = np.where(eta != 0, eta * np.arctan(u / np.where(eta != 0, eta, 1.0)), 0.0)
        return lg - u + at

    return -(F(L[None, :] - s0) - F(-s0)) / (2 * math.pi)


def panel_double(x, panels):
    """int_{panel j} -(x_i - y).n_j / (2 pi |x_i - y|^2) ds_y (the paper's
    double-layer sign): -(1/2 pi) [atan((L - s0)/eta) - atan(-s0/eta)], and 0
    on the panel's own line (principal value)."""
    A = np.asarray(panels, np.float64)[:, 0:2]
    _, L, t, nrm = panel_geometry(panels)
    s0, eta = _local(np.asarray(x, np.float64), A, t, nrm)
    tiny = 1e-11 * L[None, :]  # on the panel's line (rounding of the frame)
    on_line = np.abs(eta) < tiny
    e = np.where(on_line, 1.0, eta)
    val = -(np.arctan((L[None, :] - s0) / e) - np.arctan(-s0 / e)) / (2 * math.pi)
    return np.where(on_line, 0.0, val)


# ------------------------------------------------------------------ stencils

def _offsets(order):
    if order == 2:
        return np.array([-1, 0, 1])
    if order == 3:
        return np.array([-1, 0, 1, 2])
    raise ValueError("stencil order must be 2 or 3")


def anchors(m, h, order):
    """Anchor node per axis of each point (see the module docstring)."""
    u = np.asarray(m, np.float64) / h - 0.5
    return (np.floor(u + 0.5) if order == 2 else np.floor(u)).astype(np.int64)


def lagrange_1d(xi, order):
    """Weights and derivatives (per unit of the node spacing) of the
    Lagrange polynomials on the order's offsets, at local coordinates xi."""
    o = _offsets(order)
    xi = np.asarray(xi, np.float64)
    W = np.ones(xi.shape + (o.size,))
    dW = np.zeros(xi.shape + (o.size,))
    for a in range(o.size):
        den = 1.0
        for b in range(o.size):
            if b != a:
                den *= o[a] - o[b]
        num = np.ones_like(xi)
        for b in range(o.size):
            if b != a:
                num = num * (xi - o[b])
        W[..., a] = num / den
        # derivative: sum over the left-out factor
        d = np.zeros_like(xi)
        for c in range(o.size):
            if c == a:
                continue
            term = np.ones_like(xi)
            for b in range(o.size):
                if b != a and b != c:
                    term = term * (xi - o[b])
            d = d + term
        dW[..., a] = d / den
    return W, dW


def stencils(m, h, order):
    """For points m (nb, 2): node indices (nb, S, 2), weights L (nb, S) and
    physical gradients grad L (nb, S, 2), S = (order + 1)^2, node k = (kx, ky)
    enumerated kx fastest."""
    m = np.asarray(m, np.float64)
    a = anchors(m, h, order)
    u = m / h - 0.5
    o = _offsets(order)
    Wx, dWx = lagrange_1d(u[:, 0] - a[:, 0], order)
    Wy, dWy = lagrange_1d(u[:, 1] - a[:, 1], order)
    nb, q = m.shape[0], o.size
    idx = np.empty((nb, q * q, 2), np.int64)
    L = np.empty((nb, q * q))
    G = np.empty((nb, q * q, 2))
    for by in range(q):
        for bx in range(q):
            s = by * q + bx
            idx[:, s, 0] = a[:, 0] + o[bx]
            idx[:, s, 1] = a[:, 1] + o[by]
            L[:, s] = Wx[:, bx] * Wy[:, by]
            G[:, s, 0] = dWx[:, bx] * Wy[:, by] / h
            G[:, s, 1] = Wx[:, bx] * dWy[:, by] / h
    return idx, L, G


def near_mask(m, h, order, R):
    a = anchors(m, h, order)
    d = np.abs(a[:, None, :] - a[None, :, :]).max(axis=2)
    return d <= R


# ------------------------------------------------------------------ operators

def o2_matrices(panels):
    """Dense O2 single- and double-layer matrices (nb, nb): every entry the
    exact panel integral at the collocation points."""
    m, _, _, _ = panel_geometry(panels)
    return panel_single(m, panels), panel_double(m, panels)


def grid_kernel(dk, h):
    """U_grid between nodes at integer offsets dk (..., 2)."""
    r = h * np.hypot(dk[..., 0], dk[..., 1])
    with np.errstate(divide="ignore"):
        v = -np.log(np.where(r > 0, r, 1.0)) / (2 * math.pi)
    return np.where(r > 0, v, -(math.log(h) + L2_CONST) / (2 * math.pi))


def projection_weights(panels, h, order):
    """Stencil nodes of each panel's midpoint (nb, S, 2) and the panel's
    moments on them: PS (nb, S) = int L_l ds, PD (nb, S) = -int n . grad L_l ds
    (Gauss-Legendre, order + 1 points)."""
    P = np.asarray(panels, np.float64)
    m, L, t, nrm = panel_geometry(P)
    idx, _, _ = stencils(m, h, order)
    a = anchors(m, h, order)
    o = _offsets(order)
    q = o.size
    gx, gw = np.polynomial.legendre.leggauss(order + 1)
    PS = np.zeros((m.shape[0], q * q))
    PD = np.zeros((m.shape[0], q * q))
    for g in range(gx.size):
        y = P[:, 0:2] + (0.5 * (gx[g] + 1.0) * L)[:, None] * t  # Gauss point on [A, B]
        u = y / h - 0.5
        Wx, dWx = lagrange_1d(u[:, 0] - a[:, 0], order)
        Wy, dWy = lagrange_1d(u[:, 1] - a[:, 1], order)
        ww = 0.5 * gw[g] * L
        for by in range(q):
            for bx in range(q):
                sidx = by * q + bx
                PS[:, sidx] += ww * Wx[:, bx] * Wy[:, by]
                ng = (dWx[:, bx] * Wy[:, by] * nrm[:, 0] + Wx[:, bx] * dWy[:, by] * nrm[:, 1]) / h
                PD[:, sidx] -= ww * ng
    return idx, PS, PD


def accelerated_parts(panels, h, order=3, R=3):
    """The pieces of the accelerated operator: interpolation I (nb, nodes),
    grid kernel G (nodes, nodes), projections PS, PD (nodes, nb), the near
    mask and the exact matrices (module docstring)."""
    if R < order:
        raise ValueError("R must be at least the stencil order")
    m, _, _, _ = panel_geometry(panels)
    idx, PSw, PDw = projection_weights(panels, h, order)
    _, W, _ = stencils(m, h, order)
    nb, S = W.shape
    keys = idx[..., 1] * (1 << 32) + idx[..., 0]
    nodes, inv = np.unique(keys.ravel(), return_inverse=True)
    inv = inv.reshape(nb, S)
    nk = np.stack([nodes % (1 << 32), nodes // (1 << 32)], axis=1)
    I = np.zeros((nb, nodes.size))        # interpolation: target i from node k
    PS = np.zeros((nodes.size, nb))       # single-layer projection
    PD = np.zeros((nodes.size, nb))       # dipole projection
    rows = np.repeat(np.arange(nb), S)
    np.add.at(I, (rows, inv.ravel()), W.ravel())
    np.add.at(PS, (inv.ravel(), rows), PSw.ravel())
    np.add.at(PD, (inv.ravel(), rows), PDw.ravel())
    Gn = grid_kernel(nk[:, None, :] - nk[None, :, :], h)
    near = near_mask(m, h, order, R)
    S_ex, D_ex = o2_matrices(panels)
    return I, Gn, PS, PD, near, S_ex, D_ex


def accelerated_matrices(panels, h, order=3, R=3):
    """Dense single- and double-layer matrices of the grid-accelerated
    operator: near entries exact (as O2), far entries through the projected
    moments, the grid kernel and the interpolation, and the double layer's
    row-sum term (module docstring)."""
    I, Gn, PS, PD, near, S_ex, D_ex = accelerated_parts(panels, h, order, R)
    S_acc = np.where(near, S_ex, I @ Gn @ PS)
    D_acc = np.where(near, D_ex, I @ Gn @ PD)
    D_acc = D_acc + np.diag(0.5 - D_acc.sum(axis=1))
    return S_acc, D_acc


def system(S, D, bc, c=0.5):
    """BC split (Eq. 4 with c = 1/2): Dirichlet panels carry the unknown flux
    (column of S), Neumann panels the unknown potential (column of D minus
    c on the diagonal).  Returns A; the right-hand side is rhs()."""
    bc = np.asarray(bc)
    A = np.where(bc[None, :] == 0, S, D)
    A = A - c * np.diag((bc == 1).astype(np.float64))
    return A


def rhs(S, D, bc, u_known, q_known, c=0.5):
    """b = c u_D - D u_D - S q_N (known data moved to the right)."""
    bc = np.asarray(bc)
    uD = np.where(bc == 0, u_known, 0.0)
    qN = np.where(bc == 1, q_known, 0.0)
    return c * uD - D @ uD - S @ qN


def interior_potential(x, panels, q, u):
    """Representation formula at interior points x (m, 2): u(x) = S q + D u
    (c = 1 inside), panel integrals evaluated exactly."""
    return panel_single(x, panels) @ q + panel_double(x, panels) @ u


def accelerated_rows(panels, h, order, R, x, rows, layer, bc=None, c=0.5):
    """Rows `rows` of the accelerated operator applied to x, for grids too large
    for the dense matrices: (A x)_i = sum_s L_s(m_i) sum_l U_grid(x_s - x_l) rho_l
    (rho = the projection of x, all panels) plus, for the near pairs, the exact
    integral minus the grid-mediated value of the pair, plus the double layer's
    row-sum term (module docstring).  layer: "single", "double" or "system"
    (with bc: 0 = the column carries the flux through S, 1 = the potential
    through D, minus c on the diagonal)."""
    P = np.asarray(panels, np.float64)
    x = np.asarray(x, np.float64)
    rows = np.asarray(rows)
    m, _, _, _ = panel_geometry(P)
    idx, PSw, PDw = projection_weights(P, h, order)
    _, W, _ = stencils(m, h, order)
    nb, S = W.shape
    keys = idx[..., 1] * (1 << 32) + idx[..., 0]
    nodes, inv = np.unique(keys.ravel(), return_inverse=True)
    inv = inv.reshape(nb, S)
    nk = np.stack([nodes % (1 << 32), nodes // (1 << 32)], axis=1)
    bc = np.zeros(nb, np.uint8) if bc is None else np.asarray(bc)
    if layer == "single":
        dip = np.zeros(nb, bool)
    elif layer == "double":
        dip = np.ones(nb, bool)
    else:
        dip = bc == 1
    Pw = np.where(dip[:, None], PDw, PSw)
    rho = np.zeros(nodes.size)
    np.add.at(rho, inv.ravel(), (Pw * x[:, None]).ravel())
    rho1 = np.zeros(nodes.size)  # the double layer of x = 1, for its row-sum term
    np.add.at(rho1, inv.ravel(), PDw.ravel())
    a = anchors(m, h, order)
    out = np.zeros(rows.size)
    for r, i in enumerate(rows):
        Gi = grid_kernel(nk[inv[i]][:, None, :] - nk[None, :, :], h)  # (S, nodes)
        far = W[i] @ (Gi @ rho)
        near = np.nonzero(np.abs(a - a[i]).max(axis=1) <= R)[0]
        ex_s = panel_single(m[i:i + 1], P[near])[0]
        ex_d = panel_double(m[i:i + 1], P[near])[0]
        # grid-mediated value of each near pair: sum_s W_is sum_t U(x_s - x_t) P_jt
        cols = inv[near]  # (k, S) node indices of the sources' stencils
        Gn = Gi[:, cols]  # (S, k, S)
        grid_s = np.einsum("s,skt,kt->k", W[i], Gn, PSw[near])
        grid_d = np.einsum("s,skt,kt->k", W[i], Gn, PDw[near])
        corr = np.where(dip[near], ex_d - grid_d, ex_s - grid_s)
        val = far + corr @ x[near]
        if layer == "double" or (layer == "system" and bc[i] == 1):
            delta = 0.5 - (W[i] @ (Gi @ rho1) + (ex_d - grid_d).sum())
            val += delta * x[i] - (c * x[i] if layer == "system" else 0.0)
        out[r] = val
    return out
