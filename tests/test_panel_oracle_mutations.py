"""Planted mistakes in a temporary copy of the accuracy-mode oracle (CPU only).

Each case rewrites one expression of a copy of ``oracle/panel_oracle.py``,
loads it as a module of its own and runs the pins of
``test_panel_oracle_pins.py`` against it (every pin, so that the case passes
when any one of them fails).  The committed oracle is never modified.
"""
import importlib.util
import os

import pytest

pytest.importorskip("scipy")
from paper_1809_00845_gb300 import inputs as I  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PANEL_ORACLE = os.path.join(ROOT, "oracle", "panel_oracle.py")
PINS_PATH = os.path.join(ROOT, "tests", "test_panel_oracle_pins.py")


def _load(name, path):
    spec = importlib.util.spec_from_file_location(name, path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _pins_against(oracle_module):
    """The pin functions, bound to the given oracle module (their global PO)."""
    pins = _load(f"panel_pins_{id(oracle_module)}", PINS_PATH)
    pins.PO = oracle_module
    return [
        pins.test_panel_integrals_match_adaptive_quadrature,
        lambda: pins.test_gauss_law_double_layer_of_one_is_one_half(I.star_curve(0.3, 0.3, 5)),
        pins.test_o2_converges_to_the_analytic_flux_on_the_circle,
        lambda: pins.test_o2_solve_on_the_star_reaches_the_analytic_field("dirichlet"),
        lambda: pins.test_o2_solve_on_the_star_reaches_the_analytic_field("mixed"),
        lambda: pins.test_stencils_reproduce_polynomials(3),
        lambda: pins.test_stencils_reproduce_polynomials(2),
        pins.test_accelerated_equals_o2_when_every_pair_is_near,
        pins.test_accelerated_error_falls_with_stencil_order_and_radius,
        lambda: pins.test_grid_kernel_self_term_is_the_cell_average(1.0 / 64),
        lambda: pins.test_row_wise_accelerated_operator_equals_the_dense_one("single"),
        lambda: pins.test_row_wise_accelerated_operator_equals_the_dense_one("double"),
        lambda: pins.test_row_wise_accelerated_operator_equals_the_dense_one("system"),
    ]


def mutant(tmp_path, old, new):
    src = open(PANEL_ORACLE).read()
    assert src.count(old) == 1, f"mutation site not unique: {old!r}"
    path = tmp_path / "panel_oracle_mutant.py"
    path.write_text(src.replace(old, new))
    return _load(f"panel_oracle_mutant_{abs(hash((old, new)))}", str(path))


MUTATIONS = [
    ("single-layer atan term sign", "return lg - u + at", "return lg - u - at"),
    ("single-layer linear term dropped", "return lg - u + at", "return lg + at"),
    ("double-layer sign", "val = -(np.arctan((L[None, :] - s0) / e) - np.arctan(-s0 / e)) / (2 * math.pi)",
     "val = (np.arctan((L[None, :] - s0) / e) - np.arctan(-s0 / e)) / (2 * math.pi)"),
    ("normal points inward", "nrm = np.stack([t[:, 1], -t[:, 0]], axis=1)", "nrm = np.stack([-t[:, 1], t[:, 0]], axis=1)"),
    ("Lagrange derivative sign", "d = d + term", "d = d - term"),
    ("Lagrange denominator dropped", "W[..., a] = num / den", "W[..., a] = num"),
    ("dipole moment sign", "PD[:, sidx] -= ww * ng", "PD[:, sidx] += ww * ng"),
    ("Gauss weight factor", "ww = 0.5 * gw[g] * L", "ww = gw[g] * L"),
    ("Gauss point map", "y = P[:, 0:2] + (0.5 * (gx[g] + 1.0) * L)[:, None] * t",
     "y = P[:, 0:2] + (0.5 * gx[g] * L)[:, None] * t"),
    ("row-sum term dropped", "D_acc = D_acc + np.diag(0.5 - D_acc.sum(axis=1))", "D_acc = D_acc"),
    ("row-sum term sign", "D_acc = D_acc + np.diag(0.5 - D_acc.sum(axis=1))",
     "D_acc = D_acc + np.diag(D_acc.sum(axis=1) - 0.5)"),
    ("grid kernel self-term sign", "return np.where(r > 0, v, -(math.log(h) + L2_CONST) / (2 * math.pi))",
     "return np.where(r > 0, v, (math.log(h) + L2_CONST) / (2 * math.pi))"),
    ("grid kernel cell-average constant", "L2_CONST = math.pi / 4 - 1.5 - 0.5 * math.log(2.0)",
     "L2_CONST = math.pi / 4 - 1.5 - math.log(2.0)"),
    ("near and far swapped", "S_acc = np.where(near, S_ex, I @ Gn @ PS)", "S_acc = np.where(near, I @ Gn @ PS, S_ex)"),
    ("system diagonal sign", "A = A - c * np.diag((bc == 1).astype(np.float64))",
     "A = A + c * np.diag((bc == 1).astype(np.float64))"),
    ("right-hand side double-layer sign", "return c * uD - D @ uD - S @ qN", "return c * uD + D @ uD - S @ qN"),
    ("row-wise row-sum term sign", "delta = 0.5 - (W[i] @ (Gi @ rho1) + (ex_d - grid_d).sum())",
     "delta = (W[i] @ (Gi @ rho1) + (ex_d - grid_d).sum()) - 0.5"),
    ("row-wise near correction sign", "val = far + corr @ x[near]", "val = far - corr @ x[near]"),
]


def test_unmutated_copy_passes_the_pins(tmp_path):
    o = mutant(tmp_path, "# ------------------------------------------------------------------ geometry", "# geometry")
    for pin in _pins_against(o):
        pin()


@pytest.mark.parametrize("what,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, what, old, new):
    o = mutant(tmp_path, old, new)
    failed = []
    for pin in _pins_against(o):
        try:
            pin()
        except (AssertionError, ValueError, FloatingPointError, IndexError, ZeroDivisionError):
            failed.append(pin)
            break
    assert failed, f"no pin sees the planted mistake: {what}"
