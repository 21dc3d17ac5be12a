"""Planted mistakes in a temporary copy of the oracle (CPU only).

Each case rewrites one expression of a copy of ``oracle/bem_oracle.c`` (a
wrong sign, prefactor, power or constant, a dropped term, a transposed or
reversed offset, a dropped weight; compiled with gcc into a library of its
own) or of ``oracle/oracle.py`` (the boundary-condition split), and runs the
pins of ``test_oracle_pins.py`` against it: at least one of them must fail.
The committed oracle is never modified; the pins are shown to see the
mistakes they are there to see.
"""
import importlib.util
import os
import shutil

import pytest

pytest.importorskip("scipy")
from paper_1809_00845_gb300 import inputs as I  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_PY = os.path.join(ROOT, "oracle", "oracle.py")
ORACLE_C = os.path.join(ROOT, "oracle", "bem_oracle.c")


def _load_by_path(name, path):
    spec = importlib.util.spec_from_file_location(name, path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


PINS = _load_by_path("oracle_pins_for_mutants", os.path.join(ROOT, "tests", "test_oracle_pins.py"))


def mutant_oracle(tmp_path, old, new):
    """A fresh oracle module whose C source has `old` replaced by `new`."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = open(ORACLE_C).read()
    assert src.count(old) == 1, f"mutation site not unique: {old!r}"
    cdir = tmp_path / "oracle"
    cdir.mkdir()
    (cdir / "bem_oracle.c").write_text(src.replace(old, new))
    mod = _load_by_path(f"oracle_mutant_{abs(hash((old, new)))}", ORACLE_PY)
    mod._SRC = str(cdir / "bem_oracle.c")
    mod._BUILD = str(cdir / "_build")
    mod._LIB_PATH = str(cdir / "_build" / "libbem_oracle.so")
    mod._lib = None
    return mod


def python_mutant(tmp_path, old, new):
    """A fresh oracle module whose Python source has `old` replaced by `new`
    (the compiled kernels unchanged)."""
    src = open(ORACLE_PY).read()
    assert src.count(old) == 1, f"mutation site not unique: {old!r}"
    path = tmp_path / "oracle_py_mutant.py"
    path.write_text(src.replace(old, new))
    mod = _load_by_path(f"oracle_py_mutant_{abs(hash((old, new)))}", str(path))
    here = os.path.dirname(ORACLE_PY)
    mod._SRC = ORACLE_C
    mod._BUILD = os.path.join(here, "_build")
    mod._LIB_PATH = os.path.join(here, "_build", "libbem_oracle.so")
    mod._lib = None
    return mod


# pins (functions of the oracle module) that each mutation must break
green2d = lambda o: PINS.test_green_identity_2d(o, I.field_x2y2)  # noqa: E731
green3d = lambda o: PINS.test_green_identity_3d(o)  # noqa: E731
somigliana = lambda o: PINS.test_somigliana_kelvin(o, "general")  # noqa: E731
L2_pin = lambda o: PINS.test_L2_closed_form_matches_quadrature(o)  # noqa: E731
C3_pin = lambda o: PINS.test_C3_closed_form_matches_quadrature(o)  # noqa: E731
cell2d = lambda o: PINS.test_2d_singular_cell_is_cell_average(o, 1.0 / 128)  # noqa: E731
cell3d = lambda o: PINS.test_3d_singular_cell_is_cell_average(o, 1.0 / 16)  # noqa: E731
cell_kelvin = lambda o: PINS.test_kelvin_singular_cell_is_cell_average(o)  # noqa: E731
plane_D = lambda o: PINS.test_full_plane_is_plain_convolution(o, 1)  # noqa: E731
plane_S = lambda o: PINS.test_full_plane_is_plain_convolution(o, 0)  # noqa: E731
const2d = lambda o: PINS.test_discrete_double_layer_of_a_constant(o, "laplace2d")  # noqa: E731
const3d = lambda o: PINS.test_discrete_double_layer_of_a_constant(o, "laplace3d")  # noqa: E731
const_kelvin = lambda o: PINS.test_discrete_double_layer_of_a_constant(o, "kelvin3d")  # noqa: E731


def split_pins(o):
    for kernel in ("laplace2d", "kelvin3d"):
        PINS.test_split_system_is_the_unsplit_equation(o, kernel)


MUTATIONS = [
    # 2D Laplace (Eq. 15)
    ("2d double-layer sign", "return -da / (2.0 * BO_PI * r2);", "return da / (2.0 * BO_PI * r2);", green2d),
    ("2d single-layer prefactor", "return -0.5 * log(r2) / (2.0 * BO_PI);", "return -0.5 * log(r2) / (4.0 * BO_PI);",
     green2d),
    ("2d double-layer power", "return -da / (2.0 * BO_PI * r2);", "return -da / (2.0 * BO_PI * sqrt(r2));", green2d),
    ("L2 constant", "return BO_PI / 4.0 - 1.5 - 0.5 * log(2.0);", "return BO_PI / 4.0 - 1.5 - log(2.0);", L2_pin),
    ("2d self-term sign", "if (r2 == 0.0) return -(log(h) + bo_L2()) / (2.0 * BO_PI);",
     "if (r2 == 0.0) return (log(h) + bo_L2()) / (2.0 * BO_PI);", cell2d),
    # 3D Laplace
    ("3d single-layer prefactor", "return 1.0 / (4.0 * BO_PI * sqrt(r2));", "return 1.0 / (2.0 * BO_PI * sqrt(r2));",
     green3d),
    ("3d double-layer power", "return -d[a] / (4.0 * BO_PI * r2 * r);", "return -d[a] / (4.0 * BO_PI * r2);", green3d),
    ("C3 constant", "3.0 * log(2.0 + sqrt(3.0)) - BO_PI / 2.0", "3.0 * log(2.0 + sqrt(3.0)) - BO_PI / 3.0", C3_pin),
    ("3d self-term h power", "if (r2 == 0.0) return bo_C3() / (4.0 * BO_PI * h);",
     "if (r2 == 0.0) return bo_C3() / (4.0 * BO_PI * h * h);", cell3d),
    # Kelvin (Eq. 7, Eq. 8)
    ("Kelvin U Poisson factor", "(3.0 - 4.0 * nu) / r", "(3.0 - 2.0 * nu) / r", somigliana),
    ("Kelvin U prefactor", "double pref = 1.0 / (16.0 * BO_PI * mu * (1.0 - nu));",
     "double pref = 1.0 / (8.0 * BO_PI * mu * (1.0 - nu));", somigliana),
    ("Kelvin T antisymmetric term dropped", " - c * (rd[a] * n[b] - rd[b] * n[a]);", ";", somigliana),
    ("Kelvin T antisymmetric term transposed", "(rd[a] * n[b] - rd[b] * n[a])", "(rd[b] * n[a] - rd[a] * n[b])",
     somigliana),
    ("Kelvin T direction cosines reversed", "double rd[3] = {-d[0] / r, -d[1] / r, -d[2] / r};",
     "double rd[3] = {d[0] / r, d[1] / r, d[2] / r};", somigliana),
    ("Kelvin self term", "(3.0 - 4.0 * nu + 1.0 / 3.0)", "(3.0 - 4.0 * nu)", cell_kelvin),
    # assembly of the discrete operator (bo_block)
    ("offset reversed (source minus target)", "d[a] = (double)(ci[a] - cj[a]) * h;",
     "d[a] = (double)(cj[a] - ci[a]) * h;", plane_D),
    ("weight dropped from the 2d single layer", "blk[0] = bo_lap2d_U(d[0], d[1], h) * wj;",
     "blk[0] = bo_lap2d_U(d[0], d[1], h);", plane_S),
    ("normal components swapped in the 2d double layer",
     "bo_lap2d_Q(0, d[0], d[1]) * nj[0] + bo_lap2d_Q(1, d[0], d[1]) * nj[1]) * wj;",
     "bo_lap2d_Q(0, d[0], d[1]) * nj[1] + bo_lap2d_Q(1, d[0], d[1]) * nj[0]) * wj;", plane_D),
    ("offset reversed, seen by the constant-density invariant", "d[a] = (double)(ci[a] - cj[a]) * h;",
     "d[a] = (double)(cj[a] - ci[a]) * h;", const2d),
    ("weight dropped from the 3d double layer", "               wj;", "               1.0;", const3d),
    ("normal components permuted in the 3d double layer",
     "bo_lap3d_Q(0, d[0], d[1], d[2]) * nj[0] + bo_lap3d_Q(1, d[0], d[1], d[2]) * nj[1] +",
     "bo_lap3d_Q(0, d[0], d[1], d[2]) * nj[1] + bo_lap3d_Q(1, d[0], d[1], d[2]) * nj[0] +", const3d),
    ("weight dropped from the Kelvin blocks", "for (int k = 0; k < 9; ++k) blk[k] = K[k] * wj;",
     "for (int k = 0; k < 9; ++k) blk[k] = K[k];", const_kelvin),
]


PY_MUTATIONS = [
    ("Navier double-layer sign", "return -1.0 if _kernel_id(kernel) == KELVIN_3D else 1.0", "return 1.0"),
    ("split diagonal sign", "A = K1 * mD[None, :] + K2 * mN[None, :] - np.diag(c * mN)",
     "A = K1 * mD[None, :] + K2 * mN[None, :] + np.diag(c * mN)"),
    ("split masks swapped", "A = K1 * mD[None, :] + K2 * mN[None, :] - np.diag(c * mN)",
     "A = K1 * mN[None, :] + K2 * mD[None, :] - np.diag(c * mN)"),
    ("split right-hand side sign", "b = c * u * mD - K2 @ (u * mD) - K1 @ (q * mN)",
     "b = c * u * mD + K2 @ (u * mD) - K1 @ (q * mN)"),
    ("matrix-free split diagonal sign", "return y1 + double_sign(k) * y2 - c * (x * mN)[sl]",
     "return y1 + double_sign(k) * y2 + c * (x * mN)[sl]"),
    ("matrix-free right-hand side sign", "return c * u * mD - double_sign(k) * k2u - k1q",
     "return c * u * mD + double_sign(k) * k2u - k1q"),
]


def test_unmutated_copy_passes_the_pins(tmp_path):
    """The harness itself: a copy with a no-op rewrite passes every pin used below."""
    o = mutant_oracle(tmp_path, "/* ---------------------------------------------------------------- kernels -- */",
                      "/* kernels */")
    for pin in (green2d, green3d, somigliana, L2_pin, C3_pin, cell2d, cell3d, cell_kelvin, plane_D, plane_S,
                const2d, const3d, const_kelvin, split_pins):
        pin(o)
    split_pins(python_mutant(tmp_path, "_lock = threading.Lock()", "_lock = threading.Lock()  # copy"))


@pytest.mark.parametrize("what,old,new,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, what, old, new, pin):
    o = mutant_oracle(tmp_path, old, new)
    with pytest.raises(AssertionError):
        pin(o)


@pytest.mark.parametrize("what,old,new", PY_MUTATIONS, ids=[m[0] for m in PY_MUTATIONS])
def test_planted_mistake_in_the_split_fails_a_pin(tmp_path, what, old, new):
    o = python_mutant(tmp_path, old, new)
    with pytest.raises(AssertionError):
        split_pins(o)
