"""Planted mistakes in a temporary copy of the learned-guess network oracle
(CPU only): each rewrites one expression of ``oracle/net_oracle.py`` and must
fail at least one pin of ``test_net_oracle_pins.py``.  The committed oracle is
never modified."""
import importlib.util
import os

import pytest

pytest.importorskip("scipy")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NET_ORACLE = os.path.join(ROOT, "oracle", "net_oracle.py")
PINS_PATH = os.path.join(ROOT, "tests", "test_net_oracle_pins.py")


def _load(name, path):
    spec = importlib.util.spec_from_file_location(name, path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _pins_against(oracle_module):
    pins = _load(f"net_pins_{id(oracle_module)}", PINS_PATH)
    pins.N = oracle_module
    return [pins.test_bf16_round_to_nearest_even, pins.test_circular_conv_matches_scipy_correlate,
            lambda: pins.test_gradient_matches_finite_differences([1, 2, 4]), pins.test_bf16_rounding_points]


def mutant(tmp_path, old, new):
    src = open(NET_ORACLE).read()
    assert src.count(old) == 1, f"mutation site not unique: {old!r}"
    path = tmp_path / "net_oracle_mutant.py"
    path.write_text(src.replace(old, new))
    return _load(f"net_oracle_mutant_{abs(hash((old, new)))}", str(path))


MUTATIONS = [
    ("BF16 ties away from even", "u = (u + 0x7FFF + lsb) & 0xFFFF0000", "u = (u + 0x8000) & 0xFFFF0000"),
    ("BF16 truncation", "u = (u + 0x7FFF + lsb) & 0xFFFF0000", "u = u & 0xFFFF0000"),
    ("layer input not rounded", "x = rnd(np.maximum(y, 0.0))", "x = np.maximum(y, 0.0)"),
    ("weights not rounded", "Wr = rnd(W)", "Wr = W"),
    ("convolution instead of correlation", "shift = (k - K // 2) * d\n", "shift = (K // 2 - k) * d\n"),
    ("bias dropped", "acc = np.tile(b, (L, 1))", "acc = np.zeros((L, co))"),
    ("ReLU mask dropped in the backward pass", "g = g * (yl > 0)", "g = g"),
    ("loss gradient factor", "g = (2.0 * e / T)[:, None]", "g = (e / T)[:, None]"),
    ("input gradient scattered without the shift", "np.add.at(gx, s0 + idx, g[s0:s1] @ Wr[:, :, k])",
     "np.add.at(gx, s0 + np.arange(L), g[s0:s1] @ Wr[:, :, k])"),
]


def test_unmutated_copy_passes_the_pins(tmp_path):
    o = mutant(tmp_path, "from __future__ import annotations", "from __future__ import annotations  # copy")
    for pin in _pins_against(o):
        pin()


@pytest.mark.parametrize("what,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, what, old, new):
    o = mutant(tmp_path, old, new)
    failed = False
    for pin in _pins_against(o):
        try:
            pin()
        except AssertionError:
            failed = True
            break
    assert failed, f"no pin sees the planted mistake: {what}"
