"""Stored expected values (tests/golden/, written by tests/golden/make_golden.py
from the CPU oracle).

CPU: the stored singular-cell constants agree with numerical quadrature, and
the oracle still reproduces every stored operator output (any change of its
arithmetic shows here).  GPU: the CUDA path, planned from the stored geometry
alone, matches the stored outputs of the single and double layer operators
and of the boundary-condition split (Eq. 4 / Eq. 8 at c = 1/2): relative L2
<= 1e-12 in FP64 and 2e-6 in FP32, the parity tolerances of every other test.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
OPERATOR_FIXTURES = ["circle_n16_laplace2d.txt", "cube_n16_laplace3d.txt", "cube_n16_kelvin3d.txt"]
TOL = {"f64": 1e-12, "f32": 2e-6}


def read_fixture(name):
    """key -> list of tokens, for every non-comment line."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            out.setdefault(key, []).append(vals)
    return out


def operator_fixture(name):
    raw = read_fixture(name)
    one = {k: v[0] for k, v in raw.items()}
    dim, nb, nc = int(one["dim"][0]), int(one["nb"][0]), int(one["ncomp"][0])
    f = lambda k: np.array(one[k], dtype=np.float64)  # noqa: E731
    fx = dict(kernel=one["kernel"][0], dim=dim, n=int(one["n"][0]), h=float(one["h"][0]), nu=float(one["nu"][0]),
              mu=float(one["mu"][0]), c=float(one["c"][0]), nb=nb, ncomp=nc,
              cell=np.array(one["cell"], dtype=np.int32).reshape(nb, dim), w=f("w"),
              normal=f("normal").reshape(nb, dim), bc=np.array(one["bc"], dtype=np.uint8),
              x=f("x"), single=f("single"), double=f("double"), system=f("system"))
    for k in ("bc", "x", "single", "double", "system"):
        assert fx[k].size == nb * nc, k
    return fx


def rel_l2(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ------------------------------------------------------------------ CPU side

def test_stored_self_terms_match_quadrature():
    integrate = pytest.importorskip("scipy.integrate")
    st = {k: v for k, v in read_fixture("self_terms.txt").items()}
    L2 = float(st["L2"][0][0])
    C3 = float(st["C3"][0][0])
    # mean of ln r over [-1/2, 1/2]^2 and integral of 1/r over [-1/2, 1/2]^3
    # (z-integral in closed form), by adaptive quadrature
    q2, _ = integrate.dblquad(lambda y, x: 0.5 * math.log(x * x + y * y), 0.0, 0.5, 0.0, 0.5,
                              epsabs=1e-13, epsrel=1e-13)
    q3, _ = integrate.dblquad(lambda y, x: math.asinh(0.5 / math.hypot(x, y)) if (x > 0 or y > 0) else 0.0,
                              0.0, 0.5, 0.0, 0.5, epsabs=1e-13, epsrel=1e-13)
    assert abs(L2 - 4.0 * q2) < 1e-10
    assert abs(C3 - 8.0 * q3) < 1e-9
    # scaling in h of the cell averages: -ln h / (2 pi) shift in 2D, 1/h in 3D
    (h1, u1), (h2, u2) = [(float(a), float(b)) for a, b in st["lap2d_U0"]]
    assert abs((u2 - u1) - (-(math.log(h2) - math.log(h1)) / (2 * math.pi))) < 1e-13
    for key in ("lap3d_U0", "kelvin_U0_diag"):
        (h1, u1), (h2, u2) = [(float(a), float(b)) for a, b in st[key]]
        assert abs(u1 * h1 - u2 * h2) < 1e-13 * abs(u1 * h1), key


def test_oracle_reproduces_stored_self_terms(oracle_mod):
    st = read_fixture("self_terms.txt")
    lib = oracle_mod._load()
    assert abs(oracle_mod.L2() - float(st["L2"][0][0])) < 1e-15
    assert abs(oracle_mod.C3() - float(st["C3"][0][0])) < 1e-15
    for h, v in st["lap2d_U0"]:
        assert abs(lib.bo_lap2d_U(0.0, 0.0, float(h)) - float(v)) < 1e-14 * abs(float(v))
    for h, v in st["lap3d_U0"]:
        assert abs(lib.bo_lap3d_U(0.0, 0.0, 0.0, float(h)) - float(v)) < 1e-14 * abs(float(v))


@pytest.mark.parametrize("name", OPERATOR_FIXTURES)
def test_oracle_reproduces_stored_operators(oracle_mod, name):
    fx = operator_fixture(name)
    kw = dict(nu=fx["nu"], mu=fx["mu"])
    args = (fx["cell"], fx["h"], fx["w"], fx["normal"])
    got = {"single": oracle_mod.apply(fx["kernel"], 0, *args, fx["x"], **kw),
           "double": oracle_mod.apply(fx["kernel"], 1, *args, fx["x"], **kw),
           "system": oracle_mod.system_apply(fx["kernel"], *args, fx["bc"], fx["x"], c=fx["c"], **kw)}
    for layer, y in got.items():
        ref = fx[layer]
        # the same sums in the same order; libm and FMA contraction may differ between hosts
        assert np.max(np.abs(np.reshape(y, -1) - ref)) <= 1e-13 * np.max(np.abs(ref)), layer


# ------------------------------------------------------------------ GPU side

@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_00845_gb300 import build
    build.build()
    return torch


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name", OPERATOR_FIXTURES)
def test_cuda_path_matches_stored_operators(torch_cuda, name, prec):
    from paper_1809_00845_gb300.bem import Plan
    fx = operator_fixture(name)
    plan = Plan(fx["dim"], fx["n"], fx["h"], fx["cell"], fx["w"], fx["normal"], kernel=fx["kernel"],
                precision=prec, nu=fx["nu"], mu=fx["mu"])
    x = torch_cuda.from_numpy(fx["x"].astype(plan.np_dtype)).cuda()
    plan.set_bc(fx["bc"], fx["c"])
    for layer in ("single", "double", "system"):
        y = plan.apply(layer, x)
        torch_cuda.cuda.synchronize()
        err = rel_l2(y.cpu().numpy(), fx[layer])
        assert err <= TOL[prec], (layer, err)
