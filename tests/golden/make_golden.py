"""Writes the stored expected values under tests/golden/ (run from the repo root:
``python tests/golden/make_golden.py``).

Every value comes from the CPU oracle (FP64 direct sums, ``oracle/``) on
seeded inputs from ``paper_1809_00845_gb300.inputs``; nothing here runs the
CUDA path.  The fixtures let the GPU tests compare against stored numbers
without running the oracle, and let the CPU tests notice any change of the
oracle's arithmetic.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1809_00845_gb300 import inputs as I  # noqa: E402


def _fmt(a):
    a = np.asarray(a).reshape(-1)
    if a.dtype.kind in "iu":
        return " ".join(str(int(v)) for v in a)
    return " ".join(repr(float(v)) for v in a)


def write_operator_fixture(path, header, kernel, b, seed, nu=0.3, mu=1.0, c=0.5):
    rng = np.random.default_rng(seed)
    nc = 3 if kernel == "kelvin3d" else 1
    x = rng.standard_normal(b.nb * nc)
    bc = (rng.uniform(size=b.nb * nc) < 0.5).astype(np.int64)
    single = O.apply(kernel, 0, b.cell, b.h, b.w, b.normal, x, nu=nu, mu=mu)
    double = O.apply(kernel, 1, b.cell, b.h, b.w, b.normal, x, nu=nu, mu=mu)
    system = O.system_apply(kernel, b.cell, b.h, b.w, b.normal, bc, x, c=c, nu=nu, mu=mu)
    lines = ["# " + h for h in header]
    lines += ["# written by tests/golden/make_golden.py from the CPU oracle (FP64 direct sums)",
              f"kernel {kernel}", f"dim {b.dim}", f"n {b.n}", f"h {b.h!r}", f"nu {nu!r}", f"mu {mu!r}", f"c {c!r}",
              f"nb {b.nb}", f"ncomp {nc}",
              "cell " + _fmt(b.cell), "w " + _fmt(b.w), "normal " + _fmt(b.normal), "bc " + _fmt(bc),
              "x " + _fmt(x), "single " + _fmt(single), "double " + _fmt(double), "system " + _fmt(system)]
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def write_self_terms(path):
    lib = O._load()
    nu, mu = 0.3, 1.0
    lines = [
        "# Values on the singular cell (target node = source node) of the kernel tables on constant",
        "# elements (Section 3, the tables approximated on constant elements of the whole grid; Fig. 5).",
        "# Reading: the mean of the kernel over the h-cell (h-square, h-cube) centred at the node.",
        "#   L2 = mean of ln r over [-1/2, 1/2]^2;  C3 = integral of 1/r over [-1/2, 1/2]^3",
        "#   lap2d_U0(h) = -(ln h + L2) / (2 pi)            (Eq. 15 kernel -ln r / (2 pi))",
        "#   lap3d_U0(h) = C3 / (4 pi h)                    (kernel 1 / (4 pi r))",
        "#   kelvin_U0_diag(h) = (3 - 4 nu + 1/3) C3 / (16 pi mu (1 - nu) h)   (Eq. 7, nu = 0.3, mu = 1)",
        "# written by tests/golden/make_golden.py from the CPU oracle",
        f"L2 {O.L2()!r}",
        f"C3 {O.C3()!r}",
    ]
    for h in (1.0 / 16, 1.0 / 4096):
        lines.append(f"lap2d_U0 {h!r} {lib.bo_lap2d_U(0.0, 0.0, h)!r}")
    for h in (1.0 / 16, 1.0 / 512):
        lines.append(f"lap3d_U0 {h!r} {lib.bo_lap3d_U(0.0, 0.0, 0.0, h)!r}")
    for h in (1.0 / 16, 1.0 / 128):
        # one cell of unit weight: the matrix is the singular-cell block
        U = O.matrix("kelvin3d", 0, np.zeros((1, 3), np.int32), h, np.ones(1), np.array([[1.0, 0.0, 0.0]]), nu, mu)
        lines.append(f"kelvin_U0_diag {h!r} {float(U[0, 0])!r}")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def main():
    write_self_terms(os.path.join(HERE, "self_terms.txt"))
    write_operator_fixture(
        os.path.join(HERE, "circle_n16_laplace2d.txt"),
        ["2D Laplace, circle r = 0.35 on a 16^2 grid: single layer S x, double layer D x (Eq. 15: the",
         "discretised boundary integral as a sum over boundary cells with w = in-cell arc length) and the",
         "boundary-condition split A x of Eq. 4 at c = 1/2 (bc 0: Dirichlet, x is q; bc 1: Neumann, x is u)"],
        "laplace2d", I.circle_boundary(16), seed=1016)
    cube = I.cube_boundary(16, 7, 9)
    write_operator_fixture(
        os.path.join(HERE, "cube_n16_laplace3d.txt"),
        ["3D Laplace, surface cells of the cube [7, 9]^3 on a 16^3 grid: S x, D x and the split A x",
         "(the 3D analogue of Eq. 15 and Eq. 4, kernel 1 / (4 pi r), c = 1/2)"],
        "laplace3d", cube, seed=308)
    write_operator_fixture(
        os.path.join(HERE, "cube_n16_kelvin3d.txt"),
        ["Kelvin (3D elasticity), same cube, nu = 0.3, mu = 1: U t (Eq. 7), T u (traction kernel) and",
         "the split A x of Eq. 8 at c = 1/2 (A x = U (x on Dirichlet) - T (x on Neumann) - c x on Neumann)"],
        "kelvin3d", cube, seed=708)


if __name__ == "__main__":
    main()
