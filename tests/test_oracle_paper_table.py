"""Pin against the paper's printed numbers: Table tab:fixedHorizon, constant kernel, 6x6, h=0.004.

Setting of Sec. 6.2: constant l-infinity kernel 3/(4 delta^4) (eq. constantkernel),
delta = 0.008, u = x1^2 x2 + x2^2 with g = u on the collar and the forcing read as
f = -2(1 + x2) = -Lap(u) (the printed -2(1 + x1) does not match the stated u; the
reported rates of convergence require a consistent pair).

Facts checked:
* with delta/h = 2 the discrete solution is exact at the nodes (the interpolation error
  of a cubic is reproduced by the exact l-infinity quadrature on this mesh), so the L2
  error equals the interpolation error of u;
* that L2 error brackets the paper's 3.47e-6: it depends on the cell diagonal
  (5.9e-6 for the diagonal used here, 3.1e-6 for the mirrored one), so the test accepts
  a factor of two either way;
* FETI reaches the single-domain solution and its iteration count is of the paper's
  order (the paper does not state the norm of its stopping test: sanity band only).
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import feti, problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_table_fixed_horizon.txt")


def _golden_row(kernel, K):
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] == kernel and f[1] == K:
            return dict(h=float(f[2]), feti_its=int(f[5]), l2=float(f[7]))
    raise KeyError((kernel, K))


@pytest.mark.slow
def test_constant_kernel_6x6_row():
    row = _golden_row("constant", "6x6")
    N = int(round(1.0 / row["h"]))
    delta = 0.008
    mesh = W.make_mesh(2, N, W.collar_cells(delta, N))
    kern = W.Kernel(W.KERNEL_CONST_LINF, delta)
    kern.scale = W.default_scale(kern, 2)
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    exact = lambda a, b: a * a * b + b * b
    u = exact(x, y).reshape(-1, 1)
    f = (-2.0 * (1.0 + y)).reshape(-1, 1)
    mono = problem.Monolithic(mesh, kern)
    uh = mono.solve(f, 0, u)[:, 0]
    free = mesh.node_is_dirichlet == 0
    assert np.abs(uh - u[:, 0])[free].max() < 1e-10
    l2 = problem.l2_error(mesh, uh, exact)
    assert 0.5 * row["l2"] <= l2 <= 2.0 * row["l2"], l2
    labels = W.rect_labels(mesh, 6, 6)
    fo = feti.Feti(mesh, kern, labels, 36)
    uf, info = fo.solve(f, 0, u)
    assert np.abs(uf[:, 0] - uh)[free].max() < 1e-9
    its = int(info["iterations"][0])
    assert 0.6 * row["feti_its"] <= its <= 1.5 * row["feti_its"], its
