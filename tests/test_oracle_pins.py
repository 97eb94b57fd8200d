"""Pins of the FP64 oracle's assembly against facts the paper and the mathematics fix.

* 1-D constant kernel, uniform mesh, delta/h integer: for quadratic u the P1
  interpolation error is h-periodic, so every interior row satisfies
  sum_j A_ij x_j^2 = -(4 c delta^3 / 3) h exactly (c = 3/delta^3 gives -4h), with zero
  row sums and sum_j A_ij x_j = 0; the solve with g = x^2/2, f = -2 returns x^2/2.
* 2-D l-infinity constant kernel 3/(4 delta^4) (eq. constantkernel), delta/h integer:
  the same argument gives A I_h u = -Lap(u) h^2 in every interior row for quadratic u.
* Difference form: constants are in the kernel of [A  B] for every kernel (row sums 0);
  for peridynamics both translations and the rotation are (Sec. 5.2).
* Continuous limits of the kernel constants (Sec. 6.1): interior rows of A I_h u approach
  -Lap(u) h^2 (constant l2, fractional s=0.4, 0.5) and the Navier operator
  -pi/4 Lap u - pi/2 grad div u (peridynamics) for quadratic u.
* Symmetry and positive definiteness of A (Sec. 2.3.3).
"""
import numpy as np
import pytest

import workloads as W
from oracle import assembly, problem


def _rows_free(mesh, kern):
    free = np.flatnonzero(mesh.node_is_dirichlet == 0)
    nc = kern.ncomp
    dofs = (free[:, None] * nc + np.arange(nc)[None, :]).ravel()
    return dofs, assembly.assemble_rows(mesh, kern, kern.scale, dofs)


@pytest.mark.parametrize("N", [200, 250])
def test_1d_quadratic_row_identity(N):
    w = W.const_1d(N=N, K=2)
    dofs, rows = _rows_free(w.mesh, w.kernel)
    x = w.mesh.xy[:, 0]
    h = 1.0 / N
    scale = np.abs(rows).max()
    assert np.abs(rows.sum(axis=1)).max() <= 1e-12 * scale
    assert np.abs(rows @ x).max() <= 1e-12 * scale
    np.testing.assert_allclose(rows @ (x * x), -4.0 * h, rtol=0, atol=1e-11 * scale)


def test_1d_quadratic_solution_exact():
    w = W.manufactured_1d_quadratic(N=200, K=3)
    mono = problem.Monolithic(w.mesh, w.kernel)
    u = mono.solve(w.rhs, w.rhs_kind, w.g)
    x = w.mesh.xy[:, 0]
    assert np.abs(u[:, 0] - 0.5 * x * x).max() < 1e-12


def test_1d_alternative_scale_solution_exact():
    # with c = 3/(2 delta^3) the operator tends to -u'', so u = x^2 solves f = -2
    w = W.manufactured_1d_quadratic(N=100, K=2)
    w.kernel.scale = 3.0 / (2.0 * w.kernel.delta ** 3)
    x = w.mesh.xy[:, 0]
    w.g = (x * x).reshape(-1, 1)
    mono = problem.Monolithic(w.mesh, w.kernel)
    u = mono.solve(w.rhs, w.rhs_kind, w.g)
    assert np.abs(u[:, 0] - x * x).max() < 1e-12


@pytest.mark.parametrize("N,dcells", [(16, 2), (20, 3)])
def test_2d_linf_quadratic_rows(N, dcells):
    delta = dcells / N
    mesh = W.make_mesh(2, N, W.collar_cells(delta, N))
    kern = W.Kernel(W.KERNEL_CONST_LINF, delta)
    kern.scale = W.default_scale(kern, 2)
    _, rows = _rows_free(mesh, kern)
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    h = 1.0 / N
    for u, lap in [(x * x, 2.0), (x * y, 0.0), (y * y, 2.0), (3 * x * x - x * y + 0.5 * y * y + x - 2 * y + 1, 7.0)]:
        assert np.abs(rows @ u + lap * h * h).max() <= 5e-12 * h * h


def test_2d_linf_quadratic_solution_exact():
    N, delta = 16, 2 / 16
    mesh = W.make_mesh(2, N, W.collar_cells(delta, N))
    kern = W.Kernel(W.KERNEL_CONST_LINF, delta)
    kern.scale = W.default_scale(kern, 2)
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    u = (x * x + 2 * x * y - y * y + 0.3 * x).reshape(-1, 1)   # Laplacian 0 -> f = 0
    mono = problem.Monolithic(mesh, kern)
    sol = mono.solve(np.zeros_like(u), 0, u)
    assert np.abs(sol - u).max() < 1e-12


@pytest.mark.parametrize("kt,s", [(W.KERNEL_CONST_L2, 0.0), (W.KERNEL_FRACTIONAL, 0.4), (W.KERNEL_FRACTIONAL, 0.5),
                                  (W.KERNEL_PERIDYNAMIC, 0.0)])
def test_difference_form_kernel(kt, s):
    N, delta = 12, 0.25
    mesh = W.make_mesh(2, N, W.collar_cells(delta, N))
    kern = W.Kernel(kt, delta, s=s)
    kern.scale = W.default_scale(kern, 2)
    _, rows = _rows_free(mesh, kern)
    sc = np.abs(rows).max()
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    if kern.ncomp == 1:
        assert np.abs(rows.sum(axis=1)).max() <= 1e-12 * sc
    else:
        tx = np.zeros(2 * mesh.n_nodes); tx[0::2] = 1.0
        ty = np.zeros(2 * mesh.n_nodes); ty[1::2] = 1.0
        rot = np.zeros(2 * mesh.n_nodes); rot[0::2] = -y; rot[1::2] = x
        for v in (tx, ty, rot):
            assert np.abs(rows @ v).max() <= 1e-12 * sc


@pytest.mark.parametrize("kt,N,delta,s", [(W.KERNEL_CONST_L2, 64, 0.1, 0.0), (W.KERNEL_FRACTIONAL, 48, 0.125, 0.4),
                                          (W.KERNEL_FRACTIONAL, 48, 0.125, 0.5)])
def test_scalar_kernel_constants_continuous_limit(kt, N, delta, s):
    mesh = W.make_mesh(2, N, W.collar_cells(delta, N))
    kern = W.Kernel(kt, delta, s=s)
    kern.scale = W.default_scale(kern, 2)
    c = np.flatnonzero((np.abs(mesh.xy[:, 0] - 0.5) < 1e-12) & (np.abs(mesh.xy[:, 1] - 0.5) < 1e-12))
    rows = assembly.assemble_rows(mesh, kern, kern.scale, c)
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    h = 1.0 / N
    assert abs((rows @ (x * x))[0] / (-2 * h * h) - 1.0) < 0.01
    assert abs((rows @ (y * y))[0] / (-2 * h * h) - 1.0) < 0.01
    assert abs((rows @ (x * y))[0] / (h * h)) < 0.01


def test_peridynamic_constant_navier_limit():
    N, delta = 48, 6 / 48
    mesh = W.make_mesh(2, N, W.collar_cells(delta, N))
    kern = W.Kernel(W.KERNEL_PERIDYNAMIC, delta)
    kern.scale = W.default_scale(kern, 2)
    c = np.flatnonzero((np.abs(mesh.xy[:, 0] - 0.5) < 1e-12) & (np.abs(mesh.xy[:, 1] - 0.5) < 1e-12))[0]
    rows = assembly.assemble_rows(mesh, kern, kern.scale, [2 * c, 2 * c + 1])
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    h = 1.0 / N
    U = np.zeros(2 * mesh.n_nodes); U[0::2] = x * x          # Lap = (2,0), grad div = (2,0)
    r = rows @ U / (h * h)
    assert abs(r[0] / (-1.5 * np.pi) - 1) < 0.01 and abs(r[1]) < 0.01
    U = np.zeros(2 * mesh.n_nodes); U[1::2] = x * y          # Lap = 0, grad div = (1,0)
    r = rows @ U / (h * h)
    assert abs(r[0] / (-0.5 * np.pi) - 1) < 0.01 and abs(r[1]) < 0.01


@pytest.mark.parametrize("maker", [lambda: W.const_l2_2d(N=16, k=2, nrhs=1),
                                   lambda: W.fractional_2d(N=12, k=2, nrhs=1),
                                   lambda: W.peridynamic_2d(N=16, k=2, nrhs=1, jitter=0.0)])
def test_symmetric_positive_definite(maker):
    w = maker()
    mono = problem.Monolithic(w.mesh, w.kernel, dense=True)
    A = mono.A
    assert np.abs(A - A.T).max() <= 1e-15 * np.abs(A).max() * 8
    assert np.linalg.eigvalsh(0.5 * (A + A.T))[0] > 0
