"""Load vectors, the single-domain (monolithic) solve and error measures (test infrastructure only).

* Load vector (eq. bil1, F(v) = int_Omega v f): for nodal values of f, the P1
  interpolant of f integrated against each basis function over the interior
  elements, i.e. the consistent P1 mass matrix (|E|/12 [2 1 1; 1 2 1; 1 1 2] in
  2-D, h/6 [2 1; 1 2] in 1-D), per component for the vector kernel.
* Single-domain system (Sec. 2.3.3): A u = f - B g over the non-Dirichlet dofs,
  A symmetric positive definite because Gamma^D is non-empty; solved by LAPACK
  Cholesky (dense, or banded for lexicographic 2-D numbering).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import assembly


def load_vector(mesh, ncomp, rhs, rhs_kind):
    """Global load vector (n_nodes*ncomp, nrhs); Dirichlet entries are present but unused."""
    rhs = np.asarray(rhs, dtype=np.float64)
    if rhs.ndim == 1:
        rhs = rhs[:, None]
    if rhs_kind == 1:
        return rhs.copy()
    nv = mesh.dim + 1
    F = np.zeros_like(rhs)
    els = np.flatnonzero(mesh.elem_is_dirichlet == 0)
    P = mesh.xy[mesh.elems[els]]
    if mesh.dim == 1:
        meas = np.abs(P[:, 1, 0] - P[:, 0, 0])
        Mloc = np.array([[2.0, 1.0], [1.0, 2.0]]) / 6.0
    else:
        meas = 0.5 * np.abs((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1])
                            - (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0]))
        Mloc = np.array([[2.0, 1.0, 1.0], [1.0, 2.0, 1.0], [1.0, 1.0, 2.0]]) / 12.0
    for c in range(ncomp):
        for a in range(nv):
            na = mesh.elems[els, a]
            acc = np.zeros((els.size, rhs.shape[1]))
            for b in range(nv):
                nb = mesh.elems[els, b]
                acc += Mloc[a, b] * rhs[nb * ncomp + c]
            np.add.at(F, na * ncomp + c, meas[:, None] * acc)
    return F


def global_dofs(mesh, ncomp):
    free = np.flatnonzero(mesh.node_is_dirichlet == 0)
    dofs = (free[:, None] * ncomp + np.arange(ncomp)[None, :]).ravel()
    dof_of = np.full(mesh.n_nodes * ncomp, -1, dtype=np.int32)
    dof_of[dofs] = np.arange(dofs.size, dtype=np.int32)
    return dofs, dof_of


def _band_guess(mesh, kernel, ncomp):
    if mesh.dim == 1:
        return None
    row = mesh.N + 2 * mesh.m + 1
    reach = int(np.ceil(kernel.delta * mesh.N)) + 2
    return (reach * row + reach + 2) * ncomp


class Monolithic:
    """Assembled single-domain operator; solve() returns nodal solutions."""

    def __init__(self, mesh, kernel, nthreads=None, dense=None):
        self.mesh, self.kernel = mesh, kernel
        nc = kernel.ncomp
        self.dofs, self.dof_of = global_dofs(mesh, nc)
        n = self.dofs.size
        kd = _band_guess(mesh, kernel, nc)
        if dense is None:
            dense = kd is None or kd >= n or n <= 4000
        self.dense = dense
        if dense:
            A, _ = assembly.assemble(mesh, kernel, kernel.scale, self.dof_of, n, nthreads=nthreads)
            self.A = A
            self.chol = sla.cho_factor(A, lower=True)
        else:
            while True:
                try:
                    ab, _ = assembly.assemble(mesh, kernel, kernel.scale, self.dof_of, n, band=kd, nthreads=nthreads)
                    break
                except RuntimeError:
                    kd *= 2
            self.kd = kd
            self.ab = ab
            self.cb = sla.cholesky_banded(ab, lower=True)

    def dirichlet_term(self, g):
        """B g for one Dirichlet data vector g (n_nodes*nc,)."""
        n = self.dofs.size
        _, Bg = assembly.assemble(self.mesh, self.kernel, self.kernel.scale, self.dof_of, n, g=g, matrix=False)
        return Bg

    def matvec(self, u):
        if self.dense:
            return self.A @ u
        # symmetric lower band product
        n = self.dofs.size
        y = self.ab[0][:, None] * u
        for d in range(1, self.ab.shape[0]):
            a = self.ab[d, : n - d][:, None]
            y[d:] += a * u[: n - d]
            y[: n - d] += a * u[d:]
        return y

    def solve(self, rhs, rhs_kind, g=None):
        mesh, nc = self.mesh, self.kernel.ncomp
        F = load_vector(mesh, nc, rhs, rhs_kind)
        b = F[self.dofs].copy()
        if g is not None:
            g = np.asarray(g, dtype=np.float64)
            if g.ndim == 1:
                g = g[:, None]
            for j in range(b.shape[1]):
                b[:, j] -= self.dirichlet_term(g[:, j])
        if self.dense:
            x = sla.cho_solve(self.chol, b)
        else:
            x = sla.cho_solve_banded((self.cb, True), b)
        u = np.zeros((mesh.n_nodes * nc, b.shape[1]))
        if g is not None:
            u[:] = g
            u[self.dofs] = x
        else:
            u[self.dofs] = x
        return u


def rel_nodal_error(u, ref, mesh, ncomp):
    """max_i |u_i - ref_i| / max_i |ref_i| over non-Dirichlet dofs, per right-hand side."""
    free = np.flatnonzero(mesh.node_is_dirichlet == 0)
    dofs = (free[:, None] * ncomp + np.arange(ncomp)[None, :]).ravel()
    d = np.abs(u[dofs] - ref[dofs]).max(axis=0)
    s = np.abs(ref[dofs]).max(axis=0)
    return d / np.where(s > 0, s, 1.0)


def l2_error(mesh, u_nodal, exact, comp=None):
    """L2 norm over the interior elements of (u_h - u), by the 7-point degree-5 rule per triangle.

    exact(x, y) returns the exact solution at points; u_nodal has one value per node (one component)."""
    els = np.flatnonzero(mesh.elem_is_dirichlet == 0)
    r15 = np.sqrt(15.0)
    a1, a2 = (6 - r15) / 21, (6 + r15) / 21
    B = np.array([[1 / 3, 1 / 3, 1 / 3], [a1, a1, 1 - 2 * a1], [a1, 1 - 2 * a1, a1], [1 - 2 * a1, a1, a1],
                  [a2, a2, 1 - 2 * a2], [a2, 1 - 2 * a2, a2], [1 - 2 * a2, a2, a2]])
    Wq = np.array([9 / 40] + [(155 - r15) / 1200] * 3 + [(155 + r15) / 1200] * 3)
    tri = mesh.elems[els]
    P = mesh.xy[tri]                                   # (ne, 3, 2)
    area = 0.5 * np.abs((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1])
                        - (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0]))
    uv = u_nodal[tri]                                  # (ne, 3)
    s = np.zeros(els.size)
    for q in range(7):
        xq = (B[q][None, :, None] * P).sum(axis=1)     # (ne, 2)
        uh = uv @ B[q]
        s += Wq[q] * (uh - exact(xq[:, 0], xq[:, 1])) ** 2
    return float(np.sqrt((s * area).sum()))
