"""One-level FETI (Algorithm 1) in FP64 numpy (test infrastructure only).

Steps follow Algorithm 1 of the paper and the formulas it cites:

1. substructures, zeta, Z, B, B_D                 -- ``decomposition.build_decomposition``
2. subdomain matrices A^k (eq. subStiffnessMatrix, kernel weighted by 1/zeta) and
   loads f~^k (eq. bilinear-multi5: F_m / zeta(x_m), minus the Dirichlet coupling)
3. d = B S^+ f, e = Z^T f, G = B Z                 -- eq. FETIproblem, p. G
4. Cholesky factors: A_OO^k (Dirichlet solves for S_k, eq. subSchurComplement),
   the pinned Neumann matrix (Sec. 5.3, eq. neumannSubproblem) for S_k^+, G^T G
5. F = B S^+ B^T, P = I - G (G^T G)^-1 G^T (eq. P), M^-1 = B_D S B_D^T (eq. preconditioner)
6. lambda^0 = G (G^T G)^-1 e
7. projected preconditioned CG on P F lambda = P d
8. alpha = (G^T G)^-1 G^T (d - F lambda)           -- eq. forAlpha
9. u = S^+ (f - B^T lambda) - Z alpha              -- eq. forU; then the back
   substitution u_O = A_OO^-1 (f~_O - A_OG u_G)     -- eq. backwardSubstitution

Reduced forcing f_k = f~_G - A_GO A_OO^-1 f~_O (eq. subForcing).  Nodal output:
copies of an interface node are averaged (they agree to the solver tolerance).

PCG (readings: the paper names a projected PCG with tolerance 1e-10, norm unstated):
w = P r; stop when ||w||_2 <= tol ||P d||_2 (per right-hand side); z = M^-1 w;
y = P z; beta = (y,w)/(y_old,w_old); p = y + beta p; eta = (y,w)/(p,F p);
lambda += eta p; r -= eta F p.  A constraint right-hand side c (B u = c, used by
iterative refinement) enters as d - c.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import assembly
from .decomposition import build_decomposition
from .problem import load_vector


class SubdomainOps:
    def __init__(self, A, n_omega, pinned, Zk):
        self.A = A
        self.nO = n_omega
        self.nG = A.shape[0] - n_omega
        nO = n_omega
        self.AOO = A[:nO, :nO]
        self.AOG = A[:nO, nO:]
        self.AGO = A[nO:, :nO]
        self.AGG = A[nO:, nO:]
        self.cOO = sla.cho_factor(self.AOO, lower=True) if nO > 0 else None
        # Neumann matrix with artificial Dirichlet conditions at the pinned dofs (Sec. 5.3)
        At = A.copy()
        for p in pinned:
            i = nO + int(p)
            At[i, :] = 0.0
            At[:, i] = 0.0
            At[i, i] = 1.0
        self.pinned = np.asarray(pinned, dtype=np.int64)
        self.cN = sla.cho_factor(At, lower=True)
        if Zk is not None and Zk.shape[1] > 0:
            self.Q, _ = np.linalg.qr(Zk)
        else:
            self.Q = None

    def proj(self, v):
        """Orthogonal projection onto range(S_k) = ker(Z_k^T)."""
        if self.Q is None:
            return v
        return v - self.Q @ (self.Q.T @ v)

    def solve_OO(self, b):
        if self.nO == 0:
            return np.zeros((0,) + b.shape[1:])
        return sla.cho_solve(self.cOO, b)

    def S(self, v):
        """S_k v by a Dirichlet solve (eq. subSchurComplement)."""
        if self.nO == 0:
            return self.AGG @ v
        return self.AGG @ v - self.AGO @ self.solve_OO(self.AOG @ v)

    def S_plus(self, v):
        """Moore-Penrose S_k^+ v through the pinned Neumann problem, then removing ker(S_k)."""
        v = self.proj(v)
        rhs = np.zeros((self.nO + self.nG,) + v.shape[1:])
        rhs[self.nO:] = v
        for p in self.pinned:
            rhs[self.nO + p] = 0.0
        w = sla.cho_solve(self.cN, rhs)[self.nO:]
        return self.proj(w)

    def reduced_forcing(self, fO, fG):
        if self.nO == 0:
            return fG.copy()
        return fG - self.AGO @ self.solve_OO(fO)

    def back_substitute(self, fO, uG):
        if self.nO == 0:
            return np.zeros((0,) + uG.shape[1:])
        return self.solve_OO(fO - self.AOG @ uG)


class Feti:
    def __init__(self, mesh, kernel, labels, K, dec=None, nthreads=None):
        self.mesh, self.kernel = mesh, kernel
        self.dec = dec if dec is not None else build_decomposition(mesh, kernel, labels, K)
        d = self.dec
        nc = kernel.ncomp
        self.nc = nc
        self.A = []
        self.ops = []
        self.dof_maps = []
        for k in range(d.K):
            dofs = d.dofs(k)
            dof_of = np.full(mesh.n_nodes * nc, -1, dtype=np.int32)
            dof_of[dofs] = np.arange(dofs.size, dtype=np.int32)
            Ak, _ = assembly.assemble(mesh, kernel, kernel.scale, dof_of, dofs.size, elem_mask=d.elem_mask, k=k,
                                      nthreads=nthreads)
            self.A.append(Ak)
            self.dof_maps.append((dofs, dof_of))
            Zk = d.Z[d.u_offset[k]:d.u_offset[k + 1], d.coarse_offset[k]:d.coarse_offset[k + 1]]
            self.ops.append(SubdomainOps(Ak, d.n_omega(k), d.subs[k].pinned, Zk if Zk.shape[1] else None))
        nl, nu = d.n_lambda, d.n_u
        r = np.arange(nl)
        self.B = sp.csr_matrix((np.concatenate([np.ones(nl), -np.ones(nl)]),
                                (np.concatenate([r, r]), np.concatenate([d.B_plus, d.B_minus]))), shape=(nl, nu))
        self.BD = sp.csr_matrix(d.B_D_dense()) if nl > 0 else sp.csr_matrix((0, nu))
        self.G = self.B @ d.Z                     # dense (n_lambda, n_coarse)
        self.nco = self.G.shape[1]
        if self.nco > 0:
            self.GtG = self.G.T @ self.G
            self.cG = sla.cho_factor(self.GtG, lower=True)

    # ----------------------------------------------------------------- operators
    def _split_U(self, x):
        d = self.dec
        return [x[d.u_offset[k]:d.u_offset[k + 1]] for k in range(d.K)]

    def S_plus(self, x):
        return np.concatenate([op.S_plus(xk) for op, xk in zip(self.ops, self._split_U(x))], axis=0)

    def S(self, x):
        return np.concatenate([op.S(xk) for op, xk in zip(self.ops, self._split_U(x))], axis=0)

    def F(self, lam):
        return self.B @ self.S_plus(self.B.T @ lam)

    def Minv(self, w):
        return self.BD @ self.S(self.BD.T @ w)

    def P(self, w):
        if self.nco == 0:
            return w
        return w - self.G @ sla.cho_solve(self.cG, self.G.T @ w)

    # --------------------------------------------------------------------- loads
    def subdomain_loads(self, rhs, rhs_kind, g=None):
        """f~^k for each subdomain: F_m / zeta(x_m) minus the Dirichlet coupling of A^k (eq. bilinear-multi5)."""
        mesh, nc, d = self.mesh, self.nc, self.dec
        Fg = load_vector(mesh, nc, rhs, rhs_kind)
        zeta = np.repeat(d.node_zeta, nc).astype(np.float64)
        zeta[zeta == 0] = 1.0
        out = []
        for k in range(d.K):
            dofs, dof_of = self.dof_maps[k]
            f = Fg[dofs] / zeta[dofs][:, None]
            if g is not None:
                g2 = np.asarray(g, dtype=np.float64)
                if g2.ndim == 1:
                    g2 = g2[:, None]
                for j in range(f.shape[1]):
                    _, Bg = assembly.assemble(mesh, self.kernel, self.kernel.scale, dof_of, dofs.size,
                                              elem_mask=d.elem_mask, k=k, g=g2[:, j], matrix=False)
                    f[:, j] -= Bg
            out.append(f)
        return out

    # ------------------------------------------------------------------- solver
    def solve_torn(self, ftil, c=None, tol=1e-10, max_it=1000, lam_init=None):
        """Solve the torn system for subdomain loads ftil (list of (n_k, R)); returns per-subdomain u and info."""
        d = self.dec
        R = ftil[0].shape[1]
        fU = np.concatenate([op.reduced_forcing(f[:op.nO], f[op.nO:]) for op, f in zip(self.ops, ftil)], axis=0) \
            if d.n_u > 0 else np.zeros((0, R))
        nl = d.n_lambda
        info = dict(iterations=np.zeros(R, dtype=np.int64))
        if nl > 0:
            dvec = self.B @ self.S_plus(fU)
            if c is not None:
                dvec = dvec - c
            e = d.Z.T @ fU if self.nco > 0 else np.zeros((0, R))
            lam = self.G @ sla.cho_solve(self.cG, e) if self.nco > 0 else np.zeros((nl, R))
            lam0 = lam.copy()
            r = dvec - self.F(lam)
            Pd = self.P(dvec)
            nPd = np.linalg.norm(Pd, axis=0)
            p = np.zeros_like(lam)
            yw_old = np.ones(R)
            active = np.ones(R, dtype=bool)
            hist = []
            for it in range(max_it + 1):
                w = self.P(r)
                nw = np.linalg.norm(w, axis=0)
                hist.append(nw / np.where(nPd > 0, nPd, 1.0))
                active &= ~(nw <= tol * nPd)
                if not active.any():
                    break
                if it == max_it:
                    break
                z = self.Minv(w)
                y = self.P(z)
                yw = (y * w).sum(axis=0)
                beta = np.where(it == 0, 0.0, yw / np.where(yw_old != 0, yw_old, 1.0))
                p = y + beta[None, :] * p
                q = self.F(p)
                pq = (p * q).sum(axis=0)
                eta = np.where(active, yw / np.where(pq != 0, pq, 1.0), 0.0)
                lam = lam + eta[None, :] * p
                r = r - eta[None, :] * q
                yw_old = np.where(active, yw, yw_old)
                info["iterations"] += active
            alpha = sla.cho_solve(self.cG, self.G.T @ (dvec - self.F(lam))) if self.nco > 0 else np.zeros((0, R))
            uU = self.S_plus(fU - self.B.T @ lam) - (d.Z @ alpha if self.nco > 0 else 0.0)
            info.update(d=dvec, e=e, lam0=lam0, lam=lam, alpha=alpha, hist=np.array(hist))
        else:
            uU = self.S_plus(fU) if d.n_u > 0 else np.zeros((0, R))
            info.update(lam=np.zeros((0, R)), alpha=np.zeros((0, R)))
        info["fU"] = fU
        uk = []
        for k, (op, f) in enumerate(zip(self.ops, ftil)):
            uG = uU[d.u_offset[k]:d.u_offset[k + 1]]
            uO = op.back_substitute(f[:op.nO], uG)
            uk.append(np.concatenate([uO, uG], axis=0))
        return uk, info

    def nodal(self, uk, g=None):
        """Average the copies of each node (zeta-weighted mean); Dirichlet entries get g (or 0)."""
        mesh, nc, d = self.mesh, self.nc, self.dec
        R = uk[0].shape[1]
        u = np.zeros((mesh.n_nodes * nc, R))
        cnt = np.zeros(mesh.n_nodes * nc)
        for k in range(d.K):
            dofs, _ = self.dof_maps[k]
            u[dofs] += uk[k]
            cnt[dofs] += 1
        free = cnt > 0
        u[free] /= cnt[free][:, None]
        if g is not None:
            g2 = np.asarray(g, dtype=np.float64)
            if g2.ndim == 1:
                g2 = g2[:, None]
            dn = np.repeat(mesh.node_is_dirichlet == 1, nc)
            u[dn] = g2[dn]
        return u

    def solve(self, rhs, rhs_kind, g=None, tol=1e-10, max_it=1000):
        ftil = self.subdomain_loads(rhs, rhs_kind, g)
        uk, info = self.solve_torn(ftil, tol=tol, max_it=max_it)
        return self.nodal(uk, g), info
