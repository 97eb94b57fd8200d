"""Nonlocal subdivision and the FETI index structures, FP64 / integer (test infrastructure only).

Follows Sec. 3.1 (Def. nonlocalsubdivision, eq. subdomainDefinitions), eq. zeta,
Sec. 3.3 (index sets I_k, G_k; the jump matrix B, eq. constraintSpace), eq. matKerS,
Sec. 4.1 (B_D, D) and Sec. 5.1 (construction from a local decomposition).

Readings taken where the paper leaves a choice:

* Extension (Sec. 5.1): an interior element E joins Omega-hat_k when the l-infinity
  distance between the bounding box of E and that of some element of the local
  part Omega-tilde_k is <= delta/2 (times 1+1e-9); a collar element joins
  Gamma^D_k under the same test with delta.  Bounding boxes only enlarge the
  sets, which the definition allows (supersets are admissible).
* zeta at element pairs counts the subdomains whose Omega-hat_k u Gamma^D_k holds
  both elements; zeta at a node counts the Omega-hat_k holding the node.
* Dofs of k: non-Dirichlet nodes of Omega-hat_k, ordered Omega_k first (zeta=1)
  then Gamma_k (zeta>=2), each by ascending node id; vector kernels add the
  component as the fastest index.
* B: for every interface node (ascending id), its subdomains k_1<...<k_z, one row
  per chain link j (+1 on k_j, -1 on k_j+1), the component fastest.
* Pinned dofs of floating subdomains (Sec. 5.3): scalar -- the lowest-id node of
  Gamma_k; vector -- both components of that node a, and at the Gamma_k node b
  farthest from a (ties: lowest id) the component along which |x_b - x_a| is smaller.
* Z_k: constants on Gamma_k (scalar); (e_x, e_y, (-(y-yc), x-xc)) with the Gamma_k
  centroid (vector).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.spatial import cKDTree


@dataclass
class Subdomain:
    k: int
    elems_hat: np.ndarray        # elements of Omega-hat_k
    elems_dir: np.ndarray        # elements of Gamma^D_k
    omega_nodes: np.ndarray      # I_k nodes (ascending)
    gamma_nodes: np.ndarray      # G_k nodes (ascending)
    floating: bool
    pinned: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))  # Gamma-local dof indices

    @property
    def nodes(self) -> np.ndarray:
        return np.concatenate([self.omega_nodes, self.gamma_nodes])


@dataclass
class Decomposition:
    K: int
    ncomp: int
    subs: list
    node_zeta: np.ndarray        # (n_nodes,) number of Omega-hat_k holding the node
    elem_mask: np.ndarray        # (n_elems, ceil(K / 64)) uint64: bit k % 64 of word k // 64 <=> element in
                                 # Omega-hat_k u Gamma^D_k
    u_offset: np.ndarray         # (K+1,) offsets of Gamma_k blocks in U (in dofs)
    B_plus: np.ndarray           # (M_C,) U index with +1
    B_minus: np.ndarray          # (M_C,) U index with -1
    B_node: np.ndarray           # (M_C,) interface node of each row
    floating: np.ndarray         # (K,) bool
    Z: np.ndarray                # (U, n_coarse) dense
    coarse_offset: np.ndarray    # (K+1,) columns of Z per subdomain

    @property
    def n_lambda(self) -> int:
        return self.B_plus.size

    @property
    def n_u(self) -> int:
        return int(self.u_offset[-1])

    def in_sub(self, k):
        """(n_elems,) bool: the element belongs to Omega-hat_k u Gamma^D_k."""
        return ((self.elem_mask[:, k // 64] >> np.uint64(k % 64)) & np.uint64(1)).astype(bool)

    def dofs(self, k):
        """Global dof ids (node*nc + comp) of subdomain k, Omega block first."""
        s = self.subs[k]
        nc = self.ncomp
        return (s.nodes[:, None] * nc + np.arange(nc)[None, :]).ravel()

    def n_omega(self, k):
        return self.subs[k].omega_nodes.size * self.ncomp

    def n_gamma(self, k):
        return self.subs[k].gamma_nodes.size * self.ncomp

    def B_dense(self):
        B = np.zeros((self.n_lambda, self.n_u))
        r = np.arange(self.n_lambda)
        B[r, self.B_plus] += 1.0
        B[r, self.B_minus] -= 1.0
        return B

    def B_D_dense(self):
        """B_D = (B D^-1 B^T)^-1 B D^-1 with D = diag(zeta) on U (eq. preconditioner), per node block."""
        B = self.B_dense()
        zeta_u = np.zeros(self.n_u)
        for k, s in enumerate(self.subs):
            z = self.node_zeta[s.gamma_nodes]
            zeta_u[self.u_offset[k]:self.u_offset[k + 1]] = np.repeat(z, self.ncomp)
        Dinv = 1.0 / zeta_u
        BD = np.zeros_like(B)
        # B D^-1 B^T is block diagonal: one block per (interface node, component)
        comp = np.arange(self.n_lambda) % self.ncomp if self.ncomp > 1 else np.zeros(self.n_lambda, np.int64)
        keys = self.B_node * self.ncomp + comp
        order = np.argsort(keys, kind="stable")
        ks = keys[order]
        bounds = np.flatnonzero(np.diff(ks)) + 1
        for rows in np.split(order, bounds):
            Bb = B[rows] * Dinv[None, :]
            Sb = Bb @ B[rows].T
            BD[rows] = np.linalg.solve(Sb, Bb)
        return BD


def _bbox(mesh):
    P = mesh.xy[mesh.elems]                  # (n_elems, nv, dim)
    return P.min(axis=1), P.max(axis=1)


def _within(mesh, lo, hi, src_elems, cand_mask, r):
    """Elements in cand_mask whose bbox is within l-infinity distance r of the bbox of some src element."""
    n = mesh.n_elems
    out = np.zeros(n, dtype=bool)
    if src_elems.size == 0:
        return out
    cen = 0.5 * (lo + hi)
    half = 0.5 * (hi - lo)
    hmax = float(half.max())
    cand = np.flatnonzero(cand_mask)
    if cand.size == 0:
        return out
    tree = cKDTree(cen[cand])
    rad = r + 2.0 * hmax + 1e-12
    for c0 in range(0, src_elems.size, 512):
        src = src_elems[c0:c0 + 512]
        lists = tree.query_ball_point(cen[src], rad, p=np.inf)
        cnt = np.array([len(l) for l in lists])
        if cnt.sum() == 0:
            continue
        ii = np.repeat(src, cnt)
        jj = cand[np.concatenate([np.asarray(l, dtype=np.int64) for l in lists])]
        gap = np.maximum(0.0, np.maximum(lo[jj] - hi[ii], lo[ii] - hi[jj]))   # (pairs, dim)
        dist = gap.max(axis=1)
        ok = dist <= r
        out[jj[ok]] = True
    return out


def build_decomposition(mesh, kernel, labels, K) -> Decomposition:
    delta = kernel.delta
    nc = kernel.ncomp
    lo, hi = _bbox(mesh)
    interior = mesh.elem_is_dirichlet == 0
    collar = ~interior
    r_ext = (0.5 * delta) * (1.0 + 1e-9)
    r_dir = delta * (1.0 + 1e-9)
    elem_mask = np.zeros((mesh.n_elems, (K + 63) // 64), dtype=np.uint64)
    hat_sets, dir_sets = [], []
    for k in range(K):
        src = np.flatnonzero(labels == k)
        if src.size == 0:
            raise ValueError(f"empty local subdomain {k}")
        hat = _within(mesh, lo, hi, src, interior, r_ext)
        hat[src] = True
        dirk = _within(mesh, lo, hi, src, collar, r_dir)
        hat_sets.append(np.flatnonzero(hat))
        dir_sets.append(np.flatnonzero(dirk))
        elem_mask[hat, k // 64] |= np.uint64(1) << np.uint64(k % 64)
        elem_mask[dirk, k // 64] |= np.uint64(1) << np.uint64(k % 64)
    # nodes of each Omega-hat_k (non-Dirichlet)
    node_sets = []
    node_zeta = np.zeros(mesh.n_nodes, dtype=np.int64)
    for k in range(K):
        nodes = np.unique(mesh.elems[hat_sets[k]].ravel())
        nodes = nodes[mesh.node_is_dirichlet[nodes] == 0]
        node_sets.append(nodes)
        node_zeta[nodes] += 1
    subs = []
    for k in range(K):
        nodes = node_sets[k]
        z = node_zeta[nodes]
        om = nodes[z == 1]
        ga = nodes[z >= 2]
        floating = dir_sets[k].size == 0
        subs.append(Subdomain(k, hat_sets[k], dir_sets[k], om, ga, floating))
    # U layout
    u_off = np.zeros(K + 1, dtype=np.int64)
    for k in range(K):
        u_off[k + 1] = u_off[k] + subs[k].gamma_nodes.size * nc
    # position of each node in each Gamma_k
    gpos = [dict(zip(s.gamma_nodes.tolist(), range(s.gamma_nodes.size))) for s in subs]
    # B rows (chain per interface node)
    owners = {}
    for k in range(K):
        for n in subs[k].gamma_nodes.tolist():
            owners.setdefault(n, []).append(k)
    bp, bm, bn = [], [], []
    for n in sorted(owners):
        ks = sorted(owners[n])
        for j in range(len(ks) - 1):
            ka, kb = ks[j], ks[j + 1]
            for c in range(nc):
                bp.append(u_off[ka] + gpos[ka][n] * nc + c)
                bm.append(u_off[kb] + gpos[kb][n] * nc + c)
                bn.append(n)
    floating = np.array([s.floating for s in subs], dtype=bool)
    # pinned dofs and Z
    ncols = []
    for k, s in enumerate(subs):
        if not s.floating or s.gamma_nodes.size == 0:
            ncols.append(0)
            continue
        if nc == 1:
            s.pinned = np.array([0], dtype=np.int64)       # lowest id node of Gamma_k
            ncols.append(1)
        else:
            xa = mesh.xy[s.gamma_nodes[0]]
            d2 = ((mesh.xy[s.gamma_nodes] - xa) ** 2).sum(axis=1)
            b = int(np.flatnonzero(d2 == d2.max())[0])
            dx = np.abs(mesh.xy[s.gamma_nodes[b]] - xa)
            comp = 0 if dx[0] < dx[1] else 1
            s.pinned = np.array([0, 1, 2 * b + comp], dtype=np.int64)
            ncols.append(3)
    c_off = np.concatenate([[0], np.cumsum(ncols)]).astype(np.int64)
    n_u = int(u_off[-1])
    Z = np.zeros((n_u, int(c_off[-1])))
    for k, s in enumerate(subs):
        if ncols[k] == 0:
            continue
        r0, r1 = u_off[k], u_off[k + 1]
        if nc == 1:
            Z[r0:r1, c_off[k]] = 1.0
        else:
            X = mesh.xy[s.gamma_nodes]
            xc = X.mean(axis=0)
            Z[r0:r1:2, c_off[k]] = 1.0
            Z[r0 + 1:r1:2, c_off[k] + 1] = 1.0
            Z[r0:r1:2, c_off[k] + 2] = -(X[:, 1] - xc[1])
            Z[r0 + 1:r1:2, c_off[k] + 2] = X[:, 0] - xc[0]
    return Decomposition(K, nc, subs, node_zeta, elem_mask, u_off, np.array(bp, dtype=np.int64),
                         np.array(bm, dtype=np.int64), np.array(bn, dtype=np.int64), floating, Z, c_off)
