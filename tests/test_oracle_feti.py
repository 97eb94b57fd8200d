"""Pins of the oracle's decomposition and FETI against the paper's structural facts.

* Nonlocal subdivision covers every interacting element pair (Def.
  nonlocalsubdivision) and 1/zeta is a partition of unity: sum_k R_k^T A^k R_k = A
  (eq. zeta, eq. bilinear-multi1, the equivalence of the multi-domain problem).
* B has one +1 and one -1 per row, full row rank, M_C = sum(zeta - 1) rows per
  component (eq. constraintSpace); G = B Z; B D^-1 B^T is block diagonal with
  blocks smaller than max zeta (Sec. 5.1).
* Floating blocks: A^k Z_k = 0 (Remark floating, Sec. 5.2); A^k_OO and the pinned
  Neumann matrix are positive definite (Sec. 3.3, Sec. 5.3).
* The pinning pseudo-inverse is the Moore-Penrose inverse (Sec. 5.3 and eq. forU):
  compared with an SVD pseudo-inverse; S S^+ S = S.
* FETI solution == single-domain solution (Sec. 4); K = 1 reproduces it.
* Brute force: the dense torn KKT system (eq. discreteKKT) solved by Gaussian
  elimination gives the same multipliers lambda.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import assembly, feti, problem
from oracle.decomposition import build_decomposition

CASES = {
    "1d_k4": lambda: W.const_1d(N=120, K=4, nrhs=2),
    "l2_3x3": lambda: W.const_l2_2d(N=24, k=3, nrhs=2, delta=0.1),
    "frac_3x3": lambda: W.fractional_2d(N=24, k=3, nrhs=2, delta=0.1),
    "frac_deg": lambda: W.fractional_2d(N=24, k=3, nrhs=2, delta=0.25),   # Omega_k empty
    "pd_3x3_jit": lambda: W.peridynamic_2d(N=30, k=3, nrhs=2, delta_cells=3, jitter=0.2),
    "l2_unstructured": lambda: W.unstructured_l2(N=20, K=5, nrhs=2),      # irregular mesh, graph parts
    "pd_unstructured": lambda: W.unstructured_pd(N=20, K=4, nrhs=2),
    "l2_neumann": lambda: W.neumann_l2(N=20, k=3, nrhs=2),                # Neumann region on two sides
    "pd_neumann": lambda: W.neumann_pd(N=24, k=3, nrhs=2),
    "l2_rounded_collar": lambda: W.l2_collar_const(N=20, k=3, nrhs=2, delta=0.15),
    "l2_9x9": lambda: W.const_l2_2d(N=36, k=9, nrhs=1, delta=2.0 / 36),   # K = 81: more than 64 subdomains
}


@pytest.fixture(scope="module")
def built():
    out = {}
    for name, mk in CASES.items():
        w = mk()
        out[name] = (w, feti.Feti(w.mesh, w.kernel, w.labels, w.K))
    return out


def _pairs_within(mesh, delta):
    P = mesh.xy[mesh.elems]
    lo, hi = P.min(axis=1), P.max(axis=1)
    gap = np.maximum(0.0, np.maximum(lo[:, None, :] - hi[None, :, :], lo[None, :, :] - hi[:, None, :])).max(axis=2)
    return gap <= delta


@pytest.mark.parametrize("name", list(CASES))
def test_subdivision_covers_interactions(built, name):
    w, f = built[name]
    d = f.dec
    near = _pairs_within(w.mesh, w.kernel.delta)
    both_dir = (w.mesh.elem_is_dirichlet[:, None] == 1) & (w.mesh.elem_is_dirichlet[None, :] == 1)
    need = near & ~both_dir
    zeta = np.zeros(need.shape, dtype=np.int64)
    for k in range(d.K):
        b = d.in_sub(k)
        zeta += (b[:, None] & b[None, :])
    assert (zeta[need] >= 1).all()
    # every non-Dirichlet node is a dof of some subdomain
    assert (d.node_zeta[w.mesh.node_is_dirichlet == 0] >= 1).all()


@pytest.mark.parametrize("name", list(CASES))
def test_partition_of_unity(built, name):
    w, f = built[name]
    mono = problem.Monolithic(w.mesh, w.kernel, dense=True)
    n = mono.dofs.size
    S = np.zeros((n, n))
    for k in range(f.dec.K):
        dofs, _ = f.dof_maps[k]
        idx = mono.dof_of[dofs]
        S[np.ix_(idx, idx)] += f.A[k]
    assert np.abs(S - mono.A).max() <= 1e-13 * np.abs(mono.A).max()


@pytest.mark.parametrize("name", list(CASES))
def test_jump_operator_structure(built, name):
    w, f = built[name]
    d = f.dec
    B = d.B_dense()
    assert (np.sort(B, axis=1)[:, 0] == -1).all() and (np.sort(B, axis=1)[:, -1] == 1).all()
    assert (np.abs(B).sum(axis=1) == 2).all()
    z = d.node_zeta[d.node_zeta >= 2]
    assert d.n_lambda == int((z - 1).sum()) * d.ncomp
    if d.n_lambda:
        assert np.linalg.matrix_rank(B) == d.n_lambda
        np.testing.assert_allclose(f.G, B @ d.Z)
        # B D^-1 B^T blocks smaller than max zeta
        zeta_u = np.concatenate([np.repeat(d.node_zeta[s.gamma_nodes], d.ncomp) for s in d.subs])
        M = B @ np.diag(1.0 / zeta_u) @ B.T
        nz = M != 0
        for r in range(d.n_lambda):
            assert nz[r].sum() < d.node_zeta.max()
        BD = d.B_D_dense()
        np.testing.assert_allclose(BD @ B.T, np.eye(d.n_lambda), atol=1e-13)


@pytest.mark.parametrize("name", list(CASES))
def test_floating_kernels_and_definiteness(built, name):
    w, f = built[name]
    d = f.dec
    for k in range(d.K):
        op = f.ops[k]
        if op.nO:
            assert np.linalg.eigvalsh(op.AOO)[0] > 0
        nullity = 0
        if d.floating[k]:
            Zk = d.Z[d.u_offset[k]:d.u_offset[k + 1], d.coarse_offset[k]:d.coarse_offset[k + 1]]
            Zfull = np.concatenate([np.zeros((op.nO, Zk.shape[1])), Zk])
            # rigid modes extended to Omega_k: constants / rigid motions on all subdomain nodes
            nodes = d.subs[k].nodes
            if d.ncomp == 1:
                Zfull = np.ones((nodes.size, 1))
            else:
                X = w.mesh.xy[nodes]
                xc = w.mesh.xy[d.subs[k].gamma_nodes].mean(axis=0)
                Zfull = np.zeros((2 * nodes.size, 3))
                Zfull[0::2, 0] = 1
                Zfull[1::2, 1] = 1
                Zfull[0::2, 2] = -(X[:, 1] - xc[1])
                Zfull[1::2, 2] = X[:, 0] - xc[0]
            assert np.abs(f.A[k] @ Zfull).max() <= 1e-12 * np.abs(f.A[k]).max()
            nullity = Zfull.shape[1]
        S = op.S(np.eye(op.nG))
        ev = np.linalg.eigvalsh(0.5 * (S + S.T))
        tol = 1e-10 * ev[-1]
        assert (np.abs(ev) <= tol).sum() == nullity
        assert ev[0] >= -tol


@pytest.mark.parametrize("name", list(CASES))
def test_pseudo_inverse_is_moore_penrose(built, name):
    w, f = built[name]
    for k in range(f.dec.K):
        op = f.ops[k]
        S = op.S(np.eye(op.nG))
        Sp = op.S_plus(np.eye(op.nG))
        ref = np.linalg.pinv(0.5 * (S + S.T), rcond=1e-11, hermitian=True)
        assert np.abs(Sp - ref).max() <= 1e-8 * np.abs(ref).max()
        assert np.abs(S @ Sp @ S - S).max() <= 1e-9 * np.abs(S).max()
        assert np.abs(Sp - Sp.T).max() <= 1e-9 * np.abs(Sp).max()


@pytest.mark.parametrize("name", list(CASES))
def test_feti_equals_monolithic(built, name):
    w, f = built[name]
    mono = problem.Monolithic(w.mesh, w.kernel)
    um = mono.solve(w.rhs, w.rhs_kind, w.g)
    uf, info = f.solve(w.rhs, w.rhs_kind, w.g)
    err = problem.rel_nodal_error(uf, um, w.mesh, w.kernel.ncomp)
    assert (err < 1e-8).all(), err
    if f.dec.n_lambda:
        # admissibility G^T lambda = e and the constraint B u = 0 on U
        lam = info["lam"]
        if f.nco:
            np.testing.assert_allclose(f.G.T @ lam, info["e"], atol=1e-9 * np.abs(info["e"]).max())


def test_single_subdomain_is_monolithic():
    w = W.const_l2_2d(N=16, k=1, nrhs=2)
    f = feti.Feti(w.mesh, w.kernel, w.labels, w.K)
    assert f.dec.n_lambda == 0 and not f.dec.floating.any()
    mono = problem.Monolithic(w.mesh, w.kernel)
    um = mono.solve(w.rhs, w.rhs_kind)
    uf, _ = f.solve(w.rhs, w.rhs_kind)
    assert (problem.rel_nodal_error(uf, um, w.mesh, 1) < 1e-12).all()


@pytest.mark.parametrize("name", ["1d_k4", "l2_3x3", "pd_3x3_jit"])
def test_kkt_brute_force_multipliers(built, name):
    """Dense torn KKT system A^k u_k + R^T B_k^T lambda = f~_k, B u_G = 0 solved directly."""
    w, f = built[name]
    d = f.dec
    ftil = f.subdomain_loads(w.rhs, w.rhs_kind, w.g)
    nks = [A.shape[0] for A in f.A]
    ntot = sum(nks)
    off = np.concatenate([[0], np.cumsum(nks)])
    K = np.zeros((ntot + d.n_lambda, ntot + d.n_lambda))
    rhs = np.zeros((ntot + d.n_lambda, ftil[0].shape[1]))
    # map U index -> torn index
    u2t = np.zeros(d.n_u, dtype=np.int64)
    for k in range(d.K):
        K[off[k]:off[k + 1], off[k]:off[k + 1]] = f.A[k]
        rhs[off[k]:off[k + 1]] = ftil[k]
        nO = d.n_omega(k)
        u2t[d.u_offset[k]:d.u_offset[k + 1]] = off[k] + nO + np.arange(d.n_gamma(k))
    Bt = np.zeros((d.n_lambda, ntot))
    r = np.arange(d.n_lambda)
    Bt[r, u2t[d.B_plus]] += 1
    Bt[r, u2t[d.B_minus]] -= 1
    K[ntot:, :ntot] = Bt
    K[:ntot, ntot:] = Bt.T
    sol = np.linalg.solve(K, rhs)
    uk, info = f.solve_torn(ftil)
    np.testing.assert_allclose(info["lam"], sol[ntot:], atol=1e-8 * np.abs(sol[ntot:]).max())
    ut = np.concatenate(uk)
    np.testing.assert_allclose(ut, sol[:ntot], atol=1e-8 * np.abs(sol[:ntot]).max())
