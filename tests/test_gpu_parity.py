"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

* decomposition, index maps and B: bit-exact;
* assembled subdomain matrices A^k: <= 1e-12 relative (same quadrature rule, two codes);
* S_k, S_k^+ (FP64 operators): <= 1e-9 relative to the oracle's Dirichlet / pinned
  Neumann solves; the FP32 operators within their rounding (1e-4 relative);
* F, M^-1, P applied to random vectors (FP64 operators): <= 1e-9;
* end to end: relative nodal error vs the oracle's single-domain solve <= 1e-8 for the
  FP64 path and for the mixed path after refinement (the tolerance of the paper's solver
  target), on small workloads spanning several tiles with ragged tails, floating
  subdomains, the Omega_k = empty degeneracy, the vector kernel, K = 1, unstructured
  meshes (irregular nodes and diagonals) with graph-grown local parts, the whole-element
  approximate balls (barycenter, 123vertices, 23vertices), the approxcaps ball (cap
  triangles on the nocaps polygon; structured and unstructured), Neumann volume constraints
  (a free, loaded collar region on two sides), the l2 (rounded-corner) collar, and 81
  subdomains (subdomain masks of more than one 64-bit word).
"""
import numpy as np
import pytest

import workloads as W
from oracle import feti as ofeti
from oracle import problem as oprob

pytestmark = pytest.mark.gpu

CASES = {
    "1d_k4": lambda: W.const_1d(N=200, K=4, nrhs=2),
    "l2_3x3": lambda: W.const_l2_2d(N=24, k=3, nrhs=3, delta=0.1),
    "linf_2x2": lambda: W.Workload("linf", *_linf(20, 2)),
    "frac_3x3": lambda: W.fractional_2d(N=24, k=3, nrhs=2, delta=0.1),
    "frac_deg": lambda: W.fractional_2d(N=24, k=3, nrhs=2, delta=0.25),
    "pd_3x3_jit": lambda: W.peridynamic_2d(N=30, k=3, nrhs=2, delta_cells=3, jitter=0.2),
    "k1": lambda: W.const_l2_2d(N=16, k=1, nrhs=2),
    "l2_unstructured": lambda: W.unstructured_l2(N=24, K=5, nrhs=2),
    "pd_unstructured": lambda: W.unstructured_pd(N=24, K=4, nrhs=2),
    "l2_ball_barycenter": lambda: _ball(W.const_l2_2d(N=24, k=3, nrhs=2, delta=0.1), 1),
    "frac_ball_123v": lambda: _ball(W.fractional_2d(N=24, k=3, nrhs=2, delta=0.1), 2),
    "pd_ball_23v": lambda: _ball(W.peridynamic_2d(N=30, k=3, nrhs=2, delta_cells=3, jitter=0.2), 3),
    "l2_approxcaps": lambda: _ball(W.const_l2_2d(N=24, k=3, nrhs=2, delta=0.1), 4),
    "frac_approxcaps": lambda: _ball(W.fractional_2d(N=24, k=3, nrhs=2, delta=0.1), 4),
    "pd_approxcaps": lambda: _ball(W.peridynamic_2d(N=30, k=3, nrhs=2, delta_cells=3, jitter=0.2), 4),
    "l2_unstructured_approxcaps": lambda: _ball(W.unstructured_l2(N=24, K=5, nrhs=2), 4),
    "l2_neumann": lambda: W.neumann_l2(N=24, k=3, nrhs=2),
    "pd_neumann": lambda: W.neumann_pd(N=30, k=3, nrhs=2),
    "l2_rounded_collar": lambda: W.l2_collar_const(N=24, k=3, nrhs=2, delta=0.15),
    "l2_9x9": lambda: W.const_l2_2d(N=36, k=9, nrhs=2, delta=2.0 / 36),   # K = 81: more than 64 subdomains
    "pd_9x9": lambda: W.peridynamic_2d(N=36, k=9, nrhs=2),   # 147 rigid modes: coarse matrix past 128
}


def _ball(w, ball):
    w.kernel.ball = ball
    return w


def _linf(N, k):
    delta = 2.0 / N
    mesh = W.make_mesh(2, N, W.collar_cells(delta, N))
    kern = W.Kernel(W.KERNEL_CONST_LINF, delta)
    kern.scale = W.default_scale(kern, 2)
    labels = W.rect_labels(mesh, k, k)
    rhs = W.nodal_loads(mesh, 1, 2, 11, "normal")
    return mesh, kern, labels, k * k, rhs, 1


@pytest.fixture(scope="module")
def ctx():
    from paper_2306_00094_gb300 import binding
    return binding.Context()


@pytest.fixture(scope="module")
def built(ctx):
    from paper_2306_00094_gb300 import binding
    out = {}
    for name, mk in CASES.items():
        w = mk()
        p = binding.Problem.from_workload(ctx, w)
        p.factor(3)
        o = ofeti.Feti(w.mesh, w.kernel, w.labels, w.K)
        out[name] = (w, p, o)
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_decomposition_bit_exact(built, name):
    w, p, o = built[name]
    d = p.decomposition()
    dec = o.dec
    assert list(d["n_k"]) == [dec.dofs(k).size for k in range(dec.K)]
    assert list(d["n_gamma"]) == [dec.n_gamma(k) for k in range(dec.K)]
    assert np.array_equal(d["nodes"], np.concatenate([s.nodes for s in dec.subs]))
    assert np.array_equal(d["B_plus"], dec.B_plus) and np.array_equal(d["B_minus"], dec.B_minus)
    assert np.array_equal(d["floating"].astype(bool), dec.floating)


@pytest.mark.parametrize("name", list(CASES))
def test_assembled_matrices(built, name):
    w, p, o = built[name]
    for k in range(o.dec.K):
        A = p.operator(k, 0)
        ref = o.A[k]
        assert np.abs(A - ref).max() <= 1e-12 * np.abs(ref).max(), (k, np.abs(A - ref).max())
        assert np.array_equal(A, A.T)


@pytest.mark.parametrize("name", list(CASES))
def test_schur_and_pseudo_inverse(built, name):
    w, p, o = built[name]
    for k in range(o.dec.K):
        op = o.ops[k]
        if op.nG == 0:
            continue
        S_ref = op.S(np.eye(op.nG))
        Sp_ref = op.S_plus(np.eye(op.nG))
        for prec, tol in [(0, 1e-9), (1, 1e-4)]:
            S = p.operator(k, 1, prec)
            Sp = p.operator(k, 2, prec)
            assert np.abs(S - S_ref).max() <= tol * np.abs(S_ref).max(), (k, prec, "S")
            assert np.abs(Sp - Sp_ref).max() <= tol * 10 * np.abs(Sp_ref).max(), (k, prec, "S+")


@pytest.mark.parametrize("name", [n for n in CASES if n != "k1"])
def test_feti_operators(built, name):
    w, p, o = built[name]
    rng = np.random.default_rng(5)
    nl = o.dec.n_lambda
    X = rng.standard_normal((nl, 3))
    for op, ref in [(0, o.F), (1, o.Minv), (2, o.P)]:
        Y = p.apply(op, 0, X)
        R = ref(X)
        assert np.abs(Y - R).max() <= 1e-9 * max(np.abs(R).max(), 1e-300), (op, np.abs(Y - R).max())


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [0, 1])
def test_end_to_end_vs_oracle(built, name, precision):
    from paper_2306_00094_gb300 import binding
    w, p, o = built[name]
    mono = oprob.Monolithic(w.mesh, w.kernel)
    ref = mono.solve(w.rhs, w.rhs_kind, w.g)
    p.set_options(binding.default_options(precision=precision))
    u, st = p.solve(w.rhs, w.rhs_kind, w.g)
    err = oprob.rel_nodal_error(u, ref, w.mesh, w.kernel.ncomp)
    assert (err <= 1e-8).all(), (err, st)


def test_quadratic_closed_form_1d_on_gpu(ctx):
    from paper_2306_00094_gb300 import binding
    w = W.manufactured_1d_quadratic(N=400, K=4)
    p = binding.Problem.from_workload(ctx, w)
    p.factor(1)
    u, st = p.solve(w.rhs, w.rhs_kind, w.g)
    x = w.mesh.xy[:, 0]
    assert np.abs(u[:, 0] - 0.5 * x * x).max() < 1e-10


def test_approxcaps_rejects_short_horizon(ctx):
    from paper_2306_00094_gb300 import binding
    w = _ball(W.const_l2_2d(N=24, k=2, nrhs=1, delta=0.02), 4)     # 2 delta < the diagonal h sqrt(2)
    with pytest.raises(binding.NlfetiError) as e:
        binding.Problem.from_workload(ctx, w)
    assert e.value.status == binding.E_INVALID


def test_empty_and_invalid_requests_rejected(ctx):
    """Zero right-hand sides and an unknown load kind are refused with NLFETI_E_INVALID by the
    FETI solve, the CG solve and the operator apply; the problem stays usable afterwards."""
    from paper_2306_00094_gb300 import binding
    w = W.const_l2_2d(N=16, k=2, nrhs=1)
    p = binding.Problem.from_workload(ctx, w)
    p.factor(3)
    empty = np.zeros((w.rhs.shape[0], 0), order="F")
    for call in (lambda: p.solve(empty, w.rhs_kind), lambda: p.solve(w.rhs, 2),
                 lambda: p.solve_cg(empty, w.rhs_kind), lambda: p.apply(0, 0, np.zeros((p.info()["n_lambda"], 0)))):
        with pytest.raises(binding.NlfetiError) as e:
            call()
        assert e.value.status == binding.E_INVALID
    u, st = p.solve(w.rhs, w.rhs_kind)
    assert np.isfinite(u).all() and st["iterations"] > 0
    p.close()
