"""The paper's baseline solver on the GPU: diagonally preconditioned CG on the single-domain
system, through the C ABI (nlfeti_solve_cg).

* the CG solution equals the oracle's single-domain FP64 Cholesky solve to the parity
  tolerance (relative nodal error <= 1e-8) on small workloads: 1-D, 2-D l2 constant, the
  Omega_k = empty fractional case, the vector peridynamic kernel (jittered parts), K = 1,
  unstructured meshes, Neumann regions, the rounded collar, the approxcaps ball;
* the 1-D quadratic with Dirichlet data is reproduced (closed form, |u - x^2/2| <= 1e-10);
* graph loop and plain launches agree bit for bit, and a column gives bitwise the same
  result alone or batched (reductions in an order independent of the batch);
* more than 32 right-hand sides are rejected (NLFETI_E_INVALID).
"""
import numpy as np
import pytest

import workloads as W
from oracle import problem as oprob

pytestmark = pytest.mark.gpu

CASES = {
    "1d_k4": lambda: W.const_1d(N=200, K=4, nrhs=2),
    "l2_3x3": lambda: W.const_l2_2d(N=24, k=3, nrhs=3, delta=0.1),
    "frac_deg": lambda: W.fractional_2d(N=24, k=3, nrhs=2, delta=0.25),
    "pd_3x3_jit": lambda: W.peridynamic_2d(N=30, k=3, nrhs=2, delta_cells=3, jitter=0.2),
    "k1": lambda: W.const_l2_2d(N=16, k=1, nrhs=2),
    "l2_unstructured": lambda: W.unstructured_l2(N=24, K=5, nrhs=2),
    "l2_neumann": lambda: W.neumann_l2(N=24, k=3, nrhs=2),
    "l2_rounded_collar": lambda: W.l2_collar_const(N=24, k=3, nrhs=2, delta=0.15),
    "frac_approxcaps": lambda: _approxcaps(W.fractional_2d(N=24, k=3, nrhs=2, delta=0.1)),
}


def _approxcaps(w):
    w.kernel.ball = 4
    return w


@pytest.fixture(scope="module")
def ctx():
    from paper_2306_00094_gb300 import binding
    return binding.Context()


def _problem(ctx, w, **opt):
    from paper_2306_00094_gb300 import binding
    p = binding.Problem.from_workload(ctx, w)
    o = binding.default_options(tol=1e-12, max_it=20000, **opt)
    p.set_options(o)
    return p


@pytest.mark.parametrize("name", list(CASES))
def test_cg_vs_single_domain_oracle(ctx, name):
    w = CASES[name]()
    p = _problem(ctx, w)
    u, st = p.solve_cg(w.rhs, w.rhs_kind, w.g)
    ref = oprob.Monolithic(w.mesh, w.kernel).solve(w.rhs, w.rhs_kind, w.g)
    err = oprob.rel_nodal_error(u, ref, w.mesh, w.kernel.ncomp)
    assert (err <= 1e-8).all(), (err, st)
    assert st["iterations"] > 0 and st["final_rel_residual"] <= 1e-12
    p.close()


def test_cg_quadratic_closed_form_1d(ctx):
    w = W.manufactured_1d_quadratic(N=400, K=4)
    p = _problem(ctx, w)
    u, st = p.solve_cg(w.rhs, w.rhs_kind, w.g)
    x = w.mesh.xy[:, 0]
    assert np.abs(u[:, 0] - 0.5 * x * x).max() < 1e-10, st
    p.close()


def test_cg_graph_eager_and_column_independence(ctx):
    from paper_2306_00094_gb300 import binding
    w = CASES["l2_3x3"]()
    p = _problem(ctx, w)
    u_graph, st_g = p.solve_cg(w.rhs, w.rhs_kind)
    p.set_options(binding.default_options(tol=1e-12, max_it=20000, batched=0))
    u_eager, st_e = p.solve_cg(w.rhs, w.rhs_kind)
    assert np.array_equal(u_graph, u_eager)
    assert st_g["iterations"] == st_e["iterations"]
    u_one, _ = p.solve_cg(w.rhs[:, 1:2], w.rhs_kind)
    assert np.array_equal(u_one[:, 0], u_graph[:, 1])
    p.close()


def test_cg_rejects_more_than_32_rhs(ctx):
    from paper_2306_00094_gb300 import binding
    w = CASES["1d_k4"]()
    p = _problem(ctx, w)
    with pytest.raises(binding.NlfetiError) as e:
        p.solve_cg(np.tile(w.rhs, (1, 17)), w.rhs_kind)
    assert e.value.status == binding.E_INVALID
    p.close()
