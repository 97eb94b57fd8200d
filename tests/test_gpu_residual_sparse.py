"""The refinement residual r = f~ - A^k u - [0; B_k^T lambda] with A^k kept as a CSR of FP32
pairs or as dense FP32 pairs, both in double-single arithmetic (options.residual_format: 0
from the sparsity of A^k, 1 dense, 2 CSR):

* the CSR holds exactly the nonzeros of the assembled A^k (an integer count, bit-exact), and
  the automatic choice takes it when at most an eighth of the dense entries are nonzero;
* with either operator the mixed solve (FP32 operators + FP64 refinement) is within 1e-8 of
  the oracle's single-domain solve (eq. discreteKKT solved to the paper's tolerance), in the
  same number of refinement sweeps, and the two solutions agree to the refinement's stopping
  tolerance (refine_tol = 1e-9; the residuals differ in rounding only, a few 1e-13);
* the CSR kernel gives every (row, column) the same bits whatever the number of right-hand
  sides (one, two and three columns run different lane layouts): a batch of three solves
  column by column to the same bits.
"""
import numpy as np
import pytest

import workloads as W
from oracle import problem as oprob

pytestmark = pytest.mark.gpu

CASES = {
    "pd_3x3_jit": lambda: W.peridynamic_2d(N=30, k=3, nrhs=3, delta_cells=3, jitter=0.2),
    "pd_n48": lambda: W.peridynamic_2d(N=48, k=3, nrhs=3, delta_cells=3),
    "l2_wide": lambda: W.const_l2_2d(N=24, k=2, nrhs=3, delta=0.3),
}


@pytest.fixture(scope="module")
def ctx():
    from paper_2306_00094_gb300 import binding
    return binding.Context()


@pytest.mark.parametrize("name", list(CASES))
def test_residual_formats(ctx, name):
    from paper_2306_00094_gb300 import binding
    w = CASES[name]()
    ref = oprob.Monolithic(w.mesh, w.kernel).solve(w.rhs, w.rhs_kind)
    p = binding.Problem.from_workload(ctx, w)
    sols = {}
    for fmt in (0, 1, 2):
        p.set_options(binding.default_options(precision=1, residual_format=fmt))
        p.factor(2)
        info = p.info()
        nnz = sum(int(np.count_nonzero(p.operator(k, 0))) for k in range(info["K"]))
        csr = fmt == 2 or (fmt == 0 and 8 * nnz <= info["sum_nk2"])
        assert info["residual_nnz"] == (nnz if csr else 0), (fmt, nnz, info)
        u, st = p.solve(w.rhs, w.rhs_kind)
        assert (oprob.rel_nodal_error(u, ref, w.mesh, w.kernel.ncomp) <= 1e-8).all(), (fmt, st)
        sols[fmt] = (u, st["refine_sweeps"])
        if fmt == 2:
            for c in range(w.rhs.shape[1]):
                uc, _ = p.solve(w.rhs[:, c:c + 1], w.rhs_kind)
                assert np.array_equal(uc[:, 0], u[:, c]), (name, c)
    (ud, sd), (us, ss) = sols[1], sols[2]
    assert sd == ss
    # each stops refining once its correction is below refine_tol (1e-9): they agree to that
    assert np.abs(us - ud).max() <= 1e-9 * np.abs(ud).max()
    p.close()


def test_residual_format_validated(ctx):
    from paper_2306_00094_gb300 import binding
    w = CASES["pd_3x3_jit"]()
    p = binding.Problem.from_workload(ctx, w)
    code = ctx.lib.nlfeti_problem_set_options(p.h, binding.C.byref(binding.default_options(residual_format=3)))
    assert code == binding.E_INVALID
    p.close()
