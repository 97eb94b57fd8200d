"""The factorization sweeps with their rank-64 updates on the tensor cores (factor_tc = 1:
tcgen05 kind::tf32, three-term TF32 splits of the FP32 panels, two accumulators in tensor
memory) against the FP64 oracle (eq. subSchurComplement for S_k, the pinned Neumann solve of
Sec. 5.3 for S_k^+): S_k and S_k^+ within the FP32 operators' tolerance, and the mixed solve
(FP32 operators + FP64 refinement) within 1e-8 of the oracle's single-domain solution, on
workloads with several 128-row tiles and ragged tails, floating subdomains, the vector kernel
and the Omega_k = empty degeneracy."""
import numpy as np
import pytest

import workloads as W
from oracle import feti as ofeti
from oracle import problem as oprob

pytestmark = pytest.mark.gpu

CASES = {
    "l2_4x4_n48": lambda: W.const_l2_2d(N=48, k=4, nrhs=3, delta=0.1),
    "pd_3x3_jit": lambda: W.peridynamic_2d(N=30, k=3, nrhs=2, delta_cells=3, jitter=0.2),
    "frac_deg": lambda: W.fractional_2d(N=24, k=3, nrhs=2, delta=0.25),
    "1d_k4": lambda: W.const_1d(N=400, K=4, nrhs=2),
}


@pytest.fixture(scope="module")
def ctx():
    from paper_2306_00094_gb300 import binding
    return binding.Context()


@pytest.mark.parametrize("name", list(CASES))
def test_tensor_core_factorization(ctx, name):
    from paper_2306_00094_gb300 import binding
    w = CASES[name]()
    p = binding.Problem.from_workload(ctx, w)
    p.set_options(binding.default_options(precision=1, factor_tc=1))
    p.factor(2)
    o = ofeti.Feti(w.mesh, w.kernel, w.labels, w.K)
    assert max(o.ops[k].nO + o.ops[k].nG for k in range(o.dec.K)) > 128   # several tensor-core tiles
    for k in range(o.dec.K):
        op = o.ops[k]
        if op.nG == 0:
            continue
        S_ref = op.S(np.eye(op.nG))
        Sp_ref = op.S_plus(np.eye(op.nG))
        S = p.operator(k, 1, 1)
        Sp = p.operator(k, 2, 1)
        assert np.abs(S - S_ref).max() <= 1e-4 * np.abs(S_ref).max(), (k, "S")
        assert np.abs(Sp - Sp_ref).max() <= 1e-3 * np.abs(Sp_ref).max(), (k, "S+")
    u, st = p.solve(w.rhs, w.rhs_kind)
    ref = oprob.Monolithic(w.mesh, w.kernel).solve(w.rhs, w.rhs_kind)
    assert (oprob.rel_nodal_error(u, ref, w.mesh, w.kernel.ncomp) <= 1e-8).all(), st
    p.close()
