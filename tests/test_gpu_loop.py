"""The three ways the PCG loop of a pass can run give the same solution.

* batched, no profiling: the loop is one cached graph with a device-side WHILE node;
* batched, profiling on or graph_loop = 0: graphs of 4 iterations (event-timed applies when
  profiling) with host checks in between;
* not batched: one launch per subdomain per stage, no graphs.

The arithmetic of every iteration is the same in all three (inactive right-hand sides are
frozen by their flags), so the graph loop and the chunked loop must agree bit for bit, and
the per-subdomain launches (same kernels on subsets of the work items) as well.  The cached
graph must follow a refactorization and option changes.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2306_00094_gb300 import binding
    ctx = binding.Context()
    w = W.const_l2_2d(N=24, k=3, nrhs=3, delta=0.1)
    p = binding.Problem.from_workload(ctx, w)
    p.factor(3)
    yield binding, w, p
    p.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_while_chunked_eager_agree(setup, precision):
    binding, w, p = setup
    p.set_options(binding.default_options(precision=precision, batched=1))
    u_while, st_w = p.solve(w.rhs, w.rhs_kind)
    u_again, _ = p.solve(w.rhs, w.rhs_kind)              # cached graph reused
    assert np.array_equal(u_while, u_again)
    p.profile()
    p.set_profiling(True)
    u_chunk, st_c = p.solve(w.rhs, w.rhs_kind)
    p.set_profiling(False)
    prof = p.profile()
    assert prof["apply_launches"] > 0 and prof["apply_ms"] > 0 and prof["kernel_launches"] > 0
    assert np.array_equal(u_while, u_chunk)
    assert st_w["iterations"] == st_c["iterations"]
    p.set_options(binding.default_options(precision=precision, batched=1, graph_loop=0))
    u_host, st_h = p.solve(w.rhs, w.rhs_kind)
    assert np.array_equal(u_while, u_host)
    assert st_w["iterations"] == st_h["iterations"]
    p.set_options(binding.default_options(precision=precision, batched=0))
    u_eager, st_e = p.solve(w.rhs, w.rhs_kind)
    assert np.array_equal(u_while, u_eager)
    assert st_w["iterations"] == st_e["iterations"]


def test_graph_follows_refactor_and_options(setup):
    binding, w, p = setup
    p.set_options(binding.default_options(precision=1, batched=1))
    u1, _ = p.solve(w.rhs, w.rhs_kind)
    p.factor(2)                                            # operator buffers are rebuilt
    u2, _ = p.solve(w.rhs, w.rhs_kind)
    assert np.array_equal(u1, u2)
    loose = binding.default_options(precision=1, batched=1)
    loose.inner_tol = 1e-2
    p.set_options(loose)
    u3, st3 = p.solve(w.rhs, w.rhs_kind)
    scale = np.abs(u1).max()
    assert np.abs(u3 - u1).max() <= 1e-8 * scale
    p.set_options(binding.default_options(precision=1, batched=1))
    u4, _ = p.solve(w.rhs, w.rhs_kind)
    assert np.array_equal(u1, u4)


def test_launch_count_of_graph_loop(setup):
    binding, w, p = setup
    p.set_options(binding.default_options(precision=1, batched=1))
    p.solve(w.rhs, w.rhs_kind)
    p.profile()
    _, st = p.solve(w.rhs, w.rhs_kind)
    n = p.profile()["kernel_launches"]
    # at least the interface applies of every iteration (two per iteration) were counted
    assert n >= 2 * st["iterations"]


def test_fp16_preconditioner_reaches_the_same_accuracy(setup):
    """The 16-bit copies of S_k (BF16 on the tensor cores, FP16 on the FP32 pipes) only steer
    the PCG: with them and without them the mixed path reaches the oracle's solution to the
    same tolerance (the refinement fixes the fixed point) in about as many iterations."""
    from oracle import problem as oprob
    binding, w, p = setup
    ref = oprob.Monolithic(w.mesh, w.kernel).solve(w.rhs, w.rhs_kind)
    out = {}
    for fp16 in (0, 1, 2):
        p.set_options(binding.default_options(precision=1, precond_fp16=fp16))
        u, st = p.solve(w.rhs, w.rhs_kind)
        assert (oprob.rel_nodal_error(u, ref, w.mesh, w.kernel.ncomp) <= 1e-8).all()
        out[fp16] = (u, st)
    scale = np.abs(out[0][0]).max()
    for fp16 in (1, 2):
        assert np.abs(out[fp16][0] - out[0][0]).max() <= 1e-8 * scale
        assert abs(out[fp16][1]["iterations"] - out[0][1]["iterations"]) <= max(3, out[0][1]["iterations"] // 5)


@pytest.mark.parametrize("precision", [0, 1])
def test_columns_bitwise_independent_of_batch_size(setup, precision):
    """Every kernel treats a column the same whatever batch it is part of; the Lambda
    reductions sum it over the same rows in the same tree in the coalesced layout (up to 8
    columns) and in the one-column-per-block layout (more columns).  So one right-hand side
    solved alone, in a batch of 8 and in a batch of 9 identical columns (the same iterations
    and sweeps) gives bitwise the same solution."""
    binding, w, p = setup
    p.set_options(binding.default_options(precision=precision))
    col = np.asfortranarray(w.rhs[:, :1])
    u1, s1 = p.solve(col, w.rhs_kind)
    u8, s8 = p.solve(np.asfortranarray(np.tile(col, (1, 8))), w.rhs_kind)
    u9, s9 = p.solve(np.asfortranarray(np.tile(col, (1, 9))), w.rhs_kind)
    assert s1["iterations"] == s8["iterations"] == s9["iterations"]
    for u in (u8, u9):
        for c in range(u.shape[1]):
            assert np.array_equal(u[:, c], u1[:, 0]), (u.shape[1], c, np.abs(u[:, c] - u1[:, 0]).max())
