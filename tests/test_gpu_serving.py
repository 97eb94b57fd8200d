"""Serving: requests of different problems, sizes and right-hand-side counts run concurrently
(continuous batching across slots), and each result equals the same request solved alone.
Failure handling is exercised on the host: over-budget admission and a wait that times out."""
import numpy as np
import pytest

import workloads as W
from oracle import problem as oprob

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2306_00094_gb300 import binding
    ctx = binding.Context()
    work = [W.const_1d(N=300, K=4, nrhs=3), W.const_l2_2d(N=32, k=4, nrhs=5, delta=0.1),
            W.fractional_2d(N=24, k=3, nrhs=2, delta=0.1), W.peridynamic_2d(N=24, k=3, nrhs=1, jitter=0.2)]
    probs = []
    for w in work:
        p = binding.Problem.from_workload(ctx, w)
        p.factor(2)
        p.set_options(binding.default_options(precision=1))
        probs.append(p)
    return ctx, work, probs


def test_alone_equals_mix(setup):
    from paper_2306_00094_gb300 import binding
    ctx, work, probs = setup
    alone = []
    srv1 = binding.Server(ctx, max_slots=1)
    for w, p in zip(work, probs):
        t = srv1.submit(p, w.rhs, w.rhs_kind)
        alone.append(srv1.wait(t)[0])
    srv1.close()
    srv = binding.Server(ctx, max_slots=4)
    order = [0, 1, 2, 3, 1, 0, 3, 2, 1, 1]
    tickets = [(i, srv.submit(probs[i], work[i].rhs, work[i].rhs_kind)) for i in order]
    for i, t in tickets:
        u, st = srv.wait(t, timeout_ms=120000)
        assert np.array_equal(u, alone[i]), (i, np.abs(u - alone[i]).max())
    srv.close()
    for w, u in zip(work, alone):
        ref = oprob.Monolithic(w.mesh, w.kernel).solve(w.rhs, w.rhs_kind)
        assert (oprob.rel_nodal_error(u, ref, w.mesh, w.kernel.ncomp) <= 1e-8).all()


def test_admission_rejects_oversize_request(setup):
    from paper_2306_00094_gb300 import binding
    ctx, work, probs = setup
    srv = binding.Server(ctx, hbm_budget=1 << 16, max_slots=2)
    with pytest.raises(binding.NlfetiError) as e:
        srv.submit(probs[1], work[1].rhs, work[1].rhs_kind)
    assert e.value.status == binding.E_NOMEM
    srv.close()


def test_wait_times_out_then_completes(setup):
    from paper_2306_00094_gb300 import binding
    ctx, work, probs = setup
    srv = binding.Server(ctx, max_slots=1)
    big = np.tile(work[1].rhs, (1, 8))
    t1 = srv.submit(probs[1], big, 1)
    t2 = srv.submit(probs[1], big, 1)
    with pytest.raises(binding.NlfetiError) as e:
        srv.wait(t2, timeout_ms=0)
    assert e.value.status == binding.E_TIMEOUT
    u1, _ = srv.wait(t1)
    u2, _ = srv.wait(t2)
    assert np.array_equal(u1, u2)
    srv.close()


def test_server_matches_direct_solve_for_odd_rhs_counts(setup):
    """The server rounds right-hand-side counts up to bucket sizes (zero columns) and keeps
    workspaces per (problem, count); results equal the direct solve of the same columns."""
    from paper_2306_00094_gb300 import binding
    ctx, work, probs = setup
    w, p = work[1], probs[1]
    srv = binding.Server(ctx, max_slots=2)
    for R in (1, 3, 5, 3, 5):
        rhs = np.asfortranarray(np.tile(w.rhs, (1, 2))[:, :R])
        u_direct, _ = p.solve(rhs, w.rhs_kind)
        u_srv, st = srv.wait(srv.submit(p, rhs, w.rhs_kind), timeout_ms=120000)
        assert u_srv.shape == u_direct.shape
        assert np.abs(u_srv - u_direct).max() <= 1e-12 * np.abs(u_direct).max()
        assert st["ms_queue"] >= 0.0
    srv.close()
