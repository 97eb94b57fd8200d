"""Serving: requests of different problems, sizes and right-hand-side counts run concurrently
(slots on their own streams) and requests on the same problem share batched solves
(continuous batching); each result equals the same request solved alone, bitwise.  The
server's device bytes stay within its HBM budget; requests given by their inputs go through
the factorization cache (created and factored once per key, evicted least recently used
first when the budget needs the room).  Failure handling is exercised on the host:
over-budget admission, invalid inputs and a wait that times out."""
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
    order = [0, 1, 2, 3, 1, 0, 3, 2, 1, 1, 1, 2, 0, 1]
    tickets = [(i, srv.submit(probs[i], work[i].rhs, work[i].rhs_kind)) for i in order]
    for i, t in tickets:
        u, st = srv.wait(t, timeout_ms=120000)
        assert np.array_equal(u, alone[i]), (i, np.abs(u - alone[i]).max())
    inf = srv.info()
    srv.close()
    # the requests overlapped on the device, and some ran in shared batches
    assert inf["requests_done"] == len(order)
    assert inf["peak_active"] >= 2
    assert inf["merged_requests"] >= 2 and inf["batches"] < len(order)
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


def test_budget_holds_with_slots_and_odd_counts(setup):
    """The server's device bytes (workspaces in use and kept) never exceed its budget."""
    from paper_2306_00094_gb300 import binding
    ctx, work, probs = setup
    budget = 24 << 20
    srv = binding.Server(ctx, hbm_budget=budget, max_slots=4)
    reqs = []
    for R in (1, 3, 5, 7, 9, 11, 2, 13):
        for i in (0, 1, 2):
            rhs = np.asfortranarray(np.tile(work[i].rhs, (1, 16))[:, :R])
            reqs.append((i, rhs, srv.submit(probs[i], rhs, work[i].rhs_kind)))
    for i, rhs, t in reqs:
        u, _ = srv.wait(t, timeout_ms=120000)
        u_direct, _ = probs[i].solve(rhs, work[i].rhs_kind)
        assert np.abs(u - u_direct).max() <= 1e-12 * np.abs(u_direct).max()
    inf = srv.info()
    srv.close()
    assert 0 < inf["peak_bytes"] <= budget, inf


def test_factorization_cache_by_inputs(setup):
    """Requests given by their inputs: created and factored once per key, reused after."""
    from paper_2306_00094_gb300 import binding
    ctx, work, probs = setup
    opt = binding.default_options(precision=1)
    srv = binding.Server(ctx, max_slots=2)
    a, b = work[1], work[2]
    ta = srv.submit_workload(a, opt=opt)
    ua, sa = srv.wait(ta, timeout_ms=120000)
    assert sa["ms_factor"] > 0.0                       # a miss: created and factored here
    for _ in range(2):
        u, s = srv.wait(srv.submit_workload(a, opt=opt), timeout_ms=120000)
        assert np.array_equal(u, ua) and s["ms_factor"] == 0.0
    ub, _ = srv.wait(srv.submit_workload(b, opt=opt), timeout_ms=120000)
    inf = srv.info()
    srv.close()
    assert inf["problem_misses"] == 2 and inf["problem_hits"] == 2 and inf["problems_cached"] == 2
    for w, u in ((a, ua), (b, ub)):
        ref = oprob.Monolithic(w.mesh, w.kernel).solve(w.rhs, w.rhs_kind)
        assert (oprob.rel_nodal_error(u, ref, w.mesh, w.kernel.ncomp) <= 1e-8).all()


def test_factorization_cache_evicts_within_budget(setup):
    """With room for one cached problem only, alternating keys evict the idle one and the
    server's bytes stay within the budget."""
    from paper_2306_00094_gb300 import binding
    ctx, work, probs = setup
    opt = binding.default_options(precision=1)
    a = W.const_l2_2d(N=48, k=3, nrhs=2, delta=0.1)
    b = W.const_l2_2d(N=48, k=4, nrhs=2, delta=0.1)
    alone = {}
    for name, w in (("a", a), ("b", b)):
        srv = binding.Server(ctx, max_slots=1)
        u, _ = srv.wait(srv.submit_workload(w, opt=opt), timeout_ms=120000)
        alone[name] = (u, srv.info()["peak_bytes"])
        srv.close()
    pa, pb = alone["a"][1], alone["b"][1]
    budget = max(pa, pb) + min(pa, pb) // 2           # one problem with its workspace, not two
    srv = binding.Server(ctx, hbm_budget=budget, max_slots=1)
    for name, w in (("a", a), ("b", b), ("a", a), ("b", b)):
        u, _ = srv.wait(srv.submit_workload(w, opt=opt), timeout_ms=120000)
        # a re-created problem is assembled again (FP64 atomics: summation order may differ)
        ref = alone[name][0]
        assert np.abs(u - ref).max() <= 1e-10 * np.abs(ref).max()
    inf = srv.info()
    srv.close()
    assert inf["problem_misses"] == 4 and inf["problems_evicted"] >= 3
    assert inf["peak_bytes"] <= budget


def test_invalid_inputs_fail_the_request(setup):
    from paper_2306_00094_gb300 import binding
    ctx, work, probs = setup
    w = W.const_l2_2d(N=16, k=2, nrhs=1, delta=0.1)
    w.K = 0                                             # no local parts
    srv = binding.Server(ctx, max_slots=1)
    t = srv.submit_workload(w)
    with pytest.raises(binding.NlfetiError) as e:
        srv.wait(t, timeout_ms=60000)
    assert e.value.status == binding.E_INVALID
    u, _ = srv.wait(srv.submit(probs[1], work[1].rhs, work[1].rhs_kind), timeout_ms=60000)
    assert np.isfinite(u).all()
    srv.close()
