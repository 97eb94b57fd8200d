"""Failure paths through the C ABI, each made on the host or by a bounded device wait that is
given nothing to wait for (no fault, trap or endless wait on the GPU), and each followed by a
clean solve of the same problem that matches the oracle:

* NLFETI_E_NOT_SPD: a subdomain matrix replaced by its negative (nlfeti_problem_set_matrix),
  so the first pivot of the sweep is negative; the device status word reports it, both
  precisions refuse to factor, solves are refused until a valid matrix is factored again;
* NLFETI_E_NOT_CONVERGED: the PCG iteration limit (max_it = 2, FP64 path);
* NLFETI_E_NOMEM: the allocator callback returns NULL for the solve's workspace;
* NLFETI_E_TIMEOUT: the batched interface apply's producer withholds its copies and the
  consumers' stage waits are bounded to a few thousand polls, so the first wait runs out with
  no copy in flight; the CTAs return and the error word reaches the host;
* NLFETI_E_INVALID: malformed meshes, kernels and decompositions, refused on the host.
"""
import numpy as np
import pytest

import workloads as W
from oracle import problem as oprob

pytestmark = pytest.mark.gpu


def _work():
    return W.const_l2_2d(N=24, k=3, nrhs=2, delta=0.1)


@pytest.fixture(scope="module")
def ref():
    w = _work()
    return w, oprob.Monolithic(w.mesh, w.kernel).solve(w.rhs, w.rhs_kind)


def _check(w, u, ref_u):
    assert (oprob.rel_nodal_error(u, ref_u, w.mesh, w.kernel.ncomp) <= 1e-8).all()


def test_not_spd_then_recover(ref):
    from paper_2306_00094_gb300 import binding
    w, ref_u = ref
    ctx = binding.Context()
    p = binding.Problem.from_workload(ctx, w)
    k = 4                                               # the interior (floating) subdomain
    A0 = p.operator(k, 0)
    p.set_matrix(k, -A0)
    for mask in (1, 2):
        with pytest.raises(binding.NlfetiError) as e:
            p.factor(mask)
        assert e.value.status == binding.E_NOT_SPD
    for precision in (0, 1):
        p.set_options(binding.default_options(precision=precision))
        code = ctx.lib.nlfeti_solve(p.h, 1, w.rhs_kind, np.asfortranarray(w.rhs[:, :1]).ctypes.data, None,
                                    np.zeros((p.n_dofs, 1)).ctypes.data, None)
        assert code == binding.E_INVALID                # not factored
    # a non-finite entry is refused and leaves the matrix as it was
    bad = A0.copy()
    bad[0, 0] = np.nan
    assert p.set_matrix(k, bad, raise_on_error=False) == binding.E_INVALID
    assert np.array_equal(p.operator(k, 0), -A0)
    p.set_matrix(k, A0)
    p.factor(3)
    for precision in (0, 1):
        p.set_options(binding.default_options(precision=precision))
        u, _ = p.solve(w.rhs, w.rhs_kind)
        _check(w, u, ref_u)
    p.close()
    ctx.close()


def test_not_converged_then_solves(ref):
    from paper_2306_00094_gb300 import binding
    w, ref_u = ref
    ctx = binding.Context()
    p = binding.Problem.from_workload(ctx, w)
    p.factor(1)
    p.set_options(binding.default_options(precision=0, max_it=2))
    out = np.zeros((p.n_dofs, w.nrhs), order="F")
    st = binding.Stats()
    code = ctx.lib.nlfeti_solve(p.h, w.nrhs, w.rhs_kind, np.asfortranarray(w.rhs).ctypes.data, None,
                                out.ctypes.data, st)
    assert code == binding.E_NOT_CONVERGED
    assert st.iterations <= 3 and st.final_rel_residual > 1e-10
    assert np.isfinite(out).all()
    p.set_options(binding.default_options(precision=0))
    u, s = p.solve(w.rhs, w.rhs_kind)
    _check(w, u, ref_u)
    p.close()
    ctx.close()


def test_allocator_null_then_solves(ref):
    from paper_2306_00094_gb300 import binding
    w, ref_u = ref
    state = {"ok": True, "refused": 0}

    def gate(n):
        if not state["ok"]:
            state["refused"] += 1
        return state["ok"]

    ctx = binding.Context(alloc_filter=gate)
    p = binding.Problem.from_workload(ctx, w)
    p.factor(2)
    p.set_options(binding.default_options(precision=1))
    state["ok"] = False                                 # the solve's workspace cannot be allocated
    with pytest.raises(binding.NlfetiError) as e:
        p.solve(w.rhs, w.rhs_kind)
    assert e.value.status == binding.E_NOMEM and state["refused"] >= 1
    assert "NULL" in ctx.lib.nlfeti_last_error(ctx.h).decode()
    state["ok"] = True
    u, _ = p.solve(w.rhs, w.rhs_kind)
    _check(w, u, ref_u)
    p.close()
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_apply_wait_runs_out_then_solves(ref, precision):
    from paper_2306_00094_gb300 import binding
    w, ref_u = ref
    ctx = binding.Context()
    p = binding.Problem.from_workload(ctx, w)
    p.factor(3)
    p.set_options(binding.default_options(precision=precision, batched=1, max_it=3, max_refine=1))
    p.debug_apply_waits(wait_tries=4096, withhold_copies=1)
    with pytest.raises(binding.NlfetiError) as e:
        p.solve(w.rhs, w.rhs_kind)
    assert e.value.status == binding.E_TIMEOUT
    p.debug_apply_waits(0, 0)
    p.set_options(binding.default_options(precision=precision, batched=1))
    u, _ = p.solve(w.rhs, w.rhs_kind)
    _check(w, u, ref_u)
    # a short limit alone (copies issued) still lets a solve through or reports a timeout;
    # either way the next default solve is clean
    p.debug_apply_waits(wait_tries=4096, withhold_copies=0)
    p.solve(w.rhs, w.rhs_kind, raise_on_error=False)
    p.debug_apply_waits(0, 0)
    u, _ = p.solve(w.rhs, w.rhs_kind)
    _check(w, u, ref_u)
    p.close()
    ctx.close()


def test_malformed_inputs_rejected(ref):
    """A malformed mesh, kernel or decomposition is refused on the host with NLFETI_E_INVALID and
    a message, before any device work; a valid problem on the same context then solves."""
    from paper_2306_00094_gb300 import binding
    w, ref_u = ref
    m, k = w.mesh, w.kernel
    ctx = binding.Context()

    def make(**kw):
        a = dict(dim=m.dim, xy=m.xy, elems=m.elems, node_is_dirichlet=m.node_is_dirichlet,
                 elem_is_dirichlet=m.elem_is_dirichlet, kernel_type=k.type, delta=k.delta, s=k.s,
                 scale=k.scale, labels=w.labels, K=w.K)
        a.update(kw)
        return binding.Problem(ctx, **a)

    bad_el = m.elems.copy()
    bad_el.flat[7] = m.xy.shape[0]                       # a node index past the last node
    bad_xy = m.xy.copy()
    bad_xy[3, 1] = np.inf
    bad_lab = w.labels.copy()
    bad_lab[np.flatnonzero(m.elem_is_dirichlet == 0)[0]] = w.K   # a label past the last subdomain
    gap_lab = np.where(w.labels == 2, 1, w.labels)       # subdomain 2 left empty
    cases = {"element node index out of range": dict(elems=bad_el),
             "non-finite node coordinate": dict(xy=bad_xy),
             "the Dirichlet volume constraint is empty": dict(
                 node_is_dirichlet=np.zeros_like(m.node_is_dirichlet),
                 elem_is_dirichlet=np.zeros_like(m.elem_is_dirichlet)),
             "delta must be positive": dict(delta=-k.delta),
             "unknown kernel type": dict(kernel_type=9),
             "element label out of range": dict(labels=bad_lab),
             "empty local subdomain": dict(labels=gap_lab),
             "K must be in": dict(K=0)}
    for msg, kw in cases.items():
        with pytest.raises(binding.NlfetiError) as e:
            make(**kw)
        assert e.value.status == binding.E_INVALID, msg
        assert msg in ctx.lib.nlfeti_last_error(ctx.h).decode(), msg
    p = make()
    p.factor(2)
    p.set_options(binding.default_options(precision=1))
    u, _ = p.solve(w.rhs, w.rhs_kind)
    _check(w, u, ref_u)
    p.close()
    ctx.close()
