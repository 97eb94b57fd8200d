"""The autotuner of the batched interface apply (nlfeti_autotune / nlfeti_set_apply_choice):

* every candidate shape (right-hand sides per streamed pass 1..16, one or two CTAs per SM, 4 or
  8 rows per consumer warp) gives bitwise the same S_k^+ and S_k products, in both precisions
  and for the FP16 preconditioner copy, with ragged right-hand-side counts (9 and 17);
* the tuner keeps a valid shape per operator kind (for the FP16 preconditioner copy possibly the
  tensor-core apply), writes its choices to the JSON cache, and a second call reads them back
  without timing;
* a solve after tuning gives bitwise the solution of the untuned solve (to 1e-8 when the
  tensor-core preconditioner was chosen, which steers the PCG differently);
* shapes outside the lists are refused.
"""
import json

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

R = 9


@pytest.fixture(scope="module")
def prob():
    from paper_2306_00094_gb300 import binding
    ctx = binding.Context()
    w = W.const_l2_2d(N=32, k=4, nrhs=R, delta=0.1)
    p = binding.Problem.from_workload(ctx, w)
    p.factor(3)
    yield binding, w, p
    p.close()


@pytest.mark.parametrize("nrhs", [R, 17])
def test_every_shape_gives_the_same_products(prob, nrhs):
    binding, w, p = prob
    n_u = p.info()["n_u"]
    X = np.random.default_rng(3).standard_normal((n_u, nrhs))
    for kind, precision, ops in ((0, 1, (3, 4)), (2, 0, (3, 4)), (1, 1, (5,))):
        p.set_options(binding.default_options(precision=precision, batched=1, precond_fp16=1))
        refs = {op: p.apply(op, precision, X) for op in ops}
        for rc in (1, 2, 4, 8, 16):
            if rc > nrhs or (kind == 2 and rc > 8):
                assert p.set_apply_choice(kind, nrhs, rc, 2, raise_on_error=False) == binding.E_INVALID
                continue
            for per_sm in (1, 2):
                for rpw in (4, 8):
                    if rpw == 8 and (kind == 2 or rc < 4):
                        assert p.set_apply_choice(kind, nrhs, rc, per_sm, rpw,
                                                  raise_on_error=False) == binding.E_INVALID
                        continue
                    p.set_apply_choice(kind, nrhs, rc, per_sm, rpw)
                    for op in ops:
                        assert np.array_equal(p.apply(op, precision, X), refs[op]), (kind, rc, per_sm, rpw, op)
        p.set_apply_choice(kind, nrhs, 0)
    assert p.set_apply_choice(0, R, 3, 2, raise_on_error=False) == binding.E_INVALID
    assert p.set_apply_choice(0, R, 4, 3, raise_on_error=False) == binding.E_INVALID
    assert p.set_apply_choice(0, R, 4, 2, 6, raise_on_error=False) == binding.E_INVALID


def test_tuner_cache_and_solution(prob, tmp_path):
    binding, w, p = prob
    p.set_options(binding.default_options(precision=1, batched=1))
    u0, _ = p.solve(w.rhs, w.rhs_kind)
    path = str(tmp_path / "tune.json")
    first = p.autotune(R, path)
    assert sorted(e["kind"] for e in first) == [0, 1, 2]
    for e in first:
        assert e["nrhs"] == R and e["from_cache"] == 0 and e["us"] > 0
        if e["kind"] == 1 and e["rc"] == -1:           # the tensor-core preconditioner apply
            continue
        assert e["rc"] in (1, 2, 4, 8, 16) and e["rc"] <= R and e["ctas_per_sm"] in (1, 2)
        assert e["rows_per_warp"] == 4 or (e["rows_per_warp"] == 8 and e["kind"] < 2 and e["rc"] >= 4)
    doc = json.load(open(path))
    assert len(doc["entries"]) == 3
    again = p.autotune(R, path)
    assert all(e["from_cache"] == 1 for e in again)
    assert sorted((e["kind"], e["rc"], e["ctas_per_sm"], e["rows_per_warp"]) for e in again) == \
        sorted((e["kind"], e["rc"], e["ctas_per_sm"], e["rows_per_warp"]) for e in first)
    u1, _ = p.solve(w.rhs, w.rhs_kind)
    if any(e["kind"] == 1 and e["rc"] == -1 for e in first):
        # the tensor-core preconditioner steers the PCG differently: the same accuracy
        assert np.abs(u1 - u0).max() <= 1e-8 * np.abs(u0).max()
    else:
        assert np.array_equal(u0, u1)
    # the tensor-core preconditioner pinned by hand: a solve of the same accuracy
    p.set_apply_choice(1, R, -1)
    u2, _ = p.solve(w.rhs, w.rhs_kind)
    assert np.abs(u2 - u0).max() <= 1e-8 * np.abs(u0).max()
    assert p.set_apply_choice(0, R, -1, raise_on_error=False) == binding.E_INVALID
    for kind in (0, 1, 2):
        p.set_apply_choice(kind, R, 0)
