"""The preconditioner's S_k apply on the tensor cores (FP16 S_k scaled by a power of two, x
scaled per column by a power of two, FP32 accumulation in tensor memory), through
nlfeti_apply op 5 with precond_fp16 = 2, against the oracle's S_k (FP64 Dirichlet solves).

* elementwise error bound of an FP16 product: |y - S x| <= 1.5e-3 (|S| |x|) per entry (two
  FP16 roundings of 2^-11 each, the FP32 operator's own error and the FP32 accumulation over
  at most a few thousand terms stay below that; entries of x below 2^-14 of the column's
  largest lose bits, which the bound on |S| |x| absorbs), and the relative error is that of
  FP16 (at most 1e-3 in the Frobenius norm: a wrong tile layout or a dropped K block gives
  errors of order one);
* right-hand-side counts 1, 3, 8, 16 (N = 16), 17, 32 (N = 32), 33, 64 (N = 64) and 80 (the
  FP16 path on the FP32 pipes, which precond_fp16 = 1 selects at every count), on workloads
  whose n_gamma is below, around and well above
  the 128-row item and the 64-column stage (ragged tails in both), scalar and vector kernels;
* the FP16 copy on the FP32 pipes (precond_fp16 = 1) within the same kind of bound;
* the batched persistent launch and the per-subdomain launches give the same bits;
* op 4 (FP32 S_k) matches the oracle to 1e-5 on the same vectors (the U ordering is the
  oracle's).
"""
import numpy as np
import pytest

import workloads as W
from oracle import feti as ofeti

pytestmark = pytest.mark.gpu

CASES = {
    "l2_3x3": lambda: W.const_l2_2d(N=24, k=3, nrhs=1, delta=0.1),
    "l2_2x2_big": lambda: W.const_l2_2d(N=64, k=2, nrhs=1, delta=0.1),
    "pd_3x3": lambda: W.peridynamic_2d(N=30, k=3, nrhs=1, delta_cells=3, jitter=0.2),
    "l2_unstructured": lambda: W.unstructured_l2(N=32, K=5, nrhs=1),
}


@pytest.fixture(scope="module")
def built():
    from paper_2306_00094_gb300 import binding
    ctx = binding.Context()
    out = {}
    for name, mk in CASES.items():
        w = mk()
        p = binding.Problem.from_workload(ctx, w)
        p.factor(3)
        o = ofeti.Feti(w.mesh, w.kernel, w.labels, w.K)
        blocks = [op.S(np.eye(op.nG)) if op.nG else np.zeros((0, 0)) for op in o.ops]
        n = sum(b.shape[0] for b in blocks)
        S = np.zeros((n, n))
        off = 0
        for b in blocks:
            S[off:off + b.shape[0], off:off + b.shape[0]] = b
            off += b.shape[0]
        out[name] = (binding, p, S)
    yield out
    for _, p, _ in out.values():
        p.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("R", [1, 3, 8, 16, 17, 32, 33, 64, 80])
def test_tensor_core_apply_vs_oracle(built, name, R):
    binding, p, S = built[name]
    n = S.shape[0]
    assert p.info()["n_u"] == n
    rng = np.random.default_rng(1000 + R)
    X = rng.standard_normal((n, R))
    ref = S @ X
    bound = np.abs(S) @ np.abs(X)
    Y4 = p.apply(4, 1, X)
    assert np.abs(Y4 - ref).max() <= 1e-5 * np.abs(ref).max()
    p.set_options(binding.default_options(precision=1, precond_fp16=2))
    Y = p.apply(5, 1, X)
    assert np.isfinite(Y).all()
    assert (np.abs(Y - ref) <= 1.5e-3 * bound + 1e-300).all(), np.max(np.abs(Y - ref) / bound)
    rel = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
    assert rel <= 1e-3, rel
    p.set_options(binding.default_options(precision=1, precond_fp16=2, batched=0))
    Y_each = p.apply(5, 1, X)
    assert np.array_equal(Y, Y_each)
    p.set_options(binding.default_options(precision=1))


@pytest.mark.parametrize("name", ["l2_2x2_big"])
def test_fp16_pipes_copy_vs_oracle(built, name):
    binding, p, S = built[name]
    rng = np.random.default_rng(7)
    X = rng.standard_normal((S.shape[0], 8))
    ref = S @ X
    p.set_options(binding.default_options(precision=1, precond_fp16=1))
    Y = p.apply(5, 1, X)
    p.set_options(binding.default_options(precision=1))
    assert (np.abs(Y - ref) <= 2e-3 * (np.abs(S) @ np.abs(X)) + 1e-300).all()
