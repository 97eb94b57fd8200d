"""The no-allocation interface apply (nlfeti_apply_schur_noalloc) against nlfeti_apply and
against the FP64 oracle's S_k^+ (pinned Neumann solve, Sec. 5.3) and S_k (Dirichlet solve,
eq. subSchurComplement) applied to the same vectors.

The file name makes pytest collect it last: it has to pass in a fresh process and after every
other GPU test, since all its calls on a device share the library's scratch array.  Each
configuration is applied twice in a row, so a second call must not depend on what the first
left in the scratch.
"""
import numpy as np
import pytest

import workloads as W
from oracle import feti as ofeti

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    from paper_2306_00094_gb300 import binding
    ctx = binding.Context()
    w = W.const_l2_2d(N=24, k=3, nrhs=3, delta=0.1)
    p = binding.Problem.from_workload(ctx, w)
    p.factor(3)
    o = ofeti.Feti(w.mesh, w.kernel, w.labels, w.K)
    yield torch, binding, p, o
    p.close()


@pytest.mark.parametrize("R", [1, 3, 9])
def test_noalloc_apply_matches_apply(setup, R):
    torch, binding, p, o = setup
    n_u = p.info()["n_u"]
    rng = np.random.default_rng(100 + R)
    X = rng.standard_normal((n_u, R))
    d_in = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()      # column-major n_u x R
    oracle_ref = {0: o.S_plus(X), 1: o.S(X)}
    for precision, tol, otol in ((0, 1e-12, 1e-9), (1, 1e-6, 1e-3)):
        for which, op in ((0, 3), (1, 4)):                          # S^+ and S
            ref = p.apply(op, precision, X)
            scale = np.abs(ref).max()
            oref = oracle_ref[which]
            assert np.abs(ref - oref).max() <= otol * np.abs(oref).max()
            for _ in range(2):
                d_out = torch.full_like(d_in, float("nan"))
                p.apply_schur_noalloc(which, precision, d_in, d_out, R)
                torch.cuda.synchronize()
                got = d_out.cpu().numpy().T
                assert np.isfinite(got).all()
                assert np.abs(got - ref).max() <= tol * scale, (precision, which, R)
                assert np.abs(got - oref).max() <= otol * np.abs(oref).max(), (precision, which, R)


def test_noalloc_apply_rejects_oversize(setup):
    torch, binding, p, o = setup
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    code = p.apply_schur_noalloc(0, 0, d, d, 10 ** 6, raise_on_error=False)
    assert code == binding.E_INVALID
    msg = p.ctx.lib.nlfeti_last_error(p.ctx.h).decode()
    assert "bytes of scratch" in msg
    assert torch.all(d == 0)
