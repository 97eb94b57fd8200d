"""Pins of the oracle's whole-element approximate balls (Fig. approximate-ball (a)-(d)):
the barycenter ball, 123vertices (at least one vertex in the disc) and 23vertices (at least
two), against facts that follow from their definitions rather than from the code:

* difference form: every row of A sums to zero, and A is symmetric;
* monotonicity: the quadratic form is an integral of a non-negative integrand over the
  selected region, and the regions are nested (23vertices within 123vertices, the nocaps
  polygon of E' within 123vertices), so v^T A v is ordered the same way for every v;
* consistency: as h -> 0 at fixed delta the selected elements approach the disc, so the
  action on x^2 at the centre tends to the local limit -2 h^2 (the same limit as nocaps),
  with an error that shrinks at every refinement (first order for 123vertices, whose
  region overshoots the disc by about one element layer: +66 %, +30 %, +14 % at delta/h =
  4, 8, 16);
* FETI with a whole-element ball equals the single-domain solve (the subdivision still
  covers every interacting pair: a selected E' lies within delta of the outer point).
"""
import numpy as np
import pytest

import workloads as W
from oracle import assembly, feti, problem

BALLS = {"barycenter": 1, "123vertices": 2, "23vertices": 3}


def _mono(N, delta, kt, ball, s=0.0):
    mesh = W.make_mesh(2, N, W.collar_cells(delta, N))
    kern = W.Kernel(kt, delta, s=s, ball=ball)
    kern.scale = W.default_scale(kern, 2)
    return mesh, kern, problem.Monolithic(mesh, kern, dense=True)


@pytest.mark.parametrize("ball", list(BALLS))
@pytest.mark.parametrize("kt,s", [(W.KERNEL_CONST_L2, 0.0), (W.KERNEL_FRACTIONAL, 0.5)])
def test_difference_form_and_symmetry(ball, kt, s):
    mesh, kern, _ = _mono(10, 0.25, kt, BALLS[ball], s)
    free = np.flatnonzero(mesh.node_is_dirichlet == 0)
    rows = assembly.assemble_rows(mesh, kern, kern.scale, free)
    sc = np.abs(rows).max()
    assert np.abs(rows.sum(axis=1)).max() <= 1e-12 * sc
    sub = rows[:, free]
    assert np.abs(sub - sub.T).max() <= 1e-13 * sc


@pytest.mark.parametrize("kt,s", [(W.KERNEL_CONST_L2, 0.0), (W.KERNEL_FRACTIONAL, 0.5)])
def test_quadratic_forms_follow_nested_regions(kt, s):
    A = {name: _mono(10, 0.25, kt, b, s)[2].A for name, b in [("nocaps", 0), *BALLS.items()]}
    rng = np.random.default_rng(4)
    for _ in range(5):
        v = rng.standard_normal(A["nocaps"].shape[0])
        q = {k: v @ M @ v for k, M in A.items()}
        tol = 1e-12 * q["123vertices"]
        assert q["23vertices"] <= q["123vertices"] + tol
        assert q["nocaps"] <= q["123vertices"] + tol
        assert min(q.values()) > 0


@pytest.mark.parametrize("ball", list(BALLS))
def test_local_limit_on_quadratics(ball):
    delta = 0.125
    errs = []
    for N in (32, 64, 128):
        mesh = W.make_mesh(2, N, W.collar_cells(delta, N))
        kern = W.Kernel(W.KERNEL_CONST_L2, delta, ball=BALLS[ball])
        kern.scale = W.default_scale(kern, 2)
        c = np.flatnonzero((np.abs(mesh.xy[:, 0] - 0.5) < 1e-12) & (np.abs(mesh.xy[:, 1] - 0.5) < 1e-12))
        rows = assembly.assemble_rows(mesh, kern, kern.scale, c)
        x = mesh.xy[:, 0]
        h = 1.0 / N
        errs.append((rows @ (x * x))[0] / (-2 * h * h) - 1.0)
    a = np.abs(errs)
    assert a[2] < a[1] < a[0] and a[2] < a[0] / 3, errs       # converges as h -> 0
    if ball == "123vertices":
        assert min(errs) > 0, errs      # a superset of the region of the nocaps rule: larger form


@pytest.mark.parametrize("ball", list(BALLS))
def test_feti_equals_single_domain(ball):
    w = W.cfg2_const_l2(N=16, k=3, nrhs=2, delta=0.15)
    w.kernel.ball = BALLS[ball]
    ref = problem.Monolithic(w.mesh, w.kernel).solve(w.rhs, w.rhs_kind)
    u, _ = feti.Feti(w.mesh, w.kernel, w.labels, w.K).solve(w.rhs, w.rhs_kind)
    assert (problem.rel_nodal_error(u, ref, w.mesh, 1) <= 1e-9).all()
