"""Pins of the oracle's other approximate balls (Fig. approximate-ball): the whole-element
balls (a)-(d) -- barycenter, 123vertices (at least one vertex in the disc), 23vertices (at
least two) -- and approxcaps (f), the nocaps polygon with each left-out cap replaced by the
triangle on its chord and arc midpoint, against facts that follow from their definitions
rather than from the code:

* cap geometry (approxcaps): for a single inner element and outer point, the region's area
  (read off the inner integral of the constant kernel, whose integrand is c on disjoint
  elements for the indicator of the inner nodes) lies between the nocaps area and the exact
  area of disc cap E' (computed independently by adaptive quadrature in polar angle), and
  the area still missing is the fraction 1 - sin(phi)(1 - cos(phi)) / (phi - sin(phi) cos(phi))
  of each cap of half-angle phi: 1/4 for small caps, at most 0.2548 when the chord is at most
  delta / 1.41 -- including a circle that enters and leaves E' through one edge (nocaps:
  nothing; approxcaps: the lone cap triangle);

* difference form: every row of A sums to zero, and A is symmetric;
* monotonicity: the quadratic form is an integral of a non-negative integrand over the
  selected region, and the regions are nested (23vertices within 123vertices, the nocaps
  polygon of E' within 123vertices), so v^T A v is ordered the same way for every v;
* consistency: as h -> 0 at fixed delta the selected elements approach the disc, so the
  action on x^2 at the centre tends to the local limit -2 h^2 (the same limit as nocaps),
  with an error that shrinks at every refinement (first order for 123vertices, whose
  region overshoots the disc by about one element layer: +66 %, +30 %, +14 % at delta/h =
  4, 8, 16); the approxcaps error is 1/4 of the nocaps error (the caps' share of the
  second moment, all at radius delta, shrinks to 1/4 as well) and falls as h^2;
* FETI with a whole-element ball equals the single-domain solve (the subdivision still
  covers every interacting pair: a selected E' lies within delta of the outer point).
"""
import numpy as np
import pytest
from scipy.integrate import quad

import workloads as W
from oracle import assembly, feti, problem

BALLS = {"barycenter": 1, "123vertices": 2, "23vertices": 3, "approxcaps": 4}


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
        assert q["nocaps"] <= q["approxcaps"] + tol
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
    w = W.const_l2_2d(N=16, k=3, nrhs=2, delta=0.15)
    w.kernel.ball = BALLS[ball]
    ref = problem.Monolithic(w.mesh, w.kernel).solve(w.rhs, w.rhs_kind)
    u, _ = feti.Feti(w.mesh, w.kernel, w.labels, w.K).solve(w.rhs, w.rhs_kind)
    assert (problem.rel_nodal_error(u, ref, w.mesh, 1) <= 1e-9).all()


def _disc_triangle_area(T, x, d):
    """Exact area of the closed disc |y - x| <= d intersected with triangle T: the sum over the
    edges of the signed areas of disc cap triangle(x, A, B), each the integral over the polar
    angle of min(rho, d)^2 / 2 with rho the distance from x to the edge's line."""
    tot = 0.0
    for k in range(3):
        A, B = T[k] - x, T[(k + 1) % 3] - x
        ta = np.arctan2(A[1], A[0])
        dth = (np.arctan2(B[1], B[0]) - ta + np.pi) % (2 * np.pi) - np.pi
        e = B - A
        nrm = np.array([e[1], -e[0]]) / np.hypot(e[0], e[1])
        p = float(A @ nrm)
        if p < 0:
            nrm, p = -nrm, -p
        if p == 0.0 or dth == 0.0:
            continue
        tn = np.arctan2(nrm[1], nrm[0])
        kinks = []
        if p < d:
            for sg in (-1.0, 1.0):
                u = (tn + sg * np.arccos(p / d) - ta + np.pi) % (2 * np.pi) - np.pi
                if 0.0 < u / dth < 1.0:
                    kinks.append(u)
        lo, hi = (0.0, dth) if dth > 0 else (dth, 0.0)
        v, _ = quad(lambda t: 0.5 * min(p / np.cos(ta + t - tn), d) ** 2, lo, hi,
                    points=sorted(kinks) or None, epsabs=1e-16, epsrel=1e-13, limit=200)
        tot += v if dth > 0 else -v
    return abs(tot)


def _region_area(mesh, delta, ball, e, ep, x):
    M, nodes = assembly.point_integral(mesh, W.Kernel(W.KERNEL_CONST_L2, delta, ball=ball), 1.0, e, ep, x)
    assert len(nodes) == 6          # disjoint pair: the inner nodes have zero outer values
    s = np.r_[np.zeros(3), np.ones(3)]
    return float(s @ M @ s)


@pytest.mark.parametrize("meshkind", ["structured", "unstructured"])
def test_approxcaps_cap_geometry(meshkind):
    N, rng = 20, np.random.default_rng(7)
    h = 1.0 / N
    delta = 2.5 * h
    if meshkind == "structured":
        mesh = W.make_mesh(2, N, W.collar_cells(delta, N))
    else:
        mesh = W.unstructured_mesh(N, W.collar_cells(delta, N), seed=3)
    cen_all = mesh.xy[mesh.elems].mean(axis=1)
    diam = max(np.linalg.norm(mesh.xy[mesh.elems[:, i]] - mesh.xy[mesh.elems[:, (i + 1) % 3]], axis=1).max()
               for i in range(3))
    assert 2 * delta > diam          # every arc inside an element is a minor arc
    checked = dips = 0
    for trial in range(60):
        ep = int(rng.integers(mesh.n_elems))
        T = mesh.xy[mesh.elems[ep]]
        e = int(np.flatnonzero(np.abs(cen_all - T.mean(0)).max(axis=1) > 4 * h)[0])
        if trial % 3 == 0:
            # the circle dips into E' through one edge only
            k = int(rng.integers(3))
            A, B, C = T[k], T[(k + 1) % 3], T[(k + 2) % 3]
            nrm = np.array([B[1] - A[1], A[0] - B[0]]) / np.linalg.norm(B - A)
            if (C - 0.5 * (A + B)) @ nrm > 0:
                nrm = -nrm
            x = 0.5 * (A + B) + nrm * (delta - rng.uniform(0.002, 0.02) * h)
        else:
            ang = rng.uniform(0, 2 * np.pi)
            x = T.mean(0) + (delta + rng.uniform(-0.8, 0.8) * h) * np.array([np.cos(ang), np.sin(ang)])
        a_no = _region_area(mesh, delta, 0, e, ep, x)
        a_ap = _region_area(mesh, delta, 4, e, ep, x)
        a_ex = _disc_triangle_area(T, x, delta)
        tol = 1e-12 * h * h
        assert a_no <= a_ap + tol and a_ap <= a_ex + tol, (a_no, a_ap, a_ex)
        if a_ex - a_no > 1e-6 * h * h:
            ratio = (a_ex - a_ap) / (a_ex - a_no)
            assert 0.2499 <= ratio <= 0.2548, (ratio, a_no, a_ap, a_ex)
            checked += 1
            dips += a_no == 0.0
    assert checked >= 30 and dips >= 10, (checked, dips)


def test_approxcaps_local_limit_quarter_of_nocaps():
    delta = 0.125
    errs = {}
    for ball in (0, 4):
        errs[ball] = []
        for N in (32, 64, 128):
            mesh = W.make_mesh(2, N, W.collar_cells(delta, N))
            kern = W.Kernel(W.KERNEL_CONST_L2, delta, ball=ball)
            kern.scale = W.default_scale(kern, 2)
            c = np.flatnonzero((np.abs(mesh.xy[:, 0] - 0.5) < 1e-12) & (np.abs(mesh.xy[:, 1] - 0.5) < 1e-12))
            rows = assembly.assemble_rows(mesh, kern, kern.scale, c)
            x = mesh.xy[:, 0]
            errs[ball].append((rows @ (x * x))[0] / (-2.0 / N ** 2) - 1.0)
    no, ap = np.array(errs[0]), np.array(errs[4])
    assert (no < 0).all() and (ap < 0).all(), errs          # both regions inside the disc
    assert np.all(np.abs(ap / no - 0.25) < 0.01), ap / no
    assert np.all(3.5 < ap[:-1] / ap[1:]) and np.all(ap[:-1] / ap[1:] < 4.5), ap    # O(h^2)
