"""Brute-force pins of the oracle's inner integrals on tiny meshes.

The oracle integrates, for an outer point x, over the inner region E' cap B^h(x)
(l2 "nocaps" polygon of Fig. approximate-ball (e), or the l-infinity square), with
exact rules for constant kernels and a polar rule (radial integral in closed form,
8-point Gauss-Legendre in the angle) for the fractional and peridynamic kernels.

Here the region is rebuilt independently (edge/circle crossings by root bracketing,
ordering by a convex hull) and the integral is evaluated by other means:

* constant kernels: Duffy-mapped tensor Gauss-Legendre on a fan of the polygon
  (exact for the quadratic integrand) -> agreement to rounding;
* singular kernels, x inside E' = E: the integral over each triangle (x, V_k, V_k+1)
  factorises into a radial power integral (closed form) times an adaptive integral
  along the edge -> agreement to ~1e-9 (the oracle's polar rule with the geometric
  angular split);
* singular kernels, touching pairs: nested adaptive integration over the polygon in
  Duffy coordinates -> agreement to ~1e-9;
* singular kernels, separated pairs: high-order tensor Gauss on a fan of the polygon
  (the integrand is smooth there) -> agreement to the accuracy of the oracle's
  7-point rule per fan triangle.

1-D: the whole pair integral is compared with an adaptive double integral over
E x E' restricted to |x - y| <= delta (exact for delta/h integer).
"""
import numpy as np
import pytest
from scipy import integrate, optimize
from scipy.spatial import ConvexHull

import workloads as W
from oracle import assembly


def _bary_solve(tri, y):
    """Barycentric coordinates of y (..., 2) in triangle tri (3, 2) by a linear solve."""
    T = np.array([[tri[0][0], tri[1][0], tri[2][0]], [tri[0][1], tri[1][1], tri[2][1]], [1.0, 1.0, 1.0]])
    y = np.atleast_2d(y)
    rhs = np.vstack([y[:, 0], y[:, 1], np.ones(y.shape[0])])
    return np.linalg.solve(T, rhs).T


def _nocaps_polygon(tri, x, delta):
    pts = [v for v in tri if np.hypot(*(v - x)) <= delta]
    for k in range(3):
        A, B = tri[k], tri[(k + 1) % 3]
        f = lambda t: np.hypot(*(A + t * (B - A) - x)) - delta
        ts = np.linspace(0, 1, 2001)
        vals = np.array([f(t) for t in ts])
        for i in range(len(ts) - 1):
            if vals[i] == 0:
                continue
            if vals[i] * vals[i + 1] < 0:
                t = optimize.brentq(f, ts[i], ts[i + 1], xtol=1e-15, rtol=1e-15)
                pts.append(A + t * (B - A))
    if len(pts) < 3:
        return None
    P = np.array(pts)
    hull = ConvexHull(P)
    return P[hull.vertices]


def _square_polygon(tri, x, delta):
    # sample-free construction: vertices of the triangle inside the square, triangle edges
    # crossing the square's sides, square corners inside the triangle
    pts = [v for v in tri if np.max(np.abs(v - x)) <= delta]
    for k in range(3):
        A, B = tri[k], tri[(k + 1) % 3]
        for ax in range(2):
            for side in (-1, 1):
                if B[ax] != A[ax]:
                    t = (x[ax] + side * delta - A[ax]) / (B[ax] - A[ax])
                    if 0 < t < 1:
                        p = A + t * (B - A)
                        if np.max(np.abs(p - x)) <= delta * (1 + 1e-14):
                            pts.append(p)
    for sx in (-1, 1):
        for sy in (-1, 1):
            c = x + delta * np.array([sx, sy])
            b = _bary_solve(tri, c)[0]
            if (b >= -1e-15).all():
                pts.append(c)
    if len(pts) < 3:
        return None
    P = np.array(pts)
    return P[ConvexHull(P).vertices]


def _tri_rule(n):
    """Duffy-collapsed tensor Gauss-Legendre on the unit triangle: points (n*n, 2), weights."""
    t, w = np.polynomial.legendre.leggauss(n)
    u = 0.5 * (t + 1)
    wu = 0.5 * w
    U, V = np.meshgrid(u, u, indexing="ij")
    WU, WV = np.meshgrid(wu, wu, indexing="ij")
    # (u, v) -> (u (1 - v), u v), Jacobian u
    pts = np.stack([(U * (1 - V)).ravel(), (U * V).ravel()], axis=1)
    return pts, (WU * WV * U).ravel()


def _integrand(kt, c, s, x, y, dv):
    """kernel-weighted products for local dofs; dv: (npts, nl) differences psi(y)-psi(x)."""
    xi = y - x
    r = np.hypot(xi[:, 0], xi[:, 1])
    if kt in (W.KERNEL_CONST_L2, W.KERNEL_CONST_LINF):
        return c * dv[:, :, None] * dv[:, None, :]
    if kt == W.KERNEL_FRACTIONAL:
        return (c * r ** (-2 - 2 * s))[:, None, None] * dv[:, :, None] * dv[:, None, :]
    th = xi / r[:, None]
    base = (c / r)[:, None, None] * dv[:, :, None] * dv[:, None, :]        # (n, nl, nl)
    nl = dv.shape[1]
    out = np.zeros((y.shape[0], 2 * nl, 2 * nl))
    for a in range(2):
        for b in range(2):
            out[:, a::2, b::2] = base * (th[:, a] * th[:, b])[:, None, None]
    return out


def _local_setup(mesh, e, ep, nodes, x):
    tri_o = mesh.xy[mesh.elems[e]]
    tri_i = mesh.xy[mesh.elems[ep]]
    bo = _bary_solve(tri_o, x)[0]
    a = np.array([bo[list(mesh.elems[e]).index(n)] if n in mesh.elems[e] else 0.0 for n in nodes])
    return tri_o, tri_i, a


def _psi_inner(mesh, ep, nodes, y):
    tri_i = mesh.xy[mesh.elems[ep]]
    b = _bary_solve(tri_i, y)
    out = np.zeros((y.shape[0], len(nodes)))
    for j, n in enumerate(nodes):
        if n in mesh.elems[ep]:
            out[:, j] = b[:, list(mesh.elems[ep]).index(n)]
    return out


def _brute_outside(mesh, kern, e, ep, x, nodes, P, order=40):
    _, _, a = _local_setup(mesh, e, ep, nodes, x)
    pts, wts = _tri_rule(order)
    nl = len(nodes) * kern.ncomp
    acc = np.zeros((nl, nl))
    for k in range(1, P.shape[0] - 1):
        V0, V1, V2 = P[0], P[k], P[k + 1]
        J = abs((V1[0] - V0[0]) * (V2[1] - V0[1]) - (V1[1] - V0[1]) * (V2[0] - V0[0]))
        y = V0 + pts[:, :1] * (V1 - V0) + pts[:, 1:] * (V2 - V0)
        dv = _psi_inner(mesh, ep, nodes, y) - a[None, :]
        acc += np.einsum("n,nij->ij", wts * J, _integrand(kern.type, kern.scale, kern.s, x, y, dv))
    return acc


def _brute_adaptive(mesh, kern, e, ep, x, nodes, P, eps=1e-12):
    """Nested adaptive integration (Duffy coordinates) over each fan triangle of the polygon."""
    _, _, a = _local_setup(mesh, e, ep, nodes, x)
    nl = len(nodes) * kern.ncomp
    acc = np.zeros((nl, nl))
    for k in range(1, P.shape[0] - 1):
        V0, V1, V2 = P[0], P[k], P[k + 1]
        J = abs((V1[0] - V0[0]) * (V2[1] - V0[1]) - (V1[1] - V0[1]) * (V2[0] - V0[0]))

        def inner(u):
            def f(v):
                y = (V0 + u * (1 - v) * (V1 - V0) + u * v * (V2 - V0))[None, :]
                dv = _psi_inner(mesh, ep, nodes, y) - a[None, :]
                return _integrand(kern.type, kern.scale, kern.s, x, y, dv)[0] * u * J
            return integrate.quad_vec(f, 0.0, 1.0, epsabs=0.0, epsrel=eps)[0]
        acc += integrate.quad_vec(inner, 0.0, 1.0, epsabs=0.0, epsrel=eps)[0]
    return acc


def _brute_inside(mesh, kern, e, x, nodes, P, nv=64):
    """x inside the polygon, E' = E: psi(y)-psi(x) = g.(y-x); per fan triangle from x the radial
    factor integrates in closed form and the edge factor by Gauss-Legendre."""
    tri = mesh.xy[mesh.elems[e]]
    # gradients of the P1 basis by solving
    T = np.array([[tri[0][0], tri[0][1], 1.0], [tri[1][0], tri[1][1], 1.0], [tri[2][0], tri[2][1], 1.0]])
    coef = np.linalg.solve(T, np.eye(3))      # columns: [gx, gy, c] for each basis
    g = np.array([[coef[0, list(mesh.elems[e]).index(n)], coef[1, list(mesh.elems[e]).index(n)]] for n in nodes])
    s, c = kern.s, kern.scale
    nl = len(nodes) * kern.ncomp
    acc = np.zeros((nl, nl))
    for k in range(P.shape[0]):
        A, B = P[k] - x, P[(k + 1) % P.shape[0]] - x
        J = A[0] * (B - A)[1] - A[1] * (B - A)[0]               # signed; xi = u (A + v (B - A)), dy = u J du dv

        def f(v):
            Wv = A + v * (B - A)
            rw = np.hypot(Wv[0], Wv[1])
            gw = g @ Wv                                          # (nl_nodes,)
            if kern.type == W.KERNEL_FRACTIONAL:
                # c |u w|^{-2-2s} (u g.w)(u g.w) u J  ->  u^{1-2s}: integral over u in [0,1] = 1/(2-2s)
                return c * rw ** (-2 - 2 * s) * J * np.outer(gw, gw) / (2 - 2 * s)
            # c (w w^T/|w|^3)(g.w)(g.w) u^{4-3} u J -> integral of u^2 over [0,1] = 1/3
            th = Wv / rw
            out = np.zeros((nl, nl))
            base = c / rw * J / 3.0 * np.outer(gw, gw)
            for a_ in range(2):
                for b_ in range(2):
                    out[a_::2, b_::2] = base * th[a_] * th[b_]
            return out
        acc += integrate.quad_vec(f, 0.0, 1.0, epsabs=0.0, epsrel=1e-13)[0]
    return acc


def _mesh_kernel(kt, N=8, delta=0.3, s=0.5):
    mesh = W.make_mesh(2, N, W.collar_cells(delta, N))
    kern = W.Kernel(kt, delta, s=s)
    kern.scale = W.default_scale(kern, 2)
    return mesh, kern


def _elem_at(mesh, cx, cy, upper):
    M = mesh.N + 2 * mesh.m
    return 2 * ((cy + mesh.m) * M + (cx + mesh.m)) + upper


RNG = np.random.default_rng(7)
POINTS = [RNG.dirichlet([2, 2, 2]) for _ in range(3)]


@pytest.mark.parametrize("kt", [W.KERNEL_CONST_L2, W.KERNEL_CONST_LINF])
@pytest.mark.parametrize("offset", [(0, 0, 1), (1, 0, 0), (2, 1, 1), (2, 2, 0), (3, 0, 1)])
def test_constant_kernels_inner_integral(kt, offset):
    mesh, kern = _mesh_kernel(kt, N=8, delta=0.3)
    e = _elem_at(mesh, 3, 3, 0)
    ep = _elem_at(mesh, 3 + offset[0], 3 + offset[1], offset[2])
    tri_o = mesh.xy[mesh.elems[e]]
    tri_i = mesh.xy[mesh.elems[ep]]
    for bc in POINTS:
        x = bc @ tri_o
        L, nodes = assembly.point_integral(mesh, kern, kern.scale, e, ep, x)
        P = _nocaps_polygon(tri_i, x, kern.delta) if kt == W.KERNEL_CONST_L2 else _square_polygon(tri_i, x, kern.delta)
        if P is None:
            assert np.abs(L).max() == 0.0
            continue
        ref = _brute_outside(mesh, kern, e, ep, x, list(nodes), P, order=6)
        assert np.abs(L - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1e-300), (np.abs(L - ref).max(), np.abs(ref).max())


@pytest.mark.parametrize("kt,s", [(W.KERNEL_FRACTIONAL, 0.5), (W.KERNEL_FRACTIONAL, 0.4), (W.KERNEL_PERIDYNAMIC, 0.0)])
def test_singular_kernels_self_pair(kt, s):
    mesh, kern = _mesh_kernel(kt, N=8, delta=0.3, s=s)
    e = _elem_at(mesh, 3, 3, 1)
    tri = mesh.xy[mesh.elems[e]]
    for bc in POINTS:
        x = bc @ tri
        L, nodes = assembly.point_integral(mesh, kern, kern.scale, e, e, x)
        P = _nocaps_polygon(tri, x, kern.delta)
        ref = _brute_inside(mesh, kern, e, x, list(nodes), P)
        assert np.abs(L - ref).max() <= 1e-9 * np.abs(ref).max(), (np.abs(L - ref).max(), np.abs(ref).max())


@pytest.mark.parametrize("kt,s", [(W.KERNEL_FRACTIONAL, 0.5), (W.KERNEL_FRACTIONAL, 0.4), (W.KERNEL_PERIDYNAMIC, 0.0)])
@pytest.mark.parametrize("offset", [(0, 0, 1), (1, 0, 0), (1, 0, 1), (0, 1, 0), (1, 1, 0), (-1, -1, 1)])
def test_singular_kernels_touching_pair(kt, s, offset):
    """Touching pairs use the polar rule with the geometric angular split: near machine precision."""
    mesh, kern = _mesh_kernel(kt, N=8, delta=0.3, s=s)
    e = _elem_at(mesh, 3, 3, 0)
    ep = _elem_at(mesh, 3 + offset[0], 3 + offset[1], offset[2])
    tri_o = mesh.xy[mesh.elems[e]]
    tri_i = mesh.xy[mesh.elems[ep]]
    for bc in POINTS[:2]:
        x = bc @ tri_o
        L, nodes = assembly.point_integral(mesh, kern, kern.scale, e, ep, x)
        P = _nocaps_polygon(tri_i, x, kern.delta)
        ref = _brute_adaptive(mesh, kern, e, ep, x, list(nodes), P)
        assert np.abs(L - ref).max() <= 1e-9 * np.abs(ref).max(), (np.abs(L - ref).max(), np.abs(ref).max())


@pytest.mark.parametrize("kt,s", [(W.KERNEL_FRACTIONAL, 0.5), (W.KERNEL_FRACTIONAL, 0.4), (W.KERNEL_PERIDYNAMIC, 0.0)])
@pytest.mark.parametrize("offset", [(2, 0, 0), (2, 1, 1), (1, 2, 0), (3, 1, 1)])
def test_singular_kernels_separated_pair(kt, s, offset):
    mesh, kern = _mesh_kernel(kt, N=8, delta=0.3, s=s)
    e = _elem_at(mesh, 3, 3, 0)
    ep = _elem_at(mesh, 3 + offset[0], 3 + offset[1], offset[2])
    tri_o = mesh.xy[mesh.elems[e]]
    tri_i = mesh.xy[mesh.elems[ep]]
    for bc in POINTS:
        x = bc @ tri_o
        L, nodes = assembly.point_integral(mesh, kern, kern.scale, e, ep, x)
        P = _nocaps_polygon(tri_i, x, kern.delta)
        if P is None:
            assert np.abs(L).max() == 0.0
            continue
        ref = _brute_outside(mesh, kern, e, ep, x, list(nodes), P, order=40)
        # separated pairs use a 7-point rule per fan triangle: agreement to that rule's accuracy
        assert np.abs(L - ref).max() <= 2e-3 * np.abs(ref).max(), (np.abs(L - ref).max(), np.abs(ref).max())


@pytest.mark.parametrize("pair", [(10, 10), (10, 11), (10, 13), (10, 14), (9, 12), (3, 5)])
def test_1d_pair_matrix_double_integral(pair):
    N, delta = 20, 0.2                 # delta/h = 4 (integer): the outer 4-point rule is exact
    mesh = W.make_mesh(1, N, W.collar_cells(delta, N))
    kern = W.Kernel(W.KERNEL_CONST_LINF, delta)
    kern.scale = W.default_scale(kern, 1)
    e, ep = pair
    L, nodes = assembly.pair_matrix(mesh, kern, kern.scale, e, ep)
    a, b = mesh.xy[mesh.elems[e], 0]
    c0, c1 = mesh.xy[mesh.elems[ep], 0]

    def psi(n, el, t):
        p, q = mesh.xy[mesh.elems[el], 0]
        if mesh.elems[el][0] == n:
            return (q - t) / (q - p)
        if mesh.elems[el][1] == n:
            return (t - p) / (q - p)
        return 0.0

    for i, ni in enumerate(nodes):
        for j, nj in enumerate(nodes):
            f = lambda y, x: kern.scale * (psi(ni, ep, y) - psi(ni, e, x)) * (psi(nj, ep, y) - psi(nj, e, x))
            val, _ = integrate.dblquad(f, a, b, lambda x: max(c0, x - delta), lambda x: min(c1, x + delta),
                                       epsabs=1e-13, epsrel=1e-12)
            # dblquad returns 0 when the inner interval is empty at every x
            assert abs(L[i, j] - val) <= 1e-10 * max(1.0, abs(val))
