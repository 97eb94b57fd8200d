"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module holds input generation only: structured P1 meshes with a Dirichlet
collar, rectangular local decompositions (element labels), and seeded load
vectors. It contains none of the method's arithmetic (no quadrature, no
decomposition extension, no solver step), so that the oracle and the CUDA path
stay independent while consuming identical inputs.

Problem setting follows Sec. 6.2 of the paper: the domain is the open unit
square (or unit interval in 1-D), the Dirichlet volume constraint occupies the
collar around it, the triangulation is regular, and the local decomposition
is a k1 x k2 grid of rectangles.  Mesh conventions:

* nodes on the grid (i, j), 0 <= i, j <= N + 2m, coordinate (i - m) / N,
  numbered lexicographically with x fastest; m = ceil(delta / h) collar cells;
* each cell (ci, cj) is split by its diagonal (ci, cj) -> (ci+1, cj+1) into a
  lower triangle [(ci,cj), (ci+1,cj), (ci+1,cj+1)] and an upper triangle
  [(ci,cj), (ci+1,cj+1), (ci,cj+1)], both counter-clockwise; element id is
  2 * (cj * (N + 2m) + ci) + (0 lower | 1 upper);
* a node is Dirichlet when it lies on the boundary of the unit square or
  outside it; an element is Dirichlet when its cell lies outside the square.

Unstructured variants (`unstructured_mesh`, `graph_labels`): irregular node positions and
cell diagonals with the same collar, and local parts grown on the element graph instead of
rectangles (the paper's general setting, Sec. 5.1: Omega-tilde_k from a graph partitioner).
"""
from __future__ import annotations

import heapq
import math
from dataclasses import dataclass, field

import numpy as np

KERNEL_CONST_LINF = 0      # constant kernel on an l-infinity ball (1-D: interval)
KERNEL_CONST_L2 = 1        # constant kernel on an l2 ball (nocaps polygon)
KERNEL_FRACTIONAL = 2      # c / |x-y|^(d+2s) on an l2 ball
KERNEL_PERIDYNAMIC = 3     # c (x-y)(x-y)^T / |x-y|^3 on an l2 ball, 2 dofs / node


@dataclass
class Mesh:
    dim: int
    N: int                  # cells per unit length
    m: int                  # collar cells
    xy: np.ndarray          # (n_nodes, dim) float64
    elems: np.ndarray       # (n_elems, dim+1) int32
    node_is_dirichlet: np.ndarray  # (n_nodes,) int8
    elem_is_dirichlet: np.ndarray  # (n_elems,) int8

    @property
    def h(self) -> float:
        return 1.0 / self.N

    @property
    def n_nodes(self) -> int:
        return self.xy.shape[0]

    @property
    def n_elems(self) -> int:
        return self.elems.shape[0]


@dataclass
class Kernel:
    type: int
    delta: float
    s: float = 0.0
    scale: float = 0.0      # <= 0 selects the default constant for the type
    ball: int = 0           # 2-D l2 kernels: 0 nocaps, 1 barycenter, 2 123vertices, 3 23vertices, 4 approxcaps

    @property
    def ncomp(self) -> int:
        return 2 if self.type == KERNEL_PERIDYNAMIC else 1


@dataclass
class Workload:
    name: str
    mesh: Mesh
    kernel: Kernel
    labels: np.ndarray          # (n_elems,) int32 local subdomain label, -1 on Dirichlet elements
    K: int
    rhs: np.ndarray             # (n_nodes * ncomp, nrhs) float64, column-major semantics
    rhs_kind: int               # 0 nodal values of f, 1 load vector
    g: np.ndarray | None = None  # (n_nodes * ncomp, nrhs) Dirichlet data or None
    meta: dict = field(default_factory=dict)

    @property
    def nrhs(self) -> int:
        return self.rhs.shape[1]


def collar_cells(delta: float, N: int) -> int:
    """Number of collar cells m = ceil(delta / h) (ties within 1e-9 cells round down)."""
    return int(math.ceil(delta * N - 1e-9))


def make_mesh(dim: int, N: int, m: int) -> Mesh:
    if dim == 1:
        n = N + 2 * m + 1
        i = np.arange(n)
        xy = ((i - m) / N).astype(np.float64).reshape(n, 1)
        elems = np.stack([np.arange(n - 1), np.arange(1, n)], axis=1).astype(np.int32)
        nd = ((i <= m) | (i >= m + N)).astype(np.int8)
        c = np.arange(n - 1)
        ed = ((c < m) | (c >= m + N)).astype(np.int8)
        return Mesh(1, N, m, xy, elems, nd, ed)
    if dim != 2:
        raise ValueError("dim must be 1 or 2")
    M = N + 2 * m                       # cells per side
    n1 = M + 1
    j, i = np.meshgrid(np.arange(n1), np.arange(n1), indexing="ij")
    i = i.ravel()
    j = j.ravel()
    xy = np.stack([(i - m) / N, (j - m) / N], axis=1).astype(np.float64)
    nd = ((i <= m) | (i >= m + N) | (j <= m) | (j >= m + N)).astype(np.int8)
    cj, ci = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")
    ci = ci.ravel()
    cj = cj.ravel()
    v00 = cj * n1 + ci
    v10 = v00 + 1
    v11 = v00 + n1 + 1
    v01 = v00 + n1
    lower = np.stack([v00, v10, v11], axis=1)
    upper = np.stack([v00, v11, v01], axis=1)
    elems = np.empty((2 * M * M, 3), dtype=np.int32)
    elems[0::2] = lower
    elems[1::2] = upper
    cell_out = (ci < m) | (ci >= m + N) | (cj < m) | (cj >= m + N)
    ed = np.repeat(cell_out, 2).astype(np.int8)
    return Mesh(2, N, m, xy, elems, nd, ed)


def rect_cuts(N: int, k: int, jitter: float = 0.0, rng: np.random.Generator | None = None) -> np.ndarray:
    """Cut positions (in cells of the unit square) for k slabs: round(i N / k), optionally jittered
    by U(-jitter, jitter) * N / k for the interior cuts."""
    cuts = np.array([i * N / k for i in range(k + 1)], dtype=np.float64)
    if jitter > 0.0:
        assert rng is not None
        u = rng.uniform(-jitter, jitter, size=k - 1)
        cuts[1:-1] = cuts[1:-1] + u * N / k
    c = np.rint(cuts).astype(np.int64)
    c[0], c[-1] = 0, N
    if np.any(np.diff(c) <= 0):
        raise ValueError("degenerate cuts")
    return c


def rect_labels(mesh: Mesh, kx: int, ky: int = 1, jitter: float = 0.0, seed: int | None = None) -> np.ndarray:
    """Label each non-Dirichlet element with the rectangle containing its barycenter.

    Rectangles are k_x x k_y slabs of the unit square bounded by grid lines
    (Sec. 6.2: the domain is substructured into K = k1 x k2 rectangles)."""
    rng = np.random.default_rng(seed) if jitter > 0.0 else None
    cx = rect_cuts(mesh.N, kx, jitter, rng)
    cy = rect_cuts(mesh.N, ky, jitter, rng) if mesh.dim == 2 else np.array([0, mesh.N])
    labels = np.full(mesh.n_elems, -1, dtype=np.int32)
    inside = mesh.elem_is_dirichlet == 0
    bary = mesh.xy[mesh.elems].mean(axis=1)          # (n_elems, dim)
    # barycenter in cells of the unit square; strictly inside one cell
    bx = bary[:, 0] * mesh.N
    ix = np.searchsorted(cx, bx, side="right") - 1
    if mesh.dim == 2:
        by = bary[:, 1] * mesh.N
        iy = np.searchsorted(cy, by, side="right") - 1
    else:
        iy = np.zeros_like(ix)
    lab = iy * kx + ix
    labels[inside] = lab[inside].astype(np.int32)
    return labels


def unstructured_mesh(N: int, m: int, amp: float = 0.15, seed: int = 7) -> Mesh:
    """2-D P1 mesh of [-m h, 1 + m h]^2 with irregular geometry and connectivity: the grid
    nodes strictly inside the unit square move by U(-amp, amp) h in each coordinate
    (amp <= 0.15 keeps every triangle counter-clockwise: a vertex moves less than 0.22 h,
    its distance to the opposite edge is at least 0.7 h), and each cell takes one of its two
    diagonals at random.  Nodes on the boundary of the unit square and outside it stay on
    the grid, so the Dirichlet nodes and elements are those of make_mesh(2, N, m)."""
    base = make_mesh(2, N, m)
    rng = np.random.default_rng(seed)
    xy = base.xy.copy()
    eps = 1e-12
    inside = (xy[:, 0] > eps) & (xy[:, 0] < 1 - eps) & (xy[:, 1] > eps) & (xy[:, 1] < 1 - eps)
    xy[inside] += rng.uniform(-amp, amp, size=(int(inside.sum()), 2)) / N
    M = N + 2 * m
    n1 = M + 1
    cj, ci = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")
    v00 = (cj * n1 + ci).ravel()
    v10, v11, v01 = v00 + 1, v00 + n1 + 1, v00 + n1
    anti = rng.random(M * M) < 0.5
    t0 = np.where(anti[:, None], np.stack([v00, v10, v01], 1), np.stack([v00, v10, v11], 1))
    t1 = np.where(anti[:, None], np.stack([v10, v11, v01], 1), np.stack([v00, v11, v01], 1))
    elems = np.empty((2 * M * M, 3), dtype=np.int32)
    elems[0::2] = t0
    elems[1::2] = t1
    return Mesh(2, N, m, xy, elems, base.node_is_dirichlet.copy(), base.elem_is_dirichlet.copy())


def graph_labels(mesh: Mesh, K: int, seed: int = 0) -> np.ndarray:
    """Local parts grown on the graph of non-Dirichlet elements (edges between elements that
    share a mesh edge): K seeds by farthest-point sampling of the barycenters (the first one
    at random), then the part with the fewest elements takes, one at a time, the unassigned
    neighbour of its region nearest to its seed (a greedy graph-growing partition; every part
    is connected).  Labels -1 on Dirichlet elements."""
    rng = np.random.default_rng(seed)
    inside = np.flatnonzero(mesh.elem_is_dirichlet == 0)
    pos = {int(e): i for i, e in enumerate(inside)}
    nv = mesh.elems.shape[1]
    edge_owner: dict = {}
    nbr = [[] for _ in inside]
    for i, e in enumerate(inside):
        vs = mesh.elems[e]
        for a in range(nv):
            for b in range(a + 1, nv):
                key = (min(vs[a], vs[b]), max(vs[a], vs[b]))
                if key in edge_owner:
                    j = edge_owner[key]
                    nbr[i].append(j)
                    nbr[j].append(i)
                else:
                    edge_owner[key] = i
    bary = mesh.xy[mesh.elems[inside]].mean(axis=1)
    seeds = [int(rng.integers(len(inside)))]
    dmin = np.linalg.norm(bary - bary[seeds[0]], axis=1)
    while len(seeds) < K:
        s = int(np.argmax(dmin))
        seeds.append(s)
        dmin = np.minimum(dmin, np.linalg.norm(bary - bary[s], axis=1))
    lab = np.full(len(inside), -1, dtype=np.int32)
    size = np.zeros(K, dtype=np.int64)
    heaps = [[] for _ in range(K)]
    for k, s in enumerate(seeds):
        lab[s] = k
        size[k] = 1
        for j in nbr[s]:
            heapq.heappush(heaps[k], (float(np.linalg.norm(bary[j] - bary[s])), j))
    left = len(inside) - K
    while left > 0:
        for k in np.argsort(size, kind="stable"):
            h = heaps[k]
            while h and lab[h[0][1]] >= 0:
                heapq.heappop(h)
            if h:
                break
        else:
            raise RuntimeError("graph partition: unreachable elements")
        _, j = heapq.heappop(heaps[k])
        lab[j] = k
        size[k] += 1
        left -= 1
        for i in nbr[j]:
            if lab[i] < 0:
                heapq.heappush(heaps[k], (float(np.linalg.norm(bary[i] - bary[seeds[k]])), i))
    labels = np.full(mesh.n_elems, -1, dtype=np.int32)
    labels[inside] = lab
    return labels


def unstructured_l2(N: int = 24, K: int = 5, nrhs: int = 2, delta: float = 0.1, seed: int = 7) -> Workload:
    """Constant l2 kernel on an unstructured mesh with graph-grown local parts, N(0,1) loads."""
    m = collar_cells(delta, N)
    mesh = unstructured_mesh(N, m, seed=seed)
    kern = Kernel(KERNEL_CONST_L2, delta)
    kern.scale = default_scale(kern, 2)
    labels = graph_labels(mesh, K, seed=seed)
    rhs = nodal_loads(mesh, 1, nrhs, seed + 1, "normal")
    return Workload("unstructured_l2", mesh, kern, labels, K, rhs, 1, meta=dict(N=N, delta=delta, K=K))


def unstructured_pd(N: int = 24, K: int = 4, nrhs: int = 2, delta_cells: int = 3, seed: int = 9) -> Workload:
    """Bond-based peridynamic kernel (2 dofs per node) on an unstructured mesh with graph-grown
    local parts, N(0,1) loads per dof."""
    delta = delta_cells / N
    m = collar_cells(delta, N)
    mesh = unstructured_mesh(N, m, seed=seed)
    kern = Kernel(KERNEL_PERIDYNAMIC, delta)
    kern.scale = default_scale(kern, 2)
    labels = graph_labels(mesh, K, seed=seed)
    rhs = nodal_loads(mesh, 2, nrhs, seed + 1, "normal")
    return Workload("unstructured_pd", mesh, kern, labels, K, rhs, 1, meta=dict(N=N, delta=delta, K=K))


def l2_collar(mesh: Mesh, delta: float) -> Mesh:
    """Keep only the collar elements that meet the l2 delta-neighbourhood of the unit square
    (the Dirichlet region of an l2 ball has rounded corners; the simplest discretization of
    it takes every triangle that meets it, Sec. 2.3.1), then drop unused nodes.  The distance
    between a triangle and the square (both convex) is the smallest distance from a vertex of
    one of them to the other."""
    P = mesh.xy[mesh.elems]                              # (n_elems, 3, 2)
    nE = P.shape[0]
    # vertex of a triangle to the square
    dv = np.linalg.norm(P - np.clip(P, 0.0, 1.0), axis=2).min(axis=1)
    # corner of the square to a triangle (zero when inside)
    dc = np.full(nE, np.inf)
    for cx, cy in ((0.0, 0.0), (1.0, 0.0), (0.0, 1.0), (1.0, 1.0)):
        q = np.array([cx, cy])
        d = np.minimum(np.minimum(_seg_dist_many(q, P[:, 0], P[:, 1]), _seg_dist_many(q, P[:, 1], P[:, 2])),
                       _seg_dist_many(q, P[:, 2], P[:, 0]))
        v0, v1, v2 = P[:, 0] - q, P[:, 1] - q, P[:, 2] - q
        c0 = v0[:, 0] * v1[:, 1] - v0[:, 1] * v1[:, 0]
        c1 = v1[:, 0] * v2[:, 1] - v1[:, 1] * v2[:, 0]
        c2 = v2[:, 0] * v0[:, 1] - v2[:, 1] * v0[:, 0]
        inside = (c0 >= 0) & (c1 >= 0) & (c2 >= 0)
        dc = np.minimum(dc, np.where(inside, 0.0, d))
    keep = (mesh.elem_is_dirichlet == 0) | (np.minimum(dv, dc) <= delta * (1 + 1e-12))
    elems = mesh.elems[keep]
    used = np.zeros(mesh.n_nodes, dtype=bool)
    used[elems.ravel()] = True
    new_id = np.full(mesh.n_nodes, -1, dtype=np.int64)
    new_id[used] = np.arange(int(used.sum()))
    return Mesh(mesh.dim, mesh.N, mesh.m, mesh.xy[used].copy(), new_id[elems].astype(np.int32),
                mesh.node_is_dirichlet[used].copy(), mesh.elem_is_dirichlet[keep].copy())


def _seg_dist_many(q, a, b):
    """distance from the point q to each segment [a_i, b_i]"""
    ab = b - a
    t = np.clip(np.einsum("ij,ij->i", q - a, ab) / np.maximum(np.einsum("ij,ij->i", ab, ab), 1e-300), 0.0, 1.0)
    return np.linalg.norm(q - (a + t[:, None] * ab), axis=1)


def l2_collar_const(N: int = 24, k: int = 3, nrhs: int = 2, delta: float = 0.15, seed: int = 17) -> Workload:
    """Constant l2 kernel on a mesh whose Dirichlet collar is the l2 delta-neighbourhood of
    the square (rounded corners), k x k rectangles, N(0,1) loads."""
    mesh = l2_collar(make_mesh(2, N, collar_cells(delta, N)), delta)
    kern = Kernel(KERNEL_CONST_L2, delta)
    kern.scale = default_scale(kern, 2)
    labels = rect_labels(mesh, k, k)
    rhs = nodal_loads(mesh, 1, nrhs, seed, "normal")
    return Workload("l2_collar", mesh, kern, labels, k * k, rhs, 1, meta=dict(N=N, delta=delta, k=k))


def neumann_sides(mesh: Mesh) -> Mesh:
    """The same mesh with the Dirichlet volume constraint kept only on the left (x < 0) and
    bottom (y < 0) parts of the collar; the rest of the collar (x > 1 or y > 1, corners
    included) becomes a Neumann region Gamma^N: free nodes and elements that belong to
    Omega_h = Omega u Gamma^N (Sec. 2.1), loaded like the interior.  Nodes on x = 0 or
    y = 0 stay Dirichlet."""
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    eps = 1e-12
    nd = ((x <= eps) | (y <= eps)).astype(np.int8)
    cen = mesh.xy[mesh.elems].mean(axis=1)
    ed = ((cen[:, 0] < 0) | (cen[:, 1] < 0)).astype(np.int8)
    return Mesh(mesh.dim, mesh.N, mesh.m, mesh.xy, mesh.elems, nd, ed)


def clamped_rect_labels(mesh: Mesh, kx: int, ky: int) -> np.ndarray:
    """rect_labels with the barycenters clamped into the unit square first, so that free
    collar elements (a Neumann region) join the nearest rectangle."""
    cx = rect_cuts(mesh.N, kx)
    cy = rect_cuts(mesh.N, ky)
    bary = np.clip(mesh.xy[mesh.elems].mean(axis=1) * mesh.N, 1e-9, mesh.N - 1e-9)
    ix = np.searchsorted(cx, bary[:, 0], side="right") - 1
    iy = np.searchsorted(cy, bary[:, 1], side="right") - 1
    labels = np.full(mesh.n_elems, -1, dtype=np.int32)
    free = mesh.elem_is_dirichlet == 0
    labels[free] = (iy * kx + ix)[free].astype(np.int32)
    return labels


def neumann_l2(N: int = 24, k: int = 3, nrhs: int = 2, delta: float = 0.1, seed: int = 13) -> Workload:
    """Constant l2 kernel with Dirichlet constraint on the left and bottom collar and a
    Neumann region on the rest, k x k rectangles (clamped labels), N(0,1) loads."""
    mesh = neumann_sides(make_mesh(2, N, collar_cells(delta, N)))
    kern = Kernel(KERNEL_CONST_L2, delta)
    kern.scale = default_scale(kern, 2)
    labels = clamped_rect_labels(mesh, k, k)
    rhs = nodal_loads(mesh, 1, nrhs, seed, "normal")
    return Workload("neumann_l2", mesh, kern, labels, k * k, rhs, 1, meta=dict(N=N, delta=delta, k=k))


def neumann_pd(N: int = 30, k: int = 3, nrhs: int = 2, delta_cells: int = 3, seed: int = 15) -> Workload:
    """Bond-based peridynamics with the same mixed volume constraints (2 dofs per node)."""
    delta = delta_cells / N
    mesh = neumann_sides(make_mesh(2, N, collar_cells(delta, N)))
    kern = Kernel(KERNEL_PERIDYNAMIC, delta)
    kern.scale = default_scale(kern, 2)
    labels = clamped_rect_labels(mesh, k, k)
    rhs = nodal_loads(mesh, 2, nrhs, seed, "normal")
    return Workload("neumann_pd", mesh, kern, labels, k * k, rhs, 1, meta=dict(N=N, delta=delta, k=k))


def nodal_loads(mesh: Mesh, ncomp: int, nrhs: int, seed: int, dist: str) -> np.ndarray:
    rng = np.random.default_rng(seed)
    n = mesh.n_nodes * ncomp
    if dist == "normal":
        return np.asfortranarray(rng.standard_normal((n, nrhs)))
    raise ValueError(dist)


def default_scale(kernel: Kernel, dim: int) -> float:
    """Kernel constants used by the workloads (the reading of each config is documented in DESIGN)."""
    d = kernel.delta
    if kernel.scale > 0:
        return kernel.scale
    if kernel.type == KERNEL_CONST_LINF:
        return 3.0 / d ** 3 if dim == 1 else 3.0 / (4.0 * d ** 4)
    if kernel.type == KERNEL_CONST_L2:
        return 4.0 / (math.pi * d ** 4)
    if kernel.type == KERNEL_FRACTIONAL:
        s = kernel.s
        return (2.0 - 2.0 * s) / (math.pi * d ** (2.0 - 2.0 * s))
    if kernel.type == KERNEL_PERIDYNAMIC:
        return 3.0 / d ** 3
    raise ValueError(kernel.type)


# --------------------------------------------------------------------------------------
# The five workload shapes (1-D constant, 2-D constant l2, fractional, peridynamic) at full
# size and at reduced sizes that keep the same structure for fast parity runs.
# --------------------------------------------------------------------------------------

def const_1d(N: int = 1000, K: int = 4, seed: int = 1, delta: float = 0.1, nrhs: int = 1) -> Workload:
    """1-D constant kernel 3/delta^3 on |x-y|<delta, h=1/N, K equal subdomains, nodal f=-2+U(-0.1,0.1)."""
    m = collar_cells(delta, N)
    mesh = make_mesh(1, N, m)
    kern = Kernel(KERNEL_CONST_LINF, delta)
    kern.scale = default_scale(kern, 1)
    labels = rect_labels(mesh, K)
    rng = np.random.default_rng(seed)
    f = -2.0 + rng.uniform(-0.1, 0.1, size=(mesh.n_nodes, nrhs))
    return Workload("1d_const", mesh, kern, labels, K, np.asfortranarray(f), 0,
                    meta=dict(N=N, delta=delta, kx=K, ky=1))


def const_l2_2d(N: int = 128, k: int = 4, nrhs: int = 8, seed: int = 2, delta: float = 0.1) -> Workload:
    """2-D constant kernel 4/(pi delta^4) on the l2 ball (nocaps), h=1/N, k x k subdomains, N(0,1) loads."""
    m = collar_cells(delta, N)
    mesh = make_mesh(2, N, m)
    kern = Kernel(KERNEL_CONST_L2, delta)
    kern.scale = default_scale(kern, 2)
    labels = rect_labels(mesh, k, k)
    rhs = nodal_loads(mesh, 1, nrhs, seed, "normal")
    return Workload("2d_const_l2", mesh, kern, labels, k * k, rhs, 1,
                    meta=dict(N=N, delta=delta, kx=k, ky=k))


def fractional_2d(N: int = 96, k: int = 6, nrhs: int = 64, seed: int = 3, delta: float = 0.2,
                    s: float = 0.5) -> Workload:
    """2-D fractional-type kernel (2-2s)/(pi delta^(2-2s)) |x-y|^-(2+2s), s=0.5, delta=0.2, h=1/N, k x k."""
    m = collar_cells(delta, N)
    mesh = make_mesh(2, N, m)
    kern = Kernel(KERNEL_FRACTIONAL, delta, s=s)
    kern.scale = default_scale(kern, 2)
    labels = rect_labels(mesh, k, k)
    rhs = nodal_loads(mesh, 1, nrhs, seed, "normal")
    return Workload("2d_fractional", mesh, kern, labels, k * k, rhs, 1,
                    meta=dict(N=N, delta=delta, kx=k, ky=k, s=s))


def peridynamic_2d(N: int = 256, k: int = 8, nrhs: int = 16, seed_cuts: int = 4, seed_rhs: int = 5,
                     delta_cells: int = 3, jitter: float = 0.2) -> Workload:
    """2-D bond-based peridynamics 3/delta^3 xi xi^T/|xi|^3, delta=3h, h=1/N, k x k jittered cuts."""
    delta = delta_cells / N
    m = collar_cells(delta, N)
    mesh = make_mesh(2, N, m)
    kern = Kernel(KERNEL_PERIDYNAMIC, delta)
    kern.scale = default_scale(kern, 2)
    labels = rect_labels(mesh, k, k, jitter=jitter, seed=seed_cuts)
    rhs = nodal_loads(mesh, 2, nrhs, seed_rhs, "normal")
    return Workload("2d_peridynamic", mesh, kern, labels, k * k, rhs, 1,
                    meta=dict(N=N, delta=delta, kx=k, ky=k, jitter=jitter))


def manufactured_1d_quadratic(N: int = 1000, K: int = 4, delta: float = 0.1) -> Workload:
    """1-D closed-form case: c=3/delta^3, nodal f=-2, g = x^2/2 on the collar; the discrete
    solution is x^2/2 at every node (uniform mesh, delta/h integer)."""
    w = const_1d(N=N, K=K, delta=delta)
    x = w.mesh.xy[:, 0]
    w.rhs = np.asfortranarray(np.full((w.mesh.n_nodes, 1), -2.0))
    w.g = np.asfortranarray((0.5 * x * x).reshape(-1, 1))
    w.name = "1d_quadratic"
    return w


WORKLOADS = {
    "const_1d": const_1d,
    "const_l2_2d": const_l2_2d,
    "fractional_2d": fractional_2d,
    "peridynamic_2d": peridynamic_2d,
}
