"""Inputs of the unstructured cases: valid meshes (every triangle counter-clockwise with a
positive area, the same collar as the structured mesh) and graph-grown local parts (every
non-Dirichlet element labelled, every part connected through shared edges, seeded)."""
import numpy as np

import workloads as W


def _areas(mesh):
    P = mesh.xy[mesh.elems]
    return 0.5 * ((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) -
                  (P[:, 2, 0] - P[:, 0, 0]) * (P[:, 1, 1] - P[:, 0, 1]))


def test_unstructured_mesh_valid():
    N, m = 20, 3
    mesh = W.unstructured_mesh(N, m, seed=3)
    base = W.make_mesh(2, N, m)
    assert (_areas(mesh) > 0.2 / N ** 2).all()
    assert np.isclose(_areas(mesh).sum(), _areas(base).sum())           # same domain covered
    assert np.array_equal(mesh.node_is_dirichlet, base.node_is_dirichlet)
    assert np.array_equal(mesh.elem_is_dirichlet, base.elem_is_dirichlet)
    moved = np.abs(mesh.xy - base.xy).max(axis=1) > 0
    assert moved[base.node_is_dirichlet == 0].mean() > 0.9 and not moved[base.node_is_dirichlet == 1].any()
    assert not np.array_equal(mesh.elems, base.elems)                   # diagonals differ


def test_graph_labels_cover_and_connect():
    w = W.unstructured_l2(N=20, K=5)
    inside = w.mesh.elem_is_dirichlet == 0
    assert (w.labels[~inside] == -1).all() and (w.labels[inside] >= 0).all()
    sizes = np.bincount(w.labels[inside], minlength=w.K)
    assert sizes.min() > 0.5 * sizes.mean()
    ids = np.flatnonzero(inside)
    edges = {}
    for e in ids:
        v = w.mesh.elems[e]
        for a, b in ((0, 1), (1, 2), (0, 2)):
            edges.setdefault((min(v[a], v[b]), max(v[a], v[b])), []).append(e)
    adj = {e: [] for e in ids}
    for es in edges.values():
        if len(es) == 2:
            adj[es[0]].append(es[1])
            adj[es[1]].append(es[0])
    for k in range(w.K):
        part = set(ids[w.labels[ids] == k])
        start = next(iter(part))
        seen, stack = {start}, [start]
        while stack:
            for j in adj[stack.pop()]:
                if j in part and j not in seen:
                    seen.add(j)
                    stack.append(j)
        assert seen == part
    assert np.array_equal(w.labels, W.unstructured_l2(N=20, K=5).labels)   # seeded


def test_l2_collar_keeps_exactly_the_elements_meeting_the_disc_neighbourhood():
    N, delta = 24, 0.15
    base = W.make_mesh(2, N, W.collar_cells(delta, N))
    mesh = W.l2_collar(base, delta)
    # distance of a triangle to the unit square by dense barycentric sampling (resolution h / 40)
    t = np.linspace(0.0, 1.0, 41)
    a, b = np.meshgrid(t, t, indexing="ij")
    ok = (a + b) <= 1.0
    lam = np.stack([a[ok], b[ok], 1.0 - a[ok] - b[ok]], axis=1)

    def dist(P):
        pts = lam @ P
        return np.linalg.norm(pts - np.clip(pts, 0.0, 1.0), axis=1).min()

    kept = {tuple(np.round(mesh.xy[e].mean(axis=0), 12)) for e in mesh.elems}
    for e in range(base.n_elems):
        if base.elem_is_dirichlet[e] == 0:
            continue
        P = base.xy[base.elems[e]]
        d = dist(P)
        key = tuple(np.round(P.mean(axis=0), 12))
        if d <= delta - 1.0 / (40 * N):
            assert key in kept
        elif d > delta + 1e-12:
            assert key not in kept
    assert mesh.n_elems < base.n_elems and (mesh.elem_is_dirichlet == 0).sum() == (base.elem_is_dirichlet == 0).sum()
