// Host construction of the nonlocal subdivision and the FETI index structures.
//
// Sec. 5.1: each local part Omega-tilde_k is extended by an approximate
// delta/2-neighbourhood to Omega-hat_k, and Gamma^D_k collects the collar elements
// within delta of Omega-tilde_k.  The neighbourhood test is the l-infinity gap between
// element bounding boxes (a superset of the exact criterion, admissible by
// Def. nonlocalsubdivision), with radii (delta/2)(1+1e-9) and delta(1+1e-9).
// zeta (eq. zeta) counts at nodes the Omega-hat_k holding the node and at element
// pairs the Omega-hat_k u Gamma^D_k holding both.  Dofs of k are the non-Dirichlet
// nodes of Omega-hat_k, Omega_k (zeta = 1) first, Gamma_k (zeta >= 2) after, each
// ascending (Sec. 3.3, index sets I_k and G_k).  B (eq. constraintSpace) has, per
// interface node in ascending order, one row per link of the chain of its
// subdomains k_1 < ... < k_z (+1 on k_j, -1 on k_{j+1}), the component fastest.
// Pinned dofs of floating subdomains (Sec. 5.3): scalar -- the first Gamma_k node;
// vector -- both components of that node a and, at the Gamma_k node b farthest from
// a (first on ties), the component along which |x_b - x_a| is smaller.
#include <algorithm>
#include <cmath>
#include <map>

#include "internal.hpp"

namespace nlf {

namespace {

struct Box {
    double lo[2], hi[2];
};

struct Buckets {
    int dim;
    double org[2], H;
    int64_t nb[2];
    std::vector<int64_t> start, items;
};

void make_boxes(const MeshHost &m, std::vector<Box> &bb) {
    int nv = m.dim + 1;
    bb.resize(m.n_elems);
    for (int64_t e = 0; e < m.n_elems; ++e) {
        Box b;
        for (int a = 0; a < 2; ++a) { b.lo[a] = 0; b.hi[a] = 0; }
        for (int a = 0; a < m.dim; ++a) { b.lo[a] = INFINITY; b.hi[a] = -INFINITY; }
        for (int i = 0; i < nv; ++i) {
            int32_t n = m.elems[e * nv + i];
            for (int a = 0; a < m.dim; ++a) {
                double x = m.xy[(int64_t)n * m.dim + a];
                b.lo[a] = std::min(b.lo[a], x);
                b.hi[a] = std::max(b.hi[a], x);
            }
        }
        bb[e] = b;
    }
}

void make_buckets(const MeshHost &m, const std::vector<Box> &bb, Buckets &G) {
    G.dim = m.dim;
    double lo[2] = {INFINITY, INFINITY}, hi[2] = {-INFINITY, -INFINITY}, ext = 0;
    for (const Box &b : bb)
        for (int a = 0; a < m.dim; ++a) {
            lo[a] = std::min(lo[a], b.lo[a]);
            hi[a] = std::max(hi[a], b.hi[a]);
            ext = std::max(ext, b.hi[a] - b.lo[a]);
        }
    G.H = ext > 0 ? ext : 1.0;
    for (int a = 0; a < 2; ++a) {
        G.org[a] = a < m.dim ? lo[a] : 0.0;
        G.nb[a] = a < m.dim ? (int64_t)std::floor((hi[a] - lo[a]) / G.H) + 1 : 1;
    }
    int64_t nbt = G.nb[0] * G.nb[1];
    G.start.assign(nbt + 1, 0);
    std::vector<int64_t> cell(bb.size());
    for (size_t e = 0; e < bb.size(); ++e) {
        int64_t c[2] = {0, 0};
        for (int a = 0; a < m.dim; ++a)
            c[a] = std::clamp<int64_t>((int64_t)std::floor((bb[e].lo[a] - G.org[a]) / G.H), 0, G.nb[a] - 1);
        cell[e] = c[1] * G.nb[0] + c[0];
        G.start[cell[e] + 1]++;
    }
    for (int64_t i = 0; i < nbt; ++i) G.start[i + 1] += G.start[i];
    G.items.resize(bb.size());
    std::vector<int64_t> fill(G.start.begin(), G.start.end() - 1);
    for (size_t e = 0; e < bb.size(); ++e) G.items[fill[cell[e]]++] = (int64_t)e;
}

inline double box_gap(const Box &a, const Box &b, int dim) {
    double g = 0.0;
    for (int k = 0; k < dim; ++k) {
        double d1 = a.lo[k] - b.hi[k], d2 = b.lo[k] - a.hi[k];
        double d = d1 > d2 ? d1 : d2;
        if (d > g) g = d;
    }
    return g;
}

// mark every element within gap r of box b
template <typename F> void for_near(const Buckets &G, const std::vector<Box> &bb, const Box &b, double r, F &&f) {
    int64_t lo[2] = {0, 0}, hi[2] = {0, 0};
    for (int a = 0; a < G.dim; ++a) {
        lo[a] = std::max<int64_t>(0, (int64_t)std::floor((b.lo[a] - r - G.H - G.org[a]) / G.H) - 1);
        hi[a] = std::min<int64_t>(G.nb[a] - 1, (int64_t)std::floor((b.hi[a] + r - G.org[a]) / G.H) + 1);
    }
    for (int64_t cy = lo[1]; cy <= hi[1]; ++cy)
        for (int64_t cx = lo[0]; cx <= hi[0]; ++cx) {
            int64_t c = cy * G.nb[0] + cx;
            for (int64_t t = G.start[c]; t < G.start[c + 1]; ++t) {
                int64_t e = G.items[t];
                if (box_gap(bb[e], b, G.dim) <= r) f(e);
            }
        }
}

}  // namespace

void build_decomposition(const MeshHost &m, const nlfeti_kernel &kern, const std::vector<int32_t> &labels, int K,
                         Decomp &d) {
    if (K < 1 || K > kMaxSubdomains) fail(NLFETI_E_INVALID, "K must be in [1, 4096]");
    d.K = K;
    const int W = (K + 63) / 64;
    d.mask_words = W;
    d.nc = kern.type == NLFETI_K_PERIDYNAMIC ? 2 : 1;
    const int nc = d.nc;
    const int nv = m.dim + 1;
    std::vector<Box> bb;
    make_boxes(m, bb);
    Buckets G;
    make_buckets(m, bb, G);
    const double r_ext = (0.5 * kern.delta) * (1.0 + 1e-9);
    const double r_dir = kern.delta * (1.0 + 1e-9);
    d.elem_mask.assign((size_t)m.n_elems * W, 0);
    std::vector<std::vector<int64_t>> parts(K);
    for (int64_t e = 0; e < m.n_elems; ++e) {
        if (m.elem_dir[e]) continue;
        int32_t l = labels[e];
        if (l < 0 || l >= K) fail(NLFETI_E_INVALID, "element label out of range");
        parts[l].push_back(e);
    }
    std::vector<char> has_dir(K, 0);
    for (int k = 0; k < K; ++k) {
        if (parts[k].empty()) fail(NLFETI_E_INVALID, "empty local subdomain");
        const uint64_t bit = uint64_t(1) << (k % 64);
        const int wk = k / 64;
        for (int64_t f : parts[k]) {
            d.elem_mask[f * W + wk] |= bit;
            for_near(G, bb, bb[f], r_dir, [&](int64_t e) {
                if (d.elem_mask[e * W + wk] & bit) return;
                if (m.elem_dir[e]) {
                    d.elem_mask[e * W + wk] |= bit;
                    has_dir[k] = 1;
                } else if (box_gap(bb[e], bb[f], m.dim) <= r_ext) {
                    d.elem_mask[e * W + wk] |= bit;
                }
            });
        }
    }
    // nodes of Omega-hat_k and their zeta
    d.node_zeta.assign(m.n_nodes, 0);
    std::vector<std::vector<int32_t>> hat_nodes(K), dnodes(K);
    {
        std::vector<uint64_t> node_mask((size_t)m.n_nodes * W, 0), node_dmask((size_t)m.n_nodes * W, 0);
        for (int64_t e = 0; e < m.n_elems; ++e) {
            if (!d.any_sub(e)) continue;
            for (int i = 0; i < nv; ++i) {
                int32_t n = m.elems[e * nv + i];
                for (int w = 0; w < W; ++w) {
                    const uint64_t msk = d.elem_mask[e * W + w];
                    if (m.node_dir[n]) node_dmask[(int64_t)n * W + w] |= msk;
                    else if (!m.elem_dir[e]) node_mask[(int64_t)n * W + w] |= msk;
                }
            }
        }
        for (int64_t n = 0; n < m.n_nodes; ++n) {
            int z = 0;
            for (int w = 0; w < W; ++w) {
                uint64_t msk = node_mask[n * W + w];
                z += __builtin_popcountll(msk);
                while (msk) {
                    int k = 64 * w + __builtin_ctzll(msk);
                    hat_nodes[k].push_back((int32_t)n);
                    msk &= msk - 1;
                }
                uint64_t dm = node_dmask[n * W + w];
                while (dm) {
                    int k = 64 * w + __builtin_ctzll(dm);
                    dnodes[k].push_back((int32_t)n);
                    dm &= dm - 1;
                }
            }
            d.node_zeta[n] = z;
        }
    }
    d.nodes.assign(K, {});
    d.n_omega_nodes.assign(K, 0);
    d.n_gamma_nodes.assign(K, 0);
    d.dir_nodes = dnodes;
    d.floating.assign(K, 0);
    d.pinned.assign(K, {});
    d.u_off.assign(K + 1, 0);
    std::vector<std::map<int32_t, int32_t>> gpos(K);
    for (int k = 0; k < K; ++k) {
        std::vector<int32_t> om, ga;
        for (int32_t n : hat_nodes[k]) (d.node_zeta[n] == 1 ? om : ga).push_back(n);
        d.n_omega_nodes[k] = (int32_t)om.size();
        d.n_gamma_nodes[k] = (int32_t)ga.size();
        for (size_t i = 0; i < ga.size(); ++i) gpos[k][ga[i]] = (int32_t)i;
        d.nodes[k] = om;
        d.nodes[k].insert(d.nodes[k].end(), ga.begin(), ga.end());
        d.floating[k] = has_dir[k] ? 0 : 1;
        d.u_off[k + 1] = d.u_off[k] + (int64_t)ga.size() * nc;
        if (d.floating[k] && !ga.empty()) {
            if (nc == 1) {
                d.pinned[k] = {0};
            } else {
                const double xa = m.xy[2 * (int64_t)ga[0]], ya = m.xy[2 * (int64_t)ga[0] + 1];
                double best = -1.0;
                int32_t b = 0;
                for (size_t i = 0; i < ga.size(); ++i) {
                    double dx = m.xy[2 * (int64_t)ga[i]] - xa, dy = m.xy[2 * (int64_t)ga[i] + 1] - ya;
                    double d2 = dx * dx + dy * dy;
                    if (d2 > best) { best = d2; b = (int32_t)i; }
                }
                double ax = std::fabs(m.xy[2 * (int64_t)ga[b]] - xa), ay = std::fabs(m.xy[2 * (int64_t)ga[b] + 1] - ya);
                int comp = ax < ay ? 0 : 1;
                d.pinned[k] = {0, 1, 2 * b + comp};
            }
        }
    }
    // B: chain rows per interface node
    d.B_plus.clear(); d.B_minus.clear(); d.B_node.clear();
    // per interface node, its subdomains in ascending order
    std::vector<std::vector<int>> owners(m.n_nodes);
    for (int k = 0; k < K; ++k)
        for (const auto &kv : gpos[k]) owners[kv.first].push_back(k);
    for (int64_t n = 0; n < m.n_nodes; ++n) {
        if (d.node_zeta[n] < 2) continue;
        const std::vector<int> &ks = owners[n];
        for (size_t j = 0; j + 1 < ks.size(); ++j) {
            int ka = ks[j], kb = ks[j + 1];
            for (int c = 0; c < nc; ++c) {
                d.B_plus.push_back(d.u_off[ka] + (int64_t)gpos[ka][(int32_t)n] * nc + c);
                d.B_minus.push_back(d.u_off[kb] + (int64_t)gpos[kb][(int32_t)n] * nc + c);
                d.B_node.push_back((int32_t)n);
            }
        }
    }
    d.co_off.assign(K + 1, 0);
    for (int k = 0; k < K; ++k)
        d.co_off[k + 1] = d.co_off[k] + ((d.floating[k] && d.n_gamma_nodes[k] > 0) ? (nc == 1 ? 1 : 3) : 0);
}

}  // namespace nlf
