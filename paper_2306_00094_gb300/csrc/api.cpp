// C ABI of the nlfeti library: contexts, problems (setup + assembly), factorization,
// solves, operator application and introspection.  Every entry point converts internal
// errors into an nlfeti_status and records the message in the context.
#include <atomic>
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "solve.hpp"

namespace nlf {

void fail(nlfeti_status st, const std::string &msg) { throw Error{st, msg}; }

void check_cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        fail(NLFETI_E_NOMEM, std::string("device allocation failed in ") + what);
    }
    fail(NLFETI_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void set_error(nlfeti_ctx *c, const std::string &msg) {
    if (!c) return;
    std::lock_guard<std::mutex> g(c->mu);
    c->err = msg;
}

void stream_enter(nlfeti_ctx *c) {
    NLF_CUDA(cudaEventRecord(c->ev_in, c->user_stream));
    NLF_CUDA(cudaStreamWaitEvent(c->stream, c->ev_in, 0));
}

void stream_leave(nlfeti_ctx *c) {
    NLF_CUDA(cudaEventRecord(c->ev_out, c->stream));
    NLF_CUDA(cudaStreamWaitEvent(c->user_stream, c->ev_out, 0));
}

void DevMem::alloc(nlfeti_ctx *c, size_t n) {
    release();
    ctx = c;
    async = false;
    n = std::max<size_t>(n, 16);
    {
        std::lock_guard<std::mutex> g(c->mu);
        if (c->opt.hbm_budget && c->bytes_in_use + n > c->opt.hbm_budget)
            fail(NLFETI_E_NOMEM, "allocation exceeds the context HBM budget");
    }
    void *q = nullptr;
    if (c->dev_alloc) {
        q = c->dev_alloc(n, c->alloc_user);
        if (!q) fail(NLFETI_E_NOMEM, "device allocator returned NULL");
    } else {
        cudaError_t e = cudaMalloc(&q, n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail(NLFETI_E_NOMEM, "cudaMalloc failed");
        }
    }
    p = q;
    bytes = n;
    std::lock_guard<std::mutex> g(c->mu);
    c->bytes_in_use += n;
}

void DevMem::alloc_async(cudaStream_t s, size_t n) {
    release();
    ctx = nullptr;
    async = true;
    astream = s;
    n = std::max<size_t>(n, 16);
    void *q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, n, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(NLFETI_E_NOMEM, "cudaMallocAsync failed");
    }
    p = q;
    bytes = n;
}

void DevMem::release() {
    if (!p) return;
    if (async) {
        cudaFreeAsync(p, astream);
    } else if (ctx) {
        if (ctx->dev_free) ctx->dev_free(p, ctx->alloc_user);
        else cudaFree(p);
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->bytes_in_use -= std::min(ctx->bytes_in_use, bytes);
    }
    p = nullptr;
    bytes = 0;
}

}  // namespace nlf

nlfeti_problem::~nlfeti_problem() = default;

using namespace nlf;

namespace {

template <typename F> nlfeti_status guarded(nlfeti_ctx *c, F &&f) {
    try {
        f();
        return NLFETI_OK;
    } catch (const Error &e) {
        set_error(c, e.msg);
        return e.st;
    } catch (const std::bad_alloc &) {
        set_error(c, "host allocation failed");
        return NLFETI_E_NOMEM;
    } catch (const std::exception &e) {
        set_error(c, e.what());
        return NLFETI_E_INVALID;
    }
}

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int round8(int n) { return (n + 7) / 8 * 8; }

void validate_mesh(const nlfeti_mesh *m) {
    if (!m || (m->dim != 1 && m->dim != 2)) fail(NLFETI_E_INVALID, "mesh dim must be 1 or 2");
    if (m->n_nodes <= 0 || m->n_elems <= 0) fail(NLFETI_E_INVALID, "empty mesh");
    if (m->n_nodes > INT32_MAX || m->n_elems > INT32_MAX) fail(NLFETI_E_INVALID, "mesh too large");
    if (!m->xy || !m->elems || !m->node_is_dirichlet || !m->elem_is_dirichlet) fail(NLFETI_E_INVALID, "null mesh array");
    const int nv = m->dim + 1;
    for (int64_t i = 0; i < m->n_elems * nv; ++i)
        if (m->elems[i] < 0 || m->elems[i] >= m->n_nodes) fail(NLFETI_E_INVALID, "element node index out of range");
    for (int64_t i = 0; i < m->n_nodes * m->dim; ++i)
        if (!std::isfinite(m->xy[i])) fail(NLFETI_E_INVALID, "non-finite node coordinate");
    bool any_dir = false;
    for (int64_t i = 0; i < m->n_nodes; ++i) any_dir |= m->node_is_dirichlet[i] != 0;
    if (!any_dir) fail(NLFETI_E_INVALID, "the Dirichlet volume constraint is empty");
}

void validate_kernel(const nlfeti_kernel *k, int dim) {
    if (!k) fail(NLFETI_E_INVALID, "null kernel");
    if (k->type < 0 || k->type > 3) fail(NLFETI_E_INVALID, "unknown kernel type");
    if (!(k->delta > 0) || !std::isfinite(k->delta)) fail(NLFETI_E_INVALID, "delta must be positive");
    if (!(k->scale > 0)) fail(NLFETI_E_INVALID, "kernel scale must be positive");
    if (k->type == NLFETI_K_FRACTIONAL && !(k->s > 0 && k->s < 1)) fail(NLFETI_E_INVALID, "fractional s must be in (0,1)");
    if (dim == 1 && k->type != NLFETI_K_CONST_LINF) fail(NLFETI_E_INVALID, "1-D meshes support the constant kernel only");
    if (k->ball < 0 || k->ball > 4) fail(NLFETI_E_INVALID, "unknown approximate ball");
    if (k->ball != 0 && (dim == 1 || k->type == NLFETI_K_CONST_LINF))
        fail(NLFETI_E_INVALID, "approximate balls apply to the 2-D l2 kernels only");
}

// approxcaps fills each cap with the triangle on its chord and the midpoint of its arc, which
// lies in E' when the arc is a minor arc; that holds for every element when 2 delta exceeds
// the longest element edge (an arc of at least half the circle inside E' would put two
// antipodal points, 2 delta apart, in E').
void validate_ball_mesh(const nlfeti_kernel *k, const nlfeti_mesh *m) {
    if (k->ball != 4) return;
    double longest = 0.0;
    for (int64_t e = 0; e < m->n_elems; ++e)
        for (int i = 0; i < 3; ++i) {
            const int32_t a = m->elems[3 * e + i], b = m->elems[3 * e + (i + 1) % 3];
            longest = std::max(longest, std::hypot(m->xy[2 * a] - m->xy[2 * b], m->xy[2 * a + 1] - m->xy[2 * b + 1]));
        }
    if (!(2.0 * k->delta > longest)) fail(NLFETI_E_INVALID, "approxcaps needs 2 delta above the longest element edge");
}

void build_maps(nlfeti_problem *p) {
    nlfeti_ctx *c = p->ctx;
    const Decomp &d = p->dec;
    const int K = d.K, nc = d.nc;
    const MeshHost &m = p->mesh;
    p->K = K;
    p->nc = nc;
    p->n_dofs_total = m.n_nodes * nc;
    p->n_lambda = (int64_t)d.B_plus.size();
    p->n_u = d.u_off[K];
    p->n_co = d.co_off[K];
    p->sd.assign(K, SubdomainDesc{});
    int64_t offA = 0, offAD = 0, offM = 0, offG = 0, offV = 0, offUp = 0, offVp = 0, offT = 0, offXp = 0;
    p->n_floating = 0;
    p->max_ldG = 8;
    for (int k = 0; k < K; ++k) {
        SubdomainDesc &s = p->sd[k];
        std::memset(&s, 0, sizeof(s));
        s.nk = (int32_t)d.nodes[k].size() * nc;
        s.nO = d.n_omega_nodes[k] * nc;
        s.nG = d.n_gamma_nodes[k] * nc;
        s.nD = (int32_t)d.dir_nodes[k].size() * nc;
        s.ldM = round8(s.nk);
        s.ldG = round8(std::max(s.nG, 1));
        s.offA = offA; offA += (int64_t)s.nk * s.nk;
        s.offAD = offAD; offAD += (int64_t)s.nk * s.nD;
        s.offM = offM; offM += (int64_t)s.nk * s.ldM;
        s.offS = offG; s.offSp = offG; offG += (int64_t)s.nG * s.ldG;
        s.offT = offT; offT += s.nG > 0 ? (int64_t)((s.nG + 127) / 128) * mma_ktiles(s.nG, s.ldG) : 0;
        s.offU = d.u_off[k];
        s.offUp = offUp; offUp += s.ldG;
        s.offXp = offXp; offXp += ldgx(s.ldG);
        s.offVp = offVp; offVp += s.ldM;
        s.offV = offV; offV += s.nk;
        s.co_off = d.co_off[k];
        s.n_co = d.co_off[k + 1] - d.co_off[k];
        s.floating = d.floating[k];
        s.npin = (int32_t)d.pinned[k].size();
        for (int i = 0; i < s.npin && i < 3; ++i) s.pin[i] = d.pinned[k][i];
        if (s.floating) p->n_floating++;
        p->max_ldG = std::max(p->max_ldG, s.ldG);
    }
    p->poolA = offA; p->poolAD = offAD; p->poolM = offM; p->poolG = offG; p->poolT = offT;
    p->sum_nk = offV;
    p->n_up = offUp;
    p->n_xp = offXp;
    p->n_vp = offVp;
    // node maps
    std::vector<int32_t> nodemap((size_t)K * m.n_nodes, -1);
    std::vector<int32_t> vdofs(offV);
    std::vector<int64_t> u2v(std::max<int64_t>(p->n_u, 1));
    std::vector<int32_t> u2sub(std::max<int64_t>(p->n_u, 1));
    std::vector<int32_t> ddofs;
    std::vector<int64_t> doff(K + 1, 0);
    for (int k = 0; k < K; ++k) {
        const auto &nd = d.nodes[k];
        for (size_t i = 0; i < nd.size(); ++i) {
            nodemap[(size_t)k * m.n_nodes + nd[i]] = (int32_t)i;
            for (int cc = 0; cc < nc; ++cc) vdofs[p->sd[k].offV + (int64_t)i * nc + cc] = nd[i] * nc + cc;
        }
        const auto &dn = d.dir_nodes[k];
        for (size_t i = 0; i < dn.size(); ++i) {
            nodemap[(size_t)k * m.n_nodes + dn[i]] = -(2 + (int32_t)i);
            for (int cc = 0; cc < nc; ++cc) ddofs.push_back(dn[i] * nc + cc);
        }
        doff[k + 1] = (int64_t)ddofs.size();
        for (int i = 0; i < p->sd[k].nG; ++i) {
            u2v[p->sd[k].offU + i] = p->sd[k].offV + p->sd[k].nO + i;
            u2sub[p->sd[k].offU + i] = k;
        }
    }
    // copies of each global dof
    std::vector<int64_t> cp_ptr(p->n_dofs_total + 1, 0), cp_pos(offV);
    for (int64_t v = 0; v < offV; ++v) cp_ptr[vdofs[v] + 1]++;
    for (int64_t i = 0; i < p->n_dofs_total; ++i) cp_ptr[i + 1] += cp_ptr[i];
    {
        std::vector<int64_t> fill(cp_ptr.begin(), cp_ptr.end() - 1);
        for (int64_t v = 0; v < offV; ++v) cp_pos[fill[vdofs[v]]++] = v;
    }
    std::vector<double> zeta(p->n_dofs_total, 1.0);
    for (int64_t n = 0; n < m.n_nodes; ++n)
        for (int cc = 0; cc < nc; ++cc) zeta[n * nc + cc] = d.node_zeta[n] > 0 ? (double)d.node_zeta[n] : 1.0;
    // B^T (signed rows) per U dof
    std::vector<int64_t> bt_ptr(p->n_u + 1, 0), bt_row(2 * p->n_lambda);
    for (int64_t r = 0; r < p->n_lambda; ++r) { bt_ptr[d.B_plus[r] + 1]++; bt_ptr[d.B_minus[r] + 1]++; }
    for (int64_t u = 0; u < p->n_u; ++u) bt_ptr[u + 1] += bt_ptr[u];
    {
        std::vector<int64_t> fill(bt_ptr.begin(), bt_ptr.end() - 1);
        for (int64_t r = 0; r < p->n_lambda; ++r) {
            bt_row[fill[d.B_plus[r]]++] = r + 1;
            bt_row[fill[d.B_minus[r]]++] = -(r + 1);
        }
    }
    // interior elements around each node (load vector)
    const int nv = m.dim + 1;
    std::vector<int64_t> inc_ptr(m.n_nodes + 1, 0);
    for (int64_t e = 0; e < m.n_elems; ++e)
        if (!m.elem_dir[e])
            for (int i = 0; i < nv; ++i) inc_ptr[m.elems[e * nv + i] + 1]++;
    for (int64_t i = 0; i < m.n_nodes; ++i) inc_ptr[i + 1] += inc_ptr[i];
    std::vector<int32_t> inc_el(std::max<int64_t>(inc_ptr[m.n_nodes], 1));
    {
        std::vector<int64_t> fill(inc_ptr.begin(), inc_ptr.end() - 1);
        for (int64_t e = 0; e < m.n_elems; ++e)
            if (!m.elem_dir[e])
                for (int i = 0; i < nv; ++i) inc_el[fill[m.elems[e * nv + i]]++] = (int32_t)e;
    }
    // apply work items: kApplyRows rows each
    std::vector<int32_t> items;
    p->item_off.assign(K + 1, 0);
    for (int k = 0; k < K; ++k) {
        for (int r0 = 0; r0 < p->sd[k].nG; r0 += kApplyRows) { items.push_back(k); items.push_back(r0); }
        p->item_off[k + 1] = (int)(items.size() / 2);
    }
    p->n_items = (int)(items.size() / 2);
    std::vector<int32_t> items_o;
    p->item_off_o.assign(K + 1, 0);
    for (int k = 0; k < K; ++k) {
        for (int r0 = 0; r0 < p->sd[k].nO; r0 += kApplyRows) { items_o.push_back(k); items_o.push_back(r0); }
        p->item_off_o[k + 1] = (int)(items_o.size() / 2);
    }
    upload(c, p->d_items_o, items_o);
    // persistent schedules of the bulk-copy apply (items over Gamma rows) and of the residual
    // (items over all rows of A^k): longest item first onto the least loaded CTA (cost = rows x
    // streamed columns), then each CTA's list in (subdomain, row) order
    auto schedule = [&](const std::vector<int32_t> &its, int ctas, auto rows_cols, DevMem &dptr, DevMem &ditems) {
        const int n = (int)(its.size() / 2);
        const int G = std::max(1, std::min(ctas, std::max(1, n)));
        std::vector<std::pair<int64_t, int>> order;     // (cost, item)
        for (int t = 0; t < n; ++t) {
            const auto rc = rows_cols(p->sd[its[2 * t]], its[2 * t + 1]);
            order.push_back({(int64_t)rc.first * rc.second + 256, t});
        }
        std::stable_sort(order.begin(), order.end(), [](auto a, auto b) { return a.first > b.first; });
        std::vector<int64_t> load(G, 0);
        std::vector<std::vector<int>> lists(G);
        for (auto &o : order) {
            const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            load[b] += o.first;
            lists[b].push_back(o.second);
        }
        std::vector<int32_t> sptr(G + 1, 0), sitems;
        for (int b = 0; b < G; ++b) {
            std::sort(lists[b].begin(), lists[b].end());
            for (int t : lists[b]) { sitems.push_back(its[2 * t]); sitems.push_back(its[2 * t + 1]); }
            sptr[b + 1] = (int32_t)(sitems.size() / 2);
        }
        upload(c, dptr, sptr);
        upload(c, ditems, sitems);
        return G;
    };
    p->sched_ctas = schedule(items, apply_tma_ctas(), [](const SubdomainDesc &s, int r0) {
        return std::make_pair(std::min(kApplyRows, s.nG - r0), std::min<int64_t>(s.ldG, (s.nG + 7) / 8 * 8));
    }, p->d_sched_ptr, p->d_sched_items);
    p->sched1_ctas = items.empty() ? 0 : schedule(items, device_sms(),
                                                 [](const SubdomainDesc &s, int r0) {
        return std::make_pair(std::min(kApplyRows, s.nG - r0), std::min<int64_t>(s.ldG, (s.nG + 7) / 8 * 8));
    }, p->d_sched1_ptr, p->d_sched1_items);
    p->fsched_ctas = schedule(items, apply_tma_ctas(), [](const SubdomainDesc &s, int r0) {
        return std::make_pair(std::min(kApplyRows, s.nG - r0), (int64_t)(s.nO + 7) / 8 * 8);
    }, p->d_fsched_ptr, p->d_fsched_items);
    p->osched_ctas = items_o.empty() ? 0 : schedule(items_o, apply_tma_ctas(), [](const SubdomainDesc &s, int r0) {
        return std::make_pair(std::min(kApplyRows, s.nO - r0), std::min<int64_t>(s.ldM, (s.nk + 7) / 8 * 8));
    }, p->d_osched_ptr, p->d_osched_items);
    {
        // tensor-core preconditioner apply: 128-row items, 64-column stages
        std::vector<int32_t> items_m;
        for (int k = 0; k < K; ++k)
            for (int r0 = 0; r0 < p->sd[k].nG; r0 += 128) { items_m.push_back(k); items_m.push_back(r0); }
        p->msched_ctas = items_m.empty() ? 0 : schedule(items_m, apply_mma_ctas(), [](const SubdomainDesc &s, int) {
            return std::make_pair(128, (std::min<int64_t>(s.ldG, (s.nG + 7) / 8 * 8) + 63) / 64 * 64);
        }, p->d_msched_ptr, p->d_msched_items);
        p->mitem_off.assign(K + 1, 0);
        int most = 1;
        for (int k = 0; k < K; ++k) {
            const int nk_items = (p->sd[k].nG + 127) / 128;
            p->mitem_off[k + 1] = p->mitem_off[k] + nk_items;
            most = std::max(most, nk_items);
        }
        std::vector<int32_t> iota(most + 1);
        for (int i = 0; i <= most; ++i) iota[i] = i;
        if (!items_m.empty()) upload(c, p->d_mitems, items_m);
        upload(c, p->d_iota, iota);
    }
    {
        std::vector<int32_t> items_a;
        for (int k = 0; k < K; ++k)
            for (int r0 = 0; r0 < p->sd[k].nk; r0 += 32) { items_a.push_back(k); items_a.push_back(r0); }
        p->rsched_ctas = items_a.empty() ? 0 : schedule(items_a, residual_tma_ctas(), [](const SubdomainDesc &s, int r0) {
            return std::make_pair(std::min(32, s.nk - r0), (int64_t)s.ldM);
        }, p->d_rsched_ptr, p->d_rsched_items);
    }
    std::vector<uint64_t> mask = d.elem_mask;
    upload(c, p->d_sd, p->sd);
    upload(c, p->d_xy, m.xy);
    upload(c, p->d_elems, m.elems);
    upload(c, p->d_node_dir, m.node_dir);
    upload(c, p->d_elem_mask, mask);
    upload(c, p->d_nodemap, nodemap);
    upload(c, p->d_vdofs, vdofs);
    upload(c, p->d_u2v, u2v);
    upload(c, p->d_u2sub, u2sub);
    upload(c, p->d_ddofs, ddofs);
    upload(c, p->d_doff, doff);
    upload(c, p->d_cp_ptr, cp_ptr);
    upload(c, p->d_cp_pos, cp_pos);
    upload(c, p->d_zeta_dof, zeta);
    upload(c, p->d_Bp, d.B_plus);
    upload(c, p->d_Bm, d.B_minus);
    upload(c, p->d_Bt_ptr, bt_ptr);
    upload(c, p->d_Bt_row, bt_row);
    upload(c, p->d_nodeinc_ptr, inc_ptr);
    upload(c, p->d_nodeinc_el, inc_el);
    upload(c, p->d_items, items);
    p->d_flag.alloc(c, sizeof(int) * 4);
    NLF_CUDA(cudaMemsetAsync(p->d_flag.p, 0, sizeof(int) * 4, c->stream));
    p->d_A.alloc(c, sizeof(double) * std::max<int64_t>(offA, 1));
    p->d_AD.alloc(c, sizeof(double) * std::max<int64_t>(offAD, 1));
    NLF_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace

extern "C" {

void nlfeti_default_options(nlfeti_options *o) {
    if (!o) return;
    o->precision = 0;
    o->tol = 1e-10;
    o->max_it = 1000;
    o->max_refine = 10;
    o->inner_tol = 1e-3;
    o->refine_tol = 1e-9;
    o->batched = 1;
    o->hbm_budget = 0;
    o->graph_loop = 1;
    o->precond_fp16 = 1;
    o->factor_tc = 2;
    o->residual_format = 0;
}

nlfeti_status nlfeti_create(nlfeti_ctx **out, const nlfeti_options *opt, void *cuda_stream,
                            void *(*dev_alloc)(size_t, void *), void (*dev_free)(void *, void *), void *alloc_user) {
    if (!out) return NLFETI_E_INVALID;
    if ((dev_alloc == nullptr) != (dev_free == nullptr)) return NLFETI_E_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return NLFETI_E_CUDA;
    }
    nlfeti_ctx *c = new (std::nothrow) nlfeti_ctx();
    if (!c) return NLFETI_E_NOMEM;
    nlfeti_default_options(&c->opt);
    if (opt) c->opt = *opt;
    c->user_stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return NLFETI_E_CUDA;
    }
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return NLFETI_E_CUDA;
    }
    c->dev_alloc = dev_alloc;
    c->dev_free = dev_free;
    c->alloc_user = alloc_user;
    *out = c;
    return NLFETI_OK;
}

static void ctx_free(nlfeti_ctx *ctx) {
    if (ctx->stream) {
        cudaStreamSynchronize(ctx->stream);
        cudaStreamDestroy(ctx->stream);
    }
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    delete ctx;
}

// A context outlives its problems and servers: destroying it while they are alive only
// marks it, and the last of them to be destroyed frees it.
void nlfeti_destroy(nlfeti_ctx *ctx) {
    if (!ctx) return;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        if (ctx->children > 0) {
            ctx->destroy_pending = true;
            return;
        }
    }
    ctx_free(ctx);
}

}  // extern "C"

namespace nlf {
void ctx_attach(nlfeti_ctx *c) {
    std::lock_guard<std::mutex> g(c->mu);
    c->children++;
}

void ctx_detach(nlfeti_ctx *c) {
    bool free_now;
    {
        std::lock_guard<std::mutex> g(c->mu);
        c->children--;
        free_now = c->destroy_pending && c->children == 0;
    }
    if (free_now) ctx_free(c);
}
}  // namespace nlf

namespace nlf {

// Device bytes a problem holds once created and factored with the precisions of mask (bit 0
// FP64, bit 1 FP32): the assembled matrices, the operator pools in the layout of build_maps,
// the sweep scratch and the node maps, plus a margin for the index maps and tensor maps.
size_t problem_bytes(const Decomp &d, int64_t n_nodes, int mask) {
    const int K = d.K, nc = d.nc;
    double b = 0, sum_nk = 0;
    for (int k = 0; k < K; ++k) {
        const double nk = (double)d.nodes[k].size() * nc, nG = (double)d.n_gamma_nodes[k] * nc;
        const double nD = (double)d.dir_nodes[k].size() * nc;
        const double ldM = (double)round8((int)nk), ldG = (double)round8(std::max((int)nG, 1));
        sum_nk += nk;
        b += 8.0 * nk * nk + 8.0 * nk * nD;                               // A^k and its Dirichlet block
        if (mask & 1) b += 8.0 * nk * ldM + 2 * 8.0 * nG * ldG;           // FP64 swept matrix, S, S^+
        if (mask & 2) b += 4.0 * nk * ldM * 3 + 2 * 4.0 * nG * ldG + 2.0 * nG * ldG;   // FP32 + A pairs, S, S^+, FP16 S
    }
    const double scr = sum_nk * 64 * 2 + (double)K * 64 * 64;              // sweep panels
    if (mask & 1) b += 8.0 * scr;
    if (mask & 2) b += 4.0 * scr;
    b += 4.0 * (double)K * (double)n_nodes;                               // node -> subdomain-local maps
    b += 64.0 * sum_nk;                                                   // index maps, vectors, tensor maps
    // (G^T G)^-1 in FP64 and its FP32 copy, at most every subdomain floating (1 kernel vector
    // per scalar subdomain, 3 rigid modes per 2-D peridynamic one)
    const double nco = (double)K * (nc == 1 ? 1 : 3);
    b += 8.0 * nco * nco + ((mask & 2) ? 4.0 * nco * nco : 0.0);
    return (size_t)(b * 1.05) + (size_t(16) << 20);
}

size_t predict_problem_bytes(const nlfeti_mesh *mesh, const nlfeti_kernel *kernel, const nlfeti_decomp *decomp,
                             int mask) {
    validate_mesh(mesh);
    validate_kernel(kernel, mesh->dim);
    validate_ball_mesh(kernel, mesh);
    if (!decomp || !decomp->elem_subdomain) fail(NLFETI_E_INVALID, "null decomposition");
    MeshHost m;
    m.dim = mesh->dim;
    m.n_nodes = mesh->n_nodes;
    m.n_elems = mesh->n_elems;
    m.xy.assign(mesh->xy, mesh->xy + mesh->n_nodes * mesh->dim);
    m.elems.assign(mesh->elems, mesh->elems + mesh->n_elems * (mesh->dim + 1));
    m.node_dir.assign(mesh->node_is_dirichlet, mesh->node_is_dirichlet + mesh->n_nodes);
    m.elem_dir.assign(mesh->elem_is_dirichlet, mesh->elem_is_dirichlet + mesh->n_elems);
    std::vector<int32_t> labels(decomp->elem_subdomain, decomp->elem_subdomain + mesh->n_elems);
    Decomp d;
    build_decomposition(m, *kernel, labels, decomp->K, d);
    return problem_bytes(d, mesh->n_nodes, mask);
}

}  // namespace nlf

extern "C" {

const char *nlfeti_last_error(const nlfeti_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

nlfeti_status nlfeti_problem_create(nlfeti_ctx *ctx, const nlfeti_mesh *mesh, const nlfeti_kernel *kernel,
                                    const nlfeti_decomp *decomp, nlfeti_problem **out) {
    if (!ctx || !out) return NLFETI_E_INVALID;
    nlfeti_problem *p = nullptr;
    nlfeti_status st = guarded(ctx, [&] {
        double t0 = now_ms();
        validate_mesh(mesh);
        validate_kernel(kernel, mesh->dim);
        validate_ball_mesh(kernel, mesh);
        if (!decomp || !decomp->elem_subdomain) fail(NLFETI_E_INVALID, "null decomposition");
        std::unique_ptr<nlfeti_problem> q(new nlfeti_problem());
        static std::atomic<uint64_t> next_uid{1};
        q->uid = next_uid++;
        q->ctx = ctx;
        q->opt = ctx->opt;
        q->kern = *kernel;
        MeshHost &m = q->mesh;
        m.dim = mesh->dim;
        m.n_nodes = mesh->n_nodes;
        m.n_elems = mesh->n_elems;
        m.xy.assign(mesh->xy, mesh->xy + mesh->n_nodes * mesh->dim);
        m.elems.assign(mesh->elems, mesh->elems + mesh->n_elems * (mesh->dim + 1));
        m.node_dir.assign(mesh->node_is_dirichlet, mesh->node_is_dirichlet + mesh->n_nodes);
        m.elem_dir.assign(mesh->elem_is_dirichlet, mesh->elem_is_dirichlet + mesh->n_elems);
        std::vector<int32_t> labels(decomp->elem_subdomain, decomp->elem_subdomain + mesh->n_elems);
        build_decomposition(m, *kernel, labels, decomp->K, q->dec);
        build_maps(q.get());
        assemble_all(q.get());
        setup_jump_weights(q.get());
        setup_coarse(q.get());
        int flag[4] = {0, 0, 0, 0};
        NLF_CUDA(cudaMemcpy(flag, q->d_flag.p, sizeof(flag), cudaMemcpyDeviceToHost));
        if (flag[1]) fail(NLFETI_E_INVALID, "an interface node belongs to more than 16 subdomains");
        if (flag[0]) fail(NLFETI_E_NOT_SPD, "the coarse matrix G^T G is not positive definite");
        q->ms_setup = now_ms() - t0;
        p = q.release();
    });
    if (st == NLFETI_OK) {
        ctx_attach(ctx);
        *out = p;
    }
    return st;
}

void nlfeti_problem_destroy(nlfeti_problem *p) {
    if (!p) return;
    nlfeti_ctx *c = p->ctx;
    if (c && c->stream) cudaStreamSynchronize(c->stream);
    delete p;
    if (c) ctx_detach(c);
}

nlfeti_status nlfeti_problem_info(const nlfeti_problem *p, nlfeti_info *info) {
    if (!p || !info) return NLFETI_E_INVALID;
    info->K = p->K;
    info->ncomp = p->nc;
    info->n_floating = p->n_floating;
    info->n_coarse = p->n_co;
    info->n_lambda = p->n_lambda;
    info->n_u = p->n_u;
    info->sum_nk = p->sum_nk;
    int64_t s2 = 0, g2 = 0;
    int mk = 0, mg = 0;
    for (auto &d : p->sd) {
        s2 += (int64_t)d.nk * d.nk;
        g2 += (int64_t)d.nG * d.nG;
        mk = std::max(mk, d.nk);
        mg = std::max(mg, d.nG);
    }
    info->sum_nk2 = s2;
    info->sum_ngamma2 = g2;
    info->max_nk = mk;
    info->max_ngamma = mg;
    info->residual_nnz = (p->op32.ready && p->op32.a_sparse) ? p->op32.a_nnz : 0;
    return NLFETI_OK;
}

nlfeti_status nlfeti_problem_set_options(nlfeti_problem *p, const nlfeti_options *opt) {
    if (!p || !opt) return NLFETI_E_INVALID;
    if (opt->precision != 0 && opt->precision != 1) return NLFETI_E_INVALID;
    if (opt->precond_fp16 < 0 || opt->precond_fp16 > 2) return NLFETI_E_INVALID;
    if (opt->factor_tc < 0 || opt->factor_tc > 2) return NLFETI_E_INVALID;
    if (opt->residual_format < 0 || opt->residual_format > 2) return NLFETI_E_INVALID;
    return guarded(p->ctx, [&] {
        p->opt = *opt;
        if (p->opt.precond_fp16 == 2 && p->op32.ready) build_tiled_half(p);
    });
}

nlfeti_status nlfeti_factor(nlfeti_problem *p, int mask) {
    if (!p) return NLFETI_E_INVALID;
    return guarded(p->ctx, [&] {
        if (mask & ~3) fail(NLFETI_E_INVALID, "precision mask must use bits 0 and 1");
        double t0 = now_ms();
        ++p->factor_gen;
        if (mask & 1) factor_ops<double>(p, p->op64);
        if (mask & 2) factor_ops<float>(p, p->op32);
        p->ms_factor = now_ms() - t0;
    });
}

}  // extern "C"

namespace {
using SolveFn = void (*)(nlfeti_problem *, SolveWS &, cudaStream_t, int, int, const double *, const double *, double *,
                         nlfeti_stats *);

nlfeti_status solve_on_device(nlfeti_problem *p, SolveFn fn, int nrhs, int rhs_kind, const double *d_rhs,
                              const double *d_g, double *d_u_out, nlfeti_stats *stats) {
    if (!p) return NLFETI_E_INVALID;
    return guarded(p->ctx, [&] {
        if (nrhs < 1 || (rhs_kind != 0 && rhs_kind != 1) || !d_rhs || !d_u_out) fail(NLFETI_E_INVALID, "bad solve arguments");
        if (!p->ws) p->ws.reset(new SolveWS());
        double t0 = now_ms();
        nlfeti_stats s{};
        stream_enter(p->ctx);
        try {
            fn(p, *p->ws, p->ctx->stream, nrhs, rhs_kind, d_rhs, d_g, d_u_out, &s);
        } catch (...) {
            if (stats) *stats = s;
            stream_leave(p->ctx);
            throw;
        }
        stream_leave(p->ctx);
        s.ms_setup = p->ms_setup;
        s.ms_factor = p->ms_factor;
        s.ms_solve = now_ms() - t0;
        if (stats) *stats = s;
    });
}

nlfeti_status solve_on_host(nlfeti_problem *p, SolveFn fn, int nrhs, int rhs_kind, const double *rhs, const double *g,
                            double *u_out, nlfeti_stats *stats) {
    if (!p) return NLFETI_E_INVALID;
    return guarded(p->ctx, [&] {
        if (nrhs < 1 || (rhs_kind != 0 && rhs_kind != 1) || !rhs || !u_out) fail(NLFETI_E_INVALID, "bad solve arguments");
        if (!p->ws) p->ws.reset(new SolveWS());
        SolveWS &ws = *p->ws;
        cudaStream_t st = p->ctx->stream;
        const size_t bytes = sizeof(double) * (size_t)p->n_dofs_total * nrhs;
        if (ws.in_rhs.bytes < bytes) ws.in_rhs.alloc(p->ctx, bytes);
        if (ws.out_u.bytes < bytes) ws.out_u.alloc(p->ctx, bytes);
        if (g && ws.in_g.bytes < bytes) ws.in_g.alloc(p->ctx, bytes);
        double t0 = now_ms();
        NLF_CUDA(cudaMemcpyAsync(ws.in_rhs.p, rhs, bytes, cudaMemcpyHostToDevice, st));
        if (g) NLF_CUDA(cudaMemcpyAsync(ws.in_g.p, g, bytes, cudaMemcpyHostToDevice, st));
        nlfeti_stats s{};
        nlfeti_status inner = NLFETI_OK;
        try {
            fn(p, ws, st, nrhs, rhs_kind, ws.in_rhs.as<double>(), g ? ws.in_g.as<double>() : nullptr,
               ws.out_u.as<double>(), &s);
        } catch (const Error &e) {
            if (e.st != NLFETI_E_NOT_CONVERGED) throw;
            inner = e.st;
            set_error(p->ctx, e.msg);
        }
        NLF_CUDA(cudaMemcpyAsync(u_out, ws.out_u.p, bytes, cudaMemcpyDeviceToHost, st));
        NLF_CUDA(cudaStreamSynchronize(st));
        s.ms_setup = p->ms_setup;
        s.ms_factor = p->ms_factor;
        s.ms_solve = now_ms() - t0;
        if (stats) *stats = s;
        if (inner != NLFETI_OK) fail(inner, p->ctx->err);
    });
}
}  // namespace

extern "C" {

nlfeti_status nlfeti_solve_device(nlfeti_problem *p, int nrhs, int rhs_kind, const double *d_rhs, const double *d_g,
                                  double *d_u_out, nlfeti_stats *stats) {
    return solve_on_device(p, solve_device, nrhs, rhs_kind, d_rhs, d_g, d_u_out, stats);
}

nlfeti_status nlfeti_solve(nlfeti_problem *p, int nrhs, int rhs_kind, const double *rhs, const double *g,
                           double *u_out, nlfeti_stats *stats) {
    return solve_on_host(p, solve_device, nrhs, rhs_kind, rhs, g, u_out, stats);
}

nlfeti_status nlfeti_cg_prepare(nlfeti_problem *p) {
    if (!p) return NLFETI_E_INVALID;
    return guarded(p->ctx, [&] { cg_prepare(p); });
}

nlfeti_status nlfeti_solve_cg_device(nlfeti_problem *p, int nrhs, int rhs_kind, const double *d_rhs, const double *d_g,
                                     double *d_u_out, nlfeti_stats *stats) {
    return solve_on_device(p, cg_solve_device, nrhs, rhs_kind, d_rhs, d_g, d_u_out, stats);
}

nlfeti_status nlfeti_solve_cg(nlfeti_problem *p, int nrhs, int rhs_kind, const double *rhs, const double *g,
                              double *u_out, nlfeti_stats *stats) {
    return solve_on_host(p, cg_solve_device, nrhs, rhs_kind, rhs, g, u_out, stats);
}

nlfeti_status nlfeti_set_profiling(nlfeti_problem *p, int on) {
    if (!p) return NLFETI_E_INVALID;
    p->prof_on = on != 0;
    return NLFETI_OK;
}

nlfeti_status nlfeti_get_profile(nlfeti_problem *p, nlfeti_profile *out) {
    if (!p || !out) return NLFETI_E_INVALID;
    std::lock_guard<std::mutex> g(p->prof_mu);
    *out = p->prof;
    p->prof = nlfeti_profile{};
    return NLFETI_OK;
}

nlfeti_status nlfeti_get_decomposition(const nlfeti_problem *p, int32_t *n_k, int32_t *n_gamma, int32_t *node_lists,
                                       int64_t *B_plus, int64_t *B_minus, int8_t *floating) {
    if (!p) return NLFETI_E_INVALID;
    int64_t off = 0;
    for (int k = 0; k < p->K; ++k) {
        if (n_k) n_k[k] = p->sd[k].nk;
        if (n_gamma) n_gamma[k] = p->sd[k].nG;
        if (floating) floating[k] = p->dec.floating[k];
        if (node_lists) std::copy(p->dec.nodes[k].begin(), p->dec.nodes[k].end(), node_lists + off);
        off += (int64_t)p->dec.nodes[k].size();
    }
    if (B_plus) std::copy(p->dec.B_plus.begin(), p->dec.B_plus.end(), B_plus);
    if (B_minus) std::copy(p->dec.B_minus.begin(), p->dec.B_minus.end(), B_minus);
    return NLFETI_OK;
}

nlfeti_status nlfeti_autotune(nlfeti_problem *p, int nrhs, const char *cache_path, nlfeti_tune_entry *out,
                              int *n_out) {
    if (!p || nrhs < 1) return NLFETI_E_INVALID;
    return guarded(p->ctx, [&] {
        std::vector<TuneEntry> res;
        autotune_applies(p, nrhs, cache_path, res);
        if (n_out) *n_out = (int)res.size();
        if (out)
            for (size_t i = 0; i < res.size() && i < 3; ++i) {
                out[i].kind = res[i].kind;
                out[i].nrhs = res[i].R;
                out[i].rc = res[i].rc;
                out[i].ctas_per_sm = res[i].per_sm;
                out[i].us = res[i].us;
                out[i].from_cache = res[i].from_cache ? 1 : 0;
                out[i].rows_per_warp = res[i].rpw;
            }
    });
}

nlfeti_status nlfeti_set_apply_choice(nlfeti_problem *p, int kind, int nrhs, int rc, int ctas_per_sm,
                                      int rows_per_warp) {
    if (!p || kind < 0 || kind > 2 || nrhs < 1) return NLFETI_E_INVALID;
    if (rows_per_warp == 0) rows_per_warp = 4;
    return guarded(p->ctx, [&] {
        if (rc == 0) {
            p->tune.erase({kind, nrhs});
        } else if (rc == -1) {
            if (kind != 1 || nrhs > MMA_MAX_RHS || !p->op32.ready)
                fail(NLFETI_E_INVALID, "the tensor-core apply serves the FP16 copy of S_k (kind 1), at most 64 "
                                       "right-hand sides, with FP32 operators factored");
            build_tiled_half(p);
            p->tune[{kind, nrhs}] = ApplyChoice{0, 2, 1};
        } else {
            const bool pow2 = rc == 1 || rc == 2 || rc == 4 || rc == 8 || rc == 16;
            if (!pow2 || (kind == 2 && rc > 8) || (rc > nrhs && rc > 1) || (ctas_per_sm != 1 && ctas_per_sm != 2))
                fail(NLFETI_E_INVALID, "column block must be 1, 2, 4, 8 or 16 (8 for FP64) and at most nrhs; "
                                       "CTAs per SM 1 or 2");
            if (rows_per_warp != 4 && (rows_per_warp != 8 || kind == 2 || rc < 4))
                fail(NLFETI_E_INVALID, "rows per warp must be 4, or 8 for the FP32 and FP16 operators with a "
                                       "column block of at least 4");
            p->tune[{kind, nrhs}] = ApplyChoice{rc, ctas_per_sm, 0, rows_per_warp};
        }
        ++p->tune_gen;
    });
}

nlfeti_status nlfeti_debug_apply_waits(nlfeti_problem *p, long long wait_tries, int withhold_copies) {
    if (!p || wait_tries < 0 || (withhold_copies != 0 && withhold_copies != 1)) return NLFETI_E_INVALID;
    p->dbg_wait_tries = wait_tries;
    p->dbg_withhold = withhold_copies;
    return NLFETI_OK;
}

nlfeti_status nlfeti_problem_set_matrix(nlfeti_problem *p, int k, const double *A) {
    if (!p || !A || k < 0 || k >= p->K) return NLFETI_E_INVALID;
    return guarded(p->ctx, [&] {
        const SubdomainDesc &d = p->sd[k];
        const size_t n = (size_t)d.nk * (size_t)d.nk;
        for (size_t t = 0; t < n; ++t)
            if (!std::isfinite(A[t])) fail(NLFETI_E_INVALID, "the subdomain matrix has a non-finite entry");
        if (n) NLF_CUDA(cudaMemcpy(p->d_A.as<double>() + d.offA, A, sizeof(double) * n, cudaMemcpyHostToDevice));
        // every operator derived from A^k is stale: refactor before the next solve
        p->op64.ready = false;
        p->op32.ready = false;
        p->cg_ready = false;
        ++p->factor_gen;
    });
}

nlfeti_status nlfeti_get_operator(const nlfeti_problem *p, int k, int which, int precision, double *out) {
    if (!p || !out || k < 0 || k >= p->K) return NLFETI_E_INVALID;
    nlfeti_problem *q = const_cast<nlfeti_problem *>(p);
    return guarded(q->ctx, [&] {
        const SubdomainDesc &d = p->sd[k];
        if (which == 0) {
            NLF_CUDA(cudaMemcpy(out, p->d_A.as<double>() + d.offA, sizeof(double) * d.nk * d.nk, cudaMemcpyDeviceToHost));
            return;
        }
        if (which != 1 && which != 2) fail(NLFETI_E_INVALID, "which must be 0, 1 or 2");
        const int64_t n = d.nG, ld = d.ldG;
        const int64_t off = which == 1 ? d.offS : d.offSp;
        if (precision == 0) {
            if (!p->op64.ready) fail(NLFETI_E_INVALID, "FP64 operators not factored");
            std::vector<double> tmp(n * ld);
            const nlf::DevMem &src = which == 1 ? p->op64.S : p->op64.Sp;
            if (n) NLF_CUDA(cudaMemcpy(tmp.data(), src.as<double>() + off, sizeof(double) * n * ld, cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < n; ++i)
                for (int64_t l = 0; l < n; ++l) out[i * n + l] = tmp[i * ld + l];
        } else {
            if (!p->op32.ready) fail(NLFETI_E_INVALID, "FP32 operators not factored");
            std::vector<float> tmp(n * ld);
            const nlf::DevMem &src = which == 1 ? p->op32.S : p->op32.Sp;
            if (n) NLF_CUDA(cudaMemcpy(tmp.data(), src.as<float>() + off, sizeof(float) * n * ld, cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < n; ++i)
                for (int64_t l = 0; l < n; ++l) out[i * n + l] = tmp[i * ld + l];
        }
    });
}

nlfeti_status nlfeti_apply(nlfeti_problem *p, int op, int precision, int nrhs, const double *in, double *out) {
    if (!p || !in || !out || nrhs < 1) return NLFETI_E_INVALID;
    return guarded(p->ctx, [&] {
        if (op < 0 || op > 5) fail(NLFETI_E_INVALID, "unknown operator");
        const int64_t n = (op <= 2) ? p->n_lambda : p->n_u;
        if (n == 0) return;
        cudaStream_t st = p->ctx->stream;
        DevMem a, b, ai, bi;
        a.alloc(p->ctx, sizeof(double) * n * nrhs);
        b.alloc(p->ctx, sizeof(double) * n * nrhs);
        ai.alloc(p->ctx, sizeof(double) * n * nrhs);
        bi.alloc(p->ctx, sizeof(double) * n * nrhs);
        NLF_CUDA(cudaMemcpyAsync(a.p, in, sizeof(double) * n * nrhs, cudaMemcpyHostToDevice, st));
        to_interleaved(a.as<double>(), ai.as<double>(), n, nrhs, st);
        SolveWS ws;
        apply_operator(p, ws, st, op, precision, nrhs, ai.as<double>(), bi.as<double>());
        to_colmajor(bi.as<double>(), b.as<double>(), n, nrhs, st);
        NLF_CUDA(cudaMemcpyAsync(out, b.p, sizeof(double) * n * nrhs, cudaMemcpyDeviceToHost, st));
        NLF_CUDA(cudaStreamSynchronize(st));
    });
}

}  // extern "C"
