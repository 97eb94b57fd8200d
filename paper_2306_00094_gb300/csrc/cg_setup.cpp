// Global matrix of the single-domain system for the diagonally preconditioned CG that the
// paper uses as its performance baseline (section "Considered solver strategies": CG with a
// diagonal preconditioner on the discrete nonlocal problem, rows distributed without
// duplicated unknowns).
//
// The subdomain matrices A^k carry the zeta weights of the subdivision, so that
// sum_k R_k^T A^k R_k is the single-domain matrix A on the non-Dirichlet dofs (the partition
// of unity of the zeta weights, eqs. bilinear-multi1..5).  Row g of A is therefore the sum,
// over the subdomain copies of dof g (ascending subdomain), of their rows of A^k mapped to
// global columns.  The rows are assembled on the host from a copy of the A^k (exact zeros of
// non-interacting pairs are dropped), by row ranges on several threads, into CSR: int64 row
// pointers, int32 columns ascending, FP64 values.  Dofs without a subdomain copy (Dirichlet
// dofs) get an identity row.  The values are kept on the device as FP32 pairs
// (hi = fl32(a), lo = fl32(a - hi), 2^-48 relative), the operands of the double-single
// product of the CG (FP64 accuracy on the FP32 pipes).  Setup only: the solve runs on the
// device (iterate.cu).
#include <algorithm>
#include <thread>

#include "internal.hpp"

namespace nlf {

namespace {
template <typename T> std::vector<T> download(const DevMem &m, size_t n) {
    std::vector<T> v(n);
    if (n) NLF_CUDA(cudaMemcpy(v.data(), m.p, sizeof(T) * n, cudaMemcpyDeviceToHost));
    return v;
}
}  // namespace

void cg_prepare(nlfeti_problem *p) {
    if (p->cg_ready) return;
    nlfeti_ctx *c = p->ctx;
    NLF_CUDA(cudaStreamSynchronize(c->stream));
    const int64_t n = p->n_dofs_total, nv = p->sum_nk;
    const int K = p->K;
    int64_t na = 0;
    for (const auto &d : p->sd) na = std::max<int64_t>(na, d.offA + (int64_t)d.nk * d.nk);
    const std::vector<double> A = download<double>(p->d_A, (size_t)na);
    const std::vector<int32_t> vdofs = download<int32_t>(p->d_vdofs, (size_t)nv);
    const std::vector<int64_t> cp_ptr = download<int64_t>(p->d_cp_ptr, (size_t)n + 1);
    const std::vector<int64_t> cp_pos = download<int64_t>(p->d_cp_pos, (size_t)cp_ptr[n]);
    // subdomain of each subdomain-vector entry
    std::vector<int32_t> v2k((size_t)nv);
    for (int k = 0; k < K; ++k)
        for (int32_t i = 0; i < p->sd[k].nk; ++i) v2k[p->sd[k].offV + i] = k;

    const int T = (int)std::max<unsigned>(1, std::min<unsigned>(16, std::thread::hardware_concurrency()));
    struct Chunk {
        std::vector<int64_t> len;
        std::vector<int32_t> col;
        std::vector<double> val, diag;
    };
    std::vector<Chunk> ch(T);
    auto work = [&](int t) {
        const int64_t g0 = n * t / T, g1 = n * (t + 1) / T;
        Chunk &o = ch[t];
        std::vector<double> acc((size_t)n, 0.0);
        std::vector<char> mark((size_t)n, 0);
        std::vector<int32_t> touched;
        for (int64_t g = g0; g < g1; ++g) {
            touched.clear();
            for (int64_t q = cp_ptr[g]; q < cp_ptr[g + 1]; ++q) {
                const int64_t v = cp_pos[q];
                const SubdomainDesc &d = p->sd[v2k[v]];
                const int64_t li = v - d.offV;
                const double *row = A.data() + d.offA + li * d.nk;
                const int32_t *cols = vdofs.data() + d.offV;
                for (int32_t lj = 0; lj < d.nk; ++lj) {
                    const double a = row[lj];
                    if (a == 0.0) continue;
                    const int32_t gj = cols[lj];
                    if (!mark[gj]) {
                        mark[gj] = 1;
                        touched.push_back(gj);
                    }
                    acc[gj] += a;
                }
            }
            double dg = 1.0;
            if (touched.empty()) {            // no subdomain copy: identity row
                o.col.push_back((int32_t)g);
                o.val.push_back(1.0);
                o.len.push_back(1);
            } else {
                std::sort(touched.begin(), touched.end());
                dg = 0.0;
                for (int32_t gj : touched) {
                    o.col.push_back(gj);
                    o.val.push_back(acc[gj]);
                    if (gj == g) dg = acc[gj];
                    acc[gj] = 0.0;
                    mark[gj] = 0;
                }
                o.len.push_back((int64_t)touched.size());
            }
            o.diag.push_back(dg);
        }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < T; ++t) th.emplace_back(work, t);
    work(0);
    for (auto &x : th) x.join();

    std::vector<int64_t> ptr((size_t)n + 1, 0);
    std::vector<int32_t> col;
    std::vector<double> val, dinv;
    std::vector<float> vhi, vlo;
    int64_t r = 0;
    for (int t = 0; t < T; ++t) {
        for (size_t i = 0; i < ch[t].len.size(); ++i, ++r) ptr[r + 1] = ptr[r] + ch[t].len[i];
        col.insert(col.end(), ch[t].col.begin(), ch[t].col.end());
        val.insert(val.end(), ch[t].val.begin(), ch[t].val.end());
        for (double dg : ch[t].diag) {
            if (!(dg > 0.0)) fail(NLFETI_E_NOT_SPD, "the single-domain matrix has a non-positive diagonal entry");
            dinv.push_back(1.0 / dg);
        }
        Chunk().len.swap(ch[t].len);
    }
    vhi.resize(val.size());
    vlo.resize(val.size());
    for (size_t i = 0; i < val.size(); ++i) {
        vhi[i] = (float)val[i];
        vlo[i] = (float)(val[i] - (double)vhi[i]);
    }
    upload(c, p->d_cg_ptr, ptr);
    upload(c, p->d_cg_col, col);
    upload(c, p->d_cg_vhi, vhi);
    upload(c, p->d_cg_vlo, vlo);
    upload(c, p->d_cg_dinv, dinv);
    NLF_CUDA(cudaStreamSynchronize(c->stream));
    p->cg_nnz = ptr[n];
    p->cg_ready = true;
}

}  // namespace nlf
