// Internal declarations of the nlfeti library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/nlfeti.h"

struct nlfeti_ctx {
    nlfeti_options opt;
    int device = 0;                       // the device current at nlfeti_create (its streams and memory)
    cudaStream_t stream = nullptr;        // the library's own non-blocking stream (capturable)
    cudaStream_t user_stream = nullptr;   // the caller's stream (may be the legacy stream)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    void *(*dev_alloc)(size_t, void *) = nullptr;
    void (*dev_free)(void *, void *) = nullptr;
    void *alloc_user = nullptr;
    std::string err;
    std::mutex mu;                // guards err, bytes_in_use and the child count
    size_t bytes_in_use = 0;
    int children = 0;             // live problems and servers
    bool destroy_pending = false; // nlfeti_destroy was called while children were alive
};

namespace nlf {

// ------------------------------------------------------------------ errors
struct Error {
    nlfeti_status st;
    std::string msg;
};
[[noreturn]] void fail(nlfeti_status st, const std::string &msg);
void check_cuda(cudaError_t e, const char *what);
#define NLF_CUDA(x) ::nlf::check_cuda((x), #x)

// ------------------------------------------------------------------ device memory
// Owned device buffer.  With a context: the context's allocator (or cudaMalloc), counted
// against the context budget.  With a stream (no context): stream-ordered cudaMallocAsync.
struct DevMem {
    nlfeti_ctx *ctx = nullptr;
    cudaStream_t astream = nullptr;
    bool async = false;
    void *p = nullptr;
    size_t bytes = 0;
    DevMem() = default;
    DevMem(const DevMem &) = delete;
    DevMem &operator=(const DevMem &) = delete;
    DevMem(DevMem &&o) noexcept { *this = std::move(o); }
    DevMem &operator=(DevMem &&o) noexcept {
        release();
        ctx = o.ctx; astream = o.astream; async = o.async; p = o.p; bytes = o.bytes;
        o.p = nullptr; o.bytes = 0;
        return *this;
    }
    ~DevMem() { release(); }
    void alloc(nlfeti_ctx *c, size_t n);
    void alloc_async(cudaStream_t s, size_t n);
    void release();
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

template <typename T> void upload(nlfeti_ctx *c, DevMem &m, const std::vector<T> &v) {
    m.alloc(c, sizeof(T) * (v.empty() ? 1 : v.size()));
    if (!v.empty())
        NLF_CUDA(cudaMemcpyAsync(m.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, c->stream));
}

// ------------------------------------------------------------------ host decomposition
constexpr int kMaxSubdomains = 4096;
constexpr int kMaxCoarse = 3 * kMaxSubdomains;     // coarse columns: at most three rigid modes per subdomain

struct Decomp {
    int K = 0, nc = 1;
    int mask_words = 1;                   // words of an element's subdomain mask: ceil(K / 64)
    std::vector<uint64_t> elem_mask;      // per element mask_words words, bit k % 64 of word k / 64:
                                          // element in Omega-hat_k u Gamma^D_k
    bool in_sub(int64_t e, int k) const { return (elem_mask[e * mask_words + k / 64] >> (k % 64)) & 1u; }
    bool any_sub(int64_t e) const {
        for (int w = 0; w < mask_words; ++w)
            if (elem_mask[e * mask_words + w]) return true;
        return false;
    }
    bool share_sub(int64_t e, int64_t f) const {
        for (int w = 0; w < mask_words; ++w)
            if (elem_mask[e * mask_words + w] & elem_mask[f * mask_words + w]) return true;
        return false;
    }
    std::vector<int32_t> node_zeta;       // number of Omega-hat_k holding the node
    std::vector<std::vector<int32_t>> nodes;   // per k: Omega nodes then Gamma nodes (ascending each)
    std::vector<int32_t> n_omega_nodes, n_gamma_nodes;
    std::vector<std::vector<int32_t>> dir_nodes;  // per k: Dirichlet nodes of Omega-hat_k u Gamma^D_k (ascending)
    std::vector<int8_t> floating;
    std::vector<std::vector<int32_t>> pinned;     // Gamma-local dof indices
    std::vector<int64_t> u_off;                   // K+1, in dofs
    std::vector<int64_t> B_plus, B_minus;         // U indices
    std::vector<int32_t> B_node;
    std::vector<int32_t> co_off;                  // K+1 coarse columns per subdomain
};

struct MeshHost {
    int dim = 2;
    int64_t n_nodes = 0, n_elems = 0;
    std::vector<double> xy;
    std::vector<int32_t> elems;
    std::vector<int8_t> node_dir, elem_dir;
};

void build_decomposition(const MeshHost &m, const nlfeti_kernel &kern, const std::vector<int32_t> &labels, int K,
                         Decomp &d);

}  // namespace nlf

// ------------------------------------------------------------------ device-side problem data
struct SubdomainDesc {      // per subdomain, device resident (POD)
    int32_t nk, nO, nG;     // dofs
    int32_t nD;             // Dirichlet dofs coupled (columns of AD)
    int64_t offA;           // FP64 assembled matrix (nk x nk, ld nk)
    int64_t offAD;          // FP64 Dirichlet coupling (nk x nD)
    int64_t offM;           // swept matrix (nk x ldM) in the operator pool of a precision
    int64_t offS;           // S_k (nG x ldG)
    int64_t offSp;          // S_k^+ (nG x ldG)
    int64_t offU;           // start of Gamma_k in U
    int64_t offV;           // start of the subdomain in the concatenated subdomain vectors (sum nk)
    int32_t co_off, n_co;   // coarse columns
    int32_t floating;
    int32_t npin;
    int32_t pin[3];
    int32_t ldM;            // nk rounded up to 8
    int32_t ldG;            // nG rounded up to 8
    int32_t pad;
    int64_t offUp;          // start of Gamma_k in the padded U layout (sum of ldG); the apply input
                            // for R right-hand sides sits at offUp*R as R columns of ldG entries
    int64_t offVp;          // start of the subdomain in the padded subdomain-vector layout (sum of
                            // ldM): R columns of ldM entries at offVp*R (refinement residual input)
    int64_t offT;           // first tile of S_k in the tiled FP16 copy (tensor-core apply): tiles of
                            // 128 rows x 64 columns, ceil(nG/128) row tiles x mma_ktiles(nG, ldG)
    int64_t offXp;          // start of Gamma_k in the paired FP32 apply input (sum of ldG rounded up
                            // to 128): for R right-hand sides at offXp * R2 (R2 = R rounded up to
                            // even), see apply_paired_index
};

// the paired FP32 apply input: the right-hand sides of a subdomain taken two at a time (pair
// row cp = columns 2 cp, 2 cp + 1; R2 / 2 pair rows of 2 ldgx(ldG) floats), and within a pair row
// the 128-column group g of operator columns in the order a lane of the apply reads them: lane k
// (columns 4k .. 4k+3 of the group) finds columns 4k, 4k+1 of both right-hand sides as one float4
// at 256 g + 4 k and columns 4k+2, 4k+3 as one float4 128 floats further
__host__ __device__ inline int64_t ldgx(int ldG) { return (int64_t)(ldG + 127) / 128 * 128; }
__host__ __device__ inline int64_t paired_col(int j) {
    return 256 * (int64_t)(j >> 7) + 128 * ((j >> 1) & 1) + 4 * ((j & 127) >> 2) + 2 * (j & 1);
}
__host__ __device__ inline int64_t apply_paired_index(int64_t offXp, int ldG, int j, int c, int R) {
    const int R2 = (R + 1) / 2 * 2;
    return offXp * R2 + (int64_t)(c >> 1) * 2 * ldgx(ldG) + paired_col(j) + (c & 1);
}

// column tiles of 64 of an operator in the tiled FP16 copy: the streamed columns, min(ldG,
// nG rounded up to 8), in 64-column tiles
__host__ __device__ inline int mma_ktiles(int nG, int ldG) {
    const int ncp = ldG < (nG + 7) / 8 * 8 ? ldG : (nG + 7) / 8 * 8;
    return (ncp + 63) / 64;
}

constexpr int kApplyRows = 32;          // rows of an interface-apply work item
constexpr int MMA_MAX_RHS = 64;         // right-hand sides of the tensor-core preconditioner apply

template <typename T> struct OpPool {   // operators of one precision
    nlf::DevMem M, S, Sp;                // swept matrices, Schur complements, pseudo-inverses
    nlf::DevMem scratch;                 // panel scratch of the sweeps
    nlf::DevMem maps;                    // tensor maps of S_k and S_k^+ (2 per subdomain) for the apply
    nlf::DevMem fmaps, omaps;            // tensor maps of the swept matrix blocks the forcing (rows n_O..,
                                         // columns ..n_O) and the back substitution (rows ..n_O) stream
    nlf::DevMem Ahi, Alo;                // FP32 pool only: A^k = Ahi + Alo (FP32 pairs, swept-matrix layout),
                                         // for the double-single refinement residual
    nlf::DevMem amaps;                   // FP32 pool only: tensor maps of Ahi and Alo (2 per subdomain)
    bool a_sparse = false;               // FP32 pool only: A^k kept as a CSR of FP32 pairs instead of
    int64_t a_nnz = 0;                   // Ahi / Alo (a_nnz entries, at most a third of sum n_k^2)
    nlf::DevMem Aptr, Aent;              // row pointers (int64, sum n_k + 1) and entries (int4: column
                                         // position, hi bits, lo bits, 0) of that CSR
    nlf::DevMem row_u;                   // per subdomain-vector row: U index (Gamma dof) or -1
    nlf::DevMem Sh;                      // FP32 pool only: S_k * hscale in FP16 (preconditioner of the PCG)
    nlf::DevMem hmaps;                   // FP32 pool only: tensor maps of Sh (slot 2k per subdomain)
    double hscale = 1.0;                 // power of two: largest |S_k| entry * hscale in [2^13, 2^14)
    nlf::DevMem St;                      // FP32 pool only: Sh tiled for the tensor-core apply: 128 x 64 tiles
                                         // of 16 KB, each in the 128-byte swizzled K-major order of the MMA
                                         // operand (zeros past n_gamma and ld_gamma)
    bool ready = false;
};

namespace nlf { struct SolveWS; }

// a configuration of the bulk-copy interface apply: right-hand sides per streamed pass (1, 2,
// 4, 8 or 16) and CTAs per SM of its persistent grid (1 or 2); for the FP16 copy of S_k the
// tensor-core apply instead (mma)
struct ApplyChoice {
    int rc = 0;
    int per_sm = 2;
    int mma = 0;
    int rpw = 4;      // rows per consumer warp of the bulk-copy apply (4 or 8)
};

struct nlfeti_problem {
    nlfeti_ctx *ctx = nullptr;
    uint64_t uid = 0;                   // unique per problem of the process (workspaces and graphs key on it)
    uint64_t factor_gen = 0;            // bumped by every factorization (operator buffers may move)
    nlfeti_options opt;
    nlf::MeshHost mesh;
    nlfeti_kernel kern;
    nlf::Decomp dec;
    int K = 0, nc = 1;
    int64_t n_lambda = 0, n_u = 0, sum_nk = 0, n_dofs_total = 0, n_up = 0, n_vp = 0, n_xp = 0;
    int n_co = 0, n_floating = 0, max_ldG = 0;
    std::vector<SubdomainDesc> sd;      // host copy
    nlf::DevMem d_sd;
    // mesh on device
    nlf::DevMem d_xy, d_elems, d_node_dir, d_elem_mask;
    // node -> subdomain-local node index map (K x n_nodes): >= 0 dof node, <= -2 Dirichlet column node
    // -(2 + index), -1 none
    nlf::DevMem d_nodemap;
    // assembled FP64 matrices
    nlf::DevMem d_A, d_AD;
    int64_t poolA = 0, poolAD = 0, poolM = 0, poolG = 0, poolT = 0;
    // jump operators
    nlf::DevMem d_Bp, d_Bm;              // int64 U index per Lambda row
    nlf::DevMem d_Bt_ptr, d_Bt_row;      // per U dof: rows, signed (r+1 for +1, -(r+1) for -1)
    nlf::DevMem d_BD_ptr, d_BD_col, d_BD_val;    // B_D rows (U index, value)
    nlf::DevMem d_BDt_ptr, d_BDt_row, d_BDt_val; // B_D^T rows per U dof
    nlf::DevMem d_BD_val32, d_BDt_val32;         // FP32 copies of the values (FP32 PCG iterations)
    nlf::DevMem d_Z;                     // (n_u x 3) FP64 kernel basis of floating subdomains
    nlf::DevMem d_Q;                     // (n_u x 3) FP64 orthonormal kernel basis
    nlf::DevMem d_GtGinv;                // n_co x n_co FP64
    nlf::DevMem d_GtGinv32;              // its FP32 copy, transposed (FP32 PCG iterations)
    // rows of G = B Z: per Lambda row gw slots (coarse column, value), the first gw/2 for the
    // +1 side (Z rows of B_plus), the rest for the -1 side; empty slots have column -1
    int gw = 0;
    nlf::DevMem d_Gcol, d_Gval, d_Gval32;        // d_Gval32: FP32 copy
    nlf::DevMem d_float_ids;             // floating subdomains (int32)
    // G^T gathers per floating subdomain f: entry ranges (4 int64: Lambda-mode e0, e1 into the
    // B^T entries, U-mode u0, u1), (co_off, n_co), and per B^T entry its Lambda row and the
    // weights sign * Z[u] (3 doubles)
    nlf::DevMem d_gt_range, d_gt_co, d_gt_rows, d_gt_w, d_gt_w32;   // d_gt_w32: FP32 copy
    nlf::DevMem d_u2sub;                 // per U dof: subdomain (int32)
    nlf::DevMem d_u2v;                   // per U dof: position in the subdomain vectors (int64)
    nlf::DevMem d_vdofs;                 // per subdomain-vector entry: global dof (int32)
    nlf::DevMem d_cp_ptr, d_cp_pos;      // per global dof: positions of its copies (int64)
    nlf::DevMem d_ddofs, d_doff;         // per subdomain: global dofs of the Dirichlet columns
    nlf::DevMem d_nodeinc_ptr, d_nodeinc_el;  // node -> interior elements (load vector gather)
    nlf::DevMem d_zeta_dof;              // per global dof: zeta (double)
    nlf::DevMem d_items;                 // row-product work items over Gamma rows: (k, first row) pairs
    int n_items = 0;
    std::vector<int> item_off;           // K+1
    nlf::DevMem d_items_o;               // work items over Omega rows (back substitution)
    std::vector<int> item_off_o;         // K+1
    // persistent schedule of the refinement residual: 32-row items over all rows of A^k
    int rsched_ctas = 0;
    nlf::DevMem d_rsched_ptr, d_rsched_items;
    // persistent schedule of the bulk-copy interface apply: CTA b runs the work items
    // sched_items[sched_ptr[b] .. sched_ptr[b+1]) (pairs (k, first row)), balanced by cost
    int sched_ctas = 0;
    nlf::DevMem d_sched_ptr, d_sched_items;
    // the same items over one CTA per SM (an autotuner candidate)
    int sched1_ctas = 0;
    nlf::DevMem d_sched1_ptr, d_sched1_items;
    // the autotuner's choices for the bulk-copy apply per (operator kind, right-hand sides):
    // kind 0 = FP32 operators, 1 = the FP16 copy of S_k, 2 = FP64 operators
    std::map<std::pair<int, int>, ApplyChoice> tune;
    uint64_t tune_gen = 0;               // bumped by every change of tune (captured graphs key on it)
    // the same for the tensor-core preconditioner apply: 128-row items; and, for the launches
    // per subdomain, the items in subdomain order (subdomain k: mitem_off[k] .. mitem_off[k+1])
    // with the identity schedule 0, 1, 2, ... (one item per CTA)
    int msched_ctas = 0;
    nlf::DevMem d_msched_ptr, d_msched_items;
    // and for the forcing (items over Gamma rows, n_O columns) and the back substitution (items
    // over Omega rows, n_k columns) on the same pipeline
    int fsched_ctas = 0, osched_ctas = 0;
    nlf::DevMem d_fsched_ptr, d_fsched_items, d_osched_ptr, d_osched_items;
    nlf::DevMem d_mitems, d_iota;
    std::vector<int> mitem_off;
    nlf::DevMem d_flag;                  // device status words
    OpPool<double> op64;
    OpPool<float> op32;
    std::unique_ptr<nlf::SolveWS> ws;
    // Diagonally preconditioned CG on the single-domain system (the paper's comparison
    // solver): the global FP64 matrix as CSR over the n_dofs_total dofs (int64 row pointers,
    // int32 columns, values as FP32 hi / lo pairs), assembled from the A^k by
    // nlfeti_cg_prepare or the first CG solve, and the inverse of its diagonal
    nlf::DevMem d_cg_ptr, d_cg_col, d_cg_vhi, d_cg_vlo, d_cg_dinv;
    int64_t cg_nnz = 0;
    bool cg_ready = false;
    double ms_setup = 0, ms_factor = 0;
    // fault injection for tests of the bounded waits of the interface apply (nlfeti_debug_apply_waits):
    // the consumers' stage-wait limit (0 = the default) and whether the producer withholds its copies
    long long dbg_wait_tries = 0;
    int dbg_withhold = 0;
    bool prof_on = false;
    std::mutex prof_mu;
    nlfeti_profile prof{};
    ~nlfeti_problem();
};

// kernels and launchers (defined in the .cu files)
namespace nlf {
void assemble_all(nlfeti_problem *p);
template <typename T> void factor_ops(nlfeti_problem *p, OpPool<T> &pool);
// the FP16 copy of S_k tiled for the tensor-core preconditioner apply (FP32 operators factored)
void build_tiled_half(nlfeti_problem *p);
void setup_coarse(nlfeti_problem *p);
void setup_jump_weights(nlfeti_problem *p);
void set_error(nlfeti_ctx *c, const std::string &msg);
// order the library stream after the caller's stream (enter) and the caller's after it (leave)
void stream_enter(nlfeti_ctx *c);
void stream_leave(nlfeti_ctx *c);
// a live problem or server keeps its context alive
void ctx_attach(nlfeti_ctx *c);
void ctx_detach(nlfeti_ctx *c);
// the apply configuration used for operator kind (0 FP32, 1 FP16 copy, 2 FP64) and R: the
// autotuner's choice if one was made, else the default (apply_rc(R), two CTAs per SM)
ApplyChoice apply_choice(const nlfeti_problem *p, int kind, int R);
// streaming multiprocessors of the current device
int device_sms();
// CTAs of the bulk-copy interface apply / refinement residual that fit on the device at once
int apply_tma_ctas();
int apply_mma_ctas();
int residual_tma_ctas();
// tensor maps of a pool's S_k and S_k^+ for the bulk-copy apply (after the factorization)
template <typename T> void encode_apply_maps(nlfeti_problem *p, OpPool<T> &pool);
// global CSR of the single-domain matrix for the CG baseline (once per problem; host sync)
void cg_prepare(nlfeti_problem *p);
// device bytes of a problem created from these inputs and factored in the precisions of mask
// (bit 0 FP64, bit 1 FP32): validates the inputs and runs the host decomposition (throws Error)
size_t predict_problem_bytes(const nlfeti_mesh *mesh, const nlfeti_kernel *kernel, const nlfeti_decomp *decomp,
                             int mask);
}  // namespace nlf
