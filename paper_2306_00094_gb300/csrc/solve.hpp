// Solve-phase workspace and entry points (internal).
#pragma once

#include "internal.hpp"

namespace nlf {

// An instantiated PCG loop of one pass (the body captured once and launched by every later
// pass with the same problem, factorization, precision, tolerance and iteration limit).
struct PcgGraph {
    uint64_t factor_gen = 0;
    int precision = 0, max_it = 0;
    double tol = 0;
    cudaGraphExec_t exec = nullptr;
    int64_t body_launches = 0;      // kernels per loop iteration
    int precond_fp16 = 0;           // the preconditioner apply it was captured with
    int kind = 0;                   // 0: FETI PCG loop, 1: single-domain CG loop
    long long wait_tries = 0;       // the apply's stage-wait limit and withheld copies it was
    int withhold = 0;               // captured with (fault injection for tests)
    uint64_t tune_gen = 0;          // the apply configurations it was captured with
};

constexpr int kSlotFlags = 1024;   // flag words of the timed applies: half for graphs, half eager

struct SolveWS {
    nlfeti_problem *prob = nullptr;
    uint64_t prob_uid = 0;
    int R = 0;
    DevMem lam, r, w, z, y, pv, q, d, cvec, dlam;      // Lambda space (FP64)
    DevMem lamf;                                        // r, w, z, y, p, q, lambda of the FP32 pass (FP32)
    DevMem fU, yU, uU, xU;                              // U space (xU: apply input, FP64 and FP16 layouts)
    DevMem xP;                                          // FP32 apply input, paired layout (apply_paired_index)
    DevMem xmaps[2];                                    // tensor maps of xU per subdomain (FP32, FP64),
                                                        // tiles of the default column block apply_rc(R)
    DevMem xmaps_rc[2][5];                              // the same for column blocks 1, 2, 4, 8, 16 (the
                                                        // autotuner's choices; 16 for FP32 only)
    DevMem xhmaps;                                      // xU read as FP16 (tensor-core apply; R <= 64)
    DevMem xscale;                                      // per column: power of two x is scaled by (FP16 x)
    DevMem slot_flags;                                  // gates seen by the timed applies (profiling)
    DevMem rxs;                                         // right-hand sides of the forcing / back substitution
                                                        // (R columns of ld_M entries at offVp * R per subdomain)
    DevMem rxmaps[2];                                   // tensor maps of rxs per subdomain (FP32, FP64)
    DevMem ftil, res, u, du;                            // concatenated subdomain vectors
    DevMem uhl;                                         // u as FP32 hi / lo pairs, padded layout
    DevMem umaps;                                       // tensor maps of uh and ul per subdomain
    DevMem F;                                           // global load vector per dof
    DevMem gco, gsum, alpha;                            // coarse space
    DevMem partial, partial2, scal;                     // reductions and PCG scalars
    DevMem frozen;                                      // per column: refinement finished (mixed path)
    DevMem in_rhs, in_g, out_u;                         // staging for host-array solves
    DevMem cg_u, cg_r, cg_z, cg_p, cg_q, cg_b, cg_part;  // single-domain CG (global dofs x R)
    DevMem cg_ph, cg_pl;                                // p as FP32 hi / lo pairs (SpMV operand)
    std::vector<int> host_flag;
    cudaStream_t async_stream = nullptr;   // set: the stream the workspace works on (a server slot's)
    cudaStream_t alloc_stream = nullptr;   // set: stream-ordered allocations and frees of its buffers
                                           // on this stream (a server's, never captured), so that a
                                           // workspace freed by another slot never enqueues into a
                                           // stream that is capturing a graph
    std::vector<PcgGraph> graphs;
    void ensure(nlfeti_problem *p, int R);
    void drop_graphs();
    SolveWS() = default;
    SolveWS(const SolveWS &) = delete;
    SolveWS &operator=(const SolveWS &) = delete;
    ~SolveWS() { drop_graphs(); }
};

// Full solve on device arrays: rhs / g column-major (n_dofs x R), out column-major.
void solve_device(nlfeti_problem *p, SolveWS &ws, cudaStream_t st, int R, int rhs_kind, const double *d_rhs,
                  const double *d_g, double *d_out, nlfeti_stats *stats);

// Single-domain diagonally preconditioned CG (the paper's baseline solver) on device arrays,
// same arguments as solve_device; at most 32 right-hand sides.
void cg_solve_device(nlfeti_problem *p, SolveWS &ws, cudaStream_t st, int R, int rhs_kind, const double *d_rhs,
                     const double *d_g, double *d_out, nlfeti_stats *stats);

// Apply one operator (0 F, 1 M^-1, 2 P, 3 S^+, 4 S) to device vectors in the interleaved layout.
void apply_operator(nlfeti_problem *p, SolveWS &ws, cudaStream_t st, int op, int precision, int R, const double *in,
                    double *out);

// Autotuner of the bulk-copy interface apply for R right-hand sides: per operator kind the
// problem has (FP32 S^+, FP16 copy of S_k, FP64 S^+), every column block 1..16 (<= R) and one or
// two CTAs per SM, timed with CUDA events on the problem's operators; the fastest is kept in
// the problem.  With a cache path, choices found there (same device, subdomain shapes, kind and
// R) are used without timing, and new ones are written back (JSON).
struct TuneEntry {
    int kind = 0, R = 0, rc = 0, per_sm = 0, rpw = 4;
    double us = 0;
    bool from_cache = false;
};
void autotune_applies(nlfeti_problem *p, int R, const char *cache_path, std::vector<TuneEntry> &out);

// Interleaved <-> column-major conversions (device).
void to_interleaved(const double *colmajor, double *inter, int64_t n, int R, cudaStream_t st);
void to_colmajor(const double *inter, double *colmajor, int64_t n, int R, cudaStream_t st);

}  // namespace nlf
