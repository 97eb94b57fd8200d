// FETI solve phase on the GPU: Algorithm 1 steps 3 and 6-9, the projected PCG of step 7
// with the scaled Dirichlet preconditioner (eq. preconditioner), and for the mixed path FP64
// iterative refinement on the torn system (eq. discreteKKT).
//
// Vectors hold R right-hand sides interleaved (entry i of column c at i*R + c).
// Lambda-space vectors, coarse vectors and all scalars are FP64; the subdomain operators
// S_k^+, S_k and the swept matrices are FP64 (plain path) or FP32 (mixed path).
//
// PCG iteration (per right-hand side; converged columns are frozen with eta = 0):
//   w = P r;  z = B_D S B_D^T w;  y = P z;  beta = (y,w)/(y,w)_old;  p = y + beta p;
//   q = B S^+ B^T p;  eta = (y,w)/(p,q);  lambda += eta p;  r -= eta q
// with P = I - G (G^T G)^-1 G^T (eq. P), G = B Z, stopping when ||w||_2 <= tol ||P d||_2.
// A pass solves for subdomain loads f: reduced forcing f_U (eq. subForcing),
// d = B S^+ f_U - c, e = Z^T f_U, lambda^0 = G (G^T G)^-1 e, PCG, then
// alpha = (G^T G)^-1 G^T (d - F lambda) (eq. forAlpha), u_G = S^+ (f_U - B^T lambda) - Z alpha
// (eq. forU) and u_O by back substitution (eq. backwardSubstitution).
// Mixed refinement: r = f~ - A u - [0; B^T lambda] and c = -B u_G in FP64, a pass with the
// FP32 operators gives the correction, u += du, lambda += dlambda, until the relative nodal
// correction is below refine_tol.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>

#include <cuda_fp16.h>

#include "solve.hpp"

namespace nlf {
namespace {

template <typename X> struct TypeTag { using type = X; };

constexpr int RED_BLOCKS = 304;     // two CTAs per SM for reductions
constexpr int RED_THREADS = 256;

template <typename V> __device__ __forceinline__ V warp_sum(V v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

inline unsigned grid_for(int64_t n, int threads = 256) {
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

__global__ void k_sub(const double *a, const double *b, double *out, int64_t n) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = a[t] - b[t];
}

// zero the columns c with frozen[c] != 0 of an interleaved n x R vector
__global__ void k_zero_frozen(double *v, int64_t n, int R, const int *frozen) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * R; t += (int64_t)gridDim.x * blockDim.x)
        if (frozen[t % R]) v[t] = 0.0;
}

__global__ void k_axpy(double *y, const double *x, double a, int64_t n) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        y[t] += a * x[t];
}

__global__ void k_transpose_cr(const double *src, double *dst, int64_t n, int R, int to_inter) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * R; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = t / R;
        int c = (int)(t % R);
        if (to_inter) dst[t] = src[(int64_t)c * n + i];
        else dst[(int64_t)c * n + i] = src[t];
    }
}

// ------------------------------------------------------------------ gathers between U and Lambda
// x_U = B^T v (cast to T); rows stored signed: r+1 for +1, -(r+1) for -1
template <typename T>
__global__ void k_gather_bt(const int64_t *ptr, const int64_t *row, const double *v, T *x, int64_t nu, int R) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nu * R; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t u = t / R;
        int c = (int)(t % R);
        double s = 0;
        for (int64_t q = ptr[u]; q < ptr[u + 1]; ++q) {
            int64_t r = row[q];
            s += r > 0 ? v[(r - 1) * R + c] : -v[(-r - 1) * R + c];
        }
        x[t] = (T)s;
    }
}

// x_U = B_D^T v (cast to T)
// out = B y - c (c optional)
__global__ void k_gather_b(const int64_t *Bp, const int64_t *Bm, const double *y, const double *cvec, double *out,
                           int64_t nl, int R) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nl * R; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = t / R;
        int c = (int)(t % R);
        double v = y[Bp[r] * R + c] - y[Bm[r] * R + c];
        if (cvec) v -= cvec[t];
        out[t] = v;
    }
}

// c = -B u_G read from the subdomain vectors through the U -> vector position map
__global__ void k_constraint_residual(const int64_t *Bp, const int64_t *Bm, const int64_t *u2v, const double *u,
                                      double *cvec, int64_t nl, int R) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nl * R; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = t / R;
        int c = (int)(t % R);
        cvec[t] = -(u[u2v[Bp[r]] * R + c] - u[u2v[Bm[r]] * R + c]);
    }
}

// out = B_D y (y, the sum and out in the type L of the Lambda vectors)
template <typename L>
__global__ void k_gather_bd(const int64_t *ptr, const int64_t *col, const L *val, const L *y, L *out, int64_t nl,
                            int R) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nl * R; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = t / R;
        int c = (int)(t % R);
        L s = 0;
        for (int64_t q = ptr[r]; q < ptr[r + 1]; ++q) s += val[q] * y[col[q] * R + c];
        out[t] = s;
    }
}

#include "rows.cuh"
#include "apply_tma.cuh"
#include "apply_mma.cuh"
#include "residual_tma.cuh"
#include "residual_csr.cuh"

__global__ void k_scatter_u(const int64_t *u2v, const double *uU, double *v, int64_t nu, int R) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nu * R; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / R;
        const int c = (int)(t % R);
        v[u2v[i] * R + c] = uU[t];
    }
}

// ------------------------------------------------------------------ loads and output
// global load vector per dof; rhs column-major with leading dimension ndof.
// kind 0: consistent P1 mass matrix over interior elements ((1 + [i==j]) |E| / ((d+1)(d+2)))
__global__ void k_load_vector(const double *rhs, int kind, const double *xy, const int32_t *elems, int dim,
                              const int64_t *inc_ptr, const int32_t *inc_el, int nc, int64_t ndof, int R, double *F) {
    const int nv = dim + 1;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ndof * R; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t g = t / R;
        int c = (int)(t % R);
        if (kind == 1) { F[t] = rhs[(int64_t)c * ndof + g]; continue; }
        int64_t node = g / nc;
        int comp = (int)(g % nc);
        double s = 0;
        for (int64_t q = inc_ptr[node]; q < inc_ptr[node + 1]; ++q) {
            const int32_t *en = elems + (int64_t)inc_el[q] * nv;
            double meas;
            if (dim == 1) meas = fabs(xy[en[1]] - xy[en[0]]);
            else {
                double ax = xy[2 * (int64_t)en[1]] - xy[2 * (int64_t)en[0]], ay = xy[2 * (int64_t)en[1] + 1] - xy[2 * (int64_t)en[0] + 1];
                double bx = xy[2 * (int64_t)en[2]] - xy[2 * (int64_t)en[0]], by = xy[2 * (int64_t)en[2] + 1] - xy[2 * (int64_t)en[0] + 1];
                meas = 0.5 * fabs(ax * by - ay * bx);
            }
            const double denom = dim == 1 ? 6.0 : 12.0;
            for (int b = 0; b < nv; ++b)
                s += (en[b] == node ? 2.0 : 1.0) * meas / denom * rhs[(int64_t)c * ndof + (int64_t)en[b] * nc + comp];
        }
        F[t] = s;
    }
}

// subdomain loads f~ = F / zeta at the subdomain's dofs (eq. bilinear-multi5)
__global__ void k_split_loads(const double *F, const int32_t *vdofs, const double *zeta_dof, int64_t nv, int R,
                              double *f) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nv * R; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = t / R;
        int c = (int)(t % R);
        int64_t g = vdofs[i];
        f[t] = F[g * R + c] / zeta_dof[g];
    }
}

// f~ -= A^k_D g (Dirichlet coupling), warp per row; g column-major with leading dimension ndof
__global__ void k_dirichlet(const double *AD, const SubdomainDesc *sd, const int32_t *ddofs, const int64_t *doff,
                            const double *g, int64_t ndof, double *f, int R) {
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int k = blockIdx.y;
    const SubdomainDesc d = sd[k];
    const int32_t *dd = ddofs + doff[k];
    for (int i = blockIdx.x * 8 + warp; i < d.nk; i += gridDim.x * 8) {
        const double *Ai = AD + d.offAD + (int64_t)i * d.nD;
        for (int c = 0; c < R; ++c) {
            double s = 0;
            for (int l = lane; l < d.nD; l += 32) s += Ai[l] * g[(int64_t)c * ndof + dd[l]];
            s = warp_sum(s);
            if (lane == 0) f[(d.offV + i) * R + c] -= s;
        }
    }
}

// nodal output: mean of the copies; Dirichlet dofs take g (or 0); column-major
__global__ void k_output(const double *u, const int64_t *cp_ptr, const int64_t *cp_pos, const int8_t *node_dir, int nc,
                         const double *g, int64_t ndof, int R, double *out) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ndof * R; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t gd = t % ndof;
        int c = (int)(t / ndof);
        double v = 0;
        if (node_dir[gd / nc]) v = g ? g[(int64_t)c * ndof + gd] : 0.0;
        else {
            int64_t a = cp_ptr[gd], b = cp_ptr[gd + 1];
            for (int64_t q = a; q < b; ++q) v += u[cp_pos[q] * R + c];
            if (b > a) v /= (double)(b - a);
        }
        out[t] = v;
    }
}

__device__ __forceinline__ double z_alpha(const SubdomainDesc *sd, const int32_t *u2sub, const double *Z,
                                          const double *alpha, int64_t u, int c, int R) {
    const SubdomainDesc d = sd[u2sub[u]];
    double s = 0;
    for (int a = 0; a < d.n_co; ++a) s += Z[u * 3 + a] * alpha[(int64_t)(d.co_off + a) * R + c];
    return s;
}

// (G alpha)_r for column c from the slots of row r of G = B Z, in the arithmetic type L of
// the Lambda vectors (FP64, or FP32 in the FP32 pass with FP32 copies of G and alpha)
template <typename L>
__device__ __forceinline__ L g_alpha(const int32_t *gcol, const L *gval, int gw, const L *alpha, int64_t r, int c,
                                     int R) {
    const int h = gw / 2;
    L sp = 0, sm = 0;
    for (int e = 0; e < h; ++e) {
        const int cp = gcol[r * gw + e], cm = gcol[r * gw + h + e];
        if (cp >= 0) sp += gval[r * gw + e] * alpha[(int64_t)cp * R + c];
        if (cm >= 0) sm += gval[r * gw + h + e] * alpha[(int64_t)cm * R + c];
    }
    return sp - sm;
}

// out = base + sign * G alpha on Lambda
__global__ void k_apply_galpha(const int32_t *gcol, const double *gval, int gw, const double *alpha,
                               const double *base, double sign, double *out, int64_t nl, int R) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nl * R; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / R;
        const int c = (int)(t % R);
        out[t] = (base ? base[t] : 0.0) + sign * g_alpha(gcol, gval, gw, alpha, r, c, R);
    }
}

// uU += sign * Z alpha
__global__ void k_apply_zalpha(const SubdomainDesc *sd, const int32_t *u2sub, const double *Z, const double *alpha,
                               double sign, double *uU, int64_t nu, int R) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nu * R; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t u = t / R;
        int c = (int)(t % R);
        uU[t] += sign * z_alpha(sd, u2sub, Z, alpha, u, c, R);
    }
}

// PCG scalar state, per right-hand side
struct PcgScalars {
    double *nPd, *yw_old, *yw, *eta, *beta, *relres, *corr;
    double *xscale;        // per column: 2^-floor(log2 ||w||) (FP16 input of the tensor-core apply)
    float *eta_f, *beta_f, *xscale_f;   // FP32 copies of eta, beta, xscale (the FP32 pass's steps)
    int *active, *iters, *n_active;
    int *loops;            // PCG iterations run by the current graph loop
    int *err;              // set by a device wait that ran out (checked after the solve)
    unsigned *counter;     // arrival counter of the fused reductions (reset by the last block)
    unsigned *colcnt;      // per column: arrival counters of the per-column coarse solve
};

enum { FIN_NPD = 0, FIN_CHECK = 1, FIN_BETA = 2, FIN_ETA = 3 };

// the step scalars in the arithmetic type L of the Lambda vectors
template <typename L> __device__ __forceinline__ const L *eta_of(const PcgScalars &s) {
    if constexpr (std::is_same<L, float>::value) return s.eta_f;
    else return s.eta;
}
template <typename L> __device__ __forceinline__ const L *beta_of(const PcgScalars &s) {
    if constexpr (std::is_same<L, float>::value) return s.beta_f;
    else return s.beta;
}
template <typename L> __device__ __forceinline__ const L *xscale_of(const PcgScalars &s) {
    if constexpr (std::is_same<L, float>::value) return s.xscale_f;
    else return s.xscale;
}
__device__ __forceinline__ double fma_l(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_l(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Reductions over Lambda: grid (row blocks, right-hand sides), one thread per row of one
// column.  The row blocks depend on the vector length only, so every column is summed in the
// same order whatever batch it is part of: per thread over its rows, a warp tree, the warps
// in order, and the row blocks in order by the last block to arrive.
inline dim3 red_grid(int64_t n, int R) {
    return dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(RED_BLOCKS, (n + RED_THREADS - 1) / RED_THREADS)),
                (unsigned)R);
}

// block sum of one value per thread into partial[blockIdx.x][blockIdx.y]
__device__ __forceinline__ void block_partial(double acc, double *partial, int R) {
    __shared__ double red[RED_THREADS / 32];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    acc = warp_sum(acc);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0;
        for (int w = 0; w < RED_THREADS / 32; ++w) x += red[w];
        partial[(int64_t)blockIdx.x * R + blockIdx.y] = x;
    }
}

// true in the last block of the grid to arrive (after every block's partials are visible)
__device__ __forceinline__ bool arrive_last(unsigned *counter) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x * gridDim.y * gridDim.z - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Coalesced reductions over Lambda with R interleaved right-hand sides (entry (i, c) at
// i R + c).  The rows are cut into tiles of RT = 8 rows; block b owns the contiguous tiles
// [b tpb, (b + 1) tpb) (tpb from n and the grid only).  A (tile, chunk of cw columns) unit
// takes 4 cw lanes: lane (h, j), h = 0..3, adds rows h and h + 4 of column c0 + j, and the
// four lanes of a column are added as ((h0 + h2) + (h1 + h3)).  The block adds its tile sums
// per column in tile order (rounds of up to RSMEM / R tiles through shared memory), and
// finish_scalars adds the blocks' partials in block order.  cw = min(8, R rounded up to a
// power of two) and the round size only decide which lanes run a unit and when, never the
// order of the additions, so every column is summed in the same order whatever the batch it
// is part of; the lanes of a unit read 4 rows x cw consecutive columns per step, and each lane
// has two rows in flight.  f(i, c) is called once per entry (i < n, c < R) and returns its
// addend; a unit's sum is formed in the addends' type (FP32 in the FP32 pass), the tile sums
// onward in FP64.  The block partials are stored column by column (partial[c * blocks + b]), so that the
// last block reads each column's partials as whole lines (measured: the finish of 608 blocks x 16
// columns took 10 us with the partials row by row, 6 us column by column).
constexpr int RT = 8;
constexpr int RSMEM = 2048;             // doubles of tile sums per round (16 KB)
constexpr int TILE_THREADS = 1024;      // threads of a tile-reduction block (one block per SM)
constexpr int RCOLS = TILE_THREADS;     // columns per pass (one accumulating thread each)

// one 1024-thread CTA per SM: the warps of four 256-thread CTAs, a quarter of the partials for
// the last block to add (measured: the finish with 608 blocks took about 6 us of each fused
// reduction, its loads in several dependent rounds)
constexpr int TILE_MAX_BLOCKS = 152;
inline int tile_blocks(int64_t n) {
    const int64_t nt = (n + RT - 1) / RT;
    return (int)std::max<int64_t>(1, std::min<int64_t>(TILE_MAX_BLOCKS, (nt + 1) / 2));
}

template <typename F>
__device__ __forceinline__ void tile_reduce(int64_t n, int R, double *partial, F &&f) {
    using A = decltype(f(int64_t(0), 0));   // the addends' type: the four-lane unit sums in it
    __shared__ double ts[RSMEM];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t ntiles = (n + RT - 1) / RT;
    const int64_t tpb = (ntiles + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * tpb, t1 = min(ntiles, t0 + tpb);
    const int cw = R >= 5 ? 8 : (R >= 3 ? 4 : (R == 2 ? 2 : 1));
    const int ulanes = 4 * cw, upw = 32 / ulanes;
    const int ju = lane / ulanes, jl = lane % ulanes, h = jl / cw, cj = jl % cw;
    for (int cc0 = 0; cc0 < R; cc0 += RCOLS) {
        const int ncol = min(RCOLS, R - cc0);
        const int nchunk = (ncol + cw - 1) / cw;
        const int rtiles = max(1, min(256, RSMEM / ncol));
        double acc = 0;
        for (int64_t tb = t0; tb < t1; tb += rtiles) {
            const int ntl = (int)min((int64_t)rtiles, t1 - tb);
            const int units = ntl * nchunk;
            for (int ub = warp * upw; ub < units; ub += (TILE_THREADS / 32) * upw) {
                const int u = ub + ju;
                const int tl = u / nchunk, cl = (u % nchunk) * cw + cj;
                const bool ok = u < units && cl < ncol;
                A v = 0;
                if (ok) {
                    const int64_t i0 = (tb + tl) * RT + h;
                    if (i0 < n) v += f(i0, cc0 + cl);
                    if (i0 + 4 < n) v += f(i0 + 4, cc0 + cl);
                }
                v += __shfl_down_sync(0xffffffffu, v, 2 * cw);
                v += __shfl_down_sync(0xffffffffu, v, cw);
                if (ok && h == 0) ts[tl * ncol + cl] = (double)v;
            }
            __syncthreads();
            if (threadIdx.x < ncol)
                for (int tl = 0; tl < ntl; ++tl) acc += ts[tl * ncol + threadIdx.x];
            __syncthreads();
        }
        if (threadIdx.x < ncol) partial[(int64_t)(cc0 + threadIdx.x) * gridDim.x + blockIdx.x] = acc;
    }
}

// last block: column totals over the nb row-block partials (warp per column, fixed order)
// and the PCG scalar update:
//   NPD:   ||P d|| and the initial state;      CHECK: ||w|| and the active mask;
//   BETA:  (y,w) and beta = (y,w)/(y,w)_old;    ETA:   (p,q) and eta = (y,w)/(p,q).
constexpr int FIN_GROUP = 8;            // partials per lane loaded together by the last block
template <int MODE>
__device__ void finish_scalars(const double *partial, int nb, int R, PcgScalars s, double tol, int max_it) {
    __shared__ int n_act;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) n_act = 0;
    __syncthreads();
    for (int c = warp; c < R; c += TILE_THREADS / 32) {
        // the column's nb partials are contiguous: each group of loads reads whole lines, with
        // FIN_GROUP loads of a lane in flight together, added in block order
        const double *pc = partial + (int64_t)c * nb;
        double v = 0;
        for (int b0 = lane; b0 < nb; b0 += 32 * FIN_GROUP) {
            double pv[FIN_GROUP];
#pragma unroll
            for (int m = 0; m < FIN_GROUP; ++m) pv[m] = b0 + 32 * m < nb ? __ldcg(pc + b0 + 32 * m) : 0.0;
#pragma unroll
            for (int m = 0; m < FIN_GROUP; ++m)
                if (b0 + 32 * m < nb) v += pv[m];
        }
        v = warp_sum(v);
        if (lane == 0) {
            if (MODE == FIN_NPD) {
                s.nPd[c] = sqrt(v);
                s.active[c] = 1;
                s.iters[c] = 0;
                s.yw_old[c] = 1.0;
                s.relres[c] = 1.0;
                s.eta[c] = 0.0;
                s.beta[c] = 0.0;
                s.eta_f[c] = 0.0f;
                s.beta_f[c] = 0.0f;
                s.xscale_f[c] = 1.0f;
            } else if (MODE == FIN_CHECK) {
                const double nw = sqrt(v), ref = s.nPd[c];
                // a power of two that FP32 holds too (the FP32 pass scales with the same factor)
                const double xs = (nw > 0.0 && nw < INFINITY) ? ldexp(1.0, max(-126, min(126, -ilogb(nw)))) : 1.0;
                s.xscale[c] = xs;
                s.xscale_f[c] = (float)xs;
                int act = s.active[c];
                if (act) s.relres[c] = ref > 0 ? nw / ref : 0.0;
                if (act && (nw <= tol * ref || s.iters[c] >= max_it)) act = 0;
                s.active[c] = act;
                if (act) atomicAdd(&n_act, 1);
            } else if (MODE == FIN_BETA) {
                s.yw[c] = v;
                const double b = (s.iters[c] == 0 || s.yw_old[c] == 0.0) ? 0.0 : v / s.yw_old[c];
                s.beta[c] = b;
                s.beta_f[c] = (float)b;
            } else {
                const bool act = s.active[c] != 0;
                const double e = (act && v != 0.0) ? s.yw[c] / v : 0.0;
                s.eta[c] = e;
                s.eta_f[c] = (float)e;
                if (act) { s.yw_old[c] = s.yw[c]; s.iters[c] += 1; }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (MODE == FIN_NPD) *s.n_active = R;
        if (MODE == FIN_CHECK) *s.n_active = n_act;
        *s.counter = 0u;
    }
}

// (a, b) per column with the scalar update of MODE (grid tile_blocks(n))
template <int MODE>
__global__ void __launch_bounds__(TILE_THREADS) k_dot_final(const double *__restrict__ a, const double *__restrict__ b,
                                                            int64_t n, int R, double *partial, PcgScalars s, double tol,
                                                            int max_it) {
    tile_reduce(n, R, partial, [&](int64_t i, int c) { return a[i * R + c] * b[i * R + c]; });
    if (arrive_last(s.counter)) finish_scalars<MODE>(partial, gridDim.x, R, s, tol, max_it);
}

// The updates of p, lambda and r are stored one iteration late, by the kernel that starts the
// next iteration; until then the kernels that read p_new or r_new form them per row with these
// (the same bits everywhere):
//   p_new = y + beta p on active columns (p unchanged on converged ones),
//   r_new = r - eta q (eta = 0 on converged columns and before the first iteration).
// L: the arithmetic type of the Lambda vectors (FP64; FP32 in the FP32 pass).
template <typename L> __device__ __forceinline__ L p_next(L p, L y, L beta, bool active) {
    return active ? fma_l(beta, p, y) : p;
}
template <typename L> __device__ __forceinline__ L r_next(L r, L q, L eta) { return fma_l(-eta, q, r); }

// out = P v = v - G alpha (alpha from k_proj_g; NULL when there is no coarse space), with the
// dot product of MODE: CHECK (out, out), BETA (out, other).  Grid tile_blocks(nl).
template <int MODE, typename L>
__global__ void __launch_bounds__(TILE_THREADS) k_project_dot(const int32_t *__restrict__ gcol,
                                                              const L *__restrict__ gval, int gw,
                                                              const L *__restrict__ alpha,
                                                              const L *__restrict__ v,
                                                              const L *__restrict__ other,
                                                              L *__restrict__ out, int64_t nl, int R,
                                                              double *partial, PcgScalars s, double tol, int max_it) {
    tile_reduce(nl, R, partial, [&](int64_t i, int c) {
        const int64_t t = i * R + c;
        L x = v[t];
        if (alpha) x += -g_alpha(gcol, gval, gw, alpha, i, c, R);
        out[t] = x;
        return x * (MODE == FIN_CHECK ? x : other[t]);
    });
    if (arrive_last(s.counter)) finish_scalars<MODE>(partial, gridDim.x, R, s, tol, max_it);
}

// q = B y_U with (p_new, q) and the ETA update (p_new formed per row, stored by the next
// iteration's k_check_update).  Grid tile_blocks(nl).
template <typename L>
__global__ void __launch_bounds__(TILE_THREADS) k_gather_b_eta(const int64_t *__restrict__ Bp,
                                                               const int64_t *__restrict__ Bm,
                                                               const L *__restrict__ yU,
                                                               const L *__restrict__ pv,
                                                               const L *__restrict__ y, L *__restrict__ q,
                                                               int64_t nl, int R, double *partial, PcgScalars s) {
    const L *beta = beta_of<L>(s);
    tile_reduce(nl, R, partial, [&](int64_t i, int c) {
        const int64_t t = i * R + c;
        const L x = yU[Bp[i] * R + c] - yU[Bm[i] * R + c];
        q[t] = x;
        return p_next(pv[t], y[t], beta[c], s.active[c] != 0) * x;
    });
    if (arrive_last(s.counter)) finish_scalars<FIN_ETA>(partial, gridDim.x, R, s, 0.0, 0);
}

// Start of a PCG iteration (after k_proj_g formed alpha from G^T r_new): the previous
// iteration's updates p = p_new, lambda += eta p, r = r_new, then w = P r = r - G alpha,
// (w, w) and the stop test.  The active flags read here are those p_new was formed with: the
// last block changes them only after every block has arrived.  COND: the last block also
// counts the iteration and sets the condition of the WHILE loop (continue while a
// right-hand side is active and fewer than limit iterations have run, so the loop ends
// whatever the scalars hold); a separate instantiation, as profilers skip kernels that set
// graph conditions.
template <int COND, typename L>
__global__ void __launch_bounds__(TILE_THREADS) k_check_update(const int32_t *__restrict__ gcol,
                                                               const L *__restrict__ gval, int gw,
                                                               const L *__restrict__ alpha,
                                                               const L *__restrict__ y, L *__restrict__ pv,
                                                               L *__restrict__ lam, L *__restrict__ r,
                                                               const L *__restrict__ q, L *__restrict__ w,
                                                               int64_t nl, int R, double *partial, PcgScalars s,
                                                               double tol, int max_it, cudaGraphConditionalHandle cond,
                                                               int limit) {
    const L *eta = eta_of<L>(s), *beta = beta_of<L>(s);
    tile_reduce(nl, R, partial, [&](int64_t i, int c) {
        const int64_t t = i * R + c;
        const L e = eta[c];
        const L pn = p_next(pv[t], y[t], beta[c], s.active[c] != 0);
        pv[t] = pn;
        lam[t] = fma_l(e, pn, lam[t]);
        const L rn = r_next(r[t], q[t], e);
        r[t] = rn;
        L x = rn;
        if (alpha) x += -g_alpha(gcol, gval, gw, alpha, i, c, R);
        w[t] = x;
        return x * x;
    });
    if (arrive_last(s.counter)) {
        finish_scalars<FIN_CHECK>(partial, gridDim.x, R, s, tol, max_it);
        if (COND && threadIdx.x == 0) {
            const int l = *s.loops + 1;
            *s.loops = l;
            cudaGraphSetConditional(cond, (*s.n_active > 0 && l < limit) ? 1u : 0u);
        }
    }
}

// Entry of the FP32 pass's iterations: r and lambda rounded to FP32, p, y and q zero; and its
// exit: lambda and r back in FP64.  n = n_lambda R entries.
__global__ void k_lam_enter(const double *r, const double *lam, float *rf, float *lf, float *pf, float *yf, float *qf,
                            int64_t n) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        rf[t] = (float)r[t];
        lf[t] = (float)lam[t];
        pf[t] = 0.0f;
        yf[t] = 0.0f;
        qf[t] = 0.0f;
    }
}
__global__ void k_lam_exit(const float *lf, const float *rf, double *lam, double *r, int64_t n) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        lam[t] = (double)lf[t];
        r[t] = (double)rf[t];
    }
}

// x (apply layout) = B^T p_new (B^T rows signed r+1 / -(r+1)), p_new formed per row: the input
// of the S^+ apply of a PCG iteration
template <typename T, typename L>
__global__ void k_gather_apply_p(const int64_t *ptr, const int64_t *row, const L *pv, const L *y, const L *beta,
                                 const int *active, T *x, const SubdomainDesc *sd, const int32_t *u2sub, int64_t nu,
                                 int R, const int *gate) {
    if (gate && *gate == 0) return;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nu * R; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / nu);
        const int64_t u = t % nu;
        const bool act = active[c] != 0;
        const L be = beta[c];
        L s = 0;
        for (int64_t q = ptr[u]; q < ptr[u + 1]; ++q) {
            const int64_t r = row[q], i = r > 0 ? r - 1 : -r - 1;
            const L pn = p_next(pv[i * R + c], y[i * R + c], be, act);
            s += r > 0 ? pn : -pn;
        }
        apply_store<T>(x, sd, u2sub, u, c, R, (T)s);
    }
}

// Gathers into the apply layout through shared memory: a block takes GX_U consecutive U dofs
// with all R columns; the sums are formed with the columns fastest (the R entries of a Lambda
// row are consecutive: coalesced reads), staged as [c][u], and stored with the U dofs fastest
// (coalesced stores into the per-subdomain columns).  Each sum runs over its CSR entries in the
// same order as in the column-major kernels, so the stored values are the same bits.  The sums
// are staged in their own type (that of the Lambda vectors).  Dynamic shared memory GX_U * R
// doubles (R <= GX_MAXR).
constexpr int GX_U = 32;
constexpr int GX_MAXR = 64;

template <typename T, typename G>
__device__ __forceinline__ void gather_x_block(T *x, const SubdomainDesc *sd, const int32_t *u2sub, int64_t nu, int R,
                                               G &&g) {
    using S = decltype(g(int64_t(0), 0));
    extern __shared__ double gx_raw[];
    S *gx_sm = reinterpret_cast<S *>(gx_raw);
    const int64_t u0 = (int64_t)blockIdx.x * GX_U;
    const int nuu = (int)min((int64_t)GX_U, nu - u0);
    for (int t = threadIdx.x; t < nuu * R; t += blockDim.x) {
        const int ul = t / R, c = t % R;
        gx_sm[c * GX_U + ul] = g(u0 + ul, c);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nuu * R; t += blockDim.x) {
        const int c = t / nuu, ul = t % nuu;
        apply_store<T>(x, sd, u2sub, u0 + ul, c, R, (T)gx_sm[c * GX_U + ul]);
    }
}

// x = B^T p_new (as k_gather_apply_p)
template <typename T, typename L>
__global__ void __launch_bounds__(256) k_gather_apply_p_t(const int64_t *__restrict__ ptr,
                                                          const int64_t *__restrict__ row,
                                                          const L *__restrict__ pv, const L *__restrict__ y,
                                                          const L *beta, const int *active, T *x,
                                                          const SubdomainDesc *sd, const int32_t *u2sub, int64_t nu,
                                                          int R, const int *gate) {
    if (gate && *gate == 0) return;
    gather_x_block<T>(x, sd, u2sub, nu, R, [&](int64_t u, int c) {
        const bool act = active[c] != 0;
        const L be = beta[c];
        L s = 0;
        for (int64_t q = ptr[u]; q < ptr[u + 1]; ++q) {
            const int64_t r = row[q], i = r > 0 ? r - 1 : -r - 1;
            const L pn = p_next(pv[i * R + c], y[i * R + c], be, act);
            s += r > 0 ? pn : -pn;
        }
        return s;
    });
}

// x = B^T v, or B_D^T v when val is given (as k_gather_apply)
template <typename T, typename L>
__global__ void __launch_bounds__(256) k_gather_apply_t(const int64_t *__restrict__ ptr,
                                                        const int64_t *__restrict__ row,
                                                        const L *__restrict__ val,
                                                        const L *__restrict__ v, T *x, const SubdomainDesc *sd,
                                                        const int32_t *u2sub, int64_t nu, int R, const int *gate) {
    if (gate && *gate == 0) return;
    gather_x_block<T>(x, sd, u2sub, nu, R, [&](int64_t u, int c) {
        L s = 0;
        if (val) {
            for (int64_t q = ptr[u]; q < ptr[u + 1]; ++q) s += val[q] * v[row[q] * R + c];
        } else {
            for (int64_t q = ptr[u]; q < ptr[u + 1]; ++q) {
                const int64_t r = row[q];
                s += r > 0 ? v[(r - 1) * R + c] : -v[(-r - 1) * R + c];
            }
        }
        return s;
    });
}

// store v * xscale (a power of two), rounded once to FP16, at (U dof u, column c) of the
// apply layout; the thread of the last Gamma dof of a subdomain zeroes the column's padding
__device__ __forceinline__ __half to_half(double v) { return __double2half(v); }
__device__ __forceinline__ __half to_half(float v) { return __float2half_rn(v); }
template <typename V>
__device__ __forceinline__ void store_f16(__half *x, const SubdomainDesc *sd, const int32_t *u2sub, int64_t u, int c,
                                          int R, V v) {
    const SubdomainDesc &d = sd[u2sub[u]];
    const int64_t col = d.offUp * R + (int64_t)c * d.ldG;
    const int j = (int)(u - d.offU);
    x[col + j] = to_half(v);
    if (j == d.nG - 1)
        for (int q = d.nG; q < d.ldG; ++q) x[col + q] = __float2half(0.0f);
}

// x (apply layout, FP16) = xscale B_D^T v for the tensor-core preconditioner apply (the sums
// of k_gather_apply in the type of the Lambda vectors, scaled exactly, rounded once)
template <typename L>
__global__ void k_gather_apply_f16(const int64_t *ptr, const int64_t *row, const L *val, const L *v, const L *xscale,
                                   __half *x, const SubdomainDesc *sd, const int32_t *u2sub, int64_t nu, int R,
                                   const int *gate) {
    if (gate && *gate == 0) return;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nu * R; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / nu);
        const int64_t u = t % nu;
        L s = 0;
        for (int64_t q = ptr[u]; q < ptr[u + 1]; ++q) s += val[q] * v[row[q] * R + c];
        store_f16(x, sd, u2sub, u, c, R, s * xscale[c]);
    }
}

// xscale[c] = 2^-floor(log2 max_u |v[u][c]|) (1 for a zero column); grid R blocks
__global__ void __launch_bounds__(256) k_col_scale(const double *v, int64_t n, int R, double *xscale) {
    __shared__ double red[8];
    const int c = blockIdx.x;
    double m = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(v[i * R + c]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) m = fmax(m, red[w]);
        m = fmax(m, red[0]);
        xscale[c] = (m > 0.0 && m < INFINITY) ? ldexp(1.0, -ilogb(m)) : 1.0;
    }
}

// U vectors (interleaved, FP64) -> FP16 apply layout, column c scaled by xscale[c]
__global__ void k_to_apply_f16(const double *uU, const double *xscale, __half *x, const SubdomainDesc *sd,
                               const int32_t *u2sub, int64_t nu, int R) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nu * R; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / nu);
        const int64_t u = t % nu;
        store_f16(x, sd, u2sub, u, c, R, uU[u * R + c] * xscale[c]);
    }
}

// right-hand side of the forcing (MODE ROWS_FORCING: f_O) or of the back substitution
// (ROWS_BACKSUB: [f_O; u_G]) per subdomain, R columns of ld_M entries at offVp * R, zero past
// the block's columns: the values (and conversions) k_rows stages in shared memory.  Grid (K, R).
template <typename T, int MODE>
__global__ void k_stage_rows_x(const double *xa, const double *xb, const SubdomainDesc *sd, T *xs, int R) {
    const SubdomainDesc d = sd[blockIdx.x];
    const int c = blockIdx.y;
    const int ncols = MODE == ROWS_FORCING ? d.nO : d.nk;
    for (int l = threadIdx.x; l < d.ldM; l += blockDim.x) {
        T v = T(0);
        if (l < ncols) {
            if (MODE == ROWS_FORCING || l < d.nO) v = (T)xa[(d.offV + l) * R + c];
            else v = (T)xb[(d.offU + l - d.nO) * R + c];
        }
        xs[d.offVp * R + (int64_t)c * d.ldM + l] = v;
    }
}

// alpha = (G^T G)^-1 G^T v.  G^T v is gathered from flat entry lists per floating subdomain
// f: for v on Lambda, entry e of B^T restricted to Gamma_f is (Lambda row rows[e], weights
// w[e][q] = sign(e) Z[u(e)][q]); for v on U, the entries are the U dofs of Gamma_f with
// weights Z.  Grid (floating subdomains, psplit slices of the entry range, right-hand sides):
// block (f, j, c) sums slice j into gpart.  Small coarse spaces (fused): the last block to
// arrive adds the slices in order (into shared memory when they fit, else gsum) and applies
// (G^T G)^-1.  Large ones: k_coarse_solve does that over many CTAs (FP64 runs at a small
// fraction of the FP32 rate here, so one CTA would take ~100 us for n_co = 108 and 16
// right-hand sides).  In the FP32 pass the large ones are fused per column instead (fused = 2,
// one slice): the last of a column's blocks to arrive applies the FP32 copy of (G^T G)^-1,
// stored transposed (GtGinv32[j n_co + i] = (G^T G)^-1[i][j]), to that column, thread i
// summing over j in ascending order (n_co^2 FP32 FMAs per column: a few thousand cycles of
// one SM).  psplit and the choice depend on the problem only, so every column is summed in the
// same order whatever batch it is part of.
// v_mode: PG_U v on U; PG_LAM v on Lambda; PG_LAM_R r_new = r - eta q on Lambda (v = r)
constexpr int PSPLIT = 8;
constexpr int kCoarseFusedMax = 16;     // n_co up to which the last block of k_proj_g solves
constexpr int kCoarseColMax = 2048;     // n_co up to which the FP32 pass fuses per column
enum { PG_U = 0, PG_LAM = 1, PG_LAM_R = 2 };

// true in the last of column c's blocks (gridDim.x gridDim.y of them) to arrive
__device__ __forceinline__ bool arrive_last_col(unsigned *counters, int c) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&counters[c], 1u) == gridDim.x * gridDim.y - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// L: the type of v, q, the weights, the per-block sums and alpha (FP32 in the FP32 pass, with
// FP32 copies of the weights); the slices' sums and (G^T G)^-1 are FP64 (but for fused = 2).
template <int VMODE, typename L>
__global__ void __launch_bounds__(256) k_proj_g(const int64_t *range, const int32_t *fco, const int64_t *rows,
                                                const L *w, const L *v, const L *q, const L *eta, double *gpart,
                                                double *gsum, const double *GtGinv, int nco, L *alpha, int R,
                                                unsigned *counter, int psplit, int fused,
                                                const float *GtGinv32 = nullptr, unsigned *colcnt = nullptr) {
    constexpr int lam_mode = VMODE != PG_U;
    extern __shared__ double gs_dyn[];
    __shared__ L red[8][3];
    const int f = blockIdx.x, c = blockIdx.z;
    const int64_t e0 = range[4 * f + (lam_mode ? 0 : 2)], e1 = range[4 * f + (lam_mode ? 1 : 3)];
    const int co_off = fco[2 * f], nq = fco[2 * f + 1];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t chunk = (e1 - e0 + psplit - 1) / psplit;
    const int64_t l0 = e0 + blockIdx.y * chunk, l1 = min(e1, l0 + chunk);
    L acc[3] = {0, 0, 0};
    const L eta_c = VMODE == PG_LAM_R ? eta[c] : L(0);
    // a thread's entries e0, e0 + 256, ... taken PGU at a time: the loads of PGU entries (row
    // index, then the gathered value) in flight together, the products added in ascending e
    constexpr int PGU = 8;
    for (int64_t e0 = l0 + threadIdx.x; e0 < l1; e0 += PGU * (int64_t)blockDim.x) {
        int64_t rr[PGU];
        L xv[PGU];
#pragma unroll
        for (int m = 0; m < PGU; ++m) {
            const int64_t e = e0 + (int64_t)m * blockDim.x;
            rr[m] = (VMODE != PG_U && e < l1) ? rows[e] : 0;
        }
#pragma unroll
        for (int m = 0; m < PGU; ++m) {
            const int64_t e = e0 + (int64_t)m * blockDim.x;
            L x = 0;
            if (e < l1) {
                if (VMODE == PG_U) x = v[e * R + c];
                else if (VMODE == PG_LAM) x = v[rr[m] * R + c];
                else x = r_next(v[rr[m] * R + c], q[rr[m] * R + c], eta_c);
            }
            xv[m] = x;
        }
#pragma unroll
        for (int m = 0; m < PGU; ++m) {
            const int64_t e = e0 + (int64_t)m * blockDim.x;
            if (e < l1) {
#pragma unroll
                for (int qq = 0; qq < 3; ++qq) acc[qq] += w[e * 3 + qq] * xv[m];
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) acc[q] = warp_sum(acc[q]);
    if (lane == 0)
        for (int q = 0; q < 3; ++q) red[warp][q] = acc[q];
    __syncthreads();
    if (threadIdx.x < nq) {
        L x = 0;
        for (int ww = 0; ww < 8; ++ww) x += red[ww][threadIdx.x];
        gpart[((int64_t)(co_off + threadIdx.x) * psplit + blockIdx.y) * R + c] = (double)x;
    }
    if (!fused) return;
    if constexpr (std::is_same<L, float>::value) {
        if (fused == 2) {
            if (!arrive_last_col(colcnt, c)) return;
            float *gc = reinterpret_cast<float *>(gs_dyn);       // n_co entries of G^T v, column c
            for (int j = threadIdx.x; j < nco; j += blockDim.x) {
                double g = 0;
                for (int s = 0; s < psplit; ++s) g += __ldcg(gpart + ((int64_t)j * psplit + s) * R + c);
                gc[j] = (float)g;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < nco; i += blockDim.x) {
                // j ascending; the loads of 16 consecutive j in flight together
                float a = 0.0f;
                int j = 0;
                for (; j + 16 <= nco; j += 16) {
                    float gv[16];
#pragma unroll
                    for (int m = 0; m < 16; ++m) gv[m] = __ldg(GtGinv32 + (int64_t)(j + m) * nco + i);
#pragma unroll
                    for (int m = 0; m < 16; ++m) a = __fmaf_rn(gv[m], gc[j + m], a);
                }
                for (; j < nco; ++j) a = __fmaf_rn(__ldg(GtGinv32 + (int64_t)j * nco + i), gc[j], a);
                alpha[(int64_t)i * R + c] = a;
            }
            if (threadIdx.x == 0) colcnt[c] = 0u;
            return;
        }
    }
    if (!arrive_last(counter)) return;
    double *gs = gsum ? gsum : gs_dyn;
    for (int t = threadIdx.x; t < nco * R; t += blockDim.x) {
        const int i = t / R, cc = t % R;
        double g = 0;
        for (int j = 0; j < psplit; ++j) g += __ldcg(gpart + ((int64_t)i * psplit + j) * R + cc);
        gs[t] = g;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nco * R; t += blockDim.x) {
        const int i = t / R, cc = t % R;
        double a = 0;
        for (int j = 0; j < nco; ++j) a += GtGinv[(int64_t)i * nco + j] * gs[(int64_t)j * R + cc];
        alpha[t] = (L)a;
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// alpha[i][c] = sum_j (G^T G)^-1[i][j] (G^T v)[j][c], G^T v summed from the psplit slices of
// k_proj_g: one warp per (i, c), lanes over j (fixed order: per lane ascending, then the warp
// tree).  Grid (ceil(n_co / 8), R), 256 threads.
template <typename L>
__global__ void __launch_bounds__(256) k_coarse_solve(const double *gpart, int psplit, const double *GtGinv, int nco,
                                                      L *alpha, int R) {
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int i = blockIdx.x * 8 + warp, c = blockIdx.y;
    if (i >= nco) return;
    double a = 0;
    for (int j = lane; j < nco; j += 32) {
        double g = 0;
        for (int s = 0; s < psplit; ++s) g += __ldcg(gpart + ((int64_t)j * psplit + s) * R + c);
        a += GtGinv[(int64_t)i * nco + j] * g;
    }
    a = warp_sum(a);
    if (lane == 0) alpha[(int64_t)i * R + c] = (L)a;
}

// refinement update u += du with corr = max |du| / max |u| per column: grid (row blocks,
// right-hand sides), per-block maxima, the last block to arrive writes corr (maxima do not
// depend on the order)
__global__ void __launch_bounds__(RED_THREADS) k_refine_update(double *u, const double *du, int64_t n, int R,
                                                                double *pa, double *pb, PcgScalars s) {
    __shared__ double ra[RED_THREADS / 32], rb[RED_THREADS / 32];
    const int c = blockIdx.y, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    double ma = 0, mb = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = du[i * R + c], v = u[i * R + c] + d;
        u[i * R + c] = v;
        ma = fmax(ma, fabs(d));
        mb = fmax(mb, fabs(v));
    }
    for (int o = 16; o > 0; o >>= 1) {
        ma = fmax(ma, __shfl_xor_sync(0xffffffffu, ma, o));
        mb = fmax(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    }
    if (lane == 0) { ra[warp] = ma; rb[warp] = mb; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, y = 0;
        for (int w = 0; w < RED_THREADS / 32; ++w) { x = fmax(x, ra[w]); y = fmax(y, rb[w]); }
        pa[(int64_t)blockIdx.x * R + c] = x;
        pb[(int64_t)blockIdx.x * R + c] = y;
    }
    if (!arrive_last(s.counter)) return;
    for (int cc = warp; cc < R; cc += RED_THREADS / 32) {
        double x = 0, y = 0;
        for (int bl = lane; bl < (int)gridDim.x; bl += 32) {
            x = fmax(x, __ldcg(pa + (int64_t)bl * R + cc));
            y = fmax(y, __ldcg(pb + (int64_t)bl * R + cc));
        }
        for (int o = 16; o > 0; o >>= 1) {
            x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
            y = fmax(y, __shfl_xor_sync(0xffffffffu, y, o));
        }
        if (lane == 0) s.corr[cc] = y > 0 ? x / y : (x > 0 ? 1.0 : 0.0);
    }
    if (threadIdx.x == 0) *s.counter = 0u;
}

// ====================================================================== single-domain CG
//
// Diagonally preconditioned CG on A u = b over the global dofs: the performance baseline of
// the paper's experiments (section "Considered solver strategies"), FP64, R right-hand sides
// interleaved (entry g of column c at g*R + c), each column frozen once ||r|| <= tol ||b|| or
// after max_it iterations:
//   q = A p;  alpha = (r, z) / (p, q);  u += alpha p;  r -= alpha q;  z = D^-1 r;
//   beta = (r, z)_new / (r, z)_old;  p = z + beta p.
// A is the CSR of cg_prepare; b = sum over the subdomain copies of each dof of the split
// loads (they sum to F - A_D g).  FP64 has a small share of this GPU's arithmetic, so the
// SpMV runs in double-single arithmetic on the FP32 pipes: A and p as FP32 pairs (hi + lo,
// 2^-48 relative), each product's rounding error kept exactly (fma), sums by TwoSum per lane
// (the scheme of the refinement residual), lane sums in FP64.  The scalar block holds the CG state in the PCG's slots:
// nPd = ||b||, yw = (r, z), eta = alpha, beta, relres = ||r|| / ||b||, active, iters,
// n_active, loops.  Every reduction has a fixed order that does not depend on R.

constexpr int CG_WARPS = 8;                   // warps (rows at a time) of a SpMV block
constexpr int CG_BLOCKS = 8 * 152;            // SpMV blocks (rows strided over them; 64 warps per SM)
constexpr int CG_MAX_R = 32;                  // right-hand sides per CG call
constexpr int CG_U = 8;                       // nonzeros per SpMV slot loaded at a time

// b[g] = sum of f~ over the copies of dof g
__global__ void k_cg_rhs(const double *ftil, const int64_t *cp_ptr, const int64_t *cp_pos, int64_t n, int R,
                         double *b) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * R; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = t / R;
        const int c = (int)(t % R);
        double s = 0;
        for (int64_t q = cp_ptr[g]; q < cp_ptr[g + 1]; ++q) s += ftil[cp_pos[q] * R + c];
        b[t] = s;
    }
}

// p as FP32 pairs for the SpMV: hi = fl32(p), lo = fl32(p - hi)
__device__ __forceinline__ void split_f2(double v, float *hi, float *lo, int64_t t) {
    const float h = __double2float_rn(v);
    hi[t] = h;
    lo[t] = __double2float_rn(v - (double)h);
}

// u = 0, r = b, z = D^-1 b, p = z; (r, z) and (b, b); the initial state
__global__ void __launch_bounds__(RED_THREADS) k_cg_init(const double *b, const double *dinv, double *u, double *r,
                                                          double *z, double *p, float *ph, float *pl, int64_t n, int R,
                                                          double *pa, double *pb, PcgScalars s) {
    const int c = blockIdx.y;
    double a1 = 0, a2 = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i * R + c;
        const double bv = b[t], zv = dinv[i] * bv;
        u[t] = 0.0;
        r[t] = bv;
        z[t] = zv;
        p[t] = zv;
        split_f2(zv, ph, pl, t);
        a1 += bv * zv;
        a2 += bv * bv;
    }
    block_partial(a1, pa, R);
    __syncthreads();
    block_partial(a2, pb, R);
    if (!arrive_last(s.counter)) return;
    __shared__ int n_act;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) n_act = 0;
    __syncthreads();
    for (int cc = warp; cc < R; cc += RED_THREADS / 32) {
        double rz = 0, bb = 0;
        for (int bl = lane; bl < (int)gridDim.x; bl += 32) {
            rz += __ldcg(pa + (int64_t)bl * R + cc);
            bb += __ldcg(pb + (int64_t)bl * R + cc);
        }
        rz = warp_sum(rz);
        bb = warp_sum(bb);
        if (lane == 0) {
            const int act = bb > 0.0 ? 1 : 0;
            s.nPd[cc] = sqrt(bb);
            s.yw[cc] = rz;
            s.eta[cc] = 0.0;
            s.beta[cc] = 0.0;
            s.relres[cc] = act ? 1.0 : 0.0;
            s.iters[cc] = 0;
            s.active[cc] = act;
            if (act) atomicAdd(&n_act, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *s.n_active = n_act;
        *s.counter = 0u;
    }
}

// q = A p (warp per row, double-single products), (p, q) per column, alpha for the active
// columns.  Lanes are (nonzero slot kg = lane / 8, column cl = lane % 8): the 8 lanes of a slot
// read one nonzero and the 8 consecutive p entries of its column index (one 32-byte segment
// of hi and one of lo), the 4 slots take every 4th nonzero of the row; the slots are summed by
// two shuffles.  Columns come in blocks of 8; each column's arithmetic is the same whatever R.
__global__ void __launch_bounds__(CG_WARPS * 32) k_cg_spmv(const int64_t *ptr, const int32_t *col, const float *vhi,
                                                           const float *vlo, const float *ph, const float *pl,
                                                           const double *p, double *q, int64_t n, int R, double *part,
                                                           PcgScalars s) {
    __shared__ double red[CG_WARPS][CG_MAX_R];
    if (*s.n_active == 0) return;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, kg = lane >> 3, cl = lane & 7;
    constexpr int NCB = CG_MAX_R / 8;
    double dacc[NCB];
#pragma unroll
    for (int cb = 0; cb < NCB; ++cb) dacc[cb] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * CG_WARPS + warp; i < n; i += (int64_t)gridDim.x * CG_WARPS) {
        const int64_t a = ptr[i], e = ptr[i + 1];
#pragma unroll
        for (int cb = 0; cb < NCB; ++cb) {
            const int c = cb * 8 + cl;
            if (cb * 8 < R) {
                const bool on = c < R;
                float sh = 0.f, sl = 0.f;
                // CG_U nonzeros per slot at a time: their matrix loads first, then their p
                // gathers, then the products in order (loads in flight cover DRAM latency)
                for (int64_t k0 = a + kg; k0 < e; k0 += 4 * CG_U) {
                    float ahv[CG_U], alv[CG_U];
                    int64_t jv[CG_U];
#pragma unroll
                    for (int u = 0; u < CG_U; ++u) {
                        const int64_t k = k0 + 4 * u;
                        const bool in = k < e;
                        ahv[u] = in ? __ldg(vhi + k) : 0.f;
                        alv[u] = in ? __ldg(vlo + k) : 0.f;
                        jv[u] = in ? (int64_t)__ldg(col + k) : -1;
                    }
                    float xhv[CG_U], xlv[CG_U];
#pragma unroll
                    for (int u = 0; u < CG_U; ++u) {
                        const bool in = on && jv[u] >= 0;
                        xhv[u] = in ? __ldg(ph + jv[u] * R + c) : 0.f;
                        xlv[u] = in ? __ldg(pl + jv[u] * R + c) : 0.f;
                    }
#pragma unroll
                    for (int u = 0; u < CG_U; ++u) {
                        if (!on || jv[u] < 0) continue;
                        const float ah = ahv[u], al = alv[u], xh = xhv[u], xl = xlv[u];
                        // explicit round-to-nearest intrinsics: no contraction into fma
                        const float pr = __fmul_rn(ah, xh);
                        const float pe = fmaf(ah, xh, -pr);              // ah*xh - pr exactly
                        const float sum = __fadd_rn(sh, pr);             // TwoSum(sh, pr)
                        const float bb = __fsub_rn(sum, sh);
                        const float se = __fadd_rn(__fsub_rn(sh, __fsub_rn(sum, bb)), __fsub_rn(pr, bb));
                        sh = sum;
                        sl = __fadd_rn(sl, __fadd_rn(se, fmaf(ah, xl, fmaf(al, xh, pe))));
                    }
                }
                double acc = (double)sh + (double)sl;
                acc += __shfl_xor_sync(0xffffffffu, acc, 8);
                acc += __shfl_xor_sync(0xffffffffu, acc, 16);
                if (kg == 0 && on) {
                    q[i * R + c] = acc;
                    dacc[cb] += p[i * R + c] * acc;
                }
            }
        }
    }
    // block sums per column, warps in order
#pragma unroll
    for (int cb = 0; cb < NCB; ++cb) {
        const int c = cb * 8 + cl;
        if (kg == 0 && c < R) red[warp][c] = dacc[cb];
    }
    __syncthreads();
    if (threadIdx.x < R) {
        double x = 0;
        for (int w = 0; w < CG_WARPS; ++w) x += red[w][threadIdx.x];
        part[(int64_t)blockIdx.x * R + threadIdx.x] = x;
    }
    if (!arrive_last(s.counter)) return;
    for (int cc = warp; cc < R; cc += CG_WARPS) {
        double pq = 0;
        for (int bl = lane; bl < (int)gridDim.x; bl += 32) pq += __ldcg(part + (int64_t)bl * R + cc);
        pq = warp_sum(pq);
        if (lane == 0) s.eta[cc] = (s.active[cc] && pq != 0.0) ? s.yw[cc] / pq : 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) *s.counter = 0u;
}

// u += alpha p, r -= alpha q, z = D^-1 r; (r, z), (r, r); beta and the stop test.  COND: the
// last block also counts the iteration and sets the WHILE condition (continue while a column
// is active and fewer than limit iterations have run)
template <int COND>
__global__ void __launch_bounds__(RED_THREADS) k_cg_update(const double *dinv, const double *p, const double *q,
                                                            double *u, double *r, double *z, int64_t n, int R,
                                                            double *pa, double *pb, PcgScalars s, double tol,
                                                            int max_it, cudaGraphConditionalHandle cond, int limit) {
    if (*s.n_active == 0) {
        if (COND && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
        return;
    }
    const int c = blockIdx.y;
    const double al = s.eta[c];
    double a1 = 0, a2 = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i * R + c;
        u[t] = __fma_rn(al, p[t], u[t]);
        const double rn = __fma_rn(-al, q[t], r[t]), zn = dinv[i] * rn;
        r[t] = rn;
        z[t] = zn;
        a1 += rn * zn;
        a2 += rn * rn;
    }
    block_partial(a1, pa, R);
    __syncthreads();
    block_partial(a2, pb, R);
    if (!arrive_last(s.counter)) return;
    __shared__ int n_act;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) n_act = 0;
    __syncthreads();
    for (int cc = warp; cc < R; cc += RED_THREADS / 32) {
        double rz = 0, rr = 0;
        for (int bl = lane; bl < (int)gridDim.x; bl += 32) {
            rz += __ldcg(pa + (int64_t)bl * R + cc);
            rr += __ldcg(pb + (int64_t)bl * R + cc);
        }
        rz = warp_sum(rz);
        rr = warp_sum(rr);
        if (lane == 0) {
            int act = s.active[cc];
            if (act) {
                const int it = s.iters[cc] + 1;
                s.iters[cc] = it;
                const double nb = s.nPd[cc], rel = nb > 0 ? sqrt(rr) / nb : 0.0;
                s.relres[cc] = rel;
                s.beta[cc] = s.yw[cc] != 0.0 ? rz / s.yw[cc] : 0.0;
                s.yw[cc] = rz;
                if (rel <= tol || it >= max_it) act = 0;
                s.active[cc] = act;
            }
            if (act) atomicAdd(&n_act, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *s.n_active = n_act;
        *s.counter = 0u;
        if (COND) {
            const int l = *s.loops + 1;
            *s.loops = l;
            cudaGraphSetConditional(cond, (n_act > 0 && l < limit) ? 1u : 0u);
        }
    }
}

// p = z + beta p on the active columns (and its FP32 pair)
__global__ void k_cg_p(const double *z, double *p, float *ph, float *pl, int64_t n, int R, PcgScalars s) {
    if (*s.n_active == 0) return;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * R; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t % R);
        if (s.active[c]) {
            const double v = __fma_rn(s.beta[c], p[t], z[t]);
            p[t] = v;
            split_f2(v, ph, pl, t);
        }
    }
}

// nodal output of the CG solution: u on the free dofs, g (or 0) on the Dirichlet dofs
__global__ void k_cg_output(const double *u, const int8_t *node_dir, int nc, const double *g, int64_t ndof, int R,
                            double *out) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ndof * R; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t gd = t % ndof;
        const int c = (int)(t / ndof);
        out[t] = node_dir[gd / nc] ? (g ? g[(int64_t)c * ndof + gd] : 0.0) : u[gd * R + c];
    }
}

// ====================================================================== host orchestration

// the workspace's error word (set by a device wait that ran out)
inline int *ws_err(SolveWS &ws, int R) { return reinterpret_cast<int *>(ws.scal.as<double>() + 7 * R) + 2 * R + 3; }

// ws.res = ftil - A^k u - [0; B^T lambda] on every subdomain (double-single, FP32 pool pairs):
// u is first split into FP32 hi / lo pairs, then the sparse kernel (A^k kept as a CSR) or the
// dense pipeline kernel runs.  Returns the number of kernels launched.
int residual_ds(nlfeti_problem *p, SolveWS &ws, cudaStream_t st, int R, const double *lam) {
    const OpPool<float> &pool = p->op32;
    if (pool.a_sparse) {
        const int64_t nrows = p->sum_nk;
        if (nrows == 0) return 0;
        const int P = (R + 1) / 2;
        int sms = 0;
        NLF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->ctx->device));
        float2 *uh = reinterpret_cast<float2 *>(ws.uhl.as<float>()), *ul = uh + nrows * P;
        k_split_u_rows<<<grid_for(nrows * P), 256, 0, st>>>(ws.u.as<double>(), uh, ul, nrows, R);
        auto go = [&](auto lpr_tag) {
            constexpr int LPR = decltype(lpr_tag)::value;
            // one CTA per SM, each over a contiguous range of rows
            const int ctas = (int)std::max<int64_t>(1, std::min<int64_t>(sms, (nrows * LPR + RES_CSR_THREADS - 1) /
                                                                                 RES_CSR_THREADS));
            k_residual_csr<LPR><<<ctas, RES_CSR_THREADS, 0, st>>>(
                pool.Aptr.as<int64_t>(), pool.Aent.as<int4>(), pool.row_u.as<int32_t>(), uh, ul, ws.ftil.as<double>(),
                p->d_Bt_ptr.as<int64_t>(), p->d_Bt_row.as<int64_t>(), lam, ws.res.as<double>(), nrows, R);
        };
        if (P > 16) go(std::integral_constant<int, 32>{});
        else if (P > 8) go(std::integral_constant<int, 16>{});
        else if (P > 4) go(std::integral_constant<int, 8>{});
        else if (P > 2) go(std::integral_constant<int, 4>{});
        else if (P > 1) go(std::integral_constant<int, 2>{});
        else go(std::integral_constant<int, 1>{});
        return 2;
    }
    if (p->rsched_ctas == 0) return 0;
    const int R2 = (R + 1) / 2 * 2;
    float *uh = ws.uhl.as<float>(), *ul = uh + std::max<int64_t>(1, p->n_vp) * R2;
    k_split_u<<<dim3(p->K, R2), 256, 0, st>>>(ws.u.as<double>(), p->d_sd.as<SubdomainDesc>(), uh, ul, R);
    auto go = [&](auto rc_tag) {
        constexpr int RC = decltype(rc_tag)::value;
        k_residual_tma<RC><<<p->rsched_ctas, RES_THREADS, res_smem_bytes(RC), st>>>(
            pool.amaps.as<CUtensorMap>(), ws.umaps.as<CUtensorMap>(), p->d_sd.as<SubdomainDesc>(),
            p->d_rsched_ptr.as<int32_t>(), p->d_rsched_items.as<int32_t>(), ws.ftil.as<double>(),
            p->d_Bt_ptr.as<int64_t>(), p->d_Bt_row.as<int64_t>(), lam, ws.res.as<double>(), R, ws_err(ws, R));
    };
    if (R >= 8) go(std::integral_constant<int, 8>{});
    else if (R >= 4) go(std::integral_constant<int, 4>{});
    else if (R >= 2) go(std::integral_constant<int, 2>{});
    else go(std::integral_constant<int, 1>{});
    return 2;
}

// the interface apply's input buffer of an arithmetic type: FP32 in the paired layout (xP),
// FP64 in the column layout (xU)
template <typename T> T *apply_input(SolveWS &ws) {
    if constexpr (std::is_same<T, float>::value) return ws.xP.as<float>();
    else return ws.xU.as<T>();
}

struct Runner {
    nlfeti_problem *p;
    SolveWS &ws;
    cudaStream_t st;
    int R;
    PcgScalars S;
    const SubdomainDesc *sd;
    // kernel accounting: launches made eagerly, launches recorded into the graph being
    // captured, and event pairs around the interface applies (graph slots are re-recorded
    // by every launch of the graph)
    bool capturing = false;
    int64_t eager_launches = 0, cap_launches = 0;
    struct Slot {
        cudaEvent_t a, b;
        int launches;
        double bytes;
        bool half;          // an apply of the FP16 preconditioner copy
        int flag = -1;      // word of ws.slot_flags holding the gate (active columns) the apply saw
    };
    std::vector<Slot> graph_slots, eager_slots;
    int next_graph_flag = 0, next_eager_flag = 0;
    // inside PCG iterations: the interface applies and their gathers return at once when no
    // right-hand side is active any more (every later update is masked by the active flags)
    const int *gate = nullptr;
    int64_t loop_body_launches = 0;     // kernels per iteration of the last device-side loop
    // the WHILE node of the graph loop being captured (set by k_check_update)
    cudaGraphConditionalHandle cond = 0;
    // set (FP32 PCG iterations): the interface applies store their results here in FP32 instead
    // of the FP64 output they are given
    float *yout_f = nullptr;
    bool use_cond = false;
    int64_t apply_launches = 0, half_launches = 0;
    double apply_ms = 0, apply_bytes = 0, half_ms = 0, half_bytes = 0;
    std::vector<int> slot_flags_host;

    Runner(nlfeti_problem *pp, SolveWS &w, cudaStream_t s) : p(pp), ws(w), st(s), R(w.R) {
        double *b = ws.scal.as<double>();
        S.nPd = b; S.yw_old = b + R; S.yw = b + 2 * R; S.eta = b + 3 * R; S.beta = b + 4 * R; S.relres = b + 5 * R;
        S.corr = b + 6 * R;
        S.xscale = ws.xscale.as<double>();
        int *ib = reinterpret_cast<int *>(b + 7 * R);
        S.active = ib; S.iters = ib + R; S.n_active = ib + 2 * R; S.loops = ib + 2 * R + 1;
        S.counter = reinterpret_cast<unsigned *>(ib + 2 * R + 2);
        S.err = ib + 2 * R + 3;
        float *fb = reinterpret_cast<float *>(ib + 2 * R + 8);
        S.eta_f = fb; S.beta_f = fb + R; S.xscale_f = fb + 2 * R;
        S.colcnt = reinterpret_cast<unsigned *>(fb + 3 * R);
        sd = p->d_sd.as<SubdomainDesc>();
        set_attributes();
    }

    template <int MODE> void dot_final(const double *a, const double *b, int64_t n, double tol = 0, int max_it = 0) {
        k_dot_final<MODE><<<tile_blocks(n), TILE_THREADS, 0, st>>>(a, b, n, R, ws.partial.as<double>(), S, tol, max_it);
        note_launch();
    }

    ~Runner() {
        harvest(eager_slots, true);
        drop(graph_slots);
        std::lock_guard<std::mutex> g(p->prof_mu);
        p->prof.kernel_launches += eager_launches;
        p->prof.apply_launches += apply_launches;
        p->prof.apply_ms += apply_ms;
        p->prof.apply_bytes += apply_bytes;
        p->prof.half_apply_launches += half_launches;
        p->prof.half_apply_ms += half_ms;
        p->prof.half_apply_bytes += half_bytes;
    }

    // read the error word of the bounded waits and report a wait that ran out
    void check_waits_now() {
        NLF_CUDA(cudaMemcpyAsync(ws.host_flag.data(), S.n_active, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
        NLF_CUDA(cudaStreamSynchronize(st));
        check_waits();
    }

    // after a read-back of the scalar words n_active .. err into host_flag
    void check_waits() {
        if (ws.host_flag[3] == 0) return;
        NLF_CUDA(cudaMemsetAsync(S.err, 0, sizeof(int), st));
        fail(NLFETI_E_TIMEOUT, "a device-side wait of the interface apply ran out of time");
    }

    void note_launch() {
        if (capturing) ++cap_launches;
        else ++eager_launches;
    }

    void drop(std::vector<Slot> &v) {
        for (auto &s : v) { cudaEventDestroy(s.a); cudaEventDestroy(s.b); }
        v.clear();
        if (&v == &graph_slots) next_graph_flag = 0;
        else next_eager_flag = 0;
    }

    // a timed apply inside the PCG loop copies its gate (the number of active columns) into a
    // flag word, so that the harvest counts only the launches that did the work (a gated
    // launch returns at once; the chunked loop runs up to chunk - 1 of them per pass)
    int snapshot_gate() {
        if (!gate) return -1;
        int idx = -1;
        if (capturing && next_graph_flag < kSlotFlags / 2) idx = next_graph_flag++;
        if (!capturing && next_eager_flag < kSlotFlags / 2) idx = kSlotFlags / 2 + next_eager_flag++;
        if (idx >= 0)
            NLF_CUDA(cudaMemcpyAsync(ws.slot_flags.as<int>() + idx, gate, sizeof(int), cudaMemcpyDeviceToDevice, st));
        return idx;
    }

    // add the elapsed times of completed slots (the stream has been synchronized); slots whose
    // gate was zero (the apply returned at once) are left out
    void harvest(std::vector<Slot> &v, bool clear) {
        bool any = false;
        for (auto &s : v) any |= s.flag >= 0;
        if (any) {
            slot_flags_host.resize(kSlotFlags);
            NLF_CUDA(cudaMemcpyAsync(slot_flags_host.data(), ws.slot_flags.p, sizeof(int) * kSlotFlags,
                                     cudaMemcpyDeviceToHost, st));
            NLF_CUDA(cudaStreamSynchronize(st));
        }
        for (auto &s : v) {
            float ms = 0.f;
            if (s.flag >= 0 && slot_flags_host[s.flag] == 0) continue;
            if (cudaEventElapsedTime(&ms, s.a, s.b) == cudaSuccess) {
                (s.half ? half_ms : apply_ms) += ms;
                (s.half ? half_launches : apply_launches) += s.launches;
                (s.half ? half_bytes : apply_bytes) += s.bytes;
            } else {
                cudaGetLastError();
            }
        }
        if (clear) drop(v);
    }

    // The arithmetic type L of the Lambda vectors: FP64, or FP32 in the PCG iterations of the
    // FP32 pass, which read FP32 copies of the weights of G, G^T and B_D.
    template <typename L> static const L *wt(const DevMem &d64, const DevMem &d32) {
        if constexpr (std::is_same<L, float>::value) return d32.as<float>();
        else return d64.as<double>();
    }
    template <typename L> const L *eta_ptr() const {
        if constexpr (std::is_same<L, float>::value) return S.eta_f;
        else return S.eta;
    }
    template <typename L> const L *beta_ptr() const {
        if constexpr (std::is_same<L, float>::value) return S.beta_f;
        else return S.beta;
    }
    template <typename L> const L *xscale_ptr() const {
        if constexpr (std::is_same<L, float>::value) return S.xscale_f;
        else return ws.xscale.as<double>();
    }
    // the PCG vectors of the iterations (r, w, z, y, p, q, lambda) in L
    template <typename L> struct LamVecs { L *r, *w, *z, *y, *pv, *q, *lam; };
    template <typename L> LamVecs<L> lam_vecs() {
        if constexpr (std::is_same<L, float>::value) {
            const int64_t n = std::max<int64_t>(1, p->n_lambda) * R;
            float *b = ws.lamf.as<float>();
            return {b, b + n, b + 2 * n, b + 3 * n, b + 4 * n, b + 5 * n, b + 6 * n};
        } else {
            return {ws.r.as<double>(), ws.w.as<double>(), ws.z.as<double>(), ws.y.as<double>(), ws.pv.as<double>(),
                    ws.q.as<double>(), ws.dlam.as<double>()};
        }
    }

    // alpha = (G^T G)^-1 G^T v: v on U (PG_U, FP64), on Lambda (PG_LAM) or r_new = v - eta q
    // (PG_LAM_R); alpha in L
    template <typename L> void coarse_alpha(const L *v, int vmode, const L *q = nullptr) {
        const bool fused = p->n_co <= kCoarseFusedMax;
        const bool colfused = std::is_same<L, float>::value && !fused && p->n_co <= kCoarseColMax;
        const int psplit = fused ? PSPLIT : 1;
        const size_t gs_bytes = sizeof(double) * (size_t)p->n_co * R;
        const bool in_smem = fused && gs_bytes <= 32768;
        const size_t smem = in_smem ? gs_bytes : (colfused ? sizeof(float) * (size_t)p->n_co : 0);
        L *alpha = ws.alpha.as<L>();
        auto go = [&](auto kern, const L *w) {
            kern<<<dim3(p->n_floating, psplit, R), 256, smem, st>>>(
                p->d_gt_range.as<int64_t>(), p->d_gt_co.as<int32_t>(), p->d_gt_rows.as<int64_t>(), w, v, q,
                eta_ptr<L>(), ws.gco.as<double>(), in_smem ? nullptr : ws.gsum.as<double>(), p->d_GtGinv.as<double>(),
                p->n_co, alpha, R, S.counter, psplit, fused ? 1 : (colfused ? 2 : 0), p->d_GtGinv32.as<float>(),
                S.colcnt);
        };
        if (vmode == PG_U) {
            if constexpr (std::is_same<L, double>::value) go(k_proj_g<PG_U, double>, p->d_Z.as<double>());
            else fail(NLFETI_E_INVALID, "the U-space coarse gather runs in FP64");
        } else if (vmode == PG_LAM) {
            go(k_proj_g<PG_LAM, L>, wt<L>(p->d_gt_w, p->d_gt_w32));
        } else {
            go(k_proj_g<PG_LAM_R, L>, wt<L>(p->d_gt_w, p->d_gt_w32));
        }
        note_launch();
        if (!fused && !colfused) {
            k_coarse_solve<L><<<dim3((p->n_co + 7) / 8, R), 256, 0, st>>>(ws.gco.as<double>(), psplit,
                                                                         p->d_GtGinv.as<double>(), p->n_co, alpha, R);
            note_launch();
        }
    }

    // out = P v (out may alias v)
    void project(const double *v, double *out) {
        const int64_t nl = p->n_lambda;
        if (p->n_co == 0) {
            if (out != v) NLF_CUDA(cudaMemcpyAsync(out, v, sizeof(double) * nl * R, cudaMemcpyDeviceToDevice, st));
            return;
        }
        coarse_alpha(v, PG_LAM);
        k_apply_galpha<<<grid_for(nl * R), 256, 0, st>>>(p->d_Gcol.as<int32_t>(), p->d_Gval.as<double>(), p->gw,
                                                         ws.alpha.as<double>(), v, -1.0, out, nl, R);
        note_launch();
    }

    // out = P v with the PCG dot product of MODE fused in (CHECK: (out, out); BETA: (out, other))
    template <int MODE, typename L> void project_dot(const L *v, const L *other, L *out, double tol = 0,
                                                     int max_it = 0) {
        const int64_t nl = p->n_lambda;
        if (p->n_co > 0) coarse_alpha<L>(v, PG_LAM);
        k_project_dot<MODE, L><<<tile_blocks(nl), TILE_THREADS, 0, st>>>(
            p->d_Gcol.as<int32_t>(), wt<L>(p->d_Gval, p->d_Gval32), p->gw, p->n_co > 0 ? ws.alpha.as<L>() : nullptr, v,
            other, out, nl, R, ws.partial.as<double>(), S, tol, max_it);
        note_launch();
    }

    template <typename T, int RC, int MODE, typename MT> void rows_launch(const MT *base, int use_sp, const int32_t *it,
                                                                         int nitems, const T *x, const double *xa,
                                                                         const double *xb, double *y, double oscale) {
        k_rows<T, RC, MODE, MT><<<nitems, 256, 0, st>>>(base, use_sp, sd, it, x, xa, xb, y, R,
                                                        MODE == ROWS_APPLY ? gate : nullptr, oscale,
                                                        MODE == ROWS_APPLY ? yout_f : nullptr);
        note_launch();
    }

    // one row-product stage over every subdomain: one launch (batched) or one per subdomain;
    // returns the number of launches.  MT: stored operator type (FP16 copy of S_k, result
    // scaled by oscale)
    template <typename T, int MODE, typename MT = T>
    int rows(const MT *base, int use_sp, const T *x, const double *xa, const double *xb, double *y, const DevMem &items,
             const std::vector<int> &off, double oscale = 1.0) {
        const int rc = R >= 8 ? 8 : (R >= 4 ? 4 : (R >= 2 ? 2 : 1));
        auto go = [&](const int32_t *it, int nitems) {
            if (nitems <= 0) return 0;
            switch (rc) {
                case 8: rows_launch<T, 8, MODE, MT>(base, use_sp, it, nitems, x, xa, xb, y, oscale); break;
                case 4: rows_launch<T, 4, MODE, MT>(base, use_sp, it, nitems, x, xa, xb, y, oscale); break;
                case 2: rows_launch<T, 2, MODE, MT>(base, use_sp, it, nitems, x, xa, xb, y, oscale); break;
                default: rows_launch<T, 1, MODE, MT>(base, use_sp, it, nitems, x, xa, xb, y, oscale); break;
            }
            return 1;
        };
        const int32_t *it = items.as<int32_t>();
        const int K = p->K;
        if (p->opt.batched) return go(it, off[K]);
        int launches = 0;
        for (int k = 0; k < K; ++k) launches += go(it + 2 * off[k], off[k + 1] - off[k]);
        return launches;
    }

    void set_attributes() {}

    // forcing / back substitution on the bulk-copy pipeline (batched): the right-hand sides are
    // staged once (k_stage_rows_x), then k_apply_tma in the row mode over its schedule
    template <typename T, int MODE> void rows_tma(const OpPool<T> &pool, const double *xa, const double *xb, double *y) {
        const int ctas = MODE == ROWS_FORCING ? p->fsched_ctas : p->osched_ctas;
        if (ctas <= 0) return;
        T *xs = ws.rxs.as<T>();
        k_stage_rows_x<T, MODE><<<dim3(p->K, R), 256, 0, st>>>(xa, xb, sd, xs, R);
        note_launch();
        const CUtensorMap *om = (MODE == ROWS_FORCING ? pool.fmaps : pool.omaps).template as<CUtensorMap>();
        const CUtensorMap *xm = ws.rxmaps[sizeof(T) == 8 ? 1 : 0].template as<CUtensorMap>();
        const int32_t *sp = (MODE == ROWS_FORCING ? p->d_fsched_ptr : p->d_osched_ptr).template as<int32_t>();
        const int32_t *si = (MODE == ROWS_FORCING ? p->d_fsched_items : p->d_osched_items).template as<int32_t>();
        const int rc = apply_rc(R, (int)sizeof(T));
        auto go = [&](auto rc_tag) {
            constexpr int RCT = decltype(rc_tag)::value;
            k_apply_tma<T, RCT, APPLY_NS, APPLY_MINB, T, MODE><<<ctas, APPLY_THREADS, apply_smem_bytes(RCT, APPLY_NS), st>>>(
                om, xm, 0, sd, sp, si, y, R, nullptr, S.err, 1.0, xa);
        };
        switch (rc) {
            case 16:
                if constexpr (sizeof(T) == 4) go(std::integral_constant<int, 16>{});
                break;
            case 8: go(std::integral_constant<int, 8>{}); break;
            case 4: go(std::integral_constant<int, 4>{}); break;
            case 2: go(std::integral_constant<int, 2>{}); break;
            default: go(std::integral_constant<int, 1>{}); break;
        }
        note_launch();
    }

    // the batched interface apply: persistent tensor-copy pipeline over the balanced schedule;
    // x is read through the workspace's tensor maps of xU
    // half: S_k from the FP16 copy (FP32 pool, use_sp = 0)
    long long wait_tries() const { return p->dbg_wait_tries > 0 ? p->dbg_wait_tries : APPLY_WAIT_TRIES; }


    template <typename T> int apply_tma(const OpPool<T> &pool, int use_sp, double *y, bool half = false) {
        // the autotuner's choice for this operator kind and R (column block, CTAs per SM), else
        // the default block and two CTAs per SM
        const ApplyChoice ch = apply_choice(p, half ? 1 : (sizeof(T) == 8 ? 2 : 0), R);
        const int rc = ch.rc > 0 ? ch.rc : apply_rc(R, (int)sizeof(T));
        const int ri = rc >= 16 ? 4 : (rc >= 8 ? 3 : (rc >= 4 ? 2 : (rc >= 2 ? 1 : 0)));
        const CUtensorMap *xm = ws.xmaps_rc[sizeof(T) == 8 ? 1 : 0][ri].template as<CUtensorMap>();
        const bool one = ch.rc > 0 && ch.per_sm == 1 && p->sched1_ctas > 0;
        const int ctas = one ? p->sched1_ctas : p->sched_ctas;
        const int32_t *sptr = (one ? p->d_sched1_ptr : p->d_sched_ptr).as<int32_t>();
        const int32_t *sitems = (one ? p->d_sched1_items : p->d_sched_items).as<int32_t>();
        if (!xm) fail(NLFETI_E_INVALID, "no tensor maps for the chosen column block");
        // one variant of the kernel: NS stages, MINB CTAs per SM in its register budget, RPW rows
        // per consumer warp, operator stored as MT
        auto launch = [&](auto ns_tag, auto minb_tag, auto rpw_tag, auto rc_tag, auto mt_tag) {
            constexpr int NS = decltype(ns_tag)::value, MINB = decltype(minb_tag)::value;
            constexpr int RPW = decltype(rpw_tag)::value, RCT = decltype(rc_tag)::value;
            using MT = typename decltype(mt_tag)::type;
            constexpr int MROW = APPLY_CB / (int)sizeof(T) * (int)sizeof(MT);
            const CUtensorMap *maps = std::is_same<MT, T>::value ? pool.maps.template as<CUtensorMap>()
                                                                 : pool.hmaps.template as<CUtensorMap>();
            k_apply_tma<T, RCT, NS, MINB, MT, ROWS_APPLY, RPW>
                <<<ctas, apply_threads(RPW), apply_smem_bytes(RCT, NS, MROW, std::is_same<T, float>::value), st>>>(
                    maps, xm, std::is_same<MT, T>::value ? use_sp : 0, sd, sptr, sitems, y, R, gate, S.err,
                    std::is_same<MT, T>::value ? 1.0 : 1.0 / pool.hscale, nullptr, wait_tries(), p->dbg_withhold,
                    yout_f);
        };
        using I1 = std::integral_constant<int, 1>;
        using I2 = std::integral_constant<int, 2>;
        using I4 = std::integral_constant<int, 4>;
        using I8 = std::integral_constant<int, 8>;
        auto go = [&](auto rc_tag) {
            constexpr int RCT = decltype(rc_tag)::value;
            if constexpr (std::is_same<T, float>::value) {
                // one CTA per SM with eight or more columns: its own instantiation (the register
                // budget of one CTA, a deeper ring)
                if constexpr (RCT >= 8) {
                  if (one) {
                    if (half) {
                        using NS1 = std::integral_constant<int, apply_ns_one(RCT, APPLY_CB / 2)>;
                        if (ch.rpw == 8) launch(NS1{}, I1{}, I8{}, rc_tag, TypeTag<__half>{});
                        else launch(NS1{}, I1{}, I4{}, rc_tag, TypeTag<__half>{});
                    } else {
                        using NS1 = std::integral_constant<int, apply_ns_one(RCT, APPLY_CB)>;
                        if (ch.rpw == 8) launch(NS1{}, I1{}, I8{}, rc_tag, TypeTag<float>{});
                        else launch(NS1{}, I1{}, I4{}, rc_tag, TypeTag<float>{});
                    }
                    return;
                  }
                }
                if (half) {
                    using NSH = std::integral_constant<int, RCT >= 16 ? APPLY_NS_H16 : APPLY_NS_H>;
                    if constexpr (RCT >= 4)
                        if (ch.rpw == 8) return launch(NSH{}, I2{}, I8{}, rc_tag, TypeTag<__half>{});
                    return launch(NSH{}, I2{}, I4{}, rc_tag, TypeTag<__half>{});
                }
                using NSF = std::integral_constant<int, APPLY_NS>;
                if constexpr (RCT >= 4)
                    if (ch.rpw == 8) return launch(NSF{}, I2{}, I8{}, rc_tag, TypeTag<float>{});
            }
            k_apply_tma<T, RCT><<<ctas, APPLY_THREADS, apply_smem_bytes(RCT, APPLY_NS, APPLY_CB, std::is_same<T, float>::value),
                                  st>>>(pool.maps.template as<CUtensorMap>(), xm, use_sp, sd, sptr, sitems, y, R, gate,
                                        S.err, 1.0, nullptr, wait_tries(), p->dbg_withhold, yout_f);
        };
        switch (rc) {
            case 16:
                if constexpr (sizeof(T) == 4) go(std::integral_constant<int, 16>{});
                break;
            case 8: go(std::integral_constant<int, 8>{}); break;
            case 4: go(std::integral_constant<int, 4>{}); break;
            case 2: go(std::integral_constant<int, 2>{}); break;
            default: go(std::integral_constant<int, 1>{}); break;
        }
        note_launch();
        return 1;
    }

    // y = S^+ x (use_sp = 1) or S x (use_sp = 0) on every subdomain.  precond: the apply is
    // the preconditioner's, which takes S_k from its FP16 copy in the mixed path (when enabled)
    template <typename T> void symv(const OpPool<T> &pool, int use_sp, const T *x, double *y, bool precond = false) {
        if (p->n_u == 0) return;
        const bool half = std::is_same<T, float>::value && precond && !use_sp && p->opt.precond_fp16 != 0 && pool.Sh.p;
        const T *base = use_sp ? pool.Sp.template as<T>() : pool.S.template as<T>();
        Slot slot{};
        const bool timed = p->prof_on;
        // inside a capture the records must become event nodes of the graph to be timed
        const unsigned rec_flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
        if (timed) {
            NLF_CUDA(cudaEventCreate(&slot.a));
            NLF_CUDA(cudaEventCreate(&slot.b));
            slot.flag = snapshot_gate();
            NLF_CUDA(cudaEventRecordWithFlags(slot.a, st, rec_flags));
        }
        int launches = 0;
        if (p->opt.batched && p->sched_ctas > 0) {
            launches = apply_tma<T>(pool, use_sp, y, half);
        } else if (half) {
            if constexpr (std::is_same<T, float>::value)
                launches = rows<T, ROWS_APPLY, __half>(pool.Sh.template as<__half>(), 0, x, nullptr, nullptr, y,
                                                       p->d_items, p->item_off, 1.0 / pool.hscale);
        } else {
            launches = rows<T, ROWS_APPLY>(base, use_sp, x, nullptr, nullptr, y, p->d_items, p->item_off);
        }
        if (timed) {
            NLF_CUDA(cudaEventRecordWithFlags(slot.b, st, rec_flags));
            double bytes = 0;
            const double me = half ? 2.0 : (double)sizeof(T);
            const double ob = yout_f ? sizeof(float) : sizeof(double);      // the output's type
            for (const auto &d : p->sd) bytes += (double)d.nG * d.ldG * me + (double)d.nG * R * (sizeof(T) + ob);
            slot.launches = launches;
            slot.bytes = bytes;
            slot.half = half;
            (capturing ? graph_slots : eager_slots).push_back(slot);
        }
    }

    // y = S x on every subdomain on the tensor cores (FP16 S_k and x in xU, x scaled per column
    // by xscale, FP32 accumulators), timed like the other preconditioner applies
    template <typename T> void symv_mma(const OpPool<T> &pool, double *y) {
        Slot slot{};
        const bool timed = p->prof_on;
        const unsigned rec_flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
        if (timed) {
            NLF_CUDA(cudaEventCreate(&slot.a));
            NLF_CUDA(cudaEventCreate(&slot.b));
            slot.flag = snapshot_gate();
            NLF_CUDA(cudaEventRecordWithFlags(slot.a, st, rec_flags));
        }
        const __half *am = pool.St.template as<__half>();
        const CUtensorMap *xm = ws.xhmaps.as<CUtensorMap>();
        const double osc = 1.0 / pool.hscale;
        const double *xs = ws.xscale.as<double>();
        auto go = [&](int ctas, const int32_t *sp, const int32_t *si) {
            if (ctas <= 0) return 0;
            switch (mma_np(R)) {
                case 16:
                    k_apply_mma<16><<<ctas, MMA_THREADS, mma_smem_bytes(16), st>>>(am, xm, sd, sp, si, y, R, gate, S.err,
                                                                                    osc, xs, yout_f);
                    break;
                case 32:
                    k_apply_mma<32><<<ctas, MMA_THREADS, mma_smem_bytes(32), st>>>(am, xm, sd, sp, si, y, R, gate, S.err,
                                                                                    osc, xs, yout_f);
                    break;
                default:
                    k_apply_mma<64><<<ctas, MMA_THREADS, mma_smem_bytes(64), st>>>(am, xm, sd, sp, si, y, R, gate, S.err,
                                                                                    osc, xs, yout_f);
                    break;
            }
            note_launch();
            return 1;
        };
        // batched: the balanced persistent schedule; else one launch per subdomain, one item per
        // CTA (every item runs the same MMA sequence either way: the same bits)
        int launches = 0;
        if (p->opt.batched) {
            launches = go(p->msched_ctas, p->d_msched_ptr.as<int32_t>(), p->d_msched_items.as<int32_t>());
        } else {
            for (int k = 0; k < p->K; ++k)
                launches += go(p->mitem_off[k + 1] - p->mitem_off[k], p->d_iota.as<int32_t>(),
                               p->d_mitems.as<int32_t>() + 2 * p->mitem_off[k]);
        }
        if (timed) {
            NLF_CUDA(cudaEventRecordWithFlags(slot.b, st, rec_flags));
            double bytes = 0;
            const double ob = yout_f ? sizeof(float) : sizeof(double);
            for (const auto &d : p->sd) bytes += (double)d.nG * d.ldG * 2.0 + (double)d.nG * R * (2.0 + ob);
            slot.launches = launches;
            slot.bytes = bytes;
            slot.half = true;
            (capturing ? graph_slots : eager_slots).push_back(slot);
        }
    }

    // x (apply layout) = B^T v, or B_D^T v with weights
    template <typename T, typename L>
    void gather_x(const int64_t *ptr, const int64_t *row, const L *val, const L *v, T *x) {
        const int64_t nu = p->n_u;
        if (R <= GX_MAXR)
            k_gather_apply_t<T, L><<<(unsigned)((nu + GX_U - 1) / GX_U), 256, sizeof(double) * GX_U * R, st>>>(
                ptr, row, val, v, x, sd, p->d_u2sub.as<int32_t>(), nu, R, gate);
        else
            k_gather_apply<T, L><<<grid_for(nu * R), 256, 0, st>>>(ptr, row, val, v, x, sd, p->d_u2sub.as<int32_t>(),
                                                                   nu, R, gate);
        note_launch();
    }

    template <typename T> void applyF(const OpPool<T> &pool, const double *v, double *out, const double *cvec = nullptr) {
        const int64_t nl = p->n_lambda, nu = p->n_u;
        T *x = apply_input<T>(ws);
        if (nu > 0) gather_x<T, double>(p->d_Bt_ptr.as<int64_t>(), p->d_Bt_row.as<int64_t>(), nullptr, v, x);
        symv<T>(pool, 1, x, ws.yU.as<double>());
        k_gather_b<<<grid_for(nl * R), 256, 0, st>>>(p->d_Bp.as<int64_t>(), p->d_Bm.as<int64_t>(), ws.yU.as<double>(),
                                                     cvec, out, nl, R);
                                                     note_launch();
    }

    // the preconditioner's S_k apply runs on the tensor cores (FP16 copy, FP16 x): mixed path
    // with precond_fp16 = 2, at most MMA_MAX_R right-hand sides
    template <typename T> bool use_mma(const OpPool<T> &pool, bool precond) const {
        const bool want = p->opt.precond_fp16 == 2 || (p->opt.precond_fp16 == 1 && apply_choice(p, 1, R).mma);
        return std::is_same<T, float>::value && precond && want && p->msched_ctas > 0 && R <= MMA_MAX_R &&
               pool.St.p && ws.xhmaps.p;
    }

    // out = M^-1 v (the scaled Dirichlet preconditioner), v and out in L
    template <typename T, typename L = double>
    void applyMinv(const OpPool<T> &pool, const L *v, L *out, bool precond = false) {
        const int64_t nl = p->n_lambda, nu = p->n_u;
        T *x = apply_input<T>(ws);
        float *const saved_out = yout_f;
        yout_f = std::is_same<L, float>::value ? ws.yU.as<float>() : nullptr;   // y_U in L
        if (use_mma(pool, precond)) {
            if (nu > 0) {
                k_gather_apply_f16<L><<<grid_for(nu * R), 256, 0, st>>>(
                    p->d_BDt_ptr.as<int64_t>(), p->d_BDt_row.as<int64_t>(), wt<L>(p->d_BDt_val, p->d_BDt_val32), v,
                    xscale_ptr<L>(), ws.xU.as<__half>(), sd, p->d_u2sub.as<int32_t>(), nu, R, gate);
                note_launch();
                symv_mma(pool, ws.yU.as<double>());
            }
        } else {
            if (nu > 0)
                gather_x<T, L>(p->d_BDt_ptr.as<int64_t>(), p->d_BDt_row.as<int64_t>(),
                               wt<L>(p->d_BDt_val, p->d_BDt_val32), v, x);
            symv<T>(pool, 0, x, ws.yU.as<double>(), precond);
        }
        yout_f = saved_out;
        k_gather_bd<L><<<grid_for(nl * R), 256, 0, st>>>(p->d_BD_ptr.as<int64_t>(), p->d_BD_col.as<int64_t>(),
                                                         wt<L>(p->d_BD_val, p->d_BD_val32), ws.yU.as<L>(), out, nl, R);
        note_launch();
    }

    // One PCG iteration, ten kernels.  The updates of p, lambda and r are stored by the next
    // iteration's k_check_update (kernels before it form p_new and r_new per row), and
    // k_check_update sets the loop condition inside a graph loop.  The Lambda vectors and their
    // arithmetic are in the operators' type T: FP64 in the FP64 pass; FP32 in the FP32 pass,
    // whose iterations only have to reduce the residual by inner_tol (the refinement's FP64
    // residual corrects what FP32 leaves).  The dot products' tile sums and the PCG scalars are
    // FP64 in both.
    template <typename T> void iteration(const OpPool<T> &pool, double tol, int max_it) {
        using L = T;
        const int64_t nl = p->n_lambda, nu = p->n_u;
        const LamVecs<L> v = lam_vecs<L>();
        L *yU = ws.yU.as<L>();          // the applies' output, in L
        T *x = apply_input<T>(ws);
        const L *alpha = p->n_co > 0 ? ws.alpha.as<L>() : nullptr;
        // p, lambda, r updated; w = P r, ||w||, stop test
        if (p->n_co > 0) coarse_alpha<L>(v.r, PG_LAM_R, v.q);
        auto check = [&](auto kern) {
            kern<<<tile_blocks(nl), TILE_THREADS, 0, st>>>(p->d_Gcol.as<int32_t>(), wt<L>(p->d_Gval, p->d_Gval32), p->gw,
                                                          alpha, v.y, v.pv, v.lam, v.r, v.q, v.w, nl, R,
                                                          ws.partial.as<double>(), S, tol, max_it, cond, max_it + 1);
        };
        if (use_cond) check(k_check_update<1, L>);
        else check(k_check_update<0, L>);
        note_launch();
        gate = S.n_active;
        applyMinv<T, L>(pool, v.w, v.z, true);                   // z = M^-1 w
        project_dot<FIN_BETA, L>(v.z, v.w, v.y);                 // y = P z, (y, w), beta
        // q = F p_new, (p_new, q), eta
        if (R <= GX_MAXR)
            k_gather_apply_p_t<T, L><<<(unsigned)((nu + GX_U - 1) / GX_U), 256, sizeof(double) * GX_U * R, st>>>(
                p->d_Bt_ptr.as<int64_t>(), p->d_Bt_row.as<int64_t>(), v.pv, v.y, beta_ptr<L>(), S.active, x, sd,
                p->d_u2sub.as<int32_t>(), nu, R, gate);
        else
            k_gather_apply_p<T, L><<<grid_for(nu * R), 256, 0, st>>>(p->d_Bt_ptr.as<int64_t>(),
                                                                     p->d_Bt_row.as<int64_t>(), v.pv, v.y,
                                                                     beta_ptr<L>(), S.active, x, sd,
                                                                     p->d_u2sub.as<int32_t>(), nu, R, gate);
        note_launch();
        yout_f = std::is_same<L, float>::value ? ws.yU.as<float>() : nullptr;
        symv<T>(pool, 1, x, ws.yU.as<double>());
        yout_f = nullptr;
        k_gather_b_eta<L><<<tile_blocks(nl), TILE_THREADS, 0, st>>>(p->d_Bp.as<int64_t>(), p->d_Bm.as<int64_t>(), yU,
                                                                  v.pv, v.y, v.q, nl, R, ws.partial.as<double>(), S);
        note_launch();
        gate = nullptr;
    }

    // The PCG loop of a pass as one graph: a WHILE node whose body is one iteration; cached
    // in the workspace and reused by every pass with the same factorization and settings.
    template <typename T> const PcgGraph &while_graph(const OpPool<T> &pool, double tol, int max_it) {
        const int prec = std::is_same<T, float>::value ? 1 : 0;
        for (const auto &g : ws.graphs)
            if (g.kind == 0 && g.factor_gen == p->factor_gen && g.precision == prec && g.tol == tol &&
                g.max_it == max_it && g.precond_fp16 == p->opt.precond_fp16 && g.wait_tries == wait_tries() &&
                g.withhold == p->dbg_withhold && g.tune_gen == p->tune_gen)
                return g;
        PcgGraph g;
        g.wait_tries = wait_tries();
        g.withhold = p->dbg_withhold;
        g.tune_gen = p->tune_gen;
        g.precond_fp16 = p->opt.precond_fp16;
        g.factor_gen = p->factor_gen;
        g.precision = prec;
        g.tol = tol;
        g.max_it = max_it;
        cudaGraph_t graph = nullptr;
        NLF_CUDA(cudaGraphCreate(&graph, 0));
        try {
            NLF_CUDA(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
            cudaGraphNodeParams np = {};
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = cond;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            cudaGraphNode_t node;
            NLF_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np));
            cudaGraph_t body = np.conditional.phGraph_out[0];
            capturing = true;
            use_cond = true;
            cap_launches = 0;
            NLF_CUDA(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
            iteration<T>(pool, tol, max_it);
            cudaGraph_t captured = nullptr;
            capturing = false;
            use_cond = false;
            NLF_CUDA(cudaStreamEndCapture(st, &captured));
            NLF_CUDA(cudaGraphInstantiate(&g.exec, graph, 0));
        } catch (...) {
            if (capturing) {
                cudaGraph_t junk = nullptr;
                cudaStreamEndCapture(st, &junk);
                capturing = false;
                use_cond = false;
            }
            cudaGetLastError();
            cudaGraphDestroy(graph);
            throw;
        }
        cudaGraphDestroy(graph);
        g.body_launches = cap_launches;
        ws.graphs.push_back(g);
        return ws.graphs.back();
    }

    // ---------------------------------------------------------------- single-domain CG
    void cg_iteration(double tol, int max_it) {
        const int64_t n = p->n_dofs_total;
        double *u = ws.cg_u.as<double>(), *r = ws.cg_r.as<double>(), *z = ws.cg_z.as<double>(),
               *pv = ws.cg_p.as<double>(), *q = ws.cg_q.as<double>();
        k_cg_spmv<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(CG_BLOCKS, (n + CG_WARPS - 1) / CG_WARPS)),
                    CG_WARPS * 32, 0, st>>>(p->d_cg_ptr.as<int64_t>(), p->d_cg_col.as<int32_t>(),
                                            p->d_cg_vhi.as<float>(), p->d_cg_vlo.as<float>(), ws.cg_ph.as<float>(),
                                            ws.cg_pl.as<float>(), pv, q, n, R, ws.cg_part.as<double>(), S);
        note_launch();
        auto upd = [&](auto kern) {
            kern<<<red_grid(n, R), RED_THREADS, 0, st>>>(p->d_cg_dinv.as<double>(), pv, q, u, r, z, n, R,
                                                         ws.partial.as<double>(), ws.partial2.as<double>(), S, tol,
                                                         max_it, cond, max_it + 1);
        };
        if (use_cond) upd(k_cg_update<1>);
        else upd(k_cg_update<0>);
        note_launch();
        k_cg_p<<<grid_for(n * R), 256, 0, st>>>(z, pv, ws.cg_ph.as<float>(), ws.cg_pl.as<float>(), n, R, S);
        note_launch();
    }

    // the CG loop: one cached WHILE graph (batched, no profiling), else chunks of 4
    // iterations with a host check (graphs when batched, plain launches otherwise)
    void cg_loop(double tol, int max_it) {
        const bool batched = p->opt.batched != 0;
        if (batched && !p->prof_on && p->opt.graph_loop) {
            const PcgGraph *found = nullptr;
            for (const auto &g : ws.graphs)
                if (g.kind == 1 && g.tol == tol && g.max_it == max_it) found = &g;
            if (!found) {
                PcgGraph g;
                g.kind = 1;
                g.tol = tol;
                g.max_it = max_it;
                cudaGraph_t graph = nullptr;
                NLF_CUDA(cudaGraphCreate(&graph, 0));
                try {
                    NLF_CUDA(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
                    cudaGraphNodeParams np = {};
                    np.type = cudaGraphNodeTypeConditional;
                    np.conditional.handle = cond;
                    np.conditional.type = cudaGraphCondTypeWhile;
                    np.conditional.size = 1;
                    cudaGraphNode_t node;
                    NLF_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np));
                    cudaGraph_t body = np.conditional.phGraph_out[0];
                    capturing = true;
                    use_cond = true;
                    cap_launches = 0;
                    NLF_CUDA(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0,
                                                           cudaStreamCaptureModeThreadLocal));
                    cg_iteration(tol, max_it);
                    cudaGraph_t captured = nullptr;
                    capturing = false;
                    use_cond = false;
                    NLF_CUDA(cudaStreamEndCapture(st, &captured));
                    NLF_CUDA(cudaGraphInstantiate(&g.exec, graph, 0));
                } catch (...) {
                    if (capturing) {
                        cudaGraph_t junk = nullptr;
                        cudaStreamEndCapture(st, &junk);
                        capturing = false;
                        use_cond = false;
                    }
                    cudaGetLastError();
                    cudaGraphDestroy(graph);
                    throw;
                }
                cudaGraphDestroy(graph);
                g.body_launches = cap_launches;
                ws.graphs.push_back(g);
                found = &ws.graphs.back();
            }
            NLF_CUDA(cudaMemsetAsync(S.loops, 0, sizeof(int), st));
            NLF_CUDA(cudaGraphLaunch(found->exec, st));
            loop_body_launches = found->body_launches;
            return;
        }
        const int chunk = 4;
        cudaGraphExec_t exec = nullptr;
        if (batched) {
            cudaGraph_t graph;
            capturing = true;
            cap_launches = 0;
            NLF_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            for (int i = 0; i < chunk; ++i) cg_iteration(tol, max_it);
            NLF_CUDA(cudaStreamEndCapture(st, &graph));
            capturing = false;
            NLF_CUDA(cudaGraphInstantiate(&exec, graph, 0));
            NLF_CUDA(cudaGraphDestroy(graph));
        }
        for (int done = 0; done <= max_it; done += chunk) {
            if (batched) {
                NLF_CUDA(cudaGraphLaunch(exec, st));
                eager_launches += cap_launches;
            } else {
                for (int i = 0; i < chunk; ++i) cg_iteration(tol, max_it);
            }
            NLF_CUDA(cudaMemcpyAsync(ws.host_flag.data(), S.n_active, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
            NLF_CUDA(cudaStreamSynchronize(st));
            check_waits();
            if (ws.host_flag[0] == 0) break;
        }
        if (exec) NLF_CUDA(cudaGraphExecDestroy(exec));
    }

    // one FETI pass on subdomain loads ws.res; constraint right-hand side ws.cvec when with_c.
    // Output: ws.du (subdomain vectors) and ws.dlam.
    template <typename T> void pass(const OpPool<T> &pool, double tol, int max_it, bool with_c) {
        const int64_t nl = p->n_lambda, nu = p->n_u;
        const double *f = ws.res.as<double>();
        const bool batched = p->opt.batched != 0;
        if (nu > 0) {
            if (batched && p->fsched_ctas > 0) rows_tma<T, ROWS_FORCING>(pool, f, nullptr, ws.fU.as<double>());
            else rows<T, ROWS_FORCING>(pool.M.template as<T>(), 0, nullptr, f, nullptr, ws.fU.as<double>(), p->d_items,
                                       p->item_off);
        }
        double *lam = ws.dlam.as<double>();
        T *x = apply_input<T>(ws);
        if (nl > 0) {
            k_to_apply<T><<<grid_for(nu * R), 256, 0, st>>>(ws.fU.as<double>(), x, sd, p->d_u2sub.as<int32_t>(), nu, R);
            note_launch();
            symv<T>(pool, 1, x, ws.yU.as<double>());
            k_gather_b<<<grid_for(nl * R), 256, 0, st>>>(p->d_Bp.as<int64_t>(), p->d_Bm.as<int64_t>(), ws.yU.as<double>(),
                                                         with_c ? ws.cvec.as<double>() : nullptr, ws.d.as<double>(), nl, R);
                                                         note_launch();
            if (p->n_co > 0) {
                coarse_alpha(ws.fU.as<double>(), PG_U);
                k_apply_galpha<<<grid_for(nl * R), 256, 0, st>>>(p->d_Gcol.as<int32_t>(), p->d_Gval.as<double>(),
                                                                 p->gw, ws.alpha.as<double>(), nullptr, 1.0, lam, nl, R);
                                                                 note_launch();
            } else {
                NLF_CUDA(cudaMemsetAsync(lam, 0, sizeof(double) * nl * R, st));
            }
            applyF<T>(pool, lam, ws.q.as<double>());
            k_sub<<<grid_for(nl * R), 256, 0, st>>>(ws.d.as<double>(), ws.q.as<double>(), ws.r.as<double>(), nl * R);
            note_launch();
            project(ws.d.as<double>(), ws.w.as<double>());
            dot_final<FIN_NPD>(ws.w.as<double>(), ws.w.as<double>(), nl);
            // p, y and q start at zero and FIN_NPD set eta = beta = 0: the updates the first
            // iteration stores are empty.  The FP32 pass iterates on FP32 copies of r and lambda.
            if constexpr (std::is_same<T, float>::value) {
                const LamVecs<float> v = lam_vecs<float>();
                k_lam_enter<<<grid_for(nl * R), 256, 0, st>>>(ws.r.as<double>(), lam, v.r, v.lam, v.pv, v.y, v.q,
                                                              nl * R);
                note_launch();
            } else {
                NLF_CUDA(cudaMemsetAsync(ws.pv.p, 0, sizeof(double) * nl * R, st));
                NLF_CUDA(cudaMemsetAsync(ws.y.p, 0, sizeof(double) * nl * R, st));
                NLF_CUDA(cudaMemsetAsync(ws.q.p, 0, sizeof(double) * nl * R, st));
            }
            const int chunk = 4;
            int done = 0, n_active = R;
            cudaGraphExec_t exec = nullptr;
            if (batched && !p->prof_on && p->opt.graph_loop) {
                // device-side loop: one launch, one read-back per pass
                const PcgGraph &g = while_graph<T>(pool, tol, max_it);
                NLF_CUDA(cudaMemsetAsync(S.loops, 0, sizeof(int), st));
                NLF_CUDA(cudaGraphLaunch(g.exec, st));
                loop_body_launches = g.body_launches;   // counted when the scalars are read back
                done = max_it + 1;                      // skip the chunked loop below
            } else if (batched) {
                // host-checked chunks of iterations (profiling: with event-timed applies, as
                // event nodes are not allowed inside a WHILE body)
                cudaGraph_t graph;
                capturing = true;
                cap_launches = 0;
                NLF_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                for (int i = 0; i < chunk; ++i) iteration<T>(pool, tol, max_it);
                NLF_CUDA(cudaStreamEndCapture(st, &graph));
                capturing = false;
                NLF_CUDA(cudaGraphInstantiate(&exec, graph, 0));
                NLF_CUDA(cudaGraphDestroy(graph));
            }
            while (done <= max_it) {
                if (batched) {
                    NLF_CUDA(cudaGraphLaunch(exec, st));
                    eager_launches += cap_launches;
                } else {
                    for (int i = 0; i < chunk; ++i) iteration<T>(pool, tol, max_it);
                }
                done += chunk;
                NLF_CUDA(cudaMemcpyAsync(ws.host_flag.data(), S.n_active, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
                NLF_CUDA(cudaStreamSynchronize(st));
                check_waits();
                harvest(graph_slots, false);
                harvest(eager_slots, true);
                n_active = ws.host_flag[0];
                if (n_active == 0) break;
            }
            if (exec) NLF_CUDA(cudaGraphExecDestroy(exec));
            drop(graph_slots);
            if constexpr (std::is_same<T, float>::value) {
                const LamVecs<float> v = lam_vecs<float>();
                k_lam_exit<<<grid_for(nl * R), 256, 0, st>>>(v.lam, v.r, lam, ws.r.as<double>(), nl * R);
                note_launch();
            }
            // alpha from the PCG residual r = d - F lambda, kept current by the recurrence
            // (eq. forAlpha); u_G = S^+ (fU - B^T lambda) - Z alpha  (eq. forU)
            k_gather_sub_apply<T><<<grid_for(nu * R), 256, 0, st>>>(p->d_Bt_ptr.as<int64_t>(), p->d_Bt_row.as<int64_t>(),
                                                                   lam, ws.fU.as<double>(), x, sd,
                                                                   p->d_u2sub.as<int32_t>(), nu, R);
            note_launch();
            symv<T>(pool, 1, x, ws.uU.as<double>());
            if (p->n_co > 0) {
                coarse_alpha(ws.r.as<double>(), PG_LAM);
                k_apply_zalpha<<<grid_for(nu * R), 256, 0, st>>>(sd, p->d_u2sub.as<int32_t>(), p->d_Z.as<double>(),
                                                                 ws.alpha.as<double>(), -1.0, ws.uU.as<double>(), nu, R);
                note_launch();
            }
        } else if (nu > 0) {
            k_to_apply<T><<<grid_for(nu * R), 256, 0, st>>>(ws.fU.as<double>(), x, sd, p->d_u2sub.as<int32_t>(), nu, R);
            note_launch();
            symv<T>(pool, 1, x, ws.uU.as<double>());
        }
        if (batched && p->osched_ctas > 0)
            rows_tma<T, ROWS_BACKSUB>(pool, f, ws.uU.as<double>(), ws.du.as<double>());
        else
            rows<T, ROWS_BACKSUB>(pool.M.template as<T>(), 0, nullptr, f, ws.uU.as<double>(), ws.du.as<double>(),
                                  p->d_items_o, p->item_off_o);
        if (nu > 0) {
            k_scatter_u<<<grid_for(nu * R), 256, 0, st>>>(p->d_u2v.as<int64_t>(), ws.uU.as<double>(), ws.du.as<double>(),
                                                          nu, R);
            note_launch();
        }
        NLF_CUDA(cudaGetLastError());
    }

    // One read-back of the scalar block (doubles nPd .. corr, then active, iters, n_active,
    // loops, counter, err) after the work of a sweep; checks the error word and counts the
    // kernels of the last device-side loop.
    struct State {
        int iterations = 0, n_active = 0;
        double relres = 0;
        bool all_within = true;
        std::vector<double> corr;
    };
    State read_state(double tol) {
        const size_t nd = 7 * (size_t)R, ni = 2 * (size_t)R + 4;
        std::vector<unsigned char> buf(nd * sizeof(double) + ni * sizeof(int));
        NLF_CUDA(cudaMemcpyAsync(buf.data(), ws.scal.p, buf.size(), cudaMemcpyDeviceToHost, st));
        NLF_CUDA(cudaStreamSynchronize(st));
        const double *d = reinterpret_cast<const double *>(buf.data());
        const int *iv = reinterpret_cast<const int *>(buf.data() + nd * sizeof(double));
        for (int k = 0; k < 4; ++k) ws.host_flag[k] = iv[2 * R + k];
        check_waits();
        eager_launches += (int64_t)iv[2 * R + 1] * loop_body_launches;
        loop_body_launches = 0;
        State out;
        out.n_active = iv[2 * R];
        out.corr.assign(d + 6 * R, d + 7 * R);
        for (int c = 0; c < R; ++c) {
            out.iterations = std::max(out.iterations, iv[R + c]);
            out.relres = std::max(out.relres, d[5 * R + c]);
            if (!(d[5 * R + c] <= tol)) out.all_within = false;
        }
        return out;
    }
};

}  // namespace

namespace {
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        NLF_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q));
        if (!f || q != cudaDriverEntryPointSuccess) fail(NLFETI_E_CUDA, "cuTensorMapEncodeTiled is not available");
        fn = reinterpret_cast<EncodeTiledFn>(f);
    }
    return fn;
}
}  // namespace

void SolveWS::drop_graphs() {
    if (graphs.empty()) return;
    // a graph may still run on the workspace's stream (a server's workspaces are idle when they
    // are dropped: their slot synchronized its stream, which another slot's thread may be
    // capturing into now, so it is not touched here)
    if (alloc_stream) {
    } else if (async_stream) {
        cudaStreamSynchronize(async_stream);
    } else if (prob) {
        cudaStreamSynchronize(prob->ctx->stream);
    }
    for (auto &g : graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    graphs.clear();
}

void SolveWS::ensure(nlfeti_problem *p, int nR) {
    nlfeti_ctx *c = p->ctx;
    if (R == nR && prob == p && prob_uid == p->uid) return;
    // buffers about to be replaced may still be read by queued work
    NLF_CUDA(cudaStreamSynchronize(async_stream ? async_stream : c->stream));
    drop_graphs();
    // marked complete only once every buffer below exists: a failed allocation leaves the
    // workspace empty, so that the next call sizes it again
    R = 0;
    prob = nullptr;
    prob_uid = 0;
    const int R = nR;
    const int64_t nl = std::max<int64_t>(1, p->n_lambda), nu = std::max<int64_t>(1, p->n_u),
                  nv = std::max<int64_t>(1, p->sum_nk), nd = std::max<int64_t>(1, p->n_dofs_total);
    const int64_t nco = std::max(1, p->n_co);
    auto alloc = [&](DevMem &m, size_t bytes) {
        if (alloc_stream) m.alloc_async(alloc_stream, bytes);
        else if (async_stream) m.alloc_async(async_stream, bytes);
        else m.alloc(c, bytes);
    };
    auto A = [&](DevMem &m, int64_t n) { alloc(m, sizeof(double) * n * R); };
    A(lam, nl); A(r, nl); A(w, nl); A(z, nl); A(y, nl); A(pv, nl); A(q, nl); A(d, nl); A(cvec, nl); A(dlam, nl);
    A(fU, nu); A(yU, nu); A(uU, nu);
    A(xU, std::max<int64_t>(1, p->n_up));   // apply layout (padding zeroed by the gathers)
    const int R2x = (R + 1) / 2 * 2;
    alloc(xP, sizeof(float) * std::max<int64_t>(1, p->n_xp) * R2x);   // paired FP32 layout, zeroed below
    alloc(uhl, sizeof(float) * 2 * std::max<int64_t>(1, p->n_vp) * ((R + 1) / 2 * 2));
    alloc(xscale, sizeof(double) * R);
    if (alloc_stream) NLF_CUDA(cudaStreamSynchronize(alloc_stream));
    {
        const std::vector<double> ones(R, 1.0);
        NLF_CUDA(cudaMemcpyAsync(xscale.p, ones.data(), sizeof(double) * R, cudaMemcpyHostToDevice,
                                 async_stream ? async_stream : c->stream));
        NLF_CUDA(cudaStreamSynchronize(async_stream ? async_stream : c->stream));
    }
    NLF_CUDA(cudaMemsetAsync(xU.p, 0, xU.bytes, async_stream ? async_stream : c->stream));
    // the paired FP32 input: its padding (columns past n_gamma of each 128-column group, the
    // partner of an odd last right-hand side) is never written again and stays zero
    NLF_CUDA(cudaMemsetAsync(xP.p, 0, xP.bytes, async_stream ? async_stream : c->stream));
    // tensor maps of xU per subdomain (R rows of ld_gamma entries at offUp * R), read as FP32
    // and as FP64, tiles of rc rows as the apply kernel of this R uses
    {
        const int rcb = apply_rc(R, 8);          // at most 8 (the FP64 pipeline and the residual)
        for (int e = 0; e < 2; ++e) {
            const int es = e ? 8 : 4;
            for (int ri = 0; ri < 5; ++ri) {
                const int rce = 1 << ri;
                xmaps_rc[e][ri].release();
                if (rce > R && rce > 1) continue;
                if (e == 1 && rce > 8) continue;
                std::vector<CUtensorMap> maps(std::max(1, p->K));
                std::memset(maps.data(), 0, sizeof(CUtensorMap) * maps.size());
                for (int k = 0; k < p->K; ++k) {
                    const SubdomainDesc &d = p->sd[k];
                    if (d.nG == 0) continue;
                    CUresult er;
                    if (e == 0) {
                        // FP32: the paired layout, R2 / 2 pair rows of ldgx(ld_gamma) 8-byte pairs,
                        // tiles of 256 pairs (one stage of columns) x max(1, rce / 2) pair rows
                        const float *b = xP.as<float>() + d.offXp * R2x;
                        er = encode_apply_map(encode_tiled(), &maps[k], b, (int)ldgx(d.ldG), R2x / 2, 8,
                                              std::max(1, rce / 2), 2 * APPLY_CB);
                    } else {
                        const unsigned char *b = xU.as<unsigned char>() + d.offUp * R * es;
                        er = encode_apply_map(encode_tiled(), &maps[k], b, d.ldG, R, es, rce);
                    }
                    if (er != CUDA_SUCCESS) fail(NLFETI_E_CUDA, "cuTensorMapEncodeTiled failed for the apply input");
                }
                alloc(xmaps_rc[e][ri], sizeof(CUtensorMap) * maps.size());
                NLF_CUDA(cudaMemcpyAsync(xmaps_rc[e][ri].p, maps.data(), sizeof(CUtensorMap) * maps.size(),
                                         cudaMemcpyHostToDevice, async_stream ? async_stream : c->stream));
                NLF_CUDA(cudaStreamSynchronize(async_stream ? async_stream : c->stream));
                if (rce == apply_rc(R, es)) {
                    alloc(xmaps[e], sizeof(CUtensorMap) * maps.size());
                    NLF_CUDA(cudaMemcpyAsync(xmaps[e].p, maps.data(), sizeof(CUtensorMap) * maps.size(),
                                             cudaMemcpyHostToDevice, async_stream ? async_stream : c->stream));
                    NLF_CUDA(cudaStreamSynchronize(async_stream ? async_stream : c->stream));
                }
            }
        }
        // the forcing / back-substitution right-hand sides (R rows of ld_M entries at offVp * R),
        // read as FP32 and as FP64, tiles of rcb rows
        alloc(rxs, sizeof(double) * std::max<int64_t>(1, p->n_vp) * R);
        for (int e = 0; e < 2; ++e) {
            const int es = e ? 8 : 4;
            const int rce = apply_rc(R, es);
            std::vector<CUtensorMap> rm(std::max(1, p->K));
            std::memset(rm.data(), 0, sizeof(CUtensorMap) * rm.size());
            for (int k = 0; k < p->K; ++k) {
                const SubdomainDesc &d = p->sd[k];
                if (d.nk == 0) continue;
                const unsigned char *b = rxs.as<unsigned char>() + d.offVp * R * es;
                if (encode_apply_map(encode_tiled(), &rm[k], b, d.ldM, R, es, rce) != CUDA_SUCCESS)
                    fail(NLFETI_E_CUDA, "cuTensorMapEncodeTiled failed for the forcing input");
            }
            alloc(rxmaps[e], sizeof(CUtensorMap) * rm.size());
            NLF_CUDA(cudaMemcpyAsync(rxmaps[e].p, rm.data(), sizeof(CUtensorMap) * rm.size(), cudaMemcpyHostToDevice,
                                     async_stream ? async_stream : c->stream));
            NLF_CUDA(cudaStreamSynchronize(async_stream ? async_stream : c->stream));
        }
        // xU read as FP16 by the tensor-core apply: tiles of 64 columns x (R rounded up to 16)
        // rows, 128-byte swizzle (rows past R arrive as zeros)
        if (R <= MMA_MAX_R) {
            std::vector<CUtensorMap> bm(std::max(1, p->K));
            std::memset(bm.data(), 0, sizeof(CUtensorMap) * bm.size());
            for (int k = 0; k < p->K; ++k) {
                const SubdomainDesc &d = p->sd[k];
                if (d.nG == 0) continue;
                const unsigned char *b = xU.as<unsigned char>() + d.offUp * R * 2;
                if (encode_mma_map(encode_tiled(), &bm[k], b, d.ldG, R, mma_np(R)) != CUDA_SUCCESS)
                    fail(NLFETI_E_CUDA, "cuTensorMapEncodeTiled failed for the FP16 apply input");
            }
            alloc(xhmaps, sizeof(CUtensorMap) * bm.size());
            NLF_CUDA(cudaMemcpyAsync(xhmaps.p, bm.data(), sizeof(CUtensorMap) * bm.size(), cudaMemcpyHostToDevice,
                                     async_stream ? async_stream : c->stream));
            NLF_CUDA(cudaStreamSynchronize(async_stream ? async_stream : c->stream));
        }
        // uh and ul (FP32, column pairs: R2 / 2 rows of 2 ld_M entries at offVp * R2 each) for the
        // refinement residual, tiles of (rc + 1) / 2 pair rows
        std::vector<CUtensorMap> um(2 * std::max(1, p->K));
        std::memset(um.data(), 0, sizeof(CUtensorMap) * um.size());
        const int R2 = (R + 1) / 2 * 2;
        const float *uh = uhl.as<float>(), *ul = uh + std::max<int64_t>(1, p->n_vp) * R2;
        for (int k = 0; k < p->K; ++k) {
            const SubdomainDesc &d = p->sd[k];
            if (d.nk == 0) continue;
            if (encode_apply_map(encode_tiled(), &um[2 * k], uh + d.offVp * R2, 2 * d.ldM, R2 / 2, 4, (rcb + 1) / 2,
                                 2 * RES_CB) != CUDA_SUCCESS ||
                encode_apply_map(encode_tiled(), &um[2 * k + 1], ul + d.offVp * R2, 2 * d.ldM, R2 / 2, 4, (rcb + 1) / 2,
                                 2 * RES_CB) != CUDA_SUCCESS)
                fail(NLFETI_E_CUDA, "cuTensorMapEncodeTiled failed for the residual input");
        }
        alloc(umaps, sizeof(CUtensorMap) * um.size());
        NLF_CUDA(cudaMemcpyAsync(umaps.p, um.data(), sizeof(CUtensorMap) * um.size(), cudaMemcpyHostToDevice,
                                 async_stream ? async_stream : c->stream));
        NLF_CUDA(cudaStreamSynchronize(async_stream ? async_stream : c->stream));
    }
    A(ftil, nv); A(res, nv); A(u, nv); A(du, nv);
    A(F, nd);
    A(gco, nco * PSPLIT); A(gsum, nco); A(alpha, nco);
    alloc(partial, sizeof(double) * std::max(RED_BLOCKS, TILE_MAX_BLOCKS) * R);
    alloc(partial2, sizeof(double) * std::max(RED_BLOCKS, TILE_MAX_BLOCKS) * R);
    alloc(scal, sizeof(double) * R * 7 + sizeof(int) * (2 * R + 8) + sizeof(float) * 3 * R + sizeof(unsigned) * R);
    alloc(lamf, sizeof(float) * 7 * nl * R);
    alloc(slot_flags, sizeof(int) * kSlotFlags);
    alloc(frozen, sizeof(int) * R);
    if (alloc_stream) NLF_CUDA(cudaStreamSynchronize(alloc_stream));
    NLF_CUDA(cudaMemsetAsync(scal.p, 0, scal.bytes, async_stream ? async_stream : c->stream));
    host_flag.assign(4, 0);
    this->R = nR;
    prob = p;
    prob_uid = p->uid;
}

void to_interleaved(const double *colmajor, double *inter, int64_t n, int R, cudaStream_t st) {
    k_transpose_cr<<<grid_for(n * R), 256, 0, st>>>(colmajor, inter, n, R, 1);
}
void to_colmajor(const double *inter, double *colmajor, int64_t n, int R, cudaStream_t st) {
    k_transpose_cr<<<grid_for(n * R), 256, 0, st>>>(inter, colmajor, n, R, 0);
}

void solve_device(nlfeti_problem *p, SolveWS &ws, cudaStream_t st, int R, int rhs_kind, const double *d_rhs,
                  const double *d_g, double *d_out, nlfeti_stats *stats) {
    ws.ensure(p, R);
    Runner run(p, ws, st);
    const int64_t ndof = p->n_dofs_total, nv = p->sum_nk, nl = p->n_lambda;
    const MeshHost &m = p->mesh;
    // loads (eq. bil1 load functional, split by zeta as eq. bilinear-multi5)
    k_load_vector<<<grid_for(ndof * R), 256, 0, st>>>(d_rhs, rhs_kind, p->d_xy.as<double>(), p->d_elems.as<int32_t>(),
                                                      m.dim, p->d_nodeinc_ptr.as<int64_t>(), p->d_nodeinc_el.as<int32_t>(),
                                                      p->nc, ndof, R, ws.F.as<double>());
    k_split_loads<<<grid_for(nv * R), 256, 0, st>>>(ws.F.as<double>(), p->d_vdofs.as<int32_t>(),
                                                    p->d_zeta_dof.as<double>(), nv, R, ws.ftil.as<double>());
    if (d_g)
        k_dirichlet<<<dim3(32, p->K), 256, 0, st>>>(p->d_AD.as<double>(), p->d_sd.as<SubdomainDesc>(),
                                                    p->d_ddofs.as<int32_t>(), p->d_doff.as<int64_t>(), d_g, ndof,
                                                    ws.ftil.as<double>(), R);
    NLF_CUDA(cudaGetLastError());
    run.eager_launches += 2 + (d_g ? 1 : 0);
    nlfeti_stats s{};
    const bool mixed = p->opt.precision == 1;
    if (!mixed) {
        if (!p->op64.ready) fail(NLFETI_E_INVALID, "FP64 operators not factored");
        NLF_CUDA(cudaMemcpyAsync(ws.res.p, ws.ftil.p, sizeof(double) * nv * R, cudaMemcpyDeviceToDevice, st));
        run.pass<double>(p->op64, p->opt.tol, p->opt.max_it, false);
        NLF_CUDA(cudaMemcpyAsync(ws.u.p, ws.du.p, sizeof(double) * nv * R, cudaMemcpyDeviceToDevice, st));
        const auto state = run.read_state(p->opt.tol);
        s.iterations = state.iterations;
        s.refine_sweeps = 1;
        s.final_rel_residual = state.relres;
        if (nl > 0 && !state.all_within) {
            k_output<<<grid_for(ndof * R), 256, 0, st>>>(ws.u.as<double>(), p->d_cp_ptr.as<int64_t>(), p->d_cp_pos.as<int64_t>(),
                                                         p->d_node_dir.as<int8_t>(), p->nc, d_g, ndof, R, d_out);
            if (stats) *stats = s;
            fail(NLFETI_E_NOT_CONVERGED, "PCG did not reach the tolerance within max_it");
        }
    } else {
        if (!p->op32.ready) fail(NLFETI_E_INVALID, "FP32 operators not factored");
        NLF_CUDA(cudaMemsetAsync(ws.u.p, 0, sizeof(double) * nv * R, st));
        if (nl > 0) NLF_CUDA(cudaMemsetAsync(ws.lam.p, 0, sizeof(double) * nl * R, st));
        bool ok = false;
        std::vector<double> prev_corr;
        // a right-hand side whose refinement has finished is frozen: its residual is zeroed
        // before the later sweeps, so their corrections of it are exact zeros and its result
        // is the one it would have alone (its sweeps depend on its own corrections only)
        std::vector<int> frozen(R, 0);
        bool any_frozen = false;
        for (int sw = 0; sw < std::max(1, p->opt.max_refine); ++sw) {
            if (sw == 0) {
                NLF_CUDA(cudaMemcpyAsync(ws.res.p, ws.ftil.p, sizeof(double) * nv * R, cudaMemcpyDeviceToDevice, st));
            } else {
                run.eager_launches += residual_ds(p, ws, st, R, nl > 0 ? ws.lam.as<double>() : nullptr);
                if (nl > 0)
                    k_constraint_residual<<<grid_for(nl * R), 256, 0, st>>>(p->d_Bp.as<int64_t>(), p->d_Bm.as<int64_t>(),
                                                                            p->d_u2v.as<int64_t>(), ws.u.as<double>(),
                                                                            ws.cvec.as<double>(), nl, R);
                run.eager_launches += (nl > 0);
                if (any_frozen) {
                    NLF_CUDA(cudaMemcpyAsync(ws.frozen.p, frozen.data(), sizeof(int) * R, cudaMemcpyHostToDevice, st));
                    k_zero_frozen<<<grid_for(nv * R), 256, 0, st>>>(ws.res.as<double>(), nv, R, ws.frozen.as<int>());
                    if (nl > 0)
                        k_zero_frozen<<<grid_for(nl * R), 256, 0, st>>>(ws.cvec.as<double>(), nl, R, ws.frozen.as<int>());
                    run.eager_launches += 1 + (nl > 0);
                }
            }
            run.pass<float>(p->op32, p->opt.inner_tol, p->opt.max_it, sw > 0);
            if (nl > 0) k_axpy<<<grid_for(nl * R), 256, 0, st>>>(ws.lam.as<double>(), ws.dlam.as<double>(), 1.0, nl * R);
            k_refine_update<<<red_grid(nv, R), RED_THREADS, 0, st>>>(ws.u.as<double>(), ws.du.as<double>(), nv, R,
                                                                     ws.partial.as<double>(), ws.partial2.as<double>(),
                                                                     run.S);
            run.eager_launches += 1 + (nl > 0);
            const auto state = run.read_state(p->opt.inner_tol);
            if (nl > 0) {
                s.iterations += state.iterations;
                s.final_rel_residual = state.relres;
            }
            s.refine_sweeps = sw + 1;
            const std::vector<double> &corr = state.corr;
            s.rel_correction = *std::max_element(corr.begin(), corr.end());
            // stop when every column's correction, or its estimated remaining error, is within
            // refine_tol: with the observed contraction rho = corr_k / corr_{k-1} < 1/2 the
            // corrections still to come sum to about corr_k rho / (1 - rho)
            bool done = true;
            for (int c = 0; c < R; ++c) {
                if (frozen[c]) continue;
                bool fin = corr[c] <= p->opt.refine_tol;
                if (!fin) {
                    const double rho = prev_corr.empty() || prev_corr[c] <= 0 ? 1.0 : corr[c] / prev_corr[c];
                    fin = rho < 0.5 && corr[c] * rho / (1.0 - rho) <= p->opt.refine_tol;
                }
                if (fin) {
                    frozen[c] = 1;
                    any_frozen = true;
                } else {
                    done = false;
                }
            }
            prev_corr = corr;
            if (done) { ok = true; break; }
        }
        if (!ok) {
            k_output<<<grid_for(ndof * R), 256, 0, st>>>(ws.u.as<double>(), p->d_cp_ptr.as<int64_t>(), p->d_cp_pos.as<int64_t>(),
                                                         p->d_node_dir.as<int8_t>(), p->nc, d_g, ndof, R, d_out);
            if (stats) *stats = s;
            fail(NLFETI_E_NOT_CONVERGED, "iterative refinement did not reach refine_tol within max_refine sweeps");
        }
    }
    k_output<<<grid_for(ndof * R), 256, 0, st>>>(ws.u.as<double>(), p->d_cp_ptr.as<int64_t>(), p->d_cp_pos.as<int64_t>(),
                                                 p->d_node_dir.as<int8_t>(), p->nc, d_g, ndof, R, d_out);
    NLF_CUDA(cudaGetLastError());
    run.eager_launches += 1;
    if (stats) *stats = s;
}

ApplyChoice apply_choice(const nlfeti_problem *p, int kind, int R) {
    auto it = p->tune.find({kind, R});
    if (it != p->tune.end()) return it->second;
    ApplyChoice c;
    c.rc = apply_rc(R, kind == 2 ? 8 : 4);
    c.per_sm = 2;
    return c;
}

int device_sms() {
    int dev = 0, sms = 0;
    NLF_CUDA(cudaGetDevice(&dev));
    NLF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return sms;
}

namespace {

// key of a tuning result: the device, the subdomain operator shapes, the kind and R
std::string tune_key(const nlfeti_problem *p, int kind, int R) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void *q, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(q);
        for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ull; }
    };
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    mix(prop.name, strnlen(prop.name, sizeof(prop.name)));
    mix(&prop.multiProcessorCount, sizeof(int));
    mix(&kind, sizeof(kind));
    mix(&R, sizeof(R));
    for (const auto &d : p->sd) {
        mix(&d.nG, sizeof(d.nG));
        mix(&d.ldG, sizeof(d.ldG));
    }
    char buf[32];
    snprintf(buf, sizeof(buf), "%016llx", (unsigned long long)h);
    return buf;
}

struct CacheLine {
    std::string key;
    int kind = 0, R = 0, rc = 0, per_sm = 0, rpw = 4;
    double us = 0;
};

// the cache: {"entries": [ one object per line ]}
std::vector<CacheLine> read_tune_cache(const char *path) {
    std::vector<CacheLine> out;
    FILE *f = path ? fopen(path, "r") : nullptr;
    if (!f) return out;
    char line[512];
    while (fgets(line, sizeof(line), f)) {
        CacheLine c;
        char key[64] = {0};
        if (sscanf(line, " {\"key\": \"%63[0-9a-f]\", \"kind\": %d, \"R\": %d, \"rc\": %d, \"ctas_per_sm\": %d, \"us\": %lf",
                   key, &c.kind, &c.R, &c.rc, &c.per_sm, &c.us) == 6) {
            c.key = key;
            const char *w = strstr(line, "\"rows_per_warp\": ");
            if (w && sscanf(w, "\"rows_per_warp\": %d", &c.rpw) != 1) c.rpw = 4;
            if (c.rpw != 4 && c.rpw != 8) c.rpw = 4;
            out.push_back(c);
        }
    }
    fclose(f);
    return out;
}

void write_tune_cache(const char *path, const std::vector<CacheLine> &v) {
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\"entries\": [\n");
    for (size_t i = 0; i < v.size(); ++i)
        fprintf(f,
                "  {\"key\": \"%s\", \"kind\": %d, \"R\": %d, \"rc\": %d, \"ctas_per_sm\": %d, \"us\": %.3f, "
                "\"rows_per_warp\": %d}%s\n",
                v[i].key.c_str(), v[i].kind, v[i].R, v[i].rc, v[i].per_sm, v[i].us, v[i].rpw,
                i + 1 < v.size() ? "," : "");
    fprintf(f, "]}\n");
    fclose(f);
    std::rename(tmp.c_str(), path);
}

}  // namespace

void autotune_applies(nlfeti_problem *p, int R, const char *cache_path, std::vector<TuneEntry> &out) {
    out.clear();
    if (p->n_u == 0 || p->sched_ctas == 0) return;
    if (!p->ws) p->ws.reset(new SolveWS());
    SolveWS &ws = *p->ws;
    cudaStream_t st = p->ctx->stream;
    ws.ensure(p, R);
    NLF_CUDA(cudaMemsetAsync(ws.xU.p, 0, ws.xU.bytes, st));
    NLF_CUDA(cudaMemsetAsync(ws.xP.p, 0, ws.xP.bytes, st));
    std::vector<CacheLine> cache = read_tune_cache(cache_path);
    const int saved_batched = p->opt.batched, saved_fp16 = p->opt.precond_fp16;
    p->opt.batched = 1;
    bool changed = false;
    cudaEvent_t ea = nullptr, eb = nullptr;
    NLF_CUDA(cudaEventCreate(&ea));
    NLF_CUDA(cudaEventCreate(&eb));
    try {
        Runner run(p, ws, st);
        for (int kind = 0; kind < 3; ++kind) {
            if (kind < 2 && !p->op32.ready) continue;
            if (kind == 1 && !p->op32.Sh.p) continue;
            if (kind == 2 && !p->op64.ready) continue;
            TuneEntry te;
            te.kind = kind;
            te.R = R;
            const std::string key = tune_key(p, kind, R);
            for (const auto &c : cache)
                if (c.key == key && c.kind == kind && c.R == R) {
                    te.rc = c.rc;
                    te.per_sm = c.per_sm;
                    te.rpw = c.rpw;
                    te.us = c.us;
                    te.from_cache = true;
                }
            if (!te.from_cache) {
                p->opt.precond_fp16 = kind == 1 ? 1 : saved_fp16;
                double best = 1e30;
                for (int rc = 1; rc <= 16; rc *= 2) {
                    if (rc > R && rc > 1) break;
                    if (kind == 2 && rc > 8) break;
                    for (int per_sm = 1; per_sm <= 2; ++per_sm)
                    for (int rpw = 4; rpw <= 8; rpw += 4) {
                        // eight rows per warp: the FP32 and FP16 operators, four or more columns
                        if (rpw == 8 && (kind == 2 || rc < 4)) continue;
                        p->tune[{kind, R}] = ApplyChoice{rc, per_sm, 0, rpw};
                        auto launch = [&] {
                            if (kind == 0) run.symv<float>(p->op32, 1, ws.xP.as<float>(), ws.yU.as<double>());
                            else if (kind == 1) run.symv<float>(p->op32, 0, ws.xP.as<float>(), ws.yU.as<double>(), true);
                            else run.symv<double>(p->op64, 1, ws.xU.as<double>(), ws.yU.as<double>());
                        };
                        launch();
                        NLF_CUDA(cudaEventRecord(ea, st));
                        for (int r = 0; r < 3; ++r) launch();
                        NLF_CUDA(cudaEventRecord(eb, st));
                        NLF_CUDA(cudaEventSynchronize(eb));
                        float ms = 0.f;
                        NLF_CUDA(cudaEventElapsedTime(&ms, ea, eb));
                        const double us = 1e3 * ms / 3.0;
                        if (us < best) {
                            best = us;
                            te.rc = rc;
                            te.per_sm = per_sm;
                            te.rpw = rpw;
                            te.us = us;
                        }
                    }
                }
                // the preconditioner's copy of S_k also on the tensor cores (FP16 x scaled per column)
                if (kind == 1 && R <= MMA_MAX_R && p->msched_ctas > 0) {
                    build_tiled_half(p);
                    if (p->op32.St.p && ws.xhmaps.p) {
                        auto launch = [&] { run.symv_mma<float>(p->op32, ws.yU.as<double>()); };
                        launch();
                        NLF_CUDA(cudaEventRecord(ea, st));
                        for (int r = 0; r < 3; ++r) launch();
                        NLF_CUDA(cudaEventRecord(eb, st));
                        NLF_CUDA(cudaEventSynchronize(eb));
                        float ms = 0.f;
                        NLF_CUDA(cudaEventElapsedTime(&ms, ea, eb));
                        const double us = 1e3 * ms / 3.0;
                        if (us < best) {
                            best = us;
                            te.rc = -1;
                            te.per_sm = 1;
                            te.rpw = 4;
                            te.us = us;
                        }
                    }
                }
                run.check_waits_now();
                CacheLine c;
                c.key = key;
                c.kind = kind;
                c.R = R;
                c.rc = te.rc;
                c.per_sm = te.per_sm;
                c.rpw = te.rpw;
                c.us = te.us;
                cache.push_back(c);
                changed = true;
            }
            if (te.rc == -1) {
                build_tiled_half(p);
                p->tune[{kind, R}] = ApplyChoice{apply_rc(R, 4), 2, 1};
            } else {
                p->tune[{kind, R}] = ApplyChoice{te.rc, te.per_sm, 0, te.rpw};
            }
            out.push_back(te);
        }
    } catch (...) {
        p->opt.batched = saved_batched;
        p->opt.precond_fp16 = saved_fp16;
        ++p->tune_gen;
        cudaEventDestroy(ea);
        cudaEventDestroy(eb);
        throw;
    }
    p->opt.batched = saved_batched;
    p->opt.precond_fp16 = saved_fp16;
    ++p->tune_gen;
    cudaEventDestroy(ea);
    cudaEventDestroy(eb);
    if (changed && cache_path) write_tune_cache(cache_path, cache);
}

void apply_operator(nlfeti_problem *p, SolveWS &ws, cudaStream_t st, int op, int precision, int R, const double *in,
                    double *out) {
    ws.ensure(p, R);
    Runner run(p, ws, st);
    const int64_t nl = p->n_lambda, nu = p->n_u;
    auto go = [&](auto &pool, auto tag) {
        using T = decltype(tag);
        if (!pool.ready) fail(NLFETI_E_INVALID, "operators of the requested precision are not factored");
        switch (op) {
            case 0: run.applyF<T>(pool, in, out); break;
            case 1: run.applyMinv<T>(pool, in, out); break;
            case 2: run.project(in, out); break;
            case 3:
            case 4: {
                T *x = apply_input<T>(ws);
                k_to_apply<T><<<grid_for(nu * R), 256, 0, st>>>(in, x, run.sd, p->d_u2sub.as<int32_t>(), nu, R);
                run.symv<T>(pool, op == 3 ? 1 : 0, x, out);
                break;
            }
            case 5: {    // S through the preconditioner's copy (the path precond_fp16 selects)
                if (nu == 0) break;
                if (run.use_mma(pool, true)) {
                    k_col_scale<<<R, 256, 0, st>>>(in, nu, R, ws.xscale.as<double>());
                    k_to_apply_f16<<<grid_for(nu * R), 256, 0, st>>>(in, ws.xscale.as<double>(), ws.xU.as<__half>(),
                                                                     run.sd, p->d_u2sub.as<int32_t>(), nu, R);
                    run.symv_mma(pool, out);
                } else {
                    T *x = apply_input<T>(ws);
                    k_to_apply<T><<<grid_for(nu * R), 256, 0, st>>>(in, x, run.sd, p->d_u2sub.as<int32_t>(), nu, R);
                    run.symv<T>(pool, 0, x, out, true);
                }
                break;
            }
            default: fail(NLFETI_E_INVALID, "unknown operator");
        }
    };
    (void)nl;
    if (precision == 0) go(p->op64, double{});
    else go(p->op32, float{});
    NLF_CUDA(cudaGetLastError());
    NLF_CUDA(cudaMemcpyAsync(ws.host_flag.data(), run.S.n_active, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    NLF_CUDA(cudaStreamSynchronize(st));
    run.check_waits();
}

void cg_solve_device(nlfeti_problem *p, SolveWS &ws, cudaStream_t st, int R, int rhs_kind, const double *d_rhs,
                     const double *d_g, double *d_out, nlfeti_stats *stats) {
    if (R > CG_MAX_R) fail(NLFETI_E_INVALID, "the CG solve takes at most 32 right-hand sides per call");
    cg_prepare(p);
    ws.ensure(p, R);
    const int64_t n = p->n_dofs_total, nv = p->sum_nk;
    auto need = [&](DevMem &m, size_t bytes) {
        if (m.bytes >= bytes) return;
        if (ws.alloc_stream) {
            m.alloc_async(ws.alloc_stream, bytes);
            NLF_CUDA(cudaStreamSynchronize(ws.alloc_stream));
        } else if (ws.async_stream) {
            m.alloc_async(ws.async_stream, bytes);
        } else {
            m.alloc(p->ctx, bytes);
        }
    };
    const size_t vb = sizeof(double) * (size_t)std::max<int64_t>(1, n) * R;
    need(ws.cg_u, vb); need(ws.cg_r, vb); need(ws.cg_z, vb); need(ws.cg_p, vb); need(ws.cg_q, vb); need(ws.cg_b, vb);
    need(ws.cg_part, sizeof(double) * CG_BLOCKS * (size_t)R);
    need(ws.cg_ph, vb / 2);
    need(ws.cg_pl, vb / 2);
    Runner run(p, ws, st);
    const MeshHost &m = p->mesh;
    // loads, split per subdomain as for FETI (eq. bilinear-multi5), with the Dirichlet coupling
    k_load_vector<<<grid_for(n * R), 256, 0, st>>>(d_rhs, rhs_kind, p->d_xy.as<double>(), p->d_elems.as<int32_t>(),
                                                   m.dim, p->d_nodeinc_ptr.as<int64_t>(), p->d_nodeinc_el.as<int32_t>(),
                                                   p->nc, n, R, ws.F.as<double>());
    k_split_loads<<<grid_for(nv * R), 256, 0, st>>>(ws.F.as<double>(), p->d_vdofs.as<int32_t>(),
                                                    p->d_zeta_dof.as<double>(), nv, R, ws.ftil.as<double>());
    if (d_g)
        k_dirichlet<<<dim3(32, p->K), 256, 0, st>>>(p->d_AD.as<double>(), p->d_sd.as<SubdomainDesc>(),
                                                    p->d_ddofs.as<int32_t>(), p->d_doff.as<int64_t>(), d_g, n,
                                                    ws.ftil.as<double>(), R);
    k_cg_rhs<<<grid_for(n * R), 256, 0, st>>>(ws.ftil.as<double>(), p->d_cp_ptr.as<int64_t>(),
                                              p->d_cp_pos.as<int64_t>(), n, R, ws.cg_b.as<double>());
    k_cg_init<<<red_grid(n, R), RED_THREADS, 0, st>>>(ws.cg_b.as<double>(), p->d_cg_dinv.as<double>(),
                                                      ws.cg_u.as<double>(), ws.cg_r.as<double>(),
                                                      ws.cg_z.as<double>(), ws.cg_p.as<double>(), ws.cg_ph.as<float>(),
                                                      ws.cg_pl.as<float>(), n, R, ws.partial.as<double>(),
                                                      ws.partial2.as<double>(), run.S);
    NLF_CUDA(cudaGetLastError());
    run.eager_launches += 4 + (d_g ? 1 : 0);
    run.cg_loop(p->opt.tol, p->opt.max_it);
    const auto state = run.read_state(p->opt.tol);
    k_cg_output<<<grid_for(n * R), 256, 0, st>>>(ws.cg_u.as<double>(), p->d_node_dir.as<int8_t>(), p->nc, d_g, n, R,
                                                 d_out);
    NLF_CUDA(cudaGetLastError());
    run.eager_launches += 1;
    nlfeti_stats s{};
    s.iterations = state.iterations;
    s.final_rel_residual = state.relres;
    if (stats) *stats = s;
    if (!state.all_within) fail(NLFETI_E_NOT_CONVERGED, "CG did not reach the tolerance within max_it");
}

int apply_tma_ctas() {
    int dev = 0, sms = 0;
    NLF_CUDA(cudaGetDevice(&dev));
    NLF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int per_sm = 1 << 20;
    auto fit = [&](auto kern, int rc, bool paired = false) {
        const int smem = apply_smem_bytes(rc, APPLY_NS, APPLY_CB, paired);
        NLF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        int b = 0;
        NLF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, APPLY_THREADS, smem));
        per_sm = std::min(per_sm, b);
    };
    fit(k_apply_tma<float, 1>, 1, true); fit(k_apply_tma<float, 2>, 2, true); fit(k_apply_tma<float, 4>, 4, true);
    fit(k_apply_tma<float, 8>, 8, true); fit(k_apply_tma<float, 16>, 16, true);
    fit(k_apply_tma<double, 1>, 1); fit(k_apply_tma<double, 2>, 2);
    fit(k_apply_tma<double, 4>, 4); fit(k_apply_tma<double, 8>, 8);
    // the forcing and back-substitution modes (same pipeline and shared memory)
    fit(k_apply_tma<float, 1, APPLY_NS, APPLY_MINB, float, ROWS_FORCING>, 1);
    fit(k_apply_tma<float, 2, APPLY_NS, APPLY_MINB, float, ROWS_FORCING>, 2);
    fit(k_apply_tma<float, 4, APPLY_NS, APPLY_MINB, float, ROWS_FORCING>, 4);
    fit(k_apply_tma<float, 8, APPLY_NS, APPLY_MINB, float, ROWS_FORCING>, 8);
    fit(k_apply_tma<float, 16, APPLY_NS, APPLY_MINB, float, ROWS_FORCING>, 16);
    fit(k_apply_tma<float, 1, APPLY_NS, APPLY_MINB, float, ROWS_BACKSUB>, 1);
    fit(k_apply_tma<float, 2, APPLY_NS, APPLY_MINB, float, ROWS_BACKSUB>, 2);
    fit(k_apply_tma<float, 4, APPLY_NS, APPLY_MINB, float, ROWS_BACKSUB>, 4);
    fit(k_apply_tma<float, 8, APPLY_NS, APPLY_MINB, float, ROWS_BACKSUB>, 8);
    fit(k_apply_tma<float, 16, APPLY_NS, APPLY_MINB, float, ROWS_BACKSUB>, 16);
    fit(k_apply_tma<double, 1, APPLY_NS, APPLY_MINB, double, ROWS_FORCING>, 1);
    fit(k_apply_tma<double, 2, APPLY_NS, APPLY_MINB, double, ROWS_FORCING>, 2);
    fit(k_apply_tma<double, 4, APPLY_NS, APPLY_MINB, double, ROWS_FORCING>, 4);
    fit(k_apply_tma<double, 8, APPLY_NS, APPLY_MINB, double, ROWS_FORCING>, 8);
    fit(k_apply_tma<double, 1, APPLY_NS, APPLY_MINB, double, ROWS_BACKSUB>, 1);
    fit(k_apply_tma<double, 2, APPLY_NS, APPLY_MINB, double, ROWS_BACKSUB>, 2);
    fit(k_apply_tma<double, 4, APPLY_NS, APPLY_MINB, double, ROWS_BACKSUB>, 4);
    fit(k_apply_tma<double, 8, APPLY_NS, APPLY_MINB, double, ROWS_BACKSUB>, 8);
    auto fit_h = [&](auto kern, int rc) {
        const int smem = apply_smem_bytes(rc, APPLY_NS_H, APPLY_CB / 2, true);
        NLF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        int b = 0;
        NLF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, APPLY_THREADS, smem));
        per_sm = std::min(per_sm, b);
    };
    fit_h(k_apply_tma<float, 1, APPLY_NS_H, APPLY_MINB, __half>, 1); fit_h(k_apply_tma<float, 2, APPLY_NS_H, APPLY_MINB, __half>, 2);
    fit_h(k_apply_tma<float, 4, APPLY_NS_H, APPLY_MINB, __half>, 4); fit_h(k_apply_tma<float, 8, APPLY_NS_H, APPLY_MINB, __half>, 8);
    {
        const int smem = apply_smem_bytes(16, APPLY_NS_H16, APPLY_CB / 2);
        auto kern = k_apply_tma<float, 16, APPLY_NS_H16, APPLY_MINB, __half>;
        NLF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        int b = 0;
        NLF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, APPLY_THREADS, smem));
        per_sm = std::min(per_sm, b);
    }
    // eight rows per consumer warp (four consumer warps)
    auto fit8 = [&](auto kern, int smem) {
        NLF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        int b = 0;
        NLF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, apply_threads(8), smem));
        per_sm = std::min(per_sm, b);
    };
    fit8(k_apply_tma<float, 4, APPLY_NS, APPLY_MINB, float, ROWS_APPLY, 8>, apply_smem_bytes(4, APPLY_NS));
    fit8(k_apply_tma<float, 8, APPLY_NS, APPLY_MINB, float, ROWS_APPLY, 8>, apply_smem_bytes(8, APPLY_NS));
    fit8(k_apply_tma<float, 16, APPLY_NS, APPLY_MINB, float, ROWS_APPLY, 8>, apply_smem_bytes(16, APPLY_NS));
    fit8(k_apply_tma<float, 4, APPLY_NS_H, APPLY_MINB, __half, ROWS_APPLY, 8>,
         apply_smem_bytes(4, APPLY_NS_H, APPLY_CB / 2));
    fit8(k_apply_tma<float, 8, APPLY_NS_H, APPLY_MINB, __half, ROWS_APPLY, 8>,
         apply_smem_bytes(8, APPLY_NS_H, APPLY_CB / 2));
    fit8(k_apply_tma<float, 16, APPLY_NS_H16, APPLY_MINB, __half, ROWS_APPLY, 8>,
         apply_smem_bytes(16, APPLY_NS_H16, APPLY_CB / 2));
    if (per_sm < 1) fail(NLFETI_E_CUDA, "the interface apply does not fit on an SM");
    // the one-CTA-per-SM variants (schedules of one CTA per SM): their attributes only
    int one = 1 << 20;
    auto fit1 = [&](auto kern, int rpw, int smem) {
        NLF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        int b = 0;
        NLF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, apply_threads(rpw), smem));
        one = std::min(one, b);
    };
    constexpr int F8 = apply_ns_one(8, APPLY_CB), F16 = apply_ns_one(16, APPLY_CB);
    constexpr int H8 = apply_ns_one(8, APPLY_CB / 2), H16 = apply_ns_one(16, APPLY_CB / 2);
    fit1(k_apply_tma<float, 8, F8, 1, float, ROWS_APPLY, 4>, 4, apply_smem_bytes(8, F8));
    fit1(k_apply_tma<float, 16, F16, 1, float, ROWS_APPLY, 4>, 4, apply_smem_bytes(16, F16));
    fit1(k_apply_tma<float, 8, F8, 1, float, ROWS_APPLY, 8>, 8, apply_smem_bytes(8, F8));
    fit1(k_apply_tma<float, 16, F16, 1, float, ROWS_APPLY, 8>, 8, apply_smem_bytes(16, F16));
    fit1(k_apply_tma<float, 8, H8, 1, __half, ROWS_APPLY, 4>, 4, apply_smem_bytes(8, H8, APPLY_CB / 2));
    fit1(k_apply_tma<float, 16, H16, 1, __half, ROWS_APPLY, 4>, 4, apply_smem_bytes(16, H16, APPLY_CB / 2));
    fit1(k_apply_tma<float, 8, H8, 1, __half, ROWS_APPLY, 8>, 8, apply_smem_bytes(8, H8, APPLY_CB / 2));
    fit1(k_apply_tma<float, 16, H16, 1, __half, ROWS_APPLY, 8>, 8, apply_smem_bytes(16, H16, APPLY_CB / 2));
    if (one < 1) fail(NLFETI_E_CUDA, "the one-CTA-per-SM interface apply does not fit on an SM");
    return sms * per_sm;
}

int apply_mma_ctas() {
    int dev = 0, sms = 0;
    NLF_CUDA(cudaGetDevice(&dev));
    NLF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int per_sm = 1 << 20;
    auto fit = [&](auto kern, int np) {
        const int smem = mma_smem_bytes(np);
        NLF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        int b = 0;
        NLF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, MMA_THREADS, smem));
        per_sm = std::min(per_sm, b);
    };
    fit(k_apply_mma<16>, 16); fit(k_apply_mma<32>, 32); fit(k_apply_mma<64>, 64);
    if (per_sm < 1) fail(NLFETI_E_CUDA, "the tensor-core apply does not fit on an SM");
    return sms * per_sm;
}

int residual_tma_ctas() {
    int dev = 0, sms = 0;
    NLF_CUDA(cudaGetDevice(&dev));
    NLF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int per_sm = 1 << 20;
    auto fit = [&](auto kern, int rc) {
        const int smem = res_smem_bytes(rc);
        NLF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        int b = 0;
        NLF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, RES_THREADS, smem));
        per_sm = std::min(per_sm, b);
    };
    fit(k_residual_tma<1>, 1); fit(k_residual_tma<2>, 2); fit(k_residual_tma<4>, 4); fit(k_residual_tma<8>, 8);
    if (per_sm < 1) fail(NLFETI_E_CUDA, "the refinement residual does not fit on an SM");
    return sms * per_sm;
}


template <typename T> void encode_apply_maps(nlfeti_problem *p, OpPool<T> &pool) {
    std::vector<CUtensorMap> maps(2 * std::max(1, p->K));
    std::memset(maps.data(), 0, sizeof(CUtensorMap) * maps.size());
    for (int k = 0; k < p->K; ++k) {
        const SubdomainDesc &d = p->sd[k];
        if (d.nG == 0) continue;                      // no work items
        for (int sp = 0; sp < 2; ++sp) {
            const T *m = (sp ? pool.Sp.template as<T>() + d.offSp : pool.S.template as<T>() + d.offS);
            const CUresult r = encode_apply_map(encode_tiled(), &maps[2 * k + sp], m, d.ldG, d.nG, (int)sizeof(T));
            if (r != CUDA_SUCCESS) fail(NLFETI_E_CUDA, "cuTensorMapEncodeTiled failed for an interface operator");
        }
    }
    pool.maps.alloc(p->ctx, sizeof(CUtensorMap) * maps.size());
    NLF_CUDA(cudaMemcpyAsync(pool.maps.p, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice,
                             p->ctx->stream));

    // swept-matrix blocks of the forcing (rows n_O.., columns ..n_O) and of the back
    // substitution (rows ..n_O, all columns)
    std::vector<CUtensorMap> fm(std::max(1, p->K)), om(std::max(1, p->K));
    std::memset(fm.data(), 0, sizeof(CUtensorMap) * fm.size());
    std::memset(om.data(), 0, sizeof(CUtensorMap) * om.size());
    for (int k = 0; k < p->K; ++k) {
        const SubdomainDesc &d = p->sd[k];
        if (d.nO == 0) continue;                      // nothing to stream
        const T *m = pool.M.template as<T>() + d.offM;
        if ((d.nG > 0 && encode_block_map(encode_tiled(), &fm[k], m + (int64_t)d.nO * d.ldM, d.nO, d.nG, d.ldM,
                                          (int)sizeof(T)) != CUDA_SUCCESS) ||
            encode_block_map(encode_tiled(), &om[k], m, d.nk, d.nO, d.ldM, (int)sizeof(T)) != CUDA_SUCCESS)
            fail(NLFETI_E_CUDA, "cuTensorMapEncodeTiled failed for a swept-matrix block");
    }
    pool.fmaps.alloc(p->ctx, sizeof(CUtensorMap) * fm.size());
    pool.omaps.alloc(p->ctx, sizeof(CUtensorMap) * om.size());
    NLF_CUDA(cudaMemcpyAsync(pool.fmaps.p, fm.data(), sizeof(CUtensorMap) * fm.size(), cudaMemcpyHostToDevice,
                             p->ctx->stream));
    NLF_CUDA(cudaMemcpyAsync(pool.omaps.p, om.data(), sizeof(CUtensorMap) * om.size(), cudaMemcpyHostToDevice,
                             p->ctx->stream));
    if constexpr (std::is_same<T, float>::value) {
        // A^k as FP32 pairs (n_k rows of ld_M) for the refinement residual
        std::vector<CUtensorMap> am(2 * std::max(1, p->K));
        std::memset(am.data(), 0, sizeof(CUtensorMap) * am.size());
        for (int k = 0; k < p->K && !pool.a_sparse; ++k) {
            const SubdomainDesc &d = p->sd[k];
            if (d.nk == 0) continue;
            if (encode_apply_map(encode_tiled(), &am[2 * k], pool.Ahi.template as<float>() + d.offM, d.ldM, d.nk, 4, 32,
                                 RES_CB) != CUDA_SUCCESS ||
                encode_apply_map(encode_tiled(), &am[2 * k + 1], pool.Alo.template as<float>() + d.offM, d.ldM, d.nk, 4, 32,
                                 RES_CB) != CUDA_SUCCESS)
                fail(NLFETI_E_CUDA, "cuTensorMapEncodeTiled failed for the residual operator");
        }
        pool.amaps.alloc(p->ctx, sizeof(CUtensorMap) * am.size());
        NLF_CUDA(cudaMemcpyAsync(pool.amaps.p, am.data(), sizeof(CUtensorMap) * am.size(), cudaMemcpyHostToDevice,
                                 p->ctx->stream));
        // the FP16 copy of S_k: tiles of 32 rows x 256 entries (512 bytes), the columns of a
        // stage of the FP32 x tiles
        std::vector<CUtensorMap> hm(2 * std::max(1, p->K));
        std::memset(hm.data(), 0, sizeof(CUtensorMap) * hm.size());
        for (int k = 0; k < p->K; ++k) {
            const SubdomainDesc &d = p->sd[k];
            if (d.nG == 0) continue;
            if (encode_apply_map(encode_tiled(), &hm[2 * k], pool.Sh.template as<__half>() + d.offS, d.ldG, d.nG, 2, 32,
                                 APPLY_CB / 2) != CUDA_SUCCESS)
                fail(NLFETI_E_CUDA, "cuTensorMapEncodeTiled failed for the FP16 preconditioner operator");
        }
        pool.hmaps.alloc(p->ctx, sizeof(CUtensorMap) * hm.size());
        NLF_CUDA(cudaMemcpyAsync(pool.hmaps.p, hm.data(), sizeof(CUtensorMap) * hm.size(), cudaMemcpyHostToDevice,
                                 p->ctx->stream));

    }
    NLF_CUDA(cudaStreamSynchronize(p->ctx->stream));
}
template void encode_apply_maps<float>(nlfeti_problem *, OpPool<float> &);
template void encode_apply_maps<double>(nlfeti_problem *, OpPool<double> &);

}  // namespace nlf
