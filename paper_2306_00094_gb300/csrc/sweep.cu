// Subdomain operators by blocked symmetric sweeps, batched over all subdomains.
//
// The sweep operator on a pivot block J of a symmetric matrix M replaces
//   M_JJ -> -M_JJ^-1,  M_iJ -> M_iJ M_JJ^-1,  M_Jl -> M_JJ^-1 M_Jl,  M_il -> M_il - M_iJ M_JJ^-1 M_Jl.
// Sweeping every Omega_k pivot block of the subdomain matrix A^k (Omega-first order)
// yields in one pass (the block Cholesky identity eq. splittingBlockCholesky):
//   [ -A_OO^-1            A_OO^-1 A_OG ]
//   [ A_GO A_OO^-1        S_k          ]   with S_k = A_GG - A_GO A_OO^-1 A_OG (eq. subSchurComplement).
// A copy of S_k with the pinned dofs of a floating subdomain replaced by unit rows and
// columns (Sec. 5.3) is swept over all its pivots to give -S~_k^-1; zeroing the pinned
// rows/columns and projecting onto range(S_k) = ker(Z_k^T) gives the Moore-Penrose
// pseudo-inverse S_k^+ (eq. forU), stored explicitly.  Every FETI iteration then needs
// only dense symmetric products with S_k^+ and S_k.
//
// Pivot blocks are NB = 64 wide; a step is three launches over all subdomains: invert
// the pivot block (one CTA per subdomain, in shared memory), form the pivot panels,
// update all tiles (64x64 CTA tiles, 4x4 register blocking; for the FP32 operators per the
// factor_tc option 128x128 tiles on the tensor cores, split-TF32, in sweep_tc.cuh: by default
// in the Omega sweep of A^k, the sweep of the pinned S_k staying on the FP32 pipes).  A non-positive pivot
// sets the device status word (NLFETI_E_NOT_SPD) instead of trapping.
#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstring>

#include <cuda_fp16.h>

#include "internal.hpp"

namespace nlf {
namespace {

constexpr int NB = 64;
constexpr int TILE = 64;

template <typename T> struct SweepArgs {
    T *M;               // pool base
    T *pan;             // per subdomain: n x NB (M_iJ D^-1)
    T *old;             // per subdomain: n x NB (M_iJ before the step)
    T *dinv;            // per subdomain: NB x NB
    const SubdomainDesc *sd;
    const int64_t *moff;      // per subdomain: matrix offset in the pool
    const int32_t *mdim;      // per subdomain: matrix order
    const int32_t *mld;       // per subdomain: leading dimension
    const int32_t *pend;      // per subdomain: pivots [0, pend) are swept in this phase
    const int64_t *scr_off;   // per subdomain: scratch offset (rows)
    int j0;                   // first pivot of this step
    int *flag;
};

// sweep a small symmetric block (n <= 128) held in shared memory, row stride ld
template <typename T>
__device__ bool sweep_block_shared(T *S, int n, int ld, T *rowp) {
    bool ok = true;
    for (int p = 0; p < n; ++p) {
        __syncthreads();
        T d = S[p * ld + p];
        for (int i = threadIdx.x; i < n; i += blockDim.x) rowp[i] = S[p * ld + i];
        __syncthreads();
        if (!(d > T(0))) ok = false;
        T inv = T(1) / d;
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            int i = t / n, l = t % n;
            T v;
            if (i == p && l == p) v = -inv;
            else if (i == p) v = rowp[l] * inv;
            else if (l == p) v = rowp[i] * inv;
            else v = S[i * ld + l] - rowp[i] * rowp[l] * inv;
            S[i * ld + l] = v;
        }
    }
    __syncthreads();
    return ok;
}

template <typename T> __global__ void k_pivot(SweepArgs<T> a) {
    const int k = blockIdx.x;
    const int pend = a.pend[k];
    if (a.j0 >= pend) return;
    const int b = min(NB, pend - a.j0);
    const int ld = a.mld[k];
    T *M = a.M + a.moff[k];
    __shared__ T S[NB * NB];
    __shared__ T rowp[NB];
    for (int t = threadIdx.x; t < b * b; t += blockDim.x) {
        int i = t / b, l = t % b;
        S[i * NB + l] = M[(int64_t)(a.j0 + i) * ld + a.j0 + l];
    }
    bool ok = sweep_block_shared(S, b, NB, rowp);
    if (!ok && threadIdx.x == 0) atomicMax(a.flag, 1);
    T *D = a.dinv + (int64_t)k * NB * NB;
    for (int t = threadIdx.x; t < b * b; t += blockDim.x) {
        int i = t / b, l = t % b;
        D[i * NB + l] = -S[i * NB + l];       // D^-1
    }
}

// panels: old_i = M_iJ, pan_i = M_iJ D^-1 for every row i
template <typename T> __global__ void k_panel(SweepArgs<T> a) {
    const int k = blockIdx.y;
    const int pend = a.pend[k];
    if (a.j0 >= pend) return;
    const int b = min(NB, pend - a.j0);
    const int n = a.mdim[k];
    const int ld = a.mld[k];
    const int i = blockIdx.x * (blockDim.x / NB) + threadIdx.x / NB;
    const int t = threadIdx.x % NB;
    if (i >= n) return;
    const T *M = a.M + a.moff[k];
    const T *D = a.dinv + (int64_t)k * NB * NB;
    T *old = a.old + a.scr_off[k] * NB;
    T *pan = a.pan + a.scr_off[k] * NB;
    if (t < b) {
        T acc = 0;
        for (int s = 0; s < b; ++s) acc += M[(int64_t)i * ld + a.j0 + s] * D[s * NB + t];
        old[(int64_t)i * NB + t] = M[(int64_t)i * ld + a.j0 + t];
        pan[(int64_t)i * NB + t] = acc;
    }
}

// tile update of every entry (i, l)
template <typename T> __global__ void __launch_bounds__(256) k_update(SweepArgs<T> a) {
    const int k = blockIdx.z;
    const int pend = a.pend[k];
    if (a.j0 >= pend) return;
    const int n = a.mdim[k];
    const int ld = a.mld[k];
    const int nt = (n + TILE - 1) / TILE;
    const int ti = blockIdx.y, tl = blockIdx.x;
    if (ti >= nt || tl >= nt) return;
    const int b = min(NB, pend - a.j0);
    const int j0 = a.j0, j1 = a.j0 + b;
    T *M = a.M + a.moff[k];
    const T *old = a.old + a.scr_off[k] * NB;
    const T *pan = a.pan + a.scr_off[k] * NB;
    const T *D = a.dinv + (int64_t)k * NB * NB;
    extern __shared__ unsigned char smraw[];
    T *Ps = reinterpret_cast<T *>(smraw);            // [NB][TILE] : pan rows of tile i, transposed
    T *Os = Ps + NB * TILE;                            // [NB][TILE] : old rows of tile l, transposed
    const int r0 = ti * TILE, c0 = tl * TILE;
    for (int t = threadIdx.x; t < NB * TILE; t += blockDim.x) {
        int rr = t / NB, s = t % NB;
        int gi = r0 + rr, gl = c0 + rr;
        Ps[s * TILE + rr] = (gi < n && s < b) ? pan[(int64_t)gi * NB + s] : T(0);
        Os[s * TILE + rr] = (gl < n && s < b) ? old[(int64_t)gl * NB + s] : T(0);
    }
    __syncthreads();
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    T acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0;
    for (int s = 0; s < b; ++s) {
        T pa[4], ob[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) pa[u] = Ps[s * TILE + ty * 4 + u];
#pragma unroll
        for (int v = 0; v < 4; ++v) ob[v] = Os[s * TILE + tx * 4 + v];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] += pa[u] * ob[v];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = r0 + ty * 4 + u;
        if (i >= n) continue;
        const bool iJ = (i >= j0 && i < j1);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int l = c0 + tx * 4 + v;
            if (l >= n) continue;
            const bool lJ = (l >= j0 && l < j1);
            T *dst = M + (int64_t)i * ld + l;
            if (!iJ && !lJ) *dst = *dst - acc[u][v];
            else if (!iJ && lJ) *dst = pan[(int64_t)i * NB + (l - j0)];
            else if (iJ && !lJ) *dst = pan[(int64_t)l * NB + (i - j0)];
            else *dst = -D[(i - j0) * NB + (l - j0)];
        }
    }
}

#include "sweep_tc.cuh"

// copy A^k (FP64, ld = nk) into the swept-matrix pool (type T, ld = ldM, zero padding)
template <typename T> __global__ void k_load_matrix(const double *A, T *Mpool, const SubdomainDesc *sd) {
    const SubdomainDesc d = sd[blockIdx.y];
    const int64_t ld = d.ldM;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)d.nk * ld; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = t / ld, l = t % ld;
        Mpool[d.offM + t] = l < d.nk ? (T)A[d.offA + i * d.nk + l] : T(0);
    }
}

// A^k (FP64) -> hi + lo FP32 pairs in the swept-matrix layout (ld_M, zero padding):
// hi = fl32(a), lo = fl32(a - hi), so hi + lo equals a to about 2^-48 relative
// nonzeros per row of A^k (warp per row), at the row's subdomain-vector position
__global__ void k_row_nnz(const double *A, const SubdomainDesc *sd, int64_t *cnt) {
    const SubdomainDesc d = sd[blockIdx.y];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int i = blockIdx.x * 8 + warp; i < d.nk; i += gridDim.x * 8) {
        const double *Ai = A + d.offA + (int64_t)i * d.nk;
        unsigned n = 0;
        for (int l = lane; l < d.nk; l += 32) n += Ai[l] != 0.0 ? 1u : 0u;
        n = __reduce_add_sync(0xffffffffu, n);
        if (lane == 0) cnt[d.offV + i] = n;
    }
}

// the CSR entries of A^k, in ascending column order per row (warp per row, ballot compaction):
// column position offV + l, hi = A rounded to FP32, lo = the rest rounded to FP32
__global__ void k_fill_csr(const double *A, const SubdomainDesc *sd, const int64_t *ptr, int4 *ent) {
    const SubdomainDesc d = sd[blockIdx.y];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int i = blockIdx.x * 8 + warp; i < d.nk; i += gridDim.x * 8) {
        const double *Ai = A + d.offA + (int64_t)i * d.nk;
        int64_t base = ptr[d.offV + i];
        for (int l0 = 0; l0 < d.nk; l0 += 32) {
            const int l = l0 + lane;
            const double a = l < d.nk ? Ai[l] : 0.0;
            const unsigned m = __ballot_sync(0xffffffffu, a != 0.0);
            if (a != 0.0) {
                const float h = (float)a;
                ent[base + __popc(m & ((1u << lane) - 1u))] =
                    make_int4((int)(d.offV + l), __float_as_int(h), __float_as_int((float)(a - (double)h)), 0);
            }
            base += __popc(m);
        }
    }
}

__global__ void k_split_ds(const double *A, float *hi, float *lo, const SubdomainDesc *sd) {
    const SubdomainDesc d = sd[blockIdx.y];
    const int64_t ld = d.ldM;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)d.nk * ld; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / ld, l = t % ld;
        const double a = l < d.nk ? A[d.offA + i * d.nk + l] : 0.0;
        const float h = (float)a;
        hi[d.offM + t] = h;
        lo[d.offM + t] = (float)(a - (double)h);
    }
}

// copy the Gamma block of the swept matrix into S (and into Sp with pinning)
// largest |entry| of an FP32 array into *mx (bits of a non-negative float order as unsigned)
__global__ void k_absmax(const float *a, int64_t n, unsigned *mx) {
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(a[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(mx, __float_as_uint(m));
}

// h = half(a * scale), scale a power of two (the product is exact)
__global__ void k_to_half(const float *a, int64_t n, float scale, __half *h) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        h[i] = __float2half_rn(a[i] * scale);
}

// Sh tiled for the tensor-core apply: tile t of subdomain k (row tile t / kt, column tile
// t % kt, kt = mma_ktiles) holds rows 128 (t / kt) .. +127 and columns 64 (t % kt) .. +63 of
// S_k * scale in FP16 (zero past n_gamma or ld_gamma), row r at byte 128 r, its 16-byte chunk j
// (columns 8j..8j+7) at chunk position j ^ (r mod 8): the order of a 1 KB-aligned 128-byte
// swizzled K-major operand.  Grid (tiles of the largest subdomain / 4 blocks, K); 256 threads.
__global__ void k_tile_half(const float *S, float scale, const SubdomainDesc *sd, __half *T) {
    const SubdomainDesc d = sd[blockIdx.y];
    if (d.nG == 0) return;
    const int kt = mma_ktiles(d.nG, d.ldG);
    const int64_t ntiles = (int64_t)((d.nG + 127) / 128) * kt;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ntiles * 8192;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = e / 8192;
        const int w = (int)(e % 8192), r = w / 64, cl = w % 64;
        const int64_t i = (t / kt) * 128 + r, l = (t % kt) * 64 + cl;
        const float v = (i < d.nG && l < d.ldG) ? S[d.offS + i * d.ldG + l] * scale : 0.f;
        const int j = cl / 8, pos = r * 64 + ((j ^ (r & 7)) * 8) + cl % 8;
        T[(d.offT + t) * 8192 + pos] = __float2half_rn(v);
    }
}

template <typename T> __global__ void k_extract(const T *Mpool, T *Spool, T *Sppool, const SubdomainDesc *sd) {
    const SubdomainDesc d = sd[blockIdx.y];
    const int64_t nG = d.nG, ld = d.ldG;
    const T *M = Mpool + d.offM;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nG * ld; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = t / ld, l = t % ld;
        if (l >= nG) { Spool[d.offS + t] = T(0); Sppool[d.offSp + t] = T(0); continue; }
        T v = M[(d.nO + i) * d.ldM + d.nO + l];
        Spool[d.offS + t] = v;
        bool pi = false, pl = false;
        for (int q = 0; q < d.npin; ++q) { pi |= (d.pin[q] == i); pl |= (d.pin[q] == l); }
        Sppool[d.offSp + t] = (pi || pl) ? (i == l ? T(1) : T(0)) : v;
    }
}

// orthonormal basis of the kernel of a floating subdomain's S_k, restricted to Gamma_k
// (constants; or the two translations and the rotation about the Gamma_k centroid)
__global__ void k_kernel_basis(const double *xy, const int32_t *gnodes, const int64_t *goff, const SubdomainDesc *sd,
                               int nc, double *Z, double *Q) {
    const SubdomainDesc d = sd[blockIdx.x];
    if (!d.floating || d.nG == 0) return;
    const int ng = d.nG / nc;
    const int32_t *nodes = gnodes + goff[blockIdx.x];
    __shared__ double red[3][256];
    __shared__ double cen[2];
    const int m = nc == 1 ? 1 : 3;
    double *Zk = Z + d.offU * 3;
    double *Qk = Q + d.offU * 3;
    if (nc == 2) {
        double sx = 0, sy = 0;
        for (int i = threadIdx.x; i < ng; i += blockDim.x) { sx += xy[2 * (int64_t)nodes[i]]; sy += xy[2 * (int64_t)nodes[i] + 1]; }
        red[0][threadIdx.x] = sx; red[1][threadIdx.x] = sy;
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0, b = 0;
            for (int t = 0; t < blockDim.x; ++t) { a += red[0][t]; b += red[1][t]; }
            cen[0] = a / ng; cen[1] = b / ng;
        }
        __syncthreads();
    }
    for (int r = threadIdx.x; r < d.nG; r += blockDim.x) {
        for (int c = 0; c < 3; ++c) Zk[(int64_t)r * 3 + c] = 0.0;
        if (nc == 1) Zk[(int64_t)r * 3] = 1.0;
        else {
            int node = nodes[r / 2], comp = r % 2;
            Zk[(int64_t)r * 3 + comp] = 1.0;
            Zk[(int64_t)r * 3 + 2] = comp == 0 ? -(xy[2 * (int64_t)node + 1] - cen[1]) : (xy[2 * (int64_t)node] - cen[0]);
        }
        for (int c = 0; c < 3; ++c) Qk[(int64_t)r * 3 + c] = c < m ? Zk[(int64_t)r * 3 + c] : 0.0;
    }
    __syncthreads();
    // modified Gram-Schmidt, two passes
    for (int pass = 0; pass < 2; ++pass)
        for (int c = 0; c < m; ++c) {
            for (int pc = 0; pc < c; ++pc) {
                double s = 0;
                for (int r = threadIdx.x; r < d.nG; r += blockDim.x) s += Qk[(int64_t)r * 3 + c] * Qk[(int64_t)r * 3 + pc];
                red[0][threadIdx.x] = s;
                __syncthreads();
                if (threadIdx.x == 0) { double t = 0; for (int i = 0; i < blockDim.x; ++i) t += red[0][i]; red[1][0] = t; }
                __syncthreads();
                double proj = red[1][0];
                for (int r = threadIdx.x; r < d.nG; r += blockDim.x) Qk[(int64_t)r * 3 + c] -= proj * Qk[(int64_t)r * 3 + pc];
                __syncthreads();
            }
            double s = 0;
            for (int r = threadIdx.x; r < d.nG; r += blockDim.x) s += Qk[(int64_t)r * 3 + c] * Qk[(int64_t)r * 3 + c];
            red[0][threadIdx.x] = s;
            __syncthreads();
            if (threadIdx.x == 0) { double t = 0; for (int i = 0; i < blockDim.x; ++i) t += red[0][i]; red[1][0] = sqrt(t); }
            __syncthreads();
            double nrm = red[1][0];
            for (int r = threadIdx.x; r < d.nG; r += blockDim.x) Qk[(int64_t)r * 3 + c] /= nrm;
            __syncthreads();
        }
}

// W = -(swept pinned S~) with pinned rows/columns zeroed; then V = W Q (FP64)
template <typename T> __global__ void k_finish_inverse(T *Sppool, const SubdomainDesc *sd) {
    const SubdomainDesc d = sd[blockIdx.y];
    const int64_t nG = d.nG, ld = d.ldG;
    T *W = Sppool + d.offSp;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nG * ld; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = t / ld, l = t % ld;
        if (l >= nG) continue;
        bool pz = false;
        for (int q = 0; q < d.npin; ++q) pz |= (d.pin[q] == i) || (d.pin[q] == l);
        W[t] = pz ? T(0) : -W[t];
    }
}

template <typename T> __global__ void k_wq(const T *Sppool, const SubdomainDesc *sd, const double *Q, double *V) {
    const SubdomainDesc d = sd[blockIdx.y];
    if (!d.floating || d.nG == 0) return;
    const int m = d.n_co;
    const int64_t nG = d.nG;
    const T *W = Sppool + d.offSp;
    const double *Qk = Q + d.offU * 3;
    double *Vk = V + d.offU * 3;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + warp; i < nG; i += (int64_t)gridDim.x * (blockDim.x / 32)) {
        double s[3] = {0, 0, 0};
        for (int64_t l = lane; l < nG; l += 32) {
            double w = (double)W[i * d.ldG + l];
            for (int c = 0; c < m; ++c) s[c] += w * Qk[l * 3 + c];
        }
        for (int c = 0; c < m; ++c)
            for (int o = 16; o > 0; o >>= 1) s[c] += __shfl_xor_sync(0xffffffffu, s[c], o);
        if (lane == 0)
            for (int c = 0; c < 3; ++c) Vk[i * 3 + c] = c < m ? s[c] : 0.0;
    }
}

// C = Q^T V (m x m), one CTA per floating subdomain
__global__ void k_qtv(const SubdomainDesc *sd, const double *Q, const double *V, double *C) {
    const SubdomainDesc d = sd[blockIdx.x];
    if (!d.floating || d.nG == 0) return;
    const int m = d.n_co;
    __shared__ double red[256];
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) {
            double s = 0;
            for (int64_t r = threadIdx.x; r < d.nG; r += blockDim.x) s += Q[(d.offU + r) * 3 + a] * V[(d.offU + r) * 3 + b];
            red[threadIdx.x] = s;
            __syncthreads();
            for (int o = blockDim.x / 2; o > 0; o >>= 1) {
                if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
                __syncthreads();
            }
            if (threadIdx.x == 0) C[blockIdx.x * 9 + a * 3 + b] = red[0];
            __syncthreads();
        }
}

// S^+ = W - Q V^T - V Q^T + Q C Q^T
template <typename T> __global__ void k_project(T *Sppool, const SubdomainDesc *sd, const double *Q, const double *V,
                                               const double *C) {
    const SubdomainDesc d = sd[blockIdx.y];
    if (!d.floating || d.nG == 0) return;
    const int m = d.n_co;
    const int64_t nG = d.nG;
    T *W = Sppool + d.offSp;
    const double *Ck = C + blockIdx.y * 9;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nG * nG; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = t / nG, l = t % nG;
        const double *qi = Q + (d.offU + i) * 3, *ql = Q + (d.offU + l) * 3;
        T *Wt = W + i * d.ldG + l;
        const double *vi = V + (d.offU + i) * 3, *vl = V + (d.offU + l) * 3;
        double corr = 0;
        for (int a = 0; a < m; ++a) {
            corr -= qi[a] * vl[a] + vi[a] * ql[a];
            for (int b = 0; b < m; ++b) corr += qi[a] * Ck[a * 3 + b] * ql[b];
        }
        *Wt = (T)((double)*Wt + corr);
    }
}

template <typename T> void run_sweeps(nlfeti_problem *p, T *pool, const std::vector<int64_t> &moff,
                                      const std::vector<int32_t> &mdim, const std::vector<int32_t> &mld,
                                      const std::vector<int32_t> &pend, DevMem &scratch, bool allow_tc) {
    nlfeti_ctx *c = p->ctx;
    const int K = p->K;
    std::vector<int64_t> soff(K);
    int64_t rows = 0;
    int maxn = 0, maxp = 0;
    for (int k = 0; k < K; ++k) {
        soff[k] = rows;
        rows += mdim[k];
        maxn = std::max(maxn, mdim[k]);
        maxp = std::max(maxp, pend[k]);
    }
    if (maxp == 0) return;
    size_t need = sizeof(T) * ((size_t)rows * NB * 2 + (size_t)K * NB * NB);
    if (scratch.bytes < need) scratch.alloc(c, need);
    DevMem d_moff, d_mdim, d_mld, d_pend, d_soff;
    upload(c, d_moff, moff);
    upload(c, d_mdim, mdim);
    upload(c, d_mld, mld);
    upload(c, d_pend, pend);
    upload(c, d_soff, soff);
    SweepArgs<T> a;
    a.M = pool;
    a.pan = scratch.as<T>();
    a.old = a.pan + rows * NB;
    a.dinv = a.old + rows * NB;
    a.sd = p->d_sd.as<SubdomainDesc>();
    a.moff = d_moff.as<int64_t>();
    a.mdim = d_mdim.as<int32_t>();
    a.mld = d_mld.as<int32_t>();
    a.pend = d_pend.as<int32_t>();
    a.scr_off = d_soff.as<int64_t>();
    a.flag = p->d_flag.as<int>();
    const int nt = (maxn + TILE - 1) / TILE;
    const size_t smu = sizeof(T) * 2 * NB * TILE;
    NLF_CUDA(cudaFuncSetAttribute(k_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smu));
    // FP32 operators with factor_tc: the rank-64 updates on the tensor cores (split-TF32)
    const bool tc = std::is_same<T, float>::value && allow_tc;
    const int ntc = (maxn + TC_TILE - 1) / TC_TILE;
    if (tc) NLF_CUDA(cudaFuncSetAttribute(k_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    for (int j0 = 0; j0 < maxp; j0 += NB) {
        a.j0 = j0;
        k_pivot<T><<<K, 256, 0, c->stream>>>(a);
        k_panel<T><<<dim3((maxn + 3) / 4, K), 256, 0, c->stream>>>(a);
        if constexpr (std::is_same<T, float>::value) {
            if (tc) {
                k_update_tc<<<dim3(ntc, ntc, K), TC_THREADS, TC_SMEM, c->stream>>>(a, p->d_flag.as<int>() + 2);
                continue;
            }
        }
        k_update<T><<<dim3(nt, nt, K), 256, smu, c->stream>>>(a);
    }
    NLF_CUDA(cudaGetLastError());
    NLF_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace

// the FP16 copy of S_k tiled for the tensor-core apply (after the FP32 factorization)
void build_tiled_half(nlfeti_problem *p) {
    nlfeti_ctx *c = p->ctx;
    OpPool<float> &pool = p->op32;
    if (!pool.S.p || pool.St.p) return;
    pool.St.alloc(c, sizeof(__half) * 8192 * std::max<int64_t>(p->poolT, 1));
    if (p->poolT > 0 && p->K > 0) {
        k_tile_half<<<dim3(256, p->K), 256, 0, c->stream>>>(pool.S.as<float>(), (float)pool.hscale,
                                                            p->d_sd.as<SubdomainDesc>(), pool.St.as<__half>());
        NLF_CUDA(cudaGetLastError());
    }
    NLF_CUDA(cudaStreamSynchronize(c->stream));
}

// The operator of the refinement residual: A^k as a CSR of FP32 pairs when at most an eighth
// of the dense entries are nonzero (kernels of compact support with a horizon of a few mesh
// sizes), else dense FP32 pairs in the swept-matrix layout (Ahi, Alo); opt.residual_format 1 / 2
// forces one of the two.  The crossover: per nonzero the CSR kernel gathers the 8 R bytes of u
// it multiplies through L1 / L2, where the dense kernel stages u once per 32 rows, and measured
// about 7.5 times the dense kernel's time per entry.  Depends on A^k and the option only.
void build_residual_operator(nlfeti_problem *p, OpPool<float> &pool) {
    nlfeti_ctx *c = p->ctx;
    const int K = p->K;
    const int64_t nrows = p->sum_nk;
    pool.a_sparse = false;
    pool.a_nnz = 0;
    pool.Aptr.release();
    pool.Aent.release();
    pool.row_u.release();
    double dense = 0;
    for (const auto &d : p->sd) dense += (double)d.nk * d.nk;
    if (nrows > 0 && K > 0) {
        DevMem cnt;
        cnt.alloc(c, sizeof(int64_t) * nrows);
        k_row_nnz<<<dim3(64, K), 256, 0, c->stream>>>(p->d_A.as<double>(), p->d_sd.as<SubdomainDesc>(),
                                                      cnt.as<int64_t>());
        NLF_CUDA(cudaGetLastError());
        std::vector<int64_t> h(nrows), ptr(nrows + 1, 0);
        NLF_CUDA(cudaMemcpyAsync(h.data(), cnt.p, sizeof(int64_t) * nrows, cudaMemcpyDeviceToHost, c->stream));
        NLF_CUDA(cudaStreamSynchronize(c->stream));
        for (int64_t g = 0; g < nrows; ++g) ptr[g + 1] = ptr[g] + h[g];
        const int64_t nnz = ptr[nrows];
        const int fmt = p->opt.residual_format;
        if (fmt == 2 || (fmt == 0 && 8.0 * (double)nnz <= dense)) {
            upload(c, pool.Aptr, ptr);
            pool.Aent.alloc(c, sizeof(int4) * std::max<int64_t>(1, nnz));
            k_fill_csr<<<dim3(64, K), 256, 0, c->stream>>>(p->d_A.as<double>(), p->d_sd.as<SubdomainDesc>(),
                                                           pool.Aptr.as<int64_t>(), pool.Aent.as<int4>());
            NLF_CUDA(cudaGetLastError());
            std::vector<int32_t> ru(nrows, -1);
            for (const auto &d : p->sd)
                for (int i = d.nO; i < d.nk; ++i) ru[d.offV + i] = (int32_t)(d.offU + (i - d.nO));
            upload(c, pool.row_u, ru);
            NLF_CUDA(cudaStreamSynchronize(c->stream));
            pool.Ahi.release();
            pool.Alo.release();
            pool.a_sparse = true;
            pool.a_nnz = nnz;
            return;
        }
    }
    const int64_t poolM = p->poolM;
    pool.Ahi.alloc(c, sizeof(float) * std::max<int64_t>(poolM, 1));
    pool.Alo.alloc(c, sizeof(float) * std::max<int64_t>(poolM, 1));
    k_split_ds<<<dim3(256, std::max(1, K)), 256, 0, c->stream>>>(p->d_A.as<double>(), pool.Ahi.as<float>(),
                                                                 pool.Alo.as<float>(), p->d_sd.as<SubdomainDesc>());
    NLF_CUDA(cudaGetLastError());
}

template <typename T> void factor_ops(nlfeti_problem *p, OpPool<T> &pool) {
    nlfeti_ctx *c = p->ctx;
    const int K = p->K;
    pool.ready = false;          // until this factorization has succeeded
    int64_t poolM = p->poolM, poolG = p->poolG;
    pool.M.alloc(c, sizeof(T) * std::max<int64_t>(poolM, 1));
    pool.S.alloc(c, sizeof(T) * std::max<int64_t>(poolG, 1));
    pool.Sp.alloc(c, sizeof(T) * std::max<int64_t>(poolG, 1));
    NLF_CUDA(cudaMemsetAsync(p->d_flag.p, 0, sizeof(int) * 4, c->stream));
    // phase 1: sweep the Omega pivots of A^k
    NLF_CUDA(cudaMemsetAsync(pool.S.p, 0, pool.S.bytes, c->stream));
    NLF_CUDA(cudaMemsetAsync(pool.Sp.p, 0, pool.Sp.bytes, c->stream));
    k_load_matrix<T><<<dim3(256, K), 256, 0, c->stream>>>(p->d_A.as<double>(), pool.M.template as<T>(),
                                                          p->d_sd.as<SubdomainDesc>());
    if constexpr (std::is_same<T, float>::value) build_residual_operator(p, pool);
    NLF_CUDA(cudaGetLastError());
    std::vector<int64_t> moff(K), soff(K);
    std::vector<int32_t> mdim(K), mld(K), pend(K), gdim(K), gld(K), gend(K);
    for (int k = 0; k < K; ++k) {
        moff[k] = p->sd[k].offM;
        mdim[k] = p->sd[k].nk;
        mld[k] = p->sd[k].ldM;
        pend[k] = p->sd[k].nO;
        soff[k] = p->sd[k].offSp;
        gdim[k] = p->sd[k].nG;
        gld[k] = p->sd[k].ldG;
        gend[k] = p->sd[k].nG;
    }
    run_sweeps<T>(p, pool.M.template as<T>(), moff, mdim, mld, pend, pool.scratch, p->opt.factor_tc != 0);
    // S_k and the pinned copy
    int maxg = 0;
    for (auto &d : p->sd) maxg = std::max(maxg, d.nG);
    if (maxg > 0) {
        dim3 g(256, K);
        k_extract<T><<<g, 256, 0, c->stream>>>(pool.M.template as<T>(), pool.S.template as<T>(),
                                               pool.Sp.template as<T>(), p->d_sd.as<SubdomainDesc>());
        NLF_CUDA(cudaGetLastError());
        // phase 2: sweep all pivots of the pinned S~_k
        run_sweeps<T>(p, pool.Sp.template as<T>(), soff, gdim, gld, gend, pool.scratch, p->opt.factor_tc == 1);
        k_finish_inverse<T><<<g, 256, 0, c->stream>>>(pool.Sp.template as<T>(), p->d_sd.as<SubdomainDesc>());
        if (p->n_floating > 0) {
            DevMem V, C;
            V.alloc(c, sizeof(double) * 3 * std::max<int64_t>(p->n_u, 1));
            C.alloc(c, sizeof(double) * 9 * K);
            k_wq<T><<<dim3(64, K), 256, 0, c->stream>>>(pool.Sp.template as<T>(), p->d_sd.as<SubdomainDesc>(),
                                                         p->d_Q.as<double>(), V.as<double>());
            k_qtv<<<K, 256, 0, c->stream>>>(p->d_sd.as<SubdomainDesc>(), p->d_Q.as<double>(), V.as<double>(),
                                            C.as<double>());
            k_project<T><<<g, 256, 0, c->stream>>>(pool.Sp.template as<T>(), p->d_sd.as<SubdomainDesc>(),
                                                   p->d_Q.as<double>(), V.as<double>(), C.as<double>());
            NLF_CUDA(cudaGetLastError());
            NLF_CUDA(cudaStreamSynchronize(c->stream));
        }
    }
    NLF_CUDA(cudaStreamSynchronize(c->stream));
    int flag[3] = {0, 0, 0};
    NLF_CUDA(cudaMemcpy(flag, p->d_flag.p, sizeof(flag), cudaMemcpyDeviceToHost));
    if (flag[2]) {
        NLF_CUDA(cudaMemset(p->d_flag.as<int>() + 2, 0, sizeof(int)));
        fail(NLFETI_E_TIMEOUT, "a tensor-core update of the factorization did not complete in time");
    }
    if (flag[0]) fail(NLFETI_E_NOT_SPD, "a pivot block of a subdomain operator was not positive definite");
    if constexpr (std::is_same<T, float>::value) {
        // FP16 copy of S_k for the preconditioner, scaled by one power of two so that the
        // largest entry lies in [2^13, 2^14) (FP16 keeps 11 bits from 2^-14 up to 65504)
        DevMem mx;
        mx.alloc(c, sizeof(unsigned));
        NLF_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(unsigned), c->stream));
        const int64_t n = std::max<int64_t>(poolG, 1);
        k_absmax<<<256, 256, 0, c->stream>>>(pool.S.template as<float>(), n, mx.as<unsigned>());
        unsigned bits = 0;
        NLF_CUDA(cudaMemcpyAsync(&bits, mx.p, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
        NLF_CUDA(cudaStreamSynchronize(c->stream));
        float m;
        std::memcpy(&m, &bits, sizeof(m));
        pool.hscale = (m > 0.f && std::isfinite(m)) ? std::ldexp(1.0, 13 - std::ilogb(m)) : 1.0;
        pool.Sh.alloc(c, sizeof(__half) * n);
        k_to_half<<<512, 256, 0, c->stream>>>(pool.S.template as<float>(), n, (float)pool.hscale,
                                              pool.Sh.template as<__half>());
        NLF_CUDA(cudaGetLastError());
        // the tiled copy for the tensor-core apply only when that apply is selected (else built
        // by nlfeti_problem_set_options when it is)
        pool.St.release();
        if (p->opt.precond_fp16 == 2) build_tiled_half(p);
    }
    encode_apply_maps<T>(p, pool);
    pool.ready = true;
}

template void factor_ops<double>(nlfeti_problem *, OpPool<double> &);
template void factor_ops<float>(nlfeti_problem *, OpPool<float> &);

// ------------------------------------------------------------------ coarse problem and weights

namespace {

__global__ void k_gtg(const int64_t *Bp, const int64_t *Bm, int64_t nl, const int32_t *u2sub, const SubdomainDesc *sd,
                      const double *Z, int nco, double *GtG) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nl; r += (int64_t)gridDim.x * blockDim.x) {
        int64_t up = Bp[r], um = Bm[r];
        int kp = u2sub[up], km = u2sub[um];
        const SubdomainDesc dp = sd[kp], dm = sd[km];
        // G row r: +Z[up, :] on columns of kp, -Z[um, :] on columns of km
        int cols[6];
        double vals[6];
        int n = 0;
        for (int c = 0; c < dp.n_co; ++c) { cols[n] = dp.co_off + c; vals[n++] = Z[up * 3 + c]; }
        for (int c = 0; c < dm.n_co; ++c) { cols[n] = dm.co_off + c; vals[n++] = -Z[um * 3 + c]; }
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b)
                if (vals[a] != 0.0 && vals[b] != 0.0) atomicAdd(GtG + (int64_t)cols[a] * nco + cols[b], vals[a] * vals[b]);
    }
}

// per B^T entry e of U dof u: its Lambda row and sign(e) Z[u][0..2]
__global__ void k_gt_entries(const int64_t *bt_ptr, const int64_t *bt_row, const double *Z, int64_t nu, int64_t *rows,
                             double *w) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += (int64_t)gridDim.x * blockDim.x)
        for (int64_t e = bt_ptr[u]; e < bt_ptr[u + 1]; ++e) {
            const int64_t r = bt_row[e];
            const double sg = r > 0 ? 1.0 : -1.0;
            rows[e] = (r > 0 ? r : -r) - 1;
            for (int q = 0; q < 3; ++q) w[e * 3 + q] = sg * Z[u * 3 + q];
        }
}

// slots of the rows of G = B Z (see nlfeti_problem::gw)
__global__ void k_g_rows(const int64_t *Bp, const int64_t *Bm, int64_t nl, const int32_t *u2sub,
                         const SubdomainDesc *sd, const double *Z, int gw, int32_t *gcol, double *gval) {
    const int h = gw / 2;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nl; r += (int64_t)gridDim.x * blockDim.x) {
        for (int side = 0; side < 2; ++side) {
            const int64_t u = side ? Bm[r] : Bp[r];
            const SubdomainDesc d = sd[u2sub[u]];
            for (int a = 0; a < h; ++a) {
                const int64_t slot = r * gw + side * h + a;
                gcol[slot] = a < d.n_co ? d.co_off + a : -1;
                gval[slot] = a < d.n_co ? Z[u * 3 + a] : 0.0;
            }
        }
    }
}

// in-place inverse of a small SPD matrix (n <= 128) by one CTA; result written back
__global__ void k_small_inverse(double *A, int n, int *flag) {
    extern __shared__ double sm[];
    double *S = sm;
    double *rowp = sm + n * n;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) S[t] = A[t];
    bool ok = sweep_block_shared(S, n, n, rowp);
    if (!ok && threadIdx.x == 0) atomicMax(flag, 1);
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) A[t] = -S[t];
}

// The same sweep for a coarse matrix too large for shared memory (n_co > 128: the peridynamic
// kernel's three rigid modes on many floating subdomains), one pivot per launch: every entry
// (i, l) of the n x n matrix in global memory takes pivot p from rowp_in (row p before this
// pivot, = column p by symmetry) exactly as sweep_block_shared does, and the thread of row
// p + 1 also writes that row's new values to rowp_out for the next launch.  Grid over n^2.
__global__ void k_sweep_pivot_global(double *S, int n, int p, const double *rowp_in, double *rowp_out, int *flag) {
    const double d = rowp_in[p];
    const double inv = 1.0 / d;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)n * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / n), l = (int)(t % n);
        double v;
        if (i == p && l == p) v = -inv;
        else if (i == p) v = rowp_in[l] * inv;
        else if (l == p) v = rowp_in[i] * inv;
        else v = S[t] - rowp_in[i] * rowp_in[l] * inv;
        S[t] = v;
        if (i == p + 1) rowp_out[l] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && !(d > 0.0)) atomicMax(flag, 1);
}

__global__ void k_negate(double *A, int64_t n) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        A[t] = -A[t];
}

// B_D = (B D^-1 B^T)^-1 B D^-1 per node block (chain rows, D = zeta on every copy):
// B B^T = tridiag(-1, 2, -1) on the z-1 links of a node with z copies
__global__ void k_bd_blocks(const int32_t *blk_ptr, int64_t nblk, const int32_t *blk_rows, const int64_t *bd_ptr,
                            double *bd_val, int *flag) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += (int64_t)gridDim.x * blockDim.x) {
        const int r0 = blk_ptr[b], r1 = blk_ptr[b + 1];
        const int m = r1 - r0;             // rows in the block = zeta - 1
        const int z = m + 1;               // copies
        if (m > 15) { atomicMax(flag, 1); continue; }
        double S[15][15], Binv[15][15];
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                S[i][j] = (i == j ? 2.0 : (abs(i - j) == 1 ? -1.0 : 0.0)) / (double)z;
                Binv[i][j] = i == j ? 1.0 : 0.0;
            }
        for (int p = 0; p < m; ++p) {        // Gauss-Jordan on the SPD block
            double d = S[p][p];
            for (int j = 0; j < m; ++j) { S[p][j] /= d; Binv[p][j] /= d; }
            for (int i = 0; i < m; ++i)
                if (i != p) {
                    double f = S[i][p];
                    for (int j = 0; j < m; ++j) { S[i][j] -= f * S[p][j]; Binv[i][j] -= f * Binv[p][j]; }
                }
        }
        // row i of B_D: sum_j Binv[i][j] (row j of B) / z; row j has +1 at copy j, -1 at copy j+1
        for (int i = 0; i < m; ++i) {
            const int64_t row = blk_rows[r0 + i];
            for (int cpy = 0; cpy < z; ++cpy) {
                double v = 0;
                if (cpy < m) v += Binv[i][cpy] / (double)z;
                if (cpy >= 1) v -= Binv[i][cpy - 1] / (double)z;
                bd_val[bd_ptr[row] + cpy] = v;
            }
        }
    }
}

__global__ void k_gather_vals(const int64_t *src_idx, const double *src, double *dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[src_idx[i]];
}

// dst[j n + i] = src[i n + j] rounded to FP32 (n x n)
__global__ void k_round_f32_t(const double *src, float *dst, int n) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)n * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / n, i = t % n;
        dst[t] = (float)src[i * n + j];
    }
}

__global__ void k_round_f32(const double *src, float *dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

// dst = src (n doubles) rounded to FP32: the weights the FP32 PCG iterations read
void f32_copy(nlfeti_ctx *c, DevMem &dst, const DevMem &src, int64_t n) {
    dst.alloc(c, sizeof(float) * std::max<int64_t>(1, n));
    if (n > 0) k_round_f32<<<256, 256, 0, c->stream>>>(src.as<double>(), dst.as<float>(), n);
    NLF_CUDA(cudaGetLastError());
}

}  // namespace

void setup_coarse(nlfeti_problem *p) {
    nlfeti_ctx *c = p->ctx;
    // kernel bases on Gamma_k (all subdomains get Z, Q rows; only floating ones are filled)
    std::vector<int32_t> gnodes;
    std::vector<int64_t> goff(p->K + 1, 0);
    for (int k = 0; k < p->K; ++k) {
        const auto &nd = p->dec.nodes[k];
        int nO = p->dec.n_omega_nodes[k];
        gnodes.insert(gnodes.end(), nd.begin() + nO, nd.end());
        goff[k + 1] = goff[k] + (int64_t)(nd.size() - nO);
    }
    DevMem d_gn, d_goff;
    upload(c, d_gn, gnodes);
    upload(c, d_goff, goff);
    p->d_Z.alloc(c, sizeof(double) * 3 * std::max<int64_t>(p->n_u, 1));
    p->d_Q.alloc(c, sizeof(double) * 3 * std::max<int64_t>(p->n_u, 1));
    NLF_CUDA(cudaMemsetAsync(p->d_Z.p, 0, p->d_Z.bytes, c->stream));
    NLF_CUDA(cudaMemsetAsync(p->d_Q.p, 0, p->d_Q.bytes, c->stream));
    k_kernel_basis<<<p->K, 256, 0, c->stream>>>(p->d_xy.as<double>(), d_gn.as<int32_t>(), d_goff.as<int64_t>(),
                                                 p->d_sd.as<SubdomainDesc>(), p->nc, p->d_Z.as<double>(),
                                                 p->d_Q.as<double>());
    NLF_CUDA(cudaGetLastError());
    const int nco = p->n_co;
    int max_nco = 0;
    std::vector<int32_t> fl;
    for (int k = 0; k < p->K; ++k) {
        max_nco = std::max(max_nco, (int)p->sd[k].n_co);
        if (p->sd[k].n_co > 0) fl.push_back(k);
    }
    upload(c, p->d_float_ids, fl);
    {
        // G^T entry ranges of the floating subdomains (B^T entries of Gamma_f are contiguous)
        std::vector<int64_t> bt_ptr(p->n_u + 1, 0);
        NLF_CUDA(cudaMemcpyAsync(bt_ptr.data(), p->d_Bt_ptr.p, sizeof(int64_t) * (p->n_u + 1), cudaMemcpyDeviceToHost,
                                 c->stream));
        NLF_CUDA(cudaStreamSynchronize(c->stream));
        std::vector<int64_t> range;
        std::vector<int32_t> co;
        for (int k : fl) {
            const SubdomainDesc &d = p->sd[k];
            range.push_back(bt_ptr[d.offU]);
            range.push_back(bt_ptr[d.offU + d.nG]);
            range.push_back(d.offU);
            range.push_back(d.offU + d.nG);
            co.push_back(d.co_off);
            co.push_back(d.n_co);
        }
        upload(c, p->d_gt_range, range);
        upload(c, p->d_gt_co, co);
        const int64_t ne = std::max<int64_t>(1, bt_ptr[p->n_u]);
        p->d_gt_rows.alloc(c, sizeof(int64_t) * ne);
        p->d_gt_w.alloc(c, sizeof(double) * 3 * ne);
        if (p->n_u > 0)
            k_gt_entries<<<256, 256, 0, c->stream>>>(p->d_Bt_ptr.as<int64_t>(), p->d_Bt_row.as<int64_t>(),
                                                     p->d_Z.as<double>(), p->n_u, p->d_gt_rows.as<int64_t>(),
                                                     p->d_gt_w.as<double>());
        f32_copy(c, p->d_gt_w32, p->d_gt_w, p->n_u > 0 ? 3 * ne : 0);
    }
    p->gw = 2 * max_nco;
    p->d_Gcol.alloc(c, sizeof(int32_t) * std::max<int64_t>(1, p->n_lambda * p->gw));
    p->d_Gval.alloc(c, sizeof(double) * std::max<int64_t>(1, p->n_lambda * p->gw));
    if (p->gw > 0 && p->n_lambda > 0)
        k_g_rows<<<256, 256, 0, c->stream>>>(p->d_Bp.as<int64_t>(), p->d_Bm.as<int64_t>(), p->n_lambda,
                                             p->d_u2sub.as<int32_t>(), p->d_sd.as<SubdomainDesc>(), p->d_Z.as<double>(),
                                             p->gw, p->d_Gcol.as<int32_t>(), p->d_Gval.as<double>());
    f32_copy(c, p->d_Gval32, p->d_Gval, (p->gw > 0 && p->n_lambda > 0) ? p->n_lambda * p->gw : 0);
    p->d_GtGinv.alloc(c, sizeof(double) * std::max(1, nco * nco));
    if (nco > 0) {
        if (nco > kMaxCoarse) fail(NLFETI_E_INVALID, "more than 12288 coarse columns");
        NLF_CUDA(cudaMemsetAsync(p->d_GtGinv.p, 0, sizeof(double) * (size_t)nco * nco, c->stream));
        if (p->n_lambda > 0)
            k_gtg<<<256, 256, 0, c->stream>>>(p->d_Bp.as<int64_t>(), p->d_Bm.as<int64_t>(), p->n_lambda,
                                              p->d_u2sub.as<int32_t>(), p->d_sd.as<SubdomainDesc>(),
                                              p->d_Z.as<double>(), nco, p->d_GtGinv.as<double>());
        if (nco <= 128) {
            size_t sm = sizeof(double) * (nco * nco + nco);
            NLF_CUDA(cudaFuncSetAttribute(k_small_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            k_small_inverse<<<1, 256, sm, c->stream>>>(p->d_GtGinv.as<double>(), nco, p->d_flag.as<int>());
        } else {
            DevMem rows;
            rows.alloc(c, sizeof(double) * 2 * (size_t)nco);
            double *r0 = rows.as<double>(), *r1 = r0 + nco;
            double *G = p->d_GtGinv.as<double>();
            NLF_CUDA(cudaMemcpyAsync(r0, G, sizeof(double) * nco, cudaMemcpyDeviceToDevice, c->stream));
            const int blocks = (int)std::min<int64_t>(4096, ((int64_t)nco * nco + 255) / 256);
            for (int q = 0; q < nco; ++q) {
                k_sweep_pivot_global<<<blocks, 256, 0, c->stream>>>(G, nco, q, (q & 1) ? r1 : r0, (q & 1) ? r0 : r1,
                                                                    p->d_flag.as<int>());
            }
            k_negate<<<blocks, 256, 0, c->stream>>>(G, (int64_t)nco * nco);
            NLF_CUDA(cudaStreamSynchronize(c->stream));
        }
        NLF_CUDA(cudaGetLastError());
    }
    p->d_GtGinv32.alloc(c, sizeof(float) * std::max(1, nco * nco));
    if (nco > 0) k_round_f32_t<<<256, 256, 0, c->stream>>>(p->d_GtGinv.as<double>(), p->d_GtGinv32.as<float>(), nco);
    NLF_CUDA(cudaGetLastError());
    NLF_CUDA(cudaStreamSynchronize(c->stream));
}

void setup_jump_weights(nlfeti_problem *p) {
    nlfeti_ctx *c = p->ctx;
    // blocks: consecutive B rows of one (node, component); rows of a node are chain links
    // j = 0..z-2 with the component fastest, so the rows of (node, comp) are r0 + comp + nc*j.
    const int nc = p->nc;
    const auto &Bn = p->dec.B_node;
    const int64_t nl = p->n_lambda;
    std::vector<int32_t> blk_ptr{0}, blk_rows;
    std::vector<int64_t> bd_ptr(nl + 1, 0), bd_col;
    // copies of each block (U indices in chain order)
    std::vector<std::vector<int64_t>> blk_copies;
    int64_t r = 0;
    while (r < nl) {
        int64_t s = r;
        while (s < nl && Bn[s] == Bn[r]) ++s;
        const int64_t links = (s - r) / nc;
        for (int comp = 0; comp < nc; ++comp) {
            std::vector<int64_t> copies;
            for (int64_t j = 0; j < links; ++j) {
                int64_t row = r + comp + nc * j;
                blk_rows.push_back((int32_t)row);
                if (j == 0) copies.push_back(p->dec.B_plus[row]);
                copies.push_back(p->dec.B_minus[row]);
            }
            blk_ptr.push_back((int32_t)blk_rows.size());
            blk_copies.push_back(copies);
        }
        r = s;
    }
    // B_D CSR: each row of a block has one entry per copy of its block
    {
        int64_t nb = (int64_t)blk_copies.size();
        std::vector<int64_t> row_len(nl, 0);
        for (int64_t b = 0; b < nb; ++b)
            for (int32_t i = blk_ptr[b]; i < blk_ptr[b + 1]; ++i) row_len[blk_rows[i]] = (int64_t)blk_copies[b].size();
        for (int64_t i = 0; i < nl; ++i) bd_ptr[i + 1] = bd_ptr[i] + row_len[i];
        bd_col.assign(bd_ptr[nl], 0);
        for (int64_t b = 0; b < nb; ++b)
            for (int32_t i = blk_ptr[b]; i < blk_ptr[b + 1]; ++i)
                for (size_t cp = 0; cp < blk_copies[b].size(); ++cp) bd_col[bd_ptr[blk_rows[i]] + cp] = blk_copies[b][cp];
    }
    DevMem d_blk_ptr, d_blk_rows;
    upload(c, d_blk_ptr, blk_ptr);
    upload(c, d_blk_rows, blk_rows);
    upload(c, p->d_BD_ptr, bd_ptr);
    upload(c, p->d_BD_col, bd_col);
    p->d_BD_val.alloc(c, sizeof(double) * std::max<int64_t>(1, bd_ptr[nl]));
    const int64_t nblk = (int64_t)blk_copies.size();
    if (nblk > 0) {
        k_bd_blocks<<<(unsigned)((nblk + 127) / 128), 128, 0, c->stream>>>(
            d_blk_ptr.as<int32_t>(), nblk, d_blk_rows.as<int32_t>(), p->d_BD_ptr.as<int64_t>(),
            p->d_BD_val.as<double>(), p->d_flag.as<int>() + 1);
        NLF_CUDA(cudaGetLastError());
    }
    f32_copy(c, p->d_BD_val32, p->d_BD_val, nblk > 0 ? bd_ptr[nl] : 0);
    // transpose CSR (per U dof: rows and value positions)
    std::vector<int64_t> t_ptr(p->n_u + 1, 0), t_row, t_src;
    for (int64_t i = 0; i < (int64_t)bd_col.size(); ++i) t_ptr[bd_col[i] + 1]++;
    for (int64_t u = 0; u < p->n_u; ++u) t_ptr[u + 1] += t_ptr[u];
    t_row.assign(bd_col.size(), 0);
    t_src.assign(bd_col.size(), 0);
    {
        std::vector<int64_t> fill(t_ptr.begin(), t_ptr.end() - 1);
        for (int64_t row = 0; row < nl; ++row)
            for (int64_t q = bd_ptr[row]; q < bd_ptr[row + 1]; ++q) {
                int64_t u = bd_col[q];
                t_row[fill[u]] = row;
                t_src[fill[u]] = q;
                fill[u]++;
            }
    }
    upload(c, p->d_BDt_ptr, t_ptr);
    upload(c, p->d_BDt_row, t_row);
    DevMem d_src;
    upload(c, d_src, t_src);
    p->d_BDt_val.alloc(c, sizeof(double) * std::max<size_t>(1, t_src.size()));
    if (!t_src.empty()) {
        k_gather_vals<<<256, 256, 0, c->stream>>>(d_src.as<int64_t>(), p->d_BD_val.as<double>(),
                                                  p->d_BDt_val.as<double>(), (int64_t)t_src.size());
        NLF_CUDA(cudaGetLastError());
    }
    f32_copy(c, p->d_BDt_val32, p->d_BDt_val, (int64_t)t_src.size());
    NLF_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace nlf
