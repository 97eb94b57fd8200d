// Streaming row-product kernel: the per-iteration interface applies with S_k^+ and S_k,
// and the per-sweep reduced forcing and back substitution on the swept matrices.
//
// Work item = (subdomain k, first of 32 rows).  Each warp owns 4 rows; each lane streams 4
// (FP32) or 2 (FP64) consecutive columns of all 4 rows per step with 16-byte streaming
// loads, two steps unrolled (8 loads in flight per lane), and reuses every x vector for the
// 4 rows.  Products accumulate in T per lane; the lane sum is a shuffle tree in T.
//
// Modes (same streaming structure, different rows / columns / vectors):
//   ROWS_APPLY:   y_U = M x_U with M = S_k^+ or S_k (rows and columns Gamma_k).  x is read
//                 directly (L1-cached) from the apply input written by the gathers: FP64, for
//                 subdomain k R columns of ldG entries at offUp*R (zero padded); FP32, the paired
//                 layout (apply_paired_index).
//   ROWS_FORCING: f_U = f_G - (A_GO A_OO^-1) f_O, rows Gamma / columns Omega of the swept
//                 matrix (eq. subForcing);
//   ROWS_BACKSUB: u_O = -(M_OO f_O + M_OG u_G) = A_OO^-1 (f_O - A_OG u_G), rows Omega / all
//                 columns of the swept matrix (eq. backwardSubstitution).
//   For these two, x comes from FP64 subdomain vectors and is staged in shared memory in
//   chunks of ROWS_CW columns ([c][column], row stride padded by 4 against bank conflicts).
#pragma once

// needs <cuda_fp16.h> and <type_traits>, included before the enclosing namespace

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int W = 2; };

// W consecutive operator entries of type MT at p (16-byte aligned for MT = T, 8-byte for an
// FP16 copy) as the arithmetic vector of T; widening FP16 to FP32 is exact
template <typename T, typename MT>
__device__ __forceinline__ typename Vec<T>::type load_widen(const MT *p) {
    if constexpr (std::is_same<MT, T>::value) {
        return *reinterpret_cast<const typename Vec<T>::type *>(p);
    } else {
        static_assert(std::is_same<T, float>::value && std::is_same<MT, __half>::value, "FP16 copies widen to FP32");
        const uint2 raw = *reinterpret_cast<const uint2 *>(p);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&raw.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&raw.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
}
// the same from global memory, streamed (not kept in L1)
template <typename T, typename MT>
__device__ __forceinline__ typename Vec<T>::type ldcs_widen(const MT *p) {
    if constexpr (std::is_same<MT, T>::value) {
        return __ldcs(reinterpret_cast<const typename Vec<T>::type *>(p));
    } else {
        const uint2 raw = __ldcs(reinterpret_cast<const uint2 *>(p));
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&raw.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&raw.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
}

static_assert(kApplyRows == 32, "the row kernel owns 32 rows per CTA (8 warps x 4)");
constexpr int ROWS_CW = 512;      // staged columns per chunk (forcing / back substitution)

enum { ROWS_APPLY = 0, ROWS_FORCING = 1, ROWS_BACKSUB = 2 };

// store v at (U dof u, column c) of the apply layout; the thread of the last Gamma dof of a
// subdomain also zeroes the column's padding [n_gamma, ld_gamma), so that the padding never
// holds stale bits (the buffer is shared by both precisions and every column count)
// FP32 (the paired layout, apply_paired_index): only the dof's own entry is written; the
// padding of that buffer (columns past n_gamma, the missing partner of an odd R) is zeroed when
// it is allocated and never written, so it stays zero
template <typename T>
__device__ __forceinline__ void apply_store(T *x, const SubdomainDesc *sd, const int32_t *u2sub, int64_t u, int c, int R,
                                            T v) {
    const SubdomainDesc &d = sd[u2sub[u]];
    const int j = (int)(u - d.offU);
    if constexpr (std::is_same<T, float>::value) {
        x[apply_paired_index(d.offXp, d.ldG, j, c, R)] = v;
    } else {
        const int64_t col = d.offUp * R + (int64_t)c * d.ldG;
        const int nG = d.nG, ldG = d.ldG;
        x[col + j] = v;
        if (j == nG - 1)
            for (int q = nG; q < ldG; ++q) x[col + q] = T(0);
    }
}

// entries j .. j + W - 1 (j a multiple of W) of right-hand side c of subdomain d in the apply input
template <typename T>
__device__ __forceinline__ typename Vec<T>::type load_apply_x(const T *x, const SubdomainDesc &d, int j, int c, int R) {
    if constexpr (std::is_same<T, float>::value) {
        const float *p = x + apply_paired_index(d.offXp, d.ldG, j, c, R);
        return make_float4(__ldg(p), __ldg(p + 2), __ldg(p + 128), __ldg(p + 130));
    } else {
        return __ldg(reinterpret_cast<const typename Vec<T>::type *>(x + d.offUp * R + (int64_t)c * d.ldG + j));
    }
}

// NR-row x RC-column update from one step of the stream: acc[r][c] += M[r][l..l+W) . x[c][l..l+W)
// (one FMA per product in the order w = 0 .. W-1; packed FP32-pair FMAs over two columns were
// measured slower here: 128 vs 107 us per launch on the peridynamic workload)
template <typename T, int RC, typename XF, int NR = 4>
__device__ __forceinline__ void rows_step(const typename Vec<T>::type (&mv)[NR], XF &&xload, T (&acc)[NR][RC]) {
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
#pragma unroll
    for (int c = 0; c < RC; ++c) {
        V xv = xload(c);
        const T *xp = reinterpret_cast<const T *>(&xv);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const T *mp = reinterpret_cast<const T *>(&mv[r]);
#pragma unroll
            for (int w = 0; w < W; ++w) acc[r][c] += mp[w] * xp[w];
        }
    }
}

// The update of rows_step for NR rows and RC (even) right-hand sides with x in the paired layout:
// per pair row cp of the stage (512 floats: 256 columns of two right-hand sides), the lane's
// columns l .. l+3 of both right-hand sides are the float4s at xq + 512 cp and xq + 512 cp + 128
// ((x[2cp][l], x[2cp+1][l], x[2cp][l+1], x[2cp+1][l+1]) and the same for l+2, l+3), and
// acc[r][cp] holds the sums of right-hand sides 2cp and 2cp+1 as one pair.  Each element gets
// fma(m, x, acc) in the order w = 0 .. 3, as in rows_step, with one packed FMA per two
// right-hand sides: bitwise the result of rows_step.  MT: stored operator type (FP32, or an
// FP16 copy widened exactly).
template <int RC, int NR, typename MT>
__device__ __forceinline__ void rows_step_paired(const MT *mrow0, int mstride, const float *xq,
                                                 float2 (&acc)[NR][RC / 2]) {
    float4 mv[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) mv[r] = load_widen<float, MT>(mrow0 + r * mstride);
#pragma unroll
    for (int cp = 0; cp < RC / 2; ++cp) {
        const float4 xa = *reinterpret_cast<const float4 *>(xq + 512 * cp);
        const float4 xb = *reinterpret_cast<const float4 *>(xq + 512 * cp + 128);
        const float2 x0 = make_float2(xa.x, xa.y), x1 = make_float2(xa.z, xa.w);
        const float2 x2 = make_float2(xb.x, xb.y), x3 = make_float2(xb.z, xb.w);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            float2 a = acc[r][cp];
            a = __ffma2_rn(make_float2(mv[r].x, mv[r].x), x0, a);
            a = __ffma2_rn(make_float2(mv[r].y, mv[r].y), x1, a);
            a = __ffma2_rn(make_float2(mv[r].z, mv[r].z), x2, a);
            a = __ffma2_rn(make_float2(mv[r].w, mv[r].w), x3, a);
            acc[r][cp] = a;
        }
    }
}

// Warp reduce-scatter of V values per lane (V a power of two, 4 <= V <= 32): at the level
// with xor offset o the lanes with bit o set keep the upper half of their values and hand the
// lower half to their partner (the others the reverse), so each level halves the values per
// lane; once one value is left the remaining offsets add it plainly.  The additions form the
// same tree as a plain xor-shuffle sum of each value (offsets 16, 8, 4, 2, 1), so every sum
// is bitwise that of a plain per-value reduction, with V - 1 + log2(32 / V) shuffles instead
// of 5 V.  Returns the sum of value index lane / (32 / V).
template <typename T, int V>
__device__ __forceinline__ T warp_reduce_scatter(T (&v)[V], int lane) {
    static_assert(V >= 1 && V <= 32 && (V & (V - 1)) == 0, "V must be a power of two <= 32");
#pragma unroll
    for (int h = V / 2, o = 16; h >= 1; h /= 2, o /= 2) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const T send = upper ? v[i] : v[i + h];
            const T keep = upper ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    T t = v[0];
#pragma unroll
    for (int o = 16 / V; o >= 1; o /= 2) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

// MT: type of the stored operator (APPLY with the FP16 copy of S_k: __half, the result scaled by
// oscale); T otherwise.  yf (APPLY, FP32 only): the result stored in FP32 there instead of y
// (the FP32 PCG iterations; the sums are FP32 either way)
template <typename T, int RC, int MODE, typename MT = T>
__global__ void __launch_bounds__(256, 2) k_rows(const MT *base, int use_sp, const SubdomainDesc *sd, const int32_t *items,
                                                 const T *x, const double *xa, const double *xb, double *y, int R,
                                                 const int *gate, double oscale = 1.0, float *yf = nullptr) {
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    constexpr int XS = ROWS_CW + 4;
    __shared__ __align__(16) T xs[MODE == ROWS_APPLY ? 4 : RC * XS];
    if (gate && *gate == 0) return;
    const int k = items[2 * blockIdx.x], row0 = items[2 * blockIdx.x + 1];
    const SubdomainDesc d = sd[k];
    const int n = MODE == ROWS_BACKSUB ? d.nO : d.nG;                       // rows
    const int ncols = MODE == ROWS_APPLY ? d.nG : (MODE == ROWS_FORCING ? d.nO : d.nk);
    const int ld = MODE == ROWS_APPLY ? d.ldG : d.ldM;
    const int ncp = min(ld, (ncols + 7) / 8 * 8);                           // padded columns
    const int rbase = MODE == ROWS_FORCING ? d.nO : 0;                      // first matrix row
    const MT *M = base + (MODE == ROWS_APPLY ? (use_sp ? d.offSp : d.offS) : d.offM);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int ib = row0 + warp * 4;
    const MT *Mr[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) Mr[r] = M + (int64_t)(rbase + min(ib + r, n - 1)) * ld;
    for (int c0 = 0; c0 < R; c0 += RC) {
        const int rc = min(RC, R - c0);
        T acc[4][RC];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < RC; ++c) acc[r][c] = T(0);
        if constexpr (MODE == ROWS_APPLY) {
            if (ib < n) {
                int l = lane * W;
                for (; l + 32 * W < ncp; l += 64 * W) {
                    V mv[2][4];
#pragma unroll
                    for (int u = 0; u < 2; ++u)
#pragma unroll
                        for (int r = 0; r < 4; ++r) mv[u][r] = ldcs_widen<T, MT>(Mr[r] + l + u * 32 * W);
#pragma unroll
                    for (int u = 0; u < 2; ++u)
                        rows_step<T, RC>(mv[u], [&](int c) {
                            return c < rc ? load_apply_x<T>(x, d, l + u * 32 * W, c0 + c, R) : V{};
                        }, acc);
                }
                for (; l < ncp; l += 32 * W) {
                    V mv[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) mv[r] = ldcs_widen<T, MT>(Mr[r] + l);
                    rows_step<T, RC>(mv, [&](int c) { return c < rc ? load_apply_x<T>(x, d, l, c0 + c, R) : V{}; },
                                     acc);
                }
            }
        } else {
            for (int l0 = 0; l0 < ncp; l0 += ROWS_CW) {
                const int cw = min(ROWS_CW, ncp - l0);
                __syncthreads();
                for (int t = threadIdx.x; t < RC * cw; t += blockDim.x) {
                    const int l = t / RC, c = t % RC, gl = l0 + l;
                    T v = T(0);
                    if (c < rc && gl < ncols) {
                        if (MODE == ROWS_FORCING || gl < d.nO) v = (T)xa[(d.offV + gl) * R + c0 + c];
                        else v = (T)xb[(d.offU + gl - d.nO) * R + c0 + c];
                    }
                    xs[c * XS + l] = v;
                }
                __syncthreads();
                if (ib < n) {
                    for (int l = lane * W; l < cw; l += 32 * W) {
                        V mv[4];
#pragma unroll
                        for (int r = 0; r < 4; ++r) mv[r] = ldcs_widen<T, MT>(Mr[r] + l0 + l);
                        rows_step<T, RC>(mv, [&](int c) { return *reinterpret_cast<const V *>(xs + c * XS + l); },
                                         acc);
                    }
                }
            }
        }
        // reduce-scatter across the warp: afterwards the lanes with (lane % (32 / V)) == 0 hold the
        // lane sums of value index lane / (32 / V) (value r * RC + c = row r, column c)
        constexpr int V = 4 * RC;
        T v[V];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < RC; ++c) v[r * RC + c] = acc[r][c];
        const T tot = warp_reduce_scatter<T, V>(v, lane);
        constexpr int G = 32 / V;
        const int idx = lane / G, r = idx / RC, c = idx % RC;
        const int i = ib + r;
        if (lane % G == 0 && c < rc && i < n) {
            if (MODE == ROWS_APPLY && std::is_same<T, float>::value && yf)
                yf[(d.offU + i) * R + c0 + c] = (float)tot * (float)oscale;
            else if (MODE == ROWS_APPLY) y[(d.offU + i) * R + c0 + c] = (double)tot * oscale;
            else if (MODE == ROWS_FORCING)
                y[(d.offU + i) * R + c0 + c] = xa[(d.offV + d.nO + i) * R + c0 + c] - (double)tot;
            else y[(d.offV + i) * R + c0 + c] = -(double)tot;
        }
    }
}

// x (apply layout) = B^T v, or B_D^T v when val is given (CSR per U dof; B^T rows signed r+1 /
// -(r+1)); consecutive threads take consecutive U dofs of one column (coalesced stores)
// (the sums in the type L of the Lambda vectors)
template <typename T, typename L>
__global__ void k_gather_apply(const int64_t *ptr, const int64_t *row, const L *val, const L *v, T *x,
                               const SubdomainDesc *sd, const int32_t *u2sub, int64_t nu, int R, const int *gate) {
    if (gate && *gate == 0) return;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nu * R; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / nu);
        const int64_t u = t % nu;
        L s = 0;
        if (val) {
            for (int64_t q = ptr[u]; q < ptr[u + 1]; ++q) s += val[q] * v[row[q] * R + c];
        } else {
            for (int64_t q = ptr[u]; q < ptr[u + 1]; ++q) {
                const int64_t r = row[q];
                s += r > 0 ? v[(r - 1) * R + c] : -v[(-r - 1) * R + c];
            }
        }
        apply_store<T>(x, sd, u2sub, u, c, R, (T)s);
    }
}

// x (apply layout) = base - B^T v (B^T rows signed r+1 / -(r+1)), the apply input of u_G
template <typename T>
__global__ void k_gather_sub_apply(const int64_t *ptr, const int64_t *row, const double *v, const double *base, T *x,
                                   const SubdomainDesc *sd, const int32_t *u2sub, int64_t nu, int R) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nu * R; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / nu);
        const int64_t u = t % nu;
        double s = 0;
        for (int64_t q = ptr[u]; q < ptr[u + 1]; ++q) {
            const int64_t r = row[q];
            s += r > 0 ? v[(r - 1) * R + c] : -v[(-r - 1) * R + c];
        }
        apply_store<T>(x, sd, u2sub, u, c, R, (T)(base[u * R + c] - s));
    }
}

// x (apply layout) = uU (interleaved U vector) cast to T
template <typename T>
__global__ void k_to_apply(const double *uU, T *x, const SubdomainDesc *sd, const int32_t *u2sub, int64_t nu, int R) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nu * R; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / nu);
        const int64_t u = t % nu;
        apply_store<T>(x, sd, u2sub, u, c, R, (T)uU[u * R + c]);
    }
}

// u (interleaved subdomain vectors, FP64) -> FP32 pairs uh + ul in the padded layout, the
// columns taken two at a time: for subdomain k, R2 / 2 rows (R2 = R rounded up to even) at
// offVp * R2, row q holding columns 2q and 2q + 1 interleaved entry by entry (2 ld_M floats),
// zero beyond n_k and in the pad column.  Grid (K, R2).
__global__ void k_split_u(const double *u, const SubdomainDesc *sd, float *uh, float *ul, int R) {
    const SubdomainDesc d = sd[blockIdx.x];
    const int c = blockIdx.y, R2 = (R + 1) / 2 * 2;          // grid (K, R2): the pad column is zero
    for (int l = threadIdx.x; l < d.ldM; l += blockDim.x) {
        const double v = (l < d.nk && c < R) ? u[(d.offV + l) * R + c] : 0.0;
        const float h = (float)v;
        const int64_t o = d.offVp * R2 + (int64_t)(c / 2) * 2 * d.ldM + 2 * l + (c & 1);
        uh[o] = h;
        ul[o] = (float)(v - (double)h);
    }
}
