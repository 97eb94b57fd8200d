// Symmetric interface apply: y_U = M x_U for M = S_k^+ or S_k, reading only the lower triangle
// of M (plus the diagonal block), i.e. the entries that determine a symmetric matrix.
//
// Work item = (subdomain k, block I of 32 rows [i0, i0 + 32)).  The item computes
//   y_I = M_{I, [0, i0+32)} x_{[0, i0+32)}          (row strip: left of and including the
//                                                   diagonal block, rows streamed by warps)
//       + M_{[i0+32, n), I}^T x_{[i0+32, n)}        (column strip below the diagonal block:
//                                                   the upper triangle by symmetry)
// Every entry strictly below the diagonal blocks is read by two items (once in a row strip,
// once in a column strip); items of one subdomain run together, so the second read hits L2
// and HBM sees each such entry once.  Each item reads 32 n entries in all, so items are even.
//
// Row strip: warp w owns rows i0 + 4w .. i0 + 4w + 3 and streams their columns with 16-byte
// loads (4 FP32 / 2 FP64 per lane), sums per lane, then a warp reduce-scatter.
// Column strip: a warp instruction covers 32 / (32 / W) rows of the 32 strip columns, each
// lane W consecutive columns of one row; rows go round-robin over the warps; the lane sums
// of the row groups are combined by xor shuffles and then across warps in shared memory in
// a fixed order.  Every sum is taken in an order that depends neither on the number of
// right-hand sides nor on a column's position among them.
//
// x sits in the apply layout: for subdomain k, R columns of ld_gamma entries at offUp * R,
// zero padded beyond n_gamma (the matrix padding columns are zero as well).
#pragma once

template <typename T, int RC>
__global__ void __launch_bounds__(256, 2) k_symm(const T *base, int use_sp, const SubdomainDesc *sd,
                                                 const int32_t *items, const T *x, double *y, int R) {
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    constexpr int CQ = 32 / W;          // lanes per strip row (32 columns)
    constexpr int RS = 32 / CQ;         // strip rows per warp instruction
    constexpr int UB = 4;               // strip steps in flight per lane
    __shared__ T partA[32][RC];
    __shared__ T partB[8][32][RC];
    const int k = items[2 * blockIdx.x], i0 = items[2 * blockIdx.x + 1];
    const SubdomainDesc d = sd[k];
    const int n = d.nG, ld = d.ldG;
    const T *M = base + (use_sp ? d.offSp : d.offS);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int ib = i0 + warp * 4;
    const int ncp = min(ld, (n + 7) / 8 * 8);
    const int cA = min(i0 + 32, ncp);                 // row strip columns [0, cA)
    const T *Mr[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) Mr[r] = M + (int64_t)min(ib + r, n - 1) * ld;
    const int rs = lane / CQ, cq = lane % CQ;
    const int j0 = i0 + 32;                           // column strip rows [j0, n)
    for (int c0 = 0; c0 < R; c0 += RC) {
        const int rc = min(RC, R - c0);
        const T *xk = x + d.offUp * R + (int64_t)c0 * ld;
        // ---------------------------------------------------------------- row strip
        {
            T acc[4][RC];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < RC; ++c) acc[r][c] = T(0);
            if (ib < n) {
                for (int l = lane * W; l < cA; l += 32 * W) {
                    V mv[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) mv[r] = __ldcs(reinterpret_cast<const V *>(Mr[r] + l));
#pragma unroll
                    for (int c = 0; c < RC; ++c) {
                        const V xv = c < rc ? __ldg(reinterpret_cast<const V *>(xk + (int64_t)c * ld + l)) : V{};
                        const T *xp = reinterpret_cast<const T *>(&xv);
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            const T *mp = reinterpret_cast<const T *>(&mv[r]);
#pragma unroll
                            for (int e = 0; e < W; ++e) acc[r][c] += mp[e] * xp[e];
                        }
                    }
                }
            }
            constexpr int NV = 4 * RC;
            T v[NV];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < RC; ++c) v[r * RC + c] = acc[r][c];
            const T tot = warp_reduce_scatter<T, NV>(v, lane);
            constexpr int G = 32 / NV;
            if (lane % G == 0) {
                const int idx = lane / G;
                partA[warp * 4 + idx / RC][idx % RC] = tot;
            }
        }
        // ---------------------------------------------------------------- column strip
        {
            T acc[W][RC];
#pragma unroll
            for (int e = 0; e < W; ++e)
#pragma unroll
                for (int c = 0; c < RC; ++c) acc[e][c] = T(0);
            const T *Mc = M + i0 + cq * W;                // column block of the strip
            // rows j = j0 + s * 8 * RS + warp * RS + rs, steps s
            for (int jb = j0 + warp * RS + rs; jb < n; jb += UB * 8 * RS) {
                V mv[UB];
                T xv[UB][RC];
#pragma unroll
                for (int u = 0; u < UB; ++u) {
                    const int j = jb + u * 8 * RS;
                    const bool ok = j < n;
                    mv[u] = ok ? __ldcs(reinterpret_cast<const V *>(Mc + (int64_t)j * ld)) : V{};
#pragma unroll
                    for (int c = 0; c < RC; ++c) xv[u][c] = (ok && c < rc) ? __ldg(xk + (int64_t)c * ld + j) : T(0);
                }
#pragma unroll
                for (int u = 0; u < UB; ++u) {
                    const T *mp = reinterpret_cast<const T *>(&mv[u]);
#pragma unroll
                    for (int e = 0; e < W; ++e)
#pragma unroll
                        for (int c = 0; c < RC; ++c) acc[e][c] += mp[e] * xv[u][c];
                }
            }
            // combine the RS row groups (lanes cq, cq + CQ, ...), fixed xor order
#pragma unroll
            for (int o = CQ; o < 32; o *= 2)
#pragma unroll
                for (int e = 0; e < W; ++e)
#pragma unroll
                    for (int c = 0; c < RC; ++c) acc[e][c] += __shfl_xor_sync(0xffffffffu, acc[e][c], o);
            if (rs == 0)
#pragma unroll
                for (int e = 0; e < W; ++e)
#pragma unroll
                    for (int c = 0; c < RC; ++c) partB[warp][cq * W + e][c] = acc[e][c];
        }
        __syncthreads();
        for (int t = threadIdx.x; t < 32 * RC; t += blockDim.x) {
            const int a = t / RC, c = t % RC, i = i0 + a;
            T s = partA[a][c];
#pragma unroll
            for (int w = 0; w < 8; ++w) s += partB[w][a][c];
            if (c < rc && i < n) y[(d.offU + i) * R + c0 + c] = (double)s;
        }
        __syncthreads();
    }
}
