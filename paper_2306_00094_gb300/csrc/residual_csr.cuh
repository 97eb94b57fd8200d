// Refinement residual of the torn system (eq. discreteKKT) with FP64 accuracy on the FP32
// pipes, for sparse A^k:
//     r = f~ - A^k u - [0; B_k^T lambda]   on every subdomain.
//
// With a kernel of compact support (radius delta) the entries of A^k couple only dofs whose
// element supports interact within delta, so for a horizon of a few mesh sizes most of the
// dense n_k x n_k block is exact zeros.  The factorization then (at most an eighth of the
// entries nonzero, or when asked) keeps A^k as one CSR over the concatenated subdomain rows
// (row g = offV_k + i, columns as positions offV_k + j, entries in ascending column order),
// each entry an FP32 pair hi + lo (A^k to 2^-48 relative) with its column in one 16-byte
// record, and this kernel replaces the dense streamed one.
//
// The arithmetic per product is that of the dense kernel: p = hi*uh rounded and its exact
// error (fma), p added to a running FP32 sum by TwoSum (exact error), the errors and the cross
// terms hi*ul + lo*uh collected in a second FP32 sum, lo*ul (2^-48 relative) dropped, and the
// two sums added in FP64.  Here one lane owns one (row, column pair) and runs over the row's
// entries in order: two right-hand sides per instruction (the float2 operations, each element
// rounded as the scalar operation), no cross-lane reduction.  A warp takes 32 / LPR
// consecutive rows with LPR lanes each (LPR = column pairs per pass, a power of two up to 32).
// One 1024-thread CTA per SM walks a contiguous range of rows, 32 * 32 / LPR rows at a time, so
// that the u entries of neighbouring rows (the columns their horizons share) stay in L1 from
// one step to the next.  u is read as hi / lo FP32
// pairs with the right-hand sides of a row consecutive (k_split_u_rows); every (row, column)
// is computed by the same operations whatever the number of right-hand sides.
#pragma once

// u (interleaved subdomain vectors, FP64) -> uh + ul FP32 pairs, row g holding P = ceil(R / 2)
// float2 (columns 2q, 2q + 1), the pad column zero
__global__ void k_split_u_rows(const double *u, float2 *uh, float2 *ul, int64_t nrows, int R) {
    const int P = (R + 1) / 2;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nrows * P; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = t / P;
        const int q = (int)(t % P);
        const double a = u[g * R + 2 * q];
        const double b = 2 * q + 1 < R ? u[g * R + 2 * q + 1] : 0.0;
        const float ah = (float)a, bh = (float)b;
        uh[t] = make_float2(ah, bh);
        ul[t] = make_float2((float)(a - (double)ah), (float)(b - (double)bh));
    }
}

// one CSR entry: column position, hi, lo (as bits), unused
__device__ __forceinline__ void csr_entry(const int4 &e, int &col, float &hi, float &lo) {
    col = e.x;
    hi = __int_as_float(e.y);
    lo = __int_as_float(e.z);
}

// row_u[g]: the U index of row g (a Gamma dof) or -1 (an Omega dof)
constexpr int RES_CSR_THREADS = 1024;

template <int LPR>
__global__ void __launch_bounds__(RES_CSR_THREADS) k_residual_csr(const int64_t *__restrict__ rowptr, const int4 *__restrict__ ent,
                                                      const int32_t *__restrict__ row_u, const float2 *__restrict__ uh,
                                                      const float2 *__restrict__ ul, const double *__restrict__ f,
                                                      const int64_t *__restrict__ bt_ptr,
                                                      const int64_t *__restrict__ bt_row, const double *__restrict__ lam,
                                                      double *__restrict__ r, int64_t nrows, int R) {
    constexpr int RPW = 32 / LPR;
    const int lane = threadIdx.x & 31, sub = lane / LPR, lp = lane % LPR;
    const int P = (R + 1) / 2;
    const int64_t chunk = (nrows + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(nrows, r0 + chunk);
    const int warp = threadIdx.x / 32, nw = blockDim.x / 32;
    for (int64_t g0 = r0 + (int64_t)warp * RPW; g0 < r1; g0 += (int64_t)nw * RPW) {
        const int64_t g = g0 + sub;
        if (g >= r1) continue;
        const int64_t t0 = rowptr[g], t1 = rowptr[g + 1];
        for (int p0 = 0; p0 < P; p0 += LPR) {
            const int q = p0 + lp;
            if (q >= P) continue;
            float2 sh = make_float2(0.f, 0.f), sl = make_float2(0.f, 0.f);
#pragma unroll 4
            for (int64_t t = t0; t < t1; ++t) {
                int col;
                float ah, al;
                csr_entry(__ldg(ent + t), col, ah, al);
                const float2 xh = __ldg(uh + (int64_t)col * P + q), xl = __ldg(ul + (int64_t)col * P + q);
                // round-to-nearest pair operations (no contraction); x - y as x + (-y)
                const float2 h2 = make_float2(ah, ah), l2 = make_float2(al, al);
                const float2 pp = __fmul2_rn(h2, xh);
                const float2 pe = __ffma2_rn(h2, xh, make_float2(-pp.x, -pp.y));      // hi*uh - p exactly
                const float2 sum = __fadd2_rn(sh, pp);                                 // TwoSum(sh, p)
                const float2 bb = __fadd2_rn(sum, make_float2(-sh.x, -sh.y));
                const float2 sb = __fadd2_rn(sum, make_float2(-bb.x, -bb.y));
                const float2 se = __fadd2_rn(__fadd2_rn(sh, make_float2(-sb.x, -sb.y)),
                                             __fadd2_rn(pp, make_float2(-bb.x, -bb.y)));
                sh = sum;
                sl = __fadd2_rn(sl, __fadd2_rn(se, __ffma2_rn(h2, xl, __ffma2_rn(l2, xh, pe))));
            }
            const int u = row_u[g];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = 2 * q + h;
                if (c >= R) break;
                const double tot = h ? (double)sh.y + (double)sl.y : (double)sh.x + (double)sl.x;
                double res = f[g * R + c] - tot;
                if (u >= 0 && lam) {
                    for (int64_t t = bt_ptr[u]; t < bt_ptr[u + 1]; ++t) {
                        const int64_t rr = bt_row[t];
                        res -= rr > 0 ? lam[(rr - 1) * R + c] : -lam[(-rr - 1) * R + c];
                    }
                }
                r[g * R + c] = res;
            }
        }
    }
}
