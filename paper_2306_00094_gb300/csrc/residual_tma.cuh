// Refinement residual of the torn system (eq. discreteKKT) with FP64 accuracy on the FP32
// pipes, streamed by the tensor-copy engine:
//     r = f~ - A^k u - [0; B_k^T lambda]   on every subdomain.
//
// A^k is held as FP32 pairs (hi + lo = A^k to 2^-48 relative, swept-matrix layout) and u as
// FP32 pairs (uh + ul, k_split_u, padded layout with the right-hand sides interleaved two by
// two).  For each product a lane keeps hi*uh rounded (p) and its exact rounding error (fma),
// adds p to a running FP32 sum with TwoSum (exact error), and collects the errors and the
// cross terms hi*ul + lo*uh in a second FP32 sum; lo*ul (2^-48 relative) is dropped.  The two
// sums of each lane are added in FP64 and reduced across the warp in FP64.  Relative to
// sum_j |a_ij u_j| the result is accurate to a few 1e-13, the limit being the FP32 sum of the
// small terms over a lane's columns.  Two right-hand sides go through each step together as
// packed FP32 pairs (the float2 add / mul / fma instructions, each element rounded as the
// scalar operation: the same bits as one right-hand side at a time, with half the
// instructions): one 16-byte shared load yields the pairs of two columns.
//
// Same pipeline as k_apply_tma: persistent CTAs over a balanced schedule of 32-row items,
// warp 16 produces (per stage: 32 rows x RES_CB bytes of hi and of lo, (RC + 1) / 2 pair rows
// of 2 RES_CB bytes of uh and of ul, four 2-D tensor copies on one mbarrier), warps 0..15 consume (warp w: rows 2w, 2w + 1,
// each lane 4 consecutive columns per stage; sixteen warps, four per scheduler, hide the
// latency of the dependent TwoSum chains), bounded waits with the same error protocol.
#pragma once

constexpr int RES_CB = 512;                       // bytes of a row (or a u column) per stage
constexpr int RES_NS = 5;                         // stages
constexpr int RES_CONS = 16;                      // consumer warps (2 rows each)
constexpr int RES_THREADS = (RES_CONS + 1) * 32;
__host__ __device__ constexpr int res_pairs(int rc) { return (rc + 1) / 2; }
__host__ __device__ constexpr int res_stage_bytes(int rc) { return (64 + 4 * res_pairs(rc)) * RES_CB; }
__host__ __device__ constexpr int res_smem_bytes(int rc) { return RES_NS * res_stage_bytes(rc) + 1024; }

__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }

template <int RC>
__global__ void __launch_bounds__(RES_THREADS)
    k_residual_tma(const CUtensorMap *amaps, const CUtensorMap *umaps, const SubdomainDesc *sd,
                   const int32_t *sched_ptr, const int32_t *sched_items, const double *f, const int64_t *bt_ptr,
                   const int64_t *bt_row, const double *lam, double *r, int R, int *err) {
    constexpr int CW = RES_CB / 4;                // columns per stage (128)
    constexpr int STAGE = res_stage_bytes(RC);
    extern __shared__ __align__(128) unsigned char ring_raw[];
    unsigned char *ring = ring_raw + ((1024u - (smem_u32(ring_raw) & 1023u)) & 1023u);
    __shared__ uint64_t full[RES_NS], empty[RES_NS];
    __shared__ volatile int abort_flag;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < RES_NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], RES_CONS);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int it0 = sched_ptr[blockIdx.x], it1 = sched_ptr[blockIdx.x + 1];
    if (warp == RES_CONS) {
        // ------------------------------------------------------------------ producer
        int q = 0;
        bool ok = true;
        const uint64_t stream_policy = l2_evict_first_policy();
        for (int it = it0; it < it1 && ok; ++it) {
            const int k = sched_items[2 * it], i0 = sched_items[2 * it + 1];
            const int ld = sd[k].ldM, n = sd[k].nk;
            const int ncp = min(ld, (n + 7) / 8 * 8);
            const CUtensorMap *ahi = amaps + 2 * k, *alo = amaps + 2 * k + 1, *uhm = umaps + 2 * k,
                              *ulm = umaps + 2 * k + 1;
            for (int c0 = 0; c0 < R && ok; c0 += RC)
                for (int l0 = 0; l0 < ncp; l0 += CW, ++q) {
                    const int s = q % RES_NS;
                    // warp-uniform decisions: every lane takes the same branch
                    if (__any_sync(0xffffffffu, (q >= RES_NS && !mbar_wait(&empty[s], ((q / RES_NS) - 1) & 1)) || abort_flag)) {
                        ok = false;
                        break;
                    }
                    if (lane == 0) {
                        unsigned char *stg = ring + s * STAGE;
                        mbar_arrive_expect_tx(&full[s], STAGE);
                        tile_g2s_hint(stg, ahi, l0, i0, &full[s], stream_policy);
                        tile_g2s_hint(stg + 32 * RES_CB, alo, l0, i0, &full[s], stream_policy);
                        tile_g2s(stg + 64 * RES_CB, uhm, 2 * l0, c0 / 2, &full[s]);
                        tile_g2s(stg + (64 + 2 * res_pairs(RC)) * RES_CB, ulm, 2 * l0, c0 / 2, &full[s]);
                    }
                    __syncwarp();
                }
        }
        if (!ok) {
            if (lane == 0) { atomicExch(err, 1); abort_flag = 1; }
            for (int t = max(0, q - RES_NS); t < q; ++t) mbar_wait(&full[t % RES_NS], (t / RES_NS) & 1);
        }
        return;
    }
    // ---------------------------------------------------------------------- consumers
    int q = 0;
    for (int it = it0; it < it1; ++it) {
        const int k = sched_items[2 * it], i0 = sched_items[2 * it + 1];
        const int ld = sd[k].ldM, n = sd[k].nk, nO = sd[k].nO;
        const int64_t offV = sd[k].offV, offU = sd[k].offU;
        const int ncp = min(ld, (n + 7) / 8 * 8);
        const int ib = i0 + warp * 2;
        for (int c0 = 0; c0 < R; c0 += RC) {
            constexpr int NP2 = res_pairs(RC);
            // accumulators of rows ib, ib + 1 for the column pairs (c0 + 2q, c0 + 2q + 1)
            float2 sh[2][NP2], sl[2][NP2];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int q2 = 0; q2 < NP2; ++q2) { sh[a][q2] = make_float2(0.f, 0.f); sl[a][q2] = make_float2(0.f, 0.f); }
            for (int l0 = 0; l0 < ncp; l0 += CW, ++q) {
                const int s = q % RES_NS;
                if (__any_sync(0xffffffffu, !mbar_wait(&full[s], (q / RES_NS) & 1) || abort_flag)) {
                    if (lane == 0) { atomicExch(err, 1); abort_flag = 1; }
                    return;                           // the whole warp (the vote is uniform)
                }
                const float *st = reinterpret_cast<const float *>(ring + s * STAGE);
                const float *sth = st, *stl = st + 32 * CW;
                const float2 *xh = reinterpret_cast<const float2 *>(st + 64 * CW), *xl = xh + NP2 * CW;
                if (ib < n && l0 + lane * 4 < ncp) {
                    const int l = lane * 4;
                    float4 mh[2], ml[2];
#pragma unroll
                    for (int a = 0; a < 2; ++a) {
                        const int row = warp * 2 + a;
                        mh[a] = *reinterpret_cast<const float4 *>(sth + row * CW + l);
                        ml[a] = *reinterpret_cast<const float4 *>(stl + row * CW + l);
                    }
#pragma unroll
                    for (int q2 = 0; q2 < NP2; ++q2) {
                        // u of columns l..l+3 for the pair: (c, c + 1) per column
                        const float4 h01 = *reinterpret_cast<const float4 *>(xh + q2 * CW + l);
                        const float4 h23 = *reinterpret_cast<const float4 *>(xh + q2 * CW + l + 2);
                        const float4 l01 = *reinterpret_cast<const float4 *>(xl + q2 * CW + l);
                        const float4 l23 = *reinterpret_cast<const float4 *>(xl + q2 * CW + l + 2);
                        const float2 uh[4] = {make_float2(h01.x, h01.y), make_float2(h01.z, h01.w),
                                              make_float2(h23.x, h23.y), make_float2(h23.z, h23.w)};
                        const float2 ul[4] = {make_float2(l01.x, l01.y), make_float2(l01.z, l01.w),
                                              make_float2(l23.x, l23.y), make_float2(l23.z, l23.w)};
#pragma unroll
                        for (int a = 0; a < 2; ++a) {
                            const float ah[4] = {mh[a].x, mh[a].y, mh[a].z, mh[a].w};
                            const float al[4] = {ml[a].x, ml[a].y, ml[a].z, ml[a].w};
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                // round-to-nearest pair operations (no contraction); x - y as x + (-y)
                                const float2 h2 = make_float2(ah[e], ah[e]), l2 = make_float2(al[e], al[e]);
                                const float2 pp = __fmul2_rn(h2, uh[e]);
                                const float2 pe = __ffma2_rn(h2, uh[e], neg2(pp));          // hi*uh - p exactly
                                const float2 sum = __fadd2_rn(sh[a][q2], pp);               // TwoSum(sh, p)
                                const float2 bb = __fadd2_rn(sum, neg2(sh[a][q2]));
                                const float2 se = __fadd2_rn(__fadd2_rn(sh[a][q2], neg2(__fadd2_rn(sum, neg2(bb)))),
                                                             __fadd2_rn(pp, neg2(bb)));
                                sh[a][q2] = sum;
                                sl[a][q2] = __fadd2_rn(sl[a][q2],
                                                       __fadd2_rn(se, __ffma2_rn(h2, ul[e], __ffma2_rn(l2, uh[e], pe))));
                            }
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
            }
            const int rc = min(RC, R - c0);
            constexpr int V = 2 * RC;
            double v[V];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int c = 0; c < RC; ++c) {
                    const float2 hh = sh[a][c / 2], ll = sl[a][c / 2];
                    v[a * RC + c] = (c & 1) ? (double)hh.y + (double)ll.y : (double)hh.x + (double)ll.x;
                }
            const double tot = warp_reduce_scatter<double, V>(v, lane);
            constexpr int G = 32 / V;
            const int idx = lane / G, a = idx / RC, c = idx % RC, i = ib + a;
            if (lane % G == 0 && c < rc && i < n) {
                const int cc = c0 + c;
                double res = f[(offV + i) * R + cc] - tot;
                if (i >= nO && lam) {
                    const int64_t ui = offU + (i - nO);
                    for (int64_t t = bt_ptr[ui]; t < bt_ptr[ui + 1]; ++t) {
                        const int64_t rr = bt_row[t];
                        res -= rr > 0 ? lam[(rr - 1) * R + cc] : -lam[(-rr - 1) * R + cc];
                    }
                }
                r[(offV + i) * R + cc] = res;
            }
        }
    }
}
