// Interface apply y_U = M x_U (M = S_k^+ or S_k on every subdomain) with the operator rows
// streamed by the bulk-copy engine.
//
// Persistent CTAs (a host-built schedule gives each CTA a list of 32-row work items, balanced
// by their cost).  The last warp is the producer: for every item of the CTA and every chunk of
// APPLY_CB bytes of columns it loads the 32 x APPLY_CB tile of the item's rows and the same
// columns of RC right-hand sides of x with two 2-D tensor copies (tensor maps per subdomain
// operator and per subdomain block of x in the apply layout; rows past n_gamma or past R
// arrive as zeros) into a ring of NS shared-memory stages, each signalled by an mbarrier
// with the byte count of its copies.  The other warps consume: with RPW rows per warp (4:
// eight consumer warps; 8: four, each x vector read from shared memory then serves 8 rows),
// warp w owns rows RPW w .. RPW w + RPW - 1 of the item, each lane 4 (FP32) or 2 (FP64)
// consecutive columns per 128-/64-column step, in the same per-lane order of operations as the
// register-streaming row kernel, so every variant gives bitwise the same y.  A consumed stage
// is released to the producer through a second mbarrier.  The producer runs ahead across item
// boundaries, so the copy engine keeps up to NS stages per CTA in flight while the consumers
// compute.
// The FP32 interface apply reads x in the paired layout (apply_paired_index: two right-hand
// sides interleaved, and each 128-column group in the order the lanes read it), one pair row
// per two right-hand sides of the stage, so that a lane's columns of two right-hand sides are
// two conflict-free 16-byte shared loads and their products are packed FMAs (fma.rn.f32x2), each
// element rounded as the scalar FMA: bitwise the sums of the scalar step, with half the FMA
// instructions (the consumers were issue-bound: the producer waited on free stages, the
// consumers about a tenth of their time on data).
// With more than RC right-hand sides the rows of an item are streamed once per block of RC.
// The operator may be stored in a narrower type MT than the arithmetic type T (FP16 copy of
// S_k for the preconditioner of the mixed path): a stage then holds the same columns with
// rows of CW * sizeof(MT) bytes, the consumers widen each 4-entry group to T before the same
// row step, and the result is multiplied by oscale (the power of two the copy was scaled by).
//
// Every wait is bounded: a wait that runs out sets *err (the workspace's error word, read by
// the host after the solve), the consumers stop, the producer waits (again bounded, with the
// default limit) for the copies it has issued and the CTA returns.  The consumers' stage waits
// take their limit from wait_tries (the problem's setting; tests make it short).
#pragma once

#include <cuda.h>

constexpr int APPLY_CB = 1024;                      // bytes of one row (or one x column) per stage
// Two CTAs per SM (18 warps): the consumers of one CTA wait on shared-memory loads and on
// their stage barrier often enough that a second CTA's warps are needed to keep the FMA
// pipes and the copy engine busy; the ring per CTA is smaller accordingly.
constexpr int APPLY_MINB = 2;                       // CTAs per SM
constexpr int APPLY_NS = 2;                         // stages per CTA (40 KB each at RC = 8)
constexpr int APPLY_NS_H = 4;                       // stages with an FP16 operator (24 KB each at RC = 8)
constexpr int APPLY_NS_H16 = 3;                     // ... at RC = 16 (32 KB each), two CTAs per SM
// right-hand sides per streamed pass: the FP32 operators stream once for up to 16 columns (the
// FP64 ones, whose accumulators take twice the registers, for up to 8)
__host__ __device__ constexpr int apply_rc(int R, int elem_size) {
    return (R >= 16 && elem_size == 4) ? 16 : (R >= 8 ? 8 : (R >= 4 ? 4 : (R >= 2 ? 2 : 1)));
}
// a stage: 32 operator rows of mrow bytes, then the RC columns of x: RC rows of APPLY_CB bytes,
// or (paired: the FP32 interface apply) (RC + 1) / 2 pair rows of 2 APPLY_CB bytes
__host__ __device__ constexpr int apply_stage_bytes(int rc, int mrow = APPLY_CB, bool paired = false) {
    return 32 * mrow + (paired ? (rc + 1) / 2 * 2 : rc) * APPLY_CB;
}
// the ring is aligned to 1 KB inside the dynamic shared memory (tensor copies want 128 B)
__host__ __device__ constexpr int apply_smem_bytes(int rc, int ns, int mrow = APPLY_CB, bool paired = false) {
    return ns * apply_stage_bytes(rc, mrow, paired) + 1024;
}
// rows of an item per consumer warp: 4 (eight consumer warps) or 8 (four consumer warps, twice
// the accumulators per lane; each x vector loaded from shared memory serves 8 rows instead of 4)
__host__ __device__ constexpr int apply_threads(int rpw) { return (32 / rpw + 1) * 32; }
constexpr int APPLY_THREADS = apply_threads(4);     // 8 consumer warps + 1 producer warp
// stages of a one-CTA-per-SM variant: as many as fit in 200 KB, at most 8
__host__ __device__ constexpr int apply_ns_one(int rc, int mrow) {
    return (200 * 1024) / (32 * mrow + rc * APPLY_CB) < 8 ? (200 * 1024) / (32 * mrow + rc * APPLY_CB) : 8;
}
constexpr long long APPLY_WAIT_TRIES = 1ll << 24;   // bounded mbarrier waits (seconds)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// true once the phase with the given parity has completed; false when the tries run out (or,
// with an abort word, once another warp of the CTA has set it)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, long long tries = APPLY_WAIT_TRIES,
                                          const volatile int *abort_word = nullptr) {
    const uint32_t a = smem_u32(bar);
    for (long long i = 0; i < tries; ++i) {
        if (abort_word && (i & 63) == 63 && *abort_word) return false;
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 2-D tile (box of the tensor map) at coordinates (x = column, y = row) -> shared memory,
// completing on an mbarrier; x * element size must be a multiple of 16 bytes
__device__ __forceinline__ void tile_g2s(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// L2 policy of the streamed operator tiles: evicted first, so that a stream of operators larger
// than L2 does not push out the vectors the next kernels read (the Lambda and U vectors of the
// PCG, a few tens of MB, stay in L2 between the interface applies)
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// tile_g2s with an L2 cache policy for the source
__device__ __forceinline__ void tile_g2s_hint(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar,
                                              uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// tensor map of a row-major block (n rows of ld entries, 16-byte aligned rows) for tiles of
// box_rows rows x box_bytes bytes: an operator (box_rows 32) or the R columns of x of one
// subdomain in the apply layout (box_rows RC); encode: the driver's cuTensorMapEncodeTiled
template <typename Encode>
inline CUresult encode_apply_map(Encode encode, CUtensorMap *map, const void *base, int ld, int n, int elem_size,
                                 int box_rows = 32, int box_bytes = APPLY_CB) {
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * (cuuint64_t)elem_size};
    const cuuint32_t box[2] = {(cuuint32_t)(box_bytes / elem_size), (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUtensorMapDataType dt = elem_size == 2   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                   : elem_size == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                    : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    return encode(map, dt, 2u,
                  const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

// tensor map of a block of a row-major matrix (rows of `stride` entries, 16-byte aligned; the
// block cols x rows from base) for tiles of 32 rows x APPLY_CB bytes: the sub-blocks of the
// swept matrix that the forcing and back-substitution modes stream
template <typename Encode>
inline CUresult encode_block_map(Encode encode, CUtensorMap *map, const void *base, int cols, int rows, int stride,
                                 int elem_size) {
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)stride * (cuuint64_t)elem_size};
    const cuuint32_t box[2] = {(cuuint32_t)(APPLY_CB / elem_size), 32u};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUtensorMapDataType dt = elem_size == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    return encode(map, dt, 2u, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

// rows and streamed columns of an item's operator per mode: the interface apply (S_k or S_k^+,
// n_gamma x n_gamma), the forcing (rows n_O.. of the swept matrix, columns 0..n_O-1: T_k) and
// the back substitution (rows 0..n_O-1, all n_k columns)
template <int MODE>
__device__ __forceinline__ void apply_shape(const SubdomainDesc &d, int &n, int &ncp) {
    if (MODE == ROWS_APPLY) { n = d.nG; ncp = min(d.ldG, (d.nG + 7) / 8 * 8); }
    else if (MODE == ROWS_FORCING) { n = d.nG; ncp = (d.nO + 7) / 8 * 8; }
    else { n = d.nO; ncp = min(d.ldM, (d.nk + 7) / 8 * 8); }
}

// an item's fields, loaded one item ahead (the chain schedule -> subdomain descriptor is two
// dependent global loads; issued while the previous item streams, it no longer stalls the warps
// at item boundaries)
struct ApplyItem {
    int k, i0, n, ncp;
    int64_t yoff, voff, nO;
};
template <int MODE>
__device__ __forceinline__ ApplyItem load_apply_item(const int32_t *sched_items, const SubdomainDesc *sd, int it) {
    ApplyItem a;
    a.k = sched_items[2 * it];
    a.i0 = sched_items[2 * it + 1];
    const SubdomainDesc &d = sd[a.k];
    apply_shape<MODE>(d, a.n, a.ncp);
    a.yoff = d.offU;
    a.voff = d.offV;
    a.nO = d.nO;
    return a;
}

// MODE (ROWS_APPLY, ROWS_FORCING, ROWS_BACKSUB) selects the operator block (above), the tensor
// maps (APPLY: 2 per subdomain, use_sp picks; else 1 per subdomain) and the output:
//   APPLY     y[(offU + i) R + c] = acc * oscale   (FP32 into yf instead when given, T = float);
//   FORCING   y[(offU + i) R + c] = xa[(offV + n_O + i) R + c] - acc   (reduced forcing, f_G - T_k f_O);
//   BACKSUB   y[(offV + i) R + c] = -acc                              (u_O from the swept -A_OO^-1 rows),
// the same outputs, in the same order of operations per lane, as k_rows.
template <typename T, int RC, int NS = APPLY_NS, int MINB = APPLY_MINB, typename MT = T, int MODE = ROWS_APPLY,
          int RPW = 4>
__global__ void __launch_bounds__(apply_threads(RPW), MINB)
    k_apply_tma(const CUtensorMap *maps, const CUtensorMap *xmaps, int use_sp, const SubdomainDesc *sd,
                const int32_t *sched_ptr, const int32_t *sched_items, double *y, int R, const int *gate, int *err,
                double oscale = 1.0, const double *xa = nullptr, long long wait_tries = APPLY_WAIT_TRIES,
                int withhold = 0, float *yf = nullptr) {
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    constexpr int NCW = 32 / RPW;                   // consumer warps (the producer is warp NCW)
    static_assert(RPW == 4 || RPW == 8, "4 or 8 rows per consumer warp");
    constexpr int CW = APPLY_CB / (int)sizeof(T);   // columns per stage row
    constexpr int MROW = CW * (int)sizeof(MT);      // operator bytes per stage row
    // FP32 interface apply: x in the paired layout (apply_paired_index), two right-hand sides per
    // pair row, so that the products of two right-hand sides are one packed FMA
    constexpr bool PAIRED = std::is_same<T, float>::value && MODE == ROWS_APPLY;
    constexpr bool PAIRS = PAIRED && RC >= 2;
    constexpr int STAGE = apply_stage_bytes(RC, MROW, PAIRED);
    extern __shared__ __align__(128) unsigned char ring_raw[];
    unsigned char *ring = ring_raw + ((1024u - (smem_u32(ring_raw) & 1023u)) & 1023u);
    __shared__ uint64_t full[NS], empty[NS];
    __shared__ volatile int abort_flag;
    if (gate && *gate == 0) return;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int it0 = sched_ptr[blockIdx.x], it1 = sched_ptr[blockIdx.x + 1];
    if (warp == NCW) {
        // ------------------------------------------------------------------ producer
        // withhold (fault injection for tests of the bounded waits): issue nothing, so that the
        // consumers' first stage wait runs out with no copy in flight
        if (withhold) return;
        int q = 0;
        bool ok = true;
        const uint64_t stream_policy = l2_evict_first_policy();
        ApplyItem nxt{};
        if (it0 < it1) nxt = load_apply_item<MODE>(sched_items, sd, it0);
        for (int it = it0; it < it1 && ok; ++it) {
            // descriptor fields in registers (the asm statements below clobber memory); the next
            // item's are loaded now and used one item later
            const ApplyItem cur = nxt;
            if (it + 1 < it1) nxt = load_apply_item<MODE>(sched_items, sd, it + 1);
            const int k = cur.k, i0 = cur.i0, ncp = cur.ncp;
            const CUtensorMap *map = MODE == ROWS_APPLY ? maps + 2 * k + use_sp : maps + k, *xmap = xmaps + k;
            for (int c0 = 0; c0 < R && ok; c0 += RC)        // the rows again for every column block
            for (int l0 = 0; l0 < ncp; l0 += CW, ++q) {
                const int s = q % NS;
                // warp-uniform decisions: every lane takes the same branch
                if (__any_sync(0xffffffffu,
                               (q >= NS && !mbar_wait(&empty[s], ((q / NS) - 1) & 1, APPLY_WAIT_TRIES, &abort_flag)) ||
                                   abort_flag)) {
                    ok = false;
                    break;
                }
                // the tiles always land whole (out-of-range rows and columns as zeros)
                if (lane == 0) {
                    unsigned char *stg = ring + s * STAGE;
                    mbar_arrive_expect_tx(&full[s], STAGE);
                    tile_g2s_hint(stg, map, l0, i0, &full[s], stream_policy);
                    tile_g2s(stg + 32 * MROW, xmap, l0, PAIRED ? c0 / 2 : c0, &full[s]);
                }
                __syncwarp();
            }
        }
        if (!ok) {
            if (lane == 0) { atomicExch(err, 1); abort_flag = 1; }
            // let the copies already issued land before the CTA leaves
            for (int t = max(0, q - NS); t < q; ++t) mbar_wait(&full[t % NS], (t / NS) & 1);
        }
        return;
    }
    // ---------------------------------------------------------------------- consumers
    int q = 0;
    ApplyItem nxt{};
    if (it0 < it1) nxt = load_apply_item<MODE>(sched_items, sd, it0);
    for (int it = it0; it < it1; ++it) {
        const ApplyItem cur = nxt;
        if (it + 1 < it1) nxt = load_apply_item<MODE>(sched_items, sd, it + 1);
        const int i0 = cur.i0, n = cur.n, ncp = cur.ncp;
        const int64_t yoff = cur.yoff, voff = cur.voff, nO = cur.nO;
        const int ib = i0 + warp * RPW;
        for (int c0 = 0; c0 < R; c0 += RC) {
            const int rc = min(RC, R - c0);
            T acc[RPW][PAIRS ? 1 : RC];
            float2 acc2[RPW][PAIRS ? RC / 2 : 1];
#pragma unroll
            for (int r = 0; r < RPW; ++r) {
#pragma unroll
                for (int c = 0; c < (PAIRS ? 1 : RC); ++c) acc[r][c] = T(0);
#pragma unroll
                for (int c = 0; c < (PAIRS ? RC / 2 : 1); ++c) acc2[r][c] = make_float2(0.f, 0.f);
            }
            for (int l0 = 0; l0 < ncp; l0 += CW, ++q) {
                const int s = q % NS;
                if (__any_sync(0xffffffffu, !mbar_wait(&full[s], (q / NS) & 1, wait_tries, &abort_flag) || abort_flag)) {
                    if (lane == 0) { atomicExch(err, 1); abort_flag = 1; }
                    return;                           // the whole warp (the vote is uniform)
                }
                const MT *st = reinterpret_cast<const MT *>(ring + s * STAGE);
                const T *xs = reinterpret_cast<const T *>(ring + s * STAGE + 32 * MROW);
                // the tiles land whole, with zeros past n_gamma, ld_gamma and R (and the operator's
                // padding columns and x's padding are zero), so every lane runs the full stage
                // without bounds tests: the extra products are exact zeros and the rows and
                // columns past the operator are never stored
                if (ib < n) {
#pragma unroll
                    for (int j = 0; j < CW / (32 * W); ++j) {
                        const int l = lane * W + j * 32 * W;
                        if constexpr (PAIRS) {
                            // the lane's float4s of each pair row: j * 256 + 4 lane and 128 further
                            rows_step_paired<RC, RPW, MT>(st + (warp * RPW) * CW + l, CW,
                                                          reinterpret_cast<const float *>(xs) + j * 256 + lane * 4,
                                                          acc2);
                        } else {
                            V mv[RPW];
#pragma unroll
                            for (int r = 0; r < RPW; ++r) mv[r] = load_widen<T, MT>(st + (warp * RPW + r) * CW + l);
                            if constexpr (PAIRED) {
                                // one right-hand side: its slot of the pair row
                                const float *q = reinterpret_cast<const float *>(xs) + j * 256 + lane * 4 + (c0 & 1);
                                const V xv = make_float4(q[0], q[2], q[128], q[130]);
                                rows_step<T, RC>(mv, [&](int) { return xv; }, acc);
                            } else {
                                rows_step<T, RC>(mv, [&](int c) { return *reinterpret_cast<const V *>(xs + c * CW + l); },
                                                 acc);
                            }
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
            }
            // lane sums by reduce-scatter in groups of 4 rows and at most 8 columns (4 x 8 = 32
            // values, one per lane): every sum takes the same shuffle tree whatever RC and RPW are
            constexpr int CG = RC < 8 ? RC : 8;
#pragma unroll
            for (int rh = 0; rh < RPW; rh += 4)
#pragma unroll
            for (int g0 = 0; g0 < RC; g0 += CG) {
                constexpr int NV = 4 * CG;
                T v[NV];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < CG; ++c) {
                        if constexpr (PAIRS) {
                            const float2 a2 = acc2[rh + r][(g0 + c) / 2];
                            v[r * CG + c] = ((g0 + c) & 1) ? a2.y : a2.x;
                        } else {
                            v[r * CG + c] = acc[rh + r][g0 + c];
                        }
                    }
                const T tot = warp_reduce_scatter<T, NV>(v, lane);
                constexpr int G = 32 / NV;
                const int idx = lane / G, r = idx / CG, c = g0 + idx % CG, i = ib + rh + r;
                if (lane % G == 0 && c < rc && i < n) {
                    if (MODE == ROWS_APPLY && std::is_same<T, float>::value && yf)
                        yf[(yoff + i) * R + c0 + c] = (float)tot * (float)oscale;
                    else if (MODE == ROWS_APPLY) y[(yoff + i) * R + c0 + c] = (double)tot * oscale;
                    else if (MODE == ROWS_FORCING)
                        y[(yoff + i) * R + c0 + c] = xa[(voff + nO + i) * R + c0 + c] - (double)tot;
                    else y[(voff + i) * R + c0 + c] = -(double)tot;
                }
            }
        }
    }
}
