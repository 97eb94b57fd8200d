// Preconditioner apply y_U = S x_U (the S_k of the scaled Dirichlet preconditioner,
// eq. preconditioner) on the fifth-generation tensor cores.
//
// y_k = S_k x_k is a skinny product: S_k is n_gamma x n_gamma and x_k holds R <= 64 columns.
// Operands in FP16: the copy of S_k scaled by the power of two hscale (largest entry in
// [2^13, 2^14)) and x scaled per column by the power of two xscale[c] (set from the column's
// norm before the apply, so that the entries lie below about 2^5 and keep 11 bits down to
// 2^-14 of the norm); products accumulated in FP32 in tensor memory; the epilogue multiplies
// by oscale / xscale[c] (oscale = 1 / hscale; exact).  The preconditioner only steers the PCG,
// so its rounding changes iteration counts, not the solution the refinement reaches.
//
// Work item: 128 rows of one S_k (M = 128, one TMEM lane per row) times all R columns of x_k
// (N = NP, R rounded up to 16; rows past R of the x tile arrive as zeros).  The K loop streams
// 64 columns per stage: the 128 x 64 tile of S_k, stored contiguously (16 KB) in the tiled
// copy already in the 128-byte swizzled K-major order and loaded by one bulk copy (one
// contiguous DRAM stream per stage instead of 128 rows of 128 bytes; on the 2-D constant-kernel
// workload with h = 1/128, 4 x 4 subdomains and 8 right-hand sides both forms measured the
// same), and the NP x 64 tile of x_k by a 2-D tensor copy with the same swizzle; 8-row atoms
// of 1 KB, stage buffers 1 KB aligned, four MMAs of K = 16 per stage.  Rows and columns past
// the operator (n_gamma, ld_gamma) are zeros in the tiles.
//
// Persistent CTAs of six warps over a host-built schedule of items (longest first onto the
// least loaded CTA):
//   warp 4      producer: one lane issues the two copies of every stage into a ring
//               of mma_ns stages (full[s]: copy bytes landed; empty[s]: MMAs done reading);
//   warp 5      owns the tensor-memory allocation; one lane issues the MMAs of an item, the
//               k-th MMA of every stage into accumulator k of MMA_ACC (each cleared by its
//               first MMA: independent chains) of the item's set (items alternate between two
//               sets, so that an item's MMAs run while the epilogue drains the one before),
//               commits every stage to empty[s] and the item to tmem_full[set];
//   warps 0..3  epilogue: wait tmem_full[set], read the MMA_ACC 128 x NP accumulators (warp w
//               reads lanes 32w..32w+31, its row of the item) and add them in order, release
//               them through tmem_empty[set], and store y[(offU + row) * R + c] for rows < n_gamma,
//               columns < R, times oscale / xscale[c] (a power of two formed once per column;
//               the FP64 pipe of this GPU runs at a small fraction of the FP32 rate, and a division
//               per entry kept it a third busy: 63.6 -> 37.8 us per apply on the peridynamic
//               workload once hoisted), applied to the exponent with integer operations; as
//               FP64 into y, or (yf given: the FP32 PCG iterations) as FP32 into yf.
//
// Every wait is bounded: a wait that runs out sets *err and the abort flag, the other roles
// stop at their next wait, outstanding copies and MMAs are waited for (bounded), and the
// tensor memory is freed before the CTA returns.
#pragma once

#include <cuda_fp16.h>

constexpr int MMA_M = 128;                           // operator rows per item (TMEM lanes)
constexpr int MMA_KB = 64;                           // FP16 columns per stage (128-byte rows)
constexpr int MMA_THREADS = 6 * 32;                  // epilogue warps 0..3, producer 4, MMA 5
constexpr int MMA_MAX_R = 64;                        // right-hand sides of one pass
constexpr int MMA_A_BYTES = MMA_M * 128;             // 16 KB operator tile
// ring stages: one CTA per SM with about 200 KB in flight (two CTAs per SM let the block
// scheduler put both on one SM while others idle when there are about as many items as SMs)
__host__ __device__ constexpr int mma_ns(int np) { return np <= 16 ? 11 : (np <= 32 ? 10 : 8); }
__host__ __device__ constexpr int mma_stage_bytes(int np) { return MMA_A_BYTES + np * 128; }
__host__ __device__ constexpr int mma_smem_bytes(int np) { return mma_ns(np) * mma_stage_bytes(np) + 1024; }
// MMA_ACC accumulators per item (the k-th MMA of every stage adds into accumulator k), so
// that no chain of dependent accumulations into one tile can set the pace of the small
// 128 x 16 x 16 MMAs (on that workload one accumulator measured the same: the copies set it)
constexpr int MMA_ACC = 4;
// two accumulator sets (items alternate between them, so that the MMAs of an item overlap the
// epilogue of the one before)
__host__ __device__ constexpr int mma_tmem_cols(int np) {
    return 2 * MMA_ACC * np <= 32 ? 32
                                  : (2 * MMA_ACC * np <= 64 ? 64
                                                            : (2 * MMA_ACC * np <= 128 ? 128
                                                                                       : (2 * MMA_ACC * np <= 256 ? 256 : 512)));
}

// N of the MMA for R right-hand sides (R <= MMA_MAX_R): 16, 32 or 64
__host__ __device__ constexpr int mma_np(int R) { return R <= 16 ? 16 : (R <= 32 ? 32 : 64); }

// tensor map of a row-major FP16 block (n rows of ld entries, 16-byte aligned rows) for tiles
// of box_rows rows x 64 columns in the 128-byte swizzled layout the MMA descriptors expect:
// an operator (box_rows 128) or the R columns of x of one subdomain (box_rows mma_np(R));
// encode: the driver's cuTensorMapEncodeTiled
template <typename Encode>
inline CUresult encode_mma_map(Encode encode, CUtensorMap *map, const void *base, int ld, int n, int box_rows) {
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2u};
    const cuuint32_t box[2] = {(cuuint32_t)MMA_KB, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1u, 1u};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2u, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1 KB apart
// (start address and stride byte offset in 16-byte units; leading byte offset unused by the
// swizzled K-major layout, set to 1; descriptor version 1; layout type 2 = 128-byte swizzle)
__device__ __forceinline__ uint64_t mma_smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)2u << 61;
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B FP16
// (bits 7-9 and 10-12 = 0), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t mma_idesc_f16(int m, int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D (+)= A B with A, B from shared-memory descriptors, D in tensor memory
__device__ __forceinline__ void tc_mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

// arrive (once) on the mbarrier when every tcgen05 operation issued so far by this thread is done
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 lanes x 16 columns of 32 bits from tensor memory (lane quarter of the calling warp)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 1-D bulk copy global -> shared memory completing on an mbarrier (16-byte aligned, bytes a
// multiple of 16), with an L2 cache policy for the source
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, unsigned bytes, uint64_t *bar,
                                              uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// 1-D bulk copy global -> shared memory completing on an mbarrier (16-byte aligned, bytes a
// multiple of 16)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// v * 2^e as a double (fac = 2^e), exactly: the double's bits composed with integer
// operations for a normal v whose scaled exponent stays in range; otherwise (zero, subnormal,
// inf, nan, out of range) by the FP64 product.  The same bits as (double)v * fac either way.
__device__ __forceinline__ double f2d_pow2(float v, int e, double fac) {
    const uint32_t b = __float_as_uint(v);
    const int ex = (int)((b >> 23) & 0xffu);
    const int de = ex - 127 + 1023 + e;
    if (ex == 0 || ex == 0xff || de <= 0 || de >= 2047) return (double)v * fac;
    const uint64_t d = ((uint64_t)(b >> 31) << 63) | ((uint64_t)de << 52) | ((uint64_t)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}

// v * 2^e as a float, exactly while the result is a normal float (the exponent field set with
// integer operations); otherwise ldexpf
__device__ __forceinline__ float f2f_pow2(float v, int e) {
    const uint32_t b = __float_as_uint(v);
    const int ex = (int)((b >> 23) & 0xffu);
    const int de = ex + e;
    if (ex == 0 || ex == 0xff || de <= 0 || de >= 255) return ldexpf(v, e);
    return __uint_as_float((b & 0x807fffffu) | ((uint32_t)de << 23));
}

// yf: the result stored in FP32 there instead of y (the FP32 PCG iterations)
template <int NP>
__global__ void __launch_bounds__(MMA_THREADS, 1)
    k_apply_mma(const __half *St, const CUtensorMap *xmaps, const SubdomainDesc *sd, const int32_t *sched_ptr,
                const int32_t *sched_items, double *y, int R, const int *gate, int *err, double oscale,
                const double *xscale, float *yf = nullptr) {
    static_assert(NP % 16 == 0 && NP >= 16 && NP <= MMA_MAX_R, "N of the MMA");
    constexpr int MMA_NS = mma_ns(NP);
    constexpr int STAGE = mma_stage_bytes(NP);
    constexpr int TCOLS = mma_tmem_cols(NP);
    constexpr uint32_t IDESC = mma_idesc_f16(MMA_M, NP);
    extern __shared__ __align__(128) unsigned char mma_raw[];
    unsigned char *ring = mma_raw + ((1024u - (smem_u32(mma_raw) & 1023u)) & 1023u);
    __shared__ uint64_t full[MMA_NS], empty[MMA_NS], tmem_full[2], tmem_empty[2], drain;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    __shared__ double colfac[NP];       // oscale / xscale[c] (a power of two): formed once per column
    __shared__ int colexp[NP];          // its exponent
    if (gate && *gate == 0) return;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x < NP) {
        const double f = threadIdx.x < R ? oscale / xscale[threadIdx.x] : 0.0;
        colfac[threadIdx.x] = f;
        colexp[threadIdx.x] = f != 0.0 ? ilogb(f) : 0;
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < MMA_NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tmem_full[b], 1);
            mbar_init(&tmem_empty[b], 4 * 32);
        }
        mbar_init(&drain, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const int it0 = sched_ptr[blockIdx.x], it1 = sched_ptr[blockIdx.x + 1];
    auto fail = [&]() {
        atomicExch(err, 1);
        abort_flag = 1;
    };

    if (warp == 4) {
        // ------------------------------------------------------------------ producer
        if (lane == 0) {
            int q = 0;
            bool ok = true;
            const uint64_t stream_policy = l2_evict_first_policy();
            for (int it = it0; it < it1 && ok; ++it) {
                const int k = sched_items[2 * it], i0 = sched_items[2 * it + 1];
                const int ncp = min(sd[k].ldG, (sd[k].nG + 7) / 8 * 8);
                const int kt = mma_ktiles(sd[k].nG, sd[k].ldG);
                const __half *tiles = St + (sd[k].offT + (int64_t)(i0 / MMA_M) * kt) * (MMA_A_BYTES / 2);
                const CUtensorMap *xmap = xmaps + k;
                for (int l0 = 0; l0 < ncp; l0 += MMA_KB, ++q) {
                    const int s = q % MMA_NS;
                    if (abort_flag || (q >= MMA_NS && !mbar_wait(&empty[s], ((q / MMA_NS) - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    unsigned char *stg = ring + s * STAGE;
                    mbar_arrive_expect_tx(&full[s], STAGE);
                    bulk_g2s_hint(stg, tiles + (int64_t)(l0 / MMA_KB) * (MMA_A_BYTES / 2), MMA_A_BYTES, &full[s],
                                  stream_policy);
                    tile_g2s(stg + MMA_A_BYTES, xmap, l0, 0, &full[s]);
                }
            }
            if (!ok) {
                fail();
                for (int t = max(0, q - MMA_NS); t < q; ++t) mbar_wait(&full[t % MMA_NS], (t / MMA_NS) & 1);
            }
        }
    } else if (warp == 5) {
        // ------------------------------------------------------------------ MMA issue
        if (lane == 0) {
            int q = 0, j = 0;
            bool ok = true, issued = false;
            for (int it = it0; it < it1 && ok; ++it, ++j) {
                const int k = sched_items[2 * it];
                const int ncp = min(sd[k].ldG, (sd[k].nG + 7) / 8 * 8);
                const uint32_t acc0 = tmem + (uint32_t)((j & 1) * MMA_ACC * NP);
                if (j > 1) {
                    // accumulator set j & 1 was last used by item j - 2
                    if (abort_flag || !mbar_wait(&tmem_empty[j & 1], ((j - 2) >> 1) & 1)) { ok = false; break; }
                    tc_fence_after();
                }
                for (int l0 = 0; l0 < ncp; l0 += MMA_KB, ++q) {
                    const int s = q % MMA_NS;
                    if (abort_flag || !mbar_wait(&full[s], (q / MMA_NS) & 1)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a = smem_u32(ring + s * STAGE), b = a + MMA_A_BYTES;
                    static_assert(MMA_KB / 16 == MMA_ACC, "one accumulator per K step of a stage");
#pragma unroll
                    for (int kk = 0; kk < MMA_KB / 16; ++kk)    // K = 16 per MMA: 32 bytes along the row
                        tc_mma_f16(acc0 + (uint32_t)(kk * NP), mma_smem_desc(a + 32 * kk), mma_smem_desc(b + 32 * kk),
                                   IDESC, l0 > 0 ? 1 : 0);
                    issued = true;
                    tc_commit(&empty[s]);
                }
                if (ok) tc_commit(&tmem_full[j & 1]);
            }
            if (!ok) {
                fail();
                if (issued) {
                    tc_commit(&drain);
                    mbar_wait(&drain, 0);
                }
            }
        }
    } else {
        // ------------------------------------------------------------------ epilogue
        int j = 0;
        for (int it = it0; it < it1; ++it, ++j) {
            const int k = sched_items[2 * it], i0 = sched_items[2 * it + 1];
            bool ok = !abort_flag && mbar_wait(&tmem_full[j & 1], (j >> 1) & 1);
            if (__any_sync(0xffffffffu, !ok)) {
                if (lane == 0) fail();
                break;
            }
            tc_fence_after();
            const int n = sd[k].nG, row = i0 + 32 * warp + lane;
            const int64_t yoff = sd[k].offU;
#pragma unroll
            for (int c0 = 0; c0 < NP; c0 += 16) {
                float v[16], t[16];
                const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)((j & 1) * MMA_ACC * NP + c0);
                tc_ld16(ta, v);
#pragma unroll
                for (int a = 1; a < MMA_ACC; ++a) {
                    tc_ld16(ta + (uint32_t)(a * NP), t);
#pragma unroll
                    for (int c = 0; c < 16; ++c) v[c] += t[c];
                }
                if (row < n && yf) {
#pragma unroll
                    for (int c = 0; c < 16; ++c)
                        if (c0 + c < R) yf[(yoff + row) * R + c0 + c] = f2f_pow2(v[c], colexp[c0 + c]);
                } else if (row < n) {
#pragma unroll
                    for (int c = 0; c < 16; ++c)
                        if (c0 + c < R) y[(yoff + row) * R + c0 + c] = f2d_pow2(v[c], colexp[c0 + c], colfac[c0 + c]);
                }
            }
            tc_fence_before();
            mbar_arrive(&tmem_empty[j & 1]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    __syncwarp();
    if (warp == 5)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
}
