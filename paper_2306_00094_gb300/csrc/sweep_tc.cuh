// Rank-64 update of the FP32 sweeps on the fifth-generation tensor cores, split-TF32.
//
// One sweep step over a pivot block J (64 wide) updates every entry of the subdomain matrix
// outside J by M_il -= sum_s pan_is old_ls, a product of the n x 64 panels pan = M_iJ D^-1 and
// old = M_lJ (eq. splittingBlockCholesky: the Schur-complement update of the swept block), and
// writes the J rows and columns from pan and D^-1.  Here a CTA takes a 128 x 128 tile of M:
//   staging  (256 threads): rows r0.. of pan and rows c0.. of old (64 columns, zeros past n and
//            past the block width) are split into three TF32 terms x = hi + mid + lo (each the
//            remainder rounded to TF32: about 33 bits, so the split is exact for FP32 x) and
//            stored in the 128-byte-swizzled K-major layout of the MMA operands: two atoms of 32
//            columns (16 KB each: 8-row groups 1 KB apart, row r at 128 (r mod 8) in its group,
//            16-byte chunk j at position j ^ (r mod 8));
//   MMA      (one thread): tcgen05.mma kind::tf32, M = N = 128, K = 8; per K step the leading
//            product hi hi into accumulator 0 and the five next-order products (hi mid, mid hi,
//            hi lo, lo hi, mid mid; the rest lie below 2^-33 of the product) into accumulator 1,
//            both FP32 in tensor memory (128 lanes = rows, 2 x 128 columns), so that the small
//            terms are not added to the large ones inside the tensor core; committed to an
//            mbarrier.  The tensor core truncates while it accumulates, so the update carries a
//            few times the rounding error of the FP32-pipe kernel: measured, harmless in the Omega
//            sweep of A^k, but in the sweep of the pinned S_k it cost the mixed solve of the
//            2-D constant-kernel workload an extra refinement sweep (26 -> 32 PCG iterations), so
//            by default only the Omega sweep runs here;
//   epilogue (8 warps): warp w reads lanes 32 (w mod 4).. of its column half, adds the two
//            accumulators (acc0 + acc1) and stages the tile in shared memory; then the tile of M
//            is read, updated (or given the J-block values, as the SIMT kernel does) and written
//            with 16-byte accesses along the rows.
// The MMA wait is bounded: if it runs out the CTA sets the sweep's timeout word, waits once more
// (bounded) for its MMAs, frees its tensor memory and returns without writing.
#pragma once

constexpr int TC_TILE = 128;                        // tile rows and columns (MMA M and N)
constexpr int TC_THREADS = 256;
constexpr int TC_ATOM = TC_TILE * 128;              // one 128-byte K atom of 128 rows: 16 KB
constexpr int TC_OP = 2 * TC_ATOM;                  // a 128 x 64 FP32 operand: 32 KB
constexpr int TC_SMEM = 6 * TC_OP + 1024;           // A hi, mid, lo and B hi, mid, lo (+ 1 KB alignment)
constexpr int TC_TMEM_COLS = 2 * TC_TILE;           // two FP32 accumulators
constexpr int TC_CT = TC_TILE + 4;                  // row stride of the staged tile (floats)
constexpr long long TC_WAIT_TRIES = 1ll << 24;

__device__ __forceinline__ uint32_t tc_s32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// byte offset of entry (row r, column k) of a 128 x 64 operand in the swizzled layout
__device__ __forceinline__ int tc_off(int r, int k) {
    return (k >> 5) * TC_ATOM + (r >> 3) * 1024 + (r & 7) * 128 + ((((k & 31) >> 2) ^ (r & 7)) << 4) + ((k & 3) << 2);
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1 KB apart
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)2u << 61;
    return d;
}

// instruction descriptor of kind::tf32: FP32 accumulator (bits 4-5 = 1), A and B TF32 (format 2
// at bits 7-9 and 10-12), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int m, int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ bool tc_wait(uint64_t *bar, unsigned parity, long long tries) {
    const uint32_t a = tc_s32(bar);
    for (long long i = 0; i < tries; ++i) {
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

__device__ __forceinline__ void tc_load16(uint32_t taddr, float (&v)[16]) {
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

// grid (tiles per row, tiles per column, K) of the largest subdomain; TC_SMEM dynamic shared memory
__global__ void __launch_bounds__(TC_THREADS, 1) k_update_tc(SweepArgs<float> a, int *tflag) {
    constexpr uint32_t IDESC = tc_idesc_tf32(TC_TILE, TC_TILE);
    const int k = blockIdx.z;
    const int pend = a.pend[k];
    if (a.j0 >= pend) return;
    const int n = a.mdim[k];
    const int ld = a.mld[k];
    const int nt = (n + TC_TILE - 1) / TC_TILE;
    const int ti = blockIdx.y, tl = blockIdx.x;
    if (ti >= nt || tl >= nt) return;
    const int b = min(NB, pend - a.j0);
    const int j0 = a.j0, j1 = a.j0 + b;
    float *M = a.M + a.moff[k];
    const float *old = a.old + a.scr_off[k] * NB;
    const float *pan = a.pan + a.scr_off[k] * NB;
    const float *D = a.dinv + (int64_t)k * NB * NB;
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    unsigned char *sm = tc_raw + ((1024u - (tc_s32(tc_raw) & 1023u)) & 1023u);
    __shared__ uint64_t done_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int tc_fail;
    const int r0 = ti * TC_TILE, c0 = tl * TC_TILE;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    // ---- staging: three-term TF32 splits of the panels (A at 0, 1, 2 TC_OP; B at 3, 4, 5 TC_OP)
    for (int t = threadIdx.x; t < TC_TILE * (NB / 4); t += TC_THREADS) {
        const int r = t / (NB / 4), kk = (t % (NB / 4)) * 4;
        float4 pa = make_float4(0.f, 0.f, 0.f, 0.f), ob = pa;
        if (r0 + r < n) pa = *reinterpret_cast<const float4 *>(pan + (int64_t)(r0 + r) * NB + kk);
        if (c0 + r < n) ob = *reinterpret_cast<const float4 *>(old + (int64_t)(c0 + r) * NB + kk);
        float x[2][4] = {{pa.x, pa.y, pa.z, pa.w}, {ob.x, ob.y, ob.z, ob.w}};
        const int off = tc_off(r, kk);
#pragma unroll
        for (int o = 0; o < 2; ++o) {
            float hi[4], mid[4], lo[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float v = kk + e < b ? x[o][e] : 0.f;
                hi[e] = tf32_rna(v);
                const float r1 = v - hi[e];
                mid[e] = tf32_rna(r1);
                lo[e] = tf32_rna(r1 - mid[e]);
            }
            unsigned char *base = sm + 3 * o * TC_OP + off;
            *reinterpret_cast<float4 *>(base) = make_float4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<float4 *>(base + TC_OP) = make_float4(mid[0], mid[1], mid[2], mid[3]);
            *reinterpret_cast<float4 *>(base + 2 * TC_OP) = make_float4(lo[0], lo[1], lo[2], lo[3]);
        }
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_s32(&tmem_base)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        tc_fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_s32(&done_bar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the operands were written by ordinary stores: make them visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    // ---- MMAs over K = 64 in steps of 8: D0 = A_hi B_hi, D1 = the next-order products
    if (threadIdx.x == 0) {
        const uint32_t a0 = tc_s32(sm), b0 = a0 + 3 * TC_OP;
        const uint32_t d0 = tmem, d1 = tmem + TC_TILE;
#pragma unroll
        for (int ks = 0; ks < NB / 8; ++ks) {
            const uint32_t o = (uint32_t)((ks >> 2) * TC_ATOM + (ks & 3) * 32);
            const uint32_t ah = a0 + o, am = a0 + TC_OP + o, al = a0 + 2 * TC_OP + o;
            const uint32_t bh = b0 + o, bm = b0 + TC_OP + o, bl = b0 + 2 * TC_OP + o;
            tc_mma_tf32(d1, tc_desc(am), tc_desc(bm), IDESC, ks > 0 ? 1 : 0);
            tc_mma_tf32(d1, tc_desc(ah), tc_desc(bl), IDESC, 1);
            tc_mma_tf32(d1, tc_desc(al), tc_desc(bh), IDESC, 1);
            tc_mma_tf32(d1, tc_desc(ah), tc_desc(bm), IDESC, 1);
            tc_mma_tf32(d1, tc_desc(am), tc_desc(bh), IDESC, 1);
            tc_mma_tf32(d0, tc_desc(ah), tc_desc(bh), IDESC, ks > 0 ? 1 : 0);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         tc_s32(&done_bar))
                     : "memory");
    }
    const bool ok = tc_wait(&done_bar, 0, TC_WAIT_TRIES);
    if (__any_sync(0xffffffffu, !ok)) {
        if (lane == 0) {
            atomicExch(tflag, 1);
            tc_fail = 1;
        }
        tc_wait(&done_bar, 0, TC_WAIT_TRIES);           // let the MMAs finish before freeing
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- epilogue, 1: warp w reads lane quarter w mod 4 (one row per lane) of its column half
    // w / 4 from tensor memory, adds the two accumulators and stages the tile in shared memory
    // (the operand buffers, no longer read once the MMAs are done), row stride TC_CT floats
    float *ct = reinterpret_cast<float *>(sm);
    {
        const int q4 = warp & 3, hf = warp >> 2;
        const int rl = 32 * q4 + lane;
#pragma unroll 1
        for (int cc = 0; cc < TC_TILE / 2; cc += 16) {
            const int lc = hf * (TC_TILE / 2) + cc;
            float v[16], v1[16];
            tc_load16(tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)lc, v);
            tc_load16(tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(TC_TILE + lc), v1);
#pragma unroll
            for (int e = 0; e < 16; ++e) ct[rl * TC_CT + lc + e] = v[e] + v1[e];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- epilogue, 2: the tile of M read, updated and written with the columns fastest (a warp
    // covers one row of 128 columns); J rows and columns take their values from pan and D^-1
    if (!tc_fail) {
        const int c4 = (threadIdx.x % 32) * 4, rw = threadIdx.x / 32;
        constexpr int RPT = TC_TILE / (TC_THREADS / 32);          // rows per thread: 16
        const bool interior = r0 + TC_TILE <= n && c0 + TC_TILE <= n && (j1 <= r0 || j0 >= r0 + TC_TILE) &&
                              (j1 <= c0 || j0 >= c0 + TC_TILE);
        if (interior) {
            // all 16 rows of the thread in flight at once (64 KB per CTA), then the updates
            float4 m[RPT];
#pragma unroll
            for (int q = 0; q < RPT; ++q)
                m[q] = *reinterpret_cast<const float4 *>(M + (int64_t)(r0 + rw + q * (TC_THREADS / 32)) * ld + c0 + c4);
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int rr = rw + q * (TC_THREADS / 32);
                const float4 u = *reinterpret_cast<const float4 *>(ct + rr * TC_CT + c4);
                m[q].x -= u.x; m[q].y -= u.y; m[q].z -= u.z; m[q].w -= u.w;
                *reinterpret_cast<float4 *>(M + (int64_t)(r0 + rr) * ld + c0 + c4) = m[q];
            }
        }
#pragma unroll 1
        for (int rr = rw; rr < TC_TILE && !interior; rr += TC_THREADS / 32) {
            const int i = r0 + rr;
            const float4 u = *reinterpret_cast<const float4 *>(ct + rr * TC_CT + c4);
            if (i >= n) continue;
            const bool iJ = i >= j0 && i < j1;
            const float uv[4] = {u.x, u.y, u.z, u.w};
            float *row = M + (int64_t)i * ld;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int l = c0 + c4 + e;
                if (l >= n) break;
                const bool lJ = l >= j0 && l < j1;
                if (!iJ && !lJ) row[l] = row[l] - uv[e];
                else if (!iJ && lJ) row[l] = pan[(int64_t)i * NB + (l - j0)];
                else if (iJ && !lJ) row[l] = pan[(int64_t)l * NB + (i - j0)];
                else row[l] = -D[(i - j0) * NB + (l - j0)];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
}
