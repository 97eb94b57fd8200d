// nlfeti_apply_schur_noalloc: the interface apply (S_k^+ or S_k on every subdomain) for
// callers that cannot allocate device memory during the call.
//
// Who needs it: code that runs under a fixed device-memory plan (a serving loop whose pool
// is sized and frozen after warm-up, a framework that forbids allocations between its own
// planned ones, or a caller whose allocator would synchronise the device).  The other entry
// points size their workspaces on first use through the context's allocator; this one uses
// no cudaMalloc, cudaFree, allocator callback or allocating library routine.  It stages its
// input in the scratch array below, which belongs to the library's device image, and reads the
// operators already resident in the problem (factored before).
//
// The scratch: kNoallocScratchBytes (8 MiB) per device.  A call needs n_up * nrhs * sizeof(T)
// bytes of it (n_up = sum_k ld_gamma,k, T = double for precision 0, float for 1); larger
// requests are rejected with NLFETI_E_INVALID before anything is launched.  Every call on a
// device shares the one array, so calls that overlap in time (other host threads, other
// streams) race and must be serialised by the caller.  Nothing in it has to start at zero:
// every call writes each entry it reads, the zero padding included.
//
// Set-up: the first call on a device, with that device current, resolves the array's address
// with cudaGetSymbolAddress (once per device, under a lock) and every later call reuses it.
// A caller that captures streams should make that first call before capturing.  A call made
// with another device current than the one the problem's context was created on is rejected
// (NLFETI_E_INVALID): its operators live on that device.  The resolved address stays valid for
// the life of the process's primary context on the device; a caller that resets the device
// (cudaDeviceReset) has destroyed its problems with it and does not call this again.
#include <mutex>
#include <string>
#include <type_traits>

#include <cuda_fp16.h>

#include "internal.hpp"

constexpr size_t kNoallocScratchBytes = NLFETI_NOALLOC_SCRATCH_BYTES;

// the scratch of nlfeti_apply_schur_noalloc (one per device, part of the library image)
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace nlf {
namespace {

#include "rows.cuh"

constexpr int kMaxDevices = 64;

std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// address of the scratch array on the problem's device, which must be the current one (resolved
// once per device)
void *scratch_for_device(const nlfeti_problem *p) {
    int dev = 0;
    NLF_CUDA(cudaGetDevice(&dev));
    if (dev != p->ctx->device)
        fail(NLFETI_E_INVALID, "the no-allocation apply must be called with the problem's device current (device " +
                                   std::to_string(p->ctx->device) + ", current " + std::to_string(dev) + ")");
    if (dev < 0 || dev >= kMaxDevices) fail(NLFETI_E_INVALID, "device ordinal out of range for the no-allocation apply");
    std::lock_guard<std::mutex> g(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            fail(NLFETI_E_CUDA, std::string("cudaGetSymbolAddress of the no-allocation scratch failed: ") +
                                    cudaGetErrorString(e));
        }
        g_scratch_ptr[dev] = ptr;
    }
    return g_scratch_ptr[dev];
}

// column-major input (n_u x R, FP64) -> the apply layout in the scratch (R columns of ld_gamma
// entries per subdomain at offUp * R, padding zeroed), converted to T
template <typename T>
__global__ void k_stage_colmajor(const double *in, T *x, const SubdomainDesc *sd, const int32_t *u2sub, int64_t nu,
                                 int R) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nu * R; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / nu);
        const int64_t u = t % nu;
        const SubdomainDesc &d = sd[u2sub[u]];
        const int64_t col = d.offUp * R + (int64_t)c * d.ldG;
        const int j = (int)(u - d.offU);
        x[col + j] = (T)in[t];
        if (j == d.nG - 1)
            for (int q = d.nG; q < d.ldG; ++q) x[col + q] = T(0);
    }
}

// The register-streaming interface apply (k_rows in apply mode) with its input read from the
// scratch and its output written column-major (n_u x R) into the caller's array.  Work item =
// (subdomain k, 32 rows); warp w owns rows 4w..4w+3, each lane streams 4 (FP32) or 2 (FP64)
// consecutive columns per step, sums per lane in T, then a warp reduce-scatter.
template <typename T, int RC>
__global__ void __launch_bounds__(256, 2) k_apply_colmajor(const T *base, int use_sp, const SubdomainDesc *sd,
                                                           const int32_t *items, const T *x, double *y, int64_t nu,
                                                           int R) {
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    const int k = items[2 * blockIdx.x], row0 = items[2 * blockIdx.x + 1];
    const SubdomainDesc d = sd[k];
    const int n = d.nG, ld = d.ldG;
    const int ncp = min(ld, (n + 7) / 8 * 8);
    const T *M = base + (use_sp ? d.offSp : d.offS);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int ib = row0 + warp * 4;
    const T *Mr[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) Mr[r] = M + (int64_t)min(ib + r, n - 1) * ld;
    for (int c0 = 0; c0 < R; c0 += RC) {
        const int rc = min(RC, R - c0);
        const T *xk = x + d.offUp * R + (int64_t)c0 * ld;
        T acc[4][RC];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < RC; ++c) acc[r][c] = T(0);
        if (ib < n) {
            for (int l = lane * W; l < ncp; l += 32 * W) {
                V mv[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) mv[r] = __ldcs(reinterpret_cast<const V *>(Mr[r] + l));
                rows_step<T, RC>(mv, [&](int c) {
                    return c < rc ? __ldg(reinterpret_cast<const V *>(xk + (int64_t)c * ld + l)) : V{};
                }, acc);
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
        const int idx = lane / G, r = idx / RC, c = idx % RC, i = ib + r;
        if (lane % G == 0 && c < rc && i < n) y[(int64_t)(c0 + c) * nu + d.offU + i] = (double)tot;
    }
}

template <typename T>
void apply_noalloc(nlfeti_problem *p, const OpPool<T> &pool, int use_sp, int R, const double *d_in, double *d_out,
                   void *scratch) {
    cudaStream_t st = p->ctx->stream;
    const int64_t nu = p->n_u;
    T *x = static_cast<T *>(scratch);
    const int64_t blocks = std::min<int64_t>((nu * R + 255) / 256, 152 * 16);
    k_stage_colmajor<T><<<(unsigned)std::max<int64_t>(1, blocks), 256, 0, st>>>(
        d_in, x, p->d_sd.as<SubdomainDesc>(), p->d_u2sub.as<int32_t>(), nu, R);
    const T *base = use_sp ? pool.Sp.template as<T>() : pool.S.template as<T>();
    auto go = [&](auto rc_tag) {
        constexpr int RC = decltype(rc_tag)::value;
        k_apply_colmajor<T, RC><<<p->n_items, 256, 0, st>>>(base, use_sp, p->d_sd.as<SubdomainDesc>(),
                                                            p->d_items.as<int32_t>(), x, d_out, nu, R);
    };
    if (R >= 8) go(std::integral_constant<int, 8>{});
    else if (R >= 4) go(std::integral_constant<int, 4>{});
    else if (R >= 2) go(std::integral_constant<int, 2>{});
    else go(std::integral_constant<int, 1>{});
    NLF_CUDA(cudaGetLastError());
}

}  // namespace
}  // namespace nlf

using namespace nlf;

extern "C" nlfeti_status nlfeti_apply_schur_noalloc(nlfeti_problem *p, int which, int precision, int nrhs,
                                                    const double *d_in, double *d_out) {
    if (!p) return NLFETI_E_INVALID;
    try {
        if ((which != 0 && which != 1) || (precision != 0 && precision != 1) || nrhs < 1 || !d_in || !d_out)
            fail(NLFETI_E_INVALID, "bad no-allocation apply arguments");
        const size_t elem = precision == 0 ? sizeof(double) : sizeof(float);
        const size_t need = (size_t)std::max<int64_t>(p->n_up, 1) * (size_t)nrhs * elem;
        if (need > kNoallocScratchBytes)
            fail(NLFETI_E_INVALID, "the no-allocation apply needs " + std::to_string(need) +
                                       " bytes of scratch for this problem and nrhs; it holds " +
                                       std::to_string(kNoallocScratchBytes) + " bytes (use fewer right-hand sides "
                                       "per call, or nlfeti_apply)");
        if ((precision == 0 && !p->op64.ready) || (precision == 1 && !p->op32.ready))
            fail(NLFETI_E_INVALID, "operators of the requested precision are not factored");
        if (p->n_u == 0 || p->n_items == 0) return NLFETI_OK;
        void *scratch = scratch_for_device(p);
        stream_enter(p->ctx);
        try {
            if (precision == 0) apply_noalloc<double>(p, p->op64, which == 0 ? 1 : 0, nrhs, d_in, d_out, scratch);
            else apply_noalloc<float>(p, p->op32, which == 0 ? 1 : 0, nrhs, d_in, d_out, scratch);
        } catch (...) {
            stream_leave(p->ctx);
            throw;
        }
        stream_leave(p->ctx);
        return NLFETI_OK;
    } catch (const Error &e) {
        set_error(p->ctx, e.msg);
        return e.st;
    } catch (const std::exception &e) {
        set_error(p->ctx, e.what());
        return NLFETI_E_INVALID;
    }
}
