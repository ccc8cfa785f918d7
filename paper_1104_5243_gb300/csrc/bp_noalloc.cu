// Allocation-free variant of the row-filter gradient (bp_row_filter_bwd).
//
// bp_row_filter_bwd reduces the tap gradient through a scratch buffer that it
// obtains from the stream-ordered allocator on every call.  Some callers
// cannot allow that: an acquisition or reconstruction loop that budgets all
// device memory once at start-up and must not allocate while images stream
// in, or a host framework whose own allocator owns the device and forbids
// allocations behind its back.  bp_row_filter_bwd_noalloc computes the same
// gradients with its scratch in a fixed, file-scope device array instead.
//
// The scratch (kNoAllocBlocks x kNoAllocTaps floats, 128 KiB) lives in every
// GPU that loads the library until the process exits.  In host code the
// array's name only stands for the device symbol, so its device address is
// looked up with cudaGetSymbolAddress: once per CUDA context (keyed by the
// context's unique ID, so a context created after cudaDeviceReset, or a
// non-primary context, gets its own lookup), on the first call made in that
// context.  All calls share the array, so calls whose work overlaps on the
// GPU (for example on two streams) race on it and must be serialised by the
// caller.
#include <mutex>

#include "bp_internal.cuh"

namespace bp {

constexpr int kNoAllocTaps = 128;      // largest filter the scratch serves
constexpr int kNoAllocBlocks = 256;    // persistent grid, one scratch row each
constexpr int kNoAllocRows = 4;        // rows per work item
constexpr int kNoAllocMaxContexts = 64;

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocBlocks * kNoAllocTaps];

// Same arithmetic as the regular gradient kernel, but a fixed grid of at
// most kNoAllocBlocks blocks walks the row groups (block b takes groups
// b, b + grid, ...), so each block leaves exactly one row of T partial sums
// and the scratch size does not depend on the number of rows.  Every block
// writes its whole row, so nothing has to be cleared between calls.
__global__ void __launch_bounds__(256)
row_filter_bwd_noalloc_kernel(long long rows, int isx, int T, const float *__restrict__ h,
                              const float *__restrict__ in, const float *__restrict__ g,
                              float *__restrict__ gin, float *__restrict__ partial)
{
    extern __shared__ float sm[];
    __shared__ float hs[kNoAllocTaps];
    __shared__ float red[256];
    const int pitch = isx + 2 * T;
    float *xs = sm;
    float *gs = sm + kNoAllocRows * pitch;
    for (int t = threadIdx.x; t < T; t += blockDim.x)
        hs[t] = h[t];
    const long long groups = (rows + kNoAllocRows - 1) / kNoAllocRows;
    const int ngrp = blockDim.x / T;
    const int tap = threadIdx.x % T, grp = threadIdx.x / T;
    float acc = 0.f;
    for (long long rg = blockIdx.x; rg < groups; rg += gridDim.x) {
        const long long r0 = rg * kNoAllocRows;
        __syncthreads();   // previous group's readers are done with smem
        for (int q = threadIdx.x; q < kNoAllocRows * pitch; q += blockDim.x) {
            const int rr = q / pitch, c = q % pitch - T;
            const long long r = r0 + rr;
            const bool ok = r < rows && c >= 0 && c < isx;
            xs[q] = ok ? in[r * isx + c] : 0.f;
            gs[q] = ok ? g[r * isx + c] : 0.f;
        }
        __syncthreads();
        if (gin != nullptr) {
            for (int q = threadIdx.x; q < kNoAllocRows * isx; q += blockDim.x) {
                const int rr = q / isx, s = q % isx;
                const long long r = r0 + rr;
                if (r >= rows)
                    break;
                const float *c = gs + rr * pitch + T + s + T / 2;   // c[-t] = g[s - t + T/2]
                float v = 0.f;
                for (int t = 0; t < T; ++t)
                    v = fmaf(hs[t], c[-t], v);
                gin[r * isx + s] = v;
            }
        }
        if (partial != nullptr && grp < ngrp) {
            // the group's terms summed on their own, then added to the
            // block's running sum once: the running sum then takes one term
            // per row group instead of one per product, which keeps its
            // float32 rounding at the level of the regular kernel's
            float part = 0.f;
            for (int rr = 0; rr < kNoAllocRows; ++rr) {
                const float *xr = xs + rr * pitch + T + tap - T / 2;    // xr[j] = in[j + tap - T/2]
                const float *gr = gs + rr * pitch + T;
                for (int j = grp; j < isx; j += ngrp)
                    part = fmaf(gr[j], xr[j], part);
            }
            acc += part;
        }
    }
    if (partial == nullptr)
        return;
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < T) {
        float s = 0.f;
        for (int q = 0; q < ngrp; ++q)
            s += red[q * T + threadIdx.x];
        partial[(long long)blockIdx.x * T + threadIdx.x] = s;
    }
}

// gh[t] = sum over the grid's blocks of partial[b][t], fixed order.
__global__ void __launch_bounds__(256)
reduce_noalloc_kernel(int nblk, int T, const float *__restrict__ partial, float *__restrict__ gh)
{
    __shared__ float red[256];
    const int t = blockIdx.x;
    float s = 0.f;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
        s += partial[(long long)b * T + t];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        gh[t] = red[0];
}

// Device address of g_noalloc_scratch in the current context, looked up
// once per context.  In host code the array's name only stands for the
// device symbol; only the address returned here may be handed to a kernel.
// The context is identified by cuCtxGetId (unique over the process's life,
// unlike a context handle or a device ordinal, which a context created after
// cudaDeviceReset may reuse), taken from the driver through the runtime's
// entry-point query.
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

static cudaError_t current_context_id(unsigned long long *id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(p);
    });
    if (get_current == nullptr || get_id == nullptr)
        return cudaErrorNotSupported;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS)
        return cudaErrorDeviceUninitialized;
    if (ctx == nullptr) {
        // no context on this thread yet: cudaSetDevice initialises the
        // current device's primary context and makes it current (a context
        // the caller made current is left as it is); nothing is allocated
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess)
            e = cudaSetDevice(dev);
        if (e != cudaSuccess)
            return e;
        if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr)
            return cudaErrorDeviceUninitialized;
    }
    if (get_id(ctx, id) != CUDA_SUCCESS)
        return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}

static cudaError_t noalloc_scratch(float **out)
{
    static std::mutex mu;
    static unsigned long long ids[kNoAllocMaxContexts] = {};
    static float *addr[kNoAllocMaxContexts] = {};
    static int used = 0;
    unsigned long long id = 0;
    cudaError_t e = current_context_id(&id);
    if (e != cudaSuccess)
        return e;
    std::lock_guard<std::mutex> lock(mu);
    for (int q = 0; q < used; ++q) {
        if (ids[q] == id) {
            *out = addr[q];
            return cudaSuccess;
        }
    }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
        return e;
    // the table keeps the most recent contexts; a context dropped from it
    // is looked up again on its next call
    const int slot = used < kNoAllocMaxContexts ? used++ : (int)(id % kNoAllocMaxContexts);
    ids[slot] = id;
    addr[slot] = static_cast<float *>(p);
    *out = addr[slot];
    return cudaSuccess;
}

}  // namespace bp

using namespace bp;

extern "C" bp_status bp_row_filter_bwd_noalloc(long long rows, int isx, int T, const float *h,
                                               const float *in, const float *g, float *gin,
                                               float *gh, void *stream)
{
    const size_t smem = sizeof(float) * 2 * kNoAllocRows * (size_t)(isx + 2 * (size_t)(T > 0 ? T : 0));
    if (T > kNoAllocTaps) {
        set_thread_error("bp_row_filter_bwd_noalloc: %d taps exceed the fixed scratch, which holds "
                         "%d taps x %d blocks", T, kNoAllocTaps, kNoAllocBlocks);
        return BP_EINVAL;
    }
    if (rows < 0 || isx < 1 || T < 1 || smem > 200 * 1024) {
        set_thread_error("bp_row_filter_bwd_noalloc: invalid argument (rows >= 0, isx >= 1, "
                         "1 <= T <= %d, row too long for shared memory)", kNoAllocTaps);
        return BP_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (rows == 0) {
        if (gh != nullptr) {
            cudaError_t e = cudaMemsetAsync(gh, 0, sizeof(float) * T, s);
            if (e != cudaSuccess) {
                set_thread_error("bp_row_filter_bwd_noalloc: %s", cudaGetErrorString(e));
                return BP_ECUDA;
            }
        }
        return BP_OK;
    }
    if (gin == nullptr && gh == nullptr)
        return BP_OK;
    if (h == nullptr || in == nullptr || g == nullptr) {
        set_thread_error("bp_row_filter_bwd_noalloc: NULL pointer");
        return BP_EINVAL;
    }
    float *scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e == cudaSuccess && smem > 48 * 1024)
        e = cudaFuncSetAttribute(row_filter_bwd_noalloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
    const long long groups = (rows + kNoAllocRows - 1) / kNoAllocRows;
    const int grid = groups < kNoAllocBlocks ? (int)groups : kNoAllocBlocks;
    if (e == cudaSuccess) {
        row_filter_bwd_noalloc_kernel<<<grid, 256, smem, s>>>(rows, isx, T, h, in, g, gin,
                                                             gh != nullptr ? scratch : nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && gh != nullptr) {
        reduce_noalloc_kernel<<<T, 256, 0, s>>>(grid, T, scratch, gh);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_thread_error("bp_row_filter_bwd_noalloc: %s", cudaGetErrorString(e));
        return BP_ECUDA;
    }
    return BP_OK;
}
