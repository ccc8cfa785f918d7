// Measurement support: the texture unit's 2x2-gather throughput on this GPU,
// the speed-of-light of Part 2 of Listing 1 (Sect. 3.1) as the backprojection
// kernel performs it.  The paper derives its bounds from measured machine
// figures (Sect. 2, Table 1 update benchmark; Sect. 3.2 bounds); this is the
// GPU counterpart for the gather.
//
// Every block gathers from a small (L1-resident) patch with the kernel's warp
// shape (8 lanes along u, 4 along v, neighbouring texels) and times itself
// with the SM clock; with all blocks co-resident the per-SM rate is
// (blocks per SM * threads * gathers) / cycles.
#include <cstring>
#include <vector>

#include "bp_internal.cuh"

namespace bp {

constexpr int kProbeIters = 2048, kProbeThreads = 256, kProbeBlocksPerSM = 4, kProbeSize = 256;

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads)
gather_probe_kernel(cudaTextureObject_t t, float *__restrict__ sink, long long *__restrict__ cycles)
{
    const int lane = threadIdx.x & 31;
    const float bx = (float)(1 + (blockIdx.x % 4) * 64), by = (float)(1 + (blockIdx.x / 4 % 4) * 48);
    const int lx = lane & 7, ly = (lane >> 3) + 4 * (threadIdx.x >> 5);
    float acc = 0.f;
    const long long c0 = clock64();
    for (int i = 0; i < kProbeIters; ++i) {
        const float x = bx + (float)((lx + 3 * i) & 63);
        const float y = by + (float)((ly + i) & 31);
        if constexpr (KIND == kTexFloat) {
            const float4 q = tex2Dgather<float4>(t, x, y, 0);
            acc += (q.x + q.y) + (q.z + q.w);
        } else {
            const uint4 q = tex2Dgather<uint4>(t, x, y, 0);
            acc += (__uint_as_float(q.x << 16) + __uint_as_float(q.y << 16)) +
                   (__uint_as_float(q.z << 16) + __uint_as_float(q.w << 16));
        }
    }
    const long long c1 = clock64();
    sink[blockIdx.x * kProbeThreads + threadIdx.x] = acc;
    if (threadIdx.x == 0)
        cycles[blockIdx.x] = c1 - c0;
}

}  // namespace bp

using namespace bp;

extern "C" bp_status bp_probe_gather(bp_dtype dtype, double *gathers_per_sm_clk)
{
    if (gathers_per_sm_clk == nullptr || (dtype != BP_F32 && dtype != BP_F16 && dtype != BP_BF16)) {
        set_thread_error("bp_probe_gather: invalid argument");
        return BP_EINVAL;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaChannelFormatDesc fmt = dtype == BP_F32   ? cudaCreateChannelDesc(32, 0, 0, 0, cudaChannelFormatKindFloat)
                                : dtype == BP_F16 ? cudaCreateChannelDesc(16, 0, 0, 0, cudaChannelFormatKindFloat)
                                                  : cudaCreateChannelDesc(16, 0, 0, 0, cudaChannelFormatKindUnsigned);
    const size_t es = dtype == BP_F32 ? 4 : 2;
    cudaArray_t arr = nullptr;
    cudaTextureObject_t tex = 0;
    float *sink = nullptr;
    long long *cyc = nullptr;
    const int blocks = sms * kProbeBlocksPerSM;
    std::vector<unsigned short> host(kProbeSize * kProbeSize * es / 2);
    for (size_t q = 0; q < host.size(); ++q)
        host[q] = (unsigned short)(0x3c00 + (q * 7919 % 1021));   // finite f16 / bf16 / f32 bit patterns
    if (e == cudaSuccess)
        e = cudaMallocArray(&arr, &fmt, kProbeSize, kProbeSize);
    if (e == cudaSuccess)
        e = cudaMemcpy2DToArray(arr, 0, 0, host.data(), kProbeSize * es, kProbeSize * es, kProbeSize,
                                cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        cudaResourceDesc res;
        memset(&res, 0, sizeof res);
        res.resType = cudaResourceTypeArray;
        res.res.array.array = arr;
        cudaTextureDesc td;
        memset(&td, 0, sizeof td);
        td.addressMode[0] = td.addressMode[1] = cudaAddressModeBorder;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        e = cudaCreateTextureObject(&tex, &res, &td, nullptr);
    }
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&sink, sizeof(float) * blocks * kProbeThreads);
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&cyc, sizeof(long long) * blocks);
    double best = 0.0;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        if (dtype == BP_BF16)
            gather_probe_kernel<kTexBF16><<<blocks, kProbeThreads>>>(tex, sink, cyc);
        else
            gather_probe_kernel<kTexFloat><<<blocks, kProbeThreads>>>(tex, sink, cyc);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaDeviceSynchronize();
        std::vector<long long> c(blocks);
        if (e == cudaSuccess)
            e = cudaMemcpy(c.data(), cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) {
            double mean = 0.0;
            for (long long v : c)
                mean += (double)v;
            mean /= blocks;
            const double rate = (double)kProbeBlocksPerSM * kProbeThreads * kProbeIters / mean;
            best = rate > best ? rate : best;
        }
    }
    if (tex)
        cudaDestroyTextureObject(tex);
    if (arr)
        cudaFreeArray(arr);
    if (sink)
        cudaFree(sink);
    if (cyc)
        cudaFree(cyc);
    if (e != cudaSuccess) {
        set_thread_error("bp_probe_gather: %s", cudaGetErrorString(e));
        return BP_ECUDA;
    }
    *gathers_per_sm_clk = best;
    return BP_OK;
}
