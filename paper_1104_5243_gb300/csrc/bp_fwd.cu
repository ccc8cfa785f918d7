// Voxel-driven cone-beam backprojection kernel (Sect. 3.1, Listing 1) for
// sm_103a.
//
// For every voxel x and projection i:  (uw, vw, w) = A_i (x, 1),
// u = uw / w, v = vw / w, VOL[x] += bilinear(I_i, u, v) / w^2, with pixels
// outside the detector reading zero.
//
// GPU mapping (what differs from the paper's SSE/AVX line kernel):
//  * Part 2 of the listing (the four scattered corner loads, the bottleneck
//    of every SIMD variant in Sect. 4) is ONE texture gather per update: the
//    image lives in a block-linear CUDA array, tex2Dgather returns the 2x2
//    neighbourhood, and the border address mode supplies the zero padding of
//    Sect. 3.3 without masks.  Interpolation weights are computed in float32
//    here, never by the texture unit's reduced-precision filter.
//  * The gather coordinate is the exact integer floor(u)+1: with texel
//    centres at j + 0.5 the 2x2 footprint is then texels floor(u), floor(u)+1
//    with no rounding in the selection.  The host folds an integer centring
//    offset and the +1 into the matrix in float64, so the kernel works with
//    u' = u - ku + 1, a small number whose float32 rounding error is a
//    fraction of that of u itself, and gathers at floor(u') + ku.
//  * One reciprocal per update (Sect. 3.3); the weight 1/w^2 is r*r.
//  * A thread keeps 4 voxels' sums in registers over the whole batch of
//    projections (the b-way image blocking of Sect. 6.2 with b = the batch
//    size): the volume is read and written once per batch.  The 32 lanes of
//    a warp take neighbouring voxels (LX along x by 32/LX along z) so one
//    gather instruction touches a compact detector patch; each lane's 4
//    voxels are LX apart along x, and every volume access of the warp covers
//    whole 32-byte sectors.
//  * The matrices and texture handles of the batch are kernel parameters,
//    read through the constant cache with a warp-uniform index.
//  * Brick culling (the line-wise clipping of Sect. 3.3 at block
//    granularity): a pre-pass marks, per thread block, the projections whose
//    footprint can reach the block's voxels; the others are skipped with a
//    block-uniform branch.  Skipped terms are exactly zero, so culling does
//    not change a single bit of the volume.
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "bp_internal.cuh"

namespace bp {

template <bool IEEE>
__device__ __forceinline__ float recip(float w)
{
    if constexpr (IEEE) {
        return __frcp_rn(w);
    } else {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(w));
        return r;
    }
}

// 2x2 neighbourhood at exact integer texture coordinate (x, y):
// returns (bl, br, tr, tl) in (.x, .y, .z, .w) -- texels (i0, j1), (i1, j1),
// (i1, j0), (i0, j0) with i0 = x - 1, j0 = y - 1.
template <int KIND>
__device__ __forceinline__ float4 gather(cudaTextureObject_t t, float x, float y)
{
    if constexpr (KIND == kTexFloat) {
        return tex2Dgather<float4>(t, x, y, 0);
    } else {
        uint4 q = tex2Dgather<uint4>(t, x, y, 0);   // raw BF16 bits, zero-extended
        return make_float4(__uint_as_float(q.x << 16), __uint_as_float(q.y << 16),
                           __uint_as_float(q.z << 16), __uint_as_float(q.w << 16));
    }
}

template <int KIND, bool IEEE, int LX, int LY, int VPL>
__global__ void __launch_bounds__(kThreads, VPL == 4 ? 6 : 4)
bp_fwd_kernel(const __grid_constant__ FwdBatch b, float *__restrict__ vol, const VolGeom g,
              int accumulate, const unsigned long long *__restrict__ masks)
{
    constexpr int LZ = 32 / (LX * LY);          // lanes along z
    constexpr int TX = LX * VPL;                // x extent of the block tile
    const int lane = threadIdx.x & 31;
    const int tx = lane % LX, ty = (lane / LX) % LY, tz = lane / (LX * LY);
    const int L = g.L;
    const int xb = blockIdx.x * TX + tx;        // this lane's voxels: xb + LX k
    const int y = (blockIdx.y * kWarpsY + (threadIdx.x >> 5)) * LY + ty;
    const int z = blockIdx.z * LZ + tz;
    if (y >= L || z >= L)
        return;

    float X[VPL];
#pragma unroll
    for (int k = 0; k < VPL; ++k)
        X[k] = fmaf(g.R, (float)(xb + LX * k), g.Ox);
    const float Y = fmaf(g.R, (float)y, g.Oy);
    const float Z = fmaf(g.R, (float)z, g.Oz);

    float acc[VPL];
#pragma unroll
    for (int k = 0; k < VPL; ++k)
        acc[k] = 0.f;
    // projections that can reach this block (all of them without culling)
    const unsigned long long visible =
        masks ? masks[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] : ~0ull;
#pragma unroll 1
    for (int i = 0; i < b.n; ++i) {
        if (!((visible >> i) & 1ull))
            continue;   // every term of this projection is exactly zero here
        const float4 ru = b.m[i][0], rv = b.m[i][1], rw = b.m[i][2];
        const float2 kc = b.k[i];
        const cudaTextureObject_t t = b.tex[i];
        // Part 1: geometry; the y, z terms are shared by the lane's voxels.
        const float bu = fmaf(ru.y, Y, fmaf(ru.z, Z, ru.w));
        const float bv = fmaf(rv.y, Y, fmaf(rv.z, Z, rv.w));
        const float bw = fmaf(rw.y, Y, fmaf(rw.z, Z, rw.w));
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            const float uw = fmaf(ru.x, X[k], bu);
            const float vw = fmaf(rv.x, X[k], bv);
            const float w = fmaf(rw.x, X[k], bw);
            const float r = recip<IEEE>(w);
            const float u = uw * r, v = vw * r;       // centred: u - ku + 1
            const float fu0 = floorf(u), fv0 = floorf(v);
            // Part 2: the four corners in one gather at floor(u) + 1.
            const float4 q = gather<KIND>(t, fu0 + kc.x, fv0 + kc.y);
            // Part 3: bilinear interpolation and the 1/w^2 weight.
            const float fu = u - fu0, fv = v - fv0;
            const float top = fmaf(fu, q.z - q.w, q.w);
            const float bot = fmaf(fu, q.y - q.x, q.x);
            const float fx = fmaf(fv, bot - top, top);
            acc[k] = fmaf(fx, r * r, acc[k]);
        }
    }

    float *row = vol + ((size_t)z * L + y) * L;
#pragma unroll
    for (int k = 0; k < VPL; ++k) {
        const int x = xb + LX * k;
        if (x < L)
            row[x] = (accumulate ? row[x] : 0.f) + acc[k];
    }
}

// Block tile of a layout: (TX, TY, TZ) voxels.
static void layout_tile(int lanes_x, int *tx, int *ty, int *tz)
{
    int lx = 8, ly = 1, vpl = kVoxPerLane;
    switch (lanes_x) {
    case 108: vpl = 8; break;
    case 32: lx = 32; break;
    case 16: lx = 16; break;
    case 44: lx = 4; ly = 4; break;
    case 42: lx = 4; ly = 2; break;
    case 82: lx = 8; ly = 2; break;
    case 24: lx = 2; ly = 4; break;
    default: break;
    }
    *tx = lx * vpl;
    *ty = kWarpsY * ly;
    *tz = 32 / (lx * ly);
}

long long fwd_blocks(int L, int lanes_x)
{
    int tx, ty, tz;
    layout_tile(lanes_x, &tx, &ty, &tz);
    return (long long)((L + tx - 1) / tx) * ((L + ty - 1) / ty) * ((L + tz - 1) / tz);
}

template <int KIND, bool IEEE, int LX, int LY, int VPL = kVoxPerLane>
static cudaError_t launch_lx(const FwdBatch &b, float *vol, const VolGeom &g, bool acc,
                             const unsigned long long *masks, cudaStream_t s)
{
    constexpr int TX = LX * VPL, TY = kWarpsY * LY, LZ = 32 / (LX * LY);
    dim3 grid((g.L + TX - 1) / TX, (g.L + TY - 1) / TY, (g.L + LZ - 1) / LZ);
    bp_fwd_kernel<KIND, IEEE, LX, LY, VPL><<<grid, kThreads, 0, s>>>(b, vol, g, acc ? 1 : 0, masks);
    return cudaGetLastError();
}

// Visibility mask of one thread block of the texture kernel: project the 8
// corners of the block's voxel box (clamped to the volume) for every
// projection of the batch, with the kernel's float32 arithmetic, and keep
// the projection when the footprint, widened by one pixel, touches
// [-1, isx] x [-1, isy].  Returns the number of voxel updates it keeps.
__device__ unsigned long long block_mask(const FwdBatch &b, const VolGeom &g, int isx, int isy, int x0, int y0,
                                         int z0, int x1, int y1, int z1, unsigned long long *mask)
{
    unsigned long long m = 0;
    for (int i = 0; i < b.n; ++i) {
        const float4 ru = b.m[i][0], rv = b.m[i][1], rw = b.m[i][2];
        float umin = 3.0e38f, umax = -3.0e38f, vmin = 3.0e38f, vmax = -3.0e38f;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float X = fmaf(g.R, (float)((c & 1) ? x1 : x0), g.Ox);
            const float Y = fmaf(g.R, (float)((c & 2) ? y1 : y0), g.Oy);
            const float Z = fmaf(g.R, (float)((c & 4) ? z1 : z0), g.Oz);
            const float w = fmaf(rw.x, X, fmaf(rw.y, Y, fmaf(rw.z, Z, rw.w)));
            const float r = 1.0f / w;
            const float u = fmaf(ru.x, X, fmaf(ru.y, Y, fmaf(ru.z, Z, ru.w))) * r;
            const float v = fmaf(rv.x, X, fmaf(rv.y, Y, fmaf(rv.z, Z, rv.w))) * r;
            umin = fminf(umin, u);
            umax = fmaxf(umax, u);
            vmin = fminf(vmin, v);
            vmax = fmaxf(vmax, v);
        }
        // centred coordinates: pixel u = u' + ku - 1; keep unless the box,
        // widened by a pixel, lies entirely left of -1 or right of isx
        const float2 kc = b.k[i];
        const float pu0 = umin + kc.x - 2.f, pu1 = umax + kc.x;
        const float pv0 = vmin + kc.y - 2.f, pv1 = vmax + kc.y;
        const bool miss = pu1 < -1.f || pu0 > (float)isx || pv1 < -1.f || pv0 > (float)isy;
        if (!miss)
            m |= 1ull << i;
    }
    *mask = m;
    return (unsigned long long)__popcll(m) * (x1 - x0 + 1) * (y1 - y0 + 1) * (z1 - z0 + 1);
}

// One thread per block of the texture kernel; the kept updates are summed
// per warp into the context's work counter (for the roofline).
__global__ void __launch_bounds__(256)
cull_mask_kernel(const __grid_constant__ FwdBatch b, const VolGeom g, int isx, int isy, int tx, int ty,
                 int tz, int nbx, int nby, long long nblocks, unsigned long long *__restrict__ masks,
                 unsigned long long *__restrict__ work)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long done = 0;
    if (q < nblocks) {
        const int bx = (int)(q % nbx), by = (int)((q / nbx) % nby), bz = (int)(q / ((long long)nbx * nby));
        const int x0 = bx * tx, y0 = by * ty, z0 = bz * tz;
        done = block_mask(b, g, isx, isy, x0, y0, z0, min(x0 + tx, g.L) - 1, min(y0 + ty, g.L) - 1,
                          min(z0 + tz, g.L) - 1, &masks[q]);
    }
    for (int o = 16; o > 0; o >>= 1)
        done += __shfl_down_sync(0xffffffffu, done, o);
    if ((threadIdx.x & 31) == 0 && done)
        atomicAdd(work, done);
}

cudaError_t launch_cull_masks(const FwdBatch &b, const VolGeom &g, int isx, int isy, int lanes_x,
                              unsigned long long *masks, unsigned long long *work, cudaStream_t s)
{
    int tx, ty, tz;
    layout_tile(lanes_x, &tx, &ty, &tz);
    const int nbx = (g.L + tx - 1) / tx, nby = (g.L + ty - 1) / ty;
    const long long nblocks = fwd_blocks(g.L, lanes_x);
    cull_mask_kernel<<<(unsigned)((nblocks + 255) / 256), 256, 0, s>>>(b, g, isx, isy, tx, ty, tz, nbx, nby,
                                                                      nblocks, masks, work);
    return cudaGetLastError();
}

// Warp layouts (bp_set_option BP_OPT_LANES_X): 8, 16, 32 = lanes along x
// (the rest along z); two-digit codes XY = X lanes along x by Y along y
// (the rest along z): 44, 42, 82, 24; 108 = 8 lanes along x with 8 voxels
// per lane (instead of 4).
template <int KIND, bool IEEE>
static cudaError_t launch_kind(const FwdBatch &b, float *vol, const VolGeom &g, bool acc, int layout,
                               const unsigned long long *m, cudaStream_t s)
{
    switch (layout) {
    case 32: return launch_lx<KIND, IEEE, 32, 1>(b, vol, g, acc, m, s);
    case 16: return launch_lx<KIND, IEEE, 16, 1>(b, vol, g, acc, m, s);
    case 44: return launch_lx<KIND, IEEE, 4, 4>(b, vol, g, acc, m, s);
    case 42: return launch_lx<KIND, IEEE, 4, 2>(b, vol, g, acc, m, s);
    case 82: return launch_lx<KIND, IEEE, 8, 2>(b, vol, g, acc, m, s);
    case 24: return launch_lx<KIND, IEEE, 2, 4>(b, vol, g, acc, m, s);
    case 108: return launch_lx<KIND, IEEE, 8, 1, 8>(b, vol, g, acc, m, s);
    default: return launch_lx<KIND, IEEE, 8, 1>(b, vol, g, acc, m, s);
    }
}

cudaError_t launch_bp_fwd(const FwdBatch &b, float *vol, const VolGeom &g, int tex_kind,
                          bool accumulate, bool ieee_rcp, int lanes_x, const unsigned long long *masks,
                          cudaStream_t s)
{
    if (b.n <= 0)
        return cudaSuccess;
    if (tex_kind == kTexFloat)
        return ieee_rcp ? launch_kind<kTexFloat, true>(b, vol, g, accumulate, lanes_x, masks, s)
                        : launch_kind<kTexFloat, false>(b, vol, g, accumulate, lanes_x, masks, s);
    return ieee_rcp ? launch_kind<kTexBF16, true>(b, vol, g, accumulate, lanes_x, masks, s)
                    : launch_kind<kTexBF16, false>(b, vol, g, accumulate, lanes_x, masks, s);
}

// ---------------------------------------------------------------------------
// FP32 images -> projection arrays: copied as float32 (MODE 0) or rounded to
// FP16 (1) / BF16 (2) with round-to-nearest-even, written through surfaces
// into the block-linear arrays; one thread per pixel, grid.z = image index.
template <int MODE>
__global__ void __launch_bounds__(256)
convert_kernel(const __grid_constant__ ConvBatch b, int isx, int isy)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    const int i = blockIdx.z;
    if (j >= isx || i >= b.n)
        return;
    const float f = b.src[i][(size_t)k * isx + j];
    if constexpr (MODE == 0) {
        surf2Dwrite<float>(f, b.surf[i], j * (int)sizeof(float), k);
    } else {
        const unsigned short bits = MODE == 2 ? __bfloat16_as_ushort(__float2bfloat16_rn(f))
                                              : __half_as_ushort(__float2half_rn(f));
        surf2Dwrite<unsigned short>(bits, b.surf[i], j * (int)sizeof(unsigned short), k);
    }
}

cudaError_t launch_convert(const ConvBatch &b, int isx, int isy, int mode, cudaStream_t s)
{
    if (b.n <= 0)
        return cudaSuccess;
    dim3 grid((isx + 255) / 256, isy, b.n);
    if (mode == 0)
        convert_kernel<0><<<grid, 256, 0, s>>>(b, isx, isy);
    else if (mode == 2)
        convert_kernel<2><<<grid, 256, 0, s>>>(b, isx, isy);
    else
        convert_kernel<1><<<grid, 256, 0, s>>>(b, isx, isy);
    return cudaGetLastError();
}

}  // namespace bp
