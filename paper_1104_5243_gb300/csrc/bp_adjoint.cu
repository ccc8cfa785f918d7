// Adjoint (transpose) of the voxel-driven backprojection: a voxel-driven
// forward projection.  For every voxel value f(x) and projection i the value
// s = f(x) / w^2 is spread onto the four pixels around (u, v) = (uw/w, vw/w)
// with the bilinear weights of Listing 1 (Sect. 3.1), dropping pixels
// outside the detector.  This is exactly B^T for the map of bp_fwd.cu, so
// <B p, f> = <p, B^T f>.
//
// Scatter with float32 atomics (red.global.add).  Threads own the same voxel
// tile as the forward kernel and work in the same centred coordinates
// (u' = u - ku with an integer ku folded into the matrix in float64).  For one
// projection the 32 lanes of a warp hit 32 neighbouring 2x2 neighbourhoods
// (neighbouring voxels land 1..5 pixels apart), so same-address conflicts
// inside a warp are rare and contention is across warps and blocks, along
// the rays.
#include "bp_internal.cuh"

namespace bp {

template <bool IEEE>
__device__ __forceinline__ float recip_adj(float w)
{
    if constexpr (IEEE) {
        return __frcp_rn(w);
    } else {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(w));
        return r;
    }
}

template <bool IEEE>
__global__ void __launch_bounds__(kThreads)
bp_adjoint_kernel(const __grid_constant__ AdjBatch b, const float *__restrict__ vol,
                  const VolGeom g, float *__restrict__ out, int isx, int isy)
{
    constexpr int LX = 8, LZ = 32 / LX, TX = LX * kVoxPerLane;
    const int lane = threadIdx.x & 31;
    const int tx = lane % LX, tz = lane / LX;
    const int L = g.L;
    const int xb = blockIdx.x * TX + tx;
    const int y = blockIdx.y * kWarpsY + (threadIdx.x >> 5);
    const int z = blockIdx.z * LZ + tz;
    if (y >= L || z >= L)
        return;

    const float *row = vol + ((size_t)z * L + y) * L;
    float f[kVoxPerLane], X[kVoxPerLane];
#pragma unroll
    for (int k = 0; k < kVoxPerLane; ++k) {
        const int x = xb + LX * k;
        f[k] = x < L ? row[x] : 0.f;
        X[k] = fmaf(g.R, (float)x, g.Ox);
    }
    const float Y = fmaf(g.R, (float)y, g.Oy);
    const float Z = fmaf(g.R, (float)z, g.Oz);

#pragma unroll 1
    for (int i = 0; i < b.n; ++i) {
        const float4 ru = b.m[i][0], rv = b.m[i][1], rw = b.m[i][2];
        const int2 kc = b.k[i];
        // bounds of the centred coordinates u' = u - ku, v' = v - kv
        const float ulo = (float)(-1 - kc.x), uhi = (float)(isx - kc.x);
        const float vlo = (float)(-1 - kc.y), vhi = (float)(isy - kc.y);
        float *img = out + b.out_off[i];
        const float bu = fmaf(ru.y, Y, fmaf(ru.z, Z, ru.w));
        const float bv = fmaf(rv.y, Y, fmaf(rv.z, Z, rv.w));
        const float bw = fmaf(rw.y, Y, fmaf(rw.z, Z, rw.w));
#pragma unroll
        for (int k = 0; k < kVoxPerLane; ++k) {
            if (f[k] == 0.f)
                continue;
            const float uw = fmaf(ru.x, X[k], bu);
            const float vw = fmaf(rv.x, X[k], bv);
            const float w = fmaf(rw.x, X[k], bw);
            const float r = recip_adj<IEEE>(w);
            const float u = uw * r, v = vw * r;
            // Every corner is outside the detector unless -1 < u < isx and
            // -1 < v < isy (this also keeps the int conversion in range).
            if (!(u > ulo && u < uhi && v > vlo && v < vhi))
                continue;
            const float fu0 = floorf(u), fv0 = floorf(v);
            const int iu = (int)fu0 + kc.x, iv = (int)fv0 + kc.y;
            const float fu = u - fu0, fv = v - fv0;
            const float s = f[k] * (r * r);
            const float sb = s * fv, st = s - sb;          // s fv, s (1 - fv)
            const float w_tr = st * fu, w_tl = st - w_tr;  // s fu (1-fv), s (1-fu)(1-fv)
            const float w_br = sb * fu, w_bl = sb - w_br;  // s fu fv, s (1-fu) fv
            const bool in_l = iu >= 0, in_r = iu + 1 < isx;
            const long long base = (long long)iv * isx + iu;
            if (iv >= 0) {
                if (in_l) atomicAdd(img + base, w_tl);
                if (in_r) atomicAdd(img + base + 1, w_tr);
            }
            if (iv + 1 < isy) {
                if (in_l) atomicAdd(img + base + isx, w_bl);
                if (in_r) atomicAdd(img + base + isx + 1, w_br);
            }
        }
    }
}

cudaError_t launch_bp_adjoint(const AdjBatch &b, const float *vol, const VolGeom &g, float *out,
                              int isx, int isy, bool ieee_rcp, cudaStream_t s)
{
    if (b.n <= 0)
        return cudaSuccess;
    constexpr int TX = 8 * kVoxPerLane, LZ = 4;
    dim3 grid((g.L + TX - 1) / TX, (g.L + kWarpsY - 1) / kWarpsY, (g.L + LZ - 1) / LZ);
    if (ieee_rcp)
        bp_adjoint_kernel<true><<<grid, kThreads, 0, s>>>(b, vol, g, out, isx, isy);
    else
        bp_adjoint_kernel<false><<<grid, kThreads, 0, s>>>(b, vol, g, out, isx, isy);
    return cudaGetLastError();
}

}  // namespace bp
