// Direct (one thread per voxel group, no staging) forms of the
// backprojection and of its transpose, as templates on the scalar type T.
//
// The float instantiation of direct_adjoint_kernel is the library's
// per-update-atomic adjoint (bp_adjoint with BP_OPT_CULL 0).  The double
// instantiations of both kernels are compiled only into the gradient-check
// library (csrc/check/bp_f64.cu): in float64 a finite-difference gradient
// check of B against its transpose is exact to about 1e-10, which float32
// cannot give.  Neither double instantiation is on a product path.
//
// Both follow Sect. 3.1, Listing 1: (uw, vw, w) = A_i (x, 1), u = uw / w,
// v = vw / w, the four pixels around (u, v) with bilinear weights, zero
// outside the detector (Sect. 3.3), weight 1 / w^2.  The rows are centred in
// float64 on the host: row_u' = row_u - ku row_w, so u' = u - ku and the
// pixel index is floor(u') + ku.
#pragma once

#include "bp_internal.cuh"

namespace bp {

template <typename T, bool IEEE>
__device__ __forceinline__ T direct_recip(T w)
{
    if constexpr (sizeof(T) == 8) {
        return T(1) / w;
    } else if constexpr (IEEE) {
        return __frcp_rn(w);
    } else {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(w));
        return r;
    }
}

// Adjoint (transpose) of the backprojection: a voxel-driven forward
// projection.  For every voxel value f(x) and projection i the value
// s = f(x) / w^2 is spread onto the four pixels around (u, v) with the
// bilinear weights, dropping pixels outside the detector, by atomic adds.
// Threads: 8 lanes along x by 4 along z per warp, one warp per y row of a
// 32 x 8 x 4 tile, each lane 4 voxels along x (8 apart).  For one
// projection the lanes of a warp hit neighbouring 2x2 neighbourhoods, so
// same-address conflicts inside a warp are rare.
template <typename T, bool IEEE>
__global__ void __launch_bounds__(kThreads)
direct_adjoint_kernel(const __grid_constant__ AdjBatchT<T> b, const T *__restrict__ vol,
                      const VolGeomT<T> g, T *__restrict__ out, int isx, int isy)
{
    constexpr int LX = 8, LZ = 32 / LX, TX = LX * kVoxPerLane;
    const int lane = threadIdx.x & 31;
    const int tx = lane % LX, tz = lane / LX;
    const int L = g.L;
    const int xb = blockIdx.x * TX + tx;
    const int y = blockIdx.y * kWarpsY + (threadIdx.x >> 5);
    const int z = blockIdx.z * LZ + tz;
    if (y >= L || z >= g.Lz)
        return;

    const T *row = vol + ((size_t)z * L + y) * L;
    T f[kVoxPerLane], X[kVoxPerLane];
#pragma unroll
    for (int k = 0; k < kVoxPerLane; ++k) {
        const int x = xb + LX * k;
        f[k] = x < L ? row[x] : T(0);
        X[k] = fma(g.R, (T)x, g.Ox);
    }
    const T Y = fma(g.R, (T)y, g.Oy);
    const T Z = fma(g.R, (T)(z + g.z0), g.Oz);

#pragma unroll 1
    for (int i = 0; i < b.n; ++i) {
        const Vec4<T> ru = b.m[i][0], rv = b.m[i][1], rw = b.m[i][2];
        const int2 kc = b.k[i];
        // bounds of the centred coordinates u' = u - ku, v' = v - kv
        const T ulo = (T)(-1 - kc.x), uhi = (T)(isx - kc.x);
        const T vlo = (T)(-1 - kc.y), vhi = (T)(isy - kc.y);
        T *img = out + b.out_off[i];
        const T bu = fma(ru.y, Y, fma(ru.z, Z, ru.w));
        const T bv = fma(rv.y, Y, fma(rv.z, Z, rv.w));
        const T bw = fma(rw.y, Y, fma(rw.z, Z, rw.w));
#pragma unroll
        for (int k = 0; k < kVoxPerLane; ++k) {
            if (f[k] == T(0))
                continue;
            const T uw = fma(ru.x, X[k], bu);
            const T vw = fma(rv.x, X[k], bv);
            const T w = fma(rw.x, X[k], bw);
            const T r = direct_recip<T, IEEE>(w);
            const T u = uw * r, v = vw * r;
            // Every corner is outside the detector unless -1 < u < isx and
            // -1 < v < isy (this also keeps the int conversion in range).
            if (!(u > ulo && u < uhi && v > vlo && v < vhi))
                continue;
            const T fu0 = floor(u), fv0 = floor(v);
            const int iu = (int)fu0 + kc.x, iv = (int)fv0 + kc.y;
            const T fu = u - fu0, fv = v - fv0;
            const T s = f[k] * (r * r);
            const T sb = s * fv, st = s - sb;          // s fv, s (1 - fv)
            const T w_tr = st * fu, w_tl = st - w_tr;  // s fu (1-fv), s (1-fu)(1-fv)
            const T w_br = sb * fu, w_bl = sb - w_br;  // s fu fv, s (1-fu) fv
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

// The backprojection in its plain form: one thread per voxel, the four
// corners read from the images in global memory (zero outside the
// detector), accumulated over the batch in a register and added to the
// volume once.  Same centred rows and coordinates as the adjoint above, so
// the two kernels are exact transposes of each other up to rounding.
template <typename T>
struct DirectBatchT {
    Vec4<T> m[kMaxBatch][3];
    int2 k[kMaxBatch];
    long long img_off[kMaxBatch];   // offset of projection i's image in the stack
    int n;
};

template <typename T, bool IEEE>
__global__ void __launch_bounds__(256)
direct_backproject_kernel(const __grid_constant__ DirectBatchT<T> b, const T *__restrict__ images,
                          T *__restrict__ vol, const VolGeomT<T> g, int isx, int isy)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    const int L = g.L;
    if (x >= L)
        return;
    const T X = fma(g.R, (T)x, g.Ox), Y = fma(g.R, (T)y, g.Oy), Z = fma(g.R, (T)(z + g.z0), g.Oz);
    T acc = T(0);
#pragma unroll 1
    for (int i = 0; i < b.n; ++i) {
        const Vec4<T> ru = b.m[i][0], rv = b.m[i][1], rw = b.m[i][2];
        const int2 kc = b.k[i];
        const T uw = fma(ru.x, X, fma(ru.y, Y, fma(ru.z, Z, ru.w)));
        const T vw = fma(rv.x, X, fma(rv.y, Y, fma(rv.z, Z, rv.w)));
        const T w = fma(rw.x, X, fma(rw.y, Y, fma(rw.z, Z, rw.w)));
        const T r = direct_recip<T, IEEE>(w);
        const T u = uw * r, v = vw * r;
        if (!(u > (T)(-1 - kc.x) && u < (T)(isx - kc.x) && v > (T)(-1 - kc.y) && v < (T)(isy - kc.y)))
            continue;
        const T fu0 = floor(u), fv0 = floor(v);
        const int iu = (int)fu0 + kc.x, iv = (int)fv0 + kc.y;
        const T fu = u - fu0, fv = v - fv0;
        const T *img = images + b.img_off[i];
        const bool in_l = iu >= 0, in_r = iu + 1 < isx, in_t = iv >= 0, in_b = iv + 1 < isy;
        const long long base = (long long)iv * isx + iu;
        const T tl = in_t && in_l ? img[base] : T(0);
        const T tr = in_t && in_r ? img[base + 1] : T(0);
        const T bl = in_b && in_l ? img[base + isx] : T(0);
        const T br = in_b && in_r ? img[base + isx + 1] : T(0);
        const T t = fma(fu, tr - tl, tl);
        const T bt = fma(fu, br - bl, bl);
        const T fx = fma(fv, bt - t, t);
        acc = fma(fx, r * r, acc);
    }
    vol[((size_t)z * L + y) * L + x] += acc;
}

}  // namespace bp
