// Adjoint (transpose) of the voxel-driven backprojection: a voxel-driven
// forward projection.  For every voxel value f(x) and projection i the value
// s = f(x) / w^2 is spread onto the four pixels around (u, v) = (uw/w, vw/w)
// with the bilinear weights of Listing 1 (Sect. 3.1), dropping pixels
// outside the detector.  This is exactly B^T for the map of bp_fwd.cu, so
// <B p, f> = <p, B^T f>.
//
// Two kernels: the shared-tile kernel below (the default: each block
// accumulates its footprint in shared memory and flushes it with one atomic
// per pixel), and the direct kernel of bp_direct.cuh (float32 atomics per
// update; BP_OPT_CULL 0).
#include "bp_direct.cuh"
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

// Shared-memory accumulation.  Per projection, 8 lanes of warp 0 project
// the corners of the block's voxel box and the block agrees on its footprint
// (with a pixel of margin, not clipped to the detector, so that every corner
// of every voxel falls inside it without a test).  Then
//   * footprint off the detector: the projection is skipped (all of its
//     terms would be dropped -- block culling, as in the forward kernel);
//   * footprint of at most kAdjTile pixels: the block scatters its 4
//     weighted corners per update into a tile of that size, and adds the
//     tile's nonzero pixels on the detector to the image with one global
//     atomic each (a few hundred per block instead of 4 per update),
//     zeroing each word it reads (the tile starts zeroed, so it is zero
//     again for the next projection without a pass of its own);
//   * larger footprint: global atomics per update, as in the direct kernel.
// The tile accumulates in 32-bit fixed point with native integer
// shared-memory atomics: float, and 64-bit integer, shared-memory atomics
// are emulated with compare-and-swap loops on this GPU (measured 196 and 123
// against 306 GUP/s).  The scale is a power of two chosen per projection
// from a bound: a voxel's four weights go to four different pixels, so it
// adds at most |f| r^2 to any pixel, and r^2 = 1/w^2 is largest at a corner
// of the block's box (w is affine).  A pixel's terms therefore sum in
// magnitude to at most B = (sum of |f| over the block) * (max r^2 over the
// box).  With B mapped to 2^30 no partial sum can overflow; a term is
// rounded to 2^-31 B (float32 rounds to 2^-24 of the term itself): about
// 1e-6 relative error on coarse detectors, below float32 order effects on
// fine ones.
// Same coordinates and weights as direct_adjoint_kernel.
using AdjAcc = int;
constexpr int kAccBits = 8 * (int)sizeof(AdjAcc);
constexpr float kFloorMagic = 12582912.0f;          // 1.5 * 2^23
constexpr unsigned kFloorMagicBits = 0x4B400000u;   // its bits

// Blocks of 32 x 32 x 4 voxels: each lane takes 4 voxels along x (8 apart)
// and kAdjVPY along y (one per warp row, kWarpsY apart).  A block's
// footprint grows with its x and y extent in u but its update count with
// x * y, so the per-projection work of a block (plan, zeroing and flushing
// its tile, barriers) is spread over 4096 updates.
constexpr int kAdjVPY = 4;

// BLK: per-block centring, as in the forward kernels: the block stages its
// centring records of the batch (u row, v row, (w_c, ku_b, kv_b); written by
// the per-tile pre-pass with this kernel's block as the tile) and works
// with offsets from the centre of its voxel box, so u and v stay within the
// block's footprint.  The records centre u' = u - ku_b + 1; the kernel's
// pixel offsets are ku_b - 1, kv_b - 1.
// Four blocks per SM (measured: 538 GUP/s against 521 with three; with the
// earlier four-barrier loop, 533 against 510 with the compiler's own
// register choice, 500 with five blocks, 495 with six).
template <bool IEEE, bool BLK>
__global__ void __launch_bounds__(kThreads, 4)
bp_adjoint_smem_kernel(const __grid_constant__ AdjBatch b, const float *__restrict__ vol, const VolGeom g,
                       float *__restrict__ out, int isx, int isy)
{
    constexpr int LX = 8, LZ = 32 / LX, TX = LX * kVoxPerLane, TY = kWarpsY * kAdjVPY;
    static_assert(TX == kAdjBlockX && TY == kAdjBlockY && LZ == kAdjBlockZ, "pre-pass tile must be the block");
    __shared__ __align__(16) AdjAcc tile[kAdjTile];
    // (x0, y0, W, H); W = 0 culled, W < 0 too large.  Two slots: warp 0
    // plans the next projection after its own scatter, while slower warps
    // may still read this one; the barrier that ends the scatter publishes
    // it.  A projection thus costs two block barriers (end of the scatter,
    // end of the flush) and one when it is culled or untiled.
    __shared__ int4 plan[2];
    __shared__ float2 plan_scale[2];   // (scale, 1 / scale) of the fixed-point tile
    __shared__ float fsum_warp[kThreads / 32];
    __shared__ float4 rec[3][BLK ? kMaxBatch : 1];
    const int lane = threadIdx.x & 31;
    const int tx = lane % LX, tz = lane / LX;
    const int L = g.L;
    const int bx0 = blockIdx.x * TX, by0 = blockIdx.y * TY, bz0 = blockIdx.z * LZ;
    const int xb = bx0 + tx;
    const int yb = by0 + (threadIdx.x >> 5);   // this lane's rows: yb + kWarpsY * ky
    const int z = bz0 + tz;

    // voxel coordinates: absolute, or with BLK offsets from the centre of the
    // block's voxel box clipped to the volume ((x0 + x1) / 2 etc., a multiple
    // of 1/2, as in the pre-pass)
    const int xe = min(bx0 + TX, L) - 1, ye = min(by0 + TY, L) - 1, ze = min(bz0 + LZ, g.Lz) - 1;
    const float hx = 0.5f * (float)(bx0 + xe), hy = 0.5f * (float)(by0 + ye), hz = 0.5f * (float)(bz0 + ze);
    float f[kAdjVPY][kVoxPerLane], X[kVoxPerLane], Y[kAdjVPY];
#pragma unroll
    for (int k = 0; k < kVoxPerLane; ++k)
        X[k] = BLK ? g.R * ((float)(xb + LX * k) - hx) : fmaf(g.R, (float)(xb + LX * k), g.Ox);
#pragma unroll
    for (int ky = 0; ky < kAdjVPY; ++ky) {
        const int y = yb + kWarpsY * ky;
        const bool live = y < L && z < g.Lz;
        Y[ky] = BLK ? g.R * ((float)y - hy) : fmaf(g.R, (float)y, g.Oy);
#pragma unroll
        for (int k = 0; k < kVoxPerLane; ++k) {
            const int x = xb + LX * k;
            f[ky][k] = (live && x < L) ? vol[((size_t)z * L + y) * L + x] : 0.f;
        }
    }
    const float Z = BLK ? g.R * ((float)z - hz) : fmaf(g.R, (float)(z + g.z0), g.Oz);
    if constexpr (BLK) {
        if (threadIdx.x < 3 * kMaxBatch) {
            const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
            const int part = threadIdx.x / kMaxBatch, i = threadIdx.x % kMaxBatch;
            if (i < b.n)
                rec[part][i] = b.centres[((size_t)part * kMaxBatch + i) * b.blocks + blk];
        }
    }
    // sum of |f| over the block, for the fixed-point scale (rounded up by
    // the factor applied to B below)
    float fm = 0.f;
#pragma unroll
    for (int ky = 0; ky < kAdjVPY; ++ky)
#pragma unroll
        for (int k = 0; k < kVoxPerLane; ++k)
            fm += fabsf(f[ky][k]);
    for (int o = 16; o > 0; o >>= 1)
        fm += __shfl_xor_sync(0xffffffffu, fm, o);
    if (lane == 0)
        fsum_warp[threadIdx.x >> 5] = fm;
    __syncthreads();
    float fsum_blk = 0.f;
#pragma unroll
    for (int w8 = 0; w8 < kThreads / 32; ++w8)
        fsum_blk += fsum_warp[w8];
    // corner of the block's voxel box taken by lane c < 8 of warp 0
    const float CX = fmaf(g.R, (float)((lane & 1) ? xe : bx0), g.Ox);
    const float CY = fmaf(g.R, (float)((lane & 2) ? ye : by0), g.Oy);
    const float CZ = fmaf(g.R, (float)(((lane & 4) ? ze : bz0) + g.z0), g.Oz);

    // warp 0: the footprint box and fixed-point scale of projection i into
    // plan slot i & 1
    auto plan_projection = [&](int i) {
        const float4 ru = b.m[i][0], rv = b.m[i][1], rw = b.m[i][2];
        const int2 kc = b.k[i];
        if (threadIdx.x < 32) {
            const float w = fmaf(rw.x, CX, fmaf(rw.y, CY, fmaf(rw.z, CZ, rw.w)));
            const float r = 1.0f / w;
            float umin = fmaf(ru.x, CX, fmaf(ru.y, CY, fmaf(ru.z, CZ, ru.w))) * r, umax = umin;
            float vmin = fmaf(rv.x, CX, fmaf(rv.y, CY, fmaf(rv.z, CZ, rv.w))) * r, vmax = vmin;
            float wmin = w;
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                umin = fminf(umin, __shfl_xor_sync(0xffffffffu, umin, o));
                umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, o));
                vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
                vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
                wmin = fminf(wmin, __shfl_xor_sync(0xffffffffu, wmin, o));
            }
            if (lane == 0) {
                umin = fminf(fmaxf(umin, -1.0e6f), 1.0e6f);   // keep the int conversions in range
                umax = fminf(fmaxf(umax, -1.0e6f), 1.0e6f);
                vmin = fminf(fmaxf(vmin, -1.0e6f), 1.0e6f);
                vmax = fminf(fmaxf(vmax, -1.0e6f), 1.0e6f);
                // pixels touched: floor(u) .. floor(u) + 1 with u = u' + ku, one of
                // margin; the box is not clipped to the detector, so every
                // corner of every voxel of the block lies inside it (the
                // projection of the block is the hull of its corners'), and
                // the flush drops the pixels outside the detector
                const int x0 = (int)floorf(umin) + kc.x - 1, x1 = (int)floorf(umax) + kc.x + 2;
                const int y0 = (int)floorf(vmin) + kc.y - 1, y1 = (int)floorf(vmax) + kc.y + 2;
                int4 p = make_int4(x0, y0, 0, 0);
                if (x1 >= 0 && x0 <= isx - 1 && y1 >= 0 && y0 <= isy - 1) {
                    const int W = x1 - x0 + 1, H = y1 - y0 + 1;   // at least 4 each
                    p.z = (W <= kAdjTile && H <= kAdjTile && W * H <= kAdjTile) ? W : -1;
                    p.w = H;
                }
                // fixed-point scale 2^e with B * 2^e <= 2^(kAccBits - 2), B the
                // bound on a pixel's summed term magnitudes (1.01: the voxels'
                // float32 w may fall a little below the corners', and the
                // float32 sum of |f| is rounded)
                const float B = fsum_blk * 1.01f / (wmin * wmin);
                int e = 0;
                if (B > 0.f && isfinite(B)) {
                    e = (kAccBits - 2) - (int)ceilf(log2f(B));
                    e = max(-100, min(e, 100));
                }
                plan_scale[i & 1] = make_float2(ldexpf(1.f, e), ldexpf(1.f, -e));
                plan[i & 1] = p;
            }
        }
    };

    // the tile starts zeroed; every flush leaves the part it used zeroed
    for (int q = threadIdx.x; q < kAdjTile / 4; q += kThreads)
        reinterpret_cast<int4 *>(tile)[q] = make_int4(0, 0, 0, 0);
    plan_projection(0);
    __syncthreads();
#pragma unroll 1
    for (int i = 0; i < b.n; ++i) {
        const float4 ru = b.m[i][0], rv = b.m[i][1], rw = b.m[i][2];
        const int2 kc = b.k[i];
        const int4 p = plan[i & 1];
        const float2 sc = plan_scale[i & 1];
        float *img = out + b.out_off[i];
        const bool tiled = p.z > 0;
        if (p.z != 0) {
            // the voxels' rows and pixel offsets: the projection's (the plan
            // above), or with BLK the block's recentred ones
            float4 vu = ru, vv = rv, vw4 = rw;
            int2 kb = kc;
            if constexpr (BLK) {
                vu = rec[0][i];
                vv = rec[1][i];
                vw4.w = rec[2][i].x;
                kb = make_int2((int)rec[2][i].y - 1, (int)rec[2][i].z - 1);
            }
            if (tiled) {
                // Every corner lands in the tile (the box covers the block's
                // footprint with a pixel of margin), so there is no per-corner
                // test; the clamp keeps the four addresses inside the array
                // whatever the rounding.  The fixed-point scale (a power of two)
                // is folded into the weight: the terms equal the scaled ones of
                // the global path exactly.
                const int W = p.z;
                const unsigned qmax = (unsigned)(W * p.w - W - 2);
                const int du = kb.x - p.x, dv = kb.y - p.y;
                // the tile index of the top-left corner from the bits of the
                // round-down sums (below): (bits(mv) - M) * W + bits(mu) - M +
                // dv * W + du, in 32-bit unsigned arithmetic
                const unsigned qoff = (unsigned)(dv * W + du) - kFloorMagicBits * (unsigned)(W + 1);
    #pragma unroll
                for (int ky = 0; ky < kAdjVPY; ++ky) {
                    const float bu = fmaf(vu.y, Y[ky], fmaf(vu.z, Z, vu.w));
                    const float bv = fmaf(vv.y, Y[ky], fmaf(vv.z, Z, vv.w));
                    const float bw = fmaf(vw4.y, Y[ky], fmaf(vw4.z, Z, vw4.w));
    #pragma unroll
                    for (int k = 0; k < kVoxPerLane; ++k) {
                        if (f[ky][k] == 0.f)
                            continue;
                        const float uw = fmaf(vu.x, X[k], bu);
                        const float vw = fmaf(vv.x, X[k], bv);
                        const float w = fmaf(vw4.x, X[k], bw);
                        const float r = recip_adj<IEEE>(w);
                        const float u = uw * r, v = vw * r;
                        // floor without the conversion unit, which the
                        // reciprocal and the four fixed-point conversions keep
                        // busy (the floors and int conversions made it the
                        // binding pipe: 9 of its operations per update): u +
                        // 1.5 * 2^23 rounded down is floor(u) + 1.5 * 2^23
                        // exactly for |u| < 2^22 (u stays within the block's
                        // footprint), and its bits are the integer
                        const float mu = __fadd_rd(u, kFloorMagic), mv = __fadd_rd(v, kFloorMagic);
                        const float fu0 = mu - kFloorMagic, fv0 = mv - kFloorMagic;
                        const unsigned q0 = min((unsigned)__float_as_int(mv) * (unsigned)W +
                                                    (unsigned)__float_as_int(mu) + qoff, qmax);
                        const float fu = u - fu0, fv = v - fv0;
                        const float s = f[ky][k] * ((r * sc.x) * r);
                        const float sb = s * fv, st = s - sb;
                        const float w_tr = st * fu, w_tl = st - w_tr;
                        const float w_br = sb * fu, w_bl = sb - w_br;
                        atomicAdd(&tile[q0], __float2int_rn(w_tl));
                        atomicAdd(&tile[q0 + 1], __float2int_rn(w_tr));
                        atomicAdd(&tile[q0 + W], __float2int_rn(w_bl));
                        atomicAdd(&tile[q0 + W + 1], __float2int_rn(w_br));
                    }
                }
            } else {
                // footprint larger than the tile: global atomics, pixels outside
                // the detector dropped
                const float ulo = (float)(-1 - kb.x), uhi = (float)(isx - kb.x);
                const float vlo = (float)(-1 - kb.y), vhi = (float)(isy - kb.y);
    #pragma unroll
                for (int ky = 0; ky < kAdjVPY; ++ky) {
                    const float bu = fmaf(vu.y, Y[ky], fmaf(vu.z, Z, vu.w));
                    const float bv = fmaf(vv.y, Y[ky], fmaf(vv.z, Z, vv.w));
                    const float bw = fmaf(vw4.y, Y[ky], fmaf(vw4.z, Z, vw4.w));
    #pragma unroll
                    for (int k = 0; k < kVoxPerLane; ++k) {
                        if (f[ky][k] == 0.f)
                            continue;
                        const float uw = fmaf(vu.x, X[k], bu);
                        const float vw = fmaf(vv.x, X[k], bv);
                        const float w = fmaf(vw4.x, X[k], bw);
                        const float r = recip_adj<IEEE>(w);
                        const float u = uw * r, v = vw * r;
                        if (!(u > ulo && u < uhi && v > vlo && v < vhi))
                            continue;
                        const float fu0 = floorf(u), fv0 = floorf(v);
                        const int iu = (int)fu0 + kb.x, iv = (int)fv0 + kb.y;
                        const float fu = u - fu0, fv = v - fv0;
                        const float s = f[ky][k] * (r * r);
                        const float sb = s * fv, st = s - sb;
                        const float w_tr = st * fu, w_tl = st - w_tr;
                        const float w_br = sb * fu, w_bl = sb - w_br;
                        const bool in_l = iu >= 0, in_r = iu + 1 < isx, in_t = iv >= 0, in_b = iv + 1 < isy;
                        const long long base = (long long)iv * isx + iu;
                        if (in_t) {
                            if (in_l) atomicAdd(img + base, w_tl);
                            if (in_r) atomicAdd(img + base + 1, w_tr);
                        }
                        if (in_b) {
                            if (in_l) atomicAdd(img + base + isx, w_bl);
                            if (in_r) atomicAdd(img + base + isx + 1, w_br);
                        }
                    }
                }
            }
        }
        if (i + 1 < b.n)
            plan_projection(i + 1);
        __syncthreads();   // the scatter is done; the next plan is visible
        if (tiled) {
            // one warp per tile row, lanes along the row; the pixels on the
            // detector go to the image, and every word used is left zero
            const int c0 = max(0, -p.x), c1 = min(p.z, isx - p.x);
            const int r0 = max(0, -p.y), r1 = min(p.w, isy - p.y);
            for (int row = threadIdx.x >> 5; row < p.w; row += kThreads / 32) {
                float *dst = img + (long long)(p.y + row) * isx + p.x;
                AdjAcc *src = tile + row * p.z;
                const bool on_row = row >= r0 && row < r1;
                for (int col = lane; col < p.z; col += 32) {
                    const AdjAcc v = src[col];
                    if (v != 0) {
                        src[col] = 0;
                        if (on_row && col >= c0 && col < c1)
                            atomicAdd(dst + col, (float)v * sc.y);
                    }
                }
            }
            // the next projection scatters into the tile only if it is tiled
            if (i + 1 < b.n && plan[(i + 1) & 1].z > 0)
                __syncthreads();
        }
    }
}

cudaError_t launch_bp_adjoint(const AdjBatch &b, const float *vol, const VolGeom &g, float *out,
                              int isx, int isy, bool ieee_rcp, bool smem, cudaStream_t s)
{
    if (b.n <= 0)
        return cudaSuccess;
    constexpr int TX = 8 * kVoxPerLane, LZ = 4;
    dim3 grid((g.L + TX - 1) / TX, (g.L + kWarpsY - 1) / kWarpsY, (g.Lz + LZ - 1) / LZ);
    if (smem) {
        grid.y = (g.L + kWarpsY * kAdjVPY - 1) / (kWarpsY * kAdjVPY);
        if (b.centres) {
            if (ieee_rcp)
                bp_adjoint_smem_kernel<true, true><<<grid, kThreads, 0, s>>>(b, vol, g, out, isx, isy);
            else
                bp_adjoint_smem_kernel<false, true><<<grid, kThreads, 0, s>>>(b, vol, g, out, isx, isy);
        } else if (ieee_rcp) {
            bp_adjoint_smem_kernel<true, false><<<grid, kThreads, 0, s>>>(b, vol, g, out, isx, isy);
        } else {
            bp_adjoint_smem_kernel<false, false><<<grid, kThreads, 0, s>>>(b, vol, g, out, isx, isy);
        }
    } else if (ieee_rcp) {
        direct_adjoint_kernel<float, true><<<grid, kThreads, 0, s>>>(b, vol, g, out, isx, isy);
    } else {
        direct_adjoint_kernel<float, false><<<grid, kThreads, 0, s>>>(b, vol, g, out, isx, isy);
    }
    return cudaGetLastError();
}

}  // namespace bp
