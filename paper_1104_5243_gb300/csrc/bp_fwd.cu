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
//  * Per-block centring (float32 form): the same pre-pass gives every
//    (block, projection) integer offsets near the block centre's projection
//    and the centred homogeneous values there, exact to float-float
//    precision.  The kernel adds offsets from the block centre, so u' and v'
//    stay within the block's footprint (tens of pixels) instead of the
//    volume's, and their float32 rounding shrinks accordingly.
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

template <int KIND, bool IEEE, int LX, int LY, int VPL, bool BLK>
__global__ void __launch_bounds__(kThreads, VPL == 4 ? 6 : 4)
bp_fwd_kernel(const __grid_constant__ FwdBatch b, float *__restrict__ vol, const VolGeom g,
              int accumulate, const unsigned long long *__restrict__ masks,
              const float4 *__restrict__ centres)
{
    constexpr int LZ = 32 / (LX * LY);          // lanes along z
    constexpr int TX = LX * VPL;                // x extent of the block tile
    constexpr int TY = kWarpsY * LY;
    const int lane = threadIdx.x & 31;
    const int tx = lane % LX, ty = (lane / LX) % LY, tz = lane / (LX * LY);
    const int L = g.L;
    const int xb = blockIdx.x * TX + tx;        // this lane's voxels: xb + LX k
    const int y = blockIdx.y * TY + (threadIdx.x >> 5) * LY + ty;
    const int z = blockIdx.z * LZ + tz;
    const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    // projections that can reach this block (all of them without culling)
    const unsigned long long visible = masks ? masks[blk] : ~0ull;
    // BLK: the block's centring records of those projections (three float4
    // planes: u row, v row, (w_c, gather offsets)), staged once
    __shared__ float4 cen[BLK ? 3 * kMaxBatch : 1];
    if constexpr (BLK) {
        const size_t nblk = (size_t)gridDim.x * gridDim.y * gridDim.z;
        if (threadIdx.x < 3 * kMaxBatch) {
            const int j = threadIdx.x / kMaxBatch, i = threadIdx.x % kMaxBatch;
            if (i < b.n && ((visible >> i) & 1ull))
                cen[threadIdx.x] = centres[((size_t)j * kMaxBatch + i) * nblk + blk];
        }
        __syncthreads();
    }
    if (y >= L || z >= g.Lz)
        return;

    // Voxel coordinates: absolute, or with BLK offsets from the centre of the
    // block's voxel box clipped to the volume, (x0 + x1) / 2 etc.  The centre
    // index is a multiple of 1/2, so the offsets are exact before the product
    // with R.
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * LZ;
    const float hx = 0.5f * (float)(x0 + min(x0 + TX, L) - 1);
    const float hy = 0.5f * (float)(y0 + min(y0 + TY, L) - 1);
    const float hz = 0.5f * (float)(z0 + min(z0 + LZ, g.Lz) - 1);
    float X[VPL];
#pragma unroll
    for (int k = 0; k < VPL; ++k)
        X[k] = BLK ? g.R * ((float)(xb + LX * k) - hx) : fmaf(g.R, (float)(xb + LX * k), g.Ox);
    const float Y = BLK ? g.R * ((float)y - hy) : fmaf(g.R, (float)y, g.Oy);
    const float Z = BLK ? g.R * ((float)z - hz) : fmaf(g.R, (float)(z + g.z0), g.Oz);

    float acc[VPL];
#pragma unroll
    for (int k = 0; k < VPL; ++k)
        acc[k] = 0.f;
#pragma unroll 1
    for (int i = 0; i < b.n; ++i) {
        if (!((visible >> i) & 1ull))
            continue;   // every term of this projection is exactly zero here
        float4 ru, rv, rw = b.m[i][2];
        float2 kc;
        if constexpr (BLK) {
            // rows recentred on the block: (row_u'' x, y, z, value at the
            // block centre), likewise v, and (w_c, gather offsets)
            ru = cen[i];
            rv = cen[kMaxBatch + i];
            const float4 c = cen[2 * kMaxBatch + i];
            rw.w = c.x;
            kc = make_float2(c.y, c.z);
        } else {
            ru = b.m[i][0];
            rv = b.m[i][1];
            kc = b.k[i];
        }
        const cudaTextureObject_t t = b.tex[i];
        // Part 1: geometry; the y, z terms are shared by the lane's voxels
        // (z outermost, y inside: the order the TMA kernel uses, which
        // shares the y term across a lane's z values)
        const float bu = fmaf(ru.z, Z, fmaf(ru.y, Y, ru.w));
        const float bv = fmaf(rv.z, Z, fmaf(rv.y, Y, rv.w));
        const float bw = fmaf(rw.z, Z, fmaf(rw.y, Y, rw.w));
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

    // a batch stored with a power-of-four scale 2^(-2k) (b.pmax): the sums
    // times 2^(2k), exactly; 1 otherwise
    const float vs = b.pmax ? pow2f(2 * proj_scale_k(*b.pmax)) : 1.f;
    float *row = vol + ((size_t)z * L + y) * L;
#pragma unroll
    for (int k = 0; k < VPL; ++k) {
        const int x = xb + LX * k;
        if (x < L)
            row[x] = (accumulate ? row[x] : 0.f) + acc[k] * vs;
    }
}

// Block tile of a layout: (TX, TY, TZ) voxels.
void fwd_tile(int lanes_x, int *tx, int *ty, int *tz)
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

long long tile_count(int L, int Lz, int tx, int ty, int tz)
{
    return (long long)((L + tx - 1) / tx) * ((L + ty - 1) / ty) * ((Lz + tz - 1) / tz);
}


template <int KIND, bool IEEE, int LX, int LY, int VPL = kVoxPerLane>
static cudaError_t launch_lx(const FwdBatch &b, float *vol, const VolGeom &g, bool acc,
                             const unsigned long long *masks, const float4 *centres, cudaStream_t s)
{
    constexpr int TX = LX * VPL, TY = kWarpsY * LY, LZ = 32 / (LX * LY);
    dim3 grid((g.L + TX - 1) / TX, (g.L + TY - 1) / TY, (g.Lz + LZ - 1) / LZ);
    if constexpr (KIND == kTexFloat) {
        if (centres) {
            bp_fwd_kernel<KIND, IEEE, LX, LY, VPL, true><<<grid, kThreads, 0, s>>>(b, vol, g, acc ? 1 : 0, masks,
                                                                                    centres);
            return cudaGetLastError();
        }
    }
    bp_fwd_kernel<KIND, IEEE, LX, LY, VPL, false><<<grid, kThreads, 0, s>>>(b, vol, g, acc ? 1 : 0, masks, nullptr);
    return cudaGetLastError();
}

// Float-float arithmetic (Dekker, Knuth): a value is the unevaluated sum
// hi + lo of two float32 numbers.  The explicit _rn intrinsics keep the
// compiler from contracting the error terms into FMAs.
struct Ff {
    float hi, lo;
};

__device__ __forceinline__ Ff two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ Ff ff_norm(float hi, float lo)   // needs |hi| >= |lo| or hi == 0
{
    const float s = __fadd_rn(hi, lo);
    return {s, __fsub_rn(lo, __fsub_rn(s, hi))};
}

__device__ __forceinline__ Ff ff_add(Ff a, Ff b)
{
    const Ff s = two_sum(a.hi, b.hi);
    return ff_norm(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

// a * n for an integer-valued float n (|n| < 2^24): the product of the high
// parts is split exactly with an FMA.
__device__ __forceinline__ Ff ff_mul_int(Ff a, float n)
{
    const float p = __fmul_rn(a.hi, n);
    const float e = fmaf(a.lo, n, fmaf(a.hi, n, -p));
    return ff_norm(p, e);
}

// Footprint test of one (block, projection): project the 8 corners of the
// block's voxel box (clamped to the volume) with float32 arithmetic and keep
// the projection when the footprint, widened by one pixel, touches
// [-1, isx] x [-1, isy].  The kernel's coordinates differ from these by far
// less than the pixel of margin.
__device__ bool footprint_hits(const FwdBatch &b, int i, const VolGeom &g, int isx, int isy, int x0, int y0,
                               int z0, int x1, int y1, int z1)
{
    const float4 ru = b.m[i][0], rv = b.m[i][1], rw = b.m[i][2];
    float umin = 3.0e38f, umax = -3.0e38f, vmin = 3.0e38f, vmax = -3.0e38f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float X = fmaf(g.R, (float)((c & 1) ? x1 : x0), g.Ox);
        const float Y = fmaf(g.R, (float)((c & 2) ? y1 : y0), g.Oy);
        const float Z = fmaf(g.R, (float)(((c & 4) ? z1 : z0) + g.z0), g.Oz);
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
    return !(pu1 < -1.f || pu0 > (float)isx || pv1 < -1.f || pv0 > (float)isy);
}

// Centring record of the block whose clipped voxel box has its centre at
// voxel index (cx2, cy2, cz2) / 2, for projection i.  The rows' values there
// are float-float sums C + cx2 Hx + cy2 Hy + cz2 Hz; with the offsets
// dku = round(u'_c), dkv = round(v'_c) (any integer is valid; these make
// u'' and v'' smallest near the centre) the record holds
//   u: (row_u'' x, y, z, uw_c - dku w_c),  row_u'' = row_u' - dku row_w,
//   v: the same for v,
//   w: (w_c, ku + dku, kv + dkv, 0),
// the centre values rounded to float32 once.  The centre lies in the volume,
// where the host has checked w > 0.
struct BlockRec {
    float4 u, v, w;
};

__device__ BlockRec block_centre(const FwdBatch &b, const CentreBatch &cb, int i, int cx2, int cy2, int cz2)
{
    Ff val[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float2 *c = cb.c[i][r];
        const Ff sx = ff_mul_int({c[1].x, c[1].y}, (float)cx2);
        const Ff sy = ff_mul_int({c[2].x, c[2].y}, (float)cy2);
        const Ff sz = ff_mul_int({c[3].x, c[3].y}, (float)cz2);
        val[r] = ff_add(ff_add({c[0].x, c[0].y}, sx), ff_add(sy, sz));
    }
    float dku = rintf(val[0].hi / val[2].hi), dkv = rintf(val[1].hi / val[2].hi);
    if (!(fabsf(dku) <= 1048576.f))
        dku = 0.f;
    if (!(fabsf(dkv) <= 1048576.f))
        dkv = 0.f;
    const Ff du = ff_mul_int(val[2], -dku), dv = ff_mul_int(val[2], -dkv);
    const float4 ru = b.m[i][0], rv = b.m[i][1], rw = b.m[i][2];
    const float2 kc = b.k[i];
    BlockRec rec;
    rec.u = make_float4(fmaf(-dku, rw.x, ru.x), fmaf(-dku, rw.y, ru.y), fmaf(-dku, rw.z, ru.z), ff_add(val[0], du).hi);
    rec.v = make_float4(fmaf(-dkv, rw.x, rv.x), fmaf(-dkv, rw.y, rv.y), fmaf(-dkv, rw.z, rv.z), ff_add(val[1], dv).hi);
    rec.w = make_float4(val[2].hi, kc.x + dku, kc.y + dkv, 0.f);
    return rec;
}

// TMA-path box decision of one (brick, projection): the element columns
// and rows the brick's corner projections touch, with a pixel of margin,
// decide between culling, one staged box, and the global-memory path.  An
// update at pixel (iu, iv) reads element column iu + 1 = floor(u') + ku, and
// row iv = floor(v') + kv - 1 (pair images: rows iv and iv + 1) or stored row
// iv + 1 (column quads, whose element at stored row k + 1 carries image rows
// k and k + 1).  kb are the offsets the kernel's floor(u'), floor(v') are
// relative to.
__device__ int4 tma_box(const FwdBatch &b, int i, const VolGeom &g, int isx, int isy, int x0, int y0, int z0,
                        int x1, int y1, int z1, int2 kb, const BoxSpec &bs)
{
    const float4 ru = b.m[i][0], rv = b.m[i][1], rw = b.m[i][2];
    float umin = 3.0e38f, umax = -3.0e38f, vmin = 3.0e38f, vmax = -3.0e38f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float X = fmaf(g.R, (float)((c & 1) ? x1 : x0), g.Ox);
        const float Y = fmaf(g.R, (float)((c & 2) ? y1 : y0), g.Oy);
        const float Z = fmaf(g.R, (float)(((c & 4) ? z1 : z0) + g.z0), g.Oz);
        const float w = fmaf(rw.x, X, fmaf(rw.y, Y, fmaf(rw.z, Z, rw.w)));
        const float r = 1.0f / w;
        const float u = fmaf(ru.x, X, fmaf(ru.y, Y, fmaf(ru.z, Z, ru.w))) * r;
        const float v = fmaf(rv.x, X, fmaf(rv.y, Y, fmaf(rv.z, Z, rv.w))) * r;
        umin = fminf(umin, u);
        umax = fmaxf(umax, u);
        vmin = fminf(vmin, v);
        vmax = fmaxf(vmax, v);
    }
    // keep the int conversions in range
    umin = fminf(fmaxf(umin, -1.0e6f), 1.0e6f);
    umax = fminf(fmaxf(umax, -1.0e6f), 1.0e6f);
    vmin = fminf(fmaxf(vmin, -1.0e6f), 1.0e6f);
    vmax = fminf(fmaxf(vmax, -1.0e6f), 1.0e6f);
    const int ku = (int)b.k[i].x, kv = (int)b.k[i].y;
    // stored row of the update's (top) element: floor(v') + kv - 1 + quad
    const int rs = bs.quad ? 0 : -1;
    const int cmin = (int)floorf(umin) + ku - 1, cmax = (int)floorf(umax) + ku + 1;
    const int rmin = (int)floorf(vmin) + kv + rs - 1, rmax = (int)floorf(vmax) + kv + rs + (bs.quad ? 1 : 2);
    const int rows = bs.quad ? isy + 1 : isy;   // stored rows of the image
    if (cmax < 0 || cmin > isx || rmax < 0 || rmin > rows - 1)
        return make_int4(0, 0, 0, 0);   // nothing of this brick lands on the detector
    const int cx0 = cmin & ~(bs.align - 1), ry0 = rmin;
    if (cmax < cx0 + bs.bu && rmax < ry0 + bs.bv) {
        const int cu = kb.x - cx0, cv = kb.y + rs - ry0;
        return make_int4(1, __float_as_int((float)(cv * bs.bu + cu) + 12582912.0f), cx0, ry0);
    }
    return make_int4(2, kb.x, kb.y + rs, 0);
}

// One thread per tile (the texture kernel's block or the TMA path's brick),
// looping over the projections of the batch (a warp-uniform index: the
// matrices are read from kernel parameter space by broadcast).  Records are stored as three planes
// (u, v, w parts), projection-major within each, centres[(part * 64 + i) *
// nblocks + block], so a warp's stores are contiguous.  The kept
// updates are summed per warp into the context's work counter (for the
// roofline).
template <bool CENTRES>
__global__ void __launch_bounds__(256)
block_prepass_kernel(const __grid_constant__ FwdBatch b, const __grid_constant__ CentreBatch cb, const VolGeom g,
                     int isx, int isy, int tx, int ty, int tz, int zoff2, int nbx, int nby, long long nblocks,
                     unsigned long long *__restrict__ masks, float4 *__restrict__ centres, const BoxSpec bs,
                     int4 *__restrict__ boxes, unsigned long long *__restrict__ work)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long done = 0;
    if (q < nblocks) {
        const int bx = (int)(q % nbx), by = (int)((q / nbx) % nby), bz = (int)(q / ((long long)nbx * nby));
        const int x0 = bx * tx, y0 = by * ty, z0 = bz * tz;
        const int x1 = min(x0 + tx, g.L) - 1, y1 = min(y0 + ty, g.L) - 1, z1 = min(z0 + tz, g.Lz) - 1;
        unsigned long long m = 0;
        for (int i = 0; i < b.n; ++i) {
            if (masks && footprint_hits(b, i, g, isx, isy, x0, y0, z0, x1, y1, z1))
                m |= 1ull << i;
            int2 kb = make_int2((int)b.k[i].x, (int)b.k[i].y);
            if constexpr (CENTRES) {
                const BlockRec rec = block_centre(b, cb, i, x0 + x1, y0 + y1, z0 + z1 + zoff2);
                centres[((size_t)0 * kMaxBatch + i) * nblocks + q] = rec.u;
                centres[((size_t)1 * kMaxBatch + i) * nblocks + q] = rec.v;
                centres[((size_t)2 * kMaxBatch + i) * nblocks + q] = rec.w;
                kb = make_int2((int)rec.w.y, (int)rec.w.z);
            }
            if (boxes)
                boxes[(size_t)i * nblocks + q] = tma_box(b, i, g, isx, isy, x0, y0, z0, x1, y1, z1, kb, bs);
        }
        if (masks) {
            masks[q] = m;
            done = (unsigned long long)__popcll(m) * (x1 - x0 + 1) * (y1 - y0 + 1) * (z1 - z0 + 1);
        }
    }
    for (int o = 16; o > 0; o >>= 1)
        done += __shfl_down_sync(0xffffffffu, done, o);
    if ((threadIdx.x & 31) == 0 && done && work)
        atomicAdd(work, done);
}

cudaError_t launch_block_prepass(const FwdBatch &b, const CentreBatch *cb, const VolGeom &g, int isx, int isy,
                                 int tx, int ty, int tz, int zoff2, unsigned long long *masks, float4 *centres,
                                 const BoxSpec *box, int4 *boxes, unsigned long long *work, cudaStream_t s)
{
    if (b.n <= 0 || (!masks && !centres && !boxes))
        return cudaSuccess;
    const BoxSpec bs = box ? *box : BoxSpec{1, 1, 1};
    if (!box)
        boxes = nullptr;
    const int nbx = (g.L + tx - 1) / tx, nby = (g.L + ty - 1) / ty;
    const long long nblocks = tile_count(g.L, g.Lz, tx, ty, tz);
    const unsigned grid = (unsigned)((nblocks + 255) / 256);
    if (centres && cb) {
        block_prepass_kernel<true><<<grid, 256, 0, s>>>(b, *cb, g, isx, isy, tx, ty, tz, zoff2, nbx, nby, nblocks,
                                                        masks, centres, bs, boxes, work);
    } else {
        static const CentreBatch none = {};
        block_prepass_kernel<false><<<grid, 256, 0, s>>>(b, none, g, isx, isy, tx, ty, tz, zoff2, nbx, nby, nblocks,
                                                         masks, nullptr, bs, boxes, work);
    }
    return cudaGetLastError();
}

// Host side of the centring records: rows holds, per projection, the
// per-projection-centred rows u', v', w in float64 (n x 3 x 4).  Each row is
// stored as its value at voxel (0,0,0), X = O, and its change per half voxel
// along x, y and z.
void centre_batch(CentreBatch *cb, const double *rows, int n, const double O[3], double R)
{
    auto split = [](double v) {
        const float hi = (float)v;
        return make_float2(hi, (float)(v - (double)hi));
    };
    for (int i = 0; i < n; ++i)
        for (int r = 0; r < 3; ++r) {
            const double *a = rows + 12 * i + 4 * r;
            cb->c[i][r][0] = split(a[0] * O[0] + a[1] * O[1] + a[2] * O[2] + a[3]);
            cb->c[i][r][1] = split(a[0] * 0.5 * R);
            cb->c[i][r][2] = split(a[1] * 0.5 * R);
            cb->c[i][r][3] = split(a[2] * 0.5 * R);
        }
}

// Warp layouts (bp_set_option BP_OPT_LANES_X): 8, 16, 32 = lanes along x
// (the rest along z); two-digit codes XY = X lanes along x by Y along y
// (the rest along z): 44, 42, 82, 24; 108 = 8 lanes along x with 8 voxels
// per lane (instead of 4).
template <int KIND, bool IEEE>
static cudaError_t launch_kind(const FwdBatch &b, float *vol, const VolGeom &g, bool acc, int layout,
                               const unsigned long long *m, const float4 *c, cudaStream_t s)
{
    switch (layout) {
    case 32: return launch_lx<KIND, IEEE, 32, 1>(b, vol, g, acc, m, c, s);
    case 16: return launch_lx<KIND, IEEE, 16, 1>(b, vol, g, acc, m, c, s);
    case 44: return launch_lx<KIND, IEEE, 4, 4>(b, vol, g, acc, m, c, s);
    case 42: return launch_lx<KIND, IEEE, 4, 2>(b, vol, g, acc, m, c, s);
    case 82: return launch_lx<KIND, IEEE, 8, 2>(b, vol, g, acc, m, c, s);
    case 24: return launch_lx<KIND, IEEE, 2, 4>(b, vol, g, acc, m, c, s);
    case 108: return launch_lx<KIND, IEEE, 8, 1, 8>(b, vol, g, acc, m, c, s);
    default: return launch_lx<KIND, IEEE, 8, 1>(b, vol, g, acc, m, c, s);
    }
}

cudaError_t launch_bp_fwd(const FwdBatch &b, float *vol, const VolGeom &g, int tex_kind,
                          bool accumulate, bool ieee_rcp, int lanes_x, const unsigned long long *masks,
                          const float4 *centres, cudaStream_t s)
{
    if (b.n <= 0)
        return cudaSuccess;
    if (tex_kind == kTexFloat)
        return ieee_rcp ? launch_kind<kTexFloat, true>(b, vol, g, accumulate, lanes_x, masks, centres, s)
                        : launch_kind<kTexFloat, false>(b, vol, g, accumulate, lanes_x, masks, centres, s);
    return ieee_rcp ? launch_kind<kTexBF16, true>(b, vol, g, accumulate, lanes_x, masks, nullptr, s)
                    : launch_kind<kTexBF16, false>(b, vol, g, accumulate, lanes_x, masks, nullptr, s);
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
    float f = b.src[i][(size_t)k * isx + j];
    if (b.pmax)
        f *= pow2f(-2 * proj_scale_k(*b.pmax));   // the batch's power-of-four scale (exact)
    if constexpr (MODE == 0) {
        surf2Dwrite<float>(f, b.surf[i], j * (int)sizeof(float), k);
    } else {
        const unsigned short bits = MODE == 2 ? __bfloat16_as_ushort(__float2bfloat16_rn(f))
                                              : __half_as_ushort(__float2half_rn(f));
        surf2Dwrite<unsigned short>(bits, b.surf[i], j * (int)sizeof(unsigned short), k);
    }
}

// max|p| over the batch's images as float bits (non-negative floats order
// like their bits): a grid-stride pass per image (16-byte loads where every
// image of the batch is 16-byte aligned and a multiple of 4 pixels), a warp
// maximum, one atomic per warp.
__device__ __forceinline__ unsigned abs_bits(float f)
{
    return __float_as_uint(f) & 0x7fffffffu;
}

template <bool VEC>
__global__ void __launch_bounds__(256)
proj_absmax_kernel(const __grid_constant__ ConvBatch b, long long pixels, unsigned *pmax)
{
    const int i = blockIdx.y;
    if (i >= b.n)
        return;
    const float *src = b.src[i];
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, step = (long long)gridDim.x * blockDim.x;
    unsigned m0 = 0u, m1 = 0u;
    if constexpr (VEC) {
        const float4 *src4 = reinterpret_cast<const float4 *>(src);
        const long long n4 = pixels / 4;
        for (long long j = t0; j < n4; j += step) {
            const float4 v = src4[j];
            m0 = max(m0, max(abs_bits(v.x), abs_bits(v.y)));
            m1 = max(m1, max(abs_bits(v.z), abs_bits(v.w)));
        }
    } else {
        for (long long j = t0; j < pixels; j += step)
            m0 = max(m0, abs_bits(src[j]));
    }
    unsigned m = __reduce_max_sync(0xffffffffu, max(m0, m1));
    if ((threadIdx.x & 31) == 0 && m != 0u)
        atomicMax(pmax, m);
}

cudaError_t launch_proj_absmax(const ConvBatch &b, long long pixels, unsigned *pmax, cudaStream_t s)
{
    if (b.n <= 0 || pixels <= 0)
        return cudaSuccess;
    bool vec = pixels % 4 == 0;
    for (int j = 0; j < b.n; ++j)
        vec = vec && reinterpret_cast<uintptr_t>(b.src[j]) % 16 == 0;
    const long long work = vec ? pixels / 4 : pixels;
    const long long blocks = (work + 255) / 256;
    dim3 grid((unsigned)(blocks < 64 ? blocks : 64), b.n);
    if (vec)
        proj_absmax_kernel<true><<<grid, 256, 0, s>>>(b, pixels, pmax);
    else
        proj_absmax_kernel<false><<<grid, 256, 0, s>>>(b, pixels, pmax);
    return cudaGetLastError();
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
