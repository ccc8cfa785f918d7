// Backprojection with projections staged through TMA into shared memory
// (Sect. 3.1, Listing 1; the same geometry as bp_fwd.cu, different data
// path).
//
// Why: the texture unit returns 2x2 gathers of 32-bit texels at half the
// rate of 16-bit ones, which bounds the float32 form of the texture kernel.
// Here each block owns a 32 x 16 x (2 ZPL) voxel brick.  For every
// projection the per-tile pre-pass (bp_fwd.cu) has projected the brick's 8
// corners and decided to
//   * cull the projection when the footprint misses the detector (every
//     term is then exactly zero -- the line-wise clipping of Sect. 3.3 at
//     brick granularity), or
//   * load the footprint box of the projection's staged image with one
//     cp.async.bulk.tensor.2d into a stage of a shared-memory ring,
//     completing on an mbarrier; out-of-range rows/columns are zero-filled
//     by the TMA unit, which is the zero padding of Sect. 3.3, or
//   * (footprint larger than the box) use the bounds-checked global-memory
//     path.
// The block stages those decisions; one producer lane issues the copies of
// the projections the brick computes, and the consumers skip culled ones
// without touching the ring.
//
// Staged images hold 8-byte elements, so that the four corners of an update
// come from one or two shared-memory loads:
//   * float32 pair images: element c of row k = (p[k][c-1], p[k][c] -
//     p[k][c-1]); an update loads row iv and row iv + 1, and the difference
//     is the float32 subtraction the horizontal interpolation needs anyway,
//     done once per pixel instead of once per update;
//   * 16-bit column quads: element c of stored row k + 1 = the 16-bit pairs
//     (p[k][c-1], p[k+1][c-1] - p[k][c-1]) and (p[k][c] - p[k][c-1],
//     (p[k+1][c] - p[k+1][c-1]) - (p[k][c] - p[k][c-1])): the bilinear
//     coefficients of the pixel cell; an update loads one element, forms
//     both coefficient pairs along u with one packed two-lane FMA (fractions
//     rounded to the storage type), and the interpolant with one
//     mixed-precision FMA into float32.
// Coordinates, the weight 1/w^2 and the accumulation are float32 in every
// form (Sect. 3.1's single precision; the 16-bit forms only store the
// projections in 16 bits).
//
// Each thread accumulates its 4 ZPL voxels over the whole batch in
// registers; at the end the block stages its sums in shared memory and
// updates the volume with float4 loads and stores (coalesced rows of 32
// voxels), so the volume crosses HBM once per batch.
//
// Every wait on an mbarrier is bounded; on timeout the block records an
// error flag the host turns into BP_ETIMEOUT, the producer waits (bounded)
// for the copies it has in flight, and the block returns.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "bp_internal.cuh"

namespace bp {

template <bool IEEE>
__device__ __forceinline__ float recip_tma(float w)
{
    if constexpr (IEEE) {
        return __frcp_rn(w);
    } else {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(w));
        return r;
    }
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// try_wait with a suspend-time hint: a waiting warp sleeps (for at most
// the hint) until the phase completes instead of spinning on issue slots.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kTmaSuspendNs)
        : "memory");
    return done != 0;
}

// Bounded wait: at most iters suspensions of kTmaSuspendNs each.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int iters = kTmaWaitIters)
{
    for (int it = 0; it < iters; ++it)
        if (mbar_try_wait(bar, parity))
            return true;
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Barrier of the 256 consumer threads only (the producer warp has left).
__device__ __forceinline__ void consumers_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");
}

// Integer value of an integer-valued float with |f| < 2^22, without the
// float-to-int conversion unit: adding 1.5 * 2^23 puts the integer in the
// low mantissa bits.
constexpr float kIntMagic = 12582912.0f;
constexpr uint32_t kIntMagicBits = 0x4B400000u;
__device__ __forceinline__ int int_of_integral(float f)
{
    return __float_as_int(f + kIntMagic) - (int)kIntMagicBits;
}

// 8-byte shared-memory load at a 32-bit shared address plus a constant.
template <int OFF>
__device__ __forceinline__ uint2 lds_u2(uint32_t a)
{
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2+%3];" : "=r"(v.x), "=r"(v.y) : "r"(a), "n"(OFF));
    return v;
}

// The interpolated projection value fx of one update from its staged
// element(s).  e0: the element of row iv (pair column iu + 1); e1: the
// element of row iv + 1 (pair images only).  fu, fv: the fractions.
template <int KIND>
struct Interp;

template <>
struct Interp<kPairF32> {
    static constexpr bool kQuad = false;
    __device__ static float fx(uint2 e0, uint2 e1, float fu, float fv)
    {
        const float t = fmaf(fu, __uint_as_float(e0.y), __uint_as_float(e0.x));
        const float bt = fmaf(fu, __uint_as_float(e1.y), __uint_as_float(e1.x));
        return fmaf(fv, bt - t, t);
    }
};

// Coefficient quads: the element holds (tl, dv) and (dt, dd), with
// dv = bl - tl, dt = tr - tl and dd = (br - bl) - (tr - tl), so that
// fx = (tl + fu dt) + fv (dv + fu dd).  One conversion packs (fu, fv) into
// the storage type, one two-lane FMA gives (t, g) = (tl, dv) + fu (dt, dd),
// and one mixed-precision FMA (16-bit fv and g, float32 t widened exactly)
// gives fx = fv g + t in float32: four instructions per update (a form that
// interpolated the rows (tl, bl) + fu (dt, db) and subtracted them in
// float32 took five; measured 24.3 against 23.3 per update, 1527 against
// 1575 GUP/s f16, with 1.35x its rounding error, far inside the 16-bit
// forms' bars).
template <>
struct Interp<kQuadF16> {
    static constexpr bool kQuad = true;
    __device__ static float fx(uint2 e0, uint2, float fu, float fv)
    {
        unsigned f2, tg;
        float fx;
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(f2) : "f"(fv), "f"(fu));
        asm("{\n\t.reg .b16 lo, hi;\n\t.reg .b32 ff;\n\tmov.b32 {lo, hi}, %1;\n\tmov.b32 ff, {lo, lo};\n\t"
            "fma.rn.f16x2 %0, ff, %2, %3;\n\t}"
            : "=r"(tg) : "r"(f2), "r"(e0.y), "r"(e0.x));
        asm("{\n\t.reg .b16 tl, gh, fl, fh;\n\t.reg .f32 t;\n\tmov.b32 {tl, gh}, %1;\n\tmov.b32 {fl, fh}, %2;\n\t"
            "cvt.f32.f16 t, tl;\n\tfma.rn.f32.f16 %0, fh, gh, t;\n\t}"
            : "=f"(fx) : "r"(tg), "r"(f2));
        return fx;
    }
};

template <>
struct Interp<kQuadBF16> {
    static constexpr bool kQuad = true;
    __device__ static float fx(uint2 e0, uint2, float fu, float fv)
    {
        unsigned f2, tg;
        float fx;
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(f2) : "f"(fv), "f"(fu));
        asm("{\n\t.reg .b16 lo, hi;\n\t.reg .b32 ff;\n\tmov.b32 {lo, hi}, %1;\n\tmov.b32 ff, {lo, lo};\n\t"
            "fma.rn.bf16x2 %0, ff, %2, %3;\n\t}"
            : "=r"(tg) : "r"(f2), "r"(e0.y), "r"(e0.x));
        asm("{\n\t.reg .b16 tl, gh, fl, fh;\n\t.reg .f32 t;\n\tmov.b32 {tl, gh}, %1;\n\tmov.b32 {fl, fh}, %2;\n\t"
            "cvt.f32.bf16 t, tl;\n\tfma.rn.f32.bf16 %0, fh, gh, t;\n\t}"
            : "=f"(fx) : "r"(tg), "r"(f2));
        return fx;
    }
};

// Shared-memory stride of a ring stage: the box rounded up to a multiple of
// 128 bytes, the alignment a tensor copy's shared-memory destination needs.
template <int KIND, int ZPL>
struct TmaStage {
    static constexpr int BU = kTmaBU;
    static constexpr int BV = tma_rows(ZPL, Interp<KIND>::kQuad);
    static constexpr int kBytes = 8 * BU * BV;
    static constexpr int kElems = (kBytes + 127) / 128 * 128 / 8;
    static_assert(kElems * 8 % 128 == 0, "stage stride must be 128-byte aligned");
    // the brick's sums staged for the float4 epilogue: rows of 32 voxels at a
    // pitch of 40 floats (the 4 y-rows of a warp land 8 banks apart)
    static constexpr int kSumPitch = 40;
    static_assert(kTmaStages * kElems * 8 >= kSumPitch * kBrickY * 2 * ZPL * 4, "sums must fit the ring");
};

// The 4 ZPL updates of one consumer lane for projection i (matrix rows ru,
// rv, rw), reading the staged box (SMEM) or the global image; the two forms
// are separate loop bodies so neither carries the other's work.  Lane
// voxels: X[kx] (kx = 0..3, 8 apart), one Y, Z[q] (q < ZPL, adjacent);
// absolute, or offsets from the brick centre with per-brick centring.  The
// row terms nest z outside y, so the y term is formed once per projection.
template <int KIND, int ZPL, bool IEEE, bool SMEM>
__device__ __forceinline__ void tma_updates(const TmaBatch &b, int i, const float4 ru, const float4 rv,
                                            const float4 rw, int4 mt, uint32_t tile, const float (&X)[4], const float Y, const float (&Z)[ZPL],
                                            float (&acc)[4 * ZPL])
{
    using I = Interp<KIND>;
    constexpr int BU = kTmaBU;
    // mt is the box decision (1, off, cx0, ry0) or (2, cu, cv, 0).  SMEM:
    // off (mt.y) holds the bits of (row offset) * BU + (column offset) +
    // 1.5 * 2^23; off8 = 8 (off - 1.5 * 2^23) + 1.5 * 2^23, so
    // 8 fv0 BU + 8 fu0 + off8 is 8 times the element index in the staged box
    // (its byte offset), plus the magic, exactly (all integers far below
    // 2^22), and its bits plus (tile - magic bits) modulo 2^32 are the shared
    // address: two FP32 multiply-adds and one integer add per update (the
    // index times 8 in integer arithmetic took about three integer
    // instructions: 26.3 against 24.4 instructions per update, measured).
    // Global: element column floor(u') + cu, stored row floor(v') + cv.
    const float off8 = fmaf(__int_as_float(mt.y) - kIntMagic, 8.f, kIntMagic);
    const uint32_t base8 = tile - kIntMagicBits;
    const float cu = fmaf(ru.y, Y, ru.w), cv = fmaf(rv.y, Y, rv.w), cw = fmaf(rw.y, Y, rw.w);
#pragma unroll
    for (int q = 0; q < ZPL; ++q) {
        const float bu = fmaf(ru.z, Z[q], cu);
        const float bv = fmaf(rv.z, Z[q], cv);
        const float bw = fmaf(rw.z, Z[q], cw);
#pragma unroll
        for (int kx = 0; kx < 4; ++kx) {
            const float w = fmaf(rw.x, X[kx], bw);
            const float r = recip_tma<IEEE>(w);
            const float uw = fmaf(ru.x, X[kx], bu);
            const float vw = fmaf(rv.x, X[kx], bv);
            const float u = uw * r, v = vw * r;
            const float fu0 = floorf(u), fv0 = floorf(v);
            uint2 e0, e1 = make_uint2(0u, 0u);
            if constexpr (SMEM) {
                // every lane's coordinates lie in the volume (clamped at
                // setup) and the box covers the brick's footprint with a pixel
                // of margin, so the address is inside the staged box
                const float e8 = fmaf(fv0, (float)(8 * BU), fmaf(fu0, 8.f, off8));
                const uint32_t a = (uint32_t)__float_as_int(e8) + base8;
                e0 = lds_u2<0>(a);
                if constexpr (!I::kQuad)
                    e1 = lds_u2<BU * 8>(a);
            } else {
                // stored rows outside the image are zero (the TMA fill)
                const int col = int_of_integral(fu0) + mt.y;
                const int row = int_of_integral(fv0) + mt.z;
                const int rows = tma_image_rows(I::kQuad ? kQuadF16 : kPairF32, b.isy);
                const uint2 *img = reinterpret_cast<const uint2 *>(b.img[i]);
                const bool cok = col >= 0 && col <= b.isx;
                const uint2 *p = img + (long long)row * b.pitch + col;
                const uint2 zero = make_uint2(0u, 0u);
                e0 = cok && row >= 0 && row < rows ? p[0] : zero;
                if constexpr (!I::kQuad)
                    e1 = cok && row + 1 >= 0 && row + 1 < rows ? p[b.pitch] : zero;
            }
            const float fu = u - fu0, fv = v - fv0;
            const float fx = I::fx(e0, e1, fu, fv);
            acc[q * 4 + kx] = fmaf(fx, r * r, acc[q * 4 + kx]);
        }
    }
}

// Warp-specialised pipeline: warps 0..7 compute (256 consumer threads,
// 4 ZPL voxels each), warp 8 is the producer.  Stage s of the ring has a
// "full" barrier (the producer's arrival, plus the TMA bytes when a tile is
// loaded) and an "empty" barrier (one arrival per consumer warp when it is
// done with the stage).  No block-wide barrier inside the loop.
// BLK: per-brick centring; the block stages the brick's centring records
// (u row, v row, (w_c, ku_b, kv_b)) of every projection in shared memory at
// the start, and consumers work with offsets from the brick centre, as the
// texture kernel does per block.
template <int KIND, bool IEEE, bool BLK, int ZPL>
__global__ void __launch_bounds__(kThreads + 32, ZPL == 4 ? 3 : 2)
bp_tma_kernel(const __grid_constant__ TmaBatch b, float *__restrict__ vol, const VolGeom g, int accumulate,
              int *__restrict__ err, unsigned long long *__restrict__ work)
{
    using St = TmaStage<KIND, ZPL>;
    constexpr int kBufElems = St::BU * St::BV;       // elements one box copy writes
    constexpr int kStageElems = St::kElems;         // stage stride: 128-byte multiple
    constexpr int S = kTmaStages;
    constexpr int BZ = 2 * ZPL;
    constexpr int kConsumerWarps = kThreads / 32;
    // consumer layout: 8 x-lanes by 4 y-lanes per warp, warps 0-3 and 4-7
    // on the two ZPL-deep z halves; each lane 4 voxels along x (8 apart) and
    // ZPL along z, covering the brick once
    static_assert(kBrickX == 8 * 4 && kBrickY == 4 * 4 && kConsumerWarps == 8,
                  "the consumer layout tiles a 32 x 16 x 2 ZPL brick with 8 warps");
    extern __shared__ __align__(128) unsigned char dyn_smem[];   // the ring: S stages of kStageElems
    uint2(*buf)[kStageElems] = reinterpret_cast<uint2(*)[kStageElems]>(dyn_smem);
    __shared__ __align__(8) uint64_t full[S], empty[S];
    // the brick's box decision for every projection of the batch (made by
    // the pre-pass: culled / staged box / global path, with its offsets),
    // and with BLK its centring records (u row, v row, (w_c, ku_b, kv_b)),
    // staged once
    __shared__ int4 box[kMaxBatch];
    __shared__ float4 rec[3][BLK ? kMaxBatch : 1];
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = g.L;
    const int bx0 = blockIdx.x * kBrickX, by0 = blockIdx.y * kBrickY, bz0 = blockIdx.z * BZ;
    const size_t brick = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;

    if (threadIdx.x == 0) {
        for (int q = 0; q < S; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], kConsumerWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    if (threadIdx.x < kMaxBatch && threadIdx.x < b.n)
        box[threadIdx.x] = b.boxes[(size_t)threadIdx.x * b.bricks + brick];
    if constexpr (BLK) {
        if (threadIdx.x < 3 * kMaxBatch) {
            const int part = threadIdx.x / kMaxBatch, i = threadIdx.x % kMaxBatch;
            if (i < b.n)
                rec[part][i] = b.centres[((size_t)part * kMaxBatch + i) * b.bricks + brick];
        }
    }
    __syncthreads();

    if (warp == kConsumerWarps) {
        // ---------------- producer: one lane starts the copies of the
        // projections the brick computes, in order, into the ring
        if (lane != 0)
            return;
        int issued = 0;            // stages whose tile may still be in flight
        unsigned last_par = 0;     // bit q: phase parity of stage q's last tile
        unsigned long long computed = 0;
        int k = 0;                 // projections computed so far
        for (int i = 0; i < b.n; ++i) {
            const int4 bi = box[i];
            if (bi.x == 0)
                continue;          // culled: no stage, no barrier
            const int st = k % S, use = k / S;
            ++k;
            if (use > 0 && !mbar_wait_bounded(&empty[st], (use - 1) & 1)) {
                atomicExch(&abort_flag, 1);
                atomicExch(err, 1);
                break;
            }
            if (*(volatile int *)&abort_flag)
                break;
            ++computed;
            if (bi.x == 1) {
                mbar_expect_tx(&full[st], (uint32_t)(kBufElems * 8));
                tma_load_2d(buf[st], &b.map[i], bi.z * 2, bi.w, &full[st]);
                issued |= 1 << st;
                last_par = (last_par & ~(1u << st)) | ((unsigned)(use & 1) << st);
            } else {
                mbar_arrive(&full[st]);
                issued &= ~(1 << st);
            }
        }
        if (computed) {
            const int xe = min(bx0 + kBrickX, L) - 1, ye = min(by0 + kBrickY, L) - 1;
            const int ze = min(bz0 + BZ, g.Lz) - 1;
            atomicAdd(work, computed * (unsigned long long)((xe - bx0 + 1) * (ye - by0 + 1) * (ze - bz0 + 1)));
        }
        if (*(volatile int *)&abort_flag) {
            // let copies still in flight land before the block's memory goes away
            for (int q = 0; q < S; ++q)
                if (issued & (1 << q))
                    mbar_wait_bounded(&full[q], (last_par >> q) & 1u);
        }
        return;
    }

    // ---------------- consumers
    // A warp is 8 lanes along x by 4 along y in one z plane of the brick,
    // numbered so that each half-warp is a 4 x 4 patch (x 0-3 and x 4-7):
    // the shared-memory unit serves a warp's 8-byte loads per half-warp, and
    // a compact patch's corners span few elements of one or two detector
    // rows (a z-spread warp spans rows whose pitch aliases the banks; an
    // 8 x 2 half-warp spans more elements than the 16 banks pairs).
    const int tx = (lane & 3) | ((lane >> 4) << 2), ty = (lane >> 2) & 3;
    const int yl = 4 * (warp & 3) + ty, zl0 = ZPL * (warp >> 2);
    // this lane's voxels: x0 + {0, 8, 16, 24}, y0, z0 + {0 .. ZPL-1};
    // lanes beyond a ragged edge compute with the last voxel's coordinates
    // (inside the brick box, so their loads stay in the staged tile) and
    // store nothing
    // (BLK: offsets from the centre of the brick's voxel box clipped to the
    // volume, (x0 + x1) / 2 etc., a multiple of 1/2, as in the pre-pass)
    const int x0 = bx0 + tx, y0 = by0 + yl, z0 = bz0 + zl0;
    const float hx = 0.5f * (float)(bx0 + min(bx0 + kBrickX, L) - 1);
    const float hy = 0.5f * (float)(by0 + min(by0 + kBrickY, L) - 1);
    const float hz = 0.5f * (float)(bz0 + min(bz0 + BZ, g.Lz) - 1);
    float X[4], Z[ZPL];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int x = min(x0 + 8 * k, L - 1);
        X[k] = BLK ? g.R * ((float)x - hx) : fmaf(g.R, (float)x, g.Ox);
    }
#pragma unroll
    for (int q = 0; q < ZPL; ++q) {
        const int z = min(z0 + q, g.Lz - 1);
        Z[q] = BLK ? g.R * ((float)z - hz) : fmaf(g.R, (float)(z + g.z0), g.Oz);
    }
    const int yc = min(y0, L - 1);
    const float Y = BLK ? g.R * ((float)yc - hy) : fmaf(g.R, (float)yc, g.Oy);

    float acc[4 * ZPL];
#pragma unroll
    for (int k = 0; k < 4 * ZPL; ++k)
        acc[k] = 0.f;
    int s = 0;
    uint32_t phase = 0;
#pragma unroll 1
    for (int i = 0; i < b.n; ++i) {
        const int4 mt = box[i];
        if (mt.x == 0)
            continue;   // culled by the pre-pass: every term is exactly zero
        if (!mbar_wait_bounded(&full[s], phase)) {
            if (lane == 0) {
                atomicExch(&abort_flag, 1);
                atomicExch(err, 1);
            }
            break;
        }
        {
            float4 ru, rv, rw = b.m[i][2];
            if constexpr (BLK) {
                ru = rec[0][i];
                rv = rec[1][i];
                rw.w = rec[2][i].x;
            } else {
                ru = b.m[i][0];
                rv = b.m[i][1];
            }
            if (mt.x == 1)   // tile in shared memory (the common case)
                tma_updates<KIND, ZPL, IEEE, true>(b, i, ru, rv, rw, mt, smem_u32(buf[s]), X, Y, Z, acc);
            else             // footprint larger than the tile
                tma_updates<KIND, ZPL, IEEE, false>(b, i, ru, rv, rw, mt, 0u, X, Y, Z, acc);
        }
        __syncwarp();
        if (lane == 0)
            mbar_arrive(&empty[s]);   // this warp is done with stage s
        if (++s == S) {
            s = 0;
            phase ^= 1u;
        }
    }

    // Every consumer warp is past its last wait, so every copy the producer
    // issued has landed and the ring is free.
    consumers_sync();
    if (*(volatile int *)&abort_flag)
        return;
    // The brick's sums, staged as rows of 32 voxels (x fastest), then the
    // volume's read-modify-write with float4 accesses: 8 threads per row of
    // 32 voxels.  With final_out the same values also go to the caller's
    // destination (mapped host memory: the read-back of the finished volume
    // then overlaps this launch instead of following it).
    float *sums = reinterpret_cast<float *>(dyn_smem);
    constexpr int P = St::kSumPitch;
    // a batch staged with a power-of-four scale 2^(-2k) (b.pmax, 16-bit
    // storage): the sums times 2^(2k), exactly
    float vs = 1.f;
    if constexpr (KIND != kPairF32)
        vs = b.pmax ? pow2f(2 * proj_scale_k(*b.pmax)) : 1.f;
#pragma unroll
    for (int q = 0; q < ZPL; ++q)
#pragma unroll
        for (int kx = 0; kx < 4; ++kx)
            sums[((zl0 + q) * kBrickY + yl) * P + tx + 8 * kx] = acc[q * 4 + kx] * vs;
    consumers_sync();
    float *const fin = b.final_out;
#pragma unroll
    for (int f = threadIdx.x; f < kBrickX / 4 * kBrickY * BZ; f += kThreads) {
        const int xq = f & 7, ys = (f >> 3) % kBrickY, zs = (f >> 3) / kBrickY;
        const int x = bx0 + 4 * xq, y = by0 + ys, z = bz0 + zs;
        if (y >= L || z >= g.Lz || x >= L)
            continue;
        const float4 a = *reinterpret_cast<const float4 *>(&sums[(zs * kBrickY + ys) * P + 4 * xq]);
        const size_t o = ((size_t)z * L + y) * L + x;
        if (b.vec4 && x + 3 < L) {
            float4 v = a;
            if (accumulate) {
                const float4 old = *reinterpret_cast<const float4 *>(vol + o);
                v = make_float4(old.x + a.x, old.y + a.y, old.z + a.z, old.w + a.w);
            }
            *reinterpret_cast<float4 *>(vol + o) = v;
            if (fin)
                *reinterpret_cast<float4 *>(fin + o) = v;
        } else {
            const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (x + j < L) {
                    const float v = (accumulate ? vol[o + j] : 0.f) + av[j];
                    vol[o + j] = v;
                    if (fin)
                        fin[o + j] = v;
                }
            }
        }
    }
}

template <int KIND, bool IEEE, bool BLK, int ZPL>
static cudaError_t launch_tma_zpl(const TmaBatch &b, float *vol, const VolGeom &g, bool acc, int *err,
                                  unsigned long long *work, cudaStream_t s)
{
    dim3 grid((g.L + kBrickX - 1) / kBrickX, (g.L + kBrickY - 1) / kBrickY, (g.Lz + 2 * ZPL - 1) / (2 * ZPL));
    const size_t smem = 8 * (size_t)TmaStage<KIND, ZPL>::kElems * kTmaStages;
    // the ring exceeds the 48 KB default (set per call: cheap, and correct
    // on whichever device is current)
    cudaError_t e = cudaFuncSetAttribute(bp_tma_kernel<KIND, IEEE, BLK, ZPL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    bp_tma_kernel<KIND, IEEE, BLK, ZPL><<<grid, kThreads + 32, smem, s>>>(b, vol, g, acc ? 1 : 0, err, work);
    return cudaGetLastError();
}

template <int KIND, bool IEEE, bool BLK>
static cudaError_t launch_tma_blk(const TmaBatch &b, float *vol, const VolGeom &g, bool acc, int *err,
                                  unsigned long long *work, cudaStream_t s)
{
    switch (b.zpl) {
    case 8:
        return launch_tma_zpl<KIND, IEEE, BLK, 8>(b, vol, g, acc, err, work, s);
    case 6:
        return launch_tma_zpl<KIND, IEEE, BLK, 6>(b, vol, g, acc, err, work, s);
    default:
        return launch_tma_zpl<KIND, IEEE, BLK, 4>(b, vol, g, acc, err, work, s);
    }
}

// Per-brick centring exists for the float32 pairs only (16-bit storage
// rounds far above the coordinate error it removes).
template <int KIND, bool IEEE>
static cudaError_t launch_tma_kind(const TmaBatch &b, float *vol, const VolGeom &g, bool acc, int *err,
                                   unsigned long long *work, cudaStream_t s)
{
    if constexpr (KIND == kPairF32) {
        if (b.centres)
            return launch_tma_blk<KIND, IEEE, true>(b, vol, g, acc, err, work, s);
    }
    return launch_tma_blk<KIND, IEEE, false>(b, vol, g, acc, err, work, s);
}

cudaError_t launch_bp_tma(const TmaBatch &b, float *vol, const VolGeom &g, int pair_kind, bool accumulate,
                          bool ieee_rcp, int *err, unsigned long long *work, cudaStream_t s)
{
    if (b.n <= 0)
        return cudaSuccess;
    if (b.zpl != 4 && b.zpl != 6 && b.zpl != 8)
        return cudaErrorInvalidValue;
    switch (pair_kind) {
    case kPairF32:
        return ieee_rcp ? launch_tma_kind<kPairF32, true>(b, vol, g, accumulate, err, work, s)
                        : launch_tma_kind<kPairF32, false>(b, vol, g, accumulate, err, work, s);
    case kQuadF16:
        return ieee_rcp ? launch_tma_kind<kQuadF16, true>(b, vol, g, accumulate, err, work, s)
                        : launch_tma_kind<kQuadF16, false>(b, vol, g, accumulate, err, work, s);
    default:
        return ieee_rcp ? launch_tma_kind<kQuadBF16, true>(b, vol, g, accumulate, err, work, s)
                        : launch_tma_kind<kQuadBF16, false>(b, vol, g, accumulate, err, work, s);
    }
}

// ---------------------------------------------------------------------------
// Staged images, one thread per element (zero outside the detector):
//   float32 pairs: element c of row k = (p[k][c-1], p[k][c] - p[k][c-1]),
//     rows k = 0 .. isy - 1;
//   16-bit column quads: element c of stored row j (image row k = j - 1,
//     j = 0 .. isy) = ((tl, bl - tl), (tr - tl, (br - bl) - (tr - tl))) with
//     tl = p[k][c-1], tr = p[k][c], bl = p[k+1][c-1], br = p[k+1][c], each
//     value rounded once to the storage type (the differences taken in
//     float32 first);
// for c = 0 .. isx; elements c > isx of the padded row are zero.
__device__ __forceinline__ float pix(const float *src, int isx, int isy, int k, int c)
{
    return (k >= 0 && k < isy && c >= 0 && c < isx) ? src[(size_t)k * isx + c] : 0.f;
}

template <int KIND>
__global__ void __launch_bounds__(256)
pair_image_kernel(const __grid_constant__ PairBatch b, int isx, int isy, int pitch)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int i = blockIdx.z;
    if (c >= pitch || i >= b.n)
        return;
    const float *src = b.src[i];
    const size_t o = (size_t)j * pitch + c;
    uint2 *dst = reinterpret_cast<uint2 *>(b.dst[i]);
    const bool in = c <= isx;
    if constexpr (KIND == kPairF32) {
        const float l = in ? pix(src, isx, isy, j, c - 1) : 0.f;
        const float r = in ? pix(src, isx, isy, j, c) : 0.f;
        dst[o] = make_uint2(__float_as_uint(l), __float_as_uint(__fsub_rn(r, l)));
    } else {
        const int k = j - 1;
        // the batch's power-of-four scale (exact; 1 without one)
        const float sc = b.pmax ? pow2f(-2 * proj_scale_k(*b.pmax)) : 1.f;
        const float tl = (in ? pix(src, isx, isy, k, c - 1) : 0.f) * sc;
        const float tr = (in ? pix(src, isx, isy, k, c) : 0.f) * sc;
        const float bl = (in ? pix(src, isx, isy, k + 1, c - 1) : 0.f) * sc;
        const float br = (in ? pix(src, isx, isy, k + 1, c) : 0.f) * sc;
        // (tl, dv) and (dt, dd): dv = bl - tl, dt = tr - tl, dd = (br - bl) - dt
        const float dt = __fsub_rn(tr, tl), dv = __fsub_rn(bl, tl), dd = __fsub_rn(__fsub_rn(br, bl), dt);
        unsigned lo, hi;
        if constexpr (KIND == kQuadF16) {
            lo = (unsigned)__half_as_ushort(__float2half_rn(tl)) | ((unsigned)__half_as_ushort(__float2half_rn(dv)) << 16);
            hi = (unsigned)__half_as_ushort(__float2half_rn(dt)) | ((unsigned)__half_as_ushort(__float2half_rn(dd)) << 16);
        } else {
            lo = (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(tl)) |
                 ((unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(dv)) << 16);
            hi = (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(dt)) |
                 ((unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(dd)) << 16);
        }
        dst[o] = make_uint2(lo, hi);
    }
}

cudaError_t launch_pair_images(const PairBatch &b, int isx, int isy, int pitch, int pair_kind, cudaStream_t s)
{
    if (b.n <= 0)
        return cudaSuccess;
    dim3 grid((pitch + 255) / 256, tma_image_rows(pair_kind, isy), b.n);
    if (pair_kind == kPairF32)
        pair_image_kernel<kPairF32><<<grid, 256, 0, s>>>(b, isx, isy, pitch);
    else if (pair_kind == kQuadF16)
        pair_image_kernel<kQuadF16><<<grid, 256, 0, s>>>(b, isx, isy, pitch);
    else
        pair_image_kernel<kQuadBF16><<<grid, 256, 0, s>>>(b, isx, isy, pitch);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Self-test of the bounded wait (failure detection without a GPU fault): one
// warp waits, with the backprojection kernel's helper, on an mbarrier that
// lane 0 completes (arrive) or that nothing completes; after iters
// suspensions the wait gives up, and lane 0 records the error flag the host
// turns into BP_ETIMEOUT, as the backprojection kernel does.
__global__ void __launch_bounds__(32) wait_selftest_kernel(int arrive, int iters, int *err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (arrive && threadIdx.x == 0)
        mbar_arrive(&bar);
    __syncwarp();
    if (!mbar_wait_bounded(&bar, 0, iters) && threadIdx.x == 0)
        atomicExch(err, 1);
}

}  // namespace bp

extern "C" bp_status bp_selftest_bounded_wait(int arrive, int iters)
{
    if ((arrive != 0 && arrive != 1) || iters < 1 || iters > (1 << 20)) {
        bp::set_thread_error("bp_selftest_bounded_wait: arrive must be 0 or 1 and iters in [1, 2^20]");
        return BP_EINVAL;
    }
    int *err = nullptr, flag = 0;
    cudaError_t e = cudaMalloc((void **)&err, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess) {
        bp::wait_selftest_kernel<<<1, 32>>>(arrive, iters, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(&flag, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (err)
        cudaFree(err);
    if (e != cudaSuccess) {
        bp::set_thread_error("bp_selftest_bounded_wait: %s", cudaGetErrorString(e));
        return BP_ECUDA;
    }
    if (flag) {
        bp::set_thread_error("bp_selftest_bounded_wait: the wait gave up after %d suspensions", iters);
        return BP_ETIMEOUT;
    }
    return BP_OK;
}
