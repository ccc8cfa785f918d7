// Backprojection with projections staged through TMA into shared memory
// (Sect. 3.1, Listing 1; the same arithmetic as bp_fwd.cu, different data
// path).
//
// Why: the texture unit returns 2x2 gathers of 32-bit texels at half the
// rate of 16-bit ones, which bounds the float32 form of the texture kernel.
// Here each block owns a 32 x 16 x 8 voxel brick.  For every projection the
// per-tile pre-pass (bp_fwd.cu) has projected the brick's 8 corners and
// decided to
//   * cull the projection when the footprint misses the detector (every
//     term is then exactly zero -- the line-wise clipping of Sect. 3.3 at
//     brick granularity), or
//   * load the footprint box of the projection's "pair image" with one
//     cp.async.bulk.tensor.2d into a stage of a shared-memory ring,
//     completing on an mbarrier; out-of-range rows/columns are zero-filled
//     by the TMA unit, which is the zero padding of Sect. 3.3, or
//   * (footprint larger than the box) use the bounds-checked global-memory
//     path.
// The block stages those decisions; one producer lane issues the copies of
// the projections the brick computes, and the consumers skip culled ones
// without touching the ring.
// The pair image stores element c = (p[c-1], p[c]) of each row (zero outside
// the detector), so the four corners of an update are two shared-memory
// loads: (tl, tr) from row iv and (bl, br) from row iv+1.  Float32 pairs
// hold (p[c-1], p[c] - p[c-1]) instead: the difference is the float32
// subtraction the horizontal interpolation needs anyway (the texture kernel
// computes the same one), done once per pixel instead of once per update.
//
// The coordinates, fractions and interpolation are computed exactly as in
// the texture kernel, so both paths give bit-identical volumes.
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

// Integer value of an integer-valued float with |f| < 2^22, without the
// float-to-int conversion unit: adding 1.5 * 2^23 puts the integer in the
// low mantissa bits.
constexpr float kIntMagic = 12582912.0f;
constexpr uint32_t kIntMagicBits = 0x4B400000u;
__device__ __forceinline__ int int_of_integral(float f)
{
    return __float_as_int(f + kIntMagic) - (int)kIntMagicBits;
}

// Shared-memory loads at a 32-bit shared address plus a constant offset.
template <int OFF>
__device__ __forceinline__ float2 lds_f2(uint32_t a)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2+%3];" : "=f"(v.x), "=f"(v.y) : "r"(a), "n"(OFF));
    return v;
}
template <int OFF>
__device__ __forceinline__ unsigned int lds_u32(uint32_t a)
{
    unsigned int v;
    asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(a), "n"(OFF));
    return v;
}

// The four corners of an update from two pair loads.  Pair = (left, right).
template <int KIND>
struct Pairs;

template <>
struct Pairs<kPairF32> {
    using T = float2;
    static constexpr bool kDiff = true;   // (left, right - left)
    __device__ static float2 unpack(float2 p) { return p; }
    template <int OFF>
    __device__ static float2 load(uint32_t a) { return lds_f2<OFF>(a); }
};

// 16-bit pairs unpack to (left, right - left) as well: the left pixel
// widened to float32, and the difference by one mixed-precision subtraction
// (the 16-bit right pixel widened exactly, minus the float32 left, rounded
// once: the float32 subtraction the texture kernel performs on the same two
// widened values).
template <>
struct Pairs<kPairF16> {
    using T = unsigned int;
    static constexpr bool kDiff = true;
    __device__ static float2 unpack(unsigned int p)
    {
        float l, d;
        asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\tcvt.f32.f16 %0, lo;\n\t"
            "sub.rn.f32.f16 %1, hi, %0;\n\t}"
            : "=f"(l), "=f"(d) : "r"(p));
        return make_float2(l, d);
    }
    template <int OFF>
    __device__ static float2 load(uint32_t a) { return unpack(lds_u32<OFF>(a)); }
};

template <>
struct Pairs<kPairBF16> {
    using T = unsigned int;
    static constexpr bool kDiff = true;
    __device__ static float2 unpack(unsigned int p)
    {
        float l, d;
        asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\tcvt.f32.bf16 %0, lo;\n\t"
            "sub.rn.f32.bf16 %1, hi, %0;\n\t}"
            : "=f"(l), "=f"(d) : "r"(p));
        return make_float2(l, d);
    }
    template <int OFF>
    __device__ static float2 load(uint32_t a) { return unpack(lds_u32<OFF>(a)); }
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Shared-memory stride of a ring stage: the box rounded up to a multiple of
// 128 bytes, the alignment a tensor copy's shared-memory destination needs.
template <int KIND>
struct TmaStage {
    static constexpr int kBytes = (int)sizeof(typename Pairs<KIND>::T) * TmaBox<KIND>::BU * TmaBox<KIND>::BV;
    static constexpr int kElems = ((kBytes + 127) / 128 * 128) / (int)sizeof(typename Pairs<KIND>::T);
    static_assert(kElems * (int)sizeof(typename Pairs<KIND>::T) % 128 == 0, "stage stride must be 128-byte aligned");
};

// The 16 updates of one consumer lane for projection i (matrix rows ru, rv,
// rw), reading the corner pairs from the staged tile (SMEM) or from the
// global pair image; the two forms are separate loop bodies so neither
// carries the other's work.  Lane voxels: X[kx] (kx = 0..3, 8 apart), one
// Y, Z[kz] (kz = 0..3, adjacent); absolute, or offsets from the brick
// centre with per-brick centring.  The row terms nest z outside y (as the
// texture kernel does), so the y term is formed once per projection.
template <int KIND, bool IEEE, bool SMEM>
__device__ __forceinline__ void tma_updates(const TmaBatch &b, int i, const float4 ru, const float4 rv,
                                            const float4 rw, int4 mt, uint32_t tile, const float (&X)[4],
                                            const float Y, const float (&Z)[4], float (&acc)[16])
{
    using P = Pairs<KIND>;
    using T = typename P::T;
    constexpr int BU = TmaBox<KIND>::BU;
    // mt is the box decision (1, off, cx0, ry0) or (2, cu, cv, 0).  SMEM:
    // off holds the bits of (row offset) * BU + (column offset) + 1.5 * 2^23,
    // so fv0 * BU + fu0 + off is the element index of the top pair in the
    // staged box, plus the magic, exactly (all integers far below 2^22); its
    // bits times the pair size, plus (tile - magic bits * pair size) modulo
    // 2^32, are the shared address.  Global: pair column floor(u') + cu, top
    // row floor(v') + cv.
    const float off = __int_as_float(mt.y);
    const uint32_t base = tile - kIntMagicBits * (uint32_t)sizeof(T);
    const float cu = fmaf(ru.y, Y, ru.w), cv = fmaf(rv.y, Y, rv.w), cw = fmaf(rw.y, Y, rw.w);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float bu = fmaf(ru.z, Z[q], cu);
        const float bv = fmaf(rv.z, Z[q], cv);
        const float bw = fmaf(rw.z, Z[q], cw);
#pragma unroll
        for (int kx = 0; kx < 4; ++kx) {
            const float uw = fmaf(ru.x, X[kx], bu);
            const float vw = fmaf(rv.x, X[kx], bv);
            const float w = fmaf(rw.x, X[kx], bw);
            const float r = recip_tma<IEEE>(w);
            const float u = uw * r, v = vw * r;
            const float fu0 = floorf(u), fv0 = floorf(v);
            float2 top, bot;
            if constexpr (SMEM) {
                // every lane's coordinates lie in the volume (clamped at
                // setup) and the box covers the brick's footprint with a pixel
                // of margin, so the address is inside the staged box
                const float e = fmaf(fv0, (float)BU, fu0 + off);
                const uint32_t a = (uint32_t)__float_as_int(e) * (uint32_t)sizeof(T) + base;
                top = P::template load<0>(a);
                bot = P::template load<BU * (int)sizeof(T)>(a);
            } else {
                // rows outside the detector are zero
                const int col = int_of_integral(fu0) + mt.y;
                const int row = int_of_integral(fv0) + mt.z;
                const T *img = reinterpret_cast<const T *>(b.img[i]);
                const bool cok = col >= 0 && col <= b.isx;
                const T *p = img + (long long)row * b.pitch + col;
                const T zero{};
                top = P::unpack(cok && row >= 0 && row < b.isy ? p[0] : zero);
                bot = P::unpack(cok && row + 1 >= 0 && row + 1 < b.isy ? p[b.pitch] : zero);
            }
            const float fu = u - fu0, fv = v - fv0;
            const float dt = P::kDiff ? top.y : top.y - top.x;
            const float db = P::kDiff ? bot.y : bot.y - bot.x;
            const float t = fmaf(fu, dt, top.x);
            const float bt = fmaf(fu, db, bot.x);
            const float fx = fmaf(fv, bt - t, t);
            acc[q * 4 + kx] = fmaf(fx, r * r, acc[q * 4 + kx]);
        }
    }
}

// Warp-specialised pipeline: warps 0..7 compute (256 consumer threads, 16
// voxels each), warp 8 is the producer.  Stage s of the S-deep ring
// has a "full" barrier (the producer's arrival, plus the TMA bytes when a
// tile is loaded) and an "empty" barrier (one arrival per consumer warp when
// it is done with the stage).  No block-wide barrier inside the loop.
// BLK: per-brick centring; the block stages the brick's centring records
// (u row, v row, (w_c, ku_b, kv_b)) of every projection in shared memory at
// the start, and consumers work with offsets from the brick centre, as the
// texture kernel does per block.
template <int KIND, bool IEEE, bool BLK>
__global__ void __launch_bounds__(kThreads + 32, 3)
bp_tma_kernel(const __grid_constant__ TmaBatch b, float *__restrict__ vol, const VolGeom g, int accumulate,
              int *__restrict__ err, unsigned long long *__restrict__ work)
{
    using P = Pairs<KIND>;
    using T = typename P::T;
    constexpr int BU = TmaBox<KIND>::BU, BV = TmaBox<KIND>::BV;
    constexpr int kBufElems = BU * BV;                  // pairs one box copy writes
    constexpr int kStageElems = TmaStage<KIND>::kElems;   // stage stride: 128-byte multiple
    constexpr int S = TmaBox<KIND>::S;
    constexpr int kConsumerWarps = kThreads / 32;
    // consumer layout: 8 x-lanes by 4 y-lanes per warp, warps 0-3 and 4-7
    // on the two 4-deep z halves; each lane 4 voxels along x (8 apart) and
    // 4 along z, covering the brick once
    static_assert(kBrickX == 8 * 4 && kBrickY == 4 * 4 && kBrickZ == 2 * 4 && kConsumerWarps == 8,
                  "the consumer layout tiles a 32 x 16 x 8 brick with 8 warps");
    extern __shared__ __align__(128) unsigned char dyn_smem[];   // the ring: S stages of kStageElems pairs
    T (*buf)[kStageElems] = reinterpret_cast<T (*)[kStageElems]>(dyn_smem);
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
    const int bx0 = blockIdx.x * kBrickX, by0 = blockIdx.y * kBrickY, bz0 = blockIdx.z * kBrickZ;
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
                mbar_expect_tx(&full[st], (uint32_t)(kBufElems * sizeof(T)));
                tma_load_2d(buf[st], &b.map[i], bi.z * kPairWords<KIND>, bi.w, &full[st]);
                issued |= 1 << st;
                last_par = (last_par & ~(1u << st)) | ((unsigned)(use & 1) << st);
            } else {
                mbar_arrive(&full[st]);
                issued &= ~(1 << st);
            }
        }
        if (computed) {
            const int xe = min(bx0 + kBrickX, L) - 1, ye = min(by0 + kBrickY, L) - 1;
            const int ze = min(bz0 + kBrickZ, g.Lz) - 1;
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
    // A warp is 8 lanes along x by 4 along y in one z plane of the brick:
    // its 32 voxels land on about the same detector rows, spread along
    // them, which keeps the shared-memory bank conflicts of the corner loads
    // low (a z-spread warp spans rows whose pitch aliases the banks).
    const int tx = lane & 7, ty = lane >> 3;
    // this lane's voxels: x0 + {0, 8, 16, 24}, y0, z0 + {0, 1, 2, 3};
    // lanes beyond a ragged edge compute with the last voxel's coordinates
    // (inside the brick box, so their loads stay in the staged tile) and
    // store nothing
    // (BLK: offsets from the centre of the brick's voxel box clipped to the
    // volume, (x0 + x1) / 2 etc., a multiple of 1/2, as in the pre-pass)
    const int x0 = bx0 + tx, y0 = by0 + 4 * (warp & 3) + ty, z0 = bz0 + 4 * (warp >> 2);
    const float hx = 0.5f * (float)(bx0 + min(bx0 + kBrickX, L) - 1);
    const float hy = 0.5f * (float)(by0 + min(by0 + kBrickY, L) - 1);
    const float hz = 0.5f * (float)(bz0 + min(bz0 + kBrickZ, g.Lz) - 1);
    float X[4], Z[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int x = min(x0 + 8 * k, L - 1), z = min(z0 + k, g.Lz - 1);
        X[k] = BLK ? g.R * ((float)x - hx) : fmaf(g.R, (float)x, g.Ox);
        Z[k] = BLK ? g.R * ((float)z - hz) : fmaf(g.R, (float)z, g.Oz);
    }
    const int yc = min(y0, L - 1);
    const float Y = BLK ? g.R * ((float)yc - hy) : fmaf(g.R, (float)yc, g.Oy);

    float acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k)
        acc[k] = 0.f;
    bool ok = true;
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
            ok = false;
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
                tma_updates<KIND, IEEE, true>(b, i, ru, rv, rw, mt, smem_u32(buf[s]), X, Y, Z, acc);
            else             // footprint larger than the tile
                tma_updates<KIND, IEEE, false>(b, i, ru, rv, rw, mt, 0u, X, Y, Z, acc);
        }
        __syncwarp();
        if (lane == 0)
            mbar_arrive(&empty[s]);   // this warp is done with stage s
        if (++s == S) {
            s = 0;
            phase ^= 1u;
        }
    }

    if (!ok)
        return;
    // the volume's read-modify-write; with final_out the same values also go
    // to the caller's destination (mapped host memory: the read-back of the
    // finished volume then overlaps this launch instead of following it)
    float *const fin = b.final_out;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int y = y0, z = z0 + q;
        if (y >= L || z >= g.Lz)
            continue;
        const size_t r0 = ((size_t)z * L + y) * L;
        float *row = vol + r0;
#pragma unroll
        for (int kx = 0; kx < 4; ++kx) {
            const int x = x0 + 8 * kx;
            if (x < L) {
                const float v = (accumulate ? row[x] : 0.f) + acc[q * 4 + kx];
                row[x] = v;
                if (fin)
                    fin[r0 + x] = v;
            }
        }
    }
}

template <int KIND, bool IEEE, bool BLK>
static cudaError_t launch_tma_blk(const TmaBatch &b, float *vol, const VolGeom &g, bool acc, int *err,
                                  unsigned long long *work, cudaStream_t s)
{
    dim3 grid((g.L + kBrickX - 1) / kBrickX, (g.L + kBrickY - 1) / kBrickY, (g.Lz + kBrickZ - 1) / kBrickZ);
    using T = typename Pairs<KIND>::T;
    const size_t smem = sizeof(T) * TmaStage<KIND>::kElems * TmaBox<KIND>::S;
    // the ring exceeds the 48 KB default for float32 pairs (set per call:
    // cheap, and correct on whichever device is current)
    cudaError_t e = cudaFuncSetAttribute(bp_tma_kernel<KIND, IEEE, BLK>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    bp_tma_kernel<KIND, IEEE, BLK><<<grid, kThreads + 32, smem, s>>>(b, vol, g, acc ? 1 : 0, err, work);
    return cudaGetLastError();
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
    switch (pair_kind) {
    case kPairF32:
        return ieee_rcp ? launch_tma_kind<kPairF32, true>(b, vol, g, accumulate, err, work, s)
                        : launch_tma_kind<kPairF32, false>(b, vol, g, accumulate, err, work, s);
    case kPairF16:
        return ieee_rcp ? launch_tma_kind<kPairF16, true>(b, vol, g, accumulate, err, work, s)
                        : launch_tma_kind<kPairF16, false>(b, vol, g, accumulate, err, work, s);
    default:
        return ieee_rcp ? launch_tma_kind<kPairBF16, true>(b, vol, g, accumulate, err, work, s)
                        : launch_tma_kind<kPairBF16, false>(b, vol, g, accumulate, err, work, s);
    }
}

// ---------------------------------------------------------------------------
// Pair images: element c of row k holds (p[k][c-1], p[k][c]) for
// c = 0 .. isx (zero outside the detector), in the storage type, or for
// float32 (p[k][c-1], p[k][c] - p[k][c-1]); elements c > isx of the padded
// row are zero.  One thread per element.
template <int KIND>
__global__ void __launch_bounds__(256)
pair_image_kernel(const __grid_constant__ PairBatch b, int isx, int isy, int pitch)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    const int i = blockIdx.z;
    if (c >= pitch || i >= b.n)
        return;
    const float *src = b.src[i] + (size_t)k * isx;
    const float l = (c >= 1 && c <= isx) ? src[c - 1] : 0.f;
    const float r = (c < isx) ? src[c] : 0.f;
    const size_t o = (size_t)k * pitch + c;
    if constexpr (KIND == kPairF32) {
        reinterpret_cast<float2 *>(b.dst[i])[o] = make_float2(l, __fsub_rn(r, l));
    } else if constexpr (KIND == kPairF16) {
        const __half2 h = __floats2half2_rn(l, r);
        reinterpret_cast<__half2 *>(b.dst[i])[o] = h;
    } else {
        const unsigned int lo = __bfloat16_as_ushort(__float2bfloat16_rn(l));
        const unsigned int hi = __bfloat16_as_ushort(__float2bfloat16_rn(r));
        reinterpret_cast<unsigned int *>(b.dst[i])[o] = lo | (hi << 16);
    }
}

cudaError_t launch_pair_images(const PairBatch &b, int isx, int isy, int pitch, int pair_kind, cudaStream_t s)
{
    if (b.n <= 0)
        return cudaSuccess;
    dim3 grid((pitch + 255) / 256, isy, b.n);
    if (pair_kind == kPairF32)
        pair_image_kernel<kPairF32><<<grid, 256, 0, s>>>(b, isx, isy, pitch);
    else if (pair_kind == kPairF16)
        pair_image_kernel<kPairF16><<<grid, 256, 0, s>>>(b, isx, isy, pitch);
    else
        pair_image_kernel<kPairBF16><<<grid, 256, 0, s>>>(b, isx, isy, pitch);
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
