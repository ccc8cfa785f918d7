// Internal declarations shared by the library's translation units.
// Nothing here is part of the C ABI (that is include/bp1104.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "../../include/bp1104.h"

namespace bp {

// Projections per volume pass: the kernel keeps its voxels' sums in
// registers over the whole batch, so the volume crosses HBM once per batch
// (the image blocking of Sect. 6.2, with b = kMaxBatch).
constexpr int kMaxBatch = 64;

// Thread blocks of 256 threads = 8 warps, one warp per y row of the tile.
// A warp is LX lanes along x by 32/LX lanes along z; each lane owns
// kVoxPerLane voxels along x at stride LX, so for each of them the warp's 32
// samples are neighbouring voxels whose projections form a compact patch on
// the detector (texture-cache friendly).
constexpr int kThreads = 256, kWarpsY = 8, kVoxPerLane = 4;

// One batch of projections for the backprojection kernel, passed by value
// (kernel parameter space): per projection the three matrix rows as float4
// (a0, a1, a2, a3), the integer offsets (ku, kv) the u and v rows were
// centred on, and the texture holding the image.  The host folds the
// centring into the rows in float64: row_u' = row_u - (ku - 1) row_w (and
// likewise for v), so u' = u - ku + 1 stays small (precise in float32) and
// the gather coordinate floor(u') + ku = floor(u) + 1 is an exact integer.
struct FwdBatch {
    float4 m[kMaxBatch][3];
    float2 k[kMaxBatch];
    cudaTextureObject_t tex[kMaxBatch];
    const unsigned *pmax;              // the batch's max|p| bits (proj_scale_k), NULL: no scale
    int n;
};

// Power-of-four scale of 16-bit storage (BP_OPT_PROJ_SCALE), one per batch.
// From the bits of max|p| over the batch's projections (a non-negative
// float, whose bits order like the values), the k for which
// max|p| * 2^(-2k) lies in [2^12, 2^14): the staged values are p * 2^(-2k),
// far from float16's overflow (65504, also for the pair differences, at
// most twice the maximum) and from its subnormals (below 2^-14), and the
// kernels multiply the batch's sums by 2^(2k).  Every term of a sum carries
// the same factor 2^(-2k), so the scaled sums are the unscaled ones times
// that power of two, exactly: the volume is bit-identical wherever the
// unscaled staging is exact in its range.  k = 0 for an all-zero, infinite
// or NaN batch; k is clamped to [-63, 63] (maxima below 2^-113 or above
// 2^127 keep a smaller scaled maximum, or a larger one).
__host__ __device__ inline int proj_scale_k(unsigned max_bits)
{
    if (max_bits == 0u || max_bits >= 0x7f800000u)
        return 0;
    const unsigned ex = max_bits >> 23, man = max_bits & 0x7fffffu;
    int e;   // floor(log2(max|p|))
    if (ex != 0) {
        e = (int)ex - 127;
    } else {
        int hb = 22;
        while (((man >> hb) & 1u) == 0u)
            --hb;
        e = hb - 149;
    }
    const int t = e - 13;
    const int k = (t + (t & 1)) / 2;
    return k < -63 ? -63 : k > 63 ? 63 : k;   // 2^(-2k) stays a normal float
}

// 2^q as a float for |q| <= 126.
__host__ __device__ inline float pow2f(int q)
{
    union {
        unsigned u;
        float f;
    } v;
    v.u = (unsigned)(127 + q) << 23;
    return v.f;
}

// Four values of the scalar type T: float4 for float, a plain aggregate for
// double (the direct kernels are templates on T; the float64 instantiation
// serves gradient checks only).
struct Dbl4 {
    double x, y, z, w;
};
template <typename T> struct Vec4Of;
template <> struct Vec4Of<float> { using type = float4; };
template <> struct Vec4Of<double> { using type = Dbl4; };
template <typename T> using Vec4 = typename Vec4Of<T>::type;

// Same for the adjoint: centred matrix rows (row_u - ku row_w), the offsets
// as integers, and the output image offset.
template <typename T>
struct AdjBatchT {
    Vec4<T> m[kMaxBatch][3];
    int2 k[kMaxBatch];
    long long out_off[kMaxBatch];
    const float4 *centres;   // per-block centring records (shared-tile kernel; NULL: per projection)
    long long blocks;        // blocks of the volume (record plane stride)
    int n;
};
using AdjBatch = AdjBatchT<float>;
// The shared-tile adjoint kernel's block of voxels (the pre-pass tile for
// its centring records).
constexpr int kAdjBlockX = 32, kAdjBlockY = 32, kAdjBlockZ = 4;

// Volume: L x L x Lz voxels (x fastest; Lz = L for a cube, Lz < L for a
// z-slab of an L^3 grid), voxel size R, centre of voxel (0,0,0) at O.
template <typename T>
struct VolGeomT {
    int L, Lz;
    T R, Ox, Oy, Oz;
    // first slice of a z-slab in the L^3 grid (0 for the whole cube); Oz is
    // the cube's origin, so a slice's z coordinate R (z + z0) + Oz is formed
    // identically by a slab context and by one holding the whole cube
    int z0;
};
using VolGeom = VolGeomT<float>;

// Texture storage kinds: float channel (FP32 or FP16 arrays; the texture
// unit widens FP16 exactly) or raw 16-bit words holding BF16.
enum TexKind { kTexFloat = 0, kTexBF16 = 1 };

// Per-block centring (float32 form).  Centring once per projection leaves
// |u'| up to the half-width of the volume's footprint (hundreds of pixels on
// a full detector), and the float32 rounding of u' there is what limits the
// accuracy.  With per-block centring, every (thread block, projection) gets
// its own integer offsets ku_b = ku + dku, kv_b = kv + dkv (the pixel the
// block centre projects to).  It also gets the centred rows' values at the
// block centre, uw_c = (row_u - (ku_b - 1) row_w) . (x_c, 1), likewise vw_c,
// and w_c.  These are computed as float-float sums (about 44 significant bits)
// and rounded to float32 once.  The kernel then works with offsets from the
// block centre, where every float32 quantity stays small.
//
// CentreBatch: for each projection and row r = (u', v', w) of the
// per-projection-centred matrix, the row's value at voxel (0,0,0) and its
// change per half voxel along x, y, z, each a float64 value split into a
// float32 (hi, lo) pair.  A block is centred on the centre of its voxel box
// clipped to the volume, at half-integer voxel indices.  The pre-pass writes
// three float4 per (block, projection): the u row recentred on the block,
// (row_u'' x, y, z, uw_c), the same for v, and (w_c, ku_b, kv_b, 0), in three
// planes at index (part * 64 + projection) * blocks + block.
struct CentreBatch {
    float2 c[kMaxBatch][3][4];
};

// Fills cb from the float64 centred rows (n x 3 x 4: u', v', w).
void centre_batch(CentreBatch *cb, const double *rows, int n, const double O[3], double R);

// masks: one 64-bit word per thread block of the texture kernel, bit i set
// when projection i of the batch can reach the block's voxels (NULL: no
// culling).  centres: the per-block centring records (NULL: per-projection
// centring; only the float-channel kind supports it).  Both are built by
// launch_block_prepass for the same layout.
cudaError_t launch_bp_fwd(const FwdBatch &b, float *vol, const VolGeom &g, int tex_kind,
                          bool accumulate, bool ieee_rcp, int lanes_x, const unsigned long long *masks,
                          const float4 *centres, cudaStream_t s);

// The per-tile pre-pass (one thread per tile of voxels: the texture
// kernel's block, fwd_tile of its layout; the TMA path's brick; the tile
// adjoint's block), writing for every projection of the batch
// - masks (if not NULL): a tile's bit for projection i is cleared when the
//   projections of its voxel box miss the detector by more than a pixel
//   (every term of those updates is exactly zero);
// - centres (if not NULL, with cb): the tile's centring records;
// - boxes (if not NULL, with box): the TMA path's box decisions (below);
// - work (if not NULL): the kept updates are added to *work.
// tile_count: tiles of an L x L x Lz volume.
void fwd_tile(int lanes_x, int *tx, int *ty, int *tz);
long long tile_count(int L, int Lz, int tx, int ty, int tz);
// TMA-path box decision per (brick, projection), made by the pre-pass
// (boxes, one int4 per pair at index projection * bricks + brick):
//   (0, 0, 0, 0)            the footprint misses the detector: skip;
//   (1, off, cx0, ry0)      load the BU x BV pair box at pair column cx0,
//                           row ry0; off = float bits of (row offset * BU +
//                           column offset + 1.5 * 2^23), see bp_tma.cu;
//   (2, cu, cv, 0)          footprint larger than the box: read the pair
//                           image from global memory, pair column floor(u')
//                           + cu, top row floor(v') + cv.
// The offsets are relative to the brick's centring offsets with per-brick
// centring, else to the projection's.
struct BoxSpec {
    int bu, bv, align;   // box columns and rows (elements), column alignment (elements)
    int quad;            // column quads: an element carries rows k and k + 1, stored at row k + 1
};
// zoff2: twice the global index of the volume's first slice (a z-slab of
// the L^3 grid), so that the centring records of a slab's tiles are those
// of the same tiles of the whole grid (cb built from the grid's origin).
cudaError_t launch_block_prepass(const FwdBatch &b, const CentreBatch *cb, const VolGeom &g, int isx, int isy,
                                 int tx, int ty, int tz, int zoff2, unsigned long long *masks, float4 *centres,
                                 const BoxSpec *box, int4 *boxes, unsigned long long *work, cudaStream_t s);

// smem: accumulate each block's footprint in shared memory (kAdjTile pixels
// at most) and add it to the image with one atomic per touched pixel.
constexpr int kAdjTile = 3072;
cudaError_t launch_bp_adjoint(const AdjBatch &b, const float *vol, const VolGeom &g,
                              float *out, int isx, int isy, bool ieee_rcp, bool smem, cudaStream_t s);

// ---------------------------------------------------------------------------
// TMA / shared-memory path (bp_tma.cu).  Bricks of 32 x 16 x (2 ZPL) voxels
// per block of 256 consumer threads (4 ZPL voxels each) and one producer
// warp; projections staged as images of 8-byte elements, loaded per brick
// and projection as one TMA box of BU element columns by BV rows:
//   * float32 "pair images": element c of row k holds (p[k][c-1],
//     p[k][c] - p[k][c-1]); an update reads two elements (rows iv, iv+1);
//   * 16-bit "column quads": element c of stored row j (image row k = j - 1)
//     holds the pixel cell's bilinear coefficients as 16-bit pairs
//     (tl, bl - tl) and (tr - tl, (br - bl) - (tr - tl)) (tl = p[k][c-1],
//     tr = p[k][c], bl = p[k+1][c-1], br = p[k+1][c]), the differences taken
//     in float32 and rounded once; an update reads one element, forms both
//     coefficient pairs along u with one packed two-lane FMA and the
//     interpolant with one mixed-precision FMA.
// ZPL (voxels per lane along z) sets the brick depth: 4, 6 or 8 (8-, 12-
// and 16-deep bricks).  Deeper bricks spread the per-projection work of a
// thread over more updates but need taller boxes; the host picks, per
// batch, the deepest brick whose box holds the sampled footprints.  The box
// heights come from a CPU model of the pre-pass's box rule over the 512^3
// C-arm scan: 36 rows hold 99.7 % of the visible 8-deep footprints, 48 rows
// 99.7 % of the 12-deep ones and 58 rows (as tall as two blocks per SM
// allow) 98.9 % of the 16-deep ones; larger footprints (bricks near the
// source, near the top and bottom of the volume) read the image from
// global memory.
//
// The box is 120 elements wide (114 hold 99.99 % of the footprints): its row
// pitch of 240 words is 16 modulo 32, so an element and the one a row below
// it sit 16 banks apart.  A warp's 8-byte loads are served per half-warp;
// a half-warp covers 4 x 4 voxels, whose corners span about 10 elements of
// one or two rows, and the 16-bank shift keeps two rows' elements apart
// (a CPU model of the bank accounting, checked against ncu: 1.34 wavefronts
// per load against 1.84 with a 114-element pitch and 8 x 2 half-warps).
constexpr int kBrickX = 32, kBrickY = 16;
enum PairKind { kPairF32 = 0, kQuadF16 = 1, kQuadBF16 = 2 };
constexpr int kTmaBU = 120;   // element columns (and row pitch) of a staged box
constexpr int kTmaAlign = 2;  // element-column alignment that keeps the box origin on 16 bytes
// Box rows of the float32 pair images per ZPL; a column-quad box is one row
// shorter (each element carries the row below).
__host__ __device__ constexpr int tma_rows(int zpl, bool quad)
{
    return (zpl == 4 ? 36 : zpl == 6 ? 48 : 58) - (quad ? 1 : 0);
}
constexpr int kTmaStages = 2;
constexpr int kTmaWaitIters = 1 << 14;          // bounded waits: at most ~2 s
constexpr unsigned kTmaSuspendNs = 100000;        // suspend hint per try, ns

struct TmaBatch {
    CUtensorMap map[kMaxBatch];        // one per projection's image (box of this batch's ZPL)
    float4 m[kMaxBatch][3];            // rows as in FwdBatch (centred, +1 folded)
    int2 k[kMaxBatch];                 // integer centring offsets (ku, kv)
    const void *img[kMaxBatch];        // image base, for the global path
    const float4 *centres;             // per-brick centring records (NULL: per projection)
    const int4 *boxes;                 // per-(brick, projection) box decisions (pre-pass)
    long long bricks;                  // bricks of the volume (record plane stride)
    const unsigned *pmax;              // the batch's max|p| bits (proj_scale_k), NULL: no scale
    float *final_out;                  // NULL, or a second destination of the updated volume
                                       // (device-addressable, same layout): the finished
                                       // volume written by the last batch's launch
    int n, isx, isy, pitch;            // pitch: elements per row
    int zpl;                           // voxels per lane along z (4, 6, 8)
    int vec4;                          // volume (and final_out) rows 16-byte aligned: float4 I/O
};

cudaError_t launch_bp_tma(const TmaBatch &b, float *vol, const VolGeom &g, int pair_kind, bool accumulate,
                          bool ieee_rcp, int *err, unsigned long long *work, cudaStream_t s);

struct PairBatch {
    const float *src[kMaxBatch];
    void *dst[kMaxBatch];
    const unsigned *pmax;              // the batch's max|p| bits (proj_scale_k), NULL: no scale
    int n;
};
// Images of the TMA path: rows() of them per projection (isy for pair
// images, isy + 1 for column quads).
__host__ __device__ constexpr int tma_image_rows(int pair_kind, int isy) { return pair_kind == kPairF32 ? isy : isy + 1; }
cudaError_t launch_pair_images(const PairBatch &b, int isx, int isy, int pitch, int pair_kind, cudaStream_t s);

// Copy (mode 0) or FP16 (1) / BF16 (2) conversion of up to kMaxBatch FP32
// images into the projection arrays' surfaces.
struct ConvBatch {
    const float *src[kMaxBatch];
    cudaSurfaceObject_t surf[kMaxBatch];
    const unsigned *pmax;              // the batch's max|p| bits (proj_scale_k), NULL: no scale
    int n;
};
cudaError_t launch_convert(const ConvBatch &b, int isx, int isy, int mode, cudaStream_t s);
// max|p| over the batch's images (src, n; `pixels` each) as float bits into
// *pmax, which the caller has zeroed.
cudaError_t launch_proj_absmax(const ConvBatch &b, long long pixels, unsigned *pmax, cudaStream_t s);

// Thread-local message for context-free entry points.
void set_thread_error(const char *fmt, ...);

}  // namespace bp
