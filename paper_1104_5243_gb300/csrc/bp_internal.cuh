// Internal declarations shared by the library's translation units.
// Nothing here is part of the C ABI (that is include/bp1104.h).
#pragma once

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
    int n;
};

// Same for the adjoint: centred matrix rows (row_u - ku row_w), the offsets
// as integers, and the output image offset.
struct AdjBatch {
    float4 m[kMaxBatch][3];
    int2 k[kMaxBatch];
    long long out_off[kMaxBatch];
    int n;
};

struct VolGeom {
    int L;
    float R, Ox, Oy, Oz;
};

// Texture storage kinds: float channel (FP32 or FP16 arrays; the texture
// unit widens FP16 exactly) or raw 16-bit words holding BF16.
enum TexKind { kTexFloat = 0, kTexBF16 = 1 };

cudaError_t launch_bp_fwd(const FwdBatch &b, float *vol, const VolGeom &g, int tex_kind,
                          bool accumulate, bool ieee_rcp, int lanes_x, cudaStream_t s);

cudaError_t launch_bp_adjoint(const AdjBatch &b, const float *vol, const VolGeom &g,
                              float *out, int isx, int isy, bool ieee_rcp, cudaStream_t s);

// Copy (mode 0) or FP16 (1) / BF16 (2) conversion of up to kMaxBatch FP32
// images into the projection arrays' surfaces.
struct ConvBatch {
    const float *src[kMaxBatch];
    cudaSurfaceObject_t surf[kMaxBatch];
    int n;
};
cudaError_t launch_convert(const ConvBatch &b, int isx, int isy, int mode, cudaStream_t s);

// Thread-local message for context-free entry points.
void set_thread_error(const char *fmt, ...);

}  // namespace bp
