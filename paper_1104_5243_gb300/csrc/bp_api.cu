// C ABI of the backprojection context (include/bp1104.h): argument checks,
// device allocations, the projection staging pipeline and kernel launches.
//
// Pipeline of bp_add_projections (images arrive one by one or in batches,
// Sect. 6): batches of up to kMaxBatch images alternate between two sets of
// texture-backed CUDA arrays.  A copy stream fills one set (host or device
// source; FP16/BF16 conversion included) while the compute stream
// backprojects the other; events order the two streams, so the compute
// stream never reads a set before its copy finished and the copy stream
// never overwrites a set the compute stream still reads.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "bp_internal.cuh"

namespace bp {
const char *thread_error();
}

// cuTensorMapEncodeTiled from the driver, through the runtime's entry-point
// query (no link against libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled()
{
    // looked up once, thread-safely (contexts may be used from several
    // host threads, one thread per context)
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

using namespace bp;

struct bp_ctx {
    int L = 0, Lz = 0;   // volume L x L x Lz (Lz < L: a z-slab of the L^3 grid)
    int nz_cap = 0;      // slab depth the volume was allocated for
    double R = 0, O[3] = {0, 0, 0};
    double O_cube[3] = {0, 0, 0};   // centre of voxel (0,0,0) of the L^3 grid
    int z0 = 0;                     // the slab's first slice in the L^3 grid
    int isx = 0, isy = 0;
    bp_dtype dtype = BP_F32;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t copy_stream = nullptr;
    float *vol = nullptr;
    bool vol_zero = true;         // volume known to be all zeros
    long long n_added = 0;
    int batch = kMaxBatch;
    bool ieee_rcp = false;
    int lanes_x = 0;              // warp layout of the texture kernel (0: automatic)
    int last_lanes = 0;           // layout of the last texture-path batch
    cudaArray_t arr[2][kMaxBatch] = {};
    cudaTextureObject_t tex[2][kMaxBatch] = {};
    cudaSurfaceObject_t surf[2][kMaxBatch] = {};
    float *staging[2] = {nullptr, nullptr};   // host-input staging for FP16/BF16
    bool proj_scale = false;      // BP_OPT_PROJ_SCALE
    unsigned *pmax[2] = {nullptr, nullptr};   // per input set: max|p| bits of the batch
    cudaEvent_t inputs_ready = nullptr;
    cudaEvent_t copy_done[2] = {nullptr, nullptr};
    cudaEvent_t kern_done[2] = {nullptr, nullptr};
    int next_set = 0;
    bool timing = false;
    std::vector<cudaEvent_t> ev;   // start/stop pairs, reused
    int path = 0;                  // BP_OPT_PATH: 0 auto, 1 texture, 2 TMA
    int last_path = 0;             // path of the last batch (1 or 2)
    // TMA path: staged images per set (kMaxBatch slots each) and their
    // tensor maps, one set of maps per brick depth (the box height differs)
    void *pairs[2] = {nullptr, nullptr};
    size_t pair_pitch = 0;         // 8-byte elements per row
    size_t pair_slot_bytes = 0;
    CUtensorMap maps[3][2][kMaxBatch];
    bool maps_ready[3] = {false, false, false};
    int brick_depth = 0;           // BP_OPT_BRICK_DEPTH (0 automatic)
    int last_depth = 0;            // brick depth of the last TMA batch
    int *err_dev = nullptr;        // set by a kernel whose bounded wait gave up
    bool cull = true;              // BP_OPT_CULL
    bool host_direct = true;       // BP_OPT_HOST_DIRECT (f32 host images: copy engine into arrays)
    bool arrays_ready = false;     // texture path's arrays allocated (ensure_arrays)
    unsigned long long *work_dev = nullptr;   // updates computed by culled launches
    unsigned long long work_host = 0;         // updates of launches without culling
    // texture path, per input set: per-block visibility masks and
    // per-(block, projection) centring records, built on the copy stream
    unsigned long long *masks[2] = {nullptr, nullptr};
    long long mask_blocks[2] = {0, 0};
    bool block_centre = true;      // BP_OPT_BLOCK_CENTRE (float32 projections)
    float4 *centres[2] = {nullptr, nullptr};
    long long centre_blocks[2] = {0, 0};
    int4 *boxes[2] = {nullptr, nullptr};   // TMA path: per-(brick, projection) box decisions
    long long box_bricks[2] = {0, 0};
    float4 *adj_centres = nullptr;         // adjoint: per-(block, projection) centring records
    long long adj_blocks = 0;
    size_t ev_used = 0;
    char err[1024] = "no error";
};

static bp_status fail(bp_ctx *c, bp_status st, const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c)
        snprintf(c->err, sizeof c->err, "%s", buf);
    else
        set_thread_error("%s", buf);
    return st;
}

#define CTX_CK(c, call)                                                              \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return fail((c), e_ == cudaErrorMemoryAllocation ? BP_ENOMEM : BP_ECUDA, \
                        "%s: %s", #call, cudaGetErrorString(e_));                    \
    } while (0)

static void release(bp_ctx *c)
{
    cudaStreamSynchronize(c->stream);
    if (c->copy_stream)
        cudaStreamSynchronize(c->copy_stream);
    for (int s = 0; s < 2; ++s) {
        for (int j = 0; j < kMaxBatch; ++j) {
            if (c->tex[s][j])
                cudaDestroyTextureObject(c->tex[s][j]);
            if (c->surf[s][j])
                cudaDestroySurfaceObject(c->surf[s][j]);
            if (c->arr[s][j])
                cudaFreeArray(c->arr[s][j]);
        }
        if (c->staging[s])
            cudaFree(c->staging[s]);
        if (c->pairs[s])
            cudaFree(c->pairs[s]);
        if (c->copy_done[s])
            cudaEventDestroy(c->copy_done[s]);
        if (c->kern_done[s])
            cudaEventDestroy(c->kern_done[s]);
    }
    if (c->inputs_ready)
        cudaEventDestroy(c->inputs_ready);
    for (cudaEvent_t e : c->ev)
        cudaEventDestroy(e);
    if (c->vol)
        cudaFree(c->vol);
    if (c->err_dev)
        cudaFree(c->err_dev);
    for (int s = 0; s < 2; ++s) {
        if (c->pmax[s])
            cudaFree(c->pmax[s]);
        if (c->masks[s])
            cudaFree(c->masks[s]);
        if (c->centres[s])
            cudaFree(c->centres[s]);
        if (c->boxes[s])
            cudaFree(c->boxes[s]);
    }
    if (c->adj_centres)
        cudaFree(c->adj_centres);
    if (c->work_dev)
        cudaFree(c->work_dev);
    if (c->copy_stream)
        cudaStreamDestroy(c->copy_stream);
}

static bp_status alloc_slot(bp_ctx *c, int s, int j)
{
    if (c->arr[s][j] != nullptr)
        return BP_OK;   // allocated by an earlier (possibly interrupted) pass
    cudaChannelFormatDesc fmt;
    if (c->dtype == BP_F32)
        fmt = cudaCreateChannelDesc(32, 0, 0, 0, cudaChannelFormatKindFloat);
    else if (c->dtype == BP_F16)
        fmt = cudaCreateChannelDesc(16, 0, 0, 0, cudaChannelFormatKindFloat);
    else
        fmt = cudaCreateChannelDesc(16, 0, 0, 0, cudaChannelFormatKindUnsigned);
    CTX_CK(c, cudaMallocArray(&c->arr[s][j], &fmt, c->isx, c->isy, cudaArraySurfaceLoadStore));
    cudaResourceDesc res;
    memset(&res, 0, sizeof res);
    res.resType = cudaResourceTypeArray;
    res.res.array.array = c->arr[s][j];
    cudaTextureDesc td;
    memset(&td, 0, sizeof td);
    td.addressMode[0] = cudaAddressModeBorder;   // zero outside the detector
    td.addressMode[1] = cudaAddressModeBorder;
    td.filterMode = cudaFilterModePoint;
    td.readMode = cudaReadModeElementType;
    td.normalizedCoords = 0;
    CTX_CK(c, cudaCreateTextureObject(&c->tex[s][j], &res, &td, nullptr));
    CTX_CK(c, cudaCreateSurfaceObject(&c->surf[s][j], &res));
    return BP_OK;
}

// The texture path's projection arrays (two sets of kMaxBatch, with their
// texture and surface objects), allocated on the path's first use: the
// default TMA path never touches them.
static bp_status ensure_arrays(bp_ctx *c)
{
    if (c->arrays_ready)
        return BP_OK;
    for (int s = 0; s < 2; ++s)
        for (int j = 0; j < kMaxBatch; ++j) {
            const bp_status st = alloc_slot(c, s, j);
            if (st != BP_OK)
                return st;
        }
    c->arrays_ready = true;
    return BP_OK;
}

static bp_status create_context(bp_ctx **out, int L, int nz, int z0, double R, const double O[3], int isx, int isy,
                                bp_dtype proj_dtype, void *cuda_stream)
{
    if (out == nullptr)
        return fail(nullptr, BP_EINVAL, "bp_create: out is NULL");
    *out = nullptr;
    if (L < 1 || L > 4096 || !(R > 0) || !std::isfinite(R) || O == nullptr ||
        !std::isfinite(O[0]) || !std::isfinite(O[1]) || !std::isfinite(O[2]))
        return fail(nullptr, BP_EINVAL, "bp_create: invalid volume (1 <= L <= 4096, R > 0, finite O)");
    if (nz < 1 || z0 < 0 || z0 > L - nz)
        return fail(nullptr, BP_EINVAL, "bp_create_slab: the slab must satisfy 1 <= nz and 0 <= z0 <= L - nz");
    if (isx < 1 || isy < 1 || isx > 32768 || isy > 32768)
        return fail(nullptr, BP_EINVAL, "bp_create: detector size must be in [1, 32768]");
    if (proj_dtype != BP_F32 && proj_dtype != BP_F16 && proj_dtype != BP_BF16)
        return fail(nullptr, BP_EINVAL, "bp_create: unknown projection dtype %d", (int)proj_dtype);
    bp_ctx *c = new (std::nothrow) bp_ctx;
    if (c == nullptr)
        return fail(nullptr, BP_ENOMEM, "bp_create: out of host memory");
    c->L = L;
    c->Lz = nz;
    c->nz_cap = nz;
    c->R = R;
    for (int q = 0; q < 3; ++q)
        c->O_cube[q] = O[q];
    c->z0 = z0;
    c->O[0] = O[0];
    c->O[1] = O[1];
    c->O[2] = O[2] + R * z0;   // centre of the slab's voxel (0,0,0)
    c->isx = isx;
    c->isy = isy;
    c->dtype = proj_dtype;
    c->lanes_x = 0;   // automatic, per batch (texture_layout)
    bp_status st = BP_OK;
    auto check = [&](cudaError_t e, const char *what) {
        if (st == BP_OK && e != cudaSuccess)
            st = fail(nullptr, e == cudaErrorMemoryAllocation ? BP_ENOMEM : BP_ECUDA, "bp_create: %s: %s",
                      what, cudaGetErrorString(e));
    };
    check(cudaGetDevice(&c->device), "cudaGetDevice");
    c->stream = (cudaStream_t)cuda_stream;   // NULL: the legacy default stream
    check(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking), "cudaStreamCreate(copy)");
    check(cudaEventCreateWithFlags(&c->inputs_ready, cudaEventDisableTiming), "cudaEventCreate");
    for (int s = 0; s < 2; ++s) {
        check(cudaEventCreateWithFlags(&c->copy_done[s], cudaEventDisableTiming), "cudaEventCreate");
        check(cudaEventCreateWithFlags(&c->kern_done[s], cudaEventDisableTiming), "cudaEventCreate");
    }
    const size_t nvox = (size_t)L * L * nz;
    check(cudaMalloc((void **)&c->vol, nvox * sizeof(float)), "cudaMalloc(volume)");
    check(cudaMalloc((void **)&c->err_dev, sizeof(int)), "cudaMalloc(error flag)");
    if (st == BP_OK)
        check(cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->stream), "cudaMemsetAsync");
    check(cudaMalloc((void **)&c->work_dev, sizeof(unsigned long long)), "cudaMalloc(work counter)");
    if (st == BP_OK)
        check(cudaMemsetAsync(c->work_dev, 0, sizeof(unsigned long long), c->stream), "cudaMemsetAsync");
    if (st == BP_OK)
        check(cudaMemsetAsync(c->vol, 0, nvox * sizeof(float), c->stream), "cudaMemsetAsync");
    if (st == BP_OK)
        check(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    if (st != BP_OK) {
        release(c);
        delete c;
        return st;
    }
    *out = c;
    return BP_OK;
}

extern "C" bp_status bp_create(bp_ctx **out, int L, double R, const double O[3], int isx, int isy,
                               bp_dtype proj_dtype, void *cuda_stream)
{
    return create_context(out, L, L, 0, R, O, isx, isy, proj_dtype, cuda_stream);
}

extern "C" bp_status bp_create_slab(bp_ctx **out, int L, int nz, int z0, double R, const double O[3], int isx,
                                    int isy, bp_dtype proj_dtype, void *cuda_stream)
{
    return create_context(out, L, nz, z0, R, O, isx, isy, proj_dtype, cuda_stream);
}

extern "C" bp_status bp_move_slab(bp_ctx *c, int z0, int nz)
{
    if (c == nullptr)
        return fail(nullptr, BP_EINVAL, "bp_move_slab: NULL context");
    if (nz < 1 || nz > c->nz_cap || z0 < 0 || z0 > c->L - nz)
        return fail(c, BP_EINVAL, "bp_move_slab: the slab must satisfy 1 <= nz <= %d and 0 <= z0 <= L - nz",
                    c->nz_cap);
    CTX_CK(c, cudaSetDevice(c->device));
    // the kernels in flight still address the old slab
    CTX_CK(c, cudaStreamSynchronize(c->stream));
    CTX_CK(c, cudaStreamSynchronize(c->copy_stream));
    c->Lz = nz;
    c->z0 = z0;
    c->O[2] = c->O_cube[2] + c->R * z0;
    return bp_reset(c);
}

extern "C" bp_status bp_destroy(bp_ctx *c)
{
    if (c == nullptr)
        return BP_OK;
    release(c);
    delete c;
    return BP_OK;
}

extern "C" const char *bp_last_error(const bp_ctx *c)
{
    return c ? c->err : thread_error();
}

extern "C" bp_status bp_set_option(bp_ctx *c, int option, long long value)
{
    if (c == nullptr)
        return fail(nullptr, BP_EINVAL, "bp_set_option: NULL context");
    switch (option) {
    case BP_OPT_IEEE_RCP:
        if (value != 0 && value != 1)
            return fail(c, BP_EINVAL, "bp_set_option: IEEE_RCP takes 0 or 1");
        c->ieee_rcp = value != 0;
        return BP_OK;
    case BP_OPT_BATCH:
        if (value < 1 || value > kMaxBatch)
            return fail(c, BP_EINVAL, "bp_set_option: BATCH must be in [1, %d]", kMaxBatch);
        c->batch = (int)value;
        return BP_OK;
    case BP_OPT_LANES_X:
        if (value != 0 && value != 8 && value != 16 && value != 32 && value != 44 && value != 42 && value != 82 &&
            value != 24 && value != 108)
            return fail(c, BP_EINVAL, "bp_set_option: LANES_X takes 0, 8, 16, 32, 44, 42, 82, 24 or 108");
        c->lanes_x = (int)value;
        return BP_OK;
    case BP_OPT_HOST_DIRECT:
        if (value != 0 && value != 1)
            return fail(c, BP_EINVAL, "bp_set_option: HOST_DIRECT takes 0 or 1");
        c->host_direct = value != 0;
        return BP_OK;
    case BP_OPT_BLOCK_CENTRE:
        if (value != 0 && value != 1)
            return fail(c, BP_EINVAL, "bp_set_option: BLOCK_CENTRE takes 0 or 1");
        c->block_centre = value != 0;
        return BP_OK;
    case BP_OPT_PROJ_SCALE:
        if (value != 0 && value != 1)
            return fail(c, BP_EINVAL, "bp_set_option: PROJ_SCALE takes 0 or 1");
        c->proj_scale = value != 0;
        return BP_OK;
    case BP_OPT_CULL:
        if (value != 0 && value != 1)
            return fail(c, BP_EINVAL, "bp_set_option: CULL takes 0 or 1");
        c->cull = value != 0;
        return BP_OK;
    case BP_OPT_PATH:
        if (value < 0 || value > 2)
            return fail(c, BP_EINVAL, "bp_set_option: PATH takes 0 (auto), 1 (texture) or 2 (TMA)");
        c->path = (int)value;
        return BP_OK;
    case BP_OPT_TIMING:
        if (value != 0 && value != 1)
            return fail(c, BP_EINVAL, "bp_set_option: TIMING takes 0 or 1");
        c->timing = value != 0;
        return BP_OK;
    case BP_OPT_BRICK_DEPTH:
        if (value != 0 && value != 8 && value != 12 && value != 16)
            return fail(c, BP_EINVAL, "bp_set_option: BRICK_DEPTH takes 0 (automatic), 8, 12 or 16");
        c->brick_depth = (int)value;
        return BP_OK;
    default:
        return fail(c, BP_EINVAL, "bp_set_option: unknown option %d", option);
    }
}

extern "C" bp_status bp_reset(bp_ctx *c)
{
    if (c == nullptr)
        return fail(nullptr, BP_EINVAL, "bp_reset: NULL context");
    CTX_CK(c, cudaSetDevice(c->device));
    CTX_CK(c, cudaMemsetAsync(c->vol, 0, sizeof(float) * (size_t)c->L * c->L * c->Lz, c->stream));
    c->vol_zero = true;
    c->n_added = 0;
    return BP_OK;
}

// Host-side checks of the matrices: finite entries and w > 0 at the eight
// corners of the volume box (w is affine in x, so then w > 0 everywhere).
static bp_status check_matrices(bp_ctx *c, const char *who, const double *A, int n)
{
    for (int i = 0; i < n; ++i) {
        const double *a = A + 12 * (size_t)i;
        for (int q = 0; q < 12; ++q)
            if (!std::isfinite(a[q]))
                return fail(c, BP_EINVAL, "%s: matrix %d has a non-finite entry", who, i);
        for (int corner = 0; corner < 8; ++corner) {
            const double X = c->O[0] + c->R * ((corner & 1) ? c->L - 1 : 0);
            const double Y = c->O[1] + c->R * ((corner & 2) ? c->L - 1 : 0);
            const double Z = c->O[2] + c->R * ((corner & 4) ? c->Lz - 1 : 0);
            const double w = a[8] * X + a[9] * Y + a[10] * Z + a[11];
            if (!(w > 0))
                return fail(c, BP_EINVAL,
                            "%s: matrix %d puts part of the volume behind the source (w <= 0)", who, i);
        }
    }
    return BP_OK;
}

static inline float4 row4(const double *a, int r, double add_w)
{
    // row r of A, plus add_w times the w row (folds the centring and gather
    // offsets in float64 before rounding to float32)
    return make_float4((float)(a[4 * r] + add_w * a[8]), (float)(a[4 * r + 1] + add_w * a[9]),
                       (float)(a[4 * r + 2] + add_w * a[10]), (float)(a[4 * r + 3] + add_w * a[11]));
}

// Integer centring offsets (ku, kv): the pixel the centre of the L^3 grid
// projects to, rounded.  Over the volume |u - ku| then stays within the
// volume's footprint half-width, far below |u|.  A z-slab takes the whole
// grid's offsets, so that its float32 rows (and the per-block centring
// records built from them) equal the cube's.
static inline void centre_offsets(const bp_ctx *c, const double *a, double *ku, double *kv)
{
    const double h = 0.5 * (c->L - 1) * c->R;
    const double X = c->O_cube[0] + h, Y = c->O_cube[1] + h, Z = c->O_cube[2] + h;
    const double w = a[8] * X + a[9] * Y + a[10] * Z + a[11];
    const double u = (a[0] * X + a[1] * Y + a[2] * Z + a[3]) / w;
    const double v = (a[4] * X + a[5] * Y + a[6] * Z + a[7]) / w;
    *ku = std::fmin(std::fmax(std::nearbyint(u), -1048576.0), 1048576.0);
    *kv = std::fmin(std::fmax(std::nearbyint(v), -1048576.0), 1048576.0);
}

static VolGeom vol_geom(const bp_ctx *c)
{
    VolGeom g;
    g.L = c->L;
    g.Lz = c->Lz;
    g.R = (float)c->R;
    g.Ox = (float)c->O[0];
    g.Oy = (float)c->O[1];
    g.Oz = (float)c->O_cube[2];
    g.z0 = c->z0;
    return g;
}

static int pair_kind(const bp_ctx *c)
{
    return c->dtype == BP_F32 ? kPairF32 : c->dtype == BP_F16 ? kQuadF16 : kQuadBF16;
}

// Staged images for the TMA path (float32 pair images or 16-bit column
// quads, 8-byte elements), allocated on first use; the slots' addresses
// never change.
static bp_status ensure_pairs(bp_ctx *c)
{
    if (c->pairs[0] != nullptr)
        return BP_OK;
    if (encode_tiled() == nullptr)
        return fail(c, BP_ECUDA, "TMA path: cuTensorMapEncodeTiled is not available from the driver");
    const size_t width = (size_t)c->isx + 1;                     // element columns 0 .. isx
    c->pair_pitch = (width + kTmaAlign - 1) / kTmaAlign * kTmaAlign;
    c->pair_slot_bytes = c->pair_pitch * 8 * (size_t)tma_image_rows(pair_kind(c), c->isy);
    for (int s = 0; s < 2; ++s)
        CTX_CK(c, cudaMalloc(&c->pairs[s], c->pair_slot_bytes * kMaxBatch));
    return BP_OK;
}

static int depth_index(int zpl) { return zpl == 4 ? 0 : zpl == 6 ? 1 : 2; }

// One tensor map per slot for the box of brick depth 2 zpl (two 32-bit
// words per element; rows of the staged image).
static bp_status ensure_maps(bp_ctx *c, int zpl)
{
    const int di = depth_index(zpl);
    if (c->maps_ready[di])
        return BP_OK;
    EncodeTiledFn enc = encode_tiled();
    const int kind = pair_kind(c);
    const size_t width = (size_t)c->isx + 1;
    for (int s = 0; s < 2; ++s) {
        for (int j = 0; j < kMaxBatch; ++j) {
            void *base = static_cast<char *>(c->pairs[s]) + c->pair_slot_bytes * j;
            const cuuint64_t dims[2] = {width * 2, (cuuint64_t)tma_image_rows(kind, c->isy)};
            const cuuint64_t strides[1] = {c->pair_pitch * 8};
            const cuuint32_t box[2] = {(cuuint32_t)(kTmaBU * 2), (cuuint32_t)tma_rows(zpl, kind != kPairF32)};
            const cuuint32_t estr[2] = {1, 1};
            CUresult r = enc(&c->maps[di][s][j], CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, base, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS)
                return fail(c, BP_ECUDA, "TMA path: cuTensorMapEncodeTiled failed (%d)", (int)r);
        }
    }
    c->maps_ready[di] = true;
    return BP_OK;
}

// Host model of the pre-pass's box rule on a sample of bricks (the bricks
// at the centres of a 6 x 6 x 6 partition of the volume, so that every part
// of the volume weighs the same) and up to 16 projections of the batch, in
// float64: of the sampled (brick, projection) pairs whose
// footprint reaches the detector, the fraction whose box fits kTmaBU
// element columns by bv rows (pair-image rule: rows floor(v) - 1 ..
// floor(v_max) + 2) for bricks 32 x 16 x bz; 1 if no sampled pair is
// visible.
static double box_fit_fraction(const bp_ctx *c, const double *A, int m, int bz, int bv)
{
    const int nb[3] = {(c->L + kBrickX - 1) / kBrickX, (c->L + kBrickY - 1) / kBrickY, (c->Lz + bz - 1) / bz};
    const int ext[3] = {kBrickX, kBrickY, bz}, lim[3] = {c->L, c->L, c->Lz};
    constexpr int K = 6;
    long vis = 0, fit = 0;
    const int pstep = m > 16 ? m / 16 : 1;
    for (int p = 0; p < m; p += pstep) {
        const double *a = A + 12 * (size_t)p;
        for (int q = 0; q < K * K * K; ++q) {
            int lo[3], hi[3];
            for (int d = 0, qq = q; d < 3; ++d, qq /= K) {
                const int bi = std::min(nb[d] - 1, (int)(((double)(qq % K) + 0.5) * nb[d] / K));
                lo[d] = bi * ext[d];
                hi[d] = std::min(lo[d] + ext[d], lim[d]) - 1;
            }
            double umin = 1e300, umax = -1e300, vmin = 1e300, vmax = -1e300;
            for (int cn = 0; cn < 8; ++cn) {
                const double X = c->O[0] + c->R * ((cn & 1) ? hi[0] : lo[0]);
                const double Y = c->O[1] + c->R * ((cn & 2) ? hi[1] : lo[1]);
                const double Z = c->O[2] + c->R * ((cn & 4) ? hi[2] : lo[2]);
                const double w = a[8] * X + a[9] * Y + a[10] * Z + a[11];
                const double u = (a[0] * X + a[1] * Y + a[2] * Z + a[3]) / w;
                const double v = (a[4] * X + a[5] * Y + a[6] * Z + a[7]) / w;
                umin = std::fmin(umin, u), umax = std::fmax(umax, u);
                vmin = std::fmin(vmin, v), vmax = std::fmax(vmax, v);
            }
            const double cmin = std::floor(umin), cmax = std::floor(umax) + 2;
            const double rmin = std::floor(vmin) - 1, rmax = std::floor(vmax) + 2;
            if (cmax < 0 || cmin > c->isx || rmax < 0 || rmin > c->isy - 1)
                continue;
            ++vis;
            const double cx0 = std::floor(cmin / kTmaAlign) * kTmaAlign;
            if (cmax - cx0 + 1 <= kTmaBU && rmax - rmin + 1 <= bv)
                ++fit;
        }
    }
    return vis ? (double)fit / (double)vis : 1.0;
}

// Data path and brick depth of a batch.  Forced depths and the forced TMA
// path take the caller's choice; otherwise 16-deep bricks when their box
// holds the sampled footprints of 98 % of the visible pairs (the rest take
// the slower global-memory branch), else 8-deep bricks, and the texture path
// when even the 8-deep box holds fewer than 40 % of them (coarse voxels).
// The 40 % is measured: at 384^3 on the 1248x960 detector the 8-deep box
// holds 60-75 % of the footprints and the TMA path still wins (f32 978
// against 732 GUP/s, f16 1125 against 1105); at 256^3 it holds under 1 %
// (468 against 593).
// Measured on GB300 at 512^3 x 496 x 1248x960 (GUP/s per step for depths
// 8 / 12 / 16): f32 1403 / 1379 / 1413, f16 1511 / 1497 / 1536; so 12 is
// never the automatic choice.
static void choose_path(const bp_ctx *c, const double *A, int m, bool *tma, int *zpl)
{
    *zpl = c->brick_depth ? c->brick_depth / 2 : 4;
    *tma = c->path != 1;
    if (c->path == 1 || c->brick_depth)
        return;
    if (box_fit_fraction(c, A, m, 16, tma_rows(8, false)) >= 0.98) {
        *zpl = 8;
        return;
    }
    if (c->path == 0 && box_fit_fraction(c, A, m, 8, tma_rows(4, false)) < 0.4)
        *tma = false;
}

// Pixels spanned by one voxel step in the x-y plane at the volume centre,
// R |grad_xy u| (u = a_u.X / a_w.X, so grad u = (a_u - u a_w) / w), averaged
// over up to 16 projections of the batch: about R times the magnification
// over the pixel pitch for a scan about the z axis.
static double voxel_pixels(const bp_ctx *c, const double *A, int m)
{
    const double X = c->O[0] + 0.5 * c->R * (c->L - 1), Y = c->O[1] + 0.5 * c->R * (c->L - 1);
    const double Z = c->O[2] + 0.5 * c->R * (c->Lz - 1);
    const int pstep = m > 16 ? m / 16 : 1;
    double sum = 0.0;
    int cnt = 0;
    for (int p = 0; p < m; p += pstep, ++cnt) {
        const double *a = A + 12 * (size_t)p;
        const double w = a[8] * X + a[9] * Y + a[10] * Z + a[11];
        const double u = (a[0] * X + a[1] * Y + a[2] * Z + a[3]) / w;
        const double gx = (a[0] - u * a[8]) / w, gy = (a[1] - u * a[9]) / w;
        sum += c->R * std::sqrt(gx * gx + gy * gy);
    }
    return cnt ? sum / cnt : 0.0;
}

// Warp layout of a texture-path batch: the caller's, or automatically
//   * 2 lanes along x by 4 along y (code 24) for coarse voxels, whose step
//     spans 4 pixels or more: a warp's gathers then cover a compact patch of
//     the detector at every angle, where 8 lanes along x spread over 8 voxel
//     steps when x runs across the rays.  Measured on GB300 (GUP/s per step
//     on the 1248x960 detector, f32 / f16): 256^3 (5.0 pixels per voxel)
//     633 / 802 against 590 / 791 for the finer voxels' layouts, 128^3 254 /
//     316 against 241 / 272;
//   * else 8 lanes along x with 4 voxels per lane (code 8) for float32
//     projections, 8 voxels per lane (code 108) for 16-bit ones: 512^3 (2.5
//     pixels per voxel) f32 795 against 791 for code 24, f16 1217 against
//     1127.
static int texture_layout(const bp_ctx *c, const double *A, int m)
{
    if (c->lanes_x)
        return c->lanes_x;
    if (voxel_pixels(c, A, m) >= 4.0)
        return 24;
    return c->dtype == BP_F32 ? 8 : 108;
}

static bp_status record_start(bp_ctx *c, cudaEvent_t *stop)
{
    *stop = nullptr;
    if (!c->timing)
        return BP_OK;
    while (c->ev.size() < c->ev_used + 2) {
        cudaEvent_t e;
        CTX_CK(c, cudaEventCreate(&e));
        c->ev.push_back(e);
    }
    CTX_CK(c, cudaEventRecord(c->ev[c->ev_used], c->stream));
    *stop = c->ev[c->ev_used + 1];
    c->ev_used += 2;
    return BP_OK;
}

// bp_add_projections; with final_out (device-addressable, or NULL) the last
// batch's TMA launch also stores the finished volume there.
static bp_status add_projections(bp_ctx *c, const float *images, int images_on_device, const double *A, int n,
                                 float *final_out)
{
    if (c == nullptr)
        return fail(nullptr, BP_EINVAL, "bp_add_projections: NULL context");
    if (n < 0)
        return fail(c, BP_EINVAL, "bp_add_projections: n < 0");
    if (n == 0)
        return BP_OK;
    if (images == nullptr || A == nullptr)
        return fail(c, BP_EINVAL, "bp_add_projections: NULL images or matrices");
    bp_status st = check_matrices(c, "bp_add_projections", A, n);
    if (st != BP_OK)
        return st;
    CTX_CK(c, cudaSetDevice(c->device));
    const size_t img_elems = (size_t)c->isx * c->isy;
    const size_t row_bytes = sizeof(float) * c->isx;
    // Work queued on the caller's stream before this call (e.g. the producer
    // of device images) must finish before the copy stream reads.
    CTX_CK(c, cudaEventRecord(c->inputs_ready, c->stream));
    CTX_CK(c, cudaStreamWaitEvent(c->copy_stream, c->inputs_ready, 0));
    const VolGeom g = vol_geom(c);
    for (int c0 = 0; c0 < n; c0 += c->batch) {
        const int m = n - c0 < c->batch ? n - c0 : c->batch;
        const double *A0 = A + 12 * (size_t)c0;
        // Automatic choice, by measurement on GB300: the TMA path wherever its
        // boxes hold the bricks' footprints (512^3 x 1248x960: f32 1388
        // against 796 GUP/s on the texture path, whose 32-bit gathers the
        // texture unit returns at half the 16-bit rate), the texture path for
        // coarse voxels (256^3 on that detector: 593 against 468 GUP/s for
        // the TMA path's global-memory branch).
        bool tma = true;
        int zpl = 4;
        choose_path(c, A0, m, &tma, &zpl);
        const int lanes = tma ? 0 : texture_layout(c, A0, m);
        st = tma ? ensure_pairs(c) : ensure_arrays(c);
        if (st == BP_OK && tma)
            st = ensure_maps(c, zpl);
        if (st != BP_OK)
            return st;
        const int s = c->next_set;
        c->next_set ^= 1;
        CTX_CK(c, cudaStreamWaitEvent(c->copy_stream, c->kern_done[s], 0));
        const float *src0 = images + (size_t)c0 * img_elems;
        // float16 storage with BP_OPT_PROJ_SCALE: a power-of-four scale per
        // batch (proj_scale_k), from the images' maximum on the copy stream
        const bool scaled = c->proj_scale && c->dtype == BP_F16;
        if (scaled && c->pmax[s] == nullptr)
            CTX_CK(c, cudaMalloc((void **)&c->pmax[s], sizeof(unsigned)));
        const unsigned *pmax = scaled ? c->pmax[s] : nullptr;
        if (!tma && c->dtype == BP_F32 && !images_on_device && c->host_direct) {
            // host images straight into the arrays on the copy engine
            for (int j = 0; j < m; ++j)
                CTX_CK(c, cudaMemcpy2DToArrayAsync(c->arr[s][j], 0, 0, src0 + (size_t)j * img_elems, row_bytes,
                                                   row_bytes, c->isy, cudaMemcpyHostToDevice, c->copy_stream));
        } else {
            const float *src = src0;
            if (!images_on_device) {
                if (c->staging[s] == nullptr)
                    CTX_CK(c, cudaMalloc((void **)&c->staging[s], sizeof(float) * img_elems * kMaxBatch));
                CTX_CK(c, cudaMemcpyAsync(c->staging[s], src0, sizeof(float) * img_elems * m,
                                          cudaMemcpyHostToDevice, c->copy_stream));
                src = c->staging[s];
            }
            if (scaled) {
                // max|p| over the batch's images, for its power-of-four scale
                CTX_CK(c, cudaMemsetAsync(c->pmax[s], 0, sizeof(unsigned), c->copy_stream));
                ConvBatch mb;
                mb.n = m;
                mb.pmax = nullptr;
                for (int j = 0; j < m; ++j)
                    mb.src[j] = src + (size_t)j * img_elems;
                CTX_CK(c, launch_proj_absmax(mb, (long long)img_elems, c->pmax[s], c->copy_stream));
            }
            if (tma) {
                PairBatch pb;
                pb.n = m;
                pb.pmax = pmax;
                for (int j = 0; j < m; ++j) {
                    pb.src[j] = src + (size_t)j * img_elems;
                    pb.dst[j] = static_cast<char *>(c->pairs[s]) + c->pair_slot_bytes * j;
                }
                CTX_CK(c, launch_pair_images(pb, c->isx, c->isy, (int)c->pair_pitch, pair_kind(c), c->copy_stream));
            } else {
                ConvBatch cb;
                cb.n = m;
                cb.pmax = pmax;
                for (int j = 0; j < m; ++j) {
                    cb.src[j] = src + (size_t)j * img_elems;
                    cb.surf[j] = c->surf[s][j];
                }
                const int mode = c->dtype == BP_F32 ? 0 : c->dtype == BP_F16 ? 1 : 2;
                CTX_CK(c, launch_convert(cb, c->isx, c->isy, mode, c->copy_stream));
            }
        }
        // The batch's kernel parameters, and the per-tile pre-pass on the copy
        // stream: culling masks (texture path; the TMA producer culls per
        // brick itself) and centring records (float32 projections).  It needs
        // only the matrices, so it overlaps the previous batch's
        // backprojection; its buffers belong to this input set, which the
        // copy stream has waited for.  Tiles: the texture kernel's blocks or
        // the TMA path's bricks.
        FwdBatch b;
        b.pmax = pmax;
        unsigned long long *masks = nullptr;
        float4 *centres = nullptr;
        int tile[3] = {kBrickX, kBrickY, 2 * zpl};
        if (!tma)
            fwd_tile(lanes, &tile[0], &tile[1], &tile[2]);
        const long long nb = tile_count(c->L, c->Lz, tile[0], tile[1], tile[2]);
        {
            b.n = m;
            double rows[kMaxBatch][3][4];   // the same centred rows in float64
            for (int j = 0; j < m; ++j) {
                const double *a = A0 + 12 * (size_t)j;
                // u' = u - ku + 1 = (uw - (ku - 1) w) / w; gather at floor(u') + ku
                double ku, kv;
                centre_offsets(c, a, &ku, &kv);
                b.m[j][0] = row4(a, 0, 1.0 - ku);
                b.m[j][1] = row4(a, 1, 1.0 - kv);
                b.m[j][2] = row4(a, 2, 0.0);
                b.k[j] = make_float2((float)ku, (float)kv);
                b.tex[j] = c->tex[s][j];
                for (int q = 0; q < 4; ++q) {
                    rows[j][0][q] = a[q] + (1.0 - ku) * a[8 + q];
                    rows[j][1][q] = a[4 + q] + (1.0 - kv) * a[8 + q];
                    rows[j][2][q] = a[8 + q];
                }
            }
            if (c->cull && !tma) {
                if (nb > c->mask_blocks[s]) {
                    if (c->masks[s])
                        CTX_CK(c, cudaFree(c->masks[s]));
                    c->masks[s] = nullptr;
                    c->mask_blocks[s] = 0;
                    CTX_CK(c, cudaMalloc((void **)&c->masks[s], sizeof(unsigned long long) * nb));
                    c->mask_blocks[s] = nb;
                }
                masks = c->masks[s];
            } else if (!tma) {
                c->work_host += (unsigned long long)m * c->L * c->L * c->Lz;
            }
            CentreBatch cb;
            if (c->dtype == BP_F32 && c->block_centre) {
                if (nb > c->centre_blocks[s]) {
                    if (c->centres[s])
                        CTX_CK(c, cudaFree(c->centres[s]));
                    c->centres[s] = nullptr;
                    c->centre_blocks[s] = 0;
                    CTX_CK(c, cudaMalloc((void **)&c->centres[s], sizeof(float4) * 3 * kMaxBatch * nb));
                    c->centre_blocks[s] = nb;
                }
                centres = c->centres[s];
                centre_batch(&cb, &rows[0][0][0], m, c->O_cube, c->R);
            }
            int4 *boxes = nullptr;
            BoxSpec bs{};
            if (tma) {
                if (nb > c->box_bricks[s]) {
                    if (c->boxes[s])
                        CTX_CK(c, cudaFree(c->boxes[s]));
                    c->boxes[s] = nullptr;
                    c->box_bricks[s] = 0;
                    CTX_CK(c, cudaMalloc((void **)&c->boxes[s], sizeof(int4) * kMaxBatch * nb));
                    c->box_bricks[s] = nb;
                }
                boxes = c->boxes[s];
                const bool quad = pair_kind(c) != kPairF32;
                bs = BoxSpec{kTmaBU, tma_rows(zpl, quad), kTmaAlign, quad ? 1 : 0};
            }
            CTX_CK(c, launch_block_prepass(b, centres ? &cb : nullptr, g, c->isx, c->isy, tile[0], tile[1], tile[2],
                                           2 * c->z0, masks, centres, boxes ? &bs : nullptr, boxes,
                                           masks ? c->work_dev : nullptr, c->copy_stream));
        }
        CTX_CK(c, cudaEventRecord(c->copy_done[s], c->copy_stream));
        CTX_CK(c, cudaStreamWaitEvent(c->stream, c->copy_done[s], 0));
        cudaEvent_t ev_stop;
        st = record_start(c, &ev_stop);
        if (st != BP_OK)
            return st;
        if (tma) {
            TmaBatch tb;   // 12 KB of kernel parameters
            tb.n = m;
            tb.pmax = pmax;
            tb.isx = c->isx;
            tb.isy = c->isy;
            tb.pitch = (int)c->pair_pitch;
            for (int j = 0; j < m; ++j) {
                const double *a = A0 + 12 * (size_t)j;
                double ku, kv;
                centre_offsets(c, a, &ku, &kv);
                tb.m[j][0] = row4(a, 0, 1.0 - ku);
                tb.m[j][1] = row4(a, 1, 1.0 - kv);
                tb.m[j][2] = row4(a, 2, 0.0);
                tb.k[j] = make_int2((int)ku, (int)kv);
                tb.map[j] = c->maps[depth_index(zpl)][s][j];
                tb.img[j] = static_cast<const char *>(c->pairs[s]) + c->pair_slot_bytes * j;
            }
            tb.centres = centres;
            tb.boxes = c->boxes[s];
            tb.bricks = nb;
            tb.final_out = c0 + m == n ? final_out : nullptr;
            tb.zpl = zpl;
            tb.vec4 = c->L % 4 == 0 && (tb.final_out == nullptr || reinterpret_cast<uintptr_t>(tb.final_out) % 16 == 0);
            CTX_CK(c, launch_bp_tma(tb, c->vol, g, pair_kind(c), !c->vol_zero, c->ieee_rcp, c->err_dev, c->work_dev,
                                    c->stream));
        } else {
            CTX_CK(c, launch_bp_fwd(b, c->vol, g, c->dtype == BP_BF16 ? kTexBF16 : kTexFloat, !c->vol_zero,
                                    c->ieee_rcp, lanes, masks, centres, c->stream));
        }
        if (ev_stop)
            CTX_CK(c, cudaEventRecord(ev_stop, c->stream));
        c->last_path = tma ? 2 : 1;
        if (tma)
            c->last_depth = 2 * zpl;
        else
            c->last_lanes = lanes;
        c->vol_zero = false;
        CTX_CK(c, cudaEventRecord(c->kern_done[s], c->stream));
    }
    c->n_added += n;
    return BP_OK;
}

extern "C" bp_status bp_add_projections(bp_ctx *c, const float *images, int images_on_device,
                                        const double *A, int n)
{
    return add_projections(c, images, images_on_device, A, n, nullptr);
}

// Turn the device-side error flag (a bounded wait that gave up) into a
// status; clears the flag.  The caller has synchronised the stream.
static bp_status check_device_error(bp_ctx *c, const char *who)
{
    int flag = 0;
    CTX_CK(c, cudaMemcpy(&flag, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        CTX_CK(c, cudaMemset(c->err_dev, 0, sizeof(int)));
        return fail(c, BP_ETIMEOUT, "%s: a backprojection block gave up waiting for its projection tile; "
                                    "the volume is incomplete", who);
    }
    return BP_OK;
}

extern "C" bp_status bp_query(bp_ctx *c, int what, long long *value)
{
    if (c == nullptr || value == nullptr)
        return fail(nullptr, BP_EINVAL, "bp_query: NULL argument");
    switch (what) {
    case BP_QUERY_LAST_PATH:
        *value = c->last_path;
        return BP_OK;
    case BP_QUERY_PROJECTIONS_ADDED:
        *value = c->n_added;
        return BP_OK;
    case BP_QUERY_LAST_BRICK_DEPTH:
        *value = c->last_depth;
        return BP_OK;
    case BP_QUERY_LAST_LANES_X:
        *value = c->last_lanes;
        return BP_OK;
    case BP_QUERY_UPDATES_COMPUTED: {
        unsigned long long dev = 0;
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpy(&dev, c->work_dev, sizeof dev, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess)
            return fail(nullptr, BP_ECUDA, "bp_query: %s", cudaGetErrorString(e));
        *value = (long long)(dev + c->work_host);
        return BP_OK;
    }
    default:
        return fail(nullptr, BP_EINVAL, "bp_query: unknown query %d", what);
    }
}

extern "C" bp_status bp_kernel_stats(bp_ctx *c, long long *launches, double *total_ms)
{
    if (c == nullptr)
        return fail(nullptr, BP_EINVAL, "bp_kernel_stats: NULL context");
    CTX_CK(c, cudaSetDevice(c->device));
    CTX_CK(c, cudaStreamSynchronize(c->stream));
    bp_status st = check_device_error(c, "bp_kernel_stats");
    if (st != BP_OK)
        return st;
    double ms = 0.0;
    for (size_t q = 0; q + 1 < c->ev_used; q += 2) {
        float t = 0.f;
        CTX_CK(c, cudaEventElapsedTime(&t, c->ev[q], c->ev[q + 1]));
        ms += t;
    }
    if (launches)
        *launches = (long long)(c->ev_used / 2);
    if (total_ms)
        *total_ms = ms;
    c->ev_used = 0;
    return BP_OK;
}

extern "C" bp_status bp_finalize(bp_ctx *c, float *vol_out, int on_device)
{
    if (c == nullptr)
        return fail(nullptr, BP_EINVAL, "bp_finalize: NULL context");
    if (vol_out == nullptr)
        return fail(c, BP_EINVAL, "bp_finalize: NULL output");
    CTX_CK(c, cudaSetDevice(c->device));
    const size_t bytes = sizeof(float) * (size_t)c->L * c->L * c->Lz;
    CTX_CK(c, cudaMemcpyAsync(vol_out, c->vol, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              c->stream));
    CTX_CK(c, cudaStreamSynchronize(c->stream));
    return check_device_error(c, "bp_finalize");
}

extern "C" bp_status bp_add_projections_finalize(bp_ctx *c, const float *images, int images_on_device,
                                                 const double *A, int n, float *vol_out, int out_on_device)
{
    if (c == nullptr)
        return fail(nullptr, BP_EINVAL, "bp_add_projections_finalize: NULL context");
    if (vol_out == nullptr)
        return fail(c, BP_EINVAL, "bp_add_projections_finalize: NULL output");
    CTX_CK(c, cudaSetDevice(c->device));
    // the destination as the kernel can address it: device memory as it is,
    // page-locked host memory through its mapping; other host memory (no
    // mapping) is copied after the last launch as bp_finalize does
    float *direct = nullptr;
    if (n > 0 && c->path != 1) {
        if (out_on_device) {
            direct = vol_out;
        } else {
            cudaPointerAttributes at{};
            if (cudaPointerGetAttributes(&at, vol_out) == cudaSuccess && at.type == cudaMemoryTypeHost &&
                at.devicePointer != nullptr)
                direct = static_cast<float *>(at.devicePointer);
            else
                (void)cudaGetLastError();   // not a CUDA allocation: not an error here
        }
    }
    bp_status st = add_projections(c, images, images_on_device, A, n, direct);
    if (st != BP_OK)
        return st;
    if (direct != nullptr) {
        CTX_CK(c, cudaStreamSynchronize(c->stream));
        return check_device_error(c, "bp_add_projections_finalize");
    }
    return bp_finalize(c, vol_out, out_on_device);
}

extern "C" bp_status bp_get_state(bp_ctx *c, float *vol_out, int on_device, long long *n_added)
{
    if (c == nullptr)
        return fail(nullptr, BP_EINVAL, "bp_get_state: NULL context");
    if (vol_out != nullptr) {
        bp_status st = bp_finalize(c, vol_out, on_device);
        if (st != BP_OK)
            return st;
    }
    if (n_added)
        *n_added = c->n_added;
    return BP_OK;
}

extern "C" bp_status bp_set_state(bp_ctx *c, const float *vol_in, int on_device, long long n_added)
{
    if (c == nullptr)
        return fail(nullptr, BP_EINVAL, "bp_set_state: NULL context");
    if (vol_in == nullptr || n_added < 0)
        return fail(c, BP_EINVAL, "bp_set_state: NULL volume or negative counter");
    CTX_CK(c, cudaSetDevice(c->device));
    const size_t bytes = sizeof(float) * (size_t)c->L * c->L * c->Lz;
    CTX_CK(c, cudaMemcpyAsync(c->vol, vol_in, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              c->stream));
    CTX_CK(c, cudaStreamSynchronize(c->stream));
    c->vol_zero = false;
    c->n_added = n_added;
    return BP_OK;
}

extern "C" bp_status bp_adjoint(bp_ctx *c, const float *vol, int vol_on_device, const double *A, int n,
                                float *images_out, int out_on_device)
{
    if (c == nullptr)
        return fail(nullptr, BP_EINVAL, "bp_adjoint: NULL context");
    if (n < 0)
        return fail(c, BP_EINVAL, "bp_adjoint: n < 0");
    if (n == 0)
        return BP_OK;
    if (vol == nullptr || A == nullptr || images_out == nullptr)
        return fail(c, BP_EINVAL, "bp_adjoint: NULL volume, matrices or output");
    bp_status st = check_matrices(c, "bp_adjoint", A, n);
    if (st != BP_OK)
        return st;
    CTX_CK(c, cudaSetDevice(c->device));
    const size_t nvox = (size_t)c->L * c->L * c->Lz;
    const size_t img_elems = (size_t)c->isx * c->isy;
    const float *dvol = vol;
    float *dvol_tmp = nullptr, *dout = images_out;
    cudaError_t e = cudaSuccess;
    if (!vol_on_device) {
        e = cudaMallocAsync((void **)&dvol_tmp, sizeof(float) * nvox, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dvol_tmp, vol, sizeof(float) * nvox, cudaMemcpyHostToDevice, c->stream);
        dvol = dvol_tmp;
    }
    float *dout_tmp = nullptr;
    if (e == cudaSuccess && !out_on_device) {
        e = cudaMallocAsync((void **)&dout_tmp, sizeof(float) * img_elems * n, c->stream);
        dout = dout_tmp;
    }
    if (e == cudaSuccess)
        e = cudaMemsetAsync(dout, 0, sizeof(float) * img_elems * n, c->stream);
    const VolGeom g = vol_geom(c);
    // The shared-tile kernel (BP_OPT_CULL) centres per block with
    // BP_OPT_BLOCK_CENTRE: its records come from the per-tile pre-pass, on
    // this stream, with the kernel's block as the tile.
    const bool blk = c->cull && c->block_centre;
    const long long nb = tile_count(c->L, c->Lz, kAdjBlockX, kAdjBlockY, kAdjBlockZ);
    if (e == cudaSuccess && blk && nb > c->adj_blocks) {
        if (c->adj_centres)
            e = cudaFree(c->adj_centres);
        c->adj_centres = nullptr;
        c->adj_blocks = 0;
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&c->adj_centres, sizeof(float4) * 3 * kMaxBatch * nb);
        if (e == cudaSuccess)
            c->adj_blocks = nb;
    }
    for (int c0 = 0; e == cudaSuccess && c0 < n; c0 += kMaxBatch) {
        const int m = n - c0 < kMaxBatch ? n - c0 : kMaxBatch;
        AdjBatch b;
        b.n = m;
        b.centres = nullptr;
        b.blocks = nb;
        FwdBatch fb;   // the same rows in the forward convention, for the pre-pass
        fb.n = m;
        fb.pmax = nullptr;
        double rows[kMaxBatch][3][4];
        for (int j = 0; j < m; ++j) {
            const double *a = A + 12 * (size_t)(c0 + j);
            double ku, kv;
            centre_offsets(c, a, &ku, &kv);
            b.m[j][0] = row4(a, 0, -ku);
            b.m[j][1] = row4(a, 1, -kv);
            b.m[j][2] = row4(a, 2, 0.0);
            b.k[j] = make_int2((int)ku, (int)kv);
            b.out_off[j] = (long long)(c0 + j) * (long long)img_elems;
            if (blk) {
                fb.m[j][0] = row4(a, 0, 1.0 - ku);
                fb.m[j][1] = row4(a, 1, 1.0 - kv);
                fb.m[j][2] = row4(a, 2, 0.0);
                fb.k[j] = make_float2((float)ku, (float)kv);
                for (int q = 0; q < 4; ++q) {
                    rows[j][0][q] = a[q] + (1.0 - ku) * a[8 + q];
                    rows[j][1][q] = a[4 + q] + (1.0 - kv) * a[8 + q];
                    rows[j][2][q] = a[8 + q];
                }
            }
        }
        if (blk) {
            CentreBatch cb;
            centre_batch(&cb, &rows[0][0][0], m, c->O_cube, c->R);
            e = launch_block_prepass(fb, &cb, g, c->isx, c->isy, kAdjBlockX, kAdjBlockY, kAdjBlockZ, 2 * c->z0, nullptr,
                                     c->adj_centres, nullptr, nullptr, nullptr, c->stream);
            b.centres = c->adj_centres;
        }
        if (e == cudaSuccess)
            e = launch_bp_adjoint(b, dvol, g, dout, c->isx, c->isy, c->ieee_rcp, c->cull, c->stream);
    }
    if (e == cudaSuccess && !out_on_device) {
        e = cudaMemcpyAsync(images_out, dout, sizeof(float) * img_elems * n, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(c->stream);
    }
    if (dvol_tmp)
        cudaFreeAsync(dvol_tmp, c->stream);
    if (dout_tmp)
        cudaFreeAsync(dout_tmp, c->stream);
    if (e != cudaSuccess)
        return fail(c, e == cudaErrorMemoryAllocation ? BP_ENOMEM : BP_ECUDA, "bp_adjoint: %s",
                    cudaGetErrorString(e));
    return BP_OK;
}
