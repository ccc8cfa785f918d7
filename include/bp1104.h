/*
 * bp1104.h -- C ABI of the GB300 voxel-driven cone-beam backprojection
 * library (libbp1104.so).
 *
 * The method is the Feldkamp backprojection step studied by Treibig, Hager,
 * Hofmann, Hornegger and Wellein, "Pushing the limits for medical image
 * reconstruction on recent standard multicore processors" (Sect. 3.1,
 * Listing 1): for every voxel x of an L^3 volume and every filtered
 * projection image I_i with 3x4 projection matrix A_i,
 *
 *     (uw, vw, w) = A_i (x, 1),   u = uw / w,   v = vw / w
 *     VOL[x] += bilinear(I_i, u, v) / w^2
 *
 * where pixel (j, k) of an ISX x ISY image sits at (u, v) = (j, k) and pixels
 * outside the detector read as zero (the zero-padded image buffers of
 * Sect. 3.3).  The integer part of u and v is floor().
 *
 * Conventions for every entry point:
 *   - Volumes are L^3 float32, x fastest: index z*L*L + y*L + x.  Voxel
 *     (x, y, z) sits at world position O + R (x, y, z) in mm (Sect. 3.1: the
 *     volume is a 256 mm cube, R = 256 / L).
 *   - Projection stacks are n x ISY x ISX float32, row-major (I[k*ISX + j]).
 *   - Matrices are n x 3 x 4 float64, ROW-major (A[r*4 + c]; rows give uw,
 *     vw, w).  The paper's listing indexes the same matrix column-major.
 *   - "on_device" flags say whether a pointer is device memory (1) or host
 *     memory (0).  Host buffers should be page-locked for asynchronous copies.
 *   - The caller owns every buffer it passes.  Calls are asynchronous on the
 *     context's CUDA stream unless stated otherwise: buffers must stay valid
 *     and unmodified until the next bp_finalize / bp_get_state or a stream
 *     synchronisation.
 *   - Errors are status codes; nothing aborts or throws.  bp_last_error(ctx)
 *     returns the message of the last failure on that context
 *     (bp_last_error(NULL): the calling thread's last failure in a function
 *     without a context).
 *   - All arithmetic on the GPU is float32 except where noted; float64 is used
 *     on the GPU only to build and invert projection matrices.
 */
#ifndef BP1104_H
#define BP1104_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bp_ctx bp_ctx;

typedef enum {
    BP_OK = 0,        /* success */
    BP_EINVAL = 1,    /* invalid argument (size, pointer, geometry) */
    BP_ENOMEM = 2,    /* device or pinned allocation failed */
    BP_ECUDA = 3,     /* a CUDA runtime call failed; see bp_last_error */
    BP_ESTATE = 4,    /* call not allowed in the context's current state */
    BP_ETIMEOUT = 5   /* a bounded device-side wait gave up */
} bp_status;

/* Storage type of the projections inside the library (Sect. 3.1 uses single
 * precision; FP16 / BF16 halve the bytes gathered per update).  Coordinates,
 * the 1/w^2 weight and the accumulation are float32 for every type. */
typedef enum { BP_F32 = 0, BP_F16 = 1, BP_BF16 = 2 } bp_dtype;

/* Options for bp_set_option. */
typedef enum {
    /* 1: reciprocal 1/w by the IEEE round-to-nearest division; 0 (default):
     * the hardware approximate reciprocal (about 1 ulp).  Sect. 7.2 compares
     * the same two choices (divps against rcpps). */
    BP_OPT_IEEE_RCP = 1,
    /* Projections per volume pass, 1..64 (default 64).  The volume is read
     * and written once per pass (the image blocking of Sect. 6.2). */
    BP_OPT_BATCH = 2,
    /* 1: record a CUDA event pair around every backprojection kernel launch
     * on the context's stream, for bp_kernel_stats; 0 (default): off. */
    BP_OPT_TIMING = 3,
    /* Warp layout of the texture path's kernel: 8, 16 or 32 lanes along x
     * (the rest along z), or a two-digit code XY = X lanes along x by Y along
     * y (44, 42, 82, 24; the rest along z), or 108 (8 lanes along x, 8
     * voxels per lane instead of 4), or 0 (default): automatic, per batch --
     * 24 where one voxel step spans 4 or more pixels at the volume centre
     * (coarse voxels: 256^3 and coarser on a 1248x960 detector), else 8 for
     * BP_F32 projections and 108 for BP_F16 / BP_BF16 (the fastest layouts
     * measured on GB300 in each regime).  bp_query(BP_QUERY_LAST_LANES_X)
     * reports the layout used.  Every voxel sums its projections in the same
     * order whatever the layout; with per-projection centring the volumes
     * are bit-identical, with per-block centring (the BP_F32 default) the
     * blocks, and so the centring offsets, follow the layout and the float32
     * rounding differs within the same accuracy. */
    BP_OPT_LANES_X = 4,
    /* Data path of the backprojection: 0 (default) automatic, 1 texture
     * gathers, 2 TMA-staged shared-memory tiles.  With per-projection
     * centring (BP_OPT_BLOCK_CENTRE 0) the two give bit-identical BP_F32
     * volumes; 16-bit storage differs between them by the rounding of the
     * staged differences (the TMA path stores each pixel difference rounded
     * once, the texture path differences the rounded pixels).  The automatic
     * choice, made per batch, is the TMA path wherever the sampled
     * footprints of its bricks fit its staged boxes (fine voxels: 512^3 and
     * finer on the 1248x960 detector), else the texture path (coarse voxels,
     * whose footprints are too wide to stage: 256^3 on that detector).  The
     * TMA path allocates two sets of 64 staged images on first use (1.2 GB
     * for a 1248x960 detector).  bp_query(BP_QUERY_LAST_PATH) reports the
     * path taken. */
    BP_OPT_PATH = 5,
    /* 1 (default): skip, per block of voxels, the projections whose footprint
     * misses the detector (the line-wise clipping of Sect. 3.3 at block
     * granularity; the skipped terms are exactly zero, so the volume is
     * bit-identical); 0: compute every term.  For bp_adjoint, 1 also
     * accumulates each block's footprint in a shared-memory tile (32-bit
     * fixed point, scaled per block and projection so that no sum can
     * overflow) before adding it to the images with one atomic per pixel;
     * 0 uses float32 global atomics per update (the sums agree to about
     * 1e-6). */
    BP_OPT_CULL = 6,
    /* Host float32 images with the texture path: 1 (default) copy-engine
     * transfers straight into the arrays, image by image; 0 one linear
     * host-to-device copy per batch into a staging buffer, then a copy
     * kernel into the arrays. */
    BP_OPT_HOST_DIRECT = 7,
    /* 1 (default): centre the detector coordinates per block of voxels and
     * projection, 0: once per projection.  Applies to BP_F32 projections in
     * bp_add_projections (blocks: the texture kernel's thread block or the
     * TMA path's brick) and to bp_adjoint's shared-tile kernel
     * (32x32x4 blocks; BP_OPT_CULL 1).  Per-block centring costs a pre-pass
     * and 48 bytes of device memory per (block, projection of a batch), per
     * input set for bp_add_projections (768 MiB for a 512^3 volume on the
     * texture path, 192 MiB on the TMA path, 96 MiB for the adjoint), and
     * cuts the float32 rounding of u and v by the ratio of block to volume
     * footprint (rel-L2 5e-7 instead of 1e-5 for the backprojection on a
     * full 1248x960 detector, 6e-7 instead of 4e-6 for the adjoint).  16-bit
     * storage always centres per projection. */
    BP_OPT_BLOCK_CENTRE = 8,
    /* Depth of the TMA path's bricks of 32 x 16 x D voxels: 0 (default)
     * automatic, or D = 8, 12, 16.  Deeper bricks give each thread more
     * voxels per staged projection (less per-projection work per update) but
     * need taller staged boxes; the automatic choice takes, per batch, the
     * deepest brick whose box holds the footprints of a sample of bricks
     * (16 for 512^3 and 1024^3 on a 1248x960 detector).  With
     * per-projection centring (16-bit storage, or BP_OPT_BLOCK_CENTRE 0)
     * the depth changes speed only: every voxel sums the same float32 terms
     * in the same order.  With per-brick centring (the BP_F32 default) the
     * centring offsets follow the brick, so the float32 rounding differs
     * between depths within the same accuracy.
     * bp_query(BP_QUERY_LAST_BRICK_DEPTH) reports the depth used. */
    BP_OPT_BRICK_DEPTH = 9,
    /* BP_F16 storage: 1 scales each batch of projections by a power of four
     * before rounding it to float16, 0 (default) stores the float32 values as
     * they are.  Float16 overflows above 65504 and loses relative precision
     * below 2^-14 (subnormals); ramp-filtered projections in physical units
     * can fall outside that range.  With 1, a pass over each batch (on the
     * copy stream) finds max|p| over its images; they are stored as
     * p * 2^-2k with k chosen so that the largest value lies in
     * [2^12, 2^14), and the kernels multiply the batch's sums by 2^2k (the
     * scale folded into the weight 1/w^2 of every term; every step exact).
     * Where the unscaled float16 values and their pair differences are
     * normal numbers, the volume is bit-identical to the unscaled one;
     * elsewhere the scaled form keeps float16's relative precision.  No
     * effect for BP_F32 and BP_BF16 (bfloat16 has float32's exponent
     * range). */
    BP_OPT_PROJ_SCALE = 10
} bp_option;

/* Queries for bp_query. */
typedef enum {
    BP_QUERY_LAST_PATH = 1,          /* data path of the last batch: 1 texture, 2 TMA, 0 none yet */
    BP_QUERY_PROJECTIONS_ADDED = 2,  /* projections accumulated since create / reset / set_state */
    BP_QUERY_UPDATES_COMPUTED = 3,   /* voxel updates actually computed since create (culled blocks
                                      * excluded; synchronises the stream) */
    BP_QUERY_LAST_BRICK_DEPTH = 4,   /* brick depth of the last TMA-path batch (8, 12, 16; 0 none yet) */
    BP_QUERY_LAST_LANES_X = 5        /* warp layout of the last texture-path batch (BP_OPT_LANES_X codes; 0 none yet) */
} bp_query_what;

/* ---------------------------------------------------------------- context */

/* Create a backprojection context for an L^3 volume of voxel size R (mm)
 * whose voxel (0,0,0) centre is at O[0..2] (mm), and ISX x ISY projections
 * stored as proj_dtype.  cuda_stream is the cudaStream_t every later call on
 * this context is ordered on (NULL: the legacy default stream); it is fixed
 * for the context's lifetime.  The context allocates the
 * device volume (zeroed) and the projection staging on the current device.
 * Sect. 3.1 (problem statement: L, MM, offsets, ISX x ISY images).
 * Returns BP_EINVAL for L < 1, R <= 0, ISX or ISY outside [1, 32768], or
 * a NULL out; BP_ENOMEM when the device allocations fail. */
bp_status bp_create(bp_ctx **out, int L, double R, const double O[3],
                    int isx, int isy, bp_dtype proj_dtype, void *cuda_stream);

/* Like bp_create, for a z-slab of the L^3 grid: the context's volume is the
 * nz slices z0 .. z0 + nz - 1 of the grid (L x L x nz voxels, x fastest;
 * 1 <= nz, 0 <= z0 <= L - nz).  O is still the centre of the grid's voxel
 * (0,0,0).  Every call on the context (bp_add_projections, bp_finalize,
 * bp_get_state / bp_set_state, bp_adjoint, which reads an L x L x nz
 * volume) then works on the slab alone.  Slabs reconstruct a volume larger
 * than one context can hold (each slab takes every projection; the paper's
 * split of the z loop, Sect. 6), or split one volume across GPUs.
 * bp_create(L, ...) is bp_create_slab(L, L, 0, ...).  Other errors as
 * bp_create. */
bp_status bp_create_slab(bp_ctx **out, int L, int nz, int z0, double R, const double O[3],
                         int isx, int isy, bp_dtype proj_dtype, void *cuda_stream);

/* Re-target a context to the z-slab of slices z0 .. z0+nz-1 of the same
 * L^3 grid (same L, R, O, detector and storage type), keeping its device
 * allocations: 1 <= nz <= the slab depth the context was created with (L for
 * bp_create), 0 <= z0 <= L - nz.  Waits for the context's work in flight,
 * then zeroes the volume and the projection counter.  A volume larger than
 * the device is reconstructed by moving one or two slab contexts over it
 * (Sect. 6's split of the z loop), without a context per slab.  BP_EINVAL for
 * a NULL context or a slab outside those bounds. */
bp_status bp_move_slab(bp_ctx *ctx, int z0, int nz);

/* Release everything the context owns (synchronises its stream first).
 * NULL is accepted and ignored. */
bp_status bp_destroy(bp_ctx *ctx);

/* Set a bp_option (see above).  BP_EINVAL for an unknown option or value. */
bp_status bp_set_option(bp_ctx *ctx, int option, long long value);

/* Zero the volume and the projection counter (asynchronous). */
bp_status bp_reset(bp_ctx *ctx);

/* Accumulate n projections into the volume (Sect. 3.1, Listing 1; images
 * arrive one by one or in batches, Sect. 6):
 *   images: n x ISY x ISX float32, host (images_on_device = 0) or device;
 *   A:      n x 3 x 4 float64 row-major, HOST memory, read before return.
 * VOL += sum_i bilinear(I_i, A_i x) / w^2 over the n images.  Every voxel of
 * the volume must lie in front of every source (w > 0 at the 8 corners of
 * the volume box), else BP_EINVAL.  n = 0 is a no-op.  Host images are
 * copied while earlier batches compute; the call returns when the last copy
 * has been queued. */
bp_status bp_add_projections(bp_ctx *ctx, const float *images, int images_on_device,
                             const double *A, int n);

/* Synchronise the stream and copy the volume (L^3 float32) to vol_out (host
 * or device).  The context stays usable; further bp_add_projections keep
 * accumulating onto the same volume until bp_reset. */
bp_status bp_finalize(bp_ctx *ctx, float *vol_out, int on_device);

/* bp_add_projections followed by bp_finalize, in one call (Sect. 3.1: the
 * images of a scan in, the finished volume out):
 *   images, images_on_device, A, n: as bp_add_projections;
 *   vol_out: the volume's L x L x Lz float32 destination, host
 *            (out_on_device = 0) or device, owned by the caller.
 * The result equals bp_add_projections + bp_finalize bit for bit, and the
 * context keeps the volume as after them.  On the TMA path the last batch's
 * launch also stores every voxel's final value into vol_out directly: device
 * memory, or page-locked host memory (cudaHostAlloc, cudaHostRegister),
 * through its device mapping, so the read-back overlaps that launch instead
 * of following it.  Other host memory is copied after the launch.  The call
 * synchronises.  n = 0 is bp_finalize.  Errors as bp_add_projections and
 * bp_finalize (BP_EINVAL for a NULL context or output). */
bp_status bp_add_projections_finalize(bp_ctx *ctx, const float *images, int images_on_device,
                                      const double *A, int n, float *vol_out, int out_on_device);

/* Checkpoint: copy the partial volume and the number of projections added so
 * far (synchronous).  vol_out may be NULL to read only the counter. */
bp_status bp_get_state(bp_ctx *ctx, float *vol_out, int on_device, long long *n_added);

/* Resume: replace the volume by vol_in (L^3 float32, host or device) and set
 * the projection counter.  Continuing from a saved state gives the same
 * volume, bit for bit, as one uninterrupted run with the same batches. */
bp_status bp_set_state(bp_ctx *ctx, const float *vol_in, int on_device, long long n_added);

/* Adjoint (transpose) of the backprojection: for every voxel value f(x) and
 * projection i, spread f(x) / w^2 onto the four pixels around (u, v) with the
 * bilinear weights (1-fu)(1-fv), fu(1-fv), (1-fu)fv, fu fv; pixels outside
 * the detector are dropped.  This is the transpose of the sum in Listing 1
 * (Sect. 3.1): <B p, f> = <p, B^T f>.
 *   vol:        L^3 float32 (host or device per vol_on_device);
 *   A:          n x 3 x 4 float64 row-major, HOST memory;
 *   images_out: n x ISY x ISX float32 (host or device per out_on_device),
 *               overwritten (the callee zeroes it first).
 * With BP_OPT_CULL 1 (the default) each block of 32x32x4 voxels sums its
 * terms for a projection in a shared-memory tile in 32-bit fixed point
 * (native integer atomics; the scale is a power of two per block and
 * projection, bounded so that no sum overflows, each term rounded to 2^-31
 * of the block's bound), then adds each nonzero tile pixel to the image with
 * one float32 global atomic; blocks whose footprint exceeds the tile, and
 * BP_OPT_CULL 0, add every term with float32 global atomics.  The float32
 * atomics make the summation order (and the last bits) vary between runs.
 * Leaves the context's volume untouched. */
bp_status bp_adjoint(bp_ctx *ctx, const float *vol, int vol_on_device,
                     const double *A, int n, float *images_out, int out_on_device);

/* Read a bp_query_what value into *value.  BP_EINVAL for an unknown query. */
bp_status bp_query(bp_ctx *ctx, int what, long long *value);

/* Device time of the backprojection kernel launches recorded while
 * BP_OPT_TIMING was on (measurement support, in the spirit of the paper's
 * hardware-counter timelines, Sect. 7): synchronises the stream, returns the
 * number of launches and their summed CUDA-event time in ms, and clears the
 * record.  Either output pointer may be NULL. */
bp_status bp_kernel_stats(bp_ctx *ctx, long long *launches, double *total_ms);

/* Measured speed of light of Part 2 of Listing 1 (Sect. 3.1) on this GPU:
 * the texture unit's 2x2-gather rate for projections stored as `dtype`, in
 * gathers per SM per clock, with the backprojection kernel's warp shape
 * (lanes on neighbouring pixels) and an L1-resident footprint.  The paper
 * bases its bounds on measured machine figures (Sect. 2, Table 1; Sect. 3.2);
 * this is the GPU counterpart used for the roofline.  Synchronous (runs a
 * short kernel on the current device, allocating and freeing a 256 x 256
 * array). */
bp_status bp_probe_gather(bp_dtype dtype, double *gathers_per_sm_clk);

/* Self-test of the failure detection of the TMA path's device-side waits (no
 * counterpart in the paper).  One warp waits, with the bounded wait the
 * backprojection kernel uses, on a barrier that is completed (arrive = 1)
 * or that nothing completes (arrive = 0), at most iters (1 .. 2^20)
 * suspensions of 100 us each.  Returns BP_OK when the wait succeeded and
 * BP_ETIMEOUT when it gave up; nothing faults or hangs, and the device stays
 * usable.  BP_EINVAL for bad arguments (checked before any CUDA call).
 * Synchronous, on the current device. */
bp_status bp_selftest_bounded_wait(int arrive, int iters);

/* Message of the last failure on ctx (or, for ctx == NULL, of the calling
 * thread's last failing context-free call).  Never NULL. */
const char *bp_last_error(const bp_ctx *ctx);

/* ------------------------------------------------------ context-free calls
 * All pointers below are DEVICE pointers unless stated; work is queued on
 * `stream` (a cudaStream_t, NULL = legacy default stream). */

/* Projection matrices of a circular C-arm scan about z, built in float64 on
 * the GPU: source at sid (cos b, sin b, 0), detector at distance sdd from the
 * source with u axis (-sin b, cos b, 0), v axis (0, 0, 1), square pixels of
 * `pitch` mm and principal point (cu, cv); scaled so that w = depth / sid.
 * beta: n angles in radians (HOST); A_out: n x 12 float64 (device). */
bp_status bp_carm_matrices(int n, const double *beta, double sid, double sdd, double pitch,
                           double cu, double cv, double *A_out, void *stream);

/* Analytic line integrals of an additive ellipsoid phantom (test data for
 * the FDK pipeline, Sect. 1.1): out[i][k][j] = sum_e rho_e * chord length of
 * the ray from the source of A_i through pixel (j, k).  A: n x 12 float64
 * (device; sources and ray directions are found by inverting A in float64);
 * ell: count x 16 float64 (device; centre 3, semi-axes 3, row-major rotation
 * 9 whose columns are the axes, density 1); out: n x isy x isx float32. */
bp_status bp_ellipsoid_project(int n, const double *A, int isx, int isy, int count,
                               const double *ell, float *out, void *stream);

/* Phantom density at every voxel centre of an L^3 grid (R, O as above):
 * vol[z][y][x] = sum of rho_e over ellipsoids containing the centre. */
bp_status bp_ellipsoid_voxelize(int L, double R, const double O[3], int count,
                                const double *ell, float *vol, void *stream);

/* FDK pre-weighting (Sect. 1.1, 2-D pre-processing): out = in * scale *
 * sdd / sqrt(sdd^2 + ut^2 + vt^2) * parker(b_i, atan(ut / sdd)) with
 * ut = (j - cu) pitch, vt = (k - cv) pitch, b_i = beta[i] - beta[0] and the
 * Parker short-scan weight for a scan of beta[n-1] - beta[0] = pi + 2 delta
 * (parker = 0 drops that factor).  beta: HOST, n values; in/out: n x isy x
 * isx float32 device (in == out allowed). */
bp_status bp_fdk_preweight(int n, int isx, int isy, double pitch, double sdd, double cu,
                           double cv, const double *beta, int parker, double scale,
                           const float *in, float *out, void *stream);

/* Ramp filter: row-wise linear (zero-padded) convolution with the Ram-Lak
 * kernel h(0) = 1/(4 tau^2), h(odd m) = -1/(m^2 pi^2 tau^2), h(even) = 0:
 * out[r][j] = tau * sum_j' h(j - j') in[r][j'], rows rows of isx floats.
 * in and out must not overlap. */
bp_status bp_ramp_filter(long long rows, int isx, double tau, const float *in, float *out,
                         void *stream);

/* Short per-row filter (the learned replacement of the ramp, T <= 256 taps):
 * out[r][j] = sum_t h[t] in[r][j + t - T/2], zero outside the row.
 * h: T float32 (device).  in and out must not overlap. */
bp_status bp_row_filter_fwd(long long rows, int isx, int T, const float *h, const float *in,
                            float *out, void *stream);

/* Gradients of bp_row_filter_fwd for dL/dout = g:
 *   gin[r][s] = sum_t h[t] g[r][s - t + T/2]           (may be NULL to skip)
 *   gh[t]     = sum_{r,j} g[r][j] in[r][j + t - T/2]   (may be NULL to skip)
 * gh is reduced deterministically in two passes through a scratch buffer the
 * call allocates (stream-ordered) and frees. */
bp_status bp_row_filter_bwd(long long rows, int isx, int T, const float *h, const float *in,
                            const float *g, float *gin, float *gh, void *stream);

/* Allocation-free form of bp_row_filter_bwd (the paper has no counterpart:
 * this serves callers of the library, not the method).  Same arguments and
 * results (gh summed in a different but fixed order, so within float32
 * rounding of bp_row_filter_bwd's, and deterministic), for callers that must
 * not allocate device memory once running -- e.g. a reconstruction loop that
 * budgets all device memory at start-up, or a host framework whose allocator
 * owns the device.  Its scratch is a fixed 128 KiB device array inside the
 * library (256 blocks x 128 taps of float32), held by every GPU that loads
 * the library until the process exits; T above 128 is rejected with
 * BP_EINVAL.  The first call in each CUDA context (the device's primary
 * context, a context created after cudaDeviceReset, or a non-primary
 * context made current by the caller) looks up the array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream capture.
 * All calls share the array: calls that overlap on the GPU (e.g. on two
 * streams) race and must be serialised by the caller.  Makes no call to
 * cudaMalloc, cudaMallocAsync or cudaFree. */
bp_status bp_row_filter_bwd_noalloc(long long rows, int isx, int T, const float *h,
                                    const float *in, const float *g, float *gin, float *gh,
                                    void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BP1104_H */
