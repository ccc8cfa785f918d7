// Support kernels around the backprojection: projection matrices (float64,
// the only float64 on the GPU), analytic phantom projections and
// voxelisation (test data), the FDK 2-D pre-processing (cosine + Parker
// weights, Ram-Lak ramp filter; Sect. 1.1 names the step) and the short
// learned per-row filter with its gradients.
#include <cmath>
#include <cstdarg>
#include <cstdio>

#include "bp_internal.cuh"

namespace bp {

static thread_local char g_thread_err[1024] = "no error";

void set_thread_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_thread_err, sizeof g_thread_err, fmt, ap);
    va_end(ap);
}

const char *thread_error() { return g_thread_err; }

static bp_status cuda_fail(cudaError_t e, const char *what)
{
    set_thread_error("%s: %s", what, cudaGetErrorString(e));
    return BP_ECUDA;
}

#define BP_CK(call)                                  \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess)                       \
            return cuda_fail(e_, #call);             \
    } while (0)

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// Matrices of a circular C-arm scan (float64).  Chunks of angles travel as
// kernel parameters.
constexpr int kAngleChunk = 480;
struct AngleChunk {
    double beta[kAngleChunk];
    int n;
};

__global__ void carm_matrices_kernel(const __grid_constant__ AngleChunk c, double sid, double sdd,
                                     double pitch, double cu, double cv, double *A)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.n)
        return;
    double sb, cb;
    sincos(c.beta[i], &sb, &cb);
    const double g = sdd / (pitch * sid);
    // w = (d . X + sid) / sid with d = -(cos b, sin b, 0)
    const double w0 = -cb / sid, w1 = -sb / sid;
    double *a = A + 12 * (long long)i;
    // uw = g (e_u . X) + cu w, e_u = (-sin b, cos b, 0); vw = g z + cv w
    a[0] = fma(cu, w0, -g * sb);
    a[1] = fma(cu, w1, g * cb);
    a[2] = 0.0;
    a[3] = cu;
    a[4] = cv * w0;
    a[5] = cv * w1;
    a[6] = g;
    a[7] = cv;
    a[8] = w0;
    a[9] = w1;
    a[10] = 0.0;
    a[11] = 1.0;
}

// Source position and inverse of the left 3x3 block, float64: with
// A = [M | a], the source is S = -M^{-1} a and the ray through pixel (u, v)
// points along M^{-1} (u, v, 1).  Output per projection (12 doubles):
// Minv row-major (9) then S (3).
__global__ void invert_kernel(int n, const double *__restrict__ A, double *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const double *a = A + 12 * (long long)i;
    const double m00 = a[0], m01 = a[1], m02 = a[2];
    const double m10 = a[4], m11 = a[5], m12 = a[6];
    const double m20 = a[8], m21 = a[9], m22 = a[10];
    const double c00 = m11 * m22 - m12 * m21;
    const double c01 = m12 * m20 - m10 * m22;
    const double c02 = m10 * m21 - m11 * m20;
    const double det = m00 * c00 + m01 * c01 + m02 * c02;
    const double id = 1.0 / det;
    double Mi[9] = {c00 * id, (m02 * m21 - m01 * m22) * id, (m01 * m12 - m02 * m11) * id,
                    c01 * id, (m00 * m22 - m02 * m20) * id, (m02 * m10 - m00 * m12) * id,
                    c02 * id, (m01 * m20 - m00 * m21) * id, (m00 * m11 - m01 * m10) * id};
    double *o = out + 12 * (long long)i;
    for (int r = 0; r < 9; ++r)
        o[r] = Mi[r];
    for (int r = 0; r < 3; ++r)
        o[9 + r] = -(Mi[3 * r] * a[3] + Mi[3 * r + 1] * a[7] + Mi[3 * r + 2] * a[11]);
}

// ---------------------------------------------------------------------------
// Ellipsoid phantoms.  Per ellipsoid (float32 in shared memory): centre (3),
// rows of Q^T scaled by 1/a_k (9: maps X - c to the unit-sphere frame),
// density.
constexpr int kEllStride = 13;
constexpr int kMaxEll = 256;

__device__ __forceinline__ void load_ellipsoids(const double *__restrict__ ell, int count,
                                                float *sm)
{
    for (int e = threadIdx.x; e < count; e += blockDim.x) {
        const double *q = ell + 16 * e;
        float *s = sm + kEllStride * e;
        s[0] = (float)q[0];
        s[1] = (float)q[1];
        s[2] = (float)q[2];
        for (int k = 0; k < 3; ++k)       // row k of Q^T / a_k = column k of Q / a_k
            for (int c = 0; c < 3; ++c)
                s[3 + 3 * k + c] = (float)(q[6 + 3 * c + k] / q[3 + k]);
        s[12] = (float)q[15];
    }
}

// Chord length of the ray P0 + t d (|d| = 1) inside one ellipsoid.  In the
// unit-sphere frame the ray is p(t) = s0 + t sd; with t* = -(s0.sd)/|sd|^2
// the closest point m = s0 + t* sd gives the chord 2 sqrt((1 - |m|^2)/|sd|^2)
// (|m|^2 is formed from m itself, avoiding the cancellation of the
// discriminant).  P0 is taken near the ellipsoid, at the foot of its centre
// on the ray, so that s0 is small.
__device__ __forceinline__ float chord_len(const float *e, float Sx, float Sy, float Sz, float dx,
                                           float dy, float dz)
{
    const float cx = e[0] - Sx, cy = e[1] - Sy, cz = e[2] - Sz;
    const float tc = cx * dx + cy * dy + cz * dz;
    const float px = fmaf(tc, dx, -cx), py = fmaf(tc, dy, -cy), pz = fmaf(tc, dz, -cz);
    float s0[3], sd[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float *row = e + 3 + 3 * k;
        s0[k] = row[0] * px + row[1] * py + row[2] * pz;
        sd[k] = row[0] * dx + row[1] * dy + row[2] * dz;
    }
    const float qa = sd[0] * sd[0] + sd[1] * sd[1] + sd[2] * sd[2];
    const float ts = -(s0[0] * sd[0] + s0[1] * sd[1] + s0[2] * sd[2]) / qa;
    const float m0 = fmaf(ts, sd[0], s0[0]), m1 = fmaf(ts, sd[1], s0[1]), m2 = fmaf(ts, sd[2], s0[2]);
    const float h = 1.f - (m0 * m0 + m1 * m1 + m2 * m2);
    return h > 0.f ? 2.f * sqrtf(h / qa) : 0.f;
}

__global__ void __launch_bounds__(256)
ellipsoid_project_kernel(const double *__restrict__ inv, int isx, int isy, int count,
                         const double *__restrict__ ell, float *__restrict__ out)
{
    __shared__ float sm[kEllStride * kMaxEll];
    __shared__ float geo[12];
    const int i = blockIdx.z;
    load_ellipsoids(ell, count, sm);
    if (threadIdx.x < 12)
        geo[threadIdx.x] = (float)inv[12 * (long long)i + threadIdx.x];
    __syncthreads();
    const int j = blockIdx.x * 32 + (threadIdx.x & 31);
    const int k = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (j >= isx || k >= isy)
        return;
    const float fj = (float)j, fk = (float)k;
    float dx = fmaf(geo[0], fj, fmaf(geo[1], fk, geo[2]));
    float dy = fmaf(geo[3], fj, fmaf(geo[4], fk, geo[5]));
    float dz = fmaf(geo[6], fj, fmaf(geo[7], fk, geo[8]));
    const float nd = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= nd;
    dy *= nd;
    dz *= nd;
    float acc = 0.f;
    for (int e = 0; e < count; ++e)
        acc = fmaf(sm[kEllStride * e + 12], chord_len(sm + kEllStride * e, geo[9], geo[10], geo[11], dx, dy, dz), acc);
    out[((long long)i * isy + k) * isx + j] = acc;
}

__global__ void __launch_bounds__(256)
ellipsoid_voxelize_kernel(int L, float R, float Ox, float Oy, float Oz, int count,
                          const double *__restrict__ ell, float *__restrict__ vol)
{
    __shared__ float sm[kEllStride * kMaxEll];
    load_ellipsoids(ell, count, sm);
    __syncthreads();
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int z = blockIdx.z;
    if (x >= L || y >= L)
        return;
    const float X = fmaf(R, (float)x, Ox), Y = fmaf(R, (float)y, Oy), Z = fmaf(R, (float)z, Oz);
    float acc = 0.f;
    for (int e = 0; e < count; ++e) {
        const float *s = sm + kEllStride * e;
        const float px = X - s[0], py = Y - s[1], pz = Z - s[2];
        float r2 = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float t = s[3 + 3 * k] * px + s[4 + 3 * k] * py + s[5 + 3 * k] * pz;
            r2 = fmaf(t, t, r2);
        }
        if (r2 <= 1.f)
            acc += s[12];
    }
    vol[((long long)z * L + y) * L + x] = acc;
}

// ---------------------------------------------------------------------------
// FDK pre-weighting: cosine weight times the Parker short-scan weight.
constexpr int kWeightChunk = 960;
struct WeightChunk {
    float b[kWeightChunk];   // scan angle beta_i - beta_0 of each image
    int n;
};

__device__ __forceinline__ float parker_f(float b, float g, float delta)
{
    const float gs = -g;  // this geometry's conjugate ray is (b + pi - 2g, -g)
    const float pi = 3.14159265358979f;
    if (b < 0.f || b > pi + 2.f * delta)
        return 0.f;
    if (b < 2.f * (delta - gs)) {
        const float t = sinf(0.25f * pi * b / (delta - gs));
        return t * t;
    }
    if (b <= pi - 2.f * gs)
        return 1.f;
    const float t = sinf(0.25f * pi * (pi + 2.f * delta - b) / (delta + gs));
    return t * t;
}

__global__ void __launch_bounds__(256)
preweight_kernel(const __grid_constant__ WeightChunk c, int isx, int isy, float pitch, float sdd,
                 float cu, float cv, int parker, float delta, float scale,
                 const float *__restrict__ in, float *__restrict__ out)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    const int i = blockIdx.z;
    if (j >= isx)
        return;
    const float ut = ((float)j - cu) * pitch, vt = ((float)k - cv) * pitch;
    float wgt = scale * sdd * rsqrtf(sdd * sdd + ut * ut + vt * vt);
    if (parker)
        wgt *= parker_f(c.b[i], atanf(ut / sdd), delta);
    const long long q = ((long long)i * isy + k) * isx + j;
    out[q] = wgt * in[q];
}

// ---------------------------------------------------------------------------
// Ram-Lak ramp filter, one row per block.  The row sits in shared memory
// between isx zeros on each side; with the symmetric kernel
// out[j] = tau (h0 x[j] + sum_{odd m} h_m (x[j-m] + x[j+m])) the loop over m
// is uniform across the block and needs no bounds tests.
__global__ void __launch_bounds__(256)
ramp_kernel(long long rows, int isx, float tau, const float *__restrict__ in, float *__restrict__ out)
{
    extern __shared__ float sm[];
    float *xs = sm;                 // 3 * isx: zeros | row | zeros
    float *hm = sm + 3 * isx;       // h_m for odd m at hm[(m-1)/2]
    const long long r = blockIdx.x;
    const float *x = in + r * isx;
    for (int t = threadIdx.x; t < 3 * isx; t += blockDim.x)
        xs[t] = (t >= isx && t < 2 * isx) ? x[t - isx] : 0.f;
    const float pi2tau2 = 9.8696044010893586f * tau * tau;
    for (int t = threadIdx.x; t < (isx + 1) / 2; t += blockDim.x) {
        const float m = (float)(2 * t + 1);
        hm[t] = -1.f / (m * m * pi2tau2);
    }
    __syncthreads();
    const float h0 = 0.25f / (tau * tau);
    for (int j = threadIdx.x; j < isx; j += blockDim.x) {
        const float *c = xs + isx + j;
        float acc = h0 * c[0];
        for (int t = 0, m = 1; m < isx; ++t, m += 2)
            acc = fmaf(hm[t], c[-m] + c[m], acc);
        out[r * isx + j] = tau * acc;
    }
}

// ---------------------------------------------------------------------------
// Learned per-row filter.  kRowsPerBlock rows per block; each row sits in
// shared memory with T zeros on the left and T on the right.
constexpr int kMaxTaps = 256;
constexpr int kRowsPerBlock = 4;

__global__ void __launch_bounds__(256)
row_filter_fwd_kernel(long long rows, int isx, int T, const float *__restrict__ h,
                      const float *__restrict__ in, float *__restrict__ out)
{
    extern __shared__ float sm[];
    __shared__ float hs[kMaxTaps];
    const int pitch = isx + 2 * T;
    const long long r0 = (long long)blockIdx.x * kRowsPerBlock;
    for (int t = threadIdx.x; t < T; t += blockDim.x)
        hs[t] = h[t];
    for (int q = threadIdx.x; q < kRowsPerBlock * pitch; q += blockDim.x) {
        const int rr = q / pitch, c = q % pitch - T;
        const long long r = r0 + rr;
        sm[q] = (r < rows && c >= 0 && c < isx) ? in[r * isx + c] : 0.f;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kRowsPerBlock * isx; q += blockDim.x) {
        const int rr = q / isx, j = q % isx;
        const long long r = r0 + rr;
        if (r >= rows)
            break;
        const float *c = sm + rr * pitch + T + j - T / 2;   // c[t] = in[j + t - T/2]
        float acc = 0.f;
        for (int t = 0; t < T; ++t)
            acc = fmaf(hs[t], c[t], acc);
        out[r * isx + j] = acc;
    }
}

// gin[s] = sum_t h[t] g[s - t + T/2]; partial[blk][t] = sum over the block's
// rows of sum_j g[j] in[j + t - T/2].
__global__ void __launch_bounds__(256)
row_filter_bwd_kernel(long long rows, int isx, int T, const float *__restrict__ h,
                      const float *__restrict__ in, const float *__restrict__ g,
                      float *__restrict__ gin, float *__restrict__ partial)
{
    extern __shared__ float sm[];
    __shared__ float hs[kMaxTaps];
    __shared__ float red[256];
    const int pitch = isx + 2 * T;
    float *xs = sm;                            // inputs, padded
    float *gs = sm + kRowsPerBlock * pitch;    // upstream gradient, padded
    const long long r0 = (long long)blockIdx.x * kRowsPerBlock;
    for (int t = threadIdx.x; t < T; t += blockDim.x)
        hs[t] = h[t];
    for (int q = threadIdx.x; q < kRowsPerBlock * pitch; q += blockDim.x) {
        const int rr = q / pitch, c = q % pitch - T;
        const long long r = r0 + rr;
        const bool ok = r < rows && c >= 0 && c < isx;
        xs[q] = ok ? in[r * isx + c] : 0.f;
        gs[q] = ok ? g[r * isx + c] : 0.f;
    }
    __syncthreads();
    if (gin != nullptr) {
        for (int q = threadIdx.x; q < kRowsPerBlock * isx; q += blockDim.x) {
            const int rr = q / isx, s = q % isx;
            const long long r = r0 + rr;
            if (r >= rows)
                break;
            const float *c = gs + rr * pitch + T + s + T / 2;   // c[-t] = g[s - t + T/2]
            float acc = 0.f;
            for (int t = 0; t < T; ++t)
                acc = fmaf(hs[t], c[-t], acc);
            gin[r * isx + s] = acc;
        }
    }
    if (partial != nullptr) {
        // 256 threads: tap t = tid % T, lane group sweeps a slice of columns;
        // fixed-order reduction of the groups keeps the result deterministic.
        const int groups = blockDim.x / T;
        const int t = threadIdx.x % T, grp = threadIdx.x / T;
        float acc = 0.f;
        if (grp < groups) {
            for (int rr = 0; rr < kRowsPerBlock; ++rr) {
                const float *xr = xs + rr * pitch + T + t - T / 2;   // xr[j] = in[j + t - T/2]
                const float *gr = gs + rr * pitch + T;
                for (int j = grp; j < isx; j += groups)
                    acc = fmaf(gr[j], xr[j], acc);
            }
        }
        red[threadIdx.x] = acc;
        __syncthreads();
        if (threadIdx.x < T) {
            float s = 0.f;
            for (int q = 0; q < groups; ++q)
                s += red[q * T + threadIdx.x];
            partial[(long long)blockIdx.x * T + threadIdx.x] = s;
        }
    }
}

// Sum partial[b][t] over blocks b, fixed order: one block per tap.
__global__ void __launch_bounds__(256)
reduce_taps_kernel(long long nblk, int T, const float *__restrict__ partial, float *__restrict__ gh)
{
    __shared__ float red[256];
    const int t = blockIdx.x;
    float s = 0.f;
    for (long long b = threadIdx.x; b < nblk; b += blockDim.x)
        s += partial[b * T + t];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        gh[t] = red[0];
}

}  // namespace bp

// ============================================================================
// C ABI (context-free entry points)
using namespace bp;

extern "C" bp_status bp_carm_matrices(int n, const double *beta, double sid, double sdd,
                                      double pitch, double cu, double cv, double *A_out,
                                      void *stream)
{
    if (n < 0 || (n > 0 && (beta == nullptr || A_out == nullptr)) || !(sid > 0) || !(sdd > 0) ||
        !(pitch > 0)) {
        set_thread_error("bp_carm_matrices: invalid argument");
        return BP_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    for (int c0 = 0; c0 < n; c0 += kAngleChunk) {
        AngleChunk c;
        c.n = n - c0 < kAngleChunk ? n - c0 : kAngleChunk;
        for (int i = 0; i < c.n; ++i)
            c.beta[i] = beta[c0 + i];
        carm_matrices_kernel<<<(c.n + 127) / 128, 128, 0, s>>>(c, sid, sdd, pitch, cu, cv,
                                                               A_out + 12 * (long long)c0);
        BP_CK(cudaGetLastError());
    }
    return BP_OK;
}

extern "C" bp_status bp_ellipsoid_project(int n, const double *A, int isx, int isy, int count,
                                          const double *ell, float *out, void *stream)
{
    if (n < 0 || isx < 1 || isy < 1 || count < 0 || count > kMaxEll || isy > 65535 * 8 ||
        (n > 0 && (A == nullptr || out == nullptr)) || (count > 0 && ell == nullptr)) {
        set_thread_error("bp_ellipsoid_project: invalid argument (count <= %d)", kMaxEll);
        return BP_EINVAL;
    }
    if (n == 0)
        return BP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    double *inv = nullptr;
    BP_CK(cudaMallocAsync((void **)&inv, sizeof(double) * 12 * (size_t)n, s));
    invert_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, A, inv);
    cudaError_t e = cudaGetLastError();
    for (int i0 = 0; e == cudaSuccess && i0 < n; i0 += 65535) {
        const int m = n - i0 < 65535 ? n - i0 : 65535;
        dim3 grid((isx + 31) / 32, (isy + 7) / 8, m);
        ellipsoid_project_kernel<<<grid, 256, 0, s>>>(inv + 12 * (long long)i0, isx, isy, count, ell,
                                                      out + (long long)i0 * isx * isy);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaFreeAsync(inv, s);
    BP_CK(e);
    BP_CK(e2);
    return BP_OK;
}

extern "C" bp_status bp_ellipsoid_voxelize(int L, double R, const double O[3], int count,
                                           const double *ell, float *vol, void *stream)
{
    if (L < 1 || L > 65535 || !(R > 0) || O == nullptr || vol == nullptr || count < 0 ||
        count > kMaxEll || (count > 0 && ell == nullptr)) {
        set_thread_error("bp_ellipsoid_voxelize: invalid argument");
        return BP_EINVAL;
    }
    dim3 grid((L + 31) / 32, (L + 7) / 8, L);
    ellipsoid_voxelize_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(
        L, (float)R, (float)O[0], (float)O[1], (float)O[2], count, ell, vol);
    BP_CK(cudaGetLastError());
    return BP_OK;
}

extern "C" bp_status bp_fdk_preweight(int n, int isx, int isy, double pitch, double sdd, double cu,
                                      double cv, const double *beta, int parker, double scale,
                                      const float *in, float *out, void *stream)
{
    if (n < 0 || isx < 1 || isy < 1 || isy > 65535 || !(pitch > 0) || !(sdd > 0) ||
        (n > 0 && (beta == nullptr || in == nullptr || out == nullptr))) {
        set_thread_error("bp_fdk_preweight: invalid argument");
        return BP_EINVAL;
    }
    if (n == 0)
        return BP_OK;
    const double delta = n > 1 ? 0.5 * (std::fabs(beta[n - 1] - beta[0]) - kPi) : 0.0;
    for (int c0 = 0; c0 < n; c0 += kWeightChunk) {
        WeightChunk c;
        c.n = n - c0 < kWeightChunk ? n - c0 : kWeightChunk;
        for (int i = 0; i < c.n; ++i)
            c.b[i] = (float)std::fabs(beta[c0 + i] - beta[0]);
        const long long off = (long long)c0 * isx * isy;
        dim3 grid((isx + 255) / 256, isy, c.n);
        preweight_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(
            c, isx, isy, (float)pitch, (float)sdd, (float)cu, (float)cv, parker, (float)delta,
            (float)scale, in + off, out + off);
        BP_CK(cudaGetLastError());
    }
    return BP_OK;
}

extern "C" bp_status bp_ramp_filter(long long rows, int isx, double tau, const float *in, float *out,
                                    void *stream)
{
    if (rows < 0 || isx < 1 || isx > 8192 || !(tau > 0) ||
        (rows > 0 && (in == nullptr || out == nullptr))) {
        set_thread_error("bp_ramp_filter: invalid argument (isx <= 8192)");
        return BP_EINVAL;
    }
    if (rows == 0)
        return BP_OK;
    const size_t smem = sizeof(float) * (3 * (size_t)isx + (isx + 1) / 2);
    if (smem > 48 * 1024)
        BP_CK(cudaFuncSetAttribute(ramp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (long long r0 = 0; r0 < rows; r0 += 0x7fffffffLL) {
        const long long m = rows - r0 < 0x7fffffffLL ? rows - r0 : 0x7fffffffLL;
        ramp_kernel<<<(unsigned)m, 256, smem, (cudaStream_t)stream>>>(m, isx, (float)tau, in + r0 * isx,
                                                                      out + r0 * isx);
        BP_CK(cudaGetLastError());
    }
    return BP_OK;
}

static bp_status check_row_filter(const char *who, long long rows, int isx, int T)
{
    const size_t smem = sizeof(float) * 2 * kRowsPerBlock * (size_t)(isx + 2 * T);
    if (rows < 0 || isx < 1 || T < 1 || T > kMaxTaps || smem > 200 * 1024) {
        set_thread_error("%s: invalid argument (1 <= T <= %d, row too long)", who, kMaxTaps);
        return BP_EINVAL;
    }
    return BP_OK;
}

extern "C" bp_status bp_row_filter_fwd(long long rows, int isx, int T, const float *h,
                                       const float *in, float *out, void *stream)
{
    bp_status st = check_row_filter("bp_row_filter_fwd", rows, isx, T);
    if (st != BP_OK)
        return st;
    if (rows == 0)
        return BP_OK;
    if (h == nullptr || in == nullptr || out == nullptr) {
        set_thread_error("bp_row_filter_fwd: NULL pointer");
        return BP_EINVAL;
    }
    const size_t smem = sizeof(float) * kRowsPerBlock * (size_t)(isx + 2 * T);
    if (smem > 48 * 1024)
        BP_CK(cudaFuncSetAttribute(row_filter_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long nblk = (rows + kRowsPerBlock - 1) / kRowsPerBlock;
    if (nblk > 0x7fffffffLL) {
        set_thread_error("bp_row_filter_fwd: too many rows");
        return BP_EINVAL;
    }
    row_filter_fwd_kernel<<<(unsigned)nblk, 256, smem, (cudaStream_t)stream>>>(rows, isx, T, h, in, out);
    BP_CK(cudaGetLastError());
    return BP_OK;
}

extern "C" bp_status bp_row_filter_bwd(long long rows, int isx, int T, const float *h,
                                       const float *in, const float *g, float *gin, float *gh,
                                       void *stream)
{
    bp_status st = check_row_filter("bp_row_filter_bwd", rows, isx, T);
    if (st != BP_OK)
        return st;
    if (gh != nullptr && rows == 0) {
        BP_CK(cudaMemsetAsync(gh, 0, sizeof(float) * T, (cudaStream_t)stream));
        return BP_OK;
    }
    if (rows == 0 || (gin == nullptr && gh == nullptr))
        return BP_OK;
    if (h == nullptr || in == nullptr || g == nullptr) {
        set_thread_error("bp_row_filter_bwd: NULL pointer");
        return BP_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t smem = sizeof(float) * 2 * kRowsPerBlock * (size_t)(isx + 2 * T);
    if (smem > 48 * 1024)
        BP_CK(cudaFuncSetAttribute(row_filter_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long nblk = (rows + kRowsPerBlock - 1) / kRowsPerBlock;
    if (nblk > 0x7fffffffLL) {
        set_thread_error("bp_row_filter_bwd: too many rows");
        return BP_EINVAL;
    }
    float *partial = nullptr;
    if (gh != nullptr)
        BP_CK(cudaMallocAsync((void **)&partial, sizeof(float) * (size_t)nblk * T, s));
    row_filter_bwd_kernel<<<(unsigned)nblk, 256, smem, s>>>(rows, isx, T, h, in, g, gin, partial);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && gh != nullptr) {
        reduce_taps_kernel<<<T, 256, 0, s>>>(nblk, T, partial, gh);
        e = cudaGetLastError();
    }
    cudaError_t e2 = partial ? cudaFreeAsync(partial, s) : cudaSuccess;
    BP_CK(e);
    BP_CK(e2);
    return BP_OK;
}
