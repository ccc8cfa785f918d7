// Float64 instantiations of the direct backprojection and direct adjoint
// kernels (bp_direct.cuh), for gradient checks only (include/bp1104_f64.h).
// Built into libbp1104_f64.so, separate from the product library.
#include <cmath>
#include <cstdarg>
#include <cstdio>

#include "../bp_direct.cuh"
#include "../../../include/bp1104_f64.h"

namespace {

thread_local char g_err[512] = "no error";

bp_status f64_fail(bp_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

bool bad_args(int L, double R, const double *O, int isx, int isy, int n, const double *A)
{
    return L < 1 || L > 1024 || !(R > 0) || O == nullptr || isx < 1 || isy < 1 || isx > 32768 || isy > 32768 ||
           n < 0 || (n > 0 && A == nullptr);
}

// Rows of A_i centred on the integer offsets (ku, kv), the pixel the volume
// centre projects to: u' = u - ku (float64 throughout).
template <typename Batch>
void centred_rows(Batch &b, const double *A, int c0, int m, int L, double R, const double *O)
{
    const double h = 0.5 * (L - 1) * R;
    const double X = O[0] + h, Y = O[1] + h, Z = O[2] + h;
    for (int j = 0; j < m; ++j) {
        const double *a = A + 12 * (size_t)(c0 + j);
        const double w = a[8] * X + a[9] * Y + a[10] * Z + a[11];
        const double ku = std::nearbyint((a[0] * X + a[1] * Y + a[2] * Z + a[3]) / w);
        const double kv = std::nearbyint((a[4] * X + a[5] * Y + a[6] * Z + a[7]) / w);
        b.m[j][0] = bp::Dbl4{a[0] - ku * a[8], a[1] - ku * a[9], a[2] - ku * a[10], a[3] - ku * a[11]};
        b.m[j][1] = bp::Dbl4{a[4] - kv * a[8], a[5] - kv * a[9], a[6] - kv * a[10], a[7] - kv * a[11]};
        b.m[j][2] = bp::Dbl4{a[8], a[9], a[10], a[11]};
        b.k[j] = make_int2((int)ku, (int)kv);
    }
}

bp::VolGeomT<double> geom(int L, double R, const double *O)
{
    bp::VolGeomT<double> g;
    g.L = L;
    g.Lz = L;
    g.R = R;
    g.Ox = O[0];
    g.Oy = O[1];
    g.Oz = O[2];
    g.z0 = 0;
    return g;
}

}  // namespace

extern "C" bp_status bp_f64_backproject(int L, double R, const double O[3], int isx, int isy, const double *images,
                                        const double *A, int n, double *vol, void *stream)
{
    if (bad_args(L, R, O, isx, isy, n, A) || (n > 0 && (images == nullptr || vol == nullptr)))
        return f64_fail(BP_EINVAL, "bp_f64_backproject: invalid argument");
    const auto g = geom(L, R, O);
    cudaStream_t s = (cudaStream_t)stream;
    for (int c0 = 0; c0 < n; c0 += bp::kMaxBatch) {
        const int m = n - c0 < bp::kMaxBatch ? n - c0 : bp::kMaxBatch;
        bp::DirectBatchT<double> b;
        b.n = m;
        centred_rows(b, A, c0, m, L, R, O);
        for (int j = 0; j < m; ++j)
            b.img_off[j] = (long long)(c0 + j) * isx * isy;
        dim3 grid((L + 255) / 256, L, L);
        bp::direct_backproject_kernel<double, true><<<grid, 256, 0, s>>>(b, images, vol, g, isx, isy);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return f64_fail(BP_ECUDA, "bp_f64_backproject: %s", cudaGetErrorString(e));
    }
    return BP_OK;
}

extern "C" bp_status bp_f64_adjoint(int L, double R, const double O[3], int isx, int isy, const double *vol,
                                    const double *A, int n, double *images, void *stream)
{
    if (bad_args(L, R, O, isx, isy, n, A) || (n > 0 && (images == nullptr || vol == nullptr)))
        return f64_fail(BP_EINVAL, "bp_f64_adjoint: invalid argument");
    const auto g = geom(L, R, O);
    cudaStream_t s = (cudaStream_t)stream;
    for (int c0 = 0; c0 < n; c0 += bp::kMaxBatch) {
        const int m = n - c0 < bp::kMaxBatch ? n - c0 : bp::kMaxBatch;
        bp::AdjBatchT<double> b;
        b.n = m;
        b.centres = nullptr;
        b.blocks = 0;
        centred_rows(b, A, c0, m, L, R, O);
        for (int j = 0; j < m; ++j)
            b.out_off[j] = (long long)(c0 + j) * isx * isy;
        constexpr int TX = 8 * bp::kVoxPerLane, LZ = 4;
        dim3 grid((L + TX - 1) / TX, (L + bp::kWarpsY - 1) / bp::kWarpsY, (L + LZ - 1) / LZ);
        bp::direct_adjoint_kernel<double, true><<<grid, bp::kThreads, 0, s>>>(b, vol, g, images, isx, isy);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return f64_fail(BP_ECUDA, "bp_f64_adjoint: %s", cudaGetErrorString(e));
    }
    return BP_OK;
}

extern "C" const char *bp_f64_last_error(void)
{
    return g_err;
}
