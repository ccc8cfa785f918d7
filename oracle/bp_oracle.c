/*
 * CPU oracle for the voxel-driven cone-beam backprojection -- TEST
 * INFRASTRUCTURE ONLY.  Plain, slow, obviously correct FP64 code.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark load
 * it; the product library never does.  It shares no code with the CUDA path.
 *
 * What it computes (Treibig et al., "Pushing the limits for medical image
 * reconstruction on recent standard multicore processors"):
 *
 *   backprojection (Sect. 3.1, Listing 1): for every voxel x and projection i
 *     (uw, vw, w) = A_i (x, 1),  u = uw / w,  v = vw / w
 *     fx = bilinear sample of image i at (u, v), zero outside the detector
 *     VOL[x] += fx / w^2
 *
 * Readings of the listing (the paper is silent or garbled there):
 *   - the integer part of u, v is floor(), not truncation toward zero, and a
 *     corner pixel outside [0,ISX) x [0,ISY) reads 0 (the zero-padded image
 *     buffers of Sect. 3.3);
 *   - the four corner values are reset for every voxel;
 *   - the update statement is VOL[z*L*L + y*L + x] += fx / (w*w);
 *   - matrices are given row-major here: A[r*4 + c], rows (uw, vw, w);
 *   - a voxel with w <= 0 (behind the source) contributes nothing.
 *
 * Every routine is FP64 and deterministic: each voxel sums its projections in
 * index order, and OpenMP splits only over independent outputs (z slices with
 * schedule(static,1), the paper's Sect. 6 scheme, or whole images).
 *
 * Parity pins for each routine live in tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Pixel (j, k) of one image, zero outside the detector (Sect. 3.3). */
static double pix(const float *img, int isx, int isy, long long j, long long k)
{
    if (j < 0 || j >= isx || k < 0 || k >= isy)
        return 0.0;
    return (double)img[k * (long long)isx + j];
}

/* Bilinear sample at (u, v) with the listing's corner naming:
 * tl = (iu, iv), tr = (iu+1, iv), bl = (iu, iv+1), br = (iu+1, iv+1). */
static double bilinear(const float *img, int isx, int isy, double u, double v)
{
    /* Far outside the detector every corner is zero; this also keeps the
     * integer conversion below in range. */
    if (!(u > -2.0 && u < isx + 1.0 && v > -2.0 && v < isy + 1.0))
        return 0.0;
    double fu0 = floor(u), fv0 = floor(v);
    long long iu = (long long)fu0, iv = (long long)fv0;
    double scalx = u - fu0, scaly = v - fv0;
    double valtl = pix(img, isx, isy, iu, iv);
    double valtr = pix(img, isx, isy, iu + 1, iv);
    double valbl = pix(img, isx, isy, iu, iv + 1);
    double valbr = pix(img, isx, isy, iu + 1, iv + 1);
    double vall = scaly * valbl + (1.0 - scaly) * valtl;
    double valr = scaly * valbr + (1.0 - scaly) * valtr;
    return scalx * valr + (1.0 - scalx) * vall;
}

/* ------------------------------------------------------------------------ */
/* Geometry: C-arm circular scan about z (the workloads' acquisition).
 *
 * Source at S = sid (cos b, sin b, 0); central ray direction d = -(cos b,
 * sin b, 0); detector plane at distance sdd from the source, perpendicular to
 * d, with u axis e_u = (-sin b, cos b, 0) and v axis e_v = (0, 0, 1); pixel
 * (j, k) sits at detector coordinates ((j - cu) p, (k - cv) p).  The matrix is
 * scaled so that w = depth / sid (w = 1 at the isocenter).                  */
void orc_carm_matrices(int n, const double *beta, double sid, double sdd,
                       double pitch, double cu, double cv, double *A)
{
    for (int i = 0; i < n; ++i) {
        double c = cos(beta[i]), s = sin(beta[i]);
        double *a = A + 12 * (long long)i;
        double g = sdd / (pitch * sid);
        /* w row: (d . X + sid) / sid */
        double w0 = -c / sid, w1 = -s / sid, w2 = 0.0, w3 = 1.0;
        /* uw row: g (e_u . X) + cu w ;  vw row: g (e_v . X) + cv w */
        a[0] = g * (-s) + cu * w0; a[1] = g * c + cu * w1; a[2] = cu * w2; a[3] = cu * w3;
        a[4] = cv * w0;            a[5] = cv * w1;         a[6] = g + cv * w2; a[7] = cv * w3;
        a[8] = w0;                 a[9] = w1;              a[10] = w2;        a[11] = w3;
    }
}

/* ------------------------------------------------------------------------ */
/* Backprojection, the plain definition (Sect. 3.1, Listing 1).
 * vol: L^3 doubles, index z*L*L + y*L + x, ACCUMULATED into.
 * images: n x isy x isx float32, row-major.  A: n x 12 row-major.          */
void orc_backproject(int L, double R, const double *O, int isx, int isy,
                     int n, const float *images, const double *A, double *vol)
{
    for (int i = 0; i < n; ++i) {
        const float *img = images + (long long)i * isx * isy;
        const double *a = A + 12 * (long long)i;
        #pragma omp parallel for schedule(static, 1)
        for (int z = 0; z < L; ++z) {
            double wz = O[2] + R * z;
            for (int y = 0; y < L; ++y) {
                double wy = O[1] + R * y;
                for (int x = 0; x < L; ++x) {
                    double wx = O[0] + R * x;
                    double uw = a[0] * wx + a[1] * wy + a[2] * wz + a[3];
                    double vw = a[4] * wx + a[5] * wy + a[6] * wz + a[7];
                    double w = a[8] * wx + a[9] * wy + a[10] * wz + a[11];
                    if (w <= 0.0)
                        continue;
                    double fx = bilinear(img, isx, isy, uw / w, vw / w);
                    vol[((long long)z * L + y) * L + x] += fx / (w * w);
                }
            }
        }
    }
}

/* Same sum for a list of voxels only (idx = z*L*L + y*L + x); out[m] is SET.
 * Used to check full-size volumes on sampled voxels.                       */
void orc_backproject_voxels(int L, double R, const double *O, int isx, int isy,
                            int n, const float *images, const double *A,
                            long long m, const long long *idx, double *out)
{
    #pragma omp parallel for schedule(static, 1)
    for (long long t = 0; t < m; ++t) {
        long long q = idx[t];
        int x = (int)(q % L), y = (int)((q / L) % L), z = (int)(q / ((long long)L * L));
        double wx = O[0] + R * x, wy = O[1] + R * y, wz = O[2] + R * z;
        double acc = 0.0;
        for (int i = 0; i < n; ++i) {
            const double *a = A + 12 * (long long)i;
            double uw = a[0] * wx + a[1] * wy + a[2] * wz + a[3];
            double vw = a[4] * wx + a[5] * wy + a[6] * wz + a[7];
            double w = a[8] * wx + a[9] * wy + a[10] * wz + a[11];
            if (w <= 0.0)
                continue;
            acc += bilinear(images + (long long)i * isx * isy, isx, isy, uw / w, vw / w) / (w * w);
        }
        out[t] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the backprojection (the transpose of the linear map above):
 * every voxel value f scaled by 1/w^2 is spread onto the four corner pixels
 * with the bilinear weights; corners outside the detector are dropped.
 * images_out: n x isy x isx doubles, ACCUMULATED into.  Parallel over images,
 * each image sums its voxels in index order.                               */
void orc_adjoint(int L, double R, const double *O, int isx, int isy, int n,
                 const double *vol, const double *A, double *images_out)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n; ++i) {
        double *img = images_out + (long long)i * isx * isy;
        const double *a = A + 12 * (long long)i;
        for (int z = 0; z < L; ++z) {
            double wz = O[2] + R * z;
            for (int y = 0; y < L; ++y) {
                double wy = O[1] + R * y;
                for (int x = 0; x < L; ++x) {
                    double wx = O[0] + R * x;
                    double uw = a[0] * wx + a[1] * wy + a[2] * wz + a[3];
                    double vw = a[4] * wx + a[5] * wy + a[6] * wz + a[7];
                    double w = a[8] * wx + a[9] * wy + a[10] * wz + a[11];
                    if (w <= 0.0)
                        continue;
                    double u = uw / w, v = vw / w;
                    if (!(u > -2.0 && u < isx + 1.0 && v > -2.0 && v < isy + 1.0))
                        continue;
                    double s = vol[((long long)z * L + y) * L + x] / (w * w);
                    double fu0 = floor(u), fv0 = floor(v);
                    long long iu = (long long)fu0, iv = (long long)fv0;
                    double fu = u - fu0, fv = v - fv0;
                    double wt[4] = {(1.0 - fu) * (1.0 - fv), fu * (1.0 - fv), (1.0 - fu) * fv, fu * fv};
                    long long ju[4] = {iu, iu + 1, iu, iu + 1};
                    long long kv[4] = {iv, iv, iv + 1, iv + 1};
                    for (int c = 0; c < 4; ++c)
                        if (ju[c] >= 0 && ju[c] < isx && kv[c] >= 0 && kv[c] < isy)
                            img[kv[c] * isx + ju[c]] += s * wt[c];
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Source position and ray directions from a projection matrix: with
 * A = [M | a], the source S solves M S = -a and the ray through pixel (u, v)
 * has direction M^{-1} (u, v, 1).  3x3 inverse by cofactors, FP64.          */
static int inv3(const double *A, double *Mi)
{
    double m00 = A[0], m01 = A[1], m02 = A[2];
    double m10 = A[4], m11 = A[5], m12 = A[6];
    double m20 = A[8], m21 = A[9], m22 = A[10];
    double c00 = m11 * m22 - m12 * m21, c01 = m12 * m20 - m10 * m22, c02 = m10 * m21 - m11 * m20;
    double det = m00 * c00 + m01 * c01 + m02 * c02;
    if (det == 0.0)
        return -1;
    double id = 1.0 / det;
    Mi[0] = c00 * id; Mi[1] = (m02 * m21 - m01 * m22) * id; Mi[2] = (m01 * m12 - m02 * m11) * id;
    Mi[3] = c01 * id; Mi[4] = (m00 * m22 - m02 * m20) * id; Mi[5] = (m02 * m10 - m00 * m12) * id;
    Mi[6] = c02 * id; Mi[7] = (m01 * m20 - m00 * m21) * id; Mi[8] = (m00 * m11 - m01 * m10) * id;
    return 0;
}

void orc_source_position(int n, const double *A, double *S)
{
    for (int i = 0; i < n; ++i) {
        const double *a = A + 12 * (long long)i;
        double Mi[9];
        inv3(a, Mi);
        for (int r = 0; r < 3; ++r)
            S[3 * i + r] = -(Mi[3 * r] * a[3] + Mi[3 * r + 1] * a[7] + Mi[3 * r + 2] * a[11]);
    }
}

/* Chord length of the line S + t d (|d| = 1) through one ellipsoid
 * (centre c, semi-axes ax, rotation Q whose columns are the axes).         */
static double chord(const double *S, const double *d, const double *e)
{
    const double *c = e, *ax = e + 3, *Q = e + 6;
    double p[3] = {S[0] - c[0], S[1] - c[1], S[2] - c[2]};
    double s0[3], sd[3];
    for (int k = 0; k < 3; ++k) {   /* Q^T p / a_k and Q^T d / a_k */
        s0[k] = (Q[k] * p[0] + Q[3 + k] * p[1] + Q[6 + k] * p[2]) / ax[k];
        sd[k] = (Q[k] * d[0] + Q[3 + k] * d[1] + Q[6 + k] * d[2]) / ax[k];
    }
    double qa = sd[0] * sd[0] + sd[1] * sd[1] + sd[2] * sd[2];
    double qb = s0[0] * sd[0] + s0[1] * sd[1] + s0[2] * sd[2];
    double qc = s0[0] * s0[0] + s0[1] * s0[1] + s0[2] * s0[2] - 1.0;
    double disc = qb * qb - qa * qc;
    if (disc <= 0.0)
        return 0.0;
    return 2.0 * sqrt(disc) / qa;
}

/* Analytic line integrals of an ellipsoid phantom (additive densities):
 * out[i][k][j] = sum_e rho_e * chord_e(ray through pixel (j, k)), SET.
 * ell: count x 16 (centre, semi-axes, row-major rotation, density).       */
void orc_ellipsoid_project(int n, const double *A, int isx, int isy,
                           int count, const double *ell, double *out)
{
    for (int i = 0; i < n; ++i) {
        const double *a = A + 12 * (long long)i;
        double Mi[9], S[3];
        inv3(a, Mi);
        for (int r = 0; r < 3; ++r)
            S[r] = -(Mi[3 * r] * a[3] + Mi[3 * r + 1] * a[7] + Mi[3 * r + 2] * a[11]);
        #pragma omp parallel for schedule(static, 1)
        for (int k = 0; k < isy; ++k) {
            for (int j = 0; j < isx; ++j) {
                double d[3];
                for (int r = 0; r < 3; ++r)
                    d[r] = Mi[3 * r] * j + Mi[3 * r + 1] * k + Mi[3 * r + 2];
                double nd = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                d[0] /= nd; d[1] /= nd; d[2] /= nd;
                double acc = 0.0;
                for (int e = 0; e < count; ++e)
                    acc += ell[16 * e + 15] * chord(S, d, ell + 16 * e);
                out[((long long)i * isy + k) * isx + j] = acc;
            }
        }
    }
}

/* Phantom density at every voxel centre (point sampling), SET.            */
void orc_ellipsoid_voxelize(int L, double R, const double *O, int count,
                            const double *ell, double *vol)
{
    #pragma omp parallel for schedule(static, 1)
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                double X[3] = {O[0] + R * x, O[1] + R * y, O[2] + R * z};
                double acc = 0.0;
                for (int e = 0; e < count; ++e) {
                    const double *c = ell + 16 * e, *ax = c + 3, *Q = c + 6;
                    double p[3] = {X[0] - c[0], X[1] - c[1], X[2] - c[2]};
                    double r2 = 0.0;
                    for (int k = 0; k < 3; ++k) {
                        double t = (Q[k] * p[0] + Q[3 + k] * p[1] + Q[6 + k] * p[2]) / ax[k];
                        r2 += t * t;
                    }
                    if (r2 <= 1.0)
                        acc += c[15];
                }
                vol[((long long)z * L + y) * L + x] = acc;
            }
}

/* ------------------------------------------------------------------------ */
/* FDK 2-D preprocessing (Sect. 1.1 names it; the paper gives no formulas,
 * these follow the standard Feldkamp weighting for a flat detector).
 *
 * Pre-weight (SET into out): cosine weight sdd / sqrt(sdd^2 + ut^2 + vt^2)
 * with ut = (j - cu) p, vt = (k - cv) p, times the Parker short-scan weight
 * of the ray (scan angle b = beta_i - beta_0, fan angle g = atan(ut / sdd),
 * half over-scan delta), times scale.  parker = 0 turns the Parker factor
 * off.  With this geometry the conjugate of ray (b, g) is (b + pi - 2g, -g). */
static double parker_weight(double b, double g, double delta)
{
    double gs = -g;   /* textbook form has conjugate (b + pi + 2 gs, -gs) */
    if (b < 0.0 || b > M_PI + 2.0 * delta)
        return 0.0;
    if (b < 2.0 * (delta - gs)) {
        double t = sin(M_PI / 4.0 * b / (delta - gs));
        return t * t;
    }
    if (b <= M_PI - 2.0 * gs)
        return 1.0;
    double t = sin(M_PI / 4.0 * (M_PI + 2.0 * delta - b) / (delta + gs));
    return t * t;
}

double orc_parker(double b, double g, double delta)
{
    return parker_weight(b, g, delta);
}

void orc_fdk_preweight(int n, int isx, int isy, double pitch, double sdd,
                       double cu, double cv, const double *beta, int parker,
                       double scale, const double *in, double *out)
{
    double delta = n > 1 ? 0.5 * (fabs(beta[n - 1] - beta[0]) - M_PI) : 0.0;
    for (int i = 0; i < n; ++i) {
        double b = fabs(beta[i] - beta[0]);
        for (int k = 0; k < isy; ++k)
            for (int j = 0; j < isx; ++j) {
                double ut = (j - cu) * pitch, vt = (k - cv) * pitch;
                double wgt = scale * sdd / sqrt(sdd * sdd + ut * ut + vt * vt);
                if (parker)
                    wgt *= parker_weight(b, atan(ut / sdd), delta);
                long long q = ((long long)i * isy + k) * isx + j;
                out[q] = wgt * in[q];
            }
    }
}

/* Ram-Lak ramp kernel sampled at integer offsets with spacing tau:
 * h(0) = 1/(4 tau^2), h(odd m) = -1/(m^2 pi^2 tau^2), h(even m != 0) = 0.   */
double orc_ramlak(long long m, double tau)
{
    if (m == 0)
        return 1.0 / (4.0 * tau * tau);
    if (m % 2 == 0)
        return 0.0;
    return -1.0 / ((double)m * (double)m * M_PI * M_PI * tau * tau);
}

/* Row-wise linear (zero-padded) convolution with the Ram-Lak kernel:
 * out[r][j] = tau * sum_j' h(j - j') in[r][j'], SET.  rows = n * isy.      */
void orc_ramp_filter(long long rows, int isx, double tau, const double *in, double *out)
{
    #pragma omp parallel for schedule(static, 1)
    for (long long r = 0; r < rows; ++r) {
        const double *x = in + r * isx;
        double *q = out + r * isx;
        for (int j = 0; j < isx; ++j) {
            double acc = 0.0;
            for (int jp = 0; jp < isx; ++jp)
                acc += orc_ramlak(j - jp, tau) * x[jp];
            q[j] = tau * acc;
        }
    }
}

/* Short per-row filter with T taps (the learned filter):
 * out[r][j] = sum_t h[t] in[r][j + t - T/2], zero outside the row, SET.    */
void orc_row_filter_fwd(long long rows, int isx, int T, const double *h,
                        const double *in, double *out)
{
    #pragma omp parallel for schedule(static, 1)
    for (long long r = 0; r < rows; ++r)
        for (int j = 0; j < isx; ++j) {
            double acc = 0.0;
            for (int t = 0; t < T; ++t) {
                long long s = (long long)j + t - T / 2;
                if (s >= 0 && s < isx)
                    acc += h[t] * in[r * isx + s];
            }
            out[r * isx + j] = acc;
        }
}

/* Gradients of the row filter given dL/dout (g):
 * gin[r][s] = sum_t h[t] g[r][s - t + T/2] (SET);
 * gh[t] = sum_{r,j} g[r][j] in[r][j + t - T/2] (SET).                      */
void orc_row_filter_bwd(long long rows, int isx, int T, const double *h,
                        const double *in, const double *g, double *gin, double *gh)
{
    #pragma omp parallel for schedule(static, 1)
    for (long long r = 0; r < rows; ++r)
        for (int s = 0; s < isx; ++s) {
            double acc = 0.0;
            for (int t = 0; t < T; ++t) {
                long long j = (long long)s - t + T / 2;
                if (j >= 0 && j < isx)
                    acc += h[t] * g[r * isx + j];
            }
            gin[r * isx + s] = acc;
        }
    #pragma omp parallel for schedule(static, 1)
    for (int t = 0; t < T; ++t) {
        double acc = 0.0;
        for (long long r = 0; r < rows; ++r)
            for (int j = 0; j < isx; ++j) {
                long long s = (long long)j + t - T / 2;
                if (s >= 0 && s < isx)
                    acc += g[r * isx + j] * in[r * isx + s];
            }
        gh[t] = acc;
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
