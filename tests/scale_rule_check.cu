// Host-side check of the float16 storage scale rule (proj_scale_k, pow2f in
// the library's internal header): for maxima across the whole float range,
// the scaled maximum max * 2^(-2k) lies in [2^12, 2^14) unless k is clamped
// at +-63, and zero, infinite and NaN maxima take k = 0.  Prints one line per
// failure and "ok <cases>" at the end; exit status 1 on any failure.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "../paper_1104_5243_gb300/csrc/bp_internal.cuh"

static unsigned bits(float f)
{
    unsigned u;
    std::memcpy(&u, &f, sizeof u);
    return u;
}

int main()
{
    int bad = 0, cases = 0;
    // every float exponent, a few mantissas each, plus subnormals
    for (int e = -149; e <= 127; ++e) {
        for (double m : {1.0, 1.2345, 1.5, 1.999999}) {
            const float mx = (float)std::ldexp(m, e);
            if (!(mx > 0.f) || std::isinf(mx))
                continue;
            ++cases;
            const int k = bp::proj_scale_k(bits(mx));
            const double scaled = std::ldexp((double)mx, -2 * k);
            const bool clamped = k == 63 || k == -63;
            if (!clamped && !(scaled >= 4096.0 && scaled < 16384.0)) {
                std::printf("max %.9g: k %d, scaled %.9g\n", mx, k, scaled);
                ++bad;
            }
            if (clamped && ((k == 63 && scaled >= 16384.0 && e < 127) || (k == -63 && scaled < 4096.0 && e > -114))) {
                std::printf("max %.9g: clamped k %d too early, scaled %.9g\n", mx, k, scaled);
                ++bad;
            }
            // pow2f is exact for the factors the kernels use
            if ((double)bp::pow2f(-2 * k) != std::ldexp(1.0, -2 * k) || (double)bp::pow2f(2 * k) != std::ldexp(1.0, 2 * k)) {
                std::printf("pow2f(%d) inexact\n", 2 * k);
                ++bad;
            }
        }
    }
    const float specials[] = {0.f, INFINITY, NAN};
    for (float f : specials) {
        ++cases;
        const float a = std::fabs(f);
        if (bp::proj_scale_k(bits(a)) != 0) {
            std::printf("special %g: k %d\n", (double)f, bp::proj_scale_k(bits(a)));
            ++bad;
        }
    }
    if (bad)
        return 1;
    std::printf("ok %d\n", cases);
    return 0;
}
