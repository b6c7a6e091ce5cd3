// Rational approximation of A^-1/2 for the non-degenerate doublet (Sec. 4.2's
// rational monomials and their correction term, Fig. 4), host side, and the
// FP64 linear combination of fields its application needs.
//
// Coefficients.  The best relative approximation of type (n, n) to x^-1/2 on
// [eps, 1] (Zolotarev) has its poles and zeros at x = -eps c_{2l-1} and
// x = -eps c_{2l}, c_j = sn^2(j K / (2n+1); k) / (1 - sn^2(j K / (2n+1); k)),
// k = sqrt(1 - eps), K = K(k); sn and K come from the arithmetic-geometric mean
// (Abramowitz and Stegun 16.4).  The constant factor centres the relative error
// sqrt(x) r(x) - 1 about zero (equioscillation), found on a logarithmic grid of
// 200001 points; [lo, hi] maps to [eps, 1] with eps = lo / hi.
#include <cmath>
#include <vector>

#include "rational.h"

namespace tmk {

// sn(u | k) by the arithmetic-geometric mean (A&S 16.4.3)
static double agm_sn(double u, double k) {
    std::vector<double> a{1.0}, c{k};
    double b = std::sqrt(1.0 - k * k);
    while (std::fabs(c.back()) > 1e-18 && a.size() < 80) {
        const double an = 0.5 * (a.back() + b);
        c.push_back(0.5 * (a.back() - b));
        b = std::sqrt(a.back() * b);
        a.push_back(an);
    }
    const int n = (int)a.size() - 1;
    double phi = std::ldexp(a[n] * u, n);
    for (int i = n; i > 0; --i) phi = 0.5 * (phi + std::asin(c[i] / a[i] * std::sin(phi)));
    return std::sin(phi);
}

// complete elliptic integral K(k) = pi / (2 AGM(1, sqrt(1 - k^2)))
static double ellip_k(double k) {
    double a = 1.0, b = std::sqrt(1.0 - k * k);
    for (int i = 0; i < 80 && std::fabs(a - b) > 1e-17 * a; ++i) {
        const double an = 0.5 * (a + b);
        b = std::sqrt(a * b);
        a = an;
    }
    return M_PI / (2.0 * a);
}

bool zolotarev_inv_sqrt(int n, double lo, double hi, double* a0, double* a, double* sigma, double* delta) {
    if (n < 1 || !(lo > 0.0) || !(hi > lo)) return false;
    const double eps = lo / hi;
    const double k = std::sqrt(1.0 - eps);
    const double K = ellip_k(k);
    std::vector<double> p(n), z(n);
    for (int j = 1; j <= 2 * n; ++j) {
        const double s = agm_sn(j * K / (2 * n + 1), k);
        const double cj = eps * s * s / (1.0 - s * s);
        if (j % 2) p[(j - 1) / 2] = cj;   // poles at -c_{2l-1}
        else z[j / 2 - 1] = cj;           // zeros at -c_{2l}
    }
    const int grid = 200001;
    double gmax = -1.0, gmin = 1e300;
    const double l0 = std::log(eps);
    for (int i = 0; i < grid; ++i) {
        const double x = std::exp(l0 + (0.0 - l0) * i / (grid - 1));
        double g = std::sqrt(x);
        for (int l = 0; l < n; ++l) g *= (x + z[l]) / (x + p[l]);
        gmax = std::max(gmax, g);
        gmin = std::min(gmin, g);
    }
    const double d = 2.0 / (gmax + gmin);
    *delta = (gmax - gmin) / (gmax + gmin);
    // residues of d prod (x + z) / (x + p) at x = -p_l, then [eps, 1] -> [lo, hi]
    const double s = 1.0 / std::sqrt(hi);
    for (int l = 0; l < n; ++l) {
        double num = 1.0, den = 1.0;
        for (int m = 0; m < n; ++m) {
            num *= z[m] - p[l];
            if (m != l) den *= p[m] - p[l];
        }
        a[l] = d * num / den * hi * s;
        sigma[l] = p[l] * hi;
    }
    *a0 = d * s;
    return true;
}

__global__ void k_lincomb64(const __grid_constant__ LinComb p) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < p.len; i += (long)gridDim.x * blockDim.x) {
        const double2 bv = p.b[i];
        double re = p.a0 * bv.x, im = p.a0 * bv.y;
        for (int k = 0; k < p.n; ++k) {
            const double2 v = p.x[k][i];
            re = fma(p.a[k], v.x, re);
            im = fma(p.a[k], v.y, im);
        }
        p.y[i] = make_double2(re, im);
    }
}

cudaError_t launch_lincomb64(const LinComb& p, cudaStream_t st) {
    if (p.len <= 0) return cudaSuccess;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long want = (p.len + 255) / 256;
    const long cap = (long)nsm * 8;
    k_lincomb64<<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace tmk
