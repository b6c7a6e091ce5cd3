// Rational approximation of A^-1/2 for the non-degenerate doublet (Sec. 4.2's
// rational monomials and their correction term, Fig. 4), host side, and the
// FP64 linear combination of fields its application needs.
//
// Coefficients.  The best relative approximation of type (n, n) to x^-1/2 on
// [eps, 1] (Zolotarev) has its poles and zeros at x = -c_{2l-1} and x = -c_{2l},
//   c_j = eps sc^2(j K / (2n+1); k),  k = sqrt(1 - eps),  sc = sn / cn.
// sc is evaluated here through Jacobi theta functions of the nome
// q = exp(-pi K'/K) (DLMF 22.2.4-5):
//   sc(u; k) = [theta3(0) / theta4(0)] theta1(zeta) / theta2(zeta),
//   zeta = pi u / (2K),
// so c_j = eps [theta3(0) theta1(zeta_j) / (theta4(0) theta2(zeta_j))]^2 with
// zeta_j = pi j / (2 (2n+1)); the ratio avoids the cancellation of 1 - sn^2 near
// u = K.  K and K' are complete elliptic integrals (arithmetic-geometric mean).
// The constant factor centres the relative error sqrt(x) r(x) - 1 about zero
// (equioscillation): the extrema of g(x) = sqrt(x) prod (x + z) / (x + p) are the
// end points and the roots of d log g / d log x, bracketed on a logarithmic grid
// and refined by bisection.  delta is the resulting maximum relative error,
// close to 4 q^(2n+1) for the sizes used here.  [lo, hi] maps to [eps, 1] with
// eps = lo / hi.
#include <cmath>
#include <vector>

#include "rational.h"

namespace tmk {

// complete elliptic integral K of modulus k from its complement kc = sqrt(1 - k^2):
// K = pi / (2 AGM(1, kc))
static double ellip_k_from_kc(double kc) {
    double a = 1.0, b = kc;
    for (int i = 0; i < 100 && std::fabs(a - b) > 1e-17 * a; ++i) {
        const double an = 0.5 * (a + b);
        b = std::sqrt(a * b);
        a = an;
    }
    return M_PI / (2.0 * a);
}

// Jacobi theta functions theta_1 .. theta_4 (z, q), 0 <= q < 1 (DLMF 20.2.1-4),
// summed until the terms fall below 1e-18 of the leading one
struct Theta {
    double t1, t2, t3, t4;
};
static Theta theta(double z, double q) {
    Theta t{0.0, 0.0, 1.0, 1.0};
    for (int n = 0; n < 200; ++n) {
        const double e = (n + 0.5) * (n + 0.5);
        const double w = std::pow(q, e);
        const double sgn = (n & 1) ? -1.0 : 1.0;
        t.t1 += 2.0 * sgn * w * std::sin((2 * n + 1) * z);
        t.t2 += 2.0 * w * std::cos((2 * n + 1) * z);
        if (n >= 1) {
            const double v = std::pow(q, (double)n * n);
            t.t3 += 2.0 * v * std::cos(2.0 * n * z);
            t.t4 += 2.0 * sgn * v * std::cos(2.0 * n * z);
        }
        if (w < 1e-18) break;
    }
    return t;
}

bool zolotarev_inv_sqrt(int n, double lo, double hi, double* a0, double* a, double* sigma, double* delta) {
    if (n < 1 || !(lo > 0.0) || !(hi > lo)) return false;
    const double eps = lo / hi;
    const double K = ellip_k_from_kc(std::sqrt(eps));          // modulus k = sqrt(1 - eps)
    const double Kp = ellip_k_from_kc(std::sqrt(1.0 - eps));   // complementary modulus sqrt(eps)
    const double q = std::exp(-M_PI * Kp / K);
    const Theta t0 = theta(0.0, q);
    std::vector<double> p(n), z(n);
    for (int j = 1; j <= 2 * n; ++j) {
        const Theta tz = theta(M_PI * j / (2.0 * (2 * n + 1)), q);
        const double sc = t0.t3 * tz.t1 / (t0.t4 * tz.t2);
        const double cj = eps * sc * sc;
        if (j % 2) p[(j - 1) / 2] = cj;   // poles at -c_{2l-1}
        else z[j / 2 - 1] = cj;           // zeros at -c_{2l}
    }
    auto logg = [&](double x) {
        double v = 0.5 * std::log(x);
        for (int l = 0; l < n; ++l) v += std::log((x + z[l]) / (x + p[l]));
        return v;
    };
    auto dlogg = [&](double lx) {   // d log g / d log x
        const double x = std::exp(lx);
        double v = 0.5;
        for (int l = 0; l < n; ++l) v += x / (x + z[l]) - x / (x + p[l]);
        return v;
    };
    // extrema of g: both ends and every sign change of d log g / d log x
    std::vector<double> ext{std::log(eps), 0.0};
    const int grid = 8192;
    const double l0 = std::log(eps);
    double tprev = l0, hprev = dlogg(l0);
    for (int i = 1; i < grid; ++i) {
        const double tc = l0 * (1.0 - (double)i / (grid - 1));
        const double hc = dlogg(tc);
        if ((hprev < 0.0) != (hc < 0.0)) {
            double ta = tprev, tb = tc, ha = hprev;
            for (int it = 0; it < 100 && tb - ta > 1e-15; ++it) {
                const double tm = 0.5 * (ta + tb);
                const double hm = dlogg(tm);
                if ((hm < 0.0) == (ha < 0.0)) { ta = tm; ha = hm; } else tb = tm;
            }
            ext.push_back(0.5 * (ta + tb));
        }
        tprev = tc;
        hprev = hc;
    }
    double lmax = -1e300, lmin = 1e300;
    for (double te : ext) {
        const double v = logg(std::exp(te));
        lmax = std::max(lmax, v);
        lmin = std::min(lmin, v);
    }
    const double gmax = std::exp(lmax), gmin = std::exp(lmin);
    const double d = 2.0 / (gmax + gmin);
    *delta = std::tanh(0.5 * (lmax - lmin));   // (gmax - gmin) / (gmax + gmin)
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
