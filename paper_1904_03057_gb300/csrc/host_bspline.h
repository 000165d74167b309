// host_bspline.h -- host-side B-spline values and Gauss rules for the tables the kernels take
// (variable-coefficient quadrature tables, Robin boundary rows, transfer matrices).
#pragma once

#include <cmath>

namespace bsk {
namespace host {

// Centred B-spline beta^n(x) from its truncated-power form
// beta^n(x) = (1/n!) sum_k (-1)^k C(n+1, k) (x + (n+1)/2 - k)_+^n (Table tblBsplines).
inline double bspline(int n, double x)
{
    if (n == 0) return (x >= -0.5 && x < 0.5) ? 1.0 : 0.0;
    double s = 0.0, binom = 1.0, fact = 1.0;
    for (int i = 2; i <= n; i++) fact *= i;
    for (int k = 0; k <= n + 1; k++) {
        const double t = x + 0.5 * (n + 1) - k;
        if (t > 0.0) s += ((k & 1) ? -binom : binom) * std::pow(t, n);
        binom = binom * (n + 1 - k) / (k + 1);
    }
    return s / fact;
}

// beta^n'(x) = beta^{n-1}(x + 1/2) - beta^{n-1}(x - 1/2) (Table tblBsplines, derivative row).
inline double bspline_deriv(int n, double x)
{
    return bspline(n - 1, x + 0.5) - bspline(n - 1, x - 0.5);
}

// Gauss-Legendre rule of q points on [0, 1]: Newton iteration on the three-term recurrence of
// the Legendre polynomials, weights 2 / ((1 - x^2) P_q'(x)^2), mapped from [-1, 1].
inline void gauss_unit(int q, double* xi, double* w)
{
    const double pi = 3.14159265358979323846;
    auto legendre = [q](double x, double& p1, double& p0) {
        p0 = 1.0;
        p1 = x;
        for (int k = 2; k <= q; k++) {
            const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
    };
    for (int i = 0; i < q; i++) {
        double x = std::cos(pi * (i + 0.75) / (q + 0.5)), p1, p0;
        for (int it = 0; it < 100; it++) {
            legendre(x, p1, p0);
            const double dp = q * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        legendre(x, p1, p0);
        const double dp = q * (x * p1 - p0) / (x * x - 1.0);
        xi[i] = 0.5 * (1.0 - x);
        w[i] = 1.0 / ((1.0 - x * x) * dp * dp);
    }
}

// integral over [a, b] of f, by q-point Gauss-Legendre on each of the unit-length pieces
// [a + k s, a + (k + 1) s] with s = (b - a) / pieces.
template <typename F>
inline double integrate(double a, double b, int pieces, int q, F f)
{
    double xi[16], w[16];
    gauss_unit(q, xi, w);
    const double s = (b - a) / pieces;
    double acc = 0.0;
    for (int k = 0; k < pieces; k++)
        for (int g = 0; g < q; g++) acc += s * w[g] * f(a + s * (k + xi[g]));
    return acc;
}

}  // namespace host
}  // namespace bsk
