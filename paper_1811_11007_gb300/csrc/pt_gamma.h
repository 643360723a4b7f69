// Discrete Gamma rate categories, shared by the host model set-up and the
// device kernel that re-derives them when a visit re-optimises the shape.
#pragma once

#include <cmath>

#include "pt_internal.h"

#ifdef __CUDACC__
#define PT_HD __host__ __device__
#else
#define PT_HD
#endif

namespace pt {

// Regularised lower incomplete gamma P(a, x): series for x < a + 1, else
// 1 - Q(a, x) with Q as a continued fraction (modified Lentz).
PT_HD inline double inc_gamma_p(double a, double x) {
    if (x <= 0) return 0.0;
    const double lead = exp(a * log(x) - x - lgamma(a));
    if (x < a + 1.0) {
        double sum = 1.0 / a, term = sum;
        for (int k = 1; k < 10000; ++k) {
            term *= x / (a + k);
            sum += term;
            if (term < sum * 1e-17) break;
        }
        return sum * lead;
    }
    double f = x + 1.0 - a;
    if (fabs(f) < 1e-300) f = 1e-300;
    double Cc = f, D = 0.0;
    for (int k = 1; k < 10000; ++k) {
        double an = k * (a - k), bn = x + 2.0 * k + 1.0 - a;
        D = bn + an * D;
        if (fabs(D) < 1e-300) D = 1e-300;
        Cc = bn + an / Cc;
        if (fabs(Cc) < 1e-300) Cc = 1e-300;
        D = 1.0 / D;
        double delta = Cc * D;
        f *= delta;
        if (fabs(delta - 1.0) < 1e-16) break;
    }
    return 1.0 - lead / f;
}

// y with P(a, y) = q: Newton on P (derivative = Gamma(a) density), kept in a
// shrinking bracket, bisection when a step leaves it.
PT_HD inline double inc_gamma_inv(double a, double q) {
    double lo = 0.0, hi = a > 1.0 ? a : 1.0;
    for (int k = 0; k < 2000 && inc_gamma_p(a, hi) < q; ++k) hi *= 2.0;
    double y = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        double f = inc_gamma_p(a, y) - q;
        if (f < 0) lo = y; else hi = y;
        double dens = exp((a - 1.0) * log(y) - y - lgamma(a));
        double yn = y - f / dens;
        if (!(yn > lo && yn < hi)) yn = 0.5 * (lo + hi);
        if (fabs(yn - y) <= 1e-15 * y || hi - lo <= 1e-300) { y = yn; break; }
        y = yn;
    }
    return y;
}

// Mean rate of each of C equal-probability categories of Gamma(alpha, rate alpha).
PT_HD inline bool discrete_gamma(double alpha, int C, double* rates) {
    if (C == 1) { rates[0] = 1.0; return true; }
    if (!(alpha > 0.0) || C < 1 || C > kMaxCat) return false;
    double prev = 0.0, tot = 0.0;
    for (int k = 0; k < C; ++k) {
        double cum = 1.0;
        if (k + 1 < C) {
            double b = inc_gamma_inv(alpha, (double)(k + 1) / C) / alpha;  // category bound on the rate scale
            cum = inc_gamma_p(alpha + 1.0, alpha * b);
        }
        rates[k] = (cum - prev) * C;
        prev = cum;
        tot += rates[k];
    }
    for (int k = 0; k < C; ++k) rates[k] *= C / tot;
    return true;
}

}  // namespace pt
