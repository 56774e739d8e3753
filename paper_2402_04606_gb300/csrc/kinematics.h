// Prescribed pitch angles of the paper's moving-body cases, shared by the host
// planner (api.cpp) and the kernels (kernels.cu).  Time is in finest steps
// unless stated otherwise.
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define SBOT_HD __host__ __device__
#else
#define SBOT_HD
#endif

namespace sbot_kin {

// log cosh x as |x| + log(1 + e^(-2|x|)) - log 2: the same value, no overflow
SBOT_HD inline double log_cosh(double x) {
    const double ax = fabs(x);
    return ax + log1p(exp(-2.0 * ax)) - 0.69314718055994530942;
}

// Sec. 3.4, Eqs. 20-21: the smoothed pitch-up ramp from 0 to A at
// nondimensional time ts = t U / c.  G = log[cosh(a_s (ts - t1)) /
// cosh(a_s (ts - t2))] - a_s (t1 - t2) with t2 = t1 + A / (2 K), normalised
// by its supremum 2 a_s (t2 - t1), the value G reaches after the ramp.
SBOT_HD inline double ramp_alpha(double A, double as, double K, double t1, double ts) {
    const double t2 = t1 + A / (2.0 * K);
    const double G = log_cosh(as * (ts - t1)) - log_cosh(as * (ts - t2)) + as * (t2 - t1);
    return A * G / (2.0 * as * (t2 - t1));
}

// Sec. 3.5, Eqs. 22-24: the smoothed asymmetric triangular pitch of
// amplitude a0 and period T.  The upstroke takes xi T and the downstroke
// (1 - xi) T; alpha rises through 0 at t = 0, peaks at xi T / 2, reaches -a0
// at T - xi T / 2.  Each corner is rounded by two quartic pieces of length
// t_a = acc T that join the linear strokes with matching slope and
// curvature; the linear rates are 2 a0 / (xi T - t_a) and
// -2 a0 / ((1 - xi) T - t_a).
SBOT_HD inline double triangle_alpha(double a0, double xi, double acc, double T, double t) {
    const double tt = t - T * floor(t / T);
    const double ta = acc * T, ta2 = ta * ta, ta3 = ta2 * ta;
    const double up = 2.0 * a0 / (xi * T - ta);
    const double dn = -2.0 * a0 / ((1.0 - xi) * T - ta);
    const double tpk = 0.5 * xi * T, ttr = T - 0.5 * xi * T;  // peak, trough
    double u;
    if (tt < tpk - ta) return up * tt;
    if (tt < tpk) {
        u = tt - tpk;
        return a0 + u * u * u * (up / ta2 + u * up / (2.0 * ta3));
    }
    if (tt < tpk + ta) {
        u = tt - tpk;
        return a0 + u * u * u * (dn / ta2 - u * dn / (2.0 * ta3));
    }
    if (tt < ttr - ta) return dn * (tt - ttr + ta) - 0.5 * dn * ta - a0;
    if (tt < ttr) {
        u = tt - ttr;
        return -a0 + u * u * u * (dn / ta2 + u * dn / (2.0 * ta3));
    }
    if (tt < ttr + ta) {
        u = tt - ttr;
        return -a0 + u * u * u * (up / ta2 - u * up / (2.0 * ta3));
    }
    return up * (tt - T);
}

}  // namespace sbot_kin
