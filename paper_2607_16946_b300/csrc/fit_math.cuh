// The torus fit of one point from its six coefficients (Sec. 4.1, App. C),
// written once over a scalar type T: double for sdf_build, and Dual6 (a value
// with six partial derivatives) for the parameter backward, which needs the
// Jacobian of the packed torus record with respect to (a00, a01, a10, a11,
// a02, a20).
#pragma once

#include <cuda_runtime.h>

#include <cmath>

namespace ptsdf {

// |kappa| at or below this (coordinates are O(1)) is a zero curvature.
constexpr double kFlatKappa = 1e-8;

struct Dual6 {
    double v;
    double d[6];
};

__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ double val(const Dual6& x) { return x.v; }

__device__ __forceinline__ Dual6 dconst(double v) {
    Dual6 r;
    r.v = v;
#pragma unroll
    for (int k = 0; k < 6; ++k) r.d[k] = 0.0;
    return r;
}
__device__ __forceinline__ Dual6 operator+(const Dual6& a, const Dual6& b) {
    Dual6 r;
    r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < 6; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
}
__device__ __forceinline__ Dual6 operator-(const Dual6& a, const Dual6& b) {
    Dual6 r;
    r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < 6; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
}
__device__ __forceinline__ Dual6 operator-(const Dual6& a) {
    Dual6 r;
    r.v = -a.v;
#pragma unroll
    for (int k = 0; k < 6; ++k) r.d[k] = -a.d[k];
    return r;
}
__device__ __forceinline__ Dual6 operator*(const Dual6& a, const Dual6& b) {
    Dual6 r;
    r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < 6; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
__device__ __forceinline__ Dual6 operator/(const Dual6& a, const Dual6& b) {
    Dual6 r;
    r.v = a.v / b.v;
    const double ib = 1.0 / b.v;
#pragma unroll
    for (int k = 0; k < 6; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
}
__device__ __forceinline__ Dual6 operator+(const Dual6& a, double b) { return a + dconst(b); }
__device__ __forceinline__ Dual6 operator+(double a, const Dual6& b) { return dconst(a) + b; }
__device__ __forceinline__ Dual6 operator-(const Dual6& a, double b) { return a - dconst(b); }
__device__ __forceinline__ Dual6 operator-(double a, const Dual6& b) { return dconst(a) - b; }
__device__ __forceinline__ Dual6 operator*(const Dual6& a, double b) {
    Dual6 r;
    r.v = a.v * b;
#pragma unroll
    for (int k = 0; k < 6; ++k) r.d[k] = a.d[k] * b;
    return r;
}
__device__ __forceinline__ Dual6 operator*(double a, const Dual6& b) { return b * a; }
__device__ __forceinline__ Dual6 operator/(const Dual6& a, double b) { return a * (1.0 / b); }
__device__ __forceinline__ Dual6 operator/(double a, const Dual6& b) { return dconst(a) / b; }

__device__ __forceinline__ double fsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ Dual6 fsqrt(const Dual6& a) {
    Dual6 r;
    r.v = sqrt(a.v);
    const double s = r.v > 0.0 ? 0.5 / r.v : 0.0;   // d sqrt at 0 taken as 0
#pragma unroll
    for (int k = 0; k < 6; ++k) r.d[k] = a.d[k] * s;
    return r;
}
__device__ __forceinline__ double fabsT(double x) { return fabs(x); }
__device__ __forceinline__ Dual6 fabsT(const Dual6& a) { return a.v < 0.0 ? -a : a; }
__device__ __forceinline__ double zero_like(double) { return 0.0; }
__device__ __forceinline__ Dual6 zero_like(const Dual6&) { return dconst(0.0); }
__device__ __forceinline__ double one_like(double) { return 1.0; }
__device__ __forceinline__ Dual6 one_like(const Dual6&) { return dconst(1.0); }

// sgn with zero counted as negative (a zero curvature is convex)
__device__ __forceinline__ double sgn_convex(double v) { return v > 0.0 ? 1.0 : -1.0; }

template <typename T>
struct FitPoint {
    T kmin, kmax;            // signed principal curvatures, |kmin| <= |kmax|
    T q[3];                  // Q*(0,0) = p + a00 n
    T nstar[3];              // unit normal of the patch at (0,0)
    T u[3];                  // axis of revolution n* x v_min
};

// Branchless orthonormal frame (s, t) of a unit normal n (Duff et al. 2017,
// "Building an Orthonormal Basis, Revisited"): the frame the six
// coefficients are expressed in.
__host__ __device__ inline void duff_frame(const double n[3], double s[3], double t[3]) {
    const double sg = n[2] >= 0.0 ? 1.0 : -1.0;
    const double fa = -1.0 / (sg + n[2]);
    const double fb = n[0] * n[1] * fa;
    s[0] = 1.0 + sg * n[0] * n[0] * fa;
    s[1] = sg * fb;
    s[2] = -sg * n[0];
    t[0] = fb;
    t[1] = sg + n[1] * n[1] * fa;
    t[2] = -n[1];
}

// n must be unit length.  a = {a00, a01, a10, a11, a02, a20}.
template <typename T>
__device__ void fit_point(const double p[3], const double n[3], const T a[6], FitPoint<T>& f) {
    const T& a00 = a[0];
    const T& a01 = a[1];
    const T& a10 = a[2];
    const T& a11 = a[3];
    const T& a02 = a[4];
    const T& a20 = a[5];
    double s[3], t[3];
    duff_frame(n, s, t);

    // fundamental forms at (0,0): I = [[E, F], [F, G]], II = [[2 a20, a11], [a11, 2 a02]] / A
    const T E = 1.0 + a10 * a10, G = 1.0 + a01 * a01, F = a10 * a01;
    const T A2 = 1.0 + a01 * a01 + a10 * a10;
    const T A = fsqrt(A2);
    // mean and Gauss curvature (Eq. MeanAndGaussCurvatures)
    const T H = (a02 * E + a20 * G - a11 * F) / (A2 * A);
    const T K = (4.0 * a02 * a20 - a11 * a11) / (A2 * A2);
    T disc = H * H - K;
    if (val(disc) < 0.0) disc = zero_like(disc);
    const T root = fsqrt(disc);
    const T kp = H + root, km = H - root;
    // kappa_min has the smaller magnitude; a tie keeps kappa_- as kappa_min
    const bool plus_is_min = fabs(val(kp)) < fabs(val(km));
    f.kmin = plus_is_min ? kp : km;
    f.kmax = plus_is_min ? km : kp;
    if (fabs(val(f.kmin)) <= kFlatKappa) f.kmin = zero_like(f.kmin);
    if (fabs(val(f.kmax)) <= kFlatKappa) f.kmax = zero_like(f.kmax);

    // principal direction of kappa_min: (II - kappa I) w = 0 (Eq. PrincipalDirections).
    // Each row of the 2x2 system gives a candidate; the longer is kept (the
    // printed one vanishes when a11 = 0 and kappa = 2 a20).  Umbilic: w = (1, 0).
    const T kA = f.kmin * A;
    const T w1x = kA * F - a11, w1y = 2.0 * a20 - kA * E;
    const T w2x = 2.0 * a02 - kA * G, w2y = kA * F - a11;
    const double l1 = val(w1x) * val(w1x) + val(w1y) * val(w1y);
    const double l2 = val(w2x) * val(w2x) + val(w2y) * val(w2y);
    T wx = l1 >= l2 ? w1x : w2x, wy = l1 >= l2 ? w1y : w2y;
    const double scale = fabs(val(a20)) + fabs(val(a02)) + fabs(val(a11)) +
                         fabs(val(kA)) * (val(E) + val(G)) + 1e-300;
    if (sqrt(fmax(l1, l2)) <= 1e-12 * scale) {
        wx = one_like(wx);
        wy = zero_like(wy);
    }
    T v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = wx * (s[k] + a10 * n[k]) + wy * (t[k] + a01 * n[k]);
    const T vl = fsqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        v[k] = v[k] / vl;
        f.nstar[k] = (n[k] - a10 * s[k] - a01 * t[k]) / A;   // (n - a10 s - a01 t) / A
        f.q[k] = p[k] + a00 * n[k];                            // Q*(0,0)
    }
    f.u[0] = f.nstar[1] * v[2] - f.nstar[2] * v[1];
    f.u[1] = f.nstar[2] * v[0] - f.nstar[0] * v[2];
    f.u[2] = f.nstar[0] * v[1] - f.nstar[1] * v[0];
}

}  // namespace ptsdf
