// Device helpers shared by the PIC kernels: complex arithmetic on double2/float2,
// the B-spline particle shapes, periodic wrap and the spectral wavenumbers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gpic {

// ------------------------------------------------------------ types -------

template <typename T> struct Cplx;
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<float> { using type = float2; };
template <typename T> using cplx_t = typename Cplx<T>::type;

template <typename C> __host__ __device__ __forceinline__ C mk(double re, double im) {
    C z;
    z.x = (decltype(z.x))re;
    z.y = (decltype(z.y))im;
    return z;
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by s*i (s = +-1)
__device__ __forceinline__ double2 cmul_si(double2 a, int s) { return make_double2(-s * a.y, s * a.x); }
__device__ __forceinline__ float2 cmul_si(float2 a, int s) { return make_float2(-s * a.y, s * a.x); }

// Complex numbers in FP64 used by the per-mode kernels whatever the storage type.
struct zd {
    double re, im;
};
__device__ __forceinline__ zd zmk(double r, double i) { return zd{r, i}; }
__device__ __forceinline__ zd operator+(zd a, zd b) { return zd{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ zd operator-(zd a, zd b) { return zd{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ zd operator*(double s, zd a) { return zd{s * a.re, s * a.im}; }
__device__ __forceinline__ zd operator-(zd a) { return zd{-a.re, -a.im}; }
__device__ __forceinline__ zd zconj(zd a) { return zd{a.re, -a.im}; }
__device__ __forceinline__ zd zi(zd a) { return zd{-a.im, a.re}; }  // i * a
__device__ __forceinline__ double znorm2(zd a) { return a.re * a.re + a.im * a.im; }
template <typename C> __device__ __forceinline__ zd zload(const C* p) {
    C v = *p;
    return zd{(double)v.x, (double)v.y};
}
template <typename C> __device__ __forceinline__ void zstore(C* p, zd v) {
    C w;
    w.x = (decltype(w.x))v.re;
    w.y = (decltype(w.y))v.im;
    *p = w;
}

// ------------------------------------------------------------ grid --------

// Spectral wavenumber of index m on an n-point periodic grid of length L:
// 2 pi m'/L with m' = m (m < n/2), m - n (m > n/2) and 0 at the Nyquist index.
__device__ __forceinline__ double wavenumber(int m, int n, double two_pi_over_l) {
    int s = (2 * m < n) ? m : ((2 * m == n) ? 0 : m - n);
    return two_pi_over_l * (double)s;
}

// Periodic wrap after a move of less than one period.
template <typename T> __device__ __forceinline__ T wrap_pos(T x, T l) {
    if (x >= l) x -= l;
    if (x < (T)0) x += l;
    return x;
}

__device__ __forceinline__ int wrap_idx(int i, int n) {
    if (i < 0) i += n;
    if (i >= n) i -= n;
    return i;
}

// ------------------------------------------------------------ shapes ------
//
// Centred cardinal B-spline of degree P (unit integral) in closed form.  For a
// particle at xi = x/dx (cell units) the first node with nonzero weight is
// floor(xi - (P+1)/2) + 1 and w[a] = W_P(xi - first - a), a = 0..P.

template <int P, typename T> struct Shape;

template <typename T> struct Shape<2, T> {
    static __device__ __forceinline__ int weights(T xi, T* w) {
        T f = floor(xi + (T)0.5);
        T d = xi - f;
        T hm = (T)0.5 - d, hp = (T)0.5 + d;
        w[0] = (T)0.5 * hm * hm;
        w[1] = (T)0.75 - d * d;
        w[2] = (T)0.5 * hp * hp;
        return (int)f - 1;
    }
};

template <typename T> struct Shape<3, T> {
    static __device__ __forceinline__ int weights(T xi, T* w) {
        T f = floor(xi);
        T d = xi - f;
        T e = (T)1 - d;
        const T s6 = (T)(1.0 / 6.0), t3 = (T)(2.0 / 3.0);
        w[0] = s6 * e * e * e;
        w[1] = t3 - d * d + (T)0.5 * d * d * d;
        w[2] = t3 - e * e + (T)0.5 * e * e * e;
        w[3] = s6 * d * d * d;
        return (int)f - 1;
    }
};

template <typename T> struct Shape<4, T> {
    static __device__ __forceinline__ T mid(T t) {  // 1/2 <= |t| < 3/2
        return ((T)55 + t * ((T)20 + t * ((T)-120 + t * ((T)80 - (T)16 * t)))) * (T)(1.0 / 96.0);
    }
    static __device__ __forceinline__ int weights(T xi, T* w) {
        T f = floor(xi + (T)0.5);
        T d = xi - f;
        T a = (T)1 - (T)2 * d, b = (T)1 + (T)2 * d;
        T a2 = a * a, b2 = b * b, d2 = d * d;
        const T s384 = (T)(1.0 / 384.0);
        w[0] = s384 * a2 * a2;
        w[1] = mid((T)1 + d);
        w[2] = ((T)115 - (T)120 * d2 + (T)48 * d2 * d2) * (T)(1.0 / 192.0);
        w[3] = mid((T)1 - d);
        w[4] = s384 * b2 * b2;
        return (int)f - 2;
    }
};

}  // namespace gpic
