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

// ------------------------------------------------------------ launch chain ---
//
// Programmatic dependent launch (sm_90 and later).  A kernel launched with the
// programmatic stream-serialization attribute (launch_pdl) may start while the kernel
// before it in the stream is still running.  griddep_wait() blocks until that kernel
// has completed and its writes are visible; griddep_launch() allows the next kernel to
// start launching.  Every kernel of the step calls griddep_launch() only after its own
// griddep_wait(), so when a kernel starts, all kernels but its immediate predecessor
// have completed: before its wait it may read what those earlier kernels wrote, and it
// writes nothing.  Both are no-ops in a kernel launched without the attribute.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
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

// ------------------------------------------------------------ exact ops -----
//
// Round-to-nearest arithmetic that the compiler may not contract or reorder: the shape
// weights, the move and the current contributions are written with these, so every
// kernel that evaluates them (tiled or not, FP32 or FP64) produces the same bits.

__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

__device__ __forceinline__ float rdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double rdiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float rsqrt_rn(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double rsqrt_rn(double a) { return __dsqrt_rn(a); }

// x + v dt, wrapped (the IAEM position update)
template <typename T> __device__ __forceinline__ T move_pos(T x, T v, T dt, T l) {
    return wrap_pos(rfma(v, dt, x), l);
}

// ------------------------------------------------------------ shapes ------
//
// Centred cardinal B-spline of degree P (unit integral) in closed form.  For a
// particle at xi = x/dx (cell units) the first node with nonzero weight is
// floor(xi - (P+1)/2) + 1 and w[a] = W_P(xi - first - a), a = 0..P.

template <int P, typename T> struct Shape;

template <typename T> struct Shape<2, T> {
    // d in [-1/2, 1/2): w = ((1/2 - d)^2/2, 3/4 - d^2, (1/2 + d)^2/2)
    static __device__ __forceinline__ int weights(T xi, T* w) {
        const T h = (T)0.5;
        T f = floor(radd(xi, h));
        T d = rsub(xi, f);
        T hm = rsub(h, d), hp = radd(h, d);
        w[0] = rmul(h, rmul(hm, hm));
        w[1] = rfma(-d, d, (T)0.75);
        w[2] = rmul(h, rmul(hp, hp));
        return (int)f - 1;
    }
};

template <typename T> struct Shape<3, T> {
    // d in [0, 1), e = 1 - d: w = (e^3/6, 2/3 - d^2 + d^3/2, 2/3 - e^2 + e^3/2, d^3/6)
    static __device__ __forceinline__ int weights(T xi, T* w) {
        T f = floor(xi);
        T d = rsub(xi, f);
        T e = rsub((T)1, d);
        const T s6 = (T)(1.0 / 6.0), t3 = (T)(2.0 / 3.0), h = (T)0.5;
        T d2 = rmul(d, d), e2 = rmul(e, e);
        T d3 = rmul(d2, d), e3 = rmul(e2, e);
        w[0] = rmul(s6, e3);
        w[1] = rfma(h, d3, rsub(t3, d2));
        w[2] = rfma(h, e3, rsub(t3, e2));
        w[3] = rmul(s6, d3);
        return (int)f - 1;
    }
};

template <typename T> struct Shape<4, T> {
    // |t| in [1/2, 3/2): (55 + 20|t| - 120 t^2 + 80 |t|^3 - 16 t^4)/96, Horner form
    static __device__ __forceinline__ T mid(T t) {
        T r = rfma((T)-16, t, (T)80);
        r = rfma(r, t, (T)-120);
        r = rfma(r, t, (T)20);
        r = rfma(r, t, (T)55);
        return rmul(r, (T)(1.0 / 96.0));
    }
    // d in [-1/2, 1/2): w = ((1-2d)^4/384, mid(1+d), (115 - 120 d^2 + 48 d^4)/192,
    //                       mid(1-d), (1+2d)^4/384)
    static __device__ __forceinline__ int weights(T xi, T* w) {
        T f = floor(radd(xi, (T)0.5));
        T d = rsub(xi, f);
        T a = rfma((T)-2, d, (T)1), b = rfma((T)2, d, (T)1);
        T a2 = rmul(a, a), b2 = rmul(b, b), d2 = rmul(d, d);
        const T s384 = (T)(1.0 / 384.0);
        w[0] = rmul(s384, rmul(a2, a2));
        w[1] = mid(radd((T)1, d));
        w[2] = rmul(rfma(rmul((T)48, d2), d2, rfma((T)-120, d2, (T)115)), (T)(1.0 / 192.0));
        w[3] = mid(rsub((T)1, d));
        w[4] = rmul(s384, rmul(b2, b2));
        return (int)f - 2;
    }
};

}  // namespace gpic
