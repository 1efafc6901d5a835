// Particle kernels of one PIC step (Algorithm 1, section 4.2), plain path.
//
//   move + deposit : x^{n+1} = x^n + v^n dt (wrapped), then J^{n+1} gets
//                    q_p v^n W(x^{n+1}/dx - i) W(y^{n+1}/dy - j) / (dx dy) at the
//                    (p+1)^2 nodes of the tensor-product B-spline (sections 2.2, 4).
//                    The kernel accumulates sum_p v W; q_p/(dx dy) is applied per mode.
//   gather + push  : the same shape gathers the eight fields (grad phi~, A, grad A)
//                    at x^{n+1}; then IAEM (section 4.1): v* = 2v^n - v^{n-1},
//                    P^{n+1} = P^n + q dt (-grad phi~ + grad A . v*),
//                    v^{n+1} = c^2 (P - qA) / sqrt(c^2 |P - qA|^2 + (m c^2)^2),
//                    written over v^{n-1} (the caller swaps the velocity buffers).
//   init           : wrap x^0, P^0 = gamma m v^0, v^{-1} by one Taylor step back in E^0.
// Particles are SoA arrays; one thread per particle in a grid-stride loop.  A
// position outside [0, L] (including NaN) is never used to index the grid: the
// particle is skipped and the non-finite bit of the device error word is set.
#include "common.cuh"
#include "gpic_internal.h"
#include "launch.cuh"

namespace gpic {

namespace {

constexpr int kThreads = 256;

// Geometry and push constants in the storage precision, converted once on the host so
// the per-thread set-up of the FP32 kernels issues no FP64 conversions (GB300 has little
// FP64 throughput).
template <typename T>
struct GeomT {
    int nx, ny;
    T lx, ly, inv_dx, inv_dy, dt;
};
template <typename T>
GeomT<T> typed(const ParticleGeom& g) {
    return GeomT<T>{g.nx, g.ny, (T)g.lx, (T)g.ly, (T)g.inv_dx, (T)g.inv_dy, (T)g.dt};
}
template <typename T>
struct PushT {
    T q, qdt, c2, mc2;
    double c, m, weight;  // FP64 kinetic-energy diagnostic
    int diag;
};
template <typename T>
PushT<T> typed(const PushParams& pp) {
    return PushT<T>{(T)pp.q, (T)(pp.q * pp.dt), (T)(pp.c * pp.c), (T)(pp.m * pp.c * pp.c),
                    pp.c, pp.m, pp.weight, pp.diag};
}

// The deposit factors q_s w_s of a species table in the storage precision.
template <typename T>
struct SpeciesT {
    int n;
    T qw[kMaxSpecies];
};
template <typename T>
SpeciesT<T> typed_species(const SpeciesParams* spp) {
    SpeciesT<T> r{};
    if (spp) {
        r.n = spp->n;
        for (int k = 0; k < kMaxSpecies; ++k) r.qw[k] = (T)spp->qw[k];
    }
    return r;
}
// q_s w_s of particle p (1 without a table); false for an index outside the table.
template <typename T>
__device__ __forceinline__ bool species_factor(const int32_t* __restrict__ sp,
                                               const SpeciesT<T>& spt, int64_t p, T& f) {
    f = (T)1;
    if (!sp) return true;
    const int s = sp[p];
    if ((unsigned)s >= (unsigned)spt.n) return false;
    f = spt.qw[s];
    return true;
}

inline int blocks_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    const int64_t cap = 152 * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// The eight gather fields of one node ([node][4] complex, 32 B in FP32, 64 B in FP64) with
// 16-byte loads.
__device__ __forceinline__ void load_node(const float2* node, float* g) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(node));
    const float4 b = __ldg(reinterpret_cast<const float4*>(node) + 1);
    g[0] = a.x; g[1] = a.y; g[2] = a.z; g[3] = a.w;
    g[4] = b.x; g[5] = b.y; g[6] = b.z; g[7] = b.w;
}
__device__ __forceinline__ void load_node(const double2* node, double* g) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double2 v = __ldg(node + k);
        g[2 * k] = v.x;
        g[2 * k + 1] = v.y;
    }
}

// Asks the L2 to fetch the 16-byte-aligned part of [p, p + bytes) (a bulk prefetch: one
// instruction, no registers, no completion to wait for).
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uintptr_t lo = (a + 15) & ~(uintptr_t)15, hi = (a + bytes) & ~(uintptr_t)15;
    if (hi > lo)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((unsigned)(hi - lo))
                     : "memory");
}

template <typename T>
__device__ __forceinline__ bool in_domain(T xi, int n) {
    return xi >= (T)0 && xi <= (T)n;
}

// Current accumulation policies.  AccF64: FP64 atomics (plain path).  AccFix: each
// contribution is rounded to an integer multiple of 1/scale and summed with int64
// atomics, so the grid total does not depend on the order of the additions.
struct AccF64 {
    double2* J;
    template <typename T>
    __device__ __forceinline__ T pre(T v) const { return v; }
    // (tx wy, ty wy) to node: the two current components of one stencil node
    template <typename T>
    __device__ __forceinline__ void add2(size_t node, T tx, T ty, T wy) const {
        atomicAdd(&J[node].x, (double)rmul(tx, wy));
        atomicAdd(&J[node].y, (double)rmul(ty, wy));
    }
    template <typename T>
    __device__ __forceinline__ void add1f(size_t node, T t, T w) const {
        atomicAdd(&J[node].x, (double)rmul(t, w));
    }
    template <typename T>
    __device__ __forceinline__ void add1(size_t node, T a) const {
        atomicAdd(&J[node].x, (double)a);
    }
};

struct AccFix {
    longlong2* J;
    float scale;     // 1 / quantum, a power of two
    float s_hi;      // scale 2^-19
    template <typename T>
    __device__ __forceinline__ T pre(T v) const { return v; }
    static AccFix make(void* j, float scale) {
        return AccFix{(longlong2*)j, scale, scale * (1.0f / 524288.0f)};
    }
    // round(v * scale), the contribution in units of the quantum (the deposited charge of
    // the naive update only: the float-to-int64 conversion runs on the FP64 pipe)
    __device__ __forceinline__ static long long q(float v, float s) {
        return __float2ll_rn(__fmul_rn(v, s));
    }
    // The contribution of a current component to one node is t w (t = v W_x rounded to
    // FP32, w = W_y): its exact product, rounded once to the quantum, rne(t w scale), split
    // as hi 2^19 + lo with three FMAs, for |t w scale| <= 2^38.  wh = w scale 2^-19 and
    // ws = w scale are exact (power-of-two scalings, see scaled()).  With M = 1.5 2^23:
    //   m1 = rne(t wh + M)             = M + hi,   hi = rne(t w scale 2^-19), |hi| <= 2^19
    //   mt = m1 (-2^19) + M (2^19 + 1) = M - hi 2^19   (exact: a multiple of 2^19 below 2^39)
    //   l  = rne(t ws + mt)            = M + lo,   lo = rne(t w scale - hi 2^19), |lo| <= 2^18
    // (every FMA rounds the exact a b + c once; results in [2^23, 2^24) round to integers).
    // hi 2^19 is even, so hi 2^19 + lo = rne(t w scale).
    __device__ __forceinline__ static void split2(float t, float wh, float ws, int& hi, int& lo) {
        const float m1 = __fmaf_rn(t, wh, 12582912.0f);
        const float mt = __fmaf_rn(m1, -524288.0f, 6597082349568.0f);
        hi = __float_as_int(m1) - 0x4B400000;
        lo = __float_as_int(__fmaf_rn(t, ws, mt)) - 0x4B400000;
    }
    __device__ __forceinline__ void scaled(float w, float& wh, float& ws) const {
        wh = __fmul_rn(w, s_hi);
        ws = __fmul_rn(w, scale);
    }
    __device__ __forceinline__ static unsigned long long join(int hi, int lo) {
        return (unsigned long long)((long long)hi * 524288ll + (long long)lo);
    }
    template <typename T>
    __device__ __forceinline__ void add2(size_t node, T tx, T ty, T wy) const {
        float wh, ws;
        scaled((float)wy, wh, ws);
        int ha, la, hb, lb;
        split2((float)tx, wh, ws, ha, la);
        split2((float)ty, wh, ws, hb, lb);
        atomicAdd(reinterpret_cast<unsigned long long*>(&J[node].x), join(ha, la));
        atomicAdd(reinterpret_cast<unsigned long long*>(&J[node].y), join(hb, lb));
    }
    template <typename T>
    __device__ __forceinline__ void add1f(size_t node, T t, T w) const {
        float wh, ws;
        scaled((float)w, wh, ws);
        int h, l;
        split2((float)t, wh, ws, h, l);
        atomicAdd(reinterpret_cast<unsigned long long*>(&J[node].x), join(h, l));
    }
    template <typename T>
    __device__ __forceinline__ void add1(size_t node, T a) const {
        atomicAdd(reinterpret_cast<unsigned long long*>(&J[node].x), (unsigned long long)q((float)a, scale));
    }
};

// FP64 path: each contribution is rounded once to an integer multiple of the quantum
// 1/scale (|x| <= 2^60 by the choice of scale, a power of two) and summed exactly as a
// 128-bit integer per node and component: a low word (unsigned, modulo 2^64) and a high
// word.  The atomic on the low word returns the word it added to, so the carry out of
// each addition is known exactly; the carry and the sign extension of x go to the high
// word, which changes only when the low word wraps.  Integer sums do not depend on the
// order of the additions, so the deposit is bit-for-bit deterministic.
struct AccFix128 {
    longlong2* J;  // [node]: the low words (x, y); [ng + node]: the high words
    size_t ng;
    double scale;
    // the velocity factor carries the scale (exact: a power of two), so each contribution
    // is rounded to an integer once
    template <typename T>
    __device__ __forceinline__ T pre(T v) const { return v * (T)scale; }
    __device__ __forceinline__ void add_word(size_t node, int comp, long long x) const {
        unsigned long long* lo = reinterpret_cast<unsigned long long*>(J + node) + comp;
        const unsigned long long ux = (unsigned long long)x;
        const unsigned long long old = atomicAdd(lo, ux);
        const long long dh = (x < 0 ? -1ll : 0ll) + (old + ux < old ? 1ll : 0ll);
        if (dh != 0)
            atomicAdd(reinterpret_cast<unsigned long long*>(J + ng + node) + comp,
                      (unsigned long long)dh);
    }
    template <typename T>
    __device__ __forceinline__ void add2(size_t node, T tx, T ty, T wy) const {
        add_word(node, 0, __double2ll_rn((double)rmul(tx, wy)));
        add_word(node, 1, __double2ll_rn((double)rmul(ty, wy)));
    }
    template <typename T>
    __device__ __forceinline__ void add1f(size_t node, T t, T w) const {
        add_word(node, 0, __double2ll_rn((double)rmul(t, w)));
    }
    template <typename T>
    __device__ __forceinline__ void add1(size_t node, T a) const {
        add_word(node, 0, __double2ll_rn((double)a * scale));
    }
};

// hi 2^64 + lo (two's complement over 128 bits) times unscale, rounded to FP64: the
// magnitude is exact below 2^64 before its one rounding, and rounded twice above.
__device__ __forceinline__ double fix128_value(long long hi, unsigned long long lo,
                                               double unscale) {
    const bool neg = hi < 0;
    if (neg) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ll : 0ll);
    }
    const double m = fma((double)hi, 18446744073709551616.0, (double)lo);
    return (neg ? -m : m) * unscale;
}

template <typename T, int P, typename Acc>
__global__ void __launch_bounds__(kThreads)
k_move_deposit(GeomT<T> g, T* __restrict__ x, T* __restrict__ y, const T* __restrict__ vx,
               const T* __restrict__ vy, int64_t n, Acc acc, unsigned int* __restrict__ err,
               const int32_t* __restrict__ sp, SpeciesT<T> spt) {
    const T dt = g.dt, lx = g.lx, ly = g.ly, idx_ = g.inv_dx, idy = g.inv_dy;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        T vxi = vx[p], vyi = vy[p];
        T xp = move_pos(x[p], vxi, dt, lx);
        T yp = move_pos(y[p], vyi, dt, ly);
        x[p] = xp;
        y[p] = yp;
        const T xi = rmul(xp, idx_), yj = rmul(yp, idy);
        T fq;
        if (!in_domain(xi, g.nx) || !in_domain(yj, g.ny) || !species_factor(sp, spt, p, fq)) {
            atomicOr(err, (unsigned)ERR_NONFINITE);
            continue;
        }
        if (sp) {  // each contribution carries the particle's q_s w_s
            vxi = rmul(vxi, fq);
            vyi = rmul(vyi, fq);
        }
        vxi = acc.pre(vxi);
        vyi = acc.pre(vyi);
        T wx[P + 1], wy[P + 1];
        const int ix = Shape<P, T>::weights(xi, wx);
        const int iy = Shape<P, T>::weights(yj, wy);
#pragma unroll
        for (int a = 0; a <= P; ++a) {
            const int gi = wrap_idx(ix + a, g.nx);
            const T tx = rmul(vxi, wx[a]), ty = rmul(vyi, wx[a]);
            const size_t row = (size_t)gi * g.ny;
#pragma unroll
            for (int b = 0; b <= P; ++b) acc.add2(row + wrap_idx(iy + b, g.ny), tx, ty, wy[b]);
        }
    }
}

template <typename T, int P, typename Acc>
__global__ void __launch_bounds__(kThreads)
k_deposit_charge(ParticleGeom g, const T* __restrict__ x, const T* __restrict__ y, int64_t n,
                 Acc acc, unsigned int* __restrict__ err, const int32_t* __restrict__ sp,
                 SpeciesT<T> spt) {
    const T idx_ = (T)g.inv_dx, idy = (T)g.inv_dy;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const T xi = rmul(x[p], idx_), yj = rmul(y[p], idy);
        T fq;
        if (!in_domain(xi, g.nx) || !in_domain(yj, g.ny) || !species_factor(sp, spt, p, fq)) {
            atomicOr(err, (unsigned)ERR_NONFINITE);
            continue;
        }
        T wx[P + 1], wy[P + 1];
        const int ix = Shape<P, T>::weights(xi, wx);
        const int iy = Shape<P, T>::weights(yj, wy);
#pragma unroll
        for (int a = 0; a <= P; ++a) {
            const int gi = wrap_idx(ix + a, g.nx);
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                const int gj = wrap_idx(iy + b, g.ny);
                const T wab = rmul(wx[a], wy[b]);
                acc.add1((size_t)gi * g.ny + gj, sp ? rmul(wab, fq) : wab);
            }
        }
    }
}


// The binned FP32 pass keeps its 32-bit region sums in two parts of a contribution:
// node totals are hi 2^kLoBits + lo (see AccFix::split2).
constexpr int kLoBits = 19;

// Fixed-point (Jx, Jy) sums to complex storage values, times `unscale`.
template <typename T>
__global__ void k_fix_to_cplx(const longlong2* __restrict__ J, double unscale,
                              cplx_t<T>* __restrict__ out, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const longlong2 v = J[k];
        out[k] = mk<cplx_t<T>>((double)v.x * unscale, (double)v.y * unscale);
    }
}

// FP64 path: the 128-bit sums of AccFix128 to complex FP64 values, times `unscale`.
__global__ void k_fix128_to_cplx(const longlong2* __restrict__ J, size_t ng, double unscale,
                                 double2* __restrict__ out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < (int64_t)ng;
         k += (int64_t)gridDim.x * blockDim.x) {
        const longlong2 lo = J[k], hi = J[ng + k];
        out[k] = make_double2(fix128_value(hi.x, (unsigned long long)lo.x, unscale),
                              fix128_value(hi.y, (unsigned long long)lo.y, unscale));
    }
}

__global__ void k_extract_fix(const longlong2* __restrict__ J, int comp, double scale,
                              double* __restrict__ dst, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const longlong2 v = J[k];
        dst[k] = scale * (double)(comp ? v.y : v.x);
    }
}

// Gather of the eight fields at one particle: f += W_x[a] W_y[b] g(node), nodes in the
// order a = 0..P, b = 0..P (the same order and roundings in every gather kernel).
template <typename T>
__device__ __forceinline__ void gather_node(T w, const T* g, T* f) {
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] = rfma(w, g[k], f[k]);
}

// IAEM push of particle p from its gathered fields (section 3.3):
//   P^{n+1} = P^n + q dt (-grad phi + (grad A) . v*),  v* = 2 v^n - v^{n-1}
//   u = P^{n+1} - q A,  v^{n+1} = c^2 u / sqrt(c^2 |u|^2 + (m c^2)^2)
// f = (dphi/dx, dphi/dy, Ax, Ay, dAx/dx, dAx/dy, dAy/dx, dAy/dy).  v^{n+1} overwrites
// v^{n-1}.  Written with explicit roundings, so every kernel gives the same bits.
// m c^2 (gamma - 1) per unit weight from |u|^2 (u = P - q A), accumulated in FP64.  FP64
// storage: in FP64 from the identity gamma m c^2 = sqrt(c^2 |u|^2 + (m c^2)^2).  FP32
// form: in FP32 as c^2 |u|^2 / (m c^2 (gamma + 1)), gamma = sqrt(1 + c^2 |u|^2 / (m c^2)^2),
// which has no cancellation at small |u| (the FP32 momenta carry 2^-24 relative error
// already, and the FP64 sqrt per particle would cost the FP32 kernels more than their
// whole push).
template <typename T>
__device__ __forceinline__ double kinetic(T c2, T mc2, double c, double m, T u2) {
    if constexpr (sizeof(T) == 4) {
        const float t = __fmul_rn(c2, u2);
        const float g = __fsqrt_rn(__fadd_rn(1.0f, __fdiv_rn(t, __fmul_rn(mc2, mc2))));
        return (double)__fdiv_rn(t, __fmul_rn(mc2, __fadd_rn(g, 1.0f)));
    } else {
        const double c2d = c * c, mc2d = m * c2d;
        return sqrt(c2d * (double)u2 + mc2d * mc2d) - mc2d;
    }
}

// The push from the particle's values (P^n, v^n, v^{n-1}): returns P^{n+1} and v^{n+1}.
template <typename T>
__device__ __forceinline__ void push_core(const PushT<T>& pp, const T* f, T px, T py, T vx, T vy,
                                          T vxo, T vyo, unsigned& bad, double& kin, T& Px_new,
                                          T& Py_new, T& vx_new, T& vy_new) {
    const T vsx = rfma((T)2, vx, -vxo);
    const T vsy = rfma((T)2, vy, -vyo);
    const T fx = rfma(f[6], vsy, rfma(f[4], vsx, -f[0]));
    const T fy = rfma(f[7], vsy, rfma(f[5], vsx, -f[1]));
    const T Px = rfma(pp.qdt, fx, px);
    const T Py = rfma(pp.qdt, fy, py);
    const T ux = rfma(-pp.q, f[2], Px), uy = rfma(-pp.q, f[3], Py);
    const T den = rsqrt_rn(rfma(pp.c2, rfma(ux, ux, rmul(uy, uy)), rmul(pp.mc2, pp.mc2)));
    const T rc = rdiv(pp.c2, den);
    const T vxn1 = rmul(rc, ux), vyn1 = rmul(rc, uy);
    Px_new = Px;
    Py_new = Py;
    vx_new = vxn1;
    vy_new = vyn1;
    if (!isfinite(vxn1) || !isfinite(vyn1)) bad |= ERR_NONFINITE;
    if (pp.diag) kin += kinetic(pp.c2, pp.mc2, pp.c, pp.m, rfma(ux, ux, rmul(uy, uy)));
}

template <typename T>
__device__ __forceinline__ void push_one(const PushT<T>& pp, const T* f, int64_t p,
                                         T* __restrict__ px, T* __restrict__ py,
                                         const T* __restrict__ vx, const T* __restrict__ vy,
                                         T* __restrict__ vxo, T* __restrict__ vyo, unsigned& bad,
                                         double& kin, T& vx_new, T& vy_new) {
    T Px, Py;
    push_core(pp, f, px[p], py[p], vx[p], vy[p], vxo[p], vyo[p], bad, kin, Px, Py, vx_new,
              vy_new);
    px[p] = Px;
    py[p] = Py;
    vxo[p] = vx_new;
    vyo[p] = vy_new;
}

template <typename T>
__device__ __forceinline__ void push_finish(const PushT<T>& pp, unsigned bad, double kin,
                                            double* __restrict__ diag,
                                            unsigned int* __restrict__ err) {
    if (bad) atomicOr(err, bad);
    if (pp.diag) {
        for (int o = 16; o > 0; o >>= 1) kin += __shfl_down_sync(0xffffffffu, kin, o);
        if ((threadIdx.x & 31) == 0 && kin != 0.0) atomicAdd(diag + D_KIN, kin * pp.weight);
    }
}

template <typename T, int P>
__global__ void __launch_bounds__(kThreads)
k_gather_push(GeomT<T> g, PushT<T> pp, const T* __restrict__ x, const T* __restrict__ y,
              T* __restrict__ px, T* __restrict__ py, const T* __restrict__ vx,
              const T* __restrict__ vy, T* __restrict__ vxo, T* __restrict__ vyo, int64_t n,
              const cplx_t<T>* __restrict__ F, double* __restrict__ gout, int gout_short,
              double* __restrict__ diag, unsigned int* __restrict__ err) {
    using C = cplx_t<T>;
    const T idx_ = g.inv_dx, idy = g.inv_dy;
    double kin = 0.0;
    unsigned bad = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const T xi = rmul(x[p], idx_), yj = rmul(y[p], idy);
        if (!in_domain(xi, g.nx) || !in_domain(yj, g.ny)) {
            bad |= ERR_NONFINITE;
            continue;
        }
        T wx[P + 1], wy[P + 1];
        const int ix = Shape<P, T>::weights(xi, wx);
        const int iy = Shape<P, T>::weights(yj, wy);
        T f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int a = 0; a <= P; ++a) {
            const int gi = wrap_idx(ix + a, g.nx);
            const C* row = F + (size_t)gi * g.ny * 4;
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                const int gj = wrap_idx(iy + b, g.ny);
                T gv[8];
                load_node(row + (size_t)gj * 4, gv);
                gather_node(rmul(wx[a], wy[b]), gv, f);
            }
        }
        T vxn1, vyn1;
        push_one(pp, f, p, px, py, vx, vy, vxo, vyo, bad, kin, vxn1, vyn1);
        if (gout) {  // the adjoint's record of this step (see launcher)
            gout[p] = (double)px[p];
            gout[(size_t)n + p] = (double)py[p];
            gout[2 * (size_t)n + p] = (double)vxn1;
            gout[3 * (size_t)n + p] = (double)vyn1;
            if (!gout_short) {
#pragma unroll
                for (int k = 2; k < 8; ++k) gout[(size_t)(k + 2) * n + p] = (double)f[k];
            }
        }
    }
    push_finish(pp, bad, kin, diag, err);
}

// Gather + push over particles sorted by tile and cell (see sort.cu), FP32 form.
//
// CTA (tile, split) copies the gather fields of the tile's node region (the tile plus a
// halo: rx x ry nodes, 32 B each) into shared memory, then pushes a contiguous share of
// the tile's particles.  Consecutive particles mostly sit in one cell, so the lanes of a
// warp read the same node: shared-memory broadcasts.  A particle whose stencil leaves the
// region (it drifted further than the halo) reads the global fields.  Node order and
// roundings are those of k_gather_push, so the two give the same bits.
template <int P>
__global__ void __launch_bounds__(kThreads, 4)
k_gather_push_tiled(GeomT<float> g, PushT<float> pp, TileGeom tg, const float* __restrict__ x,
                    const float* __restrict__ y, float* __restrict__ px,
                    float* __restrict__ py, const float* __restrict__ vx,
                    const float* __restrict__ vy, float* __restrict__ vxo,
                    float* __restrict__ vyo,
                    const int* __restrict__ off, int nsplit, const float2* __restrict__ F,
                    double* __restrict__ diag, unsigned int* __restrict__ err) {
    extern __shared__ float4 sf[];  // [rx][ry] nodes, two float4 each
    const int tt = tg.t * tg.t;
    const int tile = blockIdx.x / nsplit, split = blockIdx.x - tile * nsplit;
    const int64_t t0 = off[tile * tt], cnt = (int64_t)off[(tile + 1) * tt] - t0;
    const int64_t p0 = t0 + cnt * split / nsplit, p1 = t0 + cnt * (split + 1) / nsplit;
    if (p0 == p1) return;  // uniform for the CTA
    if (threadIdx.x < 8) {  // the CTA's particles come to L2 while it stages the fields
        const float* arr[8] = {x, y, px, py, vx, vy, vxo, vyo};
        prefetch_l2(arr[threadIdx.x] + p0, (size_t)(p1 - p0) * sizeof(float));
    }
    const int tx = tile / tg.nty, ty = tile - tx * tg.nty;
    int bi = (tx * tg.t - tg.halo) % g.nx, bj = (ty * tg.t - tg.halo) % g.ny;
    if (bi < 0) bi += g.nx;
    if (bj < 0) bj += g.ny;
    const int rx = tg.rx, ry = tg.ry;
    const float4* F4 = reinterpret_cast<const float4*>(F);
    griddep_wait();  // the fields are the previous kernel's output
    griddep_launch();
    for (int k = threadIdx.x; k < 2 * rx * ry; k += blockDim.x) {
        const int node = k >> 1;
        const int ri = node / ry, rj = node - ri * ry;
        int gi = bi + ri, gj = bj + rj;
        if (gi >= g.nx) gi -= g.nx;
        if (gj >= g.ny) gj -= g.ny;
        sf[k] = __ldg(F4 + ((size_t)gi * g.ny + gj) * 2 + (k & 1));
    }
    __syncthreads();
    const float idx_ = g.inv_dx, idy = g.inv_dy;
    double kin = 0.0;
    unsigned bad = 0;
    for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const float xp = x[p], yp = y[p];
        const float xi = rmul(xp, idx_), yj = rmul(yp, idy);
        if (!in_domain(xi, g.nx) || !in_domain(yj, g.ny)) {
            bad |= ERR_NONFINITE;
            continue;
        }
        float wx[P + 1], wy[P + 1];
        const int ix = wrap_idx(Shape<P, float>::weights(xi, wx), g.nx);
        const int iy = wrap_idx(Shape<P, float>::weights(yj, wy), g.ny);
        int ri0 = ix - bi, rj0 = iy - bj;
        if (ri0 < 0) ri0 += g.nx;
        if (rj0 < 0) rj0 += g.ny;
        float f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (ri0 + P < rx && rj0 + P < ry) {
            const float4* row = sf + 2 * (ri0 * ry + rj0);
#pragma unroll
            for (int a = 0; a <= P; ++a) {
#pragma unroll
                for (int b = 0; b <= P; ++b) {
                    const float4 u = row[2 * b], v = row[2 * b + 1];
                    const float gv[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
                    gather_node(rmul(wx[a], wy[b]), gv, f);
                }
                row += 2 * ry;
            }
        } else {
#pragma unroll
            for (int a = 0; a <= P; ++a) {
                const int gi = wrap_idx(ix + a, g.nx);
#pragma unroll
                for (int b = 0; b <= P; ++b) {
                    const int gj = wrap_idx(iy + b, g.ny);
                    float gv[8];
                    load_node(F + ((size_t)gi * g.ny + gj) * 4, gv);
                    gather_node(rmul(wx[a], wy[b]), gv, f);
                }
            }
        }
        float vxn1, vyn1;
        push_one(pp, f, p, px, py, vx, vy, vxo, vyo, bad, kin, vxn1, vyn1);
    }
    push_finish(pp, bad, kin, diag, err);
}

// ------------------------------------------------------------ binned FP32 pass -----
//
// Move + deposit of the FP32 form over tile-sorted particles, and the same pass fused
// with the gather + push of the step before it (kFused).
//
// CTA (tile, split) takes a contiguous share [p0, p1) of one tile's particles and works
// through it in the fewest batches of at most `cap` particles, of equal sizes (a batch
// costs the same barriers, scan and region flush whatever its size, so a share of
// cap + 20 runs as two halves, not as cap and 20):
//   A  consecutive lanes take consecutive particles (the SoA loads and stores coalesce;
//      unfused, each thread's next particle is loaded while it works on the current one).
//      Fused: gather the eight fields of the step at x^{n+1} from the tile's field region
//      staged in shared memory, IAEM push (section 4.1) -> P^{n+1}, v^{n+1}.  Then the move
//      x^{n+2} = x^{n+1} + v^{n+1} dt (the next step's first operation, Algorithm 1).  The
//      moved particle (x, y, vx, vy) goes to a staging slot, keyed by the region node of its
//      stencil base; a shared atomic on that key's count gives its rank there.
//   B  an exclusive scan of the counts over the region's nodes.
//   C  each staged slot is written at its key's offset plus its rank: the batch is now
//      binned by stencil base.
//   D  thread t takes an equal slice of the binned particles (slices spread over the
//      threads so that the lanes of a warp work in different cells).  Consecutive
//      particles of a slice mostly share their stencil base and so all (p+1)^2 nodes:
//      their fixed-point contributions rne(t_a W_y,b scale) are summed exactly in
//      registers (int32 hi and lo parts, AccFix::split2) and added to the CTA's shared
//      node region with one set of atomics whenever the base changes, instead of
//      4 (p+1)^2 atomics per particle.  The stencil rows are summed in passes of at most
//      two rows (three for quadratic shapes) over the slice, which keeps the sums within
//      the register budget of four CTAs per SM.
//   The region is added to the global int64 grid after every batch, which keeps every
//   32-bit sum exact: a batch adds at most cap <= kBinBatchMax = 1152 contributions of
//   magnitude <= 2^19 to a node, less than 2^30 in all.
// A particle whose stencil leaves the region (it drifted further than the halo) adds its
// contributions straight to the global grid.  The integer sums make J independent of the
// order of the particles and of how they are grouped, so the result is the same bits as
// every other deposit of the FP32 form.
// Batch capacity: kBinBatchMax where four CTAs per SM still fit (a tile share of about
// 1024 particles then runs as one batch even when sampling noise puts it a little above
// 1024), else kBinBatchMin; whether a tiling can use the pass at all is judged at the
// smaller one.
constexpr int kBinBatchMin = 1024;
constexpr int kBinBatchMax = 1152;
constexpr int kBinSmemMax = 100 * 1024;  // four CTAs per SM fit up to 56 KB each

// Byte offsets in the binned pass's dynamic shared memory (stage first: 16-byte aligned).
// The species constants of the binned pass (FP32 form): the deposit factor q_s w_s, the
// push constants of k_gather_push3 (q_s, q_s dt, m_s c^2 in FP32) and the FP64 mass and
// weight of the kinetic-energy diagnostic.
struct BinSpecies {
    int n;
    float qw[kMaxSpecies], q[kMaxSpecies], qdt[kMaxSpecies], mc2[kMaxSpecies];
    double m[kMaxSpecies], w[kMaxSpecies];
};

struct BinLayout {
    int fields;   // kFused: the gather fields of the region, [rx][ry] x 2 float4
    int stz;      // 2D-3V: float [cap]: v_z of each staged particle
    int kr;       // int [cap]: key | rank << 16 of each staged particle (-1: none)
    int idx;      // uint16 [cap]: staging slots in binned order
    int racc;     // int [4 rx ry] (2D-3V: 6): lo_x, lo_y, hi_x, hi_y (lo_z, hi_z) node sums
    int cnt;      // int [rx ry + 1]: counts, then offsets
    int bytes;
};
__host__ __device__ inline BinLayout bin_layout(const TileGeom& tg, int p, bool fused,
                                                bool z = false, int cap = kBinBatchMin) {
    BinLayout l;
    int o = cap * 16;  // stage: (x, y, vx, vy) of each particle, arrival order
    l.fields = o;
    if (fused) o += tg.rx * tg.ry * 32;
    l.stz = o;
    if (z) o += cap * 4;
    l.kr = o;
    o += cap * 4;
    l.idx = o;
    o += cap * 2;
    o = (o + 15) & ~15;
    l.racc = o;
    o += (z ? 6 : 4) * tg.rx * tg.ry * 4;
    l.cnt = o;
    o += (tg.rx * tg.ry + 1) * 4;
    l.bytes = (o + 15) & ~15;
    return l;
}

// Exclusive scan of one value per thread over the CTA (kThreads); sets *total.
__device__ __forceinline__ int cta_exclusive_scan(int v, int* wsum, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int w = lane < kThreads / 32 ? wsum[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < kThreads / 32) wsum[lane] = wi - w;
        if (lane == 31) wsum[32] = wi;
    }
    __syncthreads();
    *total = wsum[32];
    return wsum[warp] + inc - v;
}

// Register sums of stencil rows A0..A1-1 of one base node: s[a][b] = (lo_x, lo_y, hi_x,
// hi_y) and, in 2D-3V (NQ = 6), (lo_z, hi_z).
template <int P, int NA, int NQ = 4>
struct RowSums {
    int s[NA][P + 1][NQ];
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int b = 0; b <= P; ++b)
#pragma unroll
                for (int q = 0; q < NQ; ++q) s[a][b][q] = 0;
    }
    // adds them to the region at node0 (rows of ry nodes; the NQ planes R apart)
    __device__ __forceinline__ void flush(int* __restrict__ node0, int ry, int R) const {
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            int* row = node0 + a * ry;
#pragma unroll
            for (int b = 0; b <= P; ++b)
#pragma unroll
                for (int q = 0; q < NQ; ++q) atomicAdd(row + q * R + b, s[a][b][q]);
        }
    }
};

// Deposit of the binned particles [k0, k1) (sidx order) for stencil rows A0..A1-1: the
// contributions are summed in registers while the key (the region node of the stencil
// base) stays the same.
template <int P, int A0, int A1, bool kZ = false>
__device__ __forceinline__ void bin_slice_rows(const float4* __restrict__ stage,
                                               const int* __restrict__ kr,
                                               const uint16_t* __restrict__ sidx, int k0, int k1,
                                               float idx_, float idy, const AccFix& acc,
                                               int* __restrict__ racc, int ry, int R,
                                               const float* __restrict__ stz = nullptr) {
    RowSums<P, A1 - A0, kZ ? 6 : 4> rs;
    rs.clear();
    int cur = -1;
#pragma unroll 1
    for (int k = k0; k < k1; ++k) {
        const int slot = sidx[k];
        const int key = kr[slot] & 0xFFFF;
        const float4 q4 = stage[slot];
        if (key != cur) {
            if (cur >= 0) {
                rs.flush(racc + cur + A0 * ry, ry, R);
                rs.clear();
            }
            cur = key;
        }
        float wx[P + 1], wy[P + 1];
        Shape<P, float>::weights(rmul(q4.x, idx_), wx);
        Shape<P, float>::weights(rmul(q4.y, idy), wy);
        float vzs = 0.f;
        if (kZ) vzs = stz[slot];
#pragma unroll
        for (int a = 0; a < A1 - A0; ++a) {
            const float tx = rmul(q4.z, wx[A0 + a]), ty = rmul(q4.w, wx[A0 + a]);
            float tz = 0.f;
            if (kZ) tz = rmul(vzs, wx[A0 + a]);
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                float wh, ws;
                acc.scaled(wy[b], wh, ws);
                int hx, lx, hy, ly;
                AccFix::split2(tx, wh, ws, hx, lx);
                AccFix::split2(ty, wh, ws, hy, ly);
                rs.s[a][b][0] += lx;
                rs.s[a][b][1] += ly;
                rs.s[a][b][2] += hx;
                rs.s[a][b][3] += hy;
                if constexpr (kZ) {
                    int hz, lz;
                    AccFix::split2(tz, wh, ws, hz, lz);
                    rs.s[a][b][4] += lz;
                    rs.s[a][b][5] += hz;
                }
            }
        }
    }
    if (cur >= 0) rs.flush(racc + cur + A0 * ry, ry, R);
}

// Gather of the eight fields at (xi, yj) (cell units) from the region staged in shared
// memory (sf: [rx][ry] nodes of two float4), or from the global fields F when the stencil
// leaves the region; the node order and roundings of k_gather_push.
template <int P>
__device__ __forceinline__ void gather_region(const GeomT<float>& g, const float4* sf,
                                              const float2* __restrict__ F, int bi, int bj,
                                              int rx, int ry, float xi, float yj, float* f) {
    float wx[P + 1], wy[P + 1];
    const int ix = wrap_idx(Shape<P, float>::weights(xi, wx), g.nx);
    const int iy = wrap_idx(Shape<P, float>::weights(yj, wy), g.ny);
    int ri0 = ix - bi, rj0 = iy - bj;
    if (ri0 < 0) ri0 += g.nx;
    if (rj0 < 0) rj0 += g.ny;
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] = 0.f;
    if (ri0 + P < rx && rj0 + P < ry) {
        const float4* row = sf + 2 * (ri0 * ry + rj0);
#pragma unroll
        for (int a = 0; a <= P; ++a) {
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                const float4 u = row[2 * b], v = row[2 * b + 1];
                const float gv[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
                gather_node(rmul(wx[a], wy[b]), gv, f);
            }
            row += 2 * ry;
        }
    } else {
#pragma unroll 1
        for (int a = 0; a <= P; ++a) {
            const int gi = wrap_idx(ix + a, g.nx);
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                const int gj = wrap_idx(iy + b, g.ny);
                float gv[8];
                load_node(F + ((size_t)gi * g.ny + gj) * 4, gv);
                gather_node(rmul(wx[a], wy[b]), gv, f);
            }
        }
    }
}

// Stencil base node (first node with a nonzero weight) of a position in cell units: the
// node Shape<P>::weights returns.
template <int P>
__device__ __forceinline__ int stencil_base(float xi) {
    if constexpr (P % 2 == 0) return (int)floor(radd(xi, 0.5f)) - P / 2;
    return (int)floor(xi) - (P - 1) / 2;
}

template <int P, bool kFused, bool kSpecies, bool kZ>
__global__ void __launch_bounds__(kThreads, 4)
k_deposit_binned(GeomT<float> g, PushT<float> pp, TileGeom tg, const float* __restrict__ x,
                 const float* __restrict__ y, float* __restrict__ xo, float* __restrict__ yo,
                 float* __restrict__ px, float* __restrict__ py,
                 const float* __restrict__ vx, const float* __restrict__ vy,
                 float* __restrict__ vxo, float* __restrict__ vyo, const int* __restrict__ off,
                 int nsplit, const float2* __restrict__ F, AccFix acc,
                 double* __restrict__ diag, unsigned int* __restrict__ err,
                 const int32_t* __restrict__ sp, BinSpecies bs, const float* __restrict__ vz,
                 AccFix accz, int cap) {
    static_assert(!(kZ && kFused), "2D-3V runs the binned deposit on its own");
    constexpr int NF = kFused ? 8 : (kZ ? 5 : 4);  // values loaded per particle
    constexpr int NQ = kZ ? 6 : 4;                 // region planes
    extern __shared__ float4 bin_smem[];
    __shared__ int wsum[33];
    const BinLayout L = bin_layout(tg, P, kFused, kZ, cap);
    char* base = reinterpret_cast<char*>(bin_smem);
    float4* stage = bin_smem;
    const float4* sf = reinterpret_cast<const float4*>(base + L.fields);
    int* kr = reinterpret_cast<int*>(base + L.kr);
    uint16_t* sidx = reinterpret_cast<uint16_t*>(base + L.idx);
    int* racc = reinterpret_cast<int*>(base + L.racc);
    int* cnt = reinterpret_cast<int*>(base + L.cnt);
    float* stz = reinterpret_cast<float*>(base + L.stz);

    const int tt = tg.t * tg.t;
    const int tile = blockIdx.x / nsplit, split = blockIdx.x - tile * nsplit;
    const int64_t t0 = off[tile * tt], tcnt = (int64_t)off[(tile + 1) * tt] - t0;
    const int64_t p0 = t0 + tcnt * split / nsplit, p1 = t0 + tcnt * (split + 1) / nsplit;
    if (p0 == p1) return;  // uniform for the CTA
    const int rx = tg.rx, ry = tg.ry, R = rx * ry;
    if (threadIdx.x < NF) {  // the CTA's particles come to L2 meanwhile
        const float* arr[8] = {x, y, vx, vy, kZ ? vz : px, py, vxo, vyo};
        prefetch_l2(arr[threadIdx.x] + p0, (size_t)(p1 - p0) * sizeof(float));
    }
    for (int k = threadIdx.x; k < NQ * R; k += kThreads) racc[k] = 0;
    for (int k = threadIdx.x; k <= R; k += kThreads) cnt[k] = 0;
    const int tx = tile / tg.nty, ty = tile - tx * tg.nty;
    // region origin, reduced into [0, n): then gi - bi lies in (-n, n) and bi + ri in
    // [0, 2n), so one correction wraps each exactly (whatever the halo)
    int bi = (tx * tg.t - tg.halo) % g.nx, bj = (ty * tg.t - tg.halo) % g.ny;
    if (bi < 0) bi += g.nx;
    if (bj < 0) bj += g.ny;
    griddep_wait();  // particles, fields and J come from the previous operations
    griddep_launch();
    if (kFused) {
        float4* sfw = reinterpret_cast<float4*>(base + L.fields);
        const float4* F4 = reinterpret_cast<const float4*>(F);
        for (int k = threadIdx.x; k < 2 * R; k += kThreads) {
            const int node = k >> 1;
            const int ri = node / ry, rj = node - ri * ry;
            int gi = bi + ri, gj = bj + rj;
            if (gi >= g.nx) gi -= g.nx;
            if (gj >= g.ny) gj -= g.ny;
            sfw[k] = __ldg(F4 + ((size_t)gi * g.ny + gj) * 2 + (k & 1));
        }
    }
    __syncthreads();
    const float dt = g.dt, lx = g.lx, ly = g.ly, idx_ = g.inv_dx, idy = g.inv_dy;
    // per-thread segment of the region's nodes for the scan
    const int seg = (R + kThreads - 1) / kThreads;
    const int c0 = min(R, (int)threadIdx.x * seg), c1 = min(R, c0 + seg);
    // the slice of the binned particles this thread deposits: 33 is odd, so t -> 33 t mod
    // kThreads is a permutation, and the lanes of a warp take slices 33 apart
    const int slice = (33 * (int)threadIdx.x) & (kThreads - 1);
    double kin = 0.0;
    unsigned bad = 0;
    const int64_t nbat = (p1 - p0 + cap - 1) / cap;
    for (int64_t bq = 0; bq < nbat; ++bq) {
        const int64_t b0 = p0 + (p1 - p0) * bq / nbat;
        const int nb = (int)(p0 + (p1 - p0) * (bq + 1) / nbat - b0);
        // A: (gather + push,) move, stage and count; without the gather, the next particle's
        // loads are in flight meanwhile (the fused kernel keeps its registers for the gather)
        constexpr bool kAhead = !kFused;
        float cur[NF], nxt[NF];
        auto load = [&](float* r, int i) {
            if (i < nb) {
                const int64_t p = b0 + i;
                r[0] = x[p];
                r[1] = y[p];
                r[2] = vx[p];
                r[3] = vy[p];
                if (kFused) {
                    r[4] = px[p];
                    r[5] = py[p];
                    r[6] = vxo[p];
                    r[7] = vyo[p];
                } else if (kZ) {
                    r[NF - 1] = vz[p];
                }
            }
        };
        if (kAhead) load(cur, threadIdx.x);
#pragma unroll 1
        for (int i = threadIdx.x; i < nb; i += kThreads) {
            if (kAhead) {
                load(nxt, i + kThreads);
            } else {
                load(cur, i);
            }
            const int64_t p = b0 + i;
            float xs = cur[0], ys = cur[1], vxs = cur[2], vys = cur[3];
            int key = -1;
            bool ok = true;
            int sidx_p = 0;  // the particle's species (kSpecies)
            if (kSpecies) {
                sidx_p = sp[p];
                if ((unsigned)sidx_p >= (unsigned)bs.n) {
                    bad |= ERR_NONFINITE;
                    ok = false;
                }
            }
            if (kFused && ok) {
                const float xi = rmul(xs, idx_), yj = rmul(ys, idy);
                if (!in_domain(xi, g.nx) || !in_domain(yj, g.ny)) {
                    bad |= ERR_NONFINITE;
                    ok = false;
                } else {
                    float f[8];
                    gather_region<P>(g, sf, F, bi, bj, rx, ry, xi, yj, f);
                    float Px, Py;
                    if (kSpecies) {  // the species' charge and mass, its weight on the energy
                        PushT<float> ps = pp;
                        ps.q = bs.q[sidx_p];
                        ps.qdt = bs.qdt[sidx_p];
                        ps.mc2 = bs.mc2[sidx_p];
                        ps.m = bs.m[sidx_p];
                        double ks = 0.0;
                        push_core(ps, f, cur[4], cur[5], cur[2], cur[3], cur[6], cur[7], bad, ks,
                                  Px, Py, vxs, vys);
                        kin += bs.w[sidx_p] * ks;
                    } else {
                        push_core(pp, f, cur[4], cur[5], cur[2], cur[3], cur[6], cur[7], bad,
                                  kin, Px, Py, vxs, vys);
                    }
                    px[p] = Px;
                    py[p] = Py;
                    vxo[p] = vxs;
                    vyo[p] = vys;
                }
            }
            if (ok) {
                xs = move_pos(xs, vxs, dt, lx);
                ys = move_pos(ys, vys, dt, ly);
                xo[p] = xs;
                yo[p] = ys;
                float vzs = kZ ? cur[NF - 1] : 0.f;
                if (kSpecies) {  // each contribution carries the particle's q_s w_s
                    vxs = rmul(vxs, bs.qw[sidx_p]);
                    vys = rmul(vys, bs.qw[sidx_p]);
                    if (kZ) vzs = rmul(vzs, bs.qw[sidx_p]);
                }
                if (kZ) stz[i] = vzs;
                const float xi = rmul(xs, idx_), yj = rmul(ys, idy);
                if (!in_domain(xi, g.nx) || !in_domain(yj, g.ny)) {
                    bad |= ERR_NONFINITE;
                } else {
                    const int ix = wrap_idx(stencil_base<P>(xi), g.nx);
                    const int iy = wrap_idx(stencil_base<P>(yj), g.ny);
                    int ri0 = ix - bi, rj0 = iy - bj;
                    if (ri0 < 0) ri0 += g.nx;
                    if (rj0 < 0) rj0 += g.ny;
                    if (ri0 + P < rx && rj0 + P < ry) {
                        key = ri0 * ry + rj0;
                    } else {  // beyond the region: straight to the global grid
                        float wx[P + 1], wy[P + 1];
                        Shape<P, float>::weights(xi, wx);
                        Shape<P, float>::weights(yj, wy);
#pragma unroll 1
                        for (int a = 0; a <= P; ++a) {
                            const int gi = wrap_idx(ix + a, g.nx);
                            const float tx_ = rmul(vxs, wx[a]), ty_ = rmul(vys, wx[a]);
#pragma unroll
                            for (int b = 0; b <= P; ++b)
                                acc.add2((size_t)gi * g.ny + wrap_idx(iy + b, g.ny), tx_, ty_,
                                         wy[b]);
                            if (kZ) {
                                const float tz_ = rmul(vzs, wx[a]);
#pragma unroll
                                for (int b = 0; b <= P; ++b)
                                    accz.add1f((size_t)gi * g.ny + wrap_idx(iy + b, g.ny), tz_,
                                               wy[b]);
                            }
                        }
                    }
                }
            }
            if (key >= 0) {
                stage[i] = make_float4(xs, ys, vxs, vys);
                kr[i] = key | (atomicAdd(cnt + key, 1) << 16);
            } else {
                kr[i] = -1;
            }
            if (kAhead) {
#pragma unroll
                for (int q = 0; q < NF; ++q) cur[q] = nxt[q];
            }
        }
        __syncthreads();
        // B: exclusive scan of the counts over the region's nodes
        int local = 0;
        for (int c = c0; c < c1; ++c) local += cnt[c];
        int total;
        int run = cta_exclusive_scan(local, wsum, &total);
        for (int c = c0; c < c1; ++c) {
            const int v = cnt[c];
            cnt[c] = run;
            run += v;
        }
        __syncthreads();
        // C: binned order of the staging slots
        for (int i = threadIdx.x; i < nb; i += kThreads) {
            const int k = kr[i];
            if (k >= 0) sidx[cnt[k & 0xFFFF] + (k >> 16)] = (uint16_t)i;
        }
        __syncthreads();
        // D: equal slices of the binned particles, summed in registers per key
        {
            const int per = (total + kThreads - 1) / kThreads;
            const int k0 = min(total, slice * per), k1 = min(total, k0 + per);
            if constexpr (kZ) {  // six planes: one stencil row a pass
                bin_slice_rows<P, 0, 1, true>(stage, kr, sidx, k0, k1, idx_, idy, acc, racc, ry, R, stz);
                bin_slice_rows<P, 1, 2, true>(stage, kr, sidx, k0, k1, idx_, idy, acc, racc, ry, R, stz);
                bin_slice_rows<P, 2, 3, true>(stage, kr, sidx, k0, k1, idx_, idy, acc, racc, ry, R, stz);
                if constexpr (P >= 3)
                    bin_slice_rows<P, 3, 4, true>(stage, kr, sidx, k0, k1, idx_, idy, acc, racc, ry, R, stz);
                if constexpr (P == 4)
                    bin_slice_rows<P, 4, 5, true>(stage, kr, sidx, k0, k1, idx_, idy, acc, racc, ry, R, stz);
            } else if constexpr (P == 2) {
                bin_slice_rows<P, 0, 3>(stage, kr, sidx, k0, k1, idx_, idy, acc, racc, ry, R);
            } else {
                bin_slice_rows<P, 0, 2>(stage, kr, sidx, k0, k1, idx_, idy, acc, racc, ry, R);
                bin_slice_rows<P, 2, 4>(stage, kr, sidx, k0, k1, idx_, idy, acc, racc, ry, R);
                if constexpr (P == 4)
                    bin_slice_rows<P, 4, 5>(stage, kr, sidx, k0, k1, idx_, idy, acc, racc, ry, R);
            }
        }
        __syncthreads();
        // the batch's region sums to the global grid; counts cleared for the next batch
        for (int k = threadIdx.x; k < R; k += kThreads) {
            const int lx_ = racc[k], ly_ = racc[R + k];
            const int hx = racc[2 * R + k], hy = racc[3 * R + k];
            int lz = 0, hz = 0;
            if (kZ) {
                lz = racc[4 * R + k];
                hz = racc[5 * R + k];
            }
            if (!(lx_ | ly_ | hx | hy | lz | hz)) continue;
            racc[k] = racc[R + k] = racc[2 * R + k] = racc[3 * R + k] = 0;
            if (kZ) racc[4 * R + k] = racc[5 * R + k] = 0;
            const int ri = k / ry, rj = k - ri * ry;
            int gi = bi + ri, gj = bj + rj;
            if (gi >= g.nx) gi -= g.nx;
            if (gj >= g.ny) gj -= g.ny;
            const size_t node = (size_t)gi * g.ny + gj;
            const long long sx = (long long)hx * (1ll << kLoBits) + (long long)lx_;
            const long long sy = (long long)hy * (1ll << kLoBits) + (long long)ly_;
            if (sx) atomicAdd(reinterpret_cast<unsigned long long*>(&acc.J[node].x), (unsigned long long)sx);
            if (sy) atomicAdd(reinterpret_cast<unsigned long long*>(&acc.J[node].y), (unsigned long long)sy);
            if (kZ) {
                const long long sz = (long long)hz * (1ll << kLoBits) + (long long)lz;
                if (sz) atomicAdd(reinterpret_cast<unsigned long long*>(&accz.J[node].x), (unsigned long long)sz);
            }
        }
        for (int k = threadIdx.x; k <= R; k += kThreads) cnt[k] = 0;
        __syncthreads();
    }
    if (kFused) {
        push_finish(pp, bad, kin, diag, err);
    } else if (bad) {
        atomicOr(err, bad);
    }
}

template <typename T, int P>
__global__ void __launch_bounds__(kThreads)
k_init_particles(ParticleGeom g, PushParams pp, T* __restrict__ x, T* __restrict__ y,
                 T* __restrict__ px, T* __restrict__ py, const T* __restrict__ vx,
                 const T* __restrict__ vy, T* __restrict__ vxo, T* __restrict__ vyo, int64_t n,
                 const cplx_t<T>* __restrict__ E, unsigned int* __restrict__ err) {
    using C = cplx_t<T>;
    const T idx_ = (T)g.inv_dx, idy = (T)g.inv_dy;
    const double c2 = pp.c * pp.c;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const T xi = rmul(x[p], idx_), yj = rmul(y[p], idy);
        const double vxn = (double)vx[p], vyn = (double)vy[p];
        const double v2 = vxn * vxn + vyn * vyn;
        if (!in_domain(xi, g.nx) || !in_domain(yj, g.ny) || !(v2 < c2)) {
            atomicOr(err, (unsigned)ERR_NONFINITE);
            continue;
        }
        T wx[P + 1], wy[P + 1];
        const int ix = Shape<P, T>::weights(xi, wx);
        const int iy = Shape<P, T>::weights(yj, wy);
        T ex = 0, ey = 0;
#pragma unroll
        for (int a = 0; a <= P; ++a) {
            const int gi = wrap_idx(ix + a, g.nx);
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                const int gj = wrap_idx(iy + b, g.ny);
                const C e = E[(size_t)gi * g.ny + gj];
                const T w = wx[a] * wy[b];
                ex += w * e.x;
                ey += w * e.y;
            }
        }
        const double gamma = 1.0 / sqrt(1.0 - v2 / c2);
        px[p] = (T)(gamma * pp.m * vxn);
        py[p] = (T)(gamma * pp.m * vyn);
        // Taylor step back: d v/dt = (q/(gamma m)) (E - v (v.E)/c^2)
        const double coef = pp.dt * pp.q / (gamma * pp.m);
        const double vdote = vxn * (double)ex + vyn * (double)ey;
        vxo[p] = (T)(vxn - coef * ((double)ex - vxn * vdote / c2));
        vyo[p] = (T)(vyn - coef * ((double)ey - vyn * vdote / c2));
    }
}

template <typename T>
__global__ void k_wrap_positions(T* __restrict__ x, T* __restrict__ y, int64_t n, T lx, T ly) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        x[p] = wrap_pos(x[p], lx);
        y[p] = wrap_pos(y[p], ly);
    }
}

template <typename Ts, typename Td>
__global__ void k_convert(const Ts* __restrict__ s, Td* __restrict__ d, int64_t n) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        d[p] = (Td)s[p];
}

template <typename T>
__global__ void k_scatter_by_id(const T* __restrict__ s, const int32_t* __restrict__ id,
                                double* __restrict__ d, int64_t n) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        int32_t k = id[p];
        if (k >= 0 && k < n) d[k] = (double)s[p];
    }
}

// Replay of one FP64 step's particle update from the adjoint's record of that step:
// state n -> state n+1 with the move of k_move_deposit (the same operations, so the same
// bits) and the recorded P^{n+1}, v^{n+1}.  States are eight arrays of n in the order x, y,
// Px, Py, v^n (x, y), v^{n-1} (x, y); rec is the step's record (P^{n+1}, v^{n+1} first).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_replay_step(GeomT<T> g, const T* __restrict__ s0, T* __restrict__ s1,
              const double* __restrict__ rec, int64_t n) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const T vxi = s0[4 * n + p], vyi = s0[5 * n + p];
        s1[p] = move_pos(s0[p], vxi, g.dt, g.lx);
        s1[n + p] = move_pos(s0[n + p], vyi, g.dt, g.ly);
        s1[2 * n + p] = (T)rec[p];
        s1[3 * n + p] = (T)rec[n + p];
        s1[4 * n + p] = (T)rec[2 * n + p];
        s1[5 * n + p] = (T)rec[3 * n + p];
        s1[6 * n + p] = vxi;
        s1[7 * n + p] = vyi;
    }
}

// ------------------------------------------------------------ 2D-3V, species ----
//
// Section 2.2 writes the particle equations with three-component P and A and each
// particle's own charge and mass.  On the plane d/dz = 0: J_z is deposited like J_x, A_z
// gathered with its in-plane gradient, (grad A . v*)_l gains d_l A_z v*_z for l = x, y,
// P_z is constant, and u = P - q A has three components.

// J_z of the moved particles (after the move of k_move_deposit): x^{n+1}, v_z^n.
template <typename T, int P, typename Acc>
__global__ void __launch_bounds__(kThreads)
k_deposit_z(GeomT<T> g, const T* __restrict__ x, const T* __restrict__ y,
            const T* __restrict__ vz, int64_t n, const int32_t* __restrict__ sp, SpeciesT<T> spt,
            Acc acc, unsigned int* __restrict__ err) {
    const T idx_ = g.inv_dx, idy = g.inv_dy;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const T xi = rmul(x[p], idx_), yj = rmul(y[p], idy);
        T fq;
        if (!in_domain(xi, g.nx) || !in_domain(yj, g.ny) || !species_factor(sp, spt, p, fq)) {
            atomicOr(err, (unsigned)ERR_NONFINITE);
            continue;
        }
        T wx[P + 1], wy[P + 1];
        const int ix = Shape<P, T>::weights(xi, wx);
        const int iy = Shape<P, T>::weights(yj, wy);
        const T vzi = acc.pre(sp ? rmul(vz[p], fq) : vz[p]);
#pragma unroll
        for (int a = 0; a <= P; ++a) {
            const size_t row = (size_t)wrap_idx(ix + a, g.nx) * g.ny;
            const T tz = rmul(vzi, wx[a]);
#pragma unroll
            for (int b = 0; b <= P; ++b) acc.add1f(row + wrap_idx(iy + b, g.ny), tz, wy[b]);
        }
    }
}

// Species constants of particle p in the storage precision (the table's, or the single
// species' q, m, weight).
template <typename T>
struct PushConst {
    T q, qdt, mc2;
    double qd, m, w;
};
template <typename T>
__device__ __forceinline__ bool push_const(const PushParams& pp, const int32_t* __restrict__ sp,
                                           const SpeciesParams& spp, int64_t p, PushConst<T>& k) {
    double q = pp.q, m = pp.m, w = pp.weight;
    if (sp) {
        const int s = sp[p];
        if ((unsigned)s >= (unsigned)spp.n) return false;
        q = spp.q[s];
        m = spp.m[s];
        w = spp.w[s];
    }
    k.q = (T)q;
    k.qdt = (T)(q * pp.dt);
    k.mc2 = (T)(m * pp.c * pp.c);
    k.qd = q;
    k.m = m;
    k.w = w;
    return true;
}

template <typename T, int P, bool Z3>
__global__ void __launch_bounds__(kThreads)
k_gather_push3(GeomT<T> g, PushParams pp, const T* __restrict__ x, const T* __restrict__ y,
               T* __restrict__ px, T* __restrict__ py, const T* __restrict__ pz,
               const T* __restrict__ vx, const T* __restrict__ vy, const T* __restrict__ vz,
               T* __restrict__ vxo, T* __restrict__ vyo, T* __restrict__ vzo,
               const int32_t* __restrict__ sp, SpeciesParams spp, int64_t n,
               const cplx_t<T>* __restrict__ F, const cplx_t<T>* __restrict__ Fz,
               double* __restrict__ diag, unsigned int* __restrict__ err) {
    using C = cplx_t<T>;
    const T idx_ = g.inv_dx, idy = g.inv_dy, c2 = (T)(pp.c * pp.c);
    double kin = 0.0;
    unsigned bad = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const T xi = rmul(x[p], idx_), yj = rmul(y[p], idy);
        PushConst<T> k;
        if (!in_domain(xi, g.nx) || !in_domain(yj, g.ny) || !push_const(pp, sp, spp, p, k)) {
            bad |= ERR_NONFINITE;
            continue;
        }
        T wx[P + 1], wy[P + 1];
        const int ix = Shape<P, T>::weights(xi, wx);
        const int iy = Shape<P, T>::weights(yj, wy);
        T f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        T fz[3] = {0, 0, 0};  // dAz/dx, dAz/dy, Az
#pragma unroll
        for (int a = 0; a <= P; ++a) {
            const size_t row = (size_t)wrap_idx(ix + a, g.nx) * g.ny;
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                const size_t nd = row + wrap_idx(iy + b, g.ny);
                T gv[8];
                load_node(F + nd * 4, gv);
                const T w = rmul(wx[a], wy[b]);
                gather_node(w, gv, f);
                if (Z3) {
                    const C z0 = Fz[nd * 2], z1 = Fz[nd * 2 + 1];
                    fz[0] = rfma(w, z0.x, fz[0]);
                    fz[1] = rfma(w, z0.y, fz[1]);
                    fz[2] = rfma(w, z1.x, fz[2]);
                }
            }
        }
        const T vsx = rfma((T)2, vx[p], -vxo[p]);
        const T vsy = rfma((T)2, vy[p], -vyo[p]);
        T fx = rfma(f[6], vsy, rfma(f[4], vsx, -f[0]));
        T fy = rfma(f[7], vsy, rfma(f[5], vsx, -f[1]));
        T vsz = (T)0;
        if (Z3) {
            vsz = rfma((T)2, vz[p], -vzo[p]);
            fx = rfma(fz[0], vsz, fx);
            fy = rfma(fz[1], vsz, fy);
        }
        const T Px = rfma(k.qdt, fx, px[p]);
        const T Py = rfma(k.qdt, fy, py[p]);
        const T ux = rfma(-k.q, f[2], Px), uy = rfma(-k.q, f[3], Py);
        T u2 = rfma(ux, ux, rmul(uy, uy));
        T uz = (T)0;
        if (Z3) {
            uz = rfma(-k.q, fz[2], pz[p]);
            u2 = rfma(uz, uz, u2);
        }
        const T den = rsqrt_rn(rfma(c2, u2, rmul(k.mc2, k.mc2)));
        const T rc = rdiv(c2, den);
        const T vxn1 = rmul(rc, ux), vyn1 = rmul(rc, uy);
        px[p] = Px;
        py[p] = Py;
        vxo[p] = vxn1;
        vyo[p] = vyn1;
        if (Z3) vzo[p] = rmul(rc, uz);
        if (!isfinite(vxn1) || !isfinite(vyn1)) bad |= ERR_NONFINITE;
        if (pp.diag) kin += k.w * kinetic(c2, k.mc2, pp.c, k.m, u2);  // w m c^2 (gamma - 1)
    }
    if (bad) atomicOr(err, bad);
    if (pp.diag) {
        for (int o = 16; o > 0; o >>= 1) kin += __shfl_down_sync(0xffffffffu, kin, o);
        if ((threadIdx.x & 31) == 0 && kin != 0.0) atomicAdd(diag + D_KIN, kin);
    }
}

// t = 0 with species and/or three velocity components: P^0 = gamma m_s v^0 and the Taylor
// start v^{-1} = v^0 - kappa (E - v (v . E)/c^2), kappa = dt q_s/(gamma m_s), E = (Ex, Ey, 0).
template <typename T, int P>
__global__ void __launch_bounds__(kThreads)
k_init_particles3(ParticleGeom g, PushParams pp, T* __restrict__ x, T* __restrict__ y,
                  T* __restrict__ px, T* __restrict__ py, T* __restrict__ pz,
                  const T* __restrict__ vx, const T* __restrict__ vy, const T* __restrict__ vz,
                  T* __restrict__ vxo, T* __restrict__ vyo, T* __restrict__ vzo,
                  const int32_t* __restrict__ sp, SpeciesParams spp, int64_t n,
                  const cplx_t<T>* __restrict__ E, unsigned int* __restrict__ err) {
    using C = cplx_t<T>;
    const T idx_ = (T)g.inv_dx, idy = (T)g.inv_dy;
    const double c2 = pp.c * pp.c;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const T xi = rmul(x[p], idx_), yj = rmul(y[p], idy);
        const double vxn = (double)vx[p], vyn = (double)vy[p], vzn = vz ? (double)vz[p] : 0.0;
        const double v2 = vxn * vxn + vyn * vyn + vzn * vzn;
        PushConst<T> k;
        if (!in_domain(xi, g.nx) || !in_domain(yj, g.ny) || !(v2 < c2) ||
            !push_const(pp, sp, spp, p, k)) {
            atomicOr(err, (unsigned)ERR_NONFINITE);
            continue;
        }
        T wx[P + 1], wy[P + 1];
        const int ix = Shape<P, T>::weights(xi, wx);
        const int iy = Shape<P, T>::weights(yj, wy);
        T ex = 0, ey = 0;
#pragma unroll
        for (int a = 0; a <= P; ++a) {
            const int gi = wrap_idx(ix + a, g.nx);
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                const C e = E[(size_t)gi * g.ny + wrap_idx(iy + b, g.ny)];
                const T w = wx[a] * wy[b];
                ex += w * e.x;
                ey += w * e.y;
            }
        }
        const double m = k.m, qs = k.qd;
        const double gamma = 1.0 / sqrt(1.0 - v2 / c2);
        px[p] = (T)(gamma * m * vxn);
        py[p] = (T)(gamma * m * vyn);
        if (vz) pz[p] = (T)(gamma * m * vzn);
        const double coef = pp.dt * qs / (gamma * m);
        const double vdote = vxn * (double)ex + vyn * (double)ey;
        vxo[p] = (T)(vxn - coef * ((double)ex - vxn * vdote / c2));
        vyo[p] = (T)(vyn - coef * ((double)ey - vyn * vdote / c2));
        if (vz) vzo[p] = (T)(vzn + coef * vzn * vdote / c2);
    }
}

template <typename T>
__global__ void k_extract(const cplx_t<T>* __restrict__ src, int stride, int comp, double scale,
                          double* __restrict__ dst, int64_t n) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        cplx_t<T> v = src[p * stride];
        dst[p] = scale * (double)(comp ? v.y : v.x);
    }
}

}  // namespace

#define GPIC_DISPATCH_P(p, KERNEL, ...)                                    \
    switch (p) {                                                           \
        case 2: KERNEL<T, 2><<<blocks_for(n), kThreads, 0, s>>>(__VA_ARGS__); break; \
        case 3: KERNEL<T, 3><<<blocks_for(n), kThreads, 0, s>>>(__VA_ARGS__); break; \
        case 4: KERNEL<T, 4><<<blocks_for(n), kThreads, 0, s>>>(__VA_ARGS__); break; \
        default: return cudaErrorInvalidValue;                             \
    }

#define GPIC_DISPATCH_PA(p, KERNEL, ACC, ...)                                               \
    switch (p) {                                                                           \
        case 2: KERNEL<T, 2, ACC><<<blocks_for(n), kThreads, 0, s>>>(__VA_ARGS__); break; \
        case 3: KERNEL<T, 3, ACC><<<blocks_for(n), kThreads, 0, s>>>(__VA_ARGS__); break; \
        case 4: KERNEL<T, 4, ACC><<<blocks_for(n), kThreads, 0, s>>>(__VA_ARGS__); break; \
        default: return cudaErrorInvalidValue;                                             \
    }

template <typename T>
cudaError_t launch_move_deposit(int p, const ParticleGeom& g, T* x, T* y, const T* vx,
                                const T* vy, int64_t n, double2* j, unsigned int* err,
                                cudaStream_t s, const int32_t* sp, const SpeciesParams* spp) {
    if (n == 0) return cudaSuccess;
    GPIC_DISPATCH_PA(p, k_move_deposit, AccF64, typed<T>(g), x, y, vx, vy, n, AccF64{j}, err,
                     sp, typed_species<T>(spp))
    return cudaGetLastError();
}

cudaError_t launch_move_deposit_fix128(int p, const ParticleGeom& g, double* x, double* y,
                                       const double* vx, const double* vy, int64_t n,
                                       longlong2* j, size_t ng, double scale, unsigned int* err,
                                       cudaStream_t s, const int32_t* sp,
                                       const SpeciesParams* spp) {
    using T = double;
    if (n == 0) return cudaSuccess;
    GPIC_DISPATCH_PA(p, k_move_deposit, AccFix128, typed<T>(g), x, y, vx, vy, n,
                     (AccFix128{j, ng, scale}), err, sp, typed_species<T>(spp))
    return cudaGetLastError();
}

cudaError_t launch_deposit_charge_fix128(int p, const ParticleGeom& g, const double* x,
                                         const double* y, int64_t n, longlong2* j, size_t ng,
                                         double scale, unsigned int* err, cudaStream_t s,
                                         const int32_t* sp, const SpeciesParams* spp) {
    using T = double;
    if (n == 0) return cudaSuccess;
    GPIC_DISPATCH_PA(p, k_deposit_charge, AccFix128, g, x, y, n, (AccFix128{j, ng, scale}), err,
                     sp, typed_species<T>(spp))
    return cudaGetLastError();
}

cudaError_t launch_fix128_to_cplx(const longlong2* j, size_t ng, double unscale, double2* out,
                                  cudaStream_t s) {
    k_fix128_to_cplx<<<blocks_for((int64_t)ng), kThreads, 0, s>>>(j, ng, unscale, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_deposit_charge(int p, const ParticleGeom& g, const T* x, const T* y, int64_t n,
                                  double2* j, unsigned int* err, cudaStream_t s,
                                  const int32_t* sp, const SpeciesParams* spp) {
    if (n == 0) return cudaSuccess;
    GPIC_DISPATCH_PA(p, k_deposit_charge, AccF64, g, x, y, n, AccF64{j}, err, sp,
                     typed_species<T>(spp))
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_move_deposit_fix(int p, const ParticleGeom& g, T* x, T* y, const T* vx,
                                    const T* vy, int64_t n, longlong2* j, float scale,
                                    unsigned int* err, cudaStream_t s, const int32_t* sp,
                                    const SpeciesParams* spp) {
    if (n == 0) return cudaSuccess;
    GPIC_DISPATCH_PA(p, k_move_deposit, AccFix, typed<T>(g), x, y, vx, vy, n, (AccFix::make(j, scale)),
                     err, sp, typed_species<T>(spp))
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_deposit_charge_fix(int p, const ParticleGeom& g, const T* x, const T* y,
                                      int64_t n, longlong2* j, float scale, unsigned int* err,
                                      cudaStream_t s, const int32_t* sp, const SpeciesParams* spp) {
    if (n == 0) return cudaSuccess;
    GPIC_DISPATCH_PA(p, k_deposit_charge, AccFix, g, x, y, n, (AccFix::make(j, scale)), err, sp,
                     typed_species<T>(spp))
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_replay_step(const ParticleGeom& g, const T* s0, T* s1, const double* rec,
                               int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_replay_step<T><<<blocks_for(n), kThreads, 0, s>>>(typed<T>(g), s0, s1, rec, n);
    return cudaGetLastError();
}
template cudaError_t launch_replay_step<double>(const ParticleGeom&, const double*, double*,
                                                const double*, int64_t, cudaStream_t);
template cudaError_t launch_replay_step<float>(const ParticleGeom&, const float*, float*,
                                               const double*, int64_t, cudaStream_t);

template <typename T>
cudaError_t launch_deposit_z(int p, const ParticleGeom& g, const T* x, const T* y, const T* vz,
                             int64_t n, const int32_t* sp, const SpeciesParams& spp, void* jz,
                             size_t ng, double scale, unsigned int* err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int32_t* spi = spp.n > 0 ? sp : nullptr;
    if constexpr (sizeof(T) == 4) {
        GPIC_DISPATCH_PA(p, k_deposit_z, AccFix, typed<T>(g), x, y, vz, n, spi,
                         typed_species<T>(&spp), (AccFix::make(jz, (float)scale)), err)
    } else {
        GPIC_DISPATCH_PA(p, k_deposit_z, AccFix128, typed<T>(g), x, y, vz, n, spi,
                         typed_species<T>(&spp), (AccFix128{(longlong2*)jz, ng, scale}), err)
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather_push3(int p, const ParticleGeom& g, const PushParams& pp, const T* x,
                                const T* y, T* px, T* py, const T* pz, const T* vx, const T* vy,
                                const T* vz, T* vx_old, T* vy_old, T* vz_old, const int32_t* sp,
                                const SpeciesParams& spp, int64_t n, const void* fields4,
                                const void* fz, double* diag, unsigned int* err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    using C = cplx_t<T>;
    const int32_t* spi = spp.n > 0 ? sp : nullptr;
    const bool z3 = vz != nullptr;
#define GPIC_GP3(PP)                                                                           \
    if (z3)                                                                                    \
        k_gather_push3<T, PP, true><<<blocks_for(n), kThreads, 0, s>>>(                        \
            typed<T>(g), pp, x, y, px, py, pz, vx, vy, vz, vx_old, vy_old, vz_old, spi, spp, n, \
            (const C*)fields4, (const C*)fz, diag, err);                                       \
    else                                                                                       \
        k_gather_push3<T, PP, false><<<blocks_for(n), kThreads, 0, s>>>(                       \
            typed<T>(g), pp, x, y, px, py, pz, vx, vy, vz, vx_old, vy_old, vz_old, spi, spp, n, \
            (const C*)fields4, (const C*)fz, diag, err);
    switch (p) {
        case 2: GPIC_GP3(2) break;
        case 3: GPIC_GP3(3) break;
        case 4: GPIC_GP3(4) break;
        default: return cudaErrorInvalidValue;
    }
#undef GPIC_GP3
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_particles3(int p, const ParticleGeom& g, const PushParams& pp, T* x, T* y,
                                   T* px, T* py, T* pz, const T* vx, const T* vy, const T* vz,
                                   T* vx_old, T* vy_old, T* vz_old, const int32_t* sp,
                                   const SpeciesParams& spp, int64_t n, const void* e2,
                                   unsigned int* err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int32_t* spi = spp.n > 0 ? sp : nullptr;
    GPIC_DISPATCH_P(p, k_init_particles3, g, pp, x, y, px, py, pz, vx, vy, vz, vx_old, vy_old,
                    vz_old, spi, spp, n, (const cplx_t<T>*)e2, err)
    return cudaGetLastError();
}


template <typename T>
cudaError_t launch_fix_to_cplx(const longlong2* j, double unscale, void* out, int64_t n,
                               cudaStream_t s) {
    k_fix_to_cplx<T><<<blocks_for(n), kThreads, 0, s>>>(j, unscale, (cplx_t<T>*)out, n);
    return cudaGetLastError();
}

cudaError_t launch_extract_fix(const longlong2* j, int comp, double scale, double* dst, int64_t n,
                               cudaStream_t s) {
    k_extract_fix<<<blocks_for(n), kThreads, 0, s>>>(j, comp, scale, dst, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather_push(int p, const ParticleGeom& g, const PushParams& pp, const T* x,
                               const T* y, T* px, T* py, const T* vx, const T* vy, T* vxo,
                               T* vyo, int64_t n, const void* f, double* gout, double* diag,
                               unsigned int* err, cudaStream_t s, bool gout_short) {
    if (n == 0) return cudaSuccess;
    GPIC_DISPATCH_P(p, k_gather_push, typed<T>(g), typed<T>(pp), x, y, px, py, vx, vy, vxo, vyo, n,
                    (const cplx_t<T>*)f, gout, gout_short ? 1 : 0, diag, err)
    return cudaGetLastError();
}

cudaError_t launch_gather_push_tiled(int p, const ParticleGeom& g, const PushParams& pp,
                                    const TileGeom& tg, const float* x, const float* y, float* px,
                                    float* py, const float* vx, const float* vy, float* vxo,
                                    float* vyo, int64_t n, const int* off,
                                    const void* f, double* diag, unsigned int* err,
                                    cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    // splits per tile: about 2048 particles per CTA at the mean density (so that a grid of
    // 64-per-cell tiles is a single wave of four CTAs per SM)
    const int ntiles = tg.ntx * tg.nty;
    int nsplit = (int)((n + (int64_t)ntiles * 2048 - 1) / ((int64_t)ntiles * 2048));
    if (nsplit < 1) nsplit = 1;
    if (nsplit > 64) nsplit = 64;
    const int blocks = ntiles * nsplit;
    const size_t smem = (size_t)tg.rx * tg.ry * 2 * sizeof(float4);
    if (smem > 100 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
#define GPIC_GTILED(PP)                                                                        \
    {                                                                                          \
        static const cudaError_t attr = cudaFuncSetAttribute(                                  \
            k_gather_push_tiled<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024); \
        e = attr;                                                                              \
        if (e == cudaSuccess)                                                                  \
            e = launch_pdl(k_gather_push_tiled<PP>, dim3(blocks), dim3(kThreads), smem, s,     \
                           typed<float>(g), typed<float>(pp), tg, x, y, px, py, vx, vy, vxo,   \
                           vyo, off, nsplit, (const float2*)f, diag, err);                     \
    }
    switch (p) {
        case 2: GPIC_GTILED(2) break;
        case 3: GPIC_GTILED(3) break;
        case 4: GPIC_GTILED(4) break;
        default: return cudaErrorInvalidValue;
    }
#undef GPIC_GTILED
    return e;
}

bool deposit_binned_fits(const TileGeom& tg, int p, bool fused, bool z) {
    return tg.rx > p && tg.ry > p && tg.rx * tg.ry < (1 << 16) && !(fused && z) &&
           bin_layout(tg, p, fused, z).bytes <= kBinSmemMax;
}

cudaError_t launch_deposit_binned(int p, const ParticleGeom& g, const PushParams& pp,
                                  const TileGeom& tg, const float* x, const float* y, float* xo,
                                  float* yo, float* px, float* py, const float* vx,
                                  const float* vy, float* vxo, float* vyo, int64_t n,
                                  const int* off, const void* fields4, void* j, float scale,
                                  double* diag, unsigned int* err, cudaStream_t s, bool fused,
                                  int per_cta, const int32_t* sp, const SpeciesParams* spp,
                                  const float* vz, void* jz) {
    if (n == 0) return cudaSuccess;
    const bool z = vz != nullptr;
    if (z && (fused || !jz)) return cudaErrorInvalidValue;
    const bool species = sp && spp && spp->n > 0;
    BinSpecies bs{};
    PushT<float> ptyped = typed<float>(pp);
    if (species) {
        bs.n = spp->n;
        for (int k = 0; k < spp->n; ++k) {
            bs.qw[k] = (float)spp->qw[k];
            bs.q[k] = (float)spp->q[k];
            bs.qdt[k] = (float)(spp->q[k] * pp.dt);
            bs.mc2[k] = (float)(spp->m[k] * pp.c * pp.c);
            bs.m[k] = spp->m[k];
            bs.w[k] = spp->w[k];
        }
        ptyped.weight = 1.0;  // the energy sum carries each particle's w_s already
    }
    if (!deposit_binned_fits(tg, p, fused, z) || per_cta < 1) return cudaErrorInvalidValue;
    const int ntiles = tg.ntx * tg.nty;
    int nsplit = (int)((n + (int64_t)ntiles * per_cta - 1) / ((int64_t)ntiles * per_cta));
    if (nsplit < 1) nsplit = 1;
    if (nsplit > 64) nsplit = 64;
    const int blocks = ntiles * nsplit;
    const AccFix acc = AccFix::make(j, scale);
    const AccFix accz = AccFix::make(jz, scale);
    cudaError_t e = cudaSuccess;
    // the larger batch capacity where the occupancy calculator still puts four CTAs on an
    // SM (shared memory is what limits it), else the smaller one
#define GPIC_BINNED(PP, FF, SS, ZZ)                                                            \
    {                                                                                          \
        static const cudaError_t attr = cudaFuncSetAttribute(                                  \
            k_deposit_binned<PP, FF, SS, ZZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
            kBinSmemMax);                                                                      \
        e = attr;                                                                              \
        int cap = kBinBatchMin, per_sm = 0;                                                    \
        const size_t big = (size_t)bin_layout(tg, p, fused, z, kBinBatchMax).bytes;            \
        if (e == cudaSuccess && big <= (size_t)kBinSmemMax)                                    \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(                                 \
                &per_sm, k_deposit_binned<PP, FF, SS, ZZ>, kThreads, big);                     \
        if (per_sm >= 4) cap = kBinBatchMax;                                                   \
        const size_t smem = (size_t)bin_layout(tg, p, fused, z, cap).bytes;                    \
        if (e == cudaSuccess)                                                                  \
            e = launch_pdl(k_deposit_binned<PP, FF, SS, ZZ>, dim3(blocks), dim3(kThreads),     \
                           smem, s, typed<float>(g), ptyped, tg, x, y, xo, yo, px, py, vx, vy, \
                           vxo, vyo, off, nsplit, (const float2*)fields4, acc, diag, err,      \
                           species ? sp : nullptr, bs, vz, accz, cap);                         \
    }
#define GPIC_BINNED_S(PP, FF)                       \
    if (species && z) GPIC_BINNED(PP, false, true, true) \
    else if (z) GPIC_BINNED(PP, false, false, true)     \
    else if (species) GPIC_BINNED(PP, FF, true, false)  \
    else GPIC_BINNED(PP, FF, false, false)
    switch (p * 2 + (fused ? 1 : 0)) {
        case 4: GPIC_BINNED_S(2, false) break;
        case 5: GPIC_BINNED_S(2, true) break;
        case 6: GPIC_BINNED_S(3, false) break;
        case 7: GPIC_BINNED_S(3, true) break;
        case 8: GPIC_BINNED_S(4, false) break;
        case 9: GPIC_BINNED_S(4, true) break;
        default: return cudaErrorInvalidValue;
    }
#undef GPIC_BINNED_S
#undef GPIC_BINNED
    return e;
}

template <typename T>
cudaError_t launch_init_particles(int p, const ParticleGeom& g, const PushParams& pp, T* x, T* y,
                                  T* px, T* py, const T* vx, const T* vy, T* vxo, T* vyo,
                                  int64_t n, const void* e, unsigned int* err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_wrap_positions<T><<<blocks_for(n), kThreads, 0, s>>>(x, y, n, (T)g.lx, (T)g.ly);
    GPIC_DISPATCH_P(p, k_init_particles, g, pp, x, y, px, py, vx, vy, vxo, vyo, n,
                    (const cplx_t<T>*)e, err)
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_wrap_positions(T* x, T* y, int64_t n, double lx, double ly, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_wrap_positions<T><<<blocks_for(n), kThreads, 0, s>>>(x, y, n, (T)lx, (T)ly);
    return cudaGetLastError();
}

template <typename Ts, typename Td>
cudaError_t launch_convert(const Ts* src, Td* dst, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_convert<Ts, Td><<<blocks_for(n), kThreads, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scatter_by_id(const T* src, const int32_t* id, double* dst, int64_t n,
                                 cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_scatter_by_id<T><<<blocks_for(n), kThreads, 0, s>>>(src, id, dst, n);
    return cudaGetLastError();
}

__global__ void k_scatter_by_id_i32(const int32_t* __restrict__ src, const int32_t* __restrict__ id,
                                    int32_t* __restrict__ dst, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        dst[id[k]] = src[k];
}

cudaError_t launch_scatter_by_id_i32(const int32_t* src, const int32_t* id, int32_t* dst,
                                     int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_scatter_by_id_i32<<<blocks_for(n), kThreads, 0, s>>>(src, id, dst, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_extract(const void* src, int stride, int comp, double scale, double* dst,
                           int64_t n, cudaStream_t s) {
    k_extract<T><<<blocks_for(n), kThreads, 0, s>>>((const cplx_t<T>*)src, stride, comp, scale,
                                                    dst, n);
    return cudaGetLastError();
}

#define GPIC_INST(T)                                                                            \
    template cudaError_t launch_move_deposit<T>(int, const ParticleGeom&, T*, T*, const T*,     \
                                                const T*, int64_t, double2*, unsigned int*,     \
                                                cudaStream_t, const int32_t*,                   \
                                                const SpeciesParams*);                          \
    template cudaError_t launch_deposit_charge<T>(int, const ParticleGeom&, const T*, const T*, \
                                                  int64_t, double2*, unsigned int*,             \
                                                  cudaStream_t, const int32_t*,                 \
                                                  const SpeciesParams*);                        \
    template cudaError_t launch_deposit_z<T>(int, const ParticleGeom&, const T*, const T*,      \
                                             const T*, int64_t, const int32_t*,                 \
                                             const SpeciesParams&, void*, size_t, double,       \
                                             unsigned int*, cudaStream_t);                      \
    template cudaError_t launch_gather_push3<T>(int, const ParticleGeom&, const PushParams&,    \
                                                const T*, const T*, T*, T*, const T*, const T*, \
                                                const T*, const T*, T*, T*, T*, const int32_t*, \
                                                const SpeciesParams&, int64_t, const void*,     \
                                                const void*, double*, unsigned int*,            \
                                                cudaStream_t);                                  \
    template cudaError_t launch_init_particles3<T>(int, const ParticleGeom&, const PushParams&, \
                                                   T*, T*, T*, T*, T*, const T*, const T*,      \
                                                   const T*, T*, T*, T*, const int32_t*,        \
                                                   const SpeciesParams&, int64_t, const void*,  \
                                                   unsigned int*, cudaStream_t);                \
    template cudaError_t launch_gather_push<T>(int, const ParticleGeom&, const PushParams&,     \
                                               const T*, const T*, T*, T*, const T*, const T*,  \
                                               T*, T*, int64_t, const void*, double*, double*,  \
                                               unsigned int*, cudaStream_t, bool);                    \
    template cudaError_t launch_init_particles<T>(int, const ParticleGeom&, const PushParams&,  \
                                                  T*, T*, T*, T*, const T*, const T*, T*, T*,   \
                                                  int64_t, const void*, unsigned int*,          \
                                                  cudaStream_t);                                \
    template cudaError_t launch_scatter_by_id<T>(const T*, const int32_t*, double*, int64_t,    \
                                                 cudaStream_t);                                 \
    template cudaError_t launch_extract<T>(const void*, int, int, double, double*, int64_t,     \
                                           cudaStream_t);                                       \
    template cudaError_t launch_wrap_positions<T>(T*, T*, int64_t, double, double, cudaStream_t); \
    template cudaError_t launch_move_deposit_fix<T>(int, const ParticleGeom&, T*, T*, const T*,   \
                                                    const T*, int64_t, longlong2*, float,         \
                                                    unsigned int*, cudaStream_t, const int32_t*,  \
                                                    const SpeciesParams*);                        \
    template cudaError_t launch_deposit_charge_fix<T>(int, const ParticleGeom&, const T*,         \
                                                      const T*, int64_t, longlong2*, float,       \
                                                      unsigned int*, cudaStream_t,                \
                                                      const int32_t*, const SpeciesParams*);      \
    template cudaError_t launch_fix_to_cplx<T>(const longlong2*, double, void*, int64_t,          \
                                               cudaStream_t);
GPIC_INST(double)
GPIC_INST(float)
#undef GPIC_INST
template cudaError_t launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template cudaError_t launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template cudaError_t launch_convert<double, double>(const double*, double*, int64_t, cudaStream_t);

}  // namespace gpic
