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

namespace gpic {

namespace {

constexpr int kThreads = 256;

inline int blocks_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    const int64_t cap = 152 * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
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
    __device__ __forceinline__ void add(size_t node, T a, T b) const {
        atomicAdd(&J[node].x, (double)a);
        atomicAdd(&J[node].y, (double)b);
    }
    template <typename T>
    __device__ __forceinline__ void add1(size_t node, T a) const {
        atomicAdd(&J[node].x, (double)a);
    }
};

struct AccFix {
    longlong2* J;
    float scale;
    __device__ __forceinline__ static unsigned long long q(float v, float s) {
        return (unsigned long long)__float2ll_rn(v * s);
    }
    template <typename T>
    __device__ __forceinline__ void add(size_t node, T a, T b) const {
        atomicAdd(reinterpret_cast<unsigned long long*>(&J[node].x), q((float)a, scale));
        atomicAdd(reinterpret_cast<unsigned long long*>(&J[node].y), q((float)b, scale));
    }
    template <typename T>
    __device__ __forceinline__ void add1(size_t node, T a) const {
        atomicAdd(reinterpret_cast<unsigned long long*>(&J[node].x), q((float)a, scale));
    }
};

template <typename T, int P, typename Acc>
__global__ void __launch_bounds__(kThreads)
k_move_deposit(ParticleGeom g, T* __restrict__ x, T* __restrict__ y, const T* __restrict__ vx,
               const T* __restrict__ vy, int64_t n, Acc acc, unsigned int* __restrict__ err) {
    const T dt = (T)g.dt, lx = (T)g.lx, ly = (T)g.ly, idx_ = (T)g.inv_dx, idy = (T)g.inv_dy;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const T vxi = vx[p], vyi = vy[p];
        T xp = wrap_pos(x[p] + vxi * dt, lx);
        T yp = wrap_pos(y[p] + vyi * dt, ly);
        x[p] = xp;
        y[p] = yp;
        const T xi = xp * idx_, yj = yp * idy;
        if (!in_domain(xi, g.nx) || !in_domain(yj, g.ny)) {
            atomicOr(err, (unsigned)ERR_NONFINITE);
            continue;
        }
        T wx[P + 1], wy[P + 1];
        const int ix = Shape<P, T>::weights(xi, wx);
        const int iy = Shape<P, T>::weights(yj, wy);
#pragma unroll
        for (int a = 0; a <= P; ++a) {
            const int gi = wrap_idx(ix + a, g.nx);
            const T tx = vxi * wx[a], ty = vyi * wx[a];
            const size_t row = (size_t)gi * g.ny;
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                const int gj = wrap_idx(iy + b, g.ny);
                acc.add(row + gj, tx * wy[b], ty * wy[b]);
            }
        }
    }
}

template <typename T, int P, typename Acc>
__global__ void __launch_bounds__(kThreads)
k_deposit_charge(ParticleGeom g, const T* __restrict__ x, const T* __restrict__ y, int64_t n,
                 Acc acc, unsigned int* __restrict__ err) {
    const T idx_ = (T)g.inv_dx, idy = (T)g.inv_dy;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const T xi = x[p] * idx_, yj = y[p] * idy;
        if (!in_domain(xi, g.nx) || !in_domain(yj, g.ny)) {
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
                acc.add1((size_t)gi * g.ny + gj, wx[a] * wy[b]);
            }
        }
    }
}

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

__global__ void k_extract_fix(const longlong2* __restrict__ J, int comp, double scale,
                              double* __restrict__ dst, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const longlong2 v = J[k];
        dst[k] = scale * (double)(comp ? v.y : v.x);
    }
}

template <typename T, int P>
__global__ void __launch_bounds__(kThreads)
k_gather_push(ParticleGeom g, PushParams pp, const T* __restrict__ x, const T* __restrict__ y,
              T* __restrict__ px, T* __restrict__ py, const T* __restrict__ vx,
              const T* __restrict__ vy, T* __restrict__ vxo, T* __restrict__ vyo, int64_t n,
              const cplx_t<T>* __restrict__ F, double* __restrict__ diag,
              unsigned int* __restrict__ err) {
    using C = cplx_t<T>;
    const T idx_ = (T)g.inv_dx, idy = (T)g.inv_dy;
    const T q = (T)pp.q, qdt = (T)(pp.q * pp.dt), c2 = (T)(pp.c * pp.c);
    const T mc2 = (T)(pp.m * pp.c * pp.c);
    double kin = 0.0;
    unsigned bad = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const T xi = x[p] * idx_, yj = y[p] * idy;
        if (!in_domain(xi, g.nx) || !in_domain(yj, g.ny)) {
            bad |= ERR_NONFINITE;
            continue;
        }
        T wx[P + 1], wy[P + 1];
        const int ix = Shape<P, T>::weights(xi, wx);
        const int iy = Shape<P, T>::weights(yj, wy);
        T f0 = 0, f1 = 0, f2 = 0, f3 = 0, f4 = 0, f5 = 0, f6 = 0, f7 = 0;
#pragma unroll
        for (int a = 0; a <= P; ++a) {
            const int gi = wrap_idx(ix + a, g.nx);
            const C* row = F + (size_t)gi * g.ny * 4;
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                const int gj = wrap_idx(iy + b, g.ny);
                const T w = wx[a] * wy[b];
                const C* node = row + (size_t)gj * 4;
                const C g0 = node[0], g1 = node[1], g2 = node[2], g3 = node[3];
                f0 += w * g0.x;  // dphi/dx
                f1 += w * g0.y;  // dphi/dy
                f2 += w * g1.x;  // Ax
                f3 += w * g1.y;  // Ay
                f4 += w * g2.x;  // dAx/dx
                f5 += w * g2.y;  // dAx/dy
                f6 += w * g3.x;  // dAy/dx
                f7 += w * g3.y;  // dAy/dy
            }
        }
        const T vxn = vx[p], vyn = vy[p];
        const T vsx = (T)2 * vxn - vxo[p];
        const T vsy = (T)2 * vyn - vyo[p];
        const T Px = px[p] + qdt * (-f0 + f4 * vsx + f6 * vsy);
        const T Py = py[p] + qdt * (-f1 + f5 * vsx + f7 * vsy);
        const T ux = Px - q * f2, uy = Py - q * f3;
        const T den = sqrt(c2 * (ux * ux + uy * uy) + mc2 * mc2);
        const T vxn1 = c2 * ux / den, vyn1 = c2 * uy / den;
        px[p] = Px;
        py[p] = Py;
        vxo[p] = vxn1;
        vyo[p] = vyn1;
        if (!isfinite(vxn1) || !isfinite(vyn1)) bad |= ERR_NONFINITE;
        if (pp.diag) {  // m c^2 (gamma - 1) per unit weight, in FP64 for either storage type
            const double uxd = ux, uyd = uy, c2d = pp.c * pp.c, mc2d = pp.m * c2d;
            kin += sqrt(c2d * (uxd * uxd + uyd * uyd) + mc2d * mc2d) - mc2d;
        }
    }
    if (bad) atomicOr(err, bad);
    if (pp.diag) {
        for (int o = 16; o > 0; o >>= 1) kin += __shfl_down_sync(0xffffffffu, kin, o);
        if ((threadIdx.x & 31) == 0 && kin != 0.0) atomicAdd(diag + D_KIN, kin * pp.weight);
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
        const T xi = x[p] * idx_, yj = y[p] * idy;
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
                                cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    GPIC_DISPATCH_PA(p, k_move_deposit, AccF64, g, x, y, vx, vy, n, AccF64{j}, err)
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_deposit_charge(int p, const ParticleGeom& g, const T* x, const T* y, int64_t n,
                                  double2* j, unsigned int* err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    GPIC_DISPATCH_PA(p, k_deposit_charge, AccF64, g, x, y, n, AccF64{j}, err)
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_move_deposit_fix(int p, const ParticleGeom& g, T* x, T* y, const T* vx,
                                    const T* vy, int64_t n, longlong2* j, float scale,
                                    unsigned int* err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    GPIC_DISPATCH_PA(p, k_move_deposit, AccFix, g, x, y, vx, vy, n, (AccFix{j, scale}), err)
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_deposit_charge_fix(int p, const ParticleGeom& g, const T* x, const T* y,
                                      int64_t n, longlong2* j, float scale, unsigned int* err,
                                      cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    GPIC_DISPATCH_PA(p, k_deposit_charge, AccFix, g, x, y, n, (AccFix{j, scale}), err)
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
                               T* vyo, int64_t n, const void* f, double* diag, unsigned int* err,
                               cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    GPIC_DISPATCH_P(p, k_gather_push, g, pp, x, y, px, py, vx, vy, vxo, vyo, n,
                    (const cplx_t<T>*)f, diag, err)
    return cudaGetLastError();
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
                                                cudaStream_t);                                  \
    template cudaError_t launch_deposit_charge<T>(int, const ParticleGeom&, const T*, const T*, \
                                                  int64_t, double2*, unsigned int*,             \
                                                  cudaStream_t);                                \
    template cudaError_t launch_gather_push<T>(int, const ParticleGeom&, const PushParams&,     \
                                               const T*, const T*, T*, T*, const T*, const T*,  \
                                               T*, T*, int64_t, const void*, double*,           \
                                               unsigned int*, cudaStream_t);                    \
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
                                                    unsigned int*, cudaStream_t);                 \
    template cudaError_t launch_deposit_charge_fix<T>(int, const ParticleGeom&, const T*,         \
                                                      const T*, int64_t, longlong2*, float,       \
                                                      unsigned int*, cudaStream_t);               \
    template cudaError_t launch_fix_to_cplx<T>(const longlong2*, double, void*, int64_t,          \
                                               cudaStream_t);
GPIC_INST(double)
GPIC_INST(float)
#undef GPIC_INST
template cudaError_t launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template cudaError_t launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template cudaError_t launch_convert<double, double>(const double*, double*, int64_t, cudaStream_t);

}  // namespace gpic
