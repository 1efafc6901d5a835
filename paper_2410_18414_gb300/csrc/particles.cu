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

// Round-to-nearest-even integer of a float with |x| < 2^22, without a conversion
// instruction: adding 1.5 * 2^23 leaves the rounded integer in the low mantissa bits.
__device__ __forceinline__ int round_small(float x) {
    return __float_as_int(__fadd_rn(x, 12582912.0f)) - 0x4B400000;
}

struct AccFix {
    longlong2* J;
    float scale;
    // round(v * scale), the contribution in units of the quantum 1/scale (set-up only:
    // the float-to-int64 conversion runs on the FP64 pipe)
    __device__ __forceinline__ static long long q(float v, float s) {
        return __float2ll_rn(__fmul_rn(v, s));
    }
    // The same integer round(v * scale) as hi * 2^19 + lo with FP32 and integer operations
    // only, for |v * scale| < 2^38: t = v * scale, hi = floor(t / 2^19) (exact),
    // lo = round(t - hi 2^19) with t - hi 2^19 in [0, 2^19] exact.  hi 2^19 is an even
    // integer, so rounding t - hi 2^19 to nearest even gives round(t) - hi 2^19.
    __device__ __forceinline__ static void split(float v, float s, int& hi, int& lo) {
        const float t = __fmul_rn(v, s);
        const float hf = floorf(__fmul_rn(t, 1.0f / 524288.0f));
        hi = round_small(hf);
        lo = round_small(__fmaf_rn(-hf, 524288.0f, t));
    }
    __device__ __forceinline__ static unsigned long long join(int hi, int lo) {
        return (unsigned long long)((long long)hi * 524288ll + (long long)lo);
    }
    template <typename T>
    __device__ __forceinline__ void add(size_t node, T a, T b) const {
        int ha, la, hb, lb;
        split((float)a, scale, ha, la);
        split((float)b, scale, hb, lb);
        atomicAdd(reinterpret_cast<unsigned long long*>(&J[node].x), join(ha, la));
        atomicAdd(reinterpret_cast<unsigned long long*>(&J[node].y), join(hb, lb));
    }
    template <typename T>
    __device__ __forceinline__ void add1(size_t node, T a) const {
        atomicAdd(reinterpret_cast<unsigned long long*>(&J[node].x), (unsigned long long)q((float)a, scale));
    }
};

template <typename T, int P, typename Acc>
__global__ void __launch_bounds__(kThreads)
k_move_deposit(GeomT<T> g, T* __restrict__ x, T* __restrict__ y, const T* __restrict__ vx,
               const T* __restrict__ vy, int64_t n, Acc acc, unsigned int* __restrict__ err) {
    const T dt = g.dt, lx = g.lx, ly = g.ly, idx_ = g.inv_dx, idy = g.inv_dy;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const T vxi = vx[p], vyi = vy[p];
        T xp = move_pos(x[p], vxi, dt, lx);
        T yp = move_pos(y[p], vyi, dt, ly);
        x[p] = xp;
        y[p] = yp;
        const T xi = rmul(xp, idx_), yj = rmul(yp, idy);
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
            const T tx = rmul(vxi, wx[a]), ty = rmul(vyi, wx[a]);
            const size_t row = (size_t)gi * g.ny;
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                const int gj = wrap_idx(iy + b, g.ny);
                acc.add(row + gj, rmul(tx, wy[b]), rmul(ty, wy[b]));
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
        const T xi = rmul(x[p], idx_), yj = rmul(y[p], idy);
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
                acc.add1((size_t)gi * g.ny + gj, rmul(wx[a], wy[b]));
            }
        }
    }
}


// Move + deposit over particles sorted by tile (see sort.cu), FP32 form.  CTA b owns
// particles [b*chunk, (b+1)*chunk); for each run of particles of one tile it accumulates
// the fixed-point contributions into a shared-memory copy of that tile's node region (the
// tile plus a halo) and adds the region to the global grid once.
//
// Shared atomics are native for 32-bit integers, so each contribution q is split exactly
// as q = hi * 2^19 + lo with lo in [0, 2^19] and |hi| <= 2^(k-19) <= 2^19 (the quantum is
// 2^-k c with k <= 38, see pic_api.cu; AccFix::split), and hi and lo are summed apart.
// A node receives at most one contribution per particle and a CTA at most kDepositChunk
// particles, so both 32-bit sums stay within 2^30 + 2^11.  The flush recombines them.
// A node outside the region (a particle that drifted further than the halo since the
// last sort) goes straight to the global grid.  Integer sums make the result independent
// of the order of the particles.
constexpr int kDepositChunk = 2048;
constexpr int kLoBits = 19;

__device__ __forceinline__ int64_t gcd64(int64_t a, int64_t b) {
    while (b) {
        const int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

template <typename T, int P>
__global__ void __launch_bounds__(kThreads)
k_move_deposit_tiled(GeomT<T> g, TileGeom tg, T* __restrict__ x, T* __restrict__ y,
                     const T* __restrict__ vx, const T* __restrict__ vy, int64_t n,
                     const int* __restrict__ keys, const int* __restrict__ off, AccFix acc,
                     unsigned int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // four int arrays of R words (lo_x, lo_y, hi_x, hi_y): a node's word k sits in bank
    // k mod 32, so lanes hitting different nodes rarely share a bank
    const int R = tg.rx * tg.ry;
    int* lo_x = reinterpret_cast<int*>(smem_raw);
    int* lo_y = lo_x + R;
    int* hi_x = lo_y + R;
    int* hi_y = hi_x + R;
    const int64_t c0 = (int64_t)blockIdx.x * kDepositChunk;
    if (c0 >= n) return;
    const int64_t c1 = c0 + kDepositChunk < n ? c0 + kDepositChunk : n;
    const T dt = g.dt, lx = g.lx, ly = g.ly, idx_ = g.inv_dx, idy = g.inv_dy;
    const int tt = tg.t * tg.t;
    __shared__ int64_t stride_sh;
    unsigned bad = 0;
    int64_t p0 = c0;
    while (p0 < c1) {
        const int tile = keys[p0] / tt;
        const int64_t tend = (int64_t)off[(tile + 1) * tt];
        const int64_t seg_end = tend < c1 ? tend : c1;
        const int tx = tile / tg.nty, ty = tile - tx * tg.nty;
        // region origin, reduced into [0, n): then gi - bi lies in (-n, n) and bi + ri in
        // [0, 2n), so one correction wraps each exactly (whatever the halo)
        int bi = (tx * tg.t - tg.halo) % g.nx, bj = (ty * tg.t - tg.halo) % g.ny;
        if (bi < 0) bi += g.nx;
        if (bj < 0) bj += g.ny;
        // Walk the segment in a stride permutation pos = j s mod L (gcd(s, L) = 1,
        // s ~ L/32): the particles are stored by cell, so consecutive positions share
        // nodes, while the 32 lanes of a warp then sit in ~32 different cells and their
        // shared atomics rarely hit the same word.
        const int64_t L = seg_end - p0;
        if (threadIdx.x == 0) {
            int64_t st = L / 32;
            st |= 1;
            while (gcd64(st, L) != 1) st += 2;
            stride_sh = st;
        }
        for (int k = threadIdx.x; k < 4 * R; k += blockDim.x) lo_x[k] = 0;
        __syncthreads();
        const int64_t st = stride_sh;
        const int64_t step = (int64_t)((unsigned long long)blockDim.x * (unsigned long long)st %
                                       (unsigned long long)L);
        int64_t pos = (int64_t)((unsigned long long)threadIdx.x * (unsigned long long)st %
                                (unsigned long long)L);
        for (int64_t j = threadIdx.x; j < L; j += blockDim.x) {
            const int64_t p = p0 + pos;
            pos += step;
            if (pos >= L) pos -= L;
            const T vxi = vx[p], vyi = vy[p];
            const T xp = move_pos(x[p], vxi, dt, lx);
            const T yp = move_pos(y[p], vyi, dt, ly);
            x[p] = xp;
            y[p] = yp;
            const T xi = rmul(xp, idx_), yj = rmul(yp, idy);
            if (!in_domain(xi, g.nx) || !in_domain(yj, g.ny)) {
                bad |= ERR_NONFINITE;
                continue;
            }
            T wx[P + 1], wy[P + 1];
            const int ix = Shape<P, T>::weights(xi, wx);
            const int iy = Shape<P, T>::weights(yj, wy);
#pragma unroll
            for (int a = 0; a <= P; ++a) {
                const int gi = wrap_idx(ix + a, g.nx);
                int ri = gi - bi;
                if (ri < 0) ri += g.nx;
                const T tx_ = rmul(vxi, wx[a]), ty_ = rmul(vyi, wx[a]);
#pragma unroll
                for (int b = 0; b <= P; ++b) {
                    const int gj = wrap_idx(iy + b, g.ny);
                    int rj = gj - bj;
                    if (rj < 0) rj += g.ny;
                    const T cx = rmul(tx_, wy[b]), cy = rmul(ty_, wy[b]);
                    if (ri < tg.rx && rj < tg.ry) {
                        int hx, lx2, hy, ly2;
                        AccFix::split((float)cx, acc.scale, hx, lx2);
                        AccFix::split((float)cy, acc.scale, hy, ly2);
                        const int k = ri * tg.ry + rj;
                        atomicAdd(lo_x + k, lx2);
                        atomicAdd(lo_y + k, ly2);
                        atomicAdd(hi_x + k, hx);
                        atomicAdd(hi_y + k, hy);
                    } else {
                        acc.add((size_t)gi * g.ny + gj, cx, cy);
                    }
                }
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < R; k += blockDim.x) {
            const int lx_ = lo_x[k], ly_ = lo_y[k], hx = hi_x[k], hy = hi_y[k];
            if (!(lx_ | ly_ | hx | hy)) continue;
            const long long sx = (long long)hx * (1ll << kLoBits) + (long long)lx_;
            const long long sy = (long long)hy * (1ll << kLoBits) + (long long)ly_;
            const int ri = k / tg.ry, rj = k - ri * tg.ry;
            int gi = bi + ri, gj = bj + rj;
            if (gi >= g.nx) gi -= g.nx;
            if (gj >= g.ny) gj -= g.ny;
            const size_t node = (size_t)gi * g.ny + gj;
            if (sx) atomicAdd(reinterpret_cast<unsigned long long*>(&acc.J[node].x), (unsigned long long)sx);
            if (sy) atomicAdd(reinterpret_cast<unsigned long long*>(&acc.J[node].y), (unsigned long long)sy);
        }
        __syncthreads();
        p0 = seg_end;
    }
    if (bad) atomicOr(err, bad);
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
k_gather_push(GeomT<T> g, PushT<T> pp, const T* __restrict__ x, const T* __restrict__ y,
              T* __restrict__ px, T* __restrict__ py, const T* __restrict__ vx,
              const T* __restrict__ vy, T* __restrict__ vxo, T* __restrict__ vyo, int64_t n,
              const cplx_t<T>* __restrict__ F, double* __restrict__ diag,
              unsigned int* __restrict__ err) {
    using C = cplx_t<T>;
    const T idx_ = g.inv_dx, idy = g.inv_dy;
    const T q = pp.q, qdt = pp.qdt, c2 = pp.c2, mc2 = pp.mc2;
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
                T g[8];
                load_node(node, g);  // dphi/dx, dphi/dy, Ax, Ay, dAx/dx, dAx/dy, dAy/dx, dAy/dy
                f0 += w * g[0];
                f1 += w * g[1];
                f2 += w * g[2];
                f3 += w * g[3];
                f4 += w * g[4];
                f5 += w * g[5];
                f6 += w * g[6];
                f7 += w * g[7];
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
    GPIC_DISPATCH_PA(p, k_move_deposit, AccF64, typed<T>(g), x, y, vx, vy, n, AccF64{j}, err)
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
    GPIC_DISPATCH_PA(p, k_move_deposit, AccFix, typed<T>(g), x, y, vx, vy, n, (AccFix{j, scale}),
                     err)
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
cudaError_t launch_move_deposit_tiled(int p, const ParticleGeom& g, const TileGeom& tg, T* x,
                                      T* y, const T* vx, const T* vy, int64_t n, const int* keys,
                                      const int* off, void* j, bool fix, float scale,
                                      unsigned int* err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (!fix) return cudaErrorInvalidValue;  // the tiled pass is the fixed-point form's
    const int blocks = (int)((n + kDepositChunk - 1) / kDepositChunk);
    const size_t smem = (size_t)tg.rx * tg.ry * 4 * sizeof(int);
    if (smem > 96 * 1024) return cudaErrorInvalidValue;
    AccFix acc{(longlong2*)j, scale};
    cudaError_t e = cudaSuccess;
#define GPIC_TILED(PP)                                                                             \
    {                                                                                              \
        auto kern = k_move_deposit_tiled<T, PP>;                                                   \
        if (smem > 48 * 1024)                                                                      \
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e == cudaSuccess)                                                                      \
            kern<<<blocks, kThreads, smem, s>>>(typed<T>(g), tg, x, y, vx, vy, n, keys, off, acc, \
                                                err);                                           \
    }
    switch (p) {
        case 2: GPIC_TILED(2) break;
        case 3: GPIC_TILED(3) break;
        case 4: GPIC_TILED(4) break;
        default: return cudaErrorInvalidValue;
    }
#undef GPIC_TILED
    if (e != cudaSuccess) return e;
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
    GPIC_DISPATCH_P(p, k_gather_push, typed<T>(g), typed<T>(pp), x, y, px, py, vx, vy, vxo, vyo, n,
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
                                               cudaStream_t);                                     \
    template cudaError_t launch_move_deposit_tiled<T>(int, const ParticleGeom&, const TileGeom&,  \
                                                      T*, T*, const T*, const T*, int64_t,        \
                                                      const int*, const int*, void*, bool, float, \
                                                      unsigned int*, cudaStream_t);
GPIC_INST(double)
GPIC_INST(float)
#undef GPIC_INST
template cudaError_t launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template cudaError_t launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template cudaError_t launch_convert<double, double>(const double*, double*, int64_t, cudaStream_t);

}  // namespace gpic
