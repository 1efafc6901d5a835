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
    float scale;     // 1 / quantum, a power of two
    float s_hi;      // scale 2^-19
    float neg_step;  // -2^19 / scale
    static AccFix make(void* j, float scale) {
        return AccFix{(longlong2*)j, scale, scale * (1.0f / 524288.0f), -524288.0f / scale};
    }
    // round(v * scale), the contribution in units of the quantum (set-up only: the
    // float-to-int64 conversion runs on the FP64 pipe)
    __device__ __forceinline__ static long long q(float v, float s) {
        return __float2ll_rn(__fmul_rn(v, s));
    }
    // The same integer round(v * scale) as hi * 2^19 + lo with |hi| <= 2^19 and
    // |lo| <= 2^18, by FP32 and integer operations only, for |v * scale| <= 2^38:
    //   hi = rne(v scale 2^-19)   -- fma with 1.5 * 2^23 leaves it in the low mantissa bits
    //   d  = v - hi 2^19 / scale  -- exact (a power-of-two scale, |d scale| <= 2^18)
    //   lo = rne(d scale)         -- the same trick, d scale is exact
    // hi 2^19 is even, so rne(v scale - hi 2^19) = rne(v scale) - hi 2^19.
    __device__ __forceinline__ void split(float v, int& hi, int& lo) const {
        const float m1 = __fmaf_rn(v, s_hi, 12582912.0f);
        hi = __float_as_int(m1) - 0x4B400000;
        const float d = __fmaf_rn(__fsub_rn(m1, 12582912.0f), neg_step, v);
        lo = __float_as_int(__fmaf_rn(d, scale, 12582912.0f)) - 0x4B400000;
    }
    __device__ __forceinline__ static unsigned long long join(int hi, int lo) {
        return (unsigned long long)((long long)hi * 524288ll + (long long)lo);
    }
    template <typename T>
    __device__ __forceinline__ void add(size_t node, T a, T b) const {
        int ha, la, hb, lb;
        split((float)a, ha, la);
        split((float)b, hb, lb);
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


// Move + deposit over particles sorted by tile and cell (see sort.cu), FP32 form.
//
// CTA (tile, split) deposits the particles of one tile into a shared-memory copy of the
// tile's node region (the tile plus a halo, rows of `pitch` words) and adds the region
// to the global grid.  Traversal: thread tid serves local cell c = tid mod t^2 and phase
// f = tid div t^2 and takes, one per round, the particles f, f + F, f + 2F, ... of the
// CTA's share of that cell (F = threads per cell).  The 32 lanes of a warp thus work on 32
// consecutive local cells -- a block of 32/t x t cells -- and the row pitch is = t
// (mod 32), so for each stencil offset their nodes fall in 32 different banks while the
// particles sit in their sorted cells.
//
// Shared atomics are native for 32-bit integers, so each contribution is split exactly
// into hi * 2^19 + lo (AccFix::split) and the parts are summed apart.  The region is
// flushed to the global grid every kFlushRounds rounds: a round adds at most one
// contribution per thread to a node, so between flushes a 32-bit sum holds at most
// kFlushRounds * 256 = 2^11 terms of magnitude <= 2^19 (< 2^31).  A particle whose
// stencil leaves the region (it drifted further than the halo) adds the nodes outside
// straight to the global grid.  Integer sums make the result independent of the order
// of the particles.
constexpr int kFlushRounds = 8;
constexpr int kLoBits = 19;
constexpr int kRegionCap = 2560;  // largest region (rx * pitch words), 40 KB for four arrays

template <typename T, int P>
__global__ void __launch_bounds__(kThreads, 5)
k_move_deposit_tiled(GeomT<T> g, TileGeom tg, T* __restrict__ x, T* __restrict__ y,
                     const float4* __restrict__ p4, const int* __restrict__ off, int nsplit,
                     AccFix acc, unsigned int* __restrict__ err) {
    // four arrays of R = rx * pitch words: lo_x, lo_y, hi_x, hi_y (sized to the region,
    // so that the rest of the L1 caches the scattered particle loads)
    extern __shared__ int sacc[];
    __shared__ int max_rounds;
    const int pitch = tg.pitch;
    const int R = tg.rx * pitch;
    const int tt = tg.t * tg.t;
    const int tile = blockIdx.x / nsplit, split = blockIdx.x - tile * nsplit;
    const int cell = threadIdx.x % tt;
    const int phases = blockDim.x / tt;   // threads per cell in this CTA
    const int phase = threadIdx.x / tt;
    const int key = tile * tt + cell;
    if (threadIdx.x == 0) {  // the tile's particles come to L2 while the region is cleared
        const int64_t a0 = off[tile * tt], a1 = off[(tile + 1) * tt];
        prefetch_l2(p4 + a0, (size_t)(a1 - a0) * sizeof(float4));
    }
    const int o0 = off[key], count = off[key + 1] - o0;
    // split s takes the contiguous share [s count / nsplit, (s+1) count / nsplit) of the
    // cell, so the particles of one 32-byte sector are read by one CTA
    const int lo_ = (int)((int64_t)count * split / nsplit);
    const int hi_ = (int)((int64_t)count * (split + 1) / nsplit);
    const int64_t cbeg = (int64_t)o0 + lo_ + phase;
    const int streams = phases;
    const int len = hi_ - lo_;
    const int mine = len > phase ? (len - phase + phases - 1) / phases : 0;
    if (threadIdx.x == 0) max_rounds = 0;
    for (int k = threadIdx.x; k < R; k += blockDim.x) {
#pragma unroll
        for (int q = 0; q < 4; ++q) sacc[q * R + k] = 0;
    }
    __syncthreads();
    atomicMax(&max_rounds, mine);
    __syncthreads();
    const int rounds = max_rounds;
    if (rounds == 0) return;  // empty tile (uniform for the CTA)
    griddep_wait();  // particles and J come from the previous operations of the stream
    griddep_launch();
    const int tx = tile / tg.nty, ty = tile - tx * tg.nty;
    // region origin, reduced into [0, n): then gi - bi lies in (-n, n) and bi + ri in
    // [0, 2n), so one correction wraps each exactly (whatever the halo)
    int bi = (tx * tg.t - tg.halo) % g.nx, bj = (ty * tg.t - tg.halo) % g.ny;
    if (bi < 0) bi += g.nx;
    if (bj < 0) bj += g.ny;
    const T dt = g.dt, lx = g.lx, ly = g.ly, idx_ = g.inv_dx, idy = g.inv_dy;
    unsigned bad = 0;
    for (int r = 0; r < rounds; ++r) {
        if (r < mine) {
            const int64_t p = cbeg + (int64_t)r * streams;
            const float4 q4 = p4[p];  // one 16-byte load: x, y, vx, vy
            const T vxi = (T)q4.z, vyi = (T)q4.w;
            const T xp = move_pos((T)q4.x, vxi, dt, lx);
            const T yp = move_pos((T)q4.y, vyi, dt, ly);
            x[p] = xp;
            y[p] = yp;
            const T xi = rmul(xp, idx_), yj = rmul(yp, idy);
            if (!in_domain(xi, g.nx) || !in_domain(yj, g.ny)) {
                bad |= ERR_NONFINITE;
            } else {
                T wx[P + 1], wy[P + 1];
                const int ix = wrap_idx(Shape<P, T>::weights(xi, wx), g.nx);
                const int iy = wrap_idx(Shape<P, T>::weights(yj, wy), g.ny);
                int ri0 = ix - bi, rj0 = iy - bj;
                if (ri0 < 0) ri0 += g.nx;
                if (rj0 < 0) rj0 += g.ny;
                if (ri0 + P < tg.rx && rj0 + P < tg.ry) {
                    // whole stencil in the region: rows ri0.., columns rj0.. (no wrap)
                    int* row = sacc + ri0 * pitch + rj0;
#pragma unroll
                    for (int a = 0; a <= P; ++a) {
                        const T tx_ = rmul(vxi, wx[a]), ty_ = rmul(vyi, wx[a]);
#pragma unroll
                        for (int b = 0; b <= P; ++b) {
                            int hx, lx2, hy, ly2;
                            acc.split((float)rmul(tx_, wy[b]), hx, lx2);
                            acc.split((float)rmul(ty_, wy[b]), hy, ly2);
                            atomicAdd(row + b, lx2);
                            atomicAdd(row + R + b, ly2);
                            atomicAdd(row + 2 * R + b, hx);
                            atomicAdd(row + 3 * R + b, hy);
                        }
                        row += pitch;
                    }
                } else {
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
                                acc.split((float)cx, hx, lx2);
                                acc.split((float)cy, hy, ly2);
                                int* c = sacc + ri * pitch + rj;
                                atomicAdd(c, lx2);
                                atomicAdd(c + R, ly2);
                                atomicAdd(c + 2 * R, hx);
                                atomicAdd(c + 3 * R, hy);
                            } else {
                                acc.add((size_t)gi * g.ny + gj, cx, cy);
                            }
                        }
                    }
                }
            }
        }
        if ((r + 1) % kFlushRounds == 0 || r == rounds - 1) {  // uniform in the CTA
            __syncthreads();
            for (int k = threadIdx.x; k < R; k += blockDim.x) {
                const int lx_ = sacc[k], ly_ = sacc[R + k];
                const int hx = sacc[2 * R + k], hy = sacc[3 * R + k];
                if (!(lx_ | ly_ | hx | hy)) continue;
                sacc[k] = sacc[R + k] = sacc[2 * R + k] = sacc[3 * R + k] = 0;
                const int ri = k / pitch, rj = k - ri * pitch;
                int gi = bi + ri, gj = bj + rj;
                if (gi >= g.nx) gi -= g.nx;
                if (gj >= g.ny) gj -= g.ny;
                const size_t node = (size_t)gi * g.ny + gj;
                const long long sx = (long long)hx * (1ll << kLoBits) + (long long)lx_;
                const long long sy = (long long)hy * (1ll << kLoBits) + (long long)ly_;
                if (sx) atomicAdd(reinterpret_cast<unsigned long long*>(&acc.J[node].x), (unsigned long long)sx);
                if (sy) atomicAdd(reinterpret_cast<unsigned long long*>(&acc.J[node].y), (unsigned long long)sy);
            }
            __syncthreads();
        }
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
template <typename T>
__device__ __forceinline__ void push_one(const PushT<T>& pp, const T* f, int64_t p,
                                         T* __restrict__ px, T* __restrict__ py,
                                         const T* __restrict__ vx, const T* __restrict__ vy,
                                         T* __restrict__ vxo, T* __restrict__ vyo, unsigned& bad,
                                         double& kin, T& vx_new, T& vy_new) {
    const T vsx = rfma((T)2, vx[p], -vxo[p]);
    const T vsy = rfma((T)2, vy[p], -vyo[p]);
    const T fx = rfma(f[6], vsy, rfma(f[4], vsx, -f[0]));
    const T fy = rfma(f[7], vsy, rfma(f[5], vsx, -f[1]));
    const T Px = rfma(pp.qdt, fx, px[p]);
    const T Py = rfma(pp.qdt, fy, py[p]);
    const T ux = rfma(-pp.q, f[2], Px), uy = rfma(-pp.q, f[3], Py);
    const T den = rsqrt_rn(rfma(pp.c2, rfma(ux, ux, rmul(uy, uy)), rmul(pp.mc2, pp.mc2)));
    const T rc = rdiv(pp.c2, den);
    const T vxn1 = rmul(rc, ux), vyn1 = rmul(rc, uy);
    px[p] = Px;
    py[p] = Py;
    vxo[p] = vxn1;
    vyo[p] = vyn1;
    vx_new = vxn1;
    vy_new = vyn1;
    if (!isfinite(vxn1) || !isfinite(vyn1)) bad |= ERR_NONFINITE;
    if (pp.diag) {  // m c^2 (gamma - 1) per unit weight, in FP64 for either storage type
        const double uxd = ux, uyd = uy, c2d = pp.c * pp.c, mc2d = pp.m * c2d;
        kin += sqrt(c2d * (uxd * uxd + uyd * uyd) + mc2d * mc2d) - mc2d;
    }
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
              const cplx_t<T>* __restrict__ F, double* __restrict__ gout,
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
        if (gout) {  // the adjoint's record of this step (ten arrays of n, see launcher)
            gout[p] = (double)px[p];
            gout[(size_t)n + p] = (double)py[p];
            gout[2 * (size_t)n + p] = (double)vxn1;
            gout[3 * (size_t)n + p] = (double)vyn1;
#pragma unroll
            for (int k = 2; k < 8; ++k) gout[(size_t)(k + 2) * n + p] = (double)f[k];
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
                    float* __restrict__ vyo, float4* __restrict__ p4,
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
        p4[p] = make_float4(xp, yp, vxn1, vyn1);  // the next deposit's packed input
    }
    push_finish(pp, bad, kin, diag, err);
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
        const T vzi = sp ? rmul(vz[p], fq) : vz[p];
#pragma unroll
        for (int a = 0; a <= P; ++a) {
            const size_t row = (size_t)wrap_idx(ix + a, g.nx) * g.ny;
            const T tz = rmul(vzi, wx[a]);
#pragma unroll
            for (int b = 0; b <= P; ++b) acc.add1(row + wrap_idx(iy + b, g.ny), rmul(tz, wy[b]));
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
        if (pp.diag) {  // w m c^2 (gamma - 1) in FP64
            const double c2d = pp.c * pp.c, mc2d = k.m * c2d;
            const double ud2 = (double)ux * ux + (double)uy * uy + (double)uz * uz;
            kin += k.w * (sqrt(c2d * ud2 + mc2d * mc2d) - mc2d);
        }
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

cudaError_t launch_replay_step(const ParticleGeom& g, const double* s0, double* s1,
                               const double* rec, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_replay_step<double><<<blocks_for(n), kThreads, 0, s>>>(typed<double>(g), s0, s1, rec, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_deposit_z(int p, const ParticleGeom& g, const T* x, const T* y, const T* vz,
                             int64_t n, const int32_t* sp, const SpeciesParams& spp, void* jz,
                             bool fix, float scale, unsigned int* err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int32_t* spi = spp.n > 0 ? sp : nullptr;
    if (fix) {
        GPIC_DISPATCH_PA(p, k_deposit_z, AccFix, typed<T>(g), x, y, vz, n, spi,
                         typed_species<T>(&spp), (AccFix::make(jz, scale)), err)
    } else {
        GPIC_DISPATCH_PA(p, k_deposit_z, AccF64, typed<T>(g), x, y, vz, n, spi,
                         typed_species<T>(&spp), AccF64{(double2*)jz}, err)
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
cudaError_t launch_move_deposit_tiled(int p, const ParticleGeom& g, const TileGeom& tg, T* x,
                                      T* y, const float4* p4, int64_t n, const int* off,
                                      void* j, bool fix, float scale, unsigned int* err,
                                      cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (!fix) return cudaErrorInvalidValue;  // the tiled pass is the fixed-point form's
    if (tg.t * tg.t > kThreads || kThreads % (tg.t * tg.t) != 0) return cudaErrorInvalidValue;
    // splits per tile: about 1366 particles (5 or 6 rounds of 256) per CTA at the mean
    // density, so that a grid of 64-per-cell tiles holds about five CTAs per SM (timed
    // fastest of 512..2048 on a 128 x 128 grid with 2^20 particles)
    const int ntiles = tg.ntx * tg.nty;
    int nsplit = (int)((n + (int64_t)ntiles * 1366 - 1) / ((int64_t)ntiles * 1366));
    if (nsplit < 1) nsplit = 1;
    if (nsplit > 64) nsplit = 64;
    const int blocks = ntiles * nsplit;
    if (tg.rx * tg.pitch > kRegionCap || tg.ry > tg.pitch) return cudaErrorInvalidValue;
    const AccFix acc = AccFix::make(j, scale);
    const size_t smem = (size_t)4 * tg.rx * tg.pitch * sizeof(int);
#define GPIC_TILED(PP)                                                                     \
    e = launch_pdl(k_move_deposit_tiled<T, PP>, dim3(blocks), dim3(kThreads), smem, s,        \
                   typed<T>(g), tg, x, y, p4, off, nsplit, acc, err);
    cudaError_t e = cudaSuccess;
    switch (p) {
        case 2: GPIC_TILED(2) break;
        case 3: GPIC_TILED(3) break;
        case 4: GPIC_TILED(4) break;
        default: return cudaErrorInvalidValue;
    }
#undef GPIC_TILED
    return e;
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
                               unsigned int* err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    GPIC_DISPATCH_P(p, k_gather_push, typed<T>(g), typed<T>(pp), x, y, px, py, vx, vy, vxo, vyo, n,
                    (const cplx_t<T>*)f, gout, diag, err)
    return cudaGetLastError();
}

cudaError_t launch_gather_push_tiled(int p, const ParticleGeom& g, const PushParams& pp,
                                    const TileGeom& tg, const float* x, const float* y, float* px,
                                    float* py, const float* vx, const float* vy, float* vxo,
                                    float* vyo, float4* p4, int64_t n, const int* off,
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
                           vyo, p4, off, nsplit, (const float2*)f, diag, err);                 \
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
                                                cudaStream_t, const int32_t*,                   \
                                                const SpeciesParams*);                          \
    template cudaError_t launch_deposit_charge<T>(int, const ParticleGeom&, const T*, const T*, \
                                                  int64_t, double2*, unsigned int*,             \
                                                  cudaStream_t, const int32_t*,                 \
                                                  const SpeciesParams*);                        \
    template cudaError_t launch_deposit_z<T>(int, const ParticleGeom&, const T*, const T*,      \
                                             const T*, int64_t, const int32_t*,                 \
                                             const SpeciesParams&, void*, bool, float,          \
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
                                                    unsigned int*, cudaStream_t, const int32_t*,  \
                                                    const SpeciesParams*);                        \
    template cudaError_t launch_deposit_charge_fix<T>(int, const ParticleGeom&, const T*,         \
                                                      const T*, int64_t, longlong2*, float,       \
                                                      unsigned int*, cudaStream_t,                \
                                                      const int32_t*, const SpeciesParams*);      \
    template cudaError_t launch_fix_to_cplx<T>(const longlong2*, double, void*, int64_t,          \
                                               cudaStream_t);                                     \
    template cudaError_t launch_move_deposit_tiled<T>(int, const ParticleGeom&, const TileGeom&,  \
                                                      T*, T*, const float4*, int64_t,             \
                                                      const int*, void*, bool, float,             \
                                                      unsigned int*, cudaStream_t);
GPIC_INST(double)
GPIC_INST(float)
#undef GPIC_INST
template cudaError_t launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template cudaError_t launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template cudaError_t launch_convert<double, double>(const double*, double*, int64_t, cudaStream_t);

}  // namespace gpic
