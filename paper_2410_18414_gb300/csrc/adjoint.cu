// Discrete adjoint of the step: the transpose of the Jacobian of one step of
// Algorithm 1 (section 4.2) with the BDF-k (section 3.2), CDF-2 (section 3.1) or DIRK
// (section 3.3) field solve, applied in reverse, for the gradient of an objective of the
// final state with respect to the initial velocities.
//
// Adjoint of a quantity z is written zb; the pairing is the plain sum over particles and
// grid nodes, and Re sum conj(zb) dz for a spectrum.  Reverse of step n -> n+1:
//
//   push + gather (k_adj_push_gather), per particle at x^{n+1}, from the fields the
//   forward push gathered (kept by the recording step):
//     u = P^{n+1} - q A_p, v^{n+1} = c^2 u / D, D = sqrt(c^2 |u|^2 + (m c^2)^2)
//     ub = (c^2/D) (vb - c^2 u (u . vb)/D^2);  Pb += ub;  A_p b = -q ub
//     P^{n+1} = P^n + q dt (-grad phi + (grad A) . v*):  (grad phi)b = -q dt Pb,
//       (d_l A_m)b = q dt Pb_l v*_m,  v*b_m = q dt sum_l Pb_l d_l A_m
//     v* = 2 v^n - v^{n-1}:  v^n b += 2 v*b,  v^{n-1} b = -v*b
//     the gather's transpose deposits the eight field adjoints with the same weights,
//     and x^{n+1} b gets sum_f gb_f grad(sum_node F_f W)
//   field solve (k_adj_modes / k_adj_columns), per mode, after forward transforms of the
//     deposited field adjoints: conj(i k) = -i k for the spectral gradients, then the
//     stepper's recurrences run backwards with their real per-mode multipliers (DIRK:
//     the transpose of the forward's per-mode 2 x 4 step matrix), ending in the
//     adjoint of the current spectrum, inverse-transformed to the mesh
//   deposit + move (k_adj_deposit_move), per particle:
//     J = q_p v^n W(x^{n+1}) / (dx dy):  v^n b += gather(Jb),
//       x^{n+1} b += v^n . grad gather(Jb)   (q_p/(dx dy) folded into Jb)
//     x^{n+1} = x^n + dt v^n:  x^n b = x^{n+1} b,  v^n b += dt x^{n+1} b
//   t = 0 (k_adj_init): P^0 = gamma m v^0 and the Taylor start v^{-1}(v^0, E^0).
//
// One thread per particle or per mode.  The particle kernels run in the storage type T of
// the forward they reverse: FP64 for the plain path, FP32 for the FP32 form (the adjoint
// of the step in exact arithmetic, evaluated along the FP32 form's trajectory; the
// fixed-point rounding of its current, piecewise constant, is differentiated as the
// identity).  The field adjoints they deposit are summed in FP64 (FP32 form: in FP32, the
// eight values of a node in two vector atomics, then converted), and the reverse field
// solve is FP64 in both forms, as the forward's per-mode update is.  Shape weights come
// from Shape<P, T> (the forward's), their derivatives from the closed forms below.
#include <algorithm>

#include "common.cuh"
#include "fft_device.cuh"
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

// d w[a] / d xi for the weights of Shape<P, T>, from the same offset d.
template <int P, typename T> struct DShape;
template <typename T> struct DShape<2, T> {
    // w = ((1/2 - d)^2/2, 3/4 - d^2, (1/2 + d)^2/2)
    static __device__ __forceinline__ void dweights(T xi, T* dw) {
        const T d = xi - floor(xi + (T)0.5);
        dw[0] = d - (T)0.5;
        dw[1] = (T)-2 * d;
        dw[2] = d + (T)0.5;
    }
};
template <typename T> struct DShape<3, T> {
    // w = (e^3/6, 2/3 - d^2 + d^3/2, 2/3 - e^2 + e^3/2, d^3/6), e = 1 - d
    static __device__ __forceinline__ void dweights(T xi, T* dw) {
        const T d = xi - floor(xi), e = (T)1 - d;
        dw[0] = (T)-0.5 * e * e;
        dw[1] = d * ((T)1.5 * d - (T)2);
        dw[2] = e * ((T)2 - (T)1.5 * e);
        dw[3] = (T)0.5 * d * d;
    }
};
template <typename T> struct DShape<4, T> {
    // derivative of (55 + 20 t - 120 t^2 + 80 t^3 - 16 t^4)/96
    static __device__ __forceinline__ T dmid(T t) {
        return ((T)20 + t * ((T)-240 + t * ((T)240 - (T)64 * t))) * (T)(1.0 / 96.0);
    }
    // w = ((1-2d)^4/384, mid(1+d), (115 - 120 d^2 + 48 d^4)/192, mid(1-d), (1+2d)^4/384)
    static __device__ __forceinline__ void dweights(T xi, T* dw) {
        const T d = xi - floor(xi + (T)0.5);
        const T a = (T)1 - (T)2 * d, b = (T)1 + (T)2 * d;
        dw[0] = -a * a * a * (T)(1.0 / 48.0);
        dw[1] = dmid((T)1 + d);
        dw[2] = d * (d * d - (T)1.25);
        dw[3] = -dmid((T)1 - d);
        dw[4] = b * b * b * (T)(1.0 / 48.0);
    }
};

template <typename T>
__device__ __forceinline__ bool inside(T xi, int n) { return xi >= (T)0 && xi <= (T)n; }

template <typename T, int P>
__global__ void __launch_bounds__(kThreads, 3)
k_adj_push_gather(ParticleGeom g, PushParams pp, const T* __restrict__ x1,
                  const T* __restrict__ y1, const T* __restrict__ px1,
                  const T* __restrict__ py1, const T* __restrict__ vx,
                  const T* __restrict__ vy, const T* __restrict__ vxo,
                  const T* __restrict__ vyo, const double* __restrict__ gfa,
                  const cplx_t<T>* __restrict__ F, AdjParticlesT<T> ab, double2* __restrict__ Fb,
                  float4* __restrict__ Fb32, int64_t n, unsigned int* __restrict__ err) {
    using C = cplx_t<T>;
    const size_t ng = (size_t)g.nx * g.ny;
    const T q = (T)pp.q, qdt = (T)(pp.q * pp.dt), c2 = (T)(pp.c * pp.c),
            mc2 = (T)(pp.m * pp.c * pp.c);
    const T idx_ = (T)g.inv_dx, idy = (T)g.inv_dy;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const T xi = rmul(x1[p], idx_), yj = rmul(y1[p], idy);
        if (!inside(xi, g.nx) || !inside(yj, g.ny)) {
            atomicOr(err, (unsigned)ERR_NONFINITE);
            continue;
        }
        T wx[P + 1], wy[P + 1], dwx[P + 1], dwy[P + 1];
        const int ix = Shape<P, T>::weights(xi, wx);
        const int iy = Shape<P, T>::weights(yj, wy);
        // the fields the forward push gathered at x^{n+1} (dphi/dx, dphi/dy, Ax, Ay,
        // dAx/dx, dAx/dy, dAy/dx, dAy/dy): from the record, or (gfa == NULL, the lean
        // record) gathered again from the step's fields F in the forward gather's node
        // order and roundings, which gives the same bits
        T f[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // f[0], f[1] (grad phi) are not needed here
        if (gfa) {
#pragma unroll
            for (int k = 2; k < 8; ++k) f[k] = (T)gfa[(size_t)(k - 2) * n + p];
        } else {
#pragma unroll 1
            for (int a = 0; a <= P; ++a) {
                const C* row = F + (size_t)wrap_idx(ix + a, g.nx) * g.ny * 4;
#pragma unroll
                for (int b = 0; b <= P; ++b) {
                    const C* node = row + (size_t)wrap_idx(iy + b, g.ny) * 4;
                    const T w = rmul(wx[a], wy[b]);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const C v = __ldg(node + k);
                        f[2 * k] = rfma(w, v.x, f[2 * k]);
                        f[2 * k + 1] = rfma(w, v.y, f[2 * k + 1]);
                    }
                }
            }
        }
        // velocity: v = c^2 u / D
        const T ux = px1[p] - q * f[2], uy = py1[p] - q * f[3];
        const T D = sqrt(c2 * (ux * ux + uy * uy) + mc2 * mc2);
        const T id = (T)1 / D;
        const T vbx = ab.vx[p], vby = ab.vy[p];
        const T cd = c2 * id, udv = (ux * vbx + uy * vby) * cd * id;
        const T ubx = cd * (vbx - ux * udv), uby = cd * (vby - uy * udv);
        const T pbx = ab.px[p] + ubx, pby = ab.py[p] + uby;
        // momentum: P^{n+1} = P^n + q dt (-grad phi + (grad A) . v*)
        const T vsx = (T)2 * vx[p] - vxo[p], vsy = (T)2 * vy[p] - vyo[p];
        T gb[8];
        gb[0] = -qdt * pbx;
        gb[1] = -qdt * pby;
        gb[2] = -q * ubx;
        gb[3] = -q * uby;
        gb[4] = qdt * pbx * vsx;
        gb[5] = qdt * pby * vsx;
        gb[6] = qdt * pbx * vsy;
        gb[7] = qdt * pby * vsy;
        const T vsbx = qdt * (pbx * f[4] + pby * f[5]);
        const T vsby = qdt * (pbx * f[6] + pby * f[7]);
        DShape<P, T>::dweights(xi, dwx);
        DShape<P, T>::dweights(yj, dwy);
        // one pass over the stencil: s = sum_f gb_f F_f at each node gives the position
        // gradient (separable: along y in the row, then across rows), and gb is deposited
        T xg = 0, yg = 0;
#pragma unroll 1
        for (int a = 0; a <= P; ++a) {
            const size_t row = (size_t)wrap_idx(ix + a, g.nx) * g.ny;
            const T wxa = wx[a];
            T sx = 0, sy = 0;
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                const size_t nd = row + wrap_idx(iy + b, g.ny);
                const C* node = F + nd * 4;
                T sn = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const C v = __ldg(node + k);
                    sn += gb[2 * k] * v.x + gb[2 * k + 1] * v.y;
                }
                sx += wy[b] * sn;
                sy += dwy[b] * sn;
                const T w = wxa * wy[b];
                if constexpr (sizeof(T) == 4) {  // the node's eight values, four an atomic
                    atomicAdd(Fb32 + 2 * nd,
                              make_float4(w * gb[0], w * gb[1], w * gb[2], w * gb[3]));
                    atomicAdd(Fb32 + 2 * nd + 1,
                              make_float4(w * gb[4], w * gb[5], w * gb[6], w * gb[7]));
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        atomicAdd(&Fb[k * ng + nd].x, (double)(w * gb[2 * k]));
                        atomicAdd(&Fb[k * ng + nd].y, (double)(w * gb[2 * k + 1]));
                    }
                }
            }
            xg += dwx[a] * sx;
            yg += wxa * sy;
        }
        ab.x[p] += idx_ * xg;
        ab.y[p] += idy * yg;
        ab.px[p] = pbx;
        ab.py[p] = pby;
        ab.vx[p] = ab.vxo[p] + (T)2 * vsbx;
        ab.vy[p] = ab.vyo[p] + (T)2 * vsby;
        ab.vxo[p] = -vsbx;
        ab.vyo[p] = -vsby;
    }
}

template <typename T, int P>
__global__ void __launch_bounds__(kThreads)
k_adj_deposit_move(ParticleGeom g, const T* __restrict__ x1, const T* __restrict__ y1,
                   const T* __restrict__ vx, const T* __restrict__ vy,
                   const double2* __restrict__ Jb, AdjParticlesT<T> ab, int64_t n,
                   unsigned int* __restrict__ err) {
    const T idx_ = (T)g.inv_dx, idy = (T)g.inv_dy, dt = (T)g.dt;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const T xi = rmul(x1[p], idx_), yj = rmul(y1[p], idy);
        if (!inside(xi, g.nx) || !inside(yj, g.ny)) {
            atomicOr(err, (unsigned)ERR_NONFINITE);
            continue;
        }
        T wx[P + 1], wy[P + 1], dwx[P + 1], dwy[P + 1];
        const int ix = Shape<P, T>::weights(xi, wx);
        const int iy = Shape<P, T>::weights(yj, wy);
        DShape<P, T>::dweights(xi, dwx);
        DShape<P, T>::dweights(yj, dwy);
        // separable sums: row a first along y with wy and dwy, then across rows
        T sx = 0, sy = 0, dxx = 0, dxy = 0, dyx = 0, dyy = 0;
#pragma unroll
        for (int a = 0; a <= P; ++a) {
            const size_t row = (size_t)wrap_idx(ix + a, g.nx) * g.ny;
            T rx = 0, ry = 0, rdx = 0, rdy = 0;
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                const double2 jd = __ldg(Jb + row + wrap_idx(iy + b, g.ny));
                const T jx = (T)jd.x, jy = (T)jd.y;
                rx += wy[b] * jx;
                ry += wy[b] * jy;
                rdx += dwy[b] * jx;
                rdy += dwy[b] * jy;
            }
            sx += wx[a] * rx;
            sy += wx[a] * ry;
            dxx += dwx[a] * rx;  // d/dxi of the gathered Jx adjoint
            dxy += dwx[a] * ry;  // d/dxi of the gathered Jy adjoint
            dyx += wx[a] * rdx;
            dyy += wx[a] * rdy;
        }
        const T vxp = vx[p], vyp = vy[p];
        const T xb = ab.x[p] + idx_ * (vxp * dxx + vyp * dxy);
        const T yb = ab.y[p] + idy * (vxp * dyx + vyp * dyy);
        ab.x[p] = xb;
        ab.y[p] = yb;
        ab.vx[p] = ab.vx[p] + sx + dt * xb;
        ab.vy[p] = ab.vy[p] + sy + dt * yb;
    }
}

constexpr int kModeThreads = 256;

__device__ __forceinline__ zd zl(const double2* p) { return zd{p->x, p->y}; }
__device__ __forceinline__ void zs(double2* p, zd v) { *p = make_double2(v.re, v.im); }

// The eight field adjoints' spectra / (nx ny) of mode (kx, ky), from the packed pairs
// za[k] = F(f_2k + i f_2k+1)(k) and zb[k] = the same at -k, folded into the adjoints of
// the three potentials they are taken from: gradient fields i k_l u get -i k_l, the A
// fields themselves 1.  (The particles' phi is phi~ for CDF-2, the new level otherwise.)
__device__ __forceinline__ void gathered_adjoints(const ModeCommon& mc, double kx, double ky,
                                                  const zd* za, const zd* zb, zd& phi, zd& ax,
                                                  zd& ay) {
    zd a[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const zd c = zconj(zb[k]);
        const double h = 0.5 * mc.inv_n;
        a[2 * k] = h * (za[k] + c);
        const zd d = za[k] - c;  // 2i F(f_2k+1)
        a[2 * k + 1] = zd{h * d.im, -h * d.re};
    }
    phi = zi(-kx * a[0]) - zi(ky * a[1]);
    ax = a[2] - zi(kx * a[4]) - zi(ky * a[5]);
    ay = a[3] - zi(kx * a[6]) - zi(ky * a[7]);
}

// Reverse BDF-k field step of mode idx = i ny + j.  Updates the history adjoints of the
// mode and returns the packed adjoint current (Jx + i Jy) q_p/(dx dy).
__device__ __forceinline__ zd adj_mode(const ModeCommon& mc, const AdjModeParams& ap, int idx,
                                       double kx, double ky, const zd* za, const zd* zb) {
    zd phis, axs, ays;
    gathered_adjoints(mc, kx, ky, za, zb, phis, axs, ays);
    phis = zl(ap.phi[0] + idx) + phis;
    axs = zl(ap.ax[0] + idx) + axs;
    ays = zl(ap.ay[0] + idx) + ays;
    // u^{n+1} = (g S - sum_d C_d u^{n+1-d}) / (C_0 + g K)
    const double inv = mc.invd[idx];
    const int L = 2 * ap.k;
    for (int d = 1; d < L; ++d) {
        const double c = ap.C[d] * inv;
        zs(ap.phi[d] + idx, zl(ap.phi[d] + idx) - c * phis);
        zs(ap.ax[d] + idx, zl(ap.ax[d] + idx) - c * axs);
        zs(ap.ay[d] + idx, zl(ap.ay[d] + idx) - c * ays);
    }
    const double cl = ap.C[L] * inv;
    zs(ap.phi[0] + idx, -(cl * phis));
    zs(ap.ax[0] + idx, -(cl * axs));
    zs(ap.ay[0] + idx, -(cl * ays));
    // rho^{n+1} = -sum_j a_j rho^{n+1-j} - beta dt i k . J   (a_0 = 1); phi's source rho/eps0
    const zd rhos = zl(ap.rho[0] + idx) + (ap.g * inv / mc.eps0) * phis;
    for (int d = 1; d < ap.k; ++d) zs(ap.rho[d] + idx, zl(ap.rho[d] + idx) - ap.a[d] * rhos);
    zs(ap.rho[0] + idx, -(ap.a[ap.k] * rhos));
    // current: -beta dt i k_l (continuity) and g mu0 / (C_0 + g K) (A's source)
    const double ga = ap.g * mc.mu0 * inv;
    const zd jx = zi(ap.bdt * kx * rhos) + ga * axs;
    const zd jy = zi(ap.bdt * ky * rhos) + ga * ays;
    // packed (Jx + i Jy), times q_p/(dx dy): the adjoint of the raw deposit sums after
    // the unnormalised inverse transform
    return mc.jscale * (jx + zi(jy));
}

// Reverse CDF-2 field step of mode idx (section 3.1; form 0 implicit, 1 semi-implicit,
// 2 explicit).  cp holds the adjoints of the levels after the step by role (cur, prev);
// the adjoints of the levels before it are written into the other buffer of each pair
// (cur into prev, prev into cur), so the host swaps each pair after the launch, the
// mirror of the forward's swap.  The particles' phi~ = (phi^{n+3/2} + phi^{n+1/2})/2.
__device__ __forceinline__ zd adj_mode(const ModeCommon& mc, const CdfParams& cp, int idx,
                                       double kx, double ky, const zd* za, const zd* zb) {
    auto L = [&](void* p) { return zl(reinterpret_cast<const double2*>(p) + idx); };
    auto S = [&](void* p, zd v) { zs(reinterpret_cast<double2*>(p) + idx, v); };
    zd phic, axc, ayc;
    gathered_adjoints(mc, kx, ky, za, zb, phic, axc, ayc);
    const zd phin = L(cp.phi) + 0.5 * phic;   // phi^{n+3/2}
    zd phih = L(cp.phi_prev) + 0.5 * phic;    // phi^{n+1/2}
    zd rhon = L(cp.rho), rhoh = L(cp.rho_prev);
    const zd axn = L(cp.ax) + axc, ayn = L(cp.ay) + ayc;  // A^{n+1}
    zd axh = L(cp.ax_prev), ayh = L(cp.ay_prev);          // A^n
    zd jxn = L(cp.jx), jyn = L(cp.jy);                    // J^{n+1} (this step's)
    zd jxh = L(cp.jx_prev), jyh = L(cp.jy_prev);          // J^n
    zd rhop{0.0, 0.0}, jxp{0.0, 0.0}, jyp{0.0, 0.0};      // the oldest levels read
    const double dt = mc.dt, h2 = mc.c * mc.c * dt * dt;
    if (cp.form == 0) {
        // u^{n+1} = inv (2 u^n + th (S^{n+1} + S^{n-1})) - u^{n-1}, th = c^2 dt^2 / 2
        const double inv = mc.invd[idx], ts = inv * 0.5 * h2;
        phih = phih + (2.0 * inv) * phin;
        rhon = rhon + (ts / mc.eps0) * phin;
        rhop = (ts / mc.eps0) * phin;
        axh = axh + (2.0 * inv) * axn;
        ayh = ayh + (2.0 * inv) * ayn;
        jxn = jxn + (ts * mc.mu0) * axn;
        jyn = jyn + (ts * mc.mu0) * ayn;
        jxp = (ts * mc.mu0) * axn;
        jyp = (ts * mc.mu0) * ayn;
    } else {
        // semi: u^{n+1} = inv (2 u^n + c^2 dt^2 S^n) - u^{n-1};
        // explicit: u^{n+1} = (2 - c^2 dt^2 K) u^n - u^{n-1} + c^2 dt^2 S^n
        const double K = kx * kx + ky * ky;
        const double inv = cp.form == 1 ? mc.invd[idx] : 1.0;
        const double mu = cp.form == 1 ? 2.0 * inv : 2.0 - h2 * K, ss = inv * h2;
        phih = phih + mu * phin;
        rhoh = rhoh + (ss / mc.eps0) * phin;
        axh = axh + mu * axn;
        ayh = ayh + mu * ayn;
        jxh = jxh + (ss * mc.mu0) * axn;
        jyh = jyh + (ss * mc.mu0) * ayn;
    }
    // rho^{n+3/2} = rho^{n+1/2} - dt i k . J^{n+1}
    rhoh = rhoh + rhon;
    jxn = jxn + zi(dt * kx * rhon);
    jyn = jyn + zi(dt * ky * rhon);
    S(cp.phi_prev, phih);
    S(cp.phi, -phin);
    S(cp.rho_prev, rhoh);
    S(cp.rho, rhop);
    S(cp.ax_prev, axh);
    S(cp.ax, -axn);
    S(cp.ay_prev, ayh);
    S(cp.ay, -ayn);
    S(cp.jx_prev, jxh);
    S(cp.jx, jxp);
    S(cp.jy_prev, jyh);
    S(cp.jy, jyp);
    return mc.jscale * (jxn + zi(jyn));
}

// Reverse DIRK field step of mode idx (section 3.3): dp's state pointers hold the
// adjoints of the state after the step (phi, v_phi, A, v_A, rho, J^{n+1}), overwritten in
// place with those of the state before it (J^n in the J slots).
__device__ __forceinline__ zd adj_mode(const ModeCommon& mc, const DirkParams& dp, int idx,
                                       double kx, double ky, const zd* za, const zd* zb) {
    auto L = [&](void* p) { return zl(reinterpret_cast<const double2*>(p) + idx); };
    auto S = [&](void* p, zd v) { zs(reinterpret_cast<double2*>(p) + idx, v); };
    zd phic, axc, ayc;
    gathered_adjoints(mc, kx, ky, za, zb, phic, axc, ayc);
    // the forward's step matrix of this mode (mc.dirkm, built once from the stage
    // recurrence on unit inputs): the step is that linear map, so its transpose is exact
    double M[2][4];
    const double* Mf = mc.dirkm + (size_t)idx * 8;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        M[0][k] = __ldg(Mf + k);
        M[1][k] = __ldg(Mf + 4 + k);
    }
    const zd phiu = L(dp.phi) + phic, phiv = L(dp.vphi);
    const zd axu = L(dp.ax) + axc, axv = L(dp.vax);
    const zd ayu = L(dp.ay) + ayc, ayv = L(dp.vay);
    // transpose: input i gets M[0][i] u_bar' + M[1][i] v_bar'
    S(dp.phi, M[0][0] * phiu + M[1][0] * phiv);
    S(dp.vphi, M[0][1] * phiu + M[1][1] * phiv);
    S(dp.ax, M[0][0] * axu + M[1][0] * axv);
    S(dp.vax, M[0][1] * axu + M[1][1] * axv);
    S(dp.ay, M[0][0] * ayu + M[1][0] * ayv);
    S(dp.vay, M[0][1] * ayu + M[1][1] * ayv);
    // phi's sources rho^n/eps0 and rho^{n+1}/eps0; A's mu0 J^n and mu0 J^{n+1}
    const zd rhon = L(dp.rho) + (M[0][3] / mc.eps0) * phiu + (M[1][3] / mc.eps0) * phiv;
    // rho^{n+1} = rho^n - dt (r0 i k . J^n + r1 i k . J^{n+1})
    S(dp.rho, rhon + (M[0][2] / mc.eps0) * phiu + (M[1][2] / mc.eps0) * phiv);
    const double dt = mc.dt;
    const zd jxn = L(dp.jx) + mc.mu0 * (M[0][3] * axu + M[1][3] * axv) + zi(dt * dp.r1 * kx * rhon);
    const zd jyn = L(dp.jy) + mc.mu0 * (M[0][3] * ayu + M[1][3] * ayv) + zi(dt * dp.r1 * ky * rhon);
    S(dp.jx, mc.mu0 * (M[0][2] * axu + M[1][2] * axv) + zi(dt * dp.r0 * kx * rhon));
    S(dp.jy, mc.mu0 * (M[0][2] * ayu + M[1][2] * ayv) + zi(dt * dp.r0 * ky * rhon));
    return mc.jscale * (jxn + zi(jyn));
}

// One thread per mode over the transformed planes Zb (four planes of nx ny).
template <typename Params>
__global__ void __launch_bounds__(kModeThreads)
k_adj_modes(ModeCommon mc, Params ap, const double2* __restrict__ Zb, double2* __restrict__ Js) {
    const int ng = mc.nx * mc.ny;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ng) return;
    const int i = idx / mc.ny, j = idx - i * mc.ny;
    const int ip = (i == 0) ? 0 : mc.nx - i;
    const int jp = (j == 0) ? 0 : mc.ny - j;
    const int idm = ip * mc.ny + jp;
    zd za[4], zb[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        za[k] = zl(Zb + (size_t)k * ng + idx);
        zb[k] = zl(Zb + (size_t)k * ng + idm);
    }
    zs(Js + idx, adj_mode(mc, ap, idx, mc.kxt[i], mc.kyt[j], za, zb));
}

// Fused column pass of the reverse field step.  CTA j loads columns j and ny - j (mod ny)
// of the four row-transformed planes, transforms them along x in shared memory, updates
// the modes of column j and transforms column j of the adjoint current back along x;
// the caller finishes with the inverse transform along y.
template <typename Params>
__global__ void __launch_bounds__(kModeThreads)
k_adj_columns(ModeCommon mc, Params ap, const double2* __restrict__ Zb,
              double2* __restrict__ Js, FftDesc fd, const double2* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = mc.nx, ny = mc.ny;
    const size_t ng = (size_t)nx * ny;
    const int j = blockIdx.x;
    const int jp = (j == 0) ? 0 : ny - j;
    const int ncols = (jp == j) ? 1 : 2;
    double2* bufA = reinterpret_cast<double2*>(smem_raw);  // 8 lines of nx: line c*4 + k
    double2* bufB = bufA + 8 * nx;
    double2* tws = bufB + 8 * nx;
    stage_twiddles(tw, tws, nx);
    for (int t = threadIdx.x; t < 4 * ncols * nx; t += blockDim.x) {
        const int l = t / nx, i = t - l * nx;
        const int c = l >> 2, k = l & 3;
        bufA[t] = Zb[k * ng + (size_t)i * ny + (c ? jp : j)];
    }
    __syncthreads();
    double2* zc = run_passes(bufA, bufB, fd, 4 * ncols, (const double2*)tws, -1);
    double2* out = (zc == bufA) ? bufB : bufA;
    const double2* zp = zc + (size_t)(ncols - 1) * 4 * nx;
    const double ky = mc.kyt[j];
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const int ip = (i == 0) ? 0 : nx - i;
        zd za[4], zb[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            za[k] = zl(zc + k * nx + i);
            zb[k] = zl(zp + k * nx + ip);
        }
        zs(out + i, adj_mode(mc, ap, i * ny + j, mc.kxt[i], ky, za, zb));
    }
    __syncthreads();
    double2* res = run_passes(out, zc, fd, 1, (const double2*)tws, +1);
    for (int i = threadIdx.x; i < nx; i += blockDim.x) Js[(size_t)i * ny + j] = res[i];
}

// Final-level seed of an objective sum bzb B_z: B_z = IDFT(i kx Ay - i ky Ax), so
// Ay b += -i kx DFT(bzb)/N and Ax b += i ky DFT(bzb)/N.
__global__ void __launch_bounds__(kModeThreads)
k_adj_seed(ModeCommon mc, const double2* __restrict__ zs_, double2* __restrict__ ax,
           double2* __restrict__ ay) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= mc.nx * mc.ny) return;
    const int i = idx / mc.ny, j = idx - i * mc.ny;
    const double kx = mc.kxt[i], ky = mc.kyt[j];
    const zd z = mc.inv_n * zl(zs_ + idx);
    zs(ay + idx, zl(ay + idx) - zi(kx * z));
    zs(ax + idx, zl(ax + idx) + zi(ky * z));
}

// (Ex + i Ey)/(nx ny) of E = -grad phi, for an inverse transform to the mesh E^0.
__global__ void __launch_bounds__(kModeThreads)
k_adj_e0(ModeCommon mc, const double2* __restrict__ phi, double2* __restrict__ out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= mc.nx * mc.ny) return;
    const int i = idx / mc.ny, j = idx - i * mc.ny;
    const double kx = mc.kxt[i], ky = mc.kyt[j];
    const zd ph = zl(phi + idx);
    const zd ex = -zi(kx * ph), ey = -zi(ky * ph);
    zs(out + idx, mc.inv_n * (ex + zi(ey)));
}

// dst[k n + i] = src.p[k][i] (pack) or dst.p[k][i] = src[k n + i] (unpack), k = blockIdx.y.
template <typename T>
__global__ void k_pack8(Ptr8T<T> src, T* __restrict__ dst, int64_t n) {
    const T* s = src.p[blockIdx.y];
    T* d = dst + (size_t)blockIdx.y * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        d[i] = s[i];
}
template <typename T>
__global__ void k_unpack8(const T* __restrict__ src, Ptr8T<T> dst, int64_t n) {
    const T* s = src + (size_t)blockIdx.y * n;
    T* d = const_cast<T*>(dst.p[blockIdx.y]);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        d[i] = s[i];
}

__global__ void k_real_to_cplx(const double* __restrict__ src, double2* __restrict__ dst,
                               int64_t n) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        dst[p] = make_double2(src[p], 0.0);
}

// t = 0: P^0 = gamma m v^0 and v^{-1} = v^0 - kappa (E - v (v . E)/c^2), kappa =
// dt q/(gamma m), E = E^0 gathered at x^0.  Gradient with respect to v^0 (gv) and, with
// P^0 as the independent variable, with respect to P^0 (gp = (dv/dP)^T gv).
template <typename T, int P>
__global__ void __launch_bounds__(kThreads)
k_adj_init(ParticleGeom g, PushParams pp, const T* __restrict__ x0, const T* __restrict__ y0,
           const T* __restrict__ vx0, const T* __restrict__ vy0, const double2* __restrict__ E,
           AdjParticlesT<T> ab, double* __restrict__ gvx, double* __restrict__ gvy,
           double* __restrict__ gpx, double* __restrict__ gpy, int64_t n,
           unsigned int* __restrict__ err) {
    const T c2 = (T)(pp.c * pp.c), m = (T)pp.m;
    const T idx_ = (T)g.inv_dx, idy = (T)g.inv_dy;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const T xi = x0[p] * idx_, yj = y0[p] * idy;
        if (!inside(xi, g.nx) || !inside(yj, g.ny)) {
            atomicOr(err, (unsigned)ERR_NONFINITE);
            continue;
        }
        T wx[P + 1], wy[P + 1];
        const int ix = Shape<P, T>::weights(xi, wx);
        const int iy = Shape<P, T>::weights(yj, wy);
        T ex = 0, ey = 0;
#pragma unroll
        for (int a = 0; a <= P; ++a) {
            const size_t row = (size_t)wrap_idx(ix + a, g.nx) * g.ny;
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                const double2 e = E[row + wrap_idx(iy + b, g.ny)];
                const T w = wx[a] * wy[b];
                ex += w * (T)e.x;
                ey += w * (T)e.y;
            }
        }
        const T vx = vx0[p], vy = vy0[p];
        const T gam = (T)1 / sqrt((T)1 - (vx * vx + vy * vy) / c2);
        // dP/dv = gamma m (I + gamma^2 v v^T / c^2)
        const T pbx = ab.px[p], pby = ab.py[p];
        const T pvb = vx * pbx + vy * pby;
        T gx = ab.vx[p] + gam * m * (pbx + gam * gam * vx * pvb / c2);
        T gy = ab.vy[p] + gam * m * (pby + gam * gam * vy * pvb / c2);
        // v^{-1}: transpose of I + kappa gamma^2 T v^T / c^2 + kappa (v E^T + (v.E) I)/c^2
        const T wxb = ab.vxo[p], wyb = ab.vyo[p];
        const T kap = (T)(pp.dt * pp.q) / (gam * m);
        const T vde = vx * ex + vy * ey;
        const T tx = ex - vx * vde / c2, ty = ey - vy * vde / c2;
        const T tw = tx * wxb + ty * wyb, vw = vx * wxb + vy * wyb;
        gx += wxb + kap * gam * gam * vx * tw / c2 + (kap / c2) * (ex * vw + vde * wxb);
        gy += wyb + kap * gam * gam * vy * tw / c2 + (kap / c2) * (ey * vw + vde * wyb);
        if (gvx) gvx[p] = (double)gx;
        if (gvy) gvy[p] = (double)gy;
        // dv/dP = (I - v v^T / c^2) / (gamma m)
        const T vg = vx * gx + vy * gy;
        if (gpx) gpx[p] = (double)((gx - vx * vg / c2) / (gam * m));
        if (gpy) gpy[p] = (double)((gy - vy * vg / c2) / (gam * m));
    }
}

// The FP32 form's field adjoints, [node][2] float4 (fields 0-3, 4-7), to the four FP64
// planes of the reverse field solve: plane k holds fields (2k, 2k + 1) of each node.
__global__ void k_fb32_to_planes(const float4* __restrict__ fb32, double2* __restrict__ Fb,
                                 int64_t ng) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ng;
         k += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = fb32[2 * k], b = fb32[2 * k + 1];
        Fb[k] = make_double2(a.x, a.y);
        Fb[ng + k] = make_double2(a.z, a.w);
        Fb[2 * ng + k] = make_double2(b.x, b.y);
        Fb[3 * ng + k] = make_double2(b.z, b.w);
    }
}

inline int mode_blocks(const ModeCommon& mc) {
    return (mc.nx * mc.ny + kModeThreads - 1) / kModeThreads;
}

}  // namespace

#define GPIC_ADJ_DISPATCH(p, KERNEL, ...)                                                  \
    switch (p) {                                                                         \
        case 2: KERNEL<T, 2><<<blocks_for(n), kThreads, 0, s>>>(__VA_ARGS__); break;    \
        case 3: KERNEL<T, 3><<<blocks_for(n), kThreads, 0, s>>>(__VA_ARGS__); break;    \
        case 4: KERNEL<T, 4><<<blocks_for(n), kThreads, 0, s>>>(__VA_ARGS__); break;    \
        default: return cudaErrorInvalidValue;                                          \
    }

template <typename T>
cudaError_t launch_adj_push_gather(int p, const ParticleGeom& g, const PushParams& pp,
                                   const T* x1, const T* y1, const T* px1, const T* py1,
                                   const T* vx, const T* vy, const T* vxo, const T* vyo,
                                   const double* gf, bool lean, const void* F,
                                   AdjParticlesT<T> ab, double2* Fb, void* fb32, int64_t n,
                                   unsigned int* err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (sizeof(T) == 4 && !fb32) return cudaErrorInvalidValue;
    const double* gfa = lean ? nullptr : gf + 4 * n;  // the gathered values of the record
    GPIC_ADJ_DISPATCH(p, k_adj_push_gather, g, pp, x1, y1, px1, py1, vx, vy, vxo, vyo, gfa,
                      (const cplx_t<T>*)F, ab, Fb, (float4*)fb32, n, err)
    return cudaGetLastError();
}

cudaError_t launch_fb32_to_planes(const void* fb32, double2* Fb, int64_t ng, cudaStream_t s) {
    k_fb32_to_planes<<<blocks_for(ng), kThreads, 0, s>>>((const float4*)fb32, Fb, ng);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_deposit_move(int p, const ParticleGeom& g, const T* x1, const T* y1,
                                    const T* vx, const T* vy, const double2* Jb,
                                    AdjParticlesT<T> ab, int64_t n, unsigned int* err,
                                    cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    GPIC_ADJ_DISPATCH(p, k_adj_deposit_move, g, x1, y1, vx, vy, Jb, ab, n, err)
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_init(int p, const ParticleGeom& g, const PushParams& pp, const T* x0,
                            const T* y0, const T* vx0, const T* vy0, const double2* E,
                            AdjParticlesT<T> ab, double* gvx, double* gvy, double* gpx,
                            double* gpy, int64_t n, unsigned int* err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    GPIC_ADJ_DISPATCH(p, k_adj_init, g, pp, x0, y0, vx0, vy0, E, ab, gvx, gvy, gpx, gpy, n, err)
    return cudaGetLastError();
}

template <typename Params>
cudaError_t adj_modes(const ModeCommon& mc, const Params& ap, const double2* Zb, double2* Js,
                      cudaStream_t s) {
    k_adj_modes<Params><<<mode_blocks(mc), kModeThreads, 0, s>>>(mc, ap, Zb, Js);
    return cudaGetLastError();
}

cudaError_t launch_adj_modes(const ModeCommon& mc, int kind, const AdjModeParams& ap,
                             const CdfParams& cp, const DirkParams& dp, const double2* Zb,
                             double2* Js, cudaStream_t s) {
    if (kind == K_CDF2) return adj_modes(mc, cp, Zb, Js, s);
    if (kind == K_DIRK) return adj_modes(mc, dp, Zb, Js, s);
    return adj_modes(mc, ap, Zb, Js, s);
}

size_t adj_columns_smem(int nx) { return 17 * (size_t)nx * sizeof(double2); }

template <typename Params>
cudaError_t adj_columns(const ModeCommon& mc, const Params& ap, const double2* Zb, double2* Js,
                        const FftDesc& fd, const double2* tw, cudaStream_t s) {
    const size_t sm = adj_columns_smem(mc.nx);
    cudaError_t e = cudaFuncSetAttribute(k_adj_columns<Params>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_adj_columns<Params><<<mc.ny, kModeThreads, sm, s>>>(mc, ap, Zb, Js, fd, tw);
    return cudaGetLastError();
}

cudaError_t launch_adj_columns(const ModeCommon& mc, int kind, const AdjModeParams& ap,
                               const CdfParams& cp, const DirkParams& dp, const double2* Zb,
                               double2* Js, const FftDesc& fd, const double2* tw,
                               cudaStream_t s) {
    if (kind == K_CDF2) return adj_columns(mc, cp, Zb, Js, fd, tw, s);
    if (kind == K_DIRK) return adj_columns(mc, dp, Zb, Js, fd, tw, s);
    return adj_columns(mc, ap, Zb, Js, fd, tw, s);
}

cudaError_t launch_adj_seed(const ModeCommon& mc, const double2* zs_, double2* ax, double2* ay,
                            cudaStream_t s) {
    k_adj_seed<<<mode_blocks(mc), kModeThreads, 0, s>>>(mc, zs_, ax, ay);
    return cudaGetLastError();
}

cudaError_t launch_adj_e0(const ModeCommon& mc, const double2* phi, double2* out, cudaStream_t s) {
    k_adj_e0<<<mode_blocks(mc), kModeThreads, 0, s>>>(mc, phi, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pack8(Ptr8T<T> src, T* dst, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int bx = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 2);
    k_pack8<T><<<dim3(bx, 8), kThreads, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_unpack8(const T* src, Ptr8T<T> dst, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int bx = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 2);
    k_unpack8<T><<<dim3(bx, 8), kThreads, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_real_to_cplx(const double* src, double2* dst, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_real_to_cplx<<<blocks_for(n), kThreads, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

#define GPIC_ADJ_INST(T)                                                                    \
    template cudaError_t launch_adj_push_gather<T>(                                         \
        int, const ParticleGeom&, const PushParams&, const T*, const T*, const T*, const T*, \
        const T*, const T*, const T*, const T*, const double*, bool, const void*,            \
        AdjParticlesT<T>, double2*, void*, int64_t, unsigned int*, cudaStream_t);           \
    template cudaError_t launch_adj_deposit_move<T>(int, const ParticleGeom&, const T*,     \
                                                    const T*, const T*, const T*,           \
                                                    const double2*, AdjParticlesT<T>,       \
                                                    int64_t, unsigned int*, cudaStream_t);  \
    template cudaError_t launch_adj_init<T>(int, const ParticleGeom&, const PushParams&,    \
                                            const T*, const T*, const T*, const T*,         \
                                            const double2*, AdjParticlesT<T>, double*,      \
                                            double*, double*, double*, int64_t,             \
                                            unsigned int*, cudaStream_t);                   \
    template cudaError_t launch_pack8<T>(Ptr8T<T>, T*, int64_t, cudaStream_t);              \
    template cudaError_t launch_unpack8<T>(const T*, Ptr8T<T>, int64_t, cudaStream_t);
GPIC_ADJ_INST(double)
GPIC_ADJ_INST(float)
#undef GPIC_ADJ_INST

}  // namespace gpic
