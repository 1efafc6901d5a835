// Per-mode field solve: charge from continuity, implicit wave update of phi, Ax, Ay
// and the spectral gradients the particles gather, one thread per Fourier mode.
//
// With the spectral discretisation every mode k evolves independently (the
// Laplacian becomes -K, K = |k|^2, and the inverse of L = I - alpha^-2 Laplacian is a
// division), so the time steppers of section 3 reduce to short scalar recurrences:
//   BDF-k   (section 3.2):  rho^{n+1} = -sum_{j>=1} a_j rho^{n+1-j} - beta dt i k.J^{n+1}
//                           u^{n+1} = (g S^{n+1} - sum_{d>=1} C_d u^{n+1-d}) / (C_0 + g K),
//                           g = (c beta dt)^2, C = coefficients of the twice-applied BDF
//   CDF-2   (section 3.1):  rho^{n+3/2} = rho^{n+1/2} - dt i k.J^{n+1}
//                           u^{n+1} = (2u^n + th (S^{n+1} + S^{n-1}))/(1 + th K) - u^{n-1},
//                           th = c^2 dt^2 / 2
//   DIRK-s  (section 3.3):  rho^{n+1} = rho^n - h sum_i b_i i k.J^(i); stage pairs solved
//                           with d_i = 1 + (h a_ii c)^2 K
// All coefficients and the recurrences run in FP64, and the time histories are stored in
// FP64 in both precision forms; only the transform inputs/outputs use the storage type C.
// The packed current spectrum Z = FFT(Jx + i Jy) is split with the Hermitian pair
// (k, -k):  Jx = (Z(k) + conj Z(-k))/2,  Jy = (Z(k) - conj Z(-k))/(2i).
// Outputs are four packed spectra whose inverse FFTs give the real field pairs
// (dphi/dx, dphi/dy), (Ax, Ay), (dAx/dx, dAx/dy), (dAy/dx, dAy/dy).
#include "common.cuh"
#include "gpic_internal.h"

namespace gpic {

namespace {

constexpr int kModeThreads = 256;

struct ModeIn {
    int idx;
    double kx, ky, K;
    zd jx, jy, divj;
};

template <typename C>
__device__ __forceinline__ ModeIn mode_in(const ModeCommon& mc, const C* z, int idx) {
    ModeIn m;
    m.idx = idx;
    int i = idx / mc.ny, j = idx - i * mc.ny;
    int ip = (i == 0) ? 0 : mc.nx - i;
    int jp = (j == 0) ? 0 : mc.ny - j;
    m.kx = wavenumber(i, mc.nx, mc.kx_scale);
    m.ky = wavenumber(j, mc.ny, mc.ky_scale);
    m.K = m.kx * m.kx + m.ky * m.ky;
    if (z) {
        zd a = zload(z + idx);
        zd b = zconj(zload(z + (ip * mc.ny + jp)));
        double hs = 0.5 * mc.jscale;
        m.jx = hs * (a + b);
        zd d = a - b;  // = 2i Jy / jscale
        m.jy = zd{hs * d.im, -hs * d.re};
        m.divj = zi(m.kx * m.jx + m.ky * m.jy);
    } else {
        m.jx = m.jy = m.divj = zd{0, 0};
    }
    return m;
}

__device__ __forceinline__ zd div2(double kx, double ky, zd ax, zd ay) {
    return zi(kx * ax + ky * ay);
}

// (i kx - ky) u : the packed gradient (du/dx) + i (du/dy).
__device__ __forceinline__ zd grad_packed(double kx, double ky, zd u) {
    return zi(kx * u) - ky * u;
}

template <typename C>
__device__ __forceinline__ void store_outputs(const ModeCommon& mc, C* f4, int idx, double kx,
                                              double ky, zd phit, zd ax, zd ay) {
    const size_t N = (size_t)mc.nx * mc.ny;
    const double s = mc.inv_n;
    zstore(f4 + idx, s * grad_packed(kx, ky, phit));
    zstore(f4 + N + idx, s * (ax + zi(ay)));
    zstore(f4 + 2 * N + idx, s * grad_packed(kx, ky, ax));
    zstore(f4 + 3 * N + idx, s * grad_packed(kx, ky, ay));
}

// Block-wide sum of D_NSLOTS accumulators, then one atomicAdd per slot.
__device__ void reduce_diag(double* acc, double* diag) {
    __shared__ double red[kModeThreads / 32][D_NSLOTS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < D_NSLOTS; ++s) {
        double v = acc[s];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][s] = v;
    }
    __syncthreads();
    if (threadIdx.x < D_NSLOTS) {
        double v = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
        if (v != 0.0) atomicAdd(diag + threadIdx.x, v);
    }
}

__device__ __forceinline__ void diag_fields(double* acc, const ModeCommon& mc, double kx,
                                            double ky, zd ex, zd ey, zd ax, zd ay) {
    acc[D_WE] += znorm2(ex) + znorm2(ey);
    zd bz = zi(kx * ay) - zi(ky * ax);
    acc[D_WB] += znorm2(bz);
    acc[D_DIVA] += znorm2(div2(kx, ky, ax, ay));
}

template <typename C>
__global__ void __launch_bounds__(kModeThreads)
k_mode_bdf(ModeCommon mc, BdfParams bp, const C* __restrict__ z, C* __restrict__ f4,
           C* __restrict__ epk, double* __restrict__ diag) {
    const int nmodes = mc.nx * mc.ny;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[D_NSLOTS];
#pragma unroll
    for (int s = 0; s < D_NSLOTS; ++s) acc[s] = 0.0;
    if (idx < nmodes) {
        ModeIn m = mode_in(mc, z, idx);
        const int k = bp.k;
        zd rho_new = -bp.bdt * m.divj;
        for (int d = 1; d <= k; ++d) rho_new = rho_new - bp.a[d] * zload((const double2*)bp.rho[d - 1] + idx);
        rho_new = (1.0 / bp.a[0]) * rho_new;
        const double inv = 1.0 / (bp.C[0] + bp.g * m.K);
        zd sphi = (bp.g / mc.eps0) * rho_new;
        zd sax = (bp.g * mc.mu0) * m.jx;
        zd say = (bp.g * mc.mu0) * m.jy;
        for (int d = 1; d <= 2 * k; ++d) {
            sphi = sphi - bp.C[d] * zload((const double2*)bp.phi[d - 1] + idx);
            sax = sax - bp.C[d] * zload((const double2*)bp.ax[d - 1] + idx);
            say = say - bp.C[d] * zload((const double2*)bp.ay[d - 1] + idx);
        }
        zd phi_new = inv * sphi, ax_new = inv * sax, ay_new = inv * say;
        if (mc.diag) {
            // section 3.2: gauge eps_1, continuity eps_2, and Gauss with
            // E^{n+1} = -grad phi^{n+1} - (1/(beta dt)) sum_j a_j A^{n+1-j}
            zd dphi = bp.a[0] * phi_new, dax = bp.a[0] * ax_new, day = bp.a[0] * ay_new;
            zd drho = bp.a[0] * rho_new;
            for (int d = 1; d <= k; ++d) {
                dphi = dphi + bp.a[d] * zload((const double2*)bp.phi[d - 1] + idx);
                dax = dax + bp.a[d] * zload((const double2*)bp.ax[d - 1] + idx);
                day = day + bp.a[d] * zload((const double2*)bp.ay[d - 1] + idx);
                drho = drho + bp.a[d] * zload((const double2*)bp.rho[d - 1] + idx);
            }
            const double ibdt = 1.0 / bp.bdt;
            zd diva = div2(m.kx, m.ky, ax_new, ay_new);
            zd gauge = (ibdt / (mc.c * mc.c)) * dphi + diva;
            zd cont = ibdt * drho + m.divj;
            zd ex = -zi(m.kx * phi_new) - ibdt * dax;
            zd ey = -zi(m.ky * phi_new) - ibdt * day;
            zd rs = (1.0 / mc.eps0) * rho_new;
            zd gauss = div2(m.kx, m.ky, ex, ey) - rs;
            acc[D_GAUGE] += znorm2(gauge);
            acc[D_CONT] += znorm2(cont);
            acc[D_GAUSS] += znorm2(gauss);
            acc[D_RHO] += znorm2(rs);
            diag_fields(acc, mc, m.kx, m.ky, ex, ey, ax_new, ay_new);
            zstore(epk + idx, mc.inv_n * (ex + zi(ey)));
        }
        zstore((double2*)bp.rho_new + idx, rho_new);
        zstore((double2*)bp.phi_new + idx, phi_new);
        zstore((double2*)bp.ax_new + idx, ax_new);
        zstore((double2*)bp.ay_new + idx, ay_new);
        store_outputs(mc, f4, idx, m.kx, m.ky, phi_new, ax_new, ay_new);
    }
    if (mc.diag) reduce_diag(acc, diag);
}

template <typename C>
__global__ void __launch_bounds__(kModeThreads)
k_mode_cdf2(ModeCommon mc, CdfParams cp, const C* __restrict__ z, C* __restrict__ f4,
            C* __restrict__ epk, double* __restrict__ diag) {
    const int nmodes = mc.nx * mc.ny;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[D_NSLOTS];
#pragma unroll
    for (int s = 0; s < D_NSLOTS; ++s) acc[s] = 0.0;
    if (idx < nmodes) {
        ModeIn m = mode_in(mc, z, idx);
        const double dt = mc.dt;
        const double th = 0.5 * mc.c * mc.c * dt * dt;
        const double inv = 1.0 / (1.0 + th * m.K);
        zd phi = zload((const double2*)cp.phi + idx), phi_prev = zload((const double2*)cp.phi_prev + idx);
        zd rho = zload((const double2*)cp.rho + idx), rho_prev = zload((const double2*)cp.rho_prev + idx);
        zd ax = zload((const double2*)cp.ax + idx), ax_prev = zload((const double2*)cp.ax_prev + idx);
        zd ay = zload((const double2*)cp.ay + idx), ay_prev = zload((const double2*)cp.ay_prev + idx);
        zd jx_prev = zload((const double2*)cp.jx_prev + idx), jy_prev = zload((const double2*)cp.jy_prev + idx);
        zd rho_new = rho - dt * m.divj;                                    // rho^{n+3/2}
        zd phi_new = inv * (2.0 * phi + (th / mc.eps0) * (rho_new + rho_prev)) - phi_prev;
        zd ax_new = inv * (2.0 * ax + (th * mc.mu0) * (m.jx + jx_prev)) - ax_prev;
        zd ay_new = inv * (2.0 * ay + (th * mc.mu0) * (m.jy + jy_prev)) - ay_prev;
        if (mc.diag) {
            // section 3.1: eps_1^{n+1}, eps_2^{n+1} and Gauss at t^{n+1/2}
            zd diva = div2(m.kx, m.ky, ax_new, ay_new);
            zd gauge = (1.0 / (mc.c * mc.c * dt)) * (phi_new - phi) + diva;
            zd cont = (1.0 / dt) * (rho_new - rho) + m.divj;
            zd pavg = 0.5 * (phi_new + phi_prev);
            zd ex = -zi(m.kx * pavg) - (1.0 / dt) * (ax_new - ax);
            zd ey = -zi(m.ky * pavg) - (1.0 / dt) * (ay_new - ay);
            zd rs = (0.5 / mc.eps0) * (rho_new + rho_prev);
            zd gauss = div2(m.kx, m.ky, ex, ey) - rs;
            acc[D_GAUGE] += znorm2(gauge);
            acc[D_CONT] += znorm2(cont);
            acc[D_GAUSS] += znorm2(gauss);
            acc[D_RHO] += znorm2((1.0 / mc.eps0) * rho_new);
            diag_fields(acc, mc, m.kx, m.ky, ex, ey, ax_new, ay_new);
            zstore(epk + idx, mc.inv_n * (ex + zi(ey)));
        }
        zstore((double2*)cp.phi_prev + idx, phi_new);
        zstore((double2*)cp.rho_prev + idx, rho_new);
        zstore((double2*)cp.ax_prev + idx, ax_new);
        zstore((double2*)cp.ay_prev + idx, ay_new);
        zstore((double2*)cp.jx_prev + idx, m.jx);
        zstore((double2*)cp.jy_prev + idx, m.jy);
        store_outputs(mc, f4, idx, m.kx, m.ky, 0.5 * (phi_new + phi), ax_new, ay_new);
    }
    if (mc.diag) reduce_diag(acc, diag);
}

// One s-stage DIRK step of d/dt (v, u) = (c^2 (S - K u), v) for one mode (section 3.3.1).
__device__ __forceinline__ void dirk_mode(const DirkParams& dp, double K, double c, double h,
                                          zd u, zd v, zd sn, zd snew, zd& uo, zd& vo) {
    zd ku[kMaxDirk], kv[kMaxDirk];
    const double c2 = c * c;
    uo = u;
    vo = v;
    for (int i = 0; i < dp.s; ++i) {
        zd ub = u, vb = v;
        for (int j = 0; j < i; ++j) {
            ub = ub + (h * dp.a[i * kMaxDirk + j]) * ku[j];
            vb = vb + (h * dp.a[i * kMaxDirk + j]) * kv[j];
        }
        zd src = (1.0 - dp.c[i]) * sn + dp.c[i] * snew;
        const double gam = h * dp.a[i * kMaxDirk + i];
        const double d = 1.0 / (1.0 + (gam * c) * (gam * c) * K);
        zd force = c2 * (src - K * ub);
        ku[i] = d * (vb + gam * force);
        kv[i] = d * (force - (gam * c2 * K) * vb);
    }
    for (int i = 0; i < dp.s; ++i) {
        uo = uo + (h * dp.b[i]) * ku[i];
        vo = vo + (h * dp.b[i]) * kv[i];
    }
}

template <typename C>
__global__ void __launch_bounds__(kModeThreads)
k_mode_dirk(ModeCommon mc, DirkParams dp, const C* __restrict__ z, C* __restrict__ f4,
            C* __restrict__ epk, double* __restrict__ diag) {
    const int nmodes = mc.nx * mc.ny;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[D_NSLOTS];
#pragma unroll
    for (int s = 0; s < D_NSLOTS; ++s) acc[s] = 0.0;
    if (idx < nmodes) {
        ModeIn m = mode_in(mc, z, idx);
        const double h = mc.dt;
        zd phi = zload((const double2*)dp.phi + idx), vphi = zload((const double2*)dp.vphi + idx);
        zd ax = zload((const double2*)dp.ax + idx), vax = zload((const double2*)dp.vax + idx);
        zd ay = zload((const double2*)dp.ay + idx), vay = zload((const double2*)dp.vay + idx);
        zd rho = zload((const double2*)dp.rho + idx);
        zd jxn = zload((const double2*)dp.jx + idx), jyn = zload((const double2*)dp.jy + idx);
        zd divjn = div2(m.kx, m.ky, jxn, jyn);
        zd rho_new = rho;
        for (int i = 0; i < dp.s; ++i)
            rho_new = rho_new - (h * dp.b[i]) * ((1.0 - dp.c[i]) * divjn + dp.c[i] * m.divj);
        zd phi_new, vphi_new, ax_new, vax_new, ay_new, vay_new;
        const double ie = 1.0 / mc.eps0;
        dirk_mode(dp, m.K, mc.c, h, phi, vphi, ie * rho, ie * rho_new, phi_new, vphi_new);
        dirk_mode(dp, m.K, mc.c, h, ax, vax, mc.mu0 * jxn, mc.mu0 * m.jx, ax_new, vax_new);
        dirk_mode(dp, m.K, mc.c, h, ay, vay, mc.mu0 * jyn, mc.mu0 * m.jy, ay_new, vay_new);
        if (mc.diag) {
            // section 3.3.2: eps_1, eps_2 and eps_3; Gauss with E = -grad phi - v_A (reported only)
            const double c2h = mc.c * mc.c * h;
            zd diva_n = div2(m.kx, m.ky, ax, ay), diva = div2(m.kx, m.ky, ax_new, ay_new);
            zd divva_n = div2(m.kx, m.ky, vax, vay), divva = div2(m.kx, m.ky, vax_new, vay_new);
            zd gauge = -(phi_new - phi) - c2h * (dp.r0 * diva_n + dp.r1 * diva);
            zd gauge_dt = -(vphi_new - vphi) - c2h * (dp.r0 * divva_n + dp.r1 * divva);
            zd cont = -(rho_new - rho) - h * (dp.r0 * divjn + dp.r1 * m.divj);
            zd ex = -zi(m.kx * phi_new) - vax_new;
            zd ey = -zi(m.ky * phi_new) - vay_new;
            zd rs = ie * rho_new;
            zd gauss = div2(m.kx, m.ky, ex, ey) - rs;
            acc[D_GAUGE] += znorm2(gauge);
            acc[D_GAUGE_DT] += znorm2(gauge_dt);
            acc[D_CONT] += znorm2(cont);
            acc[D_GAUSS] += znorm2(gauss);
            acc[D_RHO] += znorm2(rs);
            diag_fields(acc, mc, m.kx, m.ky, ex, ey, ax_new, ay_new);
            zstore(epk + idx, mc.inv_n * (ex + zi(ey)));
        }
        zstore((double2*)dp.phi + idx, phi_new);
        zstore((double2*)dp.vphi + idx, vphi_new);
        zstore((double2*)dp.ax + idx, ax_new);
        zstore((double2*)dp.vax + idx, vax_new);
        zstore((double2*)dp.ay + idx, ay_new);
        zstore((double2*)dp.vay + idx, vay_new);
        zstore((double2*)dp.rho + idx, rho_new);
        zstore((double2*)dp.jx + idx, m.jx);
        zstore((double2*)dp.jy + idx, m.jy);
        store_outputs(mc, f4, idx, m.kx, m.ky, phi_new, ax_new, ay_new);
    }
    if (mc.diag) reduce_diag(acc, diag);
}

// t = 0: rho^0 (deposited charge, K = 0 modes removed), phi^0 from Poisson, and the
// packed E^0 = -grad phi^0 for the Taylor start of v^{-1}.
template <typename C>
__global__ void __launch_bounds__(kModeThreads)
k_mode_init(ModeCommon mc, const C* __restrict__ zq, double2* __restrict__ rho_out,
            double2* __restrict__ phi_out, C* __restrict__ epk) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= mc.nx * mc.ny) return;
    ModeIn m = mode_in(mc, zq, idx);
    zd rho = (m.K > 0.0) ? m.jx : zd{0.0, 0.0};
    zd phi = (m.K > 0.0) ? (1.0 / (mc.eps0 * m.K)) * rho : zd{0.0, 0.0};
    zstore(rho_out + idx, rho);
    zstore(phi_out + idx, phi);
    zd ex = -zi(m.kx * phi), ey = -zi(m.ky * phi);
    zstore(epk + idx, mc.inv_n * (ex + zi(ey)));
}

// out = inv_n * (A + i B) with (op 0) A = a, B = b, or (op 1) A = i kx b - i ky a, B = 0.
template <typename C>
__global__ void __launch_bounds__(kModeThreads)
k_mode_pack2(ModeCommon mc, const double2* __restrict__ a, const double2* __restrict__ b, int op,
             C* __restrict__ out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= mc.nx * mc.ny) return;
    zd va = a ? zload(a + idx) : zd{0, 0};
    zd vb = b ? zload(b + idx) : zd{0, 0};
    zd r;
    if (op == 1) {
        int i = idx / mc.ny, j = idx - i * mc.ny;
        double kx = wavenumber(i, mc.nx, mc.kx_scale), ky = wavenumber(j, mc.ny, mc.ky_scale);
        r = zi(kx * vb) - zi(ky * va);
    } else {
        r = va + zi(vb);
    }
    zstore(out + idx, mc.inv_n * r);
}

inline int mode_blocks(const ModeCommon& mc) {
    return (mc.nx * mc.ny + kModeThreads - 1) / kModeThreads;
}

}  // namespace

template <typename T>
cudaError_t launch_mode_bdf(const ModeCommon& mc, const BdfParams& bp, const void* z, void* f4,
                            void* e, double* diag, cudaStream_t s) {
    using C = cplx_t<T>;
    k_mode_bdf<C><<<mode_blocks(mc), kModeThreads, 0, s>>>(mc, bp, (const C*)z, (C*)f4, (C*)e, diag);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_mode_cdf2(const ModeCommon& mc, const CdfParams& cp, const void* z, void* f4,
                             void* e, double* diag, cudaStream_t s) {
    using C = cplx_t<T>;
    k_mode_cdf2<C><<<mode_blocks(mc), kModeThreads, 0, s>>>(mc, cp, (const C*)z, (C*)f4, (C*)e, diag);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_mode_dirk(const ModeCommon& mc, const DirkParams& dp, const void* z, void* f4,
                             void* e, double* diag, cudaStream_t s) {
    using C = cplx_t<T>;
    k_mode_dirk<C><<<mode_blocks(mc), kModeThreads, 0, s>>>(mc, dp, (const C*)z, (C*)f4, (C*)e, diag);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_mode_init(const ModeCommon& mc, const void* zq, void* rho, void* phi, void* e,
                             cudaStream_t s) {
    using C = cplx_t<T>;
    k_mode_init<C><<<mode_blocks(mc), kModeThreads, 0, s>>>(mc, (const C*)zq, (double2*)rho, (double2*)phi, (C*)e);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_mode_pack2(const ModeCommon& mc, const void* a, const void* b, int op,
                              void* out, cudaStream_t s) {
    using C = cplx_t<T>;
    k_mode_pack2<C><<<mode_blocks(mc), kModeThreads, 0, s>>>(mc, (const double2*)a, (const double2*)b, op, (C*)out);
    return cudaGetLastError();
}

#define GPIC_INST(T)                                                                              \
    template cudaError_t launch_mode_bdf<T>(const ModeCommon&, const BdfParams&, const void*,     \
                                            void*, void*, double*, cudaStream_t);                 \
    template cudaError_t launch_mode_cdf2<T>(const ModeCommon&, const CdfParams&, const void*,    \
                                             void*, void*, double*, cudaStream_t);                \
    template cudaError_t launch_mode_dirk<T>(const ModeCommon&, const DirkParams&, const void*,   \
                                             void*, void*, double*, cudaStream_t);                \
    template cudaError_t launch_mode_init<T>(const ModeCommon&, const void*, void*, void*, void*, \
                                             cudaStream_t);                                       \
    template cudaError_t launch_mode_pack2<T>(const ModeCommon&, const void*, const void*, int,  \
                                              void*, cudaStream_t);
GPIC_INST(double)
GPIC_INST(float)
#undef GPIC_INST

}  // namespace gpic
