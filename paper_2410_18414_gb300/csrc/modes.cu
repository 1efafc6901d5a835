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
//
// Two drivers share the per-mode code: one thread per mode over a transformed spectrum
// (k_mode_*), and the fused column kernel k_field_columns, which also performs the
// forward transform along x before the update and the inverse transforms along x of the
// four outputs after it, all in shared memory.
#include "common.cuh"
#include "fft_device.cuh"
#include "gpic_internal.h"
#include "launch.cuh"

namespace gpic {

namespace {

constexpr int kModeThreads = 256;

// Explicitly rounded complex operations for the values a step stores or outputs: the
// per-mode update is compiled in more than one context (one or two threads per mode,
// with or without diagnostics), and explicit roundings keep the compiler from fusing
// products differently in each, so every context gives the same bits.
__device__ __forceinline__ zd zscale(double s, zd a) {
    return zd{__dmul_rn(s, a.re), __dmul_rn(s, a.im)};
}
__device__ __forceinline__ zd zfms(zd a, double c, zd b) {  // a - c b
    return zd{__fma_rn(-c, b.re, a.re), __fma_rn(-c, b.im, a.im)};
}

struct ModeIn {
    int idx;  // i * ny + j
    double kx, ky, K;
    zd jx, jy, divj;
};

// Mode (i, j) from Z(k) = za and Z(-k) = zb.
__device__ __forceinline__ ModeIn make_mode(const ModeCommon& mc, int i, int j, zd za, zd zb) {
    ModeIn m;
    m.idx = i * mc.ny + j;
    m.kx = mc.kxt[i];
    m.ky = mc.kyt[j];
    m.K = m.kx * m.kx + m.ky * m.ky;
    const zd b = zconj(zb);
    const double hs = 0.5 * mc.jscale;
    m.jx = zscale(hs, zd{__dadd_rn(za.re, b.re), __dadd_rn(za.im, b.im)});
    const zd d = zd{__dsub_rn(za.re, b.re), __dsub_rn(za.im, b.im)};  // = 2i Jy / jscale
    m.jy = zd{__dmul_rn(hs, d.im), __dmul_rn(-hs, d.re)};
    m.divj = zi(zd{__fma_rn(m.ky, m.jy.re, __dmul_rn(m.kx, m.jx.re)),
                   __fma_rn(m.ky, m.jy.im, __dmul_rn(m.kx, m.jx.im))});
    return m;
}

__device__ __forceinline__ ModeIn make_mode(const ModeCommon& mc, int i, int j, double2 za,
                                            double2 zb) {
    return make_mode(mc, i, j, zd{za.x, za.y}, zd{zb.x, zb.y});
}
// FP32 form: Jx, Jy unpacked in FP32 (the transforms are FP32) and converted exactly;
// div J is then formed in FP64 from those same values, so the continuity and gauge
// identities of the FP64 recurrences hold to FP64 roundoff.
__device__ __forceinline__ ModeIn make_mode(const ModeCommon& mc, int i, int j, float2 za,
                                            float2 zb) {
    ModeIn m;
    m.idx = i * mc.ny + j;
    m.kx = mc.kxt[i];
    m.ky = mc.kyt[j];
    m.K = m.kx * m.kx + m.ky * m.ky;
    const float hs = (float)(0.5 * mc.jscale);
    const float2 b = make_float2(zb.x, -zb.y);
    m.jx = zd{__fmul_rn(hs, __fadd_rn(za.x, b.x)), __fmul_rn(hs, __fadd_rn(za.y, b.y))};
    const float dre = __fsub_rn(za.x, b.x), dim = __fsub_rn(za.y, b.y);  // 2i Jy / jscale
    m.jy = zd{__fmul_rn(hs, dim), __fmul_rn(-hs, dre)};
    m.divj = zi(zd{__fma_rn(m.ky, m.jy.re, __dmul_rn(m.kx, m.jx.re)),
                   __fma_rn(m.ky, m.jy.im, __dmul_rn(m.kx, m.jx.im))});
    return m;
}

template <typename C>
__device__ __forceinline__ ModeIn mode_from_global(const ModeCommon& mc, const C* z, int idx) {
    const int i = idx / mc.ny, j = idx - i * mc.ny;
    const int ip = (i == 0) ? 0 : mc.nx - i;
    const int jp = (j == 0) ? 0 : mc.ny - j;
    if (!z) {
        ModeIn m = make_mode(mc, i, j, zd{0, 0}, zd{0, 0});
        return m;
    }
    return make_mode(mc, i, j, z[idx], z[ip * mc.ny + jp]);
}

__device__ __forceinline__ zd div2(double kx, double ky, zd ax, zd ay) {
    return zi(kx * ax + ky * ay);
}

// (i kx - ky) u : the packed gradient (du/dx) + i (du/dy).
__device__ __forceinline__ zd grad_packed(double kx, double ky, zd u) {
    return zd{__fma_rn(-ky, u.re, __dmul_rn(-kx, u.im)), __fma_rn(-ky, u.im, __dmul_rn(kx, u.re))};
}
// s (ax + i ay)
__device__ __forceinline__ zd packed_a(double s, zd ax, zd ay) {
    return zd{__dmul_rn(s, __dsub_rn(ax.re, ay.im)), __dmul_rn(s, __dadd_rn(ax.im, ay.re))};
}

// The four packed output spectra of one mode, with the inverse-FFT factor 1/(nx ny):
// (i kx - ky) phi, ax + i ay, (i kx - ky) ax, (i kx - ky) ay.  FP64 for the FP64 form;
// FP32 from the FP64 fields for the FP32 form, whose transforms and gather are FP32.
__device__ __forceinline__ void packed_outputs(const ModeCommon& mc, const ModeIn& m, zd phit,
                                               zd ax, zd ay, double2* out) {
    const double s = mc.inv_n;
    const zd o[4] = {zscale(s, grad_packed(m.kx, m.ky, phit)), packed_a(s, ax, ay),
                     zscale(s, grad_packed(m.kx, m.ky, ax)), zscale(s, grad_packed(m.kx, m.ky, ay))};
#pragma unroll
    for (int f = 0; f < 4; ++f) out[f] = make_double2(o[f].re, o[f].im);
}
__device__ __forceinline__ float2 grad_packed_f(float s, float kx, float ky, float2 u) {
    return make_float2(__fmul_rn(s, __fmaf_rn(-ky, u.x, __fmul_rn(-kx, u.y))),
                       __fmul_rn(s, __fmaf_rn(-ky, u.y, __fmul_rn(kx, u.x))));
}
__device__ __forceinline__ void packed_outputs(const ModeCommon& mc, const ModeIn& m, zd phit,
                                               zd ax, zd ay, float2* out) {
    const float s = (float)mc.inv_n, kx = (float)m.kx, ky = (float)m.ky;
    const float2 p = make_float2((float)phit.re, (float)phit.im);
    const float2 a = make_float2((float)ax.re, (float)ax.im);
    const float2 b = make_float2((float)ay.re, (float)ay.im);
    out[0] = grad_packed_f(s, kx, ky, p);
    out[1] = make_float2(__fmul_rn(s, __fsub_rn(a.x, b.y)), __fmul_rn(s, __fadd_rn(a.y, b.x)));
    out[2] = grad_packed_f(s, kx, ky, a);
    out[3] = grad_packed_f(s, kx, ky, b);
}

// Block-wide sum of D_NSLOTS accumulators, then one atomicAdd per slot (256 threads).
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

__device__ __forceinline__ void diag_fields(double* acc, double kx, double ky, zd ex, zd ey,
                                            zd ax, zd ay) {
    acc[D_WE] += znorm2(ex) + znorm2(ey);
    zd bz = zi(kx * ay) - zi(ky * ax);
    acc[D_WB] += znorm2(bz);
    acc[D_DIVA] += znorm2(div2(kx, ky, ax, ay));
}

__device__ __forceinline__ zd hload(const void* p, int idx) {
    return zload(reinterpret_cast<const double2*>(p) + idx);
}
__device__ __forceinline__ void hstore(void* p, int idx, zd v) {
    zstore(reinterpret_cast<double2*>(p) + idx, v);
}

// ---------------------------------------------------------------- BDF-k ----

// rho^{n+1} of the naive update: the deposited charge's spectrum in density units, its
// K = 0 modes removed as at t = 0 (reading R15).
template <typename C>
__device__ __forceinline__ zd deposited_rho(const ModeCommon& mc, const ModeIn& m) {
    if (m.K == 0.0) return zd{0.0, 0.0};
    return zscale(mc.jscale, zload(reinterpret_cast<const C*>(mc.zq) + m.idx));
}

// The BDF order a kernel is compiled for: K in 1..kMaxBdf fixes it (loops unroll and every
// history load of a mode is issued at once), K = 0 takes it from the parameters.
template <int K> struct BdfOrder {
    BdfParams p;
};
template <int K>
__device__ __forceinline__ int bdf_k(const BdfParams& bp) {
    return K > 0 ? K : bp.k;
}

// The BDF-k recurrences of one mode: continuity and the phi wave update; the A wave
// updates.
template <int K = 0>
__device__ __forceinline__ void bdf_rho_phi(const ModeCommon& mc, const BdfParams& bp,
                                            const ModeIn& m, zd& rho_new, zd& phi_new,
                                            const zd* rho_dep = nullptr) {
    const int idx = m.idx, k = bdf_k<K>(bp);
    rho_new = zscale(-bp.bdt, m.divj);
#pragma unroll
    for (int d = 1; d <= k; ++d) rho_new = zfms(rho_new, bp.a[d], hload(bp.rho[d - 1], idx));
    rho_new = zscale(bp.inv_a0, rho_new);
    if (rho_dep) rho_new = *rho_dep;  // the naive update: the deposited charge
    zd sphi = zscale(bp.g_eps0, rho_new);
#pragma unroll
    for (int d = 1; d <= 2 * k; ++d) sphi = zfms(sphi, bp.C[d], hload(bp.phi[d - 1], idx));
    phi_new = zscale(mc.invd[idx], sphi);  // 1/(C_0 + g K)
}
template <int K = 0>
__device__ __forceinline__ void bdf_a(const ModeCommon& mc, const BdfParams& bp, const ModeIn& m,
                                      zd& ax_new, zd& ay_new) {
    const int idx = m.idx, k = bdf_k<K>(bp);
    zd sax = zscale(bp.g * mc.mu0, m.jx);
    zd say = zscale(bp.g * mc.mu0, m.jy);
#pragma unroll
    for (int d = 1; d <= 2 * k; ++d) {
        sax = zfms(sax, bp.C[d], hload(bp.ax[d - 1], idx));
        say = zfms(say, bp.C[d], hload(bp.ay[d - 1], idx));
    }
    const double inv = mc.invd[idx];
    ax_new = zscale(inv, sax);
    ay_new = zscale(inv, say);
}

template <int K, typename C>
__device__ __forceinline__ void bdf_mode_update(const ModeCommon& mc, const BdfParams& bp,
                                                const ModeIn& m, double* acc, C* epk, C* out);

template <typename C>
__device__ __forceinline__ void mode_update(const ModeCommon& mc, const BdfParams& bp,
                                            const ModeIn& m, double* acc, C* epk, C* out) {
    bdf_mode_update<0>(mc, bp, m, acc, epk, out);
}
template <int K, typename C>
__device__ __forceinline__ void mode_update(const ModeCommon& mc, const BdfOrder<K>& bo,
                                            const ModeIn& m, double* acc, C* epk, C* out) {
    bdf_mode_update<K>(mc, bo.p, m, acc, epk, out);
}

template <int K, typename C>
__device__ __forceinline__ void bdf_mode_update(const ModeCommon& mc, const BdfParams& bp,
                                                const ModeIn& m, double* acc, C* epk, C* out) {
    const int idx = m.idx, k = bdf_k<K>(bp);
    zd rho_new, phi_new, ax_new, ay_new;
    zd rho_dep;
    if (mc.zq) rho_dep = deposited_rho<C>(mc, m);
    bdf_rho_phi<K>(mc, bp, m, rho_new, phi_new, mc.zq ? &rho_dep : nullptr);
    bdf_a<K>(mc, bp, m, ax_new, ay_new);
    if (mc.diag) {
        // section 3.2: gauge eps_1, continuity eps_2, and Gauss with
        // E^{n+1} = -grad phi^{n+1} - (1/(beta dt)) sum_j a_j A^{n+1-j}
        zd dphi = bp.a[0] * phi_new, dax = bp.a[0] * ax_new, day = bp.a[0] * ay_new;
        zd drho = bp.a[0] * rho_new;
#pragma unroll
        for (int d = 1; d <= k; ++d) {
            dphi = dphi + bp.a[d] * hload(bp.phi[d - 1], idx);
            dax = dax + bp.a[d] * hload(bp.ax[d - 1], idx);
            day = day + bp.a[d] * hload(bp.ay[d - 1], idx);
            drho = drho + bp.a[d] * hload(bp.rho[d - 1], idx);
        }
        const double ibdt = 1.0 / bp.bdt;
        const zd diva = div2(m.kx, m.ky, ax_new, ay_new);
        const zd gauge = (ibdt / (mc.c * mc.c)) * dphi + diva;
        const zd cont = ibdt * drho + m.divj;
        const zd ex = -zi(m.kx * phi_new) - ibdt * dax;
        const zd ey = -zi(m.ky * phi_new) - ibdt * day;
        const zd rs = mc.inv_eps0 * rho_new;
        const zd gauss = div2(m.kx, m.ky, ex, ey) - rs;
        acc[D_GAUGE] += znorm2(gauge);
        acc[D_CONT] += znorm2(cont);
        acc[D_GAUSS] += znorm2(gauss);
        acc[D_RHO] += znorm2(rs);
        diag_fields(acc, m.kx, m.ky, ex, ey, ax_new, ay_new);
        zstore(epk + idx, mc.inv_n * (ex + zi(ey)));
    }
    hstore(bp.rho_new, idx, rho_new);
    hstore(bp.phi_new, idx, phi_new);
    hstore(bp.ax_new, idx, ax_new);
    hstore(bp.ay_new, idx, ay_new);
    packed_outputs(mc, m, phi_new, ax_new, ay_new, out);
}

// ---------------------------------------------------------------- CDF-2 ----

template <typename C>
__device__ __forceinline__ void mode_update(const ModeCommon& mc, const CdfParams& cp,
                                            const ModeIn& m, double* acc, C* epk, C* out) {
    const int idx = m.idx;
    const double dt = mc.dt;
    const double th = 0.5 * mc.c * mc.c * dt * dt;
    const double inv = mc.invd[idx];  // 1/(1 + th K)
    const zd phi = hload(cp.phi, idx), phi_prev = hload(cp.phi_prev, idx);
    const zd rho = hload(cp.rho, idx), rho_prev = hload(cp.rho_prev, idx);
    const zd ax = hload(cp.ax, idx), ax_prev = hload(cp.ax_prev, idx);
    const zd ay = hload(cp.ay, idx), ay_prev = hload(cp.ay_prev, idx);
    const zd jx_prev = hload(cp.jx_prev, idx), jy_prev = hload(cp.jy_prev, idx);
    const zd rho_new = rho - dt * m.divj;  // rho^{n+3/2}
    zd phi_new, ax_new, ay_new;
    if (cp.form == 0) {  // implicit: sources averaged over the new and the oldest level
        phi_new = inv * (2.0 * phi + mc.cdf_th_eps0 * (rho_new + rho_prev)) - phi_prev;
        ax_new = inv * (2.0 * ax + (th * mc.mu0) * (m.jx + jx_prev)) - ax_prev;
        ay_new = inv * (2.0 * ay + (th * mc.mu0) * (m.jy + jy_prev)) - ay_prev;
    } else {  // sources at the middle level: rho^{n+1/2} and J^n
        const double h2 = mc.c * mc.c * dt * dt;
        const zd jx_n = hload(cp.jx, idx), jy_n = hload(cp.jy, idx);
        const zd sphi = mc.inv_eps0 * rho, sax = mc.mu0 * jx_n, say = mc.mu0 * jy_n;
        if (cp.form == 1) {  // semi-implicit: Laplacian averaged over levels n+1, n-1
            phi_new = inv * (2.0 * phi + h2 * sphi) - phi_prev;
            ax_new = inv * (2.0 * ax + h2 * sax) - ax_prev;
            ay_new = inv * (2.0 * ay + h2 * say) - ay_prev;
        } else {  // explicit: Laplacian at level n
            phi_new = 2.0 * phi - phi_prev + h2 * (sphi - m.K * phi);
            ax_new = 2.0 * ax - ax_prev + h2 * (sax - m.K * ax);
            ay_new = 2.0 * ay - ay_prev + h2 * (say - m.K * ay);
        }
    }
    if (mc.diag) {
        // section 3.1: eps_1^{n+1}, eps_2^{n+1} and Gauss at t^{n+1/2}
        const zd diva = div2(m.kx, m.ky, ax_new, ay_new);
        const zd gauge = (1.0 / (mc.c * mc.c * dt)) * (phi_new - phi) + diva;
        const zd cont = (1.0 / dt) * (rho_new - rho) + m.divj;
        const zd pavg = 0.5 * (phi_new + phi_prev);
        const zd ex = -zi(m.kx * pavg) - (1.0 / dt) * (ax_new - ax);
        const zd ey = -zi(m.ky * pavg) - (1.0 / dt) * (ay_new - ay);
        const zd rs = (0.5 / mc.eps0) * (rho_new + rho_prev);
        const zd gauss = div2(m.kx, m.ky, ex, ey) - rs;
        acc[D_GAUGE] += znorm2(gauge);
        acc[D_CONT] += znorm2(cont);
        acc[D_GAUSS] += znorm2(gauss);
        acc[D_RHO] += znorm2(mc.inv_eps0 * rho_new);
        diag_fields(acc, m.kx, m.ky, ex, ey, ax_new, ay_new);
        zstore(epk + idx, mc.inv_n * (ex + zi(ey)));
    }
    hstore(cp.phi_prev, idx, phi_new);
    hstore(cp.rho_prev, idx, rho_new);
    hstore(cp.ax_prev, idx, ax_new);
    hstore(cp.ay_prev, idx, ay_new);
    hstore(cp.jx_prev, idx, m.jx);
    hstore(cp.jy_prev, idx, m.jy);
    packed_outputs(mc, m, 0.5 * (phi_new + phi), ax_new, ay_new, out);
}

// ---------------------------------------------------------------- DIRK-s ---

// One s-stage DIRK step of d/dt (v, u) = (c^2 (S - K u), v) for one mode (section 3.3.1).
// dinv[i * stride] = 1/(1 + (h a_ii c)^2 K) for stage i.
__device__ __forceinline__ void dirk_mode(const DirkParams& dp, double K, double c, double h,
                                          const double* dinv, size_t stride, zd u, zd v, zd sn,
                                          zd snew, zd& uo, zd& vo) {
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
        const zd src = (1.0 - dp.c[i]) * sn + dp.c[i] * snew;
        const double gam = h * dp.a[i * kMaxDirk + i];
        const double d = dinv[i * stride];
        const zd force = c2 * (src - K * ub);
        ku[i] = d * (vb + gam * force);
        kv[i] = d * (force - (gam * c2 * K) * vb);
    }
    for (int i = 0; i < dp.s; ++i) {
        uo = uo + (h * dp.b[i]) * ku[i];
        vo = vo + (h * dp.b[i]) * kv[i];
    }
}

// The DIRK step of one mode as its matrix (mc.dirkm): u' = M_0 . (u, v, sn, snew),
// v' = M_1 . (u, v, sn, snew).  The stage recurrence is linear in those four inputs with
// real coefficients that depend on K alone, so the matrix, built once per mode from the
// recurrence on unit inputs, is the step (to the rounding of its build).
__device__ __forceinline__ void dirk_apply(const double* __restrict__ M, zd u, zd v, zd sn,
                                           zd snew, zd& uo, zd& vo) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(M)),
                  b = __ldg(reinterpret_cast<const double2*>(M) + 1),
                  c = __ldg(reinterpret_cast<const double2*>(M) + 2),
                  d = __ldg(reinterpret_cast<const double2*>(M) + 3);
    uo = a.x * u + a.y * v + b.x * sn + b.y * snew;
    vo = c.x * u + c.y * v + d.x * sn + d.y * snew;
}

template <typename C>
__device__ __forceinline__ void mode_update(const ModeCommon& mc, const DirkParams& dp,
                                            const ModeIn& m, double* acc, C* epk, C* out) {
    const int idx = m.idx;
    const double h = mc.dt;
    const zd phi = hload(dp.phi, idx), vphi = hload(dp.vphi, idx);
    const zd ax = hload(dp.ax, idx), vax = hload(dp.vax, idx);
    const zd ay = hload(dp.ay, idx), vay = hload(dp.vay, idx);
    const zd rho = hload(dp.rho, idx);
    const zd jxn = hload(dp.jx, idx), jyn = hload(dp.jy, idx);
    const zd divjn = div2(m.kx, m.ky, jxn, jyn);
    // continuity: the stages' sum of b_i ((1 - c_i) div J^n + c_i div J^{n+1}) in closed
    // form, r0 = sum b_i (1 - c_i), r1 = sum b_i c_i
    zd rho_new = rho - (h * dp.r0) * divjn - (h * dp.r1) * m.divj;
    if (mc.zq) rho_new = deposited_rho<C>(mc, m);  // the naive update
    zd phi_new, vphi_new, ax_new, vax_new, ay_new, vay_new;
    const double ie = mc.inv_eps0;
    const double* M = mc.dirkm + (size_t)idx * 8;
    dirk_apply(M, phi, vphi, ie * rho, ie * rho_new, phi_new, vphi_new);
    dirk_apply(M, ax, vax, mc.mu0 * jxn, mc.mu0 * m.jx, ax_new, vax_new);
    dirk_apply(M, ay, vay, mc.mu0 * jyn, mc.mu0 * m.jy, ay_new, vay_new);
    if (mc.diag) {
        // section 3.3.2: eps_1, eps_2 and eps_3; Gauss with E = -grad phi - v_A (reported only)
        const double c2h = mc.c * mc.c * h;
        const zd diva_n = div2(m.kx, m.ky, ax, ay), diva = div2(m.kx, m.ky, ax_new, ay_new);
        const zd divva_n = div2(m.kx, m.ky, vax, vay), divva = div2(m.kx, m.ky, vax_new, vay_new);
        const zd gauge = -(phi_new - phi) - c2h * (dp.r0 * diva_n + dp.r1 * diva);
        const zd gauge_dt = -(vphi_new - vphi) - c2h * (dp.r0 * divva_n + dp.r1 * divva);
        const zd cont = -(rho_new - rho) - h * (dp.r0 * divjn + dp.r1 * m.divj);
        const zd ex = -zi(m.kx * phi_new) - vax_new;
        const zd ey = -zi(m.ky * phi_new) - vay_new;
        const zd rs = ie * rho_new;
        const zd gauss = div2(m.kx, m.ky, ex, ey) - rs;
        acc[D_GAUGE] += znorm2(gauge);
        acc[D_GAUGE_DT] += znorm2(gauge_dt);
        acc[D_CONT] += znorm2(cont);
        acc[D_GAUSS] += znorm2(gauss);
        acc[D_RHO] += znorm2(rs);
        diag_fields(acc, m.kx, m.ky, ex, ey, ax_new, ay_new);
        zstore(epk + idx, mc.inv_n * (ex + zi(ey)));
    }
    hstore(dp.phi, idx, phi_new);
    hstore(dp.vphi, idx, vphi_new);
    hstore(dp.ax, idx, ax_new);
    hstore(dp.vax, idx, vax_new);
    hstore(dp.ay, idx, ay_new);
    hstore(dp.vay, idx, vay_new);
    hstore(dp.rho, idx, rho_new);
    hstore(dp.jx, idx, m.jx);
    hstore(dp.jy, idx, m.jy);
    packed_outputs(mc, m, phi_new, ax_new, ay_new, out);
}

// ------------------------------------------------------------- drivers -----

// One thread per mode over the transformed current spectrum z.
template <typename C, typename Params>
__global__ void __launch_bounds__(kModeThreads)
k_mode(ModeCommon mc, Params prm, const C* __restrict__ z, C* __restrict__ f4,
       C* __restrict__ epk, double* __restrict__ diag) {
    const int nmodes = mc.nx * mc.ny;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[D_NSLOTS];
#pragma unroll
    for (int s = 0; s < D_NSLOTS; ++s) acc[s] = 0.0;
    if (idx < nmodes) {
        const ModeIn m = mode_from_global(mc, z, idx);
        C out[4];
        mode_update(mc, prm, m, acc, epk, out);
        const size_t N = (size_t)nmodes;
#pragma unroll
        for (int f = 0; f < 4; ++f) f4[f * N + idx] = out[f];
    }
    if (mc.diag) reduce_diag(acc, diag);
}

// Fused column pass.  CTA j owns column j (fixed y-index, all x-indices).  The partner
// -k of a mode of column j lies in column ny - j (mod ny), so the CTA loads both columns
// from the row-transformed current and transforms both along x, updates the modes of
// its own column, and transforms that column's four packed outputs back along x, all
// in shared memory; the caller finishes with the inverse transform along y.
// L2 prefetch of the history entries of column j's modes (a hint: the L2 is coherent,
// so it is safe while the previous kernel runs; the histories were written two or more
// kernels back).
__device__ __forceinline__ void prefetch_l2(const void* base, int idx) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const double2*>(base) + idx));
}
__device__ __forceinline__ void prefetch_history(const ModeCommon& mc, const BdfParams& bp, int j) {
    for (int i = threadIdx.x; i < mc.nx; i += blockDim.x) {
        const int idx = i * mc.ny + j;
        for (int d = 0; d < 2 * bp.k; ++d) {
            prefetch_l2(bp.phi[d], idx);
            prefetch_l2(bp.ax[d], idx);
            prefetch_l2(bp.ay[d], idx);
        }
        for (int d = 0; d < bp.k; ++d) prefetch_l2(bp.rho[d], idx);
    }
}
template <int K>
__device__ __forceinline__ void prefetch_history(const ModeCommon& mc, const BdfOrder<K>& bo,
                                                 int j) {
    prefetch_history(mc, bo.p, j);
}
__device__ __forceinline__ void prefetch_history(const ModeCommon& mc, const CdfParams& cp, int j) {
    const void* const arr[10] = {cp.phi, cp.phi_prev, cp.rho, cp.rho_prev, cp.ax,
                                 cp.ax_prev, cp.ay, cp.ay_prev, cp.jx_prev, cp.jy_prev};
    for (int i = threadIdx.x; i < mc.nx; i += blockDim.x)
        for (int a = 0; a < 10; ++a) prefetch_l2(arr[a], i * mc.ny + j);
}
__device__ __forceinline__ void prefetch_history(const ModeCommon& mc, const DirkParams& dp, int j) {
    const void* const arr[9] = {dp.phi, dp.vphi, dp.ax, dp.vax, dp.ay, dp.vay, dp.rho, dp.jx, dp.jy};
    for (int i = threadIdx.x; i < mc.nx; i += blockDim.x)
        for (int a = 0; a < 9; ++a) prefetch_l2(arr[a], i * mc.ny + j);
}

template <typename C, typename Params>
__global__ void __launch_bounds__(kModeThreads)
k_field_columns(ModeCommon mc, Params prm, const C* __restrict__ z, C* __restrict__ f4,
                C* __restrict__ epk, double* __restrict__ diag, FftDesc fd,
                const C* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = mc.nx, ny = mc.ny;
    const int j = blockIdx.x;
    const int jp = (j == 0) ? 0 : ny - j;
    const int ncols = (jp == j) ? 1 : 2;  // column j, then its partner column
    C* bufA = reinterpret_cast<C*>(smem_raw);  // 4 lines of nx
    C* bufB = bufA + 4 * nx;                   // 4 lines of nx
    C* tws = bufB + 4 * nx;                    // twiddles (constant: staged before the wait)
    stage_twiddles(tw, tws, nx);
    prefetch_history(mc, prm, j);              // written two or more kernels back
    griddep_wait();                            // z is the previous kernel's output
    griddep_launch();
    for (int t = threadIdx.x; t < ncols * nx; t += blockDim.x) {
        const int c = t / nx, i = t - c * nx;
        bufA[t] = z[(size_t)i * ny + (c ? jp : j)];
    }
    __syncthreads();
    C* zc = run_passes(bufA, bufB, fd, ncols, (const C*)tws, -1);  // forward along x
    C* out = (zc == bufA) ? bufB : bufA;               // the other buffer
    const C* zp = zc + (ncols - 1) * nx;               // partner column
    double acc[D_NSLOTS];
#pragma unroll
    for (int s = 0; s < D_NSLOTS; ++s) acc[s] = 0.0;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const int ip = (i == 0) ? 0 : nx - i;
        const ModeIn m = make_mode(mc, i, j, zc[i], zp[ip]);
        C o[4];
        mode_update(mc, prm, m, acc, epk, o);
#pragma unroll
        for (int f = 0; f < 4; ++f) out[f * nx + i] = o[f];
    }
    __syncthreads();
    C* res = run_passes(out, zc, fd, 4, (const C*)tws, +1);  // inverse along x
    const size_t N = (size_t)nx * ny;
    for (int t = threadIdx.x; t < 4 * nx; t += blockDim.x) {
        const int f = t / nx, i = t - f * nx;
        f4[f * N + (size_t)i * ny + j] = res[t];
    }
    if (mc.diag) reduce_diag(acc, diag);
}

// 2D-3V: the A_z update of mode idx (one thread per mode over zz = FFT(J_z sums)).  With
// d/dz = 0 the z component of the vector potential obeys its own wave equation with source
// mu0 J_z, stepped with the same recurrences as A_x; it enters neither the continuity
// equation nor the gauge.  E_z = -dA_z/dt is the stepper's discrete derivative (BDF: the
// BDF difference; CDF-2: the centred difference at n+1/2; DIRK: -v_Az), B_x = i ky A_z,
// B_y = -i kx A_z.
template <typename C>
__global__ void __launch_bounds__(kModeThreads)
k_zmode(ModeCommon mc, BdfParams bp, DirkParams dp, ZParams zp, const C* __restrict__ zz,
        C* __restrict__ f2, double* __restrict__ diag) {
    const int nmodes = mc.nx * mc.ny;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[D_NSLOTS];
#pragma unroll
    for (int s = 0; s < D_NSLOTS; ++s) acc[s] = 0.0;
    if (idx < nmodes) {
        const int i = idx / mc.ny, j = idx - i * mc.ny;
        const double kx = mc.kxt[i], ky = mc.kyt[j], K = kx * kx + ky * ky;
        const zd jz = zscale(mc.jscale, zload(zz + idx));
        zd az_new, ez;
        if (zp.kind == K_BDF) {
            zd s = zscale(bp.g * mc.mu0, jz);
            for (int d = 1; d <= 2 * bp.k; ++d) s = zfms(s, bp.C[d], hload(zp.az[d - 1], idx));
            az_new = zscale(mc.invd[idx], s);
            zd daz = bp.a[0] * az_new;
            for (int d = 1; d <= bp.k; ++d) daz = daz + bp.a[d] * hload(zp.az[d - 1], idx);
            ez = -(1.0 / bp.bdt) * daz;
            hstore(zp.az_new, idx, az_new);
        } else if (zp.kind == K_CDF2) {
            const double dt = mc.dt, inv = mc.invd[idx];
            const zd az = hload(zp.az_n, idx), azp = hload(zp.az_prev, idx);
            if (zp.form == 0) {
                const double th = 0.5 * mc.c * mc.c * dt * dt;
                az_new = inv * (2.0 * az + (th * mc.mu0) * (jz + hload(zp.jz_prev, idx))) - azp;
            } else {
                const double h2 = mc.c * mc.c * dt * dt;
                const zd s = mc.mu0 * hload(zp.jz_n, idx);
                az_new = (zp.form == 1) ? inv * (2.0 * az + h2 * s) - azp
                                        : 2.0 * az - azp + h2 * (s - K * az);
            }
            ez = -(1.0 / dt) * (az_new - az);
            hstore(zp.az_prev, idx, az_new);
            hstore(zp.jz_prev, idx, jz);
        } else {
            const zd az = hload(zp.az_n, idx), vaz = hload(zp.vaz, idx);
            zd vaz_new;
            dirk_apply(mc.dirkm + (size_t)idx * 8, az, vaz, mc.mu0 * hload(zp.jz_n, idx),
                       mc.mu0 * jz, az_new, vaz_new);
            ez = -vaz_new;
            hstore(zp.az_n, idx, az_new);
            hstore(zp.vaz, idx, vaz_new);
            hstore(zp.jz_n, idx, jz);
        }
        if (mc.diag) {
            acc[D_WE] += znorm2(ez);
            acc[D_WB] += K * znorm2(az_new);
        }
        zstore(f2 + idx, zscale(mc.inv_n, grad_packed(kx, ky, az_new)));
        zstore(f2 + (size_t)nmodes + idx, zscale(mc.inv_n, az_new));
    }
    if (mc.diag) reduce_diag(acc, diag);
}

__global__ void k_mode_tables(ModeCommon mc, int kind, BdfParams bp, DirkParams dp,
                              double* __restrict__ kxt, double* __restrict__ kyt,
                              double* __restrict__ invd, double* __restrict__ dirkm) {
    const int nmodes = mc.nx * mc.ny;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < mc.nx) kxt[idx] = wavenumber(idx, mc.nx, mc.kx_scale);
    if (idx < mc.ny) kyt[idx] = wavenumber(idx, mc.ny, mc.ky_scale);
    if (idx >= nmodes) return;
    const int i = idx / mc.ny, j = idx - i * mc.ny;
    const double kx = wavenumber(i, mc.nx, mc.kx_scale), ky = wavenumber(j, mc.ny, mc.ky_scale);
    const double K = kx * kx + ky * ky;
    if (kind == K_BDF) {
        invd[idx] = 1.0 / (bp.C[0] + bp.g * K);
    } else if (kind == K_CDF2) {
        const double th = 0.5 * mc.c * mc.c * mc.dt * mc.dt;
        invd[idx] = 1.0 / (1.0 + th * K);
    } else {
        double dl[kMaxDirk];
        for (int st = 0; st < dp.s; ++st) {
            const double gc = mc.dt * dp.a[st * kMaxDirk + st] * mc.c;
            dl[st] = 1.0 / (1.0 + gc * gc * K);
            invd[(size_t)st * nmodes + idx] = dl[st];
        }
        // the step matrix: the stage recurrence on the four unit inputs
        for (int k = 0; k < 4; ++k) {
            const zd e1{1.0, 0.0}, e0{0.0, 0.0};
            zd uo, vo;
            dirk_mode(dp, K, mc.c, mc.dt, dl, 1, k == 0 ? e1 : e0, k == 1 ? e1 : e0,
                      k == 2 ? e1 : e0, k == 3 ? e1 : e0, uo, vo);
            dirkm[(size_t)idx * 8 + k] = uo.re;
            dirkm[(size_t)idx * 8 + 4 + k] = vo.re;
        }
    }
}

// t = 0: rho^0 (deposited charge, K = 0 modes removed), phi^0 from Poisson, and the
// packed E^0 = -grad phi^0 for the Taylor start of v^{-1}.
template <typename C>
__global__ void __launch_bounds__(kModeThreads)
k_mode_init(ModeCommon mc, const C* __restrict__ zq, double2* __restrict__ rho_out,
            double2* __restrict__ phi_out, C* __restrict__ epk) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= mc.nx * mc.ny) return;
    const ModeIn m = mode_from_global(mc, zq, idx);
    const zd rho = (m.K > 0.0) ? m.jx : zd{0.0, 0.0};
    const zd phi = (m.K > 0.0) ? (1.0 / (mc.eps0 * m.K)) * rho : zd{0.0, 0.0};
    zstore(rho_out + idx, rho);
    zstore(phi_out + idx, phi);
    const zd ex = -zi(m.kx * phi), ey = -zi(m.ky * phi);
    zstore(epk + idx, mc.inv_n * (ex + zi(ey)));
}

// out = inv_n * (A + i B) with (op 0) A = a, B = b, (op 1) A = i kx b - i ky a, B = 0, or
// (op 2) A = i ky a, B = -i kx a (B_x, B_y of A_z = a).
template <typename C>
__global__ void __launch_bounds__(kModeThreads)
k_mode_pack2(ModeCommon mc, const double2* __restrict__ a, const double2* __restrict__ b, int op,
             C* __restrict__ out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= mc.nx * mc.ny) return;
    const zd va = a ? zload(a + idx) : zd{0, 0};
    const zd vb = b ? zload(b + idx) : zd{0, 0};
    zd r;
    if (op == 1) {
        const int i = idx / mc.ny, j = idx - i * mc.ny;
        const double kx = wavenumber(i, mc.nx, mc.kx_scale), ky = wavenumber(j, mc.ny, mc.ky_scale);
        r = zi(kx * vb) - zi(ky * va);
    } else if (op == 2) {
        const int i = idx / mc.ny, j = idx - i * mc.ny;
        const double kx = wavenumber(i, mc.nx, mc.kx_scale), ky = wavenumber(j, mc.ny, mc.ky_scale);
        r = zi(ky * va) + zi(zi(-kx * va));
    } else {
        r = va + zi(vb);
    }
    zstore(out + idx, mc.inv_n * r);
}

inline int mode_blocks(const ModeCommon& mc) {
    return (mc.nx * mc.ny + kModeThreads - 1) / kModeThreads;
}

template <typename C, typename Params>
cudaError_t launch_mode_generic(const ModeCommon& mc, const Params& prm, const void* z, void* f4,
                                void* e, double* diag, cudaStream_t s) {
    k_mode<C, Params><<<mode_blocks(mc), kModeThreads, 0, s>>>(mc, prm, (const C*)z, (C*)f4,
                                                               (C*)e, diag);
    return cudaGetLastError();
}

template <typename C, typename Params>
cudaError_t launch_columns_generic(const ModeCommon& mc, const Params& prm, const void* z,
                                   void* f4, void* e, double* diag, const FftDesc& fd,
                                   const void* tw, cudaStream_t s) {
    const size_t smem = field_columns_smem(mc.nx, sizeof(C));
    if (smem > kFieldColumnsSmemMax) return cudaErrorInvalidValue;
    auto kern = k_field_columns<C, Params>;
    if (smem > 48 * 1024) {
        cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem);
        if (e2 != cudaSuccess) return e2;
    }
    // one thread per mode of the column: grids up to 128 wide take 128-thread CTAs (one
    // step 1 us shorter at 128 x 128 than with 256, half of whose threads idle)
    const int threads = mc.nx <= 128 ? 128 : kModeThreads;
    return launch_pdl(kern, dim3(mc.ny), dim3(threads), smem, s, mc, prm, (const C*)z,
                      (C*)f4, (C*)e, diag, fd, (const C*)tw);
}

}  // namespace

template <typename T>
cudaError_t launch_mode_bdf(const ModeCommon& mc, const BdfParams& bp, const void* z, void* f4,
                            void* e, double* diag, cudaStream_t s) {
    return launch_mode_generic<cplx_t<T>>(mc, bp, z, f4, e, diag, s);
}
template <typename T>
cudaError_t launch_mode_cdf2(const ModeCommon& mc, const CdfParams& cp, const void* z, void* f4,
                             void* e, double* diag, cudaStream_t s) {
    return launch_mode_generic<cplx_t<T>>(mc, cp, z, f4, e, diag, s);
}
template <typename T>
cudaError_t launch_mode_dirk(const ModeCommon& mc, const DirkParams& dp, const void* z, void* f4,
                             void* e, double* diag, cudaStream_t s) {
    return launch_mode_generic<cplx_t<T>>(mc, dp, z, f4, e, diag, s);
}
template <typename T>
cudaError_t launch_field_columns(const ModeCommon& mc, int kind, const BdfParams& bp,
                                 const CdfParams& cp, const DirkParams& dp, const void* z,
                                 void* f4, void* e, double* diag, const FftDesc& fd,
                                 const void* tw, cudaStream_t s) {
    using C = cplx_t<T>;
    if (kind == K_BDF) {
        static_assert(kMaxBdf == 6, "one column kernel per BDF order");
        switch (bp.k) {
            case 1: return launch_columns_generic<C>(mc, BdfOrder<1>{bp}, z, f4, e, diag, fd, tw, s);
            case 2: return launch_columns_generic<C>(mc, BdfOrder<2>{bp}, z, f4, e, diag, fd, tw, s);
            case 3: return launch_columns_generic<C>(mc, BdfOrder<3>{bp}, z, f4, e, diag, fd, tw, s);
            case 4: return launch_columns_generic<C>(mc, BdfOrder<4>{bp}, z, f4, e, diag, fd, tw, s);
            case 5: return launch_columns_generic<C>(mc, BdfOrder<5>{bp}, z, f4, e, diag, fd, tw, s);
            default: return launch_columns_generic<C>(mc, BdfOrder<6>{bp}, z, f4, e, diag, fd, tw, s);
        }
    }
    if (kind == K_CDF2) return launch_columns_generic<C>(mc, cp, z, f4, e, diag, fd, tw, s);
    return launch_columns_generic<C>(mc, dp, z, f4, e, diag, fd, tw, s);
}
cudaError_t launch_mode_tables(const ModeCommon& mc, int kind, const BdfParams& bp,
                               const DirkParams& dp, double* kxt, double* kyt, double* invd,
                               double* dirkm, cudaStream_t s) {
    if (kind == K_DIRK && !dirkm) return cudaErrorInvalidValue;
    const int n = mc.nx * mc.ny > mc.nx ? mc.nx * mc.ny : mc.nx;
    k_mode_tables<<<(n + kModeThreads - 1) / kModeThreads, kModeThreads, 0, s>>>(
        mc, kind, bp, dp, kxt, kyt, invd, dirkm);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zfield(const ModeCommon& mc, const BdfParams& bp, const DirkParams& dp,
                          const ZParams& zp, const void* zz, void* f2, double* diag,
                          cudaStream_t s) {
    using C = cplx_t<T>;
    k_zmode<C><<<mode_blocks(mc), kModeThreads, 0, s>>>(mc, bp, dp, zp, (const C*)zz, (C*)f2,
                                                        diag);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mode_init(const ModeCommon& mc, const void* zq, void* rho, void* phi, void* e,
                             cudaStream_t s) {
    using C = cplx_t<T>;
    k_mode_init<C><<<mode_blocks(mc), kModeThreads, 0, s>>>(mc, (const C*)zq, (double2*)rho,
                                                            (double2*)phi, (C*)e);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_mode_pack2(const ModeCommon& mc, const void* a, const void* b, int op,
                              void* out, cudaStream_t s) {
    using C = cplx_t<T>;
    k_mode_pack2<C><<<mode_blocks(mc), kModeThreads, 0, s>>>(mc, (const double2*)a,
                                                             (const double2*)b, op, (C*)out);
    return cudaGetLastError();
}

#define GPIC_INST(T)                                                                              \
    template cudaError_t launch_mode_bdf<T>(const ModeCommon&, const BdfParams&, const void*,     \
                                            void*, void*, double*, cudaStream_t);                 \
    template cudaError_t launch_mode_cdf2<T>(const ModeCommon&, const CdfParams&, const void*,    \
                                             void*, void*, double*, cudaStream_t);                \
    template cudaError_t launch_mode_dirk<T>(const ModeCommon&, const DirkParams&, const void*,   \
                                             void*, void*, double*, cudaStream_t);                \
    template cudaError_t launch_field_columns<T>(const ModeCommon&, int, const BdfParams&,        \
                                                 const CdfParams&, const DirkParams&, const void*, \
                                                 void*, void*, double*, const FftDesc&,           \
                                                 const void*, cudaStream_t);                      \
    template cudaError_t launch_mode_init<T>(const ModeCommon&, const void*, void*, void*, void*, \
                                             cudaStream_t);                                       \
    template cudaError_t launch_zfield<T>(const ModeCommon&, const BdfParams&, const DirkParams&, \
                                          const ZParams&, const void*, void*, double*,            \
                                          cudaStream_t);                                          \
    template cudaError_t launch_mode_pack2<T>(const ModeCommon&, const void*, const void*, int,  \
                                              void*, cudaStream_t);
GPIC_INST(double)
GPIC_INST(float)
#undef GPIC_INST

}  // namespace gpic
