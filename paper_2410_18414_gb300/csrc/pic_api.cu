// Host side of the C ABI declared in include/pic.h: the simulation handle, argument
// checks, the t = 0 set-up and the three phases of one step (Algorithm 1, section 4.2).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gpic_internal.h"
#include "handle.h"
#include "pic.h"

using namespace gpic;

namespace {
thread_local std::string g_init_error;
}


namespace gpic {

nvtxDomainHandle_t nvtx_domain() {
    static const nvtxDomainHandle_t d = nvtxDomainCreateA("gpic");
    return d;
}

void nvtx_push(const char* name) {
    nvtxEventAttributes_t a = {};
    a.version = NVTX_VERSION;
    a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
    a.messageType = NVTX_MESSAGE_TYPE_ASCII;
    a.message.ascii = name;
    nvtxDomainRangePushEx(nvtx_domain(), &a);
}

const char* timer_name(int which) {
    static const char* const names[PIC_KT_COUNT] = {
        "sort", "deposit", "field_solve", "gather_push", "adj_push", "adj_field", "adj_deposit",
        "gather_deposit"};
    return which >= 0 && which < PIC_KT_COUNT ? names[which] : "?";
}

pic_status fail(pic_handle* h, pic_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h)
        h->errmsg = buf;
    else
        g_init_error = buf;
    return st;
}


cudaError_t forward_fft(pic_handle* h, const void* in, void* out) {
    return by_prec(h, [&](auto t) {
        using T = decltype(t);
        cudaError_t e = launch_fft_y<T>(in, out, h->nx, h->ny, 1, h->fy, h->twy, -1, 0, h->s);
        if (e != cudaSuccess) return e;
        return launch_fft_x<T>(out, out, h->nx, h->ny, 1, h->fx, h->twx, -1, h->s);
    });
}

// Inverse transform of nb packed spectra in `buf` (in place along x), then along y
// into `out` (interleaved by array when nb > 1).
cudaError_t inverse_fft(pic_handle* h, void* buf, void* out, int nb) {
    return by_prec(h, [&](auto t) {
        using T = decltype(t);
        cudaError_t e = launch_fft_x<T>(buf, buf, h->nx, h->ny, nb, h->fx, h->twx, +1, h->s);
        if (e != cudaSuccess) return e;
        return launch_fft_y<T>(buf, out, h->nx, h->ny, nb, h->fy, h->twy, +1, nb > 1, h->s);
    });
}

cudaError_t drop_pending(pic_handle* h) {
    if (!h->pending) return cudaSuccess;
    h->pending = false;
    return cudaMemsetAsync(h->Jalt, 0, h->ng * sizeof(double2), h->s);
}

pic_status check_device_error(pic_handle* h) {
    unsigned int e = 0;
    CK(cudaMemcpyAsync(&e, h->err, sizeof e, cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    if (e & ERR_OVERFLOW) return fail(h, PIC_ERR_OVERFLOW, "fixed-point current overflow");
    if (e & ERR_TIMEOUT) return fail(h, PIC_ERR_TIMEOUT, "a bounded device wait gave up");
    if (e & ERR_NONFINITE)
        return fail(h, PIC_ERR_NONFINITE, "non-finite or out-of-domain particle data");
    return PIC_OK;
}

}  // namespace gpic

namespace {

bool factor_23(int n, FftDesc& d) {
    d.n = n;
    d.nf = 0;
    int m = n;
    while (m % 4 == 0 && d.nf < kMaxRadices) { d.radix[d.nf++] = 4; m /= 4; }
    while (m % 2 == 0 && d.nf < kMaxRadices) { d.radix[d.nf++] = 2; m /= 2; }
    while (m % 3 == 0 && d.nf < kMaxRadices) { d.radix[d.nf++] = 3; m /= 3; }
    if (m != 1) return false;
    auto magic = [](int div) -> unsigned {  // ceil(2^32 / div); 0 marks div = 1
        return div == 1 ? 0u : (unsigned)(((1ull << 32) + div - 1) / div);
    };
    int Ns = 1;
    for (int f = 0; f < d.nf; ++f) {
        const int R = d.radix[f];
        d.ns[f] = Ns;
        d.nr[f] = n / R;
        d.twstep[f] = n / (Ns * R);
        d.m_nr[f] = magic(n / R);
        d.m_ns[f] = magic(Ns);
        Ns *= R;
    }
    return true;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

pic_status validate(const pic_config* c, const pic_particles_in* in) {
    pic_handle* h = nullptr;
    if (!c || !in) return fail(h, PIC_ERR_INVALID_ARG, "cfg and init must not be NULL");
    for (int i = 0; i < 4; ++i)
        if (c->reserved[i] != 0) return fail(h, PIC_ERR_INVALID_ARG, "reserved fields must be 0");
    if (c->tile != 0 && c->tile != 4 && c->tile != 8 && c->tile != 16)
        return fail(h, PIC_ERR_INVALID_ARG, "tile must be 0, 4, 8 or 16");
    if (c->vdim != 0 && c->vdim != 2 && c->vdim != 3)
        return fail(h, PIC_ERR_INVALID_ARG, "vdim must be 0, 2 or 3");
    if (c->nspecies < 0 || c->nspecies > kMaxSpecies)
        return fail(h, PIC_ERR_INVALID_ARG, "nspecies must be 0..%d", kMaxSpecies);
    for (int i = 0; i < c->nspecies; ++i)
        if (!std::isfinite(c->species_q[i]) || !finite_pos(c->species_m[i]) ||
            !std::isfinite(c->species_w[i]) || c->species_w[i] < 0)
            return fail(h, PIC_ERR_INVALID_ARG,
                        "species %d: q finite, m finite and > 0, weight finite and >= 0", i);
    if (c->charge != PIC_CHARGE_CONTINUITY && c->charge != PIC_CHARGE_DEPOSIT)
        return fail(h, PIC_ERR_INVALID_ARG, "unknown charge source %d", c->charge);
    if (c->charge == PIC_CHARGE_DEPOSIT &&
        (c->stepper == PIC_STEPPER_CDF2 || c->stepper == PIC_STEPPER_CDF2_SEMI ||
         c->stepper == PIC_STEPPER_CDF2_EXPLICIT))
        return fail(h, PIC_ERR_UNSUPPORTED,
                    "a deposited charge needs integer time levels: BDF-k or DIRK, not CDF-2");
    FftDesc d;
    for (int n : {c->nx, c->ny})
        if (n < 8 || n > 1024 || (n & 1) || !factor_23(n, d))
            return fail(h, PIC_ERR_INVALID_ARG,
                        "grid size %d must be even, 8..1024 and of the form 2^a 3^b", n);
    if (c->spline_order < 2 || c->spline_order > 4)
        return fail(h, PIC_ERR_INVALID_ARG, "spline_order must be 2, 3 or 4");
    if (!finite_pos(c->lx) || !finite_pos(c->ly) || !finite_pos(c->c) || !finite_pos(c->eps0) ||
        !finite_pos(c->dt) || !finite_pos(c->m) || !std::isfinite(c->q) ||
        !std::isfinite(c->weight) || c->weight < 0)
        return fail(h, PIC_ERR_INVALID_ARG,
                    "lx, ly, c, eps0, dt, m must be finite and > 0; q finite; weight >= 0");
    if (c->precision == PIC_FP32_FIX64 && (c->c < 0x1p-60 || c->c > 0x1p60))
        return fail(h, PIC_ERR_INVALID_ARG, "the FP32 form needs 2^-60 <= c <= 2^60");
    if (c->c * c->dt >= std::fmin(c->lx, c->ly))
        return fail(h, PIC_ERR_INVALID_ARG, "c*dt must be below the domain size");
    if (c->stepper == PIC_STEPPER_BDF) {
        if (c->bdf_order < 1 || c->bdf_order > kMaxBdf)
            return fail(h, PIC_ERR_INVALID_ARG, "bdf_order must be 1..6");
    } else if (c->stepper == PIC_STEPPER_DIRK) {
        const int s = c->dirk_stages;
        if (s < 1 || s > kMaxDirk) return fail(h, PIC_ERR_INVALID_ARG, "dirk_stages must be 1..4");
        for (int i = 0; i < s; ++i) {
            if (!std::isfinite(c->dirk_b[i]) || !std::isfinite(c->dirk_c[i]))
                return fail(h, PIC_ERR_INVALID_ARG, "DIRK tableau must be finite");
            for (int j = 0; j < s; ++j) {
                const double a = c->dirk_a[i * s + j];
                if (!std::isfinite(a))
                    return fail(h, PIC_ERR_INVALID_ARG, "DIRK tableau must be finite");
                if (j > i && a != 0.0)
                    return fail(h, PIC_ERR_INVALID_ARG, "DIRK matrix must be lower triangular");
                if (j == i && a < 0.0)
                    return fail(h, PIC_ERR_INVALID_ARG, "DIRK diagonal must be >= 0");
            }
        }
    } else if (c->stepper != PIC_STEPPER_CDF2 && c->stepper != PIC_STEPPER_CDF2_SEMI &&
               c->stepper != PIC_STEPPER_CDF2_EXPLICIT) {
        return fail(h, PIC_ERR_INVALID_ARG, "unknown stepper %d", c->stepper);
    }
    if (c->precision != PIC_FP64 && c->precision != PIC_FP32_FIX64)
        return fail(h, PIC_ERR_INVALID_ARG, "unknown precision %d", c->precision);
    if (c->sort_interval < 0) return fail(h, PIC_ERR_INVALID_ARG, "sort_interval must be >= 0");
    if (in->n < 0 || in->n > 2147483647LL)
        return fail(h, PIC_ERR_INVALID_ARG, "particle count must be 0..2^31-1");
    if (in->n > 0 && (!in->x || !in->y || !in->vx || !in->vy))
        return fail(h, PIC_ERR_INVALID_ARG, "particle arrays must not be NULL");
    if (in->n > 0 && c->vdim == 3 && !in->vz)
        return fail(h, PIC_ERR_INVALID_ARG, "vdim 3 needs the z velocities");
    if (in->n > 0 && c->nspecies > 0 && !in->species)
        return fail(h, PIC_ERR_INVALID_ARG, "a species table needs each particle's species");
    return PIC_OK;
}

cudaError_t dalloc(pic_handle* h, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) h->allocs.push_back(*p);
    return e;
}

void free_timers(pic_handle* h) {
    for (auto& t : h->kt) {
        for (cudaEvent_t e : t.ev) cudaEventDestroy(e);
        t.ev.clear();
        t.used = 0;
    }
}


void free_all(pic_handle* h) {
    free_timers(h);
    for (void* p : h->allocs) cudaFree(p);
    h->allocs.clear();
}

// Newest spectral level: 0 phi, 1 Ax, 2 Ay, 3 rho, 4 Az (2D-3V).
void* newest(pic_handle* h, int which) {
    if (which == 4) return h->cfg.stepper == PIC_STEPPER_BDF ? h->az_l[h->head] : h->az;
    switch (h->cfg.stepper) {
        case PIC_STEPPER_BDF:
            if (which == 3) return h->rho_l[h->head_r];
            return (which == 0 ? h->phi_l : which == 1 ? h->ax_l : h->ay_l)[h->head];
        case PIC_STEPPER_CDF2:
            return which == 0 ? h->cdf.phi : which == 1 ? h->cdf.ax : which == 2 ? h->cdf.ay : h->cdf.rho;
        default:
            return which == 0 ? h->dirk.phi : which == 1 ? h->dirk.ax : which == 2 ? h->dirk.ay : h->dirk.rho;
    }
}


pic_status alloc_state(pic_handle* h) {
    const pic_config& c = h->cfg;
    const size_t cs = 2 * h->rsz;
    const size_t pn = (size_t)std::max<int64_t>(h->n, 1) * h->rsz;
    if (!h->bound) {  // else the caller's arrays, set by pic_init_bound
        CK(dalloc(h, &h->x, pn));
        CK(dalloc(h, &h->y, pn));
        CK(dalloc(h, &h->px, pn));
        CK(dalloc(h, &h->py, pn));
        for (int b = 0; b < 2; ++b)
            for (int k = 0; k < 2; ++k) CK(dalloc(h, &h->v[b][k], pn));
    }
    CK(dalloc(h, (void**)&h->stage, (size_t)std::max<int64_t>(h->n, 1) * sizeof(double)));
    if (h->sorting) {
        const size_t ni = (size_t)std::max<int64_t>(h->n, 1) * sizeof(int);
        for (int a = 0; a < 8; ++a) CK(dalloc(h, &h->alt[a], pn));
        if (h->fp32) {  // the moved positions of a pending deposit
            CK(dalloc(h, &h->xnext, pn));
            CK(dalloc(h, &h->ynext, pn));
        }
        CK(dalloc(h, (void**)&h->id, ni));
        CK(dalloc(h, (void**)&h->id_alt, ni));
        CK(dalloc(h, (void**)&h->keys, ni));
        const size_t nt = (size_t)h->tg.nkeys() + 1;
        CK(dalloc(h, (void**)&h->hist, nt * sizeof(int)));
        CK(cudaMemsetAsync(h->hist, 0, nt * sizeof(int), h->s));  // kept zero by the sort's scan
        CK(dalloc(h, (void**)&h->off, nt * sizeof(int)));
        CK(dalloc(h, (void**)&h->cursor, nt * sizeof(int)));
        CK(dalloc(h, (void**)&h->bsum, sort_scan_chunks(h->tg.nkeys()) * sizeof(int)));
        CK(launch_iota(h->id, h->n, h->s));
    }
    if (h->vdim == 3) {
        CK(dalloc(h, &h->pz, pn));
        CK(dalloc(h, &h->vz[0], pn));
        CK(dalloc(h, &h->vz[1], pn));
        CK(dalloc(h, &h->Jz, h->jbytes));
        CK(dalloc(h, &h->Zz, h->ng * cs));
        CK(dalloc(h, &h->F2, 2 * h->ng * cs));
        CK(dalloc(h, &h->Gz, 2 * h->ng * cs));
    }
    if (h->spp.n > 0)
        CK(dalloc(h, (void**)&h->species, (size_t)std::max<int64_t>(h->n, 1) * sizeof(int32_t)));
    if (h->sorting && h->spp.n > 0)  // the sort's second set
        CK(dalloc(h, (void**)&h->species_alt,
                  (size_t)std::max<int64_t>(h->n, 1) * sizeof(int32_t)));
    if (h->sorting && h->vdim == 3)
        for (int a = 0; a < 3; ++a) CK(dalloc(h, &h->z_alt[a], pn));
    CK(dalloc(h, (void**)&h->J, h->jbytes));
    if (h->fp32) {
        CK(dalloc(h, (void**)&h->Jalt, h->ng * sizeof(double2)));
        CK(cudaMemsetAsync(h->Jalt, 0, h->ng * sizeof(double2), h->s));
    }
    CK(dalloc(h, &h->Z, h->ng * cs));
    if (h->cfg.charge == PIC_CHARGE_DEPOSIT) {
        CK(dalloc(h, &h->rhoq, h->jbytes));
        CK(dalloc(h, &h->ZQ, h->ng * cs));
        h->mc.zq = h->ZQ;
    }
    CK(dalloc(h, &h->F4, 4 * h->ng * cs));
    CK(dalloc(h, &h->G, 4 * h->ng * cs));
    CK(dalloc(h, &h->E, h->ng * cs));
    CK(dalloc(h, &h->tmp, h->ng * cs));
    CK(dalloc(h, (void**)&h->tmpd, h->ng * sizeof(double)));
    CK(dalloc(h, &h->twx, (size_t)c.nx * cs));
    CK(dalloc(h, &h->twy, (size_t)c.ny * cs));
    CK(dalloc(h, (void**)&h->diag, D_NSLOTS * sizeof(double)));
    {
        const int stages = c.stepper == PIC_STEPPER_DIRK ? c.dirk_stages : 1;
        double *kxt = nullptr, *kyt = nullptr, *invd = nullptr;
        CK(dalloc(h, (void**)&kxt, (size_t)c.nx * sizeof(double)));
        CK(dalloc(h, (void**)&kyt, (size_t)c.ny * sizeof(double)));
        CK(dalloc(h, (void**)&invd, (size_t)stages * h->ng * sizeof(double)));
        h->mc.kxt = kxt;
        h->mc.kyt = kyt;
        h->mc.invd = invd;
        h->mc.dirkm = nullptr;
        if (c.stepper == PIC_STEPPER_DIRK) {  // the per-mode step matrices
            double* dirkm = nullptr;
            CK(dalloc(h, (void**)&dirkm, 8 * h->ng * sizeof(double)));
            h->mc.dirkm = dirkm;
        }
    }
    CK(dalloc(h, (void**)&h->err, sizeof(unsigned int)));
    CK(cudaMemsetAsync(h->err, 0, sizeof(unsigned int), h->s));
    CK(cudaMemsetAsync(h->diag, 0, D_NSLOTS * sizeof(double), h->s));

    // time histories are FP64 complex spectra in both precision forms
    auto spec = [&](void** p) {
        cudaError_t e = dalloc(h, p, h->ng * sizeof(double2));
        if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, h->ng * sizeof(double2), h->s);
        return e;
    };
    if (c.stepper == PIC_STEPPER_BDF) {
        const int k = c.bdf_order;
        h->L = 2 * k;
        h->Lr = k;
        h->phi_l.assign(h->L, nullptr);
        h->ax_l.assign(h->L, nullptr);
        h->ay_l.assign(h->L, nullptr);
        h->rho_l.assign(h->Lr, nullptr);
        for (int i = 0; i < h->L; ++i) {
            CK(spec(&h->phi_l[i]));
            CK(spec(&h->ax_l[i]));
            CK(spec(&h->ay_l[i]));
        }
        for (int i = 0; i < h->Lr; ++i) CK(spec(&h->rho_l[i]));
        if (h->vdim == 3) {
            h->az_l.assign(h->L, nullptr);
            for (int i = 0; i < h->L; ++i) CK(spec(&h->az_l[i]));
        }
        // BDF-k with a_0 = 1 (section 3.2) from sum_{j=1..k} (1/j) nabla^j u = dt u'.
        double alpha[kMaxBdf + 1] = {0};
        for (int j = 1; j <= k; ++j) {
            double binom = 1.0;
            for (int i = 0; i <= j; ++i) {
                alpha[i] += ((i & 1) ? -binom : binom) / j;
                binom = binom * (j - i) / (i + 1);
            }
        }
        h->bdf.k = k;
        for (int i = 0; i <= k; ++i) h->bdf.a[i] = alpha[i] / alpha[0];
        const double beta = 1.0 / alpha[0];
        // C = a * a: coefficients of the twice-applied BDF operator (Table 1).
        for (int d = 0; d <= 2 * k; ++d) {
            double s = 0;
            for (int j = 0; j <= d; ++j)
                if (j <= k && d - j <= k) s += h->bdf.a[j] * h->bdf.a[d - j];
            h->bdf.C[d] = s;
        }
        h->bdf.bdt = beta * c.dt;
        h->bdf.inv_a0 = 1.0 / h->bdf.a[0];
        h->bdf.g = (c.c * beta * c.dt) * (c.c * beta * c.dt);
        h->bdf.g_eps0 = h->bdf.g / c.eps0;
    } else if (c.stepper == PIC_STEPPER_CDF2) {
        void** slots[] = {&h->cdf.phi, &h->cdf.phi_prev, &h->cdf.rho, &h->cdf.rho_prev,
                          &h->cdf.ax,  &h->cdf.ax_prev,  &h->cdf.ay,  &h->cdf.ay_prev,
                          &h->cdf.jx,  &h->cdf.jx_prev,  &h->cdf.jy,  &h->cdf.jy_prev};
        for (void** sl : slots) CK(spec(sl));
        if (h->vdim == 3)
            for (void** sl : {&h->az, &h->az_prev, &h->jz, &h->jz_prev}) CK(spec(sl));
    } else {
        void** slots[] = {&h->dirk.phi, &h->dirk.vphi, &h->dirk.ax, &h->dirk.vax, &h->dirk.ay,
                          &h->dirk.vay, &h->dirk.rho,  &h->dirk.jx, &h->dirk.jy};
        for (void** sl : slots) CK(spec(sl));
        if (h->vdim == 3)
            for (void** sl : {&h->az, &h->vaz, &h->jz}) CK(spec(sl));
        const int s = c.dirk_stages;
        h->dirk.s = s;
        double r0 = 0, r1 = 0;
        for (int i = 0; i < s; ++i) {
            for (int j = 0; j < s; ++j) h->dirk.a[i * kMaxDirk + j] = c.dirk_a[i * s + j];
            h->dirk.b[i] = c.dirk_b[i];
            h->dirk.c[i] = c.dirk_c[i];
            r0 += c.dirk_b[i] * (1.0 - c.dirk_c[i]);
            r1 += c.dirk_b[i] * c.dirk_c[i];
        }
        h->dirk.r0 = r0;
        h->dirk.r1 = r1;
    }
    {
        const int kind = c.stepper == PIC_STEPPER_BDF ? K_BDF : (c.stepper == PIC_STEPPER_CDF2 ? K_CDF2 : K_DIRK);
        CK(launch_mode_tables(h->mc, kind, h->bdf, h->dirk, const_cast<double*>(h->mc.kxt),
                              const_cast<double*>(h->mc.kyt), const_cast<double*>(h->mc.invd),
                              const_cast<double*>(h->mc.dirkm), h->s));
    }
    return PIC_OK;
}

// t = 0 state (Algorithm 1 set-up): wrap x^0, deposit the charge, remove its K = 0
// modes, solve Poisson for phi^0, gather E^0 = -grad phi^0 for P^0 and v^{-1}, and
// fill every history level with its t = 0 value.
pic_status setup(pic_handle* h, const pic_particles_in* in) {
    const pic_config& c = h->cfg;
    CK(by_prec(h, [&](auto t) {
        using T = decltype(t);
        cudaError_t r = launch_twiddles<T>(h->twx, c.nx, h->s);
        return r != cudaSuccess ? r : launch_twiddles<T>(h->twy, c.ny, h->s);
    }));

    const int64_t n = h->n;
    const size_t nb64 = (size_t)n * sizeof(double);
    const double* src[5] = {in->x, in->y, in->vx, in->vy, in->vz};
    void* dst[5] = {h->x, h->y, h->v[0][0], h->v[0][1], h->vz[0]};
    const int narr = h->vdim == 3 ? 5 : 4;
    if (h->spp.n > 0 && n > 0)
        CK(cudaMemcpyAsync(h->species, in->species, (size_t)n * sizeof(int32_t), cudaMemcpyDefault,
                           h->s));
    const int32_t* sp = h->spp.n > 0 ? h->species : nullptr;
    for (int i = 0; i < narr && n > 0 && !h->bound; ++i) {  // bound: in place already
        if (h->fp32) {
            CK(cudaMemcpyAsync(h->stage, src[i], nb64, cudaMemcpyDefault, h->s));
            CK(launch_convert<double, float>(h->stage, (float*)dst[i], n, h->s));
        } else {
            CK(cudaMemcpyAsync(dst[i], src[i], nb64, cudaMemcpyDefault, h->s));
        }
    }

    void* rho0 = newest(h, 3);
    void* phi0 = newest(h, 0);
    CK(cudaMemsetAsync(h->J, 0, h->jbytes, h->s));
    CK(by_prec(h, [&](auto t) -> cudaError_t {
        using T = decltype(t);
        cudaError_t r = launch_wrap_positions<T>((T*)h->x, (T*)h->y, n, c.lx, c.ly, h->s);
        if (r != cudaSuccess) return r;
        if (h->fp32) {
            r = launch_deposit_charge_fix<T>(h->p, h->geom, (const T*)h->x, (const T*)h->y, n,
                                             (longlong2*)h->J, h->fix_scale_q, h->err, h->s, sp,
                                             &h->spp);
            if (r != cudaSuccess) return r;
            r = launch_fix_to_cplx<T>((const longlong2*)h->J, h->fix_unscale_q, h->tmp, h->ng, h->s);
            if (r != cudaSuccess) return r;
            r = forward_fft(h, h->tmp, h->Z);
        } else {
            r = launch_deposit_charge_fix128(h->p, h->geom, (const double*)h->x,
                                             (const double*)h->y, n, (longlong2*)h->J, h->ng,
                                             h->fix64_scale_q, h->err, h->s, sp, &h->spp);
            if (r != cudaSuccess) return r;
            r = launch_fix128_to_cplx((const longlong2*)h->J, h->ng, h->fix64_unscale_q,
                                      (double2*)h->tmp, h->s);
            if (r != cudaSuccess) return r;
            r = forward_fft(h, h->tmp, h->Z);
        }
        if (r != cudaSuccess) return r;
        r = launch_mode_init<T>(h->mc, h->Z, rho0, phi0, h->F4, h->s);
        if (r != cudaSuccess) return r;
        r = inverse_fft(h, h->F4, h->tmp, 1);  // grid (Ex, Ey) at t = 0
        if (r != cudaSuccess) return r;
        if (h->vdim == 3 || h->spp.n > 0)
            return launch_init_particles3<T>(h->p, h->geom, h->push, (T*)h->x, (T*)h->y,
                                             (T*)h->px, (T*)h->py, (T*)h->pz, (const T*)h->v[0][0],
                                             (const T*)h->v[0][1], (const T*)h->vz[0],
                                             (T*)h->v[1][0], (T*)h->v[1][1], (T*)h->vz[1], sp,
                                             h->spp, n, h->tmp, h->err, h->s);
        return launch_init_particles<T>(h->p, h->geom, h->push, (T*)h->x, (T*)h->y, (T*)h->px,
                                        (T*)h->py, (const T*)h->v[0][0], (const T*)h->v[0][1],
                                        (T*)h->v[1][0], (T*)h->v[1][1], n, h->tmp, h->err, h->s);
    }));
    h->vcur = 0;

    const size_t bytes = h->ng * sizeof(double2);
    if (c.stepper == PIC_STEPPER_BDF) {
        for (int i = 1; i < h->L; ++i)
            CK(cudaMemcpyAsync(h->phi_l[i], phi0, bytes, cudaMemcpyDeviceToDevice, h->s));
        for (int i = 1; i < h->Lr; ++i)
            CK(cudaMemcpyAsync(h->rho_l[i], rho0, bytes, cudaMemcpyDeviceToDevice, h->s));
        h->head = 0;
        h->head_r = 0;
    } else if (c.stepper == PIC_STEPPER_CDF2) {
        CK(cudaMemcpyAsync(h->cdf.phi_prev, phi0, bytes, cudaMemcpyDeviceToDevice, h->s));
        CK(cudaMemcpyAsync(h->cdf.rho_prev, rho0, bytes, cudaMemcpyDeviceToDevice, h->s));
    }
    return check_device_error(h);
}

bool diag_due(const pic_handle* h) {
    return h->diag_every > 0 && ((h->step + 1) % h->diag_every) == 0;
}

// Particles per CTA of the binned FP32 deposit at the mean density: one batch of its
// shared-memory binning.  Measured on the 128 x 128 workload (2^20 particles, tiles of
// about 4096): 1024 a CTA (one batch each) 51 us for the fused kernel, 2048 (two batches)
// 58 us.
constexpr int kBinPerCta = 1024;

// Whether the gather + push of the step now finishing may run fused with the next step's
// move + deposit: the sorted FP32 form (2D-2V, one species) when the tile regions fit the
// fused kernel's shared memory.  A sort due at the next step then follows its deposit.
// The sorted FP32 form's deposit runs in the binned pass (with J_z in 2D-3V) when the
// tiles' regions fit its shared memory.
bool binned_deposit(const pic_handle* h) {
    return h->sorting && h->fp32 && deposit_binned_fits(h->tg, h->p, false, h->vdim == 3);
}

bool fuse_next(const pic_handle* h) {
    if (!(h->sorting && h->fp32) || h->vdim != 2) return false;
    return deposit_binned_fits(h->tg, h->p, true);
}

pic_status gather_push_step(pic_handle* h, bool fuse, bool defer);

// The tile sort.  moved = false: keyed by the positions after this step's move (the sort
// comes before the step's deposit); true: keyed by the current positions (the step's move
// and deposit are done).  The current sums do not depend on the order of the particles.
pic_status sort_particles(pic_handle* h, bool moved) {
    void** cur[8] = {&h->x, &h->y, &h->px, &h->py, &h->v[0][0], &h->v[0][1], &h->v[1][0], &h->v[1][1]};
    void** curz[3] = {&h->pz, &h->vz[0], &h->vz[1]};
    const bool z3 = h->vdim == 3, spec = h->spp.n > 0;
    CK(by_prec(h, [&](auto t) {
        using T = decltype(t);
        SortArrays<T> src, dst;
        for (int a = 0; a < 8; ++a) {
            src.a[a] = (T*)*cur[a];
            dst.a[a] = (T*)h->alt[a];
        }
        src.id = h->id;
        dst.id = h->id_alt;
        if (spec) {
            src.sp = h->species;
            dst.sp = h->species_alt;
        }
        if (z3)
            for (int a = 0; a < 3; ++a) {
                src.z[a] = (T*)*curz[a];
                dst.z[a] = (T*)h->z_alt[a];
            }
        // cur[4 + 2 vcur] is v^n_x, the velocity of this step's move
        return launch_tile_sort<T>(h->tg, src, dst, h->n, moved ? -1 : 4 + 2 * h->vcur,
                                   h->keys, h->hist, h->off, h->cursor, h->bsum, h->s);
    }));
    for (int a = 0; a < 8; ++a) std::swap(*cur[a], h->alt[a]);
    std::swap(h->id, h->id_alt);
    if (spec) std::swap(h->species, h->species_alt);
    if (z3)
        for (int a = 0; a < 3; ++a) std::swap(*curz[a], h->z_alt[a]);
    h->launches_now += 4;
    return PIC_OK;
}

}  // namespace

extern "C" {

static pic_status init_impl(const pic_config* cfg, const pic_particles_in* init,
                            const pic_particles_bound* bound, void* stream, pic_handle** out);

pic_status pic_init(const pic_config* cfg, const pic_particles_in* init, void* stream,
                    pic_handle** out) {
    return init_impl(cfg, init, nullptr, stream, out);
}

pic_status pic_init_bound(const pic_config* cfg, const pic_particles_bound* p, void* stream,
                          pic_handle** out) {
    if (out) *out = nullptr;
    if (!cfg || !p) return fail(nullptr, PIC_ERR_INVALID_ARG, "cfg and particles must not be NULL");
    if (cfg->sort_interval != 0 || (cfg->vdim != 0 && cfg->vdim != 2) || cfg->nspecies != 0)
        return fail(nullptr, PIC_ERR_UNSUPPORTED,
                    "bound particle arrays need an unsorted 2D-2V single-species configuration");
    void* const arr[8] = {p->x, p->y, p->px, p->py, p->vx, p->vy, p->vx_old, p->vy_old};
    for (int a = 0; a < 8 && p->n > 0; ++a) {
        if (!arr[a]) return fail(nullptr, PIC_ERR_INVALID_ARG, "bound particle array %d is NULL", a);
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, arr[a]) != cudaSuccess ||
            (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();  // a host pointer is not an error of the context
            return fail(nullptr, PIC_ERR_INVALID_ARG, "bound particle array %d is not device memory",
                        a);
        }
    }
    // the positions and velocities are read in place; the descriptor only carries n
    const pic_particles_in in{(const double*)p->x, (const double*)p->y, (const double*)p->vx,
                              (const double*)p->vy, p->n, nullptr, nullptr};
    return init_impl(cfg, &in, p, stream, out);
}

static pic_status init_impl(const pic_config* cfg, const pic_particles_in* init,
                            const pic_particles_bound* bound, void* stream, pic_handle** out) {
    if (!out) return fail(nullptr, PIC_ERR_INVALID_ARG, "out must not be NULL");
    *out = nullptr;
    pic_status st = validate(cfg, init);
    if (st != PIC_OK) return st;
    pic_handle* h = new pic_handle();
    h->cfg = *cfg;
    // the CDF-2 forms share its buffers and kernels; the form goes with the parameters
    int cdf_form = 0;
    if (cfg->stepper == PIC_STEPPER_CDF2_SEMI) cdf_form = 1;
    if (cfg->stepper == PIC_STEPPER_CDF2_EXPLICIT) cdf_form = 2;
    if (cdf_form) h->cfg.stepper = PIC_STEPPER_CDF2;
    h->cdf.form = cdf_form;
    h->s = (cudaStream_t)stream;
    cudaGetDevice(&h->device);
    h->nx = cfg->nx;
    h->ny = cfg->ny;
    h->ng = (size_t)cfg->nx * cfg->ny;
    h->p = cfg->spline_order;
    h->n = init->n;
    h->fp32 = cfg->precision == PIC_FP32_FIX64;
    h->rsz = h->fp32 ? 4 : 8;
    factor_23(cfg->nx, h->fx);
    factor_23(cfg->ny, h->fy);
    const double dx = cfg->lx / cfg->nx, dy = cfg->ly / cfg->ny;
    h->mc.nx = cfg->nx;
    h->mc.ny = cfg->ny;
    h->mc.kx_scale = 2.0 * M_PI / cfg->lx;
    h->mc.ky_scale = 2.0 * M_PI / cfg->ly;
    h->mc.jscale = cfg->weight * cfg->q / (dx * dy);
    h->vdim = cfg->vdim == 3 ? 3 : 2;
    double rmax = 1.0;  // bound on a deposit factor: 1, or max |q_s w_s| of a species table
    if (cfg->nspecies > 0) {
        // the deposits multiply each contribution by q_s w_s; the grid scale is 1/(dx dy)
        h->spp.n = cfg->nspecies;
        rmax = 0.0;
        for (int i = 0; i < cfg->nspecies; ++i) {
            h->spp.q[i] = cfg->species_q[i];
            h->spp.m[i] = cfg->species_m[i];
            h->spp.w[i] = cfg->species_w[i];
            h->spp.qw[i] = cfg->species_q[i] * cfg->species_w[i];
            rmax = std::max(rmax, std::fabs(h->spp.qw[i]));
        }
        if (!(rmax > 0.0)) rmax = 1.0;
        h->mc.jscale = 1.0 / (dx * dy);
    }
    h->mc.inv_n = 1.0 / (double)h->ng;
    h->mc.eps0 = cfg->eps0;
    h->mc.inv_eps0 = 1.0 / cfg->eps0;
    h->mc.cdf_th_eps0 = (0.5 * cfg->c * cfg->c * cfg->dt * cfg->dt) / cfg->eps0;
    h->mc.mu0 = 1.0 / (cfg->eps0 * cfg->c * cfg->c);
    h->mc.c = cfg->c;
    h->mc.dt = cfg->dt;
    h->geom = ParticleGeom{cfg->nx, cfg->ny, cfg->lx, cfg->ly, 1.0 / dx, 1.0 / dy, cfg->dt};
    h->push = PushParams{cfg->q, cfg->m, cfg->c, cfg->dt, cfg->weight, 0};
    h->sorting = cfg->sort_interval > 0;
    if (h->sorting) {
        // Tiles of t x t cells holding about 4096 particles at the mean density.  Between
        // two sorts a particle moves at most c dt per step, so a CTA's shared-memory region
        // is its tile plus a halo of that drift and the stencil reach (capped so the region
        // stays within 2048 nodes); nodes beyond it fall back to global atomics.
        TileGeom& tg = h->tg;
        tg.nx = cfg->nx;
        tg.ny = cfg->ny;
        const double ppc = (double)std::max<int64_t>(h->n, 1) / ((double)cfg->nx * cfg->ny);
        tg.t = 4;
        if (cfg->tile > 0) {  // the caller's (an autotuner's) choice, within the grid
            while (tg.t < cfg->tile && 2 * tg.t <= std::min(cfg->nx, cfg->ny)) tg.t *= 2;
        } else {
            while (tg.t < 16 && (double)(2 * tg.t) * (2 * tg.t) * ppc <= 8192.0 &&
                   2 * tg.t <= std::min(cfg->nx, cfg->ny))
                tg.t *= 2;
        }
        tg.ntx = (cfg->nx + tg.t - 1) / tg.t;
        tg.nty = (cfg->ny + tg.t - 1) / tg.t;
        const double drift = cfg->c * cfg->dt * cfg->sort_interval / std::fmin(dx, dy);
        tg.halo = (int)std::ceil(drift) + cfg->spline_order / 2 + 2;
        while (tg.halo > 1 && (tg.t + 2 * tg.halo) * (tg.t + 2 * tg.halo + 31) > 2560) --tg.halo;
        tg.rx = std::min(tg.t + 2 * tg.halo, cfg->nx);
        tg.ry = std::min(tg.t + 2 * tg.halo, cfg->ny);
        // row pitch = t (mod 32): the 32/t x t cells a warp serves map their nodes to
        // 32 different shared-memory banks
        tg.pitch = tg.ry + ((tg.t - tg.ry % 32) % 32 + 32) % 32;
        tg.inv_dx = 1.0 / dx;
        tg.inv_dy = 1.0 / dy;
        tg.dt = cfg->dt;
        tg.lx = cfg->lx;
        tg.ly = cfg->ly;
        tg.half = (cfg->spline_order % 2 == 0) ? 1 : 0;
    }
    if (h->fp32) {
        // Current quantum: the power of two 2^(kc - k) >= c 2^-k, with c <= 2^kc and
        // k = min(38, 62 - ceil(log2 n)).  A contribution |v| W_x W_y is below c, i.e.
        // below 2^k quanta, so no int64 node total can reach 2^62 whatever the
        // distribution, and k <= 38 lets the deposit split each contribution exactly into
        // two parts that fit 32-bit shared atomics (the power of two makes the split's
        // scalings exact).  At k = 38 the quantum (3.6e-12 c for c = 1) is far below the
        // FP32 rounding of a contribution.
        int kj = 38;
        if (h->n > 1) kj = std::min(38, 62 - (int)std::ceil(std::log2((double)h->n)));
        // (with a species table the bound is c max |q_s w_s|: the quantum scales with it)
        const int kc = (int)std::ceil(std::log2(cfg->c)) + (int)std::ceil(std::log2(rmax));
        h->fix_scale_j = (float)std::ldexp(1.0, kj - kc);
        h->fix_unscale_j = 1.0 / (double)h->fix_scale_j;
        // Charge at t = 0 (only the untiled pass): W_x W_y <= 1 (times max |q_s w_s|) with
        // 2^k quanta, k = 62 - ceil(log2 n), so no node total can reach 2^62.
        int k = 46;
        if (h->n > 1) k = std::min(46, 62 - (int)std::ceil(std::log2((double)h->n)));
        k -= (int)std::ceil(std::log2(rmax));
        h->fix_scale_q = (float)std::ldexp(1.0, k);
        h->fix_unscale_q = std::ldexp(1.0, -k);
    } else {
        // FP64 path: |v W_x W_y| < c and |W_x W_y| <= 1 (times max |q_s w_s|), so quanta of
        // 2^-60 of those bounds keep every contribution below 2^60 (one int64 word); the
        // 128-bit sums have room for any number of them.  The quantum (8.7e-19 c for the
        // current) is far below FP64 rounding of a node's total.
        const int kc = (int)std::ceil(std::log2(cfg->c)) + (int)std::ceil(std::log2(rmax));
        h->fix64_scale_j = std::ldexp(1.0, 60 - kc);
        h->fix64_unscale_j = std::ldexp(1.0, kc - 60);
        const int kq = (int)std::ceil(std::log2(rmax));
        h->fix64_scale_q = std::ldexp(1.0, 60 - kq);
        h->fix64_unscale_q = std::ldexp(1.0, kq - 60);
    }
    h->jbytes = h->ng * (h->fp32 ? sizeof(longlong2) : 2 * sizeof(longlong2));
    if (bound) {
        h->bound = true;
        h->x = bound->x;
        h->y = bound->y;
        h->px = bound->px;
        h->py = bound->py;
        h->v[0][0] = bound->vx;
        h->v[0][1] = bound->vy;
        h->v[1][0] = bound->vx_old;
        h->v[1][1] = bound->vy_old;
    }
    st = alloc_state(h);
    if (st == PIC_OK) st = setup(h, init);
    if (st != PIC_OK) {
        g_init_error = h->errmsg;
        cudaStreamSynchronize(h->s);
        free_all(h);
        delete h;
        return st;
    }
    *out = h;
    return PIC_OK;
}

pic_status pic_deposit(pic_handle* h) {
    if (!h) return fail(nullptr, PIC_ERR_INVALID_ARG, "NULL handle");
    if (h->phase != 0) return fail(h, PIC_ERR_STATE, "pic_deposit: the previous step is not finished");
    h->launches_now = 0;
    const bool sort_due = h->sorting && h->step % h->cfg.sort_interval == 0;
    if (h->pending) {  // the last step of the previous pic_step call did this deposit
        std::swap(h->x, h->xnext);
        std::swap(h->y, h->ynext);
        std::swap(h->J, h->Jalt);
        h->pending = false;
        h->phase = 1;
        if (sort_due) {
            TimedScope ts(h, PIC_KT_SORT);
            return sort_particles(h, true);
        }
        return PIC_OK;
    }
    if (sort_due) {
        TimedScope ts(h, PIC_KT_SORT);
        pic_status st = sort_particles(h, false);
        if (st != PIC_OK) return st;
    }
    if (h->fp32) {
        // the buffer the previous field solve zeroed (a memset here would break the chain
        // of dependent launches); J^n stays readable until then
        std::swap(h->J, h->Jalt);
    } else {
        CK(cudaMemsetAsync(h->J, 0, h->jbytes, h->s));
    }
    if (h->vdim == 3 && binned_deposit(h))  // the binned pass adds J_z to it
        CK(cudaMemsetAsync(h->Jz, 0, h->jbytes, h->s));
    h->launches_now += 1;
    TimedScope ts(h, PIC_KT_DEPOSIT);
    CK(by_prec(h, [&](auto t) {
        using T = decltype(t);
        if (binned_deposit(h)) {  // 2D-3V: J_z in the same pass
            const int vo = 1 - h->vcur;
            const bool z3 = h->vdim == 3;
            return launch_deposit_binned(h->p, h->geom, h->push, h->tg, (const float*)h->x,
                                         (const float*)h->y, (float*)h->x, (float*)h->y,
                                         (float*)h->px, (float*)h->py,
                                         (const float*)h->v[h->vcur][0],
                                         (const float*)h->v[h->vcur][1], (float*)h->v[vo][0],
                                         (float*)h->v[vo][1], h->n, h->off, nullptr, h->J,
                                         h->fix_scale_j, h->diag, h->err, h->s, false,
                                         kBinPerCta, h->species, &h->spp,
                                         z3 ? (const float*)h->vz[h->vcur] : nullptr,
                                         z3 ? h->Jz : nullptr);
        }
        const int32_t* sp = h->spp.n > 0 ? h->species : nullptr;
        if constexpr (sizeof(T) == 4) {
            return launch_move_deposit_fix<T>(h->p, h->geom, (T*)h->x, (T*)h->y,
                                              (const T*)h->v[h->vcur][0], (const T*)h->v[h->vcur][1],
                                              h->n, (longlong2*)h->J, h->fix_scale_j, h->err, h->s,
                                              sp, &h->spp);
        } else {
            return launch_move_deposit_fix128(h->p, h->geom, (T*)h->x, (T*)h->y,
                                              (const T*)h->v[h->vcur][0],
                                              (const T*)h->v[h->vcur][1], h->n, (longlong2*)h->J,
                                              h->ng, h->fix64_scale_j, h->err, h->s, sp, &h->spp);
        }
    }));
    if (h->vdim == 3 && !binned_deposit(h)) {  // J_z of the moved particles
        CK(cudaMemsetAsync(h->Jz, 0, h->jbytes, h->s));
        CK(by_prec(h, [&](auto t) {
            using T = decltype(t);
            return launch_deposit_z<T>(h->p, h->geom, (const T*)h->x, (const T*)h->y,
                                       (const T*)h->vz[h->vcur], h->n, h->species, h->spp, h->Jz,
                                       h->ng, h->fp32 ? (double)h->fix_scale_j : h->fix64_scale_j,
                                       h->err, h->s);
        }));
        h->launches_now += 1;
    }
    h->phase = 1;
    return PIC_OK;
}

pic_status pic_field_solve(pic_handle* h) {
    if (!h) return fail(nullptr, PIC_ERR_INVALID_ARG, "NULL handle");
    if (h->phase != 1) return fail(h, PIC_ERR_STATE, "pic_field_solve needs pic_deposit first");
    h->diag_now = diag_due(h);
    h->mc.diag = h->diag_now ? 1 : 0;
    if (h->diag_now) CK(cudaMemsetAsync(h->diag, 0, D_NSLOTS * sizeof(double), h->s));
    const bool fused = field_columns_smem(h->nx, 2 * h->rsz) <= kFieldColumnsSmemMax;
    TimedScope ts(h, PIC_KT_FIELD);

    // forward transform along y (the FP32 form converts the fixed-point sums on load)
    if (h->fp32) {
        CK(launch_fft_y_from_fix<float>((const longlong2*)h->J, h->fix_unscale_j, h->Z, h->nx,
                                        h->ny, h->fy, h->twy, (longlong2*)h->Jalt, h->s));
    } else {  // the 128-bit sums to FP64, then the transform
        CK(launch_fix128_to_cplx((const longlong2*)h->J, h->ng, h->fix64_unscale_j,
                                 (double2*)h->tmp, h->s));
        CK(launch_fft_y<double>(h->tmp, h->Z, h->nx, h->ny, 1, h->fy, h->twy, -1, 0, h->s));
        h->launches_now += 1;
    }
    if (!fused) CK(by_prec(h, [&](auto t) {
        using T = decltype(t);
        return launch_fft_x<T>(h->Z, h->Z, h->nx, h->ny, 1, h->fx, h->twx, -1, h->s);
    }));

    // the naive update takes rho^{n+1} from the charge deposited at x^{n+1}, transformed
    // like the t = 0 charge
    const int32_t* sp = h->spp.n > 0 ? h->species : nullptr;
    if (h->cfg.charge == PIC_CHARGE_DEPOSIT) {
        CK(cudaMemsetAsync(h->rhoq, 0, h->jbytes, h->s));
        CK(by_prec(h, [&](auto t) -> cudaError_t {
            using T = decltype(t);
            cudaError_t r;
            if (h->fp32) {
                r = launch_deposit_charge_fix<T>(h->p, h->geom, (const T*)h->x, (const T*)h->y,
                                                 h->n, (longlong2*)h->rhoq, h->fix_scale_q,
                                                 h->err, h->s, sp, &h->spp);
                if (r == cudaSuccess)
                    r = launch_fix_to_cplx<T>((const longlong2*)h->rhoq, h->fix_unscale_q, h->tmp,
                                              h->ng, h->s);
                return r == cudaSuccess ? forward_fft(h, h->tmp, h->ZQ) : r;
            }
            r = launch_deposit_charge_fix128(h->p, h->geom, (const double*)h->x,
                                             (const double*)h->y, h->n, (longlong2*)h->rhoq,
                                             h->ng, h->fix64_scale_q, h->err, h->s, sp, &h->spp);
            if (r == cudaSuccess)
                r = launch_fix128_to_cplx((const longlong2*)h->rhoq, h->ng, h->fix64_unscale_q,
                                          (double2*)h->tmp, h->s);
            return r == cudaSuccess ? forward_fft(h, h->tmp, h->ZQ) : r;
        }));
    }

    // per-mode update with the stepper's history levels
    const int st = h->cfg.stepper;
    BdfParams bp = h->bdf;
    ZParams zp{};
    int nslot = 0, nr = 0;
    if (st == PIC_STEPPER_BDF) {
        const int k = bp.k;
        for (int d = 1; d <= 2 * k; ++d) {
            const int slot = ((h->head - (d - 1)) % h->L + h->L) % h->L;
            bp.phi[d - 1] = h->phi_l[slot];
            bp.ax[d - 1] = h->ax_l[slot];
            bp.ay[d - 1] = h->ay_l[slot];
            if (h->vdim == 3) zp.az[d - 1] = h->az_l[slot];
        }
        for (int d = 1; d <= k; ++d) bp.rho[d - 1] = h->rho_l[((h->head_r - (d - 1)) % h->Lr + h->Lr) % h->Lr];
        nslot = (h->head + 1) % h->L;
        nr = (h->head_r + 1) % h->Lr;
        bp.phi_new = h->phi_l[nslot];
        bp.ax_new = h->ax_l[nslot];
        bp.ay_new = h->ay_l[nslot];
        bp.rho_new = h->rho_l[nr];
        if (h->vdim == 3) zp.az_new = h->az_l[nslot];
    }
    const int kind = st == PIC_STEPPER_BDF ? K_BDF : (st == PIC_STEPPER_CDF2 ? K_CDF2 : K_DIRK);
    zp.kind = kind;
    zp.form = h->cdf.form;
    zp.az_n = h->az;
    zp.az_prev = h->az_prev;
    zp.jz_n = h->jz;
    zp.jz_prev = h->jz_prev;
    zp.vaz = h->vaz;
    CK(by_prec(h, [&](auto t) {
        using T = decltype(t);
        if (fused)
            return launch_field_columns<T>(h->mc, kind, bp, h->cdf, h->dirk, h->Z, h->F4, h->E,
                                           h->diag, h->fx, h->twx, h->s);
        if (kind == K_BDF) return launch_mode_bdf<T>(h->mc, bp, h->Z, h->F4, h->E, h->diag, h->s);
        if (kind == K_CDF2) return launch_mode_cdf2<T>(h->mc, h->cdf, h->Z, h->F4, h->E, h->diag, h->s);
        return launch_mode_dirk<T>(h->mc, h->dirk, h->Z, h->F4, h->E, h->diag, h->s);
    }));
    if (st == PIC_STEPPER_BDF) {
        h->head = nslot;
        h->head_r = nr;
    } else if (st == PIC_STEPPER_CDF2) {
        std::swap(h->cdf.phi, h->cdf.phi_prev);
        std::swap(h->cdf.rho, h->cdf.rho_prev);
        std::swap(h->cdf.ax, h->cdf.ax_prev);
        std::swap(h->cdf.ay, h->cdf.ay_prev);
        std::swap(h->cdf.jx, h->cdf.jx_prev);
        std::swap(h->cdf.jy, h->cdf.jy_prev);
    }

    // inverse transforms: along x (unless fused above), then along y into the [node][4]
    // gather layout
    CK(by_prec(h, [&](auto t) {
        using T = decltype(t);
        cudaError_t r = cudaSuccess;
        if (!fused) r = launch_fft_x<T>(h->F4, h->F4, h->nx, h->ny, 4, h->fx, h->twx, +1, h->s);
        if (r != cudaSuccess) return r;
        return launch_fft_y<T>(h->F4, h->G, h->nx, h->ny, 4, h->fy, h->twy, +1, 1, h->s);
    }));
    h->launches_now += fused ? 3 : 5;

    // 2D-3V: A_z by the same stepper from J_z, and its gather fields (Gz)
    if (h->vdim == 3) {
        CK(by_prec(h, [&](auto t) -> cudaError_t {
            using T = decltype(t);
            cudaError_t r;
            if (h->fp32) {
                r = launch_fix_to_cplx<T>((const longlong2*)h->Jz, h->fix_unscale_j, h->tmp, h->ng,
                                          h->s);
                if (r == cudaSuccess) r = forward_fft(h, h->tmp, h->Zz);
            } else {  // J_z in the real parts
                r = launch_fix128_to_cplx((const longlong2*)h->Jz, h->ng, h->fix64_unscale_j,
                                          (double2*)h->tmp, h->s);
                if (r == cudaSuccess) r = forward_fft(h, h->tmp, h->Zz);
            }
            if (r != cudaSuccess) return r;
            r = launch_zfield<T>(h->mc, bp, h->dirk, zp, h->Zz, h->F2, h->diag, h->s);
            if (r != cudaSuccess) return r;
            r = launch_fft_x<T>(h->F2, h->F2, h->nx, h->ny, 2, h->fx, h->twx, +1, h->s);
            if (r != cudaSuccess) return r;
            return launch_fft_y<T>(h->F2, h->Gz, h->nx, h->ny, 2, h->fy, h->twy, +1, 1, h->s);
        }));
        if (st == PIC_STEPPER_CDF2) {
            std::swap(h->az, h->az_prev);
            std::swap(h->jz, h->jz_prev);
        }
        h->launches_now += h->fp32 ? 6 : 5;
    }
    h->phase = 2;
    return PIC_OK;
}

pic_status pic_gather_push(pic_handle* h) { return gather_push_step(h, false, false); }

pic_status pic_step(pic_handle* h, int32_t nsteps) {
    if (!h) return fail(nullptr, PIC_ERR_INVALID_ARG, "NULL handle");
    if (nsteps < 0) return fail(h, PIC_ERR_INVALID_ARG, "nsteps must be >= 0");
    for (int32_t i = 0; i < nsteps; ++i) {
        NvtxRange r("step");
        pic_status st = PIC_OK;
        if (h->phase == 1 && h->fused_deposit) {
            // this step's deposit ran fused with the previous gather; a sort due now
            // follows it
            h->fused_deposit = false;
            if (h->sorting && h->step % h->cfg.sort_interval == 0) {
                TimedScope ts(h, PIC_KT_SORT);
                st = sort_particles(h, true);
            }
        } else {
            st = pic_deposit(h);
        }
        if (st == PIC_OK) st = pic_field_solve(h);
        // the last step of the call leaves the next deposit pending (the call still
        // returns between two steps), or, in an ensemble's capture, is not fused
        const bool last = i + 1 == nsteps;
        if (st == PIC_OK)
            st = gather_push_step(h, fuse_next(h) && !(last && h->no_defer), last);
        if (st != PIC_OK) return st;
    }
    return PIC_OK;
}

}  // extern "C"

namespace {

// Gather + push of the step (a8, a9); with `fuse`, the sorted FP32 form's binned kernel
// also moves the particles and deposits the next step's current (its a2, a3) into the
// buffer the field solve just cleared, and the handle is left with that deposit done; with
// `defer` as well, the moved positions go to xnext, ynext and the deposit stays pending
// until the next step, so the handle's particle state is that of the end of this step.
pic_status gather_push_step(pic_handle* h, bool fuse, bool defer) {
    if (!h) return fail(nullptr, PIC_ERR_INVALID_ARG, "NULL handle");
    if (h->phase != 2) return fail(h, PIC_ERR_STATE, "pic_gather_push needs pic_field_solve first");
    PushParams pp = h->push;
    pp.diag = h->diag_now ? 1 : 0;
    const int vo = 1 - h->vcur;
    if (fuse) {
        TimedScope ts(h, PIC_KT_GATHER_DEPOSIT);
        void* xo = defer ? h->xnext : h->x;
        void* yo = defer ? h->ynext : h->y;
        CK(launch_deposit_binned(h->p, h->geom, pp, h->tg, (const float*)h->x,
                                 (const float*)h->y, (float*)xo, (float*)yo, (float*)h->px,
                                 (float*)h->py, (const float*)h->v[h->vcur][0],
                                 (const float*)h->v[h->vcur][1], (float*)h->v[vo][0],
                                 (float*)h->v[vo][1], h->n, h->off, h->G, h->Jalt,
                                 h->fix_scale_j, h->diag, h->err, h->s, true, kBinPerCta,
                                 h->species, &h->spp));
    } else if (h->sorting && h->fp32 && h->vdim == 2 && h->spp.n == 0) {
        TimedScope ts(h, PIC_KT_GATHER);
        CK(launch_gather_push_tiled(h->p, h->geom, pp, h->tg, (const float*)h->x,
                                    (const float*)h->y, (float*)h->px, (float*)h->py,
                                    (const float*)h->v[h->vcur][0], (const float*)h->v[h->vcur][1],
                                    (float*)h->v[vo][0], (float*)h->v[vo][1], h->n,
                                    h->off, h->G,
                                    h->diag, h->err, h->s));
    } else if (h->vdim == 3 || h->spp.n > 0) {
        TimedScope ts(h, PIC_KT_GATHER);
        const bool z3 = h->vdim == 3;
        CK(by_prec(h, [&](auto t) {
            using T = decltype(t);
            return launch_gather_push3<T>(
                h->p, h->geom, pp, (const T*)h->x, (const T*)h->y, (T*)h->px, (T*)h->py,
                (const T*)h->pz, (const T*)h->v[h->vcur][0], (const T*)h->v[h->vcur][1],
                z3 ? (const T*)h->vz[h->vcur] : nullptr, (T*)h->v[vo][0], (T*)h->v[vo][1],
                z3 ? (T*)h->vz[vo] : nullptr, h->species, h->spp, h->n, h->G, h->Gz, h->diag,
                h->err, h->s);
        }));
    } else {
        TimedScope ts(h, PIC_KT_GATHER);
        CK(by_prec(h, [&](auto t) {
            using T = decltype(t);
            return launch_gather_push<T>(h->p, h->geom, pp, (const T*)h->x, (const T*)h->y,
                                         (T*)h->px, (T*)h->py, (const T*)h->v[h->vcur][0],
                                         (const T*)h->v[h->vcur][1], (T*)h->v[vo][0],
                                         (T*)h->v[vo][1], h->n, h->G, h->gather_out, h->diag,
                                         h->err, h->s, h->gather_out_short);
        }));
    }
    h->vcur = vo;
    h->launches_now += 1;
    h->launches_last = h->launches_now;
    h->step += 1;
    h->stepped = true;
    h->e_valid = h->diag_now;
    if (h->diag_now) {
        h->diag_valid = true;
        h->diag_step = h->step;
        if (h->diag_ring) {  // this step's record, stream-ordered after its reductions
            const int64_t slot = h->ring_written % PIC_DIAG_HISTORY;
            CK(cudaMemcpyAsync(h->diag_ring + slot * D_NSLOTS, h->diag,
                               D_NSLOTS * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
            h->ring_step[slot] = h->step;
            ++h->ring_written;
        }
    }
    h->phase = 0;
    h->fused_deposit = false;
    if (fuse && defer) {
        h->pending = true;
    } else if (fuse) {  // the next step's deposit is done: its current is in the buffer it reads
        std::swap(h->J, h->Jalt);
        h->launches_now = 0;
        h->phase = 1;
        h->fused_deposit = true;
    }
    return PIC_OK;
}

}  // namespace

// ------------------------------------------------------------ ensembles ----

struct pic_ensemble {
    std::vector<pic_handle*> runs;
    std::vector<int64_t> step0;  // each run's step count when the graph was captured
    cudaStream_t s = nullptr;
    int period = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev = nullptr;    // fork / join marks on the ensemble's stream
    std::vector<cudaEvent_t> ev_run;
};

namespace {

int64_t lcm64(int64_t a, int64_t b) { return a / std::gcd(a, b) * b; }

// Steps after which every per-step rotation of the run's buffers is back where it was:
// velocity buffers (2), BDF rings (L, Lr), CDF-2 level swaps (2), the FP32 current
// buffers (2), the sort's particle sets (two sorts, 2 S).
int64_t step_period(const pic_handle* h) {
    int64_t p = 2;
    if (h->cfg.stepper == PIC_STEPPER_BDF) p = lcm64(lcm64(p, h->L), h->Lr);
    if (h->sorting) p = lcm64(p, 2 * (int64_t)h->cfg.sort_interval);
    return p;
}

void ensemble_release(pic_ensemble* e) {
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    if (e->ev) cudaEventDestroy(e->ev);
    for (cudaEvent_t v : e->ev_run) cudaEventDestroy(v);
    delete e;
}

pic_status efail(pic_ensemble* e, pic_status st, const char* msg, cudaError_t ce = cudaSuccess) {
    if (e) ensemble_release(e);
    if (ce != cudaSuccess) return fail(nullptr, st, "%s: %s", msg, cudaGetErrorString(ce));
    return fail(nullptr, st, "%s", msg);
}

}  // namespace

extern "C" {

pic_status pic_ensemble_create(pic_handle* const* runs, int32_t count, void* stream,
                               pic_ensemble** out) {
    if (!runs || !out || count < 1 || count > 4096)
        return fail(nullptr, PIC_ERR_INVALID_ARG, "runs, out must not be NULL; 1 <= count <= 4096");
    if (!stream)
        return fail(nullptr, PIC_ERR_INVALID_ARG, "the ensemble needs a stream other than NULL");
    *out = nullptr;
    int64_t period = 1;
    for (int32_t i = 0; i < count; ++i) {
        const pic_handle* h = runs[i];
        if (!h) return fail(nullptr, PIC_ERR_INVALID_ARG, "run %d is NULL", i);
        for (int32_t k = 0; k < i; ++k)
            if (runs[k] == h) return fail(nullptr, PIC_ERR_INVALID_ARG, "run %d repeats run %d", i, k);
        if (!h->s) return fail(nullptr, PIC_ERR_INVALID_ARG, "run %d uses the NULL stream", i);
        if (h->phase != 0) return fail(nullptr, PIC_ERR_STATE, "run %d is in the middle of a step", i);
        if (h->diag_every > 0 || h->ktiming)
            return fail(nullptr, PIC_ERR_STATE, "run %d has diagnostics or kernel timing on", i);
        period = lcm64(period, step_period(h));
        if (period > (1 << 16)) return fail(nullptr, PIC_ERR_INVALID_ARG, "common period too long");
    }
    pic_ensemble* e = new pic_ensemble;
    e->runs.assign(runs, runs + count);
    e->s = (cudaStream_t)stream;
    e->period = (int)period;
    cudaError_t ce = cudaEventCreateWithFlags(&e->ev, cudaEventDisableTiming);
    for (int32_t i = 0; i < count && ce == cudaSuccess; ++i) {
        cudaEvent_t v = nullptr;
        ce = cudaEventCreateWithFlags(&v, cudaEventDisableTiming);
        if (ce == cudaSuccess) e->ev_run.push_back(v);
    }
    if (ce != cudaSuccess) return efail(e, PIC_ERR_CUDA, "event creation failed", ce);
    // nothing of the runs may be pending outside the capture (a pending deposit is redone
    // by the graph's first step)
    for (pic_handle* h : e->runs) {
        if ((ce = drop_pending(h)) != cudaSuccess)
            return efail(e, PIC_ERR_CUDA, "clearing a pending deposit failed", ce);
        if ((ce = cudaStreamSynchronize(h->s)) != cudaSuccess)
            return efail(e, PIC_ERR_CUDA, "synchronising a run failed", ce);
    }
    if ((ce = cudaStreamSynchronize(e->s)) != cudaSuccess)
        return efail(e, PIC_ERR_CUDA, "synchronising the ensemble stream failed", ce);
    // Capturing runs the step functions on the host: their buffer rotations advance by
    // the period and so end where they started; the step counts are put back.
    std::vector<pic_handle> saved;
    saved.reserve(count);
    for (pic_handle* h : e->runs) {
        saved.push_back(*h);
        e->step0.push_back(h->step);
    }
    auto restore = [&] {
        for (int32_t i = 0; i < count; ++i) *e->runs[i] = saved[i];
    };
    ce = cudaStreamBeginCapture(e->s, cudaStreamCaptureModeRelaxed);
    if (ce != cudaSuccess) return efail(e, PIC_ERR_CUDA, "cudaStreamBeginCapture failed", ce);
    pic_status st = PIC_OK;
    int32_t failed = 0;
    cudaError_t cap = cudaEventRecord(e->ev, e->s);
    for (int32_t i = 0; i < count && cap == cudaSuccess && st == PIC_OK; ++i) {
        pic_handle* h = e->runs[i];
        failed = i;
        cap = cudaStreamWaitEvent(h->s, e->ev, 0);  // the run's stream joins the capture
        h->no_defer = true;  // the captured period ends between two steps
        if (cap == cudaSuccess) st = pic_step(h, e->period);
        h->no_defer = false;
        if (cap == cudaSuccess && st == PIC_OK) cap = cudaEventRecord(e->ev_run[i], h->s);
        if (cap == cudaSuccess && st == PIC_OK) cap = cudaStreamWaitEvent(e->s, e->ev_run[i], 0);
    }
    cudaGraph_t g = nullptr;
    ce = cudaStreamEndCapture(e->s, &g);
    e->graph = g;
    std::string why = st != PIC_OK ? "capturing the steps of run " + std::to_string(failed) +
                                         " failed: " + e->runs[failed]->errmsg
                                   : "";
    restore();
    if (st != PIC_OK) return efail(e, st, why.c_str());
    if (cap != cudaSuccess) return efail(e, PIC_ERR_CUDA, "capture failed", cap);
    if (ce != cudaSuccess || !g) return efail(e, PIC_ERR_CUDA, "cudaStreamEndCapture failed", ce);
    ce = cudaGraphInstantiate(&e->exec, e->graph, 0);
    if (ce != cudaSuccess) return efail(e, PIC_ERR_CUDA, "cudaGraphInstantiate failed", ce);
    *out = e;
    return PIC_OK;
}

pic_status pic_ensemble_step(pic_ensemble* e, int32_t nsteps) {
    if (!e) return fail(nullptr, PIC_ERR_INVALID_ARG, "NULL ensemble");
    if (nsteps < 0 || nsteps % e->period != 0)
        return fail(nullptr, PIC_ERR_INVALID_ARG, "nsteps must be a non-negative multiple of %d",
                    e->period);
    const size_t n = e->runs.size();
    for (size_t i = 0; i < n; ++i) {
        const pic_handle* h = e->runs[i];
        if (h->phase != 0 || h->diag_every > 0 || h->ktiming ||
            (h->step - e->step0[i]) % e->period != 0)
            return fail(nullptr, PIC_ERR_STATE,
                        "run %d no longer matches the captured graph (mid-step, diagnostics or "
                        "timing on, or advanced alone by a number of steps that is not a "
                        "multiple of %d)", (int)i, e->period);
    }
    if (nsteps == 0) return PIC_OK;
    cudaError_t ce = cudaSuccess;
    // a run stepped alone since may hold a pending deposit: the graph redoes it
    for (size_t i = 0; i < n && ce == cudaSuccess; ++i) ce = drop_pending(e->runs[i]);
    for (size_t i = 0; i < n && ce == cudaSuccess; ++i) {  // after the runs' pending work
        ce = cudaEventRecord(e->ev_run[i], e->runs[i]->s);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(e->s, e->ev_run[i], 0);
    }
    for (int32_t k = 0; k < nsteps / e->period && ce == cudaSuccess; ++k)
        ce = cudaGraphLaunch(e->exec, e->s);
    if (ce == cudaSuccess) ce = cudaEventRecord(e->ev, e->s);
    for (size_t i = 0; i < n && ce == cudaSuccess; ++i)  // later work on a run comes after
        ce = cudaStreamWaitEvent(e->runs[i]->s, e->ev, 0);
    if (ce != cudaSuccess) return fail(nullptr, PIC_ERR_CUDA, "ensemble launch failed: %s",
                                       cudaGetErrorString(ce));
    for (pic_handle* h : e->runs) {
        h->step += nsteps;
        h->stepped = true;
    }
    return PIC_OK;
}

int32_t pic_ensemble_period(const pic_ensemble* e) { return e ? e->period : 0; }

void pic_ensemble_destroy(pic_ensemble* e) {
    if (!e) return;
    cudaStreamSynchronize(e->s);
    ensemble_release(e);
}

pic_status pic_set_diagnostics(pic_handle* h, int32_t every) {
    if (!h) return fail(nullptr, PIC_ERR_INVALID_ARG, "NULL handle");
    if (every < 0) return fail(h, PIC_ERR_INVALID_ARG, "every must be >= 0");
    if (every > 0 && !h->diag_ring) {
        void* p = nullptr;
        CK(dalloc(h, &p, (size_t)PIC_DIAG_HISTORY * D_NSLOTS * sizeof(double)));
        h->diag_ring = static_cast<double*>(p);
        h->ring_step.assign(PIC_DIAG_HISTORY, -1);
    }
    h->diag_every = every;
    h->ring_read = h->ring_written;  // the history starts here
    return PIC_OK;
}

namespace {

// The diagnostics of one step from its raw accumulators (sums over modes and particles).
void to_diagnostics(const pic_handle* h, const double* acc, int64_t step, pic_diagnostics* out) {
    const double N = (double)h->ng;
    const double area = (h->cfg.lx / h->nx) * (h->cfg.ly / h->ny);
    // Parseval: grid mean of |f|^2 = (1/N^2) sum_k |f_hat|^2
    auto rms = [&](double s) { return std::sqrt(s) / N; };
    out->gauge_rms = rms(acc[D_GAUGE]);
    out->gauss_rms = rms(acc[D_GAUSS]);
    out->continuity_rms = rms(acc[D_CONT]);
    out->gauge_dt_rms = rms(acc[D_GAUGE_DT]);
    out->rho_rms = rms(acc[D_RHO]);
    out->div_a_rms = rms(acc[D_DIVA]);
    out->w_e = 0.5 * h->cfg.eps0 * area * acc[D_WE] / N;
    out->w_b = 0.5 / h->mc.mu0 * area * acc[D_WB] / N;
    out->kinetic = acc[D_KIN];
    out->step = step;
}

}  // namespace

pic_status pic_residuals(pic_handle* h, pic_diagnostics* out) {
    if (!h || !out) return fail(h, PIC_ERR_INVALID_ARG, "NULL argument");
    double acc[D_NSLOTS];
    CK(cudaMemcpyAsync(acc, h->diag, sizeof acc, cudaMemcpyDeviceToHost, h->s));
    pic_status st = check_device_error(h);
    if (st != PIC_OK) return st;
    if (!h->diag_valid) return fail(h, PIC_ERR_STATE, "no step has been diagnosed yet");
    to_diagnostics(h, acc, h->diag_step, out);
    return PIC_OK;
}

pic_status pic_diagnostics_history(pic_handle* h, pic_diagnostics* out, int32_t capacity,
                                   int32_t* count) {
    if (!h || !count || (capacity > 0 && !out))
        return fail(h, PIC_ERR_INVALID_ARG, "NULL argument");
    if (capacity < 0) return fail(h, PIC_ERR_INVALID_ARG, "capacity must be >= 0");
    *count = 0;
    pic_status st = check_device_error(h);  // also waits for the ring's copies
    if (st != PIC_OK) return st;
    // the unread records still in the ring, the newest `capacity` of them
    int64_t first = std::max(h->ring_read, h->ring_written - (int64_t)PIC_DIAG_HISTORY);
    first = std::max(first, h->ring_written - (int64_t)capacity);
    const int64_t nrec = h->ring_written - first;
    if (nrec > 0) {
        std::vector<double> acc((size_t)nrec * D_NSLOTS);
        for (int64_t r = first; r < h->ring_written; ) {  // at most two contiguous pieces
            const int64_t slot = r % PIC_DIAG_HISTORY;
            const int64_t len = std::min(h->ring_written - r, (int64_t)PIC_DIAG_HISTORY - slot);
            CK(cudaMemcpyAsync(acc.data() + (size_t)(r - first) * D_NSLOTS,
                               h->diag_ring + slot * D_NSLOTS,
                               (size_t)len * D_NSLOTS * sizeof(double), cudaMemcpyDeviceToHost,
                               h->s));
            r += len;
        }
        CK(cudaStreamSynchronize(h->s));
        for (int64_t r = first; r < h->ring_written; ++r)
            to_diagnostics(h, acc.data() + (size_t)(r - first) * D_NSLOTS,
                           h->ring_step[r % PIC_DIAG_HISTORY], out + (r - first));
    }
    h->ring_read = h->ring_written;
    *count = (int32_t)nrec;
    return PIC_OK;
}

pic_status pic_get_field(pic_handle* h, int32_t which, double* dst) {
    if (!h || !dst) return fail(h, PIC_ERR_INVALID_ARG, "NULL argument");
    if (which < PIC_FIELD_JX || which > PIC_FIELD_DAZDY)
        return fail(h, PIC_ERR_INVALID_ARG, "unknown field %d", which);
    if (which >= PIC_FIELD_JZ && h->vdim != 3)
        return fail(h, PIC_ERR_STATE, "field %d needs 2D-3V (vdim 3)", which);
    if (!h->stepped && which != PIC_FIELD_RHO && which != PIC_FIELD_PHI)
        return fail(h, PIC_ERR_STATE, "field %d needs a completed step", which);
    if ((which == PIC_FIELD_EX || which == PIC_FIELD_EY) && !h->e_valid)
        return fail(h, PIC_ERR_STATE, "E needs diagnostics on the last step");
    const int64_t n = (int64_t)h->ng;
    cudaError_t e = by_prec(h, [&](auto t) -> cudaError_t {
        using T = decltype(t);
        const size_t cs = sizeof(T) * 2;
        cudaError_t r0;
        switch (which) {
            case PIC_FIELD_JX:
            case PIC_FIELD_JY:
                if (h->fp32)
                    return launch_extract_fix((const longlong2*)h->J, which == PIC_FIELD_JY,
                                              h->fix_unscale_j * h->mc.jscale, h->tmpd, n, h->s);
                r0 = launch_fix128_to_cplx((const longlong2*)h->J, h->ng, h->fix64_unscale_j,
                                           (double2*)h->tmp, h->s);
                if (r0 != cudaSuccess) return r0;
                return launch_extract<double>(h->tmp, 1, which == PIC_FIELD_JY, h->mc.jscale,
                                              h->tmpd, n, h->s);
            case PIC_FIELD_JZ:
                if (h->fp32)
                    return launch_extract_fix((const longlong2*)h->Jz, 0,
                                              h->fix_unscale_j * h->mc.jscale, h->tmpd, n, h->s);
                r0 = launch_fix128_to_cplx((const longlong2*)h->Jz, h->ng, h->fix64_unscale_j,
                                           (double2*)h->tmp, h->s);
                if (r0 != cudaSuccess) return r0;
                return launch_extract<double>(h->tmp, 1, 0, h->mc.jscale, h->tmpd, n, h->s);
            case PIC_FIELD_DAZDX: case PIC_FIELD_DAZDY:  // Gz: [node][2], (dAz/dx, dAz/dy) first
                return launch_extract<T>(h->Gz, 2, which == PIC_FIELD_DAZDY, 1.0, h->tmpd, n, h->s);
            case PIC_FIELD_DPHIDX: case PIC_FIELD_DPHIDY: case PIC_FIELD_GAX: case PIC_FIELD_GAY:
            case PIC_FIELD_DAXDX: case PIC_FIELD_DAXDY: case PIC_FIELD_DAYDX: case PIC_FIELD_DAYDY: {
                const int f = which - PIC_FIELD_DPHIDX;
                return launch_extract<T>((const char*)h->G + (f / 2) * cs, 4, f & 1, 1.0, h->tmpd, n, h->s);
            }
            default: break;
        }
        cudaError_t r;
        int comp = 0;
        if (which == PIC_FIELD_EX || which == PIC_FIELD_EY) {
            r = cudaMemcpyAsync(h->tmp, h->E, h->ng * cs, cudaMemcpyDeviceToDevice, h->s);
            comp = which == PIC_FIELD_EY;
        } else if (which == PIC_FIELD_RHO) {
            r = launch_mode_pack2<T>(h->mc, newest(h, 3), nullptr, 0, h->tmp, h->s);
        } else if (which == PIC_FIELD_PHI) {
            r = launch_mode_pack2<T>(h->mc, newest(h, 0), nullptr, 0, h->tmp, h->s);
        } else if (which == PIC_FIELD_BZ) {
            r = launch_mode_pack2<T>(h->mc, newest(h, 1), newest(h, 2), 1, h->tmp, h->s);
        } else if (which == PIC_FIELD_AZ) {
            r = launch_mode_pack2<T>(h->mc, newest(h, 4), nullptr, 0, h->tmp, h->s);
        } else if (which == PIC_FIELD_BX || which == PIC_FIELD_BY) {
            r = launch_mode_pack2<T>(h->mc, newest(h, 4), nullptr, 2, h->tmp, h->s);
            comp = which == PIC_FIELD_BY;
        } else {
            r = launch_mode_pack2<T>(h->mc, newest(h, 1), newest(h, 2), 0, h->tmp, h->s);
            comp = which == PIC_FIELD_AY;
        }
        if (r != cudaSuccess) return r;
        r = inverse_fft(h, h->tmp, h->tmp, 1);
        if (r != cudaSuccess) return r;
        return launch_extract<T>(h->tmp, 1, comp, 1.0, h->tmpd, n, h->s);
    });
    CK(e);
    CK(cudaMemcpyAsync(dst, h->tmpd, h->ng * sizeof(double), cudaMemcpyDefault, h->s));
    return check_device_error(h);
}

pic_status pic_read_particles(pic_handle* h, double* x, double* y, double* px, double* py,
                              double* vx, double* vy, double* vx_old, double* vy_old) {
    if (!h) return fail(nullptr, PIC_ERR_INVALID_ARG, "NULL handle");
    if (h->phase != 0) return fail(h, PIC_ERR_STATE, "pic_read_particles inside a step");
    const void* src[8] = {h->x, h->y, h->px, h->py, h->v[h->vcur][0], h->v[h->vcur][1],
                          h->v[1 - h->vcur][0], h->v[1 - h->vcur][1]};
    double* dst[8] = {x, y, px, py, vx, vy, vx_old, vy_old};
    const size_t nb = (size_t)h->n * sizeof(double);
    for (int i = 0; i < 8; ++i) {
        if (!dst[i] || h->n == 0) continue;
        if (h->sorting) {  // restore the order given to pic_init
            CK(by_prec(h, [&](auto t) {
                using T = decltype(t);
                return launch_scatter_by_id<T>((const T*)src[i], h->id, h->stage, h->n, h->s);
            }));
            CK(cudaMemcpyAsync(dst[i], h->stage, nb, cudaMemcpyDefault, h->s));
            CK(cudaStreamSynchronize(h->s));
            continue;
        }
        if (h->fp32) {
            CK(launch_convert<float, double>((const float*)src[i], h->stage, h->n, h->s));
            CK(cudaMemcpyAsync(dst[i], h->stage, nb, cudaMemcpyDefault, h->s));
            CK(cudaStreamSynchronize(h->s));  // the staging buffer is reused
        } else {
            CK(cudaMemcpyAsync(dst[i], src[i], nb, cudaMemcpyDefault, h->s));
        }
    }
    return check_device_error(h);
}

pic_status pic_read_particles_z(pic_handle* h, double* pz, double* vz, double* vz_old,
                                int32_t* species) {
    if (!h) return fail(nullptr, PIC_ERR_INVALID_ARG, "NULL handle");
    if (h->phase != 0) return fail(h, PIC_ERR_STATE, "pic_read_particles_z inside a step");
    if ((pz || vz || vz_old) && h->vdim != 3)
        return fail(h, PIC_ERR_STATE, "no z components: the handle is 2D-2V");
    if (species && h->spp.n == 0) return fail(h, PIC_ERR_STATE, "the handle has no species table");
    const size_t nb = (size_t)h->n * sizeof(double);
    const void* src[3] = {h->pz, h->vz[h->vcur], h->vz[1 - h->vcur]};
    double* dst[3] = {pz, vz, vz_old};
    for (int i = 0; i < 3 && h->n > 0; ++i) {
        if (!dst[i]) continue;
        if (h->sorting) {  // restore the order given to pic_init
            CK(by_prec(h, [&](auto t) {
                using T = decltype(t);
                return launch_scatter_by_id<T>((const T*)src[i], h->id, h->stage, h->n, h->s);
            }));
            CK(cudaMemcpyAsync(dst[i], h->stage, nb, cudaMemcpyDefault, h->s));
            CK(cudaStreamSynchronize(h->s));
            continue;
        }
        if (h->fp32) {
            CK(launch_convert<float, double>((const float*)src[i], h->stage, h->n, h->s));
            CK(cudaMemcpyAsync(dst[i], h->stage, nb, cudaMemcpyDefault, h->s));
            CK(cudaStreamSynchronize(h->s));  // the staging buffer is reused
        } else {
            CK(cudaMemcpyAsync(dst[i], src[i], nb, cudaMemcpyDefault, h->s));
        }
    }
    if (species && h->n > 0) {
        const int32_t* from = h->species;
        if (h->sorting) {  // restore the order given to pic_init (in the staging buffer)
            CK(launch_scatter_by_id_i32(h->species, h->id, (int32_t*)h->stage, h->n, h->s));
            from = (const int32_t*)h->stage;
        }
        CK(cudaMemcpyAsync(species, from, (size_t)h->n * sizeof(int32_t), cudaMemcpyDefault,
                           h->s));
    }
    return check_device_error(h);
}

pic_status pic_sync(pic_handle* h) {
    if (!h) return fail(nullptr, PIC_ERR_INVALID_ARG, "NULL handle");
    CK(cudaStreamSynchronize(h->s));
    return check_device_error(h);
}

int64_t pic_step_count(const pic_handle* h) { return h ? h->step : -1; }

int32_t pic_velocity_slot(const pic_handle* h) { return h ? h->vcur : -1; }

int32_t pic_kernels_per_step(const pic_handle* h) {
    if (!h) return 0;
    // Kernels the most recent complete step launched: move_deposit, the row transform,
    // the fused column pass (or column transforms and the per-mode update on grids too
    // large for it), the inverse row transform, gather_push; a sort step adds its 3
    // kernels.  Before any step: the count of a step without a sort.
    if (!h->stepped) {
        const bool fused = field_columns_smem(h->nx, 2 * h->rsz) <= kFieldColumnsSmemMax;
        const int z = h->vdim == 3 ? (h->fp32 ? 7 : 6) : 0;  // J_z deposit and the A_z solve
        return (fused ? 5 : 7) + z;
    }
    return h->launches_last;
}

const char* pic_last_error(const pic_handle* h) {
    return h ? h->errmsg.c_str() : g_init_error.c_str();
}

pic_status pic_set_kernel_timing(pic_handle* h, int32_t max_launches) {
    if (!h) return fail(nullptr, PIC_ERR_INVALID_ARG, "NULL handle");
    if (max_launches < 0 || max_launches > (1 << 20))
        return fail(h, PIC_ERR_INVALID_ARG, "max_launches must be in 0..2^20");
    if (max_launches == 0) {
        h->ktiming = false;
        return PIC_OK;
    }
    CK(cudaStreamSynchronize(h->s));  // no recorded pair is still pending
    for (auto& t : h->kt) {
        t.used = 0;
        while ((int64_t)t.ev.size() < 2 * (int64_t)max_launches) {
            cudaEvent_t e;
            const cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) {
                h->ktiming = false;
                return fail(h, PIC_ERR_CUDA, "kernel timing: %s", cudaGetErrorString(r));
            }
            t.ev.push_back(e);
        }
    }
    h->kt_cap = max_launches;
    h->ktiming = true;
    return PIC_OK;
}

pic_status pic_kernel_time(pic_handle* h, int32_t which, double* total_ms, int64_t* launches) {
    if (!h) return fail(nullptr, PIC_ERR_INVALID_ARG, "NULL handle");
    if (which < 0 || which >= PIC_KT_COUNT || !total_ms || !launches)
        return fail(h, PIC_ERR_INVALID_ARG, "unknown timer or NULL output");
    CK(cudaStreamSynchronize(h->s));
    const auto& t = h->kt[which];
    double sum = 0.0;
    for (int64_t i = 0; i < t.used; ++i) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, t.ev[2 * i], t.ev[2 * i + 1]));
        sum += ms;
    }
    *total_ms = sum;
    *launches = t.used;
    return PIC_OK;
}

void pic_destroy(pic_handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->s);
    free_all(h);
    delete h;
}

}  // extern "C"
