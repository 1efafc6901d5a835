// Host side of pic_save_state / pic_load_state (include/pic.h): the handle's state between
// two steps as one host byte string -- a header of the configuration and the rotation
// state, then every device buffer a later step reads, in a fixed order.
//
// Buffers are taken by role, never by address: the CDF-2 levels by their current meaning
// (phi^{n+1/2}, phi^{n-1/2}, ...), the BDF rings slot by slot with the head, the velocity
// buffers by index with vcur.  Loading writes the same roles of the target handle, so the
// target steps on exactly as the source would have.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstring>
#include <vector>

#include "gpic_internal.h"
#include "handle.h"
#include "pic.h"

using namespace gpic;

namespace {

// The configuration a state was saved under: the integer layout fields and every FP64
// parameter a later step uses (box, constants, time step, particle constants, the DIRK
// tableau and the species table).  A load compares them bit for bit.
struct StateHeader {
    char magic[8];
    int32_t nx, ny, p, stepper, cdf_form, bdf_order, dirk_stages, precision;
    int32_t sort_interval, vdim, nspecies, charge, tile, pad;
    int64_t n, step;
    int32_t vcur, head, head_r, stepped;
    uint64_t payload;
    double lx, ly, c, eps0, dt, q, m, weight;
    double dirk_a[16], dirk_b[4], dirk_c[4];
    double species_q[4], species_m[4], species_w[4];
};
constexpr char kMagic[8] = {'G', 'P', 'I', 'C', 'S', 'T', 'A', '4'};

struct Seg {
    void* p;
    size_t bytes;
};

std::vector<Seg> segments(pic_handle* h) {
    std::vector<Seg> s;
    const size_t pn = (size_t)h->n * h->rsz, cs = 2 * h->rsz, ng = h->ng;
    const size_t sb = ng * sizeof(double2);  // spectral histories are FP64 in both forms
    auto add = [&](void* p, size_t b) {
        if (p && b) s.push_back({p, b});
    };
    for (void* p : {h->x, h->y, h->px, h->py, h->v[0][0], h->v[0][1], h->v[1][0], h->v[1][1]})
        add(p, pn);
    if (h->vdim == 3)
        for (void* p : {h->pz, h->vz[0], h->vz[1]}) add(p, pn);
    if (h->spp.n > 0) add(h->species, (size_t)h->n * sizeof(int32_t));
    if (h->sorting) {
        add(h->id, (size_t)h->n * sizeof(int32_t));
        add(h->off, ((size_t)h->tg.nkeys() + 1) * sizeof(int));
    }
    add(h->J, h->jbytes);  // last step's current (128-bit sums, or int64 sums)
    add(h->G, 4 * ng * cs);
    if (h->vdim == 3) {
        add(h->Jz, h->jbytes);
        add(h->Gz, 2 * ng * cs);
    }
    switch (h->cfg.stepper) {
        case PIC_STEPPER_BDF:
            for (auto* l : {&h->phi_l, &h->ax_l, &h->ay_l, &h->rho_l, &h->az_l})
                for (void* p : *l) add(p, sb);
            break;
        case PIC_STEPPER_CDF2:
            for (void* p : {h->cdf.phi, h->cdf.phi_prev, h->cdf.rho, h->cdf.rho_prev, h->cdf.ax,
                            h->cdf.ax_prev, h->cdf.ay, h->cdf.ay_prev, h->cdf.jx, h->cdf.jx_prev,
                            h->cdf.jy, h->cdf.jy_prev, h->az, h->az_prev, h->jz, h->jz_prev})
                add(p, sb);
            break;
        default:
            for (void* p : {h->dirk.phi, h->dirk.vphi, h->dirk.ax, h->dirk.vax, h->dirk.ay,
                            h->dirk.vay, h->dirk.rho, h->dirk.jx, h->dirk.jy, h->az, h->vaz, h->jz})
                add(p, sb);
    }
    return s;
}

StateHeader header_of(pic_handle* h, uint64_t payload) {
    StateHeader hd{};
    std::memcpy(hd.magic, kMagic, 8);
    const pic_config& c = h->cfg;
    hd.nx = c.nx;
    hd.ny = c.ny;
    hd.p = c.spline_order;
    hd.stepper = c.stepper;
    hd.cdf_form = h->cdf.form;
    hd.bdf_order = c.bdf_order;
    hd.dirk_stages = c.dirk_stages;
    hd.precision = c.precision;
    hd.sort_interval = c.sort_interval;
    hd.vdim = h->vdim;
    hd.nspecies = h->spp.n;
    hd.charge = c.charge;
    hd.tile = h->sorting ? h->tg.t : 0;  // the tiles the saved order and offsets belong to
    hd.n = h->n;
    hd.step = h->step;
    hd.vcur = h->vcur;
    hd.head = h->head;
    hd.head_r = h->head_r;
    hd.stepped = h->stepped ? 1 : 0;
    hd.payload = payload;
    hd.lx = c.lx;
    hd.ly = c.ly;
    hd.c = c.c;
    hd.eps0 = c.eps0;
    hd.dt = c.dt;
    hd.q = c.q;
    hd.m = c.m;
    hd.weight = c.weight;
    // only the entries the configuration uses (the rest of a caller's struct may hold
    // anything); unused entries stay zero
    if (c.stepper == PIC_STEPPER_DIRK) {
        const int st = c.dirk_stages;
        for (int i = 0; i < st; ++i) {
            for (int j = 0; j < st; ++j) hd.dirk_a[i * st + j] = c.dirk_a[i * st + j];
            hd.dirk_b[i] = c.dirk_b[i];
            hd.dirk_c[i] = c.dirk_c[i];
        }
    }
    for (int k = 0; k < h->spp.n; ++k) {
        hd.species_q[k] = c.species_q[k];
        hd.species_m[k] = c.species_m[k];
        hd.species_w[k] = c.species_w[k];
    }
    return hd;
}

// Bitwise equality of the FP64 parameters of two headers (a state saved under another
// dt, box, constant, tableau or species table belongs to another configuration).
bool same_parameters(const StateHeader& a, const StateHeader& b) {
    const size_t first = offsetof(StateHeader, lx);
    const size_t last = offsetof(StateHeader, species_w) + sizeof(a.species_w);
    return std::memcmp(reinterpret_cast<const char*>(&a) + first,
                       reinterpret_cast<const char*>(&b) + first, last - first) == 0;
}

uint64_t payload_bytes(const std::vector<Seg>& segs) {
    uint64_t b = 0;
    for (const Seg& g : segs) b += g.bytes;
    return b;
}

}  // namespace

extern "C" {

pic_status pic_save_state(pic_handle* h, void* dst, size_t* size) {
    if (!h || !size) return fail(h, PIC_ERR_INVALID_ARG, "NULL argument");
    if (h->phase != 0) return fail(h, PIC_ERR_STATE, "pic_save_state inside a step");
    const std::vector<Seg> segs = segments(h);
    const uint64_t payload = payload_bytes(segs);
    const size_t need = sizeof(StateHeader) + payload;
    if (!dst) {
        *size = need;
        return PIC_OK;
    }
    if (*size < need) {
        *size = need;
        return fail(h, PIC_ERR_INVALID_ARG, "state buffer too small: %zu bytes needed", need);
    }
    const StateHeader hd = header_of(h, payload);
    std::memcpy(dst, &hd, sizeof hd);
    char* out = static_cast<char*>(dst) + sizeof hd;
    for (const Seg& g : segs) {
        CK(cudaMemcpyAsync(out, g.p, g.bytes, cudaMemcpyDefault, h->s));
        out += g.bytes;
    }
    *size = need;
    return check_device_error(h);  // synchronizes: dst is complete on return
}

pic_status pic_load_state(pic_handle* h, const void* src, size_t size) {
    if (!h || !src) return fail(h, PIC_ERR_INVALID_ARG, "NULL argument");
    if (h->phase != 0) return fail(h, PIC_ERR_STATE, "pic_load_state inside a step");
    if (size < sizeof(StateHeader)) return fail(h, PIC_ERR_INVALID_ARG, "not a saved state");
    StateHeader hd;
    std::memcpy(&hd, src, sizeof hd);
    if (std::memcmp(hd.magic, kMagic, 8) != 0)
        return fail(h, PIC_ERR_INVALID_ARG, "not a saved state of this library");
    const std::vector<Seg> segs = segments(h);
    const uint64_t payload = payload_bytes(segs);
    const StateHeader mine = header_of(h, payload);
    const bool same = hd.nx == mine.nx && hd.ny == mine.ny && hd.p == mine.p &&
                      hd.stepper == mine.stepper && hd.cdf_form == mine.cdf_form &&
                      hd.bdf_order == mine.bdf_order && hd.dirk_stages == mine.dirk_stages &&
                      hd.precision == mine.precision && hd.sort_interval == mine.sort_interval &&
                      hd.vdim == mine.vdim && hd.nspecies == mine.nspecies &&
                      hd.charge == mine.charge && hd.tile == mine.tile && hd.n == mine.n &&
                      hd.payload == payload &&
                      same_parameters(hd, mine);
    if (!same)
        return fail(h, PIC_ERR_INVALID_ARG,
                    "the saved state belongs to another configuration or particle count");
    if (size < sizeof hd + payload) return fail(h, PIC_ERR_INVALID_ARG, "truncated state");
    if (hd.vcur < 0 || hd.vcur > 1 || (h->L && (hd.head < 0 || hd.head >= h->L)) ||
        (h->Lr && (hd.head_r < 0 || hd.head_r >= h->Lr)))
        return fail(h, PIC_ERR_INVALID_ARG, "corrupt saved state");
    const char* in = static_cast<const char*>(src) + sizeof hd;
    for (const Seg& g : segs) {
        CK(cudaMemcpyAsync(g.p, in, g.bytes, cudaMemcpyDefault, h->s));
        in += g.bytes;
    }
    h->step = hd.step;
    h->vcur = hd.vcur;
    h->head = hd.head;
    h->head_r = hd.head_r;
    h->stepped = hd.stepped != 0;
    h->diag_valid = h->e_valid = false;
    // the diagnostics log restarts: records of steps before the load are not returned
    h->ring_read = h->ring_written;
    h->pending = false;  // a pending deposit of the old state is void
    if (h->fp32)  // the buffer the next deposit sums into starts at zero (the row
                  // transform keeps it so)
        CK(cudaMemsetAsync(h->Jalt, 0, h->ng * sizeof(double2), h->s));
    CK(cudaStreamSynchronize(h->s));  // src may be released on return
    return check_device_error(h);
}

}  // extern "C"
