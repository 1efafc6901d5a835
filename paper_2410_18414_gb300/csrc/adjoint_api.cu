// Host side of the adjoint API (include/pic.h): checkpoints of the forward run, the
// segment-by-segment recomputation and the reverse sweep of the step (BDF-k, the three
// CDF-2 forms or DIRK), for the plain FP64 path and the (unsorted) FP32 form.
//
// Storage (device; particle values in the handle's storage type T, everything else FP64):
//   state     the eight particle arrays of one time level, in the order x, y, Px, Py,
//             v^n (x, y), v^{n-1} (x, y): 8 n values
//   ck[c]     checkpoint c: the state at step c K and the field history (BDF: the ring
//             contents in slot order and the ring heads; CDF-2, DIRK: the levels by
//             role); ck[nseg] is the end of the run, with the last step's J and gather
//             fields, so the handle can be put back after the sweep
//   rec[j]    the state after step c0 + j of the segment being swept (j = 0..K-1)
//   records   per step (every step in the replay mode, the segment's in the recompute
//             mode): the gather fields the step used (recg, in T) and recf (FP64): P^{n+1},
//             v^{n+1} and the gathered A and grad A of each particle (10 n)
//   adjoint   particle adjoints (8 n, in T), the history adjoints (BDF: 3 L + k spectra, slot
//             of time level t = t mod L; CDF-2: 12 by role, each (cur, prev) pair swapped
//             after every reverse step; DIRK: 9 by role, in place), field-adjoint planes
//             and transform scratch, and FP64 twiddle tables for the reverse field solve
//             (an FP32-form handle's own tables are FP32)
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "gpic_internal.h"
#include "handle.h"
#include "pic.h"

using namespace gpic;

struct pic_adjoint {
    pic_handle* h = nullptr;
    int32_t nsteps = 0, K = 0, nseg = 0;
    int L = 0, Lr = 0;
    int kind = K_BDF;  // StepperKind of the handle
    int nh = 0;        // history spectra: 3 L + Lr (BDF), 12 (CDF-2), 9 (DIRK)
    size_t n = 0, ng = 0;
    bool f32 = false;  // the FP32 form: particle values in float
    size_t rsz = 8;    // bytes of one particle value
    struct Ck {
        void* state = nullptr;
        double2* hist = nullptr;  // nh spectra, slot or role order
        int head = 0, head_r = 0;
        int64_t step = 0;
    };
    std::vector<Ck> ck;
    double2* final_j = nullptr;  // J of the last step (the handle's sums, jbytes)
    void* final_g = nullptr;     // gather fields of the last step (4 ng complex of T)
    void* rec = nullptr;         // K states
    void* recg = nullptr;        // K x 4 ng complex of T
    double* recf = nullptr;      // per step 10 n: P^{n+1}, v^{n+1} and the gathered A, grad A
    int seg_held = -1;           // segment whose states rec holds
    int mode = 0;                // PIC_ADJ_REPLAY, PIC_ADJ_RECOMPUTE or PIC_ADJ_REPLAY_LEAN
    bool lean = false;           // records without the gathered values (re-gathered)
    void* ab = nullptr;          // particle adjoints, 8 n
    double2* twx = nullptr;      // FP64 twiddles along x and y
    double2* twy = nullptr;
    void* fb32 = nullptr;        // FP32 form: the field adjoints as summed, [node][8] float
    double2* hb = nullptr;       // history adjoints, nh ng
    double2* role[12] = {};      // CDF-2, DIRK: the history adjoint of each role
    double2* fb = nullptr;       // field-adjoint planes, 4 ng
    double2* zb = nullptr;       // their transforms, 4 ng
    double2* js = nullptr;       // adjoint current spectrum, ng
    double2* jg = nullptr;       // adjoint current on the mesh, ng
    double2* e0 = nullptr;       // E^0 on the mesh, ng (Ex, Ey)
    double2* tmp = nullptr;      // ng
    bool forward_done = false;
    std::vector<void*> allocs;
};

namespace {

cudaError_t aalloc(pic_adjoint* a, void** p, size_t bytes) {
    *p = nullptr;
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e == cudaSuccess) a->allocs.push_back(*p);
    return e;
}

void release(pic_adjoint* a) {
    for (void* p : a->allocs) cudaFree(p);
    a->allocs.clear();
}

// The handle's particle arrays in state order (v^n first).
void handle_arrays(pic_handle* h, void* arr[8]) {
    arr[0] = h->x;
    arr[1] = h->y;
    arr[2] = h->px;
    arr[3] = h->py;
    arr[4] = h->v[h->vcur][0];
    arr[5] = h->v[h->vcur][1];
    arr[6] = h->v[1 - h->vcur][0];
    arr[7] = h->v[1 - h->vcur][1];
}

// The field history of the handle: the BDF ring slots, or the CDF-2 and DIRK levels in
// role order (the buffer now in each role: CDF-2 swaps pairs every step).
std::vector<void*> ring_slots(pic_handle* h) {
    std::vector<void*> s;
    if (h->cfg.stepper == PIC_STEPPER_CDF2) {
        const CdfParams& c = h->cdf;
        return {c.phi, c.phi_prev, c.rho, c.rho_prev, c.ax, c.ax_prev,
                c.ay,  c.ay_prev,  c.jx,  c.jx_prev,  c.jy, c.jy_prev};
    }
    if (h->cfg.stepper == PIC_STEPPER_DIRK) {
        const DirkParams& d = h->dirk;
        return {d.phi, d.vphi, d.ax, d.vax, d.ay, d.vay, d.rho, d.jx, d.jy};
    }
    for (void* p : h->phi_l) s.push_back(p);
    for (void* p : h->ax_l) s.push_back(p);
    for (void* p : h->ay_l) s.push_back(p);
    for (void* p : h->rho_l) s.push_back(p);
    return s;
}

template <typename T>
Ptr8T<T> handle_ptrs(pic_handle* h) {
    void* arr[8];
    handle_arrays(h, arr);
    Ptr8T<T> p;
    for (int k = 0; k < 8; ++k) p.p[k] = (const T*)arr[k];
    return p;
}

// Byte offset of state j (or array k of a state) in a block of states.
size_t state_bytes(const pic_adjoint* a) { return 8 * a->n * a->rsz; }

pic_status save_state(pic_adjoint* a, void* dst) {
    pic_handle* h = a->h;
    CK(by_prec(h, [&](auto t) {
        using T = decltype(t);
        return launch_pack8<T>(handle_ptrs<T>(h), (T*)dst, (int64_t)a->n, h->s);
    }));
    return PIC_OK;
}

// FP64 2-D transforms with the adjoint's own twiddles (whatever the handle's precision).
cudaError_t fft64_forward(pic_adjoint* a, const double2* in, double2* out) {
    pic_handle* h = a->h;
    cudaError_t e = launch_fft_y<double>(in, out, h->nx, h->ny, 1, h->fy, a->twy, -1, 0, h->s);
    if (e != cudaSuccess) return e;
    return launch_fft_x<double>(out, out, h->nx, h->ny, 1, h->fx, a->twx, -1, h->s);
}
cudaError_t fft64_inverse(pic_adjoint* a, double2* buf, double2* out) {
    pic_handle* h = a->h;
    cudaError_t e = launch_fft_x<double>(buf, buf, h->nx, h->ny, 1, h->fx, a->twx, +1, h->s);
    if (e != cudaSuccess) return e;
    return launch_fft_y<double>(buf, out, h->nx, h->ny, 1, h->fy, a->twy, +1, 0, h->s);
}

pic_status save_checkpoint(pic_adjoint* a, pic_adjoint::Ck& c) {
    pic_handle* h = a->h;
    pic_status st = save_state(a, c.state);
    if (st != PIC_OK) return st;
    const std::vector<void*> slots = ring_slots(h);
    for (size_t i = 0; i < slots.size(); ++i)
        CK(cudaMemcpyAsync(c.hist + i * a->ng, slots[i], a->ng * sizeof(double2),
                           cudaMemcpyDeviceToDevice, h->s));
    c.head = h->head;
    c.head_r = h->head_r;
    c.step = h->step;
    return PIC_OK;
}

pic_status restore_checkpoint(pic_adjoint* a, const pic_adjoint::Ck& c) {
    pic_handle* h = a->h;
    h->vcur = 0;
    CK(by_prec(h, [&](auto t) {
        using T = decltype(t);
        return launch_unpack8<T>((const T*)c.state, handle_ptrs<T>(h), (int64_t)a->n, h->s);
    }));
    const std::vector<void*> slots = ring_slots(h);
    for (size_t i = 0; i < slots.size(); ++i)
        CK(cudaMemcpyAsync(slots[i], c.hist + i * a->ng, a->ng * sizeof(double2),
                           cudaMemcpyDeviceToDevice, h->s));
    h->head = c.head;
    h->head_r = c.head_r;
    h->step = c.step;
    h->phase = 0;
    return PIC_OK;
}

// Arrays of n in one step's record: P^{n+1} (2), v^{n+1} (2) and the gathered A, grad A
// (6); the lean record keeps the first four.
size_t rec_width(const pic_adjoint* a) { return a->lean ? 4 : 10; }

int seg_begin(const pic_adjoint* a, int c) { return c * a->K; }
int seg_end(const pic_adjoint* a, int c) { return std::min(a->nsteps, (c + 1) * a->K); }

// Record slot of step s: every step has its own in the replay mode; in the recompute mode
// the slots are reused by each segment.
size_t rec_slot(const pic_adjoint* a, int s) {
    return a->mode != PIC_ADJ_RECOMPUTE ? (size_t)s : (size_t)(s % a->K);
}

// One forward step of h (step s of the run), keeping the step's gather fields and the
// values its push gathered, and (state_j >= 0) the new state in segment slot state_j.
pic_status step_and_record(pic_adjoint* a, int s, int state_j) {
    pic_handle* h = a->h;
    const size_t r = rec_slot(a, s);
    h->gather_out = a->recf + r * rec_width(a) * a->n;
    h->gather_out_short = a->lean;
    pic_status st = pic_step(h, 1);
    h->gather_out = nullptr;
    h->gather_out_short = false;
    if (st != PIC_OK) return st;
    if (state_j >= 0) {
        st = save_state(a, (char*)a->rec + (size_t)state_j * state_bytes(a));
        if (st != PIC_OK) return st;
    }
    const size_t gbytes = 4 * a->ng * 2 * a->rsz;
    CK(cudaMemcpyAsync((char*)a->recg + r * gbytes, h->G, gbytes, cudaMemcpyDeviceToDevice,
                       h->s));
    return PIC_OK;
}

template <typename T>
AdjParticlesT<T> adjoint_arrays(pic_adjoint* a) {
    T* b = (T*)a->ab;
    const size_t n = a->n;
    return AdjParticlesT<T>{b, b + n, b + 2 * n, b + 3 * n, b + 4 * n, b + 5 * n, b + 6 * n,
                            b + 7 * n};
}

double2* hist_slot(pic_adjoint* a, int field, int64_t t) {
    // field 0..2: phi, Ax, Ay (L slots each); 3: rho (Lr slots)
    if (field == 3) {
        const int s = (int)(((t % a->Lr) + a->Lr) % a->Lr);
        return a->hb + (size_t)(3 * a->L + s) * a->ng;
    }
    const int s = (int)(((t % a->L) + a->L) % a->L);
    return a->hb + (size_t)(field * a->L + s) * a->ng;
}

// Reverse of step n (from level n+1 to level n): s0 = state n, s1 = state n+1 (in T),
// g = the gather fields of the step.
pic_status backward_step(pic_adjoint* a, int64_t n, const void* s0v, const void* s1v,
                         const double* gf, const void* g) {
    pic_handle* h = a->h;
    const size_t np = a->n, ng = a->ng;
    if (a->f32)
        CK(cudaMemsetAsync(a->fb32, 0, ng * 8 * sizeof(float), h->s));
    else
        CK(cudaMemsetAsync(a->fb, 0, 4 * ng * sizeof(double2), h->s));
    TimedScope tp(h, PIC_KT_ADJ_PUSH);
    CK(by_prec(h, [&](auto t) {
        using T = decltype(t);
        const T* s0 = (const T*)s0v;
        const T* s1 = (const T*)s1v;
        return launch_adj_push_gather<T>(h->p, h->geom, h->push, s1, s1 + np, s1 + 2 * np,
                                         s1 + 3 * np, s0 + 4 * np, s0 + 5 * np, s0 + 6 * np,
                                         s0 + 7 * np, gf, a->lean, g, adjoint_arrays<T>(a),
                                         a->fb, a->fb32, (int64_t)np, h->err, h->s);
    }));
    if (a->f32) CK(launch_fb32_to_planes(a->fb32, a->fb, (int64_t)ng, h->s));
    tp.end();
    TimedScope tf(h, PIC_KT_ADJ_FIELD);
    CK(launch_fft_y<double>(a->fb, a->zb, h->nx, h->ny, 4, h->fy, a->twy, -1, 0, h->s));
    const bool fused = adj_columns_smem(h->nx) <= kFieldColumnsSmemMax;
    if (!fused) CK(launch_fft_x<double>(a->zb, a->zb, h->nx, h->ny, 4, h->fx, a->twx, -1, h->s));
    AdjModeParams ap{};
    CdfParams cp{};
    DirkParams dp{};
    if (a->kind == K_BDF) {
        ap.k = h->bdf.k;
        for (int i = 0; i <= ap.k; ++i) ap.a[i] = h->bdf.a[i];
        for (int d = 0; d <= 2 * ap.k; ++d) ap.C[d] = h->bdf.C[d];
        ap.g = h->bdf.g;
        ap.bdt = h->bdf.bdt;
        for (int d = 0; d < a->L; ++d) {
            ap.phi[d] = hist_slot(a, 0, n + 1 - d);
            ap.ax[d] = hist_slot(a, 1, n + 1 - d);
            ap.ay[d] = hist_slot(a, 2, n + 1 - d);
        }
        for (int d = 0; d < a->Lr; ++d) ap.rho[d] = hist_slot(a, 3, n + 1 - d);
    } else if (a->kind == K_CDF2) {
        cp.form = h->cdf.form;
        void** roles[12] = {&cp.phi, &cp.phi_prev, &cp.rho, &cp.rho_prev, &cp.ax, &cp.ax_prev,
                            &cp.ay,  &cp.ay_prev,  &cp.jx,  &cp.jx_prev,  &cp.jy, &cp.jy_prev};
        for (int r = 0; r < 12; ++r) *roles[r] = a->role[r];
    } else {
        dp = h->dirk;  // the stage table; the state pointers become the adjoints
        void** roles[9] = {&dp.phi, &dp.vphi, &dp.ax, &dp.vax, &dp.ay, &dp.vay, &dp.rho, &dp.jx, &dp.jy};
        for (int r = 0; r < 9; ++r) *roles[r] = a->role[r];
    }
    if (fused) {
        CK(launch_adj_columns(h->mc, a->kind, ap, cp, dp, a->zb, a->js, h->fx, a->twx, h->s));
        CK(launch_fft_y<double>(a->js, a->jg, h->nx, h->ny, 1, h->fy, a->twy, +1, 0, h->s));
    } else {
        CK(launch_adj_modes(h->mc, a->kind, ap, cp, dp, a->zb, a->js, h->s));
        CK(fft64_inverse(a, a->js, a->jg));
    }
    // CDF-2: the adjoints before the step were written into the other buffer of each pair
    if (a->kind == K_CDF2)
        for (int r = 0; r < 12; r += 2) std::swap(a->role[r], a->role[r + 1]);
    tf.end();
    TimedScope td(h, PIC_KT_ADJ_DEPOSIT);
    CK(by_prec(h, [&](auto t) {
        using T = decltype(t);
        const T* s0 = (const T*)s0v;
        const T* s1 = (const T*)s1v;
        return launch_adj_deposit_move<T>(h->p, h->geom, s1, s1 + np, s0 + 4 * np, s0 + 5 * np,
                                          a->jg, adjoint_arrays<T>(a), (int64_t)np, h->err,
                                          h->s);
    }));
    return PIC_OK;
}

}  // namespace

extern "C" {

pic_status pic_adjoint_create(pic_handle* h, int32_t nsteps, int32_t checkpoint_every,
                              pic_adjoint** out) {
    return pic_adjoint_create_ex(h, nsteps, checkpoint_every, PIC_ADJ_REPLAY, out);
}

pic_status pic_adjoint_create_ex(pic_handle* h, int32_t nsteps, int32_t checkpoint_every,
                                 int32_t mode, pic_adjoint** out) {
    if (!out) return fail(h, PIC_ERR_INVALID_ARG, "out must not be NULL");
    if (mode != PIC_ADJ_REPLAY && mode != PIC_ADJ_RECOMPUTE && mode != PIC_ADJ_REPLAY_LEAN)
        return fail(h, PIC_ERR_INVALID_ARG, "unknown adjoint record mode %d", mode);
    *out = nullptr;
    if (!h) return fail(nullptr, PIC_ERR_INVALID_ARG, "NULL handle");
    if (nsteps < 1) return fail(h, PIC_ERR_INVALID_ARG, "nsteps must be >= 1");
    if (h->cfg.charge != PIC_CHARGE_CONTINUITY || h->sorting || h->vdim == 3 || h->spp.n > 0)
        return fail(h, PIC_ERR_UNSUPPORTED,
                    "the adjoint needs the continuity charge, one species in 2D-2V and no "
                    "sorting");
    if (h->step != 0 || h->phase != 0)
        return fail(h, PIC_ERR_STATE, "the adjoint needs a handle fresh from pic_init");
    pic_adjoint* a = new pic_adjoint();
    a->h = h;
    a->nsteps = nsteps;
    a->K = std::max(1, std::min(checkpoint_every, nsteps));
    a->nseg = (nsteps + a->K - 1) / a->K;
    a->mode = mode;
    a->lean = mode == PIC_ADJ_REPLAY_LEAN;
    const size_t nrec = mode != PIC_ADJ_RECOMPUTE ? (size_t)nsteps : (size_t)a->K;
    a->L = h->L;
    a->Lr = h->Lr;
    a->kind = h->cfg.stepper == PIC_STEPPER_BDF ? K_BDF
              : h->cfg.stepper == PIC_STEPPER_CDF2 ? K_CDF2 : K_DIRK;
    a->nh = a->kind == K_BDF ? 3 * a->L + a->Lr : a->kind == K_CDF2 ? 12 : 9;
    a->n = (size_t)h->n;
    a->ng = h->ng;
    a->f32 = h->fp32;
    a->rsz = h->rsz;
    const size_t sb = 8 * std::max<size_t>(a->n, 1) * a->rsz;
    const size_t hbytes = (size_t)a->nh * a->ng * sizeof(double2);
    const size_t gb = a->ng * sizeof(double2);
    cudaError_t e = cudaSuccess;
    a->ck.resize(a->nseg + 1);
    for (auto& c : a->ck) {
        if (e == cudaSuccess) e = aalloc(a, (void**)&c.state, sb);
        if (e == cudaSuccess) e = aalloc(a, (void**)&c.hist, hbytes);
    }
    const size_t gfb = 4 * a->ng * 2 * a->rsz;  // one step's gather fields
    if (e == cudaSuccess) e = aalloc(a, (void**)&a->final_j, h->jbytes);
    if (e == cudaSuccess) e = aalloc(a, &a->final_g, gfb);
    if (e == cudaSuccess) e = aalloc(a, &a->rec, (size_t)a->K * sb);
    if (e == cudaSuccess) e = aalloc(a, &a->recg, nrec * gfb);
    if (e == cudaSuccess)
        e = aalloc(a, (void**)&a->recf,
                   nrec * rec_width(a) * std::max<size_t>(a->n, 1) * sizeof(double));
    if (e == cudaSuccess) e = aalloc(a, &a->ab, sb);
    if (e == cudaSuccess && a->f32) e = aalloc(a, &a->fb32, a->ng * 8 * sizeof(float));
    if (e == cudaSuccess) e = aalloc(a, (void**)&a->twx, (size_t)h->nx * sizeof(double2));
    if (e == cudaSuccess) e = aalloc(a, (void**)&a->twy, (size_t)h->ny * sizeof(double2));
    if (e == cudaSuccess) e = launch_twiddles<double>(a->twx, h->nx, h->s);
    if (e == cudaSuccess) e = launch_twiddles<double>(a->twy, h->ny, h->s);
    if (e == cudaSuccess) e = aalloc(a, (void**)&a->hb, hbytes);
    if (e == cudaSuccess) e = aalloc(a, (void**)&a->fb, 4 * gb);
    if (e == cudaSuccess) e = aalloc(a, (void**)&a->zb, 4 * gb);
    if (e == cudaSuccess) e = aalloc(a, (void**)&a->js, gb);
    if (e == cudaSuccess) e = aalloc(a, (void**)&a->jg, gb);
    if (e == cudaSuccess) e = aalloc(a, (void**)&a->e0, gb);
    if (e == cudaSuccess) e = aalloc(a, (void**)&a->tmp, gb);
    // E^0 = -grad phi^0 on the mesh (every phi level holds phi^0 at step 0)
    const void* phi0 = a->kind == K_BDF ? h->phi_l[h->head] : a->kind == K_CDF2 ? h->cdf.phi : h->dirk.phi;
    if (e == cudaSuccess) e = launch_adj_e0(h->mc, (const double2*)phi0, a->tmp, h->s);
    if (e == cudaSuccess) e = fft64_inverse(a, a->tmp, a->e0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    if (e != cudaSuccess) {
        release(a);
        delete a;
        return fail(h, PIC_ERR_CUDA, "pic_adjoint_create: %s", cudaGetErrorString(e));
    }
    *out = a;
    return PIC_OK;
}

pic_status pic_adjoint_forward(pic_adjoint* a) {
    NvtxRange r("adjoint_forward");
    if (!a) return fail(nullptr, PIC_ERR_INVALID_ARG, "NULL adjoint");
    pic_handle* h = a->h;
    if (a->forward_done) return fail(h, PIC_ERR_STATE, "pic_adjoint_forward runs once");
    if (h->step != 0 || h->phase != 0)
        return fail(h, PIC_ERR_STATE, "the handle has stepped since pic_adjoint_create");
    a->forward_done = true;
    const bool replay = a->mode != PIC_ADJ_RECOMPUTE;
    for (int c = 0; c < a->nseg; ++c) {
        pic_status st = save_checkpoint(a, a->ck[c]);
        if (st != PIC_OK) return st;
        const bool last = c == a->nseg - 1;
        for (int s = seg_begin(a, c); s < seg_end(a, c); ++s) {
            // replay: every step's records, no states; recompute: the last segment's
            // records and states, which the backward pass then need not recompute
            if (replay)
                st = step_and_record(a, s, -1);
            else
                st = last ? step_and_record(a, s, s - seg_begin(a, c)) : pic_step(h, 1);
            if (st != PIC_OK) return st;
        }
    }
    a->seg_held = replay ? -1 : a->nseg - 1;
    pic_status st = save_checkpoint(a, a->ck[a->nseg]);
    if (st != PIC_OK) return st;
    CK(cudaMemcpyAsync(a->final_j, h->J, h->jbytes, cudaMemcpyDeviceToDevice, h->s));
    CK(cudaMemcpyAsync(a->final_g, h->G, 4 * a->ng * 2 * a->rsz, cudaMemcpyDeviceToDevice,
                       h->s));
    return PIC_OK;
}

pic_status pic_adjoint_backward(pic_adjoint* a, const double* bz_bar, const double* px_bar,
                                const double* py_bar, double* dvx0, double* dvy0, double* dpx0,
                                double* dpy0) {
    NvtxRange r("adjoint_backward");
    if (!a) return fail(nullptr, PIC_ERR_INVALID_ARG, "NULL adjoint");
    pic_handle* h = a->h;
    if (!a->forward_done) return fail(h, PIC_ERR_STATE, "pic_adjoint_backward needs pic_adjoint_forward");
    if (h->phase != 0) return fail(h, PIC_ERR_STATE, "pic_adjoint_backward inside a step");
    const size_t np = a->n, ng = a->ng;
    const size_t hbytes = (size_t)a->nh * ng * sizeof(double2);
    CK(cudaMemsetAsync(a->ab, 0, 8 * std::max<size_t>(np, 1) * a->rsz, h->s));
    CK(cudaMemsetAsync(a->hb, 0, hbytes, h->s));
    if (a->kind != K_BDF)
        for (int r = 0; r < a->nh; ++r) a->role[r] = a->hb + (size_t)r * ng;
    // momentum seeds, converted to the particle storage type (through the FP64 staging
    // buffer of the handle)
    const double* pbar[2] = {px_bar, py_bar};
    for (int c = 0; c < 2; ++c) {
        if (!pbar[c] || !np) continue;
        void* dst = (char*)a->ab + (2 + c) * np * a->rsz;
        if (!a->f32) {
            CK(cudaMemcpyAsync(dst, pbar[c], np * sizeof(double), cudaMemcpyDefault, h->s));
        } else {
            CK(cudaMemcpyAsync(h->stage, pbar[c], np * sizeof(double), cudaMemcpyDefault, h->s));
            CK(launch_convert<double, float>(h->stage, (float*)dst, (int64_t)np, h->s));
        }
    }
    if (bz_bar) {
        CK(launch_real_to_cplx(bz_bar, a->tmp, (int64_t)ng, h->s));
        CK(fft64_forward(a, a->tmp, a->js));
        // the newest A: the BDF ring slot of the last level, else the A role (CDF-2: 4, 6;
        // DIRK: 2, 4)
        double2* sax = a->kind == K_BDF ? hist_slot(a, 1, a->nsteps)
                       : a->role[a->kind == K_CDF2 ? 4 : 2];
        double2* say = a->kind == K_BDF ? hist_slot(a, 2, a->nsteps)
                       : a->role[a->kind == K_CDF2 ? 6 : 4];
        CK(launch_adj_seed(h->mc, a->js, sax, say, h->s));
    }
    for (int c = a->nseg - 1; c >= 0; --c) {
        const int c0 = seg_begin(a, c), c1 = seg_end(a, c);
        if (a->seg_held != c) {
            if (a->mode != PIC_ADJ_RECOMPUTE) {
                // the segment's particle states from its checkpoint and the recorded fields
                for (int s = c0; s < c1; ++s) {
                    const int j = s - c0;
                    const void* s0 = j == 0 ? a->ck[c].state
                                            : (char*)a->rec + (size_t)(j - 1) * state_bytes(a);
                    void* s1 = (char*)a->rec + (size_t)j * state_bytes(a);
                    const double* rf = a->recf + rec_slot(a, s) * rec_width(a) * np;
                    CK(by_prec(h, [&](auto t) {
                        using T = decltype(t);
                        return launch_replay_step<T>(h->geom, (const T*)s0, (T*)s1, rf,
                                                     (int64_t)np, h->s);
                    }));
                }
            } else {
                pic_status st = restore_checkpoint(a, a->ck[c]);
                if (st != PIC_OK) return st;
                for (int s = c0; s < c1; ++s) {
                    st = step_and_record(a, s, s - c0);
                    if (st != PIC_OK) return st;
                }
            }
            a->seg_held = c;
        }
        for (int s = c1 - 1; s >= c0; --s) {
            const int j = s - c0;
            const void* s0 = j == 0 ? a->ck[c].state
                                    : (char*)a->rec + (size_t)(j - 1) * state_bytes(a);
            const void* s1 = (char*)a->rec + (size_t)j * state_bytes(a);
            pic_status st = backward_step(a, s, s0, s1,
                                          a->recf + rec_slot(a, s) * rec_width(a) * np,
                                          (char*)a->recg + rec_slot(a, s) * 4 * ng * 2 * a->rsz);
            if (st != PIC_OK) return st;
        }
    }
    CK(by_prec(h, [&](auto t) {
        using T = decltype(t);
        const T* x0 = (const T*)a->ck[0].state;
        return launch_adj_init<T>(h->p, h->geom, h->push, x0, x0 + np, x0 + 4 * np, x0 + 5 * np,
                                  a->e0, adjoint_arrays<T>(a), dvx0, dvy0, dpx0, dpy0,
                                  (int64_t)np, h->err, h->s);
    }));
    // put the handle back at the end of the forward run
    pic_status st = restore_checkpoint(a, a->ck[a->nseg]);
    if (st != PIC_OK) return st;
    CK(cudaMemcpyAsync(h->J, a->final_j, h->jbytes, cudaMemcpyDeviceToDevice, h->s));
    CK(cudaMemcpyAsync(h->G, a->final_g, 4 * ng * 2 * a->rsz, cudaMemcpyDeviceToDevice, h->s));
    return check_device_error(h);
}

int32_t pic_adjoint_checkpoint_every(const pic_adjoint* a) { return a ? a->K : 0; }

void pic_adjoint_destroy(pic_adjoint* a) {
    if (!a) return;
    if (a->h) cudaStreamSynchronize(a->h->s);
    release(a);
    delete a;
}

}  // extern "C"
