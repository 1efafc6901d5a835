// The simulation handle behind the opaque pic_handle of include/pic.h and the host
// helpers the library's API translation units share.  Internal: not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <string>
#include <vector>

#include "gpic_internal.h"
#include "pic.h"

struct pic_handle {
    pic_config cfg{};
    // kernel timing (pic_set_kernel_timing): per timer, event pairs created up front
    struct KTimer {
        std::vector<cudaEvent_t> ev;  // start, stop, start, stop, ...
        int64_t used = 0;             // pairs recorded since timing started
    };
    KTimer kt[PIC_KT_COUNT];
    bool ktiming = false;
    int64_t kt_cap = 0;  // pairs each timer may record since timing started
    cudaStream_t s = nullptr;
    int device = 0;
    int64_t n = 0;
    bool fp32 = false;
    size_t rsz = 8;
    int p = 2;
    int nx = 0, ny = 0;
    size_t ng = 0;
    // particle state (FP64 or FP32 by precision); v[buffer][component]
    void *x = nullptr, *y = nullptr, *px = nullptr, *py = nullptr;
    void* v[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int vcur = 0;             // v[vcur] holds v^n, v[1 - vcur] holds v^{n-1}
    bool bound = false;       // x, y, px, py, v are the caller's arrays (pic_init_bound)
    double* stage = nullptr;  // FP64 staging for conversions (n values)
    // tile sort (sort_interval > 0): second set of particle arrays, original indices, keys
    bool sorting = false;
    gpic::TileGeom tg{};
    void* alt[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int32_t *id = nullptr, *id_alt = nullptr;
    int32_t* species_alt = nullptr;                 // species indices (a species table)
    void* z_alt[3] = {nullptr, nullptr, nullptr};   // 2D-3V: P_z, v_z[0], v_z[1]
    int *keys = nullptr, *hist = nullptr, *off = nullptr, *cursor = nullptr, *bsum = nullptr;
    int launches_now = 0, launches_last = 0;
    // grid buffers
    double2* J = nullptr;    // deposit accumulator (sum_p v W): 128-bit sums (FP64 path:
                             // longlong2 low words, then high words), or int64 pairs (FP32 form)
    double2* Jalt = nullptr; // FP32 form: the other int64 buffer, zeroed by the row transform
    // FP32 form: a contribution a is summed as round(a * fix_scale_*) in int64
    float fix_scale_j = 0.f, fix_scale_q = 0.f;
    double fix_unscale_j = 0.0, fix_unscale_q = 0.0;
    // FP64 path: round(a * fix64_scale_*) summed as 128-bit integers (two words a value)
    double fix64_scale_j = 0.0, fix64_scale_q = 0.0;
    double fix64_unscale_j = 0.0, fix64_unscale_q = 0.0;
    size_t jbytes = 0;  // bytes of one current, charge or J_z buffer: 16 or 32 a node
    void* Z = nullptr;       // spectrum of J (complex)
    void* F4 = nullptr;      // 4 packed field spectra, inverse-transformed in place
    void* G = nullptr;       // [node][4] complex: the eight real gather fields
    double* gather_out = nullptr;  // where gather_push also writes the adjoint's record of
                                   // the step (its recording steps), else NULL
    bool gather_out_short = false; // the record without the gathered values (P, v only)
    void* E = nullptr;       // packed E spectrum of the last diagnosed step
    void* tmp = nullptr;     // complex scratch (ng)
    // naive update (PIC_CHARGE_DEPOSIT): the deposited charge (FP64 pairs, or int64 sums
    // in the FP32 form) and its spectrum
    void* rhoq = nullptr;
    void* ZQ = nullptr;
    double* tmpd = nullptr;  // real scratch (ng)
    void *twx = nullptr, *twy = nullptr;
    gpic::FftDesc fx{}, fy{};
    // 2D-3V (vdim 3) and species tables
    int vdim = 2;
    gpic::SpeciesParams spp{};        // spp.n = 0: one species (q, m, weight of cfg)
    int32_t* species = nullptr;       // each particle's species index (device)
    void* pz = nullptr;               // P_z (constant: d/dz = 0)
    void* vz[2] = {nullptr, nullptr}; // v_z, rotated with v
    void* Jz = nullptr;               // J_z sums in the .x parts (double2, or longlong2)
    void* Zz = nullptr;               // spectrum of J_z
    void* F2 = nullptr;               // the two packed A_z output spectra
    void* Gz = nullptr;               // [node][2] complex: (dAz/dx, dAz/dy), (Az, 0)
    std::vector<void*> az_l;          // BDF: A_z ring (the slots and head of phi, Ax, Ay)
    void *az = nullptr, *az_prev = nullptr, *jz = nullptr, *jz_prev = nullptr,
         *vaz = nullptr;              // CDF-2: A_z^n, A_z^{n-1}, J_z^n, J_z^{n-1}; DIRK: az, vaz, jz
    // time histories (BDF rings; CDF pairs; DIRK state)
    std::vector<void*> phi_l, ax_l, ay_l, rho_l;
    int L = 0, Lr = 0, head = 0, head_r = 0;
    gpic::BdfParams bdf{};
    gpic::CdfParams cdf{};
    gpic::DirkParams dirk{};
    // diagnostics and errors
    double* diag = nullptr;
    unsigned int* err = nullptr;
    int diag_every = 0;
    bool diag_now = false, diag_valid = false, e_valid = false;
    int64_t diag_step = -1;
    // per-step records (pic_diagnostics_history): a device ring of PIC_DIAG_HISTORY x
    // D_NSLOTS accumulators, each slot's step on the host, the records not yet read
    double* diag_ring = nullptr;
    std::vector<int64_t> ring_step;
    int64_t ring_written = 0, ring_read = 0;
    int64_t step = 0;
    int phase = 0;  // 0: ready to deposit, 1: deposited, 2: fields solved
    bool fused_deposit = false;  // phase 1 reached by the fused gather + deposit of pic_step
    // The sorted FP32 form ends a pic_step call with the fused kernel too: the next step's
    // moved positions wait in xnext, ynext and its current in Jalt (pending); the handle's
    // state is unchanged otherwise.  The next deposit swaps them in; anything else that
    // changes the state drops them (drop_pending).
    void *xnext = nullptr, *ynext = nullptr;
    bool pending = false;
    bool no_defer = false;  // set while an ensemble captures the run's steps
    bool stepped = false;
    std::vector<void*> allocs;
    gpic::ModeCommon mc{};
    gpic::ParticleGeom geom{};
    gpic::PushParams push{};
    std::string errmsg;
};

namespace gpic {

// Records the formatted message on h (or as the last pic_init error when h is NULL) and
// returns st.
pic_status fail(pic_handle* h, pic_status st, const char* fmt, ...);

// Run f with a value of the storage type (double or float).
template <typename F>
cudaError_t by_prec(pic_handle* h, F&& f) {
    if (h->fp32) return f(float{});
    return f(double{});
}

// Forward 2-D transform of one complex array (along y, then along x in place).
cudaError_t forward_fft(pic_handle* h, const void* in, void* out);
// Inverse transform of nb packed spectra in `buf` (in place along x), then along y into
// `out` (interleaved by array when nb > 1).
cudaError_t inverse_fft(pic_handle* h, void* buf, void* out, int nb);
// Waits for the stream and maps the device error word to a status.
pic_status check_device_error(pic_handle* h);
// Forgets a pending deposit (see pic_handle::pending): the current buffer it filled is
// cleared for the next deposit.
cudaError_t drop_pending(pic_handle* h);

// NVTX ranges of the library, in the domain "gpic" (host-side markers for timeline and
// profiler tools: nsys, or ncu --nvtx --nvtx-include "gpic@deposit/"); a push without an
// attached tool is a check of a function pointer.
nvtxDomainHandle_t nvtx_domain();
void nvtx_push(const char* name);
inline void nvtx_pop() { nvtxDomainRangePop(nvtx_domain()); }
// The range names of the kernel timers (PIC_KT_*): sort, deposit, field_solve,
// gather_push, adj_push, adj_field, adj_deposit, gather_deposit.
const char* timer_name(int which);

class NvtxRange {
  public:
    explicit NvtxRange(const char* name) { nvtx_push(name); }
    ~NvtxRange() { nvtx_pop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Brackets one launch group with an NVTX range named for the timer and, when timing is
// on and a pair is left, with the timer's next event pair; the range ends and the stop
// event is recorded by end() or when the scope ends, early returns included.
class TimedScope {
  public:
    TimedScope(pic_handle* h, int which) {
        nvtx_push(timer_name(which));
        open_ = true;
        if (!h->ktiming) return;
        auto& t = h->kt[which];
        if (t.used >= h->kt_cap || 2 * (t.used + 1) > (int64_t)t.ev.size()) return;
        stop_ = t.ev[2 * t.used + 1];
        s_ = h->s;
        cudaEventRecord(t.ev[2 * t.used], s_);
        ++t.used;
    }
    ~TimedScope() { end(); }
    // Records the stop event and ends the range now (once).
    void end() {
        if (stop_) cudaEventRecord(stop_, s_);
        stop_ = nullptr;
        if (open_) nvtx_pop();
        open_ = false;
    }
    TimedScope(const TimedScope&) = delete;
    TimedScope& operator=(const TimedScope&) = delete;

  private:
    cudaEvent_t stop_ = nullptr;
    cudaStream_t s_ = nullptr;
    bool open_ = false;
};

}  // namespace gpic

// Returns PIC_ERR_CUDA from the enclosing function (with the call's text as the message
// on h) when a CUDA runtime call fails.
#define CK(...)                                                                           \
    do {                                                                                  \
        cudaError_t e_ = (__VA_ARGS__);                                                        \
        if (e_ != cudaSuccess)                                                            \
            return fail(h, PIC_ERR_CUDA, "%s failed: %s", #__VA_ARGS__, cudaGetErrorString(e_)); \
    } while (0)
