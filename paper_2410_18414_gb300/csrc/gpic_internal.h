// Internal declarations shared by the translation units of libgpic: kernel
// launchers and their parameter blocks.  Not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gpic {

constexpr int kMaxRadices = 16;
constexpr int kMaxBdf = 6;
constexpr int kMaxDirk = 4;
constexpr int kMaxSpecies = 4;

// Per-particle constants from a species table: section 2.2 writes the equations of motion
// and the densities with each particle's own charge and mass, section 2.1 sums the
// densities over species.  n = 0: one species (the kernels take the plain path and never
// read the index array).  With a table the deposits multiply each contribution by q_s w_s
// (the handle's current scale is then 1/(dx dy)).
struct SpeciesParams {
    int n;
    double qw[kMaxSpecies];
    double q[kMaxSpecies], m[kMaxSpecies], w[kMaxSpecies];
};

// 1-D transform description: length n = prod(radix[0..nf-1]), radices in {2,3,4}.
// Per pass f, precomputed on the host: Ns (product of the earlier radices), nr = n / R,
// the twiddle stride n / (Ns R), and multipliers ceil(2^32 / d) that divide indices
// below 2^16 exactly by d = nr or Ns with one multiply-high (0 when d = 1).
struct FftDesc {
    int n;
    int nf;
    int radix[kMaxRadices];
    int ns[kMaxRadices];
    int nr[kMaxRadices];
    int twstep[kMaxRadices];
    unsigned m_nr[kMaxRadices];
    unsigned m_ns[kMaxRadices];
};

// Diagnostic accumulators (device, FP64): sums of |.|^2 over modes and particles.
enum DiagSlot {
    D_GAUGE = 0, D_GAUSS, D_CONT, D_GAUGE_DT, D_RHO, D_DIVA, D_WE, D_WB, D_KIN, D_NSLOTS
};

// Per-mode kernel parameters common to all steppers.
struct ModeCommon {
    int nx, ny;
    double kx_scale, ky_scale;  // 2 pi / L
    double jscale;              // q_p / (dx dy): raw deposit sums -> current density
    double inv_n;               // 1 / (nx ny): inverse-FFT normalisation folded in
    double eps0, mu0, c, dt;
    // host-computed constants of the per-mode updates (the same roundings as the device
    // expressions they replace, so no mode divides): 1/eps0 and CDF-2's th/eps0 with
    // th = 0.5 c^2 dt^2
    double inv_eps0, cdf_th_eps0;
    int diag;                   // accumulate diagnostics this step
    // precomputed FP64 tables (pic_init): wavenumbers per axis and the inverse implicit-
    // solve denominator per mode (BDF: 1/(C_0 + g K); CDF: 1/(1 + th K); DIRK stage i:
    // invd[i*nx*ny + mode] = 1/(1 + (h a_ii c)^2 K))
    const double* kxt;
    const double* kyt;
    const double* invd;
    // DIRK: the step as one real 2 x 4 matrix per mode, (u', v') = M (u, v, S^n, S^{n+1}),
    // dirkm[8 mode + 4 r + k] (built from the stage recurrence on unit inputs); else NULL
    const double* dirkm;
    // naive update (PIC_CHARGE_DEPOSIT): spectrum of the charge deposited at x^{n+1}
    // (raw shape-weight sums, storage type of the form); NULL: continuity
    const void* zq;
};

struct BdfParams {
    int k;
    double a[kMaxBdf + 1];
    double C[2 * kMaxBdf + 1];
    double g;       // (c beta dt)^2
    double bdt;     // beta dt
    double inv_a0;  // 1 / a[0] (host-computed, so no mode divides)
    double g_eps0;  // g / eps0 (host-computed)
    // history, newest first: hist[d-1] is level n+1-d
    void* phi[2 * kMaxBdf];
    void* ax[2 * kMaxBdf];
    void* ay[2 * kMaxBdf];
    void* rho[kMaxBdf];
    // where the new level goes (the slot of the oldest level, read first)
    void* phi_new;
    void* ax_new;
    void* ay_new;
    void* rho_new;
};

struct CdfParams {
    // levels: phi^{n+1/2}, phi^{n-1/2} (new phi^{n+3/2} overwrites phi_prev), same for rho;
    // A^n, A^{n-1} (new A^{n+1} overwrites *_prev); J^n, J^{n-1} (new J overwrites j_prev)
    void *phi, *phi_prev, *rho, *rho_prev, *ax, *ax_prev, *ay, *ay_prev;
    void *jx, *jx_prev, *jy, *jy_prev;
    int form;  // 0 implicit, 1 semi-implicit, 2 explicit (section 3.1)
};

struct DirkParams {
    int s;
    double a[kMaxDirk * kMaxDirk];
    double b[kMaxDirk];
    double c[kMaxDirk];
    double r0, r1;
    // state at level n, updated in place
    void *phi, *vphi, *ax, *vax, *ay, *vay, *rho, *jx, *jy;
};

enum StepperKind { K_BDF = 0, K_CDF2 = 1, K_DIRK = 2 };

// ---------------------------------------------------------------- launchers

// In-place or out-of-place 1-D transforms of nb arrays of shape (nx, ny).
// Along y (contiguous); out_interleave != 0 writes out[(i*ny + j)*nb + b].
template <typename T>
cudaError_t launch_fft_y(const void* in, void* out, int nx, int ny, int nb, const FftDesc& d,
                         const void* twiddle, int sign, int out_interleave, cudaStream_t s);
// Forward transform along y of the fixed-point current (converted on load); zeroes
// `clear` (same shape, may be NULL) on the way, the buffer the next deposit sums into.
template <typename T>
cudaError_t launch_fft_y_from_fix(const longlong2* j, double unscale, void* out, int nx, int ny,
                                  const FftDesc& d, const void* tw, longlong2* clear,
                                  cudaStream_t s);
// Along x (stride ny).
template <typename T>
cudaError_t launch_fft_x(const void* in, void* out, int nx, int ny, int nb, const FftDesc& d,
                         const void* twiddle, int sign, cudaStream_t s);
// exp(-2 pi i m / n), m = 0..n-1, computed in FP64.
template <typename T>
cudaError_t launch_twiddles(void* tw, int n, cudaStream_t s);

// Per-mode kernels.
template <typename T>
cudaError_t launch_mode_init(const ModeCommon& mc, const void* zq, void* rho_out, void* phi_out,
                             void* e_packed, cudaStream_t s);
template <typename T>
cudaError_t launch_mode_bdf(const ModeCommon& mc, const BdfParams& bp, const void* z, void* f4,
                            void* e_packed, double* diag, cudaStream_t s);
template <typename T>
cudaError_t launch_mode_cdf2(const ModeCommon& mc, const CdfParams& cp, const void* z, void* f4,
                             void* e_packed, double* diag, cudaStream_t s);
template <typename T>
cudaError_t launch_mode_dirk(const ModeCommon& mc, const DirkParams& dp, const void* z, void* f4,
                             void* e_packed, double* diag, cudaStream_t s);
// Fused column pass of the field solve (forward transform along x, per-mode update,
// inverse transforms along x of the four outputs): one CTA per column, 8 lines of nx
// complex values in shared memory.  `kind` is a StepperKind.
inline size_t field_columns_smem(int nx, size_t complex_bytes) {
    return 9 * (size_t)nx * complex_bytes;  // two buffers of 4 lines, the twiddles
}
constexpr size_t kFieldColumnsSmemMax = 200 * 1024;
template <typename T>
cudaError_t launch_field_columns(const ModeCommon& mc, int kind, const BdfParams& bp,
                                 const CdfParams& cp, const DirkParams& dp, const void* z,
                                 void* f4, void* e, double* diag, const FftDesc& fd,
                                 const void* tw, cudaStream_t s);
// 2D-3V: the A_z wave update of the stepper in use (the same recurrences as A_x with the
// source mu0 J_z), from zz = FFT(J_z sums); writes the two packed outputs
// f2 = [(i kx - ky) A_z, A_z] / (nx ny) for the inverse transforms, and adds |E_z|^2 and
// |B_x|^2 + |B_y|^2 to the diagnostics when mc.diag.
struct ZParams {
    int kind, form;
    void* az[2 * kMaxBdf];   // BDF: history newest first; az_new: the slot of the new level
    void* az_new;
    void *az_n, *az_prev;    // CDF: A_z^n, A_z^{n-1} (the new level overwrites az_prev);
    void *jz_n, *jz_prev;    //      J_z^n, J_z^{n-1} (the new current overwrites jz_prev)
    void* vaz;               // DIRK: dA_z/dt; az_n and jz_n hold A_z^n and J_z^n
};
template <typename T>
cudaError_t launch_zfield(const ModeCommon& mc, const BdfParams& bp, const DirkParams& dp,
                          const ZParams& zp, const void* zz, void* f2, double* diag,
                          cudaStream_t s);
// Fill the wavenumber and inverse-denominator tables of mc (kind: StepperKind).
cudaError_t launch_mode_tables(const ModeCommon& mc, int kind, const BdfParams& bp,
                               const DirkParams& dp, double* kxt, double* kyt, double* invd,
                               double* dirkm, cudaStream_t s);
// Pack two spectra a + i b (scaled by inv_n) for an inverse transform to two real fields.
template <typename T>
cudaError_t launch_mode_pack2(const ModeCommon& mc, const void* a, const void* b, int op,
                              void* out, cudaStream_t s);

// Particle kernels.
struct ParticleGeom {
    int nx, ny;
    double lx, ly, inv_dx, inv_dy, dt;
};

// sp/spp (optional): each particle's species index and the table; the contributions are
// then multiplied by q_s w_s.
template <typename T>
cudaError_t launch_move_deposit(int p, const ParticleGeom& g, T* x, T* y, const T* vx,
                                const T* vy, int64_t n, double2* j, unsigned int* err,
                                cudaStream_t s, const int32_t* sp = nullptr,
                                const SpeciesParams* spp = nullptr);
template <typename T>
cudaError_t launch_deposit_charge(int p, const ParticleGeom& g, const T* x, const T* y, int64_t n,
                                  double2* j, unsigned int* err, cudaStream_t s,
                                  const int32_t* sp = nullptr, const SpeciesParams* spp = nullptr);
// Fixed-point current (int64 per component, contribution = round(value * scale)).
template <typename T>
cudaError_t launch_move_deposit_fix(int p, const ParticleGeom& g, T* x, T* y, const T* vx,
                                    const T* vy, int64_t n, longlong2* j, float scale,
                                    unsigned int* err, cudaStream_t s, const int32_t* sp = nullptr,
                                    const SpeciesParams* spp = nullptr);
template <typename T>
cudaError_t launch_deposit_charge_fix(int p, const ParticleGeom& g, const T* x, const T* y,
                                      int64_t n, longlong2* j, float scale, unsigned int* err,
                                      cudaStream_t s, const int32_t* sp = nullptr,
                                      const SpeciesParams* spp = nullptr);
// FP64 path, deterministic: contribution = round(value * scale) summed exactly as 128-bit
// integers; j holds 2 ng longlong2, the low words (x, y) of each node, then the high words.
cudaError_t launch_move_deposit_fix128(int p, const ParticleGeom& g, double* x, double* y,
                                       const double* vx, const double* vy, int64_t n,
                                       longlong2* j, size_t ng, double scale, unsigned int* err,
                                       cudaStream_t s, const int32_t* sp = nullptr,
                                       const SpeciesParams* spp = nullptr);
cudaError_t launch_deposit_charge_fix128(int p, const ParticleGeom& g, const double* x,
                                         const double* y, int64_t n, longlong2* j, size_t ng,
                                         double scale, unsigned int* err, cudaStream_t s,
                                         const int32_t* sp = nullptr,
                                         const SpeciesParams* spp = nullptr);
// out[k] = the 128-bit sums (x, y) of node k times unscale, as complex FP64.
cudaError_t launch_fix128_to_cplx(const longlong2* j, size_t ng, double unscale, double2* out,
                                  cudaStream_t s);
// 2D-3V: J_z of the moved particles (x^{n+1}, v_z^n) into the .x parts of jz: int64 sums
// (FP32 form, float `scale`) or 128-bit sums (FP64, layout of launch_move_deposit_fix128).
template <typename T>
cudaError_t launch_deposit_z(int p, const ParticleGeom& g, const T* x, const T* y, const T* vz,
                             int64_t n, const int32_t* sp, const SpeciesParams& spp, void* jz,
                             size_t ng, double scale, unsigned int* err, cudaStream_t s);
// out[k] = (J[k].x, J[k].y) * unscale in complex storage type T.
template <typename T>
cudaError_t launch_fix_to_cplx(const longlong2* j, double unscale, void* out, int64_t n,
                               cudaStream_t s);
cudaError_t launch_extract_fix(const longlong2* j, int comp, double scale, double* dst, int64_t n,
                               cudaStream_t s);
// dst[k] = component `comp` of the complex array src (element stride `stride` complex
// values) times `scale`, as FP64.
template <typename T>
cudaError_t launch_extract(const void* src, int stride, int comp, double scale, double* dst,
                           int64_t n, cudaStream_t s);

struct PushParams {
    double q, m, c, dt, weight;
    int diag;
};

// gout (FP64, may be NULL): the adjoint's record of the step, ten arrays of n: P^{n+1}
// (x, y), v^{n+1} (x, y), then the gathered Ax, Ay, dAx/dx, dAx/dy, dAy/dx, dAy/dy.
template <typename T>
cudaError_t launch_gather_push(int p, const ParticleGeom& g, const PushParams& pp, const T* x,
                               const T* y, T* px, T* py, const T* vx, const T* vy, T* vx_old,
                               T* vy_old, int64_t n, const void* fields4, double* gout,
                               double* diag, unsigned int* err, cudaStream_t s,
                               bool gout_short = false);
// Gather + push with a species table and/or three velocity components (vz == NULL: 2D-2V):
// fz holds the A_z fields as [node][2] complex ((dAz/dx, dAz/dy), (Az, 0)); P_z is constant.
template <typename T>
cudaError_t launch_gather_push3(int p, const ParticleGeom& g, const PushParams& pp, const T* x,
                                const T* y, T* px, T* py, const T* pz, const T* vx, const T* vy,
                                const T* vz, T* vx_old, T* vy_old, T* vz_old, const int32_t* sp,
                                const SpeciesParams& spp, int64_t n, const void* fields4,
                                const void* fz, double* diag, unsigned int* err, cudaStream_t s);
// t = 0 with a species table and/or three velocity components.
template <typename T>
cudaError_t launch_init_particles3(int p, const ParticleGeom& g, const PushParams& pp, T* x, T* y,
                                   T* px, T* py, T* pz, const T* vx, const T* vy, const T* vz,
                                   T* vx_old, T* vy_old, T* vz_old, const int32_t* sp,
                                   const SpeciesParams& spp, int64_t n, const void* e2,
                                   unsigned int* err, cudaStream_t s);
template <typename T>
cudaError_t launch_init_particles(int p, const ParticleGeom& g, const PushParams& pp, T* x, T* y,
                                  T* px, T* py, const T* vx, const T* vy, T* vx_old, T* vy_old,
                                  int64_t n, const void* e2, unsigned int* err, cudaStream_t s);
template <typename T>
cudaError_t launch_wrap_positions(T* x, T* y, int64_t n, double lx, double ly, cudaStream_t s);
template <typename Tsrc, typename Tdst>
cudaError_t launch_convert(const Tsrc* src, Tdst* dst, int64_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_scatter_by_id(const T* src, const int32_t* id, double* dst, int64_t n,
                                 cudaStream_t s);
// dst[id[k]] = src[k] for int32 values (the species indices of a sorted handle).
cudaError_t launch_scatter_by_id_i32(const int32_t* src, const int32_t* id, int32_t* dst,
                                     int64_t n, cudaStream_t s);

// Tiles for the particle sort and the shared-memory deposit: t x t cells per tile,
// ntx x nty tiles; a CTA accumulates into an rx x ry node region starting `halo` nodes
// before its tile's first node (wrapping periodically).
struct TileGeom {
    int nx, ny, t, ntx, nty, halo, rx, ry;
    int pitch;  // shared-memory row pitch of the region (>= ry, = t mod 32)
    double inv_dx, inv_dy;
    double dt, lx, ly;  // the sort keys a particle by its position after this step's move
    int half;  // 1 for even spline degree: the stencil base cell is floor(x/dx + 1/2)
    // sort key of a particle: tile-major, then the stencil base cell inside the tile,
    // key = tile * t * t + (bx mod t) * t + (by mod t); nkeys = ntx * nty * t * t
    __host__ __device__ int nkeys() const { return ntx * nty * t * t; }
};

// Particle arrays moved by the sort: x, y, Px, Py, v[0].x, v[0].y, v[1].x, v[1].y, and the
// particle's index at pic_init.
template <typename T>
struct SortArrays {
    T* a[8];
    int32_t* id;
    int32_t* sp = nullptr;                  // species indices (a species table), else NULL
    T* z[3] = {nullptr, nullptr, nullptr};  // 2D-3V: P_z, v_z (both buffers), else NULL
};

int sort_scan_chunks(int nkeys);  // chunk totals the scan keeps (size of its bsum array)
// vidx: index in src.a of the x velocity the keys' move uses (4 or 6; y velocity: vidx + 1),
// or -1: keys at the current positions (particles that have moved already).
template <typename T>
cudaError_t launch_tile_sort(const TileGeom& tg, SortArrays<T> src, SortArrays<T> dst, int64_t n,
                             int vidx, int* keys, int* hist, int* off, int* cursor, int* bsum,
                             cudaStream_t s);
cudaError_t launch_iota(int32_t* id, int64_t n, cudaStream_t s);

// Binned move + deposit of the FP32 form over tile-sorted particles (x, y, v^n = vx, vy)
// into the int64 current j (the moved positions go to xo, yo, which may be x, y): each CTA
// bins its particles by stencil base in shared memory and sums each base's contributions
// in registers before its shared atomics.  fused: the gather + push of the step before runs
// first on each particle (fields4 = that step's gather fields, P and v^{n+1} -> px, py,
// vxo, vyo; the move and deposit then use v^{n+1}), as launch_gather_push_tiled does it.
// per_cta: particles per CTA at the mean density.  deposit_binned_fits: whether the tile's
// regions fit the pass's shared memory.  sp/spp: a species table (each contribution times
// q_s w_s; the fused push with each species' charge and mass).  vz/jz (2D-3V, not fused):
// v_z^n of the particles and the int64 J_z sums (.x parts), deposited in the same pass.
bool deposit_binned_fits(const TileGeom& tg, int p, bool fused, bool z = false);
cudaError_t launch_deposit_binned(int p, const ParticleGeom& g, const PushParams& pp,
                                  const TileGeom& tg, const float* x, const float* y, float* xo,
                                  float* yo, float* px, float* py, const float* vx,
                                  const float* vy, float* vxo, float* vyo, int64_t n,
                                  const int* off, const void* fields4, void* j, float scale,
                                  double* diag, unsigned int* err, cudaStream_t s, bool fused,
                                  int per_cta, const int32_t* sp = nullptr,
                                  const SpeciesParams* spp = nullptr, const float* vz = nullptr,
                                  void* jz = nullptr);

// Gather + push of particles sorted by launch_tile_sort (FP32 form), fields staged per tile.
cudaError_t launch_gather_push_tiled(int p, const ParticleGeom& g, const PushParams& pp,
                                    const TileGeom& tg, const float* x, const float* y, float* px,
                                    float* py, const float* vx, const float* vy, float* vx_old,
                                    float* vy_old, int64_t n, const int* off,
                                    const void* fields4, double* diag, unsigned int* err,
                                    cudaStream_t s);

// ---------------------------------------------------------------- adjoint (FP64)
//
// Adjoints of the eight particle arrays of one state: x, y, Px, Py, v^n (vx, vy) and
// v^{n-1} (vxo, vyo).
template <typename T>
struct AdjParticlesT {
    T *x, *y, *px, *py, *vx, *vy, *vxo, *vyo;
};
using AdjParticles = AdjParticlesT<double>;
// Reverse BDF-k field step: the history adjoints, slot of level d (time n+1-d) for
// d = 0..2k-1 (rho: d = 0..k-1); level 0 is read first and rewritten with the new
// oldest level, which shares its slot.
struct AdjModeParams {
    int k;
    double a[kMaxBdf + 1];
    double C[2 * kMaxBdf + 1];
    double g, bdt;
    double2* phi[2 * kMaxBdf];
    double2* ax[2 * kMaxBdf];
    double2* ay[2 * kMaxBdf];
    double2* rho[kMaxBdf];
};
// The reverse particle kernels run in the forward's storage type T (double: the plain
// path; float: the FP32 form); the current adjoint they read (Jb) is FP64 in both, the
// field adjoints they add are FP64 (Fb) or, for T = float, FP32 sums (fb32).
//
// Reverse push + gather of one step: reads x^{n+1}, P^{n+1} (state n+1), v^n, v^{n-1}
// (state n), the step's record (gf: the gathered A and grad A at 4 n .. 10 n, FP64, see
// launch_gather_push; lean: the record stops at 4 n and they are gathered again from F)
// and the step's gather fields F ([node][4] complex of T); updates the particle adjoints
// and adds the eight field adjoints into Fb (four planes [k][node] of (f_2k, f_2k+1)).
template <typename T>
cudaError_t launch_adj_push_gather(int p, const ParticleGeom& g, const PushParams& pp,
                                   const T* x1, const T* y1, const T* px1, const T* py1,
                                   const T* vx, const T* vy, const T* vxo, const T* vyo,
                                   const double* gf, bool lean, const void* F,
                                   AdjParticlesT<T> ab, double2* Fb, void* fb32, int64_t n,
                                   unsigned int* err, cudaStream_t s);
// The FP32 form's field adjoints (fb32: [node][2] float4, fields 0-3 and 4-7, summed by
// launch_adj_push_gather<float>) to the four FP64 planes Fb of the reverse field solve.
cudaError_t launch_fb32_to_planes(const void* fb32, double2* Fb, int64_t ng, cudaStream_t s);
// Reverse field solve per mode of the stepper `kind` (a StepperKind: ap, cp or dp used,
// their pointers the history adjoints): Zb = forward transforms of the four Fb planes;
// writes the packed adjoint current spectrum Js (unnormalised inverse transform -> mesh).
// CDF-2 writes the adjoints before the step into the other buffer of each (cur, prev)
// pair, for the caller to swap; BDF and DIRK update in place.
cudaError_t launch_adj_modes(const ModeCommon& mc, int kind, const AdjModeParams& ap,
                             const CdfParams& cp, const DirkParams& dp, const double2* Zb,
                             double2* Js, cudaStream_t s);
// Fused column pass of the same (Zb transformed along y only; Js transformed back along x
// only), when adj_columns_smem(nx) fits kFieldColumnsSmemMax.
size_t adj_columns_smem(int nx);
cudaError_t launch_adj_columns(const ModeCommon& mc, int kind, const AdjModeParams& ap,
                               const CdfParams& cp, const DirkParams& dp, const double2* Zb,
                               double2* Js, const FftDesc& fd, const double2* tw,
                               cudaStream_t s);
// Reverse deposit + move: gathers the mesh current adjoint Jb ([node] (jx, jy)) at x^{n+1}.
template <typename T>
cudaError_t launch_adj_deposit_move(int p, const ParticleGeom& g, const T* x1, const T* y1,
                                    const T* vx, const T* vy, const double2* Jb,
                                    AdjParticlesT<T> ab, int64_t n, unsigned int* err,
                                    cudaStream_t s);
// Objective seed sum bzb B_z at the final level, from zs = DFT(bzb).
cudaError_t launch_adj_seed(const ModeCommon& mc, const double2* zs, double2* ax, double2* ay,
                            cudaStream_t s);
// (Ex + i Ey)/(nx ny) of E = -grad phi (for the mesh E^0 by an inverse transform).
cudaError_t launch_adj_e0(const ModeCommon& mc, const double2* phi, double2* out, cudaStream_t s);
// t = 0 reverse: gradients with respect to v^0 and P^0 (any output may be NULL).
template <typename T>
cudaError_t launch_adj_init(int p, const ParticleGeom& g, const PushParams& pp, const T* x0,
                            const T* y0, const T* vx0, const T* vy0, const double2* E,
                            AdjParticlesT<T> ab, double* gvx, double* gvy, double* gpx,
                            double* gpy, int64_t n, unsigned int* err, cudaStream_t s);
cudaError_t launch_real_to_cplx(const double* src, double2* dst, int64_t n, cudaStream_t s);
// Replay of one step's particle update from its record (FP64 values): state s0 -> state s1
// (eight arrays of n each, storage type T), bit for bit the step's own.
template <typename T>
cudaError_t launch_replay_step(const ParticleGeom& g, const T* s0, T* s1, const double* rec,
                               int64_t n, cudaStream_t s);
// Eight arrays of n values <-> one contiguous block of 8 n (array k at k n).
template <typename T>
struct Ptr8T {
    const T* p[8];
};
using Ptr8 = Ptr8T<double>;
template <typename T>
cudaError_t launch_pack8(Ptr8T<T> src, T* dst, int64_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_unpack8(const T* src, Ptr8T<T> dst, int64_t n, cudaStream_t s);

// Device error word bits.
enum ErrBits { ERR_NONFINITE = 1u, ERR_OVERFLOW = 2u, ERR_TIMEOUT = 4u };

}  // namespace gpic
