// pic_move_deposit_noalloc: one move-and-deposit pass that never allocates device memory.
//
// Some callers cannot let a library call cudaMalloc: hosts whose device memory is owned
// entirely by their own pool allocator (a framework's caching allocator that has already
// reserved the GPU, where a hidden cudaMalloc either fails or escapes the pool's
// accounting), and latency-critical loops in which the implicit device-wide
// synchronisation of cudaMalloc/cudaFree is not acceptable.  This entry point serves
// them: its only scratch -- the (Jx, Jy) accumulation grid that the regular path keeps in
// the simulation handle -- is a fixed-size array in this file, resident on every device
// that loads the library until the process exits.
//
// Host code must not hand the array's name to a kernel (in host code that name is only a
// stand-in for the device symbol); the device address comes from cudaGetSymbolAddress,
// taken once per device with that device current, on the first call made on it.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "gpic_internal.h"
#include "pic.h"

using namespace gpic;

// Largest grid the fixed scratch holds: nx * ny <= 262,144 nodes (a 512 x 512 grid).
constexpr int kMaxNoallocNodes = 512 * 512;

// The accumulation grid (16 bytes per node, 4 MiB), followed by 256 bytes whose first
// word is the pass's error flag.
static __device__ __align__(256) double2 g_noalloc_scratch[kMaxNoallocNodes + 16];

namespace {

constexpr int kMaxDevices = 64;

struct DeviceScratch {
    double2* j = nullptr;
    unsigned int* err = nullptr;
    bool ready = false;
};
DeviceScratch g_scratch[kMaxDevices];
std::mutex g_scratch_mutex;

// Failures are reported by status code only (the message documents the reason).
pic_status noalloc_fail(pic_status st, const char* /*reason*/) { return st; }

// Device addresses of the static scratch on the current device (set-up on first use).
pic_status scratch_for_current_device(DeviceScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(PIC_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(PIC_ERR_UNSUPPORTED, "device ordinal >= 64");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    DeviceScratch& s = g_scratch[dev];
    if (!s.ready) {
        void* base = nullptr;
        e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
        if (e != cudaSuccess) return noalloc_fail(PIC_ERR_CUDA, cudaGetErrorString(e));
        s.j = static_cast<double2*>(base);
        s.err = reinterpret_cast<unsigned int*>(s.j + kMaxNoallocNodes);
        s.ready = true;
    }
    *out = &s;
    return PIC_OK;
}

// J = jscale * (accumulated sum of v W), split into the caller's two real grids.
__global__ void k_noalloc_finish(const double2* __restrict__ acc, double jscale,
                                 double* __restrict__ jx, double* __restrict__ jy, int nodes) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nodes; k += gridDim.x * blockDim.x) {
        const double2 a = acc[k];
        jx[k] = jscale * a.x;
        jy[k] = jscale * a.y;
    }
}

bool pos_finite(double v) { return std::isfinite(v) && v > 0.0; }

}  // namespace

extern "C" pic_status pic_move_deposit_noalloc(const pic_config* cfg, int64_t n, double* x,
                                               double* y, const double* vx, const double* vy,
                                               double* jx, double* jy, void* cuda_stream) {
    if (!cfg) return noalloc_fail(PIC_ERR_INVALID_ARG, "cfg must not be NULL");
    if (cfg->precision != PIC_FP64)
        return noalloc_fail(PIC_ERR_UNSUPPORTED, "only the FP64 path has an allocation-free pass");
    if (cfg->nx < 8 || cfg->ny < 8)
        return noalloc_fail(PIC_ERR_INVALID_ARG, "nx and ny must be >= 8");
    if ((int64_t)cfg->nx * cfg->ny > kMaxNoallocNodes)
        return noalloc_fail(PIC_ERR_INVALID_ARG,
                            "grid too large: nx*ny must be <= 262144 (the fixed scratch holds a "
                            "512x512 grid)");
    if (cfg->spline_order < 2 || cfg->spline_order > 4)
        return noalloc_fail(PIC_ERR_INVALID_ARG, "spline_order must be 2, 3 or 4");
    if (!pos_finite(cfg->lx) || !pos_finite(cfg->ly) || !pos_finite(cfg->dt) ||
        !pos_finite(cfg->c) || !std::isfinite(cfg->q) || !std::isfinite(cfg->weight))
        return noalloc_fail(PIC_ERR_INVALID_ARG, "lx, ly, dt, c must be finite and > 0");
    if (cfg->c * cfg->dt >= std::fmin(cfg->lx, cfg->ly))
        return noalloc_fail(PIC_ERR_INVALID_ARG, "c*dt must be below the domain size");
    if (n < 0 || n > 2147483647LL) return noalloc_fail(PIC_ERR_INVALID_ARG, "n must be 0..2^31-1");
    if (!jx || !jy || (n > 0 && (!x || !y || !vx || !vy)))
        return noalloc_fail(PIC_ERR_INVALID_ARG, "array pointers must not be NULL");

    DeviceScratch* s = nullptr;
    pic_status st = scratch_for_current_device(&s);
    if (st != PIC_OK) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const int nodes = cfg->nx * cfg->ny;
    const double dx = cfg->lx / cfg->nx, dy = cfg->ly / cfg->ny;
    const ParticleGeom g{cfg->nx, cfg->ny, cfg->lx, cfg->ly, 1.0 / dx, 1.0 / dy, cfg->dt};

    // The scratch keeps the previous call's contents: clear what must start at zero.
    cudaError_t e = cudaMemsetAsync(s->j, 0, (size_t)nodes * sizeof(double2), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->err, 0, sizeof(unsigned int), stream);
    if (e == cudaSuccess)
        e = launch_move_deposit<double>(cfg->spline_order, g, x, y, vx, vy, n, s->j, s->err, stream);
    if (e == cudaSuccess) {
        k_noalloc_finish<<<(nodes + 255) / 256, 256, 0, stream>>>(s->j, cfg->weight * cfg->q / (dx * dy),
                                                                 jx, jy, nodes);
        e = cudaGetLastError();
    }
    unsigned int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, s->err, sizeof flag, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return noalloc_fail(PIC_ERR_CUDA, cudaGetErrorString(e));
    if (flag & ERR_NONFINITE)
        return noalloc_fail(PIC_ERR_NONFINITE, "a particle position left the domain or is not finite");
    return PIC_OK;
}
