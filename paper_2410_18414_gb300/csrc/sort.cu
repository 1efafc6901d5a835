// Counting sort of the particles by tile and cell (every sort_interval steps).
//
// The domain is cut into tiles of T x T cells; a particle's key is its stencil base
// cell, numbered tile by tile, so the particles of one tile are contiguous and, inside
// it, those of one cell are.  Three or four kernels: the keys with their histogram, an
// exclusive scan giving each key's first slot (one CTA for up to 16384 keys, else two
// passes), and a scatter that moves all particle
// arrays (and the particle's original index) to the slots of its key.  The order inside
// a cell is not fixed; nothing depends on it: the FP32 form sums the current in integers,
// the push is per particle, and read-back restores the caller's order through the index
// array.  Sorting keeps the particles of one CTA inside one tile, so
// the deposit can accumulate in shared memory and the gather reuses cached field tiles.
#include "common.cuh"
#include "gpic_internal.h"
#include "launch.cuh"

namespace gpic {

namespace {

constexpr int kThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kScanChunk = 4 * kScanThreads;  // keys per CTA of the scan
constexpr int kKeysPer = 4;                   // particles per thread in the keys
constexpr int kScanSinglePer = 16;            // keys per thread of the one-CTA scan
// particles per thread in the scatter (their payload is held in registers)
template <typename T>
constexpr int scatter_per() { return sizeof(T) == 4 ? 4 : 2; }

inline int blocks_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b > 152 * 8) b = 152 * 8;
    return (int)(b < 1 ? 1 : b);
}

// Stencil base cell of a position (floor(x/dx) for odd spline degree, floor(x/dx + 1/2)
// for even degree: particles with equal base cells share all their stencil nodes),
// wrapped into the grid, then the tile-major key of that cell.
template <typename T>
__device__ __forceinline__ int tile_key(T x, T y, const TileGeom& tg) {
    const T h = tg.half ? (T)0.5 : (T)0;
    int bx = (int)floor(radd(rmul(x, (T)tg.inv_dx), h));  // in the storage precision: FP32
    int by = (int)floor(radd(rmul(y, (T)tg.inv_dy), h));  // keys stay off the FP64 pipe
    bx = bx < 0 ? 0 : (bx >= tg.nx ? bx - tg.nx : bx);
    by = by < 0 ? 0 : (by >= tg.ny ? by - tg.ny : by);
    bx = bx >= tg.nx ? tg.nx - 1 : bx;
    by = by >= tg.ny ? tg.ny - 1 : by;
    const int tx = bx / tg.t, ty = by / tg.t;
    return ((tx * tg.nty + ty) * tg.t + (bx - tx * tg.t)) * tg.t + (by - ty * tg.t);
}

// Keys and their histogram.  Particles arrive in the order of the previous sort, so the
// lanes of a warp mostly share a key: one lane adds the group's count (no return value).
// A thread takes kKeysPer particles kThreads apart and issues all their loads first.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_sort_keys(TileGeom tg, const T* __restrict__ x, const T* __restrict__ y,
            const T* __restrict__ vx, const T* __restrict__ vy, int64_t n,
            int* __restrict__ keys, int* __restrict__ hist) {
    griddep_wait();
    griddep_launch();
    const T dt = (T)tg.dt, lx = (T)tg.lx, ly = (T)tg.ly;
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * kKeysPer + threadIdx.x;
    T xs[kKeysPer], ys[kKeysPer], us[kKeysPer], ws[kKeysPer];
#pragma unroll
    for (int i = 0; i < kKeysPer; ++i) {
        const int64_t p = base + (int64_t)i * blockDim.x;
        xs[i] = ys[i] = us[i] = ws[i] = (T)0;
        if (p < n) {
            xs[i] = x[p];
            ys[i] = y[p];
            if (vx) {
                us[i] = vx[p];
                ws[i] = vy[p];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < kKeysPer; ++i) {  // warp-uniform: every lane reaches the match
        const int64_t p = base + (int64_t)i * blockDim.x;
        int k = -1;
        if (p < n) {
            // the cell the particle will deposit from after this step's move (vx NULL: the
            // particle has moved already), so that the deposit right after a sort sees no
            // drift from the sorted cells
            k = vx ? tile_key(move_pos(xs[i], us[i], dt, lx), move_pos(ys[i], ws[i], dt, ly), tg)
                   : tile_key(xs[i], ys[i], tg);
            keys[p] = k;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, k);
        if (k >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(hist + k, __popc(peers));
    }
}

// Exclusive scan of the thread sums of a CTA (blockDim.x = kScanThreads); returns the
// thread's exclusive prefix and sets *total.
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_sums, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = warp_sums[lane];
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        warp_sums[lane] = wi - w;  // exclusive prefix of the warp totals
        if (lane == 31) warp_sums[32] = wi;
    }
    __syncthreads();
    *total = warp_sums[32];
    return warp_sums[warp] + inc - v;
}

// Scan, pass 1: CTA b scans keys [b C, (b+1) C) locally (C = kScanChunk) into off and
// stores the chunk total in bsum[b].  It leaves the histogram zeroed for the next sort.
__global__ void __launch_bounds__(kScanThreads)
k_scan_local(int* __restrict__ hist, int nkeys, int* __restrict__ off, int* __restrict__ bsum) {
    __shared__ int warp_sums[33];
    const int i0 = blockIdx.x * kScanChunk + 4 * threadIdx.x;
    griddep_wait();
    griddep_launch();
    int v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        v[j] = 0;
        if (i0 + j < nkeys) {
            v[j] = hist[i0 + j];
            hist[i0 + j] = 0;
        }
    }
    int total;
    int run = block_exclusive_scan(v[0] + v[1] + v[2] + v[3], warp_sums, &total);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (i0 + j < nkeys) off[i0 + j] = run;
        run += v[j];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// Scan, pass 2: adds the totals of the earlier chunks; cursor = off; off[nkeys] = n.
__global__ void __launch_bounds__(kScanThreads)
k_scan_add(int nkeys, int nchunks, const int* __restrict__ bsum, int* __restrict__ off,
           int* __restrict__ cursor) {
    __shared__ int warp_sums[33];
    griddep_wait();
    griddep_launch();
    int s = 0;
    for (int c = threadIdx.x; c < blockIdx.x; c += blockDim.x) s += bsum[c];
    int total;
    block_exclusive_scan(s, warp_sums, &total);  // total = sum of bsum[0 .. blockIdx.x)
    const int base = total;
    const int i0 = blockIdx.x * kScanChunk;
    for (int i = i0 + threadIdx.x; i < i0 + kScanChunk && i < nkeys; i += blockDim.x) {
        const int o = off[i] + base;
        off[i] = o;
        cursor[i] = o;
    }
    if (blockIdx.x == nchunks - 1 && threadIdx.x == 0) off[nkeys] = base + bsum[nchunks - 1];
}

// Scatter: every particle claims a slot of its key (warp-aggregated atomics on the key
// cursors).  A thread handles PER particles: it loads their keys and particle values
// first, so the loads are in flight while the claims go out and come back, then stores
// the particle arrays and the original index at the claimed slots.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_sort_scatter(SortArrays<T> src, SortArrays<T> dst, const int* __restrict__ keys, int64_t n,
               int* __restrict__ cursor) {
    constexpr int PER = scatter_per<T>();
    const int lane = threadIdx.x & 31;
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * PER + threadIdx.x;
    griddep_wait();
    griddep_launch();
    int k[PER], slot[PER], leader[PER];
    unsigned peers[PER];
    T v[PER][8];
    int32_t id[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int64_t p = base + (int64_t)i * blockDim.x;
        k[i] = p < n ? keys[p] : -1;
        id[i] = 0;
#pragma unroll
        for (int a = 0; a < 8; ++a) v[i][a] = (T)0;
        if (p < n) {
#pragma unroll
            for (int a = 0; a < 8; ++a) v[i][a] = src.a[a][p];
            id[i] = src.id[p];
        }
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        peers[i] = __match_any_sync(0xffffffffu, k[i]);
        leader[i] = __ffs(peers[i]) - 1;
        slot[i] = 0;
        if (lane == leader[i] && k[i] >= 0) slot[i] = atomicAdd(cursor + k[i], __popc(peers[i]));
    }
#pragma unroll
    for (int i = 0; i < PER; ++i)
        slot[i] = __shfl_sync(0xffffffffu, slot[i], leader[i]) +
                  __popc(peers[i] & ((1u << lane) - 1u));
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int64_t p = base + (int64_t)i * blockDim.x;
        if (k[i] >= 0) {
            const int q = slot[i];
#pragma unroll
            for (int a = 0; a < 8; ++a) dst.a[a][q] = v[i][a];
            dst.id[q] = id[i];
            if (src.sp) dst.sp[q] = src.sp[p];
            if (src.z[0]) {
#pragma unroll
                for (int a = 0; a < 3; ++a) dst.z[a][q] = src.z[a][p];
            }
        }
    }
}

// Scan of a histogram of at most kScanThreads * kScanSinglePer keys in one CTA: the
// exclusive offsets into off and cursor, off[nkeys] = the total; the histogram is left
// zeroed for the next sort.  (Larger key counts take k_scan_local + k_scan_add.)  Warp w
// owns the contiguous block [w B, (w + 1) B) of keys, B = 32 per; its lanes read, clear
// and write the block 32 consecutive keys at a time (coalesced), scanning each group of
// 32 with shuffles and carrying the running total from group to group.
__global__ void __launch_bounds__(kScanThreads)
k_scan_single(int* __restrict__ hist, int nkeys, int* __restrict__ off,
              int* __restrict__ cursor) {
    __shared__ int warp_sums[33];
    griddep_wait();
    griddep_launch();
    constexpr int kWarps = kScanThreads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = (nkeys + kWarps * 32 - 1) / (kWarps * 32);  // groups a warp, <= 16
    const int w0 = warp * per * 32;
    int v[kScanSinglePer];
#pragma unroll
    for (int j = 0; j < kScanSinglePer; ++j) {
        const int i = w0 + j * 32 + lane;
        v[j] = 0;
        if (j < per && i < nkeys) {
            v[j] = hist[i];
            hist[i] = 0;
        }
    }
    int carry = 0;  // the warp's keys before the current group
#pragma unroll
    for (int j = 0; j < kScanSinglePer; ++j) {
        int inc = v[j];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        const int excl = carry + inc - v[j];
        carry += __shfl_sync(0xffffffffu, inc, 31);
        v[j] = excl;  // from here on: the exclusive prefix inside the warp's block
    }
    if (lane == 0) warp_sums[warp] = carry;
    __syncthreads();
    if (warp == 0) {
        const int t = warp_sums[lane];
        int inc = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        warp_sums[lane] = inc - t;
        if (lane == 31) warp_sums[32] = inc;
    }
    __syncthreads();
    const int wbase = warp_sums[warp];
#pragma unroll
    for (int j = 0; j < kScanSinglePer; ++j) {
        const int i = w0 + j * 32 + lane;
        if (j < per && i < nkeys) {
            off[i] = wbase + v[j];
            cursor[i] = wbase + v[j];
        }
    }
    if (threadIdx.x == 0) off[nkeys] = warp_sums[32];
}

__global__ void k_iota(int32_t* __restrict__ id, int64_t n) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        id[p] = (int32_t)p;
}

}  // namespace

int sort_scan_chunks(int nkeys) { return (nkeys + kScanChunk - 1) / kScanChunk; }

template <typename T>
cudaError_t launch_tile_sort(const TileGeom& tg, SortArrays<T> src, SortArrays<T> dst, int64_t n,
                             int vidx, int* keys, int* hist, int* off, int* cursor, int* bsum,
                             cudaStream_t s) {
    if (vidx != 4 && vidx != 6 && vidx != -1) return cudaErrorInvalidValue;
    // hist is all zero on entry: zeroed once at allocation, then by every scan
    const int nkeys = tg.nkeys();  // number of sort keys (cells, tile-major)
    if (n == 0) return cudaMemsetAsync(off, 0, sizeof(int) * (nkeys + 1), s);
    const int64_t keys_cta = (int64_t)kThreads * kKeysPer;
    cudaError_t e = launch_pdl(k_sort_keys<T>, dim3((unsigned)((n + keys_cta - 1) / keys_cta)),
                   dim3(kThreads), 0, s, tg, (const T*)src.a[0], (const T*)src.a[1],
                   vidx < 0 ? nullptr : (const T*)src.a[vidx],
                   vidx < 0 ? nullptr : (const T*)src.a[vidx + 1], n, keys, hist);
    const int nchunks = sort_scan_chunks(nkeys);
    if (nkeys <= kScanThreads * kScanSinglePer) {  // one CTA (the 128 x 128 grid: 16 keys each)
        if (e == cudaSuccess)
            e = launch_pdl(k_scan_single, dim3(1), dim3(kScanThreads), 0, s, hist, nkeys, off,
                           cursor);
    } else {
        if (e == cudaSuccess)
            e = launch_pdl(k_scan_local, dim3(nchunks), dim3(kScanThreads), 0, s, hist, nkeys,
                           off, bsum);
        if (e == cudaSuccess)
            e = launch_pdl(k_scan_add, dim3(nchunks), dim3(kScanThreads), 0, s, nkeys, nchunks,
                           (const int*)bsum, off, cursor);
    }
    const int64_t per_cta = (int64_t)kThreads * scatter_per<T>();
    if (e == cudaSuccess)
        e = launch_pdl(k_sort_scatter<T>, dim3((unsigned)((n + per_cta - 1) / per_cta)),
                       dim3(kThreads), 0, s, src, dst, (const int*)keys, n, cursor);
    return e;
}

cudaError_t launch_iota(int32_t* id, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_iota<<<blocks_for(n), kThreads, 0, s>>>(id, n);
    return cudaGetLastError();
}

template cudaError_t launch_tile_sort<float>(const TileGeom&, SortArrays<float>, SortArrays<float>,
                                             int64_t, int, int*, int*, int*, int*, int*,
                                             cudaStream_t);
template cudaError_t launch_tile_sort<double>(const TileGeom&, SortArrays<double>,
                                              SortArrays<double>, int64_t, int, int*, int*, int*,
                                              int*, int*, cudaStream_t);

}  // namespace gpic
