// Counting sort of the particles by tile and cell (every sort_interval steps).
//
// The domain is cut into tiles of T x T cells; a particle's key is its stencil base
// cell, numbered tile by tile, so the particles of one tile are contiguous and, inside
// it, those of one cell are.  Three kernels: a histogram of keys (shared-memory privatised), one
// single-CTA exclusive scan giving each tile's first slot, and a scatter that moves all
// particle arrays (and the particle's original index) to the slots of its tile.  The
// scatter order inside a tile is not fixed; nothing depends on it: the FP32 form sums the
// current in int64, the push is per particle, and read-back restores the caller's order
// through the index array.  Sorting keeps the particles of one CTA inside one tile, so
// the deposit can accumulate in shared memory and the gather reuses cached field tiles.
#include "common.cuh"
#include "gpic_internal.h"

namespace gpic {

namespace {

constexpr int kThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kSmemHistMax = 12 * 1024;  // tiles held in a shared-memory histogram

inline int blocks_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b > 152 * 8) b = 152 * 8;
    return (int)(b < 1 ? 1 : b);
}

// Lanes of the calling warp holding the same key: one of them adds the group's count
// to *counter; every lane returns its slot (old value + rank inside the group).  All 32
// lanes must call it (invalid lanes pass key = -1 and get -1 back).
__device__ __forceinline__ int warp_aggregated_claim(int* counter_base, int key) {
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    int start = 0;
    if (lane == leader && key >= 0) start = atomicAdd(counter_base + key, __popc(peers));
    start = __shfl_sync(0xffffffffu, start, leader);
    return key >= 0 ? start + rank : -1;
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

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_tile_hist(TileGeom tg, const T* __restrict__ x, const T* __restrict__ y, int64_t n,
            int* __restrict__ keys, int* __restrict__ hist) {
    extern __shared__ int sh[];
    const int ntiles = tg.nkeys();
    const bool priv = ntiles <= kSmemHistMax;
    if (priv) {
        for (int i = threadIdx.x; i < ntiles; i += blockDim.x) sh[i] = 0;
        __syncthreads();
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < n; b += stride) {  // warp-uniform
        const int64_t p = b + threadIdx.x;
        int k = -1;
        if (p < n) {
            k = tile_key(x[p], y[p], tg);
            keys[p] = k;
        }
        warp_aggregated_claim(priv ? sh : hist, k);
    }
    if (priv) {
        __syncthreads();
        for (int i = threadIdx.x; i < ntiles; i += blockDim.x)
            if (sh[i]) atomicAdd(&hist[i], sh[i]);
    }
}

// Exclusive scan of hist[0..ntiles) into off[0..ntiles] (off[ntiles] = n); cursor = off.
__global__ void __launch_bounds__(kScanThreads)
k_tile_scan(const int* __restrict__ hist, int ntiles, int* __restrict__ off,
            int* __restrict__ cursor) {
    __shared__ int part[kScanThreads];
    const int per = (ntiles + kScanThreads - 1) / kScanThreads;
    const int b = threadIdx.x * per;
    int s = 0;
    for (int i = 0; i < per && b + i < ntiles; ++i) s += hist[b + i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {  // Hillis-Steele inclusive scan
        int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = part[threadIdx.x] - s;  // exclusive prefix of this thread's block
    for (int i = 0; i < per && b + i < ntiles; ++i) {
        off[b + i] = run;
        cursor[b + i] = run;
        run += hist[b + i];
    }
    if (threadIdx.x == kScanThreads - 1) off[ntiles] = part[kScanThreads - 1];
}

// Scatter with per-CTA slot reservation: CTA b counts its chunk's particles per tile in
// shared memory, reserves each tile's slots with one global atomic, then hands out slots
// from the reservation with shared-memory atomics.  (One global atomic per particle on a
// few dozen tile cursors serialises badly.)
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_tile_scatter(SortArrays<T> src, SortArrays<T> dst, const int* __restrict__ keys, int64_t n,
               int ntiles, int chunk, int* __restrict__ cursor, int* __restrict__ keys_out) {
    extern __shared__ int base[];
    const int64_t c0 = (int64_t)blockIdx.x * chunk;
    if (c0 >= n) return;
    const int64_t c1 = c0 + chunk < n ? c0 + chunk : n;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) base[t] = 0;
    __syncthreads();
    for (int64_t b = c0; b < c1; b += blockDim.x) {  // warp-uniform trip count
        const int64_t p = b + threadIdx.x;
        warp_aggregated_claim(base, p < c1 ? keys[p] : -1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        const int c = base[t];
        base[t] = c ? atomicAdd(&cursor[t], c) : 0;
    }
    __syncthreads();
    for (int64_t b = c0; b < c1; b += blockDim.x) {
        const int64_t p = b + threadIdx.x;
        const int k = p < c1 ? keys[p] : -1;
        const int q = warp_aggregated_claim(base, k);
        if (k >= 0) {
#pragma unroll
            for (int a = 0; a < 8; ++a) dst.a[a][q] = src.a[a][p];
            dst.id[q] = src.id[p];
            keys_out[q] = k;
        }
    }
}

// Fallback for more tiles than fit a shared-memory table: one global atomic per particle.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_tile_scatter_global(SortArrays<T> src, SortArrays<T> dst, const int* __restrict__ keys,
                      int64_t n, int* __restrict__ cursor, int* __restrict__ keys_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < n; b += stride) {
        const int64_t p = b + threadIdx.x;
        const int k = p < n ? keys[p] : -1;
        const int q = warp_aggregated_claim(cursor, k);
        if (k >= 0) {
#pragma unroll
            for (int a = 0; a < 8; ++a) dst.a[a][q] = src.a[a][p];
            dst.id[q] = src.id[p];
            keys_out[q] = k;
        }
    }
}

__global__ void k_iota(int32_t* __restrict__ id, int64_t n) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        id[p] = (int32_t)p;
}

}  // namespace

template <typename T>
cudaError_t launch_tile_sort(const TileGeom& tg, SortArrays<T> src, SortArrays<T> dst, int64_t n,
                             int* keys, int* keys_out, int* hist, int* off, int* cursor,
                             cudaStream_t s) {
    const int ntiles = tg.nkeys();  // number of sort keys (cells, tile-major)
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int) * ntiles, s);
    if (e != cudaSuccess || n == 0) {
        if (e == cudaSuccess) e = cudaMemsetAsync(off, 0, sizeof(int) * (ntiles + 1), s);
        return e;
    }
    const size_t sh = ntiles <= kSmemHistMax ? sizeof(int) * ntiles : 0;
    if (sh > 48 * 1024) {
        e = cudaFuncSetAttribute(k_tile_hist<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        if (e != cudaSuccess) return e;
    }
    k_tile_hist<T><<<blocks_for(n), kThreads, sh, s>>>(tg, src.a[0], src.a[1], n, keys, hist);
    k_tile_scan<<<1, kScanThreads, 0, s>>>(hist, ntiles, off, cursor);
    if (ntiles <= kSmemHistMax) {
        const int chunk = 1024;
        const int blocks = (int)((n + chunk - 1) / chunk);
        if (sh > 48 * 1024) {
            e = cudaFuncSetAttribute(k_tile_scatter<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sh);
            if (e != cudaSuccess) return e;
        }
        k_tile_scatter<T><<<blocks, kThreads, sh, s>>>(src, dst, keys, n, ntiles, chunk, cursor,
                                                       keys_out);
    } else {
        k_tile_scatter_global<T><<<blocks_for(n), kThreads, 0, s>>>(src, dst, keys, n, cursor,
                                                                    keys_out);
    }
    return cudaGetLastError();
}

cudaError_t launch_iota(int32_t* id, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_iota<<<blocks_for(n), kThreads, 0, s>>>(id, n);
    return cudaGetLastError();
}

template cudaError_t launch_tile_sort<float>(const TileGeom&, SortArrays<float>, SortArrays<float>,
                                             int64_t, int*, int*, int*, int*, int*, cudaStream_t);
template cudaError_t launch_tile_sort<double>(const TileGeom&, SortArrays<double>,
                                              SortArrays<double>, int64_t, int*, int*, int*, int*,
                                              int*, cudaStream_t);

}  // namespace gpic
