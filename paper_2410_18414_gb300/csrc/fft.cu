// Shared-memory mixed-radix (4, 2, 3) Stockham FFT for the spectral field solve.
//
// The paper inverts the modified Helmholtz operator and takes every spatial
// derivative with the FFT on the periodic grid (sections 3.1 and 4).  Grids here
// are at most a few thousand points per side, so each CTA loads whole lines into
// shared memory, runs all radix passes there (ping-pong buffers, autosort
// Stockham ordering: no bit reversal) and writes the lines back once.
//
// Pass with radix R on lines of length n, Ns = product of the earlier radices:
//   for j in [0, n/R):  k = j mod Ns
//     a_r = src[j + r n/R] * w^(r k n/(Ns R)),  r = 0..R-1   (w = exp(sign 2 pi i / n))
//     b   = R-point DFT of a
//     dst[(j div Ns) Ns R + k + r Ns] = b_r
// which leaves the transform in natural order after the last pass.
#include "common.cuh"
#include "fft_device.cuh"
#include "gpic_internal.h"
#include "launch.cuh"

namespace gpic {

namespace {

constexpr int kThreads = 256;

// Transforms along y (contiguous): CTA = `rows` consecutive x-indices of all nb arrays.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_fft_y(const cplx_t<T>* __restrict__ in, cplx_t<T>* __restrict__ out, int nx, int ny, int nb,
        int rows, FftDesc d, const cplx_t<T>* __restrict__ tw, int sign, int interleave,
        const longlong2* __restrict__ fix_in, double unscale, longlong2* __restrict__ clear) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* b0 = reinterpret_cast<C*>(smem_raw);
    const int lines = nb * rows;
    C* b1 = b0 + lines * ny;
    C* tws = b1 + lines * ny;  // twiddles, staged before the wait (they are constant)
    stage_twiddles(tw, tws, ny);
    const int i0 = blockIdx.x * rows;
    const size_t plane = (size_t)nx * ny;
    griddep_wait();  // the input is the previous kernel's output
    griddep_launch();
    for (int e = threadIdx.x; e < lines * ny; e += blockDim.x) {
        int l = e / ny, jj = e - l * ny;
        int b = l / rows, r = l - b * rows;
        const size_t src = b * plane + (size_t)(i0 + r) * ny + jj;
        if (fix_in) {  // fixed-point current sums, converted on load
            const longlong2 v = fix_in[src];
            if (clear) clear[src] = longlong2{0, 0};  // the other buffer, for the next deposit
            b0[e] = mk<C>((double)v.x * unscale, (double)v.y * unscale);
        } else {
            b0[e] = in[src];
        }
    }
    __syncthreads();
    C* res = run_passes(b0, b1, d, lines, (const C*)tws, sign);
    if (interleave) {
        for (int e = threadIdx.x; e < lines * ny; e += blockDim.x) {
            int b = e % nb, t = e / nb;
            int jj = t % ny, r = t / ny;
            out[((size_t)(i0 + r) * ny + jj) * nb + b] = res[(b * rows + r) * ny + jj];
        }
    } else {
        for (int e = threadIdx.x; e < lines * ny; e += blockDim.x) {
            int l = e / ny, jj = e - l * ny;
            int b = l / rows, r = l - b * rows;
            out[b * plane + (size_t)(i0 + r) * ny + jj] = res[e];
        }
    }
}

// Transforms along x (stride ny): CTA = `cols` consecutive y-indices of one array.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_fft_x(const cplx_t<T>* __restrict__ in, cplx_t<T>* __restrict__ out, int nx, int ny, int cols,
        FftDesc d, const cplx_t<T>* __restrict__ tw, int sign) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* b0 = reinterpret_cast<C*>(smem_raw);
    C* b1 = b0 + cols * nx;
    const int j0 = blockIdx.x * cols;
    const size_t off = (size_t)blockIdx.y * nx * ny;
    for (int t = threadIdx.x; t < nx * cols; t += blockDim.x) {
        int e = t / cols, c = t - e * cols;
        b0[c * nx + e] = in[off + (size_t)e * ny + j0 + c];
    }
    __syncthreads();
    C* res = run_passes(b0, b1, d, cols, tw, sign);
    for (int t = threadIdx.x; t < nx * cols; t += blockDim.x) {
        int e = t / cols, c = t - e * cols;
        out[off + (size_t)e * ny + j0 + c] = res[c * nx + e];
    }
}

template <typename T>
__global__ void k_twiddles(cplx_t<T>* tw, int n) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < n) {
        double s, c;
        sincospi(2.0 * (double)m / (double)n, &s, &c);
        tw[m] = mk<cplx_t<T>>(c, -s);
    }
}

constexpr size_t kSmemBudget = 96 * 1024;

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

template <typename T>
static cudaError_t fft_y_impl(const void* in, void* out, int nx, int ny, int nb, const FftDesc& d,
                              const void* tw, int sign, int interleave, const longlong2* fix_in,
                              double unscale, longlong2* clear, cudaStream_t s) {
    using C = cplx_t<T>;
    const size_t per_line = 2 * (size_t)ny * sizeof(C);
    const size_t tw_bytes = (size_t)ny * sizeof(C);
    // few lines per CTA: these transforms are latency-bound, so favour CTAs (one row of
    // all nb arrays each, or two rows when there is a single array)
    int rows = nb == 1 && nx % 2 == 0 ? 2 : 1;
    if ((size_t)rows * nb * per_line + tw_bytes > 200 * 1024) rows = 1;
    if ((size_t)rows * nb * per_line + tw_bytes > 200 * 1024) return cudaErrorInvalidValue;
    size_t smem = (size_t)rows * nb * per_line + tw_bytes;
    cudaError_t e = set_smem(k_fft_y<T>, smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_fft_y<T>, dim3(nx / rows), dim3(kThreads), smem, s, (const C*)in, (C*)out,
                      nx, ny, nb, rows, d, (const C*)tw, sign, interleave, fix_in, unscale, clear);
}

template <typename T>
cudaError_t launch_fft_y(const void* in, void* out, int nx, int ny, int nb, const FftDesc& d,
                         const void* tw, int sign, int interleave, cudaStream_t s) {
    return fft_y_impl<T>(in, out, nx, ny, nb, d, tw, sign, interleave, nullptr, 0.0, nullptr, s);
}

template <typename T>
cudaError_t launch_fft_y_from_fix(const longlong2* j, double unscale, void* out, int nx, int ny,
                                  const FftDesc& d, const void* tw, longlong2* clear,
                                  cudaStream_t s) {
    return fft_y_impl<T>(nullptr, out, nx, ny, 1, d, tw, -1, 0, j, unscale, clear, s);
}

template <typename T>
cudaError_t launch_fft_x(const void* in, void* out, int nx, int ny, int nb, const FftDesc& d,
                         const void* tw, int sign, cudaStream_t s) {
    using C = cplx_t<T>;
    const size_t per_line = 2 * (size_t)nx * sizeof(C);
    int cols = 1;
    while (cols * 2 <= 16 && ny % (cols * 2) == 0 && (size_t)(cols * 2) * per_line <= kSmemBudget)
        cols *= 2;
    if ((size_t)cols * per_line > 200 * 1024) return cudaErrorInvalidValue;
    size_t smem = (size_t)cols * per_line;
    cudaError_t e = set_smem(k_fft_x<T>, smem);
    if (e != cudaSuccess) return e;
    dim3 grid(ny / cols, nb);
    k_fft_x<T><<<grid, kThreads, smem, s>>>((const C*)in, (C*)out, nx, ny, cols, d, (const C*)tw,
                                            sign);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_twiddles(void* tw, int n, cudaStream_t s) {
    k_twiddles<T><<<(n + 255) / 256, 256, 0, s>>>((cplx_t<T>*)tw, n);
    return cudaGetLastError();
}

template cudaError_t launch_fft_y<double>(const void*, void*, int, int, int, const FftDesc&,
                                          const void*, int, int, cudaStream_t);
template cudaError_t launch_fft_y<float>(const void*, void*, int, int, int, const FftDesc&,
                                         const void*, int, int, cudaStream_t);
template cudaError_t launch_fft_x<double>(const void*, void*, int, int, int, const FftDesc&,
                                          const void*, int, cudaStream_t);
template cudaError_t launch_fft_x<float>(const void*, void*, int, int, int, const FftDesc&,
                                         const void*, int, cudaStream_t);
template cudaError_t launch_fft_y_from_fix<double>(const longlong2*, double, void*, int, int,
                                                   const FftDesc&, const void*, longlong2*,
                                                   cudaStream_t);
template cudaError_t launch_fft_y_from_fix<float>(const longlong2*, double, void*, int, int,
                                                  const FftDesc&, const void*, longlong2*,
                                                  cudaStream_t);
template cudaError_t launch_twiddles<double>(void*, int, cudaStream_t);
template cudaError_t launch_twiddles<float>(void*, int, cudaStream_t);

}  // namespace gpic
