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
#include "gpic_internal.h"

namespace gpic {

namespace {

constexpr int kThreads = 256;

template <typename C>
__device__ __forceinline__ void small_dft(C* a, int R, int sign) {
    if (R == 2) {
        C t = a[0];
        a[0] = cadd(t, a[1]);
        a[1] = csub(t, a[1]);
    } else if (R == 4) {
        C t0 = cadd(a[0], a[2]);
        C t1 = csub(a[0], a[2]);
        C t2 = cadd(a[1], a[3]);
        C t3 = cmul_si(csub(a[1], a[3]), sign);
        a[0] = cadd(t0, t2);
        a[2] = csub(t0, t2);
        a[1] = cadd(t1, t3);
        a[3] = csub(t1, t3);
    } else {  // R == 3
        using T = decltype(a[0].x);
        const T h = (T)0.86602540378443864676;  // sqrt(3)/2
        C t = cadd(a[1], a[2]);
        C d = csub(a[1], a[2]);
        C u = cmul_si(d, sign);
        u.x *= h;
        u.y *= h;
        C m = a[0];
        m.x -= (T)0.5 * t.x;
        m.y -= (T)0.5 * t.y;
        a[0] = cadd(a[0], t);
        a[1] = cadd(m, u);
        a[2] = csub(m, u);
    }
}

template <typename C>
__device__ __forceinline__ void stockham_pass(const C* __restrict__ src, C* __restrict__ dst,
                                              int n, int R, int Ns, int lines,
                                              const C* __restrict__ tw, int sign) {
    const int nr = n / R;
    const int twstep = n / (Ns * R);
    for (int idx = threadIdx.x; idx < lines * nr; idx += blockDim.x) {
        int line = idx / nr;
        int j = idx - line * nr;
        int k = j % Ns;
        const C* s = src + line * n;
        C a[4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (r < R) a[r] = s[j + r * nr];
#pragma unroll
        for (int r = 1; r < 4; ++r) {
            if (r < R && k != 0) {
                C w = __ldg(tw + r * k * twstep);
                if (sign > 0) w.y = -w.y;
                a[r] = cmul(a[r], w);
            }
        }
        small_dft(a, R, sign);
        int base = (j / Ns) * Ns * R + k;
        C* d = dst + line * n;
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (r < R) d[base + r * Ns] = a[r];
    }
}

// Runs all passes; returns the buffer that holds the result.
template <typename C>
__device__ C* run_passes(C* b0, C* b1, const FftDesc& d, int lines, const C* tw, int sign) {
    C* src = b0;
    C* dst = b1;
    int Ns = 1;
    for (int f = 0; f < d.nf; ++f) {
        int R = d.radix[f];
        stockham_pass(src, dst, d.n, R, Ns, lines, tw, sign);
        __syncthreads();
        C* t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

// Transforms along y (contiguous): CTA = `rows` consecutive x-indices of all nb arrays.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_fft_y(const cplx_t<T>* __restrict__ in, cplx_t<T>* __restrict__ out, int nx, int ny, int nb,
        int rows, FftDesc d, const cplx_t<T>* __restrict__ tw, int sign, int interleave) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* b0 = reinterpret_cast<C*>(smem_raw);
    const int lines = nb * rows;
    C* b1 = b0 + lines * ny;
    const int i0 = blockIdx.x * rows;
    const size_t plane = (size_t)nx * ny;
    for (int e = threadIdx.x; e < lines * ny; e += blockDim.x) {
        int l = e / ny, jj = e - l * ny;
        int b = l / rows, r = l - b * rows;
        b0[e] = in[b * plane + (size_t)(i0 + r) * ny + jj];
    }
    __syncthreads();
    C* res = run_passes(b0, b1, d, lines, tw, sign);
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
cudaError_t launch_fft_y(const void* in, void* out, int nx, int ny, int nb, const FftDesc& d,
                         const void* tw, int sign, int interleave, cudaStream_t s) {
    using C = cplx_t<T>;
    const size_t per_line = 2 * (size_t)ny * sizeof(C);
    int rows = 1;
    while (rows * 2 <= 8 && nx % (rows * 2) == 0 &&
           (size_t)(rows * 2) * nb * per_line <= kSmemBudget)
        rows *= 2;
    if ((size_t)rows * nb * per_line > 200 * 1024) return cudaErrorInvalidValue;
    size_t smem = (size_t)rows * nb * per_line;
    cudaError_t e = set_smem(k_fft_y<T>, smem);
    if (e != cudaSuccess) return e;
    k_fft_y<T><<<nx / rows, kThreads, smem, s>>>((const C*)in, (C*)out, nx, ny, nb, rows, d,
                                                 (const C*)tw, sign, interleave);
    return cudaGetLastError();
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
template cudaError_t launch_twiddles<double>(void*, int, cudaStream_t);
template cudaError_t launch_twiddles<float>(void*, int, cudaStream_t);

}  // namespace gpic
