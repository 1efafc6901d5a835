// Shared-memory Stockham FFT passes (radices 4, 2, 3), shared by the transform kernels
// and the fused column kernel of the field solve.
//
// Pass with radix R on lines of length n, Ns = product of the earlier radices:
//   for j in [0, n/R):  k = j mod Ns
//     a_r = src[j + r n/R] * w^(r k n/(Ns R)),  r = 0..R-1   (w = exp(sign 2 pi i / n))
//     b   = R-point DFT of a
//     dst[(j div Ns) Ns R + k + r Ns] = b_r
// which leaves the transform in natural order after the last pass.
#pragma once

#include "common.cuh"
#include "gpic_internal.h"

namespace gpic {

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
__device__ __forceinline__ C* run_passes(C* b0, C* b1, const FftDesc& d, int lines, const C* tw, int sign) {
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


}  // namespace gpic
