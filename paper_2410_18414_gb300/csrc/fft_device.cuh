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

// x / d for x < 2^16 by one multiply-high with m = ceil(2^32 / d) (m = 0: d = 1).
__device__ __forceinline__ int fdiv(int x, unsigned m) {
    return m ? (int)__umulhi((unsigned)x, m) : x;
}

template <int R, typename C>
__device__ __forceinline__ void small_dft_r(C* a, int sign) {
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

// One radix-R pass of pass index f over `lines` lines.
template <int R, typename C>
__device__ __forceinline__ void stockham_pass(const C* __restrict__ src, C* __restrict__ dst,
                                              const FftDesc& d, int f, int lines,
                                              const C* __restrict__ tw, int sign) {
    const int n = d.n, Ns = d.ns[f], nr = d.nr[f], twstep = d.twstep[f];
    const unsigned m_nr = d.m_nr[f], m_ns = d.m_ns[f];
    for (int idx = threadIdx.x; idx < lines * nr; idx += blockDim.x) {
        const int line = fdiv(idx, m_nr);
        const int j = idx - line * nr;
        const int q = fdiv(j, m_ns);
        const int k = j - q * Ns;
        const C* s = src + line * n;
        C a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = s[j + r * nr];
        if (k != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = tw[r * k * twstep];
                if (sign > 0) w.y = -w.y;
                a[r] = cmul(a[r], w);
            }
        }
        small_dft_r<R>(a, sign);
        C* o = dst + line * n + q * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) o[r * Ns] = a[r];
    }
}

// Copies the n twiddles to shared memory (all threads of the CTA; the caller syncs).
// They are constant, so a kernel may do this before waiting on its predecessor.
template <typename C>
__device__ __forceinline__ void stage_twiddles(const C* __restrict__ tw, C* __restrict__ dst, int n) {
    for (int m = threadIdx.x; m < n; m += blockDim.x) dst[m] = __ldg(tw + m);
}

// Runs all passes (tw may point to global or shared memory); returns the buffer that
// holds the result.
template <typename C>
__device__ __forceinline__ C* run_passes(C* b0, C* b1, const FftDesc& d, int lines, const C* tw, int sign) {
    C* src = b0;
    C* dst = b1;
    for (int f = 0; f < d.nf; ++f) {
        switch (d.radix[f]) {
            case 4: stockham_pass<4>(src, dst, d, f, lines, tw, sign); break;
            case 2: stockham_pass<2>(src, dst, d, f, lines, tw, sign); break;
            default: stockham_pass<3>(src, dst, d, f, lines, tw, sign); break;
        }
        __syncthreads();
        C* t = src;
        src = dst;
        dst = t;
    }
    return src;
}


}  // namespace gpic
