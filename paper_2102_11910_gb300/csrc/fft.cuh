// Shared-memory Stockham FFT executed by one thread block (internal).
//
// Length N is a power of two (4 <= N <= 4096).  Radix-4 passes, plus one
// radix-2 pass when log2(N) is odd.  Forward transform: X(k) = sum_n x(n)
// exp(-2 pi i k n / N); inverse: the same with +i, unnormalised.
// tw[m] = exp(-2 pi i m / N), m in [0, N).
#pragma once
#include "common.cuh"

template <typename C, bool INV>
__device__ __forceinline__ C* block_fft(C* a, C* b, int N, const C* __restrict__ tw) {
    C* src = a;
    C* dst = b;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int N4 = N >> 2;
    int Ns = 1;
    while (Ns * 4 <= N) {
        const int stride = N / (4 * Ns);
        for (int j = tid; j < N4; j += nt) {
            const int k = j & (Ns - 1);
            C v0 = src[j], v1 = src[j + N4], v2 = src[j + 2 * N4], v3 = src[j + 3 * N4];
            if (Ns > 1) {
                C t1 = tw[k * stride], t2 = tw[2 * k * stride], t3 = tw[3 * k * stride];
                if (INV) { t1 = conjc(t1); t2 = conjc(t2); t3 = conjc(t3); }
                v1 = v1 * t1; v2 = v2 * t2; v3 = v3 * t3;
            }
            const C a0 = v0 + v2, a1 = v0 - v2, b0 = v1 + v3, b1 = v1 - v3;
            const int d = (j - k) * 4 + k;
            dst[d] = a0 + b0;
            dst[d + 2 * Ns] = a0 - b0;
            if (!INV) { dst[d + Ns] = a1 + mul_mi(b1); dst[d + 3 * Ns] = a1 + mul_i(b1); }
            else      { dst[d + Ns] = a1 + mul_i(b1);  dst[d + 3 * Ns] = a1 + mul_mi(b1); }
        }
        __syncthreads();
        C* t = src; src = dst; dst = t;
        Ns *= 4;
    }
    if (Ns < N) {
        const int N2 = N >> 1, stride = N / (2 * Ns);
        for (int j = tid; j < N2; j += nt) {
            const int k = j & (Ns - 1);
            C v0 = src[j], v1 = src[j + N2];
            C t = tw[k * stride];
            if (INV) t = conjc(t);
            v1 = v1 * t;
            const int d = (j - k) * 2 + k;
            dst[d] = v0 + v1;
            dst[d + Ns] = v0 - v1;
        }
        __syncthreads();
        C* t = src; src = dst; dst = t;
    }
    return src;
}
