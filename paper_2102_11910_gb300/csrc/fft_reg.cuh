// Register-resident FFT of length N = 256 * R3 (R3 in {1, 2, 4, 8, 16}) run by
// T = N / 16 threads, each holding 16 elements (internal).
//
// Layout: thread t holds x[t + T r], r = 0..15, on input AND on output, so a
// transform's output can feed the next transform (or a pointwise multiply)
// without leaving registers.  Stockham autosort passes of radix 16, 16, R3;
// data cross between threads through one shared buffer of N complex values,
// twice.  Forward: X(k) = sum_n x(n) exp(-2 pi i k n / N); inverse: +i,
// unnormalised.  tw256[m] = exp(-2 pi i m / 256), twN[m] = exp(-2 pi i m / N).
#pragma once
#include "common.cuh"

template <typename C> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };
// (double-float complex: dfloat.cuh)

// cos(2 pi m / 16) for a compile-time m
template <int M>
__host__ __device__ constexpr double cos16() {
    constexpr int m = M & 15;
    constexpr double a = 0.92387953251128674, b = 0.70710678118654752, c = 0.38268343236508977;
    return m == 0 ? 1.0 : m == 1 ? a : m == 2 ? b : m == 3 ? c : m == 4 ? 0.0 : m == 5 ? -c : m == 6 ? -b
         : m == 7 ? -a : m == 8 ? -1.0 : m == 9 ? -a : m == 10 ? -b : m == 11 ? -c : m == 12 ? 0.0
         : m == 13 ? c : m == 14 ? b : a;
}

// x * exp(-+ 2 pi i m / 16) for a compile-time m (forward: minus sign)
template <typename C, bool INV, int M>
__device__ __forceinline__ C rot16(C x) {
    using R = typename real_of<C>::type;
    constexpr int m = M & 15;
    if (m == 0) return x;
    if (m == 4) return INV ? mul_i(x) : mul_mi(x);
    if (m == 8) { x.x = -x.x; x.y = -x.y; return x; }
    if (m == 12) return INV ? mul_mi(x) : mul_i(x);
    constexpr R c = (R)cos16<m>();
    constexpr R s = (R)(INV ? cos16<m + 12>() : -cos16<m + 12>());   // sin(t) = cos(t - pi/2)
    C r;
    r.x = x.x * c - x.y * s;
    r.y = x.x * s + x.y * c;
    return r;
}

template <typename C, bool INV>
__device__ __forceinline__ void dft2(C& a, C& b) {
    const C t = a - b;
    a = a + b;
    b = t;
}

template <typename C, bool INV>
__device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
    const C a0 = v0 + v2, a1 = v0 - v2, b0 = v1 + v3, b1 = v1 - v3;
    v0 = a0 + b0;
    v2 = a0 - b0;
    if (!INV) { v1 = a1 + mul_mi(b1); v3 = a1 + mul_i(b1); }
    else      { v1 = a1 + mul_i(b1);  v3 = a1 + mul_mi(b1); }
}

template <typename C, bool INV>
__device__ __forceinline__ void dft8(C* v) {   // v[0..7] natural order in and out
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<C, INV>(e0, e1, e2, e3);
    dft4<C, INV>(o0, o1, o2, o3);
    o1 = rot16<C, INV, 2>(o1);
    o2 = rot16<C, INV, 4>(o2);
    o3 = rot16<C, INV, 6>(o3);
    v[0] = e0 + o0; v[4] = e0 - o0;
    v[1] = e1 + o1; v[5] = e1 - o1;
    v[2] = e2 + o2; v[6] = e2 - o2;
    v[3] = e3 + o3; v[7] = e3 - o3;
}

template <typename C, bool INV, int N2>
__device__ __forceinline__ void dft16_col(C* v, C* y) {
    C a0 = v[N2], a1 = v[4 + N2], a2 = v[8 + N2], a3 = v[12 + N2];
    dft4<C, INV>(a0, a1, a2, a3);
    y[N2 * 4 + 0] = a0;
    y[N2 * 4 + 1] = rot16<C, INV, N2 * 1>(a1);
    y[N2 * 4 + 2] = rot16<C, INV, N2 * 2>(a2);
    y[N2 * 4 + 3] = rot16<C, INV, N2 * 3>(a3);
}

template <typename C, bool INV, int K1>
__device__ __forceinline__ void dft16_row(C* v, const C* y) {
    C b0 = y[K1], b1 = y[4 + K1], b2 = y[8 + K1], b3 = y[12 + K1];
    dft4<C, INV>(b0, b1, b2, b3);
    v[K1] = b0; v[K1 + 4] = b1; v[K1 + 8] = b2; v[K1 + 12] = b3;
}

template <typename C, bool INV>
__device__ __forceinline__ void dft16(C* v) {   // natural order in and out
    C y[16];
    dft16_col<C, INV, 0>(v, y);
    dft16_col<C, INV, 1>(v, y);
    dft16_col<C, INV, 2>(v, y);
    dft16_col<C, INV, 3>(v, y);
    dft16_row<C, INV, 0>(v, y);
    dft16_row<C, INV, 1>(v, y);
    dft16_row<C, INV, 2>(v, y);
    dft16_row<C, INV, 3>(v, y);
}

template <typename C, bool INV, int R>
__device__ __forceinline__ void dft_r(C* v) {
    if (R == 16) dft16<C, INV>(v);
    else if (R == 8) dft8<C, INV>(v);
    else if (R == 4) dft4<C, INV>(v[0], v[1], v[2], v[3]);
    else if (R == 2) dft2<C, INV>(v[0], v[1]);
}

template <typename C, bool INV>
__device__ __forceinline__ C twiddle(const C* __restrict__ tw, int m) {
    C w = tw[m];
    if (INV) w.y = -w.y;
    return w;
}

// shared-buffer index with one pad slot per 16 elements (pass 1 writes with a
// stride of 16 elements, which would otherwise hit one bank)
__device__ __forceinline__ int spad(int i) { return i + (i >> 4); }
template <int N> struct SBuf { static constexpr int size = N + N / 16; };

// One length-N transform by the T = N/16 threads t = 0..T-1 of a group.  `buf`
// is the group's shared buffer (SBuf<N>::size complex).  All threads of the
// block must call this the same number of times (it contains __syncthreads).
template <typename C, bool INV, int R3>
__device__ __forceinline__ void fft_strided(C (&v)[16], C* buf, int t, const C* __restrict__ tw256,
                                            const C* __restrict__ twN) {
    constexpr int N = 256 * R3;
    constexpr int T = N / 16;
    // pass 1: radix 16, Ns = 1; inputs v[r] = x[t + T r]; outputs to 16 t + r
    dft16<C, INV>(v);
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[spad(16 * t + r)] = v[r];
    __syncthreads();
    // pass 2: radix 16, Ns = 16
    {
        const int k = t & 15;
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = buf[spad(t + T * r)];
#pragma unroll
        for (int r = 1; r < 16; ++r) v[r] = v[r] * twiddle<C, INV>(tw256, r * k);
        dft16<C, INV>(v);
        __syncthreads();
        if (R3 == 1) return;          // N = 256: outputs t + 16 r already in place
        const int d = (t - k) * 16 + k;
#pragma unroll
        for (int r = 0; r < 16; ++r) buf[spad(d + 16 * r)] = v[r];
    }
    __syncthreads();
    // pass 3: radix R3, Ns = 256, butterflies j = t + m T, m < 16 / R3;
    // outputs j + 256 r = t + T (m + r 16/R3) stay in registers
    // (v was stored to buf by pass 2, so the outputs go straight into v)
    if (R3 > 1) {
        constexpr int M = 16 / R3;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int j = t + m * T;
            C u[R3 > 1 ? R3 : 1];
#pragma unroll
            for (int r = 0; r < R3; ++r) u[r] = buf[spad(j + 256 * r)];
#pragma unroll
            for (int r = 1; r < R3; ++r) u[r] = u[r] * twiddle<C, INV>(twN, r * j);
            dft_r<C, INV, R3>(u);
#pragma unroll
            for (int r = 0; r < R3; ++r) v[m + r * M] = u[r];
        }
        __syncthreads();
    }
}
