// Unbounded Poisson solve psi = -L^{-1} w by zero-padded FFT convolution with
// the real, even LGF spectrum (Sec. 2.1), and the spectral node velocity.
//
// Layout of the three passes (w real, ny rows of nx nodes; torus P x Q):
//   1. rows:    two real rows j, j+1 packed as one complex row, length-P FFT,
//               split into the two half spectra A_j(k), k in [0, P/2]; the
//               generic kernels store them column-major T1[k*ny + j], the
//               register-resident ones in groups of four rows (see below).
//   2. columns: for each k, length-Q FFT of T1[k, 0..ny) (zero padded),
//               multiply by the kernel spectrum (psi: -dx^2 Ghat/(PQ); for the
//               node velocity the spectra of the centred-differenced LGF,
//               u: -dx/2 D_y G, v: +dx/2 D_x G, which is exactly the central
//               difference of psi), inverse FFT, keep rows [0, ny).
//   3. rows:    rebuild full Hermitian rows from the half spectra of two real
//               outputs (psi_j + i psi_{j+1}, or u_j + i v_j), inverse FFT,
//               keep nodes [0, nx).
#include <type_traits>

#include "dfloat.cuh"
#include "fft.cuh"
#include "fft_reg.cuh"

template <> struct real_of<dfc> { using type = dfl; };

template <typename T>
__global__ void __launch_bounds__(512) k_rows_fwd(const T* __restrict__ w, C_t<T>* __restrict__ T1, int nx, int ny,
                                                  int P, const C_t<T>* __restrict__ tw) {
    using C = C_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* A = reinterpret_cast<C*>(smem_raw);
    C* B = A + P;
    const int j0 = 2 * blockIdx.x;
    const bool has2 = (j0 + 1) < ny;
    for (int n = threadIdx.x; n < P; n += blockDim.x) {
        T a = 0, b = 0;
        if (n < nx) {
            a = w[(size_t)j0 * nx + n];
            if (has2) b = w[(size_t)(j0 + 1) * nx + n];
        }
        A[n] = cmake<C>(a, b);
    }
    __syncthreads();
    C* Z = block_fft<C, false>(A, B, P, tw);
    for (int k = threadIdx.x; k <= P / 2; k += blockDim.x) {
        const C z1 = Z[k], z2 = conjc(Z[(P - k) & (P - 1)]);
        T1[(size_t)k * ny + j0] = (z1 + z2) * T(0.5);
        if (has2) T1[(size_t)k * ny + j0 + 1] = mul_mi(z1 - z2) * T(0.5);
    }
}

template <typename T>
__global__ void __launch_bounds__(512) k_cols(const C_t<T>* __restrict__ T1, C_t<T>* __restrict__ T2a,
                                              C_t<T>* __restrict__ T2b, int ny, int Q, int mode,
                                              const T* __restrict__ H, const T* __restrict__ Hu,
                                              const T* __restrict__ Hv, int Hld, const C_t<T>* __restrict__ tw,
                                              const int* __restrict__ rows) {
    using C = C_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* A = reinterpret_cast<C*>(smem_raw);
    C* B = A + Q;
    C* D = B + Q;
    // rows (nullable, mode CONV_PSI): only output rows rows[0] .. rows[1] are
    // needed; the row pass takes rows in (even, odd) pairs, so both rows of
    // every pair that holds a needed one are written (a pair's other row
    // enters its arithmetic, and must be finite)
    const int jlo = rows ? max(rows[0], 0) & ~1 : 0, jhi = rows ? min(rows[1] | 1, ny - 1) : ny - 1;
    const int k = blockIdx.x;
    for (int l = threadIdx.x; l < Q; l += blockDim.x)
        A[l] = l < ny ? T1[(size_t)k * ny + l] : cmake<C>(T(0), T(0));
    __syncthreads();
    C* Z = block_fft<C, false>(A, B, Q, tw);
    C* other = (Z == A) ? B : A;
    const size_t row = (size_t)k * Hld;
    if (mode == CONV_UV) {
        for (int l = threadIdx.x; l < Q; l += blockDim.x) {
            const bool lo = l <= Q / 2;
            const int lq = lo ? l : Q - l;
            const C iw = mul_i(Z[l]);
            const T hu = Hu[row + lq];
            D[l] = iw * (lo ? hu : -hu);      // odd in l
            Z[l] = iw * Hv[row + lq];         // even in l
        }
        __syncthreads();
        C* U = block_fft<C, true>(D, other, Q, tw);
        for (int j = threadIdx.x; j < ny; j += blockDim.x) T2a[(size_t)k * ny + j] = U[j];
        __syncthreads();
        C* scratch = (U == D) ? other : D;
        C* V = block_fft<C, true>(Z, scratch, Q, tw);
        for (int j = threadIdx.x; j < ny; j += blockDim.x) T2b[(size_t)k * ny + j] = V[j];
    } else {
        for (int l = threadIdx.x; l < Q; l += blockDim.x) Z[l] = Z[l] * H[row + (l <= Q / 2 ? l : Q - l)];
        __syncthreads();
        C* R = block_fft<C, true>(Z, other, Q, tw);
        for (int j = jlo + (int)threadIdx.x; j <= jhi && j < ny; j += blockDim.x) T2a[(size_t)k * ny + j] = R[j];
    }
}

template <typename T>
__global__ void __launch_bounds__(512) k_rows_inv(const C_t<T>* __restrict__ T2a, const C_t<T>* __restrict__ T2b,
                                                  T* __restrict__ out, int nx, int ny, int P, int mode, T Uinf,
                                                  T Vinf, const C_t<T>* __restrict__ tw,
                                                  const int* __restrict__ rows) {
    using C = C_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* A = reinterpret_cast<C*>(smem_raw);
    C* B = A + P;
    int ja, jb;
    const C_t<T>* Sb;
    bool has_b = true;
    if (mode == CONV_UV) {
        ja = jb = blockIdx.x;
        Sb = T2b;
    } else {
        ja = 2 * blockIdx.x;
        jb = ja + 1;
        has_b = jb < ny;
        Sb = T2a;
        // rows (nullable): blocks whose two rows are not read later do nothing
        if (rows && (jb < rows[0] || ja > rows[1])) return;
    }
    const int h = P / 2;
    for (int k = threadIdx.x; k <= h; k += blockDim.x) {
        C a = T2a[(size_t)k * ny + ja];
        C b = has_b ? Sb[(size_t)k * ny + jb] : cmake<C>(T(0), T(0));
        if (k == 0 || k == h) { a.y = 0; b.y = 0; }
        A[k] = a + mul_i(b);
        if (k > 0 && k < h) A[P - k] = conjc(a) + mul_i(conjc(b));
    }
    __syncthreads();
    C* Z = block_fft<C, true>(A, B, P, tw);
    if (mode == CONV_UV) {
        T* o = out + (size_t)2 * ja * nx;
        for (int n = threadIdx.x; n < nx; n += blockDim.x) {
            o[2 * n] = Z[n].x + Uinf;
            o[2 * n + 1] = Z[n].y + Vinf;
        }
    } else {
        for (int n = threadIdx.x; n < nx; n += blockDim.x) {
            out[(size_t)ja * nx + n] = Z[n].x;
            if (has_b) out[(size_t)jb * nx + n] = Z[n].y;
        }
    }
}

// generic in-place complex FFTs of a row-major (rows x len) array, used once per
// plan to transform the LGF torus
template <typename C>
__global__ void __launch_bounds__(256) k_fft_rows_inplace(C* data, int len, const C* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* A = reinterpret_cast<C*>(smem_raw);
    C* B = A + len;
    C* row = data + (size_t)blockIdx.x * len;
    for (int n = threadIdx.x; n < len; n += blockDim.x) A[n] = row[n];
    __syncthreads();
    C* Z = block_fft<C, false>(A, B, len, tw);
    for (int n = threadIdx.x; n < len; n += blockDim.x) row[n] = Z[n];
}

template <typename C>
__global__ void __launch_bounds__(256) k_fft_cols_inplace(C* data, int width, int len, const C* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* A = reinterpret_cast<C*>(smem_raw);
    C* B = A + len;
    const int c = blockIdx.x;
    for (int n = threadIdx.x; n < len; n += blockDim.x) A[n] = data[(size_t)n * width + c];
    __syncthreads();
    C* Z = block_fft<C, false>(A, B, len, tw);
    for (int n = threadIdx.x; n < len; n += blockDim.x) data[(size_t)n * width + c] = Z[n];
}

pf_status fft2d_inplace_f64(pf_plan p, double2* data) {
    const size_t sr = 2 * (size_t)p->P * sizeof(double2), sc = 2 * (size_t)p->Q * sizeof(double2);
    PF_CUDA(p, set_smem(k_fft_rows_inplace<double2>, sr));
    PF_CUDA(p, set_smem(k_fft_cols_inplace<double2>, sc));
    k_fft_rows_inplace<double2><<<p->Q, 256, sr, p->stream>>>(data, p->P, p->twP64);
    PF_LAUNCH_CHECK(p);
    k_fft_cols_inplace<double2><<<p->P, 256, sc, p->stream>>>(data, p->P, p->Q, p->twQ64);
    PF_LAUNCH_CHECK(p);
    return PF_OK;
}


// ---------------------------------------------------------------------------
// Register-resident variants for P, Q = 256 * R3 (256 <= P, Q <= 4096).
//
// Half-spectrum layout shared by T1, T2a, T2b: rows in groups of four,
// element (j, k) at ((j / 4) * nk + k) * 4 + j % 4 with nk = P/2 + 1.  The
// forward row pass (four rows per block) then writes one contiguous run, and
// a column k is read and written as full 32-byte sectors of four rows.
__device__ __forceinline__ size_t spec_at(int j, int k, int nk) {
    return ((size_t)(j >> 2) * nk + k) * 4 + (j & 3);
}

// Two consecutive rows j, j + 1 (j even) of a half spectrum are adjacent in
// this layout: one 16-byte access in FP32, two in FP64.
template <typename C>
__device__ __forceinline__ void ld_pair(const C* p, C& a, C& b) { a = p[0]; b = p[1]; }
template <>
__device__ __forceinline__ void ld_pair<float2>(const float2* p, float2& a, float2& b) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    a = make_float2(q.x, q.y);
    b = make_float2(q.z, q.w);
}
template <typename C>
__device__ __forceinline__ void st_pair(C* p, C a, C b) { p[0] = a; p[1] = b; }
template <>
__device__ __forceinline__ void st_pair<float2>(float2* p, float2 a, float2 b) {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}

// Row groups (one complex transform of two real rows, or of one row of u + i v)
// per block of the inverse row pass: one for P >= 1024 (a 1024-row grid's
// velocity then runs as 1024 blocks of 128 threads, eight an SM, in one wave),
// two for shorter rows (a whole warp or more a block).  The forward pass keeps
// two (four rows a block: its 32-byte sectors of T1 written whole by one
// block measured faster than twice the blocks writing halves).
template <int R3> struct RowGroups { static constexpr int value = R3 >= 4 ? 1 : 2; };
constexpr int FWD_GROUPS = 2;

template <typename T, int R3>
__global__ void __launch_bounds__(16 * R3 * FWD_GROUPS) k_rows_fwd_r(const T* __restrict__ w,
                                                                                C_t<T>* __restrict__ T1, int nx,
                                                                                int ny, const C_t<T>* __restrict__ tw256,
                                                                                const C_t<T>* __restrict__ twP) {
    using C = C_t<T>;
    constexpr int P = 256 * R3, TP = P / 16, SB = SBuf<P>::size, NK = P / 2 + 1, G = FWD_GROUPS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* bufs = reinterpret_cast<C*>(smem_raw);
    const int g = threadIdx.x / TP, t = threadIdx.x % TP;
    C* buf = bufs + g * SB;
    const int r0 = 2 * G * blockIdx.x;          // the block's first row (even)
    const int j0 = r0 + 2 * g;
    const bool h0 = j0 < ny, h1 = j0 + 1 < ny;
    pdl_wait();
    C v[16];
    const int ja = h0 ? j0 : ny - 1, jb = h1 ? j0 + 1 : ny - 1;     // clamped rows: loads never branch
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int n = t + TP * r;
        const int nc = n < nx ? n : nx - 1;
        const T a = w[(size_t)ja * nx + nc], b = w[(size_t)jb * nx + nc];
        v[r] = cmake<C>(n < nx && h0 ? a : T(0), n < nx && h1 ? b : T(0));
    }
    fft_strided<C, false, R3>(v, buf, t, tw256, twP);
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[spad(t + TP * r)] = v[r];
    __syncthreads();
    // per k, the half spectra of the rows j0, j0 + 1 of each group are adjacent
    // (rows past ny get the zero spectrum of their zero input)
    C* dst = T1 + (size_t)(r0 >> 2) * NK * 4 + (r0 & 3);
    for (int e = threadIdx.x; e < NK * G; e += blockDim.x) {
        const int k = e / G, gg = e % G;
        const C* bz = bufs + gg * SB;
        const C z1 = bz[spad(k)], z2 = conjc(bz[spad((P - k) & (P - 1))]);
        st_pair(dst + 4 * k + 2 * gg, (z1 + z2) * T(0.5), mul_mi(z1 - z2) * T(0.5));
    }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

// Column pass.  The block's rows of the kernel spectra (Hu and Hv, or H) are
// copied into shared memory by cp.async as the block starts, so their loads
// overlap the column load and the forward transform.
template <typename T, int R3>
__global__ void __launch_bounds__(16 * R3, sizeof(T) == 4 ? 32 / R3 : 1) k_cols_r(
    const C_t<T>* __restrict__ T1, C_t<T>* __restrict__ T2a, C_t<T>* __restrict__ T2b, int ny, int nk, int mode,
    const T* __restrict__ H, const T* __restrict__ Hu, const T* __restrict__ Hv, int Hld,
    const C_t<T>* __restrict__ tw256, const C_t<T>* __restrict__ twQ) {
    using C = C_t<T>;
    constexpr int Q = 256 * R3, TQ = Q / 16, SB = SBuf<Q>::size;
    constexpr int NH = (Q / 2 + 1 + 3) / 4 * 4, PER = 16 / sizeof(T);   // spectrum row length, elements per copy
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* keep = buf + SB;
    T* hs0 = reinterpret_cast<T*>(keep + SB);
    T* hs1 = hs0 + NH;
    const int k = blockIdx.x, t = threadIdx.x;
    const size_t row = (size_t)k * Hld;
    pdl_wait();
    {
        const T* s0 = mode == CONV_UV ? Hu : H;
        for (int i = PER * t; i < NH; i += PER * TQ) {
            cp_async16(hs0 + i, s0 + row + i);
            if (mode == CONV_UV) cp_async16(hs1 + i, Hv + row + i);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    C v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {            // clamped row: loads never branch
        const int l = t + TQ * r;
        const C x = T1[spec_at(l < ny ? l : ny - 1, k, nk)];
        v[r] = l < ny ? x : cmake<C>(T(0), T(0));
    }
    fft_strided<C, false, R3>(v, buf, t, tw256, twQ);
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (mode == CONV_UV) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int l = t + TQ * r;
            const bool lo = l <= Q / 2;
            const int lq = lo ? l : Q - l;
            const C iw = mul_i(v[r]);
            const T hu = hs0[lq];
            keep[spad(l)] = iw * hs1[lq];          // even in l
            v[r] = iw * (lo ? hu : -hu);            // odd in l
        }
        fft_strided<C, true, R3>(v, buf, t, tw256, twQ);
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int l = t + TQ * r;
            if (l < ny) T2a[spec_at(l, k, nk)] = v[r];
            v[r] = keep[spad(l)];                    // written by this thread
        }
        fft_strided<C, true, R3>(v, buf, t, tw256, twQ);
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int l = t + TQ * r;
            if (l < ny) T2b[spec_at(l, k, nk)] = v[r];
        }
    } else {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int l = t + TQ * r;
            v[r] = v[r] * hs0[l <= Q / 2 ? l : Q - l];
        }
        fft_strided<C, true, R3>(v, buf, t, tw256, twQ);
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int l = t + TQ * r;
            if (l < ny) T2a[spec_at(l, k, nk)] = v[r];
        }
    }
}

// Inverse row pass.  A group's complex row is u_j + i v_j (node velocity: one
// row, half spectra from T2a and T2b) or psi_j + i psi_{j+1} (two rows of
// T2a).  Where the block's rows start at an even row, each k's values of two
// rows come as one 16-byte pair.  FP32 at P = 2048: one group (128 threads) a
// block at most 64 registers, eight blocks an SM, so a 1024-row grid's 1024
// blocks run in one wave.
template <typename T, int R3>
__global__ void __launch_bounds__(16 * R3 * RowGroups<R3>::value,
                                  sizeof(T) == 4 && R3 == 8 ? 8 : 1) k_rows_inv_r(const C_t<T>* __restrict__ T2a,
                                                                             const C_t<T>* __restrict__ T2b,
                                                                             T* __restrict__ out, int nx, int ny,
                                                                             int mode, T Uinf, T Vinf,
                                                                             const C_t<T>* __restrict__ tw256,
                                                                             const C_t<T>* __restrict__ twP) {
    using C = C_t<T>;
    constexpr int P = 256 * R3, TP = P / 16, SB = SBuf<P>::size, NK = P / 2 + 1, G = RowGroups<R3>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* bufs = reinterpret_cast<C*>(smem_raw);
    const int g = threadIdx.x / TP, t = threadIdx.x % TP;
    const bool uv = mode == CONV_UV;
    const int rows = uv ? G : 2 * G;                 // rows of the block
    const int r0 = rows * blockIdx.x;                // <= ny - 1: every row read lies in a stored group of four
    const int h = P / 2;
    pdl_wait();
#pragma unroll 2
    for (int k = threadIdx.x; k <= h; k += blockDim.x) {
        C a[2], b[2];
        const size_t at = spec_at(r0, k, NK);
        if (uv) {                                     // group gg takes row r0 + gg
            if (G == 2) {
                ld_pair(T2a + at, a[0], a[1]);
                ld_pair(T2b + at, b[0], b[1]);
            } else {                                  // one row a block: r0 may be odd
                a[0] = T2a[at];
                b[0] = T2b[at];
            }
#pragma unroll
            for (int gg = 0; gg < G; ++gg)
                if (r0 + gg >= ny) a[gg] = b[gg] = cmake<C>(T(0), T(0));
        } else {                                      // group gg takes rows r0 + 2 gg, r0 + 2 gg + 1
#pragma unroll
            for (int gg = 0; gg < G; ++gg) {
                ld_pair(T2a + at + 2 * gg, a[gg], b[gg]);
                if (r0 + 2 * gg >= ny) a[gg] = cmake<C>(T(0), T(0));
                if (r0 + 2 * gg + 1 >= ny) b[gg] = cmake<C>(T(0), T(0));
            }
        }
#pragma unroll
        for (int gg = 0; gg < G; ++gg) {
            C x = a[gg], y = b[gg];
            if (k == 0 || k == h) { x.y = 0; y.y = 0; }
            C* buf = bufs + gg * SB;
            buf[spad(k)] = x + mul_i(y);
            if (k > 0 && k < h) buf[spad(P - k)] = conjc(x) + mul_i(conjc(y));
        }
    }
    __syncthreads();
    C* buf = bufs + g * SB;
    C v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = buf[spad(t + TP * r)];
    __syncthreads();
    fft_strided<C, true, R3>(v, buf, t, tw256, twP);
    if (uv) {
        const int j = r0 + g;
        if (j < ny) {
            C* o = reinterpret_cast<C*>(out) + (size_t)j * nx;
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const int n = t + TP * r;
                if (n < nx) o[n] = cmake<C>(v[r].x + Uinf, v[r].y + Vinf);
            }
        }
    } else {
        const int ja = r0 + 2 * g, jb = ja + 1;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int n = t + TP * r;
            if (n < nx) {
                if (ja < ny) out[(size_t)ja * nx + n] = v[r].x;
                if (jb < ny) out[(size_t)jb * nx + n] = v[r].y;
            }
        }
    }
}

// workspaces of one convolution (half spectra of the rows, column outputs)
struct ConvWs {
    void* T1;
    void* T2a;
    void* T2b;
};

template <typename T, int R3P, int R3Q>
static pf_status conv_solve_r(pf_plan p, const T* w, T* out, int mode, T Uinf, T Vinf, const T* H, const T* Hu,
                              const T* Hv, const C_t<T>* twP, const C_t<T>* twQ, const C_t<T>* tw256, ConvWs ws) {
    using C = C_t<T>;
    constexpr int P = 256 * R3P, Q = 256 * R3Q;
    const int nx = p->nx, ny = p->ny;
    constexpr int G = RowGroups<R3P>::value;
    const size_t sf = FWD_GROUPS * (size_t)SBuf<P>::size * sizeof(C), sr = G * (size_t)SBuf<P>::size * sizeof(C);
    const size_t sc = 2 * (size_t)SBuf<Q>::size * sizeof(C) + 2 * (size_t)((Q / 2 + 1 + 3) / 4 * 4) * sizeof(T);
    PF_CUDA(p, set_smem(k_rows_fwd_r<T, R3P>, sf));
    PF_CUDA(p, set_smem(k_cols_r<T, R3Q>, sc));
    PF_CUDA(p, set_smem(k_rows_inv_r<T, R3P>, sr));
    C* T1 = reinterpret_cast<C*>(ws.T1);
    C* T2a = reinterpret_cast<C*>(ws.T2a);
    C* T2b = reinterpret_cast<C*>(ws.T2b);
    PF_KERNEL(p, "fft_rows_fwd", PF_CUDA(p, pf_launch(k_rows_fwd_r<T, R3P>, ceil_div(ny, 2 * FWD_GROUPS), 16 * R3P * FWD_GROUPS, sf, p->stream, w, T1,
                                                      nx, ny, tw256, twP)));
    PF_KERNEL(p, "fft_cols_conv", PF_CUDA(p, pf_launch(k_cols_r<T, R3Q>, P / 2 + 1, 16 * R3Q, sc, p->stream, T1, T2a,
                                                       T2b, ny, P / 2 + 1, mode, H, Hu, Hv, p->Hld, tw256, twQ)));
    const int nb = mode == CONV_UV ? ceil_div(ny, G) : ceil_div(ny, 2 * G);
    PF_KERNEL(p, "fft_rows_inv", PF_CUDA(p, pf_launch(k_rows_inv_r<T, R3P>, nb, 16 * R3P * G, sr, p->stream, T2a, T2b, out,
                                                      nx, ny, mode, Uinf, Vinf, tw256, twP)));
    return PF_OK;
}

template <typename T, int R3P>
static pf_status conv_dispatch_q(pf_plan p, const T* w, T* out, int mode, T Uinf, T Vinf, const T* H, const T* Hu,
                                 const T* Hv, const C_t<T>* twP, const C_t<T>* twQ, const C_t<T>* tw256, ConvWs ws) {
    switch (p->Q) {
        case 256: return conv_solve_r<T, R3P, 1>(p, w, out, mode, Uinf, Vinf, H, Hu, Hv, twP, twQ, tw256, ws);
        case 512: return conv_solve_r<T, R3P, 2>(p, w, out, mode, Uinf, Vinf, H, Hu, Hv, twP, twQ, tw256, ws);
        case 1024: return conv_solve_r<T, R3P, 4>(p, w, out, mode, Uinf, Vinf, H, Hu, Hv, twP, twQ, tw256, ws);
        case 2048: return conv_solve_r<T, R3P, 8>(p, w, out, mode, Uinf, Vinf, H, Hu, Hv, twP, twQ, tw256, ws);
        case 4096: return conv_solve_r<T, R3P, 16>(p, w, out, mode, Uinf, Vinf, H, Hu, Hv, twP, twQ, tw256, ws);
    }
    return PF_ERR_ARG;
}

template <typename T>
static pf_status conv_dispatch(pf_plan p, const T* w, T* out, int mode, T Uinf, T Vinf, const T* H, const T* Hu,
                               const T* Hv, const C_t<T>* twP, const C_t<T>* twQ, const C_t<T>* tw256, ConvWs ws) {
    switch (p->P) {
        case 256: return conv_dispatch_q<T, 1>(p, w, out, mode, Uinf, Vinf, H, Hu, Hv, twP, twQ, tw256, ws);
        case 512: return conv_dispatch_q<T, 2>(p, w, out, mode, Uinf, Vinf, H, Hu, Hv, twP, twQ, tw256, ws);
        case 1024: return conv_dispatch_q<T, 4>(p, w, out, mode, Uinf, Vinf, H, Hu, Hv, twP, twQ, tw256, ws);
        case 2048: return conv_dispatch_q<T, 8>(p, w, out, mode, Uinf, Vinf, H, Hu, Hv, twP, twQ, tw256, ws);
        case 4096: return conv_dispatch_q<T, 16>(p, w, out, mode, Uinf, Vinf, H, Hu, Hv, twP, twQ, tw256, ws);
    }
    return PF_ERR_ARG;
}

template <typename T>
static pf_status conv_solve_t(pf_plan p, const T* w, T* out, int mode, T Uinf, T Vinf, const T* H, const T* Hu,
                              const T* Hv, const C_t<T>* twP, const C_t<T>* twQ, ConvWs ws,
                              const int* rows = nullptr) {
    using C = C_t<T>;
    const int P = p->P, Q = p->Q, nx = p->nx, ny = p->ny;
    // the third column buffer holds the second component (mode CONV_UV) only;
    // the double-float passes of 2048 points and more run 512 threads a block,
    // one radix-4 butterfly each per pass (their arithmetic, not shared memory,
    // bounds them; shorter transforms keep 256, which have work for no more)
    const size_t sr = 2 * (size_t)P * sizeof(C), sc = (mode == CONV_UV ? 3 : 2) * (size_t)Q * sizeof(C);
    const bool df = std::is_same<T, dfl>::value;
    const int ntP = df && P >= 2048 ? 512 : 256, ntQ = df && Q >= 2048 ? 512 : 256;
    PF_CUDA(p, set_smem(k_rows_fwd<T>, sr));
    PF_CUDA(p, set_smem(k_cols<T>, sc));
    PF_CUDA(p, set_smem(k_rows_inv<T>, sr));
    C* T1 = reinterpret_cast<C*>(ws.T1);
    C* T2a = reinterpret_cast<C*>(ws.T2a);
    C* T2b = reinterpret_cast<C*>(ws.T2b);
    PF_KERNEL(p, "fft_rows_fwd", k_rows_fwd<T><<<(ny + 1) / 2, ntP, sr, p->stream>>>(w, T1, nx, ny, P, twP));
    PF_KERNEL(p, "fft_cols_conv", k_cols<T><<<P / 2 + 1, ntQ, sc, p->stream>>>(T1, T2a, T2b, ny, Q, mode, H, Hu, Hv, p->Hld, twQ,
                                                                              rows));
    const int nb = mode == CONV_UV ? ny : (ny + 1) / 2;
    PF_KERNEL(p, "fft_rows_inv", k_rows_inv<T><<<nb, ntP, sr, p->stream>>>(T2a, T2b, out, nx, ny, P, mode, Uinf, Vinf, twP,
                                                                               rows));
    return PF_OK;
}

pf_status conv_solve(pf_plan p, const void* w, void* out, int mode, double Uinf, double Vinf) {
    // register-resident kernels unless the plan is configured for the shared-memory
    // ones; grids below 256 x 256 padded nodes always take the shared-memory ones
    const bool reg = p->fft_impl == 0 && p->P >= 256 && p->Q >= 256;
    const ConvWs ws{p->T1, p->T2a, p->T2b};
    if (p->prec == PF_FP64) {
        if (reg)
            return conv_dispatch<double>(p, (const double*)w, (double*)out, mode, Uinf, Vinf, p->H64, p->Hu64, p->Hv64,
                                         p->twP64, p->twQ64, p->tw256_64, ws);
        return conv_solve_t<double>(p, (const double*)w, (double*)out, mode, Uinf, Vinf, p->H64, p->Hu64, p->Hv64,
                                    p->twP64, p->twQ64, ws);
    }
    if (reg)
        return conv_dispatch<float>(p, (const float*)w, (float*)out, mode, (float)Uinf, (float)Vinf, p->H32, p->Hu32,
                                    p->Hv32, p->twP32, p->twQ32, p->tw256_32, ws);
    return conv_solve_t<float>(p, (const float*)w, (float*)out, mode, (float)Uinf, (float)Vinf, p->H32, p->Hu32,
                               p->Hv32, p->twP32, p->twQ32, ws);
}

// psi = -L^-1 w in FP64 for either precision of plan, on the register-resident
// path (P, Q >= 256), with caller-given FP64 workspaces T1, T2 (ldT x ldK
// complex each): the surface right-hand side of the sheet solves.
pf_status conv_psi_f64(pf_plan p, const double* w, double* psi, void* T1, void* T2) {
    if (p->P < 256 || p->Q < 256) return PF_ERR_ARG;
    return conv_dispatch<double>(p, w, psi, CONV_PSI, 0.0, 0.0, p->H64, p->Hu64, p->Hv64, p->twP64, p->twQ64,
                                 p->tw256_64, ConvWs{T1, T2, T2});
}

// ---------------------------------------------------------------- double-float route
// psi = -L^-1 w for a mixed plan's FP32 w with the shared-memory passes run
// in double-float (dfloat.cuh): the FP64-class surface right-hand side of the
// sheet solves at the FP32 pipe's rate.  (The register-resident passes, fully
// unrolled, grow too large in double-float to compile in reasonable time.)
// w is widened exactly (lo = 0); psi is returned as doubles (hi + lo).

namespace {

__global__ void k_df_table(const double* __restrict__ src, int64_t n, dfl* __restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = dfl(src[i]);
}

__global__ void k_widen_df(const float* __restrict__ w, int64_t n, dfl* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = dfl(w[i], 0.0f);
}

// in place: element i of a dfl array becomes element i of a double array (same
// size), over rows rows[0] .. rows[1] (clamped to [0, ny)) of nx elements
__global__ void k_df_to_double(void* data, int nx, int ny, const int* __restrict__ rows) {
    const int64_t i0 = (int64_t)max(rows[0], 0) * nx, i1 = (int64_t)(min(rows[1], ny - 1) + 1) * nx;
    for (int64_t i = i0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < i1; i += (int64_t)gridDim.x * blockDim.x) {
        const dfl v = reinterpret_cast<const dfl*>(data)[i];
        reinterpret_cast<double*>(data)[i] = df_to_double(v);
    }
}

struct DfTables {
    const dfl* H;
    const dfc *twP, *twQ;
};

pf_status df_tables(pf_plan p, DfTables& t) {
    PlanTables* sh = p->shared;
    const size_t nh = (size_t)(p->P / 2 + 1) * p->Hld;
    std::lock_guard<std::mutex> lock(sh->mu);
    if (!sh->df) {
        const size_t bytes = nh * sizeof(dfl) + (size_t)(p->P + p->Q) * sizeof(dfc);
        void* d = nullptr;
        PF_CUDA(p, cudaMalloc(&d, bytes));
        dfl* h = (dfl*)d;
        dfc* tp = (dfc*)(h + nh);
        dfc* tq = tp + p->P;
        k_df_table<<<152 * 2, 256, 0, p->stream>>>(p->H64, (int64_t)nh, h);
        k_df_table<<<8, 256, 0, p->stream>>>((const double*)p->twP64, 2 * (int64_t)p->P, (dfl*)tp);
        k_df_table<<<8, 256, 0, p->stream>>>((const double*)p->twQ64, 2 * (int64_t)p->Q, (dfl*)tq);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);    // complete before any stream reads them
        if (e != cudaSuccess) {
            cudaFree(d);
            snprintf(p->err, sizeof(p->err), "double-float tables: %s", cudaGetErrorString(e));
            return PF_ERR_CUDA;
        }
        sh->df = d;
    }
    t.H = (const dfl*)sh->df;
    t.twP = (const dfc*)(t.H + nh);
    t.twQ = t.twP + p->P;
    return PF_OK;
}

}  // namespace

pf_status df_tables_ready(pf_plan p) {
    if (p->P < 256 || p->Q < 256) return PF_ERR_ARG;
    DfTables t;
    return df_tables(p, t);
}

// wdf: scratch of nx ny double-floats (8 bytes each); psi: nx ny doubles, of
// which only rows rows[0] .. rows[1] (device, within [0, ny)) are computed
pf_status conv_psi_df(pf_plan p, const float* w, double* psi, void* T1, void* T2, void* wdf, const int* rows) {
    if (p->P < 256 || p->Q < 256) return PF_ERR_ARG;
    DfTables t;
    PF_TRY(df_tables(p, t));
    const int64_t M = (int64_t)p->nx * p->ny;
    const int nb = (int)std::min<int64_t>(ceil_div(M, 256), 152 * 4);
    k_widen_df<<<nb, 256, 0, p->stream>>>(w, M, (dfl*)wdf);
    PF_LAUNCH_CHECK(p);
    PF_TRY(conv_solve_t<dfl>(p, (const dfl*)wdf, (dfl*)psi, CONV_PSI, dfl(0.0), dfl(0.0), t.H, t.H, t.H, t.twP, t.twQ,
                             ConvWs{T1, T2, T2}, rows));
    k_df_to_double<<<nb, 256, 0, p->stream>>>(psi, p->nx, p->ny, rows);
    PF_LAUNCH_CHECK(p);
    return PF_OK;
}
