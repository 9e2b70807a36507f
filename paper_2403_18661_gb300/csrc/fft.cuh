// Shared-memory FFT building blocks, templated on the complex type; the FP64
// filter build uses them (the FP32 Welch and whitening transforms are in
// fft16.cuh).
//
// Complex FFT of NC = 8192 points as a Stockham auto-sort sequence of
// radix-8 passes (8*8*8*8) plus one radix-2 pass (and of 2048 points:
// 8*8*8*4, and of 512: 8*8*8).  Each pass reads R points
// at stride NC/R into registers, applies the twiddles, does an in-register
// DFT of size R and writes the R results at stride Ns; in place, with a
// barrier between the reads and the writes.  Twiddles come from a table
// tw[k] = exp(-2 pi i k / NFFT) (NFFT = 2 NC), which also serves the real-FFT
// split.  All index arithmetic is power-of-two.
#pragma once

#include <cuda_runtime.h>

#include "afg_internal.cuh"

template <typename T> struct Cx;
template <> struct Cx<float> { using t = float2; };
template <> struct Cx<double> { using t = double2; };

template <typename C> __device__ __forceinline__ C cmk(decltype(C::x) a, decltype(C::x) b) { C r; r.x = a; r.y = b; return r; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) { return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmk<C>(a.x, -a.y); }
// multiply by (SIGN * i)
template <typename C, int SIGN> __device__ __forceinline__ C cmul_i(C a) {
    return SIGN < 0 ? cmk<C>(a.y, -a.x) : cmk<C>(-a.y, a.x);
}

// twiddle exp(SIGN * 2 pi i idx / NFFT) from the forward table
template <typename C, int SIGN> __device__ __forceinline__ C twiddle(const C *tw, int idx) {
    C w = tw[idx & (NFFT - 1)];
    return SIGN < 0 ? w : cconj(w);
}

template <typename C, int SIGN> __device__ __forceinline__ void dft2(C &a, C &b) {
    C t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <typename C, int SIGN> __device__ __forceinline__ void dft4(C &v0, C &v1, C &v2, C &v3) {
    C e0 = cadd(v0, v2), e1 = csub(v0, v2);
    C o0 = cadd(v1, v3), o1 = cmul_i<C, SIGN>(csub(v1, v3));
    v0 = cadd(e0, o0);
    v2 = csub(e0, o0);
    v1 = cadd(e1, o1);
    v3 = csub(e1, o1);
}

template <typename C, int SIGN> __device__ __forceinline__ void dft8(C *v) {
    using T = decltype(C::x);
    const T h = (T)0.70710678118654752440084436210485;
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<C, SIGN>(e0, e1, e2, e3);
    dft4<C, SIGN>(o0, o1, o2, o3);
    // W8^k = exp(SIGN 2 pi i k / 8)
    C w1 = cmk<C>(h, SIGN * h);
    C w3 = cmk<C>(-h, SIGN * h);
    o1 = cmul(o1, w1);
    o2 = cmul_i<C, SIGN>(o2);
    o3 = cmul(o3, w3);
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

// One Stockham pass of radix R over LEN points held in shared memory `d`.
template <typename C, int R, int SIGN, int NT, int LEN = NC>
__device__ __forceinline__ void stockham_pass(C *d, int Ns, const C *tw) {
    constexpr int NB = LEN / R;         // butterflies in the pass
    constexpr int BPT = (NB + NT - 1) / NT;
    C v[BPT][R];
    const int tid = threadIdx.x;
    // twiddle step on the NFFT table: exp(SIGN 2 pi i r k / (Ns R)) = tw[r k NFFT/(Ns R)]
    const int tscale = NFFT / (Ns * R);
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
        int j = tid + q * NT;
        if (NB % NT == 0 || j < NB) {
            int k = j & (Ns - 1);
#pragma unroll
            for (int r = 0; r < R; ++r) v[q][r] = d[j + r * NB];
            if (Ns > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) v[q][r] = cmul(v[q][r], twiddle<C, SIGN>(tw, r * k * tscale));
            }
            if (R == 8) dft8<C, SIGN>(v[q]);
            else if (R == 4) dft4<C, SIGN>(v[q][0], v[q][1], v[q][2], v[q][3]);
            else dft2<C, SIGN>(v[q][0], v[q][1]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
        int j = tid + q * NT;
        if (NB % NT == 0 || j < NB) {
            int k = j & (Ns - 1);
            int base = (j - k) * R + k;  // (j / Ns) * Ns * R + k
#pragma unroll
            for (int r = 0; r < R; ++r) d[base + r * Ns] = v[q][r];
        }
    }
    __syncthreads();
}

// Complex FFT of NC points in shared memory, natural order in and out,
// unnormalised: X_k = sum_n x_n exp(SIGN 2 pi i k n / NC).  Caller syncs before.
template <typename C, int SIGN, int NT>
__device__ __forceinline__ void fft_nc(C *d, const C *tw) {
    stockham_pass<C, 8, SIGN, NT>(d, 1, tw);
    stockham_pass<C, 8, SIGN, NT>(d, 8, tw);
    stockham_pass<C, 8, SIGN, NT>(d, 64, tw);
    stockham_pass<C, 8, SIGN, NT>(d, 512, tw);
    stockham_pass<C, 2, SIGN, NT>(d, 4096, tw);
}

// Complex FFT of 2048 points in shared memory (radix 8, 8, 8, 4), natural order in and
// out, unnormalised, twiddles from the same NFFT table.  Caller syncs before.
template <typename C, int SIGN, int NT>
__device__ __forceinline__ void fft_2048(C *d, const C *tw) {
    stockham_pass<C, 8, SIGN, NT, 2048>(d, 1, tw);
    stockham_pass<C, 8, SIGN, NT, 2048>(d, 8, tw);
    stockham_pass<C, 8, SIGN, NT, 2048>(d, 64, tw);
    stockham_pass<C, 4, SIGN, NT, 2048>(d, 512, tw);
}

// Complex FFT of 512 points in shared memory (radix 8, 8, 8), as fft_2048.
template <typename C, int SIGN, int NT>
__device__ __forceinline__ void fft_512(C *d, const C *tw) {
    stockham_pass<C, 8, SIGN, NT, 512>(d, 1, tw);
    stockham_pass<C, 8, SIGN, NT, 512>(d, 8, tw);
    stockham_pass<C, 8, SIGN, NT, 512>(d, 64, tw);
}

// Real-FFT split after a forward complex FFT of z_j = x_{2j} + i x_{2j+1}:
// d[0..NC) holds Z on entry; on exit d[0..NC] holds X_k, k in [0, NC], the
// first half of the DFT of the NFFT real samples.  d must have NC+1 slots.
template <typename C, int NT>
__device__ __forceinline__ void real_split_forward(C *d, const C *tw) {
    using T = decltype(C::x);
    const T half = (T)0.5;
    for (int k = threadIdx.x; k <= NC / 2; k += NT) {
        int nk = (NC - k) & (NC - 1);
        C zk = d[k], zn = cconj(d[nk]);
        C e = cmk<C>(half * (zk.x + zn.x), half * (zk.y + zn.y));
        C o = cmul_i<C, -1>(cmk<C>(half * (zk.x - zn.x), half * (zk.y - zn.y)));  // (zk - zn) / (2i)
        C xk = cadd(e, cmul(twiddle<C, -1>(tw, k), o));
        // partner bin NC - k: Z_{NC-k} and conj(Z_k)
        C zk2 = d[nk], zn2 = cconj(d[k]);
        C e2 = cmk<C>(half * (zk2.x + zn2.x), half * (zk2.y + zn2.y));
        C o2 = cmul_i<C, -1>(cmk<C>(half * (zk2.x - zn2.x), half * (zk2.y - zn2.y)));
        C xn = cadd(e2, cmul(twiddle<C, -1>(tw, NC - k), o2));
        if (k == 0) {
            d[0] = xk;       // X_0
            d[NC] = xn;      // X_NC (Nyquist): computed with k' = NC
        } else {
            d[k] = xk;
            d[NC - k] = xn;
        }
    }
    __syncthreads();
}

// Inverse split: d[0..NC] holds X_k (Hermitian half spectrum of a real
// signal of NFFT samples); on exit d[0..NC) holds Z with
// IDFT_NC(Z) = NC * (x_even + i x_odd), where x = IDFT_NFFT(X) / NFFT.
template <typename C, int NT>
__device__ __forceinline__ void real_split_inverse(C *d, const C *tw) {
    using T = decltype(C::x);
    const T half = (T)0.5;
    for (int k = threadIdx.x; k <= NC / 2; k += NT) {
        int nk = NC - k;  // in [NC/2, NC]
        C xk = d[k], xn = d[nk];
        // Z_k from X_k and conj(X_{NC-k})
        C a = xk, b = cconj(xn);
        C e = cmk<C>(half * (a.x + b.x), half * (a.y + b.y));
        C o = cmul(cmk<C>(half * (a.x - b.x), half * (a.y - b.y)), twiddle<C, +1>(tw, k));
        C zk = cadd(e, cmul_i<C, +1>(o));
        // Z_{NC-k} from X_{NC-k} and conj(X_k)
        C a2 = xn, b2 = cconj(xk);
        C e2 = cmk<C>(half * (a2.x + b2.x), half * (a2.y + b2.y));
        C o2 = cmul(cmk<C>(half * (a2.x - b2.x), half * (a2.y - b2.y)), twiddle<C, +1>(tw, nk));
        C zn = cadd(e2, cmul_i<C, +1>(o2));
        d[k] = zk;
        if (k != 0) d[nk] = zn;  // k == 0: nk == NC is outside the NC-point array
    }
    __syncthreads();
}
