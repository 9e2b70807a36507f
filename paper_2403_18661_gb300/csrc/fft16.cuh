// Radix-16 FP32 transforms of NC = 8192 complex points for the Welch and
// whitening kernels (Sec. IV ("Noise sampling"): the PSD and the frequency-domain whitening
// are FFTs of the strain).
//
// Layout: 512 threads, one radix-16 butterfly per thread per pass; the 8192
// points live in shared memory with one pad slot after every 16, so that
// every pass below reads and writes without bank conflicts.  A butterfly
// reads three twiddles (its base angle's and the 4th and 8th multiples', FP32
// values rounded from FP64 ones) from a per-pass table ordered by butterfly
// offset, so a warp's reads coalesce; the other powers are products of those.
//
// Forward transform (Stockham auto-sort, natural order in and out): radix 16
// at strides Ns = 1, 16, 256, then radix 2 at Ns = 4096.  The first pass takes
// its 16 inputs from the caller's registers (loaded straight from global
// memory); the radix-2 pass is fused with the real-FFT split by the caller
// (mid-pass helpers below).  Inverse transform: radix 2 at Ns = 1 (fused in
// the same mid pass), then radix 16 at Ns = 2, 32, 512; the last pass returns
// its outputs in registers.
//
// Real transforms of NFFT = 16384 samples use z_n = x_2n + i x_2n+1 and the
// split X_k = E_k + W^k O_k, E_k = (Z_k + conj Z_{NC-k}) / 2,
// O_k = (Z_k - conj Z_{NC-k}) / 2i, W = exp(-2 pi i / NFFT).
//
// A 2048-point variant (real transforms of 4096 samples, 512 threads, radix-4
// passes and the fused radix 2) serves short whitening pieces of streams.
#pragma once

#include <cuda_runtime.h>

#include "afg_internal.cuh"

namespace r16 {

constexpr int NT = 512;                // threads per CTA
constexpr int SLOTS = NC + NC / 16;    // padded shared-memory slots (float2)
static_assert(NC == 16 * 16 * 16 * 2, "radix plan assumes NC = 8192");
static_assert(NC / 16 == NT, "one radix-16 butterfly per thread per pass");

__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 conj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * (S i)
template <int S> __device__ __forceinline__ float2 mul_i(float2 a) {
    return S < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}
// Packed complex add and subtract: one FP32x2 instruction each (a - b as the exact fma(b, -1, a)).
__device__ __forceinline__ float2 cadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }

// ---- twiddle table: FP32 values of exp(-i pi a), rounded from FP64 (k_tw32 fills it once per device)
//   [tw16_off(Ns), +3 Ns): radix-16 passes of the 8192-point plan, Ns in {2, 16, 32, 256, 512}:
//       w1, w4, w8 of butterfly offset k < Ns at +k, +Ns + k, +2 Ns + k (a = m k / 8 Ns, m = 1, 4, 8)
//   [tw4_off(Ns), +Ns): radix-4 passes of the 2048-point plan, Ns = 2 .. 512: w1 (a = k / 2 Ns)
//   [TW_SPLIT, +4097): the split and radix-2 table, a = j / 8192 for j = 0 .. 4096
__host__ __device__ constexpr int tw16_off(int Ns) {
    return Ns == 2 ? 0 : Ns == 16 ? 6 : Ns == 32 ? 54 : Ns == 256 ? 150 : Ns == 512 ? 918 : -1;
}
constexpr int TW16_END = 918 + 3 * 512;
__host__ __device__ constexpr int tw4_off(int Ns) { return TW16_END + Ns - 2; }  // 2 + 4 + .. + Ns/2 = Ns - 2
constexpr int TW_SPLIT = tw4_off(1024);
constexpr int TW_TOTAL = TW_SPLIT + 4097;
static_assert(tw16_off(16) == 3 * 2 && tw16_off(32) == tw16_off(16) + 3 * 16 && tw16_off(256) == tw16_off(32) + 3 * 32 &&
                  tw16_off(512) == tw16_off(256) + 3 * 256,
              "radix-16 pass tables are packed back to back");
static __device__ float2 g_tw[TW_TOTAL];

// exp(S i pi a) from table entry i (the table holds the S = -1 value)
template <int S> __device__ __forceinline__ float2 tw_at(int i) {
    const float2 w = __ldg(&g_tw[i]);
    return S < 0 ? w : make_float2(w.x, -w.y);
}
// exp(S i pi j / 8192), 0 <= j <= 4096
template <int S> __device__ __forceinline__ float2 tw_split(int j) { return tw_at<S>(TW_SPLIT + j); }

// DFT of 4 points in natural order, kernel exp(S 2 pi i / 4)
// (The sums whose operands are register pairs as they stand are packed; the two that take S i (v1 - v3),
// whose parts trade places, stay scalar.)
template <int S> __device__ __forceinline__ void dft4(float2 &v0, float2 &v1, float2 &v2, float2 &v3) {
    const float2 e0 = cadd2(v0, v2), e1 = csub2(v0, v2);
    const float2 o0 = cadd2(v1, v3), o1 = mul_i<S>(csub2(v1, v3));
    v0 = cadd2(e0, o0);
    v2 = csub2(e0, o0);
    v1 = cadd(e1, o1);
    v3 = csub(e1, o1);
}

// multiply by exp(S 2 pi i M / 16) for a constant M in {1, 2, 3, 6, 9}
template <int S, int M> __device__ __forceinline__ float2 w16(float2 a) {
    constexpr float C1 = 0.923879532511286756128f;  // cos(pi / 8)
    constexpr float S1 = 0.382683432365089771728f;  // sin(pi / 8)
    constexpr float H = 0.707106781186547524401f;   // cos(pi / 4)
    constexpr float c = M == 1 ? C1 : M == 2 ? H : M == 3 ? S1 : M == 6 ? -H : -C1;
    constexpr float s = M == 1 ? S1 : M == 2 ? H : M == 3 ? C1 : M == 6 ? H : -S1;
    return cmul(a, make_float2(c, S < 0 ? -s : s));
}

// DFT of 16 points, kernel exp(S 2 pi i / 16), as 4 x 4: n = 4 n1 + n2,
// k = k1 + 4 k2.  On return X_q is in v[4 (q & 3) + (q >> 2)]; out16() reads
// it back in natural order.
template <int S> __device__ __forceinline__ void dft16(float2 (&v)[16]) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<S>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
    v[5] = w16<S, 1>(v[5]);
    v[6] = w16<S, 2>(v[6]);
    v[7] = w16<S, 3>(v[7]);
    v[9] = w16<S, 2>(v[9]);
    v[10] = mul_i<S>(v[10]);
    v[11] = w16<S, 6>(v[11]);
    v[13] = w16<S, 3>(v[13]);
    v[14] = w16<S, 6>(v[14]);
    v[15] = w16<S, 9>(v[15]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<S>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
}
__device__ __forceinline__ int out16(int q) { return 4 * (q & 3) + (q >> 2); }

// v[r] *= exp(S i pi x r), r = 1..15 (x = k / 8 Ns for butterfly offset k < Ns)
template <int S, int Ns> __device__ __forceinline__ void twiddle16(float2 (&v)[16], int k) {
    constexpr int T = tw16_off(Ns);
    static_assert(T >= 0, "no twiddle table for this stride");
    const float2 w1 = tw_at<S>(T + k), w4 = tw_at<S>(T + Ns + k), w8 = tw_at<S>(T + 2 * Ns + k);
    const float2 w2 = cmul(w1, w1), w3 = cmul(w2, w1), w12 = cmul(w8, w4);
    v[1] = cmul(v[1], w1);
    v[2] = cmul(v[2], w2);
    v[3] = cmul(v[3], w3);
    v[4] = cmul(v[4], w4);
    v[5] = cmul(v[5], cmul(w4, w1));
    v[6] = cmul(v[6], cmul(w4, w2));
    v[7] = cmul(v[7], cmul(w4, w3));
    v[8] = cmul(v[8], w8);
    v[9] = cmul(v[9], cmul(w8, w1));
    v[10] = cmul(v[10], cmul(w8, w2));
    v[11] = cmul(v[11], cmul(w8, w3));
    v[12] = cmul(v[12], w12);
    v[13] = cmul(v[13], cmul(w12, w1));
    v[14] = cmul(v[14], cmul(w12, w2));
    v[15] = cmul(v[15], cmul(w12, w3));
}

// Radix-16 butterfly of thread j at stride Ns on inputs already in v (read
// from positions j + 512 r): twiddles, DFT; outputs stay in v (out16 order).
template <int S, int Ns> __device__ __forceinline__ void butterfly16(float2 (&v)[16], int j) {
    if constexpr (Ns > 1) twiddle16<S, Ns>(v, j & (Ns - 1));
    dft16<S>(v);
}

// Store thread j's butterfly outputs of a pass at stride Ns (Stockham order).
// (For a power-of-two Ns, pad(base + q Ns) = pad(base) + off(q) with the constant off(q) = q Ns + (q Ns >> 4):
// base = 16 (j - k) + k with k < Ns, so adding q Ns to base & 15 = k crosses a multiple of 16 exactly when
// q Ns does.  The same holds for the radix-4 bases 4 (j - k) + k, whose low four bits plus r Ns stay below
// the next multiple of 16 that r Ns passes.)
__host__ __device__ constexpr int pad_off(int i) { return i + (i >> 4); }
template <int Ns> __device__ __forceinline__ void store16(float2 *d, const float2 (&v)[16], int j) {
    const int k = j & (Ns - 1);
    float2 *p = d + pad((j - k) * 16 + k);
#pragma unroll
    for (int q = 0; q < 16; ++q) p[pad_off(q * Ns)] = v[out16(q)];
}

// the 16 inputs of butterfly j of a radix-16 pass over LEN = 16 NTX points
template <int NTX = NT> __device__ __forceinline__ void load16(float2 (&v)[16], const float2 *d, int j) {
    static_assert(NTX % 16 == 0, "pad(j + NTX r) = pad(j) + pad(NTX r)");
    const float2 *p = d + pad(j);
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = p[pad_off(NTX * r)];
}

// One in-place Stockham radix-16 pass at stride Ns over 16 NTX points (NTX threads;
// reads, barrier, writes, barrier).
template <int S, int Ns, int NTX = NT> __device__ __forceinline__ void pass16(float2 *d) {
    const int j = threadIdx.x;
    float2 v[16];
    load16<NTX>(v, d, j);
    butterfly16<S, Ns>(v, j);
    __syncthreads();
    store16<Ns>(d, v, j);
    __syncthreads();
}

// Forward transform, first three passes: v holds z[j + 512 r] of thread j on
// entry; on exit d holds the outputs of the Ns = 256 pass (synchronised).
__device__ __forceinline__ void forward_r16(float2 *d, float2 (&v)[16]) {
    const int j = threadIdx.x;
    dft16<-1>(v);
    store16<1>(d, v, j);
    __syncthreads();
    pass16<-1, 16>(d);
    pass16<-1, 256>(d);
}

// Inverse transform after the fused mid pass: the passes at Ns = 2 and 32 in
// shared memory, then the Ns = 512 pass, whose output q of thread j is
// complex sample j + 512 q, returned in v[out16(q)].
__device__ __forceinline__ void inverse_r16(float2 *d, float2 (&v)[16]) {
    const int j = threadIdx.x;
    pass16<+1, 2>(d);
    pass16<+1, 32>(d);
    load16(v, d, j);
    butterfly16<+1, 512>(v, j);
}

// Forward split of the pair (k, NC - k): X_k and X_{NC-k} from Z_k, Z_{NC-k}
// and w = W^k.  (Uses E_{NC-k} = conj E_k, O_{NC-k} = conj O_k and
// W^{NC-k} = -conj W^k, so X_{NC-k} = conj(E_k - W^k O_k).)
__device__ __forceinline__ void split_fwd(float2 zk, float2 znk, float2 w, float2 &xk, float2 &xnk) {
    const float2 zc = conj(znk);
    const float2 e = cscale(cadd(zk, zc), 0.5f);
    const float2 o = cscale(mul_i<-1>(csub(zk, zc)), 0.5f);
    const float2 wo = cmul(w, o);
    xk = cadd(e, wo);
    xnk = conj(csub(e, wo));
}

// Inverse split of the pair (k, NC - k): Z'_k and Z'_{NC-k} from the half
// spectrum Y_k, Y_{NC-k} of a real signal, so that the inverse complex
// transform of Z' is NC (y_even + i y_odd) for y = IDFT_NFFT(Y) / NFFT.
// (Z'_k = e + i o with e = (Y_k + conj Y_{NC-k}) / 2, o = (Y_k - conj Y_{NC-k}) / 2 conj W^k;
// Z'_{NC-k} = conj(e - i o).)
__device__ __forceinline__ void split_inv(float2 yk, float2 ynk, float2 w, float2 &zk, float2 &znk) {
    const float2 yc = conj(ynk);
    const float2 e = cscale(cadd(yk, yc), 0.5f);
    const float2 o = cmul(cscale(csub(yk, yc), 0.5f), conj(w));
    const float2 io = mul_i<+1>(o);
    zk = cadd(e, io);
    znk = conj(csub(e, io));
}

// ---- 2048-point variant (real transforms of 4096 samples) on NT_S = 512 threads, one
// radix-4 butterfly per thread per pass: forward radix 4 at Ns = 1, 4, 16, 64, 256, then the
// fused radix-2 pass at 1024; inverse (after the fused pass) radix 4 at Ns = 2, 8, 32, 128, 512.
// (Short pieces are latency-bound: four points per thread and more threads beat sixteen.)
constexpr int NC_S = 2048;
constexpr int NT_S = NC_S / 4;
constexpr int SLOTS_S = NC_S + NC_S / 16;

// radix-4 butterfly of thread j at stride Ns: twiddles exp(S 2 pi i r k / 4 Ns), k = j mod Ns, DFT
template <int S, int Ns> __device__ __forceinline__ void butterfly4_s(float2 (&v)[4], int j) {
    if constexpr (Ns > 1) {
        const float2 w1 = tw_at<S>(tw4_off(Ns) + (j & (Ns - 1)));
        const float2 w2 = cmul(w1, w1), w3 = cmul(w2, w1);
        v[1] = cmul(v[1], w1);
        v[2] = cmul(v[2], w2);
        v[3] = cmul(v[3], w3);
    }
    dft4<S>(v[0], v[1], v[2], v[3]);
}

template <int Ns> __device__ __forceinline__ void store4_s(float2 *d, const float2 (&v)[4], int j) {
    const int k = j & (Ns - 1);
    float2 *p = d + pad((j - k) * 4 + k);
#pragma unroll
    for (int r = 0; r < 4; ++r) p[pad_off(r * Ns)] = v[r];
}

__device__ __forceinline__ void load4_s(float2 (&v)[4], const float2 *d, int j) {
    const float2 *p = d + pad(j);
#pragma unroll
    for (int r = 0; r < 4; ++r) v[r] = p[pad_off(NT_S * r)];
}

template <int S, int Ns> __device__ __forceinline__ void pass4_s(float2 *d) {
    const int j = threadIdx.x;
    float2 v[4];
    load4_s(v, d, j);
    butterfly4_s<S, Ns>(v, j);
    __syncthreads();
    store4_s<Ns>(d, v, j);
    __syncthreads();
}

// forward passes before the fused one: v holds z[t + 512 r] on entry
__device__ __forceinline__ void forward_s(float2 *d, float2 (&v)[4]) {
    const int j = threadIdx.x;
    butterfly4_s<-1, 1>(v, j);
    store4_s<1>(d, v, j);
    __syncthreads();
    pass4_s<-1, 4>(d);
    pass4_s<-1, 16>(d);
    pass4_s<-1, 64>(d);
    pass4_s<-1, 256>(d);
}

// inverse passes after the fused one; output r of thread t is complex sample t + 512 r, in v[r]
__device__ __forceinline__ void inverse_s(float2 *d, float2 (&v)[4]) {
    pass4_s<+1, 2>(d);
    pass4_s<+1, 8>(d);
    pass4_s<+1, 32>(d);
    pass4_s<+1, 128>(d);
    load4_s(v, d, threadIdx.x);
    butterfly4_s<+1, NC_S / 4>(v, threadIdx.x);
}

}  // namespace r16
