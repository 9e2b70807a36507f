// Welch PSD, whitening-filter build and FFT-domain whitening
// (Sec. IV, "Noise sampling" paragraph: PSD from 8 s, frequency-domain whitening,
// 0.5 s crop at each edge; Sec. VI: PSD from the first 64 s of state).
//
// Kernels
//   k_twiddles        exp(-2 pi i k / NFFT) table in double (filter build)
//   k_periodogram     one Hann-windowed segment per CTA: FP32 real FFT in
//                     shared memory (radix-16 passes, fft16.cuh), the window
//                     applied to the spectrum (a three-bin convolution),
//                     |X_k|^2 formed in FP32 after an exact power-of-two
//                     scaling of the segment's spectrum, stored in FP64
//   k_psd_mean        FP64 mean over the K segments of each epoch (a sliding
//                     sum over a run of epochs per thread), density scaling
//                     and one-sided doubling
//   k_filter_build    one (detector, epoch) per CTA, all FP64: amplitude
//                     response psd^-1/2 above the highpass, zero-phase
//                     inverse real FFT, Hann taper of F taps, sqrt(2/fs),
//                     forward real FFT at the whitening size -> real gains
//   k_whiten          one 8192-output overlap-save block per CTA: FP32 real
//                     FFT of 8192 + F - 1 samples (zero padded to NFFT),
//                     multiply by the epoch's gains, inverse FFT, keep the
//                     outputs whose support lies inside the block.  The
//                     forward transform's last pass, the split, the gains,
//                     the inverse split and the inverse transform's first
//                     pass are one fused shared-memory pass.
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "afg_internal.cuh"
#include "fft.cuh"
#include "fft16.cuh"

namespace {

constexpr int NT64 = 1024;  // threads of the FP64 filter kernel

__global__ void k_twiddles(double2 *tw64) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NFFT) return;
    double s, c;
    sincospi(2.0 * (double)k / (double)NFFT, &s, &c);
    tw64[k] = make_double2(c, -s);
}

// The taper of the many-CTA filter build with its constant factors: tap[m + FILTER_LAGS / 2] =
// sqrt(2 / fs) (1 - cos(2 pi (m + F/2) / F)) / 2 / (2 NFFT NC) for the F taps m in [-F/2, F/2), else 0.
// The 1 / NFFT of the inverse transform, the 1 / 2 of the inverse stage's Hermitian split and the
// 1 / NC the gains are stored with are powers of two and every later step is linear, so folding them
// in here is exact.
__global__ void k_taper64(double *tap, double fs, int F) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= FILTER_LAGS) return;
    const int m = i - FILTER_LAGS / 2, half = F / 2;
    tap[i] = (m >= -half && m < half)
                 ? sqrt(2.0 / fs) * (0.5 - 0.5 * cospi(2.0 * (double)(m + half) / (double)F)) /
                       (2.0 * (double)NFFT * (double)NC)
                 : 0.0;
}

// The FP32 transforms' twiddle table (layout in fft16.cuh): entry i = exp(-i pi a_i), a_i an exact
// binary fraction, evaluated in FP64 and rounded to FP32.
__global__ void k_tw32() {
    using namespace r16;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= TW_TOTAL) return;
    double a;
    if (i < TW16_END) {
        const int ns = i < tw16_off(16) ? 2 : i < tw16_off(32) ? 16 : i < tw16_off(256) ? 32 : i < tw16_off(512) ? 256 : 512;
        const int loc = i - tw16_off(ns), m = loc / ns, k = loc % ns;  // m = 0, 1, 2: w1, w4, w8
        a = (double)((m == 0 ? 1 : m == 1 ? 4 : 8) * k) / (double)(8 * ns);
    } else if (i < TW_SPLIT) {
        const int loc = i - TW16_END;  // Ns - 2 <= loc < 2 Ns - 2
        int ns = 2;
        while (loc >= 2 * ns - 2) ns *= 2;
        a = (double)(loc - (ns - 2)) / (double)(2 * ns);
    } else {
        a = (double)(i - TW_SPLIT) / 8192.0;
    }
    double s, c;
    sincospi(a, &s, &c);
    g_tw[i] = make_float2((float)c, (float)-s);
}

// Forward radix-2 pass (Ns = 4096) and real-FFT split for task j of the
// Welch kernel, 1 <= j <= 2048: the butterflies j and 4096 - j give Z at
// j, j + 4096, 4096 - j and 8192 - j, i.e. the split pairs (j, NC - j) and
// (j + 4096, 4096 - j).  The four spectrum values U at bins j, 8192 - j, j + 4096
// and 4096 - j replace the four Z values they came from (the same slots: tasks
// touch disjoint slot sets).  (At j = 2048 the two butterflies coincide and only
// the first pair is written.)
__device__ __forceinline__ void welch_mid_task(float2 *d, int j) {
    using namespace r16;
    const float2 a = d[pad(j)], b = d[pad(j + 4096)], c = d[pad(4096 - j)], e = d[pad(8192 - j)];
    const float2 w = tw_split<-1>(j);      // W^j
    const float2 u = tw_split<-1>(2 * j);  // radix-2 twiddle of butterfly j
    const float2 u2 = make_float2(-u.x, u.y);      // of butterfly 4096 - j: -conj(u)
    const float2 ub = cmul(u, b), ue = cmul(u2, e);
    const float2 zj = cadd(a, ub), zj4 = csub(a, ub), zc = cadd(c, ue), zc4 = csub(c, ue);
    float2 x1, x1n, x2, x2n;
    split_fwd(zj, zc4, w, x1, x1n);             // bins j, 8192 - j
    split_fwd(zj4, zc, mul_i<-1>(w), x2, x2n);  // bins j + 4096, 4096 - j (W^{j+4096} = -i W^j)
    d[pad(j)] = x1;
    d[pad(8192 - j)] = x1n;
    if (j < 2048) {
        d[pad(j + 4096)] = x2;
        d[pad(4096 - j)] = x2n;
    }
}

// grid (n_seg, n_det), r16::NT threads; segment g of detector d covers x[d][g*hop, g*hop + NFFT).
// The periodic Hann window is applied in the frequency domain: its DFT has three non-zero bins,
// so the windowed spectrum is X_k = U_k / 2 - (U_{k-1} + U_{k+1}) / 4 with U the spectrum of the
// unwindowed segment (U_{-1} = conj U_1, U_{NC+1} = conj U_{NC-1} for a real segment).
__global__ void __launch_bounds__(r16::NT, 2) k_periodogram(const float *__restrict__ x, int64_t x_stride, int hop,
                                                             double *__restrict__ P, int64_t n_seg,
                                                             const float *const *__restrict__ rows, float scale) {
    using namespace r16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *d = reinterpret_cast<float2 *>(smem_raw);
    float2 *u_nyq = d + SLOTS;  // U_NC (real)
    const int64_t g = blockIdx.x;
    const int det = blockIdx.y;
    const int t = threadIdx.x;
    // row det starts at x + det * x_stride, or at rows[det] (rows of unrelated buffers)
    const float *src = (rows ? rows[det] : x + det * x_stride) + g * (int64_t)hop;
    // z_n = x_2n + i x_2n+1, n = t + 512 r (the first pass's inputs)
    float2 v[16];
    if ((reinterpret_cast<uintptr_t>(src) & 7) == 0) {  // 8-byte loads of (x_2n, x_2n+1)
        const float2 *s2 = reinterpret_cast<const float2 *>(src);
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = s2[t + NT * r];
    } else {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int i0 = 2 * (t + NT * r);
            v[r] = make_float2(src[i0], src[i0 + 1]);
        }
    }
    forward_r16(d, v);
    // the unwindowed spectrum U_0 .. U_NC into the transform's slots
    if (t == 0) {
        // butterfly 0: Z_0, Z_4096; bins 0, NC (from the self-pair k = 0) and 4096
        const float2 a = d[pad(0)], b = d[pad(4096)];
        float2 x0, xn, x4, x4d;
        split_fwd(cadd(a, b), cadd(a, b), make_float2(1.0f, 0.0f), x0, xn);
        split_fwd(csub(a, b), csub(a, b), make_float2(0.0f, -1.0f), x4, x4d);
        d[pad(0)] = x0;
        *u_nyq = xn;
        d[pad(4096)] = x4;
    } else {
        welch_mid_task(d, t);
    }
#pragma unroll
    for (int m = 1; m < 4; ++m) welch_mid_task(d, t + NT * m);
    if (t == NT - 1) welch_mid_task(d, 2048);
    __syncthreads();
    // windowed bins k = t + 512 m (and NC) in registers, and the largest component magnitude of the block
    double *out = P + ((int64_t)det * n_seg + g) * NBIN;
    auto U = [&](int k) -> float2 {
        if (k < 0) return conj(d[pad(-k)]);
        if (k == NC) return *u_nyq;
        if (k > NC) return conj(d[pad(2 * NC - k)]);
        return d[pad(k)];
    };
    auto windowed = [&](int k) {
        const float2 l = U(k - 1), c = U(k), r = U(k + 1);
        return make_float2(0.5f * c.x - 0.25f * (l.x + r.x), 0.5f * c.y - 0.25f * (l.y + r.y));
    };
    float2 X[16];
    float mx = 0.f;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        X[m] = windowed(t + NT * m);
        mx = fmaxf(mx, fmaxf(fabsf(X[m].x), fabsf(X[m].y)));
    }
    float2 Xn = make_float2(0.f, 0.f);
    if (t == NT - 1) {
        Xn = windowed(NC);
        mx = fmaxf(mx, fmaxf(fabsf(Xn.x), fabsf(Xn.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float *wmax = reinterpret_cast<float *>(u_nyq + 1);  // [NT / 32]
    if ((t & 31) == 0) wmax[t >> 5] = mx;
    __syncthreads();
    mx = 0.f;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) mx = fmaxf(mx, wmax[w]);
    // |X_k|^2 = 2^-2s ((2^s X.re)^2 + (2^s X.im)^2): the power-of-two scale is exact and brings the largest
    // component near 2^40, so the FP32 squares neither overflow nor underflow (strain spectra sit near
    // 1e-19, whose squares are below FP32's range); the sum is rounded once in FP32 (relative 1.2e-7, far
    // below the FP32 transform's own error) and rebuilt as the double with the exponent lowered by 2s, bit
    // by bit, so no FP64 instruction runs here (the mean over segments is FP64).  NaN and infinity pass through.
    int e = 0;
    frexpf(mx, &e);
    const int sc = min(40 - e, 120);
    const float s2 = __int_as_float((127 + sc) << 23);  // 2^sc (sc >= -88)
    const int ebias = 896 - 2 * sc;
    // c_k scale |X_k|^2 (the density scale and one-sided doubling of the mean, applied here in FP32 so
    // that the mean over segments is a plain FP64 sum)
    auto p2 = [&](float2 q, float f) -> double {
        const float a = q.x * s2, b = q.y * s2;
        const uint32_t u = __float_as_uint(fmaf(b, b, a * a) * f);
        const uint32_t E = u >> 23, m23 = u & 0x7FFFFFu;
        if (E == 0) return 0.0;  // zero (or below 2^-126 of the scaled range)
        if (E == 255) return __hiloint2double((int)(0x7FF00000u | (m23 ? 0x80000u : 0u)), 0);
        return __hiloint2double((int)((uint32_t)((int)E + ebias) << 20 | (m23 >> 3)), (int)((m23 & 7u) << 29));
    };
    const float f2 = 2.0f * scale;
#pragma unroll
    for (int m = 0; m < 16; ++m) out[t + NT * m] = p2(X[m], (t | m) ? f2 : scale);
    if (t == NT - 1) out[NC] = p2(Xn, scale);
}

// Epochs e0 .. e0 + PSD_EPT - 1 (those below n_psd) of one bin for a fixed segment step SS and count KK:
// with the running prefix Q[n] of the run's segments (Q[0] = 0), epoch e0 + i is Q[i SS + KK] - Q[i SS];
// the prefix passes Q[i SS] before it reaches Q[i SS + KK], so those values wait in registers.  One FP64
// add per segment and one per epoch, every periodogram value of the run loaded once.
template <int SS, int KK>
__device__ __forceinline__ void psd_run_fixed(const double *src, double *dst, int64_t e0, int64_t n_psd) {
    constexpr int E = PSD_EPT, NMAX = (E - 1) * SS + KK;
    const int n_e = (int)min((int64_t)E, n_psd - e0);
    const int n_used = (n_e - 1) * SS + KK;
    const double *s0 = src + e0 * SS * NBIN;
    double trail[E];
    double q = 0.0;
#pragma unroll
    for (int n = 0; n <= NMAX; ++n) {
        if (n % SS == 0 && n / SS < E) trail[n / SS] = q;
        if (n >= KK && (n - KK) % SS == 0 && (n - KK) / SS < n_e) dst[(e0 + (n - KK) / SS) * NBIN] = q - trail[(n - KK) / SS];
        if (n < NMAX && n < n_used) q += s0[(int64_t)n * NBIN];
    }
}

// grid (ceil(NBIN/256), ceil(n_psd/PSD_EPT), n_det): bin k of epochs [e0, e0 + PSD_EPT) as FP64 sums of the
// periodograms (already scaled by the density factor; epoch e sums segments [e seg_step, e seg_step + K)):
// a running prefix for the 8 s epochs of 64 s PSDs at 50 % overlap (step 2, 15 segments), else a sliding sum
__global__ void k_psd_mean(const double *__restrict__ P, int64_t n_seg, int seg_step, int K,
                           double *__restrict__ psd, int64_t n_psd) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NBIN) return;
    const int64_t e0 = (int64_t)blockIdx.y * PSD_EPT;
    const int det = blockIdx.z;
    const double *src = P + (int64_t)det * n_seg * NBIN + k;
    double *dst = psd + (int64_t)det * n_psd * NBIN + k;
    if (seg_step == 2 && K == 15) {
        psd_run_fixed<2, 15>(src, dst, e0, n_psd);
        return;
    }
    double acc = 0.0;
    for (int q = 0; q < K; ++q) acc += src[(e0 * seg_step + q) * NBIN];
    dst[e0 * NBIN] = acc;
    for (int64_t e = e0 + 1; e < e0 + PSD_EPT && e < n_psd; ++e) {
        const int64_t s_old = (e - 1) * seg_step, s_new = s_old + K;
        for (int q = 0; q < seg_step; ++q) acc += src[(s_new + q) * NBIN] - src[(s_old + q) * NBIN];
        dst[e * NBIN] = acc;
    }
}

// grid (n_psd, n_det); builds the whitening gains of one (detector, epoch)
__global__ void __launch_bounds__(NT64) k_filter_build(const double *__restrict__ psd, int64_t n_psd, double fs,
                                                        double f_hp, int F, const double2 *__restrict__ tw,
                                                        float *__restrict__ gains) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *d = reinterpret_cast<double2 *>(smem_raw);
    const int64_t e = blockIdx.x;
    const int det = blockIdx.y;
    const double *p = psd + ((int64_t)det * n_psd + e) * NBIN;
    // amplitude response: psd^-1/2 at and above the highpass, zero below
    for (int k = threadIdx.x; k < NBIN; k += NT64) {
        double f = (double)k * fs / (double)NFFT;
        double pk = p[k];
        double a = (f >= f_hp && pk > 0.0) ? rsqrt(pk) : 0.0;
        d[k] = make_double2(a, 0.0);
    }
    __syncthreads();
    // zero-phase impulse response h = IDFT_NFFT(A) / NFFT (real, even)
    real_split_inverse<double2, NT64>(d, tw);
    fft_nc<double2, +1, NT64>(d, tw);
    // taper to F taps about m = 0 and rescale; zero every other sample.
    // Sample i of the circular buffer is lag m = i (i < NFFT/2) or i - NFFT.
    const double norm = sqrt(2.0 / fs) / (double)NC;
    double *t = reinterpret_cast<double *>(d);
    const int half = F / 2;
    for (int i = threadIdx.x; i < NFFT; i += NT64) {
        int m = i < NFFT / 2 ? i : i - NFFT;
        double v = 0.0;
        if (m >= -half && m < half) {
            double taper = 0.5 - 0.5 * cospi(2.0 * (double)(m + half) / (double)F);
            v = t[i] * norm * taper;
        }
        t[i] = v;
    }
    __syncthreads();
    // gains G_k = DFT_NFFT(g)_k (real for the even g); stored divided by NC,
    // the factor the inverse half-length transform of k_whiten leaves over
    fft_nc<double2, -1, NT64>(d, tw);
    real_split_forward<double2, NT64>(d, tw);
    float *out = gains + ((int64_t)det * n_psd + e) * NBIN;
    for (int k = threadIdx.x; k < NBIN; k += NT64) out[k] = (float)(d[k].x / (double)NC);
}

// ---- filter build spread over many CTAs (fir_len <= 2048).  With the 16384-point grid
// N, P sub-transforms of L = N / P points (L = 2048, or 512 when few filters are built):
//   inverse:  h_m = (1/N) sum_r e^{+2 pi i r m / N} Z_r[m mod L],
//             Z_r = sum_j A_{P j + r} e^{+2 pi i j n / L}      (P inverse FFTs of L points)
//   taper:    g_m = sqrt(2/fs) taper(m) h_m,  m in [-1024, 1024) (the F <= 2048 taps lie inside)
//   forward:  G_{P j + r} = sum_n y_r[n] e^{-2 pi i j n / L},
//             y_r[n] = sum_{m = n mod L} g_m e^{-2 pi i r m / N}   (P forward FFTs of L points;
//             at L = 2048 each slot n holds one lag, at L = 512 it folds four)
// The same FP64 arithmetic as k_filter_build (up to rounding order), on many CTAs per filter
// instead of one.  A and G are real and even in k, so residue P - r is residue r reversed:
// A_{P j + P - r} = A_{P (L - 1 - j) + r}, hence Z_{P-r}[n] = e^{-2 pi i n / L} conj Z_r[n], and
// the same for G.  Only the residues r = 0 .. P/2 are transformed:
//   h_m = (1/N) (Re Z_0[n] + Re(e^{+2 pi i (P/2) m / N} Z_{P/2}[n]) + 2 sum_{0<r<P/2} Re(e^{+2 pi i r m / N} Z_r[n]))
// and G at bins k > N/2 of residues 0 < r < P/2 is written to bin N - k (residue P - r).
// Each stage pairs two real sub-transforms into one complex FFT (real amplitude response;
// Hermitian folded taps): CTA (b, f) takes residues (0, P/2) of filter f for b = 0, (2b - 1, 2b)
// for 0 < b < P/4, and for b = P/4 residue P/2 - 1 of the filters f and f + 1 (f even; the
// CTAs of odd f at b = P/4 have no work).  P / 4 + 1 CTAs per filter and stage.
constexpr int FB_LAGS = FILTER_LAGS;  // lags m in [-FB_LAGS / 2, FB_LAGS / 2)
constexpr int FB_T = 256;

template <int L>
__device__ __forceinline__ void fb_fft(double2 *d, const double2 *tw, bool inverse) {
    if (L == 2048) {
        if (inverse) fft_2048<double2, +1, FB_T>(d, tw);
        else fft_2048<double2, -1, FB_T>(d, tw);
    } else {
        if (inverse) fft_512<double2, +1, FB_T>(d, tw);
        else fft_512<double2, -1, FB_T>(d, tw);
    }
}

// The two real sub-transforms (filter f1, residue r1) and (f2, r2) of CTA (b, f) of the inverse
// and forward stages (r2 < 0: the first alone); false for a CTA without work.
template <int P>
__device__ __forceinline__ bool fb_task(int b, int64_t f, int64_t nf, int64_t &f1, int &r1, int64_t &f2, int &r2) {
    f1 = f2 = f;
    if (b < P / 4) {
        r1 = b == 0 ? 0 : 2 * b - 1;
        r2 = b == 0 ? P / 2 : 2 * b;
        return true;
    }
    if (f & 1) return false;
    r1 = r2 = P / 2 - 1;
    f2 = f + 1;
    if (f2 >= nf) r2 = -1;
    return true;
}

// grid (P / 4 + 1, n_filters): Z_r1 of filter f1 and Z_r2 of filter f2 (fb_task; filter
// f = det * n_psd + e) from one complex transform.  Both inputs A_{P j + r} are real, so each Z
// is Hermitian and C = IFFT(A_r1 + i A_r2) splits as 2 Z_r1[n] = C[n] + conj C[-n],
// 2 Z_r2[n] = (C[n] - conj C[-n]) / i.  Z holds 2 Z_r (the 1/2 is in the taper table).
template <int L>
__global__ void __launch_bounds__(FB_T) k_fb_inverse(const double *__restrict__ psd, double fs, double f_hp,
                                                     const double2 *__restrict__ tw, double2 *__restrict__ Z) {
    constexpr int P = NFFT / L;
    __shared__ double2 d[L];
    int r1, r2;
    int64_t f1, f2;
    if (!fb_task<P>(blockIdx.x, blockIdx.y, gridDim.y, f1, r1, f2, r2)) return;
    // The highpass test fr >= f_hp with fr = kk fs / NFFT, as the first bin k_hp that passes it (the same
    // FP64 expression, evaluated once per thread), and pk > 0 as a test of its bits (a positive finite or
    // infinite double; NaN and -0 fail as they do in the FP64 comparison): no FP64 instruction per bin but
    // the reciprocal square root.
    const double k0 = floor(f_hp * (double)NFFT / fs) - 1.0;
    int k_hp = f_hp != f_hp ? NFFT / 2 + 1 : k0 <= 0.0 ? 0 : k0 >= (double)NFFT ? NFFT / 2 + 1 : (int)k0;  // NaN: none
    while (k_hp <= NFFT / 2 && (double)k_hp * fs / (double)NFFT < f_hp) ++k_hp;
    auto amp = [&](const double *p, int k) {
        const int kk = k <= NFFT / 2 ? k : NFFT - k;  // the amplitude response is even in k
        const double pk = p[kk];
        const long long b = __double_as_longlong(pk);
        return (kk >= k_hp && b > 0 && b <= 0x7FF0000000000000LL) ? rsqrt(pk) : 0.0;
    };
    const double *p1 = psd + f1 * NBIN, *p2 = psd + f2 * NBIN;
    if (blockIdx.x == 0) {
        // residues 0 and P/2 are their own mirrors: A_{P j} = A_{P (L - j)}, A_{P j + P/2} = A_{P (L - 1 - j) + P/2};
        // each amplitude is evaluated once and copied to its mirror
        for (int j = threadIdx.x; j <= L / 2; j += FB_T) {
            d[j].x = amp(p1, P * j);
            if (j < L / 2) d[j].y = amp(p1, P * j + P / 2);
        }
        __syncthreads();
        for (int j = L / 2 + threadIdx.x; j < L; j += FB_T) {
            if (j > L / 2) d[j].x = d[L - j].x;
            d[j].y = d[L - 1 - j].y;
        }
    } else {
        for (int j = threadIdx.x; j < L; j += FB_T)
            d[j] = make_double2(amp(p1, P * j + r1), r2 >= 0 ? amp(p2, P * j + r2) : 0.0);
    }
    __syncthreads();
    fb_fft<L>(d, tw, true);
    double2 *z1 = Z + (f1 * P + r1) * L, *z2 = Z + (f2 * P + (r2 >= 0 ? r2 : 0)) * L;
    for (int n = threadIdx.x; n < L; n += FB_T) {
        const double2 c = d[n], cm = d[(L - n) & (L - 1)];
        z1[n] = make_double2(c.x + cm.x, c.y - cm.y);        // 2 Z_r1 (the 1/2 is in the taper table)
        if (r2 >= 0) z2[n] = make_double2(c.y + cm.y, cm.x - c.x);  // 2 Z_r2
    }
}

// g_m of lag m from the P partial transforms (slot m mod L), with the taper table tap
template <int P, int L>
__device__ __forceinline__ double fb_tap(const double2 *__restrict__ Zf, int m, const double *__restrict__ tap,
                                         const double2 *__restrict__ tw) {
    const int slot = m & (L - 1);
    double s = 0.0;
#pragma unroll 8
    for (int r = 1; r < P / 2; ++r) {
        const double2 w = tw[(r * m) & (NFFT - 1)];  // e^{-2 pi i r m / N}; use its conjugate
        const double2 v = Zf[(int64_t)r * L + slot];
        s += w.x * v.x + w.y * v.y;  // Re(conj(w) v)
    }
    const double2 wh = tw[((P / 2) * m) & (NFFT - 1)], vh = Zf[(int64_t)(P / 2) * L + slot];
    const double h = Zf[slot].x + (wh.x * vh.x + wh.y * vh.y) + 2.0 * s;
    return h * tap[m + FB_LAGS / 2];
}

// L = 2048: grid (FB_LAGS / FB_T, n_filters), one lag per thread, one lag per slot
__global__ void __launch_bounds__(FB_T) k_fb_taper(const double2 *__restrict__ Z, const double *__restrict__ tap,
                                                   const double2 *__restrict__ tw, double2 *__restrict__ Y) {
    constexpr int L = 2048, P = NFFT / L;
    const int64_t f = blockIdx.y;
    const int m = blockIdx.x * FB_T + threadIdx.x - FB_LAGS / 2;  // lag in [-1024, 1024)
    const double g = fb_tap<P, L>(Z + f * P * L, m, tap, tw);
    double2 *y = Y + f * P * L + (m & (L - 1));
#pragma unroll
    y[0] = make_double2(g, 0.0);  // residue 0: twiddle 1
#pragma unroll
    for (int r = 1; r <= P / 2; ++r) {  // the other residues the forward stage transforms
        const double2 w = tw[(r * m) & (NFFT - 1)];
        y[(int64_t)r * L] = make_double2(g * w.x, g * w.y);
    }
}

// L = 512: grid (L / FB_FS, n_filters), FB_FS slots x 4 lags per CTA.  Thread (slot n, lag t)
// forms g_m of m = n + L t - 1024, then y_r[n] for every fourth r <= P/2 from r = t, summed over
// the slot's four lags.
constexpr int FB_FS = 32;
__global__ void __launch_bounds__(FB_FS * 4) k_fb_taper_fold(const double2 *__restrict__ Z,
                                                             const double *__restrict__ tap,
                                                             const double2 *__restrict__ tw,
                                                             double2 *__restrict__ Y) {
    constexpr int L = 512, P = NFFT / L, FOLD = FB_LAGS / L;
    static_assert(FOLD == 4, "four lags per slot");
    __shared__ double gs[FOLD][FB_FS];
    const int64_t f = blockIdx.y;
    const int nl = threadIdx.x % FB_FS, t = threadIdx.x / FB_FS;
    const int n = blockIdx.x * FB_FS + nl;
    gs[t][nl] = fb_tap<P, L>(Z + f * P * L, n + L * t - FB_LAGS / 2, tap, tw);
    __syncthreads();
    double2 *y = Y + f * P * L + n;
    for (int r = t; r <= P / 2; r += FOLD) {  // the residues the forward stage transforms
        double ax = 0.0, ay = 0.0;
#pragma unroll
        for (int u = 0; u < FOLD; ++u) {
            const int m = n + L * u - FB_LAGS / 2;
            const double2 w = tw[(r * m) & (NFFT - 1)];
            ax += gs[u][nl] * w.x;
            ay += gs[u][nl] * w.y;
        }
        y[(int64_t)r * L] = make_double2(ax, ay);
    }
}

// grid (P / 4 + 1, n_filters): gains G_k / NC for k <= NFFT / 2 of the residue r1 of filter f1
// and r2 of f2 (fb_task) from one complex transform.  The taps are even, so each y_r is Hermitian and its transform
// real: FFT(y_r1 + i y_r2) = G_{P j + r1} + i G_{P j + r2}.  Bins k > NFFT / 2 of residues
// 0 < r < P/2 give bin NFFT - k (G is even), which belongs to residue P - r.
template <int L>
__global__ void __launch_bounds__(FB_T) k_fb_forward(const double2 *__restrict__ Y, const double2 *__restrict__ tw,
                                                     float *__restrict__ gains) {
    constexpr int P = NFFT / L;
    __shared__ double2 d[L];
    int r1, r2;
    int64_t f1, f2;
    if (!fb_task<P>(blockIdx.x, blockIdx.y, gridDim.y, f1, r1, f2, r2)) return;
    const double2 *y1 = Y + (f1 * P + r1) * L, *y2 = Y + (f2 * P + (r2 >= 0 ? r2 : 0)) * L;
    for (int n = threadIdx.x; n < L; n += FB_T) {
        const double2 a = y1[n], b = r2 >= 0 ? y2[n] : make_double2(0.0, 0.0);
        d[n] = make_double2(a.x - b.y, a.y + b.x);
    }
    __syncthreads();
    fb_fft<L>(d, tw, false);
    auto put = [&](float *out, int r, int k, double v) {
        if (k <= NFFT / 2) out[k] = (float)v;  // G_k / NC (the 1 / NC is in the taper table)
        else if (r != 0 && r != P / 2) out[NFFT - k] = (float)v;
    };
    float *out1 = gains + f1 * NBIN, *out2 = gains + f2 * NBIN;
    for (int j = threadIdx.x; j < L; j += FB_T) {
        put(out1, r1, P * j + r1, d[j].x);
        if (r2 >= 0) put(out2, r2, P * j + r2, d[j].y);
    }
}

// 4-byte asynchronous copy global -> shared (completes at cp_async_wait_all)
__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

// Fused mid pass of the whitening kernel for task j, 1 <= j <= NCX / 4, of a
// transform of NCX complex points (H = NCX / 2): the forward radix-2 butterflies j
// and H - j (Ns = H) give Z at j, j + H, H - j, NCX - j; the split pairs (j, NCX - j)
// and (j + H, H - j) are multiplied by the gains g (on the transform's own grid) and
// split back; the inverse radix-2 butterflies j and H - j (Ns = 1) produce o[0..1]
// for d[2j], d[2j + 1] and o[2..3] for d[2(H - j)], d[2(H - j) + 1].
template <int NCX>
__device__ __forceinline__ void whiten_mid_task(const float2 *d, const float *g, int j, float2 (&o)[4]) {
    using namespace r16;
    constexpr int H = NCX / 2;
    const float2 a = d[pad(j)], b = d[pad(j + H)], c = d[pad(H - j)], e = d[pad(NCX - j)];
    static_assert(8192 % NCX == 0, "split table step");
    constexpr int SP = 8192 / NCX;
    const float2 w = tw_split<-1>(SP * j);      // W^j, W = exp(-2 pi i / 2 NCX)
    const float2 u = tw_split<-1>(2 * SP * j);  // radix-2 twiddle of butterfly j
    const float2 u2 = make_float2(-u.x, u.y);               // of butterfly H - j
    const float2 ub = cmul(u, b), ue = cmul(u2, e);
    const float2 zj = cadd(a, ub), zj4 = csub(a, ub), zc = cadd(c, ue), zc4 = csub(c, ue);
    const float2 w4 = mul_i<-1>(w);                         // W^{j + H}
    float2 x1, x1n, x2, x2n, p1, p1n, p2, p2n;
    split_fwd(zj, zc4, w, x1, x1n);
    split_fwd(zj4, zc, w4, x2, x2n);
    split_inv(cscale(x1, g[j]), cscale(x1n, g[NCX - j]), w, p1, p1n);     // Z'_j, Z'_{NCX-j}
    split_inv(cscale(x2, g[j + H]), cscale(x2n, g[H - j]), w4, p2, p2n);  // Z'_{j+H}, Z'_{H-j}
    o[0] = cadd(p1, p2);
    o[1] = csub(p1, p2);
    o[2] = cadd(p2n, p1n);
    o[3] = csub(p2n, p1n);
}

// Task 0 of the mid pass: butterfly 0 gives Z_0 and Z_H, each its own split partner
// (bin 0 with the Nyquist bin NCX, and bin H); o[0..1] go to d[0], d[1].
template <int NCX>
__device__ __forceinline__ void whiten_mid_task0(const float2 *d, const float *g, float2 (&o)[4]) {
    using namespace r16;
    constexpr int H = NCX / 2;
    const float2 a = d[pad(0)], b = d[pad(H)];
    const float2 z0 = cadd(a, b), z4 = csub(a, b);
    const float2 one = make_float2(1.0f, 0.0f), mi = make_float2(0.0f, -1.0f);  // W^0, W^H
    float2 x0, xn, x4, x4d, p0, pn, p4, p4d;
    split_fwd(z0, z0, one, x0, xn);
    split_inv(cscale(x0, g[0]), cscale(xn, g[NCX]), one, p0, pn);
    split_fwd(z4, z4, mi, x4, x4d);
    split_inv(cscale(x4, g[H]), cscale(x4d, g[H]), mi, p4, p4d);
    o[0] = cadd(p0, p4);
    o[1] = csub(p0, p4);
    o[2] = o[0];
    o[3] = o[1];
}

constexpr int WHITEN_SMEM = r16::SLOTS * (int)sizeof(float2) + NBIN * (int)sizeof(float);
// density factor of the mean of K periodograms (periodic Hann: sum w^2 = 3 NFFT / 8), applied per segment
inline float psd_scale(int64_t K, int fs) { return (float)(1.0 / ((double)K * (double)fs * (3.0 * NFFT / 8.0))); }

constexpr int WELCH_SMEM = (r16::SLOTS + 1) * (int)sizeof(float2) + (r16::NT / 32) * (int)sizeof(float);

// One overlap-save block: the FIR of src[0 .. cnt + F - 1) (cnt <= 16385 - F; samples past
// `avail` read as zero) -> outputs q in [0, cnt) written as out(q, value), or straight to lin[q]
// when the caller's destination is the linear row lin (nullptr: always through out).
// smem: r16::SLOTS float2 for the transform, then NBIN floats for the gains gk,
// which are copied in asynchronously while the forward transform runs.
template <typename Out>
__device__ __forceinline__ void whiten_block(unsigned char *smem, const float *__restrict__ src, int64_t avail,
                                             const float *__restrict__ gk, int F, int64_t cnt, Out out,
                                             float *__restrict__ lin = nullptr) {
    using namespace r16;
    float2 *d = reinterpret_cast<float2 *>(smem);
    float *gs = reinterpret_cast<float *>(smem + SLOTS * sizeof(float2));
    const int t = threadIdx.x;
    for (int k = t; k < NBIN; k += NT) cp_async4(gs + k, gk + k);
    const int half = F / 2;
    // samples that reach a kept output (cnt + F - 1 <= 16384: indices within the block are ints)
    const int need = (int)cnt + F - 1;
    const int lim = avail <= 0 ? 0 : avail < (int64_t)need ? (int)avail : need;
    float2 v[16];
    if (avail >= 2 * NC && (reinterpret_cast<uintptr_t>(src) & 7) == 0) {  // whole block in memory: 8-byte loads
        const float2 *s2 = reinterpret_cast<const float2 *>(src);
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = s2[t + NT * r];
        if (2 * (t + NT * 15) + 1 >= lim) {  // this thread holds samples past `need`: they read as zero
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const int i0 = 2 * (t + NT * r);
                if (i0 >= lim) v[r].x = 0.0f;
                if (i0 + 1 >= lim) v[r].y = 0.0f;
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int i0 = 2 * (t + NT * r);
            v[r] = make_float2(i0 < lim ? src[i0] : 0.0f, i0 + 1 < lim ? src[i0 + 1] : 0.0f);
        }
    }
    forward_r16(d, v);
    cp_async_wait_all();
    __syncthreads();
    float2 o[4][4], ox[4];
    if (t == 0) whiten_mid_task0<NC>(d, gs, o[0]);
    else whiten_mid_task<NC>(d, gs, t, o[0]);
#pragma unroll
    for (int m = 1; m < 4; ++m) whiten_mid_task<NC>(d, gs, t + NT * m, o[m]);
    if (t == NT - 1) whiten_mid_task<NC>(d, gs, 2048, ox);
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int j = t + NT * m, jc = 4096 - j;
        d[pad(2 * j)] = o[m][0];
        d[pad(2 * j + 1)] = o[m][1];
        if (j != 0) {
            d[pad(2 * jc)] = o[m][2];
            d[pad(2 * jc + 1)] = o[m][3];
        }
    }
    if (t == NT - 1) {
        d[pad(4096)] = ox[0];
        d[pad(4097)] = ox[1];
    }
    __syncthreads();
    inverse_r16(d, v);
    // complex sample c = t + 512 q holds real samples 2c, 2c + 1; output q0 = 2c - F/2
    const int cnt32 = (int)cnt;
    // outputs (q0, q0 + 1) as one 8-byte store where the destination is linear and q0 lands 8-byte aligned
    const bool pairs = lin != nullptr && (half & 1) == 0 && (reinterpret_cast<uintptr_t>(lin) & 7) == 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const float2 y = v[out16(q)];
        const int q0 = 2 * (t + NT * q) - half;
        if (pairs && q0 >= 0 && q0 + 1 < cnt32) {
            *reinterpret_cast<float2 *>(lin + q0) = y;
        } else {
            if (q0 >= 0 && q0 < cnt32) out(q0, y.x);
            if (q0 + 1 >= 0 && q0 + 1 < cnt32) out(q0 + 1, y.y);
        }
    }
}

template <typename Out>
__device__ __forceinline__ void whiten_block_s(unsigned char *smem, const float *__restrict__ src, int64_t avail,
                                               const float *__restrict__ stg, int64_t i_new,
                                               const float *__restrict__ gk, int F, int64_t cnt, Out out);

// Block layout of one whitening launch.  Every filter epoch (the whole span when epoch_len is 0) is covered by
// blocks of bl = 16385 - F outputs (rounded down to 64) on the 16384-point transform, the most its circular
// convolution keeps, and the epoch's remainder by one more block: on the 4096-point transform where it fits
// (4097 - F outputs; 2048 of a 16384-sample epoch with F = 2048), else on the 16384-point one.  An 8192-output
// block instead would keep half of every 16384-point transform.
struct WhitenLayout {
    int64_t span, bl, n_full, rem, bpe, n_blocks;
    bool small_rem;
};
__host__ __device__ inline WhitenLayout whiten_layout(int64_t out_len, int64_t epoch_len, int F) {
    WhitenLayout w;
    w.span = epoch_len > 0 ? epoch_len : out_len;
    w.bl = ((int64_t)(2 * r16::NT * 16 + 1 - F) / 64) * 64;
    w.n_full = w.span / w.bl;
    w.rem = w.span - w.n_full * w.bl;
    w.bpe = w.n_full + (w.rem > 0 ? 1 : 0);
    w.small_rem = w.rem > 0 && w.rem <= (int64_t)(2 * r16::NC_S + 1 - F);
    const int64_t n_ep = epoch_len > 0 ? (out_len + epoch_len - 1) / epoch_len : 1;
    w.n_blocks = out_len > 0 ? n_ep * w.bpe : 0;
    return w;
}

// Block (e, i) of a whitening launch: y[d][e span + i bl, + cnt) with the gains of epoch e (cnt <= 0: none)
struct WhitenBlock {
    int64_t o, cnt, ep;
};
__device__ __forceinline__ WhitenBlock whiten_block_at(const WhitenLayout &L, int64_t e, int64_t i, int64_t out_len,
                                                       int64_t epoch_len, int64_t n_psd) {
    WhitenBlock b;
    b.o = e * L.span + i * L.bl;
    b.cnt = i < L.n_full ? L.bl : L.rem;
    if (b.cnt > out_len - b.o) b.cnt = out_len - b.o;
    b.ep = epoch_len > 0 ? e : 0;
    if (b.ep > n_psd - 1) b.ep = n_psd - 1;
    return b;
}

// grid (n_ep * n16, n_det): the blocks on the 16384-point transform, n16 per epoch (bpe, or n_full where the
// remainder goes to k_whiten_rem); block (e, i) = (blockIdx.x / n16, blockIdx.x % n16)
__global__ void __launch_bounds__(r16::NT, 2) k_whiten(const float *__restrict__ x, int64_t n, int64_t x_stride,
                                                        const float *__restrict__ gains, int64_t n_psd,
                                                        int64_t out_first, int64_t out_len, int64_t epoch_len, int F,
                                                        float *__restrict__ y, int64_t y_stride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const WhitenLayout L = whiten_layout(out_len, epoch_len, F);
    const int64_t n16 = L.small_rem ? L.n_full : L.bpe;
    const int64_t e = (int64_t)blockIdx.x / n16;
    const WhitenBlock b = whiten_block_at(L, e, (int64_t)blockIdx.x - e * n16, out_len, epoch_len, n_psd);
    if (b.cnt <= 0) return;
    const int det = blockIdx.y;
    const int64_t s0 = out_first + b.o - F / 2;  // raw index of block sample 0
    float *dst = y + det * y_stride + b.o;
    whiten_block(smem_raw, x + det * x_stride + s0, n - s0, gains + ((int64_t)det * n_psd + b.ep) * NBIN, F, b.cnt,
                 [dst](int64_t q, float v) { dst[q] = v; }, dst);
}

// grid (n_ep, n_det): each epoch's remainder block on the 4096-point transform (whiten_layout().small_rem).
// A launch of its own: its 26 KB of shared memory lets several CTAs share an SM, which the short transform's
// barrier-bound passes need.
__global__ void __launch_bounds__(r16::NT_S) k_whiten_rem(const float *__restrict__ x, int64_t n, int64_t x_stride,
                                                         const float *__restrict__ gains, int64_t n_psd,
                                                         int64_t out_first, int64_t out_len, int64_t epoch_len, int F,
                                                         float *__restrict__ y, int64_t y_stride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const WhitenLayout L = whiten_layout(out_len, epoch_len, F);
    const WhitenBlock b = whiten_block_at(L, blockIdx.x, L.n_full, out_len, epoch_len, n_psd);
    if (b.cnt <= 0) return;
    const int det = blockIdx.y;
    const int64_t s0 = out_first + b.o - F / 2;
    float *dst = y + det * y_stride + b.o;
    whiten_block_s(smem_raw, x + det * x_stride + s0, n - s0, nullptr, 0, gains + ((int64_t)det * n_psd + b.ep) * NBIN,
                   F, b.cnt, [dst](int64_t q, float v) { dst[q] = v; });
}

// Whitening pieces of many streams in one launch: grid (n_desc, 2).  Piece i
// whitens raw samples src(d) = desc.x + d * x_stride + [0, cnt + F - 1) with
// gains desc.gains + d * NBIN into the mirrored ring desc.y (row stride
// y_stride, ring length y_ring): output q goes to ring slots
// (y_pos + q) mod y_ring and that + y_ring.
// (Launched as a programmatic dependent of the scatter or gains refresh before it.)
__global__ void __launch_bounds__(r16::NT, 2) k_whiten_multi(const WhitenPiece *__restrict__ pieces, int F) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_trigger();
    const WhitenPiece pc = pieces[blockIdx.x];
    pdl_wait();  // raw rings (scatter) and gains (refresh) come from the kernels before
    const int det = blockIdx.y;
    float *yr = pc.y + det * pc.y_stride;
    const int64_t ring = pc.y_ring, pos = pc.y_pos;
    whiten_block(smem_raw, pc.x + det * pc.x_stride, pc.cnt + F - 1, pc.gains + det * NBIN, F, pc.cnt,
                 [yr, ring, pos](int64_t q, float v) {
                     int64_t m = pos + q;
                     if (m >= ring) m -= ring;
                     yr[m] = v;
                     yr[m + ring] = v;
                 });
}

constexpr int WHITEN_SMEM_S = r16::SLOTS_S * (int)sizeof(float2) + (r16::NC_S + 1) * (int)sizeof(float);

// Largest piece of the 4096-point block for a filter of F taps (0 if F leaves too few).
int whiten_piece_max_s(int F) {
    const int m = 2 * r16::NC_S - F + 1;
    return m >= 512 ? m : 0;
}

// One overlap-save block of the 4096-point transform: the FIR of src[0 .. cnt + F - 1)
// (cnt <= 4097 - F, samples past `avail` read as zero) -> outputs q in [0, cnt) written as
// out(q, value).  The taps span fewer than 4096 lags, so the gains of this grid are those
// of the 16384-point grid at every 4th bin; they are rescaled by 4 for the shorter
// transform's 1 / 2048 normalisation (exact in FP32).
// stg (may be null): input i >= i_new comes from stg[i - i_new] instead of src[i].
template <typename Out>
__device__ __forceinline__ void whiten_block_s(unsigned char *smem, const float *__restrict__ src, int64_t avail,
                                               const float *__restrict__ stg, int64_t i_new,
                                               const float *__restrict__ gk, int F, int64_t cnt, Out out) {
    using namespace r16;
    constexpr int GS = NC / NC_S;  // bins of the 16384-point grid per bin of this one
    float2 *d = reinterpret_cast<float2 *>(smem);
    float *gs = reinterpret_cast<float *>(smem + SLOTS_S * sizeof(float2));
    const int t = threadIdx.x;
    for (int k = t; k <= NC_S; k += NT_S) cp_async4(gs + k, gk + GS * k);
    const int half = F / 2;
    const int64_t need = cnt + F - 1;
    const int64_t lim = need < avail ? need : avail;
    auto sample = [&](int64_t i) -> float {
        if (i >= lim) return 0.0f;
        return (stg && i >= i_new) ? stg[i - i_new] : src[i];
    };
    float2 v[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t i0 = 2 * (int64_t)(t + NT_S * r);
        v[r] = make_float2(sample(i0), sample(i0 + 1));
    }
    forward_s(d, v);
    cp_async_wait_all();
    __syncthreads();
    for (int k = t; k <= NC_S; k += NT_S) gs[k] *= (float)GS;
    __syncthreads();
    // one task per thread (tasks 0 .. NC_S / 4 - 1), the last thread also task NC_S / 4
    static_assert(NT_S == NC_S / 4, "one mid-pass task per thread");
    float2 o[4], ox[4];
    if (t == 0) whiten_mid_task0<NC_S>(d, gs, o);
    else whiten_mid_task<NC_S>(d, gs, t, o);
    if (t == NT_S - 1) whiten_mid_task<NC_S>(d, gs, NC_S / 4, ox);
    __syncthreads();
    {
        const int j = t, jc = NC_S / 2 - j;
        d[pad(2 * j)] = o[0];
        d[pad(2 * j + 1)] = o[1];
        if (j != 0) {
            d[pad(2 * jc)] = o[2];
            d[pad(2 * jc + 1)] = o[3];
        }
    }
    if (t == NT_S - 1) {
        d[pad(NC_S / 2)] = ox[0];
        d[pad(NC_S / 2 + 1)] = ox[1];
    }
    __syncthreads();
    float2 y[4];
    inverse_s(d, y);
    // complex sample c = t + 512 r holds real samples 2c, 2c + 1; output q0 = 2c - F/2
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t q0 = 2 * (int64_t)(t + NT_S * r) - half;
        if (q0 >= 0 && q0 < cnt) out(q0, y[r].x);
        if (q0 + 1 >= 0 && q0 + 1 < cnt) out(q0 + 1, y[r].y);
    }
}

// k_whiten_multi with the 4096-point block (512 threads): pieces of at most 4097 - F outputs.
__global__ void __launch_bounds__(r16::NT_S) k_whiten_multi_s(const WhitenPiece *__restrict__ pieces, int F) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_trigger();
    const WhitenPiece pc = pieces[blockIdx.x];
    pdl_wait();  // raw rings (scatter) and gains (refresh) come from the kernels before
    const int det = blockIdx.y;
    const float *stg = pc.stg ? pc.stg + det * pc.stg_stride : nullptr;
    if (pc.sc_ring) {  // the stream's new samples into its mirrored raw ring (read by later steps)
        float *row = pc.sc_ring + det * 2 * pc.sc_R;
        for (int64_t k = threadIdx.x; k < pc.sc_n; k += r16::NT_S) {
            int64_t m = pc.sc_pos + k;
            if (m >= pc.sc_R) m -= pc.sc_R;
            const float v = stg[k];
            row[m] = v;
            row[m + pc.sc_R] = v;
        }
    }
    float *yr = pc.y + det * pc.y_stride;
    const int64_t ring = pc.y_ring, pos = pc.y_pos;
    whiten_block_s(smem_raw, pc.x + det * pc.x_stride, pc.cnt + F - 1, stg, pc.i_new, pc.gains + det * NBIN, F,
                   pc.cnt,
                   [yr, ring, pos](int64_t q, float v) {
                       int64_t m = pos + q;
                       if (m >= ring) m -= ring;
                       yr[m] = v;
                       yr[m + ring] = v;
                   });
}

bool g_attrs_set = false;

int set_attrs(afg_ctx *ctx) {
    if (g_attrs_set) return AFG_OK;
    AFG_CUDA(ctx, cudaFuncSetAttribute(k_periodogram, cudaFuncAttributeMaxDynamicSharedMemorySize, WELCH_SMEM));
    AFG_CUDA(ctx, cudaFuncSetAttribute(k_whiten, cudaFuncAttributeMaxDynamicSharedMemorySize, WHITEN_SMEM));
    AFG_CUDA(ctx, cudaFuncSetAttribute(k_whiten_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, WHITEN_SMEM));
    AFG_CUDA(ctx, cudaFuncSetAttribute(k_whiten_multi_s, cudaFuncAttributeMaxDynamicSharedMemorySize, WHITEN_SMEM_S));
    AFG_CUDA(ctx, cudaFuncSetAttribute(k_filter_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)((NC + 1) * sizeof(double2))));
    g_attrs_set = true;
    return AFG_OK;
}

}  // namespace

// device scratch of building nf filters at once: two FP64 complex transforms of NFFT points per
// filter for the many-CTA build (fir_len <= 2048), none for the one-CTA build
size_t filter_build_scratch_bytes(const afg_ctx *ctx, int64_t nf) {
    if (ctx->cfg.fir_len > FB_LAGS || nf > 65535) return 0;
    return (size_t)2 * nf * NFFT * sizeof(double2);
}

// gains [n_det][n_psd][NBIN] from psd: the many-CTA FP64 build where fir_len <= 2048,
// else one CTA per filter
int filter_build(afg_ctx *ctx, const double *psd, int n_det, int64_t n_psd, float *gains, cudaStream_t st) {
    const int64_t nf = (int64_t)n_det * n_psd;
    if (nf <= 0) return AFG_OK;
    // algorithmic FP64 work of one filter: an inverse and a forward transform of a real, even
    // sequence of NFFT points (the amplitude response and the taps), 1.25 N log2 N flops each
    // (half of a real FFT's 2.5 N log2 N)
    const double flops = (double)nf * 2.0 * 1.25 * NFFT * 14.0;
    static_assert(NFFT == 1 << 14, "flop count assumes log2(NFFT) = 14");
    if (ctx->cfg.fir_len <= FB_LAGS && nf <= 65535) {
        void *scr = nullptr;
        int rc = afg_ws_reserve(ctx, WS_FB_SCRATCH, filter_build_scratch_bytes(ctx, nf), &scr);
        if (rc) return rc;
        double2 *Z = static_cast<double2 *>(scr), *Y = Z + nf * NFFT;
        KScope ks(ctx, st, KK_FILTER, flops, (double)nf * NBIN * (8.0 + 4.0));
        if (nf * (NFFT / 2048) >= 152) {  // enough filters to fill the GPU with 2048-point transforms
            constexpr int L = 2048, P = NFFT / L;
            k_fb_inverse<L><<<dim3(P / 4 + 1, (unsigned)nf), FB_T, 0, st>>>(psd, (double)ctx->cfg.fs,
                                                                        ctx->cfg.f_highpass, ctx->tw64, Z);
            k_fb_taper<<<dim3(FB_LAGS / FB_T, (unsigned)nf), FB_T, 0, st>>>(Z, ctx->taper64, ctx->tw64, Y);
            k_fb_forward<L><<<dim3(P / 4 + 1, (unsigned)nf), FB_T, 0, st>>>(Y, ctx->tw64, gains);
        } else {  // few filters: 32 sub-transforms of 512 points each (16 paired transforms per stage)
            constexpr int L = 512, P = NFFT / L;
            k_fb_inverse<L><<<dim3(P / 4 + 1, (unsigned)nf), FB_T, 0, st>>>(psd, (double)ctx->cfg.fs,
                                                                        ctx->cfg.f_highpass, ctx->tw64, Z);
            k_fb_taper_fold<<<dim3(L / FB_FS, (unsigned)nf), FB_FS * 4, 0, st>>>(Z, ctx->taper64, ctx->tw64, Y);
            k_fb_forward<L><<<dim3(P / 4 + 1, (unsigned)nf), FB_T, 0, st>>>(Y, ctx->tw64, gains);
        }
    } else {
        KScope ks(ctx, st, KK_FILTER, flops, (double)nf * NBIN * (8.0 + 4.0));
        k_filter_build<<<dim3((unsigned)n_psd, n_det), NT64, (NC + 1) * sizeof(double2), st>>>(
            psd, n_psd, (double)ctx->cfg.fs, ctx->cfg.f_highpass, ctx->cfg.fir_len, ctx->tw64, gains);
    }
    AFG_LAUNCH_CHECK(ctx, "filter build");
    return AFG_OK;
}

// Fill the FP32 twiddle table of the current device once per process (it is a per-module device variable;
// every context on the device and the context-free Welch entry point share it).  Synchronous: the table is
// complete when this returns, before any transform can be launched on the device.
static cudaError_t ensure_tw32() {
    static std::mutex mu;
    static bool done[256] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    cudaStream_t st;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return e;
    k_tw32<<<(r16::TW_TOTAL + 255) / 256, 256, 0, st>>>();
    e = cudaGetLastError();
    const cudaError_t e2 = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

int afg_make_twiddles(afg_ctx *ctx) {
    {
        KScope ks(ctx, 0, KK_TWIDDLES, 0.0, (double)NFFT * sizeof(double2));
        k_twiddles<<<NFFT / 256, 256>>>(ctx->tw64);
        if (ctx->cfg.fir_len <= FILTER_LAGS)
            k_taper64<<<FILTER_LAGS / 256, 256>>>(ctx->taper64, (double)ctx->cfg.fs, ctx->cfg.fir_len);
    }
    AFG_LAUNCH_CHECK(ctx, "k_twiddles");
    if (ensure_tw32() != cudaSuccess) return AFG_ERR_CUDA;
    return set_attrs(ctx);
}

int launch_psd(afg_ctx *ctx, const float *x, int64_t n, int n_det, int64_t n_psd, int64_t psd_step,
               int64_t psd_span, double *psd, cudaStream_t st, int64_t x_stride) {
    if (x_stride <= 0) x_stride = n;
    const int hop = ctx->cfg.hop;
    const int64_t K = (psd_span - NFFT) / hop + 1;
    const int64_t seg_step = n_psd > 1 ? psd_step / hop : 0;
    const int64_t n_seg = (n_psd - 1) * seg_step + K;
    double *P = nullptr;
    int rc = afg_ws_reserve(ctx, WS_PERIODOGRAM, (size_t)n_det * n_seg * NBIN * sizeof(double), (void **)&P);
    if (rc) return rc;
    if (n_seg > 0x7fffffff) return afg_fail(ctx, AFG_ERR_ARG, "psd_estimate: too many segments");
    {
        // one read of every segment, one FP64 periodogram written per segment
        KScope ks(ctx, st, KK_PERIODOGRAM, 0.0, (double)n_det * n_seg * (NFFT * 4.0 + NBIN * 8.0));
        k_periodogram<<<dim3((unsigned)n_seg, n_det), r16::NT, WELCH_SMEM, st>>>(x, x_stride, hop, P, n_seg, nullptr,
                                                                                 psd_scale(K, ctx->cfg.fs));
    }
    AFG_LAUNCH_CHECK(ctx, "k_periodogram");
    {
        KScope ks(ctx, st, KK_PSD_MEAN, 0.0, (double)n_det * (n_seg + n_psd) * NBIN * 8.0);
        k_psd_mean<<<dim3((NBIN + 255) / 256, (unsigned)((n_psd + PSD_EPT - 1) / PSD_EPT), n_det), 256, 0, st>>>(
            P, n_seg, (int)seg_step, (int)K, psd, n_psd);
    }
    AFG_LAUNCH_CHECK(ctx, "k_psd_mean");
    return AFG_OK;
}

int launch_whiten(afg_ctx *ctx, const float *x, int64_t n, int n_det, const double *psd, int64_t n_psd,
                  int64_t out_first, int64_t out_len, int64_t epoch_len, float *y, int64_t y_stride,
                  cudaStream_t st, int64_t x_stride) {
    if (x_stride <= 0) x_stride = n;
    float *gains = nullptr;
    int rc = afg_ws_reserve(ctx, WS_FILTER, (size_t)n_det * n_psd * NBIN * sizeof(float), (void **)&gains);
    if (rc) return rc;
    rc = filter_build(ctx, psd, n_det, n_psd, gains, st);
    if (rc) return rc;
    if (out_len <= 0) return AFG_OK;
    const WhitenLayout wl = whiten_layout(out_len, epoch_len, ctx->cfg.fir_len);
    const int64_t n_ep = wl.bpe > 0 ? wl.n_blocks / wl.bpe : 0;
    const int64_t nb = n_ep * (wl.small_rem ? wl.n_full : wl.bpe);
    if (nb > 0x7fffffff) return afg_fail(ctx, AFG_ERR_ARG, "whiten: too many blocks");
    {
        // algorithmic: read the cropped span once, write the output once, read the gains
        const double F = ctx->cfg.fir_len;
        KScope ks(ctx, st, KK_WHITEN, 0.0, (double)n_det * ((2.0 * out_len + F - 1.0) * 4.0 + n_psd * NBIN * 4.0));
        if (nb > 0)
            k_whiten<<<dim3((unsigned)nb, n_det), r16::NT, WHITEN_SMEM, st>>>(x, n, x_stride, gains, n_psd, out_first,
                                                                              out_len, epoch_len, ctx->cfg.fir_len, y,
                                                                              y_stride);
    }
    AFG_LAUNCH_CHECK(ctx, "k_whiten");
    if (wl.small_rem && n_ep > 0) {
        KScope ks(ctx, st, KK_WHITEN, 0.0, 0.0);  // (the bytes are counted with the launch above)
        k_whiten_rem<<<dim3((unsigned)n_ep, n_det), r16::NT_S, WHITEN_SMEM_S, st>>>(
            x, n, x_stride, gains, n_psd, out_first, out_len, epoch_len, ctx->cfg.fir_len, y, y_stride);
    }
    AFG_LAUNCH_CHECK(ctx, "k_whiten_rem");
    return AFG_OK;
}

bool whiten_multi_takes_staging(const afg_ctx *ctx) { return whiten_piece_max_s(ctx->cfg.fir_len) != 0; }

// Most outputs one piece of launch_whiten_multi may hold.
int whiten_multi_piece_max(const afg_ctx *ctx) {
    const int m = whiten_piece_max_s(ctx->cfg.fir_len);
    return m ? m : WB;
}

// Filter build only: gains [n_det][n_psd][NBIN] from psd (FP64), on st.
int launch_filter(afg_ctx *ctx, const double *psd, int n_det, int64_t n_psd, float *gains, cudaStream_t st) {
    return filter_build(ctx, psd, n_det, n_psd, gains, st);
}

// One PSD per row of psd_span samples, row r starting at rows_dev[r] (device array of n_rows
// pointers): the Welch periodograms of all rows in one launch and their means in another, into
// psd [n_rows][NBIN].  The same kernels and arithmetic as launch_psd with n_psd = 1.
int launch_psd_rows(afg_ctx *ctx, const float *const *rows_dev, int n_rows, int64_t psd_span, double *psd,
                    cudaStream_t st) {
    if (n_rows <= 0) return AFG_OK;
    const int hop = ctx->cfg.hop;
    const int64_t K = (psd_span - NFFT) / hop + 1;
    double *P = nullptr;
    int rc = afg_ws_reserve(ctx, WS_PERIODOGRAM, (size_t)n_rows * K * NBIN * sizeof(double), (void **)&P);
    if (rc) return rc;
    {
        KScope ks(ctx, st, KK_PERIODOGRAM, 0.0, (double)n_rows * K * (NFFT * 4.0 + NBIN * 8.0));
        k_periodogram<<<dim3((unsigned)K, (unsigned)n_rows), r16::NT, WELCH_SMEM, st>>>(nullptr, 0, hop, P, K,
                                                                                        rows_dev, psd_scale(K, ctx->cfg.fs));
    }
    AFG_LAUNCH_CHECK(ctx, "k_periodogram");
    {
        KScope ks(ctx, st, KK_PSD_MEAN, 0.0, (double)n_rows * (K + 1) * NBIN * 8.0);
        k_psd_mean<<<dim3((NBIN + 255) / 256, 1, (unsigned)n_rows), 256, 0, st>>>(P, K, 0, (int)K, psd, 1);
    }
    AFG_LAUNCH_CHECK(ctx, "k_psd_mean");
    return AFG_OK;
}

// grid (n_rows): row r of src [n_rows][len] to dst_dev[r] (device array of n_rows pointers)
__global__ void k_scatter_rows(const float *__restrict__ src, float *const *__restrict__ dst, int len) {
    const float *s = src + (int64_t)blockIdx.x * len;
    float *d = dst[blockIdx.x];
    for (int i = threadIdx.x; i < len; i += blockDim.x) d[i] = s[i];
}

int launch_scatter_rows(afg_ctx *ctx, const float *src, float *const *dst_dev, int n_rows, int len, cudaStream_t st) {
    if (n_rows <= 0) return AFG_OK;
    k_scatter_rows<<<n_rows, 256, 0, st>>>(src, dst_dev, len);
    AFG_LAUNCH_CHECK(ctx, "k_scatter_rows");
    return AFG_OK;
}

int launch_whiten_multi(afg_ctx *ctx, const WhitenPiece *pieces_dev, int n_pieces, int64_t total_out,
                        cudaStream_t st) {
    if (n_pieces <= 0) return AFG_OK;
    const double F = ctx->cfg.fir_len;
    KScope ks(ctx, st, KK_WHITEN, 0.0, 2.0 * ((2.0 * total_out + n_pieces * (F - 1.0)) * 4.0 + n_pieces * NBIN * 4.0));
    if (whiten_piece_max_s(ctx->cfg.fir_len))  // pieces were cut to the 4096-point block
        AFG_CUDA(ctx, launch_pdl(k_whiten_multi_s, dim3((unsigned)n_pieces, 2), dim3(r16::NT_S), WHITEN_SMEM_S, st,
                                 pieces_dev, ctx->cfg.fir_len));
    else
        AFG_CUDA(ctx, launch_pdl(k_whiten_multi, dim3((unsigned)n_pieces, 2), dim3(r16::NT), WHITEN_SMEM, st,
                                 pieces_dev, ctx->cfg.fir_len));
    return AFG_OK;
}

// The Welch kernels on caller-provided scratch and twiddles (no workspace,
// no context, no accounting).  P must hold n_det * n_seg * NBIN doubles.
cudaError_t launch_psd_on(const float *x, int64_t n, int n_det, int64_t n_psd, int64_t psd_step, int64_t psd_span,
                          int hop, int fs, double *P, double *psd, cudaStream_t st) {
    const int64_t K = (psd_span - NFFT) / hop + 1;
    const int64_t seg_step = n_psd > 1 ? psd_step / hop : 0;
    const int64_t n_seg = (n_psd - 1) * seg_step + K;
    k_periodogram<<<dim3((unsigned)n_seg, n_det), r16::NT, WELCH_SMEM, st>>>(x, n, hop, P, n_seg, nullptr,
                                                                             psd_scale(K, fs));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_psd_mean<<<dim3((NBIN + 255) / 256, (unsigned)((n_psd + PSD_EPT - 1) / PSD_EPT), n_det), 256, 0, st>>>(
        P, n_seg, (int)seg_step, (int)K, psd, n_psd);
    return cudaGetLastError();
}

// Fill the twiddle table and opt the periodogram kernel into its 68 KiB of dynamic shared memory on the
// current device.
cudaError_t prepare_psd_kernels() {
    const cudaError_t e = ensure_tw32();
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_periodogram, cudaFuncAttributeMaxDynamicSharedMemorySize, WELCH_SMEM);
}
