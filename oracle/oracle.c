/*
 * oracle.c -- plain FP64 CPU oracle for the Aframe detection path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; it exists so that tests, the package smoke check and the
 * CPU baseline of the benchmark can compare the CUDA library against a slow,
 * obviously correct statement of what the path computes.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * Every routine follows a definition of the paper (arXiv 2403.18661):
 *   Welch PSD + whitening filter + whitening, 0.5 s crop .. Sec. IV, "Noise
 *                                                           sampling", Sec. VI
 *   1D ResNet34 with GroupNorm, scalar output ............. Sec. II, Sec. IX
 *   1 s top-hat integration, 8 s max clustering ........... Sec. II
 *   sliding windows (4 Hz, 1.5 s) ......................... Sec. II, Sec. VI
 *   timeslides (L1 shifted in 1 s steps) .................. Sec. IX
 * Readings of points the paper leaves open are stated beside each routine.
 *
 * Double precision throughout.  OpenMP (if enabled) only splits independent
 * windows / outputs across threads; it never changes an operation order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* FFT: iterative radix-2 decimation in time, complex double, in place.      */
/* X_k = sum_n x_n exp(sign * 2 pi i k n / N), no normalisation.            */
/* Returns -1 if n is not a power of two.                                    */
/* ------------------------------------------------------------------------ */
int orc_fft(double *re, double *im, int64_t n, int sign) {
    if (n < 1 || (n & (n - 1)) != 0) return -1;
    /* bit-reversal permutation */
    for (int64_t i = 1, j = 0; i < n; ++i) {
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    /* twiddles w_k = exp(sign 2 pi i k / n), k < n/2, each from cos/sin directly */
    int64_t half = n / 2;
    double *wr = (double *)malloc(sizeof(double) * (size_t)(half > 0 ? half : 1));
    double *wi = (double *)malloc(sizeof(double) * (size_t)(half > 0 ? half : 1));
    for (int64_t k = 0; k < half; ++k) {
        double a = 2.0 * ORC_PI * (double)k / (double)n;
        wr[k] = cos(a);
        wi[k] = sign * sin(a);
    }
    for (int64_t len = 2; len <= n; len <<= 1) {
        int64_t h = len / 2, step = n / len;
        for (int64_t s = 0; s < n; s += len) {
            for (int64_t k = 0; k < h; ++k) {
                double c = wr[k * step], d = wi[k * step];
                double xr = re[s + k + h], xi = im[s + k + h];
                double tr = xr * c - xi * d, ti = xr * d + xi * c;
                re[s + k + h] = re[s + k] - tr;
                im[s + k + h] = im[s + k] - ti;
                re[s + k] += tr;
                im[s + k] += ti;
            }
        }
    }
    free(wr);
    free(wi);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Welch one-sided PSD density (Sec. IV ("Noise sampling"): "the first 8 s is used to        */
/* estimate the power spectral density"; Sec. VI: "the first 64 seconds").  */
/* Readings: segments of nfft samples every hop samples (K = (n-nfft)/hop+1),*/
/* periodic Hann window w_j = 1/2 - 1/2 cos(2 pi j / nfft), no detrending,   */
/* mean over segments, density scaling 1/(fs sum w^2), one-sided doubling of */
/* every bin except DC and Nyquist.                                          */
/* psd has nfft/2+1 entries.  Returns the number of segments, or -1.         */
/* ------------------------------------------------------------------------ */
int orc_welch(const double *x, int64_t n, int nfft, int hop, double fs, double *psd) {
    if (nfft < 2 || hop < 1 || n < nfft) return -1;
    int64_t K = (n - nfft) / hop + 1;
    int nb = nfft / 2 + 1;
    double *w = (double *)malloc(sizeof(double) * (size_t)nfft);
    double *re = (double *)malloc(sizeof(double) * (size_t)nfft);
    double *im = (double *)malloc(sizeof(double) * (size_t)nfft);
    double s2 = 0.0;
    for (int j = 0; j < nfft; ++j) {
        w[j] = 0.5 - 0.5 * cos(2.0 * ORC_PI * (double)j / (double)nfft);
        s2 += w[j] * w[j];
    }
    for (int k = 0; k < nb; ++k) psd[k] = 0.0;
    for (int64_t s = 0; s < K; ++s) {
        const double *seg = x + s * hop;
        for (int j = 0; j < nfft; ++j) { re[j] = w[j] * seg[j]; im[j] = 0.0; }
        if (orc_fft(re, im, nfft, -1) != 0) { K = -1; break; }
        for (int k = 0; k < nb; ++k) psd[k] += re[k] * re[k] + im[k] * im[k];
    }
    if (K > 0) {
        for (int k = 0; k < nb; ++k) {
            double onesided = (k == 0 || k == nfft / 2) ? 1.0 : 2.0;
            psd[k] = onesided * psd[k] / ((double)K * fs * s2);
        }
    }
    free(w); free(re); free(im);
    return (int)K;
}

/* ------------------------------------------------------------------------ */
/* Inverse-ASD whitening filter (Sec. IV, "Noise sampling": "filter construction"; 1 s FIR,  */
/* 32 Hz highpass).  Readings:                                              */
/*   A_k = psd_k^{-1/2} for k*fs/nfft >= f_hp, else 0 (hard highpass);      */
/*   h_m = (1/nfft) sum_k A_k e^{+2 pi i k m / nfft}  (real, even: the      */
/*         zero-phase inverse DFT of the amplitude response on the nfft grid);*/
/*   g_m = sqrt(2/fs) h_m (1/2 - 1/2 cos(2 pi (m + F/2) / F)),              */
/*         m in [-F/2, F/2), F = fir_len (periodic Hann taper).             */
/* The sqrt(2/fs) factor makes white input of PSD S produce unit variance.  */
/* taps[j] holds g_{j - F/2}.  Returns 0, or -1 on bad arguments.            */
/* ------------------------------------------------------------------------ */
int orc_whitening_taps(const double *psd, int nfft, double fs, double f_hp, int fir_len, double *taps) {
    if (nfft < 2 || (nfft & (nfft - 1)) || fir_len < 2 || fir_len > nfft || (fir_len & 1)) return -1;
    double *re = (double *)malloc(sizeof(double) * (size_t)nfft);
    double *im = (double *)malloc(sizeof(double) * (size_t)nfft);
    int nb = nfft / 2 + 1;
    for (int k = 0; k < nb; ++k) {
        double f = (double)k * fs / (double)nfft;
        double a = (f >= f_hp && psd[k] > 0.0) ? 1.0 / sqrt(psd[k]) : 0.0;
        re[k] = a;
        im[k] = 0.0;
        if (k > 0 && k < nfft / 2) { re[nfft - k] = a; im[nfft - k] = 0.0; }
    }
    int rc = orc_fft(re, im, nfft, +1);
    if (rc == 0) {
        int half = fir_len / 2;
        for (int j = 0; j < fir_len; ++j) {
            int m = j - half;
            int64_t idx = m >= 0 ? m : (int64_t)nfft + m;
            double h = re[idx] / (double)nfft;
            double taper = 0.5 - 0.5 * cos(2.0 * ORC_PI * (double)j / (double)fir_len);
            taps[j] = sqrt(2.0 / fs) * h * taper;
        }
    }
    free(re); free(im);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Whitening as a direct linear FIR (Sec. IV ("Noise sampling"): whitened, transformed back, */
/* 0.5 s corrupted on both ends and removed).                                */
/* y_j = sum_{i=0}^{F-1} taps[i] * x[first + j - (i - F/2)],  j in [0,len). */
/* Requires first >= F/2 and first + len - 1 + F/2 - 1 < n, so that the      */
/* support of every output lies inside x (the "crop").  Returns 0 or -1.     */
/* ------------------------------------------------------------------------ */
int orc_fir(const double *x, int64_t n, const double *taps, int fir_len, int64_t first, int64_t len, double *y) {
    int half = fir_len / 2;
    if (first < half || first + len - 1 + (half - 1) >= n) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < len; ++j) {
        double acc = 0.0;
        int64_t c = first + j;
        for (int i = 0; i < fir_len; ++i) acc += taps[i] * x[c - (i - half)];
        y[j] = acc;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Network layers (Sec. II: ResNet34 with 1D convolutions and GroupNorm;    */
/* Sec. IX: kernel length 3, global pooling).                                */
/* Tensors are [C][L] row-major.                                             */
/* ------------------------------------------------------------------------ */

/* out[co][t] = sum_ci sum_r w[co][ci][r] * in[ci][t*stride + r - pad], zero outside [0,L) */
void orc_conv1d(const double *in, int cin, int L, const double *w, int cout, int k, int stride, int pad,
                double *out, int Lout) {
    for (int co = 0; co < cout; ++co) {
        double *o = out + (int64_t)co * Lout;
        for (int t = 0; t < Lout; ++t) o[t] = 0.0;
        for (int ci = 0; ci < cin; ++ci) {
            const double *src = in + (int64_t)ci * L;
            for (int r = 0; r < k; ++r) {
                double wv = w[((int64_t)co * cin + ci) * k + r];
                for (int t = 0; t < Lout; ++t) {
                    int64_t s = (int64_t)t * stride + r - pad;
                    if (s >= 0 && s < L) o[t] += wv * src[s];
                }
            }
        }
    }
}

/* GroupNorm (Wu & He): per group of C/G channels, mean and biased variance  */
/* over (channels in group) x L, y = (x - mu)/sqrt(var + eps) * gamma_c + beta_c. */
void orc_group_norm(double *x, int C, int L, int G, const double *gamma, const double *beta, double eps) {
    int cg = C / G;
    for (int g = 0; g < G; ++g) {
        double *base = x + (int64_t)g * cg * L;
        int64_t cnt = (int64_t)cg * L;
        double mu = 0.0;
        for (int64_t i = 0; i < cnt; ++i) mu += base[i];
        mu /= (double)cnt;
        double var = 0.0;
        for (int64_t i = 0; i < cnt; ++i) { double d = base[i] - mu; var += d * d; }
        var /= (double)cnt;
        double inv = 1.0 / sqrt(var + eps);
        for (int c = 0; c < cg; ++c) {
            int cc = g * cg + c;
            double *row = base + (int64_t)c * L;
            for (int t = 0; t < L; ++t) row[t] = (row[t] - mu) * inv * gamma[cc] + beta[cc];
        }
    }
}

static void relu(double *x, int64_t n) {
    for (int64_t i = 0; i < n; ++i) if (x[i] < 0.0) x[i] = 0.0;
}

/* max-pool k3 s2 p1; padding never wins (PyTorch semantics) */
static void maxpool3s2(const double *in, int C, int L, double *out, int Lout) {
    for (int c = 0; c < C; ++c)
        for (int t = 0; t < Lout; ++t) {
            double m = -INFINITY;
            for (int r = 0; r < 3; ++r) {
                int s = 2 * t + r - 1;
                if (s >= 0 && s < L && in[(int64_t)c * L + s] > m) m = in[(int64_t)c * L + s];
            }
            out[(int64_t)c * Lout + t] = m;
        }
}

/* Network description: spec[] = {in_ch, stem_k, stem_stride, stem_pool, groups,
 * n_stages, width_0..width_{n-1}, blocks_0..blocks_{n-1}}.  Weight layout: stem.w
 * [C0][in][k], stem gamma, beta; per block c1.w [C][Cin][3], g1 gamma, beta, c2.w
 * [C][C][3], g2 gamma, beta, and for a block that changes stride or width
 * sc.w [C][Cin][1], gsc gamma, beta; then fc.w [C_last], fc.b. */
typedef struct { const double *p; } wcursor;
static const double *take(wcursor *c, int64_t n) { const double *r = c->p; c->p += n; return r; }

static int conv_len(int L, int k, int s, int p) { return (L + 2 * p - k) / s + 1; }

/* One window x [in_ch][W] -> logit.  Scratch-free: allocates its own buffers. */
int orc_network(const int *spec, double eps, const double *weights, const double *x, int W, double *logit) {
    int in_ch = spec[0], stem_k = spec[1], stem_s = spec[2], stem_pool = spec[3], G = spec[4], ns = spec[5];
    const int *widths = spec + 6, *blocks = spec + 6 + ns;
    int cmax = in_ch;
    for (int s = 0; s < ns; ++s) if (widths[s] > cmax) cmax = widths[s];
    int64_t cap = (int64_t)cmax * W;
    double *a = (double *)calloc((size_t)cap, sizeof(double));
    double *b = (double *)calloc((size_t)cap, sizeof(double));
    double *c = (double *)calloc((size_t)cap, sizeof(double));
    double *d = (double *)calloc((size_t)cap, sizeof(double));
    if (!a || !b || !c || !d) { free(a); free(b); free(c); free(d); return -1; }
    wcursor wc = { weights };

    /* stem */
    int C = widths[0];
    int L = conv_len(W, stem_k, stem_s, stem_k / 2);
    const double *sw = take(&wc, (int64_t)C * in_ch * stem_k);
    const double *sg = take(&wc, C), *sb = take(&wc, C);
    orc_conv1d(x, in_ch, W, sw, C, stem_k, stem_s, stem_k / 2, a, L);
    orc_group_norm(a, C, L, G, sg, sb, eps);
    relu(a, (int64_t)C * L);
    if (stem_pool) {
        int Lp = conv_len(L, 3, 2, 1);
        maxpool3s2(a, C, L, b, Lp);
        memcpy(a, b, sizeof(double) * (size_t)C * Lp);
        L = Lp;
    }
    /* stages of BasicBlocks: out = relu(gn2(conv2(relu(gn1(conv1(x))))) + shortcut(x)) */
    int cin = C;
    for (int s = 0; s < ns; ++s) {
        for (int bi = 0; bi < blocks[s]; ++bi) {
            int stride = (s > 0 && bi == 0) ? 2 : 1;
            int width = widths[s];
            int Lo = conv_len(L, 3, stride, 1);
            const double *w1 = take(&wc, (int64_t)width * cin * 3);
            const double *g1 = take(&wc, width), *b1 = take(&wc, width);
            const double *w2 = take(&wc, (int64_t)width * width * 3);
            const double *g2 = take(&wc, width), *b2 = take(&wc, width);
            orc_conv1d(a, cin, L, w1, width, 3, stride, 1, b, Lo);
            orc_group_norm(b, width, Lo, G, g1, b1, eps);
            relu(b, (int64_t)width * Lo);
            orc_conv1d(b, width, Lo, w2, width, 3, 1, 1, c, Lo);
            orc_group_norm(c, width, Lo, G, g2, b2, eps);
            if (stride != 1 || cin != width) {
                const double *ws = take(&wc, (int64_t)width * cin);
                const double *gs = take(&wc, width), *bs = take(&wc, width);
                orc_conv1d(a, cin, L, ws, width, 1, stride, 0, d, Lo);
                orc_group_norm(d, width, Lo, G, gs, bs, eps);
            } else {
                memcpy(d, a, sizeof(double) * (size_t)width * Lo);
            }
            for (int64_t i = 0; i < (int64_t)width * Lo; ++i) {
                double v = c[i] + d[i];
                a[i] = v > 0.0 ? v : 0.0;
            }
            cin = width;
            L = Lo;
        }
    }
    /* global average pool + linear head */
    const double *fw = take(&wc, cin), *fb = take(&wc, 1);
    double z = fb[0];
    for (int ch = 0; ch < cin; ++ch) {
        double m = 0.0;
        for (int t = 0; t < L; ++t) m += a[(int64_t)ch * L + t];
        z += fw[ch] * (m / (double)L);
    }
    *logit = z;
    free(a); free(b); free(c); free(d);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sliding windows over whitened two-detector data (Sec. II, Sec. VI:      */
/* windows shifted by the inference stride) with an optional timeslide      */
/* (Sec. IX: H1 fixed, L1 shifted).  Window j:                              */
/*   det 0 samples y0[first + j*stride + t]                                 */
/*   det 1 samples y1[(first + j*stride + shift + t) mod n_y]  (circular)   */
/* for t in [0, W).  logits[j] = network(window j).                          */
/* ------------------------------------------------------------------------ */
int orc_infer_windows(const int *spec, double eps, const double *weights, const double *y0, const double *y1,
                      int64_t n_y, int W, int64_t first, int64_t stride, int64_t n_win, int64_t shift,
                      double *logits) {
    if (first < 0 || first + (n_win - 1) * stride + W > n_y) return -1;
    int in_ch = spec[0];
    if (in_ch != 2) return -1;
    int err = 0;
#pragma omp parallel
    {
        double *x = (double *)malloc(sizeof(double) * 2 * (size_t)W);
#pragma omp for schedule(dynamic, 1)
        for (int64_t j = 0; j < n_win; ++j) {
            int64_t s0 = first + j * stride;
            for (int t = 0; t < W; ++t) {
                x[t] = y0[s0 + t];
                int64_t i1 = (s0 + shift + t) % n_y;
                if (i1 < 0) i1 += n_y;
                x[W + t] = y1[i1];
            }
            if (orc_network(spec, eps, weights, x, W, &logits[j]) != 0) err = 1;
        }
        free(x);
    }
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Integration: 1 s top-hat (Sec. II).  Reading: causal, "valid" mode,       */
/* I_j = (1/n_int) sum_{i=0}^{n_int-1} z_{j+i}, j in [0, n - n_int], stamped */
/* at the newest window (index j + n_int - 1).                               */
/* ------------------------------------------------------------------------ */
int orc_integrate(const double *z, int64_t n, int n_int, double *out) {
    if (n_int < 1 || n < n_int) return -1;
    for (int64_t j = 0; j + n_int <= n; ++j) {
        double s = 0.0;
        for (int i = 0; i < n_int; ++i) s += z[j + i];
        out[j] = s / (double)n_int;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Clustering (Sec. II: the maximum integrated value over an 8 s window).   */
/* Reading: j is a trigger iff I_j >= I_i for every |i - j| <= half and      */
/* I_j > I_i for every i in [j - half, j) (ties go to the earliest index).   */
/* Writes trigger indices in increasing order; returns their number (or the */
/* number found if more than cap; only cap are written).                    */
/* ------------------------------------------------------------------------ */
int64_t orc_triggers(const double *I, int64_t n, int half, int64_t *idx, int64_t cap) {
    int64_t cnt = 0;
    for (int64_t j = 0; j < n; ++j) {
        int ok = 1;
        for (int64_t i = j - half; i <= j + half && ok; ++i) {
            if (i < 0 || i >= n || i == j) continue;
            if (i < j ? !(I[j] > I[i]) : !(I[j] >= I[i])) ok = 0;
        }
        if (ok) {
            if (cnt < cap) idx[cnt] = j;
            ++cnt;
        }
    }
    return cnt;
}
