/*
 * aframe_gb.h -- C ABI of the GB300 (sm_103a) detection path of Aframe
 * (Marx et al., "A machine-learning pipeline for real-time detection of
 * gravitational waves from compact binary coalescences", arXiv 2403.18661).
 *
 * The path (Sec. II, Sec. IV, "Noise sampling" paragraph, Sec. VI "Inference"):
 *   two-detector strain --Welch PSD--> inverse-ASD whitening filter -->
 *   FFT-domain whitening with 0.5 s crop --> overlapping 1.5 s windows -->
 *   1D ResNet with GroupNorm (one logit per window) --> 1 s top-hat
 *   integration --> maxima over 8 s (triggers).
 *
 * Conventions shared by every entry point
 *   - Every call returns an int status: AFG_OK (0) or a negative AFG_ERR_*.
 *     A failed call leaves its outputs unspecified and records a message
 *     that afg_last_error() returns until the next call on the same context.
 *   - Array arguments are DEVICE pointers (CUDA global memory of the
 *     context's device) owned by the caller, unless the name ends in _host.
 *     The library never frees caller memory.  It owns only its context:
 *     weights, twiddle tables and workspaces, released by afg_ctx_destroy.
 *   - Compute calls are asynchronous on the given stream (a cudaStream_t
 *     passed as void*; NULL is the legacy default stream) and may be
 *     captured in a CUDA graph once the context's workspaces have grown to
 *     the sizes the captured calls need (make one uncaptured call first).
 *     Calls that return values through host pointers synchronise the stream.
 *   - Strain arrays are row-major [n_det][n] float32 (H1 = row 0, L1 = row 1),
 *     sampled at cfg.fs.  Sizes are in samples.
 *   - A context is not thread-safe: serialise calls that share one.
 */
#ifndef AFRAME_GB_H
#define AFRAME_GB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define AFG_OK 0
#define AFG_ERR_ARG (-1)         /* invalid argument (size, pointer, layout) */
#define AFG_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define AFG_ERR_OOM (-3)         /* device allocation failed */
#define AFG_ERR_BUDGET (-4)      /* refused: would exceed the context's HBM budget */
#define AFG_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up */
#define AFG_ERR_STATE (-6)       /* call not valid in the current state */
#define AFG_ERR_NAN (-7)         /* non-finite input detected */
#define AFG_ERR_UNSUPPORTED (-8) /* configuration this build does not implement */

/* precision of the network's convolutions */
#define AFG_FP32 0 /* FP32 SIMT implicit-GEMM convolutions ("plain") */
#define AFG_BF16 1 /* BF16 operands, FP32 accumulation on tcgen05 tensor cores */

typedef struct afg_ctx afg_ctx;

/* 1D ResNet with GroupNorm (Sec. II: ResNet34 with 1D convolutions and GN;
 * Sec. IX: kernel length 3, global pooling).
 * stem: conv(in_ch -> widths[0], kernel stem_k, stride stem_stride, padding
 * stem_k/2) + GN + ReLU, then max-pool(3, stride 2, padding 1) if stem_pool.
 * n_stages stages; stage s holds blocks[s] BasicBlocks of width widths[s]:
 * out = ReLU(GN(conv3(ReLU(GN(conv3(x))))) + shortcut(x)); the first block of
 * stages s > 0 has stride 2 in its first conv and a 1x1 stride-2 conv + GN
 * shortcut (also used whenever the width changes).  Head: mean over time,
 * then linear(widths[n_stages-1] -> 1) + bias; the output is the raw logit.
 * All convolutions are bias-free with zero padding at window edges. */
typedef struct afg_net {
    int32_t in_ch;       /* must be 2 (H1, L1) */
    int32_t stem_k;      /* odd, <= 7 */
    int32_t stem_stride; /* 1 or 2 */
    int32_t stem_pool;   /* 0 or 1 */
    int32_t groups;      /* GroupNorm groups; divides every width */
    int32_t n_stages;    /* 1..4 */
    int32_t widths[4];   /* powers of two in [16, 512] */
    int32_t blocks[4];   /* >= 1 */
    float eps;           /* GroupNorm epsilon */
} afg_net;

typedef struct afg_config {
    int32_t fs;         /* sample rate (Hz), Sec. IV.A: 2048 */
    int32_t nfft;       /* Welch segment length; this build: 16384 (8 s) */
    int32_t hop;        /* Welch hop (50 % overlap: nfft/2); divides nfft */
    int32_t fir_len;    /* whitening FIR length F (1 s = fs), even, <= 8192 */
    double f_highpass;  /* whitening highpass (Hz), 32 */
    int32_t win_len;    /* network window length W (1.5 s = 3072), multiple of 32 */
    int32_t precision;  /* AFG_FP32 or AFG_BF16 */
    int64_t hbm_budget; /* bytes the context may hold on the device; 0 = no limit */
    afg_net net;
} afg_config;

/* Window-level parameters of one analysis span (see afg_analyze). */
typedef struct afg_run_params {
    int64_t n_raw;        /* raw samples per detector in x */
    int64_t epoch_len;    /* 0: plain mode; else PSD epoch length in samples */
    int64_t psd_len;      /* epoch mode: PSD look-back span in samples */
    int64_t stride;       /* window stride S (fs / inference rate) */
    int64_t n_win;        /* windows to analyse */
    int64_t shift;        /* L1 timeslide shift in samples (0 = zero lag) */
    int32_t n_int;        /* integration length in windows (1 s * rate) */
    int32_t cluster_half; /* trigger half-width in statistic samples (4 s * rate) */
} afg_run_params;

/* ---------------------------------------------------------------- context */

/* Library version string (static storage). */
const char *afg_version(void);

/* Human-readable name of a status code (static storage). */
const char *afg_status_string(int status);

/* Number of float32 weights the network `net` takes (flat layout below).
 * Returns AFG_ERR_ARG for an invalid description.
 * Flat layout, in order: stem.w [C0][in_ch][stem_k], stem.gamma [C0],
 * stem.beta [C0]; per block c1.w [C][Cin][3], g1.gamma [C], g1.beta [C],
 * c2.w [C][C][3], g2.gamma, g2.beta, and for a downsampling block
 * sc.w [C][Cin][1], gsc.gamma, gsc.beta; finally fc.w [C_last], fc.b [1]. */
int afg_weights_count(const afg_net *net, int64_t *n_out);

/* Create a context on the current CUDA device: validates cfg, copies the
 * weights (host, n_weights float32 in the flat layout) to the device in the
 * library's own layouts and builds the FFT twiddle tables.  Synchronous.
 * *out receives the context (NULL on failure). */
int afg_ctx_create(const afg_config *cfg, const float *weights_host, int64_t n_weights, afg_ctx **out);

/* Release every device resource of the context.  Waits for its work. */
int afg_ctx_destroy(afg_ctx *ctx);

/* Message of the last failed call on ctx ("" if none); valid until the next call. */
const char *afg_last_error(const afg_ctx *ctx);

/* Device bytes currently held by the context (weights + workspaces + streams). */
int afg_ctx_bytes(const afg_ctx *ctx, int64_t *bytes);

/* Wait for the work queued on `stream`, then report device-side failures
 * the library's kernels recorded since the last call: AFG_ERR_TIMEOUT if a
 * bounded wait inside a kernel gave up (that kernel returned early and its
 * outputs are unspecified).  Clears the record. */
int afg_sync(afg_ctx *ctx, void *stream);

/* Check of the bounded device-side waits (failure detection; the paper has no
 * counterpart: it concerns this library's kernels, not the method).  The
 * tensor-core kernels wait on mbarriers for their MMAs and bulk copies, each
 * wait limited in time; when one gives up, the kernel records it, returns
 * early (its outputs are then unspecified) and afg_sync reports
 * AFG_ERR_TIMEOUT.  This call exercises that path without a fault: n_blocks
 * CTAs each wait, through the same bounded wait and the same record, on an
 * mbarrier that nothing arrives on, so every wait ends by its limit
 * (limit_ns, at most 1e10) with nothing in flight, and the kernel exits
 * normally.  waited_ns: device int64 [n_blocks], the time each CTA waited.
 * Asynchronous on `stream`; call afg_sync(ctx, stream) to read the result
 * (AFG_ERR_TIMEOUT, which also clears the record).  The context stays
 * usable.  Errors: AFG_ERR_ARG for out-of-range arguments. */
int afg_wait_check(afg_ctx *ctx, int64_t limit_ns, int32_t n_blocks, int64_t *waited_ns, void *stream);

/* ---------------------------------------------------------------- hot path */

/* Welch PSD (Sec. IV ("Noise sampling"): the first 8 s of a window estimate the PSD; Sec. VI:
 * the first 64 s of the stream state).  For detector d and epoch e in
 * [0, n_psd): one-sided density of x[d][e*psd_step, e*psd_step + psd_span),
 * averaged (mean) over K = (psd_span - nfft)/hop + 1 segments of nfft
 * samples every hop samples, each multiplied by the periodic Hann window,
 * transformed with a real FFT in FP32, squared in FP32 after an exact
 * power-of-two scaling of the segment's spectrum (so that no square under- or
 * overflows; relative rounding 1.2e-7) and summed in FP64:
 *   psd[d][e][k] = c_k / (K fs sum w^2) sum_s |X_s(k)|^2, k in [0, nfft/2],
 *   c_k = 1 for k = 0 and k = nfft/2, else 2.
 * x: [n_det][n] float32.  psd: [n_det][n_psd][nfft/2+1] float64.
 * Requirements: psd_span >= nfft, (psd_span - nfft) % hop == 0,
 * psd_step % hop == 0 (each segment's periodogram is computed once and shared
 * by the epochs that contain it), (n_psd-1)*psd_step + psd_span <= n.
 * Errors: AFG_ERR_ARG on a violated requirement. */
int afg_psd_estimate(afg_ctx *ctx, const float *x, int64_t n, int32_t n_det, int64_t n_psd, int64_t psd_step,
                     int64_t psd_span, double *psd, void *stream);

/* Whitening (Sec. IV ("Noise sampling"): whitened in the frequency domain, transformed back,
 * 0.5 s corrupted at each end removed; Sec. VI).  For each detector d and
 * output j in [0, out_len):
 *   y[d][j] = sum_{m=-F/2}^{F/2-1} g^{(e)}_m x[d][out_first + j - m],
 *   e = (epoch_len > 0) ? min(j / epoch_len, n_psd - 1) : 0,
 * with the FIR g^{(e)} built in FP64 from psd[d][e] (amplitude psd^{-1/2},
 * zero below f_highpass, zero-phase inverse DFT on the nfft grid, periodic
 * Hann taper of length F, scale sqrt(2/fs): unit variance for white input),
 * applied in FP32 by overlap-save FFT blocks whose circular convolution
 * equals this linear one on every output.
 * x: [n_det][n] float32; psd: [n_det][n_psd][nfft/2+1] float64 (device);
 * y: [n_det][out_len] float32.
 * Requirements: out_first >= F/2 and out_first + out_len + F/2 - 1 <= n
 * (the crop), epoch_len % 8192 == 0 when epoch_len > 0.
 * out_len = 0 writes nothing (y may then be NULL). */
int afg_whiten(afg_ctx *ctx, const float *x, int64_t n, int32_t n_det, const double *psd, int64_t n_psd,
               int64_t out_first, int64_t out_len, int64_t epoch_len, float *y, void *stream);

/* Network over sliding windows (Sec. II: windows shifted by 1/rate; Sec. VI:
 * the whitened data is unfolded into overlapping windows; Sec. IX: L1
 * shifted for timeslides).  Window j in [0, n_win) holds
 *   H1: y[0][first + j*stride + t],  L1: y[1][(first + j*stride + shift + t) mod n_y],
 * t in [0, W).  Windows are never materialised: the first convolution reads
 * them from y.  logits[j] = network(window j), float32.
 * y: [2][n_y] float32 whitened.  logits: [n_win] float32.
 * Requirements: first >= 0, first + (n_win-1)*stride + W <= n_y, 0 <= shift < n_y.
 * n_win = 0 launches nothing (logits may then be NULL). */
int afg_infer_windows(afg_ctx *ctx, const float *y, int64_t n_y, int64_t first, int64_t stride, int64_t n_win,
                      int64_t shift, float *logits, void *stream);

/* Integration and clustering (Sec. II: 1 s top-hat, maximum over 8 s).
 *   stat[j] = (1/n_int) sum_{i<n_int} logits[j+i],  j in [0, n_win - n_int]
 * (valid mode; stat[j] is stamped at window j + n_int - 1, the newest).
 * Index j is a trigger iff stat[j] >= stat[i] for all |i-j| <= cluster_half
 * and stat[j] > stat[i] for i in [j - cluster_half, j) (ties go to the
 * earliest).  Trigger indices are written to trig_idx in increasing order;
 * *n_trig (device int64) receives their count, which may exceed trig_cap
 * (only trig_cap are written).
 * logits: [n_win] f32; stat: [n_win-n_int+1] f32; trig_idx: [trig_cap] i64. */
int afg_integrate(afg_ctx *ctx, const float *logits, int64_t n_win, int32_t n_int, int32_t cluster_half,
                  float *stat, int64_t *trig_idx, int64_t trig_cap, int64_t *n_trig, void *stream);

/* The whole path on one two-detector span, in one call.
 * Plain mode (p->epoch_len == 0): the PSD of all of x whitens all of x; the
 * whitened stream starts at raw sample F/2 (crop) and window j starts at
 * whitened sample j*stride.  Epoch mode: whitened sample j is raw sample
 * psd_len + j and uses the PSD of raw [e*epoch_len, e*epoch_len + psd_len),
 * e = j / epoch_len (the look-back immediately before its epoch, Sec. VI);
 * window j starts at whitened sample j*stride.
 * x: [2][p->n_raw] float32.  logits: [n_win] f32; stat: [n_win-n_int+1] f32;
 * trig_idx / n_trig as in afg_integrate.  Workspaces are the context's. */
int afg_analyze(afg_ctx *ctx, const float *x, const afg_run_params *p, float *logits, float *stat,
                int64_t *trig_idx, int64_t trig_cap, int64_t *n_trig, void *stream);

/* afg_analyze with HOST buffers: copies x_host (pinned or pageable) to a
 * context workspace, runs the path, and copies stat and the triggers back.
 * stat_host: [n_win-n_int+1]; trig_idx_host: [trig_cap]; *n_trig_host is the
 * trigger count.  Synchronises the stream before returning. */
int afg_analyze_host(afg_ctx *ctx, const float *x_host, const afg_run_params *p, float *stat_host,
                     int64_t *trig_idx_host, int64_t trig_cap, int64_t *n_trig_host, void *stream);



/* ---------------------------------------------------------------- timeslide batches */

/* One strain segment inside a longer two-detector buffer. */
typedef struct afg_segment {
    int64_t offset; /* first raw sample of the segment in each detector row */
    int64_t n_raw;  /* raw samples of the segment */
} afg_segment;

typedef struct afg_batch_params {
    int64_t psd_len;      /* PSD look-back (64 s = 131072 samples); nfft + a multiple of hop */
    int64_t epoch_len;    /* PSD epoch (8 s = 16384 samples); a multiple of 8192 */
    int64_t stride;       /* window stride in samples */
    int64_t shift_step;   /* timeslide step in samples (1 s = fs) */
    int32_t n_shift;      /* timeslides k = shift_first .. shift_first + n_shift - 1 */
    int32_t n_int;        /* integration length in windows */
    int32_t cluster_half; /* trigger half-width in statistic samples */
    int32_t use_graph;    /* 1: capture the whole batch into a CUDA graph on the first call
                             and replay it while the arguments stay the same */
    int64_t shift_first;  /* first timeslide k of this call (>= 1: zero lag is not background;
                             0 is read as 1), so that several calls (or GPUs) can each take a
                             contiguous range of the timeslides of one background */
} afg_batch_params;

/* Sizes of a batch (host only, no GPU work): for every segment, the windows
 * of one timeslide (n_win_host[i], may be NULL), the total windows over all
 * segments and timeslides, and the total statistic samples.  Segment i is
 * analysed in epoch mode (Sec. VI: the first 64 s estimate the PSD and the
 * rest is whitened): it yields floor((n_raw - psd_len - fir_len/2) /
 * epoch_len) whole epochs of whitened data and (n_white - W)/stride + 1
 * windows.  AFG_ERR_ARG if a segment is too short for one epoch, n_int
 * windows, or (shift_first + n_shift - 1) * shift_step whitened samples. */
int afg_batch_layout(afg_ctx *ctx, const afg_segment *segs_host, int32_t n_seg, const afg_batch_params *p,
                     int64_t *n_win_host, int64_t *total_windows, int64_t *total_stat);

/* Timeslide background over many segments in one call (Sec. IX: Hanford
 * fixed, Livingston shifted in 1 s steps until the livetime is reached).
 * Each detector of each segment is whitened once on its own axis (epoch
 * mode); series s = i * n_shift + (k - shift_first) pairs H1 of segment i with
 * its L1 circularly shifted by k * shift_step samples within the segment's whitened
 * span.  All windows of all series go through one persistent network launch.
 * Outputs, concatenated in series order: logits [total_windows] (may be
 * NULL: a context workspace is used), stat [total_stat] (each series
 * integrated on its own, valid mode), and the triggers of every series (its
 * own 8 s clustering) as indices into stat, in increasing order; *n_trig
 * (device) is their count (only trig_cap are written).
 * x: [2][x_len] float32, segments given by offset/n_raw. */
int afg_batch_run(afg_ctx *ctx, const float *x, int64_t x_len, const afg_segment *segs_host, int32_t n_seg,
                  const afg_batch_params *p, float *logits, float *stat, int64_t *trig_idx, int64_t trig_cap,
                  int64_t *n_trig, void *stream);


/* ---------------------------------------------------------------- resampling */

/* Decimation of raw strain by an integer factor M (Sec. IV.A: the strain is
 * resampled to 2048 Hz, e.g. 16384 Hz with M = 8 or 4096 Hz with M = 2;
 * Table III: the filter's edge costs latency).  Anti-aliasing filter: a
 * Kaiser-windowed sinc (beta = 5), 2L + 1 taps with L = 10 M, cutoff at the
 * output Nyquist frequency, normalised to unit gain at DC.  Valid mode:
 * output j is the filter centred on input sample (j0 + j) * M with
 * j0 = ceil(L / M), for every centre whose taps lie inside the input:
 *   y[d][j] = sum_{k=-L..L} h_k x[d][(j0 + j) M + k].
 * x: [n_det][x_stride] f32 (device; x_stride 0 = n_in); y: [n_det][y_stride]
 * f32 (device; y_stride 0 = the output count).  *n_out (host, may be NULL)
 * receives the output count.  The first call with a given factor builds the
 * taps on this context and synchronises; later calls only launch.
 * Errors: AFG_ERR_ARG for NULL pointers, n_det < 1, a factor outside 2..16,
 * or strides smaller than the rows. */
int afg_resample(afg_ctx *ctx, const float *x, int64_t n_in, int32_t n_det, int64_t x_stride, int32_t factor, float *y,
                 int64_t y_stride, int64_t *n_out, void *stream);

/* Output count of afg_resample and the input sample of output 0 (host only). */
int afg_resample_size(int64_t n_in, int32_t factor, int64_t *n_out, int64_t *first_input);

/* ---------------------------------------------------------------- false-alarm rates, trigger times */

/* False-alarm rates from a timeslide background (Sec. IX: the FAR assigned to an
 * event is the number of background events with a detection statistic greater
 * than the event's, divided by the background livetime).
 * Background events: bg_stat[bg_idx[i]] for i < n (bg_idx NULL: bg_stat[i]),
 * where n = min(*n_bg_dev, bg_cap) is read on the device, so the trigger list
 * and count that afg_batch_run writes can be passed directly (bg_stat = its
 * stat, bg_idx = its trig_idx, n_bg_dev = its n_trig, bg_cap = its trig_cap).
 * For each of the n_fg foreground statistics fg[j] (device f32):
 *   n_above[j] = #{background statistics > fg[j]}  (device i64, may be NULL)
 *   far[j]     = n_above[j] / livetime_s            (device f64, per second, may be NULL)
 * bg_sorted (device f32 [bg_cap], may be NULL) receives the background
 * statistics in decreasing order (the first n entries).  The sort runs on the
 * device (radix sort of order-preserving keys); nothing synchronises, so the
 * call can follow afg_batch_run on the same stream or inside a graph capture.
 * NaN statistics give unspecified counts.  Errors: AFG_ERR_ARG for NULL
 * inputs, bg_cap < 0, n_fg < 0 or livetime_s <= 0. */
int afg_far(afg_ctx *ctx, const float *bg_stat, const int64_t *bg_idx, const int64_t *n_bg_dev, int64_t bg_cap,
            double livetime_s, const float *fg, int64_t n_fg, int64_t *n_above, double *far, float *bg_sorted,
            void *stream);

/* Times of statistic samples (host only, no GPU work).  For indices idx[i]
 * into the statistic of one span analysed with run parameters p (as in
 * afg_analyze), with t0 the time of raw sample 0:
 *   t_peak[i] = t0 + (base + (idx[i] + n_int - 1) * stride + W) / fs
 * (Sec. II: the statistic is stamped at the right edge of the newest window
 * it integrates; base = fir_len/2 in plain mode, psd_len in epoch mode), and
 * the coalescence-time estimate (Sec. II: correct for the integration length,
 * the whitening settle-in and where the coalescence sat in the training
 * kernel; Fig. 1: full activation comes 0.75 s after coalescence)
 *   t_c[i] = t_peak[i] - (n_int - 1) * stride / fs - gap_s,
 * i.e. the time at which a response that switches on gap_s after coalescence
 * and lasts at least the integration length first reaches the maximum of its
 * causal average.  gap_s = 0.75 reproduces the paper's offsets.  t_peak or
 * t_c may be NULL.  Errors: AFG_ERR_ARG for NULL ctx/p/idx, n < 0, or an index
 * outside [0, n_win - n_int]. */
int afg_trigger_times(const afg_ctx *ctx, const afg_run_params *p, const int64_t *idx, int64_t n, double t0,
                      double gap_s, double *t_peak, double *t_c);

/* ---------------------------------------------------------------- streaming */

/* Streaming analysis with continuous batching (Sec. VI: clients send strain
 * updates; a snapshotter caches the overlapping state on the server; the
 * whitener estimates the PSD from the first 64 s of that state and whitens
 * the rest; overlapping windows go to the network; Sec. II: 1 s
 * integration).  Per stream the device holds a ring of raw strain, a ring of
 * whitened strain, the whitening gains of two epochs and a ring of logits.
 * Whitened sample j of a stream is raw sample psd_len + j, whitened with the
 * PSD of raw [e*epoch_len, e*epoch_len + psd_len), e = j / epoch_len (the
 * 64 s before its epoch; refreshed every epoch_len samples); window w covers
 * whitened [w*stride, w*stride + W); its statistic is the mean of the logits
 * of windows w - n_int + 1 .. w.  Results appear once a window's data,
 * including the 0.5 s whitening crop after it, has been pushed.
 * A host engine thread per context forms one GPU step from every chunk
 * pushed so far (all streams, one launch per stage); chunks pushed while a
 * step runs join the next step.  When idle, the engine polls for the next push
 * for 20 ms before it sleeps (a sleeping thread wakes tens of microseconds
 * late), so it keeps one host core busy while pushes keep arriving.  PSD
 * refreshes are built after a step's results, ahead of the epoch that needs
 * them.  Streams run the BF16 tensor-core network
 * (precision AFG_BF16, a 16-channel one-stage network).  While streams are
 * active, make no other calls on the same context except the stream calls. */
typedef struct afg_stream_params {
    int64_t psd_len;     /* PSD look-back (64 s = 131072) */
    int64_t epoch_len;   /* PSD refresh period (8 s = 16384) */
    int64_t stride;      /* window stride (16 Hz = 128) */
    int32_t n_int;       /* integration length in windows (<= 64) */
    int32_t max_streams; /* stream slots */
    int32_t max_chunk;   /* largest push in samples per detector (<= 8192 - W - stride) */
} afg_stream_params;

typedef struct afg_stream_result {
    int64_t window; /* window index w within the stream */
    float stat;     /* integrated statistic of windows w - n_int + 1 .. w */
    float logit;    /* logit of window w */
    double t_push;  /* host monotonic time (s) of the push that completed the window's data */
    double t_done;  /* host monotonic time (s) at which the result reached the host */
} afg_stream_result;

/* Start the engine (allocates its step buffers; once per context). */
int afg_stream_start(afg_ctx *ctx, const afg_stream_params *p);

/* Admit a stream: allocates its device state (~3 MB).  AFG_ERR_BUDGET when
 * every slot is taken or the context's hbm_budget would be exceeded. */
int afg_stream_open(afg_ctx *ctx, int64_t *stream_id);

/* Queue n samples per detector (chunk_host: [2][n] float32, host memory;
 * copied before returning).  Returns immediately; *ticket (may be NULL)
 * receives the push's sequence number within the stream.  AFG_ERR_NAN for a
 * non-finite sample, AFG_ERR_STATE for a stream that is not open. */
int afg_stream_push(afg_ctx *ctx, int64_t id, const float *chunk_host, int64_t n, int64_t *ticket);

/* Push n_push chunks of n samples per detector at once (a burst of arrivals):
 * chunk k goes to stream ids[k] and is chunks_host[k][2][n] (host memory,
 * row-major, copied before returning); the same as n_push calls of
 * afg_stream_push in order, under one lock, with one push time.  tickets
 * (NULL or n_push entries) receives each push's sequence number within its
 * stream.  Every chunk and id is checked first: AFG_ERR_NAN (a non-finite
 * sample) or AFG_ERR_STATE (a stream that is not open) pushes nothing.
 * AFG_ERR_ARG for n outside 1..max_chunk or missing arrays. */
int afg_stream_push_many(afg_ctx *ctx, int64_t n_push, const int64_t *ids, const float *chunks_host, int64_t n,
                         int64_t *tickets);

/* Move up to cap available results of the stream (oldest first) to out;
 * waits up to wait_s seconds if none is available yet. */
int afg_stream_poll(afg_ctx *ctx, int64_t id, afg_stream_result *out, int64_t cap, int64_t *n_out, double wait_s);

/* Wait up to wait_s seconds until every pushed chunk has been processed
 * (AFG_ERR_TIMEOUT otherwise). */
int afg_stream_flush(afg_ctx *ctx, double wait_s);

/* Close a stream: drops its queued chunks and results; its device state is
 * released once its work in flight completes. */
int afg_stream_close(afg_ctx *ctx, int64_t id);

/* Engine counters: GPU steps, windows evaluated, samples per detector ingested. */
int afg_stream_stats(afg_ctx *ctx, int64_t *steps, int64_t *windows, int64_t *samples);

/* ---------------------------------------------------------------- profiling */

/* Per-kernel accounting of the library's own launches.  `algo_flops` and
 * `algo_bytes` are the algorithmic work of the recorded launches (the FLOPs
 * of the operation's definition, the bytes a single pass over its inputs and
 * outputs moves), summed; `total_ms` sums CUDA-event durations taken on the
 * stream each kernel was launched on (only while profiling is enabled). */
typedef struct afg_kernel_stat {
    char name[48];
    int64_t launches;   /* launches since the last afg_profile_enable / read */
    int64_t timed;      /* launches with event timings */
    double total_ms;
    double algo_flops;
    double algo_bytes;
} afg_kernel_stat;

/* on != 0: reset the counters and record a pair of CUDA events around every
 * subsequent launch.  on == 0: stop recording (counters keep counting). */
int afg_profile_enable(afg_ctx *ctx, int32_t on);

/* Synchronise the device, fold the recorded events into per-kernel totals,
 * write up to cap entries (kernels with at least one launch) to out, set
 * *n_out, and reset the counters.  Errors: AFG_ERR_ARG for NULL pointers. */
int afg_profile_read(afg_ctx *ctx, afg_kernel_stat *out, int32_t cap, int32_t *n_out);

/* ---------------------------------------------------------------- conv tile autotuning */

/* Tile of one convolution of the BF16 tensor-core path for wide networks
 * (widths 64..512: every convolution after the stem is one tcgen05 implicit
 * GEMM launch).  The network is the 1D ResNet of Sec. II; the tiles are an
 * implementation choice with no counterpart in the paper.  Every tile of a
 * layer computes the same convolution (accumulation order aside). */
typedef struct afg_tile {
    int32_t layer;        /* convolution index in execution order (1 = first after the stem) */
    int32_t cin, cout, lin, lout, stride, taps;
    int32_t residual;     /* 1 if the epilogue adds the block's shortcut */
    int32_t orient;       /* 0: position-major (M = 128 positions, N = C_out, C_out <= 128);
                             1: channel-major (M = 128 output channels, N = positions of `wpc` windows) */
    int32_t wpc;          /* windows per tile (1 for position-major) */
    int32_t kb;           /* input channels per K-block (32, 64 or 128; C_in for position-major) */
    int32_t stages;       /* shared-memory ring depth, 1..8 */
    int32_t acc_bufs;     /* TMEM accumulator buffers: 2 overlaps a tile's epilogue with the next tile's MMAs */
    int32_t tuned;        /* 1: chosen by afg_autotune (or set so by afg_tiles_set); 0: default heuristic */
    int32_t n_candidates; /* tiles timed for this layer's geometry */
    float us_chosen;      /* microseconds per launch of the chosen tile at the tuning size (0: not timed) */
    float us_default;     /* microseconds per launch of the default tile at the tuning size (0: not timed) */
} afg_tile;

/* Wide networks: time every valid tile of each distinct layer geometry
 * (channels, lengths, stride, taps, residual) on n_win synthetic windows
 * (n_win <= 0: 1024; at most 4096) and keep the fastest for later inference
 * calls; uses the context's activation workspaces.
 * The fused 16-channel network (BF16, 8 GroupNorm groups, 3072-position
 * windows, whose geometry is compiled with fixed counts): time every
 * candidate of afg_fused_tuning_candidates (epilogue warps, MMA-issue warps,
 * polling sleep) on n_win windows, 64 samples apart, of synthetic whitened
 * strain (n_win <= 0: 4096; at most 65536) and keep the fastest; uses the
 * context's whitened-strain and logit workspaces.
 * Synchronous: synchronises `stream` and returns when done.  Errors:
 * AFG_ERR_UNSUPPORTED if the context has neither (FP32 contexts, or a fused
 * network of another geometry); AFG_ERR_STATE if `stream` is capturing;
 * AFG_ERR_TIMEOUT if a bounded device wait gave up; AFG_ERR_CUDA /
 * AFG_ERR_OOM / AFG_ERR_BUDGET. */
int afg_autotune(afg_ctx *ctx, int64_t n_win, void *stream);

/* Current tile of every convolution after the stem, in execution order:
 * writes min(cap, count) entries to out and the count to *n_out. */
int afg_tiles_get(afg_ctx *ctx, afg_tile *out, int32_t cap, int32_t *n_out);

/* Every tile the tuner would time for `layer` (the timing fields are 0). */
int afg_tile_candidates(afg_ctx *ctx, int32_t layer, afg_tile *out, int32_t cap, int32_t *n_out);

/* Apply tiles (e.g. a saved tuning): each entry's layer, orient, wpc, kb,
 * stages and acc_bufs.  All entries are checked first; AFG_ERR_ARG (and no
 * change) if one does not fit its layer. */
int afg_tiles_set(afg_ctx *ctx, const afg_tile *tiles, int32_t n);

/* Launch knobs of the fused 16-channel BF16 network (one window per CTA
 * pass, its layers pipelined; Sec. II network, Sec. IX batches).  Every
 * candidate computes the same network (up to the summation order of the
 * GroupNorm statistics across warps); they differ in speed only. */
typedef struct afg_fused_tuning {
    int32_t epi_warps;    /* epilogue warps: 8 or 12 (2 or 3 quads of four) */
    int32_t issue_warps;  /* MMA-issue warps: 1 or 2 */
    int32_t spin_ns;      /* the issue warps' sleep between polls of an incomplete barrier (0: spin) */
    int32_t tuned;        /* 1: chosen by afg_autotune (or set so by afg_fused_tuning_set) */
    int32_t n_candidates; /* candidates timed */
    float us_chosen;      /* microseconds per launch of the chosen candidate at the tuning size (0: not timed) */
    float us_default;     /* microseconds per launch of the default (12, 2, 64) (0: not timed) */
} afg_fused_tuning;

/* Current knobs of the context's fused network.  AFG_ERR_UNSUPPORTED without a
 * fused 16-channel BF16 network. */
int afg_fused_tuning_get(afg_ctx *ctx, afg_fused_tuning *out);

/* Every candidate afg_autotune times (timing fields 0): writes min(cap, count)
 * entries and the count to *n_out.  AFG_ERR_UNSUPPORTED unless the fused
 * network has the tunable geometry (8 groups, 3072 positions). */
int afg_fused_tuning_candidates(afg_ctx *ctx, afg_fused_tuning *out, int32_t cap, int32_t *n_out);

/* Apply knobs (e.g. a saved tuning): epi_warps 8 or 12, issue_warps 1 or 2,
 * spin_ns in [0, 100000]; AFG_ERR_ARG (and no change) otherwise,
 * AFG_ERR_UNSUPPORTED as for afg_fused_tuning_candidates. */
int afg_fused_tuning_set(afg_ctx *ctx, const afg_fused_tuning *in);

/* ---------------------------------------------------------------- allocation-free PSD */

/* Largest n_det * (distinct Welch segments) one afg_psd_estimate_noalloc call accepts. */
#define AFG_NOALLOC_MAX_PERIODOGRAMS 64

/* Welch PSD for callers that cannot allocate device memory.  The paper has
 * no counterpart to this entry point; it exists for integrations of this
 * library, not for the method.  Some hosts cannot call cudaMalloc: an
 * application (an inference-server backend, a framework plugin) that owns
 * every byte of device memory through its own pool and forbids allocations
 * behind its back, or a latency-critical loop where cudaMalloc/cudaFree
 * would add an implicit device-wide synchronisation.  The context API
 * allocates its workspaces on first use, so such callers use this instead.
 *
 * Result: exactly what afg_psd_estimate computes (same kernels, same
 * arguments, nfft = 16384, periodic Hann, FP32 FFT, FP64 averaging), but
 * without a context: fs and hop are passed directly.
 * x: [n_det][n] float32 (device); psd: [n_det][n_psd][8193] float64 (device).
 *
 * Memory: the periodogram scratch (AFG_NOALLOC_MAX_PERIODOGRAMS x 8193
 * doubles, 4.2 MB) and the FP32 transforms' twiddle table (60 KB) are static
 * __device__ arrays that every GPU which loads the library holds until the
 * process exits.
 * This call allocates and frees nothing.  It refuses with AFG_ERR_BUDGET
 * when n_det * ((n_psd-1)*psd_step/hop + (psd_span-nfft)/hop + 1) exceeds
 * AFG_NOALLOC_MAX_PERIODOGRAMS, and with AFG_ERR_ARG on the requirements of
 * afg_psd_estimate.  AFG_ERR_CUDA if a launch or the set-up fails.
 *
 * Set-up: the first call on each device (made with that device current)
 * resolves the array's device address, fills the twiddle table (unless a
 * context on that device already has: one small kernel on a stream of its
 * own, waited for) and configures the kernel, all synchronous; make that
 * first call before any stream capture.  Later calls only launch kernels on
 * `stream`.
 *
 * Sharing: all calls on a device use the same scratch, which keeps the last
 * call's contents (every value a call reads is written earlier in that same
 * call, so nothing needs clearing).  Calls that overlap on the GPU (other
 * streams, other host threads) race on the scratch: serialise them. */
int afg_psd_estimate_noalloc(const float *x, int64_t n, int32_t n_det, int64_t n_psd, int64_t psd_step,
                             int64_t psd_span, int32_t fs, int32_t hop, double *psd, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* AFRAME_GB_H */
