// Internal declarations of the GB300 detection-path library (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/aframe_gb.h"

// ----------------------------------------------------------------------------
// Fixed transform geometry.  Welch segments and whitening blocks both use a
// real FFT of NFFT = 16384 samples, computed as a complex FFT of NC = 8192
// points in shared memory plus the even/odd split.  Whitening blocks are laid
// out per PSD epoch (up to 16385 - F outputs on that transform, the epoch's
// remainder on a 4096-point one), so no block straddles an epoch; epochs are
// multiples of WB = 8192 samples, and a stream piece holds at most WB outputs.
// ----------------------------------------------------------------------------
constexpr int NFFT = 16384;
constexpr int NC = NFFT / 2;
constexpr int NBIN = NFFT / 2 + 1;
constexpr int FILTER_LAGS = 2048;  // lags of the tapered taps the many-CTA filter build keeps
constexpr int WB = 8192;

// Epochs per thread of the Welch averaging kernel; its grid's y extent is
// ceil(n_psd / PSD_EPT), which must stay within 65535.
constexpr int PSD_EPT = 32;

// Validate the layout of a Welch request (x: [n_det][n], n_psd epochs of
// psd_span samples every psd_step, segments of NFFT every hop) without
// forming any product that could overflow: every product is bounded by a
// division first.  On success returns true and the number of distinct
// segments each detector needs (every epoch's segments, shared ones once).
inline bool psd_request_ok(int64_t n, int n_det, int64_t n_psd, int64_t psd_step, int64_t psd_span, int hop,
                           int64_t *n_seg_out) {
    if (n_det < 1 || n_det > 65535 || n_psd < 1 || hop < 1 || NFFT % hop) return false;
    if (psd_span < NFFT || psd_span > n || (psd_span - NFFT) % hop) return false;
    int64_t seg_step = 0;
    if (n_psd > 1) {
        if (psd_step <= 0 || psd_step % hop || psd_step > n) return false;
        if (n_psd - 1 > (n - psd_span) / psd_step) return false;  // (n_psd - 1) psd_step + psd_span <= n
        seg_step = psd_step / hop;
    }
    if ((n_psd + PSD_EPT - 1) / PSD_EPT > 65535) return false;
    const int64_t n_seg = (n_psd - 1) * seg_step + (psd_span - NFFT) / hop + 1;  // <= n / hop + 1
    if (n_seg > 0x7fffffff) return false;
    *n_seg_out = n_seg;
    return true;
}

// ----------------------------------------------------------------------------
// Network plan: one entry per convolution, in execution order.
// ----------------------------------------------------------------------------
struct ConvLayer {
    int cin, cout, k, stride, pad;
    int lin, lout;            // input / output positions per window
    float *wt;                // [k*cin][cout] (row = tap-major then input channel)
    float *gamma, *beta;      // GroupNorm affine [cout]
    __nv_bfloat16_raw *wt_bf16;  // bf16 copy for the tensor-core path, [cout][k*cin] (K-major)
};

struct BlockPlan {
    int c1, c2, sc;  // indices into convs (sc = -1 for identity shortcut)
};

struct NetPlan {
    afg_net net;
    std::vector<ConvLayer> convs;  // convs[0] is the stem
    std::vector<BlockPlan> blocks;
    int l_stem_out;                // positions after the stem conv
    int l_after_stem;              // after the optional max-pool
    float *fc_w, *fc_b;
    int c_last, l_last;
    int64_t max_act_per_window;    // floats of the largest padded activation of one window
    float *tc_params = nullptr;    // fused tensor-core network: FP32 parameter block
    unsigned char *tc_wimg = nullptr;  // and BF16 weight image in shared-memory order
    // fused network's tuning (afg_autotune / afg_fused_tuning_*): epilogue and issue warps, polling sleep
    int tiny_ew = 12, tiny_mw = 2;
    uint32_t tiny_spin_ns = 64;
    int tiny_tuned = 0, tiny_n_cand = 0;
    float tiny_us_chosen = 0.f, tiny_us_default = 0.f;
};

// One segment of a timeslide batch: its whitened span in the concatenated
// whitened buffer and the windows it contributes (n_shift x n_win).
struct SegDesc {
    int64_t y_off;        // first whitened sample of the segment (per detector row)
    int64_t n_y;          // whitened samples of the segment
    int64_t n_win;        // windows per timeslide
    int64_t win_first;    // first global window index of the segment (all its timeslides)
    int64_t shift_first;  // timeslide step of the segment's first series (1 for k = 1)
};

// One window of a list-mode network launch: H1 and L1 rows (W contiguous
// samples each) and where its logit goes.
struct WinPtr {
    const float *y0;
    const float *y1;
    float *out;
};

// One piece of a multi-stream whitening launch (at most whiten_multi_piece_max outputs, one epoch's gains)
struct WhitenPiece {
    const float *x;     // raw sample of output 0 minus F/2, detector row 0
    int64_t x_stride;   // samples between detector rows of x
    const float *gains; // [2][NBIN] gains of the piece's epoch
    float *y;           // mirrored whitened ring, detector row 0
    int64_t y_stride;   // samples between detector rows of y
    int64_t y_ring;     // ring length (each row holds 2 * y_ring samples)
    int64_t y_pos;      // ring slot of output 0 (< y_ring)
    int64_t cnt;        // outputs of the piece (<= WB)
    // Samples not yet in the raw ring (4096-point kernel only): input i >= i_new is
    // stg[i - i_new] (detector row d at stg + d * stg_stride) instead of x[i]; stg null: all from x.
    const float *stg;
    int64_t stg_stride, i_new;
    // If sc_ring is set, this piece's CTAs also write those sc_n samples into the stream's mirrored
    // raw ring (row stride 2 sc_R) at slot sc_pos: one piece per stream, so no separate scatter.
    float *sc_ring;
    int64_t sc_R, sc_pos, sc_n;
};

// One new window of a stream whose 1 s statistic a serving step produces: the mean of the
// logits of windows w - n_int + 1 .. w, read from the stream's logit ring (STREAM_LR slots).
constexpr int STREAM_LR = 64;
struct IntegDesc {
    const float *ring;  // logits ring of the stream
    int64_t w;          // window index
    float *out;         // (stat, logit) pair
};

struct Workspace {
    void *p = nullptr;
    size_t bytes = 0;
};

// ----------------------------------------------------------------------------
// Launch accounting (afg_profile_*): every library launch goes through a
// KScope, which counts it and, while profiling is on, brackets it with two
// events on its stream.
// ----------------------------------------------------------------------------
enum KernelKind {
    KK_TWIDDLES = 0,
    KK_PERIODOGRAM,
    KK_PSD_MEAN,
    KK_FILTER,
    KK_WHITEN,
    KK_STEM,
    KK_GROUPNORM,
    KK_CONV_FP32,
    KK_HEAD,
    KK_INTEGRATE,
    KK_TRIGGERS,
    KK_CONV_TC,
    KK_TINY_TC,
    KK_SCATTER,
    KK_CONVERT,
    KK_FAR,
    KK_RESAMPLE,
    KK_COUNT
};
extern const char *const kKernelNames[KK_COUNT];

struct ProfRec {
    int kind;
    cudaEvent_t e0, e1;
};

struct Prof {
    bool on = false;
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    size_t pool_used = 0;
    int64_t launches[KK_COUNT] = {};
    double flops[KK_COUNT] = {};
    double bytes[KK_COUNT] = {};
};

struct BatchCache;
struct ServeEngine;
struct TcPlan;

struct afg_ctx {
    Prof prof;
    BatchCache *batch = nullptr;      // captured timeslide-batch graph (batch.cu)
    ServeEngine *serve = nullptr;     // streaming engine (serve.cu)
    TcPlan *tcplan = nullptr;         // per-layer tensor-core plan of wide networks (net_tc_layers.cu)
    afg_config cfg;
    int device = 0;
    std::string err;
    NetPlan plan;
    float *d_params = nullptr;        // all network parameters (device)
    size_t d_params_bytes = 0;
    double2 *tw64 = nullptr;          // exp(-2 pi i k / NFFT), k < NFFT, double (filter build)
    double *taper64 = nullptr;        // sqrt(2 / fs) taper(m) / (2 NFFT NC) at m + FILTER_LAGS / 2, m in
                                      // [-FILTER_LAGS / 2, FILTER_LAGS / 2) (after tw64, same allocation)
    int64_t bytes_held = 0;
    int *d_err = nullptr;             // device-side failure record (bounded waits that gave up)
    Workspace ws[32];
    float *rs_taps[17] = {};          // decimation filters by factor (resample.cu)
};

// workspace slots
enum {
    WS_PERIODOGRAM = 0,
    WS_FILTER,
    WS_PSD,
    WS_WHITE,
    WS_ACT0,
    WS_ACT1,
    WS_ACT2,
    WS_ACT3,
    WS_GNSTAT,
    WS_LOGITS,
    WS_STAT,
    WS_X,
    WS_TRIG,
    WS_SCAN,
    WS_BATCH_SEGS,
    WS_BATCH_SERIES,
    WS_FAR_KEYS,
    WS_FAR_HIST,
    WS_FAR_SORTED,
    WS_TRIG_A,
    WS_TRIG_B,
    WS_TRIG_FLAG,
    WS_TRIG_COUNT,
    WS_FB_SCRATCH,
};

struct KScope {
    afg_ctx *ctx;
    cudaStream_t st;
    int kind;
    cudaEvent_t e0 = nullptr;
    KScope(afg_ctx *c, cudaStream_t s, int k, double flops, double bytes);
    ~KScope();
};

// ----------------------------------------------------------------------------
// Programmatic dependent launch: a kernel launched with launch_pdl may start
// (and run its set-up) while the previous kernel on the stream finishes; it
// calls pdl_wait() before it touches anything that kernel writes, which
// returns once that kernel has completed and its writes are visible.
// pdl_trigger() in the earlier kernel lets the dependent launch start early.
// Both are no-ops for kernels launched without the attribute.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// cluster > 1 also groups the CTAs into clusters of that many along x.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl_cluster(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                               int cluster, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    int n = 1;
    if (cluster > 1) {
        attr[1].id = cudaLaunchAttributeClusterDimension;
        attr[1].val.clusterDim.x = (unsigned)cluster;
        attr[1].val.clusterDim.y = 1;
        attr[1].val.clusterDim.z = 1;
        n = 2;
    }
    cfg.attrs = attr;
    cfg.numAttrs = n;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
    return launch_pdl_cluster(kernel, grid, block, smem, st, 1, args...);
}

// ----------------------------------------------------------------------------
// Error plumbing
// ----------------------------------------------------------------------------
int afg_fail(afg_ctx *ctx, int code, const char *fmt, ...);
int afg_cuda_fail(afg_ctx *ctx, cudaError_t e, const char *what);
size_t filter_build_scratch_bytes(const afg_ctx *ctx, int64_t nf);
int afg_ws_reserve(afg_ctx *ctx, int slot, size_t bytes, void **out);
void batch_cache_release(afg_ctx *ctx);
void serve_release(afg_ctx *ctx);

#define AFG_CUDA(ctx, call)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return afg_cuda_fail(ctx, e_, #call); \
    } while (0)

#define AFG_LAUNCH_CHECK(ctx, what)                                   \
    do {                                                              \
        cudaError_t e_ = cudaGetLastError();                          \
        if (e_ != cudaSuccess) return afg_cuda_fail(ctx, e_, what);   \
    } while (0)

// ----------------------------------------------------------------------------
// Host-side launchers implemented in the .cu files
// ----------------------------------------------------------------------------
// spectral.cu
int afg_make_twiddles(afg_ctx *ctx);
// x_stride: samples between detector rows of x (0: n)
int launch_psd(afg_ctx *ctx, const float *x, int64_t n, int n_det, int64_t n_psd, int64_t psd_step,
               int64_t psd_span, double *psd, cudaStream_t st, int64_t x_stride = 0);
int launch_whiten(afg_ctx *ctx, const float *x, int64_t n, int n_det, const double *psd, int64_t n_psd,
                  int64_t out_first, int64_t out_len, int64_t epoch_len, float *y, int64_t y_stride,
                  cudaStream_t st, int64_t x_stride = 0);
cudaError_t launch_psd_on(const float *x, int64_t n, int n_det, int64_t n_psd, int64_t psd_step, int64_t psd_span,
                          int hop, int fs, double *P, double *psd, cudaStream_t st);
cudaError_t prepare_psd_kernels();
int launch_filter(afg_ctx *ctx, const double *psd, int n_det, int64_t n_psd, float *gains, cudaStream_t st);
int launch_psd_rows(afg_ctx *ctx, const float *const *rows_dev, int n_rows, int64_t psd_span, double *psd,
                    cudaStream_t st);
int launch_scatter_rows(afg_ctx *ctx, const float *src, float *const *dst_dev, int n_rows, int len, cudaStream_t st);
int launch_whiten_multi(afg_ctx *ctx, const WhitenPiece *pieces_dev, int n_pieces, int64_t total_out,
                        cudaStream_t st);
int whiten_multi_piece_max(const afg_ctx *ctx);  // outputs per piece of launch_whiten_multi
bool whiten_multi_takes_staging(const afg_ctx *ctx);  // pieces may carry stg / sc_ring
// net_fp32.cu
int net_plan_build(afg_ctx *ctx, const float *weights_host, int64_t n_weights);
int launch_infer_fp32(afg_ctx *ctx, const float *y, int64_t n_y, int64_t y_stride, int64_t first,
                      int64_t stride, int64_t n_win, int64_t shift, float *logits, cudaStream_t st);
int launch_stem_gn_fp32(afg_ctx *ctx, const float *y, int64_t n_y, int64_t y_stride, int64_t first, int64_t stride,
                        int64_t shift, int64_t w0, int nw, float *f0, float *f1, cudaStream_t st);
// net_tc_layers.cu
int net_tc_layers_prepare(afg_ctx *ctx);
void net_tc_layers_release(afg_ctx *ctx);
bool net_tc_layers_available(const afg_ctx *ctx);
int launch_infer_bf16_full(afg_ctx *ctx, const float *y, int64_t n_y, int64_t y_stride, int64_t first,
                           int64_t stride, int64_t n_win, int64_t shift, float *logits, cudaStream_t st);
int net_tc_autotune(afg_ctx *ctx, int64_t n_win, cudaStream_t st);
bool net_tc_tiny_tunable(const afg_ctx *ctx);
int net_tc_tiny_autotune(afg_ctx *ctx, int64_t n_win, cudaStream_t st);
int net_tc_tiny_tuning_get(afg_ctx *ctx, afg_fused_tuning *out);
int net_tc_tiny_tuning_candidates(afg_ctx *ctx, afg_fused_tuning *out, int cap, int *n_out);
int net_tc_tiny_tuning_set(afg_ctx *ctx, const afg_fused_tuning *in);
int net_tc_tiles_get(afg_ctx *ctx, afg_tile *out, int cap, int *n_out);
int net_tc_tile_candidates(afg_ctx *ctx, int layer, afg_tile *out, int cap, int *n_out);
int net_tc_tiles_set(afg_ctx *ctx, const afg_tile *in, int n);
// net_tc.cu
int net_tc_prepare(afg_ctx *ctx);
int launch_infer_bf16_batch(afg_ctx *ctx, const float *white, int64_t y_stride, const SegDesc *segs_dev, int n_seg,
                            int64_t total_win, int64_t stride, int64_t shift_step, float *logits, cudaStream_t st);
// integ (n_integ entries, may be 0): statistics the launch computes once all its windows are
// done (the last CTA to finish, counted in *done, which must be 0 on entry and is left at 0)
int launch_infer_bf16_list(afg_ctx *ctx, const WinPtr *wins_dev, int64_t n_win, const IntegDesc *integ,
                           int n_integ, int n_int, unsigned *done, cudaStream_t st);
int launch_infer_bf16(afg_ctx *ctx, const float *y, int64_t n_y, int64_t y_stride, int64_t first,
                      int64_t stride, int64_t n_win, int64_t shift, float *logits, cudaStream_t st);
// resample.cu
int64_t resample_count(int64_t n_in, int M, int64_t *j0_out);
int launch_resample(afg_ctx *ctx, const float *x, int64_t n_in, int n_det, int64_t x_stride, int M, float *y,
                    int64_t y_stride, int64_t *n_out_host, cudaStream_t st);
// far.cu
int launch_far(afg_ctx *ctx, const float *bg_stat, const int64_t *bg_idx, const int64_t *n_bg_dev, int64_t bg_cap,
               double livetime_s, const float *fg, int64_t n_fg, int64_t *n_above, double *far, float *bg_sorted,
               cudaStream_t st);
// integrate.cu
int launch_integrate(afg_ctx *ctx, const float *logits, int64_t n_win, int n_int, int cluster_half,
                     float *stat, int64_t *trig_idx, int64_t trig_cap, int64_t *n_trig, cudaStream_t st);
