// C-ABI entry points of the detection-path library: argument validation,
// context and workspace management, and the composition of the kernels.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "afg_internal.cuh"

#define AFG_VERSION "aframe-gb300 0.1 (sm_103a)"

// ---------------------------------------------------------------- errors
int afg_fail(afg_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

int afg_cuda_fail(afg_ctx *ctx, cudaError_t e, const char *what) {
    return afg_fail(ctx, e == cudaErrorMemoryAllocation ? AFG_ERR_OOM : AFG_ERR_CUDA, "%s: %s (%s)", what,
                    cudaGetErrorString(e), cudaGetErrorName(e));
}

// Grow-only workspace slot.  Growing frees the old buffer (synchronising
// the device through cudaFree), so steady-state calls never allocate.
int afg_ws_reserve(afg_ctx *ctx, int slot, size_t bytes, void **out) {
    Workspace &w = ctx->ws[slot];
    if (bytes == 0) bytes = 256;
    if (w.bytes < bytes) {
        size_t grow = std::max(bytes, w.bytes + w.bytes / 4);
        int64_t after = ctx->bytes_held - (int64_t)w.bytes + (int64_t)grow;
        if (ctx->cfg.hbm_budget > 0 && after > ctx->cfg.hbm_budget) {
            grow = bytes;
            after = ctx->bytes_held - (int64_t)w.bytes + (int64_t)grow;
            if (after > ctx->cfg.hbm_budget)
                return afg_fail(ctx, AFG_ERR_BUDGET, "workspace %d: %zu bytes would exceed the HBM budget (%lld)",
                                slot, bytes, (long long)ctx->cfg.hbm_budget);
        }
        if (w.p) {
            cudaFree(w.p);
            ctx->bytes_held -= (int64_t)w.bytes;
            w.p = nullptr;
            w.bytes = 0;
        }
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, grow);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return afg_fail(ctx, AFG_ERR_OOM, "workspace %d: cudaMalloc(%zu) failed: %s", slot, grow,
                            cudaGetErrorString(e));
        }
        w.p = p;
        w.bytes = grow;
        ctx->bytes_held += (int64_t)grow;
    }
    *out = w.p;
    return AFG_OK;
}

void prof_release(afg_ctx *ctx);

static inline cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// ---------------------------------------------------------------- validation
static int check_net(const afg_net *n, char *why, size_t len) {
    if (!n) { snprintf(why, len, "net is NULL"); return 0; }
    if (n->in_ch != 2) { snprintf(why, len, "net.in_ch must be 2"); return 0; }
    if (n->stem_k < 1 || n->stem_k > 7 || !(n->stem_k & 1)) { snprintf(why, len, "net.stem_k must be odd, <= 7"); return 0; }
    if (n->stem_stride != 1 && n->stem_stride != 2) { snprintf(why, len, "net.stem_stride must be 1 or 2"); return 0; }
    if (n->stem_pool != 0 && n->stem_pool != 1) { snprintf(why, len, "net.stem_pool must be 0 or 1"); return 0; }
    if (n->n_stages < 1 || n->n_stages > 4) { snprintf(why, len, "net.n_stages must be 1..4"); return 0; }
    if (n->groups < 1 || n->groups > 32) { snprintf(why, len, "net.groups must be 1..32"); return 0; }
    if (!(n->eps > 0.f)) { snprintf(why, len, "net.eps must be > 0"); return 0; }
    for (int s = 0; s < n->n_stages; ++s) {
        int w = n->widths[s];
        if (w < 16 || w > 512 || (w & (w - 1))) { snprintf(why, len, "net.widths[%d] must be a power of two in [16, 512]", s); return 0; }
        if (w % n->groups) { snprintf(why, len, "net.groups must divide widths[%d]", s); return 0; }
        if (n->blocks[s] < 1 || n->blocks[s] > 64) { snprintf(why, len, "net.blocks[%d] must be 1..64", s); return 0; }
    }
    return 1;
}

extern "C" {

const char *afg_version(void) { return AFG_VERSION; }

const char *afg_status_string(int status) {
    switch (status) {
        case AFG_OK: return "AFG_OK";
        case AFG_ERR_ARG: return "AFG_ERR_ARG";
        case AFG_ERR_CUDA: return "AFG_ERR_CUDA";
        case AFG_ERR_OOM: return "AFG_ERR_OOM";
        case AFG_ERR_BUDGET: return "AFG_ERR_BUDGET";
        case AFG_ERR_TIMEOUT: return "AFG_ERR_TIMEOUT";
        case AFG_ERR_STATE: return "AFG_ERR_STATE";
        case AFG_ERR_NAN: return "AFG_ERR_NAN";
        case AFG_ERR_UNSUPPORTED: return "AFG_ERR_UNSUPPORTED";
        default: return "AFG_ERR_UNKNOWN";
    }
}

int afg_weights_count(const afg_net *n, int64_t *n_out) {
    char why[160];
    if (!n_out || !check_net(n, why, sizeof why)) return AFG_ERR_ARG;
    int64_t c = 0;
    int C0 = n->widths[0];
    c += (int64_t)C0 * n->in_ch * n->stem_k + 2 * C0;
    int cin = C0;
    for (int s = 0; s < n->n_stages; ++s)
        for (int b = 0; b < n->blocks[s]; ++b) {
            int w = n->widths[s];
            int stride = (s > 0 && b == 0) ? 2 : 1;
            c += (int64_t)w * cin * 3 + 2 * w + (int64_t)w * w * 3 + 2 * w;
            if (stride != 1 || cin != w) c += (int64_t)w * cin + 2 * w;
            cin = w;
        }
    c += cin + 1;
    *n_out = c;
    return AFG_OK;
}

int afg_ctx_create(const afg_config *cfg, const float *weights_host, int64_t n_weights, afg_ctx **out) {
    if (!out) return AFG_ERR_ARG;
    *out = nullptr;
    if (!cfg || !weights_host) return AFG_ERR_ARG;
    char why[160];
    if (!check_net(&cfg->net, why, sizeof why)) return AFG_ERR_ARG;
    if (cfg->nfft != NFFT) return AFG_ERR_UNSUPPORTED;
    if (cfg->hop < 1 || NFFT % cfg->hop) return AFG_ERR_ARG;
    if (cfg->fir_len < 2 || (cfg->fir_len & 1) || cfg->fir_len > WB) return AFG_ERR_ARG;
    if (cfg->fs < 1 || !(cfg->f_highpass >= 0.0)) return AFG_ERR_ARG;
    if (cfg->win_len < 32 || cfg->win_len % 32 || cfg->win_len > 16384) return AFG_ERR_ARG;
    if (cfg->precision != AFG_FP32 && cfg->precision != AFG_BF16) return AFG_ERR_ARG;
    int64_t need = 0;
    afg_weights_count(&cfg->net, &need);
    if (n_weights != need) return AFG_ERR_ARG;
    afg_ctx *ctx = new afg_ctx();
    ctx->cfg = *cfg;
    cudaGetDevice(&ctx->device);
    size_t tw_bytes = NFFT * sizeof(double2) + FILTER_LAGS * sizeof(double);
    cudaError_t e = cudaMalloc(&ctx->tw64, tw_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        afg_ctx_destroy(ctx);
        return AFG_ERR_OOM;
    }
    ctx->bytes_held += (int64_t)tw_bytes;
    ctx->taper64 = reinterpret_cast<double *>(ctx->tw64 + NFFT);
    if (cudaMalloc(&ctx->d_err, 256) != cudaSuccess || cudaMemset(ctx->d_err, 0, 256) != cudaSuccess) {
        cudaGetLastError();
        afg_ctx_destroy(ctx);
        return AFG_ERR_OOM;
    }
    ctx->bytes_held += 256;
    int rc = afg_make_twiddles(ctx);
    if (rc == AFG_OK) rc = net_plan_build(ctx, weights_host, n_weights);
    if (rc == AFG_OK) rc = net_tc_prepare(ctx);
    if (rc == AFG_OK && cfg->precision == AFG_BF16) rc = net_tc_layers_prepare(ctx);
    if (rc == AFG_OK && cudaDeviceSynchronize() != cudaSuccess) rc = AFG_ERR_CUDA;
    if (rc != AFG_OK) {
        afg_ctx_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return AFG_OK;
}

int afg_ctx_destroy(afg_ctx *ctx) {
    if (!ctx) return AFG_ERR_ARG;
    serve_release(ctx);
    cudaDeviceSynchronize();
    prof_release(ctx);
    batch_cache_release(ctx);
    net_tc_layers_release(ctx);
    for (auto &w : ctx->ws)
        if (w.p) cudaFree(w.p);
    if (ctx->d_params) cudaFree(ctx->d_params);
    if (ctx->plan.tc_params) cudaFree(ctx->plan.tc_params);
    if (ctx->d_err) cudaFree(ctx->d_err);
    for (float *t : ctx->rs_taps)
        if (t) cudaFree(t);
    if (ctx->tw64) cudaFree(ctx->tw64);
    delete ctx;
    return AFG_OK;
}

const char *afg_last_error(const afg_ctx *ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

int afg_ctx_bytes(const afg_ctx *ctx, int64_t *bytes) {
    if (!ctx || !bytes) return AFG_ERR_ARG;
    *bytes = ctx->bytes_held;
    return AFG_OK;
}

int afg_sync(afg_ctx *ctx, void *stream) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    AFG_CUDA(ctx, cudaStreamSynchronize(S(stream)));
    int flag = 0;
    AFG_CUDA(ctx, cudaMemcpy(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        AFG_CUDA(ctx, cudaMemset(ctx->d_err, 0, sizeof(int)));
        return afg_fail(ctx, AFG_ERR_TIMEOUT, "a bounded device-side wait gave up (kernel returned early)");
    }
    return AFG_OK;
}

int afg_psd_estimate(afg_ctx *ctx, const float *x, int64_t n, int32_t n_det, int64_t n_psd, int64_t psd_step,
                     int64_t psd_span, double *psd, void *stream) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    const int hop = ctx->cfg.hop;
    if (!x || !psd || n_det < 1 || n_psd < 1) return afg_fail(ctx, AFG_ERR_ARG, "psd_estimate: null pointer or empty");
    if (psd_span < NFFT || (psd_span - NFFT) % hop)
        return afg_fail(ctx, AFG_ERR_ARG, "psd_estimate: psd_span must be nfft + a multiple of hop");
    if (n_psd > 1 && (psd_step <= 0 || psd_step % hop))
        return afg_fail(ctx, AFG_ERR_ARG, "psd_estimate: psd_step must be a positive multiple of hop");
    int64_t n_seg = 0;
    if (!psd_request_ok(n, n_det, n_psd, psd_step, psd_span, hop, &n_seg))
        return afg_fail(ctx, AFG_ERR_ARG, "psd_estimate: epochs reach past the end of x (or too many epochs)");
    return launch_psd(ctx, x, n, n_det, n_psd, psd_step, psd_span, psd, S(stream));
}

static int check_whiten(afg_ctx *ctx, int64_t n, int64_t n_psd, int64_t out_first, int64_t out_len, int64_t epoch_len) {
    const int half = ctx->cfg.fir_len / 2;
    if (n_psd < 1) return afg_fail(ctx, AFG_ERR_ARG, "whiten: n_psd must be >= 1");
    if (out_len < 0) return afg_fail(ctx, AFG_ERR_ARG, "whiten: out_len < 0");
    if (out_first < half) return afg_fail(ctx, AFG_ERR_ARG, "whiten: out_first must be >= fir_len/2 (crop)");
    if (out_first + out_len + half - 1 > n)
        return afg_fail(ctx, AFG_ERR_ARG, "whiten: outputs reach within fir_len/2 of the end of x (crop)");
    if (epoch_len < 0 || (epoch_len > 0 && epoch_len % WB))
        return afg_fail(ctx, AFG_ERR_ARG, "whiten: epoch_len must be 0 or a multiple of 8192");
    return AFG_OK;
}

int afg_whiten(afg_ctx *ctx, const float *x, int64_t n, int32_t n_det, const double *psd, int64_t n_psd,
               int64_t out_first, int64_t out_len, int64_t epoch_len, float *y, void *stream) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    if (!x || !psd || (!y && out_len > 0) || n_det < 1)
        return afg_fail(ctx, AFG_ERR_ARG, "whiten: null pointer or n_det < 1");
    int rc = check_whiten(ctx, n, n_psd, out_first, out_len, epoch_len);
    if (rc) return rc;
    return launch_whiten(ctx, x, n, n_det, psd, n_psd, out_first, out_len, epoch_len, y, out_len, S(stream));
}

static int infer(afg_ctx *ctx, const float *y, int64_t n_y, int64_t y_stride, int64_t first, int64_t stride,
                 int64_t n_win, int64_t shift, float *logits, cudaStream_t st) {
    if (n_win == 0) return AFG_OK;
    if (ctx->cfg.precision == AFG_BF16)
        return launch_infer_bf16(ctx, y, n_y, y_stride, first, stride, n_win, shift, logits, st);
    return launch_infer_fp32(ctx, y, n_y, y_stride, first, stride, n_win, shift, logits, st);
}

int afg_infer_windows(afg_ctx *ctx, const float *y, int64_t n_y, int64_t first, int64_t stride, int64_t n_win,
                      int64_t shift, float *logits, void *stream) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    const int W = ctx->cfg.win_len;
    if (!y || (!logits && n_win > 0) || n_win < 0 || stride < 1 || first < 0)
        return afg_fail(ctx, AFG_ERR_ARG, "infer_windows: bad pointer, n_win, stride or first");
    if (n_win > 0 && first + (n_win - 1) * stride + W > n_y)
        return afg_fail(ctx, AFG_ERR_ARG, "infer_windows: last window reaches past n_y");
    if (shift < 0 || shift >= n_y) return afg_fail(ctx, AFG_ERR_ARG, "infer_windows: shift must be in [0, n_y)");
    return infer(ctx, y, n_y, n_y, first, stride, n_win, shift, logits, S(stream));
}

int afg_integrate(afg_ctx *ctx, const float *logits, int64_t n_win, int32_t n_int, int32_t cluster_half,
                  float *stat, int64_t *trig_idx, int64_t trig_cap, int64_t *n_trig, void *stream) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    if (!logits || !stat || !n_trig || (trig_cap > 0 && !trig_idx) || trig_cap < 0)
        return afg_fail(ctx, AFG_ERR_ARG, "integrate: null pointer");
    if (n_int < 1 || n_win < n_int) return afg_fail(ctx, AFG_ERR_ARG, "integrate: need n_win >= n_int >= 1");
    if (cluster_half < 0) return afg_fail(ctx, AFG_ERR_ARG, "integrate: cluster_half < 0");
    return launch_integrate(ctx, logits, n_win, n_int, cluster_half, stat, trig_idx, trig_cap, n_trig, S(stream));
}

int afg_analyze(afg_ctx *ctx, const float *x, const afg_run_params *p, float *logits, float *stat,
                int64_t *trig_idx, int64_t trig_cap, int64_t *n_trig, void *stream) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    if (!x || !p || !logits || !stat || !n_trig) return afg_fail(ctx, AFG_ERR_ARG, "analyze: null pointer");
    const cudaStream_t st = S(stream);
    const int F = ctx->cfg.fir_len, half = F / 2, W = ctx->cfg.win_len, hop = ctx->cfg.hop;
    if (p->n_win < p->n_int || p->n_int < 1 || p->stride < 1 || p->cluster_half < 0)
        return afg_fail(ctx, AFG_ERR_ARG, "analyze: need n_win >= n_int >= 1, stride >= 1");
    int64_t n_psd, psd_step, psd_span, out_first, out_len;
    if (p->epoch_len == 0) {
        if (p->n_raw < NFFT || p->n_raw < F + W)
            return afg_fail(ctx, AFG_ERR_ARG, "analyze: plain span shorter than one Welch segment");
        n_psd = 1;
        psd_step = 0;
        psd_span = (p->n_raw - NFFT) / hop * hop + NFFT;
        out_first = half;
        out_len = p->n_raw - F;
    } else {
        if (p->epoch_len % WB || p->psd_len < NFFT || (p->psd_len - NFFT) % hop || p->epoch_len % hop)
            return afg_fail(ctx, AFG_ERR_ARG, "analyze: epoch_len must be a multiple of 8192, psd_len nfft + k*hop");
        const int64_t need = (p->n_win - 1) * p->stride + W;
        n_psd = (need + p->epoch_len - 1) / p->epoch_len;
        psd_step = p->epoch_len;
        psd_span = p->psd_len;
        out_first = p->psd_len;
        out_len = n_psd * p->epoch_len;
        if (out_first + out_len + half - 1 > p->n_raw)
            return afg_fail(ctx, AFG_ERR_ARG, "analyze: n_raw %lld too short for %lld epochs (need %lld)",
                            (long long)p->n_raw, (long long)n_psd, (long long)(out_first + out_len + half - 1));
    }
    const int64_t n_y = out_len;
    if ((p->n_win - 1) * p->stride + W > n_y) return afg_fail(ctx, AFG_ERR_ARG, "analyze: windows exceed the whitened span");
    if (p->shift < 0 || p->shift >= n_y) return afg_fail(ctx, AFG_ERR_ARG, "analyze: shift must be in [0, n_y)");
    double *psd = nullptr;
    float *white = nullptr;
    int rc = afg_ws_reserve(ctx, WS_PSD, (size_t)2 * n_psd * NBIN * sizeof(double), (void **)&psd);
    if (!rc) rc = afg_ws_reserve(ctx, WS_WHITE, (size_t)2 * n_y * sizeof(float), (void **)&white);
    if (!rc) rc = launch_psd(ctx, x, p->n_raw, 2, n_psd, psd_step, psd_span, psd, st);
    if (!rc) rc = launch_whiten(ctx, x, p->n_raw, 2, psd, n_psd, out_first, out_len, p->epoch_len, white, n_y, st);
    if (!rc) rc = infer(ctx, white, n_y, n_y, 0, p->stride, p->n_win, p->shift, logits, st);
    if (!rc) rc = launch_integrate(ctx, logits, p->n_win, p->n_int, p->cluster_half, stat, trig_idx, trig_cap, n_trig, st);
    return rc;
}

int afg_analyze_host(afg_ctx *ctx, const float *x_host, const afg_run_params *p, float *stat_host,
                     int64_t *trig_idx_host, int64_t trig_cap, int64_t *n_trig_host, void *stream) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    if (!x_host || !p || !stat_host || !n_trig_host || trig_cap < 0 || (trig_cap > 0 && !trig_idx_host))
        return afg_fail(ctx, AFG_ERR_ARG, "analyze_host: null pointer");
    if (p->n_raw < 1 || p->n_win < p->n_int || p->n_int < 1) return afg_fail(ctx, AFG_ERR_ARG, "analyze_host: sizes");
    const cudaStream_t st = S(stream);
    const int64_t n_stat = p->n_win - p->n_int + 1;
    float *x = nullptr, *logits = nullptr, *stat = nullptr;
    int64_t *trig = nullptr;
    int rc = afg_ws_reserve(ctx, WS_X, (size_t)2 * p->n_raw * sizeof(float), (void **)&x);
    if (!rc) rc = afg_ws_reserve(ctx, WS_LOGITS, (size_t)p->n_win * sizeof(float), (void **)&logits);
    if (!rc) rc = afg_ws_reserve(ctx, WS_STAT, (size_t)n_stat * sizeof(float), (void **)&stat);
    if (!rc) rc = afg_ws_reserve(ctx, WS_TRIG, (size_t)(trig_cap + 1) * sizeof(int64_t), (void **)&trig);
    if (rc) return rc;
    AFG_CUDA(ctx, cudaMemcpyAsync(x, x_host, (size_t)2 * p->n_raw * sizeof(float), cudaMemcpyHostToDevice, st));
    rc = afg_analyze(ctx, x, p, logits, stat, trig + 1, trig_cap, trig, stream);
    if (rc) return rc;
    AFG_CUDA(ctx, cudaMemcpyAsync(stat_host, stat, (size_t)n_stat * sizeof(float), cudaMemcpyDeviceToHost, st));
    AFG_CUDA(ctx, cudaMemcpyAsync(n_trig_host, trig, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    if (trig_cap > 0)
        AFG_CUDA(ctx, cudaMemcpyAsync(trig_idx_host, trig + 1, (size_t)trig_cap * sizeof(int64_t),
                                      cudaMemcpyDeviceToHost, st));
    AFG_CUDA(ctx, cudaStreamSynchronize(st));
    return AFG_OK;
}

int afg_autotune(afg_ctx *ctx, int64_t n_win, void *stream) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    if (net_tc_tiny_tunable(ctx)) return net_tc_tiny_autotune(ctx, n_win, S(stream));
    return net_tc_autotune(ctx, n_win, S(stream));
}

int afg_fused_tuning_get(afg_ctx *ctx, afg_fused_tuning *out) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    if (!out) return afg_fail(ctx, AFG_ERR_ARG, "fused_tuning_get: null output");
    return net_tc_tiny_tuning_get(ctx, out);
}

int afg_fused_tuning_candidates(afg_ctx *ctx, afg_fused_tuning *out, int32_t cap, int32_t *n_out) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    if (!n_out || cap < 0 || (cap > 0 && !out))
        return afg_fail(ctx, AFG_ERR_ARG, "fused_tuning_candidates: bad output arguments");
    int n = 0;
    int rc = net_tc_tiny_tuning_candidates(ctx, out, cap, &n);
    *n_out = n;
    return rc;
}

int afg_fused_tuning_set(afg_ctx *ctx, const afg_fused_tuning *in) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    if (!in) return afg_fail(ctx, AFG_ERR_ARG, "fused_tuning_set: null input");
    return net_tc_tiny_tuning_set(ctx, in);
}

int afg_tiles_get(afg_ctx *ctx, afg_tile *out, int32_t cap, int32_t *n_out) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    if (!n_out || cap < 0 || (cap > 0 && !out)) return afg_fail(ctx, AFG_ERR_ARG, "tiles_get: bad output arguments");
    int n = 0;
    int rc = net_tc_tiles_get(ctx, out, cap, &n);
    *n_out = n;
    return rc;
}

int afg_tile_candidates(afg_ctx *ctx, int32_t layer, afg_tile *out, int32_t cap, int32_t *n_out) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    if (!n_out || cap < 0 || (cap > 0 && !out))
        return afg_fail(ctx, AFG_ERR_ARG, "tile_candidates: bad output arguments");
    int n = 0;
    int rc = net_tc_tile_candidates(ctx, layer, out, cap, &n);
    *n_out = n;
    return rc;
}

int afg_tiles_set(afg_ctx *ctx, const afg_tile *tiles, int32_t n) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    if (n < 0 || (n > 0 && !tiles)) return afg_fail(ctx, AFG_ERR_ARG, "tiles_set: bad arguments");
    return net_tc_tiles_set(ctx, tiles, n);
}

int afg_far(afg_ctx *ctx, const float *bg_stat, const int64_t *bg_idx, const int64_t *n_bg_dev, int64_t bg_cap,
            double livetime_s, const float *fg, int64_t n_fg, int64_t *n_above, double *far, float *bg_sorted,
            void *stream) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    if (!bg_stat || !n_bg_dev || bg_cap < 0 || n_fg < 0 || (n_fg > 0 && !fg))
        return afg_fail(ctx, AFG_ERR_ARG, "far: null input or negative size");
    if (!(livetime_s > 0.0)) return afg_fail(ctx, AFG_ERR_ARG, "far: livetime_s must be > 0");
    return launch_far(ctx, bg_stat, bg_idx, n_bg_dev, bg_cap, livetime_s, fg, n_fg, n_above, far, bg_sorted,
                      S(stream));
}

int afg_trigger_times(const afg_ctx *ctx, const afg_run_params *p, const int64_t *idx, int64_t n, double t0,
                      double gap_s, double *t_peak, double *t_c) {
    if (!ctx || !p || n < 0 || (n > 0 && !idx)) return AFG_ERR_ARG;
    const double fs = (double)ctx->cfg.fs;
    const int64_t base = p->epoch_len == 0 ? ctx->cfg.fir_len / 2 : p->psd_len;
    const int64_t n_stat = p->n_win - p->n_int + 1;
    for (int64_t i = 0; i < n; ++i)
        if (idx[i] < 0 || idx[i] >= n_stat) return AFG_ERR_ARG;
    for (int64_t i = 0; i < n; ++i) {
        const double tp = t0 + (double)(base + (idx[i] + p->n_int - 1) * p->stride + ctx->cfg.win_len) / fs;
        if (t_peak) t_peak[i] = tp;
        if (t_c) t_c[i] = tp - (double)((int64_t)(p->n_int - 1) * p->stride) / fs - gap_s;
    }
    return AFG_OK;
}

int afg_resample_size(int64_t n_in, int32_t factor, int64_t *n_out, int64_t *first_input) {
    if (!n_out || n_in < 0 || factor < 2 || factor > 16) return AFG_ERR_ARG;
    int64_t j0 = 0;
    *n_out = resample_count(n_in, factor, &j0);
    if (first_input) *first_input = j0 * factor;
    return AFG_OK;
}

int afg_resample(afg_ctx *ctx, const float *x, int64_t n_in, int32_t n_det, int64_t x_stride, int32_t factor, float *y,
                 int64_t y_stride, int64_t *n_out, void *stream) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    if (!x || !y || n_in < 0 || n_det < 1 || factor < 2 || factor > 16)
        return afg_fail(ctx, AFG_ERR_ARG, "resample: null pointer, n_in < 0, n_det < 1 or factor outside 2..16");
    if (x_stride == 0) x_stride = n_in;
    const int64_t cnt = resample_count(n_in, factor, nullptr);
    if (y_stride == 0) y_stride = cnt;
    if (x_stride < n_in || y_stride < cnt) return afg_fail(ctx, AFG_ERR_ARG, "resample: row strides too small");
    return launch_resample(ctx, x, n_in, n_det, x_stride, factor, y, y_stride, n_out, S(stream));
}

}  // extern "C"
