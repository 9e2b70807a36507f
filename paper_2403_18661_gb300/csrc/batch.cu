// Timeslide background batches (Sec. IX: Hanford held fixed, Livingston
// shifted in 1 s steps until the required livetime is reached; every trigger
// of a shifted series is background) over many uneven strain segments, each
// whitened once per detector in epoch mode (Sec. VI).
//
// Per call: Welch + filter + whitening of every segment (4 launches per
// segment), one persistent network launch over every (segment, timeslide,
// window), and four launches for the integration and clustering of every
// series.  With use_graph the whole sequence is captured into a CUDA graph
// on the first call and replayed while the arguments are unchanged.
#include <string.h>

#include <algorithm>
#include <vector>

#include "afg_internal.cuh"

namespace {

struct SeriesDesc {
    int64_t logit_off;  // first logit of the series
    int64_t stat_off;   // first statistic sample of the series
    int64_t n_win;      // windows of the series
};

struct Plan {
    std::vector<SegDesc> segs;
    std::vector<SeriesDesc> series;
    std::vector<int64_t> n_ep;
    int64_t total_white = 0, total_win = 0, total_stat = 0, max_ep = 0, max_nseg = 0, max_nstat = 0;
};

int make_plan(afg_ctx *ctx, const afg_segment *segs, int n_seg, const afg_batch_params *p, Plan &P) {
    const int W = ctx->cfg.win_len, half = ctx->cfg.fir_len / 2, hop = ctx->cfg.hop;
    if (!segs || n_seg < 1 || !p) return afg_fail(ctx, AFG_ERR_ARG, "batch: no segments");
    if (p->epoch_len <= 0 || p->epoch_len % WB || p->epoch_len % hop || p->psd_len < NFFT ||
        (p->psd_len - NFFT) % hop || p->stride < 1 || p->n_shift < 1 || p->shift_step < 0 || p->n_int < 1 ||
        p->cluster_half < 0 || p->shift_first < 0 || p->shift_first > (int64_t)1 << 40)
        return afg_fail(ctx, AFG_ERR_ARG, "batch: bad parameters");
    const int64_t k0 = p->shift_first > 0 ? p->shift_first : 1;  // first timeslide of this call
    P = Plan();
    for (int i = 0; i < n_seg; ++i) {
        const int64_t n = segs[i].n_raw;
        const int64_t n_ep = (n - p->psd_len - half) / p->epoch_len;
        if (segs[i].offset < 0 || n_ep < 1)
            return afg_fail(ctx, AFG_ERR_ARG, "batch: segment %d (%lld samples) is shorter than look-back + one epoch",
                            i, (long long)n);
        const int64_t n_white = n_ep * p->epoch_len;
        const int64_t n_win = n_white >= W ? (n_white - W) / p->stride + 1 : 0;
        if (n_win < p->n_int)
            return afg_fail(ctx, AFG_ERR_ARG, "batch: segment %d has %lld windows, fewer than n_int", i,
                            (long long)n_win);
        if ((k0 + p->n_shift - 1) * p->shift_step >= n_white)
            return afg_fail(ctx, AFG_ERR_ARG, "batch: segment %d is shorter than the largest timeslide", i);
        SegDesc d;
        d.y_off = P.total_white;
        d.n_y = n_white;
        d.n_win = n_win;
        d.win_first = P.total_win;
        d.shift_first = k0;
        P.segs.push_back(d);
        P.n_ep.push_back(n_ep);
        for (int k = 0; k < p->n_shift; ++k) {
            SeriesDesc s;
            s.logit_off = P.total_win + (int64_t)k * n_win;
            s.stat_off = P.total_stat;
            s.n_win = n_win;
            P.series.push_back(s);
            P.total_stat += n_win - p->n_int + 1;
        }
        P.total_white += n_white;
        P.total_win += (int64_t)p->n_shift * n_win;
        P.max_ep = std::max(P.max_ep, n_ep);
        const int64_t K = (p->psd_len - NFFT) / hop + 1;
        P.max_nseg = std::max(P.max_nseg, (n_ep - 1) * (p->epoch_len / hop) + K);
        P.max_nstat = std::max(P.max_nstat, n_win - p->n_int + 1);
    }
    return AFG_OK;
}

// ---------------------------------------------------------------- kernels
__global__ void k_integrate_multi(const float *__restrict__ logits, const SeriesDesc *__restrict__ sd, int n_int,
                                  float *__restrict__ stat) {
    const SeriesDesc d = sd[blockIdx.y];
    const int64_t n_out = d.n_win - n_int + 1;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_out) return;
    float s = 0.f;
    for (int i = 0; i < n_int; ++i) s += logits[d.logit_off + j + i];
    stat[d.stat_off + j] = s / (float)n_int;
}

constexpr int TT = 1024;

// One CTA per series: flag the cluster maxima of its statistic (earliest
// index wins ties) and either count them (WRITE = false, into cnt[s]) or write
// their global statistic indices from offset cnt[s] on (WRITE = true).
template <bool WRITE>
__global__ void __launch_bounds__(TT) k_trig_multi(const float *__restrict__ stat, const SeriesDesc *__restrict__ sd,
                                                   int n_int, int half, int64_t *__restrict__ cnt,
                                                   int64_t *__restrict__ idx, int64_t cap) {
    __shared__ int warp_tot[TT / 32];
    __shared__ int64_t base_s;
    const SeriesDesc d = sd[blockIdx.x];
    const int64_t n = d.n_win - n_int + 1;
    const float *I = stat + d.stat_off;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) base_s = WRITE ? cnt[blockIdx.x] : 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < n; c0 += TT) {
        const int64_t j = c0 + tid;
        int flag = 0;
        if (j < n) {
            const float v = I[j];
            flag = 1;
            const int64_t lo = j - half < 0 ? 0 : j - half;
            const int64_t hi = j + half >= n ? n - 1 : j + half;
            for (int64_t i = lo; i < j && flag; ++i) flag = v > I[i];
            for (int64_t i = j + 1; i <= hi && flag; ++i) flag = v >= I[i];
        }
        const unsigned m = __ballot_sync(0xffffffffu, flag);
        if (lane == 0) warp_tot[wid] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < TT / 32; ++w) {
            const int t = warp_tot[w];
            if (w < wid) before += t;
            total += t;
        }
        const int64_t base = base_s;
        if (WRITE && flag) {
            const int64_t pos = base + before + __popc(m & ((1u << lane) - 1u));
            if (pos < cap) idx[pos] = d.stat_off + j;
        }
        __syncthreads();
        if (tid == 0) base_s = base + total;
        __syncthreads();
    }
    if (!WRITE && tid == 0) cnt[blockIdx.x] = base_s;
}

// exclusive prefix sum of cnt[0..n) in place (one CTA); total -> *n_trig
__global__ void __launch_bounds__(TT) k_scan_counts(int64_t *__restrict__ cnt, int n, int64_t *__restrict__ n_trig) {
    __shared__ int64_t part[TT];
    const int tid = threadIdx.x;
    const int per = (n + TT - 1) / TT;
    const int lo = tid * per, hi = min(n, lo + per);
    int64_t s = 0;
    for (int i = lo; i < hi; ++i) s += cnt[i];
    part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        int64_t run = 0;
        for (int t = 0; t < TT; ++t) {
            const int64_t v = part[t];
            part[t] = run;
            run += v;
        }
        *n_trig = run;
    }
    __syncthreads();
    int64_t run = part[tid];
    for (int i = lo; i < hi; ++i) {
        const int64_t v = cnt[i];
        cnt[i] = run;
        run += v;
    }
}

struct GraphKey {
    const void *x, *logits, *stat, *trig, *ntrig, *stream;
    int64_t x_len, trig_cap;
    afg_batch_params p;
    uint64_t seg_hash;
    int n_seg;
};

uint64_t hash_segs(const afg_segment *s, int n) {
    uint64_t h = 1469598103934665603ull;
    const unsigned char *b = reinterpret_cast<const unsigned char *>(s);
    for (size_t i = 0; i < (size_t)n * sizeof(afg_segment); ++i) h = (h ^ b[i]) * 1099511628211ull;
    return h;
}

struct BatchGraph {
    bool valid = false;
    GraphKey key;
    cudaGraphExec_t exec = nullptr;
    int64_t launches[KK_COUNT] = {};
    double flops[KK_COUNT] = {}, bytes[KK_COUNT] = {};
};

}  // namespace

// per-context graph cache
struct BatchCache {
    BatchGraph g;
};

void batch_cache_release(afg_ctx *ctx) {
    if (!ctx->batch) return;
    if (ctx->batch->g.exec) cudaGraphExecDestroy(ctx->batch->g.exec);
    delete ctx->batch;
    ctx->batch = nullptr;
}

static int enqueue(afg_ctx *ctx, const Plan &P, const float *x, int64_t x_len, const afg_batch_params *p,
                   const SegDesc *segs_dev, const SeriesDesc *series_dev, int64_t *cnt, double *psd, float *white,
                   float *logits, float *stat, int64_t *trig_idx, int64_t trig_cap, int64_t *n_trig,
                   const afg_segment *segs, cudaStream_t st) {
    const int n_seg = (int)P.segs.size();
    for (int i = 0; i < n_seg; ++i) {
        const float *xs = x + segs[i].offset;
        int rc = launch_psd(ctx, xs, segs[i].n_raw, 2, P.n_ep[i], p->epoch_len, p->psd_len, psd, st, x_len);
        if (!rc)
            rc = launch_whiten(ctx, xs, segs[i].n_raw, 2, psd, P.n_ep[i], p->psd_len, P.segs[i].n_y, p->epoch_len,
                               white + P.segs[i].y_off, P.total_white, st, x_len);
        if (rc) return rc;
    }
    int rc;
    if (ctx->cfg.precision == AFG_BF16) {
        rc = launch_infer_bf16_batch(ctx, white, P.total_white, segs_dev, n_seg, P.total_win, p->stride,
                                     p->shift_step, logits, st);
    } else {
        rc = AFG_OK;
        for (int i = 0; i < n_seg && !rc; ++i)
            for (int k = 0; k < p->n_shift && !rc; ++k) {
                const SegDesc &d = P.segs[i];
                rc = launch_infer_fp32(ctx, white + d.y_off, d.n_y, P.total_white, 0, p->stride, d.n_win,
                                       ((d.shift_first + k) * p->shift_step) % d.n_y,
                                       logits + d.win_first + (int64_t)k * d.n_win, st);
            }
    }
    if (rc) return rc;
    const int n_series = (int)P.series.size();
    {
        KScope ks(ctx, st, KK_INTEGRATE, (double)P.total_stat * p->n_int, (double)(P.total_win + P.total_stat) * 4.0);
        k_integrate_multi<<<dim3((unsigned)((P.max_nstat + 255) / 256), (unsigned)n_series), 256, 0, st>>>(
            logits, series_dev, p->n_int, stat);
    }
    AFG_LAUNCH_CHECK(ctx, "k_integrate_multi");
    {
        KScope ks(ctx, st, KK_TRIGGERS, 0.0, (double)P.total_stat * 4.0);
        k_trig_multi<false><<<n_series, TT, 0, st>>>(stat, series_dev, p->n_int, p->cluster_half, cnt, nullptr, 0);
    }
    {
        KScope ks(ctx, st, KK_TRIGGERS, 0.0, (double)n_series * 16.0);
        k_scan_counts<<<1, TT, 0, st>>>(cnt, n_series, n_trig);
    }
    {
        KScope ks(ctx, st, KK_TRIGGERS, 0.0, (double)P.total_stat * 4.0);
        k_trig_multi<true><<<n_series, TT, 0, st>>>(stat, series_dev, p->n_int, p->cluster_half, cnt, trig_idx,
                                                   trig_cap);
    }
    AFG_LAUNCH_CHECK(ctx, "k_trig_multi");
    return AFG_OK;
}

extern "C" int afg_batch_layout(afg_ctx *ctx, const afg_segment *segs_host, int32_t n_seg,
                                const afg_batch_params *p, int64_t *n_win_host, int64_t *total_windows,
                                int64_t *total_stat) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    Plan P;
    int rc = make_plan(ctx, segs_host, n_seg, p, P);
    if (rc) return rc;
    if (n_win_host)
        for (int i = 0; i < n_seg; ++i) n_win_host[i] = P.segs[i].n_win;
    if (total_windows) *total_windows = P.total_win;
    if (total_stat) *total_stat = P.total_stat;
    return AFG_OK;
}

extern "C" int afg_batch_run(afg_ctx *ctx, const float *x, int64_t x_len, const afg_segment *segs_host, int32_t n_seg,
                             const afg_batch_params *p, float *logits, float *stat, int64_t *trig_idx,
                             int64_t trig_cap, int64_t *n_trig, void *stream) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    if (!x || !stat || !n_trig || trig_cap < 0 || (trig_cap > 0 && !trig_idx))
        return afg_fail(ctx, AFG_ERR_ARG, "batch_run: null pointer");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const bool graph = p && p->use_graph && st != nullptr;
    if (graph && ctx->batch && ctx->batch->g.valid) {
        const GraphKey &k = ctx->batch->g.key;
        if (k.x == x && k.logits == logits && k.stat == stat && k.trig == trig_idx && k.ntrig == n_trig &&
            k.stream == stream && k.x_len == x_len && k.trig_cap == trig_cap && k.n_seg == n_seg &&
            memcmp(&k.p, p, sizeof *p) == 0 && k.seg_hash == hash_segs(segs_host, n_seg)) {
            AFG_CUDA(ctx, cudaGraphLaunch(ctx->batch->g.exec, st));
            for (int i = 0; i < KK_COUNT; ++i) {
                ctx->prof.launches[i] += ctx->batch->g.launches[i];
                ctx->prof.flops[i] += ctx->batch->g.flops[i];
                ctx->prof.bytes[i] += ctx->batch->g.bytes[i];
            }
            return AFG_OK;
        }
    }
    Plan P;
    int rc = make_plan(ctx, segs_host, n_seg, p, P);
    if (rc) return rc;
    for (int i = 0; i < n_seg; ++i)
        if (segs_host[i].offset + segs_host[i].n_raw > x_len)
            return afg_fail(ctx, AFG_ERR_ARG, "batch_run: segment %d reaches past x_len", i);
    // every workspace at its final size before anything is queued (graph capture allows no allocation)
    const int hop = ctx->cfg.hop;
    (void)hop;
    double *psd = nullptr;
    float *white = nullptr, *lg = logits;
    void *tmp = nullptr;
    SegDesc *segs_dev = nullptr;
    SeriesDesc *series_dev = nullptr;
    rc = afg_ws_reserve(ctx, WS_PSD, (size_t)2 * P.max_ep * NBIN * sizeof(double), (void **)&psd);
    if (!rc) rc = afg_ws_reserve(ctx, WS_WHITE, (size_t)2 * P.total_white * sizeof(float), (void **)&white);
    if (!rc) rc = afg_ws_reserve(ctx, WS_PERIODOGRAM, (size_t)2 * P.max_nseg * NBIN * sizeof(double), &tmp);
    if (!rc) rc = afg_ws_reserve(ctx, WS_FILTER, (size_t)2 * P.max_ep * NBIN * sizeof(float), &tmp);
    if (!rc && !lg) rc = afg_ws_reserve(ctx, WS_LOGITS, (size_t)P.total_win * sizeof(float), (void **)&lg);
    if (!rc) rc = afg_ws_reserve(ctx, WS_BATCH_SEGS, P.segs.size() * sizeof(SegDesc), (void **)&segs_dev);
    const size_t ser_bytes = P.series.size() * sizeof(SeriesDesc);
    if (!rc) rc = afg_ws_reserve(ctx, WS_BATCH_SERIES, ser_bytes + P.series.size() * sizeof(int64_t) + 256,
                                 (void **)&series_dev);
    if (rc) return rc;
    int64_t *cnt = reinterpret_cast<int64_t *>(reinterpret_cast<char *>(series_dev) + ((ser_bytes + 255) / 256) * 256);
    if (ctx->cfg.precision == AFG_FP32) {
        // the FP32 network's activation workspaces at the size of the longest series
        int64_t max_win = 0;
        for (const SegDesc &d : P.segs) max_win = std::max(max_win, d.n_win);
        int64_t per_win = ctx->plan.max_act_per_window * (int64_t)sizeof(float);
        int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(max_win, ((int64_t)4 << 30) / per_win));
        chunk = std::min<int64_t>(chunk, 16384);
        for (int i = 0; i < 4 && !rc; ++i) rc = afg_ws_reserve(ctx, WS_ACT0 + i, (size_t)(chunk * per_win), &tmp);
        if (rc) return rc;
    }
    // descriptors are uploaded synchronously: they are constant for a captured graph
    AFG_CUDA(ctx, cudaMemcpy(segs_dev, P.segs.data(), P.segs.size() * sizeof(SegDesc), cudaMemcpyHostToDevice));
    AFG_CUDA(ctx, cudaMemcpy(series_dev, P.series.data(), ser_bytes, cudaMemcpyHostToDevice));
    if (!graph)
        return enqueue(ctx, P, x, x_len, p, segs_dev, series_dev, cnt, psd, white, lg, stat, trig_idx, trig_cap,
                       n_trig, segs_host, st);
    // capture
    if (!ctx->batch) ctx->batch = new BatchCache();
    BatchGraph &g = ctx->batch->g;
    if (g.exec) {
        cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
    }
    g.valid = false;
    int64_t l0[KK_COUNT];
    double f0[KK_COUNT], b0[KK_COUNT];
    memcpy(l0, ctx->prof.launches, sizeof l0);
    memcpy(f0, ctx->prof.flops, sizeof f0);
    memcpy(b0, ctx->prof.bytes, sizeof b0);
    AFG_CUDA(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    rc = enqueue(ctx, P, x, x_len, p, segs_dev, series_dev, cnt, psd, white, lg, stat, trig_idx, trig_cap, n_trig,
                 segs_host, st);
    cudaGraph_t graph_obj = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &graph_obj);
    if (rc) {
        if (graph_obj) cudaGraphDestroy(graph_obj);
        return rc;
    }
    if (e != cudaSuccess) return afg_cuda_fail(ctx, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&g.exec, graph_obj, 0);
    cudaGraphDestroy(graph_obj);
    if (e != cudaSuccess) return afg_cuda_fail(ctx, e, "cudaGraphInstantiate");
    for (int i = 0; i < KK_COUNT; ++i) {
        g.launches[i] = ctx->prof.launches[i] - l0[i];
        g.flops[i] = ctx->prof.flops[i] - f0[i];
        g.bytes[i] = ctx->prof.bytes[i] - b0[i];
    }
    g.key = GraphKey{x, logits, stat, trig_idx, n_trig, stream, x_len, trig_cap, *p, hash_segs(segs_host, n_seg),
                     n_seg};
    g.valid = true;
    AFG_CUDA(ctx, cudaGraphLaunch(g.exec, st));
    return AFG_OK;
}
