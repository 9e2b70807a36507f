// Streaming detection with continuous batching (Sec. VI: clients stream
// strain updates to a snapshotter that caches the overlapping state, a
// whitener estimates the PSD from the first 64 s of that state and whitens
// the rest, and the network analyses overlapping windows; Sec. II: the
// outputs are integrated with a 1 s top-hat).
//
// Per stream, on the device: a mirrored ring of raw strain (every span of up
// to R samples is contiguous), a mirrored ring of whitened strain, the
// whitening gains of two epochs, and a ring of logits.  Whitened
// sample j of a stream is raw sample psd_len + j, whitened with the PSD of
// raw [e * epoch_len, e * epoch_len + psd_len), e = j / epoch_len (the 64 s
// before its epoch); window w covers whitened [w * stride, w * stride + W).
//
// The engine (one host thread per context) forms a step from every chunk
// pushed so far: one H2D copy and a scatter kernel into the raw rings, one
// whitening launch for every stream's new samples, one network launch for
// every new window (whose last CTA also integrates them in small steps; an
// integration launch in large ones) and one D2H copy.  PSD and filter
// refreshes are enqueued after a step's result event, as soon as a stream's
// raw strain covers the 64 s before an epoch, ahead of that epoch's first
// whitened sample; all of a step's refreshes are batched (per 16 streams: one
// periodogram launch, one mean launch, one filter build over every detector,
// one launch that copies the gains to the streams' slots).  Chunks pushed
// while a step runs join the next one; two steps may be in flight.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "afg_internal.cuh"

namespace {

constexpr int LR = STREAM_LR;  // logits ring per stream
constexpr double kPollS = 20e-3;  // the idle engine polls for pushes this long before it sleeps
constexpr int kFuseInteg = 64;   // steps with at most this many new statistics integrate in the network launch

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ScatterDesc {
    float *ring;      // raw ring, detector row 0 (row stride 2R)
    int64_t ring_n;   // R
    int64_t pos;      // slot of the first new sample (< R)
    int64_t n;        // new samples per detector
    int64_t src;      // offset of the chunk in the staging buffer ([2][n] per chunk)
};

// grid (n_desc): copy each staged chunk into its stream's mirrored raw ring
__global__ void k_scatter(const ScatterDesc *__restrict__ d, const float *__restrict__ stage) {
    pdl_trigger();
    const ScatterDesc s = d[blockIdx.x];
    for (int64_t i = threadIdx.x; i < 2 * s.n; i += blockDim.x) {
        const int det = i >= s.n;
        const int64_t k = i - det * s.n;
        int64_t m = s.pos + k;
        if (m >= s.ring_n) m -= s.ring_n;
        const float v = stage[s.src + i];
        float *row = s.ring + det * 2 * s.ring_n;
        row[m] = v;
        row[m + s.ring_n] = v;
    }
}

// one thread per new window: stat = mean of the last n_int logits (oldest first); for large
// steps, where the network launch's last CTA would integrate them one warp at a time
// (launched as a programmatic dependent of the network launch)
__global__ void k_stream_integrate(const IntegDesc *__restrict__ d, int n, int n_int) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const IntegDesc s = d[i < n ? i : 0];
    pdl_wait();  // logits of the network launch before
    if (i >= n) return;
    float acc = 0.f;
    for (int64_t j = s.w - n_int + 1; j <= s.w; ++j) acc += s.ring[j % LR];
    s.out[0] = acc / (float)n_int;
    s.out[1] = s.ring[s.w % LR];
}

struct Chunk {
    std::vector<float> data;  // [2][n]
    int64_t n;
    double t_push;
};

struct Slot {
    bool open = false, closing = false;
    float *raw = nullptr, *white = nullptr, *gains = nullptr, *logits = nullptr;
    void *mem = nullptr;
    int64_t bytes = 0;
    int64_t P = 0, Q = 0, n_win = 0;      // raw committed, whitened produced, windows evaluated
    int64_t gains_epoch[2] = {-1, -1};
    std::deque<Chunk> pending;
    std::vector<afg_stream_result> results;
    int inflight = 0;
    int64_t pushed = 0, delivered = 0;
};

struct PendingResult {
    int slot;
    int64_t w;
    double t_push;
};

struct StepBuf {
    bool busy = false;
    // one pinned host block and its device copy per step: the staged chunks, then the
    // step's scatter, whitening, window and integration descriptors (one H2D copy)
    float *h_stage = nullptr, *d_stage = nullptr;
    size_t stage_cap = 0, blk_bytes = 0;
    ScatterDesc *h_sc = nullptr;
    WhitenPiece *h_wp = nullptr;
    WinPtr *h_win = nullptr;
    IntegDesc *h_int = nullptr;
    float *d_out = nullptr, *h_out = nullptr;
    int cap_sc = 0, cap_wp = 0, cap_win = 0;
    int cap_rf = 0;  // gains-refresh rows per list (two detectors per refresh)
    cudaEvent_t ev = nullptr;
    std::vector<PendingResult> res;
    std::vector<int> slots;  // streams with chunks in this step
};

}  // namespace

struct ServeEngine {
    afg_ctx *ctx;
    afg_stream_params p;
    int64_t R, Wr, per_stream_new;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::atomic<uint64_t> pushes{0};  // chunks pushed so far (polled by the idle engine without the lock)
    bool stop = false;
    std::thread th;
    cudaStream_t st = nullptr;
    unsigned *d_done = nullptr;  // completion counter of the network launch (integration by its last CTA)
    StepBuf buf[2];
    int rb_rows = 0;                // rows (detector PSDs) per batched gains refresh
    double *d_rf_psd = nullptr;     // [rb_rows][NBIN] PSDs of a refresh batch
    float *d_rf_gains = nullptr;    // [rb_rows][NBIN] their gains, before the scatter to the streams' slots
    int err = AFG_OK;
    int64_t steps = 0, windows = 0, samples = 0;
};

namespace {

size_t align16(size_t n) { return (n + 15) & ~(size_t)15; }

int alloc_step(afg_ctx *ctx, StepBuf &b, int max_streams, int64_t per_stream_new, int64_t stride) {
    b.stage_cap = (size_t)max_streams * 2 * per_stream_new;
    b.cap_sc = max_streams;
    b.cap_wp = max_streams * (int)(per_stream_new / 512 + 3);  // pieces of >= 512 outputs, one epoch break
    b.cap_win = (int)(max_streams * (per_stream_new / stride + 2));
    b.cap_rf = 4 * max_streams;  // two epochs of two detectors per stream
    b.blk_bytes = align16(b.stage_cap * sizeof(float)) + align16(b.cap_sc * sizeof(ScatterDesc)) +
                  align16(b.cap_wp * sizeof(WhitenPiece)) + align16(b.cap_win * sizeof(WinPtr)) +
                  align16(b.cap_win * sizeof(IntegDesc)) + 2 * align16((size_t)b.cap_rf * 2 * sizeof(void *));
    AFG_CUDA(ctx, cudaHostAlloc(&b.h_stage, b.blk_bytes, cudaHostAllocDefault));
    AFG_CUDA(ctx, cudaMalloc(&b.d_stage, b.blk_bytes));
    AFG_CUDA(ctx, cudaHostAlloc(&b.h_sc, b.cap_sc * sizeof(ScatterDesc), cudaHostAllocDefault));
    AFG_CUDA(ctx, cudaHostAlloc(&b.h_wp, b.cap_wp * sizeof(WhitenPiece), cudaHostAllocDefault));
    AFG_CUDA(ctx, cudaHostAlloc(&b.h_win, b.cap_win * sizeof(WinPtr), cudaHostAllocDefault));
    AFG_CUDA(ctx, cudaHostAlloc(&b.h_int, b.cap_win * sizeof(IntegDesc), cudaHostAllocDefault));
    AFG_CUDA(ctx, cudaHostAlloc(&b.h_out, b.cap_win * 2 * sizeof(float), cudaHostAllocDefault));
    AFG_CUDA(ctx, cudaMalloc(&b.d_out, b.cap_win * 2 * sizeof(float)));
    AFG_CUDA(ctx, cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming));
    ctx->bytes_held += (int64_t)(b.blk_bytes + b.cap_win * 8);
    return AFG_OK;
}

void free_step(StepBuf &b) {
    cudaFreeHost(b.h_stage); cudaFree(b.d_stage);
    cudaFreeHost(b.h_sc);
    cudaFreeHost(b.h_wp);
    cudaFreeHost(b.h_win);
    cudaFreeHost(b.h_int);
    cudaFreeHost(b.h_out); cudaFree(b.d_out);
    if (b.ev) cudaEventDestroy(b.ev);
    b = StepBuf();
}

// Wait for a launched step and hand its results to the streams.
int complete(ServeEngine &E, StepBuf &b) {
    if (!b.busy) return AFG_OK;
    cudaError_t e = cudaEventSynchronize(b.ev);
    const double t_done = now_s();
    std::lock_guard<std::mutex> lock(E.mu);
    if (e != cudaSuccess) E.err = afg_cuda_fail(E.ctx, e, "stream step");
    for (size_t i = 0; i < b.res.size(); ++i) {
        const PendingResult &r = b.res[i];
        afg_stream_result o;
        o.window = r.w;
        o.stat = b.h_out[2 * i];
        o.logit = b.h_out[2 * i + 1];
        o.t_push = r.t_push;
        o.t_done = t_done;
        E.slots[r.slot].results.push_back(o);
        E.slots[r.slot].delivered++;
    }
    for (int s : b.slots) E.slots[s].inflight--;
    b.busy = false;
    b.res.clear();
    b.slots.clear();
    E.cv_done.notify_all();
    return AFG_OK;
}

// Gains refreshes of one list, batched: for every (slot, epoch) the PSD of raw [e * epoch_len,
// e * epoch_len + psd_len) of both detectors and their gains into the stream's gains slot e & 1.
// The host writes, into the step's staging block, the list's source rows (each detector's raw
// samples) followed by its destination rows (gains slots); per batch of rb_rows rows one
// periodogram launch, one mean launch and one filter build cover every row, and one launch
// copies the gains to their slots.
struct RefreshList {
    size_t off = 0;  // byte offset of the pointer rows in the staging block
    int n = 0;       // refreshes
};

void refresh_plan(ServeEngine &E, StepBuf &b, char *hb, RefreshList &L,
                  const std::vector<std::pair<int, int64_t>> &list) {
    const afg_stream_params &p = E.p;
    L.n = (int)list.size();
    const float **src = reinterpret_cast<const float **>(hb + L.off);
    float **dst = reinterpret_cast<float **>(hb + L.off) + b.cap_rf;
    for (int i = 0; i < L.n; ++i) {
        Slot &sl = E.slots[list[i].first];
        const int64_t e = list[i].second;
        const float *xr = sl.raw + (e * p.epoch_len) % E.R;
        float *g = sl.gains + (int64_t)(e & 1) * 2 * NBIN;
        src[2 * i] = xr;
        src[2 * i + 1] = xr + 2 * E.R;
        dst[2 * i] = g;
        dst[2 * i + 1] = g + NBIN;
        sl.gains_epoch[e & 1] = e;
    }
}

int refresh_run(ServeEngine &E, StepBuf &b, char *db, const RefreshList &L, cudaStream_t st) {
    afg_ctx *ctx = E.ctx;
    const float *const *src = reinterpret_cast<const float *const *>(db + L.off);
    float *const *dst = reinterpret_cast<float *const *>(db + L.off) + b.cap_rf;
    for (int r0 = 0; r0 < 2 * L.n; r0 += E.rb_rows) {
        const int nr = std::min(E.rb_rows, 2 * L.n - r0);
        int rc = launch_psd_rows(ctx, src + r0, nr, E.p.psd_len, E.d_rf_psd, st);
        if (!rc) rc = launch_filter(ctx, E.d_rf_psd, nr, 1, E.d_rf_gains, st);
        if (!rc) rc = launch_scatter_rows(ctx, E.d_rf_gains, dst + r0, nr, NBIN, st);
        if (rc) return rc;
    }
    return AFG_OK;
}

// Plan and launch one step from the pending chunks.  Returns 1 if a step was launched.
int launch_step(ServeEngine &E, StepBuf &b) {
    afg_ctx *ctx = E.ctx;
    const afg_stream_params &p = E.p;
    const int W = ctx->cfg.win_len, F = ctx->cfg.fir_len;
    struct Taken {
        int slot;
        std::vector<Chunk> chunks;
    };
    std::vector<Taken> taken;
    {
        std::lock_guard<std::mutex> lock(E.mu);
        for (int s = 0; s < (int)E.slots.size(); ++s) {
            Slot &sl = E.slots[s];
            if (!sl.open || sl.pending.empty()) continue;
            Taken t;
            t.slot = s;
            int64_t n = 0;
            while (!sl.pending.empty() && n + sl.pending.front().n <= E.per_stream_new) {
                n += sl.pending.front().n;
                t.chunks.push_back(std::move(sl.pending.front()));
                sl.pending.pop_front();
            }
            if (!t.chunks.empty()) {
                sl.inflight++;
                taken.push_back(std::move(t));
            }
        }
    }
    if (taken.empty()) return 0;
    const cudaStream_t st = E.st;
    int n_sc = 0, n_wp = 0, n_win = 0;
    size_t stage_off = 0;
    int64_t total_white = 0;
    b.res.clear();
    b.slots.clear();
    // 1) stage the chunks and describe their scatter into the raw rings
    std::vector<ScatterDesc> scs(taken.size());
    std::vector<int64_t> p_old(taken.size());
    for (size_t ti = 0; ti < taken.size(); ++ti) {
        Taken &t = taken[ti];
        Slot &sl = E.slots[t.slot];
        int64_t n = 0;
        for (Chunk &c : t.chunks) n += c.n;
        // rows: [det0 all chunks][det1 all chunks]
        int64_t k = 0;
        for (Chunk &c : t.chunks) {
            memcpy(b.h_stage + stage_off + k, c.data.data(), c.n * sizeof(float));
            memcpy(b.h_stage + stage_off + n + k, c.data.data() + c.n, c.n * sizeof(float));
            k += c.n;
        }
        ScatterDesc d;
        d.ring = sl.raw;
        d.ring_n = E.R;
        d.pos = sl.P % E.R;
        d.n = n;
        d.src = (int64_t)stage_off;
        scs[ti] = d;
        p_old[ti] = sl.P;
        stage_off += 2 * n;
        sl.P += n;
        b.slots.push_back(t.slot);
    }
    // 2) whitening pieces (and the gains refreshes they still need); 3) windows
    std::vector<std::pair<int, int64_t>> refresh;  // (slot, epoch) built after the scatter, before the pieces
    const int64_t piece_max = whiten_multi_piece_max(ctx);
    const bool staged = whiten_multi_takes_staging(ctx);
    std::vector<int> first_piece(taken.size(), -1);  // a stream's first piece also scatters its chunk
    for (size_t ti = 0; ti < taken.size(); ++ti) {
        Taken &t = taken[ti];
        Slot &sl = E.slots[t.slot];
        const double t_push = t.chunks.back().t_push;
        const int64_t q_new = std::max(sl.Q, sl.P - p.psd_len - F / 2 + 1);
        int64_t j = sl.Q;
        while (j < q_new) {
            const int64_t e = j / p.epoch_len;
            const int64_t end = std::min({q_new, (e + 1) * p.epoch_len, j + piece_max});
            const int slot_g = (int)(e & 1);
            if (sl.gains_epoch[slot_g] != e) {  // not built ahead (chunks longer than F/2)
                sl.gains_epoch[slot_g] = e;
                refresh.emplace_back(t.slot, e);
            }
            WhitenPiece wp;
            wp.x = sl.raw + (p.psd_len + j - F / 2) % E.R;
            wp.x_stride = 2 * E.R;
            wp.gains = sl.gains + (int64_t)slot_g * 2 * NBIN;
            wp.y = sl.white;
            wp.y_stride = 2 * E.Wr;
            wp.y_ring = E.Wr;
            wp.y_pos = j % E.Wr;
            wp.cnt = end - j;
            // samples from the step's chunks come straight from the staging copy
            wp.stg = staged ? b.d_stage + scs[ti].src : nullptr;
            wp.stg_stride = scs[ti].n;
            wp.i_new = p_old[ti] - (p.psd_len + j - F / 2);
            wp.sc_ring = nullptr;
            wp.sc_R = E.R;
            wp.sc_pos = scs[ti].pos;
            wp.sc_n = scs[ti].n;
            if (first_piece[ti] < 0) first_piece[ti] = n_wp;
            b.h_wp[n_wp++] = wp;
            total_white += end - j;
            j = end;
        }
        sl.Q = q_new;
        while (sl.n_win * p.stride + W <= sl.Q) {
            const int64_t w = sl.n_win++;
            WinPtr wptr;
            wptr.y0 = sl.white + (w * p.stride) % E.Wr;
            wptr.y1 = wptr.y0 + 2 * E.Wr;
            wptr.out = sl.logits + (w % LR);
            if (w >= p.n_int - 1) {
                IntegDesc id;
                id.ring = sl.logits;
                id.w = w;
                id.out = b.d_out + 2 * (int64_t)b.res.size();
                b.h_int[b.res.size()] = id;
                b.res.push_back(PendingResult{t.slot, w, t_push});
            }
            b.h_win[n_win++] = wptr;
        }
    }
    // Refreshes ahead of need: a stream whose raw strain now covers the 64 s before its current or
    // next epoch gets that epoch's PSD and gains, enqueued after this step's result event so that
    // no push waits for them.  The data is complete F/2 samples before the epoch's first output can
    // be whitened, so a later step (same CUDA stream) finds the gains built; the gains slot they
    // take held the epoch before the previous one, which no pending or later piece reads.
    std::vector<std::pair<int, int64_t>> ahead;
    for (Taken &t : taken) {
        Slot &sl = E.slots[t.slot];
        for (int64_t e = sl.Q / p.epoch_len; e <= sl.Q / p.epoch_len + 1; ++e)
            if (sl.gains_epoch[e & 1] != e && sl.P >= e * p.epoch_len + p.psd_len) {
                sl.gains_epoch[e & 1] = e;  // (set again by refresh_plan)
                ahead.emplace_back(t.slot, e);
            }
    }
    // Scatter: inside the whitening launch (a stream's first piece) unless a gains refresh must read
    // the new samples from the ring first, or the stream has no piece this step, or the whitening
    // kernel reads only the ring; those go through k_scatter.
    const bool fuse = staged && refresh.empty();
    for (size_t ti = 0; ti < taken.size(); ++ti) {
        if (fuse && first_piece[ti] >= 0) b.h_wp[first_piece[ti]].sc_ring = scs[ti].ring;
        else b.h_sc[n_sc++] = scs[ti];
    }
    if (!fuse)
        for (int i = 0; i < n_wp; ++i) b.h_wp[i].stg = nullptr;
    // one H2D copy: chunks, then the descriptors
    const int n_res = (int)b.res.size();
    char *hb = reinterpret_cast<char *>(b.h_stage), *db = reinterpret_cast<char *>(b.d_stage);
    size_t off = align16(stage_off * sizeof(float));
    const size_t o_sc = off;
    off += align16(n_sc * sizeof(ScatterDesc));
    const size_t o_wp = off;
    off += align16(n_wp * sizeof(WhitenPiece));
    const size_t o_win = off;
    off += align16(n_win * sizeof(WinPtr));
    const size_t o_int = off;
    off += align16(n_res * sizeof(IntegDesc));
    // the refresh pointer rows: in-step refreshes, then refreshes ahead of need
    RefreshList rf_in, rf_ahead;
    if ((int)(2 * refresh.size()) > b.cap_rf || (int)(2 * ahead.size()) > b.cap_rf)
    {
        afg_fail(ctx, AFG_ERR_STATE, "stream step: more gains refreshes than planned for");
        return -1;
    }
    if (!refresh.empty()) {
        rf_in.off = off;
        off += 2 * align16((size_t)b.cap_rf * sizeof(void *));
        refresh_plan(E, b, hb, rf_in, refresh);
    }
    if (!ahead.empty()) {
        rf_ahead.off = off;
        off += 2 * align16((size_t)b.cap_rf * sizeof(void *));
        refresh_plan(E, b, hb, rf_ahead, ahead);
    }
    memcpy(hb + o_sc, b.h_sc, n_sc * sizeof(ScatterDesc));
    memcpy(hb + o_wp, b.h_wp, n_wp * sizeof(WhitenPiece));
    memcpy(hb + o_win, b.h_win, n_win * sizeof(WinPtr));
    memcpy(hb + o_int, b.h_int, n_res * sizeof(IntegDesc));
    AFG_CUDA(ctx, cudaMemcpyAsync(db, hb, off, cudaMemcpyHostToDevice, st));
    if (n_sc) {
        {
            KScope ks(ctx, st, KK_SCATTER, 0.0, (double)stage_off * 12.0);
            k_scatter<<<n_sc, 256, 0, st>>>(reinterpret_cast<const ScatterDesc *>(db + o_sc), b.d_stage);
        }
        AFG_LAUNCH_CHECK(ctx, "k_scatter");
    }
    if (rf_in.n && refresh_run(E, b, db, rf_in, st)) return -1;
    if (n_wp && launch_whiten_multi(ctx, reinterpret_cast<const WhitenPiece *>(db + o_wp), n_wp, total_white, st))
        return -1;
    // small steps: the network launch also integrates the new windows (its last CTA, after every
    // logit); large ones use one thread per statistic in a launch of their own
    const IntegDesc *integ = reinterpret_cast<const IntegDesc *>(db + o_int);
    const bool fuse_integ = n_res <= kFuseInteg;
    if (n_win && launch_infer_bf16_list(ctx, reinterpret_cast<const WinPtr *>(db + o_win), n_win, integ,
                                        fuse_integ ? n_res : 0, (int)p.n_int, E.d_done, st))
        return -1;
    if (n_res && !fuse_integ) {
        KScope ks(ctx, st, KK_INTEGRATE, (double)n_res * p.n_int, (double)n_res * (p.n_int + 2) * 4.0);
        AFG_CUDA(ctx, launch_pdl(k_stream_integrate, dim3((unsigned)((n_res + 127) / 128)), dim3(128), 0, st, integ,
                                 n_res, (int)p.n_int));
    }
    if (n_res) AFG_CUDA(ctx, cudaMemcpyAsync(b.h_out, b.d_out, n_res * 2 * sizeof(float), cudaMemcpyDeviceToHost, st));
    AFG_CUDA(ctx, cudaEventRecord(b.ev, st));
    // the refreshes ahead of need (planned above), after the step's result event
    if (rf_ahead.n && refresh_run(E, b, db, rf_ahead, st)) return -1;
    b.busy = true;
    E.steps++;
    E.windows += n_win;
    E.samples += (int64_t)stage_off / 2;
    return 1;
}

void engine_main(ServeEngine *E) {
    cudaSetDevice(E->ctx->device);
    int cur = 0;
    while (true) {
        {
            std::unique_lock<std::mutex> lock(E->mu);
            // release closed streams with no work in flight
            for (Slot &s : E->slots)
                if (s.closing && s.inflight == 0 && s.pending.empty()) {
                    cudaFree(s.mem);
                    E->ctx->bytes_held -= s.bytes;
                    s = Slot();
                }
            bool any = false;
            for (const Slot &s : E->slots) any = any || (s.open && !s.pending.empty());
            if (!any && !E->buf[0].busy && !E->buf[1].busy) {
                if (E->stop) break;
                // Idle: poll for the next push for up to kPollS before sleeping, since a thread woken
                // from a condition variable starts tens of microseconds late (one busy core while
                // pushes keep coming; arrivals further apart pay the wake-up).
                const uint64_t seen = E->pushes.load(std::memory_order_acquire);
                lock.unlock();
                const double t0 = now_s();
                bool got = false;
                while (now_s() - t0 < kPollS)
                    if (E->pushes.load(std::memory_order_acquire) != seen) {
                        got = true;
                        break;
                    }
                if (got) continue;
                lock.lock();
                E->cv_work.wait_for(lock, std::chrono::milliseconds(50), [&] {
                    if (E->stop) return true;
                    for (const Slot &s : E->slots)
                        if (s.open && !s.pending.empty()) return true;
                    return false;
                });
                continue;
            }
        }
        if (E->buf[cur].busy) complete(*E, E->buf[cur]);
        const int launched = launch_step(*E, E->buf[cur]);
        if (launched < 0) {
            std::lock_guard<std::mutex> lock(E->mu);
            if (E->err == AFG_OK) E->err = AFG_ERR_CUDA;
            E->stop = true;
            E->cv_done.notify_all();
            break;
        }
        cur ^= 1;
        if (!launched) {
            // nothing new: finish whatever is in flight
            complete(*E, E->buf[cur]);
            complete(*E, E->buf[cur ^ 1]);
        }
    }
    complete(*E, E->buf[0]);
    complete(*E, E->buf[1]);
}

int64_t slot_bytes(const ServeEngine &E) {
    return (int64_t)(2 * 2 * E.R + 2 * 2 * E.Wr + 2 * 2 * NBIN + LR) * 4 + 1024;
}

}  // namespace

void serve_release(afg_ctx *ctx) {
    ServeEngine *E = ctx->serve;
    if (!E) return;
    {
        std::lock_guard<std::mutex> lock(E->mu);
        E->stop = true;
        for (Slot &s : E->slots) s.pending.clear();
    }
    E->cv_work.notify_all();
    if (E->th.joinable()) E->th.join();
    for (Slot &s : E->slots)
        if (s.mem) cudaFree(s.mem);
    free_step(E->buf[0]);
    free_step(E->buf[1]);
    if (E->st) cudaStreamDestroy(E->st);
    if (E->d_done) cudaFree(E->d_done);
    if (E->d_rf_psd) cudaFree(E->d_rf_psd);
    if (E->d_rf_gains) cudaFree(E->d_rf_gains);
    delete E;
    ctx->serve = nullptr;
}

extern "C" int afg_stream_start(afg_ctx *ctx, const afg_stream_params *p) {
    if (!ctx || !p) return AFG_ERR_ARG;
    ctx->err.clear();
    if (ctx->serve) return afg_fail(ctx, AFG_ERR_STATE, "stream_start: the engine is already running");
    const int hop = ctx->cfg.hop, W = ctx->cfg.win_len;
    if (p->epoch_len <= 0 || p->epoch_len % hop || p->psd_len < NFFT || (p->psd_len - NFFT) % hop ||
        p->stride < 1 || p->n_int < 1 || p->n_int > LR || p->max_streams < 1 || p->max_chunk < 1)
        return afg_fail(ctx, AFG_ERR_ARG, "stream_start: bad parameters");
    if (ctx->cfg.precision != AFG_BF16 || !ctx->plan.tc_params)
        return afg_fail(ctx, AFG_ERR_UNSUPPORTED, "stream_start: streams run the BF16 tensor-core network");
    ServeEngine *E = new ServeEngine();
    E->ctx = ctx;
    E->p = *p;
    E->Wr = 8192;
    // new samples per stream per step: every window that a step evaluates must still be in the whitened ring
    E->per_stream_new = E->Wr - W - p->stride;
    if (p->max_chunk > E->per_stream_new) {
        const long long lim = (long long)E->per_stream_new;
        delete E;
        return afg_fail(ctx, AFG_ERR_ARG, "stream_start: max_chunk must be <= %lld samples", lim);
    }
    E->R = p->psd_len + p->epoch_len + E->per_stream_new + ctx->cfg.fir_len + WB;
    int rc = alloc_step(ctx, E->buf[0], p->max_streams, E->per_stream_new, p->stride);
    if (!rc) rc = alloc_step(ctx, E->buf[1], p->max_streams, E->per_stream_new, p->stride);
    if (!rc && cudaStreamCreateWithFlags(&E->st, cudaStreamNonBlocking) != cudaSuccess) rc = AFG_ERR_CUDA;
    if (!rc && (cudaMalloc(&E->d_done, 16) != cudaSuccess || cudaMemset(E->d_done, 0, 16) != cudaSuccess))
        rc = AFG_ERR_CUDA;
    // the scratch of a batch of gains refreshes (up to 16 streams: the Welch periodograms of their
    // detectors, the FP64 transforms of their filters, their PSDs and gains), reserved and counted
    // against the HBM budget here, before any stream is admitted: steps never allocate, and the
    // engine thread never changes bytes_held outside E->mu
    void *tmp = nullptr;
    const int64_t K = (p->psd_len - NFFT) / hop + 1;
    E->rb_rows = 2 * std::min(p->max_streams, 16);
    if (!rc) rc = afg_ws_reserve(ctx, WS_PERIODOGRAM, (size_t)E->rb_rows * K * NBIN * sizeof(double), &tmp);
    if (!rc) rc = afg_ws_reserve(ctx, WS_FB_SCRATCH, filter_build_scratch_bytes(ctx, E->rb_rows), &tmp);
    if (!rc && (cudaMalloc(&E->d_rf_psd, (size_t)E->rb_rows * NBIN * sizeof(double)) != cudaSuccess ||
                cudaMalloc(&E->d_rf_gains, (size_t)E->rb_rows * NBIN * sizeof(float)) != cudaSuccess)) {
        cudaGetLastError();
        rc = afg_fail(ctx, AFG_ERR_OOM, "stream_start: refresh buffers");
    }
    if (!rc) ctx->bytes_held += (int64_t)E->rb_rows * NBIN * (sizeof(double) + sizeof(float));
    if (rc) {
        ctx->serve = E;
        serve_release(ctx);
        return rc;
    }
    E->slots.resize(p->max_streams);
    ctx->serve = E;
    E->th = std::thread(engine_main, E);
    return AFG_OK;
}

extern "C" int afg_stream_open(afg_ctx *ctx, int64_t *stream_id) {
    if (!ctx || !stream_id) return AFG_ERR_ARG;
    ctx->err.clear();
    ServeEngine *E = ctx->serve;
    if (!E) return afg_fail(ctx, AFG_ERR_STATE, "stream_open: call afg_stream_start first");
    std::lock_guard<std::mutex> lock(E->mu);
    int s = -1;
    for (int i = 0; i < (int)E->slots.size(); ++i)
        if (!E->slots[i].open && !E->slots[i].closing && !E->slots[i].mem) {
            s = i;
            break;
        }
    if (s < 0) return afg_fail(ctx, AFG_ERR_BUDGET, "stream_open: all %d stream slots are in use", (int)E->slots.size());
    const int64_t bytes = slot_bytes(*E);
    if (ctx->cfg.hbm_budget > 0 && ctx->bytes_held + bytes > ctx->cfg.hbm_budget)
        return afg_fail(ctx, AFG_ERR_BUDGET, "stream_open: %lld more bytes would exceed the HBM budget (%lld held)",
                        (long long)bytes, (long long)ctx->bytes_held);
    cudaSetDevice(ctx->device);
    void *m = nullptr;
    if (cudaMalloc(&m, bytes) != cudaSuccess) {
        cudaGetLastError();
        return afg_fail(ctx, AFG_ERR_OOM, "stream_open: cudaMalloc(%lld) failed", (long long)bytes);
    }
    if (cudaMemset(m, 0, bytes) != cudaSuccess) {
        cudaFree(m);
        return afg_fail(ctx, AFG_ERR_CUDA, "stream_open: cudaMemset failed");
    }
    Slot &sl = E->slots[s];
    sl = Slot();
    sl.mem = m;
    sl.bytes = bytes;
    char *c = static_cast<char *>(m);
    sl.raw = reinterpret_cast<float *>(c);
    c += 2 * 2 * E->R * 4;
    sl.white = reinterpret_cast<float *>(c);
    c += 2 * 2 * E->Wr * 4;
    sl.gains = reinterpret_cast<float *>(c);
    c += 2 * 2 * NBIN * 4;
    sl.logits = reinterpret_cast<float *>(c);
    sl.open = true;
    ctx->bytes_held += bytes;
    *stream_id = s;
    return AFG_OK;
}

extern "C" int afg_stream_push(afg_ctx *ctx, int64_t id, const float *chunk_host, int64_t n, int64_t *ticket) {
    if (!ctx) return AFG_ERR_ARG;
    ServeEngine *E = ctx->serve;
    if (!E) return afg_fail(ctx, AFG_ERR_STATE, "stream_push: no engine");
    if (!chunk_host || n < 1 || n > E->p.max_chunk) return afg_fail(ctx, AFG_ERR_ARG, "stream_push: bad chunk");
    for (int64_t i = 0; i < 2 * n; ++i)
        if (!(chunk_host[i] == chunk_host[i]) || chunk_host[i] - chunk_host[i] != 0.0f)
            return afg_fail(ctx, AFG_ERR_NAN, "stream_push: non-finite sample at %lld", (long long)i);
    Chunk c;
    c.data.assign(chunk_host, chunk_host + 2 * n);
    c.n = n;
    c.t_push = now_s();
    {
        std::lock_guard<std::mutex> lock(E->mu);
        if (E->err) return afg_fail(ctx, E->err, "stream_push: the engine stopped after an error");
        if (id < 0 || id >= (int64_t)E->slots.size() || !E->slots[id].open)
            return afg_fail(ctx, AFG_ERR_STATE, "stream_push: stream %lld is not open", (long long)id);
        Slot &sl = E->slots[id];
        if (ticket) *ticket = sl.pushed;
        sl.pushed++;
        sl.pending.push_back(std::move(c));
    }
    E->pushes.fetch_add(1, std::memory_order_release);
    E->cv_work.notify_one();
    return AFG_OK;
}

extern "C" int afg_stream_push_many(afg_ctx *ctx, int64_t n_push, const int64_t *ids, const float *chunks_host,
                                    int64_t n, int64_t *tickets) {
    if (!ctx) return AFG_ERR_ARG;
    ServeEngine *E = ctx->serve;
    if (!E) return afg_fail(ctx, AFG_ERR_STATE, "stream_push_many: no engine");
    if (n_push < 0 || (n_push > 0 && (!ids || !chunks_host)) || n < 1 || n > E->p.max_chunk)
        return afg_fail(ctx, AFG_ERR_ARG, "stream_push_many: bad arguments");
    if (n_push == 0) return AFG_OK;
    // every check before anything is queued: a refused call pushes nothing
    for (int64_t i = 0; i < 2 * n * n_push; ++i)
        if (!(chunks_host[i] == chunks_host[i]) || chunks_host[i] - chunks_host[i] != 0.0f)
            return afg_fail(ctx, AFG_ERR_NAN, "stream_push_many: non-finite sample in push %lld",
                            (long long)(i / (2 * n)));
    std::vector<Chunk> cs((size_t)n_push);
    const double t = now_s();
    for (int64_t k = 0; k < n_push; ++k) {
        cs[k].data.assign(chunks_host + 2 * n * k, chunks_host + 2 * n * (k + 1));
        cs[k].n = n;
        cs[k].t_push = t;
    }
    {
        std::lock_guard<std::mutex> lock(E->mu);
        if (E->err) return afg_fail(ctx, E->err, "stream_push_many: the engine stopped after an error");
        for (int64_t k = 0; k < n_push; ++k)
            if (ids[k] < 0 || ids[k] >= (int64_t)E->slots.size() || !E->slots[ids[k]].open)
                return afg_fail(ctx, AFG_ERR_STATE, "stream_push_many: stream %lld is not open", (long long)ids[k]);
        for (int64_t k = 0; k < n_push; ++k) {
            Slot &sl = E->slots[ids[k]];
            if (tickets) tickets[k] = sl.pushed;
            sl.pushed++;
            sl.pending.push_back(std::move(cs[k]));
        }
    }
    E->pushes.fetch_add((uint64_t)n_push, std::memory_order_release);
    E->cv_work.notify_one();
    return AFG_OK;
}

extern "C" int afg_stream_poll(afg_ctx *ctx, int64_t id, afg_stream_result *out, int64_t cap, int64_t *n_out,
                               double wait_s) {
    if (!ctx || !n_out || (cap > 0 && !out)) return AFG_ERR_ARG;
    ServeEngine *E = ctx->serve;
    if (!E) return afg_fail(ctx, AFG_ERR_STATE, "stream_poll: no engine");
    std::unique_lock<std::mutex> lock(E->mu);
    if (id < 0 || id >= (int64_t)E->slots.size() || !(E->slots[id].open || E->slots[id].closing))
        return afg_fail(ctx, AFG_ERR_STATE, "stream_poll: stream %lld is not open", (long long)id);
    if (wait_s > 0 && E->slots[id].results.empty())
        E->cv_done.wait_for(lock, std::chrono::duration<double>(wait_s),
                            [&] { return !E->slots[id].results.empty() || E->err; });
    Slot &sl = E->slots[id];
    const int64_t n = std::min<int64_t>(cap, (int64_t)sl.results.size());
    for (int64_t i = 0; i < n; ++i) out[i] = sl.results[i];
    sl.results.erase(sl.results.begin(), sl.results.begin() + n);
    *n_out = n;
    return E->err ? afg_fail(ctx, E->err, "stream_poll: the engine stopped after an error") : AFG_OK;
}

extern "C" int afg_stream_flush(afg_ctx *ctx, double wait_s) {
    if (!ctx) return AFG_ERR_ARG;
    ServeEngine *E = ctx->serve;
    if (!E) return afg_fail(ctx, AFG_ERR_STATE, "stream_flush: no engine");
    std::unique_lock<std::mutex> lock(E->mu);
    E->cv_work.notify_all();
    const bool ok = E->cv_done.wait_for(lock, std::chrono::duration<double>(wait_s), [&] {
        for (const Slot &s : E->slots)
            if (!s.pending.empty() || s.inflight) return false;
        return true;
    });
    if (E->err) return afg_fail(ctx, E->err, "stream_flush: the engine stopped after an error");
    return ok ? AFG_OK : afg_fail(ctx, AFG_ERR_TIMEOUT, "stream_flush: work still pending after %.3f s", wait_s);
}

extern "C" int afg_stream_close(afg_ctx *ctx, int64_t id) {
    if (!ctx) return AFG_ERR_ARG;
    ServeEngine *E = ctx->serve;
    if (!E) return afg_fail(ctx, AFG_ERR_STATE, "stream_close: no engine");
    {
        std::lock_guard<std::mutex> lock(E->mu);
        if (id < 0 || id >= (int64_t)E->slots.size() || !E->slots[id].open)
            return afg_fail(ctx, AFG_ERR_STATE, "stream_close: stream %lld is not open", (long long)id);
        E->slots[id].open = false;
        E->slots[id].closing = true;
        E->slots[id].pending.clear();
        E->slots[id].results.clear();
    }
    E->cv_work.notify_all();
    return AFG_OK;
}

extern "C" int afg_stream_stats(afg_ctx *ctx, int64_t *steps, int64_t *windows, int64_t *samples) {
    if (!ctx || !ctx->serve) return AFG_ERR_ARG;
    std::lock_guard<std::mutex> lock(ctx->serve->mu);
    if (steps) *steps = ctx->serve->steps;
    if (windows) *windows = ctx->serve->windows;
    if (samples) *samples = ctx->serve->samples;
    return AFG_OK;
}
