// Integration and clustering of the per-window outputs (Sec. II: the
// predictions are integrated with a 1 s top-hat filter; the maximum
// integrated value over an 8 s window is the detection statistic of a
// candidate).
//
//   k_integrate   stat[j] = (1/n_int) sum_{i<n_int} z[j+i], summed in index order
//   k_triggers    one CTA: flags the cluster maxima (earliest index wins ties)
//                 and compacts them in increasing index order with a
//                 block-wide prefix sum over 1024-index chunks.
#include "afg_internal.cuh"

namespace {

__global__ void k_integrate(const float *__restrict__ z, int64_t n_out, int n_int, float *__restrict__ stat) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_out) return;
    float s = 0.f;
    for (int i = 0; i < n_int; ++i) s += z[j + i];
    stat[j] = s / (float)n_int;
}

constexpr int TT = 1024;

__global__ void __launch_bounds__(TT) k_triggers(const float *__restrict__ I, int64_t n, int half,
                                                 int64_t *__restrict__ idx, int64_t cap, int64_t *__restrict__ n_trig) {
    __shared__ int warp_tot[TT / 32];
    __shared__ int64_t base_s;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) base_s = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < n; c0 += TT) {
        const int64_t j = c0 + tid;
        int flag = 0;
        if (j < n) {
            const float v = I[j];
            flag = 1;
            int64_t lo = j - half < 0 ? 0 : j - half;
            int64_t hi = j + half >= n ? n - 1 : j + half;
            for (int64_t i = lo; i < j && flag; ++i) flag = v > I[i];
            for (int64_t i = j + 1; i <= hi && flag; ++i) flag = v >= I[i];
        }
        unsigned m = __ballot_sync(0xffffffffu, flag);
        int in_warp = __popc(m & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[wid] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < TT / 32; ++w) {
            int t = warp_tot[w];
            if (w < wid) before += t;
            total += t;
        }
        const int64_t base = base_s;
        if (flag) {
            int64_t pos = base + before + in_warp;
            if (pos < cap) idx[pos] = j;
        }
        __syncthreads();
        if (tid == 0) base_s = base + total;
        __syncthreads();
    }
    if (tid == 0) *n_trig = base_s;
}

}  // namespace

int launch_integrate(afg_ctx *ctx, const float *logits, int64_t n_win, int n_int, int cluster_half, float *stat,
                     int64_t *trig_idx, int64_t trig_cap, int64_t *n_trig, cudaStream_t st) {
    const int64_t n_out = n_win - n_int + 1;
    {
        KScope ks(ctx, st, KK_INTEGRATE, (double)n_out * n_int, (double)(n_win + n_out) * 4.0);
        k_integrate<<<(unsigned)((n_out + 255) / 256), 256, 0, st>>>(logits, n_out, n_int, stat);
    }
    AFG_LAUNCH_CHECK(ctx, "k_integrate");
    {
        KScope ks(ctx, st, KK_TRIGGERS, 0.0, (double)n_out * 4.0);
        k_triggers<<<1, TT, 0, st>>>(stat, n_out, cluster_half, trig_idx, trig_cap, n_trig);
    }
    AFG_LAUNCH_CHECK(ctx, "k_triggers");
    return AFG_OK;
}
