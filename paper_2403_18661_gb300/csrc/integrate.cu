// Integration and clustering of the per-window outputs (Sec. II: the
// predictions are integrated with a 1 s top-hat filter; the maximum
// integrated value over an 8 s window is the detection statistic of a
// candidate).
//
//   k_integrate   stat[j] = (1/n_int) sum_{i<n_int} z[j+i], summed in index order
//   triggers      the cluster maxima (earliest index wins ties): short series by a
//                 direct scan in one CTA; long ones from windowed maxima built by
//                 doubling, O(n log h), compacted in increasing index order across
//                 blocks (counts, one scan, writes).
#include <math.h>

#include <algorithm>

#include "afg_internal.cuh"

namespace {

__global__ void k_integrate(const float *__restrict__ z, int64_t n_out, int n_int, float *__restrict__ stat) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_out) return;
    float s = 0.f;
    for (int i = 0; i < n_int; ++i) s += z[j + i];
    stat[j] = s / (float)n_int;
}

// Short series: one CTA scans each index's neighbourhood directly (early exit on the first
// larger neighbour) and compacts in index order over 1024-index chunks.
constexpr int TT = 1024;

__global__ void __launch_bounds__(TT) k_triggers_small(const float *__restrict__ I, int64_t n, int half,
                                                       int64_t *__restrict__ idx, int64_t cap,
                                                       int64_t *__restrict__ n_trig) {
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
            const int64_t lo = j - half < 0 ? 0 : j - half;
            const int64_t hi = j + half >= n ? n - 1 : j + half;
            for (int64_t i = lo; i < j && flag; ++i) flag = v > I[i];
            for (int64_t i = j + 1; i <= hi && flag; ++i) flag = v >= I[i];
        }
        const unsigned m = __ballot_sync(0xffffffffu, flag);
        const int in_warp = __popc(m & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[wid] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < TT / 32; ++w) {
            const int t = warp_tot[w];
            if (w < wid) before += t;
            total += t;
        }
        const int64_t base = base_s;
        if (flag) {
            const int64_t pos = base + before + in_warp;
            if (pos < cap) idx[pos] = j;
        }
        __syncthreads();
        if (tid == 0) base_s = base + total;
        __syncthreads();
    }
    if (tid == 0) *n_trig = base_s;
}

// ---- clustering: j is a trigger iff I[j] > max I[j-h .. j-1] and I[j] >= max I[j+1 .. j+h]
// (earliest index wins ties).  The statistic is padded with -inf on both sides (h each), so
// every window is full; M_k[i] = max P[i .. i + 2^k) is built by k doubling passes
// (2^k <= h < 2^(k+1)), and each half-window is the union of two overlapping 2^k windows.
constexpr int TB = 1024;  // indices per compaction block

__global__ void k_trig_pad(const float *__restrict__ I, int64_t n, int h, float *__restrict__ P) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n + 2 * (int64_t)h;
         i += (int64_t)gridDim.x * blockDim.x)
        P[i] = (i >= h && i < n + h) ? I[i - h] : -INFINITY;
}

__global__ void k_trig_double(const float *__restrict__ A, int64_t len, int64_t step, float *__restrict__ B) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        B[i] = fmaxf(A[i], A[i + step]);
}

// flags and per-block counts (M: level-k maxima of the padded statistic, or the statistic when h = 0)
__global__ void __launch_bounds__(TB) k_trig_flag(const float *__restrict__ I, const float *__restrict__ M,
                                                  int64_t n, int h, int64_t w, uint8_t *__restrict__ flag,
                                                  int *__restrict__ counts) {
    __shared__ int wc[TB / 32];
    const int64_t j = (int64_t)blockIdx.x * TB + threadIdx.x;
    int f = 0;
    if (j < n) {
        if (h == 0) {
            f = 1;
        } else {
            const int64_t p = j + h;  // padded index of j
            const float v = I[j];
            const float left = fmaxf(M[p - h], M[p - w]);
            const float right = fmaxf(M[p + 1], M[p + h - w + 1]);
            f = (v > left) && (v >= right);
        }
        flag[j] = (uint8_t)f;
    }
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < TB / 32; ++i) t += wc[i];
        counts[blockIdx.x] = t;
    }
}

// exclusive scan of the block counts (one block, fixed order) and the total
__global__ void __launch_bounds__(1024) k_trig_scan(int *__restrict__ counts, int nb, int64_t *__restrict__ n_trig) {
    __shared__ int64_t s[1024];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < nb; c0 += 1024) {
        const int i = c0 + threadIdx.x;
        const int64_t v = i < nb ? counts[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int64_t t = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) counts[i] = (int)(carry + s[threadIdx.x] - v);
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_trig = carry;
}

__global__ void __launch_bounds__(TB) k_trig_write(const uint8_t *__restrict__ flag, int64_t n,
                                                   const int *__restrict__ base, int64_t *__restrict__ idx,
                                                   int64_t cap) {
    __shared__ int wc[TB / 32];
    const int64_t j = (int64_t)blockIdx.x * TB + threadIdx.x;
    const int f = j < n ? flag[j] : 0;
    const unsigned m = __ballot_sync(0xffffffffu, f);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) wc[wid] = __popc(m);
    __syncthreads();
    int before = 0;
    for (int i = 0; i < wid; ++i) before += wc[i];
    if (f) {
        const int64_t pos = (int64_t)base[blockIdx.x] + before + __popc(m & ((1u << lane) - 1u));
        if (pos < cap) idx[pos] = j;
    }
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
    if (n_out <= 0) {
        AFG_CUDA(ctx, cudaMemsetAsync(n_trig, 0, sizeof(int64_t), st));
        return AFG_OK;
    }
    const int h = cluster_half;
    if (n_out <= 16384 && h <= 256) {  // short series: the direct scan needs one launch
        KScope ks(ctx, st, KK_TRIGGERS, 0.0, (double)n_out * 4.0);
        k_triggers_small<<<1, TT, 0, st>>>(stat, n_out, h, trig_idx, trig_cap, n_trig);
        AFG_LAUNCH_CHECK(ctx, "k_triggers_small");
        return AFG_OK;
    }
    int k = 0;
    while (h > 0 && ((int64_t)2 << k) <= h) ++k;  // 2^k <= h < 2^(k+1)
    const int64_t w = h > 0 ? ((int64_t)1 << k) : 0;
    const int64_t N = n_out + 2 * (int64_t)h;
    const int nb = (int)((n_out + TB - 1) / TB);
    void *pa = nullptr, *pb = nullptr, *pf = nullptr, *pc = nullptr;
    int rc = afg_ws_reserve(ctx, WS_TRIG_A, (size_t)N * sizeof(float), &pa);
    if (!rc && h > 0) rc = afg_ws_reserve(ctx, WS_TRIG_B, (size_t)N * sizeof(float), &pb);
    if (!rc) rc = afg_ws_reserve(ctx, WS_TRIG_FLAG, (size_t)n_out, &pf);
    if (!rc) rc = afg_ws_reserve(ctx, WS_TRIG_COUNT, (size_t)nb * sizeof(int), &pc);
    if (rc) return rc;
    float *A = static_cast<float *>(pa), *B = static_cast<float *>(pb);
    const unsigned g = (unsigned)std::min<int64_t>((N + 255) / 256, 152 * 32);
    {
        KScope ks(ctx, st, KK_TRIGGERS, 0.0, (double)n_out * 4.0 * (3 + 2 * k));
        const float *M = stat;
        if (h > 0) {
            k_trig_pad<<<g, 256, 0, st>>>(stat, n_out, h, A);
            int64_t len = N;
            for (int l = 1; l <= k; ++l) {  // M_l[i] = max(M_{l-1}[i], M_{l-1}[i + 2^(l-1)])
                const int64_t step = (int64_t)1 << (l - 1);
                len -= step;
                k_trig_double<<<g, 256, 0, st>>>(A, len, step, B);
                std::swap(A, B);
            }
            M = A;
        }
        uint8_t *flag = static_cast<uint8_t *>(pf);
        int *counts = static_cast<int *>(pc);
        k_trig_flag<<<nb, TB, 0, st>>>(stat, M, n_out, h, w, flag, counts);
        k_trig_scan<<<1, 1024, 0, st>>>(counts, nb, n_trig);
        k_trig_write<<<nb, TB, 0, st>>>(flag, n_out, counts, trig_idx, trig_cap);
    }
    AFG_LAUNCH_CHECK(ctx, "k_triggers");
    return AFG_OK;
}
