// False-alarm rates from a timeslide background (Sec. IX: the FAR of an event is
// the number of background events whose detection statistic is greater than the
// event's, divided by the background livetime).
//
// The background statistics are sorted in decreasing order on the device by an
// LSD radix sort of order-preserving 32-bit keys (4 passes of 8 bits, each pass
// stable: per-tile digit histograms, one exclusive scan over (digit, tile), and a
// scatter that ranks equal digits in input order).  Launches are sized by the
// capacity; only the tiles that hold keys do work.  Each foreground statistic x
// then gets count = #{background > x} by binary search, and FAR = count / livetime.
// The background count may live on the device (as afg_batch_run writes it), so
// every kernel reads n = min(*n_dev, cap) itself and nothing synchronises.
#include <stdint.h>

#include <algorithm>

#include "afg_internal.cuh"

namespace {

constexpr int RS_T = 256;              // threads per tile
constexpr int RS_ROUNDS = 8;           // keys per thread per tile
constexpr int RS_TILE = RS_T * RS_ROUNDS;
constexpr int RS_WARPS = RS_T / 32;

__device__ __forceinline__ int64_t dev_count(const int64_t *n_dev, int64_t cap) {
    const int64_t n = *n_dev;
    return n < 0 ? 0 : (n < cap ? n : cap);
}

// Ascending order of keys = decreasing order of statistics.
__device__ __forceinline__ uint32_t key_of(float v) {
    uint32_t b = __float_as_uint(v);
    b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);  // ascending with v
    return ~b;                                        // descending with v
}

__device__ __forceinline__ float value_of(uint32_t k) {
    uint32_t b = ~k;
    b = (b & 0x80000000u) ? (b & 0x7fffffffu) : ~b;
    return __uint_as_float(b);
}

__global__ void k_far_keys(const float *__restrict__ stat, const int64_t *__restrict__ idx, const int64_t *n_dev,
                           int64_t cap, uint32_t *__restrict__ keys) {
    const int64_t n = dev_count(n_dev, cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = key_of(stat[idx ? idx[i] : i]);
}

// tiles that hold keys
__device__ __forceinline__ int occupied_tiles(int64_t n) { return (int)((n + RS_TILE - 1) / RS_TILE); }

// hist[d * n_eff + tile] = keys of the tile whose digit (at `shift`) is d, over the
// n_eff = ceil(n / RS_TILE) tiles that hold keys (blocks past them return at once)
__global__ void __launch_bounds__(RS_T) k_rs_hist(const uint32_t *__restrict__ keys, const int64_t *n_dev,
                                                  int64_t cap, int shift, uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[256];
    const int64_t n = dev_count(n_dev, cap);
    const int n_eff = occupied_tiles(n);
    if ((int)blockIdx.x >= n_eff) return;
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const int64_t i = base + r * RS_T + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * n_eff + blockIdx.x] = h[threadIdx.x];
}

// In-place exclusive scan of the 256 n_eff histogram entries (digit-major, so the scan
// order is (digit, tile)), one block walking chunks of 1024 with a running carry.  Each
// chunk: a warp scan, the 32 warp totals through shared memory (double-buffered, so one
// barrier per chunk), and every warp scans those totals itself.  Loads run SCAN_AHEAD
// chunks ahead of the chunk being scanned.
constexpr int SCAN_AHEAD = 4;
__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t *__restrict__ a, const int64_t *n_dev, int64_t cap) {
    __shared__ uint32_t wsum[2][32];
    const int64_t n = dev_count(n_dev, cap);
    const int64_t m = (int64_t)256 * occupied_tiles(n);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    uint32_t v[SCAN_AHEAD];
#pragma unroll
    for (int k = 0; k < SCAN_AHEAD; ++k) {
        const int64_t i = (int64_t)k * 1024 + t;
        v[k] = i < m ? a[i] : 0u;
    }
    uint32_t carry = 0;
    int buf = 0;
    for (int64_t c0 = 0; c0 < m; c0 += 1024 * SCAN_AHEAD) {
        uint32_t nxt[SCAN_AHEAD];
#pragma unroll
        for (int k = 0; k < SCAN_AHEAD; ++k) {
            const int64_t i = c0 + (int64_t)(SCAN_AHEAD + k) * 1024 + t;
            nxt[k] = i < m ? a[i] : 0u;
        }
#pragma unroll
        for (int k = 0; k < SCAN_AHEAD; ++k) {
            uint32_t x = v[k];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) wsum[buf][warp] = x;
            __syncthreads();
            uint32_t w = wsum[buf][lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            const uint32_t before = __shfl_sync(0xffffffffu, w, (warp + 31) & 31);
            const uint32_t total = __shfl_sync(0xffffffffu, w, 31);
            const int64_t i = c0 + (int64_t)k * 1024 + t;
            if (i < m) a[i] = carry + (warp ? before : 0u) + x - v[k];
            carry += total;
            buf ^= 1;
        }
#pragma unroll
        for (int k = 0; k < SCAN_AHEAD; ++k) v[k] = nxt[k];
    }
}

// Stable scatter of one tile: key index base + r * RS_T + t is processed in round r by
// thread t, so (round, thread) order is input order; inside a round, equal digits are
// ranked by warp (lower warps first) and by lane (match_any peers with lower lanes).
__global__ void __launch_bounds__(RS_T) k_rs_scatter(const uint32_t *__restrict__ kin, uint32_t *__restrict__ kout,
                                                     const int64_t *n_dev, int64_t cap, int shift,
                                                     const uint32_t *__restrict__ hist) {
    __shared__ uint32_t running[256];          // keys of each digit placed by earlier rounds (+ tile base)
    __shared__ uint32_t wcnt[RS_WARPS][257];   // per-warp digit counts of the current round
    const int64_t n = dev_count(n_dev, cap);
    const int n_eff = occupied_tiles(n);
    if ((int)blockIdx.x >= n_eff) return;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    running[t] = hist[(size_t)t * n_eff + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const uint32_t lt = (1u << lane) - 1u;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        for (int i = t; i < RS_WARPS * 257; i += RS_T) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        const int64_t i = base + r * RS_T + t;
        const bool valid = i < n;
        const uint32_t key = valid ? kin[i] : 0u;
        const uint32_t d = valid ? ((key >> shift) & 255u) : 256u;  // 256: no key
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lt);
        if (rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        uint32_t before = 0;  // same-digit keys of lower warps in this round
        for (int w = 0; w < warp; ++w) before += wcnt[w][d];
        if (valid) kout[running[d] + before + rank] = key;
        __syncthreads();
        uint32_t tot = 0;  // thread t advances digit t
        for (int w = 0; w < RS_WARPS; ++w) tot += wcnt[w][t];
        running[t] += tot;
        __syncthreads();
    }
}

__global__ void k_far_values(const uint32_t *__restrict__ keys, const int64_t *n_dev, int64_t cap,
                             float *__restrict__ sorted) {
    const int64_t n = dev_count(n_dev, cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        sorted[i] = value_of(keys[i]);
}

// count = #{sorted > x}: the first index whose value is <= x in the decreasing array
__global__ void k_far_count(const float *__restrict__ sorted, const int64_t *n_dev, int64_t cap,
                            const float *__restrict__ fg, int64_t n_fg, double livetime, int64_t *__restrict__ n_above,
                            double *__restrict__ far) {
    const int64_t n = dev_count(n_dev, cap);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_fg; j += (int64_t)gridDim.x * blockDim.x) {
        const float x = fg[j];
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (sorted[mid] > x) lo = mid + 1;
            else hi = mid;
        }
        if (n_above) n_above[j] = lo;
        if (far) far[j] = (double)lo / livetime;
    }
}

}  // namespace

int launch_far(afg_ctx *ctx, const float *bg_stat, const int64_t *bg_idx, const int64_t *n_bg_dev, int64_t bg_cap,
               double livetime_s, const float *fg, int64_t n_fg, int64_t *n_above, double *far, float *bg_sorted,
               cudaStream_t st) {
    const int n_tiles = (int)std::max<int64_t>(1, (bg_cap + RS_TILE - 1) / RS_TILE);
    const int64_t m = (int64_t)256 * n_tiles;
    void *wk = nullptr, *wh = nullptr, *ws = nullptr;
    int rc = afg_ws_reserve(ctx, WS_FAR_KEYS, (size_t)2 * std::max<int64_t>(bg_cap, 1) * sizeof(uint32_t), &wk);
    if (!rc) rc = afg_ws_reserve(ctx, WS_FAR_HIST, (size_t)m * sizeof(uint32_t), &wh);
    if (!rc && !bg_sorted) {
        rc = afg_ws_reserve(ctx, WS_FAR_SORTED, (size_t)std::max<int64_t>(bg_cap, 1) * sizeof(float), &ws);
        bg_sorted = static_cast<float *>(ws);
    }
    if (rc) return rc;
    uint32_t *ka = static_cast<uint32_t *>(wk), *kb = ka + std::max<int64_t>(bg_cap, 1);
    uint32_t *hist = static_cast<uint32_t *>(wh);
    const unsigned g1 = (unsigned)std::min<int64_t>((bg_cap + 255) / 256 + 1, 152 * 16);
    {
        KScope ks(ctx, st, KK_FAR, 0.0, (double)bg_cap * (4.0 + 8.0 + 4.0 * 4 * 4 + 4.0) + n_fg * 20.0);
        k_far_keys<<<g1, 256, 0, st>>>(bg_stat, bg_idx, n_bg_dev, bg_cap, ka);
        for (int pass = 0; pass < 4; ++pass) {
            k_rs_hist<<<n_tiles, RS_T, 0, st>>>(ka, n_bg_dev, bg_cap, 8 * pass, hist);
            k_rs_scan<<<1, 1024, 0, st>>>(hist, n_bg_dev, bg_cap);
            k_rs_scatter<<<n_tiles, RS_T, 0, st>>>(ka, kb, n_bg_dev, bg_cap, 8 * pass, hist);
            std::swap(ka, kb);
        }
        k_far_values<<<g1, 256, 0, st>>>(ka, n_bg_dev, bg_cap, bg_sorted);
        if (n_fg > 0)
            k_far_count<<<(unsigned)std::min<int64_t>((n_fg + 255) / 256, 152 * 16), 256, 0, st>>>(
                bg_sorted, n_bg_dev, bg_cap, fg, n_fg, livetime_s, n_above, far);
    }
    AFG_LAUNCH_CHECK(ctx, "far (radix sort + rank count)");
    return AFG_OK;
}
