// 1D ResNet on tcgen05 tensor cores: BF16 operands in shared memory, FP32
// accumulators in TMEM (Sec. II: ResNet with 1D convolutions and GroupNorm;
// Sec. IX: kernel length 3).
//
// k_tiny_fused: the whole 16-channel network for one window per CTA pass,
// persistent over windows, with every activation resident in shared memory:
//   stem (SIMT FP32, reads the window from the whitened stream; GN statistics
//   in a first pass, GN + ReLU + BF16 store in a second)
//   -> per conv: one thread issues, for each 128-position M-subtile j and tap
//      r, tcgen05.mma(M=128, N=16, K=16) with A = activation rows
//      128 j + r .. + 127 (the tap shift is a 16-byte shift of the descriptor
//      start) and B = the tap's 16x16 weights; the accumulators of the whole
//      window (W/128 x 16 columns) live in TMEM.  The epilogue (16 warps)
//      reads TMEM twice: GroupNorm statistics, then normalise (+ residual)
//      + ReLU -> BF16 into the other activation buffer.
//   -> head: the last epilogue keeps per-channel sums (global mean pool),
//      then the linear layer.
// Activation layout in shared memory (K-major, no swizzle): channel chunk c
// (8 channels, 16 bytes) of padded row p at c * (W + 2) * 16 + p * 16, i.e.
// core matrices of 8 rows x 16 B with SBO = 128 B and LBO = (W + 2) * 16 B;
// rows 0 and W + 1 are the zero padding of the k3 convolutions.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "afg_internal.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int TF_THREADS = 512;
constexpr int TF_WARPS = TF_THREADS / 32;
constexpr int TF_C = 16;                   // channels of the fused network
constexpr int TF_WIMG = 3 * 2 * TF_C * 16;  // bytes of one conv's weight image (3 taps x 512 B)
constexpr int TF_GROUPS = 3;                // MMA commit groups per conv (8 M subtiles each at W = 3072)
constexpr int TF_CLUSTER = 8;               // list mode, few windows: CTAs sharing one window
// cluster exchange area after the shared-memory layout (floats): [0, 32) stem moments, [32, 48)
// GroupNorm partials, [48, 64) head sums, then per layer parity p the raw accumulators of the
// CTA's first and last positions at 64 + 48 p + 16 side and their residual rows (BF16 pairs) at
// 64 + 48 p + 32 + 8 side
constexpr int TF_XCH = (64 + 2 * 48) * 4;
constexpr int TF_SMEM_MAX = 227 * 1024;     // opt-in shared memory per CTA

// segment descriptors a batch launch keeps in shared memory (after the layout of total bytes)
__host__ inline int tiny_seg_cache_cap(size_t total) {
    const int64_t room = ((int64_t)TF_SMEM_MAX - (int64_t)total) / (int64_t)sizeof(SegDesc);
    return (int)std::max<int64_t>(0, std::min<int64_t>(room, 256));
}

struct TinyArgs {
    const float *y;
    int64_t n_y, y_stride, first, stride, shift, n_win;
    const SegDesc *segs;            // batch mode (n_seg > 0): per-segment window descriptors
    int n_seg;
    int seg_cache;                  // batch mode: n_seg if the descriptors are copied to shared memory, else 0
    const WinPtr *wins;             // list mode (non-null): window i reads wins[i].y0 / y1, writes *wins[i].out
    const IntegDesc *integ;         // list mode: statistics to form once every window is done (or null)
    int n_integ, n_int;
    unsigned *done;                 // windows completed (integ only); the last CTA integrates and resets it
    int64_t shift_step;
    const float *params;            // stem w [16][2][k], stem gamma/beta, per conv gamma/beta, fc w [16], fc b
    const unsigned char *wimg;      // n_conv x TF_WIMG bytes, BF16, shared-memory image order
    float *logits;
    int *err;
    int n_conv, k_stem, W, G;
    float eps;
    uint32_t spin_ns;               // k_tiny_pipe: the issue warps' sleep between polls of an incomplete barrier
};

__host__ __device__ inline int tiny_param_count(int k_stem, int n_conv) {
    return TF_C * 2 * k_stem + 2 * TF_C + n_conv * 2 * TF_C + TF_C + 1;
}

struct Smem {
    size_t off_a, off_b, off_w, off_p, off_s, off_r, off_misc, total;
};

__host__ __device__ inline Smem tiny_smem(int W, int n_conv, int k_stem) {
    Smem s;
    const size_t act = (size_t)2 * (W + 2) * 16;
    s.off_a = 0;
    s.off_b = act;
    s.off_w = 2 * act;
    s.off_p = s.off_w + (size_t)n_conv * TF_WIMG;
    s.off_s = s.off_p + (((size_t)tiny_param_count(k_stem, n_conv) * 4 + 15) / 16) * 16;
    s.off_r = s.off_s + 2 * TF_C * 4;
    s.off_misc = s.off_r + (size_t)(TF_WARPS * 32 + 64) * 4;  // partials [16][32] + moments and channel stats
    s.total = s.off_misc + 64;
    return s;
}


// x rounded to BF16 (nearest even) and back: the operand precision of the tensor-core stem
__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Sum NV per-lane values over the warp (NV a power of two <= 32) so that lane l ends with
// the warp total of value l / (32 / NV) in v[0]: each butterfly stage keeps the half of the
// values selected by the lane's bit and adds the partner's copy (NV - 1 shuffles in all,
// instead of 5 per value), then plain butterflies finish the lanes that share a value.
template <int NV>
__device__ __forceinline__ void warp_reduce_scatter(float (&v)[NV], int lane) {
#pragma unroll
    for (int off = 16, h = NV / 2; h >= 1; off >>= 1, h >>= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = up ? v[i] : v[i + h];
            const float keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
#pragma unroll
    for (int off = 16 / NV; off >= 1; off >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
}

// Reduce per-thread group sums (s[g], q[g], g < G) over the block and write the
// per-channel affine map of GroupNorm: scale[c] = rstd_g * gamma_c,
// shift[c] = beta_c - mean_g * scale[c].  cnt = elements per group.
template <int G>
__device__ __forceinline__ void gn_reduce(float (&s)[TF_C], float (&q)[TF_C], float cnt, float eps,
                                          const float *gamma, const float *beta, float *red, float *scale,
                                          float *shift) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NV = 2 * G;  // sums then sums of squares
    float v[NV];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        v[g] = s[g];
        v[G + g] = q[g];
    }
    warp_reduce_scatter<NV>(v, lane);
    if ((lane & (32 / NV - 1)) == 0) red[warp * 2 * TF_C + lane / (32 / NV)] = v[0];  // [warp][s(G) q(G)]
    __syncthreads();
    if (threadIdx.x < TF_C) {
        const int c = threadIdx.x;
        const int cg = TF_C / G;
        const int g = c / cg;
        float ts = 0.f, tq = 0.f;
        for (int w = 0; w < TF_WARPS; ++w) {
            ts += red[w * 2 * TF_C + g];
            tq += red[w * 2 * TF_C + G + g];
        }
        const float mean = ts / cnt;
        const float var = fmaxf(tq / cnt - mean * mean, 0.f);
        const float a = rsqrtf(var + eps) * gamma[c];
        scale[c] = a;
        shift[c] = beta[c] - mean * a;
    }
    __syncthreads();
}

// ---- clusters of CTAs sharing one window (list mode with few windows): barrier over all
// threads of the cluster (release/acquire orders shared-memory writes before it with reads
// after it in every CTA) and loads from another CTA's shared memory
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// address of shared variable p in the shared memory of cluster CTA `rank`
__device__ __forceinline__ uint32_t dsmem_addr(const void *p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(tc::smem_addr(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ float dsmem_ld(const float *p, uint32_t rank) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(dsmem_addr(p, rank)) : "memory");
    return v;
}
// sum of x[i] over the CL CTAs of the cluster, in rank order (the same total in every CTA)
template <int CL> __device__ __forceinline__ float cluster_sum(const float *x) {
    float t = 0.f;
#pragma unroll
    for (int r = 0; r < CL; ++r) t += dsmem_ld(x, (uint32_t)r);
    return t;
}

// gn_reduce for a window split over a cluster of CL CTAs: the block totals of the
// 2 G group sums go through xch (shared memory, 2 G floats) to every CTA of the cluster
template <int G, int CL>
__device__ __forceinline__ void gn_reduce_cluster(float (&s)[TF_C], float (&q)[TF_C], float cnt, float eps,
                                                  const float *gamma, const float *beta, float *red, float *scale,
                                                  float *shift, float *xch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NV = 2 * G;
    float v[NV];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        v[g] = s[g];
        v[G + g] = q[g];
    }
    warp_reduce_scatter<NV>(v, lane);
    if ((lane & (32 / NV - 1)) == 0) red[warp * 2 * TF_C + lane / (32 / NV)] = v[0];
    __syncthreads();
    if (threadIdx.x < NV) {
        float t = 0.f;
        for (int w = 0; w < TF_WARPS; ++w) t += red[w * 2 * TF_C + threadIdx.x];
        xch[threadIdx.x] = t;
    }
    cluster_sync_all();
    if (threadIdx.x < TF_C) {
        const int c = threadIdx.x, g = c / (TF_C / G);
        const float mean = cluster_sum<CL>(xch + g) / cnt;
        const float var = fmaxf(cluster_sum<CL>(xch + G + g) / cnt - mean * mean, 0.f);
        const float a = rsqrtf(var + eps) * gamma[c];
        scale[c] = a;
        shift[c] = beta[c] - mean * a;
    }
    __syncthreads();
}

// One conv of the fused network as straight-line MMAs (M subtile j, tap r): A = activation
// rows 128 j + r .. (a 16-byte shift per row), B = the tap's 16 x 16 weights.  Issued without
// loops: a loop around single tcgen05.mma instructions costs 150-270 cycles per iteration.
template <int MT>
__device__ __forceinline__ void tiny_issue(uint32_t tmem, uint64_t ad00, uint64_t bd00, uint32_t idesc) {
#pragma unroll
    for (int j = 0; j < MT; ++j)
#pragma unroll
        for (int r = 0; r < 3; ++r)
            tc::mma_bf16(tmem + (uint32_t)(j * TF_C), ad00 + (uint64_t)(128 * j + r), bd00 + (uint64_t)(32 * r), idesc,
                         r > 0 ? 1u : 0u);
}

// Where window `win` lives: single series, (segment, timeslide, window) in batch mode, or an
// explicit pointer pair in list mode.  start + t < n_y and l1_shift < n_y, so one conditional
// subtraction wraps the shifted L1 index.
struct WinLoc {
    const float *y0, *y1;
    float *out_ptr;
    int64_t n_y, start, l1_shift, out;
};

// segs: the segment descriptors (the kernel's shared-memory copy where it made one)
__device__ __forceinline__ WinLoc locate_window(const TinyArgs &args, int64_t win, const SegDesc *segs) {
    WinLoc w;
    w.y0 = args.y;
    w.y1 = nullptr;
    w.out_ptr = nullptr;
    w.n_y = args.n_y;
    w.start = args.first + win * args.stride;
    w.l1_shift = args.shift;
    w.out = win;
    if (win >= args.n_win) return w;
    if (args.wins) {
        const WinPtr wp = args.wins[win];
        w.y0 = wp.y0;
        w.y1 = wp.y1;
        w.out_ptr = wp.out;
        w.start = 0;
        w.l1_shift = 0;
        w.n_y = INT64_MAX / 4;
    } else if (args.n_seg > 0) {
        int lo = 0, hi = args.n_seg - 1;  // last segment with win_first <= win
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (segs[mid].win_first <= win) lo = mid;
            else hi = mid - 1;
        }
        const SegDesc sd = segs[lo];
        const int64_t local = win - sd.win_first;
        const int64_t k = local / sd.n_win;  // timeslide index (0-based)
        const int64_t j = local - k * sd.n_win;
        w.y0 = args.y + sd.y_off;
        w.n_y = sd.n_y;
        w.start = j * args.stride;
        w.l1_shift = ((sd.shift_first + k) * args.shift_step) % w.n_y;
    }
    if (!w.y1) w.y1 = w.y0 + args.y_stride;
    return w;
}

// Stage the window into xs: detector d's sample s at xs[d * (W + 8) + 4 + s] (16-byte
// aligned), zero pads just before and after each row.  Plain loads, or cp.async copies that
// the caller waits for: 16 bytes at a time where both rows are 16-byte aligned and the
// circular L1 index cannot wrap inside 4 samples, else 4 bytes.
__device__ __forceinline__ void load_window(const TinyArgs &args, const WinLoc &w, float *xs, int W, int pad,
                                            bool async, int nthreads = TF_THREADS) {
    const int RP = W + 8;
    if (threadIdx.x < 4 * pad) {  // zero pads (pad <= 3) of both rows
        const int d = threadIdx.x & 1, i = threadIdx.x >> 1;  // i < pad: left; i >= pad: right
        const int s = i < pad ? -1 - i : W + (i - pad);
        if (s < W + pad) xs[d * RP + 4 + s] = 0.f;
    }
    const bool vec = async && ((w.start | w.l1_shift | w.n_y) & 3) == 0 &&
                     ((reinterpret_cast<uintptr_t>(w.y0 + w.start) | reinterpret_cast<uintptr_t>(w.y1)) & 15) == 0;
    if (vec) {
        for (int c = threadIdx.x; c < 2 * (W / 4); c += nthreads) {
            const int d = c >= W / 4, s = 4 * (c - d * (W / 4));
            const float *src;
            if (d == 0) {
                src = w.y0 + w.start + s;
            } else {
                int64_t i1 = w.start + w.l1_shift + s;
                if (i1 >= w.n_y) i1 -= w.n_y;
                src = w.y1 + i1;
            }
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_addr(xs + d * RP + 4 + s)),
                         "l"(src)
                         : "memory");
        }
    } else {
        for (int c = threadIdx.x; c < 2 * W; c += nthreads) {
            const int d = c >= W, s = c - d * W;
            const float *src;
            if (d == 0) {
                src = w.y0 + w.start + s;
            } else {
                int64_t i1 = w.start + w.l1_shift + s;
                if (i1 >= w.n_y) i1 -= w.n_y;
                src = w.y1 + i1;
            }
            if (async)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(tc::smem_addr(xs + d * RP + 4 + s)),
                             "l"(src)
                             : "memory");
            else
                xs[d * RP + 4 + s] = *src;
        }
    }
    if (async) asm volatile("cp.async.commit_group;" ::: "memory");
}

// CL > 1 (list mode only): a cluster of CL CTAs shares each window, CTA rank q taking
// positions [q W / CL, (q + 1) W / CL); GroupNorm statistics, the stem moments and the
// pooled head sums are summed over the cluster.  The halo rows (one neighbour position per
// side) are built locally: the stem's from one more input sample per side, a conv's from
// the neighbours' raw boundary accumulators and residuals, published with the GroupNorm
// partials, so each layer costs one cluster barrier.  Every CTA of a cluster
// runs the same sequence of cluster barriers whatever happens, so none can wait alone.
template <int G, int CL = 1>
__global__ void __launch_bounds__(TF_THREADS, 1) k_tiny_fused(const TinyArgs args) {
    extern __shared__ __align__(1024) unsigned char sm[];
    pdl_trigger();
    const int W = args.W, Wl = W / CL, k = args.k_stem, pad = k / 2, n_conv = args.n_conv;
    const Smem L = tiny_smem(Wl, n_conv, k);
    const uint32_t rank = CL > 1 ? cluster_rank() : 0u;
    float *xch = reinterpret_cast<float *>(sm + L.total);  // CL > 1: exchange area (TF_XCH)
    unsigned char *actA = sm + L.off_a;
    unsigned char *actB = sm + L.off_b;
    unsigned char *wimg = sm + L.off_w;
    float *prm = reinterpret_cast<float *>(sm + L.off_p);
    float *scale = reinterpret_cast<float *>(sm + L.off_s);
    float *shift = scale + TF_C;
    float *red = reinterpret_cast<float *>(sm + L.off_r);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L.off_misc);  // [TF_GROUPS]: MMA groups of a conv
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + L.off_misc + 8 * TF_GROUPS);
    int *abort_flag = reinterpret_cast<int *>(sm + L.off_misc + 8 * TF_GROUPS + 4);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t act_chunk = (size_t)(Wl + 2) * 16;  // bytes of one 8-channel chunk
    const int MT = Wl / 128;

    // ---- one-time set-up: parameters, weight image, zero pad rows, barrier, TMEM
    const int n_prm = tiny_param_count(k, n_conv);
    for (int i = tid; i < n_prm; i += TF_THREADS) prm[i] = args.params[i];
    for (int i = tid; i < n_conv * TF_WIMG / 16; i += TF_THREADS)
        reinterpret_cast<uint4 *>(wimg)[i] = reinterpret_cast<const uint4 *>(args.wimg)[i];
    if (tid < 8) {
        unsigned char *buf = (tid & 4) ? actB : actA;
        const int c = (tid >> 1) & 1, row = (tid & 1) ? Wl + 1 : 0;
        *reinterpret_cast<uint4 *>(buf + c * act_chunk + (size_t)row * 16) = make_uint4(0, 0, 0, 0);
    }
    // batch mode: the segment descriptors in shared memory (after the layout), so that locating a
    // window (a binary search per window, on every window's critical path) reads no global memory
    if (CL == 1 && args.seg_cache > 0) {
        SegDesc *seg_sm = reinterpret_cast<SegDesc *>(sm + L.total);
        for (int i = tid; i < args.seg_cache; i += TF_THREADS) seg_sm[i] = args.segs[i];
    }
    // (recomputed where used: keeping the pointer live across the window loop costs a register)
    auto segs_at = [&]() -> const SegDesc * {
        return (CL == 1 && args.seg_cache > 0) ? reinterpret_cast<const SegDesc *>(sm + tiny_smem(Wl, n_conv, k).total)
                                               : args.segs;
    };
    if (tid == 0) {
        for (int g = 0; g < TF_GROUPS; ++g) tc::mbar_init(&bar[g], 1);
        tc::fence_mbar_init();
        *abort_flag = 0;
    }
    // a split window needs at most 96 columns: 128 leaves room for CTAs of one cluster that share an SM
    if (warp == 0) {
        tc::tmem_alloc(tmem_slot, CL > 1 ? 128 : 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const float *stem_w = prm;
    const float *stem_g = prm + TF_C * 2 * k;
    const float *stem_b = stem_g + TF_C;
    const float *conv_gb = stem_b + TF_C;           // per conv: gamma[16], beta[16]
    const float *fc_w = conv_gb + n_conv * 2 * TF_C;
    const float fc_b = fc_w[TF_C];
    const uint32_t idesc = tc::idesc_bf16_f32(128, TF_C);
    const float cnt = (float)W * (float)(TF_C / G);
    uint32_t phase = 0;

    // staging for the raw window (2 rows of Wl + 8 floats) inside buffer B, past its first pad row
    float *xs = reinterpret_cast<float *>(actB + 16);
    const float *xs0 = xs + 4 - pad, *xs1 = xs + (Wl + 8) + 4 - pad;  // padded index p of each detector row

    const int64_t win0 = blockIdx.x / CL, win_step = gridDim.x / CL;
    WinLoc cur = locate_window(args, win0, segs_at());
    bool prefetched = false;  // the window's samples were copied asynchronously during the previous one
    pdl_wait();  // list mode: the whitened rings come from the whitening launch before (set-up above overlaps it)
    for (int64_t win = win0; win < args.n_win; win += win_step) {
        if (CL > 1) {
            // this CTA's slice of the window with pad samples each side (zero beyond the window)
            cur = locate_window(args, win, segs_at());
            // pad + 1 samples each side: the stem of the halo positions -1 and Wl is computed here too
            const int q0 = (int)rank * Wl, mg = pad + 1, n = Wl + 2 * mg, RP = Wl + 8;
            for (int c = tid; c < 2 * n; c += TF_THREADS) {
                const int d = c >= n, sl = c - d * n - mg, g = q0 + sl;
                xs[d * RP + 4 + sl] = (g >= 0 && g < W) ? (d ? cur.y1 : cur.y0)[g] : 0.f;
            }
        } else if (prefetched) {
            asm volatile("cp.async.wait_all;" ::: "memory");
        } else {
            load_window(args, cur, xs, W, pad, false);
        }
        __syncthreads();
        const int64_t out = cur.out;
        float *out_ptr = cur.out_ptr;
        const int64_t win_next = win + win_step;
        prefetched = false;
        // ---- stem pass 1: GroupNorm statistics of the k = 3 stem from the moments
        // of its six inputs u = (x0[t..t+2], x1[t..t+2]):  sum_t y_c = w_c . S and
        // sum_t y_c^2 = w_c^T M w_c, with S = sum_t u and M = sum_t u u^T
        {
            float S[6], M[21];
#pragma unroll
            for (int i = 0; i < 6; ++i) S[i] = 0.f;
#pragma unroll
            for (int i = 0; i < 21; ++i) M[i] = 0.f;
#pragma unroll 2
            for (int t = tid; t < Wl; t += TF_THREADS) {
                float u[6];
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    u[r] = bf16_round(xs0[t + r]);
                    u[3 + r] = bf16_round(xs1[t + r]);
                }
                // upper triangle row by row; two entries of a row per packed FP32x2 FMA
                int m = 0;
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    S[i] += u[i];
#pragma unroll
                    for (int jj = i; jj < 6; jj += 2) {
                        if (jj + 1 < 6) {
                            const float2 r2 = __ffma2_rn(make_float2(u[jj], u[jj + 1]), make_float2(u[i], u[i]),
                                                         make_float2(M[m], M[m + 1]));
                            M[m] = r2.x;
                            M[m + 1] = r2.y;
                            m += 2;
                        } else {
                            M[m] = fmaf(u[i], u[jj], M[m]);
                            ++m;
                        }
                    }
                }
            }
            // block reduction of the 27 moments (fixed order): warp reduce-scatter, then warps
            {
                float v[32];
#pragma unroll
                for (int i = 0; i < 6; ++i) v[i] = S[i];
#pragma unroll
                for (int i = 0; i < 21; ++i) v[6 + i] = M[i];
#pragma unroll
                for (int i = 27; i < 32; ++i) v[i] = 0.f;
                warp_reduce_scatter<32>(v, lane);  // lane i holds the warp's moment i
                if (lane < 27) red[warp * 32 + lane] = v[0];
            }
            __syncthreads();
            if (tid < 27) {
                float tot = 0.f;
                for (int w = 0; w < TF_WARPS; ++w) tot += red[w * 32 + tid];
                if (CL > 1) xch[tid] = tot;
                else red[TF_WARPS * 32 + tid] = tot;
            }
            if (CL > 1) {
                cluster_sync_all();
                if (tid < 27) red[TF_WARPS * 32 + tid] = cluster_sum<CL>(xch + tid);
            }
            __syncthreads();
            if (tid < TF_C) {
                const float *mom = red + TF_WARPS * 32;
                float wc[6];  // [ci][r] = u order
#pragma unroll
                for (int i = 0; i < 6; ++i) wc[i] = bf16_round(stem_w[tid * 6 + i]);
                float mean = 0.f, e2 = 0.f;
#pragma unroll
                for (int i = 0; i < 6; ++i) mean = fmaf(wc[i], mom[i], mean);
                int m = 6;
#pragma unroll
                for (int i = 0; i < 6; ++i)
#pragma unroll
                    for (int jj = i; jj < 6; ++jj) {
                        const float v = wc[i] * wc[jj] * mom[m++];
                        e2 += (jj == i) ? v : 2.f * v;
                    }
                red[TF_WARPS * 32 + 32 + tid] = mean / (float)W;
                red[TF_WARPS * 32 + 48 + tid] = e2 / (float)W;
            }
            __syncthreads();
            if (tid < TF_C) {
                const int cg = TF_C / G, g = tid / cg;
                const float *cm = red + TF_WARPS * 32 + 32, *ce = red + TF_WARPS * 32 + 48;
                float mean = 0.f, e2 = 0.f;
                for (int c = g * cg; c < (g + 1) * cg; ++c) {
                    mean += cm[c];
                    e2 += ce[c];
                }
                mean /= (float)cg;
                e2 /= (float)cg;
                const float a = rsqrtf(fmaxf(e2 - mean * mean, 0.f) + args.eps) * stem_g[tid];
                scale[tid] = a;
                shift[tid] = stem_b[tid] - mean * a;
            }
            __syncthreads();
        }
        // ---- stem pass 2: conv + GN + ReLU -> BF16 into A (rows 1..W); each thread
        // owns one 8-channel chunk with its 48 weights in registers
        {
            const int h = tid & 1;
            float wr[8][6], sc8[8], sh8[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
#pragma unroll
                for (int i = 0; i < 6; ++i) wr[c][i] = bf16_round(stem_w[(h * 8 + c) * 6 + i]);
                sc8[c] = scale[h * 8 + c];
                sh8[c] = shift[h * 8 + c];
            }
            unsigned char *dstc = actA + h * act_chunk;
#pragma unroll 2
            for (int t = tid >> 1; t < Wl; t += TF_THREADS / 2) {
                float u[6];
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    u[r] = bf16_round(xs0[t + r]);
                    u[3 + r] = bf16_round(xs1[t + r]);
                }
                uint32_t pk[4];
#pragma unroll
                for (int c = 0; c < 8; c += 2) {
                    float a0 = 0.f, a1 = 0.f;
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        a0 = fmaf(wr[c][i], u[i], a0);
                        a1 = fmaf(wr[c + 1][i], u[i], a1);
                    }
                    pk[c / 2] = tc::pack_bf16x2_relu(fmaf(a0, sc8[c], sh8[c]), fmaf(a1, sc8[c + 1], sh8[c + 1]));
                }
                *reinterpret_cast<uint4 *>(dstc + (size_t)(t + 1) * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
            if (CL > 1 && tid < 4) {
                // halo rows 0 and Wl + 1: the stem at local positions -1 and Wl, the neighbours' edge
                // positions, from the same samples, weights and cluster statistics (zero outside the window)
                const int t = (tid >> 1) ? Wl : -1, g = (int)rank * Wl + t;
                uint32_t pk[4] = {0u, 0u, 0u, 0u};
                if (g >= 0 && g < W) {
                    float u[6];
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        u[r] = bf16_round(xs0[t + r]);
                        u[3 + r] = bf16_round(xs1[t + r]);
                    }
#pragma unroll
                    for (int c = 0; c < 8; c += 2) {
                        float a0 = 0.f, a1 = 0.f;
#pragma unroll
                        for (int i = 0; i < 6; ++i) {
                            a0 = fmaf(wr[c][i], u[i], a0);
                            a1 = fmaf(wr[c + 1][i], u[i], a1);
                        }
                        pk[c / 2] = tc::pack_bf16x2_relu(fmaf(a0, sc8[c], sh8[c]), fmaf(a1, sc8[c + 1], sh8[c + 1]));
                    }
                }
                *reinterpret_cast<uint4 *>(dstc + (size_t)(t + 1) * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
        }
        tc::fence_proxy_async_smem();
        __syncthreads();

        float hs[TF_C];
#pragma unroll
        for (int c = 0; c < TF_C; ++c) hs[c] = 0.f;
        bool aborted = false;
        for (int l = 0; l < n_conv; ++l) {
            const bool second = (l & 1) != 0;  // second conv of a block: residual from A
            unsigned char *src = second ? actB : actA;
            unsigned char *dst = second ? actA : actB;
            const bool last = l == n_conv - 1;
            // ---- issue the conv as MT x 3 MMAs in TF_GROUPS commit groups of M subtiles, so that
            // the statistics of a group are read while the later groups still run
            const int GS = (MT + TF_GROUPS - 1) / TF_GROUPS;
            if (tid == 0) {
                tc::fence_after_sync();
                const uint64_t ad00 = tc::desc_kmajor_noswizzle(tc::smem_addr(src), (uint32_t)act_chunk, 128);
                const uint64_t bd00 = tc::desc_kmajor_noswizzle(tc::smem_addr(wimg + (size_t)l * TF_WIMG), 256, 128);
                for (int g = 0; g < TF_GROUPS; ++g) {
                    const int j_lo = g * GS, j_hi = min(MT, j_lo + GS);
                    if (MT == 24) {
                        tiny_issue<8>(tmem + (uint32_t)(j_lo * TF_C), ad00 + (uint64_t)(128 * j_lo), bd00,
                                      idesc);  // 1.5 s windows at 2048 Hz
                    } else if (MT == 6) {
                        tiny_issue<2>(tmem + (uint32_t)(j_lo * TF_C), ad00 + (uint64_t)(128 * j_lo), bd00,
                                      idesc);  // a quarter of such a window (cluster of 4)
                    } else if (MT == 3) {
                        tiny_issue<1>(tmem + (uint32_t)(j_lo * TF_C), ad00 + (uint64_t)(128 * j_lo), bd00,
                                      idesc);  // an eighth of such a window (cluster of 8)
                    } else {
                        for (int j = j_lo; j < j_hi; ++j)
                            for (int r = 0; r < 3; ++r)
                                tc::mma_bf16(tmem + (uint32_t)(j * TF_C), ad00 + (uint64_t)(128 * j + r),
                                             bd00 + (uint64_t)(32 * r), idesc, r > 0 ? 1u : 0u);
                    }
                    tc::mma_commit(&bar[g]);
                }
            }
            const uint32_t tq = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
            // ---- epilogue pass 1: GroupNorm statistics, group by group as the MMAs complete;
            // (sum, sum of squares) of a group as one packed FP32x2 FMA per value
            {
                float2 sq[G];
#pragma unroll
                for (int g = 0; g < G; ++g) sq[g] = make_float2(0.f, 0.f);
                bool ok = true;
                for (int grp = 0; grp < TF_GROUPS; ++grp) {
                    if (!tc::mbar_wait(&bar[grp], phase & 1, 1000000000ull)) ok = false;
                    tc::fence_after_sync();
                    const int j_lo = grp * GS, j_hi = min(MT, j_lo + GS);
                    for (int j0 = j_lo + (warp >> 2); j0 < j_hi; j0 += 2 * (TF_WARPS / 4)) {
                        const int j1 = j0 + TF_WARPS / 4;
                        uint32_t r0[16], r1[16];
                        tc::tmem_ld16_nowait(tq + (uint32_t)(j0 * TF_C), r0);
                        if (j1 < j_hi) tc::tmem_ld16_nowait(tq + (uint32_t)(j1 * TF_C), r1);
                        tc::tmem_wait_ld();
                        if (CL > 1 && !last) {
                            // raw accumulators of the CTA's first position (subtile 0, lane 0) and last
                            // (subtile MT - 1, lane 127): the neighbours build their halo rows from them
                            float *bnd = xch + 64 + 48 * (l & 1);
                            if ((warp & 3) == 0 && lane == 0 && j0 == 0)
#pragma unroll
                                for (int c = 0; c < TF_C; ++c) bnd[c] = __uint_as_float(r0[c]);
                            if ((warp & 3) == 3 && lane == 31) {
                                if (j0 == MT - 1) {
#pragma unroll
                                    for (int c = 0; c < TF_C; ++c) bnd[16 + c] = __uint_as_float(r0[c]);
                                } else if (j1 == MT - 1 && j1 < j_hi) {
#pragma unroll
                                    for (int c = 0; c < TF_C; ++c) bnd[16 + c] = __uint_as_float(r1[c]);
                                }
                            }
                        }
#pragma unroll
                        for (int c = 0; c < TF_C; ++c) {
                            const float v = __uint_as_float(r0[c]);
                            sq[c / (TF_C / G)] = __ffma2_rn(make_float2(v, v), make_float2(1.f, v), sq[c / (TF_C / G)]);
                        }
                        if (j1 < j_hi) {
#pragma unroll
                            for (int c = 0; c < TF_C; ++c) {
                                const float v = __uint_as_float(r1[c]);
                                sq[c / (TF_C / G)] =
                                    __ffma2_rn(make_float2(v, v), make_float2(1.f, v), sq[c / (TF_C / G)]);
                            }
                        }
                    }
                }
                phase++;
                if (!ok) {
                    atomicExch(args.err, 1);
                    *abort_flag = 1;
                }
                __syncthreads();
                if (*abort_flag && CL == 1) {  // (a cluster CTA carries on: its partners wait at barriers)
                    aborted = true;
                    break;
                }
                if (CL == 1 && last && win_next < args.n_win) {
                    // buffer B (the staging of the raw window) is free once the last conv's MMAs
                    // have read it: copy the next window's samples meanwhile
                    cur = locate_window(args, win_next, segs_at());
                    load_window(args, cur, xs, W, pad, true);
                    prefetched = true;
                }
                float s[TF_C], q[TF_C];
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    s[g] = sq[g].x;
                    q[g] = sq[g].y;
                }
                const float *gb = conv_gb + l * 2 * TF_C;
                if (CL > 1 && !last && second && tid < 4) {
                    // the residual (block input) of the first and last positions, before pass 2 overwrites it
                    const int side = tid >> 1, ch = tid & 1;
                    *reinterpret_cast<uint4 *>(xch + 64 + 48 * (l & 1) + 32 + 8 * side + 4 * ch) =
                        *reinterpret_cast<const uint4 *>(actA + ch * act_chunk + (size_t)(side ? Wl : 1) * 16);
                }
                if (CL > 1) gn_reduce_cluster<G, CL>(s, q, cnt, args.eps, gb, gb + TF_C, red, scale, shift, xch + 32);
                else gn_reduce<G>(s, q, cnt, args.eps, gb, gb + TF_C, red, scale, shift);
                if (CL > 1 && !last && tid < 4) {
                    // halo rows of dst: the neighbours' edge outputs, computed here with the same arithmetic
                    // as pass 2 (normalise, residual, ReLU in the BF16 conversion) from their raw accumulators
                    const int side = tid >> 1, ch = tid & 1;
                    if (side ? rank + 1 < (uint32_t)CL : rank > 0) {
                        const uint32_t nb = side ? rank + 1 : rank - 1;
                        const float *bnd = xch + 64 + 48 * (l & 1);
                        const int from = side ? 0 : 16;  // right neighbour's first position, left's last
                        uint32_t pk[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int c = ch * 8 + 2 * e;
                            float2 v = __ffma2_rn(make_float2(dsmem_ld(bnd + from + c, nb), dsmem_ld(bnd + from + c + 1, nb)),
                                                  make_float2(scale[c], scale[c + 1]), make_float2(shift[c], shift[c + 1]));
                            if (second) {
                                const uint32_t w = __float_as_uint(dsmem_ld(bnd + 32 + 8 * (side ? 0 : 1) + 4 * ch + e, nb));
                                v = __fadd2_rn(v, make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u)));
                            }
                            pk[e] = tc::pack_bf16x2_relu(v.x, v.y);
                        }
                        *reinterpret_cast<uint4 *>(dst + ch * act_chunk + (size_t)(side ? Wl + 1 : 0) * 16) =
                            make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    }
                }
            }
            // ---- epilogue pass 2: normalise (+ residual) + ReLU -> BF16 (two subtiles per TMEM wait)
            {
                float sc[TF_C], sh[TF_C];
#pragma unroll
                for (int c = 0; c < TF_C; ++c) {
                    sc[c] = scale[c];
                    sh[c] = shift[c];
                }
                for (int j0 = warp >> 2; j0 < MT; j0 += 2 * (TF_WARPS / 4)) {
                    const int j1 = j0 + TF_WARPS / 4;
                    const bool two = j1 < MT;
                    uint32_t r0[16], r1[16];
                    tc::tmem_ld16_nowait(tq + (uint32_t)(j0 * TF_C), r0);
                    if (two) tc::tmem_ld16_nowait(tq + (uint32_t)(j1 * TF_C), r1);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        if (half == 1 && !two) break;
                        const int j = half ? j1 : j0;
                        const uint32_t *rr = half ? r1 : r0;
                        const int row = 128 * j + 32 * (warp & 3) + lane + 1;
#pragma unroll
                        for (int ch = 0; ch < 2; ++ch) {
                            // normalise, residual add, ReLU two channels per instruction (packed FP32x2);
                            // the ReLU of stored values is folded into the BF16 conversion
                            float2 val[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                val[e] = __ffma2_rn(make_float2(__uint_as_float(rr[ch * 8 + 2 * e]),
                                                                __uint_as_float(rr[ch * 8 + 2 * e + 1])),
                                                    make_float2(sc[ch * 8 + 2 * e], sc[ch * 8 + 2 * e + 1]),
                                                    make_float2(sh[ch * 8 + 2 * e], sh[ch * 8 + 2 * e + 1]));
                            if (second) {
                                const uint4 u = *reinterpret_cast<const uint4 *>(actA + ch * act_chunk +
                                                                                 (size_t)row * 16);
                                const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                                for (int e = 0; e < 4; ++e)
                                    val[e] = __fadd2_rn(val[e], make_float2(__uint_as_float(w4[e] << 16),
                                                                            __uint_as_float(w4[e] & 0xffff0000u)));
                            }
                            if (last) {
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    hs[ch * 8 + 2 * e] += fmaxf(val[e].x, 0.f);
                                    hs[ch * 8 + 2 * e + 1] += fmaxf(val[e].y, 0.f);
                                }
                            } else {
                                uint32_t pk[4];
#pragma unroll
                                for (int e = 0; e < 4; ++e) pk[e] = tc::pack_bf16x2_relu(val[e].x, val[e].y);
                                *reinterpret_cast<uint4 *>(dst + ch * act_chunk + (size_t)row * 16) =
                                    make_uint4(pk[0], pk[1], pk[2], pk[3]);
                            }
                        }
                    }
                }
            }
            tc::fence_before_sync();
            tc::fence_proxy_async_smem();
            __syncthreads();
        }
        if (aborted) break;
        // ---- head: global mean pool of the last block's output, then linear
        warp_reduce_scatter<TF_C>(hs, lane);  // lane 2c holds the warp's sum of channel c
        if (!(lane & 1)) red[warp * 2 * TF_C + (lane >> 1)] = hs[0];
        __syncthreads();
        if (CL > 1) {  // channel sums of the cluster: each CTA's block totals through xch
            if (tid < TF_C) {
                float t = 0.f;
                for (int w = 0; w < TF_WARPS; ++w) t += red[w * 2 * TF_C + tid];
                xch[48 + tid] = t;
            }
            cluster_sync_all();
        }
        if (tid < 32 && (CL == 1 || rank == 0)) {
            float part = 0.f;  // lanes 0..15: channel lane over all warps, times its weight
            if (lane < TF_C) {
                if (CL > 1) {
                    part = cluster_sum<CL>(xch + 48 + lane);
                } else {
                    for (int w = 0; w < TF_WARPS; ++w) part += red[w * 2 * TF_C + lane];
                }
                part = fc_w[lane] * (part / (float)W);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            bool last_win = false;
            if (lane == 0) {
                const float z = fc_b + part;
                if (out_ptr) *out_ptr = z;
                else args.logits[out] = z;
                if (args.integ) {  // publish the logit, then count the window
                    __threadfence();
                    last_win = atomicAdd(args.done, 1u) == (unsigned)(args.n_win - 1);
                }
            }
            if (__shfl_sync(0xffffffffu, last_win, 0)) {
                // every logit of the launch is written: the statistics of the new windows, lane l
                // loading logit w - n_int + 1 + l (+ 32 ...) of 8 statistics at a time, then a warp sum
                // in a fixed order (the loads of a batch are all in flight together)
                __threadfence();
                for (int i0 = 0; i0 < args.n_integ; i0 += 8) {
                    float v[8];
#pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        v[b] = 0.f;
                        if (i0 + b < args.n_integ) {
                            const IntegDesc d = args.integ[i0 + b];
                            for (int l = lane; l < args.n_int; l += 32)
                                v[b] += __ldcg(d.ring + (d.w - args.n_int + 1 + l) % STREAM_LR);
                        }
                    }
#pragma unroll
                    for (int b = 0; b < 8; ++b)
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) v[b] += __shfl_xor_sync(0xffffffffu, v[b], o);
                    if (lane < 8 && i0 + lane < args.n_integ) {
                        float tot = v[0];
#pragma unroll
                        for (int b = 1; b < 8; ++b)
                            if (lane == b) tot = v[b];
                        const IntegDesc d = args.integ[i0 + lane];
                        d.out[0] = tot / (float)args.n_int;
                        d.out[1] = __ldcg(d.ring + d.w % STREAM_LR);
                    }
                }
                if (lane == 0) *args.done = 0u;
            }
        }
        __syncthreads();
    }
    // ---- teardown (a prefetch may still be in flight after an abort); a cluster CTA waits
    // until every partner has finished reading its shared memory
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (CL > 1) cluster_sync_all();
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, CL > 1 ? 128 : 512);
}

// ============================================================================
// k_tiny_pipe: the fused 16-channel network with its layers pipelined inside a
// window (one window per CTA pass, persistent over windows).
//
// Warp roles (448 threads):
//   warps 0..11  epilogue: build the stem's im2col tile, then per layer a
//                statistics pass and a normalise pass over the TMEM accumulators;
//                quad q = warp / 4 owns the units u = q, q + 3, .. (a unit is two
//                128-position subtiles, 2u and 2u + 1; each warp reads its TMEM
//                lane quarter warp % 4)
//   warps 12, 13 MMA issue, warp 12 + m for the units u = m, m + 2, .. (one elected
//                lane issues, the warp uniform; two issuing warps because the issue
//                latency of these small MMAs, not the tensor core, bounds one warp)
// Every layer, stem included, is an implicit GEMM with M = 128 positions, N = 16
// channels, accumulators for the whole window in TMEM (W / 128 subtiles x 16
// columns).  Per unit u two mbarriers link the roles:
//   rows_ready[u]  the input rows of unit u of the next layer are in shared
//                  memory (one arrival per warp of the owning quad, after the
//                  warp's writes and proxy fences): its im2col rows for the stem,
//                  else the previous layer's normalised output; the tensor core
//                  also reads the first row of unit u + 1 (the k = 3 halo), so
//                  the MMAs of unit u need rows_ready[u] and [u + 1].
//                  The arrival also releases unit u's accumulator columns,
//                  which the layer's MMAs overwrite (their old values were read
//                  by the normalise pass that produced these rows).
//   mma_done[u]    the MMAs of unit u of the current layer have completed.
// Issue latency, not the tensor core, bounds an issue loop at this size (an M = 128,
// N = 16, K = 16 MMA issues in about 40 cycles when its operands are warp-uniform,
// several times slower when they come from per-lane registers; a wait on a barrier,
// even a completed one, costs about 235): an MMA warp polls every unit's barrier at
// once (lane i tests unit i, then a ballot) and issues its units that are ready.
// So the MMAs of layer k + 1 run while the normalise pass of layer k is still
// writing later subtiles, and the statistics pass of layer k + 1 reads each
// subtile as soon as its MMAs are done; only GroupNorm's block-wide reduction
// separates the layers.  Each barrier completes once per layer, so both roles
// wait on the parity of a running layer count.
//
// Stem (2 -> 16 channels, k = 3): row t of the im2col tile holds the six BF16 taps
// (x0[t-1], x0[t], x0[t+1], x1[t-1], x1[t], x1[t+1], 0, 0): one 16-byte row per
// position, read as the first K half of an M = 128, N = 16, K = 16 MMA.  The
// second K half is addressed 16 bytes on (the next row, finite data) and meets
// zero weights.  The tile sits in buffer B's second channel chunk, the raw FP32
// window (staged by cp.async during the previous window's last layer) in its
// first; both are free by then.
// Shared memory: activation buffers A and B ([2 chunks][W + 2 rows][16 B], rows
// 0 and W + 1 zero), the BF16 weight images (convs, then the stem), the FP32
// parameters, reduction scratch and barriers, then the batch segment table.
// ============================================================================
// The epilogue and issue warp counts are tunable (afg_autotune picks among 8 or 12 epilogue warps and 1 or 2
// issue warps for the fixed geometry); the shared-memory layout is sized for the largest.
constexpr int TP_EPI_WARPS = 12;           // default and largest: 3 quads of epilogue warps
constexpr int TP_MMA_WARPS = 2;             // default: issue warps for the even and odd units
constexpr int TP_MT_MAX = 32;
constexpr int TP_STEM_IMG = 512;  // BF16 image of the stem weights: 16 channels x K = 16
constexpr uint64_t TP_WAIT_NS = 1000000000ull;
constexpr uint32_t TP_SPIN_NS = 64;  // default sleep of the issue warps between polls of an incomplete barrier
constexpr int TP_EPI_RED = TP_EPI_WARPS * 32 + 32;  // floats of one reduction scratch

struct PipeSmem {
    size_t off_a, off_b, off_w, off_p, off_s, off_r, off_bar, total;
};

__host__ __device__ inline PipeSmem pipe_smem(int W, int n_conv, int k_stem) {
    PipeSmem s;
    const size_t act = (size_t)2 * (W + 2) * 16;
    s.off_a = 0;
    s.off_b = act;
    s.off_w = 2 * act;
    s.off_p = s.off_w + (size_t)n_conv * TF_WIMG + TP_STEM_IMG;
    s.off_s = s.off_p + (((size_t)tiny_param_count(k_stem, n_conv) * 4 + 15) / 16) * 16;
    s.off_r = s.off_s + 2 * TF_C * 4;
    // reduction scratch: two halves (layer parity) of [TP_EPI_WARPS][32] floats + a stop flag, then the head's,
    // then per epilogue warp the 16 scales and 16 shifts of the current GroupNorm
    s.off_bar = s.off_r + (size_t)(3 * TP_EPI_RED + TP_EPI_WARPS * 32) * 4;
    // mma_done[TP_MT_MAX], rows_ready[TP_MT_MAX] (per unit; the first MT / 2 used), drain, then the
    // tmem slot, abort flag, stop flag
    s.total = s.off_bar + (2 * TP_MT_MAX + 1) * 8 + 16;
    return s;
}

// Per-channel (sum, sum of squares) of one position's 16 accumulators, adjacent channels as packed pairs
// (the loaded registers are the FP32x2 operands as they are: no register moves).
__device__ __forceinline__ void acc_channel_pairs(const uint32_t (&r)[16], float2 (&s2)[TF_C / 2],
                                                  float2 (&q2)[TF_C / 2]) {
#pragma unroll
    for (int i = 0; i < TF_C / 2; ++i) {
        const float2 v = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
        s2[i] = __fadd2_rn(s2[i], v);
        q2[i] = __ffma2_rn(v, v, q2[i]);
    }
}

// GroupNorm reduction over the epilogue warps, one named barrier (id 1): per-thread group sums
// (x: sum, y: sum of squares) -> every warp's lanes hold the per-channel affine map
// (sc[c] = rstd_g gamma_c, sh[c] = beta_c - mean_g sc[c]) and a consistent copy of the abort
// flag (stop).  red is this layer's half of a double buffer: a warp that runs ahead writes the
// next layer's sums into the other half, and cannot get two layers ahead past the barrier.
template <int G, int EW>
__device__ __forceinline__ void gn_reduce_epi(const float2 (&sq)[G], float inv_cnt, float eps, const float *gamma,
                                              const float *beta, float *red, float *maps, float (&sc)[TF_C],
                                              float (&sh)[TF_C], const volatile int *abort_flag, bool &stop) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NV = 2 * G;
    float v[NV];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        v[g] = sq[g].x;
        v[G + g] = sq[g].y;
    }
    warp_reduce_scatter<NV>(v, lane);
    if ((lane & (32 / NV - 1)) == 0) red[warp * 32 + lane / (32 / NV)] = v[0];
    int *stop_slot = reinterpret_cast<int *>(red + TP_EPI_WARPS * 32);
    if (threadIdx.x == 0) *stop_slot = *abort_flag;
    tc::named_bar_sync(1, EW * 32);
    // lane i < 2G: total i over the warps (sums, then sums of squares); lane c (mod 16) then forms
    // channel c's affine map, and the 16 maps are broadcast to every lane
    float t = 0.f;
    if (lane < NV)
#pragma unroll
        for (int w = 0; w < EW; ++w) t += red[w * 32 + lane];
    const int c = lane & (TF_C - 1), g = c / (TF_C / G);
    const float s_g = __shfl_sync(0xffffffffu, t, g), q_g = __shfl_sync(0xffffffffu, t, G + g);
    const float mean = s_g * inv_cnt;  // (a multiply by the reciprocal of the group's element count: no divide)
    const float a = rsqrtf(fmaxf(q_g * inv_cnt - mean * mean, 0.f) + eps) * gamma[c];
    const float b = beta[c] - mean * a;
    // the 16 maps to every lane through the warp's own slot (broadcast loads, adjacent pairs aligned for
    // the packed normalisation)
    float *mw = maps + warp * 32;
    if (lane < TF_C) {
        mw[lane] = a;
        mw[TF_C + lane] = b;
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < TF_C; i += 4) {
        const float4 va = *reinterpret_cast<const float4 *>(mw + i);
        const float4 vb = *reinterpret_cast<const float4 *>(mw + TF_C + i);
        sc[i] = va.x; sc[i + 1] = va.y; sc[i + 2] = va.z; sc[i + 3] = va.w;
        sh[i] = vb.x; sh[i + 1] = vb.y; sh[i + 2] = vb.z; sh[i + 3] = vb.w;
    }
    __syncwarp();  // (the slot is rewritten at the next layer only after every lane has read it)
    stop = *stop_slot != 0;
}

// Window output: the logit (and, in list mode, the statistics of the launch once its last
// window is done; executed by one warp, lane 0 holding z).
__device__ __forceinline__ void tiny_emit(const TinyArgs &args, int64_t out, float *out_ptr, float z, int lane) {
    bool last_win = false;
    if (lane == 0) {
        if (out_ptr) *out_ptr = z;
        else args.logits[out] = z;
        if (args.integ) {  // publish the logit, then count the window
            __threadfence();
            last_win = atomicAdd(args.done, 1u) == (unsigned)(args.n_win - 1);
        }
    }
    if (__shfl_sync(0xffffffffu, last_win, 0)) {
        // every logit of the launch is written: the statistics of the new windows, lane l
        // loading logit w - n_int + 1 + l (+ 32 ...) of 8 statistics at a time, then a warp sum
        // in a fixed order (the loads of a batch are all in flight together)
        __threadfence();
        for (int i0 = 0; i0 < args.n_integ; i0 += 8) {
            float v[8];
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                v[b] = 0.f;
                if (i0 + b < args.n_integ) {
                    const IntegDesc d = args.integ[i0 + b];
                    for (int l = lane; l < args.n_int; l += 32)
                        v[b] += __ldcg(d.ring + (d.w - args.n_int + 1 + l) % STREAM_LR);
                }
            }
#pragma unroll
            for (int b = 0; b < 8; ++b)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v[b] += __shfl_xor_sync(0xffffffffu, v[b], o);
            if (lane < 8 && i0 + lane < args.n_integ) {
                float tot = v[0];
#pragma unroll
                for (int b = 1; b < 8; ++b)
                    if (lane == b) tot = v[b];
                const IntegDesc d = args.integ[i0 + lane];
                d.out[0] = tot / (float)args.n_int;
                d.out[1] = __ldcg(d.ring + d.w % STREAM_LR);
            }
        }
        if (lane == 0) *args.done = 0u;
    }
}

// MTS: the window's subtiles as a compile-time constant (0: from args.W); with a constant that is even
// and whose units divide evenly among the quads and issue warps, every loop over units has a fixed
// trip count and no partial unit
// EW epilogue warps (EW / 4 quads) and MW issue warps.
template <int G, int MTS = 0, int EW = TP_EPI_WARPS, int MW = TP_MMA_WARPS>
__global__ void __launch_bounds__((EW + MW) * 32, 1) k_tiny_pipe(const TinyArgs args) {
    extern __shared__ __align__(1024) unsigned char sm[];
    pdl_trigger();
    constexpr int NQ = EW / 4, EPI = EW * 32, THREADS = (EW + MW) * 32;
    static_assert(EW % 4 == 0 && EW <= TP_EPI_WARPS, "whole quads, within the shared-memory layout");
    constexpr bool FIXED = MTS > 0 && MTS % 2 == 0 && (MTS / 2) % NQ == 0 && (MTS / 2) % MW == 0;
    const int W = MTS > 0 ? 128 * MTS : args.W, n_conv = args.n_conv, MT = W / 128, k_stem = args.k_stem;
    const PipeSmem L = pipe_smem(W, n_conv, k_stem);
    unsigned char *actA = sm + L.off_a;
    unsigned char *actB = sm + L.off_b;
    unsigned char *wimg = sm + L.off_w;
    float *prm = reinterpret_cast<float *>(sm + L.off_p);
    float *red = reinterpret_cast<float *>(sm + L.off_r);
    uint64_t *mma_done = reinterpret_cast<uint64_t *>(sm + L.off_bar);
    uint64_t *rows_ready = mma_done + TP_MT_MAX;
    uint64_t *drain = rows_ready + TP_MT_MAX;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t act_chunk = (size_t)(W + 2) * 16;

    // ---- one-time set-up: parameters, weight images, zero pad rows, barriers, TMEM
    const int n_prm = tiny_param_count(k_stem, n_conv);
    for (int i = tid; i < n_prm; i += THREADS) prm[i] = args.params[i];
    for (int i = tid; i < (n_conv * TF_WIMG + TP_STEM_IMG) / 16; i += THREADS)
        reinterpret_cast<uint4 *>(wimg)[i] = reinterpret_cast<const uint4 *>(args.wimg)[i];
    if (tid < 8) {
        unsigned char *buf = (tid & 4) ? actB : actA;
        const int c = (tid >> 1) & 1, row = (tid & 1) ? W + 1 : 0;
        *reinterpret_cast<uint4 *>(buf + c * act_chunk + (size_t)row * 16) = make_uint4(0, 0, 0, 0);
    }
    // the im2col tile's rows start finite (zero): the stem MMA's second K half (zero weights) also
    // reads the first row of the next subtile, which another quad may not have written yet
    for (int i = tid; i < W; i += THREADS)
        *reinterpret_cast<uint4 *>(actB + act_chunk + 16 + (size_t)i * 16) = make_uint4(0, 0, 0, 0);
    if (args.seg_cache > 0) {
        SegDesc *seg_sm = reinterpret_cast<SegDesc *>(sm + L.total);
        for (int i = tid; i < args.seg_cache; i += THREADS) seg_sm[i] = args.segs[i];
    }
    if (tid == 0) {
        for (int j = 0; j < TP_MT_MAX; ++j) {
            tc::mbar_init(&mma_done[j], 1);
            tc::mbar_init(&rows_ready[j], 4);
        }
        tc::mbar_init(drain, MW);
        tc::fence_mbar_init();
        *abort_flag = 0;
    }
    if (warp == EW) {
        tc::tmem_alloc(tmem_slot, 512);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async_smem();  // weight images and zero rows -> the tensor core
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const SegDesc *segs = args.seg_cache > 0 ? reinterpret_cast<const SegDesc *>(sm + L.total) : args.segs;
    const int64_t win0 = blockIdx.x, win_step = gridDim.x;
    pdl_wait();  // list mode: the whitened rings come from the whitening launch before

    if (warp >= EW) {
        // ================================================================ MMA warps
        const int mw = warp - EW;  // this warp issues the units u = mw, mw + MW, ..
        const uint32_t idesc = tc::idesc_bf16_f32(128, TF_C);
        const uint64_t d_stem_a = tc::desc_kmajor_noswizzle(tc::smem_addr(actB + act_chunk + 16), 16, 128);
        const uint64_t d_stem_b = tc::desc_kmajor_noswizzle(tc::smem_addr(wimg + (size_t)n_conv * TF_WIMG), 256, 128);
        const uint64_t d_a = tc::desc_kmajor_noswizzle(tc::smem_addr(actA), (uint32_t)act_chunk, 128);
        const uint64_t d_b = tc::desc_kmajor_noswizzle(tc::smem_addr(actB), (uint32_t)act_chunk, 128);
        const uint64_t d_w = tc::desc_kmajor_noswizzle(tc::smem_addr(wimg), 256, 128);
        const int NU = (MT + 1) / 2;  // units of two subtiles
        // The issue loops have warp-uniform trip counts and no early exit, so their counters, and the
        // descriptors derived from them, stay warp-uniform.  After a failed wait `ok` turns false and the
        // remaining waits are skipped (the MMAs still issue: they only read shared memory and write
        // accumulators that nothing reads any more).
        uint32_t seq = 0;
        bool ok = true;
        // wait until the leading `need` units have their rows: one poll tests every unit (lane i unit i)
        auto wait_rows = [&](int &ready, int need, uint32_t par) {
            while (ready < need) {
                const bool rdy = lane >= NU || tc::mbar_test_wait(&rows_ready[lane], par);
                const unsigned m = __ballot_sync(0xffffffffu, rdy);
                ready = m == 0xffffffffu ? 32 : __ffs(~m) - 1;
                if (ready < need && !tc::mbar_spin_warp(&rows_ready[ready], par, TP_WAIT_NS, args.spin_ns)) {
                    ok = false;
                    ready = NU;
                }
            }
            tc::fence_after_sync();
        };
        // this warp's i-th unit of a layer, and its count
        const int n_mu = FIXED ? NU / MW : (NU - mw + MW - 1) / MW;
        for (int64_t win = win0; win < args.n_win; win += win_step) {
            {   // stem: one K = 16 MMA per subtile over the im2col tile
                const uint32_t par = seq & 1;
                int ready = ok ? 0 : NU;
                for (int i = 0; i < n_mu; ++i) {
                    const int u = mw + MW * i;
                    wait_rows(ready, u + 1, par);
                    const int j0 = 2 * u;
                    tc::mma_bf16_elect(tmem + (uint32_t)(j0 * TF_C), d_stem_a + (uint64_t)(128 * j0), d_stem_b, idesc, 0u);
                    if (FIXED || j0 + 1 < MT)
                        tc::mma_bf16_elect(tmem + (uint32_t)((j0 + 1) * TF_C), d_stem_a + (uint64_t)(128 * (j0 + 1)),
                                           d_stem_b, idesc, 0u);
                    tc::mma_commit_elect(&mma_done[u]);
                }
                ++seq;
            }
            for (int l = 0; l < n_conv; ++l, ++seq) {  // convs: three taps, a conv also reads the next unit's first row
                const uint32_t par = seq & 1;
                const uint64_t ad = (l & 1) ? d_b : d_a;  // the second conv of a block reads B
                const uint64_t bd = d_w + (uint64_t)(l * (TF_WIMG / 16));
                int ready = ok ? 0 : NU;
                for (int i = 0; i < n_mu; ++i) {
                    const int u = mw + MW * i;
                    wait_rows(ready, min(u + 2, NU), par);
                    const int j0 = 2 * u;
                    const uint64_t a0 = ad + (uint64_t)(128 * j0);
                    const uint32_t t0 = tmem + (uint32_t)(j0 * TF_C);
                    tc::mma_bf16_elect(t0, a0, bd, idesc, 0u);
                    tc::mma_bf16_elect(t0, a0 + 1, bd + 32, idesc, 1u);
                    tc::mma_bf16_elect(t0, a0 + 2, bd + 64, idesc, 1u);
                    if (FIXED || j0 + 1 < MT) {
                        tc::mma_bf16_elect(t0 + TF_C, a0 + 128, bd, idesc, 0u);
                        tc::mma_bf16_elect(t0 + TF_C, a0 + 129, bd + 32, idesc, 1u);
                        tc::mma_bf16_elect(t0 + TF_C, a0 + 130, bd + 64, idesc, 1u);
                    }
                    tc::mma_commit_elect(&mma_done[u]);
                }
            }
            if (*abort_flag) ok = false;  // the epilogue gave up: skip the waits from now on
            ok = __all_sync(0xffffffffu, ok);
        }
        if (!ok) {
            if (lane == 0) atomicExch(args.err, 1);
            *abort_flag = 1;
        }
        // every MMA issued above completes before the accumulators are released
        tc::mma_commit_elect(drain);
        if (!tc::mbar_wait(drain, 0, TP_WAIT_NS) && lane == 0) atomicExch(args.err, 1);
    } else {
        // ================================================================ epilogue warps
        const int q = warp >> 2, lq = warp & 3;
        const uint32_t tq = tmem + ((uint32_t)(32 * lq) << 16);
        const float *stem_g = prm + TF_C * 2 * k_stem;
        const float *stem_b = stem_g + TF_C;
        const float *conv_gb = stem_b + TF_C;
        const float *fc_w = conv_gb + n_conv * 2 * TF_C;
        const float fc_b = fc_w[TF_C];
        const float cnt = (float)W * (float)(TF_C / G);
        float *xs = reinterpret_cast<float *>(actB + 16);   // raw window, [2][W + 8] FP32
        unsigned char *im2col = actB + act_chunk + 16;       // stem im2col tile, [W][16 B]
        const int RP = W + 8;
        uint32_t seq = 0;
        // this quad's i-th unit is u = q + NQ i, i < n_qu
        const int n_qu = FIXED ? (MT / 2) / NQ : ((MT + 1) / 2 - q + NQ - 1) / NQ;
        WinLoc cur = locate_window(args, win0, segs);
        if (win0 < args.n_win) load_window(args, cur, xs, W, 1, true, EPI);
        for (int64_t win = win0; win < args.n_win; win += win_step) {
            const int64_t out = cur.out;
            float *out_ptr = cur.out_ptr;
            asm volatile("cp.async.wait_all;" ::: "memory");
            tc::named_bar_sync(1, EPI);
            // ---- stem im2col rows of this quad's units (BF16, six taps per 16-byte row)
            for (int i = 0; i < n_qu; ++i) {
                const int u = q + NQ * i;
                for (int j = 2 * u; j < (FIXED ? 2 * u + 2 : min(2 * u + 2, MT)); ++j) {
                    const int t = 128 * j + 32 * lq + lane;
                    const float *p0 = xs + 4 + t - 1, *p1 = xs + RP + 4 + t - 1;
                    const uint4 row = make_uint4(tc::pack_bf16x2(p0[0], p0[1]), tc::pack_bf16x2(p0[2], p1[0]),
                                                 tc::pack_bf16x2(p1[1], p1[2]), 0u);
                    *reinterpret_cast<uint4 *>(im2col + (size_t)t * 16) = row;
                }
                tc::fence_proxy_async_smem();
                tc::fence_before_sync();  // (this unit's accumulators were read by the last layer)
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&rows_ready[u]);
            }
            float2 hs2[TF_C / 2];  // pooled sums of adjacent channel pairs (last layer)
#pragma unroll
            for (int c = 0; c < TF_C / 2; ++c) hs2[c] = make_float2(0.f, 0.f);
            bool stopped = false;
            for (int k = 0; k <= n_conv; ++k, ++seq) {
                const uint32_t par = seq & 1;
                const int l = k - 1;
                const bool last = k == n_conv;
                const bool res = k > 0 && (l & 1);  // second conv of a block: residual from A
                unsigned char *dst = (k == 0 || (l & 1)) ? actA : actB;
                const float *gam = k == 0 ? stem_g : conv_gb + l * 2 * TF_C;
                // ---- statistics pass: each subtile as soon as its MMAs are done; per-channel sums and sums
                // of squares of adjacent channel pairs as packed FP32x2 adds and FMAs on the loaded registers
                float2 s2[TF_C / 2], q2[TF_C / 2];
#pragma unroll
                for (int i = 0; i < TF_C / 2; ++i) s2[i] = q2[i] = make_float2(0.f, 0.f);
                bool ok = true;
                for (int i = 0; i < n_qu; ++i) {
                    const int u = q + NQ * i;
                    const int j0 = 2 * u, j1 = j0 + 1;
                    const bool two = FIXED || j1 < MT;
                    uint32_t r0[16], r1[16];
                    // (after a failed wait the rest are skipped: the MMA warp has stopped)
                    if (ok) ok = tc::mbar_wait_warp_tested(&mma_done[u], par, TP_WAIT_NS);
                    tc::fence_after_sync();
                    tc::tmem_ld16_nowait(tq + (uint32_t)(j0 * TF_C), r0);
                    if (two) tc::tmem_ld16_nowait(tq + (uint32_t)(j1 * TF_C), r1);
                    tc::tmem_wait_ld();
                    tc::tmem_regs_ready(r0);
                    tc::tmem_regs_ready(r1);
                    acc_channel_pairs(r0, s2, q2);
                    if (two) acc_channel_pairs(r1, s2, q2);
                }
                float2 sq[G];  // (sum, sum of squares) per group
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    float s = 0.f, qq = 0.f;
#pragma unroll
                    for (int c = g * (TF_C / G); c < (g + 1) * (TF_C / G); ++c) {
                        s += (c & 1) ? s2[c >> 1].y : s2[c >> 1].x;
                        qq += (c & 1) ? q2[c >> 1].y : q2[c >> 1].x;
                    }
                    sq[g] = make_float2(s, qq);
                }
                if (!ok) {
                    atomicExch(args.err, 1);
                    *abort_flag = 1;
                }
                float sc[TF_C], sh[TF_C];
                bool stop_now = false;
                gn_reduce_epi<G, EW>(sq, 1.0f / cnt, args.eps, gam, gam + TF_C, red + (seq & 1) * TP_EPI_RED, red + 3 * TP_EPI_RED,
                                 sc, sh, abort_flag, stop_now);
                if (stop_now) {
                    stopped = true;
                    break;
                }
                if (last && win + win_step < args.n_win) {
                    // every MMA of the last layer is done (its statistics are complete), so buffer B,
                    // its input, is free: stage the next window's samples while this one finishes
                    cur = locate_window(args, win + win_step, segs);
                    load_window(args, cur, xs, W, 1, true, EPI);
                }
                // ---- normalise pass (+ residual) + ReLU -> BF16 rows of dst, or the pooled sums
                for (int i = 0; i < n_qu; ++i) {
                    const int u = q + NQ * i;
                    const int j0 = 2 * u, j1 = j0 + 1;
                    const bool two = FIXED || j1 < MT;
                    uint32_t ra[16], rb[16];
                    tc::tmem_ld16_nowait(tq + (uint32_t)(j0 * TF_C), ra);
                    if (two) tc::tmem_ld16_nowait(tq + (uint32_t)(j1 * TF_C), rb);
                    tc::tmem_wait_ld();
                    tc::tmem_regs_ready(ra);
                    tc::tmem_regs_ready(rb);
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        if (half == 1 && !two) break;
                        const int j = half ? j1 : j0;
                        const uint32_t *rr = half ? rb : ra;
                        const size_t row = (size_t)(128 * j + 32 * lq + lane + 1) * 16;
#pragma unroll
                        for (int ch = 0; ch < 2; ++ch) {
                            float2 v[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                v[e] = __ffma2_rn(make_float2(__uint_as_float(rr[ch * 8 + 2 * e]),
                                                              __uint_as_float(rr[ch * 8 + 2 * e + 1])),
                                                  make_float2(sc[ch * 8 + 2 * e], sc[ch * 8 + 2 * e + 1]),
                                                  make_float2(sh[ch * 8 + 2 * e], sh[ch * 8 + 2 * e + 1]));
                            if (last) {
                                // the block's residual in FP32, ReLU, pooled sums (nothing stored)
                                const uint4 rv = *reinterpret_cast<const uint4 *>(actA + ch * act_chunk + row);
                                const uint32_t w4[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    const float2 y = __fadd2_rn(v[e], make_float2(__uint_as_float(w4[e] << 16),
                                                                                  __uint_as_float(w4[e] & 0xffff0000u)));
                                    hs2[ch * 4 + e] = __fadd2_rn(hs2[ch * 4 + e], make_float2(fmaxf(y.x, 0.f), fmaxf(y.y, 0.f)));
                                }
                            } else if (res) {
                                // + the block's residual in FP32, ReLU folded into the BF16 conversion
                                const uint4 rv = *reinterpret_cast<const uint4 *>(actA + ch * act_chunk + row);
                                const uint32_t w4[4] = {rv.x, rv.y, rv.z, rv.w};
                                uint32_t pk[4];
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    const float2 y = __fadd2_rn(v[e], make_float2(__uint_as_float(w4[e] << 16),
                                                                                  __uint_as_float(w4[e] & 0xffff0000u)));
                                    pk[e] = tc::pack_bf16x2_relu(y.x, y.y);
                                }
                                *reinterpret_cast<uint4 *>(dst + ch * act_chunk + row) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                            } else {
                                *reinterpret_cast<uint4 *>(dst + ch * act_chunk + row) =
                                    make_uint4(tc::pack_bf16x2_relu(v[0].x, v[0].y), tc::pack_bf16x2_relu(v[1].x, v[1].y),
                                               tc::pack_bf16x2_relu(v[2].x, v[2].y), tc::pack_bf16x2_relu(v[3].x, v[3].y));
                            }
                        }
                    }
                    if (!last) {
                        tc::fence_proxy_async_smem();
                        tc::fence_before_sync();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&rows_ready[u]);
                    }
                }
                if (last) tc::fence_before_sync();
            }
            if (stopped) break;
            // ---- head: global mean pool, then the linear layer
            float *hred = red + 2 * TP_EPI_RED;
            float hs[TF_C];
#pragma unroll
            for (int c = 0; c < TF_C / 2; ++c) {
                hs[2 * c] = hs2[c].x;
                hs[2 * c + 1] = hs2[c].y;
            }
            warp_reduce_scatter<TF_C>(hs, lane);  // lane 2c holds the warp's sum of channel c
            if (!(lane & 1)) hred[warp * 32 + (lane >> 1)] = hs[0];
            tc::named_bar_sync(1, EPI);
            if (warp == 0) {
                float part = 0.f;
                if (lane < TF_C) {
                    for (int w = 0; w < EW; ++w) part += hred[w * 32 + lane];
                    part = fc_w[lane] * (part / (float)W);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                tiny_emit(args, out, out_ptr, fc_b + part, lane);
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    // ---- teardown: the MMA warp has drained its MMAs
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == EW) tc::tmem_dealloc(tmem, 512);
}

bool tiny_compatible(const afg_ctx *ctx) {
    const afg_net &n = ctx->cfg.net;
    const int W = ctx->cfg.win_len;
    const int g = n.groups;
    return n.n_stages == 1 && n.widths[0] == TF_C && n.stem_k == 3 && n.stem_stride == 1 && n.stem_pool == 0 &&
           W % 128 == 0 &&
           (W / 128) * TF_C <= 512 && (g == 1 || g == 2 || g == 4 || g == 8 || g == 16) &&
           tiny_smem(W, 2 * n.blocks[0], n.stem_k).total <= 227 * 1024 &&
           pipe_smem(W, 2 * n.blocks[0], n.stem_k).total <= 227 * 1024;
}

// batch segment descriptors the pipelined kernel keeps in shared memory after its layout
__host__ inline int pipe_seg_cache_cap(size_t total) { return tiny_seg_cache_cap(total); }

// subtiles of the 1.5 s window at 2048 Hz (3072 positions): compiled with a fixed geometry
constexpr int TP_MT_FIXED = 24;

template <int G, int MTS, int EW = TP_EPI_WARPS, int MW = TP_MMA_WARPS>
cudaError_t launch_pipe_t(const TinyArgs &a, unsigned grid, size_t smem, cudaStream_t st, bool pdl) {
    constexpr int threads = (EW + MW) * 32;
    if (pdl) return launch_pdl(k_tiny_pipe<G, MTS, EW, MW>, dim3(grid), dim3(threads), smem, st, a);
    k_tiny_pipe<G, MTS, EW, MW><<<grid, threads, smem, st>>>(a);
    return cudaGetLastError();
}

// Tuning candidates of the pipelined network's fixed geometry (8 groups, 3072 positions): epilogue warps,
// issue warps and the issue warps' polling sleep; candidate 0 is the default.
struct PipeVariant {
    int ew, mw;
    uint32_t spin_ns;
};
constexpr PipeVariant kPipeVariants[] = {{12, 2, 64}, {12, 2, 0}, {12, 2, 256}, {12, 1, 64},
                                         {8, 2, 64},  {8, 1, 64}, {8, 1, 0},   {12, 1, 0}};
constexpr int kNPipeVariants = (int)(sizeof(kPipeVariants) / sizeof(kPipeVariants[0]));

// The pipelined network over a.n_win windows (a.spin_ns set by the caller); the fixed-geometry build for
// 8 groups and 3072 positions, with the warp counts ew / mw the context chose
cudaError_t launch_pipe(const TinyArgs &a, unsigned grid, size_t smem, cudaStream_t st, bool pdl, int ew = TP_EPI_WARPS,
                        int mw = TP_MMA_WARPS) {
    switch (a.G) {
        case 1: return launch_pipe_t<1, 0>(a, grid, smem, st, pdl);
        case 2: return launch_pipe_t<2, 0>(a, grid, smem, st, pdl);
        case 4: return launch_pipe_t<4, 0>(a, grid, smem, st, pdl);
        case 8:
            if (a.W != 128 * TP_MT_FIXED) return launch_pipe_t<8, 0>(a, grid, smem, st, pdl);
            if (ew == 8) return mw == 1 ? launch_pipe_t<8, TP_MT_FIXED, 8, 1>(a, grid, smem, st, pdl)
                                        : launch_pipe_t<8, TP_MT_FIXED, 8, 2>(a, grid, smem, st, pdl);
            return mw == 1 ? launch_pipe_t<8, TP_MT_FIXED, 12, 1>(a, grid, smem, st, pdl)
                           : launch_pipe_t<8, TP_MT_FIXED, 12, 2>(a, grid, smem, st, pdl);
        default: return launch_pipe_t<16, 0>(a, grid, smem, st, pdl);
    }
}

}  // namespace

// Build the fused kernel's parameter block and BF16 weight image (device).
int net_tc_prepare(afg_ctx *ctx) {
    NetPlan &P = ctx->plan;
    if (!tiny_compatible(ctx)) return AFG_OK;
    const int k = P.net.stem_k;
    const int n_conv = (int)P.convs.size() - 1;
    std::vector<float> prm((size_t)tiny_param_count(k, n_conv));
    // conv images, then the stem's image (K = ci * 3 + r, zero for K >= 6) for the pipelined kernel
    std::vector<unsigned short> img(((size_t)n_conv * TF_WIMG + TP_STEM_IMG) / 2, 0);
    std::vector<float> host_w;
    // copy the device parameter image back to read the layers' weights
    std::vector<float> all(ctx->d_params_bytes / sizeof(float));
    AFG_CUDA(ctx, cudaMemcpy(all.data(), ctx->d_params, ctx->d_params_bytes, cudaMemcpyDeviceToHost));
    auto at = [&](const float *dptr) { return all.data() + (dptr - ctx->d_params); };
    size_t o = 0;
    const ConvLayer &S = P.convs[0];
    for (int i = 0; i < TF_C * 2 * k; ++i) prm[o++] = at(S.wt)[i];
    // stem weights [co][ci][r] -> image[k = ci * 3 + r][co] (K-major, no swizzle, as the convs' taps)
    for (int co = 0; co < TF_C; ++co)
        for (int kk = 0; kk < 2 * k; ++kk) {
            const size_t byte = (size_t)n_conv * TF_WIMG + (kk / 8) * 256 + co * 16 + (kk % 8) * 2;
            __nv_bfloat16 b = __float2bfloat16_rn(at(S.wt)[co * 2 * k + kk]);
            img[byte / 2] = *reinterpret_cast<unsigned short *>(&b);
        }
    for (int c = 0; c < TF_C; ++c) prm[o++] = at(S.gamma)[c];
    for (int c = 0; c < TF_C; ++c) prm[o++] = at(S.beta)[c];
    for (int l = 0; l < n_conv; ++l) {
        const ConvLayer &C = P.convs[1 + l];
        for (int c = 0; c < TF_C; ++c) prm[o++] = at(C.gamma)[c];
        for (int c = 0; c < TF_C; ++c) prm[o++] = at(C.beta)[c];
        // Wt[(r*cin + ci)*cout + co] -> image[l][r][chunk][co][8] (K-major, no swizzle)
        const float *wt = at(C.wt);
        for (int r = 0; r < 3; ++r)
            for (int ci = 0; ci < TF_C; ++ci)
                for (int co = 0; co < TF_C; ++co) {
                    const float v = wt[((size_t)r * TF_C + ci) * TF_C + co];
                    const size_t byte = (size_t)l * TF_WIMG + r * 512 + (ci / 8) * 256 + co * 16 + (ci % 8) * 2;
                    __nv_bfloat16 b = __float2bfloat16_rn(v);
                    img[byte / 2] = *reinterpret_cast<unsigned short *>(&b);
                }
    }
    for (int c = 0; c < TF_C; ++c) prm[o++] = at(P.fc_w)[c];
    prm[o++] = at(P.fc_b)[0];
    size_t pbytes = prm.size() * sizeof(float), ibytes = img.size() * 2;
    void *d = nullptr;
    if (cudaMalloc(&d, pbytes + ibytes + 256) != cudaSuccess) {
        cudaGetLastError();
        return afg_fail(ctx, AFG_ERR_OOM, "tensor-core weight image: cudaMalloc failed");
    }
    ctx->bytes_held += (int64_t)(pbytes + ibytes + 256);
    P.tc_params = static_cast<float *>(d);
    P.tc_wimg = static_cast<unsigned char *>(d) + ((pbytes + 255) / 256) * 256;
    AFG_CUDA(ctx, cudaMemcpy(P.tc_params, prm.data(), pbytes, cudaMemcpyHostToDevice));
    AFG_CUDA(ctx, cudaMemcpy(P.tc_wimg, img.data(), ibytes, cudaMemcpyHostToDevice));
    const size_t pbase = pipe_smem(ctx->cfg.win_len, n_conv, k).total;
    const int psmem = (int)(pbase + pipe_seg_cache_cap(pbase) * sizeof(SegDesc));
    AFG_CUDA(ctx, cudaFuncSetAttribute(k_tiny_pipe<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, psmem));
    AFG_CUDA(ctx, cudaFuncSetAttribute(k_tiny_pipe<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, psmem));
    AFG_CUDA(ctx, cudaFuncSetAttribute(k_tiny_pipe<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, psmem));
    AFG_CUDA(ctx, cudaFuncSetAttribute(k_tiny_pipe<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, psmem));
    AFG_CUDA(ctx, cudaFuncSetAttribute(k_tiny_pipe<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, psmem));
    AFG_CUDA(ctx, cudaFuncSetAttribute(k_tiny_pipe<8, TP_MT_FIXED, 12, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, psmem));
    AFG_CUDA(ctx, cudaFuncSetAttribute(k_tiny_pipe<8, TP_MT_FIXED, 12, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, psmem));
    AFG_CUDA(ctx, cudaFuncSetAttribute(k_tiny_pipe<8, TP_MT_FIXED, 8, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, psmem));
    AFG_CUDA(ctx, cudaFuncSetAttribute(k_tiny_pipe<8, TP_MT_FIXED, 8, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, psmem));
    if (ctx->cfg.win_len % (128 * TF_CLUSTER) == 0) {  // list mode on clusters: a quarter window per CTA
        const int smem_c = (int)tiny_smem(ctx->cfg.win_len / TF_CLUSTER, n_conv, k).total + TF_XCH;
        AFG_CUDA(ctx, cudaFuncSetAttribute(k_tiny_fused<1, TF_CLUSTER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           smem_c));
        AFG_CUDA(ctx, cudaFuncSetAttribute(k_tiny_fused<2, TF_CLUSTER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           smem_c));
        AFG_CUDA(ctx, cudaFuncSetAttribute(k_tiny_fused<4, TF_CLUSTER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           smem_c));
        AFG_CUDA(ctx, cudaFuncSetAttribute(k_tiny_fused<8, TF_CLUSTER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           smem_c));
        AFG_CUDA(ctx, cudaFuncSetAttribute(k_tiny_fused<16, TF_CLUSTER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           smem_c));
    }
    return AFG_OK;
}

int launch_infer_bf16_batch(afg_ctx *ctx, const float *white, int64_t y_stride, const SegDesc *segs_dev, int n_seg,
                            int64_t total_win, int64_t stride, int64_t shift_step, float *logits, cudaStream_t st) {
    const NetPlan &P = ctx->plan;
    if (!tiny_compatible(ctx) || !P.tc_params)
        return afg_fail(ctx, AFG_ERR_UNSUPPORTED, "batch: the BF16 path covers one-stage 16-channel networks");
    const int n_conv = (int)P.convs.size() - 1;
    const int W = ctx->cfg.win_len;
    TinyArgs a;
    memset(&a, 0, sizeof a);
    a.y = white;
    a.n_y = 0;
    a.y_stride = y_stride;
    a.first = 0;
    a.stride = stride;
    a.shift = 0;
    a.n_win = total_win;
    a.segs = segs_dev;
    a.n_seg = n_seg;
    a.wins = nullptr;
    a.shift_step = shift_step;
    a.params = P.tc_params;
    a.wimg = P.tc_wimg;
    a.logits = logits;
    a.err = ctx->d_err;
    a.n_conv = n_conv;
    a.k_stem = P.net.stem_k;
    a.W = W;
    a.G = P.net.groups;
    a.eps = P.net.eps;
    const PipeSmem L = pipe_smem(W, n_conv, a.k_stem);
    a.seg_cache = n_seg <= pipe_seg_cache_cap(L.total) ? n_seg : 0;
    const size_t smem = L.total + (size_t)a.seg_cache * sizeof(SegDesc);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const unsigned grid = (unsigned)std::min<int64_t>(total_win, std::max(sms, 1));
    const double flops = 2.0 * total_win * W * TF_C * ((3.0 * TF_C) * n_conv + 2.0 * a.k_stem);
    KScope ks(ctx, st, KK_TINY_TC, flops, (double)total_win * (2.0 * W * 4.0 + 4.0));
    a.spin_ns = P.tiny_spin_ns;
    cudaError_t e = launch_pipe(a, grid, smem, st, false, P.tiny_ew, P.tiny_mw);
    if (e != cudaSuccess) return afg_cuda_fail(ctx, e, "k_tiny_pipe(batch)");
    return AFG_OK;
}

int launch_infer_bf16_list(afg_ctx *ctx, const WinPtr *wins_dev, int64_t n_win, const IntegDesc *integ,
                           int n_integ, int n_int, unsigned *done, cudaStream_t st) {
    const NetPlan &P = ctx->plan;
    if (!tiny_compatible(ctx) || !P.tc_params)
        return afg_fail(ctx, AFG_ERR_UNSUPPORTED, "streams: the BF16 path covers one-stage 16-channel networks");
    if (n_win <= 0) return AFG_OK;
    const int n_conv = (int)P.convs.size() - 1;
    const int W = ctx->cfg.win_len;
    TinyArgs a;
    memset(&a, 0, sizeof a);
    a.wins = wins_dev;
    a.n_win = n_win;
    if (n_integ > 0) {
        a.integ = integ;
        a.n_integ = n_integ;
        a.n_int = n_int;
        a.done = done;
    }
    a.stride = 1;
    a.params = P.tc_params;
    a.wimg = P.tc_wimg;
    a.err = ctx->d_err;
    a.n_conv = n_conv;
    a.k_stem = P.net.stem_k;
    a.W = W;
    a.G = P.net.groups;
    a.eps = P.net.eps;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const unsigned grid = (unsigned)std::min<int64_t>(n_win, std::max(sms, 1));
    const double flops = 2.0 * n_win * W * TF_C * ((3.0 * TF_C) * n_conv + 2.0 * a.k_stem);
    KScope ks(ctx, st, KK_TINY_TC, flops, (double)n_win * (2.0 * W * 4.0 + 4.0));
    // a programmatic dependent of the whitening launch: set-up overlaps its tail
    cudaError_t e;
    if (W % (128 * TF_CLUSTER) == 0 && n_win * TF_CLUSTER <= sms) {
        // few windows (a latency-bound step): one cluster of TF_CLUSTER CTAs per window
        const size_t smem_c = tiny_smem(W / TF_CLUSTER, n_conv, a.k_stem).total + TF_XCH;
        const dim3 gc((unsigned)(n_win * TF_CLUSTER));
        switch (a.G) {
            case 1: e = launch_pdl_cluster(k_tiny_fused<1, TF_CLUSTER>, gc, dim3(TF_THREADS), smem_c, st, TF_CLUSTER, a); break;
            case 2: e = launch_pdl_cluster(k_tiny_fused<2, TF_CLUSTER>, gc, dim3(TF_THREADS), smem_c, st, TF_CLUSTER, a); break;
            case 4: e = launch_pdl_cluster(k_tiny_fused<4, TF_CLUSTER>, gc, dim3(TF_THREADS), smem_c, st, TF_CLUSTER, a); break;
            case 8: e = launch_pdl_cluster(k_tiny_fused<8, TF_CLUSTER>, gc, dim3(TF_THREADS), smem_c, st, TF_CLUSTER, a); break;
            default: e = launch_pdl_cluster(k_tiny_fused<16, TF_CLUSTER>, gc, dim3(TF_THREADS), smem_c, st, TF_CLUSTER, a); break;
        }
        AFG_CUDA(ctx, e);
        return AFG_OK;
    }
    const size_t psmem = pipe_smem(W, n_conv, a.k_stem).total;
    a.spin_ns = P.tiny_spin_ns;
    AFG_CUDA(ctx, launch_pipe(a, grid, psmem, st, true, P.tiny_ew, P.tiny_mw));
    return AFG_OK;
}

int launch_infer_bf16(afg_ctx *ctx, const float *y, int64_t n_y, int64_t y_stride, int64_t first, int64_t stride,
                      int64_t n_win, int64_t shift, float *logits, cudaStream_t st) {
    const NetPlan &P = ctx->plan;
    if (!tiny_compatible(ctx) || !P.tc_params) {
        if (net_tc_layers_available(ctx))
            return launch_infer_bf16_full(ctx, y, n_y, y_stride, first, stride, n_win, shift, logits, st);
        return afg_fail(ctx, AFG_ERR_UNSUPPORTED,
                        "infer_windows: no BF16 tensor-core path for this network (widths 16 fused, or 64..512)");
    }
    const int n_conv = (int)P.convs.size() - 1;
    const int W = ctx->cfg.win_len;
    TinyArgs a;
    memset(&a, 0, sizeof a);
    a.segs = nullptr;
    a.n_seg = 0;
    a.wins = nullptr;
    a.shift_step = 0;
    a.y = y;
    a.n_y = n_y;
    a.y_stride = y_stride;
    a.first = first;
    a.stride = stride;
    a.shift = shift;
    a.n_win = n_win;
    a.params = P.tc_params;
    a.wimg = P.tc_wimg;
    a.logits = logits;
    a.err = ctx->d_err;
    a.n_conv = n_conv;
    a.k_stem = P.net.stem_k;
    a.W = W;
    a.G = P.net.groups;
    a.eps = P.net.eps;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const unsigned grid = (unsigned)std::min<int64_t>(n_win, std::max(sms, 1));
    const double flops_conv = 2.0 * n_win * W * TF_C * (3.0 * TF_C) * n_conv;
    const double flops_stem = 2.0 * n_win * W * TF_C * 2.0 * a.k_stem;
    KScope ks(ctx, st, KK_TINY_TC, flops_conv + flops_stem, (double)n_win * (2.0 * W * 4.0 + 4.0));
    const size_t psmem = pipe_smem(W, n_conv, a.k_stem).total;
    a.spin_ns = P.tiny_spin_ns;
    cudaError_t e = launch_pipe(a, grid, psmem, st, false, P.tiny_ew, P.tiny_mw);
    if (e != cudaSuccess) return afg_cuda_fail(ctx, e, "k_tiny_pipe");
    return AFG_OK;
}

namespace {

__global__ void k_fill_f32(float *x, int64_t n, uint32_t seed) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 0x9E3779B1u ^ seed;
        h ^= h >> 16;
        h *= 0x85EBCA6Bu;
        h ^= h >> 13;
        x[i] = (float)(h >> 8) * (4.0f / 16777216.0f) - 2.0f;
    }
}

void tiny_tuning_record(const NetPlan &P, afg_fused_tuning &t) {
    memset(&t, 0, sizeof t);
    t.epi_warps = P.tiny_ew;
    t.issue_warps = P.tiny_mw;
    t.spin_ns = (int32_t)P.tiny_spin_ns;
    t.tuned = P.tiny_tuned;
    t.n_candidates = P.tiny_n_cand;
    t.us_chosen = P.tiny_us_chosen;
    t.us_default = P.tiny_us_default;
}

}  // namespace

// The fused 16-channel network's knobs are tuned where its fixed geometry is compiled (BF16 context,
// 8 GroupNorm groups, 3072-position windows).
bool net_tc_tiny_tunable(const afg_ctx *ctx) {
    return ctx->cfg.precision == AFG_BF16 && tiny_compatible(ctx) && ctx->plan.tc_params &&
           ctx->plan.net.groups == 8 && ctx->cfg.win_len == 128 * TP_MT_FIXED;
}

// Time every candidate of kPipeVariants on nw windows (stride 64) of synthetic whitened strain and keep the fastest.
int net_tc_tiny_autotune(afg_ctx *ctx, int64_t n_win, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    AFG_CUDA(ctx, cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return afg_fail(ctx, AFG_ERR_STATE, "autotune: stream is capturing");
    NetPlan &P = ctx->plan;
    const int64_t nw = std::max<int64_t>(1, std::min<int64_t>(n_win > 0 ? n_win : 4096, 65536));
    const int64_t stride = 64, n_y = (nw - 1) * stride + ctx->cfg.win_len;
    float *y = nullptr, *z = nullptr;
    int rc = afg_ws_reserve(ctx, WS_WHITE, (size_t)2 * n_y * sizeof(float), (void **)&y);
    if (!rc) rc = afg_ws_reserve(ctx, WS_LOGITS, (size_t)nw * sizeof(float), (void **)&z);
    if (rc) return rc;
    k_fill_f32<<<1024, 256, 0, st>>>(y, 2 * n_y, 0x2468ACEu);
    AFG_LAUNCH_CHECK(ctx, "k_fill_f32");
    cudaEvent_t e0, e1;
    AFG_CUDA(ctx, cudaEventCreate(&e0));
    AFG_CUDA(ctx, cudaEventCreate(&e1));
    const int saved_ew = P.tiny_ew, saved_mw = P.tiny_mw;
    const uint32_t saved_spin = P.tiny_spin_ns;
    const int reps = 3;
    float best = 0.f, t_dflt = 0.f;
    int best_i = 0, err = AFG_OK;
    for (int i = 0; i < kNPipeVariants && !err; ++i) {
        P.tiny_ew = kPipeVariants[i].ew;
        P.tiny_mw = kPipeVariants[i].mw;
        P.tiny_spin_ns = kPipeVariants[i].spin_ns;
        err = launch_infer_bf16(ctx, y, n_y, n_y, 0, stride, nw, 0, z, st);  // warm
        if (err) break;
        if (cudaEventRecord(e0, st) != cudaSuccess) err = afg_cuda_fail(ctx, cudaGetLastError(), "autotune: event");
        for (int r = 0; r < reps && !err; ++r) err = launch_infer_bf16(ctx, y, n_y, n_y, 0, stride, nw, 0, z, st);
        if (err) break;
        float ms = 0.f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            err = afg_cuda_fail(ctx, cudaGetLastError(), "autotune: event timing");
            break;
        }
        const float us = ms * 1000.f / reps;
        if (i == 0) t_dflt = us;
        if (best == 0.f || us < best) {
            best = us;
            best_i = i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err) {
        P.tiny_ew = saved_ew;
        P.tiny_mw = saved_mw;
        P.tiny_spin_ns = saved_spin;
        return err;
    }
    P.tiny_ew = kPipeVariants[best_i].ew;
    P.tiny_mw = kPipeVariants[best_i].mw;
    P.tiny_spin_ns = kPipeVariants[best_i].spin_ns;
    P.tiny_tuned = 1;
    P.tiny_n_cand = kNPipeVariants;
    P.tiny_us_chosen = best;
    P.tiny_us_default = t_dflt;
    AFG_CUDA(ctx, cudaStreamSynchronize(st));
    int flag = 0;
    AFG_CUDA(ctx, cudaMemcpy(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        AFG_CUDA(ctx, cudaMemset(ctx->d_err, 0, sizeof(int)));
        return afg_fail(ctx, AFG_ERR_TIMEOUT, "autotune: a bounded device-side wait gave up");
    }
    return AFG_OK;
}

int net_tc_tiny_tuning_get(afg_ctx *ctx, afg_fused_tuning *out) {
    if (ctx->cfg.precision != AFG_BF16 || !tiny_compatible(ctx) || !ctx->plan.tc_params)
        return afg_fail(ctx, AFG_ERR_UNSUPPORTED, "fused tuning: the context has no fused 16-channel BF16 network");
    tiny_tuning_record(ctx->plan, *out);
    return AFG_OK;
}

int net_tc_tiny_tuning_candidates(afg_ctx *ctx, afg_fused_tuning *out, int cap, int *n_out) {
    if (!net_tc_tiny_tunable(ctx))
        return afg_fail(ctx, AFG_ERR_UNSUPPORTED, "fused tuning: no tunable fused network (BF16, 8 groups, 3072 positions)");
    *n_out = kNPipeVariants;
    for (int i = 0; i < kNPipeVariants && i < cap; ++i) {
        memset(&out[i], 0, sizeof out[i]);
        out[i].epi_warps = kPipeVariants[i].ew;
        out[i].issue_warps = kPipeVariants[i].mw;
        out[i].spin_ns = (int32_t)kPipeVariants[i].spin_ns;
    }
    return AFG_OK;
}

int net_tc_tiny_tuning_set(afg_ctx *ctx, const afg_fused_tuning *in) {
    if (!net_tc_tiny_tunable(ctx))
        return afg_fail(ctx, AFG_ERR_UNSUPPORTED, "fused tuning: no tunable fused network (BF16, 8 groups, 3072 positions)");
    if ((in->epi_warps != 8 && in->epi_warps != 12) || (in->issue_warps != 1 && in->issue_warps != 2) ||
        in->spin_ns < 0 || in->spin_ns > 100000)
        return afg_fail(ctx, AFG_ERR_ARG, "fused tuning: epi_warps 8 or 12, issue_warps 1 or 2, spin_ns in [0, 1e5]");
    NetPlan &P = ctx->plan;
    P.tiny_ew = in->epi_warps;
    P.tiny_mw = in->issue_warps;
    P.tiny_spin_ns = (uint32_t)in->spin_ns;
    P.tiny_tuned = in->tuned ? 1 : 0;
    P.tiny_us_chosen = in->us_chosen;
    P.tiny_us_default = in->us_default;
    P.tiny_n_cand = in->n_candidates;
    return AFG_OK;
}
