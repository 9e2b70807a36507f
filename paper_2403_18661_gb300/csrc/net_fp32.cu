// 1D ResNet with GroupNorm over sliding windows, FP32 SIMT path
// (Sec. II: ResNet34 with 1D convolutions and GroupNorm, scalar output;
// Sec. IX: kernel length 3 and global pooling).
//
// Activation layout: per window, channels-last with one zero row before and
// after the data ([L + 2][C]), windows packed back to back.  With this layout
// the K = k*Cin operand row of output position t (taps r = 0..k-1, channels
// ci) is the contiguous run of k*Cin floats starting at padded row
// t*stride + (1 - pad), so every convolution is a GEMM whose A operand is a
// strided view of the activation buffer (implicit GEMM, no im2col copy).
//
// Per conv: k_conv_fp32 (tiled SIMT GEMM) writes the raw output; then
// k_groupnorm computes the group statistics of each window (two passes,
// one warp per group), and applies the affine map, the optional residual and
// ReLU in place (or max-pools into another buffer for the stem).
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "afg_internal.cuh"

namespace {

inline int conv_len(int L, int k, int s, int p) { return (L + 2 * p - k) / s + 1; }

// ---------------------------------------------------------------- stem
// grid (n_win); reads the window straight from the whitened stream.
// out: [n_win][L0 + 2][C0], raw conv output (GroupNorm follows).
__global__ void k_stem(const float *__restrict__ y, int64_t n_y, int64_t y_stride, int64_t first, int64_t stride,
                       int64_t shift, int64_t w0, const float *__restrict__ w, int C0, int k, int s, int W, int L0,
                       float *__restrict__ out) {
    extern __shared__ float xs[];  // [2][W + 2*pad]
    const int pad = k / 2;
    const int Wp = W + 2 * pad;
    const int64_t win = w0 + blockIdx.x;
    const int64_t start = first + win * stride;
    const float *y0 = y, *y1 = y + y_stride;
    for (int t = threadIdx.x; t < Wp; t += blockDim.x) {
        int tt = t - pad;
        float a = 0.f, b = 0.f;
        if (tt >= 0 && tt < W) {
            a = y0[start + tt];
            int64_t i1 = start + shift + tt;
            if (i1 >= n_y) i1 -= n_y;
            b = y1[i1];
        }
        xs[t] = a;
        xs[Wp + t] = b;
    }
    __syncthreads();
    float *o = out + (int64_t)blockIdx.x * (L0 + 2) * C0;
    for (int idx = threadIdx.x; idx < (L0 + 2) * C0; idx += blockDim.x) {
        int row = idx / C0, co = idx - row * C0;
        float acc = 0.f;
        if (row >= 1 && row <= L0) {
            int t = row - 1;
            const float *wc = w + co * 2 * k;
            for (int ci = 0; ci < 2; ++ci)
                for (int r = 0; r < k; ++r) acc = fmaf(wc[ci * k + r], xs[ci * Wp + t * s + r], acc);
        }
        o[idx] = acc;
    }
}

// ---------------------------------------------------------------- GroupNorm
// grid (n_win), block GN_T.  x: [n_win][L+2][C] padded, normalised in place;
// res (optional) same layout, added before ReLU; if pool_out is given, the
// result is max-pooled (k3, s2, p1) into pool_out [n_win][L/2 + 2][C]
// instead (x left untouched).  Pad rows of the written tile are set to zero.
// Thread t reads float4 chunks t, t + GN_T, ... of the tile; since C/4
// divides GN_T, its 4 channels are fixed.  Per-channel partial sums are
// reduced in a fixed order (two passes: mean, then centred variance).
constexpr int GN_T = 256;

__device__ __forceinline__ void gn_channel_reduce(float (&a)[4], float *red, float *chs, int C) {
    // red: [GN_T][4] partials; chs: [C] per-channel totals
    const int tid = threadIdx.x;
    for (int e = 0; e < 4; ++e) red[tid * 4 + e] = a[e];
    __syncthreads();
    const int q = C / 4;  // channel quads
    for (int c = tid; c < C; c += GN_T) {
        const int quad = c / 4, e = c % 4;
        float s = 0.f;
        for (int t = quad; t < GN_T; t += q) s += red[t * 4 + e];
        chs[c] = s;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(GN_T) k_groupnorm(float *__restrict__ x, int L, int C, int G,
                                                    const float *__restrict__ gamma, const float *__restrict__ beta,
                                                    float eps, const float *__restrict__ res, int relu,
                                                    float *__restrict__ pool_out) {
    __shared__ float red[GN_T * 4];
    __shared__ float chs[512];
    __shared__ float gmean[32], grstd[32];
    const int tid = threadIdx.x;
    const int cg = C / G;
    const int64_t tile = (int64_t)(L + 2) * C;
    float *xt = x + (int64_t)blockIdx.x * tile + C;  // row 0 of data
    const int n4 = L * C / 4;
    const int c0 = (tid % (C / 4)) * 4;  // first channel of this thread's float4s
    const float4 *x4 = reinterpret_cast<const float4 *>(xt);
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    for (int i = tid; i < n4; i += GN_T) {
        const float4 v = x4[i];
        a[0] += v.x; a[1] += v.y; a[2] += v.z; a[3] += v.w;
    }
    gn_channel_reduce(a, red, chs, C);
    if (tid < G) {
        float s = 0.f;
        for (int c = tid * cg; c < (tid + 1) * cg; ++c) s += chs[c];
        gmean[tid] = s / (float)(L * cg);
    }
    __syncthreads();
    float mu[4];
    for (int e = 0; e < 4; ++e) mu[e] = gmean[(c0 + e) / cg];
    for (int e = 0; e < 4; ++e) a[e] = 0.f;
    for (int i = tid; i < n4; i += GN_T) {
        const float4 v = x4[i];
        float d;
        d = v.x - mu[0]; a[0] = fmaf(d, d, a[0]);
        d = v.y - mu[1]; a[1] = fmaf(d, d, a[1]);
        d = v.z - mu[2]; a[2] = fmaf(d, d, a[2]);
        d = v.w - mu[3]; a[3] = fmaf(d, d, a[3]);
    }
    gn_channel_reduce(a, red, chs, C);
    if (tid < G) {
        float s = 0.f;
        for (int c = tid * cg; c < (tid + 1) * cg; ++c) s += chs[c];
        grstd[tid] = rsqrtf(s / (float)(L * cg) + eps);
    }
    __syncthreads();
    float sc[4], sh[4];
    for (int e = 0; e < 4; ++e) {
        const int c = c0 + e, g = c / cg;
        sc[e] = grstd[g] * gamma[c];
        sh[e] = beta[c] - gmean[g] * sc[e];
    }
    if (pool_out == nullptr) {
        const float4 *r4 = res ? reinterpret_cast<const float4 *>(res + (int64_t)blockIdx.x * tile + C) : nullptr;
        float4 *w4 = reinterpret_cast<float4 *>(xt);
        for (int i = tid; i < n4; i += GN_T) {
            float4 v = x4[i];
            float o[4] = {fmaf(v.x, sc[0], sh[0]), fmaf(v.y, sc[1], sh[1]), fmaf(v.z, sc[2], sh[2]),
                          fmaf(v.w, sc[3], sh[3])};
            if (r4) {
                const float4 r = r4[i];
                o[0] += r.x; o[1] += r.y; o[2] += r.z; o[3] += r.w;
            }
            if (relu)
                for (int e = 0; e < 4; ++e) o[e] = fmaxf(o[e], 0.f);
            w4[i] = make_float4(o[0], o[1], o[2], o[3]);
        }
        for (int c = tid; c < C; c += GN_T) {
            xt[-C + c] = 0.f;
            xt[(int64_t)L * C + c] = 0.f;
        }
    } else {
        const int Lp = (L + 2 - 3) / 2 + 1;
        float *po = pool_out + (int64_t)blockIdx.x * (Lp + 2) * C + C;
        float4 *p4 = reinterpret_cast<float4 *>(po);
        const int C4 = C / 4;
        for (int i = tid; i < Lp * C4; i += GN_T) {
            const int row = i / C4, q = i - row * C4;
            float m[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
            for (int r = -1; r <= 1; ++r) {
                const int src = 2 * row + r;
                if (src < 0 || src >= L) continue;
                const float4 v = x4[(int64_t)src * C4 + q];
                float o[4] = {fmaf(v.x, sc[0], sh[0]), fmaf(v.y, sc[1], sh[1]), fmaf(v.z, sc[2], sh[2]),
                              fmaf(v.w, sc[3], sh[3])};
                for (int e = 0; e < 4; ++e) {
                    if (relu) o[e] = fmaxf(o[e], 0.f);
                    m[e] = fmaxf(m[e], o[e]);
                }
            }
            p4[i] = make_float4(m[0], m[1], m[2], m[3]);
        }
        for (int c = tid; c < C; c += GN_T) {
            po[-C + c] = 0.f;
            po[(int64_t)Lp * C + c] = 0.f;
        }
    }
}

// GroupNorm with the window's tile staged in shared memory (every tile of the 16-channel and
// ResNet34-GN networks has L * C = 49,152 floats, 192 KB): thread t copies float4 chunks t, t + GN_ST,
// ... of the window with cp.async (all copies in flight together, no registers held), and after its
// own copies have landed reads only those chunks back, so the tile is read from HBM once.  The mean
// and the centred variance come from shared memory (the same two-pass definition, partial sums
// reduced in a fixed order), and the normalised tile (+ residual, ReLU) is written once.  C/4
// divides GN_ST, so a thread's 4 channels are fixed.
constexpr int GN_ST = 512;
constexpr int GN_ST_MAX4 = 12288;  // float4 chunks of the largest staged tile (192 KB)

__device__ __forceinline__ void gn_channel_reduce_st(float (&a)[4], float *red, float *chs, int C) {
    const int tid = threadIdx.x;
    for (int e = 0; e < 4; ++e) red[tid * 4 + e] = a[e];
    __syncthreads();
    const int q = C / 4;
    for (int c = tid; c < C; c += GN_ST) {
        const int quad = c / 4, e = c % 4;
        float s = 0.f;
        for (int t = quad; t < GN_ST; t += q) s += red[t * 4 + e];
        chs[c] = s;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(GN_ST, 1) k_groupnorm_st(float *__restrict__ x, int L, int C, int G,
                                                          const float *__restrict__ gamma,
                                                          const float *__restrict__ beta, float eps,
                                                          const float *__restrict__ res, int relu) {
    extern __shared__ __align__(16) float4 gn_tile[];  // [L * C / 4]
    __shared__ float red[GN_ST * 4];
    __shared__ float chs[512];
    __shared__ float gmean[32], grstd[32];
    const int tid = threadIdx.x;
    const int cg = C / G;
    const int n4 = L * C / 4;
    const int64_t tile = (int64_t)(L + 2) * C;
    float *xt = x + (int64_t)blockIdx.x * tile + C;  // row 0 of data
    const int c0 = (tid % (C / 4)) * 4;
    const float4 *x4 = reinterpret_cast<const float4 *>(xt);
    for (int i = tid; i < n4; i += GN_ST)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(gn_tile + i)),
                     "l"(x4 + i)
                     : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_all;" ::: "memory");
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    for (int i = tid; i < n4; i += GN_ST) {
        const float4 v = gn_tile[i];
        a[0] += v.x; a[1] += v.y; a[2] += v.z; a[3] += v.w;
    }
    gn_channel_reduce_st(a, red, chs, C);
    if (tid < G) {
        float s = 0.f;
        for (int c = tid * cg; c < (tid + 1) * cg; ++c) s += chs[c];
        gmean[tid] = s / (float)(L * cg);
    }
    __syncthreads();
    float mu[4];
    for (int e = 0; e < 4; ++e) mu[e] = gmean[(c0 + e) / cg];
    for (int e = 0; e < 4; ++e) a[e] = 0.f;
    for (int i = tid; i < n4; i += GN_ST) {
        const float4 v = gn_tile[i];
        float d;
        d = v.x - mu[0]; a[0] = fmaf(d, d, a[0]);
        d = v.y - mu[1]; a[1] = fmaf(d, d, a[1]);
        d = v.z - mu[2]; a[2] = fmaf(d, d, a[2]);
        d = v.w - mu[3]; a[3] = fmaf(d, d, a[3]);
    }
    gn_channel_reduce_st(a, red, chs, C);
    if (tid < G) {
        float s = 0.f;
        for (int c = tid * cg; c < (tid + 1) * cg; ++c) s += chs[c];
        grstd[tid] = rsqrtf(s / (float)(L * cg) + eps);
    }
    __syncthreads();
    float sc[4], sh[4];
    for (int e = 0; e < 4; ++e) {
        const int c = c0 + e, g = c / cg;
        sc[e] = grstd[g] * gamma[c];
        sh[e] = beta[c] - gmean[g] * sc[e];
    }
    const float4 *r4 = res ? reinterpret_cast<const float4 *>(res + (int64_t)blockIdx.x * tile + C) : nullptr;
    float4 *w4 = reinterpret_cast<float4 *>(xt);
    constexpr int RB = 8;  // residual loads in flight per thread
    for (int i0 = tid; i0 < n4; i0 += RB * GN_ST) {
        float4 r[RB];
#pragma unroll
        for (int k = 0; k < RB; ++k) {
            const int i = i0 + k * GN_ST;
            r[k] = (r4 && i < n4) ? r4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < RB; ++k) {
            const int i = i0 + k * GN_ST;
            if (i >= n4) break;
            const float4 u = gn_tile[i];
            float o[4] = {fmaf(u.x, sc[0], sh[0]) + r[k].x, fmaf(u.y, sc[1], sh[1]) + r[k].y,
                          fmaf(u.z, sc[2], sh[2]) + r[k].z, fmaf(u.w, sc[3], sh[3]) + r[k].w};
            if (relu)
                for (int e = 0; e < 4; ++e) o[e] = fmaxf(o[e], 0.f);
            w4[i] = make_float4(o[0], o[1], o[2], o[3]);
        }
    }
    for (int c = tid; c < C; c += GN_ST) {
        xt[-C + c] = 0.f;
        xt[(int64_t)L * C + c] = 0.f;
    }
}

// ---------------------------------------------------------------- conv GEMM
// out[w][t+1][n] = sum_kk A[w,t][kk] * Wt[kk][n],  A[w,t][kk] = in[w][t*s + off][kk]
// (kk runs over k*Cin contiguous floats).  M = n_win * Lout rows.
// Tiles of BM x BN per CTA (256 threads, TM x TN outputs each), K in steps of BK,
// double-buffered in shared memory with one barrier per step: the next step's A
// and B tiles are copied by cp.async while the current step is multiplied (A into
// a staging area; after the copies land, each thread rewrites the A values it
// copied itself into the layout below, so no extra barrier is needed).
//
// The products are packed FP32x2 FMAs (fma.rn.f32x2: two independent FMAs, each
// rounded once like fmaf), so every output is accumulated in exactly the order
// k = 0 .. K-1 with one rounding per step.  Each pair is (a_m, a_m) x (b_n, b_n+1),
// the (a, a) pair built in registers from the transposed A tile.
// A thread's TM rows and TN columns are runs of 4 spaced BM / (TM/4) and BN / (TN/4)
// apart, so the 16-byte B loads of a warp touch consecutive addresses.
template <int BM, int BN, int BK>
struct ConvSmem {
    static constexpr int A_LD = BM + 4;  // +4 floats spreads the transposed stores over the banks
    static constexpr size_t bytes = sizeof(float) * (2 * BK * (A_LD + BN) + BM * BK);
};

template <int BM, int BN, int TM, int TN, int BK>
__global__ void __launch_bounds__(256, 2) k_conv_fp32(const float *__restrict__ in, const float *__restrict__ wt,
                                                   float *__restrict__ out, int M, int Lout, int Lp_in, int Lp_out,
                                                   int Cin, int Cout, int K, int s, int off) {
    constexpr int TX = BN / TN, TY = BM / TM;
    static_assert(TX * TY == 256 && TM % 4 == 0 && TN % 4 == 0, "tile shape");
    constexpr int A_LD = ConvSmem<BM, BN, BK>::A_LD;
    constexpr int A_F4 = BM * BK / 4;  // float4 loads per A tile
    constexpr int B_F4 = BK * BN / 4;  // 16-byte copies per B tile
    constexpr int A_PER = (A_F4 + 255) / 256;
    constexpr int B_PER = (B_F4 + 255) / 256;
    extern __shared__ __align__(16) float conv_smem[];
    float *As = conv_smem;                     // [2][BK][A_LD]
    float *Bs = conv_smem + 2 * BK * A_LD;     // [2][BK][BN]
    float *Ast = Bs + 2 * BK * BN;             // [BM][BK] staging of the next A tile
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;

    const float *arow[A_PER];
#pragma unroll
    for (int i = 0; i < A_PER; ++i) {
        const int f = tid + i * 256;
        const int m = m0 + f / (BK / 4);
        if (f < A_F4 && m < M) {
            const int w = m / Lout, t = m - w * Lout;
            arow[i] = in + ((int64_t)w * Lp_in + (int64_t)t * s + off) * Cin + (f % (BK / 4)) * 4;
        } else {
            arow[i] = nullptr;
        }
    }
    auto copy_tiles = [&](int k0, int buf) {
#pragma unroll
        for (int i = 0; i < A_PER; ++i) {
            const int f = tid + i * 256;
            if (f < A_F4) {  // rows past M are zero-filled (source size 0)
                const uint32_t dst = (uint32_t)__cvta_generic_to_shared(Ast + f * 4);
                const float *src = arow[i] ? arow[i] + k0 : in;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                             "r"(arow[i] ? 16 : 0)
                             : "memory");
            }
        }
#pragma unroll
        for (int i = 0; i < B_PER; ++i) {
            const int f = tid + i * 256;
            if (f < B_F4) {
                const int r = f / (BN / 4), c = (f % (BN / 4)) * 4;
                const uint32_t dst = (uint32_t)__cvta_generic_to_shared(Bs + (buf * BK + r) * BN + c);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst),
                             "l"(wt + (int64_t)(k0 + r) * Cout + n0 + c)
                             : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // after cp.async.wait_all: the thread's own staged A values -> the transposed A tile
    auto store_a = [&](int buf) {
#pragma unroll
        for (int i = 0; i < A_PER; ++i) {
            const int f = tid + i * 256;
            if (f < A_F4) {
                const float4 v = *reinterpret_cast<const float4 *>(Ast + f * 4);
                float *d = As + (buf * BK + (f % (BK / 4)) * 4) * A_LD + (f / (BK / 4));
                d[0] = v.x;
                d[A_LD] = v.y;
                d[2 * A_LD] = v.z;
                d[3 * A_LD] = v.w;
            }
        }
    };
    float2 acc[TM][TN / 2];  // acc[i][j] = columns (2j, 2j+1) of the thread's row i
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN / 2; ++j) acc[i][j] = make_float2(0.f, 0.f);

    copy_tiles(0, 0);
    asm volatile("cp.async.wait_all;" ::: "memory");
    store_a(0);
    __syncthreads();
    int cur = 0;
    for (int k0 = 0; k0 < K; k0 += BK) {
        const bool more = k0 + BK < K;
        if (more) copy_tiles(k0 + BK, cur ^ 1);  // copies in flight during the math below
        const float *Ac = As + cur * BK * A_LD;
        const float *Bc = Bs + cur * BK * BN;
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float4 ap[TM / 4];
            float4 bq[TN / 4];
#pragma unroll
            for (int h = 0; h < TM / 4; ++h) {
                ap[h] = *reinterpret_cast<const float4 *>(Ac + kk * A_LD + h * TY * 4 + ty * 4);
            }
#pragma unroll
            for (int h = 0; h < TN / 4; ++h)
                bq[h] = *reinterpret_cast<const float4 *>(Bc + kk * BN + h * TX * 4 + tx * 4);
#pragma unroll
            for (int i = 0; i < TM; ++i) {
                const float4 &a4 = ap[i / 4];
                const float av = (i % 4 == 0) ? a4.x : (i % 4 == 1) ? a4.y : (i % 4 == 2) ? a4.z : a4.w;
                const float2 a2 = make_float2(av, av);
#pragma unroll
                for (int j = 0; j < TN / 2; ++j) {
                    const float2 b2 = (j & 1) ? make_float2(bq[j / 2].z, bq[j / 2].w)
                                              : make_float2(bq[j / 2].x, bq[j / 2].y);
                    acc[i][j] = __ffma2_rn(a2, b2, acc[i][j]);
                }
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (more) store_a(cur ^ 1);
        __syncthreads();
        cur ^= 1;
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int m = m0 + (i / 4) * TY * 4 + ty * 4 + (i % 4);
        if (m >= M) continue;
        const int w = m / Lout, t = m - w * Lout;
        float *o = out + ((int64_t)w * Lp_out + t + 1) * Cout + n0 + tx * 4;
#pragma unroll
        for (int h = 0; h < TN / 4; ++h)
            *reinterpret_cast<float4 *>(o + h * TX * 4) =
                make_float4(acc[i][2 * h].x, acc[i][2 * h].y, acc[i][2 * h + 1].x, acc[i][2 * h + 1].y);
    }
}

// ---------------------------------------------------------------- head
// grid (n_win), block 256: logit = fc_b + sum_c fc_w[c] * mean_t x[t][c]
__global__ void k_head(const float *__restrict__ x, int L, int C, const float *__restrict__ fc_w,
                       const float *__restrict__ fc_b, float *__restrict__ logits, int64_t w0) {
    __shared__ float part[512];
    const float *xt = x + (int64_t)blockIdx.x * (L + 2) * C + C;
    const int tid = threadIdx.x;
    if (C <= 256) {
        const int phases = 256 / C;
        const int c = tid % C, p = tid / C;
        float s = 0.f;
        for (int r = p; r < L; r += phases) s += xt[(int64_t)r * C + c];
        part[tid] = s;
        __syncthreads();
        if (tid < C) {
            float tot = 0.f;
            for (int q = 0; q < phases; ++q) tot += part[q * C + tid];
            part[256 + tid] = fc_w[tid] * (tot / (float)L);
        }
    } else {
        for (int c = tid; c < C; c += 256) {
            float s = 0.f;
            for (int r = 0; r < L; ++r) s += xt[(int64_t)r * C + c];
            part[c] = fc_w[c] * (s / (float)L);
        }
    }
    __syncthreads();
    if (tid == 0) {
        const float *v = C <= 256 ? part + 256 : part;
        float z = fc_b[0];
        for (int c = 0; c < C; ++c) z += v[c];
        logits[w0 + blockIdx.x] = z;
    }
}

template <int BM, int BN, int TM, int TN, int BK>
void conv_launch(afg_ctx *ctx, const float *in, const float *wt, float *out, int nw, const ConvLayer &L,
                 cudaStream_t st) {
    const int M = nw * L.lout;
    const int K = L.k * L.cin;
    const int off = 1 - L.pad;
    dim3 grid((M + BM - 1) / BM, L.cout / BN);
    // algorithmic: 2 M N K FLOPs; one read of the input activations and weights, one write of the output
    KScope ks(ctx, st, KK_CONV_FP32, 2.0 * M * L.cout * K,
              4.0 * ((double)nw * L.lin * L.cin + (double)K * L.cout + (double)M * L.cout));
    constexpr size_t smem = ConvSmem<BM, BN, BK>::bytes;
    static bool attr_set = false;  // per instantiation; one device per process
    if (!attr_set) {
        cudaFuncSetAttribute(k_conv_fp32<BM, BN, TM, TN, BK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set = true;
    }
    k_conv_fp32<BM, BN, TM, TN, BK><<<grid, 256, smem, st>>>(in, wt, out, M, L.lout, L.lin + 2, L.lout + 2, L.cin,
                                                             L.cout, K, L.stride, off);
}

// K = k * Cin is a multiple of 16 for every convolution of the networks (Cin >= 16)
void conv_dispatch(afg_ctx *ctx, const float *in, float *out, int nw, const ConvLayer &L, cudaStream_t st) {
    if (L.cout % 128 == 0) conv_launch<128, 128, 8, 8, 16>(ctx, in, L.wt, out, nw, L, st);
    else if (L.cout % 64 == 0) conv_launch<256, 64, 8, 8, 16>(ctx, in, L.wt, out, nw, L, st);  // 8 x 8 per thread too
    else conv_launch<256, 16, 4, 4, 16>(ctx, in, L.wt, out, nw, L, st);
}

// GroupNorm launch with its accounting: one read (+ residual read) and one write of the tile
void gn_launch(afg_ctx *ctx, float *x, int nw, int L, int C, int G, const float *gamma, const float *beta, float eps,
               const float *res, int relu, float *pool_out, cudaStream_t st) {
    double tile = (double)nw * L * C * 4.0;
    double bytes = tile * (res ? 3.0 : 2.0);
    if (pool_out) bytes = tile * 1.5;
    KScope ks(ctx, st, KK_GROUPNORM, 0.0, bytes);
    const int64_t n4 = (int64_t)L * C / 4;
    if (!pool_out && C % 4 == 0 && C <= 512 && GN_ST % (C / 4) == 0 && n4 >= GN_ST && n4 <= GN_ST_MAX4) {
        static bool attr_set = false;  // one device per process
        if (!attr_set) {
            cudaFuncSetAttribute(k_groupnorm_st, cudaFuncAttributeMaxDynamicSharedMemorySize, GN_ST_MAX4 * 16);
            attr_set = true;
        }
        k_groupnorm_st<<<nw, GN_ST, (size_t)n4 * 16, st>>>(x, L, C, G, gamma, beta, eps, res, relu);
    } else {
        k_groupnorm<<<nw, GN_T, 0, st>>>(x, L, C, G, gamma, beta, eps, res, relu, pool_out);
    }
}

}  // namespace

// ---------------------------------------------------------------- plan
int net_plan_build(afg_ctx *ctx, const float *weights_host, int64_t n_weights) {
    NetPlan &P = ctx->plan;
    const afg_net &n = ctx->cfg.net;
    P.net = n;
    P.convs.clear();
    P.blocks.clear();
    const int W = ctx->cfg.win_len;
    // host-side parameter image: per conv Wt [k*cin][cout], gamma, beta; stem raw [C0][2][k]
    std::vector<float> img;
    const float *src = weights_host;
    auto take = [&](int64_t cnt) { const float *r = src; src += cnt; return r; };
    struct Pending { int64_t wt, gamma, beta; };
    std::vector<Pending> pend;
    auto add_conv = [&](int cin, int cout, int k, int s, int lin) {
        ConvLayer L{};
        L.cin = cin; L.cout = cout; L.k = k; L.stride = s; L.pad = k / 2;
        L.lin = lin; L.lout = conv_len(lin, k, s, k / 2);
        const float *w = take((int64_t)cout * cin * k);
        const float *g = take(cout), *b = take(cout);
        Pending pd;
        pd.wt = (int64_t)img.size();
        img.resize(img.size() + (size_t)cout * cin * k);
        bool stem = P.convs.empty();
        for (int co = 0; co < cout; ++co)
            for (int ci = 0; ci < cin; ++ci)
                for (int r = 0; r < k; ++r) {
                    float v = w[((int64_t)co * cin + ci) * k + r];
                    if (stem) img[pd.wt + ((int64_t)co * cin + ci) * k + r] = v;
                    else img[pd.wt + ((int64_t)r * cin + ci) * cout + co] = v;
                }
        pd.gamma = (int64_t)img.size();
        img.insert(img.end(), g, g + cout);
        pd.beta = (int64_t)img.size();
        img.insert(img.end(), b, b + cout);
        pend.push_back(pd);
        P.convs.push_back(L);
        return (int)P.convs.size() - 1;
    };
    int C0 = n.widths[0];
    add_conv(n.in_ch, C0, n.stem_k, n.stem_stride, W);
    P.l_stem_out = P.convs[0].lout;
    P.l_after_stem = n.stem_pool ? conv_len(P.l_stem_out, 3, 2, 1) : P.l_stem_out;
    int cin = C0, L = P.l_after_stem;
    int64_t maxact = (int64_t)(P.l_stem_out + 2) * C0;
    for (int s = 0; s < n.n_stages; ++s) {
        for (int b = 0; b < n.blocks[s]; ++b) {
            int stride = (s > 0 && b == 0) ? 2 : 1;
            int width = n.widths[s];
            BlockPlan bp;
            bp.c1 = add_conv(cin, width, 3, stride, L);
            int Lo = P.convs[bp.c1].lout;
            bp.c2 = add_conv(width, width, 3, 1, Lo);
            bp.sc = -1;
            if (stride != 1 || cin != width) bp.sc = add_conv(cin, width, 1, stride, L);
            P.blocks.push_back(bp);
            maxact = std::max(maxact, (int64_t)(L + 2) * cin);
            maxact = std::max(maxact, (int64_t)(Lo + 2) * width);
            cin = width;
            L = Lo;
        }
    }
    P.c_last = cin;
    P.l_last = L;
    const float *fw = take(cin), *fb = take(1);
    int64_t fc_off = (int64_t)img.size();
    img.insert(img.end(), fw, fw + cin);
    img.push_back(fb[0]);
    if (src - weights_host != n_weights)
        return afg_fail(ctx, AFG_ERR_ARG, "weights: expected %lld floats, got %lld",
                        (long long)(src - weights_host), (long long)n_weights);
    P.max_act_per_window = maxact;
    // upload
    size_t bytes = img.size() * sizeof(float);
    float *d = nullptr;
    cudaError_t e = cudaMalloc(&d, bytes);
    if (e != cudaSuccess) return afg_fail(ctx, AFG_ERR_OOM, "weights: cudaMalloc(%zu) failed", bytes);
    ctx->d_params = d;
    ctx->d_params_bytes = bytes;
    ctx->bytes_held += (int64_t)bytes;
    AFG_CUDA(ctx, cudaMemcpy(d, img.data(), bytes, cudaMemcpyHostToDevice));
    for (size_t i = 0; i < P.convs.size(); ++i) {
        P.convs[i].wt = d + pend[i].wt;
        P.convs[i].gamma = d + pend[i].gamma;
        P.convs[i].beta = d + pend[i].beta;
        P.convs[i].wt_bf16 = nullptr;
    }
    P.fc_w = d + fc_off;
    P.fc_b = d + fc_off + cin;
    return AFG_OK;
}

// Stem conv (reading the windows from the whitened stream) + GroupNorm + ReLU
// (+ max-pool) for windows [w0, w0 + nw): raw conv output in f0, the result
// in f0 (no pool) or f1 (pool).
int launch_stem_gn_fp32(afg_ctx *ctx, const float *y, int64_t n_y, int64_t y_stride, int64_t first, int64_t stride,
                        int64_t shift, int64_t w0, int nw, float *f0, float *f1, cudaStream_t st) {
    const NetPlan &P = ctx->plan;
    const ConvLayer &S = P.convs[0];
    const int W = ctx->cfg.win_len, G = P.net.groups, pad = S.k / 2;
    {
        KScope ks(ctx, st, KK_STEM, 2.0 * nw * S.lout * S.cout * S.cin * S.k,
                  4.0 * nw * ((double)2 * W + (double)(S.lout + 2) * S.cout));
        k_stem<<<nw, 256, 2 * (W + 2 * pad) * sizeof(float), st>>>(y, n_y, y_stride, first, stride, shift, w0, S.wt,
                                                                  S.cout, S.k, S.stride, W, S.lout, f0);
    }
    AFG_LAUNCH_CHECK(ctx, "k_stem");
    gn_launch(ctx, f0, nw, S.lout, S.cout, G, S.gamma, S.beta, P.net.eps, nullptr, 1, P.net.stem_pool ? f1 : nullptr,
              st);
    AFG_LAUNCH_CHECK(ctx, "k_groupnorm(stem)");
    return AFG_OK;
}

// ---------------------------------------------------------------- forward
int launch_infer_fp32(afg_ctx *ctx, const float *y, int64_t n_y, int64_t y_stride, int64_t first, int64_t stride,
                      int64_t n_win, int64_t shift, float *logits, cudaStream_t st) {
    const NetPlan &P = ctx->plan;
    const int G = P.net.groups;
    const float eps = P.net.eps;
    const int W = ctx->cfg.win_len;
    // windows per chunk: keep each activation buffer under ~4 GiB
    int64_t per_win = P.max_act_per_window * (int64_t)sizeof(float);
    int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(n_win, ((int64_t)4 << 30) / per_win));
    chunk = std::min<int64_t>(chunk, 16384);
    float *buf[4];
    for (int i = 0; i < 4; ++i) {
        int rc = afg_ws_reserve(ctx, WS_ACT0 + i, (size_t)(chunk * per_win), (void **)&buf[i]);
        if (rc) return rc;
    }
    const ConvLayer &S = P.convs[0];
    for (int64_t w0 = 0; w0 < n_win; w0 += chunk) {
        const int nw = (int)std::min<int64_t>(chunk, n_win - w0);
        const int pad = S.k / 2;
        {
            KScope ks(ctx, st, KK_STEM, 2.0 * nw * S.lout * S.cout * S.cin * S.k,
                      4.0 * nw * ((double)2 * W + (double)(S.lout + 2) * S.cout));
            k_stem<<<nw, 256, 2 * (W + 2 * pad) * sizeof(float), st>>>(y, n_y, y_stride, first, stride, shift, w0,
                                                                      S.wt, S.cout, S.k, S.stride, W, S.lout, buf[0]);
        }
        AFG_LAUNCH_CHECK(ctx, "k_stem");
        float *A = buf[0], *B = buf[1], *Cb = buf[2], *D = buf[3];
        if (P.net.stem_pool) {
            gn_launch(ctx, buf[0], nw, S.lout, S.cout, G, S.gamma, S.beta, eps, nullptr, 1, buf[1], st);
            A = buf[1];
            B = buf[0];
        } else {
            gn_launch(ctx, buf[0], nw, S.lout, S.cout, G, S.gamma, S.beta, eps, nullptr, 1, nullptr, st);
        }
        AFG_LAUNCH_CHECK(ctx, "k_groupnorm(stem)");
        for (const BlockPlan &bp : P.blocks) {
            const ConvLayer &c1 = P.convs[bp.c1], &c2 = P.convs[bp.c2];
            conv_dispatch(ctx, A, B, nw, c1, st);
            gn_launch(ctx, B, nw, c1.lout, c1.cout, G, c1.gamma, c1.beta, eps, nullptr, 1, nullptr, st);
            conv_dispatch(ctx, B, Cb, nw, c2, st);
            const float *res = A;
            if (bp.sc >= 0) {
                const ConvLayer &sc = P.convs[bp.sc];
                conv_dispatch(ctx, A, D, nw, sc, st);
                gn_launch(ctx, D, nw, sc.lout, sc.cout, G, sc.gamma, sc.beta, eps, nullptr, 0, nullptr, st);
                res = D;
            }
            gn_launch(ctx, Cb, nw, c2.lout, c2.cout, G, c2.gamma, c2.beta, eps, res, 1, nullptr, st);
            AFG_LAUNCH_CHECK(ctx, "residual block");
            std::swap(A, Cb);
        }
        {
            KScope ks(ctx, st, KK_HEAD, 2.0 * nw * P.l_last * P.c_last, 4.0 * nw * (double)P.l_last * P.c_last);
            k_head<<<nw, 256, 0, st>>>(A, P.l_last, P.c_last, P.fc_w, P.fc_b, logits, w0);
        }
        AFG_LAUNCH_CHECK(ctx, "k_head");
    }
    return AFG_OK;
}
