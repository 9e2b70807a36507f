// Per-layer tcgen05 implicit-GEMM convolutions for wide 1D ResNets (the
// ResNet34 with GroupNorm of Sec. II): BF16 activations in HBM, chunk-major:
// per window, C/8 chunks of 8 channels, each (L + 2) rows of 16 bytes with a
// zero row before and after ([W][C/8][L + 2][8]).  A chunk is the no-swizzle
// K-major core-matrix layout the tensor core reads, so the chunks of one
// K-block of a window are one contiguous run in HBM, copied to shared memory
// unchanged by one bulk copy.  An activation that feeds a stride-2
// convolution is written parity-split instead: each chunk holds the even rows,
// then the odd rows ([W][C/8][2][(L + 2)/2][8]), so that stride-2 taps are
// contiguous too.
//
// One kernel per convolution, persistent over tiles, warp-specialised:
//   warp 0  producer: bulk copies of the K-block's activation chunks into
//           shared memory [chunk][row][16 B] (plus, for channel-major tiles,
//           the weight block)
//   warp 1  MMA issuer: tcgen05.mma kind::f16, FP32 accumulators in TMEM
//   warps 4..11 epilogue: GroupNorm statistics from TMEM, normalise,
//           optional residual, optional ReLU, BF16 store (+ zero pad rows)
// Taps are 16-byte row shifts of the activation descriptor; stride-2 convs
// read parity-split chunks, where tap 0/1/2 are the even rows / odd rows /
// even rows one row down (the 1x1 stride-2 shortcut loads only the odd rows).
//
// Orientations:
//   POS  M = 128 output positions per MMA, N = C_out; a tile is one window;
//        weights resident in shared memory; the window's input is one K-block.
//   CH   M = 128 output channels per MMA, N = L_out positions; a tile is a
//        128-channel slice x wpc windows; K-blocks of KB input channels
//        stream weights (bulk copy) and activations (TMA) through a ring.
// A tile's accumulators take at most 512 TMEM columns; tiles of at most 256
// columns may use two accumulator buffers, so that the epilogue of one tile
// overlaps the MMAs of the next.  The tile knobs (orientation, windows per
// tile, KB, ring depth, accumulator buffers) are chosen per layer geometry by
// measurement (net_tc_autotune) or by a default heuristic.
//
// Weight image of a layer (BF16, K-major core matrices): slices of
// Ms = min(C_out, 128) output channels, [slice][C_in/8][tap][Ms][8], so one
// K-block of any KB is a contiguous run and one image serves every knob.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "afg_internal.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int LT = 448;            // threads: 14 warps
constexpr int EPI_W0 = 2;          // first epilogue warp
constexpr int EPI_WARPS = 12;      // three per TMEM lane quarter
constexpr int EPI_T = EPI_WARPS * 32;
constexpr int EPI_PARTS = EPI_WARPS / 4;  // the epilogue splits positions (subtiles) into this many parts
constexpr int XCH_FLOATS = EPI_PARTS * 128 * 2;  // channel-major GroupNorm exchange (one window at a time)
constexpr int CH_SCR_BYTES = 256;                     // channel-major transpose scratch per epilogue warp
// epilogue region: position-major [red][scale][shift] or channel-major [exchange][scratch]
constexpr int POS_EPI_BYTES = EPI_WARPS * 32 * 4 + 2 * 512 * 4;
constexpr int CH_EPI_BYTES = XCH_FLOATS * 4 + EPI_WARPS * CH_SCR_BYTES;
constexpr int EPI_BYTES = POS_EPI_BYTES > CH_EPI_BYTES ? POS_EPI_BYTES : CH_EPI_BYTES;
constexpr uint64_t WAIT_NS = 2000000000ull;
constexpr int NB_MAX = 8;          // deepest shared-memory ring
constexpr uint32_t SMEM_LIMIT = 227 * 1024;

struct LayerArgs {
    int orient;          // 0 POS, 1 CH
    int n_win;
    int Lout, Cout, Cin, stride, taps;
    int rows;            // 16-byte rows per chunk in shared memory
    int in_rows;         // rows per chunk of the input in HBM (L_in + 2)
    int KB;              // input channels per K-block
    int odd_only;        // 1: load only the odd half of parity-split chunks (1x1 stride-2 shortcut)
    int out_split;       // 1: write the output parity-split (it feeds a stride-2 convolution)
    int n_kb;            // K-blocks per tile
    int wpc, slices;     // CH tiling
    int nsplit;          // CH: MMAs per window along N (L_out / nsplit <= 256 positions each)
    int NB;              // pipeline stages (<= NB_MAX)
    int shape;           // index of the unrolled MMA sequence of one stage (-1: generic loops)
    int nacc;            // TMEM accumulator buffers (1, or 2 with buffer b at column 256 b)
    int nparts;          // CH: parts the epilogue splits each window's positions into (2 or 3)
    int pair;            // CH: the two windows of a tile share each MMA along N: per chunk, window 0's rows
                         // in a slot of win_cols rows (rows rounded up to 8), then window 1's rows
    int mma_n;           // CH: N of one MMA (L_out / nsplit, or win_cols + L_out rounded up to 16 for a pair)
    int win_cols;        // CH: TMEM columns from one window of the tile to the next (L_out, or the pair slot)
    int G;
    float eps;
    int relu;
    uint32_t act_stage_bytes;  // activation bytes per stage (all tile windows)
    uint32_t w_block_bytes;    // CH: weight bytes per K-block; POS: whole image
    const unsigned char *wimg;
    const float *gamma, *beta;
    const __nv_bfloat16 *in;
    const __nv_bfloat16 *res;
    __nv_bfloat16 *out;
    int *err;
};

struct LSmem {
    uint32_t off_w, off_act, off_red, off_sc, off_bar, total;
};

__host__ __device__ inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline LSmem layer_smem(const LayerArgs &a) {
    LSmem s;
    const uint32_t wbytes = a.orient == 0 ? a.w_block_bytes : a.w_block_bytes * a.NB;
    s.off_w = 0;
    s.off_act = align_up(wbytes, 1024);
    s.off_red = align_up(s.off_act + a.act_stage_bytes * a.NB, 16);
    s.off_sc = s.off_red + EPI_WARPS * 32 * 4;  // position-major scale, shift
    s.off_bar = align_up(s.off_red + EPI_BYTES, 16);
    s.total = s.off_bar + 8 * (2 * NB_MAX + 5) + 16;  // full, empty, acc_full[2], acc_empty[2], wbar; slot, flag
    return s;
}

// row offset of tap r inside a shared-memory chunk (16-byte units): stride 1 reads rows
// p + r; stride 2 reads padded rows 2p, 2p + 1, 2p + 2 = even p, odd p, even p + 1 of a
// parity-split chunk (odd rows start at (L_in + 2) / 2); the 1x1 shortcut's odd rows alone
__host__ __device__ inline uint32_t tap_row(const LayerArgs &a, int r) {
    if (a.stride == 1) return (uint32_t)r;
    if (a.odd_only) return 0u;
    return r == 1 ? (uint32_t)(a.in_rows / 2) : (uint32_t)(r == 2 ? 1 : 0);
}

// padded output row R of a chunk in HBM, plain or parity-split (L + 2 even)
__device__ __forceinline__ size_t out_row(int R, int split, int Lout) {
    return split ? (size_t)((R & 1) * ((Lout + 2) >> 1) + (R >> 1)) : (size_t)R;
}

__device__ __forceinline__ bool bounded_wait(uint64_t *bar, uint32_t parity, int *abort_flag, int *err) {
    if (tc::mbar_wait(bar, parity, WAIT_NS)) return true;
    atomicExch(err, 1);
    *(volatile int *)abort_flag = 1;
    return false;
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"r"(EPI_T) : "memory"); }

// Sum 32 per-lane values over the warp so that lane l ends with the total of value l
// (butterfly reduce-scatter: 16 + 8 + 4 + 2 + 1 shuffles).
__device__ __forceinline__ float warp_reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = up ? v[i] : v[i + o];
            const float keep = up ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

// Position-major GroupNorm partials of one warp: the thread's rows (positions) of its
// subtiles j = hsel, hsel + EPI_PARTS, ... folded into the CO / CG groups (value g: sum,
// value 16 + g: sum of squares), 16 channels per TMEM wait; lane l returns the warp's total
// of value l.
template <int CO, int CG>
__device__ __forceinline__ float pos_group_partials(uint32_t tb, int hsel, int MT, int lane) {
    static_assert(CO / CG <= 16 && CO % 32 == 0 && CG % 2 == 0, "at most 16 groups of an even channel count");
    // per group: the sums and the sums of squares of its even and of its odd channels, one packed add and one
    // packed FMA per two adjacent channels (the loaded registers are the operand pairs as they stand)
    float2 s2[16], q2[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) s2[i] = q2[i] = make_float2(0.f, 0.f);
    for (int j = hsel; j < MT; j += EPI_PARTS) {
#pragma unroll
        for (int c0 = 0; c0 < CO; c0 += 16) {
            uint32_t r[16];
            tc::tmem_ld16_nowait(tb + (uint32_t)(j * CO + c0), r);
            tc::tmem_wait_ld();
#pragma unroll
            for (int c = 0; c < 16; c += 2) {
                const float2 v = make_float2(__uint_as_float(r[c]), __uint_as_float(r[c + 1]));
                const int g = (c0 + c) / CG;
                s2[g] = __fadd2_rn(s2[g], v);
                q2[g] = __ffma2_rn(v, v, q2[g]);
            }
        }
    }
    float gp[32];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        gp[i] = s2[i].x + s2[i].y;
        gp[16 + i] = q2[i].x + q2[i].y;
    }
    return warp_reduce_scatter32(gp, lane);
}

// Stage shapes with a fully unrolled MMA sequence.  A loop around single tcgen05.mma
// instructions costs 150-270 cycles per iteration on the issuing thread (measured), so
// one stage's MMAs are issued as straight-line code: channel-major (taps, k-steps,
// windows, N splits) and position-major (taps, k-steps, M subtiles).
#define AFG_CH_SHAPES(X) \
    X(0, 3, 2, 1, 2) X(1, 3, 4, 1, 2) X(2, 3, 8, 1, 2) X(3, 1, 2, 1, 2) X(4, 1, 4, 1, 2) \
    X(5, 1, 8, 1, 2) X(6, 3, 2, 1, 1) X(7, 3, 4, 1, 1) X(8, 3, 8, 1, 1) X(9, 1, 2, 1, 1) \
    X(10, 1, 4, 1, 1) X(11, 1, 8, 1, 1) X(12, 3, 2, 2, 1) X(13, 3, 4, 2, 1) X(14, 3, 8, 2, 1) \
    X(15, 1, 2, 2, 1) X(16, 1, 4, 2, 1) X(17, 1, 8, 2, 1) X(18, 3, 2, 3, 1) X(19, 3, 4, 3, 1) \
    X(20, 3, 8, 3, 1) X(21, 1, 2, 3, 1) X(22, 1, 4, 3, 1) X(23, 1, 8, 3, 1) X(24, 3, 2, 4, 1) \
    X(25, 3, 4, 4, 1) X(26, 3, 8, 4, 1) X(27, 1, 2, 4, 1) X(28, 1, 4, 4, 1) X(29, 1, 8, 4, 1) \
    X(30, 3, 2, 5, 1) X(31, 3, 4, 5, 1) X(32, 3, 8, 5, 1) X(33, 1, 2, 5, 1) X(34, 1, 4, 5, 1) \
    X(35, 1, 8, 5, 1)
#define AFG_POS_SHAPES(X) \
    X(0, 3, 4, 6) X(1, 3, 4, 3) X(2, 1, 4, 3) X(3, 3, 8, 3) X(4, 1, 8, 3) X(5, 3, 8, 6)

struct StageGeo {
    uint32_t dt;              // TMEM accumulator base of the tile
    uint64_t wd00, ad00;      // weight / activation descriptors of (tap 0, k-step 0)
    uint32_t toff0, toff1, toff2;  // activation descriptor offset of each tap (16-byte units)
    uint64_t w_tap, w_kk, a_kk, a_win;
    uint32_t n_step;          // TMEM columns between the N splits (= descriptor rows of a split)
    uint32_t win_cols;        // TMEM columns per window (channel-major) / per M subtile (position-major)
    uint32_t idesc;
    uint32_t first;           // 1 for the tile's first K-block (the first MMA of each accumulator overwrites)
};

__device__ __forceinline__ uint32_t tap_off(const StageGeo &g, int r) {
    return r == 0 ? g.toff0 : r == 1 ? g.toff1 : g.toff2;
}

template <int TAPS, int NKK, int WPC, int NSPLIT>
__device__ __forceinline__ void issue_ch(const StageGeo &g) {
#pragma unroll
    for (int r = 0; r < TAPS; ++r)
#pragma unroll
        for (int kk = 0; kk < NKK; ++kk) {
            const uint64_t wd = g.wd00 + (uint64_t)r * g.w_tap + (uint64_t)kk * g.w_kk;
            const uint64_t adk = g.ad00 + (uint64_t)tap_off(g, r) + (uint64_t)kk * g.a_kk;
            const uint32_t acc = (g.first && r == 0 && kk == 0) ? 0u : 1u;
#pragma unroll
            for (int i = 0; i < WPC; ++i)
#pragma unroll
                for (int h = 0; h < NSPLIT; ++h)
                    tc::mma_bf16(g.dt + (uint32_t)i * g.win_cols + (uint32_t)h * g.n_step, wd,
                                 adk + (uint64_t)i * g.a_win + (uint64_t)(h * g.n_step), g.idesc, acc);
        }
}

template <int TAPS, int NKK, int MT>
__device__ __forceinline__ void issue_pos(const StageGeo &g) {
#pragma unroll
    for (int r = 0; r < TAPS; ++r)
#pragma unroll
        for (int kk = 0; kk < NKK; ++kk) {
            const uint64_t wd = g.wd00 + (uint64_t)r * g.w_tap + (uint64_t)kk * g.w_kk;
            const uint64_t adk = g.ad00 + (uint64_t)tap_off(g, r) + (uint64_t)kk * g.a_kk;
            const uint32_t acc = (g.first && r == 0 && kk == 0) ? 0u : 1u;
#pragma unroll
            for (int j = 0; j < MT; ++j)
                tc::mma_bf16(g.dt + (uint32_t)j * g.win_cols, adk + (uint64_t)(128 * j), wd, g.idesc, acc);
        }
}

// host: index of (taps, k-steps, windows | subtiles, splits) in the shape tables, -1 if absent
static int stage_shape(int orient, int taps, int nkk, int wpc_or_mt, int nsplit) {
#define AFG_FIND_CH(I, T, K, W, S) \
    if (orient == 1 && taps == T && nkk == K && wpc_or_mt == W && nsplit == S) return I;
#define AFG_FIND_POS(I, T, K, M) \
    if (orient == 0 && taps == T && nkk == K && wpc_or_mt == M) return I;
    AFG_CH_SHAPES(AFG_FIND_CH)
    AFG_POS_SHAPES(AFG_FIND_POS)
#undef AFG_FIND_CH
#undef AFG_FIND_POS
    return -1;
}

// device: issue one stage with the unrolled sequence of shape `shape` (false if none)
template <int ORIENT>
__device__ __forceinline__ bool issue_stage(int shape, const StageGeo &g) {
    if (ORIENT == 1) {
        switch (shape) {
#define AFG_CASE_CH(I, T, K, W, S) \
    case I: issue_ch<T, K, W, S>(g); return true;
            AFG_CH_SHAPES(AFG_CASE_CH)
#undef AFG_CASE_CH
            default: return false;
        }
    } else {
        switch (shape) {
#define AFG_CASE_POS(I, T, K, M) \
    case I: issue_pos<T, K, M>(g); return true;
            AFG_POS_SHAPES(AFG_CASE_POS)
#undef AFG_CASE_POS
            default: return false;
        }
    }
}

// Residual rows of a channel-major epilogue unit (16 * NQ positions from p_first): lane e of
// each octet loads rows p_first + 8 b + e + 1 of the octet's chunk (issued one unit ahead).
template <int NQ>
__device__ __forceinline__ void ch_res_load(const __nv_bfloat16 *__restrict__ rw8, int p_first, int lane,
                                            uint4 (&rr)[4]) {
#pragma unroll
    for (int b = 0; b < 2 * NQ; ++b)
        rr[b] = __ldg(reinterpret_cast<const uint4 *>(rw8 + (size_t)(p_first + 8 * b + (lane & 7) + 1) * 8));
}

// Channel-major epilogue of 16 * NQ consecutive positions of the warp's 32 channels: the
// accumulators are read in the MMA fragment layout (lane t: channels t/4, 8 + t/4, 16 + t/4,
// 24 + t/4 of the warp at positions 2 (t % 4) and 2 (t % 4) + 1 of each group of 8), normalised
// (sc4[k], sh4[k]: channel 8 k + t/4), the residual added, ReLU'd and packed to BF16.  Per
// group, stmatrix.trans turns the four 8 x 8 fragments (one per 8-channel chunk) into chunk
// rows in the warp's 256-byte scratch (two chunks at a time), and every lane stores one
// 16-byte row: position p_first + 8 g + lane % 8 of chunk lane / 8.  The residual rows
// (rr[g], loaded by ch_res_load) come in through ldmatrix.trans the same way.
template <int NQ>
__device__ __forceinline__ void ch_store(uint32_t taddr, int p_first, const float (&sc4)[4], const float (&sh4)[4],
                                         bool has_res, const uint4 (&rr)[4], __nv_bfloat16 *__restrict__ ow8,
                                         int relu, int lane, int split, int Lout, uint32_t scr) {
    constexpr int NG = 2 * NQ;
    uint32_t A[4 * NG], B[4 * NG];  // TMEM lanes 0..15 and 16..31 of the warp's quarter
    if constexpr (NG == 4) {
        tc::tmem_ld16x256b_x4_nowait(taddr, A);
        tc::tmem_ld16x256b_x4_nowait(taddr + (16u << 16), B);
    } else {
        tc::tmem_ld16x256b_x2_nowait(taddr, A);
        tc::tmem_ld16x256b_x2_nowait(taddr + (16u << 16), B);
    }
    tc::tmem_wait_ld();
    const uint32_t my_row = scr + (uint32_t)(lane & 15) * 16;  // row address this thread gives stmatrix
    const int half = lane >> 4;                                  // which pass stores this lane's chunk
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        float2 x[4];  // x[k]: chunk k's channel at the lane's two positions
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t *src = k < 2 ? &A[4 * g + 2 * k] : &B[4 * g + 2 * (k - 2)];
            x[k] = __ffma2_rn(make_float2(__uint_as_float(src[0]), __uint_as_float(src[1])),
                              make_float2(sc4[k], sc4[k]), make_float2(sh4[k], sh4[k]));
        }
        if (has_res) {
            uint32_t Q[4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {  // rows of chunks 2h, 2h + 1 -> their fragments
                if (half == h)
                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(my_row), "r"(rr[g].x), "r"(rr[g].y),
                                 "r"(rr[g].z), "r"(rr[g].w)
                                 : "memory");
                __syncwarp();
                tc::ldmatrix_x2_trans(my_row, Q[2 * h], Q[2 * h + 1]);
                __syncwarp();
            }
#pragma unroll
            for (int k = 0; k < 4; ++k)
                x[k] = __fadd2_rn(x[k], make_float2(__uint_as_float(Q[k] << 16), __uint_as_float(Q[k] & 0xffff0000u)));
        }
        uint32_t R[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            R[k] = relu ? tc::pack_bf16x2_relu(x[k].x, x[k].y) : tc::pack_bf16x2(x[k].x, x[k].y);
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // fragments of chunks 2h, 2h + 1 -> their rows
            tc::stmatrix_x2_trans(my_row, R[2 * h], R[2 * h + 1]);
            __syncwarp();
            if (half == h) {
                uint4 v;
                asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                             : "r"(my_row)
                             : "memory");
                *reinterpret_cast<uint4 *>(ow8 + out_row(p_first + 8 * g + (lane & 7) + 1, split, Lout) * 8) = v;
            }
            __syncwarp();
        }
    }
}

template <int ORIENT>
__global__ void __launch_bounds__(LT, 1) k_conv_tc(const LayerArgs a) {
    // ORIENT (= a.orient) is compile-time: each instantiation keeps only its own path
    extern __shared__ __align__(1024) unsigned char sm[];
    const LSmem L = layer_smem(a);
    unsigned char *wsm = sm + L.off_w;
    unsigned char *act = sm + L.off_act;
    float *red = reinterpret_cast<float *>(sm + L.off_red);
    float *scale = reinterpret_cast<float *>(sm + L.off_sc);
    float *shift = scale + 512;
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + L.off_bar);
    uint64_t *empty = full + NB_MAX;
    uint64_t *acc_full = empty + NB_MAX;  // [2]
    uint64_t *acc_empty = acc_full + 2;   // [2]
    uint64_t *wbar = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(wbar + 1);
    int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_tiles = ORIENT == 0 ? a.n_win : ((a.n_win + a.wpc - 1) / a.wpc) * a.slices;
    const uint32_t chunk_bytes = (uint32_t)a.rows * 16;
    const uint32_t win_bytes = (uint32_t)(a.KB / 8) * chunk_bytes;  // one window's K-block activations
    const int Nw = ORIENT == 0 ? a.Cout : 128;                  // rows of the weight tile

    if (tid == 0) {
        for (int i = 0; i < a.NB; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&acc_full[b], 1);
            tc::mbar_init(&acc_empty[b], 1);
        }
        tc::mbar_init(wbar, 1);
        tc::fence_mbar_init();
        *abort_flag = 0;
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        // the whole warp walks the stages: lane 0 waits for the slot and arms its barrier (and
        // copies the weights), then the lanes issue the activation copies, in parallel where a
        // window pair needs one small copy per (chunk, window)
        if (ORIENT == 0 && lane == 0) {
            tc::mbar_expect_tx(wbar, a.w_block_bytes);
            for (uint32_t o = 0; o < a.w_block_bytes; o += 32768)
                tc::bulk_load(wsm + o, a.wimg + o, min(32768u, a.w_block_bytes - o), wbar);
        }
        uint32_t k = 0;  // stage uses
        bool stop = false;
        for (int t = blockIdx.x; t < n_tiles && !stop; t += gridDim.x) {
            if (__shfl_sync(0xffffffffu, lane == 0 ? *(volatile int *)abort_flag : 0, 0)) break;
            const int slice = ORIENT == 0 ? 0 : t % a.slices;
            const int w0 = ORIENT == 0 ? t : (t / a.slices) * a.wpc;
            const int nwt = ORIENT == 0 ? 1 : a.wpc;
            const int n_here = min(nwt, a.n_win - w0);  // absent windows: stale data, never stored
            for (int kb = 0; kb < a.n_kb; ++kb, ++k) {
                const int s = k % a.NB;
                int ok = 1;
                if (lane == 0) {
                    if (k >= (uint32_t)a.NB && !bounded_wait(&empty[s], ((k / a.NB) - 1) & 1, abort_flag, a.err)) {
                        ok = 0;
                    } else {
                        const uint32_t wb = ORIENT == 1 ? a.w_block_bytes : 0;
                        tc::mbar_expect_tx(&full[s], (uint32_t)n_here * win_bytes + wb);
                        if (ORIENT == 1) {
                            const unsigned char *src = a.wimg + ((size_t)slice * a.n_kb + kb) * a.w_block_bytes;  // [slice][C_in/8][tap][128][8]
                            unsigned char *dst = wsm + (size_t)s * a.w_block_bytes;
                            for (uint32_t o = 0; o < a.w_block_bytes; o += 32768)
                                tc::bulk_load(dst + o, src + o, min(32768u, a.w_block_bytes - o), &full[s]);
                        }
                    }
                }
                if (!__shfl_sync(0xffffffffu, ok, 0)) {
                    stop = true;
                    break;
                }
                unsigned char *ab = act + (size_t)s * a.act_stage_bytes;
                const size_t in_chunk = (size_t)a.in_rows * 16;  // bytes of one input chunk in HBM
                if (ORIENT == 1 && a.pair) {
                    // lane 2 c + i: chunk c of window i, at row (win_cols + rows) c + win_cols i
                    const int c = lane >> 1, i = lane & 1;
                    if (c < a.KB / 8 && i < n_here) {
                        const unsigned char *src = reinterpret_cast<const unsigned char *>(a.in) +
                                                   ((size_t)(w0 + i) * (a.Cin / 8) + (size_t)kb * (a.KB / 8) + c) * in_chunk;
                        tc::bulk_load(ab + ((size_t)c * (a.win_cols + a.rows) + (size_t)i * a.win_cols) * 16, src,
                                      chunk_bytes, &full[s]);
                    }
                } else if (lane == 0) {
                    for (int i = 0; i < n_here; ++i) {
                        const unsigned char *src = reinterpret_cast<const unsigned char *>(a.in) +
                                                   ((size_t)(w0 + i) * (a.Cin / 8) + (size_t)kb * (a.KB / 8)) * in_chunk;
                        unsigned char *d = ab + (size_t)i * win_bytes;
                        if (!a.odd_only) {
                            for (uint32_t o = 0; o < win_bytes; o += 32768)
                                tc::bulk_load(d + o, src + o, min(32768u, win_bytes - o), &full[s]);
                        } else {
                            for (int c = 0; c < a.KB / 8; ++c)
                                tc::bulk_load(d + (size_t)c * chunk_bytes, src + (size_t)c * in_chunk + chunk_bytes,
                                              chunk_bytes, &full[s]);
                        }
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            if (ORIENT == 0) bounded_wait(wbar, 0, abort_flag, a.err);
            const uint32_t idesc =
                ORIENT == 0 ? tc::idesc_bf16_f32(128, a.Cout) : tc::idesc_bf16_f32(128, a.mma_n);
            // activation chunk stride along K: one chunk, or a pair of window chunks
            const uint32_t a_lbo = (ORIENT == 1 && a.pair) ? (uint32_t)(a.win_cols + a.rows) * 16 : chunk_bytes;
            const int wpc_mma = (ORIENT == 1 && a.pair) ? 1 : a.wpc;
            const uint32_t wlbo = (uint32_t)(a.taps * Nw * 16);  // next 8-channel chunk of a weight tile
            const uint32_t toff0 = tap_row(a, 0), toff1 = tap_row(a, 1), toff2 = tap_row(a, 2);
            uint32_t k = 0, tiles = 0;
            for (int t = blockIdx.x; t < n_tiles && !*(volatile int *)abort_flag; t += gridDim.x, ++tiles) {
                const int buf = (int)(tiles % (uint32_t)a.nacc);
                const uint32_t use = tiles / (uint32_t)a.nacc;
                if (use > 0 && !bounded_wait(&acc_empty[buf], (use - 1) & 1, abort_flag, a.err)) break;
                tc::fence_after_sync();
                const uint32_t dt = tmem + (uint32_t)(buf * 256);
                bool ok = true;
                for (int kb = 0; kb < a.n_kb; ++kb, ++k) {
                    const int s = k % a.NB;
                    if (!bounded_wait(&full[s], (k / a.NB) & 1, abort_flag, a.err)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t ab = tc::smem_addr(act + (size_t)s * a.act_stage_bytes);
                    const uint32_t wb = tc::smem_addr(wsm + (ORIENT == 1 ? (size_t)s * a.w_block_bytes : 0));
                    // descriptors of (tap 0, k-step 0); every other MMA adds address deltas (in 16-byte
                    // units) to these, which stay inside the 14-bit start-address field (smem < 256 KB)
                    // weight tile [KB/8][tap][Nw][8] (POS: the whole image, n_kb = 1)
                    StageGeo g;
                    g.dt = dt;
                    g.wd00 = tc::desc_kmajor_noswizzle(wb, wlbo, 128);
                    g.ad00 = tc::desc_kmajor_noswizzle(ab, a_lbo, 128);
                    g.w_tap = (uint64_t)Nw;                // (Nw * 16) >> 4
                    g.w_kk = (uint64_t)(2 * a.taps * Nw);  // two chunks
                    g.a_kk = (uint64_t)(2 * a_lbo / 16);
                    g.a_win = (uint64_t)(win_bytes / 16);
                    g.toff0 = toff0;
                    g.toff1 = toff1;
                    g.toff2 = toff2;
                    g.n_step = ORIENT == 1 ? (uint32_t)(a.Lout / a.nsplit) : 0u;
                    g.win_cols = ORIENT == 1 ? (uint32_t)a.win_cols : (uint32_t)a.Cout;
                    g.idesc = idesc;
                    g.first = kb == 0 ? 1u : 0u;
                    if (!issue_stage<ORIENT>(a.shape, g)) {
                        // generic loops (shapes without an unrolled sequence)
                        const int MT = a.Lout / 128;
                        for (int r = 0; r < a.taps; ++r)
                            for (int kk = 0; kk < a.KB / 16; ++kk) {
                                const uint64_t wd = g.wd00 + (uint64_t)r * g.w_tap + (uint64_t)kk * g.w_kk;
                                const uint64_t adk = g.ad00 + (uint64_t)tap_off(g, r) + (uint64_t)kk * g.a_kk;
                                const uint32_t acc = (kb > 0 || r > 0 || kk > 0) ? 1u : 0u;
                                if (ORIENT == 0) {
                                    for (int j = 0; j < MT; ++j)
                                        tc::mma_bf16(dt + (uint32_t)(j * a.Cout), adk + (uint64_t)(128 * j), wd, idesc, acc);
                                } else {
                                    for (int i = 0; i < wpc_mma; ++i)
                                        for (int h = 0; h < a.nsplit; ++h)
                                            tc::mma_bf16(dt + (uint32_t)(i * a.Lout) + (uint32_t)h * g.n_step, wd,
                                                         adk + (uint64_t)i * g.a_win + (uint64_t)(h * g.n_step), idesc, acc);
                                }
                            }
                    }
                    tc::mma_commit(&empty[s]);
                }
                if (!ok) break;
                tc::mma_commit(&acc_full[buf]);
            }
        }
    } else if (warp >= EPI_W0) {
        // ------------------------------------------------------------ epilogue
        const int e = warp - EPI_W0;        // 0 .. EPI_WARPS - 1
        const int q = warp & 3;             // TMEM lane quarter (warp w reaches lanes 32 (w % 4) ..)
        const int hsel = e >> 2;            // which part of the subtiles / positions
        const int et = tid - EPI_W0 * 32;   // 0 .. EPI_T - 1
        const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16);
        uint32_t tiles = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++tiles) {
            const int buf = (int)(tiles % (uint32_t)a.nacc);
            bounded_wait(&acc_full[buf], (tiles / (uint32_t)a.nacc) & 1, abort_flag, a.err);
            epi_sync();  // every epilogue thread sees the same abort decision
            if (*(volatile int *)abort_flag) break;
            tc::fence_after_sync();
            const uint32_t tb = tq + (uint32_t)(buf * 256);
            if (ORIENT == 0) {
                // rows = positions; thread: row 32q + lane of subtiles j = hsel, hsel + 2, ...
                const int w = t;
                const int MT = a.Lout / 128;
                const int cg = a.Cout / a.G;
                const size_t ld = (size_t)(a.Lout + 2) * a.Cout;  // elements per window
                const size_t cs = (size_t)(a.Lout + 2) * 8;       // elements per chunk
                const __nv_bfloat16 *__restrict__ rw = a.res ? a.res + (size_t)w * ld : nullptr;
                // residual units (subtile j, 32 channels from c0) are loaded one unit ahead; the
                // first is issued before the statistics pass
                uint4 cur[4], nxt[4];
                if (rw && hsel < MT) {
                    const size_t o0 = (size_t)(128 * hsel + 32 * q + lane + 1) * 8;
#pragma unroll
                    for (int i = 0; i < 4; ++i) cur[i] = __ldg(reinterpret_cast<const uint4 *>(rw + o0 + i * cs));
                }
                // per-warp group partials: red[e][g] (sum) and red[e][16 + g] (sum of squares)
                float part;
                if (a.Cout == 64) part = pos_group_partials<64, 4>(tb, hsel, MT, lane);
                else part = pos_group_partials<128, 8>(tb, hsel, MT, lane);  // the two geometries the host admits
                red[e * 32 + lane] = part;
                epi_sync();
                if (et < a.Cout) {
                    const int g = et / cg;
                    float ts = 0.f, tq2 = 0.f;
                    for (int i = 0; i < EPI_WARPS; ++i) {
                        ts += red[i * 32 + g];
                        tq2 += red[i * 32 + 16 + g];
                    }
                    const float cnt = (float)a.Lout * (float)cg;
                    const float mean = ts / cnt;
                    const float var = fmaxf(tq2 / cnt - mean * mean, 0.f);
                    const float sc = rsqrtf(var + a.eps) * a.gamma[et];
                    scale[et] = sc;
                    shift[et] = a.beta[et] - mean * sc;
                }
                epi_sync();
                __nv_bfloat16 *__restrict__ ow = a.out + (size_t)w * ld;
                for (int j = hsel; j < MT; j += EPI_PARTS) {
                    const int row = 128 * j + 32 * q + lane + 1;
                    for (int c0 = 0; c0 < a.Cout; c0 += 32) {
                        const size_t s0 = (size_t)(c0 / 8) * cs + out_row(row, a.out_split, a.Lout) * 8;
                        if (rw) {  // prefetch the next unit: (j, c0 + 32) or (j + EPI_PARTS, 0)
                            const int cn = c0 + 32 < a.Cout ? c0 + 32 : 0;
                            const int jn = c0 + 32 < a.Cout ? j : j + EPI_PARTS;
                            if (jn < MT) {
                                const size_t on = (size_t)(cn / 8) * cs + (size_t)(128 * jn + 32 * q + lane + 1) * 8;
#pragma unroll
                                for (int i = 0; i < 4; ++i)
                                    nxt[i] = __ldg(reinterpret_cast<const uint4 *>(rw + on + i * cs));
                            }
                        }
                        uint4 rr[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) rr[i] = cur[i];
#pragma unroll
                        for (int i = 0; i < 4; ++i) cur[i] = nxt[i];
                        float v[32];
                        tc::tmem_ld32(tb + (uint32_t)(j * a.Cout + c0), v);
                        uint32_t pk[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) {  // channels c0 + 2i, c0 + 2i + 1 as one packed pair
                            float2 x = __ffma2_rn(make_float2(v[2 * i], v[2 * i + 1]),
                                                  *reinterpret_cast<const float2 *>(scale + c0 + 2 * i),
                                                  *reinterpret_cast<const float2 *>(shift + c0 + 2 * i));
                            if (rw) {
                                const uint32_t u = (i & 3) == 0 ? rr[i >> 2].x
                                                   : (i & 3) == 1 ? rr[i >> 2].y
                                                   : (i & 3) == 2 ? rr[i >> 2].z
                                                                  : rr[i >> 2].w;
                                x = __fadd2_rn(x, make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u)));
                            }
                            pk[i] = a.relu ? tc::pack_bf16x2_relu(x.x, x.y) : tc::pack_bf16x2(x.x, x.y);
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            *reinterpret_cast<uint4 *>(ow + s0 + i * cs) =
                                make_uint4(pk[4 * i], pk[4 * i + 1], pk[4 * i + 2], pk[4 * i + 3]);
                    }
                    if (row == 1 || row == a.Lout) {  // zero pad rows
                        const size_t pr = out_row(row == 1 ? 0 : a.Lout + 1, a.out_split, a.Lout) * 8;
                        for (int c = 0; c < a.Cout / 8; ++c)
                            *reinterpret_cast<uint4 *>(ow + (size_t)c * cs + pr) = make_uint4(0, 0, 0, 0);
                    }
                }
            } else {
                // rows = channels of the slice; thread: channel 32q + lane; the warps of a lane quarter
                // take the parts of every window's positions and exchange GroupNorm partials
                const int slice = t % a.slices;
                const int w0 = (t / a.slices) * a.wpc;
                const int cl = 32 * q + lane;
                const int c = slice * 128 + cl;
                const int cg = a.Cout / a.G;  // <= 32: lanes of one group are contiguous
                const float gam = a.gamma[c], bet = a.beta[c];
                const int np = a.nparts;       // 2 or 3; warps of an unused part only keep the barriers
                const bool active = hsel < np;
                const int Lh = a.Lout / np;
                const int pb = hsel * Lh;
                float *xch = red;  // [part][128 channels][sum, sum of squares] of the current window
                const uint32_t scr = tc::smem_addr(reinterpret_cast<unsigned char *>(red) + XCH_FLOATS * 4 +
                                                   e * CH_SCR_BYTES);
                const size_t ld = (size_t)(a.Lout + 2) * a.Cout;
                const int n32 = Lh / 32, tail16 = Lh % 32;
                for (int i = 0; i < a.wpc; ++i) {
                    const int w = w0 + i;
                    const uint32_t tw = tb + (uint32_t)(i * a.win_cols + pb);
                    const size_t co = (size_t)w * ld + (size_t)(c >> 3) * (a.Lout + 2) * 8;  // row 0 of c's chunk
                    const bool has_res = active && a.res != nullptr && w < a.n_win;
                    const __nv_bfloat16 *__restrict__ rw = has_res ? a.res + co : nullptr;
                    uint4 cur[4], nxt[4];  // residual of the current / next unit (loads in flight meanwhile)
                    if (has_res) {
                        if (n32 > 0) ch_res_load<2>(rw, pb, lane, cur);
                        else ch_res_load<1>(rw, pb, lane, cur);
                    }
                    float s = 0.f, qq = 0.f;
                    if (active) {
                        // sums and sums of squares of adjacent positions as packed pairs: one packed add and
                        // one packed FMA per two values, on the loaded registers as they stand
                        float2 s0 = make_float2(0.f, 0.f), q0 = s0, s1 = s0, q1 = s0;
                        int p0 = 0;
                        for (; p0 + 32 <= Lh; p0 += 32) {
                            uint32_t r0[16], r1[16];
                            tc::tmem_ld16_nowait(tw + (uint32_t)p0, r0);
                            tc::tmem_ld16_nowait(tw + (uint32_t)(p0 + 16), r1);
                            tc::tmem_wait_ld();
#pragma unroll
                            for (int p = 0; p < 16; p += 2) {
                                const float2 v0 = make_float2(__uint_as_float(r0[p]), __uint_as_float(r0[p + 1]));
                                const float2 v1 = make_float2(__uint_as_float(r1[p]), __uint_as_float(r1[p + 1]));
                                s0 = __fadd2_rn(s0, v0);
                                q0 = __ffma2_rn(v0, v0, q0);
                                s1 = __fadd2_rn(s1, v1);
                                q1 = __ffma2_rn(v1, v1, q1);
                            }
                        }
                        if (p0 < Lh) {
                            uint32_t r0[16];
                            tc::tmem_ld16_nowait(tw + (uint32_t)p0, r0);
                            tc::tmem_wait_ld();
#pragma unroll
                            for (int p = 0; p < 16; p += 2) {
                                const float2 v0 = make_float2(__uint_as_float(r0[p]), __uint_as_float(r0[p + 1]));
                                s0 = __fadd2_rn(s0, v0);
                                q0 = __ffma2_rn(v0, v0, q0);
                            }
                        }
                        s = (s0.x + s0.y) + (s1.x + s1.y);
                        qq = (q0.x + q0.y) + (q1.x + q1.y);
                        for (int o = cg / 2; o > 0; o >>= 1) {
                            s += __shfl_xor_sync(0xffffffffu, s, o);
                            qq += __shfl_xor_sync(0xffffffffu, qq, o);
                        }
                        float *mine = xch + (hsel * 128 + cl) * 2;
                        mine[0] = s;
                        mine[1] = qq;
                    }
                    epi_sync();  // the partials are written
                    // every part sums the parts in the same order, so all get the same statistics
                    s = 0.f;
                    qq = 0.f;
                    if (active)
                        for (int k = 0; k < np; ++k) {
                            const float *pk = xch + (k * 128 + cl) * 2;
                            s += pk[0];
                            qq += pk[1];
                        }
                    epi_sync();  // ... and read: the next window may overwrite them
                    if (!active || w >= a.n_win) continue;
                    const float cnt = (float)a.Lout * (float)cg;
                    const float mean = s / cnt;
                    const float var = fmaxf(qq / cnt - mean * mean, 0.f);
                    const float sc = rsqrtf(var + a.eps) * gam;
                    const float sh = bet - mean * sc;
                    float sc4[4], sh4[4];  // of the channels this lane holds in the fragment layout
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        sc4[k] = __shfl_sync(0xffffffffu, sc, 8 * k + (lane >> 2));
                        sh4[k] = __shfl_sync(0xffffffffu, sh, 8 * k + (lane >> 2));
                    }
                    __nv_bfloat16 *__restrict__ ow = a.out + co;
                    for (int u = 0; u < n32; ++u) {
                        const int p0 = 32 * u;
                        if (has_res) {
                            if (u + 1 < n32) ch_res_load<2>(rw, pb + p0 + 32, lane, nxt);
                            else if (tail16) ch_res_load<1>(rw, pb + p0 + 32, lane, nxt);
                        }
                        ch_store<2>(tw + (uint32_t)p0, pb + p0, sc4, sh4, has_res, cur, ow, a.relu, lane, a.out_split,
                                    a.Lout, scr);
#pragma unroll
                        for (int b = 0; b < 4; ++b) cur[b] = nxt[b];
                    }
                    if (tail16)
                        ch_store<1>(tw + (uint32_t)(32 * n32), pb + 32 * n32, sc4, sh4, has_res, cur, ow, a.relu, lane,
                                    a.out_split, a.Lout, scr);
                    if ((lane & 7) == 0) {  // zero pad rows of the chunk
                        if (hsel == 0)
                            *reinterpret_cast<uint4 *>(ow + out_row(0, a.out_split, a.Lout) * 8) = make_uint4(0, 0, 0, 0);
                        if (hsel == np - 1)
                            *reinterpret_cast<uint4 *>(ow + out_row(a.Lout + 1, a.out_split, a.Lout) * 8) =
                                make_uint4(0, 0, 0, 0);
                    }
                }
            }
            tc::fence_before_sync();
            epi_sync();
            if (et == 0) tc::mbar_arrive(&acc_empty[buf]);
        }
    }
    // ---- teardown: every role is done; free TMEM
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 512);
    }
}

// Stem of the wide network in one pass per window, straight into the first tensor-core
// layer's input: conv (k taps, stride s, 2 -> C0 channels) read from the whitened stream,
// GroupNorm, ReLU, optional max-pool (k3, s2, p1), BF16 chunk-major [C0/8][L + 2][8].
// grid (n_win), block STEM_T; warp w owns the 8-channel chunks w, w + 8, ... (their 16 k
// weights in registers), lanes own positions.  Pass 1 gets the GroupNorm sums (sum and sum of
// squares per channel) from the first and second moments of the conv inputs; pass 2 computes
// the conv, normalises, and pools across neighbouring lanes before writing.
constexpr int STEM_T = 256;
constexpr int STEM_KMAX = 7;
constexpr int STEM_NMOM = 2 * STEM_KMAX + STEM_KMAX * (2 * STEM_KMAX + 1);  // S and the upper triangle of M

// weights [c][ci][r] of the 8 channels of chunk ch, zero past k taps
__device__ __forceinline__ void stem_weights(const float *__restrict__ wt, int ch, int k, float (&wa)[8][STEM_KMAX],
                                             float (&wb)[8][STEM_KMAX]) {
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int r = 0; r < STEM_KMAX; ++r) {
            wa[c][r] = r < k ? wt[(ch * 8 + c) * 2 * k + r] : 0.f;
            wb[c][r] = r < k ? wt[(ch * 8 + c) * 2 * k + k + r] : 0.f;
        }
}

// conv of the 8 channels at the window position whose first padded input is x0
__device__ __forceinline__ void stem_conv8(const float *xs, int Wp, int x0, int k, const float (&wa)[8][STEM_KMAX],
                                           const float (&wb)[8][STEM_KMAX], float (&acc)[8]) {
    float u0[STEM_KMAX], u1[STEM_KMAX];
#pragma unroll
    for (int r = 0; r < STEM_KMAX; ++r) {
        u0[r] = r < k ? xs[x0 + r] : 0.f;
        u1[r] = r < k ? xs[Wp + x0 + r] : 0.f;
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        float a = 0.f;
#pragma unroll
        for (int r = 0; r < STEM_KMAX; ++r) {
            a = fmaf(wa[c][r], u0[r], a);
            a = fmaf(wb[c][r], u1[r], a);
        }
        acc[c] = a;
    }
}

__global__ void __launch_bounds__(STEM_T) k_stem_bf16(const float *__restrict__ y, int64_t n_y, int64_t y_stride,
                                                      int64_t first, int64_t stride, int64_t shift, int64_t w0,
                                                      const float *__restrict__ wt, const float *__restrict__ gamma,
                                                      const float *__restrict__ beta, int C0, int k, int s, int W,
                                                      int L0, int pool, int G, float eps,
                                                      __nv_bfloat16 *__restrict__ out) {
    extern __shared__ float xs[];  // [2][W + 2 pad], per-channel sums [2][C0], scale/shift [2][C0], moments
    const int pad = k / 2, Wp = W + 2 * pad;
    float *csum = xs + 2 * Wp, *csq = csum + C0, *scl = csq + C0, *shf = scl + C0;
    float *red = shf + C0, *mom = red + (STEM_T / 32) * STEM_NMOM;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t win = w0 + blockIdx.x;
    const int64_t start = first + win * stride;
    const float *y0 = y, *y1 = y + y_stride;
    for (int t = tid; t < Wp; t += STEM_T) {
        const int tt = t - pad;
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
    const int nch = C0 / 8;
    // ---- pass 1: per-channel sum and sum of squares of the raw conv output from the moments
    // of its inputs u_t = (x0[t s + r], x1[t s + r]), r < k:  sum_t y_c = w_c . S and
    // sum_t y_c^2 = w_c^T M w_c with S = sum_t u_t, M = sum_t u_t u_t^T (upper triangle)
    {
        constexpr int D = 2 * STEM_KMAX, NM = D * (D + 1) / 2;
        float S[D], M[NM];
#pragma unroll
        for (int i = 0; i < D; ++i) S[i] = 0.f;
#pragma unroll
        for (int i = 0; i < NM; ++i) M[i] = 0.f;
        for (int t = tid; t < L0; t += STEM_T) {
            float u[D];
#pragma unroll
            for (int r = 0; r < STEM_KMAX; ++r) {
                u[r] = r < k ? xs[t * s + r] : 0.f;
                u[STEM_KMAX + r] = r < k ? xs[Wp + t * s + r] : 0.f;
            }
            int m = 0;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                S[i] += u[i];
#pragma unroll
                for (int j = i; j < D; ++j) {
                    M[m] = fmaf(u[i], u[j], M[m]);
                    ++m;
                }
            }
        }
        // block reduction in a fixed order: warp butterflies, then the warps' rows in order
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) S[i] += __shfl_xor_sync(0xffffffffu, S[i], o);
#pragma unroll
        for (int i = 0; i < NM; ++i)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) M[i] += __shfl_xor_sync(0xffffffffu, M[i], o);
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < D; ++i) red[warp * STEM_NMOM + i] = S[i];
#pragma unroll
            for (int i = 0; i < NM; ++i) red[warp * STEM_NMOM + D + i] = M[i];
        }
        __syncthreads();
        for (int i = tid; i < STEM_NMOM; i += STEM_T) {
            float v = 0.f;
            for (int w8 = 0; w8 < STEM_T / 32; ++w8) v += red[w8 * STEM_NMOM + i];
            mom[i] = v;
        }
        __syncthreads();
        for (int c = tid; c < C0; c += STEM_T) {
            float wv[D];
#pragma unroll
            for (int r = 0; r < STEM_KMAX; ++r) {
                wv[r] = r < k ? wt[c * 2 * k + r] : 0.f;
                wv[STEM_KMAX + r] = r < k ? wt[c * 2 * k + k + r] : 0.f;
            }
            float sm = 0.f, sq = 0.f;
            int m = 0;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                sm = fmaf(wv[i], mom[i], sm);
#pragma unroll
                for (int j = i; j < D; ++j) {
                    const float v = wv[i] * wv[j] * mom[D + m++];
                    sq += (j == i) ? v : 2.f * v;
                }
            }
            csum[c] = sm;
            csq[c] = sq;
        }
    }
    __syncthreads();
    // ---- GroupNorm affine map per channel
    const int cg = C0 / G;
    for (int c = tid; c < C0; c += STEM_T) {
        const int g0 = (c / cg) * cg;
        float a = 0.f, b = 0.f;
        for (int j = g0; j < g0 + cg; ++j) {
            a += csum[j];
            b += csq[j];
        }
        const float cnt = (float)L0 * (float)cg;
        const float mean = a / cnt;
        const float var = fmaxf(b / cnt - mean * mean, 0.f);
        const float sc = rsqrtf(var + eps) * gamma[c];
        scl[c] = sc;
        shf[c] = beta[c] - mean * sc;
    }
    __syncthreads();
    // ---- pass 2: normalise + ReLU (+ max-pool) -> BF16 chunk-major
    const int Lo = pool ? (L0 + 2 - 3) / 2 + 1 : L0;
    const size_t cstride = (size_t)(Lo + 2) * 8;
    __nv_bfloat16 *ow = out + (size_t)blockIdx.x * nch * cstride;
    for (int ch = warp; ch < nch; ch += STEM_T / 32) {
        float wa[8][STEM_KMAX], wb[8][STEM_KMAX], sc8[8], sh8[8];
        stem_weights(wt, ch, k, wa, wb);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            sc8[c] = scl[ch * 8 + c];
            sh8[c] = shf[ch * 8 + c];
        }
        __nv_bfloat16 *oc = ow + (size_t)ch * cstride;
        // lanes take 32 consecutive conv positions; a pooled output u (window t = 2u-1..2u+1)
        // is formed by the even lane t = 2u from its neighbours' values (shuffles), the value
        // of t = 2u-1 at a warp boundary carried over from the previous pass
        float carry[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) carry[c] = -INFINITY;
        for (int t0 = 0; t0 < L0; t0 += 32) {
            const int t = t0 + lane;
            float z[8];
            if (t < L0) {
                float acc[8];
                stem_conv8(xs, Wp, t * s, k, wa, wb, acc);
#pragma unroll
                for (int c = 0; c < 8; ++c) z[c] = fmaxf(fmaf(acc[c], sc8[c], sh8[c]), 0.f);
            } else {
#pragma unroll
                for (int c = 0; c < 8; ++c) z[c] = -INFINITY;
            }
            float m[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                float lo = __shfl_up_sync(0xffffffffu, z[c], 1);
                const float hi = __shfl_down_sync(0xffffffffu, z[c], 1);
                if (lane == 0) lo = carry[c];
                m[c] = pool ? fmaxf(fmaxf(lo, z[c]), lane < 31 ? hi : -INFINITY) : z[c];
                carry[c] = __shfl_sync(0xffffffffu, z[c], 31);
            }
            const int u = pool ? t >> 1 : t;
            if (t < L0 && (!pool || !(lane & 1)) && u < Lo) {
                __nv_bfloat162 b0 = __floats2bfloat162_rn(m[0], m[1]), b1 = __floats2bfloat162_rn(m[2], m[3]);
                __nv_bfloat162 b2 = __floats2bfloat162_rn(m[4], m[5]), b3 = __floats2bfloat162_rn(m[6], m[7]);
                *reinterpret_cast<uint4 *>(oc + (size_t)(u + 1) * 8) =
                    make_uint4(*reinterpret_cast<uint32_t *>(&b0), *reinterpret_cast<uint32_t *>(&b1),
                               *reinterpret_cast<uint32_t *>(&b2), *reinterpret_cast<uint32_t *>(&b3));
            }
        }
        if (lane == 0) *reinterpret_cast<uint4 *>(oc) = make_uint4(0, 0, 0, 0);
        if (lane == 1) *reinterpret_cast<uint4 *>(oc + (size_t)(Lo + 1) * 8) = make_uint4(0, 0, 0, 0);
    }
}

// ---------------------------------------------------------------- stem on the tensor cores
// The stem conv (C0 = 64 outputs, 2 inputs, k <= 8 taps, stride s) as an implicit GEMM per
// window: M = the L0 output positions in subtiles of 128, N = 64, K = 2k zero-padded to 16,
// one tcgen05.mma per subtile.  A is an im2col tile built in shared memory from the window's
// samples (row t = x0[s t - pad + r], r < k, then x1[...], BF16, K-major without swizzle:
// element (t, kk) at (kk / 8) * L0 * 16 + t * 16 + (kk % 8) * 2), B the 64 x 16 weight tile.
// Rounds of 4 subtiles (256 TMEM columns, so two CTAs share an SM) run twice: first for the
// GroupNorm sums (read from TMEM), then to normalise, apply ReLU and max-pool (neighbouring
// positions are neighbouring lanes; the position before each 32-lane block comes through a
// shared edge table) and store BF16 chunk-major rows.
constexpr int STC_T = 256;      // threads: 8 warps, two per TMEM lane quarter (32 columns each)
constexpr int STC_C = 64;       // output channels
constexpr int STC_RS = 4;       // subtiles per round
constexpr int STC_COLS = 256;   // TMEM columns per CTA (STC_RS x 64)

struct StemTcSmem {
    size_t xs, a, b, edge, red, scl, bar, total;
};
__host__ __device__ inline StemTcSmem stem_tc_smem(int W, int k, int L0) {
    StemTcSmem m;
    const int pad = k / 2, Wp = W + 2 * pad;
    m.xs = 0;
    m.a = ((size_t)2 * Wp * 4 + 127) / 128 * 128;
    m.b = m.a + (size_t)2 * L0 * 16;
    m.edge = m.b + (size_t)2 * STC_C * 16;
    m.red = m.edge + (size_t)(L0 / 32) * STC_C * 4;
    m.scl = m.red + (size_t)(STC_T / 32) * 32 * 4;
    m.bar = m.scl + (size_t)2 * STC_C * 4;
    m.total = m.bar + 16;
    return m;
}

// CG: channels per GroupNorm group (a divisor of 32)
template <int CG>
__global__ void __launch_bounds__(STC_T, 2) k_stem_tc(const float *__restrict__ y, int64_t n_y, int64_t y_stride,
                                                      int64_t first, int64_t stride, int64_t shift, int64_t w0,
                                                      const float *__restrict__ wt, const float *__restrict__ gamma,
                                                      const float *__restrict__ beta, int k, int s, int W, int L0,
                                                      int pool, float eps, int *err, __nv_bfloat16 *__restrict__ out) {
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int NLG = 32 / CG;  // groups in a warp's 32 channels
    const StemTcSmem L = stem_tc_smem(W, k, L0);
    float *xs = reinterpret_cast<float *>(sm + L.xs);
    unsigned char *As = sm + L.a, *Bs = sm + L.b;
    float *edge = reinterpret_cast<float *>(sm + L.edge);
    float *red = reinterpret_cast<float *>(sm + L.red);
    float *scl = reinterpret_cast<float *>(sm + L.scl), *shf = scl + STC_C;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L.bar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + L.bar + 8);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q = warp & 3, ch = warp >> 2;  // TMEM lane quarter, column half
    const int pad = k / 2, Wp = W + 2 * pad;
    const int64_t win = w0 + blockIdx.x;
    const int64_t start = first + win * stride;

    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, STC_COLS);
        tc::tmem_relinquish();
    }
    // the window's samples (zero outside it), FP32
    for (int t = tid; t < Wp; t += STC_T) {
        const int tt = t - pad;
        float a = 0.f, b = 0.f;
        if (tt >= 0 && tt < W) {
            a = y[start + tt];
            int64_t i1 = start + shift + tt;
            if (i1 >= n_y) i1 -= n_y;
            b = y[y_stride + i1];
        }
        xs[t] = a;
        xs[Wp + t] = b;
    }
    // weight tile: element (c, kk), kk = ci * k + r, from wt[c][ci][r]
    for (int i = tid; i < STC_C * 16; i += STC_T) {
        const int c = i >> 4, kk = i & 15;
        const float v = kk < 2 * k ? wt[c * 2 * k + kk] : 0.f;
        reinterpret_cast<__nv_bfloat16 *>(Bs + (kk >> 3) * STC_C * 16 + c * 16)[kk & 7] = __float2bfloat16_rn(v);
    }
    __syncthreads();
    // im2col rows, 16 bytes per K half
    for (int t = tid; t < L0; t += STC_T) {
        uint32_t pk[8];
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            float v[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int kk = 2 * h + e, ci = kk >= k ? 1 : 0, r = kk - ci * k;
                v[e] = kk < 2 * k ? xs[ci * Wp + t * s + r] : 0.f;
            }
            pk[h] = tc::pack_bf16x2(v[0], v[1]);
        }
        *reinterpret_cast<uint4 *>(As + (size_t)t * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        *reinterpret_cast<uint4 *>(As + (size_t)L0 * 16 + (size_t)t * 16) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * ch);
    const uint32_t idesc = tc::idesc_bf16_f32(128, STC_C);
    const uint64_t ad0 = tc::desc_kmajor_noswizzle(tc::smem_addr(As), (uint32_t)(L0 * 16), 128);
    const uint64_t bd0 = tc::desc_kmajor_noswizzle(tc::smem_addr(Bs), STC_C * 16, 128);
    const int MT = L0 / 128, rounds = MT / STC_RS;
    uint32_t phase = 0;
    bool ok = true;
    // one round: MMAs of subtiles RS*rd .. + RS into columns 64 m, then wait for them
    auto mma_round = [&](int rd) {
        if (tid == 0) {
            tc::fence_after_sync();
#pragma unroll
            for (int m = 0; m < STC_RS; ++m)
                tc::mma_bf16(tmem + (uint32_t)(64 * m), ad0 + (uint64_t)((128 * (STC_RS * rd + m) * 16) >> 4), bd0,
                             idesc, 0u);
            tc::mma_commit(bar);
        }
        if (!tc::mbar_wait(bar, phase & 1, 1000000000ull)) ok = false;
        phase++;
        tc::fence_after_sync();
    };

    // ---- pass 1: GroupNorm sums (sum, sum of squares) of the warp's NLG groups
    float2 gs2[NLG], gq2[NLG];  // per group: sums and sums of squares of its even and odd channels
#pragma unroll
    for (int g = 0; g < NLG; ++g) gs2[g] = gq2[g] = make_float2(0.f, 0.f);
    for (int rd = 0; rd < rounds; ++rd) {
        mma_round(rd);
#pragma unroll 1
        for (int m = 0; m < STC_RS; ++m) {
            float v[32];
            tc::tmem_ld32(tq + (uint32_t)(64 * m), v);
#pragma unroll
            for (int c = 0; c < 32; c += 2) {  // adjacent channels of a group as packed pairs
                const float2 vv = make_float2(v[c], v[c + 1]);
                gs2[c / CG] = __fadd2_rn(gs2[c / CG], vv);
                gq2[c / CG] = __ffma2_rn(vv, vv, gq2[c / CG]);
            }
        }
        tc::fence_before_sync();
        __syncthreads();  // every TMEM read of the round is done before the next round's MMAs
    }
    float2 gs[NLG];
#pragma unroll
    for (int g = 0; g < NLG; ++g) gs[g] = make_float2(gs2[g].x + gs2[g].y, gq2[g].x + gq2[g].y);
#pragma unroll
    for (int g = 0; g < NLG; ++g)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            gs[g].x += __shfl_xor_sync(0xffffffffu, gs[g].x, o);
            gs[g].y += __shfl_xor_sync(0xffffffffu, gs[g].y, o);
        }
    if (lane == 0)
#pragma unroll
        for (int g = 0; g < NLG; ++g) {
            red[warp * 32 + 2 * g] = gs[g].x;
            red[warp * 32 + 2 * g + 1] = gs[g].y;
        }
    __syncthreads();
    if (tid < STC_C) {
        const int c = tid, h = c >> 5, g = (c & 31) / CG;
        float a = 0.f, b = 0.f;
        for (int qq = 0; qq < 4; ++qq) {  // the four warps of column half h
            a += red[(h * 4 + qq) * 32 + 2 * g];
            b += red[(h * 4 + qq) * 32 + 2 * g + 1];
        }
        const float cnt = (float)L0 * (float)CG;
        const float mean = a / cnt;
        const float var = fmaxf(b / cnt - mean * mean, 0.f);
        const float sc = rsqrtf(var + eps) * gamma[c];
        scl[c] = sc;
        shf[c] = beta[c] - mean * sc;
    }
    __syncthreads();

    // ---- pass 2: normalise + ReLU (+ max-pool) -> BF16 chunk-major rows
    const int Lo = pool ? (L0 + 2 - 3) / 2 + 1 : L0;
    const size_t cstride = (size_t)(Lo + 2) * 8;
    __nv_bfloat16 *ow = out + (size_t)blockIdx.x * (STC_C / 8) * cstride;
    const float *sc = scl + 32 * ch, *sh = shf + 32 * ch;  // (warp-uniform shared reads)
    for (int rd = 0; rd < rounds; ++rd) {
        mma_round(rd);
#pragma unroll 1
        for (int m = 0; m < STC_RS; ++m) {
            const int j = STC_RS * rd + m, blk = 4 * j + q, t = 32 * blk + lane;
            float z[32];
            tc::tmem_ld32(tq + (uint32_t)(64 * m), z);
#pragma unroll
            for (int c = 0; c < 32; ++c) z[c] = fmaxf(fmaf(z[c], sc[c], sh[c]), 0.f);
            if (pool && lane == 31)
#pragma unroll
                for (int c = 0; c < 32; ++c) edge[blk * STC_C + 32 * ch + c] = z[c];
            __syncthreads();  // the edge of the block before this one is written
            uint32_t pk[16];
            if (pool) {
#pragma unroll
                for (int c = 0; c < 32; c += 2) {
                    float lo0 = __shfl_up_sync(0xffffffffu, z[c], 1), lo1 = __shfl_up_sync(0xffffffffu, z[c + 1], 1);
                    const float hi0 = __shfl_down_sync(0xffffffffu, z[c], 1);
                    const float hi1 = __shfl_down_sync(0xffffffffu, z[c + 1], 1);
                    if (lane == 0) {
                        lo0 = blk > 0 ? edge[(blk - 1) * STC_C + 32 * ch + c] : -INFINITY;
                        lo1 = blk > 0 ? edge[(blk - 1) * STC_C + 32 * ch + c + 1] : -INFINITY;
                    }
                    pk[c / 2] = tc::pack_bf16x2(fmaxf(fmaxf(lo0, z[c]), hi0), fmaxf(fmaxf(lo1, z[c + 1]), hi1));
                }
            } else {
#pragma unroll
                for (int c = 0; c < 32; c += 2) pk[c / 2] = tc::pack_bf16x2(z[c], z[c + 1]);
            }
            const int u = pool ? t >> 1 : t;
            if ((!pool || !(lane & 1)) && u < Lo) {
#pragma unroll
                for (int c8 = 0; c8 < 4; ++c8)  // chunks 4 ch .. 4 ch + 3, row u + 1
                    *reinterpret_cast<uint4 *>(ow + (size_t)(4 * ch + c8) * cstride + (size_t)(u + 1) * 8) =
                        make_uint4(pk[4 * c8], pk[4 * c8 + 1], pk[4 * c8 + 2], pk[4 * c8 + 3]);
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    // zero pad rows of the 8 chunks
    if (tid < 16) {
        const int c8 = tid >> 1, row = (tid & 1) ? Lo + 1 : 0;
        *reinterpret_cast<uint4 *>(ow + (size_t)c8 * cstride + (size_t)row * 8) = make_uint4(0, 0, 0, 0);
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, STC_COLS);
}

// grid (n_win), block 256: logit = fc_b + sum_c fc_w[c] * mean_t x[t][c] (bf16 chunk-major input,
// C / 8 <= 256 chunks); each thread sums 8 channels of one chunk over a subset of rows
__global__ void k_head_bf16(const __nv_bfloat16 *__restrict__ x, int L, int C, const float *__restrict__ fc_w,
                            const float *__restrict__ fc_b, float *__restrict__ logits, int64_t w0) {
    __shared__ float part[256][9];
    const int tid = threadIdx.x, nch = C / 8, tpc = 256 / nch;  // threads per chunk
    const int ch = tid % nch, r0 = tid / nch;
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (r0 < tpc) {
        const uint4 *xc = reinterpret_cast<const uint4 *>(x + ((int64_t)blockIdx.x * nch + ch) * (L + 2) * 8) + 1;
        for (int r = r0; r < L; r += tpc) {
            const uint4 u = __ldg(xc + r);
            const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                s[2 * e] += __uint_as_float(w4[e] << 16);
                s[2 * e + 1] += __uint_as_float(w4[e] & 0xffff0000u);
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) part[tid][e] = s[e];
    __syncthreads();
    __shared__ float term[512];
    for (int c = tid; c < C; c += 256) {
        float t = 0.f;
        for (int g = 0; g < tpc; ++g) t += part[g * nch + c / 8][c % 8];
        term[c] = fc_w[c] * (t / (float)L);
    }
    __syncthreads();
    if (tid < 32) {
        float z = 0.f;
        for (int c = tid; c < C; c += 32) z += term[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
        if (tid == 0) logits[w0 + blockIdx.x] = fc_b[0] + z;
    }
}

}  // namespace

// Tile knobs of one convolution (see the header comment).
struct TileKnobs {
    int orient = 1, wpc = 1, KB = 64, NB = 1, nacc = 1;
    bool operator==(const TileKnobs &o) const {
        return orient == o.orient && wpc == o.wpc && KB == o.KB && NB == o.NB && nacc == o.nacc;
    }
};

// Per-layer plan of the tensor-core path (built once per context).
struct TcLayer {
    LayerArgs a;                 // everything but pointers and n_win
    TileKnobs knobs;
    unsigned char *wimg = nullptr;
    int residual = 0, relu = 1;  // epilogue of this layer in the network
    int out_split = 0;           // output feeds a stride-2 convolution: written parity-split
    int tuned = 0, n_cand = 0;
    float us_chosen = 0.f, us_default = 0.f;
};

struct TcPlan {
    std::vector<TcLayer> layers;  // indexed like NetPlan::convs (index 0 unused: the stem runs SIMT)
    void *mem = nullptr;
};

// Geometry of a layer under the given knobs; false if the knobs do not fit the layer.
static bool layer_geometry(const ConvLayer &C, int G, float eps, const TileKnobs &k, LayerArgs &a) {
    memset(&a, 0, sizeof a);
    a.Lout = C.lout;
    a.Cout = C.cout;
    a.Cin = C.cin;
    a.stride = C.stride;
    a.taps = C.k;
    a.G = G;
    a.eps = eps;
    a.orient = k.orient;
    a.nacc = k.nacc;
    a.NB = k.NB;
    if (k.nacc != 1 && k.nacc != 2) return false;
    if (k.NB < 1 || k.NB > NB_MAX) return false;
    if (C.cin % 32 || C.cout % 16 || G < 1 || C.cout % G) return false;
    if (!((C.k == 3 && C.stride <= 2) || (C.k == 1 && C.stride == 2))) return false;
    if (C.stride == 2 && (C.lin % 2 || C.lout != C.lin / 2)) return false;
    const int cg = C.cout / G;
    if (cg & (cg - 1)) return false;
    const int acc_cols = k.nacc == 2 ? 256 : 512;
    a.in_rows = C.lin + 2;
    a.odd_only = (C.stride == 2 && C.k == 1) ? 1 : 0;
    a.rows = a.odd_only ? a.in_rows / 2 : a.in_rows;
    if (k.orient == 0) {
        // position-major: one window per tile, all input channels one K-block, weights resident
        if (C.cout > 128 || C.lout % 128 || (C.lout / 128) * C.cout > acc_cols) return false;
        // the statistics pass is unrolled for 16 groups of 64 or 128 channels
        if (G != 16 || (C.cout != 64 && C.cout != 128)) return false;
        if (k.wpc != 1) return false;
        a.KB = C.cin;
        a.n_kb = 1;
        a.wpc = 1;
        a.slices = 1;
        a.nsplit = 1;
        a.nparts = EPI_PARTS;
        a.pair = 0;
        a.mma_n = C.cout;
        a.win_cols = C.cout;
        a.w_block_bytes = (uint32_t)(C.k * C.cin * C.cout * 2);
    } else {
        if (C.cout % 128 || cg > 32) return false;
        if (!(k.KB == 32 || k.KB == 64 || k.KB == 128) || C.cin % k.KB) return false;
        a.nsplit = (C.lout + 255) / 256;
        if (C.lout % 32 || C.lout % a.nsplit || (C.lout / a.nsplit) % 16) return false;
        a.nparts = C.lout % (16 * EPI_PARTS) == 0 ? EPI_PARTS : 2;
        if (k.wpc < 1 || k.wpc * C.lout > acc_cols) return false;
        a.wpc = k.wpc;
        a.slices = C.cout / 128;
        a.KB = k.KB;
        // two windows per MMA where their rows fit one N <= 256 (stride 1: every row is read); window
        // 1 starts at an 8-aligned row (and TMEM column) so the epilogue reads whole 8-column groups
        const int pslot = (a.rows + 7) / 8 * 8;
        const int pair_n = (pslot + C.lout + 15) / 16 * 16;
        a.pair = (k.wpc == 2 && C.stride == 1 && a.nsplit == 1 && pair_n <= acc_cols && pair_n <= 256) ? 1 : 0;
        a.mma_n = a.pair ? pair_n : C.lout / a.nsplit;
        a.win_cols = a.pair ? pslot : C.lout;
        a.n_kb = C.cin / k.KB;
        a.w_block_bytes = (uint32_t)(C.k * a.KB * 128 * 2);
    }
    a.act_stage_bytes = (uint32_t)a.wpc * (a.KB / 8) * (uint32_t)a.rows * 16;
    if (a.pair) {
        a.act_stage_bytes = (uint32_t)(a.KB / 8) * (uint32_t)(a.win_cols + a.rows) * 16;
        if (layer_smem(a).total > SMEM_LIMIT) {  // the padded pair does not fit: one MMA per window
            a.pair = 0;
            a.mma_n = C.lout / a.nsplit;
            a.win_cols = C.lout;
            a.act_stage_bytes = (uint32_t)a.wpc * (a.KB / 8) * (uint32_t)a.rows * 16;
        }
    }
    a.shape = stage_shape(a.orient, a.taps, a.KB / 16, a.orient == 0 ? a.Lout / 128 : (a.pair ? 1 : a.wpc), a.nsplit);
    return layer_smem(a).total <= SMEM_LIMIT;
}

// deepest ring that fits (0 if none)
static int deepest_ring(const ConvLayer &C, int G, float eps, TileKnobs k) {
    LayerArgs a;
    for (int nb = NB_MAX; nb >= 1; --nb) {
        k.NB = nb;
        if (layer_geometry(C, G, eps, k, a)) return nb;
    }
    return 0;
}

// The heuristic used until the layer is tuned: position-major tiles only where a
// 128-channel slice does not exist, about 384 accumulator columns per tile.
static TileKnobs default_knobs(const ConvLayer &C, int G, float eps) {
    TileKnobs k;
    k.orient = C.cout < 128 ? 0 : 1;
    k.wpc = k.orient == 0 ? 1 : std::max(1, 384 / C.lout);
    k.KB = (C.stride == 2 && C.k == 3) ? 32 : 64;
    k.nacc = 1;
    k.NB = std::min(4, deepest_ring(C, G, eps, k));
    return k;
}

// Every knob combination the tuner times for this layer (deepest ring for each).
static void tile_candidates(const ConvLayer &C, int G, float eps, std::vector<TileKnobs> &out) {
    out.clear();
    for (int orient = 0; orient < 2; ++orient)
        for (int nacc = 1; nacc <= 2; ++nacc)
            for (int wpc = 1; wpc <= (orient == 0 ? 1 : 8); ++wpc)
                for (int KB : {32, 64, 128}) {
                    if (orient == 0 && KB != 64) continue;  // KB is C_in for position-major tiles
                    TileKnobs k;
                    k.orient = orient;
                    k.nacc = nacc;
                    k.wpc = wpc;
                    k.KB = orient == 0 ? C.cin : KB;
                    k.NB = deepest_ring(C, G, eps, k);
                    if (k.NB > 0) out.push_back(k);
                }
}

static bool build_layer(const ConvLayer &C, int G, float eps, const TileKnobs &k, TcLayer &T) {
    LayerArgs a;
    if (!layer_geometry(C, G, eps, k, a)) return false;
    T.a = a;
    T.knobs = k;
    return true;
}

// BF16 weight image of one conv: [slice][C_in/8][tap][Ms][8], Ms = min(C_out, 128)
static void pack_weights(const ConvLayer &C, const float *wt_host /* [(r*cin+ci)*cout+co] */,
                         std::vector<unsigned short> &img) {
    auto bf = [](float v) {
        __nv_bfloat16 b = __float2bfloat16_rn(v);
        return *reinterpret_cast<unsigned short *>(&b);
    };
    const int Ms = std::min(C.cout, 128);
    img.assign((size_t)C.k * C.cin * C.cout, 0);
    for (int r = 0; r < C.k; ++r)
        for (int ci = 0; ci < C.cin; ++ci)
            for (int co = 0; co < C.cout; ++co) {
                const int sl = co / Ms, m = co % Ms;
                const size_t idx = ((((size_t)sl * (C.cin / 8) + ci / 8) * C.k + r) * Ms + m) * 8 + ci % 8;
                img[idx] = bf(wt_host[((size_t)r * C.cin + ci) * C.cout + co]);
            }
}

static bool full_net_supported(const afg_ctx *ctx) {
    const NetPlan &P = ctx->plan;
    if (P.blocks.empty() || P.convs[P.blocks[0].c1].stride != 1) return false;  // the stem output is not split
    for (const BlockPlan &bp : P.blocks)
        if (P.convs[bp.c2].lout % 2) return false;  // parity-split outputs need L + 2 even
    for (size_t i = 1; i < P.convs.size(); ++i) {
        const ConvLayer &C = P.convs[i];
        if (C.cin % 64 || C.cout % 64 || C.cout > 512) return false;
        const TileKnobs k = default_knobs(C, P.net.groups, P.net.eps);
        if (k.NB < 1) return false;
        TcLayer T;
        if (!build_layer(C, P.net.groups, P.net.eps, k, T)) return false;
    }
    return true;
}

int net_tc_layers_prepare(afg_ctx *ctx) {
    NetPlan &P = ctx->plan;
    if (P.convs.size() < 2 || !full_net_supported(ctx)) return AFG_OK;
    TcPlan *tp = new TcPlan();
    tp->layers.resize(P.convs.size());
    for (size_t b = 0; b < P.blocks.size(); ++b) {
        const BlockPlan &bp = P.blocks[b];
        tp->layers[bp.c2].residual = 1;
        if (bp.sc >= 0) tp->layers[bp.sc].relu = 0;
        // the block's output feeds the next block's stride-2 convolutions
        if (b + 1 < P.blocks.size() && P.convs[P.blocks[b + 1].c1].stride == 2) tp->layers[bp.c2].out_split = 1;
    }
    std::vector<float> all(ctx->d_params_bytes / sizeof(float));
    AFG_CUDA(ctx, cudaMemcpy(all.data(), ctx->d_params, ctx->d_params_bytes, cudaMemcpyDeviceToHost));
    std::vector<std::vector<unsigned short>> imgs(P.convs.size());
    size_t total = 0;
    for (size_t i = 1; i < P.convs.size(); ++i) {
        const ConvLayer &C = P.convs[i];
        build_layer(C, P.net.groups, P.net.eps, default_knobs(C, P.net.groups, P.net.eps), tp->layers[i]);
        pack_weights(C, all.data() + (C.wt - ctx->d_params), imgs[i]);
        total += (imgs[i].size() * 2 + 1023) / 1024 * 1024;
    }
    void *d = nullptr;
    if (cudaMalloc(&d, total) != cudaSuccess) {
        cudaGetLastError();
        delete tp;
        return afg_fail(ctx, AFG_ERR_OOM, "tensor-core weight images: cudaMalloc(%zu) failed", total);
    }
    ctx->bytes_held += (int64_t)total;
    tp->mem = d;
    size_t off = 0;
    for (size_t i = 1; i < P.convs.size(); ++i) {
        tp->layers[i].wimg = static_cast<unsigned char *>(d) + off;
        AFG_CUDA(ctx, cudaMemcpy(tp->layers[i].wimg, imgs[i].data(), imgs[i].size() * 2, cudaMemcpyHostToDevice));
        off += (imgs[i].size() * 2 + 1023) / 1024 * 1024;
    }
    AFG_CUDA(ctx, cudaFuncSetAttribute(k_conv_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT));
    AFG_CUDA(ctx, cudaFuncSetAttribute(k_conv_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT));
    {
        const ConvLayer &S = P.convs[0];
        const int smem = (int)stem_tc_smem(ctx->cfg.win_len, S.k, S.lout).total;
        AFG_CUDA(ctx, cudaFuncSetAttribute(k_stem_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        AFG_CUDA(ctx, cudaFuncSetAttribute(k_stem_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        AFG_CUDA(ctx, cudaFuncSetAttribute(k_stem_tc<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        AFG_CUDA(ctx, cudaFuncSetAttribute(k_stem_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        AFG_CUDA(ctx, cudaFuncSetAttribute(k_stem_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    }
    ctx->tcplan = tp;
    return AFG_OK;
}

// The stem runs on the tensor cores where its shape fits k_stem_tc: 64 outputs, 2 k <= 16,
// whole rounds of 4 subtiles of 128 positions, groups of 2..32 channels.
static bool stem_tc_fits(const afg_ctx *ctx) {
    const ConvLayer &S = ctx->plan.convs[0];
    const int G = ctx->plan.net.groups;
    if (S.cout != STC_C || S.cin != 2 || 2 * S.k > 16 || S.lout % (128 * STC_RS) || G < 2 || STC_C % G) return false;
    const int cg = STC_C / G;
    return cg >= 2 && cg <= 32 && !(cg & (cg - 1)) &&
           stem_tc_smem(ctx->cfg.win_len, S.k, S.lout).total <= (size_t)SMEM_LIMIT;
}

void net_tc_layers_release(afg_ctx *ctx) {
    if (!ctx->tcplan) return;
    if (ctx->tcplan->mem) cudaFree(ctx->tcplan->mem);
    delete ctx->tcplan;
    ctx->tcplan = nullptr;
}

bool net_tc_layers_available(const afg_ctx *ctx) { return ctx->tcplan != nullptr; }

// launch one layer (no accounting)
static int conv_tc_raw(afg_ctx *ctx, const TcLayer &T, const __nv_bfloat16 *in, const __nv_bfloat16 *res, int relu,
                       __nv_bfloat16 *out, int nw, const ConvLayer &C, cudaStream_t st) {
    (void)C;
    LayerArgs a = T.a;
    a.n_win = nw;
    a.relu = relu;
    a.out_split = T.out_split;
    a.wimg = T.wimg;
    a.gamma = C.gamma;
    a.beta = C.beta;
    a.in = in;
    a.res = res;
    a.out = out;
    a.err = ctx->d_err;
    const int n_tiles = a.orient == 0 ? nw : ((nw + a.wpc - 1) / a.wpc) * a.slices;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const unsigned grid = (unsigned)std::max(1, std::min(n_tiles, sms));
    if (a.orient == 0) k_conv_tc<0><<<grid, LT, layer_smem(a).total, st>>>(a);
    else k_conv_tc<1><<<grid, LT, layer_smem(a).total, st>>>(a);
    AFG_LAUNCH_CHECK(ctx, "k_conv_tc");
    return AFG_OK;
}

static int conv_tc(afg_ctx *ctx, const TcLayer &T, const __nv_bfloat16 *in, const __nv_bfloat16 *res, int relu,
                   __nv_bfloat16 *out, int nw, const ConvLayer &C, cudaStream_t st) {
    const double flops = 2.0 * nw * C.lout * C.cout * (double)C.k * C.cin;
    const double bytes = 2.0 * nw * ((double)(C.lin + 2) * C.cin + (double)(C.lout + 2) * C.cout * (res ? 2 : 1)) +
                         2.0 * C.k * C.cin * C.cout;
    KScope ks(ctx, st, KK_CONV_TC, flops, bytes);
    return conv_tc_raw(ctx, T, in, res, relu, out, nw, C, st);
}

// deterministic pseudo-random BF16 in [-1, 1) (tuning inputs)
__global__ void k_fill_bf16(__nv_bfloat16 *x, int64_t n, uint32_t seed) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 0x9E3779B1u ^ seed;
        h ^= h >> 16;
        h *= 0x85EBCA6Bu;
        h ^= h >> 13;
        x[i] = __float2bfloat16_rn((float)(h >> 8) * (2.0f / 16777216.0f) - 1.0f);
    }
}

// Time every candidate tile of each distinct layer geometry on nw synthetic windows and
// keep the fastest.  Synchronises the device; refuses during stream capture.
int net_tc_autotune(afg_ctx *ctx, int64_t n_win, cudaStream_t st) {
    if (!ctx->tcplan) return afg_fail(ctx, AFG_ERR_UNSUPPORTED, "autotune: no per-layer tensor-core plan");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    AFG_CUDA(ctx, cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return afg_fail(ctx, AFG_ERR_STATE, "autotune: stream is capturing");
    const NetPlan &P = ctx->plan;
    TcPlan &TP = *ctx->tcplan;
    const int nw = (int)std::max<int64_t>(1, std::min<int64_t>(n_win > 0 ? n_win : 1024, 4096));
    const int64_t per_win16 = P.max_act_per_window * 2;
    __nv_bfloat16 *in = nullptr, *res = nullptr, *out = nullptr;
    int rc = afg_ws_reserve(ctx, WS_ACT0, (size_t)(nw * per_win16), (void **)&in);
    if (!rc) rc = afg_ws_reserve(ctx, WS_ACT1, (size_t)(nw * per_win16), (void **)&res);
    if (!rc) rc = afg_ws_reserve(ctx, WS_ACT2, (size_t)(nw * per_win16), (void **)&out);
    if (rc) return rc;
    const int64_t n_el = nw * P.max_act_per_window;
    k_fill_bf16<<<1024, 256, 0, st>>>(in, n_el, 0x1234567u);
    k_fill_bf16<<<1024, 256, 0, st>>>(res, n_el, 0x7654321u);
    AFG_LAUNCH_CHECK(ctx, "k_fill_bf16");
    cudaEvent_t e0, e1;
    AFG_CUDA(ctx, cudaEventCreate(&e0));
    AFG_CUDA(ctx, cudaEventCreate(&e1));
    const int reps = 3;
    auto time_layer = [&](const TcLayer &T, const ConvLayer &C, float &us) -> int {
        const __nv_bfloat16 *r = T.residual ? res : nullptr;
        int e = conv_tc_raw(ctx, T, in, r, T.relu, out, nw, C, st);  // warm
        if (e) return e;
        AFG_CUDA(ctx, cudaEventRecord(e0, st));
        for (int i = 0; i < reps && !e; ++i) e = conv_tc_raw(ctx, T, in, r, T.relu, out, nw, C, st);
        if (e) return e;
        AFG_CUDA(ctx, cudaEventRecord(e1, st));
        AFG_CUDA(ctx, cudaEventSynchronize(e1));
        float ms = 0.f;
        AFG_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
        us = ms * 1000.f / reps;
        return AFG_OK;
    };
    int err = AFG_OK;
    for (size_t i = 1; i < P.convs.size() && !err; ++i) {
        const ConvLayer &C = P.convs[i];
        TcLayer &L = TP.layers[i];
        // a layer with the geometry and epilogue of an earlier one takes its result
        size_t same = 0;
        for (size_t j = 1; j < i && !same; ++j) {
            const ConvLayer &D = P.convs[j];
            if (D.cin == C.cin && D.cout == C.cout && D.lin == C.lin && D.lout == C.lout && D.stride == C.stride &&
                D.k == C.k && TP.layers[j].residual == L.residual && TP.layers[j].relu == L.relu)
                same = j;
        }
        if (same) {
            const TcLayer &S = TP.layers[same];
            build_layer(C, P.net.groups, P.net.eps, S.knobs, L);
            L.tuned = S.tuned;
            L.n_cand = S.n_cand;
            L.us_chosen = S.us_chosen;
            L.us_default = S.us_default;
            continue;
        }
        std::vector<TileKnobs> cands;
        tile_candidates(C, P.net.groups, P.net.eps, cands);
        const TileKnobs dflt = default_knobs(C, P.net.groups, P.net.eps);
        if (std::find(cands.begin(), cands.end(), dflt) == cands.end()) cands.push_back(dflt);
        float best = 0.f, t_dflt = 0.f;
        TileKnobs best_k = dflt;
        for (const TileKnobs &k : cands) {
            TcLayer T = L;
            if (!build_layer(C, P.net.groups, P.net.eps, k, T)) continue;
            float us = 0.f;
            err = time_layer(T, C, us);
            if (err) break;
            if (k == dflt) t_dflt = us;
            if (best == 0.f || us < best) {
                best = us;
                best_k = k;
            }
        }
        if (err) break;
        build_layer(C, P.net.groups, P.net.eps, best_k, L);
        L.tuned = 1;
        L.n_cand = (int)cands.size();
        L.us_chosen = best;
        L.us_default = t_dflt;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err) return err;
    AFG_CUDA(ctx, cudaStreamSynchronize(st));
    int flag = 0;
    AFG_CUDA(ctx, cudaMemcpy(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        AFG_CUDA(ctx, cudaMemset(ctx->d_err, 0, sizeof(int)));
        return afg_fail(ctx, AFG_ERR_TIMEOUT, "autotune: a bounded device-side wait gave up");
    }
    return AFG_OK;
}

static void tile_record(const ConvLayer &C, const TcLayer &L, int layer, const TileKnobs &k, afg_tile &t) {
    memset(&t, 0, sizeof t);
    t.layer = layer;
    t.cin = C.cin;
    t.cout = C.cout;
    t.lin = C.lin;
    t.lout = C.lout;
    t.stride = C.stride;
    t.taps = C.k;
    t.residual = L.residual;
    t.orient = k.orient;
    t.wpc = k.wpc;
    t.kb = k.orient == 0 ? C.cin : k.KB;
    t.stages = k.NB;
    t.acc_bufs = k.nacc;
}

int net_tc_tiles_get(afg_ctx *ctx, afg_tile *out, int cap, int *n_out) {
    if (!ctx->tcplan) return afg_fail(ctx, AFG_ERR_UNSUPPORTED, "tiles: no per-layer tensor-core plan");
    const NetPlan &P = ctx->plan;
    const TcPlan &TP = *ctx->tcplan;
    int n = 0;
    for (size_t i = 1; i < P.convs.size(); ++i, ++n) {
        if (n >= cap) continue;
        const TcLayer &L = TP.layers[i];
        tile_record(P.convs[i], L, (int)i, L.knobs, out[n]);
        out[n].tuned = L.tuned;
        out[n].n_candidates = L.n_cand;
        out[n].us_chosen = L.us_chosen;
        out[n].us_default = L.us_default;
    }
    *n_out = n;
    return AFG_OK;
}

int net_tc_tile_candidates(afg_ctx *ctx, int layer, afg_tile *out, int cap, int *n_out) {
    if (!ctx->tcplan) return afg_fail(ctx, AFG_ERR_UNSUPPORTED, "tiles: no per-layer tensor-core plan");
    const NetPlan &P = ctx->plan;
    if (layer < 1 || layer >= (int)P.convs.size()) return afg_fail(ctx, AFG_ERR_ARG, "tiles: layer out of range");
    std::vector<TileKnobs> cands;
    tile_candidates(P.convs[layer], P.net.groups, P.net.eps, cands);
    int n = 0;
    for (const TileKnobs &k : cands) {
        if (n < cap) tile_record(P.convs[layer], ctx->tcplan->layers[layer], layer, k, out[n]);
        ++n;
    }
    *n_out = n;
    return AFG_OK;
}

int net_tc_tiles_set(afg_ctx *ctx, const afg_tile *in, int n) {
    if (!ctx->tcplan) return afg_fail(ctx, AFG_ERR_UNSUPPORTED, "tiles: no per-layer tensor-core plan");
    const NetPlan &P = ctx->plan;
    TcPlan &TP = *ctx->tcplan;
    std::vector<TcLayer> next = TP.layers;
    for (int j = 0; j < n; ++j) {
        const afg_tile &t = in[j];
        if (t.layer < 1 || t.layer >= (int)P.convs.size())
            return afg_fail(ctx, AFG_ERR_ARG, "tiles_set: entry %d: layer %d out of range", j, t.layer);
        const ConvLayer &C = P.convs[t.layer];
        TileKnobs k;
        k.orient = t.orient;
        k.wpc = t.wpc;
        k.KB = t.kb;
        k.NB = t.stages;
        k.nacc = t.acc_bufs;
        if ((k.orient != 0 && k.orient != 1) || (k.orient == 0 && k.KB != C.cin) ||
            !build_layer(C, P.net.groups, P.net.eps, k, next[t.layer]))
            return afg_fail(ctx, AFG_ERR_ARG, "tiles_set: entry %d: knobs do not fit layer %d", j, t.layer);
        next[t.layer].tuned = t.tuned;
        next[t.layer].n_cand = t.n_candidates;
        next[t.layer].us_chosen = t.us_chosen;
        next[t.layer].us_default = t.us_default;
    }
    TP.layers = next;
    return AFG_OK;
}

// Full-network BF16 forward over sliding windows (stem in FP32 SIMT, every
// other convolution on tcgen05).
int launch_infer_bf16_full(afg_ctx *ctx, const float *y, int64_t n_y, int64_t y_stride, int64_t first,
                           int64_t stride, int64_t n_win, int64_t shift, float *logits, cudaStream_t st) {
    const NetPlan &P = ctx->plan;
    const TcPlan &TP = *ctx->tcplan;
    const ConvLayer &S = P.convs[0];
    const int64_t per_win16 = P.max_act_per_window * 2;
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(n_win, 8192));
    __nv_bfloat16 *bA = nullptr, *bB = nullptr, *bC = nullptr, *bD = nullptr;
    int rc = afg_ws_reserve(ctx, WS_ACT0, (size_t)(chunk * per_win16), (void **)&bA);
    if (!rc) rc = afg_ws_reserve(ctx, WS_ACT1, (size_t)(chunk * per_win16), (void **)&bB);
    if (!rc) rc = afg_ws_reserve(ctx, WS_ACT2, (size_t)(chunk * per_win16), (void **)&bC);
    if (!rc) rc = afg_ws_reserve(ctx, WS_ACT3, (size_t)(chunk * per_win16), (void **)&bD);
    if (rc) return rc;
    const int W = ctx->cfg.win_len;
    const int pad = S.k / 2;
    const size_t stem_smem = (size_t)(2 * (W + 2 * pad) + 4 * S.cout + (STEM_T / 32 + 1) * STEM_NMOM) * sizeof(float);
    for (int64_t w0 = 0; w0 < n_win; w0 += chunk) {
        const int nw = (int)std::min<int64_t>(chunk, n_win - w0);
        {
            const double fl = 2.0 * nw * (double)S.lout * S.cout * 2.0 * S.k;
            const double by = (double)nw * (2.0 * W * 4.0 + 2.0 * (P.l_after_stem + 2) * S.cout);
            KScope ks(ctx, st, KK_STEM, fl, by);
            if (stem_tc_fits(ctx)) {
                const size_t sm_tc = stem_tc_smem(W, S.k, S.lout).total;
                const int cg = S.cout / P.net.groups;
#define AFG_STEM_TC(CGV)                                                                                         \
    k_stem_tc<CGV><<<nw, STC_T, sm_tc, st>>>(y, n_y, y_stride, first, stride, shift, w0, S.wt, S.gamma, S.beta, \
                                             S.k, S.stride, W, S.lout, P.net.stem_pool, P.net.eps, ctx->d_err, bA)
                switch (cg) {
                    case 2: AFG_STEM_TC(2); break;
                    case 4: AFG_STEM_TC(4); break;
                    case 8: AFG_STEM_TC(8); break;
                    case 16: AFG_STEM_TC(16); break;
                    default: AFG_STEM_TC(32); break;
                }
#undef AFG_STEM_TC
            } else {
                k_stem_bf16<<<nw, STEM_T, stem_smem, st>>>(y, n_y, y_stride, first, stride, shift, w0, S.wt, S.gamma,
                                                           S.beta, S.cout, S.k, S.stride, W, S.lout, P.net.stem_pool,
                                                           P.net.groups, P.net.eps, bA);
            }
        }
        AFG_LAUNCH_CHECK(ctx, "stem");
        __nv_bfloat16 *A = bA, *Cb = bC, *B = bB, *D = bD;
        for (const BlockPlan &bp : P.blocks) {
            const ConvLayer &c1 = P.convs[bp.c1], &c2 = P.convs[bp.c2];
            int e = conv_tc(ctx, TP.layers[bp.c1], A, nullptr, 1, B, nw, c1, st);
            const __nv_bfloat16 *res = A;
            if (!e && bp.sc >= 0) {
                e = conv_tc(ctx, TP.layers[bp.sc], A, nullptr, 0, D, nw, P.convs[bp.sc], st);
                res = D;
            }
            if (!e) e = conv_tc(ctx, TP.layers[bp.c2], B, res, 1, Cb, nw, c2, st);
            if (e) return e;
            std::swap(A, Cb);
        }
        {
            KScope ks(ctx, st, KK_HEAD, 2.0 * nw * P.l_last * P.c_last, 2.0 * nw * (double)P.l_last * P.c_last);
            k_head_bf16<<<nw, 256, 0, st>>>(A, P.l_last, P.c_last, P.fc_w, P.fc_b, logits, w0);
        }
        AFG_LAUNCH_CHECK(ctx, "k_head_bf16");
    }
    return AFG_OK;
}
