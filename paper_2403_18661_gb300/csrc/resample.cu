// Integer-factor decimation of raw strain to the analysis rate (Sec. IV.A: the
// strain is resampled to 2048 Hz; Table III: the edge it corrupts costs 1 s of
// latency).  Anti-aliasing FIR: a Kaiser-windowed sinc (beta = 5) with
// half-length L = 10 M taps and cutoff at the output Nyquist frequency,
// normalised to unit gain at DC (the design of the widely used polyphase
// resampler of Harris, "Multirate Signal Processing", with the defaults of
// scipy.signal.resample_poly).  Output j is the filter centred on input
// sample c_j = (j0 + j) M, j0 = ceil(L / M), for every centre whose taps lie
// inside the input ("valid" mode):
//   y[j] = sum_{k=-L..L} h_k x[c_j + k]
// Only the kept outputs are computed (polyphase).  Each block stages its input
// span in shared memory de-interleaved by phase (sample i at [i mod M][i / M]),
// so that the lanes of a warp, which compute consecutive outputs, read
// consecutive words for every tap.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "afg_internal.cuh"

namespace {

// taps of the compiled factors 2, 4, 8, 16 (41 + 81 + 161 + 321 values), written once per process
__constant__ float c_taps[604];
__host__ __device__ constexpr int c_taps_off(int M) { return M == 2 ? 0 : M == 4 ? 41 : M == 8 ? 122 : 283; }

constexpr int RSMP_T = 256;
constexpr int RSMP_OUT = 4 * RSMP_T;  // outputs per block
constexpr int RSMP_Q = 21;            // taps per phase at L = 10 M (phase 0: 21, others 20)
constexpr int RSMP_WIN = 24;          // window of one thread per phase: 4 outputs + 20, rounded to float4
// words per phase row: a multiple of 4 (16-byte rows) that is 4 mod 8, so the rows p and p + 4
// written from one 16-byte load of a warp fall in different shared-memory banks
constexpr int RSMP_PITCH = RSMP_OUT + RSMP_WIN + 4;
static_assert(RSMP_PITCH % 8 == 4, "phase-row layout");

// MF: the factor at compile time (0: runtime M).  Thread t computes the 4 consecutive
// outputs 4t .. 4t + 3 of its block's tile.  For each phase p it holds a sliding window of
// 4 + 20 consecutive samples of that phase's row in registers (six 16-byte shared loads),
// and the tap h[q M + p] multiplies window entries q .. q + 3.
template <int MF>
__global__ void __launch_bounds__(RSMP_T) k_decimate(const float *__restrict__ x, int64_t x_stride, int64_t n_in,
                                                     const float *__restrict__ taps, int M_rt, int L, int64_t j0,
                                                     int64_t n_out, float *__restrict__ y, int64_t y_stride,
                                                     int vec_store, int vec_load) {
    extern __shared__ __align__(16) float sm[];
    const int M = MF ? MF : M_rt;
    const int ntap = 2 * L + 1;                     // L = 10 M: 21 taps in phase 0, 20 in the others
    const int pitch = RSMP_PITCH;
    float *h = sm;                                  // [ntap], padded to a multiple of 4
    float *xs = sm + ((ntap + 3) / 4) * 4;          // [M][pitch]
    const float *xd = x + (int64_t)blockIdx.y * x_stride;
    float *yd = y + (int64_t)blockIdx.y * y_stride;
    const int64_t o0 = (int64_t)blockIdx.x * RSMP_OUT;
    const int64_t first = (j0 + o0) * M - L;  // input sample of local index 0 (>= 0 by the choice of j0)
    const int span = M * pitch;               // staged samples (zero past the input)
    if (!MF)
        for (int k = threadIdx.x; k < ntap; k += RSMP_T) h[k] = taps[k];
    // stage the span de-interleaved by phase: local sample li at [li % M][li / M]
    if (MF >= 4 && vec_load && first + span <= n_in) {
        // 16-byte loads (first is a multiple of 4: x rows 16-byte aligned), 4 phases per load;
        // all of a thread's loads are issued before the first shared store
        constexpr int NV = ((MF ? MF : 1) * RSMP_PITCH / 4 + RSMP_T - 1) / RSMP_T;
        const float4 *x4 = reinterpret_cast<const float4 *>(xd + first);
        float4 u[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const int v = threadIdx.x + k * RSMP_T;
            u[k] = v < span / 4 ? __ldg(x4 + v) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const int v = threadIdx.x + k * RSMP_T;
            if (v < span / 4) {
                const int li = 4 * v, p = li & ((MF ? MF : 1) - 1), m = li / (MF ? MF : 1);
                xs[p * pitch + m] = u[k].x;
                xs[(p + 1) * pitch + m] = u[k].y;
                xs[(p + 2) * pitch + m] = u[k].z;
                xs[(p + 3) * pitch + m] = u[k].w;
            }
        }
    } else {
        for (int li = threadIdx.x; li < span; li += RSMP_T) {
            const int64_t i = first + li;
            const int p = MF ? (li & (MF - 1)) : li % M;
            const int m = MF ? (li / MF) : li / M;
            xs[p * pitch + m] = (i < n_in) ? __ldg(xd + i) : 0.f;
        }
    }
    __syncthreads();
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const int base = 4 * threadIdx.x;
    if (MF) {  // every tap a compile-time constant-bank operand
#pragma unroll
        for (int p = 0; p < (MF ? MF : 1); ++p) {
            float win[RSMP_WIN];
            const float4 *row = reinterpret_cast<const float4 *>(xs + p * pitch + base);
#pragma unroll
            for (int v = 0; v < RSMP_WIN / 4; ++v) {
                const float4 u = row[v];
                win[4 * v] = u.x;
                win[4 * v + 1] = u.y;
                win[4 * v + 2] = u.z;
                win[4 * v + 3] = u.w;
            }
#pragma unroll
            for (int q = 0; q < RSMP_Q; ++q) {
                const int k = q * (MF ? MF : 1) + p;
                if (k < 20 * (MF ? MF : 1) + 1) {
                    const float hk = c_taps[c_taps_off(MF) + k];
#pragma unroll
                    for (int r = 0; r < 4; ++r) acc[r] = fmaf(hk, win[q + r], acc[r]);
                }
            }
        }
    } else
#pragma unroll 1
    for (int p = 0; p < M; ++p) {
        float win[RSMP_WIN];
        const float4 *row = reinterpret_cast<const float4 *>(xs + p * pitch + base);
#pragma unroll
        for (int v = 0; v < RSMP_WIN / 4; ++v) {
            const float4 u = row[v];
            win[4 * v] = u.x;
            win[4 * v + 1] = u.y;
            win[4 * v + 2] = u.z;
            win[4 * v + 3] = u.w;
        }
#pragma unroll
        for (int q = 0; q < RSMP_Q; ++q) {
            const int k = q * M + p;
            const float hk = k < ntap ? h[k] : 0.f;
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[r] = fmaf(hk, win[q + r], acc[r]);
        }
    }
    const int64_t o = o0 + base;
    if (vec_store && o + 3 < n_out) {  // rows 16-byte aligned (checked on the host), o a multiple of 4
        *reinterpret_cast<float4 *>(yd + o) = make_float4(acc[0], acc[1], acc[2], acc[3]);
    } else {
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (o + r < n_out) yd[o + r] = acc[r];
    }
}

// modified Bessel function of the first kind, order 0, by its power series
double bessel_i0(double x) {
    double sum = 1.0, term = 1.0;
    const double q = 0.25 * x * x;
    for (int k = 1; k < 500; ++k) {
        term *= q / ((double)k * (double)k);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

}  // namespace

// Taps of the decimation filter for factor M (host, double precision).
void resample_taps(int M, std::vector<double> &h) {
    const int L = 10 * M, N = 2 * L + 1;
    const double beta = 5.0, fc = 1.0 / M, pi = 3.14159265358979323846;
    h.assign(N, 0.0);
    double sum = 0.0;
    const double i0b = bessel_i0(beta);
    for (int k = 0; k < N; ++k) {
        const double r = 2.0 * k / (N - 1) - 1.0;
        const double w = bessel_i0(beta * sqrt(std::max(0.0, 1.0 - r * r))) / i0b;
        const double t = fc * (k - L);
        const double s = t == 0.0 ? 1.0 : sin(pi * t) / (pi * t);
        h[k] = fc * s * w;
        sum += h[k];
    }
    for (double &v : h) v /= sum;
}

int64_t resample_count(int64_t n_in, int M, int64_t *j0_out) {
    const int L = 10 * M;
    const int64_t j0 = (L + M - 1) / M;
    if (j0_out) *j0_out = j0;
    if (n_in - 1 - L < j0 * M) return 0;
    return (n_in - 1 - L) / M - j0 + 1;
}

int launch_resample(afg_ctx *ctx, const float *x, int64_t n_in, int n_det, int64_t x_stride, int M, float *y,
                    int64_t y_stride, int64_t *n_out_host, cudaStream_t st) {
    int64_t j0 = 0;
    const int64_t n_out = resample_count(n_in, M, &j0);
    if (n_out_host) *n_out_host = n_out;
    if (n_out == 0) return AFG_OK;
    const int L = 10 * M, ntap = 2 * L + 1;
    // the taps of each factor are built once per context (the first call synchronises)
    if (!ctx->rs_taps[M]) {
        std::vector<double> hd;
        resample_taps(M, hd);
        std::vector<float> hf(hd.begin(), hd.end());
        void *d = nullptr;
        if (cudaMalloc(&d, (size_t)ntap * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return afg_fail(ctx, AFG_ERR_OOM, "resample: cudaMalloc of the taps failed");
        }
        ctx->bytes_held += (int64_t)ntap * sizeof(float);
        ctx->rs_taps[M] = static_cast<float *>(d);
        AFG_CUDA(ctx, cudaMemcpy(d, hf.data(), (size_t)ntap * sizeof(float), cudaMemcpyHostToDevice));
    }
    const float *dt = ctx->rs_taps[M];
    static std::once_flag once;
    static cudaError_t const_err = cudaSuccess;
    std::call_once(once, [] {
        std::vector<float> all(604);
        for (int f : {2, 4, 8, 16}) {
            std::vector<double> t;
            resample_taps(f, t);
            for (size_t k = 0; k < t.size(); ++k) all[c_taps_off(f) + k] = (float)t[k];
        }
        const_err = cudaMemcpyToSymbol(c_taps, all.data(), all.size() * sizeof(float));
    });
    if (const_err != cudaSuccess) return afg_cuda_fail(ctx, const_err, "resample: constant taps");
    const int pitch = RSMP_PITCH;
    const size_t smem = (size_t)(((ntap + 3) / 4) * 4 + M * pitch) * sizeof(float);
    auto kern = M == 2 ? k_decimate<2> : M == 4 ? k_decimate<4> : M == 8 ? k_decimate<8> : M == 16 ? k_decimate<16>
                                                                                                   : k_decimate<0>;
    AFG_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const dim3 grid((unsigned)((n_out + RSMP_OUT - 1) / RSMP_OUT), (unsigned)n_det);
    {
        KScope ks(ctx, st, KK_RESAMPLE, 2.0 * n_det * n_out * ntap,
                  (double)n_det * ((double)n_out * M * 4.0 + n_out * 4.0));
        const int vec = ((reinterpret_cast<uintptr_t>(y) & 15) == 0 && y_stride % 4 == 0) ? 1 : 0;
        const int vec_in = ((reinterpret_cast<uintptr_t>(x) & 15) == 0 && x_stride % 4 == 0) ? 1 : 0;
        kern<<<grid, RSMP_T, smem, st>>>(x, x_stride, n_in, dt, M, L, j0, n_out, y, y_stride, vec, vec_in);
    }
    AFG_LAUNCH_CHECK(ctx, "k_decimate");
    return AFG_OK;
}
