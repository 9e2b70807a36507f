// Launch accounting behind afg_profile_enable / afg_profile_read.
#include <string.h>

#include "afg_internal.cuh"

const char *const kKernelNames[KK_COUNT] = {
    "twiddles", "welch_periodogram", "welch_mean", "filter_build_fp64", "whiten_overlap_save",
    "stem_conv", "groupnorm", "conv_gemm_fp32_simt", "pool_linear_head", "integrate", "triggers",
    "conv_gemm_bf16_tcgen05", "resnet_tiny_fused_bf16_tcgen05", "stream_scatter", "to_bf16",
    "far_sort_rank", "resample_decimate",
};

static cudaEvent_t take_event(Prof &p) {
    if (p.pool_used == p.pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        p.pool.push_back(e);
    }
    return p.pool[p.pool_used++];
}

KScope::KScope(afg_ctx *c, cudaStream_t s, int k, double flops, double bytes) : ctx(c), st(s), kind(k) {
    Prof &p = ctx->prof;
    p.launches[k] += 1;
    p.flops[k] += flops;
    p.bytes[k] += bytes;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    // no event timing while a stream is being captured into a graph
    if (p.on && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
        e0 = take_event(p);
        if (e0) cudaEventRecord(e0, st);
    }
}

KScope::~KScope() {
    Prof &p = ctx->prof;
    if (p.on && e0) {
        cudaEvent_t e1 = take_event(p);
        if (e1) {
            cudaEventRecord(e1, st);
            p.recs.push_back(ProfRec{kind, e0, e1});
        }
    }
}

static void prof_reset(Prof &p) {
    p.recs.clear();
    p.pool_used = 0;
    for (int k = 0; k < KK_COUNT; ++k) {
        p.launches[k] = 0;
        p.flops[k] = 0;
        p.bytes[k] = 0;
    }
}

void prof_release(afg_ctx *ctx) {
    for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
    ctx->prof.pool.clear();
}

extern "C" int afg_profile_enable(afg_ctx *ctx, int32_t on) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    if (on) {
        cudaDeviceSynchronize();
        prof_reset(ctx->prof);
    }
    ctx->prof.on = on != 0;
    return AFG_OK;
}

extern "C" int afg_profile_read(afg_ctx *ctx, afg_kernel_stat *out, int32_t cap, int32_t *n_out) {
    if (!ctx || !n_out || (cap > 0 && !out)) return AFG_ERR_ARG;
    ctx->err.clear();
    AFG_CUDA(ctx, cudaDeviceSynchronize());
    double ms[KK_COUNT] = {};
    int64_t timed[KK_COUNT] = {};
    for (const ProfRec &r : ctx->prof.recs) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.e0, r.e1) == cudaSuccess) {
            ms[r.kind] += t;
            timed[r.kind] += 1;
        }
    }
    cudaGetLastError();
    int n = 0;
    for (int k = 0; k < KK_COUNT; ++k) {
        if (ctx->prof.launches[k] == 0) continue;
        if (n < cap) {
            afg_kernel_stat &s = out[n];
            memset(&s, 0, sizeof s);
            strncpy(s.name, kKernelNames[k], sizeof s.name - 1);
            s.launches = ctx->prof.launches[k];
            s.timed = timed[k];
            s.total_ms = ms[k];
            s.algo_flops = ctx->prof.flops[k];
            s.algo_bytes = ctx->prof.bytes[k];
        }
        ++n;
    }
    *n_out = n;
    prof_reset(ctx->prof);
    return AFG_OK;
}
