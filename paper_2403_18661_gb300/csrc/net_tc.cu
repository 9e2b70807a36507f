// 1D ResNet on tcgen05 tensor cores (BF16 operands, FP32 accumulation in TMEM).
#include "afg_internal.cuh"

int launch_infer_bf16(afg_ctx *ctx, const float *, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, float *,
                      cudaStream_t) {
    return afg_fail(ctx, AFG_ERR_UNSUPPORTED, "infer_windows: the BF16 tensor-core path is not built yet");
}
