// Check of the library's bounded device-side waits (failure detection).
//
// The tensor-core kernels wait on mbarriers for their MMAs and bulk copies
// with tc::mbar_wait, which gives up after a time limit; the kernel then
// records the failure in the context's device flag, leaves its work early,
// and afg_sync reports AFG_ERR_TIMEOUT.  Making one of those waits run out
// would need a copy or an MMA that never completes.  Instead this kernel
// waits, through the same helper and the same flag, on an mbarrier that
// nothing ever arrives on: nothing is in flight, so the wait ends only by
// its limit, and the kernel then exits normally.
#include "afg_internal.cuh"
#include "tc_ptx.cuh"

namespace {

__global__ void k_wait_check(uint64_t limit_ns, int *err, unsigned long long *waited_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);  // one arrival expected, and none will come
        tc::fence_mbar_init();
    }
    __syncthreads();
    const uint64_t t0 = tc::globaltimer_ns();
    const bool ok = tc::mbar_wait(&bar, 0, limit_ns);
    const uint64_t t1 = tc::globaltimer_ns();
    if (threadIdx.x == 0) {
        if (!ok) atomicExch(err, 1);
        waited_ns[blockIdx.x] = (unsigned long long)(t1 - t0);
    }
}

}  // namespace

extern "C" int afg_wait_check(afg_ctx *ctx, int64_t limit_ns, int32_t n_blocks, int64_t *waited_ns, void *stream) {
    if (!ctx) return AFG_ERR_ARG;
    ctx->err.clear();
    if (limit_ns < 0 || limit_ns > 10000000000LL || n_blocks < 1 || n_blocks > 1024 || !waited_ns)
        return afg_fail(ctx, AFG_ERR_ARG, "wait_check: limit_ns in [0, 1e10], 1 <= n_blocks <= 1024, waited_ns set");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    k_wait_check<<<n_blocks, 128, 0, st>>>((uint64_t)limit_ns, ctx->d_err,
                                           reinterpret_cast<unsigned long long *>(waited_ns));
    AFG_LAUNCH_CHECK(ctx, "k_wait_check");
    return AFG_OK;
}
