// Self-test of the bounded-wait protocol that the tensor-core and tensor-copy kernels use for their
// mbarrier waits: every thread polls mbarrier.try_wait at most `limit` times, the block decides
// together (__syncthreads_or) whether the wait gave up, records that in a device flag and returns
// normally; the host reads the flag after synchronising and reports CS_ERR_TIMEOUT.  With
// arrive = 0 nothing ever arrives on the barrier, so the wait must give up on its own and the
// context stays usable (no trap, no fault, no endless loop).
#include "cs_internal.cuh"

namespace cs {

__device__ int g_wait_selftest_error = 0;

__global__ void wait_selftest_kernel(int arrive, long long limit) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t addr = (uint32_t)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(1u));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (arrive && threadIdx.x == 0)
        asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(addr) : "memory");
    long long spins = 0;
    uint32_t done = 0;
    while (!done) {
        asm volatile(
            "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\nselp.b32 %0, 1, 0, P1;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(0u)
            : "memory");
        if (!done && ++spins > limit) break;
    }
    if (__syncthreads_or(!done) && threadIdx.x == 0) atomicExch(&g_wait_selftest_error, 1);
}

}  // namespace cs

using namespace cs;

extern "C" cs_status cs_wait_selftest(int arrive, int64_t limit, void* stream) {
    clear_error();
    CS_REQUIRE(limit >= 1 && limit <= (1ll << 24), CS_ERR_INVALID_ARG, "poll limit must be in [1, 2^24]");
    cudaStream_t st = (cudaStream_t)stream;
    wait_selftest_kernel<<<1, 128, 0, st>>>(arrive, (long long)limit);
    CS_LAUNCH_CHECK();
    CS_TRY_CUDA(cudaStreamSynchronize(st));
    int v = 0;
    CS_TRY_CUDA(cudaMemcpyFromSymbol(&v, g_wait_selftest_error, sizeof(int)));
    if (v) {
        const int zero = 0;
        CS_TRY_CUDA(cudaMemcpyToSymbol(g_wait_selftest_error, &zero, sizeof(int)));
        set_error("bounded mbarrier wait gave up after %lld polls", (long long)limit);
        return CS_ERR_TIMEOUT;
    }
    return CS_OK;
}
