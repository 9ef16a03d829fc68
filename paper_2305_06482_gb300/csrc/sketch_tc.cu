// Tensor-core split-precision contraction for the sketched maps (Eq. 8, random block):
//   maps_s[s][d] = sum_j S~_S[s][j] maps_rot[V + j][d],   s < S <= 16, j < K = C - V <= 64.
//
// Viewed as a real GEMM D[r][s] = sum_j A[r][j] B[s][j] with r running over the re/im components
// of a tile of 64 voxels (M = 128), s over the sketch rows (N = 16) and j over the low-energy
// coils (K padded to a multiple of 16).  The sketch entries are BF16-exact (sketch_draw rounds
// them), the FP32 maps are split into hi = bf16(m) and lo = bf16(m - hi), and
//   D = A_hi B + A_lo B
// accumulates in FP32 in tensor memory (tcgen05.mma kind::f16, BF16 x BF16 products are exact
// in FP32), leaving a relative error of about 2^-17 per term.
//
// Per CTA (128 threads, one output row per thread): the threads convert and store their rows of
// A_hi / A_lo straight into the K-major no-swizzle canonical layout (8x16-byte core matrices,
// K-adjacent core matrices 128 B apart, M-adjacent ones 256 B apart), one elected thread issues
// the MMAs and commits them to an mbarrier, every thread waits on it (bounded), reads its TMEM
// lane with tcgen05.ld and stores the 16 results.
#include <cstdio>

#include "cs_internal.cuh"

namespace cs {

constexpr int kTcM = 128;          // output rows per tile (64 voxels x re/im)
constexpr int kTcN = 16;           // sketch rows (padded)
constexpr int kTcMaxK = 64;        // low-energy coils (padded to 16)
constexpr int kTcTileBytes = kTcM * 16 * 2;   // one 128 x 16 bf16 k-block of A: 4 KiB
constexpr int kTcBBytes = kTcN * 16 * 2;      // one 16 x 16 bf16 k-block of B: 512 B
constexpr long long kSpinLimit = 1ll << 22;   // bounded mbarrier waits (seconds at most)

__device__ int g_tc_error = 0;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (row, k) inside one K-major no-swizzle k-block (16 wide)
__device__ __forceinline__ int kmajor_off(int row, int k) {
    return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    const uint64_t lbo = 128 >> 4, sbo = 256 >> 4;
    return (uint64_t)((addr >> 4) & 0x3FFF) | (lbo << 16) | (sbo << 32) | (1ull << 46);
}

// instruction descriptor: D F32, A/B BF16, both K-major, N = 16, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ unsigned short bf16_bits_rn(float f) {
    uint32_t b = __float_as_uint(f);
    const uint32_t lsb = (b >> 16) & 1u;
    b += 0x7FFFu + lsb;
    return (unsigned short)(b >> 16);
}

__device__ __forceinline__ float bf16_to_float(unsigned short h) { return __uint_as_float((uint32_t)h << 16); }

__global__ void __launch_bounds__(128) sketch_tc_kernel(const float* __restrict__ Sk, const int* __restrict__ tsel,
                                                        const float2* __restrict__ mrot, int64_t D, int V, int K, int Sn,
                                                        float2* __restrict__ out) {
    if (tsel) Sk += (int64_t)(*tsel) * Sn * K;
    extern __shared__ __align__(1024) unsigned char tsm[];
    const int kblocks = (K + 15) / 16;
    unsigned char* a_hi = tsm;
    unsigned char* a_lo = tsm + kblocks * kTcTileBytes;
    unsigned char* b_sm = tsm + 2 * kblocks * kTcTileBytes;
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) uint64_t s_mbar;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_taddr)),
                     "r"(32u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&s_mbar)), "r"(1u));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // B: the sketch block, zero-padded to 16 x (16 kblocks), K-major
    for (int e = tid; e < kTcN * kblocks * 16; e += blockDim.x) {
        const int n = e / (kblocks * 16), k = e % (kblocks * 16);
        const float v = (n < Sn && k < K) ? Sk[n * K + k] : 0.f;
        *reinterpret_cast<unsigned short*>(b_sm + (k >> 4) * kTcBBytes + kmajor_off(n, k & 15)) = bf16_bits_rn(v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = s_taddr;
    const uint32_t mbar = smem_u32(&s_mbar);
    uint32_t phase = 0;
    bool failed = false;

    const int64_t ntiles = (D + 63) / 64;
    for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
        // ---- this thread's row of A: component (tid & 1) of voxel d0 + tid / 2 ----
        const int64_t d = tile * 64 + (tid >> 1);
        const bool dv = d < D;
        for (int k = 0; k < kblocks * 16; ++k) {
            float m = 0.f;
            if (dv && k < K) {
                const float2 v = mrot[(int64_t)(V + k) * D + d];
                m = (tid & 1) ? v.y : v.x;
            }
            const unsigned short hi = bf16_bits_rn(m);
            const unsigned short lo = bf16_bits_rn(m - bf16_to_float(hi));
            const int off = (k >> 4) * kTcTileBytes + kmajor_off(tid, k & 15);
            *reinterpret_cast<unsigned short*>(a_hi + off) = hi;
            *reinterpret_cast<unsigned short*>(a_lo + off) = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            for (int kb = 0; kb < kblocks; ++kb) {
                const uint64_t bdesc = smem_desc(smem_u32(b_sm + kb * kTcBBytes));
                const uint64_t ahd = smem_desc(smem_u32(a_hi + kb * kTcTileBytes));
                const uint64_t ald = smem_desc(smem_u32(a_lo + kb * kTcTileBytes));
                const uint32_t acc_first = kb > 0 ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
                    "l"(ahd), "l"(bdesc), "r"(kIdesc), "r"(acc_first));
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
                    "l"(ald), "l"(bdesc), "r"(kIdesc), "r"(1u));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                         : "memory");
        }
        // ---- bounded wait for the MMAs of this tile ----
        long long spins = 0;
        uint32_t done = 0;
        while (!done) {
            asm volatile(
                "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\nselp.b32 %0, 1, 0, P1;\n}\n"
                : "=r"(done)
                : "r"(mbar), "r"(phase)
                : "memory");
            if (!done && ++spins > kSpinLimit) break;
        }
        // one decision for the whole CTA: give up together if any thread timed out
        if (__syncthreads_or(!done)) {
            if (tid == 0) atomicExch(&g_tc_error, 1);
            // drain: wait once more (bounded) for the MMAs in flight before the tensor memory is freed
            for (long long k = 0; !done && k < kSpinLimit; ++k)
                asm volatile(
                    "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\nselp.b32 %0, 1, 0, P1;\n}\n"
                    : "=r"(done)
                    : "r"(mbar), "r"(phase)
                    : "memory");
            failed = true;
            break;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // ---- TMEM -> registers: lane = output row, 16 columns = sketch rows ----
        uint32_t r[16];
        const uint32_t lane_addr = taddr + ((uint32_t)(warp * 32) << 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(lane_addr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (dv) {
            float* o = reinterpret_cast<float*>(out);
#pragma unroll
            for (int s = 0; s < kTcN; ++s)
                if (s < Sn) o[2 * ((int64_t)s * D + d) + (tid & 1)] = __uint_as_float(r[s]);
        }
        // the next tile overwrites A and D only after every thread has read its results
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(32u));
    }
}

cs_status tc_init_attrs() {
    CS_TRY_CUDA(cudaFuncSetAttribute(sketch_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(2 * 4 * kTcTileBytes + 4 * kTcBBytes)));
    return CS_OK;
}

static int sm_count_tc() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 148;
}

cs_status sketched_maps_bf16split(const float* S, const int* tsel, const float2* mrot, int64_t D, int C, int V, int Sn,
                                  float2* out, cudaStream_t st) {
    const int K = C - V;
    CS_REQUIRE(Sn <= kTcN && K <= kTcMaxK, CS_ERR_UNSUPPORTED_SIZE,
               "CS_PREC_BF16_SPLIT supports S <= %d and C - V <= %d", kTcN, kTcMaxK);
    if (K <= 0) return CS_ERR_INVALID_ARG;
    const int kblocks = (K + 15) / 16;
    const size_t sm = (size_t)2 * kblocks * kTcTileBytes + (size_t)kblocks * kTcBBytes;
    const int64_t tiles = (D + 63) / 64;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sm_count_tc() * 8));
    sketch_tc_kernel<<<grid, 128, sm, st>>>(S, tsel, mrot, D, V, K, Sn, out);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

// reads and clears the tensor-core timeout flag (after the caller synchronised the stream)
cs_status tc_check_and_clear() {
    int v = 0;
    CS_TRY_CUDA(cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int)));
    if (v) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(int));
        set_error("a tensor-core contraction gave up waiting for its MMAs (bounded wait)");
        return CS_ERR_TIMEOUT;
    }
    return CS_OK;
}

}  // namespace cs
