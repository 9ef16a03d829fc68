// Building blocks of the learned warm start: a 3D U-Net that maps (x^t, d) of a sketched
// sub-problem (Eq. 9-10) to a correction of x^t.  Activations are voxel-major with channels
// fastest ([nz][ny][nx][C], FP32); 3x3x3 convolutions (zero padding 1, stride 1) run as BF16
// implicit GEMMs on the tensor cores with FP32 accumulation in tensor memory:
//   forward:  out[v][co] = b[co] + sum_{tap, ci} in[v + off(tap)][ci] w[co][tap][ci]
//             (GEMM M = 128 voxels, N = C_out padded to 16/32/64, K = 27 C_in padded to 16)
//   data gradient: the same kernel with the taps flipped and the weights transposed,
//             gin[v][ci] = sum_{tap, co} gout[v - off(tap)][co] w[co][tap][ci]
//   weight gradient: gw[co][tap][ci] = sum_v gout[v][co] in[v + off(tap)][ci]
//             (GEMM M = 27 C_in rows of the transposed im2col, N = C_out padded, K = voxels)
// Max-pools, stride-2 transposed convolutions, channel slices (skip concatenation), the 1x1x1
// output layer, ReLU masks, the loss and Adam run on CUDA cores.
#include <cstdio>

#include "cs_internal.cuh"

namespace cs {

constexpr int kNnM = 128;
constexpr int kNnChunk = 8;                 // k-blocks (16 wide) staged per MMA batch
constexpr int kNnABytes = kNnM * 16 * 2;    // one 128 x 16 bf16 k-block
constexpr long long kNnSpin = 1ll << 22;

__device__ int g_nn_error = 0;

__device__ __forceinline__ uint32_t nn_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ int nn_kmajor_off(int row, int k) {
    return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t nn_desc(uint32_t addr) {
    const uint64_t lbo = 128 >> 4, sbo = 256 >> 4;
    return (uint64_t)((addr >> 4) & 0x3FFF) | (lbo << 16) | (sbo << 32) | (1ull << 46);
}

__device__ __forceinline__ unsigned short nn_bf16(float f) {
    uint32_t b = __float_as_uint(f);
    b += 0x7FFFu + ((b >> 16) & 1u);
    return (unsigned short)(b >> 16);
}

// two floats rounded to the nearest BF16 (ties to even) and packed, lo in the low half
__device__ __forceinline__ uint32_t nn_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

template <int NPAD>
__global__ void __launch_bounds__(128) conv3_tc_kernel(const float* __restrict__ in, int nz, int ny, int nx, int cin,
                                                       const unsigned short* __restrict__ wpk, int kpad, int nout,
                                                       const float* __restrict__ bias, int relu, int flip,
                                                       float* __restrict__ out, int ldo, int coff) {
    constexpr int kBBytes = NPAD * 16 * 2;
    constexpr uint32_t kCols = NPAD < 32 ? 32u : (uint32_t)NPAD;
    constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NPAD >> 3) << 17) | ((uint32_t)(kNnM >> 4) << 24);
    extern __shared__ __align__(1024) unsigned char nsm[];
    unsigned char* a_sm = nsm;
    unsigned char* b_sm = nsm + kNnChunk * kNnABytes;
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) uint64_t s_mbar;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(nn_smem_u32(&s_taddr)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(nn_smem_u32(&s_mbar)), "r"(1u));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = s_taddr, mbar = nn_smem_u32(&s_mbar);
    uint32_t phase = 0;
    const int64_t nvox = (int64_t)nz * ny * nx;
    const int ktot = 27 * cin;
    const int kblocks = kpad / 16;
    const int64_t ntiles = (nvox + kNnM - 1) / kNnM;
    const int sgn = flip ? -1 : 1;
    const bool vec4 = (cin & 3) == 0 && ((reinterpret_cast<uintptr_t>(in) & 15) == 0);
    bool failed = false;
    for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
        const int64_t v = tile * kNnM + tid;
        const bool vv = v < nvox;
        int x = 0, y = 0, z = 0;
        if (vv) {
            x = (int)(v % nx);
            y = (int)((v / nx) % ny);
            z = (int)(v / ((int64_t)nx * ny));
        }
        for (int c0 = 0; c0 < kblocks; c0 += kNnChunk) {
            const int nkb = min(kNnChunk, kblocks - c0);
            // A: this thread's voxel row of the implicit im2col matrix.  With cin a multiple of 4
            // every group of 4 consecutive k is 4 channels of one tap: one float4 load each, and
            // 8 consecutive k are one 16-byte row of a core matrix.
            for (int kb = 0; kb < nkb; ++kb) {
                unsigned char* arow = a_sm + kb * kNnABytes + nn_kmajor_off(tid, 0);
                if (vec4) {
                    uint32_t pk[8];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int k = (c0 + kb) * 16 + 4 * q;
                        float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (vv && k < ktot) {
                            const int tap = k / cin, ci = k - tap * cin;
                            const int zz = z + sgn * (tap / 9 - 1), yy = y + sgn * ((tap / 3) % 3 - 1),
                                      xx = x + sgn * (tap % 3 - 1);
                            if (zz >= 0 && zz < nz && yy >= 0 && yy < ny && xx >= 0 && xx < nx)
                                val = *reinterpret_cast<const float4*>(in + (((int64_t)zz * ny + yy) * nx + xx) * cin + ci);
                        }
                        pk[2 * q] = (uint32_t)nn_bf16(val.x) | ((uint32_t)nn_bf16(val.y) << 16);
                        pk[2 * q + 1] = (uint32_t)nn_bf16(val.z) | ((uint32_t)nn_bf16(val.w) << 16);
                    }
                    *reinterpret_cast<uint4*>(arow) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    *reinterpret_cast<uint4*>(arow + 128) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                } else {
                    for (int kk = 0; kk < 16; ++kk) {
                        const int k = (c0 + kb) * 16 + kk;
                        float val = 0.f;
                        if (vv && k < ktot) {
                            const int tap = k / cin, ci = k - tap * cin;
                            const int zz = z + sgn * (tap / 9 - 1), yy = y + sgn * ((tap / 3) % 3 - 1),
                                      xx = x + sgn * (tap % 3 - 1);
                            if (zz >= 0 && zz < nz && yy >= 0 && yy < ny && xx >= 0 && xx < nx)
                                val = in[(((int64_t)zz * ny + yy) * nx + xx) * cin + ci];
                        }
                        *reinterpret_cast<unsigned short*>(a_sm + kb * kNnABytes + nn_kmajor_off(tid, kk)) = nn_bf16(val);
                    }
                }
            }
            // B: the packed BF16 weights of these k-blocks, 8 k (16 bytes) per copy
            for (int e = tid; e < NPAD * nkb * 2; e += blockDim.x) {
                const int n = e / (nkb * 2), kr = e % (nkb * 2);
                const int kb = kr >> 1, h = kr & 1;
                *reinterpret_cast<uint4*>(b_sm + kb * kBBytes + nn_kmajor_off(n, 8 * h)) =
                    *reinterpret_cast<const uint4*>(wpk + (int64_t)n * kpad + (c0 + kb) * 16 + 8 * h);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (tid == 0) {
                for (int kb = 0; kb < nkb; ++kb) {
                    const uint64_t ad = nn_desc(nn_smem_u32(a_sm + kb * kNnABytes));
                    const uint64_t bd = nn_desc(nn_smem_u32(b_sm + kb * kBBytes));
                    const uint32_t acc = (c0 + kb > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
                        "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                             : "memory");
            }
            long long spins = 0;
            uint32_t done = 0;
            while (!done) {
                asm volatile(
                    "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\nselp.b32 %0, 1, 0, P1;\n}\n"
                    : "=r"(done)
                    : "r"(mbar), "r"(phase)
                    : "memory");
                if (!done && ++spins > kNnSpin) break;
            }
            if (__syncthreads_or(!done)) {
                if (tid == 0) atomicExch(&g_nn_error, 1);
                // drain: wait once more (bounded) for the MMAs in flight before the tensor memory is freed
                for (long long k = 0; !done && k < kNnSpin; ++k)
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
        }
        if (failed) break;
        // epilogue: TMEM lane = voxel, columns = output channels
#pragma unroll
        for (int j = 0; j < NPAD / 16; ++j) {
            uint32_t r[16];
            const uint32_t a = taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * 16);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(a));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (vv) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int n = j * 16 + q;
                    if (n < nout) {
                        float val = __uint_as_float(r[q]) + (bias ? bias[n] : 0.f);
                        if (relu) val = fmaxf(val, 0.f);
                        out[v * ldo + coff + n] = val;
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kCols));
}

// ---- halo-brick implicit GEMM (cin a multiple of 4) ----
// A CTA tile is TZ planes x 8 rows x 14 columns of output voxels.  The input brick around it,
// (TZ + 2) x 10 x 16 voxels, is staged once per 16 input channels as BF16 in two 8-channel slabs
// whose voxels sit 16 bytes apart, x fastest, rows 256 bytes apart.  Then the 128 rows
// (8 rows x 16 columns) of one plane, shifted by a tap (dz, dy, dx), are one K-major operand
// with 8-row core-matrix groups 128 bytes apart (SBO) and the two slabs as its two K halves
// (LBO = slab size): each tap is one MMA straight from the brick, no im2col copy.  Columns 0
// and 15 of each row see a neighbouring row through the shift and are discarded, so 14 of 16
// columns are outputs.  Weights of all 27 taps for the 16 channels are staged beside the brick.
constexpr int kBrX = 16, kBrY = 10, kTileX = 14, kTileY = 8, kBrTZ = 4;
constexpr int kBrGuard = 128;    // shifted rows reach 16 bytes before the brick

template <int NPAD, int TZ>
struct BrickCfg {
    static constexpr int kSlab = (TZ + 2) * kBrY * kBrX * 16;     // bytes of one 8-channel slab
    static constexpr int kWTap = NPAD * 16 * 2;                   // bytes of one tap's B operand
    static constexpr int kSmem = kBrGuard + 2 * kSlab + 27 * kWTap + 128;
    static constexpr uint32_t kColsNeed = (uint32_t)(TZ * NPAD);
    static constexpr uint32_t kCols = kColsNeed <= 32 ? 32u : kColsNeed <= 64 ? 64u : kColsNeed <= 128 ? 128u
                                      : kColsNeed <= 256 ? 256u : 512u;
};

__device__ __forceinline__ uint64_t nn_desc2(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

template <int NPAD, int TZ>
__global__ void __launch_bounds__(128, 1) conv3_brick_kernel(const float* __restrict__ in, int nz, int ny, int nx,
                                                          int cin, const unsigned short* __restrict__ wpk, int kpad,
                                                          int nout, const float* __restrict__ bias, int relu, int flip,
                                                          float* __restrict__ out, int ldo, int coff) {
    using Cfg = BrickCfg<NPAD, TZ>;
    constexpr int kSlab = Cfg::kSlab, kWTap = Cfg::kWTap;
    constexpr int kBz = TZ + 2;
    constexpr int kVox = kBz * kBrY * kBrX;
    constexpr int kItems = kVox * 4;
    constexpr int kBrBatch = 8;
    constexpr int kItemsPerThread = (kItems + 127) / 128;
    constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NPAD >> 3) << 17) | ((uint32_t)(kNnM >> 4) << 24);
    extern __shared__ __align__(1024) unsigned char nsm[];
    unsigned char* brick = nsm + kBrGuard;                 // slab 0, then slab 1
    unsigned char* wsm = brick + 2 * kSlab + 128;          // 27 taps x [NPAD][16] bf16
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) uint64_t s_mbar;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(nn_smem_u32(&s_taddr)),
                     "r"(Cfg::kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(nn_smem_u32(&s_mbar)), "r"(1u));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the guard bytes before the brick and the gap after it are read by discarded rows only;
    // clear them once so that they hold finite values
    for (int e = tid; e < kBrGuard / 4; e += blockDim.x) reinterpret_cast<uint32_t*>(nsm)[e] = 0u;
    for (int e = tid; e < 128 / 4; e += blockDim.x) reinterpret_cast<uint32_t*>(brick + 2 * kSlab)[e] = 0u;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = s_taddr, mbar = nn_smem_u32(&s_mbar);
    uint32_t phase = 0;
    const int tx = (nx + kTileX - 1) / kTileX, ty = (ny + kTileY - 1) / kTileY, tz = (nz + TZ - 1) / TZ;
    const int64_t ntiles = (int64_t)tx * ty * tz;
    const int kpairs = (cin + 15) / 16;
    const bool wvec = (cin & 15) == 0;
    const bool vec_out = ((ldo | coff) & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;
    bool failed = false;
    for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
        const int itx = (int)(tile % tx), ity = (int)((tile / tx) % ty), itz = (int)(tile / ((int64_t)tx * ty));
        const int x0 = itx * kTileX - 1, y0 = ity * kTileY - 1, z0 = itz * TZ - 1;   // brick origin
        for (int kp = 0; kp < kpairs; ++kp) {
            // input brick of channels kp*16 .. kp*16+15, zero outside the volume / channel range:
            // item i = 4 channels (q = i & 3) of brick voxel i >> 2, loaded in batches so that
            // each thread has kBrBatch loads in flight
            for (int j0 = 0; j0 < kItemsPerThread; j0 += kBrBatch) {
                float4 v[kBrBatch];
#pragma unroll
                for (int j = 0; j < kBrBatch; ++j) {
                    const int i = tid + 128 * (j0 + j);
                    v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                    const int vb = i >> 2, q = i & 3;
                    if (i < kItems && kp * 16 + 4 * q < cin) {
                        const int bx = vb % kBrX, by = (vb / kBrX) % kBrY, bz = vb / (kBrX * kBrY);
                        const int gx = x0 + bx, gy = y0 + by, gz = z0 + bz;
                        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz)
                            v[j] = *reinterpret_cast<const float4*>(in + (((int64_t)gz * ny + gy) * nx + gx) * cin + kp * 16 + 4 * q);
                    }
                }
#pragma unroll
                for (int j = 0; j < kBrBatch; ++j) {
                    const int i = tid + 128 * (j0 + j);
                    if (i < kItems) {
                        const int vb = i >> 2, q = i & 3;
                        *reinterpret_cast<uint2*>(brick + (q >> 1) * kSlab + vb * 16 + (q & 1) * 8) =
                            make_uint2((uint32_t)nn_bf16(v[j].x) | ((uint32_t)nn_bf16(v[j].y) << 16),
                                       (uint32_t)nn_bf16(v[j].z) | ((uint32_t)nn_bf16(v[j].w) << 16));
                    }
                }
            }
            // B operands of the 27 taps for these channels (tap slot t holds tap 26 - t when flipped)
            if (wvec) {
                for (int e = tid; e < 27 * NPAD * 2; e += blockDim.x) {
                    const int h = e & 1, n = (e >> 1) % NPAD, t = (e >> 1) / NPAD;
                    const int ts = flip ? 26 - t : t;
                    *reinterpret_cast<uint4*>(wsm + t * kWTap + nn_kmajor_off(n, 8 * h)) =
                        *reinterpret_cast<const uint4*>(wpk + (int64_t)n * kpad + ts * cin + kp * 16 + 8 * h);
                }
            } else {
                for (int e = tid; e < 27 * NPAD * 16; e += blockDim.x) {
                    const int c = e & 15, n = (e >> 4) % NPAD, t = (e >> 4) / NPAD;
                    const int ts = flip ? 26 - t : t;
                    const int ch = kp * 16 + c;
                    *reinterpret_cast<unsigned short*>(wsm + t * kWTap + nn_kmajor_off(n, c)) =
                        ch < cin ? wpk[(int64_t)n * kpad + ts * cin + ch] : (unsigned short)0;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (tid == 0) {
                const uint32_t b0 = nn_smem_u32(brick), w0 = nn_smem_u32(wsm);
                for (int p = 0; p < TZ; ++p) {
                    for (int t = 0; t < 27; ++t) {
                        const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
                        const uint32_t aaddr = b0 + (uint32_t)((p + dz + 1) * (kBrY * kBrX * 16) + (dy + 1) * (kBrX * 16) + dx * 16);
                        const uint64_t ad = nn_desc2(aaddr, (uint32_t)kSlab, 128u);
                        const uint64_t bd = nn_desc2(w0 + (uint32_t)(t * kWTap), 128u, 256u);
                        const uint32_t acc = (kp > 0 || t > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr + (uint32_t)(p * NPAD)),
                            "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                             : "memory");
            }
            long long spins = 0;
            uint32_t done = 0;
            while (!done) {
                asm volatile(
                    "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\nselp.b32 %0, 1, 0, P1;\n}\n"
                    : "=r"(done)
                    : "r"(mbar), "r"(phase)
                    : "memory");
                if (!done && ++spins > kNnSpin) break;
            }
            if (__syncthreads_or(!done)) {
                if (tid == 0) atomicExch(&g_nn_error, 1);
                // drain: wait once more (bounded) for the MMAs in flight before the tensor memory is freed
                for (long long k = 0; !done && k < kNnSpin; ++k)
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
        }
        if (failed) break;
        // epilogue: TMEM lane = row r = 16 y + c of the plane, columns p * NPAD + channel
        const int yy = tid >> 4, cc = tid & 15;
        const int gx = x0 + cc, gy = y0 + 1 + yy;
        const bool colok = cc >= 1 && cc <= kTileX && gx < nx && gy < ny;
        for (int p = 0; p < TZ; ++p) {
            const int gz = z0 + 1 + p;
            const bool ok = colok && gz < nz;
#pragma unroll
            for (int j = 0; j < NPAD / 16; ++j) {
                uint32_t r[16];
                const uint32_t a = taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(p * NPAD + j * 16);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                    : "r"(a));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (ok) {
                    float* o = out + (((int64_t)gz * ny + gy) * nx + gx) * ldo + coff;
                    float vals[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int n = j * 16 + q;
                        float val = __uint_as_float(r[q]) + ((bias && n < nout) ? bias[n] : 0.f);
                        vals[q] = relu ? fmaxf(val, 0.f) : val;
                    }
                    if (vec_out && j * 16 + 16 <= nout) {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            *reinterpret_cast<float4*>(o + j * 16 + 4 * q) =
                                make_float4(vals[4 * q], vals[4 * q + 1], vals[4 * q + 2], vals[4 * q + 3]);
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q)
                            if (j * 16 + q < nout) o[j * 16 + q] = vals[q];
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(Cfg::kCols));
}

// packed BF16 weights [npad][kpad]: forward rows co with k = tap*cin + ci; transposed (data
// gradient) rows ci with k = tap*cout + co.  Zero padding outside.
__global__ void pack_weights_kernel(const float* __restrict__ w, int cout, int cin, int transpose, int npad, int kpad,
                                    unsigned short* __restrict__ pk) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)npad * kpad) return;
    const int n = (int)(e / kpad), k = (int)(e % kpad);
    float v = 0.f;
    if (!transpose) {
        if (n < cout && k < 27 * cin) v = w[(int64_t)n * 27 * cin + k];   // w[co][tap][ci]
    } else {
        if (n < cin && k < 27 * cout) {
            const int tap = k / cout, co = k % cout;
            v = w[((int64_t)co * 27 + tap) * cin + n];
        }
    }
    pk[e] = nn_bf16(v);
}

// weight gradient: gw[co][tap][ci] += sum_v gout[v][co] in[v + off(tap)][ci], gb[co] += sum_v gout[v][co].
constexpr int kWgVox = 128;    // voxels staged per round by the transposed convolution's weight gradient

// Weight gradient of the 3x3x3 convolution as a BF16 implicit GEMM on the tensor cores:
//   gw[co][m] += sum_v gout[v][co] in[v + off(tap_m)][ci_m],   m = tap * cin + ci,
// with the rows m of the transposed im2col matrix of the input as GEMM rows (tiles of 128), the
// output channels as columns (N = NPAD) and the voxels as the reduction (k-blocks of 16).  Both
// operands are rounded to BF16 as they are staged in the same K-major core-matrix layout as the
// forward kernel's, and the products accumulate in FP32 in tensor memory.  A CTA takes up to
// kWtTiles row tiles (one accumulator each) and one contiguous range of voxel rounds; it writes its
// accumulators to its own partial-sum slot [blockIdx.x][row][NPAD], and wgrad_sum_kernel adds the
// slots in slot order, so the gradient is bit-reproducible.
constexpr int kWtKB = 4;                  // k-blocks (16 voxels each) per MMA round
constexpr int kWtTiles = 4;               // row tiles (accumulators) per CTA
constexpr int kWtVox = 16 * kWtKB;        // voxels per round

template <int NPAD>
__global__ void __launch_bounds__(128) wgrad_tc_kernel(const float* __restrict__ in, const float* __restrict__ gout, int nz,
                                                       int ny, int nx, int cin, int cout, int mtiles, int tpc,
                                                       int rounds_per_cta, float* __restrict__ part) {
    constexpr int kBBytes = NPAD * 16 * 2;
    // tensor-memory columns: tpc accumulators of NPAD columns, rounded up to a power of two >= 32
    uint32_t kCols = 32;
    while (kCols < (uint32_t)(tpc * NPAD)) kCols <<= 1;
    constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NPAD >> 3) << 17) | ((uint32_t)(kNnM >> 4) << 24);
    extern __shared__ __align__(1024) unsigned char nsm[];
    unsigned char* a_sm = nsm;                                  // [tpc][kWtKB] blocks of 128 x 16
    unsigned char* b_sm = nsm + tpc * kWtKB * kNnABytes;         // [kWtKB] blocks of NPAD x 16
    __shared__ int s_vlin[kWtVox];          // linear voxel index of the round's voxels
    __shared__ uint32_t s_vmask[kWtVox];    // bit tap: the voxel exists and its tap neighbour is inside
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) uint64_t s_mbar;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(nn_smem_u32(&s_taddr)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(nn_smem_u32(&s_mbar)), "r"(1u));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = s_taddr, mbar = nn_smem_u32(&s_mbar);
    uint32_t phase = 0;
    const int64_t nvox = (int64_t)nz * ny * nx;
    const int64_t rounds = (nvox + kWtVox - 1) / kWtVox;
    const int64_t r0 = (int64_t)blockIdx.x * rounds_per_cta;
    const int64_t r1 = min(rounds, r0 + rounds_per_cta);
    const int rows = 27 * cin;
    const int tile0 = blockIdx.y * tpc;
    const int nt = min(tpc, mtiles - tile0);
    bool failed = false;
    for (int64_t r = r0; r < r1 && !failed; ++r) {
        const int64_t v0 = r * kWtVox;
        if (tid < kWtVox) {
            const int64_t v = v0 + tid;
            uint32_t mask = 0;
            if (v < nvox) {
                const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((int64_t)nx * ny));
                for (int t = 0; t < 27; ++t) {
                    const int zz = z + t / 9 - 1, yy = y + (t / 3) % 3 - 1, xx = x + t % 3 - 1;
                    if (zz >= 0 && zz < nz && yy >= 0 && yy < ny && xx >= 0 && xx < nx) mask |= 1u << t;
                }
            }
            s_vlin[tid] = (int)(v < nvox ? v : 0);   // volumes hold fewer than 2^31 voxels
            s_vmask[tid] = mask;
        }
        __syncthreads();
        // B: the output gradient of the round's voxels, row n = output channel, k = voxel
        for (int e = tid; e < NPAD * kWtKB * 2; e += blockDim.x) {
            const int n = e % NPAD, kh = e / NPAD, kb = kh >> 1, h = kh & 1;
            uint32_t pk[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = kb * 16 + h * 8 + 2 * q;
                const float g0 = (n < cout && v0 + j < nvox) ? gout[(v0 + j) * cout + n] : 0.f;
                const float g1 = (n < cout && v0 + j + 1 < nvox) ? gout[(v0 + j + 1) * cout + n] : 0.f;
                pk[q] = nn_bf16x2(g0, g1);
            }
            *reinterpret_cast<uint4*>(b_sm + kb * kBBytes + nn_kmajor_off(n, 8 * h)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
        // A: this thread's row m of each of the CTA's tiles, the input at the row's tap for every voxel
        for (int i = 0; i < nt; ++i) {
            const int m = (tile0 + i) * kNnM + tid;
            const bool mv = m < rows;
            const int tap = mv ? m / cin : 13, ci = mv ? m - tap * cin : 0;
            const int toff = ((tap / 9 - 1) * ny + (tap / 3) % 3 - 1) * nx + tap % 3 - 1;   // linear tap offset
            const uint32_t bit = mv ? 1u << tap : 0u;
            const float* src = in + ci;
            for (int kb = 0; kb < kWtKB; ++kb) {
                uint32_t pk[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float a2[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int j = kb * 16 + 2 * q + u;
                        a2[u] = (s_vmask[j] & bit) ? src[(int64_t)(s_vlin[j] + toff) * cin] : 0.f;
                    }
                    pk[q] = nn_bf16x2(a2[0], a2[1]);
                }
                unsigned char* arow = a_sm + (i * kWtKB + kb) * kNnABytes + nn_kmajor_off(tid, 0);
                *reinterpret_cast<uint4*>(arow) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                *reinterpret_cast<uint4*>(arow + 128) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            for (int i = 0; i < nt; ++i) {
                for (int kb = 0; kb < kWtKB; ++kb) {
                    const uint64_t ad = nn_desc(nn_smem_u32(a_sm + (i * kWtKB + kb) * kNnABytes));
                    const uint64_t bd = nn_desc(nn_smem_u32(b_sm + kb * kBBytes));
                    const uint32_t acc = (r > r0 || kb > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr + (uint32_t)(i * NPAD)),
                        "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                         : "memory");
        }
        long long spins = 0;
        uint32_t done = 0;
        while (!done) {
            asm volatile(
                "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\nselp.b32 %0, 1, 0, P1;\n}\n"
                : "=r"(done)
                : "r"(mbar), "r"(phase)
                : "memory");
            if (!done && ++spins > kNnSpin) break;
        }
        if (__syncthreads_or(!done)) {
            if (tid == 0) atomicExch(&g_nn_error, 1);
            // drain: wait once more (bounded) for the MMAs in flight before the tensor memory is freed
            for (long long k = 0; !done && k < kNnSpin; ++k)
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
    }
    if (!failed && r0 < r1) {
        // accumulators -> this CTA's partial-sum slot: TMEM lane = row m, columns = output channels
        const int64_t mrows = (int64_t)mtiles * kNnM;
        for (int i = 0; i < nt; ++i) {
            const int m = (tile0 + i) * kNnM + warp * 32 + lane;
#pragma unroll
            for (int j = 0; j < NPAD / 16; ++j) {
                uint32_t rr[16];
                const uint32_t ta = taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(i * NPAD + j * 16);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                    : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]), "=r"(rr[7]),
                      "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]), "=r"(rr[14]), "=r"(rr[15])
                    : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (m < rows) {
                    float* dst = part + ((int64_t)blockIdx.x * mrows + m) * NPAD + j * 16;
#pragma unroll
                    for (int q = 0; q < 16; ++q) dst[q] = __uint_as_float(rr[q]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kCols));
}

// gw[co][m] += sum over the partial-sum slots (in slot order) of part[slot][m][co]
__global__ void wgrad_sum_kernel(const float* __restrict__ part, int nslots, int64_t mrows, int npad, int rows, int cout,
                                 float* __restrict__ gw) {
    // one warp per gw entry: lane l adds slots l, l + 32, ... in order, then a fixed shuffle tree
    const int lane = threadIdx.x & 31;
    const int64_t n = (int64_t)rows * cout;
    for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < n;
         e += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int co = (int)(e / rows), m = (int)(e % rows);
        float acc = 0.f;
        for (int s = lane; s < nslots; s += 32) acc += part[((int64_t)s * mrows + m) * npad + co];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) gw[e] += acc;
    }
}

// bias gradient partials: part[block][co] = sum of gout[v][co] over the block's contiguous voxel
// range; the block's lanes (threads with the same co) take voxels in turn and are added in lane order
__global__ void bias_part_kernel(const float* __restrict__ gout, int64_t nvox, int cout, int64_t per_block,
                                 float* __restrict__ part) {
    __shared__ float red[256];
    const int lanes = max(1, (int)blockDim.x / cout);
    const int co = threadIdx.x % cout, l = threadIdx.x / cout;
    const int64_t v0 = (int64_t)blockIdx.x * per_block, v1 = min(nvox, v0 + per_block);
    float acc = 0.f;
    if (l < lanes)
        for (int64_t v = v0 + l; v < v1; v += lanes) acc += gout[v * cout + co];
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < cout) {
        float t = 0.f;
        for (int k = 0; k < lanes; ++k) t += red[k * cout + threadIdx.x];
        part[(int64_t)blockIdx.x * cout + threadIdx.x] = t;
    }
}

// g *= (act > 0)
__global__ void relu_bwd_kernel(const float* __restrict__ act, float* __restrict__ g, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!(act[i] > 0.f)) g[i] = 0.f;
}

// 1x1x1 layer: out[v][o] = b[o] + sum_c w[o][c] in[v][c]
__global__ void conv1_fwd_kernel(const float* __restrict__ in, int64_t nvox, int cin, int cout, const float* __restrict__ w,
                                 const float* __restrict__ b, float* __restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nvox * cout; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e / cout;
        const int o = (int)(e % cout);
        float a = b[o];
        for (int c = 0; c < cin; ++c) a = fmaf(w[o * cin + c], in[v * cin + c], a);
        out[e] = a;
    }
}

// 1x1x1 layer backward: gin[v][c] = sum_o w[o][c] gout[v][o]
__global__ void conv1_gin_kernel(const float* __restrict__ gout, int64_t nvox, int cin, int cout, const float* __restrict__ w,
                                 float* __restrict__ gin) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (int64_t)gridDim.x * blockDim.x) {
        for (int c = 0; c < cin; ++c) {
            float a = 0.f;
            for (int o = 0; o < cout; ++o) a = fmaf(w[o * cin + c], gout[v * cout + o], a);
            gin[v * cin + c] = a;
        }
    }
}

// 1x1x1 layer weight partials: block b sums its contiguous voxel chunk in voxel order; thread e
// owns gw entry e (< cout cin) or bias entry e - cout cin.  part [gridDim.x][cout cin + cout].
__global__ void conv1_wpart_kernel(const float* __restrict__ in, const float* __restrict__ gout, int64_t nvox, int cin,
                                   int cout, float* __restrict__ part) {
    const int nw = cout * cin + cout;
    const int e = threadIdx.x;
    if (e >= nw) return;
    const int64_t chunk = (nvox + gridDim.x - 1) / gridDim.x;
    const int64_t v0 = (int64_t)blockIdx.x * chunk, v1 = min(nvox, v0 + chunk);
    float acc = 0.f;
    if (e < cout * cin) {
        const int o = e / cin, c = e % cin;
        for (int64_t v = v0; v < v1; ++v) acc = fmaf(gout[v * cout + o], in[v * cin + c], acc);
    } else {
        const int o = e - cout * cin;
        for (int64_t v = v0; v < v1; ++v) acc += gout[v * cout + o];
    }
    part[(int64_t)blockIdx.x * nw + e] = acc;
}

// dst[i] += sum over the nb partial rows (in row order) of part[b * stride + i], i < n
__global__ void wsum_kernel(const float* __restrict__ part, int nb, int64_t stride, int64_t n, float* __restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int b = 0; b < nb; ++b) acc += part[(int64_t)b * stride + i];
        dst[i] += acc;
    }
}

// mean squared error: g = 2 (out - tgt) / n and the block partials of sum (out - tgt)^2 / n
// (part[blockIdx.x]; the loss is their sum in block order)
__global__ void mse_kernel(const float* __restrict__ out, const float* __restrict__ tgt, int64_t n, float* __restrict__ g,
                           float* __restrict__ part) {
    __shared__ float red[8];
    float acc = 0.f;
    const float inv = 1.0f / (float)n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = out[i] - tgt[i];
        g[i] = 2.f * d * inv;
        acc += d * d * inv;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

// Adam (Kingma & Ba) with bias correction; step is 1-based
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            int64_t n, float lr, float b1, float b2, float eps, int step) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Network input: [Re x^t, Im x^t] / s and [Re d, Im d] * eta / s with s the RMS of (x^t, eta d)
// over the voxels (non-zero from the first outer iteration, where x^t = 0), summed reproducibly:
// per-block FP64 partials over a fixed grid of
// kFeatBlocks blocks, summed in block order by every consumer, so the network input (and with it
// the prediction) is bit-identical from run to run.  eta is read from eta_dev when that is given
// (the solver's step lives on the device), else the host value is used.
__global__ void feat_part_kernel(const float2* __restrict__ x, const float2* __restrict__ d, float eta_h,
                                 const double* __restrict__ eta_dev, int64_t n, double* __restrict__ part) {
    __shared__ double red[8];
    const float eta = eta_dev ? (float)*eta_dev : eta_h;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = x[i], b = d[i];
        acc += (double)(a.x * a.x + a.y * a.y) + (double)(eta * eta) * (double)(b.x * b.x + b.y * b.y);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

__global__ void features_det_kernel(const float2* __restrict__ x, const float2* __restrict__ d, int64_t n, float eta_h,
                                    const double* __restrict__ eta_dev, const double* __restrict__ part,
                                    float* __restrict__ ss, float* __restrict__ f) {
    __shared__ float s_inv;
    const float eta = eta_dev ? (float)*eta_dev : eta_h;
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int b = 0; b < kFeatBlocks; ++b) tot += part[b];
        const float ssf = (float)tot;
        if (blockIdx.x == 0) ss[0] = ssf;
        s_inv = 1.f / (sqrtf(ssf / (float)n) + 1e-12f);
    }
    __syncthreads();
    const float inv = s_inv;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        f[4 * i + 0] = x[i].x * inv;
        f[4 * i + 1] = x[i].y * inv;
        f[4 * i + 2] = d[i].x * eta * inv;
        f[4 * i + 3] = d[i].y * eta * inv;
    }
}

// out = x + s * delta (delta [n][2] in units of s)
__global__ void apply_delta_kernel(const float2* __restrict__ x, const float* __restrict__ delta, int64_t n,
                                   const float* __restrict__ ss, float2* __restrict__ out) {
    const float s = sqrtf(ss[0] / (float)n) + 1e-12f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = make_float2(fmaf(s, delta[2 * i], x[i].x), fmaf(s, delta[2 * i + 1], x[i].y));
}

// target: (x_target - x^t) / s as [n][2]
__global__ void target_kernel(const float2* __restrict__ xt, const float2* __restrict__ xs, int64_t n,
                              const float* __restrict__ ss, float* __restrict__ tgt) {
    const float inv = 1.f / (sqrtf(ss[0] / (float)n) + 1e-12f);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        tgt[2 * i] = (xs[i].x - xt[i].x) * inv;
        tgt[2 * i + 1] = (xs[i].y - xt[i].y) * inv;
    }
}

// ---- U-Net pieces.  Child a = 4 dz + 2 dy + dx of a 2x2x2 block; coarse sizes (nz, ny, nx). ----

// 2x2x2 max-pool: out[v][c] = max over the children of v; idx = first child reaching the maximum
__global__ void maxpool2_kernel(const float* __restrict__ in, int nz, int ny, int nx, int C, float* __restrict__ out,
                                unsigned char* __restrict__ idx) {
    const int64_t n = (int64_t)nz * ny * nx * C;
    const int64_t fy = 2 * nx, fz = (int64_t)4 * ny * nx;   // fine strides in voxels
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        const int64_t v = e / C;
        const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((int64_t)nx * ny));
        const int64_t base = (int64_t)(2 * z) * fz + (int64_t)(2 * y) * fy + 2 * x;
        float best = 0.f;
        int arg = 0;
        for (int a = 0; a < 8; ++a) {
            const int64_t f = base + (a >> 2) * fz + ((a >> 1) & 1) * fy + (a & 1);
            const float val = in[f * C + c];
            if (a == 0 || val > best) {
                best = val;
                arg = a;
            }
        }
        out[e] = best;
        idx[e] = (unsigned char)arg;
    }
}

// gin (fine) = the pooled gradient routed to each block's argmax child, zero elsewhere
__global__ void maxpool2_bwd_kernel(const float* __restrict__ g, const unsigned char* __restrict__ idx, int nz, int ny,
                                    int nx, int C, float* __restrict__ gin) {
    const int64_t n = (int64_t)nz * ny * nx * C;
    const int64_t fy = 2 * nx, fz = (int64_t)4 * ny * nx;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        const int64_t v = e / C;
        const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((int64_t)nx * ny));
        const int64_t base = (int64_t)(2 * z) * fz + (int64_t)(2 * y) * fy + 2 * x;
        const int arg = idx[e];
        const float gv = g[e];
        for (int a = 0; a < 8; ++a) {
            const int64_t f = base + (a >> 2) * fz + ((a >> 1) & 1) * fy + (a & 1);
            gin[f * C + c] = (a == arg) ? gv : 0.f;
        }
    }
}

// stride-2 transposed convolution (kernel 2): out[child a of v][coff + co] = b[co] + sum_ci in[v][ci] w[co][a][ci].
// A thread takes one coarse voxel and one group of 4 output channels (blockIdx.y) for all 8
// children; the block's 4 x 8 weight rows sit in shared memory and are read as broadcasts.
constexpr int kUpThreads = 256;
__global__ void __launch_bounds__(kUpThreads) upconv2_kernel(const float* __restrict__ in, int nz, int ny, int nx, int cin,
                                                             const float* __restrict__ w, const float* __restrict__ b,
                                                             int cout, float* __restrict__ out, int ldo, int coff, int vec) {
    extern __shared__ float4 usw[];            // [cin / 4][4 r][8 a] float4 (vec) or [cin][4][8] floats
    float* uss = reinterpret_cast<float*>(usw);
    const int co0 = blockIdx.y * 4;
    const int nr = min(4, cout - co0);
    for (int e = threadIdx.x; e < cin * 32; e += blockDim.x) {
        const int ci = e / 32, ra = e % 32, r = ra / 8, a = ra % 8;
        const float val = r < nr ? w[((int64_t)(co0 + r) * 8 + a) * cin + ci] : 0.f;
        if (vec)
            uss[(((ci >> 2) * 4 + r) * 8 + a) * 4 + (ci & 3)] = val;
        else
            uss[(ci * 4 + r) * 8 + a] = val;
    }
    __syncthreads();
    const int64_t nvox = (int64_t)nz * ny * nx;
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    float acc[8][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const float bb = (b && r < nr) ? b[co0 + r] : 0.f;
#pragma unroll
        for (int a = 0; a < 8; ++a) acc[a][r] = bb;
    }
    const float* iv = in + v * cin;
    if (vec) {
        for (int c4 = 0; c4 < cin / 4; ++c4) {
            const float4 xi = *reinterpret_cast<const float4*>(iv + 4 * c4);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    const float4 wv = usw[(c4 * 4 + r) * 8 + a];
                    acc[a][r] = fmaf(xi.x, wv.x, fmaf(xi.y, wv.y, fmaf(xi.z, wv.z, fmaf(xi.w, wv.w, acc[a][r]))));
                }
            }
        }
    } else {
        for (int ci = 0; ci < cin; ++ci) {
            const float xi = iv[ci];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int a = 0; a < 8; ++a) acc[a][r] = fmaf(xi, uss[(ci * 4 + r) * 8 + a], acc[a][r]);
        }
    }
    const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((int64_t)nx * ny));
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int64_t f = ((int64_t)(2 * z + (a >> 2)) * (2 * ny) + (2 * y + ((a >> 1) & 1))) * (2 * nx) + 2 * x + (a & 1);
        float* o = out + f * ldo + coff + co0;
        if (nr == 4 && (reinterpret_cast<uintptr_t>(o) & 15) == 0) {
            *reinterpret_cast<float4*>(o) = make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (r < nr) o[r] = acc[a][r];
        }
    }
}

// data gradient of upconv2: gin[v][ci] = sum_{a, co} gout[child a of v][goff + co] w[co][a][ci]
__global__ void upconv2_bwd_kernel(const float* __restrict__ gout, int ldg, int goff, int nz, int ny, int nx, int cin,
                                   const float* __restrict__ w, int cout, float* __restrict__ gin) {
    const int64_t n = (int64_t)nz * ny * nx * cin;
    const int64_t fy = 2 * nx, fz = (int64_t)4 * ny * nx;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int ci = (int)(e % cin);
        const int64_t v = e / cin;
        const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((int64_t)nx * ny));
        const int64_t base = (int64_t)(2 * z) * fz + (int64_t)(2 * y) * fy + 2 * x;
        float acc = 0.f;
        for (int a = 0; a < 8; ++a) {
            const float* gf = gout + (base + (a >> 2) * fz + ((a >> 1) & 1) * fy + (a & 1)) * ldg + goff;
            for (int co = 0; co < cout; ++co) acc = fmaf(gf[co], w[((int64_t)co * 8 + a) * cin + ci], acc);
        }
        gin[e] = acc;
    }
}

// weight gradient of upconv2: gw[co][a][ci] += sum_v gout[child a of v][goff + co] in[v][ci];
// gb[co] += sum over fine voxels of gout (blocks with blockIdx.z == 0 only).  Grid (x, 8 = a, pair chunks).
__global__ void upconv2_wgrad_kernel(const float* __restrict__ in, const float* __restrict__ gout, int ldg, int goff, int nz,
                                     int ny, int nx, int cin, int cout, float* __restrict__ gw, float* __restrict__ gb) {
    extern __shared__ float usm[];
    float* sg = usm;                      // [kWgVox][cout]
    float* si = usm + kWgVox * cout;      // [kWgVox][cin]
    const int a = blockIdx.y;
    const int64_t nvox = (int64_t)nz * ny * nx;
    const int64_t fy = 2 * nx, fz = (int64_t)4 * ny * nx;
    const int pairs = cout * cin;
    const int pbase = blockIdx.z * 4 * blockDim.x;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    float bacc = 0.f;
    for (int64_t v0 = (int64_t)blockIdx.x * kWgVox; v0 < nvox; v0 += (int64_t)gridDim.x * kWgVox) {
        __syncthreads();
        for (int e = threadIdx.x; e < kWgVox * cout; e += blockDim.x) {
            const int64_t v = v0 + e / cout;
            float val = 0.f;
            if (v < nvox) {
                const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((int64_t)nx * ny));
                const int64_t f = (int64_t)(2 * z + (a >> 2)) * fz + (int64_t)(2 * y + ((a >> 1) & 1)) * fy + 2 * x + (a & 1);
                val = gout[f * ldg + goff + e % cout];
            }
            sg[e] = val;
        }
        for (int e = threadIdx.x; e < kWgVox * cin; e += blockDim.x) {
            const int64_t v = v0 + e / cin;
            si[e] = (v < nvox) ? in[v * cin + e % cin] : 0.f;
        }
        __syncthreads();
        for (int q = 0; q < 4; ++q) {
            const int pr = pbase + threadIdx.x + q * blockDim.x;
            if (pr < pairs) {
                const int co = pr / cin, ci = pr % cin;
                float s = 0.f;
                for (int t = 0; t < kWgVox; ++t) s = fmaf(sg[t * cout + co], si[t * cin + ci], s);
                acc[q] += s;
            }
        }
        if (blockIdx.z == 0 && threadIdx.x < cout)
            for (int t = 0; t < kWgVox; ++t) bacc += sg[t * cout + threadIdx.x];
    }
    float* pw = gw + (int64_t)blockIdx.x * cout * 8 * cin;   // this voxel block's partial sums
    for (int q = 0; q < 4; ++q) {
        const int pr = pbase + threadIdx.x + q * blockDim.x;
        if (pr < pairs) {
            const int co = pr / cin, ci = pr % cin;
            pw[((int64_t)co * 8 + a) * cin + ci] = acc[q];
        }
    }
    if (blockIdx.z == 0 && threadIdx.x < cout && gb) gb[((int64_t)blockIdx.x * 8 + a) * cout + threadIdx.x] = bacc;
}

// channel slices: dst[v][doff + j] (+)= src[v][soff + j], j < n; with n, the offsets and strides
// multiples of 4 (and aligned pointers) a thread moves 4 channels
__global__ void slice_kernel(const float* __restrict__ src, int lds, int soff, int n, float* __restrict__ dst, int ldd,
                             int doff, int64_t nvox, int accumulate, int vec) {
    const int per = vec ? n >> 2 : n;
    const int64_t tot = nvox * per;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e / per;
        const int j = (int)(e - v * per);
        if (vec) {
            const float4 sv = *reinterpret_cast<const float4*>(src + v * lds + soff + 4 * j);
            float4* d = reinterpret_cast<float4*>(dst + v * ldd + doff + 4 * j);
            if (accumulate) {
                const float4 dv = *d;
                *d = make_float4(dv.x + sv.x, dv.y + sv.y, dv.z + sv.z, dv.w + sv.w);
            } else {
                *d = sv;
            }
        } else {
            const float sv = src[v * lds + soff + j];
            float* d = dst + v * ldd + doff + j;
            *d = accumulate ? *d + sv : sv;
        }
    }
}

// box crop of a complex volume: dst[z][y][x] = src[oz + z][oy + y][ox + x] (the box lies inside src)
__global__ void crop3d_kernel(const float2* __restrict__ src, int ny, int nx, int oz, int oy, int ox, int cz, int cy,
                              int cx, float2* __restrict__ dst) {
    const int64_t n = (int64_t)cz * cy * cx;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(e % cx);
        const int64_t r = e / cx;
        const int y = (int)(r % cy), z = (int)(r / cy);
        dst[e] = src[((int64_t)(oz + z) * ny + (oy + y)) * nx + (ox + x)];
    }
}

static int nn_grid(int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096));
}

cs_status nn_init_attrs() {
    CS_TRY_CUDA(cudaFuncSetAttribute(conv3_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kNnChunk * kNnABytes + kNnChunk * 16 * 32));
    CS_TRY_CUDA(cudaFuncSetAttribute(conv3_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kNnChunk * kNnABytes + kNnChunk * 32 * 32));
    CS_TRY_CUDA(cudaFuncSetAttribute(conv3_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kNnChunk * kNnABytes + kNnChunk * 64 * 32));
    CS_TRY_CUDA(cudaFuncSetAttribute(conv3_brick_kernel<16, kBrTZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     BrickCfg<16, kBrTZ>::kSmem));
    CS_TRY_CUDA(cudaFuncSetAttribute(conv3_brick_kernel<16, kBrTZ>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    CS_TRY_CUDA(cudaFuncSetAttribute(conv3_brick_kernel<32, kBrTZ>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    CS_TRY_CUDA(cudaFuncSetAttribute(conv3_brick_kernel<64, kBrTZ>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    CS_TRY_CUDA(cudaFuncSetAttribute(conv3_brick_kernel<32, kBrTZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     BrickCfg<32, kBrTZ>::kSmem));
    CS_TRY_CUDA(cudaFuncSetAttribute(conv3_brick_kernel<64, kBrTZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     BrickCfg<64, kBrTZ>::kSmem));
    // weight gradients: kWtTiles x kWtKB row blocks and kWtKB gradient blocks per round
    CS_TRY_CUDA(cudaFuncSetAttribute(wgrad_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kWtTiles * kWtKB * kNnABytes + kWtKB * 16 * 32));
    CS_TRY_CUDA(cudaFuncSetAttribute(wgrad_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kWtTiles * kWtKB * kNnABytes + kWtKB * 32 * 32));
    CS_TRY_CUDA(cudaFuncSetAttribute(wgrad_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kWtTiles * kWtKB * kNnABytes + kWtKB * 64 * 32));
    CS_TRY_CUDA(cudaFuncSetAttribute(wgrad_tc_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kWtTiles * kWtKB * kNnABytes + kWtKB * 128 * 32));
    // the transposed convolution's weight gradient stages kWgVox voxels of cin + cout <= 256 channels
    CS_TRY_CUDA(cudaFuncSetAttribute(upconv2_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(float) * kWgVox * 256));
    return CS_OK;
}

static cs_status nn_attrs_once() {
    static bool init[128] = {false};
    int dev = 0;
    CS_TRY_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 128 && !init[dev]) {
        CS_PROPAGATE(nn_init_attrs());
        init[dev] = true;
    }
    return CS_OK;
}

// persistent grid: as many CTAs per SM as shared memory and tensor memory (512 columns) allow
template <int NPAD>
static cs_status launch_brick(int64_t tiles, int sms, const float* in, int nz, int ny, int nx, int cin,
                              const unsigned short* packed, int kpad, int nout, const float* bias, int relu, int flip,
                              float* out, int ldo, int coff, cudaStream_t st) {
    using Cfg = BrickCfg<NPAD, kBrTZ>;
    // 228 KB of shared memory per SM, 1 KB of it reserved per CTA, plus this kernel's static 1 KB
    const int per_sm = std::max(1, std::min(233472 / (Cfg::kSmem + 2048), (int)(512u / Cfg::kCols)));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)std::max(sms, 1) * per_sm));
    conv3_brick_kernel<NPAD, kBrTZ><<<grid, 128, Cfg::kSmem, st>>>(in, nz, ny, nx, cin, packed, kpad, nout, bias, relu,
                                                                   flip, out, ldo, coff);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

cs_status nn_check_and_clear() {
    int v = 0;
    CS_TRY_CUDA(cudaMemcpyFromSymbol(&v, g_nn_error, sizeof(int)));
    if (v) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_nn_error, &zero, sizeof(int));
        set_error("a tensor-core convolution gave up waiting for its MMAs (bounded wait)");
        return CS_ERR_TIMEOUT;
    }
    return CS_OK;
}

}  // namespace cs

using namespace cs;

extern "C" {

cs_status cs_nn_pack_weights(const float* w, int cout, int cin, int transpose, unsigned short* packed, int npad,
                             int kpad, void* stream) {
    clear_error();
    CS_REQUIRE(w && packed && cout >= 1 && cin >= 1, CS_ERR_INVALID_ARG, "bad pack arguments");
    const int nn = transpose ? cin : cout, kk = 27 * (transpose ? cout : cin);
    CS_REQUIRE((npad == 16 || npad == 32 || npad == 64) && npad >= nn && kpad % 16 == 0 && kpad >= kk,
               CS_ERR_INVALID_ARG, "packed shape %d x %d cannot hold %d x %d", npad, kpad, nn, kk);
    const int64_t n = (int64_t)npad * kpad;
    pack_weights_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(w, cout, cin, transpose, npad, kpad,
                                                                                       packed);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

cs_status cs_nn_conv3d(const float* in, int nz, int ny, int nx, int cin, const unsigned short* packed, int npad, int kpad,
                       int nout, const float* bias, int relu, int flip, float* out, int ldo, int coff, void* stream) {
    clear_error();
    CS_REQUIRE(in && packed && out && nz > 0 && ny > 0 && nx > 0 && cin >= 1 && nout >= 1 && nout <= npad &&
                   coff >= 0 && coff + nout <= ldo && kpad >= 27 * cin && kpad % 16 == 0 &&
                   (reinterpret_cast<uintptr_t>(packed) & 15) == 0,
               CS_ERR_INVALID_ARG, "bad conv3d arguments");
    CS_PROPAGATE(nn_attrs_once());
    int dev = 0;
    CS_TRY_CUDA(cudaGetDevice(&dev));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nvox = (int64_t)nz * ny * nx;
    const int64_t tiles = (nvox + kNnM - 1) / kNnM;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)std::max(sms, 1) * 4));
    if ((cin & 3) == 0 && (reinterpret_cast<uintptr_t>(in) & 15) == 0) {
        const int64_t btiles = (int64_t)((nx + kTileX - 1) / kTileX) * ((ny + kTileY - 1) / kTileY) *
                               ((nz + kBrTZ - 1) / kBrTZ);
        switch (npad) {
            case 16: return launch_brick<16>(btiles, sms, in, nz, ny, nx, cin, packed, kpad, nout, bias, relu, flip, out, ldo, coff, st);
            case 32: return launch_brick<32>(btiles, sms, in, nz, ny, nx, cin, packed, kpad, nout, bias, relu, flip, out, ldo, coff, st);
            case 64: return launch_brick<64>(btiles, sms, in, nz, ny, nx, cin, packed, kpad, nout, bias, relu, flip, out, ldo, coff, st);
            default: set_error("npad must be 16, 32 or 64"); return CS_ERR_INVALID_ARG;
        }
    }
    const size_t sm = (size_t)kNnChunk * kNnABytes + (size_t)kNnChunk * npad * 32;
    switch (npad) {
        case 16: conv3_tc_kernel<16><<<grid, 128, sm, st>>>(in, nz, ny, nx, cin, packed, kpad, nout, bias, relu, flip, out, ldo, coff); break;
        case 32: conv3_tc_kernel<32><<<grid, 128, sm, st>>>(in, nz, ny, nx, cin, packed, kpad, nout, bias, relu, flip, out, ldo, coff); break;
        case 64: conv3_tc_kernel<64><<<grid, 128, sm, st>>>(in, nz, ny, nx, cin, packed, kpad, nout, bias, relu, flip, out, ldo, coff); break;
        default: set_error("npad must be 16, 32 or 64"); return CS_ERR_INVALID_ARG;
    }
    CS_LAUNCH_CHECK();
    return CS_OK;
}

cs_status cs_nn_conv3d_wgrad(const float* in, const float* gout, int nz, int ny, int nx, int cin, int cout, float* gw,
                             float* gb, void* stream) {
    clear_error();
    CS_REQUIRE(in && gout && gw && cin >= 1 && cout >= 1 && cin <= 128 && cout <= 128 && nz >= 1 && ny >= 1 && nx >= 1,
               CS_ERR_INVALID_ARG, "bad wgrad arguments");
    CS_PROPAGATE(nn_attrs_once());
    const int64_t nvox = (int64_t)nz * ny * nx;
    cudaStream_t st = (cudaStream_t)stream;
    const int rows = 27 * cin;
    const int mtiles = (rows + kNnM - 1) / kNnM;
    const int tpc = std::min(kWtTiles, mtiles);                 // row tiles per CTA
    const int groups = (mtiles + tpc - 1) / tpc;
    const int npad = cout <= 16 ? 16 : cout <= 32 ? 32 : cout <= 64 ? 64 : 128;
    const size_t sm = (size_t)tpc * kWtKB * kNnABytes + (size_t)kWtKB * npad * 32;
    int cols = 32;
    while (cols < tpc * npad) cols <<= 1;
    // resident CTAs per SM allowed by shared and tensor memory (at most 8); the voxel rounds are
    // split so that that many CTAs per SM run, every CTA with at least one round
    const int per_sm = (int)std::max<size_t>(
        1, std::min<size_t>(std::min<size_t>(8, (size_t)(220 * 1024) / (sm + 2048)), (size_t)(512 / cols)));
    const int64_t rounds = (nvox + kWtVox - 1) / kWtVox;
    const int64_t want = std::max<int64_t>(1, ((int64_t)per_sm * 152 + groups - 1) / groups);
    const int64_t per = (rounds + std::min(rounds, want) - 1) / std::min(rounds, want);
    const int nslots = (int)((rounds + per - 1) / per);
    const int64_t mrows = (int64_t)mtiles * kNnM;
    const int nbias = (int)std::max<int64_t>(1, std::min<int64_t>((nvox + 511) / 512, 1024));
    const int64_t bper = (nvox + nbias - 1) / nbias;
    float* part = nullptr;
    CS_TRY_CUDA(cudaMallocAsync((void**)&part, sizeof(float) * ((size_t)nslots * mrows * npad + (size_t)nbias * cout), st));
    float* pb = part + (int64_t)nslots * mrows * npad;
    const dim3 grid((unsigned)nslots, (unsigned)groups);
    switch (npad) {
        case 16: wgrad_tc_kernel<16><<<grid, 128, sm, st>>>(in, gout, nz, ny, nx, cin, cout, mtiles, tpc, (int)per, part); break;
        case 32: wgrad_tc_kernel<32><<<grid, 128, sm, st>>>(in, gout, nz, ny, nx, cin, cout, mtiles, tpc, (int)per, part); break;
        case 64: wgrad_tc_kernel<64><<<grid, 128, sm, st>>>(in, gout, nz, ny, nx, cin, cout, mtiles, tpc, (int)per, part); break;
        default: wgrad_tc_kernel<128><<<grid, 128, sm, st>>>(in, gout, nz, ny, nx, cin, cout, mtiles, tpc, (int)per, part); break;
    }
    CS_LAUNCH_CHECK();
    wgrad_sum_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(((int64_t)rows * cout + 7) / 8, 4096)), 256, 0,
                       st>>>(part, nslots, mrows, npad, rows, cout, gw);
    CS_LAUNCH_CHECK();
    if (gb) {
        bias_part_kernel<<<nbias, 256, 0, st>>>(gout, nvox, cout, bper, pb);
        CS_LAUNCH_CHECK();
        wsum_kernel<<<1, 256, 0, st>>>(pb, nbias, cout, cout, gb);
        CS_LAUNCH_CHECK();
    }
    CS_TRY_CUDA(cudaFreeAsync(part, st));
    return CS_OK;
}

cs_status cs_nn_relu_bwd(const float* act, float* g, int64_t n, void* stream) {
    clear_error();
    CS_REQUIRE(act && g && n >= 0, CS_ERR_INVALID_ARG, "bad relu_bwd arguments");
    if (n == 0) return CS_OK;
    relu_bwd_kernel<<<nn_grid(n), 256, 0, (cudaStream_t)stream>>>(act, g, n);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

cs_status cs_nn_conv1(const float* in, int64_t nvox, int cin, int cout, const float* w, const float* b, float* out,
                      void* stream) {
    clear_error();
    CS_REQUIRE(in && w && b && out && cin >= 1 && cout >= 1, CS_ERR_INVALID_ARG, "bad conv1 arguments");
    conv1_fwd_kernel<<<nn_grid(nvox * cout), 256, 0, (cudaStream_t)stream>>>(in, nvox, cin, cout, w, b, out);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

cs_status cs_nn_conv1_bwd(const float* in, const float* gout, int64_t nvox, int cin, int cout, const float* w, float* gin,
                          float* gw, float* gb, void* stream) {
    clear_error();
    CS_REQUIRE(in && gout && w && gin && gw && gb && cin * cout + cout <= 64 * 4 + 4, CS_ERR_INVALID_ARG,
               "bad conv1_bwd arguments");
    cudaStream_t st = (cudaStream_t)stream;
    conv1_gin_kernel<<<nn_grid(nvox), 256, 0, st>>>(gout, nvox, cin, cout, w, gin);
    CS_LAUNCH_CHECK();
    const int nw = cout * cin + cout, nb = kFeatBlocks;
    float* part = nullptr;
    CS_TRY_CUDA(cudaMallocAsync((void**)&part, sizeof(float) * (size_t)nb * nw, st));
    conv1_wpart_kernel<<<nb, 288, 0, st>>>(in, gout, nvox, cin, cout, part);
    CS_LAUNCH_CHECK();
    wsum_kernel<<<1, 256, 0, st>>>(part, nb, nw, (int64_t)cout * cin, gw);
    CS_LAUNCH_CHECK();
    wsum_kernel<<<1, 256, 0, st>>>(part + (int64_t)cout * cin, nb, nw, cout, gb);
    CS_LAUNCH_CHECK();
    CS_TRY_CUDA(cudaFreeAsync(part, st));
    return CS_OK;
}

cs_status cs_nn_mse(const float* out, const float* tgt, int64_t n, float* g, float* loss, void* stream) {
    clear_error();
    CS_REQUIRE(out && tgt && g && loss && n > 0, CS_ERR_INVALID_ARG, "bad mse arguments");
    cudaStream_t st = (cudaStream_t)stream;
    float* part = nullptr;
    CS_TRY_CUDA(cudaMallocAsync((void**)&part, sizeof(float) * kFeatBlocks, st));
    mse_kernel<<<kFeatBlocks, 256, 0, st>>>(out, tgt, n, g, part);
    CS_LAUNCH_CHECK();
    wsum_kernel<<<1, 32, 0, st>>>(part, kFeatBlocks, 1, 1, loss);
    CS_LAUNCH_CHECK();
    CS_TRY_CUDA(cudaFreeAsync(part, st));
    return CS_OK;
}

cs_status cs_nn_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps,
                     int step, void* stream) {
    clear_error();
    CS_REQUIRE(p && g && m && v && n >= 0 && step >= 1, CS_ERR_INVALID_ARG, "bad adam arguments");
    if (n == 0) return CS_OK;
    adam_kernel<<<nn_grid(n), 256, 0, (cudaStream_t)stream>>>(p, g, m, v, n, lr, b1, b2, eps, step);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

// ss (device float, caller-owned): cleared and set to ||x^t||^2; f [n][4]; (targets and the
// application of a prediction use the same ss)
cs_status cs_nn_features(const float* xt, const float* d, int64_t n, float eta, float* ss, float* f, void* stream) {
    clear_error();
    CS_REQUIRE(xt && d && ss && f && n > 0, CS_ERR_INVALID_ARG, "bad features arguments");
    cudaStream_t st = (cudaStream_t)stream;
    double* part = nullptr;
    CS_TRY_CUDA(cudaMallocAsync((void**)&part, sizeof(double) * kFeatBlocks, st));
    CS_PROPAGATE(nn_features_det((const float2*)xt, (const float2*)d, n, eta, nullptr, part, ss, f, st));
    CS_TRY_CUDA(cudaFreeAsync(part, st));
    return CS_OK;
}

}  // extern "C"

namespace cs {
cs_status nn_features_det(const float2* xt, const float2* d, int64_t n, float eta, const double* eta_dev, double* part,
                          float* ss, float* f, cudaStream_t st) {
    feat_part_kernel<<<kFeatBlocks, 256, 0, st>>>(xt, d, eta, eta_dev, n, part);
    CS_LAUNCH_CHECK();
    features_det_kernel<<<nn_grid(n), 256, 0, st>>>(xt, d, n, eta, eta_dev, part, ss, f);
    CS_LAUNCH_CHECK();
    return CS_OK;
}
}  // namespace cs

extern "C" {

cs_status cs_nn_target(const float* xt, const float* xs, int64_t n, const float* ss, float* tgt, void* stream) {
    clear_error();
    CS_REQUIRE(xt && xs && ss && tgt && n > 0, CS_ERR_INVALID_ARG, "bad target arguments");
    target_kernel<<<nn_grid(n), 256, 0, (cudaStream_t)stream>>>((const float2*)xt, (const float2*)xs, n, ss, tgt);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

cs_status cs_nn_apply(const float* xt, const float* delta, int64_t n, const float* ss, float* out, void* stream) {
    clear_error();
    CS_REQUIRE(xt && delta && ss && out && n > 0, CS_ERR_INVALID_ARG, "bad apply arguments");
    apply_delta_kernel<<<nn_grid(n), 256, 0, (cudaStream_t)stream>>>((const float2*)xt, delta, n, ss, (float2*)out);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

cs_status cs_nn_maxpool2(const float* in, int nz, int ny, int nx, int C, float* out, unsigned char* idx, void* stream) {
    clear_error();
    CS_REQUIRE(in && out && idx && nz >= 1 && ny >= 1 && nx >= 1 && C >= 1, CS_ERR_INVALID_ARG,
               "bad maxpool arguments (coarse sizes)");
    const int64_t n = (int64_t)nz * ny * nx * C;
    maxpool2_kernel<<<nn_grid(n), 256, 0, (cudaStream_t)stream>>>(in, nz, ny, nx, C, out, idx);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

cs_status cs_nn_maxpool2_bwd(const float* g, const unsigned char* idx, int nz, int ny, int nx, int C, float* gin,
                             void* stream) {
    clear_error();
    CS_REQUIRE(g && idx && gin && nz >= 1 && ny >= 1 && nx >= 1 && C >= 1, CS_ERR_INVALID_ARG, "bad maxpool_bwd arguments");
    const int64_t n = (int64_t)nz * ny * nx * C;
    maxpool2_bwd_kernel<<<nn_grid(n), 256, 0, (cudaStream_t)stream>>>(g, idx, nz, ny, nx, C, gin);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

cs_status cs_nn_upconv2(const float* in, int nz, int ny, int nx, int cin, const float* w, const float* b, int cout,
                        float* out, int ldo, int coff, void* stream) {
    clear_error();
    CS_REQUIRE(in && w && out && nz >= 1 && ny >= 1 && nx >= 1 && cin >= 1 && cout >= 1 && coff >= 0 && coff + cout <= ldo,
               CS_ERR_INVALID_ARG, "bad upconv arguments");
    CS_REQUIRE(cin <= 1024 && (cout + 3) / 4 <= 65535, CS_ERR_UNSUPPORTED_SIZE, "upconv: cin above 1024");
    const int groups = (cout + 3) / 4;
    const int vec = (cin % 4 == 0) && (reinterpret_cast<uintptr_t>(in) & 15) == 0;
    const int64_t nvox = (int64_t)nz * ny * nx;
    const size_t sm = sizeof(float) * 32 * (size_t)cin;
    if (sm > 48 * 1024) CS_TRY_CUDA(cudaFuncSetAttribute(upconv2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const dim3 grid((unsigned)((nvox + kUpThreads - 1) / kUpThreads), (unsigned)groups);
    upconv2_kernel<<<grid, kUpThreads, sm, (cudaStream_t)stream>>>(in, nz, ny, nx, cin, w, b, cout, out, ldo, coff, vec);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

cs_status cs_nn_upconv2_bwd(const float* in, const float* gout, int ldg, int goff, int nz, int ny, int nx, int cin,
                            const float* w, int cout, float* gin, float* gw, float* gb, void* stream) {
    clear_error();
    CS_REQUIRE(in && gout && w && nz >= 1 && ny >= 1 && nx >= 1 && cin >= 1 && cout >= 1 && cin <= 128 && cout <= 128 &&
                   goff >= 0 && goff + cout <= ldg,
               CS_ERR_INVALID_ARG, "bad upconv_bwd arguments");
    CS_PROPAGATE(nn_attrs_once());
    cudaStream_t st = (cudaStream_t)stream;
    if (gin) {
        const int64_t n = (int64_t)nz * ny * nx * cin;
        upconv2_bwd_kernel<<<nn_grid(n), 256, 0, st>>>(gout, ldg, goff, nz, ny, nx, cin, w, cout, gin);
        CS_LAUNCH_CHECK();
    }
    if (gw) {
        const int64_t nvox = (int64_t)nz * ny * nx;
        const size_t sm = sizeof(float) * kWgVox * (cin + cout);
        const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((nvox + kWgVox - 1) / kWgVox, 64));
        const int chunks = (cin * cout + 1023) / 1024;
        const int64_t wsize = (int64_t)cout * 8 * cin;
        float* part = nullptr;     // per-voxel-block partials: weights [gx][wsize], bias [gx][8][cout]
        CS_TRY_CUDA(cudaMallocAsync((void**)&part, sizeof(float) * (size_t)gx * (wsize + 8 * cout), st));
        float* pb = part + (int64_t)gx * wsize;
        upconv2_wgrad_kernel<<<dim3(gx, 8, chunks), 256, sm, st>>>(in, gout, ldg, goff, nz, ny, nx, cin, cout, part,
                                                                   gb ? pb : nullptr);
        CS_LAUNCH_CHECK();
        wsum_kernel<<<nn_grid(wsize), 256, 0, st>>>(part, gx, wsize, wsize, gw);
        CS_LAUNCH_CHECK();
        if (gb) {
            wsum_kernel<<<1, 256, 0, st>>>(pb, gx * 8, cout, cout, gb);
            CS_LAUNCH_CHECK();
        }
        CS_TRY_CUDA(cudaFreeAsync(part, st));
    }
    return CS_OK;
}

cs_status cs_nn_slice(const float* src, int lds, int soff, int n, float* dst, int ldd, int doff, int64_t nvox,
                      int accumulate, void* stream) {
    clear_error();
    CS_REQUIRE(src && dst && n >= 1 && soff >= 0 && soff + n <= lds && doff >= 0 && doff + n <= ldd && nvox >= 0,
               CS_ERR_INVALID_ARG, "bad slice arguments");
    const int vec = n % 4 == 0 && lds % 4 == 0 && ldd % 4 == 0 && soff % 4 == 0 && doff % 4 == 0 &&
                    (reinterpret_cast<uintptr_t>(src) & 15) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
    slice_kernel<<<nn_grid(nvox * (vec ? n / 4 : n)), 256, 0, (cudaStream_t)stream>>>(src, lds, soff, n, dst, ldd, doff,
                                                                                    nvox, accumulate, vec);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

cs_status cs_crop3d(const float* src, const int* dims, const int* origin, const int* box, float* dst, void* stream) {
    clear_error();
    CS_REQUIRE(src && dims && origin && box && dst, CS_ERR_INVALID_ARG, "null pointer");
    for (int a = 0; a < 3; ++a)
        CS_REQUIRE(dims[a] >= 1 && box[a] >= 1 && origin[a] >= 0 && origin[a] + box[a] <= dims[a], CS_ERR_INVALID_ARG,
                   "crop box [%d, %d) outside axis %d of size %d", origin[a], origin[a] + box[a], a, dims[a]);
    const int64_t n = (int64_t)box[0] * box[1] * box[2];
    crop3d_kernel<<<nn_grid(n), 256, 0, (cudaStream_t)stream>>>((const float2*)src, dims[1], dims[2], origin[0],
                                                                origin[1], origin[2], box[0], box[1], box[2],
                                                                (float2*)dst);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

cs_status cs_nn_status(void* stream) {
    clear_error();
    CS_TRY_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return nn_check_and_clear();
}

}  // extern "C"
