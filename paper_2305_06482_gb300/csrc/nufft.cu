// Kaiser-Bessel gridding for the non-uniform Fourier operator F~_n (Sec. 2.1, Beatty et al.
// 2005): sample binning, interpolation (forward) and spreading (adjoint).
//
// Discretisation (identical to the CPU restatement, bit for bit where integers are decided):
//   g   = fmaf(f, G, G/2) in float32 per axis            (grid coordinate of a sample)
//   j0  = floor(g) - 1                                  (first of the W = 4 box indices)
//   phi(u) = I0(beta sqrt(1 - (u/2)^2)) / I0(beta),     beta = pi sqrt((W/a)^2 (a-1/2)^2 - 0.8)
//            (tabulated in double at 2049 points of [0, 2], linearly interpolated)
//   tile = floor((j0 mod G) / T) per axis, linear id (z, y, x) with x fastest.
// The forward grid is produced without the output modulation of the centred DFT; the sign
// (-1)^(j + G/2) of every grid index is folded into the interpolation weights instead.
#include <cmath>
#include <cstdio>

#include "cs_internal.cuh"

namespace cs {

constexpr int kW = 4;

__device__ __forceinline__ int wrapi(int j, int G) {
    j %= G;
    return j < 0 ? j + G : j;
}

// ------------------------------------------------------------------------------------------
// binning
__global__ void bin_keys_kernel(const float* __restrict__ traj, int64_t N, int nd, int3 G, int3 T, int3 nt,
                                float* __restrict__ gout, int32_t* __restrict__ j0out, int32_t* __restrict__ key) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int Gs[3] = {G.x, G.y, G.z}, Ts[3] = {T.x, T.y, T.z}, nts[3] = {nt.x, nt.y, nt.z};
    int64_t lin = 0;
    for (int ax = 0; ax < 3; ++ax) {
        int jj = 0;
        float g = 0.f;
        if (ax >= 3 - nd) {
            const int a = ax - (3 - nd);
            const float f = traj[i * nd + a];
            const float Gf = (float)Gs[ax];
            g = __fmaf_rn(f, Gf, 0.5f * Gf);
            jj = (int)floorf(g) - (kW / 2 - 1);
            j0out[i * nd + a] = jj;
        }
        gout[i * 3 + ax] = g;
        const int t = wrapi(jj, Gs[ax]) / Ts[ax];
        lin = lin * nts[ax] + t;
    }
    key[i] = (int32_t)lin;
}

constexpr int kRankChunk = 2048;

// One warp per chunk of kRankChunk consecutive samples: stable rank of each sample among the
// chunk's samples of the same tile (warp match + prefix popcount, processed in index order).
__global__ void chunk_rank_kernel(const int32_t* __restrict__ key, int64_t N, int ntiles,
                                  int32_t* __restrict__ lrank, int32_t* __restrict__ counts) {
    extern __shared__ int32_t running[];
    const int lane = threadIdx.x;
    const int64_t chunk = blockIdx.x;
    for (int t = lane; t < ntiles; t += 32) running[t] = 0;
    __syncwarp();
    const int64_t s0 = chunk * kRankChunk;
    const unsigned lt = (1u << lane) - 1u;
    for (int step = 0; step < kRankChunk; step += 32) {
        const int64_t i = s0 + step + lane;
        const bool valid = i < N;
        const int k = valid ? key[i] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, k);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (valid && lane == leader) base = running[k];
        base = __shfl_sync(0xffffffffu, base, leader);
        if (valid) lrank[i] = base + __popc(peers & lt);
        __syncwarp();
        if (valid && lane == leader) running[k] = base + __popc(peers);
        __syncwarp();
    }
    for (int t = lane; t < ntiles; t += 32) counts[chunk * (int64_t)ntiles + t] = running[t];
}

// per tile: exclusive scan over chunks (in place) and the tile total
__global__ void chunk_scan_kernel(int32_t* __restrict__ counts, int64_t nchunks, int ntiles, int32_t* __restrict__ total) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    int32_t run = 0;
    for (int64_t c = 0; c < nchunks; ++c) {
        const int32_t v = counts[c * ntiles + t];
        counts[c * ntiles + t] = run;
        run += v;
    }
    total[t] = run;
}

// single-CTA exclusive scan of tile totals -> tile_off[ntiles + 1]
__global__ void tile_scan_kernel(const int32_t* __restrict__ total, int ntiles, int32_t* __restrict__ off) {
    __shared__ int32_t part[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = (ntiles + nt - 1) / nt;
    const int b = tid * per, e = min(ntiles, b + per);
    int32_t s = 0;
    for (int i = b; i < e; ++i) s += total[i];
    part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        int32_t run = 0;
        for (int i = 0; i < nt; ++i) {
            const int32_t v = part[i];
            part[i] = run;
            run += v;
        }
        off[ntiles] = run;
    }
    __syncthreads();
    int32_t run = part[tid];
    for (int i = b; i < e; ++i) {
        off[i] = run;
        run += total[i];
    }
}

__global__ void bin_scatter_kernel(const int32_t* __restrict__ key, const int32_t* __restrict__ lrank,
                                   const int32_t* __restrict__ cbase, const int32_t* __restrict__ toff, int ntiles,
                                   const float* __restrict__ g, const float* __restrict__ dcf, int64_t N,
                                   int32_t* __restrict__ perm, float* __restrict__ gs, float* __restrict__ ws) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int k = key[i];
    const int64_t chunk = i / kRankChunk;
    const int64_t pos = (int64_t)toff[k] + cbase[chunk * ntiles + k] + lrank[i];
    perm[pos] = (int32_t)i;
    gs[pos * 3 + 0] = g[i * 3 + 0];
    gs[pos * 3 + 1] = g[i * 3 + 1];
    gs[pos * 3 + 2] = g[i * 3 + 2];
    ws[pos] = sqrtf(dcf[i]);
}

cs_status nufft_bin(cs_plan* p, const float* traj, const float* dcf, cudaStream_t st) {
    const int64_t N = p->N;
    const int nd = p->ndim;
    const int ntiles = (int)p->ntiles_total;
    CS_REQUIRE(ntiles <= 49152, CS_ERR_UNSUPPORTED_SIZE, "too many tiles (%d); use a larger tile", ntiles);
    const int64_t nchunks = (N + kRankChunk - 1) / kRankChunk;
    float* g = nullptr;
    int32_t *key = nullptr, *lrank = nullptr, *counts = nullptr, *total = nullptr;
    cs_status rc = CS_OK;
    auto cleanup = [&]() {
        cudaFree(g);
        cudaFree(key);
        cudaFree(lrank);
        cudaFree(counts);
        cudaFree(total);
    };
#define BIN_TRY(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            set_error("binning: %s: %s", #call, cudaGetErrorString(e_));                \
            cleanup();                                                                  \
            return e_ == cudaErrorMemoryAllocation ? CS_ERR_OOM : CS_ERR_CUDA;          \
        }                                                                               \
    } while (0)
    BIN_TRY(cudaMalloc(&g, sizeof(float) * 3 * N));
    BIN_TRY(cudaMalloc(&key, sizeof(int32_t) * N));
    BIN_TRY(cudaMalloc(&lrank, sizeof(int32_t) * N));
    BIN_TRY(cudaMalloc(&counts, sizeof(int32_t) * nchunks * ntiles));
    BIN_TRY(cudaMalloc(&total, sizeof(int32_t) * ntiles));
    const int3 G3 = make_int3(p->grid[0], p->grid[1], p->grid[2]);
    const int3 T3 = make_int3(p->tile[0], p->tile[1], p->tile[2]);
    const int3 nt3 = make_int3(p->ntiles[0], p->ntiles[1], p->ntiles[2]);
    const unsigned nb = (unsigned)((N + 255) / 256);
    bin_keys_kernel<<<nb, 256, 0, st>>>(traj, N, nd, G3, T3, nt3, g, p->j0, key);
    BIN_TRY(cudaGetLastError());
    const size_t rsm = sizeof(int32_t) * ntiles;
    BIN_TRY(cudaFuncSetAttribute(chunk_rank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
    chunk_rank_kernel<<<(unsigned)nchunks, 32, rsm, st>>>(key, N, ntiles, lrank, counts);
    BIN_TRY(cudaGetLastError());
    chunk_scan_kernel<<<(ntiles + 127) / 128, 128, 0, st>>>(counts, nchunks, ntiles, total);
    BIN_TRY(cudaGetLastError());
    tile_scan_kernel<<<1, 1024, 0, st>>>(total, ntiles, p->tile_off);
    BIN_TRY(cudaGetLastError());
    bin_scatter_kernel<<<nb, 256, 0, st>>>(key, lrank, counts, p->tile_off, ntiles, g, dcf, N, p->perm,
                                           p->gsorted, p->wsorted);
    BIN_TRY(cudaGetLastError());
    // work items on the host (plan time): split every tile into chunks of <= spread_chunk samples
    std::vector<int32_t> off(ntiles + 1);
    BIN_TRY(cudaMemcpyAsync(off.data(), p->tile_off, sizeof(int32_t) * (ntiles + 1), cudaMemcpyDeviceToHost, st));
    BIN_TRY(cudaStreamSynchronize(st));
    std::vector<WorkItem> items;
    const int M = p->spread_chunk;
    for (int t = 0; t < ntiles; ++t) {
        for (int s = off[t]; s < off[t + 1]; s += M) {
            WorkItem w;
            w.tile = t;
            w.start = s;
            w.count = std::min(M, off[t + 1] - s);
            items.push_back(w);
        }
    }
    p->nitems = (int)items.size();
    if (p->nitems > 0) {
        BIN_TRY(cudaMalloc(&p->items, sizeof(WorkItem) * items.size()));
        BIN_TRY(cudaMemcpy(p->items, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice));
    }
    cleanup();
#undef BIN_TRY
    return rc;
}

// ------------------------------------------------------------------------------------------
// Sliding-window interpolation and spreading on the coil-interleaved grid [G][C].
//
// Samples are sorted by tile and, inside a tile, by acquisition order, so consecutive sorted
// samples lie a fraction of a grid unit apart along a readout and their W^3 boxes mostly
// coincide.  One warp walks a run of consecutive samples; its lanes are (coil, z-slice) pairs
// of one coil chunk, so every lane sees the same sample and the window updates are uniform
// across the warp.  A lane keeps P of the 4 z-planes of the box (4x4 values each) in registers:
// planes are held by z residue modulo 4, so a move along z replaces one plane in place; a move
// along y or x shifts every held plane by one row/column and touches only the entering
// (interp: loads) or leaving (spread: atomic adds) row/column.  Kernel weights phi come from a
// 2049-point table of phi on [0, 2] (linear interpolation, relative error below 3e-7, built in
// double on the host); 12 lanes evaluate one weight each and the warp shares them by shuffles.
enum { OUT_USER = 0, OUT_RESID = 1, OUT_SORTED = 2 };
constexpr int kPhiTable = 2048;

struct GridArgs {
    float2* grid;          // [G][C] (coil-interleaved)
    int C;                 // interleave stride = coils of the operator call
    int c0, gsize;         // coil chunk handled by this launch
    int Gz, Gy, Gx;
    const float* rec;      // [N][16] per-sample records (weights, box, sqrt(w), user index)
    int64_t N;
    int chunk;             // samples per warp
};

__device__ __forceinline__ float phi_lookup(const float* __restrict__ tab, float u) {
    float p = fabsf(u) * (0.5f * kPhiTable);
    int i = (int)p;
    i = min(i, kPhiTable - 1);
    const float f = p - (float)i;
    const float a = tab[i], b = tab[i + 1];
    return fmaf(f, b - a, a);
}

__device__ __forceinline__ int wrapc(int j, int G) {   // j in [-G, 2G)
    return j < 0 ? j + G : (j >= G ? j - G : j);
}

template <int ND>
struct SampleBox {
    int jz, jy, jx;        // wrapped box starts
    float wz[kW], wy[kW], wx[kW];
    float sw;              // sqrt(w)
    int perm;              // user index
};

// Per-sample record of 16 words, computed once per plan: the 12 kernel weights (z, y, x, with
// the (-1)^(j + G/2) sign of the centred DFT folded in), the wrapped box start packed as
// 10 + 10 + 10 bits, sqrt(w) and the user index of the sample.
constexpr int kRec = 16;

__global__ void sample_record_kernel(const float* __restrict__ gs, const float* __restrict__ ws,
                                     const int32_t* __restrict__ perm, const float* __restrict__ tab_g, int64_t N,
                                     int nd, int Gz, int Gy, int Gx, float* __restrict__ rec) {
    __shared__ float tab[kPhiTable + 1];
    for (int i = threadIdx.x; i <= kPhiTable; i += blockDim.x) tab[i] = tab_g[i];
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    float* r = rec + s * kRec;
    int jb[3] = {0, 0, 0};
    const int Gs[3] = {Gz, Gy, Gx};
    for (int ax = 0; ax < 3; ++ax) {
        const bool used = ax >= 3 - nd;
        const float g = gs[s * 3 + ax];
        const int j0 = used ? (int)floorf(g) - (kW / 2 - 1) : 0;
        for (int a = 0; a < kW; ++a) {
            float v = (a == 0) ? 1.f : 0.f;
            if (used) {
                const int j = j0 + a;
                v = phi_lookup(tab, g - (float)j);
                if ((j + Gs[ax] / 2) & 1) v = -v;
            }
            r[ax * kW + a] = v;
        }
        jb[ax] = used ? wrapc(j0, Gs[ax]) : 0;
    }
    r[12] = __int_as_float(jb[0] | (jb[1] << 10) | (jb[2] << 20));
    r[13] = ws[s];
    r[14] = __int_as_float(perm[s]);
    r[15] = 0.f;
}

// lane l holds word (l mod 16) of the sample's record; every lane gets the weights by shuffles
__device__ __forceinline__ float rec_word(const GridArgs& A, int64_t s, int lane) {
    return (s < A.N) ? __ldg(A.rec + s * kRec + (lane & (kRec - 1))) : 0.f;
}

template <int ND>
__device__ __forceinline__ void sample_box(float w, int lane, SampleBox<ND>& B) {
#pragma unroll
    for (int a = 0; a < kW; ++a) {
        B.wz[a] = __shfl_sync(0xffffffffu, w, a);
        B.wy[a] = __shfl_sync(0xffffffffu, w, kW + a);
        B.wx[a] = __shfl_sync(0xffffffffu, w, 2 * kW + a);
    }
    const int packed = __float_as_int(__shfl_sync(0xffffffffu, w, 12));
    B.sw = __shfl_sync(0xffffffffu, w, 13);
    B.perm = __float_as_int(__shfl_sync(0xffffffffu, w, 14));
    B.jz = packed & 1023;
    B.jy = (packed >> 10) & 1023;
    B.jx = (packed >> 20) & 1023;
}

__device__ __forceinline__ int64_t gaddr(const GridArgs& A, int z, int y, int x, int c) {
    return (((int64_t)z * A.Gy + y) * A.Gx + x) * A.C + c;
}

// Per-lane window: P planes of 4x4 values; plane p holds z residue q + p*s (s = 4 / P lanes per
// coil).  zc[p] is the (wrapped) z of the plane or -1 when empty.
template <int P>
struct Win {
    float2 v[P][kW][kW];
    int zc[P];
};

// Minimum resident CTAs per SM requested from the register allocator for the gridding kernels, by
// planes per lane P (1: 8 coils per warp, 2: 16, 4: 32); 1 leaves the allocator unconstrained. Four
// CTAs (128 registers, a few spilled words) measured faster for the spread at P = 1 and the
// interpolation at P = 2 than the unconstrained allocation (3 CTAs) on the 128^3 and
// 160x256x256 cones workloads.
#ifndef CS_INTERP_MINB_P1
#define CS_INTERP_MINB_P1 1
#endif
#ifndef CS_INTERP_MINB_P2
#define CS_INTERP_MINB_P2 4
#endif
#ifndef CS_SPREAD_MINB_P1
#define CS_SPREAD_MINB_P1 4
#endif
#ifndef CS_SPREAD_MINB_P2
#define CS_SPREAD_MINB_P2 1
#endif
#define CS_INTERP_MINB(P) ((P) == 1 ? CS_INTERP_MINB_P1 : (P) == 2 ? CS_INTERP_MINB_P2 : 1)
#define CS_SPREAD_MINB(P) ((P) == 1 ? CS_SPREAD_MINB_P1 : (P) == 2 ? CS_SPREAD_MINB_P2 : 1)

template <int ND, int P>
__global__ void __launch_bounds__(128, CS_INTERP_MINB(P)) interp_kernel(GridArgs A, int mode, const float2* __restrict__ ysub,
                                                     float2* __restrict__ out) {
    constexpr int S = (ND == 3) ? 4 / P : 1;     // lanes per coil
    const int lane = threadIdx.x & 31;
    const int coil_l = lane / S, slice = lane % S;
    const bool active = coil_l < A.gsize;
    const int c = A.c0 + (active ? coil_l : 0);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t s0 = warp * A.chunk;
    if (s0 >= A.N) return;                       // whole warp exits together
    const int64_t s1 = min(A.N, s0 + A.chunk);
    Win<P> W;
#pragma unroll
    for (int p = 0; p < P; ++p) W.zc[p] = -1;
    int cy = -100, cx = -100;
    float wnext = rec_word(A, s0, lane);
    for (int64_t s = s0; s < s1; ++s) {
        SampleBox<ND> B;
        sample_box<ND>(wnext, lane, B);
        wnext = rec_word(A, s + 1, lane);   // prefetch the next sample's record
        const int dy = B.jy - cy, dx = B.jx - cx;
        if (abs(dy) > 1 || abs(dx) > 1) {
#pragma unroll
            for (int p = 0; p < P; ++p) W.zc[p] = -1;    // reload every plane below
        } else {
            if (dy != 0) {
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    if (dy > 0) {
#pragma unroll
                        for (int b = 0; b < kW - 1; ++b)
#pragma unroll
                            for (int d = 0; d < kW; ++d) W.v[p][b][d] = W.v[p][b + 1][d];
                    } else {
#pragma unroll
                        for (int b = kW - 1; b > 0; --b)
#pragma unroll
                            for (int d = 0; d < kW; ++d) W.v[p][b][d] = W.v[p][b - 1][d];
                    }
                    if (W.zc[p] >= 0 && active) {
                        if (dy > 0) {
                            const int yy = wrapc(B.jy + kW - 1, A.Gy);
#pragma unroll
                            for (int d = 0; d < kW; ++d)
                                W.v[p][kW - 1][d] = __ldg(A.grid + gaddr(A, W.zc[p], yy, wrapc(cx + d, A.Gx), c));
                        } else {
                            const int yy = B.jy;
#pragma unroll
                            for (int d = 0; d < kW; ++d)
                                W.v[p][0][d] = __ldg(A.grid + gaddr(A, W.zc[p], yy, wrapc(cx + d, A.Gx), c));
                        }
                    }
                }
                cy = B.jy;
            }
            if (dx != 0) {
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    if (dx > 0) {
#pragma unroll
                        for (int b = 0; b < kW; ++b)
#pragma unroll
                            for (int d = 0; d < kW - 1; ++d) W.v[p][b][d] = W.v[p][b][d + 1];
                    } else {
#pragma unroll
                        for (int b = 0; b < kW; ++b)
#pragma unroll
                            for (int d = kW - 1; d > 0; --d) W.v[p][b][d] = W.v[p][b][d - 1];
                    }
                    if (W.zc[p] >= 0 && active) {
                        if (dx > 0) {
                            const int xx = wrapc(B.jx + kW - 1, A.Gx);
#pragma unroll
                            for (int b = 0; b < kW; ++b)
                                W.v[p][b][kW - 1] = __ldg(A.grid + gaddr(A, W.zc[p], wrapc(cy + b, A.Gy), xx, c));
                        } else {
                            const int xx = B.jx;
#pragma unroll
                            for (int b = 0; b < kW; ++b)
                                W.v[p][b][0] = __ldg(A.grid + gaddr(A, W.zc[p], wrapc(cy + b, A.Gy), xx, c));
                        }
                    }
                }
                cx = B.jx;
            }
        }
        cy = B.jy;
        cx = B.jx;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int p = 0; p < P; ++p) {
            // z of this plane inside the box [jz, jz+3]
            int rel = 0, zw = 0;
            if (ND == 3) {
                const int q = slice + p * S;                       // residue held by this plane
                rel = (q - B.jz) & 3;
                zw = wrapc(B.jz + rel, A.Gz);
            }
            if (W.zc[p] != zw) {
                if (active) {
#pragma unroll
                    for (int b = 0; b < kW; ++b) {
                        const int yy = wrapc(cy + b, A.Gy);
#pragma unroll
                        for (int d = 0; d < kW; ++d) W.v[p][b][d] = __ldg(A.grid + gaddr(A, zw, yy, wrapc(cx + d, A.Gx), c));
                    }
                }
                W.zc[p] = zw;
            }
            const float wzp = (rel == 0) ? B.wz[0] : (rel == 1 ? B.wz[1] : (rel == 2 ? B.wz[2] : B.wz[3]));
            float2 pa = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < kW; ++b) {
                float2 r = make_float2(0.f, 0.f);
#pragma unroll
                for (int d = 0; d < kW; ++d) {
                    r.x = fmaf(B.wx[d], W.v[p][b][d].x, r.x);
                    r.y = fmaf(B.wx[d], W.v[p][b][d].y, r.y);
                }
                pa.x = fmaf(B.wy[b], r.x, pa.x);
                pa.y = fmaf(B.wy[b], r.y, pa.y);
            }
            acc.x = fmaf(wzp, pa.x, acc.x);
            acc.y = fmaf(wzp, pa.y, acc.y);
        }
        if (S > 1) {
#pragma unroll
            for (int o = 1; o < S; o <<= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            }
        }
        if (active && slice == 0) {
            acc = cscale(acc, B.sw);
            if (mode == OUT_USER) {
                out[(int64_t)c * A.N + B.perm] = acc;
            } else if (mode == OUT_RESID) {
                out[s * A.C + c] = csub(acc, ysub[(int64_t)c * A.N + B.perm]);
            } else {
                out[s * A.C + c] = acc;
            }
        }
    }
}

__device__ __forceinline__ void red_add(float2* p, float2 v) {
    if (v.x != 0.f || v.y != 0.f) atomicAdd(p, v);
}

template <int ND, int P>
__global__ void __launch_bounds__(128, CS_SPREAD_MINB(P)) spread_kernel(GridArgs A, const float2* __restrict__ yin, int sorted_in) {
    constexpr int S = (ND == 3) ? 4 / P : 1;
    const int lane = threadIdx.x & 31;
    const int coil_l = lane / S, slice = lane % S;
    const bool active = coil_l < A.gsize;
    const int c = A.c0 + (active ? coil_l : 0);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t s0 = warp * A.chunk;
    if (s0 >= A.N) return;
    const int64_t s1 = min(A.N, s0 + A.chunk);
    Win<P> W;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        W.zc[p] = -1;
#pragma unroll
        for (int b = 0; b < kW; ++b)
#pragma unroll
            for (int d = 0; d < kW; ++d) W.v[p][b][d] = make_float2(0.f, 0.f);
    }
    int cy = -100, cx = -100;
    auto flush_plane = [&](int p) {
        if (W.zc[p] >= 0 && active) {
#pragma unroll
            for (int b = 0; b < kW; ++b) {
                const int yy = wrapc(cy + b, A.Gy);
#pragma unroll
                for (int d = 0; d < kW; ++d) red_add(A.grid + gaddr(A, W.zc[p], yy, wrapc(cx + d, A.Gx), c), W.v[p][b][d]);
            }
        }
#pragma unroll
        for (int b = 0; b < kW; ++b)
#pragma unroll
            for (int d = 0; d < kW; ++d) W.v[p][b][d] = make_float2(0.f, 0.f);
    };
    float wnext = rec_word(A, s0, lane);
    // the sample value: sorted scratch [N][C] (prefetched one sample ahead) or user order [C][N]
    auto load_v = [&](int64_t s, int perm) -> float2 {
        if (!active || s >= A.N) return make_float2(0.f, 0.f);
        return sorted_in ? yin[s * A.C + c] : yin[(int64_t)c * A.N + perm];
    };
    float2 vnext = sorted_in ? load_v(s0, 0) : make_float2(0.f, 0.f);
    for (int64_t s = s0; s < s1; ++s) {
        SampleBox<ND> B;
        sample_box<ND>(wnext, lane, B);
        float2 v = sorted_in ? vnext : load_v(s, B.perm);
        wnext = rec_word(A, s + 1, lane);
        if (sorted_in) vnext = load_v(s + 1, 0);
        const int dy = B.jy - cy, dx = B.jx - cx;
        if (abs(dy) > 1 || abs(dx) > 1) {
#pragma unroll
            for (int p = 0; p < P; ++p) {
                flush_plane(p);
                W.zc[p] = -1;
            }
        } else {
            if (dy != 0) {
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    if (dy > 0) {
                        if (W.zc[p] >= 0 && active) {
                            const int yy = cy;   // leaving row 0
#pragma unroll
                            for (int d = 0; d < kW; ++d) red_add(A.grid + gaddr(A, W.zc[p], yy, wrapc(cx + d, A.Gx), c), W.v[p][0][d]);
                        }
#pragma unroll
                        for (int b = 0; b < kW - 1; ++b)
#pragma unroll
                            for (int d = 0; d < kW; ++d) W.v[p][b][d] = W.v[p][b + 1][d];
#pragma unroll
                        for (int d = 0; d < kW; ++d) W.v[p][kW - 1][d] = make_float2(0.f, 0.f);
                    } else {
                        if (W.zc[p] >= 0 && active) {
                            const int yy = wrapc(cy + kW - 1, A.Gy);   // leaving row 3
#pragma unroll
                            for (int d = 0; d < kW; ++d) red_add(A.grid + gaddr(A, W.zc[p], yy, wrapc(cx + d, A.Gx), c), W.v[p][kW - 1][d]);
                        }
#pragma unroll
                        for (int b = kW - 1; b > 0; --b)
#pragma unroll
                            for (int d = 0; d < kW; ++d) W.v[p][b][d] = W.v[p][b - 1][d];
#pragma unroll
                        for (int d = 0; d < kW; ++d) W.v[p][0][d] = make_float2(0.f, 0.f);
                    }
                }
                cy = B.jy;
            }
            if (dx != 0) {
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    if (dx > 0) {
                        if (W.zc[p] >= 0 && active) {
                            const int xx = cx;   // leaving column 0
#pragma unroll
                            for (int b = 0; b < kW; ++b) red_add(A.grid + gaddr(A, W.zc[p], wrapc(cy + b, A.Gy), xx, c), W.v[p][b][0]);
                        }
#pragma unroll
                        for (int b = 0; b < kW; ++b)
#pragma unroll
                            for (int d = 0; d < kW - 1; ++d) W.v[p][b][d] = W.v[p][b][d + 1];
#pragma unroll
                        for (int b = 0; b < kW; ++b) W.v[p][b][kW - 1] = make_float2(0.f, 0.f);
                    } else {
                        if (W.zc[p] >= 0 && active) {
                            const int xx = wrapc(cx + kW - 1, A.Gx);   // leaving column 3
#pragma unroll
                            for (int b = 0; b < kW; ++b) red_add(A.grid + gaddr(A, W.zc[p], wrapc(cy + b, A.Gy), xx, c), W.v[p][b][kW - 1]);
                        }
#pragma unroll
                        for (int b = 0; b < kW; ++b)
#pragma unroll
                            for (int d = kW - 1; d > 0; --d) W.v[p][b][d] = W.v[p][b][d - 1];
#pragma unroll
                        for (int b = 0; b < kW; ++b) W.v[p][b][0] = make_float2(0.f, 0.f);
                    }
                }
                cx = B.jx;
            }
        }
        cy = B.jy;
        cx = B.jx;
        v = cscale(v, B.sw);
#pragma unroll
        for (int p = 0; p < P; ++p) {
            int rel = 0, zw = 0;
            if (ND == 3) {
                const int q = slice + p * S;
                rel = (q - B.jz) & 3;
                zw = wrapc(B.jz + rel, A.Gz);
            }
            if (W.zc[p] != zw) {
                flush_plane(p);
                W.zc[p] = zw;
            }
            const float wzp = (rel == 0) ? B.wz[0] : (rel == 1 ? B.wz[1] : (rel == 2 ? B.wz[2] : B.wz[3]));
            const float2 va = cscale(v, wzp);
#pragma unroll
            for (int b = 0; b < kW; ++b) {
                const float2 vb = cscale(va, B.wy[b]);
#pragma unroll
                for (int d = 0; d < kW; ++d) {
                    W.v[p][b][d].x = fmaf(B.wx[d], vb.x, W.v[p][b][d].x);
                    W.v[p][b][d].y = fmaf(B.wx[d], vb.y, W.v[p][b][d].y);
                }
            }
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) flush_plane(p);
}

static float2* grid_buffer(const cs_plan* p) { return p->ndim == 3 ? p->bufA : p->bufB; }

static GridArgs make_grid_args(const cs_plan* p, int ncoils) {
    GridArgs A;
    A.grid = grid_buffer(p);
    A.C = ncoils;
    A.c0 = 0;
    A.gsize = 0;
    A.Gz = p->grid[0];
    A.Gy = p->grid[1];
    A.Gx = p->grid[2];
    A.rec = p->rec;
    A.N = p->N;
    A.chunk = p->interp_chunk;
    return A;
}

// Launch one kernel per coil chunk: a chunk of g <= 8 coils uses 4 lanes per coil holding one
// plane each (P = 1), g <= 16 two lanes with two planes, g <= 32 one lane with all 4 planes;
// always one sample stream per warp.
template <bool SPREAD>
static cs_status launch_grid_op(const cs_plan* p, int ncoils, int mode, const float2* ysub, float2* out,
                                const float2* yin, int sorted_in, cudaStream_t st) {
    GridArgs A = make_grid_args(p, ncoils);
    const int64_t warps = (p->N + A.chunk - 1) / A.chunk;
    const unsigned nb = (unsigned)((warps * 32 + 127) / 128);
    if (nb == 0) return CS_OK;
    const int cmax = SPREAD ? p->spread_coils : p->interp_coils;   // 8, 16 or 32 coils per warp
    const int nch = (ncoils + cmax - 1) / cmax;
    const int cbal = (ncoils + nch - 1) / nch;                      // balanced chunk size
    for (int c0 = 0; c0 < ncoils; c0 += cbal) {
        const int g = std::min(cbal, ncoils - c0);
        A.c0 = c0;
        A.gsize = g;
        int P = 4;
        if (p->ndim == 3) P = (g <= 8) ? 1 : (g <= 16 ? 2 : 4);
        prof_begin(SPREAD ? ST_SPREAD : ST_INTERP, st);
        if (p->ndim == 2) {
            if (SPREAD) spread_kernel<2, 1><<<nb, 128, 0, st>>>(A, yin, sorted_in);
            else interp_kernel<2, 1><<<nb, 128, 0, st>>>(A, mode, ysub, out);
        } else if (P == 1) {
            if (SPREAD) spread_kernel<3, 1><<<nb, 128, 0, st>>>(A, yin, sorted_in);
            else interp_kernel<3, 1><<<nb, 128, 0, st>>>(A, mode, ysub, out);
        } else if (P == 2) {
            if (SPREAD) spread_kernel<3, 2><<<nb, 128, 0, st>>>(A, yin, sorted_in);
            else interp_kernel<3, 2><<<nb, 128, 0, st>>>(A, mode, ysub, out);
        } else {
            if (SPREAD) spread_kernel<3, 4><<<nb, 128, 0, st>>>(A, yin, sorted_in);
            else interp_kernel<3, 4><<<nb, 128, 0, st>>>(A, mode, ysub, out);
        }
        CS_LAUNCH_CHECK();
        prof_end(SPREAD ? ST_SPREAD : ST_INTERP, st);
    }
    return CS_OK;
}

cs_status nufft_records(cs_plan* p, cudaStream_t st) {
    CS_TRY_CUDA(cudaMalloc(&p->rec, sizeof(float) * kRec * (size_t)p->N));
    sample_record_kernel<<<(unsigned)((p->N + 255) / 256), 256, 0, st>>>(p->gsorted, p->wsorted, p->perm, p->phi, p->N,
                                                                      p->ndim, p->grid[0], p->grid[1], p->grid[2], p->rec);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

// y (user order) = sqrt(w) interp(grid); with ysub: ktmp (sorted) = sqrt(w) interp(grid) - y
cs_status nufft_interp(const cs_plan* p, int ncoils, float2* y, const float2* ysub, cudaStream_t st) {
    if (ysub) return launch_grid_op<false>(p, ncoils, OUT_RESID, ysub, p->ktmp, nullptr, 0, st);
    return launch_grid_op<false>(p, ncoils, OUT_USER, nullptr, y, nullptr, 0, st);
}

// grid = spread(sqrt(w) y); y in user order (sorted_in = 0) or the sorted scratch ktmp
cs_status nufft_spread(const cs_plan* p, int ncoils, const float2* y, int sorted_in, cudaStream_t st) {
    float2* grid = grid_buffer(p);
    CS_TRY_CUDA(cudaMemsetAsync(grid, 0, sizeof(float2) * (size_t)p->G * ncoils, st));
    if (ncoils == 0) return CS_OK;
    return launch_grid_op<true>(p, ncoils, 0, nullptr, nullptr, sorted_in ? p->ktmp : y, sorted_in, st);
}

// normal operator on the grid: ktmp = w^1/2 interp(grid) (sorted), then grid = spread(w^1/2 ktmp)
cs_status nufft_interp_spread(const cs_plan* p, int ncoils, cudaStream_t st) {
    CS_PROPAGATE(launch_grid_op<false>(p, ncoils, OUT_SORTED, nullptr, p->ktmp, nullptr, 0, st));
    return nufft_spread(p, ncoils, nullptr, 1, st);
}

}  // namespace cs
