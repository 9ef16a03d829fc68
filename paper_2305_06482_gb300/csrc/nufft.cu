// Kaiser-Bessel gridding for the non-uniform Fourier operator F~_n (Sec. 2.1, Beatty et al.
// 2005): sample binning, interpolation (forward) and spreading (adjoint).
//
// Discretisation (identical to the CPU restatement, bit for bit where integers are decided):
//   g   = fmaf(f, G, G/2) in float32 per axis            (grid coordinate of a sample)
//   j0  = floor(g) - 1                                  (first of the W = 4 box indices)
//   phi(u) = I0(beta sqrt(1 - (u/2)^2)) / I0(beta),     beta = pi sqrt((W/a)^2 (a-1/2)^2 - 0.8)
//   tile = floor((j0 mod G) / T) per axis, linear id (z, y, x) with x fastest.
// The forward grid is produced without the output modulation of the centred DFT; the sign
// (-1)^(j + G/2) of every grid index is folded into the interpolation weights instead.
#include <cmath>
#include <cstdio>

#include "cs_internal.cuh"

namespace cs {

constexpr int kW = 4;

struct KbAxis {
    int G;
    float beta;
    float inv_i0b;
};

__device__ __forceinline__ void kb_weights(float g, const KbAxis& ax, int& j0, float w[kW]) {
    const float fl = floorf(g);
    j0 = (int)fl - (kW / 2 - 1);
    const int half = ax.G / 2;
#pragma unroll
    for (int a = 0; a < kW; ++a) {
        const int j = j0 + a;
        const float u = g - (float)j;               // in [-2, 2)
        const float t = 1.0f - 0.25f * u * u;
        float v = (t > 0.f) ? cyl_bessel_i0f(ax.beta * sqrtf(t)) * ax.inv_i0b : ax.inv_i0b * (t == 0.f);
        if ((j + half) & 1) v = -v;                  // (-1)^(j + G/2) of the centred DFT
        w[a] = v;
    }
}

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
// interpolation: one thread per sorted sample, all coils (weights computed once per sample)
enum { OUT_USER = 0, OUT_RESID = 1, OUT_SORTED = 2 };

struct GridArgs {
    const float2* grid;    // [C][G]
    int64_t G;
    int Gz, Gy, Gx;
    KbAxis az, ay, ax;
    const float* gs;       // [N][3]
    const float* ws;       // [N]
    const int32_t* perm;
    int64_t N;
    int ncoils;
};

template <int ND>
__global__ void __launch_bounds__(256) interp_kernel(GridArgs A, int mode, const float2* __restrict__ ysub,
                                                     float2* __restrict__ out) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.N) return;
    int jz = 0, jy, jx;
    float wz[kW] = {1.f, 0.f, 0.f, 0.f}, wy[kW], wx[kW];
    if (ND == 3) kb_weights(A.gs[s * 3 + 0], A.az, jz, wz);
    kb_weights(A.gs[s * 3 + 1], A.ay, jy, wy);
    kb_weights(A.gs[s * 3 + 2], A.ax, jx, wx);
    int iz[kW], iy[kW], ix[kW];
#pragma unroll
    for (int a = 0; a < kW; ++a) {
        iz[a] = (ND == 3) ? wrapi(jz + a, A.Gz) : 0;
        iy[a] = wrapi(jy + a, A.Gy);
        ix[a] = wrapi(jx + a, A.Gx);
    }
    const float sw = A.ws[s];
    const int32_t ps = A.perm[s];
    for (int c = 0; c < A.ncoils; ++c) {
        const float2* gc = A.grid + (int64_t)c * A.G;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int a = 0; a < (ND == 3 ? kW : 1); ++a) {
#pragma unroll
            for (int b = 0; b < kW; ++b) {
                const float2* row = gc + ((int64_t)iz[a] * A.Gy + iy[b]) * A.Gx;
                const float wab = wz[a] * wy[b];
                float2 r = make_float2(0.f, 0.f);
#pragma unroll
                for (int d = 0; d < kW; ++d) {
                    const float2 v = __ldg(row + ix[d]);
                    r.x = fmaf(wx[d], v.x, r.x);
                    r.y = fmaf(wx[d], v.y, r.y);
                }
                acc.x = fmaf(wab, r.x, acc.x);
                acc.y = fmaf(wab, r.y, acc.y);
            }
        }
        acc = cscale(acc, sw);
        if (mode == OUT_USER) {
            out[(int64_t)c * A.N + ps] = acc;
        } else if (mode == OUT_RESID) {
            out[(int64_t)c * A.N + s] = csub(acc, ysub[(int64_t)c * A.N + ps]);
        } else {
            out[(int64_t)c * A.N + s] = acc;
        }
    }
}

// ------------------------------------------------------------------------------------------
// spreading: one CTA per (work item, coil); the tile plus its high-side halo of W-1 points is
// accumulated in shared memory, then added to the grid (wrapping modulo G).
struct SpreadArgs {
    GridArgs g;
    float2* grid;
    const float2* yin;      // user order [C][N] or sorted [C][N]
    int sorted_in;
    const WorkItem* items;
    int tz, ty, tx;         // tile sizes
    int ntz, nty, ntx;
};

template <int ND>
__global__ void __launch_bounds__(256) spread_kernel(SpreadArgs S) {
    extern __shared__ float2 reg[];
    const WorkItem it = S.items[blockIdx.x];
    const int c = blockIdx.y;
    const int Rz = (ND == 3) ? S.tz + kW - 1 : 1, Ry = S.ty + kW - 1, Rx = S.tx + kW - 1;
    const int R = Rz * Ry * Rx;
    for (int e = threadIdx.x; e < R; e += blockDim.x) reg[e] = make_float2(0.f, 0.f);
    int t = it.tile;
    const int tcx = t % S.ntx;
    t /= S.ntx;
    const int tcy = t % S.nty;
    const int tcz = t / S.nty;
    const int oz = tcz * S.tz, oy = tcy * S.ty, ox = tcx * S.tx;
    __syncthreads();
    const GridArgs& A = S.g;
    for (int s = it.start + threadIdx.x; s < it.start + it.count; s += blockDim.x) {
        int jz = 0, jy, jx;
        float wz[kW] = {1.f, 0.f, 0.f, 0.f}, wy[kW], wx[kW];
        if (ND == 3) kb_weights(A.gs[s * 3 + 0], A.az, jz, wz);
        kb_weights(A.gs[s * 3 + 1], A.ay, jy, wy);
        kb_weights(A.gs[s * 3 + 2], A.ax, jx, wx);
        const int lz = (ND == 3) ? wrapi(jz, A.Gz) - oz : 0;
        const int ly = wrapi(jy, A.Gy) - oy;
        const int lx = wrapi(jx, A.Gx) - ox;
        float2 v = S.sorted_in ? S.yin[(int64_t)c * A.N + s] : S.yin[(int64_t)c * A.N + A.perm[s]];
        v = cscale(v, A.ws[s]);
#pragma unroll
        for (int a = 0; a < (ND == 3 ? kW : 1); ++a) {
#pragma unroll
            for (int b = 0; b < kW; ++b) {
                const float wab = wz[a] * wy[b];
                float2* row = reg + ((lz + a) * Ry + (ly + b)) * Rx + lx;
#pragma unroll
                for (int d = 0; d < kW; ++d) {
                    const float w = wab * wx[d];
                    atomicAdd(&row[d].x, w * v.x);
                    atomicAdd(&row[d].y, w * v.y);
                }
            }
        }
    }
    __syncthreads();
    float2* gc = S.grid + (int64_t)c * A.G;
    for (int e = threadIdx.x; e < R; e += blockDim.x) {
        const float2 v = reg[e];
        if (v.x == 0.f && v.y == 0.f) continue;
        const int rx = e % Rx;
        const int ry = (e / Rx) % Ry;
        const int rz = e / (Rx * Ry);
        const int gz = (ND == 3) ? wrapi(oz + rz, A.Gz) : 0;
        const int gy = wrapi(oy + ry, A.Gy);
        const int gx = wrapi(ox + rx, A.Gx);
        atomicAdd(reinterpret_cast<float2*>(gc + ((int64_t)gz * A.Gy + gy) * A.Gx + gx), v);
    }
}

static GridArgs make_grid_args(const cs_plan* p, int ncoils, const float2* grid) {
    GridArgs A;
    A.grid = grid;
    A.G = p->G;
    A.Gz = p->grid[0];
    A.Gy = p->grid[1];
    A.Gx = p->grid[2];
    const float i0b = (float)(1.0 / std::cyl_bessel_i(0.0, (double)p->beta));
    A.az = KbAxis{p->grid[0], p->beta, i0b};
    A.ay = KbAxis{p->grid[1], p->beta, i0b};
    A.ax = KbAxis{p->grid[2], p->beta, i0b};
    A.gs = p->gsorted;
    A.ws = p->wsorted;
    A.perm = p->perm;
    A.N = p->N;
    A.ncoils = ncoils;
    return A;
}

static float2* grid_buffer(const cs_plan* p) { return p->ndim == 3 ? p->bufA : p->bufB; }

static cs_status launch_interp(const cs_plan* p, int ncoils, int mode, const float2* ysub, float2* out,
                               cudaStream_t st) {
    GridArgs A = make_grid_args(p, ncoils, grid_buffer(p));
    const unsigned nb = (unsigned)((p->N + 255) / 256);
    if (nb == 0) return CS_OK;
    if (p->ndim == 3) interp_kernel<3><<<nb, 256, 0, st>>>(A, mode, ysub, out);
    else interp_kernel<2><<<nb, 256, 0, st>>>(A, mode, ysub, out);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

// y (user order) = sqrt(w) interp(grid)
cs_status nufft_interp(const cs_plan* p, int ncoils, float2* y, const float2* ysub, cudaStream_t st) {
    if (ysub) return launch_interp(p, ncoils, OUT_RESID, ysub, p->ktmp, st);
    return launch_interp(p, ncoils, OUT_USER, nullptr, y, st);
}

// grid = spread(sqrt(w) y); y in user order (sorted_in = 0) or the sorted scratch (ktmp)
cs_status nufft_spread(const cs_plan* p, int ncoils, const float2* y, int sorted_in, cudaStream_t st) {
    float2* grid = grid_buffer(p);
    CS_TRY_CUDA(cudaMemsetAsync(grid, 0, sizeof(float2) * (size_t)p->G * ncoils, st));
    if (p->nitems == 0 || ncoils == 0) return CS_OK;
    SpreadArgs S;
    S.g = make_grid_args(p, ncoils, grid);
    S.grid = grid;
    S.yin = sorted_in ? p->ktmp : y;
    S.sorted_in = sorted_in;
    S.items = p->items;
    S.tz = p->tile[0];
    S.ty = p->tile[1];
    S.tx = p->tile[2];
    S.ntz = p->ntiles[0];
    S.nty = p->ntiles[1];
    S.ntx = p->ntiles[2];
    const int Rz = p->ndim == 3 ? p->tile[0] + kW - 1 : 1;
    const size_t sm = sizeof(float2) * (size_t)Rz * (p->tile[1] + kW - 1) * (p->tile[2] + kW - 1);
    dim3 grd((unsigned)p->nitems, (unsigned)ncoils);
    if (p->ndim == 3) {
        CS_TRY_CUDA(cudaFuncSetAttribute(spread_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        spread_kernel<3><<<grd, 256, sm, st>>>(S);
    } else {
        CS_TRY_CUDA(cudaFuncSetAttribute(spread_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        spread_kernel<2><<<grd, 256, sm, st>>>(S);
    }
    CS_LAUNCH_CHECK();
    return CS_OK;
}

// normal operator on the grid: ktmp = w^1/2 interp(grid) (sorted), then grid = spread(w^1/2 ktmp)
cs_status nufft_interp_spread(const cs_plan* p, int ncoils, cudaStream_t st) {
    CS_PROPAGATE(launch_interp(p, ncoils, OUT_SORTED, nullptr, p->ktmp, st));
    return nufft_spread(p, ncoils, nullptr, 1, st);
}

}  // namespace cs
