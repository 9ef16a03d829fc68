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
#include <type_traits>
#include <algorithm>
#include <vector>

#include "cs_internal.cuh"

namespace cs {

constexpr int kW = 4;

__device__ __forceinline__ int wrapi(int j, int G) {
    j %= G;
    return j < 0 ? j + G : j;
}

// ------------------------------------------------------------------------------------------
// binning
//
// Every sample gets a tile (floor(wrap(j0) / T) per axis; a remainder narrower than the kernel
// widens the last tile) and a halo class (bit a: its box reaches the next tile along axis a,
// z = 4, y = 2, x = 1; only axes with more than one tile).  Samples are stable-sorted by the key
// tile * 8 + class in two stable counting-sort passes (least significant key first: class, then
// tile), so that every tile's samples come in class runs, each in acquisition order.
__device__ __forceinline__ void tile_of(int jw, int G, int T, int nt, int* t, int* start, int* width) {
    int tt = jw / T;
    tt = tt < nt - 1 ? tt : nt - 1;
    *t = tt;
    *start = tt * T;
    *width = (tt == nt - 1) ? G - tt * T : T;
}

// coords: the trajectory [N][nd] in cycles/pixel (from_grid = 0) or grid coordinates [N][3] in
// user order (from_grid = 1, as a plan stores them)
__global__ void bin_keys_kernel(const float* __restrict__ coords, int from_grid, int64_t N, int nd, int3 G, int3 T,
                                int3 nt, float* __restrict__ gout, int32_t* __restrict__ j0out,
                                int32_t* __restrict__ tkey, int32_t* __restrict__ ckey) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int Gs[3] = {G.x, G.y, G.z}, Ts[3] = {T.x, T.y, T.z}, nts[3] = {nt.x, nt.y, nt.z};
    int64_t lin = 0;
    int cls = 0;
    for (int ax = 0; ax < 3; ++ax) {
        int jj = 0;
        float g = 0.f;
        if (ax >= 3 - nd) {
            const int a = ax - (3 - nd);
            if (from_grid) {
                g = coords[i * 3 + ax];
            } else {
                const float f = coords[i * nd + a];
                const float Gf = (float)Gs[ax];
                g = __fmaf_rn(f, Gf, 0.5f * Gf);
            }
            jj = (int)floorf(g) - (kW / 2 - 1);
            j0out[i * nd + a] = jj;
        }
        gout[i * 3 + ax] = g;
        int t, st, w;
        const int jw = wrapi(jj, Gs[ax]);
        tile_of(jw, Gs[ax], Ts[ax], nts[ax], &t, &st, &w);
        lin = lin * nts[ax] + t;
        if (ax >= 3 - nd && nts[ax] > 1 && jw - st >= w - (kW - 1)) cls |= 1 << (2 - ax);
    }
    tkey[i] = (int32_t)lin;
    ckey[i] = cls;
}

constexpr int kRankChunk = 8192;

// One warp per chunk of kRankChunk consecutive entries: stable rank of each entry among the
// chunk's entries of the same key (warp match + prefix popcount, processed in index order).
__global__ void chunk_rank_kernel(const int32_t* __restrict__ key, int64_t N, int nkeys,
                                  int32_t* __restrict__ lrank, int32_t* __restrict__ counts) {
    extern __shared__ int32_t running[];
    const int lane = threadIdx.x;
    const int64_t chunk = blockIdx.x;
    for (int t = lane; t < nkeys; t += 32) running[t] = 0;
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
    for (int t = lane; t < nkeys; t += 32) counts[chunk * (int64_t)nkeys + t] = running[t];
}

// per key: exclusive scan over chunks (in place) and the key total
__global__ void chunk_scan_kernel(int32_t* __restrict__ counts, int64_t nchunks, int nkeys, int32_t* __restrict__ total) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nkeys) return;
    int32_t run = 0;
    for (int64_t c = 0; c < nchunks; ++c) {
        const int32_t v = counts[c * nkeys + t];
        counts[c * nkeys + t] = run;
        run += v;
    }
    total[t] = run;
}

// single-CTA exclusive scan of key totals -> off[nkeys + 1]
__global__ void key_scan_kernel(const int32_t* __restrict__ total, int nkeys, int32_t* __restrict__ off) {
    __shared__ int32_t part[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = (nkeys + nt - 1) / nt;
    const int b = tid * per, e = min(nkeys, b + per);
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
        off[nkeys] = run;
    }
    __syncthreads();
    int32_t run = part[tid];
    for (int i = b; i < e; ++i) {
        off[i] = run;
        run += total[i];
    }
}

// sorted position of entry i: key offset + rank of its chunk + rank inside the chunk
__global__ void rank_scatter_kernel(const int32_t* __restrict__ key, const int32_t* __restrict__ lrank,
                                    const int32_t* __restrict__ cbase, const int32_t* __restrict__ koff, int nkeys,
                                    int64_t N, int32_t* __restrict__ order) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int k = key[i];
    const int64_t chunk = i / kRankChunk;
    order[(int64_t)koff[k] + cbase[chunk * nkeys + k] + lrank[i]] = (int32_t)i;
}

__global__ void gather_i32_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ idx, int64_t N,
                                  int32_t* __restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) dst[i] = src[idx[i]];
}

// final order: perm[pos] = sample; sorted grid coordinates, sqrt(dcf) and keys
__global__ void bin_final_kernel(const int32_t* __restrict__ perm1, const int32_t* __restrict__ perm2,
                                 const float* __restrict__ g, const float* __restrict__ w, int w_is_sqrt,
                                 const int32_t* __restrict__ tkey, const int32_t* __restrict__ ckey, int64_t N,
                                 int32_t* __restrict__ perm, float* __restrict__ gs, float* __restrict__ ws,
                                 int32_t* __restrict__ skey) {
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= N) return;
    const int32_t i = perm1[perm2[pos]];
    perm[pos] = i;
    gs[pos * 3 + 0] = g[(int64_t)i * 3 + 0];
    gs[pos * 3 + 1] = g[(int64_t)i * 3 + 1];
    gs[pos * 3 + 2] = g[(int64_t)i * 3 + 2];
    ws[pos] = w_is_sqrt ? w[i] : sqrtf(w[i]);
    skey[pos] = tkey[i] * 8 + ckey[i];
}

// off[k] = first sorted position whose key is >= k (k = 0 .. nkeys), by binary search
__global__ void lower_bound_kernel(const int32_t* __restrict__ skey, int64_t N, int nkeys, int32_t* __restrict__ off) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > nkeys) return;
    int64_t lo = 0, hi = N;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (skey[mid] < k) lo = mid + 1;
        else hi = mid;
    }
    off[k] = (int32_t)lo;
}

__global__ void tile_off_kernel(const int32_t* __restrict__ coff, int ntiles, int32_t* __restrict__ toff) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t <= ntiles) toff[t] = coff[(int64_t)t * 8];
}

// a plan's sorted grid coordinates and sqrt(dcf) back in user order (input of a re-binning)
__global__ void unsort_kernel(const int32_t* __restrict__ perm, const float* __restrict__ gs,
                              const float* __restrict__ ws, int64_t N, float* __restrict__ gu, float* __restrict__ wu) {
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= N) return;
    const int64_t i = perm[pos];
    if (!CS_INB(i, N)) return;
    gu[i * 3 + 0] = gs[pos * 3 + 0];
    gu[i * 3 + 1] = gs[pos * 3 + 1];
    gu[i * 3 + 2] = gs[pos * 3 + 2];
    wu[i] = ws[pos];
}

cs_status nufft_set_tiles(cs_plan* p, const int* tile3) {
    int t[3], nt[3], wm[3];
    int64_t tot = 1;
    const int nd = p->ndim;
    for (int a = 0; a < 3; ++a) {
        int v = (a >= 3 - nd) ? tile3[a] : 1;
        if (v <= 0) v = 16;
        v = std::min(v, p->grid[a]);
        CS_REQUIRE(a < 3 - nd || v >= kW || v == p->grid[a], CS_ERR_UNSUPPORTED_SIZE,
                   "tiles narrower than the kernel width (%d) are not supported", v);
        t[a] = v;
        const int rem = p->grid[a] % v;
        // a remainder narrower than the kernel widens the last tile instead of forming its own
        nt[a] = (rem > 0 && rem < kW && p->grid[a] >= v) ? p->grid[a] / v : (p->grid[a] + v - 1) / v;
        wm[a] = std::max(v, p->grid[a] - (nt[a] - 1) * v);
        tot *= nt[a];
    }
    CS_REQUIRE(tot <= 49152, CS_ERR_UNSUPPORTED_SIZE, "too many tiles (%lld); use a larger tile", (long long)tot);
    for (int a = 0; a < 3; ++a) {
        p->tile[a] = t[a];
        p->ntiles[a] = nt[a];
        p->wmax[a] = wm[a];
    }
    p->ntiles_total = tot;
    return CS_OK;
}

cs_status nufft_bin(cs_plan* p, const float* coords, const float* w, int from_grid, cudaStream_t st) {
    const int64_t N = p->N;
    const int nd = p->ndim;
    const int ntiles = (int)p->ntiles_total;
    CS_REQUIRE(ntiles <= 49152, CS_ERR_UNSUPPORTED_SIZE, "too many tiles (%d); use a larger tile", ntiles);
    const int64_t nchunks = (N + kRankChunk - 1) / kRankChunk;
    float* g = nullptr;
    int32_t *tkey = nullptr, *ckey = nullptr, *lrank = nullptr, *counts = nullptr, *total = nullptr, *koff = nullptr;
    int32_t *perm1 = nullptr, *key2 = nullptr, *perm2 = nullptr, *skey = nullptr;
    auto cleanup = [&]() {
        cudaFree(g);
        cudaFree(tkey);
        cudaFree(ckey);
        cudaFree(lrank);
        cudaFree(counts);
        cudaFree(total);
        cudaFree(koff);
        cudaFree(perm1);
        cudaFree(key2);
        cudaFree(perm2);
        cudaFree(skey);
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
    BIN_TRY(cudaMalloc(&tkey, sizeof(int32_t) * N));
    BIN_TRY(cudaMalloc(&ckey, sizeof(int32_t) * N));
    BIN_TRY(cudaMalloc(&lrank, sizeof(int32_t) * N));
    const int nkmax = ntiles > 8 ? ntiles : 8;   // the class pass has 8 keys
    BIN_TRY(cudaMalloc(&counts, sizeof(int32_t) * nchunks * nkmax));
    BIN_TRY(cudaMalloc(&total, sizeof(int32_t) * nkmax));
    BIN_TRY(cudaMalloc(&koff, sizeof(int32_t) * (nkmax + 1)));
    BIN_TRY(cudaMalloc(&perm1, sizeof(int32_t) * N));
    BIN_TRY(cudaMalloc(&key2, sizeof(int32_t) * N));
    BIN_TRY(cudaMalloc(&perm2, sizeof(int32_t) * N));
    BIN_TRY(cudaMalloc(&skey, sizeof(int32_t) * N));
    const int3 G3 = make_int3(p->grid[0], p->grid[1], p->grid[2]);
    const int3 T3 = make_int3(p->tile[0], p->tile[1], p->tile[2]);
    const int3 nt3 = make_int3(p->ntiles[0], p->ntiles[1], p->ntiles[2]);
    const unsigned nb = (unsigned)((N + 255) / 256);
    bin_keys_kernel<<<nb, 256, 0, st>>>(coords, from_grid, N, nd, G3, T3, nt3, g, p->j0, tkey, ckey);
    BIN_TRY(cudaGetLastError());
    // one stable counting-sort pass: order[pos] = index of the entry at sorted position pos
    auto pass = [&](const int32_t* key, int nkeys, int32_t* order) -> cudaError_t {
        const size_t rsm = sizeof(int32_t) * nkeys;
        cudaError_t e = cudaFuncSetAttribute(chunk_rank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm);
        if (e != cudaSuccess) return e;
        chunk_rank_kernel<<<(unsigned)nchunks, 32, rsm, st>>>(key, N, nkeys, lrank, counts);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        chunk_scan_kernel<<<(nkeys + 127) / 128, 128, 0, st>>>(counts, nchunks, nkeys, total);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        key_scan_kernel<<<1, 1024, 0, st>>>(total, nkeys, koff);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        rank_scatter_kernel<<<nb, 256, 0, st>>>(key, lrank, counts, koff, nkeys, N, order);
        return cudaGetLastError();
    };
    BIN_TRY(pass(ckey, 8, perm1));                                   // by class (stable)
    gather_i32_kernel<<<nb, 256, 0, st>>>(tkey, perm1, N, key2);
    BIN_TRY(cudaGetLastError());
    BIN_TRY(pass(key2, ntiles, perm2));                              // then by tile (stable)
    bin_final_kernel<<<nb, 256, 0, st>>>(perm1, perm2, g, w, from_grid, tkey, ckey, N, p->perm, p->gsorted, p->wsorted, skey);
    BIN_TRY(cudaGetLastError());
    lower_bound_kernel<<<(ntiles * 8 + 1 + 255) / 256, 256, 0, st>>>(skey, N, ntiles * 8, p->class_off);
    BIN_TRY(cudaGetLastError());
    tile_off_kernel<<<(ntiles + 1 + 255) / 256, 256, 0, st>>>(p->class_off, ntiles, p->tile_off);
    BIN_TRY(cudaGetLastError());
    BIN_TRY(cudaStreamSynchronize(st));   // the scratch buffers are freed below
    cleanup();
#undef BIN_TRY
    return CS_OK;
}

// ------------------------------------------------------------------------------------------
// Sliding-window interpolation and spreading on the coil-interleaved grid [G][C].
//
// Samples are sorted by tile and, inside a tile, by acquisition order, so consecutive sorted
// samples lie a fraction of a grid unit apart along a readout and their W^3 boxes mostly
// coincide.  One warp walks a run of consecutive samples; its lanes are (coil, z-slice) pairs
// of one coil chunk (S lanes per coil), so every lane sees the same sample and the window
// updates are uniform across the warp.  A lane keeps P of the 4 z-planes of the box (4x4 values
// each) in registers.  Every axis of the window is indexed by grid index modulo 4: the value of
// grid point (z, y, x) sits in plane z & 3 (held by lane slice (z & 3) mod S), row y & 3 and
// column x & 3.  A move of the box by one along y or x therefore leaves every other register
// where it is: only the leaving row/column (residue of the old box start for a step up, of the
// old box end for a step down) is written out (spread: atomic adds) or replaced by the entering
// one (interp: loads), and it takes the entering position; a move along z does the same for a
// whole plane.  The per-sample weights are stored rotated the same way, so the accumulation
// and the dot product use fixed register indices.  Records are staged per warp in shared memory
// (64 samples at a time), and element offsets are kept as 32-bit row/column/plane offsets
// (the plan guarantees grid points x coils < 2^31).  Kernel weights phi come from a 2049-point
// table of phi on [0, 2] (linear interpolation, relative error below 3e-7, built in double on
// the host).
enum { OUT_USER = 0, OUT_RESID = 1, OUT_SORTED = 2 };
constexpr int kPhiTable = 2048;
constexpr int kStage = 64;          // records staged per warp
constexpr int kGridWarps = 4;       // warps per CTA of the gridding kernels
constexpr int kNoPlane = -(1 << 30);

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

// Per-sample record of 16 words, computed once per plan.  Words 4a .. 4a+3 hold the kernel
// weights along axis a (z, y, x), the weight of grid index j stored at word 4a + (j & 3), with
// the (-1)^(j + G/2) sign of the centred DFT folded in; word 12 packs the unwrapped box starts
// plus 2 (10 bits per axis, z lowest), word 13 is sqrt(w) and word 14 the user index.
constexpr int kRec = 16;
// word 15: the window move from the previous sorted sample.  Bits 0-1 the y step (1 up, 2 down),
// 2-3 the x step, bit 4 a jump (a step of more than one along y or x, or the first sample), bit 5
// a z change, bits 6-7 / 8-9 the residue of the leaving row / column, bits 10-19 / 20-29 the
// wrapped grid index of the entering row / column.
constexpr int kMvJump = 1 << 4, kMvZ = 1 << 5;

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
            const int j = j0 + a;
            float v = (a == 0) ? 1.f : 0.f;
            if (used) {
                v = phi_lookup(tab, g - (float)j);
                if ((j + Gs[ax] / 2) & 1) v = -v;
            }
            r[ax * kW + (j & 3)] = v;
        }
        jb[ax] = j0 + 2;
    }
    r[12] = __int_as_float(jb[0] | (jb[1] << 10) | (jb[2] << 20));
    r[13] = ws[s];
    r[14] = __int_as_float(perm[s]);
    // the window move from the previous sorted sample (word 15): a run of samples is walked in
    // sorted order, so this is the move a warp makes unless the sample starts its run
    int code = kMvJump;
    if (s > 0) {
        int jp[3] = {0, 0, 0};
        for (int ax = 3 - nd; ax < 3; ++ax) jp[ax] = (int)floorf(gs[(s - 1) * 3 + ax]) - (kW / 2 - 1);
        const int j0[3] = {jb[0] - 2, jb[1] - 2, jb[2] - 2};
        const int dz = j0[0] - jp[0], dy = j0[1] - jp[1], dx = j0[2] - jp[2];
        if ((unsigned)(dy + 1) <= 2u && (unsigned)(dx + 1) <= 2u) {
            code = (dz != 0) ? kMvZ : 0;
            if (dy != 0) {
                const int rr = (dy > 0) ? (jp[1] & 3) : ((jp[1] + 3) & 3);
                const int yn = wrapc((dy > 0) ? jp[1] + 4 : jp[1] - 1, Gy);
                code |= ((dy > 0) ? 1 : 2) | (rr << 6) | (yn << 10);
            }
            if (dx != 0) {
                const int rr = (dx > 0) ? (jp[2] & 3) : ((jp[2] + 3) & 3);
                const int xn = wrapc((dx > 0) ? jp[2] + 4 : jp[2] - 1, Gx);
                code |= (((dx > 0) ? 1 : 2) << 2) | (rr << 8) | (xn << 20);
            }
        }
    }
    r[15] = __int_as_float(code);
}

// Stage the records of samples [base, base + n) (n <= kStage) into the warp's shared buffer.
__device__ __forceinline__ void stage_records(const float* __restrict__ rec, int64_t base, int n, float* wrec, int lane,
                                              int64_t N) {
    __syncwarp();
    const float4* src = reinterpret_cast<const float4*>(rec + base * kRec);
    float4* dst = reinterpret_cast<float4*>(wrec);
    float4 t[kStage * kRec / 4 / 32];
#pragma unroll
    for (int k = 0; k < kStage * kRec / 4 / 32; ++k) {
        const int i = lane + 32 * k;
        if (i < n * (kRec / 4))
            t[k] = CS_INB(base * (kRec / 4) + i, N * (kRec / 4)) ? __ldg(src + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < kStage * kRec / 4 / 32; ++k) {
        const int i = lane + 32 * k;
        if (i < n * (kRec / 4)) dst[i] = t[k];
    }
    __syncwarp();
}

struct BoxHead {
    int jz, jy, jx;   // unwrapped box starts
    float sw;
    int perm;
};

__device__ __forceinline__ BoxHead box_head(const float* r) {
    const float4 h = *reinterpret_cast<const float4*>(r + 12);
    const int packed = __float_as_int(h.x);
    BoxHead b;
    b.jz = (packed & 1023) - 2;
    b.jy = ((packed >> 10) & 1023) - 2;
    b.jx = ((packed >> 20) & 1023) - 2;
    b.sw = h.y;
    b.perm = __float_as_int(h.z);
    return b;
}

template <int V>
using IC = std::integral_constant<int, V>;

// call f(IC<r>) for the runtime residue r in [0, 4) (uniform across the warp)
template <class F>
__device__ __forceinline__ void with_residue(int r, F&& f) {
    switch (r) {
        case 0: f(IC<0>{}); break;
        case 1: f(IC<1>{}); break;
        case 2: f(IC<2>{}); break;
        default: f(IC<3>{}); break;
    }
}

// Window state shared by both kernels: P planes of 4x4 values and the 32-bit element offsets of
// every plane (zoff), row residue (yoff) and column residue (xoff).
template <int P>
struct Win {
    float2 v[P][kW][kW];
    int zc[P];      // unwrapped z of the plane, kNoPlane when empty
    int zoff[P];
    int yoff[kW], xoff[kW];
};

// offsets of the 4 residues of a box starting at unwrapped j0: position j0 + ((r - j0) & 3)
__device__ __forceinline__ void set_offsets(int (&off)[kW], int j0, int G, int stride) {
#pragma unroll
    for (int r = 0; r < kW; ++r) off[r] = wrapc(j0 + ((r - j0) & 3), G) * stride;
}

// Minimum resident CTAs per SM requested from the register allocator for the gridding kernels, by
// planes per lane P (1: 8 coils per warp, 2: 16, 4: 32); 1 leaves the allocator unconstrained.
#ifndef CS_INTERP_MINB_P1
#define CS_INTERP_MINB_P1 4
#endif
#ifndef CS_INTERP_MINB_P2
#define CS_INTERP_MINB_P2 4
#endif
#ifndef CS_SPREAD_MINB_P1
#define CS_SPREAD_MINB_P1 4
#endif
#ifndef CS_SPREAD_MINB_P2
#define CS_SPREAD_MINB_P2 4
#endif
// decode the next sample's record head one sample ahead in the interpolation (off: its registers
// are tight)
#ifndef CS_INTERP_HEAD_PREFETCH
#define CS_INTERP_HEAD_PREFETCH 0
#endif
#ifndef CS_SPREAD_HEAD_PREFETCH
#define CS_SPREAD_HEAD_PREFETCH 1
#endif
#define CS_INTERP_MINB(P) ((P) == 1 ? CS_INTERP_MINB_P1 : (P) == 2 ? CS_INTERP_MINB_P2 : 1)
#define CS_SPREAD_MINB(P) ((P) == 1 ? CS_SPREAD_MINB_P1 : (P) == 2 ? CS_SPREAD_MINB_P2 : 1)

// S lanes per coil, P planes per lane: S * P = 4 for 3D plans, S = P = 1 for 2D plans (one plane
// z = 0 whose z weight is 1).
// grid value at element offset off of coil c (g = grid + c); guarded in checked builds
__device__ __forceinline__ float2 gridld(const float2* __restrict__ g, int c, int off, int64_t glim) {
    return CS_INB((int64_t)c + off, glim) ? __ldg(g + off) : make_float2(0.f, 0.f);
}

template <int S, int P>
__global__ void __launch_bounds__(32 * kGridWarps, CS_INTERP_MINB(P))
    interp_kernel(GridArgs A, int mode, const float2* __restrict__ ysub, float2* __restrict__ out) {
    __shared__ __align__(16) float srec[kGridWarps * kStage * kRec];
    const int lane = threadIdx.x & 31;
    const int coil_l = lane / S, slice = lane % S;
    const bool active = coil_l < A.gsize;
    const int c = A.c0 + (active ? coil_l : 0);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t s0l = warp * A.chunk;
    if (s0l >= A.N) return;                      // whole warp exits together
    // sample indices fit in 32 bits (plans hold fewer than 2^31 samples)
    const int s0 = (int)s0l, s1 = (int)min(A.N, s0l + A.chunk);
    float* wrec = srec + (threadIdx.x >> 5) * (kStage * kRec);
    const int sy = A.Gx * A.C, sz = A.Gy * A.Gx * A.C;
    const float2* g = A.grid + c;
    const int64_t glim = (int64_t)A.Gz * A.Gy * A.Gx * A.C;
    (void)glim;
    Win<P> W;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        W.zc[p] = kNoPlane;
        W.zoff[p] = 0;
#pragma unroll
        for (int b = 0; b < kW; ++b)
#pragma unroll
            for (int d = 0; d < kW; ++d) W.v[p][b][d] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int r = 0; r < kW; ++r) W.yoff[r] = W.xoff[r] = 0;
    for (int base = s0; base < s1; base += kStage) {
        const int n = min(kStage, s1 - base);
        stage_records(A.rec, base, n, wrec, lane, A.N);
#pragma unroll 1
        for (int i = 0; i < n; ++i) {
            const float* r = wrec + i * kRec;
            // the window move was decoded at plan time (record word 15); a run's first sample jumps
            const float4 hd = *reinterpret_cast<const float4*>(r + 12);
            const int mv = __float_as_int(hd.w);
            const bool jump = (mv & kMvJump) || (i == 0 && base == s0);
            if (jump) {
                const int pk = __float_as_int(hd.x);
                set_offsets(W.yoff, ((pk >> 10) & 1023) - 2, A.Gy, sy);
                set_offsets(W.xoff, ((pk >> 20) & 1023) - 2, A.Gx, A.C);
#pragma unroll
                for (int p = 0; p < P; ++p) W.zc[p] = kNoPlane;    // every plane reloads below
            } else {
                if (mv & 3) {
                    // the leaving row takes the entering row, whose grid index has the same residue
                    const int yrow = (mv >> 10) & 1023;
                    with_residue((mv >> 6) & 3, [&](auto RC) {
                        constexpr int R = decltype(RC)::value;
                        W.yoff[R] = yrow * sy;
                        if (active) {
#pragma unroll
                            for (int p = 0; p < P; ++p)
                                if (W.zc[p] != kNoPlane) {
#pragma unroll
                                    for (int d = 0; d < kW; ++d) W.v[p][R][d] = gridld(g, c, W.zoff[p] + W.yoff[R] + W.xoff[d], glim);
                                }
                        }
                    });
                }
                if (mv & 12) {
                    const int xcol = (mv >> 20) & 1023;
                    with_residue((mv >> 8) & 3, [&](auto RC) {
                        constexpr int R = decltype(RC)::value;
                        W.xoff[R] = xcol * A.C;
                        if (active) {
#pragma unroll
                            for (int p = 0; p < P; ++p)
                                if (W.zc[p] != kNoPlane) {
#pragma unroll
                                    for (int b = 0; b < kW; ++b) W.v[p][b][R] = gridld(g, c, W.zoff[p] + W.yoff[b] + W.xoff[R], glim);
                                }
                        }
                    });
                }
            }
            if (jump || (mv & kMvZ)) {
                const int jz = (__float_as_int(hd.x) & 1023) - 2;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const int q = slice + p * S;                    // z residue held by this plane
                    const int zq = jz + ((q - jz) & 3);
                    if (zq != W.zc[p]) {
                        W.zc[p] = zq;
                        W.zoff[p] = wrapc(zq, A.Gz) * sz;
                        if (active) {
#pragma unroll
                            for (int b = 0; b < kW; ++b)
#pragma unroll
                                for (int d = 0; d < kW; ++d) W.v[p][b][d] = gridld(g, c, W.zoff[p] + W.yoff[b] + W.xoff[d], glim);
                        }
                    }
                }
            }
            const float sw = hd.y;
            const int perm = __float_as_int(hd.z);
            float2 acc = make_float2(0.f, 0.f);
            const float4 wy = *reinterpret_cast<const float4*>(r + 4);
            const float4 wx = *reinterpret_cast<const float4*>(r + 8);
            const float wyv[kW] = {wy.x, wy.y, wy.z, wy.w};
            // x weights as pairs for the paired single-precision FMA (both halves of a complex value)
            const float2 wx2[kW] = {make_float2(wx.x, wx.x), make_float2(wx.y, wx.y), make_float2(wx.z, wx.z),
                                    make_float2(wx.w, wx.w)};
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float wzp = r[slice + p * S];
                float2 pa = make_float2(0.f, 0.f);
#pragma unroll
                for (int b = 0; b < kW; ++b) {
                    float2 t = make_float2(0.f, 0.f);
#pragma unroll
                    for (int d = 0; d < kW; ++d) t = __ffma2_rn(wx2[d], W.v[p][b][d], t);
                    pa = __ffma2_rn(make_float2(wyv[b], wyv[b]), t, pa);
                }
                acc = __ffma2_rn(make_float2(wzp, wzp), pa, acc);
            }
            if (S > 1) {
#pragma unroll
                for (int o = 1; o < S; o <<= 1) {
                    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
                }
            }
            if (active && slice == 0) {
                const int64_t s = (int64_t)base + i;
                acc = cscale(acc, sw);
                const int64_t lim = (int64_t)A.C * A.N;
                if (mode == OUT_USER) {
                    if (CS_INB((int64_t)c * A.N + perm, lim)) out[(int64_t)c * A.N + perm] = acc;
                } else if (mode == OUT_RESID) {
                    if (CS_INB(s * A.C + c, lim) && CS_INB((int64_t)c * A.N + perm, lim))
                        out[s * A.C + c] = csub(acc, ysub[(int64_t)c * A.N + perm]);
                } else {
                    if (CS_INB(s * A.C + c, lim)) out[s * A.C + c] = acc;
                }
            }
        }
    }
}

// Producer-computes spreading (the default): one sample stream per warp, leaving rows, columns and
// planes added to the grid with float2 atomics, so the order of the additions to a grid point
// depends on scheduling (results equal up to rounding order).  The owner-computes kernel below is
// the deterministic alternative.
template <int S, int P>
__global__ void __launch_bounds__(32 * kGridWarps, CS_SPREAD_MINB(P))
    spread_kernel(GridArgs A, const float2* __restrict__ yin, int sorted_in) {
    __shared__ __align__(16) float srec[kGridWarps * kStage * kRec];
    const int lane = threadIdx.x & 31;
    const int coil_l = lane / S, slice = lane % S;
    const bool active = coil_l < A.gsize;
    const int c = A.c0 + (active ? coil_l : 0);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t s0l = warp * A.chunk;
    if (s0l >= A.N) return;
    const int s0 = (int)s0l, s1 = (int)min(A.N, s0l + A.chunk);
    float* wrec = srec + (threadIdx.x >> 5) * (kStage * kRec);
    const int sy = A.Gx * A.C, sz = A.Gy * A.Gx * A.C;
    float2* g = A.grid + c;
    const int64_t glim = (int64_t)A.Gz * A.Gy * A.Gx * A.C;
    (void)glim;
    Win<P> W;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        W.zc[p] = kNoPlane;
        W.zoff[p] = 0;
#pragma unroll
        for (int b = 0; b < kW; ++b)
#pragma unroll
            for (int d = 0; d < kW; ++d) W.v[p][b][d] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int r = 0; r < kW; ++r) W.yoff[r] = W.xoff[r] = 0;
    auto flush_plane = [&](int p) {
        if (active && W.zc[p] != kNoPlane) {
#pragma unroll
            for (int b = 0; b < kW; ++b)
#pragma unroll
                for (int d = 0; d < kW; ++d)
                    if (CS_INB((int64_t)c + W.zoff[p] + W.yoff[b] + W.xoff[d], glim)) atomicAdd(g + (W.zoff[p] + W.yoff[b] + W.xoff[d]), W.v[p][b][d]);
        }
#pragma unroll
        for (int b = 0; b < kW; ++b)
#pragma unroll
            for (int d = 0; d < kW; ++d) W.v[p][b][d] = make_float2(0.f, 0.f);
    };
    // the sample value: sorted scratch [N][C] or user order [C][N]
    auto load_v = [&](int s, const float* r) -> float2 {
        if (!active) return make_float2(0.f, 0.f);
        const int64_t i = sorted_in ? (int64_t)s * A.C + c : (int64_t)c * A.N + __float_as_int(r[14]);
        return CS_INB(i, (int64_t)A.C * A.N) ? yin[i] : make_float2(0.f, 0.f);
    };
    for (int base = s0; base < s1; base += kStage) {
        const int n = min(kStage, s1 - base);
        stage_records(A.rec, base, n, wrec, lane, A.N);
        float2 vnext = load_v(base, wrec);
#pragma unroll 1
        for (int i = 0; i < n; ++i) {
            const float* r = wrec + i * kRec;
            float2 v = vnext;
            if (i + 1 < n) vnext = load_v(base + i + 1, r + kRec);   // one sample ahead
            // the window move was decoded at plan time (record word 15); a run's first sample jumps
            const float4 hd = *reinterpret_cast<const float4*>(r + 12);
            const int mv = __float_as_int(hd.w);
            const bool jump = (mv & kMvJump) || (i == 0 && base == s0);
            if (jump) {
                const int pk = __float_as_int(hd.x);
#pragma unroll
                for (int p = 0; p < P; ++p) flush_plane(p);
                set_offsets(W.yoff, ((pk >> 10) & 1023) - 2, A.Gy, sy);
                set_offsets(W.xoff, ((pk >> 20) & 1023) - 2, A.Gx, A.C);
            } else {
                if (mv & 3) {
                    // write out the leaving row; its registers and residue pass to the entering row
                    const int yrow = (mv >> 10) & 1023;
                    with_residue((mv >> 6) & 3, [&](auto RC) {
                        constexpr int R = decltype(RC)::value;
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            if (active && W.zc[p] != kNoPlane) {
#pragma unroll
                                for (int d = 0; d < kW; ++d)
                                    if (CS_INB((int64_t)c + W.zoff[p] + W.yoff[R] + W.xoff[d], glim)) atomicAdd(g + (W.zoff[p] + W.yoff[R] + W.xoff[d]), W.v[p][R][d]);
                            }
#pragma unroll
                            for (int d = 0; d < kW; ++d) W.v[p][R][d] = make_float2(0.f, 0.f);
                        }
                        W.yoff[R] = yrow * sy;
                    });
                }
                if (mv & 12) {
                    const int xcol = (mv >> 20) & 1023;
                    with_residue((mv >> 8) & 3, [&](auto RC) {
                        constexpr int R = decltype(RC)::value;
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            if (active && W.zc[p] != kNoPlane) {
#pragma unroll
                                for (int b = 0; b < kW; ++b)
                                    if (CS_INB((int64_t)c + W.zoff[p] + W.yoff[b] + W.xoff[R], glim)) atomicAdd(g + (W.zoff[p] + W.yoff[b] + W.xoff[R]), W.v[p][b][R]);
                            }
#pragma unroll
                            for (int b = 0; b < kW; ++b) W.v[p][b][R] = make_float2(0.f, 0.f);
                        }
                        W.xoff[R] = xcol * A.C;
                    });
                }
            }
            if (jump || (mv & kMvZ)) {
                const int jz = (__float_as_int(hd.x) & 1023) - 2;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const int q = slice + p * S;
                    const int zq = jz + ((q - jz) & 3);
                    if (zq != W.zc[p]) {
                        flush_plane(p);
                        W.zc[p] = zq;
                        W.zoff[p] = wrapc(zq, A.Gz) * sz;
                    }
                }
            }
            v = cscale(v, hd.y);
            const float4 wy = *reinterpret_cast<const float4*>(r + 4);
            const float4 wx = *reinterpret_cast<const float4*>(r + 8);
            const float wyv[kW] = {wy.x, wy.y, wy.z, wy.w};
            // x weights as pairs for the paired single-precision FMA (both halves of a complex value)
            const float2 wx2[kW] = {make_float2(wx.x, wx.x), make_float2(wx.y, wx.y), make_float2(wx.z, wx.z),
                                    make_float2(wx.w, wx.w)};
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float2 va = cscale(v, r[slice + p * S]);
#pragma unroll
                for (int b = 0; b < kW; ++b) {
                    const float2 vb = cscale(va, wyv[b]);
#pragma unroll
                    for (int d = 0; d < kW; ++d) W.v[p][b][d] = __ffma2_rn(wx2[d], vb, W.v[p][b][d]);
                }
            }
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) flush_plane(p);
}

// Two coils per lane (3D plans, chunks of 10 .. 16 coils with even coil offsets and an even
// interleave stride): lanes are (coil pair, z-slice), 4 lanes per pair with one plane each.  The
// two coils of a pair are adjacent in the coil-interleaved grid, so every window point is one
// 16-byte value: a leaving row or column is written with half as many (vector) atomic adds, an
// entering one read with half as many loads, for the same lanes and registers as two planes of
// one coil.  Value layout (x, y) = coil c, (z, w) = coil c + 1.
__device__ __forceinline__ float4 f4scale(float4 a, float s) { return make_float4(a.x * s, a.y * s, a.z * s, a.w * s); }
__device__ __forceinline__ float4 f4fma(float w, float4 v, float4 acc) {
    const float2 ww = make_float2(w, w);
    const float2 lo = __ffma2_rn(ww, make_float2(v.x, v.y), make_float2(acc.x, acc.y));
    const float2 hi = __ffma2_rn(ww, make_float2(v.z, v.w), make_float2(acc.z, acc.w));
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}
__device__ __forceinline__ float4 gridld4(const float2* __restrict__ g, int c, int off, int64_t glim) {
    return CS_INB((int64_t)c + 1 + off, glim) ? __ldg(reinterpret_cast<const float4*>(g + off))
                                               : make_float4(0.f, 0.f, 0.f, 0.f);
}

struct Win4 {
    float4 v[kW][kW];
    int zc, zoff;
    int yoff[kW], xoff[kW];
};

__global__ void __launch_bounds__(32 * kGridWarps, CS_INTERP_MINB_P2)
    interp_pair_kernel(GridArgs A, int mode, const float2* __restrict__ ysub, float2* __restrict__ out) {
    __shared__ __align__(16) float srec[kGridWarps * kStage * kRec];
    const int lane = threadIdx.x & 31;
    const int pair_l = lane >> 2, slice = lane & 3;
    const bool active = 2 * pair_l < A.gsize;
    const int c = A.c0 + 2 * (active ? pair_l : 0);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t s0l = warp * A.chunk;
    if (s0l >= A.N) return;
    const int s0 = (int)s0l, s1 = (int)min(A.N, s0l + A.chunk);
    float* wrec = srec + (threadIdx.x >> 5) * (kStage * kRec);
    const int sy = A.Gx * A.C, sz = A.Gy * A.Gx * A.C;
    const float2* g = A.grid + c;
    const int64_t glim = (int64_t)A.Gz * A.Gy * A.Gx * A.C;
    (void)glim;
    Win4 W;
    W.zc = kNoPlane;
    W.zoff = 0;
#pragma unroll
    for (int b = 0; b < kW; ++b)
#pragma unroll
        for (int d = 0; d < kW; ++d) W.v[b][d] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < kW; ++r) W.yoff[r] = W.xoff[r] = 0;
    for (int base = s0; base < s1; base += kStage) {
        const int n = min(kStage, s1 - base);
        stage_records(A.rec, base, n, wrec, lane, A.N);
#pragma unroll 1
        for (int i = 0; i < n; ++i) {
            const float* r = wrec + i * kRec;
            const float4 hd = *reinterpret_cast<const float4*>(r + 12);
            const int mv = __float_as_int(hd.w);
            const bool jump = (mv & kMvJump) || (i == 0 && base == s0);
            if (jump) {
                const int pk = __float_as_int(hd.x);
                set_offsets(W.yoff, ((pk >> 10) & 1023) - 2, A.Gy, sy);
                set_offsets(W.xoff, ((pk >> 20) & 1023) - 2, A.Gx, A.C);
                W.zc = kNoPlane;
            } else {
                if (mv & 3) {
                    const int yrow = (mv >> 10) & 1023;
                    with_residue((mv >> 6) & 3, [&](auto RC) {
                        constexpr int R = decltype(RC)::value;
                        W.yoff[R] = yrow * sy;
                        if (active && W.zc != kNoPlane) {
#pragma unroll
                            for (int d = 0; d < kW; ++d) W.v[R][d] = gridld4(g, c, W.zoff + W.yoff[R] + W.xoff[d], glim);
                        }
                    });
                }
                if (mv & 12) {
                    const int xcol = (mv >> 20) & 1023;
                    with_residue((mv >> 8) & 3, [&](auto RC) {
                        constexpr int R = decltype(RC)::value;
                        W.xoff[R] = xcol * A.C;
                        if (active && W.zc != kNoPlane) {
#pragma unroll
                            for (int b = 0; b < kW; ++b) W.v[b][R] = gridld4(g, c, W.zoff + W.yoff[b] + W.xoff[R], glim);
                        }
                    });
                }
            }
            if (jump || (mv & kMvZ)) {
                const int jz = (__float_as_int(hd.x) & 1023) - 2;
                const int zq = jz + ((slice - jz) & 3);
                if (zq != W.zc) {
                    W.zc = zq;
                    W.zoff = wrapc(zq, A.Gz) * sz;
                    if (active) {
#pragma unroll
                        for (int b = 0; b < kW; ++b)
#pragma unroll
                            for (int d = 0; d < kW; ++d) W.v[b][d] = gridld4(g, c, W.zoff + W.yoff[b] + W.xoff[d], glim);
                    }
                }
            }
            const float sw = hd.y;
            const int perm = __float_as_int(hd.z);
            const float4 wy = *reinterpret_cast<const float4*>(r + 4);
            const float4 wx = *reinterpret_cast<const float4*>(r + 8);
            const float wyv[kW] = {wy.x, wy.y, wy.z, wy.w};
            const float wxv[kW] = {wx.x, wx.y, wx.z, wx.w};
            float4 pa = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int b = 0; b < kW; ++b) {
                float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int d = 0; d < kW; ++d) t = f4fma(wxv[d], W.v[b][d], t);
                pa = f4fma(wyv[b], t, pa);
            }
            float4 acc = f4scale(pa, r[slice]);
#pragma unroll
            for (int o = 1; o < 4; o <<= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
                acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
                acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
            }
            if (active && slice == 0) {
                const int64_t s = (int64_t)base + i;
                acc = f4scale(acc, sw);
                const int64_t lim = (int64_t)A.C * A.N;
                if (mode == OUT_USER) {
                    if (CS_INB((int64_t)(c + 1) * A.N + perm, lim)) {
                        out[(int64_t)c * A.N + perm] = make_float2(acc.x, acc.y);
                        out[(int64_t)(c + 1) * A.N + perm] = make_float2(acc.z, acc.w);
                    }
                } else if (mode == OUT_RESID) {
                    if (CS_INB(s * A.C + c + 1, lim) && CS_INB((int64_t)(c + 1) * A.N + perm, lim)) {
                        const float2 y0 = ysub[(int64_t)c * A.N + perm], y1 = ysub[(int64_t)(c + 1) * A.N + perm];
                        *reinterpret_cast<float4*>(out + s * A.C + c) = make_float4(acc.x - y0.x, acc.y - y0.y, acc.z - y1.x, acc.w - y1.y);
                    }
                } else {
                    if (CS_INB(s * A.C + c + 1, lim)) *reinterpret_cast<float4*>(out + s * A.C + c) = acc;
                }
            }
        }
    }
}

__global__ void __launch_bounds__(32 * kGridWarps, CS_SPREAD_MINB_P2)
    spread_pair_kernel(GridArgs A, const float2* __restrict__ yin, int sorted_in) {
    __shared__ __align__(16) float srec[kGridWarps * kStage * kRec];
    const int lane = threadIdx.x & 31;
    const int pair_l = lane >> 2, slice = lane & 3;
    const bool active = 2 * pair_l < A.gsize;
    const int c = A.c0 + 2 * (active ? pair_l : 0);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t s0l = warp * A.chunk;
    if (s0l >= A.N) return;
    const int s0 = (int)s0l, s1 = (int)min(A.N, s0l + A.chunk);
    float* wrec = srec + (threadIdx.x >> 5) * (kStage * kRec);
    const int sy = A.Gx * A.C, sz = A.Gy * A.Gx * A.C;
    float2* g = A.grid + c;
    const int64_t glim = (int64_t)A.Gz * A.Gy * A.Gx * A.C;
    (void)glim;
    Win4 W;
    W.zc = kNoPlane;
    W.zoff = 0;
#pragma unroll
    for (int b = 0; b < kW; ++b)
#pragma unroll
        for (int d = 0; d < kW; ++d) W.v[b][d] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < kW; ++r) W.yoff[r] = W.xoff[r] = 0;
    auto add4 = [&](int off, float4 v) {
        if (CS_INB((int64_t)c + 1 + off, glim)) atomicAdd(reinterpret_cast<float4*>(g + off), v);
    };
    auto flush_plane = [&]() {
        if (active && W.zc != kNoPlane) {
#pragma unroll
            for (int b = 0; b < kW; ++b)
#pragma unroll
                for (int d = 0; d < kW; ++d) add4(W.zoff + W.yoff[b] + W.xoff[d], W.v[b][d]);
        }
#pragma unroll
        for (int b = 0; b < kW; ++b)
#pragma unroll
            for (int d = 0; d < kW; ++d) W.v[b][d] = make_float4(0.f, 0.f, 0.f, 0.f);
    };
    // the pair's two sample values: sorted scratch [N][C] (one 16-byte load) or user order [C][N]
    auto load_v = [&](int s, const float* r) -> float4 {
        if (!active) return make_float4(0.f, 0.f, 0.f, 0.f);
        if (sorted_in) {
            const int64_t i = (int64_t)s * A.C + c;
            return CS_INB(i + 1, (int64_t)A.C * A.N) ? *reinterpret_cast<const float4*>(yin + i)
                                                     : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const int64_t i = (int64_t)c * A.N + __float_as_int(r[14]);
        if (!CS_INB(i + A.N, (int64_t)A.C * A.N)) return make_float4(0.f, 0.f, 0.f, 0.f);
        const float2 a = yin[i], b = yin[i + A.N];
        return make_float4(a.x, a.y, b.x, b.y);
    };
    for (int base = s0; base < s1; base += kStage) {
        const int n = min(kStage, s1 - base);
        stage_records(A.rec, base, n, wrec, lane, A.N);
        float4 vnext = load_v(base, wrec);
#pragma unroll 1
        for (int i = 0; i < n; ++i) {
            const float* r = wrec + i * kRec;
            float4 v = vnext;
            if (i + 1 < n) vnext = load_v(base + i + 1, r + kRec);
            const float4 hd = *reinterpret_cast<const float4*>(r + 12);
            const int mv = __float_as_int(hd.w);
            const bool jump = (mv & kMvJump) || (i == 0 && base == s0);
            if (jump) {
                const int pk = __float_as_int(hd.x);
                flush_plane();
                set_offsets(W.yoff, ((pk >> 10) & 1023) - 2, A.Gy, sy);
                set_offsets(W.xoff, ((pk >> 20) & 1023) - 2, A.Gx, A.C);
            } else {
                if (mv & 3) {
                    const int yrow = (mv >> 10) & 1023;
                    with_residue((mv >> 6) & 3, [&](auto RC) {
                        constexpr int R = decltype(RC)::value;
                        if (active && W.zc != kNoPlane) {
#pragma unroll
                            for (int d = 0; d < kW; ++d) add4(W.zoff + W.yoff[R] + W.xoff[d], W.v[R][d]);
                        }
#pragma unroll
                        for (int d = 0; d < kW; ++d) W.v[R][d] = make_float4(0.f, 0.f, 0.f, 0.f);
                        W.yoff[R] = yrow * sy;
                    });
                }
                if (mv & 12) {
                    const int xcol = (mv >> 20) & 1023;
                    with_residue((mv >> 8) & 3, [&](auto RC) {
                        constexpr int R = decltype(RC)::value;
                        if (active && W.zc != kNoPlane) {
#pragma unroll
                            for (int b = 0; b < kW; ++b) add4(W.zoff + W.yoff[b] + W.xoff[R], W.v[b][R]);
                        }
#pragma unroll
                        for (int b = 0; b < kW; ++b) W.v[b][R] = make_float4(0.f, 0.f, 0.f, 0.f);
                        W.xoff[R] = xcol * A.C;
                    });
                }
            }
            if (jump || (mv & kMvZ)) {
                const int jz = (__float_as_int(hd.x) & 1023) - 2;
                const int zq = jz + ((slice - jz) & 3);
                if (zq != W.zc) {
                    flush_plane();
                    W.zc = zq;
                    W.zoff = wrapc(zq, A.Gz) * sz;
                }
            }
            const float4 wy = *reinterpret_cast<const float4*>(r + 4);
            const float4 wx = *reinterpret_cast<const float4*>(r + 8);
            const float wyv[kW] = {wy.x, wy.y, wy.z, wy.w};
            const float wxv[kW] = {wx.x, wx.y, wx.z, wx.w};
            const float4 va = f4scale(f4scale(v, hd.y), r[slice]);
#pragma unroll
            for (int b = 0; b < kW; ++b) {
                const float4 vb = f4scale(va, wyv[b]);
#pragma unroll
                for (int d = 0; d < kW; ++d) W.v[b][d] = f4fma(wxv[d], vb, W.v[b][d]);
            }
        }
    }
    flush_plane();
}

// Owner-computes spreading.  One warp runs one work item: a tile of the grid (its region) and a
// list of sorted-sample ranges (the tile's own samples and those of its lower neighbours whose box
// reaches it, or a chunk of that list).  The warp keeps the same residue-indexed sliding window as
// the interpolation; when a row, column or plane leaves the window, the points of it that lie in
// the region are added to the target by a plain read-modify-write - the region belongs to this
// warp alone, so no other thread touches those points while it runs, and every point receives its
// contributions in the fixed order of the item's sample list.  Points outside the region are
// dropped (their owner adds them).  The target is the grid itself (item slot -1) or the item's
// private partial slot, laid out [z][y][x][coil] over the widest tile; owner_reduce_kernel later
// adds a tile's slots to the grid in slot order.  Lanes are (coil, z-slice) as in the
// interpolation; a grid plane always belongs to the same lane (see launch_spread for the z sizes
// that need the 2-lane mapping), and rows and columns stay within a lane.
struct OwnerArgs {
    float2* grid;          // [G][C] (coil-interleaved)
    int C;                 // interleave stride = coils of the operator call
    int c0, gsize;         // coil chunk handled by this launch
    int Gz, Gy, Gx;
    int Tz, Ty, Tx, ntz, nty, ntx;
    const float* rec;      // [N][16] per-sample records (sorted order)
    int64_t Nsamp;         // samples per coil (user-order input y [C][N])
    const GItem* items;
    int nitems;
    const GRange* ranges;
    float2* part;          // partial slots
    int nslots;
    int wz, wy, wx;        // slot geometry (widest tile per axis)
};

__device__ __forceinline__ void tile_region(const OwnerArgs& A, int tile, int* o, int* w) {
    const int tx = tile % A.ntx, ty = (tile / A.ntx) % A.nty, tz = tile / (A.ntx * A.nty);
    o[0] = tz * A.Tz;
    o[1] = ty * A.Ty;
    o[2] = tx * A.Tx;
    w[0] = (tz == A.ntz - 1) ? A.Gz - o[0] : A.Tz;
    w[1] = (ty == A.nty - 1) ? A.Gy - o[1] : A.Ty;
    w[2] = (tx == A.ntx - 1) ? A.Gx - o[2] : A.Tx;
}

// offsets (from the target's base b) and region membership of the 4 residues of a box starting at
// unwrapped j0 along one axis: residue r holds position j0 + ((r - j0) & 3)
__device__ __forceinline__ void set_offsets_owned(int (&off)[kW], int& in, int j0, int G, int stride, int o, int w,
                                                  int b) {
    in = 0;
#pragma unroll
    for (int r = 0; r < kW; ++r) {
        const int j = wrapc(j0 + ((r - j0) & 3), G);
        off[r] = (j - b) * stride;
        in |= ((unsigned)(j - o) < (unsigned)w) << r;
    }
}

template <int S, int P>
__global__ void __launch_bounds__(32 * kGridWarps, CS_SPREAD_MINB(P))
    spread_owner_kernel(OwnerArgs A, const float2* __restrict__ yin, int sorted_in) {
    __shared__ __align__(16) float srec[kGridWarps * kStage * kRec];
    const int lane = threadIdx.x & 31;
    const int coil_l = lane / S, slice = lane % S;
    const bool active = coil_l < A.gsize;
    const int c = A.c0 + (active ? coil_l : 0);
    const int item_i = blockIdx.x * kGridWarps + (threadIdx.x >> 5);
    if (item_i >= A.nitems) return;                // whole warp exits together
    const GItem it = A.items[item_i];
    int o[3], w[3];
    tile_region(A, it.tile, o, w);
    // target base and strides: the grid (absolute offsets) or the item's slot (offsets from o)
    float2* tgt;
    int b[3], sz, sy, sx;
    int64_t tbase, tlim;   // element offset of tgt in its buffer and the buffer length (checked builds)
    if (it.slot < 0) {
        tbase = c;
        tlim = (int64_t)A.Gz * A.Gy * A.Gx * A.C;
        tgt = A.grid + c;
        b[0] = b[1] = b[2] = 0;
        sx = A.C;
        sy = A.Gx * A.C;
        sz = A.Gy * A.Gx * A.C;
    } else {
        tbase = (int64_t)it.slot * A.wz * A.wy * A.wx * A.gsize + (active ? coil_l : 0);
        tlim = (int64_t)A.nslots * A.wz * A.wy * A.wx * A.gsize;
        tgt = A.part + (int64_t)it.slot * A.wz * A.wy * A.wx * A.gsize + (active ? coil_l : 0);
        b[0] = o[0];
        b[1] = o[1];
        b[2] = o[2];
        sx = A.gsize;
        sy = A.wx * A.gsize;
        sz = A.wy * A.wx * A.gsize;
    }
    float* wrec = srec + (threadIdx.x >> 5) * (kStage * kRec);
    Win<P> W;
    int zin = 0, yin_m = 0, xin_m = 0;   // region membership: planes (bit p), rows and columns (bit r)
#pragma unroll
    for (int p = 0; p < P; ++p) {
        W.zc[p] = kNoPlane;
        W.zoff[p] = 0;
#pragma unroll
        for (int bb = 0; bb < kW; ++bb)
#pragma unroll
            for (int d = 0; d < kW; ++d) W.v[p][bb][d] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int r = 0; r < kW; ++r) W.yoff[r] = W.xoff[r] = 0;
    int cy = kNoPlane, cx = kNoPlane;
    // a flush adds 4 points at a time: their 4 loads are issued together, then the 4 stores
    auto flush_plane = [&](int p) {
        if (active && ((zin >> p) & 1) && W.zc[p] != kNoPlane) {
#pragma unroll
            for (int bb = 0; bb < kW; ++bb) {
                if (!((yin_m >> bb) & 1)) continue;
                float2 old[kW];
#pragma unroll
                for (int d = 0; d < kW; ++d)
                    if (((xin_m >> d) & 1) && CS_INB(tbase + W.zoff[p] + W.yoff[bb] + W.xoff[d], tlim))
                        old[d] = tgt[W.zoff[p] + W.yoff[bb] + W.xoff[d]];
#pragma unroll
                for (int d = 0; d < kW; ++d)
                    if (((xin_m >> d) & 1) && CS_INB(tbase + W.zoff[p] + W.yoff[bb] + W.xoff[d], tlim))
                        tgt[W.zoff[p] + W.yoff[bb] + W.xoff[d]] =
                            make_float2(old[d].x + W.v[p][bb][d].x, old[d].y + W.v[p][bb][d].y);
            }
        }
#pragma unroll
        for (int bb = 0; bb < kW; ++bb)
#pragma unroll
            for (int d = 0; d < kW; ++d) W.v[p][bb][d] = make_float2(0.f, 0.f);
    };
    for (int ri = it.r0; ri < it.r1; ++ri) {
        const GRange rg = A.ranges[ri];
        const int rend = rg.start + rg.count;
        for (int base = rg.start; base < rend; base += kStage) {
            const int n = min(kStage, rend - base);
            stage_records(A.rec, base, n, wrec, lane, A.Nsamp);
#pragma unroll 1
            for (int i = 0; i < n; ++i) {
                const float* r = wrec + i * kRec;
                const BoxHead B = box_head(r);
                float2 v = make_float2(0.f, 0.f);
                if (active) {
                    const int64_t vi = sorted_in ? (int64_t)(base + i) * A.C + c : (int64_t)c * A.Nsamp + B.perm;
                    if (CS_INB(vi, (int64_t)A.C * A.Nsamp)) v = yin[vi];
                }
                const int dy = B.jy - cy, dx = B.jx - cx;
                if ((unsigned)(dy + 1) > 2u || (unsigned)(dx + 1) > 2u) {   // not a step of -1, 0 or +1
#pragma unroll
                    for (int p = 0; p < P; ++p) flush_plane(p);
                    set_offsets_owned(W.yoff, yin_m, B.jy, A.Gy, sy, o[1], w[1], b[1]);
                    set_offsets_owned(W.xoff, xin_m, B.jx, A.Gx, sx, o[2], w[2], b[2]);
                } else {
                    if (dy != 0) {
                        // add the leaving row (old start for a step up, old end for a step down) to
                        // the target; its registers and residue pass to the entering row
                        const int rr = (dy > 0) ? (cy & 3) : ((cy + 3) & 3);
                        const int ynew = (dy > 0) ? cy + 4 : cy - 1;
                        with_residue(rr, [&](auto RC) {
                            constexpr int R = decltype(RC)::value;
                            const bool rowin = (yin_m >> R) & 1;
#pragma unroll
                            for (int p = 0; p < P; ++p) {
                                if (active && rowin && ((zin >> p) & 1) && W.zc[p] != kNoPlane) {
                                    float2 old[kW];
#pragma unroll
                                    for (int d = 0; d < kW; ++d)
                                        if (((xin_m >> d) & 1) && CS_INB(tbase + W.zoff[p] + W.yoff[R] + W.xoff[d], tlim))
                                            old[d] = tgt[W.zoff[p] + W.yoff[R] + W.xoff[d]];
#pragma unroll
                                    for (int d = 0; d < kW; ++d)
                                        if (((xin_m >> d) & 1) && CS_INB(tbase + W.zoff[p] + W.yoff[R] + W.xoff[d], tlim))
                                            tgt[W.zoff[p] + W.yoff[R] + W.xoff[d]] =
                                                make_float2(old[d].x + W.v[p][R][d].x, old[d].y + W.v[p][R][d].y);
                                }
#pragma unroll
                                for (int d = 0; d < kW; ++d) W.v[p][R][d] = make_float2(0.f, 0.f);
                            }
                            const int jw = wrapc(ynew, A.Gy);
                            W.yoff[R] = (jw - b[1]) * sy;
                            yin_m = (yin_m & ~(1 << R)) | (((unsigned)(jw - o[1]) < (unsigned)w[1]) << R);
                        });
                    }
                    if (dx != 0) {
                        const int rr = (dx > 0) ? (cx & 3) : ((cx + 3) & 3);
                        const int xnew = (dx > 0) ? cx + 4 : cx - 1;
                        with_residue(rr, [&](auto RC) {
                            constexpr int R = decltype(RC)::value;
                            const bool colin = (xin_m >> R) & 1;
#pragma unroll
                            for (int p = 0; p < P; ++p) {
                                if (active && colin && ((zin >> p) & 1) && W.zc[p] != kNoPlane) {
                                    float2 old[kW];
#pragma unroll
                                    for (int bb = 0; bb < kW; ++bb)
                                        if (((yin_m >> bb) & 1) && CS_INB(tbase + W.zoff[p] + W.yoff[bb] + W.xoff[R], tlim))
                                            old[bb] = tgt[W.zoff[p] + W.yoff[bb] + W.xoff[R]];
#pragma unroll
                                    for (int bb = 0; bb < kW; ++bb)
                                        if (((yin_m >> bb) & 1) && CS_INB(tbase + W.zoff[p] + W.yoff[bb] + W.xoff[R], tlim))
                                            tgt[W.zoff[p] + W.yoff[bb] + W.xoff[R]] =
                                                make_float2(old[bb].x + W.v[p][bb][R].x, old[bb].y + W.v[p][bb][R].y);
                                }
#pragma unroll
                                for (int bb = 0; bb < kW; ++bb) W.v[p][bb][R] = make_float2(0.f, 0.f);
                            }
                            const int jw = wrapc(xnew, A.Gx);
                            W.xoff[R] = (jw - b[2]) * sx;
                            xin_m = (xin_m & ~(1 << R)) | (((unsigned)(jw - o[2]) < (unsigned)w[2]) << R);
                        });
                    }
                }
                cy = B.jy;
                cx = B.jx;
                v = cscale(v, B.sw);
                const float4 wy = *reinterpret_cast<const float4*>(r + 4);
                const float4 wx = *reinterpret_cast<const float4*>(r + 8);
                const float wyv[kW] = {wy.x, wy.y, wy.z, wy.w};
                const float2 wx2[kW] = {make_float2(wx.x, wx.x), make_float2(wx.y, wx.y), make_float2(wx.z, wx.z),
                                        make_float2(wx.w, wx.w)};
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const int q = slice + p * S;
                    const int zq = B.jz + ((q - B.jz) & 3);
                    if (zq != W.zc[p]) {
                        flush_plane(p);
                        W.zc[p] = zq;
                        const int jw = wrapc(zq, A.Gz);
                        W.zoff[p] = (jw - b[0]) * sz;
                        zin = (zin & ~(1 << p)) | (((unsigned)(jw - o[0]) < (unsigned)w[0]) << p);
                    }
                    const float2 va = cscale(v, r[q]);
#pragma unroll
                    for (int bb = 0; bb < kW; ++bb) {
                        const float2 vb = cscale(va, wyv[bb]);
#pragma unroll
                        for (int d = 0; d < kW; ++d) W.v[p][bb][d] = __ffma2_rn(wx2[d], vb, W.v[p][bb][d]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) flush_plane(p);
}

// grid (tile region, this launch's coils) += the tile's partial slots in slot order
__global__ void owner_reduce_kernel(OwnerArgs A, const GRed* __restrict__ reds) {
    const GRed rd = reds[blockIdx.x];
    int o[3], w[3];
    tile_region(A, rd.tile, o, w);
    const int g = A.gsize;
    const int64_t n = (int64_t)w[0] * w[1] * w[2] * g;
    const int64_t slot = (int64_t)A.wz * A.wy * A.wx * g;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
        const int cc = (int)(e % g);
        const int64_t v = e / g;
        const int lx = (int)(v % w[2]), ly = (int)((v / w[2]) % w[1]), lz = (int)(v / ((int64_t)w[2] * w[1]));
        const int64_t di = (((int64_t)(o[0] + lz) * A.Gy + (o[1] + ly)) * A.Gx + (o[2] + lx)) * A.C + A.c0 + cc;
        const int64_t loc = (((int64_t)lz * A.wy + ly) * A.wx + lx) * g + cc;
        if (!CS_INB(di, (int64_t)A.Gz * A.Gy * A.Gx * A.C)) continue;
        float2 acc = A.grid[di];
        for (int k = 0; k < rd.ns; ++k) {
            const int64_t pi = (rd.s0 + k) * slot + loc;
            if (!CS_INB(pi, (int64_t)A.nslots * slot)) continue;
            const float2 q = A.part[pi];
            acc.x += q.x;
            acc.y += q.y;
        }
        A.grid[di] = acc;
    }
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

// Coil chunks of a gridding launch: a chunk of g <= 8 coils uses 4 lanes per coil holding one
// plane each (P = 1), g <= 16 two lanes with two planes, g <= 32 one lane with all 4 planes.
template <class F>
static cs_status for_coil_chunks(const cs_plan* p, int ncoils, int cmax, F&& f) {
    const int nch = (ncoils + cmax - 1) / cmax;
    const int cbal = (ncoils + nch - 1) / nch;                      // balanced chunk size
    for (int c0 = 0; c0 < ncoils; c0 += cbal) {
        const int g = std::min(cbal, ncoils - c0);
        int P = 1;
        if (p->ndim == 3) P = (g <= 8) ? 1 : (g <= 16 ? 2 : 4);
        CS_PROPAGATE(f(c0, g, P));
    }
    return CS_OK;
}

// The two-coils-per-lane kernels need 16-byte alignment of every coil pair: an even interleave
// stride, an even first coil and an even chunk, a 16-byte aligned grid (and sorted k-space
// array, when one is read or written as pairs).
static bool pair_ok(const GridArgs& A, const float2* sorted) {
    return A.C % 2 == 0 && A.c0 % 2 == 0 && A.gsize % 2 == 0 && (reinterpret_cast<uintptr_t>(A.grid) & 15) == 0 &&
           (sorted == nullptr || (reinterpret_cast<uintptr_t>(sorted) & 15) == 0);
}

// Interpolation: one sample stream (interp_chunk consecutive sorted samples) per warp.
static cs_status launch_interp(const cs_plan* p, int ncoils, int mode, const float2* ysub, float2* out,
                               cudaStream_t st) {
    GridArgs A = make_grid_args(p, ncoils);
    A.chunk = p->interp_chunk;
    const int64_t warps = (p->N + A.chunk - 1) / A.chunk;
    const unsigned nb = (unsigned)((warps + kGridWarps - 1) / kGridWarps);
    if (nb == 0) return CS_OK;
    return for_coil_chunks(p, ncoils, p->interp_coils, [&](int c0, int g, int P) -> cs_status {
        A.c0 = c0;
        A.gsize = g;
        prof_begin(ST_INTERP, st);
        if (p->ndim == 2) interp_kernel<1, 1><<<nb, 32 * kGridWarps, 0, st>>>(A, mode, ysub, out);
        else if (P == 2 && pair_ok(A, out)) interp_pair_kernel<<<nb, 32 * kGridWarps, 0, st>>>(A, mode, ysub, out);
        else if (P == 1) interp_kernel<4, 1><<<nb, 32 * kGridWarps, 0, st>>>(A, mode, ysub, out);
        else if (P == 2) interp_kernel<2, 2><<<nb, 32 * kGridWarps, 0, st>>>(A, mode, ysub, out);
        else interp_kernel<1, 4><<<nb, 32 * kGridWarps, 0, st>>>(A, mode, ysub, out);
        CS_LAUNCH_CHECK();
        prof_end(ST_INTERP, st);
        return CS_OK;
    });
}

// Producer-computes spreading (default): one sample stream (spread_chunk sorted samples) per warp.
static cs_status launch_spread_producer(const cs_plan* p, int ncoils, const float2* yin, int sorted_in,
                                        cudaStream_t st) {
    GridArgs A = make_grid_args(p, ncoils);
    A.chunk = p->spread_chunk;
    const int64_t warps = (p->N + A.chunk - 1) / A.chunk;
    const unsigned nb = (unsigned)((warps + kGridWarps - 1) / kGridWarps);
    if (nb == 0) return CS_OK;
    return for_coil_chunks(p, ncoils, p->spread_coils, [&](int c0, int g, int P) -> cs_status {
        A.c0 = c0;
        A.gsize = g;
        prof_begin(ST_SPREAD, st);
        if (p->ndim == 2) spread_kernel<1, 1><<<nb, 32 * kGridWarps, 0, st>>>(A, yin, sorted_in);
        else if (P == 2 && pair_ok(A, sorted_in ? yin : nullptr)) spread_pair_kernel<<<nb, 32 * kGridWarps, 0, st>>>(A, yin, sorted_in);
        else if (P == 1) spread_kernel<4, 1><<<nb, 32 * kGridWarps, 0, st>>>(A, yin, sorted_in);
        else spread_kernel<2, 2><<<nb, 32 * kGridWarps, 0, st>>>(A, yin, sorted_in);
        CS_LAUNCH_CHECK();
        prof_end(ST_SPREAD, st);
        return CS_OK;
    });
}

// Owner-computes spreading (deterministic mode): per coil chunk one launch over the work items
// (one warp each), then the fixed-order addition of the partial slots.  The grid is cleared first
// (items add into it).
static cs_status launch_spread(const cs_plan* p, int ncoils, const float2* yin, int sorted_in, cudaStream_t st) {
    if (!p->deterministic) return launch_spread_producer(p, ncoils, yin, sorted_in, st);
    OwnerArgs A;
    A.grid = grid_buffer(p);
    A.C = ncoils;
    A.Gz = p->grid[0];
    A.Gy = p->grid[1];
    A.Gx = p->grid[2];
    A.Tz = p->tile[0];
    A.Ty = p->tile[1];
    A.Tx = p->tile[2];
    A.ntz = p->ntiles[0];
    A.nty = p->ntiles[1];
    A.ntx = p->ntiles[2];
    A.rec = p->rec;
    A.Nsamp = p->N;
    A.items = p->gitems;
    A.nitems = p->n_gitems;
    A.ranges = p->granges;
    A.part = p->gpart;
    A.nslots = p->n_slots;
    A.wz = p->wmax[0];
    A.wy = p->wmax[1];
    A.wx = p->wmax[2];
    if (p->n_gitems == 0) return CS_OK;
    const unsigned nb = (unsigned)((p->n_gitems + kGridWarps - 1) / kGridWarps);
    return for_coil_chunks(p, ncoils, p->spread_coils, [&](int c0, int g, int P) -> cs_status {
        A.c0 = c0;
        A.gsize = g;
        prof_begin(ST_SPREAD, st);
        if (p->n_slots > 0)
            CS_TRY_CUDA(cudaMemsetAsync(p->gpart, 0,
                                        sizeof(float2) * (size_t)p->n_slots * p->wmax[0] * p->wmax[1] * p->wmax[2] * g, st));
        // a grid plane must stay with one lane: with 4 lanes per coil (one z residue each) that needs a
        // z size that is a multiple of 4; for z sizes of 2 mod 4 the 2-lane mapping (residues r and
        // r + 2 in one lane, which a wrap maps onto each other) is used
        if (p->ndim == 2) spread_owner_kernel<1, 1><<<nb, 32 * kGridWarps, 0, st>>>(A, yin, sorted_in);
        else if (P == 1 && p->grid[0] % 4 == 0) spread_owner_kernel<4, 1><<<nb, 32 * kGridWarps, 0, st>>>(A, yin, sorted_in);
        else spread_owner_kernel<2, 2><<<nb, 32 * kGridWarps, 0, st>>>(A, yin, sorted_in);
        CS_LAUNCH_CHECK();
        if (p->n_greds > 0) {
            owner_reduce_kernel<<<p->n_greds, 256, 0, st>>>(A, p->greds);
            CS_LAUNCH_CHECK();
        }
        prof_end(ST_SPREAD, st);
        return CS_OK;
    });
}

void nufft_owner_free(cs_plan* p) {
    cudaFree(p->gitems);
    cudaFree(p->granges);
    cudaFree(p->greds);
    cudaFree(p->gpart);
    p->gitems = nullptr;
    p->granges = nullptr;
    p->greds = nullptr;
    p->gpart = nullptr;
    p->n_gitems = p->n_greds = p->n_slots = 0;
}

// Work items of the owner-computes spreading from the (tile, halo class) offsets: tile t takes its
// own samples and, for every non-empty set e of axes (z = 4, y = 2, x = 1) that have more than one
// tile, the samples of tile t - e whose class contains e.  The concatenated list is cut into items
// of at most owner_item visits; the first writes the grid, the others own partial slots.  Items
// are ordered longest first.  Synchronous (copies the offsets to the host).
cs_status nufft_owner_build(cs_plan* p) {
    nufft_owner_free(p);
    const int nt[3] = {p->ntiles[0], p->ntiles[1], p->ntiles[2]};
    const int64_t ntot = p->ntiles_total;
    std::vector<int32_t> coff((size_t)ntot * 8 + 1);
    CS_TRY_CUDA(cudaMemcpy(coff.data(), p->class_off, sizeof(int32_t) * coff.size(), cudaMemcpyDeviceToHost));
    const int nd = p->ndim;
    std::vector<GItem> items;
    std::vector<GRange> ranges;
    std::vector<GRed> reds;
    std::vector<GRange> list;
    int slots = 0;
    const int64_t Q = std::max(1, p->owner_item);
    for (int64_t t = 0; t < ntot; ++t) {
        const int tz = (int)(t / ((int64_t)nt[1] * nt[2])), ty = (int)((t / nt[2]) % nt[1]), tx = (int)(t % nt[2]);
        list.clear();
        int64_t visits = 0;
        for (int e = 0; e < 8; ++e) {
            // bits of e on the axes this plan uses; a neighbour exists only with more than one tile
            const int ez = (e >> 2) & 1, ey = (e >> 1) & 1, ex = e & 1;
            if ((ez && (nd < 3 || nt[0] == 1)) || (ey && nt[1] == 1) || (ex && nt[2] == 1)) continue;
            const int sz_ = (tz - ez + nt[0]) % nt[0], sy_ = (ty - ey + nt[1]) % nt[1], sx_ = (tx - ex + nt[2]) % nt[2];
            const int64_t src = ((int64_t)sz_ * nt[1] + sy_) * nt[2] + sx_;
            for (int cl = 0; cl < 8; ++cl) {
                if ((cl & e) != e) continue;
                const int32_t a = coff[src * 8 + cl], b = coff[src * 8 + cl + 1];
                if (b > a) {
                    list.push_back(GRange{a, b - a});
                    visits += b - a;
                }
            }
        }
        if (visits == 0) continue;
        const int nchunks = (int)((visits + Q - 1) / Q);
        size_t li = 0;
        int64_t inpos = 0;   // position inside list[li]
        for (int k = 0; k < nchunks; ++k) {
            GItem it;
            it.tile = (int)t;
            it.slot = (k == 0) ? -1 : slots + k - 1;
            it.r0 = (int)ranges.size();
            int64_t need = std::min<int64_t>(Q, visits - (int64_t)k * Q);
            while (need > 0) {
                const int64_t take = std::min<int64_t>(need, list[li].count - inpos);
                ranges.push_back(GRange{(int)(list[li].start + inpos), (int)take});
                need -= take;
                inpos += take;
                if (inpos == list[li].count) {
                    ++li;
                    inpos = 0;
                }
            }
            it.r1 = (int)ranges.size();
            items.push_back(it);
        }
        if (nchunks > 1) {
            reds.push_back(GRed{(int)t, slots, nchunks - 1});
            slots += nchunks - 1;
        }
    }
    // longest first (by visits), ties in tile order, so that the long items start first
    std::vector<int64_t> len(items.size());
    for (size_t i = 0; i < items.size(); ++i) {
        int64_t v = 0;
        for (int r = items[i].r0; r < items[i].r1; ++r) v += ranges[r].count;
        len[i] = v;
    }
    std::vector<size_t> ord(items.size());
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return len[a] > len[b]; });
    std::vector<GItem> sorted(items.size());
    for (size_t i = 0; i < ord.size(); ++i) sorted[i] = items[ord[i]];
    auto upload = [&](auto& vec, auto** dst) -> cs_status {
        if (vec.empty()) return CS_OK;
        CS_TRY_CUDA(cudaMalloc((void**)dst, sizeof(vec[0]) * vec.size()));
        CS_TRY_CUDA(cudaMemcpy(*dst, vec.data(), sizeof(vec[0]) * vec.size(), cudaMemcpyHostToDevice));
        return CS_OK;
    };
    CS_PROPAGATE(upload(sorted, &p->gitems));
    CS_PROPAGATE(upload(ranges, &p->granges));
    CS_PROPAGATE(upload(reds, &p->greds));
    p->n_gitems = (int)sorted.size();
    p->n_greds = (int)reds.size();
    p->n_slots = slots;
    if (slots > 0) {
        const size_t n = (size_t)slots * p->wmax[0] * p->wmax[1] * p->wmax[2] * 16;   // <= 16 coils per launch
        CS_TRY_CUDA(cudaMalloc(&p->gpart, sizeof(float2) * n));
    }
    return CS_OK;
}

// Re-binning for new tile sizes: the plan's sorted grid coordinates and sqrt(dcf) go back to user
// order and are binned again exactly as at plan creation (same keys, same stable order), the
// records are rewritten in the same buffer, and the deterministic-spreading work items are rebuilt
// if the plan has them.  Synchronous.  On an error after the first step the plan is unusable.
cs_status nufft_retile(cs_plan* p, const int* tile3, cudaStream_t st) {
    const int keep_t[3] = {p->tile[0], p->tile[1], p->tile[2]};
    CS_PROPAGATE(nufft_set_tiles(p, tile3));
    const int64_t N = p->N;
    float *gu = nullptr, *wu = nullptr;
    int32_t *toff = nullptr, *coff = nullptr;
    cudaError_t e = cudaMalloc(&gu, sizeof(float) * 3 * N);
    if (e == cudaSuccess) e = cudaMalloc(&wu, sizeof(float) * N);
    if (e == cudaSuccess) e = cudaMalloc(&toff, sizeof(int32_t) * (p->ntiles_total + 1));
    if (e == cudaSuccess) e = cudaMalloc(&coff, sizeof(int32_t) * (p->ntiles_total * 8 + 1));
    if (e != cudaSuccess) {
        cudaFree(gu);
        cudaFree(wu);
        cudaFree(toff);
        cudaFree(coff);
        nufft_set_tiles(p, keep_t);   // the plan is unchanged
        set_error("re-binning: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? CS_ERR_OOM : CS_ERR_CUDA;
    }
    CS_TRY_CUDA(cudaStreamSynchronize(st));    // nothing queued still reads the old order
    unsort_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(p->perm, p->gsorted, p->wsorted, N, gu, wu);
    cudaFree(p->tile_off);
    cudaFree(p->class_off);
    p->tile_off = toff;
    p->class_off = coff;
    cs_status rc = nufft_bin(p, gu, wu, 1, st);
    cudaFree(gu);
    cudaFree(wu);
    CS_PROPAGATE(rc);
    CS_PROPAGATE(nufft_records(p, st));
    CS_TRY_CUDA(cudaStreamSynchronize(st));
    if (p->gitems) CS_PROPAGATE(nufft_owner_build(p));
    p->layout_gen++;
    return CS_OK;
}

cs_status nufft_records(cs_plan* p, cudaStream_t st) {
    if (!p->rec) CS_TRY_CUDA(cudaMalloc(&p->rec, sizeof(float) * kRec * (size_t)p->N));   // rewritten in place
    sample_record_kernel<<<(unsigned)((p->N + 255) / 256), 256, 0, st>>>(p->gsorted, p->wsorted, p->perm, p->phi, p->N,
                                                                      p->ndim, p->grid[0], p->grid[1], p->grid[2], p->rec);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

// y (user order) = sqrt(w) interp(grid); with ysub: ktmp (sorted) = sqrt(w) interp(grid) - y
cs_status nufft_interp(const cs_plan* p, int ncoils, float2* y, const float2* ysub, cudaStream_t st) {
    if (ysub) return launch_interp(p, ncoils, OUT_RESID, ysub, p->ktmp, st);
    return launch_interp(p, ncoils, OUT_USER, nullptr, y, st);
}

// grid = spread(sqrt(w) y); y in user order (sorted_in = 0) or the sorted scratch ktmp
cs_status nufft_spread(const cs_plan* p, int ncoils, const float2* y, int sorted_in, cudaStream_t st) {
    float2* grid = grid_buffer(p);
    CS_TRY_CUDA(cudaMemsetAsync(grid, 0, sizeof(float2) * (size_t)p->G * ncoils, st));
    if (ncoils == 0) return CS_OK;
    return launch_spread(p, ncoils, sorted_in ? p->ktmp : y, sorted_in, st);
}

// ktmp (sorted, coil-interleaved) = w^1/2 interp(grid)
cs_status nufft_interp_sorted(const cs_plan* p, int ncoils, cudaStream_t st) {
    return launch_interp(p, ncoils, OUT_SORTED, nullptr, p->ktmp, st);
}

// normal operator on the grid: ktmp = w^1/2 interp(grid) (sorted), then grid = spread(w^1/2 ktmp)
CS_BOUNDS_READER(nufft_bounds_check)

cs_status nufft_interp_spread(const cs_plan* p, int ncoils, cudaStream_t st) {
    CS_PROPAGATE(launch_interp(p, ncoils, OUT_SORTED, nullptr, p->ktmp, st));
    return nufft_spread(p, ncoils, nullptr, 1, st);
}

}  // namespace cs
