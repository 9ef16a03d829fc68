// Coil-space operations of coil sketching (Sec. 2.3, Sec. 3.1, Algorithm 1):
//   coil_pca       SVD-based coil compression: R = Y Y^H, FP64 Hermitian Jacobi eigensolver
//   coil_rotate    c' = U^H c, y' = U^H y
//   sketch_draw    random blocks S~_S^t (Philox4x32-10, Gaussian / Rademacher)
//   sketched_maps  c^_{V+s} = sum_j S~_S[s][j] c'_{V+j}   (Eq. 8, random block only)
#include <cmath>
#include <cstdio>
#include <mutex>

#include "cs_internal.cuh"

namespace cs {

// ------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
struct Philox {
    __host__ __device__ static inline void mulhilo(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
        const uint64_t p = (uint64_t)a * (uint64_t)b;
        hi = (uint32_t)(p >> 32);
        lo = (uint32_t)p;
    }
    __host__ __device__ static inline void block(const uint32_t in[4], const uint32_t key[2], uint32_t out[4]) {
        uint32_t c0 = in[0], c1 = in[1], c2 = in[2], c3 = in[3];
        uint32_t k0 = key[0], k1 = key[1];
        for (int r = 0; r < 10; ++r) {
            if (r) {
                k0 += 0x9E3779B9u;
                k1 += 0xBB67AE85u;
            }
            uint32_t hi0, lo0, hi1, lo1;
            mulhilo(0xD2511F53u, c0, hi0, lo0);
            mulhilo(0xCD9E8D57u, c2, hi1, lo1);
            const uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
            c0 = n0;
            c1 = n1;
            c2 = n2;
            c3 = n3;
        }
        out[0] = c0;
        out[1] = c1;
        out[2] = c2;
        out[3] = c3;
    }
};

// nearest bfloat16 value (ties to even) of a float, returned as float
__host__ __device__ inline float round_bf16(float f) {
    uint32_t b;
    memcpy(&b, &f, 4);
    const uint32_t lsb = (b >> 16) & 1u;
    b = (b + 0x7FFFu + lsb) & 0xFFFF0000u;
    float r;
    memcpy(&r, &b, 4);
    return r;
}

__global__ void sketch_draw_kernel(uint32_t k0, uint32_t k1, int t0, int T, int S, int K, int dist, double scale,
                                   float* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)S * K;
    if (e >= per * T) return;
    const int t = t0 + (int)(e / per);
    const uint32_t idx = (uint32_t)(e % per);
    const uint32_t ctr[4] = {idx, (uint32_t)t, 0u, 0u};
    const uint32_t key[2] = {k0, k1};
    uint32_t o[4];
    Philox::block(ctr, key, o);
    double v;
    if (dist == CS_GAUSSIAN) {
        const double u1 = ((double)(o[0] >> 8) + 0.5) * 0x1.0p-24;
        const double u2 = ((double)(o[1] >> 8) + 0.5) * 0x1.0p-24;
        v = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
    } else {
        v = (o[2] >> 31) ? -1.0 : 1.0;
    }
    out[e] = round_bf16((float)(v * scale));
}

// ------------------------------------------------------------------------------------------
// coil covariance R = Y Y^H: 4x4 coil blocks per thread, FP32 within a 128-sample tile, FP64
// across tiles and CTAs, complex128 [C][C], upper blocks only.  With part == nullptr the thread
// sums go into R with atomic adds (order of the additions set by scheduling); otherwise every
// thread writes its 4x4 block to its own slot part[CTA][thread][16][2] and cov_reduce_kernel adds
// the slots in a fixed order, so R is bit-reproducible.
constexpr int kCovTile = 128;

__global__ void __launch_bounds__(256) cov_kernel(const float2* __restrict__ y, int C, int64_t N,
                                                  double* __restrict__ R, double* __restrict__ part) {
    extern __shared__ float2 tile[];  // [C][kCovTile]
    const int nb = (C + 3) / 4;
    const int npairs = nb * (nb + 1) / 2;
    const int groups = max(1, (int)blockDim.x / npairs);
    const int tid = threadIdx.x;
    const int pair = tid % npairs;
    const int grp = tid / npairs;
    int bi = 0, bj = 0;
    {
        int r = pair;
        while (r >= nb - bi) {
            r -= nb - bi;
            ++bi;
        }
        bj = bi + r;
    }
    const bool active = grp < groups;
    double accd[4][4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) accd[a][b][0] = accd[a][b][1] = 0.0;
    for (int64_t s0 = (int64_t)blockIdx.x * kCovTile; s0 < N; s0 += (int64_t)gridDim.x * kCovTile) {
        __syncthreads();
        for (int e = tid; e < C * kCovTile; e += blockDim.x) {
            const int c = e / kCovTile, s = e % kCovTile;
            tile[e] = (s0 + s < N) ? y[(int64_t)c * N + s0 + s] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (!active) continue;
        float acc[4][4][2];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b][0] = acc[a][b][1] = 0.f;
        for (int s = grp; s < kCovTile; s += groups) {
            float2 ya[4], yb[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int ca = bi * 4 + a, cb = bj * 4 + a;
                ya[a] = ca < C ? tile[ca * kCovTile + s] : make_float2(0.f, 0.f);
                yb[a] = cb < C ? tile[cb * kCovTile + s] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    // y_a conj(y_b)
                    acc[a][b][0] = fmaf(ya[a].x, yb[b].x, fmaf(ya[a].y, yb[b].y, acc[a][b][0]));
                    acc[a][b][1] = fmaf(ya[a].y, yb[b].x, fmaf(-ya[a].x, yb[b].y, acc[a][b][1]));
                }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                accd[a][b][0] += (double)acc[a][b][0];
                accd[a][b][1] += (double)acc[a][b][1];
            }
    }
    if (!active) return;
    if (part) {
        double* slot = part + ((int64_t)blockIdx.x * blockDim.x + tid) * 32;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                slot[(a * 4 + b) * 2 + 0] = accd[a][b][0];
                slot[(a * 4 + b) * 2 + 1] = accd[a][b][1];
            }
        return;
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int ca = bi * 4 + a, cb = bj * 4 + b;
            if (ca < C && cb < C && (bi != bj || ca <= cb)) {
                atomicAdd(&R[2 * (ca * C + cb) + 0], accd[a][b][0]);
                atomicAdd(&R[2 * (ca * C + cb) + 1], accd[a][b][1]);
            }
        }
}

// R[ca][cb] (ca <= cb) = sum over CTAs, then over the thread groups of a CTA, of the slots that
// hold block pair (ca / 4, cb / 4), in that order
__global__ void cov_reduce_kernel(const double* __restrict__ part, int nblocks, int threads, int C,
                                  double* __restrict__ R) {
    const int nb = (C + 3) / 4;
    const int npairs = nb * (nb + 1) / 2;
    const int groups = max(1, threads / npairs);
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= C * C) return;
    const int ca = e / C, cb = e % C;
    if (ca > cb) return;
    const int bi = ca / 4, bj = cb / 4, a = ca % 4, b = cb % 4;
    int pair = bj - bi;                      // the kernel's pair numbering: row bi, column bj >= bi
    for (int i = 0; i < bi; ++i) pair += nb - i;
    double re = 0.0, im = 0.0;
    for (int k = 0; k < nblocks; ++k)
        for (int g = 0; g < groups; ++g) {
            const double* slot = part + ((int64_t)k * threads + g * npairs + pair) * 32 + (a * 4 + b) * 2;
            re += slot[0];
            im += slot[1];
        }
    R[2 * e + 0] = re;
    R[2 * e + 1] = im;
}

// ------------------------------------------------------------------------------------------
// Cyclic complex Jacobi for a Hermitian matrix (FP64).  For pivot (p, q) with
// A[p][q] = |c| e^{i phi}: theta = (a_qq - a_pp) / (2|c|), t = sgn(theta) / (|theta| + sqrt(theta^2 + 1)),
// cs = 1/sqrt(1 + t^2), sn = t cs, and J = [[cs, sn e^{i phi}], [-sn e^{-i phi}, cs]] on (p, q):
// A <- J^H A J zeroes A[p][q]; eigenvectors accumulate V <- V J.
struct Rot {
    double cs, sn, er, ei;  // e^{i phi} = er + i ei
    bool skip;
};

__host__ __device__ inline Rot jacobi_rot(const double* A, int n, int p, int q) {
    Rot r;
    const double cr = A[2 * (p * n + q)], ci = A[2 * (p * n + q) + 1];
    const double mag = sqrt(cr * cr + ci * ci);
    const double app = A[2 * (p * n + p)], aqq = A[2 * (q * n + q)];
    r.skip = !(mag > 1e-300) || mag <= 1e-18 * (fabs(app) + fabs(aqq)) * 1e-2;
    if (r.skip) {
        r.cs = 1;
        r.sn = 0;
        r.er = 1;
        r.ei = 0;
        return r;
    }
    const double theta = (aqq - app) / (2.0 * mag);
    double t = 1.0 / (fabs(theta) + sqrt(theta * theta + 1.0));
    if (theta < 0) t = -t;
    r.cs = 1.0 / sqrt(1.0 + t * t);
    r.sn = t * r.cs;
    r.er = cr / mag;
    r.ei = ci / mag;
    return r;
}

// column update of rows k: M[k][p], M[k][q] <- M J
__host__ __device__ inline void rot_cols(double* M, int n, int k, int p, int q, const Rot& r) {
    const double xr = M[2 * (k * n + p)], xi = M[2 * (k * n + p) + 1];
    const double yr = M[2 * (k * n + q)], yi = M[2 * (k * n + q) + 1];
    // new_p = cs x - sn e^{-i phi} y ; new_q = sn e^{i phi} x + cs y
    const double ayr = r.er * yr + r.ei * yi, ayi = r.er * yi - r.ei * yr;   // e^{-i phi} y
    const double axr = r.er * xr - r.ei * xi, axi = r.er * xi + r.ei * xr;   // e^{i phi} x
    M[2 * (k * n + p)] = r.cs * xr - r.sn * ayr;
    M[2 * (k * n + p) + 1] = r.cs * xi - r.sn * ayi;
    M[2 * (k * n + q)] = r.sn * axr + r.cs * yr;
    M[2 * (k * n + q) + 1] = r.sn * axi + r.cs * yi;
}

// row update of columns k: A[p][k], A[q][k] <- J^H A
__host__ __device__ inline void rot_rows(double* A, int n, int k, int p, int q, const Rot& r) {
    const double xr = A[2 * (p * n + k)], xi = A[2 * (p * n + k) + 1];
    const double yr = A[2 * (q * n + k)], yi = A[2 * (q * n + k) + 1];
    // new_p = cs x - sn e^{i phi} y ; new_q = sn e^{-i phi} x + cs y
    const double ayr = r.er * yr - r.ei * yi, ayi = r.er * yi + r.ei * yr;   // e^{i phi} y
    const double axr = r.er * xr + r.ei * xi, axi = r.er * xi - r.ei * xr;   // e^{-i phi} x
    A[2 * (p * n + k)] = r.cs * xr - r.sn * ayr;
    A[2 * (p * n + k) + 1] = r.cs * xi - r.sn * ayi;
    A[2 * (q * n + k)] = r.sn * axr + r.cs * yr;
    A[2 * (q * n + k) + 1] = r.sn * axi + r.cs * yi;
}

__host__ __device__ inline double offdiag2(const double* A, int n) {
    double s = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (i != j) s += A[2 * (i * n + j)] * A[2 * (i * n + j)] + A[2 * (i * n + j) + 1] * A[2 * (i * n + j) + 1];
    return s;
}

// sort descending, fix phases (largest-magnitude entry of each column real positive)
__host__ __device__ inline void eig_finish(double* A, int n, double* V, double* ev) {
    for (int i = 0; i < n; ++i) ev[i] = A[2 * (i * n + i)];
    for (int i = 0; i < n; ++i) {
        int best = i;
        for (int j = i + 1; j < n; ++j)
            if (ev[j] > ev[best]) best = j;
        if (best != i) {
            const double t = ev[i];
            ev[i] = ev[best];
            ev[best] = t;
            for (int k = 0; k < n; ++k) {
                const double ar = V[2 * (k * n + i)], ai = V[2 * (k * n + i) + 1];
                V[2 * (k * n + i)] = V[2 * (k * n + best)];
                V[2 * (k * n + i) + 1] = V[2 * (k * n + best) + 1];
                V[2 * (k * n + best)] = ar;
                V[2 * (k * n + best) + 1] = ai;
            }
        }
    }
    for (int i = 0; i < n; ++i) {
        int jm = 0;
        double mm = -1;
        for (int k = 0; k < n; ++k) {
            const double m = V[2 * (k * n + i)] * V[2 * (k * n + i)] + V[2 * (k * n + i) + 1] * V[2 * (k * n + i) + 1];
            if (m > mm) {
                mm = m;
                jm = k;
            }
        }
        const double pr = V[2 * (jm * n + i)], pi = V[2 * (jm * n + i) + 1];
        const double pm = sqrt(pr * pr + pi * pi);
        if (pm > 0) {
            const double ur = pr / pm, ui = -pi / pm;  // conj(phase)
            for (int k = 0; k < n; ++k) {
                const double vr = V[2 * (k * n + i)], vi = V[2 * (k * n + i) + 1];
                V[2 * (k * n + i)] = vr * ur - vi * ui;
                V[2 * (k * n + i) + 1] = vr * ui + vi * ur;
            }
            V[2 * (jm * n + i) + 1] = 0.0;
        }
    }
}

constexpr int kJacobiSweeps = 40;

void hermitian_eig_serial(double* A, int n, double* V, double* ev) {
    for (int i = 0; i < n * n * 2; ++i) V[i] = 0;
    for (int i = 0; i < n; ++i) V[2 * (i * n + i)] = 1;
    double fro = 0;
    for (int i = 0; i < 2 * n * n; ++i) fro += A[i] * A[i];
    for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
        if (offdiag2(A, n) <= 1e-30 * fro) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const Rot r = jacobi_rot(A, n, p, q);
                if (r.skip) continue;
                for (int k = 0; k < n; ++k) rot_cols(A, n, k, p, q, r);
                for (int k = 0; k < n; ++k) rot_rows(A, n, k, p, q, r);
                for (int k = 0; k < n; ++k) rot_cols(V, n, k, p, q, r);
                A[2 * (p * n + q)] = A[2 * (p * n + q) + 1] = 0;
                A[2 * (q * n + p)] = A[2 * (q * n + p) + 1] = 0;
            }
    }
    eig_finish(A, n, V, ev);
}

// One CTA: the same sweeps with the O(n) row/column updates spread over threads.
// Parallel ordering of the same rotations (Brent and Luk's round robin): a sweep is m - 1 rounds
// (m = n rounded up to even; the pairs with the extra index of odd n are skipped), each of m/2
// disjoint pivot pairs.  All rotation angles of a round come from the matrix before the round;
// because the pairs are disjoint, applying every column rotation and then every row rotation is
// J^H A J for J the product of the round's rotations, and it zeroes each pivot entry exactly as
// the single rotation would.  A sweep still visits every pair once.
__global__ void jacobi_kernel(const double* __restrict__ Rin, int n, float2* __restrict__ Uout,
                              double* __restrict__ evout) {
    extern __shared__ double sm[];
    double* A = sm;
    double* V = sm + 2 * n * n;
    __shared__ Rot rots[32];
    __shared__ int pp[32], pq[32];
    __shared__ double s_off, s_fro;
    __shared__ double ev[64];
    const int tid = threadIdx.x;
    // Hermitian fill from the upper triangle
    for (int e = tid; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        if (i <= j) {
            A[2 * e] = Rin[2 * e];
            A[2 * e + 1] = (i == j) ? 0.0 : Rin[2 * e + 1];
        } else {
            A[2 * e] = Rin[2 * (j * n + i)];
            A[2 * e + 1] = -Rin[2 * (j * n + i) + 1];
        }
        V[2 * e] = (i == j) ? 1.0 : 0.0;
        V[2 * e + 1] = 0.0;
    }
    __syncthreads();
    if (tid == 0) {
        double f = 0;
        for (int i = 0; i < 2 * n * n; ++i) f += A[i] * A[i];
        s_fro = f;
    }
    __syncthreads();
    const int m = (n + 1) & ~1;
    const int half = m / 2;
    for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
        if (tid == 0) s_off = offdiag2(A, n);
        __syncthreads();
        if (s_off <= 1e-30 * s_fro) break;
        for (int round = 0; round < m - 1; ++round) {
            if (tid < half) {
                // player at seat k in this round: seat 0 fixed, the others rotate
                auto player = [&](int k) { return k == 0 ? 0 : 1 + (k - 1 + round) % (m - 1); };
                int p = player(tid), q = player(m - 1 - tid);
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                Rot r;
                if (q >= n) {
                    r.cs = 1;
                    r.sn = 0;
                    r.er = 1;
                    r.ei = 0;
                    r.skip = true;
                } else {
                    r = jacobi_rot(A, n, p, q);
                }
                rots[tid] = r;
                pp[tid] = p;
                pq[tid] = q;
            }
            __syncthreads();
            for (int e = tid; e < half * n; e += blockDim.x) {   // columns p, q of A and V
                const int i = e / n, k = e - (e / n) * n;
                if (!rots[i].skip) {
                    rot_cols(A, n, k, pp[i], pq[i], rots[i]);
                    rot_cols(V, n, k, pp[i], pq[i], rots[i]);
                }
            }
            __syncthreads();
            for (int e = tid; e < half * n; e += blockDim.x) {   // rows p, q of A
                const int i = e / n, k = e - (e / n) * n;
                if (!rots[i].skip) rot_rows(A, n, k, pp[i], pq[i], rots[i]);
            }
            __syncthreads();
            if (tid < half && !rots[tid].skip) {
                const int p = pp[tid], q = pq[tid];
                A[2 * (p * n + q)] = A[2 * (p * n + q) + 1] = 0;
                A[2 * (q * n + p)] = A[2 * (q * n + p) + 1] = 0;
            }
            __syncthreads();
        }
    }
    if (tid == 0) eig_finish(A, n, V, ev);
    __syncthreads();
    for (int e = tid; e < n * n; e += blockDim.x) Uout[e] = make_float2((float)V[2 * e], (float)V[2 * e + 1]);
    for (int e = tid; e < n; e += blockDim.x) evout[e] = ev[e];
}

// ------------------------------------------------------------------------------------------
// out[k][l] = sum_c conj(U[c][k]) in[c][l]; a CTA covers 64 columns, a thread 8 outputs k.
constexpr int kRotCols = 64;

__global__ void rotate_kernel(const float2* __restrict__ U, const float2* __restrict__ in, int C, int Cout, int64_t L,
                              float2* __restrict__ out) {
    extern __shared__ float2 rsm[];
    float2* Us = rsm;             // [C][C]
    float2* tile = rsm + C * C;   // [C][kRotCols]
    const int tid = threadIdx.x;
    for (int e = tid; e < C * C; e += blockDim.x) Us[e] = U[e];
    const int l = tid % kRotCols;
    const int kg = tid / kRotCols;
    for (int64_t l0 = (int64_t)blockIdx.x * kRotCols; l0 < L; l0 += (int64_t)gridDim.x * kRotCols) {
        __syncthreads();
        for (int e = tid; e < C * kRotCols; e += blockDim.x) {
            const int c = e / kRotCols, ll = e % kRotCols;
            tile[e] = (l0 + ll < L) ? in[(int64_t)c * L + l0 + ll] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        float2 acc[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] = make_float2(0.f, 0.f);
        for (int c = 0; c < C; ++c) {
            const float2 v = tile[c * kRotCols + l];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = kg * 8 + j;
                if (k < Cout) acc[j] = cadd(acc[j], cmulc(Us[c * C + k], v));
            }
        }
        if (l0 + l < L) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = kg * 8 + j;
                if (k < Cout) out[(int64_t)k * L + l0 + l] = acc[j];
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// FP32 sketched maps: one thread per voxel, S <= 32 outputs in registers
constexpr int kMaxSketchRows = 32;

__global__ void sketch_maps_fp32_kernel(const float* __restrict__ Sk, const int* __restrict__ tsel, const float2* __restrict__ mrot,
                                        int64_t D, int V, int K, int Sn, float2* __restrict__ out) {
    __shared__ float sS[kMaxSketchRows * 64];
    if (tsel) Sk += (int64_t)(*tsel) * Sn * K;
    for (int e = threadIdx.x; e < Sn * K; e += blockDim.x) sS[e] = Sk[e];
    __syncthreads();
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < D; d += (int64_t)gridDim.x * blockDim.x) {
        float2 acc[kMaxSketchRows];
#pragma unroll
        for (int s = 0; s < kMaxSketchRows; ++s) acc[s] = make_float2(0.f, 0.f);
        for (int j = 0; j < K; ++j) {
            const float2 m = mrot[(int64_t)(V + j) * D + d];
#pragma unroll
            for (int s = 0; s < kMaxSketchRows; ++s) {
                if (s < Sn) {
                    const float w = sS[s * K + j];
                    acc[s].x = fmaf(w, m.x, acc[s].x);
                    acc[s].y = fmaf(w, m.y, acc[s].y);
                }
            }
        }
#pragma unroll
        for (int s = 0; s < kMaxSketchRows; ++s)
            if (s < Sn) out[(int64_t)s * D + d] = acc[s];
    }
}

cs_status tc_check_and_clear();

// tensor-core split-precision variant (sketch_tc.cu)
cs_status sketched_maps_bf16split(const float* S, const int* tsel, const float2* mrot, int64_t D, int C, int V, int Sn,
                                  float2* out, cudaStream_t st);

static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}

// dynamic shared-memory limits for up to 64 coils (set once per device at plan creation)
cs_status coil_init_attrs() {
    CS_TRY_CUDA(cudaFuncSetAttribute(cov_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(float2) * 64 * kCovTile)));
    CS_TRY_CUDA(cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(double) * 4 * 64 * 64)));
    CS_TRY_CUDA(cudaFuncSetAttribute(rotate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(float2) * (64 * 64 + 64 * kRotCols))));
    return CS_OK;
}

static cs_status coil_attrs_once() {
    static std::mutex mu;
    static bool done[128] = {false};
    int dev = 0;
    CS_TRY_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 128 && !done[dev]) {
        CS_PROPAGATE(coil_init_attrs());
        done[dev] = true;
    }
    return CS_OK;
}

// the device-side index checks of every translation unit with guarded accesses (checked builds)
cs_status bounds_check_all() {
    CS_PROPAGATE(nufft_bounds_check());
    return fft_bounds_check();
}

static void cov_launch_shape(int C, int64_t N, int* threads, int* grid) {
    const int nb = (C + 3) / 4;
    const int npairs = nb * (nb + 1) / 2;
    *threads = npairs > 256 ? ((npairs + 31) / 32) * 32 : 256;
    const int64_t tiles = (N + kCovTile - 1) / kCovTile;
    *grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sm_count() * 4));
}

// doubles of the slot array of the bit-reproducible covariance
int64_t coil_cov_part_size(int C, int64_t N) {
    int threads = 0, grid = 0;
    cov_launch_shape(C, N, &threads, &grid);
    return (int64_t)grid * threads * 32;
}

// coil PCA with the covariance accumulated by atomic adds (no slot array; coil_pca_noalloc)
cs_status coil_pca_impl(const float2* y, int C, int64_t N, float2* U, double* eig, double* Rws, cudaStream_t st) {
    CS_TRY_CUDA(cudaMemsetAsync(Rws, 0, sizeof(double) * 2 * C * C, st));
    int threads = 0, grid = 0;
    cov_launch_shape(C, N, &threads, &grid);
    CS_REQUIRE(threads <= 1024, CS_ERR_UNSUPPORTED_SIZE, "too many coils for coil_pca");
    const size_t sm = sizeof(float2) * C * kCovTile;
    cov_kernel<<<grid, threads, sm, st>>>(y, C, N, Rws, nullptr);
    CS_LAUNCH_CHECK();
    const size_t jsm = sizeof(double) * 4 * C * C;
    jacobi_kernel<<<1, 256, jsm, st>>>(Rws, C, U, eig);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

// coil PCA with the bit-reproducible covariance: `part` holds coil_cov_part_size(C, N) doubles
cs_status coil_pca_det_impl(const float2* y, int C, int64_t N, float2* U, double* eig, double* Rws, double* part,
                            cudaStream_t st) {
    int threads = 0, grid = 0;
    cov_launch_shape(C, N, &threads, &grid);
    CS_REQUIRE(threads <= 1024, CS_ERR_UNSUPPORTED_SIZE, "too many coils for coil_pca");
    CS_TRY_CUDA(cudaMemsetAsync(Rws, 0, sizeof(double) * 2 * C * C, st));
    const size_t sm = sizeof(float2) * C * kCovTile;
    cov_kernel<<<grid, threads, sm, st>>>(y, C, N, Rws, part);
    CS_LAUNCH_CHECK();
    cov_reduce_kernel<<<(C * C + 255) / 256, 256, 0, st>>>(part, grid, threads, C, Rws);
    CS_LAUNCH_CHECK();
    const size_t jsm = sizeof(double) * 4 * C * C;
    jacobi_kernel<<<1, 256, jsm, st>>>(Rws, C, U, eig);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

cs_status coil_rotate_impl(const float2* U, const float2* in, int C, int Cout, int64_t L, float2* out, cudaStream_t st) {
    const int groups = (Cout + 7) / 8;
    const int threads = kRotCols * groups;
    const size_t sm = sizeof(float2) * ((size_t)C * C + (size_t)C * kRotCols);
    const int64_t blocks = (L + kRotCols - 1) / kRotCols;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sm_count() * 8));
    rotate_kernel<<<grid, threads, sm, st>>>(U, in, C, Cout, L, out);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

cs_status sketch_draw_impl(uint64_t seed, int t0, int T, int C, int V, int S, int dist, int norm, float* out,
                           cudaStream_t st) {
    const int K = C - V;
    const int64_t n = (int64_t)T * S * K;
    if (n == 0) return CS_OK;
    double scale;
    if (dist == CS_GAUSSIAN) scale = (norm == CS_NORM_UNIT_VAR) ? 1.0 / std::sqrt((double)S) : 1.0 / S;
    else scale = (norm == CS_NORM_UNIT_VAR) ? 1.0 / std::sqrt((double)S) : 1.0;
    sketch_draw_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32),
                                                                   t0, T, S, K, dist, scale, out);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

// tsel (device, nullable): use the sketch block S + (*tsel) * Sn * (C - V)
cs_status sketched_maps_impl(const float* S, const int* tsel, const float2* mrot, int64_t D, int C, int V, int Sn,
                             int precision, float2* out, cudaStream_t st) {
    const int K = C - V;
    if (Sn == 0 || D == 0) return CS_OK;
    if (precision == CS_PREC_BF16_SPLIT) return sketched_maps_bf16split(S, tsel, mrot, D, C, V, Sn, out, st);
    const int64_t blocks = (D + 255) / 256;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sm_count() * 8));
    sketch_maps_fp32_kernel<<<grid, 256, 0, st>>>(S, tsel, mrot, D, V, K, Sn, out);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

// ------------------------------------------------------------------------------------------
// Statically allocated scratch for coil_pca_noalloc: the FP64 coil covariance (complex128 C x C)
// of at most kNoAllocMaxCoils coils, 64 KiB, held by every device that loads the library.
constexpr int kNoAllocMaxCoils = 64;
static __device__ __align__(256) double g_pca_scratch[2 * kNoAllocMaxCoils * kNoAllocMaxCoils];

// Device address of g_pca_scratch for the current device.  The name g_pca_scratch in host code
// is only a host-side stand-in, so the address is looked up once per device with that device
// current and cached.
static cs_status pca_scratch_address(double** out) {
    static std::mutex mu;
    static double* addr[128] = {nullptr};
    int dev = 0;
    CS_TRY_CUDA(cudaGetDevice(&dev));
    CS_REQUIRE(dev >= 0 && dev < 128, CS_ERR_INVALID_ARG, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_pca_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_error("coil_pca_noalloc: cudaGetSymbolAddress failed on device %d: %s", dev, cudaGetErrorString(e));
            return CS_ERR_CUDA;
        }
        addr[dev] = (double*)p;
    }
    *out = addr[dev];
    return CS_OK;
}

}  // namespace cs

using namespace cs;

extern "C" {

cs_status coil_pca_noalloc(const float* y, int C, int64_t N, float* U, double* eig, void* stream) {
    clear_error();
    CS_REQUIRE(y && U && eig && N >= 1, CS_ERR_INVALID_ARG, "bad coil_pca_noalloc arguments");
    CS_REQUIRE(C >= 1 && C <= kNoAllocMaxCoils, CS_ERR_UNSUPPORTED_SIZE,
               "coil_pca_noalloc supports at most %d coils (got %d); use coil_pca", kNoAllocMaxCoils, C);
    double* R = nullptr;
    CS_PROPAGATE(coil_attrs_once());
    CS_PROPAGATE(pca_scratch_address(&R));
    // coil_pca_impl clears R on `stream` before accumulating into it
    return coil_pca_impl((const float2*)y, C, N, (float2*)U, eig, R, (cudaStream_t)stream);
}

cs_status cs_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    clear_error();
    CS_REQUIRE(ctr && key && out, CS_ERR_INVALID_ARG, "null pointer");
    Philox::block(ctr, key, out);
    return CS_OK;
}

cs_status cs_hermitian_eig_host(const double* A, int n, double* evecs, double* evals) {
    clear_error();
    CS_REQUIRE(A && evecs && evals && n >= 1 && n <= 64, CS_ERR_INVALID_ARG, "bad arguments");
    std::vector<double> W(A, A + 2 * n * n);
    hermitian_eig_serial(W.data(), n, evecs, evals);
    return CS_OK;
}

cs_status sketch_draw(uint64_t seed, int t0, int T, int C, int V, int S, int dist, int norm, float* out, void* stream) {
    clear_error();
    CS_REQUIRE(out && T >= 0 && t0 >= 0 && C >= 1 && V >= 0 && S >= 0 && V + S <= C && V <= C,
               CS_ERR_INVALID_ARG, "bad sketch sizes (C=%d V=%d S=%d)", C, V, S);
    CS_REQUIRE(S <= kMaxSketchRows && C - V <= 64, CS_ERR_UNSUPPORTED_SIZE, "sketch larger than 32 x 64");
    CS_REQUIRE(dist == CS_GAUSSIAN || dist == CS_RADEMACHER, CS_ERR_INVALID_ARG, "bad distribution");
    return sketch_draw_impl(seed, t0, T, C, V, S, dist, norm, out, (cudaStream_t)stream);
}

cs_status coil_pca(const float* y, int C, int64_t N, float* U, double* eig, void* stream) {
    clear_error();
    CS_REQUIRE(y && U && eig && C >= 1 && C <= 64 && N >= 1, CS_ERR_INVALID_ARG, "bad coil_pca arguments");
    cudaStream_t st = (cudaStream_t)stream;
    CS_PROPAGATE(coil_attrs_once());
    double* R = nullptr;
    const int64_t np = coil_cov_part_size(C, N);
    CS_TRY_CUDA(cudaMallocAsync(&R, sizeof(double) * (2 * C * C + np), st));
    cs_status rc = coil_pca_det_impl((const float2*)y, C, N, (float2*)U, eig, R, R + 2 * C * C, st);
    cudaFreeAsync(R, st);
    return rc;
}

cs_status coil_rotate(const float* U, const float* in, int C, int C_out, int64_t L, float* out, void* stream) {
    clear_error();
    CS_REQUIRE(U && in && out && C >= 1 && C <= 64 && C_out >= 0 && C_out <= C && L >= 0, CS_ERR_INVALID_ARG,
               "bad coil_rotate arguments");
    CS_REQUIRE(in != out, CS_ERR_INVALID_ARG, "coil_rotate cannot run in place");
    if (C_out == 0 || L == 0) return CS_OK;
    CS_PROPAGATE(coil_attrs_once());
    return coil_rotate_impl((const float2*)U, (const float2*)in, C, C_out, L, (float2*)out, (cudaStream_t)stream);
}

cs_status cs_device_status(void* stream) {
    clear_error();
    CS_TRY_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    CS_PROPAGATE(fft_check_and_clear());
    CS_PROPAGATE(bounds_check_all());
    return tc_check_and_clear();
}

cs_status sketched_maps(const float* S, const float* maps_rot, int64_t D, int C, int V, int Sn, int precision,
                        float* maps_s, void* stream) {
    clear_error();
    CS_REQUIRE(S && maps_rot && maps_s && D >= 0 && V >= 0 && Sn >= 0 && V <= C && Sn <= kMaxSketchRows && C - V <= 64,
               CS_ERR_INVALID_ARG, "bad sketched_maps arguments");
    CS_REQUIRE(precision == CS_PREC_FP32 || precision == CS_PREC_BF16_SPLIT, CS_ERR_INVALID_ARG, "bad precision");
    return sketched_maps_impl(S, nullptr, (const float2*)maps_rot, D, C, V, Sn, precision, (float2*)maps_s,
                              (cudaStream_t)stream);
}

}  // extern "C"
