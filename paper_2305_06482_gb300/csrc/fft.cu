// Mixed-radix Stockham FFT passes over one axis of a coil stack, with the SENSE operator's
// element-wise work fused into the first and last pass (Sec. 2.1, Eq. 5: y_c = w^1/2 F{c_c x}).
//
// A CTA transforms kLines lines of length n held in shared memory as buf[k * kLinePad + l]
// (line index fastest), so butterfly threads walk consecutive lines; buffers are coil-
// interleaved so that the kLines lines of a CTA are contiguous in global memory for every axis.  Each radix-r stage of the Stockham autosort
// formulation reads a[j + q n/r], twiddles by exp(-+2 pi i q k / (Ns r)) (k = j mod Ns, Ns the
// product of earlier radices), applies the r-point DFT and writes b[(j/Ns) Ns r + k + q Ns].
//
// Pass modes
//   EXPAND_X   x (.) c_c (.) apod -> zero-padded rows -> FFT along x        (first forward pass)
//   PLAIN      strided axis, zero-pad on input / crop on output            (middle passes)
//   GATHER_Y   FFT along y, keep the sampled entries U (Cartesian forward)
//   SCATTER_Y  U^H (zero-fill) then inverse FFT along y (Cartesian adjoint)
//   MASK_Y     FFT along y, U^H U (optionally minus the data: residual), inverse FFT
//   REDUCE_X   inverse FFT along x, crop, apod, sum_c conj(c_c) (.) (+ lambda v)  (last adjoint)
#include <cstdio>
#include <cmath>

#include "cs_internal.cuh"

namespace cs {

cs_status fft_len_init(FftLen& f, int n) {
    CS_REQUIRE(n >= 2 && n <= kMaxFft, CS_ERR_UNSUPPORTED_SIZE, "FFT length %d outside [2, %d]", n, kMaxFft);
    f.n = n;
    f.nrad = 0;
    int m = n;
    const int order[] = {8, 4, 2, 3, 5, 7, 11};
    for (int r : order) {
        while (m % r == 0) {
            CS_REQUIRE(f.nrad < kMaxRadices, CS_ERR_UNSUPPORTED_SIZE, "too many radices for %d", n);
            f.rad[f.nrad++] = r;
            m /= r;
        }
    }
    CS_REQUIRE(m == 1, CS_ERR_UNSUPPORTED_SIZE,
               "FFT length %d has a prime factor outside {2, 3, 5, 7, 11}", n);
    std::vector<float2> h(n);
    for (int k = 0; k < n; ++k) {
        double a = -2.0 * M_PI * (double)k / (double)n;
        h[k] = make_float2((float)cos(a), (float)sin(a));
    }
    CS_TRY_CUDA(cudaMalloc(&f.tw, sizeof(float2) * n));
    CS_TRY_CUDA(cudaMemcpy(f.tw, h.data(), sizeof(float2) * n, cudaMemcpyHostToDevice));
    return CS_OK;
}

void fft_len_free(FftLen& f) {
    if (f.tw) cudaFree(f.tw);
    f.tw = nullptr;
}

// ------------------------------------------------------------------------------------------
// small DFTs (sign = -1 forward, +1 inverse); roots of unity for the generic radices are read
// from the length-n twiddle table (r divides n, so exp(-2 pi i m / r) = tw[m n / r]).
template <int R>
__device__ __forceinline__ void dft_small(float2 (&v)[R], int sign, const float2* tw, int n) {
    float2 o[R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
        float2 acc = v[0];
#pragma unroll
        for (int q = 1; q < R; ++q) {
            float2 w = tw[((q * m) % R) * (n / R)];
            if (sign > 0) w.y = -w.y;
            acc = cadd(acc, cmul(v[q], w));
        }
        o[m] = acc;
    }
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = o[m];
}

__device__ __forceinline__ float2 rot_mi(float2 a, int sign) {
    // multiply by -i (forward) or +i (inverse)
    return sign < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

template <>
__device__ __forceinline__ void dft_small<2>(float2 (&v)[2], int, const float2*, int) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <>
__device__ __forceinline__ void dft_small<4>(float2 (&v)[4], int sign, const float2*, int) {
    float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    float2 s13 = cadd(v[1], v[3]), d13 = rot_mi(csub(v[1], v[3]), sign);
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
}

template <>
__device__ __forceinline__ void dft_small<8>(float2 (&v)[8], int sign, const float2*, int) {
    const float h = 0.70710678118654752440f;
    // radix-2 split into even/odd 4-point DFTs
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    dft_small<4>(e, sign, nullptr, 0);
    dft_small<4>(o, sign, nullptr, 0);
    // twiddles exp(sign * 2 pi i m / 8), m = 0..3
    float2 t1 = make_float2(h * (o[1].x - sign * o[1].y) * 1.0f, h * (o[1].y + sign * o[1].x));
    float2 t2 = rot_mi(o[2], sign);
    float2 t3 = make_float2(h * (-o[3].x - sign * o[3].y), h * (-o[3].y + sign * o[3].x));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], t1);
    v[5] = csub(e[1], t1);
    v[2] = cadd(e[2], t2);
    v[6] = csub(e[2], t2);
    v[3] = cadd(e[3], t3);
    v[7] = csub(e[3], t3);
}

// q = j / Ns for 0 <= j < 2^16 and 2 <= Ns < 2^16 via a multiply-shift with mag = floor(2^32 / Ns) + 1
// (the error of j * mag / 2^32 against j / Ns stays below 1 / Ns there); Ns = 1 is passed through
__device__ __forceinline__ int divmagic(int j, int Ns, uint32_t mag) {
    return Ns == 1 ? j : (int)__umulhi((uint32_t)j, mag);
}

template <int R>
__device__ __forceinline__ void stockham_stage(const float2* __restrict__ a, float2* __restrict__ b,
                                               const float2* tw, int n, int Ns, uint32_t mag, int sign) {
    const int nb = n / R;
    const int tstride = n / (Ns * R);
    for (int t = threadIdx.x; t < nb * kLines; t += blockDim.x) {
        const int l = t % kLines;
        const int j = t / kLines;
        const int jq = divmagic(j, Ns, mag);
        const int k = j - jq * Ns;
        float2 v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = a[(j + q * nb) * kLinePad + l];
        if (Ns > 1) {
#pragma unroll
            for (int q = 1; q < R; ++q) {
                float2 w = tw[q * k * tstride];
                if (sign > 0) w.y = -w.y;
                v[q] = cmul(v[q], w);
            }
        }
        dft_small<R>(v, sign, tw, n);
        const int base = jq * Ns * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) b[(base + q * Ns) * kLinePad + l] = v[q];
    }
}

// Transform kLines lines in shared memory; returns the buffer holding the result.
__device__ float2* fft_lines(float2* a, float2* b, const float2* tw, int n, const int* rad, int nrad,
                             int sign) {
    int Ns = 1;
    for (int s = 0; s < nrad; ++s) {
        const int r = rad[s];
        const uint32_t mag = (uint32_t)(0x100000000ull / (unsigned long long)Ns) + 1u;
        switch (r) {
            case 2: stockham_stage<2>(a, b, tw, n, Ns, mag, sign); break;
            case 3: stockham_stage<3>(a, b, tw, n, Ns, mag, sign); break;
            case 4: stockham_stage<4>(a, b, tw, n, Ns, mag, sign); break;
            case 5: stockham_stage<5>(a, b, tw, n, Ns, mag, sign); break;
            case 7: stockham_stage<7>(a, b, tw, n, Ns, mag, sign); break;
            case 8: stockham_stage<8>(a, b, tw, n, Ns, mag, sign); break;
            case 11: stockham_stage<11>(a, b, tw, n, Ns, mag, sign); break;
            default: break;
        }
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        Ns *= r;
    }
    return a;
}

// ------------------------------------------------------------------------------------------
// Pass kernels.  Coil stacks are stored coil-interleaved: element (..., k, ..., c) of an
// intermediate or grid buffer sits at ((... * n + k) * inner_rest + ...) * C + c, so a line is
// (position along the other axes, coil) and kLines consecutive lines are contiguous in memory
// for every axis, including x.
enum PassMode { EXPAND_X = 0, PLAIN = 1, GATHER_Y = 2, SCATTER_Y = 3, MASK_Y = 4, REDUCE_X = 5 };

struct PassArgs {
    int n, nrad, rad[kMaxRadices];
    const float2* tw;
    int sign;
    int64_t outer;   // PLAIN / Y modes: outer index count
    int64_t inner;   // PLAIN / Y modes: stride of the FFT axis in elements (includes the coil count)
    int n_in, in_off, n_out, out_off;
    const float2* in;
    float2* out;
    // X modes: image rows and coils
    int64_t rows;    // nz * ny image rows
    int C;           // coils (interleave stride)
    int rows_per_cta;
    // maps / image
    const float2* maps_v;
    const float2* maps_s;
    int V;
    int64_t D;
    const float2* x;
    float2* xo;
    const float2* addv;
    float lambda;
    int accumulate;
    const float* apz;
    const float* apy;
    const float* apx;
    int nyi, nxi;
    // Cartesian sampling
    const int32_t* idxmap;
    const float2* yk;
    float2* yko;
    int64_t N;
    int residual;
};

__device__ __forceinline__ const float2* coil_map(const PassArgs& A, int c) {
    return c < A.V ? A.maps_v + (int64_t)c * A.D : A.maps_s + (int64_t)(c - A.V) * A.D;
}

__device__ __forceinline__ bool cart_neg(int py, int px, int ny, int nx) {
    return (py + px + ny / 2 + nx / 2) & 1;
}

template <int MODE>
__global__ void __launch_bounds__(kPassThreads, 3) fft_pass_kernel(PassArgs A) {
    extern __shared__ float2 smem[];
    const int n = A.n;
    float2* bufa = smem;
    float2* bufb = smem + n * kLinePad;
    float2* stw = smem + 2 * n * kLinePad;
    __shared__ int srad[kMaxRadices];
    if (threadIdx.x < kMaxRadices) srad[threadIdx.x] = A.rad[threadIdx.x];
    for (int e = threadIdx.x; e < n; e += blockDim.x) stw[e] = A.tw[e];
    const int tid = threadIdx.x;

    if (MODE == REDUCE_X) {
        // ---- rows_per_cta image rows; inverse FFT of every coil's line, crop, conj(map),
        //      apodisation and the sum over coils (deterministic order) ----
        constexpr int MAXE = 4;     // rows_per_cta * nx <= 4 * kPassThreads (set by pass_reduce)
        float2 acc[MAXE];
#pragma unroll
        for (int e = 0; e < MAXE; ++e) acc[e] = make_float2(0.f, 0.f);
        const int nx = A.nxi;
        const int R = A.rows_per_cta;
        const int64_t r0 = (int64_t)blockIdx.x * R;
        const int cwmax = (A.C >= kLines) ? kLines : A.C;
        for (int c0 = 0; c0 < A.C; c0 += cwmax) {
            const int cw = min(cwmax, A.C - c0);
            const int nl = R * cw;
            __syncthreads();
            for (int e = tid; e < kLines * n; e += blockDim.x) {
                const int l = e % kLines, k = e / kLines;
                float2 v = make_float2(0.f, 0.f);
                if (l < nl) {
                    const int64_t row = r0 + l / cw;
                    const int c = c0 + l % cw;
                    if (row < A.rows) v = A.in[(row * n + k) * A.C + c];
                }
                bufa[k * kLinePad + l] = v;
            }
            __syncthreads();
            float2* res = fft_lines(bufa, bufb, stw, n, srad, A.nrad, A.sign);
#pragma unroll
            for (int e = 0; e < MAXE; ++e) {
                const int idx = tid + e * kPassThreads;
                if (idx < R * nx) {
                    const int rr = idx / nx, i = idx % nx;
                    const int64_t row = r0 + rr;
                    if (row < A.rows) {
                        for (int q = 0; q < cw; ++q) {
                            const int l = rr * cw + q;
                            const float2 v = res[(i + A.out_off) * kLinePad + l];
                            const float2 m = coil_map(A, c0 + q)[row * nx + i];
                            acc[e] = cadd(acc[e], cmulc(m, v));
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int e = 0; e < MAXE; ++e) {
            const int idx = tid + e * kPassThreads;
            if (idx < R * nx) {
                const int rr = idx / nx, i = idx % nx;
                const int64_t row = r0 + rr;
                if (row < A.rows) {
                    const int z = (int)(row / A.nyi), yy = (int)(row % A.nyi);
                    const float ap = A.apz[z] * A.apy[yy] * A.apx[i];
                    float2 r = cscale(acc[e], ap);
                    const int64_t g = row * nx + i;
                    if (A.addv) r = cadd(r, cscale(A.addv[g], A.lambda));
                    if (A.accumulate) r = cadd(r, A.xo[g]);
                    A.xo[g] = r;
                }
            }
        }
        return;
    }

    // ---------------------------------- load ----------------------------------
    int64_t o0 = 0, i0 = 0;
    if (MODE == EXPAND_X) {
        i0 = (int64_t)blockIdx.x * kLines;  // first line = row * C + c
        const int nx = A.nxi;
        const int64_t nlines = A.rows * A.C;
        __syncthreads();
        for (int e = tid; e < kLines * nx; e += blockDim.x) {
            const int l = e / nx, i = e % nx;
            const int64_t L = i0 + l;
            float2 v = make_float2(0.f, 0.f);
            if (L < nlines) {
                const int64_t row = L / A.C;
                const int c = (int)(L % A.C);
                const int z = (int)(row / A.nyi), yy = (int)(row % A.nyi);
                const float ap = A.apz[z] * A.apy[yy] * A.apx[i];
                v = cscale(cmul(A.x[row * nx + i], coil_map(A, c)[row * nx + i]), ap);
            }
            bufa[(i + A.in_off) * kLinePad + l] = v;
        }
        for (int e = tid; e < kLines * (n - nx); e += blockDim.x) {
            const int l = e % kLines, kk = e / kLines;
            const int k = (kk < A.in_off) ? kk : kk + nx;
            bufa[k * kLinePad + l] = make_float2(0.f, 0.f);
        }
    } else {
        const int64_t iblocks = (A.inner + kLines - 1) / kLines;
        o0 = blockIdx.x / iblocks;
        i0 = (blockIdx.x % iblocks) * kLines;
        __syncthreads();
        if (MODE == PLAIN) {
            // loads are issued in batches of 8 per thread before the shared-memory stores, so
            // every thread keeps 8 independent 8-byte loads in flight
            constexpr int BATCH = 8;
            constexpr int KSTEP = kPassThreads / kLines;
            const int l = tid % kLines;
            const int64_t i = i0 + l;
            const bool iv = i < A.inner;
            for (int kb = tid / kLines; kb < n; kb += BATCH * KSTEP) {
                float2 reg[BATCH];
#pragma unroll
                for (int q = 0; q < BATCH; ++q) {
                    const int k = kb + q * KSTEP;
                    const int kk = k - A.in_off;
                    reg[q] = make_float2(0.f, 0.f);
                    if (k < n && iv && kk >= 0 && kk < A.n_in) reg[q] = A.in[(o0 * A.n_in + kk) * A.inner + i];
                }
#pragma unroll
                for (int q = 0; q < BATCH; ++q) {
                    const int k = kb + q * KSTEP;
                    if (k < n) bufa[k * kLinePad + l] = reg[q];
                }
            }
        } else
        for (int e = tid; e < kLines * n; e += blockDim.x) {
            const int l = e % kLines, k = e / kLines;
            const int64_t i = i0 + l;
            float2 v = make_float2(0.f, 0.f);
            if (i < A.inner) {
                if (MODE == SCATTER_Y) {
                    const int64_t px = i / A.C;
                    const int c = (int)(i % A.C);
                    const int32_t f = A.idxmap[(int64_t)k * A.nxi + px];
                    if (f >= 0) {
                        v = A.yk[(int64_t)c * A.N + f];
                        if (cart_neg(k, (int)px, n, A.nxi)) v = make_float2(-v.x, -v.y);
                    }
                } else {
                    const int kk = k - A.in_off;
                    if (kk >= 0 && kk < A.n_in) v = A.in[(o0 * A.n_in + kk) * A.inner + i];
                }
            }
            bufa[k * kLinePad + l] = v;
        }
    }
    __syncthreads();
    float2* res = fft_lines(bufa, bufb, stw, n, srad, A.nrad, A.sign);
    float2* other = (res == bufa) ? bufb : bufa;

    if (MODE == MASK_Y) {
        // U^H U (minus data) between the forward and the inverse transform
        for (int e = tid; e < kLines * n; e += blockDim.x) {
            const int l = e % kLines, k = e / kLines;
            const int64_t i = i0 + l;
            float2 v = make_float2(0.f, 0.f);
            if (i < A.inner) {
                const int64_t px = i / A.C;
                const int c = (int)(i % A.C);
                const int32_t f = A.idxmap[(int64_t)k * A.nxi + px];
                if (f >= 0) {
                    v = res[k * kLinePad + l];
                    if (A.residual) {
                        float2 yv = A.yk[(int64_t)c * A.N + f];
                        if (cart_neg(k, (int)px, n, A.nxi)) yv = make_float2(-yv.x, -yv.y);
                        v = csub(v, yv);
                    }
                }
            }
            res[k * kLinePad + l] = v;
        }
        __syncthreads();
        res = fft_lines(res, other, stw, n, srad, A.nrad, -A.sign);
    }

    // ---------------------------------- store ----------------------------------
    if (MODE == EXPAND_X) {
        const int64_t nlines = A.rows * A.C;
        for (int e = tid; e < kLines * n; e += blockDim.x) {
            const int l = e % kLines, k = e / kLines;
            const int64_t L = i0 + l;
            if (L < nlines) {
                const int64_t row = L / A.C;
                const int c = (int)(L % A.C);
                A.out[(row * n + k) * A.C + c] = res[k * kLinePad + l];
            }
        }
    } else if (MODE == GATHER_Y) {
        for (int e = tid; e < kLines * n; e += blockDim.x) {
            const int l = e % kLines, k = e / kLines;
            const int64_t i = i0 + l;
            if (i < A.inner) {
                const int64_t px = i / A.C;
                const int c = (int)(i % A.C);
                const int32_t f = A.idxmap[(int64_t)k * A.nxi + px];
                if (f >= 0) {
                    float2 v = res[k * kLinePad + l];
                    if (cart_neg(k, (int)px, n, A.nxi)) v = make_float2(-v.x, -v.y);
                    A.yko[(int64_t)c * A.N + f] = v;
                }
            }
        }
    } else {
        for (int e = tid; e < kLines * A.n_out; e += blockDim.x) {
            const int l = e % kLines, kk = e / kLines;
            const int64_t i = i0 + l;
            if (i < A.inner) A.out[(o0 * A.n_out + kk) * A.inner + i] = res[(kk + A.out_off) * kLinePad + l];
        }
    }
}

static size_t pass_smem(int n) { return sizeof(float2) * (size_t)(2 * n * kLinePad + n); }

// dynamic shared-memory limits of every pass kernel (set once per device at plan creation,
// never inside a stream capture)
cs_status fft_init_attrs() {
    const int sm = (int)pass_smem(kMaxFft);
    CS_TRY_CUDA(cudaFuncSetAttribute(fft_pass_kernel<EXPAND_X>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    CS_TRY_CUDA(cudaFuncSetAttribute(fft_pass_kernel<PLAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    CS_TRY_CUDA(cudaFuncSetAttribute(fft_pass_kernel<GATHER_Y>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    CS_TRY_CUDA(cudaFuncSetAttribute(fft_pass_kernel<SCATTER_Y>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    CS_TRY_CUDA(cudaFuncSetAttribute(fft_pass_kernel<MASK_Y>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    CS_TRY_CUDA(cudaFuncSetAttribute(fft_pass_kernel<REDUCE_X>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    return CS_OK;
}

template <int MODE>
static cs_status launch_pass(const PassArgs& A, cudaStream_t st) {
    const size_t sm = pass_smem(A.n);
    int64_t blocks;
    if (MODE == EXPAND_X) blocks = (A.rows * A.C + kLines - 1) / kLines;
    else if (MODE == REDUCE_X) blocks = (A.rows + A.rows_per_cta - 1) / A.rows_per_cta;
    else blocks = A.outer * ((A.inner + kLines - 1) / kLines);
    if (blocks == 0) return CS_OK;
    CS_REQUIRE(blocks < (int64_t)1 << 31, CS_ERR_UNSUPPORTED_SIZE, "pass grid too large");
    const int stage = (MODE == EXPAND_X) ? ST_EXPAND : (MODE == REDUCE_X ? ST_REDUCE : ST_FFT_PLAIN);
    prof_begin(stage, st);
    fft_pass_kernel<MODE><<<(unsigned)blocks, kPassThreads, sm, st>>>(A);
    CS_LAUNCH_CHECK();
    prof_end(stage, st);
    return CS_OK;
}

static void fill_fft(PassArgs& A, const FftLen& f, int sign) {
    A.n = f.n;
    A.nrad = f.nrad;
    for (int i = 0; i < kMaxRadices; ++i) A.rad[i] = f.rad[i];
    A.tw = f.tw;
    A.sign = sign;
}

static void fill_maps(PassArgs& A, const cs_plan* p, const float2* maps_v, int V, const float2* maps_s, int S) {
    A.maps_v = maps_v;
    A.maps_s = maps_s;
    A.V = V;
    A.C = V + S;
    A.D = p->D;
    A.apz = p->apod[0];
    A.apy = p->apod[1];
    A.apx = p->apod[2];
    A.nyi = p->img[1];
    A.nxi = p->img[2];
    A.rows = (int64_t)p->img[0] * p->img[1];
}

// x (.) maps (.) apod, zero-padded rows, FFT along x -> bufA [rows][Gx][C]
static cs_status pass_expand(const cs_plan* p, const float2* x, const float2* maps_v, int V,
                             const float2* maps_s, int S, cudaStream_t st) {
    PassArgs A = {};
    fill_fft(A, p->fft[2], -1);
    fill_maps(A, p, maps_v, V, maps_s, S);
    A.in_off = p->off[2];
    A.x = x;
    A.out = p->bufA;
    return launch_pass<EXPAND_X>(A, st);
}

static cs_status pass_reduce(const cs_plan* p, const float2* maps_v, int V, const float2* maps_s, int S,
                             float2* x, int accumulate, const float2* addv, float lambda, cudaStream_t st) {
    PassArgs A = {};
    fill_fft(A, p->fft[2], +1);
    fill_maps(A, p, maps_v, V, maps_s, S);
    A.out_off = p->off[2];
    A.in = p->bufA;
    A.xo = x;
    A.accumulate = accumulate;
    A.addv = addv;
    A.lambda = lambda;
    const int C = V + S;
    A.rows_per_cta = (C >= kLines || C == 0) ? 1 : kLines / C;   // C == 0: only lambda v / accumulate
    A.rows_per_cta = std::max(1, std::min(A.rows_per_cta, 4 * kPassThreads / p->img[2]));
    return launch_pass<REDUCE_X>(A, st);
}

// strided-axis pass for 3D plans: axis 0 (z) or 1 (y); coil-interleaved buffers
static cs_status pass_plain(const cs_plan* p, int axis, int sign, const float2* in, float2* out, int C,
                            cudaStream_t st) {
    PassArgs A = {};
    fill_fft(A, p->fft[axis], sign);
    const int Gx = p->grid[2], Gy = p->grid[1];
    if (axis == 1) {
        A.outer = (p->ndim == 3) ? p->img[0] : 1;
        A.inner = (int64_t)Gx * C;
    } else {
        A.outer = 1;
        A.inner = (int64_t)Gy * Gx * C;
    }
    if (sign < 0) {  // forward: pad img -> grid
        A.n_in = p->img[axis];
        A.in_off = p->off[axis];
        A.n_out = p->grid[axis];
        A.out_off = 0;
    } else {  // adjoint: crop grid -> img
        A.n_in = p->grid[axis];
        A.in_off = 0;
        A.n_out = p->img[axis];
        A.out_off = p->off[axis];
    }
    A.in = in;
    A.out = out;
    return launch_pass<PLAIN>(A, st);
}

static cs_status pass_cart_y(const cs_plan* p, int mode, int C, const float2* yk, float2* yko, int residual,
                             cudaStream_t st) {
    PassArgs A = {};
    const int sign = (mode == SCATTER_Y) ? +1 : -1;
    fill_fft(A, p->fft[1], sign);
    A.C = C;
    A.nxi = p->img[2];
    A.outer = 1;
    A.inner = (int64_t)p->img[2] * C;
    A.n_in = p->img[1];
    A.in_off = 0;
    A.n_out = p->img[1];
    A.out_off = 0;
    A.in = p->bufA;
    A.out = p->bufA;
    A.idxmap = p->idxmap;
    A.yk = yk;
    A.yko = yko;
    A.N = p->N;
    A.residual = residual;
    switch (mode) {
        case GATHER_Y: return launch_pass<GATHER_Y>(A, st);
        case SCATTER_Y: return launch_pass<SCATTER_Y>(A, st);
        default: return launch_pass<MASK_Y>(A, st);
    }
}

// ------------------------------------------------------------------------------------------
// Public to ops.cu

// Forward chain up to the sampling step: Cartesian leaves the x-transformed rows in bufA; the
// non-Cartesian chain leaves the oversampled k-space grid [G][C] in the grid buffer.
cs_status fft_to_grid(const cs_plan* p, const float2* x, const float2* maps_v, int V,
                      const float2* maps_s, int S, cudaStream_t st) {
    const int C = V + S;
    CS_PROPAGATE(pass_expand(p, x, maps_v, V, maps_s, S, st));
    if (p->kind == CS_CARTESIAN) return CS_OK;
    if (p->ndim == 3) {
        CS_PROPAGATE(pass_plain(p, 1, -1, p->bufA, p->bufB, C, st));
        CS_PROPAGATE(pass_plain(p, 0, -1, p->bufB, p->bufA, C, st));
        return CS_OK;
    }
    return pass_plain(p, 1, -1, p->bufA, p->bufB, C, st);   // 2D: the grid lands in bufB
}

// Cartesian sampling along y: mode 0 gather (y = U F .), 1 scatter (U^H y then inverse FFT),
// 2 normal (U^H U), 3 residual (U^H (U . - y)).
cs_status fft_cart_sample(const cs_plan* p, int mode, int ncoils, const float2* yk, float2* yko, cudaStream_t st) {
    switch (mode) {
        case 0: return pass_cart_y(p, GATHER_Y, ncoils, nullptr, yko, 0, st);
        case 1: return pass_cart_y(p, SCATTER_Y, ncoils, yk, nullptr, 0, st);
        case 2: return pass_cart_y(p, MASK_Y, ncoils, nullptr, nullptr, 0, st);
        default: return pass_cart_y(p, MASK_Y, ncoils, yk, nullptr, 1, st);
    }
}

// Adjoint chain from the sampling step: (non-Cartesian: inverse z, y passes from the grid
// buffer) then the coil-combining x pass: x (+)= sum_c conj(c_c) . F^H(...) (+ lambda addv).
cs_status fft_to_image(const cs_plan* p, const float2* maps_v, int V, const float2* maps_s, int S,
                       float2* x, int accumulate, const float2* addv, float lambda, cudaStream_t st) {
    const int C = V + S;
    if (p->kind != CS_CARTESIAN && C > 0) {
        if (p->ndim == 3) {
            CS_PROPAGATE(pass_plain(p, 0, +1, p->bufA, p->bufB, C, st));
            CS_PROPAGATE(pass_plain(p, 1, +1, p->bufB, p->bufA, C, st));
        } else {
            CS_PROPAGATE(pass_plain(p, 1, +1, p->bufB, p->bufA, C, st));
        }
    }
    return pass_reduce(p, maps_v, V, maps_s, S, x, accumulate, addv, lambda, st);
}

}  // namespace cs
