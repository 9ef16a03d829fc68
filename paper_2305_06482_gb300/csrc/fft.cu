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
//   (strided)  middle passes along z / y: tensor-copy kernel below, zero-pad on input / crop on
//              output
//   GATHER_Y   FFT along y, keep the sampled entries U (Cartesian forward)
//   SCATTER_Y  U^H (zero-fill) then inverse FFT along y (Cartesian adjoint)
//   MASK_Y     FFT along y, U^H U (optionally minus the data: residual), inverse FFT
//   REDUCE_X   inverse FFT along x, crop, apod, sum_c conj(c_c) (.) (+ lambda v)  (last adjoint)
#include <cstdio>
#include <cmath>

#include <cuda.h>
#include <cudaTypedefs.h>

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
    int Ns = 1;
    for (int s = 0; s < f.nrad; ++s) {
        const int r = f.rad[s];
        f.st[s] = make_int4(r, Ns, (int)((uint32_t)(0x100000000ull / (unsigned long long)Ns) + 1u), n / (Ns * r));
        Ns *= r;
    }
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
// Small DFTs, the direction a template parameter (SIGN = -1 forward, +1 inverse).  Radices 2, 4
// and 8 are split-radix butterflies; the odd radices use the symmetric form
//   X_m = x_0 + sum_q cos(2 pi q m / R) (x_q + x_{R-q}) + SIGN i sum_q sin(2 pi q m / R) (x_q - x_{R-q})
// (q, m = 1 .. (R-1)/2, X_{R-m} with the opposite sign of the second sum), whose cosines and
// sines are compile-time constants.

// cos and sin of 2 pi k / R evaluated at compile time in double by Taylor series after reducing
// the angle to [-pi, pi] (30 terms: truncation error far below double rounding there)
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double ct_reduce(double x) {
    while (x > kTwoPi / 2) x -= kTwoPi;
    while (x < -kTwoPi / 2) x += kTwoPi;
    return x;
}
constexpr double ct_cos(double x) {
    x = ct_reduce(x);
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 30; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}
constexpr double ct_sin(double x) {
    x = ct_reduce(x);
    double term = x, sum = x;
    for (int k = 1; k < 30; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}

template <int R>
struct Roots {
    float c[R], s[R];
    constexpr Roots() : c(), s() {
        for (int k = 0; k < R; ++k) {
            c[k] = (float)ct_cos(kTwoPi * k / R);
            s[k] = (float)ct_sin(kTwoPi * k / R);
        }
    }
};

// paired single-precision add / subtract / fused multiply-add (one instruction for both halves,
// each half rounded like its scalar counterpart)
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 fma2s(float s, float2 a, float2 b) { return __ffma2_rn(make_float2(s, s), a, b); }

template <int R, int SIGN>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
    static_assert(R % 2 == 1, "odd radix");
    constexpr int H = (R - 1) / 2;
    constexpr Roots<R> rt{};
    float2 t[H], d[H];
#pragma unroll
    for (int q = 1; q <= H; ++q) {
        t[q - 1] = add2(v[q], v[R - q]);
        d[q - 1] = sub2(v[q], v[R - q]);
    }
    float2 o[R];
    o[0] = v[0];
#pragma unroll
    for (int q = 0; q < H; ++q) o[0] = add2(o[0], t[q]);
#pragma unroll
    for (int m = 1; m <= H; ++m) {
        float2 a = v[0], b = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 1; q <= H; ++q) {
            a = fma2s(rt.c[(q * m) % R], t[q - 1], a);
            b = fma2s(rt.s[(q * m) % R], d[q - 1], b);
        }
        // a + SIGN i b and a - SIGN i b
        o[m] = make_float2(a.x - SIGN * b.y, a.y + SIGN * b.x);
        o[R - m] = make_float2(a.x + SIGN * b.y, a.y - SIGN * b.x);
    }
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = o[m];
}

template <int SIGN>
__device__ __forceinline__ float2 rot_i(float2 a) {   // multiply by SIGN i
    return SIGN < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

template <>
__device__ __forceinline__ void dft<2, -1>(float2 (&v)[2]) {
    const float2 a = v[0], b = v[1];
    v[0] = add2(a, b);
    v[1] = sub2(a, b);
}
template <>
__device__ __forceinline__ void dft<2, 1>(float2 (&v)[2]) {
    const float2 a = v[0], b = v[1];
    v[0] = add2(a, b);
    v[1] = sub2(a, b);
}

template <int SIGN>
__device__ __forceinline__ void dft4(float2 (&v)[4]) {
    const float2 s02 = add2(v[0], v[2]), d02 = sub2(v[0], v[2]);
    const float2 s13 = add2(v[1], v[3]), d13 = rot_i<SIGN>(sub2(v[1], v[3]));
    v[0] = add2(s02, s13);
    v[2] = sub2(s02, s13);
    v[1] = add2(d02, d13);
    v[3] = sub2(d02, d13);
}
template <>
__device__ __forceinline__ void dft<4, -1>(float2 (&v)[4]) { dft4<-1>(v); }
template <>
__device__ __forceinline__ void dft<4, 1>(float2 (&v)[4]) { dft4<1>(v); }

template <int SIGN>
__device__ __forceinline__ void dft8(float2 (&v)[8]) {
    const float h = 0.70710678118654752440f;
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    dft4<SIGN>(e);
    dft4<SIGN>(o);
    // o[m] times exp(SIGN 2 pi i m / 8), m = 1, 2, 3
    const float2 t1 = make_float2(h * (o[1].x - SIGN * o[1].y), h * (o[1].y + SIGN * o[1].x));
    const float2 t2 = rot_i<SIGN>(o[2]);
    const float2 t3 = make_float2(h * (-o[3].x - SIGN * o[3].y), h * (-o[3].y + SIGN * o[3].x));
    v[0] = add2(e[0], o[0]);
    v[4] = sub2(e[0], o[0]);
    v[1] = add2(e[1], t1);
    v[5] = sub2(e[1], t1);
    v[2] = add2(e[2], t2);
    v[6] = sub2(e[2], t2);
    v[3] = add2(e[3], t3);
    v[7] = sub2(e[3], t3);
}
template <>
__device__ __forceinline__ void dft<8, -1>(float2 (&v)[8]) { dft8<-1>(v); }
template <>
__device__ __forceinline__ void dft<8, 1>(float2 (&v)[8]) { dft8<1>(v); }

// q = j / Ns for 0 <= j < 2^16 and 2 <= Ns < 2^16 via a multiply-shift with mag = floor(2^32 / Ns) + 1
// (the error of j * mag / 2^32 against j / Ns stays below 1 / Ns there); Ns = 1 is passed through
__device__ __forceinline__ int divmagic(int j, int Ns, uint32_t mag) {
    return Ns == 1 ? j : (int)__umulhi((uint32_t)j, mag);
}

constexpr int kJ = kPassThreads / kLines;   // threads per line

// One radix-R Stockham stage over the kLines lines of a CTA; thread (l, jt) takes butterflies
// j = jt, jt + kJ, ... of line l.  tw holds exp(-2 pi i k / n); the inverse conjugates it.
template <int R, int SIGN, int PITCH>
__device__ __forceinline__ void stockham_stage(const float2* __restrict__ a, float2* __restrict__ b,
                                               const float2* __restrict__ tw, int n, int Ns, uint32_t mag,
                                               int tstride, int l, int jt) {
    const int nb = n / R;
    for (int j = jt; j < nb; j += kJ) {
        const int jq = divmagic(j, Ns, mag);
        const int k = j - jq * Ns;
        float2 v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = a[(j + q * nb) * PITCH + l];
        if (Ns > 1) {
            const int step = k * tstride;
#pragma unroll
            for (int q = 1; q < R; ++q) {
                float2 w = tw[q * step];
                if (SIGN > 0) w.y = -w.y;
                v[q] = cmul(v[q], w);
            }
        }
        dft<R, SIGN>(v);
        const int base = jq * Ns * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) b[(base + q * Ns) * PITCH + l] = v[q];
    }
}

// Transform the kLines lines in shared memory (element k of line l at k * PITCH + l); returns the
// buffer holding the result.
template <int SIGN, int PITCH = kLinePad>
__device__ float2* fft_lines(float2* a, float2* b, const float2* tw, int n, const int4* stages, int nrad, int l,
                             int jt) {
    for (int s = 0; s < nrad; ++s) {
        const int4 g = stages[s];
        const int r = g.x, Ns = g.y, tstride = g.w;
        const uint32_t mag = (uint32_t)g.z;
        switch (r) {
            case 2: stockham_stage<2, SIGN, PITCH>(a, b, tw, n, Ns, mag, tstride, l, jt); break;
            case 3: stockham_stage<3, SIGN, PITCH>(a, b, tw, n, Ns, mag, tstride, l, jt); break;
            case 4: stockham_stage<4, SIGN, PITCH>(a, b, tw, n, Ns, mag, tstride, l, jt); break;
            case 5: stockham_stage<5, SIGN, PITCH>(a, b, tw, n, Ns, mag, tstride, l, jt); break;
            case 7: stockham_stage<7, SIGN, PITCH>(a, b, tw, n, Ns, mag, tstride, l, jt); break;
            case 8: stockham_stage<8, SIGN, PITCH>(a, b, tw, n, Ns, mag, tstride, l, jt); break;
            case 11: stockham_stage<11, SIGN, PITCH>(a, b, tw, n, Ns, mag, tstride, l, jt); break;
            default: break;
        }
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
    }
    return a;
}

// ------------------------------------------------------------------------------------------
// Pass kernels.  Coil stacks are stored coil-interleaved: element (..., k, ..., c) of an
// intermediate or grid buffer sits at ((... * n + k) * inner_rest + ...) * C + c, so a line is
// (position along the other axes, coil) and kLines consecutive lines are contiguous in memory
// for every axis, including x.  Thread t of a CTA owns line l = t mod kLines for the loads, the
// butterflies and the stores (element rows jt = t / kLines, jt + kJ, ...), so its addresses are
// one base plus a stride; per-line quantities of the x passes are computed once per CTA.
// (the strided middle passes run in fft_plain_tma_kernel below)
enum PassMode { EXPAND_X = 0, GATHER_Y = 2, SCATTER_Y = 3, MASK_Y = 4, REDUCE_X = 5 };

struct PassArgs {
    int n, nrad;
    int4 st[kMaxRadices];
    const float2* tw;
    int sign;
    int64_t outer;   // Y modes: outer index count
    int64_t inner;   // Y modes: stride of the FFT axis in elements (includes the coil count)
    int n_in, in_off, n_out, out_off;
    const float2* in;
    float2* out;
    // X modes: image rows and coils
    int64_t rows;    // nz * ny image rows
    int C;           // coils (interleave stride)
    int rows_per_cta;
    int cw;          // REDUCE_X: coils per chunk (rows_per_cta * cw <= kLines lines)
    uint32_t nx_mag; // floor(2^32 / nxi) + 1
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

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// asynchronous global -> shared copies of 8 and 4 bytes (every copy of a thread in flight at once;
// cp.async.wait_all makes them visible to the issuing thread, a barrier to the others)
__device__ __forceinline__ void cp8(float2* dst, const float2* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp4(float* dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// i / nxi for 0 <= i < 2^16 (the x-pass element loops stay below 16 * 512)
__device__ __forceinline__ int div_nx(const PassArgs& A, int i) { return (int)__umulhi((uint32_t)i, A.nx_mag); }

template <int MODE, int SIGN>
__global__ void __launch_bounds__(kPassThreads, 3) fft_pass_kernel(PassArgs A) {
    extern __shared__ float2 smem[];
    const int n = A.n;
    float2* bufa = smem;
    float2* bufb = smem + n * kLinePad;
    float2* stw = smem + 2 * n * kLinePad;
    __shared__ int4 sst[kMaxRadices];
    __shared__ int64_t sbase[kLines];          // x passes: per-line element offset
    __shared__ int srow[kLines];               // x passes: image row of the line (-1: none)
    __shared__ const float2* sxp[kLines];      // x passes: row pointers of x / the line's map
    __shared__ const float2* smp[kLines];
    __shared__ float sapzy[kLines];
    __shared__ float sapx[MODE == EXPAND_X ? 512 : 1];   // nx <= 512
    const int tid = threadIdx.x;
    const int l = tid % kLines, jt = tid / kLines;
    if (tid < kMaxRadices) sst[tid] = A.st[tid];
    for (int e = tid; e < n; e += blockDim.x) stw[e] = A.tw[e];

    if (MODE == REDUCE_X) {
        // ---- rows_per_cta image rows; inverse FFT of every coil's line, crop, conj(map),
        //      apodisation and the sum over coils (deterministic order) ----
        constexpr int MAXE = 4;     // rows_per_cta * nx <= 4 * kPassThreads (set by pass_reduce)
        float2 acc[MAXE];
        int orow[MAXE], oi[MAXE];
        const int nx = A.nxi;
        const int R = A.rows_per_cta;
        const int r0 = blockIdx.x * R;
#pragma unroll
        for (int e = 0; e < MAXE; ++e) {
            acc[e] = make_float2(0.f, 0.f);
            const int idx = tid + e * kPassThreads;
            const int rr = div_nx(A, idx);
            oi[e] = idx - rr * nx;
            orow[e] = (idx < R * nx && r0 + rr < A.rows) ? r0 + rr : -1;
            oi[e] = (orow[e] >= 0) ? oi[e] : 0;
        }
        const int cwmax = A.cw;
        for (int c0 = 0; c0 < A.C; c0 += cwmax) {
            const int cw = min(cwmax, A.C - c0);
            __syncthreads();
            if (tid < kLines) {
                const int row = r0 + tid / cw, c = c0 + tid % cw;
                const bool ok = tid < R * cw && row < A.rows;
                srow[tid] = ok ? row : -1;
                sbase[tid] = ok ? (int64_t)row * n * A.C + c : 0;
                smp[tid] = ok ? coil_map(A, c) + (int64_t)row * nx : nullptr;
            }
            __syncthreads();
            {
                const bool ok = srow[l] >= 0;
                const float2* p = A.in + sbase[l] + (int64_t)jt * A.C;
                const int64_t step = (int64_t)kJ * A.C;
                const int64_t inlim = A.rows * n * A.C;
                (void)inlim;
                for (int k = jt; k < n; k += kJ, p += step) {
                    if (ok && CS_INB(sbase[l] + (int64_t)k * A.C, inlim)) cp8(&bufa[k * kLinePad + l], p);
                    else bufa[k * kLinePad + l] = make_float2(0.f, 0.f);
                }
                cp_wait_all();
            }
            __syncthreads();
            float2* res = fft_lines<SIGN>(bufa, bufb, stw, n, sst, A.nrad, l, jt);
            // the coil maps of the chunk's lines, staged in the buffer the FFT left free:
            // mp[line * nx + i] (line = rr * cw + q)
            float2* mp = (res == bufa) ? bufb : bufa;
            for (int e = tid; e < R * cw * nx; e += kPassThreads) {
                const int ln = div_nx(A, e), i = e - ln * nx;
                if (smp[ln] && CS_INB((int64_t)srow[ln] * nx + i, A.D)) cp8(&mp[e], smp[ln] + i);
            }
            cp_wait_all();
            __syncthreads();
#pragma unroll
            for (int e = 0; e < MAXE; ++e) {
                if (orow[e] >= 0) {
                    const int idx = tid + e * kPassThreads;
                    const int rr = div_nx(A, idx);
                    const float2* rp = res + (oi[e] + A.out_off) * kLinePad + rr * cw;
                    const float2* mq = mp + rr * cw * nx + oi[e];
                    for (int q = 0; q < cw; ++q) acc[e] = cadd(acc[e], cmulc(mq[q * nx], rp[q]));
                }
            }
        }
#pragma unroll
        for (int e = 0; e < MAXE; ++e) {
            if (orow[e] >= 0) {
                const int row = orow[e], i = oi[e];
                const int z = row / A.nyi, yy = row - (row / A.nyi) * A.nyi;
                const float ap = A.apz[z] * A.apy[yy] * A.apx[i];
                float2 r = cscale(acc[e], ap);
                const int64_t g = (int64_t)row * nx + i;
                if (CS_INB(g, A.D)) {
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
    int px = 0, cc = 0;
    bool iv = true;
    if (MODE == EXPAND_X) {
        i0 = (int64_t)blockIdx.x * kLines;  // first line = row * C + c
        const int nx = A.nxi;
        if (tid < kLines) {
            const int L = (int)i0 + tid;               // rows * C < 2^31 (checked at launch)
            const bool ok = L < (int)(A.rows * A.C);
            const int row = ok ? L / A.C : 0;
            const int c = ok ? L - row * A.C : 0;
            const int z = row / A.nyi, yy = row - z * A.nyi;
            srow[tid] = ok ? row : -1;
            sapzy[tid] = A.apz[z] * A.apy[yy];
            sbase[tid] = (int64_t)row * n * A.C + c;
            sxp[tid] = ok ? A.x + (int64_t)row * nx : nullptr;
            smp[tid] = ok ? coil_map(A, c) + (int64_t)row * nx : nullptr;
        }
        // zero padding rows outside [in_off, in_off + nx)
        for (int kk = jt; kk < n - nx; kk += kJ) {
            const int k = (kk < A.in_off) ? kk : kk + nx;
            bufa[k * kLinePad + l] = make_float2(0.f, 0.f);
        }
        __syncthreads();
        // x (per line) -> bufa rows in_off.., maps -> bufb, apodisation along x -> sapx, all
        // asynchronous; then each thread forms the products of the elements it copied
        for (int i = tid; i < nx; i += kPassThreads) cp4(&sapx[i], A.apx + i);
        for (int e = tid; e < kLines * nx; e += kPassThreads) {
            const int le = div_nx(A, e), i = e - le * nx;
            float2* da = &bufa[(i + A.in_off) * kLinePad + le];
            if (sxp[le] && CS_INB((int64_t)srow[le] * nx + i, A.D)) {
                cp8(da, sxp[le] + i);
                cp8(&bufb[i * kLinePad + le], smp[le] + i);
            } else {
                *da = make_float2(0.f, 0.f);
            }
        }
        cp_wait_all();
        __syncthreads();
        for (int e = tid; e < kLines * nx; e += kPassThreads) {
            const int le = div_nx(A, e), i = e - le * nx;
            if (sxp[le]) {
                float2* d = &bufa[(i + A.in_off) * kLinePad + le];
                *d = cscale(cmul(*d, bufb[i * kLinePad + le]), sapzy[le] * sapx[i]);
            }
        }
    } else {
        o0 = blockIdx.y;
        i0 = (int64_t)blockIdx.x * kLines;
        const int64_t i = i0 + l;
        iv = i < A.inner;
        px = (int)(i / A.C);
        cc = (int)(i - (int64_t)px * A.C);
        constexpr int LB = 8;   // loads in flight per thread
        if (MODE == SCATTER_Y) {
            for (int k0 = jt; k0 < n; k0 += kJ * LB) {
                int32_t f[LB];
                float2 t[LB];
#pragma unroll
                for (int b = 0; b < LB; ++b) {
                    const int k = k0 + b * kJ;
                    f[b] = (iv && k < n && CS_INB((int64_t)k * A.nxi + px, A.D)) ? A.idxmap[(int64_t)k * A.nxi + px] : -1;
                }
#pragma unroll
                for (int b = 0; b < LB; ++b)
                    t[b] = (f[b] >= 0 && CS_INB((int64_t)cc * A.N + f[b], (int64_t)A.C * A.N)) ? A.yk[(int64_t)cc * A.N + f[b]]
                                                                                             : make_float2(0.f, 0.f);
#pragma unroll
                for (int b = 0; b < LB; ++b) {
                    const int k = k0 + b * kJ;
                    if (k < n) bufa[k * kLinePad + l] = cart_neg(k, px, n, A.nxi) ? make_float2(-t[b].x, -t[b].y) : t[b];
                }
            }
        } else {
            for (int kk = jt; kk < n - A.n_in; kk += kJ) {
                const int k = (kk < A.in_off) ? kk : kk + A.n_in;
                bufa[k * kLinePad + l] = make_float2(0.f, 0.f);
            }
            const float2* p = A.in + o0 * A.n_in * A.inner + i;
            for (int k0 = jt; k0 < A.n_in; k0 += kJ * LB) {
                float2 t[LB];
                const float2* pk = p + (int64_t)k0 * A.inner;
#pragma unroll
                for (int b = 0; b < LB; ++b) {
                    const int kk = k0 + b * kJ;
                    t[b] = (iv && kk < A.n_in && CS_INB((o0 * A.n_in + kk) * A.inner + i, A.outer * A.n_in * A.inner))
                               ? pk[(int64_t)b * kJ * A.inner]
                               : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int b = 0; b < LB; ++b) {
                    const int kk = k0 + b * kJ;
                    if (kk < A.n_in) bufa[(kk + A.in_off) * kLinePad + l] = t[b];
                }
            }
        }
    }
    __syncthreads();
    float2* res = fft_lines<SIGN>(bufa, bufb, stw, n, sst, A.nrad, l, jt);
    float2* other = (res == bufa) ? bufb : bufa;

    if (MODE == MASK_Y) {
        // U^H U (minus data) between the forward and the inverse transform
        for (int k = jt; k < n; k += kJ) {
            float2 v = make_float2(0.f, 0.f);
            if (iv && CS_INB((int64_t)k * A.nxi + px, A.D)) {
                const int32_t f = A.idxmap[(int64_t)k * A.nxi + px];
                if (f >= 0) {
                    v = res[k * kLinePad + l];
                    if (A.residual && CS_INB((int64_t)cc * A.N + f, (int64_t)A.C * A.N)) {
                        float2 yv = A.yk[(int64_t)cc * A.N + f];
                        if (cart_neg(k, px, n, A.nxi)) yv = make_float2(-yv.x, -yv.y);
                        v = csub(v, yv);
                    }
                }
            }
            res[k * kLinePad + l] = v;
        }
        __syncthreads();
        res = fft_lines<-SIGN>(res, other, stw, n, sst, A.nrad, l, jt);
    }

    // ---------------------------------- store ----------------------------------
    if (MODE == EXPAND_X) {
        if (srow[l] >= 0) {
            float2* p = A.out + sbase[l] + (int64_t)jt * A.C;
            const int64_t step = (int64_t)kJ * A.C;
            const int64_t outlim = A.rows * n * A.C;
            (void)outlim;
#pragma unroll 4
            for (int k = jt; k < n; k += kJ, p += step)
                if (CS_INB(sbase[l] + (int64_t)k * A.C, outlim)) *p = res[k * kLinePad + l];
        }
    } else if (MODE == GATHER_Y) {
        if (iv) {
            for (int k = jt; k < n; k += kJ) {
                const int32_t f = CS_INB((int64_t)k * A.nxi + px, A.D) ? A.idxmap[(int64_t)k * A.nxi + px] : -1;
                if (f >= 0 && CS_INB((int64_t)cc * A.N + f, (int64_t)A.C * A.N)) {
                    float2 v = res[k * kLinePad + l];
                    if (cart_neg(k, px, n, A.nxi)) v = make_float2(-v.x, -v.y);
                    A.yko[(int64_t)cc * A.N + f] = v;
                }
            }
        }
    } else if (iv) {
        float2* p = A.out + o0 * A.n_out * A.inner + i0 + l;
#pragma unroll 4
        for (int kk = jt; kk < A.n_out; kk += kJ)
            if (CS_INB((o0 * A.n_out + kk) * A.inner + i0 + l, A.outer * A.n_out * A.inner))
                p[(int64_t)kk * A.inner] = res[(kk + A.out_off) * kLinePad + l];
    }
}

static size_t pass_smem(int n) { return sizeof(float2) * (size_t)(2 * n * kLinePad + n); }

// dynamic shared-memory limits of every pass kernel (set once per device at plan creation,
// never inside a stream capture)
static cs_status tma_init_attrs();

cs_status fft_init_attrs() {
    CS_PROPAGATE(tma_init_attrs());
    const int sm = (int)pass_smem(kMaxFft);
    CS_TRY_CUDA(cudaFuncSetAttribute(fft_pass_kernel<EXPAND_X, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    CS_TRY_CUDA(cudaFuncSetAttribute(fft_pass_kernel<GATHER_Y, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    CS_TRY_CUDA(cudaFuncSetAttribute(fft_pass_kernel<SCATTER_Y, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    CS_TRY_CUDA(cudaFuncSetAttribute(fft_pass_kernel<MASK_Y, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    CS_TRY_CUDA(cudaFuncSetAttribute(fft_pass_kernel<REDUCE_X, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    return CS_OK;
}

template <int MODE, int SIGN>
static cs_status launch_pass(const PassArgs& A, cudaStream_t st) {
    const size_t sm = pass_smem(A.n);
    int64_t blocks, outer = 1;
    if (MODE == EXPAND_X) {
        CS_REQUIRE(A.rows * A.C < ((int64_t)1 << 31) - kLines, CS_ERR_UNSUPPORTED_SIZE, "too many x lines");
        blocks = (A.rows * A.C + kLines - 1) / kLines;
    }
    else if (MODE == REDUCE_X) blocks = (A.rows + A.rows_per_cta - 1) / A.rows_per_cta;
    else {
        blocks = (A.inner + kLines - 1) / kLines;
        outer = A.outer;
    }
    if (blocks * outer == 0) return CS_OK;
    CS_REQUIRE(blocks < (int64_t)1 << 31 && outer <= 65535, CS_ERR_UNSUPPORTED_SIZE, "pass grid too large");
    const int stage = (MODE == EXPAND_X) ? ST_EXPAND : (MODE == REDUCE_X ? ST_REDUCE : ST_FFT_PLAIN);
    prof_begin(stage, st);
    fft_pass_kernel<MODE, SIGN><<<dim3((unsigned)blocks, (unsigned)outer), kPassThreads, sm, st>>>(A);
    CS_LAUNCH_CHECK();
    prof_end(stage, st);
    return CS_OK;
}

static void fill_fft(PassArgs& A, const FftLen& f, int sign) {
    A.n = f.n;
    A.nrad = f.nrad;
    for (int i = 0; i < kMaxRadices; ++i) A.st[i] = f.st[i];
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
    A.nx_mag = (uint32_t)(0x100000000ull / (unsigned long long)p->img[2]) + 1u;
    A.rows = (int64_t)p->img[0] * p->img[1];
}

// ------------------------------------------------------------------------------------------
// Strided-axis pass with tensor-memory-access copies.  The coil-interleaved buffer is a 3D
// tensor [outer][rows][inner] of 8-byte elements; a CTA's tile is 16 consecutive lines (128 B of
// every row) by the n rows of the transform.  One thread issues the tensor loads of the whole
// tile (boxes of h_in rows; rows outside [0, n_in) after the shift by in_off read as zero, which
// is the zero padding of the forward transform), every thread waits on the mbarrier (bounded),
// the FFT runs in shared memory in the dense layout [k][16] (a half-warp touches one 128-byte
// row: no bank conflicts), and one thread stores the cropped rows [out_off, out_off + n_out)
// with tensor stores (the ragged last tile is clipped by the copy unit).
constexpr long long kTmaSpinLimit = 1ll << 24;
__device__ int g_fft_error = 0;

struct TmaPassArgs {
    int n, nrad;
    int4 st[kMaxRadices];
    const float2* tw;
    int64_t iblocks;        // tiles along the line index
    int in_off, h_in, nbox_in;
    int out_off, h_out, nbox_out;
};

template <int SIGN>
__global__ void __launch_bounds__(kPassThreads, 4)
    fft_plain_tma_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
                         const __grid_constant__ TmaPassArgs A) {
    extern __shared__ __align__(1024) float2 tsm[];
    const int n = A.n;
    float2* bufa = tsm;
    float2* bufb = tsm + n * kLines;
    float2* stw = tsm + 2 * n * kLines;
    __shared__ int4 sst[kMaxRadices];
    __shared__ __align__(8) uint64_t mbar;
    const int tid = threadIdx.x;
    const int l = tid % kLines, jt = tid / kLines;
    const int o0 = (int)blockIdx.y;
    const int i0 = (int)blockIdx.x * kLines;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar)), "r"(1u));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        const uint32_t bytes = (uint32_t)n * kLines * sizeof(float2);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&mbar)), "r"(bytes)
                     : "memory");
        for (int b = 0; b < A.nbox_in; ++b) {
            const int y = b * A.h_in - A.in_off;
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                ::"r"(smem_addr(bufa + (size_t)b * A.h_in * kLines)), "l"(&tin), "r"(i0), "r"(y), "r"(o0),
                  "r"(smem_addr(&mbar))
                : "memory");
        }
    }
    if (tid < kMaxRadices) sst[tid] = A.st[tid];
    for (int e = tid; e < n; e += blockDim.x) stw[e] = A.tw[e];
    // bounded wait for the tile (phase 0)
    int done = 0;
    long long spins = 0;
    while (!done) {
        asm volatile(
            "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\nselp.b32 %0, 1, 0, P1;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(&mbar)), "r"(0u)
            : "memory");
        if (!done && ++spins > kTmaSpinLimit) break;
    }
    if (__syncthreads_or(!done)) {
        // gave up: the flag makes the host report CS_ERR_TIMEOUT; this CTA's lines are not written,
        // so every output of the call (and of a solve that contains it) is invalid.  Before the CTA
        // leaves, wait once more (bounded) for the tile copy in flight into its shared memory.
        if (tid == 0) atomicExch(&g_fft_error, 1);
        for (long long k = 0; !done && k < kTmaSpinLimit; ++k)
            asm volatile(
                "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\nselp.b32 %0, 1, 0, P1;\n}\n"
                : "=r"(done)
                : "r"(smem_addr(&mbar)), "r"(0u)
                : "memory");
        return;
    }
    float2* res = fft_lines<SIGN, kLines>(bufa, bufb, stw, n, sst, A.nrad, l, jt);
    // make the generic-proxy shared-memory writes visible to the copy unit, then store
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
        for (int b = 0; b < A.nbox_out; ++b) {
            const int y = b * A.h_out;
            asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];"
                         ::"l"(&tout), "r"(i0), "r"(y), "r"(o0),
                           "r"(smem_addr(res + (size_t)(A.out_off + y) * kLines))
                         : "memory");
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
}

static size_t tma_pass_smem(int n) { return sizeof(float2) * (size_t)(2 * n * kLines + n); }

static cs_status tma_init_attrs() {
    const int sm = (int)tma_pass_smem(kMaxFft);
    CS_TRY_CUDA(cudaFuncSetAttribute(fft_plain_tma_kernel<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    CS_TRY_CUDA(cudaFuncSetAttribute(fft_plain_tma_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    return CS_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link)
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// smallest divisor h of n with h <= 256 and n / h boxes (the box height limit is 256 rows)
static int box_rows(int n) {
    for (int b = 1; b <= n; ++b)
        if (n % b == 0 && n / b <= 256) return n / b;
    return 1;
}

static cs_status encode_3d(CUtensorMap* m, const float2* base, int64_t inner, int rows, int64_t outer, int h) {
    auto fn = encode_fn();
    CS_REQUIRE(fn != nullptr, CS_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    CS_REQUIRE(inner % 2 == 0, CS_ERR_UNSUPPORTED_SIZE, "tensor copies need an even line count (got %lld)", (long long)inner);
    const cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)rows, (cuuint64_t)outer};
    const cuuint64_t strides[2] = {(cuuint64_t)inner * sizeof(float2), (cuuint64_t)inner * rows * sizeof(float2)};
    const cuuint32_t box[3] = {(cuuint32_t)kLines, (cuuint32_t)h, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, (void*)base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    CS_REQUIRE(r == CUDA_SUCCESS, CS_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return CS_OK;
}

// strided-axis pass for 3D plans (axis 0: z, 1: y) and the y pass of 2D plans; coil-interleaved
static cs_status pass_plain(const cs_plan* p, int axis, int sign, const float2* in, float2* out, int C,
                            cudaStream_t st) {
    const FftLen& f = p->fft[axis];
    TmaPassArgs A = {};
    A.n = f.n;
    A.nrad = f.nrad;
    for (int i = 0; i < kMaxRadices; ++i) A.st[i] = f.st[i];
    A.tw = f.tw;
    const int Gx = p->grid[2], Gy = p->grid[1];
    int64_t outer, inner;
    if (axis == 1) {
        outer = (p->ndim == 3) ? p->img[0] : 1;
        inner = (int64_t)Gx * C;
    } else {
        outer = 1;
        inner = (int64_t)Gy * Gx * C;
    }
    int n_in, n_out;
    if (sign < 0) {  // forward: pad img -> grid
        n_in = p->img[axis];
        A.in_off = p->off[axis];
        n_out = p->grid[axis];
        A.out_off = 0;
    } else {  // adjoint: crop grid -> img
        n_in = p->grid[axis];
        A.in_off = 0;
        n_out = p->img[axis];
        A.out_off = p->off[axis];
    }
    A.h_in = box_rows(A.n);
    A.nbox_in = A.n / A.h_in;
    A.h_out = box_rows(n_out);
    A.nbox_out = n_out / A.h_out;
    A.iblocks = (inner + kLines - 1) / kLines;
    if (outer * A.iblocks == 0) return CS_OK;
    CS_REQUIRE(A.iblocks < (int64_t)1 << 31 && outer <= 65535 && inner < (int64_t)1 << 31,
               CS_ERR_UNSUPPORTED_SIZE, "pass grid too large");
    const dim3 blocks((unsigned)A.iblocks, (unsigned)outer);
    // the copy unit clips every tensor copy to its tensor map; the maps must not describe more
    // than the plan buffers they address
    auto capacity = [&](const float2* b) -> int64_t {
        if (b == p->bufA) return (int64_t)p->max_coils * p->G;
        if (b == p->bufB) return (int64_t)p->max_coils * p->img[0] * p->grid[1] * p->grid[2];
        return -1;
    };
    const int64_t cin_ = capacity(in), cout_ = capacity(out);
    CS_REQUIRE((cin_ < 0 || inner * n_in * outer <= cin_) && (cout_ < 0 || inner * n_out * outer <= cout_), CS_ERR_BOUNDS,
               "a tensor-copy pass would address beyond its buffer");
    CUtensorMap tin, tout;
    CS_PROPAGATE(encode_3d(&tin, in, inner, n_in, outer, A.h_in));
    CS_PROPAGATE(encode_3d(&tout, out, inner, n_out, outer, A.h_out));
    prof_begin(ST_FFT_PLAIN, st);
    if (sign < 0)
        fft_plain_tma_kernel<-1><<<blocks, kPassThreads, tma_pass_smem(A.n), st>>>(tin, tout, A);
    else
        fft_plain_tma_kernel<1><<<blocks, kPassThreads, tma_pass_smem(A.n), st>>>(tin, tout, A);
    CS_LAUNCH_CHECK();
    prof_end(ST_FFT_PLAIN, st);
    return CS_OK;
}

CS_BOUNDS_READER(fft_bounds_check)

// reads and clears the flag of a tensor-copy wait that gave up (after the caller synchronised)
cs_status fft_check_and_clear() {
    int v = 0;
    CS_TRY_CUDA(cudaMemcpyFromSymbol(&v, g_fft_error, sizeof(int)));
    if (v) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_fft_error, &zero, sizeof(int));
        set_error("an FFT pass gave up waiting for its tensor copies (bounded wait)");
        return CS_ERR_TIMEOUT;
    }
    return CS_OK;
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
    return launch_pass<EXPAND_X, -1>(A, st);
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
    // coils per chunk cw and rows per CTA R = kLines / cw chosen to waste the fewest of the
    // kLines transform lines per image row (ceil(C / cw) chunks of R rows each), the widest
    // chunk among equals
    const int rmax = std::max(1, 4 * kPassThreads / p->img[2]);   // output elements per thread <= 4
    int best_cw = 1, best_R = 1;
    double best = 1e300;
    for (int cw = std::min(std::max(C, 1), kLines); cw >= 1; --cw) {   // ties: the widest chunk
        const int R = std::min(kLines / cw, rmax);
        const double slots = (double)((C + cw - 1) / cw) * kLines / R;
        if (slots < best - 1e-9) {
            best = slots;
            best_cw = cw;
            best_R = R;
        }
    }
    A.cw = best_cw;
    A.rows_per_cta = best_R;
    return launch_pass<REDUCE_X, 1>(A, st);
}

static cs_status pass_cart_y(const cs_plan* p, int mode, int C, const float2* yk, float2* yko, int residual,
                             cudaStream_t st) {
    PassArgs A = {};
    const int sign = (mode == SCATTER_Y) ? +1 : -1;
    fill_fft(A, p->fft[1], sign);
    A.C = C;
    A.D = p->D;
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
        case GATHER_Y: return launch_pass<GATHER_Y, -1>(A, st);
        case SCATTER_Y: return launch_pass<SCATTER_Y, 1>(A, st);
        default: return launch_pass<MASK_Y, -1>(A, st);
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
