// Solvers of coil sketching on the GPU (Sec. 2.1, 2.3, Algorithm 1):
//   CG (l2 regulariser), FISTA with a periodised db4 prox (l1-wavelets), power iteration for
//   the FISTA step, the sketched sub-problem (Eq. 9-10) and the outer loop of Algorithm 1.
// Vectors are complex64; every inner product and norm is accumulated in FP64 (per-block
// partial sums, then summed in a fixed order by the consuming kernel, so runs are
// bit-reproducible); solver scalars stay on the device (no host round trip inside the loop).
#include <cmath>
#include <complex>
#include <cstdio>
#include <vector>

#include "cs_internal.cuh"

namespace cs {

cs_status sketch_draw_impl(uint64_t seed, int t0, int T, int C, int V, int S, int dist, int norm, float* out,
                           cudaStream_t st);
cs_status sketched_maps_impl(const float* S, const int* tsel, const float2* mrot, int64_t D, int C, int V, int Sn,
                             int precision, float2* out, cudaStream_t st);
cs_status coil_pca_det_impl(const float2* y, int C, int64_t N, float2* U, double* eig, double* Rws, double* part,
                            cudaStream_t st);
int64_t coil_cov_part_size(int C, int64_t N);
cs_status coil_rotate_impl(const float2* U, const float2* in, int C, int Cout, int64_t L, float2* out, cudaStream_t st);
cs_status tc_check_and_clear();

constexpr int kRedBlocks = 296;   // partial sums per reduction (2 per SM of a 148/152-SM part)
constexpr int kRedThreads = 256;
int reduce_blocks() { return kRedBlocks; }

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[kRedThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x / 32, l = threadIdx.x % 32;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kRedThreads / 32; ++i) s += red[i];
    return s;  // valid in thread 0
}

// sum of kRedBlocks partials in a fixed order (every CTA gets the same value)
__device__ __forceinline__ double sum_partials(const double* __restrict__ part) {
    __shared__ double s_val;
    if (threadIdx.x < 32) {
        double v = 0;
        for (int i = threadIdx.x; i < kRedBlocks; i += 32) v += part[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) s_val = v;
    }
    __syncthreads();
    return s_val;
}

// Re<a, b> partials (a == b gives ||a||^2)
__global__ void __launch_bounds__(kRedThreads) dot_kernel(const float2* __restrict__ a, const float2* __restrict__ b,
                                                          int64_t n, double* __restrict__ part) {
    double acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 x = a[i], y = b[i];
        acc += (double)fmaf(x.x, y.x, x.y * y.y);
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

struct Scal {
    double rr[2];     // CG: squared residual norm, parity slots
    double L;         // power iteration: largest eigenvalue estimate
    double eta;       // FISTA step
    int nonfinite;
    int naccept;      // warm starts accepted in this solve
    double fhat, ft;  // warm start: sub-problem objective at the prediction and at x^t
    double refn2;     // trace: ||x_ref||^2
};

// CG start for the sub-problem: r = -(d + lambda x), p = r, partials of ||r||^2
__global__ void cg_init_kernel(const float2* __restrict__ d, const float2* __restrict__ x, float lambda, int64_t n,
                               float2* __restrict__ r, float2* __restrict__ p, double* __restrict__ part) {
    double acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 dv = d[i], xv = x[i];
        const float2 rv = make_float2(-(dv.x + lambda * xv.x), -(dv.y + lambda * xv.y));
        r[i] = rv;
        p[i] = rv;
        acc += (double)fmaf(rv.x, rv.x, rv.y * rv.y);
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// warm-started sub-problem CG: r = -(d + lambda u) - A_S^H A_S (u - x^t) (the last term given), p = r
__global__ void cg_init_warm_kernel(const float2* __restrict__ d, const float2* __restrict__ u, const float2* __restrict__ hdu,
                                    float lambda, int64_t n, float2* __restrict__ r, float2* __restrict__ p,
                                    double* __restrict__ part) {
    double acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 dv = d[i], uv = u[i], hv = hdu[i];
        const float2 rv = make_float2(-(dv.x + lambda * uv.x + hv.x), -(dv.y + lambda * uv.y + hv.y));
        r[i] = rv;
        p[i] = rv;
        acc += (double)fmaf(rv.x, rv.x, rv.y * rv.y);
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// plain CG start: r = b - H x (b, Hx given), p = r
__global__ void cg_init2_kernel(const float2* __restrict__ b, const float2* __restrict__ hx, int64_t n,
                                float2* __restrict__ r, float2* __restrict__ p, double* __restrict__ part) {
    double acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 rv = csub(b[i], hx[i]);
        r[i] = rv;
        p[i] = rv;
        acc += (double)fmaf(rv.x, rv.x, rv.y * rv.y);
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void store_sum_kernel(const double* __restrict__ part, double* __restrict__ dst) {
    const double s = sum_partials(part);
    if (threadIdx.x == 0) *dst = s;
}

// alpha = rr / <p, Hp>; x += alpha p; r -= alpha Hp; partials of ||r||^2
__global__ void __launch_bounds__(kRedThreads) cg_update_kernel(const double* __restrict__ php_part, Scal* sc, int par,
                                                                 const int* __restrict__ par_dev, int64_t n,
                                                                 float2* __restrict__ x, float2* __restrict__ r,
                                                                 const float2* __restrict__ p,
                                                                 const float2* __restrict__ hp, double* __restrict__ part) {
    if (par_dev) par = *par_dev & 1;
    const double php = sum_partials(php_part);
    const double rr = sc->rr[par];
    double alpha = rr / php;
    if (!isfinite(rr) || !isfinite(php) || (rr > 0 && !isfinite(alpha))) {
        if (threadIdx.x == 0 && blockIdx.x == 0) sc->nonfinite = 1;
    }
    if (!(rr > 0) || !isfinite(alpha)) alpha = 0;
    const float a = (float)alpha;
    double acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 pv = p[i], hv = hp[i];
        float2 xv = x[i], rv = r[i];
        xv.x = fmaf(a, pv.x, xv.x);
        xv.y = fmaf(a, pv.y, xv.y);
        rv.x = fmaf(-a, hv.x, rv.x);
        rv.y = fmaf(-a, hv.y, rv.y);
        x[i] = xv;
        r[i] = rv;
        acc += (double)fmaf(rv.x, rv.x, rv.y * rv.y);
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// beta = rr_new / rr; p = r + beta p; rr slot (par ^ 1) = rr_new
__global__ void __launch_bounds__(kRedThreads) cg_dir_kernel(const double* __restrict__ rr_part, Scal* sc, int par,
                                                              const int* __restrict__ par_dev, int64_t n,
                                                              const float2* __restrict__ r, float2* __restrict__ p) {
    if (par_dev) par = *par_dev & 1;
    const double rrn = sum_partials(rr_part);
    const double rr = sc->rr[par];
    double beta = (rr > 0) ? rrn / rr : 0.0;
    if (!isfinite(beta) || !isfinite(rrn)) {
        if (threadIdx.x == 0 && blockIdx.x == 0) sc->nonfinite = 1;
        beta = 0;
    }
    if (threadIdx.x == 0 && blockIdx.x == 0) sc->rr[par ^ 1] = rrn;
    const float b = (float)beta;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 rv = r[i];
        float2 pv = p[i];
        pv.x = fmaf(b, pv.x, rv.x);
        pv.y = fmaf(b, pv.y, rv.y);
        p[i] = pv;
    }
}

// out = a - b
__global__ void sub_kernel(const float2* __restrict__ a, const float2* __restrict__ b, int64_t n, float2* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = csub(a[i], b[i]);
}

// FISTA gradient step: v = z - eta (g + d)   (d may be null)
__global__ void fista_step_kernel(const float2* __restrict__ z, const float2* __restrict__ g, const float2* __restrict__ d,
                                  const Scal* sc, int64_t n, float2* __restrict__ v) {
    const float eta = (float)sc->eta;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float2 gv = g[i];
        if (d) gv = cadd(gv, d[i]);
        const float2 zv = z[i];
        v[i] = make_float2(fmaf(-eta, gv.x, zv.x), fmaf(-eta, gv.y, zv.y));
    }
}

// soft threshold with tau = eta * lambda (eta from the device scalars, or a fixed tau if sc null)
__global__ void soft_kernel(float2* __restrict__ c, int64_t n, float lambda, const Scal* sc, float tau_fixed) {
    const float tau = sc ? (float)(sc->eta * (double)lambda) : tau_fixed;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = c[i];
        const float m = sqrtf(v.x * v.x + v.y * v.y);
        const float s = (m > tau) ? (1.0f - tau / m) : 0.0f;
        c[i] = make_float2(v.x * s, v.y * s);
    }
}

// z = x + theta (x - xprev)
__global__ void momentum_kernel(const float2* __restrict__ x, const float2* __restrict__ xp, float theta,
                                const float* __restrict__ theta_dev, const int* __restrict__ kdev, int64_t n,
                                float2* __restrict__ z) {
    if (theta_dev) theta = theta_dev[*kdev];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = x[i], b = xp[i];
        z[i] = make_float2(fmaf(theta, a.x - b.x, a.x), fmaf(theta, a.y - b.y, a.y));
    }
}

// power iteration: L = ||w||, v = w / L (also sets eta = 1 / L)
__global__ void power_norm_kernel(const double* __restrict__ part, Scal* sc, const float2* __restrict__ w, int64_t n,
                                  float2* __restrict__ v, int set_eta) {
    const double nrm = sqrt(sum_partials(part));
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        sc->L = nrm;
        if (set_eta) sc->eta = (nrm > 0) ? 1.0 / nrm : 0.0;
        if (!isfinite(nrm)) sc->nonfinite = 1;
    }
    const float inv = (nrm > 0) ? (float)(1.0 / nrm) : 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = cscale(w[i], inv);
}

// out[idx] = x with idx = *idev (or the host index when idev is null); then optionally ++*inc
__global__ void copy_iter_kernel(const float2* __restrict__ x, float2* __restrict__ out, const int* __restrict__ idev,
                                 int idx, int64_t n) {
    if (idev) idx = *idev;
    float2* o = out + (int64_t)idx * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) o[i] = x[i];
}

__global__ void set_int_kernel(int* c, int v) {
    if (threadIdx.x == 0) *c = v;
}

__global__ void add_inplace_kernel(float2* __restrict__ a, const float2* __restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = cadd(a[i], b[i]);
}

// AccProxSGD: rows of the coil batch of iteration *kdev: dst[j] = src[coils[k * B + j]], j < B
__global__ void gather_coils_kernel(const float2* __restrict__ src, int64_t len, const int* __restrict__ coils, int B,
                                    const int* __restrict__ kdev, float2* __restrict__ dst) {
    const int k = *kdev;
    for (int j = blockIdx.y; j < B; j += gridDim.y) {
        const float2* s = src + (int64_t)coils[(int64_t)k * B + j] * len;
        float2* d = dst + (int64_t)j * len;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
            d[i] = s[i];
    }
}

// AccProxSGD step: alpha_k = max(beta^k alpha_0, min_frac alpha_0), alpha_0 = 1 / L (power iteration);
// u = z - alpha_k ratio g (ratio = C / B makes the batch gradient unbiased); eta = alpha_k for the
// proximal step that follows
__global__ void sgd_step_kernel(const float2* __restrict__ z, const float2* __restrict__ g, Scal* sc,
                                const int* __restrict__ kdev, double beta, double min_frac, float ratio, int64_t n,
                                float2* __restrict__ u) {
    const double a0 = 1.0 / sc->L;
    const double alpha = fmax(pow(beta, (double)*kdev) * a0, min_frac * a0);
    const float s = (float)alpha * ratio;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 zv = z[i], gv = g[i];
        u[i] = make_float2(fmaf(-s, gv.x, zv.x), fmaf(-s, gv.y, zv.y));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->eta = alpha;
}

__global__ void inc_kernel(int* c) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *c += 1;
}

__global__ void set_L_kernel(Scal* sc, double L) {
    if (threadIdx.x == 0) sc->L = L;
}

__global__ void set_eta_kernel(Scal* sc, double eta) {
    if (threadIdx.x == 0 && blockIdx.x == 0) sc->eta = eta;
}

// ---- per-iteration trace (records of CS_TRACE_FIELDS doubles, row *tdev) ----
__global__ void trace_init_kernel(double* __restrict__ tr, int rows) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * CS_TRACE_FIELDS) return;
    const int f = i % CS_TRACE_FIELDS;
    tr[i] = (f == CS_TRACE_ACCEPT || f == CS_TRACE_DIST2) ? -1.0 : __longlong_as_double(0x7ff8000000000000ll);
}

// tr[row][field] = scale * (sum of the partials in a fixed order) / (denom ? *denom : 1) (+ the
// second partial set times scale2 when part2 is given)
__global__ void trace_store_kernel(const double* __restrict__ part, double scale, const double* __restrict__ part2,
                                   double scale2, const double* __restrict__ denom, double* __restrict__ tr,
                                   const int* __restrict__ tdev, int field) {
    if (threadIdx.x < 32) {
        double a = 0, b = 0;
        for (int i = threadIdx.x; i < kRedBlocks; i += 32) {
            a += part[i];
            if (part2) b += part2[i];
        }
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        if (threadIdx.x == 0) {
            double v = scale * a + (part2 ? scale2 * b : 0.0);
            if (denom) v /= *denom;
            tr[(int64_t)(*tdev) * CS_TRACE_FIELDS + field] = v;
        }
    }
}

__global__ void trace_time_kernel(double* __restrict__ tr, const int* __restrict__ tdev, const Scal* __restrict__ sc,
                                  int have_L) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    tr[(int64_t)(*tdev) * CS_TRACE_FIELDS + CS_TRACE_TIME_NS] = (double)t;
    tr[(int64_t)(*tdev) * CS_TRACE_FIELDS + CS_TRACE_STEP_L] = have_L ? sc->L : 0.0;
}

// partials of ||a - b||^2
__global__ void __launch_bounds__(kRedThreads) diff2_kernel(const float2* __restrict__ a, const float2* __restrict__ b,
                                                            int64_t n, double* __restrict__ part) {
    double acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float dx = a[i].x - b[i].x, dy = a[i].y - b[i].y;
        acc += (double)fmaf(dx, dx, dy * dy);
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// partials of sum |c_i| (complex moduli)
__global__ void l1_kernel(const float2* __restrict__ c, int64_t n, double* __restrict__ part) {
    double acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = c[i];
        acc += (double)sqrtf(v.x * v.x + v.y * v.y);
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// warm start: *dst = 0.5 quad + lin + lambda reg from three partial sets (quad may be null: 0)
__global__ void subobj_kernel(const double* __restrict__ pq, const double* __restrict__ pl, const double* __restrict__ pr,
                              double lambda, double* __restrict__ dst) {
    if (threadIdx.x < 32) {
        double q = 0, l = 0, r = 0;
        for (int i = threadIdx.x; i < kRedBlocks; i += 32) {
            if (pq) q += pq[i];
            l += pl[i];
            r += pr[i];
        }
        for (int o = 16; o > 0; o >>= 1) {
            q += __shfl_down_sync(0xffffffffu, q, o);
            l += __shfl_down_sync(0xffffffffu, l, o);
            r += __shfl_down_sync(0xffffffffu, r, o);
        }
        if (threadIdx.x == 0) *dst = 0.5 * q + l + lambda * r;
    }
}

// warm start: keep the prediction as the sub-problem's start when its objective is lower (x = xhat),
// else leave x = x^t; record the decision in the trace (if any) and the accept count
__global__ void warm_select_kernel(Scal* __restrict__ sc, const float2* __restrict__ xhat, float2* __restrict__ x,
                                   int64_t n, double* __restrict__ tr, const int* __restrict__ tdev) {
    const double fh = sc->fhat, ft = sc->ft;
    const bool ok = isfinite(fh) && isfinite(ft) && fh < ft;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (ok) sc->naccept += 1;
        if (tr) tr[(int64_t)(*tdev) * CS_TRACE_FIELDS + CS_TRACE_ACCEPT] = ok ? 1.0 : 0.0;
    }
    if (!ok) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = xhat[i];
}

// FISTA momentum coefficients theta_k = (t_{k-1} - 1) / t_k, t_0 = 1, t_k = (1 + sqrt(1 + 4 t_{k-1}^2)) / 2
__global__ void theta_kernel(float* theta, int K) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 1.0;
        for (int k = 0; k < K; ++k) {
            const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
            theta[k] = (float)((t - 1.0) / tn);
            t = tn;
        }
    }
}

// ------------------------------------------------------------------------------------------
// periodised orthonormal db4 (8 taps) along one axis of the corner block, in place per line.
// Analysis: a[k] = sum_m h[m] x[(2k+m) mod M], d[k] = sum_m g[m] x[(2k+m) mod M], g[m] = (-1)^m h[7-m],
// stored as [a | d]; synthesis is the transpose.
__constant__ float c_h[8];
__constant__ float c_g[8];

struct WavArgs {
    float2* data;
    int nz, ny, nx;      // full array
    int bz, by, bx;      // current corner block
    int axis;            // 0 z, 1 y, 2 x
    int inverse;
    uint32_t m_mag;      // floor(2^32 / M) + 1 for the line length M of this pass
};

constexpr int kWavLines = 16;
constexpr int kWavMax = 512;

// One CTA filters kWavLines lines of length M held in shared memory (pitch M + 1).  x lines
// (axis 2) are read and written along the line (consecutive threads, consecutive elements); for
// the strided axes a thread keeps one line (t mod kWavLines) and walks its elements, so the
// kWavLines consecutive x positions of a row are one coalesced segment.  Periodic indices are
// reduced by one conditional subtraction (every tap index lies below M + 8 <= 2M).
__global__ void __launch_bounds__(256) wavelet_pass_kernel(WavArgs W) {
    extern __shared__ float2 wsm[];
    const int M = (W.axis == 0) ? W.bz : (W.axis == 1 ? W.by : W.bx);
    const int P = M + 1;
    float2* line = wsm;
    float2* outl = wsm + kWavLines * P;
    __shared__ int64_t sbase[kWavLines];
    const int tid = threadIdx.x;
    const int64_t stride = (W.axis == 2) ? 1 : (W.axis == 1 ? (int64_t)W.nx : (int64_t)W.nx * W.ny);
    if (tid < kWavLines) {
        const int64_t li = (int64_t)blockIdx.x * kWavLines + tid;
        int64_t nlines, base = -1;
        if (W.axis == 2) {
            nlines = (int64_t)W.bz * W.by;
            if (li < nlines) base = ((li / W.by) * W.ny + li % W.by) * W.nx;
        } else if (W.axis == 1) {
            nlines = (int64_t)W.bz * W.bx;
            if (li < nlines) base = (li / W.bx) * W.ny * W.nx + li % W.bx;
        } else {
            nlines = (int64_t)W.by * W.bx;
            if (li < nlines) base = (li / W.bx) * W.nx + li % W.bx;
        }
        sbase[tid] = base;
    }
    __syncthreads();
    const int H = M / 2;
    // element e of the CTA's kWavLines x M block -> (line l, position k)
    auto lk = [&](int e, int& l, int& k) {
        if (W.axis == 2) {
            l = (int)__umulhi((uint32_t)e, W.m_mag);
            k = e - l * M;
        } else {
            l = e % kWavLines;
            k = e / kWavLines;
        }
    };
    constexpr int LB = 8;
    for (int e0 = tid; e0 < kWavLines * M; e0 += 256 * LB) {
        float2 t[LB];
#pragma unroll
        for (int b = 0; b < LB; ++b) {
            const int e = e0 + 256 * b;
            int l, k;
            lk(e, l, k);
            t[b] = (e < kWavLines * M && sbase[l] >= 0) ? W.data[sbase[l] + k * stride] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int b = 0; b < LB; ++b) {
            const int e = e0 + 256 * b;
            int l, k;
            lk(e, l, k);
            if (e < kWavLines * M) line[l * P + k] = t[b];
        }
    }
    __syncthreads();
    for (int e = tid; e < kWavLines * M; e += 256) {
        int l, k;
        lk(e, l, k);
        const float2* x = line + l * P;
        float2 acc = make_float2(0.f, 0.f);
        if (!W.inverse) {
            const int kk = (k < H) ? k : k - H;
            const float* f = (k < H) ? c_h : c_g;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                int idx = 2 * kk + m;
                if (idx >= M) idx -= M;
                const float2 v = x[idx];
                acc.x = fmaf(f[m], v.x, acc.x);
                acc.y = fmaf(f[m], v.y, acc.y);
            }
        } else {
            // x[j] = sum over taps m with (j - m) even: h[m] a[k] + g[m] d[k], k = ((j - m) mod M) / 2
#pragma unroll
            for (int mm = 0; mm < 4; ++mm) {
                const int m = 2 * mm + (k & 1);
                int t = k - m;
                if (t < 0) t += M;
                const int kk = t >> 1;
                const float2 a = x[kk], d = x[H + kk];
                acc.x = fmaf(c_h[m], a.x, fmaf(c_g[m], d.x, acc.x));
                acc.y = fmaf(c_h[m], a.y, fmaf(c_g[m], d.y, acc.y));
            }
        }
        outl[l * P + k] = acc;
    }
    __syncthreads();
    for (int e = tid; e < kWavLines * M; e += 256) {
        int l, k;
        lk(e, l, k);
        if (sbase[l] >= 0) W.data[sbase[l] + k * stride] = outl[l * P + k];
    }
}

// db4 scaling filter from Daubechies' construction: |m0|^2 = cos^8(xi/2) P(sin^2(xi/2)),
// P(y) = 1 + 4y + 10y^2 + 20y^3; the roots of P (Durand-Kerner) map to z-roots of
// z^2 - (2 - 4y) z + 1 = 0, of which the one inside the unit circle is kept (minimum phase).
static void db4_filter(double h[8]) {
    typedef std::complex<double> cd;
    const double P[4] = {1.0, 4.0, 10.0, 20.0};  // coefficients of y^0..y^3
    cd r[3] = {cd(0.4, 0.9), cd(0.4, 0.9) * cd(0.4, 0.9), cd(0.4, 0.9) * cd(0.4, 0.9) * cd(0.4, 0.9)};
    for (int it = 0; it < 500; ++it) {
        for (int i = 0; i < 3; ++i) {
            cd num = P[3];
            for (int k = 2; k >= 0; --k) num = num * r[i] + P[k];
            num /= P[3];
            cd den = 1.0;
            for (int j = 0; j < 3; ++j)
                if (j != i) den *= (r[i] - r[j]);
            r[i] -= num / den;
        }
    }
    // q(z) = prod (z - z_k) with |z_k| < 1
    cd q[4] = {1.0, 0.0, 0.0, 0.0};  // q[0] z^deg + ... (highest first)
    int deg = 0;
    for (int i = 0; i < 3; ++i) {
        const cd b = -(2.0 - 4.0 * r[i]);
        const cd disc = std::sqrt(b * b - 4.0);
        cd z1 = (-b + disc) / 2.0, z2 = (-b - disc) / 2.0;
        const cd zk = (std::abs(z1) < std::abs(z2)) ? z1 : z2;
        cd nq[4] = {0.0, 0.0, 0.0, 0.0};
        for (int k = 0; k <= deg; ++k) {
            nq[k] += q[k];
            nq[k + 1] -= q[k] * zk;
        }
        ++deg;
        for (int k = 0; k < 4; ++k) q[k] = nq[k];
    }
    // h = (1 + z)^4 * q  (coefficients highest power first)
    double bin[5] = {1, 4, 6, 4, 1};
    double hh[8] = {0};
    for (int i = 0; i < 5; ++i)
        for (int k = 0; k < 4; ++k) hh[i + k] += bin[i] * q[k].real();
    double s = 0;
    for (int i = 0; i < 8; ++i) s += hh[i];
    for (int i = 0; i < 8; ++i) hh[i] *= std::sqrt(2.0) / s;
    double first = 0, second = 0;
    for (int i = 0; i < 4; ++i) {
        first += std::fabs(hh[i]);
        second += std::fabs(hh[i + 4]);
    }
    for (int i = 0; i < 8; ++i) h[i] = (first >= second) ? hh[i] : hh[7 - i];
}

constexpr int kWavSmem = (int)sizeof(float2) * 2 * kWavLines * (kWavMax + 1);

cs_status wavelet_init_constants() {
    static int done_dev[64] = {0};
    int dev = 0;
    CS_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && done_dev[dev]) return CS_OK;
    CS_TRY_CUDA(cudaFuncSetAttribute(wavelet_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kWavSmem));
    double h[8];
    db4_filter(h);
    float hf[8], gf[8];
    for (int m = 0; m < 8; ++m) {
        hf[m] = (float)h[m];
        gf[m] = (float)(((m & 1) ? -1.0 : 1.0) * h[7 - m]);
    }
    CS_TRY_CUDA(cudaMemcpyToSymbol(c_h, hf, sizeof(hf)));
    CS_TRY_CUDA(cudaMemcpyToSymbol(c_g, gf, sizeof(gf)));
    if (dev < 64) done_dev[dev] = 1;
    return CS_OK;
}

static cs_status wavelet_apply(float2* data, const int dims3[3], int nd, int levels, int inverse, cudaStream_t st) {
    CS_PROPAGATE(wavelet_init_constants());
    for (int a = 3 - nd; a < 3; ++a) {
        CS_REQUIRE(dims3[a] % (1 << levels) == 0 && (dims3[a] >> (levels - 1)) >= 8 && dims3[a] <= kWavMax,
                   CS_ERR_UNSUPPORTED_SIZE, "wavelet: axis %d (size %d) must be divisible by 2^%d, >= 8 * 2^(levels-1), <= %d",
                   a, dims3[a], levels, kWavMax);
    }
    auto run = [&](int lev, int axis) -> cs_status {
        WavArgs W;
        W.data = data;
        W.nz = dims3[0];
        W.ny = dims3[1];
        W.nx = dims3[2];
        W.bz = (nd == 3) ? dims3[0] >> lev : 1;
        W.by = dims3[1] >> lev;
        W.bx = dims3[2] >> lev;
        W.axis = axis;
        W.inverse = inverse;
        const int M = (axis == 0) ? W.bz : (axis == 1 ? W.by : W.bx);
        W.m_mag = (uint32_t)(0x100000000ull / (unsigned long long)M) + 1u;
        const size_t smem = sizeof(float2) * 2 * kWavLines * (size_t)(M + 1);
        int64_t nlines = (axis == 2) ? (int64_t)W.bz * W.by : (axis == 1 ? (int64_t)W.bz * W.bx : (int64_t)W.by * W.bx);
        wavelet_pass_kernel<<<(unsigned)((nlines + kWavLines - 1) / kWavLines), 256, smem, st>>>(W);
        CS_LAUNCH_CHECK();
        return CS_OK;
    };
    if (!inverse) {
        for (int lev = 0; lev < levels; ++lev)
            for (int axis = 2; axis >= 3 - nd; --axis) CS_PROPAGATE(run(lev, axis));
    } else {
        for (int lev = levels - 1; lev >= 0; --lev)
            for (int axis = 3 - nd; axis < 3; ++axis) CS_PROPAGATE(run(lev, axis));
    }
    return CS_OK;
}

// ------------------------------------------------------------------------------------------
// l1 total variation (Sec. 2.1: g(x) = lambda ||T x||_1, T the forward differences along every
// image axis with periodic wrap; anisotropic: the l1 norm sums the complex moduli of all
// differences) and the two element-wise steps of PDHG (Chambolle & Pock 2011) around its data
// step.  The dual variable is stored [ndim][image], component a for the a-th image axis (slow to
// fast: z, y, x; 2D images: y, x).

struct TvDims {
    int nd;            // image axes (2 or 3)
    int n[3];          // sizes slow to fast, n[0] = 1 for 2D
    int64_t D;
};

// dual step: z_a <- proj_lambda(z_a + sigma (T xbar)_a), xbar = 2 x - x_prev (x_prev null: xbar = x);
// proj_lambda scales an entry down to modulus lambda when it is larger.  One CTA per image row
// (z, y), threads along x.
__global__ void tv_dual_kernel(const float2* __restrict__ x, const float2* __restrict__ xp, float2* __restrict__ z,
                               TvDims t, float sigma, float lam) {
    const float lam2 = lam * lam;
    const int rows = t.n[0] * t.n[1];
    const int64_t sy = t.n[2], sz = (int64_t)t.n[1] * t.n[2];
    auto xbar = [&](int64_t j) {
        float2 v = x[j];
        if (xp) v = make_float2(2.f * v.x - xp[j].x, 2.f * v.y - xp[j].y);
        return v;
    };
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int iz = row / t.n[1], iy = row - iz * t.n[1];
        const int64_t base = (int64_t)row * t.n[2];
        // offsets of the +1 neighbour along z and y (periodic)
        const int64_t dz = (iz + 1 < t.n[0]) ? sz : -(int64_t)(t.n[0] - 1) * sz;
        const int64_t dy = (iy + 1 < t.n[1]) ? sy : -(int64_t)(t.n[1] - 1) * sy;
        for (int ix = threadIdx.x; ix < t.n[2]; ix += blockDim.x) {
            const int64_t i = base + ix;
            const int64_t nx1 = (ix + 1 < t.n[2]) ? i + 1 : base;
            const float2 xc = xbar(i);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a < 3 - t.nd) continue;
                const int c = a - (3 - t.nd);
                const float2 xn = xbar(a == 0 ? i + dz : (a == 1 ? i + dy : nx1));
                float2 v = z[c * t.D + i];
                v.x = fmaf(sigma, xn.x - xc.x, v.x);
                v.y = fmaf(sigma, xn.y - xc.y, v.y);
                const float m2 = fmaf(v.x, v.x, v.y * v.y);
                if (m2 > lam2) {
                    const float sc = lam * rsqrtf(m2);
                    v.x *= sc;
                    v.y *= sc;
                }
                z[c * t.D + i] = v;
            }
        }
    }
}

// data-step right-hand side: rhs = b0 + x / tau - T^H z, (T^H z)[r] = sum_a z_a[r - e_a] - z_a[r];
// x_prev (if given) receives x.  b0 may be null (zero).
__global__ void tv_rhs_kernel(const float2* __restrict__ b0, const float2* __restrict__ x, const float2* __restrict__ z,
                              TvDims t, float inv_tau, float2* __restrict__ rhs, float2* __restrict__ xp) {
    const int rows = t.n[0] * t.n[1];
    const int64_t sy = t.n[2], sz = (int64_t)t.n[1] * t.n[2];
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int iz = row / t.n[1], iy = row - iz * t.n[1];
        const int64_t base = (int64_t)row * t.n[2];
        // offsets of the -1 neighbour along z and y (periodic)
        const int64_t dz = (iz > 0) ? -sz : (int64_t)(t.n[0] - 1) * sz;
        const int64_t dy = (iy > 0) ? -sy : (int64_t)(t.n[1] - 1) * sy;
        for (int ix = threadIdx.x; ix < t.n[2]; ix += blockDim.x) {
            const int64_t i = base + ix;
            const int64_t nx1 = (ix > 0) ? i - 1 : base + t.n[2] - 1;
            float2 div = make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a < 3 - t.nd) continue;
                const int c = a - (3 - t.nd);
                const float2 zp = z[c * t.D + (a == 0 ? i + dz : (a == 1 ? i + dy : nx1))], zc = z[c * t.D + i];
                div.x += zp.x - zc.x;
                div.y += zp.y - zc.y;
            }
            const float2 xv = x[i];
            const float2 bv = b0 ? b0[i] : make_float2(0.f, 0.f);
            rhs[i] = make_float2(fmaf(inv_tau, xv.x, bv.x) - div.x, fmaf(inv_tau, xv.y, bv.y) - div.y);
            if (xp) xp[i] = xv;
        }
    }
}

static int tv_grid(const TvDims& t) { return (int)std::min<int64_t>((int64_t)t.n[0] * t.n[1], 152 * 16); }

static TvDims tv_dims(int nd, const int dims3[3]) {
    TvDims t;
    t.nd = nd;
    for (int a = 0; a < 3; ++a) t.n[a] = dims3[a];
    t.D = (int64_t)dims3[0] * dims3[1] * dims3[2];
    return t;
}

static int vec_grid(int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + kRedThreads - 1) / kRedThreads, kRedBlocks));
}

// ------------------------------------------------------------------------------------------
// recon_solve
//
// The solver's device vectors live in a per-plan workspace that persists across calls (so that
// pointers are stable and a captured CUDA graph can be replayed by later calls); all scalars of
// the iteration stay on the device.  With use_graph, one outer iteration of Algorithm 1 (true
// gradient, sketched maps selected by a device-side iteration counter, K inner iterations,
// iterate copy, counter increment) - or, for the plain solver, one iteration - is captured once,
// cached in the plan under a signature of the call's arguments, and replayed.

struct SolverWS {
    int64_t D = 0, N = 0;
    int C = 0, S = 0, Kc = 0, T = 0, K = 0;
    Scal* sc = nullptr;
    double *partA = nullptr, *partB = nullptr, *eig = nullptr, *Rws = nullptr;
    float2 *U = nullptr, *maps_r = nullptr, *y_r = nullptr, *d = nullptr, *hp = nullptr, *u = nullptr, *z = nullptr,
           *xp = nullptr, *gr = nullptr, *xt = nullptr, *r = nullptr, *pv = nullptr, *msk = nullptr;
    float* skd = nullptr;
    float* theta = nullptr;
    int* tdev = nullptr;
    float2* tvz = nullptr;   // l1-TV dual variable [ndim][image] (PDHG), allocated on first use
    int64_t tvz_n = 0;
    float2* ysk = nullptr;   // sketched k-space rows S~_S^0 y of the classical-sketch initialisation
    int64_t ysk_n = 0;
    int* tinit = nullptr;    // device index of the initialisation's sketch block
    float2 *bmaps = nullptr, *by = nullptr;   // AccProxSGD: the current coil batch's maps and data
    int64_t bmaps_n = 0, by_n = 0;
    double* trace = nullptr;   // device trace records [trace_rows][CS_TRACE_FIELDS]
    int trace_rows = 0;
    float2* kres = nullptr;    // trace objective: full forward operator output [C][N]
    int64_t kres_n = 0;
    float2 *xt0 = nullptr, *xhat = nullptr;   // warm start: saved x^t and the prediction
    double* partC = nullptr;
    float2* peig = nullptr;    // step re-estimation: the eigenvector estimate carried across outer iterations
    std::vector<void*> allocs;
    cudaGraphExec_t gexec = nullptr;
    uint64_t gsig = 0;
    cudaStream_t cap = nullptr;   // non-blocking stream used only for graph capture
    void free_all() {
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        gsig = 0;
        for (void* q : allocs) cudaFree(q);
        allocs.clear();
        tvz = nullptr;
        tvz_n = 0;
        ysk = nullptr;
        ysk_n = 0;
        tinit = nullptr;
        bmaps = by = nullptr;
        bmaps_n = by_n = 0;
        trace = nullptr;
        trace_rows = 0;
        kres = nullptr;
        kres_n = 0;
        xt0 = xhat = nullptr;
        partC = nullptr;
        peig = nullptr;
    }
    void drop_graph() {
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        gsig = 0;
    }
    cs_status ensure_trace(int rows) {
        if (trace && trace_rows >= rows) return CS_OK;
        drop_graph();
        CS_PROPAGATE(get(&trace, (size_t)rows * CS_TRACE_FIELDS));
        trace_rows = rows;
        return CS_OK;
    }
    cs_status ensure_kres(int64_t n) {
        if (kres && kres_n >= n) return CS_OK;
        drop_graph();
        CS_PROPAGATE(get(&kres, (size_t)n));
        kres_n = n;
        return CS_OK;
    }
    cs_status ensure_peig() {
        if (peig) return CS_OK;
        drop_graph();
        return get(&peig, (size_t)D);
    }
    cs_status ensure_warm() {
        if (xt0 && xhat && partC) return CS_OK;
        drop_graph();
        CS_PROPAGATE(get(&xt0, (size_t)D));
        CS_PROPAGATE(get(&xhat, (size_t)D));
        CS_PROPAGATE(get(&partC, (size_t)kRedBlocks));
        return CS_OK;
    }
    cs_status ensure_sgd(int64_t nm, int64_t ny) {
        if (bmaps && bmaps_n >= nm && by && by_n >= ny) return CS_OK;
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        gsig = 0;
        CS_PROPAGATE(get(&bmaps, (size_t)nm));
        CS_PROPAGATE(get(&by, (size_t)ny));
        bmaps_n = nm;
        by_n = ny;
        return CS_OK;
    }
    cs_status ensure_init(int64_t n) {
        if (ysk && ysk_n >= n && tinit) return CS_OK;
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        gsig = 0;
        CS_PROPAGATE(get(&ysk, (size_t)std::max<int64_t>(n, 1)));
        ysk_n = n;
        if (!tinit) CS_PROPAGATE(get(&tinit, 1));
        return CS_OK;
    }
    cs_status ensure_tv(int64_t n) {
        if (tvz && tvz_n >= n) return CS_OK;
        if (gexec) cudaGraphExecDestroy(gexec);   // a cached graph may refer to the old buffer
        gexec = nullptr;
        gsig = 0;
        CS_PROPAGATE(get(&tvz, (size_t)n));
        tvz_n = n;
        return CS_OK;
    }
    ~SolverWS() {
        free_all();
        if (cap) cudaStreamDestroy(cap);
    }
    template <typename T_>
    cs_status get(T_** out, size_t count) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, sizeof(T_) * std::max<size_t>(count, 1));
        if (e != cudaSuccess) {
            set_error("recon_solve workspace allocation (%zu bytes): %s", sizeof(T_) * count, cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? CS_ERR_OOM : CS_ERR_CUDA;
        }
        allocs.push_back(q);
        *out = (T_*)q;
        return CS_OK;
    }
    // (re)allocate for the given sizes when the current buffers are too small
    cs_status ensure(int64_t D_, int64_t N_, int C_, int S_, int Kc_, int T_, int K_) {
        if (!allocs.empty() && D_ <= D && N_ <= N && C_ <= C && S_ <= S && Kc_ <= Kc && T_ <= T && K_ <= K) return CS_OK;
        free_all();
        D = std::max(D_, D);
        N = std::max(N_, N);
        C = std::max(C_, C);
        S = std::max(S_, S);
        Kc = std::max(Kc_, Kc);
        T = std::max(T_, T);
        K = std::max(K_, K);
        CS_PROPAGATE(get(&sc, 1));
        CS_PROPAGATE(get(&partA, kRedBlocks));
        CS_PROPAGATE(get(&partB, kRedBlocks));
        CS_PROPAGATE(get(&U, (size_t)C * C));
        CS_PROPAGATE(get(&eig, (size_t)C));
        // the FP64 covariance followed by the slot array of its fixed-order reduction
        CS_PROPAGATE(get(&Rws, (size_t)(2 * C * C + coil_cov_part_size(C, N))));
        CS_PROPAGATE(get(&maps_r, (size_t)C * D));
        CS_PROPAGATE(get(&y_r, (size_t)C * N));
        for (float2** v : {&d, &hp, &u, &z, &xp, &gr, &xt, &r, &pv}) CS_PROPAGATE(get(v, (size_t)D));
        CS_PROPAGATE(get(&msk, (size_t)std::max(S, 1) * D));
        CS_PROPAGATE(get(&skd, (size_t)std::max(T * S * Kc, 1)));
        CS_PROPAGATE(get(&theta, (size_t)std::max(K, 1)));
        CS_PROPAGATE(get(&tdev, 1));
        return CS_OK;
    }
};

void solver_ws_free(cs_plan* p) {
    delete static_cast<SolverWS*>(p->solver_ws);
    p->solver_ws = nullptr;
}

struct Ctx {
    const cs_plan* p;
    cudaStream_t st;
    int64_t D;
    Scal* sc;
    double* partA;
    double* partB;
    int dims3[3];
    int nd;
    int levels;
    float lambda;
};

// z = A_S^H A_S v (+ lambda v) with the sketched maps (V rows of maps_v, S rows of maps_s)
static cs_status normal_apply(const Ctx& c, const float2* v, const float2* mv, int V, const float2* ms, int S, float lam,
                              float2* z) {
    return sketched_normal_apply(c.p, (const float*)v, (const float*)mv, V, (const float*)ms, S, lam, (float*)z, c.st);
}

static cs_status prox_wavelet(const Ctx& c, float2* v, float2* x_out, const Scal* sc, float tau_fixed) {
    // v is overwritten by its coefficients; x_out = Psi^H soft(Psi v)
    CS_PROPAGATE(wavelet_apply(v, c.dims3, c.nd, c.levels, 0, c.st));
    soft_kernel<<<vec_grid(c.D), kRedThreads, 0, c.st>>>(v, c.D, c.lambda, sc, tau_fixed);
    CS_LAUNCH_CHECK();
    CS_PROPAGATE(wavelet_apply(v, c.dims3, c.nd, c.levels, 1, c.st));
    CS_TRY_CUDA(cudaMemcpyAsync(x_out, v, sizeof(float2) * c.D, cudaMemcpyDeviceToDevice, c.st));
    return CS_OK;
}

static cs_status power_iteration(const Ctx& c, const float2* v0, int iters, const float2* mv, int V, const float2* ms,
                                 int S, float2* v, float2* w) {
    const int g = vec_grid(c.D);
    dot_kernel<<<kRedBlocks, kRedThreads, 0, c.st>>>(v0, v0, c.D, c.partA);
    CS_LAUNCH_CHECK();
    power_norm_kernel<<<g, kRedThreads, 0, c.st>>>(c.partA, c.sc, v0, c.D, v, 0);
    CS_LAUNCH_CHECK();
    for (int it = 0; it < iters; ++it) {
        CS_PROPAGATE(normal_apply(c, v, mv, V, ms, S, 0.f, w));
        dot_kernel<<<kRedBlocks, kRedThreads, 0, c.st>>>(w, w, c.D, c.partA);
        CS_LAUNCH_CHECK();
        power_norm_kernel<<<g, kRedThreads, 0, c.st>>>(c.partA, c.sc, w, c.D, v, 1);
        CS_LAUNCH_CHECK();
    }
    return CS_OK;
}

// one CG iteration on H = A^H A + lambda I (sketched or full maps); parity from host k or device counter
static cs_status cg_iter(const Ctx& c, const float2* mv, int V, const float2* ms, int S, float2* x, float2* r,
                         float2* pv, float2* hp, int par, const int* par_dev) {
    CS_PROPAGATE(normal_apply(c, pv, mv, V, ms, S, c.lambda, hp));
    dot_kernel<<<kRedBlocks, kRedThreads, 0, c.st>>>(pv, hp, c.D, c.partA);
    CS_LAUNCH_CHECK();
    cg_update_kernel<<<kRedBlocks, kRedThreads, 0, c.st>>>(c.partA, c.sc, par, par_dev, c.D, x, r, pv, hp, c.partB);
    CS_LAUNCH_CHECK();
    cg_dir_kernel<<<vec_grid(c.D), kRedThreads, 0, c.st>>>(c.partB, c.sc, par, par_dev, c.D, r, pv);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

// K CG iterations on (A_S^H A_S + lambda I) x = A_S^H A_S x^t - d from x^t (x updated in place);
// the initial residual is b - H x^t = -(d + lambda x^t)
static cs_status cg_sub(const Ctx& c, const float2* d, float2* x, int K, const float2* mv, int V, const float2* ms, int S,
                        float2* r, float2* pv, float2* hp, const float2* xt_other = nullptr, float2* tmp = nullptr) {
    if (xt_other) {
        // warm start: x holds the start u != x^t; r0 = -(d + lambda u) - A_S^H A_S (u - x^t)
        sub_kernel<<<vec_grid(c.D), kRedThreads, 0, c.st>>>(x, xt_other, c.D, tmp);
        CS_LAUNCH_CHECK();
        CS_PROPAGATE(normal_apply(c, tmp, mv, V, ms, S, 0.f, hp));
        cg_init_warm_kernel<<<kRedBlocks, kRedThreads, 0, c.st>>>(d, x, hp, c.lambda, c.D, r, pv, c.partB);
    } else {
        cg_init_kernel<<<kRedBlocks, kRedThreads, 0, c.st>>>(d, x, c.lambda, c.D, r, pv, c.partB);
    }
    CS_LAUNCH_CHECK();
    store_sum_kernel<<<1, 32, 0, c.st>>>(c.partB, &c.sc->rr[0]);
    CS_LAUNCH_CHECK();
    for (int k = 0; k < K; ++k) CS_PROPAGATE(cg_iter(c, mv, V, ms, S, x, r, pv, hp, k & 1, nullptr));
    return CS_OK;
}

// K FISTA iterations on the sketched sub-problem from x^t: grad = A_S^H A_S (z - x^t) + d
static cs_status fista_sub(const Ctx& c, const float2* d, float2* x, int K, const float2* mv, int V, const float2* ms,
                           int S, const std::vector<float>& theta, float2* z, float2* xp, float2* u, float2* gr,
                           float2* xt, const float2* xt_other = nullptr) {
    const int g = vec_grid(c.D);
    // x^t is x on entry, unless a warm start u = x was given with x^t elsewhere
    CS_TRY_CUDA(cudaMemcpyAsync(xt, xt_other ? xt_other : x, sizeof(float2) * c.D, cudaMemcpyDeviceToDevice, c.st));
    CS_TRY_CUDA(cudaMemcpyAsync(z, x, sizeof(float2) * c.D, cudaMemcpyDeviceToDevice, c.st));
    CS_TRY_CUDA(cudaMemcpyAsync(xp, x, sizeof(float2) * c.D, cudaMemcpyDeviceToDevice, c.st));
    for (int k = 0; k < K; ++k) {
        sub_kernel<<<g, kRedThreads, 0, c.st>>>(z, xt, c.D, u);
        CS_LAUNCH_CHECK();
        CS_PROPAGATE(normal_apply(c, u, mv, V, ms, S, 0.f, gr));
        fista_step_kernel<<<g, kRedThreads, 0, c.st>>>(z, gr, d, c.sc, c.D, u);
        CS_LAUNCH_CHECK();
        CS_PROPAGATE(prox_wavelet(c, u, x, c.sc, 0.f));
        momentum_kernel<<<g, kRedThreads, 0, c.st>>>(x, xp, theta[k], nullptr, nullptr, c.D, z);
        CS_LAUNCH_CHECK();
        CS_TRY_CUDA(cudaMemcpyAsync(xp, x, sizeof(float2) * c.D, cudaMemcpyDeviceToDevice, c.st));
    }
    return CS_OK;
}

// K PDHG iterations (Chambolle & Pock 2011, theta = 1) on min_x f(x) + lambda ||T x||_1 with the
// data step prox_{tau f}(v) solved by M CG iterations on (A^H A + I/tau) u = b0 + v/tau started at
// the current iterate (A: the sketched or the full model given by the maps).  For the sketched
// sub-problem f(x) = 1/2 ||A_S (x - x^t)||^2 + Re<x, d> and b0 = A_S^H A_S x^t - d (formed here
// when d is given); for the plain problem b0 = A^H y is passed in.  zd is the dual variable,
// carried in and out.  Buffers: b0, xp (previous iterate), rhs, and the CG vectors r, pv, hp.
struct PdhgArgs {
    int K, M;
    float tau, sigma, lam_tv;
    float2 *zd, *b0, *xp, *rhs, *r, *pv, *hp;
};

static cs_status pdhg_sub(const Ctx& c, const float2* d, float2* x, const float2* mv, int V, const float2* ms, int S,
                          const PdhgArgs& P) {
    const TvDims t = tv_dims(c.nd, c.dims3);
    if (d) {
        CS_PROPAGATE(normal_apply(c, x, mv, V, ms, S, 0.f, P.hp));
        sub_kernel<<<vec_grid(c.D), kRedThreads, 0, c.st>>>(P.hp, d, c.D, P.b0);
        CS_LAUNCH_CHECK();
    }
    // xbar_0 = x: the dual step of the first iteration reads 2 x - x_prev with x_prev = x
    CS_TRY_CUDA(cudaMemcpyAsync(P.xp, x, sizeof(float2) * c.D, cudaMemcpyDeviceToDevice, c.st));
    Ctx cc = c;
    cc.lambda = 1.0f / P.tau;
    for (int k = 0; k < P.K; ++k) {
        tv_dual_kernel<<<tv_grid(t), 128, 0, c.st>>>(x, P.xp, P.zd, t, P.sigma, P.lam_tv);
        CS_LAUNCH_CHECK();
        tv_rhs_kernel<<<tv_grid(t), 128, 0, c.st>>>(P.b0, x, P.zd, t, cc.lambda, P.rhs, P.xp);
        CS_LAUNCH_CHECK();
        // CG from the current iterate: r = rhs - (A^H A + I/tau) x
        CS_PROPAGATE(normal_apply(cc, x, mv, V, ms, S, cc.lambda, P.hp));
        cg_init2_kernel<<<kRedBlocks, kRedThreads, 0, c.st>>>(P.rhs, P.hp, c.D, P.r, P.pv, c.partB);
        CS_LAUNCH_CHECK();
        store_sum_kernel<<<1, 32, 0, c.st>>>(c.partB, &c.sc->rr[0]);
        CS_LAUNCH_CHECK();
        for (int m = 0; m < P.M; ++m) CS_PROPAGATE(cg_iter(cc, mv, V, ms, S, x, P.r, P.pv, P.hp, m & 1, nullptr));
    }
    return CS_OK;
}

static void pdhg_default_steps(int nd, float* tau, float* sigma) {
    // tau = sigma = 0.99 / ||T||, ||T||^2 = 4 ndim, so that tau sigma ||T||^2 < 1
    const float s = (float)(0.99 / std::sqrt(4.0 * nd));
    if (!(*tau > 0)) *tau = s;
    if (!(*sigma > 0)) *sigma = s;
}

static std::vector<float> fista_thetas(int K) {
    std::vector<float> th(K);
    double t = 1.0;
    for (int k = 0; k < K; ++k) {
        const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
        th[k] = (float)((t - 1.0) / tn);
        t = tn;
    }
    return th;
}

static uint64_t fnv(uint64_t h, const void* data, size_t n) {
    const unsigned char* b = (const unsigned char*)data;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

// Run `body(stream)` `reps` times on `st`, or - with use_graph - capture it once on the
// workspace's capture stream (the caller's stream may be the legacy default stream, which cannot
// be captured), cache the instantiated graph and launch it `reps` times on `st`.
template <typename F>
static cs_status run_body(SolverWS* ws, bool use_graph, uint64_t sig, int reps, cudaStream_t st, F body, int* graph_used) {
    if (!use_graph) {
        for (int i = 0; i < reps; ++i) CS_PROPAGATE(body(st));
        return CS_OK;
    }
    if (!ws->gexec || ws->gsig != sig) {
        if (ws->gexec) cudaGraphExecDestroy(ws->gexec);
        ws->gexec = nullptr;
        if (!ws->cap) CS_TRY_CUDA(cudaStreamCreateWithFlags(&ws->cap, cudaStreamNonBlocking));
        CS_TRY_CUDA(cudaStreamBeginCapture(ws->cap, cudaStreamCaptureModeThreadLocal));
        cs_status rc = body(ws->cap);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(ws->cap, &g);
        if (rc != CS_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) {
            set_error("graph capture failed: %s", cudaGetErrorString(e));
            return CS_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&ws->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ws->gexec = nullptr;
            set_error("graph instantiation failed: %s", cudaGetErrorString(e));
            return CS_ERR_CUDA;
        }
        ws->gsig = sig;
    }
    for (int i = 0; i < reps; ++i) CS_TRY_CUDA(cudaGraphLaunch(ws->gexec, st));
    *graph_used = 1;
    return CS_OK;
}

// Enqueue a whole solve on `st` (no host synchronisation).  With allow_graph == false the
// iterations are launched directly even if sp->use_graph is set (used inside an outer capture).
struct SolveEvents {
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
    int graph_used = 0;
    ~SolveEvents() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (e2) cudaEventDestroy(e2);
    }
};

static cs_status recon_enqueue(cs_plan* p, const cs_problem* pr, const cs_solve_params* sp, float2* x, cudaStream_t st,
                               bool allow_graph, SolveEvents* ev) {
    const int64_t D = p->D, N = p->N;
    const int C = pr->C;
    const bool sketch = sp->sketch != 0;
    const int V = sketch ? sp->V : C, S = sketch ? sp->S : 0, Kc = C - V;
    const int T = sp->T, K = sp->K;
    const int init = (sketch && sp->init) ? 1 : 0;   // classical-sketch initialisation (sketch block T)
    if (!p->solver_ws) p->solver_ws = new SolverWS();
    SolverWS* ws = static_cast<SolverWS*>(p->solver_ws);
    CS_PROPAGATE(ws->ensure(D, N, C, S, Kc, T + init, K));
    if (init) CS_PROPAGATE(ws->ensure_init((int64_t)S * N));
    Ctx c;
    c.p = p;
    c.st = st;
    c.D = D;
    c.nd = p->ndim;
    for (int a = 0; a < 3; ++a) c.dims3[a] = p->img[a];
    c.levels = pr->wavelet_levels > 0 ? pr->wavelet_levels : 4;
    c.lambda = pr->lambda;
    c.sc = ws->sc;
    c.partA = ws->partA;
    c.partB = ws->partB;
    CS_TRY_CUDA(cudaMemsetAsync(ws->sc, 0, sizeof(Scal), st));
    CS_TRY_CUDA(cudaMemsetAsync(ws->tdev, 0, sizeof(int), st));
    if (sp->step > 0) {
        set_eta_kernel<<<1, 32, 0, st>>>(ws->sc, (double)sp->step);
        CS_LAUNCH_CHECK();
    }
    if (ev) {
        CS_TRY_CUDA(cudaEventCreate(&ev->e0));
        CS_TRY_CUDA(cudaEventCreate(&ev->e1));
        CS_TRY_CUDA(cudaEventCreate(&ev->e2));
        CS_TRY_CUDA(cudaEventRecord(ev->e0, st));
    }


    const float2* maps = (const float2*)pr->maps;
    const float2* y = (const float2*)pr->y;
    if (sp->do_pca) {
        CS_PROPAGATE(coil_pca_det_impl(y, C, N, ws->U, ws->eig, ws->Rws, ws->Rws + 2 * C * C, st));
        CS_PROPAGATE(coil_rotate_impl(ws->U, maps, C, C, D, ws->maps_r, st));
        CS_PROPAGATE(coil_rotate_impl(ws->U, y, C, C, N, ws->y_r, st));
        maps = ws->maps_r;
        y = ws->y_r;
    }
    if (ev) CS_TRY_CUDA(cudaEventRecord(ev->e1, st));

    const bool fista = pr->reg == CS_REG_L1_WAVELET;
    const bool tvreg = pr->reg == CS_REG_L1_TV;
    // plain solvers: aggressive coil compression keeps the first `keep` (virtual) coils
    const int Cp = (!sketch && sp->keep > 0) ? std::min(sp->keep, C) : C;
    const bool sgd = !sketch && sp->sgd_batch > 0;
    // FISTA step re-estimated at every outer iteration (power iterations on that iteration's
    // sketched operator, warm-started from the previous eigenvector)
    const int pso = sp->step_per_outer;
    CS_REQUIRE(pso >= 0 && (pso == 0 || (sketch && fista && !(sp->step > 0))), CS_ERR_INVALID_ARG,
               "step_per_outer needs a sketched l1-wavelet (FISTA) solve with step = 0");
    if (pso > 0) CS_PROPAGATE(ws->ensure_peig());
    const int have_L = (fista && !(sp->step > 0)) ? 1 : 0;
    PdhgArgs pd = {};
    if (tvreg) {
        CS_REQUIRE(K >= 1 && sp->cg_iters >= 0, CS_ERR_INVALID_ARG, "l1-TV needs K >= 1 and cg_iters >= 0");
        CS_PROPAGATE(ws->ensure_tv((int64_t)c.nd * D));
        CS_TRY_CUDA(cudaMemsetAsync(ws->tvz, 0, sizeof(float2) * c.nd * D, st));
        pd.K = K;
        pd.M = sp->cg_iters > 0 ? sp->cg_iters : 5;
        pd.tau = sp->tv_tau;
        pd.sigma = sp->tv_sigma;
        pdhg_default_steps(c.nd, &pd.tau, &pd.sigma);
        pd.lam_tv = pr->lambda;
        pd.zd = ws->tvz;
        pd.b0 = ws->u;
        pd.xp = ws->xp;
        pd.rhs = ws->gr;
        pd.r = ws->r;
        pd.pv = ws->pv;
        pd.hp = ws->hp;
    }
    const std::vector<float> theta = fista_thetas(std::max(K, 1));
    const bool use_graph = sp->use_graph != 0 && allow_graph;
    // optional trace (one record per outer iteration, or per iteration of the plain solver) and
    // optional learned warm start; both run entirely on the device inside the loop body
    const bool tracing = sp->trace != nullptr;
    const bool trace_obj = tracing && sp->trace_objective != 0 && !tvreg;
    if (tracing) {
        const int rows = sketch ? T : K;
        CS_REQUIRE(rows >= 1, CS_ERR_INVALID_ARG, "a trace needs at least one iteration");
        CS_PROPAGATE(ws->ensure_trace(rows));
        trace_init_kernel<<<(rows * CS_TRACE_FIELDS + 255) / 256, 256, 0, st>>>(ws->trace, rows);
        CS_LAUNCH_CHECK();
        if (sp->x_ref) {
            dot_kernel<<<kRedBlocks, kRedThreads, 0, st>>>((const float2*)sp->x_ref, (const float2*)sp->x_ref, D, c.partA);
            CS_LAUNCH_CHECK();
            store_sum_kernel<<<1, 32, 0, st>>>(c.partA, &ws->sc->refn2);
            CS_LAUNCH_CHECK();
        }
        if (trace_obj) CS_PROPAGATE(ws->ensure_kres((int64_t)C * N));
    }
    const bool warm = sp->warm != nullptr;
    uint64_t wgen = 0;
    if (warm) {
        CS_REQUIRE(sketch && fista && p->ndim == 3, CS_ERR_INVALID_ARG,
                   "the warm start serves sketched l1-wavelet (FISTA) solves of 3D images");
        CS_PROPAGATE(ws->ensure_warm());
        CS_PROPAGATE(unet_prepare(sp->warm, p->img, st, &wgen));
    }
    // ||v||^2 into the trace field of the current row
    auto trace_norm2 = [&](cudaStream_t s, const float2* v, int field) -> cs_status {
        dot_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(v, v, D, ws->partA);
        CS_LAUNCH_CHECK();
        trace_store_kernel<<<1, 32, 0, s>>>(ws->partA, 1.0, nullptr, 0.0, nullptr, ws->trace, ws->tdev, field);
        CS_LAUNCH_CHECK();
        return CS_OK;
    };
    // 1/2 ||A u - y||^2 + g(u) with the first Cn coils (a forward operator into kres); `scr` is a
    // free image-sized buffer for the wavelet coefficients
    auto trace_objective = [&](cudaStream_t s, const float2* u, const float2* mp, int Cn, const float2* yv,
                               float2* scr) -> cs_status {
        CS_PROPAGATE((cs_status)sense_fwd(p, (const float*)u, (const float*)mp, Cn, (float*)ws->kres, s));
        diff2_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(ws->kres, yv, (int64_t)Cn * N, ws->partA);
        CS_LAUNCH_CHECK();
        double rscale = 0.5 * c.lambda;
        if (fista) {
            CS_TRY_CUDA(cudaMemcpyAsync(scr, u, sizeof(float2) * D, cudaMemcpyDeviceToDevice, s));
            CS_PROPAGATE(wavelet_apply(scr, c.dims3, c.nd, c.levels, 0, s));
            l1_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(scr, D, ws->partB);
            rscale = c.lambda;
        } else {
            dot_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(u, u, D, ws->partB);
        }
        CS_LAUNCH_CHECK();
        trace_store_kernel<<<1, 32, 0, s>>>(ws->partA, 0.5, ws->partB, rscale, nullptr, ws->trace, ws->tdev,
                                            CS_TRACE_OBJECTIVE);
        CS_LAUNCH_CHECK();
        return CS_OK;
    };
    // after an iteration: distance to x_ref and the device clock
    auto trace_end = [&](cudaStream_t s) -> cs_status {
        if (sp->x_ref) {
            diff2_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(x, (const float2*)sp->x_ref, D, ws->partA);
            CS_LAUNCH_CHECK();
            trace_store_kernel<<<1, 32, 0, s>>>(ws->partA, 1.0, nullptr, 0.0, &ws->sc->refn2, ws->trace, ws->tdev,
                                                CS_TRACE_DIST2);
            CS_LAUNCH_CHECK();
        }
        trace_time_kernel<<<1, 1, 0, s>>>(ws->trace, ws->tdev, ws->sc, have_L);
        CS_LAUNCH_CHECK();
        return CS_OK;
    };
    int graph_used = 0;
    // signature of everything a captured body depends on
    uint64_t sig = 1469598103934665603ull;
    const void* ptrs[] = {p, x, pr->y, pr->maps, sp->sketches, sp->iterates, sp->power_v0};
    sig = fnv(sig, ptrs, sizeof(ptrs));
    const int ints[] = {C, T, K, V, S, sp->dist, sp->norm, sp->do_pca, sp->precision, pr->reg, c.levels, (int)sketch,
                        init, Cp, sp->sgd_batch, pso};
    const void* ptrs2[] = {sp->sgd_coils};
    const float sgdf[] = {sp->sgd_beta, sp->sgd_min};
    sig = fnv(sig, ints, sizeof(ints));
    sig = fnv(sig, ptrs2, sizeof(ptrs2));
    sig = fnv(sig, sgdf, sizeof(sgdf));
    sig = fnv(sig, &pr->lambda, sizeof(float));
    sig = fnv(sig, &sp->step, sizeof(float));
    if (tvreg) {
        const int tvi[] = {pd.M};
        const float tvf[] = {pd.tau, pd.sigma};
        sig = fnv(sig, tvi, sizeof(tvi));
        sig = fnv(sig, tvf, sizeof(tvf));
    }
    sig = fnv(sig, &sp->seed, sizeof(uint64_t));
    sig = fnv(sig, &p->layout_gen, sizeof(uint64_t));     // sample order, records, gridding launches
    {
        const void* tp[] = {sp->warm, sp->x_ref};
        const int ti[] = {(int)tracing, (int)trace_obj};
        sig = fnv(sig, tp, sizeof(tp));
        sig = fnv(sig, ti, sizeof(ti));
        sig = fnv(sig, &wgen, sizeof(wgen));
    }
    const int g = vec_grid(D);
    float2* iters = (float2*)sp->iterates;

    if (sketch) {
        const float* sk = sp->sketches;
        if (!sk && S > 0) {
            CS_PROPAGATE(sketch_draw_impl(sp->seed, 0, T + init, C, V, S, sp->dist, sp->norm, ws->skd, st));
            sk = ws->skd;
        }
        float2* msk = ws->msk;
        if (init) {
            // S^0 A and S^0 y: block T of the sketch array, V rows in place + S combinations
            set_int_kernel<<<1, 32, 0, st>>>(ws->tinit, T);
            CS_LAUNCH_CHECK();
            if (S > 0) {
                CS_PROPAGATE(sketched_maps_impl(sk, ws->tinit, maps, D, C, V, S, sp->precision, msk, st));
                CS_PROPAGATE(sketched_maps_impl(sk, ws->tinit, y, N, C, V, S, sp->precision, ws->ysk, st));
            }
        }
        if (fista && !(sp->step > 0) && T + init > 0) {
            // FISTA step from the first sketched model (the initialisation's when there is one),
            // reused by every sub-problem
            CS_REQUIRE(sp->power_v0 != nullptr, CS_ERR_INVALID_ARG, "power_v0 is required when step == 0");
            if (S > 0 && !init) CS_PROPAGATE(sketched_maps_impl(sk, ws->tdev, maps, D, C, V, S, sp->precision, msk, st));
            CS_PROPAGATE(power_iteration(c, (const float2*)sp->power_v0, sp->power_iters > 0 ? sp->power_iters : 20,
                                         maps, V, msk, S, ws->u, ws->hp));
            if (pso > 0) CS_TRY_CUDA(cudaMemcpyAsync(ws->peig, ws->u, sizeof(float2) * D, cudaMemcpyDeviceToDevice, st));
        }
        if (init) {
            // argmin 1/2 ||S^0 A x - S^0 y||^2 + g(x) from x^0: the sub-problem at x^t = x^0 with
            // the sketched gradient d = (S^0 A)^H (S^0 A x^0 - S^0 y)
            if (V > 0) CS_PROPAGATE((cs_status)sense_grad(p, (const float*)x, (const float*)maps, V, (const float*)y,
                                                          (float*)ws->d, st));
            if (S > 0) {
                float2* dst = (V > 0) ? ws->hp : ws->d;
                CS_PROPAGATE((cs_status)sense_grad(p, (const float*)x, (const float*)msk, S, (const float*)ws->ysk,
                                                   (float*)dst, st));
                if (V > 0) {
                    add_inplace_kernel<<<g, kRedThreads, 0, st>>>(ws->d, ws->hp, D);
                    CS_LAUNCH_CHECK();
                }
            }
            if (fista) CS_PROPAGATE(fista_sub(c, ws->d, x, K, maps, V, msk, S, theta, ws->z, ws->xp, ws->u, ws->gr, ws->xt));
            else if (tvreg) CS_PROPAGATE(pdhg_sub(c, ws->d, x, maps, V, msk, S, pd));
            else CS_PROPAGATE(cg_sub(c, ws->d, x, K, maps, V, msk, S, ws->r, ws->pv, ws->hp));
        }
        auto body = [&](cudaStream_t s) -> cs_status {
            Ctx cc = c;
            cc.st = s;
            if (trace_obj) CS_PROPAGATE(trace_objective(s, x, maps, C, y, ws->u));
            // true gradient with all C coils
            CS_PROPAGATE((cs_status)sense_grad(p, (const float*)x, (const float*)maps, C, (const float*)y, (float*)ws->d, s));
            if (tracing) CS_PROPAGATE(trace_norm2(s, ws->d, CS_TRACE_GRAD2));
            // sketched model: V virtual coils in place + S random combinations of the rest
            if (S > 0) CS_PROPAGATE(sketched_maps_impl(sk, ws->tdev, maps, D, C, V, S, sp->precision, msk, s));
            if (pso > 0) {
                CS_PROPAGATE(power_iteration(cc, ws->peig, pso, maps, V, msk, S, ws->u, ws->hp));
                CS_TRY_CUDA(cudaMemcpyAsync(ws->peig, ws->u, sizeof(float2) * D, cudaMemcpyDeviceToDevice, s));
            }
            if (fista && warm) {
                // learned warm start: prediction xhat from (x^t, d); the sub-problem objective of
                // Eq. 9-10, F(u) = 1/2 ||A_S (u - x^t)||^2 + Re<u, d> + lambda ||Psi u||_1, at xhat
                // and at x^t decides on the device which one FISTA starts from
                CS_TRY_CUDA(cudaMemcpyAsync(ws->xt0, x, sizeof(float2) * D, cudaMemcpyDeviceToDevice, s));
                CS_PROPAGATE(unet_infer_dev(sp->warm, ws->xt0, ws->d, p->img, &ws->sc->eta, ws->xhat, s));
                sub_kernel<<<g, kRedThreads, 0, s>>>(ws->xhat, ws->xt0, D, ws->z);
                CS_LAUNCH_CHECK();
                CS_PROPAGATE(normal_apply(cc, ws->z, maps, V, msk, S, 0.f, ws->hp));
                dot_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(ws->z, ws->hp, D, ws->partA);
                CS_LAUNCH_CHECK();
                dot_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(ws->xhat, ws->d, D, ws->partB);
                CS_LAUNCH_CHECK();
                CS_TRY_CUDA(cudaMemcpyAsync(ws->u, ws->xhat, sizeof(float2) * D, cudaMemcpyDeviceToDevice, s));
                CS_PROPAGATE(wavelet_apply(ws->u, c.dims3, c.nd, c.levels, 0, s));
                l1_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(ws->u, D, ws->partC);
                CS_LAUNCH_CHECK();
                subobj_kernel<<<1, 32, 0, s>>>(ws->partA, ws->partB, ws->partC, (double)c.lambda, &ws->sc->fhat);
                CS_LAUNCH_CHECK();
                dot_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(ws->xt0, ws->d, D, ws->partB);
                CS_LAUNCH_CHECK();
                CS_TRY_CUDA(cudaMemcpyAsync(ws->u, ws->xt0, sizeof(float2) * D, cudaMemcpyDeviceToDevice, s));
                CS_PROPAGATE(wavelet_apply(ws->u, c.dims3, c.nd, c.levels, 0, s));
                l1_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(ws->u, D, ws->partC);
                CS_LAUNCH_CHECK();
                subobj_kernel<<<1, 32, 0, s>>>(nullptr, ws->partB, ws->partC, (double)c.lambda, &ws->sc->ft);
                CS_LAUNCH_CHECK();
                warm_select_kernel<<<g, kRedThreads, 0, s>>>(ws->sc, ws->xhat, x, D, tracing ? ws->trace : nullptr,
                                                             ws->tdev);
                CS_LAUNCH_CHECK();
                CS_PROPAGATE(fista_sub(cc, ws->d, x, K, maps, V, msk, S, theta, ws->z, ws->xp, ws->u, ws->gr, ws->xt,
                                       ws->xt0));
            } else if (fista) {
                CS_PROPAGATE(fista_sub(cc, ws->d, x, K, maps, V, msk, S, theta, ws->z, ws->xp, ws->u, ws->gr, ws->xt));
            } else if (tvreg) {
                CS_PROPAGATE(pdhg_sub(cc, ws->d, x, maps, V, msk, S, pd));
            } else {
                CS_PROPAGATE(cg_sub(cc, ws->d, x, K, maps, V, msk, S, ws->r, ws->pv, ws->hp));
            }
            if (tracing) CS_PROPAGATE(trace_end(s));
            if (iters) {
                copy_iter_kernel<<<g, kRedThreads, 0, s>>>(x, iters, ws->tdev, 0, D);
                CS_LAUNCH_CHECK();
            }
            inc_kernel<<<1, 32, 0, s>>>(ws->tdev);
            CS_LAUNCH_CHECK();
            return CS_OK;
        };
        CS_PROPAGATE(run_body(ws, use_graph, sig, T, st, body, &graph_used));
    } else if (tvreg) {
        // plain full-coil l1-TV: K PDHG iterations in total, each with M CG iterations on the
        // full normal operator; b0 = A^H y
        CS_PROPAGATE((cs_status)sense_adj(p, (const float*)y, (const float*)maps, Cp, (float*)ws->d, 0, st));
        pd.b0 = ws->d;
        pd.K = 1;
        CS_TRY_CUDA(cudaMemcpyAsync(ws->xp, x, sizeof(float2) * D, cudaMemcpyDeviceToDevice, st));
        const TvDims tvd = tv_dims(c.nd, c.dims3);
        auto body = [&](cudaStream_t s) -> cs_status {
            Ctx cc = c;
            cc.st = s;
            cc.lambda = 1.0f / pd.tau;
            tv_dual_kernel<<<tv_grid(tvd), 128, 0, s>>>(x, ws->xp, pd.zd, tvd, pd.sigma, pd.lam_tv);
            CS_LAUNCH_CHECK();
            tv_rhs_kernel<<<tv_grid(tvd), 128, 0, s>>>(pd.b0, x, pd.zd, tvd, cc.lambda, pd.rhs, ws->xp);
            CS_LAUNCH_CHECK();
            CS_PROPAGATE(normal_apply(cc, x, maps, Cp, nullptr, 0, cc.lambda, ws->hp));
            cg_init2_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(pd.rhs, ws->hp, D, ws->r, ws->pv, c.partB);
            CS_LAUNCH_CHECK();
            store_sum_kernel<<<1, 32, 0, s>>>(c.partB, &c.sc->rr[0]);
            CS_LAUNCH_CHECK();
            for (int m = 0; m < pd.M; ++m) CS_PROPAGATE(cg_iter(cc, maps, Cp, nullptr, 0, x, ws->r, ws->pv, ws->hp, m & 1, nullptr));
            if (tracing) CS_PROPAGATE(trace_end(s));
            if (iters) {
                copy_iter_kernel<<<g, kRedThreads, 0, s>>>(x, iters, ws->tdev, 0, D);
                CS_LAUNCH_CHECK();
            }
            inc_kernel<<<1, 32, 0, s>>>(ws->tdev);
            CS_LAUNCH_CHECK();
            return CS_OK;
        };
        CS_PROPAGATE(run_body(ws, use_graph, sig, K, st, body, &graph_used));
    } else if (sgd) {
        // AccProxSGD (plain problem, l1-wavelets): per iteration a batch of B coils (given indices),
        // unbiased batch gradient (Cp/B) sum_batch A_c^H (A_c z - y_c), step alpha_k =
        // max(beta^k alpha_0, min alpha_0) with alpha_0 = 1/L of the full-coil normal operator,
        // proximal step and Nesterov (FISTA) momentum
        const int B = sp->sgd_batch;
        CS_PROPAGATE(ws->ensure_sgd((int64_t)B * D, (int64_t)B * N));
        if (sp->step > 0) {
            set_L_kernel<<<1, 32, 0, st>>>(ws->sc, 1.0 / (double)sp->step);
            CS_LAUNCH_CHECK();
        } else {
            CS_REQUIRE(sp->power_v0 != nullptr, CS_ERR_INVALID_ARG, "power_v0 is required when step == 0");
            CS_PROPAGATE(power_iteration(c, (const float2*)sp->power_v0, sp->power_iters > 0 ? sp->power_iters : 20,
                                         maps, Cp, nullptr, 0, ws->u, ws->hp));
        }
        theta_kernel<<<1, 32, 0, st>>>(ws->theta, std::max(K, 1));
        CS_LAUNCH_CHECK();
        CS_TRY_CUDA(cudaMemcpyAsync(ws->z, x, sizeof(float2) * D, cudaMemcpyDeviceToDevice, st));
        CS_TRY_CUDA(cudaMemcpyAsync(ws->xp, x, sizeof(float2) * D, cudaMemcpyDeviceToDevice, st));
        const double beta = sp->sgd_beta > 0 ? sp->sgd_beta : 0.99;
        const double minf = sp->sgd_min > 0 ? sp->sgd_min : 0.1;
        const float ratio = (float)Cp / (float)B;
        auto body = [&](cudaStream_t s) -> cs_status {
            Ctx cc = c;
            cc.st = s;
            const dim3 gg((unsigned)std::min<int64_t>(kRedBlocks, (std::max(D, N) + kRedThreads - 1) / kRedThreads),
                          (unsigned)B);
            gather_coils_kernel<<<gg, kRedThreads, 0, s>>>(maps, D, sp->sgd_coils, B, ws->tdev, ws->bmaps);
            CS_LAUNCH_CHECK();
            gather_coils_kernel<<<gg, kRedThreads, 0, s>>>(y, N, sp->sgd_coils, B, ws->tdev, ws->by);
            CS_LAUNCH_CHECK();
            if (trace_obj) CS_PROPAGATE(trace_objective(s, ws->z, maps, Cp, y, ws->hp));
            CS_PROPAGATE((cs_status)sense_grad(p, (const float*)ws->z, (const float*)ws->bmaps, B, (const float*)ws->by,
                                               (float*)ws->gr, s));
            if (tracing) CS_PROPAGATE(trace_norm2(s, ws->gr, CS_TRACE_GRAD2));
            sgd_step_kernel<<<g, kRedThreads, 0, s>>>(ws->z, ws->gr, c.sc, ws->tdev, beta, minf, ratio, D, ws->u);
            CS_LAUNCH_CHECK();
            CS_PROPAGATE(prox_wavelet(cc, ws->u, x, c.sc, 0.f));
            momentum_kernel<<<g, kRedThreads, 0, s>>>(x, ws->xp, 0.f, ws->theta, ws->tdev, D, ws->z);
            CS_LAUNCH_CHECK();
            CS_TRY_CUDA(cudaMemcpyAsync(ws->xp, x, sizeof(float2) * D, cudaMemcpyDeviceToDevice, s));
            if (tracing) CS_PROPAGATE(trace_end(s));
            if (iters) {
                copy_iter_kernel<<<g, kRedThreads, 0, s>>>(x, iters, ws->tdev, 0, D);
                CS_LAUNCH_CHECK();
            }
            inc_kernel<<<1, 32, 0, s>>>(ws->tdev);
            CS_LAUNCH_CHECK();
            return CS_OK;
        };
        CS_PROPAGATE(run_body(ws, use_graph, sig, K, st, body, &graph_used));
    } else if (fista) {
        // plain full-coil FISTA: K iterations in total
        if (!(sp->step > 0)) {
            CS_REQUIRE(sp->power_v0 != nullptr, CS_ERR_INVALID_ARG, "power_v0 is required when step == 0");
            CS_PROPAGATE(power_iteration(c, (const float2*)sp->power_v0, sp->power_iters > 0 ? sp->power_iters : 20,
                                         maps, Cp, nullptr, 0, ws->u, ws->hp));
        }
        theta_kernel<<<1, 32, 0, st>>>(ws->theta, std::max(K, 1));
        CS_LAUNCH_CHECK();
        CS_TRY_CUDA(cudaMemcpyAsync(ws->z, x, sizeof(float2) * D, cudaMemcpyDeviceToDevice, st));
        CS_TRY_CUDA(cudaMemcpyAsync(ws->xp, x, sizeof(float2) * D, cudaMemcpyDeviceToDevice, st));
        auto body = [&](cudaStream_t s) -> cs_status {
            Ctx cc = c;
            cc.st = s;
            if (trace_obj) CS_PROPAGATE(trace_objective(s, ws->z, maps, Cp, y, ws->hp));
            CS_PROPAGATE((cs_status)sense_grad(p, (const float*)ws->z, (const float*)maps, Cp, (const float*)y, (float*)ws->gr, s));
            if (tracing) CS_PROPAGATE(trace_norm2(s, ws->gr, CS_TRACE_GRAD2));
            fista_step_kernel<<<g, kRedThreads, 0, s>>>(ws->z, ws->gr, nullptr, c.sc, D, ws->u);
            CS_LAUNCH_CHECK();
            CS_PROPAGATE(prox_wavelet(cc, ws->u, x, c.sc, 0.f));
            momentum_kernel<<<g, kRedThreads, 0, s>>>(x, ws->xp, 0.f, ws->theta, ws->tdev, D, ws->z);
            CS_LAUNCH_CHECK();
            CS_TRY_CUDA(cudaMemcpyAsync(ws->xp, x, sizeof(float2) * D, cudaMemcpyDeviceToDevice, s));
            if (tracing) CS_PROPAGATE(trace_end(s));
            if (iters) {
                copy_iter_kernel<<<g, kRedThreads, 0, s>>>(x, iters, ws->tdev, 0, D);
                CS_LAUNCH_CHECK();
            }
            inc_kernel<<<1, 32, 0, s>>>(ws->tdev);
            CS_LAUNCH_CHECK();
            return CS_OK;
        };
        CS_PROPAGATE(run_body(ws, use_graph, sig, K, st, body, &graph_used));
    } else {
        // plain full-coil CG: (A^H A + lambda I) x = A^H y from x, K iterations in total
        CS_PROPAGATE((cs_status)sense_adj(p, (const float*)y, (const float*)maps, Cp, (float*)ws->d, 0, st));   // b
        CS_PROPAGATE(normal_apply(c, x, maps, Cp, nullptr, 0, c.lambda, ws->hp));                            // H x
        cg_init2_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(ws->d, ws->hp, D, ws->r, ws->pv, c.partB);
        CS_LAUNCH_CHECK();
        store_sum_kernel<<<1, 32, 0, st>>>(c.partB, &c.sc->rr[0]);
        CS_LAUNCH_CHECK();
        auto body = [&](cudaStream_t s) -> cs_status {
            Ctx cc = c;
            cc.st = s;
            CS_PROPAGATE(cg_iter(cc, maps, Cp, nullptr, 0, x, ws->r, ws->pv, ws->hp, 0, ws->tdev));
            if (tracing) {
                CS_PROPAGATE(trace_norm2(s, ws->r, CS_TRACE_GRAD2));
                CS_PROPAGATE(trace_end(s));
            }
            if (iters) {
                copy_iter_kernel<<<g, kRedThreads, 0, s>>>(x, iters, ws->tdev, 0, D);
                CS_LAUNCH_CHECK();
            }
            inc_kernel<<<1, 32, 0, s>>>(ws->tdev);
            CS_LAUNCH_CHECK();
            return CS_OK;
        };
        CS_PROPAGATE(run_body(ws, use_graph, sig, K, st, body, &graph_used));
    }
    if (ev) {
        CS_TRY_CUDA(cudaEventRecord(ev->e2, st));
        ev->graph_used = graph_used;
    }
    return CS_OK;
}

// Synchronise, fill stats, report non-finite reductions and tensor-core timeouts.
static cs_status recon_finish(cs_plan* p, const cs_solve_params* sp, cudaStream_t st, SolveEvents* ev, cs_stats* stats) {
    SolverWS* ws = static_cast<SolverWS*>(p->solver_ws);
    CS_TRY_CUDA(cudaStreamSynchronize(st));
    Scal h;
    CS_TRY_CUDA(cudaMemcpy(&h, ws->sc, sizeof(Scal), cudaMemcpyDeviceToHost));
    if (stats) {
        float ms_all = 0, ms_pca = 0;
        if (ev && ev->e0) {
            cudaEventElapsedTime(&ms_all, ev->e0, ev->e2);
            cudaEventElapsedTime(&ms_pca, ev->e0, ev->e1);
        }
        stats->L = h.L;
        stats->final_rr = h.rr[sp->K & 1];
        stats->outer_done = sp->sketch ? sp->T : 0;
        stats->graph_used = ev ? ev->graph_used : 0;
        stats->ms_total = ms_all;
        stats->ms_pca = ms_pca;
        stats->warm_accepted = h.naccept;
    }
    if (sp->trace && ws->trace) {
        const int rows = sp->sketch ? sp->T : sp->K;
        CS_TRY_CUDA(cudaMemcpy(sp->trace, ws->trace, sizeof(double) * CS_TRACE_FIELDS * rows, cudaMemcpyDeviceToHost));
    }
    CS_PROPAGATE(fft_check_and_clear());
    CS_PROPAGATE(tc_check_and_clear());
    CS_PROPAGATE(bounds_check_all());
    CS_REQUIRE(!h.nonfinite, CS_ERR_NONFINITE, "a solver reduction produced a non-finite value");
    return CS_OK;
}

static cs_status recon_solve_impl(cs_plan* p, const cs_problem* pr, const cs_solve_params* sp, float2* x,
                                  cs_stats* stats, cudaStream_t st) {
    SolveEvents ev;
    CS_PROPAGATE(recon_enqueue(p, pr, sp, x, st, true, &ev));
    return recon_finish(p, sp, st, &ev, stats);
}

// ------------------------------------------------------------------------------------------
// Batched independent solves (many slices of uneven size): every slice has its own plan and
// workspace; the solves are forked onto a pool of streams and joined, either launched directly
// or captured once - all slices in one CUDA graph - cached and replayed.
struct BatchCache {
    std::vector<cudaStream_t> pool;
    cudaStream_t cap = nullptr;
    std::vector<cudaEvent_t> evs;
    cudaGraphExec_t gexec = nullptr;
    uint64_t sig = 0;
};

static BatchCache& batch_cache() {
    static BatchCache bc;
    return bc;
}

static cs_status batch_streams(BatchCache& bc, int n) {
    while ((int)bc.pool.size() < n) {
        cudaStream_t s = nullptr;
        CS_TRY_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        bc.pool.push_back(s);
    }
    while ((int)bc.evs.size() < 2 * n + 2) {
        cudaEvent_t e = nullptr;
        CS_TRY_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        bc.evs.push_back(e);
    }
    if (!bc.cap) CS_TRY_CUDA(cudaStreamCreateWithFlags(&bc.cap, cudaStreamNonBlocking));
    return CS_OK;
}

// fork: every branch waits for `root`; join: root waits for every branch
static cs_status batch_enqueue(BatchCache& bc, int n, const cs_batch_item* items, const cs_solve_params* sp,
                               cudaStream_t root) {
    const int nb = std::min(n, 32);
    CS_TRY_CUDA(cudaEventRecord(bc.evs[0], root));
    for (int b = 0; b < nb; ++b) CS_TRY_CUDA(cudaStreamWaitEvent(bc.pool[b], bc.evs[0], 0));
    for (int i = 0; i < n; ++i) {
        const cs_batch_item& it = items[i];
        cs_solve_params one = *sp;
        one.power_v0 = it.power_v0;
        CS_PROPAGATE(recon_enqueue(it.plan, &it.problem, &one, (float2*)it.x_inout, bc.pool[i % nb], false, nullptr));
    }
    for (int b = 0; b < nb; ++b) {
        CS_TRY_CUDA(cudaEventRecord(bc.evs[1 + b], bc.pool[b]));
        CS_TRY_CUDA(cudaStreamWaitEvent(root, bc.evs[1 + b], 0));
    }
    return CS_OK;
}

static cs_status recon_batched_impl(int n, const cs_batch_item* items, const cs_solve_params* sp, cs_stats* stats,
                                    cudaStream_t st) {
    BatchCache& bc = batch_cache();
    CS_PROPAGATE(batch_streams(bc, std::min(n, 32)));
    // make sure every slice's workspace exists before any capture (allocation is not capturable)
    for (int i = 0; i < n; ++i) {
        cs_plan* p = items[i].plan;
        const int C = items[i].problem.C;
        const int V = sp->sketch ? sp->V : C, S = sp->sketch ? sp->S : 0;
        if (!p->solver_ws) p->solver_ws = new SolverWS();
        CS_PROPAGATE(static_cast<SolverWS*>(p->solver_ws)->ensure(p->D, p->N, C, S, C - V, sp->T, sp->K));
    }
    int graph_used = 0;
    if (sp->use_graph) {
        uint64_t sig = 1469598103934665603ull;
        sig = fnv(sig, items, sizeof(cs_batch_item) * n);
        sig = fnv(sig, sp, sizeof(cs_solve_params));
        for (int i = 0; i < n; ++i) sig = fnv(sig, &items[i].plan->layout_gen, sizeof(uint64_t));
        if (!bc.gexec || bc.sig != sig) {
            if (bc.gexec) cudaGraphExecDestroy(bc.gexec);
            bc.gexec = nullptr;
            CS_TRY_CUDA(cudaStreamBeginCapture(bc.cap, cudaStreamCaptureModeThreadLocal));
            cs_status rc = batch_enqueue(bc, n, items, sp, bc.cap);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(bc.cap, &g);
            if (rc != CS_OK) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (e != cudaSuccess) {
                set_error("batched graph capture failed: %s", cudaGetErrorString(e));
                return CS_ERR_CUDA;
            }
            e = cudaGraphInstantiate(&bc.gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                bc.gexec = nullptr;
                set_error("batched graph instantiation failed: %s", cudaGetErrorString(e));
                return CS_ERR_CUDA;
            }
            bc.sig = sig;
        }
        CS_TRY_CUDA(cudaGraphLaunch(bc.gexec, st));
        graph_used = 1;
    } else {
        CS_PROPAGATE(batch_enqueue(bc, n, items, sp, st));
    }
    CS_TRY_CUDA(cudaStreamSynchronize(st));
    cs_status worst = CS_OK;
    for (int i = 0; i < n; ++i) {
        cs_stats one = {};
        cs_status rc = recon_finish(items[i].plan, sp, st, nullptr, &one);
        if (rc != CS_OK && worst == CS_OK) worst = rc;
        if (stats) {
            stats[i] = one;
            stats[i].graph_used = graph_used;
        }
    }
    return worst;
}

}  // namespace cs

using namespace cs;

extern "C" {

cs_status recon_solve(const cs_plan* p, const cs_problem* pr, const cs_solve_params* sp, float* x_inout,
                      cs_stats* stats, void* stream) {
    clear_error();
    CS_REQUIRE(p && pr && sp && x_inout, CS_ERR_INVALID_ARG, "null argument");
    CS_REQUIRE(pr->y && pr->maps && pr->C >= 1 && pr->C <= p->max_coils, CS_ERR_INVALID_ARG,
               "problem needs y, maps and 1 <= C <= max_coils");
    CS_REQUIRE(std::isfinite(pr->lambda) && pr->lambda >= 0, CS_ERR_INVALID_ARG, "lambda must be finite and >= 0");
    CS_REQUIRE(pr->reg == CS_REG_L2 || pr->reg == CS_REG_L1_WAVELET || pr->reg == CS_REG_L1_TV, CS_ERR_INVALID_ARG,
               "bad regulariser");
    CS_REQUIRE(sp->K >= 0 && sp->T >= 0 && sp->cg_iters >= 0, CS_ERR_INVALID_ARG, "negative iteration count");
    CS_REQUIRE(std::isfinite(sp->tv_tau) && sp->tv_tau >= 0 && std::isfinite(sp->tv_sigma) && sp->tv_sigma >= 0,
               CS_ERR_INVALID_ARG, "PDHG steps must be finite and >= 0 (0 = default)");
    if (sp->sketch) {
        CS_REQUIRE(sp->V >= 0 && sp->S >= 0 && sp->V + sp->S <= pr->C && sp->V + sp->S >= 1, CS_ERR_INVALID_ARG,
                   "need 1 <= V + S <= C (V=%d S=%d C=%d)", sp->V, sp->S, pr->C);
        CS_REQUIRE(sp->S == 0 || sp->V < pr->C, CS_ERR_INVALID_ARG, "S > 0 needs V < C");
    }
    CS_REQUIRE(sp->keep >= 0 && sp->sgd_batch >= 0, CS_ERR_INVALID_ARG, "keep and sgd_batch must be >= 0");
    if (!sp->sketch && sp->sgd_batch > 0) {
        const int Cp = sp->keep > 0 ? std::min(sp->keep, pr->C) : pr->C;
        CS_REQUIRE(pr->reg == CS_REG_L1_WAVELET, CS_ERR_INVALID_ARG, "AccProxSGD is implemented for l1-wavelets");
        CS_REQUIRE(sp->sgd_batch <= Cp && sp->sgd_coils != nullptr, CS_ERR_INVALID_ARG,
                   "AccProxSGD needs 1 <= sgd_batch <= coils and the coil index array");
        CS_REQUIRE(std::isfinite(sp->sgd_beta) && sp->sgd_beta >= 0 && sp->sgd_beta <= 1 && std::isfinite(sp->sgd_min) &&
                       sp->sgd_min >= 0 && sp->sgd_min <= 1,
                   CS_ERR_INVALID_ARG, "sgd_beta and sgd_min must lie in [0, 1]");
        // every batch index must name one of the Cp coils (checked on the host before anything runs)
        std::vector<int> h((size_t)sp->K * sp->sgd_batch);
        if (!h.empty()) {
            CS_TRY_CUDA(cudaMemcpy(h.data(), sp->sgd_coils, sizeof(int) * h.size(), cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < h.size(); ++i)
                CS_REQUIRE(h[i] >= 0 && h[i] < Cp, CS_ERR_INVALID_ARG, "sgd_coils[%zu] = %d outside [0, %d)", i, h[i], Cp);
        }
    }
    CS_REQUIRE(sp->trace_objective == 0 || sp->trace_objective == 1, CS_ERR_INVALID_ARG, "trace_objective is 0 or 1");
    CS_REQUIRE(!sp->trace || (sp->sketch ? sp->T : sp->K) >= 1, CS_ERR_INVALID_ARG, "a trace needs iterations");
    return recon_solve_impl(const_cast<cs_plan*>(p), pr, sp, (float2*)x_inout, stats, (cudaStream_t)stream);
}

cs_status recon_solve_batched(int nslices, const cs_batch_item* items, const cs_solve_params* params, cs_stats* stats,
                              void* stream) {
    clear_error();
    CS_REQUIRE(nslices >= 1 && items && params, CS_ERR_INVALID_ARG, "bad batched solve arguments");
    CS_REQUIRE(!params->warm && !params->trace && !params->x_ref, CS_ERR_INVALID_ARG,
               "batched solves take no warm start, trace or reference");
    for (int i = 0; i < nslices; ++i) {
        const cs_batch_item& it = items[i];
        CS_REQUIRE(it.plan && it.x_inout && it.problem.y && it.problem.maps && it.problem.C >= 1 &&
                       it.problem.C <= it.plan->max_coils,
                   CS_ERR_INVALID_ARG, "batch item %d: bad plan/problem", i);
        for (int j = 0; j < i; ++j)
            CS_REQUIRE(items[j].plan != it.plan, CS_ERR_INVALID_ARG, "batch items %d and %d share a plan", j, i);
    }
    if (params->sketch) {
        CS_REQUIRE(params->V >= 0 && params->S >= 0 && params->V + params->S >= 1, CS_ERR_INVALID_ARG, "bad V/S");
        for (int i = 0; i < nslices; ++i)
            CS_REQUIRE(params->V + params->S <= items[i].problem.C, CS_ERR_INVALID_ARG, "V + S > C in item %d", i);
        CS_REQUIRE(params->sketches == nullptr, CS_ERR_INVALID_ARG, "batched solves draw their own sketches");
    }
    CS_REQUIRE(params->iterates == nullptr, CS_ERR_INVALID_ARG, "batched solves do not record iterates");
    CS_REQUIRE(params->sgd_batch == 0, CS_ERR_INVALID_ARG, "batched solves do not run AccProxSGD");
    return recon_batched_impl(nslices, items, params, stats, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------------------------
// Pseudo-replica noise statistics (the inverse g-factor of Sec. 3.2): per pixel, in FP64 and in
// replica order, std = sqrt(mean_k |x_k - mean|^2); 1/g = std_full sqrt(R) / std_R.
__device__ __forceinline__ double replica_std(const float2* __restrict__ x, int K, int64_t D, int64_t i) {
    double mr = 0, mi = 0;
    for (int k = 0; k < K; ++k) {
        const float2 v = x[(int64_t)k * D + i];
        mr += v.x;
        mi += v.y;
    }
    mr /= K;
    mi /= K;
    double acc = 0;
    for (int k = 0; k < K; ++k) {
        const float2 v = x[(int64_t)k * D + i];
        const double dr = v.x - mr, di = v.y - mi;
        acc += dr * dr + di * di;
    }
    return sqrt(acc / K);
}

__global__ void noise_std_kernel(const float2* __restrict__ x, int K, int64_t D, float* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)replica_std(x, K, D, i);
}

__global__ void inv_gfactor_kernel(const float2* __restrict__ xr, const float2* __restrict__ xf, int K, int64_t D,
                                   double sqrtR, float* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)(replica_std(xf, K, D, i) * sqrtR / replica_std(xr, K, D, i));
}

// ---------------------------------------------------------------------------------------------
// Sub-problem pieces for callers that drive Algorithm 1 themselves (e.g. with a warm start).

static cs_status make_ctx(cs_plan* p, float lambda, int levels, cudaStream_t st, Ctx& c, SolverWS*& ws, int C, int S, int K) {
    if (!p->solver_ws) p->solver_ws = new SolverWS();
    ws = static_cast<SolverWS*>(p->solver_ws);
    CS_PROPAGATE(ws->ensure(p->D, p->N, C, S, std::max(C - 1, 1), 1, std::max(K, 1)));
    c.p = p;
    c.st = st;
    c.D = p->D;
    c.nd = p->ndim;
    for (int a = 0; a < 3; ++a) c.dims3[a] = p->img[a];
    c.levels = levels > 0 ? levels : 4;
    c.lambda = lambda;
    c.sc = ws->sc;
    c.partA = ws->partA;
    c.partB = ws->partB;
    return CS_OK;
}

cs_status sketched_subproblem_solve(const cs_plan* plan, const float* d, const float* xt, float* x_inout,
                                    const float* maps_v, int V, const float* maps_s, int S, float lambda, int reg,
                                    int wavelet_levels, int K, float step, void* stream) {
    clear_error();
    CS_REQUIRE(plan && d && xt && x_inout && K >= 0 && V >= 0 && S >= 0 && V + S >= 1 && V + S <= plan->max_coils,
               CS_ERR_INVALID_ARG, "bad sub-problem arguments");
    CS_REQUIRE(reg == CS_REG_L2 || step > 0, CS_ERR_INVALID_ARG, "FISTA needs a step > 0");
    cs_plan* p = const_cast<cs_plan*>(plan);
    cudaStream_t st = (cudaStream_t)stream;
    Ctx c;
    SolverWS* ws = nullptr;
    CS_PROPAGATE(make_ctx(p, lambda, wavelet_levels, st, c, ws, V + S, S, K));
    CS_TRY_CUDA(cudaMemsetAsync(ws->sc, 0, sizeof(Scal), st));
    const float2* mv = (const float2*)maps_v;
    const float2* ms = (const float2*)maps_s;
    float2* x = (float2*)x_inout;
    const bool same = (const float*)x_inout == xt;
    if (reg == CS_REG_L2) {
        CS_PROPAGATE(cg_sub(c, (const float2*)d, x, K, mv, V, ms, S, ws->r, ws->pv, ws->hp,
                            same ? nullptr : (const float2*)xt, ws->u));
    } else {
        set_eta_kernel<<<1, 32, 0, st>>>(ws->sc, (double)step);
        CS_LAUNCH_CHECK();
        const std::vector<float> theta = fista_thetas(std::max(K, 1));
        CS_PROPAGATE(fista_sub(c, (const float2*)d, x, K, mv, V, ms, S, theta, ws->z, ws->xp, ws->u, ws->gr, ws->xt,
                               same ? nullptr : (const float2*)xt));
    }
    return CS_OK;
}

// F(u) = 1/2 ||A_S (u - x^t)||^2 + Re<u, d> + g(u), g = lambda/2 ||u||^2 or lambda ||Psi u||_1 (Eq. 9-10)
cs_status cs_subproblem_objective(const cs_plan* plan, const float* u, const float* xt, const float* d, const float* maps_v,
                                  int V, const float* maps_s, int S, float lambda, int reg, int wavelet_levels,
                                  double* value, void* stream) {
    clear_error();
    CS_REQUIRE(plan && u && xt && d && value && V + S >= 1, CS_ERR_INVALID_ARG, "bad objective arguments");
    cs_plan* p = const_cast<cs_plan*>(plan);
    cudaStream_t st = (cudaStream_t)stream;
    Ctx c;
    SolverWS* ws = nullptr;
    CS_PROPAGATE(make_ctx(p, lambda, wavelet_levels, st, c, ws, V + S, S, 1));
    const int64_t D = p->D;
    sub_kernel<<<vec_grid(D), kRedThreads, 0, st>>>((const float2*)u, (const float2*)xt, D, ws->z);
    CS_LAUNCH_CHECK();
    CS_PROPAGATE(normal_apply(c, ws->z, (const float2*)maps_v, V, (const float2*)maps_s, S, 0.f, ws->hp));
    std::vector<double> ha(kRedBlocks), hb(kRedBlocks), hc(kRedBlocks);
    dot_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(ws->z, ws->hp, D, ws->partA);
    CS_LAUNCH_CHECK();
    CS_TRY_CUDA(cudaMemcpyAsync(ha.data(), ws->partA, sizeof(double) * kRedBlocks, cudaMemcpyDeviceToHost, st));
    dot_kernel<<<kRedBlocks, kRedThreads, 0, st>>>((const float2*)u, (const float2*)d, D, ws->partB);
    CS_LAUNCH_CHECK();
    CS_TRY_CUDA(cudaMemcpyAsync(hb.data(), ws->partB, sizeof(double) * kRedBlocks, cudaMemcpyDeviceToHost, st));
    CS_TRY_CUDA(cudaStreamSynchronize(st));
    double quad = 0, lin = 0, reg_v = 0;
    for (int i = 0; i < kRedBlocks; ++i) {
        quad += ha[i];
        lin += hb[i];
    }
    if (reg == CS_REG_L2) {
        dot_kernel<<<kRedBlocks, kRedThreads, 0, st>>>((const float2*)u, (const float2*)u, D, ws->partA);
        CS_LAUNCH_CHECK();
        CS_TRY_CUDA(cudaMemcpyAsync(hc.data(), ws->partA, sizeof(double) * kRedBlocks, cudaMemcpyDeviceToHost, st));
        CS_TRY_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i < kRedBlocks; ++i) reg_v += hc[i];
        reg_v *= 0.5 * lambda;
    } else {
        CS_TRY_CUDA(cudaMemcpyAsync(ws->gr, u, sizeof(float2) * D, cudaMemcpyDeviceToDevice, st));
        CS_PROPAGATE(wavelet_apply(ws->gr, c.dims3, c.nd, c.levels, 0, st));
        l1_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(ws->gr, D, ws->partA);
        CS_LAUNCH_CHECK();
        CS_TRY_CUDA(cudaMemcpyAsync(hc.data(), ws->partA, sizeof(double) * kRedBlocks, cudaMemcpyDeviceToHost, st));
        CS_TRY_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i < kRedBlocks; ++i) reg_v += hc[i];
        reg_v *= lambda;
    }
    *value = 0.5 * quad + lin + reg_v;
    return CS_OK;
}

// largest eigenvalue of A_S^H A_S by power iteration from v0 (synchronises)
cs_status cs_power_iteration(const cs_plan* plan, const float* v0, const float* maps_v, int V, const float* maps_s, int S,
                             int iters, double* L, void* stream) {
    clear_error();
    CS_REQUIRE(plan && v0 && L && V + S >= 1 && iters >= 1, CS_ERR_INVALID_ARG, "bad power iteration arguments");
    cs_plan* p = const_cast<cs_plan*>(plan);
    cudaStream_t st = (cudaStream_t)stream;
    Ctx c;
    SolverWS* ws = nullptr;
    CS_PROPAGATE(make_ctx(p, 0.f, 4, st, c, ws, V + S, S, 1));
    CS_PROPAGATE(power_iteration(c, (const float2*)v0, iters, (const float2*)maps_v, V, (const float2*)maps_s, S, ws->u,
                                 ws->hp));
    Scal h;
    CS_TRY_CUDA(cudaMemcpyAsync(&h, ws->sc, sizeof(Scal), cudaMemcpyDeviceToHost, st));
    CS_TRY_CUDA(cudaStreamSynchronize(st));
    *L = h.L;
    return CS_OK;
}

cs_status cs_noise_std(const float* recons, int K, int64_t D, float* std_out, void* stream) {
    clear_error();
    CS_REQUIRE(recons && std_out && K >= 1 && D >= 0, CS_ERR_INVALID_ARG, "bad noise_std arguments");
    if (D == 0) return CS_OK;
    noise_std_kernel<<<vec_grid(D), kRedThreads, 0, (cudaStream_t)stream>>>((const float2*)recons, K, D, std_out);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

cs_status cs_inverse_gfactor(const float* recons_R, const float* recons_full, int K, int64_t D, float R, float* inv_g,
                             void* stream) {
    clear_error();
    CS_REQUIRE(recons_R && recons_full && inv_g && K >= 1 && D >= 0 && R > 0, CS_ERR_INVALID_ARG,
               "bad inverse g-factor arguments");
    if (D == 0) return CS_OK;
    inv_gfactor_kernel<<<vec_grid(D), kRedThreads, 0, (cudaStream_t)stream>>>(
        (const float2*)recons_R, (const float2*)recons_full, K, D, std::sqrt((double)R), inv_g);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

cs_status wavelet_fwd(const float* x, int ndim, const int* dims, int levels, float* c, void* stream) {
    clear_error();
    CS_REQUIRE(x && c && dims && (ndim == 2 || ndim == 3) && levels >= 1, CS_ERR_INVALID_ARG, "bad wavelet arguments");
    int d3[3] = {1, 1, 1};
    for (int a = 0; a < ndim; ++a) d3[3 - ndim + a] = dims[a];
    const int64_t n = (int64_t)d3[0] * d3[1] * d3[2];
    cudaStream_t st = (cudaStream_t)stream;
    if (c != x) CS_TRY_CUDA(cudaMemcpyAsync(c, x, sizeof(float2) * n, cudaMemcpyDeviceToDevice, st));
    return wavelet_apply((float2*)c, d3, ndim, levels, 0, st);
}

cs_status wavelet_inv(const float* c, int ndim, const int* dims, int levels, float* x, void* stream) {
    clear_error();
    CS_REQUIRE(x && c && dims && (ndim == 2 || ndim == 3) && levels >= 1, CS_ERR_INVALID_ARG, "bad wavelet arguments");
    int d3[3] = {1, 1, 1};
    for (int a = 0; a < ndim; ++a) d3[3 - ndim + a] = dims[a];
    const int64_t n = (int64_t)d3[0] * d3[1] * d3[2];
    cudaStream_t st = (cudaStream_t)stream;
    if (c != x) CS_TRY_CUDA(cudaMemcpyAsync(x, c, sizeof(float2) * n, cudaMemcpyDeviceToDevice, st));
    return wavelet_apply((float2*)x, d3, ndim, levels, 1, st);
}

cs_status soft_threshold(float* z, int64_t n, float tau, void* stream) {
    clear_error();
    CS_REQUIRE(z && n >= 0 && tau >= 0, CS_ERR_INVALID_ARG, "bad soft_threshold arguments");
    if (n == 0) return CS_OK;
    soft_kernel<<<vec_grid(n), kRedThreads, 0, (cudaStream_t)stream>>>((float2*)z, n, 0.f, nullptr, tau);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

static cs_status tv_check(int ndim, const int* dims, TvDims* t) {
    CS_REQUIRE((ndim == 2 || ndim == 3) && dims, CS_ERR_INVALID_ARG, "TV needs ndim 2 or 3 and dims");
    int d3[3] = {1, 1, 1};
    for (int a = 0; a < ndim; ++a) {
        CS_REQUIRE(dims[a] >= 1, CS_ERR_INVALID_ARG, "TV dims must be positive");
        d3[3 - ndim + a] = dims[a];
    }
    *t = tv_dims(ndim, d3);
    CS_REQUIRE(t->D < ((int64_t)1 << 31), CS_ERR_UNSUPPORTED_SIZE, "TV image above 2^31 voxels");
    return CS_OK;
}

cs_status tv_dual_update(const float* x, const float* x_prev, float* z, int ndim, const int* dims, float sigma,
                         float lambda, void* stream) {
    clear_error();
    CS_REQUIRE(x && z, CS_ERR_INVALID_ARG, "null argument");
    CS_REQUIRE(std::isfinite(sigma) && std::isfinite(lambda) && lambda >= 0, CS_ERR_INVALID_ARG, "bad sigma/lambda");
    TvDims t;
    CS_PROPAGATE(tv_check(ndim, dims, &t));
    if (t.D == 0) return CS_OK;
    tv_dual_kernel<<<tv_grid(t), 128, 0, (cudaStream_t)stream>>>((const float2*)x, (const float2*)x_prev, (float2*)z, t,
                                                                   sigma, lambda);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

cs_status tv_rhs(const float* b0, const float* x, const float* z, int ndim, const int* dims, float inv_tau, float* rhs,
                 float* x_prev_out, void* stream) {
    clear_error();
    CS_REQUIRE(x && z && rhs, CS_ERR_INVALID_ARG, "null argument");
    CS_REQUIRE(std::isfinite(inv_tau), CS_ERR_INVALID_ARG, "bad 1/tau");
    TvDims t;
    CS_PROPAGATE(tv_check(ndim, dims, &t));
    if (t.D == 0) return CS_OK;
    tv_rhs_kernel<<<tv_grid(t), 128, 0, (cudaStream_t)stream>>>((const float2*)b0, (const float2*)x, (const float2*)z, t,
                                                                  inv_tau, (float2*)rhs, (float2*)x_prev_out);
    CS_LAUNCH_CHECK();
    return CS_OK;
}

}  // extern "C"
