// Plans and the SENSE operators of the C ABI (Sec. 2.1 and 2.3 of the paper):
//   sense_fwd             y = A x,            A = W^1/2 F C  (Cartesian: F = U F_u, no W)
//   sense_adj             x (+)= A^H y
//   sense_grad            d = A^H (A x - y)   (Algorithm 1, true gradient; residual fused)
//   sketched_normal_apply z = A_S^H A_S v + lambda v with the sketched maps (Eq. 7-8)
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <algorithm>
#include <atomic>
#include <mutex>

#include "cs_internal.cuh"

namespace cs {

static thread_local char g_err[1024] = {0};

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }

// ---- launch counter and stage profiler ----
static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

struct ProfRec {
    int stage;
    cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<cudaEvent_t> g_ev_pool;
static std::vector<ProfRec> g_prof_recs;
static ProfRec g_open[ST_COUNT];
static double g_prof_ms[ST_COUNT];
static long long g_prof_n[ST_COUNT];

bool profiling() { return g_prof_on; }

static cudaEvent_t ev_get() {
    if (!g_ev_pool.empty()) {
        cudaEvent_t e = g_ev_pool.back();
        g_ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

static bool capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    return cs != cudaStreamCaptureStatusNone;
}

void prof_begin(int stage, cudaStream_t st) {
    if (!g_prof_on || capturing(st)) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_open[stage].stage = stage;
    g_open[stage].a = ev_get();
    cudaEventRecord(g_open[stage].a, st);
}

void prof_end(int stage, cudaStream_t st) {
    if (!g_prof_on || capturing(st)) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfRec r = g_open[stage];
    r.b = ev_get();
    cudaEventRecord(r.b, st);
    g_prof_recs.push_back(r);
}

static void prof_drain() {
    for (ProfRec& r : g_prof_recs) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        g_prof_ms[r.stage] += ms;
        g_prof_n[r.stage] += 1;
        g_ev_pool.push_back(r.a);
        g_ev_pool.push_back(r.b);
    }
    g_prof_recs.clear();
}

// Continuous Fourier transform of the width-W Kaiser-Bessel kernel phi(u) = I0(beta sqrt(1 -
// (2u/W)^2)) / I0(beta): W sinh(z)/z / I0(beta), z = sqrt(beta^2 - (pi W nu)^2) (sin past zero).
static double kb_phi_hat(double nu, double beta, double W) {
    const double z2 = beta * beta - (M_PI * W * nu) * (M_PI * W * nu);
    double v;
    if (z2 > 0) {
        const double z = std::sqrt(z2);
        v = std::sinh(z) / z;
    } else if (z2 < 0) {
        const double z = std::sqrt(-z2);
        v = std::sin(z) / z;
    } else {
        v = 1.0;
    }
    return W * v / std::cyl_bessel_i(0.0, beta);
}

__global__ void idxmap_kernel(const int32_t* __restrict__ idx, int64_t N, int32_t* __restrict__ map) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) map[idx[i]] = (int32_t)i;
}

static void plan_free(cs_plan* p) {
    if (!p) return;
    solver_ws_free(p);
    for (int a = 0; a < 3; ++a) {
        fft_len_free(p->fft[a]);
        cudaFree(p->apod[a]);
    }
    cudaFree(p->idxmap);
    cudaFree(p->mask_idx);
    cudaFree(p->gsorted);
    cudaFree(p->wsorted);
    cudaFree(p->perm);
    cudaFree(p->j0);
    cudaFree(p->tile_off);
    cudaFree(p->class_off);
    nufft_owner_free(p);
    cudaFree(p->phi);
    cudaFree(p->rec);
    cudaFree(p->bufA);
    cudaFree(p->bufB);
    cudaFree(p->ktmp);
    delete p;
}

static cs_status device_init_once() {
    static std::mutex mu;
    static bool done[128] = {false};
    int dev = 0;
    CS_TRY_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 128 || done[dev]) return CS_OK;
    CS_PROPAGATE(fft_init_attrs());
    CS_PROPAGATE(tc_init_attrs());
    CS_PROPAGATE(wavelet_init_constants());
    CS_PROPAGATE(coil_init_attrs());
    done[dev] = true;
    return CS_OK;
}

static cs_status plan_build(cs_plan* p, const cs_geom* g, cudaStream_t st) {
    CS_TRY_CUDA(cudaGetDevice(&p->device));
    CS_PROPAGATE(device_init_once());
    const int nd = g->ndim;
    p->kind = g->kind;
    p->ndim = nd;
    p->max_coils = g->max_coils;
    for (int a = 0; a < 3; ++a) {
        p->img[a] = 1;
        p->grid[a] = 1;
    }
    for (int a = 0; a < nd; ++a) {
        p->img[3 - nd + a] = g->img[a];
        p->grid[3 - nd + a] = (g->kind == CS_CARTESIAN) ? g->img[a] : g->grid[a];
    }
    for (int a = 3 - nd; a < 3; ++a) {
        CS_REQUIRE(p->img[a] >= 2 && p->img[a] % 2 == 0, CS_ERR_UNSUPPORTED_SIZE, "image sizes must be even (got %d)", p->img[a]);
        CS_REQUIRE(p->grid[a] >= p->img[a] && p->grid[a] % 2 == 0 && (p->grid[a] - p->img[a]) % 2 == 0,
                   CS_ERR_UNSUPPORTED_SIZE, "grid %d must be even and >= image %d", p->grid[a], p->img[a]);
        p->off[a] = (p->grid[a] - p->img[a]) / 2;
    }
    CS_REQUIRE(p->img[2] <= 512, CS_ERR_UNSUPPORTED_SIZE, "nx above 512 is not supported");
    for (int a = 0; a < 3; ++a)
        CS_REQUIRE(p->grid[a] <= 1023, CS_ERR_UNSUPPORTED_SIZE, "grid size %d above 1023", p->grid[a]);
    p->D = (int64_t)p->img[0] * p->img[1] * p->img[2];
    p->G = (int64_t)p->grid[0] * p->grid[1] * p->grid[2];
    p->N = g->nsamples;
    // FFT lengths
    for (int a = 3 - nd; a < 3; ++a) CS_PROPAGATE(fft_len_init(p->fft[a], p->grid[a]));
    // per-axis input factors (centred-DFT modulation (-1)^q, deapodisation, 1/sqrt(D))
    const double W = 4.0;
    const double alpha = g->alpha > 0 ? g->alpha : 1.25;
    const double beta = M_PI * std::sqrt((W / alpha) * (W / alpha) * (alpha - 0.5) * (alpha - 0.5) - 0.8);
    p->beta = (float)beta;
    for (int a = 0; a < 3; ++a) {
        const int n = p->img[a];
        std::vector<float> h(n, 1.0f);
        if (a >= 3 - nd) {
            for (int i = 0; i < n; ++i) {
                double v = ((i + p->off[a]) & 1) ? -1.0 : 1.0;
                if (p->kind == CS_NONCARTESIAN) v /= kb_phi_hat((double)(i - n / 2) / p->grid[a], beta, W);
                if (a == 2) v /= std::sqrt((double)p->D);
                h[i] = (float)v;
            }
        }
        CS_TRY_CUDA(cudaMalloc(&p->apod[a], sizeof(float) * n));
        CS_TRY_CUDA(cudaMemcpy(p->apod[a], h.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
    }
    const size_t C = (size_t)p->max_coils;
    CS_TRY_CUDA(cudaMalloc(&p->bufA, sizeof(float2) * C * p->G));
    if (p->kind == CS_CARTESIAN) {
        CS_REQUIRE(nd == 2, CS_ERR_UNSUPPORTED_SIZE, "Cartesian plans are 2D");
        CS_REQUIRE(g->mask_idx != nullptr && p->N > 0 && p->N <= p->D, CS_ERR_INVALID_ARG, "bad Cartesian mask");
        // validate the mask list on the host: strictly ascending flat indices inside the image
        std::vector<int32_t> h(p->N);
        CS_TRY_CUDA(cudaMemcpy(h.data(), g->mask_idx, sizeof(int32_t) * p->N, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < p->N; ++i) {
            CS_REQUIRE(h[i] >= 0 && h[i] < p->D && (i == 0 || h[i] > h[i - 1]), CS_ERR_INVALID_ARG,
                       "mask indices must be strictly ascending and inside the image (index %lld)", (long long)i);
        }
        CS_TRY_CUDA(cudaMalloc(&p->mask_idx, sizeof(int32_t) * p->N));
        CS_TRY_CUDA(cudaMemcpy(p->mask_idx, h.data(), sizeof(int32_t) * p->N, cudaMemcpyHostToDevice));
        CS_TRY_CUDA(cudaMalloc(&p->idxmap, sizeof(int32_t) * p->D));
        CS_TRY_CUDA(cudaMemsetAsync(p->idxmap, 0xff, sizeof(int32_t) * p->D, st));
        idxmap_kernel<<<(unsigned)((p->N + 255) / 256), 256, 0, st>>>(p->mask_idx, p->N, p->idxmap);
        CS_LAUNCH_CHECK();
        CS_TRY_CUDA(cudaStreamSynchronize(st));
        return CS_OK;
    }
    CS_REQUIRE(g->traj != nullptr && g->dcf != nullptr && p->N > 0, CS_ERR_INVALID_ARG, "non-Cartesian plan needs traj, dcf, N > 0");
    CS_REQUIRE(p->G * (int64_t)p->max_coils < (int64_t)1 << 31, CS_ERR_UNSUPPORTED_SIZE,
               "grid points x max_coils must stay below 2^31 (32-bit gridding offsets)");
    CS_REQUIRE(p->N < (int64_t)1 << 31, CS_ERR_UNSUPPORTED_SIZE, "more than 2^31 samples");
    const int64_t bsz = (nd == 3) ? (int64_t)p->img[0] * p->grid[1] * p->grid[2] : p->G;
    CS_TRY_CUDA(cudaMalloc(&p->bufB, sizeof(float2) * C * bsz));
    CS_TRY_CUDA(cudaMalloc(&p->ktmp, sizeof(float2) * C * p->N));
    {
        int t3[3] = {1, 1, 1};
        for (int a = 3 - nd; a < 3; ++a) t3[a] = g->tile[a - (3 - nd)];
        CS_PROPAGATE(nufft_set_tiles(p, t3));
    }
    p->spread_chunk = 64;
    p->interp_chunk = 64;
    // tuning knobs (coils per warp of the gridding kernels, samples per warp)
    if (const char* e = getenv("CS_INTERP_COILS")) p->interp_coils = std::max(1, std::min(32, atoi(e)));
    if (const char* e = getenv("CS_SPREAD_COILS")) p->spread_coils = std::max(1, std::min(16, atoi(e)));
    if (const char* e = getenv("CS_GRID_CHUNK")) p->interp_chunk = p->spread_chunk = std::max(1, atoi(e));
    {
        // phi(u) = I0(beta sqrt(1 - (u/2)^2)) / I0(beta) on [0, 2], 2049 points
        const int nt = 2048;
        std::vector<float> tab(nt + 1);
        const double i0b = std::cyl_bessel_i(0.0, beta);
        for (int i = 0; i <= nt; ++i) {
            const double u = 2.0 * i / nt;
            const double t = 1.0 - 0.25 * u * u;
            tab[i] = (float)(std::cyl_bessel_i(0.0, beta * std::sqrt(t > 0 ? t : 0.0)) / i0b);
        }
        CS_TRY_CUDA(cudaMalloc(&p->phi, sizeof(float) * (nt + 1)));
        CS_TRY_CUDA(cudaMemcpy(p->phi, tab.data(), sizeof(float) * (nt + 1), cudaMemcpyHostToDevice));
    }
    CS_TRY_CUDA(cudaMalloc(&p->gsorted, sizeof(float) * 3 * p->N));
    CS_TRY_CUDA(cudaMalloc(&p->wsorted, sizeof(float) * p->N));
    CS_TRY_CUDA(cudaMalloc(&p->perm, sizeof(int32_t) * p->N));
    CS_TRY_CUDA(cudaMalloc(&p->j0, sizeof(int32_t) * nd * p->N));
    CS_TRY_CUDA(cudaMalloc(&p->tile_off, sizeof(int32_t) * (p->ntiles_total + 1)));
    CS_TRY_CUDA(cudaMalloc(&p->class_off, sizeof(int32_t) * (p->ntiles_total * 8 + 1)));
    CS_PROPAGATE(nufft_bin(p, g->traj, g->dcf, 0, st));
    CS_PROPAGATE(nufft_records(p, st));
    CS_TRY_CUDA(cudaStreamSynchronize(st));
    return CS_OK;
}

static cs_status check_plan_coils(const cs_plan* p, int ncoils) {
    CS_REQUIRE(p != nullptr, CS_ERR_INVALID_ARG, "null plan");
    CS_REQUIRE(ncoils >= 0 && ncoils <= p->max_coils, CS_ERR_INVALID_ARG,
               "coil count %d outside [0, max_coils = %d]", ncoils, p->max_coils);
    return CS_OK;
}

}  // namespace cs

using namespace cs;

extern "C" {

const char* cs_last_error(void) { return g_err; }

long long cs_launch_count(void) { return g_launches.load(); }

cs_status cs_profile(int enable) {
    clear_error();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_drain();
    for (int i = 0; i < ST_COUNT; ++i) {
        g_prof_ms[i] = 0;
        g_prof_n[i] = 0;
    }
    g_prof_on = enable != 0;
    return CS_OK;
}

cs_status cs_profile_read(int stage, double* total_ms, long long* launches) {
    clear_error();
    CS_REQUIRE(stage >= 0 && stage < ST_COUNT && total_ms && launches, CS_ERR_INVALID_ARG, "bad profile query");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_drain();
    *total_ms = g_prof_ms[stage];
    *launches = g_prof_n[stage];
    return CS_OK;
}
#ifdef CS_CHECK_BOUNDS
const char* cs_version(void) { return "coilsketch-gb300 0.2 (sm_103a, bounds-checked)"; }
#else
const char* cs_version(void) { return "coilsketch-gb300 0.2 (sm_103a)"; }
#endif

cs_status cs_plan_create(const cs_geom* g, void* stream, cs_plan** out) {
    clear_error();
    CS_REQUIRE(g != nullptr && out != nullptr, CS_ERR_INVALID_ARG, "null argument");
    CS_REQUIRE(g->ndim == 2 || g->ndim == 3, CS_ERR_INVALID_ARG, "ndim must be 2 or 3");
    CS_REQUIRE(g->kind == CS_CARTESIAN || g->kind == CS_NONCARTESIAN, CS_ERR_INVALID_ARG, "bad plan kind");
    CS_REQUIRE(g->max_coils >= 1 && g->max_coils <= 256, CS_ERR_INVALID_ARG, "max_coils must be in [1, 256]");
    *out = nullptr;
    cs_plan* p = new cs_plan();
    cs_status rc = plan_build(p, g, (cudaStream_t)stream);
    if (rc != CS_OK) {
        plan_free(p);
        return rc;
    }
    *out = p;
    return CS_OK;
}

cs_status cs_plan_destroy(cs_plan* plan) {
    plan_free(plan);
    return CS_OK;
}

cs_status cs_plan_binning(const cs_plan* p, int32_t* perm, int32_t* tile_off, int32_t* j0, int* ntiles_out,
                          void* stream) {
    clear_error();
    CS_REQUIRE(p != nullptr && p->kind == CS_NONCARTESIAN, CS_ERR_INVALID_ARG, "needs a non-Cartesian plan");
    cudaStream_t st = (cudaStream_t)stream;
    if (perm) CS_TRY_CUDA(cudaMemcpyAsync(perm, p->perm, sizeof(int32_t) * p->N, cudaMemcpyDeviceToDevice, st));
    if (tile_off)
        CS_TRY_CUDA(cudaMemcpyAsync(tile_off, p->tile_off, sizeof(int32_t) * (p->ntiles_total + 1), cudaMemcpyDeviceToDevice, st));
    if (j0) CS_TRY_CUDA(cudaMemcpyAsync(j0, p->j0, sizeof(int32_t) * p->ndim * p->N, cudaMemcpyDeviceToDevice, st));
    if (ntiles_out)
        for (int a = 0; a < 3; ++a) ntiles_out[a] = p->ntiles[a];
    return CS_OK;
}

cs_status sense_fwd(const cs_plan* p, const float* x, const float* maps, int ncoils, float* y, void* stream) {
    clear_error();
    CS_PROPAGATE(check_plan_coils(p, ncoils));
    CS_REQUIRE(x && maps && y, CS_ERR_INVALID_ARG, "null pointer");
    if (ncoils == 0) return CS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const float2* m = (const float2*)maps;
    CS_PROPAGATE(fft_to_grid(p, (const float2*)x, m, ncoils, nullptr, 0, st));
    if (p->kind == CS_CARTESIAN) return fft_cart_sample(p, 0, ncoils, nullptr, (float2*)y, st);
    return nufft_interp(p, ncoils, (float2*)y, nullptr, st);
}

cs_status sense_adj(const cs_plan* p, const float* y, const float* maps, int ncoils, float* x, int accumulate,
                    void* stream) {
    clear_error();
    CS_PROPAGATE(check_plan_coils(p, ncoils));
    CS_REQUIRE(x && maps && y, CS_ERR_INVALID_ARG, "null pointer");
    cudaStream_t st = (cudaStream_t)stream;
    if (ncoils == 0) {
        if (!accumulate) CS_TRY_CUDA(cudaMemsetAsync(x, 0, sizeof(float2) * p->D, st));
        return CS_OK;
    }
    const float2* m = (const float2*)maps;
    if (p->kind == CS_CARTESIAN) {
        CS_PROPAGATE(fft_cart_sample(p, 1, ncoils, (const float2*)y, nullptr, st));
    } else {
        CS_PROPAGATE(nufft_spread(p, ncoils, (const float2*)y, 0, st));
    }
    return fft_to_image(p, m, ncoils, nullptr, 0, (float2*)x, accumulate, nullptr, 0.f, st);
}

cs_status sense_grad(const cs_plan* p, const float* x, const float* maps, int ncoils, const float* y, float* d,
                     void* stream) {
    clear_error();
    CS_PROPAGATE(check_plan_coils(p, ncoils));
    CS_REQUIRE(x && maps && y && d, CS_ERR_INVALID_ARG, "null pointer");
    cudaStream_t st = (cudaStream_t)stream;
    const float2* m = (const float2*)maps;
    CS_PROPAGATE(fft_to_grid(p, (const float2*)x, m, ncoils, nullptr, 0, st));
    if (p->kind == CS_CARTESIAN) {
        CS_PROPAGATE(fft_cart_sample(p, 3, ncoils, (const float2*)y, nullptr, st));
    } else {
        CS_PROPAGATE(nufft_interp(p, ncoils, nullptr, (const float2*)y, st));
        CS_PROPAGATE(nufft_spread(p, ncoils, nullptr, 1, st));
    }
    return fft_to_image(p, m, ncoils, nullptr, 0, (float2*)d, 0, nullptr, 0.f, st);
}

cs_status sketched_normal_apply(const cs_plan* p, const float* v, const float* maps_v, int V, const float* maps_s,
                                int S, float lambda, float* z, void* stream) {
    clear_error();
    CS_REQUIRE(V >= 0 && S >= 0, CS_ERR_INVALID_ARG, "negative coil count");
    CS_PROPAGATE(check_plan_coils(p, V + S));
    CS_REQUIRE(v && z && (V == 0 || maps_v) && (S == 0 || maps_s), CS_ERR_INVALID_ARG, "null pointer");
    CS_REQUIRE(v != z, CS_ERR_INVALID_ARG, "v and z must not alias");
    cudaStream_t st = (cudaStream_t)stream;
    const float2* mv = (const float2*)maps_v;
    const float2* ms = (const float2*)maps_s;
    if (V + S == 0) {
        CS_TRY_CUDA(cudaMemsetAsync(z, 0, sizeof(float2) * p->D, st));
        return fft_to_image(p, mv, 0, ms, 0, (float2*)z, 1, (const float2*)v, lambda, st);
    }
    CS_PROPAGATE(fft_to_grid(p, (const float2*)v, mv, V, ms, S, st));
    if (p->kind == CS_CARTESIAN) CS_PROPAGATE(fft_cart_sample(p, 2, V + S, nullptr, nullptr, st));
    else CS_PROPAGATE(nufft_interp_spread(p, V + S, st));
    return fft_to_image(p, mv, V, ms, S, (float2*)z, 0, (const float2*)v, lambda, st);
}

cs_status cs_plan_set_gridding(cs_plan* p, int interp_coils, int interp_chunk, int spread_coils, int spread_chunk) {
    clear_error();
    CS_REQUIRE(p, CS_ERR_INVALID_ARG, "null plan");
    CS_REQUIRE(interp_coils >= 1 && interp_coils <= 32 && spread_coils >= 1 && spread_coils <= 16 && interp_chunk >= 1 &&
                   interp_chunk <= 4096 && spread_chunk >= 1 && spread_chunk <= 4096,
               CS_ERR_INVALID_ARG, "gridding parameters out of range");
    p->interp_coils = interp_coils;
    p->interp_chunk = interp_chunk;
    p->spread_coils = spread_coils;
    p->spread_chunk = spread_chunk;
    p->layout_gen++;
    return CS_OK;
}

cs_status cs_plan_set_deterministic(cs_plan* p, int on, int item_visits) {
    clear_error();
    CS_REQUIRE(p && (on == 0 || on == 1) && (item_visits == 0 || (item_visits >= 64 && item_visits <= (1 << 20))),
               CS_ERR_INVALID_ARG, "bad deterministic-spreading arguments");
    if (p->kind != CS_NONCARTESIAN) return CS_OK;
    const int q = item_visits > 0 ? item_visits : p->owner_item;
    if (on && (q != p->owner_item || !p->gitems)) {
        CS_TRY_CUDA(cudaDeviceSynchronize());      // work items and partial slots are (re)built
        p->owner_item = q;
        CS_PROPAGATE(nufft_owner_build(p));
    }
    p->owner_item = q;
    p->deterministic = on;
    p->layout_gen++;
    return CS_OK;
}

// Times the interpolation and spreading launches of `ncoils` coils for each candidate (coils per
// warp, samples per warp) on the plan's own scratch buffers and keeps the fastest of each.
cs_status cs_plan_autotune(cs_plan* p, int ncoils, int reps, int* choice, float* ms, void* stream) {
    clear_error();
    CS_REQUIRE(p && ncoils >= 1 && ncoils <= p->max_coils && reps >= 1 && reps <= 100, CS_ERR_INVALID_ARG,
               "bad autotune arguments");
    cudaStream_t st = (cudaStream_t)stream;
    float best_i = 0.f, best_s = 0.f, def_i = 0.f, def_s = 0.f;
    if (p->kind == CS_NONCARTESIAN) {
        cudaEvent_t e0, e1;
        CS_TRY_CUDA(cudaEventCreate(&e0));
        CS_TRY_CUDA(cudaEventCreate(&e1));
        cs_status rc = CS_OK;
        auto timed = [&](bool spread, float& out) -> cs_status {
            for (int r = 0; r <= reps; ++r) {
                if (r == 1) CS_TRY_CUDA(cudaEventRecord(e0, st));
                if (spread) CS_PROPAGATE(nufft_spread(p, ncoils, nullptr, 1, st));
                else CS_PROPAGATE(nufft_interp_sorted(p, ncoils, st));
            }
            CS_TRY_CUDA(cudaEventRecord(e1, st));
            CS_TRY_CUDA(cudaEventSynchronize(e1));
            CS_TRY_CUDA(cudaEventElapsedTime(&out, e0, e1));
            out /= reps;
            return CS_OK;
        };
        const int coils_i[] = {8, 16, 32}, coils_s[] = {8, 16}, chunks[] = {32, 64, 128};
        int bi_c = p->interp_coils, bi_k = p->interp_chunk, bs_c = p->spread_coils, bs_k = p->spread_chunk;
        rc = timed(false, def_i);
        if (rc == CS_OK) rc = timed(true, def_s);
        best_i = def_i;
        best_s = def_s;
        for (int c : coils_i) {
            for (int k : chunks) {
                if (rc != CS_OK) break;
                p->interp_coils = c;
                p->interp_chunk = k;
                float t = 0.f;
                rc = timed(false, t);
                if (rc == CS_OK && t < best_i) {
                    best_i = t;
                    bi_c = c;
                    bi_k = k;
                }
            }
        }
        for (int c : coils_s) {
            for (int k : chunks) {
                if (rc != CS_OK) break;
                p->spread_coils = c;
                p->spread_chunk = k;
                float t = 0.f;
                rc = timed(true, t);
                if (rc == CS_OK && t < best_s) {
                    best_s = t;
                    bs_c = c;
                    bs_k = k;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        p->interp_coils = bi_c;
        p->interp_chunk = bi_k;
        p->spread_coils = bs_c;
        p->spread_chunk = bs_k;
        p->layout_gen++;
        if (rc != CS_OK) return rc;
    }
    if (choice) {
        choice[0] = p->interp_coils;
        choice[1] = p->interp_chunk;
        choice[2] = p->spread_coils;
        choice[3] = p->spread_chunk;
    }
    if (ms) {
        ms[0] = best_i;
        ms[1] = best_s;
        ms[2] = def_i;
        ms[3] = def_s;
    }
    return CS_OK;
}

cs_status cs_plan_set_tile(cs_plan* p, const int* tile, void* stream) {
    clear_error();
    CS_REQUIRE(p && tile, CS_ERR_INVALID_ARG, "null argument");
    CS_REQUIRE(p->kind == CS_NONCARTESIAN, CS_ERR_INVALID_ARG, "needs a non-Cartesian plan");
    int t3[3] = {1, 1, 1};
    for (int a = 3 - p->ndim; a < 3; ++a) {
        t3[a] = tile[a - (3 - p->ndim)];
        CS_REQUIRE(t3[a] >= 1, CS_ERR_INVALID_ARG, "tile sizes must be positive");
    }
    return nufft_retile(p, t3, (cudaStream_t)stream);
}

// Times interpolation + spreading of `ncoils` coils for every cubic tile candidate (the plan is
// re-binned for each) and leaves the plan binned with the fastest.
cs_status cs_plan_autotune_tile(cs_plan* p, int ncoils, int reps, const int* cand, int ncand, int* best, float* ms,
                                void* stream) {
    clear_error();
    CS_REQUIRE(p && cand && ncand >= 1 && ncand <= 16 && ncoils >= 1 && ncoils <= p->max_coils && reps >= 1 &&
                   reps <= 100,
               CS_ERR_INVALID_ARG, "bad tile autotune arguments");
    CS_REQUIRE(p->kind == CS_NONCARTESIAN, CS_ERR_INVALID_ARG, "needs a non-Cartesian plan");
    for (int i = 0; i < ncand; ++i) CS_REQUIRE(cand[i] >= 4, CS_ERR_INVALID_ARG, "tile candidates must be >= 4");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    CS_TRY_CUDA(cudaEventCreate(&e0));
    CS_TRY_CUDA(cudaEventCreate(&e1));
    cs_status rc = CS_OK;
    int bi = -1;
    float bt = 0.f;
    auto timed = [&](float& out) -> cs_status {
        for (int r = 0; r <= reps; ++r) {
            if (r == 1) CS_TRY_CUDA(cudaEventRecord(e0, st));
            CS_PROPAGATE(nufft_interp_sorted(p, ncoils, st));
            CS_PROPAGATE(nufft_spread(p, ncoils, nullptr, 1, st));
        }
        CS_TRY_CUDA(cudaEventRecord(e1, st));
        CS_TRY_CUDA(cudaEventSynchronize(e1));
        CS_TRY_CUDA(cudaEventElapsedTime(&out, e0, e1));
        out /= reps;
        return CS_OK;
    };
    for (int i = 0; i < ncand && rc == CS_OK; ++i) {
        const int t3[3] = {cand[i], cand[i], cand[i]};
        rc = nufft_retile(p, t3, st);
        float t = 0.f;
        if (rc == CS_OK) rc = timed(t);
        if (rc == CS_OK) {
            if (ms) ms[i] = t;
            if (bi < 0 || t < bt) {
                bi = i;
                bt = t;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != CS_OK) return rc;
    if (bi != ncand - 1) {
        const int t3[3] = {cand[bi], cand[bi], cand[bi]};
        CS_PROPAGATE(nufft_retile(p, t3, st));
    }
    if (best) *best = cand[bi];
    return CS_OK;
}

}  // extern "C"
