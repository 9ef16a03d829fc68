// Internal declarations shared by the CUDA translation units of libcoilsketch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/coilsketch.h"

namespace cs {

// ------------------------------------------------------------------------------------------
// error plumbing (thread-local message, status codes; nothing throws across the ABI)
void set_error(const char* fmt, ...);
void clear_error();

#define CS_TRY_CUDA(call)                                                                     \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            ::cs::set_error("%s:%d: %s failed: %s", __FILE__, __LINE__, #call,               \
                            cudaGetErrorString(e_));                                          \
            return e_ == cudaErrorMemoryAllocation ? CS_ERR_OOM : CS_ERR_CUDA;                \
        }                                                                                     \
    } while (0)

// every kernel launch of the library is followed by CS_LAUNCH_CHECK, which also counts it
void count_launch();
#define CS_LAUNCH_CHECK()                                                                     \
    do {                                                                                      \
        ::cs::count_launch();                                                                 \
        CS_TRY_CUDA(cudaGetLastError());                                                      \
    } while (0)

// optional per-stage timing with CUDA events (enabled by cs_profile)
enum { ST_SPREAD = 0, ST_INTERP = 1, ST_FFT_PLAIN = 2, ST_EXPAND = 3, ST_REDUCE = 4, ST_COUNT = 5 };
bool profiling();
void prof_begin(int stage, cudaStream_t st);
void prof_end(int stage, cudaStream_t st);

#define CS_REQUIRE(cond, code, ...)                                                           \
    do {                                                                                      \
        if (!(cond)) {                                                                        \
            ::cs::set_error(__VA_ARGS__);                                                     \
            return (code);                                                                    \
        }                                                                                     \
    } while (0)

#define CS_PROPAGATE(expr)                                                                    \
    do {                                                                                      \
        cs_status s_ = (expr);                                                                \
        if (s_ != CS_OK) return s_;                                                           \
    } while (0)

// ------------------------------------------------------------------------------------------
// Bounds-checked builds (compiled with -DCS_CHECK_BOUNDS, build(checked=True)): every guarded
// global access checks its element index against the length of its buffer; an index outside
// skips the access (a guarded load reads zero) and sets the error word of its translation unit,
// which cs_device_status and recon_solve report as CS_ERR_BOUNDS.  Nothing traps: the context
// stays usable.  In normal builds a guard is the constant true and compiles away.
#ifdef CS_CHECK_BOUNDS
static __device__ unsigned int cs_bounds_word = 0;
__device__ __forceinline__ bool cs_inb(long long i, long long n) {
    if (i >= 0 && i < n) return true;
    atomicOr(&cs_bounds_word, 1u);
    return false;
}
#define CS_INB(i, n) ::cs::cs_inb((long long)(i), (long long)(n))
#define CS_BOUNDS_READER(fn)                                                                  \
    cs_status fn() {                                                                          \
        unsigned int v = 0;                                                                   \
        CS_TRY_CUDA(cudaMemcpyFromSymbol(&v, cs_bounds_word, sizeof(v)));                     \
        if (!v) return CS_OK;                                                                 \
        const unsigned int zero = 0;                                                          \
        cudaMemcpyToSymbol(cs_bounds_word, &zero, sizeof(zero));                              \
        set_error("a device-side index check failed (%s)", #fn);                             \
        return CS_ERR_BOUNDS;                                                                 \
    }
#else
#define CS_INB(i, n) true
#define CS_BOUNDS_READER(fn) \
    cs_status fn() { return CS_OK; }
#endif
// readers of the translation units with guarded accesses (after the caller synchronised)
cs_status nufft_bounds_check();
cs_status fft_bounds_check();
cs_status bounds_check_all();

// ------------------------------------------------------------------------------------------
// complex helpers (complex64 = float2)
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// ------------------------------------------------------------------------------------------
// 1D FFT length descriptor: mixed-radix Stockham factorisation + device twiddle table
constexpr int kMaxRadices = 12;
constexpr int kMaxFft = 800;   // 2 * 800 * 17 * 8 B + twiddles fits the 227 KB shared-memory limit

struct FftLen {
    int n = 0;
    int nrad = 0;
    int rad[kMaxRadices] = {0};
    // per Stockham stage: (radix r, Ns = product of the earlier radices, floor(2^32 / Ns) + 1,
    // twiddle stride n / (Ns r)), so that kernels divide by nothing at run time
    int4 st[kMaxRadices] = {};
    float2* tw = nullptr;  // device, n entries exp(-2 pi i k / n) (computed in double)
};

cs_status fft_len_init(FftLen& f, int n);
void fft_len_free(FftLen& f);

// Lines handled by one CTA of a pass kernel, threads per CTA.
constexpr int kLines = 16;
constexpr int kLinePad = 17;
constexpr int kPassThreads = 256;

// ------------------------------------------------------------------------------------------
// Owner-computes spreading (nufft.cu): every tile of the grid is accumulated by exactly one warp at
// a time, from its own samples and the samples of its lower neighbour tiles whose kernel box
// reaches it; a tile with more sample visits than the plan's item size is split into items whose
// sums land in private partial slots, added to the grid afterwards in a fixed order.
struct GItem {
    int tile;      // linear tile id (z, y, x; x fastest)
    int slot;      // partial slot, or -1: the item writes the grid itself
    int r0, r1;    // its sample ranges [r0, r1) in the plan's range list
};
struct GRange {
    int start, count;   // consecutive sorted samples
};
struct GRed {
    int tile, s0, ns;   // the tile's partial slots s0 .. s0 + ns - 1, added in this order
};

// ------------------------------------------------------------------------------------------
// Plan
}  // namespace cs

struct cs_plan {
    int kind = CS_CARTESIAN;
    int ndim = 2;
    int device = 0;
    int img[3] = {1, 1, 1};    // always 3 entries (nz, ny, nx); 2D uses nz = 1
    int grid[3] = {1, 1, 1};   // oversampled grid (Cartesian: equals img)
    int off[3] = {0, 0, 0};    // (grid - img) / 2 per axis
    int64_t D = 0;             // image voxels
    int64_t G = 0;             // grid voxels
    int64_t N = 0;             // samples per coil
    int max_coils = 0;
    float beta = 0.f;          // Kaiser-Bessel beta

    cs::FftLen fft[3];         // per axis (z, y, x)
    float* apod[3] = {nullptr, nullptr, nullptr};   // per-axis input factor (img length), device

    // Cartesian sampling
    int32_t* idxmap = nullptr;    // [D] sample index or -1
    int32_t* mask_idx = nullptr;  // [N]

    // non-Cartesian sampling
    float* gsorted = nullptr;     // [N][3] grid coordinates (float32 fmaf), sorted by tile
    float* wsorted = nullptr;     // [N] sqrt(dcf), sorted
    int32_t* perm = nullptr;      // [N] sorted position -> sample index
    int32_t* j0 = nullptr;        // [N][3] unwrapped first box index (user order), for tests
    int32_t* tile_off = nullptr;  // [ntiles + 1]
    int32_t* class_off = nullptr; // [ntiles * 8 + 1] offsets of every (tile, halo class) run
    int tile[3] = {1, 1, 1};
    int ntiles[3] = {1, 1, 1};    // a remainder narrower than the kernel widens the last tile
    int wmax[3] = {1, 1, 1};      // widest tile per axis (the partial-slot geometry)
    int64_t ntiles_total = 0;
    int interp_chunk = 0;         // consecutive sorted samples per warp, interpolation
    int spread_chunk = 0;         // consecutive sorted samples per warp, producer spreading
    int deterministic = 0;        // 1: owner-computes spreading (atomics-free, bit-reproducible)
    int owner_item = 4096;        // largest sample visits of one owner-computes work item
    cs::GItem* gitems = nullptr;  // spreading work items, longest first
    int n_gitems = 0;
    cs::GRange* granges = nullptr;
    cs::GRed* greds = nullptr;    // tiles with partial slots
    int n_greds = 0;
    int n_slots = 0;
    float2* gpart = nullptr;      // partial slots [n_slots][wmax z][wmax y][wmax x][<= 16 coils]
    int interp_coils = 16;        // coils per warp in interpolation (8, 16 or 32)
    int spread_coils = 16;        // coils per warp in spreading (8 or 16)
    float* phi = nullptr;         // KB kernel table [2049] on [0, 2]
    float* rec = nullptr;         // [N][16] per-sample gridding records (sorted order)
    uint64_t layout_gen = 0;      // bumped when the sample order, the records or the gridding launch
                                  // parameters change; part of every captured graph's signature

    // workspace (per coil up to max_coils)
    float2* bufA = nullptr;       // grid-sized per coil   [max_coils][G] (also the first-pass buffer)
    float2* bufB = nullptr;       // intermediate per coil [max_coils][nz * Gy * Gx] (3D) or unused
    float2* ktmp = nullptr;       // k-space scratch [N][max_coils] (sorted, coil-interleaved)
    void* solver_ws = nullptr;    // recon_solve workspace and cached CUDA graph (solve.cu)
};

namespace cs {

// FFT passes (fft.cu)
cs_status fft_to_grid(const cs_plan* p, const float2* x, const float2* maps_v, int V,
                      const float2* maps_s, int S, cudaStream_t st);
cs_status fft_cart_sample(const cs_plan* p, int mode, int ncoils, const float2* yk, float2* yko, cudaStream_t st);
cs_status fft_to_image(const cs_plan* p, const float2* maps_v, int V, const float2* maps_s, int S,
                       float2* x, int accumulate, const float2* addv, float lambda, cudaStream_t st);

// NUFFT binning / interpolation / spreading (nufft.cu)
// tile sizes (per axis z, y, x; validated) -> tile, ntiles, wmax, ntiles_total
cs_status nufft_set_tiles(cs_plan* p, const int* tile3);
// binning from the user's trajectory (from_grid = 0: coords = traj [N][ndim], w = dcf) or from
// grid coordinates in user order (from_grid = 1: coords [N][3], w = sqrt(dcf))
cs_status nufft_bin(cs_plan* p, const float* coords, const float* w, int from_grid, cudaStream_t st);
// re-bins a non-Cartesian plan for new tile sizes (records rewritten in place)
cs_status nufft_retile(cs_plan* p, const int* tile3, cudaStream_t st);
cs_status nufft_records(cs_plan* p, cudaStream_t st);
cs_status nufft_owner_build(cs_plan* p);   // spreading work items from the class offsets (synchronous)
void nufft_owner_free(cs_plan* p);
cs_status nufft_interp(const cs_plan* p, int ncoils, float2* y, const float2* ysub, cudaStream_t st);
cs_status nufft_spread(const cs_plan* p, int ncoils, const float2* y, int sorted_in, cudaStream_t st);
cs_status nufft_interp_spread(const cs_plan* p, int ncoils, cudaStream_t st);
cs_status nufft_interp_sorted(const cs_plan* p, int ncoils, cudaStream_t st);   // ktmp = w^1/2 interp(grid)

// Reductions and vector kernels (solve.cu)
int reduce_blocks();

void solver_ws_free(cs_plan* p);

// one-time per-device set-up (kernel attributes, filter constants), done at plan creation
cs_status fft_init_attrs();
cs_status fft_check_and_clear();
cs_status tc_init_attrs();
cs_status wavelet_init_constants();
cs_status coil_init_attrs();

// Warm-start network pieces used by recon_solve (warmnet.cu, unet.cu).  The network input scale
// is a fixed-order FP64 sum over kFeatBlocks block partials (part), so inference is reproducible.
constexpr int kFeatBlocks = 296;
cs_status nn_features_det(const float2* xt, const float2* d, int64_t n, float eta, const double* eta_dev, double* part,
                          float* ss, float* f, cudaStream_t st);
// buffers for `dims` and packed weights, done outside any stream capture; *gen changes whenever the
// network's activation buffers are reallocated (a captured graph holding the old ones is stale)
cs_status unet_prepare(cs_unet* net, const int* dims, cudaStream_t st, uint64_t* gen);
// xhat = x^t + s U-Net(x^t / s, eta d / s) with eta read on the device (capturable after unet_prepare)
cs_status unet_infer_dev(cs_unet* net, const float2* xt, const float2* d, const int* dims, const double* eta_dev,
                         float2* xhat, cudaStream_t st);

// Jacobi eigensolver (shared host/device algorithm, coil.cu)
void hermitian_eig_serial(double* A, int n, double* V, double* evals);

}  // namespace cs
