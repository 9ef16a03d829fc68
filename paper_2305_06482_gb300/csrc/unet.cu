// The warm-start network as a library object: a 3-level 3D U-Net (widths c1/c2/c3; two 3x3x3
// convolutions with ReLU per level, 2x2x2 max-pools, 2x2x2 stride-2 transposed convolutions,
// skip concatenation [up-path, encoder], a 1x1x1 layer to 2 channels) whose parameters, Adam
// state, packed tensor-core weights and activation buffers live on the device.  Inference and
// one training step are sequences of the layer kernels of warmnet.cu; the host only orders them.
// Parameter i of the 26: (w, b) pairs of the layers e1a, e1b, e2a, e2b, b1, b2 (3x3x3, w
// [cout][27][cin]), u2 (transposed, w [cout][8][cin]), d2a, d2b, u1, d1a, d1b, out (w [2][c1]).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "cs_internal.cuh"

namespace {

constexpr int kParams = 26;
enum LayerKind { L_CONV = 0, L_UP = 1, L_OUT = 2 };
struct Layer {
    int pi, kind, cin, cout;
};

int npad_of(int n) { return n <= 16 ? 16 : n <= 32 ? 32 : 64; }
int kpad_of(int k) { return (k + 15) / 16 * 16; }

}  // namespace

struct cs_unet {
    int c1 = 16, c2 = 32, c3 = 64;
    int device = 0;
    int step = 0;
    std::vector<Layer> layers;
    int64_t numel[kParams] = {};
    float* p[kParams] = {};
    float* g[kParams] = {};
    float* m[kParams] = {};
    float* v[kParams] = {};
    // packed BF16 weights of the 3x3x3 layers: forward and transposed (data gradient)
    unsigned short* pk_f[kParams] = {};
    unsigned short* pk_t[kParams] = {};
    int np_f[kParams] = {}, kp_f[kParams] = {}, np_t[kParams] = {}, kp_t[kParams] = {};
    bool packed = false;
    // activation and gradient buffers for the current volume size
    int dims[3] = {0, 0, 0};
    bool have_bwd = false;
    std::vector<void*> bufs;
    float *f = nullptr, *e1a = nullptr, *e1 = nullptr, *p1 = nullptr, *e2a = nullptr, *e2 = nullptr, *p2 = nullptr;
    float *b1 = nullptr, *b2 = nullptr, *cat2 = nullptr, *d2a = nullptr, *d2 = nullptr, *cat1 = nullptr;
    float *d1a = nullptr, *d1 = nullptr, *out = nullptr, *tgt = nullptr, *gout = nullptr, *ss = nullptr;
    unsigned char *i1 = nullptr, *i2 = nullptr;
    double* fpart = nullptr;   // kFeatBlocks partial sums of the input scale
    uint64_t gen = 0;          // bumped whenever the buffers above are reallocated
    float *gA1 = nullptr, *gB1 = nullptr, *ge1 = nullptr, *gcat1 = nullptr, *gA2 = nullptr, *gB2 = nullptr;
    float *ge2 = nullptr, *gp1 = nullptr, *gcat2 = nullptr, *gA3 = nullptr, *gB3 = nullptr, *gp2 = nullptr;
};

namespace cs {
namespace {

void free_bufs(cs_unet* n) {
    for (void* b : n->bufs) cudaFree(b);
    n->bufs.clear();
    n->dims[0] = n->dims[1] = n->dims[2] = 0;
    n->have_bwd = false;
}

template <class T>
cs_status alloc(cs_unet* n, T*& ptr, int64_t count) {
    void* q = nullptr;
    CS_TRY_CUDA(cudaMalloc(&q, (size_t)std::max<int64_t>(count, 1) * sizeof(T)));
    n->bufs.push_back(q);
    ptr = (T*)q;
    return CS_OK;
}

cs_status ensure_bufs(cs_unet* n, const int* dims, bool bwd) {
    if (n->dims[0] == dims[0] && n->dims[1] == dims[1] && n->dims[2] == dims[2] && (!bwd || n->have_bwd))
        return CS_OK;
    free_bufs(n);
    const int64_t V1 = (int64_t)dims[0] * dims[1] * dims[2], V2 = V1 / 8, V3 = V1 / 64;
    const int c1 = n->c1, c2 = n->c2, c3 = n->c3;
    CS_PROPAGATE(alloc(n, n->f, V1 * 4));
    CS_PROPAGATE(alloc(n, n->e1a, V1 * c1));
    CS_PROPAGATE(alloc(n, n->e1, V1 * c1));
    CS_PROPAGATE(alloc(n, n->p1, V2 * c1));
    CS_PROPAGATE(alloc(n, n->i1, V2 * c1));
    CS_PROPAGATE(alloc(n, n->e2a, V2 * c2));
    CS_PROPAGATE(alloc(n, n->e2, V2 * c2));
    CS_PROPAGATE(alloc(n, n->p2, V3 * c2));
    CS_PROPAGATE(alloc(n, n->i2, V3 * c2));
    CS_PROPAGATE(alloc(n, n->b1, V3 * c3));
    CS_PROPAGATE(alloc(n, n->b2, V3 * c3));
    CS_PROPAGATE(alloc(n, n->cat2, V2 * 2 * c2));
    CS_PROPAGATE(alloc(n, n->d2a, V2 * c2));
    CS_PROPAGATE(alloc(n, n->d2, V2 * c2));
    CS_PROPAGATE(alloc(n, n->cat1, V1 * 2 * c1));
    CS_PROPAGATE(alloc(n, n->d1a, V1 * c1));
    CS_PROPAGATE(alloc(n, n->d1, V1 * c1));
    CS_PROPAGATE(alloc(n, n->out, V1 * 2));
    CS_PROPAGATE(alloc(n, n->ss, 2));
    CS_PROPAGATE(alloc(n, n->fpart, kFeatBlocks));
    n->gen += 1;
    if (bwd) {
        CS_PROPAGATE(alloc(n, n->tgt, V1 * 2));
        CS_PROPAGATE(alloc(n, n->gout, V1 * 2));
        CS_PROPAGATE(alloc(n, n->gA1, V1 * c1));
        CS_PROPAGATE(alloc(n, n->gB1, V1 * c1));
        CS_PROPAGATE(alloc(n, n->ge1, V1 * c1));
        CS_PROPAGATE(alloc(n, n->gcat1, V1 * 2 * c1));
        CS_PROPAGATE(alloc(n, n->gA2, V2 * c2));
        CS_PROPAGATE(alloc(n, n->gB2, V2 * c2));
        CS_PROPAGATE(alloc(n, n->ge2, V2 * c2));
        CS_PROPAGATE(alloc(n, n->gp1, V2 * c1));
        CS_PROPAGATE(alloc(n, n->gcat2, V2 * 2 * c2));
        CS_PROPAGATE(alloc(n, n->gA3, V3 * c3));
        CS_PROPAGATE(alloc(n, n->gB3, V3 * c3));
        CS_PROPAGATE(alloc(n, n->gp2, V3 * c2));
        n->have_bwd = true;
    }
    n->dims[0] = dims[0];
    n->dims[1] = dims[1];
    n->dims[2] = dims[2];
    return CS_OK;
}

cs_status pack_all(cs_unet* n, void* st) {
    if (n->packed) return CS_OK;
    for (const Layer& L : n->layers) {
        if (L.kind != L_CONV) continue;
        CS_PROPAGATE(cs_nn_pack_weights(n->p[L.pi], L.cout, L.cin, 0, n->pk_f[L.pi], n->np_f[L.pi], n->kp_f[L.pi], st));
        if (n->pk_t[L.pi])
            CS_PROPAGATE(cs_nn_pack_weights(n->p[L.pi], L.cout, L.cin, 1, n->pk_t[L.pi], n->np_t[L.pi], n->kp_t[L.pi], st));
    }
    n->packed = true;
    return CS_OK;
}

// ReLU(conv3(in)) into out[v][coff + co] (row stride ldo)
cs_status conv(cs_unet* n, const float* in, const int* d, int pi, int cin, int cout, float* out, int ldo, int coff,
               void* st) {
    return cs_nn_conv3d(in, d[0], d[1], d[2], cin, n->pk_f[pi], n->np_f[pi], n->kp_f[pi], cout, n->p[pi + 1], 1, 0, out,
                        ldo, coff, st);
}

cs_status forward(cs_unet* n, void* st) {
    const int c1 = n->c1, c2 = n->c2, c3 = n->c3;
    const int d1[3] = {n->dims[0], n->dims[1], n->dims[2]};
    const int d2[3] = {d1[0] / 2, d1[1] / 2, d1[2] / 2};
    const int d3[3] = {d2[0] / 2, d2[1] / 2, d2[2] / 2};
    const int64_t V1 = (int64_t)d1[0] * d1[1] * d1[2], V2 = V1 / 8;
    CS_PROPAGATE(pack_all(n, st));
    CS_PROPAGATE(conv(n, n->f, d1, 0, 4, c1, n->e1a, c1, 0, st));
    CS_PROPAGATE(conv(n, n->e1a, d1, 2, c1, c1, n->e1, c1, 0, st));
    CS_PROPAGATE(cs_nn_maxpool2(n->e1, d2[0], d2[1], d2[2], c1, n->p1, n->i1, st));
    CS_PROPAGATE(conv(n, n->p1, d2, 4, c1, c2, n->e2a, c2, 0, st));
    CS_PROPAGATE(conv(n, n->e2a, d2, 6, c2, c2, n->e2, c2, 0, st));
    CS_PROPAGATE(cs_nn_maxpool2(n->e2, d3[0], d3[1], d3[2], c2, n->p2, n->i2, st));
    CS_PROPAGATE(conv(n, n->p2, d3, 8, c2, c3, n->b1, c3, 0, st));
    CS_PROPAGATE(conv(n, n->b1, d3, 10, c3, c3, n->b2, c3, 0, st));
    CS_PROPAGATE(cs_nn_upconv2(n->b2, d3[0], d3[1], d3[2], c3, n->p[12], n->p[13], c2, n->cat2, 2 * c2, 0, st));
    CS_PROPAGATE(cs_nn_slice(n->e2, c2, 0, c2, n->cat2, 2 * c2, c2, V2, 0, st));
    CS_PROPAGATE(conv(n, n->cat2, d2, 14, 2 * c2, c2, n->d2a, c2, 0, st));
    CS_PROPAGATE(conv(n, n->d2a, d2, 16, c2, c2, n->d2, c2, 0, st));
    CS_PROPAGATE(cs_nn_upconv2(n->d2, d2[0], d2[1], d2[2], c2, n->p[18], n->p[19], c1, n->cat1, 2 * c1, 0, st));
    CS_PROPAGATE(cs_nn_slice(n->e1, c1, 0, c1, n->cat1, 2 * c1, c1, V1, 0, st));
    CS_PROPAGATE(conv(n, n->cat1, d1, 20, 2 * c1, c1, n->d1a, c1, 0, st));
    CS_PROPAGATE(conv(n, n->d1a, d1, 22, c1, c1, n->d1, c1, 0, st));
    return cs_nn_conv1(n->d1, V1, c1, 2, n->p[24], n->p[25], n->out, st);
}

// ReLU mask, weight gradient and (optionally) data gradient of 3x3x3 layer pi
cs_status conv_back(cs_unet* n, float* g, const float* act_out, const float* act_in, const int* d, int pi, int cin,
                    int cout, float* gin, void* st) {
    const int64_t V = (int64_t)d[0] * d[1] * d[2];
    CS_PROPAGATE(cs_nn_relu_bwd(act_out, g, V * cout, st));
    CS_PROPAGATE(cs_nn_conv3d_wgrad(act_in, g, d[0], d[1], d[2], cin, cout, n->g[pi], n->g[pi + 1], st));
    if (!gin) return CS_OK;
    return cs_nn_conv3d(g, d[0], d[1], d[2], cout, n->pk_t[pi], n->np_t[pi], n->kp_t[pi], cin, nullptr, 0, 1, gin, cin, 0,
                        st);
}

cs_status backward(cs_unet* n, void* st) {
    const int c1 = n->c1, c2 = n->c2, c3 = n->c3;
    const int d1[3] = {n->dims[0], n->dims[1], n->dims[2]};
    const int d2[3] = {d1[0] / 2, d1[1] / 2, d1[2] / 2};
    const int d3[3] = {d2[0] / 2, d2[1] / 2, d2[2] / 2};
    const int64_t V1 = (int64_t)d1[0] * d1[1] * d1[2], V2 = V1 / 8;
    for (int i = 0; i < kParams; ++i) CS_TRY_CUDA(cudaMemsetAsync(n->g[i], 0, n->numel[i] * sizeof(float), (cudaStream_t)st));
    CS_PROPAGATE(cs_nn_conv1_bwd(n->d1, n->gout, V1, c1, 2, n->p[24], n->gA1, n->g[24], n->g[25], st));
    CS_PROPAGATE(conv_back(n, n->gA1, n->d1, n->d1a, d1, 22, c1, c1, n->gB1, st));
    CS_PROPAGATE(conv_back(n, n->gB1, n->d1a, n->cat1, d1, 20, 2 * c1, c1, n->gcat1, st));
    CS_PROPAGATE(cs_nn_upconv2_bwd(n->d2, n->gcat1, 2 * c1, 0, d2[0], d2[1], d2[2], c2, n->p[18], c1, n->gA2, n->g[18],
                                   n->g[19], st));
    CS_PROPAGATE(conv_back(n, n->gA2, n->d2, n->d2a, d2, 16, c2, c2, n->gB2, st));
    CS_PROPAGATE(conv_back(n, n->gB2, n->d2a, n->cat2, d2, 14, 2 * c2, c2, n->gcat2, st));
    CS_PROPAGATE(cs_nn_upconv2_bwd(n->b2, n->gcat2, 2 * c2, 0, d3[0], d3[1], d3[2], c3, n->p[12], c2, n->gA3, n->g[12],
                                   n->g[13], st));
    CS_PROPAGATE(conv_back(n, n->gA3, n->b2, n->b1, d3, 10, c3, c3, n->gB3, st));
    CS_PROPAGATE(conv_back(n, n->gB3, n->b1, n->p2, d3, 8, c2, c3, n->gp2, st));
    CS_PROPAGATE(cs_nn_maxpool2_bwd(n->gp2, n->i2, d3[0], d3[1], d3[2], c2, n->ge2, st));
    CS_PROPAGATE(cs_nn_slice(n->gcat2, 2 * c2, c2, c2, n->ge2, c2, 0, V2, 1, st));
    CS_PROPAGATE(conv_back(n, n->ge2, n->e2, n->e2a, d2, 6, c2, c2, n->gA2, st));
    CS_PROPAGATE(conv_back(n, n->gA2, n->e2a, n->p1, d2, 4, c1, c2, n->gp1, st));
    CS_PROPAGATE(cs_nn_maxpool2_bwd(n->gp1, n->i1, d2[0], d2[1], d2[2], c1, n->ge1, st));
    CS_PROPAGATE(cs_nn_slice(n->gcat1, 2 * c1, c1, c1, n->ge1, c1, 0, V1, 1, st));
    CS_PROPAGATE(conv_back(n, n->ge1, n->e1, n->e1a, d1, 2, c1, c1, n->gA1, st));
    return conv_back(n, n->gA1, n->e1a, n->f, d1, 0, 4, c1, nullptr, st);
}

cs_status check_dims(const cs_unet* n, const int* dims) {
    CS_REQUIRE(dims, CS_ERR_INVALID_ARG, "null dims");
    for (int a = 0; a < 3; ++a)
        CS_REQUIRE(dims[a] >= 4 && dims[a] % 4 == 0, CS_ERR_UNSUPPORTED_SIZE,
                   "U-Net volume sizes must be positive multiples of 4 (got %d x %d x %d)", dims[0], dims[1], dims[2]);
    int dev = 0;
    CS_TRY_CUDA(cudaGetDevice(&dev));
    CS_REQUIRE(dev == n->device, CS_ERR_INVALID_ARG, "network lives on device %d, current device is %d", n->device, dev);
    return CS_OK;
}

void destroy(cs_unet* n) {
    free_bufs(n);
    for (int i = 0; i < kParams; ++i) {
        cudaFree(n->p[i]);
        cudaFree(n->g[i]);
        cudaFree(n->m[i]);
        cudaFree(n->v[i]);
        cudaFree(n->pk_f[i]);
        cudaFree(n->pk_t[i]);
    }
    delete n;
}

constexpr char kMagic[8] = {'C', 'S', 'U', 'N', 'E', 'T', '1', '\0'};

}  // namespace

cs_status unet_prepare(cs_unet* net, const int* dims, cudaStream_t st, uint64_t* gen) {
    CS_REQUIRE(net, CS_ERR_INVALID_ARG, "null warm-start network");
    CS_PROPAGATE(check_dims(net, dims));
    CS_PROPAGATE(ensure_bufs(net, dims, false));
    CS_PROPAGATE(pack_all(net, st));
    *gen = net->gen;
    return CS_OK;
}

cs_status unet_infer_dev(cs_unet* net, const float2* xt, const float2* d, const int* dims, const double* eta_dev,
                         float2* xhat, cudaStream_t st) {
    CS_REQUIRE(net->dims[0] == dims[0] && net->dims[1] == dims[1] && net->dims[2] == dims[2] && net->packed,
               CS_ERR_INVALID_ARG, "warm-start network not prepared for this volume");
    const int64_t n = (int64_t)dims[0] * dims[1] * dims[2];
    CS_PROPAGATE(nn_features_det(xt, d, n, 0.f, eta_dev, net->fpart, net->ss, net->f, st));
    CS_PROPAGATE(forward(net, st));
    return cs_nn_apply((const float*)xt, net->out, n, net->ss, (float*)xhat, st);
}

}  // namespace cs

using namespace cs;

extern "C" {

cs_status ws_net_create(int c1, int c2, int c3, uint64_t seed, cs_unet** out) {
    clear_error();
    CS_REQUIRE(out, CS_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    // every convolution's outputs (and the concatenations' 2 c1, 2 c2 inputs of the data gradient)
    // fit one tensor-core tile of 64 columns
    CS_REQUIRE(c1 >= 4 && c2 >= 4 && c3 >= 4 && c1 % 4 == 0 && c2 % 4 == 0 && c3 % 4 == 0 && c1 <= 32 && c2 <= 32 &&
                   c3 <= 64,
               CS_ERR_UNSUPPORTED_SIZE, "U-Net widths must be multiples of 4 with c1, c2 <= 32 and c3 <= 64");
    cs_unet* n = new cs_unet();
    n->c1 = c1;
    n->c2 = c2;
    n->c3 = c3;
    cudaGetDevice(&n->device);
    n->layers = {{0, L_CONV, 4, c1},       {2, L_CONV, c1, c1},      {4, L_CONV, c1, c2},  {6, L_CONV, c2, c2},
                 {8, L_CONV, c2, c3},      {10, L_CONV, c3, c3},     {12, L_UP, c3, c2},   {14, L_CONV, 2 * c2, c2},
                 {16, L_CONV, c2, c2},     {18, L_UP, c2, c1},       {20, L_CONV, 2 * c1, c1}, {22, L_CONV, c1, c1},
                 {24, L_OUT, c1, 2}};
    // He-normal weights from a seeded Mersenne twister (Box-Muller), zero biases
    std::mt19937_64 rng(seed);
    auto unif = [&]() { return ((double)(rng() >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
    std::vector<float> host;
    cs_status st = CS_OK;
    for (const Layer& L : n->layers) {
        const int64_t nw = L.kind == L_CONV ? (int64_t)L.cout * 27 * L.cin : L.kind == L_UP ? (int64_t)L.cout * 8 * L.cin
                                                                                             : (int64_t)L.cout * L.cin;
        const double scale = L.kind == L_CONV ? std::sqrt(2.0 / (27.0 * L.cin))
                             : L.kind == L_UP ? std::sqrt(1.0 / L.cin)
                                              : 0.1 * std::sqrt(1.0 / L.cin);
        n->numel[L.pi] = nw;
        n->numel[L.pi + 1] = L.cout;
        host.assign((size_t)nw, 0.f);
        for (int64_t i = 0; i < nw; i += 2) {
            const double r = std::sqrt(-2.0 * std::log(unif())), th = 6.283185307179586 * unif();
            host[(size_t)i] = (float)(scale * r * std::cos(th));
            if (i + 1 < nw) host[(size_t)i + 1] = (float)(scale * r * std::sin(th));
        }
        for (int k = 0; k < 2 && st == CS_OK; ++k) {
            const int pi = L.pi + k;
            const size_t bytes = (size_t)n->numel[pi] * sizeof(float);
            if (cudaMalloc(&n->p[pi], bytes) != cudaSuccess || cudaMalloc(&n->g[pi], bytes) != cudaSuccess ||
                cudaMalloc(&n->m[pi], bytes) != cudaSuccess || cudaMalloc(&n->v[pi], bytes) != cudaSuccess) {
                set_error("U-Net parameter allocation failed");
                st = CS_ERR_OOM;
                break;
            }
            cudaMemset(n->m[pi], 0, bytes);
            cudaMemset(n->v[pi], 0, bytes);
            cudaMemset(n->g[pi], 0, bytes);
            if (k == 0) {
                if (cudaMemcpy(n->p[pi], host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) st = CS_ERR_CUDA;
            } else {
                cudaMemset(n->p[pi], 0, bytes);
            }
        }
        if (st == CS_OK && L.kind == L_CONV) {
            n->np_f[L.pi] = npad_of(L.cout);
            n->kp_f[L.pi] = kpad_of(27 * L.cin);
            if (cudaMalloc(&n->pk_f[L.pi], (size_t)n->np_f[L.pi] * n->kp_f[L.pi] * 2) != cudaSuccess) st = CS_ERR_OOM;
            if (L.pi > 0 && st == CS_OK) {
                n->np_t[L.pi] = npad_of(L.cin);
                n->kp_t[L.pi] = kpad_of(27 * L.cout);
                if (cudaMalloc(&n->pk_t[L.pi], (size_t)n->np_t[L.pi] * n->kp_t[L.pi] * 2) != cudaSuccess) st = CS_ERR_OOM;
            }
        }
        if (st != CS_OK) break;
    }
    if (st != CS_OK) {
        if (st == CS_ERR_CUDA) set_error("U-Net parameter upload failed");
        destroy(n);
        return st;
    }
    *out = n;
    return CS_OK;
}

cs_status ws_net_destroy(cs_unet* net) {
    clear_error();
    if (net) destroy(net);
    return CS_OK;
}

cs_status ws_net_param(cs_unet* net, int which, int index, const float* src, float* dst, int64_t* numel, void* stream) {
    clear_error();
    CS_REQUIRE(net && index >= 0 && index < kParams && which >= 0 && which <= 3, CS_ERR_INVALID_ARG,
               "bad parameter index");
    float* arr = which == 0 ? net->p[index] : which == 1 ? net->g[index] : which == 2 ? net->m[index] : net->v[index];
    const size_t bytes = (size_t)net->numel[index] * sizeof(float);
    cudaStream_t st = (cudaStream_t)stream;
    if (numel) *numel = net->numel[index];
    if (src) {
        CS_TRY_CUDA(cudaMemcpyAsync(arr, src, bytes, cudaMemcpyDeviceToDevice, st));
        if (which == 0) net->packed = false;
    }
    if (dst) CS_TRY_CUDA(cudaMemcpyAsync(dst, arr, bytes, cudaMemcpyDeviceToDevice, st));
    return CS_OK;
}

cs_status ws_net_infer(cs_unet* net, const float* xt, const float* d, const int* dims, float eta, float* xhat,
                       void* stream) {
    clear_error();
    CS_REQUIRE(net && xt && d && xhat, CS_ERR_INVALID_ARG, "null pointer");
    CS_PROPAGATE(check_dims(net, dims));
    CS_PROPAGATE(ensure_bufs(net, dims, false));
    const int64_t n = (int64_t)dims[0] * dims[1] * dims[2];
    CS_PROPAGATE(nn_features_det((const float2*)xt, (const float2*)d, n, eta, nullptr, net->fpart, net->ss, net->f,
                                 (cudaStream_t)stream));
    CS_PROPAGATE(forward(net, stream));
    return cs_nn_apply(xt, net->out, n, net->ss, xhat, stream);
}

cs_status ws_net_train_step(cs_unet* net, const float* xt, const float* d, const float* target, const int* dims,
                            float eta, float lr, float* loss, void* stream) {
    clear_error();
    CS_REQUIRE(net && xt && d && target && lr > 0.f, CS_ERR_INVALID_ARG, "bad train-step arguments");
    CS_PROPAGATE(check_dims(net, dims));
    CS_PROPAGATE(ensure_bufs(net, dims, true));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = (int64_t)dims[0] * dims[1] * dims[2];
    CS_PROPAGATE(nn_features_det((const float2*)xt, (const float2*)d, n, eta, nullptr, net->fpart, net->ss, net->f, st));
    CS_PROPAGATE(cs_nn_target(xt, target, n, net->ss, net->tgt, stream));
    CS_PROPAGATE(forward(net, stream));
    float* lacc = net->ss + 1;
    CS_TRY_CUDA(cudaMemsetAsync(lacc, 0, sizeof(float), st));
    CS_PROPAGATE(cs_nn_mse(net->out, net->tgt, 2 * n, net->gout, lacc, stream));
    if (loss) CS_TRY_CUDA(cudaMemcpyAsync(loss, lacc, sizeof(float), cudaMemcpyDeviceToDevice, st));
    CS_PROPAGATE(backward(net, stream));
    net->step += 1;
    for (int i = 0; i < kParams; ++i)
        CS_PROPAGATE(cs_nn_adam(net->p[i], net->g[i], net->m[i], net->v[i], net->numel[i], lr, 0.9f, 0.999f, 1e-8f,
                                net->step, stream));
    net->packed = false;
    return CS_OK;
}

cs_status ws_net_save(cs_unet* net, const char* path) {
    clear_error();
    CS_REQUIRE(net && path, CS_ERR_INVALID_ARG, "null pointer");
    CS_TRY_CUDA(cudaDeviceSynchronize());
    FILE* fp = std::fopen(path, "wb");
    CS_REQUIRE(fp, CS_ERR_INVALID_ARG, "cannot open %s for writing", path);
    const int32_t hdr[4] = {net->c1, net->c2, net->c3, net->step};
    bool ok = std::fwrite(kMagic, 1, 8, fp) == 8 && std::fwrite(hdr, sizeof(int32_t), 4, fp) == 4;
    std::vector<float> h;
    for (int i = 0; i < kParams && ok; ++i) {
        h.resize((size_t)net->numel[i]);
        for (float* arr : {net->p[i], net->m[i], net->v[i]}) {
            if (cudaMemcpy(h.data(), arr, h.size() * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
                std::fwrite(h.data(), sizeof(float), h.size(), fp) != h.size()) {
                ok = false;
                break;
            }
        }
    }
    ok = (std::fclose(fp) == 0) && ok;
    CS_REQUIRE(ok, CS_ERR_INVALID_ARG, "writing %s failed", path);
    return CS_OK;
}

cs_status ws_net_load(cs_unet* net, const char* path) {
    clear_error();
    CS_REQUIRE(net && path, CS_ERR_INVALID_ARG, "null pointer");
    FILE* fp = std::fopen(path, "rb");
    CS_REQUIRE(fp, CS_ERR_INVALID_ARG, "cannot open %s", path);
    char magic[8] = {};
    int32_t hdr[4] = {};
    bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(hdr, sizeof(int32_t), 4, fp) == 4 && hdr[0] == net->c1 && hdr[1] == net->c2 &&
              hdr[2] == net->c3 && hdr[3] >= 0;
    std::vector<float> h;
    for (int i = 0; i < kParams && ok; ++i) {
        h.resize((size_t)net->numel[i]);
        for (float* arr : {net->p[i], net->m[i], net->v[i]}) {
            if (std::fread(h.data(), sizeof(float), h.size(), fp) != h.size() ||
                cudaMemcpy(arr, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
                ok = false;
                break;
            }
        }
    }
    std::fclose(fp);
    CS_REQUIRE(ok, CS_ERR_INVALID_ARG, "%s is not a U-Net of widths %d/%d/%d saved by ws_net_save", path, net->c1,
               net->c2, net->c3);
    net->step = hdr[3];
    net->packed = false;
    return CS_OK;
}

}  // extern "C"
