// trs_mlp.cu -- the learned frontier's predictor: training kernels (forward,
// backward, Adam, all FP32), export of the BF16 inference block, inference
// kernels, and the predictor half of the C ABI.  The network and its input
// encoding are described in trs_mlp.cuh.
//
// Training is warp-cooperative like inference: lane o of a warp owns hidden
// unit o of the sample the warp is working on; the hidden vectors move between
// lanes by shuffles.  Gradients accumulate per block in shared memory (lane o
// keeps row o of dW2 in registers) and reach global memory with one atomic per
// parameter per block.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "trs_engine.h"
#include "trs_mlp.cuh"

using namespace trs;

struct trs_predictor {
    const trs_program *prog = nullptr;
    int nsym = 0, ma = 0, D = 0, F = 0;
    long long P = 0;      // parameter count
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    float *loss = nullptr;  // one float accumulator
    unsigned char *infer = nullptr;
    size_t infer_bytes = 0;
    long long step = 0;   // Adam step counter
};

namespace {

constexpr int H = kHidden;

struct PLayout {
    long long w1, b1, w2, b2, w3, b3, total;  // offsets in floats
};

PLayout playout(int D)
{
    PLayout L;
    L.w1 = 0;
    L.b1 = L.w1 + (long long)H * D;
    L.w2 = L.b1 + H;
    L.b2 = L.w2 + H * H;
    L.w3 = L.b2 + H;
    L.b3 = L.w3 + H;
    L.total = L.b3 + 1;
    return L;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

struct MemLayout {
    size_t theta, grad, m, v, loss, infer, total;
};

MemLayout mlayout(int nsym, int ma)
{
    const int D = nsym * (1 + ma) + ma;
    const size_t pb = (size_t)playout(D).total * sizeof(float);
    MemLayout L;
    size_t off = 0;
    L.theta = off; off = up256(off + pb);
    L.grad = off; off = up256(off + pb);
    L.m = off; off = up256(off + pb);
    L.v = off; off = up256(off + pb);
    L.loss = off; off = up256(off + 16);
    L.infer = off; off = up256(off + mlp_layout(nsym, ma).total);
    L.total = off;
    return L;
}

size_t train_smem_bytes(int D)
{
    // W1T, gW1T: D x H; W2, W2T, gW2: H x H; b1, b2, w3, gb1, gb2, gw3: H; b3, gb3, loss
    return ((size_t)2 * D * H + 3 * H * H + 6 * H + 8) * sizeof(float);
}

__device__ __forceinline__ float softplus(float x) { return fmaxf(x, 0.f) + log1pf(expf(-fabsf(x))); }

// One forward/backward pass over samples [lo, hi): gradients of the mean
// (over `count` samples) weighted binary cross-entropy are added to grad,
// the loss sum to *loss.
__global__ void __launch_bounds__(256)
k_mlp_grad(const float *theta, float *grad, const int32_t *feat, const float *label, long long lo,
           long long hi, int nsym, int ma, int D, float pos_weight, float inv_count, float *loss)
{
    extern __shared__ float sm[];
    float *W1T = sm;                       // [D][H]
    float *gW1T = W1T + D * H;             // [D][H]
    float *W2 = gW1T + D * H;              // [H][H] (o, i)
    float *W2T = W2 + H * H;               // [H][H] (i, o)
    float *gW2 = W2T + H * H;              // [H][H] (o, i)
    float *b1 = gW2 + H * H, *b2 = b1 + H, *w3 = b2 + H;
    float *gb1 = w3 + H, *gb2 = gb1 + H, *gw3 = gb2 + H;
    float *misc = gw3 + H;                 // b3, gb3, loss
    const long long o_b1 = (long long)H * D, o_w2 = o_b1 + H, o_b2 = o_w2 + H * H;
    const long long o_w3 = o_b2 + H, o_b3 = o_w3 + H;
    for (int t = threadIdx.x; t < D * H; t += blockDim.x) {
        const int d = t / H, o = t % H;
        W1T[t] = theta[(long long)o * D + d];
        gW1T[t] = 0.f;
    }
    for (int t = threadIdx.x; t < H * H; t += blockDim.x) {
        const int o = t / H, i = t % H;
        W2[t] = theta[o_w2 + t];
        W2T[i * H + o] = theta[o_w2 + t];
        gW2[t] = 0.f;
    }
    for (int t = threadIdx.x; t < H; t += blockDim.x) {
        b1[t] = theta[o_b1 + t];
        b2[t] = theta[o_b2 + t];
        w3[t] = theta[o_w3 + t];
        gb1[t] = gb2[t] = gw3[t] = 0.f;
    }
    if (threadIdx.x == 0) { misc[0] = theta[o_b3]; misc[1] = 0.f; misc[2] = 0.f; }
    __syncthreads();

    const unsigned full = 0xffffffffu;
    const int o = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int F = 2 + ma;
    float acc_w2[H];
#pragma unroll
    for (int i = 0; i < H; i++) acc_w2[i] = 0.f;
    float a_b1 = 0.f, a_b2 = 0.f, a_w3 = 0.f, a_b3 = 0.f, a_loss = 0.f;
    for (long long s = lo + warp; s < hi; s += nwarps) {
        const int32_t *f = feat + s * F;
        const int hsym = f[0];
        const unsigned bits = (unsigned)f[1 + ma];
        // forward
        float z1 = b1[o] + W1T[hsym * H + o];
        for (int j = 0; j < ma; j++) {
            z1 += W1T[(nsym * (1 + j) + f[1 + j]) * H + o];
            if ((bits >> j) & 1u) z1 += W1T[(nsym * (1 + ma) + j) * H + o];
        }
        const float h1 = fmaxf(z1, 0.f);
        float z2 = b2[o];
#pragma unroll
        for (int i = 0; i < H; i++) z2 = fmaf(W2T[i * H + o], __shfl_sync(full, h1, i), z2);
        const float h2 = fmaxf(z2, 0.f);
        float z = w3[o] * h2;
#pragma unroll
        for (int sft = 16; sft > 0; sft >>= 1) z += __shfl_xor_sync(full, z, sft);
        z += misc[0];
        // loss and its derivative
        const float y = label[s];
        const float sig = 1.f / (1.f + expf(-z));
        if (o == 0) a_loss += pos_weight * y * softplus(-z) + (1.f - y) * softplus(z);
        const float dz = (sig * (pos_weight * y + 1.f - y) - pos_weight * y) * inv_count;
        // backward
        const float dh2 = z2 > 0.f ? dz * w3[o] : 0.f;
        a_w3 += dz * h2;
        a_b2 += dh2;
        if (o == 0) a_b3 += dz;
        float dh1 = 0.f;
#pragma unroll
        for (int i = 0; i < H; i++) {
            acc_w2[i] = fmaf(dh2, __shfl_sync(full, h1, i), acc_w2[i]);   // dW2[o][i]
            dh1 = fmaf(W2[i * H + o], __shfl_sync(full, dh2, i), dh1);     // sum_q W2[q][o] dh2[q]
        }
        dh1 = z1 > 0.f ? dh1 : 0.f;
        a_b1 += dh1;
        atomicAdd(&gW1T[hsym * H + o], dh1);
        for (int j = 0; j < ma; j++) {
            atomicAdd(&gW1T[(nsym * (1 + j) + f[1 + j]) * H + o], dh1);
            if ((bits >> j) & 1u) atomicAdd(&gW1T[(nsym * (1 + ma) + j) * H + o], dh1);
        }
    }
#pragma unroll
    for (int i = 0; i < H; i++) atomicAdd(&gW2[o * H + i], acc_w2[i]);
    atomicAdd(&gb1[o], a_b1);
    atomicAdd(&gb2[o], a_b2);
    atomicAdd(&gw3[o], a_w3);
    if (o == 0) {
        atomicAdd(&misc[1], a_b3);
        atomicAdd(&misc[2], a_loss);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < D * H; t += blockDim.x) {
        const int d = t / H, oo = t % H;
        if (gW1T[t] != 0.f) atomicAdd(&grad[(long long)oo * D + d], gW1T[t]);
    }
    for (int t = threadIdx.x; t < H * H; t += blockDim.x) atomicAdd(&grad[o_w2 + t], gW2[t]);
    for (int t = threadIdx.x; t < H; t += blockDim.x) {
        atomicAdd(&grad[o_b1 + t], gb1[t]);
        atomicAdd(&grad[o_b2 + t], gb2[t]);
        atomicAdd(&grad[o_w3 + t], gw3[t]);
    }
    if (threadIdx.x == 0) {
        atomicAdd(&grad[o_b3], misc[1]);
        atomicAdd(loss, misc[2]);
    }
}

// Adam (bias-corrected moments, eps outside the square root); clears grad.
__global__ void k_adam(float *theta, float *grad, float *m, float *v, long long P, float lr, float b1,
                       float b2, float eps, float c1, float c2)
{
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < P;
         e += (long long)gridDim.x * blockDim.x) {
        const float g = grad[e];
        const float mm = b1 * m[e] + (1.f - b1) * g;
        const float vv = b2 * v[e] + (1.f - b2) * g * g;
        m[e] = mm;
        v[e] = vv;
        theta[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
        grad[e] = 0.f;
    }
}

// BF16 inference block from the FP32 parameters (round to nearest even).
__global__ void k_mlp_export(const float *theta, unsigned char *out, int nsym, int ma)
{
    const MlpLayout L = mlp_layout(nsym, ma);
    const int D = L.D;
    __nv_bfloat16 *w1t = (__nv_bfloat16 *)(out + L.w1t);
    __nv_bfloat16 *w2t = (__nv_bfloat16 *)(out + L.w2t);
    __nv_bfloat16 *w3 = (__nv_bfloat16 *)(out + L.w3);
    float *b1 = (float *)(out + L.b1), *b2 = (float *)(out + L.b2), *b3 = (float *)(out + L.b3);
    const long long o_b1 = (long long)H * D, o_w2 = o_b1 + H, o_b2 = o_w2 + H * H;
    const long long o_w3 = o_b2 + H, o_b3 = o_w3 + H;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < D * H; t += gridDim.x * blockDim.x) {
        const int d = t / H, o = t % H;
        w1t[t] = __float2bfloat16_rn(theta[(long long)o * D + d]);
    }
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < H * H; t += gridDim.x * blockDim.x) {
        const int i = t / H, o = t % H;
        w2t[t] = __float2bfloat16_rn(theta[o_w2 + o * H + i]);
    }
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < H; t += gridDim.x * blockDim.x) {
        w3[t] = __float2bfloat16_rn(theta[o_w3 + t]);
        b1[t] = theta[o_b1 + t];
        b2[t] = theta[o_b2 + t];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) b3[0] = theta[o_b3];
}

// BF16 inference (the engine's path): probability per feature row.
__global__ void k_mlp_infer(const unsigned char *blk, const int32_t *feat, long long n, int nsym, int ma,
                            float *prob)
{
    const MlpView M = mlp_view(blk, nsym, ma);
    const int F = 2 + ma;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (long long base = w0 * 32; base < n; base += nw * 32) {
        const long long s = base + lane;
        const bool has = s < n;
        int32_t a[TRS_MAX_ARITY] = {0, 0, 0, 0, 0, 0, 0, 0};
        int h = 0;
        unsigned bits = 0;
        if (has) {
            h = feat[s * F];
            for (int j = 0; j < ma; j++) a[j] = feat[s * F + 1 + j];
            bits = (unsigned)feat[s * F + 1 + ma];
        }
        const float p = mlp_warp_prob(M, has, h, a, bits);
        if (has) prob[s] = p;
    }
}

// FP32 logits, one thread per row (reference path for tests).
__global__ void k_mlp_logits32(const float *theta, const int32_t *feat, long long n, int nsym, int ma,
                               int D, float *out)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int F = 2 + ma;
    const int32_t *f = feat + s * F;
    const long long o_b1 = (long long)H * D, o_w2 = o_b1 + H, o_b2 = o_w2 + H * H;
    const long long o_w3 = o_b2 + H, o_b3 = o_w3 + H;
    float h1[H];
    for (int o = 0; o < H; o++) {
        const float *w = theta + (long long)o * D;
        float z = theta[o_b1 + o] + w[f[0]];
        for (int j = 0; j < ma; j++) {
            z += w[nsym * (1 + j) + f[1 + j]];
            if (((unsigned)f[1 + ma] >> j) & 1u) z += w[nsym * (1 + ma) + j];
        }
        h1[o] = fmaxf(z, 0.f);
    }
    float z = theta[o_b3];
    for (int o = 0; o < H; o++) {
        float z2 = theta[o_b2 + o];
        for (int i = 0; i < H; i++) z2 = fmaf(theta[o_w2 + o * H + i], h1[i], z2);
        z = fmaf(theta[o_w3 + o], fmaxf(z2, 0.f), z);
    }
    out[s] = z;
}

int fail(const std::string &m, int code)
{
    set_error(m);
    return code;
}

#define CKP(call, what)                                                          \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) return fail(std::string(what) + ": " + cudaGetErrorString(e_), TRS_ERR_CUDA); \
    } while (0)

int export_block(trs_predictor *p, cudaStream_t stream)
{
    k_mlp_export<<<8, 256, 0, stream>>>(p->theta, p->infer, p->nsym, p->ma);
    CKP(cudaGetLastError(), "predictor export");
    return TRS_OK;
}

size_t samples_label_offset(int F, int64_t cap)
{
    return up256((size_t)cap * F * sizeof(int32_t)) + up256((size_t)cap * sizeof(int32_t));
}

}  // namespace

namespace trs {
// used by the engine (trs_api.cu)
const unsigned char *predictor_block(const trs_predictor *p) { return p ? p->infer : nullptr; }
size_t predictor_block_bytes(const trs_predictor *p) { return p ? p->infer_bytes : 0; }
const trs_program *predictor_program(const trs_predictor *p) { return p ? p->prog : nullptr; }
}  // namespace trs

extern "C" {

int trs_predictor_bytes(const trs_program *prog, size_t *bytes)
{
    if (!prog || !bytes) return fail("trs_predictor_bytes: bad argument", TRS_ERR_ARG);
    const int nsym = prog->p.nsym, ma = prog->p.maxarity;
    const int D = nsym * (1 + ma) + ma;
    if (train_smem_bytes(D) > 200 * 1024)
        return fail("trs_predictor_bytes: signature too large for the predictor's input", TRS_ERR_TOO_BIG);
    *bytes = mlayout(nsym, ma).total;
    return TRS_OK;
}

int trs_predictor_create(const trs_program *prog, uint64_t seed, void *dev_mem, size_t bytes,
                         trs_stream stream, trs_predictor **out)
{
    if (!out) return fail("trs_predictor_create: out is NULL", TRS_ERR_ARG);
    *out = nullptr;
    size_t need = 0;
    int st = trs_predictor_bytes(prog, &need);
    if (st != TRS_OK) return st;
    if (!dev_mem || bytes < need || ((uintptr_t)dev_mem % 256) != 0)
        return fail("trs_predictor_create: memory too small or not 256-byte aligned", TRS_ERR_ARG);
    trs_predictor *p = new trs_predictor;
    p->prog = prog;
    p->nsym = prog->p.nsym;
    p->ma = prog->p.maxarity;
    p->D = p->nsym * (1 + p->ma) + p->ma;
    p->F = 2 + p->ma;
    p->P = playout(p->D).total;
    const MemLayout L = mlayout(p->nsym, p->ma);
    unsigned char *b = (unsigned char *)dev_mem;
    p->theta = (float *)(b + L.theta);
    p->grad = (float *)(b + L.grad);
    p->m = (float *)(b + L.m);
    p->v = (float *)(b + L.v);
    p->loss = (float *)(b + L.loss);
    p->infer = b + L.infer;
    p->infer_bytes = mlp_layout(p->nsym, p->ma).total;
    // He-style uniform initialisation from a splitmix64 stream; biases 0
    std::vector<float> h(p->P, 0.f);
    uint64_t x = seed ? seed : 0x9E3779B97F4A7C15ull;
    auto next = [&]() {
        x += 0x9E3779B97F4A7C15ull;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    const PLayout PL = playout(p->D);
    const double a1 = std::sqrt(6.0 / (1 + 2 * p->ma)), a2 = std::sqrt(6.0 / H), a3 = std::sqrt(3.0 / H);
    for (long long e = PL.w1; e < PL.b1; e++) h[e] = (float)((2 * next() - 1) * a1);
    for (long long e = PL.w2; e < PL.b2; e++) h[e] = (float)((2 * next() - 1) * a2);
    for (long long e = PL.w3; e < PL.b3; e++) h[e] = (float)((2 * next() - 1) * a3);
    cudaError_t e = cudaMemsetAsync(dev_mem, 0, L.total, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->theta, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) { delete p; return fail(std::string("trs_predictor_create: ") + cudaGetErrorString(e), TRS_ERR_CUDA); }
    st = export_block(p, stream);
    if (st != TRS_OK) { delete p; return st; }
    *out = p;
    return TRS_OK;
}

void trs_predictor_free(trs_predictor *p) { delete p; }

int trs_predictor_shape(const trs_predictor *p, int32_t *input_dim, int64_t *nparams)
{
    if (!p) return fail("trs_predictor_shape: bad argument", TRS_ERR_ARG);
    if (input_dim) *input_dim = p->D;
    if (nparams) *nparams = p->P;
    return TRS_OK;
}

int trs_predictor_get(trs_predictor *p, float *host, int64_t n, trs_stream stream)
{
    if (!p || !host || n != p->P) return fail("trs_predictor_get: bad argument", TRS_ERR_ARG);
    CKP(cudaMemcpyAsync(host, p->theta, n * sizeof(float), cudaMemcpyDeviceToHost, stream), "predictor get");
    CKP(cudaStreamSynchronize(stream), "predictor get");
    return TRS_OK;
}

int trs_predictor_set(trs_predictor *p, const float *host, int64_t n, trs_stream stream)
{
    if (!p || !host || n != p->P) return fail("trs_predictor_set: bad argument", TRS_ERR_ARG);
    CKP(cudaMemcpyAsync(p->theta, host, n * sizeof(float), cudaMemcpyHostToDevice, stream), "predictor set");
    CKP(cudaMemsetAsync(p->grad, 0, n * sizeof(float), stream), "predictor set");
    CKP(cudaMemsetAsync(p->m, 0, n * sizeof(float), stream), "predictor set");
    CKP(cudaMemsetAsync(p->v, 0, n * sizeof(float), stream), "predictor set");
    p->step = 0;
    int st = export_block(p, stream);
    if (st != TRS_OK) return st;
    CKP(cudaStreamSynchronize(stream), "predictor set");
    return TRS_OK;
}

void trs_train_opts_default(trs_train_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->epochs = 20;
    o->batch = 4096;
    o->lr = 1e-2f;
    o->beta1 = 0.9f;
    o->beta2 = 0.999f;
    o->eps = 1e-8f;
    o->pos_weight = 1.f;
}

int trs_samples_bytes(const trs_program *prog, int64_t cap, size_t *bytes)
{
    if (!prog || !bytes || cap <= 0) return fail("trs_samples_bytes: bad argument", TRS_ERR_ARG);
    const int F = 2 + prog->p.maxarity;
    *bytes = samples_label_offset(F, cap) + up256((size_t)cap * sizeof(float));
    return TRS_OK;
}

static int grad_pass(trs_predictor *p, const void *samples, int64_t cap, int64_t lo, int64_t hi,
                     int64_t count, float pos_weight, cudaStream_t stream)
{
    const int32_t *feat = (const int32_t *)samples;
    const float *label = (const float *)((const unsigned char *)samples + samples_label_offset(p->F, cap));
    const size_t smem = train_smem_bytes(p->D);
    CKP(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "train config");
    int dev = 0, sms = 0;
    CKP(cudaGetDevice(&dev), "train config");
    CKP(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "train config");
    const long long rows = hi - lo;
    int grid = (int)std::min<long long>(sms, std::max<long long>(1, rows / 256));
    k_mlp_grad<<<grid, 256, smem, stream>>>(p->theta, p->grad, feat, label, lo, hi, p->nsym, p->ma, p->D,
                                             pos_weight, 1.f / (float)count, p->loss);
    CKP(cudaGetLastError(), "train launch");
    return TRS_OK;
}

int trs_predictor_grad(trs_predictor *p, const void *samples, int64_t cap, int64_t n, float pos_weight,
                       float *host_grad, float *host_loss, trs_stream stream)
{
    if (!p || !samples || n <= 0 || n > cap || !host_grad)
        return fail("trs_predictor_grad: bad argument", TRS_ERR_ARG);
    CKP(cudaMemsetAsync(p->grad, 0, p->P * sizeof(float), stream), "grad");
    CKP(cudaMemsetAsync(p->loss, 0, sizeof(float), stream), "grad");
    int st = grad_pass(p, samples, cap, 0, n, n, pos_weight, stream);
    if (st != TRS_OK) return st;
    CKP(cudaMemcpyAsync(host_grad, p->grad, p->P * sizeof(float), cudaMemcpyDeviceToHost, stream), "grad");
    float l = 0.f;
    CKP(cudaMemcpyAsync(&l, p->loss, sizeof(float), cudaMemcpyDeviceToHost, stream), "grad");
    CKP(cudaMemsetAsync(p->grad, 0, p->P * sizeof(float), stream), "grad");
    CKP(cudaStreamSynchronize(stream), "grad");
    if (host_loss) *host_loss = l / (float)n;
    return TRS_OK;
}

int trs_predictor_train(trs_predictor *p, const void *samples, int64_t cap, int64_t n,
                        const trs_train_opts *opts, float *epoch_loss, trs_stream stream)
{
    if (!p || !samples || n <= 0 || n > cap) return fail("trs_predictor_train: bad argument", TRS_ERR_ARG);
    trs_train_opts o;
    if (opts) o = *opts;
    else trs_train_opts_default(&o);
    if (o.epochs <= 0 || o.batch <= 0 || !(o.lr > 0.f) || !(o.pos_weight > 0.f))
        return fail("trs_predictor_train: invalid options", TRS_ERR_ARG);
    for (int ep = 0; ep < o.epochs; ep++) {
        CKP(cudaMemsetAsync(p->loss, 0, sizeof(float), stream), "train");
        for (int64_t lo = 0; lo < n; lo += o.batch) {
            const int64_t hi = std::min<int64_t>(n, lo + o.batch);
            int st = grad_pass(p, samples, cap, lo, hi, hi - lo, o.pos_weight, stream);
            if (st != TRS_OK) return st;
            p->step++;
            const float c1 = 1.f - (float)std::pow((double)o.beta1, (double)p->step);
            const float c2 = 1.f - (float)std::pow((double)o.beta2, (double)p->step);
            k_adam<<<64, 256, 0, stream>>>(p->theta, p->grad, p->m, p->v, p->P, o.lr, o.beta1, o.beta2,
                                           o.eps, c1, c2);
            CKP(cudaGetLastError(), "adam launch");
        }
        if (epoch_loss) {
            float l = 0.f;
            CKP(cudaMemcpyAsync(&l, p->loss, sizeof(float), cudaMemcpyDeviceToHost, stream), "train loss");
            CKP(cudaStreamSynchronize(stream), "train loss");
            // sum over batches of (sum of sample losses / batch size) * batch size
            epoch_loss[ep] = l / (float)n;
        }
    }
    return export_block(p, stream);
}

int trs_predictor_infer(trs_predictor *p, const int32_t *dev_feat, int64_t n, float *dev_prob,
                        trs_stream stream)
{
    if (!p || !dev_feat || !dev_prob || n < 0) return fail("trs_predictor_infer: bad argument", TRS_ERR_ARG);
    if (n == 0) return TRS_OK;
    const long long blocks = std::min<long long>(4096, (n + 255) / 256);
    k_mlp_infer<<<(unsigned)blocks, 256, 0, stream>>>(p->infer, dev_feat, n, p->nsym, p->ma, dev_prob);
    CKP(cudaGetLastError(), "infer launch");
    return TRS_OK;
}

int trs_predictor_logits32(trs_predictor *p, const int32_t *dev_feat, int64_t n, float *dev_logit,
                           trs_stream stream)
{
    if (!p || !dev_feat || !dev_logit || n < 0) return fail("trs_predictor_logits32: bad argument", TRS_ERR_ARG);
    if (n == 0) return TRS_OK;
    k_mlp_logits32<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(p->theta, dev_feat, n, p->nsym, p->ma,
                                                                    p->D, dev_logit);
    CKP(cudaGetLastError(), "logits launch");
    return TRS_OK;
}

}  // extern "C"
