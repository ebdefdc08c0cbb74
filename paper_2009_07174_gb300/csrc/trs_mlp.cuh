// trs_mlp.cuh -- frontier predictor: feature extraction and warp-cooperative
// BF16 inference with FP32 accumulation.  Included by the engine kernel (the
// learned frontier's refresh) and by the predictor's own kernels.
//
// The predictor sees one node's local view: its head symbol h, the head
// symbols a_j of its arguments (0 where the head has fewer arguments) and the
// bits b_j telling which arguments are in normal form.  Input x is the
// concatenation of one-hot codes [h | a_0 | ... | a_{MA-1}] and the bits, of
// dimension D = nsym * (1 + MA) + MA; then h1 = relu(W1 x + b1),
// h2 = relu(W2 h1 + b2), p = sigmoid(w3 . h2 + b3), hidden width 32.
//
// Layout of the inference block (bytes, all offsets 16-aligned):
//   w1t  bf16 [D][32]   column d of W1 (one 64-byte row per input feature)
//   w2t  bf16 [32][32]  w2t[i][o] = W2[o][i]
//   w3   bf16 [32]
//   b1, b2 f32 [32], b3 f32
// Lane o of a warp owns hidden unit o: every weight read is a contiguous,
// conflict-free row of shared memory, and the hidden vector moves between
// lanes by shuffles.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace trs {

constexpr int kHidden = 32;

struct MlpLayout {
    int D;
    size_t w1t, w2t, w3, b1, b2, b3, total;
};

__host__ __device__ inline size_t mlp_up16(size_t x) { return (x + 15) / 16 * 16; }

__host__ __device__ inline MlpLayout mlp_layout(int nsym, int ma)
{
    MlpLayout L;
    L.D = nsym * (1 + ma) + ma;
    size_t off = 0;
    L.w1t = off; off = mlp_up16(off + (size_t)L.D * kHidden * 2);
    L.w2t = off; off = mlp_up16(off + (size_t)kHidden * kHidden * 2);
    L.w3 = off; off = mlp_up16(off + kHidden * 2);
    L.b1 = off; off = mlp_up16(off + kHidden * 4);
    L.b2 = off; off = mlp_up16(off + kHidden * 4);
    L.b3 = off; off = mlp_up16(off + 4);
    L.total = off;
    return L;
}

struct MlpView {
    const __nv_bfloat16 *w1t, *w2t, *w3;
    const float *b1, *b2, *b3;
    int D, nsym, ma;
};

__device__ __forceinline__ MlpView mlp_view(const unsigned char *base, int nsym, int ma)
{
    const MlpLayout L = mlp_layout(nsym, ma);
    MlpView M;
    M.w1t = (const __nv_bfloat16 *)(base + L.w1t);
    M.w2t = (const __nv_bfloat16 *)(base + L.w2t);
    M.w3 = (const __nv_bfloat16 *)(base + L.w3);
    M.b1 = (const float *)(base + L.b1);
    M.b2 = (const float *)(base + L.b2);
    M.b3 = (const float *)(base + L.b3);
    M.D = L.D;
    M.nsym = nsym;
    M.ma = ma;
    return M;
}

// Probability for the node of every lane with `has` set (0 elsewhere).  All 32
// lanes must call.  a[j] for j < ma, bits bit j = argument j in normal form.
__device__ __forceinline__ float mlp_warp_prob(const MlpView &M, bool has, int h, const int32_t *a,
                                               unsigned bits)
{
    const unsigned full = 0xffffffffu;
    const int o = threadIdx.x & 31;
    const float b1o = M.b1[o], b2o = M.b2[o];
    const float w3o = __bfloat162float(M.w3[o]);
    const float b3 = M.b3[0];
    float result = 0.f;
    unsigned todo = __ballot_sync(full, has);
    while (todo) {
        const int c = __ffs(todo) - 1;
        todo &= todo - 1;
        const int hc = __shfl_sync(full, h, c);
        const unsigned bc = __shfl_sync(full, bits, c);
        float z1 = b1o + __bfloat162float(M.w1t[hc * kHidden + o]);
        for (int j = 0; j < M.ma; j++) {
            const int ac = __shfl_sync(full, a[j], c);
            z1 += __bfloat162float(M.w1t[(M.nsym * (1 + j) + ac) * kHidden + o]);
            if ((bc >> j) & 1u) z1 += __bfloat162float(M.w1t[(M.nsym * (1 + M.ma) + j) * kHidden + o]);
        }
        const float h1 = fmaxf(z1, 0.f);
        float z2 = b2o;
#pragma unroll
        for (int i = 0; i < kHidden; i++)
            z2 = fmaf(__bfloat162float(M.w2t[i * kHidden + o]), __shfl_sync(full, h1, i), z2);
        float t = w3o * fmaxf(z2, 0.f);
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) t += __shfl_xor_sync(full, t, s);
        if (o == c) result = 1.f / (1.f + expf(-(t + b3)));
    }
    return result;
}

}  // namespace trs
