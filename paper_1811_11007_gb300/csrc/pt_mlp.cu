// Learned warm start for the proposal Newton iterations: a 69 -> 128 -> 128 -> 5
// GELU MLP with BF16 weights and activations and FP32 accumulation on the
// tensor cores (mma.sync m16n8k16), its backward pass and Adam, the feature
// kernels, and the logging of (features, optimised lengths) pairs.
//
// Features of an NNI neighbour, in post-swap member order (A, X2 at u; B, Y2
// at v): the logs of the five inherited lengths (central, A, X2, B, Y2), then
// a 16-value summary of each member's partial-likelihood vector (the
// pattern-weighted mean over sites of the site's vector divided by its sum,
// [category][state]).  Targets: the logs of the five optimised lengths in the
// same order, as log-ratios to the inherited lengths (the network predicts
// log(optimised / inherited), so an all-zero network is the plain start).  The
// prediction only sets where Newton starts; a start that is not finite or
// falls outside the length bounds is replaced by the inherited length, so
// results stay those of the plain start up to the Newton tolerance.
#include "pt_internal.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

namespace pt {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kIn = kMlpIn, kInP = kMlpInPad, kH = kMlpHidden, kOutP = kMlpOutPad;
constexpr int kRows = 64;  // rows per CTA (4 warps x 16)

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// A fragment (16 x 16) of a row-major tile at (r0, k0), leading dimension ld.
__device__ __forceinline__ void frag_a(const bf16* t, int ld, int r0, int k0, uint32_t (&a)[4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = (lane & 3) * 2;
    a[0] = ld32(t + (r0 + g) * ld + k0 + q);
    a[1] = ld32(t + (r0 + g + 8) * ld + k0 + q);
    a[2] = ld32(t + (r0 + g) * ld + k0 + 8 + q);
    a[3] = ld32(t + (r0 + g + 8) * ld + k0 + 8 + q);
}
// A fragment of the transpose of a row-major tile: A[m][k] = t[k][m].
__device__ __forceinline__ void frag_at(const bf16* t, int ld, int m0, int k0, uint32_t (&a)[4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = (lane & 3) * 2;
    a[0] = pack2(t[(k0 + q) * ld + m0 + g], t[(k0 + q + 1) * ld + m0 + g]);
    a[1] = pack2(t[(k0 + q) * ld + m0 + g + 8], t[(k0 + q + 1) * ld + m0 + g + 8]);
    a[2] = pack2(t[(k0 + q + 8) * ld + m0 + g], t[(k0 + q + 9) * ld + m0 + g]);
    a[3] = pack2(t[(k0 + q + 8) * ld + m0 + g + 8], t[(k0 + q + 9) * ld + m0 + g + 8]);
}
// B fragment (16 x 8) from an n-major tile (t[n][k], leading dimension ldk).
__device__ __forceinline__ void frag_b(const bf16* t, int ldk, int n0, int k0, uint32_t& b0, uint32_t& b1) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = (lane & 3) * 2;
    b0 = ld32(t + (n0 + g) * ldk + k0 + q);
    b1 = ld32(t + (n0 + g) * ldk + k0 + 8 + q);
}
// B fragment from a k-major tile (t[k][n], leading dimension ldn).
__device__ __forceinline__ void frag_bk(const bf16* t, int ldn, int n0, int k0, uint32_t& b0, uint32_t& b1) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = (lane & 3) * 2;
    b0 = pack2(t[(k0 + q) * ldn + n0 + g], t[(k0 + q + 1) * ldn + n0 + g]);
    b1 = pack2(t[(k0 + q + 8) * ldn + n0 + g], t[(k0 + q + 9) * ldn + n0 + g]);
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// --------------------------------------------------------------- forward
// One CTA = 64 rows (16 per warp).  Weight tiles are n-major BF16 (WT[n][k]).
struct FwdSmem {
    bf16 w1[kH * kInP];
    bf16 w2[kH * kH];
    bf16 w3[kOutP * kH];
    bf16 x[kRows * kInP];
    bf16 h1[kRows * kH];
    bf16 h2[kRows * kH];
};

template <bool kTrain>
__global__ void __launch_bounds__(128) k_mlp_fwd(MlpDev m, const bf16* __restrict__ X, DCount Nc, float* __restrict__ Y,
                                                 float* Z1, bf16* H1, float* Z2, bf16* H2) {
    extern __shared__ __align__(16) unsigned char smraw[];
    FwdSmem& sm = *reinterpret_cast<FwdSmem*>(smraw);
    const int N = dcount(Nc);
    if ((int)blockIdx.x * kRows >= N) return;  // uniform over the block
    for (int i = threadIdx.x; i < kH * kInP / 2; i += blockDim.x)
        reinterpret_cast<uint32_t*>(sm.w1)[i] = reinterpret_cast<const uint32_t*>(m.w1t)[i];
    for (int i = threadIdx.x; i < kH * kH / 2; i += blockDim.x)
        reinterpret_cast<uint32_t*>(sm.w2)[i] = reinterpret_cast<const uint32_t*>(m.w2t)[i];
    for (int i = threadIdx.x; i < kOutP * kH / 2; i += blockDim.x)
        reinterpret_cast<uint32_t*>(sm.w3)[i] = reinterpret_cast<const uint32_t*>(m.w3t)[i];
    const int row0 = blockIdx.x * kRows;
    for (int i = threadIdx.x; i < kRows * kInP / 2; i += blockDim.x) {
        int r = (2 * i) / kInP;
        uint32_t v = 0;
        if (row0 + r < N) v = reinterpret_cast<const uint32_t*>(X + (size_t)row0 * kInP)[i];
        reinterpret_cast<uint32_t*>(sm.x)[i] = v;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = (lane & 3) * 2;
    const int r0 = warp * 16;
    // layer 1: x (16 x 80) @ W1 -> 128
    for (int nt = 0; nt < kH / 8; ++nt) {
        float d[4];
        const float b0 = m.b1[nt * 8 + q], b1 = m.b1[nt * 8 + q + 1];
        d[0] = b0; d[1] = b1; d[2] = b0; d[3] = b1;
        for (int ks = 0; ks < kInP / 16; ++ks) {
            uint32_t a[4], w0, w1;
            frag_a(sm.x, kInP, r0, ks * 16, a);
            frag_b(sm.w1, kInP, nt * 8, ks * 16, w0, w1);
            mma16816(d, a, w0, w1);
        }
        const int c = nt * 8 + q;
        sm.h1[(r0 + g) * kH + c] = __float2bfloat16_rn(gelu(d[0]));
        sm.h1[(r0 + g) * kH + c + 1] = __float2bfloat16_rn(gelu(d[1]));
        sm.h1[(r0 + g + 8) * kH + c] = __float2bfloat16_rn(gelu(d[2]));
        sm.h1[(r0 + g + 8) * kH + c + 1] = __float2bfloat16_rn(gelu(d[3]));
        if (kTrain) {
            const size_t ra = (size_t)(row0 + r0 + g), rb = ra + 8;
            Z1[ra * kH + c] = d[0]; Z1[ra * kH + c + 1] = d[1];
            Z1[rb * kH + c] = d[2]; Z1[rb * kH + c + 1] = d[3];
        }
    }
    __syncwarp();
    // layer 2
    for (int nt = 0; nt < kH / 8; ++nt) {
        float d[4];
        const float b0 = m.b2[nt * 8 + q], b1 = m.b2[nt * 8 + q + 1];
        d[0] = b0; d[1] = b1; d[2] = b0; d[3] = b1;
        for (int ks = 0; ks < kH / 16; ++ks) {
            uint32_t a[4], w0, w1;
            frag_a(sm.h1, kH, r0, ks * 16, a);
            frag_b(sm.w2, kH, nt * 8, ks * 16, w0, w1);
            mma16816(d, a, w0, w1);
        }
        const int c = nt * 8 + q;
        sm.h2[(r0 + g) * kH + c] = __float2bfloat16_rn(gelu(d[0]));
        sm.h2[(r0 + g) * kH + c + 1] = __float2bfloat16_rn(gelu(d[1]));
        sm.h2[(r0 + g + 8) * kH + c] = __float2bfloat16_rn(gelu(d[2]));
        sm.h2[(r0 + g + 8) * kH + c + 1] = __float2bfloat16_rn(gelu(d[3]));
        if (kTrain) {
            const size_t ra = (size_t)(row0 + r0 + g), rb = ra + 8;
            Z2[ra * kH + c] = d[0]; Z2[ra * kH + c + 1] = d[1];
            Z2[rb * kH + c] = d[2]; Z2[rb * kH + c + 1] = d[3];
        }
    }
    __syncwarp();
    // layer 3: -> 8 (5 used)
    {
        float d[4];
        const float b0 = m.b3[q], b1 = m.b3[q + 1];
        d[0] = b0; d[1] = b1; d[2] = b0; d[3] = b1;
        for (int ks = 0; ks < kH / 16; ++ks) {
            uint32_t a[4], w0, w1;
            frag_a(sm.h2, kH, r0, ks * 16, a);
            frag_b(sm.w3, kH, 0, ks * 16, w0, w1);
            mma16816(d, a, w0, w1);
        }
        const int ra = row0 + r0 + g, rb = ra + 8;
        if (ra < N) { Y[(size_t)ra * kOutP + q] = d[0]; Y[(size_t)ra * kOutP + q + 1] = d[1]; }
        if (rb < N) { Y[(size_t)rb * kOutP + q] = d[2]; Y[(size_t)rb * kOutP + q + 1] = d[3]; }
    }
    if (kTrain) {
        __syncwarp();
        for (int i = lane; i < 16 * kH; i += 32) {
            const int r = r0 + i / kH, c = i % kH;
            H1[(size_t)(row0 + r) * kH + c] = sm.h1[r * kH + c];
            H2[(size_t)(row0 + r) * kH + c] = sm.h2[r * kH + c];
        }
    }
}

// --------------------------------------------------------------- loss
// dY = 2 (y - t) / (N * 5) on the 5 outputs (0 on the padding); loss sum.
__global__ void k_mlp_loss(const float* Y, const float* T, int N, int Npad, bf16* dY, double* loss) {
    __shared__ double red[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < Npad * kOutP) {
        const int r = i / kOutP, c = i % kOutP;
        float g = 0.f;
        if (r < N && c < kMlpOut) {
            const float e = Y[i] - T[(size_t)r * kMlpOut + c];
            l = (double)e * e / ((double)N * kMlpOut);
            g = 2.0f * e / ((float)N * kMlpOut);
        }
        dY[i] = __float2bfloat16_rn(g);
    }
    for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(loss, s);
    }
}

// --------------------------------------------------------------- backward
// One CTA = 64 rows.  dH2 = dY W3^T, dZ2 = dH2 * gelu'(Z2), dH1 = dZ2 W2^T,
// dZ1 = dH1 * gelu'(Z1); weight gradients (X^T dZ1, H1^T dZ2, H2^T dY) and
// bias gradients are accumulated with atomics into FP32 buffers.
struct BwdSmem {
    bf16 w2r[kH * kH];     // W2 as [in][out]: n-major for dH1 = dZ2 W2^T (n = in, k = out)
    bf16 w3r[kH * 16];     // W3 as [in][out padded to 16]
    bf16 x[kRows * kInP];
    bf16 h1[kRows * kH];
    bf16 h2[kRows * kH];
    bf16 dy[kRows * 16];
    bf16 dz2[kRows * kH];
    bf16 dz1[kRows * kH];
};

__global__ void __launch_bounds__(128) k_mlp_bwd(MlpDev m, const bf16* __restrict__ X, const float* __restrict__ Z1,
                                                 const bf16* __restrict__ H1, const float* __restrict__ Z2,
                                                 const bf16* __restrict__ H2, const bf16* __restrict__ dY, int N,
                                                 float* grad) {
    extern __shared__ __align__(16) unsigned char smraw[];
    BwdSmem& sm = *reinterpret_cast<BwdSmem*>(smraw);
    const int row0 = blockIdx.x * kRows;
    const bf16* w2r = reinterpret_cast<const bf16*>(m.w2r);
    const bf16* w3r = reinterpret_cast<const bf16*>(m.w3r);
    for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) sm.w2r[i] = w2r[i];
    for (int i = threadIdx.x; i < kH * 16; i += blockDim.x) {
        const int r = i / 16, c = i % 16;
        sm.w3r[i] = c < kOutP ? w3r[r * kOutP + c] : __float2bfloat16_rn(0.f);
    }
    for (int i = threadIdx.x; i < kRows * kInP; i += blockDim.x) {
        const int r = i / kInP;
        sm.x[i] = row0 + r < N ? X[(size_t)row0 * kInP + i] : __float2bfloat16_rn(0.f);
    }
    for (int i = threadIdx.x; i < kRows * kH; i += blockDim.x) {
        sm.h1[i] = H1[(size_t)row0 * kH + i];
        sm.h2[i] = H2[(size_t)row0 * kH + i];
    }
    for (int i = threadIdx.x; i < kRows * 16; i += blockDim.x) {
        const int r = i / 16, c = i % 16;
        sm.dy[i] = c < kOutP ? dY[(size_t)(row0 + r) * kOutP + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = (lane & 3) * 2;
    const int r0 = warp * 16;
    float* gW1 = grad + kOffW1;
    float* gb1 = grad + kOffB1;
    float* gW2 = grad + kOffW2;
    float* gb2 = grad + kOffB2;
    float* gW3 = grad + kOffW3;
    float* gb3 = grad + kOffB3;
    // dH2 = dY (16 x 16) @ W3^T: B[k = out][n = in] = W3[in][out] -> n-major w3r[in][out]
    for (int nt = 0; nt < kH / 8; ++nt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        uint32_t a[4], w0, w1;
        frag_a(sm.dy, 16, r0, 0, a);
        frag_b(sm.w3r, 16, nt * 8, 0, w0, w1);
        mma16816(d, a, w0, w1);
        const int c = nt * 8 + q;
        const size_t ra = (size_t)(row0 + r0 + g), rb = ra + 8;
        sm.dz2[(r0 + g) * kH + c] = __float2bfloat16_rn(d[0] * gelu_d(Z2[ra * kH + c]));
        sm.dz2[(r0 + g) * kH + c + 1] = __float2bfloat16_rn(d[1] * gelu_d(Z2[ra * kH + c + 1]));
        sm.dz2[(r0 + g + 8) * kH + c] = __float2bfloat16_rn(d[2] * gelu_d(Z2[rb * kH + c]));
        sm.dz2[(r0 + g + 8) * kH + c + 1] = __float2bfloat16_rn(d[3] * gelu_d(Z2[rb * kH + c + 1]));
    }
    __syncwarp();
    // dH1 = dZ2 (16 x 128) @ W2^T: B[k = out][n = in] = W2[in][out] -> n-major w2r[in][out]
    for (int nt = 0; nt < kH / 8; ++nt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        for (int ks = 0; ks < kH / 16; ++ks) {
            uint32_t a[4], w0, w1;
            frag_a(sm.dz2, kH, r0, ks * 16, a);
            frag_b(sm.w2r, kH, nt * 8, ks * 16, w0, w1);
            mma16816(d, a, w0, w1);
        }
        const int c = nt * 8 + q;
        const size_t ra = (size_t)(row0 + r0 + g), rb = ra + 8;
        sm.dz1[(r0 + g) * kH + c] = __float2bfloat16_rn(d[0] * gelu_d(Z1[ra * kH + c]));
        sm.dz1[(r0 + g) * kH + c + 1] = __float2bfloat16_rn(d[1] * gelu_d(Z1[ra * kH + c + 1]));
        sm.dz1[(r0 + g + 8) * kH + c] = __float2bfloat16_rn(d[2] * gelu_d(Z1[rb * kH + c]));
        sm.dz1[(r0 + g + 8) * kH + c + 1] = __float2bfloat16_rn(d[3] * gelu_d(Z1[rb * kH + c + 1]));
    }
    __syncthreads();
    // weight gradients over the CTA's 64 rows: dW[i][j] = sum_r A[r][i] D[r][j]
    // (M = i, N = j, K = rows); warps split the M tiles.
    auto wgrad = [&](const bf16* At, int lda, int Mdim, const bf16* Dt, int ldd, int Ndim, float* gW, int ldw) {
        for (int mt = warp; mt < Mdim / 16; mt += 4) {
            for (int nt = 0; nt < Ndim / 8; ++nt) {
                float d[4] = {0.f, 0.f, 0.f, 0.f};
                for (int ks = 0; ks < kRows / 16; ++ks) {
                    uint32_t a[4], w0, w1;
                    frag_at(At, lda, mt * 16, ks * 16, a);
                    frag_bk(Dt, ldd, nt * 8, ks * 16, w0, w1);
                    mma16816(d, a, w0, w1);
                }
                const int i0 = mt * 16 + g, j0 = nt * 8 + q;
                atomicAdd(&gW[i0 * ldw + j0], d[0]);
                atomicAdd(&gW[i0 * ldw + j0 + 1], d[1]);
                atomicAdd(&gW[(i0 + 8) * ldw + j0], d[2]);
                atomicAdd(&gW[(i0 + 8) * ldw + j0 + 1], d[3]);
            }
        }
    };
    wgrad(sm.x, kInP, kInP, sm.dz1, kH, kH, gW1, kH);
    wgrad(sm.h1, kH, kH, sm.dz2, kH, kH, gW2, kH);
    wgrad(sm.h2, kH, kH, sm.dy, 16, kOutP, gW3, kOutP);
    // bias gradients: column sums
    for (int j = threadIdx.x; j < kH; j += blockDim.x) {
        float s1 = 0.f, s2 = 0.f;
        for (int r = 0; r < kRows; ++r) {
            s1 += __bfloat162float(sm.dz1[r * kH + j]);
            s2 += __bfloat162float(sm.dz2[r * kH + j]);
        }
        atomicAdd(&gb1[j], s1);
        atomicAdd(&gb2[j], s2);
    }
    if (threadIdx.x < kOutP) {
        float s = 0.f;
        for (int r = 0; r < kRows; ++r) s += __bfloat162float(sm.dy[r * 16 + threadIdx.x]);
        atomicAdd(&gb3[threadIdx.x], s);
    }
}

// --------------------------------------------------------------- weights
// BF16 copies of the FP32 master weights: n-major (forward) and [in][out] (backward).
__global__ void k_mlp_cast(MlpDev m, const float* w) {
    bf16* w1t = reinterpret_cast<bf16*>(m.w1t);
    bf16* w2t = reinterpret_cast<bf16*>(m.w2t);
    bf16* w3t = reinterpret_cast<bf16*>(m.w3t);
    bf16* w2r = reinterpret_cast<bf16*>(m.w2r);
    bf16* w3r = reinterpret_cast<bf16*>(m.w3r);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kMlpParams; i += gridDim.x * blockDim.x) {
        const float x = w[i];
        if (i < kOffB1) {
            const int k = i / kH, n = i % kH;
            w1t[n * kInP + k] = __float2bfloat16_rn(x);
        } else if (i >= kOffW2 && i < kOffB2) {
            const int j = i - kOffW2, k = j / kH, n = j % kH;
            w2t[n * kH + k] = __float2bfloat16_rn(x);
            w2r[j] = __float2bfloat16_rn(x);
        } else if (i >= kOffW3 && i < kOffB3) {
            const int j = i - kOffW3, k = j / kOutP, n = j % kOutP;
            w3t[n * kH + k] = __float2bfloat16_rn(x);
            w3r[j] = __float2bfloat16_rn(x);
        }
    }
}

// Adam on the FP32 master weights (gradients are batch means already).
__global__ void k_adam(float* w, float* g, float* m1, float* m2, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.f - b1) * gi;
        const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = b;
        w[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
        g[i] = 0.f;
    }
}

// Gathers training rows idx = mix(seed, step, r) mod count.
__device__ __forceinline__ unsigned long long mixs(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
__global__ void k_mlp_gather(const float* Xf, const float* Tf, size_t count, int B, unsigned long long seed,
                             unsigned long long step, bf16* X, float* T) {
    const int r = blockIdx.x;
    const unsigned long long idx = mixs(seed + 0x9e3779b97f4a7c15ull * (step * (unsigned long long)B + r + 1)) % count;
    for (int c = threadIdx.x; c < kInP; c += blockDim.x)
        X[(size_t)r * kInP + c] = __float2bfloat16_rn(c < kIn ? Xf[idx * kIn + c] : 0.f);
    if (threadIdx.x < kMlpOut) T[(size_t)r * kMlpOut + threadIdx.x] = Tf[idx * kMlpOut + threadIdx.x];
}

// FP32 rows [N][69] -> BF16 rows [N][80].
__global__ void k_mlp_pack(const float* Xf, int N, bf16* X) {
    const int r = blockIdx.x;
    if (r >= N) return;
    for (int c = threadIdx.x; c < kInP; c += blockDim.x)
        X[(size_t)r * kInP + c] = __float2bfloat16_rn(c < kIn ? Xf[(size_t)r * kIn + c] : 0.f);
}

// --------------------------------------------------------------- features
// Summary of one stored vector (tree g, slot s): sum_p w_p v_p / sum_p w_p with
// v_p the site's 4C values divided by their sum; 16 outputs ([cat][state], zero-padded).
template <typename R, int C>
__global__ void k_slot_summary(Aln A, ClvGroup g, DCount ntrees, int nslot, float* out) {
    const int tree = blockIdx.x / nslot, slot = blockIdx.x % nslot;
    if (tree >= dcount(ntrees)) return;  // uniform over the block
    const R* base = reinterpret_cast<const R*>(g.clv) + (size_t)tree * g.tree_stride + (size_t)slot * A.P * 4 * C;
    float acc[16] = {0};
    float wsum = 0.f;
    for (int p = threadIdx.x; p < A.P; p += blockDim.x) {
        float v[4 * C], s = 0.f;
#pragma unroll
        for (int q = 0; q < 4 * C; ++q) { v[q] = (float)base[(size_t)p * 4 * C + q]; s += v[q]; }
        const float w = (float)A.w[p], f = s > 0.f ? w / s : 0.f;
#pragma unroll
        for (int q = 0; q < 4 * C; ++q) acc[q] += v[q] * f;
        wsum += w;
    }
    __shared__ float red[16][33];
    __shared__ float wred[33];
    for (int q = 0; q < 16; ++q) {
        float x = acc[q];
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = x;
    }
    float ws = wsum;
    for (int o = 16; o; o >>= 1) ws += __shfl_xor_sync(0xffffffffu, ws, o);
    if ((threadIdx.x & 31) == 0) wred[threadIdx.x >> 5] = ws;
    __syncthreads();
    if (threadIdx.x < 16) {
        float s = 0.f, w = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { s += red[threadIdx.x][i]; w += wred[i]; }
        out[(size_t)blockIdx.x * 16 + threadIdx.x] = w > 0.f ? s / w : 0.f;
    }
}

// Summary of every leaf (weighted state frequencies, gaps spread evenly).
__global__ void k_tip_summary(Aln A, int C, float* out) {
    const int leaf = blockIdx.x;
    float acc[4] = {0, 0, 0, 0}, wsum = 0.f;
    for (int p = threadIdx.x; p < A.P; p += blockDim.x) {
        const int code = A.tips[(size_t)leaf * A.P + p];
        const float w = (float)A.w[p];
        for (int i = 0; i < 4; ++i) acc[i] += w * (code >= 4 ? 0.25f : (code == i ? 1.f : 0.f));
        wsum += w;
    }
    __shared__ float red[5][33];
    for (int i = 0; i < 5; ++i) {
        float x = i < 4 ? acc[i] : wsum;
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) red[i][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        const int r = threadIdx.x >> 2, i = threadIdx.x & 3;
        float s = 0.f, w = 0.f;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) { s += red[i][j]; w += red[4][j]; }
        out[(size_t)leaf * 16 + threadIdx.x] = (r < C && w > 0.f) ? s / w / C : 0.f;
    }
}

// Feature rows of work items [i0, i1): FP32 [W][69] (for logging) and BF16 [W][80].
__global__ void k_item_features(int n, const Item* items, int i0, DCount i1, TreeSet fr, int first,
                                const float* slot_sum, int nslot, const float* tip_sum, float* Xf, bf16* Xb) {
    const int k = i0 + blockIdx.x;
    if (k >= dcount(i1)) return;
    const Item it = items[k];
    const int NN = 2 * n - 2;
    const int32_t* up = fr.up + (size_t)it.tree * NN;
    const int32_t* ch = fr.ch + (size_t)it.tree * NN * 2;
    const double* len = fr.len + (size_t)it.tree * NN;
    const int v = it.v, u = up[v];
    const int sib = ch[2 * u] == v ? ch[2 * u + 1] : ch[2 * u];
    const int c0 = ch[2 * v], c1 = ch[2 * v + 1];
    const int x2 = it.swap == 0 ? c0 : c1, y2 = it.swap == 0 ? c1 : c0;
    const int node[4] = {u, x2, sib, y2};
    const int lnode[5] = {v, u, x2, sib, y2};  // length of each member's branch
    const int gi = it.tree - first;
    float* xf = Xf + (size_t)(k - i0) * kIn;
    bf16* xb = Xb + (size_t)(k - i0) * kInP;
    for (int c = threadIdx.x; c < kInP; c += blockDim.x) {
        float val = 0.f;
        if (c < 5) {
            val = logf((float)len[lnode[c]]);
        } else if (c < kIn) {
            const int m = (c - 5) / 16, o = (c - 5) % 16, x = node[m];
            if (m == 0) {
                val = u == n ? tip_sum[o] : slot_sum[((size_t)gi * nslot + (n - 2 + (u - n - 1))) * 16 + o];
            } else if (x < n) {
                val = tip_sum[(size_t)x * 16 + o];
            } else {
                val = slot_sum[((size_t)gi * nslot + (x - n)) * 16 + o];
            }
        }
        if (c < kIn) xf[c] = val;
        xb[c] = __float2bfloat16_rn(val);
    }
}

// Whether item k of an alignment starts from the network under judge state st:
// the chosen start, except for the judge's sample, which takes the other one.
__device__ __forceinline__ bool judge_learned(int st, int k) {
    const bool sample = k % (st == kJudgeOpen ? kJudgeEveryOpen : kJudgeEvery) == 0;
    return (st != kJudgePlain) != sample;
}

// Warm starts [W][5] (branch order central, A, B, C, D) from predicted
// log-ratios in member order; NaN marks "no prediction" (the inherited length is
// kept), as for every item the judge assigns the inherited start.
__global__ void k_item_init(const Item* items, int i0, DCount i1, const float* Xf, const float* Y, double tmin,
                            double tmax, double* init, const Judge* judge) {
    const int k = i0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= dcount(i1)) return;
    const Item it = items[k];
    const int brn[5] = {0, 1, it.swap == 0 ? 3 : 4, 2, it.swap == 0 ? 4 : 3};
    const float* y = Y + (size_t)(k - i0) * kOutP;
    const float* x = Xf + (size_t)(k - i0) * kIn;
    double* o = init + (size_t)(k - i0) * 5;
    const bool plain = judge && !judge_learned(judge->state, k);
    for (int j = 0; j < 5; ++j) {
        const double t = exp((double)x[j] + (double)y[j]);
        o[brn[j]] = (!plain && isfinite(t) && t >= tmin && t <= tmax) ? t : __longlong_as_double(0x7ff8000000000000ll);
    }
}

// One block: adds a round's proposals of one alignment to its judge (group 0
// started from the network, group 1 from the inherited lengths) and, when the
// evidence suffices, chooses the start for the next rounds and halves its
// counts, so that the choice follows the recent rounds.
__global__ void k_judge(DCount count, const int32_t* evals, Judge* judge) {
    __shared__ unsigned long long red[6][32];
    const int st = judge->state;  // the state this round's starts were assigned under
    unsigned long long v[6] = {0, 0, 0, 0, 0, 0};  // evals, items, squares per group
    const int cnt = dcount(count);
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        const int g = judge_learned(st, k) ? 0 : 1;
        const unsigned long long e = (unsigned long long)evals[k];
        v[g] += e;
        v[2 + g] += 1;
        v[4 + g] += e * e;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = 0; q < 6; ++q) {
        for (int o = 16; o; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        if (lane == 0) red[q][w] = v[q];
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int q = 0; q < 6; ++q) {
        unsigned long long t = 0;
        for (int i = 0; i < nw; ++i) t += red[q][i];
        v[q] = t;
    }
    Judge& J = *judge;
    for (int g = 0; g < 2; ++g) {
        J.evals[g] += v[g];
        J.items[g] += v[2 + g];
        J.sq[g] += v[4 + g];
    }
    const double n0 = (double)J.items[0], n1 = (double)J.items[1];
    if (J.items[0] < kJudgeMinT || J.items[1] < kJudgeMinT) return;
    const double m0 = J.evals[0] / n0, m1 = J.evals[1] / n1;
    const double s0 = fmax((J.sq[0] - n0 * m0 * m0) / (n0 - 1.0), 0.0), s1 = fmax((J.sq[1] - n1 * m1 * m1) / (n1 - 1.0), 0.0);
    const double k = 1.0 - kJudgeMargin;
    // d > 0: the network saves more than the margin
    const double d = k * m1 - m0, se = sqrt(s0 / n0 + k * k * s1 / n1);
    int next = -1;
    if (se > 0.0 && d >= kJudgeT * se) next = kJudgeLearned;
    else if (se > 0.0 && -d >= kJudgeT * se) next = kJudgePlain;
    else if (J.items[0] >= kJudgeMin && J.items[1] >= kJudgeMin) next = d >= 0.0 ? kJudgeLearned : kJudgePlain;
    if (next < 0) return;
    J.state = next;
    for (int g = 0; g < 2; ++g) {
        J.evals[g] >>= 1;
        J.items[g] >>= 1;
        J.sq[g] >>= 1;
    }
}

// Logs (features, log optimised lengths in member order) of items [i0, i1).
__global__ void k_log_pairs(const Item* items, int i0, int i1, const float* Xf, const double* len5, float* LX, float* LT,
                            unsigned long long* count, size_t cap) {
    const int k = i0 + blockIdx.x;
    if (k >= i1) return;
    __shared__ unsigned long long slot;
    if (threadIdx.x == 0) slot = atomicAdd(count, 1ull);
    __syncthreads();
    if (slot >= cap) return;
    const Item it = items[k];
    const int brn[5] = {0, 1, it.swap == 0 ? 3 : 4, 2, it.swap == 0 ? 4 : 3};
    for (int c = threadIdx.x; c < kIn; c += blockDim.x) LX[slot * kIn + c] = Xf[(size_t)(k - i0) * kIn + c];
    if (threadIdx.x < 5) {  // log-ratio target, clipped to +-4 (a factor of ~55) against heavy tails at the bounds
        const double r = log(len5[(size_t)k * 5 + brn[threadIdx.x]]) - (double)Xf[(size_t)(k - i0) * kIn + threadIdx.x];
        LT[slot * kMlpOut + threadIdx.x] = (float)fmin(4.0, fmax(-4.0, r));
    }
}

inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

extern std::atomic<long long> g_launches;

size_t mlp_fwd_smem() { return sizeof(FwdSmem); }
size_t mlp_bwd_smem() { return sizeof(BwdSmem); }

void mlp_cast(cudaStream_t s, MlpDev m, const float* w) {
    k_mlp_cast<<<nblk(kMlpParams, 256), 256, 0, s>>>(m, w);
    ++g_launches;
}

void mlp_forward(cudaStream_t s, MlpDev m, const void* Xb, int N, float* Y, float* Z1, void* H1, float* Z2, void* H2,
                 bool train) {
    if (N <= 0) return;
    const int grid = nblk(N, kRows);
    if (train) {
        cudaFuncSetAttribute(k_mlp_fwd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FwdSmem));
        k_mlp_fwd<true><<<grid, 128, sizeof(FwdSmem), s>>>(m, reinterpret_cast<const bf16*>(Xb), hcount(N), Y, Z1,
                                                             reinterpret_cast<bf16*>(H1), Z2, reinterpret_cast<bf16*>(H2));
    } else {
        cudaFuncSetAttribute(k_mlp_fwd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FwdSmem));
        k_mlp_fwd<false><<<grid, 128, sizeof(FwdSmem), s>>>(m, reinterpret_cast<const bf16*>(Xb), hcount(N), Y, nullptr,
                                                              nullptr, nullptr, nullptr);
    }
    ++g_launches;
}

void mlp_forward(cudaStream_t s, MlpDev m, const void* Xb, DCount N, float* Y) {
    if (N.cap <= 0) return;
    cudaFuncSetAttribute(k_mlp_fwd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FwdSmem));
    k_mlp_fwd<false><<<nblk(N.cap, kRows), 128, sizeof(FwdSmem), s>>>(m, reinterpret_cast<const bf16*>(Xb), N, Y,
                                                                     nullptr, nullptr, nullptr, nullptr);
    ++g_launches;
}

void mlp_loss(cudaStream_t s, const float* Y, const float* T, int N, void* dY, double* loss) {
    const int Npad = nblk(N, kRows) * kRows;
    k_mlp_loss<<<nblk((long long)Npad * kOutP, 256), 256, 0, s>>>(Y, T, N, Npad, reinterpret_cast<bf16*>(dY), loss);
    ++g_launches;
}

void mlp_backward(cudaStream_t s, MlpDev m, const void* Xb, const float* Z1, const void* H1, const float* Z2,
                  const void* H2, const void* dY, int N, float* grad) {
    cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BwdSmem));
    k_mlp_bwd<<<nblk(N, kRows), 128, sizeof(BwdSmem), s>>>(
        m, reinterpret_cast<const bf16*>(Xb), Z1, reinterpret_cast<const bf16*>(H1), Z2,
        reinterpret_cast<const bf16*>(H2), reinterpret_cast<const bf16*>(dY), N, grad);
    ++g_launches;
}

void mlp_adam(cudaStream_t s, float* w, float* g, float* m1, float* m2, float lr, int t) {
    const float b1 = 0.9f, b2 = 0.999f;
    k_adam<<<nblk(kMlpParams, 256), 256, 0, s>>>(w, g, m1, m2, kMlpParams, lr, b1, b2, 1e-8f,
                                                  1.f - powf(b1, (float)t), 1.f - powf(b2, (float)t));
    ++g_launches;
}

void mlp_gather(cudaStream_t s, const float* LX, const float* LT, size_t count, int B, unsigned long long seed,
                unsigned long long step, void* Xb, float* T) {
    k_mlp_gather<<<B, 96, 0, s>>>(LX, LT, count, B, seed, step, reinterpret_cast<bf16*>(Xb), T);
    ++g_launches;
}

void mlp_pack(cudaStream_t s, const float* Xf, int N, void* Xb) {
    if (N <= 0) return;
    k_mlp_pack<<<N, 96, 0, s>>>(Xf, N, reinterpret_cast<bf16*>(Xb));
    ++g_launches;
}

void launch_slot_summary(cudaStream_t s, int prec, int C, Aln A, ClvGroup g, DCount ntrees, int nslot, float* out) {
    if (ntrees.cap <= 0 || nslot <= 0) return;
    const int grid = ntrees.cap * nslot;
    if (prec == 0) {
        if (C == 1) k_slot_summary<double, 1><<<grid, 256, 0, s>>>(A, g, ntrees, nslot, out);
        else k_slot_summary<double, 4><<<grid, 256, 0, s>>>(A, g, ntrees, nslot, out);
    } else {
        if (C == 1) k_slot_summary<float, 1><<<grid, 256, 0, s>>>(A, g, ntrees, nslot, out);
        else k_slot_summary<float, 4><<<grid, 256, 0, s>>>(A, g, ntrees, nslot, out);
    }
    ++g_launches;
}

void launch_tip_summary(cudaStream_t s, Aln A, int C, float* out) {
    k_tip_summary<<<A.n, 256, 0, s>>>(A, C, out);
    ++g_launches;
}

void launch_item_features(cudaStream_t s, int n, const Item* items, int i0, DCount i1, TreeSet fr, int first,
                          const float* slot_sum, int nslot, const float* tip_sum, float* Xf, void* Xb) {
    if (i1.cap <= i0) return;
    k_item_features<<<i1.cap - i0, 96, 0, s>>>(n, items, i0, i1, fr, first, slot_sum, nslot, tip_sum, Xf,
                                                reinterpret_cast<bf16*>(Xb));
    ++g_launches;
}

void launch_item_init(cudaStream_t s, const Item* items, int i0, DCount i1, const float* Xf, const float* Y, double tmin,
                      double tmax, double* init, const Judge* judge) {
    if (i1.cap <= i0) return;
    k_item_init<<<nblk(i1.cap - i0, 128), 128, 0, s>>>(items, i0, i1, Xf, Y, tmin, tmax, init, judge);
    ++g_launches;
}

void launch_judge(cudaStream_t s, DCount count, const int32_t* evals, Judge* judge) {
    if (count.cap <= 0 || !judge) return;
    k_judge<<<1, 256, 0, s>>>(count, evals, judge);
    ++g_launches;
}

void launch_log_pairs(cudaStream_t s, const Item* items, int i0, int i1, const float* Xf, const double* len5, float* LX,
                      float* LT, unsigned long long* count, size_t cap) {
    if (i1 <= i0) return;
    k_log_pairs<<<i1 - i0, 96, 0, s>>>(items, i0, i1, Xf, len5, LX, LT, count, cap);
    ++g_launches;
}

}  // namespace pt
