// Learned adaptation proposer (not in the paper): an MLP 8 -> 64 -> 64 -> 4
// (ReLU, ReLU, logits) that predicts from local macroscopic features which
// physical cells can decide a split/merge of the global velocity mesh, so
// that the criterion of Sec. 3.4 runs only on that check set.
//
// Tensor cores: every layer of the forward and backward pass is a BF16
// mma.sync m16n8k16 with FP32 accumulation.  A warp owns a tile of 16 cells;
// a layer's C fragments are repacked in registers as the next layer's A
// fragments.  Weight gradients contract over the cells of the tile with
// transposed BF16 copies staged in shared memory, are summed per block in
// shared memory and across blocks in a fixed order, then applied by SGD to
// the FP32 master weights.
//
// Parameter layout (FP32, AVS_MLP_NPARAM floats): W1[64][8], b1[64],
// W2[64][64], b2[64], W3[4][64], b3[4] (weights [out][in]).
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "avs_dev.cuh"
#include "avs_internal.h"
#include "avs_mlp.h"

#define CK_RET(x)                               \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return e_;       \
    } while (0)

namespace avs {

namespace {

constexpr int H = 64, NF = 8, NO = 4;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * NF, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + NO * H;
static_assert(OFF_B3 + NO == AVS_MLP_NPARAM, "parameter layout");

// BF16 operand copies: W1b[64][16] (K padded), W2b[64][64], W3b[8][64] (rows
// padded), W2t[64][64] = W2^T, W3t[64][8] = W3^T (columns padded).
constexpr int BOFF_W1 = 0, BOFF_W2 = BOFF_W1 + H * 16, BOFF_W3 = BOFF_W2 + H * H, BOFF_W2T = BOFF_W3 + 8 * H,
              BOFF_W3T = BOFF_W2T + H * H, BSIZE = BOFF_W3T + H * 8;

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, const uint32_t* b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// Forward pass of one 16-cell tile.  X rows beyond `rows` are zero.
// Returns H1, H2 (post-ReLU, FP32 C layout: [n-tile][4]) and the logits C3.
struct Fwd {
    float h1[8][4], h2[8][4], z3[4];
};

__device__ __forceinline__ void forward_tile(const __nv_bfloat16* __restrict__ Wb, const float* __restrict__ P,
                                             const uint32_t* ax, Fwd& o)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    // layer 1: [16 x 16] x [16 x 64]
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float c[4] = {0, 0, 0, 0};
        uint32_t b[2] = {ld32(Wb + BOFF_W1 + (8 * j + g) * 16 + 2 * t), 0u};
        mma16816(c, ax, b);
        const float b0 = P[OFF_B1 + 8 * j + 2 * t], b1 = P[OFF_B1 + 8 * j + 2 * t + 1];
        o.h1[j][0] = fmaxf(c[0] + b0, 0.f);
        o.h1[j][1] = fmaxf(c[1] + b1, 0.f);
        o.h1[j][2] = fmaxf(c[2] + b0, 0.f);
        o.h1[j][3] = fmaxf(c[3] + b1, 0.f);
    }
    // layer 2: [16 x 64] x [64 x 64]
    uint32_t a2[4][4];
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
        a2[kb][0] = pack2(o.h1[2 * kb][0], o.h1[2 * kb][1]);
        a2[kb][1] = pack2(o.h1[2 * kb][2], o.h1[2 * kb][3]);
        a2[kb][2] = pack2(o.h1[2 * kb + 1][0], o.h1[2 * kb + 1][1]);
        a2[kb][3] = pack2(o.h1[2 * kb + 1][2], o.h1[2 * kb + 1][3]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float c[4] = {0, 0, 0, 0};
#pragma unroll
        for (int kb = 0; kb < 4; ++kb) {
            uint32_t b[2] = {ld32(Wb + BOFF_W2 + (8 * j + g) * H + 16 * kb + 2 * t),
                             ld32(Wb + BOFF_W2 + (8 * j + g) * H + 16 * kb + 2 * t + 8)};
            mma16816(c, a2[kb], b);
        }
        const float b0 = P[OFF_B2 + 8 * j + 2 * t], b1 = P[OFF_B2 + 8 * j + 2 * t + 1];
        o.h2[j][0] = fmaxf(c[0] + b0, 0.f);
        o.h2[j][1] = fmaxf(c[1] + b1, 0.f);
        o.h2[j][2] = fmaxf(c[2] + b0, 0.f);
        o.h2[j][3] = fmaxf(c[3] + b1, 0.f);
    }
    // layer 3: [16 x 64] x [64 x 8]
    float c[4] = {0, 0, 0, 0};
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
        uint32_t a[4] = {pack2(o.h2[2 * kb][0], o.h2[2 * kb][1]), pack2(o.h2[2 * kb][2], o.h2[2 * kb][3]),
                         pack2(o.h2[2 * kb + 1][0], o.h2[2 * kb + 1][1]),
                         pack2(o.h2[2 * kb + 1][2], o.h2[2 * kb + 1][3])};
        uint32_t b[2] = {ld32(Wb + BOFF_W3 + g * H + 16 * kb + 2 * t), ld32(Wb + BOFF_W3 + g * H + 16 * kb + 2 * t + 8)};
        mma16816(c, a, b);
    }
    const int o0 = 2 * t, o1 = 2 * t + 1;
    const float b0 = o0 < NO ? P[OFF_B3 + o0] : 0.f, b1 = o1 < NO ? P[OFF_B3 + o1] : 0.f;
    o.z3[0] = c[0] + b0;
    o.z3[1] = c[1] + b1;
    o.z3[2] = c[2] + b0;
    o.z3[3] = c[3] + b1;
}

__device__ __forceinline__ void load_x(const float* __restrict__ X, int r0, int n, uint32_t* ax)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int ra = r0 + g, rb = r0 + g + 8;
    const float x0 = ra < n ? X[(size_t)ra * NF + 2 * t] : 0.f, x1 = ra < n ? X[(size_t)ra * NF + 2 * t + 1] : 0.f;
    const float y0 = rb < n ? X[(size_t)rb * NF + 2 * t] : 0.f, y1 = rb < n ? X[(size_t)rb * NF + 2 * t + 1] : 0.f;
    ax[0] = pack2(x0, x1);
    ax[1] = pack2(y0, y1);
    ax[2] = 0u;
    ax[3] = 0u;
}

}  // namespace

// ------------------------------------------------------------------ kernels
__global__ void k_mlp_prep(const float* __restrict__ P, __nv_bfloat16* Wb)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < BSIZE; e += gridDim.x * blockDim.x) {
        float v = 0.f;
        if (e < BOFF_W2) {                          // W1b[o][k], k < 16
            const int o = e / 16, k = e % 16;
            v = k < NF ? P[OFF_W1 + o * NF + k] : 0.f;
        } else if (e < BOFF_W3) {                   // W2b[o][i]
            v = P[OFF_W2 + (e - BOFF_W2)];
        } else if (e < BOFF_W2T) {                  // W3b[o][i], o < 8
            const int o = (e - BOFF_W3) / H, i = (e - BOFF_W3) % H;
            v = o < NO ? P[OFF_W3 + o * H + i] : 0.f;
        } else if (e < BOFF_W3T) {                  // W2t[i][o] = W2[o][i]
            const int i = (e - BOFF_W2T) / H, o = (e - BOFF_W2T) % H;
            v = P[OFF_W2 + o * H + i];
        } else {                                    // W3t[i][o] = W3[o][i], o < 8
            const int i = (e - BOFF_W3T) / 8, o = (e - BOFF_W3T) % 8;
            v = o < NO ? P[OFF_W3 + o * H + i] : 0.f;
        }
        Wb[e] = __float2bfloat16_rn(v);
    }
}

// logits [n][4]
__global__ void __launch_bounds__(128) k_mlp_fwd(int n, const float* __restrict__ X, const float* __restrict__ P,
                                                 const __nv_bfloat16* __restrict__ Wb, float* logits)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile * 16 < n; tile += warps) {
        const int r0 = tile * 16;
        uint32_t ax[4];
        load_x(X, r0, n, ax);
        Fwd o;
        forward_tile(Wb, P, ax, o);
        if (t < 2) {
            if (r0 + g < n) {
                logits[(size_t)(r0 + g) * NO + 2 * t] = o.z3[0];
                logits[(size_t)(r0 + g) * NO + 2 * t + 1] = o.z3[1];
            }
            if (r0 + g + 8 < n) {
                logits[(size_t)(r0 + g + 8) * NO + 2 * t] = o.z3[2];
                logits[(size_t)(r0 + g + 8) * NO + 2 * t + 1] = o.z3[3];
            }
        }
    }
}

// Forward + backward of the mean BCE-with-logits loss over n cells x 4
// outputs.  Each block accumulates the gradient of its tiles in shared memory
// and writes it to part[blockIdx.x][AVS_MLP_NPARAM + 1] (last entry: loss sum).
__global__ void __launch_bounds__(128) k_mlp_fwdbwd(int n, const float* __restrict__ X, const float* __restrict__ Y,
                                                    const float* __restrict__ P, const __nv_bfloat16* __restrict__ Wb,
                                                    float* part)
{
    __shared__ float gsum[AVS_MLP_NPARAM + 1];
    // per-warp transposed BF16 staging, columns = the 16 cells of the tile
    __shared__ __align__(16) __nv_bfloat16 XT[4][16][16], H1T[4][H][16], H2T[4][H][16], D1T[4][H][16],
        D2T[4][H][16], D3T[4][16][16];
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
    for (int e = threadIdx.x; e <= AVS_MLP_NPARAM; e += blockDim.x) gsum[e] = 0.f;
    for (int e = lane; e < 16 * 16; e += 32) {
        XT[w][e / 16][e % 16] = __float2bfloat16_rn(0.f);
        D3T[w][e / 16][e % 16] = __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    const float inv = 1.0f / (4.0f * (float)n);
    const int warps = (gridDim.x * blockDim.x) >> 5;
    float loss = 0.f;
    for (int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile * 16 < n; tile += warps) {
        const int r0 = tile * 16;
        const bool va = r0 + g < n, vb = r0 + g + 8 < n;
        uint32_t ax[4];
        load_x(X, r0, n, ax);
        Fwd o;
        forward_tile(Wb, P, ax, o);
        // dZ3 = (sigmoid(z) - y) / (4 n) on valid rows and outputs
        float d3[4] = {0, 0, 0, 0};
        if (t < 2) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool v = q < 2 ? va : vb;
                const int r = r0 + g + (q < 2 ? 0 : 8), oc = 2 * t + (q & 1);
                if (!v) continue;
                const float z = o.z3[q], y = Y[(size_t)r * NO + oc];
                const float s = 1.f / (1.f + __expf(-z));
                d3[q] = (s - y) * inv;
                loss += fmaxf(z, 0.f) - z * y + log1pf(__expf(-fabsf(z)));
            }
        }
        // stage X^T, H1^T, H2^T, dZ3^T (cells along the fast axis)
        {
            const int ra = g, rb = g + 8;
            const float x0 = va ? X[(size_t)(r0 + ra) * NF + 2 * t] : 0.f;
            const float x1 = va ? X[(size_t)(r0 + ra) * NF + 2 * t + 1] : 0.f;
            const float y0 = vb ? X[(size_t)(r0 + rb) * NF + 2 * t] : 0.f;
            const float y1 = vb ? X[(size_t)(r0 + rb) * NF + 2 * t + 1] : 0.f;
            XT[w][2 * t][ra] = __float2bfloat16_rn(x0);
            XT[w][2 * t + 1][ra] = __float2bfloat16_rn(x1);
            XT[w][2 * t][rb] = __float2bfloat16_rn(y0);
            XT[w][2 * t + 1][rb] = __float2bfloat16_rn(y1);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                H1T[w][8 * j + 2 * t][ra] = __float2bfloat16_rn(o.h1[j][0]);
                H1T[w][8 * j + 2 * t + 1][ra] = __float2bfloat16_rn(o.h1[j][1]);
                H1T[w][8 * j + 2 * t][rb] = __float2bfloat16_rn(o.h1[j][2]);
                H1T[w][8 * j + 2 * t + 1][rb] = __float2bfloat16_rn(o.h1[j][3]);
                H2T[w][8 * j + 2 * t][ra] = __float2bfloat16_rn(o.h2[j][0]);
                H2T[w][8 * j + 2 * t + 1][ra] = __float2bfloat16_rn(o.h2[j][1]);
                H2T[w][8 * j + 2 * t][rb] = __float2bfloat16_rn(o.h2[j][2]);
                H2T[w][8 * j + 2 * t + 1][rb] = __float2bfloat16_rn(o.h2[j][3]);
            }
            D3T[w][2 * t][ra] = __float2bfloat16_rn(d3[0]);
            D3T[w][2 * t + 1][ra] = __float2bfloat16_rn(d3[1]);
            D3T[w][2 * t][rb] = __float2bfloat16_rn(d3[2]);
            D3T[w][2 * t + 1][rb] = __float2bfloat16_rn(d3[3]);
        }
        // dH2 = dZ3 W3  ([16 x 8] x [8 x 64], K padded to 16); dZ2 = dH2 * (H2 > 0)
        float d2[8][4];
        {
            uint32_t a[4] = {pack2(d3[0], d3[1]), pack2(d3[2], d3[3]), 0u, 0u};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float c[4] = {0, 0, 0, 0};
                uint32_t b[2] = {ld32(Wb + BOFF_W3T + (8 * j + g) * 8 + 2 * t), 0u};
                mma16816(c, a, b);
#pragma unroll
                for (int q = 0; q < 4; ++q) d2[j][q] = o.h2[j][q] > 0.f ? c[q] : 0.f;
            }
        }
        // dH1 = dZ2 W2 ([16 x 64] x [64 x 64]); dZ1 = dH1 * (H1 > 0)
        float d1[8][4];
        {
            uint32_t a[4][4];
#pragma unroll
            for (int kb = 0; kb < 4; ++kb) {
                a[kb][0] = pack2(d2[2 * kb][0], d2[2 * kb][1]);
                a[kb][1] = pack2(d2[2 * kb][2], d2[2 * kb][3]);
                a[kb][2] = pack2(d2[2 * kb + 1][0], d2[2 * kb + 1][1]);
                a[kb][3] = pack2(d2[2 * kb + 1][2], d2[2 * kb + 1][3]);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float c[4] = {0, 0, 0, 0};
#pragma unroll
                for (int kb = 0; kb < 4; ++kb) {
                    uint32_t b[2] = {ld32(Wb + BOFF_W2T + (8 * j + g) * H + 16 * kb + 2 * t),
                                     ld32(Wb + BOFF_W2T + (8 * j + g) * H + 16 * kb + 2 * t + 8)};
                    mma16816(c, a[kb], b);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) d1[j][q] = o.h1[j][q] > 0.f ? c[q] : 0.f;
            }
        }
        // stage dZ2^T, dZ1^T; bias gradients as column sums over the tile's cells
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            D2T[w][8 * j + 2 * t][g] = __float2bfloat16_rn(d2[j][0]);
            D2T[w][8 * j + 2 * t + 1][g] = __float2bfloat16_rn(d2[j][1]);
            D2T[w][8 * j + 2 * t][g + 8] = __float2bfloat16_rn(d2[j][2]);
            D2T[w][8 * j + 2 * t + 1][g + 8] = __float2bfloat16_rn(d2[j][3]);
            D1T[w][8 * j + 2 * t][g] = __float2bfloat16_rn(d1[j][0]);
            D1T[w][8 * j + 2 * t + 1][g] = __float2bfloat16_rn(d1[j][1]);
            D1T[w][8 * j + 2 * t][g + 8] = __float2bfloat16_rn(d1[j][2]);
            D1T[w][8 * j + 2 * t + 1][g + 8] = __float2bfloat16_rn(d1[j][3]);
            // db (FP32): sum over the 16 rows = lanes with the same t
            float s0 = d2[j][0] + d2[j][2], s1 = d2[j][1] + d2[j][3];
            float u0 = d1[j][0] + d1[j][2], u1 = d1[j][1] + d1[j][3];
#pragma unroll
            for (int off = 4; off < 32; off <<= 1) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, off);
                s1 += __shfl_xor_sync(0xffffffffu, s1, off);
                u0 += __shfl_xor_sync(0xffffffffu, u0, off);
                u1 += __shfl_xor_sync(0xffffffffu, u1, off);
            }
            if (g == 0) {
                atomicAdd(&gsum[OFF_B2 + 8 * j + 2 * t], s0);
                atomicAdd(&gsum[OFF_B2 + 8 * j + 2 * t + 1], s1);
                atomicAdd(&gsum[OFF_B1 + 8 * j + 2 * t], u0);
                atomicAdd(&gsum[OFF_B1 + 8 * j + 2 * t + 1], u1);
            }
        }
        {
            float s0 = d3[0] + d3[2], s1 = d3[1] + d3[3];
#pragma unroll
            for (int off = 4; off < 32; off <<= 1) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, off);
                s1 += __shfl_xor_sync(0xffffffffu, s1, off);
            }
            if (g == 0 && t < 2) {
                atomicAdd(&gsum[OFF_B3 + 2 * t], s0);
                atomicAdd(&gsum[OFF_B3 + 2 * t + 1], s1);
            }
        }
        __syncwarp();
        // weight gradients dW = dZ^T A, contracted over the 16 cells (K)
        // dW3 [16 (4 used) x 64] = D3T x H2
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float c[4] = {0, 0, 0, 0};
            uint32_t a[4] = {ld32(&D3T[w][g][2 * t]), ld32(&D3T[w][g + 8][2 * t]), ld32(&D3T[w][g][2 * t + 8]),
                             ld32(&D3T[w][g + 8][2 * t + 8])};
            uint32_t b[2] = {ld32(&H2T[w][8 * j + g][2 * t]), ld32(&H2T[w][8 * j + g][2 * t + 8])};
            mma16816(c, a, b);
            if (g < NO) {
                atomicAdd(&gsum[OFF_W3 + g * H + 8 * j + 2 * t], c[0]);
                atomicAdd(&gsum[OFF_W3 + g * H + 8 * j + 2 * t + 1], c[1]);
            }
        }
        // dW2 [64 x 64] = D2T x H1 ; dW1 [64 x 16 (8 used)] = D1T x X
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            uint32_t a2[4] = {ld32(&D2T[w][16 * m + g][2 * t]), ld32(&D2T[w][16 * m + g + 8][2 * t]),
                              ld32(&D2T[w][16 * m + g][2 * t + 8]), ld32(&D2T[w][16 * m + g + 8][2 * t + 8])};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float c[4] = {0, 0, 0, 0};
                uint32_t b[2] = {ld32(&H1T[w][8 * j + g][2 * t]), ld32(&H1T[w][8 * j + g][2 * t + 8])};
                mma16816(c, a2, b);
                const int o0 = 16 * m + g, i0 = 8 * j + 2 * t;
                atomicAdd(&gsum[OFF_W2 + o0 * H + i0], c[0]);
                atomicAdd(&gsum[OFF_W2 + o0 * H + i0 + 1], c[1]);
                atomicAdd(&gsum[OFF_W2 + (o0 + 8) * H + i0], c[2]);
                atomicAdd(&gsum[OFF_W2 + (o0 + 8) * H + i0 + 1], c[3]);
            }
            uint32_t a1[4] = {ld32(&D1T[w][16 * m + g][2 * t]), ld32(&D1T[w][16 * m + g + 8][2 * t]),
                              ld32(&D1T[w][16 * m + g][2 * t + 8]), ld32(&D1T[w][16 * m + g + 8][2 * t + 8])};
            float c[4] = {0, 0, 0, 0};
            uint32_t b[2] = {ld32(&XT[w][g][2 * t]), ld32(&XT[w][g][2 * t + 8])};
            mma16816(c, a1, b);
            const int o0 = 16 * m + g, f0 = 2 * t;
            atomicAdd(&gsum[OFF_W1 + o0 * NF + f0], c[0]);
            atomicAdd(&gsum[OFF_W1 + o0 * NF + f0 + 1], c[1]);
            atomicAdd(&gsum[OFF_W1 + (o0 + 8) * NF + f0], c[2]);
            atomicAdd(&gsum[OFF_W1 + (o0 + 8) * NF + f0 + 1], c[3]);
        }
        __syncwarp();
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, off);
    if (lane == 0) atomicAdd(&gsum[AVS_MLP_NPARAM], loss);
    __syncthreads();
    for (int e = threadIdx.x; e <= AVS_MLP_NPARAM; e += blockDim.x)
        part[(size_t)blockIdx.x * (AVS_MLP_NPARAM + 1) + e] = gsum[e];
}

// Sum of the block partials in block order (deterministic); grad out, and
// optionally P -= lr * grad.  Entry AVS_MLP_NPARAM is the loss sum / (4 n).
__global__ void k_mlp_reduce(int nblk, const float* __restrict__ part, float* grad, float* P, float lr, float inv_loss)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e > AVS_MLP_NPARAM) return;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * (AVS_MLP_NPARAM + 1) + e];
    if (e == AVS_MLP_NPARAM) {
        grad[e] = s * inv_loss;
        return;
    }
    grad[e] = s;
    if (lr != 0.f) P[e] -= lr * s;
}

// ------------------------------------------------------------------ features and labels
// Per-cell features (rho, U, T, lambda from the cell's moments Wf and heat flux q):
// log rho, U / sqrt(R T_ref) (components; in 2D the third slot is
// |q| / (rho (RT)^1.5)), log T, log(lambda / dx), largest relative jumps of rho
// and T to the face neighbours.  lambda from Eqs. (3)-(4).  W holds NW values
// per cell; for the diatomic (Rykov) gas of Sec. 2.1 the last is rho E_rot and
// T is the translational temperature, (3/2) rho R T_t = rho E - rho U^2/2 -
// rho E_rot, the temperature of G and of the model's viscosity.
template <int D>
__device__ __forceinline__ void feat_prim(const double* W, bool rykov, double& rho, double* U, double& RT)
{
    rho = W[0];
    double m2 = 0.0;
    for (int d = 0; d < D; ++d) {
        U[d] = W[1 + d] / rho;
        m2 += W[1 + d] * W[1 + d];
    }
    double e = W[D + 1] - 0.5 * m2 / rho;
    if (rykov) e -= W[D + 2];
    RT = e / (1.5 * rho);
}

template <int D>
__global__ void k_features(int Nc, int NW, int rykov, const double* __restrict__ Wc, const double* __restrict__ q,
                           const double* __restrict__ vol, const int* __restrict__ nbr,
                           const unsigned char* __restrict__ nslot, double R, double mu_ref, double omega,
                           double T_ref, float* X)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nc) return;
    double rho, U[3], RT;
    feat_prim<D>(Wc + (size_t)i * NW, rykov != 0, rho, U, RT);
    const double T = RT / R;
    const double mu = mu_ref * pow(T / T_ref, omega);
    const double lam = 2.0 * mu * (5 - 2 * omega) * (7 - 2 * omega) / (15.0 * rho * sqrt(2 * AVS_PI * RT));
    const double dx = pow(vol[i], 1.0 / D);
    double q2 = 0.0;
    for (int d = 0; d < D; ++d) q2 += q[(size_t)i * D + d] * q[(size_t)i * D + d];
    double jr = 0.0, jt = 0.0;
    for (int s = 0; s < nslot[i]; ++s) {
        const int j = nbr[i * AVS_MAXS + s];
        if (j < 0) continue;
        double rj, Uj[3], RTj;
        feat_prim<D>(Wc + (size_t)j * NW, rykov != 0, rj, Uj, RTj);
        jr = fmax(jr, fabs(rj - rho) / rho);
        jt = fmax(jt, fabs(RTj / R - T) / T);
    }
    const double su = sqrt(R * T_ref);
    float* x = X + (size_t)i * NF;
    x[0] = (float)log(rho);
    x[1] = (float)(U[0] / su);
    x[2] = (float)(U[1] / su);
    x[3] = D == 3 ? (float)(U[2] / su) : (float)(sqrt(q2) / (rho * RT * sqrt(RT)));
    x[4] = (float)log(T);
    x[5] = (float)log(lam / dx);
    x[6] = (float)jr;
    x[7] = (float)jt;
}

// Labels from the scaled criterion values m_ik = s max(M1, M2) (same
// operation order as the criterion) and M_k:
// 0 split witness (m_ik > C1 below the level cap), 1 dominant (m_ik == M_k,
// M_k >= C2), 2 near-dominant (m_ik >= M_k / 2, M_k >= C2), 3 merge blocker
// (m_ik >= C2 at level >= 1).
template <typename T>
__global__ void k_labels(int D, int NA, int Nv, int Nvp, const T* __restrict__ f, const double* __restrict__ xi,
                         const double* __restrict__ w, const double* __restrict__ cp, const float* __restrict__ xi32,
                         const float* __restrict__ w32, const float* __restrict__ cp32, const double* __restrict__ M,
                         const float4* __restrict__ thr, const int* __restrict__ level, double s, double C1, double C2,
                         const int* __restrict__ ncap, float* Y)
{
    // Every test is first decided on the FP32 screening interval of m_ik
    // (crit32); a test whose threshold lies within 2^-20 relative of the
    // interval is decided in FP64 as in the definition.
    constexpr float eps = 0x1p-20f;
    const int i = blockIdx.x;
    const double* p = cp + (size_t)i * 5;
    const float* p32 = cp32 + (size_t)i * 8;
    const float s32 = (float)s, C1f = (float)C1 * kCritScale, C2f = (float)C2 * kCritScale;
    int y0 = 0, y1 = 0, y2 = 0, y3 = 0;
    for (int k = threadIdx.x; k < Nv; k += blockDim.x) {
        const T Gt = f[(size_t)i * NA * Nvp + k];
        float xf[3];
        for (int d = 0; d < D; ++d) xf[d] = xi32[(size_t)k * D + d];
        float m32, B;
        crit32(D, crit_scaled(Gt), w32[k], xf, p32, m32, B);
        const float lo = s32 * (m32 - B), hi = s32 * (m32 + B);
        const float4 t = thr[k];               // act, M_k, 0.5 s M_k (scaled like m32)
        const int lv = level[k], lcap = ncap[k];
        const bool act = t.x != 0.0f;
        bool amb = false;
        if (lv < lcap && !y0) {
            if (lo > C1f * (1.0f + eps)) y0 = 1;
            else if (!(hi < C1f * (1.0f - eps))) amb = true;
        }
        if (lv >= 1 && !y3) {
            if (lo > C2f * (1.0f + eps)) y3 = 1;
            else if (!(hi < C2f * (1.0f - eps))) amb = true;
        }
        if (act) {
            if (!y1 && !(m32 + B < t.y - fabsf(t.y) * eps)) amb = true;
            if (!y2) {
                if (lo > t.z + fabsf(t.z) * eps) y2 = 1;
                else if (!(hi < t.z - fabsf(t.z) * eps)) amb = true;
            }
        }
        if (!amb) continue;
        const double wg = __dmul_rn(w[k], (double)Gt);
        const double m1 = __ddiv_rn(wg, p[0]);
        double c2 = 0.0;
        for (int d = 0; d < D; ++d) {
            const double cc = __dsub_rn(xi[(size_t)k * D + d], p[1 + d]);
            c2 = __dadd_rn(c2, __dmul_rn(cc, cc));
        }
        const double m2 = __ddiv_rn(__dmul_rn(__dmul_rn(0.5, wg), c2), p[4]);
        const double mk = m1 > m2 ? m1 : m2;
        const double Mk = M[k];
        const double sm = __dmul_rn(s, mk), sM = __dmul_rn(s, Mk);
        const bool actd = sM >= C2;
        y0 |= (sm > C1 && lv < lcap);
        y1 |= (actd && sm == sM);
        y2 |= (actd && sm >= 0.5 * sM);
        y3 |= (sm >= C2 && lv >= 1);
    }
    y0 = __syncthreads_or(y0);
    y1 = __syncthreads_or(y1);
    y2 = __syncthreads_or(y2);
    y3 = __syncthreads_or(y3);
    if (threadIdx.x == 0) {
        Y[(size_t)i * NO + 0] = (float)y0;
        Y[(size_t)i * NO + 1] = (float)y1;
        Y[(size_t)i * NO + 2] = (float)y2;
        Y[(size_t)i * NO + 3] = (float)y3;
    }
}

// per-node thresholds of the label tests: (s M_k >= C2, M_k, 0.5 s M_k) in FP32,
// the last two scaled by 2^64 like the screening values
__global__ void k_label_thr(int Nv, const double* __restrict__ M, double s, double C2, float4* thr)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nv) return;
    const double sM = __dmul_rn(s, M[k]);
    thr[k] = make_float4(sM >= C2 ? 1.0f : 0.0f, (float)(M[k] * 0x1p64), (float)(0.5 * sM * 0x1p64), 0.0f);
}

// check set: cells whose dominant logit reaches the threshold.  The cell
// attaining M_k decides both the split test (M_k > C1) and whether node k
// blocks a merge (M_k >= C2); a check set holding every dominant cell would
// reproduce the full criterion's decisions, a budgeted one misses some and the
// full criterion (run every n-th adaptation) measures and repairs them.
// Appended in any order (the criterion's max is order-free).
__global__ void k_checkset(int Nc, const float* __restrict__ logits, float zthr, int* list, int* count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nc) return;
    const float* z = logits + (size_t)i * NO;
    if (z[1] >= zthr) list[atomicAdd(count, 1)] = i;
}

// nodes whose split or merge-candidate decision differs between the criterion
// over all cells (Mf) and over the check set (Ms)
__global__ void k_misses(int Nv, const double* __restrict__ Mf, const double* __restrict__ Ms, double s, double C1,
                         double C2, int* count)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nv) return;
    const double a = __dmul_rn(s, Mf[k]), b = __dmul_rn(s, Ms[k]);
    if ((a > C1) != (b > C1) || (a < C2) != (b < C2)) atomicAdd(count, 1);
}

// ------------------------------------------------------------------ launchers
// Threshold of the check set: the dominant logit that keeps the top `budget`
// fraction of the cells of the current state (order statistic on the host).
cudaError_t mlp_calibrate(avs_ctx* c, float budget)
{
    CK_RET(mlp_forward(c, c->Nc, c->mlp_X, c->mlp_logits));
    std::vector<float> z((size_t)c->Nc * NO);
    CK_RET(cudaMemcpyAsync(z.data(), c->mlp_logits, sizeof(float) * z.size(), cudaMemcpyDeviceToHost, c->stream));
    CK_RET(cudaStreamSynchronize(c->stream));
    std::vector<float> d(c->Nc);
    for (int i = 0; i < c->Nc; ++i) d[i] = z[(size_t)i * NO + 1];
    const int keep = std::max(1, std::min(c->Nc, (int)ceilf(budget * (float)c->Nc)));
    std::nth_element(d.begin(), d.begin() + (c->Nc - keep), d.end());
    c->mlp_zthr = d[c->Nc - keep] - 1e-6f * fabsf(d[c->Nc - keep]);
    return cudaSuccess;
}

cudaError_t mlp_misses(avs_ctx* c, const double* Mf, const double* Ms, int* count)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    k_misses<<<(c->Nv + 255) / 256, 256, 0, c->stream>>>(c->Nv, Mf, Ms, c->s_norm, c->cfg.C1, c->cfg.C2, count);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t mlp_prep(avs_ctx* c)
{
    k_mlp_prep<<<(BSIZE + 255) / 256, 256, 0, c->stream>>>(c->mlp_P, (__nv_bfloat16*)c->mlp_Wb);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t mlp_forward(avs_ctx* c, int n, const float* X, float* logits)
{
    const int tiles = (n + 15) / 16;
    const int blocks = std::min(1024, (tiles + 3) / 4);
    if (n > 0) {
        k_mlp_fwd<<<blocks, 128, 0, c->stream>>>(n, X, c->mlp_P, (const __nv_bfloat16*)c->mlp_Wb, logits);
        c->launches += 1;
    }
    return cudaGetLastError();
}

cudaError_t mlp_grad_step(avs_ctx* c, int n, const float* X, const float* Y, float lr, float* grad_out)
{
    if (n <= 0) return cudaSuccess;
    const int tiles = (n + 15) / 16;
    const int blocks = std::min(AVS_MLP_MAXBLK, (tiles + 3) / 4);
    k_mlp_fwdbwd<<<blocks, 128, 0, c->stream>>>(n, X, Y, c->mlp_P, (const __nv_bfloat16*)c->mlp_Wb, c->mlp_part);
    k_mlp_reduce<<<(AVS_MLP_NPARAM + 256) / 256, 256, 0, c->stream>>>(blocks, c->mlp_part, grad_out, c->mlp_P, lr,
                                                                       1.0f / (4.0f * (float)n));
    c->launches += 2;
    if (lr != 0.f) return mlp_prep(c);
    return cudaGetLastError();
}

cudaError_t mlp_features(avs_ctx* c, const double* Wc, const double* q, float* X)
{
    const int rk = c->model == AVS_RYKOV;
    if (c->D == 2)
        k_features<2><<<(c->Nc + 127) / 128, 128, 0, c->stream>>>(c->Nc, c->NW, rk, Wc, q, c->vol, c->nbr, c->nslot,
                                                                  c->cfg.R, c->mu_ref, c->cfg.omega, c->cfg.T_ref, X);
    else
        k_features<3><<<(c->Nc + 127) / 128, 128, 0, c->stream>>>(c->Nc, c->NW, rk, Wc, q, c->vol, c->nbr, c->nslot,
                                                                  c->cfg.R, c->mu_ref, c->cfg.omega, c->cfg.T_ref, X);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t mlp_labels(avs_ctx* c, const void* f, float* Y)
{
    // the criterion's per-cell inputs (crit_cp, crit_cp32) and M are those of
    // the full criterion evaluated just before
    float4* thr = (float4*)c->Mthr;
    k_label_thr<<<(c->Nv + 255) / 256, 256, 0, c->stream>>>(c->Nv, c->M, c->s_norm, c->cfg.C2, thr);
    if (c->mixed)
        k_labels<float><<<c->Nc, 256, 0, c->stream>>>(c->D, c->NA, c->Nv, c->Nvp, (const float*)f, c->xi_d, c->w_d,
                                                      c->crit_cp, c->xi_f, c->w_f, c->crit_cp32, c->M, thr, c->level,
                                                      c->s_norm, c->cfg.C1, c->cfg.C2, c->ncap, Y);
    else
        k_labels<double><<<c->Nc, 256, 0, c->stream>>>(c->D, c->NA, c->Nv, c->Nvp, (const double*)f, c->xi_d,
                                                       c->w_d, c->crit_cp, c->xi_f, c->w_f, c->crit_cp32, c->M, thr,
                                                       c->level, c->s_norm, c->cfg.C1, c->cfg.C2, c->ncap,
                                                       Y);
    c->launches += 2;
    return cudaGetLastError();
}

cudaError_t mlp_checkset(avs_ctx* c, const float* logits, float zthr, int* list, int* count)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    k_checkset<<<(c->Nc + 255) / 256, 256, 0, c->stream>>>(c->Nc, logits, zthr, list, count);
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace avs
