// mlp.cu -- learned calibration surrogate of the pseudopotential model.
//
// The paper notes that the pseudopotential model needs preliminary simulations to fix
// its parameters (Secs. 3, 5.1, 5.2: sigma^Li, kappa^P, kappa^Li and the densities,
// width and surface tension they give).  This surrogate maps (Tr, a, b, kappa^P) to the
// calibration observables (rho_l, rho_v, W, sigma) of such runs: an MLP 4 -> 128 -> 128 ->
// 128 -> 4 with GELU, 34,180 weights, trained in FP32 on the GPU by the kernels below
// (tiled SGEMM forward/backward with split-K weight gradients, GELU, MSE, Adam), and
// evaluated by one fused kernel with BF16 inputs and weights and FP32 accumulation on the
// tensor cores (mma.sync m16n8k16).  Inputs and outputs are standardised with the training
// set's statistics; rho_v is learned as ln(rho_v).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "../../include/lbm.h"

namespace {

thread_local char g_mlp_msg[256] = "";
int mfail(cudaError_t e, const char* what) {
    snprintf(g_mlp_msg, sizeof(g_mlp_msg), "%s: %s", what, cudaGetErrorString(e));
    return LBM_ERR_CUDA;
}
#define MCK(call)                                             \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return mfail(e_, #call);       \
    } while (0)

constexpr int kIn = 4, kHid = 128, kOut = 4, kLayers = 4;
__device__ constexpr int kDims[kLayers + 1] = {kIn, kHid, kHid, kHid, kOut};
// parameter offsets: W_l (out x in, row-major) then b_l
__host__ __device__ constexpr int woff(int l) {
    int o = 0;
    for (int i = 0; i < l; ++i) o += kDims[i + 1] * kDims[i] + kDims[i + 1];
    return o;
}
__host__ __device__ constexpr int boff(int l) { return woff(l) + kDims[l + 1] * kDims[l]; }
constexpr int kNumParams = woff(kLayers);
static_assert(kNumParams == 34180, "4-128-128-128-4 MLP has 34,180 parameters");

// ---------------------------------------------------------------------------------------
// FP32 kernels

// C[M x N] (+)= sum_k A(m, k) B(k, n), A element (m, k) at A[m*sam + k*sak], B (k, n) at
// B[k*sbk + n*sbn]; 64 x 64 tiles, 16-deep K slices, 4 x 4 outputs per thread.  With
// gridDim.z > 1 each z-slice handles a K range and accumulates into C atomically (C must be
// zeroed first); otherwise C = result (+ bias[n] if given).
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, const float* __restrict__ A, int sam,
                                                    int sak, const float* __restrict__ B, int sbk, int sbn,
                                                    float* __restrict__ C, int ldc, const float* __restrict__ bias) {
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int kchunk = (K + gridDim.z - 1) / gridDim.z;
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    float acc[4][4] = {};
    for (int k0 = kbeg; k0 < kend; k0 += 16) {
        // consecutive threads walk the operand's contiguous index (k or m/n) for coalescing
        for (int i = threadIdx.x; i < 16 * 64; i += 256) {
            const int kk = sak == 1 ? i % 16 : i / 64, mm = sak == 1 ? i / 16 : i % 64;
            const int gk = k0 + kk;
            As[kk][mm] = (m0 + mm < M && gk < kend) ? A[(size_t)(m0 + mm) * sam + (size_t)gk * sak] : 0.0f;
        }
        for (int i = threadIdx.x; i < 16 * 64; i += 256) {
            const int kk = sbk == 1 ? i % 16 : i / 64, nn = sbk == 1 ? i / 16 : i % 64;
            const int gk = k0 + kk;
            Bs[kk][nn] = (n0 + nn < N && gk < kend) ? B[(size_t)gk * sbk + (size_t)(n0 + nn) * sbn] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[kk][ty * 4 + i];
                b[i] = Bs[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m < M && n < N) {
                if (gridDim.z > 1)
                    atomicAdd(&C[(size_t)m * ldc + n], acc[i][j]);
                else
                    C[(size_t)m * ldc + n] = acc[i][j] + (bias ? bias[n] : 0.0f);
            }
        }
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    // d/dz [z Phi(z)] = Phi(z) + z phi(z)
    const float Phi = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
    const float phi = 0.39894228040143268f * expf(-0.5f * z * z);
    return Phi + z * phi;
}

__global__ void gelu_fwd_kernel(const float* __restrict__ Z, float* __restrict__ A, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) A[i] = gelu(Z[i]);
}

// dZ = dA * GELU'(Z) (in place on dA)
__global__ void gelu_bwd_kernel(const float* __restrict__ Z, float* __restrict__ dA, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dA[i] *= gelu_grad(Z[i]);
}

// Mean squared error over the finite targets (a NaN target is missing: no loss, no
// gradient): dZ = 2 (Z - Y) / n_valid; loss accumulated as sum of squares / n_valid.
__global__ void mse_kernel(const float* __restrict__ Z, const float* __restrict__ Y, float* __restrict__ dZ, int count,
                           float inv_valid, float* __restrict__ loss) {
    float s = 0.0f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const float y = Y[i];
        const float d = isnan(y) ? 0.0f : Z[i] - y;
        dZ[i] = 2.0f * d * inv_valid;
        s += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, s * inv_valid);
}

// db[j] = sum_i dZ[i, j]
__global__ void bias_grad_kernel(const float* __restrict__ dZ, int n, int m, float* __restrict__ db) {
    const int j = blockIdx.x;
    float s = 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += dZ[(size_t)i * m + j];
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[j] = red[0];
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, int n, float lr, float b1, float b2, float eps, float c1, float c2,
                            float wd) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.0f - b1) * gi;
        const float v = b2 * m2[i] + (1.0f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = v;
        p[i] -= lr * ((a / c1) / (sqrtf(v / c2) + eps) + wd * p[i]);
    }
}

// (raw inputs, raw targets) -> standardised network inputs / targets (rho_v as ln rho_v)
__global__ void standardise_kernel(const float* __restrict__ X, const float* __restrict__ Yraw, int n,
                                   const float* __restrict__ stats, float* __restrict__ Xn, float* __restrict__ Yn) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        for (int j = 0; j < kIn; ++j) Xn[i * kIn + j] = (X[i * kIn + j] - stats[j]) / stats[4 + j];
        if (Yraw)
            for (int j = 0; j < kOut; ++j) {
                const float y = j == 1 ? logf(Yraw[i * kOut + j]) : Yraw[i * kOut + j];
                Yn[i * kOut + j] = (y - stats[8 + j]) / stats[12 + j];
            }
    }
}

// ---------------------------------------------------------------------------------------
// Fused BF16 inference: one CTA of 128 threads (4 warps) evaluates 64 queries through all four
// layers.  Each layer is an mma.sync m16n8k16 BF16 GEMM with FP32 accumulators; bias + GELU
// run in FP32 and the activations stay FP32 in shared memory; the output layer is
// de-standardised (and rho_v exponentiated) in FP32.
//
// Split mode (kSplit): every FP32 operand x is carried as two BF16 numbers, hi = bf16(x) and
// lo = bf16(x - hi), and each tile accumulates hi*hi + lo*hi + hi*lo (the lo*lo term, below
// 2^-16 relative, is dropped): BF16 tensor-core products with FP32 accumulation that keep the
// result within ~2^-16 of the FP32 network.  Single mode rounds every operand to BF16 once
// (relative 2^-8), which costs up to ~1% in rho_v because ln rho_v spans several units.
constexpr int kQ = 64;                    // queries per CTA
constexpr int kInPad = 16;                // first layer K padded to one MMA K step
constexpr int kActStride = kHid + 4;      // floats per activation row (bank spread)
constexpr int kWStride = kHid + 8;        // bf16 elements per weight row
constexpr int kPackHalf = kHid * kInPad + 2 * kHid * kHid + 8 * kHid;  // bf16 elements of hi (or lo)

struct InferSmem {
    __nv_bfloat16 w1[2][kHid][kInPad];          // layer 1 weights (hi, lo), K padded
    __nv_bfloat16 w[2][2][kHid][kWStride];      // layers 2, 3 (layer, hi/lo)
    __nv_bfloat16 w4[2][8][kWStride];           // layer 4 (hi, lo), N padded to 8
    float bias[3][kHid];
    float b4[8];
    float act[2][kQ][kActStride];               // ping-pong FP32 activations
    float stats[16];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// (x, y) -> hi = bf16x2(x, y), lo = bf16x2(x - hi.x, y - hi.y)
__device__ __forceinline__ void split_bf16(float2 v, uint32_t& hi, uint32_t& lo) {
    __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
    const float2 hf = __bfloat1622float2(h);
    __nv_bfloat162 l = __floats2bfloat162_rn(v.x - hf.x, v.y - hf.y);
    hi = *reinterpret_cast<uint32_t*>(&h);
    lo = *reinterpret_cast<uint32_t*>(&l);
}

// D (16x8, f32) += A (16x16, bf16, row) * B (16x8, bf16, col)
__device__ __forceinline__ void mma_bf16(float d[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A fragment (rows row0..row0+15, k0..k0+15) from FP32 activations, as BF16 hi and lo parts.
__device__ __forceinline__ void load_a_frag(const float* base, int row0, int k0, int lane, uint32_t ah[4],
                                            uint32_t al[4]) {
    const int g = lane >> 2, t = lane & 3;
    const float* p0 = base + (row0 + g) * kActStride + k0 + t * 2;
    const float* p1 = base + (row0 + g + 8) * kActStride + k0 + t * 2;
    split_bf16(*reinterpret_cast<const float2*>(p0), ah[0], al[0]);
    split_bf16(*reinterpret_cast<const float2*>(p1), ah[1], al[1]);
    split_bf16(*reinterpret_cast<const float2*>(p0 + 8), ah[2], al[2]);
    split_bf16(*reinterpret_cast<const float2*>(p1 + 8), ah[3], al[3]);
}
// B fragment from a weight array stored as W[n][k] (= column-major B).
__device__ __forceinline__ void load_b_frag(const __nv_bfloat16* W, int stride, int n0, int k0, int lane,
                                            uint32_t b[2]) {
    const int g = lane >> 2, t = lane & 3;
    const __nv_bfloat16* p = W + (n0 + g) * stride + k0 + t * 2;
    b[0] = *reinterpret_cast<const uint32_t*>(p);
    b[1] = *reinterpret_cast<const uint32_t*>(p + 8);
}

template <bool kSplit>
__device__ __forceinline__ void mma_tile(float d[4], const uint32_t ah[4], const uint32_t al[4],
                                         const __nv_bfloat16* Whi, const __nv_bfloat16* Wlo, int stride, int n0,
                                         int k0, int lane) {
    uint32_t bh[2];
    load_b_frag(Whi, stride, n0, k0, lane, bh);
    mma_bf16(d, ah, bh);
    if (kSplit) {
        uint32_t bl[2];
        load_b_frag(Wlo, stride, n0, k0, lane, bl);
        mma_bf16(d, al, bh);
        mma_bf16(d, ah, bl);
    }
}

template <bool kSplit>
__global__ void __launch_bounds__(128) mlp_infer_bf16_kernel(const float* __restrict__ X, int n,
                                                             const __nv_bfloat16* __restrict__ wpack,
                                                             const float* __restrict__ bpack,
                                                             const float* __restrict__ stats, float* __restrict__ Y) {
    extern __shared__ __align__(16) unsigned char ism[];
    InferSmem& s = *reinterpret_cast<InferSmem*>(ism);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // stage weights: wpack holds [hi | lo], each w1 [128][16], w2, w3 [128][128], w4 [8][128]
    for (int h = 0; h < (kSplit ? 2 : 1); ++h) {
        const __nv_bfloat16* src = wpack + h * kPackHalf;
        for (int i = tid; i < kHid * kInPad; i += 128) (&s.w1[h][0][0])[i] = src[i];
        for (int l = 0; l < 2; ++l)
            for (int i = tid; i < kHid * kHid; i += 128)
                s.w[l][h][i / kHid][i % kHid] = src[kHid * kInPad + l * kHid * kHid + i];
        for (int i = tid; i < 8 * kHid; i += 128)
            s.w4[h][i / kHid][i % kHid] = src[kHid * kInPad + 2 * kHid * kHid + i];
    }
    for (int i = tid; i < 3 * kHid; i += 128) (&s.bias[0][0])[i] = bpack[i];
    if (tid < 8) s.b4[tid] = bpack[3 * kHid + tid];
    if (tid < 16) s.stats[tid] = stats[tid];
    __syncthreads();
    const int q0 = blockIdx.x * kQ;
    // standardised inputs (K padded to 16 with zeros)
    for (int i = tid; i < kQ * kInPad; i += 128) {
        const int r = i / kInPad, k = i % kInPad;
        float v = 0.0f;
        if (k < kIn && q0 + r < n) v = (X[(size_t)(q0 + r) * kIn + k] - s.stats[k]) / s.stats[4 + k];
        s.act[0][r][k] = v;
    }
    __syncthreads();
    // each warp owns 16 query rows; three hidden layers of N = 128 (16 n-tiles of 8)
    const int row0 = warp * 16;
    const int g = lane >> 2, t = lane & 3;
    int cur = 0;
    for (int layer = 0; layer < 3; ++layer) {
        const int ksteps = layer == 0 ? 1 : kHid / 16;
        const __nv_bfloat16* Whi = layer == 0 ? &s.w1[0][0][0] : &s.w[layer - 1][0][0][0];
        const __nv_bfloat16* Wlo = layer == 0 ? &s.w1[1][0][0] : &s.w[layer - 1][1][0][0];
        const int wstride = layer == 0 ? kInPad : kWStride;
        float acc[16][4];
#pragma unroll
        for (int nt = 0; nt < 16; ++nt)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[nt][j] = 0.0f;
        for (int ks = 0; ks < ksteps; ++ks) {
            uint32_t ah[4], al[4];
            load_a_frag(&s.act[cur][0][0], row0, ks * 16, lane, ah, al);
#pragma unroll
            for (int nt = 0; nt < 16; ++nt) mma_tile<kSplit>(acc[nt], ah, al, Whi, Wlo, wstride, nt * 8, ks * 16, lane);
        }
        // bias + GELU in FP32 into the other activation buffer (rows of this warp only)
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            const int c = nt * 8 + t * 2;
            const float b0 = s.bias[layer][c], b1 = s.bias[layer][c + 1];
            *reinterpret_cast<float2*>(&s.act[cur ^ 1][row0 + g][c]) =
                make_float2(gelu(acc[nt][0] + b0), gelu(acc[nt][1] + b1));
            *reinterpret_cast<float2*>(&s.act[cur ^ 1][row0 + g + 8][c]) =
                make_float2(gelu(acc[nt][2] + b0), gelu(acc[nt][3] + b1));
        }
        __syncwarp();
        cur ^= 1;
    }
    // output layer: N = 8 (4 used)
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int ks = 0; ks < kHid / 16; ++ks) {
        uint32_t ah[4], al[4];
        load_a_frag(&s.act[cur][0][0], row0, ks * 16, lane, ah, al);
        mma_tile<kSplit>(acc, ah, al, &s.w4[0][0][0], &s.w4[1][0][0], kWStride, 0, ks * 16, lane);
    }
    for (int half = 0; half < 2; ++half) {
        const int r = row0 + g + half * 8;
        for (int j = 0; j < 2; ++j) {
            const int c = t * 2 + j;
            if (c < kOut && q0 + r < n) {
                float y = (acc[half * 2 + j] + s.b4[c]) * s.stats[12 + c] + s.stats[8 + c];
                if (c == 1) y = expf(y);
                Y[(size_t)(q0 + r) * kOut + c] = y;
            }
        }
    }
}

// FP32 reference evaluation (the training forward pass) de-standardised, for comparison.
__global__ void destandardise_kernel(const float* __restrict__ Zn, int n, const float* __restrict__ stats,
                                     float* __restrict__ Y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * kOut; i += gridDim.x * blockDim.x) {
        const int c = i % kOut;
        float y = Zn[i] * stats[12 + c] + stats[8 + c];
        Y[i] = c == 1 ? expf(y) : y;
    }
}

// FP32 parameters -> BF16 hi and lo weight blocks (zero padded) and FP32 biases
__global__ void pack_weights_kernel(const float* __restrict__ P, __nv_bfloat16* __restrict__ wpack,
                                    float* __restrict__ bpack) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (int i = tid; i < kPackHalf; i += stride) {
        float w = 0.0f;
        if (i < kHid * kInPad) {
            const int o = i / kInPad, k = i % kInPad;
            w = k < kIn ? P[woff(0) + o * kIn + k] : 0.0f;
        } else if (i < kHid * kInPad + 2 * kHid * kHid) {
            const int j = i - kHid * kInPad, l = j / (kHid * kHid);
            w = P[woff(l + 1) + j % (kHid * kHid)];
        } else {
            const int j = i - kHid * kInPad - 2 * kHid * kHid, o = j / kHid, k = j % kHid;
            w = o < kOut ? P[woff(3) + o * kHid + k] : 0.0f;
        }
        const __nv_bfloat16 hi = __float2bfloat16_rn(w);
        wpack[i] = hi;
        wpack[kPackHalf + i] = __float2bfloat16_rn(w - __bfloat162float(hi));
    }
    for (int i = tid; i < 3 * kHid; i += stride) bpack[i] = P[boff(i / kHid) + i % kHid];
    for (int i = tid; i < 8; i += stride) bpack[3 * kHid + i] = i < kOut ? P[boff(3) + i] : 0.0f;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Host side

struct lbm_surrogate {
    int cap;                  // allocated rows
    float* d_params;          // kNumParams
    float* d_grad;
    float* d_m1;
    float* d_m2;
    float* d_stats;           // in mean[4], in std[4], out mean[4], out std[4]
    float* d_X;               // raw inputs (cap x 4)
    float* d_Yraw;            // raw targets
    float* d_Xn;              // standardised
    float* d_Yn;
    float* d_Z[kLayers];      // pre-activations per layer (cap x dim)
    float* d_A[kLayers - 1];  // activations of hidden layers
    float* d_dZ[kLayers];
    float* d_dA;              // scratch (cap x 128)
    float* d_loss;
    __nv_bfloat16* d_wpack;
    float* d_bpack;
    float* d_out;
    float h_stats[16];
    int steps_done;
    cudaStream_t stream;
    float last_loss;
};

namespace {

int sgemm(cudaStream_t s, int M, int N, int K, const float* A, int sam, int sak, const float* B, int sbk, int sbn,
          float* C, int ldc, const float* bias, int splitk) {
    dim3 grid((N + 63) / 64, (M + 63) / 64, splitk);
    if (splitk > 1) MCK(cudaMemsetAsync(C, 0, sizeof(float) * (size_t)M * ldc, s));
    sgemm_kernel<<<grid, 256, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias);
    MCK(cudaGetLastError());
    return LBM_OK;
}

int alloc_rows(lbm_surrogate* m, int n) {
    if (n <= m->cap) return LBM_OK;
    auto drop = [](float** b) {
        if (*b) cudaFree(*b);
        *b = nullptr;
    };
    float** bufs[] = {&m->d_X, &m->d_Yraw, &m->d_Xn, &m->d_Yn, &m->d_dA, &m->d_out};
    for (float** b : bufs) drop(b);
    for (int l = 0; l < kLayers; ++l) {
        drop(&m->d_Z[l]);
        drop(&m->d_dZ[l]);
        if (l < kLayers - 1) drop(&m->d_A[l]);
    }
    m->cap = 0;
    const size_t r = (size_t)n;
    MCK(cudaMalloc(&m->d_X, r * kIn * 4));
    MCK(cudaMalloc(&m->d_Yraw, r * kOut * 4));
    MCK(cudaMalloc(&m->d_Xn, r * kIn * 4));
    MCK(cudaMalloc(&m->d_Yn, r * kOut * 4));
    MCK(cudaMalloc(&m->d_dA, r * kHid * 4));
    MCK(cudaMalloc(&m->d_out, r * kOut * 4));
    for (int l = 0; l < kLayers; ++l) {
        MCK(cudaMalloc(&m->d_Z[l], r * kDims[l + 1] * 4));
        MCK(cudaMalloc(&m->d_dZ[l], r * kDims[l + 1] * 4));
        if (l < kLayers - 1) MCK(cudaMalloc(&m->d_A[l], r * kDims[l + 1] * 4));
    }
    m->cap = n;
    return LBM_OK;
}

// forward pass on d_Xn rows [0, n): fills d_Z, d_A
int forward(lbm_surrogate* m, int n) {
    const float* in = m->d_Xn;
    for (int l = 0; l < kLayers; ++l) {
        const int din = kDims[l], dout = kDims[l + 1];
        // Z[n x dout] = in[n x din] W^T + b, W row-major [dout][din]: B(k, j) = W[j*din + k]
        int rc = sgemm(m->stream, n, dout, din, in, din, 1, m->d_params + woff(l), 1, din, m->d_Z[l], dout,
                       m->d_params + boff(l), 1);
        if (rc) return rc;
        if (l < kLayers - 1) {
            gelu_fwd_kernel<<<256, 256, 0, m->stream>>>(m->d_Z[l], m->d_A[l], n * dout);
            in = m->d_A[l];
        }
    }
    MCK(cudaGetLastError());
    return LBM_OK;
}

// backward pass of the MSE loss against d_Yn (n_valid finite targets): fills d_grad and
// *loss (device)
int backward(lbm_surrogate* m, int n, long long n_valid) {
    MCK(cudaMemsetAsync(m->d_loss, 0, sizeof(float), m->stream));
    mse_kernel<<<64, 256, 0, m->stream>>>(m->d_Z[kLayers - 1], m->d_Yn, m->d_dZ[kLayers - 1], n * kOut,
                                          (float)(1.0 / (double)n_valid), m->d_loss);
    for (int l = kLayers - 1; l >= 0; --l) {
        const int din = kDims[l], dout = kDims[l + 1];
        const float* Ain = l == 0 ? m->d_Xn : m->d_A[l - 1];
        // dW[dout x din] = dZ^T[dout x n] Ain[n x din]: A(i, k) = dZ[k*dout + i], B(k, j) = Ain[k*din + j]
        const int split = std::max(1, std::min(64, n / 128));
        int rc = sgemm(m->stream, dout, din, n, m->d_dZ[l], 1, dout, Ain, din, 1, m->d_grad + woff(l), din, nullptr,
                       split);
        if (rc) return rc;
        bias_grad_kernel<<<dout, 256, 0, m->stream>>>(m->d_dZ[l], n, dout, m->d_grad + boff(l));
        if (l > 0) {
            // dA[n x din] = dZ[n x dout] W[dout x din]
            rc = sgemm(m->stream, n, din, dout, m->d_dZ[l], dout, 1, m->d_params + woff(l), din, 1, m->d_dZ[l - 1],
                       din, nullptr, 1);
            if (rc) return rc;
            gelu_bwd_kernel<<<256, 256, 0, m->stream>>>(m->d_Z[l - 1], m->d_dZ[l - 1], n * din);
        }
    }
    MCK(cudaGetLastError());
    return LBM_OK;
}

// finite target entries (each set needs a finite rho_v > 0; other outputs may be NaN = missing)
long long valid_targets(const float* Y, int n) {
    long long c = 0;
    for (long long i = 0; i < (long long)n * kOut; ++i) {
        if (i % kOut == 1 && !(Y[i] > 0.0f && std::isfinite(Y[i]))) return -1;
        c += std::isfinite(Y[i]) ? 1 : 0;
    }
    return c;
}

int upload_inputs(lbm_surrogate* m, const float* X, const float* Y, int n) {
    int rc = alloc_rows(m, n);
    if (rc) return rc;
    MCK(cudaMemcpyAsync(m->d_X, X, sizeof(float) * n * kIn, cudaMemcpyHostToDevice, m->stream));
    if (Y) MCK(cudaMemcpyAsync(m->d_Yraw, Y, sizeof(float) * n * kOut, cudaMemcpyHostToDevice, m->stream));
    standardise_kernel<<<64, 256, 0, m->stream>>>(m->d_X, Y ? m->d_Yraw : nullptr, n, m->d_stats, m->d_Xn, m->d_Yn);
    MCK(cudaGetLastError());
    return LBM_OK;
}

}  // namespace

extern "C" const char* lbm_surrogate_last_error(void) { return g_mlp_msg; }

extern "C" int lbm_surrogate_num_params(void) { return kNumParams; }

extern "C" void lbm_surrogate_destroy(lbm_surrogate* m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    float* bufs[] = {m->d_params, m->d_grad, m->d_m1, m->d_m2, m->d_stats, m->d_X, m->d_Yraw, m->d_Xn,
                     m->d_Yn, m->d_dA, m->d_loss, m->d_bpack, m->d_out};
    for (float* b : bufs)
        if (b) cudaFree(b);
    for (int l = 0; l < kLayers; ++l) {
        if (m->d_Z[l]) cudaFree(m->d_Z[l]);
        if (m->d_dZ[l]) cudaFree(m->d_dZ[l]);
        if (l < kLayers - 1 && m->d_A[l]) cudaFree(m->d_A[l]);
    }
    if (m->d_wpack) cudaFree(m->d_wpack);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

extern "C" int lbm_surrogate_create(const float* stats16, unsigned seed, lbm_surrogate** out) {
    if (!out || !stats16) return LBM_ERR_ARG;
    *out = nullptr;
    for (int j = 0; j < 4; ++j)
        if (!(stats16[4 + j] > 0) || !(stats16[12 + j] > 0)) return LBM_ERR_ARG;
    lbm_surrogate* m = new (std::nothrow) lbm_surrogate();
    if (!m) return LBM_ERR_ARG;
    auto fail = [&](int rc) {
        lbm_surrogate_destroy(m);
        return rc;
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking)) != cudaSuccess) return fail(mfail(e, "stream"));
    float** bufs[] = {&m->d_params, &m->d_grad, &m->d_m1, &m->d_m2};
    for (float** b : bufs)
        if ((e = cudaMalloc(b, sizeof(float) * kNumParams)) != cudaSuccess) return fail(mfail(e, "cudaMalloc(params)"));
    if ((e = cudaMalloc(&m->d_stats, sizeof(float) * 16)) != cudaSuccess ||
        (e = cudaMalloc(&m->d_loss, sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&m->d_wpack, sizeof(__nv_bfloat16) * 2 * kPackHalf)) !=
            cudaSuccess ||
        (e = cudaMalloc(&m->d_bpack, sizeof(float) * (3 * kHid + 8))) != cudaSuccess)
        return fail(mfail(e, "cudaMalloc"));
    std::memcpy(m->h_stats, stats16, sizeof(m->h_stats));
    // He-style initialisation (uniform, seeded); zero biases
    std::vector<float> p(kNumParams, 0.0f);
    std::mt19937 rng(seed);
    for (int l = 0; l < kLayers; ++l) {
        const float lim = std::sqrt(6.0f / kDims[l]);
        std::uniform_real_distribution<float> U(-lim, lim);
        for (int i = 0; i < kDims[l + 1] * kDims[l]; ++i) p[woff(l) + i] = U(rng) * (l == kLayers - 1 ? 0.1f : 1.0f);
    }
    if ((e = cudaMemcpy(m->d_params, p.data(), sizeof(float) * kNumParams, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(m->d_stats, stats16, sizeof(float) * 16, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(m->d_m1, 0, sizeof(float) * kNumParams)) != cudaSuccess ||
        (e = cudaMemset(m->d_m2, 0, sizeof(float) * kNumParams)) != cudaSuccess)
        return fail(mfail(e, "init"));
    *out = m;
    return LBM_OK;
}

extern "C" int lbm_surrogate_set_params(lbm_surrogate* m, const float* params) {
    if (!m || !params) return LBM_ERR_ARG;
    MCK(cudaMemcpy(m->d_params, params, sizeof(float) * kNumParams, cudaMemcpyHostToDevice));
    return LBM_OK;
}

extern "C" int lbm_surrogate_get_params(lbm_surrogate* m, float* params) {
    if (!m || !params) return LBM_ERR_ARG;
    MCK(cudaStreamSynchronize(m->stream));
    MCK(cudaMemcpy(params, m->d_params, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost));
    return LBM_OK;
}

extern "C" int lbm_surrogate_loss_grad(lbm_surrogate* m, const float* X, const float* Y, int n, float* loss,
                                       float* grad) {
    if (!m || !X || !Y || n < 1) return LBM_ERR_ARG;
    const long long nv = valid_targets(Y, n);
    if (nv < 1) return LBM_ERR_ARG;
    int rc = upload_inputs(m, X, Y, n);
    if (!rc) rc = forward(m, n);
    if (!rc) rc = backward(m, n, nv);
    if (rc) return rc;
    if (loss) MCK(cudaMemcpyAsync(loss, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    if (grad) MCK(cudaMemcpyAsync(grad, m->d_grad, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost, m->stream));
    MCK(cudaStreamSynchronize(m->stream));
    return LBM_OK;
}

extern "C" int lbm_surrogate_train(lbm_surrogate* m, const float* X, const float* Y, int n,
                                   const lbm_train_cfg* cfg, float* final_loss) {
    if (!m || !X || !Y || n < 1 || !cfg || cfg->iterations < 0 || !(cfg->lr > 0)) return LBM_ERR_ARG;
    const long long nv = valid_targets(Y, n);
    if (nv < 1) return LBM_ERR_ARG;
    int rc = upload_inputs(m, X, Y, n);
    if (rc) return rc;
    // one iteration = full-batch forward, backward and Adam update; captured once as a graph
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    MCK(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
    rc = forward(m, n);
    if (!rc) rc = backward(m, n, nv);
    cudaError_t e = cudaStreamEndCapture(m->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return mfail(e, "capture(train)");
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return mfail(e, "instantiate(train)");
    for (int it = 0; it < cfg->iterations; ++it) {
        e = cudaGraphLaunch(ge, m->stream);
        if (e != cudaSuccess) break;
        const int t = ++m->steps_done;
        // cosine learning-rate decay to lr_min over the run
        const float frac = cfg->iterations > 1 ? (float)it / (float)(cfg->iterations - 1) : 0.0f;
        const float lr = cfg->lr_min + 0.5f * (cfg->lr - cfg->lr_min) * (1.0f + std::cos(3.14159265f * frac));
        const float c1 = 1.0f - std::pow(cfg->beta1, (float)t), c2 = 1.0f - std::pow(cfg->beta2, (float)t);
        adam_kernel<<<64, 256, 0, m->stream>>>(m->d_params, m->d_grad, m->d_m1, m->d_m2, kNumParams, lr, cfg->beta1,
                                               cfg->beta2, cfg->eps, c1, c2, cfg->weight_decay);
    }
    cudaGraphExecDestroy(ge);
    if (e != cudaSuccess) return mfail(e, "train launch");
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(&m->last_loss, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    MCK(cudaStreamSynchronize(m->stream));
    if (final_loss) *final_loss = m->last_loss;
    return std::isfinite(m->last_loss) ? LBM_OK : LBM_ERR_DIVERGED;
}

extern "C" int lbm_surrogate_predict_fp32(lbm_surrogate* m, const float* X, int n, float* Y) {
    if (!m || !X || !Y || n < 1) return LBM_ERR_ARG;
    int rc = upload_inputs(m, X, nullptr, n);
    if (!rc) rc = forward(m, n);
    if (rc) return rc;
    destandardise_kernel<<<64, 256, 0, m->stream>>>(m->d_Z[kLayers - 1], n, m->d_stats, m->d_out);
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(Y, m->d_out, sizeof(float) * n * kOut, cudaMemcpyDeviceToHost, m->stream));
    MCK(cudaStreamSynchronize(m->stream));
    return LBM_OK;
}

extern "C" int lbm_surrogate_predict_device(lbm_surrogate* m, const float* X_dev, int n, float* Y_dev, int mode,
                                            void* stream) {
    if (!m || !X_dev || !Y_dev || n < 1 || (mode != LBM_INFER_SPLIT_BF16 && mode != LBM_INFER_BF16)) return LBM_ERR_ARG;
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : m->stream;
    pack_weights_kernel<<<64, 256, 0, s>>>(m->d_params, m->d_wpack, m->d_bpack);
    const int smem = (int)sizeof(InferSmem);
    const int grid = (n + kQ - 1) / kQ;
    if (mode == LBM_INFER_SPLIT_BF16) {
        MCK(cudaFuncSetAttribute(mlp_infer_bf16_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        mlp_infer_bf16_kernel<true><<<grid, 128, smem, s>>>(X_dev, n, m->d_wpack, m->d_bpack, m->d_stats, Y_dev);
    } else {
        MCK(cudaFuncSetAttribute(mlp_infer_bf16_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        mlp_infer_bf16_kernel<false><<<grid, 128, smem, s>>>(X_dev, n, m->d_wpack, m->d_bpack, m->d_stats, Y_dev);
    }
    MCK(cudaGetLastError());
    return LBM_OK;
}

extern "C" int lbm_surrogate_predict(lbm_surrogate* m, const float* X, int n, float* Y, int mode) {
    if (!m || !X || !Y || n < 1) return LBM_ERR_ARG;
    int rc = alloc_rows(m, n);
    if (rc) return rc;
    MCK(cudaMemcpyAsync(m->d_X, X, sizeof(float) * n * kIn, cudaMemcpyHostToDevice, m->stream));
    rc = lbm_surrogate_predict_device(m, m->d_X, n, m->d_out, mode, m->stream);
    if (rc) return rc;
    MCK(cudaMemcpyAsync(Y, m->d_out, sizeof(float) * n * kOut, cudaMemcpyDeviceToHost, m->stream));
    MCK(cudaStreamSynchronize(m->stream));
    return LBM_OK;
}

extern "C" int lbm_surrogate_stats(const lbm_surrogate* m, float* stats16) {
    if (!m || !stats16) return LBM_ERR_ARG;
    std::memcpy(stats16, m->h_stats, sizeof(m->h_stats));
    return LBM_OK;
}
