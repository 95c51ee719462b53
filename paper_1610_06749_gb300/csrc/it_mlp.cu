// it_mlp.cu -- the surrogate network for the collection efficiency f.
//
// A 6 -> 256 -> 256 -> 256 -> 256 -> 1 perceptron with SiLU hidden layers
// and a sigmoid output, an ensemble of independent members trained on
// solver results.  Weights are stored in bfloat16 for the matrix products
// (FP32 master copies for Adam), all products accumulate in FP32 on the
// tensor cores, bias, SiLU and its derivative are fused into the product
// epilogues, and the output layer, sigmoid, squared error and the first
// backward step are one fused kernel.  Every reduction runs in a fixed order
// (bitwise-reproducible training).
//
// Precision: weights enter the products as bf16; each layer's input enters
// as a two-term bf16 expansion hi + lo (hi = bf16(a), lo = bf16(a - hi),
// about 16 significant bits) against the weights duplicated along K, so the
// forward pass carries bf16 weights but near-FP32 activations.  A
// one-term bf16 activation added rounding noise of ~2e-4 to f on held-out
// configurations (median; FP64 activations with the same weights: ~1e-4).
// Error signals and the activations of the weight gradients stay one-term
// bf16.
//
// The 256 x 256 products (forward of layers 2-4, their data gradients and
// weight gradients) run on the 5th-generation tensor cores (it_tc.cuh:
// TMA-staged bf16 tiles, tcgen05.mma into tensor memory, fused epilogues).
// Both operands are K-major, so the data gradient reads transposed weight
// copies and the weight gradient reads transposed activations and error
// signals, which the producing epilogues write beside the row-major ones.
// The first layer (6 inputs) and its weight gradient are too narrow for
// them and stay on mma.sync tiles.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "it_device.cuh"
#include "it_internal.cuh"
#include "it_tc.cuh"

namespace itk {
namespace mlp {

constexpr int H = IT_MLP_HIDDEN;
constexpr int NIN = IT_MLP_INPUTS;
// parameter offsets inside one member (W stored out x in)
constexpr long long OW1 = 0, OB1 = OW1 + (long long)H * NIN, OW2 = OB1 + H, OB2 = OW2 + (long long)H * H,
                    OW3 = OB2 + H, OB3 = OW3 + (long long)H * H, OW4 = OB3 + H, OB4 = OW4 + (long long)H * H,
                    OW5 = OB4 + H, OB5 = OW5 + H, P = OB5 + 1;
static_assert(P == IT_MLP_PARAMS, "parameter layout");

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

// ---------------------------------------------------------------------------
// C[m][n] = sum_k A(m,k) B(k,n), A(m,k) = A[m*sam + k*sak], B(k,n) =
// B[k*sbk + n*sbn], bf16 operands, FP32 accumulation on the tensor cores.
// 64 x 64 output tile per CTA, 4 warps of 32 x 32, k-steps of 16.
// blockIdx.z selects the ensemble member (pointer strides per member).
// ---------------------------------------------------------------------------
enum { EPI_FWD = 0, EPI_BWD = 1, EPI_WGRAD = 2 };

struct GemmArgs {
    const __nv_bfloat16 *A, *B;
    long long sam, sak, sbk, sbn, za, zb;   // element strides; za, zb: per-member offsets
    int M, N, K;
    // epilogue operands (per-member offsets zc for every one of them)
    const float *bias;     // FWD: [N]
    long long zbias;
    float *Z;              // FWD: out [M][N] pre-activation; BWD: in, previous layer's pre-activation
    __nv_bfloat16 *Act;    // FWD: out bf16 SiLU(Z); BWD: out bf16 dZ
    float *Out;            // BWD: out fp32 dZ; WGRAD: out fp32 [M][N]
    long long ldc, zc;
    __nv_bfloat16 *ActT;   // FWD (optional): out bf16 SiLU(Z) transposed, [N][ldT] per member
    long long ldT, zT;
    long long ldA, zA;     // FWD: row and member stride of Act (hi at n, lo at n + H)
};

constexpr int BM = 64, BN = 64, BK = 16, LDS = 24;   // LDS: padded smem row (bf16), conflict-free fragments

template <int EPI>
__global__ void __launch_bounds__(128) gemm_bf16_kernel(const GemmArgs g) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][LDS];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][LDS];   // [n][k]
    const int z = blockIdx.z;
    const __nv_bfloat16 *A = g.A + z * g.za, *B = g.B + z * g.zb;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int grp = lane >> 2, tig = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < g.K; k0 += BK) {
        // 1024 elements of each tile, 8 per thread
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = tid + q * 128;
            const int r = e / BK, kk = e % BK;
            const int gm = m0 + r, gn = n0 + r, gk = k0 + kk;
            As[r][kk] = (gm < g.M && gk < g.K) ? A[gm * g.sam + gk * g.sak] : zero;
            Bs[r][kk] = (gn < g.N && gk < g.K) ? B[gk * g.sbk + gn * g.sbn] : zero;
        }
        __syncthreads();
        uint32_t af[2][4], bfr[4][2];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int r = wm + a * 16 + grp;
            af[a][0] = *reinterpret_cast<const uint32_t *>(&As[r][2 * tig]);
            af[a][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][2 * tig]);
            af[a][2] = *reinterpret_cast<const uint32_t *>(&As[r][2 * tig + 8]);
            af[a][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][2 * tig + 8]);
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int c = wn + b * 8 + grp;
            bfr[b][0] = *reinterpret_cast<const uint32_t *>(&Bs[c][2 * tig]);
            bfr[b][1] = *reinterpret_cast<const uint32_t *>(&Bs[c][2 * tig + 8]);
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                    "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
                    : "+f"(acc[a][b][0]), "+f"(acc[a][b][1]), "+f"(acc[a][b][2]), "+f"(acc[a][b][3])
                    : "r"(af[a][0]), "r"(af[a][1]), "r"(af[a][2]), "r"(af[a][3]), "r"(bfr[b][0]), "r"(bfr[b][1]));
        __syncthreads();
    }
    // epilogue: element (row, col) of fragment c: row = grp (+8 for c >= 2), col = 2 tig + (c & 1)
    const long long zc = z * g.zc;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int m = m0 + wm + a * 16 + grp + (c >= 2 ? 8 : 0);
                const int n = n0 + wn + b * 8 + 2 * tig + (c & 1);
                if (m >= g.M || n >= g.N) continue;
                const long long o = zc + (long long)m * g.ldc + n;
                const float v = acc[a][b][c];
                if (EPI == EPI_FWD) {
                    const float zz = v + g.bias[z * g.zbias + n];
                    g.Z[o] = zz;
                    const float s = silu(zz);
                    const __nv_bfloat16 a = __float2bfloat16_rn(s);
                    const long long oa = z * g.zA + (long long)m * g.ldA + n;
                    g.Act[oa] = a;
                    g.Act[oa + H] = __float2bfloat16_rn(s - __bfloat162float(a));
                    if (g.ActT) g.ActT[z * g.zT + (long long)n * g.ldT + m] = a;
                } else if (EPI == EPI_BWD) {
                    const float dz = v * dsilu(g.Z[o]);
                    g.Out[o] = dz;
                    g.Act[o] = __float2bfloat16_rn(dz);
                } else {
                    g.Out[o] = v;
                }
            }
}

// Output layer, sigmoid, squared error and the first backward step, one warp
// per (sample, member): z = A4 . w5 + b5, fhat = sigmoid(z); when training,
// dz = 2/B (fhat - y) fhat (1 - fhat), dZ4 = dz w5 * SiLU'(Z4) (fp32 and bf16).
__global__ void out_layer_kernel(const __nv_bfloat16 *__restrict__ A4, const float *__restrict__ Z4,
                                 const __nv_bfloat16 *__restrict__ w, const float *__restrict__ master,
                                 const float *__restrict__ y, long long ybs, int B, int train, float *__restrict__ fhat,
                                 float *__restrict__ dzout, float *__restrict__ dZ, __nv_bfloat16 *__restrict__ dZb,
                                 long long zact, __nv_bfloat16 *__restrict__ dZbT, long long zT, long long ldT,
                                 long long zA) {
    const int m = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int z = blockIdx.y, lane = threadIdx.x & 31;
    if (m >= B) return;
    const __nv_bfloat16 *w5 = w + z * P + OW5;
    const __nv_bfloat16 *a = A4 + z * zA + (long long)m * 2 * H;   // hi | lo
    float s = 0.f;
    for (int k = lane; k < H; k += 32)
        s += (__bfloat162float(a[k]) + __bfloat162float(a[k + H])) * __bfloat162float(w5[k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float zz = s + master[z * P + OB5];
    const float f = 1.f / (1.f + __expf(-zz));
    if (lane == 0) fhat[z * B + m] = f;
    if (!train) return;
    const float dz = 2.f / B * (f - y[(long long)z * ybs + m]) * f * (1.f - f);
    if (lane == 0) dzout[z * B + m] = dz;
    for (int k = lane; k < H; k += 32) {
        const long long o = z * zact + (long long)m * H + k;
        const float d = dz * __bfloat162float(w5[k]) * dsilu(Z4[o]);
        dZ[o] = d;
        const __nv_bfloat16 db = __float2bfloat16_rn(d);
        dZb[o] = db;
        dZbT[z * zT + (long long)k * ldT + m] = db;
    }
}

// grad of w5 and b5 (fixed order over the batch): g[k] = sum_m dz[m] A4[m][k]
// (A4 = hi + lo, as in the forward pass).
// Block (x, member), 8 warps: lane c of warp w sums column k = 32 x + c over
// the rows m = w, w + 8, ...; the 8 partial sums are added in warp order.
// Block x = 0 also forms b5's sum (thread t over m = t, t + 256, ..., then
// the 256 partials in thread order).
__global__ void __launch_bounds__(256)
out_grad_kernel(const __nv_bfloat16 *__restrict__ A4, const float *__restrict__ dz, int B, float *__restrict__ grad,
                long long zA) {
    __shared__ float part[8][33];
    __shared__ float bpart[256];
    const int z = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = blockIdx.x * 32 + lane;
    const __nv_bfloat16 *a = A4 + z * zA;   // rows of hi | lo
    const float *d = dz + (long long)z * B;
    float s = 0.f;
    for (int m = warp; m < B; m += 8)
        s += d[m] * (__bfloat162float(a[(long long)m * 2 * H + k]) + __bfloat162float(a[(long long)m * 2 * H + H + k]));
    part[warp][lane] = s;
    if (blockIdx.x == 0) {
        float t = 0.f;
        for (int m = threadIdx.x; m < B; m += 256) t += d[m];
        bpart[threadIdx.x] = t;
    }
    __syncthreads();
    if (warp == 0) {
        float g = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) g += part[w][lane];
        grad[z * P + OW5 + k] = g;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        float t = 0.f;
        for (int q = 0; q < 256; ++q) t += bpart[q];
        grad[z * P + OB5] = t;
    }
}

// bias gradient: column sums of dZ [B][H], fixed order.  Block (x, member),
// 8 warps: lane c of warp w sums column n = 32 x + c over the rows m = w,
// w + 8, ...; the 8 partial sums are added in warp order.
__global__ void __launch_bounds__(256)
bias_grad_kernel(const float *__restrict__ dZ, int B, float *__restrict__ grad, long long off, long long zact) {
    __shared__ float part[8][33];
    const int z = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = blockIdx.x * 32 + lane;
    const float *d = dZ + z * zact;
    float s = 0.f;
    for (int m = warp; m < B; m += 8) s += d[(long long)m * H + n];
    part[warp][lane] = s;
    __syncthreads();
    if (warp == 0) {
        float g = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) g += part[w][lane];
        grad[z * P + off + n] = g;
    }
}

// mean squared error per member, fixed order
__global__ void loss_kernel(const float *__restrict__ fhat, const float *__restrict__ y, long long ybs, int B,
                            double *__restrict__ loss, int accumulate) {
    __shared__ double red[32];
    const int z = blockIdx.x;
    double v[1] = {0.0};
    for (int m = threadIdx.x; m < B; m += blockDim.x) {
        const double d = (double)fhat[z * B + m] - (double)y[(long long)z * ybs + m];
        v[0] += d * d;
    }
    block_sum<1>(v, red);
    if (threadIdx.x == 0) loss[z] = (accumulate ? loss[z] : 0.0) + v[0] / B;
}

// Adam (Kingma & Ba) on the FP32 master weights, refreshing the bf16 copies
__global__ void adam_kernel(float *__restrict__ master, __nv_bfloat16 *__restrict__ w, const float *__restrict__ g,
                            float *__restrict__ m1, float *__restrict__ m2, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.f - b1) * gi;
        const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = b;
        const float p = master[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
        master[i] = p;
        w[i] = __float2bfloat16_rn(p);
    }
}

__global__ void to_bf16_kernel(const float *__restrict__ x, __nv_bfloat16 *__restrict__ y, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// normalised bf16 inputs of a batch for every member:
// A0[z][m][j] = hi and A0[z][m][6 + j] = lo of (x[idx[z][m]][j] - mean[j]) / std[j], yb[z][m] = y[idx[z][m]]
// (idx == NULL: sample m for every member)
// Epilogues of the tensor-core products (it_tc.cuh), called by a whole warp
// for its 32 x 32 block: lane holds row mw + lane, columns n0 .. n0+31, in
// the same operation order as the mma.sync epilogues.  Transposed copies go
// through the warp's shared-memory scratch so that each lane then writes 64
// contiguous bytes of one transposed row.

// transpose the warp's 32 x 32 bf16 block a (lane = row m) into
// dst[(n0 + c) * ld + mw + r] for rows mw + r < M
__device__ __forceinline__ void store_transposed(const __nv_bfloat16 (&a)[32], int lane, int mw, int M,
                                                 __nv_bfloat16 *dst, long long ld, float *scratch) {
    __nv_bfloat16 *t = reinterpret_cast<__nv_bfloat16 *>(scratch);   // [32 columns][40]
#pragma unroll
    for (int q = 0; q < 32; ++q) t[q * 40 + lane] = a[q];
    __syncwarp();
    __nv_bfloat16 *d = dst + (long long)lane * ld + mw;
    const __nv_bfloat16 *src = t + lane * 40;
    if (mw + 32 <= M) {
#pragma unroll
        for (int j = 0; j < 4; ++j) reinterpret_cast<uint4 *>(d)[j] = reinterpret_cast<const uint4 *>(src)[j];
    } else {
        for (int r = 0; r < M - mw; ++r) d[r] = src[r];
    }
    __syncwarp();
}

// forward: Z = D + bias, Act = bf16(SiLU(Z)), and optionally Act transposed
struct TcFwd {
    const float *bias;
    long long zbias;
    float *Z;
    long long zact;
    __nv_bfloat16 *Act;   // [member][row][hi 0..H-1 | lo H..2H-1]
    long long zA;
    __nv_bfloat16 *ActT;
    long long zT, ldT;
    __device__ __forceinline__ void operator()(int z, int mw, int lane, int M, int n0, const float (&v)[32],
                                               float *scratch) const {
        const int m = mw + lane;
        const long long o = z * zact + (long long)m * H + n0;
        const long long oa = z * zA + (long long)m * 2 * H + n0;
        const float *bb = bias + z * zbias + n0;
        float zz[32];
        __nv_bfloat16 a[32], lo[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            zz[q] = v[q] + bb[q];
            const float sq = silu(zz[q]);
            a[q] = __float2bfloat16_rn(sq);
            lo[q] = __float2bfloat16_rn(sq - __bfloat162float(a[q]));
        }
        if (m < M) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                reinterpret_cast<float4 *>(Z + o)[j] = make_float4(zz[4 * j], zz[4 * j + 1], zz[4 * j + 2], zz[4 * j + 3]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                reinterpret_cast<uint4 *>(Act + oa)[j] = reinterpret_cast<const uint4 *>(a)[j];
                reinterpret_cast<uint4 *>(Act + oa + H)[j] = reinterpret_cast<const uint4 *>(lo)[j];
            }
        }
        if (ActT) store_transposed(a, lane, mw, M, ActT + z * zT + (long long)n0 * ldT, ldT, scratch);
    }
};

// data gradient: dZ = D * SiLU'(Z of the layer below), as fp32, bf16 and
// bf16 transposed
struct TcBwd {
    const float *Zp;
    float *dZ;
    __nv_bfloat16 *dZb;
    long long zact;
    __nv_bfloat16 *dZbT;
    long long zT, ldT;
    __device__ __forceinline__ void operator()(int z, int mw, int lane, int M, int n0, const float (&v)[32],
                                               float *scratch) const {
        const int m = mw + lane;
        const long long o = z * zact + (long long)(m < M ? m : mw) * H + n0;
        float d[32];
        __nv_bfloat16 db[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            d[q] = v[q] * dsilu(Zp[o + q]);
            db[q] = __float2bfloat16_rn(d[q]);
        }
        if (m < M) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                reinterpret_cast<float4 *>(dZ + o)[j] = make_float4(d[4 * j], d[4 * j + 1], d[4 * j + 2], d[4 * j + 3]);
#pragma unroll
            for (int j = 0; j < 4; ++j) reinterpret_cast<uint4 *>(dZb + o)[j] = reinterpret_cast<const uint4 *>(db)[j];
        }
        store_transposed(db, lane, mw, M, dZbT + z * zT + (long long)n0 * ldT, ldT, scratch);
    }
};

// weight gradient [out][in] into the member's gradient vector: the block is
// reordered so that each store writes 32 consecutive floats of one row
struct TcWgrad {
    float *grad;
    long long off;
    __device__ __forceinline__ void operator()(int z, int mw, int lane, int M, int n0, const float (&v)[32],
                                               float *scratch) const {
#pragma unroll
        for (int q = 0; q < 32; ++q) scratch[lane * 33 + q] = v[q];
        __syncwarp();
        float *g = grad + z * P + off + (long long)mw * H + n0 + lane;
        for (int r = 0; r < 32 && mw + r < M; ++r) g[(long long)r * H] = scratch[r * 33 + lane];
        __syncwarp();
    }
};

// bf16 copies of the weights for the products: W2..W4 as [member][layer][out]
// [W | W] along K (the forward's A operand is [hi | lo]) and transposed as
// [member][layer][in][out] (data gradient), by 32 x 32 tiles through shared
// memory so that every write is coalesced; W1 as [member][out][W1 | W1].
// Grid (H/32, 3 H/32 + 1, members), block (32, 8): the extra row of blocks
// packs W1.
__global__ void __launch_bounds__(256)
pack_w_kernel(const __nv_bfloat16 *__restrict__ w, __nv_bfloat16 *__restrict__ wt, __nv_bfloat16 *__restrict__ wtt,
              __nv_bfloat16 *__restrict__ w1d) {
    __shared__ __nv_bfloat16 tile[32][34];
    const int z = blockIdx.z;
    if (blockIdx.y == 3 * (H / 32)) {
        const int tid = threadIdx.y * 32 + threadIdx.x;
        for (int e = blockIdx.x * 256 + tid; e < H * NIN; e += (H / 32) * 256) {
            const int o = e / NIN, i = e - o * NIN;
            const __nv_bfloat16 v = w[z * P + OW1 + e];
            w1d[((long long)z * H + o) * 2 * NIN + i] = v;
            w1d[((long long)z * H + o) * 2 * NIN + NIN + i] = v;
        }
        return;
    }
    const int l = blockIdx.y / (H / 32), to = blockIdx.y % (H / 32), ti = blockIdx.x;
    const __nv_bfloat16 *src = w + z * P + OW2 + (long long)l * (H * H + H);
    const long long blk = ((long long)z * 3 + l) * H * H;
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int o = to * 32 + j, i = ti * 32 + threadIdx.x;
        const __nv_bfloat16 v = src[o * H + i];
        tile[j][threadIdx.x] = v;
        wt[2 * blk + (long long)o * 2 * H + i] = v;
        wt[2 * blk + (long long)o * 2 * H + H + i] = v;
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int i = ti * 32 + j, o = to * 32 + threadIdx.x;
        wtt[blk + i * H + o] = tile[threadIdx.x][j];
    }
}

__global__ void gather_inputs_kernel(const float *__restrict__ X, const float *__restrict__ Y,
                                     const int *__restrict__ idx, long long istride, int B, int members, int bmax,
                                     const float *__restrict__ mean, const float *__restrict__ inv_std,
                                     __nv_bfloat16 *__restrict__ A0, float *__restrict__ yb) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)members * B * NIN) return;
    const int z = (int)(e / ((long long)B * NIN));
    const int r0 = (int)(e - (long long)z * B * NIN);
    const int m = r0 / NIN, j = r0 % NIN;
    const int r = idx ? idx[z * istride + m] : m;
    const float x = (X[(long long)r * NIN + j] - mean[j]) * inv_std[j];
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    A0[((long long)z * bmax + m) * 2 * NIN + j] = hi;
    A0[((long long)z * bmax + m) * 2 * NIN + NIN + j] = __float2bfloat16_rn(x - __bfloat162float(hi));
    if (j == 0 && Y) yb[z * bmax + m] = Y[r];
}

}  // namespace mlp
}  // namespace itk

using namespace itk;
using namespace itk::mlp;

struct it_mlp {
    int members, bmax;
    float *master, *grad, *m1, *m2;
    __nv_bfloat16 *w;
    long long adam_t;
    float *mean, *inv_std;        // device [6]
    double h_mean[NIN], h_std[NIN];
    // batch workspace (per member strides zact = bmax * H)
    __nv_bfloat16 *A0;            // [member][bmax][hi 6 | lo 6]
    float *Z[4];
    __nv_bfloat16 *Act[4];        // [member][bmax][hi 256 | lo 256]
    float *dZ[2];
    __nv_bfloat16 *dZb[2];
    float *fhat, *dz, *yb;
    int *idx;
    double *loss;
    // tensor-core operands: W2..W4 as [member][layer][out][in] and
    // [member][layer][in][out], A1..A3 transposed and the bf16 error signal
    // transposed, [member][256][bpad] (bpad: max_batch rounded up to 64)
    __nv_bfloat16 *wt, *wtt, *actT[3], *dzbT[2];
    __nv_bfloat16 *w1d;           // [member][256][W1 | W1] for the layer-1 product with [hi | lo] inputs
    long long bpad;
    int *d_err;                   // a bounded wait of the tensor-core kernel ran out
    int *eidx;                    // [members][n_data]: every member's sample order of one epoch
    long long eidx_cap;
    double *eloss;                // [members]: the epoch's summed batch losses
    // training set
    float *X, *Y;
    long long n_data;
    cudaStream_t stream;
};

namespace {

int mfail(int code, const std::string &m) {
    set_error(m);
    return code;
}

void mlp_free(it_mlp *n) {
    if (!n) return;
    if (n->stream) cudaStreamSynchronize(n->stream);
    cudaFree(n->master); cudaFree(n->grad); cudaFree(n->m1); cudaFree(n->m2); cudaFree(n->w);
    cudaFree(n->mean); cudaFree(n->inv_std); cudaFree(n->A0);
    for (int l = 0; l < 4; ++l) { cudaFree(n->Z[l]); cudaFree(n->Act[l]); }
    for (int q = 0; q < 2; ++q) { cudaFree(n->dZ[q]); cudaFree(n->dZb[q]); }
    cudaFree(n->fhat); cudaFree(n->dz); cudaFree(n->yb); cudaFree(n->idx); cudaFree(n->loss);
    cudaFree(n->eidx); cudaFree(n->eloss);
    cudaFree(n->wt); cudaFree(n->wtt); cudaFree(n->w1d); cudaFree(n->d_err);
    for (int q = 0; q < 3; ++q) cudaFree(n->actT[q]);
    for (int q = 0; q < 2; ++q) cudaFree(n->dzbT[q]);
    cudaFree(n->X); cudaFree(n->Y);
    if (n->stream) cudaStreamDestroy(n->stream);
    delete n;
}

int launch_gemm(int epi, const GemmArgs &g, int members, cudaStream_t s) {
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, members);
    if (epi == EPI_FWD) gemm_bf16_kernel<EPI_FWD><<<grid, 128, 0, s>>>(g);
    else if (epi == EPI_BWD) gemm_bf16_kernel<EPI_BWD><<<grid, 128, 0, s>>>(g);
    else gemm_bf16_kernel<EPI_WGRAD><<<grid, 128, 0, s>>>(g);
    IT_CK(cudaGetLastError());
    return IT_OK;
}

const long long kOffW[4] = {OW1, OW2, OW3, OW4};
const long long kOffB[4] = {OB1, OB2, OB3, OB4};

// D = A B^T on the tensor cores for every member: A [members][M rows][K],
// B [members][N rows][K] (bf16, K contiguous, byte strides of a row and of a
// member), N a multiple of 128
template <class Epi>
int launch_tc(it_mlp *n, const void *A, long long a_row, long long a_mem, const void *Bm, long long b_row,
              long long b_mem, int M, int N, int K, const Epi &epi) {
    CUtensorMap ta, tb;
    int rc = encode_bf16_sw128(&ta, A, K, M, n->members, a_row, a_mem);
    if (!rc) rc = encode_bf16_sw128(&tb, Bm, K, N, n->members, b_row, b_mem);
    if (rc) return rc;
    dim3 grid(N / tc::TN, (M + tc::TM - 1) / tc::TM, n->members);
    tc::tc_gemm_kernel<Epi><<<grid, 128, tc::SMEM_BYTES, n->stream>>>(ta, tb, M, N, K, epi, n->d_err);
    IT_CK(cudaGetLastError());
    return IT_OK;
}

// forward of B samples already in A0 (and yb when training)
int forward(it_mlp *n, int B, bool train) {
    const long long zact = (long long)n->bmax * H, zA = 2 * zact, zT = (long long)H * n->bpad;
    // layer 1 (6 inputs as hi | lo against W1 | W1): mma.sync tiles, also
    // writing A1 transposed
    {
        GemmArgs g{};
        g.A = n->A0; g.sam = 2 * NIN; g.sak = 1; g.za = (long long)n->bmax * 2 * NIN;
        g.B = n->w1d; g.sbk = 1; g.sbn = 2 * NIN; g.zb = (long long)H * 2 * NIN;
        g.M = B; g.N = H; g.K = 2 * NIN;
        g.bias = n->master + kOffB[0]; g.zbias = P;
        g.Z = n->Z[0]; g.Act = n->Act[0];
        g.ldc = H; g.zc = zact;
        g.ldA = 2 * H; g.zA = zA;
        g.ActT = n->actT[0]; g.ldT = n->bpad; g.zT = zT;
        int rc = launch_gemm(EPI_FWD, g, n->members, n->stream);
        if (rc) return rc;
    }
    // layers 2-4 on the tensor cores: [hi | lo] (K = 512) against [W | W]
    for (int l = 1; l < 4; ++l) {
        TcFwd e{n->master + kOffB[l], P, n->Z[l], zact, n->Act[l], zA, l < 3 ? n->actT[l] : nullptr, zT, n->bpad};
        int rc = launch_tc(n, n->Act[l - 1], 4LL * H, 2LL * zA, n->wt + (long long)(l - 1) * H * 2 * H, 4LL * H,
                           2LL * 3 * H * 2 * H, B, H, 2 * H, e);
        if (rc) return rc;
    }
    dim3 grid((B + 7) / 8, n->members);
    out_layer_kernel<<<grid, 256, 0, n->stream>>>(n->Act[3], n->Z[3], n->w, n->master, n->yb, n->bmax, B, train ? 1 : 0,
                                                  n->fhat, n->dz, n->dZ[0], n->dZb[0], zact, n->dzbT[0], zT, n->bpad,
                                                  zA);
    IT_CK(cudaGetLastError());
    return IT_OK;
}

// backward of the batch into n->grad (after forward(train = true))
int backward(it_mlp *n, int B) {
    const long long zact = (long long)n->bmax * H, zA = 2 * zact, zT = (long long)H * n->bpad;
    out_grad_kernel<<<dim3(H / 32, n->members), 256, 0, n->stream>>>(n->Act[3], n->dz, B, n->grad, zA);
    IT_CK(cudaGetLastError());
    int cur = 0;
    for (int l = 3; l >= 1; --l) {
        // weight gradient gW[o][i] = sum_m dZ[m][o] A_{l-1}[m][i] (bf16 hi part of
        // the activation): the K = batch axis is contiguous in the transposed copies
        TcWgrad w{n->grad, kOffW[l]};
        int rc = launch_tc(n, n->dzbT[cur], 2LL * n->bpad, 2LL * zT, n->actT[l - 1], 2LL * n->bpad, 2LL * zT, H, H, B,
                           w);
        if (rc) return rc;
        bias_grad_kernel<<<dim3(H / 32, n->members), 256, 0, n->stream>>>(n->dZ[cur], B, n->grad, kOffB[l], zact);
        IT_CK(cudaGetLastError());
        // data gradient into the layer below: dZ_{l-1} = (dZ_l W_l) * SiLU'(Z_{l-1})
        TcBwd d{n->Z[l - 1], n->dZ[cur ^ 1], n->dZb[cur ^ 1], zact, n->dzbT[cur ^ 1], zT, n->bpad};
        rc = launch_tc(n, n->dZb[cur], 2LL * H, 2LL * zact, n->wtt + (long long)(l - 1) * H * H, 2LL * H,
                       2LL * 3 * H * H, B, H, H, d);
        if (rc) return rc;
        cur ^= 1;
    }
    // layer 1: mma.sync weight gradient (6 inputs, their bf16 hi part)
    GemmArgs g{};
    g.A = n->dZb[cur]; g.sam = 1; g.sak = H; g.za = zact;
    g.B = n->A0; g.sbk = 2 * NIN; g.sbn = 1; g.zb = (long long)n->bmax * 2 * NIN;
    g.M = H; g.N = NIN; g.K = B;
    g.Out = n->grad + kOffW[0]; g.ldc = NIN; g.zc = P;
    int rc = launch_gemm(EPI_WGRAD, g, n->members, n->stream);
    if (rc) return rc;
    bias_grad_kernel<<<dim3(H / 32, n->members), 256, 0, n->stream>>>(n->dZ[cur], B, n->grad, kOffB[0], zact);
    IT_CK(cudaGetLastError());
    return IT_OK;
}

// the bf16 tensor-core copies of W2..W4 after the bf16 weights changed
int pack_weights(it_mlp *n) {
    pack_w_kernel<<<dim3(H / 32, 3 * (H / 32) + 1, n->members), dim3(32, 8), 0, n->stream>>>(n->w, n->wt, n->wtt,
                                                                                               n->w1d);
    IT_CK(cudaGetLastError());
    return IT_OK;
}

// IT_ETIMEOUT if a bounded wait of the tensor-core kernel ran out (the flag
// is cleared)
int check_device_error(it_mlp *n) {
    int err = 0;
    IT_CK(cudaMemcpyAsync(&err, n->d_err, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
    IT_CK(cudaStreamSynchronize(n->stream));
    if (err) {
        IT_CK(cudaMemsetAsync(n->d_err, 0, sizeof(int), n->stream));
        return mfail(IT_ETIMEOUT, "a bounded wait of the tensor-core GEMM ran out");
    }
    return IT_OK;
}

int upload_inputs(it_mlp *n, long long count, const double *x, const double *y, float **dX, float **dY) {
    std::vector<float> hx((size_t)count * NIN), hy(y ? (size_t)count : 0);
    for (long long i = 0; i < count * NIN; ++i) hx[i] = (float)x[i];
    for (long long i = 0; y && i < count; ++i) hy[i] = (float)y[i];
    IT_CK(cudaMalloc(dX, sizeof(float) * hx.size()));
    IT_CK(cudaMemcpyAsync(*dX, hx.data(), sizeof(float) * hx.size(), cudaMemcpyHostToDevice, n->stream));
    if (y) {
        IT_CK(cudaMalloc(dY, sizeof(float) * hy.size()));
        IT_CK(cudaMemcpyAsync(*dY, hy.data(), sizeof(float) * hy.size(), cudaMemcpyHostToDevice, n->stream));
    }
    IT_CK(cudaStreamSynchronize(n->stream));
    return IT_OK;
}

// idx: per member the sample rows of the batch, member z's at idx + z istride
int gather(it_mlp *n, const float *X, const float *Y, const int *idx, long long istride, int B) {
    const long long tot = (long long)n->members * B * NIN;
    gather_inputs_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, n->stream>>>(X, Y, idx, istride, B, n->members,
                                                                               n->bmax, n->mean, n->inv_std, n->A0,
                                                                               n->yb);
    IT_CK(cudaGetLastError());
    return IT_OK;
}

int adam_step(it_mlp *n, float lr) {
    n->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)n->adam_t));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)n->adam_t));
    const long long cnt = (long long)n->members * P;
    adam_kernel<<<1024, 256, 0, n->stream>>>(n->master, n->w, n->grad, n->m1, n->m2, cnt, lr, b1, b2, eps, c1, c2);
    IT_CK(cudaGetLastError());
    return pack_weights(n);
}

uint64_t splitmix_next(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int it_mlp_create(int32_t members, int32_t max_batch, it_mlp **out) {
    if (!out) return mfail(IT_EINVAL, "out is NULL");
    *out = nullptr;
    if (members < 1 || members > 64 || max_batch < 1 || max_batch > (1 << 20))
        return mfail(IT_EINVAL, "members must be 1..64 and max_batch 1..2^20");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return mfail(IT_ECUDA, "no CUDA device available");
    it_mlp *n = new (std::nothrow) it_mlp();
    if (!n) return mfail(IT_ENOMEM, "host allocation failed");
    n->members = members;
    n->bmax = max_batch;
    const long long np = (long long)members * P, za = (long long)members * max_batch * H;
    cudaError_t e;
    auto bail = [&](const char *w) { int rc = cuda_fail(e, w); mlp_free(n); return rc; };
    if ((e = cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking)) != cudaSuccess) return bail("stream");
    if ((e = cudaMalloc(&n->master, sizeof(float) * np)) != cudaSuccess ||
        (e = cudaMalloc(&n->grad, sizeof(float) * np)) != cudaSuccess ||
        (e = cudaMalloc(&n->m1, sizeof(float) * np)) != cudaSuccess ||
        (e = cudaMalloc(&n->m2, sizeof(float) * np)) != cudaSuccess ||
        (e = cudaMalloc(&n->w, sizeof(__nv_bfloat16) * np)) != cudaSuccess ||
        (e = cudaMalloc(&n->mean, sizeof(float) * NIN)) != cudaSuccess ||
        (e = cudaMalloc(&n->inv_std, sizeof(float) * NIN)) != cudaSuccess ||
        (e = cudaMalloc(&n->A0, sizeof(__nv_bfloat16) * members * max_batch * 2 * NIN)) != cudaSuccess ||
        (e = cudaMalloc(&n->fhat, sizeof(float) * members * max_batch)) != cudaSuccess ||
        (e = cudaMalloc(&n->dz, sizeof(float) * members * max_batch)) != cudaSuccess ||
        (e = cudaMalloc(&n->yb, sizeof(float) * members * max_batch)) != cudaSuccess ||
        (e = cudaMalloc(&n->idx, sizeof(int) * members * max_batch)) != cudaSuccess ||
        (e = cudaMalloc(&n->loss, sizeof(double) * members)) != cudaSuccess)
        return bail("mlp allocation");
    n->bpad = ((long long)max_batch + 63) / 64 * 64;
    const long long zw = (long long)members * 3 * H * H, zt = (long long)members * H * n->bpad;
    if ((e = cudaMalloc(&n->wt, sizeof(__nv_bfloat16) * 2 * zw)) != cudaSuccess ||
        (e = cudaMalloc(&n->w1d, sizeof(__nv_bfloat16) * members * H * 2 * NIN)) != cudaSuccess ||
        (e = cudaMalloc(&n->wtt, sizeof(__nv_bfloat16) * zw)) != cudaSuccess ||
        (e = cudaMalloc(&n->d_err, sizeof(int))) != cudaSuccess ||
        (e = cudaMemsetAsync(n->d_err, 0, sizeof(int), n->stream)) != cudaSuccess)
        return bail("mlp tensor-core operands");
    for (int q = 0; q < 3; ++q)
        if ((e = cudaMalloc(&n->actT[q], sizeof(__nv_bfloat16) * zt)) != cudaSuccess) return bail("mlp activations");
    for (int q = 0; q < 2; ++q)
        if ((e = cudaMalloc(&n->dzbT[q], sizeof(__nv_bfloat16) * zt)) != cudaSuccess) return bail("mlp gradients");
    if ((e = cudaFuncSetAttribute(tc::tc_gemm_kernel<TcFwd>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  tc::SMEM_BYTES)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(tc::tc_gemm_kernel<TcBwd>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  tc::SMEM_BYTES)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(tc::tc_gemm_kernel<TcWgrad>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  tc::SMEM_BYTES)) != cudaSuccess)
        return bail("cudaFuncSetAttribute(tensor-core GEMM)");
    for (int l = 0; l < 4; ++l)
        if ((e = cudaMalloc(&n->Z[l], sizeof(float) * za)) != cudaSuccess ||
            (e = cudaMalloc(&n->Act[l], sizeof(__nv_bfloat16) * 2 * za)) != cudaSuccess)
            return bail("mlp activations");
    for (int q = 0; q < 2; ++q)
        if ((e = cudaMalloc(&n->dZ[q], sizeof(float) * za)) != cudaSuccess ||
            (e = cudaMalloc(&n->dZb[q], sizeof(__nv_bfloat16) * za)) != cudaSuccess)
            return bail("mlp gradients");
    if ((e = cudaMemsetAsync(n->master, 0, sizeof(float) * np, n->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(n->w, 0, sizeof(__nv_bfloat16) * np, n->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(n->m1, 0, sizeof(float) * np, n->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(n->m2, 0, sizeof(float) * np, n->stream)) != cudaSuccess)
        return bail("mlp init");
    double mean[NIN] = {0}, sd[NIN] = {1, 1, 1, 1, 1, 1};
    *out = n;
    return it_mlp_set_normalization(n, mean, sd);
}

int it_mlp_set_params(it_mlp *n, int32_t member, const float *params, int64_t count) {
    if (!n || !params || member < 0 || member >= n->members || count != P) return mfail(IT_EINVAL, "bad argument");
    IT_CK(cudaMemcpyAsync(n->master + (long long)member * P, params, sizeof(float) * P, cudaMemcpyHostToDevice, n->stream));
    to_bf16_kernel<<<256, 256, 0, n->stream>>>(n->master + (long long)member * P, n->w + (long long)member * P, P);
    IT_CK(cudaGetLastError());
    if (int rc = pack_weights(n)) return rc;
    // a new starting point: the optimiser state restarts
    IT_CK(cudaMemsetAsync(n->m1 + (long long)member * P, 0, sizeof(float) * P, n->stream));
    IT_CK(cudaMemsetAsync(n->m2 + (long long)member * P, 0, sizeof(float) * P, n->stream));
    n->adam_t = 0;
    IT_CK(cudaStreamSynchronize(n->stream));
    return IT_OK;
}

int it_mlp_get_params(it_mlp *n, int32_t member, float *out, int64_t count) {
    if (!n || !out || member < 0 || member >= n->members || count != P) return mfail(IT_EINVAL, "bad argument");
    IT_CK(cudaMemcpyAsync(out, n->master + (long long)member * P, sizeof(float) * P, cudaMemcpyDeviceToHost, n->stream));
    IT_CK(cudaStreamSynchronize(n->stream));
    return IT_OK;
}

int it_mlp_set_normalization(it_mlp *n, const double *mean6, const double *std6) {
    if (!n || !mean6 || !std6) return mfail(IT_EINVAL, "bad argument");
    float m[NIN], is[NIN];
    for (int j = 0; j < NIN; ++j) {
        if (!(std::isfinite(mean6[j]) && std::isfinite(std6[j]) && std6[j] > 0)) return mfail(IT_EINVAL, "std must be > 0");
        n->h_mean[j] = mean6[j];
        n->h_std[j] = std6[j];
        m[j] = (float)mean6[j];
        is[j] = (float)(1.0 / std6[j]);
    }
    IT_CK(cudaMemcpyAsync(n->mean, m, sizeof(m), cudaMemcpyHostToDevice, n->stream));
    IT_CK(cudaMemcpyAsync(n->inv_std, is, sizeof(is), cudaMemcpyHostToDevice, n->stream));
    IT_CK(cudaStreamSynchronize(n->stream));
    return IT_OK;
}

int it_mlp_fit_normalization(it_mlp *n, int64_t count, const double *x) {
    if (!n || !x || count < 2) return mfail(IT_EINVAL, "need at least 2 samples");
    double mean[NIN] = {0}, sd[NIN] = {0};
    for (int64_t i = 0; i < count; ++i)
        for (int j = 0; j < NIN; ++j) mean[j] += x[i * NIN + j];
    for (int j = 0; j < NIN; ++j) mean[j] /= (double)count;
    for (int64_t i = 0; i < count; ++i)
        for (int j = 0; j < NIN; ++j) sd[j] += (x[i * NIN + j] - mean[j]) * (x[i * NIN + j] - mean[j]);
    for (int j = 0; j < NIN; ++j) {
        sd[j] = std::sqrt(sd[j] / (double)(count - 1));
        if (!(sd[j] > 0)) sd[j] = 1.0;
    }
    return it_mlp_set_normalization(n, mean, sd);
}

int it_mlp_set_data(it_mlp *n, int64_t count, const double *x, const double *y) {
    if (!n || !x || !y || count < 1 || count > 0x7fffffff) return mfail(IT_EINVAL, "bad argument");
    cudaFree(n->X); cudaFree(n->Y);
    n->X = n->Y = nullptr;
    n->n_data = 0;
    int rc = upload_inputs(n, count, x, y, &n->X, &n->Y);
    if (rc) return rc;
    n->n_data = count;
    return IT_OK;
}

int it_mlp_train(it_mlp *n, int32_t epochs, int32_t batch, double lr, uint64_t seed, double *loss_per_epoch) {
    if (!n || epochs < 0 || batch < 1 || batch > n->bmax || !(lr > 0)) return mfail(IT_EINVAL, "bad argument");
    if (n->n_data < 1) return mfail(IT_ESTATE, "no training data (it_mlp_set_data)");
    const long long N = n->n_data;
    const int Z = n->members;
    if (n->eidx_cap < (long long)Z * N) {
        cudaFree(n->eidx);
        n->eidx = nullptr;
        n->eidx_cap = 0;
        IT_CK(cudaMalloc(&n->eidx, sizeof(int) * (size_t)Z * N));
        n->eidx_cap = (long long)Z * N;
    }
    if (!n->eloss) IT_CK(cudaMalloc(&n->eloss, sizeof(double) * Z));
    // each member walks the data in its own order (ensemble diversity); one
    // epoch's orders go to the device at once, and the batches of the epoch
    // are enqueued without host synchronisation
    std::vector<uint64_t> st(Z);
    for (int z = 0; z < Z; ++z) st[z] = seed + 0x9E3779B97F4A7C15ULL * (uint64_t)(z + 1);
    std::vector<int> hidx((size_t)Z * N);
    std::vector<double> lossb(Z);
    for (int ep = 0; ep < epochs; ++ep) {
        for (int z = 0; z < Z; ++z) {
            int *pz = hidx.data() + (size_t)z * N;
            for (long long i = 0; i < N; ++i) pz[i] = (int)i;
            for (long long i = N - 1; i > 0; --i) {   // Fisher-Yates with SplitMix64
                const long long j = (long long)(splitmix_next(st[z]) % (uint64_t)(i + 1));
                std::swap(pz[i], pz[j]);
            }
        }
        // pageable source: the copy is staged before the call returns, so
        // hidx may be refilled for the next epoch right away
        IT_CK(cudaMemcpyAsync(n->eidx, hidx.data(), sizeof(int) * (size_t)Z * N, cudaMemcpyHostToDevice, n->stream));
        int nb = 0;
        for (long long b0 = 0; b0 + batch <= N || (b0 < N && nb == 0); b0 += batch) {
            const int B = (int)std::min<long long>(batch, N - b0);
            int rc = gather(n, n->X, n->Y, n->eidx + b0, N, B);
            if (!rc) rc = forward(n, B, true);
            if (!rc && loss_per_epoch) {
                loss_kernel<<<n->members, 256, 0, n->stream>>>(n->fhat, n->yb, n->bmax, B, n->eloss, nb > 0);
                IT_CK(cudaGetLastError());
            }
            if (!rc) rc = backward(n, B);
            if (!rc) rc = adam_step(n, (float)lr);
            if (rc) return rc;
            ++nb;
        }
        if (loss_per_epoch) {
            IT_CK(cudaMemcpyAsync(lossb.data(), n->eloss, sizeof(double) * Z, cudaMemcpyDeviceToHost, n->stream));
            IT_CK(cudaStreamSynchronize(n->stream));
            double ep_loss = 0.0;
            for (double v : lossb) ep_loss += v / Z;
            loss_per_epoch[ep] = ep_loss / std::max(nb, 1);
        }
    }
    IT_CK(cudaStreamSynchronize(n->stream));
    return check_device_error(n);
}

int it_mlp_loss_grad(it_mlp *n, int64_t count, const double *x, const double *y, float *grads, double *loss) {
    if (!n || !x || !y || count < 1 || count > n->bmax) return mfail(IT_EINVAL, "bad argument");
    float *dX = nullptr, *dY = nullptr;
    int rc = upload_inputs(n, count, x, y, &dX, &dY);
    if (!rc) rc = gather(n, dX, dY, nullptr, 0, (int)count);
    if (!rc) rc = forward(n, (int)count, true);
    if (!rc) {
        loss_kernel<<<n->members, 256, 0, n->stream>>>(n->fhat, n->yb, n->bmax, (int)count, n->loss, 0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "loss");
    }
    if (!rc) rc = backward(n, (int)count);
    if (!rc && grads) {
        cudaError_t e = cudaMemcpyAsync(grads, n->grad, sizeof(float) * n->members * P, cudaMemcpyDeviceToHost, n->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "grad copy");
    }
    if (!rc && loss) {
        cudaError_t e = cudaMemcpyAsync(loss, n->loss, sizeof(double) * n->members, cudaMemcpyDeviceToHost, n->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "loss copy");
    }
    cudaStreamSynchronize(n->stream);
    cudaFree(dX);
    cudaFree(dY);
    if (!rc) rc = check_device_error(n);
    return rc;
}

int it_mlp_adam_step(it_mlp *n, double lr) {
    if (!n || !(lr > 0)) return mfail(IT_EINVAL, "bad argument");
    int rc = adam_step(n, (float)lr);
    if (rc) return rc;
    IT_CK(cudaStreamSynchronize(n->stream));
    return IT_OK;
}

int it_mlp_predict(it_mlp *n, int64_t count, const double *x, double *mean, double *spread, double *per_member) {
    if (!n || !x || count < 0) return mfail(IT_EINVAL, "bad argument");
    if (count == 0) return IT_OK;
    float *dX = nullptr, *dYdummy = nullptr;
    int rc = upload_inputs(n, count, x, nullptr, &dX, &dYdummy);
    if (rc) return rc;
    std::vector<float> f((size_t)n->members * n->bmax);
    for (long long b0 = 0; b0 < count && !rc; b0 += n->bmax) {
        const int B = (int)std::min<long long>(n->bmax, count - b0);
        rc = gather(n, dX + b0 * NIN, nullptr, nullptr, 0, B);
        if (!rc) rc = forward(n, B, false);
        if (rc) break;
        cudaError_t e = cudaMemcpyAsync(f.data(), n->fhat, sizeof(float) * n->members * B, cudaMemcpyDeviceToHost, n->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
        if (e != cudaSuccess) { rc = cuda_fail(e, "predict copy"); break; }
        for (int m = 0; m < B; ++m) {
            double s = 0, lo = 1e300, hi = -1e300;
            for (int z = 0; z < n->members; ++z) {
                const double v = f[(size_t)z * B + m];
                s += v; lo = std::min(lo, v); hi = std::max(hi, v);
                if (per_member) per_member[(b0 + m) * n->members + z] = v;
            }
            if (mean) mean[b0 + m] = s / n->members;
            if (spread) spread[b0 + m] = hi - lo;
        }
    }
    cudaFree(dX);
    if (!rc) rc = check_device_error(n);
    return rc;
}

int it_mlp_destroy(it_mlp *n) {
    mlp_free(n);
    return IT_OK;
}

}  // extern "C"
