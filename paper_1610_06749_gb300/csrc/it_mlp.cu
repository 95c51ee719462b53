// it_mlp.cu -- the surrogate network for the collection efficiency f.
//
// A 6 -> 256 -> 256 -> 256 -> 256 -> 1 perceptron with SiLU hidden layers
// and a sigmoid output, an ensemble of independent members trained on
// solver results.  Weights are stored in bfloat16 for the matrix products
// (FP32 master copies for Adam), all products accumulate in FP32 on the
// tensor cores (mma.sync m16n8k16 bf16), bias, SiLU and its derivative are
// fused into the product epilogues, and the output layer, sigmoid, squared
// error and the first backward step are one fused kernel.  Every reduction
// runs in a fixed order (bitwise-reproducible training).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "it_device.cuh"
#include "it_internal.cuh"

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
                    g.Act[o] = __float2bfloat16_rn(silu(zz));
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
                                 long long zact) {
    const int m = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int z = blockIdx.y, lane = threadIdx.x & 31;
    if (m >= B) return;
    const __nv_bfloat16 *w5 = w + z * P + OW5;
    const __nv_bfloat16 *a = A4 + z * zact + (long long)m * H;
    float s = 0.f;
    for (int k = lane; k < H; k += 32) s += __bfloat162float(a[k]) * __bfloat162float(w5[k]);
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
        dZb[o] = __float2bfloat16_rn(d);
    }
}

// grad of w5 and b5 (fixed order over the batch): g[k] = sum_m dz[m] A4[m][k]
__global__ void out_grad_kernel(const __nv_bfloat16 *__restrict__ A4, const float *__restrict__ dz, int B,
                                float *__restrict__ grad, long long zact) {
    const int z = blockIdx.x, k = threadIdx.x;
    const __nv_bfloat16 *a = A4 + z * zact;
    const float *d = dz + (long long)z * B;
    if (k < H) {
        float s = 0.f;
        for (int m = 0; m < B; ++m) s += d[m] * __bfloat162float(a[(long long)m * H + k]);
        grad[z * P + OW5 + k] = s;
    } else if (k == H) {
        float s = 0.f;
        for (int m = 0; m < B; ++m) s += d[m];
        grad[z * P + OB5] = s;
    }
}

// bias gradient: column sums of dZ [B][H] in batch order
__global__ void bias_grad_kernel(const float *__restrict__ dZ, int B, float *__restrict__ grad, long long off,
                                 long long zact) {
    const int z = blockIdx.x, n = threadIdx.x;
    if (n >= H) return;
    const float *d = dZ + z * zact;
    float s = 0.f;
    for (int m = 0; m < B; ++m) s += d[(long long)m * H + n];
    grad[z * P + off + n] = s;
}

// mean squared error per member, fixed order
__global__ void loss_kernel(const float *__restrict__ fhat, const float *__restrict__ y, long long ybs, int B,
                            double *__restrict__ loss) {
    __shared__ double red[32];
    const int z = blockIdx.x;
    double v[1] = {0.0};
    for (int m = threadIdx.x; m < B; m += blockDim.x) {
        const double d = (double)fhat[z * B + m] - (double)y[(long long)z * ybs + m];
        v[0] += d * d;
    }
    block_sum<1>(v, red);
    if (threadIdx.x == 0) loss[z] = v[0] / B;
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
// A0[z][m][j] = (x[idx[z][m]][j] - mean[j]) / std[j], yb[z][m] = y[idx[z][m]]
// (idx == NULL: sample m for every member)
__global__ void gather_inputs_kernel(const float *__restrict__ X, const float *__restrict__ Y,
                                     const int *__restrict__ idx, int B, int members, int bmax,
                                     const float *__restrict__ mean, const float *__restrict__ inv_std,
                                     __nv_bfloat16 *__restrict__ A0, float *__restrict__ yb) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)members * B * NIN) return;
    const int z = (int)(e / ((long long)B * NIN));
    const int r0 = (int)(e - (long long)z * B * NIN);
    const int m = r0 / NIN, j = r0 % NIN;
    const int r = idx ? idx[z * bmax + m] : m;
    A0[((long long)z * bmax + m) * NIN + j] = __float2bfloat16_rn((X[(long long)r * NIN + j] - mean[j]) * inv_std[j]);
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
    __nv_bfloat16 *A0;            // [bmax][6] shared by the members
    float *Z[4];
    __nv_bfloat16 *Act[4];
    float *dZ[2];
    __nv_bfloat16 *dZb[2];
    float *fhat, *dz, *yb;
    int *idx;
    double *loss;
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

// forward of B samples already in A0 (and yb when training)
int forward(it_mlp *n, int B, bool train) {
    const long long zact = (long long)n->bmax * H;
    for (int l = 0; l < 4; ++l) {
        GemmArgs g{};
        const int K = l == 0 ? NIN : H;
        g.A = l == 0 ? n->A0 : n->Act[l - 1];
        g.sam = K; g.sak = 1;
        g.za = l == 0 ? (long long)n->bmax * NIN : zact;
        g.B = n->w + kOffW[l];
        g.sbk = 1; g.sbn = K; g.zb = P;
        g.M = B; g.N = H; g.K = K;
        g.bias = n->master + kOffB[l]; g.zbias = P;
        g.Z = n->Z[l]; g.Act = n->Act[l];
        g.ldc = H; g.zc = zact;
        int rc = launch_gemm(EPI_FWD, g, n->members, n->stream);
        if (rc) return rc;
    }
    dim3 grid((B + 7) / 8, n->members);
    out_layer_kernel<<<grid, 256, 0, n->stream>>>(n->Act[3], n->Z[3], n->w, n->master, n->yb, n->bmax, B, train ? 1 : 0,
                                                  n->fhat, n->dz, n->dZ[0], n->dZb[0], zact);
    IT_CK(cudaGetLastError());
    return IT_OK;
}

// backward of the batch into n->grad (after forward(train = true))
int backward(it_mlp *n, int B) {
    const long long zact = (long long)n->bmax * H;
    out_grad_kernel<<<n->members, H + 32, 0, n->stream>>>(n->Act[3], n->dz, B, n->grad, zact);
    IT_CK(cudaGetLastError());
    int cur = 0;
    for (int l = 3; l >= 0; --l) {
        const int K = l == 0 ? NIN : H;
        // weight gradient: gW[o][i] = sum_m dZ[m][o] A_{l-1}[m][i]
        GemmArgs g{};
        g.A = n->dZb[cur]; g.sam = 1; g.sak = H; g.za = zact;
        g.B = l == 0 ? n->A0 : n->Act[l - 1];
        g.sbk = K; g.sbn = 1; g.zb = l == 0 ? (long long)n->bmax * NIN : zact;
        g.M = H; g.N = K; g.K = B;
        g.Out = n->grad + kOffW[l]; g.ldc = K; g.zc = P;
        int rc = launch_gemm(EPI_WGRAD, g, n->members, n->stream);
        if (rc) return rc;
        bias_grad_kernel<<<n->members, H, 0, n->stream>>>(n->dZ[cur], B, n->grad, kOffB[l], zact);
        IT_CK(cudaGetLastError());
        if (l == 0) break;
        // data gradient into the layer below: dZ_{l-1} = (dZ_l W_l) * SiLU'(Z_{l-1})
        GemmArgs d{};
        d.A = n->dZb[cur]; d.sam = H; d.sak = 1; d.za = zact;
        d.B = n->w + kOffW[l]; d.sbk = K; d.sbn = 1; d.zb = P;
        d.M = B; d.N = H; d.K = H;
        d.Z = n->Z[l - 1]; d.Act = n->dZb[cur ^ 1]; d.Out = n->dZ[cur ^ 1];
        d.ldc = H; d.zc = zact;
        rc = launch_gemm(EPI_BWD, d, n->members, n->stream);
        if (rc) return rc;
        cur ^= 1;
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

int gather(it_mlp *n, const float *X, const float *Y, const int *idx, int B) {
    const long long tot = (long long)n->members * B * NIN;
    gather_inputs_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, n->stream>>>(X, Y, idx, B, n->members, n->bmax, n->mean,
                                                                               n->inv_std, n->A0, n->yb);
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
    return IT_OK;
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
        (e = cudaMalloc(&n->A0, sizeof(__nv_bfloat16) * members * max_batch * NIN)) != cudaSuccess ||
        (e = cudaMalloc(&n->fhat, sizeof(float) * members * max_batch)) != cudaSuccess ||
        (e = cudaMalloc(&n->dz, sizeof(float) * members * max_batch)) != cudaSuccess ||
        (e = cudaMalloc(&n->yb, sizeof(float) * members * max_batch)) != cudaSuccess ||
        (e = cudaMalloc(&n->idx, sizeof(int) * members * max_batch)) != cudaSuccess ||
        (e = cudaMalloc(&n->loss, sizeof(double) * members)) != cudaSuccess)
        return bail("mlp allocation");
    for (int l = 0; l < 4; ++l)
        if ((e = cudaMalloc(&n->Z[l], sizeof(float) * za)) != cudaSuccess ||
            (e = cudaMalloc(&n->Act[l], sizeof(__nv_bfloat16) * za)) != cudaSuccess)
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
    // each member walks the data in its own order (ensemble diversity)
    std::vector<std::vector<int>> perm(Z, std::vector<int>((size_t)N));
    std::vector<uint64_t> st(Z);
    for (int z = 0; z < Z; ++z) st[z] = seed + 0x9E3779B97F4A7C15ULL * (uint64_t)(z + 1);
    std::vector<int> hidx((size_t)Z * n->bmax);
    std::vector<double> lossb(Z);
    for (int ep = 0; ep < epochs; ++ep) {
        for (int z = 0; z < Z; ++z) {
            auto &pz = perm[z];
            for (long long i = 0; i < N; ++i) pz[i] = (int)i;
            for (long long i = N - 1; i > 0; --i) {   // Fisher-Yates with SplitMix64
                const long long j = (long long)(splitmix_next(st[z]) % (uint64_t)(i + 1));
                std::swap(pz[i], pz[j]);
            }
        }
        double ep_loss = 0.0;
        int nb = 0;
        for (long long b0 = 0; b0 + batch <= N || (b0 < N && nb == 0); b0 += batch) {
            const int B = (int)std::min<long long>(batch, N - b0);
            for (int z = 0; z < Z; ++z)
                std::memcpy(hidx.data() + (size_t)z * n->bmax, perm[z].data() + b0, sizeof(int) * B);
            IT_CK(cudaMemcpyAsync(n->idx, hidx.data(), sizeof(int) * Z * n->bmax, cudaMemcpyHostToDevice, n->stream));
            int rc = gather(n, n->X, n->Y, n->idx, B);
            if (!rc) rc = forward(n, B, true);
            if (!rc && loss_per_epoch) {
                loss_kernel<<<n->members, 256, 0, n->stream>>>(n->fhat, n->yb, n->bmax, B, n->loss);
                IT_CK(cudaGetLastError());
            }
            if (!rc) rc = backward(n, B);
            if (!rc) rc = adam_step(n, (float)lr);
            if (rc) return rc;
            if (loss_per_epoch) {
                IT_CK(cudaMemcpyAsync(lossb.data(), n->loss, sizeof(double) * n->members, cudaMemcpyDeviceToHost, n->stream));
                IT_CK(cudaStreamSynchronize(n->stream));
                for (double v : lossb) ep_loss += v / n->members;
            } else {
                IT_CK(cudaStreamSynchronize(n->stream));   // hidx is reused by the next batch
            }
            ++nb;
        }
        if (loss_per_epoch) loss_per_epoch[ep] = ep_loss / std::max(nb, 1);
    }
    IT_CK(cudaStreamSynchronize(n->stream));
    return IT_OK;
}

int it_mlp_loss_grad(it_mlp *n, int64_t count, const double *x, const double *y, float *grads, double *loss) {
    if (!n || !x || !y || count < 1 || count > n->bmax) return mfail(IT_EINVAL, "bad argument");
    float *dX = nullptr, *dY = nullptr;
    int rc = upload_inputs(n, count, x, y, &dX, &dY);
    if (!rc) rc = gather(n, dX, dY, nullptr, (int)count);
    if (!rc) rc = forward(n, (int)count, true);
    if (!rc) {
        loss_kernel<<<n->members, 256, 0, n->stream>>>(n->fhat, n->yb, n->bmax, (int)count, n->loss);
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
        rc = gather(n, dX + b0 * NIN, nullptr, nullptr, B);
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
    return rc;
}

int it_mlp_destroy(it_mlp *n) {
    mlp_free(n);
    return IT_OK;
}

}  // extern "C"
