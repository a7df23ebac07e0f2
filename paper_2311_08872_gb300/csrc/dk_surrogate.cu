// Learned level below level 0 (not in the paper): feature projection of the
// level-0 noise, a direct sampler of the features' exact law, and the
// kernels that train and run a 64-256-256-256-1 ReLU perceptron with BF16
// tensor-core GEMMs (dk_umma.cu), FP32 accumulation and FP32 master weights.
//
// Features.  With e_j the 32 lowest real orthonormal grid modes (cosine and
// sine per wave vector k, ordered by |k|^2) and g_j the per-step factor of the
// noise-free scheme on e_j, a level-0 sample's features are
//     F_(j,r) = sum_m g_j^(M-1-m) <Z^m_(.,r), e_j>,   r = 1, 2,
// i.e. the noise that the heat semigroup carries to time T on each low mode.
// For i.i.d. standard normals they are independent N(0, sum_i g_j^(2i)); the
// network sees F / sigma, so the level below 0 draws its inputs as plain
// standard normals, the exact law of the features of the coupled correction
// level, which keeps the telescoping sum unbiased whatever the network.
#include <cuda_bf16.h>

#include <cstdint>

#include "dk_device.cuh"
#include "dk_kernels.h"

namespace dk {

namespace {
constexpr unsigned kFullMask = 0xffffffffu;
}

// ------------------------------------------------------------------ features
// One CTA of 128 threads per sample (grid-stride over samples); thread t
// handles the cell pairs t, t + 128, ...; shared memory holds the mode table.
__global__ void __launch_bounds__(128) feature_kernel(const FeatArgs a) {
    extern __shared__ float fsm[];
    const int cells = a.n * a.n;
    float* E = fsm;                         // [32][cells]
    float* red = fsm + kModes * cells;      // [4][64]
    for (int i = threadIdx.x; i < kModes * cells; i += 128) E[i] = a.E[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long s = blockIdx.x; s < a.count; s += gridDim.x) {
        const long long sid = a.first + s;
        const uint32_t c2 = static_cast<uint32_t>(sid);
        const uint32_t c3 = a.tag | ((static_cast<uint32_t>(static_cast<unsigned long long>(sid) >> 32) & 0xffffu) << 16);
        float acc[kModes][2];
#pragma unroll
        for (int k = 0; k < kModes; ++k) acc[k][0] = acc[k][1] = 0.f;
        for (int m = 0; m < a.M; ++m) {
#pragma unroll
            for (int k = 0; k < kModes; ++k) {
                acc[k][0] *= a.g[k];
                acc[k][1] *= a.g[k];
            }
            for (int p = threadIdx.x; p < cells / 2; p += 128) {
                const uint4 x = philox10(make_uint4(static_cast<uint32_t>(p), static_cast<uint32_t>(m), c2, c3),
                                         a.key0, a.key1);
                float z1a, z2a, z1b, z2b;
                box_muller(x.x, x.y, z1a, z2a);
                box_muller(x.z, x.w, z1b, z2b);
#pragma unroll
                for (int k = 0; k < kModes; ++k) {
                    const float2 e = *reinterpret_cast<const float2*>(E + k * cells + 2 * p);
                    acc[k][0] = fmaf(e.x, z1a, fmaf(e.y, z1b, acc[k][0]));
                    acc[k][1] = fmaf(e.x, z2a, fmaf(e.y, z2b, acc[k][1]));
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kModes; ++k)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                float v = acc[k][r];
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(kFullMask, v, off);
                if (lane == 0) red[warp * kFeat + 2 * k + r] = v;
            }
        __syncthreads();
        if (threadIdx.x < kFeat) {
            const int j = threadIdx.x;
            const float f = (red[j] + red[kFeat + j] + red[2 * kFeat + j] + red[3 * kFeat + j]) * a.inv_sigma[j];
            a.X[s * kFeat + j] = __float2bfloat16_rn(f);
            if (a.Xf) a.Xf[s * kFeat + j] = f;
        }
        __syncthreads();
    }
}

// Direct draw of the standardised features: 64 normals per sample from
// Philox counters (j, 0, id, tag), j = 0..15 giving 4 normals each.
__global__ void direct_feature_kernel(const FeatArgs a) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= a.count * (kFeat / 4)) return;
    const long long s = t / (kFeat / 4);
    const int j = static_cast<int>(t % (kFeat / 4));
    const long long sid = a.first + s;
    const uint32_t c3 = a.tag | ((static_cast<uint32_t>(static_cast<unsigned long long>(sid) >> 32) & 0xffffu) << 16);
    const uint4 x = philox10(make_uint4(static_cast<uint32_t>(j), 0u, static_cast<uint32_t>(sid), c3), a.key0, a.key1);
    float z0, z1, z2, z3;
    box_muller(x.x, x.y, z0, z1);
    box_muller(x.z, x.w, z2, z3);
    __nv_bfloat16* o = a.X + s * kFeat + 4 * j;
    o[0] = __float2bfloat16_rn(z0);
    o[1] = __float2bfloat16_rn(z1);
    o[2] = __float2bfloat16_rn(z2);
    o[3] = __float2bfloat16_rn(z3);
    if (a.Xf) {
        float* of = a.Xf + s * kFeat + 4 * j;
        of[0] = z0; of[1] = z1; of[2] = z2; of[3] = z3;
    }
}

// ------------------------------------------------------------- BF16 GEMM
// The dense layers' GEMMs run on the 5th-generation tensor cores (tcgen05,
// dk_umma.cu); this file holds the output layer (K outputs, too narrow for a
// tensor-core tile), the feature kernels, Adam and the moment kernels.

// -------------------------------------------------------- small MLP kernels
// Output layer forward: y[b][o] = H3[b] . w4[o] + b4[o], o < KO (one warp per row).
__global__ void out_forward_kernel(const __nv_bfloat16* H, const float* w, const float* b, int B, int K, int KO,
                                   float* y) {
    const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= B) return;
    for (int o = 0; o < KO; ++o) {
        float s = 0.f;
        for (int k = lane; k < K; k += 32) s = fmaf(__bfloat162float(H[(size_t)row * K + k]), w[(size_t)o * K + k], s);
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(kFullMask, s, off);
        if (lane == 0) y[(size_t)row * KO + o] = s + b[o];
    }
}

// dy[b][o] = 2 (y - t) / B; dH[b][k] = (sum_o dy[b][o] w4[o][k]) (H[b][k] > 0) as BF16.
__global__ void out_backward_kernel(const float* y, const float* t, const __nv_bfloat16* H, const float* w, int B,
                                    int K, int KO, float* dy, __nv_bfloat16* dH) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)B * K) return;
    const int b = static_cast<int>(i / K), k = static_cast<int>(i % K);
    float v = 0.f;
    for (int o = 0; o < KO; ++o) {
        const size_t bo = (size_t)b * KO + o;
        const float d = 2.f * (y[bo] - t[bo]) / static_cast<float>(B);
        if (k == 0) dy[bo] = d;
        v = fmaf(d, w[(size_t)o * K + k], v);
    }
    dH[i] = __float2bfloat16_rn(__bfloat162float(H[i]) > 0.f ? v : 0.f);
}

// Column sums: out[n] = sum_b X[b][n] (X BF16 or FP32), fixed order per column.
__global__ void colsum_kernel(const __nv_bfloat16* Xb, const float* Xf, int B, int N, float* out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += Xb ? __bfloat162float(Xb[(size_t)b * N + n]) : Xf[(size_t)b * N + n];
    out[n] = s;
}

// dW4[o][k] = sum_b dy[b][o] H3[b][k]; db4[o] = sum_b dy[b][o].
__global__ void out_weight_grad_kernel(const float* dy, const __nv_bfloat16* H, int B, int K, int KO, float* dw,
                                       float* db) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < K * KO) {
        const int o = j / K, k = j % K;
        float s = 0.f;
        for (int b = 0; b < B; ++b) s = fmaf(dy[(size_t)b * KO + o], __bfloat162float(H[(size_t)b * K + k]), s);
        dw[j] = s;
    } else if (j < K * KO + KO) {
        const int o = j - K * KO;
        float s = 0.f;
        for (int b = 0; b < B; ++b) s += dy[(size_t)b * KO + o];
        db[o] = s;
    }
}

// Adam (Kingma & Ba, 2015) with bias correction; refreshes the BF16 weights.
__global__ void adam_kernel(float* theta, const float* grad, float* m1, float* m2, int P, float lr, float b1, float b2,
                            float eps, float c1, float c2, const int* bf_index, __nv_bfloat16* theta_bf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const float gi = grad[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    const float upd = lr * (a / c1) / (sqrtf(v / c2) + eps);
    const float w = theta[i] - upd;
    theta[i] = w;
    const int j = bf_index[i];
    if (j >= 0) theta_bf[j] = __float2bfloat16_rn(w);
}

__global__ void gather_kernel(const __nv_bfloat16* X, const float* T, const int* idx, int B, int KO,
                              __nv_bfloat16* Xb, float* Tb) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)B * kFeat) return;
    const int b = static_cast<int>(i / kFeat), j = static_cast<int>(i % kFeat);
    const int src = idx[b];
    Xb[i] = X[(size_t)src * kFeat + j];
    if (j < KO) Tb[(size_t)b * KO + j] = T[(size_t)src * KO + j];
}

// Squared error of a batch summed over its n values (rows x outputs) and
// divided by the rows B, FP64 accumulation, one block.
__global__ void mse_kernel(const float* y, const float* t, int n, int B, double* out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) {
        const double d = static_cast<double>(y[i]) - t[i];
        s += d * d;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] / B;
}

// Per-sample quantities of a surrogate batch into per-block FP64 partials
// (entry-major [stride][blocks]) in the moment layout of the level kernels,
// quantity by quantity: q = (j, l), j <= l when `products` (else l = j).
// That_k = network output k (sqrt(N)(Y_k - Ybar_k)); S_jl = That_j That_l.
// part = -1: dP = S (level below 0); part = 0: dP = P_0 - S with
// P_0 = N D_j D_l, D the level-0 sample's fluctuations (correction level).
__global__ void __launch_bounds__(256) surrogate_moments_kernel(const float* that, const double* d0, int d0_stride,
                                                                int part, double N, long long count, int stride,
                                                                int KO, int products, double* partials) {
    __shared__ double sh[8][12];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const double rsN = 1.0 / sqrt(N);
    int q = 0;
    for (int j = 0; j < KO; ++j) {
        const int lend = products ? KO : j + 1;
        for (int l = j; l < lend; ++l, ++q) {
            double v[12];
#pragma unroll
            for (int e = 0; e < 12; ++e) v[e] = 0.0;
            for (long long i = blockIdx.x * 256LL + threadIdx.x; i < count; i += 256LL * gridDim.x) {
                const double tj = that[i * KO + j], tl = that[i * KO + l];
                const double S = tj * tl;
                const double dj = part == 0 ? d0[i * d0_stride + j] : 0.0;
                const double dl = part == 0 ? d0[i * d0_stride + l] : 0.0;
                const double pf = part == 0 ? N * dj * dl : S;
                const double pc = part == 0 ? S : 0.0;
                const double dp = pf - pc, dp2 = dp * dp;
                v[0] += dp; v[1] += dp2; v[2] += dp2 * dp; v[3] += dp2 * dp2;
                v[4] += pf; v[5] += pf * pf; v[6] += pc; v[7] += pc * pc;
                const double yf = part == 0 ? dj : tj * rsN;
                const double yc = part == 0 ? tj * rsN : 0.0;
                v[8] += yf; v[9] += yf * yf; v[10] += yc; v[11] += yc * yc;
            }
#pragma unroll
            for (int e = 0; e < 12; ++e)
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) v[e] += __shfl_xor_sync(kFullMask, v[e], off);
            if (lane == 0)
#pragma unroll
                for (int e = 0; e < 12; ++e) sh[w][e] = v[e];
            __syncthreads();
            if (threadIdx.x < 12 && 2 + 12 * q + (int)threadIdx.x < stride) {
                double t = 0.0;
                for (int ww = 0; ww < 8; ++ww) t += sh[ww][threadIdx.x];
                partials[(size_t)(2 + 12 * q + threadIdx.x) * gridDim.x + blockIdx.x] = t;
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        // entry 0: samples of this block; entry 1: mass error (none here)
        long long c = 0;
        for (long long i = blockIdx.x * 256LL; i < count; i += 256LL * gridDim.x) c += min(256LL, count - i);
        partials[blockIdx.x] = (double)c;
        partials[(size_t)gridDim.x + blockIdx.x] = 0.0;
    }
}

// ------------------------------------------------------------------ launch
cudaError_t launch_features(const FeatArgs& a, int max_ctas, cudaStream_t st) {
    const size_t smem = sizeof(float) * (kModes * a.n * a.n + 4 * kFeat);
    cudaError_t e = cudaFuncSetAttribute(feature_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<long long>(a.count, max_ctas);
    feature_kernel<<<grid, 128, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_direct_features(const FeatArgs& a, cudaStream_t st) {
    const long long threads = a.count * (kFeat / 4);
    direct_feature_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_out_forward(const __nv_bfloat16* H, const float* w, const float* b, int B, int K, int KO, float* y,
                               cudaStream_t st) {
    out_forward_kernel<<<(B + 7) / 8, 256, 0, st>>>(H, w, b, B, K, KO, y);
    return cudaGetLastError();
}

cudaError_t launch_out_backward(const float* y, const float* t, const __nv_bfloat16* H, const float* w, int B, int K,
                                int KO, float* dy, __nv_bfloat16* dH, float* dw, float* db, cudaStream_t st) {
    out_backward_kernel<<<(unsigned)(((long long)B * K + 255) / 256), 256, 0, st>>>(y, t, H, w, B, K, KO, dy, dH);
    out_weight_grad_kernel<<<(K * KO + KO + 127) / 128, 128, 0, st>>>(dy, H, B, K, KO, dw, db);
    return cudaGetLastError();
}

cudaError_t launch_colsum(const __nv_bfloat16* Xb, const float* Xf, int B, int N, float* out, cudaStream_t st) {
    colsum_kernel<<<(N + 127) / 128, 128, 0, st>>>(Xb, Xf, B, N, out);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* theta, const float* grad, float* m1, float* m2, int P, float lr, float b1, float b2,
                        float eps, float c1, float c2, const int* bf_index, __nv_bfloat16* theta_bf,
                        cudaStream_t st) {
    adam_kernel<<<(P + 255) / 256, 256, 0, st>>>(theta, grad, m1, m2, P, lr, b1, b2, eps, c1, c2, bf_index, theta_bf);
    return cudaGetLastError();
}

cudaError_t launch_gather(const __nv_bfloat16* X, const float* T, const int* idx, int B, int KO, __nv_bfloat16* Xb,
                          float* Tb, cudaStream_t st) {
    gather_kernel<<<(unsigned)(((long long)B * kFeat + 255) / 256), 256, 0, st>>>(X, T, idx, B, KO, Xb, Tb);
    return cudaGetLastError();
}

cudaError_t launch_mse(const float* y, const float* t, int n, int B, double* out, cudaStream_t st) {
    mse_kernel<<<1, 256, 0, st>>>(y, t, n, B, out);
    return cudaGetLastError();
}

cudaError_t launch_surrogate_moments(const float* that, const double* d0, int d0_stride, int part, double N,
                                     long long count, int stride, int KO, int products, int blocks, double* partials,
                                     cudaStream_t st) {
    surrogate_moments_kernel<<<blocks, 256, 0, st>>>(that, d0, d0_stride, part, N, count, stride, KO, products,
                                                      partials);
    return cudaGetLastError();
}

}  // namespace dk
