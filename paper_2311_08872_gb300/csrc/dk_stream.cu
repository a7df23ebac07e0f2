// Streamed-state kernels for grids too large to keep a sample in registers
// (n >= 512: the finest levels of the low-density and large workloads).
//
// The state of `S` samples in flight lives in global memory (sized to stay in
// L2): the fine fixed-point state q and the coarse state qc (both double
// buffered) and the coupled coarse normal sums zt.  The scheme is the same as
// the register kernels' (Eq. FullyDiscreteDK with b0 = 0, b1 = 1; NN coupling
// of Section 3.2), in the same integer flux form and with the same FP32
// expressions for the transfers and the coupled sums, so the fine and coarse
// states agree with theirs bit for bit.
//
// One launch per fine step m: a CTA loads q^m on its tile and a one-cell halo,
// draws the normals of step m for the tile and for the halo cells (one extra
// Philox call per halo cell pair, so the transfers G^m never go to memory),
// and writes q^{m+1} and, for coupled samples, the running coarse sums zt.
// After the fourth fine step of a coarse step, a coarse launch forms the
// coarse transfers from qc and zt (tile and halo) and updates qc.  Kernel
// boundaries order all reads and writes: no kernel waits on another.
//
// Fine-step CTAs: 16 x 16 threads on a 32 x 64 tile, each thread a 2 x 4 block
// of fine cells (two coarse cells); two builds, for 4 or 5 resident CTAs per
// SM (at most 64 or 48 registers per thread), picked by the autotuner.
// The coarse step and the observables use 32 x 32 tiles.
#include <cstdint>

#include "dk_device.cuh"
#include "dk_kernels.h"

namespace dk {

namespace {

constexpr int kTile = 32;            // fine cells per tile side
constexpr int kTc = kTile / 2;       // coarse cells per tile side (= threads per side)
constexpr int kThreads = kTc * kTc;  // 256
// fine-step tiles: FR x kFC fine cells with a one-cell halo in shared memory,
// row lr = r - R0 + 1 (0 .. FR+1), column lc = c - C0 + 4 (3 .. kFC+4), so
// that each thread's own four cells sit on a 16-byte boundary
constexpr int kFC = 64;
constexpr int kFW = kFC + 8;
constexpr int kFR = 32;
constexpr int kStreamVariants = 2;
// minimum resident CTAs per SM the compiler is asked for, per variant
__host__ __device__ constexpr int fine_min_blocks(int variant) { return variant == 0 ? 4 : 5; }
__host__ __device__ constexpr int fine_threads(int fr) { return 8 * fr; }
__host__ __device__ constexpr int fine_smem(int fr) { return 3 * (fr + 2) * kFW * (int)sizeof(int32_t); }

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Transfers of the horizontal cell pair p (cells 2p, 2p+1 of the row-major
// grid) at fine step m, from the pair's state qa, qb; the normals of the pair
// are also added to the running coarse sums (z1, z2) in the register kernels'
// order (cell 2p first).
struct PairNoise {
    int32_t g1a, g2a, g1b, g2b;
};

__device__ __forceinline__ PairNoise pair_noise(const SArgs& a, uint32_t p, int m, uint32_t c2, uint32_t c3,
                                                int32_t qa, int32_t qb, float& z1, float& z2) {
    const uint4 x = philox10(make_uint4(p, static_cast<uint32_t>(m), c2, c3), a.key0, a.key1);
    float ra, ca, sa, rb, cb, sb;
    box_muller_polar(x.x, x.y, ra, ca, sa);
    box_muller_polar(x.z, x.w, rb, cb, sb);
    const float ta = noise_amp(qa, a.gf) * ra, tb = noise_amp(qb, a.gf) * rb;
    z1 = fmaf(rb, cb, fmaf(ra, ca, z1));
    z2 = fmaf(rb, sb, fmaf(ra, sa, z2));
    return {__float2int_rn(ta * ca), __float2int_rn(ta * sa), __float2int_rn(tb * cb), __float2int_rn(tb * sb)};
}

__device__ __forceinline__ void sample_counter(const SArgs& a, int s, uint32_t& c2, uint32_t& c3) {
    const long long sid = a.sid0 + s;
    c2 = static_cast<uint32_t>(sid);
    c3 = a.tag | ((static_cast<uint32_t>(static_cast<unsigned long long>(sid) >> 32) & 0xffffu) << 16);
}

}  // namespace

// Initial state.
__global__ void __launch_bounds__(kThreads) stream_init_kernel(const SArgs a) {
    const int s = blockIdx.y;
    if (s >= a.count) return;
    const int tpr = a.n / kTile;
    const int T1 = blockIdx.x / tpr, T2 = blockIdx.x % tpr;
    const int tx = threadIdx.x % kTc, ty = threadIdx.x / kTc;
    const int I = T1 * kTc + ty, J = T2 * kTc + tx;            // coarse cell
    const int r0 = 2 * I, c0 = 2 * J;
    const size_t base = (size_t)s * a.n * a.n;
#pragma unroll
    for (int i = 0; i < 2; ++i)
        *reinterpret_cast<int2*>(a.q[0] + base + (size_t)(r0 + i) * a.n + c0) =
            *reinterpret_cast<const int2*>(a.q0f + (size_t)(r0 + i) * a.n + c0);
    if (a.coupled) a.qc[0][(size_t)s * a.nc * a.nc + (size_t)I * a.nc + J] = a.q0c[(size_t)I * a.nc + J];
}

// Fine step m: noise of step m on the tile and its halo, then q^{m+1}.
// CTA: 16 x FR/2 threads on an FR x 64 tile; thread (tx, ty) owns the 2 x 4
// fine block at (R0 + 2 ty, C0 + 4 tx) = 2 coarse cells.
template <int FR, int MINB>
__global__ void __launch_bounds__(fine_threads(FR), MINB) stream_fine_kernel(const SArgs a, int m) {
    constexpr int kHaloPairs = 64 + 2 * FR;   // 2 x 32 pairs in the halo rows, one per row in the halo columns
    const int s = blockIdx.z;
    if (s >= a.count) return;
    const int n = a.n;
    const int t = threadIdx.x;
    const int tx = t % 16, ty = t / 16;
    const int R0 = blockIdx.y * FR, C0 = blockIdx.x * kFC;
    const int r0 = R0 + 2 * ty, c0 = C0 + 4 * tx;
    const size_t base = (size_t)s * n * n;
    const int32_t* qin = a.q[m & 1] + base;
    int32_t* qout = a.q[(m + 1) & 1] + base;
    uint32_t c2, c3;
    sample_counter(a, s, c2, c3);

    extern __shared__ __align__(16) int32_t smem_fine[];
    int32_t (*sq)[kFW] = reinterpret_cast<int32_t (*)[kFW]>(smem_fine);
    int32_t (*s1)[kFW] = reinterpret_cast<int32_t (*)[kFW]>(smem_fine + (FR + 2) * kFW);
    int32_t (*s2)[kFW] = reinterpret_cast<int32_t (*)[kFW]>(smem_fine + 2 * (FR + 2) * kFW);

    // own 2x4 block: state, normals of step m, transfers; coupled sums of its
    // two coarse cells in the register kernels' order
    const int lr0 = 2 * ty + 1, lc0 = 4 * tx + 4;
    int32_t q[2][4], G1[2][4], G2[2][4];
    float4* const zp = reinterpret_cast<float4*>(a.zt + (size_t)s * a.nc * a.nc + (size_t)(r0 >> 1) * a.nc + (c0 >> 1));
    float z[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    if (a.coupled && (m & 3) != 0) {
        const float4 v = *zp;
        z[0][0] = v.x; z[0][1] = v.y; z[1][0] = v.z; z[1][1] = v.w;
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int4 v = *reinterpret_cast<const int4*>(qin + (size_t)(r0 + i) * n + c0);
        q[i][0] = v.x; q[i][1] = v.y; q[i][2] = v.z; q[i][3] = v.w;
        const uint32_t p = static_cast<uint32_t>(((r0 + i) * n + c0) >> 1);
        const PairNoise g = pair_noise(a, p, m, c2, c3, v.x, v.y, z[0][0], z[0][1]);
        const PairNoise h = pair_noise(a, p + 1, m, c2, c3, v.z, v.w, z[1][0], z[1][1]);
        G1[i][0] = g.g1a; G2[i][0] = g.g2a; G1[i][1] = g.g1b; G2[i][1] = g.g2b;
        G1[i][2] = h.g1a; G2[i][2] = h.g2a; G1[i][3] = h.g1b; G2[i][3] = h.g2b;
        *reinterpret_cast<int4*>(&sq[lr0 + i][lc0]) = v;
        *reinterpret_cast<int4*>(&s1[lr0 + i][lc0]) = make_int4(g.g1a, g.g1b, h.g1a, h.g1b);
        *reinterpret_cast<int4*>(&s2[lr0 + i][lc0]) = make_int4(g.g2a, g.g2b, h.g2a, h.g2b);
    }
    // halo: rows R0-1 and R0+FR (32 pairs each: state and G1), columns C0-1
    // and C0+kFC (one pair per row: state and G2 of the cell next to the tile)
    if (t < kHaloPairs) {
        float d1 = 0.f, d2 = 0.f;   // halo normals do not enter this tile's coarse sums
        if (t < 64) {
            const int side = t >> 5, k = t & 31;
            const int r = wrapi(side ? R0 + FR : R0 - 1, n), c = C0 + 2 * k;
            const int2 v = *reinterpret_cast<const int2*>(qin + (size_t)r * n + c);
            const PairNoise g = pair_noise(a, static_cast<uint32_t>((r * n + c) >> 1), m, c2, c3, v.x, v.y, d1, d2);
            const int lr = side ? FR + 1 : 0;
            *reinterpret_cast<int2*>(&sq[lr][4 + 2 * k]) = v;
            *reinterpret_cast<int2*>(&s1[lr][4 + 2 * k]) = make_int2(g.g1a, g.g1b);
        } else {
            const int u = t - 64, side = u / FR, rr = u % FR;
            const int r = R0 + rr, c = wrapi(side ? C0 + kFC : C0 - 2, n);
            const int2 v = *reinterpret_cast<const int2*>(qin + (size_t)r * n + c);
            const PairNoise g = pair_noise(a, static_cast<uint32_t>((r * n + c) >> 1), m, c2, c3, v.x, v.y, d1, d2);
            if (side) {
                sq[rr + 1][kFC + 4] = v.x;
                s2[rr + 1][kFC + 4] = g.g2a;
            } else {
                sq[rr + 1][3] = v.y;
                s2[rr + 1][3] = g.g2b;
            }
        }
    }
    __syncthreads();

    unsigned bad = 0;
    int32_t up[4], dn[4], gu[4], gd[4];
    {
        const int4 a0 = *reinterpret_cast<const int4*>(&sq[lr0 - 1][lc0]);
        const int4 a1 = *reinterpret_cast<const int4*>(&sq[lr0 + 2][lc0]);
        const int4 b0 = *reinterpret_cast<const int4*>(&s1[lr0 - 1][lc0]);
        const int4 b1 = *reinterpret_cast<const int4*>(&s1[lr0 + 2][lc0]);
        up[0] = a0.x; up[1] = a0.y; up[2] = a0.z; up[3] = a0.w;
        dn[0] = a1.x; dn[1] = a1.y; dn[2] = a1.z; dn[3] = a1.w;
        gu[0] = b0.x; gu[1] = b0.y; gu[2] = b0.z; gu[3] = b0.w;
        gd[0] = b1.x; gd[1] = b1.y; gd[2] = b1.z; gd[3] = b1.w;
    }
    int32_t ql[2], qr[2], gl[2], gr[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        ql[i] = sq[lr0 + i][lc0 - 1];
        qr[i] = sq[lr0 + i][lc0 + 4];
        gl[i] = s2[lr0 + i][lc0 - 1];
        gr[i] = s2[lr0 + i][lc0 + 4];
    }
    // each edge flux once per block, as in the register kernels
    flux_update<2, 4>(q, G1, G2, up, gu, dn, gd, ql, gl, qr, gr, a.Af);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) bad |= (static_cast<uint32_t>(q[i][j]) + 0x40000000u) >> 31;
        *reinterpret_cast<int4*>(qout + (size_t)(r0 + i) * n + c0) = make_int4(q[i][0], q[i][1], q[i][2], q[i][3]);
    }
    if (a.coupled) *zp = make_float4(z[0][0], z[0][1], z[1][0], z[1][1]);
    if (bad) atomicOr(a.err, kErrRange);
}

// Coarse step cn (after fine step 4 cn + 3): transfers from qc^cn and the
// coupled sums on the tile and its halo, then qc^{cn+1}.
__global__ void __launch_bounds__(kThreads) stream_coarse_kernel(const SArgs a, int cn) {
    const int s = blockIdx.y;
    if (s >= a.count) return;
    const int nc = a.nc;
    const int tpr = nc / kTile;
    const int T1 = blockIdx.x / tpr, T2 = blockIdx.x % tpr;
    const size_t base = (size_t)s * nc * nc;
    const int32_t* qin = a.qc[cn & 1] + base;
    int32_t* qout = a.qc[(cn + 1) & 1] + base;
    const float2* zt = a.zt + base;
    __shared__ int32_t sq[kTile + 2][kTile + 2];
    __shared__ int2 sg[kTile + 2][kTile + 2];
    const int R0 = T1 * kTile, C0 = T2 * kTile;
    for (int k = threadIdx.x; k < (kTile + 2) * (kTile + 2); k += kThreads) {
        const int lr = k / (kTile + 2), lc = k % (kTile + 2);
        const int gr = wrapi(R0 + lr - 1, nc), gcol = wrapi(C0 + lc - 1, nc);
        const int32_t qv = qin[(size_t)gr * nc + gcol];
        const float2 z = zt[(size_t)gr * nc + gcol];
        const float amp = noise_amp(qv, a.gc);
        sq[lr][lc] = qv;
        sg[lr][lc] = make_int2(__float2int_rn(amp * z.x), __float2int_rn(amp * z.y));
    }
    __syncthreads();
    unsigned bad = 0;
    for (int k = threadIdx.x; k < kTile * kTile; k += kThreads) {
        const int lr = k / kTile + 1, lc = k % kTile + 1;
        const int32_t x = sq[lr][lc];
        const int32_t d = edge_flux(a.Ac, sq[lr + 1][lc] - x) - edge_flux(a.Ac, x - sq[lr - 1][lc]) +
                          edge_flux(a.Ac, sq[lr][lc + 1] - x) - edge_flux(a.Ac, x - sq[lr][lc - 1]);
        const int32_t v = x + d + (sg[lr + 1][lc].x - sg[lr - 1][lc].x) + (sg[lr][lc + 1].y - sg[lr][lc - 1].y);
        qout[(size_t)(R0 + lr - 1) * nc + (C0 + lc - 1)] = v;
        bad |= (static_cast<uint32_t>(v) + 0x40000000u) >> 31;
    }
    if (bad) atomicOr(a.err, kErrRange);
}

// Per-tile partial observables: sums of (q - qbar) phi_k (fine, coarse), masses.
__global__ void __launch_bounds__(kThreads) stream_observe_kernel(const SArgs a) {
    const int s = blockIdx.y;
    if (s >= a.count) return;
    const int n = a.n, nc = a.nc;
    const int tpr = n / kTile;
    const int T1 = blockIdx.x / tpr, T2 = blockIdx.x % tpr;
    const int tx = threadIdx.x % kTc, ty = threadIdx.x / kTc;
    const int I = T1 * kTc + ty, J = T2 * kTc + tx;
    const int r0 = 2 * I, c0 = 2 * J;
    const int32_t* q = a.q[a.M & 1] + (size_t)s * n * n;
    double v[2 * kMaxObs + 2];
#pragma unroll
    for (int i = 0; i < 2 * kMaxObs + 2; ++i) v[i] = 0.0;
    long long mf = 0, mc = 0;
    // FP64 products and sums against FP64 test functions (the integer
    // fluctuations are exact in FP64): the projection of a rough fluctuation on
    // a smooth phi is small, and FP32 rounding of phi or of the partial sums,
    // uncorrelated with the noise, would reach 1e-5 of it on fine grids
    double sf[kMaxObs] = {0.0, 0.0, 0.0, 0.0}, sc[kMaxObs] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const size_t x = (size_t)(r0 + i) * n + c0 + j;
            const int32_t qv = q[x];
            mf += qv;
            for (int k = 0; k < a.n_obs; ++k)
                sf[k] = fma(static_cast<double>(qv - a.qbf[x]), a.phif64[(size_t)k * n * n + x], sf[k]);
        }
    if (a.coupled) {
        const size_t xc = (size_t)I * nc + J;
        const int32_t qv = a.qc[(a.M >> 2) & 1][(size_t)s * nc * nc + xc];
        mc = qv;
        for (int k = 0; k < a.n_obs; ++k)
            sc[k] = static_cast<double>(qv - a.qbc[xc]) * a.phic64[(size_t)k * nc * nc + xc];
    }
#pragma unroll
    for (int k = 0; k < kMaxObs; ++k) {
        v[k] = sf[k];
        v[kMaxObs + k] = sc[k];
    }
    v[2 * kMaxObs] = static_cast<double>(mf);
    v[2 * kMaxObs + 1] = static_cast<double>(mc);
    // block reduction in a fixed order: warp shuffles, then warp 0
    __shared__ double red[kThreads / 32][2 * kMaxObs + 2];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
#pragma unroll
        for (int i = 0; i < 2 * kMaxObs + 2; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < 2 * kMaxObs + 2; ++i) red[w][i] = v[i];
    __syncthreads();
    if (threadIdx.x < 2 * kMaxObs + 2) {
        double t = 0.0;
        for (int ww = 0; ww < kThreads / 32; ++ww) t += red[ww][threadIdx.x];
        const int tiles = gridDim.x;
        a.tile_part[((size_t)s * tiles + blockIdx.x) * (2 * kMaxObs + 2) + threadIdx.x] = t;
    }
}

// Per sample: tiles reduced in order, then the FP64 quantities and moment sums
// of the sample added to its slot (slot = position in the wave).
__global__ void stream_finish_kernel(const SArgs a, const KArgs k, int tiles, int n_slots) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.count) return;
    constexpr int W = 2 * kMaxObs + 2;
    double v[W];
    for (int i = 0; i < W; ++i) v[i] = 0.0;
    for (int t = 0; t < tiles; ++t)
        for (int i = 0; i < W; ++i) v[i] += a.tile_part[((size_t)s * tiles + t) * W + i];
    double Df[kMaxObs], Dc[kMaxObs];
    for (int q = 0; q < kMaxObs; ++q) {
        Df[q] = k.dscale_f * v[q] + k.delta_f[q];
        Dc[q] = a.coupled ? k.dscale_c * v[kMaxObs + q] + k.delta_c[q] : 0.0;
    }
    // entry-major slot partials: partials[e * n_slots + s]
    auto P = [&](int e) -> double& { return k.partials[(size_t)e * n_slots + s]; };
    P(0) += 1.0;
    double merr = fabs(v[2 * kMaxObs] - static_cast<double>(k.mass0_f)) * k.dscale_f;
    if (a.coupled) merr = fmax(merr, fabs(v[2 * kMaxObs + 1] - static_cast<double>(k.mass0_c)) * k.dscale_c);
    P(1) = fmax(P(1), merr);
    int qi = 0;
    for (int j = 0; j < k.n_obs; ++j) {
        const int kend = k.products ? k.n_obs : j + 1;
        for (int l = j; l < kend; ++l, ++qi) {
            const double pf = k.N * Df[j] * Df[l];
            const double pc = a.coupled ? k.N * Dc[j] * Dc[l] : 0.0;
            const double dp = pf - pc, dp2 = dp * dp;
            const int b = 2 + kNSum * qi;
            P(b + 0) += dp; P(b + 1) += dp2; P(b + 2) += dp2 * dp; P(b + 3) += dp2 * dp2;
            P(b + 4) += pf; P(b + 5) += pf * pf; P(b + 6) += pc; P(b + 7) += pc * pc;
            P(b + 8) += Df[j]; P(b + 9) += Df[j] * Df[j]; P(b + 10) += Dc[j]; P(b + 11) += Dc[j] * Dc[j];
        }
    }
    if (k.samples) {
        double* o = k.samples + (a.sid0 - k.first + s) * (2 * k.n_obs + 2);
        for (int q = 0; q < k.n_obs; ++q) {
            o[q] = Df[q];
            o[k.n_obs + q] = Dc[q];
        }
        o[2 * k.n_obs] = v[2 * kMaxObs] * k.dscale_f;
        o[2 * k.n_obs + 1] = a.coupled ? v[2 * kMaxObs + 1] * k.dscale_c : 0.0;
    }
}

__global__ void zero_kernel(double* p, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        p[i] = 0.0;
}

size_t stream_bytes(int n, int S) {
    const size_t nc = n / 2, tiles = (size_t)(n / kTile) * (n / kTile);
    return (size_t)S * ((size_t)n * n * 2 * sizeof(int32_t) + nc * nc * (2 * sizeof(int32_t) + sizeof(float2)) +
                        tiles * (2 * kMaxObs + 2) * sizeof(double));
}

int stream_variant_count() { return kStreamVariants; }

template <int MINB>
static cudaError_t fine_attr() {
    return cudaFuncSetAttribute(stream_fine_kernel<kFR, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                fine_smem(kFR));
}

cudaError_t stream_variant_info(int n, int variant, VariantInfo* out) {
    if (variant < 0 || variant >= kStreamVariants) return cudaErrorInvalidValue;
    const int fr = kFR;
    cudaError_t e = variant == 0 ? fine_attr<4>() : fine_attr<5>();
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    e = variant == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stream_fine_kernel<kFR, 4>,
                                                                     fine_threads(kFR), fine_smem(kFR))
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stream_fine_kernel<kFR, 5>,
                                                                     fine_threads(kFR), fine_smem(kFR));
    if (e != cudaSuccess) return e;
    *out = VariantInfo{};
    out->supported = (n % kFC == 0 && n % fr == 0 && per_sm > 0) ? 1 : 0;
    out->threads = fine_threads(fr);
    out->cluster = 1;
    out->slots_per_cta = 0;
    out->smem = fine_smem(fr);
    out->max_ctas = sms * per_sm;
    out->C = 2;        // coarse cells per thread along a row
    out->R = 1;
    out->tile_rows = fr;
    return cudaSuccess;
}

int stream_inflight(int n, size_t budget, int variant) {
    // the largest count that fits the budget, lowered while a smaller count
    // fills the last wave of fine-step CTAs clearly better
    const int s_max = (int)std::max<size_t>(1, budget / stream_bytes(n, 1));
    VariantInfo vi{};
    if (stream_variant_info(n, variant, &vi) != cudaSuccess || !vi.supported) return s_max;
    const long long resident = vi.max_ctas, ctas = (long long)(n / kFC) * (n / vi.tile_rows);
    int best = s_max;
    double best_eff = 0.0;
    for (int S = s_max; S >= std::max(1, s_max / 2); --S) {
        const long long c = S * ctas, waves = (c + resident - 1) / resident;
        const double eff = (double)c / (double)(waves * resident);
        if (eff > best_eff + 0.01) {
            best = S;
            best_eff = eff;
        }
    }
    return best;
}

void stream_carve(SArgs* a, void* buf, int n, int S) {
    unsigned char* p = static_cast<unsigned char*>(buf);
    const size_t cf = (size_t)S * n * n, cc = (size_t)S * (n / 2) * (n / 2);
    a->q[0] = reinterpret_cast<int32_t*>(p); p += cf * sizeof(int32_t);
    a->q[1] = reinterpret_cast<int32_t*>(p); p += cf * sizeof(int32_t);
    a->qc[0] = reinterpret_cast<int32_t*>(p); p += cc * sizeof(int32_t);
    a->qc[1] = reinterpret_cast<int32_t*>(p); p += cc * sizeof(int32_t);
    a->zt = reinterpret_cast<float2*>(p); p += cc * sizeof(float2);
    a->tile_part = reinterpret_cast<double*>(p);
}

cudaError_t stream_run(const KArgs& k, SArgs a, int S, int variant, cudaStream_t st) {
    // k.partials holds S slots (entry-major, [stride][S]); zero them, run the
    // waves of S samples, accumulate per slot, then the caller reduces.
    const int n = a.n;
    if (variant < 0 || variant >= kStreamVariants) return cudaErrorInvalidValue;
    const int fr = kFR;
    if (n % kFC != 0 || n % fr != 0 || (a.coupled && (a.nc % kTile != 0 || a.M % 4 != 0))) return cudaErrorInvalidValue;
    const int tiles = (n / kTile) * (n / kTile);
    const int ctiles = a.coupled ? (a.nc / kTile) * (a.nc / kTile) : 0;
    cudaError_t e = variant == 0 ? fine_attr<4>() : fine_attr<5>();
    if (e != cudaSuccess) return e;
    zero_kernel<<<64, 256, 0, st>>>(k.partials, (size_t)k.slot_stride * S);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (long long done = 0; done < k.count; done += S) {
        a.sid0 = k.first + done;
        a.count = (int)std::min<long long>(S, k.count - done);
        const dim3 grid(tiles, a.count), cgrid(ctiles, a.count), fgrid(n / kFC, n / fr, a.count);
        stream_init_kernel<<<grid, kThreads, 0, st>>>(a);
        for (int m = 0; m < a.M; ++m) {
            if (variant == 0)
                stream_fine_kernel<kFR, 4><<<fgrid, fine_threads(kFR), fine_smem(kFR), st>>>(a, m);
            else
                stream_fine_kernel<kFR, 5><<<fgrid, fine_threads(kFR), fine_smem(kFR), st>>>(a, m);
            if (a.coupled && (m & 3) == 3) stream_coarse_kernel<<<cgrid, kThreads, 0, st>>>(a, m >> 2);
        }
        stream_observe_kernel<<<grid, kThreads, 0, st>>>(a);
        stream_finish_kernel<<<(a.count + 63) / 64, 64, 0, st>>>(a, k, tiles, S);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace dk
