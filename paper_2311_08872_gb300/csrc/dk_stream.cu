// Streamed-state kernels for grids too large to keep a sample in registers
// (n >= 512: the finest levels of the low-density and large workloads).
//
// The state of `S` samples in flight lives in global memory (sized to stay in
// L2): fine fixed-point state q and noise transfers G = (G1, G2), both double
// buffered, the coarse state qc (double buffered) with its transfers Gc, and
// the coupled coarse normal sums zt.  The scheme is the same as the register
// kernels' (Eq. FullyDiscreteDK with b0 = 0, b1 = 1; NN coupling of Section
// 3.2), in the same integer flux form, so results agree with them bit for bit
// in the state.
//
// One launch per fine step m reads q^m and G^m (own cells and the 1-cell
// halo), writes q^{m+1}, then draws the normals of step m+1 for its own cells
// and writes G^{m+1} (and the coarse sums zt).  The launch that draws the last
// fine normals of a coarse step also writes that coarse step's transfers Gc; a
// coarse launch then updates qc.  Kernel boundaries order all reads and
// writes: no kernel waits on another.
//
// CTA: 16 x 16 threads on a 32 x 32 tile of fine cells; thread (tx, ty) owns
// the 2x2 fine block = 1 coarse cell at (16 T1 + ty, 16 T2 + tx).
#include <cstdint>

#include "dk_device.cuh"
#include "dk_kernels.h"

namespace dk {

namespace {

constexpr int kTile = 32;            // fine cells per tile side
constexpr int kTc = kTile / 2;       // coarse cells per tile side (= threads per side)
constexpr int kThreads = kTc * kTc;  // 256

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Noise of fine step m for the 2x2 block at fine (r0, c0): transfers into G,
// coupled sums into zt (overwrite when m % 4 == 0).
__device__ __forceinline__ void block_noise(const SArgs& a, int s, int m, int r0, int c0, const int32_t (&q)[2][2],
                                            int2 (&G)[2][2], float2& zt) {
    const long long sid = a.sid0 + s;
    const uint32_t c2 = static_cast<uint32_t>(sid);
    const uint32_t c3 = a.tag | ((static_cast<uint32_t>(static_cast<unsigned long long>(sid) >> 32) & 0xffffu) << 16);
    float s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const uint32_t p = static_cast<uint32_t>(((r0 + i) * a.n + c0) >> 1);
        const uint4 x = philox10(make_uint4(p, static_cast<uint32_t>(m), c2, c3), a.key0, a.key1);
        float z1a, z2a, z1b, z2b;
        box_muller(x.x, x.y, z1a, z2a);
        box_muller(x.z, x.w, z1b, z2b);
        const float sa = noise_amp(q[i][0], a.gf), sb = noise_amp(q[i][1], a.gf);
        G[i][0] = make_int2(__float2int_rn(sa * z1a), __float2int_rn(sa * z2a));
        G[i][1] = make_int2(__float2int_rn(sb * z1b), __float2int_rn(sb * z2b));
        s1 += z1a + z1b;
        s2 += z2a + z2b;
    }
    if ((m & 3) == 0) zt = make_float2(s1, s2);
    else zt = make_float2(zt.x + s1, zt.y + s2);
}

}  // namespace

// Initial state and the noise of step 0.
__global__ void __launch_bounds__(kThreads) stream_init_kernel(const SArgs a) {
    const int s = blockIdx.y;
    if (s >= a.count) return;
    const int tpr = a.n / kTile;
    const int T1 = blockIdx.x / tpr, T2 = blockIdx.x % tpr;
    const int tx = threadIdx.x % kTc, ty = threadIdx.x / kTc;
    const int I = T1 * kTc + ty, J = T2 * kTc + tx;            // coarse cell
    const int r0 = 2 * I, c0 = 2 * J;
    const size_t base = (size_t)s * a.n * a.n;
    int32_t q[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int2 v = *reinterpret_cast<const int2*>(a.q0f + (size_t)(r0 + i) * a.n + c0);
        q[i][0] = v.x; q[i][1] = v.y;
        *reinterpret_cast<int2*>(a.q[0] + base + (size_t)(r0 + i) * a.n + c0) = v;
    }
    int2 G[2][2];
    float2 zt = make_float2(0.f, 0.f);
    block_noise(a, s, 0, r0, c0, q, G, zt);
#pragma unroll
    for (int i = 0; i < 2; ++i)
        *reinterpret_cast<int4*>(a.G[0] + base + (size_t)(r0 + i) * a.n + c0) =
            make_int4(G[i][0].x, G[i][0].y, G[i][1].x, G[i][1].y);
    if (a.coupled) {
        const size_t cb = (size_t)s * a.nc * a.nc + (size_t)I * a.nc + J;
        a.qc[0][cb] = a.q0c[(size_t)I * a.nc + J];
        a.zt[cb] = zt;
    }
}

// Fine step m: q^{m+1} from q^m, G^m; then the noise of step m+1.
__global__ void __launch_bounds__(kThreads) stream_fine_kernel(const SArgs a, int m) {
    const int s = blockIdx.y;
    if (s >= a.count) return;
    const int n = a.n;
    const int tpr = n / kTile;
    const int T1 = blockIdx.x / tpr, T2 = blockIdx.x % tpr;
    const int tx = threadIdx.x % kTc, ty = threadIdx.x / kTc;
    const int I = T1 * kTc + ty, J = T2 * kTc + tx;
    const int r0 = 2 * I, c0 = 2 * J;
    const size_t base = (size_t)s * n * n;
    const int32_t* qin = a.q[m & 1] + base;
    int32_t* qout = a.q[(m + 1) & 1] + base;
    const int2* Gin = a.G[m & 1] + base;
    int2* Gout = a.G[(m + 1) & 1] + base;

    // tile + 1-cell halo in shared memory: q and (G1, G2)
    __shared__ int32_t sq[kTile + 2][kTile + 2];
    __shared__ int2 sg[kTile + 2][kTile + 2];
    const int R0 = T1 * kTile, C0 = T2 * kTile;
    for (int k = threadIdx.x; k < (kTile + 2) * (kTile + 2); k += kThreads) {
        const int lr = k / (kTile + 2), lc = k % (kTile + 2);
        const int gr = wrapi(R0 + lr - 1, n), gc = wrapi(C0 + lc - 1, n);
        sq[lr][lc] = qin[(size_t)gr * n + gc];
        sg[lr][lc] = Gin[(size_t)gr * n + gc];
    }
    __syncthreads();
    int32_t q[2][2];
    const int lr0 = 2 * ty + 1, lc0 = 2 * tx + 1;
    unsigned bad = 0;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int lr = lr0 + i, lc = lc0 + j;
            const int32_t x = sq[lr][lc];
            const int32_t d = edge_flux(a.Af, sq[lr + 1][lc] - x) - edge_flux(a.Af, x - sq[lr - 1][lc]) +
                              edge_flux(a.Af, sq[lr][lc + 1] - x) - edge_flux(a.Af, x - sq[lr][lc - 1]);
            const int32_t v = x + d + (sg[lr + 1][lc].x - sg[lr - 1][lc].x) + (sg[lr][lc + 1].y - sg[lr][lc - 1].y);
            q[i][j] = v;
            bad |= (static_cast<uint32_t>(v) + 0x40000000u) >> 31;
        }
#pragma unroll
    for (int i = 0; i < 2; ++i)
        *reinterpret_cast<int2*>(qout + (size_t)(r0 + i) * n + c0) = make_int2(q[i][0], q[i][1]);
    if (bad) atomicOr(a.err, kErrRange);
    if (m + 1 >= a.M) return;
    int2 G[2][2];
    const size_t cb = (size_t)s * a.nc * a.nc + (size_t)I * a.nc + J;
    float2 zt = make_float2(0.f, 0.f);
    if (a.coupled && ((m + 1) & 3) != 0) zt = a.zt[cb];
    block_noise(a, s, m + 1, r0, c0, q, G, zt);
#pragma unroll
    for (int i = 0; i < 2; ++i)
        *reinterpret_cast<int4*>(Gout + (size_t)(r0 + i) * n + c0) =
            make_int4(G[i][0].x, G[i][0].y, G[i][1].x, G[i][1].y);
    if (a.coupled) {
        if (((m + 1) & 3) == 3) {
            // the coupled normals of coarse step (m+1)/4 are complete: its transfers
            const int cn = (m + 1) >> 2;
            const int32_t qcv = a.qc[cn & 1][cb];
            const float amp = noise_amp(qcv, a.gc);
            a.Gc[cb] = make_int2(__float2int_rn(amp * zt.x), __float2int_rn(amp * zt.y));
        } else {
            a.zt[cb] = zt;
        }
    }
}

// Coarse step cn: qc^{cn+1} from qc^cn and Gc.
__global__ void __launch_bounds__(kThreads) stream_coarse_kernel(const SArgs a, int cn) {
    const int s = blockIdx.y;
    if (s >= a.count) return;
    const int nc = a.nc;
    const int tpr = nc / kTile;
    const int T1 = blockIdx.x / tpr, T2 = blockIdx.x % tpr;
    const size_t base = (size_t)s * nc * nc;
    const int32_t* qin = a.qc[cn & 1] + base;
    int32_t* qout = a.qc[(cn + 1) & 1] + base;
    const int2* Gc = a.Gc + base;
    __shared__ int32_t sq[kTile + 2][kTile + 2];
    __shared__ int2 sg[kTile + 2][kTile + 2];
    const int R0 = T1 * kTile, C0 = T2 * kTile;
    for (int k = threadIdx.x; k < (kTile + 2) * (kTile + 2); k += kThreads) {
        const int lr = k / (kTile + 2), lc = k % (kTile + 2);
        const int gr = wrapi(R0 + lr - 1, nc), gcol = wrapi(C0 + lc - 1, nc);
        sq[lr][lc] = qin[(size_t)gr * nc + gcol];
        sg[lr][lc] = Gc[(size_t)gr * nc + gcol];
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
    float sf[kMaxObs] = {0.f, 0.f, 0.f, 0.f}, sc[kMaxObs] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const size_t x = (size_t)(r0 + i) * n + c0 + j;
            const int32_t qv = q[x];
            mf += qv;
            for (int k = 0; k < a.n_obs; ++k)
                sf[k] = fmaf(__int2float_rn(qv - a.qbf[x]), a.phif[(size_t)k * n * n + x], sf[k]);
        }
    if (a.coupled) {
        const size_t xc = (size_t)I * nc + J;
        const int32_t qv = a.qc[(a.M >> 2) & 1][(size_t)s * nc * nc + xc];
        mc = qv;
        for (int k = 0; k < a.n_obs; ++k) sc[k] = __int2float_rn(qv - a.qbc[xc]) * a.phic[(size_t)k * nc * nc + xc];
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
    return (size_t)S * ((size_t)n * n * (2 * sizeof(int32_t) + 2 * sizeof(int2)) +
                        nc * nc * (2 * sizeof(int32_t) + sizeof(int2) + sizeof(float2)) +
                        tiles * (2 * kMaxObs + 2) * sizeof(double));
}

void stream_carve(SArgs* a, void* buf, int n, int S) {
    unsigned char* p = static_cast<unsigned char*>(buf);
    const size_t cf = (size_t)S * n * n, cc = (size_t)S * (n / 2) * (n / 2);
    const size_t tiles = (size_t)(n / kTile) * (n / kTile);
    a->q[0] = reinterpret_cast<int32_t*>(p); p += cf * sizeof(int32_t);
    a->q[1] = reinterpret_cast<int32_t*>(p); p += cf * sizeof(int32_t);
    a->G[0] = reinterpret_cast<int2*>(p); p += cf * sizeof(int2);
    a->G[1] = reinterpret_cast<int2*>(p); p += cf * sizeof(int2);
    a->qc[0] = reinterpret_cast<int32_t*>(p); p += cc * sizeof(int32_t);
    a->qc[1] = reinterpret_cast<int32_t*>(p); p += cc * sizeof(int32_t);
    a->Gc = reinterpret_cast<int2*>(p); p += cc * sizeof(int2);
    a->zt = reinterpret_cast<float2*>(p); p += cc * sizeof(float2);
    a->tile_part = reinterpret_cast<double*>(p);
    (void)tiles;
}

cudaError_t stream_run(const KArgs& k, SArgs a, int S, cudaStream_t st) {
    // k.partials holds S slots (entry-major, [stride][S]); zero them, run the
    // waves of S samples, accumulate per slot, then the caller reduces.
    const int n = a.n;
    if (n % kTile != 0 || (a.coupled && (a.nc % kTile != 0 || a.M % 4 != 0))) return cudaErrorInvalidValue;
    const int tiles = (n / kTile) * (n / kTile);
    const int ctiles = a.coupled ? (a.nc / kTile) * (a.nc / kTile) : 0;
    zero_kernel<<<64, 256, 0, st>>>(k.partials, (size_t)k.slot_stride * S);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (long long done = 0; done < k.count; done += S) {
        a.sid0 = k.first + done;
        a.count = (int)std::min<long long>(S, k.count - done);
        const dim3 grid(tiles, a.count), cgrid(ctiles, a.count);
        stream_init_kernel<<<grid, kThreads, 0, st>>>(a);
        for (int m = 0; m < a.M; ++m) {
            stream_fine_kernel<<<grid, kThreads, 0, st>>>(a, m);
            if (a.coupled && (m & 3) == 2) stream_coarse_kernel<<<cgrid, kThreads, 0, st>>>(a, m >> 2);
        }
        stream_observe_kernel<<<grid, kThreads, 0, st>>>(a);
        stream_finish_kernel<<<(a.count + 63) / 64, 64, 0, st>>>(a, k, tiles, S);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace dk
