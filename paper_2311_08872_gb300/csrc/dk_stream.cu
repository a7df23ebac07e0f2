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
// boundaries order all reads and writes; in the default build the fine steps
// are programmatic dependent launches that draw their noise before waiting
// for the previous kernel.
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
constexpr int kStreamVariants = 6;
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

__device__ __forceinline__ uint4 pair_words(const SArgs& a, uint32_t p, int m, uint32_t c2, uint32_t c3) {
    return philox10(make_uint4(p, static_cast<uint32_t>(m), c2, c3), a.key0, a.key1);
}

// Box--Muller radii and directions of the pair's two cells.
struct PairNormals {
    float ra, ca, sa, rb, cb, sb;
};

__device__ __forceinline__ PairNormals pair_normals(uint4 x) {
    PairNormals z;
    box_muller_polar(x.x, x.y, z.ra, z.ca, z.sa);
    box_muller_polar(x.z, x.w, z.rb, z.cb, z.sb);
    return z;
}

// Makes the normals exist at this point of the program (an empty asm
// statement that reads and writes them): the compiler keeps their arithmetic
// before a later volatile asm statement such as the grid dependency wait.
__device__ __forceinline__ void pin(PairNormals& z) {
    asm volatile("" : "+f"(z.ra), "+f"(z.ca), "+f"(z.sa), "+f"(z.rb), "+f"(z.cb), "+f"(z.sb));
}

// The transfers from the pair's normals (drawn earlier).
__device__ __forceinline__ PairNoise pair_noise_n(const SArgs& a, const PairNormals& z, int32_t qa, int32_t qb,
                                                  float& z1, float& z2) {
    const float ta = noise_amp(qa, a.gf) * z.ra, tb = noise_amp(qb, a.gf) * z.rb;
    z1 = fmaf(z.rb, z.cb, fmaf(z.ra, z.ca, z1));
    z2 = fmaf(z.rb, z.sb, fmaf(z.ra, z.sa, z2));
    return {__float2int_rn(ta * z.ca), __float2int_rn(ta * z.sa), __float2int_rn(tb * z.cb),
            __float2int_rn(tb * z.sb)};
}


// Programmatic dependent launch: let the next kernel in the stream start its
// CTAs once every CTA of this one has started, and wait until the previous
// kernel has finished and its stores are visible.
__device__ __forceinline__ void launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void wait_previous_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

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

// Loads of the state: through L1 (one launch per step: kernel boundaries
// order every access), or from L2 only (persistent launch: tiles of other
// CTAs change between this CTA's items).
template <bool CG, typename T>
__device__ __forceinline__ T ldg(const T* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// Fine step m of the FR x 64 tile at (R0, C0) of sample s: noise of step m on
// the tile and its halo, then q^{m+1}.  Thread (tx, ty) of the 16 x FR/2
// threads owns the 2 x 4 fine block at (R0 + 2 ty, C0 + 4 tx) = 2 coarse cells.
// The barrier between the shared-memory writes and reads also decides, in the
// persistent kernel, whether any warp's wait timed out (`stop`): then no thread
// stores and the function returns true.
// With PDL (one launch per step, launched as a programmatic dependent of the
// previous kernel in the stream) the Philox words of the tile and its halo,
// which depend on no state, are drawn before the wait for the previous step:
// CTAs that start while the previous step's last wave still runs do that part
// of their work in its shadow.
template <int FR, bool PERSIST, bool PDL = false>
__device__ __forceinline__ bool fine_tile(const SArgs& a, int s, int R0, int C0, int m, int32_t* smem, int stop) {
    constexpr int kHaloPairs = 64 + 2 * FR;   // 2 x 32 pairs in the halo rows, one per row in the halo columns
    static_assert(!(PDL && PERSIST), "the persistent launch has no previous grid to wait for");
    const int n = a.n;
    const int t = threadIdx.x;
    const int tx = t % 16, ty = t / 16;
    const int r0 = R0 + 2 * ty, c0 = C0 + 4 * tx;
    const size_t base = (size_t)s * n * n;
    const int32_t* qin = a.q[m & 1] + base;
    int32_t* qout = a.q[(m + 1) & 1] + base;
    uint32_t c2, c3;
    sample_counter(a, s, c2, c3);
    // halo cell pair of this thread (t < kHaloPairs): row halo (t < 64) or column halo
    int hr = 0, hc = 0;
    auto halo_cell = [&]() {
        if (t < 64) {
            hr = wrapi((t >> 5) ? R0 + FR : R0 - 1, n);
            hc = C0 + 2 * (t & 31);
        } else {
            const int u = t - 64;
            hr = R0 + u % FR;
            hc = wrapi(u / FR ? C0 + kFC : C0 - 2, n);
        }
    };
    PairNormals w[2][2], hw{};
    if constexpr (PDL) {
        if (t < kHaloPairs) halo_cell();
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const uint32_t p = static_cast<uint32_t>(((r0 + i) * n + c0) >> 1);
            w[i][0] = pair_normals(pair_words(a, p, m, c2, c3));
            w[i][1] = pair_normals(pair_words(a, p + 1, m, c2, c3));
        }
        if (t < kHaloPairs) hw = pair_normals(pair_words(a, static_cast<uint32_t>((hr * n + hc) >> 1), m, c2, c3));
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            pin(w[i][0]);
            pin(w[i][1]);
        }
        pin(hw);
        wait_previous_grid();
    }

    int32_t (*sq)[kFW] = reinterpret_cast<int32_t (*)[kFW]>(smem);
    int32_t (*s1)[kFW] = reinterpret_cast<int32_t (*)[kFW]>(smem + (FR + 2) * kFW);
    int32_t (*s2)[kFW] = reinterpret_cast<int32_t (*)[kFW]>(smem + 2 * (FR + 2) * kFW);

    // own 2x4 block: state, normals of step m, transfers; coupled sums of its
    // two coarse cells in the register kernels' order
    const int lr0 = 2 * ty + 1, lc0 = 4 * tx + 4;
    int32_t q[2][4], G1[2][4], G2[2][4];
    float4* const zp = reinterpret_cast<float4*>(a.zt + (size_t)s * a.nc * a.nc + (size_t)(r0 >> 1) * a.nc + (c0 >> 1));
    float z[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    if (a.coupled && (m & 3) != 0) {
        const float4 v = ldg<PERSIST>(zp);
        z[0][0] = v.x; z[0][1] = v.y; z[1][0] = v.z; z[1][1] = v.w;
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int4 v = ldg<PERSIST>(reinterpret_cast<const int4*>(qin + (size_t)(r0 + i) * n + c0));
        q[i][0] = v.x; q[i][1] = v.y; q[i][2] = v.z; q[i][3] = v.w;
        const uint32_t p = static_cast<uint32_t>(((r0 + i) * n + c0) >> 1);
        if constexpr (!PDL) {
            w[i][0] = pair_normals(pair_words(a, p, m, c2, c3));
            w[i][1] = pair_normals(pair_words(a, p + 1, m, c2, c3));
        }
        const PairNoise g = pair_noise_n(a, w[i][0], v.x, v.y, z[0][0], z[0][1]);
        const PairNoise h = pair_noise_n(a, w[i][1], v.z, v.w, z[1][0], z[1][1]);
        G1[i][0] = g.g1a; G2[i][0] = g.g2a; G1[i][1] = g.g1b; G2[i][1] = g.g2b;
        G1[i][2] = h.g1a; G2[i][2] = h.g2a; G1[i][3] = h.g1b; G2[i][3] = h.g2b;
        if constexpr (!PERSIST) {
            *reinterpret_cast<int4*>(&sq[lr0 + i][lc0]) = v;
            *reinterpret_cast<int4*>(&s1[lr0 + i][lc0]) = make_int4(g.g1a, g.g1b, h.g1a, h.g1b);
            *reinterpret_cast<int4*>(&s2[lr0 + i][lc0]) = make_int4(g.g2a, g.g2b, h.g2a, h.g2b);
        }
    }
    // halo: rows R0-1 and R0+FR (32 pairs each: state and G1), columns C0-1
    // and C0+kFC (one pair per row: state and G2 of the cell next to the tile);
    // (hq, hg): the state and transfer a halo thread stores
    int32_t* hq = nullptr;
    int32_t* hg = nullptr;
    int2 hqv = make_int2(0, 0), hgv = make_int2(0, 0);
    bool hpair = false;
    if (t < kHaloPairs) {
        float d1 = 0.f, d2 = 0.f;   // halo normals do not enter this tile's coarse sums
        if (t < 64) {
            const int side = t >> 5, k = t & 31;
            const int r = PDL ? hr : wrapi(side ? R0 + FR : R0 - 1, n), c = PDL ? hc : C0 + 2 * k;
            const int2 v = ldg<PERSIST>(reinterpret_cast<const int2*>(qin + (size_t)r * n + c));
            const PairNormals x = PDL ? hw : pair_normals(pair_words(a, static_cast<uint32_t>((r * n + c) >> 1), m, c2, c3));
            const PairNoise g = pair_noise_n(a, x, v.x, v.y, d1, d2);
            const int lr = side ? FR + 1 : 0;
            if constexpr (PERSIST) {
                hq = &sq[lr][4 + 2 * k];
                hg = &s1[lr][4 + 2 * k];
                hqv = v;
                hgv = make_int2(g.g1a, g.g1b);
                hpair = true;
            } else {
                *reinterpret_cast<int2*>(&sq[lr][4 + 2 * k]) = v;
                *reinterpret_cast<int2*>(&s1[lr][4 + 2 * k]) = make_int2(g.g1a, g.g1b);
            }
        } else {
            const int u = t - 64, side = u / FR, rr = u % FR;
            const int r = PDL ? hr : R0 + rr, c = PDL ? hc : wrapi(side ? C0 + kFC : C0 - 2, n);
            const int2 v = ldg<PERSIST>(reinterpret_cast<const int2*>(qin + (size_t)r * n + c));
            const PairNormals x = PDL ? hw : pair_normals(pair_words(a, static_cast<uint32_t>((r * n + c) >> 1), m, c2, c3));
            const PairNoise g = pair_noise_n(a, x, v.x, v.y, d1, d2);
            if constexpr (PERSIST) {
                hq = side ? &sq[rr + 1][kFC + 4] : &sq[rr + 1][3];
                hg = side ? &s2[rr + 1][kFC + 4] : &s2[rr + 1][3];
                hqv.x = side ? v.x : v.y;
                hgv.x = side ? g.g2a : g.g2b;
            } else if (side) {
                sq[rr + 1][kFC + 4] = v.x;
                s2[rr + 1][kFC + 4] = g.g2a;
            } else {
                sq[rr + 1][3] = v.y;
                s2[rr + 1][3] = g.g2b;
            }
        }
    }
    if constexpr (PERSIST) {
        // shared memory is free once every warp has finished the previous item
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            *reinterpret_cast<int4*>(&sq[lr0 + i][lc0]) = make_int4(q[i][0], q[i][1], q[i][2], q[i][3]);
            *reinterpret_cast<int4*>(&s1[lr0 + i][lc0]) = make_int4(G1[i][0], G1[i][1], G1[i][2], G1[i][3]);
            *reinterpret_cast<int4*>(&s2[lr0 + i][lc0]) = make_int4(G2[i][0], G2[i][1], G2[i][2], G2[i][3]);
        }
        if (t < kHaloPairs) {
            if (hpair) {
                *reinterpret_cast<int2*>(hq) = hqv;
                *reinterpret_cast<int2*>(hg) = hgv;
            } else {
                *hq = hqv.x;
                *hg = hgv.x;
            }
        }
        if (__syncthreads_or(stop)) return true;
    } else {
        __syncthreads();
    }

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
    return false;
}

// Coarse step cn (after fine step 4 cn + 3) of the 32 x 32 coarse tile
// (T1, T2) of sample s: transfers from qc^cn and the coupled sums on the tile
// and its halo (no corners: the stencil does not use them), then qc^{cn+1}.
template <bool PERSIST>
__device__ __forceinline__ void coarse_tile(const SArgs& a, int s, int T1, int T2, int cn, int32_t* smem) {
    const int nc = a.nc;
    const size_t base = (size_t)s * nc * nc;
    const int32_t* qin = a.qc[cn & 1] + base;
    int32_t* qout = a.qc[(cn + 1) & 1] + base;
    const float2* zt = a.zt + base;
    int32_t (*sq)[kTile + 2] = reinterpret_cast<int32_t (*)[kTile + 2]>(smem);
    int2 (*sg)[kTile + 2] = reinterpret_cast<int2 (*)[kTile + 2]>(smem + (kTile + 2) * (kTile + 2));
    const int R0 = T1 * kTile, C0 = T2 * kTile;
    for (int k = threadIdx.x; k < (kTile + 2) * (kTile + 2); k += kThreads) {
        const int lr = k / (kTile + 2), lc = k % (kTile + 2);
        if ((lr == 0 || lr == kTile + 1) && (lc == 0 || lc == kTile + 1)) continue;
        const int gr = wrapi(R0 + lr - 1, nc), gcol = wrapi(C0 + lc - 1, nc);
        const int32_t qv = ldg<PERSIST>(qin + (size_t)gr * nc + gcol);
        const float2 z = ldg<PERSIST>(zt + (size_t)gr * nc + gcol);
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

// One launch per fine step m (PDL: launched as a programmatic dependent of the
// previous kernel, which it waits for after drawing its Philox words).
template <int FR, int MINB, bool PDL>
__global__ void __launch_bounds__(fine_threads(FR), MINB) stream_fine_kernel(const SArgs a, int m) {
    if constexpr (PDL) launch_dependents();
    const int s = blockIdx.z;
    if (s >= a.count) return;
    extern __shared__ __align__(16) int32_t smem_fine[];
    fine_tile<FR, false, PDL>(a, s, blockIdx.y * FR, blockIdx.x * kFC, m, smem_fine, 0);
}

// One launch per coarse step cn (after fine step 4 cn + 3).  It lets the next
// fine step's CTAs start early; launched as a dependent launch itself (with the
// dependent fine steps), its CTAs are placed while the fine step's last wave
// runs and wait there for it to finish.
__global__ void __launch_bounds__(kThreads) stream_coarse_kernel(const SArgs a, int cn) {
    launch_dependents();
    wait_previous_grid();
    const int s = blockIdx.y;
    if (s >= a.count) return;
    __shared__ __align__(16) int32_t smem_coarse[(kTile + 2) * (kTile + 2) * 3];
    const int tpr = a.nc / kTile;
    coarse_tile<false>(a, s, blockIdx.x / tpr, blockIdx.x % tpr, cn, smem_coarse);
}

// ---------------------------------------------------------------------------
// Persistent launch: all fine and coarse steps of a wave in one grid of
// resident CTAs.  Work items are taken in a fixed order from a counter:
//   for every coarse step cn: fine steps 4cn .. 4cn+3 (each: every tile of
//   every sample), then the coarse step cn (every coarse tile of every sample)
// (uncoupled: the fine steps only).  An item waits until the items it reads
// from are done, which are always earlier items: a fine tile at step m needs
// itself and its four neighbours at step m (their step m-1 done: q^m written
// and q^{m-1}, which step m overwrites, read); at m = 4cn+4 also the coarse
// tiles whose halo reads its coupled sums done with step cn.  A coarse tile at
// step cn needs the fine tiles under it and its halo done with fine step
// 4cn+3, and itself and its four neighbours done with coarse step cn-1.
// Every earlier item is held by a running CTA, so the waits end; each is
// still bounded (`wait_polls` polls), after which the kernel records
// kErrTimeout, every CTA stops at its next item, and the host reports it.
// Progress: fdone[s][tile] = 8 x fine steps done, cdone[s][ctile] = 8 x coarse
// steps done: each of an item's 8 warps adds 1 with a release after its own
// stores, so no CTA-wide barrier ends an item.  Shared memory is reused only
// after a barrier that follows the next item's noise (every warp is then past
// the previous item's reads).
// ---------------------------------------------------------------------------
constexpr unsigned kItemWarps = fine_threads(kFR) / 32;   // warps of a persistent CTA (also the coarse tiles')
static_assert(fine_threads(kFR) == kThreads, "coarse tiles run on the fine-step CTAs");

struct ItemMap {
    int tr, tc;              // fine tiles per column / row of the grid (n/FR, n/64)
    int ct;                  // coarse tiles per side (nc/32)
    long long F, C, P;       // fine items per step, coarse items per coarse step, items per period
};

__device__ __forceinline__ ItemMap item_map(const SArgs& a, int fr) {
    ItemMap im;
    im.tr = a.n / fr;
    im.tc = a.n / kFC;
    im.ct = a.coupled ? a.nc / kTile : 0;
    im.F = (long long)a.count * im.tr * im.tc;
    im.C = (long long)a.count * im.ct * im.ct;
    im.P = a.coupled ? 4 * im.F + im.C : im.F;
    return im;
}

// Item k -> kind (0 fine, 1 coarse), sample, tile coordinates, step.
struct Item {
    int kind, s, i, j, step;
};

__device__ __forceinline__ Item decode_item(const ItemMap& im, long long k, bool coupled) {
    Item it;
    const long long p = k / im.P, r = k - p * im.P;
    if (!coupled || r < 4 * im.F) {
        const long long q = coupled ? r / im.F : 0, f = coupled ? r - q * im.F : r;
        it.kind = 0;
        it.step = coupled ? (int)(4 * p + q) : (int)p;
        const long long per = (long long)im.tr * im.tc;
        it.s = (int)(f / per);
        const int t = (int)(f - it.s * per);
        it.i = t / im.tc;
        it.j = t - it.i * im.tc;
    } else {
        const long long c = r - 4 * im.F, per = (long long)im.ct * im.ct;
        it.kind = 1;
        it.step = (int)p;
        it.s = (int)(c / per);
        const int t = (int)(c - it.s * per);
        it.i = t / im.ct;
        it.j = t - it.i * im.ct;
    }
    return it;
}

__device__ __forceinline__ int wrapt(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Dependency d (0 .. 12) of an item: the counter to read and the value it must
// reach; false when the item has fewer dependencies.  Fine tiles are FR = 32
// rows high, so fine tile rows 2I and 2I+1 lie under coarse tile row I.
__device__ __forceinline__ bool item_dep(const SArgs& a, const ItemMap& im, const Item& it, int d,
                                         const unsigned*& ptr, unsigned& target) {
    const unsigned* fd = a.fdone + (size_t)it.s * im.tr * im.tc;
    const unsigned* cd = a.cdone + (size_t)it.s * im.ct * im.ct;
    if (it.kind == 0) {
        if (d < 5) {
            const int di = d == 1 ? -1 : (d == 2 ? 1 : 0), dj = d == 3 ? -1 : (d == 4 ? 1 : 0);
            ptr = fd + (size_t)wrapt(it.i + di, im.tr) * im.tc + wrapt(it.j + dj, im.tc);
            target = kItemWarps * (unsigned)it.step;
            return true;
        }
        if (!a.coupled || it.step < 4 || (it.step & 3) != 0 || d >= 9) return false;
        const int I = it.i >> 1, J = it.j;
        int ci = I, cj = J;
        if (d == 6) cj = wrapt(J - 1, im.ct);
        else if (d == 7) cj = wrapt(J + 1, im.ct);
        else if (d == 8) ci = wrapt((it.i & 1) ? I + 1 : I - 1, im.ct);
        ptr = cd + (size_t)ci * im.ct + cj;
        target = kItemWarps * (unsigned)(it.step >> 2);
        return true;
    }
    if (d < 8) {
        // fine tiles: rows 2I-1 .. 2I+2 in column J (d = 0..3), rows 2I, 2I+1
        // in column J-1 (d = 4, 5) and in column J+1 (d = 6, 7)
        const int dr = d < 4 ? d - 1 : (d & 1), dc = d < 4 ? 0 : (d < 6 ? -1 : 1);
        ptr = fd + (size_t)wrapt(2 * it.i + dr, im.tr) * im.tc + wrapt(it.j + dc, im.tc);
        target = kItemWarps * (unsigned)(4 * it.step + 4);
        return true;
    }
    if (d < 13) {
        const int e = d - 8;
        const int di = e == 1 ? -1 : (e == 2 ? 1 : 0), dj = e == 3 ? -1 : (e == 4 ? 1 : 0);
        ptr = cd + (size_t)wrapt(it.i + di, im.ct) * im.ct + wrapt(it.j + dj, im.ct);
        target = kItemWarps * (unsigned)it.step;
        return true;
    }
    return false;
}

template <int FR, int MINB>
__global__ void __launch_bounds__(fine_threads(FR), MINB) stream_persist_kernel(const SArgs a) {
    static_assert(FR == 32, "coarse tiles cover two fine tile rows");
    extern __shared__ __align__(16) int32_t smem_fine[];
    __shared__ long long s_item[2];
    const ItemMap im = item_map(a, FR);
    const long long total = a.coupled ? (long long)(a.M / 4) * im.P : (long long)a.M * im.P;
    const int lane = threadIdx.x & 31;
    // the last thread takes items from the counter: its warp has no halo
    // cells, so the atomic's latency falls where that warp waits anyway
    const bool taker = threadIdx.x == blockDim.x - 1;
    if (taker) s_item[0] = (long long)atomicAdd(a.head, 1ull);
    __syncthreads();
    for (int iter = 0;; ++iter) {
        const long long k = s_item[iter & 1];
        if (k >= total) break;
        // the next item, taken now so that its latency hides behind this one
        if (taker) {
            const long long nk = (long long)atomicAdd(a.head, 1ull);
            const unsigned err = ld_volatile(a.err);
            s_item[(iter + 1) & 1] = (err & kErrTimeout) ? total : nk;
        }
        const Item it = decode_item(im, k, a.coupled != 0);
        // every warp waits for the item's dependencies itself (lane d polls
        // dependency d), so its loads are ordered after the acquires
        int stop = 0;
        {
            const unsigned* ptr = nullptr;
            unsigned target = 0;
            bool ok = true;
            if (item_dep(a, im, it, lane, ptr, target)) {
                ok = false;
                for (unsigned poll = 0; poll < a.wait_polls; ++poll) {
                    if (static_cast<int>(ld_acquire(ptr) - target) >= 0) {
                        ok = true;
                        break;
                    }
                    if ((poll & 63u) == 63u && (ld_volatile(a.err) & kErrTimeout)) break;
                    __nanosleep(64);
                }
                if (!ok) atomicOr(a.err, kErrTimeout);
            }
            stop = __any_sync(0xffffffffu, !ok) ? 1 : 0;
            __syncwarp();
        }
        if (it.kind == 0) {
            if (fine_tile<FR, true>(a, it.s, it.i * FR, it.j * kFC, it.step, smem_fine, stop)) break;
        } else {
            if (__syncthreads_or(stop)) break;   // also frees shared memory
            coarse_tile<true>(a, it.s, it.i, it.j, it.step, smem_fine);
        }
        // this warp's stores are done: report them (the failure-detection test
        // withholds step 1 of one tile of sample 0)
        __syncwarp();
        const bool stall = it.kind == 0 && a.stall_tile >= 0 && it.step == 1 && it.s == 0 &&
                           it.i * im.tc + it.j == a.stall_tile;
        if (lane == 0 && !stall) {
            unsigned* ctr = it.kind == 0 ? a.fdone + (size_t)it.s * im.tr * im.tc + (size_t)it.i * im.tc + it.j
                                         : a.cdone + (size_t)it.s * im.ct * im.ct + (size_t)it.i * im.ct + it.j;
            red_release_add(ctr, 1u);
        }
    }
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

// Progress counters of the persistent launch: fdone [S][fine tiles], cdone
// [S][coarse tiles], then the item counter (8 bytes).
static size_t counter_bytes(int n, int S) {
    const size_t ft = (size_t)(n / kFR) * (n / kFC), ct = (size_t)(n / 2 / kTile) * (n / 2 / kTile);
    return (((size_t)S * (ft + ct) * sizeof(unsigned) + 15) & ~(size_t)15) + 16;
}

size_t stream_bytes(int n, int S) {
    const size_t nc = n / 2, tiles = (size_t)(n / kTile) * (n / kTile);
    return (size_t)S * ((size_t)n * n * 2 * sizeof(int32_t) + nc * nc * (2 * sizeof(int32_t) + sizeof(float2)) +
                        tiles * (2 * kMaxObs + 2) * sizeof(double)) +
           counter_bytes(n, S);
}

int stream_variant_count() { return kStreamVariants; }
int stream_default_variant() { return 4; }   // one programmatic dependent launch per step, 4 CTAs per SM

// Variants: 0, 1 one launch per step, 2, 3 the persistent launch, 4, 5 one
// launch per step as programmatic dependent launches; even: at most 64
// registers per thread (4 resident CTAs per SM), odd: 48 (5 CTAs).
static bool persistent_variant(int variant) { return variant == 2 || variant == 3; }
static bool pdl_variant(int variant) { return variant >= 4; }

template <typename K>
static cudaError_t fine_attr_occ(K kernel, int* per_sm) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, fine_smem(kFR));
    if (e != cudaSuccess) return e;
    return per_sm ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kernel, fine_threads(kFR), fine_smem(kFR))
                  : cudaSuccess;
}

static cudaError_t fine_attr(int variant, int* per_sm = nullptr) {
    switch (variant) {
        case 0: return fine_attr_occ(stream_fine_kernel<kFR, 4, false>, per_sm);
        case 1: return fine_attr_occ(stream_fine_kernel<kFR, 5, false>, per_sm);
        case 2: return fine_attr_occ(stream_persist_kernel<kFR, 4>, per_sm);
        case 3: return fine_attr_occ(stream_persist_kernel<kFR, 5>, per_sm);
        case 4: return fine_attr_occ(stream_fine_kernel<kFR, 4, true>, per_sm);
        case 5: return fine_attr_occ(stream_fine_kernel<kFR, 5, true>, per_sm);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t stream_variant_info(int n, int variant, VariantInfo* out) {
    if (variant < 0 || variant >= kStreamVariants) return cudaErrorInvalidValue;
    const int fr = kFR;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e;
    if ((e = fine_attr(variant, &per_sm)) != cudaSuccess) return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
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
    out->persistent = persistent_variant(variant) ? 1 : 0;
    out->pdl = pdl_variant(variant) ? 1 : 0;
    return cudaSuccess;
}

int stream_inflight(int n, size_t budget, int variant) {
    // the largest count that fits the budget, lowered while a smaller count
    // fills the last wave of fine-step CTAs clearly better
    const int s_max = (int)std::max<size_t>(1, budget / stream_bytes(n, 1));
    VariantInfo vi{};
    if (stream_variant_info(n, variant, &vi) != cudaSuccess || !vi.supported) return s_max;
    const long long resident = vi.max_ctas, ctas = (long long)(n / kFC) * (n / vi.tile_rows);
    if (vi.persistent) return s_max;   // no waves: CTAs take tiles as they free up
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
    p += (size_t)S * (n / kTile) * (n / kTile) * (2 * kMaxObs + 2) * sizeof(double);
    a->counters = p;
    a->counter_bytes = counter_bytes(n, S);
    const size_t ft = (size_t)(n / kFR) * (n / kFC);
    a->fdone = reinterpret_cast<unsigned*>(p);
    a->cdone = a->fdone + (size_t)S * ft;
    a->head = reinterpret_cast<unsigned long long*>(p + a->counter_bytes - 16);
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
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = fine_attr(variant, &per_sm);
    if (e != cudaSuccess) return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (a.wait_polls == 0) a.wait_polls = 1u << 24;
    zero_kernel<<<64, 256, 0, st>>>(k.partials, (size_t)k.slot_stride * S);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (long long done = 0; done < k.count; done += S) {
        a.sid0 = k.first + done;
        a.count = (int)std::min<long long>(S, k.count - done);
        const dim3 grid(tiles, a.count), cgrid(ctiles, a.count), fgrid(n / kFC, n / fr, a.count);
        stream_init_kernel<<<grid, kThreads, 0, st>>>(a);
        if (persistent_variant(variant)) {
            // one grid of resident CTAs (at most one per item) takes the items in order
            if ((e = cudaMemsetAsync(a.counters, 0, a.counter_bytes, st)) != cudaSuccess) return e;
            const long long items = (long long)a.count * (n / fr) * (n / kFC) * a.M +
                                    (a.coupled ? (long long)a.count * ctiles * (a.M / 4) : 0);
            const int ctas = (int)std::min<long long>((long long)sms * per_sm, items);
            if (variant == 2)
                stream_persist_kernel<kFR, 4><<<ctas, fine_threads(kFR), fine_smem(kFR), st>>>(a);
            else
                stream_persist_kernel<kFR, 5><<<ctas, fine_threads(kFR), fine_smem(kFR), st>>>(a);
        } else if (pdl_variant(variant)) {
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            cudaLaunchConfig_t cfg{};
            cfg.gridDim = fgrid;
            cfg.blockDim = dim3(fine_threads(kFR));
            cfg.dynamicSmemBytes = fine_smem(kFR);
            cfg.stream = st;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            cudaLaunchConfig_t ccfg = cfg;
            ccfg.gridDim = cgrid;
            ccfg.blockDim = dim3(kThreads);
            ccfg.dynamicSmemBytes = 0;
            for (int m = 0; m < a.M; ++m) {
                e = variant == 4 ? cudaLaunchKernelEx(&cfg, stream_fine_kernel<kFR, 4, true>, a, m)
                                 : cudaLaunchKernelEx(&cfg, stream_fine_kernel<kFR, 5, true>, a, m);
                if (e == cudaSuccess && a.coupled && (m & 3) == 3)
                    e = cudaLaunchKernelEx(&ccfg, stream_coarse_kernel, a, m >> 2);
                if (e != cudaSuccess) return e;
            }
        } else {
            for (int m = 0; m < a.M; ++m) {
                if (variant == 0)
                    stream_fine_kernel<kFR, 4, false><<<fgrid, fine_threads(kFR), fine_smem(kFR), st>>>(a, m);
                else
                    stream_fine_kernel<kFR, 5, false><<<fgrid, fine_threads(kFR), fine_smem(kFR), st>>>(a, m);
                if (a.coupled && (m & 3) == 3) stream_coarse_kernel<<<cgrid, kThreads, 0, st>>>(a, m >> 2);
            }
        }
        stream_observe_kernel<<<grid, kThreads, 0, st>>>(a);
        stream_finish_kernel<<<(a.count + 63) / 64, 64, 0, st>>>(a, k, tiles, S);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace dk
