// Band kernels: the coupled sample of a large grid (n = 128 .. 1024) spread
// over several CTAs, each holding a full-width band of coarse rows in
// registers for the whole run.
//
// The scheme, the noise counters and the integer arithmetic are those of the
// register kernels (Eq. FullyDiscreteDK with b0 = 0, b1 = 1; Right-Most NN
// coupling of Section 3.2): a thread owns a 4 x 4 block of fine cells (2 x 2
// coarse cells), draws the Philox normals of its eight cell pairs, sums the
// coupled coarse normals of its coarse cells in the same order, and applies
// the same edge fluxes and transfers, so the fine and coarse states agree with
// theirs bit for bit.
//
// Layout.  A warp covers 128 fine columns of four fine rows (a row-quad); WPR =
// n / 128 warps cover a row-quad, and a CTA holds a band of up to 16 / WPR
// row-quads.  Within a CTA the row-quads exchange their first and last fine
// rows through shared memory (double-buffered by step parity, one barrier per
// fine step) and the columns by warp shuffles (and shared memory between the
// warps of a row-quad).  Between bands the band's top and bottom fine rows
// (state and vertical transfer) and, on coarse steps, its top and bottom coarse
// rows go through global memory: the band's edge warps draw the noise of their
// edge rows first, write them, then add to a per-band counter with release
// semantics, so the neighbouring band's edge warps, which wait (acquire,
// bounded) for that counter only after the rest of their step's noise and the
// update of their inner rows, rarely wait at all.  No CTA waits for anything
// but its two neighbouring bands' counters, so the bands of a sample must be
// resident together: the grid is launched cooperatively.  Every wait gives up
// after a fixed number of polls (or as soon as another CTA has given up),
// records kErrTimeout in the error word and makes its CTA stop stepping, so a
// kernel never spins without end.
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "dk_device.cuh"
#include "dk_kernels.h"

namespace dk {

namespace {

constexpr int kW = 2 * kMaxObs + 2;              // per-band observable partials
constexpr unsigned kWaitPolls = 1u << 22;         // polls of one wait before it gives up

// Launch shape of a band kernel build: a thread owns 4 fine rows x FC fine
// columns; a warp covers 32 FC columns, WPR warps a row-quad of the n x n grid.
template <int NF_, int FC_>
struct BShape {
    static constexpr int NF = NF_, FC = FC_, CC = FC_ / 2;
    static constexpr int NC = NF / 2, NQ = NF / 4;
    static constexpr int WPR = NF / (32 * FC);
    static constexpr int MAXT = FC == 4 ? 512 : 256;   // threads of the tallest band (registers: 128 / 255)
    static_assert(WPR >= 1 && NF % (32 * FC) == 0, "a warp covers 32 FC columns of the grid");
};

// Wait until *flag >= target (counters only grow).  Returns false after
// `polls` polls, or as soon as another CTA has recorded a timeout.
__device__ bool wait_counter(const unsigned* flag, unsigned target, unsigned* err, unsigned polls) {
    for (unsigned it = 0; it < polls; ++it) {
        if (static_cast<int>(ld_acquire(flag) - target) >= 0) return true;
        if ((it & 63u) == 63u && (ld_volatile(err) & kErrTimeout)) return false;
        __nanosleep(32);
    }
    atomicOr(err, kErrTimeout);
    return false;
}

// N (q, g) pairs of one lane's part of a row as N/2 16-byte words.
template <int N>
__device__ __forceinline__ void st_pairs(int2* dst, const int32_t (&q)[N], const int32_t (&g)[N]) {
    int4* d = reinterpret_cast<int4*>(dst);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) d[k] = make_int4(q[2 * k], g[2 * k], q[2 * k + 1], g[2 * k + 1]);
}

template <int N>
__device__ __forceinline__ void ld_pairs(const int2* src, int32_t (&q)[N], int32_t (&g)[N]) {
    const int4* s = reinterpret_cast<const int4*>(src);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
        const int4 a = s[k];
        q[2 * k] = a.x; g[2 * k] = a.y; q[2 * k + 1] = a.z; g[2 * k + 1] = a.w;
    }
}

// The same from global memory through L2 (another SM wrote it).
template <int N>
__device__ __forceinline__ void ldcg_pairs(const int2* src, int32_t (&q)[N], int32_t (&g)[N]) {
    const int4* s = reinterpret_cast<const int4*>(src);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
        const int4 a = __ldcg(s + k);
        q[2 * k] = a.x; g[2 * k] = a.y; q[2 * k + 1] = a.z; g[2 * k + 1] = a.w;
    }
}

struct BandSmem {
    int2* sv;      // [2 parity][bmax][2 side][NF]: (q, G1) of each warp-row's first / last fine row
    int2* sh;      // [2 parity][bmax][WPR][2 side][4 row]: (q, G2) of each warp's first / last column
    int2* scv;     // [bmax][2 side][NC]: (qc, Gc1) of each warp-row's first / last coarse row (coarse steps)
    int2* sch;     // [bmax][WPR][2 side][2 row]: (qc, Gc2) of each warp's first / last coarse column
    double* red;   // [warps][kW]
    int* abort;    // [2]: set at step m in slot (m + 1) & 1, read after the barrier of step m + 1
};

template <class S>
__host__ __device__ constexpr size_t band_smem_bytes(int bmax) {
    return sizeof(int2) * (size_t)(2 * bmax * 2 * S::NF + 2 * bmax * S::WPR * 2 * 4 + bmax * 2 * S::NC +
                                   bmax * S::WPR * 2 * 2) +
           sizeof(double) * (size_t)(bmax * S::WPR * kW) + 2 * sizeof(int);
}

template <class S>
__device__ BandSmem carve(unsigned char* p, int bmax) {
    BandSmem s;
    s.sv = reinterpret_cast<int2*>(p);
    s.sh = s.sv + (size_t)2 * bmax * 2 * S::NF;
    s.scv = s.sh + (size_t)2 * bmax * S::WPR * 2 * 4;
    s.sch = s.scv + (size_t)bmax * 2 * S::NC;
    s.red = reinterpret_cast<double*>(s.sch + (size_t)bmax * S::WPR * 2 * 2);
    s.abort = reinterpret_cast<int*>(s.red + (size_t)bmax * S::WPR * kW);
    return s;
}

// Normals and transfers of fine row R of the thread's 4 x FC block at step m:
// the FC/2 Philox cell pairs of the row, Box--Muller, G1/G2; the normals are
// returned (radius, cos, sin per cell) for the coupled sums.
template <int R, int FC>
__device__ __forceinline__ void noise_row(const int32_t (&q)[4][FC], int32_t (&G1)[4][FC], int32_t (&G2)[4][FC],
                                          float (&nv)[FC / 2][6], uint32_t p0, uint32_t m, uint32_t c2, uint32_t c3,
                                          uint32_t k0, uint32_t k1, float gf) {
#pragma unroll
    for (int pc = 0; pc < FC / 2; ++pc) {
        const uint4 x = philox10(make_uint4(p0 + pc, m, c2, c3), k0, k1);
        float ra, ca, sa, rb, cb, sb;
        box_muller_polar(x.x, x.y, ra, ca, sa);
        box_muller_polar(x.z, x.w, rb, cb, sb);
        const float ta = noise_amp(q[R][2 * pc], gf) * ra;
        const float tb = noise_amp(q[R][2 * pc + 1], gf) * rb;
        G1[R][2 * pc] = __float2int_rn(ta * ca);
        G2[R][2 * pc] = __float2int_rn(ta * sa);
        G1[R][2 * pc + 1] = __float2int_rn(tb * cb);
        G2[R][2 * pc + 1] = __float2int_rn(tb * sb);
        nv[pc][0] = ra; nv[pc][1] = ca; nv[pc][2] = sa;
        nv[pc][3] = rb; nv[pc][4] = cb; nv[pc][5] = sb;
    }
}

// Add a row's normals to the coupled sums of its coarse row, in the register
// kernels' order (cell pair by cell pair, left cell first).
template <int CC>
__device__ __forceinline__ void add_zt(float (&z)[CC][2], const float (&nv)[CC][6]) {
#pragma unroll
    for (int pc = 0; pc < CC; ++pc) {
        z[pc][0] = fmaf(nv[pc][3], nv[pc][4], fmaf(nv[pc][0], nv[pc][1], z[pc][0]));
        z[pc][1] = fmaf(nv[pc][3], nv[pc][5], fmaf(nv[pc][0], nv[pc][2], z[pc][1]));
    }
}

// New values of fine row R of the block (Eq. FullyDiscreteDK with b0 = 0, in
// the register kernels' integer flux form): vertical fluxes Vu (upper edge) and
// Vd (lower edge), the row's horizontal fluxes from its own cells and the
// left / right neighbours, transfers from the rows above / below (g1u, g1d)
// and the neighbouring columns.
template <int R, int FC>
__device__ __forceinline__ void update_row(int32_t (&q)[4][FC], const int32_t (&G2)[4][FC], const int32_t (&Vu)[FC],
                                           const int32_t (&Vd)[FC], const int32_t (&g1u)[FC], const int32_t (&g1d)[FC],
                                           int32_t qL, int32_t gL, int32_t qR, int32_t gR, int32_t A) {
    int32_t nq[FC];
    int32_t hprev = edge_flux(A, q[R][0] - qL);
#pragma unroll
    for (int c = 0; c < FC; ++c) {
        const int32_t hnext = c < FC - 1 ? edge_flux(A, q[R][c + 1] - q[R][c]) : edge_flux(A, qR - q[R][FC - 1]);
        const int32_t g2r = c < FC - 1 ? G2[R][c + 1] : gR;
        const int32_t g2l = c > 0 ? G2[R][c - 1] : gL;
        nq[c] = q[R][c] + (Vd[c] - Vu[c]) + (hnext - hprev) + (g1d[c] - g1u[c]) + (g2r - g2l);
        hprev = hnext;
    }
#pragma unroll
    for (int c = 0; c < FC; ++c) q[R][c] = nq[c];
}

template <class S, bool CPL>
__global__ void __launch_bounds__(S::MAXT, 1) band_kernel(const KArgs a, const BArgs b) {
    constexpr int NF = S::NF, NC = S::NC, NQ = S::NQ, FC = S::FC, CC = S::CC, WPR = S::WPR;
    extern __shared__ __align__(16) unsigned char band_shared[];
    const BandSmem sm = carve<S>(band_shared, b.bmax);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int smp = blockIdx.x / b.nb, band = blockIdx.x % b.nb;
    if (smp >= b.count) return;   // the whole CTA (and every band of this sample) leaves together
    const int cr = warp / WPR, wc = warp % WPR;          // row-quad within the band, warp column
    const int r0 = (int)((long long)band * NQ / b.nb);
    const int B = (int)((long long)(band + 1) * NQ / b.nb) - r0;
    const bool live = cr < B;
    const bool top = cr == 0, bot = cr == B - 1;          // B >= 2: a warp-row is at most one band edge
    const int quad = r0 + (live ? cr : 0);
    const int frow = 4 * quad, crow = 2 * quad;
    const int col0 = (wc * 32 + lane) * FC, ccol0 = col0 / 2;
    const int up = (band + b.nb - 1) % b.nb, dn = (band + 1) % b.nb;
    const long long sid = b.sid0 + smp;
    const uint32_t c2 = static_cast<uint32_t>(sid);
    const uint32_t c3 = a.tag | ((static_cast<uint32_t>(static_cast<unsigned long long>(sid) >> 32) & 0xffffu) << 16);
    unsigned* const flags = b.flags + (size_t)smp * b.nb * 2;            // [band][side]
    int2* const edge = b.edge + (size_t)smp * b.nb * 2 * 2 * NF;         // [band][side][parity][NF]
    int2* const cedge = b.cedge + (size_t)smp * b.nb * 2 * NC;           // [band][side][NC]
    // pair index of the block's first cell pair in each fine row
    uint32_t prow[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) prow[r] = static_cast<uint32_t>(((frow + r) * NF + col0) >> 1);
    if (tid < 2) sm.abort[tid] = 0;

    int32_t q[4][FC], qc[2][CC];
    float zt[2][CC][2];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < FC; c += 4) {
            const int4 v = __ldg(reinterpret_cast<const int4*>(a.q0f + (size_t)(frow + r) * NF + col0 + c));
            q[r][c] = v.x; q[r][c + 1] = v.y; q[r][c + 2] = v.z; q[r][c + 3] = v.w;
        }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
#pragma unroll
        for (int j = 0; j < CC; j += 2) {
            if constexpr (CPL) {
                const int2 v = __ldg(reinterpret_cast<const int2*>(a.q0c + (size_t)(crow + i) * NC + ccol0 + j));
                qc[i][j] = v.x; qc[i][j + 1] = v.y;
            } else {
                qc[i][j] = qc[i][j + 1] = 0;
            }
        }
#pragma unroll
        for (int j = 0; j < CC; ++j) zt[i][j][0] = zt[i][j][1] = 0.f;
    }
    __syncthreads();
    unsigned bad = 0;
    const int M = b.steps;
    for (int m = 0; m < M; ++m) {
        const int par = m & 1;
        const bool cstep = CPL && ((m & 3) == 3);
        const uint32_t um = static_cast<uint32_t>(m);
        int32_t G1[4][FC], G2[4][FC], Gc1[2][CC], Gc2[2][CC];
        // coarse transfers of coarse row I once its coupled sums are complete
        auto coarse_row = [&](auto I_) {
            constexpr int I = decltype(I_)::value;
#pragma unroll
            for (int j = 0; j < CC; ++j) {
                const float amp = noise_amp(qc[I][j], a.gc);
                Gc1[I][j] = __float2int_rn(amp * zt[I][j][0]);
                Gc2[I][j] = __float2int_rn(amp * zt[I][j][1]);
                zt[I][j][0] = zt[I][j][1] = 0.f;
            }
        };
        // band edges to global memory, then the band's counter (release)
        auto publish = [&](auto SIDE_) {
            constexpr int SIDE = decltype(SIDE_)::value;   // 0: top edge (fine row 0), 1: bottom edge (fine row 3)
            constexpr int FRr = SIDE ? 3 : 0, CRr = SIDE ? 1 : 0;
            st_pairs<FC>(edge + (((size_t)band * 2 + SIDE) * 2 + par) * NF + col0, q[FRr], G1[FRr]);
            if (cstep) st_pairs<CC>(cedge + ((size_t)band * 2 + SIDE) * NC + ccol0, qc[CRr], Gc1[CRr]);
            __syncwarp();
            if (lane == 0 && band != b.stall_band) {   // stall_band: failure-detection test only
                __threadfence();
                red_release_add(flags + (size_t)band * 2 + SIDE, 1u);
            }
        };
        using I0 = std::integral_constant<int, 0>;
        using I1 = std::integral_constant<int, 1>;
        // ---- noise of step m; the band's edge rows first, published at once, so
        // that the neighbouring bands' waits overlap the rest of the step
        if (live) {
            float nv[CC][6], nv3[CC][6];
            if (bot) {
                // bottom edge: row 3's normals first (kept), row 2, then the coupled
                // sums of coarse row 1 in the register kernels' order (row 2, row 3)
                noise_row<3, FC>(q, G1, G2, nv3, prow[3], um, c2, c3, a.key0, a.key1, a.gf);
                noise_row<2, FC>(q, G1, G2, nv, prow[2], um, c2, c3, a.key0, a.key1, a.gf);
                if constexpr (CPL) {
                    add_zt(zt[1], nv);
                    add_zt(zt[1], nv3);
                    if (cstep) coarse_row(I1{});
                }
                publish(I1{});
                noise_row<0, FC>(q, G1, G2, nv, prow[0], um, c2, c3, a.key0, a.key1, a.gf);
                if constexpr (CPL) add_zt(zt[0], nv);
                noise_row<1, FC>(q, G1, G2, nv, prow[1], um, c2, c3, a.key0, a.key1, a.gf);
                if constexpr (CPL) {
                    add_zt(zt[0], nv);
                    if (cstep) coarse_row(I0{});
                }
            } else {
                noise_row<0, FC>(q, G1, G2, nv, prow[0], um, c2, c3, a.key0, a.key1, a.gf);
                if constexpr (CPL) add_zt(zt[0], nv);
                noise_row<1, FC>(q, G1, G2, nv, prow[1], um, c2, c3, a.key0, a.key1, a.gf);
                if constexpr (CPL) {
                    add_zt(zt[0], nv);
                    if (cstep) coarse_row(I0{});
                }
                if (top) publish(I0{});
                noise_row<2, FC>(q, G1, G2, nv, prow[2], um, c2, c3, a.key0, a.key1, a.gf);
                if constexpr (CPL) add_zt(zt[1], nv);
                noise_row<3, FC>(q, G1, G2, nv, prow[3], um, c2, c3, a.key0, a.key1, a.gf);
                if constexpr (CPL) {
                    add_zt(zt[1], nv);
                    if (cstep) coarse_row(I1{});
                }
            }
            // ---- the warp-row's edge rows and columns to shared memory
            st_pairs<FC>(sm.sv + (((size_t)par * b.bmax + cr) * 2 + 0) * NF + col0, q[0], G1[0]);
            st_pairs<FC>(sm.sv + (((size_t)par * b.bmax + cr) * 2 + 1) * NF + col0, q[3], G1[3]);
            if constexpr (WPR > 1) {
                int2* h = sm.sh + (((size_t)par * b.bmax + cr) * WPR + wc) * 8;
                if (lane == 0)
#pragma unroll
                    for (int r = 0; r < 4; ++r) h[r] = make_int2(q[r][0], G2[r][0]);
                if (lane == 31)
#pragma unroll
                    for (int r = 0; r < 4; ++r) h[4 + r] = make_int2(q[r][FC - 1], G2[r][FC - 1]);
            }
            if (cstep) {
                st_pairs<CC>(sm.scv + ((size_t)cr * 2 + 0) * NC + ccol0, qc[0], Gc1[0]);
                st_pairs<CC>(sm.scv + ((size_t)cr * 2 + 1) * NC + ccol0, qc[1], Gc1[1]);
                if constexpr (WPR > 1) {
                    int2* h = sm.sch + ((size_t)cr * WPR + wc) * 4;
                    if (lane == 0) { h[0] = make_int2(qc[0][0], Gc2[0][0]); h[1] = make_int2(qc[1][0], Gc2[1][0]); }
                    if (lane == 31) {
                        h[2] = make_int2(qc[0][CC - 1], Gc2[0][CC - 1]);
                        h[3] = make_int2(qc[1][CC - 1], Gc2[1][CC - 1]);
                    }
                }
            }
        }
        __syncthreads();
        if (sm.abort[par]) break;   // uniform: a wait of the previous step gave up
        if (!live) continue;

        // ---- fine update: the interior rows 1, 2 first (no halo), then the
        // band-edge warps wait for their neighbour's step-m edge, then rows 0, 3
        int32_t V[3][FC];   // fluxes across the block's inner edges (old state)
#pragma unroll
        for (int c = 0; c < FC; ++c) {
            V[0][c] = edge_flux(a.Af, q[1][c] - q[0][c]);
            V[1][c] = edge_flux(a.Af, q[2][c] - q[1][c]);
            V[2][c] = edge_flux(a.Af, q[3][c] - q[2][c]);
        }
        int32_t hq[4][2], hg[4][2];   // [row][left, right] column neighbours (old state)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            hq[r][0] = __shfl_sync(0xffffffffu, q[r][FC - 1], (lane + 31) & 31);
            hg[r][0] = __shfl_sync(0xffffffffu, G2[r][FC - 1], (lane + 31) & 31);
            hq[r][1] = __shfl_sync(0xffffffffu, q[r][0], (lane + 1) & 31);
            hg[r][1] = __shfl_sync(0xffffffffu, G2[r][0], (lane + 1) & 31);
        }
        if constexpr (WPR > 1) {
            if (lane == 0) {
                const int2* h = sm.sh + (((size_t)par * b.bmax + cr) * WPR + (wc + WPR - 1) % WPR) * 8 + 4;
#pragma unroll
                for (int r = 0; r < 4; ++r) { const int2 u = h[r]; hq[r][0] = u.x; hg[r][0] = u.y; }
            }
            if (lane == 31) {
                const int2* h = sm.sh + (((size_t)par * b.bmax + cr) * WPR + (wc + 1) % WPR) * 8;
#pragma unroll
                for (int r = 0; r < 4; ++r) { const int2 u = h[r]; hq[r][1] = u.x; hg[r][1] = u.y; }
            }
        }
        int32_t qU[FC], gU[FC], qD[FC], gD[FC];
        // row 1 and row 2 (their vertical neighbours are in the block)
        update_row<1, FC>(q, G2, V[0], V[1], G1[0], G1[2], hq[1][0], hg[1][0], hq[1][1], hg[1][1], a.Af);
        update_row<2, FC>(q, G2, V[1], V[2], G1[1], G1[3], hq[2][0], hg[2][0], hq[2][1], hg[2][1], a.Af);
        const int2* const svp = sm.sv + (size_t)par * b.bmax * 2 * NF + col0;
        if (top || bot) {
            if (lane == 0) {
                const bool ok = top ? wait_counter(flags + (size_t)up * 2 + 1, (unsigned)(WPR * (m + 1)), a.err, b.wait_polls)
                                    : wait_counter(flags + (size_t)dn * 2 + 0, (unsigned)(WPR * (m + 1)), a.err, b.wait_polls);
                if (!ok) sm.abort[par ^ 1] = 1;
            }
            __syncwarp();
        }
        if (top) ldcg_pairs<FC>(edge + (((size_t)up * 2 + 1) * 2 + par) * NF + col0, qU, gU);
        else ld_pairs<FC>(svp + ((size_t)(cr - 1) * 2 + 1) * NF, qU, gU);
        if (bot) ldcg_pairs<FC>(edge + (((size_t)dn * 2 + 0) * 2 + par) * NF + col0, qD, gD);
        else ld_pairs<FC>(svp + ((size_t)(cr + 1) * 2 + 0) * NF, qD, gD);
        {
            int32_t Vu[FC], Vd[FC];
#pragma unroll
            for (int c = 0; c < FC; ++c) {
                Vu[c] = edge_flux(a.Af, q[0][c] - qU[c]);
                Vd[c] = edge_flux(a.Af, qD[c] - q[3][c]);
            }
            update_row<0, FC>(q, G2, Vu, V[0], gU, G1[1], hq[0][0], hg[0][0], hq[0][1], hg[0][1], a.Af);
            update_row<3, FC>(q, G2, V[2], Vd, G1[2], gD, hq[3][0], hg[3][0], hq[3][1], hg[3][1], a.Af);
        }
        if (cstep) {
            // ---- coarse step: the same on the block's 2 x 2 coarse cells
            int32_t cqL[2], cgL[2], cqR[2], cgR[2], cqU[CC], cgU[CC], cqD[CC], cgD[CC];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                cqL[i] = __shfl_sync(0xffffffffu, qc[i][CC - 1], (lane + 31) & 31);
                cgL[i] = __shfl_sync(0xffffffffu, Gc2[i][CC - 1], (lane + 31) & 31);
                cqR[i] = __shfl_sync(0xffffffffu, qc[i][0], (lane + 1) & 31);
                cgR[i] = __shfl_sync(0xffffffffu, Gc2[i][0], (lane + 1) & 31);
            }
            if constexpr (WPR > 1) {
                if (lane == 0) {
                    const int2* h = sm.sch + ((size_t)cr * WPR + (wc + WPR - 1) % WPR) * 4 + 2;
                    cqL[0] = h[0].x; cgL[0] = h[0].y; cqL[1] = h[1].x; cgL[1] = h[1].y;
                }
                if (lane == 31) {
                    const int2* h = sm.sch + ((size_t)cr * WPR + (wc + 1) % WPR) * 4;
                    cqR[0] = h[0].x; cgR[0] = h[0].y; cqR[1] = h[1].x; cgR[1] = h[1].y;
                }
            }
            if (top) ldcg_pairs<CC>(cedge + ((size_t)up * 2 + 1) * NC + ccol0, cqU, cgU);
            else ld_pairs<CC>(sm.scv + ((size_t)(cr - 1) * 2 + 1) * NC + ccol0, cqU, cgU);
            if (bot) ldcg_pairs<CC>(cedge + ((size_t)dn * 2 + 0) * NC + ccol0, cqD, cgD);
            else ld_pairs<CC>(sm.scv + ((size_t)(cr + 1) * 2 + 0) * NC + ccol0, cqD, cgD);
            flux_update<2, CC>(qc, Gc1, Gc2, cqU, cgU, cqD, cgD, cqL, cgL, cqR, cgR, a.Ac);
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < CC; ++j) bad |= (static_cast<uint32_t>(qc[i][j]) + 0x40000000u) >> 31;
        }
        if ((m & 3) == 3 || m + 1 == M) {
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < FC; ++c) bad |= (static_cast<uint32_t>(q[r][c]) + 0x40000000u) >> 31;
        }
    }
    if (bad) atomicOr(a.err, kErrRange);

    // ---- observables of the band: FP64 fluctuation sums against FP64 test functions, masses
    double v[kW];
#pragma unroll
    for (int i = 0; i < kW; ++i) v[i] = 0.0;
    if (live) {
        long long mf = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < FC; ++c) mf += q[r][c];
        v[2 * kMaxObs] = static_cast<double>(mf);
#pragma unroll
        for (int k = 0; k < kMaxObs; ++k) {
            if (k >= a.n_obs) break;
            double sf = 0.0;
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < FC; ++c) {
                    const size_t x = (size_t)(frow + r) * NF + col0 + c;
                    sf = fma(static_cast<double>(q[r][c] - a.qbf[x]), b.phif64[(size_t)k * NF * NF + x], sf);
                }
            v[k] = sf;
        }
        if constexpr (CPL) {
            long long mc = 0;
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < CC; ++j) mc += qc[i][j];
            v[2 * kMaxObs + 1] = static_cast<double>(mc);
#pragma unroll
            for (int k = 0; k < kMaxObs; ++k) {
                if (k >= a.n_obs) break;
                double sc = 0.0;
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < CC; ++j) {
                        const size_t x = (size_t)(crow + i) * NC + ccol0 + j;
                        sc = fma(static_cast<double>(qc[i][j] - a.qbc[x]), b.phic64[(size_t)k * NC * NC + x], sc);
                    }
                v[kMaxObs + k] = sc;
            }
        }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
#pragma unroll
        for (int i = 0; i < kW; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < kW; ++i) sm.red[warp * kW + i] = v[i];
    __syncthreads();
    if (tid < kW) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm.red[w * kW + tid];   // fixed order
        b.band_part[((size_t)smp * b.nb + band) * kW + tid] = t;
    }
}

// Per sample of the wave: bands reduced in order, then the FP64 quantities and
// moment sums added to its slot (slot = position in the wave).
__global__ void band_finish_kernel(const KArgs k, const BArgs b, int n_slots) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.count) return;
    double v[kW];
    for (int i = 0; i < kW; ++i) v[i] = 0.0;
    for (int t = 0; t < b.nb; ++t)
        for (int i = 0; i < kW; ++i) v[i] += b.band_part[((size_t)s * b.nb + t) * kW + i];
    const bool cpl = b.coupled != 0;
    double Df[kMaxObs], Dc[kMaxObs];
    for (int q = 0; q < kMaxObs; ++q) {
        Df[q] = k.dscale_f * v[q] + k.delta_f[q];
        Dc[q] = cpl ? k.dscale_c * v[kMaxObs + q] + k.delta_c[q] : 0.0;
    }
    auto P = [&](int e) -> double& { return k.partials[(size_t)e * n_slots + s]; };
    P(0) += 1.0;
    double merr = fabs(v[2 * kMaxObs] - static_cast<double>(k.mass0_f)) * k.dscale_f;
    if (cpl) merr = fmax(merr, fabs(v[2 * kMaxObs + 1] - static_cast<double>(k.mass0_c)) * k.dscale_c);
    P(1) = fmax(P(1), merr);
    int qi = 0;
    for (int j = 0; j < k.n_obs; ++j) {
        const int kend = k.products ? k.n_obs : j + 1;
        for (int l = j; l < kend; ++l, ++qi) {
            const double pf = k.N * Df[j] * Df[l];
            const double pc = cpl ? k.N * Dc[j] * Dc[l] : 0.0;
            const double dp = pf - pc, dp2 = dp * dp;
            const int e = 2 + kNSum * qi;
            P(e + 0) += dp; P(e + 1) += dp2; P(e + 2) += dp2 * dp; P(e + 3) += dp2 * dp2;
            P(e + 4) += pf; P(e + 5) += pf * pf; P(e + 6) += pc; P(e + 7) += pc * pc;
            P(e + 8) += Df[j]; P(e + 9) += Df[j] * Df[j]; P(e + 10) += Dc[j]; P(e + 11) += Dc[j] * Dc[j];
        }
    }
    if (k.samples) {
        double* o = k.samples + (b.sid0 - k.first + s) * (2 * k.n_obs + 2);
        for (int q = 0; q < k.n_obs; ++q) {
            o[q] = Df[q];
            o[k.n_obs + q] = Dc[q];
        }
        o[2 * k.n_obs] = v[2 * kMaxObs] * k.dscale_f;
        o[2 * k.n_obs + 1] = cpl ? v[2 * kMaxObs + 1] * k.dscale_c : 0.0;
    }
}

__global__ void band_zero_kernel(double* p, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        p[i] = 0.0;
}

template <class S, bool CPL>
cudaError_t band_attr(int bmax) {
    return cudaFuncSetAttribute(band_kernel<S, CPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)band_smem_bytes<S>(bmax));
}

template <class S, bool CPL>
cudaError_t band_occupancy(int bmax, int* per_sm) {
    cudaError_t e = band_attr<S, CPL>(bmax);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, band_kernel<S, CPL>, bmax * S::WPR * 32,
                                                         band_smem_bytes<S>(bmax));
}

template <class S, bool CPL>
cudaError_t band_launch(const KArgs& a, const BArgs& b, cudaStream_t st) {
    cudaError_t e = band_attr<S, CPL>(b.bmax);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b.S * b.nb);
    cfg.blockDim = dim3(b.bmax * S::WPR * 32);
    cfg.dynamicSmemBytes = band_smem_bytes<S>(b.bmax);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, band_kernel<S, CPL>, a, b);
}

// The builds: 4 x 4 blocks (512 threads, 128 registers) for n = 128 .. 1024,
// 4 x 8 blocks (256 threads, 255 registers) for n = 256 .. 1024.
#define DK_BAND_BUILDS(X) X(128, 4) X(256, 4) X(512, 4) X(1024, 4) X(256, 8) X(512, 8) X(1024, 8)

template <class F>
cudaError_t band_dispatch(int n, int fc, bool coupled, F&& f) {
#define DK_BAND_CASE(NF, FC)                                                                   \
    if (n == NF && fc == FC)                                                                   \
        return coupled ? f(BShape<NF, FC>{}, std::true_type{}) : f(BShape<NF, FC>{}, std::false_type{});
    DK_BAND_BUILDS(DK_BAND_CASE)
#undef DK_BAND_CASE
    return cudaErrorInvalidValue;
}

}  // namespace

bool band_supported(int n, int fc) {
#define DK_BAND_HAS(NF, FC) if (n == NF && fc == FC) return true;
    DK_BAND_BUILDS(DK_BAND_HAS)
#undef DK_BAND_HAS
    return false;
}

cudaError_t band_plan(int n, bool coupled, int fc, BandPlan* out) {
    *out = BandPlan{};
    if (!band_supported(n, fc)) return cudaSuccess;
    const int wpr = n / (32 * fc), nq = n / 4, maxt = fc == 4 ? 512 : 256;
    const int rows_max = maxt / 32 / wpr;   // rows: row-quads (4 fine rows)
    if (rows_max < 1) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    // Bands per sample nb: the tallest band (ceil(nq / nb) row-quads) times the
    // CTAs an SM holds sets the time of a fine step, and S = floor(resident
    // CTAs / nb) samples run at once; pick the nb with the most samples per unit
    // of step time (ties: fewer, taller bands).
    double best = 0.0;
    for (int nb = std::max(2, (nq + rows_max - 1) / rows_max); nb <= nq / 2; ++nb) {
        const int bmax = (nq + nb - 1) / nb;
        if (bmax < 2) break;
        int per_sm = 0;
        e = band_dispatch(n, fc, coupled, [&](auto shape, auto cpl) {
            return band_occupancy<decltype(shape), decltype(cpl)::value>(bmax, &per_sm);
        });
        if (e != cudaSuccess) return e;
        const int S = per_sm * sms / nb;
        if (S < 1) continue;
        const int ctas_per_sm = (S * nb + sms - 1) / sms;
        const double rate = (double)S / ((double)ctas_per_sm * (double)bmax);
        if (rate > best * 1.0001) {
            best = rate;
            out->supported = 1;
            out->fc = fc;
            out->nb = nb;
            out->bmax = bmax;
            out->S = S;
            out->threads = bmax * wpr * 32;
        }
    }
    if (out->supported) {
        band_dispatch(n, fc, coupled, [&](auto shape, auto) {
            out->smem = band_smem_bytes<decltype(shape)>(out->bmax);
            return cudaSuccess;
        });
    }
    return cudaSuccess;
}

size_t band_bytes(int n, const BandPlan& p) {
    const size_t per = (size_t)p.nb * (2 * sizeof(unsigned) + sizeof(int2) * (2 * 2 * (size_t)n + 2 * (size_t)(n / 2)) +
                                       sizeof(double) * kW);
    return per * p.S + 256;
}

void band_carve(BArgs* b, void* buf, int n, const BandPlan& p) {
    unsigned char* q = static_cast<unsigned char*>(buf);
    const size_t ns = (size_t)p.S * p.nb;
    b->edge = reinterpret_cast<int2*>(q);
    q += sizeof(int2) * ns * 2 * 2 * n;
    b->cedge = reinterpret_cast<int2*>(q);
    q += sizeof(int2) * ns * 2 * (n / 2);
    b->band_part = reinterpret_cast<double*>(q);
    q += sizeof(double) * ns * kW;
    b->flags = reinterpret_cast<unsigned*>(q);
}

cudaError_t band_run(const KArgs& k, BArgs b, const BandPlan& p, cudaStream_t st) {
    // k.partials holds p.S slots (entry-major, [stride][S]); zero them, run the
    // waves of p.S samples, accumulate per slot; the caller reduces the slots.
    const int n = b.n;
    b.nb = p.nb;
    b.bmax = p.bmax;
    b.S = p.S;
    if (b.wait_polls == 0) b.wait_polls = kWaitPolls;
    cudaError_t e;
    band_zero_kernel<<<64, 256, 0, st>>>(k.partials, (size_t)k.slot_stride * p.S);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const bool cpl = b.coupled != 0;
    for (long long done = 0; done < k.count; done += p.S) {
        b.sid0 = k.first + done;
        b.count = (int)std::min<long long>(p.S, k.count - done);
        if ((e = cudaMemsetAsync(b.flags, 0, sizeof(unsigned) * (size_t)p.S * p.nb * 2, st)) != cudaSuccess) return e;
        e = band_dispatch(n, p.fc, cpl, [&](auto shape, auto c) {
            return band_launch<decltype(shape), decltype(c)::value>(k, b, st);
        });
        if (e != cudaSuccess) return e;
        band_finish_kernel<<<(b.count + 63) / 64, 64, 0, st>>>(k, b, p.S);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace dk
