// Fourier-coupled sample kernel for grids beyond one CTA (Section 3.1): the
// fine path of Eq. (FullyDiscreteDK) (b0 = 0, b1 = 1) on a 162 x 162 grid and,
// for a coupled level, the coarse path on the 54 x 54 grid with step 9 tau,
// whose noise carries every Fourier mode of the fine noise that the coarse
// grid resolves.  Same noise, arithmetic and restriction as the one-CTA
// Fourier kernel: the cell normals of the explicit kernels (same Philox
// counters), the 9 fine normal fields of a coarse step summed per cell (FP32)
// and restricted once, W = P1 S P1^T (P1: nc x n, orthonormal rows), the
// coarse transfers rint(c 2^S sqrt(rho_c^+) W / 3), integer flux form.
//
// Work decomposition.  A sample's 162^2 fine cells (and their transfers and
// summed normals) need about 630 KB, so a thread-block cluster of CL = 6 CTAs
// carries one sample: CTA `rank` holds the band of fine rows 27 rank ..
// 27 rank + 26 and the coarse rows 9 rank .. 9 rank + 8.  A thread owns a
// segment of 6 consecutive fine cells of one row in registers (3 Philox cell
// pairs) and publishes its state and transfers in shared memory; the rows just
// above and below a band come from the neighbouring CTAs' shared memory
// (distributed shared memory, periodic over the cluster).
//
// Exchanges.  State and transfers are double-buffered by the step's parity,
// so a fine step needs one cluster barrier, split: a thread arrives (release)
// after writing its transfers; the warps of the band's first and last rows,
// which read other CTAs, wait (acquire) at once, the others only before their
// next arrival, after their flux update.  At a coarse step each CTA restricts
// its own rows, T = S_band P1^T (27 x 54 per component), and forms the partial
// product P1[:, band] T (54 x 54); after a cluster barrier each CTA sums the 6
// partials of its coarse rows in rank order, forms the coarse transfers, and
// after a second barrier updates its coarse rows.
#include <cooperative_groups.h>

#include "dk_device.cuh"
#include "dk_kernels.h"

namespace cg = cooperative_groups;

namespace dk {
namespace {

constexpr unsigned kFullMaskX = 0xffffffffu;
constexpr int kRedX = 2 * kMaxObs + 2;

template <int N_, int CL_>
struct XShape {
    static constexpr int N = N_, NC = N / 3, CL = CL_;
    static constexpr int BR = N / CL;               // fine rows per CTA
    static constexpr int CBR = NC / CL;             // coarse rows per CTA
    static constexpr int SEG = 6;                   // fine cells per thread: one row segment (3 Philox pairs)
    static constexpr int SEGS = N / SEG;            // segments per row
    static constexpr int FT = BR * SEGS;            // threads that hold fine cells
    static constexpr int THREADS = (FT + 31) / 32 * 32;
    static constexpr int WARPS = THREADS / 32;
    static constexpr int BAND = BR * N;             // fine cells per CTA
    static constexpr int CBAND = CBR * NC;          // coarse cells per CTA
    static constexpr int HY = NC / 2;               // coarse column pairs
    static_assert(N % CL == 0 && NC % CL == 0 && N % SEG == 0 && NC % 2 == 0 && BR >= 2 && CBR >= 2,
                  "band shape");
    static_assert(BR * HY <= THREADS && CBAND <= THREADS && THREADS <= 1024, "one task per thread");
    // words: fine q, G1, G2 (two buffers each) of the band; for a coupled level
    // the summed normals (2 per cell), P1 transposed (N x NC), T (BR x NC x 2),
    // the partial product (NC x NC x 2), coarse q (two buffers), Gc1, Gc2
    static constexpr int WORDS_F = 6 * BAND;
    static constexpr int WORDS_C = 2 * BAND + N * NC + 2 * BR * NC + 2 * NC * NC + 4 * CBAND;
    __host__ __device__ static constexpr int words(bool cpl) { return WORDS_F + (cpl ? WORDS_C : 0); }
    static size_t smem(bool cpl, int slot_stride) {
        return sizeof(int32_t) * (size_t)((words(cpl) + 1) / 2 * 2) +
               sizeof(double) * (size_t)(WARPS * kRedX + kRedX + slot_stride);
    }
};

// Split cluster barrier: arrive with release after a write that other CTAs
// read, a CTA barrier for the rest of the CTA, then the wait with acquire at
// once (threads that read other CTAs) or before the thread's next arrival.
struct XPhase {
    bool edge;
    bool pend = false;
    __device__ __forceinline__ explicit XPhase(bool edge_) : edge(edge_) {}
    __device__ __forceinline__ static void arrive() {
        asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    }
    __device__ __forceinline__ static void wait() {
        asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
    __device__ __forceinline__ void settle() {
        if (pend) {
            wait();
            pend = false;
        }
    }
    __device__ __forceinline__ void publish() {
        settle();
        arrive();
        __syncthreads();
        if (edge) wait();
        else pend = true;
    }
    __device__ __forceinline__ void full() {
        settle();
        arrive();
        wait();
    }
};

template <int N, int CL, bool CPL>
__global__ void __launch_bounds__(XShape<N, CL>::THREADS, 1)
    fourier_cluster_kernel(const KArgs a, const FArgs f) {
    using S = XShape<N, CL>;
    constexpr int NC = S::NC, BR = S::BR, CBR = S::CBR, SEG = S::SEG, SEGS = S::SEGS, THREADS = S::THREADS;
    constexpr int BAND = S::BAND, CBAND = S::CBAND, HY = S::HY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cluster = cg::this_cluster();
    const int tid = threadIdx.x;
    const int rank = static_cast<int>(cluster.block_rank());
    int32_t* const words = reinterpret_cast<int32_t*>(smem_raw);
    // fine planes: q buffers at 0, BAND; G1 buffers at 2 BAND, 3 BAND; G2 buffers at 4 BAND, 5 BAND
    float* const Zs = reinterpret_cast<float*>(words + S::WORDS_F);        // [BAND][2] summed normals
    float* const P1t = Zs + 2 * BAND;                                      // [N][NC]
    float* const Tm = P1t + N * NC;                                        // [BR][NC][2]
    float* const Wp = Tm + 2 * BR * NC;                                    // [NC][NC][2] partial product
    int32_t* const qc0 = reinterpret_cast<int32_t*>(Wp + 2 * NC * NC);     // coarse q buffers at qc0, qc0 + CBAND
    int32_t* const Gc1 = qc0 + 2 * CBAND;
    int32_t* const Gc2 = Gc1 + CBAND;
    double* const red = reinterpret_cast<double*>(smem_raw + sizeof(int32_t) * (size_t)((S::words(CPL) + 1) / 2 * 2));
    double* const tot = red + S::WARPS * kRedX;      // this CTA's band totals
    double* const acc = tot + kRedX;                 // the slot's moment sums (rank 0)
    for (int i = tid; i < a.slot_stride; i += THREADS) acc[i] = 0.0;
    if constexpr (CPL)
        for (int i = tid; i < N * NC; i += THREADS) {
            const int x = i / NC, y = i % NC;
            P1t[i] = f.P1[(size_t)y * N + x];
        }

    // ---- the thread's fine segment and its neighbours
    const bool fine_thread = tid < S::FT;
    const int lr = fine_thread ? tid / SEGS : 0;
    const int c0 = fine_thread ? (tid % SEGS) * SEG : 0;
    const int x0 = lr * N + c0;                                   // first cell of the segment in the band
    const int gx0 = rank * BAND + x0;                             // ... on the whole grid
    const int ra = lr > 0 ? rank : (rank + CL - 1) % CL;          // CTA of the row above / below
    const int rb = lr < BR - 1 ? rank : (rank + 1) % CL;
    const int ia = lr > 0 ? x0 - N : (BR - 1) * N + c0;           // its first cell there
    const int ib = lr < BR - 1 ? x0 + N : c0;
    const int32_t* const up = ra == rank ? words : cluster.map_shared_rank(words, ra);
    const int32_t* const dn = rb == rank ? words : cluster.map_shared_rank(words, rb);
    const int lfx = c0 == 0 ? x0 + N - 1 : x0 - 1;                // left of the first cell
    const int rtx = c0 + SEG == N ? x0 + SEG - N : x0 + SEG;      // right of the last cell
    // the warps holding a cell of the band's first or last row read other CTAs
    // (rows are not warp-aligned, so the test is per warp: the cluster wait is .aligned)
    const int wf = tid & ~31, wl = min(wf + 31, S::FT - 1);
    XPhase ph(wf < S::FT && (wf / SEGS == 0 || wl / SEGS >= BR - 1));

    // ---- the thread's coarse cell (coupled levels): local index tid, global index
    // (rank CBR + tid / NC) NC + tid % NC = rank CBAND + tid
    const bool coarse_thread = CPL && tid < CBAND;

    const long long n_slots = (long long)gridDim.x / CL;
    const long long slot = (long long)blockIdx.x / CL;
    const long long iters = a.count > slot ? (a.count - slot + n_slots - 1) / n_slots : 0;
    unsigned bad = 0;
    ph.full();

    for (long long it = 0; it < iters; ++it) {
        const long long idx = slot + it * n_slots;
        const long long sid = a.first + idx;
        const uint32_t c2 = static_cast<uint32_t>(sid);
        const uint32_t c3 = a.tag | ((static_cast<uint32_t>(static_cast<unsigned long long>(sid) >> 32) & 0xffffu) << 16);
        int32_t qr[SEG];
        if (fine_thread) {
#pragma unroll
            for (int j = 0; j < SEG; j += 2) {
                qr[j] = a.q0f[gx0 + j];
                qr[j + 1] = a.q0f[gx0 + j + 1];
                *reinterpret_cast<int2*>(words + x0 + j) = make_int2(qr[j], qr[j + 1]);
            }
        }
        int cb = 0;
        if (coarse_thread) qc0[tid] = a.q0c[rank * CBAND + tid];
        ph.full();

        for (int m = 0; m < a.M; ++m) {
            const int b = m & 1;
            const bool first_of_coarse = CPL && (m % 9) == 0;
            int32_t g1[SEG], g2[SEG];
            // ---- noise of the segment: Philox4x32-10 per horizontal cell pair, Box--Muller, transfers
            if (fine_thread) {
                int2* const G1w = reinterpret_cast<int2*>(words + (2 + b) * BAND);
                int2* const G2w = reinterpret_cast<int2*>(words + (4 + b) * BAND);
#pragma unroll
                for (int j = 0; j < SEG / 2; ++j) {
                    const int p = (gx0 >> 1) + j, lp = (x0 >> 1) + j;
                    const uint4 x = philox10(make_uint4(static_cast<uint32_t>(p), static_cast<uint32_t>(m), c2, c3),
                                             a.key0, a.key1);
                    float ra_, ca, sa, rb_, cbn, sb;
                    box_muller_polar(x.x, x.y, ra_, ca, sa);
                    box_muller_polar(x.z, x.w, rb_, cbn, sb);
                    const float ta = noise_amp(qr[2 * j], a.gf) * ra_;
                    const float tb = noise_amp(qr[2 * j + 1], a.gf) * rb_;
                    g1[2 * j] = __float2int_rn(ta * ca);
                    g2[2 * j] = __float2int_rn(ta * sa);
                    g1[2 * j + 1] = __float2int_rn(tb * cbn);
                    g2[2 * j + 1] = __float2int_rn(tb * sb);
                    G1w[lp] = make_int2(g1[2 * j], g1[2 * j + 1]);
                    G2w[lp] = make_int2(g2[2 * j], g2[2 * j + 1]);
                    if constexpr (CPL) {
                        float4 z = first_of_coarse ? make_float4(0.f, 0.f, 0.f, 0.f)
                                                   : reinterpret_cast<float4*>(Zs)[lp];
                        z.x += ra_ * ca;
                        z.y += ra_ * sa;
                        z.z += rb_ * cbn;
                        z.w += rb_ * sb;
                        reinterpret_cast<float4*>(Zs)[lp] = z;
                    }
                }
            }
            ph.publish();
            // ---- explicit step of the segment in flux form (every edge flux computed
            // from the same two states by both of its cells)
            if (fine_thread) {
                const int32_t* const q = words + b * BAND;
                const int32_t* const G2 = words + (4 + b) * BAND;
                int32_t qu[SEG], qd[SEG], gu[SEG], gd[SEG];
#pragma unroll
                for (int j = 0; j < SEG; j += 2) {
                    const int2 a0 = *reinterpret_cast<const int2*>(up + b * BAND + ia + j);
                    const int2 a1 = *reinterpret_cast<const int2*>(dn + b * BAND + ib + j);
                    const int2 b0 = *reinterpret_cast<const int2*>(up + (2 + b) * BAND + ia + j);
                    const int2 b1 = *reinterpret_cast<const int2*>(dn + (2 + b) * BAND + ib + j);
                    qu[j] = a0.x; qu[j + 1] = a0.y; qd[j] = a1.x; qd[j + 1] = a1.y;
                    gu[j] = b0.x; gu[j + 1] = b0.y; gd[j] = b1.x; gd[j + 1] = b1.y;
                }
                const int32_t qlf = q[lfx], qrt = q[rtx], g2lf = G2[lfx], g2rt = G2[rtx];
                int32_t nq[SEG];
#pragma unroll
                for (int j = 0; j < SEG; ++j) {
                    const int32_t c = qr[j];
                    const int32_t lf = j == 0 ? qlf : qr[j - 1];
                    const int32_t rt = j == SEG - 1 ? qrt : qr[j + 1];
                    const int32_t g2l = j == 0 ? g2lf : g2[j - 1];
                    const int32_t g2r = j == SEG - 1 ? g2rt : g2[j + 1];
                    nq[j] = c + (edge_flux(a.Af, qd[j] - c) - edge_flux(a.Af, c - qu[j])) +
                            (edge_flux(a.Af, rt - c) - edge_flux(a.Af, c - lf)) + (gd[j] - gu[j]) + (g2r - g2l);
                    bad |= (static_cast<uint32_t>(nq[j]) + 0x40000000u) >> 31;
                }
                int32_t* const qn = words + (b ^ 1) * BAND;
#pragma unroll
                for (int j = 0; j < SEG; j += 2) {
                    qr[j] = nq[j];
                    qr[j + 1] = nq[j + 1];
                    *reinterpret_cast<int2*>(qn + x0 + j) = make_int2(nq[j], nq[j + 1]);
                }
            }
            if constexpr (CPL) {
                if ((m % 9) == 8) {
                    ph.settle();
                    // ---- T = S_band P1^T: row x1 of the band, coarse columns 2 yy and 2 yy + 1, both components
                    if (tid < BR * HY) {
                        const int lx1 = tid / HY, yy = tid % HY;
                        const float2* const zrow = reinterpret_cast<const float2*>(Zs) + lx1 * N;
                        const float2* const pcol = reinterpret_cast<const float2*>(P1t) + yy;
                        float s00 = 0.f, s01 = 0.f, s10 = 0.f, s11 = 0.f;
#pragma unroll 6
                        for (int x2 = 0; x2 < N; ++x2) {
                            const float2 z = zrow[x2], w = pcol[x2 * HY];
                            s00 = fmaf(z.x, w.x, s00);
                            s01 = fmaf(z.y, w.x, s01);
                            s10 = fmaf(z.x, w.y, s10);
                            s11 = fmaf(z.y, w.y, s11);
                        }
                        reinterpret_cast<float4*>(Tm)[lx1 * HY + yy] = make_float4(s00, s01, s10, s11);
                    }
                    __syncthreads();
                    // ---- the band's part of P1 S P1^T: every coarse point (y1, 2 yy + v)
                    for (int o = tid; o < NC * HY; o += THREADS) {
                        const int y1 = o / HY, yy = o % HY;
                        float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 9
                        for (int lx1 = 0; lx1 < BR; ++lx1) {
                            const float p = P1t[(rank * BR + lx1) * NC + y1];
                            const float4 t = reinterpret_cast<const float4*>(Tm)[lx1 * HY + yy];
                            w.x = fmaf(p, t.x, w.x);
                            w.y = fmaf(p, t.y, w.y);
                            w.z = fmaf(p, t.z, w.z);
                            w.w = fmaf(p, t.w, w.w);
                        }
                        reinterpret_cast<float4*>(Wp)[o] = w;
                    }
                    ph.full();
                    // ---- coarse transfers of the CTA's coarse rows: the partials summed in rank order
                    int32_t* const qc = qc0 + cb * CBAND;
                    if (coarse_thread) {
                        const int o = rank * CBAND + tid;   // coarse point (y1, y2), y1 = rank CBR + tid / NC
                        float w0 = 0.f, w1 = 0.f;
#pragma unroll
                        for (int r = 0; r < CL; ++r) {
                            const float* const src = r == rank ? Wp : cluster.map_shared_rank(Wp, r);
                            const float2 v = reinterpret_cast<const float2*>(src)[o];
                            w0 += v.x;
                            w1 += v.y;
                        }
                        const float amp = noise_amp(qc[tid], a.gc);   // gc includes the 1/3 of the 9-step sum
                        Gc1[tid] = __float2int_rn(amp * w0);
                        Gc2[tid] = __float2int_rn(amp * w1);
                    }
                    ph.full();
                    // ---- explicit coarse step of the CTA's coarse rows
                    if (coarse_thread) {
                        // neighbours of the coarse cell: above / below in the neighbouring CTA for
                        // the band's first / last coarse row (periodic over the cluster)
                        const int cl1 = tid / NC, cy2 = tid % NC;
                        const int cra = cl1 > 0 ? rank : (rank + CL - 1) % CL;
                        const int crb = cl1 < CBR - 1 ? rank : (rank + 1) % CL;
                        const int cia = cl1 > 0 ? tid - NC : (CBR - 1) * NC + cy2;
                        const int cib = cl1 < CBR - 1 ? tid + NC : cy2;
                        const int clf = cl1 * NC + (cy2 + NC - 1) % NC, crt = cl1 * NC + (cy2 + 1) % NC;
                        const int32_t* const cup = cra == rank ? qc0 : cluster.map_shared_rank(qc0, cra);
                        const int32_t* const cdn = crb == rank ? qc0 : cluster.map_shared_rank(qc0, crb);
                        const int32_t c = qc[tid];
                        const int32_t* const gu_p = cra == rank ? Gc1 : cluster.map_shared_rank(Gc1, cra);
                        const int32_t* const gd_p = crb == rank ? Gc1 : cluster.map_shared_rank(Gc1, crb);
                        const int32_t qu = cup[cb * CBAND + cia], qd = cdn[cb * CBAND + cib];
                        const int32_t v = c + (edge_flux(a.Ac, qd - c) - edge_flux(a.Ac, c - qu)) +
                                          (edge_flux(a.Ac, qc[crt] - c) - edge_flux(a.Ac, c - qc[clf])) +
                                          (gd_p[cib] - gu_p[cia]) + (Gc2[crt] - Gc2[clf]);
                        bad |= (static_cast<uint32_t>(v) + 0x40000000u) >> 31;
                        qc0[(cb ^ 1) * CBAND + tid] = v;
                    }
                    cb ^= 1;
                }
            }
        }

        // ---- observables of the band (fine: registers, coarse: the thread's cell), then the
        // band totals summed on rank 0 in rank order
        double v[kRedX];
#pragma unroll
        for (int i = 0; i < kRedX; ++i) v[i] = 0.0;
        if (fine_thread) {
            long long mf = 0;
#pragma unroll
            for (int j = 0; j < SEG; ++j) mf += qr[j];
            v[2 * kMaxObs] = static_cast<double>(mf);
#pragma unroll
            for (int k = 0; k < kMaxObs; ++k) {
                if (k < a.n_obs) {
                    double s = 0.0;
#pragma unroll
                    for (int j = 0; j < SEG; ++j)
                        s += static_cast<double>(qr[j] - a.qbf[gx0 + j]) * f.phif64[(size_t)k * N * N + gx0 + j];
                    v[k] = s;
                }
            }
        }
        if (coarse_thread) {
            const int cg1 = rank * CBAND + tid;
            const int32_t qv = qc0[cb * CBAND + tid];
            v[2 * kMaxObs + 1] = static_cast<double>(qv);
            const double d = static_cast<double>(qv - a.qbc[cg1]);
#pragma unroll
            for (int k = 0; k < kMaxObs; ++k)
                if (k < a.n_obs) v[kMaxObs + k] = d * f.phic64[(size_t)k * NC * NC + cg1];
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1)
#pragma unroll
            for (int i = 0; i < kRedX; ++i) v[i] += __shfl_xor_sync(kFullMaskX, v[i], off);
        if ((tid & 31) == 0)
#pragma unroll
            for (int i = 0; i < kRedX; ++i) red[(tid >> 5) * kRedX + i] = v[i];
        __syncthreads();
        if (tid < kRedX) {
            double x = 0.0;
            for (int w = 0; w < S::WARPS; ++w) x += red[w * kRedX + tid];
            tot[tid] = x;
        }
        ph.full();
        if (rank == 0 && tid == 0) {
            for (int i = 0; i < kRedX; ++i) {
                double x = 0.0;
                for (int r = 0; r < CL; ++r) x += (r == 0 ? tot : cluster.map_shared_rank(tot, r))[i];
                v[i] = x;
            }
            double Df[kMaxObs], Dc[kMaxObs];
#pragma unroll
            for (int k = 0; k < kMaxObs; ++k) {
                Df[k] = a.dscale_f * v[k] + a.delta_f[k];
                Dc[k] = CPL ? a.dscale_c * v[kMaxObs + k] + a.delta_c[k] : 0.0;
            }
            acc[0] += 1.0;
            double merr = fabs(v[2 * kMaxObs] - static_cast<double>(a.mass0_f)) * a.dscale_f;
            if (CPL) merr = fmax(merr, fabs(v[2 * kMaxObs + 1] - static_cast<double>(a.mass0_c)) * a.dscale_c);
            acc[1] = fmax(acc[1], merr);
            int qi = 0;
            for (int j = 0; j < a.n_obs; ++j) {
                const int kend = a.products ? a.n_obs : j + 1;
                for (int k = j; k < kend; ++k, ++qi) {
                    const double pf = a.N * Df[j] * Df[k];
                    const double pc = CPL ? a.N * Dc[j] * Dc[k] : 0.0;
                    const double dp = pf - pc, dp2 = dp * dp;
                    double* B = acc + 2 + kNSum * qi;
                    B[0] += dp; B[1] += dp2; B[2] += dp2 * dp; B[3] += dp2 * dp2;
                    B[4] += pf; B[5] += pf * pf; B[6] += pc; B[7] += pc * pc;
                    B[8] += Df[j]; B[9] += Df[j] * Df[j]; B[10] += Dc[j]; B[11] += Dc[j] * Dc[j];
                }
            }
            if (a.samples) {
                double* o = a.samples + idx * (2 * a.n_obs + 2);
                for (int k = 0; k < a.n_obs; ++k) {
                    o[k] = Df[k];
                    o[a.n_obs + k] = Dc[k];
                }
                o[2 * a.n_obs] = v[2 * kMaxObs] * a.dscale_f;
                o[2 * a.n_obs + 1] = CPL ? v[2 * kMaxObs + 1] * a.dscale_c : 0.0;
            }
        }
        ph.full();   // the band totals and the state planes are reused by the next sample
    }
    if (bad) atomicOr(a.err, kErrRange);

    // ---- the slot's partial sums (rank 0), entry-major [stride][n_slots]
    __syncthreads();
    if (rank == 0)
        for (int i = tid; i < a.slot_stride; i += THREADS) a.partials[(size_t)i * n_slots + slot] = acc[i];
}

constexpr int kFourierClusterN = 162, kFourierClusterCL = 6;

template <int N, int CL, bool CPL>
cudaError_t xprepare(int slot_stride, VariantInfo* out) {
    using S = XShape<N, CL>;
    const size_t smem = S::smem(CPL, slot_stride);
    cudaError_t e = cudaFuncSetAttribute(fourier_cluster_kernel<N, CL, CPL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(S::THREADS);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if ((e = cudaOccupancyMaxActiveClusters(&clusters, fourier_cluster_kernel<N, CL, CPL>, &cfg)) != cudaSuccess)
        return e;
    *out = VariantInfo{};
    out->supported = clusters > 0;
    out->threads = S::THREADS;
    out->cluster = CL;
    out->slots_per_cta = 1;   // one sample slot per cluster
    out->smem = smem;
    out->max_ctas = clusters * CL;
    return cudaSuccess;
}

template <int N, int CL, bool CPL>
cudaError_t xlaunch(const KArgs& a, const FArgs& f, int n_ctas, cudaStream_t st, int priority) {
    using S = XShape<N, CL>;
    if (n_ctas <= 0 || n_ctas % CL != 0) return cudaErrorInvalidValue;
    if (CPL && !f.P1) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(n_ctas);
    cfg.blockDim = dim3(S::THREADS);
    cfg.dynamicSmemBytes = S::smem(CPL, a.slot_stride);
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    int na = 0;
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = CL;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
    if (priority != 0) {
        attr[na].id = cudaLaunchAttributePriority;
        attr[na].val.priority = priority;
        ++na;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, fourier_cluster_kernel<N, CL, CPL>, a, f);
}

}  // namespace

bool fourier_cluster_supported(int n) { return n == kFourierClusterN; }

cudaError_t fourier_cluster_variant_info(int n, bool coupled, int slot_stride, VariantInfo* out) {
    *out = VariantInfo{};
    if (n != kFourierClusterN) return cudaSuccess;
    return coupled ? xprepare<kFourierClusterN, kFourierClusterCL, true>(slot_stride, out)
                   : xprepare<kFourierClusterN, kFourierClusterCL, false>(slot_stride, out);
}

cudaError_t launch_fourier_cluster(int n, bool coupled, const KArgs& a, const FArgs& f, int n_ctas, cudaStream_t st,
                                   int priority) {
    if (n != kFourierClusterN) return cudaErrorInvalidValue;
    return coupled ? xlaunch<kFourierClusterN, kFourierClusterCL, true>(a, f, n_ctas, st, priority)
                   : xlaunch<kFourierClusterN, kFourierClusterCL, false>(a, f, n_ctas, st, priority);
}

}  // namespace dk
