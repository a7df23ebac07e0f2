// Fused coupled fine/coarse Dean--Kawasaki sample kernel for sm_103a.
//
// One launch runs `count` independent samples of one level (Section 3.2: the
// fine path on G_{h_l} and, for l >= 1, the Right-Most NN coupled coarse path
// on G_{h_{l-1}}), each for M fine steps of Eq. (FullyDiscreteDK) with
// b0 = 0, b1 = 1 (Section 7.2), and reduces every sample on the fly to the
// observables (rho^T, I_h phi_k)_h, the quantities P = N (Y_j - Ybar_j)(Y_k -
// Ybar_k) of Eq. (eqn_MLMCLevels) and the FP64 moment sums that the estimator
// of Eq. (MLMCEstimator) and the allocation of Eq. (opt_M_ell) need.
//
// Work decomposition.  A sample's fine grid is cut into bands of FR = 2R fine
// rows; a band is held by LPB <= 32 consecutive lanes of one warp, each lane
// owning an FR x FC block (FC = 2C) of fine cells, i.e. an R x C block of the
// coarse grid, so the coupled coarse increment (the sum over the 2x2 fine
// cells to the right of each coarse point and over the 4 fine steps of one
// coarse step) is accumulated in the lane's registers.  The whole state lives
// in registers for the whole run.  Left/right neighbours come from the
// adjacent lanes by warp shuffles (the periodic wrap is the shuffle's segment
// wrap).  Up/down neighbours come
//   * by shuffles too when the whole sample fits one warp (n <= 32), so those
//     samples run without any barrier or shared memory, or
//   * through shared memory (double-buffered band edge rows, one barrier per
//     fine step) when the sample spans several warps; grids that need more
//     registers than one SM has span a thread-block cluster and read the
//     neighbouring CTA's edge rows through distributed shared memory.
//
// Arithmetic.  The state is 32-bit fixed point q = rho 2^S.  Each fine step
// computes, per cell, the noise transfers G_r = rint(c 2^S sqrt(rho^+) Z_r)
// (c = N^-1/2 sqrt(tau) / (2 h^2)) and, per edge, the diffusion flux
// rint(tau/(2h^2) (q_far - q_near)); the new state adds these integers
// exactly, so sum_x q is invariant bit for bit (the divergence form of the
// scheme) and every rounding error enters in divergence form.  Observables
// and moments are accumulated in FP64.
#include <cooperative_groups.h>

#include <atomic>
#include <mutex>

#include "dk_device.cuh"
#include "dk_kernels.h"

namespace cg = cooperative_groups;

namespace dk {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRedW = 2 * kMaxObs + 2;     // reduced values per sample
constexpr int kMaxStride = 2 + kNSum * 10;  // largest slot stride (4 obs with products)

template <int NF_, int C_, int R_, int CL_, bool COUPLED_, bool FLUCT_ = false>
struct Shape {
    static constexpr int NF = NF_, C = C_, R = R_, CL = CL_;
    static constexpr bool COUPLED = COUPLED_;
    // fluctuation state: q holds (rho - rho-bar^m) 2^S, rho-bar^m read from a
    // per-step mean-field table (see KArgs::rbf)
    static constexpr bool FLUCT = FLUCT_;
    static constexpr int NC = NF / 2;
    static constexpr int FR = 2 * R, FC = 2 * C;
    static constexpr int LPB = NC / C;            // lanes per band
    static constexpr int NB = NC / R;             // bands per sample
    static constexpr int LPS = LPB * NB;          // lanes per sample
    static constexpr bool WARP = LPS <= 32;       // sample resident in one warp
    static constexpr int SPW = WARP ? 32 / LPS : 1;
    static constexpr int THREADS = WARP ? 128 : LPS / CL;
    static constexpr int BPC = WARP ? 1 : NB / CL;   // bands per CTA
    static constexpr int SLOTS_PER_CTA = WARP ? (THREADS / 32) * SPW : 1;
    static_assert(LPB <= 32 && (LPB & (LPB - 1)) == 0, "a band must be a power-of-two warp segment");
    static_assert(NC % C == 0 && NC % R == 0, "lane blocks must tile the coarse grid");
    static_assert(WARP || (THREADS % 32 == 0 && THREADS <= 1024 && NB % CL == 0), "bad CTA shape");
    static_assert(WARP || CL == 1 || (LPS / CL) % LPB == 0, "bands may not straddle CTAs");
    static constexpr size_t fixed_smem() {
        return WARP ? 0
                    : sizeof(int2) * 2 * 2 * BPC * NF + (COUPLED ? sizeof(int2) * 2 * BPC * NC : 0) +
                          sizeof(double) * (THREADS / 32) * kRedW;
    }
};

template <int N>
__device__ __forceinline__ void load_row(int32_t (&dst)[N], const int32_t* src) {
    if constexpr (N == 1) {
        dst[0] = __ldg(src);
    } else if constexpr (N == 2) {
        const int2 v = __ldg(reinterpret_cast<const int2*>(src));
        dst[0] = v.x; dst[1] = v.y;
    } else {
        static_assert(N % 4 == 0, "");
#pragma unroll
        for (int i = 0; i < N; i += 4) {
            const int4 v = __ldg(reinterpret_cast<const int4*>(src + i));
            dst[i] = v.x; dst[i + 1] = v.y; dst[i + 2] = v.z; dst[i + 3] = v.w;
        }
    }
}

template <int N>
__device__ __forceinline__ void load_row_f(float (&dst)[N], const float* src) {
    if constexpr (N == 1) {
        dst[0] = __ldg(src);
    } else if constexpr (N == 2) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(src));
        dst[0] = v.x; dst[1] = v.y;
    } else {
#pragma unroll
        for (int i = 0; i < N; i += 4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(src + i));
            dst[i] = v.x; dst[i + 1] = v.y; dst[i + 2] = v.z; dst[i + 3] = v.w;
        }
    }
}

// Store / load the N (q, G1) pairs of one lane's part of a band edge row.
// Lane-interleaved layout: pair chunk k (columns 2k, 2k+1 of the lane) of lane
// `lib` is int4 number k*LPB + lib of the row, so a warp's store or load of one
// chunk is LPB consecutive 16-byte words (no bank conflicts).  N = 1 uses one
// int2 per lane.
template <int N, int LPB>
__device__ __forceinline__ void put_edge(int2* row, int lib, const int32_t (&qv)[N], const int32_t (&gv)[N]) {
    if constexpr (N % 2 == 0) {
        int4* r4 = reinterpret_cast<int4*>(row);
#pragma unroll
        for (int k = 0; k < N / 2; ++k) r4[k * LPB + lib] = make_int4(qv[2 * k], gv[2 * k], qv[2 * k + 1], gv[2 * k + 1]);
    } else {
        static_assert(N == 1, "odd edge chunks other than 1 are not used");
        row[lib] = make_int2(qv[0], gv[0]);
    }
}

template <int N, int LPB>
__device__ __forceinline__ void get_edge(const int2* row, int lib, int32_t (&qv)[N], int32_t (&gv)[N]) {
    if constexpr (N % 2 == 0) {
        const int4* r4 = reinterpret_cast<const int4*>(row);
#pragma unroll
        for (int k = 0; k < N / 2; ++k) {
            const int4 v = r4[k * LPB + lib];
            qv[2 * k] = v.x; gv[2 * k] = v.y; qv[2 * k + 1] = v.z; gv[2 * k + 1] = v.w;
        }
    } else {
        const int2 v = row[lib];
        qv[0] = v.x; gv[0] = v.y;
    }
}

template <class S>
__device__ __forceinline__ void block_or_cluster_sync() {
    if constexpr (S::CL > 1) {
        cg::this_cluster().sync();
    } else {
        __syncthreads();
    }
}

template <class S, class T>
__device__ __forceinline__ const T* peer(const T* local, int rank) {
    if constexpr (S::CL > 1) {
        return cg::this_cluster().map_shared_rank(const_cast<T*>(local), rank);
    } else {
        return local;
    }
}

// The same update in two phases around a split barrier: phase 1 updates the
// interior rows (1 .. RR-2), which need no vertical halo, and keeps the old
// values of rows 1 and RR-2 that the boundary rows' fluxes need; phase 2
// (after the halo arrives) updates rows 0 and RR-1.
template <int RR, int CC>
__device__ __forceinline__ void flux_update_interior(int32_t (&q)[RR][CC], const int32_t (&G1)[RR][CC],
                                                     const int32_t (&G2)[RR][CC], const int32_t (&qL)[RR],
                                                     const int32_t (&gL)[RR], const int32_t (&qR)[RR],
                                                     const int32_t (&gR)[RR], int32_t A, int32_t (&keep1)[CC],
                                                     int32_t (&keep2)[CC]) {
#pragma unroll
    for (int c = 0; c < CC; ++c) {
        keep1[c] = q[1][c];
        keep2[c] = q[RR - 2][c];
    }
    if constexpr (RR >= 3) {
        int32_t V[RR + 1][CC];
#pragma unroll
        for (int c = 0; c < CC; ++c)
#pragma unroll
            for (int r = 1; r < RR; ++r) V[r][c] = edge_flux(A, q[r][c] - q[r - 1][c]);
#pragma unroll
        for (int r = 1; r + 1 < RR; ++r) {
            int32_t H[CC + 1];
            H[0] = edge_flux(A, q[r][0] - qL[r]);
#pragma unroll
            for (int c = 1; c < CC; ++c) H[c] = edge_flux(A, q[r][c] - q[r][c - 1]);
            H[CC] = edge_flux(A, qR[r] - q[r][CC - 1]);
#pragma unroll
            for (int c = 0; c < CC; ++c) {
                const int32_t g2r = (c + 1 < CC) ? G2[r][c + 1] : gR[r];
                const int32_t g2l = (c > 0) ? G2[r][c - 1] : gL[r];
                q[r][c] += (V[r + 1][c] - V[r][c]) + (H[c + 1] - H[c]) + (G1[r + 1][c] - G1[r - 1][c]) + (g2r - g2l);
            }
        }
    }
}

template <int RR, int CC>
__device__ __forceinline__ void flux_update_boundary(int32_t (&q)[RR][CC], const int32_t (&G1)[RR][CC],
                                                     const int32_t (&G2)[RR][CC], const int32_t (&qU)[CC],
                                                     const int32_t (&gU)[CC], const int32_t (&qD)[CC],
                                                     const int32_t (&gD)[CC], const int32_t (&qL)[RR],
                                                     const int32_t (&gL)[RR], const int32_t (&qR)[RR],
                                                     const int32_t (&gR)[RR], int32_t A, const int32_t (&keep1)[CC],
                                                     const int32_t (&keep2)[CC]) {
    // row 0 (its lower neighbour is the old row 1) and row RR-1 (upper neighbour the old row RR-2)
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int r = side == 0 ? 0 : RR - 1;
        if (side == 1 && RR == 1) break;
        int32_t H[CC + 1];
        H[0] = edge_flux(A, q[r][0] - qL[r]);
#pragma unroll
        for (int c = 1; c < CC; ++c) H[c] = edge_flux(A, q[r][c] - q[r][c - 1]);
        H[CC] = edge_flux(A, qR[r] - q[r][CC - 1]);
#pragma unroll
        for (int c = 0; c < CC; ++c) {
            const int32_t up = (r == 0) ? qU[c] : keep2[c];
            const int32_t dn = (r == RR - 1) ? qD[c] : keep1[c];
            const int32_t g1u = (r == 0) ? gU[c] : G1[r - 1][c];
            const int32_t g1d = (r == RR - 1) ? gD[c] : G1[r + 1][c];
            const int32_t x = q[r][c];
            const int32_t v = edge_flux(A, dn - x) - edge_flux(A, x - up);
            const int32_t g2r = (c + 1 < CC) ? G2[r][c + 1] : gR[r];
            const int32_t g2l = (c > 0) ? G2[r][c - 1] : gL[r];
            q[r][c] = x + v + (H[c + 1] - H[c]) + (g1d - g1u) + (g2r - g2l);
        }
    }
}

__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory"); }

template <class S>
__global__ void __launch_bounds__(S::THREADS) level_kernel(const KArgs a) {
    constexpr int NF = S::NF, NC = S::NC, FR = S::FR, FC = S::FC, R = S::R, C = S::C;
    constexpr int LPB = S::LPB, LPS = S::LPS, CL = S::CL, BPC = S::BPC;
    constexpr bool CPL = S::COUPLED;
    // clusters split the per-step barrier: arrive after publishing the edge
    // rows, update the interior rows, then wait for the neighbours' rows
    constexpr bool SPLIT = !S::WARP && (CL > 1);
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int lib = lane % LPB;   // lane within its band
    int band, bl = 0, rank = 0, slot_local;
    long long slot, n_slots, base_slot;
    if constexpr (S::WARP) {
        band = (lane % LPS) / LPB;
        slot_local = (tid >> 5) * S::SPW + lane / LPS;
        slot = (long long)blockIdx.x * S::SLOTS_PER_CTA + slot_local;
        n_slots = (long long)gridDim.x * S::SLOTS_PER_CTA;
        base_slot = (long long)blockIdx.x * S::SLOTS_PER_CTA + (tid >> 5) * S::SPW;
    } else {
        if constexpr (CL > 1) rank = (int)cg::this_cluster().block_rank();
        bl = tid / LPB;
        band = rank * BPC + bl;
        slot_local = 0;
        slot = blockIdx.x / CL;
        n_slots = gridDim.x / CL;
        base_slot = slot;
    }
    const int row0 = band * FR, col0 = lib * FC;     // fine block origin
    const int crow0 = band * R, ccol0 = lib * C;      // coarse block origin
    const int left = (lib + LPB - 1) % LPB, right = (lib + 1) % LPB;
    const int up_lane = ((lane % LPS) + LPS - LPB) % LPS, dn_lane = ((lane % LPS) + LPB) % LPS;

    // shared memory: [fine edge rows][coarse edge rows][reduction][slot accumulators]
    unsigned char* sp = smem_raw;
    int2* fx = nullptr;
    int2* cx = nullptr;
    double* red = nullptr;
    if constexpr (!S::WARP) {
        fx = reinterpret_cast<int2*>(sp);
        sp += sizeof(int2) * 2 * 2 * BPC * NF;
        if constexpr (CPL) {
            cx = reinterpret_cast<int2*>(sp);
            sp += sizeof(int2) * 2 * BPC * NC;
        }
        red = reinterpret_cast<double*>(sp);
        sp += sizeof(double) * (S::THREADS / 32) * kRedW;
    }
    double* acc = reinterpret_cast<double*>(sp);
    for (int i = tid; i < S::SLOTS_PER_CTA * a.slot_stride; i += S::THREADS) acc[i] = 0.0;
    __syncthreads();

    const long long iters = a.count > base_slot ? (a.count - base_slot + n_slots - 1) / n_slots : 0;
    unsigned bad = 0;

    for (long long it = 0; it < iters; ++it) {
        const long long idx = slot + it * n_slots;
        const bool active = idx < a.count;
        const long long sid = a.first + (active ? idx : 0);
        const uint32_t c2 = static_cast<uint32_t>(sid);
        const uint32_t c3 = a.tag | ((static_cast<uint32_t>(static_cast<unsigned long long>(sid) >> 32) & 0xffffu) << 16);

        int32_t q[FR][FC];
#pragma unroll
        for (int r = 0; r < FR; ++r) load_row<FC>(q[r], a.q0f + (size_t)(row0 + r) * NF + col0);
        int32_t qc[R][C];
        float zt[R][C][2];
        if constexpr (CPL) {
#pragma unroll
            for (int i = 0; i < R; ++i) load_row<C>(qc[i], a.q0c + (size_t)(crow0 + i) * NC + ccol0);
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int j = 0; j < C; ++j) zt[i][j][0] = zt[i][j][1] = 0.f;
        }

        for (int m = 0; m < a.M; ++m) {
            // fluctuation state: the noise-free path rho-bar^m of this lane's cells
            float rb[S::FLUCT ? FR : 1][S::FLUCT ? FC : 1];
            if constexpr (S::FLUCT) {
#pragma unroll
                for (int r = 0; r < FR; ++r)
                    load_row_f<FC>(rb[r], a.rbf + (size_t)m * NF * NF + (size_t)(row0 + r) * NF + col0);
            }
            // ---- noise: Philox4x32-10 per horizontal cell pair, Box--Muller, transfers
            int32_t G1[FR][FC], G2[FR][FC];
#pragma unroll
            for (int r = 0; r < FR; ++r) {
#pragma unroll
                for (int pc = 0; pc < C; ++pc) {
                    const uint32_t p = static_cast<uint32_t>(((row0 + r) * NF + col0 + 2 * pc) >> 1);
                    const uint4 x = philox10(make_uint4(p, static_cast<uint32_t>(m), c2, c3), a.key0, a.key1);
                    // normals (ra ca, ra sa) and (rb cb, rb sb); the amplitude scales the radius
                    float ra, ca, sa, rb_, cb, sb;
                    box_muller_polar(x.x, x.y, ra, ca, sa);
                    box_muller_polar(x.z, x.w, rb_, cb, sb);
                    float ta, tb;
                    if constexpr (S::FLUCT) {
                        ta = noise_amp_fluct(q[r][2 * pc], rb[r][2 * pc], a.isf, a.gf) * ra;
                        tb = noise_amp_fluct(q[r][2 * pc + 1], rb[r][2 * pc + 1], a.isf, a.gf) * rb_;
                    } else {
                        ta = noise_amp(q[r][2 * pc], a.gf) * ra;
                        tb = noise_amp(q[r][2 * pc + 1], a.gf) * rb_;
                    }
                    G1[r][2 * pc] = __float2int_rn(ta * ca);
                    G2[r][2 * pc] = __float2int_rn(ta * sa);
                    G1[r][2 * pc + 1] = __float2int_rn(tb * cb);
                    G2[r][2 * pc + 1] = __float2int_rn(tb * sb);
                    if constexpr (CPL) {
                        zt[r >> 1][pc][0] = fmaf(rb_, cb, fmaf(ra, ca, zt[r >> 1][pc][0]));
                        zt[r >> 1][pc][1] = fmaf(rb_, sb, fmaf(ra, sa, zt[r >> 1][pc][1]));
                    }
                }
            }
            const bool cstep = CPL && ((m & 3) == 3);
            int32_t Gc1[R][C], Gc2[R][C];
            if constexpr (CPL) {
                if (cstep) {
                    float rbc[S::FLUCT ? R : 1][S::FLUCT ? C : 1];
                    if constexpr (S::FLUCT) {
#pragma unroll
                        for (int i = 0; i < R; ++i)
                            load_row_f<C>(rbc[i], a.rbc + (size_t)(m >> 2) * NC * NC + (size_t)(crow0 + i) * NC + ccol0);
                    }
#pragma unroll
                    for (int i = 0; i < R; ++i)
#pragma unroll
                        for (int j = 0; j < C; ++j) {
                            float s;
                            if constexpr (S::FLUCT) s = noise_amp_fluct(qc[i][j], rbc[i][j], a.isc, a.gc);
                            else s = noise_amp(qc[i][j], a.gc);
                            Gc1[i][j] = __float2int_rn(s * zt[i][j][0]);
                            Gc2[i][j] = __float2int_rn(s * zt[i][j][1]);
                            zt[i][j][0] = zt[i][j][1] = 0.f;
                        }
                }
            }

            if constexpr (SPLIT) {
                const int par = m & 1;
                put_edge<FC, LPB>(fx + ((par * 2 + 0) * BPC + bl) * NF, lib, q[0], G1[0]);
                put_edge<FC, LPB>(fx + ((par * 2 + 1) * BPC + bl) * NF, lib, q[FR - 1], G1[FR - 1]);
                if constexpr (CPL) {
                    if (cstep) {
                        put_edge<C, LPB>(cx + bl * NC, lib, qc[0], Gc1[0]);
                        put_edge<C, LPB>(cx + (BPC + bl) * NC, lib, qc[R - 1], Gc1[R - 1]);
                    }
                }
                cluster_arrive();
            }

            // ---- horizontal halo by shuffles within the band segment
            int32_t qL[FR], gL[FR], qR[FR], gR[FR];
#pragma unroll
            for (int r = 0; r < FR; ++r) {
                qL[r] = __shfl_sync(kFull, q[r][FC - 1], left, LPB);
                gL[r] = __shfl_sync(kFull, G2[r][FC - 1], left, LPB);
                qR[r] = __shfl_sync(kFull, q[r][0], right, LPB);
                gR[r] = __shfl_sync(kFull, G2[r][0], right, LPB);
            }
            int32_t cqL[R], cgL[R], cqR[R], cgR[R];
            if constexpr (CPL) {
                if (cstep) {
#pragma unroll
                    for (int i = 0; i < R; ++i) {
                        cqL[i] = __shfl_sync(kFull, qc[i][C - 1], left, LPB);
                        cgL[i] = __shfl_sync(kFull, Gc2[i][C - 1], left, LPB);
                        cqR[i] = __shfl_sync(kFull, qc[i][0], right, LPB);
                        cgR[i] = __shfl_sync(kFull, Gc2[i][0], right, LPB);
                    }
                }
            }

            // ---- vertical halo
            int32_t qU[FC], gU[FC], qD[FC], gD[FC];
            int32_t keep1[FC], keep2[FC];   // old rows 1 and FR-2 (split barrier only)
            int32_t cqU[C], cgU[C], cqD[C], cgD[C];
            if constexpr (S::WARP) {
#pragma unroll
                for (int c = 0; c < FC; ++c) {
                    qU[c] = __shfl_sync(kFull, q[FR - 1][c], up_lane, LPS);
                    gU[c] = __shfl_sync(kFull, G1[FR - 1][c], up_lane, LPS);
                    qD[c] = __shfl_sync(kFull, q[0][c], dn_lane, LPS);
                    gD[c] = __shfl_sync(kFull, G1[0][c], dn_lane, LPS);
                }
                if constexpr (CPL) {
                    if (cstep) {
#pragma unroll
                        for (int j = 0; j < C; ++j) {
                            cqU[j] = __shfl_sync(kFull, qc[R - 1][j], up_lane, LPS);
                            cgU[j] = __shfl_sync(kFull, Gc1[R - 1][j], up_lane, LPS);
                            cqD[j] = __shfl_sync(kFull, qc[0][j], dn_lane, LPS);
                            cgD[j] = __shfl_sync(kFull, Gc1[0][j], dn_lane, LPS);
                        }
                    }
                }
            } else {
                const int par = m & 1;
                int2* const ftop = fx + ((par * 2 + 0) * BPC) * NF;
                int2* const fbot = fx + ((par * 2 + 1) * BPC) * NF;
                int2* const ctop = cx;
                int2* const cbot = cx + BPC * NC;
                if constexpr (SPLIT) {
                    flux_update_interior<FR, FC>(q, G1, G2, qL, gL, qR, gR, a.Af, keep1, keep2);
                    cluster_wait();
                } else {
                    put_edge<FC, LPB>(ftop + bl * NF, lib, q[0], G1[0]);
                    put_edge<FC, LPB>(fbot + bl * NF, lib, q[FR - 1], G1[FR - 1]);
                    if constexpr (CPL) {
                        if (cstep) {
                            put_edge<C, LPB>(ctop + bl * NC, lib, qc[0], Gc1[0]);
                            put_edge<C, LPB>(cbot + bl * NC, lib, qc[R - 1], Gc1[R - 1]);
                        }
                    }
                    block_or_cluster_sync<S>();
                }
                const int2* above = (bl > 0) ? fbot + (bl - 1) * NF
                                             : peer<S>(fbot + (BPC - 1) * NF, (rank + CL - 1) % CL);
                const int2* below = (bl + 1 < BPC) ? ftop + (bl + 1) * NF : peer<S>(ftop, (rank + 1) % CL);
                get_edge<FC, LPB>(above, lib, qU, gU);
                get_edge<FC, LPB>(below, lib, qD, gD);
                if constexpr (CPL) {
                    if (cstep) {
                        const int2* cab = (bl > 0) ? cbot + (bl - 1) * NC
                                                   : peer<S>(cbot + (BPC - 1) * NC, (rank + CL - 1) % CL);
                        const int2* cbe = (bl + 1 < BPC) ? ctop + (bl + 1) * NC : peer<S>(ctop, (rank + 1) % CL);
                        get_edge<C, LPB>(cab, lib, cqU, cgU);
                        get_edge<C, LPB>(cbe, lib, cqD, cgD);
                    }
                }
            }

            // ---- updates
            if constexpr (SPLIT) {
                flux_update_boundary<FR, FC>(q, G1, G2, qU, gU, qD, gD, qL, gL, qR, gR, a.Af, keep1, keep2);
            } else {
                flux_update<FR, FC>(q, G1, G2, qU, gU, qD, gD, qL, gL, qR, gR, a.Af);
            }
            if constexpr (CPL) {
                if (cstep) {
                    flux_update<R, C>(qc, Gc1, Gc2, cqU, cgU, cqD, cgD, cqL, cgL, cqR, cgR, a.Ac);
#pragma unroll
                    for (int i = 0; i < R; ++i)
#pragma unroll
                        for (int j = 0; j < C; ++j) bad |= (static_cast<uint32_t>(qc[i][j]) + 0x40000000u) >> 31;
                }
            }
            if ((m & 3) == 3 || m + 1 == a.M) {
#pragma unroll
                for (int r = 0; r < FR; ++r)
#pragma unroll
                    for (int c = 0; c < FC; ++c) bad |= (static_cast<uint32_t>(q[r][c]) + 0x40000000u) >> 31;
            }
        }

        // ---- observables: fluctuation sums against the fixed-point mean field, mass
        double v[kRedW];
        {
            long long mf = 0;
#pragma unroll
            for (int r = 0; r < FR; ++r)
#pragma unroll
                for (int c = 0; c < FC; ++c) mf += q[r][c];
            v[2 * kMaxObs] = static_cast<double>(mf);
            long long mc = 0;
            if constexpr (CPL) {
#pragma unroll
                for (int i = 0; i < R; ++i)
#pragma unroll
                    for (int j = 0; j < C; ++j) mc += qc[i][j];
            }
            v[2 * kMaxObs + 1] = static_cast<double>(mc);
#pragma unroll
            for (int k = 0; k < kMaxObs; ++k) {
                float sf = 0.f, sc = 0.f;
                if (k < a.n_obs) {
#pragma unroll
                    for (int r = 0; r < FR; ++r) {
                        int32_t qb[FC];
                        float ph[FC];
                        load_row<FC>(qb, a.qbf + (size_t)(row0 + r) * NF + col0);
                        load_row_f<FC>(ph, a.phif + (size_t)k * NF * NF + (size_t)(row0 + r) * NF + col0);
#pragma unroll
                        for (int c = 0; c < FC; ++c) sf = fmaf(__int2float_rn(q[r][c] - qb[c]), ph[c], sf);
                    }
                    if constexpr (CPL) {
#pragma unroll
                        for (int i = 0; i < R; ++i) {
                            int32_t qb[C];
                            float ph[C];
                            load_row<C>(qb, a.qbc + (size_t)(crow0 + i) * NC + ccol0);
                            load_row_f<C>(ph, a.phic + (size_t)k * NC * NC + (size_t)(crow0 + i) * NC + ccol0);
#pragma unroll
                            for (int j = 0; j < C; ++j) sc = fmaf(__int2float_rn(qc[i][j] - qb[j]), ph[j], sc);
                        }
                    }
                }
                v[k] = static_cast<double>(sf);
                v[kMaxObs + k] = static_cast<double>(sc);
            }
        }
        bool leader;
        if constexpr (S::WARP) {
#pragma unroll
            for (int off = LPS / 2; off >= 1; off >>= 1)
#pragma unroll
                for (int i = 0; i < kRedW; ++i) v[i] += __shfl_xor_sync(kFull, v[i], off, LPS);
            leader = (lane % LPS) == 0;
        } else {
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1)
#pragma unroll
                for (int i = 0; i < kRedW; ++i) v[i] += __shfl_xor_sync(kFull, v[i], off);
            if (lane == 0)
#pragma unroll
                for (int i = 0; i < kRedW; ++i) red[(tid >> 5) * kRedW + i] = v[i];
            __syncthreads();
            if (tid == 0) {
                for (int w = 1; w < S::THREADS / 32; ++w)
#pragma unroll
                    for (int i = 0; i < kRedW; ++i) v[i] += red[w * kRedW + i];
#pragma unroll
                for (int i = 0; i < kRedW; ++i) red[i] = v[i];
            }
            if constexpr (CL > 1) {
                cg::this_cluster().sync();
                if (rank == 0 && tid == 0) {
                    for (int rr = 1; rr < CL; ++rr) {
                        const double* o = peer<S>(red, rr);
#pragma unroll
                        for (int i = 0; i < kRedW; ++i) v[i] += o[i];
                    }
                }
            }
            leader = (tid == 0) && (rank == 0);
        }

        // ---- FP64 quantities and moment sums (one lane per sample)
        if (leader && active) {
            double Df[kMaxObs], Dc[kMaxObs];
#pragma unroll
            for (int k = 0; k < kMaxObs; ++k) {
                Df[k] = a.dscale_f * v[k] + a.delta_f[k];
                Dc[k] = CPL ? a.dscale_c * v[kMaxObs + k] + a.delta_c[k] : 0.0;
            }
            double* A = acc + slot_local * a.slot_stride;
            A[0] += 1.0;
            double merr = fabs(v[2 * kMaxObs] - static_cast<double>(a.mass0_f)) * a.dscale_f;
            if (CPL) merr = fmax(merr, fabs(v[2 * kMaxObs + 1] - static_cast<double>(a.mass0_c)) * a.dscale_c);
            A[1] = fmax(A[1], merr);
            int qi = 0;
            for (int j = 0; j < a.n_obs; ++j) {
                const int kend = a.products ? a.n_obs : j + 1;
                for (int k = j; k < kend; ++k, ++qi) {
                    const double pf = a.N * Df[j] * Df[k];
                    const double pc = CPL ? a.N * Dc[j] * Dc[k] : 0.0;
                    const double dp = pf - pc, dp2 = dp * dp;
                    double* B = A + 2 + kNSum * qi;
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
                o[2 * a.n_obs] = v[2 * kMaxObs] * a.dscale_f + a.mass_off_f;
                o[2 * a.n_obs + 1] = CPL ? v[2 * kMaxObs + 1] * a.dscale_c + a.mass_off_c : 0.0;
            }
        }
    }
    if (bad) atomicOr(a.err, kErrRange);

    // ---- per-slot partial sums to global scratch, entry-major [stride][n_slots]
    __syncthreads();
    if (S::WARP || rank == 0) {
        const long long slot0 = S::WARP ? (long long)blockIdx.x * S::SLOTS_PER_CTA : slot;
        for (int i = tid; i < S::SLOTS_PER_CTA * a.slot_stride; i += S::THREADS) {
            const int s = i / a.slot_stride, e = i % a.slot_stride;
            a.partials[(size_t)e * n_slots + slot0 + s] = acc[i];
        }
    }
    if constexpr (CL > 1) cg::this_cluster().sync();   // peers may still read our shared memory
}

// Fixed-order reduction over slots: one block per entry.
__global__ void __launch_bounds__(256) reduce_kernel(const double* part, int n_slots, double* out) {
    const int e = blockIdx.x;
    const bool is_max = (e == 1);
    const double* row = part + (size_t)e * n_slots;
    double v = 0.0;
    for (int s = threadIdx.x; s < n_slots; s += 256) v = is_max ? fmax(v, row[s]) : v + row[s];
    __shared__ double sh[256];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const double o = sh[threadIdx.x + w];
            sh[threadIdx.x] = is_max ? fmax(sh[threadIdx.x], o) : sh[threadIdx.x] + o;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[e] = sh[0];
}

// out[e] += in[e] (entry 1, the max mass error: max): merges the sums of two
// disjoint sample ranges of one level.
__global__ void add_sums_kernel(double* out, const double* in, int stride) {
    for (int e = threadIdx.x; e < stride; e += blockDim.x) out[e] = e == 1 ? fmax(out[e], in[e]) : out[e] + in[e];
}

// Normals of one fine step, written out (the level kernel keeps them in
// registers); same device functions as the level kernel.
__global__ void noise_kernel(int n, uint32_t m, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                             float* z, uint32_t* raw) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n * n / 2) return;
    const uint4 x = philox10(make_uint4(static_cast<uint32_t>(p), m, c2, c3), k0, k1);
    if (raw) reinterpret_cast<uint4*>(raw)[p] = x;
    if (z) {
        float a1, a2, b1, b2;
        box_muller(x.x, x.y, a1, a2);
        box_muller(x.z, x.w, b1, b2);
        reinterpret_cast<float4*>(z)[p] = make_float4(a1, a2, b1, b2);
    }
}

cudaError_t launch_noise(int n, uint32_t m, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1, float* z,
                         uint32_t* raw, cudaStream_t st) {
    const int pairs = n * n / 2;
    noise_kernel<<<(pairs + 255) / 256, 256, 0, st>>>(n, m, c2, c3, k0, k1, z, raw);
    return cudaGetLastError();
}

// -------------------------------------------- statically allocated scratch
// Scratch for the per-slot partial sums of mlmc_dk_run_level_static, whose
// callers cannot allocate device memory.  Every GPU that loads the library
// holds this array until the process exits; all calls share it.
static __device__ __align__(256) double g_static_partials[kStaticScratchDoubles];

namespace {
constexpr int kMaxDevices = 64;
double* g_static_ptr[kMaxDevices] = {};
std::atomic<int> g_static_ready[kMaxDevices];
std::mutex g_static_mutex;
}  // namespace

cudaError_t static_scratch(double** out, size_t* capacity) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!g_static_ready[dev].load(std::memory_order_acquire)) {
        // Set-up, once per device, with that device current: in host code the
        // array's name is only a host-side stand-in, so the kernels get the
        // device address from the runtime.
        std::lock_guard<std::mutex> lock(g_static_mutex);
        if (!g_static_ready[dev].load(std::memory_order_relaxed)) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_partials);
            if (e != cudaSuccess) return e;
            g_static_ptr[dev] = static_cast<double*>(p);
            g_static_ready[dev].store(1, std::memory_order_release);
        }
    }
    *out = g_static_ptr[dev];
    *capacity = kStaticScratchDoubles;
    return cudaSuccess;
}

// ------------------------------------------------------------------ dispatch
template <class S>
struct Kern {
    static size_t smem_bytes(int stride) { return S::fixed_smem() + sizeof(double) * S::SLOTS_PER_CTA * stride; }

    static cudaError_t info(int stride, VariantInfo* vi) {
        auto fn = level_kernel<S>;
        const size_t smax = smem_bytes(kMaxStride);
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
        if (e != cudaSuccess) return e;
        if (S::CL > 1) {
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
        int dev = 0, sms = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        vi->supported = 1;
        vi->threads = S::THREADS;
        vi->cluster = S::CL;
        vi->slots_per_cta = S::SLOTS_PER_CTA;
        vi->smem = smem_bytes(stride);
        if (S::CL == 1) {
            int nb = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, S::THREADS, vi->smem);
            if (e != cudaSuccess) return e;
            vi->max_ctas = nb * sms;
        } else {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(S::CL * sms);
            cfg.blockDim = dim3(S::THREADS);
            cfg.dynamicSmemBytes = vi->smem;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = S::CL;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int ncl = 0;
            e = cudaOccupancyMaxActiveClusters(&ncl, fn, &cfg);
            if (e != cudaSuccess) return e;
            vi->max_ctas = ncl * S::CL;
        }
        return vi->max_ctas > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
    }

    static cudaError_t launch(const KArgs& a, int n_ctas, cudaStream_t st, int priority) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(n_ctas);
        cfg.blockDim = dim3(S::THREADS);
        cfg.dynamicSmemBytes = smem_bytes(a.slot_stride);
        cfg.stream = st;
        cudaLaunchAttribute at[2];
        int na = 0;
        if (S::CL > 1) {
            at[na].id = cudaLaunchAttributeClusterDimension;
            at[na].val.clusterDim.x = S::CL;
            at[na].val.clusterDim.y = 1;
            at[na].val.clusterDim.z = 1;
            ++na;
        }
        if (priority != 0) {
            at[na].id = cudaLaunchAttributePriority;
            at[na].val.priority = priority;
            ++na;
        }
        cfg.attrs = na ? at : nullptr;
        cfg.numAttrs = na;
        return cudaLaunchKernelEx(&cfg, level_kernel<S>, a);
    }
};

// Kernel variants: fine size n, lane block C x R coarse cells (2R x 2C fine),
// cluster size.  Every entry keeps the whole state in registers; the first
// entry for each n is the default, the others are candidates for the tuner.
#define DK_VARIANTS(X) \
    X(4, 1, 1, 1)      \
    X(8, 1, 1, 1)      \
    X(16, 1, 2, 1)     \
    X(16, 2, 2, 1)     \
    X(16, 1, 1, 1)     \
    X(32, 2, 2, 1)     \
    X(32, 1, 2, 1)     \
    X(32, 2, 1, 1)     \
    X(64, 2, 2, 1)     \
    X(64, 4, 2, 1)     \
    X(64, 2, 1, 1)     \
    X(64, 4, 1, 1)     \
    X(128, 2, 2, 2)    \
    X(128, 4, 1, 2)    \
    X(128, 2, 1, 4)    \
    X(256, 4, 2, 8)    \
    X(256, 4, 1, 8)

namespace {
struct VariantEntry {
    int n, C, R, CL;
    cudaError_t (*info)(bool coupled, int stride, VariantInfo* vi);
    cudaError_t (*launch)(bool coupled, const KArgs& a, int n_ctas, cudaStream_t st, int priority);
};

template <int NF, int C, int R, int CL, bool FL>
cudaError_t variant_info_fn(bool coupled, int stride, VariantInfo* vi) {
    return coupled ? Kern<Shape<NF, C, R, CL, true, FL>>::info(stride, vi)
                   : Kern<Shape<NF, C, R, CL, false, FL>>::info(stride, vi);
}

template <int NF, int C, int R, int CL, bool FL>
cudaError_t variant_launch_fn(bool coupled, const KArgs& a, int n_ctas, cudaStream_t st, int priority) {
    return coupled ? Kern<Shape<NF, C, R, CL, true, FL>>::launch(a, n_ctas, st, priority)
                   : Kern<Shape<NF, C, R, CL, false, FL>>::launch(a, n_ctas, st, priority);
}

#define DK_ENTRY(NF, C, R, CL) \
    {NF, C, R, CL, variant_info_fn<NF, C, R, CL, false>, variant_launch_fn<NF, C, R, CL, false>},
const VariantEntry kVariants[] = {DK_VARIANTS(DK_ENTRY)};
#undef DK_ENTRY
// Fluctuation-state builds: one lane-block shape per grid size up to 128^2
// (the grids of the high-particle-number hierarchies that need them).
#define DK_FLUCT_VARIANTS(X) \
    X(4, 1, 1, 1)            \
    X(8, 1, 1, 1)            \
    X(16, 1, 2, 1)           \
    X(32, 2, 2, 1)           \
    X(64, 2, 2, 1)           \
    X(128, 2, 2, 2)
#define DK_ENTRY(NF, C, R, CL) \
    {NF, C, R, CL, variant_info_fn<NF, C, R, CL, true>, variant_launch_fn<NF, C, R, CL, true>},
const VariantEntry kFluctVariants[] = {DK_FLUCT_VARIANTS(DK_ENTRY)};
#undef DK_ENTRY

const VariantEntry* find_variant(int n, int idx, bool fluct) {
    const VariantEntry* tab = fluct ? kFluctVariants : kVariants;
    const int count = fluct ? (int)(sizeof(kFluctVariants) / sizeof(kFluctVariants[0]))
                            : (int)(sizeof(kVariants) / sizeof(kVariants[0]));
    int k = 0;
    for (int i = 0; i < count; ++i)
        if (tab[i].n == n && k++ == idx) return &tab[i];
    return nullptr;
}
}  // namespace

int variant_count(int n, bool fluct) {
    int k = 0;
    while (find_variant(n, k, fluct)) ++k;
    return k;
}

cudaError_t variant_info(int n, bool coupled, int stride, int idx, VariantInfo* out, bool fluct) {
    *out = VariantInfo{};
    const VariantEntry* v = find_variant(n, idx, fluct);
    if (!v) return cudaSuccess;   // supported = 0
    cudaError_t e = v->info(coupled, stride, out);
    out->C = v->C;
    out->R = v->R;
    return e;
}

cudaError_t launch_level(int n, bool coupled, int idx, const KArgs& a, int n_ctas, cudaStream_t st, int priority,
                         bool fluct) {
    const VariantEntry* v = find_variant(n, idx, fluct);
    if (!v) return cudaErrorInvalidValue;
    return v->launch(coupled, a, n_ctas, st, priority);
}

cudaError_t launch_reduce(const double* partials, int n_slots, int slot_stride, double* out, cudaStream_t st) {
    reduce_kernel<<<slot_stride, 256, 0, st>>>(partials, n_slots, out);
    return cudaGetLastError();
}

cudaError_t launch_add_sums(double* out, const double* in, int slot_stride, cudaStream_t st) {
    add_sums_kernel<<<1, 256, 0, st>>>(out, in, slot_stride);
    return cudaGetLastError();
}

}  // namespace dk
