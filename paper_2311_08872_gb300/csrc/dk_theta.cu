// Theta-scheme sample kernel for sm_103a: Eq. (FullyDiscreteDK) with an
// implicit diffusion weight b0 > 0 (b1 = 1 - b0; Definition 2.1, the operator
// A_h of Appendix C), for the NN-coupled pair of Section 3.2 on grids up to
// 64 x 64.
//
// Step.  Subtracting (I - b0 tau/2 Delta_h) rho^(m-1) from both sides of the
// scheme gives the increment
//     rho^m - rho^(m-1) = H (tau/2 Delta_h rho^(m-1) + xi^(m-1)),
//     H = (I - b0 tau/2 Delta_h)^(-1) = (I + alpha L)^(-1),  alpha = b0 tau/(2 h^2),
// with L a = 4 a(x) - sum of the four neighbours (= -h^2 Delta_h) and xi the
// explicit noise divergence.  The bracket is the backward difference of a
// face flux F_r (diffusion flux across the face x -> x + e_r plus the two noise
// transfers G_r(x) + G_r(x + e_r) of the central difference), and H commutes
// with every periodic difference operator, so the increment is the backward
// difference of H F_r = F_r + u_r with (I + alpha L) u_r = -alpha L F_r.
// F_r is exact in 32/64-bit fixed point as in the explicit kernels; only the
// correction u_r is computed in FP32, by K steps of Chebyshev iteration on the
// spectrum [1, 1 + 8 alpha] of I + alpha L (K fixed on the host from the
// Chebyshev error bound), and rounded once.  Adding the integer face fluxes
// keeps sum_x q invariant bit for bit, as in the explicit kernels.  K = 0
// (b0 = 0) is exactly the explicit step.
//
// Work decomposition.  One CTA holds SPB samples; each sample uses (n/2)^2
// threads, thread t owning coarse cell t and the 2 x 2 block of fine cells to
// its right-most side (the coupling block of Section 3.2), so the coupled
// coarse increment is summed in the thread's registers.  The fine state and
// every Chebyshev operand stay in registers: a coarse row of blocks is a
// segment of n/2 consecutive lanes, so left / right neighbours come by warp
// shuffles (the segment wrap is the periodic wrap) and only the top and
// bottom rows of each block pass through shared memory for the blocks above
// and below (contiguous 8- and 16-byte accesses), one barrier per Chebyshev
// step.  The coarse step (1/16 of the work) keeps its state and operands in
// shared memory.
#include <cooperative_groups.h>

#include "dk_device.cuh"
#include "dk_kernels.h"

namespace dk {
namespace {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kRed = 2 * kMaxObs + 2;   // reduced values per sample

template <int N_>
struct TShape {
    static constexpr int N = N_, NC = N / 2;
    static constexpr int TPS = NC * NC;                    // threads per sample
    static constexpr int THREADS = TPS >= 128 ? TPS : 128;
    static constexpr int SPB = THREADS / TPS;              // samples per CTA
    // per sample: four planes of n^2 words, coarse state
    static constexpr size_t SAMPLE_BYTES = sizeof(int32_t) * (N * N * 4 + NC * NC);
    static size_t smem(int slot_stride) {
        return SAMPLE_BYTES * SPB + sizeof(double) * ((THREADS + 31) / 32) * kRed +
               sizeof(double) * SPB * slot_stride;
    }
};

__device__ __forceinline__ int32_t edge_flux64(long long A, int32_t d) {
    return static_cast<int32_t>((A * static_cast<long long>(d) + 0x80000000LL) >> 32);
}

__device__ __forceinline__ float as_f(int32_t v) { return __int_as_float(v); }
__device__ __forceinline__ int32_t as_i(float v) { return __float_as_int(v); }

// One step of the theta-scheme on an NN x NN periodic grid for the NCELL cells
// (row[i], col[i]) of this thread.  On entry sq holds the state of every cell
// and P0 / P2 the noise transfers G_1 / G_2 of every cell (as integers),
// published by a barrier.  On exit q and sq hold the new state, published by a
// barrier.  P0..P3 are NN x NN scratch planes.
template <int NN, int NCELL>
__device__ __forceinline__ void theta_step(int32_t (&q)[NCELL], const int (&row)[NCELL], const int (&col)[NCELL],
                                           int32_t* sq, float* P0, float* P1, float* P2, float* P3, long long A,
                                           const TArgs& t, unsigned& bad) {
    int idx[NCELL], dn[NCELL], rt[NCELL], up[NCELL], lf[NCELL];
#pragma unroll
    for (int i = 0; i < NCELL; ++i) {
        idx[i] = row[i] * NN + col[i];
        dn[i] = ((row[i] + 1) % NN) * NN + col[i];
        up[i] = ((row[i] + NN - 1) % NN) * NN + col[i];
        rt[i] = row[i] * NN + (col[i] + 1) % NN;
        lf[i] = row[i] * NN + (col[i] + NN - 1) % NN;
    }
    // face fluxes across x -> x + e_1 (down) and x -> x + e_2 (right), exact
    long long F1[NCELL], F2[NCELL];
#pragma unroll
    for (int i = 0; i < NCELL; ++i) {
        const int32_t g1 = as_i(P0[idx[i]]), g2 = as_i(P2[idx[i]]);
        F1[i] = (long long)edge_flux64(A, sq[dn[i]] - q[i]) + g1 + as_i(P0[dn[i]]);
        F2[i] = (long long)edge_flux64(A, sq[rt[i]] - q[i]) + g2 + as_i(P2[rt[i]]);
    }
    float u1[NCELL], u2[NCELL];
#pragma unroll
    for (int i = 0; i < NCELL; ++i) u1[i] = u2[i] = 0.f;
    float* out1 = P1;   // plane that receives the corrected fluxes
    float* out2 = P3;
    if (t.K > 0) {
        // right-hand side -alpha L F and the first Chebyshev direction (the
        // barrier after the F planes also orders every read of the G planes
        // before the direction overwrites them)
#pragma unroll
        for (int i = 0; i < NCELL; ++i) {
            P1[idx[i]] = static_cast<float>(F1[i]);
            P3[idx[i]] = static_cast<float>(F2[i]);
        }
        __syncthreads();
        float r1[NCELL], r2[NCELL], d1[NCELL], d2[NCELL];
#pragma unroll
        for (int i = 0; i < NCELL; ++i) {
            const float f1 = P1[idx[i]], f2 = P3[idx[i]];
            const float l1 = 4.f * f1 - P1[up[i]] - P1[dn[i]] - P1[lf[i]] - P1[rt[i]];
            const float l2 = 4.f * f2 - P3[up[i]] - P3[dn[i]] - P3[lf[i]] - P3[rt[i]];
            r1[i] = -t.alpha * l1;
            r2[i] = -t.alpha * l2;
            d1[i] = r1[i] * t.inv_theta;
            d2[i] = r2[i] * t.inv_theta;
            P0[idx[i]] = d1[i];
            P2[idx[i]] = d2[i];
        }
        __syncthreads();
        float *c1p = P0, *c2p = P2, *n1p = P1, *n2p = P3;   // current / next direction planes
        const float diag = 1.f + 4.f * t.alpha;
        for (int k = 0; k < t.K; ++k) {
#pragma unroll
            for (int i = 0; i < NCELL; ++i) {
                const float a1 = diag * d1[i] - t.alpha * (c1p[up[i]] + c1p[dn[i]] + c1p[lf[i]] + c1p[rt[i]]);
                const float a2 = diag * d2[i] - t.alpha * (c2p[up[i]] + c2p[dn[i]] + c2p[lf[i]] + c2p[rt[i]]);
                u1[i] += d1[i];
                u2[i] += d2[i];
                r1[i] -= a1;
                r2[i] -= a2;
            }
            if (k + 1 < t.K) {
                const float ca = t.c1[k], cb = t.c2[k];
#pragma unroll
                for (int i = 0; i < NCELL; ++i) {
                    d1[i] = ca * d1[i] + cb * r1[i];
                    d2[i] = ca * d2[i] + cb * r2[i];
                    n1p[idx[i]] = d1[i];
                    n2p[idx[i]] = d2[i];
                }
                __syncthreads();
                float* s1 = c1p; c1p = n1p; n1p = s1;
                float* s2 = c2p; c2p = n2p; n2p = s2;
            }
        }
        // the planes not read by the last Chebyshev step take the result
        out1 = n1p;
        out2 = n2p;
    }
    long long H1[NCELL], H2[NCELL];
#pragma unroll
    for (int i = 0; i < NCELL; ++i) {
        H1[i] = F1[i] + __float2ll_rn(u1[i]);
        H2[i] = F2[i] + __float2ll_rn(u2[i]);
        bad |= (H1[i] != (long long)(int32_t)H1[i]) | (H2[i] != (long long)(int32_t)H2[i]);
        out1[idx[i]] = as_f(static_cast<int32_t>(H1[i]));
        out2[idx[i]] = as_f(static_cast<int32_t>(H2[i]));
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NCELL; ++i) {
        const long long v = (long long)q[i] + (H1[i] - as_i(out1[up[i]])) + (H2[i] - as_i(out2[lf[i]]));
        bad |= (unsigned)((v >= (1LL << 30)) | (v <= -(1LL << 30)));
        q[i] = static_cast<int32_t>(v);
        sq[idx[i]] = q[i];
    }
    __syncthreads();
}

// Left / right neighbour values along a coarse row of W blocks (W lanes).
template <int W, class T>
__device__ __forceinline__ T from_left(T v, int l) {
    return __shfl_sync(kFullMask, v, (l + W - 1) % W, W);
}
template <int W, class T>
__device__ __forceinline__ T from_right(T v, int l) {
    return __shfl_sync(kFullMask, v, (l + 1) % W, W);
}

// A plane of a block field: the top rows of all blocks, then the bottom rows
// ([NC^2] float2 each, block index I1 NC + I2).
template <int NC>
struct Plane {
    float2* top;
    float2* bot;
    __device__ __forceinline__ explicit Plane(float* base) : top(reinterpret_cast<float2*>(base)), bot(top + NC * NC) {}
    __device__ __forceinline__ void put(int qi, const float (&v)[4]) const {
        top[qi] = make_float2(v[0], v[1]);
        bot[qi] = make_float2(v[2], v[3]);
    }
};

// Sum of the four periodic neighbours of each cell of the 2 x 2 block v
// (cells: 0 top-left, 1 top-right, 2 bottom-left, 3 bottom-right), the rows
// above / below from the blocks qa / qb of plane P, the columns by shuffles.
template <int NC>
__device__ __forceinline__ void neighbour_sum(const float (&v)[4], const Plane<NC>& P, int qa, int qb, int l,
                                              float (&s)[4]) {
    const float2 ab = P.bot[qa], bl = P.top[qb];
    const float l0 = from_left<NC>(v[1], l), l2 = from_left<NC>(v[3], l);
    const float r1 = from_right<NC>(v[0], l), r3 = from_right<NC>(v[2], l);
    s[0] = (ab.x + v[2]) + (l0 + v[1]);
    s[1] = (ab.y + v[3]) + (v[0] + r1);
    s[2] = (v[0] + bl.x) + (l2 + v[3]);
    s[3] = (v[1] + bl.y) + (v[2] + r3);
}

// One fine theta step for this thread's 2 x 2 block (coarse cell (I1, I2),
// lane l = I2 of its row segment); B[0..3] are four n^2-word planes.  Enters
// and leaves with the planes free (a barrier at the end).
template <int N>
__device__ __forceinline__ void theta_fine_step(int32_t (&q)[4], const int32_t (&G1)[4], const int32_t (&G2)[4],
                                                int I1, int I2, float* const (&B)[4], long long A, const TArgs& t,
                                                unsigned& bad) {
    constexpr int NC = N / 2;
    const int qi = I1 * NC + I2;
    const int qa = ((I1 + NC - 1) % NC) * NC + I2;   // block above
    const int qb = ((I1 + 1) % NC) * NC + I2;        // block below
    const int l = I2;
    // ---- exact face fluxes: the row below from the block below, the column right by shuffles
    int4* Q = reinterpret_cast<int4*>(B[0]);
    Q[qi] = make_int4(q[0], q[1], G1[0], G1[1]);
    __syncthreads();
    const int4 bq = Q[qb];
    const int32_t qr1 = from_right<NC>(q[0], l), qr3 = from_right<NC>(q[2], l);
    const int32_t gr1 = from_right<NC>(G2[0], l), gr3 = from_right<NC>(G2[2], l);
    const int32_t qdn[4] = {q[2], q[3], bq.x, bq.y}, gdn[4] = {G1[2], G1[3], bq.z, bq.w};
    const int32_t qrt[4] = {q[1], qr1, q[3], qr3}, grt[4] = {G2[1], gr1, G2[3], gr3};
    int32_t F1[4], F2[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const long long f1 = (long long)edge_flux64(A, qdn[c] - q[c]) + G1[c] + gdn[c];
        const long long f2 = (long long)edge_flux64(A, qrt[c] - q[c]) + G2[c] + grt[c];
        bad |= (unsigned)((f1 != (long long)(int32_t)f1) | (f2 != (long long)(int32_t)f2));
        F1[c] = static_cast<int32_t>(f1);
        F2[c] = static_cast<int32_t>(f2);
    }
    float u1[4] = {0.f, 0.f, 0.f, 0.f}, u2[4] = {0.f, 0.f, 0.f, 0.f};
    float* hplane = B[1];   // plane that carries the corrected fluxes of the bottom rows
    if (t.K > 0) {
        // ---- right-hand side -alpha L F and the first Chebyshev direction
        float f1[4], f2[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            f1[c] = static_cast<float>(F1[c]);
            f2[c] = static_cast<float>(F2[c]);
        }
        const Plane<NC> PF1(B[1]), PF2(B[2]);
        PF1.put(qi, f1);
        PF2.put(qi, f2);
        __syncthreads();   // also orders every read of B[0] before it is reused below
        float s1[4], s2[4], r1[4], r2[4], d1[4], d2[4];
        neighbour_sum<NC>(f1, PF1, qa, qb, l, s1);
        neighbour_sum<NC>(f2, PF2, qa, qb, l, s2);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            r1[c] = -t.alpha * (4.f * f1[c] - s1[c]);
            r2[c] = -t.alpha * (4.f * f2[c] - s2[c]);
            d1[c] = r1[c] * t.inv_theta;
            d2[c] = r2[c] * t.inv_theta;
        }
        float* cur1 = B[3];
        float* cur2 = B[0];
        float* nxt1 = B[1];
        float* nxt2 = B[2];
        Plane<NC>(cur1).put(qi, d1);
        Plane<NC>(cur2).put(qi, d2);
        __syncthreads();
        const float diag = 1.f + 4.f * t.alpha;
        for (int k = 0; k < t.K; ++k) {
            neighbour_sum<NC>(d1, Plane<NC>(cur1), qa, qb, l, s1);
            neighbour_sum<NC>(d2, Plane<NC>(cur2), qa, qb, l, s2);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                u1[c] += d1[c];
                u2[c] += d2[c];
                r1[c] -= diag * d1[c] - t.alpha * s1[c];
                r2[c] -= diag * d2[c] - t.alpha * s2[c];
            }
            if (k + 1 < t.K) {
                const float ca = t.c1[k], cb = t.c2[k];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    d1[c] = ca * d1[c] + cb * r1[c];
                    d2[c] = ca * d2[c] + cb * r2[c];
                }
                Plane<NC>(nxt1).put(qi, d1);
                Plane<NC>(nxt2).put(qi, d2);
                __syncthreads();
                float* x = cur1; cur1 = nxt1; nxt1 = x;
                x = cur2; cur2 = nxt2; nxt2 = x;
            }
        }
        hplane = nxt1;   // not read by the last Chebyshev step
    }
    // ---- corrected fluxes, rounded once; the update adds integer face fluxes
    int32_t H1[4], H2[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const long long h1 = (long long)F1[c] + __float2ll_rn(u1[c]);
        const long long h2 = (long long)F2[c] + __float2ll_rn(u2[c]);
        bad |= (unsigned)((h1 != (long long)(int32_t)h1) | (h2 != (long long)(int32_t)h2));
        H1[c] = static_cast<int32_t>(h1);
        H2[c] = static_cast<int32_t>(h2);
    }
    int2* Hb = reinterpret_cast<int2*>(hplane);
    Hb[qi] = make_int2(H1[2], H1[3]);
    __syncthreads();
    const int2 ha = Hb[qa];
    const int32_t hl0 = from_left<NC>(H2[1], l), hl2 = from_left<NC>(H2[3], l);
    const int32_t h1up[4] = {ha.x, ha.y, H1[0], H1[1]}, h2lf[4] = {hl0, H2[0], hl2, H2[2]};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const long long v = (long long)q[c] + ((long long)H1[c] - h1up[c]) + ((long long)H2[c] - h2lf[c]);
        bad |= (unsigned)((v >= (1LL << 30)) | (v <= -(1LL << 30)));
        q[c] = static_cast<int32_t>(v);
    }
    __syncthreads();
}

template <int N, bool CPL>
__global__ void __launch_bounds__(TShape<N>::THREADS) theta_kernel(const KArgs a, const TArgs t) {
    using S = TShape<N>;
    constexpr int NC = S::NC, TPS = S::TPS, SPB = S::SPB, THREADS = S::THREADS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    const int sl = tid / TPS, lt = tid % TPS;   // sample slot in the CTA, thread within the sample
    unsigned char* base = smem_raw + S::SAMPLE_BYTES * sl;
    float* P0 = reinterpret_cast<float*>(base);
    float* P1 = P0 + N * N;
    float* P2 = P1 + N * N;
    float* P3 = P2 + N * N;
    int32_t* sqc = reinterpret_cast<int32_t*>(P3 + N * N);
    double* red = reinterpret_cast<double*>(smem_raw + S::SAMPLE_BYTES * SPB);
    double* acc = red + ((THREADS + 31) / 32) * kRed;
    for (int i = tid; i < SPB * a.slot_stride; i += THREADS) acc[i] = 0.0;
    float* const planes[4] = {P0, P1, P2, P3};

    const int I1 = lt / NC, I2 = lt % NC;   // coarse cell; fine block rows 2 I1 + v1, cols 2 I2 + v2
    const int crow[1] = {I1}, ccol[1] = {I2};
    const int f00 = (2 * I1) * N + 2 * I2;  // fine index of the block's top-left cell
    const int fidx[4] = {f00, f00 + 1, f00 + N, f00 + N + 1};
    const uint32_t p_top = static_cast<uint32_t>(f00 >> 1);
    const uint32_t p_bot = static_cast<uint32_t>((f00 + N) >> 1);

    const long long n_slots = (long long)gridDim.x * SPB;
    const long long slot = (long long)blockIdx.x * SPB + sl;
    const long long cta_slot0 = (long long)blockIdx.x * SPB;
    const long long iters = a.count > cta_slot0 ? (a.count - cta_slot0 + n_slots - 1) / n_slots : 0;
    unsigned bad = 0;
    __syncthreads();

    for (long long it = 0; it < iters; ++it) {
        const long long idx = slot + it * n_slots;
        const bool active = idx < a.count;
        const long long sid = a.first + (active ? idx : 0);
        const uint32_t c2 = static_cast<uint32_t>(sid);
        const uint32_t c3 = a.tag | ((static_cast<uint32_t>(static_cast<unsigned long long>(sid) >> 32) & 0xffffu) << 16);

        int32_t q[4], qc[1] = {0};
#pragma unroll
        for (int i = 0; i < 4; ++i) q[i] = a.q0f[fidx[i]];
        float zt0 = 0.f, zt1 = 0.f;
        if constexpr (CPL) {
            qc[0] = a.q0c[lt];
            sqc[lt] = qc[0];
        }
        __syncthreads();

        for (int m = 0; m < a.M; ++m) {
            // ---- noise of the fine block: Philox4x32-10 per horizontal cell pair, Box--Muller
            int32_t G1[4], G2[4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint4 x = philox10(make_uint4(h ? p_bot : p_top, static_cast<uint32_t>(m), c2, c3), a.key0, a.key1);
                float ra, ca, sa, rb, cb, sb;
                box_muller_polar(x.x, x.y, ra, ca, sa);
                box_muller_polar(x.z, x.w, rb, cb, sb);
                const float ta = noise_amp(q[2 * h], a.gf) * ra;
                const float tb = noise_amp(q[2 * h + 1], a.gf) * rb;
                G1[2 * h] = __float2int_rn(ta * ca);
                G2[2 * h] = __float2int_rn(ta * sa);
                G1[2 * h + 1] = __float2int_rn(tb * cb);
                G2[2 * h + 1] = __float2int_rn(tb * sb);
                if constexpr (CPL) {
                    zt0 = fmaf(rb, cb, fmaf(ra, ca, zt0));
                    zt1 = fmaf(rb, sb, fmaf(ra, sa, zt1));
                }
            }
            theta_fine_step<N>(q, G1, G2, I1, I2, planes, t.Af64, t, bad);

            if constexpr (CPL) {
                if ((m & 3) == 3) {
                    // coupled coarse step: 1/4 of the 16 summed fine normals
                    const float s = noise_amp(qc[0], a.gc);
                    P0[lt] = as_f(__float2int_rn(s * zt0));
                    P2[lt] = as_f(__float2int_rn(s * zt1));
                    zt0 = zt1 = 0.f;
                    __syncthreads();
                    theta_step<NC, 1>(qc, crow, ccol, sqc, P0, P1, P2, P3, t.Ac64, t, bad);
                }
            }
        }

        // ---- observables: fluctuation sums against the fixed-point mean field (FP64), mass
        double v[kRed];
        {
            long long mf = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) mf += q[i];
            v[2 * kMaxObs] = static_cast<double>(mf);
            v[2 * kMaxObs + 1] = CPL ? static_cast<double>(qc[0]) : 0.0;
#pragma unroll
            for (int k = 0; k < kMaxObs; ++k) {
                double sf = 0.0, sc = 0.0;
                if (k < a.n_obs) {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        sf += static_cast<double>(q[i] - a.qbf[fidx[i]]) * t.phif64[(size_t)k * N * N + fidx[i]];
                    if constexpr (CPL) sc = static_cast<double>(qc[0] - a.qbc[lt]) * t.phic64[(size_t)k * NC * NC + lt];
                }
                v[k] = sf;
                v[kMaxObs + k] = sc;
            }
        }
        bool leader;
        if constexpr (TPS < 32) {
#pragma unroll
            for (int off = TPS / 2; off >= 1; off >>= 1)
#pragma unroll
                for (int i = 0; i < kRed; ++i) v[i] += __shfl_xor_sync(kFullMask, v[i], off, TPS);
            leader = lt == 0;
        } else {
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1)
#pragma unroll
                for (int i = 0; i < kRed; ++i) v[i] += __shfl_xor_sync(kFullMask, v[i], off);
            if ((tid & 31) == 0)
#pragma unroll
                for (int i = 0; i < kRed; ++i) red[(tid >> 5) * kRed + i] = v[i];
            __syncthreads();
            leader = lt == 0;
            if (leader) {
                for (int w = 1; w < TPS / 32; ++w)
#pragma unroll
                    for (int i = 0; i < kRed; ++i) v[i] += red[((tid >> 5) + w) * kRed + i];
            }
        }

        // ---- FP64 quantities and moment sums (one thread per sample)
        if (leader && active) {
            double Df[kMaxObs], Dc[kMaxObs];
#pragma unroll
            for (int k = 0; k < kMaxObs; ++k) {
                Df[k] = a.dscale_f * v[k] + a.delta_f[k];
                Dc[k] = CPL ? a.dscale_c * v[kMaxObs + k] + a.delta_c[k] : 0.0;
            }
            double* A = acc + sl * a.slot_stride;
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
                o[2 * a.n_obs] = v[2 * kMaxObs] * a.dscale_f;
                o[2 * a.n_obs + 1] = CPL ? v[2 * kMaxObs + 1] * a.dscale_c : 0.0;
            }
        }
        __syncthreads();   // the reduction scratch and the state planes are reused by the next sample
    }
    if (bad) atomicOr(a.err, kErrRange);

    // ---- per-slot partial sums to global scratch, entry-major [stride][n_slots]
    __syncthreads();
    for (int i = tid; i < SPB * a.slot_stride; i += THREADS) {
        const int s = i / a.slot_stride, e = i % a.slot_stride;
        a.partials[(size_t)e * n_slots + cta_slot0 + s] = acc[i];
    }
}

// ---------------------------------------------------------------------------
// Grids beyond one CTA (128 x 128): a thread-block cluster of CL CTAs per
// sample, CTA `rank` holding the band of BR = NC/CL block rows (its threads
// own those rows' 2 x 2 blocks as above).  The block fields live in the band's
// shared memory with the same layout in every CTA; the rows just above and
// below the band are read from the neighbouring CTAs' shared memory
// (distributed shared memory), and every barrier that orders a plane's writes
// before its reads is a cluster barrier.  The arithmetic is the one-CTA
// kernel's, so both give the same integer paths.
// ---------------------------------------------------------------------------
namespace cg = cooperative_groups;

template <int N, int CL, int NB>
struct CShape {
    static constexpr int NC = N / 2, BR = NC / CL;          // block rows per CTA
    static constexpr int RT = NC / NB;                      // threads per block row (NB blocks each)
    static constexpr int THREADS = BR * RT;
    static constexpr int BAND = BR * NC;                    // blocks (= coarse cells) per CTA
    static_assert(NC % CL == 0 && NC % NB == 0 && THREADS <= 1024 && RT % 32 == 0, "band shape");
    // four block planes of BAND x 16 bytes (top and bottom rows, or an int4 per block),
    // the coarse state of the band, reduction scratch
    static size_t smem(int slot_stride) {
        return 4 * sizeof(float) * 4 * BAND + sizeof(int32_t) * BAND + sizeof(double) * (THREADS / 32) * kRed +
               sizeof(double) * kRed + sizeof(double) * slot_stride;
    }
};

// Pointer into the shared memory of cluster rank r (this CTA's own when r == rank).
template <class T>
__device__ __forceinline__ T* band_at(T* local, int r, int rank) {
    if (r == rank) return local;
    return cg::this_cluster().map_shared_rank(local, r);
}

// Neighbours of block (or coarse cell) (lr, I2) of a band of BR rows x NC:
// left / right in the same row (periodic), above / below in the row before /
// after, in the neighbouring CTA for the band's first / last row (periodic
// over the cluster).
template <int NC, int BR>
struct BandNbr {
    int lq, il, ir, ia, ib, ra, rb, rank;
    BandNbr() = default;
    __device__ __forceinline__ BandNbr(int lr, int I2, int rank_, int cl) : rank(rank_) {
        lq = lr * NC + I2;
        il = lr * NC + (I2 + NC - 1) % NC;
        ir = lr * NC + (I2 + 1) % NC;
        if (lr > 0) { ia = lq - NC; ra = rank; } else { ia = (BR - 1) * NC + I2; ra = (rank + cl - 1) % cl; }
        if (lr < BR - 1) { ib = lq + NC; rb = rank; } else { ib = I2; rb = (rank + 1) % cl; }
    }
    template <class T> __device__ __forceinline__ T above(T* p) const { return band_at(p, ra, rank)[ia]; }
    template <class T> __device__ __forceinline__ T below(T* p) const { return band_at(p, rb, rank)[ib]; }
    template <class T> __device__ __forceinline__ T left(const T* p) const { return p[il]; }
    template <class T> __device__ __forceinline__ T right(const T* p) const { return p[ir]; }
};

// Split cluster barrier of a plane exchange.  After writing its part of a
// plane a thread arrives (release); a CTA barrier then publishes the plane
// inside the CTA.  The warps of the band's first and last block row, which
// read the neighbouring CTAs' rows, wait (acquire) at once; the other warps
// only read rows of their own CTA and defer the wait until just before they
// next write a plane that other CTAs read, so the cluster barrier's latency
// is spent on their arithmetic.  A thread always waits once between two
// arrivals, so the barrier is never more than one phase ahead of it.
struct ClPhase {
    bool edge;
    bool pend = false;
    __device__ __forceinline__ explicit ClPhase(bool edge_) : edge(edge_) {}
    __device__ __forceinline__ static void arrive() {
        asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    }
    __device__ __forceinline__ static void wait() {
        asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
    // before writing a plane that other CTAs read (or before a full barrier)
    __device__ __forceinline__ void settle() {
        if (pend) {
            wait();
            pend = false;
        }
    }
    __device__ __forceinline__ void publish() {
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

// Sum of the four neighbours of each cell of block v = (top-left, top-right,
// bottom-left, bottom-right), from the blocks above / below / left / right,
// in the one-CTA kernel's order of additions.
__device__ __forceinline__ void nsum4(const float (&v)[4], float4 A, float4 Bv, float4 L, float4 R, float (&s)[4]) {
    s[0] = (A.z + v[2]) + (L.y + v[1]);
    s[1] = (A.w + v[3]) + (v[0] + R.x);
    s[2] = (v[0] + Bv.x) + (L.w + v[3]);
    s[3] = (v[1] + Bv.y) + (v[2] + R.z);
}

template <int NC, int BR>
__device__ __forceinline__ void nsum_band(const float (&v)[4], const float4* P, const BandNbr<NC, BR>& nb,
                                          float (&s)[4]) {
    nsum4(v, nb.above(P), nb.below(P), nb.left(P), nb.right(P), s);
}

// theta_fine_step for the NB blocks of a thread in a band (B: four planes of
// one 16-byte word per block of the band; all neighbours through shared
// memory).  Every plane write is preceded by ph.settle() and followed by
// ph.publish(); the step ends with an arrival whose wait comes before the
// next plane write.
template <int NC, int BR, int NB>
__device__ __forceinline__ void theta_fine_step_cl(int32_t (&q)[NB][4], const int32_t (&G1)[NB][4],
                                                   const int32_t (&G2)[NB][4], const BandNbr<NC, BR> (&nb)[NB],
                                                   float* const (&B)[4], long long A, const TArgs& t, unsigned& bad,
                                                   ClPhase& ph) {
    // ---- exact face fluxes: the top row of the block below, the left column of the block right
    int4* Qd = reinterpret_cast<int4*>(B[0]);
    int4* Qr = reinterpret_cast<int4*>(B[3]);
    ph.settle();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        Qd[nb[b].lq] = make_int4(q[b][0], q[b][1], G1[b][0], G1[b][1]);
        Qr[nb[b].lq] = make_int4(q[b][0], q[b][2], G2[b][0], G2[b][2]);
    }
    ph.publish();
    int32_t F1[NB][4], F2[NB][4];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int4 bq = nb[b].below(Qd), rq = nb[b].right(Qr);
        const int32_t qdn[4] = {q[b][2], q[b][3], bq.x, bq.y}, gdn[4] = {G1[b][2], G1[b][3], bq.z, bq.w};
        const int32_t qrt[4] = {q[b][1], rq.x, q[b][3], rq.y}, grt[4] = {G2[b][1], rq.z, G2[b][3], rq.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const long long f1 = (long long)edge_flux64(A, qdn[c] - q[b][c]) + G1[b][c] + gdn[c];
            const long long f2 = (long long)edge_flux64(A, qrt[c] - q[b][c]) + G2[b][c] + grt[c];
            bad |= (unsigned)((f1 != (long long)(int32_t)f1) | (f2 != (long long)(int32_t)f2));
            F1[b][c] = static_cast<int32_t>(f1);
            F2[b][c] = static_cast<int32_t>(f2);
        }
    }
    float u1[NB][4], u2[NB][4];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int c = 0; c < 4; ++c) u1[b][c] = u2[b][c] = 0.f;
    float* hplane = B[1];
    if (t.K > 0) {
        float f1[NB][4], f2[NB][4];
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                f1[b][c] = static_cast<float>(F1[b][c]);
                f2[b][c] = static_cast<float>(F2[b][c]);
            }
        float4* PF1 = reinterpret_cast<float4*>(B[1]);
        float4* PF2 = reinterpret_cast<float4*>(B[2]);
        ph.settle();
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            PF1[nb[b].lq] = make_float4(f1[b][0], f1[b][1], f1[b][2], f1[b][3]);
            PF2[nb[b].lq] = make_float4(f2[b][0], f2[b][1], f2[b][2], f2[b][3]);
        }
        ph.publish();   // its wait also orders every read of B[0], B[3] before they are reused below
        float r1[NB][4], r2[NB][4], d1[NB][4], d2[NB][4];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            float s1[4], s2[4];
            nsum_band(f1[b], PF1, nb[b], s1);
            nsum_band(f2[b], PF2, nb[b], s2);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                r1[b][c] = -t.alpha * (4.f * f1[b][c] - s1[c]);
                r2[b][c] = -t.alpha * (4.f * f2[b][c] - s2[c]);
                d1[b][c] = r1[b][c] * t.inv_theta;
                d2[b][c] = r2[b][c] * t.inv_theta;
            }
        }
        float4* cur1 = reinterpret_cast<float4*>(B[3]);
        float4* cur2 = reinterpret_cast<float4*>(B[0]);
        float4* nxt1 = reinterpret_cast<float4*>(B[1]);
        float4* nxt2 = reinterpret_cast<float4*>(B[2]);
        ph.settle();
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            cur1[nb[b].lq] = make_float4(d1[b][0], d1[b][1], d1[b][2], d1[b][3]);
            cur2[nb[b].lq] = make_float4(d2[b][0], d2[b][1], d2[b][2], d2[b][3]);
        }
        ph.publish();
        const float diag = 1.f + 4.f * t.alpha;
        for (int k = 0; k < t.K; ++k) {
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                float s1[4], s2[4];
                nsum_band(d1[b], cur1, nb[b], s1);
                nsum_band(d2[b], cur2, nb[b], s2);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    u1[b][c] += d1[b][c];
                    u2[b][c] += d2[b][c];
                    r1[b][c] -= diag * d1[b][c] - t.alpha * s1[c];
                    r2[b][c] -= diag * d2[b][c] - t.alpha * s2[c];
                }
            }
            if (k + 1 < t.K) {
                const float ca = t.c1[k], cb = t.c2[k];
#pragma unroll
                for (int b = 0; b < NB; ++b)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        d1[b][c] = ca * d1[b][c] + cb * r1[b][c];
                        d2[b][c] = ca * d2[b][c] + cb * r2[b][c];
                    }
                ph.settle();
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    nxt1[nb[b].lq] = make_float4(d1[b][0], d1[b][1], d1[b][2], d1[b][3]);
                    nxt2[nb[b].lq] = make_float4(d2[b][0], d2[b][1], d2[b][2], d2[b][3]);
                }
                ph.publish();
                float4* x = cur1; cur1 = nxt1; nxt1 = x;
                x = cur2; cur2 = nxt2; nxt2 = x;
            }
        }
        hplane = reinterpret_cast<float*>(nxt1);   // not read by the last Chebyshev step
    }
    int32_t H1[NB][4], H2[NB][4];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const long long h1 = (long long)F1[b][c] + __float2ll_rn(u1[b][c]);
            const long long h2 = (long long)F2[b][c] + __float2ll_rn(u2[b][c]);
            bad |= (unsigned)((h1 != (long long)(int32_t)h1) | (h2 != (long long)(int32_t)h2));
            H1[b][c] = static_cast<int32_t>(h1);
            H2[b][c] = static_cast<int32_t>(h2);
        }
    int4* Hb = reinterpret_cast<int4*>(hplane);
    ph.settle();
#pragma unroll
    for (int b = 0; b < NB; ++b) Hb[nb[b].lq] = make_int4(H1[b][2], H1[b][3], H2[b][1], H2[b][3]);
    ph.publish();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int4 ha = nb[b].above(Hb), hl = nb[b].left(Hb);
        const int32_t h1up[4] = {ha.x, ha.y, H1[b][0], H1[b][1]}, h2lf[4] = {hl.z, H2[b][0], hl.w, H2[b][2]};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const long long v = (long long)q[b][c] + ((long long)H1[b][c] - h1up[c]) + ((long long)H2[b][c] - h2lf[c]);
            bad |= (unsigned)((v >= (1LL << 30)) | (v <= -(1LL << 30)));
            q[b][c] = static_cast<int32_t>(v);
        }
    }
    // every thread has read what it needs: arrive, wait before the next plane write
    ph.settle();
    ClPhase::arrive();
    ph.pend = true;
}

// theta_step<NC, 1> for the NB coarse cells of a thread in a band: sq the
// band's coarse state, P0 / P2 the coarse transfers G_1 / G_2 (as integers,
// published by the caller), P0..P3 band planes of one float per cell.  The
// one-CTA step's arithmetic and order of additions; plane exchanges as in the
// fine step.
template <int NC, int BR, int NB>
__device__ __forceinline__ void theta_coarse_step_cl(int32_t (&q)[NB], const BandNbr<NC, BR> (&nb)[NB], int32_t* sq,
                                                     float* P0, float* P1, float* P2, float* P3, long long A,
                                                     const TArgs& t, unsigned& bad, ClPhase& ph) {
    long long F1[NB], F2[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int idx = nb[b].lq;
        const int32_t g1 = as_i(P0[idx]), g2 = as_i(P2[idx]);
        F1[b] = (long long)edge_flux64(A, nb[b].below(sq) - q[b]) + g1 + as_i(nb[b].below(P0));
        F2[b] = (long long)edge_flux64(A, nb[b].right(sq) - q[b]) + g2 + as_i(nb[b].right(P2));
    }
    float u1[NB], u2[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) u1[b] = u2[b] = 0.f;
    float* out1 = P1;
    float* out2 = P3;
    if (t.K > 0) {
        ph.settle();
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            P1[nb[b].lq] = static_cast<float>(F1[b]);
            P3[nb[b].lq] = static_cast<float>(F2[b]);
        }
        ph.publish();   // its wait also orders every read of the G planes before they are overwritten
        float r1[NB], r2[NB], d1[NB], d2[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const BandNbr<NC, BR>& n = nb[b];
            const float f1 = P1[n.lq], f2 = P3[n.lq];
            const float l1 = 4.f * f1 - n.above(P1) - n.below(P1) - n.left(P1) - n.right(P1);
            const float l2 = 4.f * f2 - n.above(P3) - n.below(P3) - n.left(P3) - n.right(P3);
            r1[b] = -t.alpha * l1;
            r2[b] = -t.alpha * l2;
            d1[b] = r1[b] * t.inv_theta;
            d2[b] = r2[b] * t.inv_theta;
        }
        ph.settle();
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            P0[nb[b].lq] = d1[b];
            P2[nb[b].lq] = d2[b];
        }
        ph.publish();
        float *c1p = P0, *c2p = P2, *n1p = P1, *n2p = P3;
        const float diag = 1.f + 4.f * t.alpha;
        for (int k = 0; k < t.K; ++k) {
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const BandNbr<NC, BR>& n = nb[b];
                const float a1 = diag * d1[b] - t.alpha * (n.above(c1p) + n.below(c1p) + n.left(c1p) + n.right(c1p));
                const float a2 = diag * d2[b] - t.alpha * (n.above(c2p) + n.below(c2p) + n.left(c2p) + n.right(c2p));
                u1[b] += d1[b];
                u2[b] += d2[b];
                r1[b] -= a1;
                r2[b] -= a2;
            }
            if (k + 1 < t.K) {
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    d1[b] = t.c1[k] * d1[b] + t.c2[k] * r1[b];
                    d2[b] = t.c1[k] * d2[b] + t.c2[k] * r2[b];
                }
                ph.settle();
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    n1p[nb[b].lq] = d1[b];
                    n2p[nb[b].lq] = d2[b];
                }
                ph.publish();
                float* x = c1p; c1p = n1p; n1p = x;
                x = c2p; c2p = n2p; n2p = x;
            }
        }
        out1 = n1p;
        out2 = n2p;
    }
    long long H1[NB], H2[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        H1[b] = F1[b] + __float2ll_rn(u1[b]);
        H2[b] = F2[b] + __float2ll_rn(u2[b]);
        bad |= (unsigned)((H1[b] != (long long)(int32_t)H1[b]) | (H2[b] != (long long)(int32_t)H2[b]));
    }
    ph.settle();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        out1[nb[b].lq] = as_f(static_cast<int32_t>(H1[b]));
        out2[nb[b].lq] = as_f(static_cast<int32_t>(H2[b]));
    }
    ph.publish();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const long long v = (long long)q[b] + (H1[b] - as_i(nb[b].above(out1))) + (H2[b] - as_i(nb[b].left(out2)));
        bad |= (unsigned)((v >= (1LL << 30)) | (v <= -(1LL << 30)));
        q[b] = static_cast<int32_t>(v);
    }
    ph.settle();
#pragma unroll
    for (int b = 0; b < NB; ++b) sq[nb[b].lq] = q[b];
    ClPhase::arrive();
    ph.pend = true;
}

// The theta-scheme sample kernel for a cluster of CL CTAs per sample (see
// above), NB blocks of a block row per thread; a cluster is one sample
// slot of a persistent grid of clusters.
template <int N, int CL, int NB, bool CPL>
__global__ void __launch_bounds__(CShape<N, CL, NB>::THREADS, 1) theta_cluster_kernel(const KArgs a, const TArgs t) {
    using S = CShape<N, CL, NB>;
    constexpr int NC = S::NC, BR = S::BR, BAND = S::BAND, THREADS = S::THREADS, RT = S::RT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    const int rank = static_cast<int>(cg::this_cluster().block_rank());
    float* P0 = reinterpret_cast<float*>(smem_raw);
    float* P1 = P0 + 4 * BAND;
    float* P2 = P1 + 4 * BAND;
    float* P3 = P2 + 4 * BAND;
    int32_t* sqc = reinterpret_cast<int32_t*>(P3 + 4 * BAND);
    double* red = reinterpret_cast<double*>(sqc + BAND);
    double* tot = red + (THREADS / 32) * kRed;       // this CTA's band total
    double* acc = tot + kRed;                        // the slot's moment sums (rank 0)
    for (int i = tid; i < a.slot_stride; i += THREADS) acc[i] = 0.0;
    float* const planes[4] = {P0, P1, P2, P3};

    // block row within the band; the thread's blocks are columns j0, j0 + RT, ...
    // (consecutive lanes on consecutive blocks: conflict-free 16-byte plane accesses)
    const int lr = tid / RT, j0 = tid % RT;
    const int I1 = rank * BR + lr;                    // coarse row; fine block rows 2 I1 + v1, cols 2 I2 + v2
    BandNbr<NC, BR> nb[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) nb[b] = BandNbr<NC, BR>(lr, j0 + b * RT, rank, CL);
    ClPhase ph(lr == 0 || lr == BR - 1);              // the band's first and last rows read other CTAs
    int gc[NB], fidx[NB][4];
    uint32_t p_top[NB], p_bot[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int I2 = j0 + b * RT;
        gc[b] = I1 * NC + I2;                         // global coarse index
        const int f00 = (2 * I1) * N + 2 * I2;
        fidx[b][0] = f00; fidx[b][1] = f00 + 1; fidx[b][2] = f00 + N; fidx[b][3] = f00 + N + 1;
        p_top[b] = static_cast<uint32_t>(f00 >> 1);
        p_bot[b] = static_cast<uint32_t>((f00 + N) >> 1);
    }

    const long long n_slots = (long long)gridDim.x / CL;
    const long long slot = (long long)blockIdx.x / CL;
    const long long iters = a.count > slot ? (a.count - slot + n_slots - 1) / n_slots : 0;
    unsigned bad = 0;
    ph.full();

    for (long long it = 0; it < iters; ++it) {
        const long long idx = slot + it * n_slots;
        const bool active = idx < a.count;
        const long long sid = a.first + (active ? idx : 0);
        const uint32_t c2 = static_cast<uint32_t>(sid);
        const uint32_t c3 = a.tag | ((static_cast<uint32_t>(static_cast<unsigned long long>(sid) >> 32) & 0xffffu) << 16);

        int32_t q[NB][4], qc[NB];
        float zt0[NB], zt1[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
#pragma unroll
            for (int i = 0; i < 4; ++i) q[b][i] = a.q0f[fidx[b][i]];
            zt0[b] = zt1[b] = 0.f;
            qc[b] = 0;
            if constexpr (CPL) {
                qc[b] = a.q0c[gc[b]];
                sqc[nb[b].lq] = qc[b];
            }
        }
        ph.full();

        for (int m = 0; m < a.M; ++m) {
            int32_t G1[NB][4], G2[NB][4];
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint4 x = philox10(make_uint4(h ? p_bot[b] : p_top[b], static_cast<uint32_t>(m), c2, c3),
                                             a.key0, a.key1);
                    float ra, ca, sa, rb, cb, sb;
                    box_muller_polar(x.x, x.y, ra, ca, sa);
                    box_muller_polar(x.z, x.w, rb, cb, sb);
                    const float ta = noise_amp(q[b][2 * h], a.gf) * ra;
                    const float tb = noise_amp(q[b][2 * h + 1], a.gf) * rb;
                    G1[b][2 * h] = __float2int_rn(ta * ca);
                    G2[b][2 * h] = __float2int_rn(ta * sa);
                    G1[b][2 * h + 1] = __float2int_rn(tb * cb);
                    G2[b][2 * h + 1] = __float2int_rn(tb * sb);
                    if constexpr (CPL) {
                        zt0[b] = fmaf(rb, cb, fmaf(ra, ca, zt0[b]));
                        zt1[b] = fmaf(rb, sb, fmaf(ra, sa, zt1[b]));
                    }
                }
            theta_fine_step_cl<NC, BR, NB>(q, G1, G2, nb, planes, t.Af64, t, bad, ph);

            if constexpr (CPL) {
                if ((m & 3) == 3) {
                    ph.settle();
#pragma unroll
                    for (int b = 0; b < NB; ++b) {
                        const float sc = noise_amp(qc[b], a.gc);
                        P0[nb[b].lq] = as_f(__float2int_rn(sc * zt0[b]));
                        P2[nb[b].lq] = as_f(__float2int_rn(sc * zt1[b]));
                        zt0[b] = zt1[b] = 0.f;
                    }
                    ph.publish();
                    theta_coarse_step_cl<NC, BR, NB>(qc, nb, sqc, P0, P1, P2, P3, t.Ac64, t, bad, ph);
                }
            }
        }

        // ---- observables of the band, then the band totals summed on rank 0 in rank order
        double v[kRed];
        {
            long long mf = 0, mc = 0;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
#pragma unroll
                for (int i = 0; i < 4; ++i) mf += q[b][i];
                mc += qc[b];
            }
            v[2 * kMaxObs] = static_cast<double>(mf);
            v[2 * kMaxObs + 1] = CPL ? static_cast<double>(mc) : 0.0;
#pragma unroll
            for (int k = 0; k < kMaxObs; ++k) {
                double sf = 0.0, sc = 0.0;
                if (k < a.n_obs) {
#pragma unroll
                    for (int b = 0; b < NB; ++b) {
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            sf += static_cast<double>(q[b][i] - a.qbf[fidx[b][i]]) *
                                  t.phif64[(size_t)k * N * N + fidx[b][i]];
                        if constexpr (CPL)
                            sc += static_cast<double>(qc[b] - a.qbc[gc[b]]) * t.phic64[(size_t)k * NC * NC + gc[b]];
                    }
                }
                v[k] = sf;
                v[kMaxObs + k] = sc;
            }
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1)
#pragma unroll
            for (int i = 0; i < kRed; ++i) v[i] += __shfl_xor_sync(kFullMask, v[i], off);
        if ((tid & 31) == 0)
#pragma unroll
            for (int i = 0; i < kRed; ++i) red[(tid >> 5) * kRed + i] = v[i];
        __syncthreads();
        if (tid < kRed) {
            double x = 0.0;
            for (int w = 0; w < THREADS / 32; ++w) x += red[w * kRed + tid];
            tot[tid] = x;
        }
        ph.full();
        if (rank == 0 && tid == 0 && active) {
            for (int i = 0; i < kRed; ++i) {
                double x = 0.0;
                for (int r = 0; r < CL; ++r) x += band_at(tot, r, 0)[i];
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

template <int N, bool CPL>
cudaError_t prepare(int slot_stride, VariantInfo* out) {
    using S = TShape<N>;
    const size_t smem = S::smem(slot_stride);
    cudaError_t e = cudaFuncSetAttribute(theta_kernel<N, CPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, theta_kernel<N, CPL>, S::THREADS, smem)) !=
        cudaSuccess)
        return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    *out = VariantInfo{};
    out->supported = per_sm > 0;
    out->threads = S::THREADS;
    out->cluster = 1;
    out->slots_per_cta = S::SPB;
    out->smem = smem;
    out->max_ctas = per_sm * sms;
    return cudaSuccess;
}

template <int N, bool CPL>
cudaError_t launch_n(const KArgs& a, const TArgs& t, int n_ctas, cudaStream_t st, int priority) {
    using S = TShape<N>;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(n_ctas);
    cfg.blockDim = dim3(S::THREADS);
    cfg.dynamicSmemBytes = S::smem(a.slot_stride);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    int na = 0;
    if (priority != 0) {
        attr[na].id = cudaLaunchAttributePriority;
        attr[na].val.priority = priority;
        ++na;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, theta_kernel<N, CPL>, a, t);
}

// Grids beyond one CTA: clusters of CL CTAs.
constexpr int kThetaClusterN = 128, kThetaClusterCL = 4, kThetaClusterNB = 2;

template <int N, int CL, int NB, bool CPL>
cudaError_t prepare_cluster(int slot_stride, VariantInfo* out) {
    using S = CShape<N, CL, NB>;
    const size_t smem = S::smem(slot_stride);
    cudaError_t e = cudaFuncSetAttribute(theta_cluster_kernel<N, CL, NB, CPL>,
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
    if ((e = cudaOccupancyMaxActiveClusters(&clusters, theta_cluster_kernel<N, CL, NB, CPL>, &cfg)) != cudaSuccess)
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

template <int N, int CL, int NB, bool CPL>
cudaError_t launch_cluster(const KArgs& a, const TArgs& t, int n_ctas, cudaStream_t st, int priority) {
    using S = CShape<N, CL, NB>;
    if (n_ctas % CL != 0) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(n_ctas);
    cfg.blockDim = dim3(S::THREADS);
    cfg.dynamicSmemBytes = S::smem(a.slot_stride);
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
    return cudaLaunchKernelEx(&cfg, theta_cluster_kernel<N, CL, NB, CPL>, a, t);
}

}  // namespace

bool theta_supported(int n) { return n == 4 || n == 8 || n == 16 || n == 32 || n == 64 || n == kThetaClusterN; }

cudaError_t theta_variant_info(int n, bool coupled, int slot_stride, VariantInfo* out) {
    *out = VariantInfo{};
    switch (n) {
        case 4: return coupled ? prepare<4, true>(slot_stride, out) : prepare<4, false>(slot_stride, out);
        case 8: return coupled ? prepare<8, true>(slot_stride, out) : prepare<8, false>(slot_stride, out);
        case 16: return coupled ? prepare<16, true>(slot_stride, out) : prepare<16, false>(slot_stride, out);
        case 32: return coupled ? prepare<32, true>(slot_stride, out) : prepare<32, false>(slot_stride, out);
        case 64: return coupled ? prepare<64, true>(slot_stride, out) : prepare<64, false>(slot_stride, out);
        case kThetaClusterN:
            return coupled ? prepare_cluster<kThetaClusterN, kThetaClusterCL, kThetaClusterNB, true>(slot_stride, out)
                           : prepare_cluster<kThetaClusterN, kThetaClusterCL, kThetaClusterNB, false>(slot_stride, out);
        default: return cudaSuccess;   // supported = 0
    }
}

cudaError_t launch_theta(int n, bool coupled, const KArgs& a, const TArgs& t, int n_ctas, cudaStream_t st,
                         int priority) {
    if (t.K < 0 || t.K > kMaxCheb) return cudaErrorInvalidValue;
    switch (n) {
        case 4: return coupled ? launch_n<4, true>(a, t, n_ctas, st, priority) : launch_n<4, false>(a, t, n_ctas, st, priority);
        case 8: return coupled ? launch_n<8, true>(a, t, n_ctas, st, priority) : launch_n<8, false>(a, t, n_ctas, st, priority);
        case 16: return coupled ? launch_n<16, true>(a, t, n_ctas, st, priority) : launch_n<16, false>(a, t, n_ctas, st, priority);
        case 32: return coupled ? launch_n<32, true>(a, t, n_ctas, st, priority) : launch_n<32, false>(a, t, n_ctas, st, priority);
        case 64: return coupled ? launch_n<64, true>(a, t, n_ctas, st, priority) : launch_n<64, false>(a, t, n_ctas, st, priority);
        case kThetaClusterN:
            return coupled ? launch_cluster<kThetaClusterN, kThetaClusterCL, kThetaClusterNB, true>(a, t, n_ctas, st, priority)
                           : launch_cluster<kThetaClusterN, kThetaClusterCL, kThetaClusterNB, false>(a, t, n_ctas, st, priority);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace dk
