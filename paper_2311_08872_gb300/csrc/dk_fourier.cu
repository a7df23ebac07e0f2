// Fourier-coupled sample kernel for sm_103a (Section 3.1): the fine path of
// Eq. (FullyDiscreteDK) (b0 = 0, b1 = 1) on an n x n grid and, for a coupled
// level, the coarse path on the (n/3) x (n/3) grid with step 9 tau, whose
// noise carries every Fourier mode of the fine noise that the coarse grid
// resolves.
//
// Noise.  The fine Brownian increments are the cell normals of the explicit
// kernels (same Philox counters); their unitary discrete Fourier coefficients
// are exactly the independent complex-conjugate Fourier Brownian increments
// of Section 3.1.  The coarse increment of one coarse step is the restriction
// P1 S P1^T of the sum S of the 9 fine normal fields inside it, P1 (n/3 x n,
// host-built) keeping the modes -n/6..n/6 per axis, the two fine aliases of
// the coarse Nyquist mode weighted 2^-1/2 each; P1 has orthonormal rows, so
// the coarse normal field (P1 S P1^T / 3) is white with unit variance and the
// coarse path has the law of a stand-alone coarse path (Remark
// distribution_W_ell).  The restriction is linear, so the 9 fine fields are
// summed first (FP32, per fine cell) and restricted once per coarse step: two
// small dense products per component (n x n by n x n/3, then n/3 x n by
// n x n/3), under 10% of the stencil work at n = 54.
//
// Arithmetic as in the explicit kernels: int32 fixed-point state, integer
// noise transfers G = rint(c 2^S sqrt(rho^+) Z) and diffusion fluxes, every
// edge flux computed identically by both of its cells, so the mass is exact.
// With the fluctuation state (FL) the state is q = (rho - rho-bar^m) 2^S
// about the noise-free path and the amplitudes read rho-bar^m from the
// per-step tables (fine: step m; coarse: coarse step m / 9).
//
// Work decomposition.  One CTA per sample.  A thread holds a segment of 6
// consecutive fine cells of one row (3 Philox cell pairs) in registers, with
// its row's periodic neighbours fixed once, so a fine step needs no index
// arithmetic; the state and transfers are published in shared memory for the
// rows above and below and the segment ends.  The coarse grid and the
// restriction loop over cells with the CTA's stride.  Two barriers per fine
// step, two more at a coarse step.
#include "dk_device.cuh"
#include "dk_kernels.h"

namespace dk {
namespace {

constexpr unsigned kFullMaskF = 0xffffffffu;
constexpr int kRedF = 2 * kMaxObs + 2;

template <int N_>
struct FShape {
    static constexpr int N = N_, NC = N / 3;
    static constexpr int SEG = 6;                       // fine cells per thread: one row segment (3 Philox pairs)
    static constexpr int SEGS = N / SEG;                // segments per row
    static constexpr int FT = N * SEGS;                 // threads that hold fine cells
    static constexpr int THREADS = FT > 256 ? 512 : (FT > 32 ? 64 : 32);
    static_assert(N % SEG == 0 && FT <= THREADS, "fine row segments must cover the grid");
    static constexpr int MINB = THREADS >= 512 ? 2 : 1;   // two samples per SM at 54^2 (64 registers)
    static constexpr int WARPS = THREADS / 32;
    // words: q (2 buffers), G1, G2, summed normals (2), coarse q (2 buffers),
    // coarse G1, G2, the row-restricted sums T (N x NC x 2), P1 (NC x N)
    static constexpr int WORDS = 2 * N * N + 2 * N * N + 2 * N * N + 2 * NC * NC + 2 * NC * NC + 2 * N * NC + NC * N;
    static size_t smem(int slot_stride) {
        return sizeof(int32_t) * (size_t)((WORDS + 1) / 2 * 2) + sizeof(double) * WARPS * kRedF +
               sizeof(double) * slot_stride;
    }
};

// Explicit step of an NN x NN grid in flux form for the cells of this thread:
// qn(x) = q(x) + diffusion fluxes of its four edges + G1(down) - G1(up) +
// G2(right) - G2(left), every edge flux computed from the same two states by
// both cells of the edge.
template <int NN, int THREADS>
__device__ __forceinline__ void explicit_update(const int32_t* q, const int32_t* G1, const int32_t* G2, int32_t* qn,
                                                int32_t A, unsigned& bad) {
    for (int x = threadIdx.x; x < NN * NN; x += THREADS) {
        const int i1 = x / NN, i2 = x % NN;
        const int up = ((i1 + NN - 1) % NN) * NN + i2, dn = ((i1 + 1) % NN) * NN + i2;
        const int lf = i1 * NN + (i2 + NN - 1) % NN, rt = i1 * NN + (i2 + 1) % NN;
        const int32_t c = q[x];
        const int32_t v = c + (edge_flux(A, q[dn] - c) - edge_flux(A, c - q[up])) +
                          (edge_flux(A, q[rt] - c) - edge_flux(A, c - q[lf])) + (G1[dn] - G1[up]) + (G2[rt] - G2[lf]);
        bad |= (static_cast<uint32_t>(v) + 0x40000000u) >> 31;
        qn[x] = v;
    }
}

template <int N, bool CPL, bool FL>
__global__ void __launch_bounds__(FShape<N>::THREADS, FShape<N>::MINB) fourier_kernel(const KArgs a, const FArgs f) {
    using S = FShape<N>;
    constexpr int NC = S::NC, THREADS = S::THREADS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    int32_t* const qA = reinterpret_cast<int32_t*>(smem_raw);   // fine state, double buffered
    int32_t* const qB = qA + N * N;
    int32_t* G1 = qB + N * N;
    int32_t* G2 = G1 + N * N;
    float* Zs = reinterpret_cast<float*>(G2 + N * N);      // [N*N][2] summed fine normals
    int32_t* const qcA = reinterpret_cast<int32_t*>(Zs + 2 * N * N);   // coarse state, double buffered
    int32_t* const qcB = qcA + NC * NC;
    int32_t* Gc1 = qcB + NC * NC;
    int32_t* Gc2 = Gc1 + NC * NC;
    float* Tm = reinterpret_cast<float*>(Gc2 + NC * NC);    // [2][N][NC]
    float* P1 = Tm + 2 * N * NC;                            // [NC][N]
    double* red = reinterpret_cast<double*>(smem_raw + sizeof(int32_t) * (size_t)((S::WORDS + 1) / 2 * 2));
    double* acc = red + S::WARPS * kRedF;
    for (int i = tid; i < a.slot_stride; i += THREADS) acc[i] = 0.0;
    if constexpr (CPL)
        for (int i = tid; i < NC * N; i += THREADS) P1[i] = f.P1[i];

    constexpr int SEG = S::SEG, SEGS = S::SEGS;
    const bool fine_thread = tid < S::FT;
    const int frow = fine_thread ? tid / SEGS : 0;
    const int fc0 = fine_thread ? (tid % SEGS) * SEG : 0;
    const int fx0 = frow * N + fc0;                                  // first cell of the segment
    const int upo = frow == 0 ? N * (N - 1) : -N;                    // offsets to the rows above / below
    const int dno = frow == N - 1 ? -N * (N - 1) : N;
    const int lfx = fc0 == 0 ? fx0 + N - 1 : fx0 - 1;                // left of the first cell
    const int rtx = fc0 + SEG == N ? fx0 + SEG - N : fx0 + SEG;      // right of the last cell

    unsigned bad = 0;
    const long long slot = blockIdx.x, n_slots = gridDim.x;
    const long long iters = a.count > slot ? (a.count - slot + n_slots - 1) / n_slots : 0;
    __syncthreads();

    for (long long it = 0; it < iters; ++it) {
        const long long idx = slot + it * n_slots;
        const long long sid = a.first + idx;
        const uint32_t c2 = static_cast<uint32_t>(sid);
        const uint32_t c3 = a.tag | ((static_cast<uint32_t>(static_cast<unsigned long long>(sid) >> 32) & 0xffffu) << 16);
        int cur = 0, ccur = 0;
        int32_t qr[SEG];
        if (fine_thread) {
#pragma unroll
            for (int j = 0; j < SEG; ++j) {
                qr[j] = a.q0f[fx0 + j];
                qA[fx0 + j] = qr[j];
            }
        }
        if constexpr (CPL)
            for (int y = tid; y < NC * NC; y += THREADS) qcA[y] = a.q0c[y];
        __syncthreads();

        for (int m = 0; m < a.M; ++m) {
            const int32_t* q = cur ? qB : qA;
            const bool first_of_coarse = CPL && (m % 9) == 0;
            // ---- noise of the segment: Philox4x32-10 per horizontal cell pair, Box--Muller, transfers
            int32_t g1[SEG], g2[SEG];
            if (fine_thread) {
#pragma unroll
                for (int j = 0; j < SEG / 2; ++j) {
                    const int p = (fx0 >> 1) + j;
                    const uint4 x = philox10(make_uint4(static_cast<uint32_t>(p), static_cast<uint32_t>(m), c2, c3),
                                             a.key0, a.key1);
                    float ra, ca, sa, rb, cb, sb;
                    box_muller_polar(x.x, x.y, ra, ca, sa);
                    box_muller_polar(x.z, x.w, rb, cb, sb);
                    float ta, tb;
                    if constexpr (FL) {
                        const float2 rbar = reinterpret_cast<const float2*>(a.rbf + (size_t)m * N * N)[p];
                        ta = noise_amp_fluct(qr[2 * j], rbar.x, a.isf, a.gf) * ra;
                        tb = noise_amp_fluct(qr[2 * j + 1], rbar.y, a.isf, a.gf) * rb;
                    } else {
                        ta = noise_amp(qr[2 * j], a.gf) * ra;
                        tb = noise_amp(qr[2 * j + 1], a.gf) * rb;
                    }
                    g1[2 * j] = __float2int_rn(ta * ca);
                    g2[2 * j] = __float2int_rn(ta * sa);
                    g1[2 * j + 1] = __float2int_rn(tb * cb);
                    g2[2 * j + 1] = __float2int_rn(tb * sb);
                    reinterpret_cast<int2*>(G1)[p] = make_int2(g1[2 * j], g1[2 * j + 1]);
                    reinterpret_cast<int2*>(G2)[p] = make_int2(g2[2 * j], g2[2 * j + 1]);
                    if constexpr (CPL) {
                        float4 z = first_of_coarse ? make_float4(0.f, 0.f, 0.f, 0.f)
                                                   : reinterpret_cast<float4*>(Zs)[p];
                        z.x += ra * ca;
                        z.y += ra * sa;
                        z.z += rb * cb;
                        z.w += rb * sb;
                        reinterpret_cast<float4*>(Zs)[p] = z;
                    }
                }
            }
            __syncthreads();
            // ---- explicit step of the segment in flux form (every edge flux computed
            // from the same two states by both of its cells)
            if (fine_thread) {
                int32_t* qn = cur ? qA : qB;
                // the rows above and below, 8-byte loads (segments start at even cells)
                int32_t qu[SEG], qd[SEG], gu[SEG], gd[SEG];
#pragma unroll
                for (int j = 0; j < SEG; j += 2) {
                    const int2 a0 = *reinterpret_cast<const int2*>(q + fx0 + upo + j);
                    const int2 a1 = *reinterpret_cast<const int2*>(q + fx0 + dno + j);
                    const int2 b0 = *reinterpret_cast<const int2*>(G1 + fx0 + upo + j);
                    const int2 b1 = *reinterpret_cast<const int2*>(G1 + fx0 + dno + j);
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
#pragma unroll
                for (int j = 0; j < SEG; j += 2) {
                    qr[j] = nq[j];
                    qr[j + 1] = nq[j + 1];
                    *reinterpret_cast<int2*>(qn + fx0 + j) = make_int2(nq[j], nq[j + 1]);
                }
            }
            cur ^= 1;
            if constexpr (CPL) {
                if ((m % 9) == 8) {
                    // ---- coarse noise: P1 S P1^T per component (S = summed fine normals)
                    for (int o = tid; o < 2 * N * NC; o += THREADS) {
                        const int r = o / (N * NC), x1 = (o / NC) % N, y2 = o % NC;
                        float s = 0.f;
                        for (int x2 = 0; x2 < N; ++x2) s = fmaf(Zs[2 * (x1 * N + x2) + r], P1[y2 * N + x2], s);
                        Tm[o] = s;
                    }
                    __syncthreads();
                    const int32_t* qc = ccur ? qcB : qcA;
                    for (int o = tid; o < NC * NC; o += THREADS) {
                        const int y1 = o / NC, y2 = o % NC;
                        float s1 = 0.f, s2 = 0.f;
                        for (int x1 = 0; x1 < N; ++x1) {
                            const float w = P1[y1 * N + x1];
                            s1 = fmaf(w, Tm[x1 * NC + y2], s1);
                            s2 = fmaf(w, Tm[N * NC + x1 * NC + y2], s2);
                        }
                        // gc includes the 1/3 of the 9-step sum
                        const float amp = FL ? noise_amp_fluct(qc[o], a.rbc[(size_t)(m / 9) * NC * NC + o], a.isc, a.gc)
                                             : noise_amp(qc[o], a.gc);
                        Gc1[o] = __float2int_rn(amp * s1);
                        Gc2[o] = __float2int_rn(amp * s2);
                    }
                    __syncthreads();
                    explicit_update<NC, THREADS>(qc, Gc1, Gc2, ccur ? qcA : qcB, a.Ac, bad);
                    ccur ^= 1;
                }
            }
            __syncthreads();
        }

        // ---- observables against FP64 test functions, mass; CTA reduction
        double v[kRedF];
#pragma unroll
        for (int i = 0; i < kRedF; ++i) v[i] = 0.0;
        const int32_t* q = cur ? qB : qA;
        for (int x = tid; x < N * N; x += THREADS) {
            v[2 * kMaxObs] += static_cast<double>(q[x]);
            const double d = static_cast<double>(q[x] - a.qbf[x]);
            for (int k = 0; k < a.n_obs; ++k) v[k] += d * f.phif64[(size_t)k * N * N + x];
        }
        if constexpr (CPL) {
            const int32_t* qc = ccur ? qcB : qcA;
            for (int y = tid; y < NC * NC; y += THREADS) {
                v[2 * kMaxObs + 1] += static_cast<double>(qc[y]);
                const double d = static_cast<double>(qc[y] - a.qbc[y]);
                for (int k = 0; k < a.n_obs; ++k) v[kMaxObs + k] += d * f.phic64[(size_t)k * NC * NC + y];
            }
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1)
#pragma unroll
            for (int i = 0; i < kRedF; ++i) v[i] += __shfl_xor_sync(kFullMaskF, v[i], off);
        if ((tid & 31) == 0)
#pragma unroll
            for (int i = 0; i < kRedF; ++i) red[(tid >> 5) * kRedF + i] = v[i];
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < S::WARPS; ++w)
#pragma unroll
                for (int i = 0; i < kRedF; ++i) v[i] += red[w * kRedF + i];
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
                o[2 * a.n_obs] = v[2 * kMaxObs] * a.dscale_f + a.mass_off_f;
                o[2 * a.n_obs + 1] = CPL ? v[2 * kMaxObs + 1] * a.dscale_c + a.mass_off_c : 0.0;
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(a.err, kErrRange);
    __syncthreads();
    for (int i = tid; i < a.slot_stride; i += THREADS) a.partials[(size_t)i * n_slots + slot] = acc[i];
}

template <int N, bool CPL, bool FL>
cudaError_t fprepare(int slot_stride, VariantInfo* out) {
    using S = FShape<N>;
    const size_t smem = S::smem(slot_stride);
    cudaError_t e = cudaFuncSetAttribute(fourier_kernel<N, CPL, FL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fourier_kernel<N, CPL, FL>, S::THREADS, smem)) !=
        cudaSuccess)
        return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    *out = VariantInfo{};
    out->supported = per_sm > 0;
    out->threads = S::THREADS;
    out->cluster = 1;
    out->slots_per_cta = 1;
    out->smem = smem;
    out->max_ctas = per_sm * sms;
    return cudaSuccess;
}

template <int N, bool CPL, bool FL>
cudaError_t flaunch(const KArgs& a, const FArgs& f, int n_ctas, cudaStream_t st, int priority) {
    using S = FShape<N>;
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
    return cudaLaunchKernelEx(&cfg, fourier_kernel<N, CPL, FL>, a, f);
}

template <bool FL>
cudaError_t fourier_info_fl(int n, bool coupled, int slot_stride, VariantInfo* out) {
    switch (n) {
        case 6: return coupled ? cudaSuccess : fprepare<6, false, FL>(slot_stride, out);   // level 0 only
        case 18: return coupled ? fprepare<18, true, FL>(slot_stride, out) : fprepare<18, false, FL>(slot_stride, out);
        case 54: return coupled ? fprepare<54, true, FL>(slot_stride, out) : fprepare<54, false, FL>(slot_stride, out);
        default: return cudaSuccess;
    }
}

template <bool FL>
cudaError_t launch_fourier_fl(int n, bool coupled, const KArgs& a, const FArgs& f, int n_ctas, cudaStream_t st,
                              int priority) {
    switch (n) {
        case 6: return coupled ? cudaErrorInvalidValue : flaunch<6, false, FL>(a, f, n_ctas, st, priority);
        case 18: return coupled ? flaunch<18, true, FL>(a, f, n_ctas, st, priority)
                                : flaunch<18, false, FL>(a, f, n_ctas, st, priority);
        case 54: return coupled ? flaunch<54, true, FL>(a, f, n_ctas, st, priority)
                                : flaunch<54, false, FL>(a, f, n_ctas, st, priority);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool fourier_supported(int n) { return n == 6 || n == 18 || n == 54; }

cudaError_t fourier_variant_info(int n, bool coupled, int slot_stride, VariantInfo* out, bool fluct) {
    *out = VariantInfo{};
    return fluct ? fourier_info_fl<true>(n, coupled, slot_stride, out) : fourier_info_fl<false>(n, coupled, slot_stride, out);
}

cudaError_t launch_fourier(int n, bool coupled, const KArgs& a, const FArgs& f, int n_ctas, cudaStream_t st,
                           int priority, bool fluct) {
    if (fluct && (!a.rbf || (coupled && !a.rbc))) return cudaErrorInvalidValue;
    return fluct ? launch_fourier_fl<true>(n, coupled, a, f, n_ctas, st, priority)
                 : launch_fourier_fl<false>(n, coupled, a, f, n_ctas, st, priority);
}

}  // namespace dk
