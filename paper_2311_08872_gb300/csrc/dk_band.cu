// Band kernels: the coupled sample of a large grid (n = 128 .. 1024) spread
// over several CTAs, each holding a full-width band of coarse rows in
// registers for the whole run.
//
// The scheme, the noise counters and the integer arithmetic are those of the
// register kernels (Eq. FullyDiscreteDK with b0 = 0, b1 = 1; Right-Most NN
// coupling of Section 3.2): a thread owns a 2 x 4 block of fine cells (one
// coarse row, two coarse cells), draws the Philox normals of its four cell
// pairs, sums the coupled coarse normals of its two coarse cells in the same
// order, and applies the same edge fluxes and transfers, so the fine and
// coarse states agree with theirs bit for bit.
//
// Layout.  A warp covers 128 fine columns of one coarse row (two fine rows);
// WPR = n / 128 warps cover a row, and a CTA holds a band of up to 32 / WPR
// coarse rows.  Within a CTA the rows exchange their edge rows through shared
// memory (double-buffered by step parity, one barrier per fine step) and the
// columns by warp shuffles (and shared memory between the warps of a row).
// Between bands the top and bottom fine rows (state and vertical transfer)
// and, on coarse steps, the coarse rows go through global memory: the edge
// warps write them, then add to a per-band counter with release semantics;
// the neighbouring band's edge warp waits (acquire, bounded) until the counter
// shows the step, then reads them.  No CTA waits for anything but its two
// neighbouring bands' counters, so the bands of a sample must be resident
// together: the grid is launched cooperatively.  Every wait gives up after a
// fixed number of polls (or as soon as another CTA has given up), records
// kErrTimeout in the error word and makes its CTA stop stepping, so a kernel
// never spins without end.
#include <algorithm>
#include <cstdint>

#include "dk_device.cuh"
#include "dk_kernels.h"

namespace dk {

namespace {

constexpr int kBandMaxThreads = 1024;
constexpr int kW = 2 * kMaxObs + 2;              // per-band observable partials
constexpr unsigned kWaitPolls = 1u << 22;         // polls of one wait before it gives up

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
    return *reinterpret_cast<const volatile unsigned*>(p);
}

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

__device__ __forceinline__ void st_int2x4(int2* dst, const int32_t (&q)[4], const int32_t (&g)[4]) {
    int4* d = reinterpret_cast<int4*>(dst);
    d[0] = make_int4(q[0], g[0], q[1], g[1]);
    d[1] = make_int4(q[2], g[2], q[3], g[3]);
}

__device__ __forceinline__ void ld_int2x4(const int2* src, int32_t (&q)[4], int32_t (&g)[4]) {
    const int4* s = reinterpret_cast<const int4*>(src);
    const int4 a = s[0], b = s[1];
    q[0] = a.x; g[0] = a.y; q[1] = a.z; g[1] = a.w;
    q[2] = b.x; g[2] = b.y; q[3] = b.z; g[3] = b.w;
}

// The same from global memory through L2 (another SM wrote it).
__device__ __forceinline__ void ldcg_int2x4(const int2* src, int32_t (&q)[4], int32_t (&g)[4]) {
    const int4* s = reinterpret_cast<const int4*>(src);
    const int4 a = __ldcg(s), b = __ldcg(s + 1);
    q[0] = a.x; g[0] = a.y; q[1] = a.z; g[1] = a.w;
    q[2] = b.x; g[2] = b.y; q[3] = b.z; g[3] = b.w;
}

__device__ __forceinline__ void ldcg_int2x2(const int2* src, int32_t (&q)[2], int32_t (&g)[2]) {
    const int4 a = __ldcg(reinterpret_cast<const int4*>(src));
    q[0] = a.x; g[0] = a.y; q[1] = a.z; g[1] = a.w;
}

struct BandSmem {
    int2* sv;      // [2 parity][bmax][2 side][NF]: (q, G1) of each coarse row's top / bottom fine row
    int2* sh;      // [2 parity][bmax][WPR][2 side][2 row]: (q, G2) of each warp's first / last column
    int2* scv;     // [bmax][NC]: (qc, Gc1) of each coarse row (coarse steps)
    int2* sch;     // [bmax][WPR][2 side]: (qc, Gc2) of each warp's first / last coarse column
    double* red;   // [warps][kW]
    int* abort;    // [2]: set at step m in slot (m + 1) & 1, read after the barrier of step m + 1
};

template <int WPR>
__host__ __device__ constexpr size_t band_smem_bytes(int bmax) {
    return sizeof(int2) * (size_t)(2 * bmax * 2 * 128 * WPR + 2 * bmax * WPR * 2 * 2 + bmax * 64 * WPR +
                                   bmax * WPR * 2) +
           sizeof(double) * (size_t)(bmax * WPR * kW) + 2 * sizeof(int);
}

template <int WPR>
__device__ BandSmem carve(unsigned char* p, int bmax) {
    constexpr int NF = 128 * WPR, NC = NF / 2;
    BandSmem s;
    s.sv = reinterpret_cast<int2*>(p);
    s.sh = s.sv + (size_t)2 * bmax * 2 * NF;
    s.scv = s.sh + (size_t)2 * bmax * WPR * 2 * 2;
    s.sch = s.scv + (size_t)bmax * NC;
    s.red = reinterpret_cast<double*>(s.sch + (size_t)bmax * WPR * 2);
    s.abort = reinterpret_cast<int*>(s.red + (size_t)bmax * WPR * kW);
    return s;
}

template <int WPR, bool CPL>
__global__ void __launch_bounds__(kBandMaxThreads, 1) band_kernel(const KArgs a, const BArgs b) {
    constexpr int NF = 128 * WPR, NC = NF / 2;
    extern __shared__ __align__(16) unsigned char band_shared[];
    const BandSmem sm = carve<WPR>(band_shared, b.bmax);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s = blockIdx.x / b.nb, band = blockIdx.x % b.nb;
    if (s >= b.count) return;   // the whole CTA (and every band of this sample) leaves together
    const int cr = warp / WPR, wc = warp % WPR;
    const int r0 = (int)((long long)band * NC / b.nb);
    const int B = (int)((long long)(band + 1) * NC / b.nb) - r0;
    const bool live = cr < B;
    const bool top = cr == 0, bot = cr == B - 1;
    const int crow = r0 + (live ? cr : 0);
    const int frow = 2 * crow;
    const int col0 = (wc * 32 + lane) * 4, ccol0 = col0 / 2;
    const int up = (band + b.nb - 1) % b.nb, dn = (band + 1) % b.nb;
    const long long sid = b.sid0 + s;
    const uint32_t c2 = static_cast<uint32_t>(sid);
    const uint32_t c3 = a.tag | ((static_cast<uint32_t>(static_cast<unsigned long long>(sid) >> 32) & 0xffffu) << 16);
    // this sample's exchange buffers
    unsigned* const flags = b.flags + (size_t)s * b.nb * 2;            // [band][side]
    int2* const edge = b.edge + (size_t)s * b.nb * 2 * 2 * NF;         // [band][side][parity][NF]
    int2* const cedge = b.cedge + (size_t)s * b.nb * 2 * NC;           // [band][side][NC]
    if (tid < 2) sm.abort[tid] = 0;

    int32_t q[2][4], qc[1][2];
    float zt[2][2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int4 v = __ldg(reinterpret_cast<const int4*>(a.q0f + (size_t)(frow + r) * NF + col0));
        q[r][0] = v.x; q[r][1] = v.y; q[r][2] = v.z; q[r][3] = v.w;
    }
    if constexpr (CPL) {
        const int2 v = __ldg(reinterpret_cast<const int2*>(a.q0c + (size_t)crow * NC + ccol0));
        qc[0][0] = v.x; qc[0][1] = v.y;
        zt[0][0] = zt[0][1] = zt[1][0] = zt[1][1] = 0.f;
    }
    __syncthreads();
    unsigned bad = 0;
    const int M = b.steps;
    for (int m = 0; m < M; ++m) {
        const int par = m & 1;
        const bool cstep = CPL && ((m & 3) == 3);
        // ---- noise of step m: Philox4x32-10 per horizontal cell pair, Box--Muller, transfers
        // (warps below a short band's last row hold no cells and only keep the barriers)
        int32_t G1[2][4], G2[2][4];
#pragma unroll
        for (int r = 0; r < 2 && live; ++r) {
#pragma unroll
            for (int pc = 0; pc < 2; ++pc) {
                const uint32_t p = static_cast<uint32_t>(((frow + r) * NF + col0 + 2 * pc) >> 1);
                const uint4 x = philox10(make_uint4(p, static_cast<uint32_t>(m), c2, c3), a.key0, a.key1);
                float ra, ca, sa, rb, cb, sb;
                box_muller_polar(x.x, x.y, ra, ca, sa);
                box_muller_polar(x.z, x.w, rb, cb, sb);
                const float ta = noise_amp(q[r][2 * pc], a.gf) * ra;
                const float tb = noise_amp(q[r][2 * pc + 1], a.gf) * rb;
                G1[r][2 * pc] = __float2int_rn(ta * ca);
                G2[r][2 * pc] = __float2int_rn(ta * sa);
                G1[r][2 * pc + 1] = __float2int_rn(tb * cb);
                G2[r][2 * pc + 1] = __float2int_rn(tb * sb);
                if constexpr (CPL) {
                    zt[pc][0] = fmaf(rb, cb, fmaf(ra, ca, zt[pc][0]));
                    zt[pc][1] = fmaf(rb, sb, fmaf(ra, sa, zt[pc][1]));
                }
            }
        }
        int32_t Gc1[1][2], Gc2[1][2];
        if (cstep && live) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const float amp = noise_amp(qc[0][j], a.gc);
                Gc1[0][j] = __float2int_rn(amp * zt[j][0]);
                Gc2[0][j] = __float2int_rn(amp * zt[j][1]);
                zt[j][0] = zt[j][1] = 0.f;
            }
        }
        // ---- publish: edge rows to shared memory, band edges to global memory
        if (live) {
            st_int2x4(sm.sv + (((size_t)par * b.bmax + cr) * 2 + 0) * NF + col0, q[0], G1[0]);
            st_int2x4(sm.sv + (((size_t)par * b.bmax + cr) * 2 + 1) * NF + col0, q[1], G1[1]);
            if constexpr (WPR > 1) {
                int2* h = sm.sh + (((size_t)par * b.bmax + cr) * WPR + wc) * 4;
                if (lane == 0) { h[0] = make_int2(q[0][0], G2[0][0]); h[1] = make_int2(q[1][0], G2[1][0]); }
                if (lane == 31) { h[2] = make_int2(q[0][3], G2[0][3]); h[3] = make_int2(q[1][3], G2[1][3]); }
            }
            if (cstep) {
                reinterpret_cast<int4*>(sm.scv + (size_t)cr * NC + ccol0)[0] =
                    make_int4(qc[0][0], Gc1[0][0], qc[0][1], Gc1[0][1]);
                if constexpr (WPR > 1) {
                    int2* h = sm.sch + ((size_t)cr * WPR + wc) * 2;
                    if (lane == 0) h[0] = make_int2(qc[0][0], Gc2[0][0]);
                    if (lane == 31) h[1] = make_int2(qc[0][1], Gc2[0][1]);
                }
            }
            if (top || bot) {
                if (top) {
                    st_int2x4(edge + (((size_t)band * 2 + 0) * 2 + par) * NF + col0, q[0], G1[0]);
                    if (cstep)
                        reinterpret_cast<int4*>(cedge + ((size_t)band * 2 + 0) * NC + ccol0)[0] =
                            make_int4(qc[0][0], Gc1[0][0], qc[0][1], Gc1[0][1]);
                }
                if (bot) {
                    st_int2x4(edge + (((size_t)band * 2 + 1) * 2 + par) * NF + col0, q[1], G1[1]);
                    if (cstep)
                        reinterpret_cast<int4*>(cedge + ((size_t)band * 2 + 1) * NC + ccol0)[0] =
                            make_int4(qc[0][0], Gc1[0][0], qc[0][1], Gc1[0][1]);
                }
                __syncwarp();
                if (lane == 0 && band != b.stall_band) {   // stall_band: failure-detection test only
                    __threadfence();
                    if (top) red_release_add(flags + (size_t)band * 2 + 0, 1u);
                    if (bot) red_release_add(flags + (size_t)band * 2 + 1, 1u);
                }
            }
        }
        __syncthreads();
        if (sm.abort[par]) break;   // uniform: a wait of the previous step gave up

        if (!live) continue;
        // ---- the band's edge warps wait for the neighbouring bands' step-m edges
        // (lane 0 polls, the warp barrier passes the acquire on to the other lanes)
        if (top || bot) {
            if (lane == 0) {
                bool ok = true;
                if (top) ok = wait_counter(flags + (size_t)up * 2 + 1, (unsigned)(WPR * (m + 1)), a.err, b.wait_polls);
                if (bot && ok) ok = wait_counter(flags + (size_t)dn * 2 + 0, (unsigned)(WPR * (m + 1)), a.err, b.wait_polls);
                if (!ok) sm.abort[par ^ 1] = 1;
            }
            __syncwarp();
        }
        // ---- fine update, one row at a time: each edge flux once per block, as
        // in the register kernels (the integer sums are exact, so grouping them
        // by row leaves the result unchanged)
        int32_t v1[4];   // vertical fluxes between the block's two rows (old state)
#pragma unroll
        for (int c = 0; c < 4; ++c) v1[c] = edge_flux(a.Af, q[1][c] - q[0][c]);
        const int2* const svp = sm.sv + (size_t)par * b.bmax * 2 * NF + col0;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            // vertical neighbour row: the coarse row above (r = 0) / below (r = 1)
            int32_t qV[4], gV[4];
            if (r == 0) {
                if (!top) ld_int2x4(svp + ((size_t)(cr - 1) * 2 + 1) * NF, qV, gV);
                else ldcg_int2x4(edge + (((size_t)up * 2 + 1) * 2 + par) * NF + col0, qV, gV);
            } else {
                if (!bot) ld_int2x4(svp + ((size_t)(cr + 1) * 2 + 0) * NF, qV, gV);
                else ldcg_int2x4(edge + (((size_t)dn * 2 + 0) * 2 + par) * NF + col0, qV, gV);
            }
            // horizontal neighbours: shuffles, the row's other warps through shared memory
            int32_t qL = __shfl_sync(0xffffffffu, q[r][3], (lane + 31) & 31);
            int32_t gL = __shfl_sync(0xffffffffu, G2[r][3], (lane + 31) & 31);
            int32_t qR = __shfl_sync(0xffffffffu, q[r][0], (lane + 1) & 31);
            int32_t gR = __shfl_sync(0xffffffffu, G2[r][0], (lane + 1) & 31);
            if constexpr (WPR > 1) {
                if (lane == 0) {
                    const int2 u = sm.sh[(((size_t)par * b.bmax + cr) * WPR + (wc + WPR - 1) % WPR) * 4 + 2 + r];
                    qL = u.x; gL = u.y;
                }
                if (lane == 31) {
                    const int2 u = sm.sh[(((size_t)par * b.bmax + cr) * WPR + (wc + 1) % WPR) * 4 + r];
                    qR = u.x; gR = u.y;
                }
            }
            int32_t nq[4];
            int32_t hprev = edge_flux(a.Af, q[r][0] - qL);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int32_t hnext = c < 3 ? edge_flux(a.Af, q[r][c + 1] - q[r][c]) : edge_flux(a.Af, qR - q[r][3]);
                const int32_t g2r = c < 3 ? G2[r][c + 1] : gR;
                const int32_t g2l = c > 0 ? G2[r][c - 1] : gL;
                // vertical: row 0 gains v1 and loses the flux across its upper edge,
                // row 1 the flux across its lower edge minus v1; transfers likewise
                const int32_t vert = r == 0 ? (v1[c] - edge_flux(a.Af, q[0][c] - qV[c])) + (G1[1][c] - gV[c])
                                            : (edge_flux(a.Af, qV[c] - q[1][c]) - v1[c]) + (gV[c] - G1[0][c]);
                nq[c] = q[r][c] + vert + (hnext - hprev) + (g2r - g2l);
                hprev = hnext;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) q[r][c] = nq[c];
        }
        if (cstep) {
            // ---- coarse step: the same on the coarse row
            int32_t cqL[1], cgL[1], cqR[1], cgR[1], cqU[2], cgU[2], cqD[2], cgD[2];
            cqL[0] = __shfl_sync(0xffffffffu, qc[0][1], (lane + 31) & 31);
            cgL[0] = __shfl_sync(0xffffffffu, Gc2[0][1], (lane + 31) & 31);
            cqR[0] = __shfl_sync(0xffffffffu, qc[0][0], (lane + 1) & 31);
            cgR[0] = __shfl_sync(0xffffffffu, Gc2[0][0], (lane + 1) & 31);
            if constexpr (WPR > 1) {
                if (lane == 0) {
                    const int2 u = sm.sch[((size_t)cr * WPR + (wc + WPR - 1) % WPR) * 2 + 1];
                    cqL[0] = u.x; cgL[0] = u.y;
                }
                if (lane == 31) {
                    const int2 u = sm.sch[((size_t)cr * WPR + (wc + 1) % WPR) * 2 + 0];
                    cqR[0] = u.x; cgR[0] = u.y;
                }
            }
            if (!top) {
                const int4 u = reinterpret_cast<const int4*>(sm.scv + (size_t)(cr - 1) * NC + ccol0)[0];
                cqU[0] = u.x; cgU[0] = u.y; cqU[1] = u.z; cgU[1] = u.w;
            } else {
                ldcg_int2x2(cedge + ((size_t)up * 2 + 1) * NC + ccol0, cqU, cgU);
            }
            if (!bot) {
                const int4 u = reinterpret_cast<const int4*>(sm.scv + (size_t)(cr + 1) * NC + ccol0)[0];
                cqD[0] = u.x; cgD[0] = u.y; cqD[1] = u.z; cgD[1] = u.w;
            } else {
                ldcg_int2x2(cedge + ((size_t)dn * 2 + 0) * NC + ccol0, cqD, cgD);
            }
            flux_update<1, 2>(qc, Gc1, Gc2, cqU, cgU, cqD, cgD, cqL, cgL, cqR, cgR, a.Ac);
            bad |= ((static_cast<uint32_t>(qc[0][0]) + 0x40000000u) | (static_cast<uint32_t>(qc[0][1]) + 0x40000000u)) >> 31;
        }
        if ((m & 3) == 3 || m + 1 == M) {
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) bad |= (static_cast<uint32_t>(q[r][c]) + 0x40000000u) >> 31;
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
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) mf += q[r][c];
        v[2 * kMaxObs] = static_cast<double>(mf);
#pragma unroll
        for (int k = 0; k < kMaxObs; ++k) {
            if (k >= a.n_obs) break;
            double sf = 0.0;
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const size_t x = (size_t)(frow + r) * NF + col0 + c;
                    sf = fma(static_cast<double>(q[r][c] - a.qbf[x]), b.phif64[(size_t)k * NF * NF + x], sf);
                }
            v[k] = sf;
        }
        if constexpr (CPL) {
            v[2 * kMaxObs + 1] = static_cast<double>((long long)qc[0][0] + qc[0][1]);
#pragma unroll
            for (int k = 0; k < kMaxObs; ++k) {
                if (k >= a.n_obs) break;
                double sc = 0.0;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const size_t x = (size_t)crow * NC + ccol0 + j;
                    sc = fma(static_cast<double>(qc[0][j] - a.qbc[x]), b.phic64[(size_t)k * NC * NC + x], sc);
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
        b.band_part[((size_t)s * b.nb + band) * kW + tid] = t;
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

template <int WPR, bool CPL>
cudaError_t band_attr(int bmax) {
    return cudaFuncSetAttribute(band_kernel<WPR, CPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)band_smem_bytes<WPR>(bmax));
}

template <int WPR, bool CPL>
cudaError_t band_occupancy(int bmax, int* per_sm) {
    cudaError_t e = band_attr<WPR, CPL>(bmax);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, band_kernel<WPR, CPL>, bmax * WPR * 32,
                                                         band_smem_bytes<WPR>(bmax));
}

template <int WPR, bool CPL>
cudaError_t band_launch(const KArgs& a, const BArgs& b, cudaStream_t st) {
    cudaError_t e = band_attr<WPR, CPL>(b.bmax);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b.S * b.nb);
    cfg.blockDim = dim3(b.bmax * WPR * 32);
    cfg.dynamicSmemBytes = band_smem_bytes<WPR>(b.bmax);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, band_kernel<WPR, CPL>, a, b);
}

cudaError_t band_occ(int n, bool coupled, int bmax, int* per_sm) {
    switch (n) {
        case 128: return coupled ? band_occupancy<1, true>(bmax, per_sm) : band_occupancy<1, false>(bmax, per_sm);
        case 256: return coupled ? band_occupancy<2, true>(bmax, per_sm) : band_occupancy<2, false>(bmax, per_sm);
        case 512: return coupled ? band_occupancy<4, true>(bmax, per_sm) : band_occupancy<4, false>(bmax, per_sm);
        case 1024: return coupled ? band_occupancy<8, true>(bmax, per_sm) : band_occupancy<8, false>(bmax, per_sm);
        default: return cudaErrorInvalidValue;
    }
}

size_t band_smem(int n, int bmax) {
    switch (n) {
        case 128: return band_smem_bytes<1>(bmax);
        case 256: return band_smem_bytes<2>(bmax);
        case 512: return band_smem_bytes<4>(bmax);
        case 1024: return band_smem_bytes<8>(bmax);
        default: return 0;
    }
}

}  // namespace

bool band_supported(int n) { return n == 128 || n == 256 || n == 512 || n == 1024; }

cudaError_t band_plan(int n, bool coupled, BandPlan* out) {
    *out = BandPlan{};
    if (!band_supported(n)) return cudaSuccess;
    const int wpr = n / 128, nc = n / 2, rows_max = 32 / wpr;
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    // Bands per sample nb: the tallest band (ceil(nc / nb) coarse rows) times the
    // CTAs an SM holds sets the time of a fine step, and S = floor(resident
    // CTAs / nb) samples run at once; pick the nb with the most samples per unit
    // of step time (ties: fewer, taller bands).
    double best = 0.0;
    for (int nb = std::max(2, (nc + rows_max - 1) / rows_max); nb <= nc / 2; ++nb) {
        const int bmax = (nc + nb - 1) / nb;
        if (bmax < 2) break;
        int per_sm = 0;
        if ((e = band_occ(n, coupled, bmax, &per_sm)) != cudaSuccess) return e;
        const int S = per_sm * sms / nb;
        if (S < 1) continue;
        const int ctas_per_sm = (S * nb + sms - 1) / sms;
        const double rate = (double)S / ((double)ctas_per_sm * (double)bmax);
        if (rate > best * 1.0001) {
            best = rate;
            out->supported = 1;
            out->nb = nb;
            out->bmax = bmax;
            out->S = S;
            out->threads = bmax * wpr * 32;
            out->smem = band_smem(n, bmax);
        }
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
        switch (n) {
            case 128: e = cpl ? band_launch<1, true>(k, b, st) : band_launch<1, false>(k, b, st); break;
            case 256: e = cpl ? band_launch<2, true>(k, b, st) : band_launch<2, false>(k, b, st); break;
            case 512: e = cpl ? band_launch<4, true>(k, b, st) : band_launch<4, false>(k, b, st); break;
            case 1024: e = cpl ? band_launch<8, true>(k, b, st) : band_launch<8, false>(k, b, st); break;
            default: e = cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
        band_finish_kernel<<<(b.count + 63) / 64, 64, 0, st>>>(k, b, p.S);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace dk
