// Device building blocks of the coupled Dean--Kawasaki step (sm_103a).
//
// Noise source: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) evaluated in
// registers, mapped to standard normals by Box--Muller.  The paper (Definition
// 2.1) only asks for independent Brownian increments per cell, component and
// step; the counter layout that makes sample i of level l a pure function of
// (seed, l, stream, i) is documented in include/mlmc_dk.h.
#pragma once
#include <cstdint>

namespace dk {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// Ten rounds: multiply words 0 and 2 by the round multipliers, xor the high
// halves with the opposite words and the round key, swap; the key advances by
// the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += kPhiloxW0;
            k1 += kPhiloxW1;
        }
        const unsigned long long p0 = static_cast<unsigned long long>(c.x) * kPhiloxM0;
        const unsigned long long p1 = static_cast<unsigned long long>(c.z) * kPhiloxM1;
        const uint32_t hi0 = static_cast<uint32_t>(p0 >> 32), lo0 = static_cast<uint32_t>(p0);
        const uint32_t hi1 = static_cast<uint32_t>(p1 >> 32), lo1 = static_cast<uint32_t>(p1);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Box--Muller in polar form: u = (a+1) 2^-32 in (0,1], theta = 2 pi (b + 1/2)
// 2^-32; returns the radius sqrt(-2 ln u) and (cos theta, sin theta), so that
// the normals are (r cos theta, r sin theta).  theta is evaluated as
// pi ((int)b + 1/2) 2^-31 (one fused multiply-add), which differs from it by a
// multiple of 2 pi, so that the hardware sine/cosine see |x| <= pi.
__device__ __forceinline__ void box_muller_polar(uint32_t a, uint32_t b, float& r, float& c, float& s) {
    const float u = fmaf(static_cast<float>(a), 2.3283064365386963e-10f, 2.3283064365386963e-10f);
    r = sqrt_approx(-1.3862943611198906f * __log2f(u));   // sqrt(-2 ln u)
    const float th = fmaf(static_cast<float>(static_cast<int32_t>(b)), 1.4629180792671596e-09f,
                          7.314590396335798e-10f);
    __sincosf(th, &s, &c);
}

__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& z1, float& z2) {
    float r, c, s;
    box_muller_polar(a, b, r, c, s);
    z1 = r * c;
    z2 = r * s;
}

// Progress counters shared between CTAs of one launch: an acquire load, a
// release increment (after the CTA's or warp's writes), a volatile read.
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

// Noise transfer G = rint(g sqrt(max(q,0)) z) in fixed-point units.
__device__ __forceinline__ float noise_amp(int32_t q, float g) {
    return g * sqrt_approx(__int2float_rn(max(q, 0)));
}

// The same for a fluctuation state dq = (rho - rho-bar) 2^S: the transfer is
// g sqrt([rho-bar + dq 2^-S]^+) z with g = c 2^S, rho-bar the noise-free path.
__device__ __forceinline__ float noise_amp_fluct(int32_t dq, float rbar, float inv_scale, float g) {
    return g * sqrt_approx(fmaxf(fmaf(__int2float_rn(dq), inv_scale, rbar), 0.f));
}

// Diffusion flux across one edge: round(a * (q_far - q_near)) with a given as
// A = round(a 2^32); computed identically by both cells of the edge.
__device__ __forceinline__ int32_t edge_flux(int32_t A, int32_t d) {
    const long long p = static_cast<long long>(A) * static_cast<long long>(d) + 0x80000000LL;
    return static_cast<int32_t>(p >> 32);
}

// Update of an RR x CC block of cells given its halo: explicit Euler--Maruyama
// step in flux form.  up/dn are the rows above/below the block, lf/rt the
// columns left/right; G1/G2 the noise transfers (component 1 along rows).
template <int RR, int CC>
__device__ __forceinline__ void flux_update(int32_t (&q)[RR][CC], const int32_t (&G1)[RR][CC],
                                            const int32_t (&G2)[RR][CC], const int32_t (&qU)[CC],
                                            const int32_t (&gU)[CC], const int32_t (&qD)[CC],
                                            const int32_t (&gD)[CC], const int32_t (&qL)[RR],
                                            const int32_t (&gL)[RR], const int32_t (&qR)[RR],
                                            const int32_t (&gR)[RR], int32_t A) {
    // vertical edge fluxes V[r][c]: across the edge between rows r-1 and r (r = 0..RR)
    int32_t V[RR + 1][CC];
#pragma unroll
    for (int c = 0; c < CC; ++c) {
        V[0][c] = edge_flux(A, q[0][c] - qU[c]);
#pragma unroll
        for (int r = 1; r < RR; ++r) V[r][c] = edge_flux(A, q[r][c] - q[r - 1][c]);
        V[RR][c] = edge_flux(A, qD[c] - q[RR - 1][c]);
    }
    int32_t H[RR][CC + 1];
#pragma unroll
    for (int r = 0; r < RR; ++r) {
        H[r][0] = edge_flux(A, q[r][0] - qL[r]);
#pragma unroll
        for (int c = 1; c < CC; ++c) H[r][c] = edge_flux(A, q[r][c] - q[r][c - 1]);
        H[r][CC] = edge_flux(A, qR[r] - q[r][CC - 1]);
    }
#pragma unroll
    for (int r = 0; r < RR; ++r) {
#pragma unroll
        for (int c = 0; c < CC; ++c) {
            const int32_t g1d = (r + 1 < RR) ? G1[r + 1][c] : gD[c];
            const int32_t g1u = (r > 0) ? G1[r - 1][c] : gU[c];
            const int32_t g2r = (c + 1 < CC) ? G2[r][c + 1] : gR[r];
            const int32_t g2l = (c > 0) ? G2[r][c - 1] : gL[r];
            q[r][c] += (V[r + 1][c] - V[r][c]) + (H[r][c + 1] - H[r][c]) + (g1d - g1u) + (g2r - g2l);
        }
    }
}

}  // namespace dk
