// Launch interface between the host runtime (mlmc_dk.cpp) and the CUDA
// kernels (dk_kernels.cu).  Plain structs and device pointers only.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace dk {

constexpr int kMaxObs = 4;
constexpr int kNSum = 12;   // per-quantity sums, layout as in include/mlmc_dk.h

// Everything one level launch needs (passed by value as a kernel parameter).
struct KArgs {
    const int32_t* q0f;     // fine initial state, fixed point, n^2
    const int32_t* qbf;     // fine discrete mean field at T, fixed point, n^2
    const float* phif;      // fine test functions [n_obs][n^2]
    const int32_t* q0c;     // coarse (level l-1) tables, (n/2)^2
    const int32_t* qbc;
    const float* phic;
    double* partials;       // scratch: [n_slots][slot_stride] per-slot sums
    double* samples;        // optional per-sample output [count][2 n_obs + 2]
    unsigned int* err;      // sticky device error bits
    int64_t first;          // first sample id
    int64_t count;          // number of samples
    int32_t M;              // fine steps
    int32_t n_obs;
    int32_t n_quant;
    int32_t products;
    int32_t Af, Ac;         // diffusion multipliers round(tau/(2h^2) 2^32)
    float gf, gc;           // noise multipliers (gc includes the 1/4 of the coupled sum)
    uint32_t key0, key1;    // seed words
    uint32_t tag;           // (level + 1) | stream << 8
    int32_t slot_stride;    // 2 + kNSum * n_quant doubles
    double N;
    double dscale_f, dscale_c;        // h^2 2^-S: fixed-point sums -> (rho, phi)_h
    double delta_f[kMaxObs], delta_c[kMaxObs];  // (2^-S qbar - rho-bar^T, phi)_h
    double mscale_f, mscale_c;        // h^2 2^-S for the mass
    long long mass0_f, mass0_c;       // sum of the initial fixed-point states
    // fluctuation state (kernels built with it only): q = (rho - rho-bar^m) 2^S
    const float* rbf;                 // fine noise-free path rho-bar^m, [M][n^2] (m = 0 .. M-1)
    const float* rbc;                 // coarse noise-free path, [M/4][(n/2)^2]
    float isf, isc;                   // 2^-S of the fine / coarse level
    double mass_off_f, mass_off_c;    // (rho-bar, 1)_h added to the reported masses (0 for absolute states)
};

enum : unsigned int { kErrRange = 1u, kErrTimeout = 2u };

// Static facts about the kernel variant used for a grid size.
struct VariantInfo {
    int supported;
    int threads;            // threads per CTA
    int cluster;            // CTAs per cluster (1 = no cluster)
    int slots_per_cta;      // samples in flight per CTA (1/cluster for clusters)
    size_t smem;            // dynamic shared memory per CTA
    int max_ctas;           // resident CTAs on the whole GPU
    int C, R;               // lane block: C x R coarse cells (2R x 2C fine)
    int tile_rows;          // streamed kernels: fine rows per CTA tile (0 for the register kernels)
    int persistent;         // streamed kernels: 1 = one launch per wave (work items from a counter)
    int pdl;                // streamed kernels: 1 = programmatic dependent launches (one per step)
    int band;               // 1: the band kernel (a sample over several CTAs, cooperative launch)
    int bands;              // band kernel: bands (CTAs) per sample
};

// Number of kernel variants (lane-block shapes / cluster sizes) for fine size n;
// `fluct`: the builds for a fluctuation state (KArgs::rbf).
int variant_count(int n, bool fluct = false);

// Query (and prepare: attributes, occupancy) variant `idx` for fine size n;
// supported = 0 when it does not exist.
cudaError_t variant_info(int n, bool coupled, int slot_stride, int idx, VariantInfo* out, bool fluct = false);

// Launch one batch with variant `idx` on n_ctas CTAs; partials must hold
// (n_ctas / cluster) * slots_per_cta * slot_stride doubles.
// `priority` (0: none) is passed as the launch's scheduling priority (lower
// numbers are more urgent, as for streams).
cudaError_t launch_level(int n, bool coupled, int idx, const KArgs& a, int n_ctas, cudaStream_t stream,
                         int priority = 0, bool fluct = false);

// Deterministic fixed-order reduction of the per-slot partials into
// out[slot_stride]: entry 1 is a max, all others sums.
cudaError_t launch_reduce(const double* partials, int n_slots, int slot_stride, double* out,
                          cudaStream_t stream);
// out[e] += in[e] for the slot_stride entries of one level's sums (entry 1: max).
cudaError_t launch_add_sums(double* out, const double* in, int slot_stride, cudaStream_t stream);

// ---- streamed-state path (grids without a register-resident variant)
struct SArgs {
    int n, nc, M, coupled, n_obs;
    int count;                   // samples in this wave (<= samples in flight)
    long long sid0;              // sample id of the wave's first sample
    int32_t* q[2];               // [S][n][n] fine state, double buffered
    int32_t* qc[2];              // [S][n/2][n/2] coarse state, double buffered
    float2* zt;                  // [S][n/2][n/2] coupled normal sums of the current coarse step
    double* tile_part;           // [S][tiles][2 kMaxObs + 2] per-tile observables
    const int32_t* q0f; const int32_t* qbf; const float* phif;
    const int32_t* q0c; const int32_t* qbc; const float* phic;
    const double* phif64; const double* phic64;   // FP64 test functions (observables)
    int32_t Af, Ac;
    float gf, gc;
    uint32_t key0, key1, tag;
    unsigned int* err;
    // persistent launch: progress counters (fine steps done per fine tile,
    // coarse steps done per coarse tile), the item counter, their region,
    // the poll limit of every wait, and a tile (of sample 0) that never
    // reports its step 1 (-1: none; failure-detection test only)
    unsigned int* fdone;
    unsigned int* cdone;
    unsigned long long* head;
    void* counters;
    size_t counter_bytes;
    unsigned int wait_polls;
    int stall_tile;
};

// Device bytes for `S` samples in flight on an n x n grid, and their layout.
size_t stream_bytes(int n, int S);
// Fine-step tile variants of the streamed kernels (FR x 64 fine cells per CTA,
// FR = tile_rows), their launch shape on this device, and the samples in
// flight for an n x n level within `budget` bytes of working set, chosen so
// that the fine-step CTAs of `variant` fill whole waves of the GPU.
int stream_variant_count();
int stream_default_variant();
cudaError_t stream_variant_info(int n, int variant, VariantInfo* out);
int stream_inflight(int n, size_t budget, int variant);
void stream_carve(SArgs* a, void* buf, int n, int S);

// Run k.count samples (ids k.first..) in waves of S: per-slot moment sums go
// to k.partials ([k.slot_stride][S], zeroed here), per-sample outputs to
// k.samples; the caller reduces the S slots.
cudaError_t stream_run(const KArgs& k, SArgs a, int S, int variant, cudaStream_t stream);

// ---- band kernels (grids 128 .. 1024): a sample over several CTAs, each a
// full-width band of coarse rows held in registers; band edges through global
// memory with per-step counters; cooperative launch
struct BArgs {
    int n, coupled;
    int nb, bmax, S;             // bands per sample, coarse rows of the tallest band, samples in flight
    int steps;                   // fine steps (the level's M, fewer only to time variants)
    int count;                   // samples in this wave (<= S)
    long long sid0;              // sample id of the wave's first sample
    unsigned* flags;             // [S][nb][2]: published top / bottom edges (zeroed before every wave)
    int2* edge;                  // [S][nb][2 side][2 parity][n]: (q, G1) of the top / bottom fine row
    int2* cedge;                 // [S][nb][2 side][n/2]: (qc, Gc1) of the top / bottom coarse row
    double* band_part;           // [S][nb][2 kMaxObs + 2]: per-band observable partials
    const double* phif64;        // FP64 test functions [n_obs][n^2] / [n_obs][(n/2)^2]
    const double* phic64;
    unsigned wait_polls;         // polls before a wait gives up (0: the default, about a second or more)
    int stall_band;              // -1; >= 0 only in the failure-detection test: that band never publishes
};
struct BandPlan {
    int supported;
    int fc;                      // fine columns per thread (4: 4 x 4 blocks, 8: 4 x 8 blocks)
    int nb, bmax, S, threads;
    size_t smem;
};
bool band_supported(int n, int fc);
// Launch shape of the band kernel build with 4 x fc thread blocks for n x n on
// this device (see dk_band.cu); supported = 0 where that build does not exist.
cudaError_t band_plan(int n, bool coupled, int fc, BandPlan* out);
// Device bytes of the exchange buffers for `p`, and their layout.
size_t band_bytes(int n, const BandPlan& p);
void band_carve(BArgs* b, void* buf, int n, const BandPlan& p);
// Run k.count samples (ids k.first..) in waves of p.S: per-slot moment sums go
// to k.partials ([k.slot_stride][p.S], zeroed here); the caller reduces the slots.
cudaError_t band_run(const KArgs& k, BArgs b, const BandPlan& p, cudaStream_t stream);

// ---- theta-scheme (implicit diffusion weight b0 > 0), grids up to 64 x 64
constexpr int kMaxCheb = 64;   // largest number of Chebyshev steps per solve
struct TArgs {
    int K;                     // Chebyshev steps per solve (0: the explicit step)
    float alpha;               // b0 tau / (2 h^2), the same on every level
    float inv_theta;           // 1 / (1 + 4 alpha): first step of the iteration
    float c1[kMaxCheb];        // direction recurrence d <- c1[k] d + c2[k] r
    float c2[kMaxCheb];
    long long Af64, Ac64;      // round(tau / (2 h^2) 2^32) of the fine / coarse grid (64-bit: tau/h^2 may exceed 1)
    const double* phif64;      // FP64 test functions [n_obs][n^2] / [n_obs][(n/2)^2]
    const double* phic64;
};
bool theta_supported(int n);
cudaError_t theta_variant_info(int n, bool coupled, int slot_stride, VariantInfo* out);
// Launch one batch of the theta-scheme kernel on n_ctas CTAs; partials must hold
// n_ctas * slots_per_cta * slot_stride doubles.
cudaError_t launch_theta(int n, bool coupled, const KArgs& a, const TArgs& t, int n_ctas, cudaStream_t stream,
                         int priority = 0);

// ---- Fourier coupling (Section 3.1): grids 6, 18, 54 (h ratio 3, tau ratio 9)
struct FArgs {
    const float* P1;           // [n/3][n] restriction of the fine normals to the coarse grid (coupled only)
    const double* phif64;      // FP64 test functions [n_obs][n^2] / [n_obs][(n/3)^2]
    const double* phic64;
};
bool fourier_supported(int n);
// fluct: the fluctuation-state build (KArgs::rbf / rbc tables required)
cudaError_t fourier_variant_info(int n, bool coupled, int slot_stride, VariantInfo* out, bool fluct = false);
// One CTA per sample slot; partials must hold n_ctas * slot_stride doubles.
cudaError_t launch_fourier(int n, bool coupled, const KArgs& a, const FArgs& f, int n_ctas, cudaStream_t stream,
                           int priority = 0, bool fluct = false);
// Grids beyond one CTA (162^2, coupled with 54^2): clusters of 6 CTAs, one
// sample slot per cluster; n_ctas a multiple of 6.
bool fourier_cluster_supported(int n);
cudaError_t fourier_cluster_variant_info(int n, bool coupled, int slot_stride, VariantInfo* out);
cudaError_t launch_fourier_cluster(int n, bool coupled, const KArgs& a, const FArgs& f, int n_ctas,
                                   cudaStream_t stream, int priority);

// ---- learned level below level 0
constexpr int kModes = 32;     // real orthonormal modes
constexpr int kFeat = 64;      // features = modes x 2 noise components
constexpr int kHidden = 256;

struct FeatArgs {
    const float* E;            // [32][n*n] mode table (plain-sum orthonormal)
    const float* g;            // [32] per-step factor of the noise-free scheme on each mode
    const float* inv_sigma;    // [64] 1 / standard deviation of each feature
    int n, M;
    uint32_t key0, key1, tag;
    long long first, count;
    __nv_bfloat16* X;          // [count][64] standardised features
    float* Xf;                 // optional FP32 copy
};

struct GemmArgs {
    int M, N, K;
    const __nv_bfloat16* A; long long sam, sak;   // A[m][k] = A[m*sam + k*sak]
    const __nv_bfloat16* B; long long sbk, sbn;   // B[k][n] = B[k*sbk + n*sbn]
    float* C; long long ldc;                       // optional FP32 output
    __nv_bfloat16* Cb; long long ldcb;             // optional BF16 output
    const float* bias;                             // optional bias[n]
    int relu;
    const __nv_bfloat16* mask; long long ldm;      // optional: zero where mask <= 0
};

cudaError_t launch_features(const FeatArgs& a, int max_ctas, cudaStream_t st);
cudaError_t launch_direct_features(const FeatArgs& a, cudaStream_t st);
// C = A B on the 5th-generation tensor cores (dk_umma.cu): A [M][K] and B
// given as [N][K], both K-major (sak == sbk == 1), N <= 256; epilogue as in
// GemmArgs; bounded waits record kErrTimeout in *err.
cudaError_t launch_gemm_tc(const GemmArgs& g, unsigned* err, cudaStream_t st);
// out[c][r] = in[r][c] for an R x C BF16 matrix, output rows ldo >= R apart.
cudaError_t launch_transpose_bf16(const __nv_bfloat16* in, int R, int C, __nv_bfloat16* out, int ldo,
                                  cudaStream_t st);
// Output layer with KO outputs (one per test function): y [B][KO]; weights
// w4 [KO][K], biases b4 [KO].
cudaError_t launch_out_forward(const __nv_bfloat16* H, const float* w, const float* b, int B, int K, int KO, float* y,
                               cudaStream_t st);
cudaError_t launch_out_backward(const float* y, const float* t, const __nv_bfloat16* H, const float* w, int B, int K,
                                int KO, float* dy, __nv_bfloat16* dH, float* dw, float* db, cudaStream_t st);
cudaError_t launch_colsum(const __nv_bfloat16* Xb, const float* Xf, int B, int N, float* out, cudaStream_t st);
cudaError_t launch_adam(float* theta, const float* grad, float* m1, float* m2, int P, float lr, float b1, float b2,
                        float eps, float c1, float c2, const int* bf_index, __nv_bfloat16* theta_bf, cudaStream_t st);
cudaError_t launch_gather(const __nv_bfloat16* X, const float* T, const int* idx, int B, int KO, __nv_bfloat16* Xb,
                          float* Tb, cudaStream_t st);
// sum of squared differences of n values, divided by B
cudaError_t launch_mse(const float* y, const float* t, int n, int B, double* out, cudaStream_t st);
cudaError_t launch_surrogate_moments(const float* that, const double* d0, int d0_stride, int part, double N,
                                     long long count, int stride, int KO, int products, int blocks, double* partials,
                                     cudaStream_t st);

// Device address and size (doubles) of the statically allocated scratch used
// by mlmc_dk_run_level_static; the first call on a device looks the address up
// with cudaGetSymbolAddress (device must be current).
constexpr size_t kStaticScratchDoubles = size_t(1) << 19;   // 4 MiB
cudaError_t static_scratch(double** out, size_t* capacity);

// Normals (and raw Philox words) of one fine step: z [n*n][2], raw [n*n/2][4].
cudaError_t launch_noise(int n, uint32_t m, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1, float* z,
                         uint32_t* raw, cudaStream_t stream);

}  // namespace dk
