// Host runtime behind include/mlmc_dk.h: level hierarchy, discrete mean field,
// fixed-point tables, kernel launches, Algorithm 1 and checkpointing.
#include "mlmc_dk.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <numeric>
#include <random>
#include <cstring>
#include <functional>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dk_kernels.h"

namespace {

thread_local std::string g_init_error;

struct LevelTab {
    int n = 0, M = 0;
    double h = 0, tau = 0;
    int S = 24;              // fixed-point fraction bits: rho = q 2^-S
    int32_t A = 0;           // round(tau / (2 h^2) 2^32) (explicit kernels: tau/h^2 <= 1/2)
    long long A64 = 0;       // the same in 64 bits (theta-scheme kernel, where tau/h^2 may exceed 1)
    float g = 0.f;           // N^-1/2 sqrt(tau) / (2 h^2) 2^(S/2)
    double dscale = 0;       // h^2 2^-S
    long long mass0 = 0;     // sum of q0
    double ybar[MLMC_DK_MAX_OBS] = {0, 0, 0, 0};
    double delta[MLMC_DK_MAX_OBS] = {0, 0, 0, 0};
    int32_t* d_q0 = nullptr;
    int32_t* d_qbar = nullptr;
    float* d_phi = nullptr;
    double* d_phi64 = nullptr;             // the same test functions in FP64 (observables of the streamed path)
    float* d_P1 = nullptr;                 // Fourier coupling: restriction of this level's normals to level l-1
    std::vector<dk::VariantInfo> vis[2];   // kernel variants: [0] fine path only, [1] coupled pair
    int streamed = 0;                      // no register variant: state streamed through global memory
    int inflight = 0;                      // samples in flight on the streamed path (buffers sized for this)
    int inflight_v[8] = {0};               // ... per streamed tile variant
    int split_ok = 0;                      // register level that can also run samples streamed (batch split)
    double split_frac = 0.0;               // share of a batch's samples run on the streamed kernels
    int64_t batch_streamed = 0;            // samples of the last batch run on the streamed kernels
    void* d_stream = nullptr;              // their state
    double* d_spart = nullptr;             // their per-slot partial sums [stride][S]
    int sel[2] = {0, 0};                   // variant in use for each mode
    dk::BandPlan bplan[2][2] = {};         // band kernel launch shapes [mode: fine only, coupled][build: 4, 8 columns]
    void* d_band = nullptr;                // its exchange buffers
    double* d_bpart = nullptr;             // its per-slot partial sums [stride][S]
    float* d_rbar = nullptr;               // fluctuation state: noise-free path rho-bar^m, [M][n^2] FP32
    double mass_bar = 0.0;                 // fluctuation state: (rho-bar, 1)_h, added to reported masses
    const dk::VariantInfo& vi(bool coupled) const {
        static const dk::VariantInfo none{};
        const auto& v = vis[coupled ? 1 : 0];
        return v.empty() ? none : v[sel[coupled ? 1 : 0]];
    }
};

}  // namespace

struct mlmc_dk_ctx {
    double length = 1, T = 0, N = 0;
    int L_max = 0, n_obs = 1, products = 0, n_quant = 1, stride = 0, pilot = 256, L_start = 2;
    double b0 = 0;              // implicit weight of Eq. (FullyDiscreteDK)
    int theta = 0;              // every level runs on the theta-scheme kernel
    int coupling = 0;           // 0: Right-Most NN (h ratio 2); 1: Fourier (h ratio 3, Section 3.1)
    int fluct = 0;              // 1: states are fluctuations about the noise-free path (see mlmc_dk_init)
    dk::TArgs targs{};          // its Chebyshev schedule (per-level fields filled at launch)
    std::vector<LevelTab> lv;
    cudaStream_t stream = nullptr;
    double* d_partials = nullptr;
    size_t partials_cap = 0;   // doubles
    double* d_sums = nullptr;
    double* h_sums = nullptr;  // pinned
    unsigned* d_err = nullptr;
    unsigned* h_err = nullptr;  // pinned
    int64_t h2d_bytes = 0;      // bytes uploaded by mlmc_dk_init
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<int64_t> next_id[2];
    std::string err;
    // multi-level batch: one stream and one scratch buffer per level, the
    // captured CUDA graph of the last batch shape
    std::vector<cudaStream_t> lstream;
    std::vector<double*> d_lpart;
    std::vector<size_t> lpart_cap;
    std::vector<int> lprio;
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;
    std::vector<cudaEvent_t> ev_lb, ev_le;   // timing of each level inside the batch
    cudaGraphExec_t gexec = nullptr;
    // batch split: samples of a cluster level run on the streamed kernels
    // beside the graph, on the least urgent stream, on the SMs clusters leave
    cudaStream_t sstream = nullptr;
    cudaEvent_t ev_sfork = nullptr, ev_sjoin = nullptr;
    cudaEvent_t ev_graph = nullptr;        // the batch graph's completion (streamed levels start after it)
    double* d_ssums = nullptr;        // [L_max+1][stride] sums of the streamed share
    double* d_bsums = nullptr;        // device sums of mlmc_dk_run_batch
    double* h_bsums = nullptr;        // pinned host copy
    struct Surrogate* sur = nullptr;  // learned level below level 0 (mlmc_dk_surrogate_init)
};

// Learned level below level 0: mode tables, network parameters (FP32 master,
// BF16 copies of the weight matrices, Adam moments) and chunk buffers.
struct Surrogate {
    int n = 0, M = 0;
    int K = 1;                         // network outputs: one per test function
    int products = 0;                  // quantities S_jl = That_j That_l for all j <= l
    int P = 0;                         // parameters (148224 + 257 K)
    int sampw = 4;                     // doubles per level-0 per-sample output (2 K + 2)
    int chunk = 65536;                 // samples per inference chunk
    int batch_cap = 0;                 // largest training batch
    float *d_E = nullptr, *d_g = nullptr, *d_inv_sigma = nullptr;
    float *d_theta = nullptr, *d_grad = nullptr, *d_m1 = nullptr, *d_m2 = nullptr;
    __nv_bfloat16* d_wbf = nullptr;    // BF16 W1 | W2 | W3 | W4
    int* d_bfidx = nullptr;            // parameter -> BF16 index (-1 for biases)
    __nv_bfloat16 *d_X = nullptr, *d_H1 = nullptr, *d_H2 = nullptr, *d_H3 = nullptr;
    __nv_bfloat16 *d_dH1 = nullptr, *d_dH2 = nullptr, *d_dH3 = nullptr;
    // K-major operands of the backward GEMMs: dH^T, Hin^T [256][batch], W^T [256][256]
    __nv_bfloat16 *d_tA = nullptr, *d_tB = nullptr, *d_wt = nullptr;
    unsigned* err = nullptr;           // the context's device error word (bounded waits of the GEMM)
    float *d_y = nullptr, *d_dy = nullptr, *d_T = nullptr, *d_Xf = nullptr;
    double* d_samp = nullptr;          // level-0 per-sample outputs of a chunk
    double* d_D0 = nullptr;
    double* d_part = nullptr;          // moment partials [stride][blocks]
    double* d_loss = nullptr;
    __nv_bfloat16* d_trainX = nullptr; // training pairs
    float* d_trainT = nullptr;
    int* d_idx = nullptr;
    int64_t n_train = 0;
    int64_t adam_t = 0;
    int64_t next_id[2] = {0, 0};       // [0] level below 0, [1] correction level
    double kernel_s[2] = {0, 0};
};

namespace {
void free_surrogate(Surrogate* s);

int fail(mlmc_dk_ctx* ctx, int code, const std::string& msg) {
    static std::mutex m;   // the batch enqueues streamed levels from several host threads
    std::lock_guard<std::mutex> lock(m);
    if (ctx) ctx->err = msg; else g_init_error = msg;
    return code;
}

int cuda_fail(mlmc_dk_ctx* ctx, cudaError_t e, const char* what) {
    return fail(ctx, MLMC_DK_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// ---------------------------------------------------------------- FFT (FP64)
// In-place iterative radix-2 complex transform of length n (a power of two);
// sign = -1 forward, +1 inverse (unnormalised).
void fft1(std::complex<double>* a, int n, int stride, int sign) {
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[(size_t)i * stride], a[(size_t)j * stride]);
    }
    for (int len = 2; len <= n; len <<= 1) {
        const double ang = sign * 2.0 * M_PI / len;
        for (int i = 0; i < n; i += len) {
            for (int k = 0; k < len / 2; ++k) {
                const std::complex<double> w(std::cos(ang * k), std::sin(ang * k));
                std::complex<double>& x = a[(size_t)(i + k) * stride];
                std::complex<double>& y = a[(size_t)(i + k + len / 2) * stride];
                const std::complex<double> t = w * y;
                y = x - t;
                x = x + t;
            }
        }
    }
}

void fft2(std::vector<std::complex<double>>& a, int n, int sign) {
    for (int r = 0; r < n; ++r) fft1(a.data() + (size_t)r * n, n, 1, sign);
    for (int c = 0; c < n; ++c) fft1(a.data() + c, n, n, sign);
}

// Noise-free scheme iterated M times: with lam = 2 (tau/h^2)(sin^2(pi k1/n) +
// sin^2(pi k2/n)) (tau/2 Delta_h of Section 7.2 acts on discrete Fourier mode
// k as -lam), the weights (b0, b1 = 1 - b0) of Eq. (FullyDiscreteDK) multiply
// the mode by (1 - b1 lam) / (1 + b0 lam) per step (1 - lam for the explicit
// scheme).
void mean_field(int n, double h, double tau, long long M, const double* rho0, double* out, double b0 = 0.0) {
    std::vector<std::complex<double>> a((size_t)n * n);
    for (size_t i = 0; i < a.size(); ++i) a[i] = rho0[i];
    fft2(a, n, -1);
    const double mu = tau / (h * h);
    std::vector<double> s2(n);
    for (int k = 0; k < n; ++k) {
        const double s = std::sin(M_PI * k / n);
        s2[k] = s * s;
    }
    for (int k1 = 0; k1 < n; ++k1)
        for (int k2 = 0; k2 < n; ++k2) {
            const double lam = 2.0 * mu * (s2[k1] + s2[k2]);
            const double g = b0 == 0.0 ? 1.0 - lam : (1.0 - (1.0 - b0) * lam) / (1.0 + b0 * lam);
            a[(size_t)k1 * n + k2] *= std::pow(g, (double)M);
        }
    fft2(a, n, +1);
    const double inv = 1.0 / ((double)n * n);
    for (size_t i = 0; i < a.size(); ++i) out[i] = a[i].real() * inv;
}

// The same for any even n (grids of the Fourier coupling are not powers of
// two): the noise-free step applied M times in FP64 (5-point stencil; the
// implicit half, if any, by the Fourier symbol).
void mean_field_any(int n, double h, double tau, long long M, const double* rho0, double* out, double b0 = 0.0) {
    if (is_pow2(n)) {
        mean_field(n, h, tau, M, rho0, out, b0);
        return;
    }
    std::vector<double> a(rho0, rho0 + (size_t)n * n), b((size_t)n * n);
    const double w = tau / (2.0 * h * h);
    for (long long m = 0; m < M; ++m) {
        for (int i1 = 0; i1 < n; ++i1)
            for (int i2 = 0; i2 < n; ++i2) {
                const double c = a[(size_t)i1 * n + i2];
                const double s = a[(size_t)((i1 + 1) % n) * n + i2] + a[(size_t)((i1 + n - 1) % n) * n + i2] +
                                 a[(size_t)i1 * n + (i2 + 1) % n] + a[(size_t)i1 * n + (i2 + n - 1) % n];
                b[(size_t)i1 * n + i2] = c + w * (s - 4.0 * c);
            }
        a.swap(b);
    }
    std::copy(a.begin(), a.end(), out);
}

// Chebyshev iteration on the spectrum [1, 1 + 8 alpha] of I + alpha L (the
// theta-scheme's implicit operator): after K steps the error is at most
// 1 / T_K(sigma) of the initial one, sigma = (1 + 4 alpha) / (4 alpha); K is the
// first with that below 2^-27, and the direction recurrence d <- c1[k] d +
// c2[k] r follows Chebyshev acceleration (Saad, Iterative Methods for Sparse
// Linear Systems, Algorithm 12.1).  Returns false if K would exceed kMaxCheb.
bool chebyshev_schedule(double alpha, int* K_out, float* c1, float* c2) {
    *K_out = 0;
    if (!(alpha > 0.0)) return true;
    const double sigma = (1.0 + 4.0 * alpha) / (4.0 * alpha), delta = 4.0 * alpha;
    int K = 1;
    while (K <= dk::kMaxCheb && std::cosh(K * std::acosh(sigma)) < std::ldexp(1.0, 27)) ++K;
    if (K > dk::kMaxCheb) return false;
    double rho = 1.0 / sigma;
    for (int k = 0; k < K; ++k) {
        const double next = 1.0 / (2.0 * sigma - rho);
        c1[k] = (float)(next * rho);
        c2[k] = (float)(2.0 * next / delta);
        rho = next;
    }
    *K_out = K;
    return true;
}

// Restriction of the Fourier coupling (Section 3.1) along one axis, an
// (n/3) x n matrix: P1[y][x] = (n nc)^-1/2 sum_{xi=-nc/2..nc/2} w(xi)
// cos(2 pi xi (y/nc - x/n)), w = 2^-1/2 at xi = +-nc/2 (the two fine aliases of
// the coarse Nyquist mode) and 1 otherwise; coarse point y is fine point 3y.
void fourier_restriction(int n, float* P1) {
    const int nc = n / 3, K = nc / 2;
    for (int y = 0; y < nc; ++y)
        for (int x = 0; x < n; ++x) {
            double v = 0.0;
            for (int xi = -K; xi <= K; ++xi) {
                const double w = (xi == K || xi == -K) ? M_SQRT1_2 : 1.0;
                v += w * std::cos(2.0 * M_PI * xi * ((double)y / nc - (double)x / n));
            }
            P1[(size_t)y * n + x] = (float)(v / std::sqrt((double)n * nc));
        }
}

int quantities(int n_obs, int products) { return products ? n_obs * (n_obs + 1) / 2 : n_obs; }

// Fill the kernel arguments of one batch.
dk::KArgs make_args(mlmc_dk_ctx* c, int level, int stream_tag, bool coupled, int64_t first, int64_t count,
                    uint64_t seed, double* samples) {
    const LevelTab& f = c->lv[level];
    dk::KArgs a{};
    a.q0f = f.d_q0;
    a.qbf = f.d_qbar;
    a.phif = f.d_phi;
    a.partials = c->d_partials;
    a.samples = samples;
    a.err = c->d_err;
    a.first = first;
    a.count = count;
    a.M = f.M;
    a.n_obs = c->n_obs;
    a.n_quant = c->n_quant;
    a.products = c->products;
    a.Af = f.A;
    a.gf = f.g;
    a.key0 = (uint32_t)(seed & 0xffffffffu);
    a.key1 = (uint32_t)(seed >> 32);
    a.tag = ((uint32_t)(level + 1) & 0xffu) | (((uint32_t)stream_tag & 0xffu) << 8);
    a.slot_stride = c->stride;
    a.N = c->N;
    a.dscale_f = f.dscale;
    a.mass0_f = f.mass0;
    for (int k = 0; k < dk::kMaxObs; ++k) a.delta_f[k] = f.delta[k];
    if (c->fluct) {
        a.rbf = f.d_rbar;
        a.isf = (float)std::ldexp(1.0, -f.S);
        a.mass_off_f = f.mass_bar;
    }
    if (coupled) {
        const LevelTab& g = c->lv[level - 1];
        a.q0c = g.d_q0;
        a.qbc = g.d_qbar;
        a.phic = g.d_phi;
        a.Ac = g.A;
        // coupled coarse normal: NN 1/4 x (sum of 16 fine normals); Fourier 1/3 x (restriction
        // of the sum of 9 fine normal fields, each restricted field white with unit variance)
        a.gc = c->coupling == 1 ? g.g / 3.0f : 0.25f * g.g;
        a.dscale_c = g.dscale;
        a.mass0_c = g.mass0;
        for (int k = 0; k < dk::kMaxObs; ++k) a.delta_c[k] = g.delta[k];
        if (c->fluct) {
            a.rbc = g.d_rbar;
            a.isc = (float)std::ldexp(1.0, -g.S);
            a.mass_off_c = g.mass_bar;
        }
    }
    return a;
}

// Launch one batch with the given scratch and reduce it into sums_dev.
int launch_batch_into(mlmc_dk_ctx* c, int level, int stream_tag, int64_t first, int64_t count, uint64_t seed,
                      double* sums_dev, double* samples_dev, cudaStream_t st, double* partials, size_t cap,
                      int priority);

// Launch one batch and reduce it into sums_dev (device, stride doubles).
int launch_batch(mlmc_dk_ctx* c, int level, int stream_tag, int64_t first, int64_t count, uint64_t seed,
                 double* sums_dev, double* samples_dev, cudaStream_t st) {
    return launch_batch_into(c, level, stream_tag, first, count, seed, sums_dev, samples_dev, st, c->d_partials,
                             c->partials_cap, 0);
}

// Streamed level (state in global memory); `steps` > 0 truncates every sample
// to that many fine steps (used only to time the tile variants).
// `variant` >= 0 picks the fine-step tile (levels that normally run the
// register kernels); otherwise the level's tuned streamed variant.
int launch_streamed(mlmc_dk_ctx* c, int level, int stream_tag, int64_t first, int64_t count, uint64_t seed,
                    double* sums_dev, double* samples_dev, cudaStream_t st, int steps = 0, int variant = -1,
                    unsigned wait_polls = 0, int stall_tile = -1) {
    const bool coupled = (stream_tag == 0) && level > 0;
    LevelTab& t = c->lv[level];
    if (variant < 0) variant = t.sel[coupled ? 1 : 0];
    cudaError_t e;
    if (count == 0) {
        e = cudaMemsetAsync(sums_dev, 0, sizeof(double) * c->stride, st);
        return e == cudaSuccess ? MLMC_DK_OK : cuda_fail(c, e, "cudaMemsetAsync");
    }
    dk::KArgs k = make_args(c, level, stream_tag, coupled, first, count, seed, samples_dev);
    k.partials = t.d_spart;
    dk::SArgs a{};
    dk::stream_carve(&a, t.d_stream, t.n, t.inflight);
    a.n = t.n;
    a.nc = t.n / 2;
    a.M = steps > 0 ? steps : t.M;
    a.coupled = coupled ? 1 : 0;
    a.n_obs = c->n_obs;
    a.q0f = k.q0f; a.qbf = k.qbf; a.phif = k.phif;
    a.q0c = k.q0c; a.qbc = k.qbc; a.phic = k.phic;
    a.phif64 = t.d_phi64;
    a.phic64 = coupled ? c->lv[level - 1].d_phi64 : nullptr;
    a.Af = k.Af; a.Ac = k.Ac; a.gf = k.gf; a.gc = k.gc;
    a.key0 = k.key0; a.key1 = k.key1; a.tag = k.tag;
    a.err = c->d_err;
    a.wait_polls = wait_polls;
    a.stall_tile = stall_tile;
    const int S = t.inflight_v[variant];
    if ((e = dk::stream_run(k, a, S, variant, st)) != cudaSuccess) return cuda_fail(c, e, "streamed level");
    if ((e = dk::launch_reduce(t.d_spart, S, c->stride, sums_dev, st)) != cudaSuccess)
        return cuda_fail(c, e, "reduce kernel launch");
    return MLMC_DK_OK;
}

// Band-kernel level: each sample over t.bplan[mode].nb CTAs; `steps` > 0
// truncates every sample to that many fine steps (used only to time variants).
int launch_band(mlmc_dk_ctx* c, int level, int stream_tag, int64_t first, int64_t count, uint64_t seed,
                double* sums_dev, double* samples_dev, cudaStream_t st, int steps = 0, unsigned wait_polls = 0,
                int stall_band = -1) {
    const bool coupled = (stream_tag == 0) && level > 0;
    LevelTab& t = c->lv[level];
    const int fc = t.vi(coupled).band ? t.vi(coupled).band : (t.bplan[coupled ? 1 : 0][0].supported ? 4 : 8);
    const dk::BandPlan& p = t.bplan[coupled ? 1 : 0][fc == 4 ? 0 : 1];
    cudaError_t e;
    if (count == 0) {
        e = cudaMemsetAsync(sums_dev, 0, sizeof(double) * c->stride, st);
        return e == cudaSuccess ? MLMC_DK_OK : cuda_fail(c, e, "cudaMemsetAsync");
    }
    if (!p.supported || !t.d_band) return fail(c, MLMC_DK_ERR_UNSUPPORTED, "no band kernel for this level");
    dk::KArgs k = make_args(c, level, stream_tag, coupled, first, count, seed, samples_dev);
    k.partials = t.d_bpart;
    dk::BArgs b{};
    dk::band_carve(&b, t.d_band, t.n, p);
    b.n = t.n;
    b.coupled = coupled ? 1 : 0;
    b.steps = steps > 0 ? std::min(steps, t.M) : t.M;
    b.wait_polls = wait_polls;
    b.stall_band = stall_band;
    b.phif64 = t.d_phi64;
    b.phic64 = coupled ? c->lv[level - 1].d_phi64 : nullptr;
    if ((e = dk::band_run(k, b, p, st)) != cudaSuccess) return cuda_fail(c, e, "band kernel");
    if ((e = dk::launch_reduce(t.d_bpart, p.S, c->stride, sums_dev, st)) != cudaSuccess)
        return cuda_fail(c, e, "reduce kernel launch");
    return MLMC_DK_OK;
}

// The level's sample kernel: the theta-scheme kernel on a theta context, the
// register-resident kernel variant in use otherwise.
cudaError_t launch_main(const mlmc_dk_ctx* c, int level, bool coupled, const dk::KArgs& a, int n_ctas,
                        cudaStream_t st, int priority) {
    const LevelTab& t = c->lv[level];
    if (c->coupling == 1) {
        dk::FArgs fa{};
        fa.P1 = coupled ? t.d_P1 : nullptr;
        fa.phif64 = t.d_phi64;
        fa.phic64 = coupled ? c->lv[level - 1].d_phi64 : nullptr;
        if (dk::fourier_cluster_supported(t.n))
            return dk::launch_fourier_cluster(t.n, coupled, a, fa, n_ctas, st, priority);
        return dk::launch_fourier(t.n, coupled, a, fa, n_ctas, st, priority, c->fluct != 0);
    }
    if (c->theta) {
        dk::TArgs ta = c->targs;
        ta.Af64 = t.A64;
        ta.Ac64 = coupled ? c->lv[level - 1].A64 : 0;
        ta.phif64 = t.d_phi64;
        ta.phic64 = coupled ? c->lv[level - 1].d_phi64 : nullptr;
        return dk::launch_theta(t.n, coupled, a, ta, n_ctas, st, priority);
    }
    return dk::launch_level(t.n, coupled, t.sel[coupled ? 1 : 0], a, n_ctas, st, priority, c->fluct != 0);
}

int launch_batch_into(mlmc_dk_ctx* c, int level, int stream_tag, int64_t first, int64_t count, uint64_t seed,
                      double* sums_dev, double* samples_dev, cudaStream_t st, double* partials, size_t cap,
                      int priority) {
    const bool coupled = (stream_tag == 0) && level > 0;
    if (c->lv[level].vi(coupled).band)
        return launch_band(c, level, stream_tag, first, count, seed, sums_dev, samples_dev, st);
    if (c->lv[level].streamed)
        return launch_streamed(c, level, stream_tag, first, count, seed, sums_dev, samples_dev, st);
    const dk::VariantInfo& vi = c->lv[level].vi(coupled);
    if (!vi.supported)
        return fail(c, MLMC_DK_ERR_UNSUPPORTED, "no kernel variant for n = " + std::to_string(c->lv[level].n));
    cudaError_t e;
    if (count == 0) {
        e = cudaMemsetAsync(sums_dev, 0, sizeof(double) * c->stride, st);
        return e == cudaSuccess ? MLMC_DK_OK : cuda_fail(c, e, "cudaMemsetAsync");
    }
    const int64_t per_cluster = vi.slots_per_cta;            // slots per CTA (mode i) or per cluster
    const int64_t want_groups = (count + per_cluster - 1) / per_cluster;
    const int64_t max_groups = vi.max_ctas / vi.cluster;
    const int64_t groups = std::min(want_groups, max_groups);
    const int n_ctas = (int)(groups * vi.cluster);
    const int n_slots = (int)(groups * per_cluster);
    if ((size_t)n_slots * c->stride > cap) return fail(c, MLMC_DK_ERR_INVALID, "scratch too small");
    dk::KArgs a = make_args(c, level, stream_tag, coupled, first, count, seed, samples_dev);
    a.partials = partials;
    if ((e = launch_main(c, level, coupled, a, n_ctas, st, priority)) != cudaSuccess)
        return cuda_fail(c, e, "level kernel launch");
    if ((e = dk::launch_reduce(partials, n_slots, c->stride, sums_dev, st)) != cudaSuccess)
        return cuda_fail(c, e, "reduce kernel launch");
    return MLMC_DK_OK;
}

int check_device_error(mlmc_dk_ctx* c) {
    cudaError_t e = cudaMemcpyAsync(c->h_err, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "device error word");
    if (*c->h_err & dk::kErrTimeout) {
        cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->stream);
        return fail(c, MLMC_DK_ERR_TIMEOUT, "a bounded wait for another CTA's progress gave up");
    }
    if (*c->h_err & dk::kErrRange) {
        cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->stream);
        return fail(c, MLMC_DK_ERR_RANGE, "fixed-point range exceeded (|rho| too large for this level's scale)");
    }
    return MLMC_DK_OK;
}

void accumulate(const mlmc_dk_ctx* c, const double* s, mlmc_dk_level_sums* out, double cost_per, double wall,
                double kernel_s, int launches) {
    const int64_t n = (int64_t)std::llround(s[0]);
    for (int q = 0; q < c->n_quant; ++q) {
        const double* b = s + 2 + dk::kNSum * q;
        mlmc_dk_level_sums& o = out[q];
        o.n += n;
        o.dp1 += b[0]; o.dp2 += b[1]; o.dp3 += b[2]; o.dp4 += b[3];
        o.pf1 += b[4]; o.pf2 += b[5]; o.pc1 += b[6]; o.pc2 += b[7];
        o.yf1 += b[8]; o.yf2 += b[9]; o.yc1 += b[10]; o.yc2 += b[11];
        o.max_mass_err = std::max(o.max_mass_err, s[1]);
        o.cost += cost_per * (double)n;
        o.wall_s += wall;
        o.kernel_s += kernel_s;
        o.launches += launches;
        o.d2h_bytes += (int64_t)(sizeof(double) * c->stride + sizeof(unsigned));
    }
}

int run_host(mlmc_dk_ctx* c, int level, int stream_tag, int64_t n_samples, uint64_t seed, mlmc_dk_level_sums* sums) {
    if (!c) return fail(nullptr, MLMC_DK_ERR_INVALID, "null context");
    if (level < 0 || level > c->L_max) return fail(c, MLMC_DK_ERR_INVALID, "level out of range");
    if (n_samples < 0 || !sums) return fail(c, MLMC_DK_ERR_INVALID, "bad sample count or null sums");
    const auto t0 = std::chrono::steady_clock::now();
    int64_t& next = c->next_id[stream_tag][level];
    cudaError_t e = cudaEventRecord(c->ev0, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventRecord");
    int rc = launch_batch(c, level, stream_tag, next, n_samples, seed, c->d_sums, nullptr, c->stream);
    if (rc != MLMC_DK_OK) return rc;
    if ((e = cudaEventRecord(c->ev1, c->stream)) != cudaSuccess) return cuda_fail(c, e, "cudaEventRecord");
    e = cudaMemcpyAsync(c->h_sums, c->d_sums, sizeof(double) * c->stride, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "level batch");
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, c->ev0, c->ev1)) != cudaSuccess) return cuda_fail(c, e, "cudaEventElapsedTime");
    if ((rc = check_device_error(c)) != MLMC_DK_OK) return rc;
    next += n_samples;
    const double wall = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    const LevelTab& f = c->lv[level];
    double cost = (double)f.n * f.n * f.M;
    if (stream_tag == 0 && level > 0) cost += (double)c->lv[level - 1].n * c->lv[level - 1].n * c->lv[level - 1].M;
    accumulate(c, c->h_sums, sums, cost, wall, 1e-3 * ms, n_samples > 0 ? 2 : 0);
    return MLMC_DK_OK;
}

void release(mlmc_dk_ctx* c) {
    for (auto& l : c->lv) {
        cudaFree(l.d_q0);
        cudaFree(l.d_qbar);
        cudaFree(l.d_phi);
        cudaFree(l.d_phi64);
        cudaFree(l.d_P1);
        cudaFree(l.d_stream);
        cudaFree(l.d_spart);
        cudaFree(l.d_rbar);
        cudaFree(l.d_band);
        cudaFree(l.d_bpart);
    }
    cudaFree(c->d_partials);
    cudaFree(c->d_sums);
    cudaFree(c->d_err);
    if (c->h_sums) cudaFreeHost(c->h_sums);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    for (auto p : c->d_lpart) cudaFree(p);
    for (auto s : c->lstream) if (s) cudaStreamDestroy(s);
    for (auto ev : c->ev_join) if (ev) cudaEventDestroy(ev);
    for (auto ev : c->ev_lb) if (ev) cudaEventDestroy(ev);
    for (auto ev : c->ev_le) if (ev) cudaEventDestroy(ev);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->ev_sfork) cudaEventDestroy(c->ev_sfork);
    if (c->ev_sjoin) cudaEventDestroy(c->ev_sjoin);
    if (c->ev_graph) cudaEventDestroy(c->ev_graph);
    if (c->sstream) cudaStreamDestroy(c->sstream);
    cudaFree(c->d_ssums);
    cudaFree(c->d_bsums);
    if (c->h_bsums) cudaFreeHost(c->h_bsums);
    free_surrogate(c->sur);
    c->sur = nullptr;
}

}  // namespace

extern "C" {

const char* mlmc_dk_version(void) { return "mlmc_dk 0.1 (sm_103a)"; }

const char* mlmc_dk_last_error(const mlmc_dk_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

int32_t mlmc_dk_num_quantities(const mlmc_dk_ctx* ctx) { return ctx ? ctx->n_quant : 0; }

int mlmc_dk_chebyshev_schedule_host(double alpha, int32_t* K, float* c1, float* c2) {
    if (!K || !c1 || !c2 || !(alpha >= 0.0)) return fail(nullptr, MLMC_DK_ERR_INVALID, "chebyshev_schedule: bad arguments");
    int k = 0;
    if (!chebyshev_schedule(alpha, &k, c1, c2)) return fail(nullptr, MLMC_DK_ERR_UNSUPPORTED, "alpha too large");
    *K = k;
    return MLMC_DK_OK;
}

int mlmc_dk_fourier_restriction_host(int32_t n, float* P1) {
    if (!P1 || n < 6 || n % 6 != 0) return fail(nullptr, MLMC_DK_ERR_INVALID, "fourier_restriction: n must be a multiple of 6");
    fourier_restriction(n, P1);
    return MLMC_DK_OK;
}

int mlmc_dk_mean_field_host(int32_t n, double h, double tau, int64_t M, const double* rho0, double* out) {
    if (n < 2 || (n & 1) || h <= 0 || tau < 0 || M < 0 || !rho0 || !out)
        return fail(nullptr, MLMC_DK_ERR_INVALID, "mean_field_host: bad arguments");
    std::vector<double> tmp(rho0, rho0 + (size_t)n * n);
    mean_field_any(n, h, tau, M, tmp.data(), out);
    return MLMC_DK_OK;
}

int mlmc_dk_mean_field_theta_host(int32_t n, double h, double tau, int64_t M, double b0, const double* rho0,
                                  double* out) {
    if (!is_pow2(n) || n < 2 || h <= 0 || tau < 0 || M < 0 || !(b0 >= 0.0 && b0 <= 1.0) || !rho0 || !out)
        return fail(nullptr, MLMC_DK_ERR_INVALID, "mean_field_theta_host: bad arguments");
    std::vector<double> tmp(rho0, rho0 + (size_t)n * n);
    mean_field(n, h, tau, M, tmp.data(), out, b0);
    return MLMC_DK_OK;
}

int mlmc_dk_init(const mlmc_dk_config* cfg, mlmc_dk_ctx** out) {
    if (!out) return fail(nullptr, MLMC_DK_ERR_INVALID, "null output pointer");
    *out = nullptr;
    if (!cfg) return fail(nullptr, MLMC_DK_ERR_INVALID, "null config");
    const bool fourier = cfg->coupling == 1;
    if (cfg->coupling != 0 && !fourier) return fail(nullptr, MLMC_DK_ERR_INVALID, "coupling must be 0 (NN) or 1 (Fourier)");
    const int ratio = fourier ? 3 : 2;   // h_{l-1} = ratio h_l, tau_{l-1} = ratio^2 tau_l (Eq. cfl_preserved)
    if (cfg->L_max < 0 || cfg->L_max >= MLMC_DK_MAX_LEVELS)
        return fail(nullptr, MLMC_DK_ERR_INVALID, "L_max out of range");
    if (!fourier && (!is_pow2(cfg->n0) || cfg->n0 < 4 || ((long long)cfg->n0 << cfg->L_max) > 1024))
        return fail(nullptr, MLMC_DK_ERR_INVALID, "n0 must be a power of two >= 4 with n0 2^L_max <= 1024");
    if (fourier) {
        long long nl = cfg->n0;
        for (int l = 1; l <= cfg->L_max; ++l) nl *= 3;
        if (cfg->n0 != 6 || nl > 162)
            return fail(nullptr, MLMC_DK_ERR_UNSUPPORTED,
                        "Fourier coupling: levels 6^2, 18^2, 54^2, 162^2 (n0 = 6, L_max <= 3)");
        if (cfg->theta_b0 != 0.0 || cfg->theta_kernel || cfg->stream_from_n != 0)
            return fail(nullptr, MLMC_DK_ERR_UNSUPPORTED, "Fourier coupling: explicit scheme, no streamed levels");
    }
    if (!(cfg->length > 0) || !(cfg->T > 0) || !(cfg->N >= 0))
        return fail(nullptr, MLMC_DK_ERR_INVALID, "length, T must be > 0 and N >= 0");
    if (cfg->n_obs < 1 || cfg->n_obs > MLMC_DK_MAX_OBS || !cfg->rho0 || !cfg->phi)
        return fail(nullptr, MLMC_DK_ERR_INVALID, "n_obs must be 1..4 and rho0/phi non-null");
    const double h0 = cfg->length / cfg->n0;
    long long M0 = cfg->M0;
    if (M0 <= 0) {
        if (!(cfg->cfl_mu > 0)) return fail(nullptr, MLMC_DK_ERR_INVALID, "cfl_mu must be > 0 when M0 is not given");
        const double x = cfg->T / (cfg->cfl_mu * h0 * h0);
        M0 = (long long)std::ceil(x - 1e-9 * x);
    }
    const double tau0 = cfg->T / (double)M0;
    const double b0 = cfg->theta_b0, b1 = 1.0 - cfg->theta_b0;
    if (!(b0 >= 0.0 && b0 <= 1.0)) return fail(nullptr, MLMC_DK_ERR_INVALID, "theta_b0 must lie in [0, 1]");
    const bool theta = b0 > 0.0 || cfg->theta_kernel != 0;
    if (b0 == 0.0 && tau0 / (h0 * h0) > 0.5 + 1e-12)
        return fail(nullptr, MLMC_DK_ERR_INVALID,
                    "tau/h^2 > 1/2: the noise-free scheme violates the discrete maximum principle");
    // the checkerboard mode (lam = 4 tau/h^2) has factor (1 - b1 lam)/(1 + b0 lam) >= -1 iff
    // (b1 - b0) 2 tau/h^2 <= 1 (Assumption ass_stability)
    if (b0 > 0.0 && b1 > b0 && (b1 - b0) * 2.0 * tau0 / (h0 * h0) > 1.0 + 1e-12)
        return fail(nullptr, MLMC_DK_ERR_INVALID, "tau/h^2 above the theta-scheme's stability bound 1/(2 (b1 - b0))");
    dk::TArgs targs{};
    if (theta) {
        if ((cfg->n0 << cfg->L_max) > 128 || cfg->stream_from_n != 0)
            return fail(nullptr, MLMC_DK_ERR_UNSUPPORTED, "theta-scheme kernel: grids up to 128^2, no streamed levels");
        const double alpha = b0 * tau0 / (2.0 * h0 * h0);
        targs.alpha = (float)alpha;
        targs.inv_theta = (float)(1.0 / (1.0 + 4.0 * alpha));
        if (!chebyshev_schedule(alpha, &targs.K, targs.c1, targs.c2))
            return fail(nullptr, MLMC_DK_ERR_UNSUPPORTED, "b0 tau/h^2 too large for the solve's step budget");
    }
    {
        long long Mmax = M0;
        for (int l = 1; l <= cfg->L_max; ++l) Mmax *= ratio * ratio;
        if (Mmax > (1LL << 30)) return fail(nullptr, MLMC_DK_ERR_INVALID, "too many time steps");
    }

    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0)
        return fail(nullptr, MLMC_DK_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));

    mlmc_dk_ctx* c = new mlmc_dk_ctx();
    c->length = cfg->length;
    c->T = cfg->T;
    c->N = cfg->N;
    c->L_max = cfg->L_max;
    c->n_obs = cfg->n_obs;
    c->products = cfg->products ? 1 : 0;
    c->n_quant = quantities(c->n_obs, c->products);
    c->stride = 2 + dk::kNSum * c->n_quant;
    c->pilot = cfg->pilot > 1 ? cfg->pilot : 256;
    c->L_start = std::min(cfg->L_start > 0 ? cfg->L_start : 2, cfg->L_max);
    c->b0 = b0;
    c->theta = theta ? 1 : 0;
    c->coupling = fourier ? 1 : 0;
    c->targs = targs;
    c->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
    c->lv.resize(cfg->L_max + 1);
    c->next_id[0].assign(cfg->L_max + 1, 0);
    c->next_id[1].assign(cfg->L_max + 1, 0);

    // Fixed-point scales of every level and the choice of state.  An absolute
    // state q = rho 2^S needs 2^S (twice the initial range plus 12 standard
    // deviations of the per-cell fluctuation sqrt(rho/(N h^2))) below 2^29, so
    // |q| stays under the 2^30 range check with a factor 2 to spare.  A
    // fluctuation state q = (rho - rho-bar^m) 2^S, rho-bar the noise-free path
    // (the scheme is linear apart from sqrt([rho]^+), so q obeys the same
    // integer flux form and the noise alone moves it), needs only the 12
    // deviations: at large N (the paper's N = 2e9) that is many more bits, i.e.
    // finer resolution of every transfer and flux.
    std::vector<int> S_abs(cfg->L_max + 1), S_fl(cfg->L_max + 1);
    bool fl_ok = !theta && cfg->N > 0 && cfg->stream_from_n == 0;
    double table_bytes = 0.0;
    int min_gain = 1 << 20;
    for (int l = 0; l <= cfg->L_max; ++l) {
        const int n = cfg->n0 * (int)std::lround(std::pow((double)ratio, l));
        const double h = h0 / std::pow((double)ratio, l), tau = tau0 / std::pow((double)(ratio * ratio), l);
        const long long M = M0 * std::llround(std::pow((double)(ratio * ratio), l));
        const size_t cells = (size_t)n * n;
        const double* rho0 = cfg->rho0[l];
        if (!rho0) { mlmc_dk_free(c); return fail(nullptr, MLMC_DK_ERR_INVALID, "null rho0 level array"); }
        double rmax = 0;
        for (size_t i = 0; i < cells; ++i) {
            if (!std::isfinite(rho0[i])) { mlmc_dk_free(c); return fail(nullptr, MLMC_DK_ERR_INVALID, "non-finite rho0"); }
            rmax = std::max(rmax, std::fabs(rho0[i]));
        }
        const double noise_sd = cfg->N > 0 ? std::sqrt(std::max(rmax, 1e-3) / (cfg->N * h * h)) : 0.0;
        const double c_noise = cfg->N > 0 ? std::sqrt(tau) / (std::sqrt(cfg->N) * 2.0 * h * h) : 0.0;
        int S = 29 - (int)std::ceil(std::log2(std::max(2.0 * rmax + 12.0 * noise_sd, 1e-6)));
        S = std::max(16, std::min(40, S));
        // keep the noise multiplier g = c 2^(S/2) small enough that |G| stays far below 2^31
        while (S > 16 && c_noise * std::pow(2.0, 0.5 * S) > 2048.0) --S;
        if (rmax * std::ldexp(1.0, S) >= std::ldexp(1.0, 30)) {
            mlmc_dk_free(c);
            return fail(nullptr, MLMC_DK_ERR_INVALID, "|rho0| too large for the fixed-point range");
        }
        S_abs[l] = S;
        int F = 29 - (int)std::ceil(std::log2(std::max(12.0 * noise_sd, 1e-12)));
        F = std::max(16, std::min(40, F));
        // fluctuation transfers G = c 2^F sqrt(rho) z: |G| far below 2^31
        while (F > 16 && c_noise * std::ldexp(1.0, F) * std::sqrt(std::max(rmax, 1e-3)) > std::ldexp(1.0, 27)) --F;
        S_fl[l] = F;
        min_gain = std::min(min_gain, F - S);
        table_bytes += 4.0 * (double)cells * (double)M;
        // kernels built with the fluctuation state: the register kernels (NN) and
        // the one-CTA Fourier kernel
        if (fourier ? !dk::fourier_supported(n) : dk::variant_count(n, true) == 0) fl_ok = false;
    }
    fl_ok = fl_ok && table_bytes <= 512.0 * (1 << 20);
    if (cfg->state_repr == 2 && !fl_ok) {
        mlmc_dk_free(c);
        return fail(nullptr, MLMC_DK_ERR_UNSUPPORTED,
                    "fluctuation state: explicit scheme with N > 0, grids up to 128^2 (NN) or 54^2 (Fourier), "
                    "mean-field tables <= 512 MB");
    }
    if (cfg->state_repr < 0 || cfg->state_repr > 2) {
        mlmc_dk_free(c);
        return fail(nullptr, MLMC_DK_ERR_INVALID, "state_repr must be 0 (automatic), 1 (absolute) or 2 (fluctuation)");
    }
    c->fluct = (cfg->state_repr == 2 || (cfg->state_repr == 0 && fl_ok && min_gain >= 3)) ? 1 : 0;

    size_t partials_need = 0;
    for (int l = 0; l <= cfg->L_max; ++l) {
        LevelTab& t = c->lv[l];
        t.n = cfg->n0 * (int)std::lround(std::pow((double)ratio, l));
        t.h = h0 / std::pow((double)ratio, l);
        t.tau = tau0 / std::pow((double)(ratio * ratio), l);
        t.M = (int)(M0 * std::llround(std::pow((double)(ratio * ratio), l)));
        const size_t cells = (size_t)t.n * t.n;
        const double* rho0 = cfg->rho0[l];
        const double c_noise = cfg->N > 0 ? std::sqrt(t.tau) / (std::sqrt(cfg->N) * 2.0 * t.h * t.h) : 0.0;
        const int S = c->fluct ? S_fl[l] : S_abs[l];
        t.S = S;
        t.A64 = std::llround(t.tau / (2.0 * t.h * t.h) * 4294967296.0);
        t.A = t.A64 < (1LL << 31) ? (int32_t)t.A64 : 0;
        // absolute state: G = rint(c 2^S sqrt(q 2^-S) z) = rint(c 2^(S/2) sqrt(q) z);
        // fluctuation state: G = rint(c 2^S sqrt(rho-bar + q 2^-S) z)
        t.g = (float)(c_noise * (c->fluct ? std::ldexp(1.0, S) : std::pow(2.0, 0.5 * S)));
        t.dscale = t.h * t.h * std::ldexp(1.0, -S);

        std::vector<int32_t> q0(cells), qb(cells);
        std::vector<double> rbar(cells);
        long long mass = 0;
        double mass_bar = 0.0;
        for (size_t i = 0; i < cells; ++i) {
            q0[i] = c->fluct ? 0 : (int32_t)std::llrint(std::ldexp(rho0[i], S));
            mass += q0[i];
            mass_bar += rho0[i];
        }
        t.mass0 = mass;
        t.mass_bar = c->fluct ? t.h * t.h * mass_bar : 0.0;
        mean_field_any(t.n, t.h, t.tau, t.M, rho0, rbar.data(), b0);
        for (size_t i = 0; i < cells; ++i) qb[i] = c->fluct ? 0 : (int32_t)std::llrint(std::ldexp(rbar[i], S));
        if (c->fluct) {
            // the noise-free path rho-bar^m, m = 0 .. M-1, by the explicit step in
            // FP64, stored in FP32 for the transfers' amplitudes
            std::vector<float> tab(cells * (size_t)t.M);
            std::vector<double> cur(rho0, rho0 + cells), nxt(cells);
            const double a = t.tau / (2.0 * t.h * t.h);
            const int n = t.n;
            for (int m = 0; m < t.M; ++m) {
                for (size_t i = 0; i < cells; ++i) tab[(size_t)m * cells + i] = (float)cur[i];
                for (int i1 = 0; i1 < n; ++i1)
                    for (int i2 = 0; i2 < n; ++i2) {
                        const double x = cur[(size_t)i1 * n + i2];
                        const double nb = cur[(size_t)((i1 + 1) % n) * n + i2] + cur[(size_t)((i1 + n - 1) % n) * n + i2] +
                                          cur[(size_t)i1 * n + (i2 + 1) % n] + cur[(size_t)i1 * n + (i2 + n - 1) % n];
                        nxt[(size_t)i1 * n + i2] = x + a * (nb - 4.0 * x);
                    }
                cur.swap(nxt);
            }
            if ((e = cudaMalloc(&t.d_rbar, sizeof(float) * tab.size())) != cudaSuccess ||
                (e = cudaMemcpy(t.d_rbar, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
                mlmc_dk_free(c);
                return cuda_fail(nullptr, e, "noise-free path tables");
            }
            c->h2d_bytes += (int64_t)(sizeof(float) * tab.size());
        }
        // The quantised initial state q0 2^-S differs from rho0 by e0 (at most half
        // a quantum per cell); the scheme is linear apart from sqrt([rho]^+), so e0
        // reaches T as the noise-free evolution of e0 (exact, FP64 by FFT) and is
        // removed from the observables with the mean-field offset below.
        std::vector<double> e0(cells, 0.0), e0T(cells, 0.0);
        if (!c->fluct) {
            for (size_t i = 0; i < cells; ++i) e0[i] = std::ldexp((double)q0[i], -S) - rho0[i];
            mean_field_any(t.n, t.h, t.tau, t.M, e0.data(), e0T.data(), b0);
        }
        std::vector<float> phif(cells * c->n_obs);
        for (int k = 0; k < c->n_obs; ++k) {
            const double* ph = cfg->phi[(size_t)l * c->n_obs + k];
            if (!ph) { mlmc_dk_free(c); return fail(nullptr, MLMC_DK_ERR_INVALID, "null phi level array"); }
            double yb = 0, dl = 0;
            for (size_t i = 0; i < cells; ++i) {
                yb += rbar[i] * ph[i];
                if (!c->fluct) dl += (std::ldexp((double)qb[i], -S) - rbar[i] - e0T[i]) * ph[i];
                phif[(size_t)k * cells + i] = (float)ph[i];
            }
            t.ybar[k] = t.h * t.h * yb;
            t.delta[k] = t.h * t.h * dl;
        }
        // stage the level's tables in pinned memory and copy them in one transfer each
        const size_t bytes = sizeof(int32_t) * cells * 2 + sizeof(float) * cells * c->n_obs;
        unsigned char* stage = nullptr;
        if ((e = cudaMallocHost(&stage, bytes)) != cudaSuccess) {
            mlmc_dk_free(c);
            return cuda_fail(nullptr, e, "pinned staging");
        }
        std::memcpy(stage, q0.data(), sizeof(int32_t) * cells);
        std::memcpy(stage + sizeof(int32_t) * cells, qb.data(), sizeof(int32_t) * cells);
        std::memcpy(stage + sizeof(int32_t) * cells * 2, phif.data(), sizeof(float) * cells * c->n_obs);
        if ((e = cudaMalloc(&t.d_q0, sizeof(int32_t) * cells)) != cudaSuccess ||
            (e = cudaMalloc(&t.d_qbar, sizeof(int32_t) * cells)) != cudaSuccess ||
            (e = cudaMalloc(&t.d_phi, sizeof(float) * cells * c->n_obs)) != cudaSuccess ||
            (e = cudaMemcpyAsync(t.d_q0, stage, sizeof(int32_t) * cells, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(t.d_qbar, stage + sizeof(int32_t) * cells, sizeof(int32_t) * cells,
                                 cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(t.d_phi, stage + sizeof(int32_t) * cells * 2, sizeof(float) * cells * c->n_obs,
                                 cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(c->stream)) != cudaSuccess) {
            cudaFreeHost(stage);
            mlmc_dk_free(c);
            return cuda_fail(nullptr, e, "level tables");
        }
        cudaFreeHost(stage);
        c->h2d_bytes += (int64_t)bytes;
        {
            // FP64 test functions for the streamed kernels' observables: there the
            // fluctuation is projected on phi cell by cell at up to 1024^2, where FP32
            // phi (relative rounding 2^-25 per value, uncorrelated with the noise)
            // would reach 1e-5 of the projection
            std::vector<double> ph64(cells * c->n_obs);
            for (int k = 0; k < c->n_obs; ++k)
                std::memcpy(ph64.data() + (size_t)k * cells, cfg->phi[(size_t)l * c->n_obs + k], sizeof(double) * cells);
            if ((e = cudaMalloc(&t.d_phi64, sizeof(double) * ph64.size())) != cudaSuccess ||
                (e = cudaMemcpy(t.d_phi64, ph64.data(), sizeof(double) * ph64.size(), cudaMemcpyHostToDevice)) !=
                    cudaSuccess) {
                mlmc_dk_free(c);
                return cuda_fail(nullptr, e, "FP64 test functions");
            }
            c->h2d_bytes += (int64_t)(sizeof(double) * ph64.size());
        }
        if (fourier) {
            // one kernel shape per grid size: the Fourier-coupled kernel, and the
            // restriction of this level's normals to the coarse grid
            if (l > 0) {
                std::vector<float> P1((size_t)(t.n / 3) * t.n);
                fourier_restriction(t.n, P1.data());
                if ((e = cudaMalloc(&t.d_P1, sizeof(float) * P1.size())) != cudaSuccess ||
                    (e = cudaMemcpy(t.d_P1, P1.data(), sizeof(float) * P1.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
                    mlmc_dk_free(c);
                    return cuda_fail(nullptr, e, "Fourier restriction");
                }
                c->h2d_bytes += (int64_t)(sizeof(float) * P1.size());
            }
            for (int mode = 0; mode < 2; ++mode) {
                if (mode == 1 && l == 0) continue;
                dk::VariantInfo vi{};
                e = dk::fourier_cluster_supported(t.n) ? dk::fourier_cluster_variant_info(t.n, mode == 1, c->stride, &vi)
                                                       : dk::fourier_variant_info(t.n, mode == 1, c->stride, &vi,
                                                                                  c->fluct != 0);
                if (e != cudaSuccess) {
                    mlmc_dk_free(c);
                    return cuda_fail(nullptr, e, "Fourier kernel setup");
                }
                if (!vi.supported) {
                    mlmc_dk_free(c);
                    return fail(nullptr, MLMC_DK_ERR_UNSUPPORTED, "no Fourier-coupled kernel for this grid");
                }
                t.vis[mode].push_back(vi);
                partials_need = std::max(partials_need, (size_t)vi.max_ctas * vi.slots_per_cta * c->stride);
            }
            continue;
        }
        if (theta) {
            // one kernel shape per grid size: the theta-scheme kernel
            for (int mode = 0; mode < 2; ++mode) {
                if (mode == 1 && l == 0) continue;
                dk::VariantInfo vi{};
                if ((e = dk::theta_variant_info(t.n, mode == 1, c->stride, &vi)) != cudaSuccess) {
                    mlmc_dk_free(c);
                    return cuda_fail(nullptr, e, "theta kernel setup");
                }
                if (!vi.supported) {
                    mlmc_dk_free(c);
                    return fail(nullptr, MLMC_DK_ERR_UNSUPPORTED, "no theta-scheme kernel for this grid");
                }
                t.vis[mode].push_back(vi);
                partials_need = std::max(partials_need, (size_t)vi.max_ctas * vi.slots_per_cta * c->stride);
            }
            continue;
        }
        const bool force_stream = cfg->stream_from_n > 0 && t.n >= cfg->stream_from_n && t.n % 64 == 0;
        const int nv = force_stream ? 0 : dk::variant_count(t.n, c->fluct != 0);
        if (nv == 0) {
            // no register-resident variant: stream the state through global memory,
            // samples in flight within a 96 MB working set (L2-resident)
            if (t.n % 64 != 0) {
                mlmc_dk_free(c);
                return fail(nullptr, MLMC_DK_ERR_UNSUPPORTED, "grid size without a kernel");
            }
            t.streamed = 1;
            for (int v = 0; v < dk::stream_variant_count(); ++v) {
                t.inflight_v[v] = dk::stream_inflight(t.n, (size_t)96 << 20, v);
                t.inflight = std::max(t.inflight, t.inflight_v[v]);
            }
            for (int mode = 0; mode < 2; ++mode) {
                if (mode == 1 && l == 0) continue;
                for (int v = 0; v < dk::stream_variant_count(); ++v) {
                    dk::VariantInfo vi{};
                    if ((e = dk::stream_variant_info(t.n, v, &vi)) != cudaSuccess) {
                        mlmc_dk_free(c);
                        return cuda_fail(nullptr, e, "streamed kernel variant setup");
                    }
                    t.vis[mode].push_back(vi);
                }
            }
            t.sel[0] = t.sel[1] = dk::stream_default_variant();
            if ((e = cudaMalloc(&t.d_stream, dk::stream_bytes(t.n, t.inflight))) != cudaSuccess ||
                (e = cudaMalloc(&t.d_spart, sizeof(double) * c->stride * t.inflight)) != cudaSuccess) {
                mlmc_dk_free(c);
                return cuda_fail(nullptr, e, "streamed level buffers");
            }
        }
        for (int mode = 0; mode < 2; ++mode) {
            if (mode == 1 && l == 0) continue;
            for (int v = 0; v < nv; ++v) {
                dk::VariantInfo vi{};
                if ((e = dk::variant_info(t.n, mode == 1, c->stride, v, &vi, c->fluct != 0)) != cudaSuccess) {
                    mlmc_dk_free(c);
                    return cuda_fail(nullptr, e, "kernel variant setup");
                }
                t.vis[mode].push_back(vi);
                if (vi.supported)
                    partials_need = std::max(partials_need, (size_t)(vi.max_ctas / vi.cluster) * vi.slots_per_cta * c->stride);
            }
        }
        if (!c->fluct && !force_stream && (dk::band_supported(t.n, 4) || dk::band_supported(t.n, 8))) {
            // band kernels (4 x 4 and 4 x 8 thread blocks): a sample over several
            // CTAs; candidates for the tuner (the first variant stays the default)
            size_t bytes = 0;
            int S_max = 0;
            for (int mode = 0; mode < 2; ++mode) {
                if (mode == 1 && l == 0) continue;
                for (int k = 0; k < 2; ++k) {
                    if ((e = dk::band_plan(t.n, mode == 1, k == 0 ? 4 : 8, &t.bplan[mode][k])) != cudaSuccess) {
                        mlmc_dk_free(c);
                        return cuda_fail(nullptr, e, "band kernel setup");
                    }
                    if (!t.bplan[mode][k].supported) continue;
                    bytes = std::max(bytes, dk::band_bytes(t.n, t.bplan[mode][k]));
                    S_max = std::max(S_max, t.bplan[mode][k].S);
                }
            }
            if (bytes > 0) {
                if ((e = cudaMalloc(&t.d_band, bytes)) != cudaSuccess ||
                    (e = cudaMalloc(&t.d_bpart, sizeof(double) * c->stride * S_max)) != cudaSuccess) {
                    mlmc_dk_free(c);
                    return cuda_fail(nullptr, e, "band kernel buffers");
                }
                for (int mode = 0; mode < 2; ++mode) {
                    if (mode == 1 && l == 0) continue;
                    for (int k = 1; k >= 0; --k) {   // 4 x 8 blocks, then 4 x 4
                        const dk::BandPlan& p = t.bplan[mode][k];
                        if (!p.supported) continue;
                        dk::VariantInfo vi{};
                        vi.supported = 1;
                        vi.band = p.fc;
                        vi.bands = p.nb;
                        vi.threads = p.threads;
                        vi.cluster = 1;
                        vi.slots_per_cta = 0;
                        vi.smem = p.smem;
                        vi.max_ctas = p.S * p.nb;
                        vi.C = p.fc / 2;
                        vi.R = 2;
                        t.vis[mode].push_back(vi);
                    }

                }
            }
        }
        if (!t.streamed && !c->fluct && t.n >= 256 && t.n % 64 == 0) {
            // register level with 8-SM clusters: streamed buffers for a batch split
            const int dv = dk::stream_default_variant();
            t.inflight_v[dv] = dk::stream_inflight(t.n, (size_t)96 << 20, dv);
            t.inflight = t.inflight_v[dv];
            if ((e = cudaMalloc(&t.d_stream, dk::stream_bytes(t.n, t.inflight))) != cudaSuccess ||
                (e = cudaMalloc(&t.d_spart, sizeof(double) * c->stride * t.inflight)) != cudaSuccess) {
                mlmc_dk_free(c);
                return cuda_fail(nullptr, e, "batch split buffers");
            }
            t.split_ok = 1;
        }
    }
    if ((e = cudaMalloc(&c->d_partials, sizeof(double) * std::max<size_t>(partials_need, 1))) != cudaSuccess ||
        (e = cudaMalloc(&c->d_sums, sizeof(double) * c->stride)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_err, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMemset(c->d_err, 0, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMallocHost(&c->h_sums, sizeof(double) * c->stride)) != cudaSuccess ||
        (e = cudaMallocHost(&c->h_err, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaEventCreate(&c->ev0)) != cudaSuccess || (e = cudaEventCreate(&c->ev1)) != cudaSuccess) {
        mlmc_dk_free(c);
        return cuda_fail(nullptr, e, "context buffers");
    }
    c->partials_cap = partials_need;
    // per-level streams (finest level most urgent), scratch and events of the multi-level batch
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    const int nl = cfg->L_max + 1;
    c->lstream.assign(nl, nullptr);
    c->d_lpart.assign(nl, nullptr);
    c->lpart_cap.assign(nl, 0);
    c->lprio.assign(nl, 0);
    c->ev_join.assign(nl, nullptr);
    c->ev_lb.assign(nl, nullptr);
    c->ev_le.assign(nl, nullptr);
    for (int l = 0; l < nl; ++l) {
        const LevelTab& t = c->lv[l];
        size_t need = 0;
        for (int mode = 0; mode < 2; ++mode)
            for (const auto& vi : t.vis[mode])
                if (vi.supported) need = std::max(need, (size_t)(vi.max_ctas / vi.cluster) * vi.slots_per_cta * c->stride);
        c->lpart_cap[l] = need;
        // the finest level gets the most urgent priority, coarser levels fill in;
        // the streamed levels (which run side by side after the graph) share the
        // finest one's, so that the block scheduler interleaves their launches
        int rank_l = l;
        if (t.streamed) rank_l = nl - 1;
        c->lprio[l] = std::max(prio_hi, prio_lo - (rank_l * (prio_lo - prio_hi)) / std::max(1, nl - 1));
        if ((e = cudaMalloc(&c->d_lpart[l], sizeof(double) * std::max<size_t>(need, 1))) != cudaSuccess ||
            (e = cudaStreamCreateWithPriority(&c->lstream[l], cudaStreamNonBlocking, c->lprio[l])) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&c->ev_join[l], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreate(&c->ev_lb[l])) != cudaSuccess || (e = cudaEventCreate(&c->ev_le[l])) != cudaSuccess) {
            mlmc_dk_free(c);
            return cuda_fail(nullptr, e, "batch streams");
        }
    }
    if ((e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaStreamCreateWithPriority(&c->sstream, cudaStreamNonBlocking, prio_lo)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev_sfork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev_sjoin, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev_graph, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_ssums, sizeof(double) * c->stride * nl)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_bsums, sizeof(double) * c->stride * nl)) != cudaSuccess ||
        (e = cudaMallocHost(&c->h_bsums, sizeof(double) * c->stride * nl)) != cudaSuccess) {
        mlmc_dk_free(c);
        return cuda_fail(nullptr, e, "batch graph resources");
    }
    *out = c;
    return MLMC_DK_OK;
}

void mlmc_dk_free(mlmc_dk_ctx* ctx) {
    if (!ctx) return;
    release(ctx);
    delete ctx;
}

int mlmc_dk_level_info(const mlmc_dk_ctx* ctx, int32_t level, mlmc_dk_level_desc* out) {
    if (!ctx || !out || level < 0 || level > ctx->L_max)
        return fail(const_cast<mlmc_dk_ctx*>(ctx), MLMC_DK_ERR_INVALID, "level_info: bad arguments");
    const LevelTab& t = ctx->lv[level];
    *out = mlmc_dk_level_desc{};
    out->level = level;
    out->n = t.n;
    out->M = t.M;
    out->h = t.h;
    out->tau = t.tau;
    for (int k = 0; k < ctx->n_obs; ++k) {
        out->ybar_f[k] = t.ybar[k];
        out->ybar_c[k] = level > 0 ? ctx->lv[level - 1].ybar[k] : 0.0;
    }
    out->cost_mc = (double)t.n * t.n * t.M;
    out->cost = out->cost_mc + (level > 0 ? (double)ctx->lv[level - 1].n * ctx->lv[level - 1].n * ctx->lv[level - 1].M : 0.0);
    out->next_sample = ctx->next_id[0][level];
    out->h2d_bytes = ctx->h2d_bytes;
    out->frac_bits = t.S;
    out->n_variants = (int32_t)t.vis[0].size();
    out->variant_single = t.sel[0];
    out->variant_coupled = t.sel[1];
    const dk::VariantInfo& vs = t.vi(level > 0);
    out->lane_cols = vs.C;
    out->lane_rows = vs.R;
    out->cluster = vs.cluster;
    out->streamed = t.streamed;
    out->in_flight = t.streamed ? t.inflight_v[t.sel[level > 0 ? 1 : 0]]
                                : (t.split_ok ? t.inflight_v[dk::stream_default_variant()] : 0);
    out->tile_rows = vs.tile_rows;
    out->split_capable = t.split_ok;
    out->split_fraction = t.split_frac;
    out->batch_streamed = t.batch_streamed;
    out->theta = ctx->theta;
    out->theta_b0 = ctx->b0;
    out->cheb_steps = ctx->theta ? ctx->targs.K : 0;
    out->coupling = ctx->coupling;
    out->fluct = ctx->fluct;
    out->band = vs.band ? 1 : 0;
    out->bands = vs.bands;
    out->persistent = vs.persistent;
    out->pdl = vs.pdl;
    if (vs.band) out->in_flight = t.bplan[level > 0 ? 1 : 0][vs.band == 4 ? 0 : 1].S;
    return MLMC_DK_OK;
}

int mlmc_dk_run_level(mlmc_dk_ctx* ctx, int32_t level, int64_t n_samples, uint64_t seed, mlmc_dk_level_sums* sums) {
    return run_host(ctx, level, 0, n_samples, seed, sums);
}

int mlmc_dk_run_mc(mlmc_dk_ctx* ctx, int32_t level, int64_t n_samples, uint64_t seed, mlmc_dk_level_sums* sums) {
    return run_host(ctx, level, 1, n_samples, seed, sums);
}

int mlmc_dk_run_level_dev(mlmc_dk_ctx* ctx, int32_t level, int32_t stream_tag, int64_t first_sample,
                          int64_t n_samples, uint64_t seed, double* sums_dev, double* samples_dev,
                          void* cuda_stream) {
    if (!ctx) return fail(nullptr, MLMC_DK_ERR_INVALID, "null context");
    if (level < 0 || level > ctx->L_max || (stream_tag != 0 && stream_tag != 1) || first_sample < 0 ||
        n_samples < 0 || !sums_dev || ((uintptr_t)sums_dev & 7) || ((uintptr_t)samples_dev & 7))
        return fail(ctx, MLMC_DK_ERR_INVALID, "run_level_dev: bad arguments");
    cudaStream_t st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->stream;
    return launch_batch(ctx, level, stream_tag, first_sample, n_samples, seed, sums_dev, samples_dev, st);
}

int mlmc_dk_run_level_static(const mlmc_dk_ctx* ctx, int32_t level, int32_t stream_tag, int64_t first_sample,
                             int64_t n_samples, uint64_t seed, double* sums_dev, double* samples_dev,
                             unsigned int* err_dev, void* cuda_stream) {
    mlmc_dk_ctx* c = const_cast<mlmc_dk_ctx*>(ctx);   // only the error message is written
    if (!ctx) return fail(nullptr, MLMC_DK_ERR_INVALID, "null context");
    if (level < 0 || level > ctx->L_max || (stream_tag != 0 && stream_tag != 1) || first_sample < 0 ||
        n_samples < 0 || !sums_dev || ((uintptr_t)sums_dev & 7) || ((uintptr_t)samples_dev & 7) ||
        ((uintptr_t)err_dev & 3))
        return fail(c, MLMC_DK_ERR_INVALID, "run_level_static: bad arguments");
    const bool coupled = (stream_tag == 0) && level > 0;
    const dk::VariantInfo& vi = ctx->lv[level].vi(coupled);
    if (!vi.supported || ctx->lv[level].streamed || vi.band)
        return fail(c, MLMC_DK_ERR_UNSUPPORTED, "no register-resident kernel for n = " + std::to_string(ctx->lv[level].n));
    cudaStream_t st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->stream;
    cudaError_t e;
    if (n_samples == 0) {
        e = cudaMemsetAsync(sums_dev, 0, sizeof(double) * ctx->stride, st);
        return e == cudaSuccess ? MLMC_DK_OK : cuda_fail(c, e, "cudaMemsetAsync");
    }
    double* scratch = nullptr;
    size_t capacity = 0;
    if ((e = dk::static_scratch(&scratch, &capacity)) != cudaSuccess)
        return cuda_fail(c, e, "static scratch set-up (cudaGetSymbolAddress)");
    // As many sample slots as fit the static array: fewer resident slots than
    // mlmc_dk_run_level_dev may use, the same per-sample arithmetic.
    const int64_t per_group = vi.slots_per_cta;
    const size_t usable = capacity - 32;   // the last 32 doubles hold the fallback error word
    const int64_t fit_groups = (int64_t)(usable / ((size_t)ctx->stride * per_group));
    if (fit_groups < 1)
        return fail(c, MLMC_DK_ERR_INVALID, "run_level_static: one CTA's partial sums (" +
                    std::to_string(per_group * ctx->stride) + " doubles) exceed the static scratch of " +
                    std::to_string(usable) + " doubles");
    const int64_t groups = std::min({(n_samples + per_group - 1) / per_group, (int64_t)(vi.max_ctas / vi.cluster),
                                     fit_groups});
    const int n_ctas = (int)(groups * vi.cluster);
    const int n_slots = (int)(groups * per_group);
    dk::KArgs a = make_args(c, level, stream_tag, coupled, first_sample, n_samples, seed, samples_dev);
    a.partials = scratch;        // fully overwritten by the level kernel: nothing to clear
    a.err = err_dev ? err_dev : reinterpret_cast<unsigned*>(scratch + (capacity - 1));
    if ((e = launch_main(ctx, level, coupled, a, n_ctas, st, 0)) != cudaSuccess)
        return cuda_fail(c, e, "level kernel launch");
    if ((e = dk::launch_reduce(scratch, n_slots, ctx->stride, sums_dev, st)) != cudaSuccess)
        return cuda_fail(c, e, "reduce kernel launch");
    return MLMC_DK_OK;
}

int mlmc_dk_band_wait_test(mlmc_dk_ctx* ctx, int32_t level, uint32_t polls, int32_t stall_band) {
    if (!ctx) return fail(nullptr, MLMC_DK_ERR_INVALID, "null context");
    if (level < 1 || level > ctx->L_max || polls == 0 || stall_band < 0)
        return fail(ctx, MLMC_DK_ERR_INVALID, "band_wait_test: bad arguments");
    LevelTab& t = ctx->lv[level];
    const dk::VariantInfo& vi = t.vi(true);
    if (!vi.band || !t.d_band || stall_band >= t.bplan[1][vi.band == 4 ? 0 : 1].nb)
        return fail(ctx, MLMC_DK_ERR_UNSUPPORTED, "band_wait_test: the level's coupled kernel is not a band kernel");
    const int rc = launch_band(ctx, level, 0, 0, 1, 0x7465, ctx->d_sums, nullptr, ctx->stream, std::min(t.M, 64),
                               polls, stall_band);
    if (rc != MLMC_DK_OK) return rc;
    const cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "band_wait_test");
    return check_device_error(ctx);
}

int mlmc_dk_stream_wait_test(mlmc_dk_ctx* ctx, int32_t level, uint32_t polls, int32_t stall_tile) {
    if (!ctx) return fail(nullptr, MLMC_DK_ERR_INVALID, "null context");
    if (level < 0 || level > ctx->L_max || polls == 0 || stall_tile < 0)
        return fail(ctx, MLMC_DK_ERR_INVALID, "stream_wait_test: bad arguments");
    LevelTab& t = ctx->lv[level];
    if (!t.streamed) return fail(ctx, MLMC_DK_ERR_UNSUPPORTED, "stream_wait_test: the level is not streamed");
    int variant = -1;
    for (int v = 0; v < (int)t.vis[level > 0 ? 1 : 0].size(); ++v)
        if (t.vis[level > 0 ? 1 : 0][v].persistent && t.vis[level > 0 ? 1 : 0][v].supported) variant = v;
    const dk::VariantInfo* vi = variant >= 0 ? &t.vis[level > 0 ? 1 : 0][variant] : nullptr;
    if (!vi || stall_tile >= (t.n / vi->tile_rows) * (t.n / 64))
        return fail(ctx, MLMC_DK_ERR_UNSUPPORTED, "stream_wait_test: no persistent streamed kernel or no such tile");
    const int rc = launch_streamed(ctx, level, 0, 0, 1, 0x7465, ctx->d_sums, nullptr, ctx->stream, std::min(t.M, 64),
                                   variant, polls, stall_tile);
    if (rc != MLMC_DK_OK) return rc;
    const cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream_wait_test");
    return check_device_error(ctx);
}

}  // extern "C"

namespace {

// The multi-level batch with sample ids firsts[l].. on level l (the public
// entry points check the arguments).
int batch_dev(mlmc_dk_ctx* ctx, const int64_t* counts, const int64_t* firsts, uint64_t seed, double* sums_dev,
              cudaStream_t st) {
    const int nl = ctx->L_max + 1;
    cudaError_t e;
    // split: the last n_split[l] ids of a split level run streamed beside the graph
    std::vector<int64_t> n_split(nl, 0), n_reg(counts, counts + nl);
    bool any_split = false;
    // levels whose kernel runs many launches (streamed state) or a cooperative
    // grid (band kernel) run beside the graph, not inside it
    auto outside = [&](int l) { return ctx->lv[l].streamed || ctx->lv[l].vi(l > 0).band; };
    for (int l = 0; l < nl; ++l) {
        LevelTab& t = ctx->lv[l];
        t.batch_streamed = 0;
        if (t.split_ok && t.split_frac > 0 && l > 0 && counts[l] > 1 && !outside(l)) {
            n_split[l] = std::min<int64_t>(counts[l] - 1, (int64_t)std::floor(t.split_frac * (double)counts[l]));
            n_reg[l] = counts[l] - n_split[l];
            t.batch_streamed = n_split[l];
            any_split = any_split || n_split[l] > 0;
        }
    }
    if ((e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaStreamBeginCapture");
    int rc = MLMC_DK_OK;
    e = cudaEventRecord(ctx->ev_fork, ctx->cap_stream);
    // finest level first: its clusters are placed before the coarser levels fill the remaining SMs
    for (int l = nl - 1; l >= 0 && e == cudaSuccess && rc == MLMC_DK_OK; --l) {
        if (outside(l)) continue;
        double* out = sums_dev + (size_t)l * ctx->stride;
        if ((e = cudaStreamWaitEvent(ctx->lstream[l], ctx->ev_fork, 0)) != cudaSuccess) break;
        // external records become event-record nodes of the graph (timing)
        if ((e = cudaEventRecordWithFlags(ctx->ev_lb[l], ctx->lstream[l], cudaEventRecordExternal)) != cudaSuccess)
            break;
        rc = launch_batch_into(ctx, l, 0, firsts[l], n_reg[l], seed, out, nullptr, ctx->lstream[l],
                               ctx->d_lpart[l], ctx->lpart_cap[l], ctx->lprio[l]);
        if (rc != MLMC_DK_OK) break;
        if ((e = cudaEventRecordWithFlags(ctx->ev_le[l], ctx->lstream[l], cudaEventRecordExternal)) != cudaSuccess)
            break;
        if ((e = cudaEventRecord(ctx->ev_join[l], ctx->lstream[l])) != cudaSuccess) break;
        e = cudaStreamWaitEvent(ctx->cap_stream, ctx->ev_join[l], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (rc != MLMC_DK_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess || ec != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(ctx, e != cudaSuccess ? e : ec, "batch capture");
    }
    // reuse the instantiated graph when only parameters changed
    bool updated = false;
    if (ctx->gexec) {
        cudaGraphExecUpdateResultInfo info;
        updated = cudaGraphExecUpdate(ctx->gexec, graph, &info) == cudaSuccess;
        if (!updated) {
            cudaGetLastError();
            cudaGraphExecDestroy(ctx->gexec);
            ctx->gexec = nullptr;
        }
    }
    if (!updated && (e = cudaGraphInstantiate(&ctx->gexec, graph, 0)) != cudaSuccess) {
        cudaGraphDestroy(graph);
        ctx->gexec = nullptr;
        return cuda_fail(ctx, e, "cudaGraphInstantiate");
    }
    cudaGraphDestroy(graph);
    if (any_split) {
        if ((e = cudaEventRecord(ctx->ev_sfork, st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(ctx->sstream, ctx->ev_sfork, 0)) != cudaSuccess)
            return cuda_fail(ctx, e, "batch split fork");
    }
    // band-kernel levels first, each on its level's stream: their cooperative
    // grids are placed before the graph's kernels fill the remaining SMs
    bool any_band = false, any_outside = false;
    auto band_level = [&](int l) { return ctx->lv[l].vi(l > 0).band != 0; };
    for (int l = 0; l < nl; ++l) any_outside = any_outside || outside(l);
    if (any_outside && (e = cudaEventRecord(ctx->ev_fork, st)) != cudaSuccess) return cuda_fail(ctx, e, "level fork");
    for (int l = nl - 1; l >= 0; --l) {
        if (!band_level(l)) continue;
        any_band = true;
        if ((e = cudaStreamWaitEvent(ctx->lstream[l], ctx->ev_fork, 0)) != cudaSuccess ||
            (e = cudaEventRecord(ctx->ev_lb[l], ctx->lstream[l])) != cudaSuccess)
            return cuda_fail(ctx, e, "band fork");
        rc = launch_batch_into(ctx, l, 0, firsts[l], counts[l], seed, sums_dev + (size_t)l * ctx->stride, nullptr,
                               ctx->lstream[l], nullptr, 0, 0);
        if (rc != MLMC_DK_OK) return rc;
        if ((e = cudaEventRecord(ctx->ev_le[l], ctx->lstream[l])) != cudaSuccess ||
            (e = cudaEventRecord(ctx->ev_join[l], ctx->lstream[l])) != cudaSuccess)
            return cuda_fail(ctx, e, "band join");
    }
    if ((e = cudaGraphLaunch(ctx->gexec, st)) != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphLaunch");
    // streamed levels (one launch per step or per wave), each on its level's
    // stream, after the graph (whose cluster grids would otherwise wait for
    // free SMs behind the streamed levels' stream of short CTAs) and beside
    // each other: the levels fill each other's last waves.  Each level's
    // launches are enqueued by a host thread of its own, since enqueueing
    // blocks while a stream's launch queue is full.
    if ((e = cudaEventRecord(ctx->ev_graph, st)) != cudaSuccess) return cuda_fail(ctx, e, "graph event");
    std::vector<char> joined(nl, 0);
    std::vector<int> lrc(nl, MLMC_DK_OK);
    std::vector<std::thread> enq;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(ctx, e, "cudaGetDevice");
    auto enqueue = [ctx, counts, firsts, seed, sums_dev, dev, &lrc](int l) {
        cudaError_t ee = cudaSetDevice(dev);
        if (ee == cudaSuccess) ee = cudaStreamWaitEvent(ctx->lstream[l], ctx->ev_graph, 0);
        if (ee == cudaSuccess) ee = cudaEventRecord(ctx->ev_lb[l], ctx->lstream[l]);
        if (ee != cudaSuccess) {
            lrc[l] = cuda_fail(ctx, ee, "streamed level fork");
            return;
        }
        lrc[l] = launch_streamed(ctx, l, 0, firsts[l], counts[l], seed, sums_dev + (size_t)l * ctx->stride, nullptr,
                                 ctx->lstream[l]);
        if (lrc[l] != MLMC_DK_OK) return;
        if ((ee = cudaEventRecord(ctx->ev_le[l], ctx->lstream[l])) != cudaSuccess ||
            (ee = cudaEventRecord(ctx->ev_join[l], ctx->lstream[l])) != cudaSuccess)
            lrc[l] = cuda_fail(ctx, ee, "streamed level join");
    };
    for (int l = nl - 1; l >= 0; --l) {
        if (!ctx->lv[l].streamed || band_level(l)) continue;
        joined[l] = 1;
        enq.emplace_back(enqueue, l);
    }
    for (auto& th : enq) th.join();
    for (int l = nl - 1; l >= 0; --l)
        if (lrc[l] != MLMC_DK_OK) return lrc[l];
    for (int l = nl - 1; l >= 0; --l) {
        if (!joined[l] && !(any_band && band_level(l))) continue;
        if ((e = cudaStreamWaitEvent(st, ctx->ev_join[l], 0)) != cudaSuccess) return cuda_fail(ctx, e, "level join");
    }
    if (any_split) {
        for (int l = nl - 1; l >= 0; --l) {
            if (n_split[l] == 0) continue;
            rc = launch_streamed(ctx, l, 0, firsts[l] + n_reg[l], n_split[l], seed,
                                 ctx->d_ssums + (size_t)l * ctx->stride, nullptr, ctx->sstream, 0,
                                 dk::stream_default_variant());
            if (rc != MLMC_DK_OK) return rc;
        }
        if ((e = cudaEventRecord(ctx->ev_sjoin, ctx->sstream)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(st, ctx->ev_sjoin, 0)) != cudaSuccess)
            return cuda_fail(ctx, e, "batch split join");
        for (int l = 0; l < nl; ++l)
            if (n_split[l] > 0 && (e = dk::launch_add_sums(sums_dev + (size_t)l * ctx->stride,
                                                             ctx->d_ssums + (size_t)l * ctx->stride, ctx->stride,
                                                             st)) != cudaSuccess)
                return cuda_fail(ctx, e, "batch split merge");
    }
    return MLMC_DK_OK;
}

}  // namespace

extern "C" {

int mlmc_dk_run_batch_dev(mlmc_dk_ctx* ctx, const int64_t* counts, int64_t first_sample, uint64_t seed,
                          double* sums_dev, void* cuda_stream) {
    if (!ctx) return fail(nullptr, MLMC_DK_ERR_INVALID, "null context");
    if (!counts || !sums_dev || ((uintptr_t)sums_dev & 7) || first_sample < 0)
        return fail(ctx, MLMC_DK_ERR_INVALID, "run_batch_dev: bad arguments");
    const int nl = ctx->L_max + 1;
    for (int l = 0; l < nl; ++l)
        if (counts[l] < 0) return fail(ctx, MLMC_DK_ERR_INVALID, "run_batch_dev: negative count");
    cudaStream_t st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->stream;
    std::vector<int64_t> firsts(nl, first_sample);
    return batch_dev(ctx, counts, firsts.data(), seed, sums_dev, st);
}

int mlmc_dk_set_batch_split(mlmc_dk_ctx* ctx, int32_t level, double fraction) {
    if (!ctx || level < 1 || level > ctx->L_max || !(fraction >= 0.0 && fraction <= 0.5))
        return fail(ctx, MLMC_DK_ERR_INVALID, "set_batch_split: level 1..L_max, fraction in [0, 1/2]");
    LevelTab& t = ctx->lv[level];
    if (fraction > 0 && !t.split_ok)
        return fail(ctx, MLMC_DK_ERR_UNSUPPORTED, "set_batch_split: the level has no streamed share");
    t.split_frac = fraction;
    return MLMC_DK_OK;
}

int mlmc_dk_tune_batch(mlmc_dk_ctx* ctx, const int64_t* counts, int32_t repeats, double* fraction, double* seconds) {
    if (!ctx || !counts) return fail(ctx, MLMC_DK_ERR_INVALID, "tune_batch: bad arguments");
    const auto t0 = std::chrono::steady_clock::now();
    repeats = std::max(1, repeats);
    int lvl = -1;
    for (int l = ctx->L_max; l >= 1 && lvl < 0; --l)
        if (ctx->lv[l].split_ok && counts[l] > 1) lvl = l;
    double best_f = 0.0;
    if (lvl >= 0) {
        static const double kFractions[] = {0.0, 0.04, 0.06, 0.08, 0.10, 0.12};
        double best_ms = 1e300;
        cudaError_t e;
        auto time_batch = [&](double* ms) -> int {
            if ((e = cudaEventRecord(ctx->ev0, ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "tune_batch");
            int rc = mlmc_dk_run_batch_dev(ctx, counts, 0, 0x7475, ctx->d_bsums, ctx->stream);
            if (rc != MLMC_DK_OK) return rc;
            if ((e = cudaEventRecord(ctx->ev1, ctx->stream)) != cudaSuccess ||
                (e = cudaEventSynchronize(ctx->ev1)) != cudaSuccess)
                return cuda_fail(ctx, e, "tune_batch");
            float t = 0.f;
            cudaEventElapsedTime(&t, ctx->ev0, ctx->ev1);
            *ms = t;
            return MLMC_DK_OK;
        };
        // one untimed run warms the graph and the streamed path up
        ctx->lv[lvl].split_frac = kFractions[1];
        double warm = 0.0;
        int rc = time_batch(&warm);
        if (rc != MLMC_DK_OK) return rc;
        for (double f : kFractions) {
            ctx->lv[lvl].split_frac = f;
            double ms_min = 1e300;
            for (int r = 0; r < repeats; ++r) {
                double ms = 0.0;
                if ((rc = time_batch(&ms)) != MLMC_DK_OK) return rc;
                ms_min = std::min(ms_min, ms);
            }
            if (ms_min < 0.99 * best_ms) {   // a larger share only if clearly faster
                best_ms = ms_min;
                best_f = f;
            }
        }
        ctx->lv[lvl].split_frac = best_f;
    }
    int rc = check_device_error(ctx);
    if (rc != MLMC_DK_OK) return rc;
    if (fraction) *fraction = best_f;
    if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return MLMC_DK_OK;
}

int mlmc_dk_batch_level_ms(mlmc_dk_ctx* ctx, double* ms) {
    if (!ctx || !ms) return fail(ctx, MLMC_DK_ERR_INVALID, "batch_level_ms: bad arguments");
    for (int l = 0; l <= ctx->L_max; ++l) {
        float t = 0.f;
        const cudaError_t e = cudaEventElapsedTime(&t, ctx->ev_lb[l], ctx->ev_le[l]);
        if (e == cudaErrorNotReady) return cuda_fail(ctx, e, "batch still running");
        ms[l] = e == cudaSuccess ? (double)t : 0.0;
        if (e != cudaSuccess) cudaGetLastError();
    }
    return MLMC_DK_OK;
}

int mlmc_dk_run_batch(mlmc_dk_ctx* ctx, const int64_t* counts, uint64_t seed, mlmc_dk_level_sums* sums) {
    if (!ctx) return fail(nullptr, MLMC_DK_ERR_INVALID, "null context");
    if (!counts || !sums) return fail(ctx, MLMC_DK_ERR_INVALID, "run_batch: bad arguments");
    const int nl = ctx->L_max + 1;
    for (int l = 0; l < nl; ++l)
        if (counts[l] < 0) return fail(ctx, MLMC_DK_ERR_INVALID, "run_batch: negative count");
    // one id range for all levels: the batch starts after the furthest level
    int64_t first = 0;
    for (int l = 0; l < nl; ++l) first = std::max(first, ctx->next_id[0][l]);
    const auto t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaEventRecord(ctx->ev0, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventRecord");
    int rc = mlmc_dk_run_batch_dev(ctx, counts, first, seed, ctx->d_bsums, ctx->stream);
    if (rc != MLMC_DK_OK) return rc;
    if ((e = cudaEventRecord(ctx->ev1, ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "cudaEventRecord");
    e = cudaMemcpyAsync(ctx->h_bsums, ctx->d_bsums, sizeof(double) * ctx->stride * nl, cudaMemcpyDeviceToHost,
                        ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    if ((rc = check_device_error(ctx)) != MLMC_DK_OK) return rc;
    const double wall = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int active = 0;
    for (int l = 0; l < nl; ++l) active += counts[l] > 0;
    for (int l = 0; l < nl; ++l) {
        if (counts[l] == 0) continue;
        ctx->next_id[0][l] = first + counts[l];
        const LevelTab& f = ctx->lv[l];
        double cost = (double)f.n * f.n * f.M;
        if (l > 0) cost += (double)ctx->lv[l - 1].n * ctx->lv[l - 1].n * ctx->lv[l - 1].M;
        accumulate(ctx, ctx->h_bsums + (size_t)l * ctx->stride, sums + (size_t)l * ctx->n_quant, cost,
                   wall / active, 1e-3 * ms / active, 2);
    }
    return MLMC_DK_OK;
}

int mlmc_dk_set_variant(mlmc_dk_ctx* ctx, int32_t level, int32_t coupled, int32_t variant) {
    if (!ctx || level < 0 || level > ctx->L_max || (coupled && level == 0))
        return fail(ctx, MLMC_DK_ERR_INVALID, "set_variant: bad level");
    LevelTab& t = ctx->lv[level];
    const int mode = coupled ? 1 : 0;
    if (variant < 0 || variant >= (int)t.vis[mode].size() || !t.vis[mode][variant].supported)
        return fail(ctx, MLMC_DK_ERR_INVALID, "set_variant: no such variant");
    t.sel[mode] = variant;
    return MLMC_DK_OK;
}

int mlmc_dk_tune(mlmc_dk_ctx* ctx, int32_t repeats, double* seconds) {
    if (!ctx) return fail(nullptr, MLMC_DK_ERR_INVALID, "null context");
    const auto t0 = std::chrono::steady_clock::now();
    repeats = std::max(1, repeats);
    cudaError_t e;
    for (int l = 0; l <= ctx->L_max; ++l) {
        LevelTab& t = ctx->lv[l];
        for (int mode = 0; mode < 2; ++mode) {
            if (t.vis[mode].size() < 2) continue;
            double best = 1e300;
            int best_v = t.sel[mode];
            for (int v = 0; v < (int)t.vis[mode].size(); ++v) {
                const dk::VariantInfo& vi = t.vis[mode][v];
                if (!vi.supported) continue;
                t.sel[mode] = v;
                // register kernels: two full waves of resident sample slots; streamed
                // and band kernels: one wave of samples in flight over a shorter
                // horizon; compared per sample and fine step
                int steps = t.M;
                int64_t count;
                if (vi.band) {
                    count = t.bplan[mode][vi.band == 4 ? 0 : 1].S;
                    steps = std::min(t.M, 512);
                } else if (t.streamed) {
                    count = t.inflight_v[v];
                    steps = std::min(t.M, 512);
                } else {
                    count = 2LL * (vi.max_ctas / vi.cluster) * vi.slots_per_cta;
                }
                double ms_min = 1e300;
                for (int r = 0; r < repeats + 1; ++r) {
                    if ((e = cudaEventRecord(ctx->ev0, ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "tune");
                    const int tag = mode == 1 ? 0 : 1;
                    int rc = vi.band ? launch_band(ctx, l, tag, 0, count, 0x7475, ctx->d_sums, nullptr, ctx->stream, steps)
                             : t.streamed ? launch_streamed(ctx, l, tag, 0, count, 0x7475, ctx->d_sums, nullptr, ctx->stream,
                                                            steps)
                                          : launch_batch(ctx, l, tag, 0, count, 0x7475, ctx->d_sums, nullptr, ctx->stream);
                    if (rc != MLMC_DK_OK) return rc;
                    if ((e = cudaEventRecord(ctx->ev1, ctx->stream)) != cudaSuccess ||
                        (e = cudaEventSynchronize(ctx->ev1)) != cudaSuccess)
                        return cuda_fail(ctx, e, "tune");
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
                    if (r > 0) ms_min = std::min(ms_min, (double)ms);   // the first run warms up
                }
                const double per_sample = ms_min / ((double)count * (double)steps);
                if (per_sample < best) {
                    best = per_sample;
                    best_v = v;
                }
            }
            t.sel[mode] = best_v;
        }
    }
    int rc = check_device_error(ctx);
    if (rc != MLMC_DK_OK) return rc;
    if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return MLMC_DK_OK;
}

}  // extern "C"

namespace {
// Eq. (opt_M_ell) and Eq. (convergence_criterion) with the levels' mesh ratio
// r (the printed criterion has r = 2, the NN coupling's; the Fourier
// coupling's levels refine by r = 3): stop if
// max_t r^(-t alpha) |E_{L-t}| / (r^alpha - 1) < eps / sqrt 2.
int plan_ratio(int32_t L, const int64_t* n, const double* s1, const double* s2, const double* cost, double eps,
               int64_t* target, int32_t* converged, double ratio) {
    if (L < 0 || L >= MLMC_DK_MAX_LEVELS || !n || !s1 || !s2 || !cost || !target || !converged || !(eps > 0))
        return fail(nullptr, MLMC_DK_ERR_INVALID, "plan: bad arguments");
    double V[MLMC_DK_MAX_LEVELS], E[MLMC_DK_MAX_LEVELS];
    double total = 0;
    for (int l = 0; l <= L; ++l) {
        if (n[l] < 2 || !(cost[l] > 0)) return fail(nullptr, MLMC_DK_ERR_INVALID, "plan: need n >= 2 and cost > 0");
        const double m = (double)n[l];
        E[l] = s1[l] / m;
        V[l] = std::max(0.0, (s2[l] - s1[l] * s1[l] / m) / (m - 1.0));
        total += std::sqrt(V[l] * cost[l]);
    }
    // Eq. (opt_M_ell)
    for (int l = 0; l <= L; ++l) {
        const double opt = std::ceil(2.0 / (eps * eps) * std::sqrt(V[l] / cost[l]) * total);
        target[l] = std::max<int64_t>(n[l], (int64_t)std::min(opt, 9.0e18));
    }
    // Eq. (convergence_criterion), alpha = 2, P_{-1} = 0
    const double alpha = 2.0;
    double worst = 0;
    for (int t = 0; t <= 2 && L - t >= 0; ++t) worst = std::max(worst, std::pow(ratio, -t * alpha) * std::fabs(E[L - t]));
    *converged = worst / (std::pow(ratio, alpha) - 1.0) < eps / std::sqrt(2.0) ? 1 : 0;
    return MLMC_DK_OK;
}
}  // namespace

extern "C" {

int mlmc_dk_plan(int32_t L, const int64_t* n, const double* s1, const double* s2, const double* cost, double eps,
                 int64_t* target, int32_t* converged) {
    return plan_ratio(L, n, s1, s2, cost, eps, target, converged, 2.0);
}

int mlmc_dk_plan_ratio(int32_t L, const int64_t* n, const double* s1, const double* s2, const double* cost,
                       double eps, double ratio, int64_t* target, int32_t* converged) {
    if (!(ratio > 1.0)) return fail(nullptr, MLMC_DK_ERR_INVALID, "plan: ratio must exceed 1");
    return plan_ratio(L, n, s1, s2, cost, eps, target, converged, ratio);
}

}  // extern "C"

namespace {

using RoundFn = std::function<int(int32_t L, const int64_t* first, const int64_t* count, double* sums)>;
using ReduceFn = std::function<int(double* sums, int64_t n_levels, int64_t stride)>;

// Algorithm 1 (Section 7.1), the one implementation behind mlmc_dk_estimate
// (one process, the multi-level batch on the GPU) and mlmc_dk_algorithm1 (any
// sampler, several processes): start at L = L_start with `pilot` samples on
// levels 0..L; repeat {run the missing samples of every level -- each level's
// new ids cut into `world` contiguous pieces, piece `rank` run here, the
// round's sums combined over the processes by `reduce` --, set targets by
// Eq. (opt_M_ell), once no level needs more than 1% more samples apply Eq.
// (convergence_criterion) with alpha = 2 and the hierarchy's mesh ratio, and
// add a level if it fails}.  The first quantity drives the allocation; eps is
// absolute, or relative to the pilot estimate.  Sums use the device layout
// [level][2 + 12 n_quant] (entry 0 count, entry 1 max mass error).
int algorithm1_core(int32_t L_max, int32_t L_start, int64_t pilot, int32_t n_quant, const double* cost, double ratio,
                    double eps, int32_t relative, int32_t rank, int32_t world, const RoundFn& run,
                    const ReduceFn& reduce, mlmc_dk_result* out, std::vector<double>* totals, std::string* err) {
    const int nl = L_max + 1;
    const int64_t stride = 2 + (int64_t)dk::kNSum * n_quant;
    std::vector<double> tot((size_t)nl * stride, 0.0), rnd((size_t)nl * stride);
    std::vector<int64_t> target(nl, 0), next(nl, 0), first(nl, 0), count(nl, 0), need(nl, 0);
    int L = std::min(L_start, L_max);
    for (int l = 0; l <= L; ++l) target[l] = pilot;
    double eps_abs = relative ? -1.0 : eps;
    int status = MLMC_DK_OK, converged = 0;
    for (int iter = 0; iter < 1000; ++iter) {
        bool any = false;
        for (int l = 0; l < nl; ++l) {
            need[l] = l <= L ? std::max<int64_t>(0, target[l] - next[l]) : 0;
            const int64_t base = need[l] / world, extra = need[l] % world;
            count[l] = base + (rank < extra ? 1 : 0);
            first[l] = next[l] + rank * base + std::min<int64_t>(rank, extra);
            any = any || need[l] > 0;
        }
        if (any) {
            std::fill(rnd.begin(), rnd.end(), 0.0);
            int rc = run(L, first.data(), count.data(), rnd.data());
            if (rc != MLMC_DK_OK) return rc;
            if (world > 1 && reduce && (rc = reduce(rnd.data(), nl, stride)) != MLMC_DK_OK) {
                *err = "Algorithm 1: the reduction over processes failed";
                return rc;
            }
            for (int l = 0; l < nl; ++l) {
                for (int64_t e = 0; e < stride; ++e) {
                    double& t = tot[(size_t)l * stride + e];
                    const double r = rnd[(size_t)l * stride + e];
                    t = e == 1 ? std::max(t, r) : t + r;
                }
                next[l] += need[l];
            }
        }
        int64_t n[MLMC_DK_MAX_LEVELS];
        double s1[MLMC_DK_MAX_LEVELS], s2[MLMC_DK_MAX_LEVELS];
        for (int l = 0; l <= L; ++l) {
            n[l] = (int64_t)std::llround(tot[(size_t)l * stride]);
            s1[l] = tot[(size_t)l * stride + 2];
            s2[l] = tot[(size_t)l * stride + 3];
        }
        if (eps_abs < 0) {
            double mu = 0;
            for (int l = 0; l <= L; ++l) mu += s1[l] / (double)n[l];
            eps_abs = eps * std::fabs(mu);
            if (!(eps_abs > 0)) {
                *err = "relative eps with a zero pilot estimate";
                return MLMC_DK_ERR_INVALID;
            }
        }
        int64_t tgt[MLMC_DK_MAX_LEVELS];
        int32_t conv = 0;
        const int rc = plan_ratio(L, n, s1, s2, cost, eps_abs, tgt, &conv, ratio);
        if (rc != MLMC_DK_OK) {
            *err = g_init_error;
            return rc;
        }
        bool more = false;
        for (int l = 0; l <= L; ++l) {
            target[l] = std::max(target[l], tgt[l]);
            if ((double)(target[l] - n[l]) > 0.01 * (double)n[l]) more = true;
        }
        if (more) continue;
        if (conv) { converged = 1; break; }
        if (L == L_max) { status = MLMC_DK_NOT_CONVERGED; break; }
        ++L;
        target[L] = pilot;
    }
    out->L = L;
    out->converged = converged;
    out->eps_abs = eps_abs;
    for (int q = 0; q < n_quant && q < MLMC_DK_MAX_QUANT; ++q) {
        double est = 0;
        for (int l = 0; l <= L; ++l) est += tot[(size_t)l * stride + 2 + dk::kNSum * q] / tot[(size_t)l * stride];
        out->estimates[q] = est;
    }
    out->estimate = out->estimates[0];
    out->variance = 0.0;
    for (int l = 0; l <= L; ++l) {
        const double* t = tot.data() + (size_t)l * stride;
        const double m = t[0];
        out->M[l] = (int64_t)std::llround(m);
        out->E[l] = t[2] / m;
        out->V[l] = std::max(0.0, (t[3] - t[2] * t[2] / m) / (m - 1.0));
        out->C[l] = cost[l];
        out->variance += out->V[l] / m;
        out->cell_steps += m * cost[l];
        out->var_pf[l] = std::max(0.0, (t[7] - t[6] * t[6] / m) / (m - 1.0));
    }
    if (totals) totals->swap(tot);
    return status;
}

}  // namespace

extern "C" {

int mlmc_dk_algorithm1(int32_t L_max, int32_t L_start, int64_t pilot, int32_t n_quant, const double* cost,
                       double ratio, double eps, int32_t relative, int32_t rank, int32_t world,
                       mlmc_dk_round_fn run_round, mlmc_dk_reduce_fn reduce, void* user, mlmc_dk_result* out) {
    if (L_max < 0 || L_max >= MLMC_DK_MAX_LEVELS || L_start < 0 || pilot < 2 || n_quant < 1 ||
        n_quant > MLMC_DK_MAX_QUANT || !cost || !(ratio > 1.0) || !(eps > 0) || world < 1 || rank < 0 ||
        rank >= world || !run_round || !out || (world > 1 && !reduce))
        return fail(nullptr, MLMC_DK_ERR_INVALID, "algorithm1: bad arguments");
    *out = mlmc_dk_result{};
    const auto t0 = std::chrono::steady_clock::now();
    std::string err;
    const RoundFn run = [&](int32_t L, const int64_t* first, const int64_t* count, double* sums) {
        const int rc = run_round(user, L, first, count, sums);
        if (rc != 0) err = "Algorithm 1: the round callback failed";
        return rc == 0 ? MLMC_DK_OK : MLMC_DK_ERR_INVALID;
    };
    const ReduceFn red = [&](double* sums, int64_t nl, int64_t stride) {
        return reduce(user, sums, nl, stride) == 0 ? MLMC_DK_OK : MLMC_DK_ERR_INVALID;
    };
    const int rc = algorithm1_core(L_max, L_start, pilot, n_quant, cost, ratio, eps, relative, rank, world, run, red,
                                   out, nullptr, &err);
    if (rc < 0) return fail(nullptr, rc, err);
    out->wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

int mlmc_dk_estimate(mlmc_dk_ctx* ctx, double eps, int32_t relative, uint64_t seed, mlmc_dk_result* out) {
    if (!ctx || !out || !(eps > 0)) return fail(ctx, MLMC_DK_ERR_INVALID, "estimate: bad arguments");
    const auto t0 = std::chrono::steady_clock::now();
    *out = mlmc_dk_result{};
    const int nl = ctx->L_max + 1;
    std::fill(ctx->next_id[0].begin(), ctx->next_id[0].end(), 0);
    std::vector<double> cost(nl), kernel_s(nl, 0.0);
    for (int l = 0; l < nl; ++l) {
        mlmc_dk_level_desc li;
        mlmc_dk_level_info(ctx, l, &li);
        cost[l] = li.cost;
    }
    int64_t launches = 0, d2h = 0;
    // one round: the missing samples of every level at once through the
    // multi-level batch (the levels run concurrently), ids continuing each
    // level's range
    const RoundFn run = [&](int32_t, const int64_t* first, const int64_t* count, double* sums) {
        int rc = batch_dev(ctx, count, first, seed, ctx->d_bsums, ctx->stream);
        if (rc != MLMC_DK_OK) return rc;
        cudaError_t e = cudaMemcpyAsync(sums, ctx->d_bsums, sizeof(double) * ctx->stride * nl,
                                        cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "Algorithm 1 round");
        if ((rc = check_device_error(ctx)) != MLMC_DK_OK) return rc;
        for (int l = 0; l < nl; ++l) {
            if (count[l] == 0) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ctx->ev_lb[l], ctx->ev_le[l]) != cudaSuccess) {
                cudaGetLastError();
                ms = 0.f;
            }
            kernel_s[l] += 1e-3 * ms;
            launches += 2;
            d2h += (int64_t)(sizeof(double) * ctx->stride + sizeof(unsigned));
            ctx->next_id[0][l] = first[l] + count[l];
        }
        return MLMC_DK_OK;
    };
    std::string err;
    const int status = algorithm1_core(ctx->L_max, ctx->L_start, ctx->pilot, ctx->n_quant, cost.data(),
                                       ctx->coupling == 1 ? 3.0 : 2.0, eps, relative, 0, 1, run, nullptr, out,
                                       nullptr, &err);
    if (status < 0) return err.empty() ? status : fail(ctx, status, err);
    for (int l = 0; l <= out->L; ++l) {
        out->sample_steps += (double)out->M[l] * ctx->lv[l].M;
        out->kernel_s[l] = kernel_s[l];
    }
    out->launches = launches;
    out->d2h_bytes = d2h;
    out->wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return status;
}

int mlmc_dk_noise_dev(uint64_t seed, int32_t level, int32_t stream_tag, int64_t sample, int32_t m, int32_t n,
                      float* z_dev, uint32_t* raw_dev, void* cuda_stream) {
    if (n < 2 || (n & 1) || m < 0 || sample < 0 || level < -1 || level > 254 || stream_tag < 0 || stream_tag > 255 ||
        (!z_dev && !raw_dev) || ((uintptr_t)z_dev & 15) || ((uintptr_t)raw_dev & 15))
        return fail(nullptr, MLMC_DK_ERR_INVALID, "noise_dev: bad arguments");
    const uint32_t c3 = ((uint32_t)(level + 1) & 0xffu) | (((uint32_t)stream_tag & 0xffu) << 8) |
                        ((uint32_t)(((uint64_t)sample >> 32) & 0xffffu) << 16);
    cudaError_t e = dk::launch_noise(n, (uint32_t)m, (uint32_t)sample, c3, (uint32_t)(seed & 0xffffffffu),
                                     (uint32_t)(seed >> 32), z_dev, raw_dev, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? MLMC_DK_OK : cuda_fail(nullptr, e, "noise kernel");
}

int mlmc_dk_save_state(const mlmc_dk_ctx* ctx, void* buf, size_t* len) {
    if (!ctx || !len) return fail(const_cast<mlmc_dk_ctx*>(ctx), MLMC_DK_ERR_INVALID, "save_state: bad arguments");
    const size_t levels = ctx->lv.size();
    const size_t need = 16 + 2 * levels * sizeof(int64_t);
    if (!buf) { *len = need; return MLMC_DK_OK; }
    if (*len < need) return fail(const_cast<mlmc_dk_ctx*>(ctx), MLMC_DK_ERR_INVALID, "save_state: buffer too small");
    unsigned char* p = static_cast<unsigned char*>(buf);
    const uint32_t magic = 0x4d4c444bu, version = 1, nl = (uint32_t)levels, nq = (uint32_t)ctx->n_quant;
    std::memcpy(p, &magic, 4); std::memcpy(p + 4, &version, 4); std::memcpy(p + 8, &nl, 4); std::memcpy(p + 12, &nq, 4);
    std::memcpy(p + 16, ctx->next_id[0].data(), levels * sizeof(int64_t));
    std::memcpy(p + 16 + levels * sizeof(int64_t), ctx->next_id[1].data(), levels * sizeof(int64_t));
    *len = need;
    return MLMC_DK_OK;
}

int mlmc_dk_load_state(mlmc_dk_ctx* ctx, const void* buf, size_t len) {
    if (!ctx || !buf) return fail(ctx, MLMC_DK_ERR_INVALID, "load_state: bad arguments");
    const size_t levels = ctx->lv.size();
    if (len != 16 + 2 * levels * sizeof(int64_t)) return fail(ctx, MLMC_DK_ERR_STATE, "load_state: size mismatch");
    const unsigned char* p = static_cast<const unsigned char*>(buf);
    uint32_t magic, version, nl, nq;
    std::memcpy(&magic, p, 4); std::memcpy(&version, p + 4, 4); std::memcpy(&nl, p + 8, 4); std::memcpy(&nq, p + 12, 4);
    if (magic != 0x4d4c444bu || version != 1 || nl != levels || nq != (uint32_t)ctx->n_quant)
        return fail(ctx, MLMC_DK_ERR_STATE, "load_state: checkpoint does not match this context");
    std::vector<int64_t> a(levels), b(levels);
    std::memcpy(a.data(), p + 16, levels * sizeof(int64_t));
    std::memcpy(b.data(), p + 16 + levels * sizeof(int64_t), levels * sizeof(int64_t));
    for (size_t l = 0; l < levels; ++l)
        if (a[l] < 0 || b[l] < 0) return fail(ctx, MLMC_DK_ERR_STATE, "load_state: negative sample id");
    ctx->next_id[0] = a;
    ctx->next_id[1] = b;
    return MLMC_DK_OK;
}

}  // extern "C"

// ===================================================== learned level below 0
namespace {

// parameter layout (layer by layer, W [out][in] then b): 64*256+256 + 2*(256*256+256) + K*(256+1)
constexpr int kOffW1 = 0, kOffB1 = 16384, kOffW2 = 16640, kOffB2 = 82176, kOffW3 = 82432, kOffB3 = 147968,
              kOffW4 = 148224;
constexpr int kBfW1 = 0, kBfW2 = 16384, kBfW3 = 81920, kBfW4 = 147456;
constexpr int param_count(int K) { return kOffW4 + (dk::kHidden + 1) * K; }
constexpr int off_b4(int K) { return kOffW4 + dk::kHidden * K; }
constexpr int bf_total(int K) { return kBfW4 + dk::kHidden * K; }
constexpr int kMomentBlocks = 128;

void free_surrogate(Surrogate* s) {
    if (!s) return;
    for (void* p : {(void*)s->d_E, (void*)s->d_g, (void*)s->d_inv_sigma, (void*)s->d_theta, (void*)s->d_grad,
                    (void*)s->d_m1, (void*)s->d_m2, (void*)s->d_wbf, (void*)s->d_bfidx, (void*)s->d_X,
                    (void*)s->d_H1, (void*)s->d_H2, (void*)s->d_H3, (void*)s->d_dH1, (void*)s->d_dH2,
                    (void*)s->d_dH3, (void*)s->d_y, (void*)s->d_dy, (void*)s->d_T, (void*)s->d_Xf,
                    (void*)s->d_samp, (void*)s->d_D0, (void*)s->d_part, (void*)s->d_loss, (void*)s->d_trainX,
                    (void*)s->d_trainT, (void*)s->d_idx, (void*)s->d_tA, (void*)s->d_tB, (void*)s->d_wt})
        cudaFree(p);
    delete s;
}

// The 32 lowest real orthonormal modes of the n x n grid: wave vectors with
// k1 > 0, or k1 = 0 and k2 > 0 (Nyquist lines excluded), ordered by |k|^2
// then (k1, k2); a cosine and a sine mode each, scaled to unit plain-sum norm.
// With the theta-scheme's weights (b0, 1 - b0) the per-step factor of mode k is
// (1 - b1 lam)/(1 + b0 lam), and the noise of every step reaches the mode
// through the implicit operator with the constant factor 1/(1 + b0 lam), which
// the standardisation by the feature's exact deviation removes.
void build_modes(int n, double mu, int M, std::vector<float>& E, std::vector<float>& g, std::vector<float>& isig,
                 double b0) {
    std::vector<std::pair<int, int>> ks;
    for (int k1 = 0; k1 <= n / 2; ++k1)
        for (int k2 = -n / 2 + 1; k2 <= n / 2; ++k2) {
            if ((k1 == 0 && k2 <= 0) || 2 * k1 == n || 2 * std::abs(k2) == n) continue;
            ks.push_back({k1, k2});
        }
    std::sort(ks.begin(), ks.end(), [](const std::pair<int, int>& a, const std::pair<int, int>& b) {
        const int na = a.first * a.first + a.second * a.second, nb = b.first * b.first + b.second * b.second;
        return na != nb ? na < nb : a < b;  // (k1, k2) lexicographic among equal |k|^2
    });
    E.assign((size_t)dk::kModes * n * n, 0.f);
    g.assign(dk::kModes, 0.f);
    isig.assign(dk::kFeat, 0.f);
    const double scale = std::sqrt(2.0 / ((double)n * n));
    for (int j = 0; j < dk::kModes / 2; ++j) {
        const int k1 = ks[j].first, k2 = ks[j].second;
        const double lam = 2.0 * mu * (std::pow(std::sin(M_PI * k1 / n), 2) + std::pow(std::sin(M_PI * k2 / n), 2));
        const double gk = (1.0 - (1.0 - b0) * lam) / (1.0 + b0 * lam);
        double var = 0.0, p = 1.0;
        for (int i = 0; i < M; ++i, p *= gk * gk) var += p;
        for (int cs = 0; cs < 2; ++cs) {
            const int mode = 2 * j + cs;
            g[mode] = (float)gk;
            for (int i1 = 0; i1 < n; ++i1)
                for (int i2 = 0; i2 < n; ++i2) {
                    const double ang = 2.0 * M_PI * (double)(k1 * i1 + k2 * i2) / n;
                    E[(size_t)mode * n * n + i1 * n + i2] = (float)(scale * (cs == 0 ? std::cos(ang) : std::sin(ang)));
                }
            isig[2 * mode] = isig[2 * mode + 1] = (float)(1.0 / std::sqrt(var));
        }
    }
}

dk::GemmArgs gemm(int M, int N, int K, const __nv_bfloat16* A, long long sam, long long sak, const __nv_bfloat16* B,
                  long long sbk, long long sbn) {
    dk::GemmArgs g{};
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.sam = sam; g.sak = sak;
    g.B = B; g.sbk = sbk; g.sbn = sbn;
    return g;
}

// Network forward on n standardised feature rows X (n <= chunk): y = That.
// The dense layers run on the tensor cores (tcgen05): H = relu(X W^T + b),
// X [n][in] and W [out][in] both K-major.
cudaError_t mlp_forward(Surrogate* s, const __nv_bfloat16* X, int n, float* y, cudaStream_t st) {
    cudaError_t e;
    dk::GemmArgs g = gemm(n, dk::kHidden, dk::kFeat, X, dk::kFeat, 1, s->d_wbf + kBfW1, 1, dk::kFeat);
    g.Cb = s->d_H1; g.ldcb = dk::kHidden; g.bias = s->d_theta + kOffB1; g.relu = 1;
    if ((e = dk::launch_gemm_tc(g, s->err, st)) != cudaSuccess) return e;
    g = gemm(n, dk::kHidden, dk::kHidden, s->d_H1, dk::kHidden, 1, s->d_wbf + kBfW2, 1, dk::kHidden);
    g.Cb = s->d_H2; g.ldcb = dk::kHidden; g.bias = s->d_theta + kOffB2; g.relu = 1;
    if ((e = dk::launch_gemm_tc(g, s->err, st)) != cudaSuccess) return e;
    g = gemm(n, dk::kHidden, dk::kHidden, s->d_H2, dk::kHidden, 1, s->d_wbf + kBfW3, 1, dk::kHidden);
    g.Cb = s->d_H3; g.ldcb = dk::kHidden; g.bias = s->d_theta + kOffB3; g.relu = 1;
    if ((e = dk::launch_gemm_tc(g, s->err, st)) != cudaSuccess) return e;
    return dk::launch_out_forward(s->d_H3, s->d_theta + kOffW4, s->d_theta + off_b4(s->K), n, dk::kHidden, s->K, y,
                                  st);
}

// Mean-squared-error gradient of a batch (after mlp_forward on it) into d_grad.
cudaError_t mlp_backward(Surrogate* s, const __nv_bfloat16* X, const float* T, int B, cudaStream_t st) {
    cudaError_t e;
    float* G = s->d_grad;
    if ((e = dk::launch_out_backward(s->d_y, T, s->d_H3, s->d_theta + kOffW4, B, dk::kHidden, s->K, s->d_dy, s->d_dH3,
                                     G + kOffW4, G + off_b4(s->K), st)) != cudaSuccess)
        return e;
    struct Layer { const __nv_bfloat16* dH; const __nv_bfloat16* Hin; int K; float* gW; float* gb;
                   const __nv_bfloat16* W; __nv_bfloat16* dHin; };
    const Layer layers[3] = {
        {s->d_dH3, s->d_H2, dk::kHidden, G + kOffW3, G + kOffB3, s->d_wbf + kBfW3, s->d_dH2},
        {s->d_dH2, s->d_H1, dk::kHidden, G + kOffW2, G + kOffB2, s->d_wbf + kBfW2, s->d_dH1},
        {s->d_dH1, X, dk::kFeat, G + kOffW1, G + kOffB1, nullptr, nullptr}};
    for (const Layer& L : layers) {
        // dW = dH^T Hin (256 x K, summed over the batch) as a K-major product on
        // the tensor cores: A = dH^T [256][B], B operand = Hin^T [K][B]
        // rows of the transposed operands padded to 8 elements (16 bytes, the TMA
        // stride unit); the padding lies beyond K = B and is never read
        const int ldt = (B + 7) & ~7;
        if ((e = dk::launch_transpose_bf16(L.dH, B, dk::kHidden, s->d_tA, ldt, st)) != cudaSuccess ||
            (e = dk::launch_transpose_bf16(L.Hin, B, L.K, s->d_tB, ldt, st)) != cudaSuccess)
            return e;
        dk::GemmArgs g = gemm(dk::kHidden, L.K, B, s->d_tA, ldt, 1, s->d_tB, 1, ldt);
        g.C = L.gW; g.ldc = L.K;
        if ((e = dk::launch_gemm_tc(g, s->err, st)) != cudaSuccess) return e;
        if ((e = dk::launch_colsum(L.dH, nullptr, B, dk::kHidden, L.gb, st)) != cudaSuccess) return e;
        if (L.W) {
            // dHin = (dH W) * (Hin > 0): A = dH [B][256], B operand = W^T [in][out]
            if ((e = dk::launch_transpose_bf16(L.W, dk::kHidden, dk::kHidden, s->d_wt, dk::kHidden, st)) != cudaSuccess)
                return e;
            g = gemm(B, dk::kHidden, dk::kHidden, L.dH, dk::kHidden, 1, s->d_wt, 1, dk::kHidden);
            g.Cb = L.dHin; g.ldcb = dk::kHidden; g.mask = L.Hin; g.ldm = dk::kHidden;
            if ((e = dk::launch_gemm_tc(g, s->err, st)) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t upload_params(Surrogate* s, const float* theta_host, cudaStream_t st) {
    const int P = s->P, kOffB4 = off_b4(s->K), kBfTotal = bf_total(s->K);
    cudaError_t e = cudaMemcpyAsync(s->d_theta, theta_host, sizeof(float) * P, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    std::vector<__nv_bfloat16> wb(kBfTotal);
    std::vector<int> idx(P, -1);
    for (int i = 0; i < P; ++i) {
        int j = -1;
        if (i < kOffB1) j = kBfW1 + i;
        else if (i >= kOffW2 && i < kOffB2) j = kBfW2 + (i - kOffW2);
        else if (i >= kOffW3 && i < kOffB3) j = kBfW3 + (i - kOffW3);
        else if (i >= kOffW4 && i < kOffB4) j = kBfW4 + (i - kOffW4);
        idx[i] = j;
        if (j >= 0) wb[j] = __float2bfloat16_rn(theta_host[i]);
    }
    if ((e = cudaMemcpyAsync(s->d_wbf, wb.data(), sizeof(__nv_bfloat16) * kBfTotal, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(s->d_bfidx, idx.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return e;
    return cudaStreamSynchronize(st);
}

dk::FeatArgs feat_args(mlmc_dk_ctx* c, int level_tag, int stream_tag, int64_t first, int64_t n, uint64_t seed,
                       __nv_bfloat16* X, float* Xf) {
    Surrogate* s = c->sur;
    dk::FeatArgs a{};
    a.E = s->d_E; a.g = s->d_g; a.inv_sigma = s->d_inv_sigma;
    a.n = s->n; a.M = s->M;
    a.key0 = (uint32_t)(seed & 0xffffffffu);
    a.key1 = (uint32_t)(seed >> 32);
    a.tag = ((uint32_t)level_tag & 0xffu) | (((uint32_t)stream_tag & 0xffu) << 8);
    a.first = first; a.count = n;
    a.X = X; a.Xf = Xf;
    return a;
}

int sur_fail(mlmc_dk_ctx* c, cudaError_t e, const char* what) { return cuda_fail(c, e, what); }

}  // namespace

extern "C" {

int mlmc_dk_surrogate_init(mlmc_dk_ctx* ctx, uint64_t seed) {
    if (!ctx) return fail(nullptr, MLMC_DK_ERR_INVALID, "null context");
    const LevelTab& l0 = ctx->lv[0];
    if (l0.n < 8 || l0.n > 32 || l0.streamed)
        return fail(ctx, MLMC_DK_ERR_UNSUPPORTED, "surrogate: level-0 grid must be 8^2..32^2");
    free_surrogate(ctx->sur);
    Surrogate* s = ctx->sur = new Surrogate();
    s->n = l0.n;
    s->M = l0.M;
    s->K = ctx->n_obs;
    s->products = ctx->products;
    s->P = param_count(s->K);
    s->sampw = 2 * ctx->n_obs + 2;
    s->batch_cap = 4096;
    const int kP = s->P, kBfTotal = bf_total(s->K), K = s->K;
    std::vector<float> E, g, isig;
    build_modes(l0.n, l0.tau / (l0.h * l0.h), l0.M, E, g, isig, ctx->b0);
    const size_t ch = (size_t)s->chunk;
    cudaError_t e;
    auto alloc = [&](void** p, size_t bytes) { return e == cudaSuccess ? (e = cudaMalloc(p, bytes)) : e; };
    e = cudaSuccess;
    alloc((void**)&s->d_E, sizeof(float) * E.size());
    alloc((void**)&s->d_g, sizeof(float) * g.size());
    alloc((void**)&s->d_inv_sigma, sizeof(float) * isig.size());
    alloc((void**)&s->d_theta, sizeof(float) * kP);
    alloc((void**)&s->d_grad, sizeof(float) * kP);
    alloc((void**)&s->d_m1, sizeof(float) * kP);
    alloc((void**)&s->d_m2, sizeof(float) * kP);
    alloc((void**)&s->d_wbf, sizeof(__nv_bfloat16) * kBfTotal);
    alloc((void**)&s->d_bfidx, sizeof(int) * kP);
    alloc((void**)&s->d_X, sizeof(__nv_bfloat16) * ch * dk::kFeat);
    alloc((void**)&s->d_Xf, sizeof(float) * ch * dk::kFeat);
    alloc((void**)&s->d_H1, sizeof(__nv_bfloat16) * ch * dk::kHidden);
    alloc((void**)&s->d_H2, sizeof(__nv_bfloat16) * ch * dk::kHidden);
    alloc((void**)&s->d_H3, sizeof(__nv_bfloat16) * ch * dk::kHidden);
    alloc((void**)&s->d_dH1, sizeof(__nv_bfloat16) * s->batch_cap * dk::kHidden);
    alloc((void**)&s->d_dH2, sizeof(__nv_bfloat16) * s->batch_cap * dk::kHidden);
    alloc((void**)&s->d_dH3, sizeof(__nv_bfloat16) * s->batch_cap * dk::kHidden);
    alloc((void**)&s->d_tA, sizeof(__nv_bfloat16) * (s->batch_cap + 8) * dk::kHidden);
    alloc((void**)&s->d_tB, sizeof(__nv_bfloat16) * (s->batch_cap + 8) * dk::kHidden);
    alloc((void**)&s->d_wt, sizeof(__nv_bfloat16) * dk::kHidden * dk::kHidden);
    s->err = ctx->d_err;
    alloc((void**)&s->d_y, sizeof(float) * ch * K);
    alloc((void**)&s->d_dy, sizeof(float) * s->batch_cap * K);
    alloc((void**)&s->d_T, sizeof(float) * ch * K);
    alloc((void**)&s->d_samp, sizeof(double) * ch * s->sampw);
    alloc((void**)&s->d_part, sizeof(double) * ctx->stride * kMomentBlocks);
    alloc((void**)&s->d_loss, sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(s->d_E, E.data(), sizeof(float) * E.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_g, g.data(), sizeof(float) * g.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_inv_sigma, isig.data(), sizeof(float) * isig.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_surrogate(s);
        ctx->sur = nullptr;
        return sur_fail(ctx, e, "surrogate buffers");
    }
    // He-uniform weights, zero biases, from a splitmix64 stream of `seed`
    std::vector<float> theta(kP, 0.f);
    uint64_t st = seed ^ 0x5deece66dull;
    auto uni = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) / 9007199254740992.0;
    };
    const int fan[4] = {dk::kFeat, dk::kHidden, dk::kHidden, dk::kHidden};
    const int offW[4] = {kOffW1, kOffW2, kOffW3, kOffW4};
    const int cnt[4] = {dk::kFeat * dk::kHidden, dk::kHidden * dk::kHidden, dk::kHidden * dk::kHidden, dk::kHidden * K};
    for (int l = 0; l < 4; ++l) {
        const double lim = std::sqrt(6.0 / fan[l]);
        for (int i = 0; i < cnt[l]; ++i) theta[offW[l] + i] = (float)((2.0 * uni() - 1.0) * lim * (l == 3 ? 0.1 : 1.0));
    }
    if ((e = upload_params(s, theta.data(), ctx->stream)) != cudaSuccess) return sur_fail(ctx, e, "surrogate params");
    return MLMC_DK_OK;
}

int mlmc_dk_surrogate_params(mlmc_dk_ctx* ctx, float* theta_out, const float* theta_in) {
    if (!ctx || !ctx->sur) return fail(ctx, MLMC_DK_ERR_INVALID, "surrogate not initialised");
    cudaError_t e;
    if (theta_in) {
        if ((e = upload_params(ctx->sur, theta_in, ctx->stream)) != cudaSuccess) return sur_fail(ctx, e, "set params");
        ctx->sur->adam_t = 0;
    }
    if (theta_out &&
        (e = cudaMemcpy(theta_out, ctx->sur->d_theta, sizeof(float) * ctx->sur->P, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return sur_fail(ctx, e, "get params");
    return MLMC_DK_OK;
}

int mlmc_dk_surrogate_info(const mlmc_dk_ctx* ctx, int32_t* n_params, int32_t* n_outputs) {
    if (!ctx || !ctx->sur) return fail(const_cast<mlmc_dk_ctx*>(ctx), MLMC_DK_ERR_INVALID, "surrogate not initialised");
    if (n_params) *n_params = ctx->sur->P;
    if (n_outputs) *n_outputs = ctx->sur->K;
    return MLMC_DK_OK;
}

int mlmc_dk_surrogate_features(mlmc_dk_ctx* ctx, int32_t direct, int32_t stream_tag, int64_t first, int64_t n,
                               uint64_t seed, float* X_host) {
    if (!ctx || !ctx->sur || n < 0 || n > ctx->sur->chunk || !X_host)
        return fail(ctx, MLMC_DK_ERR_INVALID, "surrogate_features: bad arguments");
    Surrogate* s = ctx->sur;
    dk::FeatArgs a = feat_args(ctx, direct ? 0 : 1, stream_tag, first, n, seed, s->d_X, s->d_Xf);
    cudaError_t e = direct ? dk::launch_direct_features(a, ctx->stream)
                           : dk::launch_features(a, 152 * 8, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(X_host, s->d_Xf, sizeof(float) * n * dk::kFeat, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? MLMC_DK_OK : sur_fail(ctx, e, "surrogate features");
}

int mlmc_dk_surrogate_forward(mlmc_dk_ctx* ctx, const float* X_host, int64_t n, float* y_host) {
    if (!ctx || !ctx->sur || n < 1 || n > ctx->sur->chunk || !X_host || !y_host)
        return fail(ctx, MLMC_DK_ERR_INVALID, "surrogate_forward: bad arguments");
    Surrogate* s = ctx->sur;
    std::vector<__nv_bfloat16> xb((size_t)n * dk::kFeat);
    for (size_t i = 0; i < xb.size(); ++i) xb[i] = __float2bfloat16_rn(X_host[i]);
    cudaError_t e = cudaMemcpy(s->d_X, xb.data(), sizeof(__nv_bfloat16) * xb.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = mlp_forward(s, s->d_X, (int)n, s->d_y, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(y_host, s->d_y, sizeof(float) * n * s->K, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? MLMC_DK_OK : sur_fail(ctx, e, "surrogate forward");
}

int mlmc_dk_surrogate_loss_grad(mlmc_dk_ctx* ctx, const float* X_host, const float* T_host, int32_t B, double* loss,
                                float* grad_host) {
    if (!ctx || !ctx->sur || B < 1 || B > ctx->sur->batch_cap || !X_host || !T_host)
        return fail(ctx, MLMC_DK_ERR_INVALID, "surrogate_loss_grad: bad arguments");
    Surrogate* s = ctx->sur;
    std::vector<__nv_bfloat16> xb((size_t)B * dk::kFeat);
    for (size_t i = 0; i < xb.size(); ++i) xb[i] = __float2bfloat16_rn(X_host[i]);
    cudaError_t e = cudaMemcpy(s->d_X, xb.data(), sizeof(__nv_bfloat16) * xb.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_T, T_host, sizeof(float) * B * s->K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = mlp_forward(s, s->d_X, B, s->d_y, ctx->stream);
    if (e == cudaSuccess) e = dk::launch_mse(s->d_y, s->d_T, B * s->K, B, s->d_loss, ctx->stream);
    if (e == cudaSuccess) e = mlp_backward(s, s->d_X, s->d_T, B, ctx->stream);
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, s->d_loss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && grad_host)
        e = cudaMemcpyAsync(grad_host, s->d_grad, sizeof(float) * s->P, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? MLMC_DK_OK : sur_fail(ctx, e, "surrogate loss/grad");
}

int mlmc_dk_surrogate_train(mlmc_dk_ctx* ctx, int64_t n_pairs, int32_t epochs, int32_t batch, double lr, uint64_t seed,
                            double* train_mse, double* val_mse, double* seconds) {
    if (!ctx || !ctx->sur || n_pairs < 2 * batch || epochs < 1 || batch < 64 || batch > ctx->sur->batch_cap ||
        batch % 64 || !(lr > 0))
        return fail(ctx, MLMC_DK_ERR_INVALID, "surrogate_train: bad arguments");
    const auto t0 = std::chrono::steady_clock::now();
    Surrogate* s = ctx->sur;
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaSuccess;
    const int K = s->K, W = s->sampw, kP = s->P;
    if (s->n_train != n_pairs) {
        cudaFree(s->d_trainX);
        cudaFree(s->d_trainT);
        cudaFree(s->d_idx);
        s->d_trainX = nullptr; s->d_trainT = nullptr; s->d_idx = nullptr;
        if ((e = cudaMalloc(&s->d_trainX, sizeof(__nv_bfloat16) * n_pairs * dk::kFeat)) != cudaSuccess ||
            (e = cudaMalloc(&s->d_trainT, sizeof(float) * n_pairs * K)) != cudaSuccess ||
            (e = cudaMalloc(&s->d_idx, sizeof(int) * n_pairs)) != cudaSuccess)
            return sur_fail(ctx, e, "training buffers");
        s->n_train = n_pairs;
    }
    // training pairs: level-0 paths of the training stream (3) and their features
    std::vector<double> hs;
    std::vector<float> ht;
    const double sqrtN = std::sqrt(ctx->N);
    for (int64_t done = 0; done < n_pairs; done += s->chunk) {
        const int64_t n = std::min<int64_t>(s->chunk, n_pairs - done);
        int rc = launch_batch(ctx, 0, 3, done, n, seed, ctx->d_sums, s->d_samp, st);
        if (rc != MLMC_DK_OK) return rc;
        dk::FeatArgs a = feat_args(ctx, 1, 3, done, n, seed, s->d_trainX + done * dk::kFeat, nullptr);
        if ((e = dk::launch_features(a, 152 * 8, st)) != cudaSuccess) return sur_fail(ctx, e, "features");
        hs.resize((size_t)n * W);
        if ((e = cudaMemcpyAsync(hs.data(), s->d_samp, sizeof(double) * n * W, cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return sur_fail(ctx, e, "training targets");
        ht.resize((size_t)n * K);
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < K; ++k)
                ht[(size_t)i * K + k] = (float)(sqrtN * hs[(size_t)i * W + k]);   // sqrt(N) (Y_0k - Ybar_0k)
        if ((e = cudaMemcpy(s->d_trainT + done * K, ht.data(), sizeof(float) * n * K, cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            return sur_fail(ctx, e, "training targets");
    }
    // last 1/16 held out for validation
    const int64_t n_val = std::max<int64_t>(batch, n_pairs / 16);
    const int64_t n_fit = (n_pairs - n_val) / batch * batch;
    std::vector<int> idx(n_fit);
    std::iota(idx.begin(), idx.end(), 0);
    std::mt19937_64 rng(seed ^ 0x7261696eull);
    if ((e = cudaMemsetAsync(s->d_m1, 0, sizeof(float) * kP, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(s->d_m2, 0, sizeof(float) * kP, st)) != cudaSuccess)
        return sur_fail(ctx, e, "adam state");
    s->adam_t = 0;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    double last_loss = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(idx.begin(), idx.end(), rng);
        if ((e = cudaMemcpyAsync(s->d_idx, idx.data(), sizeof(int) * n_fit, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return sur_fail(ctx, e, "shuffle");
        // cosine-decayed step size over the epochs
        const double lr_ep = lr * 0.5 * (1.0 + std::cos(M_PI * ep / (double)epochs));
        for (int64_t b0 = 0; b0 < n_fit; b0 += batch) {
            if ((e = dk::launch_gather(s->d_trainX, s->d_trainT, s->d_idx + b0, batch, K, s->d_X, s->d_T, st)) !=
                    cudaSuccess ||
                (e = mlp_forward(s, s->d_X, batch, s->d_y, st)) != cudaSuccess ||
                (e = mlp_backward(s, s->d_X, s->d_T, batch, st)) != cudaSuccess)
                return sur_fail(ctx, e, "training step");
            ++s->adam_t;
            const float c1 = 1.f - std::pow(b1, (float)s->adam_t), c2 = 1.f - std::pow(b2, (float)s->adam_t);
            if ((e = dk::launch_adam(s->d_theta, s->d_grad, s->d_m1, s->d_m2, kP, (float)lr_ep, b1, b2, eps, c1, c2,
                                     s->d_bfidx, s->d_wbf, st)) != cudaSuccess)
                return sur_fail(ctx, e, "adam");
        }
        if (ep == epochs - 1 && train_mse) {
            // mean-squared error of the last batch's predictions (before its update)
            if ((e = dk::launch_mse(s->d_y, s->d_T, batch * K, batch, s->d_loss, st)) != cudaSuccess ||
                (e = cudaMemcpyAsync(&last_loss, s->d_loss, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess)
                return sur_fail(ctx, e, "train loss");
        }
    }
    if (train_mse) *train_mse = last_loss;
    if (val_mse) {
        double acc = 0.0;
        int64_t cnt = 0;
        for (int64_t v0 = n_pairs - n_val; v0 < n_pairs; v0 += s->chunk) {
            const int64_t n = std::min<int64_t>(s->chunk, n_pairs - v0);
            double l = 0.0;
            if ((e = mlp_forward(s, s->d_trainX + v0 * dk::kFeat, (int)n, s->d_y, st)) != cudaSuccess ||
                (e = dk::launch_mse(s->d_y, s->d_trainT + v0 * K, (int)n * K, (int)n, s->d_loss, st)) != cudaSuccess ||
                (e = cudaMemcpyAsync(&l, s->d_loss, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess)
                return sur_fail(ctx, e, "validation");
            acc += l * n;
            cnt += n;
        }
        *val_mse = acc / cnt;
    }
    if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return check_device_error(ctx);
}

int mlmc_dk_run_surrogate(mlmc_dk_ctx* ctx, int32_t part, int64_t n_samples, uint64_t seed, mlmc_dk_level_sums* sums) {
    if (!ctx || !ctx->sur || (part != -1 && part != 0) || n_samples < 0 || !sums)
        return fail(ctx, MLMC_DK_ERR_INVALID, "run_surrogate: bad arguments");
    Surrogate* s = ctx->sur;
    cudaStream_t st = ctx->stream;
    cudaError_t e;
    int64_t& next = s->next_id[part == -1 ? 0 : 1];
    const auto t0 = std::chrono::steady_clock::now();
    for (int64_t done = 0; done < n_samples; done += s->chunk) {
        const int64_t n = std::min<int64_t>(s->chunk, n_samples - done);
        const int64_t first = next + done;
        if ((e = cudaEventRecord(ctx->ev0, st)) != cudaSuccess) return sur_fail(ctx, e, "event");
        if (part == -1) {
            // level below 0: standardised features drawn from their exact law (stream 2, level tag 0)
            dk::FeatArgs a = feat_args(ctx, 0, 2, first, n, seed, s->d_X, nullptr);
            if ((e = dk::launch_direct_features(a, st)) != cudaSuccess) return sur_fail(ctx, e, "direct features");
        } else {
            // correction level: the level-0 paths of the coupled stream and their own features
            int rc = launch_batch(ctx, 0, 0, first, n, seed, ctx->d_sums, s->d_samp, st);
            if (rc != MLMC_DK_OK) return rc;
            dk::FeatArgs a = feat_args(ctx, 1, 0, first, n, seed, s->d_X, nullptr);
            if ((e = dk::launch_features(a, 152 * 8, st)) != cudaSuccess) return sur_fail(ctx, e, "features");
        }
        if ((e = mlp_forward(s, s->d_X, (int)n, s->d_y, st)) != cudaSuccess ||
            (e = dk::launch_surrogate_moments(s->d_y, s->d_samp, s->sampw, part, ctx->N, n, ctx->stride, s->K,
                                              s->products, kMomentBlocks, s->d_part, st)) != cudaSuccess ||
            (e = dk::launch_reduce(s->d_part, kMomentBlocks, ctx->stride, ctx->d_sums, st)) != cudaSuccess ||
            (e = cudaEventRecord(ctx->ev1, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(ctx->h_sums, ctx->d_sums, sizeof(double) * ctx->stride, cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return sur_fail(ctx, e, "surrogate level");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        const double cost = part == -1 ? 0.0 : (double)ctx->lv[0].n * ctx->lv[0].n * ctx->lv[0].M;
        accumulate(ctx, ctx->h_sums, sums, cost, 0.0, 1e-3 * ms, part == -1 ? 6 : 8);
    }
    next += n_samples;
    const double wall = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    sums[0].wall_s += wall;
    return check_device_error(ctx);
}

int mlmc_dk_estimate_surrogate(mlmc_dk_ctx* ctx, double eps, int32_t relative, uint64_t seed, mlmc_dk_result* out,
                               mlmc_dk_level_sums* sur_out) {
    if (!ctx || !ctx->sur || !out || !(eps > 0)) return fail(ctx, MLMC_DK_ERR_INVALID, "estimate_surrogate: bad arguments");
    const auto t0 = std::chrono::steady_clock::now();
    *out = mlmc_dk_result{};
    // virtual levels: 0 = level below 0 (S), 1 = correction (P_0 - S), 1 + l = level l >= 1
    const int VL = ctx->L_max + 2, Q = ctx->n_quant;
    std::vector<mlmc_dk_level_sums> all((size_t)VL * Q);   // [virtual level][quantity]
    auto sums = [&](int v) -> mlmc_dk_level_sums& { return all[(size_t)v * Q]; };   // the first quantity
    std::vector<int64_t> target(VL, 0);
    std::fill(ctx->next_id[0].begin(), ctx->next_id[0].end(), 0);
    ctx->sur->next_id[0] = ctx->sur->next_id[1] = 0;
    int L = ctx->L_start;
    for (int v = 0; v <= L + 1; ++v) target[v] = ctx->pilot;
    double eps_abs = relative ? -1.0 : eps;
    int status = MLMC_DK_OK, converged = 0;
    auto run = [&](int v, int64_t n) -> int {
        if (v <= 1) return mlmc_dk_run_surrogate(ctx, v == 0 ? -1 : 0, n, seed, &sums(v));
        return mlmc_dk_run_level(ctx, v - 1, n, seed, &sums(v));
    };
    for (int iter = 0; iter < 1000; ++iter) {
        for (int v = 0; v <= L + 1; ++v) {
            const int64_t need = target[v] - sums(v).n;
            if (need > 0) {
                const int rc = run(v, need);
                if (rc != MLMC_DK_OK) return rc;
            }
        }
        std::vector<double> E(L + 2), V(L + 2), C(L + 2);
        for (int v = 0; v <= L + 1; ++v) {
            const double m = (double)sums(v).n;
            E[v] = sums(v).dp1 / m;
            V[v] = std::max(0.0, (sums(v).dp2 - sums(v).dp1 * sums(v).dp1 / m) / (m - 1.0));
            C[v] = std::max(sums(v).kernel_s / m, 1e-12);   // measured device seconds per sample
        }
        if (eps_abs < 0) {
            double mu = 0;
            for (double x : E) mu += x;
            eps_abs = eps * std::fabs(mu);
            if (!(eps_abs > 0)) return fail(ctx, MLMC_DK_ERR_INVALID, "relative eps with a zero pilot estimate");
        }
        double total = 0;
        for (int v = 0; v <= L + 1; ++v) total += std::sqrt(V[v] * C[v]);
        bool more = false;
        for (int v = 0; v <= L + 1; ++v) {
            const double opt = std::ceil(2.0 / (eps_abs * eps_abs) * std::sqrt(V[v] / C[v]) * total);
            target[v] = std::max(target[v], (int64_t)std::min(opt, 9.0e18));
            if ((double)(target[v] - sums(v).n) > 0.01 * (double)sums(v).n) more = true;
        }
        if (more) continue;
        // stopping test on the level differences of the plain hierarchy (level 0 = S + (P_0 - S))
        double worst = 0;
        for (int t = 0; t <= 2 && L - t >= 0; ++t) {
            const int l = L - t;
            const double el = l == 0 ? E[0] + E[1] : E[l + 1];
            worst = std::max(worst, std::pow(4.0, -t) * std::fabs(el));
        }
        if (worst / 3.0 < eps_abs / std::sqrt(2.0)) { converged = 1; break; }
        if (L == ctx->L_max) { status = MLMC_DK_NOT_CONVERGED; break; }
        ++L;
        target[L + 1] = ctx->pilot;
    }
    out->L = L;
    out->converged = converged;
    out->eps_abs = eps_abs;
    double est = 0.0;
    for (int v = 0; v <= L + 1; ++v) {
        const mlmc_dk_level_sums& q = sums(v);
        const double m = (double)q.n;
        const double Vv = std::max(0.0, (q.dp2 - q.dp1 * q.dp1 / m) / (m - 1.0));
        est += q.dp1 / m;
        out->variance += Vv / m;
        out->cell_steps += q.cost;
        if (v >= 1) {
            const int l = v - 1;
            out->M[l] = q.n;
            out->E[l] = q.dp1 / m;
            out->V[l] = Vv;
            out->C[l] = q.kernel_s / m;
            out->kernel_s[l] = q.kernel_s;
            out->sample_steps += m * ctx->lv[l].M;
            out->var_pf[l] = std::max(0.0, (q.pf2 - q.pf1 * q.pf1 / m) / (m - 1.0));
        }
        out->launches += q.launches;
        out->d2h_bytes += q.d2h_bytes;
    }
    out->estimate = est;
    for (int q = 0; q < Q && q < MLMC_DK_MAX_QUANT; ++q) {
        double e = 0.0;
        for (int v = 0; v <= L + 1; ++v) e += all[(size_t)v * Q + q].dp1 / (double)all[(size_t)v * Q + q].n;
        out->estimates[q] = e;
    }
    if (sur_out) *sur_out = sums(0);
    out->wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return status;
}

}  // extern "C"
