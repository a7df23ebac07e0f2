/*
 * FP64 oracle for the coupled Dean--Kawasaki MLMC hot path (see dk_oracle.h).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the
 * CPU legs of bench.py; never by the product path.  Plain, slow, obviously
 * correct: every array is double, every step is written out as the paper
 * states it, nothing is fused or reordered.
 */
#include "dk_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ Philox */
/* Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3" (SC'11): ten rounds, each multiplying
 * words 0 and 2 by the two round multipliers, xoring the high halves with the
 * other two words and the round key, and swapping; the key is advanced by the
 * two Weyl constants between rounds. */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ----------------------------------------------------------------- normals */
static void box_muller(uint32_t a, uint32_t b, double* z1, double* z2)
{
    const double two32 = 4294967296.0;
    double u = ((double)a + 1.0) / two32;            /* in (0, 1] */
    double theta = 2.0 * M_PI * ((double)b + 0.5) / two32;
    double radius = sqrt(-2.0 * log(u));
    *z1 = radius * cos(theta);
    *z2 = radius * sin(theta);
}

void oracle_normals(uint64_t seed, int level, int stream, uint64_t sample, int64_t m,
                    int n, double* Z)
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t tag = ((uint32_t)(level + 1) & 0xffu) | (((uint32_t)stream & 0xffu) << 8) |
                   ((uint32_t)((sample >> 32) & 0xffffu) << 16);
    int64_t cells = (int64_t)n * n;
    for (int64_t p = 0; p < cells / 2; ++p) {
        uint32_t ctr[4] = {(uint32_t)p, (uint32_t)m, (uint32_t)(sample & 0xffffffffu), tag};
        uint32_t x[4];
        oracle_philox4x32_10(ctr, key, x);
        box_muller(x[0], x[1], &Z[(2 * p) * 2 + 0], &Z[(2 * p) * 2 + 1]);
        box_muller(x[2], x[3], &Z[(2 * p + 1) * 2 + 0], &Z[(2 * p + 1) * 2 + 1]);
    }
}

/* -------------------------------------------------------------------- step */
static inline int wrap(int i, int n) { return (i % n + n) % n; }

/* rho + w tau/2 Delta_h rho + inv_sqrt_N div_h(F): the explicit right-hand
 * side of Eq. (FullyDiscreteDK) with diffusion weight w (w = b1). */
static void explicit_part(int n, double h, double tau, double w, double inv_sqrt_N,
                          const double* rho, const double* dbeta, double* out)
{
    const int d = 2;
    const double h_pow = pow(h, -0.5 * d);   /* h^{-d/2}: grid white-noise basis scale */
    /* Flux field F_r(y) = h^{-d/2} sqrt([rho(y)]^+) dbeta_(y,r). */
    double* F = NULL;
    if (inv_sqrt_N != 0.0) {
        F = (double*)malloc(sizeof(double) * (size_t)n * n * 2);
        for (int y = 0; y < n * n; ++y) {
            double pos = rho[y] > 0.0 ? rho[y] : 0.0;
            F[2 * y + 0] = h_pow * sqrt(pos) * dbeta[2 * y + 0];
            F[2 * y + 1] = h_pow * sqrt(pos) * dbeta[2 * y + 1];
        }
    }
    for (int i1 = 0; i1 < n; ++i1) {
        for (int i2 = 0; i2 < n; ++i2) {
            int x = i1 * n + i2;
            int up = wrap(i1 - 1, n) * n + i2, down = wrap(i1 + 1, n) * n + i2;
            int left = i1 * n + wrap(i2 - 1, n), right = i1 * n + wrap(i2 + 1, n);
            /* Delta_h a(x) = (-4 a(x) + sum_{y~x} a(y)) / h^2 */
            double lap = (-4.0 * rho[x] + rho[up] + rho[down] + rho[left] + rho[right]) / (h * h);
            double value = rho[x] + w * tau * 0.5 * lap;
            if (F) {
                /* nabla_h . b(x) = sum_r ([b]_r(x + h f_r) - [b]_r(x - h f_r)) / (2h) */
                double div = (F[2 * down + 0] - F[2 * up + 0]) / (2.0 * h) +
                             (F[2 * right + 1] - F[2 * left + 1]) / (2.0 * h);
                value += inv_sqrt_N * div;
            }
            out[x] = value;
        }
    }
    free(F);
}

void oracle_dk_step(int n, double h, double tau, double inv_sqrt_N,
                    const double* rho, const double* dbeta, double* out)
{
    explicit_part(n, h, tau, 1.0, inv_sqrt_N, rho, dbeta, out);
}

/* Separable discrete Fourier transform of an n x n array held as (re, im):
 * a(k) = sum_x a(x) exp(sign 2 pi i k.x / n), along i2 for every row and then
 * along i1 for every column; cs/sn hold cos/sin(2 pi j / n). */
static void dft2(int n, int sign, const double* cs, const double* sn, double* re, double* im)
{
    double* tr = (double*)malloc(sizeof(double) * (size_t)n);
    double* ti = (double*)malloc(sizeof(double) * (size_t)n);
    for (int axis = 0; axis < 2; ++axis) {
        for (int line = 0; line < n; ++line) {
            /* element j of this line sits at base + j * step */
            const int base = axis == 0 ? line * n : line, step = axis == 0 ? 1 : n;
            for (int k = 0; k < n; ++k) {
                double sr = 0.0, si = 0.0;
                for (int j = 0; j < n; ++j) {
                    const int t = (int)(((int64_t)k * j) % n);
                    const double c = cs[t], s = sign * sn[t];
                    const double ar = re[base + j * step], ai = im[base + j * step];
                    sr += ar * c - ai * s;
                    si += ar * s + ai * c;
                }
                tr[k] = sr;
                ti[k] = si;
            }
            for (int k = 0; k < n; ++k) {
                re[base + k * step] = tr[k];
                im[base + k * step] = ti[k];
            }
        }
    }
    free(tr);
    free(ti);
}

void oracle_helmholtz_solve(int n, double c, const double* rhs, double* out)
{
    /* Every mode exp(2 pi i k.x / n) is an eigenvector of L with eigenvalue
     * 4 (sin^2(pi k1/n) + sin^2(pi k2/n)): transform, divide, transform back. */
    const size_t cells = (size_t)n * n;
    double* re = (double*)malloc(sizeof(double) * cells);
    double* im = (double*)calloc(cells, sizeof(double));
    double* cs = (double*)malloc(sizeof(double) * (size_t)n);
    double* sn = (double*)malloc(sizeof(double) * (size_t)n);
    for (int j = 0; j < n; ++j) {
        cs[j] = cos(2.0 * M_PI * j / n);
        sn[j] = sin(2.0 * M_PI * j / n);
    }
    memcpy(re, rhs, sizeof(double) * cells);
    dft2(n, -1, cs, sn, re, im);
    for (int k1 = 0; k1 < n; ++k1)
        for (int k2 = 0; k2 < n; ++k2) {
            const double s1 = sin(M_PI * k1 / n), s2 = sin(M_PI * k2 / n);
            const double lam = 4.0 * (s1 * s1 + s2 * s2);
            re[k1 * n + k2] /= 1.0 + c * lam;
            im[k1 * n + k2] /= 1.0 + c * lam;
        }
    dft2(n, +1, cs, sn, re, im);
    for (size_t x = 0; x < cells; ++x) out[x] = re[x] / (double)cells;
    free(re); free(im); free(cs); free(sn);
}

void oracle_theta_step(int n, double h, double tau, double inv_sqrt_N, double b0,
                       const double* rho, const double* dbeta, double* out)
{
    const double b1 = 1.0 - b0;
    if (b0 == 0.0) {
        explicit_part(n, h, tau, 1.0, inv_sqrt_N, rho, dbeta, out);
        return;
    }
    double* rhs = (double*)malloc(sizeof(double) * (size_t)n * n);
    explicit_part(n, h, tau, b1, inv_sqrt_N, rho, dbeta, rhs);
    /* I - b0 tau/2 Delta_h = I + c L with c = b0 tau / (2 h^2) */
    oracle_helmholtz_solve(n, b0 * tau / (2.0 * h * h), rhs, out);
    free(rhs);
}

void oracle_mean_field_theta(int n, double h, double tau, int64_t M, double b0, const double* rho0,
                             double* out)
{
    double* a = (double*)malloc(sizeof(double) * (size_t)n * n);
    double* b = (double*)malloc(sizeof(double) * (size_t)n * n);
    memcpy(a, rho0, sizeof(double) * (size_t)n * n);
    for (int64_t m = 0; m < M; ++m) {
        oracle_theta_step(n, h, tau, 0.0, b0, a, NULL, b);
        double* t = a; a = b; b = t;
    }
    memcpy(out, a, sizeof(double) * (size_t)n * n);
    free(a);
    free(b);
}

void oracle_mean_field(int n, double h, double tau, int64_t M, const double* rho0, double* out)
{
    double* a = (double*)malloc(sizeof(double) * (size_t)n * n);
    double* b = (double*)malloc(sizeof(double) * (size_t)n * n);
    memcpy(a, rho0, sizeof(double) * (size_t)n * n);
    for (int64_t m = 0; m < M; ++m) {
        oracle_dk_step(n, h, tau, 0.0, a, NULL, b);
        double* t = a; a = b; b = t;
    }
    memcpy(out, a, sizeof(double) * (size_t)n * n);
    free(a);
    free(b);
}

/* ------------------------------------------------------------------ sample */
static double inner_h(int n, double h, const double* f, const double* g)
{
    /* (f, g)_h = h^d sum_x f(x) g(x) */
    double s = 0.0;
    for (int x = 0; x < n * n; ++x) s += f[x] * g[x];
    return h * h * s;
}

/* splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the perturbation stream of oracle_sample_perturbed. */
static uint64_t splitmix64(uint64_t* state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Edge (x, x + h e_r) moves e_r(x), uniform in [-amp/2, amp/2), from cell
 * x + h e_r to cell x; transfers (optional, [n*n][2]) receives e_1, e_2. */
static void perturb_edges(int n, double amp, uint64_t* state, double* rho, double* transfers)
{
    for (int i1 = 0; i1 < n; ++i1)
        for (int i2 = 0; i2 < n; ++i2) {
            int x = i1 * n + i2;
            int down = wrap(i1 + 1, n) * n + i2, right = i1 * n + wrap(i2 + 1, n);
            double e1 = ((double)(splitmix64(state) >> 11) / 9007199254740992.0 - 0.5) * amp;
            double e2 = ((double)(splitmix64(state) >> 11) / 9007199254740992.0 - 0.5) * amp;
            rho[x] += e1 + e2;
            rho[down] -= e1;
            rho[right] -= e2;
            if (transfers) {
                transfers[2 * x + 0] = e1;
                transfers[2 * x + 1] = e2;
            }
        }
}

void oracle_perturb_field(int n, double amp, uint64_t perturb_seed, double* rho, double* transfers)
{
    uint64_t state = perturb_seed;
    perturb_edges(n, amp, &state, rho, transfers);
}

void oracle_fourier_restrict(int n, int nc, const double* fine, double* coarse)
{
    /* unitary DFT of the fine field on the kept modes (separable sums: along
     * x2 for every row, then along x1), weights, inverse DFT on the coarse grid */
    const int K = nc / 2;
    const int J = 2 * K + 1;   /* modes -K..K per axis */
    double* cs = (double*)malloc(sizeof(double) * (size_t)n);
    double* sn = (double*)malloc(sizeof(double) * (size_t)n);
    for (int j = 0; j < n; ++j) {
        cs[j] = cos(2.0 * M_PI * j / n);
        sn[j] = sin(2.0 * M_PI * j / n);
    }
    /* row transforms: t(x1, xi2) = sum_x2 f(x1, x2) exp(-2 pi i xi2 x2 / n) */
    double* tre = (double*)malloc(sizeof(double) * (size_t)n * J);
    double* tim = (double*)malloc(sizeof(double) * (size_t)n * J);
    for (int x1 = 0; x1 < n; ++x1)
        for (int b = 0; b < J; ++b) {
            double sr = 0.0, si = 0.0;
            for (int x2 = 0; x2 < n; ++x2) {
                const int t = (int)((((int64_t)(b - K) * x2) % n + n) % n);
                sr += fine[x1 * n + x2] * cs[t];
                si -= fine[x1 * n + x2] * sn[t];
            }
            tre[x1 * J + b] = sr;
            tim[x1 * J + b] = si;
        }
    /* column transforms and weights: c(xi1, xi2) */
    double* cre = (double*)malloc(sizeof(double) * (size_t)J * J);
    double* cim = (double*)malloc(sizeof(double) * (size_t)J * J);
    for (int a = 0; a < J; ++a)
        for (int b = 0; b < J; ++b) {
            double sr = 0.0, si = 0.0;
            for (int x1 = 0; x1 < n; ++x1) {
                const int t = (int)((((int64_t)(a - K) * x1) % n + n) % n);
                /* (tre + i tim) (cos - i sin) */
                sr += tre[x1 * J + b] * cs[t] + tim[x1 * J + b] * sn[t];
                si += tim[x1 * J + b] * cs[t] - tre[x1 * J + b] * sn[t];
            }
            const double w = ((a == 0 || a == J - 1) ? M_SQRT1_2 : 1.0) * ((b == 0 || b == J - 1) ? M_SQRT1_2 : 1.0);
            cre[a * J + b] = w * sr / n;
            cim[a * J + b] = w * si / n;
        }
    /* inverse on the coarse grid, real part: g(y) = nc^-1 sum c(xi) exp(2 pi i xi.y / nc) */
    double* ccs = (double*)malloc(sizeof(double) * (size_t)nc);
    double* csn = (double*)malloc(sizeof(double) * (size_t)nc);
    for (int j = 0; j < nc; ++j) {
        ccs[j] = cos(2.0 * M_PI * j / nc);
        csn[j] = sin(2.0 * M_PI * j / nc);
    }
    for (int y1 = 0; y1 < nc; ++y1)
        for (int y2 = 0; y2 < nc; ++y2) {
            double g = 0.0;
            for (int a = 0; a < J; ++a)
                for (int b = 0; b < J; ++b) {
                    const int t = (int)((((int64_t)(a - K) * y1 + (int64_t)(b - K) * y2) % nc + nc) % nc);
                    g += cre[a * J + b] * ccs[t] - cim[a * J + b] * csn[t];
                }
            coarse[y1 * nc + y2] = g / nc;
        }
    free(cs); free(sn); free(ccs); free(csn); free(tre); free(tim); free(cre); free(cim);
}

static int sample_impl(const oracle_level* lv, uint64_t seed, int stream, uint64_t sample,
                       int coupled, double amp, uint64_t perturb_seed, const double* given,
                       double* Y_f, double* Y_c, double* mass_f, double* mass_c,
                       double* rho_f_out, double* rho_c_out)
{
    uint64_t pstate = perturb_seed;
    const int fourier = lv->coupling == 1;
    const int ratio = fourier ? 3 : 2, kappa = ratio * ratio;   /* h and tau ratios (Eq. cfl_preserved) */
    const int n = lv->n, nc = n / ratio;
    if (n < 2 || (n & 1)) return -1;
    if (coupled && ((lv->M % kappa) != 0 || n % ratio != 0 || (nc & 1))) return -2;
    const size_t cf = (size_t)n * n, cc = (size_t)nc * nc;
    double* rho_f = (double*)malloc(sizeof(double) * cf);
    double* tmp_f = (double*)malloc(sizeof(double) * cf);
    double* Z = (double*)malloc(sizeof(double) * cf * 2);
    double* dbeta_f = (double*)malloc(sizeof(double) * cf * 2);
    double* rho_c = NULL, *tmp_c = NULL, *dbeta_c = NULL, *sum_f = NULL, *comp_f = NULL, *comp_c = NULL;
    memcpy(rho_f, lv->rho0_f, sizeof(double) * cf);
    if (coupled) {
        rho_c = (double*)malloc(sizeof(double) * cc);
        tmp_c = (double*)malloc(sizeof(double) * cc);
        dbeta_c = (double*)calloc(cc * 2, sizeof(double));
        memcpy(rho_c, lv->rho0_c, sizeof(double) * cc);
        if (fourier) {
            sum_f = (double*)calloc(cf * 2, sizeof(double));
            comp_f = (double*)malloc(sizeof(double) * cf);
            comp_c = (double*)malloc(sizeof(double) * cc);
        }
    }
    const double sqrt_tau = sqrt(lv->tau);
    const double block_weight = pow(2.0, -0.5 * 2);   /* 2^{-d/2} of the NN coupling */
    for (int64_t m = 0; m < lv->M; ++m) {
        if (given)
            memcpy(Z, given + (size_t)m * cf * 2, sizeof(double) * cf * 2);
        else
            oracle_normals(seed, lv->level, stream, sample, m, n, Z);
        for (size_t i = 0; i < cf * 2; ++i) dbeta_f[i] = sqrt_tau * Z[i];
        if (coupled && fourier) {
            /* Fourier coupling: the coarse increment over one coarse step carries the
             * modes of the sum of the kappa_t = 9 fine increments inside it */
            for (size_t i = 0; i < cf * 2; ++i) sum_f[i] += dbeta_f[i];
        } else if (coupled) {
            /* beta-tilde_(y,r) = 2^{-d/2} sum_{z in B->(y)} beta_(z,r), B->(y) = {y + h v}:
             * fine cells (2 I1 + v1, 2 I2 + v2).  The coarse increment over one coarse
             * step is the sum of the kappa_t = 4 fine increments inside it. */
            for (int i1 = 0; i1 < n; ++i1)
                for (int i2 = 0; i2 < n; ++i2) {
                    int z = i1 * n + i2, y = (i1 / 2) * nc + (i2 / 2);
                    dbeta_c[2 * y + 0] += block_weight * dbeta_f[2 * z + 0];
                    dbeta_c[2 * y + 1] += block_weight * dbeta_f[2 * z + 1];
                }
        }
        oracle_theta_step(n, lv->h, lv->tau, lv->inv_sqrt_N, lv->b0, rho_f, dbeta_f, tmp_f);
        double* t = rho_f; rho_f = tmp_f; tmp_f = t;
        if (amp > 0.0) perturb_edges(n, amp, &pstate, rho_f, NULL);
        if (coupled && (m % kappa) == kappa - 1) {
            if (fourier) {
                for (int r = 0; r < 2; ++r) {
                    for (size_t i = 0; i < cf; ++i) comp_f[i] = sum_f[2 * i + r];
                    oracle_fourier_restrict(n, nc, comp_f, comp_c);
                    for (size_t i = 0; i < cc; ++i) dbeta_c[2 * i + r] = comp_c[i];
                }
                memset(sum_f, 0, sizeof(double) * cf * 2);
            }
            oracle_theta_step(nc, ratio * lv->h, kappa * lv->tau, lv->inv_sqrt_N, lv->b0, rho_c, dbeta_c, tmp_c);
            double* tc = rho_c; rho_c = tmp_c; tmp_c = tc;
            memset(dbeta_c, 0, sizeof(double) * cc * 2);
            if (amp > 0.0) perturb_edges(nc, amp, &pstate, rho_c, NULL);
        }
    }
    double* ones = (double*)malloc(sizeof(double) * cf);
    for (size_t i = 0; i < cf; ++i) ones[i] = 1.0;
    for (int k = 0; k < lv->n_obs; ++k) Y_f[k] = inner_h(n, lv->h, rho_f, lv->phi_f + (size_t)k * cf);
    if (mass_f) *mass_f = inner_h(n, lv->h, rho_f, ones);
    if (rho_f_out) memcpy(rho_f_out, rho_f, sizeof(double) * cf);
    if (coupled) {
        for (int k = 0; k < lv->n_obs; ++k)
            Y_c[k] = inner_h(nc, ratio * lv->h, rho_c, lv->phi_c + (size_t)k * cc);
        if (mass_c) *mass_c = inner_h(nc, ratio * lv->h, rho_c, ones);
        if (rho_c_out) memcpy(rho_c_out, rho_c, sizeof(double) * cc);
    }
    free(ones);
    free(rho_f); free(tmp_f); free(Z); free(dbeta_f);
    free(rho_c); free(tmp_c); free(dbeta_c);
    free(sum_f); free(comp_f); free(comp_c);
    return 0;
}

int oracle_sample(const oracle_level* lv, uint64_t seed, int stream, uint64_t sample,
                  int coupled, double* Y_f, double* Y_c, double* mass_f, double* mass_c,
                  double* rho_f_out, double* rho_c_out)
{
    return sample_impl(lv, seed, stream, sample, coupled, 0.0, 0, NULL, Y_f, Y_c, mass_f, mass_c,
                       rho_f_out, rho_c_out);
}

int oracle_sample_given(const oracle_level* lv, const double* Z_all, int coupled,
                        double* Y_f, double* Y_c, double* mass_f, double* mass_c,
                        double* rho_f_out, double* rho_c_out)
{
    return sample_impl(lv, 0, 0, 0, coupled, 0.0, 0, Z_all, Y_f, Y_c, mass_f, mass_c, rho_f_out, rho_c_out);
}

int oracle_sample_perturbed(const oracle_level* lv, uint64_t seed, int stream, uint64_t sample,
                            int coupled, double amp, uint64_t perturb_seed,
                            double* Y_f, double* Y_c, double* mass_f, double* mass_c)
{
    return sample_impl(lv, seed, stream, sample, coupled, amp, perturb_seed, NULL, Y_f, Y_c, mass_f, mass_c,
                       NULL, NULL);
}
