/*
 * FP64 oracle for the coupled Dean--Kawasaki MLMC hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code with the CUDA path (paper_2311_08872_gb300/csrc) and never calls it.
 *
 * Plain, single-threaded, double precision, written to be read against the
 * paper (Cornalba & Fischer, "Multilevel Monte Carlo methods for the
 * Dean--Kawasaki equation from Fluctuating Hydrodynamics"):
 *   - Definition 2.1, Eq. (FullyDiscreteDK) with b0 = 0, b1 = 1 (Section 7.2),
 *     and with general weights b0 + b1 = 1 (the theta-scheme: an implicit
 *     diffusion half, Definition 2.1 and Appendix C, Lemma Discrete_Energy_Est),
 *   - the operators Delta_h and nabla_h. of Section 7.2,
 *   - the Right-Most Nearest-Neighbour coupling of Section 3.2 and the Fourier
 *     coupling of Section 3.1 (h_{l-1} = 3 h_l, tau_{l-1} = 9 tau_l),
 *   - the observable P_l of Eq. (eqn_MLMCLevels) with psi(x) = x^2.
 *
 * Conventions (readings where the paper is silent; same reading as the CUDA
 * path, written separately):
 *   grid point (i1,i2) at (i1*h, i2*h), flat index i1*n+i2, periodic;
 *   component r = 1 is the i1 axis, r = 2 the i2 axis;
 *   Brownian increments dbeta = sqrt(tau) * Z with Z from Philox4x32-10 +
 *   Box--Muller (see oracle_normals).
 */
#ifndef DK_ORACLE_H
#define DK_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32 with 10 rounds (Salmon et al., SC'11). */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Standard normals Z[(i1*n+i2)*2 + (r-1)] for fine step m of sample `sample`
 * at level `level` (tag level+1) in stream `stream` (0 coupled MLMC, 1 plain
 * MC), for an n x n grid (n even).  Cell pair p = (i1*n+i2)/2 uses
 *   ctr = (p, m, sample & 0xffffffff,
 *          (level+1)&0xff | (stream&0xff)<<8 | ((sample>>32)&0xffff)<<16),
 *   key = (seed & 0xffffffff, seed >> 32);
 * words (x0,x1) give cell 2p, (x2,x3) cell 2p+1 via Box--Muller with
 *   u = (x0+1) 2^-32, theta = 2 pi (x1 + 1/2) 2^-32,
 *   Z_1 = sqrt(-2 ln u) cos theta, Z_2 = sqrt(-2 ln u) sin theta. */
void oracle_normals(uint64_t seed, int level, int stream, uint64_t sample, int64_t m,
                    int n, double* Z);

/* One step of Eq. (FullyDiscreteDK), b0 = 0, b1 = 1:
 *   out = rho + tau/2 Delta_h rho + inv_sqrt_N * div_h( F ),
 *   F_r(y) = h^{-d/2} sqrt([rho(y)]^+) dbeta[(y, r)],  d = 2.
 * dbeta has layout [n*n][2]; inv_sqrt_N = 0 switches the noise off. */
void oracle_dk_step(int n, double h, double tau, double inv_sqrt_N,
                    const double* rho, const double* dbeta, double* out);

/* One step of Eq. (FullyDiscreteDK) with weights b0 >= 0, b1 = 1 - b0:
 *   (I - b0 tau/2 Delta_h) out = (I + b1 tau/2 Delta_h) rho + inv_sqrt_N * div_h( F ),
 * F as in oracle_dk_step (the noise is explicit: it uses rho).  The linear
 * system is periodic and solved exactly by discrete Fourier diagonalisation
 * (oracle_helmholtz_solve).  b0 = 0 gives oracle_dk_step. */
void oracle_theta_step(int n, double h, double tau, double inv_sqrt_N, double b0,
                       const double* rho, const double* dbeta, double* out);

/* out = (I + c L)^{-1} rhs on the periodic n x n grid, where
 * L a(x) = 4 a(x) - sum_{y~x} a(y) = -h^2 Delta_h a (c >= 0). */
void oracle_helmholtz_solve(int n, double c, const double* rhs, double* out);

typedef struct {
    int n;               /* fine cells per axis (even) */
    double h;            /* fine mesh size */
    double tau;          /* fine time step */
    int64_t M;           /* fine steps (multiple of 4 when coupled) */
    int level;           /* level index l (tag l+1) */
    double inv_sqrt_N;   /* N^{-1/2}; 0 = noise off */
    const double* rho0_f;/* I_h rho0 on the fine grid, n*n */
    const double* rho0_c;/* I_{2h} rho0 on the coarse grid, (n/2)^2 (coupled only) */
    int n_obs;
    const double* phi_f; /* [n_obs][n*n] */
    const double* phi_c; /* [n_obs][(n/2)^2] */
    double b0;           /* implicit weight of Eq. (FullyDiscreteDK) (0: explicit Euler--Maruyama) */
    int coupling;        /* 0: Right-Most NN (coarse mesh 2h, step 4 tau); 1: Fourier (3h, 9 tau) */
} oracle_level;

/* Fourier coupling of Section 3.1: the coarse-grid field carrying the fine
 * field's Fourier modes that the coarse grid (nc = n/3 points, nc even)
 * resolves.  With the unitary discrete Fourier coefficients
 * c(xi) = n^-1 sum_x f(x) exp(-2 pi i xi.x/n) of the fine field f,
 *   g(y) = nc^-1 sum_{xi in J^2} w(xi_1) w(xi_2) c(xi) exp(2 pi i xi.y/nc),
 * J = {-nc/2, ..., nc/2}, w = 1 except w(+-nc/2) = 2^-1/2 (the two fine modes
 * that alias to the coarse Nyquist mode share it), so that g is real and, for
 * a white f, white with the same variance (Remark distribution_W_ell).
 * Coarse point y is the fine point 3y. */
void oracle_fourier_restrict(int n, int nc, const double* fine, double* coarse);

/* One sample of level `lv`: fine path, and if `coupled` the coupled coarse
 * path: NN (mesh 2h, step 4 tau, increments summed over 2x2 cells and 4
 * steps) or Fourier (mesh 3h, step 9 tau, oracle_fourier_restrict of the sum
 * of the 9 fine increments);
 * both paths step with oracle_theta_step and the level's b0.
 * Outputs Y_f[k] = (rho_f^M, phi_f[k])_h, Y_c[k] likewise on the coarse grid,
 * masses (rho, 1)_h, and optionally the final fields.  Returns 0 on success. */
int oracle_sample(const oracle_level* lv, uint64_t seed, int stream, uint64_t sample,
                  int coupled, double* Y_f, double* Y_c, double* mass_f, double* mass_c,
                  double* rho_f_out, double* rho_c_out);

/* Same as oracle_sample with the fine normals supplied by the caller instead
 * of drawn: Z_all holds M arrays of n*n*2 standard normals in step order, cell
 * x = i1*n + i2, component r at 2x + r.  The coarse increments are formed from
 * them exactly as in oracle_sample (used to check properties of the coupling
 * that need chosen noise, such as its behaviour under a reflection of the
 * torus; Remark avoid_right_bias). */
int oracle_sample_given(const oracle_level* lv, const double* Z_all, int coupled,
                        double* Y_f, double* Y_c, double* mass_f, double* mass_c,
                        double* rho_f_out, double* rho_c_out);

/* Same as oracle_sample, and after every fine (coarse) step each edge of the
 * fine (coarse) grid moves a uniform random amount in [-amp/2, amp/2] from one
 * of its cells to the other (splitmix64 stream from perturb_seed).  These
 * perturbations conserve mass and have the size of one unit of a fixed-point
 * state with quantum amp; they measure how sensitive a sample path of the
 * scheme is to rounding of that size (the positive part [rho]^+ under the
 * square root makes paths ill-conditioned where rho crosses 0). */
int oracle_sample_perturbed(const oracle_level* lv, uint64_t seed, int stream, uint64_t sample,
                            int coupled, double amp, uint64_t perturb_seed,
                            double* Y_f, double* Y_c, double* mass_f, double* mass_c);

/* One application of those perturbations to an n x n field rho (in place),
 * the splitmix64 stream started at perturb_seed: edge (x, x + h e_r) moves
 * e_r(x), uniform in [-amp/2, amp/2), from cell x + h e_r to cell x
 * (transfers: NULL or [n*n][2] receiving e_1(x), e_2(x)).  Exposed so that
 * tests can pin the perturbation's law and its conservation of mass. */
void oracle_perturb_field(int n, double amp, uint64_t perturb_seed, double* rho, double* transfers);

/* Noise-free scheme (the discrete mean field rho-bar of Eq. (eqn_MLMCLevels))
 * iterated M times from rho0. */
void oracle_mean_field(int n, double h, double tau, int64_t M, const double* rho0, double* out);

/* Same for the weights (b0, 1 - b0): oracle_theta_step without noise, M times. */
void oracle_mean_field_theta(int n, double h, double tau, int64_t M, double b0, const double* rho0,
                             double* out);

#ifdef __cplusplus
}
#endif
#endif
