/*
 * twofluid_oracle.h -- plain FP64 CPU oracle for the two-fluid
 * (Maxwell + first London equation + Ohmic normal fluid) Yee scheme of
 * arXiv 2305.13419, Sec. 3, Algorithm 1.
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library; the product (CUDA) path
 * never does, and the two share no code.
 *
 * Units are SI throughout.  The state is kept at integer time levels
 * (E^n, B^n, Js^n), exactly as Algorithm 1 is written; every step runs its
 * five sub-steps in order (B half, Js half, E full with the theta scheme,
 * Js half, B half).
 *
 * Storage grid: an axis with n cells has N = n points when periodic and
 * N = n + 1 points (both walls) otherwise.  Point (i,j,k) holds
 *   Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2)
 *   Bx(i,j+1/2,k+1/2) By(i+1/2,j,k+1/2) Bz(i+1/2,j+1/2,k)
 *   Js on the E positions,
 * arrays are [k][j][i] with i fastest.  Components that fall outside the
 * domain, tangential E on a wall and normal B on a wall are never advanced
 * by the curl (PEC walls hold 0, Mur walls are set by the Mur rule).
 *
 * Parity pins: see the oracle tests (closed-form discrete dispersion, PEC
 * cavity eigenmodes, uniform-field recurrences, discrete energy identity,
 * paper's skin-depth / reflection theory and convergence orders).
 */
#ifndef TWOFLUID_ORACLE_H
#define TWOFLUID_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_BC_PERIODIC = 0, OR_BC_PEC = 1, OR_BC_MUR = 2, OR_BC_CPML = 3 };
enum { OR_SRC_GAUSS = 0, OR_SRC_SIN = 1, OR_SRC_GAUSS_SIN = 2 };

typedef struct {
    int n[3];              /* cells per axis */
    double d[3];           /* cell size per axis, m */
    double dt;             /* time step, s */
    double theta;          /* theta of the Ohmic current, Alg. 1 step 3 */
    int bc[3];             /* OR_BC_* per axis (both faces) */
    int pml_n[3];          /* CPML thickness in cells */
    double pml_m[3];       /* polynomial grading order */
    double pml_sigma_max[3];
    double pml_alpha_max[3];
    int edge_rule;         /* 0: sigma and kappa of an edge = mean over the adjacent
                              cells where they are non-zero (interface edges carry the
                              conductor's / superconductor's value); 1: plain mean */
} or_desc;

void*  or_create(const or_desc* desc);
void   or_destroy(void* h);
int    or_storage_dims(void* h, int N[3]);
/* per-cell maps [nz][ny][nx]: relative eps, relative mu, London depth (m, 0 = none), sigma (S/m) */
int    or_set_materials(void* h, const double* eps_r, const double* mu_r,
                        const double* lambda_L, const double* sigma);
/* comp 0..8 = Ex,Ey,Ez,Bx,By,Bz,Jsx,Jsy,Jsz at integer level 0 (before any step) */
int    or_set_field(void* h, int comp, const double* src);
int    or_get_field(void* h, int comp, double* dst);
int    or_add_source(void* h, int comp, const int lo[3], const int hi[3], double amp,
                     int kind, double f, double t0, double tw);
int    or_add_probe(void* h, int comp, const int p[3], const double* freqs, int nfreq,
                    int64_t n0, int64_t series_cap);
int    or_step(void* h, int64_t nsteps);
int64_t or_level(void* h);
int    or_probe_dft(void* h, int id, double* re, double* im);
int    or_probe_series(void* h, int id, double* out, int64_t n);
/* edge / face coefficients the scheme uses (for invariant checks):
   kind 0 = eps_e (F/m), 1 = sigma_e (S/m), 2 = kappa_e = mean 1/(lambda^2 mu) (1/(H m)),
   3 = mu_f (H/m), 4 = E update mask, 5 = B update mask, 6 = Js mask */
int    or_get_coeff(void* h, int kind, int comp, double* dst);
int    or_set_threads(int n);

/* Discrete adjoint of Algorithm 1 (test infrastructure, serial).
   or_adjoint_dot_test: <M v, w> and <v, M^T w> for one sub-step with random
   v, w (op 1 B half step, 2 Js half step, 3 psi_E update, 4 theta step for E,
   5 psi_B update); overwrites the state.
   or_adjoint_run: J = |X|^2 of the one-frequency probe DFT
   X = dt sum_{n0 <= n < nsteps} E_comp(p)^n exp(-i 2 pi f n dt), and dJ/d eps_r
   and dJ/d lambda_L per cell ([nz][ny][nx]), over nsteps from level 0
   (periodic, PEC or CPML walls; not Mur).  Leaves the handle at level nsteps. */
int    or_adjoint_dot_test(void* h, int op, uint64_t seed, double* lhs, double* rhs);
int    or_adjoint_run(void* h, int64_t nsteps, int comp, const int p[3], double freq, int64_t n0,
                      double* J, double* g_eps, double* g_lam);

#ifdef __cplusplus
}
#endif
#endif
