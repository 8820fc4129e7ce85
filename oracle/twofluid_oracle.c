/*
 * twofluid_oracle.c -- plain FP64 CPU oracle for the two-fluid Yee scheme of
 * arXiv 2305.13419 (Sec. 2 model, Sec. 3 Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline of the benchmark; never by the product path.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * What it computes (SI units, FP64, state at integer time levels):
 *
 *   Model (Sec. 2, Eqs. Ampere, Faraday, London1a):
 *     curl H = sigma E + Js + eps dE/dt,   curl E = -dB/dt,
 *     dJs/dt = E / (lambda^2 mu),          H = B / mu.
 *
 *   Algorithm 1, one step n -> n+1, in the paper's order:
 *     1. B^{n+1/2}  = B^n - dt/2 curl E^n
 *     2. Js^{n+1/2} = Js^n + dt/2 E^n / (lambda^2 mu)           (SC edges)
 *     3. E^{n+1}    = (1 + theta sigma dt/eps)^{-1} [ E^n + dt/eps curl H^{n+1/2}
 *                      - (1-theta) sigma dt/eps E^n - dt/eps Js^{n+1/2} ]
 *     4. Js^{n+1}   = Js^{n+1/2} + dt/2 E^{n+1} / (lambda^2 mu)  (SC edges)
 *     5. B^{n+1}    = B^{n+1/2} - dt/2 curl E^{n+1}
 *
 * Readings of points the paper leaves open:
 *   - edge material (Sec. 3: edges on an interface count as superconducting;
 *     sharp jumps in sigma or 1/lambda make the scheme first order in space,
 *     smooth ones keep second order): an edge takes the arithmetic mean of eps
 *     over the four cells that share it, and the mean of sigma and of
 *     kappa = 1/(lambda^2 mu) over those of the four cells where that property
 *     is non-zero (edge_rule 0), so an interface edge carries the full
 *     conductor / superconductor value; edge_rule 1 takes the plain mean of all
 *     four.  A face takes the mean mu of its two cells.  lambda = 0 (or inf)
 *     marks a non-superconducting cell (1/lambda -> 0).
 *   - boundaries (Sec. 3 lists periodic, PEC, PML): periodic wrap; PEC holds
 *     tangential E on a wall at 0; the PML is a Roden-Gedney convolutional PML
 *     (kappa = 1, polynomial sigma grading, linear alpha grading) backed by PEC;
 *     first-order Mur on the z walls is offered for the quasi-1-D slab.  The
 *     CPML memory variables psi_B are advanced once per level, when the E
 *     they differentiate becomes known (step 5; at level 0 from zero history),
 *     psi_E once per step in step 3.
 *   - soft source (Secs. 4.2, 5): E_c += amp * s(t^{n+1}) on the source points
 *     right after step 3.
 *   - probes (Secs. 4.2, 5 measure E at points and Fourier transform it):
 *     X_k += E_c^n exp(-i 2 pi frac(f_k dt n)) dt for levels n0 <= n < N,
 *     sampled at the start of each step.
 */
#include "twofluid_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA 2018 */
static const double C0 = 299792458.0;
static const double MU0 = 1.25663706212e-6;
static const double EPS0 = 8.8541878128e-12;
static const long double TWO_PI_L = 6.283185307179586476925286766559005768L;

#define MAXSRC 64
#define MAXPRB 64
#define MAXF 64

typedef struct {
    int comp, lo[3], hi[3], kind;
    double amp, f, t0, tw;
} src_t;

typedef struct {
    int comp, p[3], nfreq;
    double freq[MAXF], re[MAXF], im[MAXF];
    int64_t n0, cap;
    double* series;
} prb_t;

typedef struct {
    or_desc D;
    int n[3], N[3], per[3];
    long long np, nc;
    double *eps_c, *mu_c, *kap_c, *sig_c;          /* per cell */
    double *epsE[3], *sigE[3], *kapE[3], *muF[3];  /* per storage point */
    unsigned char *updE[3], *updB[3], *updJ[3], *murE[3], *keepE[3];
    double *E[3], *B[3], *J[3], *Eold[3];
    double *psiB[3][3], *psiE[3][3];               /* [component][derivative axis] */
    double *pbE[3], *pcE[3], *pbB[3], *pcB[3];     /* 1-D CPML profiles */
    int64_t level;
    int psi_ready;
    src_t src[MAXSRC];
    int nsrc;
    prb_t prb[MAXPRB];
    int nprb;
} grid_t;

static inline long long IX(const grid_t* g, int i, int j, int k) {
    return ((long long)k * g->N[1] + j) * g->N[0] + i;
}
static inline long long CI(const grid_t* g, int i, int j, int k) {
    return ((long long)k * g->n[1] + j) * g->n[0] + i;
}
/* next / previous point along axis a; wraps on periodic axes.  The update
   masks guarantee that no advanced component ever needs a point outside. */
static inline int nxt(const grid_t* g, int a, int p) { return (p + 1 < g->N[a]) ? p + 1 : (g->per[a] ? 0 : p); }
static inline int prv(const grid_t* g, int a, int p) { return (p > 0) ? p - 1 : (g->per[a] ? g->N[a] - 1 : p); }
static inline int wrapc(const grid_t* g, int a, int c) { return (c < 0) ? c + g->n[a] : c; }

/* is component c (0..2 E, 3..5 B) offset by half a cell along axis a? */
static int half(int c, int a) { return (c < 3) ? (a == c) : (a != c - 3); }
/* sign of the d/da term in component c of a curl: +1 for a = c+1, -1 for a = c+2 (mod 3) */
static int sgn(int c, int a) { return ((a - c + 3) % 3 == 1) ? 1 : -1; }

static double* dalloc(long long n) { return (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }
static unsigned char* balloc(long long n) { return (unsigned char*)calloc((size_t)(n > 0 ? n : 1), 1); }

/* ---------------------------------------------------------------- masks */
static void build_masks(grid_t* g) {
    for (int c = 0; c < 6; ++c) {
        for (int k = 0; k < g->N[2]; ++k)
            for (int j = 0; j < g->N[1]; ++j)
                for (int i = 0; i < g->N[0]; ++i) {
                    int p[3] = {i, j, k};
                    int valid = 1, interior = 1, onlyz = 1;
                    for (int a = 0; a < 3; ++a) {
                        if (g->per[a]) continue;
                        if (half(c, a)) {
                            if (p[a] >= g->n[a]) valid = 0;
                        } else if (p[a] < 1 || p[a] > g->n[a] - 1) {
                            interior = 0;
                            if (a != 2) onlyz = 0;
                        }
                    }
                    long long q = IX(g, i, j, k);
                    if (c < 3) {
                        g->updE[c][q] = (unsigned char)(valid && interior);
                        int mur = valid && !interior && onlyz && c < 2 && g->D.bc[2] == OR_BC_MUR;
                        g->murE[c][q] = (unsigned char)mur;
                        g->keepE[c][q] = (unsigned char)((valid && interior) || mur);
                    } else {
                        g->updB[c - 3][q] = (unsigned char)(valid && interior);
                    }
                }
    }
}

/* ----------------------------------------------------------- materials */
static void build_coefficients(grid_t* g) {
    for (int c = 0; c < 3; ++c) {
        #pragma omp parallel for schedule(static)
        for (int k = 0; k < g->N[2]; ++k)
            for (int j = 0; j < g->N[1]; ++j)
                for (int i = 0; i < g->N[0]; ++i) {
                    long long q = IX(g, i, j, k);
                    int p[3] = {i, j, k};
                    /* edge E_c: mean over the 4 cells sharing it */
                    if (g->updE[c][q]) {
                        int b1 = (c + 1) % 3, b2 = (c + 2) % 3;
                        double se = 0, ss = 0, sk = 0;
                        int ns = 0, nk = 0;
                        for (int u = 0; u < 2; ++u)
                            for (int v = 0; v < 2; ++v) {
                                int cc[3];
                                cc[c] = p[c];
                                cc[b1] = wrapc(g, b1, p[b1] - u);
                                cc[b2] = wrapc(g, b2, p[b2] - v);
                                long long m = CI(g, cc[0], cc[1], cc[2]);
                                se += g->eps_c[m];
                                ss += g->sig_c[m];
                                sk += g->kap_c[m];
                                ns += g->sig_c[m] > 0.0;
                                nk += g->kap_c[m] > 0.0;
                            }
                        g->epsE[c][q] = EPS0 * se / 4.0;
                        if (g->D.edge_rule == 1) {   /* plain mean of the four cells */
                            g->sigE[c][q] = ss / 4.0;
                            g->kapE[c][q] = sk / 4.0;
                        } else {                     /* mean over the conducting / SC cells */
                            g->sigE[c][q] = ns ? ss / ns : 0.0;
                            g->kapE[c][q] = nk ? sk / nk : 0.0;
                        }
                        g->updJ[c][q] = (unsigned char)(g->kapE[c][q] > 0.0);
                    } else {
                        g->epsE[c][q] = EPS0;
                        g->sigE[c][q] = 0.0;
                        g->kapE[c][q] = 0.0;
                        g->updJ[c][q] = 0;
                    }
                    /* face B_c: mean mu of the 2 cells on either side */
                    if (g->updB[c][q]) {
                        int b1 = (c + 1) % 3, b2 = (c + 2) % 3;
                        double sm = 0;
                        for (int u = 0; u < 2; ++u) {
                            int cc[3];
                            cc[c] = wrapc(g, c, p[c] - u);
                            cc[b1] = p[b1];
                            cc[b2] = p[b2];
                            sm += g->mu_c[CI(g, cc[0], cc[1], cc[2])];
                        }
                        g->muF[c][q] = MU0 * sm / 2.0;
                    } else {
                        g->muF[c][q] = MU0;
                    }
                }
    }
}

static void pml_coef(const grid_t* g, int a, double x, double* b, double* c) {
    double L = g->D.pml_n[a], n = g->n[a], rho = 0.0;
    if (x < L) rho = (L - x) / L;
    else if (x > n - L) rho = (x - (n - L)) / L;
    if (rho <= 0.0) { *b = 0.0; *c = 0.0; return; }
    double s = g->D.pml_sigma_max[a] * pow(rho, g->D.pml_m[a]);
    double al = g->D.pml_alpha_max[a] * (1.0 - rho);
    *b = exp(-(s + al) * g->D.dt / EPS0);
    *c = (s + al > 0.0) ? s * (*b - 1.0) / (s + al) : 0.0;
}

/* -------------------------------------------------------------- create */
void* or_create(const or_desc* desc) {
    if (!desc) return NULL;
    grid_t* g = (grid_t*)calloc(1, sizeof(grid_t));
    g->D = *desc;
    for (int a = 0; a < 3; ++a) {
        if (desc->n[a] < 1 || desc->d[a] <= 0) { free(g); return NULL; }
        if (desc->bc[a] == OR_BC_MUR && a != 2) { free(g); return NULL; }
        if (desc->edge_rule < 0 || desc->edge_rule > 1) { free(g); return NULL; }
        g->n[a] = desc->n[a];
        g->per[a] = desc->bc[a] == OR_BC_PERIODIC;
        g->N[a] = g->n[a] + (g->per[a] ? 0 : 1);
        if (desc->bc[a] == OR_BC_CPML && (desc->pml_n[a] < 1 || 2 * desc->pml_n[a] > desc->n[a])) {
            free(g);
            return NULL;
        }
    }
    g->np = (long long)g->N[0] * g->N[1] * g->N[2];
    g->nc = (long long)g->n[0] * g->n[1] * g->n[2];
    g->eps_c = dalloc(g->nc); g->mu_c = dalloc(g->nc); g->kap_c = dalloc(g->nc); g->sig_c = dalloc(g->nc);
    for (long long m = 0; m < g->nc; ++m) { g->eps_c[m] = 1.0; g->mu_c[m] = 1.0; }
    for (int c = 0; c < 3; ++c) {
        g->epsE[c] = dalloc(g->np); g->sigE[c] = dalloc(g->np); g->kapE[c] = dalloc(g->np);
        g->muF[c] = dalloc(g->np);
        g->updE[c] = balloc(g->np); g->updB[c] = balloc(g->np); g->updJ[c] = balloc(g->np);
        g->murE[c] = balloc(g->np); g->keepE[c] = balloc(g->np);
        g->E[c] = dalloc(g->np); g->B[c] = dalloc(g->np); g->J[c] = dalloc(g->np);
        g->Eold[c] = dalloc(g->np);
    }
    for (int a = 0; a < 3; ++a) {
        if (desc->bc[a] != OR_BC_CPML) continue;
        for (int c = 0; c < 3; ++c) {
            if (c == a) continue;
            g->psiB[c][a] = dalloc(g->np);
            g->psiE[c][a] = dalloc(g->np);
        }
        g->pbE[a] = dalloc(g->N[a]); g->pcE[a] = dalloc(g->N[a]);
        g->pbB[a] = dalloc(g->N[a]); g->pcB[a] = dalloc(g->N[a]);
        for (int p = 0; p < g->N[a]; ++p) {
            pml_coef(g, a, (double)p, &g->pbE[a][p], &g->pcE[a][p]);
            pml_coef(g, a, (double)p + 0.5, &g->pbB[a][p], &g->pcB[a][p]);
        }
    }
    build_masks(g);
    build_coefficients(g);
    return g;
}

void or_destroy(void* h) {
    grid_t* g = (grid_t*)h;
    if (!g) return;
    free(g->eps_c); free(g->mu_c); free(g->kap_c); free(g->sig_c);
    for (int c = 0; c < 3; ++c) {
        free(g->epsE[c]); free(g->sigE[c]); free(g->kapE[c]); free(g->muF[c]);
        free(g->updE[c]); free(g->updB[c]); free(g->updJ[c]); free(g->murE[c]); free(g->keepE[c]);
        free(g->E[c]); free(g->B[c]); free(g->J[c]); free(g->Eold[c]);
        for (int a = 0; a < 3; ++a) { free(g->psiB[c][a]); free(g->psiE[c][a]); }
    }
    for (int a = 0; a < 3; ++a) { free(g->pbE[a]); free(g->pcE[a]); free(g->pbB[a]); free(g->pcB[a]); }
    for (int p = 0; p < g->nprb; ++p) free(g->prb[p].series);
    free(g);
}

int or_storage_dims(void* h, int N[3]) {
    grid_t* g = (grid_t*)h;
    for (int a = 0; a < 3; ++a) N[a] = g->N[a];
    return 0;
}

int or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int or_set_materials(void* h, const double* eps_r, const double* mu_r, const double* lambda_L,
                     const double* sigma) {
    grid_t* g = (grid_t*)h;
    if (g->level != 0 || g->psi_ready) return 5;
    for (long long m = 0; m < g->nc; ++m) {
        double e = eps_r ? eps_r[m] : 1.0, u = mu_r ? mu_r[m] : 1.0;
        double l = lambda_L ? lambda_L[m] : 0.0, s = sigma ? sigma[m] : 0.0;
        if (!(e > 0) || !(u > 0) || !(s >= 0) || l < 0) return 1;
        g->eps_c[m] = e;
        g->mu_c[m] = u;
        g->sig_c[m] = s;
        /* first London equation: dJs/dt = E / (lambda^2 mu); no SC when 1/lambda -> 0 */
        g->kap_c[m] = (l > 0 && isfinite(l)) ? 1.0 / (l * l * MU0 * u) : 0.0;
    }
    build_coefficients(g);
    for (int c = 0; c < 3; ++c)
        for (long long q = 0; q < g->np; ++q)
            if (!g->updJ[c][q]) g->J[c][q] = 0.0;
    return 0;
}

int or_set_field(void* h, int comp, const double* src) {
    grid_t* g = (grid_t*)h;
    if (comp < 0 || comp > 8) return 1;
    if (g->level != 0 || g->psi_ready) return 5;
    double* dst = comp < 3 ? g->E[comp] : comp < 6 ? g->B[comp - 3] : g->J[comp - 6];
    const unsigned char* keep = comp < 3 ? g->keepE[comp] : comp < 6 ? g->updB[comp - 3] : g->updJ[comp - 6];
    for (long long q = 0; q < g->np; ++q) dst[q] = keep[q] ? src[q] : 0.0;
    return 0;
}

int or_get_field(void* h, int comp, double* dst) {
    grid_t* g = (grid_t*)h;
    if (comp < 0 || comp > 8) return 1;
    const double* s = comp < 3 ? g->E[comp] : comp < 6 ? g->B[comp - 3] : g->J[comp - 6];
    memcpy(dst, s, sizeof(double) * (size_t)g->np);
    return 0;
}

int or_get_coeff(void* h, int kind, int comp, double* dst) {
    grid_t* g = (grid_t*)h;
    if (comp < 0 || comp > 2) return 1;
    for (long long q = 0; q < g->np; ++q) {
        switch (kind) {
            case 0: dst[q] = g->epsE[comp][q]; break;
            case 1: dst[q] = g->sigE[comp][q]; break;
            case 2: dst[q] = g->kapE[comp][q]; break;
            case 3: dst[q] = g->muF[comp][q]; break;
            case 4: dst[q] = g->updE[comp][q]; break;
            case 5: dst[q] = g->updB[comp][q]; break;
            case 6: dst[q] = g->updJ[comp][q]; break;
            default: return 1;
        }
    }
    return 0;
}

int or_add_source(void* h, int comp, const int lo[3], const int hi[3], double amp, int kind,
                  double f, double t0, double tw) {
    grid_t* g = (grid_t*)h;
    if (g->nsrc >= MAXSRC || comp < 0 || comp > 2 || kind < 0 || kind > 2) return 1;
    src_t* s = &g->src[g->nsrc];
    s->comp = comp;
    for (int a = 0; a < 3; ++a) {
        s->lo[a] = lo[a] < 0 ? 0 : lo[a];
        s->hi[a] = hi[a] > g->N[a] ? g->N[a] : hi[a];
    }
    s->amp = amp; s->kind = kind; s->f = f; s->t0 = t0; s->tw = tw;
    g->nsrc++;
    return 0;
}

int or_add_probe(void* h, int comp, const int p[3], const double* freqs, int nfreq, int64_t n0,
                 int64_t series_cap) {
    grid_t* g = (grid_t*)h;
    if (g->nprb >= MAXPRB || comp < 0 || comp > 2 || nfreq < 0 || nfreq > MAXF) return 1;
    for (int a = 0; a < 3; ++a)
        if (p[a] < 0 || p[a] >= g->N[a]) return 1;
    prb_t* r = &g->prb[g->nprb];
    memset(r, 0, sizeof(*r));
    r->comp = comp;
    for (int a = 0; a < 3; ++a) r->p[a] = p[a];
    r->nfreq = nfreq;
    for (int k = 0; k < nfreq; ++k) r->freq[k] = freqs[k];
    r->n0 = n0;
    r->cap = series_cap > 0 ? series_cap : 0;
    r->series = r->cap ? dalloc(r->cap) : NULL;
    g->nprb++;
    return 0;
}

int64_t or_level(void* h) { return ((grid_t*)h)->level; }

int or_probe_dft(void* h, int id, double* re, double* im) {
    grid_t* g = (grid_t*)h;
    if (id < 0 || id >= g->nprb) return 1;
    for (int k = 0; k < g->prb[id].nfreq; ++k) { re[k] = g->prb[id].re[k]; im[k] = g->prb[id].im[k]; }
    return 0;
}

int or_probe_series(void* h, int id, double* out, int64_t n) {
    grid_t* g = (grid_t*)h;
    if (id < 0 || id >= g->nprb || n > g->prb[id].cap) return 1;
    for (int64_t q = 0; q < n; ++q) out[q] = g->prb[id].series[q];
    return 0;
}

/* ------------------------------------------------------ discrete curls */
/* forward difference of E_e along axis a at point p: (E_e(p + a) - E_e(p)) / d_a */
static inline double dE_fwd(const grid_t* g, int e, int a, const int p[3]) {
    int q[3] = {p[0], p[1], p[2]};
    q[a] = nxt(g, a, p[a]);
    return (g->E[e][IX(g, q[0], q[1], q[2])] - g->E[e][IX(g, p[0], p[1], p[2])]) / g->D.d[a];
}
/* backward difference of H_h = B_h / mu_f along axis a at point p */
static inline double dH_bwd(const grid_t* g, int h, int a, const int p[3]) {
    int q[3] = {p[0], p[1], p[2]};
    q[a] = prv(g, a, p[a]);
    long long i0 = IX(g, p[0], p[1], p[2]), i1 = IX(g, q[0], q[1], q[2]);
    return (g->B[h][i0] / g->muF[h][i0] - g->B[h][i1] / g->muF[h][i1]) / g->D.d[a];
}

/* component cb of curl E at the B_cb position of point p, with the CPML
   memory terms as they stand:
     (curl E)_x = [dEz/dy + psi_xy] - [dEy/dz + psi_xz]
     (curl E)_y = [dEx/dz + psi_yz] - [dEz/dx + psi_yx]
     (curl E)_z = [dEy/dx + psi_zx] - [dEx/dy + psi_zy]                      */
static double curlE(const grid_t* g, int cb, const int p[3]) {
    long long q = IX(g, p[0], p[1], p[2]);
    double r = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (a == cb) continue;
        int e = 3 - cb - a;
        double t = dE_fwd(g, e, a, p);
        if (g->psiB[cb][a]) t += g->psiB[cb][a][q];
        r += sgn(cb, a) * t;
    }
    return r;
}

/* component c of curl H at the E_c position of point p (backward differences) */
static double curlH(const grid_t* g, int c, const int p[3]) {
    long long q = IX(g, p[0], p[1], p[2]);
    double r = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (a == c) continue;
        int hc = 3 - c - a;
        double t = dH_bwd(g, hc, a, p);
        if (g->psiE[c][a]) t += g->psiE[c][a][q];
        r += sgn(c, a) * t;
    }
    return r;
}

/* CPML memory for the B update: psi = b psi + c dE/da, at the current E */
static void advance_psiB(grid_t* g) {
    for (int cb = 0; cb < 3; ++cb)
        for (int a = 0; a < 3; ++a) {
            double* ps = g->psiB[cb][a];
            if (!ps) continue;
            int e = 3 - cb - a;
            #pragma omp parallel for schedule(static)
            for (int k = 0; k < g->N[2]; ++k)
                for (int j = 0; j < g->N[1]; ++j)
                    for (int i = 0; i < g->N[0]; ++i) {
                        long long q = IX(g, i, j, k);
                        if (!g->updB[cb][q]) continue;
                        int p[3] = {i, j, k};
                        ps[q] = g->pbB[a][p[a]] * ps[q] + g->pcB[a][p[a]] * dE_fwd(g, e, a, p);
                    }
        }
}

/* CPML memory for the E update: psi = b psi + c dH/da, at the current B */
static void advance_psiE(grid_t* g) {
    for (int c = 0; c < 3; ++c)
        for (int a = 0; a < 3; ++a) {
            double* ps = g->psiE[c][a];
            if (!ps) continue;
            int hc = 3 - c - a;
            #pragma omp parallel for schedule(static)
            for (int k = 0; k < g->N[2]; ++k)
                for (int j = 0; j < g->N[1]; ++j)
                    for (int i = 0; i < g->N[0]; ++i) {
                        long long q = IX(g, i, j, k);
                        if (!g->updE[c][q]) continue;
                        int p[3] = {i, j, k};
                        ps[q] = g->pbE[a][p[a]] * ps[q] + g->pcE[a][p[a]] * dH_bwd(g, hc, a, p);
                    }
        }
}

/* ----------------------------------------------------- Algorithm 1 steps */
/* steps 1 and 5: B <- B - dt/2 curl E */
static void half_step_B(grid_t* g) {
    const double h = 0.5 * g->D.dt;
    for (int cb = 0; cb < 3; ++cb) {
        #pragma omp parallel for schedule(static)
        for (int k = 0; k < g->N[2]; ++k)
            for (int j = 0; j < g->N[1]; ++j)
                for (int i = 0; i < g->N[0]; ++i) {
                    long long q = IX(g, i, j, k);
                    if (!g->updB[cb][q]) continue;
                    int p[3] = {i, j, k};
                    g->B[cb][q] -= h * curlE(g, cb, p);
                }
    }
}

/* steps 2 and 4: Js <- Js + dt/2 E / (lambda^2 mu) on superconducting edges */
static void half_step_Js(grid_t* g) {
    const double h = 0.5 * g->D.dt;
    for (int c = 0; c < 3; ++c) {
        #pragma omp parallel for schedule(static)
        for (long long q = 0; q < g->np; ++q)
            if (g->updJ[c][q]) g->J[c][q] += h * g->kapE[c][q] * g->E[c][q];
    }
}

/* step 3: E^{n+1} from E^n, H^{n+1/2} and Js^{n+1/2} by the theta scheme */
static void full_step_E(grid_t* g) {
    const double dt = g->D.dt, th = g->D.theta;
    for (int c = 0; c < 3; ++c) {
        #pragma omp parallel for schedule(static)
        for (int k = 0; k < g->N[2]; ++k)
            for (int j = 0; j < g->N[1]; ++j)
                for (int i = 0; i < g->N[0]; ++i) {
                    long long q = IX(g, i, j, k);
                    if (!g->updE[c][q]) continue;
                    int p[3] = {i, j, k};
                    double eps = g->epsE[c][q], s = g->sigE[c][q] * dt / eps;
                    double rhs = g->E[c][q] + dt / eps * curlH(g, c, p) - (1.0 - th) * s * g->E[c][q]
                                 - dt / eps * g->J[c][q];
                    g->E[c][q] = rhs / (1.0 + th * s);
                }
    }
}

static double waveform(const src_t* s, double t) {
    double env = exp(-(t - s->t0) * (t - s->t0) / (2.0 * s->tw * s->tw));
    switch (s->kind) {
        case OR_SRC_GAUSS: return env;
        case OR_SRC_SIN: return sin(2.0 * M_PI * s->f * t);
        default: return env * sin(2.0 * M_PI * s->f * t);
    }
}

static void apply_sources(grid_t* g, double t) {
    for (int m = 0; m < g->nsrc; ++m) {
        const src_t* s = &g->src[m];
        double v = s->amp * waveform(s, t);
        for (int k = s->lo[2]; k < s->hi[2]; ++k)
            for (int j = s->lo[1]; j < s->hi[1]; ++j)
                for (int i = s->lo[0]; i < s->hi[0]; ++i) {
                    long long q = IX(g, i, j, k);
                    if (g->updE[s->comp][q]) g->E[s->comp][q] += v;
                }
    }
}

/* first-order Mur on the z walls: E_w^{n+1} = E_i^n + M (E_i^{n+1} - E_w^n),
   M = (c dt - dz) / (c dt + dz), E_i the first interior plane */
static void apply_mur(grid_t* g) {
    if (g->D.bc[2] != OR_BC_MUR) return;
    const double M = (C0 * g->D.dt - g->D.d[2]) / (C0 * g->D.dt + g->D.d[2]);
    const int walls[2] = {0, g->n[2]}, inner[2] = {1, g->n[2] - 1};
    for (int c = 0; c < 2; ++c)
        for (int w = 0; w < 2; ++w)
            for (int j = 0; j < g->N[1]; ++j)
                for (int i = 0; i < g->N[0]; ++i) {
                    long long qw = IX(g, i, j, walls[w]), qi = IX(g, i, j, inner[w]);
                    if (!g->murE[c][qw]) continue;
                    g->E[c][qw] = g->Eold[c][qi] + M * (g->E[c][qi] - g->Eold[c][qw]);
                }
}

static void sample_probes(grid_t* g) {
    const double dt = g->D.dt;
    for (int m = 0; m < g->nprb; ++m) {
        prb_t* r = &g->prb[m];
        double s = g->E[r->comp][IX(g, r->p[0], r->p[1], r->p[2])];
        if (g->level < r->cap) r->series[g->level] = s;
        if (g->level < r->n0) continue;
        for (int k = 0; k < r->nfreq; ++k) {
            long double ph = (long double)r->freq[k] * (long double)dt * (long double)g->level;
            ph -= floorl(ph);
            long double ang = TWO_PI_L * ph;
            r->re[k] += s * (double)cosl(ang) * dt;
            r->im[k] -= s * (double)sinl(ang) * dt;
        }
    }
}

int or_step(void* h, int64_t nsteps) {
    grid_t* g = (grid_t*)h;
    if (nsteps < 0) return 1;
    if (!g->psi_ready) {   /* psi_B at level 0 from zero history */
        advance_psiB(g);
        g->psi_ready = 1;
    }
    for (int64_t s = 0; s < nsteps; ++s) {
        sample_probes(g);
        half_step_B(g);                                  /* 1 */
        half_step_Js(g);                                 /* 2 */
        if (g->D.bc[2] == OR_BC_MUR)
            for (int c = 0; c < 2; ++c) memcpy(g->Eold[c], g->E[c], sizeof(double) * (size_t)g->np);
        advance_psiE(g);                                 /* 3 */
        full_step_E(g);
        apply_sources(g, (double)(g->level + 1) * g->D.dt);
        apply_mur(g);
        half_step_Js(g);                                 /* 4 */
        advance_psiB(g);                                 /* 5 */
        half_step_B(g);
        g->level++;
    }
    return 0;
}

/* ===================================================================== */
/* Discrete adjoint of Algorithm 1.                                       */
/*                                                                        */
/* With sources fixed, each sub-step of a step is a linear map of the     */
/* state (E, B, Js, psi_E, psi_B).  Its transpose acts on the adjoint     */
/* state; applying the transposes in reverse order, step by step from the */
/* last, and adding the derivative of the objective at each sampled level */
/* gives the adjoint trajectory.  The gradient of the objective with      */
/* respect to a coefficient is the adjoint of the sub-step's output dotted */
/* with the sub-step's derivative:                                        */
/*   step 3 (theta scheme):  (eps + theta sigma dt) E' =                 */
/*       (eps - (1 - theta) sigma dt) E + dt (curl H - Js)               */
/*       => dE'/d eps_e = (E - E') / (eps_e + theta sigma_e dt);         */
/*   steps 2 and 4:  Js' = Js + dt/2 kappa E  =>  dJs'/d kappa_e = dt/2 E. */
/* Edge values are means of cell values (build_coefficients), so a cell's */
/* gradient collects its edges' gradients with the same weights.          */
/* All loops are serial: the transposed curls scatter into neighbours.    */
/* ===================================================================== */

typedef struct {
    double *E[3], *B[3], *J[3], *psiB[3][3], *psiE[3][3];
} adj_t;

static void adj_alloc(const grid_t* g, adj_t* a) {
    memset(a, 0, sizeof(*a));
    for (int c = 0; c < 3; ++c) {
        a->E[c] = dalloc(g->np); a->B[c] = dalloc(g->np); a->J[c] = dalloc(g->np);
        for (int x = 0; x < 3; ++x) {
            if (g->psiB[c][x]) a->psiB[c][x] = dalloc(g->np);
            if (g->psiE[c][x]) a->psiE[c][x] = dalloc(g->np);
        }
    }
}

static void adj_free(adj_t* a) {
    for (int c = 0; c < 3; ++c) {
        free(a->E[c]); free(a->B[c]); free(a->J[c]);
        for (int x = 0; x < 3; ++x) { free(a->psiB[c][x]); free(a->psiE[c][x]); }
    }
}

/* transpose of half_step_B (B -= h curl E with the psi_B terms) */
static void adj_half_step_B(const grid_t* g, adj_t* A) {
    const double h = 0.5 * g->D.dt;
    for (int cb = 0; cb < 3; ++cb)
        for (int k = 0; k < g->N[2]; ++k)
            for (int j = 0; j < g->N[1]; ++j)
                for (int i = 0; i < g->N[0]; ++i) {
                    long long q = IX(g, i, j, k);
                    if (!g->updB[cb][q]) continue;
                    int p[3] = {i, j, k};
                    double v = -h * A->B[cb][q];
                    for (int a = 0; a < 3; ++a) {
                        if (a == cb) continue;
                        int e = 3 - cb - a;
                        double w = v * sgn(cb, a);
                        int r[3] = {i, j, k};
                        r[a] = nxt(g, a, p[a]);
                        A->E[e][IX(g, r[0], r[1], r[2])] += w / g->D.d[a];
                        A->E[e][q] -= w / g->D.d[a];
                        if (A->psiB[cb][a]) A->psiB[cb][a][q] += w;
                    }
                }
}

/* transpose of advance_psiB (psi = b psi + c dE/da on updated faces) */
static void adj_advance_psiB(const grid_t* g, adj_t* A) {
    for (int cb = 0; cb < 3; ++cb)
        for (int a = 0; a < 3; ++a) {
            double* ps = A->psiB[cb][a];
            if (!ps) continue;
            int e = 3 - cb - a;
            for (int k = 0; k < g->N[2]; ++k)
                for (int j = 0; j < g->N[1]; ++j)
                    for (int i = 0; i < g->N[0]; ++i) {
                        long long q = IX(g, i, j, k);
                        if (!g->updB[cb][q]) continue;
                        int p[3] = {i, j, k};
                        double w = ps[q], c = g->pcB[a][p[a]] / g->D.d[a];
                        int r[3] = {i, j, k};
                        r[a] = nxt(g, a, p[a]);
                        A->E[e][IX(g, r[0], r[1], r[2])] += c * w;
                        A->E[e][q] -= c * w;
                        ps[q] = g->pbB[a][p[a]] * w;
                    }
        }
}

/* transpose of half_step_Js; with gk != NULL also dJ/dkappa_e += dt/2 Js_adj E */
static void adj_half_step_Js(const grid_t* g, adj_t* A, double* const gk[3], double* const Ef[3]) {
    const double h = 0.5 * g->D.dt;
    for (int c = 0; c < 3; ++c)
        for (long long q = 0; q < g->np; ++q) {
            if (!g->updJ[c][q]) continue;
            A->E[c][q] += h * g->kapE[c][q] * A->J[c][q];
            if (gk) gk[c][q] += h * A->J[c][q] * Ef[c][q];
        }
}

/* transpose of full_step_E; with ge != NULL also dJ/deps_r,e (eps_e = EPS0 eps_r,e)
   += E_adj' EPS0 (E - E') / (eps_e + theta sigma_e dt), E = Eb, E' = Ea */
static void adj_full_step_E(const grid_t* g, adj_t* A, double* const ge[3], double* const Eb[3],
                            double* const Ea[3]) {
    const double dt = g->D.dt, th = g->D.theta;
    for (int c = 0; c < 3; ++c)
        for (int k = 0; k < g->N[2]; ++k)
            for (int j = 0; j < g->N[1]; ++j)
                for (int i = 0; i < g->N[0]; ++i) {
                    long long q = IX(g, i, j, k);
                    if (!g->updE[c][q]) continue;
                    int p[3] = {i, j, k};
                    double eps = g->epsE[c][q], s = g->sigE[c][q] * dt / eps;
                    if (ge) ge[c][q] += A->E[c][q] * EPS0 * (Eb[c][q] - Ea[c][q]) / (eps + th * g->sigE[c][q] * dt);
                    double e = A->E[c][q] / (1.0 + th * s);
                    A->E[c][q] = (1.0 - (1.0 - th) * s) * e;
                    double v = dt / eps * e;
                    A->J[c][q] -= v;
                    for (int a = 0; a < 3; ++a) {
                        if (a == c) continue;
                        int hc = 3 - c - a;
                        double w = v * sgn(c, a);
                        int r[3] = {i, j, k};
                        r[a] = prv(g, a, p[a]);
                        long long qr = IX(g, r[0], r[1], r[2]);
                        A->B[hc][q] += w / (g->muF[hc][q] * g->D.d[a]);
                        A->B[hc][qr] -= w / (g->muF[hc][qr] * g->D.d[a]);
                        if (A->psiE[c][a]) A->psiE[c][a][q] += w;
                    }
                }
}

/* transpose of advance_psiE (psi = b psi + c dH/da on updated edges) */
static void adj_advance_psiE(const grid_t* g, adj_t* A) {
    for (int c = 0; c < 3; ++c)
        for (int a = 0; a < 3; ++a) {
            double* ps = A->psiE[c][a];
            if (!ps) continue;
            int hc = 3 - c - a;
            for (int k = 0; k < g->N[2]; ++k)
                for (int j = 0; j < g->N[1]; ++j)
                    for (int i = 0; i < g->N[0]; ++i) {
                        long long q = IX(g, i, j, k);
                        if (!g->updE[c][q]) continue;
                        int p[3] = {i, j, k};
                        double w = ps[q], cc = g->pcE[a][p[a]] / g->D.d[a];
                        int r[3] = {i, j, k};
                        r[a] = prv(g, a, p[a]);
                        long long qr = IX(g, r[0], r[1], r[2]);
                        A->B[hc][q] += cc * w / g->muF[hc][q];
                        A->B[hc][qr] -= cc * w / g->muF[hc][qr];
                        ps[q] = g->pbE[a][p[a]] * w;
                    }
        }
}

/* ------------------------------------------------------ dot-product test */
static uint64_t sm64(uint64_t* s) {   /* SplitMix64 */
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double urand(uint64_t* s) { return (double)(sm64(s) >> 11) * (1.0 / 9007199254740992.0) - 0.5; }

/* all state arrays of g (fwd) or A (adjoint) in a fixed order */
static int state_arrays(grid_t* g, adj_t* A, double** out) {
    int n = 0;
    for (int c = 0; c < 3; ++c) out[n++] = A ? A->E[c] : g->E[c];
    for (int c = 0; c < 3; ++c) out[n++] = A ? A->B[c] : g->B[c];
    for (int c = 0; c < 3; ++c) out[n++] = A ? A->J[c] : g->J[c];
    for (int c = 0; c < 3; ++c)
        for (int a = 0; a < 3; ++a) {
            if (g->psiB[c][a]) out[n++] = A ? A->psiB[c][a] : g->psiB[c][a];
            if (g->psiE[c][a]) out[n++] = A ? A->psiE[c][a] : g->psiE[c][a];
        }
    return n;
}

/* <M v, w> and <v, M^T w> for sub-step `op` (1: B half step, 2: Js half
   step, 3: psi_E update, 4: E theta step, 5: psi_B update) with random v, w.
   Overwrites the forward state. */
int or_adjoint_dot_test(void* h, int op, uint64_t seed, double* lhs, double* rhs) {
    grid_t* g = (grid_t*)h;
    if (op < 1 || op > 5 || !lhs || !rhs) return 1;
    adj_t A;
    adj_alloc(g, &A);
    double *fs[40], *as[40];
    const int n = state_arrays(g, NULL, fs);
    state_arrays(g, &A, as);
    double** v = (double**)calloc((size_t)n, sizeof(double*));
    uint64_t s = seed;
    for (int m = 0; m < n; ++m) {
        v[m] = dalloc(g->np);
        for (long long q = 0; q < g->np; ++q) fs[m][q] = v[m][q] = urand(&s);
        for (long long q = 0; q < g->np; ++q) as[m][q] = urand(&s);
    }
    double** w = (double**)calloc((size_t)n, sizeof(double*));
    for (int m = 0; m < n; ++m) {
        w[m] = dalloc(g->np);
        memcpy(w[m], as[m], sizeof(double) * (size_t)g->np);
    }
    switch (op) {
        case 1: half_step_B(g); adj_half_step_B(g, &A); break;
        case 2: half_step_Js(g); adj_half_step_Js(g, &A, NULL, NULL); break;
        case 3: advance_psiE(g); adj_advance_psiE(g, &A); break;
        case 4: full_step_E(g); adj_full_step_E(g, &A, NULL, NULL, NULL); break;
        default: advance_psiB(g); adj_advance_psiB(g, &A); break;
    }
    long double l = 0, r = 0;
    for (int m = 0; m < n; ++m)
        for (long long q = 0; q < g->np; ++q) {
            l += (long double)fs[m][q] * w[m][q];
            r += (long double)v[m][q] * as[m][q];
        }
    *lhs = (double)l;
    *rhs = (double)r;
    for (int m = 0; m < n; ++m) { free(v[m]); free(w[m]); }
    free(v);
    free(w);
    adj_free(&A);
    return 0;
}

/* ------------------------------------------------------ adjoint gradient */
/* Objective J = |X|^2, X = dt sum_{n=n0}^{N-1} E_comp(p)^n exp(-i 2 pi f n dt)
   (the probe DFT at one frequency).  Runs nsteps of Algorithm 1 from the
   handle's current state (level 0; no Mur walls), then the adjoint back to
   level 0, and returns J and dJ/d eps_r and dJ/d lambda_L per cell (0 for
   cells that are not superconducting).  The handle is left at level nsteps. */
int or_adjoint_run(void* h, int64_t nsteps, int comp, const int pr[3], double freq, int64_t n0, double* Jout,
                   double* g_eps, double* g_lam) {
    grid_t* g = (grid_t*)h;
    if (g->level != 0 || g->D.bc[2] == OR_BC_MUR || nsteps < 1 || comp < 0 || comp > 2) return 1;
    for (int a = 0; a < 3; ++a)
        if (pr[a] < 0 || pr[a] >= g->N[a]) return 1;
    const long long np = g->np, qp = IX(g, pr[0], pr[1], pr[2]);
    const double dt = g->D.dt;
    /* forward, keeping E^n (n = 0..N) and the theta-step output before sources */
    double* Eh = dalloc(3 * np * (nsteps + 1));
    double* Ep = dalloc(3 * np * nsteps);
    if (!Eh || !Ep) { free(Eh); free(Ep); return 2; }
#define EH(n, c) (Eh + ((long long)(n) * 3 + (c)) * np)
#define EP(n, c) (Ep + ((long long)(n) * 3 + (c)) * np)
    long double xr = 0, xi = 0;
    if (!g->psi_ready) { advance_psiB(g); g->psi_ready = 1; }
    for (int64_t s = 0; s < nsteps; ++s) {
        for (int c = 0; c < 3; ++c) memcpy(EH(s, c), g->E[c], sizeof(double) * (size_t)np);
        if (g->level >= n0) {
            long double ph = (long double)freq * (long double)dt * (long double)g->level;
            ph -= floorl(ph);
            xr += g->E[comp][qp] * cosl(TWO_PI_L * ph) * dt;
            xi -= g->E[comp][qp] * sinl(TWO_PI_L * ph) * dt;
        }
        sample_probes(g);
        half_step_B(g);
        half_step_Js(g);
        advance_psiE(g);
        full_step_E(g);
        for (int c = 0; c < 3; ++c) memcpy(EP(s, c), g->E[c], sizeof(double) * (size_t)np);
        apply_sources(g, (double)(g->level + 1) * dt);
        half_step_Js(g);
        advance_psiB(g);
        half_step_B(g);
        g->level++;
    }
    for (int c = 0; c < 3; ++c) memcpy(EH(nsteps, c), g->E[c], sizeof(double) * (size_t)np);
    *Jout = (double)(xr * xr + xi * xi);
    /* adjoint sweep */
    adj_t A;
    adj_alloc(g, &A);
    double *ge[3], *gk[3];
    for (int c = 0; c < 3; ++c) { ge[c] = dalloc(np); gk[c] = dalloc(np); }
    for (int64_t s = nsteps - 1; s >= 0; --s) {
        double *Eb[3], *Ea[3], *En[3];
        for (int c = 0; c < 3; ++c) { Eb[c] = EH(s, c); Ea[c] = EP(s, c); En[c] = EH(s + 1, c); }
        adj_half_step_B(g, &A);                /* 5 */
        adj_advance_psiB(g, &A);
        adj_half_step_Js(g, &A, gk, En);       /* 4 */
        adj_full_step_E(g, &A, ge, Eb, Ea);    /* 3 */
        adj_advance_psiE(g, &A);
        adj_half_step_Js(g, &A, gk, Eb);       /* 2 */
        adj_half_step_B(g, &A);                /* 1 */
        if (s >= n0) {                          /* dJ/dE^n at the probe: 2 dt Re(conj(X) w^n) */
            long double ph = (long double)freq * (long double)dt * (long double)s;
            ph -= floorl(ph);
            A.E[comp][qp] += 2.0 * dt * (double)(xr * cosl(TWO_PI_L * ph) - xi * sinl(TWO_PI_L * ph));
        }
    }
    /* edges -> cells with the weights of build_coefficients */
    memset(g_eps, 0, sizeof(double) * (size_t)g->nc);
    memset(g_lam, 0, sizeof(double) * (size_t)g->nc);
    for (int c = 0; c < 3; ++c)
        for (int k = 0; k < g->N[2]; ++k)
            for (int j = 0; j < g->N[1]; ++j)
                for (int i = 0; i < g->N[0]; ++i) {
                    long long q = IX(g, i, j, k);
                    if (!g->updE[c][q]) continue;
                    int p[3] = {i, j, k};
                    int b1 = (c + 1) % 3, b2 = (c + 2) % 3, nk = 0;
                    long long cells[4];
                    for (int u = 0; u < 2; ++u)
                        for (int v = 0; v < 2; ++v) {
                            int cc[3];
                            cc[c] = p[c];
                            cc[b1] = wrapc(g, b1, p[b1] - u);
                            cc[b2] = wrapc(g, b2, p[b2] - v);
                            cells[2 * u + v] = CI(g, cc[0], cc[1], cc[2]);
                            nk += g->kap_c[cells[2 * u + v]] > 0.0;
                        }
                    for (int m = 0; m < 4; ++m) {
                        long long cm = cells[m];
                        g_eps[cm] += 0.25 * ge[c][q];
                        double kc = g->kap_c[cm];
                        if (kc > 0.0) {
                            double wgt = g->D.edge_rule == 1 ? 0.25 : 1.0 / nk;
                            double lam = 1.0 / sqrt(kc * MU0 * g->mu_c[cm]);
                            g_lam[cm] += gk[c][q] * wgt * (-2.0 * kc / lam);
                        }
                    }
                }
#undef EH
#undef EP
    for (int c = 0; c < 3; ++c) { free(ge[c]); free(gk[c]); }
    adj_free(&A);
    free(Eh);
    free(Ep);
    return 0;
}
