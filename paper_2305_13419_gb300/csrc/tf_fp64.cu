// tf_fp64.cu -- FP64 GPU stepper (the precision reference of the FP32 path).
//
// Runs Algorithm 1 (arXiv 2305.13419, Sec. 3) as its five sub-steps in FP64,
// SI units, on the integer-level state, in their order, one thread per
// storage point (two launches per step, three with Mur walls: see the
// fused launches below):
//   sample probes (E^n)
//   1  B  -= dt/2 curl E            (CPML memory psi_B as it stands)
//   2  Js += dt/2 kappa E           (superconducting edges)
//   3  psi_E update at the current H, then the theta step for E:
//      (eps + theta sigma dt) E' = (eps - (1 - theta) sigma dt) E + dt (curl H - Js)
//      soft sources at t^{n+1}; first-order Mur walls
//   4  Js += dt/2 kappa E
//   5  psi_B update at the new E, then B -= dt/2 curl E
// with edge values from cell values by the same rule as the FP32 path (eps:
// mean of the 4 cells; sigma, kappa: mean over the conducting /
// superconducting cells or plain mean; mu on a face: mean of its 2 cells) and
// the same Roden-Gedney CPML.  It exists to measure how far the FP32 fused
// step drifts from FP64 arithmetic; the FP64 pipe (1/64 of the FP32 rate on
// this part) bounds it.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "tf_internal.cuh"

namespace {

constexpr int kT = 256;
constexpr double kC0d = 299792458.0, kMu0d = 1.25663706212e-6, kEps0d = 8.8541878128e-12;

struct G64 {
    int n[3], N[3], per[3], bc[3], L[3], edge_rule;
    long long np;
    double d[3], id[3], dt, theta, murM;   // id: 1 / d
    double *E[3], *B[3], *J[3], *Eold[3];
    double *psiB[3][3], *psiE[3][3];
    double *caE[3], *cbE[3], *kapE[3], *imuF[3];   // theta-scheme coefficients of step 3, kappa, 1 / mu_face
    double *pbE[3], *pcE[3], *pbB[3], *pcB[3];
    const double *eps_c, *mu_c, *kap_c, *sig_c;
};

__device__ __forceinline__ long long ix(const G64& g, int i, int j, int k) {
    return ((long long)k * g.N[1] + j) * g.N[0] + i;
}
__device__ __forceinline__ long long ci(const G64& g, int i, int j, int k) {
    return ((long long)k * g.n[1] + j) * g.n[0] + i;
}
__device__ __forceinline__ int up(const G64& g, int a, int p) { return p + 1 < g.N[a] ? p + 1 : (g.per[a] ? 0 : p); }
__device__ __forceinline__ int dn(const G64& g, int a, int p) { return p > 0 ? p - 1 : (g.per[a] ? g.N[a] - 1 : p); }
__device__ __forceinline__ double sgn(int c, int a) { return ((a - c + 3) % 3 == 1) ? 1.0 : -1.0; }
// component c of E (is_b = false) or B (true) at p is advanced
__device__ __forceinline__ bool advanced(const G64& g, int c, bool is_b, const int p[3]) {
    for (int a = 0; a < 3; ++a) {
        if (g.per[a]) continue;
        const bool half = is_b ? (a != c) : (a == c);
        if (half) {
            if (p[a] >= g.n[a]) return false;
        } else if (p[a] < 1 || p[a] > g.n[a] - 1) {
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ bool slab(const G64& g, int a, int p) {
    return g.L[a] > 0 && (p < g.L[a] || p >= g.n[a] - g.L[a]);
}
__device__ __forceinline__ bool point(const G64& g, long long t, int p[3]) {
    if (t >= g.np) return false;
    p[0] = (int)(t % g.N[0]);
    p[1] = (int)((t / g.N[0]) % g.N[1]);
    p[2] = (int)(t / ((long long)g.N[0] * g.N[1]));
    return true;
}
#define POINT_OR_RETURN                                        \
    int p[3];                                                  \
    const long long t = (long long)blockIdx.x * kT + threadIdx.x; \
    if (!point(g, t, p)) return;

// edge and face coefficients from the cell maps
__global__ void k64_coeffs(G64 g) {
    POINT_OR_RETURN
    for (int c = 0; c < 3; ++c) {
        double eps = kEps0d, sig = 0.0, kap = 0.0, mu = kMu0d;
        if (advanced(g, c, false, p)) {
            const int b1 = (c + 1) % 3, b2 = (c + 2) % 3;
            double se = 0, ss = 0, sk = 0;
            int ns = 0, nk = 0;
            for (int u = 0; u < 2; ++u)
                for (int v = 0; v < 2; ++v) {
                    int cc[3];
                    cc[c] = p[c];
                    cc[b1] = p[b1] - u < 0 ? p[b1] - u + g.n[b1] : p[b1] - u;
                    cc[b2] = p[b2] - v < 0 ? p[b2] - v + g.n[b2] : p[b2] - v;
                    const long long m = ci(g, cc[0], cc[1], cc[2]);
                    se += g.eps_c[m];
                    ss += g.sig_c[m];
                    sk += g.kap_c[m];
                    ns += g.sig_c[m] > 0.0;
                    nk += g.kap_c[m] > 0.0;
                }
            eps = kEps0d * se / 4.0;
            if (g.edge_rule == TF_EDGE_PLAIN_MEAN) {
                sig = ss / 4.0;
                kap = sk / 4.0;
            } else {
                sig = ns ? ss / ns : 0.0;
                kap = nk ? sk / nk : 0.0;
            }
        }
        if (advanced(g, c, true, p)) {
            double sm = 0;
            for (int u = 0; u < 2; ++u) {
                int cc[3] = {p[0], p[1], p[2]};
                cc[c] = p[c] - u < 0 ? p[c] - u + g.n[c] : p[c] - u;
                sm += g.mu_c[ci(g, cc[0], cc[1], cc[2])];
            }
            mu = kMu0d * sm / 2.0;
        }
        // step 3: E' = ca E + cb (curl H - J), ca = (1 - (1-theta) s) / (1 + theta s),
        // cb = (dt / eps) / (1 + theta s), s = sigma dt / eps (formed once, not per step)
        const double sd = sig * g.dt / eps, den = 1.0 + g.theta * sd;
        g.caE[c][t] = (1.0 - (1.0 - g.theta) * sd) / den;
        g.cbE[c][t] = g.dt / eps / den;
        g.kapE[c][t] = kap;
        g.imuF[c][t] = 1.0 / mu;
    }
}

__device__ __forceinline__ double dE(const G64& g, int e, int a, const int p[3]) {
    int q[3] = {p[0], p[1], p[2]};
    q[a] = up(g, a, p[a]);
    return (g.E[e][ix(g, q[0], q[1], q[2])] - g.E[e][ix(g, p[0], p[1], p[2])]) * g.id[a];
}
__device__ __forceinline__ double dH(const G64& g, int h, int a, const int p[3]) {
    int q[3] = {p[0], p[1], p[2]};
    q[a] = dn(g, a, p[a]);
    const long long i0 = ix(g, p[0], p[1], p[2]), i1 = ix(g, q[0], q[1], q[2]);
    // the two products rounded on their own (no fused multiply-add), so that
    // equal neighbours give an exact zero as the oracle's divisions do
    return (__dmul_rn(g.B[h][i0], g.imuF[h][i0]) - __dmul_rn(g.B[h][i1], g.imuF[h][i1])) * g.id[a];
}

__global__ void k64_psi_B(G64 g) {
    POINT_OR_RETURN
    for (int c = 0; c < 3; ++c) {
        if (!advanced(g, c, true, p)) continue;
        for (int a = 0; a < 3; ++a)
            if (a != c && g.psiB[c][a] && slab(g, a, p[a]))
                g.psiB[c][a][t] = g.pbB[a][p[a]] * g.psiB[c][a][t] + g.pcB[a][p[a]] * dE(g, 3 - c - a, a, p);
    }
}

struct Src64 {
    int n, comp[TF_MAX_SOURCES], lo[TF_MAX_SOURCES][3], hi[TF_MAX_SOURCES][3];
    double v[TF_MAX_SOURCES];
};

struct Prb64 {
    int n, comp[TF_MAX_PROBES], nfreq[TF_MAX_PROBES];
    long long q[TF_MAX_PROBES], n0[TF_MAX_PROBES];
    const double* fdt;   // [probe][TF_MAX_FREQS]
    double *re, *im;
};

// Fused launches of the same sub-steps (one thread per point; every value a
// thread reads from another point is one that no thread of the launch
// writes):
//   k64_steps_1_2   probes at level n, step 1 (B half), step 2 (Js half)
//   k64_step_3_4    step 3 (psi_E, theta step for E), soft sources, step 4
//                   (Js half with the new E; the Mur walls carry no Js)
//   k64_steps_5_1_2 step 5 of step n (psi_B at the new E, B half) and, if
//                   `next`, steps 1 and 2 of step n+1 with the probes at
//                   level n+1 (E is not written, so both B halves use the
//                   same curl and psi_B)
// Walls of the Mur kind keep E^n of their planes and of the planes next to
// them in Eold (k64_mur_walls then applies the Mur update).
__device__ __forceinline__ void keep_mur_old(const G64& g, const int p[3], long long t) {
    if (g.bc[2] != TF_BC_MUR) return;
    if (p[2] == 0 || p[2] == 1 || p[2] == g.n[2] - 1 || p[2] == g.n[2])
        for (int c = 0; c < 2; ++c) g.Eold[c][t] = g.E[c][t];
}
__device__ __forceinline__ void probes_at(const G64& g, const Prb64& R, long long level) {
    if (blockIdx.x < (unsigned)R.n && threadIdx.x < TF_MAX_FREQS) {
        const int pr = blockIdx.x, k = threadIdx.x;
        if (k < R.nfreq[pr] && level >= R.n0[pr]) {
            const double s = g.E[R.comp[pr]][R.q[pr]];
            double ph = R.fdt[pr * TF_MAX_FREQS + k] * (double)level;
            ph -= floor(ph);
            double sn, cs;
            sincospi(2.0 * ph, &sn, &cs);
            R.re[pr * TF_MAX_FREQS + k] += s * cs * g.dt;
            R.im[pr * TF_MAX_FREQS + k] -= s * sn * g.dt;
        }
    }
}
__device__ __forceinline__ double curl_E_B(const G64& g, int c, const int p[3], long long t) {
    double r = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (a == c) continue;
        double v = dE(g, 3 - c - a, a, p);
        if (g.psiB[c][a]) v += g.psiB[c][a][t];
        r += sgn(c, a) * v;
    }
    return r;
}

__global__ void k64_steps_1_2(G64 g, Prb64 R, long long level) {
    probes_at(g, R, level);
    POINT_OR_RETURN
    keep_mur_old(g, p, t);
    for (int c = 0; c < 3; ++c)
        if (advanced(g, c, true, p)) g.B[c][t] -= 0.5 * g.dt * curl_E_B(g, c, p, t);
    for (int c = 0; c < 3; ++c)
        if (advanced(g, c, false, p) && g.kapE[c][t] > 0.0) g.J[c][t] += 0.5 * g.dt * g.kapE[c][t] * g.E[c][t];
}

__global__ void k64_step_3_4(G64 g, Src64 S) {
    POINT_OR_RETURN
    for (int c = 0; c < 3; ++c) {
        if (!advanced(g, c, false, p)) continue;
        for (int a = 0; a < 3; ++a)
            if (a != c && g.psiE[c][a] && slab(g, a, p[a]))
                g.psiE[c][a][t] = g.pbE[a][p[a]] * g.psiE[c][a][t] + g.pcE[a][p[a]] * dH(g, 3 - c - a, a, p);
        double r = 0.0;
        for (int a = 0; a < 3; ++a) {
            if (a == c) continue;
            double v = dH(g, 3 - c - a, a, p);
            if (g.psiE[c][a]) v += g.psiE[c][a][t];
            r += sgn(c, a) * v;
        }
        double e = g.caE[c][t] * g.E[c][t] + g.cbE[c][t] * (r - g.J[c][t]);
        for (int s = 0; s < S.n; ++s)
            if (S.comp[s] == c && p[0] >= S.lo[s][0] && p[0] < S.hi[s][0] && p[1] >= S.lo[s][1] &&
                p[1] < S.hi[s][1] && p[2] >= S.lo[s][2] && p[2] < S.hi[s][2])
                e += S.v[s];
        g.E[c][t] = e;
        if (g.kapE[c][t] > 0.0) g.J[c][t] += 0.5 * g.dt * g.kapE[c][t] * e;
    }
}

__global__ void k64_steps_5_1_2(G64 g, Prb64 R, long long level_next, int next) {
    if (next) probes_at(g, R, level_next);
    POINT_OR_RETURN
    if (next) keep_mur_old(g, p, t);
    for (int c = 0; c < 3; ++c) {
        if (!advanced(g, c, true, p)) continue;
        for (int a = 0; a < 3; ++a)
            if (a != c && g.psiB[c][a] && slab(g, a, p[a]))
                g.psiB[c][a][t] = g.pbB[a][p[a]] * g.psiB[c][a][t] + g.pcB[a][p[a]] * dE(g, 3 - c - a, a, p);
        const double r = curl_E_B(g, c, p, t);
        double b = g.B[c][t] - 0.5 * g.dt * r;
        if (next) b -= 0.5 * g.dt * r;
        g.B[c][t] = b;
    }
    if (next)
        for (int c = 0; c < 3; ++c)
            if (advanced(g, c, false, p) && g.kapE[c][t] > 0.0) g.J[c][t] += 0.5 * g.dt * g.kapE[c][t] * g.E[c][t];
}

// the Mur walls (planes 0 and n of z; blockIdx.y picks the wall)
__global__ void k64_mur_walls(G64 g) {
    const long long t2 = (long long)blockIdx.x * kT + threadIdx.x;
    const long long np2 = (long long)g.N[0] * g.N[1];
    if (t2 >= np2) return;
    const int p[3] = {(int)(t2 % g.N[0]), (int)(t2 / g.N[0]), blockIdx.y ? g.n[2] : 0};
    const long long t = ix(g, p[0], p[1], p[2]);
    for (int c = 0; c < 2; ++c) {
        bool ok = true;
        for (int a = 0; a < 2 && ok; ++a) {
            if (g.per[a]) continue;
            if (a == c) ok = p[a] < g.n[a];
            else ok = p[a] >= 1 && p[a] <= g.n[a] - 1;
        }
        if (!ok) continue;
        const int ki = p[2] == 0 ? 1 : g.n[2] - 1;
        const long long qi = ix(g, p[0], p[1], ki);
        g.E[c][t] = g.Eold[c][qi] + g.murM * (g.E[c][qi] - g.Eold[c][t]);
    }
}

}  // namespace

struct tf64_ctx {
    tf_grid_desc desc;
    G64 g;
    cudaStream_t st;
    double* cells;       // eps, mu, kap, sig per cell (device)
    Prb64 R;
    double freqs[TF_MAX_PROBES][TF_MAX_FREQS];
    int nsrc;
    struct {
        int comp, lo[3], hi[3], kind;
        double amp, f, t0, tw;
    } src[TF_MAX_SOURCES];
    long long level;
    int psi_ready;
};

namespace {

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

struct L64 {
    int N[3];
    long long np, nc;
    int ncpml;
    size_t bytes;
};

L64 lay(const tf_grid_desc* d) {
    L64 L{};
    const int n[3] = {d->nx, d->ny, d->nz};
    L.ncpml = 0;
    for (int a = 0; a < 3; ++a) {
        L.N[a] = n[a] + (d->bc[a].kind == TF_BC_PERIODIC ? 0 : 1);
        if (d->bc[a].kind == TF_BC_CPML) ++L.ncpml;
    }
    L.np = (long long)L.N[0] * L.N[1] * L.N[2];
    L.nc = (long long)n[0] * n[1] * n[2];
    const size_t fb = al(sizeof(double) * (size_t)L.np);
    L.bytes = (12 + 12 + 4 * (size_t)L.ncpml) * fb + 4 * al(sizeof(double) * (size_t)L.nc) +
              12 * al(sizeof(double) * (size_t)(L.N[0] + L.N[1] + L.N[2])) +
              3 * al(sizeof(double) * TF_MAX_PROBES * TF_MAX_FREQS);
    return L;
}

unsigned blocks(const G64& g) { return (unsigned)((g.np + kT - 1) / kT); }

double wave64(int kind, double amp, double f, double t0, double tw, double t) {
    const double env = exp(-(t - t0) * (t - t0) / (2.0 * tw * tw));
    const double w = 6.283185307179586476925286766559 * f * t;
    if (kind == TF_SRC_GAUSS) return amp * env;
    if (kind == TF_SRC_SIN) return amp * sin(w);
    return amp * env * sin(w);
}

#define C64(x)                                   \
    do {                                         \
        if ((x) != cudaSuccess) return TF_ECUDA; \
    } while (0)

}  // namespace

extern "C" {

size_t tf64_workspace_size(const tf_grid_desc* desc) {
    if (!desc || desc->nx < 1 || desc->ny < 1 || desc->nz < 1) return 0;
    return lay(desc).bytes;
}

tf_status tf64_create(const tf_grid_desc* d, void* ws, size_t bytes, tf64_handle* out) {
    if (!d || !ws || !out) return TF_EINVAL;
    *out = nullptr;
    const int n[3] = {d->nx, d->ny, d->nz};
    const double h[3] = {d->dx, d->dy, d->dz};
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 1 || !(h[a] > 0)) return TF_EINVAL;
        const tf_bc& b = d->bc[a];
        if (b.kind < TF_BC_PERIODIC || b.kind > TF_BC_CPML) return TF_EINVAL;
        if (b.kind == TF_BC_MUR && a != 2) return TF_ENOTSUP;
        if (b.kind == TF_BC_CPML && (b.cpml_cells < 1 || 2 * b.cpml_cells > n[a])) return TF_EINVAL;
    }
    if (!(d->theta >= 0.5 && d->theta <= 1.0) || (!(d->dt > 0) && !(d->courant > 0))) return TF_EINVAL;
    if (d->edge_rule != TF_EDGE_CONDUCTOR_MEAN && d->edge_rule != TF_EDGE_PLAIN_MEAN) return TF_EINVAL;
    if (d->max_probes < 0 || d->max_probes > TF_MAX_PROBES) return TF_EINVAL;
    const L64 L = lay(d);
    if (bytes < L.bytes || ((uintptr_t)ws & 255)) return TF_ENOMEM;
    tf64_ctx* c = new (std::nothrow) tf64_ctx();
    if (!c) return TF_ENOMEM;
    c->desc = *d;
    c->st = (cudaStream_t)d->stream;
    G64& g = c->g;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = n[a];
        g.N[a] = L.N[a];
        g.per[a] = d->bc[a].kind == TF_BC_PERIODIC;
        g.bc[a] = d->bc[a].kind;
        g.L[a] = d->bc[a].kind == TF_BC_CPML ? d->bc[a].cpml_cells : 0;
        g.d[a] = h[a];
        g.id[a] = 1.0 / h[a];
    }
    g.np = L.np;
    g.edge_rule = d->edge_rule;
    g.dt = d->dt > 0 ? d->dt : d->courant / (kC0d * sqrt(1 / (h[0] * h[0]) + 1 / (h[1] * h[1]) + 1 / (h[2] * h[2])));
    g.theta = d->theta;
    g.murM = (kC0d * g.dt - h[2]) / (kC0d * g.dt + h[2]);
    char* b = (char*)ws;
    const size_t fb = al(sizeof(double) * (size_t)L.np);
    auto take = [&](size_t nb) { char* r = b; b += nb; return r; };
    for (int k = 0; k < 3; ++k) {
        g.E[k] = (double*)take(fb); g.B[k] = (double*)take(fb); g.J[k] = (double*)take(fb);
        g.Eold[k] = (double*)take(fb);
        g.caE[k] = (double*)take(fb); g.cbE[k] = (double*)take(fb); g.kapE[k] = (double*)take(fb);
        g.imuF[k] = (double*)take(fb);
    }
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) {
            g.psiB[k][a] = nullptr;
            g.psiE[k][a] = nullptr;
        }
    for (int a = 0; a < 3; ++a) {
        if (d->bc[a].kind != TF_BC_CPML) continue;
        for (int k = 0; k < 3; ++k) {
            if (k == a) continue;
            g.psiB[k][a] = (double*)take(fb);
            g.psiE[k][a] = (double*)take(fb);
        }
    }
    const size_t cb = al(sizeof(double) * (size_t)L.nc);
    c->cells = (double*)take(4 * cb);
    g.eps_c = c->cells;
    g.mu_c = (const double*)((char*)c->cells + cb);
    g.kap_c = (const double*)((char*)c->cells + 2 * cb);
    g.sig_c = (const double*)((char*)c->cells + 3 * cb);
    const size_t pb = al(sizeof(double) * (size_t)(L.N[0] + L.N[1] + L.N[2]));
    double* prof = (double*)take(12 * pb);
    const size_t pbytes = al(sizeof(double) * TF_MAX_PROBES * TF_MAX_FREQS);
    c->R.fdt = (const double*)take(pbytes);
    c->R.re = (double*)take(pbytes);
    c->R.im = (double*)take(pbytes);
    c->R.n = 0;
    // zero state, vacuum cells, CPML profiles (Roden-Gedney, as the FP32 path)
    if (cudaMemsetAsync(ws, 0, L.bytes, c->st) != cudaSuccess) { delete c; return TF_ECUDA; }
    const size_t nprof = (size_t)(L.N[0] + L.N[1] + L.N[2]);
    double* hp = (double*)calloc(12 * nprof, sizeof(double));
    if (!hp) { delete c; return TF_ENOMEM; }
    size_t off = 0;
    for (int a = 0; a < 3; ++a) {
        double* q[4];
        for (int m = 0; m < 4; ++m) q[m] = hp + (size_t)(4 * a + m) * nprof;
        for (int pp = 0; pp < L.N[a]; ++pp)
            for (int half = 0; half < 2; ++half) {
                double bb = 0.0, cc = 0.0;
                if (d->bc[a].kind == TF_BC_CPML) {
                    const double Lc = d->bc[a].cpml_cells, x = pp + 0.5 * half;
                    double rho = 0.0;
                    if (x < Lc) rho = (Lc - x) / Lc;
                    else if (x > n[a] - Lc) rho = (x - (n[a] - Lc)) / Lc;
                    if (rho > 0.0) {
                        const double s = d->bc[a].cpml_sigma_max * pow(rho, d->bc[a].cpml_order);
                        const double alpha = d->bc[a].cpml_alpha_max * (1.0 - rho);
                        bb = exp(-(s + alpha) * g.dt / kEps0d);
                        cc = (s + alpha > 0.0) ? s * (bb - 1.0) / (s + alpha) : 0.0;
                    }
                }
                q[2 * half][pp] = bb;
                q[2 * half + 1][pp] = cc;
            }
        g.pbE[a] = prof + (size_t)(4 * a + 0) * nprof;
        g.pcE[a] = prof + (size_t)(4 * a + 1) * nprof;
        g.pbB[a] = prof + (size_t)(4 * a + 2) * nprof;
        g.pcB[a] = prof + (size_t)(4 * a + 3) * nprof;
        off += 4 * nprof;
    }
    cudaError_t e = cudaMemcpyAsync(prof, hp, sizeof(double) * 12 * nprof, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    free(hp);
    if (e != cudaSuccess) { delete c; return TF_ECUDA; }
    *out = c;
    return tf64_set_materials(c, nullptr, nullptr, nullptr, nullptr);
}

tf_status tf64_destroy(tf64_handle h) {
    if (!h) return TF_EINVAL;
    delete h;
    return TF_OK;
}

tf_status tf64_set_materials(tf64_handle h, const double* eps_r, const double* mu_r, const double* lambda_L,
                             const double* sigma) {
    if (!h) return TF_EINVAL;
    if (h->level != 0 || h->psi_ready) return TF_ESTATE;
    G64& g = h->g;
    const long long nc = (long long)g.n[0] * g.n[1] * g.n[2];
    double* hc = (double*)malloc(sizeof(double) * 4 * (size_t)nc);
    if (!hc) return TF_ENOMEM;
    for (long long m = 0; m < nc; ++m) {
        const double e = eps_r ? eps_r[m] : 1.0, u = mu_r ? mu_r[m] : 1.0;
        const double l = lambda_L ? lambda_L[m] : 0.0, s = sigma ? sigma[m] : 0.0;
        if (!(e > 0) || !(u > 0) || !(s >= 0) || l < 0) { free(hc); return TF_EINVAL; }
        hc[m] = e;
        hc[nc + m] = u;
        hc[2 * nc + m] = (l > 0 && isfinite(l)) ? 1.0 / (l * l * kMu0d * u) : 0.0;
        hc[3 * nc + m] = s;
    }
    const size_t cb = al(sizeof(double) * (size_t)nc);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync((char*)h->cells + k * cb, hc + (size_t)k * nc, sizeof(double) * nc,
                            cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    free(hc);
    if (e != cudaSuccess) return TF_ECUDA;
    k64_coeffs<<<blocks(g), kT, 0, h->st>>>(g);
    C64(cudaGetLastError());
    C64(cudaStreamSynchronize(h->st));
    return TF_OK;
}

tf_status tf64_set_field(tf64_handle h, int comp, const double* src) {
    if (!h || !src || comp < 0 || comp > 8) return TF_EINVAL;
    if (h->level != 0 || h->psi_ready) return TF_ESTATE;
    G64& g = h->g;
    double* dst = comp < 3 ? g.E[comp] : comp < 6 ? g.B[comp - 3] : g.J[comp - 6];
    C64(cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)g.np, cudaMemcpyHostToDevice, h->st));
    C64(cudaStreamSynchronize(h->st));
    return TF_OK;
}

tf_status tf64_add_source(tf64_handle h, int comp, const int lo[3], const int hi[3], double amp, int kind, double f,
                          double t0, double tw, int* id) {
    if (!h || !lo || !hi || comp < 0 || comp > 2 || kind < TF_SRC_GAUSS || kind > TF_SRC_GAUSS_SIN) return TF_EINVAL;
    if (h->nsrc >= TF_MAX_SOURCES || (kind != TF_SRC_SIN && !(tw > 0))) return TF_EINVAL;
    auto& s = h->src[h->nsrc];
    s.comp = comp;
    for (int a = 0; a < 3; ++a) {
        s.lo[a] = lo[a] < 0 ? 0 : lo[a];
        s.hi[a] = hi[a] > h->g.N[a] ? h->g.N[a] : hi[a];
    }
    s.kind = kind; s.amp = amp; s.f = f; s.t0 = t0; s.tw = tw;
    if (id) *id = h->nsrc;
    h->nsrc++;
    return TF_OK;
}

tf_status tf64_add_probe(tf64_handle h, int comp, const int p[3], const double* freqs, int nfreq, int64_t n0,
                         int* id) {
    if (!h || !p || comp < 0 || comp > 2 || nfreq < 0 || nfreq > TF_MAX_FREQS || (nfreq && !freqs)) return TF_EINVAL;
    if (h->R.n >= h->desc.max_probes) return TF_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (p[a] < 0 || p[a] >= h->g.N[a]) return TF_EINVAL;
    const int k = h->R.n;
    double fdt[TF_MAX_FREQS] = {0};
    for (int f = 0; f < nfreq; ++f) {
        h->freqs[k][f] = freqs[f];
        fdt[f] = freqs[f] * h->g.dt;
    }
    C64(cudaMemcpyAsync((double*)h->R.fdt + k * TF_MAX_FREQS, fdt, sizeof(fdt), cudaMemcpyHostToDevice, h->st));
    C64(cudaStreamSynchronize(h->st));
    h->R.nfreq[k] = nfreq;
    h->R.comp[k] = comp;
    h->R.q[k] = ((long long)p[2] * h->g.N[1] + p[1]) * h->g.N[0] + p[0];
    h->R.n0[k] = n0;
    h->R.n++;
    if (id) *id = k;
    return TF_OK;
}

tf_status tf64_step(tf64_handle h, int64_t nsteps) {
    if (!h || nsteps < 0) return TF_EINVAL;
    G64& g = h->g;
    const unsigned nb = blocks(g);
    if (!h->psi_ready && nsteps > 0) {   // psi_B at level 0 from zero history
        k64_psi_B<<<nb, kT, 0, h->st>>>(g);
        h->psi_ready = 1;
    }
    Src64 S;
    S.n = h->nsrc;
    for (int s = 0; s < h->nsrc; ++s) {
        S.comp[s] = h->src[s].comp;
        for (int a = 0; a < 3; ++a) { S.lo[s][a] = h->src[s].lo[a]; S.hi[s][a] = h->src[s].hi[a]; }
    }
    const bool mur = g.bc[2] == TF_BC_MUR;
    const unsigned nbw = (unsigned)(((long long)g.N[0] * g.N[1] + kT - 1) / kT);
    // two or three launches per step: steps 1 and 2 open the run, then per
    // step the E launch (steps 3 and 4), the Mur walls, and the B launch
    // (step 5, fused with steps 1 and 2 of the next step but the last)
    if (nsteps > 0) k64_steps_1_2<<<nb, kT, 0, h->st>>>(g, h->R, h->level);
    for (int64_t s = 0; s < nsteps; ++s) {
        const double t1 = (double)(h->level + 1) * g.dt;
        for (int q = 0; q < h->nsrc; ++q)
            S.v[q] = wave64(h->src[q].kind, h->src[q].amp, h->src[q].f, h->src[q].t0, h->src[q].tw, t1);
        k64_step_3_4<<<nb, kT, 0, h->st>>>(g, S);
        if (mur) k64_mur_walls<<<dim3(nbw, 2), kT, 0, h->st>>>(g);
        const int next = s + 1 < nsteps;
        k64_steps_5_1_2<<<nb, kT, 0, h->st>>>(g, h->R, h->level + 1, next);
        C64(cudaGetLastError());
        h->level++;
    }
    return TF_OK;
}

tf_status tf64_sync(tf64_handle h) {
    if (!h) return TF_EINVAL;
    C64(cudaStreamSynchronize(h->st));
    return TF_OK;
}

tf_status tf64_read_field(tf64_handle h, int comp, double* dst) {
    if (!h || !dst || comp < 0 || comp > 8) return TF_EINVAL;
    G64& g = h->g;
    const double* src = comp < 3 ? g.E[comp] : comp < 6 ? g.B[comp - 3] : g.J[comp - 6];
    C64(cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)g.np, cudaMemcpyDeviceToHost, h->st));
    C64(cudaStreamSynchronize(h->st));
    return TF_OK;
}

tf_status tf64_read_probe_dft(tf64_handle h, int id, double* re, double* im) {
    if (!h || !re || !im || id < 0 || id >= h->R.n) return TF_EINVAL;
    const int nf = h->R.nfreq[id];
    C64(cudaMemcpyAsync(re, h->R.re + id * TF_MAX_FREQS, sizeof(double) * nf, cudaMemcpyDeviceToHost, h->st));
    C64(cudaMemcpyAsync(im, h->R.im + id * TF_MAX_FREQS, sizeof(double) * nf, cudaMemcpyDeviceToHost, h->st));
    C64(cudaStreamSynchronize(h->st));
    return TF_OK;
}

tf_status tf64_get_time(tf64_handle h, int64_t* n, double* dt) {
    if (!h) return TF_EINVAL;
    if (n) *n = h->level;
    if (dt) *dt = h->g.dt;
    return TF_OK;
}

}  // extern "C"

namespace {
constexpr int kFmaChains = 8, kFmaThreads = 256, kFmaBlocksPerSm = 4;
// FP64 FMA throughput: kFmaChains independent chains per thread, the results
// written out so that none of the work can be dropped
__global__ void __launch_bounds__(kFmaThreads) k64_fma_rate(double* out, int iters, double a, double b) {
    const int t = blockIdx.x * kFmaThreads + threadIdx.x;
    double x[kFmaChains];
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) x[c] = 1e-3 * (t + c);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kFmaChains; ++c) x[c] = fma(x[c], a, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) s += x[c];
    out[t] = s;
}
}  // namespace

extern "C" size_t tf64_fma_rate_scratch(void) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return sizeof(double) * (size_t)sms * kFmaBlocksPerSm * kFmaThreads;
}

extern "C" tf_status tf64_fma_rate(void* dev_scratch, size_t bytes, int iters, void* stream, double* gflops) {
    if (!dev_scratch || !gflops || iters < 1) return TF_EINVAL;
    int dev = 0, sms = 0;
    C64(cudaGetDevice(&dev));
    C64(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * kFmaBlocksPerSm;
    if (bytes < sizeof(double) * (size_t)blocks * kFmaThreads) return TF_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    C64(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return TF_ECUDA;
    }
    k64_fma_rate<<<blocks, kFmaThreads, 0, st>>>((double*)dev_scratch, iters, 0.999999, 1e-7);   // warm-up
    cudaEventRecord(e0, st);
    k64_fma_rate<<<blocks, kFmaThreads, 0, st>>>((double*)dev_scratch, iters, 0.999999, 1e-7);
    cudaEventRecord(e1, st);
    float ms = 0.f;
    const cudaError_t e = cudaEventSynchronize(e1) == cudaSuccess ? cudaEventElapsedTime(&ms, e0, e1) : cudaErrorUnknown;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess || !(ms > 0.f)) return TF_ECUDA;
    *gflops = 2.0 * kFmaChains * (double)iters * blocks * kFmaThreads / (ms * 1e-3) / 1e9;
    return TF_OK;
}
