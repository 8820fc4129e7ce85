// tf_kernels.cu -- CUDA kernels of the two-fluid Yee library for sm_103a.
//
// The per-step kernels besides the fused step of tf_step.cu:
// set-up and read-back kernels (material scaling, level-0 priming
// B^{-1/2} = B^0 + dt/2 curl E^0 and Js^{-1/2} = Js^0 - dt/2 kappa E^0, and
// integer-level read-back B^n = B^{n-1/2} - dt/2 curl E^n,
// Js^n = Js^{n-1/2} + dt/2 kappa E^n).
#include <math.h>

#include "tf_internal.cuh"

namespace tf {

namespace {

constexpr int BX = 32, BY = 4, BZ = 2;  // 256-thread blocks, x rows coalesced

__device__ __forceinline__ bool point_of(const Params& P, int& i, int& j, int& k) {
    i = blockIdx.x * BX + threadIdx.x;
    j = blockIdx.y * BY + threadIdx.y;
    k = blockIdx.z * BZ + threadIdx.z;
    return i < P.N[0] && j < P.N[1] && k < P.N[2];
}

inline dim3 grid_of(const Params& P) {
    return dim3((P.N[0] + BX - 1) / BX, (P.N[1] + BY - 1) / BY, (P.N[2] + BZ - 1) / BZ);
}

// component cb of curl E at the B_cb position of p (scaled units, r_a folded
// in), with the CPML memory advanced to the current E without storing it
__device__ __forceinline__ float curl_E_peek(const Params& P, int cb, const int p[3], long long q) {
    float acc = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a == cb) continue;
        const int e = 3 - cb - a;
        int pn[3] = {p[0], p[1], p[2]};
        pn[a] = nxt(P, a, p[a]);
        const float dE = P.E[e][lin(P, pn[0], pn[1], pn[2])] - P.E[e][q];
        float t = P.r[a] * dE;
        if (P.psiB[cb][a] && in_slab(P, a, p[a]))
            t += P.pbB[a][p[a]] * P.psiB[cb][a][q] + P.pcB[a][p[a]] * dE;
        acc += curl_sign(cb, a) * t;
    }
    return acc;
}

}  // namespace

// ------------------------------------------------------------ set-up
__global__ void k_fill(float* p, long long n, float v) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (; t < n; t += (long long)gridDim.x * blockDim.x) p[t] = v;
}

__global__ void k_convert_materials(Params P, const float* eps_r, const float* mu_r, const float* lam,
                                    const float* sigma, double dt, float* eps, float* sig, float* kap,
                                    float* mu, unsigned* mm) {
    const long long ncell = (long long)P.n[0] * P.n[1] * P.n[2];
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    unsigned a_bits = 0, b_bits = 0, nonuni = 0;
    if (t < ncell) {
        const int i = (int)(t % P.n[0]);
        const long long r = t / P.n[0];
        const int j = (int)(r % P.n[1]);
        const int k = (int)(r / P.n[1]);
        const double e = eps_r ? (double)eps_r[t] : 1.0, u = mu_r ? (double)mu_r[t] : 1.0;
        const double l = lam ? (double)lam[t] : 0.0, s = sigma ? (double)sigma[t] : 0.0;
        if (!(e > 0.0) || !(u > 0.0) || !(s >= 0.0) || !(l >= 0.0) || isinf(e) || isinf(u) || isinf(s))
            atomicOr(P.status, kStatusBadMaterial);
        const double c0dt = kC0 * dt;
        // first London equation: kt = dt^2/(eps0 lambda^2 mu0 mu_r) = (c0 dt / lambda)^2 / mu_r
        const double kt = (l > 0.0 && isfinite(l)) ? (c0dt / l) * (c0dt / l) / u : 0.0;
        const long long q = lin(P, i, j, k);
        eps[q] = (float)e;
        sig[q] = (float)(s * dt / kEps0);
        kap[q] = (float)kt;
        mu[q] = (float)u;
        if (e > 0.0 && u > 0.0) {
            a_bits = __float_as_uint((float)(1.0 / (e * u)));
            b_bits = __float_as_uint((float)(kt / (4.0 * e)));
        }
        nonuni = (u != 1.0);
    }
    // non-negative floats order like their bit patterns
    a_bits = __reduce_max_sync(0xffffffffu, a_bits);
    b_bits = __reduce_max_sync(0xffffffffu, b_bits);
    nonuni = __reduce_or_sync(0xffffffffu, nonuni);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(mm + 0, a_bits);
        atomicMax(mm + 1, b_bits);
        if (nonuni) atomicOr(mm + 2, 1u);
    }
}

__global__ void k_set_field(Params P, int comp, const float* dense, float* dst, double scale) {
    const long long tot = (long long)P.N[0] * P.N[1] * P.N[2];
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= tot) return;
    const int i = (int)(t % P.N[0]);
    const long long r = t / P.N[0];
    const int p[3] = {i, (int)(r % P.N[1]), (int)(r / P.N[1])};
    bool keep;
    if (comp < 3) {
        keep = upd_E(P, comp, p) || mur_E(P, comp, p);
    } else if (comp < 6) {
        keep = upd_B(P, comp - 3, p);
    } else {   // Js lives on superconducting edges only
        keep = upd_E(P, comp - 6, p);
        if (keep) {
            float eps, st, kt;
            edge_material(P, comp - 6, p, eps, st, kt);
            keep = kt > 0.f;
        }
    }
    dst[lin(P, p[0], p[1], p[2])] = keep ? (float)((double)dense[t] * scale) : 0.f;
}

// after new materials: Js is zero on every edge that is not superconducting
__global__ void k_mask_js(Params P) {
    int i, j, k;
    if (!point_of(P, i, j, k)) return;
    const int p[3] = {i, j, k};
    const long long q = lin(P, i, j, k);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        bool keep = upd_E(P, c, p);
        if (keep) {
            float eps, st, kt;
            edge_material(P, c, p, eps, st, kt);
            keep = kt > 0.f;
        }
        if (!keep) P.J[c][q] = 0.f;
    }
}

__global__ void k_prime(Params P) {
    int i, j, k;
    if (!point_of(P, i, j, k)) return;
    const int p[3] = {i, j, k};
    const long long q = lin(P, i, j, k);
#pragma unroll
    for (int cb = 0; cb < 3; ++cb)
        if (upd_B(P, cb, p)) P.B[cb][q] += 0.5f * curl_E_peek(P, cb, p, q);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float jt = 0.f;
        if (upd_E(P, c, p)) {
            float eps, st, kt;
            edge_material(P, c, p, eps, st, kt);
            if (kt > 0.f) jt = P.J[c][q] - 0.5f * kt * P.E[c][q];
        }
        P.J[c][q] = jt;
    }
}

__global__ void k_read_field(Params P, int comp, int primed, float* dense, double scale) {
    const long long tot = (long long)P.N[0] * P.N[1] * P.N[2];
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= tot) return;
    const int i = (int)(t % P.N[0]);
    const long long r = t / P.N[0];
    const int p[3] = {i, (int)(r % P.N[1]), (int)(r / P.N[1])};
    const long long q = lin(P, p[0], p[1], p[2]);
    double v;
    if (comp < 3) {
        v = P.E[comp][q];
    } else if (comp < 6) {
        const int cb = comp - 3;
        float b = P.B[cb][q];
        if (primed && upd_B(P, cb, p)) b -= 0.5f * curl_E_peek(P, cb, p, q);
        v = b;
    } else {
        const int c = comp - 6;
        float jt = 0.f;   // Js lives on superconducting edges only
        if (upd_E(P, c, p)) {
            float eps, st, kt;
            edge_material(P, c, p, eps, st, kt);
            if (kt > 0.f) jt = P.J[c][q] + (primed ? 0.5f * kt * P.E[c][q] : 0.f);
        }
        v = jt;
    }
    dense[t] = (float)(v * scale);
}

// ------------------------------------------------------------ time step
// ------------------------------------------------------------ launchers
static inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

cudaError_t launch_convert_materials(const Params& P, const float* eps_r, const float* mu_r,
                                     const float* lam, const float* sigma, double dt, float* eps,
                                     float* sig, float* kap, float* mu, unsigned* mm, cudaStream_t st) {
    const long long tot = P.plane * P.N[2];
    k_fill<<<1024, 256, 0, st>>>(eps, tot, 1.f);
    k_fill<<<1024, 256, 0, st>>>(sig, tot, 0.f);
    k_fill<<<1024, 256, 0, st>>>(kap, tot, 0.f);
    k_fill<<<1024, 256, 0, st>>>(mu, tot, 1.f);
    const long long ncell = (long long)P.n[0] * P.n[1] * P.n[2];
    k_convert_materials<<<blocks_for(ncell, 256), 256, 0, st>>>(P, eps_r, mu_r, lam, sigma, dt, eps,
                                                                 sig, kap, mu, mm);
    return cudaGetLastError();
}

cudaError_t launch_set_field(const Params& P, int comp, const float* dense, float* dst, double scale,
                             cudaStream_t st) {
    const long long tot = (long long)P.N[0] * P.N[1] * P.N[2];
    k_set_field<<<blocks_for(tot, 256), 256, 0, st>>>(P, comp, dense, dst, scale);
    return cudaGetLastError();
}

cudaError_t launch_mask_js(const Params& P, cudaStream_t st) {
    k_mask_js<<<grid_of(P), dim3(BX, BY, BZ), 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_prime(const Params& P, cudaStream_t st) {
    k_prime<<<grid_of(P), dim3(BX, BY, BZ), 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_read_field(const Params& P, int comp, int primed, float* dense, double scale,
                              cudaStream_t st) {
    const long long tot = (long long)P.N[0] * P.N[1] * P.N[2];
    k_read_field<<<blocks_for(tot, 256), 256, 0, st>>>(P, comp, primed, dense, scale);
    return cudaGetLastError();
}


}  // namespace tf
