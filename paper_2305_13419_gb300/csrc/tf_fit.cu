// tf_fit.cu -- Q-factor of a ring-down from a probe's running DFT, FP64, one CTA.
//
// Sec. 5 of arXiv 2305.13419 extracts attenuation and phase constants of the
// resonator ring-down and reports Q.  The probe keeps
//   X_k = dt sum_{n=n0}^{N-1} s^n w_k^n,  w_k = exp(-i 2 pi f_k dt),
// and one damped mode s^n = a z^n + conj(a) conj(z)^n, z = exp((-alpha + i omega) dt)
// has the exact finite-window transform
//   M_k = dt [ a G(z w_k) + conj(a) G(conj(z) w_k) ],  G(q) = (q^n0 - q^N) / (1 - q).
// Levenberg-Marquardt over (alpha, omega, Re a, Im a) with Marquardt's
// diagonal scaling; one thread per frequency builds its residual and Jacobian
// rows, the CTA reduces J^T J and J^T r, thread 0 solves the 4 x 4 system.
// Output: f0 = omega / 2 pi, alpha, Q = omega / (2 alpha), converged flag.
#include <math.h>

#include "tf_internal.cuh"

namespace tf {

namespace {

struct C2 {
    double x, y;
};
__device__ __forceinline__ C2 cmul(C2 a, C2 b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ C2 cadd(C2 a, C2 b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ C2 csub(C2 a, C2 b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ C2 cscale(C2 a, double s) { return {a.x * s, a.y * s}; }
__device__ __forceinline__ C2 cdiv(C2 a, C2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}
// exp(m * (lr + i th))
__device__ __forceinline__ C2 cexp_m(double lr, double th, double m) {
    double s, c;
    sincos(m * th, &s, &c);
    const double r = exp(m * lr);
    return {r * c, r * s};
}

// G(q) and dG/dq for q = exp(lr + i th)
__device__ void geo(double lr, double th, long long n0, long long N, C2& G, C2& dG) {
    const C2 q = cexp_m(lr, th, 1.0);
    const C2 qa = cexp_m(lr, th, (double)n0), qb = cexp_m(lr, th, (double)N);
    const C2 one_m = {1.0 - q.x, -q.y};
    const C2 num = csub(qa, qb);
    G = cdiv(num, one_m);
    // d/dq: (n0 q^{n0-1} - N q^{N-1}) / (1-q) + (q^n0 - q^N) / (1-q)^2
    const C2 qa1 = cexp_m(lr, th, (double)(n0 - 1)), qb1 = cexp_m(lr, th, (double)(N - 1));
    const C2 t1 = cdiv(csub(cscale(qa1, (double)n0), cscale(qb1, (double)N)), one_m);
    const C2 t2 = cdiv(num, cmul(one_m, one_m));
    dG = cadd(t1, t2);
}

constexpr int kNT = TF_MAX_FREQS;  // threads

// per-thread model, residual and Jacobian row (real and imaginary parts)
__device__ void row(const double* re, const double* im, const double* fdt, int k, double dt, long long n0,
                    long long N, const double x[4], double r[2], double Jr[4], double Ji[4]) {
    const double al = x[0], om = x[1];
    const double two_pi = 6.283185307179586476925286766559;
    const double th1 = om * dt - two_pi * fdt[k], th2 = -om * dt - two_pi * fdt[k];
    const double lr = -al * dt;
    C2 G1, dG1, G2, dG2;
    geo(lr, th1, n0, N, G1, dG1);
    geo(lr, th2, n0, N, G2, dG2);
    const C2 q1 = cexp_m(lr, th1, 1.0), q2 = cexp_m(lr, th2, 1.0);
    const C2 a = {x[2], x[3]}, ac = {x[2], -x[3]};
    const C2 M = cscale(cadd(cmul(a, G1), cmul(ac, G2)), dt);
    r[0] = M.x - re[k];
    r[1] = M.y - im[k];
    // dq1/dalpha = -dt q1, dq1/domega = i dt q1; dq2/dalpha = -dt q2, dq2/domega = -i dt q2
    const C2 g1 = cmul(dG1, q1), g2 = cmul(dG2, q2);
    const C2 dal = cscale(cadd(cmul(a, g1), cmul(ac, g2)), -dt * dt);
    const C2 i_g1 = {-g1.y, g1.x}, i_g2 = {-g2.y, g2.x};
    const C2 dom = cscale(csub(cmul(a, i_g1), cmul(ac, i_g2)), dt * dt);
    const C2 dar = cscale(cadd(G1, G2), dt);
    const C2 d12 = csub(G1, G2);
    const C2 dai = cscale(C2{-d12.y, d12.x}, dt);
    Jr[0] = dal.x; Ji[0] = dal.y;
    Jr[1] = dom.x; Ji[1] = dom.y;
    Jr[2] = dar.x; Ji[2] = dar.y;
    Jr[3] = dai.x; Ji[3] = dai.y;
}

// sum a value over the CTA (kNT threads)
__device__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kNT / 32; ++w) t += sh[w];
    __syncthreads();
    return t;
}

__device__ bool solve4(double A[4][4], double b[4], double x[4]) {
    int piv[4] = {0, 1, 2, 3};
    for (int c = 0; c < 4; ++c) {
        int m = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(A[r][c]) > fabs(A[m][c])) m = r;
        if (!(fabs(A[m][c]) > 0.0)) return false;
        if (m != c) {
            for (int k = 0; k < 4; ++k) { double t = A[c][k]; A[c][k] = A[m][k]; A[m][k] = t; }
            double t = b[c]; b[c] = b[m]; b[m] = t;
            int tp = piv[c]; piv[c] = piv[m]; piv[m] = tp;
        }
        for (int r = c + 1; r < 4; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int k = c; k < 4; ++k) A[r][k] -= f * A[c][k];
            b[r] -= f * b[c];
        }
    }
    for (int c = 3; c >= 0; --c) {
        double s = b[c];
        for (int k = c + 1; k < 4; ++k) s -= A[c][k] * x[k];
        x[c] = s / A[c][c];
    }
    return true;
}

}  // namespace

__global__ void __launch_bounds__(kNT) k_fit_q(const double* re, const double* im, const double* fdt, int nf,
                                               double dt, long long n0, long long N, double f_guess,
                                               double q_guess, double* out) {
    __shared__ double sh[kNT / 32];
    __shared__ double xs[4], step[4];
    __shared__ int flag;  // 0 continue, 1 stop
    __shared__ double lam_s;
    const int k = threadIdx.x;
    const bool act = k < nf;
    const double two_pi = 6.283185307179586476925286766559;

    // start: omega from f_guess (or the strongest bin), alpha from q_guess
    if (k == 0) {
        double fg = f_guess;
        if (!(fg > 0)) {
            double best = -1.0;
            for (int j = 0; j < nf; ++j) {
                const double m = re[j] * re[j] + im[j] * im[j];
                if (m > best) { best = m; fg = fdt[j] / dt; }
            }
        }
        xs[1] = two_pi * fg;
        xs[0] = xs[1] / (2.0 * q_guess);
        xs[2] = 0.0;
        xs[3] = 0.0;
        flag = 0;
        lam_s = 1e-3;
    }
    __syncthreads();
    // amplitude by linear least squares at the starting (alpha, omega)
    {
        double x[4] = {xs[0], xs[1], 0.0, 0.0}, r[2] = {0, 0}, Jr[4] = {0, 0, 0, 0}, Ji[4] = {0, 0, 0, 0};
        if (act) row(re, im, fdt, k, dt, n0, N, x, r, Jr, Ji);
        // with a = 0 the residual is -X; normal equations in (ar, ai)
        const double a22 = block_sum(act ? Jr[2] * Jr[2] + Ji[2] * Ji[2] : 0.0, sh);
        const double a23 = block_sum(act ? Jr[2] * Jr[3] + Ji[2] * Ji[3] : 0.0, sh);
        const double a33 = block_sum(act ? Jr[3] * Jr[3] + Ji[3] * Ji[3] : 0.0, sh);
        const double b2 = block_sum(act ? -(Jr[2] * r[0] + Ji[2] * r[1]) : 0.0, sh);
        const double b3 = block_sum(act ? -(Jr[3] * r[0] + Ji[3] * r[1]) : 0.0, sh);
        if (k == 0) {
            const double det = a22 * a33 - a23 * a23;
            if (det != 0.0) {
                xs[2] = (b2 * a33 - b3 * a23) / det;
                xs[3] = (a22 * b3 - a23 * b2) / det;
            }
        }
        __syncthreads();
    }
    double cost = 0.0;
    {
        double x[4] = {xs[0], xs[1], xs[2], xs[3]}, r[2] = {0, 0}, Jr[4], Ji[4];
        if (act) row(re, im, fdt, k, dt, n0, N, x, r, Jr, Ji);
        cost = block_sum(act ? r[0] * r[0] + r[1] * r[1] : 0.0, sh);
    }
    int converged = 0;
    for (int it = 0; it < 400; ++it) {
        double x[4] = {xs[0], xs[1], xs[2], xs[3]}, r[2] = {0, 0}, Jr[4] = {0, 0, 0, 0}, Ji[4] = {0, 0, 0, 0};
        if (act) row(re, im, fdt, k, dt, n0, N, x, r, Jr, Ji);
        double A[4][4], g[4];
        for (int a = 0; a < 4; ++a) {
            for (int b = a; b < 4; ++b) A[a][b] = block_sum(act ? Jr[a] * Jr[b] + Ji[a] * Ji[b] : 0.0, sh);
            g[a] = block_sum(act ? -(Jr[a] * r[0] + Ji[a] * r[1]) : 0.0, sh);
        }
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < a; ++b) A[a][b] = A[b][a];
        // try damped steps until the cost drops (or give up)
        bool accepted = false;
        for (int tries = 0; tries < 30 && !accepted; ++tries) {
            if (k == 0) {
                double M[4][4], rhs[4], d[4];
                for (int a = 0; a < 4; ++a) {
                    for (int b = 0; b < 4; ++b) M[a][b] = A[a][b];
                    M[a][a] += lam_s * (A[a][a] > 0 ? A[a][a] : 1.0);
                    rhs[a] = g[a];
                }
                if (!solve4(M, rhs, d)) d[0] = d[1] = d[2] = d[3] = 0.0;
                for (int a = 0; a < 4; ++a) step[a] = d[a];
            }
            __syncthreads();
            double xn[4] = {xs[0] + step[0], xs[1] + step[1], xs[2] + step[2], xs[3] + step[3]};
            double rn[2] = {0, 0}, Jr2[4], Ji2[4];
            if (act) row(re, im, fdt, k, dt, n0, N, xn, rn, Jr2, Ji2);
            const double cn = block_sum(act ? rn[0] * rn[0] + rn[1] * rn[1] : 0.0, sh);
            if (cn <= cost && isfinite(cn)) {
                accepted = true;
                if (k == 0) {
                    double rel = 0.0;
                    for (int a = 0; a < 4; ++a) {
                        const double s = fabs(step[a]) / (fabs(xs[a]) + 1e-300);
                        rel = s > rel ? s : rel;
                        xs[a] = xn[a];
                    }
                    lam_s = lam_s * 0.2 > 1e-15 ? lam_s * 0.2 : 1e-15;
                    flag = (rel < 1e-14 || cost - cn <= 1e-28 * cost) ? 1 : 0;
                }
                cost = cn;
            } else if (k == 0) {
                lam_s *= 10.0;
            }
            __syncthreads();
        }
        if (!accepted) { converged = 1; break; }   // no descent left: at the minimum
        if (flag) { converged = 1; break; }
    }
    if (k == 0) {
        out[0] = xs[1] / two_pi;
        out[1] = xs[0];
        out[2] = xs[1] / (2.0 * xs[0]);
        out[3] = (converged && xs[0] > 0 && isfinite(out[2])) ? 1.0 : 0.0;
    }
}

cudaError_t launch_fit_q(const double* re, const double* im, const double* fdt, int nfreq, double dt,
                         long long n0, long long N, double f_guess, double q_guess, double* out,
                         cudaStream_t st) {
    k_fit_q<<<1, kNT, 0, st>>>(re, im, fdt, nfreq, dt, n0, N, f_guess, q_guess, out);
    return cudaGetLastError();
}

}  // namespace tf
