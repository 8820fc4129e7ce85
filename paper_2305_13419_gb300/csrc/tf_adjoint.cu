// tf_adjoint.cu -- discrete adjoint of the fused step (sm_103a).
//
// With sources fixed, one fused step of Algorithm 1 (arXiv 2305.13419,
// Sec. 3) is a linear map of the state (E, Bt, Jt, psi_B, psi_E):
//   psi_B' = bB psi_B + cB dE              (CPML slabs, updated faces)
//   Bt'    = Bt - curl_r E - sB psi_B'      (sB(c, a) = -curl_sign(c, a))
//   Jt'    = Jt + cj E
//   psi_E' = bE psi_E + cE dH(Bt'/mu)      (CPML slabs, updated edges)
//   E'     = ca E + cb (curl_r (Bt'/mu) + sE psi_E' - Jt')   (sE = curl_sign)
// (curl_r: the Yee curls with the r_a = c0 dt / d_a weights; ca, cb, cj the
// per-edge coefficients, 1, 0, 0 on edges the step leaves alone).  Its
// transpose, applied to the adjoint state (Eh, Bh, Jh, psi_Bh, psi_Eh), is
//   e          = cb Eh'
//   psi_Eh'tot = psi_Eh' + sE e
//   Bh'tot     = Bh' + (1/mu) [transposed backward differences of
//                sE r e + cE psi_Eh'tot]                     (face pass)
//   psi_Bh'tot = bB-scaled psi_Bh' + sB Bh'tot
//   Jh         = Jh' - e
//   psi_Eh     = bE psi_Eh'tot
//   Eh         = ca Eh' + cj Jh + [transposed forward differences of
//                -curl_sign r Bh'tot + cB psi_Bh'tot]         (edge pass)
// and the gradient of the objective collects, per edge,
//   dJ/d eps_e += Eh' cb (E^n - E'_no-source)     (Alg. 1 step 3, theta scheme)
//   dJ/d kt_e  += Jh E^n                           (steps 4 + 2)
// Each pass forms, once per point, the weights the other pass differences:
// the face pass stores the face weights u_c,a = -curl_sign r_a Bh'tot +
// cB psi_Bh'tot (zero on faces the step leaves alone), the edge pass the edge
// weights w_e,a = sE r_a e + cE psi_Eh'tot of the next step (zero on edges the
// step leaves alone); a pass then reads its neighbours' weights as plain
// loads.  Both passes update in place; one thread per storage point handles
// its three components, a block covers 32 x 8 points of one plane.
#include <math.h>

#include "tf_internal.cuh"

namespace tf {

namespace {

constexpr int kAX = 32, kAY = 8;

// storage point of this thread (3-D launch: x, y blocks, one plane per blockIdx.z)
__device__ __forceinline__ bool point_of(const Params& P, int p[3]) {
    p[0] = blockIdx.x * kAX + threadIdx.x;
    p[1] = blockIdx.y * kAY + threadIdx.y;
    p[2] = blockIdx.z;
    return p[0] < P.N[0] && p[1] < P.N[1];
}

__device__ __forceinline__ int lin32(const Params& P, int i, int j, int k) {
    return k * (int)P.plane + j * P.pitch + i;
}

}  // namespace

// face pass: Bh'tot = Bh' + (1/mu) sum_a [w(p) - w(p + a)], psi_Bh'tot, and the face weights
__global__ void __launch_bounds__(kAX * kAY) k_adj_faces(Params P, AdjState A) {
    int p[3];
    if (!point_of(P, p)) return;
    const int q = lin32(P, p[0], p[1], p[2]);
    // the next point along each axis (clamped at a wall, where the difference vanishes)
    const int qn[3] = {lin32(P, nxt(P, 0, p[0]), p[1], p[2]), lin32(P, p[0], nxt(P, 1, p[1]), p[2]),
                       lin32(P, p[0], p[1], nxt(P, 2, p[2]))};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (!upd_B(P, c, p)) continue;   // its weights stay zero
        const int a1 = (c + 1) % 3, a2 = (c + 2) % 3;
        const int e1 = 3 - c - a1, e2 = 3 - c - a2;
        const float hsum = (A.W[e1][a1][q] - A.W[e1][a1][qn[a1]]) + (A.W[e2][a2][q] - A.W[e2][a2][qn[a2]]);
        const float bt = A.B[c][q] + hsum * inv_mu_face(P, c, p);
        A.B[c][q] = bt;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int a = t ? a2 : a1;
            const float sg = curl_sign(c, a);
            float u = -sg * P.r[a] * bt;
            if (A.psiB[c][a] && in_slab(P, a, p[a])) {
                const float ps = __ldg(P.pbB[a] + p[a]) * A.psiB[c][a][q] - sg * bt;
                A.psiB[c][a][q] = ps;
                u += __ldg(P.pcB[a] + p[a]) * ps;
            }
            A.U[c][a][q] = u;
        }
    }
}

// edge pass: Jh, psi_Eh, Eh; per-edge gradients; the objective's derivative
// at the probe; the edge weights of the next step.  The step's coefficients
// are the ones the forward step used: the tile-plane record where the
// material of the tile-plane is uniform, else the per-point arrays; (1, 0, 0)
// on edges the step leaves alone.
__global__ void __launch_bounds__(kAX * kAY) k_adj_edges(Params P, AdjState A, Sources S, AdjStep st,
                                                        const float4* __restrict__ tilemat, int ntx) {
    int p[3];
    if (!point_of(P, p)) return;
    const int q = lin32(P, p[0], p[1], p[2]);
    // the previous point along each axis (none below a wall)
    const int qp[3] = {lin32(P, prv(P, 0, p[0]), p[1], p[2]), lin32(P, p[0], prv(P, 1, p[1]), p[2]),
                       lin32(P, p[0], p[1], prv(P, 2, p[2]))};
    const bool hp[3] = {P.per[0] || p[0] > 0, P.per[1] || p[1] > 0, P.per[2] || p[2] > 0};
    const bool in_src = S.n > 0 && p[0] >= S.bb_lo[0] && p[0] <= S.bb_hi[0] && p[1] >= S.bb_lo[1] &&
                        p[1] <= S.bb_hi[1] && p[2] >= S.bb_lo[2] && p[2] <= S.bb_hi[2];
    // the forward step's record of this point's tile-plane (points past the
    // last tile of a walled axis are walls: no record needed)
    const int tx = p[0] / kSX, ty = p[1] / kSY;
    const bool intile = p[0] < (P.per[0] ? P.N[0] : P.n[0]) && p[1] < (P.per[1] ? P.N[1] : P.n[1]);
    const float4 rec = intile ? __ldg(tilemat + (long long)(ty * ntx + tx) * P.N[2] + p[2])
                              : make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
    const bool uni = !isnan(rec.x);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const float ep = A.E[e][q];
        // transposed forward differences of the face weights
        float d = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (a == e) continue;
            const int c = 3 - e - a;
            if (hp[a]) d += A.U[c][a][qp[a]];
            d -= A.U[c][a][q];
        }
        const bool upd = upd_E(P, e, p);
        const float cb = !upd ? 0.f : uni ? rec.y : __ldg(P.cb[e] + q);
        float enew = ep + d;
        if (cb != 0.f) {
            const float ev = cb * ep, cj = uni ? rec.z : __ldg(P.cj[e] + q);
            const float jh = A.J[e][q] - ev;
            A.J[e][q] = jh;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a == e || !A.psiE[e][a] || !in_slab(P, a, p[a])) continue;
                A.psiE[e][a][q] = __ldg(P.pbE[a] + p[a]) * (A.psiE[e][a][q] + curl_sign(e, a) * ev);
            }
            enew = (uni ? rec.x : __ldg(P.ca[e] + q)) * ep + cj * jh + d;
            // gradients: E^n, and E^{n+1} without this step's soft sources
            const float en = st.En[e][q];
            float e1 = st.En1[e][q];
            if (in_src)
                for (int s = 0; s < S.n; ++s)
                    if (S.comp[s] == e && p[0] >= S.lo[s][0] && p[0] < S.hi[s][0] && p[1] >= S.lo[s][1] &&
                        p[1] < S.hi[s][1] && p[2] >= S.lo[s][2] && p[2] < S.hi[s][2])
                        e1 -= S.amp[s];
            A.gE[e][q] += (double)ep * (double)cb * (double)(en - e1);
            if (cj > 0.f) A.gK[e][q] += (double)jh * (double)en;
        }
        if (e == st.probe_comp && q == st.probe_q) enew += st.probe_src;
        A.E[e][q] = enew;
        if (cb != 0.f) {   // edge weights of the next face pass (they stay zero where cb = 0)
            const float evn = cb * enew;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a == e) continue;
                const float sg = curl_sign(e, a);
                float w = sg * P.r[a] * evn;
                if (A.psiE[e][a] && in_slab(P, a, p[a])) w += __ldg(P.pcE[a] + p[a]) * (A.psiE[e][a][q] + sg * evn);
                A.W[e][a][q] = w;
            }
        }
    }
}

// per cell: dJ/d eps_r and dJ/d lambda_L from the per-edge sums, with the
// weights of the edge rule (eps: mean of 4 cells; kt: mean over the 4 cells
// or over the superconducting ones); `unscale` undoes the seed's scaling
__global__ void __launch_bounds__(256) k_adj_cells(Params P, AdjState A, float dt_c0, double unscale, float* g_eps,
                                                   float* g_lam) {
    const long long t = (long long)blockIdx.x * 256 + threadIdx.x;
    const long long nc = (long long)P.n[0] * P.n[1] * P.n[2];
    if (t >= nc) return;
    const int cell[3] = {(int)(t % P.n[0]), (int)((t / P.n[0]) % P.n[1]), (int)(t / ((long long)P.n[0] * P.n[1]))};
    const long long m = lin(P, cell[0], cell[1], cell[2]);
    const float kc = __ldg(P.kap + m);
    double ge = 0.0, gk = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int b1 = (c + 1) % 3, b2 = (c + 2) % 3;
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                // edge E_c whose cell (p[c], p[b1] - u, p[b2] - v) is this cell
                int x[3];
                x[c] = cell[c];
                x[b1] = cell[b1] + u;
                x[b2] = cell[b2] + v;
                if (x[b1] >= P.N[b1]) { if (!P.per[b1]) continue; x[b1] -= P.N[b1]; }
                if (x[b2] >= P.N[b2]) { if (!P.per[b2]) continue; x[b2] -= P.N[b2]; }
                if (!upd_E(P, c, x)) continue;
                const long long q = lin(P, x[0], x[1], x[2]);
                ge += 0.25 * A.gE[c][q];
                if (kc > 0.f) {
                    float wgt = 0.25f;
                    if (P.edge_rule != TF_EDGE_PLAIN_MEAN) {
                        int nk = 0;
#pragma unroll
                        for (int uu = 0; uu < 2; ++uu)
#pragma unroll
                            for (int vv = 0; vv < 2; ++vv) {
                                int cc[3];
                                cc[c] = x[c];
                                cc[b1] = uu ? prv(P, b1, x[b1]) : x[b1];
                                cc[b2] = vv ? prv(P, b2, x[b2]) : x[b2];
                                nk += __ldg(P.kap + lin(P, cc[0], cc[1], cc[2])) > 0.f;
                            }
                        wgt = nk ? 1.f / (float)nk : 0.f;
                    }
                    gk += (double)wgt * A.gK[c][q];
                }
            }
    }
    g_eps[t] = (float)(ge * unscale);
    float gl = 0.f;
    if (kc > 0.f) {   // kt = (c0 dt / lambda)^2 / mu_r: d kt / d lambda = -2 kt / lambda
        const float lam = dt_c0 / sqrtf(kc * __ldg(P.mu + m));
        gl = (float)(gk * unscale * (-2.0 * (double)kc / (double)lam));
    }
    g_lam[t] = gl;
}

// E^n of the three components into the adjoint's history (16-byte aligned
// arrays of n4 float4 each), grid-stride
__global__ void __launch_bounds__(256) k_copy3(float4* d0, float4* d1, float4* d2, const float4* s0, const float4* s1,
                                               const float4* s2, long long n4) {
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n4; i += (long long)gridDim.x * 256) {
        const float4 a = __ldg(s0 + i), b = __ldg(s1 + i), c = __ldg(s2 + i);
        d0[i] = a;
        d1[i] = b;
        d2[i] = c;
    }
}

cudaError_t launch_copy3(float* const dst[3], float* const src[3], long long n, cudaStream_t stream) {
    if (n % 4 != 0) return cudaErrorInvalidValue;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess || sms < 1) sms = 1;
    k_copy3<<<4 * sms, 256, 0, stream>>>((float4*)dst[0], (float4*)dst[1], (float4*)dst[2], (const float4*)src[0],
                                          (const float4*)src[1], (const float4*)src[2], n / 4);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_step(const Params& P, const AdjState& A, const Sources& S, const AdjStep& st,
                                const float4* tilemat, int ntx, cudaStream_t stream) {
    const dim3 grid((P.N[0] + kAX - 1) / kAX, (P.N[1] + kAY - 1) / kAY, P.N[2]), block(kAX, kAY);
    k_adj_faces<<<grid, block, 0, stream>>>(P, A);
    k_adj_edges<<<grid, block, 0, stream>>>(P, A, S, st, tilemat, ntx);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_cells(const Params& P, const AdjState& A, float dt_c0, double unscale, float* g_eps,
                                 float* g_lam, cudaStream_t stream) {
    const long long nc = (long long)P.n[0] * P.n[1] * P.n[2];
    k_adj_cells<<<(unsigned)((nc + 255) / 256), 256, 0, stream>>>(P, A, dt_c0, unscale, g_eps, g_lam);
    return cudaGetLastError();
}

}  // namespace tf
