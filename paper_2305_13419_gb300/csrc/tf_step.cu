// tf_step.cu -- fused single-pass step of the two-fluid Yee scheme (sm_103a).
//
// One launch advances the whole grid by one step of Algorithm 1 (arXiv
// 2305.13419, Sec. 3) in its fused leapfrog form:
//   Bt^{n+1/2} = Bt^{n-1/2} - curl(E^n)                   (steps 5 + 1, CPML psi_B)
//   Jt^{n+1/2} = Jt^{n-1/2} + kt_e E^n                     (steps 4 + 2)
//   E^{n+1}    = ca E^n + cb (curl(Bt/mu) - Jt^{n+1/2})     (step 3, CPML psi_E)
// plus soft sources, first-order Mur z walls and the non-finite watchdog.
//
// Layout of the work: a CTA of 32 x 8 threads owns one (x, y) column per
// thread and streams along z through a chunk of planes.  The E update needs
// B^{n+1/2} at x-1 and y-1, so the tile carries one halo column and one halo
// row whose B values it recomputes (the tile advances by 31 x 7 owned
// columns).  x neighbours move by warp shuffles, y neighbours through shared
// memory, the z neighbour stays in registers (B at k-1) or is prefetched
// (E at k+1, k+2).  E, B and psi_B ping-pong between two buffers, so halo
// reads never race with another CTA's writes; Js and psi_E belong to a single
// owner and update in place.  Work items (tile, z chunk) are handed out by an
// atomic counter to a grid sized to fill every SM once.
//
// Edge material: a tile-plane whose cells are all alike carries one precomputed
// {ca, cb, cj, 1/mu} record and skips the per-cell maps entirely; elsewhere the
// edge values are averaged from the maps as the edge rule says.
#include <math.h>

#include "tf_internal.cuh"

namespace tf {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float ld(const float* p, bool ok) { return ok ? __ldg(p) : 0.f; }

// CPML memory of a B-side derivative: psi' = b psi + c d, read from the old
// buffer, written (by the owner) to the new one; returns the curl term + psi'
__device__ __forceinline__ float psi_b(float t, const float* src, float* dst, int q, float b, float c,
                                       float d, bool upd, bool owner) {
    if (!upd) return t;
    const float nv = b * __ldg(src + q) + c * d;
    if (owner) dst[q] = nv;
    return t + nv;
}

// CPML memory of an E-side derivative, in place (single owner)
__device__ __forceinline__ float psi_e(float t, float* ps, int q, float b, float c, float d) {
    const float nv = b * ps[q] + c * d;
    ps[q] = nv;
    return t + nv;
}

struct Mat {
    float ca, cb, cj;
};

__device__ __forceinline__ Mat edge_coeffs(const Params& P, int c, int gx, int gy, int k) {
    const int p[3] = {gx, gy, k};
    float eps, st, kt;
    edge_material(P, c, p, eps, st, kt);
    const float den = eps + P.theta * st;
    return {(eps - (1.f - P.theta) * st) / den, 1.f / den, kt};
}

__device__ __forceinline__ float imu(const Params& P, int c, int gx, int gy, int k) {
    const int p[3] = {gx, gy, k};
    return inv_mu_face(P, c, p);
}

}  // namespace

__global__ void __launch_bounds__(kTX* kTY, 3) k_step(Params P, StepOut O, Sources S) {
    // double-buffered exchange planes: E^n(k) {x, z} for the y+1 neighbour,
    // B^{n+1/2}(k) {x, z} for the y-1 neighbour
    __shared__ float sE[2][2][kTY][kTX], sB[2][2][kTY][kTX];
    __shared__ int s_item;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nitems = O.ntx * O.nty * O.nch;
    const int PL = (int)P.plane;

    for (;;) {
        if (tx == 0 && ty == 0) {
            const long long d = (long long)(atomicAdd(O.ctr, 1ull) - O.base);
            s_item = (d >= 0 && d < nitems) ? (int)d : -1;
        }
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item < 0) break;
        const int ch = item % O.nch;     // consecutive items: consecutive chunks of one tile
        const int tile = item / O.nch;
        const int bx = tile % O.ntx, by = tile / O.ntx;

        // ---------------------------------------------------------- column
        const int gx0 = bx * kSX - 1 + tx, gy0 = by * kSY - 1 + ty;
        int gx = gx0, gy = gy0;
        bool valid = true;
        if (gx < 0) { if (P.per[0]) gx += P.N[0]; else valid = false; }
        if (gy < 0) { if (P.per[1]) gy += P.N[1]; else valid = false; }
        if (gx >= P.N[0] || gy >= P.N[1]) valid = false;
        if (!valid) { gx = 0; gy = 0; }
        const bool owner = valid && tx >= 1 && ty >= 1;
        const int o = gy * P.pitch + gx;
        const int gxp = nxt(P, 0, gx), gyp = nxt(P, 1, gy);
        const int oxp = gy * P.pitch + gxp, oyp = gyp * P.pitch + gx;
        const bool glob_xp = (tx == kTX - 1) || (gx0 + 1 >= P.N[0]);   // x+1 not in this warp
        const bool glob_yp = (ty == kTY - 1) || (gy0 + 1 >= P.N[1]);   // y+1 not in this CTA
        const bool hvx = P.per[0] || gx < P.n[0], inx = P.per[0] || (gx >= 1 && gx <= P.n[0] - 1);
        const bool hvy = P.per[1] || gy < P.n[1], iny = P.per[1] || (gy >= 1 && gy <= P.n[1] - 1);
        const bool slx = in_slab(P, 0, gx), sly = in_slab(P, 1, gy);
        const float4* trec = O.tilemat + (long long)(by * O.ntx + bx) * P.N[2];
        const bool mur = P.bc[2] == TF_BC_MUR;

        const int kz0 = ch * kChunk;
        const int kz1 = min(kz0 + kChunk, O.kend);
        auto kn = [&](int k) { return (k + 1 < P.N[2]) ? k + 1 : (P.per[2] ? 0 : k); };
        const bool prev_plane = kz0 > 0 || P.per[2];
        const int kzm = kz0 > 0 ? kz0 - 1 : P.N[2] - 1;

        // pipeline registers: E^n at k-1, k, k+1; B^{n-1/2}(k); B^{n+1/2} at k-1 and (x, y only) k-2
        float em[3], e0[3], ep[3], bo[3], bm[3] = {0.f, 0.f, 0.f}, bmm0 = 0.f, bmm1 = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            e0[c] = ld(P.E[c] + kz0 * PL + o, valid);
            ep[c] = ld(P.E[c] + kn(kz0) * PL + o, valid);
            em[c] = ld(P.E[c] + kzm * PL + o, valid && prev_plane);
            bo[c] = ld(P.B[c] + kz0 * PL + o, valid);
        }
        // prologue: Bx, By at (x, y, kz0 - 1), the z differences of E(kz0)
        if (owner && prev_plane) {
            const int pm = kzm * PL;
            const bool hvz = P.per[2] || kzm < P.n[2];
            const bool slz = in_slab(P, 2, kzm);
            const float ez_yp = __ldg(P.E[2] + pm + oyp), ez_xp = __ldg(P.E[2] + pm + oxp);
            const bool uBx = inx && hvy && hvz, uBy = hvx && iny && hvz;
            const float dEz_y = ez_yp - em[2], dEy_z = e0[1] - em[1], dEx_z = e0[0] - em[0], dEz_x = ez_xp - em[2];
            float tx_y = P.r[1] * dEz_y, tx_z = P.r[2] * dEy_z, ty_z = P.r[2] * dEx_z, ty_x = P.r[0] * dEz_x;
            const int q = pm + o;
            if (sly && P.psiB[0][1]) tx_y = psi_b(tx_y, P.psiB[0][1], nullptr, q, P.pbB[1][gy], P.pcB[1][gy], dEz_y, uBx, false);
            if (slz && P.psiB[0][2]) tx_z = psi_b(tx_z, P.psiB[0][2], nullptr, q, P.pbB[2][kzm], P.pcB[2][kzm], dEy_z, uBx, false);
            if (slz && P.psiB[1][2]) ty_z = psi_b(ty_z, P.psiB[1][2], nullptr, q, P.pbB[2][kzm], P.pcB[2][kzm], dEx_z, uBy, false);
            if (slx && P.psiB[1][0]) ty_x = psi_b(ty_x, P.psiB[1][0], nullptr, q, P.pbB[0][gx], P.pcB[0][gx], dEz_x, uBy, false);
            const float bx_old = __ldg(P.B[0] + q), by_old = __ldg(P.B[1] + q);
            bm[0] = uBx ? bx_old - (tx_y - tx_z) : bx_old;
            bm[1] = uBy ? by_old - (ty_z - ty_x) : by_old;
        }
        float elo0 = 0.f, elo1 = 0.f;   // E^n on the low Mur wall

        // iteration k: B^{n+1/2}(k) (k < kz1) and E^{n+1}(k-1) (k > kz0)
        for (int k = kz0; k <= kz1; ++k) {
            const bool doB = k < kz1, doE = owner && k > kz0;
            const int b = k & 1;
            const int ke = k - 1;                       // plane of the E update
            const int qk = k * PL + o, qe = ke * PL + o;
            // ---- loads for this iteration and the next
            float epp[3], bon[3];
            const int kp2 = kn(kn(k)) * PL + o, kp1 = kn(k) * PL + o;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                epp[c] = ld(P.E[c] + kp2, valid && doB);
                bon[c] = ld(P.B[c] + kp1, valid && doB);
            }
            float4 rec = make_float4(0.f, 0.f, 0.f, 0.f);
            float jo[3] = {0.f, 0.f, 0.f};
            bool uni = true;
            if (doE) {
                rec = __ldg(trec + ke);
                uni = !isnan(rec.x);
                if (!uni || rec.z > 0.f) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) jo[c] = P.J[c][qe];
                }
            }
            // ---- exchange E^n(k) with the y+1 row
            sE[b][0][ty][tx] = e0[0];
            sE[b][1][ty][tx] = e0[2];
            __syncthreads();

            // ------------------------------------------------ B^{n+1/2}(k)
            float bn[3] = {bo[0], bo[1], bo[2]};
            {
                float ey_xp = __shfl_down_sync(kFull, e0[1], 1);
                float ez_xp = __shfl_down_sync(kFull, e0[2], 1);
                if (doB) {
                    const bool hvz = P.per[2] || k < P.n[2];
                    const bool inz = P.per[2] || (k >= 1 && k <= P.n[2] - 1);
                    const bool slz = in_slab(P, 2, k);
                    if (glob_xp) {
                        ey_xp = ld(P.E[1] + qk - o + oxp, valid);
                        ez_xp = ld(P.E[2] + qk - o + oxp, valid);
                    }
                    float ex_yp, ez_yp;
                    if (glob_yp) {
                        ex_yp = ld(P.E[0] + qk - o + oyp, valid);
                        ez_yp = ld(P.E[2] + qk - o + oyp, valid);
                    } else {
                        ex_yp = sE[b][0][ty + 1][tx];
                        ez_yp = sE[b][1][ty + 1][tx];
                    }
                    const float dEz_y = ez_yp - e0[2], dEy_z = ep[1] - e0[1];
                    const float dEx_z = ep[0] - e0[0], dEz_x = ez_xp - e0[2];
                    const float dEy_x = ey_xp - e0[1], dEx_y = ex_yp - e0[0];
                    float tBx_y = P.r[1] * dEz_y, tBx_z = P.r[2] * dEy_z;
                    float tBy_z = P.r[2] * dEx_z, tBy_x = P.r[0] * dEz_x;
                    float tBz_x = P.r[0] * dEy_x, tBz_y = P.r[1] * dEx_y;
                    const bool uBx = valid && inx && hvy && hvz;
                    const bool uBy = valid && hvx && iny && hvz;
                    const bool uBz = valid && hvx && hvy && inz;
                    if (sly) {
                        if (P.psiB[0][1]) tBx_y = psi_b(tBx_y, P.psiB[0][1], O.psiB[0][1], qk, P.pbB[1][gy], P.pcB[1][gy], dEz_y, uBx, owner);
                        if (P.psiB[2][1]) tBz_y = psi_b(tBz_y, P.psiB[2][1], O.psiB[2][1], qk, P.pbB[1][gy], P.pcB[1][gy], dEx_y, uBz, owner);
                    }
                    if (slz) {
                        if (P.psiB[0][2]) tBx_z = psi_b(tBx_z, P.psiB[0][2], O.psiB[0][2], qk, P.pbB[2][k], P.pcB[2][k], dEy_z, uBx, owner);
                        if (P.psiB[1][2]) tBy_z = psi_b(tBy_z, P.psiB[1][2], O.psiB[1][2], qk, P.pbB[2][k], P.pcB[2][k], dEx_z, uBy, owner);
                    }
                    if (slx) {
                        if (P.psiB[1][0]) tBy_x = psi_b(tBy_x, P.psiB[1][0], O.psiB[1][0], qk, P.pbB[0][gx], P.pcB[0][gx], dEz_x, uBy, owner);
                        if (P.psiB[2][0]) tBz_x = psi_b(tBz_x, P.psiB[2][0], O.psiB[2][0], qk, P.pbB[0][gx], P.pcB[0][gx], dEy_x, uBz, owner);
                    }
                    if (uBx) bn[0] = bo[0] - (tBx_y - tBx_z);
                    if (uBy) bn[1] = bo[1] - (tBy_z - tBy_x);
                    if (uBz) bn[2] = bo[2] - (tBz_x - tBz_y);
                    if (owner) {
                        if (uBx) O.B[0][qk] = bn[0];
                        if (uBy) O.B[1][qk] = bn[1];
                        if (uBz) O.B[2][qk] = bn[2];
                    }
                }
            }

            // ------------------------------------------------ E^{n+1}(k-1)
            {
                // B^{n+1/2}(k-1) at x-1 (shuffle) and y-1 (exchange plane of the last iteration)
                const float bz_xm = __shfl_up_sync(kFull, bm[2], 1);
                const float by_xm = __shfl_up_sync(kFull, bm[1], 1);
                if (doE) {
                    const int bb = b ^ 1;
                    const float bx_ym = sB[bb][0][ty - 1][tx];
                    const float bz_ym = sB[bb][1][ty - 1][tx];
                    const bool hvz = P.per[2] || ke < P.n[2];
                    const bool inz = P.per[2] || (ke >= 1 && ke <= P.n[2] - 1);
                    const bool slz = in_slab(P, 2, ke);
                    const bool uEx = hvx && iny && inz, uEy = inx && hvy && inz, uEz = inx && iny && hvz;
                    float hz = bm[2], hz_ym = bz_ym, hz_xm = bz_xm, hy = bm[1], hy_zm = bmm1, hy_xm = by_xm;
                    float hx = bm[0], hx_zm = bmm0, hx_ym = bx_ym;
                    if (!P.uniform_mu) {
                        if (uni) {
                            hz *= rec.w; hz_ym *= rec.w; hz_xm *= rec.w; hy *= rec.w; hy_zm *= rec.w;
                            hy_xm *= rec.w; hx *= rec.w; hx_zm *= rec.w; hx_ym *= rec.w;
                        } else {
                            const int km = ke > 0 ? ke - 1 : P.N[2] - 1;
                            const int xm = gx > 0 ? gx - 1 : P.N[0] - 1, ym = gy > 0 ? gy - 1 : P.N[1] - 1;
                            hz *= imu(P, 2, gx, gy, ke); hz_ym *= imu(P, 2, gx, ym, ke); hz_xm *= imu(P, 2, xm, gy, ke);
                            hy *= imu(P, 1, gx, gy, ke); hy_zm *= imu(P, 1, gx, gy, km); hy_xm *= imu(P, 1, xm, gy, ke);
                            hx *= imu(P, 0, gx, gy, ke); hx_zm *= imu(P, 0, gx, gy, km); hx_ym *= imu(P, 0, gx, ym, ke);
                        }
                    }
                    const float dHz_y = hz - hz_ym, dHy_z = hy - hy_zm;
                    const float dHx_z = hx - hx_zm, dHz_x = hz - hz_xm;
                    const float dHy_x = hy - hy_xm, dHx_y = hx - hx_ym;
                    float tEx_y = P.r[1] * dHz_y, tEx_z = P.r[2] * dHy_z;
                    float tEy_z = P.r[2] * dHx_z, tEy_x = P.r[0] * dHz_x;
                    float tEz_x = P.r[0] * dHy_x, tEz_y = P.r[1] * dHx_y;
                    if (sly) {
                        if (uEx && P.psiE[0][1]) tEx_y = psi_e(tEx_y, P.psiE[0][1], qe, P.pbE[1][gy], P.pcE[1][gy], dHz_y);
                        if (uEz && P.psiE[2][1]) tEz_y = psi_e(tEz_y, P.psiE[2][1], qe, P.pbE[1][gy], P.pcE[1][gy], dHx_y);
                    }
                    if (slz) {
                        if (uEx && P.psiE[0][2]) tEx_z = psi_e(tEx_z, P.psiE[0][2], qe, P.pbE[2][ke], P.pcE[2][ke], dHy_z);
                        if (uEy && P.psiE[1][2]) tEy_z = psi_e(tEy_z, P.psiE[1][2], qe, P.pbE[2][ke], P.pcE[2][ke], dHx_z);
                    }
                    if (slx) {
                        if (uEy && P.psiE[1][0]) tEy_x = psi_e(tEy_x, P.psiE[1][0], qe, P.pbE[0][gx], P.pcE[0][gx], dHz_x);
                        if (uEz && P.psiE[2][0]) tEz_x = psi_e(tEz_x, P.psiE[2][0], qe, P.pbE[0][gx], P.pcE[0][gx], dHy_x);
                    }
                    const float curl[3] = {tEx_y - tEx_z, tEy_z - tEy_x, tEz_x - tEz_y};
                    const bool upd[3] = {uEx, uEy, uEz};
                    const bool near_src = S.n > 0 && gx >= S.bb_lo[0] && gx < S.bb_hi[0] && gy >= S.bb_lo[1] &&
                                          gy < S.bb_hi[1] && ke >= S.bb_lo[2] && ke < S.bb_hi[2];
                    float enew[3];
                    bool bad = false;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        enew[c] = em[c];
                        if (!upd[c]) continue;
                        Mat m;
                        if (uni) m = {rec.x, rec.y, rec.z};
                        else m = edge_coeffs(P, c, gx, gy, ke);
                        float jt = 0.f;
                        if (m.cj > 0.f) {
                            jt = jo[c] + m.cj * em[c];
                            P.J[c][qe] = jt;
                        }
                        float e = m.ca * em[c] + m.cb * (curl[c] - jt);
                        if (near_src) {
                            for (int s = 0; s < S.n; ++s)
                                if (S.comp[s] == c && gx >= S.lo[s][0] && gx < S.hi[s][0] && gy >= S.lo[s][1] &&
                                    gy < S.hi[s][1] && ke >= S.lo[s][2] && ke < S.hi[s][2])
                                    e += S.amp[s];
                        }
                        enew[c] = e;
                        O.E[c][qe] = e;
                        bad |= !isfinite(e);
                    }
                    if (bad) atomicOr(P.status, kStatusNonFinite);
                    // first-order Mur on the z walls: E_w^{n+1} = E_i^n + M (E_i^{n+1} - E_w^n)
                    if (mur) {
                        const bool mx = hvx && iny, my = inx && hvy;
                        if (ke == 1) {
                            if (mx) O.E[0][o] = em[0] + P.mur_M * (enew[0] - elo0);
                            if (my) O.E[1][o] = em[1] + P.mur_M * (enew[1] - elo1);
                        }
                        if (ke == P.n[2] - 1) {
                            const int pw = P.n[2] * PL + o;
                            if (mx) O.E[0][pw] = em[0] + P.mur_M * (enew[0] - e0[0]);
                            if (my) O.E[1][pw] = em[1] + P.mur_M * (enew[1] - e0[1]);
                        }
                    }
                }
            }
            // publish B^{n+1/2}(k) for the y-1 reads of the next iteration
            sB[b][0][ty][tx] = bn[0];
            sB[b][1][ty][tx] = bn[2];
            if (ke == 0) { elo0 = em[0]; elo1 = em[1]; }
            bmm0 = bm[0];
            bmm1 = bm[1];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                bm[c] = bn[c];
                em[c] = e0[c];
                e0[c] = ep[c];
                ep[c] = epp[c];
                bo[c] = bon[c];
            }
        }
        __syncthreads();   // exchange planes are reused by the next work item
    }
}

// per (tile, plane): are all cells an owned edge or face of the tile-plane
// touches alike?  Then store {ca, cb, cj, 1/mu}; else ca = NaN
__global__ void k_tile_materials(Params P, float4* rec, int ntx, int nty) {
    const int bx = blockIdx.x, by = blockIdx.y;
    const int tx = threadIdx.x, ty = threadIdx.y;
    auto cellc = [&](int a, int v) {
        if (v < 0) return P.per[a] ? v + P.n[a] : 0;
        if (v >= P.n[a]) return P.per[a] ? v - P.n[a] : P.n[a] - 1;
        return v;
    };
    const int cx = cellc(0, bx * kSX - 1 + tx), cy = cellc(1, by * kSY - 1 + ty);
    __shared__ float ref[4];
    for (int k = 0; k < P.N[2]; ++k) {
        const int kz[2] = {cellc(2, k - 1), cellc(2, k)};
        if (tx == 0 && ty == 0) {
            const long long m = lin(P, cx, cy, kz[1]);
            ref[0] = P.eps[m]; ref[1] = P.sig[m]; ref[2] = P.kap[m]; ref[3] = P.mu[m];
        }
        __syncthreads();
        bool same = true;
#pragma unroll
        for (int z = 0; z < 2; ++z) {
            const long long m = lin(P, cx, cy, kz[z]);
            same &= P.eps[m] == ref[0] && P.sig[m] == ref[1] && P.kap[m] == ref[2] && P.mu[m] == ref[3];
        }
        same = __syncthreads_and(same);
        if (tx == 0 && ty == 0) {
            float4 r;
            if (same) {
                const float den = ref[0] + P.theta * ref[1];
                r = make_float4((ref[0] - (1.f - P.theta) * ref[1]) / den, 1.f / den, ref[2], 1.f / ref[3]);
            } else {
                r = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
            }
            rec[(long long)(by * ntx + bx) * P.N[2] + k] = r;
        }
        __syncthreads();
    }
}

int step_blocks_per_sm() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step, kTX * kTY, 0) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_step(const Params& P, const StepOut& O, const Sources& S, int blocks, cudaStream_t st) {
    k_step<<<blocks, dim3(kTX, kTY), 0, st>>>(P, O, S);
    return cudaGetLastError();
}

cudaError_t launch_tile_materials(const Params& P, float4* rec, int ntx, int nty, cudaStream_t st) {
    k_tile_materials<<<dim3(ntx, nty), dim3(kTX, kTY), 0, st>>>(P, rec, ntx, nty);
    return cudaGetLastError();
}

}  // namespace tf
