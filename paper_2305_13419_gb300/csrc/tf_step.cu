// tf_step.cu -- fused single-pass step of the two-fluid Yee scheme (sm_103a).
//
// One launch advances the whole grid by one step of Algorithm 1 (arXiv
// 2305.13419, Sec. 3) in its fused leapfrog form:
//   Bt^{n+1/2} = Bt^{n-1/2} - curl(E^n)                   (steps 5 + 1, CPML psi_B)
//   Jt^{n+1/2} = Jt^{n-1/2} + kt_e E^n                     (steps 4 + 2)
//   E^{n+1}    = ca E^n + cb (curl(Bt/mu) - Jt^{n+1/2})     (step 3, CPML psi_E)
// plus soft sources, first-order Mur z walls and the non-finite watchdog.
//
// Work layout.  A CTA of 32 x 8 threads owns a 32 x 8 column tile and streams
// it along z through a chunk of planes.  Each plane's E^n and B^{n-1/2}
// arrive in shared memory by TMA (cp.async.bulk.tensor) as 40 x 10 boxes
// covering the tile plus its halo, through a ring of kStages buffers whose
// mbarriers complete on the transferred byte count; one elected thread keeps
// the ring kStages - 2 planes ahead of the compute.  Per plane:
//   B phase  every thread forms B^{n+1/2} at its column (E^n of this plane and
//            the next one, old B, CPML psi_B); warps 0 and 1 also recompute
//            the y-1 row / x-1 column of B that the E update needs from the
//            neighbouring tiles; results go to shared memory, owned values to
//            the new B buffer;
//   E phase  every thread forms Js^{n+1/2} and E^{n+1} at its column from the
//            shared B plane, the previous plane's B kept in registers, and the
//            edge material.
// E, B and psi_B ping-pong between two buffers (the other tiles only ever
// read the old ones); Js and psi_E are owned by one thread and update in
// place.  Work items (tile, z chunk) come from an atomic counter; the grid
// fills every SM once.  Periodic x / y seams, which TMA cannot wrap, are
// patched from global memory after the box lands.
//
// Edge material: a tile-plane whose cells are all alike carries one precomputed
// {ca, cb, cj, 1/mu} record; elsewhere the edge values are averaged from the
// per-cell maps as the edge rule says.  An interior tile-plane (uniform
// material, no wall, no CPML slab, no source, no Mur plane) takes a path with
// none of those checks.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>

#include "tf_internal.cuh"

namespace tf {

namespace {

struct __align__(128) StageBuf {   // both TMA destinations 128-byte aligned
    alignas(128) float e[3][kBoxY][kBoxX];
    alignas(128) float b[3][kBoxY][kBoxX];
};
constexpr unsigned kBoxBytes = 3u * kBoxY * kBoxX * sizeof(float);   // one field, one box

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// bounded wait for phase `phase` of a barrier; false if it never completed
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned phase) {
    for (long long it = 0; it < kSpinLimit; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_box(void* dst, const CUtensorMap* map, int x, int y, int z, int f,
                                             unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(f), "r"(smem_u32(bar))
        : "memory");
}

// CPML memory of a B-side derivative: psi' = b psi + c d from the old buffer,
// written (by the owner) to the new one; returns the curl term + psi'
__device__ __forceinline__ float psi_b(float t, const float* src, float* dst, int q, float b, float c, float d,
                                       bool upd, bool store) {
    if (!upd) return t;
    const float nv = b * __ldg(src + q) + c * d;
    if (store) dst[q] = nv;
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

// wrap (periodic) a coordinate into [0, N); -1 if it falls outside a non-periodic axis
__device__ __forceinline__ int wrap_or_out(const Params& P, int a, int v) {
    if (v >= 0 && v < P.N[a]) return v;
    if (!P.per[a]) return -1;
    v %= P.N[a];
    return v < 0 ? v + P.N[a] : v;
}

// B^{n+1/2} at one point of a landed stage, general path (masks and CPML)
struct BPoint {
    float x, y, z;
};
__device__ __forceinline__ BPoint b_general(const Params& P, const StepOut& O, const StageBuf& s0,
                                            const StageBuf& s1, int j, int i, int gx, int gy, int k, int q,
                                            bool store_psi) {
    const float ex = s0.e[0][j][i], ey = s0.e[1][j][i], ez = s0.e[2][j][i];
    const float dEz_y = s0.e[2][j + 1][i] - ez, dEy_z = s1.e[1][j][i] - ey;
    const float dEx_z = s1.e[0][j][i] - ex, dEz_x = s0.e[2][j][i + 1] - ez;
    const float dEy_x = s0.e[1][j][i + 1] - ey, dEx_y = s0.e[0][j + 1][i] - ex;
    float tBx_y = P.r[1] * dEz_y, tBx_z = P.r[2] * dEy_z;
    float tBy_z = P.r[2] * dEx_z, tBy_x = P.r[0] * dEz_x;
    float tBz_x = P.r[0] * dEy_x, tBz_y = P.r[1] * dEx_y;
    const bool hvx = P.per[0] || gx < P.n[0], inx = P.per[0] || (gx >= 1 && gx <= P.n[0] - 1);
    const bool hvy = P.per[1] || gy < P.n[1], iny = P.per[1] || (gy >= 1 && gy <= P.n[1] - 1);
    const bool hvz = P.per[2] || k < P.n[2], inz = P.per[2] || (k >= 1 && k <= P.n[2] - 1);
    const bool uBx = inx && hvy && hvz, uBy = hvx && iny && hvz, uBz = hvx && hvy && inz;
    if (in_slab(P, 1, gy)) {
        if (P.psiB[0][1]) tBx_y = psi_b(tBx_y, P.psiB[0][1], O.psiB[0][1], q, P.pbB[1][gy], P.pcB[1][gy], dEz_y, uBx, store_psi);
        if (P.psiB[2][1]) tBz_y = psi_b(tBz_y, P.psiB[2][1], O.psiB[2][1], q, P.pbB[1][gy], P.pcB[1][gy], dEx_y, uBz, store_psi);
    }
    if (in_slab(P, 2, k)) {
        if (P.psiB[0][2]) tBx_z = psi_b(tBx_z, P.psiB[0][2], O.psiB[0][2], q, P.pbB[2][k], P.pcB[2][k], dEy_z, uBx, store_psi);
        if (P.psiB[1][2]) tBy_z = psi_b(tBy_z, P.psiB[1][2], O.psiB[1][2], q, P.pbB[2][k], P.pcB[2][k], dEx_z, uBy, store_psi);
    }
    if (in_slab(P, 0, gx)) {
        if (P.psiB[1][0]) tBy_x = psi_b(tBy_x, P.psiB[1][0], O.psiB[1][0], q, P.pbB[0][gx], P.pcB[0][gx], dEz_x, uBy, store_psi);
        if (P.psiB[2][0]) tBz_x = psi_b(tBz_x, P.psiB[2][0], O.psiB[2][0], q, P.pbB[0][gx], P.pcB[0][gx], dEy_x, uBz, store_psi);
    }
    BPoint r;
    r.x = uBx ? s0.b[0][j][i] - (tBx_y - tBx_z) : s0.b[0][j][i];
    r.y = uBy ? s0.b[1][j][i] - (tBy_z - tBy_x) : s0.b[1][j][i];
    r.z = uBz ? s0.b[2][j][i] - (tBz_x - tBz_y) : s0.b[2][j][i];
    return r;
}

}  // namespace

__global__ void __launch_bounds__(kTX* kTY, 4)
    k_step(const __grid_constant__ CUtensorMap tmap, Params P, StepOut O, Sources S) {
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    // TMA destinations must be 128-byte aligned: round the base up (128 spare bytes are allocated)
    unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    StageBuf* stg = reinterpret_cast<StageBuf*>(smem_raw);
    float(*bn)[kBoxY][kBoxX] = reinterpret_cast<float(*)[kBoxY][kBoxX]>(smem_raw + kStages * sizeof(StageBuf));
    unsigned long long* bar =
        reinterpret_cast<unsigned long long*>(smem_raw + kStages * sizeof(StageBuf) + 3 * kBoxY * kBoxX * 4);
    __shared__ int s_item;
    __shared__ float4 s_rec[kChunk + 2];   // material record of each plane of the item
    __shared__ int s_fast[kChunk + 2];     // plane takes the interior path
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTX + tx;
    const int nitems = O.ntx * O.nty * O.nch;
    const int PL = (int)P.plane;
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    unsigned long long g = 0;        // planes this CTA has pulled through the ring (stage / phase bookkeeping)
    unsigned long long issued = 0;   // planes whose copies thread 0 has started

    for (;;) {
        if (tid == 0) {
            const long long d = (long long)(atomicAdd(O.ctr, 1ull) - O.base);
            s_item = (d >= 0 && d < nitems) ? (int)d : -1;
        }
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item < 0) break;
        const int ch = item % O.nch;   // consecutive items: consecutive chunks of one tile
        const int tile = item / O.nch;
        const int bx = tile % O.ntx, by = tile / O.ntx;
        const int x0 = bx * kSX, y0 = by * kSY;
        const int kz0 = ch * kChunk, kz1 = min(kz0 + kChunk, O.kend);
        const bool prev_plane = kz0 > 0 || P.per[2];
        const int ks = prev_plane ? kz0 - 1 : kz0;
        const int nq = kz1 - ks + 1;   // planes pulled: ks .. kz1
        auto plane_of = [&](int qq) {
            int k = ks + qq;
            if (k < 0) k += P.N[2];
            if (k >= P.N[2]) k -= P.N[2];
            return k;
        };
        auto issue = [&](int qq) {   // thread 0 only
            const unsigned long long gi = g + qq;
            const int s = (int)(gi % kStages);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&bar[s], 2 * kBoxBytes);
            const int k = plane_of(qq);
            tma_load_box(&stg[s].e[0][0][0], &tmap, x0 - 4, y0 - 1, k, O.ecur, &bar[s]);
            tma_load_box(&stg[s].b[0][0][0], &tmap, x0 - 4, y0 - 1, k, O.bcur, &bar[s]);
        };
        if (tid == 0) {
            for (int qq = 0; qq < nq && qq < kStages; ++qq) issue(qq);
            issued = g + (nq < kStages ? nq : kStages);
        }

        // ------------------------------------------------------- column
        const int gx = x0 + tx, gy = y0 + ty;
        const bool valid = gx < P.N[0] && gy < P.N[1];
        const int o = (valid ? gy : 0) * P.pitch + (valid ? gx : 0);
        const int i = tx + 4, j = ty + 1;   // position in the box
        const bool hvx = P.per[0] || gx < P.n[0], inx = P.per[0] || (gx >= 1 && gx <= P.n[0] - 1);
        const bool hvy = P.per[1] || gy < P.n[1], iny = P.per[1] || (gy >= 1 && gy <= P.n[1] - 1);
        const bool slx = in_slab(P, 0, gx), sly = in_slab(P, 1, gy);
        const float4* trec = O.tilemat + (long long)(by * O.ntx + bx) * P.N[2];
        const bool mur = P.bc[2] == TF_BC_MUR;
        auto axis_clear = [&](int a, int lo, int hi) {   // columns [lo, hi] interior and outside slabs
            if (P.per[a]) return true;
            const int L = P.L[a];
            return lo >= (L > 0 ? L : 1) && hi < P.n[a] - L && hi <= P.n[a] - 1;
        };
        const bool tile_fast = axis_clear(0, x0 - 1, x0 + kSX - 1) && axis_clear(1, y0 - 1, y0 + kSY - 1);
        auto z_clear = [&](int k) {
            if (P.per[2]) return true;
            const int L = P.L[2];
            return k >= (L > 0 ? L : 1) && k < P.n[2] - L && k <= P.n[2] - 1;
        };
        int src_k0 = 1 << 30, src_k1 = -1;   // z range of source planes touching this tile
        if (S.n > 0 && x0 + kSX > S.bb_lo[0] && x0 <= S.bb_hi[0] && y0 + kSY > S.bb_lo[1] && y0 <= S.bb_hi[1]) {
            src_k0 = S.bb_lo[2];
            src_k1 = S.bb_hi[2];
        }
        // periodic seams that the TMA box cannot wrap
        const bool seam = (P.per[0] && (x0 - 4 < 0 || x0 + kBoxX - 4 > P.N[0])) ||
                          (P.per[1] && (y0 - 1 < 0 || y0 + kBoxY - 1 > P.N[1]));
        auto patch = [&](StageBuf& sb, int k) {
            for (int t = tid; t < kBoxY * kBoxX; t += kTX * kTY) {
                const int jj = t / kBoxX, ii = t % kBoxX;
                const int x = x0 - 4 + ii, y = y0 - 1 + jj;
                if (x >= 0 && x < P.N[0] && y >= 0 && y < P.N[1]) continue;
                const int xw = wrap_or_out(P, 0, x), yw = wrap_or_out(P, 1, y);
                const bool in = xw >= 0 && yw >= 0;
                const int qw = k * PL + (in ? yw : 0) * P.pitch + (in ? xw : 0);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    sb.e[c][jj][ii] = in ? P.E[c][qw] : 0.f;
                    sb.b[c][jj][ii] = in ? P.B[c][qw] : 0.f;
                }
            }
        };

        // material records and interior flags of the item's planes, read once
        for (int t = tid; t < nq - 1; t += kTX * kTY) {
            const int k = plane_of(t);
            const float4 r = __ldg(trec + k);
            s_rec[t] = r;
            s_fast[t] = tile_fast && z_clear(k) && !isnan(r.x) && (k < src_k0 || k >= src_k1) &&
                        !(mur && (k == 1 || k == P.n[2] - 1));
        }
        __syncthreads();

        float bpx = 0.f, bpy = 0.f;     // B^{n+1/2}(k-1) at the own column (z differences)
        float elo0 = 0.f, elo1 = 0.f;   // E^n on the low Mur wall
        bool abort = false;
        for (int qq = 0; qq < nq - 1; ++qq) {
            const int k = plane_of(qq);
            const bool doE = ks + qq >= kz0;
            const unsigned long long g0 = g + qq, g1 = g0 + 1;
            StageBuf& s0 = stg[g0 % kStages];
            StageBuf& s1 = stg[g1 % kStages];
            bool ok = mbar_wait(&bar[g0 % kStages], (unsigned)((g0 / kStages) & 1));
            ok = ok && mbar_wait(&bar[g1 % kStages], (unsigned)((g1 / kStages) & 1));
            if (__syncthreads_or(!ok)) {
                abort = true;
                break;
            }
            if (seam) {
                if (qq == 0) patch(s0, k);
                patch(s1, plane_of(qq + 1));
                __syncthreads();
            }
            const int q = k * PL + o;
            const float4 rec = s_rec[qq];
            const bool fast = s_fast[qq] != 0;
            // Js^{n-1/2} of this plane, requested before the B phase so the load overlaps it
            float jo0 = 0.f, jo1 = 0.f, jo2 = 0.f;
            if (doE && valid && (isnan(rec.x) || rec.z > 0.f)) {
                jo0 = P.J[0][q];
                jo1 = P.J[1][q];
                jo2 = P.J[2][q];
            }

            // ------------------------------------------------ B phase
            if (fast) {
                const float ex = s0.e[0][j][i], ey = s0.e[1][j][i], ez = s0.e[2][j][i];
                const float nbx = s0.b[0][j][i] - (P.r[1] * (s0.e[2][j + 1][i] - ez) - P.r[2] * (s1.e[1][j][i] - ey));
                const float nby = s0.b[1][j][i] - (P.r[2] * (s1.e[0][j][i] - ex) - P.r[0] * (s0.e[2][j][i + 1] - ez));
                const float nbz = s0.b[2][j][i] - (P.r[0] * (s0.e[1][j][i + 1] - ey) - P.r[1] * (s0.e[0][j + 1][i] - ex));
                bn[0][j][i] = nbx;
                bn[1][j][i] = nby;
                bn[2][j][i] = nbz;
                if (doE && valid) {
                    O.B[0][q] = nbx;
                    O.B[1][q] = nby;
                    O.B[2][q] = nbz;
                }
                if (ty == 0) {   // halo row y0 - 1: Bz, Bx
                    const int jh = 0;
                    const float hx = s0.e[0][jh][i], hy = s0.e[1][jh][i], hz = s0.e[2][jh][i];
                    bn[0][jh][i] = s0.b[0][jh][i] - (P.r[1] * (s0.e[2][jh + 1][i] - hz) - P.r[2] * (s1.e[1][jh][i] - hy));
                    bn[2][jh][i] = s0.b[2][jh][i] - (P.r[0] * (s0.e[1][jh][i + 1] - hy) - P.r[1] * (s0.e[0][jh + 1][i] - hx));
                } else if (ty == 1 && tx < kTY) {   // halo column x0 - 1: Bz, By
                    const int jh = tx + 1, ih = 3;
                    const float hx = s0.e[0][jh][ih], hy = s0.e[1][jh][ih], hz = s0.e[2][jh][ih];
                    bn[1][jh][ih] = s0.b[1][jh][ih] - (P.r[2] * (s1.e[0][jh][ih] - hx) - P.r[0] * (s0.e[2][jh][ih + 1] - hz));
                    bn[2][jh][ih] = s0.b[2][jh][ih] - (P.r[0] * (s0.e[1][jh][ih + 1] - hy) - P.r[1] * (s0.e[0][jh + 1][ih] - hx));
                }
            } else {
                const BPoint bp = b_general(P, O, s0, s1, j, i, valid ? gx : 0, valid ? gy : 0, k, q, doE && valid);
                bn[0][j][i] = bp.x;
                bn[1][j][i] = bp.y;
                bn[2][j][i] = bp.z;
                if (doE && valid) {
                    const int p3[3] = {gx, gy, k};
                    if (upd_B(P, 0, p3)) O.B[0][q] = bp.x;
                    if (upd_B(P, 1, p3)) O.B[1][q] = bp.y;
                    if (upd_B(P, 2, p3)) O.B[2][q] = bp.z;
                }
                if (ty == 0 || (ty == 1 && tx < kTY)) {
                    const int jh = ty == 0 ? 0 : tx + 1, ih = ty == 0 ? i : 3;
                    const int hxg = wrap_or_out(P, 0, x0 - 4 + ih), hyg = wrap_or_out(P, 1, y0 - 1 + jh);
                    float hxv = 0.f, hyv = 0.f, hzv = 0.f;
                    if (hxg >= 0 && hyg >= 0) {
                        const int qh = k * PL + hyg * P.pitch + hxg;
                        const BPoint h = b_general(P, O, s0, s1, jh, ih, hxg, hyg, k, qh, false);
                        hxv = h.x;
                        hyv = h.y;
                        hzv = h.z;
                    }
                    if (ty == 0) {
                        bn[0][jh][ih] = hxv;
                        bn[2][jh][ih] = hzv;
                    } else {
                        bn[1][jh][ih] = hyv;
                        bn[2][jh][ih] = hzv;
                    }
                }
            }
            __syncthreads();

            // ------------------------------------------------ E phase
            const float bxo = bn[0][j][i], byo = bn[1][j][i], bzo = bn[2][j][i];
            if (doE && valid) {
                const float em0 = s0.e[0][j][i], em1 = s0.e[1][j][i], em2 = s0.e[2][j][i];
                if (fast) {
                    const float im = P.uniform_mu ? 1.f : rec.w;
                    const float cx = im * (P.r[1] * (bzo - bn[2][j - 1][i]) - P.r[2] * (byo - bpy));
                    const float cy = im * (P.r[2] * (bxo - bpx) - P.r[0] * (bzo - bn[2][j][i - 1]));
                    const float cz = im * (P.r[0] * (byo - bn[1][j][i - 1]) - P.r[1] * (bxo - bn[0][j - 1][i]));
                    float j0 = 0.f, j1 = 0.f, j2 = 0.f;
                    if (rec.z > 0.f) {
                        j0 = jo0 + rec.z * em0;
                        j1 = jo1 + rec.z * em1;
                        j2 = jo2 + rec.z * em2;
                        P.J[0][q] = j0;
                        P.J[1][q] = j1;
                        P.J[2][q] = j2;
                    }
                    const float n0 = rec.x * em0 + rec.y * (cx - j0);
                    const float n1 = rec.x * em1 + rec.y * (cy - j1);
                    const float n2 = rec.x * em2 + rec.y * (cz - j2);
                    O.E[0][q] = n0;
                    O.E[1][q] = n1;
                    O.E[2][q] = n2;
                    if (!isfinite(n0 + n1 + n2)) atomicOr(P.status, kStatusNonFinite);
                } else {
                    const bool uni = !isnan(rec.x);
                    const bool hvz = P.per[2] || k < P.n[2], inz = P.per[2] || (k >= 1 && k <= P.n[2] - 1);
                    const bool slz = in_slab(P, 2, k);
                    const bool uEx = hvx && iny && inz, uEy = inx && hvy && inz, uEz = inx && iny && hvz;
                    float hz = bzo, hz_ym = bn[2][j - 1][i], hz_xm = bn[2][j][i - 1];
                    float hy = byo, hy_zm = bpy, hy_xm = bn[1][j][i - 1];
                    float hx = bxo, hx_zm = bpx, hx_ym = bn[0][j - 1][i];
                    if (!P.uniform_mu) {
                        if (uni) {
                            hz *= rec.w; hz_ym *= rec.w; hz_xm *= rec.w; hy *= rec.w; hy_zm *= rec.w;
                            hy_xm *= rec.w; hx *= rec.w; hx_zm *= rec.w; hx_ym *= rec.w;
                        } else {
                            const int km = k > 0 ? k - 1 : P.N[2] - 1;
                            const int xm = gx > 0 ? gx - 1 : P.N[0] - 1, ym = gy > 0 ? gy - 1 : P.N[1] - 1;
                            hz *= imu(P, 2, gx, gy, k); hz_ym *= imu(P, 2, gx, ym, k); hz_xm *= imu(P, 2, xm, gy, k);
                            hy *= imu(P, 1, gx, gy, k); hy_zm *= imu(P, 1, gx, gy, km); hy_xm *= imu(P, 1, xm, gy, k);
                            hx *= imu(P, 0, gx, gy, k); hx_zm *= imu(P, 0, gx, gy, km); hx_ym *= imu(P, 0, gx, ym, k);
                        }
                    }
                    const float dHz_y = hz - hz_ym, dHy_z = hy - hy_zm;
                    const float dHx_z = hx - hx_zm, dHz_x = hz - hz_xm;
                    const float dHy_x = hy - hy_xm, dHx_y = hx - hx_ym;
                    float tEx_y = P.r[1] * dHz_y, tEx_z = P.r[2] * dHy_z;
                    float tEy_z = P.r[2] * dHx_z, tEy_x = P.r[0] * dHz_x;
                    float tEz_x = P.r[0] * dHy_x, tEz_y = P.r[1] * dHx_y;
                    if (sly) {
                        if (uEx && P.psiE[0][1]) tEx_y = psi_e(tEx_y, P.psiE[0][1], q, P.pbE[1][gy], P.pcE[1][gy], dHz_y);
                        if (uEz && P.psiE[2][1]) tEz_y = psi_e(tEz_y, P.psiE[2][1], q, P.pbE[1][gy], P.pcE[1][gy], dHx_y);
                    }
                    if (slz) {
                        if (uEx && P.psiE[0][2]) tEx_z = psi_e(tEx_z, P.psiE[0][2], q, P.pbE[2][k], P.pcE[2][k], dHy_z);
                        if (uEy && P.psiE[1][2]) tEy_z = psi_e(tEy_z, P.psiE[1][2], q, P.pbE[2][k], P.pcE[2][k], dHx_z);
                    }
                    if (slx) {
                        if (uEy && P.psiE[1][0]) tEy_x = psi_e(tEy_x, P.psiE[1][0], q, P.pbE[0][gx], P.pcE[0][gx], dHz_x);
                        if (uEz && P.psiE[2][0]) tEz_x = psi_e(tEz_x, P.psiE[2][0], q, P.pbE[0][gx], P.pcE[0][gx], dHy_x);
                    }
                    const float curl[3] = {tEx_y - tEx_z, tEy_z - tEy_x, tEz_x - tEz_y};
                    const bool upd[3] = {uEx, uEy, uEz};
                    const float em[3] = {em0, em1, em2};
                    const float jo[3] = {jo0, jo1, jo2};
                    const bool near_src = k >= src_k0 && k < src_k1;
                    float enew[3];
                    bool bad = false;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        enew[c] = em[c];
                        if (!upd[c]) continue;
                        Mat m;
                        if (uni) m = {rec.x, rec.y, rec.z};
                        else m = edge_coeffs(P, c, gx, gy, k);
                        float jt = 0.f;
                        if (m.cj > 0.f) {
                            jt = jo[c] + m.cj * em[c];
                            P.J[c][q] = jt;
                        }
                        float e = m.ca * em[c] + m.cb * (curl[c] - jt);
                        if (near_src) {
                            for (int s = 0; s < S.n; ++s)
                                if (S.comp[s] == c && gx >= S.lo[s][0] && gx < S.hi[s][0] && gy >= S.lo[s][1] &&
                                    gy < S.hi[s][1] && k >= S.lo[s][2] && k < S.hi[s][2])
                                    e += S.amp[s];
                        }
                        enew[c] = e;
                        O.E[c][q] = e;
                        bad |= !isfinite(e);
                    }
                    if (bad) atomicOr(P.status, kStatusNonFinite);
                    // first-order Mur on the z walls: E_w^{n+1} = E_i^n + M (E_i^{n+1} - E_w^n)
                    if (mur) {
                        const bool mx = hvx && iny, my = inx && hvy;
                        if (k == 1) {
                            if (mx) O.E[0][o] = em[0] + P.mur_M * (enew[0] - elo0);
                            if (my) O.E[1][o] = em[1] + P.mur_M * (enew[1] - elo1);
                        }
                        if (k == P.n[2] - 1) {
                            const int pw = P.n[2] * PL + o;
                            if (mx) O.E[0][pw] = em[0] + P.mur_M * (enew[0] - s1.e[0][j][i]);
                            if (my) O.E[1][pw] = em[1] + P.mur_M * (enew[1] - s1.e[1][j][i]);
                        }
                    }
                }
            }
            if (k == 0) {
                elo0 = s0.e[0][j][i];
                elo1 = s0.e[1][j][i];
            }
            bpx = bxo;
            bpy = byo;
            __syncthreads();   // stage g0 and the B plane are free again
            if (tid == 0 && qq + kStages < nq) {
                issue(qq + kStages);
                ++issued;
            }
        }
        if (abort) {
            // a copy never landed: flag it, give the copies in flight a bounded
            // time to finish (they write this CTA's shared memory), stop
            if (tid == 0) {
                atomicOr(P.status, kStatusTimeout);
                for (unsigned long long gi = g; gi < issued; ++gi)
                    mbar_wait(&bar[gi % kStages], (unsigned)((gi / kStages) & 1));
            }
            __syncthreads();
            return;
        }
        g += nq;
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
    __shared__ float ref[4];
    for (int k = 0; k < P.N[2]; ++k) {
        const int kz[2] = {cellc(2, k - 1), cellc(2, k)};
        if (tx == 0 && ty == 0) {
            const long long m = lin(P, cellc(0, bx * kSX - 1), cellc(1, by * kSY - 1), kz[1]);
            ref[0] = P.eps[m];
            ref[1] = P.sig[m];
            ref[2] = P.kap[m];
            ref[3] = P.mu[m];
        }
        __syncthreads();
        bool same = true;
        // cells x0-1 .. x0+31, y0-1 .. y0+7 (the tile plus its low halo), planes k-1 and k
        for (int t = ty * kTX + tx; t < (kSX + 1) * (kSY + 1); t += kTX * kTY) {
            const int cx = cellc(0, bx * kSX - 1 + t % (kSX + 1)), cy = cellc(1, by * kSY - 1 + t / (kSX + 1));
#pragma unroll
            for (int z = 0; z < 2; ++z) {
                const long long m = lin(P, cx, cy, kz[z]);
                same &= P.eps[m] == ref[0] && P.sig[m] == ref[1] && P.kap[m] == ref[2] && P.mu[m] == ref[3];
            }
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

size_t step_smem_bytes() { return 128 + kStages * sizeof(StageBuf) + 3 * kBoxY * kBoxX * 4 + kStages * 8; }

// opt the kernel in to the dynamic shared memory it needs (above the 48 KB default)
static cudaError_t step_smem_attribute() {
    return cudaFuncSetAttribute(k_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)step_smem_bytes());
}

int step_blocks_per_sm() {
    if (step_smem_attribute() != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step, kTX * kTY, step_smem_bytes()) != cudaSuccess)
        return 1;
    return nb;
}

cudaError_t make_field_tensor_map(void* fields_base, const int N[3], int pitch, size_t field_bytes, int nfields,
                                  void* out128) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    // 4-D view of the field arrays: x (N0 of `pitch` used), y, z, field index
    const cuuint64_t dims[4] = {(cuuint64_t)N[0], (cuuint64_t)N[1], (cuuint64_t)N[2], (cuuint64_t)nfields};
    const cuuint64_t strides[3] = {(cuuint64_t)pitch * 4, (cuuint64_t)pitch * 4 * N[1], (cuuint64_t)field_bytes};
    const cuuint32_t box[4] = {kBoxX, kBoxY, 1, 3};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = encode((CUtensorMap*)out128, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, fields_base, dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_step(const void* tmap128, const Params& P, const StepOut& O, const Sources& S, int blocks,
                        cudaStream_t st) {
    const CUtensorMap* tm = (const CUtensorMap*)tmap128;
    static cudaError_t attr = step_smem_attribute();
    if (attr != cudaSuccess) return attr;
    k_step<<<blocks, dim3(kTX, kTY), step_smem_bytes(), st>>>(*tm, P, O, S);
    return cudaGetLastError();
}

cudaError_t launch_tile_materials(const Params& P, float4* rec, int ntx, int nty, cudaStream_t st) {
    k_tile_materials<<<dim3(ntx, nty), dim3(kTX, kTY), 0, st>>>(P, rec, ntx, nty);
    return cudaGetLastError();
}

}  // namespace tf
