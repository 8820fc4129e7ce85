// tf_step.cu -- fused single-pass step of the two-fluid Yee scheme (sm_103a).
//
// One launch advances the whole grid by one step of Algorithm 1 (arXiv
// 2305.13419, Sec. 3) in its fused leapfrog form:
//   Bt^{n+1/2} = Bt^{n-1/2} - curl(E^n)                   (steps 5 + 1, CPML psi_B)
//   Jt^{n+1/2} = Jt^{n-1/2} + kt_e E^n                     (steps 4 + 2)
//   E^{n+1}    = ca E^n + cb (curl(Bt/mu) - Jt^{n+1/2})     (step 3, CPML psi_E)
// plus soft sources, first-order Mur z walls and the non-finite watchdog.
//
// Work layout.  A CTA of 32 x 16 threads owns a 32 x 16 column tile and
// streams it along z through a chunk of planes.  Each plane's E^n, B^{n-1/2}
// and -- in CPML slabs -- the CPML memory of one slab axis arrive in shared
// memory by TMA (cp.async.bulk.tensor) boxes that cover the tile plus its
// halo, through a ring of kStages buffers whose mbarriers complete on the
// transferred byte count.  Thread 0 keeps the ring full, running ahead into
// the next work item (fetched one item early), so the stream of planes has
// no gap between items.  Per plane:
//   B phase  every thread forms B^{n+1/2} at its column; warps 0 and 1 also
//            recompute the y-1 row / x-1 column of B that the E update needs
//            from the neighbouring tiles; results go to shared memory, owned
//            values to the new B buffer;
//   E phase  every thread forms Js^{n+1/2} and E^{n+1} at its column from the
//            shared B plane and the previous plane's B kept in registers.
// E, B and psi_B ping-pong between two buffers (the other tiles only ever
// read the old ones); Js and psi_E are owned by one thread and update in
// place.  Work items (tile, z chunk) come from an atomic counter; the grid
// fills every SM once.  Periodic x / y seams, which TMA cannot wrap, are
// patched from global memory after the box lands.
//
// Edge material: a tile-plane whose cells are all alike carries one
// precomputed {ca, cb, cj, 1/mu} record; elsewhere per-point coefficients
// (set with the materials) are read.  An interior tile-plane (uniform
// material, no wall, no CPML slab, no source, no Mur plane) takes a path with
// none of those checks.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>

#include "tf_internal.cuh"

namespace tf {

namespace {

struct __align__(128) StageBuf {
    alignas(128) float e[3][kEY][kEX];    // E^n, tile + halo
    alignas(128) float b[3][kBY][kBX];    // B^{n-1/2}, tile + low halo
    alignas(128) float pb[2][kBY][kBX];   // psi_B (old) of the slab axis, tile + low halo
    alignas(128) float pe[2][kTY][kTX];   // psi_E of the slab axis, tile
};
constexpr unsigned kEBytes = 3u * kEY * kEX * 4, kBBytes = 3u * kBY * kBX * 4;
constexpr unsigned kPBBytes = 2u * kBY * kBX * 4, kPEBytes = 2u * kTY * kTX * 4;
constexpr int kThreads = kTX * kTY;

struct TMaps {
    CUtensorMap e, b, pb, pe;
};

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

// position (0 or 1) of component c among the two components != a
__host__ __device__ __forceinline__ int pair_pos(int c, int a) { return c < 3 - a - c ? 0 : 1; }

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

struct Tile {
    int x0, y0, kz0, kz1, ks, nq, bx, by;
};
__device__ __forceinline__ Tile tile_of(const Params& P, const StepOut& O, int item) {
    Tile t;
    const int ch = item % O.nch;   // consecutive items: consecutive chunks of one tile
    const int tile = item / O.nch;
    t.bx = tile % O.ntx;
    t.by = tile / O.ntx;
    t.x0 = t.bx * kSX;
    t.y0 = t.by * kSY;
    t.kz0 = ch * kChunk;
    t.kz1 = min(t.kz0 + kChunk, O.kend);
    t.ks = (t.kz0 > 0 || P.per[2]) ? t.kz0 - 1 : t.kz0;
    t.nq = t.kz1 - t.ks + 1;   // planes pulled: ks .. kz1
    return t;
}
__device__ __forceinline__ int plane_of(const Params& P, const Tile& t, int q) {
    int k = t.ks + q;
    if (k < 0) k += P.N[2];
    if (k >= P.N[2]) k -= P.N[2];
    return k;
}
// the slab axis whose CPML memory travels with the plane (-1: none); z slab
// planes first, then tiles that touch an x slab, then a y slab
__device__ __forceinline__ int slab_axis(const Params& P, const Tile& t, int k) {
    if (P.L[2] > 0 && in_slab(P, 2, k)) return 2;
    if (P.L[0] > 0 && (t.x0 - 1 < P.L[0] || t.x0 + kSX - 1 >= P.n[0] - P.L[0])) return 0;
    if (P.L[1] > 0 && (t.y0 - 1 < P.L[1] || t.y0 + kSY - 1 >= P.n[1] - P.L[1])) return 1;
    return -1;
}

// old psi_B of (component c, axis a) at a point: from the stage when a is the
// staged slab axis, else from global memory
__device__ __forceinline__ float psi_b_old(const Params& P, const StageBuf& s, int sax, int c, int a, int j, int i,
                                           int q) {
    if (a == sax) return s.pb[pair_pos(c, a)][j][i];
    return __ldg(P.psiB[c][a] + q);
}

// B^{n+1/2} at one point of a landed stage, general path (masks and CPML)
struct BPoint {
    float x, y, z;
};
__device__ __forceinline__ BPoint b_general(const Params& P, const StepOut& O, const StageBuf& s0,
                                            const StageBuf& s1, int sax, int j, int i, int gx, int gy, int k,
                                            int q, bool store_psi) {
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
    // psi' = b psi + c d (old buffer), stored by the owner into the new buffer
    auto psi = [&](float& t, int c, int a, int pa, float d, bool u) {
        if (!u) return;
        const float nv = P.pbB[a][pa] * psi_b_old(P, s0, sax, c, a, j, i, q) + P.pcB[a][pa] * d;
        if (store_psi) O.psiB[c][a][q] = nv;
        t += nv;
    };
    if (P.L[1] > 0 && in_slab(P, 1, gy)) {
        psi(tBx_y, 0, 1, gy, dEz_y, uBx);
        psi(tBz_y, 2, 1, gy, dEx_y, uBz);
    }
    if (P.L[2] > 0 && in_slab(P, 2, k)) {
        psi(tBx_z, 0, 2, k, dEy_z, uBx);
        psi(tBy_z, 1, 2, k, dEx_z, uBy);
    }
    if (P.L[0] > 0 && in_slab(P, 0, gx)) {
        psi(tBy_x, 1, 0, gx, dEz_x, uBy);
        psi(tBz_x, 2, 0, gx, dEy_x, uBz);
    }
    BPoint r;
    r.x = uBx ? s0.b[0][j][i] - (tBx_y - tBx_z) : s0.b[0][j][i];
    r.y = uBy ? s0.b[1][j][i] - (tBy_z - tBy_x) : s0.b[1][j][i];
    r.z = uBz ? s0.b[2][j][i] - (tBz_x - tBz_y) : s0.b[2][j][i];
    return r;
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 2)
    k_step(const __grid_constant__ TMaps tm, Params P, StepOut O, Sources S) {
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    // TMA destinations must be 128-byte aligned: round the base up (128 spare bytes are allocated)
    unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    StageBuf* stg = reinterpret_cast<StageBuf*>(smem_raw);
    float(*bn)[kBY][kBX] = reinterpret_cast<float(*)[kBY][kBX]>(smem_raw + kStages * sizeof(StageBuf));
    unsigned long long* bar =
        reinterpret_cast<unsigned long long*>(smem_raw + kStages * sizeof(StageBuf) + 3 * kBY * kBX * 4);
    __shared__ int s_item[2];               // current and next work item (-1: none)
    __shared__ float4 s_rec[2][kChunk + 2]; // material record of each plane of the two items
    __shared__ int s_fast[2][kChunk + 2];   // plane takes the interior path
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTX + tx;
    const int nitems = O.ntx * O.nty * O.nch;
    const int PL = (int)P.plane;
    const bool mur = P.bc[2] == TF_BC_MUR;

    auto fetch = [&]() -> int {   // thread 0: next work item or -1
        const long long d = (long long)(atomicAdd(O.ctr, 1ull) - O.base);
        return (d >= 0 && d < nitems) ? (int)d : -1;
    };
    // interior flags need the tile: computed where the records are stored
    auto axis_clear = [&](int a, int lo, int hi) {   // columns [lo, hi] interior and outside slabs
        if (P.per[a]) return true;
        const int L = P.L[a];
        return lo >= (L > 0 ? L : 1) && hi < P.n[a] - L && hi <= P.n[a] - 1;
    };
    auto z_clear = [&](int k) {
        if (P.per[2]) return true;
        const int L = P.L[2];
        return k >= (L > 0 ? L : 1) && k < P.n[2] - L && k <= P.n[2] - 1;
    };
    auto src_range = [&](const Tile& t, int& k0, int& k1) {   // z range of source planes touching the tile
        k0 = 1 << 30;
        k1 = -1;
        if (S.n > 0 && t.x0 + kSX > S.bb_lo[0] && t.x0 <= S.bb_hi[0] && t.y0 + kSY > S.bb_lo[1] &&
            t.y0 <= S.bb_hi[1]) {
            k0 = S.bb_lo[2];
            k1 = S.bb_hi[2];
        }
    };
    // the records of an item: loaded (by threads < nq - 1) ...
    auto rec_load = [&](int item, float4& r) {
        if (item < 0) return;
        const Tile t = tile_of(P, O, item);
        if (tid < t.nq - 1) r = __ldg(O.tilemat + (long long)(t.by * O.ntx + t.bx) * P.N[2] + plane_of(P, t, tid));
    };
    // ... and stored with the interior flag, later
    auto rec_store = [&](int item, int slot, const float4& r) {
        if (item < 0) return;
        const Tile t = tile_of(P, O, item);
        if (tid < t.nq - 1) {
            const int k = plane_of(P, t, tid);
            int sk0, sk1;
            src_range(t, sk0, sk1);
            const bool tfast = axis_clear(0, t.x0 - 1, t.x0 + kSX - 1) && axis_clear(1, t.y0 - 1, t.y0 + kSY - 1);
            s_rec[slot][tid] = r;
            s_fast[slot][tid] = tfast && z_clear(k) && !isnan(r.x) && (k < sk0 || k >= sk1) &&
                                !(mur && (k == 1 || k == P.n[2] - 1));
        }
    };

    // ---------------------------------------------- producer (thread 0 only)
    // Items are numbered in the order this CTA takes them; item m lives in
    // slot m & 1, and the slot is refilled with item m + 2 once item m is done.
    // The producer may therefore run at most one item ahead of the consumer.
    unsigned long long issued = 0, consumed = 0;   // planes through the ring
    int p_ord = 0, p_q = 0;                        // producer: item ordinal, next plane
    int c_ord = 0;                                 // consumer: item ordinal
    auto issue = [&](const Tile& t, int q, unsigned long long seq) {
        const int s = (int)(seq % kStages);
        const int k = plane_of(P, t, q);
        const int sax = slab_axis(P, t, k);
        const unsigned bytes = kEBytes + kBBytes + (sax >= 0 ? kPBBytes + kPEBytes : 0u);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bar[s], bytes);
        tma_load_box(&stg[s].e[0][0][0], &tm.e, t.x0 - 4, t.y0 - 1, k, O.ecur, &bar[s]);
        tma_load_box(&stg[s].b[0][0][0], &tm.b, t.x0 - 4, t.y0 - 1, k, O.bcur, &bar[s]);
        if (sax >= 0) {
            const int g = 6 * O.psi_slot[sax];
            tma_load_box(&stg[s].pb[0][0][0], &tm.pb, t.x0 - 4, t.y0 - 1, k, g + O.psib_cur, &bar[s]);
            tma_load_box(&stg[s].pe[0][0][0], &tm.pe, t.x0, t.y0, k, g + 4, &bar[s]);
        }
    };
    auto pump = [&]() {   // keep kStages planes in flight, crossing into the next item
        while (issued < consumed + kStages) {
            int item = s_item[p_ord & 1];
            if (item < 0) return;
            Tile t = tile_of(P, O, item);
            if (p_q >= t.nq) {
                if (p_ord > c_ord) return;   // the next slot still holds the current item
                item = s_item[(p_ord + 1) & 1];
                if (item < 0) return;
                ++p_ord;
                p_q = 0;
                t = tile_of(P, O, item);
            }
            issue(t, p_q, issued);
            ++p_q;
            ++issued;
        }
    };

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_item[0] = fetch();
        s_item[1] = s_item[0] >= 0 ? fetch() : -1;
    }
    __syncthreads();
    {
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
        rec_load(s_item[0], r0);
        rec_load(s_item[1], r1);
        rec_store(s_item[0], 0, r0);
        rec_store(s_item[1], 1, r1);
    }
    if (tid == 0) pump();
    __syncthreads();

    int cur = 0;
    bool aborted = false;
    unsigned long long seq0 = 0;   // ring sequence number of plane 0 of the current item
    while (true) {
        const int item = s_item[cur];
        if (item < 0) break;
        const Tile t = tile_of(P, O, item);
        const int x0 = t.x0, y0 = t.y0, kz0 = t.kz0, nq = t.nq;

        // ------------------------------------------------------- column
        const int gx = x0 + tx, gy = y0 + ty;
        const bool valid = gx < P.N[0] && gy < P.N[1];
        const int o = (valid ? gy : 0) * P.pitch + (valid ? gx : 0);
        const int i = tx + 4, j = ty + 1;   // position in the E / B boxes
        const bool hvx = P.per[0] || gx < P.n[0], inx = P.per[0] || (gx >= 1 && gx <= P.n[0] - 1);
        const bool hvy = P.per[1] || gy < P.n[1], iny = P.per[1] || (gy >= 1 && gy <= P.n[1] - 1);
        const bool slx = P.L[0] > 0 && in_slab(P, 0, gx), sly = P.L[1] > 0 && in_slab(P, 1, gy);
        int src_k0, src_k1;
        src_range(t, src_k0, src_k1);
        // periodic seams that the TMA box cannot wrap
        const bool seam = (P.per[0] && (x0 - 4 < 0 || x0 + kEX - 4 > P.N[0])) ||
                          (P.per[1] && (y0 - 1 < 0 || y0 + kEY - 1 > P.N[1]));
        auto patch = [&](StageBuf& sb, int k, int sax) {
            for (int u = tid; u < kEY * kEX; u += kThreads) {
                const int jj = u / kEX, ii = u % kEX;
                const int x = x0 - 4 + ii, y = y0 - 1 + jj;
                if (x >= 0 && x < P.N[0] && y >= 0 && y < P.N[1]) continue;
                const int xw = wrap_or_out(P, 0, x), yw = wrap_or_out(P, 1, y);
                const bool in = xw >= 0 && yw >= 0;
                const int qw = k * PL + (in ? yw : 0) * P.pitch + (in ? xw : 0);
                const bool inb = jj < kBY && ii < kBX;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    sb.e[c][jj][ii] = in ? P.E[c][qw] : 0.f;
                    if (inb) sb.b[c][jj][ii] = in ? P.B[c][qw] : 0.f;
                }
                if (inb && sax >= 0) {
                    for (int c = 0; c < 3; ++c) {
                        if (c == sax) continue;
                        sb.pb[pair_pos(c, sax)][jj][ii] = in ? P.psiB[c][sax][qw] : 0.f;
                    }
                }
            }
        };
        float bpx = 0.f, bpy = 0.f;     // B^{n+1/2}(k-1) at the own column (z differences)
        float elo0 = 0.f, elo1 = 0.f;   // E^n on the low Mur wall
        for (int qq = 0; qq < nq - 1; ++qq) {
            const int k = plane_of(P, t, qq);
            const bool doE = t.ks + qq >= kz0;
            const unsigned long long g0 = seq0 + qq, g1 = g0 + 1;
            StageBuf& s0 = stg[g0 % kStages];
            StageBuf& s1 = stg[g1 % kStages];
            const int sax = slab_axis(P, t, k);
            const float4 rec = s_rec[cur][qq];
            const bool fast = s_fast[cur][qq] != 0;
            const int q = k * PL + o;
            // global reads of this plane that do not depend on the stage: issue first
            float jo0 = 0.f, jo1 = 0.f, jo2 = 0.f;
            float mc[9];
            const bool uni = !isnan(rec.x);
            if (doE && valid && (!uni || rec.z > 0.f)) {
                jo0 = P.J[0][q];
                jo1 = P.J[1][q];
                jo2 = P.J[2][q];
            }
            if (doE && valid && !uni) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    mc[c] = __ldg(P.ca[c] + q);
                    mc[3 + c] = __ldg(P.cb[c] + q);
                    mc[6 + c] = __ldg(P.cj[c] + q);
                }
            }
            bool ok = mbar_wait(&bar[g0 % kStages], (unsigned)((g0 / kStages) & 1));
            ok = ok && mbar_wait(&bar[g1 % kStages], (unsigned)((g1 / kStages) & 1));
            if (__syncthreads_or(!ok)) {
                aborted = true;
                break;
            }
            if (seam) {
                if (qq == 0) patch(s0, k, sax);
                const int k1 = plane_of(P, t, qq + 1);
                patch(s1, k1, slab_axis(P, t, k1));
                __syncthreads();
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
                const BPoint bp =
                    b_general(P, O, s0, s1, sax, j, i, valid ? gx : 0, valid ? gy : 0, k, q, doE && valid);
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
                        const BPoint h = b_general(P, O, s0, s1, sax, jh, ih, hxg, hyg, k, qh, false);
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
                    const bool hvz = P.per[2] || k < P.n[2], inz = P.per[2] || (k >= 1 && k <= P.n[2] - 1);
                    const bool slz = P.L[2] > 0 && in_slab(P, 2, k);
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
                    // psi' = b psi + c d, in place; the staged copy serves the slab axis
                    auto psi = [&](float& tt, int c, int a, int pa, float d) {
                        const float old = (a == sax) ? s0.pe[pair_pos(c, a)][ty][tx] : P.psiE[c][a][q];
                        const float nv = P.pbE[a][pa] * old + P.pcE[a][pa] * d;
                        P.psiE[c][a][q] = nv;
                        tt += nv;
                    };
                    if (sly) {
                        if (uEx) psi(tEx_y, 0, 1, gy, dHz_y);
                        if (uEz) psi(tEz_y, 2, 1, gy, dHx_y);
                    }
                    if (slz) {
                        if (uEx) psi(tEx_z, 0, 2, k, dHy_z);
                        if (uEy) psi(tEy_z, 1, 2, k, dHx_z);
                    }
                    if (slx) {
                        if (uEy) psi(tEy_x, 1, 0, gx, dHz_x);
                        if (uEz) psi(tEz_x, 2, 0, gx, dHy_x);
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
                        const float ca = uni ? rec.x : mc[c], cb = uni ? rec.y : mc[3 + c],
                                    cj = uni ? rec.z : mc[6 + c];
                        float jt = 0.f;
                        if (cj > 0.f) {
                            jt = jo[c] + cj * em[c];
                            P.J[c][q] = jt;
                        }
                        float e = ca * em[c] + cb * (curl[c] - jt);
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
            __syncthreads();   // stage g0 (and, after the last plane, g1) and the B plane are free again
            if (tid == 0) {
                consumed = g0 + 1 + (qq == nq - 2 ? 1 : 0);
                pump();
            }
        }
        if (aborted) break;
        seq0 += nq;
        // this item is done: its slot takes the item after the next one
        if (tid == 0) s_item[cur] = s_item[cur ^ 1] >= 0 ? fetch() : -1;
        __syncthreads();
        {
            float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
            rec_load(s_item[cur], r);
            rec_store(s_item[cur], cur, r);
        }
        cur ^= 1;
        if (tid == 0) {
            ++c_ord;
            pump();
        }
        __syncthreads();
    }
    if (aborted) {
        // a copy never landed: flag it, give the copies in flight a bounded
        // time to finish (they write this CTA's shared memory), stop
        if (tid == 0) {
            atomicOr(P.status, kStatusTimeout);
            for (unsigned long long gi = consumed; gi < issued; ++gi)
                mbar_wait(&bar[gi % kStages], (unsigned)((gi / kStages) & 1));
        }
        __syncthreads();
    }
}

// per (tile, plane): are all cells an owned edge or face of the tile-plane
// touches alike?  Then store {ca, cb, cj, 1/mu}; else ca = NaN
__global__ void k_tile_materials(Params P, float4* rec, int ntx, int nty) {
    const int bx = blockIdx.x, by = blockIdx.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
    auto cellc = [&](int a, int v) {
        if (v < 0) return P.per[a] ? v + P.n[a] : 0;
        if (v >= P.n[a]) return P.per[a] ? v - P.n[a] : P.n[a] - 1;
        return v;
    };
    __shared__ float ref[4];
    for (int k = 0; k < P.N[2]; ++k) {
        const int kz[2] = {cellc(2, k - 1), cellc(2, k)};
        if (tid == 0) {
            const long long m = lin(P, cellc(0, bx * kSX - 1), cellc(1, by * kSY - 1), kz[1]);
            ref[0] = P.eps[m];
            ref[1] = P.sig[m];
            ref[2] = P.kap[m];
            ref[3] = P.mu[m];
        }
        __syncthreads();
        bool same = true;
        // cells x0-1 .. x0+kSX-1, y0-1 .. y0+kSY-1 (the tile plus its low halo), planes k-1 and k
        for (int t = tid; t < (kSX + 1) * (kSY + 1); t += nth) {
            const int cx = cellc(0, bx * kSX - 1 + t % (kSX + 1)), cy = cellc(1, by * kSY - 1 + t / (kSX + 1));
#pragma unroll
            for (int z = 0; z < 2; ++z) {
                const long long m = lin(P, cx, cy, kz[z]);
                same &= P.eps[m] == ref[0] && P.sig[m] == ref[1] && P.kap[m] == ref[2] && P.mu[m] == ref[3];
            }
        }
        same = __syncthreads_and(same);
        if (tid == 0) {
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

size_t step_smem_bytes() { return 128 + kStages * sizeof(StageBuf) + 3 * kBY * kBX * 4 + kStages * 8; }

// opt the kernel in to the dynamic shared memory it needs (above the 48 KB default)
static cudaError_t step_smem_attribute() {
    return cudaFuncSetAttribute(k_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)step_smem_bytes());
}

int step_blocks_per_sm() {
    if (step_smem_attribute() != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step, kThreads, step_smem_bytes()) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t make_tensor_map(void* base, const int N[3], int pitch, size_t array_bytes, int narrays, int bx, int by,
                            int bf, void* out128) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    // 4-D view: x (N0 of `pitch` used), y, z, array index
    const cuuint64_t dims[4] = {(cuuint64_t)N[0], (cuuint64_t)N[1], (cuuint64_t)N[2], (cuuint64_t)narrays};
    const cuuint64_t strides[3] = {(cuuint64_t)pitch * 4, (cuuint64_t)pitch * 4 * N[1], (cuuint64_t)array_bytes};
    const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, (cuuint32_t)bf};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = encode((CUtensorMap*)out128, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_step(const void* tmaps512, const Params& P, const StepOut& O, const Sources& S, int blocks,
                        cudaStream_t st) {
    static cudaError_t attr = step_smem_attribute();
    if (attr != cudaSuccess) return attr;
    const TMaps* tm = (const TMaps*)tmaps512;
    k_step<<<blocks, dim3(kTX, kTY), step_smem_bytes(), st>>>(*tm, P, O, S);
    return cudaGetLastError();
}

cudaError_t launch_tile_materials(const Params& P, float4* rec, int ntx, int nty, cudaStream_t st) {
    k_tile_materials<<<dim3(ntx, nty), dim3(32, 8), 0, st>>>(P, rec, ntx, nty);
    return cudaGetLastError();
}

// per-point edge coefficients of the theta scheme (used where a tile-plane's material varies)
__global__ void k_edge_coeffs(Params P) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= P.N[0] || j >= P.N[1]) return;
    const int p[3] = {i, j, k};
    const long long q = lin(P, i, j, k);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float ca = 1.f, cb = 0.f, cj = 0.f;
        if (upd_E(P, c, p)) {
            float eps, st, kt;
            edge_material(P, c, p, eps, st, kt);
            const float den = eps + P.theta * st;
            ca = (eps - (1.f - P.theta) * st) / den;
            cb = 1.f / den;
            cj = kt;
        }
        const_cast<float*>(P.ca[c])[q] = ca;
        const_cast<float*>(P.cb[c])[q] = cb;
        const_cast<float*>(P.cj[c])[q] = cj;
    }
}

cudaError_t launch_edge_coeffs(const Params& P, cudaStream_t st) {
    k_edge_coeffs<<<dim3((P.N[0] + 31) / 32, (P.N[1] + 7) / 8, P.N[2]), dim3(32, 8), 0, st>>>(P);
    return cudaGetLastError();
}

}  // namespace tf
