// tf_step.cu -- fused single-pass step of the two-fluid Yee scheme (sm_103a).
//
// One launch advances the whole grid by one step of Algorithm 1 (arXiv
// 2305.13419, Sec. 3) in its fused leapfrog form:
//   Bt^{n+1/2} = Bt^{n-1/2} - curl(E^n)                   (steps 5 + 1, CPML psi_B)
//   Jt^{n+1/2} = Jt^{n-1/2} + kt_e E^n                     (steps 4 + 2)
//   E^{n+1}    = ca E^n + cb (curl(Bt/mu) - Jt^{n+1/2})     (step 3, CPML psi_E)
// plus soft sources, first-order Mur z walls and the non-finite watchdog.
//
// Work layout.  A CTA of 32 x 8 threads owns a 32 x 16 column tile, two
// adjacent rows per thread, and streams it along z through a chunk of planes.
// Each plane's E^n, B^{n-1/2} and -- where a CPML slab reaches the tile-plane
// -- the CPML memory psi_B of one slab axis arrive in shared memory by TMA
// (cp.async.bulk.tensor) boxes covering the tile plus its halo, through a
// ring of kStages buffers whose mbarriers complete on the transferred byte
// count.  Thread 0 keeps the ring full and runs ahead into the next work
// item, so the stream of planes has no gap between items.  Per plane:
//   B phase  every thread forms B^{n+1/2} at its two points; warp 0 also forms
//            the y0-1 row and half of warp 1 the x0-1 column of B that the E
//            update needs from the neighbouring tiles; the plane of new B goes
//            to one of two shared buffers, owned values to the new B array;
//   barrier  (the only one per plane; it also frees the stage of the plane
//            before, which thread 0 then refills);
//   E phase  every thread forms Js^{n+1/2} and E^{n+1} at its two points from
//            the shared B plane and the previous plane's B kept in registers.
// E, B and psi_B ping-pong between two arrays (the other tiles only ever read
// the old ones); Js and psi_E are owned by one thread and update in place.
// Work items (tile, z chunk) come from an atomic counter, fetched one item
// ahead; the grid fills every SM twice.  Periodic x / y seams, which a TMA box
// cannot wrap, are patched from global memory after the box lands.
//
// One code path serves every plane: x / y walls by per-column masks, the z
// wall plane by plane masks, the CPML memory of the staged axis from shared
// memory and of any further slab axis from global memory, and either one
// precomputed {ca, cb, cj, 1/mu} record (all cells of the tile-plane alike)
// or per-point coefficients set with the materials.  Sources, Mur planes and
// per-face mu take branches that are uniform across the CTA.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>

#include <type_traits>

#include "tf_internal.cuh"

namespace tf {

namespace {

struct __align__(128) StageBuf {
    alignas(128) float e[3][kEY][kEX];    // E^n, tile + halo
    alignas(128) float b[3][kBY][kBX];    // B^{n-1/2}, tile + low halo
    alignas(128) float pb[2][kBY][kBX];   // old psi_B of the staged slab axis, tile + low halo
};
constexpr unsigned kEBytes = 3u * kEY * kEX * 4, kBBytes = 3u * kBY * kBX * 4, kPBBytes = 2u * kBY * kBX * 4;
constexpr int kThreadsY = kTY / kRows;
constexpr int kThreads = kTX * kThreadsY;
constexpr size_t kBPlaneBytes = 3u * kBY * kBX * 4;

// per-plane flags of a work item
enum : unsigned {
    kFCoef = 1u << 0,    // material varies across the tile-plane: per-point coefficients
    kFImu = 1u << 1,     // ... and so does mu: per-face 1/mu
    kFZlo = 1u << 2,     // the low wall plane of a walled z axis
    kFSrc = 1u << 3,     // soft sources reach the tile on this plane
    kFMurLo = 1u << 4,   // Mur: next to the low / high z wall
    kFMurHi = 1u << 5,
    kFSec0 = 1u << 6,    // CPML slabs of axis 0, 1, 2 reach the plane besides the staged one
};
constexpr int kFSaxShift = 9;   // staged slab axis + 1 (0: none), two bits

struct TMaps {
    CUtensorMap e, b, pb;
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

// the two components != a, ascending (the pair a CPML axis acts on)
__host__ __device__ __forceinline__ int pair_c1(int a) { return a == 0 ? 1 : 0; }
__host__ __device__ __forceinline__ int pair_c2(int a) { return a == 2 ? 1 : 2; }

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
// CPML slab axes reaching a tile-plane: bit a is set when the plane (z) or
// the tile's columns with their low halo (x, y) overlap the slab of axis a
__device__ __forceinline__ int slab_bits(const Params& P, const Tile& t, int k) {
    int m = 0;
    if (P.L[0] > 0 && (t.x0 - 1 < P.L[0] || t.x0 + kSX - 1 >= P.n[0] - P.L[0])) m |= 1;
    if (P.L[1] > 0 && (t.y0 - 1 < P.L[1] || t.y0 + kSY - 1 >= P.n[1] - P.L[1])) m |= 2;
    if (P.L[2] > 0 && in_slab(P, 2, k)) m |= 4;
    return m;
}
// the slab axis whose CPML memory travels with the plane: z, else x, else y (-1: none)
__device__ __forceinline__ int slab_axis(int bits) { return (bits & 4) ? 2 : (bits & 1) ? 0 : (bits & 2) ? 1 : -1; }

// position p on axis a inside its CPML slab (p may lie outside the grid)
__device__ __forceinline__ bool slab_pos(const Params& P, int a, int p) {
    return p >= 0 && p < P.N[a] && in_slab(P, a, p);
}

struct V3 {
    float x, y, z;
};

// B^{n+1/2} before masking at box position (j, i) of landed stages s0 (plane
// k) and s1 (plane k + 1): the curl update plus the CPML memory of the staged
// axis sax (coefficients bB, cB; zero outside the slab), whose new values
// come back in p0, p1 (pair order)
__device__ __forceinline__ V3 b_update(const Params& P, const StageBuf& s0, const StageBuf& s1, int j, int i,
                                       int sax, float bB, float cB, float& p0, float& p1) {
    const float ex = s0.e[0][j][i], ey = s0.e[1][j][i], ez = s0.e[2][j][i];
    const float dEz_y = s0.e[2][j + 1][i] - ez, dEy_z = s1.e[1][j][i] - ey;
    const float dEx_z = s1.e[0][j][i] - ex, dEz_x = s0.e[2][j][i + 1] - ez;
    const float dEy_x = s0.e[1][j][i + 1] - ey, dEx_y = s0.e[0][j + 1][i] - ex;
    V3 r;
    r.x = s0.b[0][j][i] - (P.r[1] * dEz_y - P.r[2] * dEy_z);
    r.y = s0.b[1][j][i] - (P.r[2] * dEx_z - P.r[0] * dEz_x);
    r.z = s0.b[2][j][i] - (P.r[0] * dEy_x - P.r[1] * dEx_y);
    p0 = 0.f;
    p1 = 0.f;
    if (sax == 0) {          // By, Bz
        p0 = bB * s0.pb[0][j][i] + cB * dEz_x;
        p1 = bB * s0.pb[1][j][i] + cB * dEy_x;
        r.y += p0;
        r.z -= p1;
    } else if (sax == 1) {   // Bx, Bz
        p0 = bB * s0.pb[0][j][i] + cB * dEz_y;
        p1 = bB * s0.pb[1][j][i] + cB * dEx_y;
        r.x -= p0;
        r.z += p1;
    } else if (sax == 2) {   // Bx, By
        p0 = bB * s0.pb[0][j][i] + cB * dEy_z;
        p1 = bB * s0.pb[1][j][i] + cB * dEx_z;
        r.x += p0;
        r.y -= p1;
    }
    return r;
}

// CPML memory of a further slab axis a at box position (j, i): old values from
// global memory (psi index q), new values added to B and returned
__device__ __forceinline__ void b_psi_extra(const Params& P, const StageBuf& s0, const StageBuf& s1, int j, int i,
                                            int a, int pos, int q, V3& b, float& p0, float& p1) {
    float d0, d1;
    if (a == 0) {
        d0 = s0.e[2][j][i + 1] - s0.e[2][j][i];
        d1 = s0.e[1][j][i + 1] - s0.e[1][j][i];
    } else if (a == 1) {
        d0 = s0.e[2][j + 1][i] - s0.e[2][j][i];
        d1 = s0.e[0][j + 1][i] - s0.e[0][j][i];
    } else {
        d0 = s1.e[1][j][i] - s0.e[1][j][i];
        d1 = s1.e[0][j][i] - s0.e[0][j][i];
    }
    const float bb = __ldg(P.pbB[a] + pos), cc = __ldg(P.pcB[a] + pos);
    p0 = bb * __ldg(P.psiB[pair_c1(a)][a] + q) + cc * d0;
    p1 = bb * __ldg(P.psiB[pair_c2(a)][a] + q) + cc * d1;
    if (a == 0) {
        b.y += p0;
        b.z -= p1;
    } else if (a == 1) {
        b.x -= p0;
        b.z += p1;
    } else {
        b.x += p0;
        b.y -= p1;
    }
}

// z range [k0, k1) of the source planes reaching a tile (empty: k0 > k1)
__device__ __forceinline__ void src_range(const Sources& S, const Tile& t, int& k0, int& k1) {
    k0 = 1 << 30;
    k1 = -1;
    if (S.n > 0 && t.x0 + kSX > S.bb_lo[0] && t.x0 <= S.bb_hi[0] && t.y0 + kSY > S.bb_lo[1] && t.y0 <= S.bb_hi[1]) {
        k0 = S.bb_lo[2];
        k1 = S.bb_hi[2];
    }
}

// an item needs the full plane loop: varying mu, a second CPML axis on one
// of its planes, a source plane or a Mur plane
__device__ __forceinline__ bool item_is_rare(const Params& P, const Sources& S, bool mur, const Tile& t) {
    if (!P.uniform_mu) return true;
    const int ka = t.ks < 0 ? 0 : t.ks, kb = t.kz1 - 1;   // planes of the item (periodic wrap: z has no slab)
    const bool sx = P.L[0] > 0 && (t.x0 - 1 < P.L[0] || t.x0 + kSX - 1 >= P.n[0] - P.L[0]);
    const bool sy = P.L[1] > 0 && (t.y0 - 1 < P.L[1] || t.y0 + kSY - 1 >= P.n[1] - P.L[1]);
    const bool sz = P.L[2] > 0 && (ka < P.L[2] || kb >= P.n[2] - P.L[2]);
    if ((int)sx + (int)sy + (int)sz >= 2) return true;
    int sk0, sk1;
    src_range(S, t, sk0, sk1);
    if (sk1 > sk0 && ((kb >= sk0 && ka < sk1) || (t.ks < 0 && P.N[2] - 1 >= sk0 && P.N[2] - 1 < sk1))) return true;
    return mur && ((ka <= 1 && 1 <= kb) || (ka <= P.n[2] - 1 && P.n[2] - 1 <= kb));
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 2)
    k_step(const __grid_constant__ TMaps tm, Params P, StepOut O, Sources S) {
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    // TMA destinations must be 128-byte aligned: round the base up (128 spare bytes are allocated)
    unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    StageBuf* stg = reinterpret_cast<StageBuf*>(smem_raw);
    float(*bplanes)[3][kBY][kBX] = reinterpret_cast<float(*)[3][kBY][kBX]>(smem_raw + kStages * sizeof(StageBuf));
    unsigned long long* bar =
        reinterpret_cast<unsigned long long*>(smem_raw + kStages * sizeof(StageBuf) + 2 * kBPlaneBytes);
    __shared__ int s_item[2];                   // current and next work item (-1: none)
    __shared__ float4 s_rec[2][kChunk + 2];     // material record of each plane of the two items
    __shared__ unsigned s_flag[2][kChunk + 2];  // plane flags
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTX + tx;
    const int nitems = O.ntx * O.nty * O.nch;
    const int PL = (int)P.plane;
    const bool mur = P.bc[2] == TF_BC_MUR;

    auto fetch = [&]() -> int {   // thread 0: next work item or -1 (items that take the full loop come first)
        const long long d = (long long)(atomicAdd(O.ctr, 1ull) - O.base);
        return (d >= 0 && d < nitems) ? __ldg(O.order + d) : -1;
    };
    // the records of an item: loaded by threads < nq - 1 ...
    auto rec_load = [&](int item, float4& r) {
        if (item < 0) return;
        const Tile t = tile_of(P, O, item);
        if (tid < t.nq - 1) r = __ldg(O.tilemat + (long long)(t.by * O.ntx + t.bx) * P.N[2] + plane_of(P, t, tid));
    };
    // ... and stored with the plane flags
    auto rec_store = [&](int item, int slot, const float4& r) {
        if (item < 0) return;
        const Tile t = tile_of(P, O, item);
        if (tid < t.nq - 1) {
            const int k = plane_of(P, t, tid);
            int sk0, sk1;
            src_range(S, t, sk0, sk1);
            const int bits = slab_bits(P, t, k);
            const int sax = slab_axis(bits);
            const int sec = bits & ~(sax >= 0 ? 1 << sax : 0);
            const bool uni = !isnan(r.x);
            unsigned f = (unsigned)(sax + 1) << kFSaxShift | (unsigned)sec * kFSec0;
            if (!uni) f |= kFCoef;
            if (!uni && !P.uniform_mu) f |= kFImu;
            if (!P.per[2] && k == 0) f |= kFZlo;
            if (k >= sk0 && k < sk1) f |= kFSrc;
            if (mur && k == 1) f |= kFMurLo;
            if (mur && k == P.n[2] - 1) f |= kFMurHi;
            s_rec[slot][tid] = r;
            s_flag[slot][tid] = f;
        }
    };

    // ---------------------------------------------- producer (thread 0 only)
    // Items are numbered in the order this CTA takes them; item m lives in
    // slot m & 1, and the slot is refilled with item m + 2 once item m is done.
    // The producer may therefore run at most one item ahead of the consumer.
    unsigned long long issued = 0, consumed = 0;   // planes through the ring
    int p_ord = 0, p_q = 0;                        // producer: item ordinal, next plane
    int c_ord = 0;                                 // consumer: item ordinal
    Tile p_t;                                      // producer: tile of item p_ord
    p_t.nq = 0;
    bool p_have = false;
    auto issue = [&](const Tile& t, int q, unsigned long long seq) {
        const int s = (int)(seq % kStages);
        const int k = plane_of(P, t, q);
        const int sax = slab_axis(slab_bits(P, t, k));
        const unsigned bytes = kEBytes + kBBytes + (sax >= 0 ? kPBBytes : 0u);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bar[s], bytes);
        tma_load_box(&stg[s].e[0][0][0], &tm.e, t.x0 - 4, t.y0 - 1, k, O.ecur, &bar[s]);
        tma_load_box(&stg[s].b[0][0][0], &tm.b, t.x0 - 4, t.y0 - 1, k, O.bcur, &bar[s]);
        if (sax >= 0)
            tma_load_box(&stg[s].pb[0][0][0], &tm.pb, t.x0 - 4, t.y0 - 1, k, 6 * O.psi_slot[sax] + O.psib_cur,
                         &bar[s]);
    };
    auto pump = [&]() {   // keep kStages planes in flight, crossing into the next item
        while (issued < consumed + kStages) {
            if (!p_have) {
                const int item = s_item[p_ord & 1];
                if (item < 0) return;
                p_t = tile_of(P, O, item);
                p_have = true;
            }
            if (p_q >= p_t.nq) {
                if (p_ord > c_ord) return;   // the next slot still holds the current item
                const int item = s_item[(p_ord + 1) & 1];
                if (item < 0) return;
                ++p_ord;
                p_q = 0;
                p_t = tile_of(P, O, item);
            }
            issue(p_t, p_q, issued);
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
    unsigned it = 0;               // planes done by this CTA (selects the shared B plane)
    int pend = -1;                 // thread 0: the item after the next one
    while (true) {
        const int item = s_item[cur];
        if (item < 0) break;
        const Tile t = tile_of(P, O, item);
        const int x0 = t.x0, y0 = t.y0, kz0 = t.kz0, nq = t.nq;

        // ------------------------------------------------------- columns
        const int gx = x0 + tx;
        const int i = tx + 4;   // x position in the E / B boxes
        const bool hvx = P.per[0] || gx < P.n[0], inx = P.per[0] || (gx >= 1 && gx <= P.n[0] - 1);
        int gy[kRows], o[kRows];
        bool valid[kRows], hvy[kRows], iny[kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            gy[r] = y0 + kRows * ty + r;
            valid[r] = gx < P.N[0] && gy[r] < P.N[1];
            o[r] = valid[r] ? gy[r] * P.pitch + gx : 0;
            hvy[r] = P.per[1] || gy[r] < P.n[1];
            iny[r] = P.per[1] || (gy[r] >= 1 && gy[r] <= P.n[1] - 1);
        }
        const int j0 = kRows * ty + 1;   // y position of row 0 in the E / B boxes
        // halo point of warp 0 (row y0 - 1) / lanes 0..15 of warp 1 (column x0 - 1)
        const bool hrow = ty == 0, hcol = ty == 1 && tx < kTY;
        const int hgx = hrow ? gx : x0 - 1, hgy = hrow ? y0 - 1 : y0 + tx;
        const int hj = hrow ? 0 : tx + 1, hi = hrow ? i : 3;
        const bool hhvx = P.per[0] || hgx < P.n[0], hinx = P.per[0] || (hgx >= 1 && hgx <= P.n[0] - 1);
        const bool hhvy = P.per[1] || hgy < P.n[1], hiny = P.per[1] || (hgy >= 1 && hgy <= P.n[1] - 1);
        const int hxw = wrap_or_out(P, 0, hgx), hyw = wrap_or_out(P, 1, hgy);
        const bool hin = hxw >= 0 && hyw >= 0;
        const int ho = hin ? hyw * P.pitch + hxw : 0;
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
                    sb.pb[0][jj][ii] = in ? P.psiB[pair_c1(sax)][sax][qw] : 0.f;
                    sb.pb[1][jj][ii] = in ? P.psiB[pair_c2(sax)][sax][qw] : 0.f;
                }
            }
        };
        float4 rnext = make_float4(0.f, 0.f, 0.f, 0.f);   // records of the next item
        V3 bprev[kRows];                                    // B^{n+1/2}(k-1) at the own points
        float elo[kRows][2];                                // E^n on the low Mur wall
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            bprev[r].x = bprev[r].y = bprev[r].z = 0.f;
            elo[r][0] = elo[r][1] = 0.f;
        }
        // the plane loop, compiled twice: items that meet a source, a Mur plane,
        // a second CPML axis or varying mu run the full version, all others a
        // version without that code
        auto planes = [&](auto rare_tag) {
            constexpr bool kRare = decltype(rare_tag)::value;
            for (int qq = 0; qq < nq - 1; ++qq, ++it) {
                const int k = plane_of(P, t, qq);
                const bool doE = t.ks + qq >= kz0;   // E update (and B store) at this plane
                const unsigned long long g0 = seq0 + qq, g1 = g0 + 1;
                StageBuf& s0 = stg[g0 % kStages];
                StageBuf& s1 = stg[g1 % kStages];
                const unsigned f = s_flag[cur][qq];
                const float4 rec = s_rec[cur][qq];
                const int sax = (int)((f >> kFSaxShift) & 3u) - 1;
                const bool coef = (f & kFCoef) != 0, zlo = (f & kFZlo) != 0;
                const unsigned sec = (f / kFSec0) & 7u;
                float(*bn)[kBY][kBX] = bplanes[it & 1];
                const int kq = k * PL;
                // global reads that do not depend on the stage: issued before the wait
                float jo[kRows][3], mc[kRows][9], pe[kRows][2];
                float bB[kRows], cB[kRows], bE[kRows], cE[kRows];
                bool insl[kRows];
    #pragma unroll
                for (int r = 0; r < kRows; ++r) {
                    const bool own = valid[r] && doE;
                    const int q = kq + o[r];
    #pragma unroll
                    for (int c = 0; c < 3; ++c) jo[r][c] = (own && (coef || rec.z > 0.f)) ? P.J[c][q] : 0.f;
                    if (own && coef) {
    #pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            mc[r][c] = __ldg(P.ca[c] + q);
                            mc[r][3 + c] = __ldg(P.cb[c] + q);
                            mc[r][6 + c] = __ldg(P.cj[c] + q);
                        }
                    } else {
    #pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            mc[r][c] = rec.x;
                            mc[r][3 + c] = rec.y;
                            mc[r][6 + c] = rec.z;
                        }
                    }
                    bB[r] = cB[r] = bE[r] = cE[r] = pe[r][0] = pe[r][1] = 0.f;
                    insl[r] = false;
                    if (sax >= 0) {
                        const int pos = sax == 0 ? gx : sax == 1 ? gy[r] : k;
                        insl[r] = slab_pos(P, sax, pos);
                        if (insl[r]) {
                            bB[r] = __ldg(P.pbB[sax] + pos);
                            cB[r] = __ldg(P.pcB[sax] + pos);
                            bE[r] = __ldg(P.pbE[sax] + pos);
                            cE[r] = __ldg(P.pcE[sax] + pos);
                            if (own) {
                                pe[r][0] = P.psiE[pair_c1(sax)][sax][q];
                                pe[r][1] = P.psiE[pair_c2(sax)][sax][q];
                            }
                        }
                    }
                }
                float hbB = 0.f, hcB = 0.f;
                if ((hrow || hcol) && sax >= 0) {
                    const int hpos = sax == 0 ? hgx : sax == 1 ? hgy : k;
                    if (slab_pos(P, sax, hpos)) {
                        hbB = __ldg(P.pbB[sax] + hpos);
                        hcB = __ldg(P.pcB[sax] + hpos);
                    }
                }
                bool ok = mbar_wait(&bar[g1 % kStages], (unsigned)((g1 / kStages) & 1));
                if (qq == 0) ok = ok && mbar_wait(&bar[g0 % kStages], (unsigned)((g0 / kStages) & 1));
                if (seam) {
                    if (qq == 0) patch(s0, k, sax);
                    const int k1 = plane_of(P, t, qq + 1);
                    patch(s1, k1, slab_axis(slab_bits(P, t, k1)));
                    __syncthreads();
                }

                // ------------------------------------------------ B phase
                V3 nb[kRows];
    #pragma unroll
                for (int r = 0; r < kRows; ++r) {
                    const int j = j0 + r;
                    const bool own = valid[r] && doE;
                    const int q = kq + o[r];
                    const bool ux = inx && hvy[r], uy = hvx && iny[r], uz = hvx && hvy[r] && !zlo;
                    float p0, p1;
                    V3 b = b_update(P, s0, s1, j, i, sax, bB[r], cB[r], p0, p1);
                    if (own && insl[r]) {
                        if (sax == 0 ? uy : ux) O.psiB[pair_c1(sax)][sax][q] = p0;
                        if (sax == 2 ? uy : uz) O.psiB[pair_c2(sax)][sax][q] = p1;
                    }
                    if (kRare && sec) {
    #pragma unroll 1
                        for (int a = 0; a < 3; ++a) {
                            if (!((sec >> a) & 1u)) continue;
                            const int pos = a == 0 ? gx : a == 1 ? gy[r] : k;
                            if (!valid[r] || !slab_pos(P, a, pos)) continue;
                            float e0, e1;
                            b_psi_extra(P, s0, s1, j, i, a, pos, q, b, e0, e1);
                            if (own) {
                                if (a == 0 ? uy : ux) O.psiB[pair_c1(a)][a][q] = e0;
                                if (a == 2 ? uy : uz) O.psiB[pair_c2(a)][a][q] = e1;
                            }
                        }
                    }
                    nb[r].x = ux ? b.x : s0.b[0][j][i];
                    nb[r].y = uy ? b.y : s0.b[1][j][i];
                    nb[r].z = uz ? b.z : s0.b[2][j][i];
                    bn[0][j][i] = nb[r].x;
                    bn[1][j][i] = nb[r].y;
                    bn[2][j][i] = nb[r].z;
                    if (own) {
                        O.B[0][q] = nb[r].x;
                        O.B[1][q] = nb[r].y;
                        O.B[2][q] = nb[r].z;
                    }
                }
                if (hrow || hcol) {
                    const bool ux = hinx && hhvy, uy = hhvx && hiny, uz = hhvx && hhvy && !zlo;
                    float p0, p1;
                    V3 b = b_update(P, s0, s1, hj, hi, sax, hbB, hcB, p0, p1);
                    if (kRare && sec && hin) {
    #pragma unroll 1
                        for (int a = 0; a < 3; ++a) {
                            if (!((sec >> a) & 1u)) continue;
                            const int pos = a == 0 ? hxw : a == 1 ? hyw : k;
                            if (slab_pos(P, a, pos)) b_psi_extra(P, s0, s1, hj, hi, a, pos, kq + ho, b, p0, p1);
                        }
                    }
                    if (hrow) {
                        bn[0][hj][hi] = ux ? b.x : s0.b[0][hj][hi];
                    } else {
                        bn[1][hj][hi] = uy ? b.y : s0.b[1][hj][hi];
                    }
                    bn[2][hj][hi] = uz ? b.z : s0.b[2][hj][hi];
                }
                if (qq == 1) rec_store(s_item[cur ^ 1], cur ^ 1, rnext);   // loaded during plane 0
                // every thread is past the E phase of the plane before: its stage is free
                if (__syncthreads_or(!ok)) {
                    aborted = true;
                    break;
                }
                if (tid == 0) {
                    consumed = g0;
                    pump();
                    if (qq == 0) pend = s_item[cur ^ 1] >= 0 ? fetch() : -1;
                }
                if (qq == 0) rec_load(s_item[cur ^ 1], rnext);

                // ------------------------------------------------ E phase
    #pragma unroll
                for (int r = 0; r < kRows; ++r) {
                    const int j = j0 + r;
                    const int q = kq + o[r];
                    if (valid[r] && doE) {
                        const float em0 = s0.e[0][j][i], em1 = s0.e[1][j][i], em2 = s0.e[2][j][i];
                        const bool ux = hvx && iny[r] && !zlo, uy = inx && hvy[r] && !zlo, uz = inx && iny[r];
                        float hx = nb[r].x, hx_zm = bprev[r].x, hx_ym = r > 0 ? nb[r - 1].x : bn[0][j - 1][i];
                        float hy = nb[r].y, hy_zm = bprev[r].y, hy_xm = bn[1][j][i - 1];
                        float hz = nb[r].z, hz_ym = r > 0 ? nb[r - 1].z : bn[2][j - 1][i], hz_xm = bn[2][j][i - 1];
                        if (kRare && (f & kFImu)) {   // mu varies: 1/mu per face
                            const int gyr = gy[r];
                            const int km = k > 0 ? k - 1 : P.N[2] - 1;
                            const int xm = gx > 0 ? gx - 1 : P.N[0] - 1, ym = gyr > 0 ? gyr - 1 : P.N[1] - 1;
                            hz *= imu(P, 2, gx, gyr, k); hz_ym *= imu(P, 2, gx, ym, k); hz_xm *= imu(P, 2, xm, gyr, k);
                            hy *= imu(P, 1, gx, gyr, k); hy_zm *= imu(P, 1, gx, gyr, km); hy_xm *= imu(P, 1, xm, gyr, k);
                            hx *= imu(P, 0, gx, gyr, k); hx_zm *= imu(P, 0, gx, gyr, km); hx_ym *= imu(P, 0, gx, ym, k);
                        } else if (!P.uniform_mu) {   // one record: one mu
                            hz *= rec.w; hz_ym *= rec.w; hz_xm *= rec.w; hy *= rec.w; hy_zm *= rec.w;
                            hy_xm *= rec.w; hx *= rec.w; hx_zm *= rec.w; hx_ym *= rec.w;
                        }
                        const float dHz_y = hz - hz_ym, dHy_z = hy - hy_zm;
                        const float dHx_z = hx - hx_zm, dHz_x = hz - hz_xm;
                        const float dHy_x = hy - hy_xm, dHx_y = hx - hx_ym;
                        float cx = P.r[1] * dHz_y - P.r[2] * dHy_z;
                        float cy = P.r[2] * dHx_z - P.r[0] * dHz_x;
                        float cz = P.r[0] * dHy_x - P.r[1] * dHx_y;
                        // CPML memory: psi' = b psi + c d, added to the curl
                        float p0 = 0.f, p1 = 0.f;
                        if (sax == 0) {          // Ey, Ez
                            p0 = bE[r] * pe[r][0] + cE[r] * dHz_x;
                            p1 = bE[r] * pe[r][1] + cE[r] * dHy_x;
                            cy -= p0;
                            cz += p1;
                        } else if (sax == 1) {   // Ex, Ez
                            p0 = bE[r] * pe[r][0] + cE[r] * dHz_y;
                            p1 = bE[r] * pe[r][1] + cE[r] * dHx_y;
                            cx += p0;
                            cz -= p1;
                        } else if (sax == 2) {   // Ex, Ey
                            p0 = bE[r] * pe[r][0] + cE[r] * dHy_z;
                            p1 = bE[r] * pe[r][1] + cE[r] * dHx_z;
                            cx -= p0;
                            cy += p1;
                        }
                        if (insl[r]) {
                            if (sax == 0 ? uy : ux) P.psiE[pair_c1(sax)][sax][q] = p0;
                            if (sax == 2 ? uy : uz) P.psiE[pair_c2(sax)][sax][q] = p1;
                        }
                        if (kRare && sec) {
    #pragma unroll 1
                            for (int a = 0; a < 3; ++a) {
                                if (!((sec >> a) & 1u)) continue;
                                const int pos = a == 0 ? gx : a == 1 ? gy[r] : k;
                                if (!slab_pos(P, a, pos)) continue;
                                const float bb = __ldg(P.pbE[a] + pos), cc = __ldg(P.pcE[a] + pos);
                                float* q1 = P.psiE[pair_c1(a)][a] + q;
                                float* q2 = P.psiE[pair_c2(a)][a] + q;
                                const float o1 = *q1, o2 = *q2;
                                if (a == 0) {
                                    const float n1 = bb * o1 + cc * dHz_x, n2 = bb * o2 + cc * dHy_x;
                                    cy -= n1;
                                    cz += n2;
                                    if (uy) *q1 = n1;
                                    if (uz) *q2 = n2;
                                } else if (a == 1) {
                                    const float n1 = bb * o1 + cc * dHz_y, n2 = bb * o2 + cc * dHx_y;
                                    cx += n1;
                                    cz -= n2;
                                    if (ux) *q1 = n1;
                                    if (uz) *q2 = n2;
                                } else {
                                    const float n1 = bb * o1 + cc * dHy_z, n2 = bb * o2 + cc * dHx_z;
                                    cx -= n1;
                                    cy += n2;
                                    if (ux) *q1 = n1;
                                    if (uy) *q2 = n2;
                                }
                            }
                        }
                        float jt0 = 0.f, jt1 = 0.f, jt2 = 0.f;
                        if (mc[r][6] > 0.f && ux) {
                            jt0 = jo[r][0] + mc[r][6] * em0;
                            P.J[0][q] = jt0;
                        }
                        if (mc[r][7] > 0.f && uy) {
                            jt1 = jo[r][1] + mc[r][7] * em1;
                            P.J[1][q] = jt1;
                        }
                        if (mc[r][8] > 0.f && uz) {
                            jt2 = jo[r][2] + mc[r][8] * em2;
                            P.J[2][q] = jt2;
                        }
                        float n0 = mc[r][0] * em0 + mc[r][3] * (cx - jt0);
                        float n1 = mc[r][1] * em1 + mc[r][4] * (cy - jt1);
                        float n2 = mc[r][2] * em2 + mc[r][5] * (cz - jt2);
                        if (kRare && (f & kFSrc)) {
                            const int gyr = gy[r];
                            for (int s = 0; s < S.n; ++s) {
                                if (gx >= S.lo[s][0] && gx < S.hi[s][0] && gyr >= S.lo[s][1] && gyr < S.hi[s][1] &&
                                    k >= S.lo[s][2] && k < S.hi[s][2]) {
                                    if (S.comp[s] == 0) n0 += S.amp[s];
                                    if (S.comp[s] == 1) n1 += S.amp[s];
                                    if (S.comp[s] == 2) n2 += S.amp[s];
                                }
                            }
                        }
                        n0 = ux ? n0 : em0;
                        n1 = uy ? n1 : em1;
                        n2 = uz ? n2 : em2;
                        O.E[0][q] = n0;
                        O.E[1][q] = n1;
                        O.E[2][q] = n2;
                        if (!isfinite(n0 + n1 + n2)) atomicOr(P.status, kStatusNonFinite);
                        // first-order Mur on the z walls: E_w^{n+1} = E_i^n + M (E_i^{n+1} - E_w^n)
                        if (kRare && (f & (kFMurLo | kFMurHi))) {
                            const bool mx = hvx && iny[r], my = inx && hvy[r];
                            if (f & kFMurLo) {
                                if (mx) O.E[0][o[r]] = em0 + P.mur_M * (n0 - elo[r][0]);
                                if (my) O.E[1][o[r]] = em1 + P.mur_M * (n1 - elo[r][1]);
                            }
                            if (f & kFMurHi) {
                                const int pw = P.n[2] * PL + o[r];
                                if (mx) O.E[0][pw] = em0 + P.mur_M * (n0 - s1.e[0][j][i]);
                                if (my) O.E[1][pw] = em1 + P.mur_M * (n1 - s1.e[1][j][i]);
                            }
                        }
                    }
                    if (kRare && zlo) {
                        elo[r][0] = s0.e[0][j][i];
                        elo[r][1] = s0.e[1][j][i];
                    }
                    bprev[r] = nb[r];
                }
            }
        };
        if (item_is_rare(P, S, mur, t))
            planes(std::true_type{});
        else
            planes(std::false_type{});
        if (aborted) break;
        seq0 += nq;
        // this item is done: its slot takes the item after the next one
        if (nq == 2) rec_store(s_item[cur ^ 1], cur ^ 1, rnext);   // a one-plane item: no plane 1
        if (tid == 0) {
            s_item[cur] = pend;
            ++c_ord;
        }
        if (nq == 2) __syncthreads();
        cur ^= 1;
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

size_t step_smem_bytes() { return 128 + kStages * sizeof(StageBuf) + 2 * kBPlaneBytes + kStages * 8; }

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

cudaError_t launch_step(const void* tmaps, const Params& P, const StepOut& O, const Sources& S, int blocks,
                        cudaStream_t st) {
    static cudaError_t attr = step_smem_attribute();
    if (attr != cudaSuccess) return attr;
    const TMaps* tm = (const TMaps*)tmaps;
    k_step<<<blocks, dim3(kTX, kThreadsY), step_smem_bytes(), st>>>(*tm, P, O, S);
    return cudaGetLastError();
}

// order of the work items of a launch: a stable partition that puts the items
// needing the full plane loop (the slow ones) first, so that the last items
// handed out are short.  One CTA.
__global__ void __launch_bounds__(1024) k_item_order(Params P, StepOut O, Sources S, int* order) {
    __shared__ int sc[1024];
    const int n = O.ntx * O.nty * O.nch;
    const int per = (n + 1023) / 1024;
    const int a = min((int)threadIdx.x * per, n), b = min(a + per, n);
    const bool mur = P.bc[2] == TF_BC_MUR;
    int cnt = 0;
    for (int d = a; d < b; ++d) cnt += item_is_rare(P, S, mur, tile_of(P, O, d)) ? 1 : 0;
    sc[threadIdx.x] = cnt;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int v = (int)threadIdx.x >= off ? sc[threadIdx.x - off] : 0;
        __syncthreads();
        sc[threadIdx.x] += v;
        __syncthreads();
    }
    const int total = sc[1023];
    int r = sc[threadIdx.x] - cnt;   // rare items before this thread's range
    int c = total + (a - r);         // position of its first common item
    for (int d = a; d < b; ++d) {
        if (item_is_rare(P, S, mur, tile_of(P, O, d)))
            order[r++] = d;
        else
            order[c++] = d;
    }
}

cudaError_t launch_item_order(const Params& P, const StepOut& O, const Sources& S, int* order, cudaStream_t st) {
    k_item_order<<<1, 1024, 0, st>>>(P, O, S, order);
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
