// tf_step.cu -- fused single-pass step of the two-fluid Yee scheme (sm_103a).
//
// One launch advances the whole grid by one step of Algorithm 1 (arXiv
// 2305.13419, Sec. 3) in its fused leapfrog form:
//   Bt^{n+1/2} = Bt^{n-1/2} - curl(E^n)                   (steps 5 + 1, CPML psi_B)
//   Jt^{n+1/2} = Jt^{n-1/2} + kt_e E^n                     (steps 4 + 2)
//   E^{n+1}    = ca E^n + cb (curl(Bt/mu) - Jt^{n+1/2})     (step 3, CPML psi_E)
// plus soft sources, first-order Mur z walls and the non-finite watchdog.
//
// Work layout.  A CTA of 32 x 8 threads owns a 32 x 16 column tile -- each
// thread an x-adjacent pair of points of one row -- and streams it along z
// through a chunk of planes.  Each plane's E^n, B^{n-1/2} and -- where a CPML
// slab reaches the tile-plane -- the CPML memory psi_B of one slab axis
// arrive in shared memory by TMA (cp.async.bulk.tensor) boxes covering the
// tile plus its halo, through a ring of kStages buffers whose mbarriers
// complete on the transferred byte count.  Lane 0 of the last warp keeps the
// ring full and runs ahead into the next work item, so the stream of planes
// has no gap between items.  Per plane:
//   B phase  every thread forms B^{n+1/2} at its pair; warp 0 also forms the
//            y0-1 row and the x0-1 column of B that the E update needs from
//            the neighbouring tiles; the plane of new B goes to one of two
//            shared buffers, owned values to the new B array;
//   barrier  (the only one per plane; it also frees the stage of the plane
//            before, which the producer then refills);
//   E phase  every thread forms Js^{n+1/2} and E^{n+1} at its pair from the
//            shared B plane and the previous plane's B kept in registers.
// A pair lives in 64-bit registers and moves with 64-bit shared / global
// accesses; its arithmetic uses the packed FP32x2 add / sub / mul / fma of
// the sm_100 family.  E, B, Js and psi_B go from one buffer to another (the
// other tiles only ever read the old ones); psi_E is owned by one thread and
// updates in place.  Work items (tile, z chunk) are handed out through an
// order that puts the slow items first, the others z chunk by z chunk and
// the last ones in short pieces; each CTA starts with two items by position
// and draws the rest from an atomic counter; the grid fills every SM twice.
// The CPML profile coefficients of an item sit in a shared table filled one
// item ahead.  The first CTAs also add E^n at the probe points to the
// running DFTs while their ring fills.  Periodic x / y seams, which a TMA
// box cannot wrap, are patched from global memory after the box lands.
//
// x / y walls are per-point masks, the low z wall a plane mask; the CPML
// memory of the staged axis comes from shared memory, that of any further
// slab axis from global memory; a tile-plane whose cells are all alike uses
// one precomputed {ca, cb, cj, 1/mu} record, the others per-point
// coefficients set with the materials.  The plane body is compiled three
// times: work items that meet a source, a Mur plane or varying mu take the
// full body, items whose planes meet a second CPML axis (and nothing else
// of those) a body with the further CPML axes only, all others a body
// without that code.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <string.h>

#include <type_traits>

#include "tf_device.cuh"
#include "tf_internal.cuh"

namespace tf {

namespace {

using namespace dev;

struct __align__(128) StageBuf {
    alignas(128) float e[3][kEY][kEX];    // E^n, tile + halo
    alignas(128) float b[3][kBY][kBX];    // B^{n-1/2}, tile + low halo
    alignas(128) float pb[2][kBY][kBX];   // old psi_B of the staged slab axis, tile + low halo
};
constexpr unsigned kEBytes = 3u * kEY * kEX * 4, kBBytes = 3u * kBY * kBX * 4, kPBBytes = 2u * kBY * kBX * 4;
constexpr int kThreadsY = kTY / kRows;
constexpr int kThreads = kTX * kThreadsY;
constexpr int kProd = kTX * (kThreadsY - 1);   // the producer: lane 0 of the last warp (warp 0 forms the halo)
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
__device__ __forceinline__ Tile tile_of(const Params& P, const StepOut& O, long long item) {
    Tile t;
    const int tile = item_tile(item);
    t.bx = tile % O.ntx;
    t.by = tile / O.ntx;
    t.x0 = t.bx * kSX;
    t.y0 = t.by * kSY;
    t.kz0 = item_kz0(item);
    t.kz1 = t.kz0 + item_len(item);
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

struct P3 {
    f2 x, y, z;
};

// bring the line holding p into L1 (no register, no wait)
__device__ __forceinline__ void prefetch_l1(const float* p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// update masks of a pair of points (gx0, gx0 + 1) on row gy: per point p, bits
// 6p + {0, 1, 2} for Bx, By, Bz and 6p + {3, 4, 5} for Ex, Ey, Ez (x / y walls)
__device__ __forceinline__ unsigned masks_of(const Params& P, int gx0, int gy) {
    const bool hvy = P.per[1] || gy < P.n[1], iny = P.per[1] || (gy >= 1 && gy <= P.n[1] - 1);
    unsigned m = 0;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int gx = gx0 + p;
        const bool hvx = P.per[0] || gx < P.n[0], inx = P.per[0] || (gx >= 1 && gx <= P.n[0] - 1);
        const unsigned b = (unsigned)(inx && hvy) | (unsigned)(hvx && iny) << 1 | (unsigned)(hvx && hvy) << 2 |
                           (unsigned)(hvx && iny) << 3 | (unsigned)(inx && hvy) << 4 | (unsigned)(inx && iny) << 5;
        m |= b << (6 * p);
    }
    return m;
}
// bits cleared on the low z wall plane: Bz, Ex, Ey of both points
constexpr unsigned kMaskZlo = (1u << 2 | 1u << 3 | 1u << 4) * 65u;
// the two point bits (low, high) of mask bit `b`
__device__ __forceinline__ unsigned mbits(unsigned m, int b) { return (m >> b & 1u) | (m >> (b + 5) & 2u); }
// B^{n+1/2} before masking at the pair of box positions (j, i0), (j, i0 + 1)
// of landed stages s0 (plane k) and s1 (plane k + 1): the curl update plus the
// CPML memory of the staged axis sax (coefficients bB, cB; zero outside the
// slab), whose new values come back in p0, p1 (pair order)
__device__ __forceinline__ P3 b_pair(const Params& P, const StageBuf& s0, const StageBuf& s1, int j, int i0, int sax,
                                     f2 bB, f2 cB, f2& p0, f2& p1) {
    const f2 ex = ld2(&s0.e[0][j][i0]), ey = ld2(&s0.e[1][j][i0]), ez = ld2(&s0.e[2][j][i0]);
    const f2 dEz_y = sub2(ld2(&s0.e[2][j + 1][i0]), ez), dEx_y = sub2(ld2(&s0.e[0][j + 1][i0]), ex);
    const f2 dEy_z = sub2(ld2(&s1.e[1][j][i0]), ey), dEx_z = sub2(ld2(&s1.e[0][j][i0]), ex);
    const f2 dEz_x = sub2(pk(hi(ez), s0.e[2][j][i0 + 2]), ez), dEy_x = sub2(pk(hi(ey), s0.e[1][j][i0 + 2]), ey);
    const f2 r0 = pk(P.r[0], P.r[0]), r1 = pk(P.r[1], P.r[1]), r2 = pk(P.r[2], P.r[2]);
    P3 b;
    // Bx - (r1 dEz/dy - r2 dEy/dz), By - (r2 dEx/dz - r0 dEz/dx), Bz - (r0 dEy/dx - r1 dEx/dy)
    b.x = fma2(r2, dEy_z, sub2(ld2(&s0.b[0][j][i0]), mul2(r1, dEz_y)));
    b.y = fma2(r0, dEz_x, sub2(ld2(&s0.b[1][j][i0]), mul2(r2, dEx_z)));
    b.z = fma2(r1, dEx_y, sub2(ld2(&s0.b[2][j][i0]), mul2(r0, dEy_x)));
    p0 = 0;
    p1 = 0;
    if (sax == 0) {          // By, Bz
        p0 = fma2(bB, ld2(&s0.pb[0][j][i0]), mul2(cB, dEz_x));
        p1 = fma2(bB, ld2(&s0.pb[1][j][i0]), mul2(cB, dEy_x));
        b.y = add2(b.y, p0);
        b.z = sub2(b.z, p1);
    } else if (sax == 1) {   // Bx, Bz
        p0 = fma2(bB, ld2(&s0.pb[0][j][i0]), mul2(cB, dEz_y));
        p1 = fma2(bB, ld2(&s0.pb[1][j][i0]), mul2(cB, dEx_y));
        b.x = sub2(b.x, p0);
        b.z = add2(b.z, p1);
    } else if (sax == 2) {   // Bx, By
        p0 = fma2(bB, ld2(&s0.pb[0][j][i0]), mul2(cB, dEy_z));
        p1 = fma2(bB, ld2(&s0.pb[1][j][i0]), mul2(cB, dEx_z));
        b.x = add2(b.x, p0);
        b.y = sub2(b.y, p1);
    }
    return b;
}

// differences of E along axis a that feed the CPML pair (c1, c2) of that axis,
// for the pair of box positions (j, i0), (j, i0 + 1)
__device__ __forceinline__ void e_diffs2(const StageBuf& s0, const StageBuf& s1, int j, int i0, int a, f2& d0, f2& d1) {
    if (a == 0) {
        const f2 ez = ld2(&s0.e[2][j][i0]), ey = ld2(&s0.e[1][j][i0]);
        d0 = sub2(pk(hi(ez), s0.e[2][j][i0 + 2]), ez);
        d1 = sub2(pk(hi(ey), s0.e[1][j][i0 + 2]), ey);
    } else if (a == 1) {
        d0 = sub2(ld2(&s0.e[2][j + 1][i0]), ld2(&s0.e[2][j][i0]));
        d1 = sub2(ld2(&s0.e[0][j + 1][i0]), ld2(&s0.e[0][j][i0]));
    } else {
        d0 = sub2(ld2(&s1.e[1][j][i0]), ld2(&s0.e[1][j][i0]));
        d1 = sub2(ld2(&s1.e[0][j][i0]), ld2(&s0.e[0][j][i0]));
    }
}
// add the new CPML memory pair (n0, n1) of axis a to B with the curl's signs
__device__ __forceinline__ void b_add_psi(int a, f2 n0, f2 n1, P3& b) {
    if (a == 0) {
        b.y = add2(b.y, n0);
        b.z = sub2(b.z, n1);
    } else if (a == 1) {
        b.x = sub2(b.x, n0);
        b.z = add2(b.z, n1);
    } else {
        b.x = add2(b.x, n0);
        b.y = sub2(b.y, n1);
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

// the plane loop an item runs: 2 (the full one) with varying mu, a source
// plane or a Mur plane; else 1 (further CPML axes only) with a second CPML
// axis on one of its planes; else 0
__device__ __forceinline__ int item_kind(const Params& P, const Sources& S, bool mur, const Tile& t) {
    if (!P.uniform_mu) return 2;
    const int ka = t.ks < 0 ? 0 : t.ks, kb = t.kz1 - 1;   // planes of the item (periodic wrap: z has no slab)
    int sk0, sk1;
    src_range(S, t, sk0, sk1);
    if (sk1 > sk0 && ((kb >= sk0 && ka < sk1) || (t.ks < 0 && P.N[2] - 1 >= sk0 && P.N[2] - 1 < sk1))) return 2;
    if (mur && ((ka <= 1 && 1 <= kb) || (ka <= P.n[2] - 1 && P.n[2] - 1 <= kb))) return 2;
    const bool sx = P.L[0] > 0 && (t.x0 - 1 < P.L[0] || t.x0 + kSX - 1 >= P.n[0] - P.L[0]);
    const bool sy = P.L[1] > 0 && (t.y0 - 1 < P.L[1] || t.y0 + kSY - 1 >= P.n[1] - P.L[1]);
    const bool sz = P.L[2] > 0 && (ka < P.L[2] || kb >= P.n[2] - P.L[2]);
    return (int)sx + (int)sy + (int)sz >= 2 ? 1 : 0;
}

}  // namespace

// batched launches: the arguments of a work item's grid as the plane loop
// reads them, staged in shared memory
struct ItemArgs {
    Params P;
    StepOut O;
    Sources S;
    const float* amp;
};
// copy `n` bytes (a multiple of 4) with every thread of the CTA
__device__ __forceinline__ void cta_copy(void* dst, const void* src, int n, int tid, int nth) {
    const unsigned* s = reinterpret_cast<const unsigned*>(src);
    unsigned* d = reinterpret_cast<unsigned*>(dst);
    for (int i = tid; i < n / 4; i += nth) d[i] = __ldg(s + i);
}

// the arguments of the grid a work item belongs to
struct GridRef {
    const TMaps* tm;
    const Params* P;
    const StepOut* O;
    const Sources* S;
    const Probes* R;
    const float* amp;   // batched: this grid's amplitude table ([step][source])
    long long level;
};

// kBatch = false: one grid, its arguments by value.  kBatch = true: one step
// of a batch of grids (tf_batch_run): the work items of every grid form one
// list (the grid's index in descriptor bits 48-62), each item runs with its
// grid's arguments from global memory, and the step number is read from the
// device (so that a captured launch can be replayed).
template <bool kBatch>
__global__ void __launch_bounds__(kThreads, 2)
    k_step_t(const __grid_constant__ TMaps tmk, const __grid_constant__ Params Pk, const __grid_constant__ StepOut Ok,
             const __grid_constant__ Sources Sk, const __grid_constant__ Probes Rk, long long levelk,
             const __grid_constant__ BatchLaunch BL) {
    const int step = kBatch ? __ldg(BL.step) : 0;
    const int par = step & 1;
    auto gridref = [&](long long item) -> GridRef {
        if constexpr (kBatch) {
            const BatchGrid& A = BL.G[(unsigned long long)item >> 48];
            return {&A.tm, &A.P[par], &A.O[par], &A.S, &A.R, A.amp, A.level0 + step};
        } else {
            return {&tmk, &Pk, &Ok, &Sk, &Rk, nullptr, levelk};
        }
    };
    const long long* order = kBatch ? BL.order : Ok.order;
    const int nitems = kBatch ? BL.nitems : Ok.nitems;
    unsigned long long* const ctr = kBatch ? BL.ctr : Ok.ctr;
    const unsigned long long obase = kBatch ? BL.base0 + (unsigned long long)step * BL.base_inc : Ok.base;
    const int gdim = (int)gridDim.x;
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    // TMA destinations must be 128-byte aligned: round the base up (128 spare bytes are allocated)
    unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    StageBuf* stg = reinterpret_cast<StageBuf*>(smem_raw);
    float(*bplanes)[3][kBY][kBX] = reinterpret_cast<float(*)[3][kBY][kBX]>(smem_raw + kStages * sizeof(StageBuf));
    unsigned long long* bar =
        reinterpret_cast<unsigned long long*>(smem_raw + kStages * sizeof(StageBuf) + 2 * kBPlaneBytes);
    __shared__ long long s_item[2];             // current and next work item (-1: none)
    __shared__ float4 s_rec[2][kItemMax + 2];     // material record of each plane of the two items
    __shared__ unsigned s_flag[2][kItemMax + 2];  // plane flags
    // CPML coefficients of the two items (zero outside the slabs): per profile
    // (b_B, c_B, b_E, c_E) the tile's columns x0-4 .. x0+31, rows y0-1 ..
    // y0+15 and the item's planes
    __shared__ __align__(16) float s_cf[2][4][kCfN];
    // batched: the grid arguments of the current and the next item (slot as s_item)
    __shared__ __align__(16) unsigned char s_args_raw[kBatch ? 2 * sizeof(ItemArgs) : 16];
    ItemArgs* s_args = reinterpret_cast<ItemArgs*>(s_args_raw);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTX + tx;
    // stage the grid arguments of `item` in slot `slot` (every thread; visible after the next barrier)
    auto stage_args = [&](long long item, int slot) {
        if constexpr (kBatch) {
            if (item < 0) return;
            const BatchGrid& A = BL.G[(unsigned long long)item >> 48];
            ItemArgs& D = s_args[slot];
            cta_copy(&D.P, &A.P[par], (int)sizeof(Params), tid, kThreads);
            cta_copy(&D.O, &A.O[par], (int)sizeof(StepOut), tid, kThreads);
            cta_copy(&D.S, &A.S, (int)sizeof(Sources), tid, kThreads);
            if (tid == 0) D.amp = A.amp;
        }
    };

    // Items 0 .. 2G - 1 (G CTAs) are handed out without the counter: CTA b
    // starts with items b and G + b.  The others come from the counter.
    // producer: a ticket from the counter, and later the work item it names
    // (or -1); the two halves are a plane apart, so that the counter's round
    // trip does not hold up the producer's warp
    auto ticket = [&]() -> unsigned long long { return atomicAdd(ctr, 1ull); };
    auto item_of = [&](unsigned long long tk) -> long long {
        const long long d = (long long)(tk - obase) + 2LL * gdim;
        return (d >= 0 && d < nitems) ? __ldg(order + d) : -1LL;
    };
    // the records of an item: loaded by threads < nq - 1 ...
    // (entry u of the coefficient table: profile u / kCfN, entry u % kCfN)
    auto cf_entry = [&](const Params& P, const Tile& t, int u) -> float {
        const int pr = u / kCfN, e = u % kCfN;
        int a = -1, pos = 0;
        if (e < kCfY) {
            a = 0;
            pos = t.x0 - 4 + e;
        } else if (e < kCfZ) {
            a = 1;
            pos = t.y0 - 1 + (e - kCfY);
        } else if (e - kCfZ < t.nq - 1) {
            a = 2;
            pos = plane_of(P, t, e - kCfZ);
        }
        if (a < 0 || !slab_pos(P, a, pos)) return 0.f;
        const float* pf = pr == 0 ? P.pbB[a] : pr == 1 ? P.pcB[a] : pr == 2 ? P.pbE[a] : P.pcE[a];
        return __ldg(pf + pos);
    };
    auto rec_load = [&](long long item, float4& r, float& cf) {
        if (item < 0) return;
        const GridRef g = gridref(item);
        const Params& P = *g.P;
        const StepOut& O = *g.O;
        const Tile t = tile_of(P, O, item);
        if (tid < t.nq - 1) r = __ldg(O.tilemat + (long long)(t.by * O.ntx + t.bx) * P.N[2] + plane_of(P, t, tid));
        // one coefficient table entry per thread; the second warp's threads,
        // which load no record, carry one more in r.x
        cf = cf_entry(P, t, tid);
        if (tid >= 32 && tid < 32 + kCfExtra) r.x = cf_entry(P, t, kThreads + tid - 32);
    };
    // ... and stored with the plane flags
    auto rec_store = [&](long long item, int slot, const float4& r, float cf) {
        if (item < 0) return;
        (&s_cf[slot][0][0])[tid] = cf;
        if (tid >= 32 && tid < 32 + kCfExtra) (&s_cf[slot][0][0])[kThreads + tid - 32] = r.x;
        const GridRef g = gridref(item);
        const Params& P = *g.P;
        const StepOut& O = *g.O;
        const Sources& S = *g.S;
        const bool mur = P.bc[2] == TF_BC_MUR;
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

    // ---------------------------------------------- producer (thread kProd only)
    // Items are numbered in the order this CTA takes them; item m lives in
    // slot m & 1, and the slot is refilled with item m + 2 once item m is done.
    // The producer may therefore run at most one item ahead of the consumer.
    unsigned long long issued = 0, consumed = 0;   // planes through the ring
    int p_ord = 0, p_q = 0;                        // producer: item ordinal, next plane
    int c_ord = 0;                                 // consumer: item ordinal
    Tile p_t;                                      // producer: tile of item p_ord
    p_t.nq = 0;
    long long p_item = -1;                         // producer: item p_ord
    bool p_have = false;
    // the arguments the producer reads for item ordinal `ord`: batched, the
    // staged copy of its slot (usable once a barrier has passed since the
    // copy), else the launch's own
    auto prod_P = [&](int ord) -> const Params& {
        if constexpr (kBatch) return s_args[ord & 1].P;
        else return Pk;
    };
    auto prod_O = [&](int ord) -> const StepOut& {
        if constexpr (kBatch) return s_args[ord & 1].O;
        else return Ok;
    };
    // stages that threads wrote with ordinary stores (periodic seam patches):
    // a proxy fence orders those writes before the stage's next TMA copy
    unsigned p_dirty = 0;
    auto issue = [&](const Tile& t, int q, unsigned long long seq) {
        const Params& P = prod_P(p_ord);
        const StepOut& O = prod_O(p_ord);
        const TMaps& tm = kBatch ? BL.G[(unsigned long long)p_item >> 48].tm : tmk;
        const int s = (int)(seq % kStages);
        const int k = plane_of(P, t, q);
        const int sax = slab_axis(slab_bits(P, t, k));
        const unsigned bytes = kEBytes + kBBytes + (sax >= 0 ? kPBBytes : 0u);
        if ((p_dirty >> s) & 1u) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            p_dirty &= ~(1u << s);
        }
        mbar_expect_tx(&bar[s], bytes);
        tma_load_box(&stg[s].e[0][0][0], &tm.e, t.x0 - 4, t.y0 - 1, k, O.ecur, &bar[s]);
        tma_load_box(&stg[s].b[0][0][0], &tm.b, t.x0 - 4, t.y0 - 1, k, O.bcur, &bar[s]);
        if (sax >= 0)
            tma_load_box(&stg[s].pb[0][0][0], &tm.pb, t.x0 - 4, t.y0 - 1, k,
                         kPsiGroup * O.psi_slot[sax] + O.psib_cur, &bar[s]);
    };
    // keep kStages planes in flight, crossing into the next item; batched,
    // the item after the consumer's only once its staged arguments are
    // visible (`next_visible`: a barrier has passed since they were copied)
    auto pump = [&](bool next_visible) {
        while (issued < consumed + kStages) {
            if (!p_have) {
                const long long item = s_item[p_ord & 1];
                if (item < 0) return;
                p_t = tile_of(prod_P(p_ord), prod_O(p_ord), item);
                p_item = item;
                p_have = true;
            }
            if (p_q >= p_t.nq) {
                if (p_ord > c_ord) return;   // the next slot still holds the current item
                if (kBatch && p_ord == c_ord && !next_visible) return;
                const long long item = s_item[(p_ord + 1) & 1];
                if (item < 0) return;
                ++p_ord;
                p_q = 0;
                p_t = tile_of(prod_P(p_ord), prod_O(p_ord), item);
                p_item = item;
            }
            issue(p_t, p_q, issued);
            ++p_q;
            ++issued;
        }
    };

    if (tid == kProd) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if constexpr (kBatch) {
            // the grids' tensor maps sit in global memory that the host rewrites
            // between runs: order those writes before the tensor-map proxy reads them
            for (int gi = 0; gi < BL.ngrids; ++gi) {
                const TMaps* m = &BL.G[gi].tm;
                asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(&m->e) : "memory");
                asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(&m->b) : "memory");
                asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(&m->pb) : "memory");
            }
        }
        const int b = (int)blockIdx.x, g = gdim;
        s_item[0] = b < nitems ? __ldg(order + b) : -1LL;
        s_item[1] = (s_item[0] >= 0 && g + b < nitems) ? __ldg(order + g + b) : -1LL;
    }
    __syncthreads();
    {
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
        float f0 = 0.f, f1 = 0.f;
        rec_load(s_item[0], r0, f0);
        rec_load(s_item[1], r1, f1);
        rec_store(s_item[0], 0, r0, f0);
        rec_store(s_item[1], 1, r1, f1);
        stage_args(s_item[0], 0);
        stage_args(s_item[1], 1);
    }
    if constexpr (kBatch) __syncthreads();   // the staged arguments, for the producer
    if (tid == kProd) pump(true);
    __syncthreads();
    // while the ring fills: E^n at the probe points into their DFTs, a probe per CTA
    if (tid < TF_MAX_FREQS)
        if constexpr (kBatch) {
            for (int pr = blockIdx.x; pr < BL.nprobes; pr += gdim) {   // (grid, probe) pairs of the batch
                const BatchGrid& A = BL.G[BL.probes[2 * pr]];
                probe_update(A.P[par].E, A.R, BL.probes[2 * pr + 1], tid, A.level0 + step);
            }
        } else {
            for (int pr = blockIdx.x; pr < Rk.n; pr += gdim) probe_update(Pk.E, Rk, pr, tid, levelk);
        }

    int cur = 0;
    bool aborted = false;
    unsigned long long seq0 = 0;   // ring sequence number of plane 0 of the current item
    unsigned it = 0;               // planes done by this CTA (selects the shared B plane)
    long long pend = -1;           // producer: the item after the next one
    unsigned long long ptk = 0;    // producer: its ticket
    bool phas = false;             // producer: a ticket was drawn for it
    unsigned* status = kBatch ? nullptr : Pk.status;   // the current item's grid's status word
    while (true) {
        const long long item = s_item[cur];
        if (item < 0) break;
        // batched: planes of this item that the producer could not issue
        // before its arguments were visible (items shorter than the ring)
        if (kBatch && tid == kProd) pump(false);
        const ItemArgs& IA = s_args[cur];
        const Params& P = kBatch ? IA.P : Pk;
        const StepOut& O = kBatch ? IA.O : Ok;
        const Sources& S = kBatch ? IA.S : Sk;
        const int PL = (int)P.plane;
        const bool mur = P.bc[2] == TF_BC_MUR;
        status = P.status;
        auto amp_of = [&](int s) -> float {
            if constexpr (kBatch) return __ldg(IA.amp + (long long)step * S.n + s);
            else return S.amp[s];
        };
        const Tile t = tile_of(P, O, item);
        const int x0 = t.x0, y0 = t.y0, kz0 = t.kz0, nq = t.nq;

        // ------------------------------------------------------- columns
        // thread: tile row `row`, x pair (gx0, gx0 + 1).  Warp 0 also forms the
        // halo: lanes 0..15 the row y0 - 1 (in pairs), lanes 16..31 the column
        // x0 - 1 of rows y0 .. y0 + 15 (as the pair x0 - 2, x0 - 1)
        const int row = 2 * ty + (tx >> 4), xi = tx & 15;
        const int gx0 = x0 + 2 * xi, gy = y0 + row;
        const int j = row + 1, i0 = 2 * xi + 4;   // position in the E / B boxes
        const bool v0 = gx0 < P.N[0] && gy < P.N[1], v1 = gx0 + 1 < P.N[0] && gy < P.N[1];
        const int o = v0 ? gy * P.pitch + gx0 : 0;
        const unsigned m = masks_of(P, gx0, gy);
        const bool hal = ty == 0, hrow = tx < 16;
        const int hj = hrow ? 0 : tx - 15, hi0 = hrow ? 2 * tx + 4 : 2;
        const int hgx0 = x0 - 4 + hi0, hgy = y0 - 1 + hj;
        const unsigned hm = masks_of(P, hgx0, hgy);
        // no x / y wall reaches the tile or its halo: masks only on the low z wall plane
        const bool open = (P.per[0] || (x0 - 2 >= 1 && x0 + kSX - 1 <= P.n[0] - 1)) &&
                          (P.per[1] || (y0 - 1 >= 1 && y0 + kSY - 1 <= P.n[1] - 1));
        // periodic seams that the TMA box cannot wrap
        const bool seam = (P.per[0] && (x0 - 4 < 0 || x0 + kEX - 4 > P.N[0])) ||
                          (P.per[1] && (y0 - 1 < 0 || y0 + kEY - 1 > P.N[1]));
        // box entries a valid point or the halo reads: columns x0-2 .. x0+kTX,
        // rows y0-1 .. y0+kTY, each clipped to one past the grid's last point
        const int pw = min(kEX - 1, min(x0 + kTX, P.N[0]) - (x0 - 4)) - 1;
        const int ph = min(kEY - 1, min(y0 + kTY, P.N[1]) - (y0 - 1)) + 1;
        auto patch = [&](StageBuf& sb, int k, int sax) {
            for (int u = tid; u < pw * ph; u += kThreads) {
                const int jj = u / pw, ii = 2 + u % pw;
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
        float cfnext = 0.f;                                 // and this thread's coefficient entry
        f2 bpx = 0, bpy = 0;     // B^{n+1/2}(k-1) at the own pair (z differences)
        f2 elo0 = 0, elo1 = 0;   // E^n on the low Mur wall
        // one plane, compiled for the three item kinds (item_kind): the full
        // version (sources, Mur planes, varying mu, further CPML axes), the
        // further CPML axes only, and neither
        auto plane = [&](auto kind_tag, int qq) -> bool {   // false: a copy never landed
            constexpr int kKind = decltype(kind_tag)::value;
            constexpr bool kSecOn = kKind >= 1, kFull = kKind == 2;
            const int k = plane_of(P, t, qq);
            const bool doE = t.ks + qq >= kz0;   // E update (and B store) at this plane
            const unsigned long long g0 = seq0 + qq, g1 = g0 + 1;
            StageBuf& s0 = stg[g0 % kStages];
            StageBuf& s1 = stg[g1 % kStages];
            const unsigned f = s_flag[cur][qq];
            const float4 rec = s_rec[cur][qq];
            const int sax = (int)((f >> kFSaxShift) & 3u) - 1;
            const bool coef = (f & kFCoef) != 0, zlo = (f & kFZlo) != 0;
            const unsigned sec = kSecOn ? (f / kFSec0) & 7u : 0u;
            const bool masked = !open || zlo;
            const unsigned mk = zlo ? m & ~kMaskZlo : m, hmk = zlo ? hm & ~kMaskZlo : hm;
            float(*bn)[kBY][kBX] = bplanes[it & 1];
            const int kq = k * PL, q = kq + o;
            const bool own = v0 && doE;
            const bool sc = coef || rec.z > 0.f;   // Js advances somewhere on the plane
            // global reads that do not depend on the stage: issued before the wait
            f2 jo0 = 0, jo1 = 0, jo2 = 0;
            if (own && sc) {
                jo0 = ld2(P.J[0] + q);
                jo1 = ld2(P.J[1] + q);
                jo2 = ld2(P.J[2] + q);
            }
            f2 ca0, ca1, ca2, cb0, cb1, cb2, cj0, cj1, cj2;
            if (own && coef) {
                ca0 = ld2(P.ca[0] + q);
                ca1 = ld2(P.ca[1] + q);
                ca2 = ld2(P.ca[2] + q);
                cb0 = ld2(P.cb[0] + q);
                cb1 = ld2(P.cb[1] + q);
                cb2 = ld2(P.cb[2] + q);
                cj0 = ld2(P.cj[0] + q);
                cj1 = ld2(P.cj[1] + q);
                cj2 = ld2(P.cj[2] + q);
            } else {
                ca0 = ca1 = ca2 = pk(rec.x, rec.x);
                cb0 = cb1 = cb2 = pk(rec.y, rec.y);
                cj0 = cj1 = cj2 = pk(rec.z, rec.z);
            }
            // CPML memory of the staged axis: coefficients (zero outside the slab), old psi_E
            f2 bB = 0, cB = 0, bE = 0, cE = 0, pe0 = 0, pe1 = 0, hbB = 0, hcB = 0;
            unsigned sl = 0;   // bit p: point p inside the slab
            if (sax >= 0) {
                const int pos0 = sax == 0 ? gx0 : sax == 1 ? gy : k, pos1 = sax == 0 ? gx0 + 1 : pos0;
                sl = (slab_pos(P, sax, pos0) ? 1u : 0u) | (slab_pos(P, sax, pos1) ? 2u : 0u);
                const float(*cf)[kCfN] = s_cf[cur];
                if (sax == 0) {
                    bB = ld2(&cf[0][i0]);
                    cB = ld2(&cf[1][i0]);
                    bE = ld2(&cf[2][i0]);
                    cE = ld2(&cf[3][i0]);
                } else {
                    const int e = sax == 1 ? kCfY + j : kCfZ + qq;
                    bB = pk(cf[0][e], cf[0][e]);
                    cB = pk(cf[1][e], cf[1][e]);
                    bE = pk(cf[2][e], cf[2][e]);
                    cE = pk(cf[3][e], cf[3][e]);
                }
                if (own && sl) {
                    pe0 = ld2(P.psiE[pair_c1(sax)][sax] + q);
                    pe1 = ld2(P.psiE[pair_c2(sax)][sax] + q);
                }
                if (hal) {
                    if (sax == 0) {
                        hbB = ld2(&cf[0][hi0]);
                        hcB = ld2(&cf[1][hi0]);
                    } else {
                        const int e = sax == 1 ? kCfY + hj : kCfZ + qq;
                        hbB = pk(cf[0][e], cf[0][e]);
                        hcB = pk(cf[1][e], cf[1][e]);
                    }
                }
            }
            f2 ho0 = 0, ho1 = 0, ho2 = 0, ho3 = 0;   // halo: old memories of the first two further axes
            unsigned hin = 0;                        // halo: bits 2a, 2a + 1: point inside the slab of axis a
            if (kSecOn && sec) {   // CPML memories of the further slab axes: into L1 while the stage lands
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (!((sec >> a) & 1u)) continue;
                    if (v0) {
                        prefetch_l1(P.psiB[pair_c1(a)][a] + q);
                        prefetch_l1(P.psiB[pair_c2(a)][a] + q);
                        prefetch_l1(P.psiE[pair_c1(a)][a] + q);
                        prefetch_l1(P.psiE[pair_c2(a)][a] + q);
                    }
                }
                if (hal) {   // halo: old memories of the further axes into registers while the stage lands
                    const int xw0 = wrap_or_out(P, 0, hgx0), xw1 = wrap_or_out(P, 0, hgx0 + 1);
                    const int yw = wrap_or_out(P, 1, hgy);
                    const int qh = kq + (yw >= 0 ? yw : 0) * P.pitch;
                    int n = 0;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        if (!((sec >> a) & 1u)) continue;
                        const bool in0 = yw >= 0 && xw0 >= 0 && slab_pos(P, a, a == 0 ? xw0 : a == 1 ? yw : k);
                        const bool in1 = yw >= 0 && xw1 >= 0 && slab_pos(P, a, a == 0 ? xw1 : a == 1 ? yw : k);
                        hin |= ((in0 ? 1u : 0u) | (in1 ? 2u : 0u)) << (2 * a);
                        const float* w1 = P.psiB[pair_c1(a)][a];
                        const float* w2 = P.psiB[pair_c2(a)][a];
                        const f2 o1 = pk(in0 ? w1[qh + xw0] : 0.f, in1 ? w1[qh + xw1] : 0.f);
                        const f2 o2 = pk(in0 ? w2[qh + xw0] : 0.f, in1 ? w2[qh + xw1] : 0.f);
                        if (n == 0) {
                            ho0 = o1;
                            ho1 = o2;
                        } else {
                            ho2 = o1;
                            ho3 = o2;
                        }
                        ++n;
                    }
                }
            }
            bool ok = mbar_wait(&bar[g1 % kStages], (unsigned)((g1 / kStages) & 1), P.wait_polls);
            if (qq == 0) ok = ok && mbar_wait(&bar[g0 % kStages], (unsigned)((g0 / kStages) & 1), P.wait_polls);
            if (seam) {
                if (qq == 0) patch(s0, k, sax);
                const int k1 = plane_of(P, t, qq + 1);
                patch(s1, k1, slab_axis(slab_bits(P, t, k1)));
                if (tid == kProd) p_dirty |= (qq == 0 ? 1u << (g0 % kStages) : 0u) | 1u << (g1 % kStages);
                __syncthreads();
            }

            // ------------------------------------------------ B phase
            f2 p0, p1;
            P3 nb = b_pair(P, s0, s1, j, i0, sax, bB, cB, p0, p1);
            if (kSecOn && sec) {   // CPML memory of further slab axes, both points at once
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (!((sec >> a) & 1u)) continue;
                    const int pos0 = a == 0 ? gx0 : a == 1 ? gy : k, pos1 = a == 0 ? gx0 + 1 : pos0;
                    const bool in0 = v0 && slab_pos(P, a, pos0), in1 = v1 && slab_pos(P, a, pos1);
                    if (!in0 && !in1) continue;
                    const int e0 = a == 0 ? i0 : a == 1 ? kCfY + j : kCfZ + qq, e1 = a == 0 ? i0 + 1 : e0;
                    const f2 bb = pk(in0 ? s_cf[cur][0][e0] : 0.f, in1 ? s_cf[cur][0][e1] : 0.f);
                    const f2 cc = pk(in0 ? s_cf[cur][1][e0] : 0.f, in1 ? s_cf[cur][1][e1] : 0.f);
                    f2 d0, d1;
                    e_diffs2(s0, s1, j, i0, a, d0, d1);
                    const f2 n0 = fma2(bb, ld2(P.psiB[pair_c1(a)][a] + q), mul2(cc, d0));
                    const f2 n1 = fma2(bb, ld2(P.psiB[pair_c2(a)][a] + q), mul2(cc, d1));
                    b_add_psi(a, n0, n1, nb);
                    if (own) {
                        const unsigned inm = (in0 ? 1u : 0u) | (in1 ? 2u : 0u);
                        st2m(O.psiB[pair_c1(a)][a] + q, n0, inm & mbits(mk, pair_c1(a)));
                        st2m(O.psiB[pair_c2(a)][a] + q, n1, inm & mbits(mk, pair_c2(a)));
                    }
                }
            }
            if (masked) {
                nb.x = sel2(nb.x, ld2(&s0.b[0][j][i0]), mbits(mk, 0));
                nb.y = sel2(nb.y, ld2(&s0.b[1][j][i0]), mbits(mk, 1));
                nb.z = sel2(nb.z, ld2(&s0.b[2][j][i0]), mbits(mk, 2));
            }
            st2(&bn[0][j][i0], nb.x);
            st2(&bn[1][j][i0], nb.y);
            st2(&bn[2][j][i0], nb.z);
            if (own) {
                st2(O.B[0] + q, nb.x);
                st2(O.B[1] + q, nb.y);
                st2(O.B[2] + q, nb.z);
                if (sl) {
                    const unsigned vm = v1 ? 3u : 1u;
                    st2m(O.psiB[pair_c1(sax)][sax] + q, p0, sl & vm & mbits(mk, pair_c1(sax)));
                    st2m(O.psiB[pair_c2(sax)][sax] + q, p1, sl & vm & mbits(mk, pair_c2(sax)));
                }
            }
            if (hal) {
                f2 hp0, hp1;
                P3 h = b_pair(P, s0, s1, hj, hi0, sax, hbB, hcB, hp0, hp1);
                if (kSecOn && sec) {   // further slab axes of the halo pair (their new memories: formed by the owner)
                    int n = 0;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        if (!((sec >> a) & 1u)) continue;
                        const unsigned m2 = (hin >> (2 * a)) & 3u;
                        const f2 o1 = n == 0 ? ho0 : ho2, o2 = n == 0 ? ho1 : ho3;
                        ++n;
                        if (!m2) continue;
                        f2 bb, cc;
                        if (a == 0) {
                            bb = ld2(&s_cf[cur][0][hi0]);
                            cc = ld2(&s_cf[cur][1][hi0]);
                        } else {
                            const int e = a == 1 ? kCfY + hj : kCfZ + qq;
                            bb = pk(s_cf[cur][0][e], s_cf[cur][0][e]);
                            cc = pk(s_cf[cur][1][e], s_cf[cur][1][e]);
                        }
                        bb = sel2(bb, 0, m2);
                        cc = sel2(cc, 0, m2);
                        f2 d0, d1;
                        e_diffs2(s0, s1, hj, hi0, a, d0, d1);
                        b_add_psi(a, fma2(bb, o1, mul2(cc, d0)), fma2(bb, o2, mul2(cc, d1)), h);
                    }
                }
                if (masked) {
                    h.x = sel2(h.x, ld2(&s0.b[0][hj][hi0]), mbits(hmk, 0));
                    h.y = sel2(h.y, ld2(&s0.b[1][hj][hi0]), mbits(hmk, 1));
                    h.z = sel2(h.z, ld2(&s0.b[2][hj][hi0]), mbits(hmk, 2));
                }
                if (hrow)
                    st2(&bn[0][hj][hi0], h.x);
                else
                    st2(&bn[1][hj][hi0], h.y);
                st2(&bn[2][hj][hi0], h.z);
            }
            if (qq == 1) rec_store(s_item[cur ^ 1], cur ^ 1, rnext, cfnext);   // loaded during plane 0
            // every thread is past the E phase of the plane before: its stage is free
            if (__syncthreads_or(!ok)) return false;
            if (tid == kProd) {
                consumed = g0;
                pump(qq >= 1);   // the next item's arguments were staged during plane 0
                if (qq == 0) {
                    phas = s_item[cur ^ 1] >= 0;
                    if (phas) ptk = ticket();
                }
                if (qq == 1 || nq == 2) pend = phas ? item_of(ptk) : -1LL;
            }
            if (qq == 0) {
                rec_load(s_item[cur ^ 1], rnext, cfnext);
                stage_args(s_item[cur ^ 1], cur ^ 1);   // read from the next item on, after a barrier
            }

            // ------------------------------------------------ E phase
            if (own) {
                const f2 em0 = ld2(&s0.e[0][j][i0]), em1 = ld2(&s0.e[1][j][i0]), em2 = ld2(&s0.e[2][j][i0]);
                f2 hx = nb.x, hx_zm = bpx, hx_ym = ld2(&bn[0][j - 1][i0]);
                f2 hy = nb.y, hy_zm = bpy, hy_xm = pk(bn[1][j][i0 - 1], lo(nb.y));
                f2 hz = nb.z, hz_ym = ld2(&bn[2][j - 1][i0]), hz_xm = pk(bn[2][j][i0 - 1], lo(nb.z));
                const bool imuf = kFull && (f & kFImu);
                if (!P.uniform_mu && !imuf) {   // one record: one mu
                    const f2 w = pk(rec.w, rec.w);
                    hx = mul2(hx, w); hx_zm = mul2(hx_zm, w); hx_ym = mul2(hx_ym, w);
                    hy = mul2(hy, w); hy_zm = mul2(hy_zm, w); hy_xm = mul2(hy_xm, w);
                    hz = mul2(hz, w); hz_ym = mul2(hz_ym, w); hz_xm = mul2(hz_xm, w);
                }
                f2 dHz_y = sub2(hz, hz_ym), dHy_z = sub2(hy, hy_zm), dHx_z = sub2(hx, hx_zm);
                f2 dHz_x = sub2(hz, hz_xm), dHy_x = sub2(hy, hy_xm), dHx_y = sub2(hx, hx_ym);
                if (imuf) {   // mu varies: 1/mu per face, point by point
                    float d[6][2];
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        const int gx = gx0 + p;
                        const int km = k > 0 ? k - 1 : P.N[2] - 1;
                        const int xm = gx > 0 ? gx - 1 : P.N[0] - 1, ym = gy > 0 ? gy - 1 : P.N[1] - 1;
                        auto h = [&](f2 v) { return p ? hi(v) : lo(v); };
                        const bool vp = p ? v1 : v0;
                        const int gxs = vp ? gx : gx0, xms = vp ? xm : gx0;
                        const float Hz = h(hz) * imu(P, 2, gxs, gy, k), Hz_ym = h(hz_ym) * imu(P, 2, gxs, ym, k);
                        const float Hz_xm = h(hz_xm) * imu(P, 2, xms, gy, k);
                        const float Hy = h(hy) * imu(P, 1, gxs, gy, k), Hy_zm = h(hy_zm) * imu(P, 1, gxs, gy, km);
                        const float Hy_xm = h(hy_xm) * imu(P, 1, xms, gy, k);
                        const float Hx = h(hx) * imu(P, 0, gxs, gy, k), Hx_zm = h(hx_zm) * imu(P, 0, gxs, gy, km);
                        const float Hx_ym = h(hx_ym) * imu(P, 0, gxs, ym, k);
                        d[0][p] = Hz - Hz_ym;
                        d[1][p] = Hy - Hy_zm;
                        d[2][p] = Hx - Hx_zm;
                        d[3][p] = Hz - Hz_xm;
                        d[4][p] = Hy - Hy_xm;
                        d[5][p] = Hx - Hx_ym;
                    }
                    dHz_y = pk(d[0][0], d[0][1]);
                    dHy_z = pk(d[1][0], d[1][1]);
                    dHx_z = pk(d[2][0], d[2][1]);
                    dHz_x = pk(d[3][0], d[3][1]);
                    dHy_x = pk(d[4][0], d[4][1]);
                    dHx_y = pk(d[5][0], d[5][1]);
                }
                const f2 r0 = pk(P.r[0], P.r[0]), r1 = pk(P.r[1], P.r[1]), r2 = pk(P.r[2], P.r[2]);
                f2 cx = sub2(mul2(r1, dHz_y), mul2(r2, dHy_z));
                f2 cy = sub2(mul2(r2, dHx_z), mul2(r0, dHz_x));
                f2 cz = sub2(mul2(r0, dHy_x), mul2(r1, dHx_y));
                // CPML memory of the staged axis: psi' = b psi + c d, added to the curl
                f2 q0 = 0, q1 = 0;
                if (sax == 0) {          // Ey, Ez
                    q0 = fma2(bE, pe0, mul2(cE, dHz_x));
                    q1 = fma2(bE, pe1, mul2(cE, dHy_x));
                    cy = sub2(cy, q0);
                    cz = add2(cz, q1);
                } else if (sax == 1) {   // Ex, Ez
                    q0 = fma2(bE, pe0, mul2(cE, dHz_y));
                    q1 = fma2(bE, pe1, mul2(cE, dHx_y));
                    cx = add2(cx, q0);
                    cz = sub2(cz, q1);
                } else if (sax == 2) {   // Ex, Ey
                    q0 = fma2(bE, pe0, mul2(cE, dHy_z));
                    q1 = fma2(bE, pe1, mul2(cE, dHx_z));
                    cx = sub2(cx, q0);
                    cy = add2(cy, q1);
                }
                if (kSecOn && sec) {   // further slab axes, both points at once
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        if (!((sec >> a) & 1u)) continue;
                        const int pos0 = a == 0 ? gx0 : a == 1 ? gy : k, pos1 = a == 0 ? gx0 + 1 : pos0;
                        const bool in0 = v0 && slab_pos(P, a, pos0), in1 = v1 && slab_pos(P, a, pos1);
                        if (!in0 && !in1) continue;
                        const int e0 = a == 0 ? i0 : a == 1 ? kCfY + j : kCfZ + qq, e1 = a == 0 ? i0 + 1 : e0;
                        const f2 bb = pk(in0 ? s_cf[cur][2][e0] : 0.f, in1 ? s_cf[cur][2][e1] : 0.f);
                        const f2 cc = pk(in0 ? s_cf[cur][3][e0] : 0.f, in1 ? s_cf[cur][3][e1] : 0.f);
                        float* w1 = P.psiE[pair_c1(a)][a] + q;
                        float* w2 = P.psiE[pair_c2(a)][a] + q;
                        const f2 d1 = a == 0 ? dHz_x : a == 1 ? dHz_y : dHy_z;
                        const f2 d2 = a == 0 ? dHy_x : a == 1 ? dHx_y : dHx_z;
                        const f2 n1 = fma2(bb, ld2(w1), mul2(cc, d1));
                        const f2 n2 = fma2(bb, ld2(w2), mul2(cc, d2));
                        // the pair of axis a enters the curl with signs (-, +), (+, -), (-, +)
                        if (a == 0) {
                            cy = sub2(cy, n1);
                            cz = add2(cz, n2);
                        } else if (a == 1) {
                            cx = add2(cx, n1);
                            cz = sub2(cz, n2);
                        } else {
                            cx = sub2(cx, n1);
                            cy = add2(cy, n2);
                        }
                        const unsigned inm = (in0 ? 1u : 0u) | (in1 ? 2u : 0u);
                        st2m(w1, n1, inm & mbits(mk, 3 + pair_c1(a)));
                        st2m(w2, n2, inm & mbits(mk, 3 + pair_c2(a)));
                    }
                }
                // Js^{n+1/2} = Js + kt E^n, E^{n+1} = ca E^n + cb (curl - Js^{n+1/2})
                f2 jt0 = 0, jt1 = 0, jt2 = 0;
                if (sc) {
                    jt0 = fma2(cj0, em0, jo0);
                    jt1 = fma2(cj1, em1, jo1);
                    jt2 = fma2(cj2, em2, jo2);
                }
                f2 n0 = fma2(cb0, sub2(cx, jt0), mul2(ca0, em0));
                f2 n1 = fma2(cb1, sub2(cy, jt1), mul2(ca1, em1));
                f2 n2 = fma2(cb2, sub2(cz, jt2), mul2(ca2, em2));
                if (kFull && (f & kFSrc)) {   // soft sources
                    float ax0 = 0.f, ax1 = 0.f, ay0 = 0.f, ay1 = 0.f, az0 = 0.f, az1 = 0.f;
                    for (int s = 0; s < S.n; ++s) {
                        if (gy < S.lo[s][1] || gy >= S.hi[s][1] || k < S.lo[s][2] || k >= S.hi[s][2]) continue;
                        const float v = amp_of(s);
                        const float u0 = (gx0 >= S.lo[s][0] && gx0 < S.hi[s][0]) ? v : 0.f;
                        const float u1 = (gx0 + 1 >= S.lo[s][0] && gx0 + 1 < S.hi[s][0]) ? v : 0.f;
                        const int c = S.comp[s];
                        if (c == 0) {
                            ax0 += u0;
                            ax1 += u1;
                        } else if (c == 1) {
                            ay0 += u0;
                            ay1 += u1;
                        } else {
                            az0 += u0;
                            az1 += u1;
                        }
                    }
                    n0 = add2(n0, pk(ax0, ax1));
                    n1 = add2(n1, pk(ay0, ay1));
                    n2 = add2(n2, pk(az0, az1));
                }
                if (masked) {
                    n0 = sel2(n0, em0, mbits(mk, 3));
                    n1 = sel2(n1, em1, mbits(mk, 4));
                    n2 = sel2(n2, em2, mbits(mk, 5));
                    jt0 = sel2(jt0, jo0, mbits(mk, 3));
                    jt1 = sel2(jt1, jo1, mbits(mk, 4));
                    jt2 = sel2(jt2, jo2, mbits(mk, 5));
                }
                st2(O.E[0] + q, n0);
                st2(O.E[1] + q, n1);
                st2(O.E[2] + q, n2);
                if (sc) {
                    st2(O.J[0] + q, jt0);
                    st2(O.J[1] + q, jt1);
                    st2(O.J[2] + q, jt2);
                }
                if (sl) {
                    const unsigned vm = v1 ? 3u : 1u;
                    st2m(P.psiE[pair_c1(sax)][sax] + q, q0, sl & vm & mbits(mk, 3 + pair_c1(sax)));
                    st2m(P.psiE[pair_c2(sax)][sax] + q, q1, sl & vm & mbits(mk, 3 + pair_c2(sax)));
                }
                const f2 sum = add2(add2(n0, n1), n2);
                if (!isfinite(lo(sum) + (v1 ? hi(sum) : 0.f))) atomicOr(P.status, kStatusNonFinite);
                // first-order Mur on the z walls: E_w^{n+1} = E_i^n + M (E_i^{n+1} - E_w^n)
                if (kFull && (f & (kFMurLo | kFMurHi))) {
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        if (!(p ? v1 : v0)) continue;
                        auto h = [&](f2 v) { return p ? hi(v) : lo(v); };
                        const bool mx = m >> (6 * p + 3) & 1u, my = m >> (6 * p + 4) & 1u;
                        const int ow = o + p, pw = P.n[2] * PL + o + p;
                        if (f & kFMurLo) {
                            if (mx) O.E[0][ow] = h(em0) + P.mur_M * (h(n0) - h(elo0));
                            if (my) O.E[1][ow] = h(em1) + P.mur_M * (h(n1) - h(elo1));
                        }
                        if (f & kFMurHi) {
                            if (mx) O.E[0][pw] = h(em0) + P.mur_M * (h(n0) - s1.e[0][j][i0 + p]);
                            if (my) O.E[1][pw] = h(em1) + P.mur_M * (h(n1) - s1.e[1][j][i0 + p]);
                        }
                    }
                }
            }
            if (kFull && zlo) {
                elo0 = ld2(&s0.e[0][j][i0]);
                elo1 = ld2(&s0.e[1][j][i0]);
            }
            bpx = nb.x;
            bpy = nb.y;
            return true;
        };
        const int kind = item_kind(P, S, mur, t);
        for (int qq = 0; qq < nq - 1; ++qq, ++it) {
            const bool ok = kind == 0   ? plane(std::integral_constant<int, 0>{}, qq)
                            : kind == 1 ? plane(std::integral_constant<int, 1>{}, qq)
                                        : plane(std::integral_constant<int, 2>{}, qq);
            if (!ok) {
                aborted = true;
                break;
            }
        }
        if (aborted) break;
        seq0 += nq;
        // this item is done: its slot takes the item after the next one
        if (nq == 2) rec_store(s_item[cur ^ 1], cur ^ 1, rnext, cfnext);   // a one-plane item: no plane 1
        if (tid == kProd) {
            s_item[cur] = pend;
            ++c_ord;
        }
        if (nq == 2) __syncthreads();
        cur ^= 1;
    }
    if (aborted) {
        // a copy never landed: flag it, give the copies in flight a bounded
        // time to finish (they write this CTA's shared memory), stop
        if (tid == kProd) {
            if constexpr (kBatch) {   // the CTA's later items, of any grid, stay undone
                for (int gi = 0; gi < BL.ngrids; ++gi) atomicOr(BL.G[gi].P[par].status, kStatusTimeout);
            } else {
                if (status) atomicOr(status, kStatusTimeout);
            }
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

// opt the kernels in to the dynamic shared memory they need (above the 48 KB default)
static cudaError_t step_smem_attribute() {
    cudaError_t e = cudaFuncSetAttribute(k_step_t<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)step_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_step_t<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)step_smem_bytes());
    return e;
}

int step_blocks_per_sm() {
    if (step_smem_attribute() != cudaSuccess) return 0;
    int nb = 0, nb2 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_t<false>, kThreads, step_smem_bytes()) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb2, k_step_t<true>, kThreads, step_smem_bytes()) !=
            cudaSuccess)
        return 0;
    return nb < nb2 ? nb : nb2;
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

cudaError_t launch_step(const void* tmaps, const Params& P, const StepOut& O, const Sources& S, const Probes& R,
                        long long n, int blocks, cudaStream_t st) {
    static cudaError_t attr = step_smem_attribute();
    if (attr != cudaSuccess) return attr;
    const TMaps* tm = (const TMaps*)tmaps;
    BatchLaunch none;
    memset(&none, 0, sizeof(none));
    k_step_t<false><<<blocks, dim3(kTX, kThreadsY), step_smem_bytes(), st>>>(*tm, P, O, S, R, n, none);
    return cudaGetLastError();
}

cudaError_t launch_step_batch(const BatchLaunch& BL, int blocks, cudaStream_t st) {
    static cudaError_t attr = step_smem_attribute();
    if (attr != cudaSuccess) return attr;
    // the by-value grid arguments are unused in a batched launch
    TMaps tm;
    memset(&tm, 0, sizeof(tm));
    Params P;
    memset(&P, 0, sizeof(P));
    StepOut O;
    memset(&O, 0, sizeof(O));
    Sources S;
    memset(&S, 0, sizeof(S));
    Probes R;
    memset(&R, 0, sizeof(R));
    k_step_t<true><<<blocks, dim3(kTX, kThreadsY), step_smem_bytes(), st>>>(tm, P, O, S, R, 0, BL);
    return cudaGetLastError();
}

__global__ void k_step_advance(int* step) { *step += 1; }

cudaError_t launch_step_advance(int* step, cudaStream_t st) {
    k_step_advance<<<1, 1, 0, st>>>(step);
    return cudaGetLastError();
}

// work items of a launch, in the order they are handed out: the (tile, z
// chunk) items that need the full plane loop come first -- on a grid with
// few items per CTA (`split`) each cut into kSub-plane pieces, so that their
// long bodies run side by side -- then the others, z chunk by z chunk (the
// CTAs at work at one time then share halos in L2), the last `tail` of them
// cut into kSub-plane pieces so that the CTAs run out of work together.
// One CTA; writes the descriptors and their count.
__global__ void __launch_bounds__(1024) k_item_order(Params P, StepOut O, Sources S, int split, int tail, int chunk,
                                                    long long* order,
                                                    int* count) {
    __shared__ int s_slow[1024], s_fast[1024], s_tail[1024];
    const int ntiles = O.ntx * O.nty, n = ntiles * ((O.kend + chunk - 1) / chunk);
    const int per = (n + 1023) / 1024;
    const int a = min((int)threadIdx.x * per, n), b = min(a + per, n);
    const bool mur = P.bc[2] == TF_BC_MUR;
    auto item_at = [&](int d, int& tile, int& kz0, int& len) {
        tile = d % ntiles;
        kz0 = (d / ntiles) * chunk;
        len = min(chunk, O.kend - kz0);
    };
    auto rare_of = [&](int tile, int kz0, int len) {
        return item_kind(P, S, mur, tile_of(P, O, make_item(tile, kz0, len))) != 0;
    };
    auto scan = [&](int* v) {   // inclusive prefix sum over the block
        for (int off = 1; off < 1024; off <<= 1) {
            const int x = (int)threadIdx.x >= off ? v[threadIdx.x - off] : 0;
            __syncthreads();
            v[threadIdx.x] += x;
            __syncthreads();
        }
    };
    int ns = 0, nf = 0;
    for (int d = a; d < b; ++d) {
        int tile, kz0, len;
        item_at(d, tile, kz0, len);
        if (rare_of(tile, kz0, len))
            ns += split ? (len + kSub - 1) / kSub : 1;
        else
            nf += 1;
    }
    s_slow[threadIdx.x] = ns;
    s_fast[threadIdx.x] = nf;
    __syncthreads();
    scan(s_slow);
    scan(s_fast);
    const int total_slow = s_slow[1023], total_fast = s_fast[1023];
    const int cut = total_fast - min(tail, total_fast);   // fast items from this rank on are cut into pieces
    int nt = 0;
    {
        int rank = s_fast[threadIdx.x] - nf;
        for (int d = a; d < b; ++d) {
            int tile, kz0, len;
            item_at(d, tile, kz0, len);
            if (rare_of(tile, kz0, len)) continue;
            if (rank >= cut) nt += (len + kSub - 1) / kSub;
            ++rank;
        }
    }
    s_tail[threadIdx.x] = nt;
    __syncthreads();
    scan(s_tail);
    int r = s_slow[threadIdx.x] - ns;                     // slow pieces before this thread's range
    int rank = s_fast[threadIdx.x] - nf;                  // fast items before it
    int c = total_slow + cut + s_tail[threadIdx.x] - nt;  // position of its first tail piece
    for (int d = a; d < b; ++d) {
        int tile, kz0, len;
        item_at(d, tile, kz0, len);
        if (rare_of(tile, kz0, len)) {
            const int piece = split ? kSub : len;
            for (int k = kz0; k < kz0 + len; k += piece) order[r++] = make_item(tile, k, min(piece, kz0 + len - k));
        } else {
            if (rank < cut) {
                order[total_slow + rank] = make_item(tile, kz0, len);
            } else {
                for (int k = kz0; k < kz0 + len; k += kSub) order[c++] = make_item(tile, k, min(kSub, kz0 + len - k));
            }
            ++rank;
        }
    }
    if (threadIdx.x == 1023) *count = total_slow + cut + s_tail[1023];
}

cudaError_t launch_item_order(const Params& P, const StepOut& O, const Sources& S, int split, int tail, int chunk,
                              long long* order, int* count, cudaStream_t st) {
    if (chunk < 1 || chunk > kItemMax) return cudaErrorInvalidValue;
    k_item_order<<<1, 1024, 0, st>>>(P, O, S, split, tail, chunk, order, count);
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
