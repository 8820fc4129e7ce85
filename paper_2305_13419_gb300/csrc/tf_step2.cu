// tf_step2.cu -- two steps of the fused leapfrog per pass (temporal
// blocking) on the interior box of a grid (sm_103a).
//
// One launch advances the points of the box from level n to level n + 2 by
// Algorithm 1 (arXiv 2305.13419, Sec. 3) in its fused form, twice:
//   B1 = Bt^{n+1/2} = Bt^{n-1/2} - curl(E^n)
//   E1 = E^{n+1}    = ca E^n + cb (curl(B1) - (Jt^{n-1/2} + kt E^n))
//   B2 = Bt^{n+3/2} = B1 - curl(E1)
//   E2 = E^{n+2}    = ca E1 + cb (curl(B2) - (Jt^{n+1/2} + kt E1))
// with the soft sources of both steps.  The box keeps every point this
// kernel computes (its tiles plus a two-point halo) off the walls, outside
// the CPML slabs and off the Mur planes, and mu is uniform, so no masks and
// no CPML memories appear here; the single-step kernel advances the rest.
//
// Work layout.  A CTA of 256 threads owns a 32 x 16 column tile (as the
// single-step kernel) and streams it along z through a work item of up to
// 24 planes.  E^n and B^{n-1/2} of each plane land by TMA boxes (x0-4 ..
// x0+35, y0-2 .. y0+17 / y0+16) through a ring of four mbarrier-guarded
// stages filled by one producer thread that runs ahead into the next item.
// The first step is formed on the tile plus a two-point halo, the second on
// the tile; the second step trails the first by one plane for B and two for
// E, so per plane k there are two phases, each closed by one barrier:
//   X(k): B1 at plane k (tile + halo)     and  E2 at plane k - 2 (tile)
//   Y(k): E1 at plane k (tile + halo)     and  B2 at plane k - 1 (tile + low halo)
// B1, E1 (two planes) and B2 live in shared memory for the neighbours'
// differences; a thread keeps its own points' previous planes in registers
// for the z differences.  Work is counted in x-adjacent point pairs
// ("slots"): each thread owns one slot of the tile, and threads 0..85 also
// one slot of the halo ring.  Every pair travels in 64-bit registers and
// uses the packed FP32x2 operations in exactly the order of the
// single-step kernel, and a halo point takes its coefficients (record or
// per-point arrays) and its current / source treatment from the tile that
// owns it, so two steps here give the same bits as two single steps.
#include <math.h>

#include "tf_device.cuh"
#include "tf_internal.cuh"

namespace tf {

namespace {

using namespace dev;

constexpr int kQX = kT2BoxX, kQEY = kT2BoxEY, kQBY = kT2BoxBY;   // stage boxes from (x0-4, y0-2)
constexpr int kW1 = 36, kR1B = 19, kR1E = 18;   // B1 / E1 planes: x0-2 .. x0+33; rows y0-2.. / y0-1..
constexpr int kW2 = 34, kR2B = 17;              // B2 plane: x0-2 .. x0+31, rows y0-1 .. y0+15
constexpr int kThr = 256, kExtra = 86;
constexpr int kProd2 = 224;                     // producer: lane 0 of the last warp (no halo slot)
constexpr int kRecN = kTBLenMax + 2;            // planes with first-step E work: kz0-1 .. kz1

struct __align__(128) Stage2 {
    alignas(128) float e[3][kQEY][kQX];
    alignas(128) float b[3][kQBY][kQX];
};
constexpr unsigned kE2Bytes = 3u * kQEY * kQX * 4, kB2Bytes = 3u * kQBY * kQX * 4;
struct Planes2 {
    float b1[3][kR1B][kW1];
    float e1[2][3][kR1E][kW1];
    float b2[3][kR2B][kW2];
};
static_assert(sizeof(Planes2) % 8 == 0, "planes are cleared as float2");

struct TMaps2 {
    CUtensorMap e, b;
};

struct It2 {
    int bx, by, x0, y0, kz0, kz1, nq;
};
__device__ __forceinline__ It2 it2_of(const Step2Out& O, long long d) {
    It2 t;
    const int tile = item_tile(d);
    t.kz0 = item_kz0(d);
    const int len = item_len(d);
    t.bx = tile % O.ntx;
    t.by = tile / O.ntx;
    t.x0 = t.bx * kSX;
    t.y0 = t.by * kSY;
    t.kz1 = t.kz0 + len;
    t.nq = len + 4;   // planes kz0-2 .. kz1+1
    return t;
}

// the halo slots: pair column px (x0-2+2px), row ry (y0-2+ry)
__device__ __forceinline__ void extra_slot(int e, int& px, int& ry) {
    if (e < 18) {
        ry = 0;
        px = e;
    } else if (e < 36) {
        ry = 1;
        px = e - 18;
    } else if (e < 54) {
        ry = 18;
        px = e - 36;
    } else if (e < 70) {
        ry = 2 + (e - 54);
        px = 0;
    } else {
        ry = 2 + (e - 70);
        px = 17;
    }
}
// tile of a slot relative to the CTA's tile: 0 .. 8 = (dy + 1) * 3 + dx + 1
__device__ __forceinline__ int slot_nb(int px, int ry) {
    const int dx = px == 0 ? -1 : px == 17 ? 1 : 0;
    const int dy = ry <= 1 ? -1 : ry == 18 ? 1 : 0;
    return (dy + 1) * 3 + dx + 1;
}

// sources at the pair (gx, gx + 1) of row gy, plane k: the per-component sums
// of the single-step kernel, in the same order
__device__ __forceinline__ void add_sources(const Sources& S, const float* amp, int gx, int gy, int k, f2& n0,
                                            f2& n1, f2& n2) {
    float ax0 = 0.f, ax1 = 0.f, ay0 = 0.f, ay1 = 0.f, az0 = 0.f, az1 = 0.f;
    for (int s = 0; s < S.n; ++s) {
        if (gy < S.lo[s][1] || gy >= S.hi[s][1] || k < S.lo[s][2] || k >= S.hi[s][2]) continue;
        const float v = amp[s];
        const float u0 = (gx >= S.lo[s][0] && gx < S.hi[s][0]) ? v : 0.f;
        const float u1 = (gx + 1 >= S.lo[s][0] && gx + 1 < S.hi[s][0]) ? v : 0.f;
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

// Bt' = Bt - curl E at a pair from E at the pair (e), its +y row (ey1), its
// +z plane (ez1) and the point past its high x end (hx: index + 2)
struct E3 {
    f2 x, y, z;
};
__device__ __forceinline__ E3 b_new(const Params& P, E3 old, E3 e, E3 ey1, E3 ez1, float ez_x2, float ey_x2) {
    const f2 dEz_y = sub2(ey1.z, e.z), dEx_y = sub2(ey1.x, e.x);
    const f2 dEy_z = sub2(ez1.y, e.y), dEx_z = sub2(ez1.x, e.x);
    const f2 dEz_x = sub2(pk(hi(e.z), ez_x2), e.z), dEy_x = sub2(pk(hi(e.y), ey_x2), e.y);
    const f2 r0 = pk(P.r[0], P.r[0]), r1 = pk(P.r[1], P.r[1]), r2 = pk(P.r[2], P.r[2]);
    E3 b;
    b.x = fma2(r2, dEy_z, sub2(old.x, mul2(r1, dEz_y)));
    b.y = fma2(r0, dEz_x, sub2(old.y, mul2(r2, dEx_z)));
    b.z = fma2(r1, dEx_y, sub2(old.z, mul2(r0, dEy_x)));
    return b;
}

// E' = ca E + cb (curl H - Jt') with Jt' = Jt + kt E (sc: the tile-plane
// carries superconducting edges, else Jt' = 0), from H at the pair (h), its
// -z plane (x, y), -y row (x, z) and the point below its low x end (y, z)
__device__ __forceinline__ void e_new(const Params& P, E3 h, f2 hx_zm, f2 hy_zm, f2 hx_ym, f2 hz_ym, float hy_x,
                                      float hz_x, const f2 em[3], const f2 ca[3], const f2 cb[3], const f2 cj[3],
                                      const f2 jo[3], bool sc, f2 n[3], f2 jt[3]) {
    const f2 hy_xm = pk(hy_x, lo(h.y)), hz_xm = pk(hz_x, lo(h.z));
    const f2 dHz_y = sub2(h.z, hz_ym), dHy_z = sub2(h.y, hy_zm), dHx_z = sub2(h.x, hx_zm);
    const f2 dHz_x = sub2(h.z, hz_xm), dHy_x = sub2(h.y, hy_xm), dHx_y = sub2(h.x, hx_ym);
    const f2 r0 = pk(P.r[0], P.r[0]), r1 = pk(P.r[1], P.r[1]), r2 = pk(P.r[2], P.r[2]);
    const f2 cx = sub2(mul2(r1, dHz_y), mul2(r2, dHy_z));
    const f2 cy = sub2(mul2(r2, dHx_z), mul2(r0, dHz_x));
    const f2 cz = sub2(mul2(r0, dHy_x), mul2(r1, dHx_y));
    jt[0] = jt[1] = jt[2] = 0;
    if (sc) {
        jt[0] = fma2(cj[0], em[0], jo[0]);
        jt[1] = fma2(cj[1], em[1], jo[1]);
        jt[2] = fma2(cj[2], em[2], jo[2]);
    }
    n[0] = fma2(cb[0], sub2(cx, jt[0]), mul2(ca[0], em[0]));
    n[1] = fma2(cb[1], sub2(cy, jt[1]), mul2(ca[1], em[1]));
    n[2] = fma2(cb[2], sub2(cz, jt[2]), mul2(ca[2], em[2]));
}

// the coefficients of a pair at padded index q from its tile-plane record
// (uniform material) or the per-point arrays
__device__ __forceinline__ void coeffs(const Params& P, float4 rec, long long q, f2 ca[3], f2 cb[3], f2 cj[3]) {
    if (isnan(rec.x)) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ca[c] = ld2(P.ca[c] + q);
            cb[c] = ld2(P.cb[c] + q);
            cj[c] = ld2(P.cj[c] + q);
        }
    } else {
        ca[0] = ca[1] = ca[2] = pk(rec.x, rec.x);
        cb[0] = cb[1] = cb[2] = pk(rec.y, rec.y);
        cj[0] = cj[1] = cj[2] = pk(rec.z, rec.z);
    }
}

}  // namespace

__global__ void __launch_bounds__(kThr, 2)
    k_step2(const __grid_constant__ TMaps2 tm, Params P, Step2Out O, Sources S) {
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    Stage2* stg = reinterpret_cast<Stage2*>(smem_raw);
    Planes2& pl = *reinterpret_cast<Planes2*>(smem_raw + kStages * sizeof(Stage2));
    unsigned long long* bar =
        reinterpret_cast<unsigned long long*>(smem_raw + kStages * sizeof(Stage2) + sizeof(Planes2));
    __shared__ long long s_item[2];            // current and next work item (-1: none)
    __shared__ float4 s_rec[2][kRecN][9];      // records of the 3 x 3 tiles around the tile, per E1 plane
    __shared__ unsigned s_flag[2][kRecN];      // bits 0-8: sources reach tile nb on the plane; 9: a probe point
    const int tid = threadIdx.x;
    const int nitems = O.nitems;
    const int PL = (int)P.plane;

    auto ticket = [&]() -> unsigned long long { return atomicAdd(O.ctr, 1ull); };
    auto item_of = [&](unsigned long long tk) -> long long {
        const long long d = (long long)(tk - O.base) + 2LL * gridDim.x;
        return (d >= 0 && d < nitems) ? __ldg(O.order + d) : -1LL;
    };
    // records and flags of an item: loaded into registers ...
    auto rec_load = [&](long long item, float4& r, unsigned& f) {
        if (item < 0) return;
        const It2 t = it2_of(O, item);
        const int npl = t.kz1 - t.kz0 + 2;
        if (tid < 9 * npl) {
            const int p = tid / 9, nb = tid % 9;
            const int tb = (t.by + nb / 3 - 1) * O.ntx + (t.bx + nb % 3 - 1);
            r = __ldg(O.tilemat + (long long)tb * P.N[2] + (t.kz0 - 1 + p));
        }
        if (tid < npl) {
            const int k = t.kz0 - 1 + tid;
            f = 0;
            if (S.n > 0 && k >= S.bb_lo[2] && k < S.bb_hi[2])
                for (int nb = 0; nb < 9; ++nb) {   // the single-step kernel's source test of that tile
                    const int tx0 = t.x0 + (nb % 3 - 1) * kSX, ty0 = t.y0 + (nb / 3 - 1) * kSY;
                    if (tx0 + kSX > S.bb_lo[0] && tx0 <= S.bb_hi[0] && ty0 + kSY > S.bb_lo[1] && ty0 <= S.bb_hi[1])
                        f |= 1u << nb;
                }
            for (int p = 0; p < O.nprobe; ++p)
                if (O.probe[p][2] == k && O.probe[p][0] >= t.x0 && O.probe[p][0] < t.x0 + kSX &&
                    O.probe[p][1] >= t.y0 && O.probe[p][1] < t.y0 + kSY)
                    f |= 1u << 9;
        }
    };
    // ... and stored in its slot
    auto rec_store = [&](long long item, int slot, const float4& r, unsigned f) {
        if (item < 0) return;
        const It2 t = it2_of(O, item);
        const int npl = t.kz1 - t.kz0 + 2;
        if (tid < 9 * npl) s_rec[slot][tid / 9][tid % 9] = r;
        if (tid < npl) s_flag[slot][tid] = f;
    };

    // ---------------------------------------------- producer (thread kProd2 only)
    unsigned long long issued = 0, consumed = 0;
    int p_ord = 0, p_q = 0, c_ord = 0;
    It2 p_t;
    p_t.nq = 0;
    bool p_have = false;
    auto issue = [&](const It2& t, int q, unsigned long long seq) {
        const int s = (int)(seq % kStages);
        const int k = t.kz0 - 2 + q;
        // no proxy fence: only TMA writes the stages, threads only read them,
        // and the barrier before every issue orders those reads first
        mbar_expect_tx(&bar[s], kE2Bytes + kB2Bytes);
        tma_load_box(&stg[s].e[0][0][0], &tm.e, t.x0 - 4, t.y0 - 2, k, O.ecur, &bar[s]);
        tma_load_box(&stg[s].b[0][0][0], &tm.b, t.x0 - 4, t.y0 - 2, k, O.bcur, &bar[s]);
    };
    auto pump = [&]() {
        while (issued < consumed + kStages) {
            if (!p_have) {
                const long long item = s_item[p_ord & 1];
                if (item < 0) return;
                p_t = it2_of(O, item);
                p_have = true;
            }
            if (p_q >= p_t.nq) {
                if (p_ord > c_ord) return;   // the next slot still holds the current item
                const long long item = s_item[(p_ord + 1) & 1];
                if (item < 0) return;
                ++p_ord;
                p_q = 0;
                p_t = it2_of(O, item);
            }
            issue(p_t, p_q, issued);
            ++p_q;
            ++issued;
        }
    };

    // shared planes start finite (the unused halo corners are read, never used)
    for (int u = tid; u < (int)(sizeof(Planes2) / 8); u += kThr) reinterpret_cast<float2*>(&pl)[u] = make_float2(0.f, 0.f);
    if (tid == kProd2) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const long long b = blockIdx.x, g = gridDim.x;
        s_item[0] = b < nitems ? __ldg(O.order + b) : -1LL;
        s_item[1] = (s_item[0] >= 0 && g + b < nitems) ? __ldg(O.order + g + b) : -1LL;
    }
    __syncthreads();
    {
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
        unsigned f0 = 0, f1 = 0;
        rec_load(s_item[0], r0, f0);
        rec_load(s_item[1], r1, f1);
        rec_store(s_item[0], 0, r0, f0);
        rec_store(s_item[1], 1, r1, f1);
    }
    if (tid == kProd2) pump();
    __syncthreads();

    // the thread's slots
    const int opx = 1 + (tid & 15), ory = 2 + (tid >> 4);   // own pair of the tile
    const bool hasx = tid < kExtra;
    int xpx = 0, xry = 0;
    if (hasx) extra_slot(tid, xpx, xry);
    const int xnb = slot_nb(xpx, xry);
    const bool x1e = hasx && xry >= 1;                           // forms E1
    const bool x2b = hasx && xpx <= 16 && xry >= 1 && xry <= 17;   // forms B2
    const f2 zero = 0;

    int cur = 0;
    bool aborted = false;
    unsigned long long seq0 = 0;
    long long pend = -1;
    unsigned long long ptk = 0;
    bool phas = false;
    while (true) {
        const long long item = s_item[cur];
        if (item < 0) break;
        const It2 t = it2_of(O, item);
        const int x0 = t.x0, y0 = t.y0, kz0 = t.kz0, kz1 = t.kz1, nq = t.nq;
        // global positions of the slots
        const int ogx = x0 - 2 + 2 * opx, ogy = y0 - 2 + ory;
        const int xgx = x0 - 2 + 2 * xpx, xgy = y0 - 2 + xry;
        const int oo = ogy * P.pitch + ogx, xo = xgy * P.pitch + xgx;
        // the ring: own pairs within two points of a face of the box
        const bool oring_xy = ogx < O.lo[0] + 2 || ogx >= O.hi[0] - 2 || ogy < O.lo[1] + 2 || ogy >= O.hi[1] - 2;
        // pipeline registers: B1 of planes k - 1 / k (both slots), the own
        // pair's Jt^{n+1/2} of the last two E1 planes and its B2 of the last two planes
        E3 ob1p = {zero, zero, zero}, ob1c = ob1p, xb1p = ob1p, xb1c = ob1p, ob2p = ob1p, ob2c = ob1p;
        f2 ja[3] = {zero, zero, zero}, jb[3] = {zero, zero, zero};   // Jt^{n+1/2} of E1 planes k - 2, k - 1
        float4 rnext = make_float4(0.f, 0.f, 0.f, 0.f);
        unsigned fnext = 0;

        for (int it = 0; it < nq; ++it) {
            const int k = kz0 - 2 + it;
            const unsigned long long g0 = seq0 + it, g1 = g0 + 1;
            const bool doB1 = k <= kz1, doE1 = k >= kz0 - 1 && k <= kz1;
            const bool doB2 = k - 1 >= kz0 - 1 && k - 1 < kz1, doE2 = k - 2 >= kz0;
            const Stage2& s0 = stg[g0 % kStages];
            const Stage2& s1 = stg[g1 % kStages];
            bool ok = true;
            if (doB1) {
                ok = mbar_wait(&bar[g1 % kStages], (unsigned)((g1 / kStages) & 1), P.wait_polls);
                if (it == 0) ok = ok && mbar_wait(&bar[g0 % kStages], (unsigned)((g0 / kStages) & 1), P.wait_polls);
            }
            // ------------------------------------------------ phase X
            if (ok && doB1) {
                auto b1_slot = [&](int px, int ry) -> E3 {
                    const int j = ry, i0 = 2 * px + 2;
                    const E3 e = {ld2(&s0.e[0][j][i0]), ld2(&s0.e[1][j][i0]), ld2(&s0.e[2][j][i0])};
                    const E3 ey1 = {ld2(&s0.e[0][j + 1][i0]), zero, ld2(&s0.e[2][j + 1][i0])};
                    const E3 ez1 = {ld2(&s1.e[0][j][i0]), ld2(&s1.e[1][j][i0]), zero};
                    const E3 old = {ld2(&s0.b[0][j][i0]), ld2(&s0.b[1][j][i0]), ld2(&s0.b[2][j][i0])};
                    const E3 b = b_new(P, old, e, ey1, ez1, s0.e[2][j][i0 + 2], s0.e[1][j][i0 + 2]);
                    st2(&pl.b1[0][ry][2 * px], b.x);
                    st2(&pl.b1[1][ry][2 * px], b.y);
                    st2(&pl.b1[2][ry][2 * px], b.z);
                    return b;
                };
                ob1c = b1_slot(opx, ory);
                if (hasx) xb1c = b1_slot(xpx, xry);
                if (k >= kz0 && k < kz1 && (oring_xy || k < O.lo[2] + 2 || k >= O.hi[2] - 2)) {
                    const int q = k * PL + oo;
                    st2(O.ZB[0] + q, ob1c.x);
                    st2(O.ZB[1] + q, ob1c.y);
                    st2(O.ZB[2] + q, ob1c.z);
                }
            }
            if (doE2) {   // E2 at plane k - 2, own pair
                const int kk = k - 2, pi = kk - (kz0 - 1);
                const float4 rec = s_rec[cur][pi][4];
                const bool sc = isnan(rec.x) || rec.z > 0.f;
                const int q = kk * PL + oo;
                f2 ca[3], cb[3], cj[3];
                coeffs(P, rec, q, ca, cb, cj);
                const float(*e0)[kR1E][kW1] = pl.e1[kk & 1];
                const int jj = ory - 1, ii = 2 * opx;
                const f2 em[3] = {ld2(&e0[0][jj][ii]), ld2(&e0[1][jj][ii]), ld2(&e0[2][jj][ii])};
                f2 n[3], jt[3];
                e_new(P, ob2c, ob2p.x, ob2p.y, ld2(&pl.b2[0][jj - 1][ii]), ld2(&pl.b2[2][jj - 1][ii]),
                      pl.b2[1][jj][ii - 1], pl.b2[2][jj][ii - 1], em, ca, cb, cj, ja, sc, n, jt);
                if (s_flag[cur][pi] & (1u << 4)) add_sources(S, O.amp2, ogx, ogy, kk, n[0], n[1], n[2]);
                st2(O.E[0] + q, n[0]);
                st2(O.E[1] + q, n[1]);
                st2(O.E[2] + q, n[2]);
                if (sc) {
                    st2(O.J[0] + q, jt[0]);
                    st2(O.J[1] + q, jt[1]);
                    st2(O.J[2] + q, jt[2]);
                }
                const f2 sum = add2(add2(n[0], n[1]), n[2]);
                if (!isfinite(lo(sum) + hi(sum))) atomicOr(P.status, kStatusNonFinite);
            }
            if (it == 1) rec_store(s_item[cur ^ 1], cur ^ 1, rnext, fnext);   // loaded during iteration 0
            if (__syncthreads_or(!ok)) {
                aborted = true;
                break;
            }
            // ------------------------------------------------ phase Y
            if (doE1) {
                const int pi = k - (kz0 - 1);
                const unsigned fl = s_flag[cur][pi];
                auto e1_slot = [&](int px, int ry, int nb, int gx, int gy, int off, const E3& bc, const E3& bp,
                                   f2 jt_out[3]) -> E3 {
                    const float4 rec = s_rec[cur][pi][nb];
                    const bool sc = isnan(rec.x) || rec.z > 0.f;
                    const int q = k * PL + off;
                    f2 ca[3], cb[3], cj[3];
                    coeffs(P, rec, q, ca, cb, cj);
                    f2 jo[3] = {zero, zero, zero};
                    if (sc) {
                        jo[0] = ld2(P.J[0] + q);
                        jo[1] = ld2(P.J[1] + q);
                        jo[2] = ld2(P.J[2] + q);
                    }
                    const int j = ry, i0 = 2 * px + 2;
                    const f2 em[3] = {ld2(&s0.e[0][j][i0]), ld2(&s0.e[1][j][i0]), ld2(&s0.e[2][j][i0])};
                    const float* b1y = &pl.b1[1][ry][0];
                    const float* b1z = &pl.b1[2][ry][0];
                    f2 n[3];
                    e_new(P, bc, bp.x, bp.y, ld2(&pl.b1[0][ry - 1][2 * px]), ld2(&pl.b1[2][ry - 1][2 * px]),
                          b1y[2 * px - 1], b1z[2 * px - 1], em, ca, cb, cj, jo, sc, n, jt_out);
                    if (fl & (1u << nb)) add_sources(S, S.amp, gx, gy, k, n[0], n[1], n[2]);
                    float(*e1)[kR1E][kW1] = pl.e1[k & 1];
                    st2(&e1[0][ry - 1][2 * px], n[0]);
                    st2(&e1[1][ry - 1][2 * px], n[1]);
                    st2(&e1[2][ry - 1][2 * px], n[2]);
                    return {n[0], n[1], n[2]};
                };
                f2 jt_o[3], jt_x[3];
                const E3 oe1 = e1_slot(opx, ory, 4, ogx, ogy, oo, ob1c, ob1p, jt_o);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    ja[c] = jb[c];
                    jb[c] = jt_o[c];
                }
                E3 xe1 = {zero, zero, zero};
                if (x1e) xe1 = e1_slot(xpx, xry, xnb, xgx, xgy, xo, xb1c, xb1p, jt_x);
                if (k >= kz0 && k < kz1) {
                    bool st = oring_xy || k < O.lo[2] + 2 || k >= O.hi[2] - 2;
                    if (!st && (fl & (1u << 9)))
                        for (int p = 0; p < O.nprobe; ++p)
                            st = st || (O.probe[p][2] == k && O.probe[p][1] == ogy &&
                                        (O.probe[p][0] == ogx || O.probe[p][0] == ogx + 1));
                    if (st) {
                        const int q = k * PL + oo;
                        st2(O.ZE[0] + q, oe1.x);
                        st2(O.ZE[1] + q, oe1.y);
                        st2(O.ZE[2] + q, oe1.z);
                    }
                    const f2 sum = add2(add2(oe1.x, oe1.y), oe1.z);
                    if (!isfinite(lo(sum) + hi(sum))) atomicOr(P.status, kStatusNonFinite);
                }
                if (doB2) {   // B2 at plane k - 1 from E1 of planes k - 1 (shared) and k (own registers)
                    const float(*e0)[kR1E][kW1] = pl.e1[(k - 1) & 1];
                    auto b2_slot = [&](int px, int ry, const E3& e1k, const E3& old) -> E3 {
                        const int jj = ry - 1, ii = 2 * px;
                        const E3 e = {ld2(&e0[0][jj][ii]), ld2(&e0[1][jj][ii]), ld2(&e0[2][jj][ii])};
                        const E3 ey1 = {ld2(&e0[0][jj + 1][ii]), zero, ld2(&e0[2][jj + 1][ii])};
                        const E3 b = b_new(P, old, e, ey1, e1k, e0[2][jj][ii + 2], e0[1][jj][ii + 2]);
                        st2(&pl.b2[0][jj][ii], b.x);
                        st2(&pl.b2[1][jj][ii], b.y);
                        st2(&pl.b2[2][jj][ii], b.z);
                        return b;
                    };
                    const E3 ob2 = b2_slot(opx, ory, oe1, ob1p);
                    if (x2b) b2_slot(xpx, xry, xe1, xb1p);
                    ob2p = ob2c;
                    ob2c = ob2;
                    if (k - 1 >= kz0) {
                        const int q = (k - 1) * PL + oo;
                        st2(O.B[0] + q, ob2.x);
                        st2(O.B[1] + q, ob2.y);
                        st2(O.B[2] + q, ob2.z);
                    }
                }
            }
            ob1p = ob1c;
            xb1p = xb1c;
            if (__syncthreads_or(!ok)) {
                aborted = true;
                break;
            }
            if (tid == kProd2) {
                consumed = g0 + 1;   // every thread is past the plane's last use of its stage
                pump();
                if (it == 0) {
                    phas = s_item[cur ^ 1] >= 0;
                    if (phas) ptk = ticket();
                }
                if (it == 1) pend = phas ? item_of(ptk) : -1LL;
            }
            if (it == 0) rec_load(s_item[cur ^ 1], rnext, fnext);
        }
        if (aborted) break;
        seq0 += nq;
        if (tid == kProd2) {
            s_item[cur] = pend;
            ++c_ord;
        }
        cur ^= 1;
    }
    if (aborted) {
        // a copy never landed: flag it, give the copies in flight a bounded
        // time to finish (they write this CTA's shared memory), stop
        if (tid == kProd2) {
            atomicOr(P.status, kStatusTimeout);
            for (unsigned long long gi = consumed; gi < issued; ++gi)
                mbar_wait(&bar[gi % kStages], (unsigned)((gi / kStages) & 1));
        }
        __syncthreads();
    }
}

static size_t step2_smem_bytes() { return 128 + kStages * sizeof(Stage2) + sizeof(Planes2) + kStages * 8; }

static cudaError_t step2_smem_attribute() {
    return cudaFuncSetAttribute(k_step2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)step2_smem_bytes());
}

int step2_blocks_per_sm() {
    if (step2_smem_attribute() != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step2, kThr, step2_smem_bytes()) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t launch_step2(const void* tmaps2, const Params& P, const Step2Out& O, const Sources& S, int blocks,
                         cudaStream_t st) {
    static cudaError_t attr = step2_smem_attribute();
    if (attr != cudaSuccess) return attr;
    const TMaps2* tm = (const TMaps2*)tmaps2;
    k_step2<<<blocks, kThr, step2_smem_bytes(), st>>>(*tm, P, O, S);
    return cudaGetLastError();
}

}  // namespace tf
