// tf_internal.cuh -- device-side layout and helpers of the two-fluid Yee
// library (arXiv 2305.13419, Sec. 3 / Algorithm 1).
//
// Units on the GPU (all FP32, all O(1) for O(1) V/m fields):
//   E                 [V/m]
//   Bt = c0 B         [V/m]
//   Jt = (dt/eps0) Js [V/m]
//   r_a = c0 dt / d_a (dimensionless)
// so that the fused leapfrog reads
//   Bt^{n+1/2} = Bt^{n-1/2} - sum_a s (r_a D_a E^n + psiB)                   (steps 5+1)
//   Jt^{n+1/2} = Jt^{n-1/2} + kt_e E^n,  kt = (c0 dt)^2 / (lambda^2 mu_r)      (steps 4+2)
//   E^{n+1}    = ca E^n + cb ( sum_a s (r_a D_a (Bt/mu_r) + psiE) - Jt^{n+1/2} ) (step 3)
//   ca = (eps_e - (1-theta) st_e) / (eps_e + theta st_e),  cb = 1 / (eps_e + theta st_e),
//   st = sigma dt / eps0.
// Per-cell maps are stored scaled (eps_r, st, kt, mu_r) on the same padded
// storage grid as the fields; edge and face values are formed in-kernel.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "twofluid.h"

namespace tf {

constexpr double kC0 = 299792458.0;
constexpr double kMu0 = 1.25663706212e-6;
constexpr double kEps0 = 8.8541878128e-12;

// status bits latched on the device
constexpr unsigned kStatusNonFinite = 1u;
constexpr unsigned kStatusBadMaterial = 2u;
constexpr unsigned kStatusTimeout = 4u;

struct Params {
    int N[3];            // storage points per axis
    int n[3];            // cells per axis
    int per[3];          // periodic flag per axis
    int bc[3];           // TF_BC_* per axis
    int L[3];            // CPML cells per axis (0 without CPML)
    int pitch;           // floats per x row (multiple of 32, at least N[0] + 1)
    long long plane;     // floats per z plane
    float r[3];          // c0 dt / d_a
    float theta;
    int edge_rule;
    int uniform_mu;      // all mu_r == 1: skip the mu map
    float mur_M;         // (c0 dt - dz) / (c0 dt + dz)
    float* E[3];
    float* B[3];
    float* J[3];
    const float* eps;    // eps_r per cell
    const float* sig;    // sigma dt / eps0 per cell
    const float* kap;    // (c0 dt)^2 / (lambda^2 mu_r) per cell
    const float* mu;     // mu_r per cell
    const float* ca[3];  // per-point edge coefficients of the theta scheme (used where the
    const float* cb[3];  //   material of a tile-plane varies): E' = ca E + cb (curl - Jt),
    const float* cj[3];  //   Jt' = Jt + cj E
    float* psiB[3][3];   // [component][derivative axis], nullptr if absent
    float* psiE[3][3];
    const float* pbE[3]; // CPML b at integer positions along axis a
    const float* pcE[3]; // CPML c * r_a at integer positions
    const float* pbB[3]; // ... at half-integer positions
    const float* pcB[3];
    unsigned* status;
    long long wait_polls;  // polls of an mbarrier before a staged plane counts as lost
};

// Fused step (tf_step.cu): E, B, Js and psi_B live in three buffers (the
// current state, the next one and a scratch state for two-step passes); a
// step reads Params' buffers and writes these.
// Field arrays of the workspace, in the field tensor map's order: buffer b
// holds E (index 9b + c), B (9b + 3 + c) and Js (9b + 6 + c).
constexpr int kFieldBuffers = 3, kFieldArrays = 9 * kFieldBuffers;
// CPML arrays of one axis, in the psi tensor map's order: the psi_B pair of
// buffers 0 and 1, the psi_E pair, the psi_B pair of buffer 2.
constexpr int kPsiGroup = 8;
__host__ __device__ __forceinline__ int psib_index(int buf) { return buf == 0 ? 0 : buf == 1 ? 2 : 6; }
constexpr int kTX = 32, kTY = 16;            // owned columns per tile (x, y)
constexpr int kRows = 2;                     // adjacent y rows per thread: kTX x kTY / kRows threads
constexpr int kSX = kTX, kSY = kTY;          // tile stride
constexpr int kEX = kTX + 8, kEY = kTY + 2;  // E box: x0-4 .. x0+35, y0-1 .. y0+kTY
constexpr int kBX = kTX + 4, kBY = kTY + 1;  // B / psi_B box: x0-4 .. x0+31, y0-1 .. y0+kTY-1
constexpr int kStages = 4;                   // planes in flight per CTA
constexpr int kChunk = 8;                    // z planes per work item of a grid stepped alone
constexpr int kItemMax = 16;                 // z planes per work item at most (a batch's items)
// The last plane an item pulls is only ever the upper plane of its last
// step, so the ring must hold the two planes the next item starts with
// while that one is still in use: four stages at least.
static_assert(kStages >= 4, "the ring must reach two planes into the next item");

// per-item CPML coefficient table: kBX columns, kBY rows, kItemMax + 2 planes
// per profile; every thread loads one entry, the kCfExtra past its 256 are
// loaded by the second warp's threads
constexpr int kCfY = kBX, kCfZ = kBX + kBY, kCfN = 72;
constexpr int kCfExtra = 4 * kCfN - kTX * (kTY / kRows);
static_assert(kCfZ + kItemMax + 2 <= kCfN && kCfExtra >= 0 && kCfExtra <= 32, "table entries per thread");
static_assert(kItemMax + 1 <= 32, "the records of an item are loaded by the first warp");
constexpr int kSub = 2;                      // planes per piece of a work item that takes the full loop
// a work item is a 64-bit descriptor: tile (bits 0-19), first plane (20-39),
// planes (40-47); -1 marks the end of the work
constexpr int kMaxTiles = 1 << 20, kMaxPlanes = 1 << 20;
__host__ __device__ __forceinline__ long long make_item(int tile, int kz0, int len) {
    return (long long)tile | (long long)kz0 << 20 | (long long)len << 40;
}
__host__ __device__ __forceinline__ int item_tile(long long d) { return (int)(d & 0xfffff); }
__host__ __device__ __forceinline__ int item_kz0(long long d) { return (int)((d >> 20) & 0xfffff); }
__host__ __device__ __forceinline__ int item_len(long long d) { return (int)((d >> 40) & 0xff); }
constexpr long long kSpinLimit = 1LL << 22;  // bounded mbarrier waits

struct StepOut {
    float* E[3];
    float* B[3];
    float* J[3];
    float* psiB[3][3];
    const float4* tilemat;   // per (tile, plane): {ca, cb, cj, 1/mu} of a uniform-material
                             // tile-plane, ca = NaN where the material varies
    int ntx, nty, nch;       // tiles along x, y; z chunks
    int kend;                // planes iterated: N2 (periodic z) or N2 - 1
    int ecur, bcur;          // index of the current E / B arrays in the field tensor map
    int psi_slot[3];         // per axis: group of kPsiGroup psi arrays in the psi tensor map, -1 if no CPML
    int psib_cur;            // 0, 2 or 6: current psi_B pair inside a group (psi_E pair at 4)
    const long long* order;  // work-item descriptors of a launch in the order they are handed out
    int nitems;              // descriptors in `order`
    unsigned long long* ctr; // work counter (monotone across launches)
    unsigned long long base; // counter value at the start of this launch
};

// watchdog statistics of one field array (tf_stats.cu)
struct StatPartial {
    double sumsq;                 // sum of squares (SI units)
    double maxabs;                // largest magnitude
    unsigned long long nonfinite; // number of NaN / Inf values
};

struct Sources {
    int n;
    int comp[TF_MAX_SOURCES];
    int lo[TF_MAX_SOURCES][3];
    int hi[TF_MAX_SOURCES][3];
    float amp[TF_MAX_SOURCES];  // amp * s(t^{n+1}) of this step
    int bb_lo[3], bb_hi[3];     // bounding box of all sources
};

struct Probes {
    int n;
    int nfreq[TF_MAX_PROBES];
    int comp[TF_MAX_PROBES];
    long long q[TF_MAX_PROBES];     // padded linear index of the probe point
    long long n0[TF_MAX_PROBES];
    const double* fdt;              // [probe][TF_MAX_FREQS]: f_k dt
    double* re;                     // [probe][TF_MAX_FREQS]
    double* im;
    double* series;                 // [probe][cap]
    long long cap;
    double dt;
};

// Two steps per pass (tf_step2.cu) on the interior box of a grid: every
// point it computes lies off the walls and outside the CPML slabs and Mur
// planes, and mu is uniform.  It reads E^n, B^{n-1/2} (TMA) and Js^{n-1/2},
// writes E^{n+2}, B^{n+3/2}, Js^{n+3/2} to the next buffer, and the level
// n+1 E / n+1/2 B of the points within two of the box faces (and of probe
// points) to the third buffer, from which the single-step kernel advances
// the rest of the grid to level n+2.
constexpr int kTBLenMax = 24, kTBLenMin = 4;   // planes per two-step work item
constexpr int kTBLenDefault = 24;
struct Step2Out {
    float* E[3];             // E^{n+2}, B^{n+3/2}, Jt^{n+3/2}
    float* B[3];
    float* J[3];
    float* ZE[3];            // E^{n+1}, B^{n+1/2} of the ring and probe points
    float* ZB[3];
    const float4* tilemat;   // per (tile, plane) records of the single-step kernel
    int ntx, nty;
    int ecur, bcur;          // TMA array index of the E^n / B^{n-1/2} arrays
    int lo[3], hi[3];        // the box, [lo, hi) in points (tile aligned in x, y)
    const long long* order;  // work-item descriptors (make_item)
    int nitems;
    unsigned long long* ctr; // work counter (monotone across launches)
    unsigned long long base; // counter value at the start of this launch
    int nprobe;
    int probe[TF_MAX_PROBES][3];
    float amp2[TF_MAX_SOURCES];  // amp * s(t^{n+2}) (Sources::amp holds t^{n+1})
};
cudaError_t launch_step2(const void* tmaps2, const Params& P, const Step2Out& O, const Sources& S, int blocks,
                         cudaStream_t st);
int step2_blocks_per_sm();
// TMA views for the two-step kernel's boxes (E^n 40 x 20, B^{n-1/2} 40 x 19)
constexpr int kT2BoxX = 40, kT2BoxEY = 20, kT2BoxBY = 19;

// running DFT of probe pr at level n (Secs. 4.2, 5): X_f += s^n e^{-2 pi i f_k n dt} dt in FP64,
// for the frequency f handled by this thread, and the series sample (f = 0)
__device__ __forceinline__ void probe_update(const float* const E[3], const Probes& R, int pr, int f, long long n) {
    const double s = (double)E[R.comp[pr]][R.q[pr]];
    if (f == 0 && n < R.cap) R.series[(long long)pr * R.cap + n] = s;
    if (f < R.nfreq[pr] && n >= R.n0[pr]) {
        double ph = R.fdt[pr * TF_MAX_FREQS + f] * (double)n;
        ph -= floor(ph);
        double sn, cs;
        sincospi(2.0 * ph, &sn, &cs);
        R.re[pr * TF_MAX_FREQS + f] += s * cs * R.dt;
        R.im[pr * TF_MAX_FREQS + f] -= s * sn * R.dt;
    }
}

__host__ __device__ __forceinline__ long long lin(const Params& P, int i, int j, int k) {
    return (long long)k * P.plane + (long long)j * P.pitch + i;
}
__device__ __forceinline__ int nxt(const Params& P, int a, int p) {
    return (p + 1 < P.N[a]) ? p + 1 : (P.per[a] ? 0 : p);
}
__device__ __forceinline__ int prv(const Params& P, int a, int p) {
    return (p > 0) ? p - 1 : (P.per[a] ? P.N[a] - 1 : p);
}
// +1 when axis a follows component c cyclically, -1 otherwise (curl sign)
__host__ __device__ __forceinline__ float curl_sign(int c, int a) {
    return ((a - c + 3) % 3 == 1) ? 1.f : -1.f;
}

// E_c at point p is advanced by the curl (not outside, not on a wall)
__device__ __forceinline__ bool upd_E(const Params& P, int c, const int p[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (P.per[a]) continue;
        if (a == c) {
            if (p[a] >= P.n[a]) return false;
        } else if (p[a] < 1 || p[a] > P.n[a] - 1) {
            return false;
        }
    }
    return true;
}
// B_c at point p is advanced (normal B on a wall is not)
__device__ __forceinline__ bool upd_B(const Params& P, int c, const int p[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (P.per[a]) continue;
        if (a != c) {
            if (p[a] >= P.n[a]) return false;
        } else if (p[a] < 1 || p[a] > P.n[a] - 1) {
            return false;
        }
    }
    return true;
}
// tangential E on a Mur z wall (z = 0 or z = nz), interior along x and y
__device__ __forceinline__ bool mur_E(const Params& P, int c, const int p[3]) {
    if (P.bc[2] != TF_BC_MUR || c > 1) return false;
    if (p[2] != 0 && p[2] != P.n[2]) return false;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        if (P.per[a]) continue;
        if (a == c) {
            if (p[a] >= P.n[a]) return false;
        } else if (p[a] < 1 || p[a] > P.n[a] - 1) {
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ bool in_slab(const Params& P, int a, int p) {
    return P.L[a] > 0 && (p < P.L[a] || p >= P.n[a] - P.L[a]);
}

// edge material of E_c at p: eps (mean of 4 cells), st and kt per edge rule
__device__ __forceinline__ void edge_material(const Params& P, int c, const int p[3], float& eps,
                                              float& st, float& kt) {
    const int b1 = (c + 1) % 3, b2 = (c + 2) % 3;
    float se = 0.f, ss = 0.f, sk = 0.f;
    int ns = 0, nk = 0;
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            int cc[3];
            cc[c] = p[c];
            cc[b1] = u ? prv(P, b1, p[b1]) : p[b1];
            cc[b2] = v ? prv(P, b2, p[b2]) : p[b2];
            const long long m = lin(P, cc[0], cc[1], cc[2]);
            const float e = __ldg(P.eps + m), s = __ldg(P.sig + m), k = __ldg(P.kap + m);
            se += e;
            ss += s;
            sk += k;
            ns += s > 0.f;
            nk += k > 0.f;
        }
    eps = 0.25f * se;
    if (P.edge_rule == TF_EDGE_PLAIN_MEAN) {
        st = 0.25f * ss;
        kt = 0.25f * sk;
    } else {
        st = ns ? ss / (float)ns : 0.f;
        kt = nk ? sk / (float)nk : 0.f;
    }
}

// 1 / mu_f of face B_c at p (mean mu_r of the two cells across the face)
__device__ __forceinline__ float inv_mu_face(const Params& P, int c, const int p[3]) {
    if (P.uniform_mu) return 1.f;
    int q[3] = {p[0], p[1], p[2]};
    q[c] = prv(P, c, p[c]);
    const float m0 = __ldg(P.mu + lin(P, p[0], p[1], p[2]));
    const float m1 = __ldg(P.mu + lin(P, q[0], q[1], q[2]));
    return 2.f / (m0 + m1);
}

// TMA views of the single-step kernel: E box, B box, psi_B box
struct TMaps {
    CUtensorMap e, b, pb;
};

// Batched stepping (tf_batch_run): one launch of the single-step kernel per
// step over every grid of a batch.  Per grid, in global memory (written by
// the host before the run):
struct __align__(128) BatchGrid {
    TMaps tm;
    Params P[2];        // the step from the current buffer (index 0) and from the next one (index 1)
    StepOut O[2];
    Sources S;          // amplitudes come from `amp`
    Probes R;
    const float* amp;   // [step][source]: amp * s(t^{n+1}) of each step of the run
    long long level0;   // level at step 0 of the run
};
// the launch: one work list over all grids (descriptor bits 48-62: the
// grid's index), its counter, and the (grid, probe) pairs sampled per step
struct BatchLaunch {
    const BatchGrid* G;
    int ngrids;
    const int* step;                  // the step number (device), advanced after each launch
    const long long* order;
    int nitems;
    unsigned long long* ctr;
    unsigned long long base0, base_inc;   // counter value at step 0, advance per step
    const int* probes;                // nprobes pairs (grid, probe)
    int nprobes;
};
__host__ __device__ __forceinline__ long long item_with_grid(long long d, int grid) {
    return d | (long long)grid << 48;
}
cudaError_t launch_step_batch(const BatchLaunch& BL, int blocks, cudaStream_t st);
cudaError_t launch_step_advance(int* step, cudaStream_t st);

// launchers (tf_kernels.cu)
cudaError_t launch_convert_materials(const Params& P, const float* eps_r, const float* mu_r,
                                     const float* lam, const float* sigma, double dt,
                                     float* eps, float* sig, float* kap, float* mu,
                                     unsigned* minmax, cudaStream_t st);
cudaError_t launch_set_field(const Params& P, int comp, const float* dense, float* dst, double scale,
                             cudaStream_t st);
cudaError_t launch_prime(const Params& P, cudaStream_t st);
cudaError_t launch_mask_js(const Params& P, cudaStream_t st);
cudaError_t launch_read_field(const Params& P, int comp, int primed, float* dense, double scale,
                              cudaStream_t st);
// 4-D TMA view (x, y, z, array index) of `narrays` equally spaced arrays with
// a box of bx x by x 1 x bf; writes a 128-byte CUtensorMap to out128
cudaError_t make_tensor_map(void* base, const int N[3], int pitch, size_t array_bytes, int narrays, int bx,
                            int by, int bf, void* out128);
// tmaps: three consecutive 128-byte maps -- E box, B box, psi_B box
// one fused step from level n; the step also adds E^n at the probe points to
// their running DFTs and series
cudaError_t launch_step(const void* tmaps, const Params& P, const StepOut& O, const Sources& S, const Probes& R,
                        long long n, int blocks, cudaStream_t st);
cudaError_t launch_edge_coeffs(const Params& P, cudaStream_t st);
size_t step_smem_bytes();
cudaError_t launch_tile_materials(const Params& P, float4* tilemat, int ntx, int nty, cudaStream_t st);
// discrete adjoint (tf_adjoint.cu): the adjoint state, in the scaled units of
// the step, and per-edge gradient sums (FP64)
struct AdjState {
    float* E[3];
    float* B[3];
    float* J[3];
    float* psiB[3][3];   // [component][axis], nullptr without CPML on the axis
    float* psiE[3][3];
    double* gE[3];       // dJ / d eps_r,e
    double* gK[3];       // dJ / d kt_e
    float* W[3][3];      // edge weights [e][a] (a != e) the face pass differences
    float* U[3][3];      // face weights [c][a] (a != c) the edge pass differences
};
struct AdjStep {
    const float* En[3];    // E^n
    const float* En1[3];   // E^{n+1} (with this step's soft sources)
    int probe_comp;        // the objective's derivative dJ/dE^n at the probe point
    long long probe_q;
    float probe_src;
};
cudaError_t launch_adjoint_step(const Params& P, const AdjState& A, const Sources& S, const AdjStep& st,
                                const float4* tilemat, int ntx, cudaStream_t stream);
// copy three float arrays of n elements (n a multiple of 4, 16-byte aligned)
cudaError_t launch_copy3(float* const dst[3], float* const src[3], long long n, cudaStream_t stream);
cudaError_t launch_adjoint_cells(const Params& P, const AdjState& A, float dt_c0, double unscale, float* g_eps,
                                 float* g_lam, cudaStream_t stream);

// order in which k_step hands out its work items (items needing the full plane loop first)
cudaError_t launch_item_order(const Params& P, const StepOut& O, const Sources& S, int split, int tail, int chunk,
                              long long* order,
                              int* count, cudaStream_t st);
int step_blocks_per_sm();
cudaError_t launch_field_stats(const float* f, int n0, int n1, int n2, int pitch, long long plane, double scale,
                               StatPartial* partials, StatPartial* out, cudaStream_t st);
cudaError_t launch_fit_q(const double* re, const double* im, const double* fdt, int nfreq,
                         double dt, long long n0, long long N, double f_guess, double q_guess,
                         double* out, cudaStream_t st);

}  // namespace tf
