// tf_api.cu -- the C ABI of include/twofluid.h: descriptor validation,
// workspace carving, coefficient set-up and the per-step launch sequence.
// All GPU work runs in the kernels of tf_kernels.cu / tf_fit.cu.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "tf_internal.cuh"

using namespace tf;

namespace {

constexpr size_t kAlign = 256;

inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct Layout {
    int N[3], pitch;
    long long total;        // floats per field array (padded)
    long long ncell, ndense;
    int ncpml_axes;         // axes with a CPML (6 psi arrays each)
    int ntx, nty, nch, kend; // fused-step tiles, z chunks, planes iterated
    size_t off_fields, off_maps, off_psi, off_prof, off_zero, off_probe, off_series, off_scratch,
        off_tiles, off_order, off_order_s, off_order_t, off_stats, off_coef, off_misc, bytes;
    long long max_s, max_t;   // capacity of the shell and two-step work lists
    long long scratch_floats;
};

double dt_of(const tf_grid_desc* d) {
    if (d->dt > 0) return d->dt;
    return d->courant / (kC0 * sqrt(1.0 / (d->dx * d->dx) + 1.0 / (d->dy * d->dy) + 1.0 / (d->dz * d->dz)));
}

tf_status validate(const tf_grid_desc* d) {
    if (!d) return TF_EINVAL;
    const int n[3] = {d->nx, d->ny, d->nz};
    const double h[3] = {d->dx, d->dy, d->dz};
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 1 || !(h[a] > 0) || !isfinite(h[a])) return TF_EINVAL;
        const tf_bc& b = d->bc[a];
        if (b.kind < TF_BC_PERIODIC || b.kind > TF_BC_CPML) return TF_EINVAL;
        if (b.kind == TF_BC_MUR && a != 2) return TF_ENOTSUP;
        if (b.kind == TF_BC_MUR && n[a] < 2) return TF_EINVAL;
        if (b.kind == TF_BC_CPML) {
            if (b.cpml_cells < 1 || 2 * b.cpml_cells > n[a]) return TF_EINVAL;
            if (!(b.cpml_order >= 0) || !(b.cpml_sigma_max >= 0) || !(b.cpml_alpha_max >= 0)) return TF_EINVAL;
        }
    }
    if (!(d->dt > 0) && !(d->courant > 0)) return TF_EINVAL;
    if (!(d->theta >= 0.5 && d->theta <= 1.0)) return TF_EINVAL;
    if (d->edge_rule != TF_EDGE_CONDUCTOR_MEAN && d->edge_rule != TF_EDGE_PLAIN_MEAN) return TF_EINVAL;
    if (d->max_probes < 0 || d->max_probes > TF_MAX_PROBES || d->series_capacity < 0) return TF_EINVAL;
    const long long pts = (long long)(n[0] + 1) * (n[1] + 1) * (n[2] + 1);
    if (pts > (1LL << 40)) return TF_EINVAL;
    // work-item descriptors hold 20 bits of tile index and 20 bits of plane
    const long long tx = (n[0] + 1 + kSX - 1) / kSX, ty = (n[1] + 1 + kSY - 1) / kSY;
    if (tx * ty > kMaxTiles || n[2] + 1 > kMaxPlanes) return TF_ENOTSUP;
    return TF_OK;
}

Layout layout_of(const tf_grid_desc* d) {
    Layout L{};
    const int n[3] = {d->nx, d->ny, d->nz};
    for (int a = 0; a < 3; ++a) L.N[a] = n[a] + (d->bc[a].kind == TF_BC_PERIODIC ? 0 : 1);
    L.pitch = (L.N[0] + 1 + 31) / 32 * 32;   // a spare column past the x end
    L.total = (long long)L.pitch * L.N[1] * L.N[2];
    L.ncell = (long long)n[0] * n[1] * n[2];
    L.ndense = (long long)L.N[0] * L.N[1] * L.N[2];
    L.ncpml_axes = 0;
    for (int a = 0; a < 3; ++a)
        if (d->bc[a].kind == TF_BC_CPML) L.ncpml_axes += 1;
    // tiles cover the cells of a walled axis (its wall plane never changes)
    // and every point of a periodic one
    const int cx = d->bc[0].kind == TF_BC_PERIODIC ? L.N[0] : n[0];
    const int cy = d->bc[1].kind == TF_BC_PERIODIC ? L.N[1] : n[1];
    L.ntx = (cx + kSX - 1) / kSX;
    L.nty = (cy + kSY - 1) / kSY;
    L.kend = d->bc[2].kind == TF_BC_PERIODIC ? L.N[2] : L.N[2] - 1;
    L.nch = (L.kend + kChunk - 1) / kChunk;
    const size_t fbytes = align_up(sizeof(float) * (size_t)L.total);
    size_t o = 0;
    L.off_fields = o; o += kFieldArrays * fbytes;   // E, B, Js in three buffers
    L.off_maps = o;   o += 4 * fbytes;
    L.off_psi = o;    o += kPsiGroup * (size_t)L.ncpml_axes * fbytes;   // per axis: psi_B pair x 3 buffers, psi_E pair
    L.off_coef = o;   o += 9 * fbytes;                             // per-point ca, cb, cj of each E component
    L.off_prof = o;
    for (int a = 0; a < 3; ++a) o += 4 * align_up(sizeof(float) * (size_t)L.N[a]);
    L.off_zero = o;
    L.off_probe = o;  o += 3 * align_up(sizeof(double) * TF_MAX_PROBES * TF_MAX_FREQS);
    L.off_series = o; o += align_up(sizeof(double) * (size_t)d->max_probes * (size_t)d->series_capacity);
    L.scratch_floats = 4 * L.ncell > L.ndense ? 4 * L.ncell : L.ndense;
    L.off_scratch = o; o += align_up(sizeof(float) * (size_t)L.scratch_floats);
    L.off_tiles = o;  o += align_up(sizeof(float4) * (size_t)L.ntx * L.nty * L.N[2]);
    L.off_order = o;  o += align_up(sizeof(long long) * (size_t)L.ntx * L.nty * L.nch * ((kChunk + kSub - 1) / kSub));
    // shell list: the chunks of every tile, two more per tile where the
    // two-step box cuts them, each chunk in pieces at most
    L.max_s = (long long)L.ntx * L.nty * (L.nch + 2) * ((kChunk + kSub - 1) / kSub);
    L.off_order_s = o; o += align_up(sizeof(long long) * (size_t)L.max_s);
    // box list: its tiles in items of at least kTBLenMin planes
    L.max_t = (long long)L.ntx * L.nty * (L.N[2] / kTBLenMin + 1);
    L.off_order_t = o; o += align_up(sizeof(long long) * (size_t)L.max_t);
    L.off_stats = o;  o += align_up(sizeof(StatPartial) * (size_t)(L.N[2] + 1));
    L.off_misc = o;   o += kAlign;
    L.bytes = o;
    return L;
}

struct SrcHost {
    int comp, lo[3], hi[3], kind;
    double amp, f, t0, tw;
};

double waveform(const SrcHost& s, double t) {
    const double env = exp(-(t - s.t0) * (t - s.t0) / (2.0 * s.tw * s.tw));
    const double two_pi = 6.283185307179586476925286766559;
    switch (s.kind) {
        case TF_SRC_GAUSS: return env;
        case TF_SRC_SIN: return sin(two_pi * s.f * t);
        default: return env * sin(two_pi * s.f * t);
    }
}

}  // namespace

struct tf_ctx {
    // TMA descriptors: the single-step E box, B box and psi_B box; the two-step E box and B box
    alignas(128) unsigned char tmap[5][128];
    tf_grid_desc desc;
    Layout L;
    Params P;           // the current state (buffer cur) ...
    StepOut O;          // ... and the next one (buffer nxt): the single-step launch
    float* fE[kFieldBuffers][3];   // the field arrays of each buffer
    float* fB[kFieldBuffers][3];
    float* fJ[kFieldBuffers][3];
    float* fPB[kFieldBuffers][3][3];   // psi_B [buffer][component][axis]
    int cur, nxt;       // buffers of the current and the next state (the third one is scratch)
    int step_blocks;
    int slots, slots2;  // resident CTAs of the single- and two-step kernels on the device
    // two-step passes: the interior box (tiles [tx0, tx1) x [ty0, ty1), planes [tz0, tz1))
    int box_ok;         // the geometry has a box (two-step passes also need uniform mu)
    int tx0, tx1, ty0, ty1, tz0, tz1;
    int nitems_s, blocks_s, nitems_t, blocks_t;
    unsigned long long* ctr_t;
    unsigned long long base_t;
    int two_step_on;    // two-step passes allowed (tf_set_two_step; on by default)
    int item_planes;    // planes per single-step work item (tf_set_item_planes)
    int tb_len;         // planes per two-step work item
    int ppos[TF_MAX_PROBES][3];   // probe points (storage coordinates)
    Probes R;
    cudaStream_t stream;
    double dt;
    long long level;
    int primed;
    int order_dirty;   // the work-item order must be rebuilt before the next step
    int fine;          // fewer items than CTA slots: every item goes out in pieces
    char* ws;
    float* scratch;
    unsigned* status;
    unsigned* mm;      // 4 words: max 1/(eps mu), max kt/(4 eps), non-uniform mu, spare
    double* fit_out;   // 4 doubles
    int nsrc;
    SrcHost src[TF_MAX_SOURCES];
    double freqs[TF_MAX_PROBES][TF_MAX_FREQS];
};

namespace {

// Params / StepOut of a step from buffer `from` to buffer `to`
void bind(const tf_ctx* h, int from, int to, Params& P, StepOut& O) {
    for (int c = 0; c < 3; ++c) {
        P.E[c] = h->fE[from][c];
        P.B[c] = h->fB[from][c];
        P.J[c] = h->fJ[from][c];
        O.E[c] = h->fE[to][c];
        O.B[c] = h->fB[to][c];
        O.J[c] = h->fJ[to][c];
        for (int a = 0; a < 3; ++a) {
            P.psiB[c][a] = h->fPB[from][c][a];
            O.psiB[c][a] = h->fPB[to][c][a];
        }
    }
    O.ecur = 9 * from;
    O.bcur = 9 * from + 3;
    O.psib_cur = psib_index(from);
}

// the counter of a work list moved once per item past the 2G handed out by
// position, and once more (the fetch that came back empty) in every CTA that
// had a second item
unsigned long long counter_advance(long long ni, long long g) {
    return (unsigned long long)((ni > 2 * g ? ni - 2 * g : 0) + (ni - g < 0 ? 0 : ni - g > g ? g : ni - g));
}

// The interior box of the two-step kernel.  Every point that kernel forms
// (its tiles plus a two-point halo: x0-2 .. x0+33, y0-2 .. y0+16, planes
// kz0-2 .. kz1) must lie off the walls and off the Mur planes (points 2 ..
// n-2 of a walled axis) and outside the CPML slabs (cells L .. n-L-1); on a
// periodic axis its TMA boxes (x0-4 .. x0+35, y0-2 .. y0+17, planes kz0-2 ..
// kz1+1) must not wrap.  Tiles are those of the single-step kernel.
void interior_box(tf_ctx* h) {
    const Params& P = h->P;
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        if (P.per[a]) {
            lo[a] = 0;
            hi[a] = P.N[a];
        } else {
            lo[a] = P.L[a] > 2 ? P.L[a] : 2;
            hi[a] = P.n[a] - (P.L[a] > 1 ? P.L[a] : 1);
        }
    }
    // x: x0 - 2 >= lo (periodic: x0 - 4 >= 0), x0 + 34 <= hi (periodic: x0 + 36 <= N)
    const int xl = P.per[0] ? 4 : lo[0] + 2, xh = P.per[0] ? hi[0] - 36 : hi[0] - 34;
    h->tx0 = (xl + kSX - 1) / kSX;
    h->tx1 = xh >= 0 ? xh / kSX + 1 : 0;
    // y: y0 - 2 >= lo, y0 + 17 <= hi (periodic: y0 + 18 <= N)
    const int yl = lo[1] + 2, yh = P.per[1] ? hi[1] - 18 : hi[1] - 17;
    h->ty0 = (yl + kSY - 1) / kSY;
    h->ty1 = yh >= 0 ? yh / kSY + 1 : 0;
    // z: kz0 - 2 >= lo, kz1 + 1 <= hi (periodic: kz1 + 2 <= N)
    h->tz0 = lo[2] + 2;
    h->tz1 = P.per[2] ? hi[2] - 2 : hi[2] - 1;
    if (h->tx1 > h->L.ntx) h->tx1 = h->L.ntx;
    if (h->ty1 > h->L.nty) h->ty1 = h->L.nty;
    h->box_ok = h->tx1 > h->tx0 && h->ty1 > h->ty0 && h->tz1 - h->tz0 >= 4;
    if (!h->box_ok) h->tx0 = h->tx1 = h->ty0 = h->ty1 = h->tz0 = h->tz1 = 0;
}

}  // namespace

#define TF_CUDA(x)                                  \
    do {                                            \
        if ((x) != cudaSuccess) return TF_ECUDA;    \
    } while (0)

extern "C" {

const char* tf_strerror(tf_status s) {
    switch (s) {
        case TF_OK: return "ok";
        case TF_EINVAL: return "invalid argument";
        case TF_ENOMEM: return "workspace too small";
        case TF_ECUDA: return "CUDA error";
        case TF_EUNSTABLE: return "time step violates the stability bound";
        case TF_ESTATE: return "call not allowed in this state";
        case TF_ETIMEOUT: return "device wait timed out";
        case TF_ENONFINITE: return "non-finite field value";
        case TF_ENOTSUP: return "not supported";
    }
    return "unknown status";
}

size_t tf_workspace_size(const tf_grid_desc* desc) {
    if (validate(desc) != TF_OK) return 0;
    return layout_of(desc).bytes;
}

static void cpml_profile(const tf_grid_desc* d, int a, double dt, double x, double r, float* b, float* c) {
    const int n[3] = {d->nx, d->ny, d->nz};
    const tf_bc& bc = d->bc[a];
    const double L = bc.cpml_cells;
    double rho = 0.0;
    if (x < L) rho = (L - x) / L;
    else if (x > n[a] - L) rho = (x - (n[a] - L)) / L;
    if (rho <= 0.0) { *b = 0.f; *c = 0.f; return; }
    const double s = bc.cpml_sigma_max * pow(rho, bc.cpml_order);
    const double al = bc.cpml_alpha_max * (1.0 - rho);
    const double bb = exp(-(s + al) * dt / kEps0);
    const double cc = (s + al > 0.0) ? s * (bb - 1.0) / (s + al) : 0.0;
    *b = (float)bb;
    *c = (float)(cc * r);   // folded with r_a = c0 dt / d_a (scaled units)
}

tf_status tf_create(const tf_grid_desc* desc, void* dev_workspace, size_t bytes, tf_handle* out) {
    if (!out || !dev_workspace) return TF_EINVAL;
    *out = nullptr;
    tf_status v = validate(desc);
    if (v != TF_OK) return v;
    if (((uintptr_t)dev_workspace) % kAlign) return TF_EINVAL;
    const Layout L = layout_of(desc);
    if (bytes < L.bytes) return TF_ENOMEM;
    const double dt = dt_of(desc);
    const double cour = kC0 * dt * sqrt(1.0 / (desc->dx * desc->dx) + 1.0 / (desc->dy * desc->dy) +
                                        1.0 / (desc->dz * desc->dz));
    if (!(cour <= 1.0)) return TF_EUNSTABLE;

    tf_ctx* h = new (std::nothrow) tf_ctx();
    if (!h) return TF_ENOMEM;
    h->desc = *desc;
    h->L = L;
    h->dt = dt;
    h->stream = (cudaStream_t)desc->stream;
    h->ws = (char*)dev_workspace;
    Params& P = h->P;
    const int n[3] = {desc->nx, desc->ny, desc->nz};
    const double dd[3] = {desc->dx, desc->dy, desc->dz};
    for (int a = 0; a < 3; ++a) {
        P.N[a] = L.N[a];
        P.n[a] = n[a];
        P.bc[a] = desc->bc[a].kind;
        P.per[a] = desc->bc[a].kind == TF_BC_PERIODIC;
        P.L[a] = desc->bc[a].kind == TF_BC_CPML ? desc->bc[a].cpml_cells : 0;
        P.r[a] = (float)(kC0 * dt / dd[a]);
    }
    P.pitch = L.pitch;
    P.plane = (long long)L.pitch * L.N[1];
    P.theta = (float)desc->theta;
    P.edge_rule = desc->edge_rule;
    P.uniform_mu = 1;
    P.mur_M = (float)((kC0 * dt - desc->dz) / (kC0 * dt + desc->dz));
    const size_t fbytes = align_up(sizeof(float) * (size_t)L.total);
    char* base = h->ws;
    StepOut& O = h->O;
    for (int b = 0; b < kFieldBuffers; ++b)
        for (int c = 0; c < 3; ++c) {
            h->fE[b][c] = (float*)(base + L.off_fields + (size_t)(9 * b + c) * fbytes);
            h->fB[b][c] = (float*)(base + L.off_fields + (size_t)(9 * b + 3 + c) * fbytes);
            h->fJ[b][c] = (float*)(base + L.off_fields + (size_t)(9 * b + 6 + c) * fbytes);
            for (int a = 0; a < 3; ++a) h->fPB[b][c][a] = nullptr;
        }
    float* maps[4];
    for (int m = 0; m < 4; ++m) maps[m] = (float*)(base + L.off_maps + m * fbytes);
    P.eps = maps[0]; P.sig = maps[1]; P.kap = maps[2]; P.mu = maps[3];
    // psi arrays: per CPML axis a (slot s), with c1 < c2 the two components != a:
    //   [psiB(c1) buf0, psiB(c2) buf0, psiB(c1) buf1, psiB(c2) buf1, psiE(c1), psiE(c2),
    //    psiB(c1) buf2, psiB(c2) buf2]
    int slot = 0;
    for (int a = 0; a < 3; ++a) {
        O.psi_slot[a] = -1;
        for (int c = 0; c < 3; ++c) P.psiE[c][a] = nullptr;
        if (desc->bc[a].kind != TF_BC_CPML) continue;
        O.psi_slot[a] = slot;
        int m = 0;
        for (int c = 0; c < 3; ++c) {
            if (c == a) continue;
            char* g0 = base + L.off_psi + (size_t)(kPsiGroup * slot) * fbytes;
            for (int b = 0; b < kFieldBuffers; ++b) h->fPB[b][c][a] = (float*)(g0 + (size_t)(psib_index(b) + m) * fbytes);
            P.psiE[c][a] = (float*)(g0 + (size_t)(4 + m) * fbytes);
            ++m;
        }
        ++slot;
    }
    for (int c = 0; c < 3; ++c) {
        P.ca[c] = (const float*)(base + L.off_coef + (size_t)(0 + c) * fbytes);
        P.cb[c] = (const float*)(base + L.off_coef + (size_t)(3 + c) * fbytes);
        P.cj[c] = (const float*)(base + L.off_coef + (size_t)(6 + c) * fbytes);
    }
    h->cur = 0;
    h->nxt = 1;
    bind(h, h->cur, h->nxt, P, O);
    if ((long long)P.plane * L.N[2] >= (1LL << 31)) { delete h; return TF_ENOTSUP; }   // 32-bit indexing
    if (make_tensor_map(base + L.off_fields, L.N, L.pitch, fbytes, kFieldArrays, kEX, kEY, 3, h->tmap[0]) !=
            cudaSuccess ||
        make_tensor_map(base + L.off_fields, L.N, L.pitch, fbytes, kFieldArrays, kBX, kBY, 3, h->tmap[1]) !=
            cudaSuccess ||
        make_tensor_map(base + L.off_fields, L.N, L.pitch, fbytes, kFieldArrays, kT2BoxX, kT2BoxEY, 3,
                        h->tmap[3]) != cudaSuccess ||
        make_tensor_map(base + L.off_fields, L.N, L.pitch, fbytes, kFieldArrays, kT2BoxX, kT2BoxBY, 3,
                        h->tmap[4]) != cudaSuccess) {
        delete h;
        return TF_ECUDA;
    }
    if (L.ncpml_axes > 0 && make_tensor_map(base + L.off_psi, L.N, L.pitch, fbytes, kPsiGroup * L.ncpml_axes, kBX,
                                            kBY, 2, h->tmap[2]) != cudaSuccess) {
        delete h;
        return TF_ECUDA;
    }
    interior_box(h);
    O.tilemat = (const float4*)(base + L.off_tiles);
    O.order = (const long long*)(base + L.off_order);
    h->order_dirty = 1;
    O.ntx = L.ntx;
    O.nty = L.nty;
    O.nch = L.nch;
    O.kend = L.kend;
    O.base = 0;
    size_t o = L.off_prof;
    float* prof_host = (float*)malloc(sizeof(float) * 4 * (size_t)(L.N[0] + L.N[1] + L.N[2] + 3));
    if (!prof_host) { delete h; return TF_ENOMEM; }
    for (int a = 0; a < 3; ++a) {
        const size_t pb = align_up(sizeof(float) * (size_t)L.N[a]);
        float* d[4];
        for (int m = 0; m < 4; ++m) d[m] = (float*)(base + o + m * pb);
        o += 4 * pb;
        P.pbE[a] = d[0]; P.pcE[a] = d[1]; P.pbB[a] = d[2]; P.pcB[a] = d[3];
        float* hb = prof_host;
        for (int p = 0; p < L.N[a]; ++p) {
            if (desc->bc[a].kind == TF_BC_CPML) {
                cpml_profile(desc, a, dt, (double)p, P.r[a], &hb[p], &hb[L.N[a] + p]);
                cpml_profile(desc, a, dt, p + 0.5, P.r[a], &hb[2 * L.N[a] + p], &hb[3 * L.N[a] + p]);
            } else {
                hb[p] = hb[L.N[a] + p] = hb[2 * L.N[a] + p] = hb[3 * L.N[a] + p] = 0.f;
            }
        }
        for (int m = 0; m < 4; ++m)
            if (cudaMemcpyAsync(d[m], hb + m * L.N[a], sizeof(float) * L.N[a], cudaMemcpyHostToDevice,
                                h->stream) != cudaSuccess) {
                free(prof_host);
                delete h;
                return TF_ECUDA;
            }
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) { free(prof_host); delete h; return TF_ECUDA; }
    }
    free(prof_host);
    const size_t pbytes = align_up(sizeof(double) * TF_MAX_PROBES * TF_MAX_FREQS);
    h->R.fdt = (const double*)(base + L.off_probe);
    h->R.re = (double*)(base + L.off_probe + pbytes);
    h->R.im = (double*)(base + L.off_probe + 2 * pbytes);
    h->R.series = desc->series_capacity > 0 ? (double*)(base + L.off_series) : nullptr;
    h->R.cap = desc->series_capacity;
    h->R.dt = dt;
    h->R.n = 0;
    h->scratch = (float*)(base + L.off_scratch);
    h->status = (unsigned*)(base + L.off_misc);
    h->mm = h->status + 4;
    h->fit_out = (double*)(base + L.off_misc + 64);
    O.ctr = (unsigned long long*)(base + L.off_misc + 128);
    h->ctr_t = (unsigned long long*)(base + L.off_misc + 160);
    h->base_t = 0;
    h->two_step_on = 1;
    h->tb_len = kTBLenDefault;
    h->item_planes = kChunk;
    P.status = h->status;
    P.wait_polls = kSpinLimit;
    {
        int dev = 0, sms = 1;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            delete h;
            return TF_ECUDA;
        }
        const long long items = (long long)L.ntx * L.nty * L.nch;
        const int per_sm = step_blocks_per_sm(), per_sm2 = step2_blocks_per_sm();
        if (per_sm < 1 || per_sm2 < 1) {
            delete h;
            return TF_ECUDA;
        }
        // one resident CTA per slot (no more than the units of work).  A grid
        // with fewer items than slots goes out in kSub-plane pieces.
        const long long slots = (long long)sms * per_sm;
        h->slots = (int)slots;
        h->slots2 = sms * per_sm2;
        h->fine = items < slots;
        const long long units = h->fine ? items * ((kChunk + kSub - 1) / kSub) : items;
        const long long nb = units < slots ? units : slots;
        h->step_blocks = (int)(nb > 0 ? nb : 1);
    }
    // zero everything but the profiles, then vacuum materials
    cudaError_t e = cudaMemsetAsync(base + L.off_fields, 0, L.off_prof - L.off_fields, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + L.off_zero, 0, L.off_misc + kAlign - L.off_zero, h->stream);
    if (e == cudaSuccess)
        e = launch_convert_materials(P, nullptr, nullptr, nullptr, nullptr, dt, maps[0], maps[1], maps[2],
                                     maps[3], h->mm, h->stream);
    if (e == cudaSuccess) e = launch_tile_materials(P, (float4*)O.tilemat, L.ntx, L.nty, h->stream);
    if (e == cudaSuccess) e = launch_edge_coeffs(P, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) { delete h; return TF_ECUDA; }
    *out = h;
    return TF_OK;
}

tf_status tf_destroy(tf_handle h) {
    if (!h) return TF_EINVAL;
    cudaStreamSynchronize(h->stream);
    delete h;
    return TF_OK;
}

tf_status tf_storage_dims(tf_handle h, int dims[3]) {
    if (!h || !dims) return TF_EINVAL;
    for (int a = 0; a < 3; ++a) dims[a] = h->L.N[a];
    return TF_OK;
}

tf_status tf_get_time(tf_handle h, int64_t* n, double* t) {
    if (!h) return TF_EINVAL;
    if (n) *n = h->level;
    if (t) *t = h->level * h->dt;
    return TF_OK;
}

tf_status tf_get_dt(tf_handle h, double* dt) {
    if (!h || !dt) return TF_EINVAL;
    *dt = h->dt;
    return TF_OK;
}

tf_status tf_set_materials(tf_handle h, const float* eps_r, const float* mu_r, const float* lambda_L,
                           const float* sigma, int on_device) {
    if (!h) return TF_EINVAL;
    if (h->level != 0 || h->primed) return TF_ESTATE;
    const long long nc = h->L.ncell;
    const float* src[4] = {eps_r, mu_r, lambda_L, sigma};
    const float* dev[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int m = 0; m < 4; ++m) {
        if (!src[m]) continue;
        if (on_device) {
            dev[m] = src[m];
        } else {
            float* st = h->scratch + m * nc;
            TF_CUDA(cudaMemcpyAsync(st, src[m], sizeof(float) * nc, cudaMemcpyHostToDevice, h->stream));
            dev[m] = st;
        }
    }
    Params& P = h->P;
    TF_CUDA(cudaMemsetAsync(h->mm, 0, 4 * sizeof(unsigned), h->stream));
    TF_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    TF_CUDA(launch_convert_materials(P, dev[0], dev[1], dev[2], dev[3], h->dt, (float*)P.eps, (float*)P.sig,
                                     (float*)P.kap, (float*)P.mu, h->mm, h->stream));
    TF_CUDA(launch_tile_materials(P, (float4*)h->O.tilemat, h->L.ntx, h->L.nty, h->stream));
    h->order_dirty = 1;
    TF_CUDA(launch_edge_coeffs(P, h->stream));
    TF_CUDA(launch_mask_js(P, h->stream));
    unsigned hm[4], st = 0;
    TF_CUDA(cudaMemcpyAsync(hm, h->mm, sizeof(hm), cudaMemcpyDeviceToHost, h->stream));
    TF_CUDA(cudaMemcpyAsync(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
    TF_CUDA(cudaStreamSynchronize(h->stream));
    TF_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    P.uniform_mu = hm[2] ? 0 : 1;
    if (st & kStatusBadMaterial) return TF_EINVAL;
    float inv_eu, lon;
    memcpy(&inv_eu, &hm[0], 4);
    memcpy(&lon, &hm[1], 4);
    const tf_grid_desc* d = &h->desc;
    const double c2 = pow(kC0 * h->dt, 2) * (1.0 / (d->dx * d->dx) + 1.0 / (d->dy * d->dy) + 1.0 / (d->dz * d->dz));
    if (c2 * inv_eu + lon > 1.0 + 1e-12) return TF_EUNSTABLE;
    return TF_OK;
}

tf_status tf_set_field(tf_handle h, int comp, const float* src, int on_device) {
    if (!h || !src || comp < 0 || comp > 8) return TF_EINVAL;
    if (h->level != 0 || h->primed) return TF_ESTATE;
    const float* dense = src;
    if (!on_device) {
        TF_CUDA(cudaMemcpyAsync(h->scratch, src, sizeof(float) * h->L.ndense, cudaMemcpyHostToDevice, h->stream));
        dense = h->scratch;
    }
    float* dst = comp < 3 ? h->P.E[comp] : comp < 6 ? h->P.B[comp - 3] : h->P.J[comp - 6];
    const double scale = comp < 3 ? 1.0 : comp < 6 ? kC0 : h->dt / kEps0;
    TF_CUDA(launch_set_field(h->P, comp, dense, dst, scale, h->stream));
    if (!on_device) TF_CUDA(cudaStreamSynchronize(h->stream));   // host buffer may be reused
    return TF_OK;
}

tf_status tf_add_source(tf_handle h, int comp, const int lo[3], const int hi[3], double amp, int kind,
                        double f, double t0, double tw, int* id) {
    if (!h || !lo || !hi || comp < 0 || comp > 2 || kind < TF_SRC_GAUSS || kind > TF_SRC_GAUSS_SIN)
        return TF_EINVAL;
    if (h->nsrc >= TF_MAX_SOURCES) return TF_EINVAL;
    if (kind != TF_SRC_SIN && !(tw > 0)) return TF_EINVAL;
    SrcHost& s = h->src[h->nsrc];
    s.comp = comp;
    for (int a = 0; a < 3; ++a) {
        s.lo[a] = lo[a] < 0 ? 0 : lo[a];
        s.hi[a] = hi[a] > h->L.N[a] ? h->L.N[a] : hi[a];
    }
    s.kind = kind; s.amp = amp; s.f = f; s.t0 = t0; s.tw = tw;
    if (id) *id = h->nsrc;
    h->nsrc++;
    h->order_dirty = 1;
    return TF_OK;
}

tf_status tf_add_probe(tf_handle h, int comp, const int p[3], const double* freqs, int nfreq, int64_t n0,
                       int* id) {
    if (!h || !p || comp < 0 || comp > 2 || nfreq < 0 || nfreq > TF_MAX_FREQS || (nfreq && !freqs))
        return TF_EINVAL;
    if (h->R.n >= h->desc.max_probes) return TF_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (p[a] < 0 || p[a] >= h->L.N[a]) return TF_EINVAL;
    const int k = h->R.n;
    double fdt[TF_MAX_FREQS] = {0};
    for (int f = 0; f < nfreq; ++f) {
        h->freqs[k][f] = freqs[f];
        fdt[f] = freqs[f] * h->dt;
    }
    TF_CUDA(cudaMemcpyAsync((double*)h->R.fdt + k * TF_MAX_FREQS, fdt, sizeof(fdt), cudaMemcpyHostToDevice,
                            h->stream));
    TF_CUDA(cudaStreamSynchronize(h->stream));
    h->R.nfreq[k] = nfreq;
    h->R.comp[k] = comp;
    h->R.q[k] = lin(h->P, p[0], p[1], p[2]);
    for (int a = 0; a < 3; ++a) h->ppos[k][a] = p[a];
    h->R.n0[k] = n0;
    h->R.n++;
    if (id) *id = k;
    return TF_OK;
}

namespace {

// per-step launch sequence (fused step with the probe DFT of E^n, buffer
// swap); with `ev` non-null events are recorded before and after the launch
cudaError_t launch_one_step(tf_ctx* h, Sources& S, cudaEvent_t* ev) {
    cudaStream_t st = h->stream;
    const double t1 = (double)(h->level + 1) * h->dt;
    for (int q = 0; q < h->nsrc; ++q) S.amp[q] = (float)(h->src[q].amp * waveform(h->src[q], t1));
    if (ev) cudaEventRecord(ev[0], st);
    cudaError_t e = launch_step(h->tmap[0], h->P, h->O, S, h->R, h->level, h->step_blocks, st);
    if (ev) cudaEventRecord(ev[1], st);
    h->O.base += counter_advance(h->O.nitems, h->step_blocks);
    // the new state is in the next buffer
    const int t = h->cur;
    h->cur = h->nxt;
    h->nxt = t;
    bind(h, h->cur, h->nxt, h->P, h->O);
    h->level++;
    return e;
}

// two steps: the two-step kernel on the interior box (current -> next
// buffer, the box's ring and probe points at level n+1 into the third
// buffer), then the single-step kernel twice on the shell (current -> third
// -> next buffer).  Events (when ev is non-null): before the two-step
// launch, between the launches, after the last.
cudaError_t launch_two_steps(tf_ctx* h, Sources& S, cudaEvent_t* ev) {
    cudaStream_t st = h->stream;
    const int x = h->cur, y = h->nxt, z = 3 - h->cur - h->nxt;
    const double t1 = (double)(h->level + 1) * h->dt, t2 = (double)(h->level + 2) * h->dt;
    Step2Out O2;
    for (int c = 0; c < 3; ++c) {
        O2.E[c] = h->fE[y][c];
        O2.B[c] = h->fB[y][c];
        O2.J[c] = h->fJ[y][c];
        O2.ZE[c] = h->fE[z][c];
        O2.ZB[c] = h->fB[z][c];
    }
    O2.tilemat = h->O.tilemat;
    O2.ntx = h->L.ntx;
    O2.nty = h->L.nty;
    O2.ecur = 9 * x;
    O2.bcur = 9 * x + 3;
    O2.lo[0] = h->tx0 * kSX;
    O2.hi[0] = h->tx1 * kSX;
    O2.lo[1] = h->ty0 * kSY;
    O2.hi[1] = h->ty1 * kSY;
    O2.lo[2] = h->tz0;
    O2.hi[2] = h->tz1;
    O2.order = (const long long*)(h->ws + h->L.off_order_t);
    O2.nitems = h->nitems_t;
    O2.ctr = h->ctr_t;
    O2.base = h->base_t;
    O2.nprobe = h->R.n;
    for (int p = 0; p < h->R.n; ++p)
        for (int a = 0; a < 3; ++a) O2.probe[p][a] = h->ppos[p][a];
    for (int q = 0; q < h->nsrc; ++q) {
        S.amp[q] = (float)(h->src[q].amp * waveform(h->src[q], t1));
        O2.amp2[q] = (float)(h->src[q].amp * waveform(h->src[q], t2));
    }
    if (ev) cudaEventRecord(ev[0], st);
    cudaError_t e = launch_step2(h->tmap[3], h->P, O2, S, h->blocks_t, st);
    h->base_t += counter_advance(h->nitems_t, h->blocks_t);
    if (ev) cudaEventRecord(ev[1], st);
    Params P1 = h->P;
    StepOut O1 = h->O;
    O1.order = (const long long*)(h->ws + h->L.off_order_s);
    O1.nitems = h->nitems_s;
    bind(h, x, z, P1, O1);
    O1.base = h->O.base;
    if (e == cudaSuccess) e = launch_step(h->tmap[0], P1, O1, S, h->R, h->level, h->blocks_s, st);
    h->O.base += counter_advance(h->nitems_s, h->blocks_s);
    if (ev) cudaEventRecord(ev[2], st);
    for (int q = 0; q < h->nsrc; ++q) S.amp[q] = O2.amp2[q];
    bind(h, z, y, P1, O1);
    O1.base = h->O.base;
    if (e == cudaSuccess) e = launch_step(h->tmap[0], P1, O1, S, h->R, h->level + 1, h->blocks_s, st);
    h->O.base += counter_advance(h->nitems_s, h->blocks_s);
    if (ev) cudaEventRecord(ev[3], st);
    h->cur = y;
    h->nxt = x;
    bind(h, h->cur, h->nxt, h->P, h->O);
    h->level += 2;
    return e;
}

bool two_step(const tf_ctx* h) { return h->two_step_on && h->box_ok && h->P.uniform_mu && h->nitems_t > 0; }

// host copy of the single-step kernel's rule for the items that take its
// full plane body (used to order the shell list; the kernel decides again)
bool rare_item(const tf_ctx* h, const Sources& S, int tile, int kz0, int len) {
    const Params& P = h->P;
    if (!P.uniform_mu) return true;
    const int x0 = (tile % h->L.ntx) * kSX, y0 = (tile / h->L.ntx) * kSY;
    const int kz1 = kz0 + len, ks = (kz0 > 0 || P.per[2]) ? kz0 - 1 : kz0;
    const int ka = ks < 0 ? 0 : ks, kb = kz1 - 1;
    const bool sx = P.L[0] > 0 && (x0 - 1 < P.L[0] || x0 + kSX - 1 >= P.n[0] - P.L[0]);
    const bool sy = P.L[1] > 0 && (y0 - 1 < P.L[1] || y0 + kSY - 1 >= P.n[1] - P.L[1]);
    const bool sz = P.L[2] > 0 && (ka < P.L[2] || kb >= P.n[2] - P.L[2]);
    if ((int)sx + (int)sy + (int)sz >= 2) return true;
    if (S.n > 0 && x0 + kSX > S.bb_lo[0] && x0 <= S.bb_hi[0] && y0 + kSY > S.bb_lo[1] && y0 <= S.bb_hi[1]) {
        const int sk0 = S.bb_lo[2], sk1 = S.bb_hi[2];
        if (sk1 > sk0 && ((kb >= sk0 && ka < sk1) || (ks < 0 && P.N[2] - 1 >= sk0 && P.N[2] - 1 < sk1))) return true;
    }
    const bool mur = P.bc[2] == TF_BC_MUR;
    return mur && ((ka <= 1 && 1 <= kb) || (ka <= P.n[2] - 1 && P.n[2] - 1 <= kb));
}

// the work lists of two-step passes, built on the host: the shell (every
// tile's z chunks outside the box; items that take the full plane body
// first, the others z chunk by z chunk, the last ones in pieces) and the
// box (its tiles in kTBLenMax-plane items, z chunk by z chunk)
cudaError_t build_two_step_lists(tf_ctx* h, const Sources& S) {
    const Layout& L = h->L;
    long long* sl = (long long*)malloc(sizeof(long long) * (size_t)L.max_s);
    long long* fa = (long long*)malloc(sizeof(long long) * (size_t)L.max_s);
    long long* tl = (long long*)malloc(sizeof(long long) * (size_t)L.max_t);
    if (!sl || !fa || !tl) {
        free(sl);
        free(fa);
        free(tl);
        return cudaErrorMemoryAllocation;
    }
    long long ns = 0, nf = 0, nt = 0, npieces = 0;
    bool ok = true;
    for (int pass = 0; pass < 2; ++pass) {   // pass 0 counts the pieces, pass 1 lists them
        const bool split = pass == 1 && npieces < 8LL * h->slots;
        for (int kz = 0; kz < L.kend; kz += h->item_planes) {
            const int ke = kz + h->item_planes < L.kend ? kz + h->item_planes : L.kend;
            for (int ty = 0; ty < L.nty; ++ty)
                for (int tx = 0; tx < L.ntx; ++tx) {
                    const int tile = ty * L.ntx + tx;
                    const bool in = tx >= h->tx0 && tx < h->tx1 && ty >= h->ty0 && ty < h->ty1;
                    int lo[2] = {kz, 0}, hi[2] = {ke, 0}, np = 1;
                    if (in) {   // the chunk minus the box's planes [tz0, tz1)
                        np = 0;
                        if (kz < h->tz0) { lo[np] = kz; hi[np] = ke < h->tz0 ? ke : h->tz0; ++np; }
                        if (ke > h->tz1) { lo[np] = kz > h->tz1 ? kz : h->tz1; hi[np] = ke; ++np; }
                    }
                    for (int p = 0; p < np; ++p) {
                        if (hi[p] <= lo[p]) continue;
                        if (pass == 0) { ++npieces; continue; }
                        if (ns + nf + (hi[p] - lo[p]) > L.max_s) { ok = false; continue; }   // never: sized for it
                        if (rare_item(h, S, tile, lo[p], hi[p] - lo[p])) {
                            const int piece = split ? kSub : hi[p] - lo[p];
                            for (int k = lo[p]; k < hi[p]; k += piece)
                                sl[ns++] = make_item(tile, k, (hi[p] - k) < piece ? hi[p] - k : piece);
                        } else {
                            fa[nf++] = make_item(tile, lo[p], hi[p] - lo[p]);
                        }
                    }
                }
        }
    }
    // the last plain items, one per CTA slot, go out in kSub-plane pieces
    const long long cut = nf > h->slots ? nf - h->slots : 0;
    for (long long i = 0; i < cut; ++i) sl[ns++] = fa[i];
    for (long long i = cut; i < nf && ok; ++i) {
        const long long d = fa[i];
        const int tile = item_tile(d), kz0 = item_kz0(d), len = item_len(d);
        for (int k = kz0; k < kz0 + len; k += kSub) {
            if (ns >= L.max_s) { ok = false; break; }
            sl[ns++] = make_item(tile, k, (kz0 + len - k) < kSub ? kz0 + len - k : kSub);
        }
    }
    for (int kz = h->tz0; kz < h->tz1; kz += h->tb_len) {
        const int len = h->tz1 - kz < h->tb_len ? h->tz1 - kz : h->tb_len;
        for (int ty = h->ty0; ty < h->ty1; ++ty)
            for (int tx = h->tx0; tx < h->tx1; ++tx) {
                if (nt >= L.max_t) { ok = false; break; }
                tl[nt++] = make_item(ty * L.ntx + tx, kz, len);
            }
    }
    if (!ok) {   // a list outgrew its region: no two-step passes (never expected)
        free(sl);
        free(fa);
        free(tl);
        h->nitems_s = h->nitems_t = 0;
        return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaSuccess;
    if (ns > 0)
        e = cudaMemcpyAsync(h->ws + L.off_order_s, sl, sizeof(long long) * (size_t)ns, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && nt > 0)
        e = cudaMemcpyAsync(h->ws + L.off_order_t, tl, sizeof(long long) * (size_t)nt, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    free(sl);
    free(fa);
    free(tl);
    h->nitems_s = (int)ns;
    h->nitems_t = (int)nt;
    const long long hs = (ns + 1) / 2, ht = (nt + 1) / 2;
    h->blocks_s = (int)(hs < h->slots ? (hs > 0 ? hs : 1) : h->slots);
    h->blocks_t = (int)(ht < h->slots2 ? (ht > 0 ? ht : 1) : h->slots2);
    return e;
}

// rebuild the work-item order after the sources or materials changed
cudaError_t refresh_order(tf_ctx* h, const Sources& S) {
    if (!h->order_dirty) return cudaSuccess;
    int* dcount = (int*)(h->ws + h->L.off_misc + 192);
    // fewer than 8 (tile, chunk) items per CTA: cut the slow ones into pieces
    const long long items = (long long)h->L.ntx * h->L.nty * ((h->L.kend + h->item_planes - 1) / h->item_planes);
    const int split = items < 8LL * h->step_blocks;
    // the last plain items of the order, one per CTA, also go out in pieces:
    // the CTAs then run out of work at nearly the same time
    const int tail = h->fine ? (int)items : h->step_blocks;
    cudaError_t e =
        launch_item_order(h->P, h->O, S, split, tail, h->item_planes, (long long*)h->O.order, dcount, h->stream);
    int n = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&n, dcount, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return e;
    h->O.nitems = n;
    h->nitems_s = h->nitems_t = 0;
    if (h->box_ok && h->P.uniform_mu && (e = build_two_step_lists(h, S)) != cudaSuccess) return e;
    h->order_dirty = 0;
    return cudaSuccess;
}

void fill_sources(const tf_ctx* h, Sources& S) {
    S.n = h->nsrc;
    for (int a = 0; a < 3; ++a) { S.bb_lo[a] = 1 << 30; S.bb_hi[a] = -1; }
    for (int s = 0; s < h->nsrc; ++s) {
        S.comp[s] = h->src[s].comp;
        S.amp[s] = 0.f;
        for (int a = 0; a < 3; ++a) {
            S.lo[s][a] = h->src[s].lo[a];
            S.hi[s][a] = h->src[s].hi[a];
            if (S.lo[s][a] < S.bb_lo[a]) S.bb_lo[a] = S.lo[s][a];
            if (S.hi[s][a] > S.bb_hi[a]) S.bb_hi[a] = S.hi[s][a];
        }
    }
}

}  // namespace

tf_status tf_step(tf_handle h, int64_t nsteps) {
    if (!h || nsteps < 0) return TF_EINVAL;
    if (nsteps == 0) return TF_OK;
    if (!h->primed) {
        TF_CUDA(launch_prime(h->P, h->stream));
        h->primed = 1;
    }
    Sources S;
    fill_sources(h, S);
    TF_CUDA(refresh_order(h, S));
    int64_t s = 0;
    if (two_step(h))
        for (; s + 2 <= nsteps; s += 2) TF_CUDA(launch_two_steps(h, S, nullptr));
    for (; s < nsteps; ++s) TF_CUDA(launch_one_step(h, S, nullptr));
    return TF_OK;
}

tf_status tf_set_two_step(tf_handle h, int planes) {
    if (!h || (planes != 0 && (planes < kTBLenMin || planes > kTBLenMax))) return TF_EINVAL;
    h->two_step_on = planes != 0;
    if (planes != 0 && planes != h->tb_len) {
        h->tb_len = planes;
        h->order_dirty = 1;   // the box's work list is cut again
    }
    return TF_OK;
}

tf_status tf_set_item_planes(tf_handle h, int planes) {
    if (!h || planes < kChunk || planes > kItemMax) return TF_EINVAL;
    if (planes != h->item_planes) {
        h->item_planes = planes;
        h->order_dirty = 1;   // the work lists are cut again
    }
    return TF_OK;
}

tf_status tf_set_wait_limit(tf_handle h, int64_t polls) {
    if (!h) return TF_EINVAL;
    h->P.wait_polls = polls < 0 ? kSpinLimit : (long long)polls;
    return TF_OK;
}

tf_status tf_two_step_box(tf_handle h, int lo[3], int hi[3], int* active) {
    if (!h || !lo || !hi) return TF_EINVAL;
    lo[0] = h->tx0 * kSX;
    hi[0] = h->tx1 * kSX;
    lo[1] = h->ty0 * kSY;
    hi[1] = h->ty1 * kSY;
    lo[2] = h->tz0;
    hi[2] = h->tz1;
    if (active) *active = two_step(h) ? 1 : 0;
    return TF_OK;
}

tf_status tf_batch_step(const tf_handle* hs, int n, int64_t nsteps) {
    if (!hs || n < 1 || nsteps < 0) return TF_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!hs[i]) return TF_EINVAL;
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return TF_EINVAL;   // a handle twice would race with itself
    }
    if (nsteps == 0) return TF_OK;
    Sources S[64];
    const int chunk = n < 64 ? n : 64;
    for (int b0 = 0; b0 < n; b0 += chunk) {
        const int nb = (n - b0) < chunk ? (n - b0) : chunk;
        for (int i = 0; i < nb; ++i) {
            tf_ctx* h = hs[b0 + i];
            if (!h->primed) {
                TF_CUDA(launch_prime(h->P, h->stream));
                h->primed = 1;
            }
            fill_sources(h, S[i]);
            TF_CUDA(refresh_order(h, S[i]));
        }
    }
    // step by step, every grid in turn: each grid's launches stay in order on
    // its own stream while the grids' streams overlap one another's tails
    for (int64_t s = 0; s < nsteps; ++s)
        for (int b0 = 0; b0 < n; b0 += chunk) {
            const int nb = (n - b0) < chunk ? (n - b0) : chunk;
            for (int i = 0; i < nb; ++i) {
                tf_ctx* h = hs[b0 + i];
                if (n > 64) fill_sources(h, S[i]);
                TF_CUDA(launch_one_step(h, S[i], nullptr));
            }
        }
    return TF_OK;
}

// ---------------------------------------------------------------- batches
namespace {

constexpr int kBatchGraphSteps = 64;   // steps per captured graph

struct BatchLayout {
    size_t off_step, off_grids, off_probes, off_order, off_amp, bytes;
    long long max_items;
};

long long order_capacity(const tf_ctx* h) {
    return (long long)h->L.ntx * h->L.nty * h->L.nch * ((kChunk + kSub - 1) / kSub);
}

BatchLayout batch_layout(const tf_handle* hs, int n, int64_t nsteps) {
    BatchLayout B{};
    size_t o = 0;
    B.off_step = o;   o += kAlign;   // step number, work counter
    B.off_grids = o;  o += align_up(sizeof(BatchGrid) * (size_t)n);
    B.off_probes = o; o += align_up(sizeof(int) * 2 * TF_MAX_PROBES * (size_t)n);
    B.max_items = 0;
    for (int i = 0; i < n; ++i) B.max_items += order_capacity(hs[i]);
    B.off_order = o;  o += align_up(sizeof(long long) * (size_t)B.max_items);
    B.off_amp = o;
    for (int i = 0; i < n; ++i) o += align_up(sizeof(float) * (size_t)nsteps * (size_t)(hs[i]->nsrc > 0 ? hs[i]->nsrc : 1));
    B.bytes = o;
    return B;
}

tf_status batch_check(const tf_handle* hs, int n, int64_t nsteps) {
    if (!hs || n < 1 || nsteps < 0) return TF_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!hs[i]) return TF_EINVAL;
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return TF_EINVAL;   // a handle twice would race with itself
    }
    return TF_OK;
}

}  // namespace

tf_status tf_batch_scratch_size(const tf_handle* hs, int n, int64_t nsteps, size_t* bytes) {
    tf_status rc = batch_check(hs, n, nsteps);
    if (rc != TF_OK) return rc;
    if (!bytes) return TF_EINVAL;
    *bytes = batch_layout(hs, n, nsteps).bytes;
    return TF_OK;
}

tf_status tf_batch_run(const tf_handle* hs, int n, int64_t nsteps, void* scratch, size_t bytes) {
    tf_status rc = batch_check(hs, n, nsteps);
    if (rc != TF_OK) return rc;
    if (!scratch || ((uintptr_t)scratch) % kAlign) return TF_EINVAL;
    const BatchLayout BL = batch_layout(hs, n, nsteps);
    if (bytes < BL.bytes) return TF_ENOMEM;
    if (nsteps == 0) return TF_OK;
    if (n > (1 << 15)) return TF_ENOTSUP;   // the grid index fills descriptor bits 48-62
    // the grids' earlier work is done before the batch reads their state
    for (int i = 0; i < n; ++i) TF_CUDA(cudaStreamSynchronize(hs[i]->stream));
    cudaStream_t st = hs[0]->stream;
    const int slots = hs[0]->slots;
    BatchGrid* G = (BatchGrid*)calloc((size_t)n, sizeof(BatchGrid));
    char* amp_host = (char*)malloc(BL.bytes - BL.off_amp);
    long long* items = (long long*)malloc(sizeof(long long) * (size_t)BL.max_items);
    long long* list = (long long*)malloc(sizeof(long long) * (size_t)BL.max_items);
    char* rare = (char*)malloc((size_t)BL.max_items);
    int* probes = (int*)malloc(sizeof(int) * 2 * TF_MAX_PROBES * (size_t)n);
    if (!G || !amp_host || !items || !list || !rare || !probes) {
        free(G); free(amp_host); free(items); free(list); free(rare); free(probes);
        return TF_ENOMEM;
    }
    // one work list over all grids: each grid's items (its own order) with
    // the grid's index in the descriptor; the items that take the full plane
    // body, of every grid, first
    long long ntot = 0, nrare = 0;
    int np = 0;
    size_t ao = 0;
    for (int i = 0; i < n && rc == TF_OK; ++i) {
        tf_ctx* h = hs[i];
        if (!h->primed) {
            if (launch_prime(h->P, h->stream) != cudaSuccess) { rc = TF_ECUDA; break; }
            h->primed = 1;
        }
        Sources S;
        fill_sources(h, S);
        // the grid's whole items, slow ones first, none cut into pieces (the
        // batch's one list balances the launch), made in the scratch's list
        // area and read back
        long long* tmp = (long long*)((char*)scratch + BL.off_order);
        int* dcount = (int*)(h->ws + h->L.off_misc + 192);
        int cnt = 0;
        if (launch_item_order(h->P, h->O, S, 0, 0, kItemMax, tmp, dcount, h->stream) != cudaSuccess ||
            cudaMemcpyAsync(&cnt, dcount, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess || cnt < 0 || ntot + cnt > BL.max_items ||
            cudaMemcpy(items + ntot, tmp, sizeof(long long) * (size_t)cnt, cudaMemcpyDeviceToHost) != cudaSuccess) {
            rc = TF_ECUDA;
            break;
        }
        for (long long k = ntot; k < ntot + cnt; ++k) {
            rare[k] = rare_item(h, S, item_tile(items[k]), item_kz0(items[k]), item_len(items[k])) ? 1 : 0;
            items[k] = item_with_grid(items[k], i);
            nrare += rare[k];
        }
        ntot += cnt;
        BatchGrid& g = G[i];
        memcpy(&g.tm, h->tmap[0], sizeof(TMaps));
        g.P[0] = h->P;
        g.O[0] = h->O;
        g.P[1] = h->P;
        g.O[1] = h->O;
        bind(h, h->cur, h->nxt, g.P[0], g.O[0]);
        bind(h, h->nxt, h->cur, g.P[1], g.O[1]);
        g.S = S;
        g.R = h->R;
        const int ns = h->nsrc > 0 ? h->nsrc : 1;
        float* amp = (float*)(amp_host + ao);
        for (int64_t k = 0; k < nsteps; ++k) {
            const double t1 = (double)(h->level + k + 1) * h->dt;
            for (int q = 0; q < h->nsrc; ++q)
                amp[k * ns + q] = (float)(h->src[q].amp * waveform(h->src[q], t1));
        }
        g.amp = (const float*)((char*)scratch + BL.off_amp + ao);
        ao += align_up(sizeof(float) * (size_t)nsteps * ns);
        g.level0 = h->level;
        for (int p = 0; p < h->R.n; ++p) {
            probes[2 * np] = i;
            probes[2 * np + 1] = p;
            ++np;
        }
    }
    long long r = 0, f = nrare;
    for (long long k = 0; k < ntot; ++k) list[rare[k] ? r++ : f++] = items[k];
    BatchLaunch L;
    L.G = (const BatchGrid*)((char*)scratch + BL.off_grids);
    L.ngrids = n;
    L.step = (const int*)((char*)scratch + BL.off_step);
    L.order = (const long long*)((char*)scratch + BL.off_order);
    L.nitems = (int)ntot;
    L.ctr = (unsigned long long*)((char*)scratch + BL.off_step + 64);
    L.base0 = 0;
    L.base_inc = counter_advance(ntot, slots);
    L.probes = (const int*)((char*)scratch + BL.off_probes);
    L.nprobes = np;
    int* dstep = (int*)((char*)scratch + BL.off_step);
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (rc == TF_OK &&
        (cudaMemcpyAsync((char*)scratch + BL.off_grids, G, sizeof(BatchGrid) * (size_t)n, cudaMemcpyHostToDevice, st) !=
             cudaSuccess ||
         cudaMemcpyAsync((char*)scratch + BL.off_probes, probes, sizeof(int) * 2 * (size_t)(np > 0 ? np : 1),
                         cudaMemcpyHostToDevice, st) != cudaSuccess ||
         cudaMemcpyAsync((char*)scratch + BL.off_order, list, sizeof(long long) * (size_t)(ntot > 0 ? ntot : 1),
                         cudaMemcpyHostToDevice, st) != cudaSuccess ||
         cudaMemcpyAsync((char*)scratch + BL.off_amp, amp_host, BL.bytes - BL.off_amp, cudaMemcpyHostToDevice, st) !=
             cudaSuccess ||
         cudaMemsetAsync((char*)scratch + BL.off_step, 0, kAlign, st) != cudaSuccess))
        rc = TF_ECUDA;
    // one launch per step over all grids, K steps captured in a CUDA graph and
    // replayed (the step number lives on the device; a one-thread launch
    // advances it after each step), the remaining steps launched directly
    const int64_t K = nsteps < kBatchGraphSteps ? nsteps : kBatchGraphSteps;
    if (rc == TF_OK && K > 1) {
        cudaStream_t cs = nullptr;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            rc = TF_ECUDA;
        } else {
            cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            for (int64_t k = 0; k < K && e == cudaSuccess; ++k) {
                e = launch_step_batch(L, slots, cs);
                if (e == cudaSuccess) e = launch_step_advance(dstep, cs);
            }
            const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
            cudaStreamDestroy(cs);
            if (e != cudaSuccess) rc = TF_ECUDA;
        }
    }
    int64_t done = 0;
    if (rc == TF_OK && exec)
        for (; done + K <= nsteps; done += K)
            if (cudaGraphLaunch(exec, st) != cudaSuccess) { rc = TF_ECUDA; break; }
    for (; rc == TF_OK && done < nsteps; ++done)
        if (launch_step_batch(L, slots, st) != cudaSuccess || launch_step_advance(dstep, st) != cudaSuccess)
            rc = TF_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == TF_OK) rc = TF_ECUDA;
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (rc == TF_OK)
        for (int i = 0; i < n; ++i) {   // each handle holds the state the run reached
            tf_ctx* h = hs[i];
            h->level += nsteps;
            if (nsteps & 1) {
                const int t = h->cur;
                h->cur = h->nxt;
                h->nxt = t;
            }
            const unsigned long long base = h->O.base;
            bind(h, h->cur, h->nxt, h->P, h->O);
            h->O.base = base;
        }
    free(G); free(amp_host); free(items); free(list); free(rare); free(probes);
    return rc;
}

tf_status tf_step_timed(tf_handle h, int64_t nsteps, double* kernel_ms, int64_t* launches, int nkinds,
                        double* total_ms) {
    if (!h || nsteps < 0 || !kernel_ms || !launches || nkinds < 1 || nkinds > 3) return TF_EINVAL;
    for (int k = 0; k < nkinds; ++k) { kernel_ms[k] = 0.0; launches[k] = 0; }
    if (total_ms) *total_ms = 0.0;
    if (nsteps == 0) return TF_OK;
    if (!h->primed) {
        TF_CUDA(launch_prime(h->P, h->stream));
        h->primed = 1;
    }
    Sources S;
    fill_sources(h, S);
    TF_CUDA(refresh_order(h, S));
    const bool two = two_step(h);
    // launch groups: two-step passes (three launches) while two steps remain, then single steps
    const int64_t ncyc = two ? nsteps / 2 : 0, nunits = ncyc + (nsteps - 2 * ncyc);
    // events for up to kBatch groups are enqueued before the stream is waited
    // on, so a run of up to kBatch groups goes out without a pause
    constexpr int64_t kBatch = 4096;
    const int64_t ring = nunits < kBatch ? nunits : kBatch;
    cudaEvent_t(*ev)[4] = (cudaEvent_t(*)[4])calloc((size_t)ring, sizeof(cudaEvent_t[4]));
    if (!ev) return TF_ENOMEM;
    tf_status rc = TF_OK;
    for (int64_t u = 0; u < ring && rc == TF_OK; ++u)
        for (int m = 0; m < 4; ++m)
            if (cudaEventCreate(&ev[u][m]) != cudaSuccess) {
                ev[u][m] = nullptr;
                rc = TF_ECUDA;
                break;
            }
    auto add = [&](int kind, cudaEvent_t a, cudaEvent_t b) {
        if (kind >= nkinds || rc != TF_OK) return;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) { rc = TF_ECUDA; return; }
        kernel_ms[kind] += ms;
        launches[kind] += 1;
    };
    int64_t done = 0;
    while (rc == TF_OK && done < nunits) {
        const int64_t m = (nunits - done) < ring ? (nunits - done) : ring;
        bool cyc[kBatch];
        for (int64_t u = 0; u < m && rc == TF_OK; ++u) {
            cyc[u] = done + u < ncyc;
            const cudaError_t e = cyc[u] ? launch_two_steps(h, S, ev[u]) : launch_one_step(h, S, ev[u]);
            if (e != cudaSuccess) rc = TF_ECUDA;
        }
        if (rc != TF_OK || cudaStreamSynchronize(h->stream) != cudaSuccess) { rc = TF_ECUDA; break; }
        for (int64_t u = 0; u < m && rc == TF_OK; ++u) {
            if (cyc[u]) {
                add(2, ev[u][0], ev[u][1]);
                add(1, ev[u][1], ev[u][2]);
                add(1, ev[u][2], ev[u][3]);
            } else {
                add(1, ev[u][0], ev[u][1]);
            }
        }
        if (rc == TF_OK && total_ms) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[0][0], ev[m - 1][cyc[m - 1] ? 3 : 1]) != cudaSuccess) rc = TF_ECUDA;
            *total_ms += ms;
        }
        done += m;
    }
    for (int64_t u = 0; u < ring; ++u)
        for (int k = 0; k < 4; ++k)
            if (ev[u][k]) cudaEventDestroy(ev[u][k]);
    free(ev);
    for (int k = 0; k < nkinds; ++k)
        if (launches[k]) kernel_ms[k] /= (double)launches[k];
    return rc;
}

tf_status tf_sync(tf_handle h) {
    if (!h) return TF_EINVAL;
    unsigned st = 0;
    TF_CUDA(cudaMemcpyAsync(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
    TF_CUDA(cudaStreamSynchronize(h->stream));
    if (st & kStatusTimeout) return TF_ETIMEOUT;
    if (st & kStatusNonFinite) return TF_ENONFINITE;
    return TF_OK;
}

tf_status tf_read_probe_dft(tf_handle h, int id, double* re, double* im) {
    if (!h || id < 0 || id >= h->R.n || !re || !im) return TF_EINVAL;
    const int nf = h->R.nfreq[id];
    TF_CUDA(cudaMemcpyAsync(re, h->R.re + id * TF_MAX_FREQS, sizeof(double) * nf, cudaMemcpyDeviceToHost, h->stream));
    TF_CUDA(cudaMemcpyAsync(im, h->R.im + id * TF_MAX_FREQS, sizeof(double) * nf, cudaMemcpyDeviceToHost, h->stream));
    TF_CUDA(cudaStreamSynchronize(h->stream));
    return TF_OK;
}

tf_status tf_read_probe_series(tf_handle h, int id, double* out, int64_t n) {
    if (!h || id < 0 || id >= h->R.n || !out || n < 0) return TF_EINVAL;
    if (n > h->R.cap || n > h->level) return TF_EINVAL;
    if (n == 0) return TF_OK;
    TF_CUDA(cudaMemcpyAsync(out, h->R.series + (long long)id * h->R.cap, sizeof(double) * n,
                            cudaMemcpyDeviceToHost, h->stream));
    TF_CUDA(cudaStreamSynchronize(h->stream));
    return TF_OK;
}

tf_status tf_read_field(tf_handle h, int comp, float* dst, int on_device) {
    if (!h || !dst || comp < 0 || comp > 8) return TF_EINVAL;
    float* out = on_device ? dst : h->scratch;
    const double scale = comp < 3 ? 1.0 : comp < 6 ? 1.0 / kC0 : kEps0 / h->dt;
    TF_CUDA(launch_read_field(h->P, comp, h->primed, out, scale, h->stream));
    if (!on_device)
        TF_CUDA(cudaMemcpyAsync(dst, out, sizeof(float) * h->L.ndense, cudaMemcpyDeviceToHost, h->stream));
    TF_CUDA(cudaStreamSynchronize(h->stream));
    return TF_OK;
}

// ------------------------------------------------------------- checkpoints
namespace {

constexpr size_t kCkptHeader = 256;

struct CkptHeader {
    char magic[8];
    int32_t N[3], pitch, bc[3], ncpml_axes, nprobes, max_probes;
    int64_t series_cap, level;
    int32_t primed, reserved;
    double dt;
    uint64_t field_bytes, total_bytes;
};
static_assert(sizeof(CkptHeader) <= kCkptHeader, "checkpoint header");

const char kCkptMagic[8] = {'T', 'F', 'C', 'K', 'P', 'T', '1', 0};

// the arrays of a blob after the header, in order: E, B, Js at the level the
// state holds them; per CPML axis the psi_B pair and the psi_E pair; the
// probe DFT accumulators; the probe series.  `cur` gives the arrays the state
// is read from / written to, `other` the second buffer of ping-pong arrays
// (nullptr where there is none)
struct CkptPart {
    float* cur;
    float* other[2];
    size_t bytes;
};

int ckpt_parts(const tf_ctx* h, CkptPart* parts) {
    const size_t fb = sizeof(float) * (size_t)h->L.total;
    const int x = h->cur, y = h->nxt, z = 3 - h->cur - h->nxt;
    int n = 0;
    for (int c = 0; c < 3; ++c) parts[n++] = {h->fE[x][c], {h->fE[y][c], h->fE[z][c]}, fb};
    for (int c = 0; c < 3; ++c) parts[n++] = {h->fB[x][c], {h->fB[y][c], h->fB[z][c]}, fb};
    for (int c = 0; c < 3; ++c) parts[n++] = {h->fJ[x][c], {h->fJ[y][c], h->fJ[z][c]}, fb};
    for (int a = 0; a < 3; ++a) {
        if (h->desc.bc[a].kind != TF_BC_CPML) continue;
        for (int c = 0; c < 3; ++c)
            if (c != a) parts[n++] = {h->fPB[x][c][a], {h->fPB[y][c][a], h->fPB[z][c][a]}, fb};
        for (int c = 0; c < 3; ++c)
            if (c != a) parts[n++] = {h->P.psiE[c][a], {nullptr, nullptr}, fb};
    }
    const size_t pb = sizeof(double) * TF_MAX_PROBES * TF_MAX_FREQS;
    parts[n++] = {(float*)h->R.re, {nullptr, nullptr}, pb};
    parts[n++] = {(float*)h->R.im, {nullptr, nullptr}, pb};
    if (h->R.series)
        parts[n++] = {(float*)h->R.series, {nullptr, nullptr}, sizeof(double) * (size_t)h->desc.max_probes * h->R.cap};
    return n;
}

size_t ckpt_bytes(const tf_ctx* h) {
    CkptPart parts[40];
    const int n = ckpt_parts(h, parts);
    size_t b = kCkptHeader;
    for (int k = 0; k < n; ++k) b += parts[k].bytes;
    return b;
}

CkptHeader ckpt_header(const tf_ctx* h) {
    CkptHeader H;
    memset(&H, 0, sizeof(H));
    memcpy(H.magic, kCkptMagic, sizeof(kCkptMagic));
    for (int a = 0; a < 3; ++a) {
        H.N[a] = h->L.N[a];
        H.bc[a] = h->desc.bc[a].kind;
    }
    H.pitch = h->L.pitch;
    H.ncpml_axes = h->L.ncpml_axes;
    H.nprobes = h->R.n;
    H.max_probes = h->desc.max_probes;
    H.series_cap = h->R.cap;
    H.level = h->level;
    H.primed = h->primed;
    H.dt = h->dt;
    H.field_bytes = sizeof(float) * (uint64_t)h->L.total;
    H.total_bytes = ckpt_bytes(h);
    return H;
}

}  // namespace

tf_status tf_checkpoint_size(tf_handle h, size_t* bytes) {
    if (!h || !bytes) return TF_EINVAL;
    *bytes = ckpt_bytes(h);
    return TF_OK;
}

tf_status tf_checkpoint_save(tf_handle h, void* dst, size_t bytes, int on_device) {
    if (!h || !dst || bytes < ckpt_bytes(h)) return TF_EINVAL;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    char* d = (char*)dst;
    const CkptHeader H = ckpt_header(h);
    if (on_device) {
        TF_CUDA(cudaMemcpyAsync(d, &H, sizeof(H), cudaMemcpyHostToDevice, h->stream));
    } else {
        memset(d, 0, kCkptHeader);
        memcpy(d, &H, sizeof(H));
    }
    CkptPart parts[40];
    const int n = ckpt_parts(h, parts);
    size_t o = kCkptHeader;
    for (int k = 0; k < n; ++k) {
        TF_CUDA(cudaMemcpyAsync(d + o, parts[k].cur, parts[k].bytes, kind, h->stream));
        o += parts[k].bytes;
    }
    TF_CUDA(cudaStreamSynchronize(h->stream));
    return TF_OK;
}

tf_status tf_checkpoint_load(tf_handle h, const void* src, size_t bytes, int on_device) {
    if (!h || !src || bytes < kCkptHeader) return TF_EINVAL;
    const char* s = (const char*)src;
    CkptHeader H;
    if (on_device) {
        TF_CUDA(cudaMemcpyAsync(&H, s, sizeof(H), cudaMemcpyDeviceToHost, h->stream));
        TF_CUDA(cudaStreamSynchronize(h->stream));
    } else {
        memcpy(&H, s, sizeof(H));
    }
    CkptHeader M = ckpt_header(h);
    bool same = memcmp(H.magic, M.magic, sizeof(H.magic)) == 0 && H.pitch == M.pitch &&
                H.ncpml_axes == M.ncpml_axes && H.nprobes == M.nprobes && H.max_probes == M.max_probes &&
                H.series_cap == M.series_cap && H.dt == M.dt && H.field_bytes == M.field_bytes &&
                H.total_bytes == M.total_bytes && bytes >= M.total_bytes;
    for (int a = 0; a < 3; ++a) same = same && H.N[a] == M.N[a] && H.bc[a] == M.bc[a];
    if (!same || (H.primed != 0 && H.primed != 1) || H.level < 0) return TF_EINVAL;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CkptPart parts[40];
    const int n = ckpt_parts(h, parts);
    size_t o = kCkptHeader;
    for (int k = 0; k < n; ++k) {
        TF_CUDA(cudaMemcpyAsync(parts[k].cur, s + o, parts[k].bytes, kind, h->stream));
        // the other buffers of a rotating array hold the same values, so that
        // points the step never writes (walls) agree in all of them
        for (int b = 0; b < 2; ++b)
            if (parts[k].other[b])
                TF_CUDA(cudaMemcpyAsync(parts[k].other[b], s + o, parts[k].bytes, kind, h->stream));
        o += parts[k].bytes;
    }
    TF_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    TF_CUDA(cudaStreamSynchronize(h->stream));
    h->level = H.level;
    h->primed = H.primed;
    return TF_OK;
}

// ---------------------------------------------------------------- adjoint
namespace {

struct AdjLayout {
    size_t ck, nck, off_ck, off_hist, off_state, off_grad, bytes;
    int64_t nseg;
};

AdjLayout adj_layout(const tf_ctx* h, int64_t nsteps, int segment) {
    AdjLayout A{};
    const size_t fb = align_up(sizeof(float) * (size_t)h->L.total);
    A.nseg = (nsteps + segment - 1) / segment;
    A.ck = align_up(ckpt_bytes(h));
    A.nck = (size_t)A.nseg + 1;
    size_t o = 0;
    A.off_ck = o;    o += A.nck * A.ck;
    A.off_hist = o;  o += 2 * (size_t)(segment + 1) * 3 * fb;   // two segments' E history
    A.off_state = o; o += (size_t)(9 + 4 * h->L.ncpml_axes + 12) * fb;   // E, B, J, psi, edge and face weights
    A.off_grad = o;  o += 6 * align_up(sizeof(double) * (size_t)h->L.total);
    A.bytes = o;
    return A;
}

// the adjoint's second stream (higher priority: the recompute's CTAs are
// placed as soon as an SM has room) and its events; released on every exit
struct AdjStreams {
    cudaStream_t rs = nullptr;
    cudaEvent_t evR[2] = {nullptr, nullptr}, evA[2] = {nullptr, nullptr};
    int sms = 1;
    bool create() {
        int dev = 0, lo = 0, hi = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            return false;
        if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) return false;
        if (cudaStreamCreateWithPriority(&rs, cudaStreamNonBlocking, hi) != cudaSuccess) return false;
        for (int b = 0; b < 2; ++b)
            if (cudaEventCreateWithFlags(&evR[b], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&evA[b], cudaEventDisableTiming) != cudaSuccess)
                return false;
        return true;
    }
    ~AdjStreams() {
        if (rs) cudaStreamSynchronize(rs);
        for (int b = 0; b < 2; ++b) {
            if (evR[b]) cudaEventDestroy(evR[b]);
            if (evA[b]) cudaEventDestroy(evA[b]);
        }
        if (rs) cudaStreamDestroy(rs);
    }
};

// a checkpoint this run wrote (so its header needs no check) back into the
// grid, enqueued on the handle's stream without waiting for it
tf_status ckpt_restore_async(tf_ctx* h, const char* src, int64_t level, int primed) {
    CkptPart parts[40];
    const int n = ckpt_parts(h, parts);
    size_t o = kCkptHeader;
    for (int k = 0; k < n; ++k) {
        TF_CUDA(cudaMemcpyAsync(parts[k].cur, src + o, parts[k].bytes, cudaMemcpyDeviceToDevice, h->stream));
        for (int b = 0; b < 2; ++b)
            if (parts[k].other[b])
                TF_CUDA(cudaMemcpyAsync(parts[k].other[b], src + o, parts[k].bytes, cudaMemcpyDeviceToDevice,
                                        h->stream));
        o += parts[k].bytes;
    }
    TF_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    h->level = level;
    h->primed = primed;
    return TF_OK;
}

}  // namespace

tf_status tf_adjoint_scratch_size(tf_handle h, int64_t nsteps, int segment, size_t* bytes) {
    if (!h || !bytes || nsteps < 1 || segment < 1) return TF_EINVAL;
    *bytes = adj_layout(h, nsteps, segment).bytes;
    return TF_OK;
}

tf_status tf_adjoint_run(tf_handle h, int64_t nsteps, int probe, int freq_index, int segment, void* scratch,
                         size_t bytes, double* J, float* grad_eps, float* grad_lambda) {
    if (!h || nsteps < 1 || segment < 1 || !scratch || !J || !grad_eps || !grad_lambda) return TF_EINVAL;
    if (probe < 0 || probe >= h->R.n || freq_index < 0 || freq_index >= h->R.nfreq[probe]) return TF_EINVAL;
    if (h->level != 0 || h->primed) return TF_ESTATE;
    if (h->desc.bc[2].kind == TF_BC_MUR) return TF_ENOTSUP;
    const AdjLayout A = adj_layout(h, nsteps, segment);
    if (bytes < A.bytes) return TF_ENOMEM;
    char* sc = (char*)scratch;
    const size_t fb = align_up(sizeof(float) * (size_t)h->L.total);
    const size_t gb = align_up(sizeof(double) * (size_t)h->L.total);
    tf_status rc;
    // forward run, a checkpoint at the start of every segment and at the end
    // (every segment but the first starts primed)
    for (int64_t s = 0; s < A.nseg; ++s) {
        if ((rc = tf_checkpoint_save(h, sc + A.off_ck + s * A.ck, A.ck, 1)) != TF_OK) return rc;
        const int64_t len = (s + 1) * segment <= nsteps ? segment : nsteps - s * segment;
        if ((rc = tf_step(h, len)) != TF_OK) return rc;
    }
    if ((rc = tf_checkpoint_save(h, sc + A.off_ck + A.nseg * A.ck, A.ck, 1)) != TF_OK) return rc;
    if ((rc = tf_sync(h)) != TF_OK) return rc;
    // objective J = |X|^2 from the probe's FP64 DFT
    double re[TF_MAX_FREQS], im[TF_MAX_FREQS];
    if ((rc = tf_read_probe_dft(h, probe, re, im)) != TF_OK) return rc;
    const double xr = re[freq_index], xi = im[freq_index];
    *J = xr * xr + xi * xi;
    const double f = h->freqs[probe][freq_index];
    // The adjoint is linear in its seed dJ/dE^n = 2 dt Re(conj(X) w^n), whose
    // size is 2 dt |X| (1e-32 for a 1 V/m source on the CPW grids): scaled by
    // a power of two to O(1), the FP32 adjoint state stays out of FP32's
    // subnormal range while it decays into the CPML; the FP64 gradient sums
    // are scaled back once at the end (exact: a power of two).
    const double seed = 2.0 * h->dt * sqrt(*J);
    const double seed_scale = seed > 0.0 && isfinite(seed) ? ldexp(1.0, -ilogb(seed)) : 1.0;
    // adjoint state and gradient sums start at zero
    TF_CUDA(cudaMemsetAsync(sc + A.off_state, 0, A.bytes - A.off_state, h->stream));
    AdjState S{};
    {
        int m = 0;
        auto fa = [&]() { return (float*)(sc + A.off_state + (size_t)(m++) * fb); };
        for (int c = 0; c < 3; ++c) S.E[c] = fa();
        for (int c = 0; c < 3; ++c) S.B[c] = fa();
        for (int c = 0; c < 3; ++c) S.J[c] = fa();
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) {
                S.psiB[c][a] = nullptr;
                S.psiE[c][a] = nullptr;
            }
        for (int a = 0; a < 3; ++a) {
            if (h->desc.bc[a].kind != TF_BC_CPML) continue;
            for (int c = 0; c < 3; ++c) {
                if (c == a) continue;
                S.psiB[c][a] = fa();
                S.psiE[c][a] = fa();
            }
        }
        for (int c = 0; c < 3; ++c)
            for (int a = 0; a < 3; ++a) {
                S.W[c][a] = S.U[c][a] = nullptr;
                if (a == c) continue;
                S.W[c][a] = fa();
                S.U[c][a] = fa();
            }
        for (int c = 0; c < 3; ++c) {
            S.gE[c] = (double*)(sc + A.off_grad + (size_t)c * gb);
            S.gK[c] = (double*)(sc + A.off_grad + (size_t)(3 + c) * gb);
        }
    }
    Sources src;
    fill_sources(h, src);
    const int64_t n0 = h->R.n0[probe];
    // E history of segment s in buffer s % 2
    auto hist = [&](int64_t s, int64_t m, int c) {
        return (float*)(sc + A.off_hist + (((size_t)(s & 1) * (segment + 1) + m) * 3 + c) * fb);
    };
    auto seg_len = [&](int64_t s) { return (s + 1) * segment <= nsteps ? segment : nsteps - s * segment; };
    // The recompute of segment s - 1 (forward steps from its checkpoint,
    // keeping E at every level) runs on a second stream, beside the adjoint
    // steps of segment s on the handle's stream: the two touch different
    // memory (the grid's fields / the adjoint state; each its own history
    // buffer).  The recompute's step kernel takes one CTA per SM, leaving
    // the rest of each SM to the adjoint passes.
    AdjStreams X;
    if (!X.create()) return TF_ECUDA;
    cudaStream_t const user = h->stream;
    const int keep_blocks = h->step_blocks;
    auto recompute = [&](int64_t s) -> tf_status {
        h->stream = X.rs;
        h->step_blocks = keep_blocks < X.sms ? keep_blocks : X.sms;
        tf_status r = ckpt_restore_async(h, sc + A.off_ck + s * A.ck, s * segment, s > 0 ? 1 : 0);
        const int64_t len = seg_len(s);
        for (int64_t m = 0; r == TF_OK && m <= len; ++m) {
            float* const dst[3] = {hist(s, m, 0), hist(s, m, 1), hist(s, m, 2)};
            if (launch_copy3(dst, h->P.E, h->L.total, h->stream) != cudaSuccess) r = TF_ECUDA;
            else if (m < len) r = tf_step(h, 1);
        }
        if (r == TF_OK && cudaEventRecord(X.evR[s & 1], X.rs) != cudaSuccess) r = TF_ECUDA;
        h->stream = user;
        h->step_blocks = keep_blocks;
        return r;
    };
    if ((rc = recompute(A.nseg - 1)) != TF_OK) return rc;
    for (int64_t s = A.nseg - 1; s >= 0; --s) {
        // this segment's history is complete
        TF_CUDA(cudaStreamWaitEvent(user, X.evR[s & 1], 0));
        if (s > 0) {   // the previous segment's recompute into the other buffer, once its last reader is done
            if (s + 1 < A.nseg) TF_CUDA(cudaStreamWaitEvent(X.rs, X.evA[(s + 1) & 1], 0));
            if ((rc = recompute(s - 1)) != TF_OK) return rc;
        }
        const int64_t len = seg_len(s);
        // adjoint steps back through the segment
        for (int64_t m = len - 1; m >= 0; --m) {
            const int64_t n = s * segment + m;
            AdjStep st;
            for (int c = 0; c < 3; ++c) {
                st.En[c] = hist(s, m, c);
                st.En1[c] = hist(s, m + 1, c);
            }
            st.probe_comp = h->R.comp[probe];
            st.probe_q = h->R.q[probe];
            st.probe_src = 0.f;
            if (n >= n0) {   // dJ/dE^n = 2 dt Re(conj(X) exp(-i 2 pi f dt n))
                double ph = f * h->dt * (double)n;
                ph -= floor(ph);
                const double ang = 6.283185307179586476925286766559 * ph;
                st.probe_src = (float)(seed_scale * 2.0 * h->dt * (xr * cos(ang) - xi * sin(ang)));
            }
            const double t1 = (double)(n + 1) * h->dt;
            for (int q = 0; q < h->nsrc; ++q) src.amp[q] = (float)(h->src[q].amp * waveform(h->src[q], t1));
            TF_CUDA(launch_adjoint_step(h->P, S, src, st, h->O.tilemat, h->L.ntx, h->stream));
        }
        TF_CUDA(cudaEventRecord(X.evA[s & 1], user));
    }
    TF_CUDA(cudaStreamWaitEvent(user, X.evR[0], 0));   // the last recompute (segment 0)
    TF_CUDA(launch_adjoint_cells(h->P, S, (float)(kC0 * h->dt), 1.0 / seed_scale, grad_eps, grad_lambda,
                                 h->stream));
    // leave the handle in the state the forward run reached
    if ((rc = tf_checkpoint_load(h, sc + A.off_ck + A.nseg * A.ck, A.ck, 1)) != TF_OK) return rc;
    TF_CUDA(cudaStreamSynchronize(h->stream));
    return TF_OK;
}

tf_status tf_field_stats(tf_handle h, int comp, double* sumsq, double* maxabs, int64_t* nonfinite) {
    if (!h || comp < 0 || comp > 8) return TF_EINVAL;
    const float* f = comp < 3 ? h->P.E[comp] : comp < 6 ? h->P.B[comp - 3] : h->P.J[comp - 6];
    const double scale = comp < 3 ? 1.0 : comp < 6 ? 1.0 / kC0 : kEps0 / h->dt;
    StatPartial* part = (StatPartial*)(h->ws + h->L.off_stats);
    StatPartial* out = part + h->L.N[2];
    TF_CUDA(launch_field_stats(f, h->L.N[0], h->L.N[1], h->L.N[2], h->L.pitch, h->P.plane, scale, part, out,
                               h->stream));
    StatPartial r;
    TF_CUDA(cudaMemcpyAsync(&r, out, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
    TF_CUDA(cudaStreamSynchronize(h->stream));
    if (sumsq) *sumsq = r.sumsq;
    if (maxabs) *maxabs = r.maxabs;
    if (nonfinite) *nonfinite = (int64_t)r.nonfinite;
    return TF_OK;
}

tf_status tf_fit_q(tf_handle h, int id, double f_guess, double q_guess, double* f0, double* alpha, double* q) {
    if (!h || id < 0 || id >= h->R.n) return TF_EINVAL;
    if (h->R.nfreq[id] < 4 || !(q_guess > 0)) return TF_EINVAL;
    if (h->level <= h->R.n0[id]) return TF_ESTATE;
    TF_CUDA(launch_fit_q(h->R.re + id * TF_MAX_FREQS, h->R.im + id * TF_MAX_FREQS,
                         h->R.fdt + id * TF_MAX_FREQS, h->R.nfreq[id], h->dt, h->R.n0[id], h->level, f_guess,
                         q_guess, h->fit_out, h->stream));
    double o[4];
    TF_CUDA(cudaMemcpyAsync(o, h->fit_out, sizeof(o), cudaMemcpyDeviceToHost, h->stream));
    TF_CUDA(cudaStreamSynchronize(h->stream));
    if (!(o[3] > 0)) return TF_ENOTSUP;   // fit did not converge
    if (f0) *f0 = o[0];
    if (alpha) *alpha = o[1];
    if (q) *q = o[2];
    return TF_OK;
}

}  // extern "C"
