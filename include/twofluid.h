/*
 * twofluid.h -- C ABI of the GB300 two-fluid (Maxwell + London + Ohmic)
 * Yee FDTD library, after arXiv 2305.13419.
 *
 * Model (Sec. 2, Eqs. Ampere, Faraday, London1a):
 *     curl H = sigma_n E + Js + eps dE/dt,   curl E = -dB/dt,
 *     dJs/dt = E / (lambda_L^2 mu),           B = mu H.
 * Discretisation (Sec. 3, Algorithm 1): Yee grid, E on edges at integer time
 * levels, B on faces and Js on E edges at half levels; the Ohmic current is
 * taken with the theta scheme of Alg. 1 step 3.  The library advances the
 * algebraically identical fused leapfrog (Alg. 1 steps 5+1 and 4+2 merged),
 * so one tf_step() call of N steps moves (E^n, B^{n-1/2}, Js^{n-1/2}) to
 * (E^{n+N}, B^{n+N-1/2}, Js^{n+N-1/2}); field reads return integer levels.
 *
 * Grid and storage convention (shared by every call that takes a field):
 *   - nx, ny, nz cells of size dx, dy, dz.  An axis has N = n points when it
 *     is periodic and N = n + 1 points (both walls) otherwise.
 *   - field arrays are dense float32 [Nz][Ny][Nx] (x fastest).  Point (i,j,k)
 *     holds Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2) Bx(i,j+1/2,k+1/2)
 *     By(i+1/2,j,k+1/2) Bz(i+1/2,j+1/2,k) and Js on the E positions.  Values
 *     that fall outside the domain, tangential E on PEC/CPML walls and normal
 *     B on walls are held at zero; Js is held at zero on edges whose material
 *     is not superconducting.
 *   - material maps are dense float32 [nz][ny][nx] over cells.
 *   - units are SI (V/m, T, A/m^2, S/m, m, s).
 *
 * Errors: every call returns a tf_status; nothing is reported any other way.
 * Arguments are validated before any GPU work is enqueued.  Device faults and
 * the non-finite watchdog are latched and surface at tf_sync().
 *
 * Ownership: the caller owns the device workspace (tf_workspace_size bytes)
 * and every host or device buffer passed in; the library copies what it
 * keeps and never allocates device memory.  A handle is not thread-safe; all
 * GPU work of a handle is enqueued on the stream given in its descriptor.
 */
#ifndef TWOFLUID_H
#define TWOFLUID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TF_MAX_PROBES 16
#define TF_MAX_FREQS 64
#define TF_MAX_SOURCES 16

typedef struct tf_ctx* tf_handle;

typedef enum {
    TF_OK = 0,
    TF_EINVAL = 1,      /* bad argument (null pointer, out of range, bad descriptor) */
    TF_ENOMEM = 2,      /* workspace smaller than tf_workspace_size() */
    TF_ECUDA = 3,       /* a CUDA runtime call failed (launch, copy, device fault) */
    TF_EUNSTABLE = 4,   /* time step violates the stability bound of the scheme */
    TF_ESTATE = 5,      /* call not allowed in the handle's current state */
    TF_ETIMEOUT = 6,    /* a bounded device wait gave up */
    TF_ENONFINITE = 7,  /* the watchdog saw a non-finite E value */
    TF_ENOTSUP = 8      /* valid request the library does not support */
} tf_status;

/* boundary kinds (Sec. 3: periodic, PEC and PML; Mur offered for quasi-1-D runs) */
enum { TF_BC_PERIODIC = 0, TF_BC_PEC = 1, TF_BC_MUR = 2, TF_BC_CPML = 3 };
/* soft-source waveforms s(t) (Secs. 4.1, 4.2, 5):
 *   GAUSS     exp(-(t-t0)^2 / (2 tw^2))
 *   SIN       sin(2 pi f t)
 *   GAUSS_SIN exp(-(t-t0)^2 / (2 tw^2)) sin(2 pi f t)                 */
enum { TF_SRC_GAUSS = 0, TF_SRC_SIN = 1, TF_SRC_GAUSS_SIN = 2 };
enum { TF_EX = 0, TF_EY, TF_EZ, TF_BX, TF_BY, TF_BZ, TF_JSX, TF_JSY, TF_JSZ };
/* edge material rule (Sec. 3: edges on an SC interface are superconducting) */
enum { TF_EDGE_CONDUCTOR_MEAN = 0, TF_EDGE_PLAIN_MEAN = 1 };

/* One axis' boundary, applied to both of its faces.
 *   TF_BC_CPML: Roden-Gedney convolutional PML, kappa = 1, backed by PEC;
 *     over `cpml_cells` cells the conductivity grows as
 *     sigma_max rho^order and the frequency shift falls as alpha_max (1-rho),
 *     rho = depth into the layer / cpml_cells.  2 cpml_cells <= n.
 *   TF_BC_MUR: first-order Mur, z axis only.                              */
typedef struct {
    int kind;
    int cpml_cells;
    double cpml_order;
    double cpml_sigma_max;   /* S/m */
    double cpml_alpha_max;   /* S/m */
} tf_bc;

typedef struct {
    int nx, ny, nz;          /* cells, each >= 1 */
    double dx, dy, dz;       /* m, > 0 */
    double dt;               /* s; if <= 0, dt = courant / (c sqrt(1/dx^2+1/dy^2+1/dz^2)) */
    double courant;          /* used only when dt <= 0; the paper's convention (Secs. 4-5) */
    double theta;            /* Ohmic time weighting of Alg. 1 step 3, in [0.5, 1] */
    tf_bc bc[3];             /* x, y, z */
    int edge_rule;           /* TF_EDGE_* */
    int max_probes;          /* 0 .. TF_MAX_PROBES */
    int64_t series_capacity; /* time levels each probe may record (0 = none) */
    void* stream;            /* cudaStream_t for all GPU work of the handle (NULL = default) */
} tf_grid_desc;

/* Bytes of device workspace a grid with this descriptor needs; 0 if the
 * descriptor is invalid.  Host-only, no GPU call. */
size_t tf_workspace_size(const tf_grid_desc* desc);

/* Create a grid in the caller's device workspace (>= tf_workspace_size bytes,
 * 256-byte aligned).  Fields start at zero, materials at vacuum
 * (eps_r = mu_r = 1, lambda_L = 0, sigma = 0).  *out receives the handle.
 * TF_EINVAL bad descriptor, TF_ENOMEM workspace too small, TF_ENOTSUP Mur on x/y,
 * TF_ECUDA failed clears. */
tf_status tf_create(const tf_grid_desc* desc, void* dev_workspace, size_t bytes, tf_handle* out);

/* Release the host side of the handle (the workspace stays the caller's). */
tf_status tf_destroy(tf_handle h);

/* Storage points per axis (N = n, or n + 1 on a non-periodic axis). */
tf_status tf_storage_dims(tf_handle h, int dims[3]);

/* Current integer level n and time n * dt; dt of the grid. */
tf_status tf_get_time(tf_handle h, int64_t* n, double* t);
tf_status tf_get_dt(tf_handle h, double* dt);

/* Per-cell material maps (Sec. 2: eps = eps0 eps_r, mu = mu0 mu_r, lambda_L
 * London depth, sigma normal-fluid conductivity; Sec. 3: 1/lambda -> 0 off
 * the superconductor, so lambda_L = 0 marks a non-superconducting cell).
 * Dense [nz][ny][nx] float32, host (on_device = 0) or device pointers; NULL
 * keeps the vacuum default for that map.  Copied; the caller keeps ownership.
 * Edge values: eps is the mean over the four cells sharing an edge; sigma and
 * kappa = 1/(lambda^2 mu) follow edge_rule; a face takes the mean mu of its two
 * cells.  Only before the first tf_step().  Checks eps_r, mu_r > 0,
 * sigma >= 0, lambda_L >= 0 (TF_EINVAL) and the stability bound
 * C^2 max 1/(eps_r mu_r) + max (c dt / (2 lambda_L))^2 / (eps_r mu_r) <= 1 (TF_EUNSTABLE).
 * Synchronises the handle's stream. */
tf_status tf_set_materials(tf_handle h, const float* eps_r, const float* mu_r,
                           const float* lambda_L, const float* sigma, int on_device);

/* Initial value (level 0) of one component, SI, dense [Nz][Ny][Nx] float32,
 * host or device.  Only before the first tf_step() (TF_ESTATE otherwise).
 * Points the convention holds at zero are zeroed. */
tf_status tf_set_field(tf_handle h, int comp, const float* src, int on_device);

/* Soft source (Secs. 4.2, 5): after each E update, E_comp += amp * s(t^{n+1})
 * on every advanced E_comp point of the storage box [lo, hi).  comp in
 * TF_EX..TF_EZ; up to TF_MAX_SOURCES; *id (may be NULL) receives its index. */
tf_status tf_add_source(tf_handle h, int comp, const int lo[3], const int hi[3], double amp,
                        int kind, double f, double t0, double tw, int* id);

/* Point probe with a running FP64 DFT (Sec. 4.2 Fourier-transforms probe
 * signals, Sec. 5 extracts Q from them): at the start of every step n the
 * library samples s^n = E_comp(p) and, for n >= n0, adds
 * s^n exp(-i 2 pi frac(f_k dt n)) dt to X_k, k < nfreq <= TF_MAX_FREQS.
 * With series_capacity > 0 it also records s^n for n < series_capacity.
 * Up to max_probes; *id (may be NULL) receives its index. */
tf_status tf_add_probe(tf_handle h, int comp, const int p[3], const double* freqs, int nfreq,
                       int64_t n0, int* id);

/* Advance nsteps >= 0 steps of Algorithm 1 (fused form) on the stream:
 * per step one probe-DFT launch and one fused launch doing the B update with
 * CPML memory, the Js update, the theta-scheme E update with sources, the
 * Mur walls and the non-finite watchdog.  Asynchronous; launch errors are
 * returned (the handle is then unusable), device-side errors latch for
 * tf_sync(). */
tf_status tf_step(tf_handle h, int64_t nsteps);

/* tf_step with per-kernel timing (the library's profiling hook): advances
 * nsteps exactly like tf_step and records a CUDA event pair on the handle's
 * stream around every kernel it launches.  On return (the stream is
 * synchronised) kernel_ms[k] is the mean duration in ms of one launch of
 * kernel kind k and launches[k] the number of launches, for k = 0 a separate
 * probe DFT kernel (no longer launched: the fused step adds E^n at the probes
 * to their DFTs while its ring fills, so launches[0] stays 0) and k = 1 the
 * fused step and k = 2 the two-step kernel of tf_set_two_step (arrays of
 * nkinds <= 3 entries; a two-step pass counts one launch of kind 2 and two
 * of kind 1).  total_ms (may be NULL)
 * receives the event time from the first launch's start to the last
 * launch's end: the same launches' whole-run time.  Up to 4096 steps are
 * enqueued before the call waits on the stream (longer runs wait once per
 * 4096 launch groups, and total_ms then sums those batches).  Host memory for the
 * events is allocated per call (TF_ENOMEM if that fails). */
tf_status tf_step_timed(tf_handle h, int64_t nsteps, double* kernel_ms, int64_t* launches, int nkinds,
                        double* total_ms);

/* Temporal blocking: two time steps of Algorithm 1 (Sec. 3) per pass over
 * the memory.  tf_step advances a grid two steps at a time where it can: a
 * two-step kernel moves the interior box -- the tiles and planes whose
 * points, with a two-point halo, lie off the walls, off the Mur planes and
 * outside the CPML slabs -- from level n to n + 2 in one pass, and the
 * single-step kernel moves the rest of the grid twice.  The results are the
 * same bits as single steps.  It is used when the box is not empty, mu is
 * uniform (tf_set_materials) and it is enabled; an odd step count ends with a
 * single step.
 *   tf_set_two_step  planes = 0 disables it for this handle; 4 .. 24 enables
 *                    it with work items of that many planes (24 by default);
 *                    other values TF_EINVAL.  A tuning switch (the project's
 *                    autotuner sets it per grid): results do not change.
 *   tf_two_step_box  the box in storage points, [lo, hi) per axis (all zero
 *                    when the geometry has none), and in *active (may be
 *                    NULL) whether tf_step uses it. */
tf_status tf_set_two_step(tf_handle h, int planes);
tf_status tf_two_step_box(tf_handle h, int lo[3], int hi[3], int* active);

/* Planes per work item of the single-step kernel (its items, and the
 * shell's items in two-step passes): 8 .. 16 (8 by default; other
 * values TF_EINVAL).  Longer items re-read fewer z halo planes and change
 * items less often; shorter ones balance a small grid's few items over the
 * CTAs better.  A tuning switch (the project's autotuner sets it per grid):
 * results do not change. */
tf_status tf_set_item_planes(tf_handle h, int planes);

/* The stepping kernels wait on an mbarrier for every plane they stage; each
 * wait polls it at most `polls` times (default 2^22, far beyond a copy's
 * latency).  A wait that runs out latches TF_ETIMEOUT for tf_sync(): the
 * CTA then waits (with the default limit) for the copies it has in flight
 * and returns, leaving the grid's fields undefined (the context stays
 * usable; reload a checkpoint or rebuild the grid).  polls < 0 restores the
 * default; polls = 0 makes every wait give up at once (a test of the error
 * path).  Applies to the handle's later launches, batched ones included. */
tf_status tf_set_wait_limit(tf_handle h, int64_t polls);

/* Advance n independent grids by nsteps steps each (the batched workload:
 * many resonator variants at once).  The grids advance together, one step
 * of every grid in turn; each grid's work goes to its own handle's stream,
 * so grids on different streams overlap (one grid's last work items run
 * beside the next grid's first ones).  Handles must be distinct; the call
 * returns after enqueueing (use tf_sync per handle). */
tf_status tf_batch_step(const tf_handle* hs, int n, int64_t nsteps);

/* One launch per step over every grid of a batch (many resonator variants
 * of uneven sizes): the work items of all grids form one list (each grid's
 * own items, the grid's index in the descriptor; the items with CPML
 * corners, sources or Mur planes of every grid first) that the single-step
 * kernel's CTAs share through one counter, each item run with its grid's
 * arguments; 64 steps at a time are captured in a CUDA graph and replayed
 * (the step number lives on the device and a one-thread launch advances it
 * after each step).  Every grid ends with the same bits as tf_step (single
 * steps) would give it.
 *   hs, n      handles (distinct, n <= 32768); the run is issued on hs[0]'s
 *              stream after every handle's stream has been synchronised, and
 *              synchronises it;
 *   scratch    caller-owned device memory (256-byte aligned) of at least
 *              tf_batch_scratch_size bytes: the per-grid arguments, the work
 *              list and the source amplitudes of every step (TF_ENOMEM if
 *              smaller).
 * Creating the CUDA graph may make the CUDA runtime allocate. */
tf_status tf_batch_scratch_size(const tf_handle* hs, int n, int64_t nsteps, size_t* bytes);
tf_status tf_batch_run(const tf_handle* hs, int n, int64_t nsteps, void* scratch, size_t bytes);

/* Wait for the stream and return the latched device status
 * (TF_ENONFINITE if the watchdog saw a non-finite E). */
tf_status tf_sync(tf_handle h);

/* Copy probe id's DFT accumulators (FP64, nfreq values each) to host arrays. */
tf_status tf_read_probe_dft(tf_handle h, int id, double* re, double* im);

/* Copy the first n recorded samples (n <= min(level, series_capacity)). */
tf_status tf_read_probe_series(tf_handle h, int id, double* out, int64_t n);

/* Integer-level value of one component at the current level (Alg. 1 steps
 * 4-5 applied to the half-level state: B^n = B^{n-1/2} - dt/2 curl E^n,
 * Js^n = Js^{n-1/2} + dt/2 E^n/(lambda^2 mu)), SI, dense [Nz][Ny][Nx]
 * float32 into a host or device buffer.  Synchronises the stream. */
tf_status tf_read_field(tf_handle h, int comp, float* dst, int on_device);

/* Checkpoint of the time-stepping state, so that a run of Algorithm 1 (the
 * paper's resonator runs take 10^5 - 10^6 steps, Sec. 5) can stop and resume
 * bit-identically.  The blob holds a header (grid sizes, level, priming
 * state), E, B, Js at the level the state holds them, the CPML memories and
 * the probe DFT accumulators and series.  It does not hold the
 * configuration: materials, sources and probe definitions must be set on the
 * handle before tf_checkpoint_load exactly as they were when the blob was
 * saved (the header checks sizes, boundary layout, probe count and dt).
 *   tf_checkpoint_size  bytes of a blob for this handle;
 *   tf_checkpoint_save  writes the blob to dst (host memory, or device memory
 *                       when on_device != 0); bytes >= tf_checkpoint_size;
 *   tf_checkpoint_load  restores the state from src; TF_EINVAL when the
 *                       header does not match this handle.
 * The caller owns dst / src.  Both synchronise the stream. */
tf_status tf_checkpoint_size(tf_handle h, size_t* bytes);
tf_status tf_checkpoint_save(tf_handle h, void* dst, size_t bytes, int on_device);
tf_status tf_checkpoint_load(tf_handle h, const void* src, size_t bytes, int on_device);

/* Discrete adjoint of the time stepping (Algorithm 1, Sec. 3): the gradient
 * of the objective J = |X_k|^2 -- X_k the FP64 DFT of probe `probe` at its
 * frequency index k over its window [n0, nsteps) -- with respect to the
 * relative permittivity and the London depth of every cell.
 *   The handle must hold the state at rest before its first step (level 0,
 *   not yet stepped; fields as set, normally zero) with materials, sources
 *   and probes configured; no Mur walls (TF_ENOTSUP).  The call runs nsteps
 *   forward, saving a checkpoint every `segment` steps into the scratch,
 *   then walks the segments backwards: each is recomputed from its
 *   checkpoint with E kept at every level, and the transposed step runs back
 *   through it, summing per-edge gradients in FP64.  The recompute of the
 *   segment before runs on a second stream of the library's (created and
 *   destroyed by the call) beside those transposed steps, into the other of
 *   two history buffers.  The adjoint's seed is
 *   scaled by a power of two to O(1) (and the gradients scaled back), so the
 *   FP32 adjoint state stays in FP32's normal range for any source size.
 *   scratch   caller-owned device memory of at least tf_adjoint_scratch_size
 *             bytes (checkpoints, two segments of E history, the adjoint
 *             state, the gradient sums); TF_ENOMEM if smaller;
 *   J         host double: the objective;
 *   grad_eps, grad_lambda  device float arrays [nz][ny][nx] (cells):
 *             dJ/d eps_r and dJ/d lambda_L (per metre), the latter 0 on
 *             cells that are not superconducting.
 * On return the handle holds the state after nsteps (as tf_step would).
 * Synchronises the stream. */
tf_status tf_adjoint_scratch_size(tf_handle h, int64_t nsteps, int segment, size_t* bytes);
tf_status tf_adjoint_run(tf_handle h, int64_t nsteps, int probe, int freq_index, int segment, void* scratch,
                         size_t bytes, double* J, float* grad_eps, float* grad_lambda);

/* Q-factor of one damped mode from probe id's DFT (Sec. 5 reports Q and the
 * resonance from the ring-down): fits X_k = dt sum_{n0<=n<N} (a z^n + c.c.)
 * w_k^n, z = exp((-alpha + i omega0) dt), in FP64 on the GPU.  f_guess and
 * q_guess start the search (f_guess <= 0: the strongest bin).  Outputs
 * f0 (Hz), alpha (1/s) and Q = omega0 / (2 alpha); any output may be NULL. */
tf_status tf_fit_q(tf_handle h, int id, double f_guess, double q_guess, double* f0,
                   double* alpha, double* q);

/* Watchdog statistics of one stored field array (the non-finite / blow-up
 * check of the step loop): sum of squares, largest magnitude and number of
 * NaN / Inf values of component comp over all storage points, in SI units.
 * E is read at the current integer level, B and Js at the half level the
 * state holds them (n - 1/2).  Uses a scratch area of the workspace (one
 * partial per z plane).  Synchronises the stream; any output may be NULL. */
tf_status tf_field_stats(tf_handle h, int comp, double* sumsq, double* maxabs, int64_t* nonfinite);

/* Allocation-free twin of tf_field_stats.  The paper has no counterpart: it
 * exists for callers that cannot allocate device memory when they need the
 * check -- a monitoring thread that must not take the CUDA allocator's lock
 * or trigger the device-wide synchronisation of cudaFree while the
 * simulation runs, or a host application whose memory pool already holds
 * (nearly) all of the device.  It allocates nothing: no cudaMalloc, no
 * cudaFree, no allocating library call.
 *   field        device pointer to one float32 array of nx_pts x ny_pts x
 *                nz_pts points, x fastest, rows `pitch` floats apart
 *                (pitch >= nx_pts), planes pitch * ny_pts floats apart;
 *   scale        factor applied to every value (1 for values already in SI);
 *   outputs      sum of squares, largest magnitude, number of NaN / Inf
 *                values (host pointers; any may be NULL);
 *   stream       cudaStream_t to run on (NULL = default stream).
 * Its scratch is a fixed 4097-entry array (about 96 KiB) inside the library
 * that every GPU loading the library keeps until the process exits; nz_pts
 * above 4096 is rejected with TF_EINVAL.  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress) with the device
 * current, so make that first call before any stream capture.  All calls
 * share the array and each one overwrites it completely; calls that overlap
 * on the GPU (different streams or threads at once) race on it.  Synchronises
 * `stream`. */
tf_status tf_field_stats_noalloc(const float* field, int nx_pts, int ny_pts, int nz_pts, int pitch, double scale,
                                 double* sumsq, double* maxabs, int64_t* nonfinite, void* stream);

/* FP64 stepper: the precision reference of the FP32 path (the study of how
 * far FP32 fields drift over long runs).  Runs Algorithm 1 (Sec. 3) as its
 * five sub-steps in FP64 and SI units on the integer-level state, with the
 * same edge/face material rule, boundaries (periodic, PEC, CPML, Mur on z),
 * soft sources and FP64 probe DFTs as the FP32 path.  Fields are dense
 * float64 [Nz][Ny][Nx] (no row padding), host buffers; materials dense
 * float64 [nz][ny][nx] on the host.  Same descriptor as tf_create; the
 * workspace is caller-owned device memory (256-byte aligned) of
 * tf64_workspace_size bytes.  tf64_step enqueues on the descriptor's
 * stream; reads synchronise it.  Errors as for the FP32 calls. */
typedef struct tf64_ctx* tf64_handle;
size_t tf64_workspace_size(const tf_grid_desc* desc);
tf_status tf64_create(const tf_grid_desc* desc, void* dev_workspace, size_t bytes, tf64_handle* out);
tf_status tf64_destroy(tf64_handle h);
tf_status tf64_set_materials(tf64_handle h, const double* eps_r, const double* mu_r, const double* lambda_L,
                             const double* sigma);
tf_status tf64_set_field(tf64_handle h, int comp, const double* src);
tf_status tf64_add_source(tf64_handle h, int comp, const int lo[3], const int hi[3], double amp, int kind,
                          double f, double t0, double tw, int* id);
tf_status tf64_add_probe(tf64_handle h, int comp, const int p[3], const double* freqs, int nfreq, int64_t n0,
                         int* id);
tf_status tf64_step(tf64_handle h, int64_t nsteps);
tf_status tf64_sync(tf64_handle h);
tf_status tf64_read_field(tf64_handle h, int comp, double* dst);
tf_status tf64_read_probe_dft(tf64_handle h, int id, double* re, double* im);
tf_status tf64_get_time(tf64_handle h, int64_t* n, double* dt);

/* The FP64 FMA rate of the current device, the arithmetic ceiling of the
 * FP64 stepper (a measurement for the FP32-vs-FP64 study; the paper has no
 * counterpart).  Runs a kernel of independent FP64 FMA chains, `iters`
 * rounds per thread, on `stream` (a cudaStream_t, NULL for the default
 * stream), timed with CUDA events after one untimed run, and writes GFLOP/s
 * (2 per FMA) to *gflops.  dev_scratch: device memory of at least
 * tf64_fma_rate_scratch() bytes (caller-owned; overwritten).  Synchronises
 * the stream.  TF_EINVAL on a null pointer or iters < 1, TF_ENOMEM if the
 * scratch is too small, TF_ECUDA on a CUDA error. */
size_t tf64_fma_rate_scratch(void);
tf_status tf64_fma_rate(void* dev_scratch, size_t bytes, int iters, void* stream, double* gflops);

const char* tf_strerror(tf_status s);

#ifdef __cplusplus
}
#endif
#endif
