/*
 * kbc.h -- C ABI of the GB300 (sm_103a) D2Q9 KBC lattice Boltzmann library.
 *
 * The library advances a doubly periodic nx x ny D2Q9 population field with
 * the fused pull-stream + collide update of Eq. Egeneral (Sec. 1), where the
 * post-collision state uses the one-parameter KBC mirror state of
 * Eq. ksh-mirror (Sec. 2) with the moment grouping of Table 1 (variants A-D)
 * and the entropic stabiliser gamma* of Eq. result21 (Sec. 4), or the plain
 * LBGK mirror of Eq. LBGKmirr.  Reference: Bosch, Chikatamarla, Karlin,
 * "Entropic multi-relaxation models for simulation of fluid turbulence".
 *
 * Conventions shared by every call
 * --------------------------------
 * Status.   Every call returns a kbc_status (0 = KBC_OK, negative = error)
 *           and never aborts, traps or exits.  kbc_last_error(h) gives a
 *           human-readable message for the last failing call on h.
 * Layout.   Scalar fields are [ny][nx] row-major, x fastest.  Velocity
 *           fields are [2][ny][nx] (u_x plane, then u_y plane).  Population
 *           fields are [9][ny][nx] with population index i = 3(b+1) + (a+1)
 *           for the lattice velocity v_i = (a, b), a, b in {-1, 0, 1}.
 *           All external fields are IEEE double.
 * Pointers. Field pointers may be host memory (pageable or pinned) or device
 *           memory of the handle's device; the library tells them apart
 *           with cudaPointerGetAttributes and stages host data through a
 *           device buffer.  Caller memory is borrowed only for the duration
 *           of the call.
 * Ordering. All device work is issued on the stream bound with
 *           kbc_set_stream (default: the legacy default stream), except the
 *           chunked host transfers of kbc_init / kbc_moments, which use a
 *           second stream owned by the handle and are ordered against the
 *           bound stream with events (the bound stream sees them as part of
 *           the call).  Calls that return device results into device memory
 *           are asynchronous on that stream; calls that return host results
 *           (host pointers, kbc_diagnostics, kbc_adjoint's scalars)
 *           synchronise that stream only, with a bounded wait
 *           (KBC_ERR_TIMEOUT).
 * Threads.  A handle is not thread-safe: calls on one handle must not run
 *           concurrently.  Different handles may be used from different
 *           host threads.
 * State.    After kbc_init and n steps the handle holds the post-collision
 *           field f'(., n) of Eq. Egeneral.  rho and u are the same for the
 *           pre- and post-collision fields because the collision conserves
 *           them (Eq. k_conservation, Eq. sh_conservation).
 * Memory.   The handle owns its device buffers (two population fields, the
 *           A-B pair, plus small scratch), obtained from the allocator set
 *           with kbc_set_allocator at kbc_create time (default cudaMalloc).
 */
#ifndef KBC_GB300_H
#define KBC_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kbc_ctx* kbc_handle;

/* Collision model: LBGK (Eq. LBGKmirr) or the KBC variants of Table 1.
 * A: s = {Pi~, N~, T~}, B: s = {Pi~, N~} (central moments, Sec. 2, Eq. cm);
 * C: s = {Pi, N, T},   D: s = {Pi, N}   (natural moments, Eq. natmoments1). */
enum kbc_variant { KBC_LBGK = 0, KBC_A = 1, KBC_B = 2, KBC_C = 3, KBC_D = 4 };

/* Storage of the population field in device memory.
 * KBC_F64:     f_i - W_i in IEEE double, arithmetic in double.
 * KBC_F32_DEV: f_i - W_i in float, arithmetic in float (moment sums and gamma
 *              in float, with an FP64 re-evaluation of nodes whose
 *              <dh|dh> falls below the guard, see kbc_set_guard).
 * KBC_F16_DEV: (f_i - W_i) / W_i * S in IEEE half with a per-run scale S
 *              (kbc_set_f16_scale), arithmetic in float. */
enum kbc_dtype { KBC_F64 = 0, KBC_F32_DEV = 1, KBC_F16_DEV = 2 };

/* gamma of Eq. result21 (entropic, the paper's choice), a fixed value (2
 * reproduces LBGK, 1/beta the regularised limit discussed after
 * Eq. dsdh1B), or the root of the exact entropic condition Eq. result1
 * (Newton from gamma*, in double precision whatever the storage, by a
 * per-node kernel; gamma* is kept where an iterate leaves the domain of
 * positive post-collision populations or 30 iterations pass). */
enum kbc_gamma_mode { KBC_GAMMA_ENTROPIC = 0, KBC_GAMMA_FIXED = 1, KBC_GAMMA_EXACT = 2 };

enum kbc_status {
    KBC_OK = 0,
    KBC_ERR_ARG = -1,       /* invalid argument or size                       */
    KBC_ERR_CUDA = -2,      /* a CUDA runtime call failed                     */
    KBC_ERR_NOMEM = -3,     /* the allocator returned NULL                    */
    KBC_ERR_NONFINITE = -4, /* the field holds NaN or Inf (the update blew up) */
    KBC_ERR_TIMEOUT = -5,   /* a bounded wait on the stream ran out           */
    KBC_ERR_STATE = -6      /* call out of order (e.g. step before init)      */
};

/* Number of doubles written by kbc_diagnostics and kbc_diagnostics_ext. */
#define KBC_DIAG_N 10
#define KBC_DIAG_EXT_N 4
/* Number of doubles in one partial diagnostics set (kbc_diagnostics_partial). */
#define KBC_DIAG_PART_N 11

/* Device allocator hook: returns a device pointer of at least `bytes` bytes
 * (256-byte aligned) or NULL; `stream` is the handle's bound stream. */
typedef void* (*kbc_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*kbc_free_fn)(void* ptr, void* stream, void* user);

/* Set the process-wide allocator used by subsequent kbc_create calls
 * (NULL, NULL restores cudaMalloc/cudaFree).  A handle frees its buffers
 * with the allocator it was created with. */
int kbc_set_allocator(kbc_alloc_fn alloc, kbc_free_fn release, void* user);

/* Create a handle for an nx x ny doubly periodic grid on the current CUDA
 * device.  beta is the relaxation parameter of Eq. Egeneral, related to the
 * kinematic viscosity by nu = cs^2 (1/(2 beta) - 1/2), cs^2 = 1/3
 * (Eq. viscosity).  Requirements: nx, ny >= 1, nx * ny <= 2^31 - 1,
 * 0 < beta <= 1, variant and dtype from their enums; else KBC_ERR_ARG.
 * Grids with nx a multiple of the vector row width (128 for F32 and F16, 64
 * for F64) take the vectorised row kernel, all others a per-node kernel
 * with the same arithmetic.  *out is NULL on failure. */
int kbc_create(int nx, int ny, int variant, double beta, int dtype, kbc_handle* out);

/* y-slab of a larger doubly periodic grid, for a domain split into
 * horizontal slabs (one per GPU or per handle).  The paper runs one periodic
 * grid; the split follows from the pull of Eq. Egeneral, which reaches one
 * row up and one row down: a step of rows [y0, y0 + ny) needs, besides
 * them, the three populations with b = +1 (i = 6, 7, 8) of row y0 - 1 and
 * the three with b = -1 (i = 0, 1, 2) of row y0 + ny, taken periodically in
 * the global grid.  The handle holds the ny interior rows plus a ghost row
 * below and above; x stays periodic within the handle.  Interior rows are
 * addressed as on a plain handle (kbc_init, kbc_set_populations,
 * kbc_get_populations, kbc_probe, kbc_moments take [.][ny][nx] fields of the
 * slab's own rows).  Before every step, each face's ghost row must be filled
 * with kbc_halo_recv from the neighbouring slab's kbc_halo_send (the slab
 * itself when it is the whole periodic grid); kbc_step then advances one
 * step (nsteps <= 1, else KBC_ERR_ARG).  Ghost rows start at f = W.
 * Global diagnostics of a split grid: kbc_diagnostics_partial per slab
 * (after full halos), combined with kbc_diagnostics_merge.
 * kbc_diagnostics, kbc_diagnostics_ext, kbc_init_grad and kbc_adjoint need
 * rows beyond the ghost rows or the whole grid and give KBC_ERR_ARG on a
 * slab handle.  Same requirements as kbc_create, with
 * nx * (ny + 2) <= 2^31 - 1. */
int kbc_create_slab(int nx, int ny, int variant, double beta, int dtype, kbc_handle* out);

/* Halo of one face of a y-slab handle, in the handle's storage encoding
 * (the stored deviations, see enum kbc_dtype), populations in increasing
 * index, each an nx-element row.
 *   full = 0: the three populations that cross the face, [3][nx] -- what a
 *   step needs:
 *     kbc_halo_send(h, 0, 0, buf): bottom interior row, populations 0, 1, 2
 *       (moving down: the lower neighbour's face-1 ghost row);
 *     kbc_halo_send(h, 1, 0, buf): top interior row, populations 6, 7, 8
 *       (moving up: the upper neighbour's face-0 ghost row);
 *     kbc_halo_recv(h, 0, 0, buf): into the ghost row below row 0,
 *       populations 6, 7, 8 (what the lower neighbour sent through face 1);
 *     kbc_halo_recv(h, 1, 0, buf): into the ghost row above row ny - 1,
 *       populations 0, 1, 2 (what the upper neighbour sent through face 0).
 *   full = 1: all nine populations of the same rows, [9][nx] -- what
 *     kbc_diagnostics_partial needs in the ghost rows (the neighbouring
 *     rows' velocity for the vorticity).
 * buf: host or device memory (KBC_ERR_ARG if NULL); device buffers are
 * asynchronous on the handle's stream, host buffers synchronise it.
 * KBC_ERR_ARG on a plain handle, a face other than 0 and 1 or full other
 * than 0 and 1; kbc_halo_send before the field is initialised gives
 * KBC_ERR_STATE. */
int kbc_halo_send(kbc_handle h, int face, int full, void* buf);
int kbc_halo_recv(kbc_handle h, int face, int full, const void* buf);

/* Bytes of one face's halo: 3 nx (full = 0) or 9 nx (full = 1) stored
 * elements. */
int kbc_halo_bytes(kbc_handle h, int full, size_t* bytes);

/* Free the handle's device buffers (after synchronising its stream). */
int kbc_destroy(kbc_handle h);

/* Bind a cudaStream_t (passed as void*); NULL = legacy default stream. */
int kbc_set_stream(kbc_handle h, void* cuda_stream);

/* gamma mode (enum kbc_gamma_mode) and the fixed gamma it uses (ignored by
 * the other modes).  Ignored by KBC_LBGK, whose mirror state has no gamma. */
int kbc_set_gamma_mode(kbc_handle h, int mode, double gamma_fixed);

/* Kernel used by kbc_step (all of them share the collision arithmetic, so
 * they give identical bits):
 *   KBC_KERNEL_AUTO  (default) the fastest choice measured on GB300 at 4096^2
 *                    and 16384^2: for F16 storage with a KBC variant the
 *                    bulk-copy kernel below where nx is a multiple of 512,
 *                    otherwise the vector-row kernel where nx is a multiple
 *                    of its row width, else the per-node kernel;
 *   KBC_KERNEL_ROWS  the vector-row kernel where nx allows it, else the
 *                    per-node kernel;
 *   KBC_KERNEL_NODES the per-node kernel;
 *   KBC_KERNEL_BULK  the persistent, warp-specialised kernel that stages each
 *                    512-node row tile in shared memory with bulk
 *                    asynchronous copies issued by a producer warp (F32/F16
 *                    with nx a multiple of 512; otherwise as AUTO). */
enum kbc_kernel { KBC_KERNEL_AUTO = 0, KBC_KERNEL_ROWS = 1, KBC_KERNEL_NODES = 2, KBC_KERNEL_BULK = 3 };
int kbc_set_kernel(kbc_handle h, int kernel);

/* kbc_step replays a CUDA graph of `steps` consecutive steps (captured once
 * per handle configuration on a private stream, then launched on the bound
 * stream) for as many whole graphs as nsteps holds, and launches the rest
 * one by one; this removes the per-launch overhead that dominates small
 * grids.  Graphs give the same bits as individual launches.  steps must be
 * even (the two population buffers return to their roles after an even
 * count); 0 disables graphs.  Default 32.  Not used while the bound stream
 * is itself being captured. */
int kbc_set_graph_steps(kbc_handle h, int steps);

/* Threshold on <dh|dh> (entropic scalar product of Sec. 4, computed with the
 * weights rho/f^eq_i) below which an F32/F16 node is recomputed entirely in
 * FP64 from its stored populations by a second pass.  0 disables the pass.
 * Defaults: 1e-16 for F32 (about 10x the float rounding level of that sum
 * for |u| ~ 0.03), 0 for F16; F64 ignores it. */
int kbc_set_guard(kbc_handle h, double threshold);

/* Number of nodes the FP64 guard pass re-evaluated in the most recent step
 * (synchronises the stream; 0 when the pass is off). */
int kbc_guard_count(kbc_handle h, long long* count);

/* Scale S of the F16 encoding (f - W)/W * S; must be set before kbc_init
 * (else KBC_ERR_STATE).  Default 1; S outside [2^-24, 2^24] (where the half
 * code or the float constants derived from S would over- or underflow) is
 * rejected with KBC_ERR_ARG. */
int kbc_set_f16_scale(kbc_handle h, double scale);

/* Initialise the field to the equilibrium f^eq(rho, u) of Eq. Eq at every
 * node.  rho: [ny][nx], u: [2][ny][nx]; host or device.  Host inputs of
 * 64 MB and more are uploaded in row chunks on a second stream owned by the
 * handle, each chunk's copy overlapping the initialisation of the previous
 * one (same result as device inputs, bit for bit). */
int kbc_init(kbc_handle h, const double* rho, const double* u);

/* Initialise with Grad's approximation (Eq. Grad) using the pressure tensor
 * Pi^eq + Pi^(1) of Eq. Peq and Eq. P1AC, velocity gradients by periodic
 * central differences of u. */
int kbc_init_grad(kbc_handle h, const double* rho, const double* u);

/* Overwrite / read the population field f[9][ny][nx] (FP64).  set rounds to
 * the handle's storage; get returns the stored values exactly. */
int kbc_set_populations(kbc_handle h, const double* f);
int kbc_get_populations(kbc_handle h, double* f);

/* Advance nsteps >= 0 time steps of Eq. Egeneral (pull f_i(x) = f'_i(x - v_i)
 * with periodic wrap, then collide).  Asynchronous: returns after enqueueing.
 * Returns KBC_ERR_NONFINITE if a NaN/Inf was detected by an earlier step of
 * this handle whose result has reached the host (the detection is copied
 * back asynchronously after each call; kbc_sync makes it current). */
int kbc_step(kbc_handle h, int nsteps);

/* Wait (bounded by timeout_s seconds; <= 0 means 600) for the handle's
 * stream; returns KBC_ERR_NONFINITE if any step so far produced NaN/Inf. */
int kbc_sync(kbc_handle h, double timeout_s);

/* Populations of selected nodes: f[k][9] (FP64) for node indices
 * nodes[k] = y * nx + x, k < count.  nodes and f may be host or device
 * memory; indices outside [0, nx*ny) give KBC_ERR_ARG (checked on the device,
 * reported after the call synchronises). */
int kbc_probe(kbc_handle h, int count, const long long* nodes, double* f);

/* rho [ny][nx] and u [2][ny][nx] of the current field (FP64); host or
 * device.  Host outputs of 64 MB and more are downloaded in row chunks on the
 * handle's second stream, overlapping the computation of the next chunk;
 * returns once the data are on the host. */
int kbc_moments(kbc_handle h, double* rho, double* u);

/* Global diagnostics (FP64 device reductions), out[KBC_DIAG_N] on the host:
 *   [0] sum rho  [1] sum rho u_x  [2] sum rho u_y
 *   [3] E = mean |u|^2/2   [4] Z = mean w^2/2, w = d_x u_y - d_y u_x by
 *       periodic central differences
 *   [5] mean, [6] min, [7] max of gamma of the collision the next step
 *       performs (2 for LBGK)
 *   [8] spatial std of |u|^2/2   [9] spatial std of w^2/2 */
int kbc_diagnostics(kbc_handle h, double* out);

/* The diagnostics of this handle's nodes as one partial set, to be combined
 * with other parts of the same grid (e.g. the slabs of a split grid, one per
 * rank) by kbc_diagnostics_merge: out[KBC_DIAG_PART_N] on the host =
 *   [0] sum rho  [1] sum rho u_x  [2] sum rho u_y  [3] node count
 *   [4] mean and [5] sum of squared deviations of |u|^2/2
 *   [6] mean and [7] sum of squared deviations of w^2/2
 *   [8] sum, [9] min, [10] max of gamma
 * with the definitions of kbc_diagnostics.  On a y-slab handle both ghost
 * rows must hold full halos (kbc_halo_recv with full = 1) received since the
 * field last changed (kbc_step, kbc_init, kbc_set_populations), else
 * KBC_ERR_STATE: the vorticity of the boundary rows and the gamma of the
 * next step's collision read them.  Synchronises the handle's stream. */
int kbc_diagnostics_partial(kbc_handle h, double* out);

/* Combines n >= 1 partial sets parts[n][KBC_DIAG_PART_N] (in that order:
 * sums added, means and sums of squared deviations by Chan, Golub and
 * LeVeque's pairwise formula, minimum and maximum) into the KBC_DIAG_N
 * values of kbc_diagnostics.  Host arithmetic only: no device, no handle;
 * parts and out are host memory.  KBC_ERR_ARG for n < 1, NULL pointers,
 * device pointers or no nodes (message: kbc_last_error(NULL)). */
int kbc_diagnostics_merge(int n, const double* parts, double* out);

/* Further diagnostics of the paper's turbulence figures (FP64 device
 * reductions), out[KBC_DIAG_EXT_N] on the host:
 *   [0] palinstrophy P = mean |grad w|^2 / 2 (w as in kbc_diagnostics, its
 *       gradient by periodic central differences)  [1] spatial std of
 *       |grad w|^2 / 2
 *   [2] mean entropy density s = -sum_i f_i ln(f_i / W_i) (Eq. S)
 *   [3] spatial std of s */
int kbc_diagnostics_ext(kbc_handle h, double* out);

/* Shell-averaged energy and enstrophy spectra of a square periodic velocity
 * field (the spectra of the paper's two-dimensional turbulence figures).
 * With u_hat the discrete Fourier coefficients of u normalised by the node
 * count, E(k) = sum over wavevectors with round(|k|) = k of |u_hat|^2 / 2,
 * so that sum_k E(k) = mean |u|^2 / 2 (Parseval), and Z(k) = (2 pi k / n)^2
 * E(k) (the paper's Z(k) = k^2 E(k)).
 *   n: grid size (nx = ny = n, even, n^2 < 2^31).  u: [2][n][n] doubles,
 *   host or device (e.g. from kbc_moments).  E, Z: nbins doubles each,
 *   host or device; shells k >= nbins are left out (all fit when nbins >=
 *   round(n sqrt(2) / 2) + 1).  stream: CUDA stream (NULL: the legacy
 *   default stream); the call synchronises it before returning.
 * The FFT is cuFFT (a library step); the binning is this library's kernel.
 * Its shell sums use atomic additions, so their last bits depend on the
 * order of the additions.  Device scratch (the velocity staging for host
 * input, the half spectrum, cuFFT's work area) comes from the allocator set
 * with kbc_set_allocator (default cudaMalloc) and is released before the
 * call returns.  Errors: KBC_ERR_ARG, KBC_ERR_NOMEM, KBC_ERR_CUDA (message:
 * kbc_last_error(NULL)). */
int kbc_spectrum(int n, const double* u, int nbins, double* E, double* Z, void* stream);

/* Diagnostics of a caller-owned population field without any device
 * allocation.  The paper has no counterpart to this call.
 *
 * For callers that cannot allocate device memory: code whose device memory
 * is fully owned by another allocator (a framework's caching pool, a fixed
 * arena sized at start-up), and code that must not trigger the implicit
 * device-wide synchronisation of cudaMalloc/cudaFree inside a timed loop.
 * It needs no handle: f is the caller's FP64 population field
 * f[9][ny][nx] in DEVICE memory of the current device (a host pointer
 * gives KBC_ERR_ARG, since staging it would need an allocation, and so does
 * a field on another device); out (host or device) receives the
 * KBC_DIAG_N values documented at kbc_diagnostics, for the given variant
 * and beta with the entropic gamma.  Work runs on `stream` (a cudaStream_t,
 * NULL = legacy default) and the call waits for it (bounded,
 * KBC_ERR_TIMEOUT).
 *
 * Scratch: a file-scope device array of about 1.4 MB that every GPU that
 * loads the library holds until the process exits; it bounds the grid to
 * nx * ny <= 2^28 nodes (e.g. 16384 x 16384); larger grids give
 * KBC_ERR_ARG.  Every failure leaves its message at kbc_last_error(NULL).  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current, and caches it
 * for that device's context (a call after cudaDeviceReset, which ends the
 * context, looks it up again); make that first call before any stream
 * capture.  All calls share the array, so calls that
 * overlap on the GPU (different streams or threads) race and must be
 * serialised by the caller.  Nothing in the array needs clearing: every
 * call overwrites the parts it reads. */
int kbc_diagnostics_noalloc(int nx, int ny, int variant, double beta, const double* f,
                            double* out, void* stream);

/* Discrete adjoint (not in the paper): J and its gradients for
 *   g^0 = f^eq(rho0, u0) (Eq. Eq), g^{n+1} = one step of kbc_step applied to g^n,
 *   objective 0: J = sum_x rho |u|^2 / 2 of g^nsteps (kinetic energy),
 *   objective 1: J = sum_x |u - u_target|^2 / 2 of g^nsteps (misfit).
 * The reverse sweep applies lambda^n = P^T (dC/df)^T lambda^{n+1} with the
 * hand-written derivative of the collision, including the dependence of
 * gamma* (Eq. result21) on f and beta; dJ/dbeta sums lambda^{n+1} . dC/dbeta.
 * Forward states are checkpointed every ckpt_every steps and each segment
 * is recomputed during the reverse sweep (bit-identical to the forward).
 *   rho0 [ny][nx], u0 [2][ny][nx], u_target [2][ny][nx] (objective 1 only,
 *   else NULL): host or device.  J, grad_beta: host doubles.  grad_u0
 *   [2][ny][nx]: host or device.  Adjoint fields are held in the arithmetic
 *   type of the storage (double for F64, float for F32/F16).
 * Device memory for the call, from the handle's allocator and released
 * before returning: ceil(nsteps/ckpt_every) + ckpt_every + 1 population
 * fields, two adjoint fields and O(nx ny) doubles.  Synchronises the
 * stream.  Afterwards the handle holds g^nsteps.  The exact-gamma mode is
 * not differentiated (KBC_ERR_ARG).  With F32/F16 storage the nodes whose
 * entropic denominator is at or below the guard (kbc_set_guard) are
 * reversed in double, as the forward step evaluates them.
 * Conditioning: where <dh|dh> is tiny (smooth, well-resolved fields)
 * gamma* of Eq. result21 is poorly determined and leaves [0, 2/beta]; there
 * the linearised relaxation of dh multiplies perturbations by |1 - beta
 * gamma| > 1, so the discrete adjoint grows step by step (the forward state
 * is unaffected because dh itself is tiny).  Over many steps the gradients
 * become rounding-dominated; single precision overflows first.
 * Errors: KBC_ERR_ARG, KBC_ERR_NOMEM, KBC_ERR_NONFINITE (the forward sweep
 * blew up, or J, grad_beta or grad_u0 is not finite; the outputs are still
 * written). */
int kbc_adjoint(kbc_handle h, const double* rho0, const double* u0, int nsteps, int ckpt_every,
                int objective, const double* u_target, double* J, double* grad_u0,
                double* grad_beta);

/* Bytes of population traffic per lattice-node update of this handle's
 * storage (9 reads + 9 writes), for roofline accounting. */
int kbc_bytes_per_update(kbc_handle h, double* bytes);

/* Measured issue rate of double-precision fused multiply-adds on the
 * current device, the ceiling of the FP64-storage path, whose step is bound
 * by the FP64 pipe rather than by memory (a measurement helper for roofline
 * accounting; the paper has no counterpart).  Launches a kernel of
 * independent DFMA chains filling every SM on `stream` (a cudaStream_t,
 * NULL = legacy default) four times, times each with CUDA events and writes
 * the best rate, in thread DFMA operations per second, to *dfma_per_s.
 * Synchronises the stream.  Errors: KBC_ERR_ARG (NULL output),
 * KBC_ERR_CUDA. */
int kbc_fp64_fma_rate(void* stream, double* dfma_per_s);

/* Message describing the last error on h (or of the last kbc_create when h
 * is NULL).  Valid until the next call on h. */
const char* kbc_last_error(kbc_handle h);

#ifdef __cplusplus
}
#endif

#endif /* KBC_GB300_H */
