/*
 * pfgrid.h - C ABI of libpfgrid.so: FP64 bus power injections and power-flow
 * Jacobians on one GPU (sm_103a), by the two methods compared in
 * "Bus Admittance Matrix Revisited: Is It Outdated on Modern Computers?"
 * (H. Cui, arXiv 2302.10736):
 *   - the Ybus method (Sec. II-A, Sec. IV-B): S = V . conj(Ybus V) (Eq. 1) and
 *     the Jacobian blocks of Eqs. (2)-(4) by a row-local two-pass sweep;
 *   - the element-wise method (Sec. II-B, Sec. IV-C): per-branch terminal
 *     flows (Eqs. 5-6) and their 16 partials, reduced onto buses (Eq. 7) and
 *     onto Jacobian slots.
 *
 * Conventions
 *   Branch l joins h = from[l] and k = to[l] (0-based).  Series admittance
 *   y_hk = g + j b (per unit); b_sh is the total line charging, split as
 *   y_h = y_k = j b_sh / 2; tap m e^{j phi} sits on the h side (Eqs. 5-6);
 *   lines have m = 1, phi = 0.  Bus shunt y_sh,i = g_s,i + j b_s,i.
 *   Voltages are polar: vm = |V| (the "V_m" of Eq. 4), va = theta (rad).
 *   All values are IEEE FP64; indices int32.
 *
 * Numerics
 *   Inputs, outputs and every sum are FP64.  Inside the kernels the sine and
 *   cosine of the angles and the complex products (V_o conj(U_q), conj(Yc) E,
 *   Y_ij U_j, V_i conj(Y_ij U_j)) are computed in 64-bit fixed point on the
 *   integer pipes and rounded once to FP64: within 2^-52 of the product's
 *   magnitude after that rounding, at least as accurate as FP64 products.
 *   Non-finite values and magnitudes outside about 2^-960 .. 2^957 take FP64
 *   products (IEEE semantics, NaN propagated).  The element-wise Jacobian's
 *   diagonal uses 1/vm, so vm must be a normal, nonzero number there.
 *
 *   Ybus pattern: every diagonal (i, i) plus (h, k) and (k, h) of every
 *   branch; parallel branches share one entry; columns sorted; explicit zeros
 *   kept (Sec. IV-B.2).
 *
 *   Canonical Jacobian J (2nb x 2nb, CSR, Eq. 2 block order), nnzJ = 4 nnzY:
 *     P-row i    (i < nb): columns = Ybus row-i columns j (theta_j), then nb + j (v_j)
 *     Q-row nb+i         : same columns
 *     rowptr[i] = 2 Yrowptr[i],  rowptr[nb + i] = 2 nnzY + 2 Yrowptr[i].
 *   With d_i the Ybus row length and k the position of column j in Ybus row i:
 *     J11 = dP_i/dtheta_j at 2 Yrowptr[i] + k
 *     J12 = dP_i/dv_j     at 2 Yrowptr[i] + d_i + k
 *     J21 = dQ_i/dtheta_j at 2 nnzY + 2 Yrowptr[i] + k
 *     J22 = dQ_i/dv_j     at 2 nnzY + 2 Yrowptr[i] + d_i + k
 *   (Alg. 2's index arrays P_xy in closed form.)
 *
 * Execution model
 *   Every evaluation entry point is asynchronous on `stream` (a cudaStream_t,
 *   NULL = the legacy default stream), allocates nothing, never synchronizes
 *   and takes device pointers the caller owns (eval_host, eval_host_async,
 *   powerflow_newton and the set-up calls are the documented exceptions).  The element-wise
 *   single evaluations (jac_elementwise, inj_elementwise, and jac_reduced /
 *   jac_target with method 1) keep their phasors in shared memory and only
 *   read the grid, so they may overlap on several streams; the Ybus-method
 *   evaluations share the grid's phasor workspace and batched and Newton
 *   calls the batch's or grid's scratch, so those must not overlap on the GPU
 *   with another call on the same grid (issue them on one stream).
 *   Input checks are done at build time; evaluation calls check only for
 *   NULL pointers and sizes.
 *   Errors: every function returns a pf_status; pf_last_error() gives a
 *   message for the calling thread.  Nothing aborts or throws across the ABI.
 */
#ifndef PFGRID_H
#define PFGRID_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t pf_status;
#define PF_OK 0
#define PF_EINVAL 1          /* bad argument (NULL pointer, size, non-finite or non-positive tap) */
#define PF_ENOMEM 2          /* device or host allocation failed */
#define PF_ECUDA 3           /* a CUDA runtime call or launch failed */
#define PF_ETOPO 4           /* bad topology: bus index out of range or self loop */
#define PF_EDEVICE 5         /* a kernel reported an error through the grid's device error word */
#define PF_ETIMEOUT 6        /* a bounded device-side wait gave up */
#define PF_EUNSUPPORTED 7    /* size beyond the int32 index range of this library */
#define PF_ENOCONV 8         /* Newton iteration did not converge, or its Jacobian was singular */

typedef void *pf_stream;            /* cudaStream_t */
typedef struct pf_grid pf_grid;     /* opaque; owns all device structure of one network */

/* Host-side network description (structure of arrays).  nb >= 0, nl >= 0.
   gs / bs may be NULL (no bus shunts). */
typedef struct {
    int32_t nb, nl;
    const int32_t *from, *to;       /* [nl] bus indices, from != to */
    const double *g, *b;            /* [nl] series conductance / susceptance (p.u.) */
    const double *bsh;              /* [nl] total line charging susceptance */
    const double *tap;              /* [nl] off-nominal ratio m > 0 (1 for lines) */
    const double *shift;            /* [nl] phase shift phi (rad) */
    const double *gs, *bs;          /* [nb] bus shunt conductance / susceptance, or NULL */
} pf_grid_desc;

/* Launch configuration (chosen by grid_autotune or set by hand). */
typedef struct {
    int32_t ybus_lanes;     /* lanes per Ybus row in the CSR kernels: 1, 2, 4, 8, 16 or 32 */
    int32_t ybus_block;     /* threads per CTA of the CSR kernels (multiple of 32, <= 512) */
    int32_t ew_window;      /* threads per CTA of the element-wise kernels: 128 or 256; a CTA owns a
                               window of consecutive buses with at most that many buses and terminals */
    int32_t ybus_fused;     /* Ybus method: 1 = the phasor step fused into the row kernel (one launch; each
                               entry forms its column's phasor), 0 = the phasor step as its own launch */
} pf_config;

/* Human-readable name of a status code (static string). */
const char *pf_status_str(pf_status s);

/* Message describing the last error on the calling thread ("" if none). */
const char *pf_last_error(void);

/*
 * Build a grid: validates the description (PF_EINVAL / PF_ETOPO), builds the
 * Ybus pattern, the canonical J pattern, the terminal layouts of both methods
 * and the per-terminal constants of Eqs. (5)-(6) (computed once ahead of time,
 * Sec. IV-C.1), uploads everything and computes the Ybus values on `stream`.
 * Synchronizes `stream` before returning (setup, not the hot path).
 * The description's arrays are read during the call only.
 */
pf_status ybus_build(const pf_grid_desc *desc, pf_stream stream, pf_grid **out);

/* Free every device and host resource of a grid (NULL is allowed). */
void grid_destroy(pf_grid *grid);

/* Sizes of a grid. Any output pointer may be NULL. */
pf_status grid_info(const pf_grid *grid, int32_t *nb, int32_t *nl, int32_t *nnzY);

/*
 * Replace the branch and bus-shunt parameters from DEVICE arrays (same
 * meaning as in pf_grid_desc: g, b, bsh, tap, shift [nl]; gs, bs [nb] or
 * NULL for zero) without changing the topology; recomputes the terminal
 * constants and the Ybus values on `stream`.  Taps are not re-validated.
 */
pf_status grid_set_params(pf_grid *grid, const double *g, const double *b, const double *bsh,
                          const double *tap, const double *shift, const double *gs, const double *bs,
                          pf_stream stream);

/*
 * Device pointers to the grid's Ybus (owned by the grid, valid until
 * grid_destroy): rowptr [nb+1], colidx [nnz], values [nnz] as interleaved
 * (re, im) pairs.
 */
pf_status ybus_get(const pf_grid *grid, int32_t *nnz, const int32_t **rowptr, const int32_t **colidx,
                   const double **values);

/*
 * The element-wise method's windows of consecutive buses (Sec. IV-C on the
 * GPU: one CTA per window, its terminals and ghost buses with it), for
 * inspection: window w is out[5w .. 5w+4] = {first bus, buses, first sorted
 * terminal, terminals, phasor slots (own and ghost buses)}.  Fills at most
 * max_windows windows (out may be NULL to query *nwin only; caller-owned
 * host memory).  Synchronous (a device-to-host copy).  Errors: PF_EINVAL for a
 * NULL grid, PF_ECUDA.
 */
pf_status grid_ew_windows(const pf_grid *grid, int32_t *out, int32_t max_windows, int32_t *nwin);

/* Device pointers to the canonical J pattern (owned by the grid):
   rowptr [2nb+1], colidx [nnzJ]. */
pf_status jac_pattern(const pf_grid *grid, int32_t *nnzJ, const int32_t **rowptr, const int32_t **colidx);

/*
 * Bus injections by the Ybus method (Eq. 1; Sec. IV-B.1 steps 1-3):
 * phasors U = e^{j theta}, V = vm U; I = Ybus V by a CSR SpMV with
 * config.ybus_lanes lanes per row; S = V . conj(I).
 * vm, va [nb] in; P, Q [nb] out (device, caller-owned).
 */
pf_status inj_ybus(pf_grid *grid, const double *vm, const double *va, double *P, double *Q, pf_stream stream);

/*
 * Bus injections by the element-wise method (Eqs. 5-7): every branch
 * terminal's flow from its precomputed constants and the gathered bus
 * phasors, then a deterministic segmented sum onto its bus plus the bus
 * shunt.  Same arguments as inj_ybus.
 */
pf_status inj_elementwise(pf_grid *grid, const double *vm, const double *va, double *P, double *Q,
                          pf_stream stream);

/*
 * Jacobian values by the Ybus method (Eqs. 2-4): per Ybus row, one sweep
 * forms Y_ij U_j, the off-diagonal entries and the row current I_i; the
 * diagonal entry is completed once I_i is known (the two passes of Alg. 1,
 * kept row-local).  Values land directly in the canonical layout (Alg. 2).
 * vm, va [nb] in; J [4 nnzY] out; P, Q [nb] out or NULL.
 */
pf_status jac_ybus(pf_grid *grid, const double *vm, const double *va, double *P, double *Q, double *J,
                   pf_stream stream);

/*
 * Jacobian values by the element-wise method: each terminal evaluates its
 * flow and 8 partials (16 per branch, Sec. II-B), which are reduced without
 * atomics onto the diagonal slot of its bus and the off-diagonal slot of its
 * (bus, other bus) pair.  Same arguments as jac_ybus.
 *
 * Throughput of many independent evaluations: one call keeps the CTAs of an
 * SM in the same phase of their windows (the integer pipes busy in the
 * sine/cosine and coupling products, then the FP64 pipe in the bus sums);
 * calls issued on two CUDA streams, each with its own outputs, share the SMs
 * in different phases (on a GB300, 70,000-bus grid: 6.7 against 8.5 us per
 * evaluation).  Element-wise calls only read the grid, so one grid may serve
 * both streams; Ybus-method calls use the grid's phasor workspace and need a
 * grid per stream.
 */
pf_status jac_elementwise(pf_grid *grid, const double *vm, const double *va, double *P, double *Q, double *J,
                          pf_stream stream);

/*
 * End-to-end evaluation from HOST buffers: copies vm, va [nb] to grid-owned
 * device buffers, runs jac_ybus (method 0) or jac_elementwise (method 1),
 * brings P, Q [nb] and J [4 nnzY] back, and synchronizes `stream`.  The
 * device staging buffers are allocated on the first call and kept by the
 * grid.  Host buffers may be pageable or page-locked; when P, Q and J are
 * page-locked and mapped (cudaHostAlloc, cudaHostRegister) the element-wise
 * kernel stores its results straight into them (and reads vm, va straight
 * from them when those are page-locked too): two CTAs per SM loop over the
 * windows, so the first windows' results cross the host link while later
 * windows are evaluated.  The host link bounds this call: 9 MB of results per
 * 70k-bus evaluation take about 50 us at the measured 180 GB/s.
 */
pf_status eval_host(pf_grid *grid, int32_t method, const double *vm, const double *va, double *P, double *Q,
                    double *J, pf_stream stream);

/*
 * eval_host without the final synchronization, for streams of evaluations:
 * the call returns once the work is enqueued on `stream`, and P, Q, J hold
 * the results once `stream` has been synchronized (or an event recorded
 * after the call has completed).  All five host buffers must be page-locked
 * (cudaHostAlloc, cudaHostRegister; PF_EINVAL otherwise, nothing enqueued),
 * and must not be touched by the host until then.  Method 1 runs the
 * element-wise kernel straight on the mapped buffers as eval_host does;
 * method 0 copies in, evaluates and copies out through the grid's staging
 * buffers, so calls on one grid that use method 0 must be issued on one
 * stream, while method-1 calls only read the grid and may overlap on several
 * streams (with distinct output buffers).  Successive calls overlap one
 * evaluation's host-side call and launch with the previous one's device
 * work: on the 70k-bus grid about 64 us per evaluation on one stream, 56 us
 * alternating two streams (the 9 MB of results take 50 us on the host link),
 * against 79 us for eval_host, whose return waits for the results.
 */
pf_status eval_host_async(pf_grid *grid, int32_t method, const double *vm, const double *va, double *P, double *Q,
                          double *J, pf_stream stream);

/*
 * The phasor step alone (Sec. IV-B.1 step 1), as run at the start of every
 * evaluation: for i < n, U[4i..4i+3] = {cos va_i, sin va_i, vm_i, 1/vm_i} and
 * V[2i..2i+1] = vm_i (cos va_i, sin va_i).  Device pointers; U 32-byte and V
 * 16-byte aligned (PF_EINVAL otherwise).  sin/cos in fixed-point integer
 * arithmetic (exact reduction to turns, a 64-entry table, Taylor polynomials;
 * absolute error within 2 ulp of 1; the library sincos for |va| >= 2^16),
 * 1/vm by two Newton steps from the hardware approximation (vm must be a
 * normal, nonzero number).  The first use of the library on a device uploads
 * a 64 KB constant table and synchronizes (ybus_build does it); make it before
 * any stream capture.
 */
pf_status phasor(int32_t n, const double *vm, const double *va, double *U, double *V, pf_stream stream);

/*
 * Bus injections by the Ybus method without any device allocation, for
 * callers that cannot call cudaMalloc: host frameworks that hand out all
 * device memory from their own pool and forbid driver allocations, or
 * latency-critical loops where an allocation is not acceptable.  The paper
 * has no counterpart; this is a deployment variant of inj_ybus.
 *   nb        buses, 0 <= nb <= 262144 (PF_EUNSUPPORTED above: the phasor
 *             scratch is a fixed 4 MiB device array in the library)
 *   rowptr [nb+1], colidx [nnz], yval [nnz][2] (re, im; 16-byte aligned):
 *             a Ybus in CSR form owned by the caller (for example the arrays
 *             returned by ybus_get), read during the call; nnz = rowptr[nb],
 *             rowptr nondecreasing from 0, every colidx entry in [0, nb).
 *             The call does not read rowptr on the host, so it cannot check
 *             these: arrays shorter than nnz, or a column outside [0, nb),
 *             make the kernels read outside the caller's buffers.
 *   vm, va [nb] in; P, Q [nb] out (device pointers on the current device,
 *             caller-owned)
 * The scratch array is shared by all calls on a device and keeps the last
 * call's contents (each call writes the entries it reads first, so nothing
 * needs clearing); calls that overlap on the GPU race on it, so issue them on
 * one stream.  The first call on a device looks up the array's device
 * address (with that device current) and keeps it for the process: make that
 * first call before any stream capture, and do not use this entry point after
 * cudaDeviceReset, which invalidates the kept address.
 */
pf_status inj_ybus_noalloc(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *yval,
                           const double *vm, const double *va, double *P, double *Q, pf_stream stream);

/*
 * Diagnostics: per-phase timing of the single-evaluation element-wise kernel
 * (the paper's per-step breakdown, Table VII, measured inside the fused
 * kernel).  Only a library built with -DPF_PHASE_PROBE records anything (its
 * kernels then write timestamps; the default build writes none and this call
 * returns PF_EUNSUPPORTED).  Copies the records of the last launch of
 * jac_elementwise / inj_elementwise, for windows 0 .. min(max_windows, 8192)-1,
 * into out (host, 9 words per window): [0] %globaltimer (ns) when the window's
 * CTA started, [1] when it ended, [2] its SM, [3..7] clock64 cycles from the
 * start to the end of the load, phasor, evaluation, reduction and store
 * phases, [8] %globaltimer when its wait for the previous kernel in the
 * stream (programmatic dependent launch) returned.  *nwin receives the number
 * of windows copied.  Synchronous.
 */
pf_status pf_phase_probe_read(uint64_t *out, int32_t max_windows, int32_t *nwin);

/*
 * Measurement: the device's FP64 fused multiply-add throughput, the
 * denominator of the FP64 roofline (the method's kernels are bound by the
 * FP64 pipe on GB300).  Launches `ctas` CTAs of 256 threads, each running 8
 * independent FMA chains for iters x 16 steps, on `stream`; the caller times
 * the launch (CUDA events) and divides *dfma_per_launch (may be NULL) by the
 * time.  sink: any device double (never written in practice).  No allocation.
 */
pf_status fp64_peak_probe(int32_t ctas, int32_t iters, double *sink, int64_t *dfma_per_launch, pf_stream stream);

/* Current launch configuration. */
pf_status grid_get_config(const pf_grid *grid, pf_config *cfg);

/*
 * Set the launch configuration.  Changing ew_window rebuilds the
 * element-wise terminal layout (host work + upload, synchronizes `stream`).
 */
pf_status grid_set_config(pf_grid *grid, const pf_config *cfg, pf_stream stream);

/*
 * Autotuner: times every candidate configuration of each kernel (CUDA
 * events, `reps` launches each, on `stream`) with the given device state
 * vm, va [nb], keeps the fastest, and writes the chosen configuration to
 * *best (may be NULL).  Allocates temporary device outputs; synchronizes.
 */
pf_status grid_autotune(pf_grid *grid, const double *vm, const double *va, int32_t reps, pf_stream stream,
                        pf_config *best);

/*
 * Synchronize `stream` and report device-side errors recorded by the grid's
 * kernels (PF_EDEVICE, PF_ETIMEOUT); clears the error word.
 */
pf_status grid_check_error(pf_grid *grid, pf_stream stream);

/*
 * Host-only self-check (no GPU needed, nothing allocated on the device):
 * validates `desc` like ybus_build, builds the index structures of the grid
 * and the element-wise windows for CTAs of `window` threads - cut at equal
 * estimated cost into at most `nwin_target` windows when nwin_target is
 * larger than the plain cut's count (ybus_build targets a whole number of
 * waves of resident CTAs), the plain cut when it is 0 - and verifies every
 * invariant the kernels' memory accesses rely on (index ranges, sorted
 * terminal order, parallel-run flags, ghost-bus slots, window descriptors,
 * staging offsets inside each window's Jacobian slice, bulk-copy alignment,
 * shared-memory size, the per-window branch lists of the small-batch adjoint:
 * every branch in exactly one window).  PF_OK or PF_EINVAL with a message.
 */
pf_status grid_selfcheck(const pf_grid_desc *desc, int32_t window, int32_t nwin_target);

/* ------------------------------------------------------------ batches -- */

typedef struct pf_batch pf_batch;   /* opaque; S scenarios over one grid */

/* Launch configuration of a batch's kernels (batch_set_config, batch_autotune). */
typedef struct {
    int32_t window;                /* threads per CTA of the batched element-wise kernels, 128 or 256: a
                                      window holds at most this many consecutive buses */
    int32_t terminals_per_thread;  /* 1, 2 or 3: a window holds at most window x this many terminals */
    int32_t ctas_per_sm;           /* CTAs per SM of the persistent batched launches: 0 = as many as fit,
                                      else at most this many (1 .. 8) */
    int32_t adjoint_form;          /* 0: one (scenario, window) item per CTA when they all fit at once,
                                      else the persistent form; 1: the persistent form always */
    int32_t ybus_lanes;            /* lanes per row of the batched Ybus kernels: 1, 2, 4, 8, 16 or 32 */
    int32_t ybus_block;            /* threads per CTA of the batched Ybus kernels (multiple of 32, <= 512) */
} pf_batch_config;

/*
 * A batch of `nscen` scenarios over `grid` (the grid must outlive the batch).
 * Scenario s has its own voltage state and, when outage != NULL and
 * outage[s] >= 0, loses branch outage[s] (an N-1 contingency: the
 * element-wise method of Sec. II-B applied to the grid without that branch).
 * Scenario s's Jacobian lives on its own pattern: the base pattern without
 * the (h, k), (k, h) entries of the removed branch, unless a parallel branch
 * keeps them; its values start at offset joff[s] of the batch's J array
 * (batch_jac_offsets), nnzJ_s = 4 (nnzY - 2 removed).  outage is a host array
 * read during the call; values outside [-1, nl) give PF_EINVAL.  Allocates
 * the batch workspaces (phasors and residuals, 64 bytes per scenario-bus) and
 * synchronizes `stream`.  If the environment variable PFGRID_TUNE_CACHE names
 * a tuning cache file (written by batch_autotune) that holds a configuration
 * for this GPU and the batch's size class, the batch starts with it.
 */
pf_status batch_create(pf_grid *grid, int32_t nscen, const int32_t *outage, pf_stream stream, pf_batch **out);

/* Free a batch (NULL is allowed). */
void batch_destroy(pf_batch *batch);

/* Number of scenarios and total Jacobian values of the batch (either may be NULL). */
pf_status batch_info(const pf_batch *batch, int32_t *nscen, int64_t *nnzJ_total);

/* The batch's current launch configuration. */
pf_status batch_get_config(const pf_batch *batch, pf_batch_config *cfg);

/*
 * Set the batch's launch configuration (PF_EINVAL for values outside the
 * ranges of pf_batch_config; PF_EUNSUPPORTED when a window would exceed
 * shared memory).  A new window size or terminal cap rebuilds the batch's
 * windows (host work and upload; synchronizes `stream`).  Results do not
 * depend on the configuration except for the rounding of loss sums: every
 * bus and Jacobian entry is summed in the same order whatever the windows.
 */
pf_status batch_set_config(pf_batch *batch, const pf_batch_config *cfg, pf_stream stream);

/*
 * Autotuner of the batched launches (no counterpart in the paper): times
 * `reps` launches (CUDA events on `stream`) of the kernels selected in
 * `kernels` (PF_TUNE_* bits; 0 means PF_TUNE_JAC | PF_TUNE_YBUS) with the
 * states vm, va [nscen * nb].  The element-wise shape (window size x terminal
 * cap x CTAs per SM, and the adjoint's form when it is selected) minimizes the
 * summed time of jac_elementwise_batched and/or adjoint_elementwise (timed with
 * targets 0 and weights 1); the batched Ybus shape (lanes x CTA size) that of
 * jac_ybus_batched.  Keeps the fastest, writes it to *best (may be NULL) and,
 * when PFGRID_TUNE_CACHE names a file, stores it there under batch_tune_key.
 * Allocates temporary outputs (the batch's full Jacobian, the adjoint's
 * arrays) and synchronizes.
 */
#define PF_TUNE_JAC 1        /* jac_elementwise_batched */
#define PF_TUNE_YBUS 2       /* jac_ybus_batched */
#define PF_TUNE_ADJOINT 4    /* adjoint_elementwise */
pf_status batch_autotune(pf_batch *batch, const double *vm, const double *va, int32_t kernels, int32_t reps,
                         pf_stream stream, pf_batch_config *best);

/*
 * The tuning-cache key of a batch: the GPU's name, the kernel family and the
 * size class (buses and scenarios rounded up to powers of two, with or
 * without outages), as a NUL-terminated string in buf[0 .. len).
 */
pf_status batch_tune_key(const pf_batch *batch, char *buf, int32_t len);

/*
 * The tuning cache itself, a JSON file mapping keys to pf_batch_config
 * fields: look a key up (*found = 1 and *cfg filled when present; a missing
 * file is an empty cache), or store a configuration under a key (the file is
 * rewritten through a temporary and a rename; other keys are kept).  Host
 * only; keys may not contain '"' or '\\'.
 */
pf_status pf_tune_cache_lookup(const char *path, const char *key, pf_batch_config *cfg, int32_t *found);
pf_status pf_tune_cache_store(const char *path, const char *key, const pf_batch_config *cfg);

/* Device pointer (owned by the batch) to the offsets joff [nscen + 1] of each
   scenario's Jacobian values in the batch's J array. */
pf_status batch_jac_offsets(const pf_batch *batch, const int64_t **offsets);

/*
 * Host copy of scenario s's Jacobian pattern in the canonical layout of this
 * header: rowptr [2nb + 1] and colidx [nnzJ_s] (either may be NULL; *nnzJ_s
 * receives the count, so a first call with NULL arrays gives the size).
 */
pf_status batch_jac_pattern(const pf_batch *batch, int32_t s, int32_t *rowptr, int32_t *colidx, int32_t *nnzJ_s);

/*
 * Element-wise injections of every scenario in one persistent cooperative
 * launch (capturable in a CUDA graph): vm, va [nscen][nb] in; P, Q
 * [nscen][nb] out (device, caller-owned).  The batch owns the phasor
 * workspace, so launches on one batch or grid must not overlap on the GPU.
 */
pf_status inj_elementwise_batched(pf_batch *batch, const double *vm, const double *va, double *P, double *Q,
                                  pf_stream stream);

/*
 * Element-wise injections and Jacobian values of every scenario in one
 * persistent cooperative launch: as inj_elementwise_batched plus J
 * [nnzJ_total] (scenario s at joff[s], on its own pattern); P, Q may be NULL.
 */
pf_status jac_elementwise_batched(pf_batch *batch, const double *vm, const double *va, double *P, double *Q,
                                  double *J, pf_stream stream);

/*
 * Ybus-method injections of every scenario (Eq. 1 per scenario): the phasor
 * step over all nscen * nb buses, then W = config.ybus_lanes lanes per
 * (scenario, row) of the shared base CSR Ybus, with the outage branch's
 * terminal constants taken out of its two end rows on the fly (the coupling
 * entry dropped when it leaves the pattern).  Two launches, capturable in a
 * CUDA graph.  Same arguments as inj_elementwise_batched; PF_EUNSUPPORTED if
 * nscen * nb exceeds 2^31 - 1.
 */
pf_status inj_ybus_batched(pf_batch *batch, const double *vm, const double *va, double *P, double *Q,
                           pf_stream stream);

/*
 * Ybus-method Jacobian values of every scenario (Eqs. 2-4 per scenario, as
 * jac_ybus on the scenario's admittance matrix), written compacted onto the
 * scenario's own pattern like jac_elementwise_batched.  Same arguments and
 * layout as jac_elementwise_batched.
 */
pf_status jac_ybus_batched(pf_batch *batch, const double *vm, const double *va, double *P, double *Q, double *J,
                           pf_stream stream);

/*
 * Adjoint of the mismatch loss, one cooperative launch (the paper has no
 * adjoint; it differentiates the element-wise flows of Eqs. 5-7):
 *   L_s = sum_i wP_i (P_si - Pspec_i)^2 + wQ_i (Q_si - Qspec_i)^2
 * for every scenario s of the batch (outages honoured), and the total
 * L_total = sum_s L_s (ascending s).  With lbar = *Lbar (device scalar; NULL
 * means 1), the upstream gradient of L_total (an autograd caller passes
 * dOut/dL_total here, so no caller-side scaling is needed):
 *   L [nscen]            the loss per scenario (may be NULL)
 *   Ltot [1]             L_total (may be NULL)
 *   gvm, gva [nscen][nb] lbar dL_s/d|V| and lbar dL_s/dtheta (J^T r without forming J)
 *   gg, gb, gbsh, gtap [nl]  lbar d(L_total)/d(g, b, b_sh, tap) per branch,
 *                        scenarios summed in ascending order (all four NULL
 *                        to skip; a branch removed in scenario s gets no
 *                        contribution from s; tap derivative at the branch's
 *                        own ratio, 1 for lines; phase shift not differentiated)
 * Pspec, Qspec, wP, wQ [nb] are shared by all scenarios.  Device pointers.
 * The loss and gradients use the grid's current parameters (grid_set_params).
 * L and Ltot are bitwise those of loss_elementwise on the same inputs.
 */
pf_status adjoint_elementwise(pf_batch *batch, const double *vm, const double *va, const double *Pspec,
                              const double *Qspec, const double *wP, const double *wQ, const double *Lbar, double *L,
                              double *Ltot, double *gvm, double *gva, double *gg, double *gb, double *gbsh,
                              double *gtap, pf_stream stream);

/*
 * The mismatch loss alone (the forward pass of the adjoint above): the
 * injections of every scenario (Eqs. 5-7), L_s and L_total, in one
 * cooperative launch that forms no residual or gradient.  L [nscen] and Ltot
 * [1] are device outputs; either may be NULL, not both.  Other arguments as in
 * adjoint_elementwise.
 */
pf_status loss_elementwise(pf_batch *batch, const double *vm, const double *va, const double *Pspec,
                           const double *Qspec, const double *wP, const double *wQ, double *L, double *Ltot,
                           pf_stream stream);

/*
 * Fault injection for tests of the bounded device-side waits (no GPU fault
 * is involved): moves the arrival counter of the grid barrier that the
 * batched element-wise and adjoint kernels of this grid's batches share out
 * of range, so in the next such launch no CTA ever sees the last arrival;
 * each CTA gives up after 2 s, skips its work and sets the device error word,
 * and grid_check_error then returns PF_ETIMEOUT and resets the barrier.
 * (The single-scenario kernels have no grid-wide wait.)  Synchronizes
 * `stream`.
 */
pf_status grid_inject_barrier_fault(pf_grid *grid, pf_stream stream);

/* --------------------------------------------- reduced Newton Jacobian -- */

/*
 * Bus types for the Newton step (codes as in MATPOWER): 1 PQ, 2 PV,
 * 3 reference (slack), 4 isolated.  The reduced system keeps, of Eq. 2's
 * blocks, the P rows and theta columns of the PV and PQ buses and the Q rows
 * and v columns of the PQ buses.  Ordering: theta / P part first
 * (n_pvpq entries), then v / Q (n_pq entries), each in ascending bus order;
 * n = n_pvpq + n_pq.  The reduced Jacobian is stored column-major (CSC:
 * colptr [n + 1], rowidx [nnz], rows ascending within a column, structural
 * zeros kept), the layout sparse direct solvers such as KLU take.
 * `bus_type` is a host array [nb]; the pattern and its gather map are built
 * on the host and uploaded (synchronizes `stream`).  PF_EINVAL for another
 * code.  May be called again to change the types.
 */
pf_status grid_set_bus_types(pf_grid *grid, const int32_t *bus_type, pf_stream stream);

/* Sizes of the reduced system (PF_EINVAL before grid_set_bus_types). */
pf_status jac_reduced_info(const pf_grid *grid, int32_t *n, int32_t *n_pvpq, int64_t *nnz);

/* Device pointers to the reduced CSC pattern, owned by the grid. */
pf_status jac_reduced_pattern(const pf_grid *grid, const int32_t **colptr, const int32_t **rowidx);

/*
 * One Newton evaluation: the mismatch vector
 *   F = [P - Pspec on the PV and PQ buses ; Q - Qspec on the PQ buses]  [n]
 * and the reduced Jacobian values Jr [nnz] in the CSC order above.  Method 1
 * (element-wise): one launch whose windows write F and Jr directly (no full
 * Jacobian is stored); the values are bit for bit those of jac_elementwise
 * selected.  Method 0 (Ybus): the full evaluation into grid-owned scratch,
 * then one gather launch.
 * vm, va, Pspec, Qspec [nb], F, Jr: device pointers owned by the caller.
 * Asynchronous; method 0 uses the grid's scratch, so those calls on one grid
 * must not overlap (method 1 only reads the grid).
 * (The paper computes the full Jacobian; the reduction is the step its
 * solver interface implies.)
 */
pf_status jac_reduced(pf_grid *grid, int32_t method, const double *vm, const double *va, const double *Pspec,
                      const double *Qspec, double *F, double *Jr, pf_stream stream);

/* ------------------------------------------- caller's Jacobian pattern -- */

/*
 * Alg. 2 (Sec. IV-B.3), the general index arrays P_xy: a caller's Jacobian
 * pattern in CSC form, 2nb x 2nb with rows and columns in the block order of
 * Eq. (2) (theta / P first, then v / Q), that contains every entry of the
 * Ybus-block pattern (jac_pattern) and may hold more (series devices such as
 * TCSC couple further buses).  colptr [2nb+1], rowidx [nnz]: host int32 arrays,
 * read during the call; rows within a column in any order (the first match
 * counts).  The library finds, by matching row and column, the position in
 * this pattern of every canonical entry and keeps that map on the device
 * (synchronizes `stream`).  PF_EINVAL if an entry of the Ybus-block pattern
 * is missing or the arrays are malformed, PF_EUNSUPPORTED if nnz >= 2^31.
 */
pf_status jac_set_target_pattern(pf_grid *grid, const int32_t *colptr, const int32_t *rowidx, int64_t nnz,
                                 pf_stream stream);

/*
 * One evaluation into that pattern: Jt[P_xy] = the Jacobian values (Jt
 * [nnz], device, caller-owned; its other entries are left as they are: they
 * belong to devices outside this library), and P, Q [nb] when both are
 * non-NULL.  Method 1 (element-wise): one launch that stores through the map;
 * method 0 (Ybus): the evaluation into grid-owned scratch, then one scatter
 * launch.  The values are bit for bit those of jac_elementwise / jac_ybus.
 * Asynchronous; PF_EINVAL before jac_set_target_pattern.
 */
pf_status jac_target(pf_grid *grid, int32_t method, const double *vm, const double *va, double *P, double *Q,
                     double *Jt, pf_stream stream);

/*
 * Solve J_r dx = F for the reduced Newton system of the grid's bus types
 * (the step the paper hands to a sparse direct solver, KLU): Jr [nnz] holds
 * the reduced Jacobian's values in jac_reduced's CSC order, F [n] the right-hand
 * side, dx [n] receives the solution (device pointers).  Sparse LU without
 * pivoting on a fill-reducing order: the first call after grid_set_bus_types
 * analyses the pattern on the host (minimum-degree order of the buses,
 * symbolic factorization, the dependency schedule of the elimination tree),
 * allocates the factor storage and synchronizes; make it before any stream
 * capture.  Every later call is asynchronous: a cooperative launch for the
 * numeric factorization with the forward solve, each column started when the
 * columns it depends on are done (bounded waits); where the top of the
 * elimination tree is a run of at least 16 narrow levels, a launch of one
 * 8-CTA thread-block cluster for it (a dense block in shared memory, both
 * triangular solves), then a cooperative launch for the backward solve below
 * it (otherwise the backward solve ends the first launch).  Bitwise
 * repeatable.  A zero
 * or non-finite pivot sets the grid's device error word (grid_check_error
 * reports PF_EDEVICE), a wait that runs out (2 s) sets it to a time-out
 * (grid_check_error reports PF_ETIMEOUT and clears it); no pivoting
 * means the matrix must admit LU in that order, which the power-flow Jacobians
 * of this library's grids do (their 2 x 2 bus blocks dominate).
 */
pf_status jac_reduced_solve(pf_grid *grid, const double *Jr, const double *F, double *dx, pf_stream stream);

/*
 * Newton-Raphson power flow on the GPU (not in the paper, which stops at the
 * Jacobian a Newton step needs): starting from vm, va [nb] (device, updated
 * in place), repeat
 *   full evaluation by `method` (0 Ybus, 1 element-wise) -> F and J_r
 *   (the reduced system of jac_reduced, J_r in CSC order) -> stop when
 *   max |F| <= tol -> solve J_r dx = F (jac_reduced_solve's sparse LU)
 *   -> theta_pvpq -= dx[0 .. n_pvpq), v_pq -= dx[n_pvpq .. n)
 * at most max_iter steps.  Requires grid_set_bus_types; PV and reference
 * magnitudes and reference angles stay as given.  *iterations and *mismatch
 * (host, may be NULL) receive the steps taken and the final max |F|.
 * PF_ENOCONV if max |F| > tol after max_iter steps or J_r is singular (vm,
 * va then hold the last iterate).  Synchronizes `stream` once per
 * iteration (the convergence test).  Allocates its workspace on the first
 * call after grid_set_bus_types.
 */
pf_status powerflow_newton(pf_grid *grid, int32_t method, double *vm, double *va, const double *Pspec,
                           const double *Qspec, double tol, int32_t max_iter, int32_t *iterations, double *mismatch,
                           pf_stream stream);

/*
 * Study entry point (the paper's two-step structure, Sec. IV-C, for
 * comparison with jac_elementwise): the phasor step, then K_t and G_t of every
 * terminal into a grid-owned intermediate, then the assembly by `strategy`:
 * 0 gather (one thread per bus, its terminals in order; deterministic) or
 * 1 copy-add (bus constants, then one thread per terminal adding with
 * floating-point atomics; the addition order, hence the last bits, vary from
 * run to run).  Same arguments and results (within rounding) as
 * jac_elementwise, P and Q required.  Uses the grid's phasor workspace and
 * intermediate: calls on one grid must not overlap.
 */
pf_status jac_elementwise_study(pf_grid *grid, int32_t strategy, const double *vm, const double *va, double *P,
                                double *Q, double *J, pf_stream stream);

/*
 * Study entry point (the paper's storage comparison, Sec. IV-B.1): the Ybus
 * method's injections with the complex voltages stored interleaved
 * (separate = 0, re/im pairs) or as separate real and imaginary arrays
 * (separate = 1): a phasor launch and a one-row-per-thread CSR SpMV, the
 * arithmetic identical.  Same arguments and results as inj_ybus.  Uses a
 * grid-owned voltage buffer: calls on one grid must not overlap.
 */
pf_status inj_ybus_study(pf_grid *grid, int32_t separate, const double *vm, const double *va, double *P, double *Q,
                         pf_stream stream);

/*
 * Test hook for the error paths: after `after` more device allocations made
 * through the library's buffer owner succeed, every later one fails (no
 * cudaMalloc is attempted) and the call reports PF_ENOMEM, releasing what it
 * had allocated.  after = -1 turns the hook off (the default).  Process-wide.
 */
pf_status pf_debug_fail_allocations(int32_t after);

/* ------------------------------------------------------------ tracing -- */

/* Kernel identifiers reported by the tracer. */
#define PF_K_PHASOR 0        /* phasor step U = e^{j theta}, V = v U (Sec. IV-B.1 step 1) */
#define PF_K_INJ_YBUS 1
#define PF_K_JAC_YBUS 2
#define PF_K_INJ_EW 3
#define PF_K_JAC_EW 4
#define PF_K_INJ_EW_BATCHED 5
#define PF_K_JAC_EW_BATCHED 6
#define PF_K_ADJOINT 7
#define PF_K_INJ_YBUS_BATCHED 8
#define PF_K_JAC_YBUS_BATCHED 9
#define PF_K_REDUCE 10       /* gather of the reduced Jacobian and mismatch vector */
#define PF_K_LOSS 11         /* the mismatch loss alone (loss_elementwise) */
#define PF_K_LU 12           /* sparse LU solve of the reduced system (jac_reduced_solve) */
#define PF_K_COUNT 13

typedef struct {
    int32_t kernel;          /* PF_K_* */
    float ms;                /* device time between CUDA events recorded around the launch */
} pf_trace_rec;

/* Static name of a kernel identifier ("?" if unknown). */
const char *pf_kernel_name(int32_t kernel);

/*
 * Per-launch tracing: with capacity > 0, every kernel launch of this grid's
 * evaluation calls is bracketed by two CUDA events recorded on the launching
 * stream, for up to `capacity` launches (later launches are not recorded).
 * capacity = 0 turns tracing off and frees the events.  Evaluation calls
 * stay asynchronous; tracing adds two cudaEventRecord calls per launch.
 */
pf_status grid_trace_enable(pf_grid *grid, int32_t capacity);

/*
 * Wait for the recorded events, copy up to `cap` records (in launch order)
 * to `out`, set *n to the number of records, and start a new trace.
 */
pf_status grid_trace_read(pf_grid *grid, pf_trace_rec *out, int32_t cap, int32_t *n);

#ifdef __cplusplus
}
#endif

#endif /* PFGRID_H */
