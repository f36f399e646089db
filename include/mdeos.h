/*
 * mdeos.h -- C ABI of the GB300 batched in-line atomistic EOS evaluation.
 *
 * Each request is one hydro element's (density, specific internal energy).
 * The library lifts it into its own periodic Lennard-Jones MD box, integrates
 * the box on the GPU and restricts the trajectory back to a time-averaged
 * pressure, temperature and stress tensor.  This follows the lifting ->
 * microscopic evolution -> restriction statement of arXiv 2508.06012,
 * Sec. III (Eq. 6-11), with one independent MD run per element and call
 * (Sec. III, last paragraph; App. C.1).
 *
 * Conventions for every entry point:
 *  - Return value: a call-level mdeos_status; per-box errors go into
 *    mdeos_result.status.  Nothing aborts or throws across the ABI.
 *  - Memory: pointers documented "host" are ordinary CPU memory owned by the
 *    caller; "device" pointers are CUDA global memory of the handle's device,
 *    owned by the caller.  The library copies what it needs before a call
 *    returns unless stated otherwise.
 *  - No CPU fallback: without a usable CUDA device mdeos_create returns
 *    MDEOS_ECUDA.
 *  - mdeos_last_error() returns a thread-local message for the most recent
 *    failing call on this thread.
 *  - Units: reduced Lennard-Jones units by default (eps = sigma = m = k_B = 1);
 *    densities are number densities, energies are per atom.
 */
#ifndef MDEOS_H
#define MDEOS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MDEOS_OK = 0,
  MDEOS_PENDING = 1,     /* mdeos_poll: not finished yet */
  MDEOS_EINVAL = -1,     /* bad argument or request */
  MDEOS_ENOMEM = -2,     /* device memory (or the HBM budget) exhausted */
  MDEOS_EUNPHYS = -3,    /* lifting temperature <= 0 (e below the cold curve) or NaN/Inf */
  MDEOS_EBOX = -4,       /* box side L below the cutoff rc */
  MDEOS_ETIMEDOUT = -5,  /* a bounded wait ran out */
  MDEOS_ECUDA = -6,      /* CUDA runtime error or no device */
  MDEOS_ECANCELLED = -7, /* request cancelled */
  MDEOS_ENBR = -8        /* neighbour-list capacity exceeded for this box */
} mdeos_status;

/* Energy zero of the lifting (Sec. III, Eq. 8-10). */
enum {
  MDEOS_REF_ECOLD = 0, /* paper: N e = E_kin + E_pot - E_cold(rho), E_cold per call */
  MDEOS_REF_FIXED = 1  /* N e = E_kin + E_pot - N e_ref, e_ref from the request */
};

/* mdeos_request.flags */
enum {
  MDEOS_REQ_TEMPERATURE = 1u /* request.e holds a temperature; lifting holds it fixed */
};

/* Library configuration.  Fill with mdeos_config_default, then override. */
typedef struct {
  int32_t device;              /* CUDA device ordinal */
  int32_t lift_iters;          /* Eq. 10 temperature updates (NVE segments); paper: 2 */
  int32_t rescale_every_equil; /* thermostat period inside a lifting segment; 0 = NVE */
  int32_t rescale_every_avg;   /* production thermostat period (NVT); 0 = NVE */
  int32_t se_blocks;           /* blocks for the standard error, 2..32 */
  int32_t energy_ref_mode;     /* MDEOS_REF_ECOLD or MDEOS_REF_FIXED */
  double eps, sigma, mass;     /* Lennard-Jones parameters */
  double rc;                   /* cutoff, truncated and shifted */
  double dt;                   /* MD time step */
  double skin;                 /* Verlet-list skin; <= 0 lets the autotuner choose */
  size_t hbm_budget_bytes;     /* cap on library device memory; 0 = no cap */
  void* cuda_stream;           /* cudaStream_t to run on; NULL = library-owned stream */
} mdeos_config;

/* One EOS query.  Layout is part of the ABI. */
typedef struct {
  double rho;          /* number density, > 0 */
  double e;            /* specific internal energy per atom (temperature with the flag) */
  double e_ref;        /* energy zero per atom, used with MDEOS_REF_FIXED */
  int32_t natoms;      /* atoms in the MD box, 2..4096 */
  int32_t steps_equil; /* lifting steps, split into lift_iters NVE segments (0 = none) */
  int32_t steps_avg;   /* production steps averaged by the restriction, >= se_blocks */
  uint32_t flags;      /* MDEOS_REQ_* */
  uint64_t seed;       /* velocity draw: Philox4x32-10 key */
  uint64_t element_id; /* caller's tag, copied to the result */
} mdeos_request;

/* One EOS answer (time averages over the production steps). */
typedef struct {
  double P;            /* pressure = mean normal stress (Eq. 11) */
  double T;            /* kinetic temperature 2 <E_kin> / N_DOF, N_DOF = 3N - 3 */
  double sigma[6];     /* stress tensor xx yy zz xy xz yz (Eq. 11, pair form) */
  double epot, ekin;   /* <E_pot>/N, <E_kin>/N */
  double e_achieved;   /* (<E_kin> + <E_pot> - E_ref)/N */
  double P_se, T_se;   /* block-average standard errors */
  double T_target;     /* last lifting temperature = production thermostat target */
  double e_cold;       /* E_cold / N of the lifted lattice */
  double L;            /* box side */
  double pairs_per_step; /* in-cutoff ordered pairs per step, mean over production steps */
  double cand_per_step;  /* pair candidates evaluated per step, same average */
  uint64_t element_id; /* copied from the request */
  int32_t natoms;
  int32_t status;      /* mdeos_status of this box */
  int32_t nlist_builds;/* neighbour-list rebuilds (diagnostic) */
  int32_t path;        /* force path used: 0 all-pairs, 1 all-pairs multi-image, 2 Verlet list */
} mdeos_result;

typedef struct mdeos_handle mdeos_handle;
typedef struct mdeos_batch mdeos_batch;

/* Fill *cfg with the defaults: device 0, lift_iters 2, NVE segments,
 * rescale_every_avg 10, se_blocks 10, REF_ECOLD, eps = sigma = mass = 1,
 * rc 2.5, dt 0.005, autotuned skin, no budget, library-owned stream. */
void mdeos_config_default(mdeos_config* cfg);

/* Create a handle on cfg->device (cfg host, copied).  *out receives an
 * opaque handle owned by the library until mdeos_destroy.
 * Errors: MDEOS_EINVAL (bad cfg), MDEOS_ECUDA (no device / CUDA error). */
mdeos_status mdeos_create(const mdeos_config* cfg, mdeos_handle** out);

/* Submit n host requests (copied before return) and start them on the GPU.
 * *ticket receives an id for mdeos_poll.  The whole batch runs as one
 * persistent kernel launch; per-box problems are reported in the results.
 * Errors: MDEOS_EINVAL (n < 1, NULL, or a request field out of range),
 * MDEOS_ENOMEM, MDEOS_ECUDA. */
mdeos_status mdeos_submit(mdeos_handle* h, const mdeos_request* reqs, int32_t n,
                          uint64_t* ticket);

/* Wait up to timeout_us microseconds (0: do not wait, < 0: wait until done)
 * for a ticket.  On MDEOS_OK the n results are written to `out` (host,
 * caller-owned, n entries, request order) and the ticket is released.
 * Returns MDEOS_PENDING if not done in time, MDEOS_EINVAL for an unknown
 * ticket, MDEOS_ECUDA if the device work failed. */
mdeos_status mdeos_poll(mdeos_handle* h, uint64_t ticket, mdeos_result* out, int32_t timeout_us);

/* Release the handle; waits for outstanding work. */
mdeos_status mdeos_destroy(mdeos_handle* h);

/* Thread-local text for the last failing call on this thread (never NULL). */
const char* mdeos_last_error(void);

/* ---- device-resident batches ------------------------------------------
 * Plan a batch once (packing, autotuned launch shape, uploads of the
 * requests and the work table, capture of one CUDA graph), then replay it
 * with inputs and outputs resident in device memory. */

/* Plan n host requests (copied) into a reusable batch.  *out owned by the
 * library until mdeos_batch_destroy. */
mdeos_status mdeos_batch_create(mdeos_handle* h, const mdeos_request* reqs, int32_t n,
                                mdeos_batch** out);
/* Launch the batch graph on `stream` (cudaStream_t; NULL = handle stream).
 * Asynchronous; results land in the batch's device result array. */
mdeos_status mdeos_batch_launch(mdeos_batch* b, void* stream);
/* Device pointer to the batch's n mdeos_result records (valid until destroy). */
mdeos_result* mdeos_batch_device_results(mdeos_batch* b);
/* Synchronise and copy the n results into host memory `out`. */
mdeos_status mdeos_batch_results(mdeos_batch* b, mdeos_result* out);
mdeos_status mdeos_batch_destroy(mdeos_batch* b);

/* Describe the plan: number of work items, CTAs launched, dynamic shared
 * memory per CTA, neighbour-list scratch bytes, and a 64-bit checksum of
 * the packing (host ints/size_t written when the pointer is non-NULL). */
mdeos_status mdeos_batch_info(const mdeos_batch* b, int32_t* n_items, int32_t* n_ctas,
                              int32_t* smem_bytes, size_t* scratch_bytes);

/* Counters of handle h: bytes copied host->device and device->host by the
 * most recent mdeos_submit, kernels launched by the library on this handle
 * since creation, and device bytes currently held (host outputs; any may be
 * NULL).  Errors: MDEOS_EINVAL for a NULL handle. */
mdeos_status mdeos_stats(const mdeos_handle* h, size_t* last_h2d_bytes, size_t* last_d2h_bytes,
                         long long* kernel_launches, size_t* device_bytes);

/* ---- evaluation without device allocation -----------------------------
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory where they need an EOS answer (a material-model
 * callback inside a hydrocode's time step, where cudaMalloc would synchronise
 * the device; code whose device memory is owned by a pool; host threads that
 * must not block).  It calls no cudaMalloc, cudaFree or other allocating
 * routine.  Its work table, queue counter and Verlet lists live in a static
 * device array of MDEOS_NOALLOC_SCRATCH_BYTES that every GPU loading this
 * library holds until exit.
 *
 * cfg:       host, copied; cfg->device must be the calling thread's current device.
 * reqs:      host array of n requests, copied before return.
 * d_results: device array of n mdeos_result, caller-owned; written in request
 *            order when the work on `stream` completes (requests rejected by
 *            the planner get their status there too).
 * stream:    cudaStream_t (NULL = legacy default stream); asynchronous.
 * The first call on a device looks up the static array's device address and
 * sets the kernel's shared-memory limit; make that first call before any
 * stream capture.  Every call reuses the same array (it keeps the previous
 * call's contents; the call clears what must start at zero): calls whose work
 * overlaps on the GPU race, so serialise them (one stream, or events).  A batch
 * whose work table plus one CTA's Verlet lists exceed the array is rejected
 * with MDEOS_EINVAL; smaller scratch per CTA runs on fewer CTAs.
 * Errors: MDEOS_EINVAL, MDEOS_ECUDA. */
#define MDEOS_NOALLOC_SCRATCH_BYTES ((size_t)128 << 20)
mdeos_status mdeos_submit_noalloc(const mdeos_config* cfg, const mdeos_request* reqs, int32_t n,
                                  mdeos_result* d_results, void* stream);

/* ---- single-box kernels exposed for parity tests ----------------------
 * These run one box through the same device code as the batch path. */

/* Lifting of one box on the device (Eq. 6, 7, 9): FCC lattice positions
 * (x4: device float4[n], w unused), Maxwell velocities at temperature T with
 * zero momentum (v4: device float4[n]) and E_cold (e_out: device double[1]).
 * L is the box side used (host double out). */
mdeos_status mdeos_debug_lift(const mdeos_config* cfg, int32_t n, double rho, double T,
                              uint64_t seed, float* x4, float* v4, double* e_out, double* L_out,
                              void* stream);

/* Forces on n atoms at device positions x4 (float4[n]) in a cubic box of side
 * L through force path `path` (0 all-pairs, 1 all-pairs multi-image, 2 Verlet
 * list with the given skin).  Writes device f4 (float4[n]) and ew (device
 * double[7]: E_pot, W_xx W_yy W_zz W_xy W_xz W_yz, W = sum_{i<j} r_ij (x) f_ij)
 * and, if pairs != NULL, the in-cutoff ordered pair count (device int64[1]). */
mdeos_status mdeos_debug_forces(const mdeos_config* cfg, const float* x4, int32_t n, double L,
                                int32_t path, double skin, float* f4, double* ew,
                                long long* pairs, void* stream);

/* Velocity-Verlet on one box from device x4/v4 (float4[n], updated in place)
 * for `steps` steps, rescaling velocities to T_target every rescale_every
 * steps (0 = NVE).  Per-step E_pot and E_kin go to device double[steps]
 * arrays epot/ekin (either may be NULL).  Positions are returned wrapped
 * into [0, L).  If cycles != NULL (device int64[11]) it receives the SM
 * cycles spent in drift, list builds, forces and kick + reductions, the number
 * of list builds, and the list build's phases (count, scan, scatter, cell sort,
 * permute, search). */
mdeos_status mdeos_debug_md(const mdeos_config* cfg, float* x4, float* v4, int32_t n, double L,
                            int32_t steps, double T_target, int32_t rescale_every, int32_t path,
                            double skin, double* epot, double* ekin, long long* cycles,
                            void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MDEOS_H */
