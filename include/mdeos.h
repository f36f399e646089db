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
  MDEOS_REQ_TEMPERATURE = 1u, /* request.e holds a temperature; lifting holds it fixed */
  MDEOS_REQ_COLD = 2u         /* lift from the lattice even if the element has a stored
                                 state (the final state is still stored) */
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
  /* Warm start (element_id != 0, mdeos_submit only): the handle keeps each
   * element's final MD state and lifts its next request from it -- positions
   * scaled affinely to the new box side, velocities kept (mean removed) and
   * rescaled to the Eq. 10 temperature of the scaled configuration, then
   * warm_lift_iters Eq. 10 segments instead of lift_iters.  The store holds
   * warm_slots elements of up to warm_atoms atoms (32 B per atom of device
   * memory, allocated by mdeos_create, counted in hbm_budget_bytes); 0 = off. */
  int32_t warm_lift_iters;     /* Eq. 10 segments after a warm start; default 1 */
  int32_t warm_slots;          /* elements kept; 0 = no warm store */
  int32_t warm_atoms;          /* atoms per stored element (>= natoms of its requests) */
  int32_t nlist_capacity;      /* Verlet-list entries per atom; 0 = from the density (1.3 x
                                  the neighbours within rc + skin at the box density, or at
                                  rho = 0.9 if higher, + 32).  A box whose list overflows is
                                  re-run by mdeos_poll with twice the capacity. */
  int32_t max_cluster;         /* CTAs per box for batches of few boxes (thread-block
                                  clusters, see mdeos_submit): 0 = up to 4, at most 8,
                                  1 = none */
} mdeos_config;

/* One EOS query.  Layout is part of the ABI. */
typedef struct {
  double rho;          /* number density, > 0 */
  double e;            /* specific internal energy per atom (temperature with the flag) */
  double e_ref;        /* energy zero per atom, used with MDEOS_REF_FIXED */
  int32_t natoms;      /* atoms in the MD box, 2..32768 (above 4096: one box per CTA with its
                          state in device memory; mdeos_submit_noalloc takes up to 4096) */
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
  int32_t warm;        /* 1 if lifted from the element's stored state, else 0 */
  int32_t nlist_retries; /* re-runs after a neighbour-list overflow (mdeos_poll) */
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
 * Launch shape: a batch that fills the GPU packs boxes into work items of one
 * CTA; one with no more boxes than SMs gives each box its own CTA; one with fewer
 * boxes than half the SMs, all of at most 768 atoms, runs each box on a
 * thread-block cluster of up to cfg.max_cluster CTAs (each holds the box and computes
 * the forces of its share of the atoms); one with fewer boxes than half the SMs, all
 * above 4096 atoms, does the same with one state per box in global memory (each CTA
 * owns a slab of the cell-ordered atoms).  Results do not depend on the launch shape.
 * Errors: MDEOS_EINVAL (n < 1, NULL, or a request field out of range),
 * MDEOS_ENOMEM, MDEOS_ECUDA. */
mdeos_status mdeos_submit(mdeos_handle* h, const mdeos_request* reqs, int32_t n,
                          uint64_t* ticket);

/* Wait up to timeout_us microseconds (0: do not wait, < 0: wait until done)
 * for a ticket.  On MDEOS_OK the n results are written to `out` (host,
 * caller-owned, n entries, request order) and the ticket is released.
 * Returns MDEOS_PENDING if not done in time, MDEOS_EINVAL for an unknown
 * ticket, MDEOS_ECUDA if the device work failed.  Boxes whose Verlet list
 * overflowed (MDEOS_ENBR) are first re-run here with twice the list capacity, as
 * often as needed up to a capacity of every other atom, with the same warm-start
 * slot; result.nlist_retries counts the re-runs.  The re-runs are synchronous, so
 * such a poll takes correspondingly longer.  Batches (mdeos_batch_*) and
 * mdeos_submit_noalloc report MDEOS_ENBR without re-running. */
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

/* Describe the plan: number of work items, CTAs launched (items x cluster size
 * for a clustered batch), dynamic shared memory per CTA and neighbour-list scratch
 * bytes (host ints/size_t written when the pointer is non-NULL). */
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
 * the device; code whose device memory is owned by a pool).  It calls no
 * cudaMalloc, cudaFree or other allocating routine.  Its work table, queue counter and Verlet lists live in a static
 * device array of MDEOS_NOALLOC_SCRATCH_BYTES that every GPU loading this
 * library holds until exit.
 *
 * cfg:       host, copied; cfg->device must be the calling thread's current device.
 * reqs:      host array of n requests, copied before return.
 * d_results: device array of n mdeos_result, caller-owned; written in request
 *            order when the work on `stream` completes (requests rejected by
 *            the planner get their status there too).
 * stream:    cudaStream_t (NULL = legacy default stream).  The kernel runs
 *            asynchronously, but the work table is copied to the device from
 *            pageable host memory that the call owns, and such a copy may wait
 *            for earlier work on `stream` before the call returns: do not rely
 *            on this call not blocking.  A stream that is being captured into a
 *            CUDA graph is refused with MDEOS_EINVAL (the recorded copies would
 *            point at host memory freed on return).
 * The first call on a device looks up the static array's device address and
 * sets the kernel's shared-memory limit.  Every call reuses the same array (it keeps the previous
 * call's contents; the call clears what must start at zero): calls whose work
 * overlaps on the GPU race, so serialise them (one stream, or events).  A batch
 * whose work table plus one CTA's Verlet lists exceed the array is rejected
 * with MDEOS_EINVAL; smaller scratch per CTA runs on fewer CTAs.  Requests above
 * 4096 atoms get MDEOS_EINVAL in their result (their per-box device state would
 * need an allocation).
 * Errors: MDEOS_EINVAL, MDEOS_ECUDA. */
#define MDEOS_NOALLOC_SCRATCH_BYTES ((size_t)128 << 20)
mdeos_status mdeos_submit_noalloc(const mdeos_config* cfg, const mdeos_request* reqs, int32_t n,
                                  mdeos_result* d_results, void* stream);

/* ---- autotuner ----------------------------------------------------------
 * Two launch choices per box size have no a-priori best value on a given GPU: the
 * Verlet skin (rarer list rebuilds with a larger skin against more pair
 * candidates per step) and the warps that run one box (more warps: more
 * parallelism per box, fewer boxes per CTA).  For every atom count among the
 * Verlet-list boxes of reqs (host, n), one full-GPU wave of such boxes (cycled from
 * reqs, `steps` MD steps each) is timed with CUDA events for every skin in
 * {0.2, 0.25, 0.3, 0.35, 0.4, 0.5} and the planner's warps per box and up to two
 * doublings of it (at most 32); the fastest shape per box whose boxes all succeed
 * (the planner's own -- skin cfg.skin, else 0.3, and its warps -- unless another is
 * faster by 2% or more: one wave's time varies by about a percent) is kept in the
 * handle and used by later planning of that atom count while
 * cfg.skin <= 0 (the skin) and for batches that fill the GPU (the warps; a batch
 * with no more boxes than SMs runs each box in its own CTA, one atom per thread).
 * table (host double[4 * max_out], may be NULL) receives (natoms, skin, warps per
 * box, ms of GPU time per box) rows and *n_out their number.  Synchronous.
 * Errors: MDEOS_EINVAL (steps < 20), MDEOS_ENOMEM, MDEOS_ECUDA. */
mdeos_status mdeos_autotune(mdeos_handle* h, const mdeos_request* reqs, int32_t n, int32_t steps,
                            double* table, int32_t max_out, int32_t* n_out);

/* ---- warm-start store -------------------------------------------------
 * Slot rules: an element_id first seen takes the next free slot (none free:
 * evaluated cold, not stored); a slot is rewritten by every successful
 * evaluation of its element and invalidated by a failed one.  When one
 * mdeos_submit holds an element_id more than once, its first request uses and
 * updates the slot and the others run cold without storing.  mdeos_batch_* and
 * mdeos_submit_noalloc never use the store.  natoms must not exceed warm_atoms
 * (larger requests run cold, not stored). */

/* Copy the stored state of element_id to host x4/v4 (float4[natoms] each:
 * positions in [0, L) with w = atom id as float bits, velocities with w = 0)
 * and its box side to *L.  Waits for the handle's outstanding work.
 * Errors: MDEOS_EINVAL (no valid stored state of that size). */
mdeos_status mdeos_warm_export(mdeos_handle* h, uint64_t element_id, int32_t natoms, float* x4,
                               float* v4, double* L);

/* Store a state for element_id (host float4[natoms] positions in a box of side L
 * and velocities; w components ignored), so its next request warm-starts from it.
 * Errors: MDEOS_EINVAL (no store, natoms > warm_atoms, L <= 0), MDEOS_ENOMEM (no
 * free slot). */
mdeos_status mdeos_warm_import(mdeos_handle* h, uint64_t element_id, int32_t natoms,
                               const float* x4, const float* v4, double L);

/* Forget every stored state (slots are reused). */
mdeos_status mdeos_warm_reset(mdeos_handle* h);

/* ---- 1D Lagrangian hydro caller (Sec. II, Eq. 2-5) ----------------------
 * Planar Lagrangian hydrodynamics on a staggered grid (node x, u; zone mass,
 * rho, e) whose closure P(rho, e) is an ideal gas, the Mie-Grueneisen form of
 * Eq. 1 (linear Us-up Hugoniot as reference curve), or the atomistic EOS of
 * this library, called once per zone and step as one batch (Sec. III, last
 * paragraph).  One step, all in FP64 on the device:
 *   closure P, c^2;  q = rho (q_quad du^2 - q_lin c du) for du = u_{z+1} - u_z < 0;
 *   dt = cfl min dx / (c + 2 q_quad max(-du, 0)), at most dt_grow * previous dt;
 *   u += dt F / M with F_i = (P+q)_{i-1} - (P+q)_i (0 outside a free end; u = 0
 *   at a wall);  x += dt (u_old + u_new) / 2;
 *   e -= dt (P+q) (uh_{z+1} - uh_z) / m (compatible form: total energy is
 *   conserved to round-off);  rho = m / (x_{z+1} - x_z).
 * The MD closure uses c^2 = sound_gamma * max(P / rho, T) (the paper gives no
 * sound speed for it). */
enum { MDEOS_CLOSURE_IDEAL_GAS = 0, MDEOS_CLOSURE_MIE_GRUNEISEN = 1, MDEOS_CLOSURE_MD = 2 };
enum { MDEOS_BC_WALL = 0, MDEOS_BC_FREE = 1 };

typedef struct {
  int32_t nzones;
  int32_t closure;             /* MDEOS_CLOSURE_* */
  int32_t bc_left, bc_right;   /* MDEOS_BC_* */
  double q_quad, q_lin;        /* artificial viscosity constants; default 2, 0.5 */
  double cfl, dt_grow;         /* default 0.5, 1.1 */
  double dt_fixed;             /* > 0: this time step instead of the CFL one */
  double gamma;                /* ideal gas */
  double mg_rho0, mg_c, mg_s, mg_gamma; /* Mie-Grueneisen: rho0, C, s, Gamma */
  /* MD closure: requests of natoms atoms; the first call of each zone uses the
   * *_first step counts (a cold lift), later calls steps_equil / steps_avg and a
   * warm start when the handle has a warm store with >= nzones free slots. */
  int32_t natoms, steps_equil, steps_avg, steps_equil_first, steps_avg_first;
  int32_t first_temperature;   /* 1: the first call lifts at temperature e0[z] and
                                  sets e to the achieved energy (MDEOS_REQ_TEMPERATURE) */
  double e_ref;                /* energy zero per atom (MDEOS_REF_FIXED handles) */
  double sound_gamma;          /* default 3 */
  uint64_t seed;               /* zone z, call k: Philox key seed + (k << 32) + z */
  uint64_t element_base;       /* zone z is element element_base + z + 1 */
} mdeos_hydro_config;

typedef struct mdeos_hydro mdeos_hydro;

/* Defaults: wall ends, q_quad 2, q_lin 0.5, cfl 0.5, dt_grow 1.1, gamma 5/3,
 * sound_gamma 3; the rest 0. */
void mdeos_hydro_config_default(mdeos_hydro_config* cfg);

/* Create a hydro problem on handle h's device and stream (h stays owned by the
 * caller and must outlive the problem).  x, u: host double[nzones + 1] node
 * positions (strictly increasing) and velocities; rho, e0: host double[nzones]
 * zone densities and specific energies (temperatures with first_temperature).
 * Copied.  Errors: MDEOS_EINVAL, MDEOS_ENOMEM, MDEOS_ECUDA. */
mdeos_status mdeos_hydro_create(mdeos_handle* h, const mdeos_hydro_config* cfg, const double* x,
                                const double* u, const double* rho, const double* e0,
                                mdeos_hydro** out);

/* Advance nsteps steps (synchronous).  Analytic closures run all steps in one
 * launch; the MD closure runs one EOS batch and one hydro launch per step.
 * Errors: MDEOS_EUNPHYS (tangled mesh, non-finite state, or an EOS box that
 * failed; the state is left at the last good step), MDEOS_ECUDA. */
mdeos_status mdeos_hydro_step(mdeos_hydro* hy, int32_t nsteps);

/* Copy the state to host arrays (any may be NULL): x, u double[nzones + 1];
 * rho, e, P, q, c2 double[nzones] (P, q, c2 of the last step);
 * clock double[3] = (time, last dt, steps taken). */
mdeos_status mdeos_hydro_state(mdeos_hydro* hy, double* x, double* u, double* rho, double* e,
                               double* P, double* q, double* c2, double* clock);

/* Results of the last MD-closure batch (host mdeos_result[nzones]).
 * Errors: MDEOS_EINVAL if the closure is not MD or no step ran. */
mdeos_status mdeos_hydro_eos_results(mdeos_hydro* hy, mdeos_result* out);

mdeos_status mdeos_hydro_destroy(mdeos_hydro* hy);

/* ---- serving loop (continuous batching) --------------------------------
 * The paper has no serving layer (each FEM element waits for its own MD run);
 * this is the many-client form of the same evaluation.  One persistent kernel
 * grid (one CTA per SM) claims work items one at a time from a queue that the
 * server's scheduler thread keeps appending to: arriving requests are planned
 * into items (boxes of one size class, LPT order within an admission step) and
 * published into host-mapped rings; every SM takes the next item as soon as it
 * finishes one, and each request is reported as soon as its box is done (result
 * and ready flag in host-mapped memory).  An idle grid exits after idle_ms and is
 * relaunched when work arrives.
 *
 * Element states (warm = 1): the server keeps each element's final MD state in a
 * device store and lifts the element's next request from it, as the handle's warm
 * store does (warm_lift_iters of the handle's configuration).  A stored element
 * takes 16 + 32 B per atom (requests above 4096 atoms run cold, not stored).  A
 * request is admitted only when its element's state has room: memory of elements
 * with no request in flight is reclaimed least recently used first; while the rest
 * of the store is held by requests in flight, the request waits in the queue and is
 * admitted as their results come back (so the store, within hbm_budget_bytes, bounds
 * the device memory however many requests arrive).  A second request for an element
 * whose previous request is still in flight waits for it.  Requests with
 * element_id 0 need no store memory. */
typedef struct {
  int32_t max_inflight;     /* requests admitted to the GPU and not finished, default 4096 */
  int32_t max_batch;        /* requests planned together per admission step, default 2048 */
  double max_wait_s;        /* waiting longer than this: shed (MDEOS_ECANCELLED); 0 = never */
  int32_t max_queue;        /* waiting requests beyond this are shed on arrival; 0 = no cap */
  int32_t idle_ms;          /* an idle kernel exits after this long, default 20 */
  size_t hbm_budget_bytes;  /* device memory the server may hold: the per-SM scratch for the
                               largest box (32768 atoms) plus the element store; creation
                               fails if the scratch alone exceeds it; 0 = no cap */
  int32_t warm;             /* 1: keep element states for warm starts (see above); 0: off */
  int32_t cluster;          /* CTAs per thread-block cluster of the serving grid (0 or 1 =
                               none, else 2, 4 or 8): in rounds, a cluster runs one
                               request above 4096 atoms on all its CTAs (each a slab of
                               the box's atoms) or lets each CTA claim items of smaller
                               boxes; large boxes finish sooner (lower p99 below
                               saturation), the rounds lower the capacity */
  size_t warm_bytes;        /* element store size; 0 = what hbm_budget_bytes leaves after the
                               scratch (1 GiB without a budget) */
} mdeos_serve_config;

/* One finished request.  Times are seconds on the server clock (mdeos_serve_clock):
 * arrival = enqueue, launch = published to the GPU queue, done = when the server saw
 * its result.  result.status: the box's status, MDEOS_ECANCELLED if shed,
 * MDEOS_ENOMEM if its box needs more per-SM scratch than the server holds,
 * MDEOS_EINVAL if rejected by the planner, MDEOS_ECUDA if the kernel failed. */
typedef struct {
  uint64_t id;
  double t_arrival, t_launch, t_done;
  mdeos_result result;
} mdeos_served;

typedef struct mdeos_server mdeos_server;

/* Defaults: 4096 in flight, admission steps of up to 2048, no shedding, idle exit
 * after 20 ms, no budget. */
void mdeos_serve_config_default(mdeos_serve_config* cfg);

/* Start a server on handle h (caller-owned, must outlive the server); cfg copied.
 * With cfg->cluster > 1 the serving grid runs in thread-block clusters (see the
 * field); results do not depend on it.
 * Errors: MDEOS_EINVAL (cluster not 0, 1, 2, 4 or 8), MDEOS_ENOMEM (budget below the
 * scratch), MDEOS_ECUDA. */
mdeos_status mdeos_serve_create(mdeos_handle* h, const mdeos_serve_config* cfg,
                                mdeos_server** out);

/* Seconds since mdeos_serve_create (steady clock). */
double mdeos_serve_clock(const mdeos_server* s);

/* Queue n host requests (copied); ids (host uint64[n], may be NULL) receives their
 * ids.  Thread-safe.  Arrivals beyond max_queue are shed at once. */
mdeos_status mdeos_serve_enqueue(mdeos_server* s, const mdeos_request* reqs, int32_t n,
                                 uint64_t* ids);

/* Move up to max finished requests into out (host, caller-owned); *n_out = count.
 * Non-blocking, thread-safe; completion order. */
mdeos_status mdeos_serve_completed(mdeos_server* s, mdeos_served* out, int32_t max,
                                   int32_t* n_out);

/* counts (host int64[7], may be NULL): enqueued, admitted, finished, shed,
 * kernel launches, waiting now, CUDA failures; bytes (host size_t[2], may be NULL):
 * device bytes held by the server and the peak number of requests in flight. */
mdeos_status mdeos_serve_stats(mdeos_server* s, long long* counts, size_t* bytes);

/* Element store counters: counts (host int64[4], may be NULL): warm-started
 * requests, admissions that waited for store memory, states evicted, elements
 * stored now; bytes (host size_t[2], may be NULL): store bytes in use (reserved by
 * stored elements) and the store's size. */
mdeos_status mdeos_serve_store_stats(mdeos_server* s, long long* counts, size_t* bytes);

/* Stop: waiting requests are shed, in-flight launches finish; then release. */
mdeos_status mdeos_serve_destroy(mdeos_server* s);

/* ---- surrogate EOS (MLP ensemble gate) ----------------------------------
 * An ensemble of n_models MLPs 2 -> 128 -> 128 -> 128 -> 2 (tanh hidden layers)
 * maps (rho, e), normalised by mean and standard deviation, to normalised (P, T).
 * BF16 weights and hidden activations, FP32 accumulation and FP32 master weights;
 * the 128-wide layers run on the tensor cores.  Trained with Adam on MD answers;
 * used as a gate: where the ensemble agrees the surrogate answers, elsewhere the
 * request goes to the MD path.  The paper runs MD for every query (Sec. III) and
 * points to learned accelerators of such couplings (Sec. I); this is one.
 * Parameter vector per model (FP32, 33,666 values): W1[128,2] b1[128] W2[128,128]
 * b2[128] W3[128,128] b3[128] W4[2,128] b4[2] (W[out,in], row-major).
 * Normalisers norm[8]: mean(rho), mean(e), sd(rho), sd(e), mean(P), mean(T), sd(P), sd(T). */
#define MDEOS_SURROGATE_NPARAM 33666
typedef struct mdeos_surrogate mdeos_surrogate;

/* Create on handle h (caller-owned, outlives it) with Glorot-uniform weights from
 * `seed`; batches up to max_batch samples per launch.  Errors: EINVAL, ECUDA. */
mdeos_status mdeos_surrogate_create(mdeos_handle* h, int32_t n_models, int32_t max_batch,
                                    uint64_t seed, mdeos_surrogate** out);

/* Set (params: host float[n_models * NPARAM], resets Adam) and/or normalisers
 * (norm: host double[8]); either may be NULL. */
mdeos_status mdeos_surrogate_set_params(mdeos_surrogate* s, const float* params,
                                        const double* norm);
mdeos_status mdeos_surrogate_get_params(mdeos_surrogate* s, float* params, double* norm);

/* Mean-squared-error gradients of one batch (x: host double[n][2] = (rho, e), y: host
 * double[n][2] = (P, T), n <= max_batch) into grads (host float[n_models * NPARAM]);
 * *loss = the batch loss averaged over the models.  No update. */
mdeos_status mdeos_surrogate_grads(mdeos_surrogate* s, const double* x, const double* y,
                                   int32_t n, float* grads, double* loss);

/* Adam training (beta 0.9 / 0.999, eps 1e-8) for `epochs` passes over n samples in
 * shuffled full batches of `batch`; set_norm != 0 first sets the normalisers from
 * the data.  loss_out (host double[epochs], may be NULL): mean batch loss per epoch. */
mdeos_status mdeos_surrogate_train(mdeos_surrogate* s, const double* x, const double* y,
                                   int32_t n, int32_t epochs, int32_t batch, double lr,
                                   uint64_t seed, int32_t set_norm, double* loss_out);

/* Ensemble prediction for n inputs (host double[n][2]): mean and population standard
 * deviation over the models of (P, T) (host double[n][2] each, may be NULL) and the
 * per-model normalised outputs (host float[n_models][n][2], may be NULL).
 * Synchronous.  ETIMEDOUT if a tensor-core completion wait ran out (about 1 s). */
mdeos_status mdeos_surrogate_predict(mdeos_surrogate* s, const double* x, int32_t n,
                                     double* mean, double* sd, float* per_model);

/* Inference paths.  TC (default): one fused kernel per 128 inputs and model; layer 1
 * on the CUDA cores, the two 128 x 128 layers as tcgen05.mma with the accumulator in
 * tensor memory, bias + tanh + the output layer in the epilogue.  MMA: the layered
 * path the training step uses (its tcgen05 GEMMs, one per layer over all inputs, and
 * elementwise kernels, activations through device memory).  Both apply the same bf16
 * roundings; they differ only in the FP32 summation order.  EINVAL for any other
 * value. */
#define MDEOS_SURROGATE_INFER_TC 0
#define MDEOS_SURROGATE_INFER_MMA 1
mdeos_status mdeos_surrogate_set_infer_path(mdeos_surrogate* s, int32_t path);

/* How the networks represent the pressure output.  LINEAR (default): P itself,
 * standardised.  ASINH: asinh(P), standardised, mapped back with sinh before the
 * ensemble mean and spread -- linear for |P| < 1 and logarithmic above, so the
 * squared-error loss weighs errors as |dP| / max(|P|, 1), the gate's error measure.
 * Set it before training (the normalisers of mdeos_surrogate_train's set_norm are
 * taken in the chosen units); predictions are always in physical units.  Errors:
 * EINVAL for any other value. */
#define MDEOS_SURROGATE_P_LINEAR 0
#define MDEOS_SURROGATE_P_ASINH 1
mdeos_status mdeos_surrogate_set_output_transform(mdeos_surrogate* s, int32_t mode);

/* Prediction on device arrays, asynchronous on `stream` (cudaStream_t; NULL = the
 * handle's stream): d_x device double[n][2] = (rho, e) in; d_mean and d_sd device
 * double[n][2] = ensemble mean and spread of (P, T) out (all caller-owned, non-NULL
 * when n > 0).  Uses the surrogate's scratch: serialise with its other calls.  A
 * tensor-core wait that ran out writes NaN for its inputs (and makes the next
 * mdeos_surrogate_predict return ETIMEDOUT).  Errors: EINVAL, ECUDA. */
mdeos_status mdeos_surrogate_infer_device(mdeos_surrogate* s, const double* d_x, int32_t n,
                                          double* d_mean, double* d_sd, void* stream);

/* Misfit map of the gate (Sec. I's learned accelerators answer only where they are
 * reliable; the members' spread does not see a region where all of them miss the
 * same rough data, such as a phase boundary).  fit_misfit predicts the ensemble mean
 * at n inputs x (host double[n][2] = (rho, e)) with MD answers y (host double[n][2] =
 * (P, T)), and keeps per cell of a bins x bins grid over the inputs' range (1..1024)
 * the RMS of |mean P - P| / max(|P|, 1); cells with fewer than min_count samples are
 * unknown (infinite).  misfit (host out double[n]) reads the map at n inputs (outside
 * the fitted range: infinite).  set_misfit_threshold: the gate also sends to MD every
 * request whose cell exceeds the threshold (INFINITY, the default: the map is not
 * used).  Errors: EINVAL (bad arguments, no map fitted), ECUDA. */
mdeos_status mdeos_surrogate_fit_misfit(mdeos_surrogate* s, const double* x, const double* y,
                                        int32_t n, int32_t bins, int32_t min_count);
mdeos_status mdeos_surrogate_misfit(const mdeos_surrogate* s, const double* x, int32_t n,
                                    double* out);
mdeos_status mdeos_surrogate_set_misfit_threshold(mdeos_surrogate* s, double threshold);

/* Gated evaluation of n requests: where sd(P) <= threshold * max(|mean P|, 1) (and
 * the request's misfit cell is within the misfit threshold, when one is set) the
 * result is the ensemble mean (path = -2, P_se / T_se = the ensemble spread), else
 * the request runs on the MD path with natoms = md_natoms (> 0) or its own.
 * used_md (host int32[n], may be NULL) marks the MD answers.  Synchronous. */
mdeos_status mdeos_surrogate_gated_eval(mdeos_surrogate* s, const mdeos_request* reqs, int32_t n,
                                        double threshold, int32_t md_natoms, mdeos_result* out,
                                        int32_t* used_md);

mdeos_status mdeos_surrogate_destroy(mdeos_surrogate* s);

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

/* The pair-force pass on its own (measurement of the force kernel): nbox boxes of
 * n atoms (device x4: float4[nbox * n], box b at x4 + 4 n b), one per CTA and at
 * most one per SM, each kept in shared memory with its Verlet list (skin) built
 * once, then `passes` force passes as the step loop runs them: mode 0 forces only,
 * mode 1 forces with energy, virial and pair count; mode 2 runs `passes` list builds
 * instead (the build measured on its own).  cycles (device int64[2 nbox])
 * receives per box the SM cycles of the passes and the list entries per pass.
 * Synchronous on `stream`.  Errors: MDEOS_EINVAL, MDEOS_ENOMEM, MDEOS_ECUDA. */
mdeos_status mdeos_debug_force_bench(const mdeos_config* cfg, const float* x4, int32_t nbox,
                                     int32_t n, double L, double skin, int32_t passes,
                                     int32_t mode, long long* cycles, void* stream);

/* The surrogate's tensor-core GEMM on its own: C(m, n) = sum_k A(m, k) B(k, n) with
 * A(m, k) = A[m * sa_m + k * sa_k], B(k, n) = B[k * sb_k + n * sb_n] (device bfloat16
 * bit patterns) and C(m, n) = C[m * sc_m + n * sc_n] (device float). */
mdeos_status mdeos_debug_gemm_bf16(const uint16_t* A, const uint16_t* B, float* C, int32_t M,
                                   int32_t N, int32_t K, int64_t sa_m, int64_t sa_k, int64_t sb_k,
                                   int64_t sb_n, int64_t sc_m, int64_t sc_n, void* stream);

/* The surrogate's hidden-layer tanh on its own: y[i] = tanh(x[i]) for n device floats
 * (relative error below 2e-6: an exp2 form, and an odd series below |x| = 1/4).
 * Synchronous on `stream` (cudaStream_t).  Errors: MDEOS_EINVAL (NULL, n < 1),
 * MDEOS_ECUDA. */
mdeos_status mdeos_debug_tanh(const float* x, float* y, int32_t n, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MDEOS_H */
