/*
 * mdeos_oracle.h -- plain FP64 CPU reference of the batched atomistic EOS
 * evaluation (lifting -> MD -> restriction) of arXiv 2508.06012, Sec. III.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library includes,
 * links or calls this code; only tests/, the smoke check and the
 * cpu_baseline / reference arm of bench.py do.  It shares no header,
 * helper or constant with the CUDA path.
 *
 * Units: Lennard-Jones reduced units are typical (eps = sigma = m = k_B = 1)
 * but eps, sigma, mass are parameters.  All arithmetic is double precision.
 */
#ifndef MDEOS_ORACLE_H
#define MDEOS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_OK = 0,
  ORC_EINVAL = -1,
  ORC_EUNPHYS = -3, /* lifting temperature <= 0, NaN/Inf in the state */
  ORC_EBOX = -4     /* box side below the cutoff */
};

enum { ORC_REF_ECOLD = 0, ORC_REF_FIXED = 1 };
enum { ORC_FORCE_ALLPAIRS = 0, ORC_FORCE_CELL = 1 };
/* request flag: the energy field holds a target temperature instead of e */
enum { ORC_REQ_TEMPERATURE = 1u };

typedef struct {
  double eps, sigma, mass, rc, dt;
  int lift_iters;          /* Eq. 10 temperature updates = NVE equilibration segments, paper: 2 */
  int rescale_every_equil; /* thermostat period inside a segment, steps (0 = NVE, the reading) */
  int rescale_every_avg;   /* thermostat period during averaging (0 = NVE) */
  int se_blocks;           /* block count for the standard error */
  int energy_ref_mode;     /* ORC_REF_ECOLD (paper) or ORC_REF_FIXED */
  int force_mode;          /* ORC_FORCE_ALLPAIRS or ORC_FORCE_CELL */
  int warm_lift_iters;     /* Eq. 10 segments after a warm start */
} orc_params;

typedef struct {
  double rho;      /* number density */
  double e;        /* specific internal energy per atom (or T if ORC_REQ_TEMPERATURE) */
  double e_ref;    /* energy zero per atom for ORC_REF_FIXED */
  int natoms, steps_equil, steps_avg;
  uint32_t flags;
  uint64_t seed;
} orc_request;

typedef struct {
  double P, T, sigma[6]; /* sigma order: xx yy zz xy xz yz */
  double epot, ekin;     /* time averages per atom */
  double e_achieved;     /* (<Ekin> + <Epot> - E_ref) / N */
  double P_se, T_se;     /* block-average standard errors */
  double T_target;       /* last lifting temperature (production thermostat target) */
  double e_cold;         /* E_cold / N */
  double L;
  int status;
} orc_result;

/* Philox4x32-10 counter-based generator (Salmon et al., SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* FCC lattice lifting (Eq. 6-7): first n sites of ceil((n/4)^(1/3))^3 cells. */
int orc_lattice_fcc(int n, double rho, double* x, double* L_out);

/* Maxwell velocities at temperature T: Philox + Box-Muller, zero momentum,
 * exact rescale to T with N_DOF = 3N - 3. */
void orc_init_velocities(int n, uint64_t seed, double T, double mass, double* v);

/* LJ forces, potential energy and pair virial W[6] = sum_{i<j} r_ij (x) f_ij.
 * Returns E_pot.  Handles every periodic image within rc (needs L >= rc). */
double orc_lj_forces(int n, const double* x, double L, const orc_params* p, int mode,
                     double* f, double W[6]);

/* In-cutoff ordered pair count (i != j, all images) of a configuration. */
long long orc_count_pairs(int n, const double* x, double L, double rc);

/* Plain velocity-Verlet steps with optional velocity rescale to T_target
 * every `rescale_every` steps (0 = NVE).  On return f holds the last forces.
 * Energies of each step are written to epot_out/ekin_out if non-NULL. */
int orc_md_steps(int n, double* x, double* v, double* f, double L, const orc_params* p,
                 int steps, double T_target, int rescale_every, double* epot_out,
                 double* ekin_out);

/* Kinetic energy 1/2 m sum v^2. */
double orc_kinetic(int n, const double* v, double mass);

/* Block-average mean and standard error of a series of m samples in nb blocks of
 * (near) equal count: the error bar of the restricted P and T (App. B). */
int orc_block_se(const double* x, int m, int nb, double* mean_out, double* se_out);

/* Full lifting -> MD -> restriction for one request (Sec. III, Eq. 6-11). */
int orc_eos_eval(const orc_request* rq, const orc_params* p, orc_result* out);

/* Same with a warm start from a previous state (x_in, v_in: 3n doubles each,
 * box side L_in; NULL = cold) and the final state written to x_out, v_out
 * (NULL = not kept).  Warm reading: positions scaled by L / L_in, velocities
 * kept with their mean removed, one Eq. 10 temperature from the scaled
 * configuration, then warm_lift_iters Eq. 10 segments before averaging. */
int orc_eos_eval_state(const orc_request* rq, const orc_params* p, const double* x_in,
                       const double* v_in, double L_in, double* x_out, double* v_out,
                       orc_result* out);

/* Batch form of orc_eos_eval_state; every request has rq[0].natoms atoms,
 * state arrays hold 3 * natoms doubles per request; L_in[i] <= 0 = cold. */
int orc_eos_batch_state(const orc_request* rq, int n, const orc_params* p, const double* x_in,
                        const double* v_in, const double* L_in, double* x_out, double* v_out,
                        orc_result* out, int nthreads);

/* Same for a batch, OpenMP over requests (nthreads <= 0: all cores). */
int orc_eos_batch(const orc_request* rq, int n, const orc_params* p, orc_result* out,
                  int nthreads);

/* Threads the batch call would use. */
int orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
