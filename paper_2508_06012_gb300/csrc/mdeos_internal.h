// Internal types shared by the host engine and the device kernels of the
// batched atomistic EOS path.  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/mdeos.h"

namespace mdeos {

// Force paths (per box, chosen by the planner).
enum Path : int {
  PATH_ALLPAIRS = 0,    // every j broadcast from shared memory, minimum image (L >= 2 rc)
  PATH_ALLPAIRS_MI = 1, // every j, the two nearest images per axis (rc <= L < 2 rc)
  PATH_NLIST = 2        // Verlet list with skin, rebuilt from a shared-memory cell list
};

constexpr int kMaxBoxesPerItem = 8;   // named barriers 1..8 (0 is the CTA barrier)
constexpr int kCtaThreads = 1024;
constexpr int kMaxAtoms = 4096;       // 1024 threads x 4 atoms per thread
constexpr int kMaxSeBlocks = 32;
constexpr int kMaxCells = 1728;       // cell-list cells per box (12 per axis)
constexpr int kRedSlots = 11;         // reduction quantities per warp (64-bit fixed point)
constexpr int kMaxCluster = 8;        // CTAs of a thread-block cluster that share one box
// boxes above kMaxAtoms run one per CTA with their state in global memory
constexpr int kMaxAtomsBig = 32768;   // uint16 neighbour indices
constexpr int kMaxCellsBig = 32768;   // cells of the list build (<= 32 per axis)
constexpr int kBigSharedBytes = 4096; // shared memory of a big-box CTA (reductions only)

// Cells per axis of a shared-memory box's Verlet-list build: side at least
// R / 2 (R = rc + skin), at most 12 per axis; 0 = no cell grid (a scan of all
// atoms, for boxes of at most kBruteMaxAtoms atoms, where it is the cheaper search).  The search walks the 5 x 5 x 5 cells around an atom's home cell, which
// is valid for any such grid once L >= 2 R (a cell reached through two images holds
// at most one image of each atom within R).
constexpr int kBruteMaxAtoms = 768;  // shared-memory boxes up to this size: no cell grid
// List entries a cell-searched list may spend on padding beyond its n - 1 neighbours:
// each of its two output streams closes at most four partial words of at most seven
// pad entries when its image code changes.
constexpr int kListPadSlack = 56;

// Threads per atom of a box whose list is built without cells (n <= kBruteMaxAtoms):
// an atom's neighbours are split by slot modulo that number into sub-lists, each with
// its own thread; the partial forces combine in a fixed order, so results depend on
// the box alone.  Boxes of up to 384 atoms are latency-bound with one thread per atom;
// from 385 atoms on, the extra sub-list work costs more than it gains (measured on
// 500-atom boxes packed many to a CTA).
__host__ __device__ inline int brute_tpa(int n) { return n <= 384 ? 4 : 1; }

// List entries per atom of such a box: brute_tpa sub-lists, each within the planner's
// capacity and within its share of the slots (which no sub-list can outgrow).
__host__ __device__ inline int brute_list_capacity(int n, int cap_total) {
  const int t = brute_tpa(n);
  const int chunk = (n + t - 1) / t;
  const int cv = ((cap_total < chunk ? cap_total : chunk) + 7) & ~7;
  return t * cv;
}

__host__ __device__ inline int list_cells_per_axis(double L, double R, int n) {
  if (!(L >= 2.0 * R) || n <= kBruteMaxAtoms) return 0;
  int nc = (int)(2.0 * L / R);
  return nc < 12 ? nc : 12;
}

// per-CTA global scratch of a big box (layout in mdeos_big.cuh)
__host__ __device__ inline int big_cap(int n) { return (n + 31) & ~31; }

__host__ __device__ inline size_t big_cells_bytes(int ncell) {
  return ((size_t)8 * (ncell + 1) + 15) & ~(size_t)15;
}

__host__ __device__ inline size_t big_scratch_bytes(int n, int ncell, int maxnb) {
  const size_t cap = (size_t)big_cap(n);
  return 80 * cap + big_cells_bytes(ncell) + (size_t)(maxnb / 8) * cap * 16;
}

// Force-field and integrator constants (FP32 where the pair loop uses them).
struct RunParams {
  float eps4, eps24, sig6, rc2, ucut;
  float rc;
  float dt, hdtm;  // dt and dt / (2 m)
  float mass_f;
  double mass;
  int lift_iters, rescale_every_equil, rescale_every_avg, se_blocks, ref_mode;
  int warm_lift_iters;
};

// One box as planned on the host.
struct BoxDesc {
  double rho, e, e_ref;
  double L;                 // box side actually simulated (float-representable)
  unsigned long long seed;
  unsigned long long element_id;
  int natoms, steps_equil, steps_avg;
  unsigned flags;
  int path;                 // Path
  int maxnb;                // neighbour capacity per atom (PATH_NLIST)
  int nc_cell;              // cells per axis for the list build (0: brute-force build)
  int nc_lat;               // FCC cells per axis of the lifted lattice
  float skin;
  int out_index;            // slot in the result array
  // warm-start slot (nullptr: none): x float4[warm_cap] then v float4[warm_cap];
  // its tag is the element_id whose valid final state the slot holds (0: none), so a
  // slot taken over by another element needs no clearing
  float4* warm_state;
  unsigned long long* warm_tag;
  double L_old;             // box side of the stored state; > 0: try a warm start
  int warm_cap;
  int warm_pad;
};

// A unit of the persistent kernel's work queue: up to 8 boxes of one size
// class, each run by `warps_per_box` warps of the CTA.
struct WorkItem {
  int nbox;
  int warps_per_box;
  int apt;                  // atoms per thread (1..4)
  int smem_stride;          // bytes of dynamic shared memory per box group
  int ncell_cap;            // cells reserved per group
  int nl_stride;            // uint16 entries of neighbour scratch per group
  int big;                  // 1: one box above the shared-memory limit (global-memory state)
  int box[kMaxBoxesPerItem];
};

// Work queue of the serving kernel: rings in host-mapped memory written by the
// host scheduler, a claim counter in device memory.  Ring slots are counter % cap.
struct ServeQueue {
  const BoxDesc* boxes;         // host-mapped, cap_boxes entries (out_index = ring slot)
  const WorkItem* items;        // host-mapped, cap_items entries (box[] = box ring slots)
  const unsigned* tail;         // host-mapped: items published so far (monotonic)
  const int* stop;              // host-mapped: 1 = exit at the next claim
  const int* linger;            // host-mapped: 1 = traffic is active, idle CTAs stay
  unsigned* head;               // device: items claimed so far (monotonic)
  int* slot_busy;               // device, nslots: per-SM scratch slots in use
  int* alive;                   // host-mapped, nslots: 1 while a CTA holds the slot
  int nslots;
  mdeos_result* results;        // host-mapped, cap_boxes entries
  int* ready;                   // host-mapped, cap_boxes flags
  unsigned cap_items, cap_boxes;
  long long idle_ns;            // a CTA with no work for this long exits (linger == 0)
  long long max_idle_ns;        // ... and after this long in any case
};

constexpr int kAccDoubles = 2 * kMaxSeBlocks + 24;  // block sums of P and T, running sums, box constants

// Shared-memory layout of one box group (host planner and device agree):
//   positions, forces, velocities  float4[npad] each (48 B per atom slot)
//   cell counts / starts           int[2 * ncell_cap + 2]
//   per-warp partials              int64[warps][kRedSlots]    (16-B aligned)
//   FP64 broadcast slots           double[8]
//   FP64 accumulators              double[kAccDoubles]
//   block counts                   int[kMaxSeBlocks]
//   control words                  int[16]
//   cluster partials               int64[kMaxCluster][kRedSlots]  (16-B aligned)
__host__ __device__ inline int group_red_offset(int warps, int apt, int ncell_cap) {
  int npad = warps * 32 * apt;
  int b = npad * 48 + (2 * ncell_cap + 2) * 4;
  return (b + 15) & ~15;
}

__host__ __device__ inline int group_cluster_offset(int warps, int apt, int ncell_cap) {
  int b = group_red_offset(warps, apt, ncell_cap);
  b += warps * kRedSlots * 8;
  b += 8 * 8 + kAccDoubles * 8 + kMaxSeBlocks * 4 + 16 * 4;
  return (b + 15) & ~15;
}

__host__ __device__ inline int group_smem_bytes(int warps, int apt, int ncell_cap) {
  const int b = group_cluster_offset(warps, apt, ncell_cap) + kMaxCluster * kRedSlots * 8;
  return (b + 127) & ~127;
}

}  // namespace mdeos
