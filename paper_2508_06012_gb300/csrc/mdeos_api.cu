// Host engine behind the C ABI (include/mdeos.h): request validation, the
// packing planner (size classes, warps per box, box-to-CTA packing, LPT
// ordering of the work queue), ticketed submit/poll, device-resident batches
// replayed as CUDA graphs, and the single-box parity entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "mdeos_host.h"

namespace mdeos {
cudaError_t set_batch_attributes(int max_smem);
cudaError_t launch_eos_batch(const BoxDesc* boxes, const WorkItem* items, int nitems, int* counter,
                             mdeos_result* results, uint16_t* nl, long long nl_elems_per_cta,
                             const RunParams& rp, int grid, int smem, cudaStream_t st,
                             int* ready, int cluster);
cudaError_t set_debug_attributes(int max_smem);
cudaError_t launch_debug_lift(const BoxDesc& bd, const RunParams& rp, double T, int apt,
                              int ncell_cap, int smem, float4* x4, float4* v4, double* e_out,
                              uint16_t* nl, cudaStream_t st);
cudaError_t launch_debug_forces(const BoxDesc& bd, const RunParams& rp, int apt, int ncell_cap,
                                int smem, const float4* x4, float4* f4, double* ew,
                                long long* pairs, uint16_t* nl, cudaStream_t st);
cudaError_t launch_debug_big_forces(const BoxDesc& bd, const RunParams& rp, unsigned char* scratch,
                                    const float4* x4, float4* f4, double* ew, long long* pairs,
                                    cudaStream_t st);
cudaError_t launch_debug_big_md(const BoxDesc& bd, const RunParams& rp, unsigned char* scratch,
                                float4* x4, float4* v4, int steps, double T, int every, double* ep,
                                double* ek, long long* cyc, cudaStream_t st);
cudaError_t launch_debug_md(const BoxDesc& bd, const RunParams& rp, int apt, int ncell_cap,
                            int smem, float4* x4, float4* v4, int steps, double T, int every,
                            double* ep, double* ek, long long* cyc, uint16_t* nl,
                            cudaStream_t st);
cudaError_t launch_debug_force_bench(const BoxDesc& bd, const RunParams& rp, int apt, int ncell_cap,
                                     int smem, const float4* x4, int nbox, int passes, int mode,
                                     long long* cyc, uint16_t* nl, long long nl_elems,
                                     cudaStream_t st);
}  // namespace mdeos

using namespace mdeos;

// ---------------------------------------------------------------------------
// errors

static thread_local std::string g_last_error = "";

static mdeos_status fail(mdeos_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

static mdeos_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return MDEOS_ECUDA;
}

#define CK(call)                                                 \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);          \
  } while (0)

extern "C" const char* mdeos_last_error(void) { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------
// configuration

extern "C" void mdeos_config_default(mdeos_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->device = 0;
  c->lift_iters = 2;
  c->rescale_every_equil = 0;
  c->rescale_every_avg = 10;
  c->se_blocks = 10;
  c->energy_ref_mode = MDEOS_REF_ECOLD;
  c->eps = 1.0;
  c->sigma = 1.0;
  c->mass = 1.0;
  c->rc = 2.5;
  c->dt = 0.005;
  c->skin = 0.0;
  c->hbm_budget_bytes = 0;
  c->cuda_stream = nullptr;
  c->warm_lift_iters = 1;
  c->warm_slots = 0;
  c->warm_atoms = 0;
}

static mdeos_status check_config(const mdeos_config* c) {
  if (!c) return fail(MDEOS_EINVAL, "config is NULL");
  if (!(c->eps > 0) || !(c->sigma > 0) || !(c->mass > 0) || !(c->rc > 0) || !(c->dt > 0))
    return fail(MDEOS_EINVAL, "eps, sigma, mass, rc and dt must be > 0");
  if (c->lift_iters < 0 || c->lift_iters > 64) return fail(MDEOS_EINVAL, "lift_iters out of range");
  if (c->se_blocks < 2 || c->se_blocks > kMaxSeBlocks)
    return fail(MDEOS_EINVAL, "se_blocks must be in 2..32");
  if (c->rescale_every_equil < 0 || c->rescale_every_avg < 0)
    return fail(MDEOS_EINVAL, "rescale periods must be >= 0");
  if (c->energy_ref_mode != MDEOS_REF_ECOLD && c->energy_ref_mode != MDEOS_REF_FIXED)
    return fail(MDEOS_EINVAL, "energy_ref_mode must be REF_ECOLD or REF_FIXED");
  if (c->skin > 2.0 * c->rc) return fail(MDEOS_EINVAL, "skin larger than 2 rc");
  if (c->warm_lift_iters < 1 || c->warm_lift_iters > 64)
    return fail(MDEOS_EINVAL, "warm_lift_iters out of range 1..64");
  if (c->nlist_capacity < 0) return fail(MDEOS_EINVAL, "nlist_capacity must be >= 0");
  if (c->max_cluster < 0) return fail(MDEOS_EINVAL, "max_cluster must be >= 0");
  if (c->warm_slots < 0 || c->warm_atoms < 0 || c->warm_atoms > kMaxAtoms ||
      (c->warm_slots > 0 && c->warm_atoms < 2))
    return fail(MDEOS_EINVAL, "warm_slots / warm_atoms out of range");
  return MDEOS_OK;
}

static RunParams make_run_params(const mdeos_config* c) {
  RunParams rp;
  double s6 = std::pow(c->sigma / c->rc, 6.0);
  rp.eps4 = (float)(4.0 * c->eps);
  rp.eps24 = (float)(24.0 * c->eps);
  rp.sig6 = (float)std::pow(c->sigma, 6.0);
  rp.rc2 = (float)(c->rc * c->rc);
  rp.ucut = (float)(4.0 * c->eps * (s6 * s6 - s6));
  rp.rc = (float)c->rc;
  rp.dt = (float)c->dt;
  rp.hdtm = (float)(0.5 * c->dt / c->mass);
  rp.mass_f = (float)c->mass;
  rp.mass = c->mass;
  rp.lift_iters = c->lift_iters;
  rp.rescale_every_equil = c->rescale_every_equil;
  rp.rescale_every_avg = c->rescale_every_avg;
  rp.se_blocks = c->se_blocks;
  rp.ref_mode = c->energy_ref_mode;
  rp.warm_lift_iters = c->warm_lift_iters;
  return rp;
}

// ---------------------------------------------------------------------------
// planner: one box

// Launch shape per atom count measured by mdeos_autotune: the Verlet skin (used
// when cfg.skin <= 0) and the warps that run one box (0 = the planner's default).
struct LaunchShape {
  float skin = 0.f;
  int warps = 0;
};
using ShapeTable = std::map<int, LaunchShape>;

// smallest power of two >= x (x <= 32)
static int pow2_ceil(int x) {
  int p = 1;
  while (p < x) p *= 2;
  return p;
}

struct BoxPlan {
  BoxDesc bd;
  int warps = 4, apt = 1;
  int ncell = 1;
  bool big = false;  // above the shared-memory limit: global-memory state, one CTA
  double cost = 0.0;
  int status = MDEOS_OK;
};

static int round_apt(int a) { return a <= 1 ? 1 : (a <= 2 ? 2 : 4); }

// Box side rounded to float so host (volume, pressure) and device (FP32
// minimum image) simulate the same box.
static double box_side(int n, double rho) { return (double)(float)std::cbrt((double)n / rho); }

// Verlet-list entries per atom: the configured capacity, else 1.3 x the neighbours
// within rs at the box density (at least the liquid's, rho = 0.9: dilute boxes in
// the coexistence region form droplets of liquid density) + 32; at least cap_min,
// at most every other atom; whole 8-entry list words.
static int list_capacity(const mdeos_config& c, int n, double rho, double rs, int cap_min) {
  int mx = c.nlist_capacity;
  if (mx <= 0) {
    const double expect_cap = 4.18879020478639 * rs * rs * rs * std::max(rho, 0.9);
    mx = (int)std::ceil(1.3 * expect_cap + 32.0) + kListPadSlack;  // + padding of coded lists
  }
  mx = std::max(mx, cap_min);
  mx = std::min(mx, n - 1 + kListPadSlack);
  return (std::max(mx, 1) + 7) & ~7;
}

static BoxPlan plan_box(const mdeos_request& r, const mdeos_config& c, int idx, bool allow_big,
                        const ShapeTable* tuned, int cap_min = 0, bool spread = false) {
  BoxPlan p;
  BoxDesc& b = p.bd;
  std::memset(&b, 0, sizeof(b));
  b.rho = r.rho;
  b.e = r.e;
  b.e_ref = r.e_ref;
  b.seed = r.seed;
  b.element_id = r.element_id;
  b.natoms = r.natoms;
  b.steps_equil = r.steps_equil;
  b.steps_avg = r.steps_avg;
  b.flags = r.flags;
  b.out_index = idx;
  const int n = r.natoms;
  const bool ok = n >= 2 && n <= (allow_big ? kMaxAtomsBig : kMaxAtoms) && std::isfinite(r.rho) &&
                  r.rho > 0 &&
                  std::isfinite(r.e) && std::isfinite(r.e_ref) && r.steps_avg >= c.se_blocks &&
                  r.steps_equil >= 0 && (long long)r.steps_equil + r.steps_avg < (1LL << 30) &&
                  (r.steps_equil == 0 || (c.lift_iters >= 1 && r.steps_equil >= c.lift_iters)) &&
                  (r.flags & ~(uint32_t)(MDEOS_REQ_TEMPERATURE | MDEOS_REQ_COLD)) == 0;
  if (!ok) {
    p.status = MDEOS_EINVAL;
    return p;
  }
  const double L = box_side(n, r.rho);
  b.L = L;
  int ncl = 1;
  while (4LL * ncl * ncl * ncl < n) ++ncl;
  b.nc_lat = ncl;
  if (L < c.rc) {
    p.status = MDEOS_EBOX;
    return p;
  }
  const double steps = (double)r.steps_equil + r.steps_avg;
  // path choice (autotuner defaults; a measured table can override per class)
  double skin = 0.3;
  if (c.skin > 0) {
    skin = c.skin;
  } else if (tuned) {
    const auto it = tuned->find(n);
    if (it != tuned->end() && it->second.skin > 0.f) skin = it->second.skin;
  }
  const double smax = 0.5 * L - c.rc;
  if (n > kMaxAtoms) {
    // above the shared-memory limit: Verlet list, state in global memory
    if (smax < 0.15) {
      p.status = MDEOS_EBOX;
      return p;
    }
    skin = std::min(skin, smax);
    const double rs = c.rc + skin;
    int nc = (int)std::floor(L / rs);
    while (nc > 3 && nc * nc * nc > kMaxCellsBig) --nc;
    if (nc < 3) {
      p.status = MDEOS_EBOX;
      return p;
    }
    b.path = PATH_NLIST;
    b.skin = (float)skin;
    b.nc_cell = nc;
    const double expect = 4.18879020478639 * rs * rs * rs * r.rho;
    b.maxnb = list_capacity(c, n, r.rho, rs, cap_min);
    p.big = true;
    p.ncell = nc * nc * nc;
    p.warps = 32;
    p.apt = 0;
    p.cost = steps * n * (expect * 1.15 + 8.0);
    return p;
  }
  if (L < 2.0 * c.rc) {
    b.path = PATH_ALLPAIRS_MI;
  } else if (n <= 128 || smax < 0.15) {
    b.path = PATH_ALLPAIRS;
  } else {
    b.path = PATH_NLIST;
    skin = std::min(skin, smax);
  }
  if (b.path == PATH_NLIST) {
    b.skin = (float)skin;
    const double rs = c.rc + skin;
    const int nc = list_cells_per_axis(L, rs, n);
    b.nc_cell = nc;
    p.ncell = nc > 0 ? nc * nc * nc : 1;
    const double expect = 4.18879020478639 * rs * rs * rs * r.rho;
    b.maxnb = list_capacity(c, n, r.rho, rs, cap_min);
    if (nc == 0) b.maxnb = brute_list_capacity(n, b.maxnb);
    p.cost = steps * n * (expect * 1.0 + 8.0);
  } else {
    b.skin = 0.f;
    b.nc_cell = 0;
    b.maxnb = 0;
    p.cost = steps * n * (double)n * (b.path == PATH_ALLPAIRS_MI ? 8.0 : 1.0) * 0.6;
  }
  // threads per box: at most 4 atoms per thread, at least 4 warps; a tuned shape
  // may give more warps; a batch that cannot fill the GPU (spread) runs every box
  // in its own CTA with one atom per thread (up to 32 warps)
  int warps = 4;
  while (warps < 32 && warps * 32 * 4 < n) warps *= 2;
  if (spread) {
    const int tpa = (b.path == PATH_NLIST && b.nc_cell == 0) ? brute_tpa(n) : 1;
    warps = std::max(warps, std::min(32, pow2_ceil((n * tpa + 31) / 32)));
  } else if (tuned) {
    const auto it = tuned->find(n);
    if (it != tuned->end() && it->second.warps > warps && it->second.warps <= 32)
      warps = it->second.warps;
  }
  p.warps = warps;
  p.apt = round_apt((n + warps * 32 - 1) / (warps * 32));
  return p;
}

// ---------------------------------------------------------------------------
// planner: packing

struct Plan {
  std::vector<BoxDesc> boxes;
  std::vector<WorkItem> items;
  std::vector<int> status;  // per request: MDEOS_OK or the planning error
  int smem = 0;
  long long nl_per_cta = 0;
  int grid = 0;
  int cluster = 1;  // CTAs per box (thread-block clusters, eos_cluster_kernel); 1: none
};

static mdeos_status make_plan(const mdeos_request* reqs, int n, const mdeos_config& c, int nsm,
                              int smem_max, Plan& plan, bool allow_big = true,
                              const ShapeTable* tuned = nullptr, const int* cap_min = nullptr,
                              bool allow_cluster = false) {
  plan.boxes.clear();
  plan.items.clear();
  plan.status.assign(n, MDEOS_OK);
  std::vector<BoxPlan> bp;
  bp.reserve(n);
  for (int i = 0; i < n; ++i) {
    BoxPlan p = plan_box(reqs[i], c, i, allow_big, tuned, cap_min ? cap_min[i] : 0);
    plan.status[i] = p.status;
    if (p.status == MDEOS_OK) bp.push_back(p);
  }
  // A batch with no more shared-memory boxes than SMs cannot fill the GPU with
  // packed items: give every such box its own CTA (spread), one atom per thread.
  int nsmall = 0;
  for (const BoxPlan& p : bp) nsmall += p.big ? 0 : 1;
  const bool spread = nsmall > 0 && nsmall <= nsm;
  if (spread) {
    for (BoxPlan& p : bp) {
      if (p.big) continue;
      const BoxPlan q = plan_box(reqs[p.bd.out_index], c, p.bd.out_index, allow_big, tuned,
                                 cap_min ? cap_min[p.bd.out_index] : 0, true);
      p.warps = q.warps;
      p.apt = q.apt;
    }
  }
  // Fewer boxes than half the SMs, all searched without cells: a thread-block
  // cluster of up to kMaxCluster CTAs per box (the whole CTA as its group), the
  // largest power of two that keeps every box's cluster on the GPU at once
  plan.cluster = 1;
  // default up to 4: clusters of 8 CTAs did not all fit on the GPU at once (16 boxes:
  // 338 EOS/s against 611 with 4 and 583 with none)
  const int cmax = c.max_cluster > 0 ? std::min(c.max_cluster, kMaxCluster) : 4;
  if (allow_cluster && spread && (int)bp.size() == nsmall) {
    bool all = true;
    for (const BoxPlan& p : bp) all = all && p.bd.path == PATH_NLIST && p.bd.nc_cell == 0;
    int C = 1;
    while (2 * C <= cmax && 2LL * C * nsmall <= nsm) C *= 2;
    if (all && C > 1) {
      plan.cluster = C;
      for (BoxPlan& p : bp) {
        p.warps = kCtaThreads / 32;
        p.apt = round_apt((p.bd.natoms + kCtaThreads - 1) / kCtaThreads);
      }
    }
  }
  // Only boxes above the shared-memory limit, fewer than half the SMs: each on a
  // cluster of CTAs sharing its global-memory state (a slab of slots per CTA), the
  // same cluster size rule
  const int nbig = (int)bp.size() - nsmall;
  if (allow_cluster && nsmall == 0 && nbig > 0) {
    int C = 1;
    while (2 * C <= cmax && 2LL * (2 * C) * nbig <= nsm) C *= 2;
    if (C > 1) plan.cluster = C;
  }
  // size classes by (warps, apt); inside a class, sort by cost so an item's
  // boxes finish together
  std::sort(bp.begin(), bp.end(), [](const BoxPlan& a, const BoxPlan& b) {
    if (a.warps != b.warps) return a.warps < b.warps;
    if (a.apt != b.apt) return a.apt < b.apt;
    return a.cost > b.cost;
  });
  struct ItemCost {
    WorkItem wi;
    double cost;
  };
  std::vector<ItemCost> items;
  plan.smem = 0;
  plan.nl_per_cta = 0;
  size_t k = 0;
  while (k < bp.size()) {
    if (bp[k].big) {  // one box per item, scratch in global memory
      WorkItem wi;
      std::memset(&wi, 0, sizeof(wi));
      wi.nbox = 1;
      wi.warps_per_box = 32;
      wi.apt = 0;
      wi.big = 1;
      wi.ncell_cap = bp[k].ncell;
      wi.smem_stride = kBigSharedBytes;
      const size_t bytes = big_scratch_bytes(bp[k].bd.natoms, bp[k].ncell, bp[k].bd.maxnb);
      wi.nl_stride = (int)(((bytes + 15) & ~(size_t)15) / 2);
      wi.box[0] = (int)plan.boxes.size();
      plan.boxes.push_back(bp[k].bd);
      // room for position windows behind the CTA's BigShared: the whole box when it
      // fits, else all the shared memory there is
      const int cache = kBigSharedBytes + 16 * big_cap(bp[k].bd.natoms);
      plan.smem = std::max(plan.smem, std::min(cache, smem_max));
      plan.nl_per_cta = std::max(plan.nl_per_cta, (long long)wi.nl_stride);
      items.push_back({wi, bp[k].cost});
      ++k;
      continue;
    }
    const int warps = bp[k].warps, apt = bp[k].apt;
    const int npad = warps * 32 * apt;
    const int per_cta = spread ? 1 : std::min(kCtaThreads / (warps * 32), kMaxBoxesPerItem);
    // boxes of this class that share one item
    WorkItem wi;
    std::memset(&wi, 0, sizeof(wi));
    wi.warps_per_box = warps;
    wi.apt = apt;
    int ncell_cap = 1, maxnb = 8;
    double cost = 0.0;
    int nb = 0;
    while (k < bp.size() && bp[k].warps == warps && bp[k].apt == apt && nb < per_cta) {
      const int nc2 = std::max(ncell_cap, bp[k].ncell);
      const int stride = group_smem_bytes(warps, apt, nc2);
      if ((nb + 1) * stride > smem_max) break;
      ncell_cap = nc2;
      maxnb = std::max(maxnb, bp[k].bd.maxnb);
      wi.box[nb++] = (int)plan.boxes.size();
      plan.boxes.push_back(bp[k].bd);
      cost += bp[k].cost;
      ++k;
    }
    if (nb == 0) return fail(MDEOS_EINVAL, "a box does not fit in shared memory");
    wi.nbox = nb;
    wi.ncell_cap = ncell_cap;
    wi.smem_stride = group_smem_bytes(warps, apt, ncell_cap);
    wi.nl_stride = ((maxnb + 7) & ~7) * npad;
    plan.smem = std::max(plan.smem, nb * wi.smem_stride);
    plan.nl_per_cta = std::max(plan.nl_per_cta, (long long)nb * wi.nl_stride);
    items.push_back({wi, cost});
  }
  // longest-processing-time first
  std::stable_sort(items.begin(), items.end(),
                   [](const ItemCost& a, const ItemCost& b) { return a.cost > b.cost; });
  for (auto& it : items) plan.items.push_back(it.wi);
  plan.grid = plan.cluster > 1 ? (int)plan.items.size() * plan.cluster
                               : std::max(1, std::min(nsm, (int)plan.items.size()));
  return MDEOS_OK;
}

namespace mdeos {
mdeos_status set_error(mdeos_status st, const std::string& msg) { return fail(st, msg); }

// Planning for the no-allocation entry point (mdeos_noalloc.cu): validation,
// packing and the host copy of the initial results, all in host memory.
mdeos_status plan_for_noalloc(const mdeos_request* reqs, int n, const mdeos_config& c, int nsm,
                              int smem_max, std::vector<BoxDesc>& boxes,
                              std::vector<WorkItem>& items, std::vector<mdeos_result>& init,
                              int& grid, int& smem, long long& nl_per_cta, RunParams& rp);
}  // namespace mdeos

static void planning_result(mdeos_result& r, int status, const mdeos_request& q);

mdeos_status mdeos::plan_for_noalloc(const mdeos_request* reqs, int n, const mdeos_config& c,
                                     int nsm, int smem_max, std::vector<BoxDesc>& boxes,
                                     std::vector<WorkItem>& items,
                                     std::vector<mdeos_result>& init, int& grid, int& smem,
                                     long long& nl_per_cta, RunParams& rp) {
  mdeos_status st = check_config(&c);
  if (st != MDEOS_OK) return st;
  Plan plan;
  st = make_plan(reqs, n, c, nsm, smem_max, plan, /*allow_big=*/false);
  if (st != MDEOS_OK) return st;
  boxes = plan.boxes;
  items = plan.items;
  init.resize(n);
  for (int i = 0; i < n; ++i) planning_result(init[i], plan.status[i], reqs[i]);
  grid = plan.grid;
  smem = plan.smem;
  nl_per_cta = plan.nl_per_cta;
  rp = make_run_params(&c);
  return MDEOS_OK;
}

// ---------------------------------------------------------------------------
// handle

struct PinnedBlock {
  void* p = nullptr;
  size_t size = 0;
};

struct PinnedBlockPtr {
  void* p = nullptr;
  size_t size = 0;
};

struct TicketState {
  int n = 0;
  cudaEvent_t done = nullptr;
  void* d_mem = nullptr;      // boxes | items | results | counter
  PinnedBlock h_in, h_out;
  std::vector<int> status;    // planning status per request
  std::vector<uint64_t> element_id;
  std::vector<int> natoms;
  std::vector<mdeos_request> reqs;  // kept to re-plan boxes whose list overflowed
  std::vector<BoxDesc> planned;     // the box each request was planned as (by index)
  bool any_device = false;
  size_t bytes = 0;
};

struct WarmSlot {
  int slot = 0;
  int natoms = 0;   // atoms of the state last planned into the slot
  double L = 0.0;   // its box side
};

struct mdeos_handle {
  mdeos_config cfg;
  ShapeTable tuned_skin;  // launch shapes from mdeos_autotune
  // warm-start store: slot k holds x float4[warm_atoms] then v float4[warm_atoms]
  float4* d_warm = nullptr;
  unsigned long long* d_warm_tag = nullptr;  // element_id of each slot's valid state
  size_t warm_bytes = 0;
  std::unordered_map<uint64_t, WarmSlot> warm_map;
  int warm_next = 0;
  // reusable device work table of eval_into_device
  void* d_eval = nullptr;
  size_t eval_bytes = 0;
  PinnedBlockPtr eval_pinned;
  RunParams rp;
  int device = 0, nsm = 0, smem_max = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint16_t* d_nl = nullptr;
  size_t nl_bytes = 0;
  size_t used_bytes = 0;
  uint64_t next_ticket = 1;
  std::unordered_map<uint64_t, TicketState> tickets;
  std::vector<PinnedBlock> pinned_free;
  std::mutex mu;
  // statistics of the last submit
  size_t last_h2d = 0, last_d2h = 0;
  long long launches = 0;
};

struct mdeos_batch {
  mdeos_handle* h = nullptr;
  int n = 0;
  Plan plan;
  void* d_mem = nullptr;
  BoxDesc* d_boxes = nullptr;
  WorkItem* d_items = nullptr;
  mdeos_result* d_results = nullptr;
  int* d_counter = nullptr;
  uint16_t* d_nl = nullptr;
  size_t bytes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<mdeos_result> init_results;
};

static mdeos_status pinned_get(mdeos_handle* h, size_t size, PinnedBlock& out) {
  for (size_t i = 0; i < h->pinned_free.size(); ++i) {
    if (h->pinned_free[i].size >= size) {
      out = h->pinned_free[i];
      h->pinned_free.erase(h->pinned_free.begin() + i);
      return MDEOS_OK;
    }
  }
  size_t sz = std::max<size_t>(size, 4096);
  CK(cudaMallocHost(&out.p, sz));
  out.size = sz;
  return MDEOS_OK;
}

static void pinned_put(mdeos_handle* h, PinnedBlock& b) {
  if (b.p) h->pinned_free.push_back(b);
  b.p = nullptr;
  b.size = 0;
}

static mdeos_status ensure_scratch(mdeos_handle* h, size_t bytes) {
  if (bytes <= h->nl_bytes) return MDEOS_OK;
  const size_t extra = bytes - h->nl_bytes;
  if (h->cfg.hbm_budget_bytes && h->used_bytes + extra > h->cfg.hbm_budget_bytes)
    return fail(MDEOS_ENOMEM, "neighbour-list scratch exceeds the HBM budget");
  if (h->d_nl) {
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaFree(h->d_nl));
    h->used_bytes -= h->nl_bytes;
    h->d_nl = nullptr;
    h->nl_bytes = 0;
  }
  CK(cudaMalloc(&h->d_nl, bytes));
  h->nl_bytes = bytes;
  h->used_bytes += bytes;
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_create(const mdeos_config* cfg, mdeos_handle** out) {
  if (!out) return fail(MDEOS_EINVAL, "out is NULL");
  *out = nullptr;
  mdeos_status st = check_config(cfg);
  if (st != MDEOS_OK) return st;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) return fail(MDEOS_ECUDA, "no CUDA device available");
  if (cfg->device < 0 || cfg->device >= ndev) return fail(MDEOS_EINVAL, "device out of range");
  mdeos_handle* h = new mdeos_handle();
  h->cfg = *cfg;
  h->rp = make_run_params(cfg);
  h->device = cfg->device;
  e = cudaSetDevice(h->device);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "cudaSetDevice");
  }
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, h->device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, h->device);
  cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device);
  cudaDeviceGetAttribute(&h->smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  h->smem_max -= 2048;  // static shared memory of the kernels (the serving kernel's is ~1.3 KB)
  e = set_batch_attributes(h->smem_max);
  if (e == cudaSuccess) e = set_debug_attributes(h->smem_max);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "kernel attributes (is this an sm_103 GPU?)");
  }
  if (cfg->warm_slots > 0) {
    const size_t slot_bytes = (size_t)2 * cfg->warm_atoms * sizeof(float4);
    h->warm_bytes = (size_t)cfg->warm_slots * (slot_bytes + sizeof(unsigned long long));
    if (cfg->hbm_budget_bytes && h->warm_bytes > cfg->hbm_budget_bytes) {
      delete h;
      return fail(MDEOS_ENOMEM, "warm-start store exceeds the HBM budget");
    }
    e = cudaMalloc(&h->d_warm, (size_t)cfg->warm_slots * slot_bytes);
    if (e == cudaSuccess)
      e = cudaMalloc(&h->d_warm_tag, (size_t)cfg->warm_slots * sizeof(unsigned long long));
    if (e == cudaSuccess)
      e = cudaMemset(h->d_warm_tag, 0, (size_t)cfg->warm_slots * sizeof(unsigned long long));
    if (e != cudaSuccess) {
      if (h->d_warm) cudaFree(h->d_warm);
      if (h->d_warm_tag) cudaFree(h->d_warm_tag);
      delete h;
      return cuda_fail(e, "warm-start store allocation");
    }
    h->used_bytes += h->warm_bytes;
  }
  if (cfg->cuda_stream) {
    h->stream = (cudaStream_t)cfg->cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete h;
      return cuda_fail(e, "cudaStreamCreate");
    }
    h->own_stream = true;
  }
  *out = h;
  return MDEOS_OK;
}

static void release_ticket(mdeos_handle* h, TicketState& t) {
  if (t.done) cudaEventDestroy(t.done);
  if (t.d_mem) cudaFreeAsync(t.d_mem, h->stream);
  h->used_bytes -= t.bytes;
  pinned_put(h, t.h_in);
  pinned_put(h, t.h_out);
}

extern "C" mdeos_status mdeos_destroy(mdeos_handle* h) {
  if (!h) return MDEOS_OK;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  for (auto& kv : h->tickets) release_ticket(h, kv.second);
  h->tickets.clear();
  cudaStreamSynchronize(h->stream);
  for (auto& b : h->pinned_free) cudaFreeHost(b.p);
  if (h->d_nl) cudaFree(h->d_nl);
  if (h->d_warm) cudaFree(h->d_warm);
  if (h->d_warm_tag) cudaFree(h->d_warm_tag);
  if (h->d_eval) cudaFree(h->d_eval);
  if (h->eval_pinned.p) cudaFreeHost(h->eval_pinned.p);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
  return MDEOS_OK;
}

// fill results of requests rejected by the planner
static void planning_result(mdeos_result& r, int status, const mdeos_request& q) {
  std::memset(&r, 0, sizeof(r));
  r.status = status;
  r.natoms = q.natoms;
  r.element_id = q.element_id;
  r.path = -1;
}

// Attach warm-start slots to the planned boxes (slot rules in mdeos.h).
static void assign_warm(mdeos_handle* h, Plan& plan, const mdeos_request* reqs) {
  if (!h->d_warm) return;
  const int cap = h->cfg.warm_atoms;
  std::unordered_set<uint64_t> seen;
  for (BoxDesc& bd : plan.boxes) {
    const mdeos_request& r = reqs[bd.out_index];
    if (r.element_id == 0 || r.natoms > cap) continue;
    if (!seen.insert(r.element_id).second) continue;  // repeated element: cold, not stored
    auto it = h->warm_map.find(r.element_id);
    if (it == h->warm_map.end()) {
      if (h->warm_next >= h->cfg.warm_slots) continue;  // store full: cold, not stored
      WarmSlot ws;
      ws.slot = h->warm_next++;
      it = h->warm_map.emplace(r.element_id, ws).first;
    }
    WarmSlot& ws = it->second;
    const bool try_warm = ws.natoms == r.natoms && ws.L > 0.0 &&
                          (r.flags & MDEOS_REQ_COLD) == 0 &&
                          (r.steps_equil == 0 || r.steps_equil >= h->cfg.warm_lift_iters);
    bd.warm_state = h->d_warm + (size_t)ws.slot * 2 * cap;
    bd.warm_tag = h->d_warm_tag + ws.slot;
    bd.warm_cap = cap;
    bd.L_old = try_warm ? ws.L : 0.0;
    ws.natoms = r.natoms;
    ws.L = bd.L;
  }
}

extern "C" mdeos_status mdeos_submit(mdeos_handle* h, const mdeos_request* reqs, int32_t n,
                                     uint64_t* ticket) {
  if (!h || !reqs || !ticket || n < 1) return fail(MDEOS_EINVAL, "bad submit arguments");
  std::lock_guard<std::mutex> lock(h->mu);
  CK(cudaSetDevice(h->device));
  Plan plan;
  mdeos_status st =
      make_plan(reqs, n, h->cfg, h->nsm, h->smem_max, plan, true, &h->tuned_skin, nullptr, true);
  if (st != MDEOS_OK) return st;
  assign_warm(h, plan, reqs);
  TicketState t;
  t.n = n;
  t.status = plan.status;
  t.element_id.resize(n);
  t.natoms.resize(n);
  for (int i = 0; i < n; ++i) {
    t.element_id[i] = reqs[i].element_id;
    t.natoms[i] = reqs[i].natoms;
  }
  t.reqs.assign(reqs, reqs + n);
  t.planned.resize(n);
  for (const BoxDesc& bd : plan.boxes) t.planned[bd.out_index] = bd;
  const size_t nb = plan.boxes.size(), ni = plan.items.size();
  const size_t off_items = (nb * sizeof(BoxDesc) + 255) & ~size_t(255);
  const size_t in_bytes = off_items + ni * sizeof(WorkItem);
  const size_t off_res = (in_bytes + 255) & ~size_t(255);
  const size_t off_cnt = off_res + (((size_t)n * sizeof(mdeos_result) + 255) & ~size_t(255));
  const size_t dev_bytes = off_cnt + 256;
  if (h->cfg.hbm_budget_bytes && h->used_bytes + dev_bytes > h->cfg.hbm_budget_bytes)
    return fail(MDEOS_ENOMEM, "batch exceeds the HBM budget");
  if ((st = pinned_get(h, in_bytes, t.h_in)) != MDEOS_OK) return st;
  if ((st = pinned_get(h, (size_t)n * sizeof(mdeos_result), t.h_out)) != MDEOS_OK) {
    pinned_put(h, t.h_in);
    return st;
  }
  std::memcpy(t.h_in.p, plan.boxes.data(), nb * sizeof(BoxDesc));
  std::memcpy((char*)t.h_in.p + off_items, plan.items.data(), ni * sizeof(WorkItem));
  t.any_device = nb > 0;
  h->last_h2d = 0;
  h->last_d2h = 0;
  if (t.any_device) {
    const size_t scratch = (size_t)plan.grid * plan.nl_per_cta * sizeof(uint16_t);
    if ((st = ensure_scratch(h, scratch)) != MDEOS_OK) {
      pinned_put(h, t.h_in);
      pinned_put(h, t.h_out);
      return st;
    }
    cudaError_t e = cudaMallocAsync(&t.d_mem, dev_bytes, h->stream);
    if (e != cudaSuccess) {
      pinned_put(h, t.h_in);
      pinned_put(h, t.h_out);
      return cuda_fail(e, "cudaMallocAsync");
    }
    t.bytes = dev_bytes;
    h->used_bytes += dev_bytes;
    char* d = (char*)t.d_mem;
    CK(cudaMemcpyAsync(d, t.h_in.p, in_bytes, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemsetAsync(d + off_cnt, 0, sizeof(int), h->stream));
    e = launch_eos_batch((BoxDesc*)d, (WorkItem*)(d + off_items), (int)ni, (int*)(d + off_cnt),
                         (mdeos_result*)(d + off_res), h->d_nl, plan.nl_per_cta, h->rp, plan.grid,
                         plan.smem, h->stream, nullptr, plan.cluster);
    if (e != cudaSuccess) return cuda_fail(e, "eos_batch_kernel launch");
    h->launches += 1;
    CK(cudaMemcpyAsync(t.h_out.p, d + off_res, (size_t)n * sizeof(mdeos_result),
                       cudaMemcpyDeviceToHost, h->stream));
    h->last_h2d = in_bytes;
    h->last_d2h = (size_t)n * sizeof(mdeos_result);
  }
  CK(cudaEventCreateWithFlags(&t.done, cudaEventDisableTiming));
  CK(cudaEventRecord(t.done, h->stream));
  const uint64_t id = h->next_ticket++;
  h->tickets.emplace(id, std::move(t));
  *ticket = id;
  return MDEOS_OK;
}

// Run one plan to completion on the handle's stream (boxes, items, results and
// queue counter in a temporary device block) and copy its results to host `out`.
static mdeos_status run_plan_sync(mdeos_handle* h, const Plan& plan, int n, mdeos_result* out) {
  const size_t nb = plan.boxes.size(), ni = plan.items.size();
  const size_t off_items = (nb * sizeof(BoxDesc) + 255) & ~size_t(255);
  const size_t off_res = (off_items + ni * sizeof(WorkItem) + 255) & ~size_t(255);
  const size_t off_cnt = off_res + (((size_t)n * sizeof(mdeos_result) + 255) & ~size_t(255));
  const size_t dev_bytes = off_cnt + 256;
  if (h->cfg.hbm_budget_bytes && h->used_bytes + dev_bytes > h->cfg.hbm_budget_bytes)
    return fail(MDEOS_ENOMEM, "re-run exceeds the HBM budget");
  mdeos_status st = ensure_scratch(h, (size_t)plan.grid * plan.nl_per_cta * sizeof(uint16_t));
  if (st != MDEOS_OK) return st;
  std::vector<char> in(off_items + ni * sizeof(WorkItem));
  std::memcpy(in.data(), plan.boxes.data(), nb * sizeof(BoxDesc));
  std::memcpy(in.data() + off_items, plan.items.data(), ni * sizeof(WorkItem));
  char* d = nullptr;
  CK(cudaMallocAsync((void**)&d, dev_bytes, h->stream));
  cudaError_t e = cudaMemcpyAsync(d, in.data(), in.size(), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d + off_cnt, 0, sizeof(int), h->stream);
  if (e == cudaSuccess)
    e = launch_eos_batch((BoxDesc*)d, (WorkItem*)(d + off_items), (int)ni, (int*)(d + off_cnt),
                         (mdeos_result*)(d + off_res), h->d_nl, plan.nl_per_cta, h->rp, plan.grid,
                         plan.smem, h->stream, nullptr, plan.cluster);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, d + off_res, (size_t)n * sizeof(mdeos_result),
                        cudaMemcpyDeviceToHost, h->stream);
  cudaFreeAsync(d, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "neighbour-list re-run");
  h->launches += 1;
  return MDEOS_OK;
}

// Boxes whose Verlet list overflowed (MDEOS_ENBR) are planned again with twice the
// list capacity (up to every other atom) and re-run, keeping the warm-start slot
// and box side of their first plan, until they succeed or the capacity is full.
// The list's content and order do not depend on its capacity, so a re-run gives
// the result a large enough list would have given at once.
static void rerun_overflowed(mdeos_handle* h, TicketState& t, mdeos_result* res) {
  std::vector<int> cap(t.n, 0);
  for (int i = 0; i < t.n; ++i) cap[i] = t.planned[i].maxnb;
  for (int round = 1; round <= 16; ++round) {
    std::vector<int> idx;
    for (int i = 0; i < t.n; ++i)
      if (t.status[i] == MDEOS_OK && res[i].status == MDEOS_ENBR && cap[i] < t.natoms[i] - 1)
        idx.push_back(i);
    if (idx.empty()) return;
    const int m = (int)idx.size();
    std::vector<mdeos_request> sub(m);
    std::vector<int> cmin(m);
    for (int k = 0; k < m; ++k) {
      sub[k] = t.reqs[idx[k]];
      cmin[k] = 2 * cap[idx[k]];
    }
    Plan plan;
    if (make_plan(sub.data(), m, h->cfg, h->nsm, h->smem_max, plan, true, &h->tuned_skin,
                  cmin.data(), true) != MDEOS_OK)
      return;
    for (BoxDesc& bd : plan.boxes) {  // same warm slot and stored box side as the first plan
      const BoxDesc& first = t.planned[idx[bd.out_index]];
      bd.warm_state = first.warm_state;
      bd.warm_tag = first.warm_tag;
      bd.warm_cap = first.warm_cap;
      bd.L_old = first.L_old;
    }
    std::vector<mdeos_result> out(m);
    if (run_plan_sync(h, plan, m, out.data()) != MDEOS_OK) return;
    for (const BoxDesc& bd : plan.boxes) {
      const int i = idx[bd.out_index];
      cap[i] = bd.maxnb;
      res[i] = out[bd.out_index];
      res[i].nlist_retries = round;
    }
  }
}

extern "C" mdeos_status mdeos_poll(mdeos_handle* h, uint64_t ticket, mdeos_result* out,
                                   int32_t timeout_us) {
  if (!h || !out) return fail(MDEOS_EINVAL, "bad poll arguments");
  std::unique_lock<std::mutex> lock(h->mu);
  auto it = h->tickets.find(ticket);
  if (it == h->tickets.end()) return fail(MDEOS_EINVAL, "unknown ticket");
  cudaEvent_t ev = it->second.done;
  lock.unlock();
  cudaSetDevice(h->device);
  cudaError_t e;
  if (timeout_us < 0) {
    e = cudaEventSynchronize(ev);
  } else {
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
      e = cudaEventQuery(ev);
      if (e != cudaErrorNotReady) break;
      auto el = std::chrono::duration_cast<std::chrono::microseconds>(
                    std::chrono::steady_clock::now() - t0)
                    .count();
      if (el >= timeout_us) return MDEOS_PENDING;
      std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
  }
  lock.lock();
  it = h->tickets.find(ticket);
  if (it == h->tickets.end()) return fail(MDEOS_EINVAL, "ticket released concurrently");
  TicketState& t = it->second;
  mdeos_status ret = MDEOS_OK;
  if (e != cudaSuccess) {
    ret = cuda_fail(e, "batch execution");
  } else {
    mdeos_result* dev = (mdeos_result*)t.h_out.p;
    rerun_overflowed(h, t, dev);
    for (int i = 0; i < t.n; ++i) {
      if (t.status[i] == MDEOS_OK) {
        out[i] = dev[i];
      } else {
        mdeos_request q;
        std::memset(&q, 0, sizeof(q));
        q.natoms = t.natoms[i];
        q.element_id = t.element_id[i];
        planning_result(out[i], t.status[i], q);
      }
    }
  }
  release_ticket(h, t);
  h->tickets.erase(it);
  return ret;
}

// ---------------------------------------------------------------------------
// device-resident batches

extern "C" mdeos_status mdeos_batch_create(mdeos_handle* h, const mdeos_request* reqs, int32_t n,
                                           mdeos_batch** out) {
  if (!h || !reqs || !out || n < 1) return fail(MDEOS_EINVAL, "bad batch arguments");
  *out = nullptr;
  std::lock_guard<std::mutex> lock(h->mu);
  CK(cudaSetDevice(h->device));
  mdeos_batch* b = new mdeos_batch();
  b->h = h;
  b->n = n;
  mdeos_status st = make_plan(reqs, n, h->cfg, h->nsm, h->smem_max, b->plan, true,
                              &h->tuned_skin, nullptr, true);
  if (st != MDEOS_OK) {
    delete b;
    return st;
  }
  const Plan& p = b->plan;
  const size_t nb = p.boxes.size(), ni = p.items.size();
  const size_t off_items = (nb * sizeof(BoxDesc) + 255) & ~size_t(255);
  const size_t off_res = (off_items + ni * sizeof(WorkItem) + 255) & ~size_t(255);
  const size_t off_cnt = off_res + (((size_t)n * sizeof(mdeos_result) + 255) & ~size_t(255));
  const size_t off_nl = off_cnt + 256;
  const size_t nl_bytes = (size_t)p.grid * p.nl_per_cta * sizeof(uint16_t);
  const size_t total = off_nl + nl_bytes;
  if (h->cfg.hbm_budget_bytes && h->used_bytes + total > h->cfg.hbm_budget_bytes) {
    delete b;
    return fail(MDEOS_ENOMEM, "batch exceeds the HBM budget");
  }
  cudaError_t e = cudaMalloc(&b->d_mem, total);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "cudaMalloc batch");
  }
  b->bytes = total;
  h->used_bytes += total;
  char* d = (char*)b->d_mem;
  b->d_boxes = (BoxDesc*)d;
  b->d_items = (WorkItem*)(d + off_items);
  b->d_results = (mdeos_result*)(d + off_res);
  b->d_counter = (int*)(d + off_cnt);
  b->d_nl = (uint16_t*)(d + off_nl);
  b->init_results.resize(n);
  for (int i = 0; i < n; ++i) planning_result(b->init_results[i], p.status[i], reqs[i]);
  CK(cudaMemcpy(b->d_boxes, p.boxes.data(), nb * sizeof(BoxDesc), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(b->d_items, p.items.data(), ni * sizeof(WorkItem), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(b->d_results, b->init_results.data(), (size_t)n * sizeof(mdeos_result),
                cudaMemcpyHostToDevice));
  // capture: reset the queue counter, run the persistent kernel
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaMemsetAsync(b->d_counter, 0, sizeof(int), cs);
  if (ni > 0)
    launch_eos_batch(b->d_boxes, b->d_items, (int)ni, b->d_counter, b->d_results, b->d_nl,
                     p.nl_per_cta, h->rp, p.grid, p.smem, cs, nullptr, p.cluster);
  e = cudaStreamEndCapture(cs, &b->graph);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    mdeos_batch_destroy(b);
    return cuda_fail(e, "graph capture");
  }
  e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) {
    mdeos_batch_destroy(b);
    return cuda_fail(e, "graph instantiate");
  }
  *out = b;
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_batch_launch(mdeos_batch* b, void* stream) {
  if (!b) return fail(MDEOS_EINVAL, "batch is NULL");
  cudaStream_t s = stream ? (cudaStream_t)stream : b->h->stream;
  CK(cudaSetDevice(b->h->device));
  CK(cudaGraphLaunch(b->exec, s));
  b->h->launches += b->plan.items.empty() ? 0 : 1;
  return MDEOS_OK;
}

extern "C" mdeos_result* mdeos_batch_device_results(mdeos_batch* b) {
  return b ? b->d_results : nullptr;
}

extern "C" mdeos_status mdeos_batch_results(mdeos_batch* b, mdeos_result* out) {
  if (!b || !out) return fail(MDEOS_EINVAL, "bad batch_results arguments");
  CK(cudaSetDevice(b->h->device));
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(out, b->d_results, (size_t)b->n * sizeof(mdeos_result), cudaMemcpyDeviceToHost));
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_batch_info(const mdeos_batch* b, int32_t* n_items, int32_t* n_ctas,
                                         int32_t* smem_bytes, size_t* scratch_bytes) {
  if (!b) return fail(MDEOS_EINVAL, "batch is NULL");
  if (n_items) *n_items = (int32_t)b->plan.items.size();
  if (n_ctas) *n_ctas = b->plan.grid;
  if (smem_bytes) *smem_bytes = b->plan.smem;
  if (scratch_bytes) *scratch_bytes = (size_t)b->plan.grid * b->plan.nl_per_cta * sizeof(uint16_t);
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_batch_destroy(mdeos_batch* b) {
  if (!b) return MDEOS_OK;
  cudaSetDevice(b->h->device);
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->d_mem) cudaFree(b->d_mem);
  b->h->used_bytes -= b->bytes;
  delete b;
  return MDEOS_OK;
}

// ---------------------------------------------------------------------------
// autotuner: Verlet skin per atom count

// Upload a plan and run it on the handle's stream, returning the kernel time
// (CUDA events on that stream) and the box statuses (host).
static mdeos_status time_plan(mdeos_handle* h, const Plan& plan, int n, float* ms,
                              std::vector<int>& status) {
  const size_t nb = plan.boxes.size(), ni = plan.items.size();
  const size_t off_items = (nb * sizeof(BoxDesc) + 255) & ~size_t(255);
  const size_t in_bytes = off_items + ni * sizeof(WorkItem);
  const size_t off_cnt = (in_bytes + 255) & ~size_t(255);
  const size_t off_res = off_cnt + 256;
  const size_t bytes = off_res + (size_t)n * sizeof(mdeos_result);
  std::vector<char> host(in_bytes);
  std::memcpy(host.data(), plan.boxes.data(), nb * sizeof(BoxDesc));
  std::memcpy(host.data() + off_items, plan.items.data(), ni * sizeof(WorkItem));
  mdeos_status st = ensure_scratch(h, (size_t)plan.grid * plan.nl_per_cta * sizeof(uint16_t));
  if (st != MDEOS_OK) return st;
  char* d = nullptr;
  CK(cudaMalloc(&d, bytes));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d, host.data(), in_bytes, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d + off_cnt, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
  if (e == cudaSuccess)
    e = launch_eos_batch((BoxDesc*)d, (WorkItem*)(d + off_items), (int)ni, (int*)(d + off_cnt),
                         (mdeos_result*)(d + off_res), h->d_nl, plan.nl_per_cta, h->rp, plan.grid,
                         plan.smem, h->stream, nullptr, plan.cluster);
  if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
  std::vector<mdeos_result> res(n);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(res.data(), d + off_res, (size_t)n * sizeof(mdeos_result),
                        cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "autotune trial");
  h->launches += 1;
  status.resize(n);
  for (int i = 0; i < n; ++i) status[i] = plan.status[i] != MDEOS_OK ? plan.status[i] : res[i].status;
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_autotune(mdeos_handle* h, const mdeos_request* reqs, int32_t n,
                                       int32_t steps, double* table, int32_t max_out,
                                       int32_t* n_out) {
  if (!h || !reqs || n < 1 || steps < 2 * 10 || max_out < 0)
    return fail(MDEOS_EINVAL, "bad autotune arguments");
  std::lock_guard<std::mutex> lock(h->mu);
  CK(cudaSetDevice(h->device));
  CK(cudaStreamSynchronize(h->stream));
  // size classes: Verlet-path boxes grouped by atom count
  std::map<int, std::vector<int>> cls;
  std::map<int, int> warps0;
  for (int i = 0; i < n; ++i) {
    const BoxPlan p = plan_box(reqs[i], h->cfg, i, true, nullptr);
    if (p.status != MDEOS_OK || p.bd.path != PATH_NLIST) continue;
    cls[reqs[i].natoms].push_back(i);
    warps0[reqs[i].natoms] = p.big ? 0 : p.warps;
  }
  // the planner's own skin: the configured one, else 0.3
  const float skin0 = h->cfg.skin > 0 ? (float)h->cfg.skin : 0.3f;
  std::vector<float> cand = {0.2f, 0.25f, 0.3f, 0.35f, 0.4f, 0.5f};
  if (std::find(cand.begin(), cand.end(), skin0) == cand.end()) cand.push_back(skin0);
  // a shape replaces the planner's own (the configured skin, its warps per box) only
  // when it is faster by this margin: one wave's timing varies by about a percent
  const float kMargin = 0.98f;
  int k_out = 0;
  for (const auto& kv : cls) {
    // warps per box: the planner's choice and up to two doublings (at most 32)
    std::vector<int> wopt;
    for (int w = warps0[kv.first]; w > 0 && w <= 32 && wopt.size() < 3; w *= 2) wopt.push_back(w);
    if (wopt.empty()) wopt.push_back(0);  // global-memory boxes: one CTA each
    float best = 0.f, base = 0.f;
    LaunchShape best_shape;
    for (int w : wopt) {
      // one full wave of the GPU: nSM CTAs, each with as many boxes as an item holds
      const int per_cta = w == 0 ? 1 : std::min(kCtaThreads / (w * 32), kMaxBoxesPerItem);
      const int count = h->nsm * per_cta;  // spread at one box per CTA changes no shape
      std::vector<mdeos_request> trial(count);
      for (int i = 0; i < count; ++i) {
        trial[i] = reqs[kv.second[i % kv.second.size()]];
        trial[i].steps_equil = steps / 2;
        trial[i].steps_avg = steps - steps / 2;
        trial[i].element_id = 0;
        trial[i].seed += (uint64_t)i;
      }
      for (float sk : cand) {
        mdeos_config c = h->cfg;
        c.skin = sk;
        ShapeTable one;
        one[kv.first].warps = w;
        Plan plan;
        if (make_plan(trial.data(), count, c, h->nsm, h->smem_max, plan, true, &one) != MDEOS_OK)
          continue;
        float ms = 0.f;
        std::vector<int> status;
        const mdeos_status st = time_plan(h, plan, count, &ms, status);
        if (st != MDEOS_OK) return st;
        bool ok = true;
        for (int v : status) ok = ok && v == MDEOS_OK;
        const float per_box = ms / count;
        if (ok && w == wopt[0] && sk == skin0) base = per_box;
        if (ok && (best_shape.skin == 0.f || per_box < best)) {
          best = per_box;
          best_shape.skin = sk;
          best_shape.warps = w;
        }
      }
    }
    if (base > 0.f && best > kMargin * base) {  // no shape clearly faster: the planner's
      best = base;
      best_shape.skin = skin0;
      best_shape.warps = wopt[0];
    }
    if (best_shape.skin > 0.f) {
      h->tuned_skin[kv.first] = best_shape;
      if (table && k_out < max_out) {
        table[4 * k_out] = kv.first;
        table[4 * k_out + 1] = best_shape.skin;
        table[4 * k_out + 2] = best_shape.warps;
        table[4 * k_out + 3] = best;  // ms of GPU time per box (one wave)
        ++k_out;
      }
    }
  }
  if (n_out) *n_out = k_out;
  return MDEOS_OK;
}

// ---------------------------------------------------------------------------
// warm-start store

extern "C" mdeos_status mdeos_warm_export(mdeos_handle* h, uint64_t element_id, int32_t natoms,
                                          float* x4, float* v4, double* L) {
  if (!h || !x4 || !v4 || !L || natoms < 2) return fail(MDEOS_EINVAL, "bad warm_export arguments");
  std::lock_guard<std::mutex> lock(h->mu);
  auto it = h->warm_map.find(element_id);
  if (!h->d_warm || it == h->warm_map.end() || it->second.natoms != natoms)
    return fail(MDEOS_EINVAL, "no stored state of this element and size");
  CK(cudaSetDevice(h->device));
  CK(cudaStreamSynchronize(h->stream));
  const WarmSlot& ws = it->second;
  unsigned long long tag = 0;
  CK(cudaMemcpy(&tag, h->d_warm_tag + ws.slot, sizeof(tag), cudaMemcpyDeviceToHost));
  if (tag != element_id) return fail(MDEOS_EINVAL, "the element's last evaluation failed");
  const float4* base = h->d_warm + (size_t)ws.slot * 2 * h->cfg.warm_atoms;
  CK(cudaMemcpy(x4, base, (size_t)natoms * sizeof(float4), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(v4, base + h->cfg.warm_atoms, (size_t)natoms * sizeof(float4),
                cudaMemcpyDeviceToHost));
  *L = ws.L;
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_warm_import(mdeos_handle* h, uint64_t element_id, int32_t natoms,
                                          const float* x4, const float* v4, double L) {
  if (!h || !x4 || !v4 || natoms < 2 || !(L > 0) || element_id == 0)
    return fail(MDEOS_EINVAL, "bad warm_import arguments");
  std::lock_guard<std::mutex> lock(h->mu);
  if (!h->d_warm || natoms > h->cfg.warm_atoms)
    return fail(MDEOS_EINVAL, "no warm store, or natoms above warm_atoms");
  auto it = h->warm_map.find(element_id);
  if (it == h->warm_map.end()) {
    if (h->warm_next >= h->cfg.warm_slots) return fail(MDEOS_ENOMEM, "warm store full");
    WarmSlot ws;
    ws.slot = h->warm_next++;
    it = h->warm_map.emplace(element_id, ws).first;
  }
  WarmSlot& ws = it->second;
  std::vector<float4> hx((size_t)natoms), hv((size_t)natoms);
  for (int i = 0; i < natoms; ++i) {
    int id = i;
    float w;
    std::memcpy(&w, &id, sizeof(float));
    hx[i] = make_float4(x4[4 * i], x4[4 * i + 1], x4[4 * i + 2], w);
    hv[i] = make_float4(v4[4 * i], v4[4 * i + 1], v4[4 * i + 2], 0.f);
  }
  CK(cudaSetDevice(h->device));
  float4* base = h->d_warm + (size_t)ws.slot * 2 * h->cfg.warm_atoms;
  const unsigned long long tag = element_id;
  CK(cudaMemcpyAsync(base, hx.data(), (size_t)natoms * sizeof(float4), cudaMemcpyHostToDevice,
                     h->stream));
  CK(cudaMemcpyAsync(base + h->cfg.warm_atoms, hv.data(), (size_t)natoms * sizeof(float4),
                     cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->d_warm_tag + ws.slot, &tag, sizeof(tag), cudaMemcpyHostToDevice,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  ws.natoms = natoms;
  ws.L = L;
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_warm_reset(mdeos_handle* h) {
  if (!h) return fail(MDEOS_EINVAL, "handle is NULL");
  std::lock_guard<std::mutex> lock(h->mu);
  if (!h->d_warm) return MDEOS_OK;
  CK(cudaSetDevice(h->device));
  CK(cudaMemsetAsync(h->d_warm_tag, 0, (size_t)h->cfg.warm_slots * sizeof(unsigned long long),
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->warm_map.clear();
  h->warm_next = 0;
  return MDEOS_OK;
}

// ---------------------------------------------------------------------------
// evaluation into a caller's device array (used by the hydro driver)

namespace mdeos {

cudaStream_t handle_stream(const mdeos_handle* h) { return h->stream; }
int handle_device(const mdeos_handle* h) { return h->device; }
const mdeos_config& handle_config(const mdeos_handle* h) { return h->cfg; }

// Plans n requests (warm store included), uploads the work table and launches
// the persistent batch kernel on the handle's stream; d_results (device, n
// records) receives every result, planning rejections included, when the
// stream reaches it.  Synchronises the stream first: the work table buffers are
// reused from call to call.
mdeos_status eval_into_device(mdeos_handle* h, const mdeos_request* reqs, int n,
                              mdeos_result* d_results) {
  if (!h || !reqs || !d_results || n < 1) return fail(MDEOS_EINVAL, "bad eval arguments");
  std::lock_guard<std::mutex> lock(h->mu);
  CK(cudaSetDevice(h->device));
  CK(cudaStreamSynchronize(h->stream));
  Plan plan;
  mdeos_status st =
      make_plan(reqs, n, h->cfg, h->nsm, h->smem_max, plan, true, &h->tuned_skin, nullptr, true);
  if (st != MDEOS_OK) return st;
  assign_warm(h, plan, reqs);
  const size_t nb = plan.boxes.size(), ni = plan.items.size();
  const size_t off_items = (nb * sizeof(BoxDesc) + 255) & ~size_t(255);
  const size_t in_bytes = off_items + ni * sizeof(WorkItem);
  const size_t off_cnt = (in_bytes + 255) & ~size_t(255);
  const size_t dev_bytes = off_cnt + 256;
  bool rejected = false;
  for (int i = 0; i < n; ++i) rejected = rejected || plan.status[i] != MDEOS_OK;
  const size_t host_bytes = std::max(in_bytes, rejected ? (size_t)n * sizeof(mdeos_result) : 0);
  if (dev_bytes > h->eval_bytes) {
    if (h->cfg.hbm_budget_bytes && h->used_bytes + dev_bytes - h->eval_bytes > h->cfg.hbm_budget_bytes)
      return fail(MDEOS_ENOMEM, "batch exceeds the HBM budget");
    if (h->d_eval) CK(cudaFree(h->d_eval));
    h->used_bytes -= h->eval_bytes;
    h->d_eval = nullptr;
    h->eval_bytes = 0;
    CK(cudaMalloc(&h->d_eval, dev_bytes));
    h->eval_bytes = dev_bytes;
    h->used_bytes += dev_bytes;
  }
  if (host_bytes > h->eval_pinned.size) {
    if (h->eval_pinned.p) CK(cudaFreeHost(h->eval_pinned.p));
    h->eval_pinned.p = nullptr;
    h->eval_pinned.size = 0;
    CK(cudaMallocHost(&h->eval_pinned.p, host_bytes));
    h->eval_pinned.size = host_bytes;
  }
  char* d = (char*)h->d_eval;
  if (rejected) {
    mdeos_result* init = (mdeos_result*)h->eval_pinned.p;
    for (int i = 0; i < n; ++i) planning_result(init[i], plan.status[i], reqs[i]);
    CK(cudaMemcpyAsync(d_results, init, (size_t)n * sizeof(mdeos_result), cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));  // the staging buffer is reused below
  }
  if (nb == 0) return MDEOS_OK;
  std::memcpy(h->eval_pinned.p, plan.boxes.data(), nb * sizeof(BoxDesc));
  std::memcpy((char*)h->eval_pinned.p + off_items, plan.items.data(), ni * sizeof(WorkItem));
  const size_t scratch = (size_t)plan.grid * plan.nl_per_cta * sizeof(uint16_t);
  if ((st = ensure_scratch(h, scratch)) != MDEOS_OK) return st;
  CK(cudaMemcpyAsync(d, h->eval_pinned.p, in_bytes, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemsetAsync(d + off_cnt, 0, sizeof(int), h->stream));
  cudaError_t e = launch_eos_batch((BoxDesc*)d, (WorkItem*)(d + off_items), (int)ni,
                                   (int*)(d + off_cnt), d_results, h->d_nl, plan.nl_per_cta, h->rp,
                                   plan.grid, plan.smem, h->stream, nullptr, plan.cluster);
  if (e != cudaSuccess) return cuda_fail(e, "eos_batch_kernel launch");
  h->launches += 1;
  return MDEOS_OK;
}

void count_launch(mdeos_handle* h, long long k) { h->launches += k; }

const RunParams& handle_run_params(const mdeos_handle* h) { return h->rp; }
int handle_sm_count(const mdeos_handle* h) { return h->nsm; }
int handle_smem_max(const mdeos_handle* h) { return h->smem_max; }

void planning_result_of(mdeos_result& r, int status, const mdeos_request& q) {
  planning_result(r, status, q);
}

// Planning with the handle's configuration and device limits (no warm store).
mdeos_status plan_requests(const mdeos_handle* h, const mdeos_request* reqs, int n, PlanOut& out,
                           const int* cap_min) {
  Plan plan;
  mdeos_status st =
      make_plan(reqs, n, h->cfg, h->nsm, h->smem_max, plan, true, &h->tuned_skin, cap_min);
  if (st != MDEOS_OK) return st;
  out.boxes.swap(plan.boxes);
  out.items.swap(plan.items);
  out.status.swap(plan.status);
  out.smem = plan.smem;
  out.grid = plan.grid;
  out.nl_per_cta = plan.nl_per_cta;
  return MDEOS_OK;
}

}  // namespace mdeos

// ---------------------------------------------------------------------------
// single-box parity entry points

static mdeos_status debug_setup(const mdeos_config* cfg, int n, double L, int path, double skin,
                                BoxDesc& bd, RunParams& rp, int& apt, int& ncell, int& smem,
                                size_t& nl_bytes) {
  mdeos_status st = check_config(cfg);
  if (st != MDEOS_OK) return st;
  if (n < 2 || n > kMaxAtoms) return fail(MDEOS_EINVAL, "n must be in 2..4096");
  if (!(L >= cfg->rc)) return fail(MDEOS_EBOX, "box side below the cutoff");
  if (path < 0 || path > 2) return fail(MDEOS_EINVAL, "path must be 0, 1 or 2");
  if (path == PATH_ALLPAIRS && L < 2 * cfg->rc)
    return fail(MDEOS_EBOX, "all-pairs minimum image needs L >= 2 rc");
  if (path == PATH_NLIST && (!(skin >= 0) || L < 2 * (cfg->rc + skin)))
    return fail(MDEOS_EBOX, "Verlet list needs L >= 2 (rc + skin)");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
    return fail(MDEOS_ECUDA, "no CUDA device available");
  static bool attr_done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  int smem_max = 0;
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  smem_max -= 1024;
  if (dev < 64 && !attr_done[dev]) {
    CK(set_debug_attributes(smem_max));
    attr_done[dev] = true;
  }
  rp = make_run_params(cfg);
  std::memset(&bd, 0, sizeof(bd));
  bd.natoms = n;
  bd.L = L;
  bd.path = path;
  bd.skin = (float)skin;
  int ncl = 1;
  while (4LL * ncl * ncl * ncl < n) ++ncl;
  bd.nc_lat = ncl;
  apt = round_apt((n + kCtaThreads - 1) / kCtaThreads);
  ncell = 1;
  nl_bytes = 0;
  if (path == PATH_NLIST) {
    const double rs = cfg->rc + skin;
    const int nc = list_cells_per_axis(L, rs, n);
    bd.nc_cell = nc;
    ncell = nc > 0 ? nc * nc * nc : 1;
    bd.maxnb = std::max(8, ((n - 1 + kListPadSlack) + 7) & ~7);  // no overflow in tests
    if (nc == 0) bd.maxnb = brute_list_capacity(n, n);
    nl_bytes = (size_t)bd.maxnb * kCtaThreads * apt * sizeof(uint16_t);
  }
  smem = group_smem_bytes(32, apt, ncell);
  if (smem > smem_max) return fail(MDEOS_EINVAL, "box does not fit in shared memory");
  return MDEOS_OK;
}

// Boxes above the shared-memory limit: Verlet path with state in global memory.
// The list capacity is twice the liquid-density estimate (tests hand in arbitrary
// configurations; an overflow is reported as a NaN energy).
static mdeos_status debug_big_setup(const mdeos_config* cfg, int n, double L, int path,
                                    double skin, BoxDesc& bd, RunParams& rp, size_t& scratch) {
  mdeos_status st = check_config(cfg);
  if (st != MDEOS_OK) return st;
  if (n <= kMaxAtoms || n > kMaxAtomsBig) return fail(MDEOS_EINVAL, "n out of range");
  if (path != PATH_NLIST) return fail(MDEOS_EINVAL, "boxes above 4096 atoms use the Verlet path");
  if (!(skin >= 0) || L < 2 * (cfg->rc + skin))
    return fail(MDEOS_EBOX, "Verlet list needs L >= 2 (rc + skin)");
  const double rs = cfg->rc + skin;
  int nc = (int)std::floor(L / rs);
  while (nc > 3 && nc * nc * nc > kMaxCellsBig) --nc;
  if (nc < 3) return fail(MDEOS_EBOX, "fewer than 3 cells per axis");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
    return fail(MDEOS_ECUDA, "no CUDA device available");
  rp = make_run_params(cfg);
  std::memset(&bd, 0, sizeof(bd));
  bd.natoms = n;
  bd.L = L;
  bd.path = PATH_NLIST;
  bd.skin = (float)skin;
  bd.nc_cell = nc;
  const double rho = n / (L * L * L);
  int mx = (int)std::ceil(2.0 * 4.18879020478639 * rs * rs * rs * std::max(rho, 0.9) + 64.0);
  bd.maxnb = (std::min(mx, n - 1) + 7) & ~7;
  scratch = big_scratch_bytes(n, nc * nc * nc, bd.maxnb);
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_debug_lift(const mdeos_config* cfg, int32_t n, double rho, double T,
                                         uint64_t seed, float* x4, float* v4, double* e_out,
                                         double* L_out, void* stream) {
  if (!x4 || !v4 || !e_out || !(rho > 0) || !(T > 0)) return fail(MDEOS_EINVAL, "bad arguments");
  const double L = box_side(n, rho);
  if (L_out) *L_out = L;
  const int path = (L < 2 * cfg->rc) ? PATH_ALLPAIRS_MI : PATH_ALLPAIRS;
  BoxDesc bd;
  RunParams rp;
  int apt, ncell, smem;
  size_t nlb;
  mdeos_status st = debug_setup(cfg, n, L, path, 0.0, bd, rp, apt, ncell, smem, nlb);
  if (st != MDEOS_OK) return st;
  bd.seed = seed;
  cudaStream_t s = (cudaStream_t)stream;
  CK(launch_debug_lift(bd, rp, T, apt, ncell, smem, (float4*)x4, (float4*)v4, e_out, nullptr, s));
  CK(cudaStreamSynchronize(s));
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_debug_forces(const mdeos_config* cfg, const float* x4, int32_t n,
                                           double L, int32_t path, double skin, float* f4,
                                           double* ew, long long* pairs, void* stream) {
  if (!x4 || !f4 || !ew) return fail(MDEOS_EINVAL, "bad arguments");
  BoxDesc bd;
  RunParams rp;
  if (n > kMaxAtoms) {
    size_t sb = 0;
    mdeos_status st = debug_big_setup(cfg, n, L, path, skin, bd, rp, sb);
    if (st != MDEOS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* scratch = nullptr;
    CK(cudaMallocAsync(&scratch, sb, s));
    cudaError_t e = launch_debug_big_forces(bd, rp, scratch, (const float4*)x4, (float4*)f4, ew,
                                            pairs, s);
    cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "debug_big_forces launch");
    CK(cudaStreamSynchronize(s));
    return MDEOS_OK;
  }
  int apt, ncell, smem;
  size_t nlb;
  mdeos_status st = debug_setup(cfg, n, L, path, skin, bd, rp, apt, ncell, smem, nlb);
  if (st != MDEOS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  uint16_t* nl = nullptr;
  if (nlb) CK(cudaMallocAsync(&nl, nlb, s));
  cudaError_t e = launch_debug_forces(bd, rp, apt, ncell, smem, (const float4*)x4, (float4*)f4, ew,
                                      pairs, nl, s);
  if (nl) cudaFreeAsync(nl, s);
  if (e != cudaSuccess) return cuda_fail(e, "debug_forces launch");
  CK(cudaStreamSynchronize(s));
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_debug_force_bench(const mdeos_config* cfg, const float* x4,
                                                int32_t nbox, int32_t n, double L, double skin,
                                                int32_t passes, int32_t mode, long long* cycles,
                                                void* stream) {
  if (!x4 || !cycles || nbox < 1 || passes < 1 || mode < 0 || mode > 2 || n > kMaxAtoms)
    return fail(MDEOS_EINVAL, "bad arguments");
  int nsm = 0, dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (nbox > nsm) return fail(MDEOS_EINVAL, "at most one box per SM");
  BoxDesc bd;
  RunParams rp;
  int apt, ncell, smem;
  size_t nlb;
  mdeos_status st = debug_setup(cfg, n, L, PATH_NLIST, skin, bd, rp, apt, ncell, smem, nlb);
  if (st != MDEOS_OK) return st;
  // list capacity as the planner sets it (liquid density at least)
  const double rs = cfg->rc + skin;
  const double expect_cap = 4.18879020478639 * rs * rs * rs * std::max(n / (L * L * L), 0.9);
  bd.maxnb = (std::min((int)std::ceil(1.3 * expect_cap + 32.0) + kListPadSlack,
                      n - 1 + kListPadSlack) + 7) & ~7;
  if (bd.nc_cell == 0) bd.maxnb = brute_list_capacity(n, bd.maxnb);
  const long long nl_elems = (long long)bd.maxnb * kCtaThreads * apt;
  cudaStream_t s = (cudaStream_t)stream;
  uint16_t* nl = nullptr;
  CK(cudaMallocAsync(&nl, (size_t)nl_elems * nbox * sizeof(uint16_t), s));
  cudaError_t e = launch_debug_force_bench(bd, rp, apt, ncell, smem, (const float4*)x4, nbox,
                                           passes, mode, cycles, nl, nl_elems, s);
  cudaFreeAsync(nl, s);
  if (e != cudaSuccess) return cuda_fail(e, "debug_force_bench launch");
  CK(cudaStreamSynchronize(s));
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_debug_md(const mdeos_config* cfg, float* x4, float* v4, int32_t n,
                                       double L, int32_t steps, double T_target,
                                       int32_t rescale_every, int32_t path, double skin,
                                       double* epot, double* ekin, long long* cycles,
                                       void* stream) {
  if (!x4 || !v4 || steps < 0 || rescale_every < 0) return fail(MDEOS_EINVAL, "bad arguments");
  BoxDesc bd;
  RunParams rp;
  if (n > kMaxAtoms) {
    size_t sb = 0;
    mdeos_status st = debug_big_setup(cfg, n, L, path, skin, bd, rp, sb);
    if (st != MDEOS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* scratch = nullptr;
    CK(cudaMallocAsync(&scratch, sb, s));
    cudaError_t e = launch_debug_big_md(bd, rp, scratch, (float4*)x4, (float4*)v4, steps, T_target,
                                        rescale_every, epot, ekin, cycles, s);
    cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "debug_big_md launch");
    CK(cudaStreamSynchronize(s));
    return MDEOS_OK;
  }
  int apt, ncell, smem;
  size_t nlb;
  mdeos_status st = debug_setup(cfg, n, L, path, skin, bd, rp, apt, ncell, smem, nlb);
  if (st != MDEOS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  uint16_t* nl = nullptr;
  if (nlb) CK(cudaMallocAsync(&nl, nlb, s));
  cudaError_t e = launch_debug_md(bd, rp, apt, ncell, smem, (float4*)x4, (float4*)v4, steps,
                                  T_target, rescale_every, epot, ekin, cycles, nl, s);
  if (nl) cudaFreeAsync(nl, s);
  if (e != cudaSuccess) return cuda_fail(e, "debug_md launch");
  CK(cudaStreamSynchronize(s));
  return MDEOS_OK;
}

// ---------------------------------------------------------------------------
// statistics for benchmarks

extern "C" mdeos_status mdeos_stats(const mdeos_handle* h, size_t* last_h2d_bytes,
                                    size_t* last_d2h_bytes, long long* kernel_launches,
                                    size_t* device_bytes) {
  if (!h) return fail(MDEOS_EINVAL, "handle is NULL");
  if (last_h2d_bytes) *last_h2d_bytes = h->last_h2d;
  if (last_d2h_bytes) *last_d2h_bytes = h->last_d2h;
  if (kernel_launches) *kernel_launches = h->launches;
  if (device_bytes) *device_bytes = h->used_bytes;
  return MDEOS_OK;
}
