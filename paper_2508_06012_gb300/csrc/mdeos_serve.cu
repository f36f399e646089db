// Serving loop of the atomistic EOS with continuous batching.
//
// Requests arrive one by one (a hydrocode's elements, many clients).  A scheduler
// thread plans whatever is waiting into work items (boxes of one size class,
// longest first) and publishes them into rings in host-mapped pinned memory; one
// persistent kernel grid (eos_serve_kernel, one CTA per SM) claims items one at a
// time, so an SM that finishes an item takes the next one at once, whichever
// admission step it came from.  Each box's result and ready flag are written to
// host-mapped memory (reached over the coherent chip-to-chip link on a
// Grace-Blackwell node), so every request is reported when its own box is done.
//
// The kernel waits for work with a bounded idle time and exits; the scheduler
// relaunches it when new items are published and no grid is running.
// Admission: at most max_inflight requests on the GPU; waiting requests older than
// max_wait_s and arrivals beyond max_queue are shed with MDEOS_ECANCELLED.  Device
// memory: per-SM scratch for the largest box, fixed at creation, and the element
// store (warm starts), whose blocks are reserved at admission and released when
// the request's result comes back; a request whose element state does not fit
// while the store is held by requests in flight waits for them.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mdeos_host.h"

using namespace mdeos;

namespace mdeos {
// the cluster form of the serving kernel (mdeos_serve_cluster.cu)
cudaError_t set_serve_cluster_attributes(int max_smem);
cudaError_t launch_eos_serve_cluster(const ServeQueue& q, const RunParams& rp, uint16_t* nl,
                                     long long nl_elems_per_cta, int grid, int smem,
                                     cudaStream_t st, int cluster);
}  // namespace mdeos

namespace {

struct Waiting {
  uint64_t id;
  mdeos_request r;
  double t_arr;
  int cap_min = 0;   // Verlet-list capacity at least (a re-run after an overflow)
  int retries = 0;   // re-runs so far
  bool waited = false;  // has waited for element-store memory
};

// One element's block of the store: [tag uint64 + pad (16 B)] [x float4[natoms]]
// [v float4[natoms]]; the device writes the tag (the element_id of a valid state).
struct StoreEntry {
  size_t off = 0, bytes = 0;
  int natoms = 0;
  double L = 0.0;         // box side of the stored state (0: none)
  double last_use = 0.0;
  int inflight = 0;       // a request of this element is on the GPU
};

struct InFlight {
  Waiting w;
  unsigned item_slot;
  double t_pub;
};

unsigned pow2_at_least(unsigned v) {
  unsigned p = 1;
  while (p < v) p <<= 1;
  return p;
}

}  // namespace

struct mdeos_server {
  mdeos_handle* h = nullptr;
  mdeos_serve_config cfg;
  int device = 0, grid = 0, smem = 0;
  int cluster = 1;  // CTAs per thread-block cluster of the serving grid (1: eos_serve_kernel)
  std::chrono::steady_clock::time_point t0;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Waiting> waiting;
  std::deque<mdeos_served> completed;
  std::atomic<bool> stop{false};
  uint64_t next_id = 1;
  long long n_enq = 0, n_admitted = 0, n_done = 0, n_cancel = 0, n_launch = 0, n_err = 0;
  // queue
  unsigned cap_items = 0, cap_boxes = 0;
  BoxDesc* h_boxes = nullptr;
  WorkItem* h_items = nullptr;
  mdeos_result* h_res = nullptr;
  int* h_ready = nullptr;
  unsigned* h_tail = nullptr;
  int* h_stop = nullptr;
  ServeQueue q;
  unsigned* d_head = nullptr;  // head counter, then nslots scratch-slot flags
  int* h_alive = nullptr;       // host-mapped, nslots
  int* h_linger = nullptr;      // host-mapped
  double last_arrival = -1.0;
  uint16_t* d_nl = nullptr;
  long long nl_per_cta = 0;
  size_t dev_bytes = 0;
  static constexpr int kGrids = 8;  // kernel grids in flight at once
  cudaStream_t st[kGrids] = {};
  cudaEvent_t ev[kGrids] = {};
  bool running[kGrids] = {};
  double last_launch = -1.0;
  long long outstanding_items = 0;
  // element store (scheduler thread only, counters read by stats)
  unsigned char* d_store = nullptr;
  size_t store_cap = 0, store_used = 0;
  std::unordered_map<uint64_t, StoreEntry> store;
  std::map<size_t, size_t> store_free;  // free blocks: offset -> bytes, coalesced
  std::atomic<long long> n_warm{0}, n_memwait{0}, n_evict{0}, n_stored{0};
  std::atomic<size_t> store_used_pub{0};
  unsigned published = 0;               // items published (= *h_tail)
  std::vector<int> item_pending;         // boxes not yet reported, per item slot
  std::vector<unsigned> free_boxes;      // free box ring slots
  std::vector<InFlight> inflight_box;    // by box slot
  std::vector<unsigned> inflight_slots;  // box slots in flight
  long long peak_inflight = 0;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

static mdeos_served make_served(const Waiting& w, double t_launch, double t_done,
                                const mdeos_result& r) {
  mdeos_served s;
  std::memset(&s, 0, sizeof(s));
  s.id = w.id;
  s.t_arrival = w.t_arr;
  s.t_launch = t_launch;
  s.t_done = t_done;
  s.result = r;
  return s;
}

static mdeos_served shed(const Waiting& w, double t, int status) {
  mdeos_result r;
  planning_result_of(r, status, w.r);
  return make_served(w, t, t, r);
}

// ---- element store (first fit over coalesced free blocks) ----------------------

static bool store_alloc(mdeos_server* s, size_t bytes, size_t& off) {
  for (auto it = s->store_free.begin(); it != s->store_free.end(); ++it) {
    if (it->second < bytes) continue;
    off = it->first;
    const size_t rest = it->second - bytes;
    s->store_free.erase(it);
    if (rest) s->store_free[off + bytes] = rest;
    s->store_used += bytes;
    return true;
  }
  return false;
}

static void store_release(mdeos_server* s, size_t off, size_t bytes) {
  s->store_used -= bytes;
  auto it = s->store_free.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != s->store_free.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    s->store_free.erase(nx);
  }
  if (it != s->store_free.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      s->store_free.erase(it);
    }
  }
}

// Reserve the element's block for a request about to be admitted: 1 = reserved,
// 0 = no state kept (no element, above 4096 atoms or larger than the store: runs
// cold), -1 = wait (the element's previous request is in flight, or the store is
// held by requests in flight).  Blocks of elements with nothing in flight are
// reclaimed least recently used first.
static int store_reserve(mdeos_server* s, const mdeos_request& r, double t) {
  if (!s->d_store || r.element_id == 0 || r.natoms > kMaxAtoms) return 0;
  const size_t bytes = (16 + 32 * (size_t)r.natoms + 255) & ~(size_t)255;
  if (bytes > s->store_cap) return 0;
  auto it = s->store.find(r.element_id);
  if (it != s->store.end()) {
    if (it->second.inflight > 0) return -1;
    if (it->second.natoms == r.natoms) {
      it->second.inflight = 1;
      it->second.last_use = t;
      return 1;
    }
    store_release(s, it->second.off, it->second.bytes);
    s->store.erase(it);
  }
  size_t off = 0;
  while (!store_alloc(s, bytes, off)) {
    auto lru = s->store.end();
    for (auto e = s->store.begin(); e != s->store.end(); ++e)
      if (e->second.inflight == 0 &&
          (lru == s->store.end() || e->second.last_use < lru->second.last_use))
        lru = e;
    if (lru == s->store.end()) {  // the rest is held by requests in flight: wait
      s->n_stored = (long long)s->store.size();
      s->store_used_pub = s->store_used;
      return -1;
    }
    store_release(s, lru->second.off, lru->second.bytes);
    s->store.erase(lru);
    ++s->n_evict;
  }
  StoreEntry e;
  e.off = off;
  e.bytes = bytes;
  e.natoms = r.natoms;
  e.last_use = t;
  e.inflight = 1;
  s->store[r.element_id] = e;
  s->n_stored = (long long)s->store.size();
  s->store_used_pub = s->store_used;
  return 1;
}

// A request's result came back (or will not): release its element's block for
// reuse and record whether the block now holds a valid state.
static void store_done(mdeos_server* s, const BoxDesc& bd, int status, double t) {
  if (!bd.warm_state) return;
  auto it = s->store.find(bd.element_id);
  if (it == s->store.end()) return;
  it->second.inflight = 0;
  it->second.last_use = t;
  if (status == MDEOS_OK)
    it->second.L = bd.L;
  else if (status != MDEOS_ENBR)
    it->second.L = 0.0;  // the device cleared the tag; an overflow left the state as it was
}

// Report every box whose ready flag is up; with fail_status != 0 (kernel failure,
// or no grid left to run them at shutdown) report the rest with that status.
static bool harvest(mdeos_server* s, int fail_status) {
  std::vector<mdeos_served> out;
  std::vector<unsigned> keep;
  keep.reserve(s->inflight_slots.size());
  std::vector<Waiting> rerun;
  for (unsigned slot : s->inflight_slots) {
    InFlight& f = s->inflight_box[slot];
    if (reinterpret_cast<volatile int*>(s->h_ready)[slot] != 0) {
      std::atomic_thread_fence(std::memory_order_acquire);
      const mdeos_result& r = s->h_res[slot];
      const int cap = s->h_boxes[slot].maxnb;
      store_done(s, s->h_boxes[slot], r.status, s->now());
      if (r.status == MDEOS_OK && r.warm == 1) ++s->n_warm;
      if (r.status == MDEOS_ENBR && cap < f.w.r.natoms - 1 && f.w.retries < 16) {
        // the box's Verlet list overflowed: run it again with twice the capacity,
        // ahead of the queue (as mdeos_poll does)
        Waiting w = f.w;
        w.cap_min = 2 * cap;
        ++w.retries;
        rerun.push_back(w);
      } else {
        mdeos_served o = make_served(f.w, f.t_pub, s->now(), r);
        o.result.nlist_retries = f.w.retries;
        out.push_back(o);
      }
    } else if (fail_status != 0) {
      store_done(s, s->h_boxes[slot], fail_status, s->now());
      out.push_back(shed(f.w, s->now(), fail_status));
      if (fail_status == MDEOS_ECUDA) ++s->n_err;
      if (fail_status == MDEOS_ECANCELLED) ++s->n_cancel;
    } else {
      keep.push_back(slot);
      continue;
    }
    if (--s->item_pending[f.item_slot] == 0) --s->outstanding_items;
    s->free_boxes.push_back(slot);
  }
  if (out.empty() && rerun.empty()) return false;
  s->inflight_slots.swap(keep);
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto& o : out) s->completed.push_back(o);
  for (auto it = rerun.rbegin(); it != rerun.rend(); ++it) s->waiting.push_front(*it);
  s->n_done += (long long)out.size();
  return true;
}

// Plan a batch of waiting requests into items and publish them.  Requests the
// queue cannot take now (ring slots) are handed back in `b`.
static void store_unreserve(mdeos_server* s, const mdeos_request& r) {
  auto it = s->store.find(r.element_id);
  if (it != s->store.end() && r.element_id != 0) it->second.inflight = 0;
}

// Plan a batch of waiting requests into items and publish them.  Requests whose
// element state has no room in the store yet, and requests the queue cannot take
// now (ring slots), are handed back in `b`.
static bool admit(mdeos_server* s, std::vector<Waiting>& b) {
  const double t = s->now();
  std::vector<Waiting> go, wait;
  std::vector<char> reserved;
  for (auto& w : b) {
    const int k = store_reserve(s, w.r, t);
    if (k < 0) {
      if (!w.waited) {
        w.waited = true;
        ++s->n_memwait;
      }
      wait.push_back(w);
    } else {
      go.push_back(w);
      reserved.push_back(k == 1 ? 1 : 0);
    }
  }
  const int n = (int)go.size();
  if (n == 0) {
    b.swap(wait);
    return false;
  }
  std::vector<mdeos_request> rq(n);
  std::vector<int> cap_min(n);
  for (int i = 0; i < n; ++i) {
    rq[i] = go[i].r;
    cap_min[i] = go[i].cap_min;
  }
  PlanOut plan;
  std::vector<mdeos_served> out;
  const int warm_iters = handle_config(s->h).warm_lift_iters;
  std::vector<Waiting> rest;
  if (plan_requests(s->h, rq.data(), n, plan, cap_min.data()) != MDEOS_OK) {
    for (int i = 0; i < n; ++i) {
      if (reserved[i]) store_unreserve(s, go[i].r);
      out.push_back(shed(go[i], t, MDEOS_EINVAL));
    }
  } else {
    std::vector<char> taken(n, 0);
    for (int i = 0; i < n; ++i)
      if (plan.status[i] != MDEOS_OK) {
        if (reserved[i]) store_unreserve(s, go[i].r);
        out.push_back(shed(go[i], t, plan.status[i]));
        taken[i] = 1;
      }
    for (const WorkItem& wi0 : plan.items) {
      // ring space: one item slot and wi0.nbox box slots
      const unsigned islot = s->published % s->cap_items;
      if (s->item_pending[islot] != 0 || (int)s->free_boxes.size() < wi0.nbox) break;
      if ((long long)wi0.nl_stride * (wi0.big ? 1 : wi0.nbox) > s->nl_per_cta ||
          wi0.nbox * wi0.smem_stride > s->smem) {
        for (int k = 0; k < wi0.nbox; ++k) {  // needs more per-SM memory than held
          const int ri = plan.boxes[wi0.box[k]].out_index;
          if (reserved[ri]) store_unreserve(s, go[ri].r);
          out.push_back(shed(go[ri], t, MDEOS_ENOMEM));
          taken[ri] = 1;
        }
        continue;
      }
      WorkItem wi = wi0;
      for (int k = 0; k < wi.nbox; ++k) {
        BoxDesc bd = plan.boxes[wi0.box[k]];
        const int ri = bd.out_index;  // request index within the batch
        if (reserved[ri]) {  // the element's block: its state, tag and box side
          const StoreEntry& e = s->store[go[ri].r.element_id];
          const mdeos_request& r = go[ri].r;
          const bool try_warm = e.L > 0.0 && (r.flags & MDEOS_REQ_COLD) == 0 &&
                                (r.steps_equil == 0 || r.steps_equil >= warm_iters);
          bd.warm_tag = reinterpret_cast<unsigned long long*>(s->d_store + e.off);
          bd.warm_state = reinterpret_cast<float4*>(s->d_store + e.off + 16);
          bd.warm_cap = e.natoms;
          bd.L_old = try_warm ? e.L : 0.0;
        }
        const unsigned slot = s->free_boxes.back();
        s->free_boxes.pop_back();
        bd.out_index = (int)slot;
        s->h_boxes[slot] = bd;
        s->h_ready[slot] = 0;
        s->inflight_box[slot] = InFlight{go[ri], islot, t};
        s->inflight_slots.push_back(slot);
        wi.box[k] = (int)slot;
        taken[ri] = 1;
      }
      s->h_items[islot] = wi;
      s->item_pending[islot] = wi.nbox;
      ++s->outstanding_items;
      std::atomic_thread_fence(std::memory_order_release);
      ++s->published;
      reinterpret_cast<std::atomic<unsigned>*>(s->h_tail)->store(s->published,
                                                                 std::memory_order_release);
      s->n_admitted += wi.nbox;
    }
    for (int i = 0; i < n; ++i)
      if (!taken[i]) {
        if (reserved[i]) store_unreserve(s, go[i].r);
        rest.push_back(go[i]);
      }
  }
  rest.insert(rest.end(), wait.begin(), wait.end());
  b.swap(rest);
  s->peak_inflight = std::max<long long>(s->peak_inflight, (long long)s->inflight_slots.size());
  if (!out.empty()) {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& o : out) s->completed.push_back(o);
    s->n_done += (long long)out.size();
  }
  return true;
}

static void serve_loop(mdeos_server* s) {
  cudaSetDevice(s->device);
  std::vector<Waiting> held;  // planned but not published (ring full): first in line
  for (;;) {
    bool did = false;
    bool failed = false;
    bool any_running = false;
    for (int g = 0; g < mdeos_server::kGrids; ++g) {
      if (!s->running[g]) continue;
      const cudaError_t q = cudaEventQuery(s->ev[g]);
      if (q != cudaErrorNotReady) {
        s->running[g] = false;
        failed = failed || q != cudaSuccess;
      } else {
        any_running = true;
      }
    }
    did = harvest(s, failed ? MDEOS_ECUDA : 0) || did;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      const double t = s->now();
      const bool stopping = s->stop.load();
      while (!s->waiting.empty() &&
             (stopping ||
              (s->cfg.max_wait_s > 0 && t - s->waiting.front().t_arr > s->cfg.max_wait_s))) {
        s->completed.push_back(shed(s->waiting.front(), t, MDEOS_ECANCELLED));
        s->waiting.pop_front();
        ++s->n_cancel;
        ++s->n_done;
        did = true;
      }
    }
    if (!s->stop.load()) {
      const int room = s->cfg.max_inflight - (int)s->inflight_slots.size();
      if (held.empty() && room > 0) {
        std::lock_guard<std::mutex> lk(s->mu);
        const int take = std::min<int>({(int)s->waiting.size(), s->cfg.max_batch, room});
        for (int i = 0; i < take; ++i) {
          held.push_back(s->waiting.front());
          s->waiting.pop_front();
        }
      }
      if (!held.empty()) {
        const size_t before = held.size();
        admit(s, held);
        did = did || held.size() != before;
      }
    }
    // idle CTAs stay while traffic is active (work outstanding or waiting, or an
    // arrival in the last 100 ms)
    {
      bool active;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        active = !s->waiting.empty() || (s->last_arrival >= 0 && s->now() - s->last_arrival < 0.1);
      }
      active = active || s->outstanding_items > 0 || !held.empty();
      reinterpret_cast<std::atomic<int>*>(s->h_linger)->store(active && !s->stop.load() ? 1 : 0,
                                                              std::memory_order_release);
    }
    // more outstanding items than live CTAs: fill the GPU to one CTA per SM; a grid
    // just launched gets 2 ms for its CTAs to start before the count is trusted
    if (!s->stop.load() && s->outstanding_items > 0) {
      int alive = 0;
      for (int k = 0; k < s->grid; ++k) alive += reinterpret_cast<volatile int*>(s->h_alive)[k];
      const double t = s->now();
      int free_g = -1;
      for (int g = 0; g < mdeos_server::kGrids && free_g < 0; ++g)
        if (!s->running[g]) free_g = g;
      const bool cold = !any_running;
      // (a whole number of clusters)
      const int nct = (s->grid - alive) / s->cluster * s->cluster;
      if (free_g >= 0 && nct > 0 && s->outstanding_items > alive &&
          (cold || t - s->last_launch > 0.002)) {
        cudaError_t e =
            s->cluster > 1
                ? launch_eos_serve_cluster(s->q, handle_run_params(s->h), s->d_nl, s->nl_per_cta,
                                           nct, s->smem, s->st[free_g], s->cluster)
                : launch_eos_serve(s->q, handle_run_params(s->h), s->d_nl, s->nl_per_cta, nct,
                                   s->smem, s->st[free_g]);
        if (e == cudaSuccess) e = cudaEventRecord(s->ev[free_g], s->st[free_g]);
        if (e == cudaSuccess) {
          s->running[free_g] = true;
          any_running = true;
          s->last_launch = t;
          ++s->n_launch;
          count_launch(s->h, 1);
        } else if (cold) {
          harvest(s, MDEOS_ECUDA);  // nothing can run what is in flight
        }
        did = true;
      }
    }
    if (s->stop.load() && !any_running) {
      harvest(s, MDEOS_ECANCELLED);  // published but never claimed
      std::lock_guard<std::mutex> lk(s->mu);
      for (auto& w : held) {
        s->completed.push_back(shed(w, s->now(), MDEOS_ECANCELLED));
        ++s->n_cancel;
        ++s->n_done;
      }
      held.clear();
      if (s->waiting.empty()) break;
      continue;
    }
    if (!did) {
      std::unique_lock<std::mutex> lk(s->mu);
      if (any_running || !held.empty())
        s->cv.wait_for(lk, std::chrono::microseconds(20));
      else
        s->cv.wait_for(lk, std::chrono::milliseconds(2),
                       [s] { return !s->waiting.empty() || s->stop.load(); });
    }
  }
}

extern "C" void mdeos_serve_config_default(mdeos_serve_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->max_inflight = 4096;
  c->max_batch = 2048;
  c->max_wait_s = 0.0;
  c->max_queue = 0;
  c->idle_ms = 20;
  c->hbm_budget_bytes = 0;
  c->cluster = 1;
}

extern "C" mdeos_status mdeos_serve_destroy(mdeos_server* s);

extern "C" mdeos_status mdeos_serve_create(mdeos_handle* h, const mdeos_serve_config* cfg,
                                           mdeos_server** out) {
  if (!h || !cfg || !out) return set_error(MDEOS_EINVAL, "bad serve_create arguments");
  *out = nullptr;
  if (cfg->max_inflight < 1 || cfg->max_inflight > (1 << 20) || cfg->max_batch < 1 ||
      cfg->max_queue < 0 || !(cfg->max_wait_s >= 0) || cfg->idle_ms < 1 || cfg->idle_ms > 60000 ||
      !(cfg->cluster == 0 || cfg->cluster == 1 || cfg->cluster == 2 || cfg->cluster == 4 ||
        cfg->cluster == 8))
    return set_error(MDEOS_EINVAL, "serve config out of range");
  mdeos_server* s = new mdeos_server();
  s->h = h;
  s->cfg = *cfg;
  s->device = handle_device(h);
  s->grid = handle_sm_count(h);
  s->smem = handle_smem_max(h);
  {  // the serving grid in thread-block clusters of cfg->cluster CTAs (a power of two
     // dividing the grid; 0 or 1: none)
    int p = 1;
    while (2 * p <= cfg->cluster && s->grid % (2 * p) == 0) p *= 2;
    s->cluster = p;
    if (p > 1) {
      const cudaError_t e = set_serve_cluster_attributes(s->smem);
      if (e != cudaSuccess) {
        delete s;
        return set_error(MDEOS_ECUDA, std::string("serving cluster kernel: ") +
                                          cudaGetErrorString(e));
      }
    }
  }
  s->t0 = std::chrono::steady_clock::now();
  // per-SM scratch: the largest item, a 32768-atom box with the list capacity of
  // the densest liquid the planner admits (or a full shared-memory item)
  const int nmax = kMaxAtomsBig;
  const size_t big = big_scratch_bytes(nmax, kMaxCellsBig, 256);
  const size_t small = (size_t)256 * kCtaThreads * 4 * sizeof(uint16_t);
  s->nl_per_cta = (long long)((std::max(big, small) + 15) / 16 * 8);
  s->dev_bytes = (size_t)s->grid * s->nl_per_cta * sizeof(uint16_t) + 256;
  if (cfg->hbm_budget_bytes && s->dev_bytes > cfg->hbm_budget_bytes) {
    delete s;
    return set_error(MDEOS_ENOMEM, "the server's per-SM scratch exceeds hbm_budget_bytes");
  }
  if (cfg->warm) {  // element store: what the budget leaves, or as configured
    size_t cap = cfg->warm_bytes;
    if (cap == 0)
      cap = cfg->hbm_budget_bytes ? cfg->hbm_budget_bytes - s->dev_bytes : (size_t(1) << 30);
    if (cfg->hbm_budget_bytes && s->dev_bytes + cap > cfg->hbm_budget_bytes) {
      delete s;
      return set_error(MDEOS_ENOMEM, "scratch plus warm_bytes exceed hbm_budget_bytes");
    }
    s->store_cap = cap & ~(size_t)255;
  }
  s->cap_items = pow2_at_least((unsigned)cfg->max_inflight * 2);
  s->cap_boxes = pow2_at_least((unsigned)cfg->max_inflight * 2);
  cudaError_t e = cudaSetDevice(s->device);
  auto halloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaHostAlloc(p, bytes, cudaHostAllocMapped);
    if (e == cudaSuccess) std::memset(*p, 0, bytes);
  };
  halloc((void**)&s->h_boxes, s->cap_boxes * sizeof(BoxDesc));
  halloc((void**)&s->h_items, s->cap_items * sizeof(WorkItem));
  halloc((void**)&s->h_res, s->cap_boxes * sizeof(mdeos_result));
  halloc((void**)&s->h_ready, s->cap_boxes * sizeof(int));
  halloc((void**)&s->h_tail, 64);
  halloc((void**)&s->h_stop, 64);
  halloc((void**)&s->h_alive, (size_t)s->grid * sizeof(int));
  halloc((void**)&s->h_linger, 64);
  const size_t head_bytes = 256 + (size_t)s->grid * sizeof(int);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_head, head_bytes);
  if (e == cudaSuccess) e = cudaMemset(s->d_head, 0, head_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_nl, (size_t)s->grid * s->nl_per_cta * sizeof(uint16_t));
  if (e == cudaSuccess && s->store_cap >= 256) {
    e = cudaMalloc(&s->d_store, s->store_cap);
    if (e == cudaSuccess) e = cudaMemset(s->d_store, 0, s->store_cap);  // no valid tags
    if (e == cudaSuccess) {
      s->store_free[0] = s->store_cap;
      s->dev_bytes += s->store_cap;
    }
  }
  for (int g = 0; g < mdeos_server::kGrids; ++g) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->st[g], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev[g], cudaEventDisableTiming);
  }
  ServeQueue& q = s->q;
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&q.boxes, s->h_boxes, 0);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&q.items, s->h_items, 0);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&q.results, s->h_res, 0);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&q.ready, s->h_ready, 0);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&q.tail, s->h_tail, 0);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&q.stop, s->h_stop, 0);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&q.alive, s->h_alive, 0);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&q.linger, s->h_linger, 0);
  if (e != cudaSuccess) {
    mdeos_serve_destroy(s);
    return set_error(MDEOS_ECUDA, std::string("serve_create: ") + cudaGetErrorString(e));
  }
  q.head = s->d_head;
  q.slot_busy = reinterpret_cast<int*>(reinterpret_cast<char*>(s->d_head) + 256);
  q.nslots = s->grid;
  q.cap_items = s->cap_items;
  q.cap_boxes = s->cap_boxes;
  q.idle_ns = (long long)cfg->idle_ms * 1000000LL;
  q.max_idle_ns = 5000000000LL;
  s->item_pending.assign(s->cap_items, 0);
  s->inflight_box.resize(s->cap_boxes);
  for (unsigned k = s->cap_boxes; k-- > 0;) s->free_boxes.push_back(k);
  s->th = std::thread(serve_loop, s);
  *out = s;
  return MDEOS_OK;
}

extern "C" double mdeos_serve_clock(const mdeos_server* s) { return s ? s->now() : 0.0; }

extern "C" mdeos_status mdeos_serve_enqueue(mdeos_server* s, const mdeos_request* reqs, int32_t n,
                                            uint64_t* ids) {
  if (!s || !reqs || n < 0) return set_error(MDEOS_EINVAL, "bad serve_enqueue arguments");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    const double t = s->now();
    if (n > 0) s->last_arrival = t;
    for (int i = 0; i < n; ++i) {
      Waiting w{s->next_id++, reqs[i], t};
      if (ids) ids[i] = w.id;
      ++s->n_enq;
      if (s->stop.load() ||
          (s->cfg.max_queue > 0 && (int)s->waiting.size() >= s->cfg.max_queue)) {
        s->completed.push_back(shed(w, t, MDEOS_ECANCELLED));  // back-pressure
        ++s->n_cancel;
        ++s->n_done;
      } else {
        s->waiting.push_back(w);
      }
    }
  }
  s->cv.notify_one();
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_serve_completed(mdeos_server* s, mdeos_served* out, int32_t max,
                                              int32_t* n_out) {
  if (!s || !out || max < 0 || !n_out)
    return set_error(MDEOS_EINVAL, "bad serve_completed arguments");
  std::lock_guard<std::mutex> lk(s->mu);
  int k = 0;
  while (k < max && !s->completed.empty()) {
    out[k++] = s->completed.front();
    s->completed.pop_front();
  }
  *n_out = k;
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_serve_stats(mdeos_server* s, long long* counts, size_t* bytes) {
  if (!s) return set_error(MDEOS_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  if (counts) {
    counts[0] = s->n_enq;
    counts[1] = s->n_admitted;
    counts[2] = s->n_done;
    counts[3] = s->n_cancel;
    counts[4] = s->n_launch;
    counts[5] = (long long)s->waiting.size();
    counts[6] = s->n_err;
  }
  if (bytes) {
    bytes[0] = s->dev_bytes;
    bytes[1] = (size_t)s->peak_inflight;
  }
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_serve_store_stats(mdeos_server* s, long long* counts,
                                                size_t* bytes) {
  if (!s) return set_error(MDEOS_EINVAL, "server is NULL");
  if (counts) {
    counts[0] = s->n_warm;
    counts[1] = s->n_memwait;
    counts[2] = s->n_evict;
    counts[3] = s->n_stored;
  }
  if (bytes) {
    bytes[0] = s->store_used_pub;
    bytes[1] = s->d_store ? s->store_cap : 0;
  }
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_serve_destroy(mdeos_server* s) {
  if (!s) return MDEOS_OK;
  s->stop.store(true);
  if (s->h_stop) reinterpret_cast<std::atomic<int>*>(s->h_stop)->store(1, std::memory_order_release);
  if (s->h_linger)
    reinterpret_cast<std::atomic<int>*>(s->h_linger)->store(0, std::memory_order_release);
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  cudaSetDevice(s->device);
  for (int g = 0; g < mdeos_server::kGrids; ++g) {
    if (s->st[g]) cudaStreamSynchronize(s->st[g]);
    if (s->ev[g]) cudaEventDestroy(s->ev[g]);
    if (s->st[g]) cudaStreamDestroy(s->st[g]);
  }
  if (s->d_nl) cudaFree(s->d_nl);
  if (s->d_store) cudaFree(s->d_store);
  if (s->d_head) cudaFree(s->d_head);
  for (void* p : {(void*)s->h_boxes, (void*)s->h_items, (void*)s->h_res, (void*)s->h_ready,
                  (void*)s->h_tail, (void*)s->h_stop, (void*)s->h_alive, (void*)s->h_linger})
    if (p) cudaFreeHost(p);
  delete s;
  return MDEOS_OK;
}
