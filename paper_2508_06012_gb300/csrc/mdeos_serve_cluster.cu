// Cluster form of the continuous-batching kernel (eos_serve_kernel): the serving
// loop's CTAs in thread-block clusters of csize, so that a box above the shared-memory
// limit runs on a whole cluster (run_big with csize > 1: a slab of its atoms per CTA)
// instead of one SM, while boxes of up to 4096 atoms still run one item per CTA
// (arXiv 2508.06012, Sec. III: one independent MD run per element and call).
//
// Rounds.  The cluster's first CTA (its thread 0, the leader) opens each round: with
// an item above the shared-memory limit in hand (claimed at the head of the queue) a
// big round for the whole cluster, otherwise a small round, in which every CTA claims
// and runs items of smaller boxes on its own.  During a small round a big item at the
// head is claimed by the first free leader for its cluster's next round; that leader
// stops claiming and raises a flag in its shared memory, which its CTAs read before
// every claim; other CTAs wait at a big head until a leader takes it.  Every wait and
// every claiming loop of a round ends after kRoundNs at the latest (items run to
// completion), so a flag seen late only delays the round.  The leader stores the
// round's command into every CTA's shared memory; a cluster barrier; every CTA runs its
// part; a cluster barrier ends the round.  Every CTA passes the same two barriers per
// round whatever it runs, and the loop ends only on the leader's command (stop flag or
// idle time, the same bounded criteria as eos_serve_kernel), so no CTA can wait on a
// barrier that another CTA skips.
#include "mdeos_big.cuh"

namespace mdeos {

namespace {

__device__ __forceinline__ unsigned long long clock_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned load_acquire_sys(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// a 32-bit word of another CTA's shared memory (the cluster's leader), read afresh
__device__ __forceinline__ int ld_cluster_s32(uint32_t a) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}

enum : int { kCmdExit = 0, kCmdBig = 1, kCmdSmall = 2 };

constexpr unsigned long long kRoundNs = 100000000ull;  // longest claiming time of a small round

}  // namespace

__global__ void __launch_bounds__(kCtaThreads, 1)
    eos_serve_cluster_kernel(ServeQueue q, RunParams rp, uint16_t* nl_scratch,
                             long long nl_elems_per_cta) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_slot, s_lslot, s_cmd;
  __shared__ int s_ok[kMaxCluster];
  __shared__ long long s_got[1];
  __shared__ BoxDesc s_bd[kMaxBoxesPerItem];
  __shared__ WorkItem s_wi;
  const int csize = cluster_size(), crank = cluster_rank();
  const int tid = threadIdx.x;
  // a per-SM scratch slot for every CTA (one CTA per SM: a free one exists); the
  // cluster goes on only if every CTA has one, and runs big items in the leader's
  if (tid == 0) {
    int slot = -1;
    for (int k = 0; k < q.nslots && slot < 0; ++k) {  // bounded: one pass over the slots
      const int c = (int)((blockIdx.x + k) % q.nslots);
      if (atomicCAS(&q.slot_busy[c], 0, 1) == 0) slot = c;
    }
    if (slot >= 0) {
      reinterpret_cast<volatile int*>(q.alive)[slot] = 1;
      __threadfence_system();
    }
    s_slot = slot;
    const uint32_t ok_a = (uint32_t)__cvta_generic_to_shared(&s_ok[crank]);
    for (int rk = 0; rk < csize; ++rk) st_cluster_s32(cluster_map(ok_a, rk), slot >= 0 ? 1 : 0);
    if (crank == 0) {
      const uint32_t ls_a = (uint32_t)__cvta_generic_to_shared(&s_lslot);
      for (int rk = 0; rk < csize; ++rk) st_cluster_s32(cluster_map(ls_a, rk), slot);
    }
  }
  cluster_sync();
  bool all_ok = true;
  for (int rk = 0; rk < csize; ++rk) all_ok = all_ok && s_ok[rk] != 0;
  const int slot = s_slot;
  if (!all_ok) {  // the same decision in every CTA; no store into another CTA follows
    if (tid == 0 && slot >= 0) {
      reinterpret_cast<volatile int*>(q.alive)[slot] = 0;
      __threadfence_system();
      atomicExch(&q.slot_busy[slot], 0);
    }
    return;
  }
  uint16_t* nl_cta = nl_scratch + (long long)slot * nl_elems_per_cta;
  uint16_t* nl_lead = nl_scratch + (long long)s_lslot * nl_elems_per_cta;
  unsigned long long idle_since = clock_ns();
  __shared__ long long s_item;
  __shared__ int s_bigflag;     // leader: a big item is claimed for the next round
  __shared__ long long s_pend;  // leader: that item
  if (tid == 0) {
    s_bigflag = 0;
    s_pend = -1;
  }
  const uint32_t flag_lead = cluster_map((uint32_t)__cvta_generic_to_shared(&s_bigflag), 0);
  for (;;) {
    if (crank == 0 && tid == 0) {
      int cmd = kCmdExit;
      long long got = -1;
      if (s_pend >= 0) {  // claimed during the last small round
        cmd = kCmdBig;
        got = s_pend;
        s_pend = -1;
        s_bigflag = 0;
      }
      for (; cmd == kCmdExit;) {
        if (*reinterpret_cast<const volatile int*>(q.stop) != 0) break;
        const unsigned t = load_acquire_sys(q.tail);
        const unsigned h = *reinterpret_cast<volatile unsigned*>(q.head);
        if ((int)(t - h) > 0) {
          const int is_big =
              *reinterpret_cast<const volatile int*>(&q.items[h % q.cap_items].big) != 0;
          if (!is_big) {
            cmd = kCmdSmall;  // every CTA claims small items itself
            break;
          }
          if (atomicCAS(q.head, h, h + 1) == h) {
            cmd = kCmdBig;
            got = h;
            break;
          }
          continue;  // another cluster took item h: look at the next one
        }
        const unsigned long long idle = clock_ns() - idle_since;
        if (idle > (unsigned long long)q.max_idle_ns) break;
        if (idle > (unsigned long long)q.idle_ns &&
            *reinterpret_cast<const volatile int*>(q.linger) == 0)
          break;
        __nanosleep(2000);
      }
      const uint32_t cmd_a = (uint32_t)__cvta_generic_to_shared(&s_cmd);
      const uint32_t got_a = (uint32_t)__cvta_generic_to_shared(&s_got[0]);
      for (int rk = 0; rk < csize; ++rk) {
        st_cluster_s32(cluster_map(cmd_a, rk), cmd);
        st_cluster_s64(cluster_map(got_a, rk), got);
      }
    }
    cluster_sync();  // the round's command is in every CTA
    const int cmd = s_cmd;
    if (cmd == kCmdExit) break;
    if (cmd == kCmdBig) {
      if (tid == 0) {
        s_wi = q.items[(unsigned)s_got[0] % q.cap_items];
        s_bd[0] = q.boxes[(unsigned)s_wi.box[0] % q.cap_boxes];
      }
      __syncthreads();
      const BoxDesc& bd = s_bd[0];
      run_big(reinterpret_cast<unsigned char*>(nl_lead), reinterpret_cast<BigShared*>(smem), bd,
              rp, q.results + bd.out_index, crank, csize);
      if (crank == 0 && tid == 0) {  // the thread that wrote the result
        __threadfence_system();
        reinterpret_cast<volatile int*>(q.ready)[bd.out_index] = 1;
      }
    } else {  // small round: items of smaller boxes, claimed by each CTA
      const unsigned long long t_round = clock_ns();
      for (;;) {
        if (tid == 0) {
          long long it = -1;
          // ends: time up, the stop flag, this cluster's leader holding a big item,
          // queue empty, a small item claimed, or (leader) a big item claimed
          for (;;) {
            if (clock_ns() - t_round >= kRoundNs) break;
            if (*reinterpret_cast<const volatile int*>(q.stop) != 0) break;
            if (ld_cluster_s32(flag_lead) != 0) break;
            const unsigned t = load_acquire_sys(q.tail);
            const unsigned h = *reinterpret_cast<volatile unsigned*>(q.head);
            if ((int)(t - h) <= 0) break;
            if (*reinterpret_cast<const volatile int*>(&q.items[h % q.cap_items].big) != 0) {
              if (crank == 0 && atomicCAS(q.head, h, h + 1) == h) {
                s_pend = h;  // for this cluster's next round
                s_bigflag = 1;
                __threadfence_block();
                break;
              }
              __nanosleep(2000);  // a leader takes it
              continue;
            }
            if (atomicCAS(q.head, h, h + 1) == h) {
              it = h;
              break;
            }
          }
          s_item = it;
          if (it >= 0) {
            s_wi = q.items[(unsigned)it % q.cap_items];
            for (int k = 0; k < s_wi.nbox; ++k)
              s_bd[k] = q.boxes[(unsigned)s_wi.box[k] % q.cap_boxes];
          }
        }
        __syncthreads();
        if (s_item < 0) break;
        const WorkItem& wi = s_wi;
        const int ntb = wi.warps_per_box * 32;
        const int grp = tid / ntb;
        if (wi.big) {  // not claimed this way (big items go to a leader): alone
          run_big(reinterpret_cast<unsigned char*>(nl_cta), reinterpret_cast<BigShared*>(smem),
                  s_bd[0], rp, q.results + s_bd[0].out_index);
          if (tid == 0) {
            __threadfence_system();
            reinterpret_cast<volatile int*>(q.ready)[s_bd[0].out_index] = 1;
          }
        } else if (grp < wi.nbox) {
          const BoxDesc& bd = s_bd[grp];
          const Group g = make_group(smem + (size_t)grp * wi.smem_stride, tid - grp * ntb,
                                     wi.warps_per_box, wi.apt, wi.ncell_cap, 1 + grp,
                                     nl_cta + (long long)grp * wi.nl_stride);
          switch (wi.apt) {
            case 1: run_box_path<1>(g, bd, rp, q.results + bd.out_index); break;
            case 2: run_box_path<2>(g, bd, rp, q.results + bd.out_index); break;
            default: run_box_path<4>(g, bd, rp, q.results + bd.out_index); break;
          }
          if (g.tid == 0) {
            __threadfence_system();
            reinterpret_cast<volatile int*>(q.ready)[bd.out_index] = 1;
          }
        }
        __syncthreads();
      }
    }
    cluster_sync();  // the round is over in every CTA
    if (crank == 0 && tid == 0) idle_since = clock_ns();
  }
  if (tid == 0) {
    reinterpret_cast<volatile int*>(q.alive)[slot] = 0;
    __threadfence_system();
    atomicExch(&q.slot_busy[slot], 0);
  }
}

cudaError_t set_serve_cluster_attributes(int max_smem) {
  return cudaFuncSetAttribute(eos_serve_cluster_kernel,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

// grid: a multiple of cluster
cudaError_t launch_eos_serve_cluster(const ServeQueue& q, const RunParams& rp, uint16_t* nl,
                                     long long nl_elems_per_cta, int grid, int smem,
                                     cudaStream_t st, int cluster) {
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)grid, 1, 1);
  lc.blockDim = dim3(kCtaThreads, 1, 1);
  lc.dynamicSmemBytes = (size_t)smem;
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  return cudaLaunchKernelEx(&lc, eos_serve_cluster_kernel, q, rp, nl, nl_elems_per_cta);
}

}  // namespace mdeos
