// Persistent batch kernel of the atomistic EOS path: one 1024-thread CTA per
// SM pulls work items (up to 8 boxes of one size class) from an atomic queue
// ordered by decreasing cost, and runs every box of the item concurrently in
// its own warp group (arXiv 2508.06012, Sec. III: one independent MD run per
// element and call).
#include "mdeos_big.cuh"

namespace mdeos {

__global__ void __launch_bounds__(kCtaThreads, 1)
    eos_batch_kernel(const BoxDesc* __restrict__ boxes, const WorkItem* __restrict__ items,
                     int nitems, int* __restrict__ counter, mdeos_result* __restrict__ results,
                     uint16_t* nl_scratch, long long nl_elems_per_cta, RunParams rp, int* ready) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_item;
  uint16_t* nl_cta = nl_scratch + (long long)blockIdx.x * nl_elems_per_cta;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= nitems) break;
    const WorkItem wi = items[it];
    if (wi.big) {  // one box above the shared-memory limit, the whole CTA
      const BoxDesc& bd = boxes[wi.box[0]];
      run_big(reinterpret_cast<unsigned char*>(nl_cta), reinterpret_cast<BigShared*>(smem), bd, rp,
              results + bd.out_index);
      if (ready != nullptr && threadIdx.x == 0) {  // the thread that wrote the result
        __threadfence_system();
        reinterpret_cast<volatile int*>(ready)[bd.out_index] = 1;
      }
      continue;
    }
    const int ntb = wi.warps_per_box * 32;
    const int grp = threadIdx.x / ntb;
    if (grp < wi.nbox) {
      const BoxDesc& bd = boxes[wi.box[grp]];
      const Group g = make_group(smem + (size_t)grp * wi.smem_stride, threadIdx.x - grp * ntb,
                                 wi.warps_per_box, wi.apt, wi.ncell_cap, 1 + grp,
                                 nl_cta + (long long)grp * wi.nl_stride);
      mdeos_result* out = results + bd.out_index;
      switch (wi.apt) {
        case 1: run_box_path<1>(g, bd, rp, out); break;
        case 2: run_box_path<2>(g, bd, rp, out); break;
        default: run_box_path<4>(g, bd, rp, out); break;
      }
      // per-box completion flag for host pollers (results in host-mapped memory):
      // the group's thread 0 wrote the result, fences it, then raises the flag
      if (ready != nullptr && g.tid == 0) {
        __threadfence_system();
        reinterpret_cast<volatile int*>(ready)[bd.out_index] = 1;
      }
    }
    __syncthreads();
  }
}

// Cluster form for batches too small to fill the GPU: one box per thread-block
// cluster of csize CTAs (cluster c runs item c, one box, the whole CTA as its group).
// Shared-memory boxes: every CTA holds the box and advances it alike; each computes
// the forces and lists of its share of the atoms and sends the forces to the others
// (run_box with Group::csize > 1).  Boxes above the shared-memory limit: one state in
// the scratch of the cluster's first CTA, each CTA owning a slab of its slots
// (run_big with csize > 1).  All CTAs of a cluster take the same path through the
// box, so they meet at the same cluster barriers; the last one below keeps every CTA
// alive until no other can still store into its shared memory.
__global__ void __launch_bounds__(kCtaThreads, 1)
    eos_cluster_kernel(const BoxDesc* __restrict__ boxes, const WorkItem* __restrict__ items,
                       int nitems, mdeos_result* __restrict__ results, uint16_t* nl_scratch,
                       long long nl_elems_per_cta, RunParams rp, int* ready) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int csize = cluster_size(), crank = cluster_rank();
  const int it = blockIdx.x / csize;
  uint16_t* nl_cta = nl_scratch + (long long)blockIdx.x * nl_elems_per_cta;
  if (it < nitems && items[it].big) {
    const BoxDesc& bd = boxes[items[it].box[0]];
    uint16_t* box_scratch = nl_scratch + (long long)(blockIdx.x - crank) * nl_elems_per_cta;
    run_big(reinterpret_cast<unsigned char*>(box_scratch), reinterpret_cast<BigShared*>(smem), bd,
            rp, results + bd.out_index, crank, csize);
    if (ready != nullptr && crank == 0 && threadIdx.x == 0) {
      __threadfence_system();
      reinterpret_cast<volatile int*>(ready)[bd.out_index] = 1;
    }
  } else if (it < nitems) {
    const WorkItem wi = items[it];
    const BoxDesc& bd = boxes[wi.box[0]];
    Group g = make_group(smem, threadIdx.x, wi.warps_per_box, wi.apt, wi.ncell_cap, 1, nl_cta);
    g.crank = crank;
    g.csize = csize;
    mdeos_result* out = results + bd.out_index;
    switch (wi.apt) {
      case 1: run_box_path<1>(g, bd, rp, out); break;
      case 2: run_box_path<2>(g, bd, rp, out); break;
      default: run_box_path<4>(g, bd, rp, out); break;
    }
    if (ready != nullptr && crank == 0 && g.tid == 0) {
      __threadfence_system();
      reinterpret_cast<volatile int*>(ready)[bd.out_index] = 1;
    }
  }
  cluster_sync();
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_sys(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Continuous-batching form of eos_batch_kernel: CTAs claim work items one at a
// time from a queue the host keeps appending to (published with a release store
// of the tail, read here with an acquire load), copy the item's box descriptors
// into shared memory, run them and raise per-box ready flags.  Waiting for work is
// bounded: a CTA exits on the stop flag, after idle_ns without work once the host
// clears `linger` (traffic over), and after max_idle_ns in any case; the host
// launches more CTAs when work outnumbers the live ones.  Each CTA holds
// one of nslots per-SM scratch slots (at most one CTA is resident per SM, so a
// free slot exists whenever a CTA starts) and shows it in the host-mapped
// alive array.
__global__ void __launch_bounds__(kCtaThreads, 1)
    eos_serve_kernel(ServeQueue q, RunParams rp, uint16_t* nl_scratch, long long nl_elems_per_cta) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ long long s_item;
  __shared__ int s_slot;
  __shared__ BoxDesc s_bd[kMaxBoxesPerItem];
  __shared__ WorkItem s_wi;
  if (threadIdx.x == 0) {
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
  }
  __syncthreads();
  const int slot = s_slot;
  if (slot < 0) return;
  uint16_t* nl_cta = nl_scratch + (long long)slot * nl_elems_per_cta;
  unsigned long long idle_since = global_ns();
  for (;;) {
    if (threadIdx.x == 0) {
      long long got = -1;
      for (;;) {
        if (*reinterpret_cast<const volatile int*>(q.stop) != 0) break;
        const unsigned t = ld_acquire_sys(q.tail);
        const unsigned h = *reinterpret_cast<volatile unsigned*>(q.head);
        if ((int)(t - h) > 0) {
          if (atomicCAS(q.head, h, h + 1) == h) {
            got = h;
            break;
          }
          continue;  // another CTA took item h: try the next one
        }
        const unsigned long long idle = global_ns() - idle_since;
        if (idle > (unsigned long long)q.max_idle_ns) break;
        if (idle > (unsigned long long)q.idle_ns &&
            *reinterpret_cast<const volatile int*>(q.linger) == 0)
          break;
        __nanosleep(2000);
      }
      s_item = got;
      if (got >= 0) {
        s_wi = q.items[(unsigned)got % q.cap_items];
        for (int k = 0; k < s_wi.nbox; ++k) s_bd[k] = q.boxes[(unsigned)s_wi.box[k] % q.cap_boxes];
      }
    }
    __syncthreads();
    const long long it = s_item;
    if (it < 0) break;
    const WorkItem& wi = s_wi;
    if (wi.big) {
      const BoxDesc& bd = s_bd[0];
      run_big(reinterpret_cast<unsigned char*>(nl_cta), reinterpret_cast<BigShared*>(smem), bd, rp,
              q.results + bd.out_index);
      if (threadIdx.x == 0) {
        __threadfence_system();
        reinterpret_cast<volatile int*>(q.ready)[bd.out_index] = 1;
      }
    } else {
      const int ntb = wi.warps_per_box * 32;
      const int grp = threadIdx.x / ntb;
      if (grp < wi.nbox) {
        const BoxDesc& bd = s_bd[grp];
        const Group g = make_group(smem + (size_t)grp * wi.smem_stride, threadIdx.x - grp * ntb,
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
    }
    __syncthreads();
    if (threadIdx.x == 0) idle_since = global_ns();
  }
  if (threadIdx.x == 0) {
    reinterpret_cast<volatile int*>(q.alive)[slot] = 0;
    __threadfence_system();
    atomicExch(&q.slot_busy[slot], 0);
  }
}

cudaError_t set_batch_attributes(int max_smem) {
  cudaError_t e = cudaFuncSetAttribute(eos_serve_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(eos_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           max_smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(eos_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              max_smem);
}

cudaError_t launch_eos_serve(const ServeQueue& q, const RunParams& rp, uint16_t* nl,
                             long long nl_elems_per_cta, int grid, int smem, cudaStream_t st) {
  eos_serve_kernel<<<grid, kCtaThreads, smem, st>>>(q, rp, nl, nl_elems_per_cta);
  return cudaGetLastError();
}

cudaError_t launch_eos_batch(const BoxDesc* boxes, const WorkItem* items, int nitems, int* counter,
                             mdeos_result* results, uint16_t* nl, long long nl_elems_per_cta,
                             const RunParams& rp, int grid, int smem, cudaStream_t st, int* ready,
                             int cluster) {
  if (cluster > 1) {  // grid = nitems * cluster CTAs in clusters of `cluster`
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
    return cudaLaunchKernelEx(&lc, eos_cluster_kernel, boxes, items, nitems, results, nl,
                              nl_elems_per_cta, rp, ready);
  }
  eos_batch_kernel<<<grid, kCtaThreads, smem, st>>>(boxes, items, nitems, counter, results, nl,
                                                    nl_elems_per_cta, rp, ready);
  return cudaGetLastError();
}

}  // namespace mdeos
