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
                     uint16_t* nl_scratch, long long nl_elems_per_cta, RunParams rp) {
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
    }
    __syncthreads();
  }
}

cudaError_t set_batch_attributes(int max_smem) {
  return cudaFuncSetAttribute(eos_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              max_smem);
}

cudaError_t launch_eos_batch(const BoxDesc* boxes, const WorkItem* items, int nitems, int* counter,
                             mdeos_result* results, uint16_t* nl, long long nl_elems_per_cta,
                             const RunParams& rp, int grid, int smem, cudaStream_t st) {
  eos_batch_kernel<<<grid, kCtaThreads, smem, st>>>(boxes, items, nitems, counter, results, nl,
                                                    nl_elems_per_cta, rp);
  return cudaGetLastError();
}

}  // namespace mdeos
