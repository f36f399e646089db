// Batch evaluation that allocates no device memory.
//
// Some callers cannot allocate device memory at the point where they need an
// equation-of-state answer: a hydrocode's material-model callback invoked
// inside its own time step (where cudaMalloc would synchronise the whole device
// and stall the caller's other streams), or code running under a memory pool that
// owns all device memory.  This entry point serves them: the caller passes the
// requests and a device result array, and every other byte the persistent kernel
// needs -- the work table, the queue counter and the Verlet lists -- lives in one
// static device array below.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "mdeos_device.cuh"

namespace mdeos {

// Static scratch of the no-allocation entry point.  Every GPU that loads the
// library holds these bytes until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(128) << 20;  // 128 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Same persistent batch loop as eos_batch_kernel; every pointer it uses beyond
// the caller's results points into the static scratch array.
__global__ void __launch_bounds__(kCtaThreads, 1)
    eos_batch_static_kernel(unsigned char* scratch, long long off_items, long long off_counter,
                            long long off_nl, int nitems, mdeos_result* results,
                            long long nl_elems_per_cta, RunParams rp) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_item;
  const BoxDesc* boxes = reinterpret_cast<const BoxDesc*>(scratch);
  const WorkItem* items = reinterpret_cast<const WorkItem*>(scratch + off_items);
  int* counter = reinterpret_cast<int*>(scratch + off_counter);
  uint16_t* nl_cta = reinterpret_cast<uint16_t*>(scratch + off_nl) +
                     (long long)blockIdx.x * nl_elems_per_cta;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= nitems) break;
    const WorkItem wi = items[it];
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

// Host side: per-device address of the static array, resolved once.
struct NoAllocDevice {
  bool ready = false;
  unsigned char* ptr = nullptr;
  int nsm = 0, smem_max = 0;
};
static std::mutex g_noalloc_mu;
static NoAllocDevice g_noalloc_dev[64];

}  // namespace mdeos

namespace mdeos {
// Planner and error helpers of the host engine (mdeos_api.cu); host memory only.
mdeos_status plan_for_noalloc(const mdeos_request* reqs, int n, const mdeos_config& c, int nsm,
                              int smem_max, std::vector<BoxDesc>& boxes,
                              std::vector<WorkItem>& items, std::vector<mdeos_result>& init,
                              int& grid, int& smem, long long& nl_per_cta, RunParams& rp);
mdeos_status set_error(mdeos_status st, const std::string& msg);
}  // namespace mdeos

using namespace mdeos;

extern "C" mdeos_status mdeos_submit_noalloc(const mdeos_config* cfg, const mdeos_request* reqs,
                                             int32_t n, mdeos_result* d_results, void* stream) {
  if (!cfg || !reqs || !d_results || n < 1)
    return set_error(MDEOS_EINVAL, "bad mdeos_submit_noalloc arguments");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(MDEOS_ECUDA, "no CUDA device available");
  if (cfg->device != dev)
    return set_error(MDEOS_EINVAL, "cfg->device must be the current device");
  if (dev < 0 || dev >= 64) return set_error(MDEOS_EINVAL, "device ordinal out of range");
  NoAllocDevice& d = g_noalloc_dev[dev];
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!d.ready) {  // once per device, with that device current
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess)
        return set_error(MDEOS_ECUDA, std::string("cudaGetSymbolAddress: ") +
                                                cudaGetErrorString(e));
      cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev);
      cudaDeviceGetAttribute(&d.smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      d.smem_max -= 1024;
      e = cudaFuncSetAttribute(eos_batch_static_kernel,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, d.smem_max);
      if (e != cudaSuccess)
        return set_error(MDEOS_ECUDA, std::string("kernel attribute: ") +
                                                cudaGetErrorString(e));
      d.ptr = static_cast<unsigned char*>(p);
      d.ready = true;
    }
  }
  std::vector<BoxDesc> boxes;
  std::vector<WorkItem> items;
  std::vector<mdeos_result> init;
  int grid = 0, smem = 0;
  long long nl_per_cta = 0;
  RunParams rp;
  mdeos_status st = plan_for_noalloc(reqs, n, *cfg, d.nsm, d.smem_max, boxes, items, init, grid,
                                     smem, nl_per_cta, rp);
  if (st != MDEOS_OK) return st;
  // layout inside the static array: boxes | items | counter | Verlet lists
  const size_t off_items = (boxes.size() * sizeof(BoxDesc) + 255) & ~size_t(255);
  const size_t off_counter = (off_items + items.size() * sizeof(WorkItem) + 255) & ~size_t(255);
  const size_t off_nl = off_counter + 256;
  const size_t per_cta = (size_t)nl_per_cta * sizeof(uint16_t);
  if (off_nl > kNoAllocScratchBytes ||
      (per_cta > 0 && off_nl + per_cta > kNoAllocScratchBytes))
    return set_error(MDEOS_EINVAL,
                           "batch exceeds the 128 MiB static scratch of mdeos_submit_noalloc "
                           "(work table plus one CTA's Verlet lists); split it");
  if (per_cta > 0) grid = std::min<long long>(grid, (kNoAllocScratchBytes - off_nl) / per_cta);
  cudaStream_t s = (cudaStream_t)stream;
  // The host tables below are pageable vectors freed on return: a copy recorded
  // into a graph would read freed memory at replay.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess)
    return set_error(MDEOS_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  if (cap != cudaStreamCaptureStatusNone)
    return set_error(MDEOS_EINVAL, "mdeos_submit_noalloc cannot be called on a capturing stream");
  // requests rejected by the planner get their status from the host copy; the
  // kernel overwrites every planned box
  e = cudaMemcpyAsync(d_results, init.data(), (size_t)n * sizeof(mdeos_result),
                      cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !items.empty()) {
    e = cudaMemcpyAsync(d.ptr, boxes.data(), boxes.size() * sizeof(BoxDesc),
                        cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d.ptr + off_items, items.data(), items.size() * sizeof(WorkItem),
                          cudaMemcpyHostToDevice, s);
    // the queue counter keeps the previous call's value: clear it
    if (e == cudaSuccess) e = cudaMemsetAsync(d.ptr + off_counter, 0, sizeof(int), s);
    if (e == cudaSuccess) {
      eos_batch_static_kernel<<<grid, kCtaThreads, smem, s>>>(
          d.ptr, (long long)off_items, (long long)off_counter, (long long)off_nl,
          (int)items.size(), d_results, nl_per_cta, rp);
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess)
    return set_error(MDEOS_ECUDA, std::string("mdeos_submit_noalloc: ") +
                                            cudaGetErrorString(e));
  return MDEOS_OK;
}
