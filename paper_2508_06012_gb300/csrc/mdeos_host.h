// Host-side declarations shared by the translation units of the library (the
// planner and handle accessors live in mdeos_api.cu).  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "mdeos_internal.h"

namespace mdeos {

// A planned batch: boxes, work items (LPT order), per-request planning status,
// launch shape and per-CTA neighbour scratch (uint16 entries).
struct PlanOut {
  std::vector<BoxDesc> boxes;
  std::vector<WorkItem> items;
  std::vector<int> status;
  int smem = 0;
  int grid = 0;
  long long nl_per_cta = 0;
  int cluster = 1;  // CTAs per box (thread-block clusters); 1: the persistent kernel
};

mdeos_status set_error(mdeos_status st, const std::string& msg);
mdeos_status plan_requests(const mdeos_handle* h, const mdeos_request* reqs, int n, PlanOut& out,
                           const int* cap_min = nullptr);
void planning_result_of(mdeos_result& r, int status, const mdeos_request& q);
cudaStream_t handle_stream(const mdeos_handle* h);
int handle_device(const mdeos_handle* h);
const mdeos_config& handle_config(const mdeos_handle* h);
const RunParams& handle_run_params(const mdeos_handle* h);
void count_launch(mdeos_handle* h, long long k);
mdeos_status eval_into_device(mdeos_handle* h, const mdeos_request* reqs, int n,
                              mdeos_result* d_results);
cudaError_t launch_eos_batch(const BoxDesc* boxes, const WorkItem* items, int nitems, int* counter,
                             mdeos_result* results, uint16_t* nl, long long nl_elems_per_cta,
                             const RunParams& rp, int grid, int smem, cudaStream_t st,
                             int* ready, int cluster = 1);

cudaError_t launch_eos_serve(const ServeQueue& q, const RunParams& rp, uint16_t* nl,
                             long long nl_elems_per_cta, int grid, int smem, cudaStream_t st);
int handle_sm_count(const mdeos_handle* h);
int handle_smem_max(const mdeos_handle* h);

}  // namespace mdeos
