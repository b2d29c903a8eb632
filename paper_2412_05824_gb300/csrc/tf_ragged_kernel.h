// Shared definitions of the persistent ragged kernel (tf_ragged_kernel.cu)
// and its host side (tf_ragged.cu).
#pragma once

#include <cuda_runtime.h>

#include "tf_device.cuh"

struct turbofft_plan;

namespace tf {

constexpr int kRgThreads = 256;  // threads per block of every size class
constexpr int kRgClasses = 15;
constexpr int kRgMaxPasses = 24;  // (member, pass) entries of one ragged plan

// a size class: kernel configuration and its shared-memory needs
struct RgClassInfo {
  int kind, ns, e, s;
  int smem_plain, smem_ft, smem_fix;
};

// queue counters, grid-barrier state and the timeout flag of one exec
// (cleared before every launch)
struct RgCtl {
  unsigned long long head[2];
  unsigned int bar_count;
  unsigned int bar_gen;
  int error;
  int pad;
};

// one pass of one member plan, run by size class `cls` in phase `phase`
struct RgPassArgs {
  PassArgs<float> A;
  int cls;
  int phase;
};

// a work item: units [u0, u1) of pass entry `ca`
struct RgItem {
  int ca;
  int pad;
  long long u0, u1;
};

struct RgParams {
  RgPassArgs ca[kRgMaxPasses];
  int num_ca;
  int num_phases;
  long long num_items[2];
  const RgItem* items[2];
  RgCtl* ctl;
};

const RgClassInfo* ragged_classes();          // kRgClasses entries
const void* ragged_kernel_fn(int ftm);        // for occupancy queries
cudaError_t launch_ragged_kernel(int ftm, const RgParams& P, int grid, size_t smem, cudaStream_t s);

}  // namespace tf

namespace tfh {
// the kernel arguments of pass pi of a float32 plan (tf_launch.cu)
void fill_pass_args_f32(const turbofft_plan* p, int pi, const void* in, void* out, const tf::InjectSite& inj,
                        tf::PassArgs<float>* A);
}  // namespace tfh
