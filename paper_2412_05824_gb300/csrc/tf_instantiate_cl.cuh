// Instantiation helpers of the cluster kernels: one ClEntry per configuration.
#pragma once

#include "tf_cluster.cuh"
#include "tf_registry.h"

namespace tf {

template <class CL, int FTM> void launch_cl(const void* a, int grid, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(CL::NT);
  cfg.dynamicSmemBytes = (size_t)cl_smem_bytes<CL>(FTM);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL::C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, tf_cl_kernel<CL, FTM>, *static_cast<const ClArgs<typename CL::real>*>(a));
}
template <class CL> void launch_cl_fix(const void* a, int grid, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(CL::NT);
  cfg.dynamicSmemBytes = (size_t)cl_smem_bytes<CL>(1);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL::C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, tf_cl_fix_kernel<CL>, *static_cast<const ClArgs<typename CL::real>*>(a));
}

template <class CL> ClEntry make_cl_entry() {
  ClEntry e;
  e.dtype = sizeof(typename CL::real) == 4 ? 0 : 1;
  e.n = (int)CL::N;
  e.n1 = CL::N1;
  e.n2 = CL::N2;
  e.e = CL::KA::E;
  e.sa = CL::SA;
  e.sb = CL::SB;
  e.cluster = CL::C;
  e.nt = CL::NT;
  e.stages_a = CL::KA::NP;
  e.stages_b = CL::KB::NP;
  e.smem[0] = cl_smem_bytes<CL>(0);
  e.smem[1] = cl_smem_bytes<CL>(1);
  e.main[0] = &launch_cl<CL, 0>;
  e.main[1] = &launch_cl<CL, 1>;
  e.fix = &launch_cl_fix<CL>;
  e.fn_main[0] = reinterpret_cast<const void*>(&tf_cl_kernel<CL, 0>);
  e.fn_main[1] = reinterpret_cast<const void*>(&tf_cl_kernel<CL, 1>);
  e.fn_fix = reinterpret_cast<const void*>(&tf_cl_fix_kernel<CL>);
  return e;
}

}  // namespace tf
