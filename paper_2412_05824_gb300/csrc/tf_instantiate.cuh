// Instantiation helpers: one KernelEntry per compile-time configuration.
#pragma once

#include "tf_device.cuh"
#include "tf_registry.h"

namespace tf {

template <class K, int FTM> void launch_main(const void* a, int grid, cudaStream_t s) {
  tf_pass_kernel<K, FTM><<<grid, K::NT, pass_smem_bytes<K, FTM>(), s>>>(
      *static_cast<const PassArgs<typename K::real>*>(a));
}
template <class K, int FTM> void launch_main_tma(const void* a, const void* tm, int grid, cudaStream_t s) {
  tf_pass_kernel_tma<K, FTM><<<grid, K::NT, tma_smem_bytes<K>(FTM), s>>>(
      *static_cast<const PassArgs<typename K::real>*>(a), *static_cast<const CUtensorMap*>(tm));
}
template <class K> void set_tma(KernelEntry& e) {
  if constexpr (tma_ok<K>()) {
    e.smem_tma[0] = tma_smem_bytes<K>(0);
    e.smem_tma[1] = tma_smem_bytes<K>(1);
    e.main_tma[0] = &launch_main_tma<K, 0>;
    e.main_tma[1] = &launch_main_tma<K, 1>;
    e.fn_main_tma[0] = reinterpret_cast<const void*>(&tf_pass_kernel_tma<K, 0>);
    e.fn_main_tma[1] = reinterpret_cast<const void*>(&tf_pass_kernel_tma<K, 1>);
  } else {
    for (int v = 0; v < 2; ++v) {
      e.smem_tma[v] = 0;
      e.main_tma[v] = nullptr;
      e.fn_main_tma[v] = nullptr;
    }
  }
}
template <class K> void launch_fix(const void* a, int grid, cudaStream_t s) {
  tf_fix_kernel<K><<<grid, K::NT, K::SMEM_BYTES, s>>>(*static_cast<const PassArgs<typename K::real>*>(a));
}
template <class K> void launch_tcfix(const void* a, int grid, cudaStream_t s) {
  tf_tc_fix_kernel<K><<<grid, K::NT, pass_smem_bytes<K, 0>(), s>>>(*static_cast<const PassArgs<typename K::real>*>(a));
}
template <class K> constexpr bool transform_level_ok() {
  return std::is_same<typename K::real, double>::value && K::KIND != KIND_SP;
}

template <class K> KernelEntry make_entry() {
  KernelEntry e;
  e.dtype = sizeof(typename K::real) == 4 ? 0 : 1;
  e.kind = K::KIND;
  e.ns = K::NS;
  e.e = K::E;
  e.s = K::S;
  e.nt = K::NT;
  e.stages = K::NP;
  e.smem_main[0] = pass_smem_bytes<K, 0>();
  e.smem_main[1] = pass_smem_bytes<K, 1>();
  e.smem_main[2] = pass_smem_bytes<K, 2>();
  e.smem_fix = K::SMEM_BYTES;
  e.main[0] = &launch_main<K, 0>;
  e.main[1] = &launch_main<K, 1>;
  e.main[2] = &launch_main<K, 2>;
  e.fix = &launch_fix<K>;
  e.fn_main[0] = reinterpret_cast<const void*>(&tf_pass_kernel<K, 0>);
  e.fn_main[1] = reinterpret_cast<const void*>(&tf_pass_kernel<K, 1>);
  e.fn_main[2] = reinterpret_cast<const void*>(&tf_pass_kernel<K, 2>);
  e.fn_fix = reinterpret_cast<const void*>(&tf_fix_kernel<K>);
  // thread-level checksums exist where one thread holds a whole transform
  if constexpr (thread_level_ok<K>()) {
    e.smem_main[3] = pass_smem_bytes<K, 3>();
    e.main[3] = &launch_main<K, 3>;
    e.fn_main[3] = reinterpret_cast<const void*>(&tf_pass_kernel<K, 3>);
  } else {
    e.smem_main[3] = 0;
    e.main[3] = nullptr;
    e.fn_main[3] = nullptr;
  }
  // transform-level checksums of float64 two-pass plans
  if constexpr (transform_level_ok<K>()) {
    e.smem_main[4] = pass_smem_bytes<K, 4>();
    e.main[4] = &launch_main<K, 4>;
    e.fn_main[4] = reinterpret_cast<const void*>(&tf_pass_kernel<K, 4>);
    e.tcfix = &launch_tcfix<K>;
    e.fn_tcfix = reinterpret_cast<const void*>(&tf_tc_fix_kernel<K>);
  } else {
    e.smem_main[4] = 0;
    e.main[4] = nullptr;
    e.fn_main[4] = nullptr;
    e.tcfix = nullptr;
    e.fn_tcfix = nullptr;
  }
  set_tma<K>(e);
  return e;
}

// Float-pair plans have no checksums: only the plain transform kernel.
template <class K> KernelEntry make_entry_plain() {
  KernelEntry e;
  e.dtype = 2;
  e.kind = K::KIND;
  e.ns = K::NS;
  e.e = K::E;
  e.s = K::S;
  e.nt = K::NT;
  e.stages = K::NP;
  e.smem_main[0] = pass_smem_bytes<K, 0>();
  e.main[0] = &launch_main<K, 0>;
  e.fn_main[0] = reinterpret_cast<const void*>(&tf_pass_kernel<K, 0>);
  e.tcfix = nullptr;
  e.fn_tcfix = nullptr;
  for (int v = 1; v < 5; ++v) {
    e.smem_main[v] = 0;
    e.main[v] = nullptr;
    e.fn_main[v] = nullptr;
  }
  e.smem_fix = 0;
  e.fix = nullptr;
  e.fn_fix = nullptr;
  for (int v = 0; v < 2; ++v) {
    e.smem_tma[v] = 0;
    e.main_tma[v] = nullptr;
    e.fn_main_tma[v] = nullptr;
  }
  return e;
}

}  // namespace tf
