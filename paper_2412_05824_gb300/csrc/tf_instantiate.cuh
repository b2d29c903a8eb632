// Instantiation helpers: one KernelEntry per compile-time configuration.
#pragma once

#include "tf_device.cuh"
#include "tf_registry.h"

namespace tf {

template <class K> void launch_plain(const void* a, int grid, cudaStream_t s) {
  tf_pass_kernel<K, false><<<grid, K::NT, pass_smem_bytes<K>(), s>>>(
      *static_cast<const PassArgs<typename K::real>*>(a));
}
template <class K> void launch_ft(const void* a, int grid, cudaStream_t s) {
  tf_pass_kernel<K, true><<<grid, K::NT, pass_smem_bytes<K>(), s>>>(
      *static_cast<const PassArgs<typename K::real>*>(a));
}
template <class K> void launch_fix(const void* a, int grid, cudaStream_t s) {
  tf_fix_kernel<K><<<grid, K::NT, K::SMEM_BYTES, s>>>(*static_cast<const PassArgs<typename K::real>*>(a));
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
  e.smem_main = pass_smem_bytes<K>();
  e.smem_fix = K::SMEM_BYTES;
  e.main_plain = &launch_plain<K>;
  e.main_ft = &launch_ft<K>;
  e.fix = &launch_fix<K>;
  e.fn_plain = reinterpret_cast<const void*>(&tf_pass_kernel<K, false>);
  e.fn_ft = reinterpret_cast<const void*>(&tf_pass_kernel<K, true>);
  e.fn_fix = reinterpret_cast<const void*>(&tf_fix_kernel<K>);
  return e;
}

}  // namespace tf
