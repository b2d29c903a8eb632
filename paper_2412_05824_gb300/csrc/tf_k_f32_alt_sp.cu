// float32 single-pass alternative shapes <real, NS, E, S, kind>: other
// radices (values per thread), threads per transform and transforms per
// block than the defaults, timed against them by the plan autotuner
#include "tf_instantiate.cuh"
namespace tf {
const KernelEntry* entries_f32_alt_sp(int* count) {
  static const KernelEntry t[] = {
      make_entry<Cfg<float, 16, 16, 64, KIND_SP>>(),   make_entry<Cfg<float, 16, 16, 128, KIND_SP>>(),
      make_entry<Cfg<float, 64, 16, 16, KIND_SP>>(),   make_entry<Cfg<float, 64, 8, 64, KIND_SP>>(),
      make_entry<Cfg<float, 128, 16, 32, KIND_SP>>(),  make_entry<Cfg<float, 128, 8, 16, KIND_SP>>(),
      make_entry<Cfg<float, 256, 16, 16, KIND_SP>>(),  make_entry<Cfg<float, 256, 8, 8, KIND_SP>>(),
      make_entry<Cfg<float, 512, 16, 8, KIND_SP>>(),   make_entry<Cfg<float, 1024, 16, 4, KIND_SP>>(),
      make_entry<Cfg<float, 2048, 16, 2, KIND_SP>>(),  make_entry<Cfg<float, 4096, 8, 1, KIND_SP>>(),
      // one thread per transform (also the shape of thread-level checksums)
      make_entry<Cfg<float, 32, 32, 64, KIND_SP>>(),
      // fewer transforms per block, for small batches (more blocks in flight)
      make_entry<Cfg<float, 128, 16, 8, KIND_SP>>(),   make_entry<Cfg<float, 256, 16, 4, KIND_SP>>(),
      make_entry<Cfg<float, 256, 16, 2, KIND_SP>>(),   make_entry<Cfg<float, 512, 16, 2, KIND_SP>>(),
      make_entry<Cfg<float, 1024, 16, 1, KIND_SP>>(),
  };
  *count = sizeof(t) / sizeof(t[0]);
  return t;
}
}  // namespace tf
