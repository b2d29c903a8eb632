// float32 single-pass configurations: <real, NS, E, S, kind>
// (shapes chosen by sweeping E and S on GB300 at 2^26 elements)
#include "tf_instantiate.cuh"
namespace tf {
const KernelEntry* entries_f32_sp(int* count) {
  static const KernelEntry t[] = {
      make_entry<Cfg<float, 8, 8, 64, KIND_SP>>(),      make_entry<Cfg<float, 16, 8, 64, KIND_SP>>(),
      make_entry<Cfg<float, 32, 8, 32, KIND_SP>>(),     make_entry<Cfg<float, 64, 8, 32, KIND_SP>>(),
      make_entry<Cfg<float, 128, 16, 16, KIND_SP>>(),   make_entry<Cfg<float, 256, 16, 8, KIND_SP>>(),
      make_entry<Cfg<float, 512, 16, 4, KIND_SP>>(),    make_entry<Cfg<float, 1024, 16, 2, KIND_SP>>(),
      make_entry<Cfg<float, 2048, 16, 1, KIND_SP>>(),   make_entry<Cfg<float, 4096, 16, 1, KIND_SP>>(),
      make_entry<Cfg<float, 8192, 16, 1, KIND_SP>>(),
  };
  *count = sizeof(t) / sizeof(t[0]);
  return t;
}
}  // namespace tf
