// float64 single-pass configurations: <real, NS, E, S, kind>
#include "tf_instantiate.cuh"
namespace tf {
const KernelEntry* entries_f64_sp(int* count) {
  static const KernelEntry t[] = {
      make_entry<Cfg<double, 8, 8, 256, KIND_SP>>(),    make_entry<Cfg<double, 16, 8, 128, KIND_SP>>(),
      make_entry<Cfg<double, 32, 8, 64, KIND_SP>>(),    make_entry<Cfg<double, 64, 8, 32, KIND_SP>>(),
      make_entry<Cfg<double, 128, 8, 16, KIND_SP>>(),   make_entry<Cfg<double, 256, 8, 8, KIND_SP>>(),
      make_entry<Cfg<double, 512, 8, 2, KIND_SP>>(),    make_entry<Cfg<double, 1024, 8, 1, KIND_SP>>(),
      make_entry<Cfg<double, 2048, 8, 1, KIND_SP>>(),   make_entry<Cfg<double, 4096, 8, 1, KIND_SP>>(),

  };
  *count = sizeof(t) / sizeof(t[0]);
  return t;
}
}  // namespace tf
