// float64 four-step second-pass (row) configurations: <real, N2, E, rows, kind>
#include "tf_instantiate.cuh"
namespace tf {
const KernelEntry* entries_f64_row(int* count) {
  static const KernelEntry t[] = {
      make_entry<Cfg<double, 64, 8, 8, KIND_ROW>>(),    make_entry<Cfg<double, 128, 8, 8, KIND_ROW>>(),   make_entry<Cfg<double, 256, 8, 8, KIND_ROW>>(),
      make_entry<Cfg<double, 512, 8, 4, KIND_ROW>>(),   make_entry<Cfg<double, 1024, 8, 2, KIND_ROW>>(),
      make_entry<Cfg<double, 2048, 8, 1, KIND_ROW>>(),  make_entry<Cfg<double, 4096, 8, 1, KIND_ROW>>(),
  };
  *count = sizeof(t) / sizeof(t[0]);
  return t;
}
}  // namespace tf
