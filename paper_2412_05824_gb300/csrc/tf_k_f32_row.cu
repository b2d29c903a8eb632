// float32 four-step second-pass (row) configurations: <real, N2, E, rows, kind>
#include "tf_instantiate.cuh"
namespace tf {
const KernelEntry* entries_f32_row(int* count) {
  static const KernelEntry t[] = {
      make_entry<Cfg<float, 128, 16, 16, KIND_ROW>>(),  make_entry<Cfg<float, 256, 16, 8, KIND_ROW>>(),
      make_entry<Cfg<float, 512, 16, 8, KIND_ROW>>() ,  make_entry<Cfg<float, 1024, 16, 8, KIND_ROW>>(),
      make_entry<Cfg<float, 2048, 16, 4, KIND_ROW>>(),  make_entry<Cfg<float, 4096, 16, 2, KIND_ROW>>(),
  };
  *count = sizeof(t) / sizeof(t[0]);
  return t;
}
}  // namespace tf
