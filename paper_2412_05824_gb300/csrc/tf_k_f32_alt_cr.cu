// float32 four-step alternative shapes <real, sub-length, E, columns/rows, kind>
// for the sub-lengths of N = 2^14..2^16, timed against the defaults by the
// plan autotuner
#include "tf_instantiate.cuh"
namespace tf {
const KernelEntry* entries_f32_alt_cr(int* count) {
  static const KernelEntry t[] = {
      make_entry<Cfg<float, 128, 16, 8, KIND_COL>>(),  make_entry<Cfg<float, 128, 16, 32, KIND_COL>>(),
      make_entry<Cfg<float, 256, 16, 16, KIND_COL>>(), make_entry<Cfg<float, 256, 16, 4, KIND_COL>>(),
      make_entry<Cfg<float, 128, 16, 8, KIND_ROW>>(),  make_entry<Cfg<float, 128, 16, 32, KIND_ROW>>(),
      make_entry<Cfg<float, 256, 16, 16, KIND_ROW>>(), make_entry<Cfg<float, 256, 16, 4, KIND_ROW>>(),
  };
  *count = sizeof(t) / sizeof(t[0]);
  return t;
}
}  // namespace tf
