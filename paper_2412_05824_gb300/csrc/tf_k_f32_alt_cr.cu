// float32 four-step alternative shapes <real, sub-length, E, columns/rows, kind>
// for the sub-lengths of N = 2^14..2^24, timed against the defaults by the
// plan autotuner
#include "tf_instantiate.cuh"
namespace tf {
const KernelEntry* entries_f32_alt_cr(int* count) {
  static const KernelEntry t[] = {
      make_entry<Cfg<float, 128, 16, 8, KIND_COL>>(),  make_entry<Cfg<float, 128, 16, 32, KIND_COL>>(),
      make_entry<Cfg<float, 256, 16, 16, KIND_COL>>(), make_entry<Cfg<float, 256, 16, 4, KIND_COL>>(),
      make_entry<Cfg<float, 128, 16, 8, KIND_ROW>>(),  make_entry<Cfg<float, 128, 16, 32, KIND_ROW>>(),
      make_entry<Cfg<float, 256, 16, 16, KIND_ROW>>(), make_entry<Cfg<float, 256, 16, 4, KIND_ROW>>(),
      // fewer columns / rows per block for the 512..2048 passes of larger N
      // (two or more blocks per SM instead of one)
      make_entry<Cfg<float, 512, 16, 16, KIND_COL>>(), make_entry<Cfg<float, 512, 16, 4, KIND_COL>>(),
      make_entry<Cfg<float, 1024, 16, 4, KIND_COL>>(), make_entry<Cfg<float, 1024, 16, 2, KIND_COL>>(),
      make_entry<Cfg<float, 2048, 16, 2, KIND_COL>>(), make_entry<Cfg<float, 512, 16, 16, KIND_ROW>>(),
      make_entry<Cfg<float, 512, 16, 4, KIND_ROW>>(),  make_entry<Cfg<float, 1024, 16, 4, KIND_ROW>>(),
      make_entry<Cfg<float, 1024, 16, 2, KIND_ROW>>(), make_entry<Cfg<float, 2048, 16, 2, KIND_ROW>>(),
      // first pass of 8192 = 64 x 128 (ragged plans run by one launch)
      make_entry<Cfg<float, 64, 8, 32, KIND_COL>>(),
  };
  *count = sizeof(t) / sizeof(t[0]);
  return t;
}
}  // namespace tf
