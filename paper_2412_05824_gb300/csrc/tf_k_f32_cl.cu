// float32 single-pass cluster configurations for N = 2^13 .. 2^16:
// ClCfg<column config <N1, E, SA, COL>, row config <N2, E, SB, ROW>>,
// C = N2 / SA = N1 / SB blocks per cluster
#include "tf_instantiate_cl.cuh"
namespace tf {
const ClEntry* entries_f32_cl(int* count) {
  static const ClEntry t[] = {
      make_cl_entry<ClCfg<Cfg<float, 128, 16, 32, KIND_COL>, Cfg<float, 64, 16, 64, KIND_ROW>>>(),   // 2^13, C=2
      make_cl_entry<ClCfg<Cfg<float, 128, 16, 32, KIND_COL>, Cfg<float, 128, 16, 32, KIND_ROW>>>(),  // 2^14, C=4
      make_cl_entry<ClCfg<Cfg<float, 128, 16, 32, KIND_COL>, Cfg<float, 256, 16, 16, KIND_ROW>>>(),  // 2^15, C=8
      make_cl_entry<ClCfg<Cfg<float, 256, 16, 32, KIND_COL>, Cfg<float, 256, 16, 32, KIND_ROW>>>(),  // 2^16, C=8
  };
  *count = sizeof(t) / sizeof(t[0]);
  return t;
}
}  // namespace tf
