// float64 alternative shapes <real, NS, E, S, kind>: twice the transforms
// (or columns / rows) per block of the defaults, one 512-thread block per SM
// instead of two of 256 threads (measured 1-3% slower on GB300 at these
// sizes), and a one-thread-per-transform N = 16 shape, timed against the
// defaults by the plan autotuner
#include "tf_instantiate.cuh"
namespace tf {
const KernelEntry* entries_f64_alt(int* count) {
  static const KernelEntry t[] = {
      make_entry<Cfg<double, 512, 8, 4, KIND_SP>>(),    make_entry<Cfg<double, 1024, 8, 2, KIND_SP>>(),
      make_entry<Cfg<double, 512, 8, 8, KIND_COL>>(),   make_entry<Cfg<double, 1024, 8, 4, KIND_COL>>(),
      make_entry<Cfg<double, 2048, 8, 2, KIND_COL>>(),  make_entry<Cfg<double, 512, 8, 8, KIND_ROW>>(),
      make_entry<Cfg<double, 1024, 8, 4, KIND_ROW>>(),  make_entry<Cfg<double, 2048, 8, 2, KIND_ROW>>(),
      // one thread per transform (also the shape of thread-level checksums)
      make_entry<Cfg<double, 16, 16, 64, KIND_SP>>(),
  };
  *count = sizeof(t) / sizeof(t[0]);
  return t;
}
}  // namespace tf
