// Float-pair configurations <dd, NS, E, S, kind>: float64 data transformed
// in float-pair arithmetic, with the float64 plans' shapes (radix 8)
#include "tf_instantiate.cuh"
namespace tf {
const KernelEntry* entries_pairs(int* count) {
  static const KernelEntry t[] = {
      make_entry_plain<Cfg<dd, 8, 8, 256, KIND_SP>>(),   make_entry_plain<Cfg<dd, 16, 8, 128, KIND_SP>>(),
      make_entry_plain<Cfg<dd, 32, 8, 64, KIND_SP>>(),   make_entry_plain<Cfg<dd, 64, 8, 32, KIND_SP>>(),
      make_entry_plain<Cfg<dd, 128, 8, 16, KIND_SP>>(),  make_entry_plain<Cfg<dd, 256, 8, 8, KIND_SP>>(),
      make_entry_plain<Cfg<dd, 512, 8, 2, KIND_SP>>(),   make_entry_plain<Cfg<dd, 1024, 8, 1, KIND_SP>>(),
      make_entry_plain<Cfg<dd, 2048, 8, 1, KIND_SP>>(),  make_entry_plain<Cfg<dd, 4096, 8, 1, KIND_SP>>(),
      make_entry_plain<Cfg<dd, 64, 8, 8, KIND_COL>>(),   make_entry_plain<Cfg<dd, 128, 8, 8, KIND_COL>>(),
      make_entry_plain<Cfg<dd, 256, 8, 8, KIND_COL>>(),  make_entry_plain<Cfg<dd, 512, 8, 4, KIND_COL>>(),
      make_entry_plain<Cfg<dd, 1024, 8, 2, KIND_COL>>(), make_entry_plain<Cfg<dd, 2048, 8, 1, KIND_COL>>(),
      make_entry_plain<Cfg<dd, 4096, 8, 1, KIND_COL>>(), make_entry_plain<Cfg<dd, 64, 8, 8, KIND_ROW>>(),
      make_entry_plain<Cfg<dd, 128, 8, 8, KIND_ROW>>(),  make_entry_plain<Cfg<dd, 256, 8, 8, KIND_ROW>>(),
      make_entry_plain<Cfg<dd, 512, 8, 4, KIND_ROW>>(),  make_entry_plain<Cfg<dd, 1024, 8, 2, KIND_ROW>>(),
      make_entry_plain<Cfg<dd, 2048, 8, 1, KIND_ROW>>(), make_entry_plain<Cfg<dd, 4096, 8, 1, KIND_ROW>>(),
  };
  *count = sizeof(t) / sizeof(t[0]);
  return t;
}
}  // namespace tf
