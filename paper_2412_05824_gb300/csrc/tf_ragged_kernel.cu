// One persistent kernel for a ragged batch of float32 transforms of mixed
// power-of-two lengths 8 .. 2^16 (the paper generates and tunes one kernel per
// length, Sec. 3.3 and Table 1; a ragged batch is served here by a single
// launch instead).
//
// Every length maps to a size class: a compile-time kernel configuration of
// 256 threads (one pass for 8 .. 4096; two four-step passes, column then
// row, for 8192 .. 2^16).  The host cuts each class's work units into items
// of a few hundred KB and sorts them by size, largest first; the blocks of
// the grid (all resident: a cooperative launch) take items from a queue with
// an atomic counter and run the class's pass body on the item's units.
// Phase 0 holds the one-pass units and the column passes, phase 1 the row
// passes; a grid barrier separates them, and with checksums on, the
// correction of the detected groups of a phase runs between that barrier and
// the next phase (delayed, batched correction, Sec. 4.1.2).
//
// The grid barrier waits on a counter with a bounded spin: after about a
// second without progress the block records an error in the control block
// and returns, and the host reports TURBOFFT_TIMEOUT.
#include <cuda_runtime.h>

#include "tf_device.cuh"
#include "tf_ragged_kernel.h"

namespace tf {

namespace {

// the size classes (order = class id of RgClassInfo)
using RC0 = Cfg<float, 8, 8, 256, KIND_SP>;
using RC1 = Cfg<float, 16, 8, 128, KIND_SP>;
using RC2 = Cfg<float, 32, 8, 64, KIND_SP>;
using RC3 = Cfg<float, 64, 8, 32, KIND_SP>;
using RC4 = Cfg<float, 128, 16, 32, KIND_SP>;
using RC5 = Cfg<float, 256, 16, 16, KIND_SP>;
using RC6 = Cfg<float, 512, 16, 8, KIND_SP>;
using RC7 = Cfg<float, 1024, 16, 4, KIND_SP>;
using RC8 = Cfg<float, 2048, 16, 2, KIND_SP>;
using RC9 = Cfg<float, 4096, 16, 1, KIND_SP>;
using RC10 = Cfg<float, 64, 8, 32, KIND_COL>;
using RC11 = Cfg<float, 128, 16, 32, KIND_COL>;
using RC12 = Cfg<float, 256, 16, 16, KIND_COL>;
using RC13 = Cfg<float, 128, 16, 32, KIND_ROW>;
using RC14 = Cfg<float, 256, 16, 16, KIND_ROW>;

template <class F> __device__ __forceinline__ void with_class(int cls, F&& f) {
  switch (cls) {
    case 0: f(RC0{}); break;
    case 1: f(RC1{}); break;
    case 2: f(RC2{}); break;
    case 3: f(RC3{}); break;
    case 4: f(RC4{}); break;
    case 5: f(RC5{}); break;
    case 6: f(RC6{}); break;
    case 7: f(RC7{}); break;
    case 8: f(RC8{}); break;
    case 9: f(RC9{}); break;
    case 10: f(RC10{}); break;
    case 11: f(RC11{}); break;
    case 12: f(RC12{}); break;
    case 13: f(RC13{}); break;
    default: f(RC14{}); break;
  }
}

template <class K> constexpr RgClassInfo info_of() {
  return RgClassInfo{K::KIND, K::NS, K::E, K::S, pass_smem_bytes<K, 0>(), pass_smem_bytes<K, 1>(), K::SMEM_BYTES};
}
constexpr RgClassInfo kClasses[kRgClasses] = {
    info_of<RC0>(),  info_of<RC1>(),  info_of<RC2>(),  info_of<RC3>(),  info_of<RC4>(),
    info_of<RC5>(),  info_of<RC6>(),  info_of<RC7>(),  info_of<RC8>(),  info_of<RC9>(),
    info_of<RC10>(), info_of<RC11>(), info_of<RC12>(), info_of<RC13>(), info_of<RC14>(),
};
static_assert(RC0::NT == kRgThreads && RC1::NT == kRgThreads && RC2::NT == kRgThreads && RC3::NT == kRgThreads &&
                  RC4::NT == kRgThreads && RC5::NT == kRgThreads && RC6::NT == kRgThreads &&
                  RC7::NT == kRgThreads && RC8::NT == kRgThreads && RC9::NT == kRgThreads &&
                  RC10::NT == kRgThreads && RC11::NT == kRgThreads && RC12::NT == kRgThreads &&
                  RC13::NT == kRgThreads && RC14::NT == kRgThreads,
              "every size class runs on blocks of kRgThreads threads");

// Grid barrier over all blocks of the (cooperative, hence co-resident) grid.
// Returns false if this block gave up waiting or another block did.
__device__ bool grid_barrier(RgCtl* ctl, unsigned nblocks, int* ok_s) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* genp = &ctl->bar_gen;
    const unsigned gen = *genp;
    __threadfence();
    if (atomicAdd(&ctl->bar_count, 1u) == nblocks - 1) {
      atomicExch(&ctl->bar_count, 0u);
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      // about 2^22 polls (an L2 read and a 64 ns sleep each): a second or more
      for (long long spins = 0; *genp == gen; ++spins) {
        if (spins > (1ll << 22)) {
          atomicExch(&ctl->error, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    *ok_s = ok && *reinterpret_cast<volatile int*>(&ctl->error) == 0;
  }
  __syncthreads();
  return *ok_s != 0;
}

// the correction path (rare) as a separate function: its register needs do
// not weigh on the transform code of the kernel
template <class K>
__device__ __noinline__ void fix_class(const PassArgs<float>& A, char* smem, double* red) {
  fix_body<K>(A, smem, red, blockIdx.x, gridDim.x);
}

template <int FTM>
__global__ void __launch_bounds__(kRgThreads, 2) tf_ragged_kernel(const __grid_constant__ RgParams P) {
  extern __shared__ __align__(128) unsigned char smem_raw_[];
  char* smem = reinterpret_cast<char*>(smem_raw_);
  __shared__ long long item_s;
  __shared__ int ok_s;
  __shared__ double red[3 * 32];
  for (int ph = 0; ph < P.num_phases; ++ph) {
    for (;;) {
      __syncthreads();  // the previous item is done with shared memory
      if (threadIdx.x == 0) item_s = (long long)atomicAdd(&P.ctl->head[ph], 1ull);
      __syncthreads();
      const long long it = item_s;
      if (it >= P.num_items[ph]) break;
      const RgItem w = P.items[ph][it];
      const RgPassArgs& C = P.ca[w.ca];
      with_class(C.cls, [&](auto k) {
        using K = decltype(k);
        pass_body<K, FTM>(C.A, smem, w.u0, 1, w.u1);
      });
    }
    const bool last = ph + 1 == P.num_phases;
    if (FTM == 0 && last) break;
    if (!grid_barrier(P.ctl, gridDim.x, &ok_s)) return;
    if constexpr (FTM != 0) {
      // corrections of this phase's detected groups
      unsigned long long nrec = 0;
      for (int i = 0; i < P.num_ca; ++i)
        if (P.ca[i].phase == ph)
          nrec += *reinterpret_cast<volatile unsigned long long*>(&P.ca[i].A.fts->num_records);
      if (nrec) {
        for (int i = 0; i < P.num_ca; ++i) {
          if (P.ca[i].phase != ph) continue;
          const RgPassArgs& C = P.ca[i];
          with_class(C.cls, [&](auto k) {
            using K = decltype(k);
            __syncthreads();
            fix_class<K>(C.A, smem, red);
          });
        }
        if (!last && !grid_barrier(P.ctl, gridDim.x, &ok_s)) return;
      }
    }
  }
}

}  // namespace

const RgClassInfo* ragged_classes() { return kClasses; }

const void* ragged_kernel_fn(int ftm) {
  return ftm ? reinterpret_cast<const void*>(&tf_ragged_kernel<1>) : reinterpret_cast<const void*>(&tf_ragged_kernel<0>);
}

cudaError_t launch_ragged_kernel(int ftm, const RgParams& P, int grid, size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)kRgThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return ftm ? cudaLaunchKernelEx(&cfg, tf_ragged_kernel<1>, P) : cudaLaunchKernelEx(&cfg, tf_ragged_kernel<0>, P);
}

}  // namespace tf
