// Host-side registry of the compiled kernel configurations.
#pragma once

#include <cuda_runtime.h>

namespace tf {

typedef void (*LaunchFn)(const void* args, int grid, cudaStream_t stream);
// pass kernel with TMA-staged tiles: args as LaunchFn, tmap a CUtensorMap
typedef void (*LaunchTmaFn)(const void* args, const void* tmap, int grid, cudaStream_t stream);

struct KernelEntry {
  int dtype;        // 0 float, 1 double, 2 double data in float-pair arithmetic
  int kind;         // Kind
  int ns;           // sub-transform length
  int e;            // complex values per thread (= radix of the first passes)
  int s;            // sub-transforms per transaction
  int nt;           // threads per block
  int stages;       // radix passes
  int smem_main[5]; // dynamic shared memory of the transform kernel per variant
  int smem_fix;     // dynamic shared memory of the correction kernel
  // transform kernel: no checksums / checksums / checksums + register sums /
  // thread-level checksums (one thread per transform only; null otherwise) /
  // transform-level checksums (float64 column and row passes; null otherwise)
  LaunchFn main[5];
  LaunchFn fix;       // correction kernel
  LaunchFn tcfix;     // transform-level correction: recompute recorded transforms' pass
  const void* fn_main[5];
  const void* fn_fix;
  const void* fn_tcfix;
  // float32 column passes: the transform kernel with TMA-staged tiles, no
  // checksums / checksums (null otherwise)
  int smem_tma[2];
  LaunchTmaFn main_tma[2];
  const void* fn_main_tma[2];
};

// all entries of one translation unit
typedef const KernelEntry* (*EntryTableFn)(int* count);

// single-pass transform of N = n1 * n2 over a cluster of `cluster` blocks
struct ClEntry {
  int dtype;
  int n, n1, n2;
  int e;            // complex values per thread (both phases)
  int sa, sb;       // columns (phase A) / rows (phase B) per block
  int cluster;      // blocks per cluster
  int nt;           // threads per block
  int stages_a, stages_b;
  int smem[2];      // dynamic shared memory: no checksums / checksums
  LaunchFn main[2];
  LaunchFn fix;
  const void* fn_main[2];
  const void* fn_fix;
};
typedef const ClEntry* (*ClTableFn)(int* count);
const ClEntry* entries_f32_cl(int* count);

const KernelEntry* entries_f32_sp(int* count);
const KernelEntry* entries_f32_col(int* count);
const KernelEntry* entries_f32_row(int* count);
const KernelEntry* entries_f64_sp(int* count);
const KernelEntry* entries_f64_col(int* count);
const KernelEntry* entries_f64_row(int* count);
// alternative shapes (registered after the defaults)
const KernelEntry* entries_f32_alt_sp(int* count);
const KernelEntry* entries_f32_alt_cr(int* count);
const KernelEntry* entries_f64_alt(int* count);
// float64 data in float-pair arithmetic (no checksum variants)
const KernelEntry* entries_pairs(int* count);

}  // namespace tf
