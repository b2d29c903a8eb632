// Types shared by the device kernels and the host side of the library.
#pragma once

#include <stdint.h>

namespace tf {

enum Kind { KIND_SP = 0, KIND_COL = 1, KIND_ROW = 2 };
enum FtMode { FT_OFF = 0, FT_DETECT = 1, FT_CORRECT = 2 };
enum FtResult {
  FT_RES_PENDING = 0,
  FT_RES_LOCATED = 1,       // DETECT mode: located, not corrected
  FT_RES_DELTA = 2,         // corrected from the right-side checksum
  FT_RES_RECOMPUTE = 3,     // corrected by recomputing from the input
  FT_RES_UNCORRECTABLE = 4,
  FT_RES_CLEAR = 5          // group alarm, but every signal passes on its own (rounding)
};

// correction records per exec (one per detected checksum group)
constexpr int MAX_RECORDS = 64;

// armed one-shot fault (kernel argument; active == 0 when not armed)
struct InjectSite {
  int active;
  int pass;
  int stage;
  int pos;        // position in the sub-transform's working array
  int comp;       // 0 real, 1 imaginary
  int bit;
  long long signal;  // sub-transform id within the pass
};

// one detected checksum group
struct FtRecord {
  int pass_id;
  int slot;
  int count;          // transactions in the group
  int located;        // transaction index of the corrupted signal, -1 ambiguous, -2 several
  long long unit0;    // first work unit of the group
  long long unit_stride;
  long long transform_base;  // offset of the launch's first transform in the caller's batch
  double s1r, s1i, s2r, s2i, tau, energy;
  int result;         // FtResult
  int has_sums;       // right-side sums stored with the record (register mode)
  long long signal;   // sub-transform id of the located signal (-1 if none)
};

// device-side fault-tolerance state of one exec
struct FtState {
  unsigned long long groups;
  unsigned long long detected;
  unsigned long long located;
  unsigned long long corrected;
  unsigned long long recomputed;
  unsigned long long uncorrectable;
  unsigned long long dropped;       // detections beyond MAX_RECORDS (counted uncorrectable)
  unsigned long long num_records;
  float max_clean_ratio;
  int error;  // nonzero: a bounded device wait of an exec expired (TURBOFFT_TIMEOUT)
  FtRecord rec[MAX_RECORDS];
};

constexpr int FT_HEADER_BYTES = 8 * 8 + 8;  // counters + max_clean_ratio + pad

}  // namespace tf
