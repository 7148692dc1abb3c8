// Optional per-kernel timing with CUDA events (dgasm_profile_enable).
#pragma once

#include <vector>

#include <cuda_runtime.h>

namespace dgasm {

enum ProfKind { PK_SPMV = 0, PK_UPDATE = 1, PK_LOCAL = 2, PK_COARSE = 3, PK_PUPDATE = 4, PK_CHOL_DIAG = 5,
                PK_CHOL_PANEL = 6, PK_CHOL_UPDATE = 7, PK_NKINDS = 8 };

bool profiling();            // some kind is timed
bool profiling(int kind);    // this kind is timed
void prof_add(int kind, double ms, long long launches);

// A set of (start, stop) event pairs, reused across calls; record with begin/end around launches,
// then accumulate() after the stream (or graph) has completed.
struct EventPairs {
  std::vector<cudaEvent_t> a, b;
  std::vector<int> kind;
  size_t used = 0;
  ~EventPairs();
  void reset() { used = 0; kind.clear(); }
  void reserve(size_t n);             // pre-create n pairs (before a stream capture)
  int begin(int k, cudaStream_t s);   // returns pair index, or -1 (kind not timed, no event left)
  void end(int idx, cudaStream_t s);
  void accumulate();                  // adds every recorded pair to the process-wide counters
  static void record(cudaEvent_t e, cudaStream_t s);
};

}  // namespace dgasm
