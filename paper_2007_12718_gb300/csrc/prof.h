// Optional per-kernel timing with CUDA events recorded on the launching
// stream (off by default; enabled through ls_profile_enable).  Each named
// slot accumulates launches, device time and the algorithmic bytes / flops
// the caller attributes to each launch.
#pragma once
#include <cuda_runtime.h>

namespace ls {

enum ProfSlot {
  PR_MV_ROWS_FWD = 0,
  PR_MV_COLS,
  PR_MV_ROWS_INV,
  PR_SPECTRUM,
  PR_CPQR,
  PR_KBLOCK,
  PR_LEAF,
  PR_MERGE_GEMM,
  PR_MERGE_INV,
  PR_APPLY,
  PR_GMRES_ORTH,
  PR_APPLY_BLOCK,
  PR_GMRES_BLOCK,
  PR_COUNT
};

// Returns an opaque token (>= 0) or -1 when profiling is off.
int prof_begin(cudaStream_t st);
void prof_end(int token, int slot, cudaStream_t st, double bytes, double flops);

}  // namespace ls
