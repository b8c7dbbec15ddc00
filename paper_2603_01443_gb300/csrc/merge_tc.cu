// Merging (Algorithm 3) on tcgen05 tensor cores -- placeholder until the
// tensor-core kernel lands; every call reports CC_EUNSUPPORTED so that
// CC_MERGE_AUTO falls back to the CUDA-core form.
#include <cuda_runtime.h>

#include "internal.h"

namespace cc {

uint64_t merge_tc_workspace_bytes(int, int, int64_t, int) { return 0; }

cc_status launch_merge_tc(const MergeStage&, int, void*, uint64_t, void*) {
  return fail(CC_EUNSUPPORTED, "tensor-core merge not available in this build");
}

}  // namespace cc
