// bounds.cuh -- index checks of the debug build (compiled with
// -DSMC_DEBUG_BOUNDS): an index that would take an access outside its array
// latches ST_BOUNDS in the status word (SMC_ERR_BOUNDS from smc_ctx_check)
// and the access is skipped or redirected to a valid element; the kernel runs
// on (no trap, no assert).  Release builds compile the checks out: the
// condition is assumed.  Placed at every access whose index comes from
// caller data (ancestor arrays) and at the resamplers' computed stores.
#pragma once
#include "device.cuh"

namespace smc {

enum : uint32_t { ST_BOUNDS = 16u };

#ifdef SMC_DEBUG_BOUNDS
__device__ __forceinline__ bool in_bounds(bool ok, uint32_t* status) {
    if (!ok) raise_status(status, ST_BOUNDS);
    return ok;
}
#define SMC_IN_BOUNDS(cond, status) (::smc::in_bounds((cond), (status)))
#else
#define SMC_IN_BOUNDS(cond, status) (true)
#endif

}  // namespace smc
