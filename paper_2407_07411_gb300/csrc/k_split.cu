// Split-precision (Ozaki) path: placeholder until the slice kernels land.
#include "../../include/dmrg_heff.h"
#include "handle.h"

namespace dmrg {
struct SplitState {};
int Handle::init_split(const double*, const int64_t*, const int64_t*, const double*) {
    return fail(DMRG_ERR_UNSUPPORTED, "split precision not built yet");
}
int Handle::apply_split(const double*, double*, int32_t, cudaStream_t) {
    return fail(DMRG_ERR_UNSUPPORTED, "split precision not built yet");
}
void Handle::release_split() { delete split; split = nullptr; }
}  // namespace dmrg
