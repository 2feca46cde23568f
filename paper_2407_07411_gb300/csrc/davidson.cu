// Block Davidson on the device: placeholder until the eigensolver kernels land.
#include "../../include/dmrg_heff.h"
#include "handle.h"

namespace dmrg {
struct DavidsonState {};
void Handle::release_davidson() { delete dav; dav = nullptr; }
}  // namespace dmrg

extern "C" int dmrg_davidson(dmrg_heff_t, int32_t, double, int32_t, int32_t, int32_t, double*, double*,
                             dmrg_davidson_info*) {
    return dmrg::fail(DMRG_ERR_UNSUPPORTED, "Davidson not built yet");
}
