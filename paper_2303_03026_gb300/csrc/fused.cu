// Fused persistent stage kernels (not yet available in this build).
#include "state.hpp"

namespace amrvac {

bool fused_supported(const amrvac_config*) { return false; }

int launch_fused_stage(amrvac_state*, int, int) { return -1; }

}  // namespace amrvac
