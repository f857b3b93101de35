// One instantiation group of the fused stage kernel, selected at compile time
// by AMRVAC_FT (float or double), AMRVAC_FD (2 or 3) and AMRVAC_FL (limiter);
// the build compiles this file once per group so the groups build in parallel.
#include "fused.cuh"

#ifndef AMRVAC_FT
#define AMRVAC_FT float
#define AMRVAC_FD 3
#define AMRVAC_FL 1
#endif

namespace amrvac {
template int launch_fused_l<AMRVAC_FT, AMRVAC_FD, AMRVAC_FL>(amrvac_state*, int, int, int);
}  // namespace amrvac
