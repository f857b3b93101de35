// Dispatch of the fused persistent stage kernel (fused.cuh) by precision,
// dimensionality and limiter; the instantiations are compiled from
// fused_inst.cu once per (precision, dimension, limiter).
#include "state.hpp"

namespace amrvac {

template <class T, int DIM, int LIM>
int launch_fused_l(amrvac_state* s, int k, int epilogue, int g);

bool fused_supported(const amrvac_config* c) {
  if (c->ndim == 2) return c->block_nx[0] == 16 && c->block_nx[1] == 16;
  if (c->ndim == 3) return c->block_nx[0] == 16 && c->block_nx[1] == 16 && c->block_nx[2] == 16;
  return false;
}

// three ghost layers (five-point limiters) on the fused path: 2D tiles, and
// 3D blocks in FP32 bulk, whose every level reconstructs with a five-point
// limiter
bool fused_supported5(const amrvac_config* c) {
  if (c->ndim == 3 && c->precision == AMRVAC_FP64) return false;
  if (c->ndim < 2 || !fused_supported(c) || !five_point_limiter(c->limiter)) return false;
  for (int L = 0; L < MAXLEV; L++)
    if (c->level_limiter[L] > 0 && !five_point_limiter(c->level_limiter[L] - 1)) return false;
  return true;
}

template <class T, int DIM> static int by_limiter(amrvac_state* s, int k, int epilogue, int g) {
  if (five_point_limiter(s->grp_lim[g])) {
    // the five-point limiters share one instantiation (three ghost layers;
    // 3D in FP32 bulk only)
    if constexpr (DIM == 2 || sizeof(T) == 4) return launch_fused_l<T, DIM, -2>(s, k, epilogue, g);
    return -1;
  }
  switch (s->grp_lim[g]) {
    case AMRVAC_LIM_MINMOD: return launch_fused_l<T, DIM, AMRVAC_LIM_MINMOD>(s, k, epilogue, g);
    case AMRVAC_LIM_VANLEER: return launch_fused_l<T, DIM, AMRVAC_LIM_VANLEER>(s, k, epilogue, g);
    case AMRVAC_LIM_KOREN: return launch_fused_l<T, DIM, AMRVAC_LIM_KOREN>(s, k, epilogue, g);
  }
  // the other limiters share one instantiation with a runtime limiter
  return launch_fused_l<T, DIM, -1>(s, k, epilogue, g);
}

// one launch per scheme group (levels sharing flux and limiter), in order
int launch_fused_stage(amrvac_state* s, int k, int epilogue) {
  const bool f64 = s->cfg.precision == AMRVAC_FP64;
  int total = 0;
  for (int g = 0; g < s->ngroups; g++) {
    int n;
    if (s->ndim == 2) n = f64 ? by_limiter<double, 2>(s, k, epilogue, g) : by_limiter<float, 2>(s, k, epilogue, g);
    else if (s->ndim == 3) n = f64 ? by_limiter<double, 3>(s, k, epilogue, g) : by_limiter<float, 3>(s, k, epilogue, g);
    else return -1;
    if (n < 0) return -1;
    total += n;
  }
  return total;
}

}  // namespace amrvac
