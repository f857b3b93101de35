// Dispatch of the fused persistent stage kernel (fused.cuh) by precision,
// dimensionality and limiter; the instantiations are compiled from
// fused_inst.cu once per (precision, dimension, limiter).
#include "state.hpp"

namespace amrvac {

template <class T, int DIM, int LIM> int launch_fused_l(amrvac_state* s, int k, int epilogue);

bool fused_supported(const amrvac_config* c) {
  if (c->ndim == 2) return c->block_nx[0] == 16 && c->block_nx[1] == 16;
  if (c->ndim == 3) return c->block_nx[0] == 16 && c->block_nx[1] == 16 && c->block_nx[2] == 16;
  return false;
}

template <class T, int DIM> static int by_limiter(amrvac_state* s, int k, int epilogue) {
  switch (s->cfg.limiter) {
    case AMRVAC_LIM_MINMOD: return launch_fused_l<T, DIM, AMRVAC_LIM_MINMOD>(s, k, epilogue);
    case AMRVAC_LIM_VANLEER: return launch_fused_l<T, DIM, AMRVAC_LIM_VANLEER>(s, k, epilogue);
    case AMRVAC_LIM_KOREN: return launch_fused_l<T, DIM, AMRVAC_LIM_KOREN>(s, k, epilogue);
  }
  // the other limiters share one instantiation with a runtime limiter
  return launch_fused_l<T, DIM, -1>(s, k, epilogue);
}

int launch_fused_stage(amrvac_state* s, int k, int epilogue) {
  const bool f64 = s->cfg.precision == AMRVAC_FP64;
  if (s->ndim == 2) return f64 ? by_limiter<double, 2>(s, k, epilogue) : by_limiter<float, 2>(s, k, epilogue);
  if (s->ndim == 3) return f64 ? by_limiter<double, 3>(s, k, epilogue) : by_limiter<float, 3>(s, k, epilogue);
  return -1;
}

}  // namespace amrvac
