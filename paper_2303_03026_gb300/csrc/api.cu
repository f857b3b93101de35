// C ABI of the amrvac GB300 library: mesh tables, workspace layout, state
// management and the stage / step drivers (see include/amrvac.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "state.hpp"

using namespace amrvac;

namespace {

constexpr size_t ALIGN = 256;

size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

struct Tables {
  std::vector<int> blk, nbr, gface, glist, gkind, rlist, lmap, lmap_off, lnb, istart, iblocks;
  std::vector<double> gamma, dx;
  // device regrid plan: per instance the deepest level, and the offsets of the
  // dense new-leaf maps of levels 0 .. deepest + 1 ([ninst * MAXLEV + 1];
  // empty when a map that fine would be too large)
  std::vector<int> maxlev, pseg;
  std::string err;
};

struct Layout {
  size_t U[3], W, F[3], part, blk, nbr, gface, glist, lmap, lmap_off, lnb, gamma, dx, istart,
      iblocks, rt, sums, err, work, work2, counter, gslab, lcf, lcd, flags, fixcount, gkind,
      rlist, fluxreg, est, eflags, rtab, pref, pfate, pmap, pseg, pmax, psums, pscal, pout,
      total;
};

bool config_ok(const amrvac_config* c, std::string& err) {
  if (!c) return err = "null config", false;
  if (c->ndim < 1 || c->ndim > 3) return err = "ndim must be 1..3", false;
  long long cells = 1;  // 64-bit: 4096^3 overflows an int
  for (int d = 0; d < c->ndim; d++) {
    if (c->block_nx[d] < 4 || c->block_nx[d] > 4096) return err = "block_nx must be 4..4096", false;
    cells *= c->block_nx[d];
  }
  if (cells > AMRVAC_MAX_BLOCK_CELLS) return err = "block larger than AMRVAC_MAX_BLOCK_CELLS", false;
  if (c->flux < AMRVAC_FLUX_HLL || c->flux > AMRVAC_FLUX_HLLC) return err = "bad flux", false;
  if (c->limiter < AMRVAC_LIM_MINMOD || c->limiter > AMRVAC_LIM_VENK)
    return err = "bad limiter", false;
  if (c->reflux != 0 && c->reflux != 1) return err = "bad reflux", false;
  for (int L = 0; L < AMRVAC_MAX_LEVELS; L++) {
    if (c->level_flux[L] < 0 || c->level_flux[L] > AMRVAC_FLUX_HLLC + 1)
      return err = "bad level_flux", false;
    if (c->level_limiter[L] < 0 || c->level_limiter[L] > AMRVAC_LIM_VENK + 1)
      return err = "bad level_limiter", false;
  }
  if (c->fix_small_values < AMRVAC_FIX_OFF || c->fix_small_values > AMRVAC_FIX_AVERAGE)
    return err = "bad fix_small_values", false;
  if (c->fix_small_values != AMRVAC_FIX_OFF &&
      !(c->small_density > 0.0 && c->small_pressure > 0.0))
    return err = "fix_small_values needs positive small_density and small_pressure", false;
  if (c->time < AMRVAC_SSPRK2 || c->time > AMRVAC_SSPRK54) return err = "bad time", false;
  if (c->precision != AMRVAC_FP64 && c->precision != AMRVAC_FP32_BULK)
    return err = "bad precision", false;
  if (!(c->courant > 0.0) || !(c->glm_alpha >= 0.0)) return err = "bad courant/glm_alpha", false;
  for (int d = 0; d < 3; d++)
    for (int s = 0; s < 2; s++)
      if (c->bc[d][s] != AMRVAC_BC_PERIODIC && c->bc[d][s] != AMRVAC_BC_OUTFLOW &&
          c->bc[d][s] != AMRVAC_BC_SYMMETRIC)
        return err = "bad bc", false;
  for (int d = 0; d < c->ndim; d++)
    if ((c->bc[d][0] == AMRVAC_BC_PERIODIC) != (c->bc[d][1] == AMRVAC_BC_PERIODIC))
      return err = "periodic bc must be set on both sides", false;
  if (c->kernel < 0 || c->kernel > 2) return err = "bad kernel", false;
  if (c->pressure != AMRVAC_PRESSURE_FP64 && c->pressure != AMRVAC_PRESSURE_FF)
    return err = "bad pressure", false;
  return true;
}

int nx_of(const amrvac_config* c, int d) { return d < c->ndim ? c->block_nx[d] : 1; }

// ghost cells per block face of the plain path: 3 when the limiter or a
// level's limiter is a five-point one, else 2
int ghost_width(const amrvac_config* c) {
  int g = five_point_limiter(c->limiter) ? NG5 : NG;
  for (int L = 0; L < AMRVAC_MAX_LEVELS; L++)
    if (c->level_limiter[L] > 0 && five_point_limiter(c->level_limiter[L] - 1)) g = NG5;
  return g;
}

// Build and validate the block tables.  Per instance and level a dense map of
// block positions: leaf id, MAP_REFINED or MAP_COARSER.
bool build_tables(const amrvac_config* c, int ninst, const amrvac_instance_desc* inst,
                  int nblocks, const int32_t* meta, Tables& T) {
  if (ninst < 1 || nblocks < 1 || !inst || !meta) return T.err = "empty mesh", false;
  std::vector<int> maxlev(ninst, -1);
  for (int q = 0; q < ninst; q++) {
    if (!(inst[q].gamma > 1.0)) return T.err = "gamma must exceed 1", false;
    for (int d = 0; d < c->ndim; d++) {
      if (inst[q].base_blocks[d] < 1) return T.err = "base_blocks must be >= 1", false;
      if (!(inst[q].xmax[d] > inst[q].xmin[d])) return T.err = "empty domain", false;
    }
  }
  for (int b = 0; b < nblocks; b++) {
    const int32_t* r = meta + 5 * b;
    if (r[0] < 0 || r[0] >= ninst) return T.err = "block instance out of range", false;
    if (r[1] < 0 || r[1] >= MAXLEV) return T.err = "block level out of range", false;
    for (int d = 0; d < c->ndim; d++) {
      long n = (long)inst[r[0]].base_blocks[d] << r[1];
      if (r[2 + d] < 0 || r[2 + d] >= n) return T.err = "block index out of range", false;
    }
    maxlev[r[0]] = std::max(maxlev[r[0]], (int)r[1]);
  }
  T.lmap_off.assign((size_t)ninst * MAXLEV, 0);
  T.lnb.assign((size_t)ninst * MAXLEV * 3, 1);
  T.dx.assign((size_t)ninst * MAXLEV * 3, 1.0);
  T.gamma.resize(ninst);
  size_t total = 0;
  for (int q = 0; q < ninst; q++) {
    if (maxlev[q] < 0) return T.err = "instance without blocks", false;
    T.gamma[q] = inst[q].gamma;
    for (int L = 0; L < MAXLEV; L++) {
      size_t cnt = 1;
      for (int d = 0; d < 3; d++) {
        long n = d < c->ndim ? ((long)inst[q].base_blocks[d] << L) : 1;
        if (L <= maxlev[q] && n > (1 << 20)) return T.err = "mesh too fine", false;
        T.lnb[(q * MAXLEV + L) * 3 + d] = (int)std::min<long>(n, 1 << 30);
        if (d < c->ndim)
          T.dx[(q * MAXLEV + L) * 3 + d] =
              (inst[q].xmax[d] - inst[q].xmin[d]) / ((double)n * c->block_nx[d]);
        cnt *= (size_t)n;
      }
      T.lmap_off[q * MAXLEV + L] = (int)total;
      if (L <= maxlev[q]) total += cnt;
      if (total > (size_t)1 << 30) return T.err = "block maps too large", false;
    }
  }
  // the dense new-leaf maps of the device regrid plan: levels 0 .. maxlev + 1
  T.maxlev = maxlev;
  {
    T.pseg.assign((size_t)ninst * MAXLEV + 1, 0);
    size_t ptot = 0;
    bool fits = true;
    for (int q = 0; q < ninst; q++)
      for (int L = 0; L < MAXLEV; L++) {
        T.pseg[q * MAXLEV + L] = (int)ptot;
        if (L > maxlev[q] + 1) continue;
        size_t cnt = 1;
        for (int d = 0; d < c->ndim; d++) cnt *= (size_t)inst[q].base_blocks[d] << L;
        ptot += cnt;
        if (ptot > ((size_t)1 << 28)) fits = false;
      }
    T.pseg[(size_t)ninst * MAXLEV] = (int)std::min<size_t>(ptot, (size_t)1 << 30);
    if (!fits) T.pseg.clear();
  }
  // the wenozp5 lambda = dx^(2/3) of every (instance, level, dimension), kept
  // after the cell sizes in the same table
  const size_t ndx = T.dx.size();
  T.dx.resize(2 * ndx);
  for (size_t i = 0; i < ndx; i++) T.dx[ndx + i] = std::pow(T.dx[i], 2.0 / 3.0);
  T.lmap.assign(total, MAP_COARSER);
  auto pos = [&](int q, int L, long i, long j, long k) -> int& {
    const int* nb = &T.lnb[(q * MAXLEV + L) * 3];
    return T.lmap[T.lmap_off[q * MAXLEV + L] + (size_t)((k * nb[1] + j) * nb[0] + i)];
  };
  for (int b = 0; b < nblocks; b++) {
    const int32_t* r = meta + 5 * b;
    long i = r[2], j = c->ndim > 1 ? r[3] : 0, k = c->ndim > 2 ? r[4] : 0;
    int& m = pos(r[0], r[1], i, j, k);
    if (m != MAP_COARSER) return T.err = "duplicate block", false;
    m = b;
  }
  for (int b = 0; b < nblocks; b++) {
    const int32_t* r = meta + 5 * b;
    long p[3] = {r[2], c->ndim > 1 ? r[3] : 0, c->ndim > 2 ? r[4] : 0};
    for (int L = r[1] - 1; L >= 0; L--) {
      for (int d = 0; d < c->ndim; d++) p[d] >>= 1;
      int& m = pos(r[0], L, p[0], p[1], p[2]);
      if (m >= 0) return T.err = "overlapping blocks", false;
      m = MAP_REFINED;
    }
  }
  // coverage
  for (int q = 0; q < ninst; q++)
    for (int L = 0; L <= maxlev[q]; L++) {
      const int* nb = &T.lnb[(q * MAXLEV + L) * 3];
      for (long k = 0; k < nb[2]; k++)
        for (long j = 0; j < nb[1]; j++)
          for (long i = 0; i < nb[0]; i++) {
            int m = pos(q, L, i, j, k);
            if (L == 0 && m == MAP_COARSER) return T.err = "hole in the base level", false;
            if (m != MAP_REFINED) continue;
            if (L + 1 > maxlev[q]) return T.err = "refined position without children", false;
            for (int oz = 0; oz < (c->ndim > 2 ? 2 : 1); oz++)
              for (int oy = 0; oy < (c->ndim > 1 ? 2 : 1); oy++)
                for (int ox = 0; ox < 2; ox++)
                  if (pos(q, L + 1, 2 * i + ox, c->ndim > 1 ? 2 * j + oy : 0,
                          c->ndim > 2 ? 2 * k + oz : 0) == MAP_COARSER)
                    return T.err = "hole below a refined block", false;
          }
    }
  // full 2:1 balance and the face neighbour table
  T.blk.resize((size_t)nblocks * 5);
  T.nbr.resize((size_t)nblocks * 6);
  for (int b = 0; b < nblocks; b++) {
    const int32_t* r = meta + 5 * b;
    const int q = r[0], L = r[1];
    long me[3] = {r[2], c->ndim > 1 ? r[3] : 0, c->ndim > 2 ? r[4] : 0};
    for (int e = 0; e < 5; e++) T.blk[b * 5 + e] = e < 2 ? r[e] : (int)me[e - 2];
    int lo[3], hi[3];
    for (int d = 0; d < 3; d++) lo[d] = d < c->ndim ? -1 : 0, hi[d] = -lo[d];
    for (int dz = lo[2]; dz <= hi[2]; dz++)
      for (int dy = lo[1]; dy <= hi[1]; dy++)
        for (int dxx = lo[0]; dxx <= hi[0]; dxx++) {
          if (!dxx && !dy && !dz) continue;
          long p[3] = {me[0] + dxx, me[1] + dy, me[2] + dz};
          bool outside = false;
          for (int d = 0; d < c->ndim; d++) {
            long n = T.lnb[(q * MAXLEV + L) * 3 + d];
            if (p[d] < 0 || p[d] >= n) {
              if (c->bc[d][p[d] < 0 ? 0 : 1] == AMRVAC_BC_PERIODIC) p[d] = ((p[d] % n) + n) % n;
              else outside = true;
            }
          }
          if (outside) continue;
          int LL = L;
          int m = pos(q, LL, p[0], p[1], p[2]);
          while (m == MAP_COARSER && LL > 0) {
            LL--;
            for (int d = 0; d < c->ndim; d++) p[d] >>= 1;
            m = pos(q, LL, p[0], p[1], p[2]);
          }
          if (m == MAP_COARSER) return T.err = "uncovered neighbour", false;
          if (LL < L - 1) return T.err = "mesh is not 2:1 balanced", false;
        }
    for (int d = 0; d < 3; d++)
      for (int side = 0; side < 2; side++) {
        int& out = T.nbr[b * 6 + d * 2 + side];
        if (d >= c->ndim) {
          out = NBR_OUTFLOW;
          continue;
        }
        long p[3] = {me[0], me[1], me[2]};
        p[d] += side ? 1 : -1;
        long n = T.lnb[(q * MAXLEV + L) * 3 + d];
        if (p[d] < 0 || p[d] >= n) {
          if (c->bc[d][side] == AMRVAC_BC_PERIODIC) p[d] = ((p[d] % n) + n) % n;
          else {
            out = c->bc[d][side] == AMRVAC_BC_SYMMETRIC ? NBR_WALL : NBR_OUTFLOW;
            continue;
          }
        }
        int m = pos(q, L, p[0], p[1], p[2]);
        out = m >= 0 ? m : NBR_GENERAL;
        if (m == MAP_REFINED) out = NBR_GENERAL_FINER;
      }
  }
  // level-change faces: one ghost slab (and flux register) each; gkind 1 when
  // the neighbour region is finer, 2 when coarser; rlist: blocks with a finer
  // neighbour (the coarse side of refluxing)
  T.gface.assign((size_t)nblocks * 6, -1);
  T.glist.clear();
  T.gkind.clear();
  T.rlist.clear();
  for (int b = 0; b < nblocks; b++) {
    bool coarse_side = false;
    for (int f = 0; f < 6; f++) {
      int& code = T.nbr[b * 6 + f];
      if (code != NBR_GENERAL && code != NBR_GENERAL_FINER) continue;
      T.gface[b * 6 + f] = (int)T.glist.size();
      T.glist.push_back(b * 6 + f);
      T.gkind.push_back(code == NBR_GENERAL_FINER ? 1 : 2);
      coarse_side |= code == NBR_GENERAL_FINER;
      code = NBR_GENERAL;
    }
    if (coarse_side) T.rlist.push_back(b);
  }
  T.istart.assign(ninst + 1, 0);
  for (int b = 0; b < nblocks; b++) T.istart[meta[5 * b] + 1]++;
  for (int q = 0; q < ninst; q++) T.istart[q + 1] += T.istart[q];
  T.iblocks.resize(nblocks);
  std::vector<int> fill(T.istart.begin(), T.istart.end() - 1);
  for (int b = 0; b < nblocks; b++) T.iblocks[fill[meta[5 * b]]++] = b;
  return true;
}

// the fused kernels take two ghost layers, or three on 2D tiles whose every
// level uses a five-point limiter
bool fused_ok(const amrvac_config* c) {
  return ghost_width(c) == NG ? fused_supported(c) : fused_supported5(c);
}

bool use_fused_for(const amrvac_config* c) {
  if (c->kernel == AMRVAC_KERNEL_PLAIN) return false;
  return fused_ok(c);
}

Layout make_layout(const amrvac_config* c, int ninst, int nblocks, const Tables& T, bool fused) {
  Layout L{};
  size_t rs = c->precision == AMRVAC_FP64 ? 8 : 4;
  size_t ncell = (size_t)nx_of(c, 0) * nx_of(c, 1) * nx_of(c, 2);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  for (int i = 0; i < 3; i++) L.U[i] = take(rs * NV * ncell * nblocks);
  if (!fused) {
    size_t np = 1;
    for (int d = 0; d < 3; d++)
      np *= (size_t)(nx_of(c, d) + (d < c->ndim ? 2 * ghost_width(c) : 0));
    L.W = take(rs * NV * np * nblocks);
    for (int d = 0; d < 3; d++) {
      size_t nf = 0;
      if (d < c->ndim) nf = ncell / nx_of(c, d) * (nx_of(c, d) + 1);
      L.F[d] = take(rs * NV * nf * nblocks);
    }
  }
  L.part = take(sizeof(double) * NPART * nblocks);
  L.blk = take(sizeof(int) * T.blk.size());
  L.nbr = take(sizeof(int) * T.nbr.size());
  L.gface = take(sizeof(int) * T.gface.size());
  L.glist = take(sizeof(int) * (T.glist.size() + 1));
  L.gkind = take(sizeof(int) * (T.gkind.size() + 1));
  L.rlist = take(sizeof(int) * (T.rlist.size() + 1));
  L.lmap = take(sizeof(int) * T.lmap.size());
  L.lmap_off = take(sizeof(int) * T.lmap_off.size());
  L.lnb = take(sizeof(int) * T.lnb.size());
  L.gamma = take(sizeof(double) * T.gamma.size());
  L.dx = take(sizeof(double) * T.dx.size());
  L.istart = take(sizeof(int) * T.istart.size());
  L.iblocks = take(sizeof(int) * T.iblocks.size());
  L.rt = take(sizeof(InstRT) * ninst);
  L.sums = take(sizeof(double) * NV * ninst);
  L.err = take(sizeof(int) * 4);
  L.work = take(sizeof(int) * (size_t)nblocks);
  L.work2 = take(sizeof(int) * (size_t)nblocks);
  L.counter = take(sizeof(int) * (MAXLEV + 4));  // one per scheme group
  L.gslab = 0;
  L.fluxreg = 0;
  if (c->reflux) {
    // flux register of every level-change face: NV x the largest face area
    size_t area = 1;
    for (int d = 0; d < c->ndim; d++) {
      size_t a = 1;
      for (int e = 0; e < c->ndim; e++)
        if (e != d) a *= (size_t)nx_of(c, e);
      area = a > area ? a : area;
    }
    L.fluxreg = take(rs * NV * area * T.glist.size());
  }
  L.flags = L.fixcount = 0;
  if (c->fix_small_values != AMRVAC_FIX_OFF) {
    L.flags = take((size_t)ncell * nblocks);
    L.fixcount = take(sizeof(unsigned long long));
  }
  L.lcf = take(sizeof(float) * LC_N * MAXLEV * ninst);
  L.lcd = take(sizeof(double) * LC_N * MAXLEV * ninst);
  // regridding: per-block estimator and flag, and the transfer table
  L.est = take(sizeof(double) * nblocks);
  L.eflags = take((size_t)nblocks);
  L.rtab = take(sizeof(int) * RTAB_N * (size_t)nblocks);
  // device regrid plan: split marks and fates per block, the dense new-leaf
  // maps, their segment table, scan sums, scalars and the new block list (at
  // most 2^ndim times as many blocks)
  L.pref = take(sizeof(int) * (size_t)nblocks);
  L.pfate = take((size_t)nblocks);
  const size_t pm = T.pseg.empty() ? 0 : (size_t)T.pseg.back();
  L.pmap = take(sizeof(int) * (pm + 1));
  L.pseg = take(sizeof(int) * (T.pseg.size() + 1));
  L.pmax = take(sizeof(int) * (size_t)ninst);
  L.psums = take(sizeof(int) * (PLAN_CTAS + 1));
  L.pscal = take(sizeof(int) * 4);
  L.pout = take(sizeof(int) * 5 * ((size_t)nblocks << c->ndim));
  if (fused) {
    size_t per = (size_t)NV * ghost_width(c) * 16 * (c->ndim == 3 ? 16 : 1);  // one face
    L.gslab = take(rs * per * T.glist.size());
  }
  L.total = off;
  return L;
}

amrvac_status cuda_status(cudaError_t e) { return e == cudaSuccess ? AMRVAC_OK : AMRVAC_E_CUDA; }

template <class T> T* at(amrvac_state* s, size_t off) { return (T*)(s->ws + off); }

amrvac_status check_launch(amrvac_state* s, int n) {
  if (n < 0) return AMRVAC_E_CUDA;
  s->launches += n;
  return AMRVAC_OK;
}

amrvac_status enqueue_stage(amrvac_state* s, int k, int epilogue, int* count) {
  // with refluxing or bootstrapping the output changes after the stage
  // kernel, so its time-step terms are taken afterwards from the final state
  const bool post = s->cfg.reflux || s->cfg.fix_small_values != AMRVAC_FIX_OFF;
  const int out = stage_buffers(s->cfg.time, k).out;
  int n = s->use_fused ? launch_fused_stage(s, k, epilogue && !post)
                       : launch_plain_stage(s, k, epilogue && !post);
  if (n < 0) return AMRVAC_E_CUDA;
  *count += n;
  // conservative coarse-fine correction, then bootstrapping (Sect. 7.4)
  n = launch_reflux(s, k);
  if (n < 0) return AMRVAC_E_CUDA;
  *count += n;
  n = launch_fix_small(s, out);
  if (n < 0) return AMRVAC_E_CUDA;
  *count += n;
  if (epilogue && post) {
    n = launch_cfl_partials(s, out);
    if (n < 0) return AMRVAC_E_CUDA;
    *count += n;
  }
  return AMRVAC_OK;
}

amrvac_status enqueue_step(amrvac_state* s, int* count) {
  const int ns = num_stages(s->cfg.time);
  for (int k = 0; k < ns; k++) {
    amrvac_status st = enqueue_stage(s, k, k == ns - 1, count);
    if (st) return st;
  }
  int n = launch_finalize(s, 1);
  if (n < 0) return AMRVAC_E_CUDA;
  *count += n;
  return AMRVAC_OK;
}

}  // namespace

extern "C" {

const char* amrvac_error_string(amrvac_status st) {
  switch (st) {
    case AMRVAC_OK: return "ok";
    case AMRVAC_E_INVALID: return "invalid argument, config or block list";
    case AMRVAC_E_NOMEM: return "workspace too small";
    case AMRVAC_E_CUDA: return "CUDA runtime error";
    case AMRVAC_E_SMALL_VALUES: return "density or pressure at or below its floor";
    case AMRVAC_E_TIMEOUT: return "bounded device wait gave up";
    case AMRVAC_E_STATE: return "call out of order or inconsistent mesh lookup";
  }
  return "unknown status";
}

amrvac_status amrvac_workspace_bytes(const amrvac_config* cfg, int32_t ninst,
                                     const amrvac_instance_desc* inst, int32_t nblocks,
                                     const int32_t* block_meta, size_t* bytes) {
  std::string err;
  if (!bytes || !config_ok(cfg, err)) return AMRVAC_E_INVALID;
  if (cfg->kernel == AMRVAC_KERNEL_FUSED && !fused_ok(cfg))
    return AMRVAC_E_INVALID;
  Tables T;
  if (!build_tables(cfg, ninst, inst, nblocks, block_meta, T)) return AMRVAC_E_INVALID;
  *bytes = make_layout(cfg, ninst, nblocks, T, use_fused_for(cfg)).total;
  return AMRVAC_OK;
}

amrvac_status amrvac_state_create(const amrvac_config* cfg, int32_t ninst,
                                  const amrvac_instance_desc* inst, int32_t nblocks,
                                  const int32_t* block_meta, void* d_workspace,
                                  size_t workspace_bytes, void* cuda_stream,
                                  amrvac_state** out) {
  std::string err;
  if (!out || !config_ok(cfg, err)) return AMRVAC_E_INVALID;
  *out = nullptr;
  if (cfg->kernel == AMRVAC_KERNEL_FUSED && !fused_ok(cfg))
    return AMRVAC_E_INVALID;
  Tables T;
  if (!build_tables(cfg, ninst, inst, nblocks, block_meta, T)) return AMRVAC_E_INVALID;
  bool fused = use_fused_for(cfg);
  Layout L = make_layout(cfg, ninst, nblocks, T, fused);
  if (!d_workspace || ((uintptr_t)d_workspace % ALIGN) != 0) return AMRVAC_E_INVALID;
  if (workspace_bytes < L.total) return AMRVAC_E_NOMEM;

  amrvac_state* s = new amrvac_state();
  s->cfg = *cfg;
  for (int d = cfg->ndim; d < 3; d++) s->cfg.block_nx[d] = 1;
  s->ninst = ninst;
  s->nblocks = nblocks;
  s->ndim = cfg->ndim;
  s->ncell = nx_of(cfg, 0) * nx_of(cfg, 1) * nx_of(cfg, 2);
  s->use_fused = fused;
  s->real_size = cfg->precision == AMRVAC_FP64 ? 8 : 4;
  s->stream = (cudaStream_t)cuda_stream;
  s->ws = (char*)d_workspace;
  s->ws_bytes = workspace_bytes;
  s->meta.assign(block_meta, block_meta + 5 * (size_t)nblocks);
  s->inst.assign(inst, inst + ninst);
  for (int i = 0; i < 3; i++) s->U[i] = s->ws + L.U[i];
  s->npad = 1;
  for (int d = 0; d < 3; d++) {
    s->P[d] = nx_of(cfg, d) + (d < cfg->ndim ? 2 * ghost_width(cfg) : 0);
    s->npad *= (size_t)s->P[d];
    s->nface[d] = d < cfg->ndim ? (size_t)s->ncell / nx_of(cfg, d) * (nx_of(cfg, d) + 1) : 0;
  }
  if (!fused) {
    s->W = s->ws + L.W;
    for (int d = 0; d < 3; d++) s->F[d] = s->ws + L.F[d];
  }
  DevMesh& M = s->mesh;
  M.ndim = cfg->ndim;
  M.ng = ghost_width(cfg);
  for (int d = 0; d < 3; d++) {
    M.nx[d] = nx_of(cfg, d);
    M.bc[d][0] = cfg->bc[d][0];
    M.bc[d][1] = cfg->bc[d][1];
  }
  M.ncell = s->ncell;
  M.nblocks = nblocks;
  M.ninst = ninst;
  M.blk = at<int>(s, L.blk);
  M.nbr = at<int>(s, L.nbr);
  M.gface = at<int>(s, L.gface);
  M.gkind = at<int>(s, L.gkind);
  M.lmap = at<int>(s, L.lmap);
  M.lmap_off = at<int>(s, L.lmap_off);
  M.lnb = at<int>(s, L.lnb);
  M.gamma = at<double>(s, L.gamma);
  M.dx = at<double>(s, L.dx);
  M.wzlam = M.dx + (size_t)ninst * MAXLEV * 3;
  M.inst_start = at<int>(s, L.istart);
  M.inst_blocks = at<int>(s, L.iblocks);
  M.rt = at<InstRT>(s, L.rt);
  M.part = at<double>(s, L.part);
  M.sums = at<double>(s, L.sums);
  M.err = at<int>(s, L.err);
  if (cfg->fix_small_values != AMRVAC_FIX_OFF) {
    s->d_flags = at<unsigned char>(s, L.flags);
    s->d_fixcount = at<unsigned long long>(s, L.fixcount);
  }
  M.lcf = at<float>(s, L.lcf);
  M.lcd = at<double>(s, L.lcd);
  s->d_work = at<int>(s, L.work);
  s->d_work_morton = s->d_work;
  s->d_work_storage = at<int>(s, L.work2);
  s->d_counter = at<int>(s, L.counter);
  s->d_est = at<double>(s, L.est);
  s->d_eflags = at<signed char>(s, L.eflags);
  s->d_rtab = at<int>(s, L.rtab);
  s->plan.ref = at<int>(s, L.pref);
  s->plan.fate = at<signed char>(s, L.pfate);
  s->plan.map = at<int>(s, L.pmap);
  s->plan.seg = at<int>(s, L.pseg);
  s->plan.maxlev = at<int>(s, L.pmax);
  s->plan.sums = at<int>(s, L.psums);
  s->plan.scal = at<int>(s, L.pscal);
  s->plan.out = at<int>(s, L.pout);
  s->plan.cap = s->nblocks << s->ndim;
  s->plan.nmap = T.pseg.empty() ? -1 : T.pseg.back();
  s->d_glist = at<int>(s, L.glist);
  s->ngen = (int)T.glist.size();
  s->d_rlist = at<int>(s, L.rlist);
  s->nrlist = (int)T.rlist.size();
  if (fused) s->gslab = s->ws + L.gslab;
  if (cfg->reflux) {
    s->fluxreg = s->ws + L.fluxreg;
    size_t area = 1;
    for (int d = 0; d < cfg->ndim; d++) {
      size_t a = 1;
      for (int e = 0; e < cfg->ndim; e++)
        if (e != d) a *= (size_t)nx_of(cfg, e);
      area = a > area ? a : area;
    }
    M.farea = (int)area;
    M.fluxreg = s->fluxreg;
  }

  std::vector<InstRT> rt(ninst);
  for (int q = 0; q < ninst; q++) rt[q] = InstRT{inst[q].t0, inst[q].t_end, 0.0, 0.0};
  cudaError_t e = cudaSuccess;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s->stream);
  };
  up((void*)M.blk, T.blk.data(), sizeof(int) * T.blk.size());
  up((void*)M.nbr, T.nbr.data(), sizeof(int) * T.nbr.size());
  up((void*)M.gface, T.gface.data(), sizeof(int) * T.gface.size());
  up((void*)s->d_glist, T.glist.data(), sizeof(int) * T.glist.size());
  up((void*)M.gkind, T.gkind.data(), sizeof(int) * T.gkind.size());
  up((void*)s->d_rlist, T.rlist.data(), sizeof(int) * T.rlist.size());
  up((void*)M.lmap, T.lmap.data(), sizeof(int) * T.lmap.size());
  up((void*)M.lmap_off, T.lmap_off.data(), sizeof(int) * T.lmap_off.size());
  up((void*)M.lnb, T.lnb.data(), sizeof(int) * T.lnb.size());
  up((void*)M.gamma, T.gamma.data(), sizeof(double) * T.gamma.size());
  up((void*)M.dx, T.dx.data(), sizeof(double) * T.dx.size());
  if (!T.pseg.empty()) up((void*)s->plan.seg, T.pseg.data(), sizeof(int) * T.pseg.size());
  up((void*)s->plan.maxlev, T.maxlev.data(), sizeof(int) * T.maxlev.size());
  up((void*)M.inst_start, T.istart.data(), sizeof(int) * T.istart.size());
  up((void*)M.inst_blocks, T.iblocks.data(), sizeof(int) * T.iblocks.size());
  up((void*)M.rt, rt.data(), sizeof(InstRT) * ninst);
  // the work list of the fused kernel: per instance, blocks along a Morton
  // (Z-order) curve of their position at the instance's finest level, so that
  // blocks processed at the same time share neighbours (and halos) in L2
  std::vector<int> work(nblocks);
  {
    std::vector<int> maxlev(ninst, 0);
    for (int b = 0; b < nblocks; b++)
      maxlev[block_meta[5 * b]] = std::max(maxlev[block_meta[5 * b]], (int)block_meta[5 * b + 1]);
    auto spread = [](uint64_t v) {  // 21 bits -> every third bit
      v &= 0x1fffff;
      v = (v | v << 32) & 0x1f00000000ffffull;
      v = (v | v << 16) & 0x1f0000ff0000ffull;
      v = (v | v << 8) & 0x100f00f00f00f00full;
      v = (v | v << 4) & 0x10c30c30c30c30c3ull;
      v = (v | v << 2) & 0x1249249249249249ull;
      return v;
    };
    std::vector<std::pair<std::pair<int, uint64_t>, int>> keys(nblocks);
    for (int b = 0; b < nblocks; b++) {
      const int32_t* r = block_meta + 5 * b;
      const int sh = maxlev[r[0]] - r[1];
      uint64_t code = spread((uint64_t)r[2] << sh) | spread((uint64_t)(cfg->ndim > 1 ? r[3] : 0) << sh) << 1 |
                      spread((uint64_t)(cfg->ndim > 2 ? r[4] : 0) << sh) << 2;
      keys[b] = {{r[0], code}, b};
    }
    std::sort(keys.begin(), keys.end());
    for (int b = 0; b < nblocks; b++) work[b] = keys[b].second;
  }
  std::vector<int> work_storage(nblocks);
  for (int b = 0; b < nblocks; b++) work_storage[b] = b;
  // scheme groups of the fused path: levels with the same (flux, limiter) share
  // one launch; both work lists become contiguous per group (order kept inside)
  {
    int gof[MAXLEV];
    s->ngroups = 0;
    for (int L = 0; L < MAXLEV; L++) {
      const int fl = cfg->level_flux[L] > 0 ? cfg->level_flux[L] - 1 : cfg->flux;
      const int li = cfg->level_limiter[L] > 0 ? cfg->level_limiter[L] - 1 : cfg->limiter;
      int g = 0;
      while (g < s->ngroups && !(s->grp_flux[g] == fl && s->grp_lim[g] == li)) g++;
      if (g == s->ngroups) {
        s->grp_flux[g] = fl;
        s->grp_lim[g] = li;
        s->ngroups++;
      }
      gof[L] = g;
    }
    auto regroup = [&](std::vector<int>& list) {
      std::vector<int> out;
      out.reserve(list.size());
      for (int g = 0; g < s->ngroups; g++) {
        s->grp_off[g] = (int)out.size();
        for (int b : list)
          if (gof[block_meta[5 * b + 1]] == g) out.push_back(b);
        s->grp_cnt[g] = (int)out.size() - s->grp_off[g];
      }
      list.swap(out);
    };
    regroup(work);
    regroup(work_storage);
  }
  up((void*)s->d_work_storage, work_storage.data(), sizeof(int) * work_storage.size());
  s->nwork = nblocks;
  up((void*)s->d_work, work.data(), sizeof(int) * work.size());
  if (e == cudaSuccess) e = cudaMemsetAsync(M.part, 0, sizeof(double) * NPART * nblocks, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(M.sums, 0, sizeof(double) * NV * ninst, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(M.err, 0, sizeof(int) * 4, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_counter, 0, sizeof(int) * (MAXLEV + 4), s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);  // host vectors die here
  if (e != cudaSuccess) {
    delete s;
    return AMRVAC_E_CUDA;
  }
  *out = s;
  return AMRVAC_OK;
}

amrvac_status amrvac_state_destroy(amrvac_state* s) {
  if (!s) return AMRVAC_E_INVALID;
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (s->graph) cudaGraphExecDestroy(s->graph);
  delete s;
  return cuda_status(e);
}

static bool buffer_ok(int b) { return b >= 0 && b < 3; }

amrvac_status amrvac_set_conserved(amrvac_state* s, int32_t buffer, const void* src,
                                   int32_t src_is_device, int32_t src_precision) {
  if (!s || !src || !buffer_ok(buffer)) return AMRVAC_E_INVALID;
  if (src_precision != AMRVAC_FP64 && src_precision != AMRVAC_FP32_BULK) return AMRVAC_E_INVALID;
  const size_t n = (size_t)NV * s->nblocks * s->ncell;
  if (buffer == 0) s->dt_valid = false;
  cudaError_t e;
  if (src_precision == s->cfg.precision) {
    e = cudaMemcpyAsync(s->U[buffer], src, n * s->real_size,
                        src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        s->stream);
    return cuda_status(e);
  }
  if (src_is_device)
    return check_launch(s, launch_convert(s, src, src_precision, s->U[buffer], s->cfg.precision, n));
  // host source of the other precision: convert on the host
  if (s->cfg.precision == AMRVAC_FP64) {
    std::vector<double> tmp(n);
    const float* f = (const float*)src;
    for (size_t i = 0; i < n; i++) tmp[i] = f[i];
    e = cudaMemcpyAsync(s->U[buffer], tmp.data(), n * 8, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  } else {
    std::vector<float> tmp(n);
    const double* d = (const double*)src;
    for (size_t i = 0; i < n; i++) tmp[i] = (float)d[i];
    e = cudaMemcpyAsync(s->U[buffer], tmp.data(), n * 4, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  }
  return cuda_status(e);
}

amrvac_status amrvac_get_conserved(amrvac_state* s, int32_t buffer, void* dst,
                                   int32_t dst_is_device, int32_t dst_precision) {
  if (!s || !dst || !buffer_ok(buffer)) return AMRVAC_E_INVALID;
  if (dst_precision != AMRVAC_FP64 && dst_precision != AMRVAC_FP32_BULK) return AMRVAC_E_INVALID;
  const size_t n = (size_t)NV * s->nblocks * s->ncell;
  cudaError_t e;
  if (dst_precision == s->cfg.precision) {
    e = cudaMemcpyAsync(dst, s->U[buffer], n * s->real_size,
                        dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        s->stream);
    return cuda_status(e);
  }
  if (dst_is_device)
    return check_launch(s, launch_convert(s, s->U[buffer], s->cfg.precision, dst, dst_precision, n));
  if (s->cfg.precision == AMRVAC_FP64) {
    std::vector<double> tmp(n);
    e = cudaMemcpyAsync(tmp.data(), s->U[buffer], n * 8, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    float* f = (float*)dst;
    for (size_t i = 0; i < n; i++) f[i] = (float)tmp[i];
  } else {
    std::vector<float> tmp(n);
    e = cudaMemcpyAsync(tmp.data(), s->U[buffer], n * 4, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    double* d = (double*)dst;
    for (size_t i = 0; i < n; i++) d[i] = tmp[i];
  }
  return cuda_status(e);
}

amrvac_status amrvac_get_primitives(amrvac_state* s, int32_t buffer, void* d_dst) {
  if (!s || !d_dst || !buffer_ok(buffer)) return AMRVAC_E_INVALID;
  return check_launch(s, launch_to_primitive(s, buffer, d_dst));
}

static amrvac_status read_rt(amrvac_state* s, std::vector<InstRT>& rt) {
  rt.resize(s->ninst);
  cudaError_t e = cudaMemcpyAsync(rt.data(), s->mesh.rt, sizeof(InstRT) * s->ninst,
                                  cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return cuda_status(e);
}

static amrvac_status write_rt(amrvac_state* s, const std::vector<InstRT>& rt) {
  cudaError_t e = cudaMemcpyAsync(s->mesh.rt, rt.data(), sizeof(InstRT) * s->ninst,
                                  cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return cuda_status(e);
}

amrvac_status amrvac_set_time(amrvac_state* s, const double* h_t, const double* h_t_end) {
  if (!s) return AMRVAC_E_INVALID;
  std::vector<InstRT> rt;
  amrvac_status st = read_rt(s, rt);
  if (st) return st;
  for (int q = 0; q < s->ninst; q++) {
    if (h_t) rt[q].t = h_t[q];
    if (h_t_end) rt[q].t_end = h_t_end[q];
  }
  s->dt_valid = false;
  return write_rt(s, rt);
}

amrvac_status amrvac_set_dt(amrvac_state* s, const double* h_dt, const double* h_ch) {
  if (!s || !h_dt || !h_ch) return AMRVAC_E_INVALID;
  std::vector<InstRT> rt;
  amrvac_status st = read_rt(s, rt);
  if (st) return st;
  for (int q = 0; q < s->ninst; q++) {
    if (!(h_dt[q] >= 0.0) || !(h_ch[q] > 0.0)) return AMRVAC_E_INVALID;
    rt[q].dt = h_dt[q];
    rt[q].ch = h_ch[q];
  }
  st = write_rt(s, rt);
  if (!st) s->dt_valid = true;
  return st;
}

amrvac_status amrvac_fill_ghosts(amrvac_state* s, int32_t buffer, void* d_padded_out) {
  if (!s || !buffer_ok(buffer) || !d_padded_out) return AMRVAC_E_INVALID;
  return check_launch(s, launch_fill_ghosts(s, buffer, d_padded_out));
}

amrvac_status amrvac_cfl_dt(amrvac_state* s, int32_t buffer, double* h_dt_out) {
  if (!s || !buffer_ok(buffer)) return AMRVAC_E_INVALID;
  amrvac_status st = check_launch(s, launch_cfl_partials(s, buffer));
  if (st) return st;
  st = check_launch(s, launch_finalize(s, 0));
  if (st) return st;
  s->dt_valid = true;
  if (h_dt_out) {
    std::vector<InstRT> rt;
    st = read_rt(s, rt);
    if (st) return st;
    for (int q = 0; q < s->ninst; q++) h_dt_out[q] = rt[q].dt;
  }
  return AMRVAC_OK;
}

amrvac_status amrvac_stage(amrvac_state* s, int32_t stage) {
  if (!s || stage < 0 || stage >= num_stages(s->cfg.time)) return AMRVAC_E_INVALID;
  if (!s->dt_valid) return AMRVAC_E_STATE;
  int count = 0;
  amrvac_status st = enqueue_stage(s, stage, stage == num_stages(s->cfg.time) - 1, &count);
  s->launches += count;
  return st;
}

amrvac_status amrvac_step(amrvac_state* s, int32_t nsteps) {
  if (!s || nsteps < 0) return AMRVAC_E_INVALID;
  if (!s->dt_valid) {
    amrvac_status st = amrvac_cfl_dt(s, 0, nullptr);
    if (st) return st;
  }
  if (nsteps == 0) return AMRVAC_OK;
  if (s->stream == nullptr) {
    for (int n = 0; n < nsteps; n++) {
      int count = 0;
      amrvac_status st = enqueue_step(s, &count);
      s->launches += count;
      if (st) return st;
    }
    return AMRVAC_OK;
  }
  if (!s->graph) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return AMRVAC_E_CUDA;
    int count = 0;
    amrvac_status st = enqueue_step(s, &count);
    e = cudaStreamEndCapture(s->stream, &g);
    if (st || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return st ? st : AMRVAC_E_CUDA;
    }
    e = cudaGraphInstantiate(&s->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      s->graph = nullptr;
      return AMRVAC_E_CUDA;
    }
    s->graph_kernels = count;
  }
  for (int n = 0; n < nsteps; n++) {
    cudaError_t e = cudaGraphLaunch(s->graph, s->stream);
    if (e != cudaSuccess) return AMRVAC_E_CUDA;
    s->launches += s->graph_kernels;
  }
  return AMRVAC_OK;
}

amrvac_status amrvac_get_diag(amrvac_state* s, double* h_t, double* h_dt, double* h_ch,
                              double* h_sums, amrvac_error_info* err) {
  if (!s) return AMRVAC_E_INVALID;
  if (h_sums) {
    amrvac_status st = check_launch(s, launch_sums(s, 0));
    if (st) return st;
  }
  std::vector<InstRT> rt;
  amrvac_status st = read_rt(s, rt);
  if (st) return st;
  int e4[4];
  cudaError_t e = cudaMemcpy(e4, s->mesh.err, sizeof(e4), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && h_sums)
    e = cudaMemcpy(h_sums, s->mesh.sums, sizeof(double) * NV * s->ninst, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return AMRVAC_E_CUDA;
  for (int q = 0; q < s->ninst; q++) {
    if (h_t) h_t[q] = rt[q].t;
    if (h_dt) h_dt[q] = rt[q].dt;
    if (h_ch) h_ch[q] = rt[q].ch;
  }
  if (err) {
    err->code = e4[0];
    err->block = e4[1];
    err->cell = e4[2];
    err->var = e4[3];
  }
  return (amrvac_status)e4[0];
}

namespace {
struct SaveHeader {
  char magic[8];
  int32_t version, ndim, nx[3], nblocks, ninst, precision;
};
}  // namespace

amrvac_status amrvac_state_save(amrvac_state* s, const char* path) {
  if (!s || !path) return AMRVAC_E_INVALID;
  std::vector<InstRT> rt;
  amrvac_status st = read_rt(s, rt);
  if (st) return st;
  const size_t n = (size_t)NV * s->nblocks * s->ncell;
  std::vector<char> u(n * s->real_size);
  cudaError_t e = cudaMemcpyAsync(u.data(), s->U[0], u.size(), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return AMRVAC_E_CUDA;
  FILE* f = fopen(path, "wb");
  if (!f) return AMRVAC_E_INVALID;
  SaveHeader h;
  memcpy(h.magic, "AMRVACGB", 8);
  h.version = 1;
  h.ndim = s->ndim;
  for (int d = 0; d < 3; d++) h.nx[d] = s->cfg.block_nx[d];
  h.nblocks = s->nblocks;
  h.ninst = s->ninst;
  h.precision = s->cfg.precision;
  bool ok = fwrite(&h, sizeof(h), 1, f) == 1;
  ok = ok && fwrite(s->meta.data(), sizeof(int32_t), s->meta.size(), f) == s->meta.size();
  for (int q = 0; q < s->ninst && ok; q++) {
    double rec[5] = {rt[q].t, rt[q].t_end, rt[q].dt, rt[q].ch, s->dt_valid ? 1.0 : 0.0};
    ok = fwrite(rec, sizeof(rec), 1, f) == 1;
  }
  ok = ok && fwrite(u.data(), 1, u.size(), f) == u.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? AMRVAC_OK : AMRVAC_E_INVALID;
}

amrvac_status amrvac_state_load(amrvac_state* s, const char* path) {
  if (!s || !path) return AMRVAC_E_INVALID;
  FILE* f = fopen(path, "rb");
  if (!f) return AMRVAC_E_INVALID;
  SaveHeader h;
  bool ok = fread(&h, sizeof(h), 1, f) == 1 && memcmp(h.magic, "AMRVACGB", 8) == 0 &&
            h.version == 1 && h.ndim == s->ndim && h.nblocks == s->nblocks &&
            h.ninst == s->ninst && h.precision == s->cfg.precision;
  for (int d = 0; d < 3 && ok; d++) ok = h.nx[d] == s->cfg.block_nx[d];
  std::vector<int32_t> meta(s->meta.size());
  ok = ok && fread(meta.data(), sizeof(int32_t), meta.size(), f) == meta.size() && meta == s->meta;
  std::vector<InstRT> rt(s->ninst);
  bool dt_valid = true;
  for (int q = 0; q < s->ninst && ok; q++) {
    double rec[5];
    ok = fread(rec, sizeof(rec), 1, f) == 1;
    rt[q] = InstRT{rec[0], rec[1], rec[2], rec[3]};
    dt_valid = dt_valid && rec[4] != 0.0;
  }
  const size_t n = (size_t)NV * s->nblocks * s->ncell;
  std::vector<char> u(n * s->real_size);
  ok = ok && fread(u.data(), 1, u.size(), f) == u.size();
  fclose(f);
  if (!ok) return AMRVAC_E_INVALID;
  cudaError_t e = cudaMemcpyAsync(s->U[0], u.data(), u.size(), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return AMRVAC_E_CUDA;
  amrvac_status st = write_rt(s, rt);
  if (st) return st;
  s->dt_valid = dt_valid;
  return AMRVAC_OK;
}

amrvac_status amrvac_set_tuning(amrvac_state* s, const amrvac_tuning* t) {
  if (!s || !t || t->ctas_per_sm < 0 || t->ctas_per_sm > 32 || (t->order != 0 && t->order != 1) ||
      (t->dynamic != 0 && t->dynamic != 1) || (t->faces != 0 && t->faces != 1))
    return AMRVAC_E_INVALID;
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return AMRVAC_E_CUDA;
  s->tune = *t;
  s->d_work = t->order == 0 ? s->d_work_morton : s->d_work_storage;
  if (s->graph) {
    cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
  }
  return AMRVAC_OK;
}

amrvac_status amrvac_get_tuning(amrvac_state* s, amrvac_tuning* t) {
  if (!s || !t) return AMRVAC_E_INVALID;
  *t = s->tune;
  return AMRVAC_OK;
}

namespace {

std::string tuning_key(const amrvac_state* s) {
  int bucket = 0;
  while ((1 << (bucket + 1)) <= s->nblocks) bucket++;
  char buf[160];
  snprintf(buf, sizeof(buf), "d%d_n%dx%dx%d_p%d_f%d_l%d_pr%d_b%d", s->ndim, s->cfg.block_nx[0],
           s->cfg.block_nx[1], s->cfg.block_nx[2], s->cfg.precision, s->cfg.flux, s->cfg.limiter,
           s->cfg.pressure, bucket);
  return buf;
}

}  // namespace

amrvac_status amrvac_autotune(amrvac_state* s, int32_t trial_steps, const char* cache_path,
                              amrvac_tuning* best) {
  if (!s || trial_steps < 1) return AMRVAC_E_INVALID;
  const std::string key = tuning_key(s);
  if (cache_path) {
    if (FILE* f = fopen(cache_path, "r")) {
      char k[160];
      amrvac_tuning t{};
      amrvac_tuning found{};
      bool have = false;
      while (fscanf(f, "%159s %d %d %d %d %lf", k, &t.ctas_per_sm, &t.order, &t.dynamic,
                    &t.faces, &t.ms_per_step) == 6)
        if (key == k) found = t, have = true;  // the last entry for a key wins
      fclose(f);
      if (have) {
        amrvac_status st = amrvac_set_tuning(s, &found);
        if (!st && best) *best = found;
        return st;
      }
    }
  }
  if (!s->use_fused) {  // the plain path has no launch shape to tune
    amrvac_tuning t{0, 0, 0, 0, 0.0};
    if (best) *best = t;
    return amrvac_set_tuning(s, &t);
  }
  // back up U^n and the clocks: every trial starts from the same state
  std::vector<InstRT> rt0;
  amrvac_status st = read_rt(s, rt0);
  if (st) return st;
  const size_t bytes = (size_t)NV * s->nblocks * s->ncell * s->real_size;
  std::vector<char> u0(bytes);
  cudaError_t e = cudaMemcpyAsync(u0.data(), s->U[0], bytes, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return AMRVAC_E_CUDA;
  const bool valid0 = s->dt_valid;
  auto restore = [&]() -> amrvac_status {
    cudaError_t r = cudaMemcpyAsync(s->U[0], u0.data(), bytes, cudaMemcpyHostToDevice, s->stream);
    if (r == cudaSuccess) r = cudaStreamSynchronize(s->stream);
    if (r != cudaSuccess) return AMRVAC_E_CUDA;
    amrvac_status w = write_rt(s, rt0);
    s->dt_valid = valid0;
    return w;
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return AMRVAC_E_CUDA;
  // face pairs apply to the lean FP32 vanleer + HLLD scheme groups; their
  // kernel holds one CTA per SM, so only the default CTA count is tried
  bool pairs = s->cfg.precision == AMRVAC_FP32_BULK && !s->cfg.reflux &&
               s->cfg.time != AMRVAC_SSPRK54;
  bool eligible = false;
  for (int d = 0; d < s->cfg.ndim; d++)
    pairs = pairs && s->cfg.bc[d][0] != AMRVAC_BC_SYMMETRIC && s->cfg.bc[d][1] != AMRVAC_BC_SYMMETRIC;
  for (int g = 0; g < s->ngroups; g++)
    eligible = eligible || (s->grp_flux[g] == AMRVAC_FLUX_HLLD && s->grp_lim[g] == AMRVAC_LIM_VANLEER);
  pairs = pairs && eligible;
  amrvac_tuning cand[12];
  int nc = 0;
  for (int faces = 0; faces <= (pairs ? 1 : 0); faces++)
    for (int ctas : {0, 1})
      for (int order : {0, 1})
        for (int dyn : {0, 1})
          if (faces == 0 || ctas == 0) cand[nc++] = amrvac_tuning{ctas, order, dyn, faces, 0.0};
  amrvac_tuning win{0, 0, 0, 0, 1e300};
  for (int c = 0; c < nc && !st; c++) {
    st = amrvac_set_tuning(s, &cand[c]);
    if (!st) st = restore();
    if (!st) st = amrvac_step(s, 1);  // warm-up and graph capture
    if (st) break;
    if (cudaEventRecord(e0, s->stream) != cudaSuccess) st = AMRVAC_E_CUDA;
    if (!st) st = amrvac_step(s, trial_steps);
    if (!st && cudaEventRecord(e1, s->stream) != cudaSuccess) st = AMRVAC_E_CUDA;
    if (!st && cudaEventSynchronize(e1) != cudaSuccess) st = AMRVAC_E_CUDA;
    float ms = 0.f;
    if (!st && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = AMRVAC_E_CUDA;
    cand[c].ms_per_step = ms / trial_steps;
    if (!st && cand[c].ms_per_step < win.ms_per_step) win = cand[c];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) {
    restore();
    return st;
  }
  st = amrvac_set_tuning(s, &win);
  if (!st) st = restore();
  if (st) return st;
  if (best) *best = win;
  if (cache_path) {
    if (FILE* f = fopen(cache_path, "a")) {
      fprintf(f, "%s %d %d %d %d %.6f\n", key.c_str(), win.ctas_per_sm, win.order, win.dynamic,
              win.faces, win.ms_per_step);
      fclose(f);
    }
  }
  return AMRVAC_OK;
}

amrvac_status amrvac_clear_error(amrvac_state* s) {
  if (!s) return AMRVAC_E_INVALID;
  return cuda_status(cudaMemsetAsync(s->mesh.err, 0, sizeof(int) * 4, s->stream));
}

int64_t amrvac_launch_count(const amrvac_state* s) { return s ? s->launches : -1; }

}  // extern "C"
