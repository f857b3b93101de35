// Ghost values of the block-AMR mesh on the device.
//
// A ghost cell of a level-L block at global level-L cell index p takes
//   - the value of the level-L leaf cell covering p (same-level copy; periodic
//     wrap or zero-gradient clamp at the domain edge);
//   - the mean of its 2^d children when finer leaves cover p (restriction;
//     recursively when a child is refined again);
//   - the coarse value plus minmod-limited slopes times +-1/4 of a coarse cell
//     when a coarser leaf covers p (prolongation on conserved variables; the
//     slopes use the coarse-level values of the neighbouring coarse cells).
// The paper gives no formulas for these operators (AMR block exchange is only
// described in words, Sect. 1 and 8); this is our stated reading.  With full
// 2:1 balance (checked on the host) a face ghost needs at most two levels of
// restriction inside a prolongation stencil, so the lookups below are bounded.
#pragma once

#include "common.cuh"

namespace amrvac {

// bring p into the domain at level L of instance q: periodic wrap, outflow
// clamp (zero gradient), or the mirror cell across a symmetric wall; returns
// the mask of the dimensions mirrored (their normal momentum and field are to
// be negated, see wall_flip)
__device__ __forceinline__ int wrap_level(const DevMesh& M, int q, int L, int* p) {
  int mask = 0;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    if (d >= M.ndim) {
      p[d] = 0;
      continue;
    }
    int N = M.lnb[(q * MAXLEV + L) * 3 + d] * M.nx[d];
    if (p[d] < 0 || p[d] >= N) {
      const int bc = M.bc[d][p[d] < 0 ? 0 : 1];
      if (bc == AMRVAC_BC_PERIODIC) {
        p[d] = ((p[d] % N) + N) % N;
      } else if (bc == AMRVAC_BC_SYMMETRIC) {
        p[d] = p[d] < 0 ? -1 - p[d] : 2 * N - 1 - p[d];
        mask |= 1 << d;
      } else {
        p[d] = p[d] < 0 ? 0 : N - 1;
      }
    }
  }
  return mask;
}

// symmetric wall: negate the normal momentum and normal field of the
// dimensions in mask
template <class T> __device__ __forceinline__ void wall_flip(int mask, T* u) {
#pragma unroll
  for (int d = 0; d < 3; d++)
    if (mask & (1 << d)) {
      u[1 + d] = -u[1 + d];
      u[5 + d] = -u[5 + d];
    }
}

// map code of the level-L block containing the (in-domain) cell p; cell index
// within that block in *cell
__device__ __forceinline__ int map_at(const DevMesh& M, int q, int L, const int* p, int* cell) {
  const int* nb = M.lnb + (q * MAXLEV + L) * 3;
  int b0 = p[0] / M.nx[0], b1 = p[1] / M.nx[1], b2 = p[2] / M.nx[2];
  int c0 = p[0] - b0 * M.nx[0], c1 = p[1] - b1 * M.nx[1], c2 = p[2] - b2 * M.nx[2];
  *cell = (c2 * M.nx[1] + c1) * M.nx[0] + c0;
  return M.lmap[M.lmap_off[q * MAXLEV + L] + (b2 * nb[1] + b1) * nb[0] + b0];
}

template <class T>
__device__ __forceinline__ void read_cell(const DevMesh& M, const T* U, size_t vs, int b,
                                          int cell, T* out) {
  const T* src = U + (size_t)b * M.ncell + cell;
#pragma unroll
  for (int v = 0; v < NV; v++) out[v] = src[(size_t)v * vs];
}

// level-L value of the in-domain cell p where p is covered at level L or finer
// (depth <= 2)
template <class T>
__device__ void level_value_in(const DevMesh& M, const T* U, size_t vs, int q, int L,
                               const int* p, T* out) {
  int cell;
  int r = map_at(M, q, L, p, &cell);
  if (r >= 0) {
    read_cell(M, U, vs, r, cell, out);
    return;
  }
  if (r != MAP_REFINED || L + 1 >= MAXLEV) {
    latch_error(M.err, AMRVAC_E_STATE, -1, L, 0);
#pragma unroll
    for (int v = 0; v < NV; v++) out[v] = T(0);
    return;
  }
  const int n1 = M.ndim > 1 ? 2 : 1, n2 = M.ndim > 2 ? 2 : 1;
  // 1 / (number of children), exact (a power of two)
  const T inv = M.ndim == 3 ? T(0.125) : (M.ndim == 2 ? T(0.25) : T(0.5));
  T sum[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) sum[v] = T(0);
  // fast path: with even block edges the children of p are one 2^d cube of
  // cells in a single level-(L+1) block; when that block is a leaf, one lookup
  // and independent loads, summed in the order of the general loop below
  if ((M.nx[0] & 1) == 0 && (M.ndim < 2 || (M.nx[1] & 1) == 0) &&
      (M.ndim < 3 || (M.nx[2] & 1) == 0)) {
    int c0[3] = {2 * p[0], M.ndim > 1 ? 2 * p[1] : 0, M.ndim > 2 ? 2 * p[2] : 0};
    int cc;
    const int r2 = map_at(M, q, L + 1, c0, &cc);
    if (r2 >= 0) {
      const T* src = U + (size_t)r2 * M.ncell + cc;
      const int sy = M.nx[0], sz = M.nx[0] * M.nx[1];
#pragma unroll
      for (int oz = 0; oz < 2; oz++)
#pragma unroll
        for (int oy = 0; oy < 2; oy++)
#pragma unroll
          for (int ox = 0; ox < 2; ox++) {
            if (oz >= n2 || oy >= n1) continue;
            const int off = ox + oy * sy + oz * sz;
#pragma unroll
            for (int v = 0; v < NV; v++) sum[v] += src[(size_t)v * vs + off];
          }
#pragma unroll
      for (int v = 0; v < NV; v++) out[v] = sum[v] * inv;
      return;
    }
  }
  for (int oz = 0; oz < n2; oz++)
    for (int oy = 0; oy < n1; oy++)
      for (int ox = 0; ox < 2; ox++) {
        int c[3] = {2 * p[0] + ox, M.ndim > 1 ? 2 * p[1] + oy : 0, M.ndim > 2 ? 2 * p[2] + oz : 0};
        int cc;
        int r2 = map_at(M, q, L + 1, c, &cc);
        T tmp[NV];
        if (r2 >= 0) {
          read_cell(M, U, vs, r2, cc, tmp);
        } else if (r2 == MAP_REFINED && L + 2 < MAXLEV) {
          T s2[NV];
#pragma unroll
          for (int v = 0; v < NV; v++) s2[v] = T(0);
          for (int gz = 0; gz < n2; gz++)
            for (int gy = 0; gy < n1; gy++)
              for (int gx = 0; gx < 2; gx++) {
                int g[3] = {2 * c[0] + gx, M.ndim > 1 ? 2 * c[1] + gy : 0,
                            M.ndim > 2 ? 2 * c[2] + gz : 0};
                int gc;
                int r3 = map_at(M, q, L + 2, g, &gc);
                T t3[NV];
                if (r3 >= 0) {
                  read_cell(M, U, vs, r3, gc, t3);
                } else {
                  latch_error(M.err, AMRVAC_E_STATE, -1, L + 2, 1);
#pragma unroll
                  for (int v = 0; v < NV; v++) t3[v] = T(0);
                }
#pragma unroll
                for (int v = 0; v < NV; v++) s2[v] += t3[v];
              }
#pragma unroll
          for (int v = 0; v < NV; v++) tmp[v] = s2[v] * inv;
        } else {
          latch_error(M.err, AMRVAC_E_STATE, -1, L + 1, 2);
#pragma unroll
          for (int v = 0; v < NV; v++) tmp[v] = T(0);
        }
#pragma unroll
        for (int v = 0; v < NV; v++) sum[v] += tmp[v];
      }
#pragma unroll
  for (int v = 0; v < NV; v++) out[v] = sum[v] * inv;
}

template <class T> __device__ __forceinline__ T minmod_g(T a, T b) {
  return (a * b > T(0)) ? ((a > T(0)) ? fmin(a, b) : fmax(a, b)) : T(0);
}

// level-L value of cell p (anywhere near the domain) where p is covered at
// level L or finer
template <class T>
__device__ void level_value_down(const DevMesh& M, const T* U, size_t vs, int q, int L,
                                 const int* pin, T* out) {
  int p[3] = {pin[0], pin[1], pin[2]};
  const int mask = wrap_level(M, q, L, p);
  level_value_in(M, U, vs, q, L, p, out);
  if (mask) wall_flip(mask, out);
}

// General ghost value of the in-domain level-L cell p of instance q (any
// coverage).
template <class T>
__device__ void ghost_value_in(const DevMesh& M, const T* U, size_t vs, int q, int L,
                               const int* p, T* out) {
  int cell;
  int r = map_at(M, q, L, p, &cell);
  if (r >= 0) {
    read_cell(M, U, vs, r, cell, out);
    return;
  }
  if (r == MAP_REFINED) {
    level_value_in(M, U, vs, q, L, p, out);
    return;
  }
  if (L == 0) {
    latch_error(M.err, AMRVAC_E_STATE, -1, 0, 3);
#pragma unroll
    for (int v = 0; v < NV; v++) out[v] = T(0);
    return;
  }
  // prolongation from the coarse cell c = floor(p/2) at level L-1
  int c[3], o[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    c[d] = d < M.ndim ? (p[d] >> 1) : 0;
    o[d] = p[d] - 2 * c[d];
  }
  T uc[NV];
  level_value_down(M, U, vs, q, L - 1, c, uc);
#pragma unroll
  for (int v = 0; v < NV; v++) out[v] = uc[v];
  for (int d = 0; d < M.ndim; d++) {
    int cm[3] = {c[0], c[1], c[2]}, cp[3] = {c[0], c[1], c[2]};
    cm[d] -= 1;
    cp[d] += 1;
    T um[NV], up[NV];
    level_value_down(M, U, vs, q, L - 1, cm, um);
    level_value_down(M, U, vs, q, L - 1, cp, up);
    T w = o[d] == 0 ? T(-0.25) : T(0.25);
#pragma unroll
    for (int v = 0; v < NV; v++) out[v] = out[v] + w * minmod_g(uc[v] - um[v], up[v] - uc[v]);
  }
}

// General ghost value of the level-L cell p of instance q, p anywhere near the
// domain (wrapped, clamped or mirrored first).
template <class T>
__device__ void ghost_value(const DevMesh& M, const T* U, size_t vs, int q, int L,
                            const int* pin, T* out) {
  int p[3] = {pin[0], pin[1], pin[2]};
  const int mask = wrap_level(M, q, L, p);
  ghost_value_in(M, U, vs, q, L, p, out);
  if (mask) wall_flip(mask, out);
}

// Conserved values of cell (i, j, k) (block-local, at most one index outside
// [0, n)) of block b: interior read, same-level neighbour read, outflow clamp,
// mirror across a symmetric wall, or the general AMR lookup.
template <class T>
__device__ __forceinline__ void block_cell_value(const DevMesh& M, const T* U, size_t vs, int b,
                                                 int i, int j, int k, T* out) {
  int c[3] = {i, j, k};
  int d = -1;
#pragma unroll
  for (int e = 0; e < 3; e++)
    if (c[e] < 0 || c[e] >= M.nx[e]) d = e;
  if (d < 0) {
    read_cell(M, U, vs, b, (k * M.nx[1] + j) * M.nx[0] + i, out);
    return;
  }
  int side = c[d] < 0 ? 0 : 1;
  int nb = M.nbr[b * 6 + d * 2 + side];
  if (nb >= 0) {
    c[d] += side ? -M.nx[d] : M.nx[d];
    read_cell(M, U, vs, nb, (c[2] * M.nx[1] + c[1]) * M.nx[0] + c[0], out);
  } else if (nb == NBR_OUTFLOW) {
    c[d] = side ? M.nx[d] - 1 : 0;
    read_cell(M, U, vs, b, (c[2] * M.nx[1] + c[1]) * M.nx[0] + c[0], out);
  } else if (nb == NBR_WALL) {
    c[d] = side ? 2 * M.nx[d] - 1 - c[d] : -1 - c[d];
    read_cell(M, U, vs, b, (c[2] * M.nx[1] + c[1]) * M.nx[0] + c[0], out);
    wall_flip(1 << d, out);
  } else {
    const int* bi = M.blk + b * 5;
    int p[3] = {bi[2] * M.nx[0] + i, bi[3] * M.nx[1] + j, bi[4] * M.nx[2] + k};
    ghost_value(M, U, vs, bi[0], bi[1], p, out);
  }
}

}  // namespace amrvac
