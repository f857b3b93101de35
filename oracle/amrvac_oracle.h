/*
 * FP64 CPU oracle for the ideal-MHD + GLM block update of MPI-AMRVAC 3.0
 * (Keppens et al. 2023, Sect. 3: conservative finite volumes in each substep of
 * an SSPRK scheme, limited reconstruction of primitives, HLL/HLLD fluxes,
 * glm monopole control, CFL time step).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is used by the tests, by the smoke
 * check and by the CPU-baseline leg of the benchmark.  The GPU library never
 * includes, links or calls it, and it shares no source with the GPU library.
 *
 * Everything is plain nested loops in double precision, compiled with
 * -ffp-contract=off.  Every quantity follows the method's definition with no
 * blocking or fusion.  Points where the paper names a method without printing
 * its formula are resolved by the published method it cites (Harten 1983 for
 * HLL, Miyoshi & Kusano 2005 for HLLD, Dedner 2002 for glm, Gottlieb 2005 and
 * Spiteri & Ruuth 2002 for SSPRK, van Leer 1974 and Koren 1993 for the
 * limiters); the readings are listed at each function.
 */
#ifndef AMRVAC_ORACLE_H
#define AMRVAC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_NVAR 9

typedef struct {
  int ndim;              /* 1, 2 or 3 */
  int nx[3];             /* cells per block per dimension (1 for unused dims) */
  int flux;              /* 0 hll, 1 hlld, 2 tvdlf, 3 hllc */
  int limiter;           /* 0 minmod, 1 vanleer, 2 koren, 3 superbee, 4 woodward,
                            5 mcbeta, 6 albada, 10 cada3; 7 mp5, 8 weno5,
                            9 wenoz5, 11 wenozp5 (five-point, 3 ghost cells) */
  int time;              /* 0 ssprk(2,2), 1 ssprk(3,3), 2 ssprk(4,3), 3 ssprk(5,4) */
  int glm;               /* 1: Dedner glm cleaning; 0: none (psi stays 0) */
  double glm_alpha;      /* psi damping parameter alpha_p */
  double courant;
  int bc[3][2];          /* 0 periodic, 1 outflow (zero gradient), 2 symmetric
                            (reflecting wall: mirror, normal m and B negated) */
  double small_density, small_pressure;
  int check_small_values;
  int fix_small_values;  /* 0 off, 1 replace, 2 average (Sect. 7.4 bootstrapping) */
  int reflux;            /* 1: coarse fluxes at level changes replaced by the mean
                            of the fine fluxes (conservative AMR) */
  int level_flux[16];    /* per AMR level: flux scheme of that level's blocks,
                            -1 = flux (Sect. 3: schemes may differ per level) */
  int level_limiter[16]; /* per AMR level: limiter, -1 = limiter */
} orc_config;

typedef struct {
  double xmin[3], xmax[3];
  int base[3];           /* level-0 blocks per dimension */
  double gamma;
} orc_instance;

typedef struct orc_mesh orc_mesh;

/* Builds the mesh; returns NULL and writes a message into err on an invalid
 * block list (overlap, hole, not 2:1 balanced across faces, edges, corners). */
orc_mesh* orc_create(const orc_config* cfg, int ninst, const orc_instance* inst,
                     int nblocks, const int32_t* meta, char* err, int errlen);
void orc_destroy(orc_mesh* m);
void orc_set_threads(orc_mesh* m, int nthreads);

/* Ghost fill: padded [var][block][(nx+2g)(ny+2g)(nz+2g) over active dims],
 * g = orc_ghost_width (3 when a level uses a five-point limiter, else 2);
 * interior and the g-deep face slabs are written, edge/corner cells are 0. */
int orc_fill_ghosts(const orc_mesh* m, const double* U, double* padded);
int orc_ghost_width(const orc_mesh* m);

/* Refluxing (with cfg.reflux) is part of every stage over all blocks: after
 * the update, the coarse cell next to a face whose neighbour is finer gets
 *   out += b c dt (+-) (F_coarse - mean of the 2^(d-1) fine fluxes) / dx,
 * + for the high face and - for the low face of the coarse cell (psi of the
 * Euler part times its damping factor; likewise for out2).  The stored face
 * fluxes are those of the same stage.  A stage restricted to a block subset
 * does not reflux. */

/* One SSPRK stage k on the listed blocks (all when sub == NULL):
 * out = a_k U0 + b_k (Uk + c_k dt L(Uk)), psi of the Euler part damped over
 * c_k dt (coefficients: orc_stage_coeffs6).  dt, ch are per instance.  Returns
 * 0 or 4 (small values found). */
int orc_stage(const orc_mesh* m, int k, const double* dt, const double* ch,
              const double* U0, const double* Uk, double* out,
              const int32_t* sub, int nsub);
/* The same with the second output of SSPRK(5,4) stage 3:
 * out2 = a2 U2 + b2 (Uk + c2 dt L(Uk)) when out2 != NULL and b2 != 0.  out may
 * be U2's array and out2 U0's (each cell is read before it is written). */
int orc_stage2(const orc_mesh* m, int k, const double* dt, const double* ch,
               const double* U0, const double* Uk, const double* U2, double* out,
               double* out2, const int32_t* sub, int nsub);

/* Bootstrapping of Sect. 7.4 on the state U in place: a cell is small when
 * rho < small_density or p < small_pressure, or either is not positive.  method 1 (replace): rho and p
 * floored to the small values, v = m/rho kept (0 if rho <= 0); method 2
 * (average): rho, v, p become the mean over the cell's face neighbours of its
 * own level that are not small themselves (the replace rule when there is
 * none).  B and psi are never changed; m and e follow from the new primitives.
 * All small cells are found before any is changed.  Returns the number of
 * cells fixed. */
long orc_fix_small(const orc_mesh* m, double* U, int method);

/* CFL: per instance dt = courant / max sum_d (|v_d|+c_f,d)/dx_d and
 * ch = max (|v_d|+c_f,d); dt clipped to t_end - t. */
int orc_cfl(const orc_mesh* m, const double* U, const double* t, const double* t_end,
            double* dt, double* ch);

/* Integral of every conserved variable per instance: sums[inst][var]. */
void orc_sums(const orc_mesh* m, const double* U, double* sums);

/* Full steps: CFL dt (or fixed_dt > 0), all stages, t += dt.  Stops early when
 * every instance reached t_end.  Returns the status; *nsteps_done written. */
int orc_run(orc_mesh* m, double* U, double* t, const double* t_end, int maxsteps,
            double fixed_dt, int* nsteps_done);

/* Pointwise pieces, exposed for the pin tests. */
void orc_cons_to_prim(double gamma, const double* u, double* w);
void orc_prim_to_cons(double gamma, const double* w, double* u);
double orc_fast_speed(double gamma, const double* w, int dir);
/* reconstruction of a 1D array: left state at i+1/2 (wl[i]) and right state at
 * i-1/2 (wr[i]) from cell i, for 1 <= i <= n-2 */
void orc_reconstruct(int limiter, const double* w, int n, double* wl, double* wr);
/* the same for the five-point limiters (7, 8, 9, 11), for 2 <= i <= n-3; dx:
 * the cell width (wenozp5's lambda = dx^(2/3)) */
void orc_reconstruct5(int limiter, const double* w, int n, double dx, double* wl, double* wr);
/* face flux along dir from primitive face states (global frame) */
void orc_face_flux(int flux, int glm, double gamma, double ch, int dir,
                   const double* wl, const double* wr, double* f);
/* stage coefficients a_k, b_k used by orc_stage */
void orc_stage_coeffs(int time, int k, double* a, double* b);
/* all six: {a, b, c, a2, b2, c2} */
void orc_stage_coeffs6(int time, int k, double* co);
int orc_num_stages(int time);

#ifdef __cplusplus
}
#endif
#endif
