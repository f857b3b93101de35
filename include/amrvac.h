/*
 * amrvac.h - C ABI of the GB300 (sm_103a) ideal-MHD block-update library.
 *
 * The library advances the ideal-MHD equations with glm divergence cleaning on
 * the blocks of a block-structured adaptive mesh, with the explicit
 * finite-volume scheme of MPI-AMRVAC 3.0 (Keppens et al. 2023):
 *   - conserved cell averages updated by interface fluxes in every substep of
 *     an SSPRK(2,2), (3,3), (4,3) or (5,4) scheme (Sect. 3, time-integration
 *     table);
 *   - limited reconstruction of primitive variables to two face states per
 *     interface with a limiter of the limiter table (Sect. 3.1.1): seven
 *     two-ghost-cell ones and three five-point ones (amrvac_limiter);
 *   - HLL (Harten 1983), HLLD (Miyoshi & Kusano 2005), TVDLF or HLLC interface
 *     fluxes (flux-scheme table of Sect. 3; Sect. 3.2.1), per AMR level if
 *     asked (level_flux / level_limiter);
 *   - `glm` monopole control (Dedner 2002; table of Sect. 3.2.2);
 *   - the CFL-limited explicit time step (Sect. 3);
 *   - ghost cells filled from same-level neighbours, from finer neighbours by
 *     restriction and from coarser neighbours by limited prolongation, i.e. the
 *     internal boundary exchange of the AMR hierarchy (Sect. 8 describes its
 *     MPI form; here it is a read from the device block pool); periodic,
 *     outflow or reflecting domain boundaries;
 *   - optional refluxing at level changes, bootstrapping of small values
 *     (Sect. 7.4) and dynamic regridding (amrvac_regrid_*).
 * One explicit substep is the paper's advect1(alpha dt, t_a, u^a, t_b, u^b) of
 * Sect. 4.2: u^b <- u^b + alpha dt F_ex(u^a) together with its boundary update.
 *
 * Conventions for every call:
 *   - Every function returns an amrvac_status and never aborts the process.
 *   - Device memory is owned by the caller: the library borrows the workspace
 *     passed to amrvac_state_create for the state's lifetime and never frees
 *     it; it allocates no device memory itself.  Host arrays are copied on call.
 *   - All device work is enqueued on the stream given at creation, in call
 *     order, and is asynchronous unless a host output pointer is given.  A
 *     state is not thread-safe.
 *   - Conserved variables, 9 per cell, in this order: rho, m_x, m_y, m_z, e,
 *     B_x, B_y, B_z, psi; B in units where the magnetic pressure is B^2/2, so
 *     p = (gamma - 1)(e - m^2/(2 rho) - B^2/2).  Three vector components are
 *     always stored, in 1D and 2D too.
 *   - Array layout [var][block][cell], cells x-fastest within a block,
 *     interior cells only (ghost cells are never stored).
 *   - Errors found on the device (small density or pressure, inconsistent
 *     mesh lookups) are latched in a device status word and reported by the
 *     next amrvac_get_diag or by any call that synchronises.
 */
#ifndef AMRVAC_H
#define AMRVAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AMRVAC_NVAR 9
#define AMRVAC_MAX_LEVELS 16
#define AMRVAC_NOALLOC_MAX_BLOCKS 65536
/* largest block: interior cells per block (product of block_nx over the active
 * dimensions, each 4..4096); larger blocks are rejected with AMRVAC_E_INVALID */
#define AMRVAC_MAX_BLOCK_CELLS (1 << 24)

typedef enum {
  AMRVAC_OK = 0,
  AMRVAC_E_INVALID = 1,      /* bad argument, config or block list            */
  AMRVAC_E_NOMEM = 2,        /* workspace too small                           */
  AMRVAC_E_CUDA = 3,         /* a CUDA runtime call failed                    */
  AMRVAC_E_SMALL_VALUES = 4, /* density or pressure at or below its floor (Sect. 7.4:
                                check_small_values stops and reports)         */
  AMRVAC_E_TIMEOUT = 5,      /* reserved: a bounded device wait gave up       */
  AMRVAC_E_STATE = 6         /* call out of order, or a mesh lookup failed    */
} amrvac_status;

/* flux-scheme table of Sect. 3.2.1: HLL (Harten 1983), HLLD (Miyoshi & Kusano
 * 2005), TVD Lax-Friedrichs (local LF with the fastest signal speed), HLLC for
 * MHD (the three-wave solver of Li 2005) */
typedef enum {
  AMRVAC_FLUX_HLL = 0,
  AMRVAC_FLUX_HLLD = 1,
  AMRVAC_FLUX_TVDLF = 2,
  AMRVAC_FLUX_HLLC = 3
} amrvac_flux;
/* limiters of the limiter table (Sect. 3.1.1).  Two ghost cells: minmod, van
 * Leer 1974, Koren 1993 (third order), superbee (Roe 1985), woodward
 * (monotonized central, van Leer 1977), mcbeta (beta = 1.4), van Albada 1982
 * (TVD form), cada3 (the compact third-order limiter function of Cada &
 * Torrilhon 2009: phi(theta) = max(0, min(phi3, max(-theta/2, min(2 theta,
 * phi3, 1.6)))), phi3 = (2 + theta)/3, theta = dm/dp; it keeps a slope at
 * extrema), venk (Venkatakrishnan 1995 in 1D form: the central increment
 * (c - a)/4 to each face times the smooth factor (D^2 + 2 D d)/(D^2 + 2 d^2 +
 * D d), d the face's increment and D the stencil's range beyond the cell value
 * on d's side, the smaller of the cell's two factors; no smoothing constant).
 * Three ghost cells (five-point, fifth order on smooth data): mp5
 * (Suresh & Huynh 1997), weno5 (Jiang & Shu 1996, eps = 1e-6), wenoz5 (Borges
 * et al. 2008, exponent 1), wenozp5 (WENO-Z+ of Acker, Borges & Costa 2016:
 * the Z weights with exponent 2 plus lambda (beta_k + eps)/(tau5 + eps),
 * lambda = dx^(2/3) of the block's level along the reconstruction).  They
 * need three ghost layers: the fused kernels take them when every level uses a
 * five-point limiter, on 2D 16x16 tiles (22x22 tiles) and on 3D 16^3 blocks in
 * FP32 bulk (a ring of six 22x22 planes, one CTA per SM), with three-layer
 * ghost slabs at level changes; otherwise (3D in FP64, or a mesh mixing two-
 * and five-point levels) they run on the PLAIN kernels (AUTO picks PLAIN,
 * FUSED is rejected). */
typedef enum {
  AMRVAC_LIM_MINMOD = 0,
  AMRVAC_LIM_VANLEER = 1,
  AMRVAC_LIM_KOREN = 2,
  AMRVAC_LIM_SUPERBEE = 3,
  AMRVAC_LIM_WOODWARD = 4,
  AMRVAC_LIM_MCBETA = 5,
  AMRVAC_LIM_ALBADA = 6,
  AMRVAC_LIM_MP5 = 7,
  AMRVAC_LIM_WENO5 = 8,
  AMRVAC_LIM_WENOZ5 = 9,
  AMRVAC_LIM_CADA3 = 10,
  AMRVAC_LIM_WENOZP5 = 11,
  AMRVAC_LIM_VENK = 12
} amrvac_limiter;
/* time-integration table of Sect. 3: SSPRK(2,2), SSPRK(3,3) (Gottlieb 2005),
 * SSPRK(4,3) and SSPRK(5,4) (Spiteri & Ruuth 2002) */
typedef enum {
  AMRVAC_SSPRK2 = 0,
  AMRVAC_SSPRK3 = 1,
  AMRVAC_SSPRK43 = 2,
  AMRVAC_SSPRK54 = 3
} amrvac_time;
/* FP64: state and arithmetic in double.  FP32_BULK: state and stencil/Riemann
 * arithmetic in float; thermal pressure recovered from the total energy in
 * double; conservation sums and the time step in double. */
typedef enum { AMRVAC_FP64 = 0, AMRVAC_FP32_BULK = 1 } amrvac_precision;
/* Boundaries: PERIODIC (both sides of a dimension); OUTFLOW (zero gradient: a
 * ghost takes the nearest in-domain cell of its level); SYMMETRIC (reflecting
 * wall: a ghost takes the mirror cell across the boundary with the normal
 * momentum and the normal magnetic field negated; density, pressure,
 * tangential components and psi are even). */
typedef enum {
  AMRVAC_BC_PERIODIC = 0,
  AMRVAC_BC_OUTFLOW = 1,
  AMRVAC_BC_SYMMETRIC = 2
} amrvac_bc;
/* Thermal-pressure recovery in FP32_BULK: the subtraction e - m^2/(2 rho) -
 * B^2/2 (and the per-thread conservation sums) in double (FP64), or in
 * float-float (FF, a pair of floats with a ~48-bit significand: the B_i^2 are
 * exact via FMA, e - m^2/(2 rho) exact via TwoSum), which avoids the scarce
 * FP64 units of GB300 at equal accuracy for float-stored inputs.  Ignored for
 * AMRVAC_FP64 states. */
typedef enum { AMRVAC_PRESSURE_FP64 = 0, AMRVAC_PRESSURE_FF = 1 } amrvac_pressure;
/* PLAIN: one kernel per step of the method per stage, staging primitives and
 * face fluxes in workspace scratch (the per-block baseline).  FUSED: one
 * persistent kernel per stage doing ghost fill, reconstruction, flux, update
 * and the time-step reduction with shared-memory staging.  AUTO picks FUSED
 * for 16x16 (2D) and 16x16x16 (3D) blocks, PLAIN otherwise. */
typedef enum { AMRVAC_KERNEL_AUTO = 0, AMRVAC_KERNEL_PLAIN = 1, AMRVAC_KERNEL_FUSED = 2 } amrvac_kernel;
/* fix_small_values (bootstrapping, Sect. 7.4).  A cell is small when its
 * density is below small_density or its pressure below small_pressure, or
 * either is not positive.  OFF: small stage inputs are reported
 * (check_small_values).  REPLACE: after every stage the small cells of its
 * output get rho = max(rho, small_density), p = max(p, small_pressure) with the
 * velocity kept (0 where rho <= 0).  AVERAGE: rho, v and p of a small cell
 * become the mean over its face neighbours of the same level that are not small
 * (REPLACE where there is none).  B and psi are never changed; momentum and
 * energy follow from the new primitives.  Both need positive floors. */
typedef enum { AMRVAC_FIX_OFF = 0, AMRVAC_FIX_REPLACE = 1, AMRVAC_FIX_AVERAGE = 2 } amrvac_fix;

typedef struct {
  int32_t ndim;           /* 1, 2 or 3                                          */
  int32_t block_nx[3];    /* interior cells per block and dimension (4..4096 in
                             active dims, at most AMRVAC_MAX_BLOCK_CELLS cells
                             per block; entries of unused dims are ignored)    */
  int32_t flux;           /* amrvac_flux                                        */
  int32_t limiter;        /* amrvac_limiter                                     */
  int32_t time;           /* amrvac_time                                        */
  int32_t precision;      /* amrvac_precision                                   */
  int32_t glm;            /* 1: glm cleaning (psi evolves); 0: psi stays 0      */
  double glm_alpha;       /* psi damping: psi *= exp(-glm_alpha c_h dt / dx_min)
                             after every Euler sub-step                         */
  double courant;         /* CFL number C (Sect. 3)                             */
  int32_t bc[3][2];       /* amrvac_bc per dimension and side                  */
  double small_density;   /* check_small_values floors (Sect. 7.4)             */
  double small_pressure;
  int32_t check_small_values;
  int32_t kernel;         /* amrvac_kernel                                      */
  int32_t pressure;       /* amrvac_pressure (FP32_BULK only)                   */
  int32_t fix_small_values; /* amrvac_fix                                       */
  int32_t reflux;         /* 1: conservative coarse-fine flux correction: after
                             every stage the coarse cell next to a finer
                             neighbour replaces that face's flux by the mean of
                             the fine fluxes through it, so AMR runs conserve
                             to round-off (off: level changes are not exactly
                             conservative)                                     */
  /* per AMR level (Sect. 3: the scheme may differ between levels): flux and
   * limiter of that level's blocks, every face of a block computed with its
   * block's scheme; 0 = the global flux / limiter above, v + 1 = amrvac_flux /
   * amrvac_limiter v (so a zero-initialised config has no overrides) */
  int32_t level_flux[AMRVAC_MAX_LEVELS];
  int32_t level_limiter[AMRVAC_MAX_LEVELS];
} amrvac_config;

/* One instance = one independent domain with its own gamma and clock. */
typedef struct {
  double xmin[3], xmax[3];
  int32_t base_blocks[3]; /* level-0 blocks per dimension                       */
  double gamma;
  double t0, t_end;       /* the time step is clipped so that t never passes t_end */
} amrvac_instance_desc;

typedef struct {
  int32_t code;           /* amrvac_status of the first device error, 0 if none */
  int32_t block;          /* block index, cell index and variable where it was found */
  int32_t cell;
  int32_t var;
} amrvac_error_info;

typedef struct amrvac_state amrvac_state;

/*
 * Workspace size in bytes for a mesh; the caller allocates that much device
 * memory (any allocator) and passes it to amrvac_state_create.
 * block_meta: host int32 [nblocks][5] = (instance, level, i, j, k); level 0 is
 * the base level, (i, j, k) the block index at that level (unused dims 0).
 * The leaves must tile every instance's domain without overlap and be graded
 * 2:1 across faces, edges and corners; otherwise AMRVAC_E_INVALID.
 */
amrvac_status amrvac_workspace_bytes(const amrvac_config* cfg, int32_t ninst,
                                     const amrvac_instance_desc* inst, int32_t nblocks,
                                     const int32_t* block_meta, size_t* bytes);

/*
 * Builds the mesh tables (neighbour table, per-level block maps) on the host,
 * uploads them into the workspace and returns a state.  d_workspace must be
 * 256-byte aligned and hold amrvac_workspace_bytes bytes.  cuda_stream is a
 * cudaStream_t; graph capture in amrvac_step needs a stream other than the
 * legacy default stream (0), otherwise steps are launched without a graph.
 */
amrvac_status amrvac_state_create(const amrvac_config* cfg, int32_t ninst,
                                  const amrvac_instance_desc* inst, int32_t nblocks,
                                  const int32_t* block_meta, void* d_workspace,
                                  size_t workspace_bytes, void* cuda_stream,
                                  amrvac_state** out);
amrvac_status amrvac_state_destroy(amrvac_state* s);

/*
 * Copies conserved variables into (set) or out of (get) state buffer 0, 1 or 2.
 * Buffer 0 holds U^n; 1 and 2 are the SSPRK stage registers.  src/dst are
 * [var][block][cell] arrays in src_precision / dst_precision (AMRVAC_FP64 =
 * double, AMRVAC_FP32_BULK = float), on the device (is_device = 1) or the host.
 * Host copies of the state's own precision are asynchronous (page-locked
 * memory is then required to stay valid until the stream reaches the copy);
 * others synchronise.
 */
amrvac_status amrvac_set_conserved(amrvac_state* s, int32_t buffer, const void* src,
                                   int32_t src_is_device, int32_t src_precision);
amrvac_status amrvac_get_conserved(amrvac_state* s, int32_t buffer, void* dst,
                                   int32_t dst_is_device, int32_t dst_precision);

/*
 * Primitive variables of buffer (the paper's snapshots can hold primitive
 * instead of conserved variables, Sect. 7.5): (rho, v_x, v_y, v_z, p, B_x,
 * B_y, B_z, psi) of every interior cell into d_dst (device memory of the
 * caller, the state's precision, the conserved layout [var][block][cell]), with
 * p = (gamma - 1)(e - m.v/2 - B^2/2) recovered exactly as the stage kernels
 * recover it: in double for FP64 states; for FP32-bulk states in float-float
 * (AMRVAC_PRESSURE_FF) or with the subtraction in double (AMRVAC_PRESSURE_FP64),
 * the kinetic part formed in float.  Asynchronous on the state's stream.
 */
amrvac_status amrvac_get_primitives(amrvac_state* s, int32_t buffer, void* d_dst);

/* Per-instance clock: t (host array [ninst]) and t_end.  Marks dt invalid. */
amrvac_status amrvac_set_time(amrvac_state* s, const double* h_t, const double* h_t_end);

/*
 * Ghost fill of buffer into d_padded_out (device, state precision):
 * [var][block][padded cell] with (n_d + 2 g) cells per active dimension, g = 3
 * when the limiter or a level's limiter is a five-point one, else 2; the
 * interior and the g-deep face slabs are written, edge and corner cells are
 * set to 0 (the unsplit scheme reads face ghosts only).  Same-level copy,
 * periodic wrap, zero-gradient outflow, restriction (mean of the 2^d children)
 * and prolongation (coarse value plus minmod-limited slopes times 1/4 of a
 * coarse cell, on conserved variables).
 */
amrvac_status amrvac_fill_ghosts(amrvac_state* s, int32_t buffer, void* d_padded_out);

/*
 * CFL time step of buffer (Sect. 3): per instance dt = C / max over cells of
 * sum_d (|v_d| + c_f,d)/dx_d, clipped to t_end - t, and the glm speed
 * c_h = max over cells and d of (|v_d| + c_f,d).  Stored on the device for the
 * next stages; also copied to h_dt_out[ninst] when it is not NULL (synchronises).
 */
amrvac_status amrvac_cfl_dt(amrvac_state* s, int32_t buffer, double* h_dt_out);

/* Overrides the device dt and c_h of every instance (host arrays [ninst]). */
amrvac_status amrvac_set_dt(amrvac_state* s, const double* h_dt, const double* h_ch);

/*
 * One SSPRK stage k (0-based) with the device-resident dt and c_h, i.e. one
 * advect1 substep plus the convex combination of the Shu-Osher form:
 *   out = a_k U0 + b_k (U_in + c_k dt L(U_in)),
 * psi of the Euler part damped by exp(-alpha c_h c_k dt / dx_min).
 *   SSPRK2  (a,b,c): (0,1,1), (1/2,1/2,1)
 *   SSPRK3:  (0,1,1), (3/4,1/4,1), (1/3,2/3,1)
 *   SSPRK43: (0,1,1/2), (0,1,1/2), (2/3,1/3,1/2), (0,1,1/2)
 *   SSPRK54: the Spiteri-Ruuth scheme; stage 3 also writes
 *            w = a2 u2 + b2 (u3 + c2 dt L(u3)) and stage 4 is
 *            u5 = w + b4 (u4 + c4 dt L(u4)) (U0 = w).
 * Buffers (U0, U_in [, U2] -> out [, out2]): stage 0: (0, 0) -> 1.
 *   SSPRK2:  stage 1: (0, 1) -> 0
 *   SSPRK3:  stage 1: (0, 1) -> 2; stage 2: (0, 2) -> 0
 *   SSPRK43: stage 1: (0, 1) -> 2; stage 2: (0, 2) -> 1; stage 3: (-, 1) -> 0
 *   SSPRK54: stage 1: (0, 1) -> 2; stage 2: (0, 2) -> 1;
 *            stage 3: (0, 1, 2) -> 2, w -> 0; stage 4: (0, 2) -> 0
 * (a buffer read and written in one stage is only read at the cells the same
 * thread writes).  After the last stage buffer 0 holds U^{n+1}.  Instances
 * whose dt is 0 are copied through unchanged.
 */
amrvac_status amrvac_stage(amrvac_state* s, int32_t stage);

/*
 * nsteps full time steps: all stages, then t += dt and the next dt and c_h
 * from U^{n+1}, all on the device (no host sync).  The
 * first call computes dt if none is valid.  With a non-default stream the
 * step is captured once as a CUDA graph and replayed.
 */
amrvac_status amrvac_step(amrvac_state* s, int32_t nsteps);

/*
 * Synchronises and reads per-instance t, dt, c_h ([ninst] each), the
 * conservation sums h_sums[ninst][9] (integral of each conserved variable of
 * buffer 0 = U^n, reduced on the device in FP64 in a fixed order when h_sums is
 * not NULL) and the latched device error.  Any pointer may be NULL.  Returns
 * the latched error code (AMRVAC_OK if none).
 */
amrvac_status amrvac_get_diag(amrvac_state* s, double* h_t, double* h_dt, double* h_ch,
                              double* h_sums, amrvac_error_info* err);

/*
 * CFL time step of a uniform mesh for callers that cannot allocate device
 * memory (no workspace, no state).  The paper has no counterpart: this is a
 * service entry point of this library.  Callers inside a host framework that
 * owns every device allocation, or in code paths where cudaMalloc is not
 * allowed, pass only their own input and output buffers.
 *   cfg, inst: one instance covered by its level-0 blocks only (nblocks =
 *     base_blocks product, blocks in any order); cfg->precision selects the
 *     element type of d_U (double or float), cfg->courant the CFL number.
 *   d_U: device [var][block][cell] conserved state; t: current time; the step
 *     is clipped to inst->t_end - t.
 *   d_out: device double[2] receiving {dt, c_h}, computed exactly as
 *     amrvac_cfl_dt computes them.
 *   cuda_stream: cudaStream_t of the two kernels (asynchronous).
 * Scratch: a file-scope device array of AMRVAC_NOALLOC_MAX_BLOCKS x 2 doubles
 * (1 MiB) that every device loading the library holds until exit.  More blocks
 * than AMRVAC_NOALLOC_MAX_BLOCKS: AMRVAC_E_INVALID.  The first call on a device
 * looks up the array's device address with cudaGetSymbolAddress (make it
 * before any stream capture).  The looked-up address is kept per device for
 * the life of the process: after cudaDeviceReset on a device it is stale, so
 * do not call this entry point on that device again.  Calls share the array:
 * calls overlapping on the GPU race.  A block larger than
 * AMRVAC_MAX_BLOCK_CELLS: AMRVAC_E_INVALID.  No allocation of any kind is
 * made.
 */
amrvac_status amrvac_cfl_dt_noalloc(const amrvac_config* cfg, const amrvac_instance_desc* inst,
                                    int32_t nblocks, const void* d_U, double t, double* d_out,
                                    void* cuda_stream);

/*
 * Checkpoint / restart (Sect. 7.5: snapshots hold the conserved variables and
 * are used to restart).  save synchronises and writes a raw binary file:
 * header {magic "AMRVACGB", version 1, ndim, block_nx[3], nblocks, ninst,
 * precision}, the block list int32 [nblocks][5], per instance {t, t_end, dt,
 * c_h, dt_valid} and buffer 0 (U^n) in the state's precision.  load reads such
 * a file into a state created with the same config and block list
 * (AMRVAC_E_INVALID otherwise) and restores U^n and the clocks, so that the
 * continued run repeats the uninterrupted one bit for bit.
 */
amrvac_status amrvac_state_save(amrvac_state* s, const char* path);
amrvac_status amrvac_state_load(amrvac_state* s, const char* path);

/*
 * Launch shape of the fused stage kernel (its tile is the 16^d block):
 * resident CTAs per SM (0 = as many as fit), work-list order (0 = Morton curve
 * per instance, 1 = storage order), block scheduling (0 = static, 1 = dynamic
 * via a device counter), and the faces a thread packs into the two lanes of
 * its FP32x2 instructions (0 = the two sides of one face: a 96-register kernel,
 * two CTAs per SM; 1 = the x and y faces of its cell together: fewer
 * instructions, a ~160-register kernel with one CTA per SM; FP32 bulk with
 * vanleer + HLLD only, ignored otherwise).  ctas_per_sm, order and dynamic do
 * not change the arithmetic (results are bit-identical across them); faces = 1
 * evaluates the same formulas with another FP32 grouping (results agree to
 * float rounding).  Setting a tuning drops the captured step graph.  Not part
 * of the paper (a GB300 launch-shape choice).
 */
typedef struct {
  int32_t ctas_per_sm;
  int32_t order;
  int32_t dynamic;
  int32_t faces;
  double ms_per_step;      /* measured by amrvac_autotune, else 0 */
} amrvac_tuning;

amrvac_status amrvac_set_tuning(amrvac_state* s, const amrvac_tuning* t);
amrvac_status amrvac_get_tuning(amrvac_state* s, amrvac_tuning* t);

/*
 * Times every launch shape (ctas_per_sm x order x dynamic, and faces where it
 * applies: 8 or 12 shapes) over trial_steps full steps on the state itself
 * (U^n and the clocks are restored after each trial and at the end), keeps the
 * fastest and returns it in *best.  With cache_path, a tuning stored there for
 * the same (ndim, block size, precision, flux, limiter, pressure, block-count
 * bucket) is applied without timing, and a new result is appended.
 */
amrvac_status amrvac_autotune(amrvac_state* s, int32_t trial_steps, const char* cache_path,
                              amrvac_tuning* best);

/* Clears the latched device error. */
amrvac_status amrvac_clear_error(amrvac_state* s);

/* Number of kernels this library launched on the state since creation. */
int64_t amrvac_launch_count(const amrvac_state* s);

/*
 * Bootstrapping (Sect. 7.4) of state register `buffer` (0..2) with the
 * configuration's fix_small_values method (AMRVAC_E_INVALID when it is OFF):
 * all small cells are found first, then repaired in place as described at
 * amrvac_fix.  Stream-ordered; with h_count != NULL the call synchronises and
 * writes the number of cells repaired.  Stages already apply it to their
 * output when the method is not OFF; this entry point serves states set by the
 * caller.
 */
amrvac_status amrvac_fix_small_values(amrvac_state* s, int32_t buffer, int64_t* h_count);

/*
 * Dynamic regridding (Sect. 1 and 3: blocks are refined and coarsened
 * automatically on weighted, user-chosen plasma quantities).  The paper
 * prints no criterion; the library uses Loehner's normalised second
 * derivative.  For a quantity q and a cell, with q_{+-} its face neighbours
 * along d (ghost values of the level across block faces, as
 * amrvac_fill_ghosts):
 *   E(q) = sqrt( sum_d (q_{+} - 2 q_0 + q_{-})^2 /
 *                sum_d (|q_{+} - q_0| + |q_0 - q_{-}|
 *                       + 0.01 (|q_{+}| + 2 |q_0| + |q_{-}|))^2 )
 * (0 where the denominator vanishes), and the cell's estimate is
 * sum_v weights[v] E(w_v) over the primitive variables w = (rho, v_x, v_y,
 * v_z, p, B_x, B_y, B_z, psi).  A regrid takes three calls:
 *
 * amrvac_regrid_estimate: per block of register `buffer`, the maximum of the
 *   estimate over its cells into h_est[nblocks] (double, may be NULL) and the
 *   flag h_flags[nblocks] (int8, may be NULL): 1 (refine) when it exceeds
 *   refine_threshold and the block's level < max_level, -1 (coarsen) when it
 *   is below derefine_ratio * refine_threshold and the level > 0, else 0.
 *   weights: host double[9], >= 0, not all 0; NULL = the density alone.
 *   Evaluated in double from the stored values.  Synchronises.
 *   AMRVAC_E_INVALID for a bad buffer, weight, threshold or max_level (0..15).
 *
 * amrvac_regrid_plan (host only, no device work): the block list after one
 *   regrid of the mesh (cfg, inst, block_meta as amrvac_workspace_bytes) with
 *   the given flags.  Flagged blocks are split in 2^ndim children; then every
 *   leaf that would touch (across faces, edges or corners) a leaf two levels
 *   finer is split too, until the mesh is 2:1 balanced.  A family of 2^ndim
 *   sibling leaves is merged into its parent only when every sibling has flag
 *   -1, none was split, and the parent keeps the mesh 2:1 balanced; families
 *   are tried in increasing (instance, level, k, j, i) order of the parent.
 *   The result is sorted by (instance, level, k, j, i) and written to
 *   new_meta[capacity][5]; *new_nblocks gets its length.  AMRVAC_E_INVALID for
 *   an invalid mesh, flags outside {-1, 0, 1}, a split beyond level 15 or
 *   capacity too small (*new_nblocks then holds the length needed).
 *
 * amrvac_regrid_transfer: fills register dst_buffer of `dst` (a state created
 *   with the planned block list and the same config and instances as `src`)
 *   from register src_buffer of `src`: a block present in both is copied; the
 *   children of a split block get its conserved value plus minmod-limited
 *   slopes times +-1/4 (the prolongation of the ghost fill, slopes across the
 *   block's faces from its ghost values); a merged parent gets the mean of the
 *   2^ndim children cells it covers.  Every conserved variable's integral is
 *   kept.  Needs even block_nx in every dimension.  Enqueued on dst's stream
 *   after the work enqueued so far on src's stream.  AMRVAC_E_INVALID when the
 *   states do not match or dst's blocks are not one regrid away from src's.
 */
amrvac_status amrvac_regrid_estimate(amrvac_state* s, int32_t buffer, const double* weights,
                                     double refine_threshold, double derefine_ratio,
                                     int32_t max_level, double* h_est, int8_t* h_flags);
amrvac_status amrvac_regrid_plan(const amrvac_config* cfg, int32_t ninst,
                                 const amrvac_instance_desc* inst, int32_t nblocks,
                                 const int32_t* block_meta, const int8_t* flags,
                                 int32_t capacity, int32_t* new_meta, int32_t* new_nblocks);
/*
 * amrvac_regrid_plan_device: the same plan (the same block list, in the same
 *   order) computed on the device from the state's own mesh tables: the
 *   splits and their 2:1 closure over the level maps (one pass per launch,
 *   repeated while a pass adds a split, at most 17 passes), the merges of
 *   complete families (each family decided independently: a merge can only
 *   be prevented by leaves of finer levels, whose families come later in the
 *   sequential order), and the compaction of the new leaves through dense
 *   per-(instance, level) maps and a prefix sum.  Flags: h_flags (host int8
 *   [nblocks], -1/0/1) when not NULL, else those of the last
 *   amrvac_regrid_estimate.  Scratch lives in the state's workspace (no
 *   allocation).  Synchronises; new_nblocks is always set; AMRVAC_E_INVALID
 *   when capacity is too small, for a bad flag, a split beyond the deepest
 *   level, or a mesh whose dense maps one level finer would be too large.
 */
amrvac_status amrvac_regrid_plan_device(amrvac_state* s, const int8_t* h_flags,
                                        int32_t capacity, int32_t* h_new_meta,
                                        int32_t* h_new_nblocks);
amrvac_status amrvac_regrid_transfer(amrvac_state* src, int32_t src_buffer, amrvac_state* dst,
                                     int32_t dst_buffer);

const char* amrvac_error_string(amrvac_status st);

#ifdef __cplusplus
}
#endif
#endif /* AMRVAC_H */
