/*
 * teno.h -- C ABI of the GB300 TENO finite-volume library (libteno.so).
 *
 * The library computes the semi-discrete finite-volume residual of 2D
 * hyperbolic conservation laws on unstructured triangular meshes with the
 * unstructured TENO reconstruction of Ji, Liang & Fu (Sec. 2.1, Eq.
 * fv_governing_equation_semi_discrete; Sec. 3, Eqs. new_scale_separation,
 * normalize, cutoff, TENO_reconstruction111/222, TENO_weight), the rotated
 * Riemann fluxes of Sec. 4, and the SSP-RK3 update of Eq.
 * fv_time_discretization_01, on one CUDA GPU.
 *
 * Conventions
 *  - Every call returns an int status: TENO_OK (0) or a negative TENO_E*
 *    code; teno_last_error() returns a message for the last failure.
 *  - The library owns everything it allocates.  Caller pointers are borrowed
 *    for the duration of the call only.
 *  - State arrays are structure-of-arrays [n_var][n_cell] of float64 in the
 *    caller's cell order ("user order").  n_var = 1 (scalar advection) or 4
 *    (2D Euler: rho, rho*u, rho*v, E).  Internally cells are renumbered along
 *    a Hilbert curve; teno_get_permutation() exposes that order.
 *  - Arguments flagged `on_device` are device pointers on the context's GPU
 *    when on_device != 0 (stream-ordered on the context's stream, not
 *    synchronised) and host pointers otherwise (the call synchronises the
 *    stream before returning).
 *  - Call order: teno_create -> teno_mesh_load -> teno_precompute_stencils ->
 *    teno_set_state -> (teno_residual | teno_rk3_step | teno_adjoint_step)*;
 *    violating it returns TENO_ESTATE.
 *  - A context is not thread safe; use one context per host thread.
 */
#ifndef TENO_H
#define TENO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct teno_ctx teno_ctx;

enum teno_status {
  TENO_OK = 0,
  TENO_EINVAL = -1,   /* bad argument (null pointer, size, option) */
  TENO_ENOMEM = -2,   /* host or device allocation failed */
  TENO_ECUDA = -3,    /* a CUDA runtime call failed */
  TENO_EMESH = -4,    /* degenerate/clockwise cell, non-manifold edge, unmatched boundary face */
  TENO_ESTENCIL = -5, /* a stencil cannot be filled or its least-squares matrix is rank deficient */
  TENO_ENONPHYS = -6, /* density or pressure <= 0, or NaN, after a stage */
  TENO_ETIMEOUT = -7, /* a bounded device-side wait gave up */
  TENO_ESTATE = -8    /* calls made in the wrong order */
};

/* Numerical fluxes (Sec. 4): upwind (scalar advection), HLL with the Einfeldt
 * wave speeds of Eq. wavespeed (the Roe sound speed with both velocity
 * components), HLLC (cited in Sec. 5) with Toro's contact speed and star
 * states on the same bounds.  The side sound speeds take a negative pressure
 * as zero (a Gauss state at the positivity floor can round below it); where
 * HLLC's contact speed is 0/0 (zero sound speed on both sides) the flux is
 * HLL's. */
enum teno_flux { TENO_FLUX_UPWIND = 0, TENO_FLUX_HLL = 1, TENO_FLUX_HLLC = 2 };
/* TENO_FP64: FP64-accurate path -- matvecs, smoothness indicators and Gauss
 *   evaluation in double-float (pairs of FP32 numbers, ~48 significant bits)
 *   on the FP32 pipe, selection decided in FP64 near the cutoff, fluxes,
 *   residual and update in FP64;
 * TENO_FP32_MIXED: matvecs and fluxes in FP32 with FP32 accumulation, the
 *   selection decision (FP64 inside a guard band of C_T) and the residual
 *   accumulation and update in FP64;
 * TENO_FP64_NATIVE: everything in FP64 on the FP64 pipe. */
enum teno_precision { TENO_FP64 = 0, TENO_FP32_MIXED = 1, TENO_FP64_NATIVE = 2 };

/* Boundary tags of non-periodic meshes (bface[:,2]); the ghost state at each
 * boundary Gauss point of the shock case (Sec. 5, double Mach reflection):
 * WALL mirrors the normal momentum; INFLOW is the post-shock state; OUTFLOW
 * copies the inner state, and a cell with an outflow face enters every face
 * flux with its cell average (first order in that cell layer: on its one-sided
 * high-order polynomial the boundary closure has a growing mode); TOP is the
 * post- or pre-shock state on either side of the exact shock trace at the
 * call's time (teno_set_time). */
enum teno_bc { TENO_BC_WALL = 1, TENO_BC_INFLOW = 2, TENO_BC_OUTFLOW = 3, TENO_BC_TOP = 4 };

/* Scheme options.  Defaults (teno_default_params) follow the paper:
 * C_T = 1e-6 (Sec. 3.3), eps = 1e-12 (Eq. new_scale_separation),
 * CFL 0.4 (Sec. 5), gamma = 1.4. */
typedef struct teno_params {
  int32_t order;     /* design order 3..6: polynomial degree r = order-1 on the large stencil */
  int32_t n_var;     /* 1: scalar advection u_t + a.grad u = 0; 4: 2D Euler */
  int32_t flux;      /* enum teno_flux; UPWIND only with n_var = 1 */
  int32_t precision; /* enum teno_precision */
  int32_t linear;    /* 1: always take the large-stencil polynomial (the paper's "Linear" rows) */
  int32_t nq;        /* Gauss points per edge; 0 = 2 for order <= 4, 3 otherwise */
  int32_t recon_variant; /* reconstruction kernel: 0 the stencil halo of each 32-cell tile
                            staged in shared memory; 1 direct gathers of neighbour states;
                            2 (default) persistent kernel whose producer lane streams the
                            per-cell matrices through a TMA bulk-copy ring while the
                            tile's stencil halo is double-buffered with cp.async (Euler,
                            TENO_FP64 and TENO_FP32_MIXED; else 0).  0 and 2 fall back to 1
                            where a tile's halo exceeds 256 cells.  Variants 0 and 1 give
                            bitwise identical results; variant 2 on TENO_FP64 evaluates
                            the large polynomial at the Gauss points through per-cell
                            products Psi' G stored at precompute and takes the cutoff
                            decision from FP32 coefficients with a rigorous error bound
                            (falling back to pairs and FP64 where the bound does not
                            separate chi from C_T): equal up to rounding; it keeps
                            4.8 KB more per cell (TENO5) in device memory. */
  double ct;         /* cutoff C_T */
  double eps;        /* epsilon of the scale separation */
  double gamma;      /* ratio of specific heats */
  double adv_x, adv_y; /* advection velocity for n_var = 1 and adv_field = 0 */
  double cfl;        /* CFL number for teno_rk3_step with dt <= 0 */
  int32_t adv_field; /* n_var = 1: 0 the constant velocity (adv_x, adv_y); 1 the rigid
                        rotation v = adv_omega phi(r) (-(y - adv_cy), x - adv_cx) of the
                        solid-body case (Sec. 5: centre (0.5, 0.5), omega 1), with the
                        radial taper phi = 1 for r <= adv_r1, a smoothstep to 0 at adv_r2
                        (no taper when adv_r2 <= adv_r1; an azimuthal field is
                        divergence-free for any phi, and the taper makes it periodic).
                        The velocity is evaluated at every face Gauss point; on a
                        periodic mesh a face on the wrap takes its points in the frame of
                        the adjacent cell with the smaller user id.  The CFL speed of a
                        cell is |omega| times the largest r phi(r) over its vertices. */
  double adv_cx, adv_cy, adv_omega;
  double adv_r1, adv_r2;
  int32_t scheme;    /* 0 TENO (the paper's scheme); 1 CWENO, the comparison scheme of
                        Sec. 2.3 on the same stencils: P = (w_K/d_K)(P_K - sum_k d_k P_k)
                        + sum_k w_k P_k with alpha = d/(beta + eps)^4, d_K = 1 - 1/cweno_dk,
                        d_k = (1 - d_K)/K over the present directional stencils (the
                        paper uses eps = 1e-14 for CWENO).  CWENO runs on the pair,
                        native and mixed paths with recon_variant 0, 1 or 2 (variant 2
                        uses the pair TMA kernel, not the W form); the adjoint entry
                        points take TENO only. */
  double cweno_dk;   /* CWENO d'_K, default 1e4 */
  int32_t charvar;   /* Euler, TENO: 1 reconstructs characteristic variables (Sec. 2.3: they
                        suppress oscillations better than conservative ones).  For every
                        local edge of a cell the large and directional coefficients of the
                        four conservative variables are projected on the characteristic
                        fields of the edge's outward normal direction at the cell-average
                        state, each field takes its own TENO selection, and the result is
                        mapped back.  The reconstruction kernels then write their
                        coefficients (FP64, 4 (m+15) values per cell) and a second kernel
                        does the projection, selection and evaluation in FP64.  The
                        selection output reports 8; the adjoint entry points take
                        conservative variables only. */
  int32_t positivity; /* Euler, conservative variables: 1 scales each cell's reconstruction
                        towards its cell average so that density, then pressure, stay at
                        least min(1e-13, the average's value) at every face Gauss point
                        (Zhang and Shu's limiter: the largest such factor <= 1; density by
                        its closed form, pressure by 60 bisection halvings).  Not in the
                        paper, which reports its schemes robust on the Mach-10 shock case
                        (Sec. 5) without stating a positivity treatment; without it that
                        case produces non-physical Gauss states at the incident front.
                        Off by default; the adjoint entry points refuse it. */
  int32_t debug;     /* test support, 0 in production.  Bit 0: the default FP64 Euler
                        reconstruction (recon_variant 2) takes every cell's cutoff decision
                        through its pair / FP64 fallback instead of the FP32 screen.  Bit 1:
                        the consumer warps of the bulk-copy reconstruction kernels wait
                        for each copy with a bound of zero polls, so the first wait of
                        every block gives up: the kernel sets the error read by
                        teno_check_state as TENO_ETIMEOUT, skips its remaining work and
                        returns once the copies its producer issued have landed (the
                        results of that call are then undefined).  This exercises the
                        give-up path of the bounded waits without a copy that never
                        lands. */
} teno_params;

/* Fills *p with the defaults above (order 5, n_var 4, HLL, FP64, recon_variant 2,
   cfl 0.4, adv (1, 1), adv_field 0, rotation centre (0.5, 0.5), omega 1, no taper,
   scheme TENO, cweno_dk 1e4, charvar 0, positivity 0, debug 0). */
void teno_default_params(teno_params* p);

/* Create a context on CUDA device `device`, launching on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *ctx receives the
 * handle, or NULL on failure.  device = -1 creates a host-only context:
 * teno_mesh_load, teno_precompute_stencils, teno_get_permutation and
 * teno_get_stencils work without a GPU, every call that needs device work
 * returns TENO_ESTATE. */
int teno_create(teno_ctx** ctx, int device, void* cuda_stream);

/* Free every host and device allocation of the context.  NULL is a no-op. */
int teno_destroy(teno_ctx* ctx);

/* Message of the last failed call on this context ("" if none).  Owned by
 * the context; valid until the next call on it. */
const char* teno_last_error(teno_ctx* ctx);

/* Change the stream later calls launch on. */
int teno_set_stream(teno_ctx* ctx, void* cuda_stream);

/* Load a triangular mesh (Sec. 2.1: elements I_i with faces j).
 *  xy     host [n_vert][2] vertex coordinates;
 *  tri    host [n_cell][3] vertex ids, counter-clockwise (the vertex order is
 *         kept: vertex 0,1,2 map to reference points (0,0),(1,0),(0,1),
 *         Eq. reconstruction_02);
 *  bface  host [n_bface][3] (v0, v1, tag) for every boundary edge, or NULL
 *         when n_bface = 0;
 *  period host {Lx, Ly} for a doubly periodic mesh whose wrapped vertices
 *         share ids (coordinates of a cell are unwrapped to lie within half
 *         a period of its vertex 0), or NULL.
 * Builds faces, normals and areas and the Hilbert-curve cell order.
 * Errors: TENO_EINVAL (null pointers, n_cell < 1 or n_vert < 3), TENO_EMESH (a
 * vertex id out of range, non-positive area, an edge shared by more than two
 * cells, a boundary edge without a bface entry).  A mesh too small for the
 * stencils of the requested order loads, and teno_precompute_stencils then
 * returns TENO_ESTENCIL. */
int teno_mesh_load(teno_ctx* ctx, int64_t n_vert, const double* xy, int64_t n_cell,
                   const int32_t* tri, int64_t n_bface, const int32_t* bface,
                   const double* period);

/* perm host [n_cell]: perm[i] = user id of internal cell i. */
int teno_get_permutation(teno_ctx* ctx, int32_t* perm);

/* Stencils and reconstruction matrices (Sec. 3.1 candidate stencils; Eqs.
 * reconstruction_03..10: A_sl, Householder QR, pseudo-inverse), computed on
 * the host in FP64 and uploaded in the device layout.  Sizes: m = N_k - 1
 * unknowns, N_s = 2 N_k large-stencil neighbours, 3 directional stencils of
 * 12 neighbours.  Errors: TENO_EINVAL, TENO_ESTENCIL, TENO_ENOMEM. */
int teno_precompute_stencils(teno_ctx* ctx, const teno_params* p);

/* Stencil members in user ids: large host [n_cell][N_s], small host
 * [n_cell][3][12] (-1 for a directional stencil that could not be filled). */
int teno_get_stencils(teno_ctx* ctx, int32_t* large, int32_t* small);

/* Slot assignment used by teno_precompute_stencils for the large stencils of
 * every 32-cell tile (the adjoint adds each lane's stencil contributions to
 * the tile's halo slot by slot; with no cell in two lanes' same slot every
 * slot takes one round).  members host [n_lanes][n_slots]: the stencil
 * members (cell ids) of each lane, distinct within a lane.  slot_of host
 * [n_lanes][n_slots] receives the slot of each member: a proper edge
 * colouring of the bipartite (lane, member) graph with n_slots colours,
 * which exists exactly when no cell is a member of more than n_slots lanes
 * (Konig's edge-colouring theorem).  Returns 1 when coloured, 0 when some
 * cell is a member of more than n_slots lanes (slot_of untouched; the
 * precompute then keeps the stencil-search order), TENO_EINVAL for n_lanes
 * < 0, n_slots < 1, null arrays or a lane with a repeated member.  Needs no
 * context and no GPU. */
int teno_colour_slots(int32_t n_lanes, int32_t n_slots, const int32_t* members,
                      int32_t* slot_of);

/* Sizes: *n_cell, *n_var, *m (unknowns), *n_s (large-stencil size). */
int teno_get_sizes(teno_ctx* ctx, int64_t* n_cell, int32_t* n_var, int32_t* m, int32_t* n_s);

/* Copy the cell averages U ([n_var][n_cell], user order) in / out. */
int teno_set_state(teno_ctx* ctx, const double* U, int on_device);
int teno_get_state(teno_ctx* ctx, double* U, int on_device);

/* Physical time of the current state (used by time-dependent boundary
 * states). */
int teno_set_time(teno_ctx* ctx, double t);

/* R = dU/dt of the current state (Eq. fv_governing_equation_semi_discrete),
 * [n_var][n_cell] user order.  sel (nullable) receives the selection per cell
 * and variable: 8 = large stencil, otherwise bit k set when directional
 * stencil k was kept (Eq. TENO_weight). */
int teno_residual(teno_ctx* ctx, double* R, uint8_t* sel, int on_device);

/* Force the selection ([n_var][n_cell] user order, bytes as above) in every
 * later residual, step and adjoint; NULL restores the computed selection. */
int teno_set_selection_override(teno_ctx* ctx, const uint8_t* sel, int on_device);

/* dt = cfl * min_i (4|V_i| / perimeter_i) / (|v_i| + c_i) of the current
 * state (host result; synchronises).  TENO_ENONPHYS when a cell is
 * non-physical (rho <= 0, p <= 0 or NaN) or every speed is zero. */
int teno_cfl_dt(teno_ctx* ctx, double* dt);

/* One SSP-RK3 step (Eq. fv_time_discretization_01) of the current state.
 * dt > 0: fixed step; dt <= 0: the CFL step computed on the device.
 * dt_used (nullable, host) receives the step; passing it (or a failing
 * positivity check, see teno_check_state) synchronises the stream. */
int teno_rk3_step(teno_ctx* ctx, double dt, double* dt_used);

/* Input state of stage `stage` (1 or 2) of the last SSP-RK3 step
 * (Eq. fv_time_discretization_01: U^(1) = U^n + dt L(U^n) for stage 1,
 * U^(2) = 3/4 U^n + 1/4 (U^(1) + dt L(U^(1))) for stage 2), [n_var][n_cell]
 * user order.  Measurement support: it lets a caller evaluate other
 * precisions on the exact states a run passed through.  TENO_ESTATE before
 * the first step; TENO_EINVAL for another stage or a null pointer. */
int teno_get_stage_state(teno_ctx* ctx, int32_t stage, double* U, int on_device);

/* n_steps SSP-RK3 steps without host synchronisation. */
int teno_rk3_steps(teno_ctx* ctx, int32_t n_steps, double dt);

/* TENO_ENONPHYS if any stage since the last check produced rho <= 0,
 * p <= 0 or NaN (Euler), else TENO_OK; clears the flag; synchronises. */
int teno_check_state(teno_ctx* ctx);

/* Discrete adjoint (no counterpart in the paper): v = (dR/dU)^T w at the
 * current state with the stencil selection and flux branches frozen at the
 * forward pass; w, v [n_var][n_cell] user order. */
int teno_residual_vjp(teno_ctx* ctx, const double* w, double* v, int on_device);

/* Adjoint of one SSP-RK3 step from the current state U^n with step dt:
 * lam_n = (dU^{n+1}/dU^n)^T lam_np1, stages replayed on the device with the
 * forward selection frozen.  The state is not changed. */
int teno_adjoint_step(teno_ctx* ctx, double dt, const double* lam_np1, double* lam_n,
                      int on_device);

/* Adjoint tape (no counterpart in the paper).  A checkpointed adjoint replays
 * each segment of steps forward before running its adjoint steps in reverse;
 * recording the replay lets the adjoint steps skip every reconstruction.
 * teno_tape_reserve allocates n_slots slots on the device (per slot the three
 * stage input states, [n_var][n_cell] FP64, and per stage the Gauss-point
 * values and selections: at 524,288 cells TENO5 about 0.5 GB); n_slots = 0
 * frees them.  teno_rk3_step_record takes one SSP-RK3 step from the current
 * state exactly as teno_rk3_step does (dt <= 0: the CFL step, host-side) and
 * records it in `slot`.  teno_adjoint_step_tape is teno_adjoint_step for the
 * recorded step: lam_n = (dU^{n+1}/dU^n)^T lam_np1 with the recorded
 * selections and Gauss-point values (the same bits as teno_adjoint_step at
 * the recorded U^n); the state is not used or changed.  Errors: TENO_EINVAL
 * (slot outside the tape or not recorded, the adjoint's restrictions),
 * TENO_ENOMEM. */
int teno_tape_reserve(teno_ctx* ctx, int32_t n_slots);
int teno_rk3_step_record(teno_ctx* ctx, int32_t slot, double dt);
int teno_adjoint_step_tape(teno_ctx* ctx, int32_t slot, const double* lam_np1, double* lam_n,
                           int on_device);

/* Values of the last reconstruction at the edge Gauss points (inspection
 * support): out host [n_cell][3][nq][n_var] in user cell order, edge e of a
 * cell running from its vertex e to vertex e+1, points in ascending order
 * along the edge; the states the face fluxes took (after the positivity
 * scaling, and the cell average for cells with an outflow face).
 * Synchronises. */
int teno_edge_values(teno_ctx* ctx, double* out);

/* Kernel timing of this context (measurement support; no counterpart in the
 * paper).  enable != 0 clears the accumulators and records a CUDA event pair
 * on the context's stream around every later kernel launch; 0 stops
 * recording.  Launch counts are kept whether or not recording is on. */
int teno_profile(teno_ctx* ctx, int enable);

/* Accumulated device time (ms, host [8]) and launch counts (host [8]) per
 * kernel kind: 0 reconstruction + selection, 1 face flux, 2 residual gather
 * + RK update, 3 CFL reduction, 4 other, 5 face-flux adjoint, 6
 * reconstruction adjoint, 7 reverse-stencil gather of the adjoint.
 * Synchronises on the recorded events; either pointer may be NULL. */
int teno_profile_read(teno_ctx* ctx, double* ms, int64_t* launches);

/* ---- Partitioned meshes (one exchange per stage; no counterpart in the
 * paper, whose code decomposes its meshes over MPI ranks, Sec. 5's
 * efficiency note).  The mesh's cells are split into n_parts contiguous
 * ranges of the Hilbert order made of whole 32-cell tiles ("owned" cells).
 * A partition reconstructs its owned cells and the first layer of cells
 * across its boundary (the face neighbours of owned cells), so that it
 * evaluates every face flux its owned cells need by itself, and keeps the
 * states of every cell those stencils reach (its "halo").  Per RK stage one
 * halo exchange brings the stage state of the halo from the owners; the
 * adjoint's reverse exchange returns the contributions to other parts' cells.
 * Each partition's stencils, matrices and slot order are those of the whole
 * mesh, and each face is evaluated with its whole-mesh orientation, so the
 * residual and the RK3 update of every owned cell are the whole-mesh results
 * bit for bit; the VJP sums the same terms in another order (equal up to
 * rounding).
 *
 * Precompute part `part` of n_parts (stencils and matrices of its compute
 * set only).  The same parameters as teno_precompute_stencils, with
 * adv_field = 0 and charvar = 0.  n_parts = 1 is the whole mesh.  On a
 * partition: teno_set_state and teno_set_selection_override take the whole
 * mesh's array ([n_var][n_cell] user order) and keep the partition's cells;
 * teno_get_state, teno_residual, teno_get_stage_state return the owned cells
 * ([n_var][n_owned], in teno_partition_cells order); teno_cfl_dt is this
 * part's step; teno_rk3_step(s), teno_residual_vjp and teno_adjoint_step
 * return TENO_EINVAL (step with teno_group_rk3_step or teno_rk3_stage).
 * Errors: those of teno_precompute_stencils; TENO_EINVAL for a bad part or
 * more parts than tiles. */
int teno_precompute_partition(teno_ctx* ctx, const teno_params* p, int32_t n_parts,
                              int32_t part);

/* *n_owned owned cells, *n_state cells of the state arrays (owned, first
 * layer, halo, and inert padding lanes); recv_counts / send_counts host
 * [n_parts] (nullable): cells received from / sent to each part per
 * exchange (send counts are 0 until teno_partition_set_send). */
int teno_partition_sizes(teno_ctx* ctx, int64_t* n_owned, int64_t* n_state, int64_t* recv_counts,
                         int64_t* send_counts);

/* owned_user host [n_owned]: user ids of the owned cells, in the order of
 * the partition's owned arrays. */
int teno_partition_cells(teno_ctx* ctx, int32_t* owned_user);

/* user_ids host [recv_counts[peer]]: the cells this partition receives from
 * `peer` per exchange, in the order the exchange buffers hold them (ascending
 * Hilbert index).  Host-only contexts too. */
int teno_partition_recv_cells(teno_ctx* ctx, int32_t peer, int32_t* user_ids);

/* Declare the cells `peer` receives from this partition (user ids, host
 * [n], in the peer's receive order: its teno_partition_recv_cells(peer ->
 * this part)); every one must be owned here.  Host-only contexts too. */
int teno_partition_set_send(teno_ctx* ctx, int32_t peer, int64_t n, const int32_t* user_ids);

/* Exchange buffers, device [n_var][count] on the context's stream.  what =
 * 0, 1, 2: the state U^n (also the state after a step), the stage-1 output
 * U^(1), the stage-2 output U^(2): pack the owned cells `peer` receives,
 * unpack the cells received from `peer` into the halo.  what = 3, the
 * adjoint's reverse exchange: pack this part's contributions to the cells
 * `peer` owns (its receive list), unpack adds the contributions from `peer`
 * to the owned cells (its send list).  Send lists must be set. */
int teno_halo_pack(teno_ctx* ctx, int32_t peer, int32_t what, double* buf);
int teno_halo_unpack(teno_ctx* ctx, int32_t peer, int32_t what, const double* buf);

/* Stage 1, 2 or 3 of an SSP-RK3 step with step dt on the updated cells
 * (Eq. fv_time_discretization_01); the halo of the stage's input state must
 * be current (U^n, U^(1), U^(2): exchange what = 0, 1, 2 first).  Stage 3
 * advances the context's time by dt. */
int teno_rk3_stage(teno_ctx* ctx, int32_t stage, double dt);

/* Largest (|v| + c) / (4|V| / perimeter) over the updated cells (host
 * result; synchronises): the CFL step of a partitioned mesh is
 * cfl / (maximum over its parts). */
int teno_local_max_speed(teno_ctx* ctx, double* lam);

/* One SSP-RK3 step of all n parts of one mesh in this process (parts[i] is
 * part i; one device and one stream): the step's dt (<= 0: the CFL step from
 * the largest speed over all parts) and after every stage the copy-based
 * halo exchange (pack on the owner, one device-to-device copy, unpack on the
 * receiver).  The first call declares the send lists from the receive lists.
 * dt_used (nullable, host) receives the step. */
int teno_group_rk3_step(teno_ctx* const* parts, int32_t n, double dt, double* dt_used);

/* v = (dR/dU)^T w for all n parts of one mesh in this process: each part
 * takes the cotangents of its owned cells from w (host [n_var][n_cell], user
 * order), runs the VJP with the selection frozen, and the reverse exchange
 * returns the contributions to other parts' cells; v host [n_var][n_cell]
 * user order (synchronises).  FP64 paths, TENO, no positivity scaling. */
int teno_group_residual_vjp(teno_ctx* const* parts, int32_t n, const double* w, double* v);

/* Measured rate (flop/s, one FMA = 2 flops) of independent fused multiply-adds
 * on every SM of `device`: precision 0 FP32, 1 FP64 (measurement support for
 * roofline fractions; no counterpart in the paper).  Runs about 0.1 s of GPU
 * work on `cuda_stream` (a cudaStream_t, NULL = legacy default) and
 * synchronises; restores the calling thread's current device.  Errors:
 * TENO_EINVAL, TENO_ECUDA. */
int teno_fma_peak(int device, void* cuda_stream, int precision, double* flops_per_s);

/* Largest n_cell that teno_cfl_dt_noalloc accepts. */
#define TENO_NOALLOC_MAX_CELLS 8388608

/* CFL step with no device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory -- code
 * running inside another framework whose caching allocator owns the GPU,
 * drivers that work to a fixed device-memory budget, real-time loops that
 * cannot afford an allocation's implicit synchronisation.
 *
 * Computes dt = cfl / max_i ((|v_i| + c_i) / cell_len_i) (scalar advection:
 * |v| = |(adv_x, adv_y)|, c = 0) -- the value teno_cfl_dt returns when
 * cell_len_i = 4 |V_i| / perimeter_i.
 *  device, cuda_stream  GPU and stream (a cudaStream_t, NULL = legacy default);
 *  U         device [n_var][n_cell] cell averages, any cell order;
 *  cell_len  device [n_cell], same cell order as U;
 *  dt        device pointer when dt_on_device != 0 (stream-ordered, not
 *            synchronised), else host pointer (the call synchronises).
 * A state with a non-physical cell (rho <= 0, p <= 0 or NaN) or with every
 * speed zero has no CFL step: the host-result call then returns
 * TENO_ENONPHYS and leaves *dt unchanged, and the device-result call writes
 * NaN to *dt (teno_cfl_dt returns TENO_ENONPHYS for the same states).
 * The caller owns every buffer.  Partial maxima go to a fixed device array of
 * (TENO_NOALLOC_MAX_CELLS / 2048 + 1) doubles = 32,776 bytes inside the
 * library, which every GPU that loads the library holds until the process
 * exits.  The first call on a device looks up that array's device address
 * with the device current and keeps it for the process; make that first call
 * before any stream capture.  A cudaDeviceReset of that device invalidates the
 * kept address: do not call this entry point for that device afterwards.
 * Every call shares the array and it keeps the last call's contents (each
 * slot is written before it is read, nothing needs clearing): calls that
 * overlap on the GPU (several streams or host threads) race and must be
 * serialised by the caller.  The calling thread's current device is restored
 * before the call returns, and a CUDA error left pending by earlier work is
 * cleared on entry rather than reported as this call's.
 * Errors: TENO_EINVAL (n_var not 1 or 4, n_cell < 1 or above
 * TENO_NOALLOC_MAX_CELLS, a null pointer, cfl <= 0, gamma <= 1 for Euler),
 * TENO_ENONPHYS (host result only, see above), TENO_ECUDA.  Calls no
 * cudaMalloc, cudaFree or allocating library routine. */
int teno_cfl_dt_noalloc(int device, void* cuda_stream, int32_t n_var, int64_t n_cell,
                        const double* U, const double* cell_len, double gamma, double adv_x,
                        double adv_y, double cfl, double* dt, int dt_on_device);

#ifdef __cplusplus
}
#endif
#endif /* TENO_H */
