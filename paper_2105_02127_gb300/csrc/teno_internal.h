// teno_internal.h -- shared declarations of the host runtime (teno_host.cpp)
// and the CUDA kernels (teno_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/teno.h"

namespace teno {

constexpr int kTile = 32;       // cells per tile of the cell-interleaved layouts
constexpr int kSmallN = 12;     // neighbours of a directional stencil (2 N_k, r = 2)
constexpr int kSmallM = 5;      // unknowns of a quadratic polynomial
constexpr int kSmallK = 3;      // directional stencils per triangle
constexpr int kMaxM = 20;
constexpr int kMaxNs = 42;
constexpr int kMaxNq = 4;
constexpr int kMaxPts = 3 * kMaxNq;

inline int unknowns(int order) {
  int r = order - 1;
  return (r + 1) * (r + 2) / 2 - 1;
}

// Per-launch constants of the reconstruction: the evaluation matrix of the
// transformed basis at the 3*nq reference edge points (row p = edge*nq + q).
struct EvalTable {
  double psi[kMaxPts * kMaxM];
};

// The same table split into FP32 (hi, lo) pairs for the double-float path.
struct DFTable {
  float2 psi[kMaxPts * kMaxM];
};

// Per-tile stencil halo: the distinct cells of a tile's stencils (internal
// ids, at most kHaloMax per tile) and the stencil slots as halo-local indices.
constexpr int kHaloMax = 256;
// nbr_loc entries: halo position in bits 0-7, and in bits 8-12 the lane's
// rank among the tile's lanes that hold the same cell in that slot (the
// order of the adjoint's halo accumulation)
constexpr int kHaloPosMask = 0xFF;
static_assert(kHaloMax <= kHaloPosMask + 1, "halo positions must fit in 8 bits");
struct HaloArgs {
  const int32_t* off = nullptr;       // [n_tiles + 1]
  const int32_t* ids = nullptr;       // [off[n_tiles]]
  const uint16_t* nbr_loc = nullptr;  // [tile][slot][32]
};

// Everything the kernels of one residual evaluation need (device pointers).
struct DeviceMesh {
  // n_cell: cells of the state arrays (stride n_pad); n_recon: cells
  // reconstructed (the first n_recon); n_update: cells whose residual is
  // gathered and updated (the first n_update).  All three are equal on a
  // whole mesh; a partition reconstructs its owned cells and the first layer
  // across its boundary, updates its owned cells and stores its halo too.
  int64_t n_cell = 0, n_pad = 0, n_face = 0, n_recon = 0, n_update = 0;
  int n_var = 1, order = 3, m = 5, ns = 12, nq = 2, e_entries = 0;
  int flux = 0, precision = 0, linear = 0;
  int variant = 0;          // reconstruction: 0 halo-staged, 1 direct gathers, 2 TMA-staged
  HaloArgs halo;            // null when some tile's halo exceeds kHaloMax
  int* err_flag = nullptr;  // device flag: bit 0 non-physical state, bit 1 a bounded wait gave up
  double ct = 1e-6, eps = 1e-12, gamma = 1.4, adv_x = 1, adv_y = 1, cfl = 0.4;
  int scheme = 0;                    // 0 TENO, 1 CWENO
  int charvar = 0;                   // Euler TENO in characteristic variables
  int positivity = 0;                // Euler: positivity scaling of the Gauss-point values
  int debug = 0;                     // teno_params.debug bits (tests only)
  double* coef_out = nullptr;        // charvar: [n_pad][4][m+15] FP64 coefficients
  double cweno_dk = 1e4;             // CWENO d'_K
  int adv_field = 0;                 // scalar velocity: 0 constant, 1 rigid rotation
  double adv_cx = 0.5, adv_cy = 0.5, adv_omega = 1.0, adv_r1 = 0.0, adv_r2 = 0.0;
  const double* cell_speed = nullptr;  // [n_pad] CFL speed per cell (rotation field)
  // reconstruction data, tile-interleaved [tile][entry][32]
  const void* ahat = nullptr;     // double (FP64_NATIVE), float2 (FP64) or float (mixed)
  const int32_t* nbr = nullptr;   // [tile][ns+36][32] internal cell ids
  const uint8_t* smask = nullptr; // [n_pad] bit k: directional stencil k present
  // Euler on the FP64 paths, recon_variant 2 (else null): FP32 matrices for
  // the selection, per slot the rows then sum_l |G_ls| ([tile][ns*(m+1) +
  // 36*6][32]), and W = Psi' G ([tile][ns*3*nq][32]) as (hi, lo) pairs on the
  // pair path, as doubles (in the same 8 bytes) on the native path
  const float* g32 = nullptr;
  const float2* wq = nullptr;
  const float2* psi_df = nullptr;   // device copy of eval_df.psi (pair W form)
  const double* psi_d = nullptr;    // device copy of eval.psi (native W form)
  // faces
  const int32_t* f_cells = nullptr; // [n_face][2] owner, neighbour (-1 boundary)
  const int8_t* f_edges = nullptr;  // [n_face][2] local edge in owner / neighbour (bc tag if boundary)
  const double* f_geom = nullptr;   // [n_face][5] nx, ny, |A| (outward from owner), x_a, y_a
  const float2* f_geom2 = nullptr;  // [n_face][3] nx, ny, |A| as (hi, lo) float pairs
  const int32_t* c_faces = nullptr; // [n_pad][3] face*2 + (1 if the cell is the neighbour)
  const double* inv_area = nullptr; // [n_pad]
  // the outflow layer: the cells (local ids, among the reconstructed ones)
  // with a face on an outflow boundary, which enter every face flux with
  // their cell average; fo_n = 0 without outflow faces
  const int32_t* fo_list = nullptr;
  int64_t fo_n = 0;
  const double* cfl_len = nullptr;    // [n_pad] 4|V|/perimeter
  const float2* cfl_ilen2 = nullptr;  // [n_pad] 1 / cfl_len as (hi, lo) pairs
  EvalTable eval;
  DFTable eval_df;
  double gw[kMaxNq];                // Gauss weights on [0,1], sum 1
  double gt[kMaxNq];                // Gauss nodes on [0,1], ascending
};

// launchers (teno_kernels.cu); all return a cudaError_t
// Us: FP32 hi/lo split of U, required by the mixed-precision path (else unused)
cudaError_t launch_recon(const DeviceMesh& dm, const double* U, const float2* Us, void* Uq,
                         uint8_t* sel_out, const uint8_t* sel_in, cudaStream_t st);
cudaError_t launch_split(const DeviceMesh& dm, const double* U, float2* Us, cudaStream_t st);
// Euler, positivity option: scale each cell's Gauss-point values towards its
// average (Zhang and Shu) in place
cudaError_t launch_positivity(const DeviceMesh& dm, const double* U, void* Uq, cudaStream_t st);
// charvar: projection, per-field selection and Gauss-point values from the
// coefficients the reconstruction wrote to dm.coef_out
cudaError_t launch_char_finish(const DeviceMesh& dm, const double* U, void* Uq, cudaStream_t st);
// the outflow layer (dm.fo_list): every Gauss value of those cells := the
// cell average (after the reconstruction and its positivity scaling)
cudaError_t launch_layer_fill(const DeviceMesh& dm, const double* U, void* Uq, cudaStream_t st);
cudaError_t launch_face_flux(const DeviceMesh& dm, const void* Uq, void* K, double time,
                             cudaStream_t st);
// mode 0: R = residual; mode 1: U_out = cn*Un + cs*(Us + dt*R), and (split
// non-null) the FP32 hi/lo split of U_out
cudaError_t launch_gather(const DeviceMesh& dm, const void* K, const double* Un, const double* Us,
                          double* out, int mode, double cn, double cs, double dt_fixed,
                          const double* max_lam, int* flag, float2* split, cudaStream_t st);
// the same maximum from the (hi, lo) state split (Euler, FP64 and mixed paths)
cudaError_t launch_max_lambda_split(const DeviceMesh& dm, const float2* Us, double* max_lam,
                                    cudaStream_t st);
cudaError_t launch_max_lambda(const DeviceMesh& dm, const double* U, double* max_lam,
                              cudaStream_t st);
cudaError_t launch_permute(const double* src, double* dst, const int32_t* perm, int64_t n,
                           int64_t ld_src, int64_t ld_dst, int n_var, int to_user,
                           cudaStream_t st);
cudaError_t launch_permute_u8(const uint8_t* src, uint8_t* dst, const int32_t* perm, int64_t n,
                              int64_t ld_src, int64_t ld_dst, int n_var, int to_user,
                              cudaStream_t st);
cudaError_t launch_axpby(double* out, const double* a, double ca, const double* b, double cb,
                         int64_t n, cudaStream_t st);
// halo exchange of a partition: pack buf[v][i] = U[v][idx[i]] (v < n_var,
// i < n); unpack writes (add = 0) or adds (add = 1) the buffer back, and the
// FP32 hi/lo split of the written states when Us is non-null
cudaError_t launch_halo_pack(const double* U, int64_t ld, const int32_t* idx, int64_t n,
                             int n_var, double* buf, cudaStream_t st);
cudaError_t launch_halo_unpack(double* U, int64_t ld, const int32_t* idx, int64_t n, int n_var,
                               const double* buf, float2* Us, int add, cudaStream_t st);
// adjoint kernels.  Uq_bar ([cell][edge point][var], 8 bytes an entry)
// holds (hi, lo) float pairs on the TENO_FP64 path and doubles on the native
// path; the reconstruction VJPs read it in the same form.
cudaError_t launch_face_flux_vjp(const DeviceMesh& dm, const void* Uq, const double* w,
                                 double* Uq_bar, double time, cudaStream_t st);
// adjoint of launch_layer_fill: ubd [cell][edge][var] := the outflow layer's
// Gauss-slot cotangents summed per edge; those slots of Uq_bar := 0
cudaError_t launch_layer_vjp(const DeviceMesh& dm, double* Uq_bar, double* ubd, cudaStream_t st);
cudaError_t launch_recon_vjp(const DeviceMesh& dm, const uint8_t* sel, const double* Uq_bar,
                             double* d_bar, double* u_self, cudaStream_t st);
// Tiled reconstruction VJP (FP64 path, Euler, per-tile halos present):
// part[halo entry][var] = pair sums of the tile's d_bar at its halo cells,
// u_self as in launch_recon_vjp; the reverse gather over halo entries
// (launch_scatter_gather with the halo reverse map) completes the VJP.
cudaError_t launch_recon_vjp_tma(const DeviceMesh& dm, const uint8_t* sel, const double* Uq_bar,
                                 double* part, double* u_self, cudaStream_t st);
cudaError_t launch_scatter_gather(const DeviceMesh& dm, const int64_t* rev_off,
                                  const int32_t* rev_idx, const double* d_bar,
                                  const double* u_self, double* v, const double* ubd,
                                  cudaStream_t st);

}  // namespace teno
