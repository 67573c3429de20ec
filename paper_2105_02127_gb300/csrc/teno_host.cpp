// teno_host.cpp -- host runtime of libteno: context, mesh topology, Hilbert
// renumbering, stencil construction and least-squares precompute (FP64), the
// device layouts, and the C ABI declared in include/teno.h.
//
// Precompute (once per mesh and order), following the paper:
//   Sec. 2.2, Eq. reconstruction_02: affine map of every target triangle onto
//     the reference triangle, vertex k of the cell -> (0,0), (1,0), (0,1);
//   Sec. 3.1: one large stencil of N_s = 2 N_k neighbours and three
//     directional stencils of 12 neighbours (sectors through the faces);
//   Eqs. reconstruction_05..08: A_sl = int_{V'_s} psi_l with exact monomial
//     moments of triangles;
//   Eqs. reconstruction_09/10: pseudo-inverse from a Householder QR,
//     Ahat = R^-1 Q_1^T;
//   Eq. WENO_smoothness: the beta quadratic form B over the reference triangle
//     (exact moments), B = L L^T; the device matrices are L^T Ahat diag|V'_s|,
//     so a kernel obtains a' = L^T a and beta = |a'|^2, and evaluates the
//     polynomial with Psi L^{-T}.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <memory>
#include <string>
#include <vector>

#include "teno_internal.h"

using namespace teno;

namespace {
constexpr int kProfKinds = 8;  // recon, face flux, gather/update, CFL, other, adjoint kernels
enum { K_RECON = 0, K_FLUX = 1, K_GATHER = 2, K_CFL = 3, K_OTHER = 4, K_FLUX_VJP = 5,
       K_RECON_VJP = 6, K_SCATTER = 7 };
}  // namespace

// ========================================================================
// context

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct teno_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  // mesh (user order unless stated)
  bool mesh_ok = false, pre_ok = false, state_ok = false;
  int64_t nv = 0, nc = 0, npad = 0, nface = 0;
  bool periodic = false;
  double L[2] = {0, 0};
  std::vector<int32_t> tri;
  std::vector<double> P;     // [nc][3][2] unwrapped vertices
  std::vector<double> cen;   // [nc][2]
  std::vector<double> area, perim;
  std::vector<int32_t> fnbr, fedge, fbc;  // [nc][3] neighbour across edge e (user), its edge, bc tag
  std::vector<int32_t> v2c_off, v2c;      // vertex -> cells (user)
  std::vector<int32_t> perm, iperm;       // perm[internal] = user, iperm[user] = internal
  bool has_time_bc = false;
  bool has_outflow = false;  // some boundary face is an outflow face
  // scheme
  teno_params prm{};
  int m = 0, ns = 0, nq = 0, E = 0, SL = 0;
  std::vector<int32_t> st_large, st_small;  // user ids, [nc][ns], [nc][36]
  // device data
  DeviceMesh dm;
  DevBuf b_halo_off, b_halo_ids, b_halo_loc, b_g32, b_wq, b_psi, b_cspeed, b_coef;
  DevBuf b_ahat, b_nbr, b_smask, b_fcells, b_fedges, b_fgeom, b_fgeom2, b_cfaces, b_inv_area, b_cfl_len, b_cfl_ilen2,
      b_perm;
  DevBuf b_fo;  // the outflow layer: local ids of the cells with an outflow face
  DevBuf b_U, b_U1, b_U2, b_R, b_tmp, b_Uq, b_K, b_sel, b_sel_ovr, b_maxlam, b_flag;
  DevBuf b_Usplit;  // FP32 hi/lo split of the state being reconstructed (mixed precision)
  bool override_on = false;
  bool split_ok = false;  // b_Usplit holds split(b_U)
  bool stages_ok = false; // b_U1, b_U2 hold the stage states of the last RK3 step
  // adjoint
  DevBuf b_rev_off, b_rev_idx, b_dbar, b_uself, b_Uqbar, b_l1, b_l2, b_lamn, b_vtmp, b_selA;
  DevBuf b_ubd;  // [cell][edge][var] cotangents of the outflow layer's cell averages
  DevBuf b_Uq_st[2], b_sel_st[2];  // stage 1, 2 reconstructions kept by the adjoint replay
  bool adj_ok = false;
  std::vector<int64_t> rev_off_h;
  std::vector<int32_t> rev_idx_h;
  // tiled adjoint (FP64 path, Euler): reverse map over the per-tile halo
  // entries and the per-entry partial sums written by the tiled VJP kernel
  DevBuf b_hrev_off, b_hrev_idx, b_hpart;
  std::vector<int64_t> hrev_off_h;
  std::vector<int32_t> hrev_idx_h;
  bool adj_tiled = false;
  double time = 0.0;
  // state and output extents: the whole mesh (sn = nc cells, stride spad =
  // npad, io_n = nc) or one partition (teno_precompute_partition)
  int64_t sn = 0, spad = 0, io_n = 0;
  int32_t part_n = 1, part_id = 0;
  int64_t n_own = 0, n_comp = 0;
  std::vector<int64_t> part_bounds;  // [part_n + 1] internal-id start of every part
  std::vector<int32_t> loc2glob;     // local cell -> global internal id
  std::vector<std::vector<int32_t>> recv_loc, send_loc;  // per peer, local cell ids
  std::vector<DevBuf> b_recv_idx, b_send_idx, b_xbuf;     // per peer
  DevBuf b_perm_in;                  // local cell -> global user id (partitions)
  // adjoint tape (teno_tape_reserve): one buffer per slot holding a step's
  // U^n, U^(1), U^(2), then per stage its Gauss-point values and selection
  std::vector<DevBuf> tape;
  std::vector<double> tape_dt, tape_t;
  std::vector<char> tape_ok;
  size_t tape_sb = 0, tape_qb = 0, tape_selb = 0;  // aligned part sizes
  // global faces (internal ids), kept on the host for partitions
  std::vector<int32_t> h_fcells, h_cfaces;
  std::vector<int8_t> h_fedges;
  std::vector<double> h_fgeom, h_inv_area, h_cfl_len;
  std::vector<uint8_t> h_fo;
  // kernel timing (teno_profile): event pairs around launches, per kind
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_kind;  // kind of the pair (2*i, 2*i+1)
  size_t ev_used = 0;
  int64_t launches[kProfKinds] = {0, 0, 0, 0, 0, 0, 0, 0};
  double prof_ms[kProfKinds] = {0, 0, 0, 0, 0, 0, 0, 0};
};

namespace {

int fail(teno_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(teno_ctx* c, cudaError_t e, const char* where) {
  cudaGetLastError();  // reported here: not left for a later call to find
  return fail(c, TENO_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(expr, where)                               \
  do {                                                \
    cudaError_t e_ = (expr);                          \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

int dev_alloc(teno_ctx* ctx, DevBuf& b, size_t bytes) {
  if (ctx->device < 0) return TENO_OK;  // host-only context
  if (b.p && b.bytes >= bytes) return TENO_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    cudaGetLastError();
    return fail(ctx, TENO_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                      cudaGetErrorString(e));
  }
  b.bytes = bytes;
  return TENO_OK;
}

void dev_free(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

// fold finished event pairs into the per-kind totals
int prof_drain(teno_ctx* ctx) {
  if (ctx->ev_used == 0) return TENO_OK;
  CK(cudaEventSynchronize(ctx->ev_pool[2 * ctx->ev_used - 1]), "event sync");
  for (size_t i = 0; i < ctx->ev_used; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev_pool[2 * i], ctx->ev_pool[2 * i + 1]), "elapsed");
    ctx->prof_ms[ctx->ev_kind[i]] += ms;
  }
  ctx->ev_used = 0;
  return TENO_OK;
}

// open a timed launch of `kind`; returns the pair index or -1
long prof_begin(teno_ctx* ctx, int kind) {
  ctx->launches[kind]++;
  if (!ctx->prof_on) return -1;
  if (ctx->ev_used == 2048 && prof_drain(ctx)) return -1;
  if (ctx->ev_pool.size() < 2 * (ctx->ev_used + 1)) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return -1;
    ctx->ev_pool.push_back(a);
    ctx->ev_pool.push_back(b);
    ctx->ev_kind.push_back(kind);
  }
  long i = (long)ctx->ev_used++;
  ctx->ev_kind[i] = kind;
  cudaEventRecord(ctx->ev_pool[2 * i], ctx->stream);
  return i;
}

void prof_end(teno_ctx* ctx, long i) {
  if (i >= 0) cudaEventRecord(ctx->ev_pool[2 * i + 1], ctx->stream);
}

int upload(teno_ctx* ctx, DevBuf& b, const void* src, size_t bytes) {
  if (ctx->device < 0) return TENO_OK;  // host-only context
  int rc = dev_alloc(ctx, b, bytes);
  if (rc) return rc;
  if (bytes == 0 || !src) return TENO_OK;  // an empty list: storage only
  CK(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, ctx->stream), "upload");
  CK(cudaStreamSynchronize(ctx->stream), "upload sync");
  return TENO_OK;
}

// ========================================================================
// mesh topology

// standard rotate/flip Hilbert mapping on an n x n grid, n = 2^16
uint64_t hilbert_index(uint32_t x, uint32_t y) {
  const uint32_t n = 1u << 16;
  uint64_t d = 0;
  for (uint32_t s = n / 2; s > 0; s /= 2) {
    uint32_t rx = (x & s) > 0;
    uint32_t ry = (y & s) > 0;
    d += (uint64_t)s * (uint64_t)s * ((3 * rx) ^ ry);
    if (ry == 0) {
      if (rx == 1) {
        x = n - 1 - x;
        y = n - 1 - y;
      }
      uint32_t t = x;
      x = y;
      y = t;
    }
  }
  return d;
}

struct EdgeRec {
  int64_t key;
  int32_t cell, edge;
};

int build_mesh(teno_ctx* ctx, const double* xy, const int32_t* tri, int64_t nbf,
               const int32_t* bface) {
  const int64_t nc = ctx->nc, nv = ctx->nv;
  ctx->tri.assign(tri, tri + 3 * nc);
  ctx->P.resize(6 * nc);
  ctx->cen.resize(2 * nc);
  ctx->area.resize(nc);
  ctx->perim.resize(nc);
  for (int64_t c = 0; c < nc; ++c) {
    double* P = &ctx->P[6 * c];
    for (int k = 0; k < 3; ++k) {
      int32_t v = tri[3 * c + k];
      if (v < 0 || v >= nv) return fail(ctx, TENO_EMESH, "vertex id out of range");
      P[2 * k] = xy[2 * v];
      P[2 * k + 1] = xy[2 * v + 1];
    }
    if (ctx->periodic) {
      for (int k = 1; k < 3; ++k)
        for (int a = 0; a < 2; ++a)
          P[2 * k + a] -= ctx->L[a] * std::round((P[2 * k + a] - P[a]) / ctx->L[a]);
    }
    ctx->cen[2 * c] = ((P[0] + P[2]) + P[4]) / 3.0;
    ctx->cen[2 * c + 1] = ((P[1] + P[3]) + P[5]) / 3.0;
    double a2 = (P[2] - P[0]) * (P[5] - P[1]) - (P[4] - P[0]) * (P[3] - P[1]);
    if (!(a2 > 0.0))
      return fail(ctx, TENO_EMESH, "cell " + std::to_string(c) + " has non-positive area");
    ctx->area[c] = 0.5 * a2;
    double pe = 0.0;
    for (int k = 0; k < 3; ++k) {
      int k1 = (k + 1) % 3;
      pe += std::hypot(P[2 * k1] - P[2 * k], P[2 * k1 + 1] - P[2 * k + 1]);
    }
    ctx->perim[c] = pe;
  }
  // vertex -> cells
  ctx->v2c_off.assign(nv + 1, 0);
  for (int64_t i = 0; i < 3 * nc; ++i) ctx->v2c_off[tri[i] + 1]++;
  for (int64_t v = 0; v < nv; ++v) ctx->v2c_off[v + 1] += ctx->v2c_off[v];
  ctx->v2c.resize(3 * nc);
  {
    std::vector<int32_t> pos(ctx->v2c_off.begin(), ctx->v2c_off.end() - 1);
    for (int64_t c = 0; c < nc; ++c)
      for (int k = 0; k < 3; ++k) ctx->v2c[pos[tri[3 * c + k]]++] = (int32_t)c;
  }
  // edges: match the two cells of every interior edge
  std::vector<EdgeRec> ed(3 * nc);
  for (int64_t c = 0; c < nc; ++c)
    for (int e = 0; e < 3; ++e) {
      int64_t a = tri[3 * c + e], b = tri[3 * c + (e + 1) % 3];
      ed[3 * c + e] = {std::min(a, b) * nv + std::max(a, b), (int32_t)c, e};
    }
  std::sort(ed.begin(), ed.end(), [](const EdgeRec& x, const EdgeRec& y) {
    return x.key != y.key ? x.key < y.key : (x.cell != y.cell ? x.cell < y.cell : x.edge < y.edge);
  });
  std::vector<std::pair<int64_t, int32_t>> bkeys;
  for (int64_t b = 0; b < nbf; ++b) {
    int64_t a0 = bface[3 * b], a1 = bface[3 * b + 1];
    bkeys.push_back({std::min(a0, a1) * nv + std::max(a0, a1), bface[3 * b + 2]});
  }
  std::sort(bkeys.begin(), bkeys.end());
  ctx->fnbr.assign(3 * nc, -1);
  ctx->fedge.assign(3 * nc, -1);
  ctx->fbc.assign(3 * nc, 0);
  for (size_t i = 0; i < ed.size();) {
    size_t j = i;
    while (j < ed.size() && ed[j].key == ed[i].key) ++j;
    if (j - i == 2) {
      const EdgeRec &x = ed[i], &y = ed[i + 1];
      ctx->fnbr[3 * x.cell + x.edge] = y.cell;
      ctx->fedge[3 * x.cell + x.edge] = y.edge;
      ctx->fnbr[3 * y.cell + y.edge] = x.cell;
      ctx->fedge[3 * y.cell + y.edge] = x.edge;
    } else if (j - i == 1) {
      auto it = std::lower_bound(bkeys.begin(), bkeys.end(), std::make_pair(ed[i].key, INT32_MIN));
      if (it == bkeys.end() || it->first != ed[i].key)
        return fail(ctx, TENO_EMESH, "boundary edge without a bface entry");
      ctx->fbc[3 * ed[i].cell + ed[i].edge] = it->second;
      if (it->second == TENO_BC_TOP) ctx->has_time_bc = true;
      if (it->second == TENO_BC_OUTFLOW) ctx->has_outflow = true;
    } else {
      return fail(ctx, TENO_EMESH, "edge shared by more than two cells");
    }
    i = j;
  }
  // Hilbert order of centroids
  double lo[2] = {1e300, 1e300}, hi[2] = {-1e300, -1e300};
  for (int64_t c = 0; c < nc; ++c)
    for (int a = 0; a < 2; ++a) {
      lo[a] = std::min(lo[a], ctx->cen[2 * c + a]);
      hi[a] = std::max(hi[a], ctx->cen[2 * c + a]);
    }
  double span = std::max(hi[0] - lo[0], hi[1] - lo[1]);
  if (!(span > 0)) span = 1.0;
  std::vector<uint64_t> key(nc);
  for (int64_t c = 0; c < nc; ++c) {
    double fx = (ctx->cen[2 * c] - lo[0]) / span, fy = (ctx->cen[2 * c + 1] - lo[1]) / span;
    uint32_t ix = (uint32_t)std::min(65535.0, std::max(0.0, fx * 65535.0));
    uint32_t iy = (uint32_t)std::min(65535.0, std::max(0.0, fy * 65535.0));
    key[c] = hilbert_index(ix, iy);
  }
  ctx->perm.resize(nc);
  for (int64_t c = 0; c < nc; ++c) ctx->perm[c] = (int32_t)c;
  std::stable_sort(ctx->perm.begin(), ctx->perm.end(),
                   [&](int32_t a, int32_t b) { return key[a] < key[b]; });
  ctx->iperm.resize(nc);
  for (int64_t i = 0; i < nc; ++i) ctx->iperm[ctx->perm[i]] = (int32_t)i;
  return TENO_OK;
}

// ========================================================================
// reference-triangle data

struct RefData {
  int m = 0, r = 0, nq = 0;
  int ex[kMaxM][2];
  double mean0[kMaxM];
  double B[kMaxM * kMaxM];
  double Lc[kMaxM * kMaxM];    // Cholesky factor, B = Lc Lc^T (lower)
  double Linv[kMaxM * kMaxM];  // Lc^{-1}
  double gt[kMaxNq], gw[kMaxNq];
  double psi_t[kMaxPts * kMaxM];  // Psi L^{-T}
};

struct FactTable {
  double f[24];
  FactTable() {
    f[0] = 1.0;
    for (int i = 1; i < 24; ++i) f[i] = f[i - 1] * i;
  }
};
const FactTable kFact;

inline double fact(int n) { return kFact.f[n]; }

// int over the reference triangle of xi^a eta^b = a! b! / (a+b+2)!
double ref_moment(int a, int b) { return fact(a) * fact(b) / fact(a + b + 2); }

double falling(int a, int i) {
  if (i > a) return 0.0;
  double c = 1.0;
  for (int k = 0; k < i; ++k) c *= (a - k);
  return c;
}

int make_ref(int order, int nq, RefData& R) {
  R.r = order - 1;
  R.nq = nq;
  int n = 0;
  for (int d = 1; d <= R.r; ++d) {  // degree by degree: xi^d, eta^d, xi^(d-1) eta, ...
    R.ex[n][0] = d; R.ex[n][1] = 0; ++n;
    R.ex[n][0] = 0; R.ex[n][1] = d; ++n;
    for (int j = 1; j < d; ++j) { R.ex[n][0] = d - j; R.ex[n][1] = j; ++n; }
  }
  R.m = n;
  const int m = n;
  for (int l = 0; l < m; ++l) R.mean0[l] = 2.0 * ref_moment(R.ex[l][0], R.ex[l][1]);
  for (int l = 0; l < m; ++l)
    for (int k = 0; k < m; ++k) {
      double s = 0.0;
      for (int q = 1; q <= R.r; ++q)
        for (int i = 0; i <= q; ++i) {
          int j = q - i;
          double cl = falling(R.ex[l][0], i) * falling(R.ex[l][1], j);
          double ck = falling(R.ex[k][0], i) * falling(R.ex[k][1], j);
          if (cl == 0.0 || ck == 0.0) continue;
          s += cl * ck *
               ref_moment(R.ex[l][0] + R.ex[k][0] - 2 * i, R.ex[l][1] + R.ex[k][1] - 2 * j);
        }
      R.B[l * m + k] = s;
    }
  // Cholesky B = Lc Lc^T
  for (int i = 0; i < m * m; ++i) R.Lc[i] = 0.0;
  for (int j = 0; j < m; ++j) {
    double d = R.B[j * m + j];
    for (int k = 0; k < j; ++k) d -= R.Lc[j * m + k] * R.Lc[j * m + k];
    if (!(d > 0.0)) return TENO_EINVAL;
    R.Lc[j * m + j] = std::sqrt(d);
    for (int i = j + 1; i < m; ++i) {
      double s = R.B[i * m + j];
      for (int k = 0; k < j; ++k) s -= R.Lc[i * m + k] * R.Lc[j * m + k];
      R.Lc[i * m + j] = s / R.Lc[j * m + j];
    }
  }
  // Linv = Lc^{-1} (lower triangular)
  for (int i = 0; i < m * m; ++i) R.Linv[i] = 0.0;
  for (int col = 0; col < m; ++col)
    for (int i = col; i < m; ++i) {
      double s = (i == col) ? 1.0 : 0.0;
      for (int k = col; k < i; ++k) s -= R.Lc[i * m + k] * R.Linv[k * m + col];
      R.Linv[i * m + col] = s / R.Lc[i * m + i];
    }
  // Gauss-Legendre nodes (closed forms) mapped to [0,1], weights summing to 1
  double x[4], w[4];
  if (nq == 1) {
    x[0] = 0.0; w[0] = 2.0;
  } else if (nq == 2) {
    x[0] = -1.0 / std::sqrt(3.0); x[1] = -x[0]; w[0] = w[1] = 1.0;
  } else if (nq == 3) {
    x[0] = -std::sqrt(0.6); x[1] = 0.0; x[2] = std::sqrt(0.6);
    w[0] = w[2] = 5.0 / 9.0; w[1] = 8.0 / 9.0;
  } else if (nq == 4) {
    double a = std::sqrt(3.0 / 7.0 - 2.0 / 7.0 * std::sqrt(1.2));
    double b = std::sqrt(3.0 / 7.0 + 2.0 / 7.0 * std::sqrt(1.2));
    x[0] = -b; x[1] = -a; x[2] = a; x[3] = b;
    w[1] = w[2] = (18.0 + std::sqrt(30.0)) / 36.0;
    w[0] = w[3] = (18.0 - std::sqrt(30.0)) / 36.0;
  } else {
    return TENO_EINVAL;
  }
  for (int k = 0; k < nq; ++k) {
    R.gt[k] = 0.5 * (x[k] + 1.0);
    R.gw[k] = 0.5 * w[k];
  }
  // Psi' = Psi L^{-T} at the 3*nq reference edge points, row p = edge*nq + q:
  // edge 0: (t, 0); edge 1: (1-t, t); edge 2: (0, 1-t)
  for (int i = 0; i < kMaxPts * kMaxM; ++i) R.psi_t[i] = 0.0;
  for (int e = 0; e < 3; ++e)
    for (int q = 0; q < nq; ++q) {
      double t = R.gt[q];
      double xi = e == 0 ? t : (e == 1 ? 1.0 - t : 0.0);
      double eta = e == 0 ? 0.0 : (e == 1 ? t : 1.0 - t);
      double psi[kMaxM];
      for (int l = 0; l < m; ++l)
        psi[l] = std::pow(xi, R.ex[l][0]) * std::pow(eta, R.ex[l][1]) - R.mean0[l];
      for (int l = 0; l < m; ++l) {
        double s = 0.0;
        for (int j = 0; j <= l; ++j) s += psi[j] * R.Linv[l * m + j];
        R.psi_t[(e * nq + q) * kMaxM + l] = s;
      }
    }
  return TENO_OK;
}

// ========================================================================
// stencils (user ids)

struct Searcher {
  const teno_ctx* ctx;
  std::vector<int32_t> mark;
  int32_t stamp = 0;
  std::vector<int32_t> cells;   // cells[0] = target, then layer by layer
  std::vector<int> layer_begin; // layer k = [layer_begin[k], layer_begin[k+1])
  bool done = false;

  explicit Searcher(const teno_ctx* c) : ctx(c), mark(c->nc, 0) {}

  void reset(int32_t t) {
    ++stamp;
    cells.clear();
    layer_begin.clear();
    cells.push_back(t);
    mark[t] = stamp;
    layer_begin.push_back(0);
    layer_begin.push_back(1);
    done = false;
  }
  int layers() const { return (int)layer_begin.size() - 2; }
  bool grow() {  // adds one vertex-neighbour layer (at most 16)
    if (done || layers() >= 16) return false;
    int b = layer_begin[layers()], e = layer_begin[layers() + 1];
    for (int i = b; i < e; ++i) {
      int32_t c = cells[i];
      for (int k = 0; k < 3; ++k) {
        int32_t v = ctx->tri[3 * c + k];
        for (int32_t p = ctx->v2c_off[v]; p < ctx->v2c_off[v + 1]; ++p) {
          int32_t x = ctx->v2c[p];
          if (mark[x] != stamp && cells.size() < 4096) {
            mark[x] = stamp;
            cells.push_back(x);
          }
        }
      }
    }
    if ((int)cells.size() == e) {
      done = true;
      return false;
    }
    layer_begin.push_back((int)cells.size());
    return true;
  }
  // centroid offset c_s - c_t, reduced to the nearest periodic image
  void offset(int32_t t, int32_t s, double* d) const {
    d[0] = ctx->cen[2 * s] - ctx->cen[2 * t];
    d[1] = ctx->cen[2 * s + 1] - ctx->cen[2 * t + 1];
    if (ctx->periodic)
      for (int a = 0; a < 2; ++a) d[a] -= ctx->L[a] * std::round(d[a] / ctx->L[a]);
  }
  double dist2(int32_t t, int32_t s) const {
    double d[2];
    offset(t, s, d);
    double x2 = d[0] * d[0];
    double y2 = d[1] * d[1];
    return x2 + y2;
  }
};

// returns TENO_OK; small[j*12..] = -1 when sector j cannot be filled
int find_stencils(Searcher& S, int32_t t, int ns, int32_t* large, int32_t* small) {
  S.reset(t);
  auto nearer = [&](int32_t a, int32_t b) {
    double da = S.dist2(t, a), db = S.dist2(t, b);
    return da != db ? da < db : a < b;
  };
  // large stencil: whole layers while the count stays <= N_s, then nearest
  int cnt = 0;
  bool ok = false;
  for (int k = 1; !ok; ++k) {
    if (k > S.layers() && !S.grow()) break;
    int b = S.layer_begin[k], e = S.layer_begin[k + 1];
    if (cnt + (e - b) <= ns) {
      for (int i = b; i < e; ++i) large[cnt++] = S.cells[i];
      ok = cnt == ns;
    } else {
      std::vector<int32_t> lay(S.cells.begin() + b, S.cells.begin() + e);
      std::sort(lay.begin(), lay.end(), nearer);
      for (int i = 0; cnt < ns; ++i) large[cnt++] = lay[i];
      ok = true;
    }
  }
  if (!ok) return TENO_ESTENCIL;
  // directional stencils: centroids in the sector from the target centroid
  // through edge j, layers added until 12 are admitted, nearest 12 kept
  const double* P = &S.ctx->P[6 * t];
  const double cx = S.ctx->cen[2 * t], cy = S.ctx->cen[2 * t + 1];
  for (int j = 0; j < kSmallK; ++j) {
    const int j1 = (j + 1) % 3;
    const double ea[2] = {P[2 * j] - cx, P[2 * j + 1] - cy};
    const double eb[2] = {P[2 * j1] - cx, P[2 * j1 + 1] - cy};
    const double D = ea[0] * eb[1] - ea[1] * eb[0];
    std::vector<int32_t> adm;
    bool filled = false;
    for (int k = 1; !filled; ++k) {
      if (k > S.layers() && !S.grow()) break;
      for (int i = S.layer_begin[k]; i < S.layer_begin[k + 1]; ++i) {
        double d[2];
        S.offset(t, S.cells[i], d);
        double al = (d[0] * eb[1] - d[1] * eb[0]) / D;
        double be = (ea[0] * d[1] - ea[1] * d[0]) / D;
        if (al >= -1e-10 && be >= -1e-10) adm.push_back(S.cells[i]);
      }
      filled = adm.size() >= (size_t)kSmallN;
    }
    if (!filled) {
      for (int i = 0; i < kSmallN; ++i) small[j * kSmallN + i] = -1;
      continue;
    }
    std::sort(adm.begin(), adm.end(), nearer);
    for (int i = 0; i < kSmallN; ++i) small[j * kSmallN + i] = adm[i];
  }
  return TENO_OK;
}

// ========================================================================
// per-cell least squares

// exact integral of xi^a eta^b over a triangle with vertices q (reference
// coordinates): expand the monomial in barycentric coordinates and use
// int lambda0^e0 lambda1^e1 lambda2^e2 = 2|T| e0! e1! e2! / (e0+e1+e2+2)!
double tri_moment(const double q[3][2], int a, int b, double two_area) {
  double px[3][8], py[3][8];
  for (int k = 0; k < 3; ++k) {
    px[k][0] = py[k][0] = 1.0;
    for (int i = 1; i < 8; ++i) {
      px[k][i] = px[k][i - 1] * q[k][0];
      py[k][i] = py[k][i - 1] * q[k][1];
    }
  }
  double s = 0.0;
  for (int i0 = 0; i0 <= a; ++i0)
    for (int i1 = 0; i1 <= a - i0; ++i1) {
      int i2 = a - i0 - i1;
      for (int j0 = 0; j0 <= b; ++j0)
        for (int j1 = 0; j1 <= b - j0; ++j1) {
          int j2 = b - j0 - j1;
          double c = fact(i0 + j0) / (fact(i0) * fact(j0)) * fact(i1 + j1) / (fact(i1) * fact(j1)) *
                     fact(i2 + j2) / (fact(i2) * fact(j2));
          s += c * px[0][i0] * py[0][j0] * px[1][i1] * py[1][j1] * px[2][i2] * py[2][j2];
        }
    }
  return two_area * fact(a) * fact(b) / fact(a + b + 2) * s;
}

// device matrix G = Lc_m^T Ahat diag(vol) (m x n) of one stencil
int stencil_matrix(const teno_ctx* ctx, const RefData& R, int32_t t, const int32_t* ids, int n,
                   int m, double* G) {
  const double* P = &ctx->P[6 * t];
  const double a = P[2] - P[0], b = P[4] - P[0], c = P[3] - P[1], d = P[5] - P[1];
  const double det = a * d - b * c;
  const double Ji[4] = {d / det, -b / det, -c / det, a / det};
  double A[kMaxNs * kMaxM], vol[kMaxNs];
  for (int s = 0; s < n; ++s) {
    const int32_t sc = ids[s];
    // image shift that brings cell s next to the target
    double off[2];
    off[0] = ctx->cen[2 * sc] - ctx->cen[2 * t];
    off[1] = ctx->cen[2 * sc + 1] - ctx->cen[2 * t + 1];
    double sh[2] = {0.0, 0.0};
    if (ctx->periodic)
      for (int k = 0; k < 2; ++k) sh[k] = -ctx->L[k] * std::round(off[k] / ctx->L[k]);
    double q[3][2];
    for (int k = 0; k < 3; ++k) {
      double x = ctx->P[6 * sc + 2 * k] + sh[0] - P[0];
      double y = ctx->P[6 * sc + 2 * k + 1] + sh[1] - P[1];
      q[k][0] = Ji[0] * x + Ji[1] * y;
      q[k][1] = Ji[2] * x + Ji[3] * y;
    }
    double two_area = std::fabs((q[1][0] - q[0][0]) * (q[2][1] - q[0][1]) -
                                (q[2][0] - q[0][0]) * (q[1][1] - q[0][1]));
    vol[s] = 0.5 * two_area;
    for (int l = 0; l < m; ++l)
      A[s * m + l] = tri_moment(q, R.ex[l][0], R.ex[l][1], two_area) - vol[s] * R.mean0[l];
  }
  // Householder QR: Qt accumulates H_m ... H_1, W becomes R
  double W[kMaxNs * kMaxM], Qt[kMaxNs * kMaxNs];
  std::copy(A, A + n * m, W);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Qt[i * n + j] = i == j ? 1.0 : 0.0;
  double rmax = 0.0, rmin = 1e300;
  for (int k = 0; k < m; ++k) {
    double sig = 0.0;
    for (int i = k; i < n; ++i) sig += W[i * m + k] * W[i * m + k];
    sig = std::sqrt(sig);
    if (sig == 0.0) return TENO_ESTENCIL;
    double v[kMaxNs];
    const double alpha = W[k * m + k] > 0 ? -sig : sig;
    for (int i = k; i < n; ++i) v[i] = W[i * m + k];
    v[k] -= alpha;
    double vv = 0.0;
    for (int i = k; i < n; ++i) vv += v[i] * v[i];
    if (vv > 0.0) {
      for (int j = k; j < m; ++j) {
        double s = 0.0;
        for (int i = k; i < n; ++i) s += v[i] * W[i * m + j];
        s *= 2.0 / vv;
        for (int i = k; i < n; ++i) W[i * m + j] -= s * v[i];
      }
      for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = k; i < n; ++i) s += v[i] * Qt[i * n + j];
        s *= 2.0 / vv;
        for (int i = k; i < n; ++i) Qt[i * n + j] -= s * v[i];
      }
    }
    rmax = std::max(rmax, std::fabs(W[k * m + k]));
    rmin = std::min(rmin, std::fabs(W[k * m + k]));
  }
  if (!(rmin > 1e-12 * rmax)) return TENO_ESTENCIL;
  // Ahat = R^-1 Q_1^T
  double Ah[kMaxM * kMaxNs];
  for (int s = 0; s < n; ++s)
    for (int i = m - 1; i >= 0; --i) {
      double x = Qt[i * n + s];
      for (int k = i + 1; k < m; ++k) x -= W[i * m + k] * Ah[k * n + s];
      Ah[i * n + s] = x / W[i * m + i];
    }
  // G = Lc^T Ahat diag(vol); Lc^T is upper triangular: G_l = sum_{j>=l} Lc[j][l] Ahat_j
  const int mr = R.m;
  for (int l = 0; l < m; ++l)
    for (int s = 0; s < n; ++s) {
      double x = 0.0;
      for (int j = l; j < m; ++j) x += R.Lc[j * mr + l] * Ah[j * n + s];
      G[l * n + s] = x * vol[s];
    }
  return TENO_OK;
}

// Assigns the ns members of each of nval lanes to the ns slots so that no
// cell is the member of two lanes in the same slot: a proper edge colouring
// of the bipartite (lane, member cell) graph with ns colours, built edge by
// edge; where the two free colours at an edge's ends differ, they are
// swapped along the alternating path from the cell end (it cannot reach the
// lane end in a bipartite graph).  Such a colouring exists exactly when no
// cell is a member of more than ns lanes (Konig's edge-colouring theorem).
// members [nval][ns] (distinct within a lane); slot_of [nval][ns] receives
// the slot of each member.  Returns 1 when coloured, 0 when some cell is a
// member of more than ns lanes (slot_of then untouched), -1 on bad input.
int colour_slots(int nval, int ns, const int32_t* members, int32_t* slot_of) {
  if (nval < 0 || ns < 1 || (nval > 0 && (!members || !slot_of))) return -1;
  std::vector<int32_t> cells(members, members + (size_t)nval * ns);
  std::sort(cells.begin(), cells.end());
  cells.erase(std::unique(cells.begin(), cells.end()), cells.end());
  const int nr = (int)cells.size();
  std::vector<int32_t> eR((size_t)nval * ns), deg(nr, 0);
  int dmax = 0;
  for (int ln = 0; ln < nval; ++ln)
    for (int s = 0; s < ns; ++s) {
      const int r = (int)(std::lower_bound(cells.begin(), cells.end(),
                                           members[(size_t)ln * ns + s]) -
                          cells.begin());
      eR[(size_t)ln * ns + s] = r;
      dmax = std::max(dmax, ++deg[r]);
    }
  for (int ln = 0; ln < nval; ++ln)  // members of a lane must be distinct
    for (int s = 0; s < ns; ++s)
      for (int s2 = 0; s2 < s; ++s2)
        if (eR[(size_t)ln * ns + s] == eR[(size_t)ln * ns + s2]) return -1;
  if (dmax > ns) return 0;
  std::vector<int32_t> colL((size_t)nval * ns, -1);  // [lane][colour] -> member index
  std::vector<int32_t> colR((size_t)nr * ns, -1);    // [member][colour] -> lane
  std::vector<int32_t> pl, pr, pc;
  for (int ln = 0; ln < nval; ++ln)
    for (int s = 0; s < ns; ++s) {
      const int w = eR[(size_t)ln * ns + s];
      int a = 0, b = 0;
      while (colL[(size_t)ln * ns + a] >= 0) ++a;
      while (colR[(size_t)w * ns + b] >= 0) ++b;
      int c = a;
      if (colR[(size_t)w * ns + a] >= 0) {
        if (colL[(size_t)ln * ns + b] < 0) {
          c = b;
        } else {
          pl.clear(), pr.clear(), pc.clear();
          int r = w, col = a;
          while (true) {
            const int l = colR[(size_t)r * ns + col];
            if (l < 0) break;
            pl.push_back(l), pr.push_back(r), pc.push_back(col);
            const int col2 = col == a ? b : a;
            const int r2 = colL[(size_t)l * ns + col2];
            if (r2 < 0) break;
            pl.push_back(l), pr.push_back(r2), pc.push_back(col2);
            r = r2;
          }
          for (size_t i = 0; i < pl.size(); ++i) {
            colL[(size_t)pl[i] * ns + pc[i]] = -1;
            colR[(size_t)pr[i] * ns + pc[i]] = -1;
          }
          for (size_t i = 0; i < pl.size(); ++i) {
            const int o = pc[i] == a ? b : a;
            colL[(size_t)pl[i] * ns + o] = pr[i];
            colR[(size_t)pr[i] * ns + o] = pl[i];
          }
        }
      }
      colL[(size_t)ln * ns + c] = w;
      colR[(size_t)w * ns + c] = ln;
    }
  // the colouring is proper: every lane has one member per colour and the
  // two tables agree
  for (int ln = 0; ln < nval; ++ln)
    for (int c = 0; c < ns; ++c) {
      const int w = colL[(size_t)ln * ns + c];
      if (w < 0 || colR[(size_t)w * ns + c] != ln) return -1;
    }
  for (int ln = 0; ln < nval; ++ln)
    for (int s = 0; s < ns; ++s) {
      const int w = eR[(size_t)ln * ns + s];
      int c = 0;
      while (colL[(size_t)ln * ns + c] != w) ++c;
      slot_of[(size_t)ln * ns + s] = c;
    }
  return 1;
}

// The cells of a partition (teno_precompute_partition): owned internal ids
// [c0, c1), a range of whole 32-cell tiles of the Hilbert order; the compute
// set (owned, then the first layer across the boundary: face neighbours of
// owned cells, ascending); the halo (every other stencil member of the
// compute set, ascending).  Local cell ids: compute set first, then halo.
struct PartCells {
  int64_t c0 = 0, c1 = 0;
  std::vector<int32_t> layer1;  // global internal ids
};

int part_cells(const teno_ctx* ctx, int32_t n_parts, int32_t part, PartCells& pc,
               std::vector<int64_t>& bounds) {
  const int64_t nc = ctx->nc, ntile = (nc + kTile - 1) / kTile;
  bounds.assign(n_parts + 1, 0);
  for (int32_t q = 0; q <= n_parts; ++q)
    bounds[q] = std::min<int64_t>(nc, kTile * (ntile * q / n_parts));
  pc.c0 = bounds[part];
  pc.c1 = bounds[part + 1];
  if (pc.c1 <= pc.c0) return TENO_EINVAL;
  std::vector<int32_t> l1;
  for (int64_t c = pc.c0; c < pc.c1; ++c) {
    const int32_t u = ctx->perm[c];
    for (int e = 0; e < 3; ++e) {
      const int32_t nu = ctx->fnbr[3 * u + e];
      if (nu < 0) continue;
      const int32_t n = ctx->iperm[nu];
      if (n < pc.c0 || n >= pc.c1) l1.push_back(n);
    }
  }
  std::sort(l1.begin(), l1.end());
  l1.erase(std::unique(l1.begin(), l1.end()), l1.end());
  pc.layer1.swap(l1);
  return TENO_OK;
}

int run_precompute(teno_ctx* ctx, int32_t n_parts = 1, int32_t part = 0) {
  const teno_params& p = ctx->prm;
  RefData R;
  if (make_ref(p.order, ctx->nq, R)) return fail(ctx, TENO_EINVAL, "reference data");
  const int m = R.m, ns = ctx->ns, SL = ctx->SL, E = ctx->E;
  const int64_t nc = ctx->nc, ntile_g = ctx->npad / kTile;
  // the global tiles whose cells are built: all of them, or those holding a
  // partition's compute set (every lane of such a tile, for its slot colouring)
  PartCells pc;
  std::vector<int64_t> tiles_g;
  if (n_parts > 1) {
    int rc0 = part_cells(ctx, n_parts, part, pc, ctx->part_bounds);
    if (rc0) return fail(ctx, rc0, "partition: empty part (more parts than tiles)");
    for (int64_t t = pc.c0 / kTile; t * kTile < pc.c1; ++t) tiles_g.push_back(t);
    for (int32_t c : pc.layer1) tiles_g.push_back(c / kTile);
    std::sort(tiles_g.begin(), tiles_g.end());
    tiles_g.erase(std::unique(tiles_g.begin(), tiles_g.end()), tiles_g.end());
  } else {
    tiles_g.resize(ntile_g);
    for (int64_t t = 0; t < ntile_g; ++t) tiles_g[t] = t;
  }
  int64_t ntile = (int64_t)tiles_g.size();
  ctx->st_large.assign(nc * ns, -1);
  ctx->st_small.assign(nc * kSmallK * kSmallN, -1);
  // matrix storage: double (native FP64), (hi, lo) float pairs (FP64 via
  // double-float) or float (mixed)
  const int store = p.precision;
  const size_t esz = store == TENO_FP32_MIXED ? sizeof(float) : 8;
  std::vector<unsigned char> ahat((size_t)ntile * E * kTile * esz, 0);
  // Euler on the FP64 paths with the bulk-copy kernel (the W form): FP32
  // selection matrices with column sums of |G| (large slots M + 1 floats,
  // directional slots 5 + 1) and W = Psi' G, the large polynomial's
  // Gauss-point values per unit difference, as (hi, lo) pairs on the pair
  // path and as doubles (the same 8 bytes) on the native path
  const bool wform = (store == TENO_FP64 || store == TENO_FP64_NATIVE) && p.n_var == 4 &&
                     p.recon_variant == 2 && p.scheme == 0 && p.charvar == 0;
  const int nq3 = 3 * ctx->nq;
  const int E32 = ns * (m + 1) + kSmallK * kSmallN * (kSmallM + 1), EW = ns * nq3;
  std::vector<float> g32(wform ? (size_t)ntile * E32 * kTile : 0, 0.f);
  std::vector<float2> wq(wform ? (size_t)ntile * EW * kTile : 0, make_float2(0.f, 0.f));
  std::vector<int32_t> nbr((size_t)ntile * SL * kTile, 0);
  std::vector<uint8_t> smask((size_t)ntile * kTile, 0);
  int rc = TENO_OK;
  int64_t bad = -1;
#pragma omp parallel
  {
    Searcher S(ctx);
    std::vector<double> G(kMaxM * kMaxNs);
#pragma omp for schedule(dynamic, 8)
    for (int64_t k = 0; k < ntile; ++k) {
      for (int64_t lane = 0; lane < kTile; ++lane) {
        const int64_t c = tiles_g[k] * kTile + lane;  // internal index
        if (c >= nc || rc != TENO_OK) continue;
        const int32_t t = ctx->perm[c];  // user id
        const int64_t tile = k;
        int32_t* lg = &ctx->st_large[(size_t)t * ns];
        int32_t* sm = &ctx->st_small[(size_t)t * kSmallK * kSmallN];
        int r = find_stencils(S, t, ns, lg, sm);
        auto put = [&](int e, double x) {
          size_t pos = ((size_t)tile * E + e) * kTile + lane;
          if (store == TENO_FP64_NATIVE) {
            reinterpret_cast<double*>(ahat.data())[pos] = x;
          } else if (store == TENO_FP64) {
            const float hi = (float)x;
            reinterpret_cast<float*>(ahat.data())[2 * pos] = hi;
            reinterpret_cast<float*>(ahat.data())[2 * pos + 1] = (float)(x - (double)hi);
          } else {
            reinterpret_cast<float*>(ahat.data())[pos] = (float)x;
          }
        };
        // FP32 rows plus an upper bound of their absolute column sum
        auto put32 = [&](int e0, const double* col, int stride, int rows) {
          double cs = 0.0;
          for (int l = 0; l < rows; ++l) {
            const float x = (float)col[l * stride];
            g32[((size_t)tile * E32 + e0 + l) * kTile + lane] = x;
            cs += std::fabs((double)x);
          }
          g32[((size_t)tile * E32 + e0 + rows) * kTile + lane] = (float)(cs * (1.0 + 1e-6));
        };
        if (!r) r = stencil_matrix(ctx, R, t, lg, ns, m, G.data());
        if (!r) {
          for (int s = 0; s < ns; ++s) {
            nbr[((size_t)tile * SL + s) * kTile + lane] = ctx->iperm[lg[s]];
            for (int l = 0; l < m; ++l) put(s * m + l, G[l * ns + s]);
            if (wform) {
              put32(s * (m + 1), &G[s], ns, m);
              for (int q = 0; q < nq3; ++q) {
                double w = 0.0;
                for (int l = 0; l < m; ++l) w += R.psi_t[q * kMaxM + l] * G[l * ns + s];
                float2& dst = wq[((size_t)tile * EW + s * nq3 + q) * kTile + lane];
                if (store == TENO_FP64_NATIVE) {
                  static_assert(sizeof(float2) == sizeof(double), "8-byte W entries");
                  memcpy(&dst, &w, sizeof(double));
                } else {
                  const float hi = (float)w;
                  dst = make_float2(hi, (float)(w - (double)hi));
                }
              }
            }
          }
          uint8_t mask = 0;
          for (int j = 0; j < kSmallK && !r; ++j) {
            const int32_t* ids = sm + j * kSmallN;
            const int slot0 = ns + j * kSmallN;
            if (ids[0] < 0) {
              for (int s = 0; s < kSmallN; ++s) {
                nbr[((size_t)tile * SL + slot0 + s) * kTile + lane] = (int32_t)c;
                for (int l = 0; l < kSmallM; ++l)
                  put(m * ns + (j * kSmallN + s) * kSmallM + l, 0.0);
              }
              continue;
            }
            r = stencil_matrix(ctx, R, t, ids, kSmallN, kSmallM, G.data());
            if (r) break;
            mask |= (uint8_t)(1u << j);
            for (int s = 0; s < kSmallN; ++s) {
              nbr[((size_t)tile * SL + slot0 + s) * kTile + lane] = ctx->iperm[ids[s]];
              for (int l = 0; l < kSmallM; ++l)
                put(m * ns + (j * kSmallN + s) * kSmallM + l, G[l * kSmallN + s]);
              if (wform)
                put32(ns * (m + 1) + (j * kSmallN + s) * (kSmallM + 1), &G[s], kSmallN, kSmallM);
            }
          }
          smask[(size_t)tile * kTile + lane] = mask;
        }
        if (r) {
#pragma omp critical
          {
            rc = r;
            bad = t;
          }
        }
      }
    }
  }
  if (rc)
    return fail(ctx, rc, "stencil or least-squares failure at user cell " + std::to_string(bad));
  // pad lanes of the last tile point at cell 0
  for (int64_t k = 0; k < ntile; ++k)
    for (int64_t lane = 0; lane < kTile; ++lane)
      if (tiles_g[k] * kTile + lane >= nc)
        for (int s = 0; s < SL; ++s) nbr[((size_t)k * SL + s) * kTile + lane] = 0;
  // Slot order of the large stencils (for the adjoint's halo accumulation):
  // within each tile the members of the cells' large stencils are assigned
  // to the ns slots by a proper edge colouring of the bipartite graph (lane,
  // member cell) with ns colours, so that no two lanes of a tile hold the
  // same cell in the same slot.  Such a colouring exists when no cell lies in
  // more than ns of the tile's large stencils (Konig's edge-colouring
  // theorem); it is built edge by edge, swapping the two colours along an
  // alternating path where needed.  Tiles with a busier cell keep the
  // stencil-search order.  Matrix columns move with their slots: the
  // reconstruction is the same sum in another order.  A partition colours
  // the global tiles its cells belong to, so every cell keeps its slot order.
  {
    const size_t E32s = wform ? (size_t)E32 : 0, EWs = wform ? (size_t)EW : 0;
#pragma omp parallel
    {
      std::vector<int32_t> members, slot_of, perm;
      std::vector<unsigned char> tmp;
#pragma omp for schedule(dynamic, 64)
      for (int64_t t = 0; t < ntile; ++t) {
        const int nval = (int)std::min<int64_t>(kTile, nc - tiles_g[t] * kTile);
        members.resize((size_t)nval * ns);
        slot_of.resize((size_t)nval * ns);
        for (int ln = 0; ln < nval; ++ln)
          for (int s = 0; s < ns; ++s)
            members[(size_t)ln * ns + s] = nbr[((size_t)t * SL + s) * kTile + ln];
        if (colour_slots(nval, ns, members.data(), slot_of.data()) != 1) continue;
        // move every lane's slot s to its colour
        perm.assign(ns, 0);
        for (int ln = 0; ln < nval; ++ln) {
          for (int s = 0; s < ns; ++s) perm[s] = slot_of[(size_t)ln * ns + s];
          // entries s * per_slot + l of lane ln in a [tile][entry][lane] array
          auto permute = [&](auto* base, size_t stride_e, size_t per_slot) {
            using T = std::remove_pointer_t<decltype(base)>;
            T* tb = reinterpret_cast<T*>(tmp.data());
            T* row = base + (size_t)t * stride_e * kTile + ln;
            for (int s = 0; s < ns; ++s)
              for (size_t l = 0; l < per_slot; ++l)
                tb[(size_t)perm[s] * per_slot + l] = row[((size_t)s * per_slot + l) * kTile];
            for (size_t e = 0; e < (size_t)ns * per_slot; ++e) row[e * kTile] = tb[e];
          };
          tmp.resize((size_t)ns * (size_t)std::max({m * 8, (m + 1) * 4, nq3 * 8, 4}));
          permute(nbr.data(), SL, 1);
          if (store == TENO_FP64_NATIVE)
            permute(reinterpret_cast<double*>(ahat.data()), E, m);
          else if (store == TENO_FP64)
            permute(reinterpret_cast<float2*>(ahat.data()), E, m);
          else
            permute(reinterpret_cast<float*>(ahat.data()), E, m);
          if (wform) {
            permute(g32.data(), E32s, m + 1);
            permute(wq.data(), EWs, nq3);
          }
        }
      }
    }
  }
  // cells reconstructed (n_valid, the first ones of the layout) and cells of
  // the state arrays (n_state; stencil ids index them)
  int64_t n_valid = nc, n_state = nc;
  if (n_parts > 1) {
    // ---- extract the partition's compute set into the local layout: owned
    // cells keep their lanes (whole tiles), the boundary layer follows in
    // ascending order, at most `fill` per tile so that each local tile's
    // stencil halo stays within kHaloMax cells (the other lanes are inert:
    // zero matrices, stencils at local cell 0, never read by a face)
    const int64_t n_own = pc.c1 - pc.c0;
    std::vector<int64_t> slot_of_tile(ntile_g, -1);
    for (int64_t k = 0; k < ntile; ++k) slot_of_tile[tiles_g[k]] = k;
    // halo-only cells: stencil members of the compute set outside it
    std::vector<int32_t> comp;
    comp.reserve(n_own + pc.layer1.size());
    for (int64_t c = pc.c0; c < pc.c1; ++c) comp.push_back((int32_t)c);
    comp.insert(comp.end(), pc.layer1.begin(), pc.layer1.end());
    std::vector<char> in_comp(nc, 0);
    for (int32_t c : comp) in_comp[c] = 1;
    std::vector<int32_t> halo;
    for (int32_t c : comp) {
      const int64_t k = slot_of_tile[c / kTile], lane = c % kTile;
      for (int s = 0; s < SL; ++s) {
        const int32_t j = nbr[((size_t)k * SL + s) * kTile + lane];
        if (!in_comp[j]) halo.push_back(j);
      }
    }
    std::sort(halo.begin(), halo.end());
    halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
    for (int fill = kTile; fill >= 4; fill /= 2) {
      // local positions of the compute set: owned cells at their own offsets,
      // then `fill` boundary cells per tile
      std::vector<int64_t> pos(comp.size());
      for (int64_t i = 0; i < n_own; ++i) pos[i] = i;
      int64_t next = (n_own + kTile - 1) / kTile * kTile;  // the owned tail tile is not shared
      if (n_own % kTile == 0) next = n_own;
      for (size_t i = 0; i < pc.layer1.size(); ++i) {
        const int64_t slot = (int64_t)i % fill;
        if (slot == 0 && i > 0) next = (next + kTile - 1) / kTile * kTile;
        pos[n_own + i] = next++;
      }
      const int64_t n_recon = comp.empty() ? 0 : pos.back() + 1;
      // local ids: compute cells at their positions (inert lanes hold no
      // cell), then the halo
      std::vector<int32_t> glob2loc(nc, -1);
      const int64_t nrp = (n_recon + kTile - 1) / kTile * kTile;
      for (size_t i = 0; i < comp.size(); ++i) glob2loc[comp[i]] = (int32_t)pos[i];
      for (size_t i = 0; i < halo.size(); ++i) glob2loc[halo[i]] = (int32_t)(nrp + i);
      const int64_t ntl = nrp / kTile;
      std::vector<unsigned char> ahat_l((size_t)ntl * E * kTile * esz, 0);
      std::vector<float> g32_l(wform ? (size_t)ntl * E32 * kTile : 0, 0.f);
      std::vector<float2> wq_l(wform ? (size_t)ntl * EW * kTile : 0, make_float2(0.f, 0.f));
      std::vector<int32_t> nbr_l((size_t)ntl * SL * kTile, 0);
      std::vector<uint8_t> smask_l((size_t)ntl * kTile, 0);
      for (size_t i = 0; i < comp.size(); ++i) {
        const int32_t c = comp[i];
        const int64_t k = slot_of_tile[c / kTile], lane = c % kTile;
        const int64_t kl = pos[i] / kTile, ll = pos[i] % kTile;
        for (int e = 0; e < E; ++e)
          memcpy(&ahat_l[(((size_t)kl * E + e) * kTile + ll) * esz],
                 &ahat[(((size_t)k * E + e) * kTile + lane) * esz], esz);
        if (wform) {
          for (int e = 0; e < E32; ++e)
            g32_l[((size_t)kl * E32 + e) * kTile + ll] = g32[((size_t)k * E32 + e) * kTile + lane];
          for (int e = 0; e < EW; ++e)
            wq_l[((size_t)kl * EW + e) * kTile + ll] = wq[((size_t)k * EW + e) * kTile + lane];
        }
        for (int s = 0; s < SL; ++s)
          nbr_l[((size_t)kl * SL + s) * kTile + ll] =
              glob2loc[nbr[((size_t)k * SL + s) * kTile + lane]];
        smask_l[(size_t)kl * kTile + ll] = smask[(size_t)k * kTile + lane];
      }
      // every local tile's halo within kHaloMax cells?
      bool ok = true;
      std::vector<int32_t> ids;
      for (int64_t t = 0; t < ntl && ok; ++t) {
        const int32_t* tn = &nbr_l[(size_t)t * SL * kTile];
        ids.assign(tn, tn + (size_t)SL * kTile);
        std::sort(ids.begin(), ids.end());
        ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
        ok = (int)ids.size() <= kHaloMax;
      }
      if (!ok && fill > 4) continue;
      ahat.swap(ahat_l);
      g32.swap(g32_l);
      wq.swap(wq_l);
      nbr.swap(nbr_l);
      smask.swap(smask_l);
      ntile = ntl;
      n_valid = n_recon;
      n_state = nrp + (int64_t)halo.size();
      ctx->n_own = n_own;
      ctx->n_comp = n_recon;
      ctx->loc2glob.assign(n_state, -1);
      for (int64_t g = 0; g < nc; ++g)
        if (glob2loc[g] >= 0) ctx->loc2glob[glob2loc[g]] = (int32_t)g;
      // receive lists: halo and boundary-layer cells by owning part, ascending
      // global id
      ctx->recv_loc.assign(n_parts, {});
      std::vector<int32_t> foreign(pc.layer1);
      foreign.insert(foreign.end(), halo.begin(), halo.end());
      std::sort(foreign.begin(), foreign.end());
      for (int32_t g : foreign) {
        const int32_t q = (int32_t)(std::upper_bound(ctx->part_bounds.begin(),
                                                     ctx->part_bounds.end(), (int64_t)g) -
                                    ctx->part_bounds.begin()) - 1;
        ctx->recv_loc[q].push_back(glob2loc[g]);
      }
      break;
    }
  }
  const int64_t npad = ntile * kTile;
  // reverse stencil adjacency (adjoint gather): for every cell the d_bar
  // entries (tile * SL + slot) * 32 + lane of the slots that hold it (int32:
  // built for meshes with npad * SL < 2^31; the adjoint refuses larger ones)
  ctx->rev_off_h.clear();
  ctx->rev_idx_h.clear();
  if ((int64_t)npad * SL < ((int64_t)1 << 31)) {
    std::vector<int64_t> cnt(n_state + 1, 0);
    for (int64_t c = 0; c < n_valid; ++c) {
      const int64_t tile = c / kTile, lane = c % kTile;
      for (int s = 0; s < SL; ++s) {
        if (s >= ns && !((smask[c] >> ((s - ns) / kSmallN)) & 1)) continue;
        cnt[nbr[((size_t)tile * SL + s) * kTile + lane] + 1]++;
      }
    }
    for (int64_t c = 0; c < n_state; ++c) cnt[c + 1] += cnt[c];
    ctx->rev_off_h = cnt;
    ctx->rev_idx_h.assign(cnt[n_state], 0);
    std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
    for (int64_t c = 0; c < n_valid; ++c) {
      const int64_t tile = c / kTile, lane = c % kTile;
      for (int s = 0; s < SL; ++s) {
        if (s >= ns && !((smask[c] >> ((s - ns) / kSmallN)) & 1)) continue;
        int32_t j = nbr[((size_t)tile * SL + s) * kTile + lane];
        ctx->rev_idx_h[pos[j]++] = (int32_t)((tile * SL + s) * kTile + lane);
      }
    }
  }
  // per-tile stencil halos (distinct stencil cells of each 32-cell tile)
  bool halo_ok = true;
  std::vector<int32_t> hoff(ntile + 1, 0), hids;
  std::vector<uint16_t> hloc((size_t)ntile * SL * kTile, 0);
  {
    std::vector<int32_t> ids;
    for (int64_t t = 0; t < ntile && halo_ok; ++t) {
      const int32_t* tn = &nbr[(size_t)t * SL * kTile];
      ids.assign(tn, tn + (size_t)SL * kTile);
      std::sort(ids.begin(), ids.end());
      ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
      if ((int)ids.size() > kHaloMax) {
        halo_ok = false;
        break;
      }
      // halo position (bits 0-7) and, for the adjoint, the lane's rank among
      // the tile's valid lanes with the same position in the slot (bits 8-12)
      const int nval = (int)std::min<int64_t>(kTile, n_valid - t * kTile);
      for (int s = 0; s < SL; ++s)
        for (int ln = 0; ln < kTile; ++ln) {
          const size_t i = (size_t)s * kTile + ln;
          const int pos = (int)(std::lower_bound(ids.begin(), ids.end(), tn[i]) - ids.begin());
          int rank = 0;
          if (ln < nval)
            for (int j = 0; j < ln; ++j) rank += tn[(size_t)s * kTile + j] == tn[i];
          hloc[(size_t)t * SL * kTile + i] = (uint16_t)(pos | (rank << 8));
        }
      hids.insert(hids.end(), ids.begin(), ids.end());
      hoff[t + 1] = (int32_t)hids.size();
    }
  }
  // reverse map of the halo entries (tiled adjoint): for every cell the
  // indices i with hids[i] == cell, in increasing i
  ctx->hrev_off_h.clear();
  ctx->hrev_idx_h.clear();
  if (halo_ok) {
    std::vector<int64_t> cnt(n_state + 1, 0);
    for (int32_t j : hids) cnt[(size_t)j + 1]++;
    for (int64_t c = 0; c < n_state; ++c) cnt[c + 1] += cnt[c];
    ctx->hrev_off_h = cnt;
    ctx->hrev_idx_h.assign(hids.size(), 0);
    std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
    for (size_t i = 0; i < hids.size(); ++i) ctx->hrev_idx_h[pos[hids[i]]++] = (int32_t)i;
  }
  int e = upload(ctx, ctx->b_ahat, ahat.data(), ahat.size());
  if (!e) e = upload(ctx, ctx->b_nbr, nbr.data(), nbr.size() * sizeof(int32_t));
  if (!e && halo_ok) e = upload(ctx, ctx->b_halo_off, hoff.data(), hoff.size() * 4);
  if (!e && halo_ok) e = upload(ctx, ctx->b_halo_ids, hids.data(), hids.size() * 4);
  if (!e && halo_ok) e = upload(ctx, ctx->b_halo_loc, hloc.data(), hloc.size() * 2);
  if (!e) e = upload(ctx, ctx->b_smask, smask.data(), smask.size());
  if (!e && wform) e = upload(ctx, ctx->b_g32, g32.data(), g32.size() * sizeof(float));
  if (!e && wform) e = upload(ctx, ctx->b_wq, wq.data(), wq.size() * sizeof(float2));
  if (e) return e;
  // device mesh descriptor
  DeviceMesh& dm = ctx->dm;
  dm.n_var = p.n_var;
  dm.order = p.order;
  dm.m = m;
  dm.ns = ns;
  dm.nq = ctx->nq;
  dm.e_entries = E;
  dm.flux = p.flux;
  dm.precision = p.precision;
  dm.linear = p.linear;
  dm.ct = p.ct;
  dm.eps = p.eps;
  dm.gamma = p.gamma;
  dm.adv_x = p.adv_x;
  dm.adv_y = p.adv_y;
  dm.adv_field = p.adv_field;
  dm.adv_cx = p.adv_cx;
  dm.adv_cy = p.adv_cy;
  dm.adv_omega = p.adv_omega;
  dm.adv_r1 = p.adv_r1;
  dm.adv_r2 = p.adv_r2;
  dm.scheme = p.scheme;
  dm.cweno_dk = p.cweno_dk;
  dm.charvar = p.charvar;
  dm.positivity = p.positivity;
  dm.debug = p.debug;
  dm.coef_out = nullptr;
  if (p.charvar && ctx->device >= 0) {
    int e4 = dev_alloc(ctx, ctx->b_coef, sizeof(double) * (size_t)npad * 4 * (m + 15));
    if (e4) return e4;
    dm.coef_out = (double*)ctx->b_coef.p;
  }
  dm.cell_speed = nullptr;
  if (p.n_var == 1 && p.adv_field == 1) {
    // CFL speed: |omega| times the largest r phi(r) over the vertices (a cell
    // at rest does not limit the step)
    auto taper = [&](double r) {
      if (!(p.adv_r2 > p.adv_r1) || r <= p.adv_r1) return 1.0;
      if (r >= p.adv_r2) return 0.0;
      const double s = (r - p.adv_r1) / (p.adv_r2 - p.adv_r1);
      return 1.0 - s * s * (3.0 - 2.0 * s);
    };
    std::vector<double> sp(npad, 1e-300);
    for (int64_t c = 0; c < nc; ++c) {
      const double* P = &ctx->P[6 * (size_t)ctx->perm[c]];
      double smax = 0.0;
      for (int k = 0; k < 3; ++k) {
        const double dx = P[2 * k] - p.adv_cx, dy = P[2 * k + 1] - p.adv_cy;
        const double r = std::sqrt(dx * dx + dy * dy);
        smax = std::max(smax, r * taper(r));
      }
      const double sc = std::fabs(p.adv_omega) * smax;
      sp[c] = sc > 0.0 ? sc : 1e-300;
    }
    int e3 = upload(ctx, ctx->b_cspeed, sp.data(), sp.size() * sizeof(double));
    if (e3) return e3;
    dm.cell_speed = (const double*)ctx->b_cspeed.p;
  }
  dm.cfl = p.cfl;
  dm.variant = p.recon_variant;
  dm.halo = HaloArgs{};
  if (halo_ok && ctx->device >= 0) {
    dm.halo.off = (const int32_t*)ctx->b_halo_off.p;
    dm.halo.ids = (const int32_t*)ctx->b_halo_ids.p;
    dm.halo.nbr_loc = (const uint16_t*)ctx->b_halo_loc.p;
  }
  dm.err_flag = (int*)ctx->b_flag.p;
  dm.ahat = ctx->b_ahat.p;
  dm.g32 = wform ? (const float*)ctx->b_g32.p : nullptr;
  dm.wq = wform ? (const float2*)ctx->b_wq.p : nullptr;
  dm.nbr = (const int32_t*)ctx->b_nbr.p;
  dm.smask = (const uint8_t*)ctx->b_smask.p;
  std::copy(R.psi_t, R.psi_t + kMaxPts * kMaxM, dm.eval.psi);
  for (int i = 0; i < kMaxPts * kMaxM; ++i) {
    const float hi = (float)R.psi_t[i];
    dm.eval_df.psi[i] = make_float2(hi, (float)(R.psi_t[i] - (double)hi));
  }
  dm.psi_df = nullptr;
  dm.psi_d = nullptr;
  if (wform && store == TENO_FP64) {
    int e2 = upload(ctx, ctx->b_psi, dm.eval_df.psi, sizeof(dm.eval_df.psi));
    if (e2) return e2;
    dm.psi_df = (const float2*)ctx->b_psi.p;
  } else if (wform) {
    int e2 = upload(ctx, ctx->b_psi, dm.eval.psi, sizeof(dm.eval.psi));
    if (e2) return e2;
    dm.psi_d = (const double*)ctx->b_psi.p;
  }
  for (int k = 0; k < kMaxNq; ++k) {
    dm.gw[k] = k < ctx->nq ? R.gw[k] : 0.0;
    dm.gt[k] = k < ctx->nq ? R.gt[k] : 0.0;
  }
  return TENO_OK;
}

int upload_mesh(teno_ctx* ctx) {
  const int64_t nc = ctx->nc, npad = ctx->npad;
  // faces in internal order: owner = the side with the smaller internal index
  std::vector<int32_t> fcells, cfaces(3 * npad, 0);
  std::vector<int8_t> fedges;
  std::vector<double> fgeom;
  for (int64_t c = 0; c < nc; ++c) {
    const int32_t u = ctx->perm[c];
    for (int e = 0; e < 3; ++e) {
      const int32_t nu = ctx->fnbr[3 * u + e];
      const int64_t n = nu >= 0 ? ctx->iperm[nu] : -1;
      if (n >= 0 && n < c) continue;
      const int64_t f = (int64_t)fcells.size() / 2;
      fcells.push_back((int32_t)c);
      fcells.push_back((int32_t)n);
      fedges.push_back((int8_t)e);
      fedges.push_back((int8_t)(n >= 0 ? ctx->fedge[3 * u + e] : ctx->fbc[3 * u + e]));
      const double* P = &ctx->P[6 * u];
      const int e1 = (e + 1) % 3;
      const double dx = P[2 * e1] - P[2 * e], dy = P[2 * e1 + 1] - P[2 * e + 1];
      const double len = std::hypot(dx, dy);
      fgeom.push_back(dy / len);
      fgeom.push_back(-dx / len);
      fgeom.push_back(len);
      // start point of the edge in the frame of the adjacent cell with the
      // smaller user id (differs from the owner's frame only across a
      // periodic wrap): there the neighbour's edge runs the other way
      if (n >= 0 && nu < u) {
        const double* Pn = &ctx->P[6 * (size_t)nu];
        const int s0 = (ctx->fedge[3 * u + e] + 1) % 3;
        fgeom.push_back(Pn[2 * s0]);
        fgeom.push_back(Pn[2 * s0 + 1]);
      } else {
        fgeom.push_back(P[2 * e]);
        fgeom.push_back(P[2 * e + 1]);
      }
      cfaces[3 * c + e] = (int32_t)(2 * f);
      if (n >= 0) cfaces[3 * n + ctx->fedge[3 * u + e]] = (int32_t)(2 * f + 1);
    }
  }
  ctx->nface = (int64_t)fcells.size() / 2;
  std::vector<double> inv_area(npad, 0.0), cfl_len(npad, 1.0);
  // the outflow layer: cells with a face on an outflow boundary enter every
  // face flux with their cell average
  std::vector<uint8_t> fo(npad, 0);
  for (int64_t c = 0; c < nc; ++c) {
    const int32_t u = ctx->perm[c];
    inv_area[c] = 1.0 / ctx->area[u];
    cfl_len[c] = 4.0 * ctx->area[u] / ctx->perim[u];
    for (int e = 0; e < 3; ++e)
      if (ctx->fnbr[3 * u + e] < 0 && ctx->fbc[3 * u + e] == TENO_BC_OUTFLOW) fo[c] = 1;
  }
  int rc = upload(ctx, ctx->b_fcells, fcells.data(), fcells.size() * 4);
  if (!rc) rc = upload(ctx, ctx->b_fedges, fedges.data(), fedges.size());
  if (!rc) rc = upload(ctx, ctx->b_fgeom, fgeom.data(), fgeom.size() * 8);
  std::vector<float2> fgeom2(3 * (size_t)ctx->nface);
  for (int64_t f = 0; f < ctx->nface; ++f)
    for (int i = 0; i < 3; ++i) {
      const double x = fgeom[5 * f + i];
      const float h = (float)x;
      fgeom2[3 * f + i] = make_float2(h, (float)(x - (double)h));
    }
  if (!rc) rc = upload(ctx, ctx->b_fgeom2, fgeom2.data(), fgeom2.size() * sizeof(float2));
  if (!rc) rc = upload(ctx, ctx->b_cfaces, cfaces.data(), cfaces.size() * 4);
  if (!rc) rc = upload(ctx, ctx->b_inv_area, inv_area.data(), inv_area.size() * 8);
  if (!rc) rc = upload(ctx, ctx->b_cfl_len, cfl_len.data(), cfl_len.size() * 8);
  if (!rc) {
    std::vector<float2> ilen2(npad);
    for (int64_t c = 0; c < npad; ++c) {
      const double x = 1.0 / cfl_len[c];
      const float h = (float)x;
      ilen2[c] = make_float2(h, (float)(x - (double)h));
    }
    rc = upload(ctx, ctx->b_cfl_ilen2, ilen2.data(), ilen2.size() * sizeof(float2));
  }
  if (!rc) rc = upload(ctx, ctx->b_perm, ctx->perm.data(), ctx->perm.size() * 4);
  std::vector<int32_t> fo_list;
  for (int64_t c = 0; c < nc; ++c)
    if (fo[c]) fo_list.push_back((int32_t)c);
  if (!rc && !fo_list.empty()) rc = upload(ctx, ctx->b_fo, fo_list.data(), fo_list.size() * 4);
  if (rc) return rc;
  DeviceMesh& dm = ctx->dm;
  dm.n_cell = nc;
  dm.n_pad = npad;
  dm.n_recon = nc;
  dm.n_update = nc;
  dm.n_face = ctx->nface;
  ctx->sn = nc;
  ctx->spad = npad;
  ctx->io_n = nc;
  ctx->part_n = 1;
  ctx->part_id = 0;
  ctx->n_own = ctx->n_comp = nc;
  ctx->h_fcells.swap(fcells);
  ctx->h_fedges.swap(fedges);
  ctx->h_fgeom.swap(fgeom);
  ctx->h_cfaces.swap(cfaces);
  ctx->h_inv_area.swap(inv_area);
  ctx->h_cfl_len.swap(cfl_len);
  ctx->h_fo.swap(fo);
  dm.fo_n = (int64_t)fo_list.size();
  dm.fo_list = dm.fo_n ? (const int32_t*)ctx->b_fo.p : nullptr;
  dm.f_cells = (const int32_t*)ctx->b_fcells.p;
  dm.f_edges = (const int8_t*)ctx->b_fedges.p;
  dm.f_geom = (const double*)ctx->b_fgeom.p;
  dm.f_geom2 = (const float2*)ctx->b_fgeom2.p;
  dm.c_faces = (const int32_t*)ctx->b_cfaces.p;
  dm.inv_area = (const double*)ctx->b_inv_area.p;
  dm.cfl_len = (const double*)ctx->b_cfl_len.p;
  dm.cfl_ilen2 = (const float2*)ctx->b_cfl_ilen2.p;
  return TENO_OK;
}

// Device mesh of a partition (after run_precompute built its layout): the
// faces touching owned cells (the global faces, owner and orientation
// unchanged, so each face flux is the same computation as on the whole
// mesh), the cell -> face map and geometry of the compute cells, and the
// permutations of the state extraction (local cell -> global user id) and of
// the owned output (identity).
int upload_partition_mesh(teno_ctx* ctx) {
  const int64_t nc = ctx->nc, n_own = ctx->n_own, n_comp = ctx->n_comp;
  const int64_t sn = (int64_t)ctx->loc2glob.size();
  const int64_t spad = (sn + kTile - 1) / kTile * kTile;
  std::vector<int32_t> glob2loc(nc, -1);
  for (int64_t l = 0; l < sn; ++l)
    if (ctx->loc2glob[l] >= 0) glob2loc[ctx->loc2glob[l]] = (int32_t)l;
  std::vector<int64_t> gf;
  for (int64_t l = 0; l < n_own; ++l) {
    const int32_t g = ctx->loc2glob[l];
    for (int e = 0; e < 3; ++e) gf.push_back(ctx->h_cfaces[3 * (size_t)g + e] >> 1);
  }
  std::sort(gf.begin(), gf.end());
  gf.erase(std::unique(gf.begin(), gf.end()), gf.end());
  const int64_t nf = (int64_t)gf.size();
  std::vector<int32_t> fcells(2 * nf), cfaces(3 * (size_t)spad, 0);
  std::vector<int8_t> fedges(2 * nf);
  std::vector<double> fgeom(5 * nf);
  std::vector<float2> fgeom2(3 * nf);
  for (int64_t f = 0; f < nf; ++f) {
    const int64_t g = gf[f];
    const int32_t o = ctx->h_fcells[2 * g], n = ctx->h_fcells[2 * g + 1];
    fcells[2 * f] = glob2loc[o];
    fcells[2 * f + 1] = n >= 0 ? glob2loc[n] : -1;
    fedges[2 * f] = ctx->h_fedges[2 * g];
    fedges[2 * f + 1] = ctx->h_fedges[2 * g + 1];
    for (int i = 0; i < 5; ++i) fgeom[5 * f + i] = ctx->h_fgeom[5 * g + i];
    for (int i = 0; i < 3; ++i) {
      const double x = fgeom[5 * f + i];
      const float h = (float)x;
      fgeom2[3 * f + i] = make_float2(h, (float)(x - (double)h));
    }
    // both sides' cell -> face entries where the side is a compute cell
    const int e0 = ctx->h_fedges[2 * g];
    cfaces[3 * (size_t)glob2loc[o] + e0] = (int32_t)(2 * f);
    if (n >= 0 && glob2loc[n] >= 0 && glob2loc[n] < n_comp)
      cfaces[3 * (size_t)glob2loc[n] + ctx->h_fedges[2 * g + 1]] = (int32_t)(2 * f + 1);
  }
  std::vector<double> inv_area(spad, 0.0), cfl_len(spad, 1.0);
  std::vector<float2> ilen2(spad);
  std::vector<int32_t> perm_in(sn, 0), perm_out(n_own);
  std::vector<int32_t> fo_list;  // outflow-layer cells among the reconstructed ones
  for (int64_t l = 0; l < spad; ++l) {
    const int32_t g = l < sn ? ctx->loc2glob[l] : -1;
    if (g >= 0 && l < n_comp) {
      inv_area[l] = ctx->h_inv_area[g];
      cfl_len[l] = ctx->h_cfl_len[g];
    }
    if (g >= 0 && l < n_comp && ctx->has_outflow && ctx->h_fo[g]) fo_list.push_back((int32_t)l);
    const double x = 1.0 / cfl_len[l];
    const float h = (float)x;
    ilen2[l] = make_float2(h, (float)(x - (double)h));
    if (l < sn) perm_in[l] = g >= 0 ? ctx->perm[g] : 0;
  }
  for (int64_t l = 0; l < n_own; ++l) perm_out[l] = (int32_t)l;
  int rc = upload(ctx, ctx->b_fcells, fcells.data(), fcells.size() * 4);
  if (!rc) rc = upload(ctx, ctx->b_fedges, fedges.data(), fedges.size());
  if (!rc) rc = upload(ctx, ctx->b_fgeom, fgeom.data(), fgeom.size() * 8);
  if (!rc) rc = upload(ctx, ctx->b_fgeom2, fgeom2.data(), fgeom2.size() * 8);
  if (!rc) rc = upload(ctx, ctx->b_cfaces, cfaces.data(), cfaces.size() * 4);
  if (!rc) rc = upload(ctx, ctx->b_inv_area, inv_area.data(), inv_area.size() * 8);
  if (!rc) rc = upload(ctx, ctx->b_cfl_len, cfl_len.data(), cfl_len.size() * 8);
  if (!rc) rc = upload(ctx, ctx->b_cfl_ilen2, ilen2.data(), ilen2.size() * sizeof(float2));
  if (!rc) rc = upload(ctx, ctx->b_perm_in, perm_in.data(), perm_in.size() * 4);
  if (!rc) rc = upload(ctx, ctx->b_perm, perm_out.data(), perm_out.size() * 4);
  if (!rc && !fo_list.empty()) rc = upload(ctx, ctx->b_fo, fo_list.data(), fo_list.size() * 4);
  const int32_t P = ctx->part_n;
  ctx->b_recv_idx.resize(P);
  ctx->b_send_idx.resize(P);
  ctx->b_xbuf.resize(2 * P);
  for (int32_t q = 0; q < P && !rc; ++q)
    rc = upload(ctx, ctx->b_recv_idx[q], ctx->recv_loc[q].data(),
                ctx->recv_loc[q].size() * 4);
  if (rc) return rc;
  DeviceMesh& dm = ctx->dm;
  dm.n_cell = sn;
  dm.n_pad = spad;
  dm.n_recon = n_comp;
  dm.n_update = n_own;
  dm.n_face = nf;
  dm.fo_n = (int64_t)fo_list.size();
  dm.fo_list = dm.fo_n ? (const int32_t*)ctx->b_fo.p : nullptr;
  dm.f_cells = (const int32_t*)ctx->b_fcells.p;
  dm.f_edges = (const int8_t*)ctx->b_fedges.p;
  dm.f_geom = (const double*)ctx->b_fgeom.p;
  dm.f_geom2 = (const float2*)ctx->b_fgeom2.p;
  dm.c_faces = (const int32_t*)ctx->b_cfaces.p;
  dm.inv_area = (const double*)ctx->b_inv_area.p;
  dm.cfl_len = (const double*)ctx->b_cfl_len.p;
  dm.cfl_ilen2 = (const float2*)ctx->b_cfl_ilen2.p;
  ctx->sn = sn;
  ctx->spad = spad;
  ctx->io_n = n_own;
  return TENO_OK;
}

// one residual evaluation of state U (internal order) into Uq / K
// split_ready: the FP32 split buffer already holds split(U) (written by the
// previous RK update); otherwise the mixed path splits U first
int stage_flux(teno_ctx* ctx, const double* U, uint8_t* sel_out, double time,
               bool split_ready = false, void* uq = nullptr) {
  if (!uq) uq = ctx->b_Uq.p;
  const uint8_t* sel_in = ctx->override_on ? (const uint8_t*)ctx->b_sel_ovr.p : nullptr;
  const bool split = ctx->prm.precision != TENO_FP64_NATIVE;
  float2* Us = split ? (float2*)ctx->b_Usplit.p : nullptr;
  if (split && !split_ready) {
    long ps = prof_begin(ctx, K_OTHER);
    CK(launch_split(ctx->dm, U, Us, ctx->stream), "split launch");
    prof_end(ctx, ps);
  }
  long pe = prof_begin(ctx, K_RECON);
  CK(launch_recon(ctx->dm, U, Us, uq, sel_out, sel_in, ctx->stream), "recon launch");
  if (ctx->dm.charvar) CK(launch_char_finish(ctx->dm, U, uq, ctx->stream), "char finish launch");
  if (ctx->dm.positivity) CK(launch_positivity(ctx->dm, U, uq, ctx->stream), "positivity launch");
  CK(launch_layer_fill(ctx->dm, U, uq, ctx->stream), "layer fill launch");
  prof_end(ctx, pe);
  pe = prof_begin(ctx, K_FLUX);
  CK(launch_face_flux(ctx->dm, uq, ctx->b_K.p, time, ctx->stream), "face flux launch");
  prof_end(ctx, pe);
  return TENO_OK;
}

int check_ready(teno_ctx* ctx, bool need_state) {
  if (!ctx) return TENO_EINVAL;
  if (ctx->device < 0) return fail(ctx, TENO_ESTATE, "host-only context: no device work");
  if (!ctx->mesh_ok || !ctx->pre_ok) return fail(ctx, TENO_ESTATE, "mesh or precompute missing");
  if (need_state && !ctx->state_ok) return fail(ctx, TENO_ESTATE, "state not set");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  return TENO_OK;
}

// copy a user-order [n_var][n_cell] array into an internal-order buffer
// (a partition extracts its state cells, owned and halo, from the whole
// mesh's array)
int to_internal(teno_ctx* ctx, const double* src, double* dst, int on_device) {
  const int64_t nc = ctx->nc;
  const int nvar = ctx->prm.n_var;
  const double* s = src;
  if (!on_device) {
    CK(cudaMemcpyAsync(ctx->b_tmp.p, src, sizeof(double) * nvar * nc, cudaMemcpyHostToDevice,
                       ctx->stream),
       "H2D");
    s = (const double*)ctx->b_tmp.p;
  }
  const bool part = ctx->part_n > 1;
  CK(launch_permute(s, dst, (const int32_t*)(part ? ctx->b_perm_in.p : ctx->b_perm.p),
                    part ? ctx->sn : nc, nc, ctx->spad, nvar, 0, ctx->stream),
     "permute");
  return TENO_OK;
}

// (a partition returns its owned cells, [n_var][n_owned] in its owned order)
int to_user(teno_ctx* ctx, const double* src, double* dst, int on_device) {
  const int64_t nc = ctx->io_n;
  const int nvar = ctx->prm.n_var;
  double* d = on_device ? dst : (double*)ctx->b_tmp.p;
  CK(launch_permute(src, d, (const int32_t*)ctx->b_perm.p, nc, ctx->spad, nc, nvar, 1,
                    ctx->stream),
     "permute");
  if (!on_device) {
    CK(cudaMemcpyAsync(dst, d, sizeof(double) * nvar * nc, cudaMemcpyDeviceToHost, ctx->stream),
       "D2H");
    CK(cudaStreamSynchronize(ctx->stream), "sync");
  }
  return TENO_OK;
}

int ensure_adjoint(teno_ctx* ctx) {
  if (ctx->adj_ok) return TENO_OK;
  const int64_t npad = ctx->spad, nc = ctx->sn;
  const int nv = ctx->prm.n_var;
  const size_t ntile = npad / kTile;
  // tiled VJP with the W-form reconstruction (variant 2, FP64 path, Euler,
  // every tile with its halo); otherwise the per-slot d_bar and the reverse
  // stencil map
  ctx->adj_tiled = ctx->prm.precision == TENO_FP64 && nv == 4 && ctx->prm.recon_variant == 2 &&
                   ctx->dm.halo.off && ctx->dm.wq && !ctx->hrev_off_h.empty() &&
                   ctx->dm.err_flag;
  if (!ctx->adj_tiled && ctx->rev_off_h.empty())
    return fail(ctx, TENO_EINVAL,
                "adjoint: mesh too large for 32-bit stencil-entry indices (cells x slots >= 2^31)");
  int rc = TENO_OK;
  if (ctx->adj_tiled) {
    rc = dev_alloc(ctx, ctx->b_hpart, sizeof(double) * std::max<size_t>(1, ctx->hrev_idx_h.size()) * nv);
    if (!rc)
      rc = upload(ctx, ctx->b_hrev_off, ctx->hrev_off_h.data(), sizeof(int64_t) * (nc + 1));
    if (!rc)
      rc = upload(ctx, ctx->b_hrev_idx, ctx->hrev_idx_h.data(),
                  sizeof(int32_t) * ctx->hrev_idx_h.size());
  } else {
    rc = dev_alloc(ctx, ctx->b_dbar, sizeof(double) * ntile * ctx->SL * nv * kTile);
    if (!rc) rc = upload(ctx, ctx->b_rev_off, ctx->rev_off_h.data(), sizeof(int64_t) * (nc + 1));
    if (!rc)
      rc = upload(ctx, ctx->b_rev_idx, ctx->rev_idx_h.data(),
                  sizeof(int32_t) * ctx->rev_idx_h.size());
    if (!rc) CK(cudaMemsetAsync(ctx->b_dbar.p, 0, ctx->b_dbar.bytes, ctx->stream), "memset");
  }
  if (!rc) rc = dev_alloc(ctx, ctx->b_uself, sizeof(double) * nv * npad);
  if (!rc) rc = dev_alloc(ctx, ctx->b_Uqbar, sizeof(double) * npad * 3 * ctx->nq * nv);
  if (!rc) rc = dev_alloc(ctx, ctx->b_l1, sizeof(double) * nv * npad);
  if (!rc) rc = dev_alloc(ctx, ctx->b_l2, sizeof(double) * nv * npad);
  if (!rc) rc = dev_alloc(ctx, ctx->b_lamn, sizeof(double) * nv * npad);
  if (!rc) rc = dev_alloc(ctx, ctx->b_vtmp, sizeof(double) * nv * npad);
  if (!rc) rc = dev_alloc(ctx, ctx->b_selA, (size_t)nv * npad);
  for (int k = 0; k < 2 && !rc; ++k) {
    rc = dev_alloc(ctx, ctx->b_Uq_st[k], ctx->b_Uq.bytes);
    if (!rc) rc = dev_alloc(ctx, ctx->b_sel_st[k], (size_t)nv * npad);
  }
  if (rc) return rc;
  // a partition's VJP leaves the Gauss slots of boundary-layer edges that
  // face no owned cell, and the own terms of halo cells, unwritten: zero
  CK(cudaMemsetAsync(ctx->b_Uqbar.p, 0, ctx->b_Uqbar.bytes, ctx->stream), "memset");
  CK(cudaMemsetAsync(ctx->b_uself.p, 0, ctx->b_uself.bytes, ctx->stream), "memset");
  if (ctx->has_outflow) {
    // written for the edges of outflow-layer cells only, zero elsewhere
    rc = dev_alloc(ctx, ctx->b_ubd, sizeof(double) * 3 * nv * npad);
    if (rc) return rc;
    CK(cudaMemsetAsync(ctx->b_ubd.p, 0, ctx->b_ubd.bytes, ctx->stream), "memset");
  }
  ctx->adj_ok = true;
  return TENO_OK;
}

// v = (dR/dU)^T w at U (all internal order).  With uq_saved / sel_saved (the
// Gauss-point values and selection a forward stage at U already produced)
// the reconstruction is not repeated.
int vjp_internal(teno_ctx* ctx, const double* U, const double* w, double* v, double time,
                 const void* uq_saved = nullptr, const uint8_t* sel_saved = nullptr) {
  int rc = ensure_adjoint(ctx);
  if (rc) return rc;
  const uint8_t* sel_in = ctx->override_on ? (const uint8_t*)ctx->b_sel_ovr.p : nullptr;
  const uint8_t* sel = sel_in ? sel_in : sel_saved;
  const void* uq = uq_saved;
  if (!uq) {
    uint8_t* sel_out = (uint8_t*)ctx->b_selA.p;
    float2* Us = nullptr;
    if (ctx->prm.precision != TENO_FP64_NATIVE) {
      Us = (float2*)ctx->b_Usplit.p;
      CK(launch_split(ctx->dm, U, Us, ctx->stream), "split launch");
      ctx->split_ok = false;
    }
    long pr = prof_begin(ctx, K_RECON);
    CK(launch_recon(ctx->dm, U, Us, ctx->b_Uq.p, sel_out, sel_in, ctx->stream), "recon launch");
    CK(launch_layer_fill(ctx->dm, U, ctx->b_Uq.p, ctx->stream), "layer fill launch");
    prof_end(ctx, pr);
    uq = ctx->b_Uq.p;
    if (!sel_in) sel = sel_out;
  }
  long pe = prof_begin(ctx, K_FLUX_VJP);
  double* ubd = ctx->dm.fo_n ? (double*)ctx->b_ubd.p : nullptr;
  CK(launch_face_flux_vjp(ctx->dm, uq, w, (double*)ctx->b_Uqbar.p, time, ctx->stream),
     "flux vjp launch");
  CK(launch_layer_vjp(ctx->dm, (double*)ctx->b_Uqbar.p, ubd, ctx->stream), "layer vjp launch");
  prof_end(ctx, pe);
  pe = prof_begin(ctx, K_RECON_VJP);
  if (ctx->adj_tiled)
    CK(launch_recon_vjp_tma(ctx->dm, sel, (const double*)ctx->b_Uqbar.p, (double*)ctx->b_hpart.p,
                            (double*)ctx->b_uself.p, ctx->stream),
       "recon vjp launch");
  else
    CK(launch_recon_vjp(ctx->dm, sel, (const double*)ctx->b_Uqbar.p, (double*)ctx->b_dbar.p,
                        (double*)ctx->b_uself.p, ctx->stream),
       "recon vjp launch");
  prof_end(ctx, pe);
  pe = prof_begin(ctx, K_SCATTER);
  if (ctx->adj_tiled)
    CK(launch_scatter_gather(ctx->dm, (const int64_t*)ctx->b_hrev_off.p,
                             (const int32_t*)ctx->b_hrev_idx.p, (const double*)ctx->b_hpart.p,
                             (const double*)ctx->b_uself.p, v, ubd, ctx->stream),
       "scatter launch");
  else
    CK(launch_scatter_gather(ctx->dm, (const int64_t*)ctx->b_rev_off.p,
                             (const int32_t*)ctx->b_rev_idx.p, (const double*)ctx->b_dbar.p,
                             (const double*)ctx->b_uself.p, v, ubd, ctx->stream),
       "scatter launch");
  prof_end(ctx, pe);
  return TENO_OK;
}

// SSP-RK3 stage: out = cn*Un + cs*(Us + dt R(Us))
// (the mixed path keeps split(U) current: each RK update writes the split of
// its output, which the next stage's reconstruction reads)
int rk_stage(teno_ctx* ctx, const double* Un, const double* Us, double* out, double cn,
             double cs, double dt, const double* max_lam, double time, bool split_ready,
             void* uq = nullptr, uint8_t* sel_out = nullptr) {
  int rc = stage_flux(ctx, Us, sel_out, time, split_ready, uq);
  if (rc) return rc;
  const bool split = ctx->prm.precision != TENO_FP64_NATIVE;
  long pe = prof_begin(ctx, K_GATHER);
  CK(launch_gather(ctx->dm, ctx->b_K.p, Un, Us, out, 1, cn, cs, dt, max_lam,
                   (int*)ctx->b_flag.p, split ? (float2*)ctx->b_Usplit.p : nullptr, ctx->stream),
     "gather launch");
  prof_end(ctx, pe);
  return TENO_OK;
}

}  // namespace

// ========================================================================
// C ABI

extern "C" {

void teno_default_params(teno_params* p) {
  if (!p) return;
  p->order = 5;
  p->n_var = 4;
  p->flux = TENO_FLUX_HLL;
  p->precision = TENO_FP64;
  p->linear = 0;
  p->nq = 0;
  p->recon_variant = 2;
  p->ct = 1e-6;
  p->eps = 1e-12;
  p->gamma = 1.4;
  p->adv_x = 1.0;
  p->adv_y = 1.0;
  p->adv_field = 0;
  p->adv_cx = 0.5;
  p->adv_cy = 0.5;
  p->adv_omega = 1.0;
  p->adv_r1 = 0.0;
  p->adv_r2 = 0.0;
  p->scheme = 0;
  p->cweno_dk = 1e4;
  p->charvar = 0;
  p->positivity = 0;
  p->debug = 0;
  p->cfl = 0.4;
}

int teno_create(teno_ctx** out, int device, void* cuda_stream) {
  if (!out) return TENO_EINVAL;
  *out = nullptr;
  if (device == -1) {  // host-only: mesh and stencil preprocessing without a GPU
    teno_ctx* ctx = new (std::nothrow) teno_ctx();
    if (!ctx) return TENO_ENOMEM;
    ctx->device = -1;
    *out = ctx;
    return TENO_OK;
  }
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return TENO_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return TENO_ECUDA;
  teno_ctx* ctx = new (std::nothrow) teno_ctx();
  if (!ctx) return TENO_ENOMEM;
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  if (dev_alloc(ctx, ctx->b_maxlam, 64) || dev_alloc(ctx, ctx->b_flag, 64)) {
    delete ctx;
    return TENO_ENOMEM;
  }
  cudaMemset(ctx->b_flag.p, 0, 64);
  cudaMemset(ctx->b_maxlam.p, 0, 64);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    delete ctx;
    return TENO_ECUDA;
  }
  *out = ctx;
  return TENO_OK;
}

int teno_destroy(teno_ctx* ctx) {
  if (!ctx) return TENO_OK;
  if (ctx->device < 0) {
    delete ctx;
    return TENO_OK;
  }
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  DevBuf* bufs[] = {&ctx->b_halo_off, &ctx->b_halo_ids, &ctx->b_halo_loc, &ctx->b_g32, &ctx->b_wq, &ctx->b_psi, &ctx->b_cspeed, &ctx->b_coef, &ctx->b_ahat, &ctx->b_nbr, &ctx->b_smask, &ctx->b_fcells, &ctx->b_fedges,
                    &ctx->b_fgeom, &ctx->b_fgeom2, &ctx->b_cfaces, &ctx->b_inv_area, &ctx->b_cfl_len, &ctx->b_cfl_ilen2,
                    &ctx->b_perm, &ctx->b_U, &ctx->b_U1, &ctx->b_U2, &ctx->b_R, &ctx->b_tmp,
                    &ctx->b_Uq, &ctx->b_K, &ctx->b_sel, &ctx->b_sel_ovr, &ctx->b_maxlam,
                    &ctx->b_Usplit,
                    &ctx->b_flag, &ctx->b_rev_off, &ctx->b_rev_idx, &ctx->b_dbar, &ctx->b_uself,
                    &ctx->b_hrev_off, &ctx->b_hrev_idx, &ctx->b_hpart,
                    &ctx->b_Uqbar, &ctx->b_l1, &ctx->b_l2, &ctx->b_lamn, &ctx->b_vtmp,
                    &ctx->b_selA, &ctx->b_Uq_st[0], &ctx->b_Uq_st[1], &ctx->b_sel_st[0],
                    &ctx->b_sel_st[1]};
  for (DevBuf* b : bufs) dev_free(*b);
  dev_free(ctx->b_perm_in);
  dev_free(ctx->b_ubd);
  for (DevBuf& b : ctx->tape) dev_free(b);
  for (auto* v : {&ctx->b_recv_idx, &ctx->b_send_idx, &ctx->b_xbuf})
    for (DevBuf& b : *v) dev_free(b);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  delete ctx;
  return TENO_OK;
}

const char* teno_last_error(teno_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int teno_set_stream(teno_ctx* ctx, void* cuda_stream) {
  if (!ctx) return TENO_EINVAL;
  ctx->stream = (cudaStream_t)cuda_stream;
  return TENO_OK;
}

int teno_mesh_load(teno_ctx* ctx, int64_t n_vert, const double* xy, int64_t n_cell,
                   const int32_t* tri, int64_t n_bface, const int32_t* bface,
                   const double* period) {
  if (!ctx) return TENO_EINVAL;
  if (!xy || !tri || n_vert < 3 || n_cell < 1 || n_bface < 0 || (n_bface > 0 && !bface))
    return fail(ctx, TENO_EINVAL, "mesh_load: bad arguments");
  if (n_cell > (int64_t)INT32_MAX / 4) return fail(ctx, TENO_EINVAL, "mesh_load: too many cells");
  if (period && !(period[0] > 0 && period[1] > 0))
    return fail(ctx, TENO_EINVAL, "mesh_load: non-positive period");
  if (ctx->device >= 0) CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  ctx->mesh_ok = ctx->pre_ok = ctx->state_ok = ctx->adj_ok = ctx->stages_ok = false;
  ctx->override_on = false;
  ctx->has_time_bc = false;
  ctx->has_outflow = false;
  ctx->nv = n_vert;
  ctx->nc = n_cell;
  ctx->npad = (n_cell + kTile - 1) / kTile * kTile;
  ctx->periodic = period != nullptr;
  ctx->L[0] = period ? period[0] : 0.0;
  ctx->L[1] = period ? period[1] : 0.0;
  int rc = build_mesh(ctx, xy, tri, n_bface, bface);
  if (!rc) rc = upload_mesh(ctx);
  if (rc) return rc;
  ctx->time = 0.0;
  ctx->mesh_ok = true;
  return TENO_OK;
}

int teno_get_permutation(teno_ctx* ctx, int32_t* perm) {
  if (!ctx || !perm) return TENO_EINVAL;
  if (!ctx->mesh_ok) return fail(ctx, TENO_ESTATE, "no mesh");
  std::copy(ctx->perm.begin(), ctx->perm.end(), perm);
  return TENO_OK;
}

static int precompute_impl(teno_ctx* ctx, const teno_params* p, int32_t n_parts, int32_t part) {
  if (!ctx || !p) return TENO_EINVAL;
  if (!ctx->mesh_ok) return fail(ctx, TENO_ESTATE, "precompute before mesh_load");
  if (p->order < 3 || p->order > 6 || (p->n_var != 1 && p->n_var != 4) ||
      p->precision < TENO_FP64 || p->precision > TENO_FP64_NATIVE || p->flux < 0 ||
      p->flux > 2 || (p->n_var == 1) != (p->flux == TENO_FLUX_UPWIND) || !(p->ct > 0) ||
      !(p->eps > 0) || !(p->gamma > 1.0) || !(p->cfl > 0) || p->recon_variant < 0 ||
      p->recon_variant > 2 || p->adv_field < 0 || p->adv_field > 1 ||
      (p->adv_field == 1 && (p->n_var != 1 || !std::isfinite(p->adv_omega) ||
                             !std::isfinite(p->adv_cx) || !std::isfinite(p->adv_cy) ||
                             !std::isfinite(p->adv_r1) || !std::isfinite(p->adv_r2))) ||
      p->scheme < 0 || p->scheme > 1 || (p->scheme == 1 && !(p->cweno_dk > 1.0)) ||
      p->charvar < 0 || p->charvar > 1 || (p->charvar == 1 && (p->n_var != 4 || p->scheme != 0)) ||
      p->positivity < 0 || p->positivity > 1 ||
      (p->positivity == 1 && (p->n_var != 4 || p->charvar != 0)) || p->debug < 0 || p->debug > 3)
    return fail(ctx, TENO_EINVAL, "precompute: bad parameters");
  const int nq_default = p->order <= 4 ? 2 : 3;
  if (p->nq != 0 && p->nq != nq_default)
    return fail(ctx, TENO_EINVAL, "precompute: only the default Gauss point count is built");
  if (!ctx->periodic && p->n_var != 4)
    return fail(ctx, TENO_EINVAL, "precompute: boundary conditions need the Euler equations");
  if (n_parts > 1 && (p->adv_field != 0 || p->charvar != 0))
    return fail(ctx, TENO_EINVAL,
                "partition: constant advection velocity and conservative variables only");
  if (ctx->device >= 0) CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  ctx->pre_ok = ctx->state_ok = ctx->adj_ok = ctx->stages_ok = false;
  if (ctx->part_n > 1 && n_parts == 1) {
    // back from a partition to the whole mesh: its faces and geometry again
    int r0 = upload_mesh(ctx);
    if (r0) return r0;
  }
  ctx->override_on = false;
  ctx->prm = *p;
  ctx->nq = nq_default;
  ctx->m = unknowns(p->order);
  ctx->ns = 2 * (ctx->m + 1);
  ctx->E = ctx->m * ctx->ns + kSmallK * kSmallN * kSmallM;
  ctx->SL = ctx->ns + kSmallK * kSmallN;
  ctx->part_n = n_parts;
  ctx->part_id = part;
  int rc = run_precompute(ctx, n_parts, part);
  if (!rc && n_parts > 1) rc = upload_partition_mesh(ctx);
  if (rc) {
    ctx->part_n = 1;
    return rc;
  }
  const int64_t npad = ctx->spad;
  const int nv = p->n_var;
  const size_t tsz = p->precision == TENO_FP32_MIXED ? 4 : 8;
  rc = dev_alloc(ctx, ctx->b_U, 8 * nv * npad);
  if (!rc) rc = dev_alloc(ctx, ctx->b_U1, 8 * nv * npad);
  if (!rc) rc = dev_alloc(ctx, ctx->b_U2, 8 * nv * npad);
  if (!rc) rc = dev_alloc(ctx, ctx->b_R, 8 * nv * npad);
  if (!rc) rc = dev_alloc(ctx, ctx->b_tmp, 8 * nv * std::max(npad, ctx->nc));
  if (!rc) rc = dev_alloc(ctx, ctx->b_Uq, tsz * npad * 3 * ctx->nq * nv);
  if (!rc) rc = dev_alloc(ctx, ctx->b_K, tsz * std::max<int64_t>(1, ctx->nface) * nv);
  if (!rc) rc = dev_alloc(ctx, ctx->b_sel, (size_t)nv * npad);
  if (!rc) rc = dev_alloc(ctx, ctx->b_sel_ovr, (size_t)nv * npad);
  if (!rc && p->precision != TENO_FP64_NATIVE) rc = dev_alloc(ctx, ctx->b_Usplit, 8 * nv * npad);
  if (rc) return rc;
  ctx->split_ok = false;
  if (ctx->device < 0) {
    ctx->pre_ok = true;
    return TENO_OK;
  }
  CK(cudaMemsetAsync(ctx->b_U.p, 0, ctx->b_U.bytes, ctx->stream), "memset");
  CK(cudaMemsetAsync(ctx->b_U1.p, 0, ctx->b_U1.bytes, ctx->stream), "memset");
  CK(cudaMemsetAsync(ctx->b_U2.p, 0, ctx->b_U2.bytes, ctx->stream), "memset");
  if (ctx->b_Usplit.p)
    CK(cudaMemsetAsync(ctx->b_Usplit.p, 0, ctx->b_Usplit.bytes, ctx->stream), "memset");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  ctx->pre_ok = true;
  return TENO_OK;
}

int teno_precompute_stencils(teno_ctx* ctx, const teno_params* p) {
  return precompute_impl(ctx, p, 1, 0);
}

int teno_precompute_partition(teno_ctx* ctx, const teno_params* p, int32_t n_parts,
                              int32_t part) {
  if (!ctx || !p) return TENO_EINVAL;
  if (n_parts < 1 || part < 0 || part >= n_parts)
    return fail(ctx, TENO_EINVAL, "partition: bad part");
  return precompute_impl(ctx, p, n_parts, part);
}

int teno_get_stencils(teno_ctx* ctx, int32_t* large, int32_t* small) {
  if (!ctx || !large || !small) return TENO_EINVAL;
  if (!ctx->pre_ok) return fail(ctx, TENO_ESTATE, "no precompute");
  std::copy(ctx->st_large.begin(), ctx->st_large.end(), large);
  std::copy(ctx->st_small.begin(), ctx->st_small.end(), small);
  return TENO_OK;
}

int teno_get_sizes(teno_ctx* ctx, int64_t* n_cell, int32_t* n_var, int32_t* m, int32_t* n_s) {
  if (!ctx) return TENO_EINVAL;
  if (n_cell) *n_cell = ctx->nc;
  if (n_var) *n_var = ctx->prm.n_var;
  if (m) *m = ctx->m;
  if (n_s) *n_s = ctx->ns;
  return TENO_OK;
}

int teno_colour_slots(int32_t n_lanes, int32_t n_slots, const int32_t* members,
                      int32_t* slot_of) {
  const int r = colour_slots(n_lanes, n_slots, members, slot_of);
  return r < 0 ? TENO_EINVAL : r;
}

int teno_set_state(teno_ctx* ctx, const double* U, int on_device) {
  int rc = check_ready(ctx, false);
  if (rc) return rc;
  if (!U) return fail(ctx, TENO_EINVAL, "set_state: null U");
  rc = to_internal(ctx, U, (double*)ctx->b_U.p, on_device);
  if (rc) return rc;
  if (!on_device) CK(cudaStreamSynchronize(ctx->stream), "sync");
  ctx->state_ok = true;
  ctx->split_ok = false;
  ctx->stages_ok = false;
  return TENO_OK;
}

int teno_get_state(teno_ctx* ctx, double* U, int on_device) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (!U) return fail(ctx, TENO_EINVAL, "get_state: null U");
  return to_user(ctx, (const double*)ctx->b_U.p, U, on_device);
}

int teno_set_time(teno_ctx* ctx, double t) {
  if (!ctx) return TENO_EINVAL;
  ctx->time = t;
  return TENO_OK;
}

int teno_residual(teno_ctx* ctx, double* R, uint8_t* sel, int on_device) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (!R) return fail(ctx, TENO_EINVAL, "residual: null R");
  rc = stage_flux(ctx, (const double*)ctx->b_U.p, (uint8_t*)ctx->b_sel.p, ctx->time,
                  ctx->split_ok);
  if (rc) return rc;
  CK(launch_gather(ctx->dm, ctx->b_K.p, nullptr, nullptr, (double*)ctx->b_R.p, 0, 0, 0, 0,
                   nullptr, nullptr, nullptr, ctx->stream),
     "gather launch");
  if (sel) {
    const uint8_t* src = ctx->override_on ? (const uint8_t*)ctx->b_sel_ovr.p
                                          : (const uint8_t*)ctx->b_sel.p;
    if (on_device) {
      CK(launch_permute_u8(src, sel, (const int32_t*)ctx->b_perm.p, ctx->io_n, ctx->spad,
                           ctx->io_n, ctx->prm.n_var, 1, ctx->stream),
         "permute");
    } else {
      rc = dev_alloc(ctx, ctx->b_vtmp, sizeof(double) * ctx->prm.n_var * ctx->spad);
      if (rc) return rc;
      uint8_t* d = (uint8_t*)ctx->b_vtmp.p;
      CK(launch_permute_u8(src, d, (const int32_t*)ctx->b_perm.p, ctx->io_n, ctx->spad,
                           ctx->io_n, ctx->prm.n_var, 1, ctx->stream),
         "permute");
      CK(cudaMemcpyAsync(sel, d, (size_t)ctx->prm.n_var * ctx->io_n, cudaMemcpyDeviceToHost,
                         ctx->stream),
         "D2H");
    }
  }
  return to_user(ctx, (const double*)ctx->b_R.p, R, on_device);
}

int teno_set_selection_override(teno_ctx* ctx, const uint8_t* sel, int on_device) {
  int rc = check_ready(ctx, false);
  if (rc) return rc;
  if (!sel) {
    ctx->override_on = false;
    return TENO_OK;
  }
  const int64_t nc = ctx->nc;
  const int nv = ctx->prm.n_var;
  const uint8_t* s = sel;
  if (!on_device) {
    CK(cudaMemcpyAsync(ctx->b_tmp.p, sel, (size_t)nv * nc, cudaMemcpyHostToDevice, ctx->stream),
       "H2D");
    s = (const uint8_t*)ctx->b_tmp.p;
  }
  const bool part = ctx->part_n > 1;
  CK(launch_permute_u8(s, (uint8_t*)ctx->b_sel_ovr.p,
                       (const int32_t*)(part ? ctx->b_perm_in.p : ctx->b_perm.p),
                       part ? ctx->sn : nc, nc, ctx->spad, nv, 0, ctx->stream),
     "permute");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  ctx->override_on = true;
  return TENO_OK;
}

int teno_cfl_dt(teno_ctx* ctx, double* dt) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (!dt) return fail(ctx, TENO_EINVAL, "cfl_dt: null dt");
  CK(launch_max_lambda(ctx->dm, (const double*)ctx->b_U.p, (double*)ctx->b_maxlam.p, ctx->stream),
     "max lambda launch");
  double lam = 0.0;
  CK(cudaMemcpyAsync(&lam, ctx->b_maxlam.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
     "D2H");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  if (!(lam > 0.0) || !std::isfinite(lam)) return fail(ctx, TENO_ENONPHYS, "cfl_dt: bad speed");
  *dt = ctx->prm.cfl / lam;
  return TENO_OK;
}

static int rk3_once(teno_ctx* ctx, double dt, double* dt_used) {
  const double* maxlam = nullptr;
  if (dt <= 0.0) {
    if (dt_used || ctx->has_time_bc) {
      int rc = teno_cfl_dt(ctx, &dt);
      if (rc) return rc;
    } else {
      long pe = prof_begin(ctx, K_CFL);
      // from the (hi, lo) split of U where the FP64 or mixed path holds it
      if (ctx->split_ok && ctx->prm.n_var == 4 && ctx->prm.precision != TENO_FP64_NATIVE)
        CK(launch_max_lambda_split(ctx->dm, (const float2*)ctx->b_Usplit.p,
                                   (double*)ctx->b_maxlam.p, ctx->stream),
           "max lambda launch");
      else
        CK(launch_max_lambda(ctx->dm, (const double*)ctx->b_U.p, (double*)ctx->b_maxlam.p,
                             ctx->stream),
           "max lambda launch");
      prof_end(ctx, pe);
      maxlam = (const double*)ctx->b_maxlam.p;
    }
  }
  double* U = (double*)ctx->b_U.p;
  double* U1 = (double*)ctx->b_U1.p;
  double* U2 = (double*)ctx->b_U2.p;
  const double t = ctx->time;
  int rc = rk_stage(ctx, U, U, U1, 0.0, 1.0, dt, maxlam, t, ctx->split_ok);
  if (!rc) rc = rk_stage(ctx, U, U1, U2, 0.75, 0.25, dt, maxlam, t + dt, true);
  if (!rc) rc = rk_stage(ctx, U, U2, U, 1.0 / 3.0, 2.0 / 3.0, dt, maxlam, t + 0.5 * dt, true);
  ctx->split_ok = ctx->prm.precision != TENO_FP64_NATIVE;
  if (rc) return rc;
  ctx->stages_ok = true;
  if (dt > 0.0) ctx->time += dt;
  if (dt_used) *dt_used = dt;
  return TENO_OK;
}

int teno_rk3_step(teno_ctx* ctx, double dt, double* dt_used) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (ctx->part_n > 1)
    return fail(ctx, TENO_EINVAL,
                "partition: step with teno_group_rk3_step, or teno_rk3_stage and halo exchanges");
  rc = rk3_once(ctx, dt, dt_used);
  if (rc) return rc;
  if (dt_used) return teno_check_state(ctx);
  return TENO_OK;
}

int teno_get_stage_state(teno_ctx* ctx, int32_t stage, double* U, int on_device) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (!U || (stage != 1 && stage != 2)) return fail(ctx, TENO_EINVAL, "get_stage_state: bad args");
  if (!ctx->stages_ok) return fail(ctx, TENO_ESTATE, "get_stage_state: no RK3 step taken");
  return to_user(ctx, (const double*)(stage == 1 ? ctx->b_U1.p : ctx->b_U2.p), U, on_device);
}

int teno_rk3_steps(teno_ctx* ctx, int32_t n_steps, double dt) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (ctx->part_n > 1)
    return fail(ctx, TENO_EINVAL,
                "partition: step with teno_group_rk3_step, or teno_rk3_stage and halo exchanges");
  if (n_steps < 0) return fail(ctx, TENO_EINVAL, "rk3_steps: negative count");
  for (int32_t i = 0; i < n_steps && !rc; ++i) rc = rk3_once(ctx, dt, nullptr);
  return rc;
}

int teno_check_state(teno_ctx* ctx) {
  if (!ctx) return TENO_EINVAL;
  if (!ctx->pre_ok) return TENO_OK;
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, ctx->b_flag.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
     "D2H");
  CK(cudaMemsetAsync(ctx->b_flag.p, 0, sizeof(int), ctx->stream), "memset");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  if (flag & 2) return fail(ctx, TENO_ETIMEOUT, "a bounded device wait gave up");
  if (flag) return fail(ctx, TENO_ENONPHYS, "non-physical state (rho <= 0, p <= 0 or NaN)");
  return TENO_OK;
}

int teno_residual_vjp(teno_ctx* ctx, const double* w, double* v, int on_device) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (ctx->part_n > 1)
    return fail(ctx, TENO_EINVAL, "partition: the VJP needs the reverse halo exchange "
                                  "(teno_group_residual_vjp)");
  if (!w || !v) return fail(ctx, TENO_EINVAL, "residual_vjp: null pointer");
  if (ctx->prm.precision == TENO_FP32_MIXED)
    return fail(ctx, TENO_EINVAL, "adjoint: FP64 precisions only");
  if (ctx->prm.scheme != 0 || ctx->prm.charvar != 0 || ctx->prm.positivity != 0)
    return fail(ctx, TENO_EINVAL,
                "adjoint: TENO in conservative variables only, without positivity scaling");
  rc = ensure_adjoint(ctx);
  if (rc) return rc;
  rc = to_internal(ctx, w, (double*)ctx->b_l1.p, on_device);
  if (!rc)
    rc = vjp_internal(ctx, (const double*)ctx->b_U.p, (const double*)ctx->b_l1.p,
                      (double*)ctx->b_vtmp.p, ctx->time);
  if (!rc) rc = to_user(ctx, (const double*)ctx->b_vtmp.p, v, on_device);
  return rc;
}

int teno_adjoint_step(teno_ctx* ctx, double dt, const double* lam_np1, double* lam_n,
                      int on_device) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (ctx->part_n > 1)
    return fail(ctx, TENO_EINVAL, "partition: adjoint steps take the whole mesh");
  if (!lam_np1 || !lam_n || !(dt > 0.0)) return fail(ctx, TENO_EINVAL, "adjoint_step: bad args");
  if (ctx->prm.precision == TENO_FP32_MIXED)
    return fail(ctx, TENO_EINVAL, "adjoint: FP64 precisions only");
  if (ctx->prm.scheme != 0 || ctx->prm.charvar != 0 || ctx->prm.positivity != 0)
    return fail(ctx, TENO_EINVAL,
                "adjoint: TENO in conservative variables only, without positivity scaling");
  rc = ensure_adjoint(ctx);
  if (rc) return rc;
  ctx->stages_ok = false;  // the replay below overwrites the stage buffers
  const int64_t n = (int64_t)ctx->prm.n_var * ctx->spad;
  double* U = (double*)ctx->b_U.p;
  double* U1 = (double*)ctx->b_U1.p;
  double* U2 = (double*)ctx->b_U2.p;
  double* lam = (double*)ctx->b_R.p;  // lambda^{n+1}, internal order
  double* l1 = (double*)ctx->b_l1.p;
  double* l2 = (double*)ctx->b_l2.p;
  double* ln = (double*)ctx->b_lamn.p;
  double* tmp = (double*)ctx->b_vtmp.p;
  const double t = ctx->time;
  rc = to_internal(ctx, lam_np1, lam, on_device);
  // forward replay of the stage states; the Gauss-point values and
  // selections of stages 1 and 2 are kept for their VJPs
  void* uq0 = ctx->b_Uq_st[0].p;
  void* uq1 = ctx->b_Uq_st[1].p;
  uint8_t* s0 = (uint8_t*)ctx->b_sel_st[0].p;
  uint8_t* s1 = (uint8_t*)ctx->b_sel_st[1].p;
  if (!rc) rc = rk_stage(ctx, U, U, U1, 0.0, 1.0, dt, nullptr, t, false, uq0, s0);
  if (!rc) rc = rk_stage(ctx, U, U1, U2, 0.75, 0.25, dt, nullptr, t + dt, false, uq1, s1);
  // stage 3: U^{n+1} = 1/3 U^n + 2/3 U2 + 2/3 dt R(U2)
  if (!rc) rc = vjp_internal(ctx, U2, lam, tmp, t + 0.5 * dt);
  if (rc) return rc;
  CK(launch_axpby(l2, lam, 2.0 / 3.0, tmp, 2.0 / 3.0 * dt, n, ctx->stream), "axpby");
  CK(launch_axpby(ln, lam, 1.0 / 3.0, lam, 0.0, n, ctx->stream), "axpby");
  // stage 2: U2 = 3/4 U^n + 1/4 U1 + 1/4 dt R(U1)
  rc = vjp_internal(ctx, U1, l2, tmp, t + dt, uq1, s1);
  if (rc) return rc;
  CK(launch_axpby(l1, l2, 0.25, tmp, 0.25 * dt, n, ctx->stream), "axpby");
  CK(launch_axpby(ln, ln, 1.0, l2, 0.75, n, ctx->stream), "axpby");
  // stage 1: U1 = U^n + dt R(U^n)
  rc = vjp_internal(ctx, U, l1, tmp, t, uq0, s0);
  if (rc) return rc;
  CK(launch_axpby(ln, ln, 1.0, l1, 1.0, n, ctx->stream), "axpby");
  CK(launch_axpby(ln, ln, 1.0, tmp, dt, n, ctx->stream), "axpby");
  return to_user(ctx, ln, lam_n, on_device);
}

int teno_edge_values(teno_ctx* ctx, double* out) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (!out) return fail(ctx, TENO_EINVAL, "edge_values: null pointer");
  const int64_t per = 3 * (int64_t)ctx->nq * ctx->prm.n_var;
  const bool f64 = ctx->prm.precision != TENO_FP32_MIXED;
  std::vector<double> h64;
  std::vector<float> h32;
  if (f64) {
    h64.resize(ctx->spad * per);
    CK(cudaMemcpyAsync(h64.data(), ctx->b_Uq.p, h64.size() * 8, cudaMemcpyDeviceToHost,
                       ctx->stream),
       "D2H");
  } else {
    h32.resize(ctx->spad * per);
    CK(cudaMemcpyAsync(h32.data(), ctx->b_Uq.p, h32.size() * 4, cudaMemcpyDeviceToHost,
                       ctx->stream),
       "D2H");
  }
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  // the FP64 path keeps Gauss-point values as (hi, lo) float pairs
  const bool pairs = ctx->prm.precision == TENO_FP64;
  const float* hp = reinterpret_cast<const float*>(h64.data());
  for (int64_t c = 0; c < ctx->io_n; ++c) {
    const int64_t u = ctx->part_n > 1 ? c : ctx->perm[c];
    for (int64_t i = 0; i < per; ++i) {
      const int64_t k = c * per + i;
      out[u * per + i] = pairs ? (double)hp[2 * k] + (double)hp[2 * k + 1]
                               : (f64 ? h64[k] : (double)h32[k]);
    }
  }
  return TENO_OK;
}

int teno_profile(teno_ctx* ctx, int enable) {
  if (!ctx) return TENO_EINVAL;
  if (ctx->device < 0) return fail(ctx, TENO_ESTATE, "host-only context");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  int rc = prof_drain(ctx);
  if (rc) return rc;
  if (enable) {
    for (int k = 0; k < kProfKinds; ++k) {
      ctx->prof_ms[k] = 0.0;
      ctx->launches[k] = 0;
    }
  }
  ctx->prof_on = enable != 0;
  return TENO_OK;
}

int teno_profile_read(teno_ctx* ctx, double* ms, int64_t* launches) {
  if (!ctx) return TENO_EINVAL;
  if (ctx->device < 0) return fail(ctx, TENO_ESTATE, "host-only context");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  int rc = prof_drain(ctx);
  if (rc) return rc;
  for (int k = 0; k < kProfKinds; ++k) {
    if (ms) ms[k] = ctx->prof_ms[k];
    if (launches) launches[k] = ctx->launches[k];
  }
  return TENO_OK;
}


// ------------------------------------------------------------------ partitions

int teno_partition_sizes(teno_ctx* ctx, int64_t* n_owned, int64_t* n_state,
                         int64_t* recv_counts, int64_t* send_counts) {
  if (!ctx) return TENO_EINVAL;
  if (!ctx->pre_ok) return fail(ctx, TENO_ESTATE, "partition_sizes: no precompute");
  if (n_owned) *n_owned = ctx->n_own;
  if (n_state) *n_state = ctx->sn;
  for (int32_t q = 0; q < ctx->part_n; ++q) {
    const bool part = ctx->part_n > 1;
    if (recv_counts) recv_counts[q] = part ? (int64_t)ctx->recv_loc[q].size() : 0;
    if (send_counts)
      send_counts[q] = part && (size_t)q < ctx->send_loc.size() ? (int64_t)ctx->send_loc[q].size()
                                                                : 0;
  }
  return TENO_OK;
}

int teno_partition_cells(teno_ctx* ctx, int32_t* owned_user) {
  if (!ctx || !owned_user) return TENO_EINVAL;
  if (!ctx->pre_ok) return fail(ctx, TENO_ESTATE, "partition_cells: no precompute");
  const int64_t c0 = ctx->part_n > 1 ? ctx->part_bounds[ctx->part_id] : 0;
  for (int64_t l = 0; l < ctx->n_own; ++l) owned_user[l] = ctx->perm[c0 + l];
  return TENO_OK;
}

int teno_partition_recv_cells(teno_ctx* ctx, int32_t peer, int32_t* user_ids) {
  if (!ctx || !user_ids) return TENO_EINVAL;
  if (!ctx->pre_ok || ctx->part_n < 2) return fail(ctx, TENO_ESTATE, "not a partition");
  if (peer < 0 || peer >= ctx->part_n) return fail(ctx, TENO_EINVAL, "bad peer");
  const std::vector<int32_t>& r = ctx->recv_loc[peer];
  for (size_t i = 0; i < r.size(); ++i) user_ids[i] = ctx->perm[ctx->loc2glob[r[i]]];
  return TENO_OK;
}

int teno_partition_set_send(teno_ctx* ctx, int32_t peer, int64_t n, const int32_t* user_ids) {
  if (!ctx || (n > 0 && !user_ids) || n < 0) return TENO_EINVAL;
  if (!ctx->pre_ok || ctx->part_n < 2) return fail(ctx, TENO_ESTATE, "not a partition");
  if (peer < 0 || peer >= ctx->part_n || peer == ctx->part_id)
    return fail(ctx, TENO_EINVAL, "bad peer");
  const int64_t c0 = ctx->part_bounds[ctx->part_id], c1 = ctx->part_bounds[ctx->part_id + 1];
  std::vector<int32_t> loc((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    const int32_t u = user_ids[i];
    if (u < 0 || u >= ctx->nc) return fail(ctx, TENO_EINVAL, "set_send: user id out of range");
    const int64_t g = ctx->iperm[u];
    if (g < c0 || g >= c1) return fail(ctx, TENO_EINVAL, "set_send: cell not owned here");
    loc[i] = (int32_t)(g - c0);
  }
  if (ctx->send_loc.size() != (size_t)ctx->part_n) ctx->send_loc.assign(ctx->part_n, {});
  ctx->send_loc[peer].swap(loc);
  if (ctx->device >= 0) {
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    int rc = upload(ctx, ctx->b_send_idx[peer], ctx->send_loc[peer].data(),
                    ctx->send_loc[peer].size() * 4);
    if (rc) return rc;
  }
  return TENO_OK;
}

}  // extern "C"

namespace {

double* stage_array(teno_ctx* ctx, int32_t what) {
  return (double*)(what == 0 ? ctx->b_U.p : what == 1 ? ctx->b_U1.p
                                          : what == 2 ? ctx->b_U2.p : ctx->b_vtmp.p);
}

// pack into buf: the owned cells `peer` receives (what 0..2: U^n, U^(1),
// U^(2)), or this partition's adjoint contributions to the halo cells `peer`
// owns (what 3)
int halo_pack(teno_ctx* ctx, int32_t peer, int32_t what, double* buf) {
  const bool rev = what == 3;
  if (!rev && (ctx->send_loc.size() != (size_t)ctx->part_n))
    return fail(ctx, TENO_ESTATE, "halo_pack: send lists not set");
  const std::vector<int32_t>& l = rev ? ctx->recv_loc[peer] : ctx->send_loc[peer];
  const DevBuf& idx = rev ? ctx->b_recv_idx[peer] : ctx->b_send_idx[peer];
  CK(launch_halo_pack(stage_array(ctx, what), ctx->spad, (const int32_t*)idx.p, (int64_t)l.size(),
                      ctx->prm.n_var, buf, ctx->stream),
     "halo pack");
  return TENO_OK;
}

// the inverse: write the received states into the halo (with their FP32
// split on the pair and mixed paths), or add the received contributions to
// the owned cells (what 3)
int halo_unpack(teno_ctx* ctx, int32_t peer, int32_t what, const double* buf) {
  const bool rev = what == 3;
  if (rev && (ctx->send_loc.size() != (size_t)ctx->part_n))
    return fail(ctx, TENO_ESTATE, "halo_unpack: send lists not set");
  const std::vector<int32_t>& l = rev ? ctx->send_loc[peer] : ctx->recv_loc[peer];
  const DevBuf& idx = rev ? ctx->b_send_idx[peer] : ctx->b_recv_idx[peer];
  float2* Us = (!rev && ctx->prm.precision != TENO_FP64_NATIVE) ? (float2*)ctx->b_Usplit.p : nullptr;
  CK(launch_halo_unpack(stage_array(ctx, what), ctx->spad, (const int32_t*)idx.p,
                        (int64_t)l.size(), ctx->prm.n_var, buf, Us, rev ? 1 : 0, ctx->stream),
     "halo unpack");
  return TENO_OK;
}

// stage 1..3 of the SSP-RK3 step (Eq. fv_time_discretization_01) on the
// updated cells; the halo of the stage's input state must be current
int rk3_stage(teno_ctx* ctx, int32_t stage, double dt) {
  double* U = (double*)ctx->b_U.p;
  double* U1 = (double*)ctx->b_U1.p;
  double* U2 = (double*)ctx->b_U2.p;
  const double t = ctx->time;
  int rc = TENO_OK;
  if (stage == 1) {
    rc = rk_stage(ctx, U, U, U1, 0.0, 1.0, dt, nullptr, t, ctx->split_ok);
    ctx->stages_ok = false;
  } else if (stage == 2) {
    rc = rk_stage(ctx, U, U1, U2, 0.75, 0.25, dt, nullptr, t + dt, true);
  } else {
    rc = rk_stage(ctx, U, U2, U, 1.0 / 3.0, 2.0 / 3.0, dt, nullptr, t + 0.5 * dt, true);
    if (!rc) {
      ctx->time += dt;
      ctx->stages_ok = true;
    }
  }
  ctx->split_ok = ctx->prm.precision != TENO_FP64_NATIVE;
  return rc;
}

// largest (|v| + c) / length over the updated cells (host; synchronises)
int local_max_speed(teno_ctx* ctx, double* lam) {
  CK(launch_max_lambda(ctx->dm, (const double*)ctx->b_U.p, (double*)ctx->b_maxlam.p, ctx->stream),
     "max lambda launch");
  CK(cudaMemcpyAsync(lam, ctx->b_maxlam.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
     "D2H");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  return TENO_OK;
}

// checks of a group of partitions driven in one process: parts[i] is part i
// of the same mesh, all on one device and one stream, with their states set
int group_check(teno_ctx* const* parts, int32_t n) {
  if (!parts || n < 1) return TENO_EINVAL;
  for (int32_t i = 0; i < n; ++i) {
    teno_ctx* c = parts[i];
    if (!c) return TENO_EINVAL;
    int rc = check_ready(c, true);
    if (rc) return rc;
    if (c->part_n != n || c->part_id != i || c->device != parts[0]->device ||
        c->stream != parts[0]->stream || c->nc != parts[0]->nc ||
        c->part_bounds != parts[0]->part_bounds || c->prm.n_var != parts[0]->prm.n_var)
      return fail(c, TENO_EINVAL, "group: parts must be parts 0..n-1 of one mesh, on one "
                                  "device and one stream");
  }
  return TENO_OK;
}

// the send lists of every part (the cells each peer receives), and the
// exchange buffers: [q] towards q, [n + q] from q
int group_link(teno_ctx* const* parts, int32_t n) {
  for (int32_t p = 0; p < n; ++p) {
    teno_ctx* cp = parts[p];
    if (cp->send_loc.size() == (size_t)n) continue;
    for (int32_t q = 0; q < n; ++q) {
      if (q == p) continue;
      const teno_ctx* cq = parts[q];
      std::vector<int32_t> users(cq->recv_loc[p].size());
      for (size_t i = 0; i < users.size(); ++i)
        users[i] = cq->perm[cq->loc2glob[cq->recv_loc[p][i]]];
      int rc = teno_partition_set_send(cp, q, (int64_t)users.size(), users.data());
      if (rc) return rc;
    }
  }
  for (int32_t p = 0; p < n; ++p) {
    teno_ctx* cp = parts[p];
    for (int32_t q = 0; q < n; ++q) {
      if (q == p) continue;
      // each buffer serves both directions: the forward exchange sends the
      // cells q receives and receives the cells q owns here; the reverse
      // exchange the other way round
      const size_t nv = cp->prm.n_var;
      const size_t cnt = std::max<size_t>(
          1, std::max(cp->send_loc[q].size(), cp->recv_loc[q].size()));
      int rc = dev_alloc(cp, cp->b_xbuf[q], 8 * nv * cnt);
      if (!rc) rc = dev_alloc(cp, cp->b_xbuf[n + q], 8 * nv * cnt);
      if (rc) return rc;
    }
  }
  return TENO_OK;
}

// forward (what 0..2): every part's halo of that state from its owners;
// reverse (what 3): every part's contributions to other parts' cells added
// there, each owner adding its peers in ascending order.  Pack on the source
// part, one device-to-device copy, unpack on the destination part.
int group_exchange(teno_ctx* const* parts, int32_t n, int32_t what) {
  const bool rev = what == 3;
  for (int32_t dst = 0; dst < n; ++dst) {
    teno_ctx* cd = parts[dst];
    for (int32_t src = 0; src < n; ++src) {
      if (src == dst) continue;
      teno_ctx* cs = parts[src];
      const size_t cnt = rev ? cs->recv_loc[dst].size() : cs->send_loc[dst].size();
      if (cnt == 0) continue;
      const size_t need = 8 * (size_t)cd->prm.n_var * cnt;
      if (cs->b_xbuf[dst].bytes < need || cd->b_xbuf[n + src].bytes < need)
        return fail(cd, TENO_EINVAL, "group exchange: buffer smaller than the list");
      int rc = halo_pack(cs, dst, what, (double*)cs->b_xbuf[dst].p);
      if (rc) return rc;
      teno_ctx* ctx = cd;
      CK(cudaMemcpyAsync(cd->b_xbuf[n + src].p, cs->b_xbuf[dst].p, 8 * cd->prm.n_var * cnt,
                         cudaMemcpyDeviceToDevice, cd->stream),
         "halo copy");
      rc = halo_unpack(cd, src, what, (const double*)cd->b_xbuf[n + src].p);
      if (rc) return rc;
    }
  }
  return TENO_OK;
}

}  // namespace

extern "C" {

int teno_halo_pack(teno_ctx* ctx, int32_t peer, int32_t what, double* buf) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (ctx->part_n < 2 || peer < 0 || peer >= ctx->part_n || peer == ctx->part_id || what < 0 ||
      what > 3 || !buf)
    return fail(ctx, TENO_EINVAL, "halo_pack: bad arguments");
  return halo_pack(ctx, peer, what, buf);
}

int teno_halo_unpack(teno_ctx* ctx, int32_t peer, int32_t what, const double* buf) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (ctx->part_n < 2 || peer < 0 || peer >= ctx->part_n || peer == ctx->part_id || what < 0 ||
      what > 3 || !buf)
    return fail(ctx, TENO_EINVAL, "halo_unpack: bad arguments");
  return halo_unpack(ctx, peer, what, buf);
}

int teno_rk3_stage(teno_ctx* ctx, int32_t stage, double dt) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (stage < 1 || stage > 3 || !(dt > 0.0)) return fail(ctx, TENO_EINVAL, "rk3_stage: bad args");
  return rk3_stage(ctx, stage, dt);
}

int teno_local_max_speed(teno_ctx* ctx, double* lam) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (!lam) return fail(ctx, TENO_EINVAL, "local_max_speed: null pointer");
  return local_max_speed(ctx, lam);
}

int teno_group_rk3_step(teno_ctx* const* parts, int32_t n, double dt, double* dt_used) {
  int rc = group_check(parts, n);
  if (rc) return rc;
  if (n > 1 && (rc = group_link(parts, n))) return rc;
  if (dt <= 0.0) {
    double lam = 0.0;
    for (int32_t i = 0; i < n; ++i) {
      double l = 0.0;
      if ((rc = local_max_speed(parts[i], &l))) return rc;
      lam = std::max(lam, l);
    }
    if (!(lam > 0.0) || !std::isfinite(lam))
      return fail(parts[0], TENO_ENONPHYS, "group step: bad speed");
    dt = parts[0]->prm.cfl / lam;
  }
  for (int32_t stage = 1; stage <= 3; ++stage) {
    for (int32_t i = 0; i < n; ++i)
      if ((rc = rk3_stage(parts[i], stage, dt))) return rc;
    if (n > 1 && (rc = group_exchange(parts, n, stage == 3 ? 0 : stage))) return rc;
  }
  if (dt_used) *dt_used = dt;
  return TENO_OK;
}

int teno_group_residual_vjp(teno_ctx* const* parts, int32_t n, const double* w, double* vout) {
  int rc = group_check(parts, n);
  if (rc) return rc;
  if (!w || !vout) return fail(parts[0], TENO_EINVAL, "group vjp: null pointer");
  if (n > 1 && (rc = group_link(parts, n))) return rc;
  for (int32_t i = 0; i < n; ++i) {
    teno_ctx* ctx = parts[i];
    if (ctx->prm.precision == TENO_FP32_MIXED || ctx->prm.scheme != 0 || ctx->prm.positivity)
      return fail(ctx, TENO_EINVAL, "adjoint: FP64 TENO without positivity scaling only");
    if ((rc = ensure_adjoint(ctx))) return rc;
    if ((rc = to_internal(ctx, w, (double*)ctx->b_l1.p, 0))) return rc;
    // cotangents of the cells this part updates only
    for (int k = 0; k < ctx->prm.n_var; ++k) {
      double* row = (double*)ctx->b_l1.p + (size_t)k * ctx->spad;
      CK(cudaMemsetAsync(row + ctx->n_own, 0, sizeof(double) * (ctx->spad - ctx->n_own),
                         ctx->stream),
         "memset");
    }
    if ((rc = vjp_internal(ctx, (const double*)ctx->b_U.p, (const double*)ctx->b_l1.p,
                           (double*)ctx->b_vtmp.p, ctx->time)))
      return rc;
  }
  if (n > 1 && (rc = group_exchange(parts, n, 3))) return rc;
  const int nv = parts[0]->prm.n_var;
  const int64_t nc = parts[0]->nc;
  std::vector<double> h;
  std::vector<int32_t> users;
  for (int32_t i = 0; i < n; ++i) {
    teno_ctx* ctx = parts[i];
    h.resize((size_t)nv * ctx->n_own);
    users.resize(ctx->n_own);
    if ((rc = to_user(ctx, (const double*)ctx->b_vtmp.p, h.data(), 0))) return rc;
    teno_partition_cells(ctx, users.data());
    for (int k = 0; k < nv; ++k)
      for (int64_t l = 0; l < ctx->n_own; ++l)
        vout[(size_t)k * nc + users[l]] = h[(size_t)k * ctx->n_own + l];
  }
  return TENO_OK;
}

// ------------------------------------------------------------------ adjoint tape

int teno_tape_reserve(teno_ctx* ctx, int32_t n_slots) {
  int rc = check_ready(ctx, false);
  if (rc) return rc;
  if (n_slots < 0) return fail(ctx, TENO_EINVAL, "tape_reserve: negative count");
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t nv = ctx->prm.n_var;
  ctx->tape_sb = al(8 * nv * ctx->spad);
  ctx->tape_qb = al(ctx->b_Uq.bytes);
  ctx->tape_selb = al(nv * ctx->spad);
  const size_t slot = 3 * (ctx->tape_sb + ctx->tape_qb + ctx->tape_selb);
  for (size_t i = (size_t)n_slots; i < ctx->tape.size(); ++i) dev_free(ctx->tape[i]);
  ctx->tape.resize(n_slots);
  for (int32_t i = 0; i < n_slots; ++i) {
    if (ctx->tape[i].bytes != slot) dev_free(ctx->tape[i]);
    if ((rc = dev_alloc(ctx, ctx->tape[i], slot))) return rc;
  }
  ctx->tape_dt.assign(n_slots, 0.0);
  ctx->tape_t.assign(n_slots, 0.0);
  ctx->tape_ok.assign(n_slots, 0);
  return TENO_OK;
}

}  // extern "C"

namespace {
// parts of tape slot i: state k (0 U^n, 1 U^(1), 2 U^(2)); Gauss values and
// selection of stage k (0..2)
unsigned char* tape_part(teno_ctx* ctx, int32_t i, int kind, int k) {
  unsigned char* b = (unsigned char*)ctx->tape[i].p;
  const size_t s = ctx->tape_sb, q = ctx->tape_qb, l = ctx->tape_selb;
  if (kind == 0) return b + k * s;
  if (kind == 1) return b + 3 * s + k * q;
  return b + 3 * s + 3 * q + k * l;
}
}  // namespace

extern "C" {

int teno_rk3_step_record(teno_ctx* ctx, int32_t slot, double dt) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (ctx->part_n > 1) return fail(ctx, TENO_EINVAL, "partition: adjoint steps take the whole mesh");
  if (slot < 0 || slot >= (int32_t)ctx->tape.size())
    return fail(ctx, TENO_EINVAL, "rk3_step_record: slot outside the reserved tape");
  if (dt <= 0.0 && (rc = teno_cfl_dt(ctx, &dt))) return rc;
  double* U = (double*)ctx->b_U.p;
  double* Un = (double*)tape_part(ctx, slot, 0, 0);
  double* U1 = (double*)tape_part(ctx, slot, 0, 1);
  double* U2 = (double*)tape_part(ctx, slot, 0, 2);
  CK(cudaMemcpyAsync(Un, U, 8 * (size_t)ctx->prm.n_var * ctx->spad, cudaMemcpyDeviceToDevice,
                     ctx->stream),
     "tape copy");
  const double t = ctx->time;
  rc = rk_stage(ctx, U, U, U1, 0.0, 1.0, dt, nullptr, t, ctx->split_ok, tape_part(ctx, slot, 1, 0),
                tape_part(ctx, slot, 2, 0));
  if (!rc)
    rc = rk_stage(ctx, U, U1, U2, 0.75, 0.25, dt, nullptr, t + dt, true,
                  tape_part(ctx, slot, 1, 1), tape_part(ctx, slot, 2, 1));
  if (!rc)
    rc = rk_stage(ctx, U, U2, U, 1.0 / 3.0, 2.0 / 3.0, dt, nullptr, t + 0.5 * dt, true,
                  tape_part(ctx, slot, 1, 2), tape_part(ctx, slot, 2, 2));
  ctx->split_ok = ctx->prm.precision != TENO_FP64_NATIVE;
  ctx->stages_ok = false;  // the stage states went to the tape
  if (rc) return rc;
  ctx->tape_dt[slot] = dt;
  ctx->tape_t[slot] = t;
  ctx->tape_ok[slot] = 1;
  ctx->time += dt;
  return TENO_OK;
}

int teno_adjoint_step_tape(teno_ctx* ctx, int32_t slot, const double* lam_np1, double* lam_n,
                           int on_device) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (!lam_np1 || !lam_n || slot < 0 || slot >= (int32_t)ctx->tape.size() || !ctx->tape_ok[slot])
    return fail(ctx, TENO_EINVAL, "adjoint_step_tape: bad arguments or an unrecorded slot");
  if (ctx->prm.precision == TENO_FP32_MIXED)
    return fail(ctx, TENO_EINVAL, "adjoint: FP64 precisions only");
  if (ctx->prm.scheme != 0 || ctx->prm.charvar != 0 || ctx->prm.positivity != 0)
    return fail(ctx, TENO_EINVAL,
                "adjoint: TENO in conservative variables only, without positivity scaling");
  rc = ensure_adjoint(ctx);
  if (rc) return rc;
  const int64_t n = (int64_t)ctx->prm.n_var * ctx->spad;
  const double dt = ctx->tape_dt[slot], t = ctx->tape_t[slot];
  double* lam = (double*)ctx->b_R.p;
  double* l1 = (double*)ctx->b_l1.p;
  double* l2 = (double*)ctx->b_l2.p;
  double* ln = (double*)ctx->b_lamn.p;
  double* tmp = (double*)ctx->b_vtmp.p;
  const double* Un = (const double*)tape_part(ctx, slot, 0, 0);
  const double* U1 = (const double*)tape_part(ctx, slot, 0, 1);
  const double* U2 = (const double*)tape_part(ctx, slot, 0, 2);
  auto uq = [&](int k) { return (const void*)tape_part(ctx, slot, 1, k); };
  auto sl = [&](int k) { return (const uint8_t*)tape_part(ctx, slot, 2, k); };
  rc = to_internal(ctx, lam_np1, lam, on_device);
  // stage 3: U^{n+1} = 1/3 U^n + 2/3 U2 + 2/3 dt R(U2)
  if (!rc) rc = vjp_internal(ctx, U2, lam, tmp, t + 0.5 * dt, uq(2), sl(2));
  if (rc) return rc;
  CK(launch_axpby(l2, lam, 2.0 / 3.0, tmp, 2.0 / 3.0 * dt, n, ctx->stream), "axpby");
  CK(launch_axpby(ln, lam, 1.0 / 3.0, lam, 0.0, n, ctx->stream), "axpby");
  // stage 2: U2 = 3/4 U^n + 1/4 U1 + 1/4 dt R(U1)
  rc = vjp_internal(ctx, U1, l2, tmp, t + dt, uq(1), sl(1));
  if (rc) return rc;
  CK(launch_axpby(l1, l2, 0.25, tmp, 0.25 * dt, n, ctx->stream), "axpby");
  CK(launch_axpby(ln, ln, 1.0, l2, 0.75, n, ctx->stream), "axpby");
  // stage 1: U1 = U^n + dt R(U^n)
  rc = vjp_internal(ctx, Un, l1, tmp, t, uq(0), sl(0));
  if (rc) return rc;
  CK(launch_axpby(ln, ln, 1.0, l1, 1.0, n, ctx->stream), "axpby");
  CK(launch_axpby(ln, ln, 1.0, tmp, dt, n, ctx->stream), "axpby");
  return to_user(ctx, ln, lam_n, on_device);
}
}  // extern "C"
