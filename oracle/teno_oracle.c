/*
 * teno_oracle.c -- plain, slow FP64 CPU oracle for the unstructured-mesh TENO
 * finite-volume residual (Ji, Liang & Fu, "A class of new high-order
 * finite-volume TENO schemes for hyperbolic conservation laws with
 * unstructured meshes").
 *
 * TEST INFRASTRUCTURE.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  The product
 * path (the CUDA library) never calls it, and this file shares no code with
 * it.  Every step follows the paper in its order and notation, with a plain
 * loop per step and no blocking, fusion or reordering:
 *
 *   Sec. 2.2, Eq. (reconstruction_02): affine map of the target triangle
 *       onto the reference triangle (v0->(0,0), v1->(1,0), v2->(0,1));
 *   Sec. 3.1: one large central stencil and K = 3 directional stencils
 *       (readings of the cited NCB / Type3 algorithms, stated below);
 *   Eq. (reconstruction_03..08): zero-mean monomial basis psi_l, matrix
 *       A_sl = int_{V'_s} psi_l and right-hand side b_s = |V'_s|(U_s-U_0),
 *       integrals by collapsed Gauss-Legendre quadrature (exact);
 *   Eq. (reconstruction_09/10): a = (R^T R)^{-1} A^T b with R from a
 *       Householder QR of A;
 *   Eq. (WENO_smoothness): beta_k = sum_{q=1..r} int_{V'_0} sum_{|alpha|=q}
 *       (d^alpha P_k)^2 over the reference target triangle;
 *   Eqs. (new_scale_separation, normalize, cutoff, TENO_reconstruction111/222,
 *       TENO_weight): gamma, chi, delta and the two-step selection;
 *   Eq. (fv_governing_equation_semi_discrete): Gauss-point evaluation on the
 *       faces, rotated flux F^n = T^-1 F^x(T U) (Sec. 4.1) with HLL and the
 *       Einfeldt wave speeds (Sec. 4.2, Eq. wavespeed), HLLC (cited in Sec. 5)
 *       or upwind for scalar advection by a constant velocity or by the rigid
 *       rotation of the solid-body case (Sec. 5); residual gather;
 *   Eq. (fv_time_discretization_01): SSP-RK3.
 * The CWENO reconstruction of Sec. 2.3 (Eqs. CWENO_reconstruction,
 * CWENOweight, CWENOOptimalLinearweight/02) on the same stencils is the
 * comparison scheme (scheme = 1).
 * The discrete adjoint (vector-Jacobian product) of a residual and of an
 * SSP-RK3 step, with the selection and the flux branches frozen at the
 * forward state, has no counterpart in the paper; flux Jacobians come from
 * forward-mode dual numbers.
 *
 * Readings where the paper is silent or garbled: m = N_k - 1 unknowns and N_s = 2 N_k neighbours excluding
 * the target; basis order per degree d: xi^d, eta^d, xi^(d-1) eta, ...,
 * xi eta^(d-1); D^q P sums every multi-index |alpha| = q once; N_q = 2 (third,
 * fourth order) or 3 (fifth, sixth order) Gauss-Legendre points per edge with
 * weights summing to one; chi_k = C_T counts as smooth; selection per cell and
 * per conservative variable; CFL length = 4|V|/perimeter; a cell with a face
 * on an outflow boundary enters every face flux with its cell average (first
 * order in that cell layer; at the outflow face both states are that average,
 * zero gradient of the cell averages): its high-order polynomial, from
 * one-sided stencils, makes a boundary closure with a growing mode.
 *
 * Stencil readings (exact, so both implementations agree index for index):
 *   centroid c = ((v0 + v1) + v2) / 3 of the unwrapped vertices; the offset
 *   of cell s from target t is dx = c_s - c_t, reduced on periodic axes by
 *   L * round(dx / L); distance key d2 = dx*dx + dy*dy (no fused multiply-add),
 *   ties broken by the smaller user cell id.  Vertex-neighbour layers: layer
 *   k+1 holds the cells that share a vertex with layer k and are in no earlier
 *   layer (layer 0 = target).
 *   Large stencil: whole layers while the running count stays <= N_s, then the
 *   nearest cells of the next layer up to N_s.
 *   Directional stencil j (edge v_j -> v_{j+1}): with ea = v_j - c_t,
 *   eb = v_{j+1} - c_t, D = ea x eb, alpha = (d x eb)/D, beta = (ea x d)/D,
 *   cell s is admitted when alpha >= -1e-10 and beta >= -1e-10; layers are
 *   added until at least 12 cells are admitted, then the 12 nearest are kept.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define MAXR 5
#define MAXM 20
#define MAXNS 42
#define MAXNQ 4
#define NSM 12 /* directional stencil size, 2 N_k for r = 2 */
#define MSM 5  /* unknowns of a third-order polynomial */
#define KSM 3  /* number of directional stencils on a triangle */
#define MAXLAYERS 16
#define MAXVAR 4
#define ST_TOTAL (MAXNS + KSM * NSM)

enum { FLUX_UPWIND = 0, FLUX_HLL = 1, FLUX_HLLC = 2 };
enum { BC_WALL = 1, BC_INFLOW = 2, BC_OUTFLOW = 3, BC_TOP = 4 };
enum { E_OK = 0, E_INVAL = -1, E_MEM = -2, E_MESH = -4, E_STENCIL = -5 };

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre nodes on [-1,1] by Newton iteration on the three-term
 * Legendre recurrence (n <= 16). */
static void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    x[i] = -z; /* ascending */
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* Collapsed (Duffy) Gauss-Legendre rule on the unit triangle u,v >= 0,
 * u + v <= 1: n*n points; weights sum to 1/2. */
typedef struct {
  int n;
  double u[256], v[256], w[256];
} trirule;

static void make_trirule(int n, trirule* R) {
  double x[16], w[16];
  gauss_legendre(n, x, w);
  R->n = n * n;
  int k = 0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double a = 0.5 * (x[i] + 1.0), b = 0.5 * (x[j] + 1.0);
      R->u[k] = a;
      R->v[k] = b * (1.0 - a);
      R->w[k] = 0.25 * w[i] * w[j] * (1.0 - a);
      ++k;
    }
}

/* ------------------------------------------------------------------------ */
/* basis exponents: degree d = 1..r, order xi^d, eta^d, xi^(d-1)eta, ... */
static int basis_exponents(int r, int ex[][2]) {
  int n = 0;
  for (int d = 1; d <= r; ++d) {
    ex[n][0] = d; ex[n][1] = 0; ++n;
    ex[n][0] = 0; ex[n][1] = d; ++n;
    for (int i = d - 1; i >= 1; --i) { ex[n][0] = i; ex[n][1] = d - i; ++n; }
  }
  return n;
}

static double ipow(double x, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

/* d^(i,j) of xi^a eta^b at (xi, eta) */
static double dmono(int a, int b, int i, int j, double xi, double eta) {
  if (i > a || j > b) return 0.0;
  double c = 1.0;
  for (int k = 0; k < i; ++k) c *= (double)(a - k);
  for (int k = 0; k < j; ++k) c *= (double)(b - k);
  return c * ipow(xi, a - i) * ipow(eta, b - j);
}

/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t nv, nc;
  const double* xy;
  const int32_t* tri;
  int periodic;
  double L[2];
  int order, r, m, ns, nq, nvar, flux, linear;
  double ct, eps, gam, adv[2], time;
  int scheme;     /* 0 TENO, 1 CWENO (the comparison scheme of Sec. 2.3) */
  int charvar;    /* Euler: reconstruct characteristic variables per face */
  int pp;         /* Euler: positivity scaling of the reconstruction (not in the paper) */
  double cw_dk;   /* CWENO d'_K (d_K = 1 - 1/d'_K) */
  int field;      /* scalar advection velocity: 0 constant adv, 1 rigid rotation */
  double rot[5];  /* rotation centre (x, y), angular velocity omega, taper radii r1 < r2 */
  /* geometry (user cell order) */
  double* P;    /* [nc][3][2] unwrapped vertices */
  double* cen;  /* [nc][2] */
  double* area; /* [nc] */
  double* perim;
  /* topology */
  int32_t* v2c_off;
  int32_t* v2c;
  int32_t* fnbr;  /* [nc][3] */
  int32_t* fedge; /* [nc][3] */
  int32_t* fbc;   /* [nc][3] */
  unsigned char* fo; /* [nc] 1: the cell has a face on an outflow boundary */
  /* stencils and reconstruction matrices, built on demand */
  unsigned char* built;
  int32_t* st;   /* [nc][ST_TOTAL] (-1 padding) */
  int32_t* nsm;  /* [nc][KSM] size of directional stencil (12, or 0 if absent) */
  double** ahat; /* per cell: large m*ns, then KSM*(MSM*NSM) */
  double** vol;  /* per cell: |V'_s| for the ST_TOTAL entries */
  /* reference-triangle data */
  int ex[MAXM][2];
  double mean0[MAXM];
  double Br[MAXM * MAXM];
  double B2[MSM * MSM];
  double gt[MAXNQ], gw[MAXNQ];
  trirule qa; /* for A_sl */
  int err;
} omesh;

static void wrap(const omesh* M, double* d) {
  if (!M->periodic) return;
  for (int a = 0; a < 2; ++a) d[a] -= M->L[a] * round(d[a] / M->L[a]);
}

/* offset c_s - c_t with periodic reduction (the stencil distance reading) */
static void cen_offset(const omesh* M, int64_t t, int64_t s, double* d) {
  d[0] = M->cen[2 * s] - M->cen[2 * t];
  d[1] = M->cen[2 * s + 1] - M->cen[2 * t + 1];
  wrap(M, d);
}

static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

/* ------------------------------------------------------------------------ */
static int setup_reference(omesh* M) {
  int n = basis_exponents(M->r, M->ex);
  if (n != M->m) return E_INVAL;
  /* means over the reference triangle V'_0 (area 1/2), Eq. reconstruction_06 */
  trirule Q;
  make_trirule(M->r + 2, &Q);
  for (int l = 0; l < M->m; ++l) {
    double s = 0.0;
    for (int q = 0; q < Q.n; ++q) s += Q.w[q] * ipow(Q.u[q], M->ex[l][0]) * ipow(Q.v[q], M->ex[l][1]);
    M->mean0[l] = s / 0.5;
  }
  /* beta quadratic forms, Eq. WENO_smoothness: B_lk = sum_{q=1..r} sum_{|alpha|=q}
   * int_{V'_0} d^alpha phi_l d^alpha phi_k  (r of the large stencil, and r = 2) */
  for (int pass = 0; pass < 2; ++pass) {
    int rr = pass == 0 ? M->r : 2;
    int mm = pass == 0 ? M->m : MSM;
    double* B = pass == 0 ? M->Br : M->B2;
    trirule QB;
    make_trirule(rr + 1, &QB);
    for (int l = 0; l < mm; ++l)
      for (int k = 0; k < mm; ++k) {
        double s = 0.0;
        for (int q = 1; q <= rr; ++q)
          for (int i = 0; i <= q; ++i) {
            int j = q - i;
            for (int g = 0; g < QB.n; ++g)
              s += QB.w[g] * dmono(M->ex[l][0], M->ex[l][1], i, j, QB.u[g], QB.v[g]) *
                   dmono(M->ex[k][0], M->ex[k][1], i, j, QB.u[g], QB.v[g]);
          }
        B[l * mm + k] = s;
      }
  }
  double x[MAXNQ], w[MAXNQ];
  gauss_legendre(M->nq, x, w);
  for (int k = 0; k < M->nq; ++k) {
    M->gt[k] = 0.5 * (x[k] + 1.0);
    M->gw[k] = 0.5 * w[k];
  }
  make_trirule(M->r / 2 + 2, &M->qa);
  return E_OK;
}

static int build_topology(omesh* M, int64_t nbf, const int32_t* bface) {
  int64_t nc = M->nc, nv = M->nv;
  M->P = (double*)malloc(sizeof(double) * nc * 6);
  M->cen = (double*)malloc(sizeof(double) * nc * 2);
  M->area = (double*)malloc(sizeof(double) * nc);
  M->perim = (double*)malloc(sizeof(double) * nc);
  for (int64_t c = 0; c < nc; ++c) {
    double* P = M->P + 6 * c;
    for (int k = 0; k < 3; ++k) {
      int32_t v = M->tri[3 * c + k];
      if (v < 0 || v >= nv) return E_MESH;
      P[2 * k] = M->xy[2 * v];
      P[2 * k + 1] = M->xy[2 * v + 1];
    }
    if (M->periodic)
      for (int k = 1; k < 3; ++k)
        for (int a = 0; a < 2; ++a) {
          double d = P[2 * k + a] - P[a];
          P[2 * k + a] -= M->L[a] * round(d / M->L[a]);
        }
    M->cen[2 * c] = ((P[0] + P[2]) + P[4]) / 3.0;
    M->cen[2 * c + 1] = ((P[1] + P[3]) + P[5]) / 3.0;
    double ar = 0.5 * ((P[2] - P[0]) * (P[5] - P[1]) - (P[4] - P[0]) * (P[3] - P[1]));
    if (!(ar > 0.0)) return E_MESH;
    M->area[c] = ar;
    double pe = 0.0;
    for (int k = 0; k < 3; ++k) {
      int k1 = (k + 1) % 3;
      pe += hypot(P[2 * k1] - P[2 * k], P[2 * k1 + 1] - P[2 * k + 1]);
    }
    M->perim[c] = pe;
  }
  /* vertex -> cell lists */
  M->v2c_off = (int32_t*)calloc(nv + 1, sizeof(int32_t));
  M->v2c = (int32_t*)malloc(sizeof(int32_t) * 3 * nc);
  for (int64_t c = 0; c < nc; ++c)
    for (int k = 0; k < 3; ++k) M->v2c_off[M->tri[3 * c + k] + 1]++;
  for (int64_t v = 0; v < nv; ++v) M->v2c_off[v + 1] += M->v2c_off[v];
  int32_t* fill = (int32_t*)calloc(nv, sizeof(int32_t));
  for (int64_t c = 0; c < nc; ++c)
    for (int k = 0; k < 3; ++k) {
      int32_t v = M->tri[3 * c + k];
      M->v2c[M->v2c_off[v] + fill[v]++] = (int32_t)c;
    }
  free(fill);
  /* face neighbours: sort (edge key, cell*3+edge) */
  int64_t ne = 3 * nc;
  int64_t* rec = (int64_t*)malloc(sizeof(int64_t) * 2 * ne);
  for (int64_t c = 0; c < nc; ++c)
    for (int k = 0; k < 3; ++k) {
      int64_t a = M->tri[3 * c + k], b = M->tri[3 * c + (k + 1) % 3];
      int64_t lo = a < b ? a : b, hi = a < b ? b : a;
      rec[2 * (3 * c + k)] = lo * nv + hi;
      rec[2 * (3 * c + k) + 1] = 3 * c + k;
    }
  qsort(rec, ne, 2 * sizeof(int64_t), cmp_i64);
  M->fnbr = (int32_t*)malloc(sizeof(int32_t) * ne);
  M->fedge = (int32_t*)malloc(sizeof(int32_t) * ne);
  M->fbc = (int32_t*)calloc(ne, sizeof(int32_t));
  int64_t i = 0;
  int rc = E_OK;
  while (i < ne) {
    int64_t j = i;
    while (j < ne && rec[2 * j] == rec[2 * i]) ++j;
    if (j - i == 2) {
      int64_t x = rec[2 * i + 1], y = rec[2 * i + 3];
      M->fnbr[x] = (int32_t)(y / 3);
      M->fedge[x] = (int32_t)(y % 3);
      M->fnbr[y] = (int32_t)(x / 3);
      M->fedge[y] = (int32_t)(x % 3);
    } else if (j - i == 1) {
      int64_t x = rec[2 * i + 1];
      M->fnbr[x] = -1;
      M->fedge[x] = -1;
      int found = 0;
      for (int64_t b = 0; b < nbf; ++b) {
        int64_t a0 = bface[3 * b], a1 = bface[3 * b + 1];
        int64_t lo = a0 < a1 ? a0 : a1, hi = a0 < a1 ? a1 : a0;
        if (lo * nv + hi == rec[2 * i]) {
          M->fbc[x] = bface[3 * b + 2];
          found = 1;
          break;
        }
      }
      if (!found) rc = E_MESH;
    } else {
      rc = E_MESH;
    }
    i = j;
  }
  free(rec);
  M->fo = (unsigned char*)calloc(nc, 1);
  for (int64_t c = 0; c < nc; ++c)
    for (int k = 0; k < 3; ++k)
      if (M->fnbr[3 * c + k] < 0 && M->fbc[3 * c + k] == BC_OUTFLOW) M->fo[c] = 1;
  return rc;
}

/* ------------------------------------------------------------------------ */
/* stencil search (readings in the file header) */
typedef struct {
  int64_t id;
  double d2;
} cand;

static int cmp_cand(const void* a, const void* b) {
  const cand* x = (const cand*)a;
  const cand* y = (const cand*)b;
  if (x->d2 < y->d2) return -1;
  if (x->d2 > y->d2) return 1;
  return (x->id > y->id) - (x->id < y->id);
}

typedef struct {
  int64_t cells[4096]; /* visited cells, layer by layer; cells[0] = target */
  int start[MAXLAYERS + 2]; /* layer k occupies [start[k], start[k+1]) */
  int nlayers;              /* layers built so far (excluding layer 0) */
  int exhausted;
} layers_t;

static void layers_init(layers_t* Ly, int64_t t, int32_t* seen, int32_t stamp) {
  Ly->cells[0] = t;
  seen[t] = stamp;
  Ly->start[0] = 0;
  Ly->start[1] = 1;
  Ly->nlayers = 0;
  Ly->exhausted = 0;
}

/* add vertex-neighbour layer nlayers+1; returns 0 if nothing new was found */
static int layers_expand(const omesh* M, layers_t* Ly, int32_t* seen, int32_t stamp) {
  if (Ly->exhausted || Ly->nlayers >= MAXLAYERS) return 0;
  int k = Ly->nlayers + 1;
  int b = Ly->start[k - 1], e = Ly->start[k];
  int n = e;
  for (int i = b; i < e; ++i) {
    int64_t c = Ly->cells[i];
    for (int q = 0; q < 3; ++q) {
      int32_t v = M->tri[3 * c + q];
      for (int p = M->v2c_off[v]; p < M->v2c_off[v + 1]; ++p) {
        int32_t x = M->v2c[p];
        if (seen[x] != stamp && n < 4096) {
          seen[x] = stamp;
          Ly->cells[n++] = x;
        }
      }
    }
  }
  if (n == e) {
    Ly->exhausted = 1;
    return 0;
  }
  Ly->start[k + 1] = n;
  Ly->nlayers = k;
  return 1;
}

static int in_sector(const omesh* M, int64_t t, int j, const double* d) {
  const double* P = M->P + 6 * t;
  int j1 = (j + 1) % 3;
  double ea[2] = {P[2 * j] - M->cen[2 * t], P[2 * j + 1] - M->cen[2 * t + 1]};
  double eb[2] = {P[2 * j1] - M->cen[2 * t], P[2 * j1 + 1] - M->cen[2 * t + 1]};
  double D = ea[0] * eb[1] - ea[1] * eb[0];
  double al = (d[0] * eb[1] - d[1] * eb[0]) / D;
  double be = (ea[0] * d[1] - ea[1] * d[0]) / D;
  return al >= -1e-10 && be >= -1e-10;
}

static int find_stencils(const omesh* M, int64_t t, int32_t* out, int32_t* nsm, int32_t* seen,
                         int32_t stamp) {
  static __thread layers_t Ly;
  static __thread cand cs[4096];
  layers_init(&Ly, t, seen, stamp);
  /* large stencil: whole layers while the count stays <= N_s, then the
   * nearest cells of the next layer */
  int cnt = 0, ok = 0;
  for (int k = 1; !ok; ++k) {
    if (k > Ly.nlayers && !layers_expand(M, &Ly, seen, stamp)) break;
    int b = Ly.start[k], e = Ly.start[k + 1];
    int sz = e - b;
    if (cnt + sz <= M->ns) {
      for (int i = b; i < e; ++i) out[cnt++] = (int32_t)Ly.cells[i];
      if (cnt == M->ns) ok = 1;
    } else {
      for (int i = b; i < e; ++i) {
        double d[2];
        cen_offset(M, t, Ly.cells[i], d);
        cs[i - b].id = Ly.cells[i];
        cs[i - b].d2 = d[0] * d[0] + d[1] * d[1];
      }
      qsort(cs, sz, sizeof(cand), cmp_cand);
      for (int i = 0; cnt < M->ns; ++i) out[cnt++] = (int32_t)cs[i].id;
      ok = 1;
    }
  }
  if (!ok) return E_STENCIL;
  /* directional stencils: sector cells of layers 1..k, k growing until at
   * least NSM are admitted; keep the NSM nearest */
  for (int j = 0; j < KSM; ++j) {
    int32_t* o = out + MAXNS + j * NSM;
    int na = 0, filled = 0;
    for (int k = 1; !filled; ++k) {
      if (k > Ly.nlayers && !layers_expand(M, &Ly, seen, stamp)) break;
      for (int i = Ly.start[k]; i < Ly.start[k + 1]; ++i) {
        double d[2];
        cen_offset(M, t, Ly.cells[i], d);
        if (in_sector(M, t, j, d)) {
          cs[na].id = Ly.cells[i];
          cs[na].d2 = d[0] * d[0] + d[1] * d[1];
          ++na;
        }
      }
      if (na >= NSM) filled = 1;
    }
    if (!filled) {
      nsm[j] = 0;
      for (int i = 0; i < NSM; ++i) o[i] = -1;
      continue;
    }
    qsort(cs, na, sizeof(cand), cmp_cand);
    for (int i = 0; i < NSM; ++i) o[i] = (int32_t)cs[i].id;
    nsm[j] = NSM;
  }
  return E_OK;
}

/* ------------------------------------------------------------------------ */
/* reference map of target t: xi = J^{-1} (x - v0) */
static void ref_map(const omesh* M, int64_t t, double* Ji, double* x0) {
  const double* P = M->P + 6 * t;
  double a = P[2] - P[0], b = P[4] - P[0], c = P[3] - P[1], d = P[5] - P[1];
  double det = a * d - b * c;
  Ji[0] = d / det;
  Ji[1] = -b / det;
  Ji[2] = -c / det;
  Ji[3] = a / det;
  x0[0] = P[0];
  x0[1] = P[1];
}

static void to_ref(const double* Ji, const double* x0, double x, double y, double* xi) {
  double dx = x - x0[0], dy = y - x0[1];
  xi[0] = Ji[0] * dx + Ji[1] * dy;
  xi[1] = Ji[2] * dx + Ji[3] * dy;
}

/* vertices of cell s in the frame of target t (nearest periodic image) */
static void cell_in_frame(const omesh* M, int64_t t, int64_t s, double* V) {
  double d[2];
  cen_offset(M, t, s, d);
  double sh0 = (M->cen[2 * t] + d[0]) - M->cen[2 * s];
  double sh1 = (M->cen[2 * t + 1] + d[1]) - M->cen[2 * s + 1];
  if (M->periodic) {
    sh0 = M->L[0] * round(sh0 / M->L[0]);
    sh1 = M->L[1] * round(sh1 / M->L[1]);
  } else {
    sh0 = sh1 = 0.0;
  }
  for (int k = 0; k < 3; ++k) {
    V[2 * k] = M->P[6 * s + 2 * k] + sh0;
    V[2 * k + 1] = M->P[6 * s + 2 * k + 1] + sh1;
  }
}

/* Householder QR of A (rows x cols, row-major) -> R (cols x cols upper) */
static int householder_r(int rows, int cols, const double* A, double* R) {
  double W[MAXNS * MAXM];
  memcpy(W, A, sizeof(double) * rows * cols);
  for (int k = 0; k < cols; ++k) {
    double nrm = 0.0;
    for (int i = k; i < rows; ++i) nrm += W[i * cols + k] * W[i * cols + k];
    nrm = sqrt(nrm);
    if (nrm == 0.0) return E_STENCIL;
    double alpha = W[k * cols + k] > 0 ? -nrm : nrm;
    double v[MAXNS];
    for (int i = 0; i < rows; ++i) v[i] = 0.0;
    for (int i = k; i < rows; ++i) v[i] = W[i * cols + k];
    v[k] -= alpha;
    double vn = 0.0;
    for (int i = k; i < rows; ++i) vn += v[i] * v[i];
    if (vn == 0.0) continue;
    for (int j = k; j < cols; ++j) {
      double s = 0.0;
      for (int i = k; i < rows; ++i) s += v[i] * W[i * cols + j];
      s = 2.0 * s / vn;
      for (int i = k; i < rows; ++i) W[i * cols + j] -= s * v[i];
    }
  }
  double dmax = 0.0, dmin = 1e300;
  for (int i = 0; i < cols; ++i) {
    for (int j = 0; j < cols; ++j) R[i * cols + j] = j >= i ? W[i * cols + j] : 0.0;
    double di = fabs(R[i * cols + i]);
    if (di > dmax) dmax = di;
    if (di < dmin) dmin = di;
  }
  if (!(dmin > 1e-12 * dmax)) return E_STENCIL;
  return E_OK;
}

/* A_sl = int_{V'_s} psi_l and |V'_s| for the given stencil cells in the
 * reference frame of target t (Eq. reconstruction_08) */
static void build_A(const omesh* M, int64_t t, int n, const int32_t* ids, int mm, double* A,
                    double* vol) {
  double Ji[4], x0[2];
  ref_map(M, t, Ji, x0);
  for (int s = 0; s < n; ++s) {
    double V[6], q[6];
    cell_in_frame(M, t, ids[s], V);
    for (int k = 0; k < 3; ++k) to_ref(Ji, x0, V[2 * k], V[2 * k + 1], q + 2 * k);
    double e1x = q[2] - q[0], e1y = q[3] - q[1], e2x = q[4] - q[0], e2y = q[5] - q[1];
    double jac = fabs(e1x * e2y - e2x * e1y);
    vol[s] = 0.5 * jac;
    for (int l = 0; l < mm; ++l) {
      double sum = 0.0;
      for (int g = 0; g < M->qa.n; ++g) {
        double xi = q[0] + M->qa.u[g] * e1x + M->qa.v[g] * e2x;
        double eta = q[1] + M->qa.u[g] * e1y + M->qa.v[g] * e2y;
        sum += M->qa.w[g] * ipow(xi, M->ex[l][0]) * ipow(eta, M->ex[l][1]);
      }
      A[s * mm + l] = jac * sum - vol[s] * M->mean0[l];
    }
  }
}

/* Ahat = (R^T R)^{-1} A^T  (Eq. reconstruction_10), A is n x mm */
static int pseudo_inverse(int n, int mm, const double* A, double* Ahat) {
  double R[MAXM * MAXM];
  int rc = householder_r(n, mm, A, R);
  if (rc) return rc;
  for (int s = 0; s < n; ++s) {
    double y[MAXM], z[MAXM];
    for (int i = 0; i < mm; ++i) { /* R^T y = A[s,:]^T */
      double v = A[s * mm + i];
      for (int k = 0; k < i; ++k) v -= R[k * mm + i] * y[k];
      y[i] = v / R[i * mm + i];
    }
    for (int i = mm - 1; i >= 0; --i) { /* R z = y */
      double v = y[i];
      for (int k = i + 1; k < mm; ++k) v -= R[i * mm + k] * z[k];
      z[i] = v / R[i * mm + i];
    }
    for (int i = 0; i < mm; ++i) Ahat[i * n + s] = z[i];
  }
  return E_OK;
}

static int ensure_cell(omesh* M, int64_t t, int32_t* seen, int32_t stamp) {
  if (M->built[t]) return M->built[t] == 1 ? E_OK : E_STENCIL;
  int32_t* st = M->st + (int64_t)ST_TOTAL * t;
  int32_t* nsm = M->nsm + (int64_t)KSM * t;
  for (int i = 0; i < ST_TOTAL; ++i) st[i] = -1;
  int rc = find_stencils(M, t, st, nsm, seen, stamp);
  if (rc) {
    M->built[t] = 2;
    return rc;
  }
  double* ah = (double*)malloc(sizeof(double) * (M->m * M->ns + KSM * MSM * NSM));
  double* vo = (double*)malloc(sizeof(double) * ST_TOTAL);
  double A[MAXNS * MAXM];
  build_A(M, t, M->ns, st, M->m, A, vo);
  rc = pseudo_inverse(M->ns, M->m, A, ah);
  for (int j = 0; j < KSM && !rc; ++j) {
    if (nsm[j] == 0) continue;
    build_A(M, t, NSM, st + MAXNS + j * NSM, MSM, A, vo + MAXNS + j * NSM);
    rc = pseudo_inverse(NSM, MSM, A, ah + M->m * M->ns + j * MSM * NSM);
  }
  if (rc) {
    free(ah);
    free(vo);
    M->built[t] = 2;
    return rc;
  }
  M->ahat[t] = ah;
  M->vol[t] = vo;
  M->built[t] = 1;
  return E_OK;
}

/* ------------------------------------------------------------------------ */
/* reconstruction of cell t: final coefficients c[var][m] (Eq. reconstruction_04
 * with the TENO selection), selection byte and cutoff margin per variable */
typedef struct {
  double coef[MAXVAR][MAXM];
  unsigned char sel[MAXVAR];
  double margin[MAXVAR];
  double beta[MAXVAR][KSM + 1];
  double a_large[MAXVAR][MAXM];
  double a_small[MAXVAR][KSM][MSM];
  double w[MAXVAR][KSM]; /* weights of the small polynomials (0 if large) */
  /* characteristic-variable reconstruction: conservative-equivalent final
   * coefficients per local edge (charf = 1), used instead of coef */
  int charf;
  double coef_f[3][MAXVAR][MAXM];
} recon_t;

static double quad_form(int n, const double* B, const double* a) {
  double s = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) s += a[i] * B[i * n + j] * a[j];
  return s;
}

/* TENO selection (Eqs. new_scale_separation, normalize, cutoff,
 * TENO_reconstruction111/222) of one field from its large and directional
 * coefficients; returns the final coefficients, the selection byte and the
 * smallest |chi - C_T| */
static unsigned char teno_field(const omesh* M, const int32_t* nsm, const double* a,
                                double as[KSM][MSM], double* c, double* margin) {
  double beta[KSM + 1];
  for (int j = 0; j < KSM; ++j) beta[j] = quad_form(MSM, M->B2, as[j]);
  beta[KSM] = quad_form(M->m, M->Br, a);
  double gam[KSM + 1], sum = 0.0;
  for (int k = 0; k <= KSM; ++k) {
    int present = k == KSM || nsm[k];
    gam[k] = present ? 1.0 / pow(beta[k] + M->eps, 6.0) : 0.0;
    sum += gam[k];
  }
  *margin = 1e300;
  if (M->linear) {
    for (int l = 0; l < M->m; ++l) c[l] = a[l];
    return 8;
  }
  for (int k = 0; k <= KSM; ++k) {
    int present = k == KSM || nsm[k];
    double d = fabs(gam[k] / sum - M->ct);
    if (present && d < *margin) *margin = d;
  }
  if (!(gam[KSM] / sum < M->ct)) {
    for (int l = 0; l < M->m; ++l) c[l] = a[l];
    return 8;
  }
  double s2 = gam[0] + gam[1] + gam[2];
  int nd = 0;
  unsigned char sel = 0;
  for (int k = 0; k < KSM; ++k) {
    if (!nsm[k]) continue;
    double chi = gam[k] / s2;
    if (fabs(chi - M->ct) < *margin) *margin = fabs(chi - M->ct);
    if (!(chi < M->ct)) {
      sel |= (unsigned char)(1 << k);
      ++nd;
    }
  }
  for (int l = 0; l < M->m; ++l) {
    double v = 0.0;
    if (l < MSM)
      for (int k = 0; k < KSM; ++k)
        if ((sel >> k) & 1) v += as[k][l] / nd;
    c[l] = v;
  }
  return sel;
}

/* Eigenvectors of the Euler flux Jacobian in the direction (nx, ny) at state
 * W (conservative), as matrices acting on conservative variables: L (rows,
 * characteristic fields u-c, u (entropy), u (shear), u+c) and R = L^-1.  They
 * are the textbook 1D eigenvectors in the face frame (normal velocity un,
 * tangential ut) composed with the rotation T: L = L' T, R = T^T R'. */
static void char_basis(double g, const double* W, double nx, double ny, double L[4][4],
                       double R[4][4]) {
  double r = W[0], un = (W[1] * nx + W[2] * ny) / r, ut = (W[2] * nx - W[1] * ny) / r;
  double q2 = un * un + ut * ut, p = (g - 1.0) * (W[3] - 0.5 * r * q2);
  double c = sqrt(g * p / r), H = (W[3] + p) / r;
  double b1 = (g - 1.0) / (c * c), b2 = 0.5 * b1 * q2;
  double Lf[4][4] = {{0.5 * (b2 + un / c), 0.5 * (-b1 * un - 1.0 / c), -0.5 * b1 * ut, 0.5 * b1},
                     {1.0 - b2, b1 * un, b1 * ut, -b1},
                     {-ut, 0.0, 1.0, 0.0},
                     {0.5 * (b2 - un / c), 0.5 * (-b1 * un + 1.0 / c), -0.5 * b1 * ut, 0.5 * b1}};
  double Rf[4][4] = {{1.0, 1.0, 0.0, 1.0},
                     {un - c, un, 0.0, un + c},
                     {ut, ut, 1.0, ut},
                     {H - un * c, 0.5 * q2, ut, H + un * c}};
  double T[4][4] = {{1, 0, 0, 0}, {0, nx, ny, 0}, {0, -ny, nx, 0}, {0, 0, 0, 1}};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double sl = 0.0, sr = 0.0;
      for (int k = 0; k < 4; ++k) {
        sl += Lf[i][k] * T[k][j];
        sr += T[k][i] * Rf[k][j];
      }
      L[i][j] = sl;
      R[i][j] = sr;
    }
}

/* Characteristic-variable reconstruction (Sec. 2.3: characteristic variables
 * suppress oscillations better than conservative ones): for each local edge
 * e of cell t, the coefficients of the four conservative variables are
 * projected on the characteristic fields of the edge's outward normal
 * direction at the cell-average state, each field takes its own TENO
 * selection, and the result is mapped back.  Since the projection is linear
 * and constant over the cell, the edge's reconstruction is again a
 * polynomial of the same basis with coefficients R c~. */
static void char_faces(const omesh* M, int64_t t, const double* U, recon_t* out) {
  const int32_t* nsm = M->nsm + (int64_t)KSM * t;
  const double* P = M->P + 6 * t;
  double W[4];
  for (int v = 0; v < 4; ++v) W[v] = U[(int64_t)v * M->nc + t];
  for (int v = 0; v < 4; ++v) out->margin[v] = 1e300;
  for (int e = 0; e < 3; ++e) {
    int e1 = (e + 1) % 3;
    double dx = P[2 * e1] - P[2 * e], dy = P[2 * e1 + 1] - P[2 * e + 1];
    double len = hypot(dx, dy);
    double L[4][4], R[4][4];
    char_basis(M->gam, W, dy / len, -dx / len, L, R);
    double cc[4][MAXM];
    for (int i = 0; i < 4; ++i) {
      double a[MAXM], as[KSM][MSM], mg;
      for (int l = 0; l < M->m; ++l) {
        double s_ = 0.0;
        for (int v = 0; v < 4; ++v) s_ += L[i][v] * out->a_large[v][l];
        a[l] = s_;
      }
      for (int k = 0; k < KSM; ++k)
        for (int l = 0; l < MSM; ++l) {
          double s_ = 0.0;
          for (int v = 0; v < 4; ++v) s_ += L[i][v] * out->a_small[v][k][l];
          as[k][l] = s_;
        }
      unsigned char sl = teno_field(M, nsm, a, as, cc[i], &mg);
      if (e == 0) out->sel[i] = sl;
      if (mg < out->margin[i]) out->margin[i] = mg;
    }
    for (int v = 0; v < 4; ++v)
      for (int l = 0; l < M->m; ++l) {
        double s_ = 0.0;
        for (int i = 0; i < 4; ++i) s_ += R[v][i] * cc[i][l];
        out->coef_f[e][v][l] = s_;
      }
  }
  out->charf = 1;
}

static void pp_scale(const omesh* M, int64_t t, const double* U, recon_t* R);

static void reconstruct(const omesh* M, int64_t t, const double* U, const unsigned char* sel_in,
                        recon_t* out) {
  const int32_t* st = M->st + (int64_t)ST_TOTAL * t;
  const int32_t* nsm = M->nsm + (int64_t)KSM * t;
  const double* ah = M->ahat[t];
  const double* vo = M->vol[t];
  for (int v = 0; v < M->nvar; ++v) {
    const double* Uv = U + (int64_t)v * M->nc;
    double u0 = Uv[t];
    /* large stencil: b_s = |V'_s| (U_s - U_0), a = Ahat b (Eq. reconstruction_08/09) */
    double a[MAXM];
    for (int l = 0; l < M->m; ++l) {
      double s = 0.0;
      for (int k = 0; k < M->ns; ++k) s += ah[l * M->ns + k] * (vo[k] * (Uv[st[k]] - u0));
      a[l] = s;
    }
    double as[KSM][MSM];
    for (int j = 0; j < KSM; ++j) {
      const double* aj = ah + M->m * M->ns + j * MSM * NSM;
      for (int l = 0; l < MSM; ++l) {
        double s = 0.0;
        if (nsm[j])
          for (int k = 0; k < NSM; ++k) {
            int idx = MAXNS + j * NSM + k;
            s += aj[l * NSM + k] * (vo[idx] * (Uv[st[idx]] - u0));
          }
        as[j][l] = s;
      }
    }
    /* smoothness indicators (Eq. WENO_smoothness); index KSM = large */
    double beta[KSM + 1];
    for (int j = 0; j < KSM; ++j) beta[j] = quad_form(MSM, M->B2, as[j]);
    beta[KSM] = quad_form(M->m, M->Br, a);
    /* scale separation, normalisation, cutoff (Eqs. new_scale_separation,
     * normalize, cutoff); absent directional stencils take no part */
    double gam[KSM + 1], sum = 0.0;
    for (int k = 0; k <= KSM; ++k) {
      int present = k == KSM || nsm[k];
      gam[k] = present ? 1.0 / pow(beta[k] + M->eps, 6.0) : 0.0;
      sum += gam[k];
    }
    double margin = 1e300;
    int delta[KSM + 1];
    for (int k = 0; k <= KSM; ++k) {
      int present = k == KSM || nsm[k];
      double chi = gam[k] / sum;
      delta[k] = present && !(chi < M->ct);
      if (present && fabs(chi - M->ct) < margin) margin = fabs(chi - M->ct);
    }
    double w[KSM] = {0, 0, 0};
    unsigned char sel;
    if (M->linear || delta[KSM]) {
      sel = 8;
    } else {
      /* step (ii): selection among the small stencils (Eq. TENO_weight) */
      double s2 = 0.0;
      for (int k = 0; k < KSM; ++k) s2 += gam[k];
      int nd = 0;
      sel = 0;
      for (int k = 0; k < KSM; ++k) {
        if (!nsm[k]) continue;
        double chi = gam[k] / s2;
        int d = !(chi < M->ct);
        if (fabs(chi - M->ct) < margin) margin = fabs(chi - M->ct);
        if (d) {
          sel |= (unsigned char)(1 << k);
          ++nd;
        }
      }
      (void)nd;
    }
    if (M->linear) margin = 1e300;
    if (sel_in) sel = sel_in[(int64_t)v * M->nc + t];
    if (M->scheme == 1 && !M->linear) {
      /* CWENO (Eqs. CWENO_reconstruction, CWENOweight,
       * CWENOOptimalLinearweight/02): d_K = 1 - 1/d'_K, d_k = (1 - d_K)/K over the K
       * present directional stencils, alpha = d / (beta + eps)^4, w = alpha / sum,
       * P = (w_K / d_K)(P_K - sum_k d_k P_k) + sum_k w_k P_k */
      int K = 0;
      for (int k = 0; k < KSM; ++k) K += nsm[k] != 0;
      double dK = K ? 1.0 - 1.0 / M->cw_dk : 1.0, dk = K ? (1.0 - dK) / K : 0.0;
      double al[KSM + 1], asum = 0.0;
      for (int k = 0; k < KSM; ++k) {
        al[k] = nsm[k] ? dk / pow(beta[k] + M->eps, 4.0) : 0.0;
        asum += al[k];
      }
      al[KSM] = dK / pow(beta[KSM] + M->eps, 4.0);
      asum += al[KSM];
      double wK = al[KSM] / asum;
      for (int l = 0; l < M->m; ++l) {
        double c = wK / dK * a[l];
        if (l < MSM)
          for (int k = 0; k < KSM; ++k)
            if (nsm[k]) c += (al[k] / asum - wK / dK * dk) * as[k][l];
        out->coef[v][l] = c;
      }
      for (int k = 0; k < KSM; ++k) w[k] = nsm[k] ? al[k] / asum : 0.0;
      sel = 8;
      margin = 1e300;
    } else if (sel & 8) {
      for (int l = 0; l < M->m; ++l) out->coef[v][l] = a[l];
    } else {
      int nd = 0;
      for (int k = 0; k < KSM; ++k) nd += (sel >> k) & 1;
      for (int k = 0; k < KSM; ++k) w[k] = ((sel >> k) & 1) ? 1.0 / nd : 0.0;
      for (int l = 0; l < M->m; ++l) {
        double s = 0.0;
        if (l < MSM)
          for (int k = 0; k < KSM; ++k) s += w[k] * as[k][l];
        out->coef[v][l] = s;
      }
    }
    out->sel[v] = sel;
    out->margin[v] = margin;
    for (int k = 0; k <= KSM; ++k) out->beta[v][k] = beta[k];
    for (int l = 0; l < M->m; ++l) out->a_large[v][l] = a[l];
    for (int k = 0; k < KSM; ++k) {
      for (int l = 0; l < MSM; ++l) out->a_small[v][k][l] = as[k][l];
      out->w[v][k] = w[k];
    }
  }
  out->charf = 0;
  if (M->charvar && M->nvar == 4 && M->scheme == 0) char_faces(M, t, U, out);
  if (M->pp) pp_scale(M, t, U, out);
}

/* value of the reconstruction of cell t at physical point (x, y) */
/* value at physical point (x, y) of the reconstruction of cell t used on its
 * local edge e (e only matters for the characteristic reconstruction) */
static void eval_point(const omesh* M, int64_t t, const double* U, const recon_t* R, int e,
                       double x, double y, double* val) {
  double Ji[4], x0[2], xi[2];
  ref_map(M, t, Ji, x0);
  /* bring (x, y) to the periodic image nearest the cell centroid */
  double d[2] = {x - M->cen[2 * t], y - M->cen[2 * t + 1]};
  if (M->periodic) {
    x -= M->L[0] * round(d[0] / M->L[0]);
    y -= M->L[1] * round(d[1] / M->L[1]);
  }
  to_ref(Ji, x0, x, y, xi);
  for (int v = 0; v < M->nvar; ++v) {
    double s = U[(int64_t)v * M->nc + t];
    const double* cf = R->charf ? R->coef_f[e][v] : R->coef[v];
    for (int l = 0; l < M->m; ++l)
      s += cf[l] * (ipow(xi[0], M->ex[l][0]) * ipow(xi[1], M->ex[l][1]) - M->mean0[l]);
    val[v] = s;
  }
}

/* Positivity scaling of a cell's reconstruction (an option, off by default;
 * the paper states no positivity treatment).  The scaling limiter of Zhang
 * and Shu: the polynomial's deviation from the cell average is multiplied by
 * the largest theta <= 1 that keeps the density, then the pressure, at least
 * eps = min(1e-13, its cell-average value) at every face Gauss point of the
 * cell.  The cell average is unchanged (the basis has zero mean).  Density:
 * theta = (rho_0 - eps) / (rho_0 - rho_q) where rho_q < eps; pressure,
 * concave in the state along the segment from the average: bisection on the
 * segment (60 halvings).  Conservative variables only. */
static double pp_press(double g, const double* W) {
  return (g - 1.0) * (W[3] - 0.5 * (W[1] * W[1] + W[2] * W[2]) / W[0]);
}
static void pp_scale(const omesh* M, int64_t t, const double* U, recon_t* R) {
  if (M->nvar != 4 || R->charf) return;
  double U0[4];
  for (int v = 0; v < 4; ++v) U0[v] = U[(int64_t)v * M->nc + t];
  const double er = fmin(1e-13, U0[0]), ep = fmin(1e-13, pp_press(M->gam, U0));
  const double* P = M->P + 6 * t;
  for (int pass = 0; pass < 2; ++pass) {  /* 0: density, 1: pressure */
    double th = 1.0;
    for (int e = 0; e < 3; ++e) {
      const int e1 = (e + 1) % 3;
      const double dx = P[2 * e1] - P[2 * e], dy = P[2 * e1 + 1] - P[2 * e + 1];
      for (int k = 0; k < M->nq; ++k) {
        double Uq[4];
        eval_point(M, t, U, R, e, P[2 * e] + M->gt[k] * dx, P[2 * e + 1] + M->gt[k] * dy, Uq);
        if (pass == 0) {
          if (Uq[0] < er) th = fmin(th, (U0[0] - er) / (U0[0] - Uq[0]));
        } else if (!(pp_press(M->gam, Uq) >= ep)) {
          double lo = 0.0, hi = 1.0;
          for (int it = 0; it < 60; ++it) {
            const double s = 0.5 * (lo + hi);
            double W[4];
            for (int v = 0; v < 4; ++v) W[v] = U0[v] + s * (Uq[v] - U0[v]);
            if (W[0] > 0.0 && pp_press(M->gam, W) >= ep)
              lo = s;
            else
              hi = s;
          }
          th = fmin(th, lo);
        }
      }
    }
    if (th < 1.0)
      for (int v = 0; v < 4; ++v)
        for (int l = 0; l < M->m; ++l) R->coef[v][l] *= th;
  }
}

/* basis values psi_l at physical point for the adjoint */
static void psi_at(const omesh* M, int64_t t, double x, double y, double* psi) {
  double Ji[4], x0[2], xi[2];
  ref_map(M, t, Ji, x0);
  double d[2] = {x - M->cen[2 * t], y - M->cen[2 * t + 1]};
  if (M->periodic) {
    x -= M->L[0] * round(d[0] / M->L[0]);
    y -= M->L[1] * round(d[1] / M->L[1]);
  }
  to_ref(Ji, x0, x, y, xi);
  for (int l = 0; l < M->m; ++l)
    psi[l] = ipow(xi[0], M->ex[l][0]) * ipow(xi[1], M->ex[l][1]) - M->mean0[l];
}

/* ------------------------------------------------------------------------ */
/* fluxes: physical flux in x of a rotated Euler state */
static void euler_fx(double g, const double* W, double* F) {
  double rho = W[0], u = W[1] / rho, v = W[2] / rho, E = W[3];
  double p = (g - 1.0) * (E - 0.5 * rho * (u * u + v * v));
  F[0] = rho * u;
  F[1] = rho * u * u + p;
  F[2] = rho * u * v;
  F[3] = u * (E + p);
}

/* Einfeldt wave speeds from Roe averages (Eq. wavespeed), in the rotated
 * frame; the Roe sound speed uses both velocity components.  The side sound
 * speeds take a negative pressure as zero (a NaN pressure stays NaN): a
 * Gauss state at the positivity floor has a pressure some 1e-15 of its
 * energy, below what a lower-precision evaluation resolves, and its wave
 * speed is then the particle speed, not the Roe bound alone. */
static void wave_speeds(double g, const double* WL, const double* WR, double* SL, double* SR) {
  double rL = WL[0], uL = WL[1] / rL, vL = WL[2] / rL;
  double rR = WR[0], uR = WR[1] / rR, vR = WR[2] / rR;
  double pL = (g - 1.0) * (WL[3] - 0.5 * rL * (uL * uL + vL * vL));
  double pR = (g - 1.0) * (WR[3] - 0.5 * rR * (uR * uR + vR * vR));
  double cL = sqrt(g * (pL < 0.0 ? 0.0 : pL) / rL), cR = sqrt(g * (pR < 0.0 ? 0.0 : pR) / rR);
  double HL = (WL[3] + pL) / rL, HR = (WR[3] + pR) / rR;
  double D = sqrt(rR / rL);
  double ut = (uL + uR * D) / (1.0 + D);
  double vt = (vL + vR * D) / (1.0 + D);
  double Ht = (HL + HR * D) / (1.0 + D);
  double ct = sqrt((g - 1.0) * (Ht - 0.5 * (ut * ut + vt * vt)));
  *SL = fmin(uL - cL, ut - ct);
  *SR = fmax(uR + cR, ut + ct);
}

static void rotate(double nx, double ny, const double* U, double* W) {
  W[0] = U[0];
  W[1] = nx * U[1] + ny * U[2];
  W[2] = -ny * U[1] + nx * U[2];
  W[3] = U[3];
}

static void unrotate(double nx, double ny, const double* W, double* U) {
  U[0] = W[0];
  U[1] = nx * W[1] - ny * W[2];
  U[2] = ny * W[1] + nx * W[2];
  U[3] = W[3];
}

/* numerical flux through a face with unit normal (nx, ny) from L to R */
/* radial taper of the rotation field: 1 for r <= r1, smoothstep to 0 at r2
 * (no taper when r2 <= r1) */
static double rot_taper(const omesh* M, double r) {
  double r1 = M->rot[3], r2 = M->rot[4];
  if (!(r2 > r1) || r <= r1) return 1.0;
  if (r >= r2) return 0.0;
  double s = (r - r1) / (r2 - r1);
  return 1.0 - s * s * (3.0 - 2.0 * s);
}

/* normal advection speed v(x, y) . n of the scalar equation: a constant
 * velocity, or the rigid rotation v = omega phi(r) (-(y - y_c), x - x_c) of the
 * solid-body rotation case (Sec. 5, v = (0.5 - y, x - 0.5)) with the radial
 * taper phi (azimuthal, hence divergence-free for any phi) */
static double adv_normal(const omesh* M, double x, double y, double nx, double ny) {
  if (M->field == 1) {
    double dx = x - M->rot[0], dy = y - M->rot[1];
    return M->rot[2] * rot_taper(M, sqrt(dx * dx + dy * dy)) * (-dy * nx + dx * ny);
  }
  return M->adv[0] * nx + M->adv[1] * ny;
}

/* numerical flux at a face point (x, y) with unit normal (nx, ny) */
static void num_flux(const omesh* M, const double* UL, const double* UR, double nx, double ny,
                     double x, double y, double* F) {
  if (M->flux == FLUX_UPWIND) {
    double an = adv_normal(M, x, y, nx, ny);
    F[0] = an * (an >= 0.0 ? UL[0] : UR[0]);
    return;
  }
  double g = M->gam;
  double WL[4], WR[4], FL[4], FR[4], Fx[4];
  rotate(nx, ny, UL, WL);
  rotate(nx, ny, UR, WR);
  euler_fx(g, WL, FL);
  euler_fx(g, WR, FR);
  double SL, SR;
  wave_speeds(g, WL, WR, &SL, &SR);
  if (M->flux == FLUX_HLL) {
    if (0.0 <= SL) {
      for (int k = 0; k < 4; ++k) Fx[k] = FL[k];
    } else if (0.0 >= SR) {
      for (int k = 0; k < 4; ++k) Fx[k] = FR[k];
    } else {
      for (int k = 0; k < 4; ++k)
        Fx[k] = (SR * FL[k] - SL * FR[k] + SL * SR * (WR[k] - WL[k])) / (SR - SL);
    }
  } else {
    /* HLLC (Toro): contact speed S* and star states.  The star energy is
     * Toro's f (E/rho + (S* - u)(S* + p / (rho (S - u)))) multiplied out, so
     * that no term divides by S - u.  S* is undefined when rho_L (S_L - u_L)
     * = rho_R (S_R - u_R), which happens only when both bounds equal the
     * particle speeds (zero sound speed on both sides, as at a reflecting
     * wall whose Gauss state has zero pressure); there the flux is HLL's. */
    double rL = WL[0], uL = WL[1] / rL, vL = WL[2] / rL;
    double rR = WR[0], uR = WR[1] / rR, vR = WR[2] / rR;
    double pL = (g - 1.0) * (WL[3] - 0.5 * rL * (uL * uL + vL * vL));
    double pR = (g - 1.0) * (WR[3] - 0.5 * rR * (uR * uR + vR * vR));
    double den = rL * (SL - uL) - rR * (SR - uR);
    double Ss = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / den;
    if (0.0 <= SL) {
      for (int k = 0; k < 4; ++k) Fx[k] = FL[k];
    } else if (0.0 >= SR) {
      for (int k = 0; k < 4; ++k) Fx[k] = FR[k];
    } else if (den == 0.0) {
      for (int k = 0; k < 4; ++k)
        Fx[k] = (SR * FL[k] - SL * FR[k] + SL * SR * (WR[k] - WL[k])) / (SR - SL);
    } else if (0.0 <= Ss) {
      double f = rL * (SL - uL) / (SL - Ss);
      double Us[4] = {f, f * Ss, f * vL,
                      ((SL - uL) * WL[3] + (Ss - uL) * (rL * (SL - uL) * Ss + pL)) / (SL - Ss)};
      for (int k = 0; k < 4; ++k) Fx[k] = FL[k] + SL * (Us[k] - WL[k]);
    } else {
      double f = rR * (SR - uR) / (SR - Ss);
      double Us[4] = {f, f * Ss, f * vR,
                      ((SR - uR) * WR[3] + (Ss - uR) * (rR * (SR - uR) * Ss + pR)) / (SR - Ss)};
      for (int k = 0; k < 4; ++k) Fx[k] = FR[k] + SR * (Us[k] - WR[k]);
    }
  }
  unrotate(nx, ny, Fx, F);
}

/* ------------------------------------------------------------------------ */
/* forward-mode dual numbers (8 directions) for flux Jacobians */
#define ND 8
typedef struct {
  double v, d[ND];
} dual;

static dual dc(double x) {
  dual r;
  r.v = x;
  for (int i = 0; i < ND; ++i) r.d[i] = 0.0;
  return r;
}
static dual dadd(dual a, dual b) {
  dual r;
  r.v = a.v + b.v;
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
static dual dsub(dual a, dual b) {
  dual r;
  r.v = a.v - b.v;
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
static dual dmul(dual a, dual b) {
  dual r;
  r.v = a.v * b.v;
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
static dual ddiv(dual a, dual b) {
  dual r;
  r.v = a.v / b.v;
  for (int i = 0; i < ND; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;
  return r;
}
static dual dscale(double s, dual a) {
  dual r;
  r.v = s * a.v;
  for (int i = 0; i < ND; ++i) r.d[i] = s * a.d[i];
  return r;
}
static dual dsqrt(dual a) {
  dual r;
  r.v = sqrt(a.v);
  /* the root of a constant zero (a clamped pressure) has no derivative */
  for (int i = 0; i < ND; ++i) r.d[i] = r.v == 0.0 ? 0.0 : a.d[i] / (2.0 * r.v);
  return r;
}
/* a negative pressure taken as zero in a sound speed (see wave_speeds) */
static dual dpos(dual a) { return a.v < 0.0 ? dc(0.0) : a; }
static dual dmin(dual a, dual b) { return a.v <= b.v ? a : b; }
static dual dmax(dual a, dual b) { return a.v >= b.v ? a : b; }

static void euler_fx_d(double g, const dual* W, dual* F) {
  dual rho = W[0], u = ddiv(W[1], rho), v = ddiv(W[2], rho), E = W[3];
  dual ke = dscale(0.5, dmul(rho, dadd(dmul(u, u), dmul(v, v))));
  dual p = dscale(g - 1.0, dsub(E, ke));
  F[0] = dmul(rho, u);
  F[1] = dadd(dmul(dmul(rho, u), u), p);
  F[2] = dmul(dmul(rho, u), v);
  F[3] = dmul(u, dadd(E, p));
}

static void num_flux_d(const omesh* M, const dual* UL, const dual* UR, double nx, double ny,
                       double x, double y, dual* F) {
  if (M->flux == FLUX_UPWIND) {
    double an = adv_normal(M, x, y, nx, ny);
    F[0] = dscale(an, an >= 0.0 ? UL[0] : UR[0]);
    return;
  }
  double g = M->gam;
  dual WL[4], WR[4], FL[4], FR[4], Fx[4];
  WL[0] = UL[0];
  WL[1] = dadd(dscale(nx, UL[1]), dscale(ny, UL[2]));
  WL[2] = dadd(dscale(-ny, UL[1]), dscale(nx, UL[2]));
  WL[3] = UL[3];
  WR[0] = UR[0];
  WR[1] = dadd(dscale(nx, UR[1]), dscale(ny, UR[2]));
  WR[2] = dadd(dscale(-ny, UR[1]), dscale(nx, UR[2]));
  WR[3] = UR[3];
  euler_fx_d(g, WL, FL);
  euler_fx_d(g, WR, FR);
  dual rL = WL[0], uL = ddiv(WL[1], rL), vL = ddiv(WL[2], rL);
  dual rR = WR[0], uR = ddiv(WR[1], rR), vR = ddiv(WR[2], rR);
  dual pL = dscale(g - 1.0, dsub(WL[3], dscale(0.5, dmul(rL, dadd(dmul(uL, uL), dmul(vL, vL))))));
  dual pR = dscale(g - 1.0, dsub(WR[3], dscale(0.5, dmul(rR, dadd(dmul(uR, uR), dmul(vR, vR))))));
  dual cL = dsqrt(ddiv(dscale(g, dpos(pL)), rL)), cR = dsqrt(ddiv(dscale(g, dpos(pR)), rR));
  dual HL = ddiv(dadd(WL[3], pL), rL), HR = ddiv(dadd(WR[3], pR), rR);
  dual D = dsqrt(ddiv(rR, rL));
  dual den = dadd(dc(1.0), D);
  dual ut = ddiv(dadd(uL, dmul(uR, D)), den);
  dual vt = ddiv(dadd(vL, dmul(vR, D)), den);
  dual Ht = ddiv(dadd(HL, dmul(HR, D)), den);
  dual ctl = dsqrt(dscale(g - 1.0, dsub(Ht, dscale(0.5, dadd(dmul(ut, ut), dmul(vt, vt))))));
  dual SL = dmin(dsub(uL, cL), dsub(ut, ctl));
  dual SR = dmax(dadd(uR, cR), dadd(ut, ctl));
  if (M->flux == FLUX_HLL) {
    if (0.0 <= SL.v) {
      for (int k = 0; k < 4; ++k) Fx[k] = FL[k];
    } else if (0.0 >= SR.v) {
      for (int k = 0; k < 4; ++k) Fx[k] = FR[k];
    } else {
      for (int k = 0; k < 4; ++k)
        Fx[k] = ddiv(dadd(dsub(dmul(SR, FL[k]), dmul(SL, FR[k])),
                          dmul(dmul(SL, SR), dsub(WR[k], WL[k]))),
                     dsub(SR, SL));
    }
  } else {
    dual aL = dmul(rL, dsub(SL, uL)), aR = dmul(rR, dsub(SR, uR));
    dual dnm = dsub(aL, aR);
    dual Ss = ddiv(dadd(dsub(pR, pL), dsub(dmul(aL, uL), dmul(aR, uR))), dnm);
    if (0.0 <= SL.v) {
      for (int k = 0; k < 4; ++k) Fx[k] = FL[k];
    } else if (0.0 >= SR.v) {
      for (int k = 0; k < 4; ++k) Fx[k] = FR[k];
    } else if (dnm.v == 0.0) {
      for (int k = 0; k < 4; ++k)
        Fx[k] = ddiv(dadd(dsub(dmul(SR, FL[k]), dmul(SL, FR[k])),
                          dmul(dmul(SL, SR), dsub(WR[k], WL[k]))),
                     dsub(SR, SL));
    } else {
      int left = 0.0 <= Ss.v;
      dual r = left ? rL : rR, u = left ? uL : uR, v = left ? vL : vR, p = left ? pL : pR;
      dual S = left ? SL : SR;
      const dual* W = left ? WL : WR;
      const dual* FK = left ? FL : FR;
      dual Smu = dsub(S, u), SmS = dsub(S, Ss);
      dual f = ddiv(dmul(r, Smu), SmS);
      dual e = ddiv(dadd(dmul(Smu, W[3]), dmul(dsub(Ss, u), dadd(dmul(dmul(r, Smu), Ss), p))), SmS);
      dual Us[4] = {f, dmul(f, Ss), dmul(f, v), e};
      for (int k = 0; k < 4; ++k) Fx[k] = dadd(FK[k], dmul(S, dsub(Us[k], W[k])));
    }
  }
  F[0] = Fx[0];
  F[1] = dsub(dscale(nx, Fx[1]), dscale(ny, Fx[2]));
  F[2] = dadd(dscale(ny, Fx[1]), dscale(nx, Fx[2]));
  F[3] = Fx[3];
}

/* Jacobians dF/dUL and dF/dUR, [nvar][nvar] each, row = flux component */
static void flux_jac(const omesh* M, const double* UL, const double* UR, double nx, double ny,
                     double x, double y, double* JL, double* JR) {
  int nv = M->nvar;
  dual L[4], R[4], F[4];
  for (int k = 0; k < 4; ++k) L[k] = R[k] = dc(0.0);
  for (int k = 0; k < nv; ++k) {
    L[k] = dc(UL[k]);
    R[k] = dc(UR[k]);
    L[k].d[k] = 1.0;
    R[k].d[nv + k] = 1.0;
  }
  num_flux_d(M, L, R, nx, ny, x, y, F);
  for (int i = 0; i < nv; ++i)
    for (int k = 0; k < nv; ++k) {
      JL[i * nv + k] = F[i].d[k];
      JR[i * nv + k] = F[i].d[nv + k];
    }
}

/* ------------------------------------------------------------------------ */
/* boundary ghost state at a boundary face point (readings for the shock case) */
static void ghost_state(const omesh* M, int tag, const double* UL, double nx, double ny, double x,
                        double y, double* UR) {
  (void)y;
  double g = M->gam;
  if (tag == BC_WALL) {
    double un = UL[1] * nx + UL[2] * ny;
    UR[0] = UL[0];
    UR[1] = UL[1] - 2.0 * un * nx;
    UR[2] = UL[2] - 2.0 * un * ny;
    UR[3] = UL[3];
    return;
  }
  double post[4] = {8.0, 7.145, -4.125, 116.8333};
  double pre[4] = {1.4, 0.0, 0.0, 1.0};
  const double* s = NULL;
  if (tag == BC_INFLOW) s = post;
  if (tag == BC_TOP) {
    double xs = 0.1667 + (1.0 + 20.0 * M->time) / 1.732;
    s = x < xs ? post : pre;
  }
  if (s) {
    UR[0] = s[0];
    UR[1] = s[0] * s[1];
    UR[2] = s[0] * s[2];
    UR[3] = s[3] / (g - 1.0) + 0.5 * s[0] * (s[1] * s[1] + s[2] * s[2]);
    return;
  }
  for (int k = 0; k < M->nvar; ++k) UR[k] = UL[k];
}

/* ------------------------------------------------------------------------ */
/* public API */

void* oracle_new(int64_t nv, const double* xy, int64_t nc, const int32_t* tri, int64_t nbf,
                 const int32_t* bface, const double* period, const int32_t* iopt,
                 const double* dopt, int32_t* status) {
  omesh* M = (omesh*)calloc(1, sizeof(omesh));
  M->nv = nv;
  M->nc = nc;
  M->xy = xy;
  M->tri = tri;
  M->periodic = period != NULL;
  if (period) {
    M->L[0] = period[0];
    M->L[1] = period[1];
  }
  M->order = iopt[0];
  M->nq = iopt[1];
  M->nvar = iopt[2];
  M->flux = iopt[3];
  M->linear = iopt[4];
  M->ct = dopt[0];
  M->eps = dopt[1];
  M->gam = dopt[2];
  M->adv[0] = dopt[3];
  M->adv[1] = dopt[4];
  M->field = iopt[5];
  M->rot[0] = dopt[5];
  M->rot[1] = dopt[6];
  M->rot[2] = dopt[7];
  M->rot[3] = dopt[8];
  M->rot[4] = dopt[9];
  M->scheme = iopt[6];
  M->charvar = iopt[7];
  M->pp = iopt[8];
  M->cw_dk = dopt[10];
  M->r = M->order - 1;
  M->m = (M->r + 1) * (M->r + 2) / 2 - 1;
  M->ns = 2 * (M->m + 1);
  *status = E_OK;
  if (M->order < 3 || M->order > 6 || M->nq < 1 || M->nq > MAXNQ ||
      (M->nvar != 1 && M->nvar != 4)) {
    *status = E_INVAL;
    return M;
  }
  int rc = setup_reference(M);
  if (!rc) rc = build_topology(M, nbf, bface);
  M->built = (unsigned char*)calloc(nc, 1);
  M->st = (int32_t*)malloc(sizeof(int32_t) * ST_TOTAL * nc);
  M->nsm = (int32_t*)calloc(KSM * nc, sizeof(int32_t));
  M->ahat = (double**)calloc(nc, sizeof(double*));
  M->vol = (double**)calloc(nc, sizeof(double*));
  *status = rc;
  return M;
}

void oracle_free(void* h) {
  omesh* M = (omesh*)h;
  if (!M) return;
  if (M->ahat)
    for (int64_t c = 0; c < M->nc; ++c) {
      free(M->ahat[c]);
      free(M->vol[c]);
    }
  free(M->ahat);
  free(M->vol);
  free(M->built);
  free(M->st);
  free(M->nsm);
  free(M->P);
  free(M->cen);
  free(M->area);
  free(M->perim);
  free(M->v2c_off);
  free(M->v2c);
  free(M->fnbr);
  free(M->fedge);
  free(M->fbc);
  free(M->fo);
  free(M);
}

/* build stencils and pseudo-inverses for the listed cells (all if cells NULL) */
int oracle_prepare(void* h, int64_t n, const int64_t* cells) {
  omesh* M = (omesh*)h;
  int64_t cnt = cells ? n : M->nc;
  int64_t* list = NULL;
  if (cells) { /* sorted, duplicate-free copy so no cell is built twice at once */
    list = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    memcpy(list, cells, sizeof(int64_t) * n);
    qsort(list, n, sizeof(int64_t), cmp_i64);
    int64_t u = 0;
    for (int64_t i = 0; i < n; ++i)
      if (u == 0 || list[u - 1] != list[i]) list[u++] = list[i];
    cnt = u;
  }
  int rc = E_OK;
#pragma omp parallel
  {
    int32_t* seen = (int32_t*)calloc(M->nc, sizeof(int32_t));
    int32_t stamp = 0;
#pragma omp for schedule(dynamic, 64)
    for (int64_t i = 0; i < cnt; ++i) {
      int64_t c = list ? list[i] : i;
      ++stamp;
      int r = ensure_cell(M, c, seen, stamp);
      if (r) {
#pragma omp critical
        rc = r;
      }
    }
    free(seen);
  }
  free(list);
  return rc;
}

int oracle_stencils(void* h, int32_t* large, int32_t* small) {
  omesh* M = (omesh*)h;
  int rc = oracle_prepare(h, 0, NULL);
  if (rc) return rc;
  for (int64_t c = 0; c < M->nc; ++c) {
    const int32_t* st = M->st + (int64_t)ST_TOTAL * c;
    for (int k = 0; k < M->ns; ++k) large[c * M->ns + k] = st[k];
    for (int k = 0; k < KSM * NSM; ++k) small[c * KSM * NSM + k] = st[MAXNS + k];
  }
  return E_OK;
}

/* reconstruction matrix access for pins: which = 0 large, 1..3 directional */
int oracle_recon_matrix(void* h, int64_t c, int which, double* A, double* Ahat, double* vol,
                        int32_t* ids) {
  omesh* M = (omesh*)h;
  int rc = oracle_prepare(h, 1, &c);
  if (rc) return rc;
  const int32_t* st = M->st + (int64_t)ST_TOTAL * c;
  int n = which == 0 ? M->ns : NSM;
  int mm = which == 0 ? M->m : MSM;
  const int32_t* sid = which == 0 ? st : st + MAXNS + (which - 1) * NSM;
  if (which > 0 && M->nsm[KSM * c + which - 1] == 0) return E_STENCIL;
  double v[MAXNS];
  if (A) build_A(M, c, n, sid, mm, A, v);
  if (vol) {
    double tmp[MAXNS * MAXM];
    build_A(M, c, n, sid, mm, tmp, vol);
  }
  if (ids)
    for (int k = 0; k < n; ++k) ids[k] = sid[k];
  if (Ahat) {
    const double* src = which == 0 ? M->ahat[c] : M->ahat[c] + M->m * M->ns + (which - 1) * MSM * NSM;
    memcpy(Ahat, src, sizeof(double) * n * mm);
  }
  return E_OK;
}

void oracle_reference_data(void* h, double* mean0, double* Br, double* B2, int32_t* ex,
                           double* gt, double* gw) {
  omesh* M = (omesh*)h;
  memcpy(mean0, M->mean0, sizeof(double) * M->m);
  memcpy(Br, M->Br, sizeof(double) * M->m * M->m);
  memcpy(B2, M->B2, sizeof(double) * MSM * MSM);
  for (int l = 0; l < M->m; ++l) {
    ex[2 * l] = M->ex[l][0];
    ex[2 * l + 1] = M->ex[l][1];
  }
  memcpy(gt, M->gt, sizeof(double) * M->nq);
  memcpy(gw, M->gw, sizeof(double) * M->nq);
}

/* per-cell reconstruction outputs for pins: coef [nvar][m], beta [nvar][4],
 * sel [nvar], margin [nvar] */
int oracle_recon_cell(void* h, const double* U, int64_t c, double* coef, double* beta,
                      uint8_t* sel, double* margin) {
  omesh* M = (omesh*)h;
  int rc = oracle_prepare(h, 1, &c);
  if (rc) return rc;
  recon_t R;
  reconstruct(M, c, U, NULL, &R);
  for (int v = 0; v < M->nvar; ++v) {
    for (int l = 0; l < M->m; ++l) coef[v * M->m + l] = R.coef[v][l];
    for (int k = 0; k <= KSM; ++k) beta[v * 4 + k] = R.beta[v][k];
    sel[v] = R.sel[v];
    margin[v] = R.margin[v];
  }
  return E_OK;
}

/* face flux K = |A| sum_k w_k F(U_L(x_k), U_R(x_k)) for owner cell c, local
 * edge e; the neighbour's reconstruction is evaluated at the same physical
 * points.  Also returns the states (for the adjoint). */
static void face_flux(const omesh* M, int64_t c, int e, const double* U, const recon_t* Rc,
                      const recon_t* Rn, double* K, double* ULq, double* URq) {
  const double* P = M->P + 6 * c;
  int e1 = (e + 1) % 3;
  double dx = P[2 * e1] - P[2 * e], dy = P[2 * e1 + 1] - P[2 * e + 1];
  double len = hypot(dx, dy);
  double nx = dy / len, ny = -dx / len;
  int64_t n = M->fnbr[3 * c + e];
  for (int v = 0; v < M->nvar; ++v) K[v] = 0.0;
  for (int k = 0; k < M->nq; ++k) {
    double x = P[2 * e] + M->gt[k] * dx, y = P[2 * e + 1] + M->gt[k] * dy;
    double UL[4], UR[4], F[4];
    /* a cell of the outflow layer enters with its cell average (at the
     * outflow face itself: zero gradient of the cell averages) */
    if (M->fo[c])
      for (int v = 0; v < M->nvar; ++v) UL[v] = U[(int64_t)v * M->nc + c];
    else
      eval_point(M, c, U, Rc, e, x, y, UL);
    if (n >= 0 && M->fo[n])
      for (int v = 0; v < M->nvar; ++v) UR[v] = U[(int64_t)v * M->nc + n];
    else if (n >= 0)
      eval_point(M, n, U, Rn, M->fedge[3 * c + e], x, y, UR);
    else
      ghost_state(M, M->fbc[3 * c + e], UL, nx, ny, x, y, UR);
    num_flux(M, UL, UR, nx, ny, x, y, F);
    for (int v = 0; v < M->nvar; ++v) {
      K[v] += M->gw[k] * F[v];
      if (ULq) ULq[k * M->nvar + v] = UL[v];
      if (URq) URq[k * M->nvar + v] = UR[v];
    }
  }
  for (int v = 0; v < M->nvar; ++v) K[v] *= len;
}

static int is_owner(const omesh* M, int64_t c, int e) {
  int64_t n = M->fnbr[3 * c + e];
  return n < 0 || c < n;
}

/* full residual R = -(1/|V|) sum_faces K (Eq. fv_governing_equation_semi_discrete);
 * sel/margin optional [nvar][nc]; sel_in optional override */
int oracle_residual(void* h, const double* U, double time, double* R, uint8_t* sel,
                    double* margin, const uint8_t* sel_in) {
  omesh* M = (omesh*)h;
  M->time = time;
  int rc = oracle_prepare(h, 0, NULL);
  if (rc) return rc;
  int64_t nc = M->nc;
  int nvar = M->nvar;
  recon_t* RC = (recon_t*)malloc(sizeof(recon_t) * nc);
  if (!RC) return E_MEM;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) reconstruct(M, c, U, sel_in, &RC[c]);
  double* K = (double*)calloc(3 * nc * nvar, sizeof(double));
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c)
    for (int e = 0; e < 3; ++e) {
      if (!is_owner(M, c, e)) continue;
      int64_t n = M->fnbr[3 * c + e];
      face_flux(M, c, e, U, &RC[c], n >= 0 ? &RC[n] : NULL, K + (3 * c + e) * nvar, NULL, NULL);
    }
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) {
    double acc[4] = {0, 0, 0, 0};
    for (int e = 0; e < 3; ++e) {
      const double* Kf;
      double s;
      if (is_owner(M, c, e)) {
        Kf = K + (3 * c + e) * nvar;
        s = 1.0;
      } else {
        int64_t n = M->fnbr[3 * c + e];
        Kf = K + (3 * n + M->fedge[3 * c + e]) * nvar;
        s = -1.0;
      }
      for (int v = 0; v < nvar; ++v) acc[v] += s * Kf[v];
    }
    for (int v = 0; v < nvar; ++v) R[v * nc + c] = -acc[v] / M->area[c];
    if (sel)
      for (int v = 0; v < nvar; ++v) sel[v * nc + c] = RC[c].sel[v];
    if (margin)
      for (int v = 0; v < nvar; ++v) margin[v * nc + c] = RC[c].margin[v];
  }
  free(K);
  free(RC);
  return E_OK;
}

/* residual at selected cells only: R_out [n][nvar]; sel_out [n][nvar] and
 * margin_out [n][nvar] of those cells and of their face neighbours folded in
 * (margin = min over the cell and its neighbours) */
/* residuals of the listed cells; optional outputs: selection, cutoff margin
 * (smallest over the cell and its face neighbours) and the flux-sum scale
 * sum_faces |K_f| / |V| per variable (the size of the terms that cancel in
 * R, for judging rounding differences) */
int oracle_residual_cells(void* h, const double* U, double time, int64_t n, const int64_t* cells,
                          double* R_out, uint8_t* sel_out, double* margin_out,
                          double* scale_out) {
  omesh* M = (omesh*)h;
  M->time = time;
  int nvar = M->nvar;
  int64_t* need = (int64_t*)malloc(sizeof(int64_t) * 4 * n);
  for (int64_t i = 0; i < n; ++i) {
    need[4 * i] = cells[i];
    for (int e = 0; e < 3; ++e) {
      int64_t nb = M->fnbr[3 * cells[i] + e];
      need[4 * i + 1 + e] = nb >= 0 ? nb : cells[i];
    }
  }
  int rc = oracle_prepare(h, 4 * n, need);
  free(need);
  if (rc) return rc;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = cells[i];
    recon_t Rc, Rn;
    reconstruct(M, c, U, NULL, &Rc);
    double acc[4] = {0, 0, 0, 0}, mag[4] = {0, 0, 0, 0};
    double mg[4];
    for (int v = 0; v < nvar; ++v) mg[v] = Rc.margin[v];
    for (int e = 0; e < 3; ++e) {
      int64_t nb = M->fnbr[3 * c + e];
      double K[4];
      if (nb >= 0) {
        reconstruct(M, nb, U, NULL, &Rn);
        for (int v = 0; v < nvar; ++v)
          if (Rn.margin[v] < mg[v]) mg[v] = Rn.margin[v];
      }
      if (is_owner(M, c, e)) {
        face_flux(M, c, e, U, &Rc, nb >= 0 ? &Rn : NULL, K, NULL, NULL);
        for (int v = 0; v < nvar; ++v) acc[v] += K[v];
      } else {
        face_flux(M, nb, M->fedge[3 * c + e], U, &Rn, &Rc, K, NULL, NULL);
        for (int v = 0; v < nvar; ++v) acc[v] -= K[v];
      }
      for (int v = 0; v < nvar; ++v) mag[v] += fabs(K[v]);
    }
    for (int v = 0; v < nvar; ++v) {
      R_out[i * nvar + v] = -acc[v] / M->area[c];
      if (scale_out) scale_out[i * nvar + v] = mag[v] / M->area[c];
      if (sel_out) sel_out[i * nvar + v] = Rc.sel[v];
      if (margin_out) margin_out[i * nvar + v] = mg[v];
    }
  }
  return err ? E_INVAL : E_OK;
}

/* dt = CFL * min_i (4|V_i|/P_i) / (|v_i| + c_i) */
double oracle_cfl_dt(void* h, const double* U, double cfl) {
  omesh* M = (omesh*)h;
  double best = 1e300;
  for (int64_t c = 0; c < M->nc; ++c) {
    double s;
    if (M->nvar == 1 && M->field == 1) {
      /* largest speed over the cell: at the vertex farthest from the centre */
      double smax = 0.0;
      for (int k = 0; k < 3; ++k) {
        double dx = M->P[6 * c + 2 * k] - M->rot[0], dy = M->P[6 * c + 2 * k + 1] - M->rot[1];
        double r = sqrt(dx * dx + dy * dy);
        double sv = r * rot_taper(M, r);
        if (sv > smax) smax = sv;
      }
      s = fabs(M->rot[2]) * smax;
      if (!(s > 0.0)) s = 1e-300; /* a cell at rest does not limit the step */
    } else if (M->nvar == 1) {
      s = sqrt(M->adv[0] * M->adv[0] + M->adv[1] * M->adv[1]);
    } else {
      double rho = U[c], u = U[M->nc + c] / rho, v = U[2 * M->nc + c] / rho;
      double p = (M->gam - 1.0) * (U[3 * M->nc + c] - 0.5 * rho * (u * u + v * v));
      s = sqrt(u * u + v * v) + sqrt(M->gam * p / rho);
    }
    double d = 4.0 * M->area[c] / M->perim[c] / s;
    if (d < best) best = d;
  }
  return cfl * best;
}

/* one SSP-RK3 step in place (Eq. fv_time_discretization_01) */
int oracle_rk3_step(void* h, double* U, double time, double dt) {
  omesh* M = (omesh*)h;
  int64_t N = M->nc * M->nvar;
  double* R = (double*)malloc(sizeof(double) * N);
  double* U1 = (double*)malloc(sizeof(double) * N);
  double* U2 = (double*)malloc(sizeof(double) * N);
  int rc = oracle_residual(h, U, time, R, NULL, NULL, NULL);
  for (int64_t i = 0; i < N && !rc; ++i) U1[i] = U[i] + dt * R[i];
  if (!rc) rc = oracle_residual(h, U1, time + dt, R, NULL, NULL, NULL);
  for (int64_t i = 0; i < N && !rc; ++i) U2[i] = 0.75 * U[i] + 0.25 * U1[i] + 0.25 * dt * R[i];
  if (!rc) rc = oracle_residual(h, U2, time + 0.5 * dt, R, NULL, NULL, NULL);
  for (int64_t i = 0; i < N && !rc; ++i)
    U[i] = U[i] / 3.0 + 2.0 / 3.0 * U2[i] + 2.0 / 3.0 * dt * R[i];
  free(R);
  free(U1);
  free(U2);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* discrete adjoint: v = (dR/dU)^T w at state U, selection frozen at U (or
 * given by sel_in), flux branches frozen at the forward states */
int oracle_residual_vjp(void* h, const double* U, double time, const double* w, double* vout,
                        const uint8_t* sel_in) {
  if (((omesh*)h)->charvar || ((omesh*)h)->scheme || ((omesh*)h)->pp)
    return E_INVAL; /* TENO in conservative variables, no positivity scaling */
  omesh* M = (omesh*)h;
  M->time = time;
  int rc = oracle_prepare(h, 0, NULL);
  if (rc) return rc;
  int64_t nc = M->nc;
  int nvar = M->nvar, nq = M->nq;
  recon_t* RC = (recon_t*)malloc(sizeof(recon_t) * nc);
  for (int64_t c = 0; c < nc; ++c) reconstruct(M, c, U, sel_in, &RC[c]);
  /* adjoint of the Gauss-point values: Ubar[c][e][k][v]; of the cell
   * averages taken directly by outflow-layer cells: direct[v][c] */
  double* Ubar = (double*)calloc(nc * 3 * nq * nvar, sizeof(double));
  double* direct = (double*)calloc(nc * nvar, sizeof(double));
  for (int64_t c = 0; c < nc; ++c)
    for (int e = 0; e < 3; ++e) {
      if (!is_owner(M, c, e)) continue;
      int64_t n = M->fnbr[3 * c + e];
      /* Kbar = dJ/dK: R_c has -K/|V_c|, R_n has +K/|V_n| */
      double Kb[4];
      for (int v = 0; v < nvar; ++v) {
        Kb[v] = -w[v * nc + c] / M->area[c];
        if (n >= 0) Kb[v] += w[v * nc + n] / M->area[n];
      }
      const double* P = M->P + 6 * c;
      int e1 = (e + 1) % 3;
      double dx = P[2 * e1] - P[2 * e], dy = P[2 * e1 + 1] - P[2 * e + 1];
      double len = hypot(dx, dy);
      double nx = dy / len, ny = -dx / len;
      for (int k = 0; k < nq; ++k) {
        double x = P[2 * e] + M->gt[k] * dx, y = P[2 * e + 1] + M->gt[k] * dy;
        double UL[4], UR[4], JL[16], JR[16];
        /* outflow-layer sides take the cell average (as in face_flux) */
        const int fl = M->fo[c], fr = n >= 0 && M->fo[n];
        if (fl)
          for (int v = 0; v < nvar; ++v) UL[v] = U[(int64_t)v * nc + c];
        else
          eval_point(M, c, U, &RC[c], e, x, y, UL);
        if (fr)
          for (int v = 0; v < nvar; ++v) UR[v] = U[(int64_t)v * nc + n];
        else if (n >= 0)
          eval_point(M, n, U, &RC[n], M->fedge[3 * c + e], x, y, UR);
        else
          ghost_state(M, M->fbc[3 * c + e], UL, nx, ny, x, y, UR);
        flux_jac(M, UL, UR, nx, ny, x, y, JL, JR);
        double wk = M->gw[k] * len;
        double bl[4] = {0, 0, 0, 0}, br[4] = {0, 0, 0, 0};
        for (int i = 0; i < nvar; ++i)
          for (int j = 0; j < nvar; ++j) {
            bl[j] += wk * JL[i * nvar + j] * Kb[i];
            br[j] += wk * JR[i * nvar + j] * Kb[i];
          }
        if (n < 0) {
          /* ghost state depends on UL: chain rule through the ghost map */
          double G[16];
          int tag = M->fbc[3 * c + e];
          for (int i = 0; i < 16; ++i) G[i] = 0.0;
          if (tag == BC_WALL) {
            G[0] = 1.0;
            G[5] = 1.0 - 2.0 * nx * nx;
            G[6] = -2.0 * nx * ny;
            G[9] = -2.0 * ny * nx;
            G[10] = 1.0 - 2.0 * ny * ny;
            G[15] = 1.0;
          } else if (tag == BC_OUTFLOW) {
            for (int i = 0; i < nvar; ++i) G[i * nvar + i] = 1.0;
          }
          for (int j = 0; j < nvar; ++j)
            for (int i = 0; i < nvar; ++i) bl[j] += G[i * nvar + j] * br[i];
        }
        for (int v = 0; v < nvar; ++v) {
          if (fl)
            direct[(int64_t)v * nc + c] += bl[v];
          else
            Ubar[((c * 3 + e) * nq + k) * nvar + v] += bl[v];
          if (fr) {
            direct[(int64_t)v * nc + n] += br[v];
          } else if (n >= 0) {
            /* the neighbour's point k on this face, stored by physical point */
            int en = M->fedge[3 * c + e];
            Ubar[((n * 3 + en) * nq + (nq - 1 - k)) * nvar + v] += br[v];
          }
        }
      }
    }
  /* adjoint of the reconstruction: P(x) = U0 + sum_l coef_l psi_l(x) */
  for (int64_t i = 0; i < nvar * nc; ++i) vout[i] = direct[i];
  free(direct);
  for (int64_t c = 0; c < nc; ++c) {
    const double* P = M->P + 6 * c;
    double cbar[MAXVAR][MAXM];
    double u0bar[MAXVAR];
    for (int v = 0; v < nvar; ++v) {
      u0bar[v] = 0.0;
      for (int l = 0; l < M->m; ++l) cbar[v][l] = 0.0;
    }
    for (int e = 0; e < 3; ++e) {
      int e1 = (e + 1) % 3;
      double dx = P[2 * e1] - P[2 * e], dy = P[2 * e1 + 1] - P[2 * e + 1];
      for (int k = 0; k < nq; ++k) {
        double x = P[2 * e] + M->gt[k] * dx, y = P[2 * e + 1] + M->gt[k] * dy;
        double psi[MAXM];
        psi_at(M, c, x, y, psi);
        for (int v = 0; v < nvar; ++v) {
          double b = Ubar[((c * 3 + e) * nq + k) * nvar + v];
          u0bar[v] += b;
          for (int l = 0; l < M->m; ++l) cbar[v][l] += b * psi[l];
        }
      }
    }
    const int32_t* st = M->st + (int64_t)ST_TOTAL * c;
    const double* ah = M->ahat[c];
    const double* vo = M->vol[c];
    for (int v = 0; v < nvar; ++v) {
      double* vv = vout + (int64_t)v * nc;
      vv[c] += u0bar[v];
      if (RC[c].sel[v] & 8) {
        for (int k = 0; k < M->ns; ++k) {
          double s = 0.0;
          for (int l = 0; l < M->m; ++l) s += ah[l * M->ns + k] * cbar[v][l];
          vv[st[k]] += vo[k] * s;
          vv[c] -= vo[k] * s;
        }
      } else {
        for (int j = 0; j < KSM; ++j) {
          double wj = RC[c].w[v][j];
          if (wj == 0.0) continue;
          const double* aj = ah + M->m * M->ns + j * MSM * NSM;
          for (int k = 0; k < NSM; ++k) {
            int idx = MAXNS + j * NSM + k;
            double s = 0.0;
            for (int l = 0; l < MSM; ++l) s += aj[l * NSM + k] * wj * cbar[v][l];
            vv[st[idx]] += vo[idx] * s;
            vv[c] -= vo[idx] * s;
          }
        }
      }
    }
  }
  free(Ubar);
  free(RC);
  return E_OK;
}

/* adjoint of one SSP-RK3 step from U^n with step dt: lam_n = (dU^{n+1}/dU^n)^T
 * lam_np1, selection frozen at each stage's state (sel1..3 optional) */
int oracle_rk3_vjp(void* h, const double* Un, double time, double dt, const double* lam_np1,
                   double* lam_n) {
  if (((omesh*)h)->charvar || ((omesh*)h)->scheme || ((omesh*)h)->pp)
    return E_INVAL; /* TENO in conservative variables, no positivity scaling */
  omesh* M = (omesh*)h;
  int64_t N = M->nc * M->nvar;
  double* R = (double*)malloc(sizeof(double) * N);
  double* U1 = (double*)malloc(sizeof(double) * N);
  double* U2 = (double*)malloc(sizeof(double) * N);
  double* l2 = (double*)malloc(sizeof(double) * N);
  double* l1 = (double*)malloc(sizeof(double) * N);
  double* tmp = (double*)malloc(sizeof(double) * N);
  int rc = oracle_residual(h, Un, time, R, NULL, NULL, NULL);
  for (int64_t i = 0; i < N; ++i) U1[i] = Un[i] + dt * R[i];
  if (!rc) rc = oracle_residual(h, U1, time + dt, R, NULL, NULL, NULL);
  for (int64_t i = 0; i < N; ++i) U2[i] = 0.75 * Un[i] + 0.25 * U1[i] + 0.25 * dt * R[i];
  /* stage 3: U^{n+1} = Un/3 + 2/3 U2 + 2/3 dt R(U2) */
  if (!rc) rc = oracle_residual_vjp(h, U2, time + 0.5 * dt, lam_np1, tmp, NULL);
  for (int64_t i = 0; i < N; ++i) {
    l2[i] = 2.0 / 3.0 * lam_np1[i] + 2.0 / 3.0 * dt * tmp[i];
    lam_n[i] = lam_np1[i] / 3.0;
  }
  /* stage 2: U2 = 3/4 Un + 1/4 U1 + 1/4 dt R(U1) */
  if (!rc) rc = oracle_residual_vjp(h, U1, time + dt, l2, tmp, NULL);
  for (int64_t i = 0; i < N; ++i) {
    l1[i] = 0.25 * l2[i] + 0.25 * dt * tmp[i];
    lam_n[i] += 0.75 * l2[i];
  }
  /* stage 1: U1 = Un + dt R(Un) */
  if (!rc) rc = oracle_residual_vjp(h, Un, time, l1, tmp, NULL);
  for (int64_t i = 0; i < N; ++i) lam_n[i] += l1[i] + dt * tmp[i];
  free(R);
  free(U1);
  free(U2);
  free(l2);
  free(l1);
  free(tmp);
  return rc;
}

/* characteristic basis of the Euler flux in direction (nx, ny) at W, for
 * pins: L, R row-major 4x4 */
void oracle_char_basis(void* h, const double* W, double nx, double ny, double* Lout,
                       double* Rout) {
  omesh* M = (omesh*)h;
  double L[4][4], R[4][4];
  char_basis(M->gam, W, nx, ny, L, R);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      Lout[4 * i + j] = L[i][j];
      Rout[4 * i + j] = R[i][j];
    }
}

/* flux access for pins at face point (x, y): F [nvar], JL/JR [nvar*nvar]
 * optional */
void oracle_flux(void* h, const double* UL, const double* UR, double nx, double ny, double x,
                 double y, double* F, double* JL, double* JR) {
  omesh* M = (omesh*)h;
  num_flux(M, UL, UR, nx, ny, x, y, F);
  if (JL && JR) flux_jac(M, UL, UR, nx, ny, x, y, JL, JR);
}

/* face flux K of owner cell c, local edge e (for pins): K [nvar]; the face
 * must be owned by c (a boundary face, or c the smaller id) */
int oracle_face_flux(void* h, const double* U, double time, int64_t c, int e, double* K) {
  omesh* M = (omesh*)h;
  if (c < 0 || c >= M->nc || e < 0 || e > 2 || !is_owner(M, c, e)) return E_INVAL;
  const int64_t n = M->fnbr[3 * c + e];
  int64_t cells[2] = {c, n >= 0 ? n : c};
  int rc = oracle_prepare(h, 2, cells);
  if (rc) return rc;
  M->time = time;
  recon_t Rc, Rn;
  reconstruct(M, c, U, NULL, &Rc);
  if (n >= 0) reconstruct(M, n, U, NULL, &Rn);
  face_flux(M, c, e, U, &Rc, n >= 0 ? &Rn : NULL, K, NULL, NULL);
  return E_OK;
}

/* boundary ghost state at face point (x, y) with outward unit normal
 * (nx, ny) at time t, for pins: UR [nvar] */
void oracle_ghost(void* h, int tag, const double* UL, double nx, double ny, double x, double y,
                  double t, double* UR) {
  omesh* M = (omesh*)h;
  const double t_saved = M->time;
  M->time = t;
  ghost_state(M, tag, UL, nx, ny, x, y, UR);
  M->time = t_saved;
}

void oracle_geometry(void* h, double* area, double* cen, int32_t* fnbr) {
  omesh* M = (omesh*)h;
  memcpy(area, M->area, sizeof(double) * M->nc);
  memcpy(cen, M->cen, sizeof(double) * 2 * M->nc);
  memcpy(fnbr, M->fnbr, sizeof(int32_t) * 3 * M->nc);
}

int oracle_gauss_legendre(int n, double* x, double* w) {
  if (n < 1 || n > 16) return E_INVAL;
  gauss_legendre(n, x, w);
  return E_OK;
}
