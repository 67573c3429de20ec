// teno_kernels.cu -- CUDA kernels of the TENO finite-volume residual for
// sm_103a (GB300).
//
// Per RK stage (Sec. 2.1, Eq. fv_governing_equation_semi_discrete):
//   recon_kernel      stencil differences, coefficient matvecs (Eqs.
//                     reconstruction_08/09 with |V'_s| folded into the
//                     matrices), smoothness indicators (Eq. WENO_smoothness in
//                     a beta-orthonormal basis, so beta = |a'|^2), TENO scale
//                     separation, cutoff and two-step selection (Eqs.
//                     new_scale_separation .. TENO_weight) and evaluation at
//                     the edge Gauss points;
//   face_flux_kernel  rotated HLL / HLLC (Sec. 4) or upwind flux at the Gauss
//                     points of each face, summed with weights and |A|;
//   gather_kernel     cell-centric, atomic-free sum of the three face fluxes
//                     (owner +, neighbour -), fused with the SSP-RK3 stage
//                     combination (Eq. fv_time_discretization_01);
//   max_lambda_kernel warp-shuffle / block reduction of the CFL signal speed.
// Adjoint (no counterpart in the paper): face_flux_vjp_kernel (dual-number
// flux Jacobians), recon_vjp_kernel (transposed matvecs with the selection
// frozen) and scatter_gather_kernel (reverse-stencil gather, no atomics).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "teno_internal.h"

namespace teno {
namespace {

constexpr int kSmallEntries = kSmallK * kSmallN * kSmallM;  // 180
// stencil slots unrolled together in the reconstruction loops (loads of that
// many slots can be in flight per thread)
#ifndef TENO_RECON_UNROLL
#define TENO_RECON_UNROLL 2
#endif
constexpr int kSlotUnroll = TENO_RECON_UNROLL;
// the FP32-mixed kernels keep more slots in flight (4 measured best, 2 for
// the double-float and FP64 kernels)
#ifndef TENO_RECON_UNROLL_MIXED
#define TENO_RECON_UNROLL_MIXED 4
#endif
constexpr int kSlotUnrollMixed = TENO_RECON_UNROLL_MIXED;
constexpr int kSmallSlots = kSmallK * kSmallN;               // 36

template <typename T>
struct TypeTag {
  using type = T;
};

// ---------------------------------------------------------------- scalars
template <typename T>
__device__ __forceinline__ T tsqrt(T x);
template <>
__device__ __forceinline__ double tsqrt<double>(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float tsqrt<float>(float x) { return sqrtf(x); }

// scalar constants of every arithmetic type used by the flux templates
template <typename T>
struct Cst {
  __device__ __forceinline__ static T from(double x) { return T(x); }
};
template <typename T>
__device__ __forceinline__ T cst(double x) {
  return Cst<T>::from(x);
}

// forward-mode dual number with N directions over scalar type S (flux
// Jacobians of the adjoint)
template <int N, typename S = double>
struct Dual {
  S v;
  S d[N];
};
template <int N, typename S>
struct Cst<Dual<N, S>> {
  __device__ __forceinline__ static Dual<N, S> from(double x) {
    Dual<N, S> r;
    r.v = Cst<S>::from(x);
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = Cst<S>::from(0.0);
    return r;
  }
};
template <int N>
__device__ __forceinline__ Dual<N> mk(double v) {
  return Cst<Dual<N>>::from(v);
}
template <int N, typename S>
__device__ __forceinline__ Dual<N, S> operator+(const Dual<N, S>& a, const Dual<N, S>& b) {
  Dual<N, S> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N, typename S>
__device__ __forceinline__ Dual<N, S> operator-(const Dual<N, S>& a, const Dual<N, S>& b) {
  Dual<N, S> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N, typename S>
__device__ __forceinline__ Dual<N, S> operator-(const Dual<N, S>& a) {
  Dual<N, S> r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int N, typename S>
__device__ __forceinline__ Dual<N, S> operator*(const Dual<N, S>& a, const Dual<N, S>& b) {
  Dual<N, S> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int N, typename S>
__device__ __forceinline__ Dual<N, S> operator*(double s, const Dual<N, S>& a) {
  const S ss = Cst<S>::from(s);
  Dual<N, S> r;
  r.v = ss * a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = ss * a.d[i];
  return r;
}
template <int N, typename S>
__device__ __forceinline__ Dual<N, S> operator/(const Dual<N, S>& a, const Dual<N, S>& b) {
  Dual<N, S> r;
  r.v = a.v / b.v;
  const S ib = Cst<S>::from(1.0) / b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
__device__ __forceinline__ double val(double x);
__device__ __forceinline__ float val(float x);
template <int N, typename S>
__device__ __forceinline__ Dual<N, S> tsqrt(const Dual<N, S>& a) {
  Dual<N, S> r;
  r.v = tsqrt(a.v);
  // the root of a zero (a clamped pressure) carries no derivative
  const bool z = val(r.v) == decltype(val(r.v))(0);
  const S h = z ? r.v : Cst<S>::from(0.5) / r.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * h;
  return r;
}
__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ float val(float x) { return x; }
template <int N, typename S>
__device__ __forceinline__ auto val(const Dual<N, S>& x) { return val(x.v); }
// min / max that ignore a NaN operand, like C's fmin / fmax (a wave speed
// from the sound speed of a state whose pressure rounds below zero is NaN;
// the other bound is then taken)
template <typename T>
__device__ __forceinline__ T vmin(const T& a, const T& b) {
  return (val(a) <= val(b) || val(b) != val(b)) ? a : b;
}
template <typename T>
__device__ __forceinline__ bool nonneg(const T& x) { return val(x) >= decltype(val(x))(0); }
template <typename T>
__device__ __forceinline__ T vmax(const T& a, const T& b) {
  return (val(a) >= val(b) || val(b) != val(b)) ? a : b;
}


// ------------------------------------------- double-float (FP32 pair) path
// Values are unevaluated sums hi + lo of two floats (|lo| <= ulp(hi)/2), about
// 48 significant bits: Dekker's double-length arithmetic ("A floating-point
// technique for extending the available precision", 1971) on FP32.  Sums use
// Knuth's two-sum (TAOCP vol. 2, 4.2.2), and Dekker's fast two-sum where the
// operands are ordered; products take the exact residual of a fused
// multiply-add in place of Dekker's splitting; the per-cell matrices are
// stored as (hi, lo) pairs.
// 8-byte aligned so that a pair moves through memory in one access
struct __align__(8) DF {
  float h, l;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
// acc += a * b with a, b pairs; acc.l collects the rounding terms (the pair
// is renormalised by the caller)
__device__ __forceinline__ void df_mac(DF& acc, float2 a, DF b) {
  const float p = a.x * b.h;
  float e = fmaf(a.x, b.h, -p);
  e = fmaf(a.x, b.l, e);
  e = fmaf(a.y, b.h, e);
  const DF s = two_sum(acc.h, p);
  acc.h = s.h;
  acc.l += s.l + e;
}
__device__ __forceinline__ DF df_norm(DF a) { return two_sum(a.h, a.l); }
__device__ __forceinline__ double df_to_double(DF a) { return (double)a.h + (double)a.l; }


// arithmetic on pairs (the Riemann flux of the FP64 path): sums renormalise
// once (Dekker's fast two-sum), products use the exact FMA residual, and
// quotients and square roots take Dekker's one correction step (div2, sqrt2
// of the 1971 paper: the exact remainder of the FP32 approximation, from an
// FMA, divided by the divisor or twice the root)
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ DF operator+(DF a, DF b) {
  DF s = two_sum(a.h, b.h);
  s.l += a.l + b.l;
  return fast_two_sum(s.h, s.l);
}
__device__ __forceinline__ DF operator-(DF a) { return {-a.h, -a.l}; }
__device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }
__device__ __forceinline__ DF operator*(DF a, DF b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return fast_two_sum(p, e);
}
// Quotients: q1 from the correctly rounded reciprocal of b.h (1.5 ulp), the
// exact remainder a - b q1 in pairs, and its quotient by the same reciprocal
// (the correction carries a relative error of about one ulp); square roots:
// the correctly rounded FP32 root and a correction scaled by rsqrt/2.  Build
// with TENO_DF_IEEE_DIV=1 for IEEE FP32 divisions in both steps instead.
#ifndef TENO_DF_IEEE_DIV
#define TENO_DF_IEEE_DIV 0
#endif
// TENO_DF_APPROX=1 (default): start from the PTX approximate reciprocal and
// square root (relative error about 2^-22 each) instead of the correctly
// rounded ones; the one exact-remainder correction squares that error, so
// the pair results keep their ~2^-44 relative accuracy (face flux 3 %, flux
// VJP 5 % faster than with the correctly rounded starts).
#ifndef TENO_DF_APPROX
#define TENO_DF_APPROX 1
#endif
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ DF operator/(DF a, DF b) {
#if TENO_DF_IEEE_DIV
  const float q1 = a.h / b.h;
  const DF r = a - b * DF{q1, 0.f};
  return fast_two_sum(q1, r.h / b.h);
#else
#if TENO_DF_APPROX
  const float rb = rcp_approx(b.h);
#else
  const float rb = __frcp_rn(b.h);
#endif
  const float q1 = a.h * rb;
  const DF r = a - b * DF{q1, 0.f};
  return fast_two_sum(q1, r.h * rb);
#endif
}
__device__ __forceinline__ DF tsqrt(DF a) {
#if TENO_DF_APPROX && !TENO_DF_IEEE_DIV
  const float s = sqrt_approx(a.h);
#else
  const float s = sqrtf(a.h);
#endif
  if (!(a.h > 0.f)) return {s, 0.f};
  const DF r = a - DF{s, 0.f} * DF{s, 0.f};
#if TENO_DF_IEEE_DIV
  return fast_two_sum(s, r.h / (2.f * s));
#else
  return fast_two_sum(s, r.h * (0.5f * rsqrtf(a.h)));
#endif
}
__device__ __forceinline__ float val(DF x) { return x.h; }
template <>
struct Cst<DF> {
  __device__ __forceinline__ static DF from(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
  }
};
__device__ __forceinline__ DF vmin(const DF& a, const DF& b) {
  return (a.h < b.h || (a.h == b.h && a.l <= b.l) || b.h != b.h) ? a : b;
}
__device__ __forceinline__ DF vmax(const DF& a, const DF& b) {
  return (a.h > b.h || (a.h == b.h && a.l >= b.l) || b.h != b.h) ? a : b;
}
// c + a*b and conversion to FP64 for every scalar type of the flux kernels
// exact zero test (pairs: both parts; dual numbers: the value)
__device__ __forceinline__ bool is_zero(double x) { return x == 0.0; }
__device__ __forceinline__ bool is_zero(float x) { return x == 0.0f; }
__device__ __forceinline__ bool is_zero(DF x) { return x.h == 0.0f && x.l == 0.0f; }
template <int N, typename S>
__device__ __forceinline__ bool is_zero(const Dual<N, S>& x) { return is_zero(x.v); }

__device__ __forceinline__ double madd(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float madd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ DF madd(DF a, DF b, DF c) { return a * b + c; }
__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return (double)x; }
__device__ __forceinline__ double to_d(DF x) { return (double)x.h + (double)x.l; }
// a stored Gauss-point value as the flux scalar type
template <typename S>
__device__ __forceinline__ S lift(double x) { return Cst<S>::from(x); }
template <typename S>
__device__ __forceinline__ S lift(float x) { return Cst<S>::from((double)x); }
template <typename S>
__device__ __forceinline__ S lift(DF x) {
  if constexpr (std::is_same<S, DF>::value)
    return x;
  else
    return S(to_d(x));
}
// branch decisions on dual numbers over pairs compare the (normalised) pairs
// lexicographically, which orders them as their exact sums; no conversion to
// FP64 on the device
__device__ __forceinline__ bool df_le(const DF& a, const DF& b) {
  return a.h < b.h || (a.h == b.h && a.l <= b.l);
}
template <int N>
__device__ __forceinline__ Dual<N, DF> vmin(const Dual<N, DF>& a, const Dual<N, DF>& b) {
  return (df_le(a.v, b.v) || b.v.h != b.v.h) ? a : b;
}
template <int N>
__device__ __forceinline__ Dual<N, DF> vmax(const Dual<N, DF>& a, const Dual<N, DF>& b) {
  return (df_le(b.v, a.v) || b.v.h != b.v.h) ? a : b;
}
template <int N>
__device__ __forceinline__ bool nonneg(const Dual<N, DF>& x) {
  return x.v.h > 0.f || (x.v.h == 0.f && x.v.l >= 0.f);
}
// a pressure in a side sound speed: negative values as zero, NaN kept.  A
// Gauss state at the positivity floor has a pressure about 1e-15 of its
// energy, below the resolution of the pair and FP32 evaluations; its sound
// speed is then zero, so the wave-speed bound is the particle speed and not
// the Roe bound alone.
template <typename T>
__device__ __forceinline__ T pos_part(const T& x) {
  return (nonneg(x) || val(x) != val(x)) ? x : x - x;
}

// ---------------------------------------------------------------- fluxes
// Euler flux through a face with unit normal n = (nx, ny): the state is
// expressed in the face frame (normal, tangential velocity), the 1D flux
// F^x is evaluated there and rotated back (Sec. 4.1, F^n = T^-1 F^x(T U)).
// constants of one face in the flux scalar type, converted once per face
template <typename T>
struct RiemannK {
  T one, half, gm1, gg, tnx, tny;
};
template <typename T>
__device__ __forceinline__ RiemannK<T> riemann_k(double nx, double ny, double g) {
  return {cst<T>(1.0), cst<T>(0.5), cst<T>(g - 1.0), cst<T>(g), cst<T>(nx), cst<T>(ny)};
}
// the same constants as dual numbers (zero derivatives; no conversion)
template <int N, typename S>
__device__ __forceinline__ RiemannK<Dual<N, S>> riemann_k_dual(const RiemannK<S>& k) {
  auto c = [](S x) {
    Dual<N, S> r = cst<Dual<N, S>>(0.0);
    r.v = x;
    return r;
  };
  return {c(k.one), c(k.half), c(k.gm1), c(k.gg), c(k.tnx), c(k.tny)};
}

template <typename T>
__device__ __forceinline__ void euler_riemann(const T* UL, const T* UR, const RiemannK<T>& K,
                                              int hllc, T* F) {
  const T one = K.one, half = K.half;
  const T gm1 = K.gm1, gg = K.gg;
  const T tnx = K.tnx, tny = K.tny;
  // left / right primitive variables in the face frame (one reciprocal per
  // density; every division below is by one of four reciprocals)
  T rL = UL[0], rR = UR[0];
  T irL = one / rL, irR = one / rR;
  T unL = (UL[1] * tnx + UL[2] * tny) * irL;
  T utL = (UL[2] * tnx - UL[1] * tny) * irL;
  T unR = (UR[1] * tnx + UR[2] * tny) * irR;
  T utR = (UR[2] * tnx - UR[1] * tny) * irR;
  T EL = UL[3], ER = UR[3];
  T pL = gm1 * (EL - half * rL * (unL * unL + utL * utL));
  T pR = gm1 * (ER - half * rR * (unR * unR + utR * utR));
  T cL = tsqrt(gg * pos_part(pL) * irL), cR = tsqrt(gg * pos_part(pR) * irR);
  T HL = (EL + pL) * irL, HR = (ER + pR) * irR;
  // Roe averages and Einfeldt wave speeds (Eq. wavespeed)
  T D = tsqrt(rR * irL);
  T iden = one / (one + D);
  T ua = (unL + unR * D) * iden;
  T va = (utL + utR * D) * iden;
  T Ha = (HL + HR * D) * iden;
  T ca = tsqrt(gm1 * (Ha - half * (ua * ua + va * va)));
  T SL = vmin(unL - cL, ua - ca);
  T SR = vmax(unR + cR, ua + ca);
  // 1D fluxes and conserved states in the face frame
  T mL = rL * unL, mR = rR * unR;
  T FL[4] = {mL, mL * unL + pL, mL * utL, unL * (EL + pL)};
  T FR[4] = {mR, mR * unR + pR, mR * utR, unR * (ER + pR)};
  T WL[4] = {rL, mL, rL * utL, EL};
  T WR[4] = {rR, mR, rR * utR, ER};
  T Fx[4];
  // HLLC's contact speed divides by aL - aR, zero only when both wave-speed
  // bounds equal the particle speeds (zero sound speed on both sides, e.g. a
  // wall Gauss state at zero pressure): the flux there is HLL's
  const T aL = rL * (SL - unL), aR = rR * (SR - unR);
  const T Dn = aL - aR;
  if (nonneg(SL)) {
#pragma unroll
    for (int k = 0; k < 4; ++k) Fx[k] = FL[k];
  } else if (nonneg(-SR)) {
#pragma unroll
    for (int k = 0; k < 4; ++k) Fx[k] = FR[k];
  } else if (!hllc || is_zero(Dn)) {
    T inv = one / (SR - SL);
    T sLR = SL * SR;
#pragma unroll
    for (int k = 0; k < 4; ++k) Fx[k] = (SR * FL[k] - SL * FR[k] + sLR * (WR[k] - WL[k])) * inv;
  } else {
    // HLLC: contact speed and star state of the side the face lies in; the
    // star energy f (E/r + (Ss - un)(Ss + p / (r (S - un)))) multiplied out,
    // so that nothing divides by S - un
    T Ss = (pR - pL + aL * unL - aR * unR) / Dn;
    bool left = nonneg(Ss);
    T r = left ? rL : rR, un = left ? unL : unR, ut = left ? utL : utR;
    T p = left ? pL : pR, S = left ? SL : SR, E = left ? EL : ER;
    T Smu = S - un, inv = one / (S - Ss);
    T gq = r * Smu;
    T f = gq * inv;
    T es = (Smu * E + (Ss - un) * (gq * Ss + p)) * inv;
    T Us[4] = {f, f * Ss, f * ut, es};
#pragma unroll
    for (int k = 0; k < 4; ++k) Fx[k] = (left ? FL[k] : FR[k]) + S * (Us[k] - (left ? WL[k] : WR[k]));
  }
  F[0] = Fx[0];
  F[1] = Fx[1] * tnx - Fx[2] * tny;
  F[2] = Fx[1] * tny + Fx[2] * tnx;
  F[3] = Fx[3];
}

// normal advection speed of the scalar equation at face point (x, y): the
// constant velocity, or the rigid rotation omega phi(r) (-(y - y_c), x - x_c)
// of the solid-body case (Sec. 5) with the smoothstep taper phi from 1 at r1
// to 0 at r2 (none when r2 <= r1)
__device__ __forceinline__ double adv_normal(int field, double ax, double ay, double cx,
                                             double cy, double om, double r1, double r2,
                                             double x, double y, double nx, double ny) {
  if (field == 1) {
    const double dx = x - cx, dy = y - cy;
    double phi = 1.0;
    if (r2 > r1) {
      const double r = sqrt(dx * dx + dy * dy);
      if (r >= r2) {
        phi = 0.0;
      } else if (r > r1) {
        const double s = (r - r1) / (r2 - r1);
        phi = 1.0 - s * s * (3.0 - 2.0 * s);
      }
    }
    return om * phi * (-dy * nx + dx * ny);
  }
  return ax * nx + ay * ny;
}

// a <= b in the order the forward solver's min/max use (pairs: lexicographic)
template <typename T>
__device__ __forceinline__ bool le_ord(const T& a, const T& b) {
  if constexpr (std::is_same<T, DF>::value)
    return a.h < b.h || (a.h == b.h && a.l <= b.l);
  else
    return a <= b;
}

// Reverse mode of euler_riemann: given Fb = dJ/dF (face frame rotated back,
// the kernel's output frame), adds (dF/dU_L)^T Fb to ULb and (dF/dU_R)^T Fb
// to URb, with every branch (wave-speed min/max, HLL/HLLC region, HLLC side)
// frozen at the forward state.  The forward values are recomputed first;
// the adjoint statements then run in reverse order of the forward ones.
template <typename T>
__device__ __forceinline__ void euler_riemann_vjp(const T* UL, const T* UR, const RiemannK<T>& K,
                                                  int hllc, const T* Fb, T* ULb, T* URb) {
  const T one = K.one, half = K.half, two = K.one + K.one;
  const T gm1 = K.gm1, gg = K.gg, tnx = K.tnx, tny = K.tny;
  const T zero = one - one;
  // ---- forward
  const T rL = UL[0], rR = UR[0];
  const T irL = one / rL, irR = one / rR;
  const T mnL = UL[1] * tnx + UL[2] * tny, mtL = UL[2] * tnx - UL[1] * tny;
  const T mnR = UR[1] * tnx + UR[2] * tny, mtR = UR[2] * tnx - UR[1] * tny;
  const T unL = mnL * irL, utL = mtL * irL, unR = mnR * irR, utR = mtR * irR;
  const T EL = UL[3], ER = UR[3];
  const T qL = unL * unL + utL * utL, qR = unR * unR + utR * utR;
  const T pL = gm1 * (EL - half * rL * qL), pR = gm1 * (ER - half * rR * qR);
  const T cL = tsqrt(gg * pos_part(pL) * irL), cR = tsqrt(gg * pos_part(pR) * irR);
  const T HL = (EL + pL) * irL, HR = (ER + pR) * irR;
  const T D = tsqrt(rR * irL);
  const T iden = one / (one + D);
  const T ua = (unL + unR * D) * iden, va = (utL + utR * D) * iden;
  const T Ha = (HL + HR * D) * iden;
  const T ca = tsqrt(gm1 * (Ha - half * (ua * ua + va * va)));
  // the branches vmin / vmax take in the forward solver (NaN operands ignored)
  const T am = ua - ca, ap = ua + ca;
  const bool sl0 = le_ord(unL - cL, am) || val(am) != val(am);  // SL from the left state
  const bool sr0 = le_ord(ap, unR + cR) || val(ap) != val(ap);  // SR from the right state
  const T SL = sl0 ? unL - cL : ua - ca;
  const T SR = sr0 ? unR + cR : ua + ca;
  const T mL = rL * unL, mR = rR * unR;
  const T FL[4] = {mL, mL * unL + pL, mL * utL, unL * (EL + pL)};
  const T FR[4] = {mR, mR * unR + pR, mR * utR, unR * (ER + pR)};
  const T WL[4] = {rL, mL, rL * utL, EL};
  const T WR[4] = {rR, mR, rR * utR, ER};
  // ---- reverse
  T Fxb[4];
  Fxb[0] = Fb[0];
  Fxb[1] = Fb[1] * tnx + Fb[2] * tny;
  Fxb[2] = Fb[2] * tnx - Fb[1] * tny;
  Fxb[3] = Fb[3];
  T FLb[4], FRb[4], WLb[4], WRb[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) FLb[k] = FRb[k] = WLb[k] = WRb[k] = zero;
  T SLb = zero, SRb = zero;
  T rLb = zero, rRb = zero, unLb = zero, unRb = zero, utLb = zero, utRb = zero;
  T pLb = zero, pRb = zero, ELb = zero, ERb = zero;
  const bool hll = !hllc || is_zero(rL * (SL - unL) - rR * (SR - unR));
  if (nonneg(SL)) {
#pragma unroll
    for (int k = 0; k < 4; ++k) FLb[k] = Fxb[k];
  } else if (nonneg(-SR)) {
#pragma unroll
    for (int k = 0; k < 4; ++k) FRb[k] = Fxb[k];
  } else if (hll) {
    const T inv = one / (SR - SL), sLR = SL * SR;
    T invb = zero, sLRb = zero;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const T G = SR * FL[k] - SL * FR[k] + sLR * (WR[k] - WL[k]);
      invb = invb + Fxb[k] * G;
      const T Gb = Fxb[k] * inv;
      FLb[k] = Gb * SR;
      FRb[k] = zero - Gb * SL;
      WRb[k] = Gb * sLR;
      WLb[k] = zero - Gb * sLR;
      SRb = SRb + Gb * FL[k];
      SLb = SLb - Gb * FR[k];
      sLRb = sLRb + Gb * (WR[k] - WL[k]);
    }
    SRb = SRb + sLRb * SL;
    SLb = SLb + sLRb * SR;
    const T db = zero - invb * inv * inv;  // d(SR - SL)
    SRb = SRb + db;
    SLb = SLb - db;
  } else {
    const T aL = rL * (SL - unL), aR = rR * (SR - unR);
    const T Nn = pR - pL + aL * unL - aR * unR, Dn = aL - aR;
    const T Ss = Nn / Dn;
    const bool left = nonneg(Ss);
    const T r = left ? rL : rR, un = left ? unL : unR, ut = left ? utL : utR;
    const T p = left ? pL : pR, S = left ? SL : SR, E = left ? EL : ER;
    const T Smu = S - un, gq = r * Smu, den = S - Ss;
    const T f = gq / den;
    const T qs = gq * Ss + p;
    const T es = (Smu * E + (Ss - un) * qs) / den;
    const T Us[4] = {f, f * Ss, f * ut, es};
    const T* Wsd = left ? WL : WR;
    T Sb = zero, Ssb = zero, rb = zero, unb = zero, utb = zero, pb = zero, Eb = zero;
    T Usb[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      Sb = Sb + Fxb[k] * (Us[k] - Wsd[k]);
      Usb[k] = S * Fxb[k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (left) {
        FLb[k] = Fxb[k];
        WLb[k] = zero - S * Fxb[k];
      } else {
        FRb[k] = Fxb[k];
        WRb[k] = zero - S * Fxb[k];
      }
    }
    // Us = (f, f Ss, f ut, es)
    const T fb = Usb[0] + Usb[1] * Ss + Usb[2] * ut;
    Ssb = Ssb + Usb[1] * f;
    utb = utb + Usb[2] * f;
    const T esb = Usb[3];
    // es = (Smu E + (Ss - un) qs) / den, qs = gq Ss + p
    const T numb = esb / den;
    T denb = zero - esb * es / den;
    T Smub = numb * E;
    Eb = Eb + numb * Smu;
    Ssb = Ssb + numb * qs;
    unb = unb - numb * qs;
    const T qsb = numb * (Ss - un);
    T gqb = qsb * Ss;
    Ssb = Ssb + qsb * gq;
    pb = pb + qsb;
    // f = gq / den, den = S - Ss, gq = r Smu, Smu = S - un
    gqb = gqb + fb / den;
    denb = denb - fb * f / den;
    Sb = Sb + denb;
    Ssb = Ssb - denb;
    rb = rb + gqb * Smu;
    Smub = Smub + gqb * r;
    Sb = Sb + Smub;
    unb = unb - Smub;
    // Ss = Nn / Dn, Nn = pR - pL + aL unL - aR unR, Dn = aL - aR
    const T Nb = Ssb / Dn, Dnb = zero - Ssb * Ss / Dn;
    pRb = pRb + Nb;
    pLb = pLb - Nb;
    const T aLb = Nb * unL + Dnb, aRb = zero - Nb * unR - Dnb;
    unLb = unLb + Nb * aL;
    unRb = unRb - Nb * aR;
    // aL = rL (SL - unL), aR = rR (SR - unR)
    rLb = rLb + aLb * (SL - unL);
    SLb = SLb + aLb * rL;
    unLb = unLb - aLb * rL;
    rRb = rRb + aRb * (SR - unR);
    SRb = SRb + aRb * rR;
    unRb = unRb - aRb * rR;
    // the chosen side's variables
    if (left) {
      rLb = rLb + rb; unLb = unLb + unb; utLb = utLb + utb; pLb = pLb + pb; SLb = SLb + Sb;
      ELb = ELb + Eb;
    } else {
      rRb = rRb + rb; unRb = unRb + unb; utRb = utRb + utb; pRb = pRb + pb; SRb = SRb + Sb;
      ERb = ERb + Eb;
    }
  }
  // wave speeds (frozen min / max branches)
  T uab = zero, cab = zero, cLb = zero, cRb = zero;
  if (sl0) {
    unLb = unLb + SLb;
    cLb = cLb - SLb;
  } else {
    uab = uab + SLb;
    cab = cab - SLb;
  }
  if (sr0) {
    unRb = unRb + SRb;
    cRb = cRb + SRb;
  } else {
    uab = uab + SRb;
    cab = cab + SRb;
  }
  // F and W of both sides
  {
    const T mLb = FLb[0] + FLb[1] * unL + FLb[2] * utL + WLb[1];
    unLb = unLb + FLb[1] * mL + FLb[3] * (EL + pL) + mLb * rL;
    pLb = pLb + FLb[1] + FLb[3] * unL;
    utLb = utLb + FLb[2] * mL + WLb[2] * rL;
    ELb = ELb + FLb[3] * unL + WLb[3];
    rLb = rLb + WLb[0] + WLb[2] * utL + mLb * unL;
    const T mRb = FRb[0] + FRb[1] * unR + FRb[2] * utR + WRb[1];
    unRb = unRb + FRb[1] * mR + FRb[3] * (ER + pR) + mRb * rR;
    pRb = pRb + FRb[1] + FRb[3] * unR;
    utRb = utRb + FRb[2] * mR + WRb[2] * rR;
    ERb = ERb + FRb[3] * unR + WRb[3];
    rRb = rRb + WRb[0] + WRb[2] * utR + mRb * unR;
  }
  // Roe averages: ca = sqrt(gm1 (Ha - (ua^2 + va^2)/2)), ua, va, Ha, iden, D
  const T ca2b = cab / (two * ca);
  const T Hab = ca2b * gm1;
  uab = uab - ca2b * gm1 * ua;
  const T vab = zero - ca2b * gm1 * va;
  unLb = unLb + uab * iden;
  unRb = unRb + uab * D * iden;
  utLb = utLb + vab * iden;
  utRb = utRb + vab * D * iden;
  T HLb = Hab * iden, HRb = Hab * D * iden;
  const T idenb = uab * (unL + unR * D) + vab * (utL + utR * D) + Hab * (HL + HR * D);
  const T Db = uab * unR * iden + vab * utR * iden + Hab * HR * iden - idenb * iden * iden;
  const T rrb = Db / (two * D);  // d(rR irL)
  rRb = rRb + rrb * irL;
  T irLb = rrb * rR, irRb = zero;
  // H, c, p, q, u of both sides
  ELb = ELb + HLb * irL;
  pLb = pLb + HLb * irL;
  irLb = irLb + HLb * (EL + pL);
  ERb = ERb + HRb * irR;
  pRb = pRb + HRb * irR;
  irRb = irRb + HRb * (ER + pR);
  {
    // a zero sound speed (clamped or zero pressure) passes nothing back
    const T c2b = is_zero(cL) ? zero : cLb / (two * cL);
    pLb = pLb + c2b * gg * irL;
    irLb = irLb + c2b * gg * pL;
    const T c2bR = is_zero(cR) ? zero : cRb / (two * cR);
    pRb = pRb + c2bR * gg * irR;
    irRb = irRb + c2bR * gg * pR;
  }
  ELb = ELb + pLb * gm1;
  rLb = rLb - pLb * gm1 * half * qL;
  const T qLb = zero - pLb * gm1 * half * rL;
  ERb = ERb + pRb * gm1;
  rRb = rRb - pRb * gm1 * half * qR;
  const T qRb = zero - pRb * gm1 * half * rR;
  unLb = unLb + two * qLb * unL;
  utLb = utLb + two * qLb * utL;
  unRb = unRb + two * qRb * unR;
  utRb = utRb + two * qRb * utR;
  const T mnLb = unLb * irL, mtLb = utLb * irL, mnRb = unRb * irR, mtRb = utRb * irR;
  irLb = irLb + unLb * mnL + utLb * mtL;
  irRb = irRb + unRb * mnR + utRb * mtR;
  rLb = rLb - irLb * irL * irL;
  rRb = rRb - irRb * irR * irR;
  ULb[0] = ULb[0] + rLb;
  ULb[1] = ULb[1] + mnLb * tnx - mtLb * tny;
  ULb[2] = ULb[2] + mnLb * tny + mtLb * tnx;
  ULb[3] = ULb[3] + ELb;
  URb[0] = URb[0] + rRb;
  URb[1] = URb[1] + mnRb * tnx - mtRb * tny;
  URb[2] = URb[2] + mnRb * tny + mtRb * tnx;
  URb[3] = URb[3] + ERb;
}

// (dU_R/dU_L)^T URb added to ULb for the ghost state of a boundary point:
// mirror at a wall, identity at an outflow, constant at inflow and top
template <typename T>
__device__ __forceinline__ void ghost_vjp(int tag, const RiemannK<T>& K, const T* URb, T* ULb) {
  if (tag == TENO_BC_WALL) {
    const T two = K.one + K.one;
    const T mnb = (URb[1] * K.tnx + URb[2] * K.tny) * two;
    ULb[0] = ULb[0] + URb[0];
    ULb[1] = ULb[1] + URb[1] - mnb * K.tnx;
    ULb[2] = ULb[2] + URb[2] - mnb * K.tny;
    ULb[3] = ULb[3] + URb[3];
  } else if (tag == TENO_BC_OUTFLOW) {
#pragma unroll
    for (int k = 0; k < 4; ++k) ULb[k] = ULb[k] + URb[k];
  }
}

// ghost state of a boundary face point (tag: enum teno_bc)
template <typename T>
__device__ __forceinline__ void ghost_state(int tag, const T* UL, double nx, double ny, double x,
                                            double time, double g, T* UR) {
  if (tag == TENO_BC_WALL) {
    T mn = UL[1] * cst<T>(nx) + UL[2] * cst<T>(ny);
    UR[0] = UL[0];
    UR[1] = UL[1] - cst<T>(2.0 * nx) * mn;
    UR[2] = UL[2] - cst<T>(2.0 * ny) * mn;
    UR[3] = UL[3];
    return;
  }
  bool post = tag == TENO_BC_INFLOW;
  if (tag == TENO_BC_TOP) post = x < 0.1667 + (1.0 + 20.0 * time) / 1.732;
  if (tag == TENO_BC_INFLOW || tag == TENO_BC_TOP) {
    double r = post ? 8.0 : 1.4, u = post ? 7.145 : 0.0, v = post ? -4.125 : 0.0;
    double p = post ? 116.8333 : 1.0;
    UR[0] = cst<T>(r);
    UR[1] = cst<T>(r * u);
    UR[2] = cst<T>(r * v);
    UR[3] = cst<T>(p / (g - 1.0) + 0.5 * r * (u * u + v * v));
    return;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) UR[k] = UL[k];
}

struct ReconArgs {
  const void* ahat;
  const int32_t* nbr;
  const uint8_t* smask;
  const double* U;
  const float2* Us;  // FP32 hi/lo split of U (mixed precision), [n_var][n_pad]
  void* Uq;
  uint8_t* sel_out;
  const uint8_t* sel_in;
  int64_t n_cell, n_pad;
  double ct, eps;
  int linear, e_entries;
  int scheme;   // 0 TENO, 1 CWENO
  double cw_dK; // CWENO d_K = 1 - 1/d'_K
  double* coef_out;  // characteristic mode: [n_pad][4][m + 15] coefficients out
  int force_near;       // W form: every cell decides through the pair / FP64 fallback
  uint32_t wait_polls;  // bulk-copy kernels: consumer mbarrier poll limit (0: give up at once)
};

// characteristic mode: store the cell's large and directional coefficients of
// variable v for the characteristic finish, in place of selection and
// evaluation: FP64 on the native path, (hi, lo) FP32 pairs on the pair and
// mixed paths (whose finish runs in pair arithmetic on the FP32 pipe)
template <int M, typename TC>
__device__ __forceinline__ void store_coefs(const ReconArgs& a, int64_t c, int v, const TC* acc,
                                            const TC (&as)[kSmallK][kSmallM]) {
  const int64_t base = ((int64_t)c * 4 + v) * (M + kSmallK * kSmallM);
  if constexpr (std::is_same<TC, double>::value) {
    double* o = a.coef_out + base;
#pragma unroll
    for (int l = 0; l < M; ++l) o[l] = acc[l];
#pragma unroll
    for (int k = 0; k < kSmallK; ++k)
#pragma unroll
      for (int l = 0; l < kSmallM; ++l) o[M + k * kSmallM + l] = as[k][l];
  } else {
    float2* o = reinterpret_cast<float2*>(a.coef_out) + base;
    auto pr = [](const TC& x) {
      if constexpr (std::is_same<TC, DF>::value)
        return make_float2(x.h, x.l);
      else
        return make_float2(x, 0.f);
    };
#pragma unroll
    for (int l = 0; l < M; ++l) o[l] = pr(acc[l]);
#pragma unroll
    for (int k = 0; k < kSmallK; ++k)
#pragma unroll
      for (int l = 0; l < kSmallM; ++l) o[M + k * kSmallM + l] = pr(as[k][l]);
  }
  if (a.sel_out) a.sel_out[(int64_t)v * a.n_pad + c] = 8;
}

// CWENO weights (Eqs. CWENOweight, CWENOOptimalLinearweight/02) from the
// smoothness indicators: alpha = d / (beta + eps)^4 with d_K = cw_dK and
// d_k = (1 - d_K)/K over the K present directional stencils; returns the
// factors of P = sK P_K + sum_k s[k] P_k, i.e. sK = w_K / d_K and
// s[k] = w_k - sK d_k (0 for absent stencils).
struct CwenoF {
  double sK, s[kSmallK];
};
// out of line: the CWENO option must not raise the register count of the
// TENO reconstruction kernels that share the finish code
__device__ __noinline__ CwenoF cweno_factors(double b0, double b1, double b2, double bK,
                                             int present, double dK_in, double eps) {
  const double beta[kSmallK + 1] = {b0, b1, b2, bK};
  CwenoF out;
  double& sK = out.sK;
  double* s = out.s;
  const int K = (present & 1) + ((present >> 1) & 1) + ((present >> 2) & 1);
  const double dK = K ? dK_in : 1.0, dk = K ? (1.0 - dK) / K : 0.0;
  double al[kSmallK + 1], sum = 0.0;
#pragma unroll
  for (int k = 0; k <= kSmallK; ++k) {
    const bool pr = k == kSmallK || ((present >> k) & 1);
    const double ib = 1.0 / (beta[k] + eps);
    const double i2 = ib * ib;
    al[k] = pr ? (k == kSmallK ? dK : dk) * (i2 * i2) : 0.0;
    sum += al[k];
  }
  sK = al[kSmallK] / sum / dK;
#pragma unroll
  for (int k = 0; k < kSmallK; ++k) s[k] = ((present >> k) & 1) ? al[k] / sum - sK * dk : 0.0;
  return out;
}

// TENO cutoff and two-step selection in FP64 (Eqs. new_scale_separation,
// normalize, cutoff, TENO_reconstruction111/222): chi_k >= C_T is evaluated as
// gamma_k >= C_T * sum_j gamma_j with gamma = (beta + eps)^-6.
__device__ __forceinline__ uint8_t select_fp64(const double* beta, int present, double ct,
                                               double eps) {
  double g[kSmallK + 1], S = 0.0;
#pragma unroll
  for (int k = 0; k <= kSmallK; ++k) {
    bool pr = k == kSmallK || ((present >> k) & 1);
    double ib = 1.0 / (beta[k] + eps);
    double i2 = ib * ib;
    g[k] = pr ? i2 * i2 * i2 : 0.0;
    S += g[k];
  }
  if (g[kSmallK] >= ct * S) return 8;
  double S2 = g[0] + g[1] + g[2];
  uint8_t sel = 0;
#pragma unroll
  for (int k = 0; k < kSmallK; ++k)
    if (((present >> k) & 1) && g[k] >= ct * S2) sel |= (uint8_t)(1u << k);
  return sel;
}

// FP32 evaluation of chi_k = 1 / sum_j ((beta_k+eps)/(beta_j+eps))^6 over the
// stencils in `mask`; *near is set when chi_k lies within the guard band
// 1e-3 C_T of C_T.  The FP32 betas are within 1.3e-6 (relative) of the FP64
// sums of the same squares, which moves chi by less than 3e-5 relative, so a
// decision outside the band equals the FP64 decision.
__device__ __forceinline__ bool chi_keep32(const float* t, int k, int mask, float ct, bool* near,
                                           float band = 1e-3f) {
  float s = 0.f;
#pragma unroll
  for (int j = 0; j <= kSmallK; ++j) {
    if (!((mask >> j) & 1)) continue;
    float r = t[k] / t[j];
    float r2 = r * r;
    s += r2 * r2 * r2;
  }
  float chi = 1.f / s;
  if (!(fabsf(chi - ct) > band * ct)) *near = true;
  return chi >= ct;
}

// As chi_keep32, for smoothness indicators known only to within a relative
// bound rho each (t_j = beta_j + eps in [t32_j / (1 + rho), t32_j / (1 - rho)]
// or tighter): every ratio t_k / t_j then lies within a factor
// (1 + rho) / (1 - rho) of its FP32 value, so chi lies within the factor
// f = ((1 + rho) / (1 - rho))^6 of the FP32 chi (times 1 + 1e-4 for the FP32
// evaluation itself); *near is set when that interval contains C_T.
__device__ __forceinline__ bool chi_keep32_bound(const float* t, int k, int mask, float ct,
                                                 float f, bool* near) {
  float s = 0.f;
#pragma unroll
  for (int j = 0; j <= kSmallK; ++j) {
    if (!((mask >> j) & 1)) continue;
    float r = t[k] / t[j];
    float r2 = r * r;
    s += r2 * r2 * r2;
  }
  const float chi = 1.f / s;
  if (!(chi > ct * f) && !(chi * f < ct)) *near = true;
  return chi >= ct;
}

// ------------------------------------------------------------ reconstruction
// thread (lane, v, z): cell tile*32 + lane, variable v.  A warp covers the 32
// cells of one tile for one variable, so every matrix entry is one coalesced
// 128/256-byte row; the other variables' warps hit it in L1.
// TA = double: the FP64 path.  TA = float: the mixed path -- stencil
// differences from the hi/lo FP32 split of U (as accurate as an FP64
// subtraction rounded to FP32), FP32 matvecs, FP32 beta and cutoff with an FP64
// fallback inside the guard band, FP32 Gauss-point values.
// selection, final coefficients and Gauss-point values of cell c, variable v
// (FP64-native and FP32-mixed paths)
// kExt: compile the CWENO and characteristic-mode branches (the TENO-only
// instantiations keep the register count of the default kernels down)
template <int M, int NQ, int NV, typename TA, typename TT, bool kExt = true>
__device__ __forceinline__ void plain_finish(const ReconArgs& a, const TT& ev, int64_t c, int v,
                                             double u0, float2 u0s, const TA (&acc)[M],
                                             const TA (&as)[kSmallK][kSmallM],
                                             TA* ostage = nullptr, int present_in = -1) {
  constexpr bool kMixed = std::is_same<TA, float>::value;
  if constexpr (kExt) {
    if (a.coef_out) {
      store_coefs<M, TA>(a, c, v, acc, as);
      return;
    }
  }
  const int present = present_in >= 0 ? present_in : a.smask[c];
  uint8_t sel;
  const bool cweno = kExt && a.scheme == 1 && !a.linear;
  TA cf[M];
  if (cweno) {
    // beta and weights in FP64 (from the FP32 coefficients on the mixed path)
    double beta[kSmallK + 1];
    double b = 0.0;
#pragma unroll
    for (int l = 0; l < M; ++l) b = fma((double)acc[l], (double)acc[l], b);
    beta[kSmallK] = b;
#pragma unroll
    for (int k = 0; k < kSmallK; ++k) {
      double q = 0.0;
#pragma unroll
      for (int l = 0; l < kSmallM; ++l) q = fma((double)as[k][l], (double)as[k][l], q);
      beta[k] = q;
    }
    const CwenoF cw = cweno_factors(beta[0], beta[1], beta[2], beta[kSmallK], present, a.cw_dK,
                                    a.eps);
    const double sK = cw.sK;
    const double* sk = cw.s;
#pragma unroll
    for (int l = 0; l < M; ++l) cf[l] = TA(sK) * acc[l];
#pragma unroll
    for (int k = 0; k < kSmallK; ++k)
#pragma unroll
      for (int l = 0; l < kSmallM; ++l) cf[l] = fma(TA(sk[k]), as[k][l], cf[l]);
    sel = 8;
  } else if (a.sel_in) {
    sel = a.sel_in[(int64_t)v * a.n_pad + c];
  } else if (a.linear) {
    sel = 8;
  } else {
    bool exact = !kMixed;
    if constexpr (kMixed) {
      // FP32 smoothness indicators (orthonormal basis: beta = |a'|^2) and cutoff
      float t[kSmallK + 1];
      {
        float b = 0.f;
#pragma unroll
        for (int l = 0; l < M; ++l) b = fmaf(acc[l], acc[l], b);
        t[kSmallK] = b + (float)a.eps;
#pragma unroll
        for (int k = 0; k < kSmallK; ++k) {
          float q = 0.f;
#pragma unroll
          for (int l = 0; l < kSmallM; ++l) q = fmaf(as[k][l], as[k][l], q);
          t[k] = q + (float)a.eps;
        }
      }
      const float ct = (float)a.ct;
      bool near = false;
      const int all = present | 8;
      if (chi_keep32(t, kSmallK, all, ct, &near)) {
        sel = 8;
      } else {
        sel = 0;
        const int smallm = present & 7;
#pragma unroll
        for (int k = 0; k < kSmallK; ++k)
          if (((present >> k) & 1) && chi_keep32(t, k, smallm, ct, &near))
            sel |= (uint8_t)(1u << k);
      }
      exact = near;
    }
    if (exact) {
      // FP64 smoothness indicators and decision
      double beta[kSmallK + 1];
      double b = 0.0;
#pragma unroll
      for (int l = 0; l < M; ++l) b = fma((double)acc[l], (double)acc[l], b);
      beta[kSmallK] = b;
#pragma unroll
      for (int k = 0; k < kSmallK; ++k) {
        double q = 0.0;
#pragma unroll
        for (int l = 0; l < kSmallM; ++l) q = fma((double)as[k][l], (double)as[k][l], q);
        beta[k] = q;
      }
      sel = select_fp64(beta, present, a.ct, a.eps);
    }
  }
  if (a.sel_out) a.sel_out[(int64_t)v * a.n_pad + c] = sel;
  // final polynomial coefficients
  if (cweno) {
    // formed above
  } else if (sel & 8) {
#pragma unroll
    for (int l = 0; l < M; ++l) cf[l] = acc[l];
  } else {
    int nd = (sel & 1) + ((sel >> 1) & 1) + ((sel >> 2) & 1);
    TA w = nd ? TA(1.0) / TA(nd) : TA(0);
#pragma unroll
    for (int l = 0; l < M; ++l) cf[l] = TA(0);
#pragma unroll
    for (int k = 0; k < kSmallK; ++k) {
      if (!((sel >> k) & 1)) continue;
#pragma unroll
      for (int l = 0; l < kSmallM; ++l) cf[l] = fma(w, as[k][l], cf[l]);
    }
  }
  // values at the 3*NQ edge Gauss points: U_0 + Psi' c' (to Uq, or to the
  // caller's shared-memory stage with the same point stride NV)
  TA* __restrict__ out = ostage ? ostage : reinterpret_cast<TA*>(a.Uq) + c * (3 * NQ * NV) + v;
#pragma unroll
  for (int p = 0; p < 3 * NQ; ++p) {
    TA s = TA(0);
#pragma unroll
    for (int l = 0; l < M; ++l) {
      if constexpr (kMixed)
        s = fmaf(cf[l], ev.psi[p * kMaxM + l].x, s);  // FP32 table: hi parts
      else
        s = fma(cf[l], ev.psi[p * kMaxM + l], s);
    }
    if constexpr (kMixed)
      out[p * NV] = u0s.x + (s + u0s.y);
    else
      out[p * NV] = u0 + s;
  }
}


template <int M, int NS, int NQ, int NV, typename TA, typename TT>
__global__ void __launch_bounds__(128) recon_kernel(const ReconArgs a, const TT ev) {
  constexpr bool kMixed = std::is_same<TA, float>::value;
  const int lane = threadIdx.x, v = threadIdx.y;
  const int64_t tile = (int64_t)blockIdx.x * blockDim.z + threadIdx.z;
  const int64_t c = tile * kTile + lane;
  if (c >= a.n_cell) return;
  constexpr int E = M * NS + kSmallEntries;
  constexpr int SL = NS + kSmallSlots;
  const double* __restrict__ Uv = a.U + (int64_t)v * a.n_pad;
  const float2* __restrict__ Usv = kMixed ? a.Us + (int64_t)v * a.n_pad : nullptr;
  double u0 = 0.0;
  float2 u0s = make_float2(0.f, 0.f);
  if constexpr (kMixed)
    u0s = Usv[c];
  else
    u0 = Uv[c];
  const TA* __restrict__ A = reinterpret_cast<const TA*>(a.ahat) + tile * (int64_t)E * kTile + lane;
  const int32_t* __restrict__ nb = a.nbr + tile * (int64_t)SL * kTile + lane;
  auto diff = [&](int j) -> TA {
    if constexpr (kMixed) {
      const float2 q = __ldg(Usv + j);
      return (q.x - u0s.x) + (q.y - u0s.y);
    } else {
      return __ldg(Uv + j) - u0;
    }
  };

  // large stencil: a' = A'' d  (d_s = U_s - U_0)
  TA acc[M];
#pragma unroll
  for (int l = 0; l < M; ++l) acc[l] = TA(0);
#pragma unroll (std::is_same<TA, float>::value ? kSlotUnrollMixed : kSlotUnroll)
  for (int s = 0; s < NS; ++s) {
    const TA d = diff(__ldg(nb + s * kTile));
    const TA* As = A + (int64_t)s * M * kTile;
#pragma unroll
    for (int l = 0; l < M; ++l) acc[l] = fma(__ldg(As + l * kTile), d, acc[l]);
  }
  // directional stencils
  TA as[kSmallK][kSmallM];
#pragma unroll
  for (int k = 0; k < kSmallK; ++k) {
#pragma unroll
    for (int l = 0; l < kSmallM; ++l) as[k][l] = TA(0);
#pragma unroll (std::is_same<TA, float>::value ? kSlotUnrollMixed : kSlotUnroll)
    for (int s = 0; s < kSmallN; ++s) {
      const TA d = diff(__ldg(nb + (NS + k * kSmallN + s) * kTile));
      const TA* As = A + (int64_t)(M * NS + (k * kSmallN + s) * kSmallM) * kTile;
#pragma unroll
      for (int l = 0; l < kSmallM; ++l) as[k][l] = fma(__ldg(As + l * kTile), d, as[k][l]);
    }
  }
  plain_finish<M, NQ, NV, TA, TT>(a, ev, c, v, u0, u0s, acc, as);
}

// FP64-accurate reconstruction with double-float arithmetic on the FP32 pipe:
// stencil differences from the (hi, lo) split of U, matvecs, beta and the
// Gauss-point evaluation in pairs (relative error ~2^-46 of the summed
// magnitudes); the cutoff is decided in FP32 with the guard band of the mixed
// path and in FP64 inside it; Gauss-point values are written in FP64.
// selection, final coefficients and Gauss-point values of cell c, variable v
// (double-float path), from the normalised stencil coefficients
template <int M, int NQ, int NV, bool kExt = true>
__device__ __forceinline__ void df_finish(const ReconArgs& a, const DFTable& ev, int64_t c, int v,
                                          const DF (&acc)[M],
                                          const DF (&as)[kSmallK][kSmallM],
                                          float2* ostage = nullptr, int present_in = -1) {
  if constexpr (kExt) {
    if (a.coef_out) {
      store_coefs<M, DF>(a, c, v, acc, as);
      return;
    }
  }
  const int present = present_in >= 0 ? present_in : a.smask[c];
  uint8_t sel;
  const bool cweno = kExt && a.scheme == 1 && !a.linear;
  DF cf[M];
  if (cweno) {
    // beta = |a'|^2 in pairs, weights in FP64, combination in pairs
    double beta[kSmallK + 1];
    {
      DF b = {0.f, 0.f};
#pragma unroll
      for (int l = 0; l < M; ++l) df_mac(b, make_float2(acc[l].h, acc[l].l), acc[l]);
      beta[kSmallK] = df_to_double(df_norm(b));
#pragma unroll
      for (int k = 0; k < kSmallK; ++k) {
        DF q = {0.f, 0.f};
#pragma unroll
        for (int l = 0; l < kSmallM; ++l) df_mac(q, make_float2(as[k][l].h, as[k][l].l), as[k][l]);
        beta[k] = df_to_double(df_norm(q));
      }
    }
    const CwenoF cw = cweno_factors(beta[0], beta[1], beta[2], beta[kSmallK], present, a.cw_dK,
                                    a.eps);
    const double sK = cw.sK;
    const double* sk = cw.s;
    const DF fK = cst<DF>(sK);
#pragma unroll
    for (int l = 0; l < M; ++l) cf[l] = fK * acc[l];
#pragma unroll
    for (int k = 0; k < kSmallK; ++k) {
      const DF fk = cst<DF>(sk[k]);
#pragma unroll
      for (int l = 0; l < kSmallM; ++l) cf[l] = cf[l] + fk * as[k][l];
    }
    sel = 8;
  } else if (a.sel_in) {
    sel = a.sel_in[(int64_t)v * a.n_pad + c];
  } else if (a.linear) {
    sel = 8;
  } else {
    // beta = |a'|^2 in pairs
    DF bt[kSmallK + 1];
    {
      DF b = {0.f, 0.f};
#pragma unroll
      for (int l = 0; l < M; ++l) df_mac(b, make_float2(acc[l].h, acc[l].l), acc[l]);
      bt[kSmallK] = df_norm(b);
#pragma unroll
      for (int k = 0; k < kSmallK; ++k) {
        DF q = {0.f, 0.f};
#pragma unroll
        for (int l = 0; l < kSmallM; ++l) df_mac(q, make_float2(as[k][l].h, as[k][l].l), as[k][l]);
        bt[k] = df_norm(q);
      }
    }
    float t[kSmallK + 1];
#pragma unroll
    for (int k = 0; k <= kSmallK; ++k) t[k] = bt[k].h + (float)a.eps;
    const float ct = (float)a.ct;
    bool near = false;
    if (chi_keep32(t, kSmallK, present | 8, ct, &near)) {
      sel = 8;
    } else {
      sel = 0;
#pragma unroll
      for (int k = 0; k < kSmallK; ++k)
        if (((present >> k) & 1) && chi_keep32(t, k, present & 7, ct, &near))
          sel |= (uint8_t)(1u << k);
    }
    if (near) {
      double beta[kSmallK + 1];
#pragma unroll
      for (int k = 0; k <= kSmallK; ++k) beta[k] = df_to_double(bt[k]);
      sel = select_fp64(beta, present, a.ct, a.eps);
    }
  }
  if (a.sel_out) a.sel_out[(int64_t)v * a.n_pad + c] = sel;
  if (cweno) {
    // coefficients formed above
  } else if (sel & 8) {
#pragma unroll
    for (int l = 0; l < M; ++l) cf[l] = acc[l];
  } else {
    // equal weights: sum the kept polynomials, then divide by their number
    const int nd = (sel & 1) + ((sel >> 1) & 1) + ((sel >> 2) & 1);
    const float fn = (float)(nd ? nd : 1);
#pragma unroll
    for (int l = 0; l < M; ++l) cf[l] = {0.f, 0.f};
#pragma unroll
    for (int l = 0; l < kSmallM; ++l) {
      DF sum = {0.f, 0.f};
#pragma unroll
      for (int k = 0; k < kSmallK; ++k) {
        if (!((sel >> k) & 1)) continue;
        DF q = two_sum(sum.h, as[k][l].h);
        q.l += sum.l + as[k][l].l;
        sum = two_sum(q.h, q.l);
      }
      const float qh = sum.h / fn;
      const float r = fmaf(-qh, fn, sum.h);  // exact remainder
      cf[l] = two_sum(qh, (r + sum.l) / fn);
      if (!nd) cf[l] = {0.f, 0.f};
    }
  }
  // Gauss-point values as (hi, lo) pairs: split(U_0) + Psi' c'
  const float2 u0s = a.Us[(int64_t)v * a.n_pad + c];
  float2* __restrict__ out =
      ostage ? ostage : reinterpret_cast<float2*>(a.Uq) + c * (3 * NQ * NV) + v;
#pragma unroll
  for (int p = 0; p < 3 * NQ; ++p) {
    DF s = {0.f, 0.f};
#pragma unroll
    for (int l = 0; l < M; ++l) df_mac(s, ev.psi[p * kMaxM + l], cf[l]);
    const DF r = DF{u0s.x, u0s.y} + df_norm(s);
    out[p * NV] = make_float2(r.h, r.l);
  }
}


template <int M, int NS, int NQ, int NV>
__global__ void __launch_bounds__(128) recon_df_kernel(const ReconArgs a, const DFTable ev) {
  const int lane = threadIdx.x, v = threadIdx.y;
  const int64_t tile = (int64_t)blockIdx.x * blockDim.z + threadIdx.z;
  const int64_t c = tile * kTile + lane;
  if (c >= a.n_cell) return;
  constexpr int E = M * NS + kSmallEntries;
  constexpr int SL = NS + kSmallSlots;
  const float2* __restrict__ Usv = a.Us + (int64_t)v * a.n_pad;
  const float2 u0s = Usv[c];
  const float2* __restrict__ A =
      reinterpret_cast<const float2*>(a.ahat) + tile * (int64_t)E * kTile + lane;
  const int32_t* __restrict__ nb = a.nbr + tile * (int64_t)SL * kTile + lane;
  auto diff = [&](int j) -> DF {
    const float2 q = __ldg(Usv + j);
    DF s = two_sum(q.x, -u0s.x);
    s.l += q.y - u0s.y;
    return two_sum(s.h, s.l);
  };
  DF acc[M];
#pragma unroll
  for (int l = 0; l < M; ++l) acc[l] = {0.f, 0.f};
#pragma unroll (kSlotUnroll)
  for (int s = 0; s < NS; ++s) {
    const DF d = diff(__ldg(nb + s * kTile));
    const float2* As = A + (int64_t)s * M * kTile;
#pragma unroll
    for (int l = 0; l < M; ++l) df_mac(acc[l], __ldg(As + l * kTile), d);
  }
#pragma unroll
  for (int l = 0; l < M; ++l) acc[l] = df_norm(acc[l]);
  DF as[kSmallK][kSmallM];
#pragma unroll
  for (int k = 0; k < kSmallK; ++k) {
#pragma unroll
    for (int l = 0; l < kSmallM; ++l) as[k][l] = {0.f, 0.f};
#pragma unroll (kSlotUnroll)
    for (int s = 0; s < kSmallN; ++s) {
      const DF d = diff(__ldg(nb + (NS + k * kSmallN + s) * kTile));
      const float2* As = A + (int64_t)(M * NS + (k * kSmallN + s) * kSmallM) * kTile;
#pragma unroll
      for (int l = 0; l < kSmallM; ++l) df_mac(as[k][l], __ldg(As + l * kTile), d);
    }
#pragma unroll
    for (int l = 0; l < kSmallM; ++l) as[k][l] = df_norm(as[k][l]);
  }
  df_finish<M, NQ, NV>(a, ev, c, v, acc, as);
}

// ------------------------------------------ halo-staged reconstruction
// The union of the stencils of a 32-cell tile (its "halo", <= kHaloMax cells,
// listed on the host) is gathered once into shared memory; every stencil
// difference then reads shared memory, and the only global stream of the
// main loop is the coalesced, independent stream of per-cell matrices.
// kMode 0: FP64 path (double-float), 1: FP32-mixed, 2: FP64 native.
template <int kMode>
struct HaloTraits;
template <>
struct HaloTraits<0> {
  using TE = float2;   // matrix entry
  using TS = float2;   // staged state (hi, lo split)
  using Acc = DF;
  using Tab = DFTable;
};
template <>
struct HaloTraits<1> {
  using TE = float;
  using TS = float2;
  using Acc = float;
  using Tab = DFTable;
};
template <>
struct HaloTraits<2> {
  using TE = double;
  using TS = double;
  using Acc = double;
  using Tab = EvalTable;
};

template <int M, int NS, int NQ, int NV, int kMode>
__global__ void __launch_bounds__(128) recon_halo_kernel(const ReconArgs a, const HaloArgs h,
                                                         const typename HaloTraits<kMode>::Tab ev) {
  using TR = HaloTraits<kMode>;
  using TE = typename TR::TE;
  using TS = typename TR::TS;
  using Acc = typename TR::Acc;
  constexpr int TZ = 4 / NV;
  constexpr int E = M * NS + kSmallEntries;
  constexpr int SL = NS + kSmallSlots;
  __shared__ TS hs[TZ][NV][kHaloMax];
  const int lane = threadIdx.x, v = threadIdx.y, z = threadIdx.z;
  const int64_t n_tiles = (a.n_cell + kTile - 1) / kTile;
  const int64_t tile = (int64_t)blockIdx.x * TZ + z;
  const bool tvalid = tile < n_tiles;
  // cooperative gather of the tile's halo states (all vars) by its NV warps
  if (tvalid) {
    const int h0 = h.off[tile], H = h.off[tile + 1] - h0;
    for (int i = lane + kTile * v; i < H; i += kTile * NV) {
      const int id = __ldg(h.ids + h0 + i);
#pragma unroll
      for (int w = 0; w < NV; ++w) {
        if constexpr (kMode == 2)
          hs[z][w][i] = __ldg(a.U + (int64_t)w * a.n_pad + id);
        else
          hs[z][w][i] = __ldg(a.Us + (int64_t)w * a.n_pad + id);
      }
    }
  }
  __syncthreads();
  if (!tvalid) return;
  const int64_t c = tile * kTile + lane;  // pad lanes compute, but store nothing
  const int64_t cc = c < a.n_cell ? c : 0;
  double u0 = 0.0;
  float2 u0s = make_float2(0.f, 0.f);
  if constexpr (kMode == 2)
    u0 = a.U[(int64_t)v * a.n_pad + cc];
  else
    u0s = a.Us[(int64_t)v * a.n_pad + cc];
  const TS* __restrict__ st = hs[z][v];
  const TE* __restrict__ A = reinterpret_cast<const TE*>(a.ahat) + tile * (int64_t)E * kTile + lane;
  const uint16_t* __restrict__ nb = h.nbr_loc + tile * (int64_t)SL * kTile + lane;
  auto dif = [&](int s) -> Acc {
    const TS q = st[__ldg(nb + s * kTile) & kHaloPosMask];
    if constexpr (kMode == 0) {
      DF t = two_sum(q.x, -u0s.x);
      t.l += q.y - u0s.y;
      return two_sum(t.h, t.l);
    } else if constexpr (kMode == 1) {
      return (q.x - u0s.x) + (q.y - u0s.y);
    } else {
      return q - u0;
    }
  };
  auto mac = [](Acc& acc, TE m, Acc d) {
    if constexpr (kMode == 0)
      df_mac(acc, m, d);
    else
      acc = fma(m, d, acc);
  };
  Acc acc[M];
#pragma unroll
  for (int l = 0; l < M; ++l) acc[l] = Acc{};
#pragma unroll (kMode == 1 ? kSlotUnrollMixed : kSlotUnroll)
  for (int s = 0; s < NS; ++s) {
    const Acc d = dif(s);
    const TE* As = A + (int64_t)s * M * kTile;
#pragma unroll
    for (int l = 0; l < M; ++l) mac(acc[l], __ldg(As + l * kTile), d);
  }
  Acc as[kSmallK][kSmallM];
#pragma unroll
  for (int k = 0; k < kSmallK; ++k) {
#pragma unroll
    for (int l = 0; l < kSmallM; ++l) as[k][l] = Acc{};
#pragma unroll (kMode == 1 ? kSlotUnrollMixed : kSlotUnroll)
    for (int s = 0; s < kSmallN; ++s) {
      const Acc d = dif(NS + k * kSmallN + s);
      const TE* As = A + (int64_t)(M * NS + (k * kSmallN + s) * kSmallM) * kTile;
#pragma unroll
      for (int l = 0; l < kSmallM; ++l) mac(as[k][l], __ldg(As + l * kTile), d);
    }
  }
  if (c >= a.n_cell) return;
  if constexpr (kMode == 0) {
#pragma unroll
    for (int l = 0; l < M; ++l) acc[l] = df_norm(acc[l]);
#pragma unroll
    for (int k = 0; k < kSmallK; ++k)
#pragma unroll
      for (int l = 0; l < kSmallM; ++l) as[k][l] = df_norm(as[k][l]);
    df_finish<M, NQ, NV, false>(a, ev, c, v, acc, as);
  } else if constexpr (kMode == 1) {
    plain_finish<M, NQ, NV, float, DFTable, false>(a, ev, c, v, 0.0, u0s, acc, as);
  } else {
    plain_finish<M, NQ, NV, double, EvalTable, false>(a, ev, c, v, u0, u0s, acc, as);
  }
}

// -------------------------------------------- TMA-staged reconstruction
// The per-cell matrices of a 32-cell tile are one contiguous block of global
// memory ([tile][entry][32]).  One producer lane streams that block into a
// ring of kRing shared-memory buffers with 1D bulk copies (cp.async.bulk,
// completion counted in bytes on the buffer's "full" mbarrier); the four
// consumer warps of the tile (one per conservative variable) wait on "full",
// accumulate from shared memory, and release the buffer on its "empty"
// mbarrier.  Every wait is bounded.  A wait that gives up sets bit 1 of the
// error flag and the block's abort flag in shared memory; from then on the
// consumers skip every wait and all work but still pass the consumer-only
// barriers of the remaining tiles (so no warp is left at a barrier), and the
// producer stops issuing, waits (bounded) for the copies it has in flight and
// returns.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
constexpr uint32_t kWaitLimit = 1u << 22;
// wait for the completion of the phase with the given parity; false on give-up
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitLimit; ++i)
    if (mbar_test(bar, parity)) return true;
  return false;
}
// as mbar_wait, also watching the block's abort flag: 1 phase complete, 0 gave
// up, 2 another thread of the block gave up first
__device__ __forceinline__ int mbar_wait_or_abort(uint64_t* bar, uint32_t parity,
                                                  const volatile int* abort,
                                                  uint32_t limit = kWaitLimit) {
  for (uint32_t i = 0; i < limit; ++i) {
    if (mbar_test(bar, parity)) return 1;
    if (*abort) return 2;
  }
  return 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

constexpr int kRing = 4;
constexpr int kConsumers = 4;  // one warp per conservative variable (Euler)

// cp.async (8-byte asynchronous global->shared copies) for the halo prefetch
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
// 16-byte asynchronous copy (both addresses 16-byte aligned), L2 only
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// barrier of the four consumer warps only (the producer warp does not take part)
__device__ __forceinline__ void consumer_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kConsumers * kTile) : "memory");
}

// Output stage of the TMA kernels.  Each variable warp writes its lanes'
// Gauss-point values to shared memory laid out [cell][point][variable] with
// an odd cell stride of kPer + 1 elements (conflict-free), and the consumer
// threads then store the tile's contiguous block of Uq with coalesced writes
// instead of one 32-sector store per point and variable.
#ifndef TENO_STAGE_OUT
#define TENO_STAGE_OUT 1
#endif
// the W-form kernel measured faster with its direct 8-byte pair stores (the
// stage costs it a ring slot and a barrier per tile)
#ifndef TENO_STAGE_OUT_W
#define TENO_STAGE_OUT_W 0
#endif
template <int kPer, typename TO>
__device__ __forceinline__ void store_out_stage(const TO* stg, TO* __restrict__ dst, int nvalid,
                                                int tid) {
#pragma unroll 3
  for (int e = tid; e < nvalid * kPer; e += kConsumers * kTile) {
    const int cl = e / kPer;
    dst[e] = stg[cl * (kPer + 1) + (e - cl * kPer)];
  }
}
template <int kPer, typename TO>
constexpr size_t out_stage_bytes() {
  return ((size_t)kTile * (kPer + 1) * sizeof(TO) + 15) / 16 * 16;
}

// Stage j of a tile's matrix block: kLPS large-stencil slots, or kSPS slots of
// one directional stencil.
template <int M, int NS, int kEsz, int kLPS, int kSPS, int kRingT = kRing>
struct StagePlan {
  static constexpr int kSlotL = M * kTile * kEsz;
  static constexpr int kSlotS = kSmallM * kTile * kEsz;
  static constexpr int kNL = (NS + kLPS - 1) / kLPS;
  static constexpr int kPerSmall = kSmallN / kSPS;
  static constexpr int kStages = kNL + kSmallK * kPerSmall;
  static constexpr int kMatL = kLPS * kSlotL, kMatS = kSPS * kSlotS;
  static constexpr int kMaxSlots = kLPS > kSPS ? kLPS : kSPS;
  static constexpr int kSlotN = kTile * 2;  // halo positions (uint16) of one slot
  // ring buffer: [matrix rows][halo positions]
  static constexpr int kNOff = kMatL > kMatS ? kMatL : kMatS;
  static constexpr int kMat = kNOff + kMaxSlots * kSlotN;
  static constexpr int kSL = NS + kSmallSlots;
  static constexpr int kE = M * NS + kSmallEntries;
  static constexpr int64_t kTileBytes = (int64_t)kE * kTile * kEsz;
  static constexpr size_t kHaloBytes = (size_t)2 * 4 * kHaloMax * sizeof(float2);
  static constexpr size_t kSmem =
      (size_t)kRingT * kMat + kHaloBytes + 2 * kRingT * sizeof(uint64_t) + 16;
  static_assert(kSmallN % kSPS == 0, "directional stencil split");
  static_assert(kMat % 16 == 0, "16-byte aligned buffers");
  __device__ static void stage(int j, int& slot0, int& nslot, int64_t& off, int& bytes, int& k) {
    if (j < kNL) {
      slot0 = j * kLPS;
      nslot = (NS - slot0) < kLPS ? (NS - slot0) : kLPS;
      off = (int64_t)slot0 * kSlotL;
      bytes = nslot * kSlotL;
      k = -1;
    } else {
      const int i = j - kNL;
      k = i / kPerSmall;
      const int s0 = (i % kPerSmall) * kSPS;
      slot0 = NS + k * kSmallN + s0;
      nslot = kSPS;
      off = (int64_t)(M * NS + (k * kSmallN + s0) * kSmallM) * kTile * kEsz;
      bytes = kSPS * kSlotS;
    }
  }
};

// Ring depth of the FP32-mixed bulk-copy reconstruction: 4 stages unless
// they keep the kernel below four blocks per SM, then 3 (TENO6: 3 -> 4 blocks,
// 7 % faster; TENO5 fits four blocks with 4 stages).  TENO_RING_MIXED > 0
// overrides.
#ifndef TENO_RING_MIXED
#define TENO_RING_MIXED 0
#endif
template <int M, int NS, int NQ>
struct MixedRing {
  static constexpr size_t kBlock4 = StagePlan<M, NS, 4, 4, 4, 4>::kSmem +
                                    (TENO_STAGE_OUT ? out_stage_bytes<3 * NQ * 4, float>() : 0) +
                                    1024;
  static constexpr int value =
      TENO_RING_MIXED > 0 ? TENO_RING_MIXED : (4 * kBlock4 <= (size_t)228 * 1024 ? 4 : 3);
};
template <bool kDF, int M, int NS, int NQ>
struct TmaTraits {
  using TE = float2;  // matrix entry: (hi, lo)
  using Acc = DF;
  static constexpr int kLPS = 4, kSPS = 4, kRing = 4;
};
template <int M, int NS, int NQ>
struct TmaTraits<false, M, NS, NQ> {
  using TE = float;
  using Acc = float;
  static constexpr int kLPS = 4, kSPS = 4, kRing = MixedRing<M, NS, NQ>::value;
};

// Halo prefetch pipeline of the bulk-copy reconstruction kernels (consumer
// threads).  The cp.async copies of a tile's halo need its halo ids, and the
// ids need the tile's halo offsets: the offsets are loaded two tiles ahead
// and the ids one tile ahead (two per thread: a halo has at most 256 cells
// and there are 128 consumer threads), so issuing the copies never waits on
// a global load.  Tiles advance by the grid size.
struct HaloPipe {
  static constexpr int kCT = kConsumers * kTile;
  static_assert(kHaloMax <= 2 * kCT, "two halo ids per consumer thread");
  const HaloArgs& h;
  const float2* Us;
  int64_t n_pad, n_tiles;
  int tid;
  int H1 = 0, id0 = 0, id1 = 0;  // ids of the next tile
  int h02 = 0, H2 = 0;           // offsets of the tile after it
  __device__ HaloPipe(const HaloArgs& h_, const float2* Us_, int64_t n_pad_, int64_t n_tiles_,
                      int tid_)
      : h(h_), Us(Us_), n_pad(n_pad_), n_tiles(n_tiles_), tid(tid_) {}
  __device__ void offsets(int64_t tile, int& h0, int& H) const {
    h0 = 0, H = 0;
    if (tile < n_tiles) {
      h0 = h.off[tile];
      H = h.off[tile + 1] - h0;
    }
  }
  __device__ void ids(int h0, int H) {
    H1 = H, id0 = 0, id1 = 0;
    if (tid < H) id0 = __ldg(h.ids + h0 + tid);
    if (tid + kCT < H) id1 = __ldg(h.ids + h0 + tid + kCT);
  }
  // copies of the halo whose ids are held into buffer hb, one commit group
  __device__ void issue(float2* halo, int hb) const {
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      if (tid < H1) cp_async8(&halo[(hb * 4 + w) * kHaloMax + tid], Us + (int64_t)w * n_pad + id0);
      if (tid + kCT < H1)
        cp_async8(&halo[(hb * 4 + w) * kHaloMax + tid + kCT], Us + (int64_t)w * n_pad + id1);
    }
    cp_async_commit();
  }
  // prologue: the first tile's halo into buffer 0 (waits once), the ids of
  // the second tile and the offsets of the third
  __device__ void start(int64_t t0, int64_t G, float2* halo) {
    int h0, H;
    offsets(t0, h0, H);
    ids(h0, H);
    issue(halo, 0);
    offsets(t0 + G, h0, H);
    ids(h0, H);
    offsets(t0 + 2 * G, h02, H2);
  }
  // at tile t: the halo of t + G into buffer hb (an empty group past the
  // end), then the ids of t + 2G and the offsets of t + 3G
  __device__ void advance(int64_t t, int64_t G, float2* halo, int hb) {
    issue(halo, hb);
    ids(h02, H2);
    offsets(t + 3 * G, h02, H2);
  }
};

// Persistent kernel, Euler only.  Producer lane: the matrix block of every
// tile in kRing-deep bulk-copy stages.  Consumer warps (one per variable):
// the tile's stencil halo in a double-buffered shared-memory area, prefetched
// with cp.async one tile ahead; stencil differences from the halo, matrices
// from the ring.  kDF: FP64 path (double-float); !kDF: FP32-mixed path.
// The pair kernel with the CWENO and characteristic branches (kDF && kExt)
// is held to two blocks per SM: uncapped it took 252 registers at TENO6, one
// block (five warps) per SM.
template <int M, int NS, int NQ, bool kDF, bool kExt>
__global__ void __launch_bounds__(kTile * (kConsumers + 1), (kDF && kExt) ? 2 : 0)
    recon_tma_kernel(const ReconArgs a, const HaloArgs h, const DFTable ev, int* err) {
  using TR = TmaTraits<kDF, M, NS, NQ>;
  using TE = typename TR::TE;
  constexpr int kRing = TR::kRing;
  using P = StagePlan<M, NS, (int)sizeof(TE), TR::kLPS, TR::kSPS, kRing>;
  constexpr int NV = 4;
  constexpr int SL = NS + kSmallSlots;
  constexpr int kPer = 3 * NQ * NV;  // Gauss-point values per cell
  // output stage on the FP32-mixed TENO path (the pair path would lose a
  // block per SM to it)
  constexpr bool kStage = TENO_STAGE_OUT && !kExt && !kDF;
  extern __shared__ __align__(128) unsigned char smem[];
  float2* halo = reinterpret_cast<float2*>(smem + (size_t)kRing * P::kMat);  // [2][NV][kHaloMax]
  float* ostg = reinterpret_cast<float*>(smem + P::kSmem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)kRing * P::kMat + P::kHaloBytes);
  uint64_t* empty = full + kRing;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + kRing);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n_tiles = (a.n_cell + kTile - 1) / kTile;
  if (threadIdx.x == 0) {
    *abort_flag = 0;
    for (int i = 0; i < kRing; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kConsumers);
    }
    mbar_fence_init();
  }
  __syncthreads();
  if (warp == kConsumers) {
    // ---- producer lane: matrix blocks, tile after tile
    if (lane == 0) {
      int64_t g = 0;
      for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const unsigned char* src =
            reinterpret_cast<const unsigned char*>(a.ahat) + tile * P::kTileBytes;
        const unsigned char* sn =
            reinterpret_cast<const unsigned char*>(h.nbr_loc) + tile * (int64_t)P::kSL * P::kSlotN;
        for (int j = 0; j < P::kStages; ++j, ++g) {
          const int b = (int)(g % kRing);
          if (g >= kRing) {
            const int w = mbar_wait_or_abort(&empty[b], (uint32_t)((g / kRing) - 1) & 1, abort_flag);
            if (w != 1) {
              if (w == 0) {
                atomicOr(err, 2);
                *abort_flag = 1;
              }
              for (int64_t i = g - kRing; i < g; ++i)
                mbar_wait(&full[i % kRing], (uint32_t)(i / kRing) & 1);
              return;
            }
          }
          int slot0, nslot, bytes, k;
          int64_t off;
          P::stage(j, slot0, nslot, off, bytes, k);
          const uint32_t bn = (uint32_t)(nslot * P::kSlotN);
          unsigned char* dst = smem + (size_t)b * P::kMat;
          mbar_expect_tx(&full[b], (uint32_t)bytes + bn);
          bulk_g2s(dst, src + off, (uint32_t)bytes, &full[b]);
          bulk_g2s(dst + P::kNOff, sn + slot0 * P::kSlotN, bn, &full[b]);
        }
      }
      // the block must not exit while a copy it issued is in flight (the
      // consumers skip their waits once a wait has given up)
      for (int64_t i = g > kRing ? g - kRing : 0; i < g; ++i)
        mbar_wait(&full[i % kRing], (uint32_t)(i / kRing) & 1);
    }
    return;
  }
  // ---- consumers
  const int v = warp, tid = threadIdx.x;
  using Acc = typename TR::Acc;
  HaloPipe hp(h, a.Us, a.n_pad, n_tiles, tid);
  auto mac = [](Acc& acc, TE m, Acc d) {
    if constexpr (kDF)
      df_mac(acc, m, d);
    else
      acc = fmaf(m, d, acc);
  };
  int64_t g = 0;
  int hb = 0;
  bool dead = false;  // a bounded wait of this block gave up: skip all work
  hp.start(blockIdx.x, gridDim.x, halo);
  // the cell's own split state and stencil mask, loaded a tile ahead
  auto own = [&](int64_t tile, float2& u, int& pm) {
    const int64_t cc = tile * kTile + lane;
    const int64_t ci = (tile < n_tiles && cc < a.n_cell) ? cc : 0;
    u = a.Us[(int64_t)v * a.n_pad + ci];
    pm = a.smask[ci];
  };
  float2 u0n;
  int pmn;
  own(blockIdx.x, u0n, pmn);
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, hb ^= 1) {
    consumer_sync();  // every consumer is done with the other halo buffer
    hp.advance(tile, gridDim.x, halo, hb ^ 1);  // halo of the next tile, ids a tile ahead
    const float2 u0s = u0n;
    const int present = pmn;
    own(tile + gridDim.x, u0n, pmn);
    cp_async_wait<1>();  // this thread's copies of the current halo have landed
    consumer_sync();     // ... and everyone's
    const float2* st = halo + (hb * NV + v) * kHaloMax;
    const uint16_t* nb = h.nbr_loc + tile * (int64_t)SL * kTile + lane;
    const int64_t c = tile * kTile + lane;  // may be a pad lane of the last tile
    auto dif = [&](int idx) -> Acc {
      const float2 q = st[idx];
      if constexpr (kDF) {
        DF t = two_sum(q.x, -u0s.x);
        t.l += q.y - u0s.y;
        return two_sum(t.h, t.l);
      } else {
        return (q.x - u0s.x) + (q.y - u0s.y);
      }
    };
    Acc acc[M];
    Acc as[kSmallK][kSmallM];
#pragma unroll
    for (int l = 0; l < M; ++l) acc[l] = Acc{};
#pragma unroll
    for (int k = 0; k < kSmallK; ++k)
#pragma unroll
      for (int l = 0; l < kSmallM; ++l) as[k][l] = Acc{};
    for (int j = 0; j < P::kStages; ++j, ++g) {
      const int b = (int)(g % kRing);
      int slot0, nslot, bytes, k;
      int64_t off;
      P::stage(j, slot0, nslot, off, bytes, k);
      if (!dead) {
        const int w =
            mbar_wait_or_abort(&full[b], (uint32_t)(g / kRing) & 1, abort_flag, a.wait_polls);
        if (w == 0) {
          atomicOr(err, 2);
          *abort_flag = 1;
        }
        dead = __any_sync(0xffffffffu, w != 1);
      }
      const TE* mat = reinterpret_cast<const TE*>(smem + (size_t)b * P::kMat) + lane;
      const uint16_t* nl = reinterpret_cast<const uint16_t*>(smem + (size_t)b * P::kMat + P::kNOff) + lane;
      if (dead) {
        // skip the stage
      } else if (k < 0) {
#pragma unroll
        for (int s = 0; s < TR::kLPS; ++s) {
          if (s < nslot) {
            const Acc d = dif(nl[s * kTile] & kHaloPosMask);
#pragma unroll
            for (int l = 0; l < M; ++l) mac(acc[l], mat[(s * M + l) * kTile], d);
          }
        }
      } else {
#pragma unroll
        for (int kk = 0; kk < kSmallK; ++kk) {
          if (kk != k) continue;
#pragma unroll
          for (int s = 0; s < TR::kSPS; ++s) {
            const Acc d = dif(nl[s * kTile] & kHaloPosMask);
#pragma unroll
            for (int l = 0; l < kSmallM; ++l) mac(as[kk][l], mat[(s * kSmallM + l) * kTile], d);
          }
        }
      }
      __syncwarp();
      if (lane == 0 && !dead) mbar_arrive(&empty[b]);
    }
    if (!dead && c < a.n_cell) {
      if constexpr (kDF) {
#pragma unroll
        for (int l = 0; l < M; ++l) acc[l] = df_norm(acc[l]);
#pragma unroll
        for (int k = 0; k < kSmallK; ++k)
#pragma unroll
          for (int l = 0; l < kSmallM; ++l) as[k][l] = df_norm(as[k][l]);
        df_finish<M, NQ, NV, kExt>(a, ev, c, v, acc, as, nullptr, present);
      } else {
        plain_finish<M, NQ, NV, float, DFTable, kExt>(a, ev, c, v, 0.0, u0s, acc, as,
                                                      kStage ? ostg + lane * (kPer + 1) + v
                                                             : nullptr,
                                                      present);
      }
    }
    if constexpr (kStage) {
      consumer_sync();  // the tile's values are staged
      if (!dead)
        store_out_stage<kPer>(ostg, reinterpret_cast<float*>(a.Uq) + tile * kTile * kPer,
                              (int)min((int64_t)kTile, a.n_cell - tile * kTile), tid);
    }
  }
  cp_async_wait<0>();
}

// ------------------------------------------- FP64 path, W form (variant 2)
// Algebraically the same reconstruction as recon_tma_kernel<kDF = true>, with
// the work split by what each quantity needs:
//  - the Gauss-point values of the large polynomial, U_0 + Psi' (G d), are
//    accumulated in pairs as U_0 + W d with W = Psi' G precomputed per cell
//    (3 N_q pair products per stencil slot instead of m);
//  - the smoothness indicators feed only the cutoff decision, so the stencil
//    coefficients for beta are FP32 products G d with a rigorous error bound
//    (per slot the column sum sum_l |G_ls| is stored next to the rows);
//    where the bound does not separate chi from C_T the coefficients and
//    beta are recomputed in pairs from the (hi, lo) matrices and the
//    decision is taken in FP64;
//  - directional-stencil values (cells where the large stencil is cut) are
//    evaluated in pairs from the (hi, lo) matrices.
#ifndef TENO_W_BLOCKS
#define TENO_W_BLOCKS 3  // 3: three blocks per SM; 0: four where the ring fits
#endif
constexpr int kWBlocks = TENO_W_BLOCKS;

template <int M, int NS, int NQ3, int kLPS, int kSPS>
struct WPlan {
  static constexpr int kG = M + 1, kGs = kSmallM + 1;
  static constexpr int kSlotG = kG * kTile * 4, kSlotW = NQ3 * kTile * 8;
  static constexpr int kSlotS = kGs * kTile * 4;
  static constexpr int kSlotN = kTile * 2;  // halo positions (uint16) of one slot
  static constexpr int kNL = (NS + kLPS - 1) / kLPS;
  static constexpr int kPerSmall = kSmallN / kSPS;
  static constexpr int kStages = kNL + kSmallK * kPerSmall;
  static constexpr int kMaxSlots = kLPS > kSPS ? kLPS : kSPS;
  // ring buffer: [FP32 rows][W pairs][halo positions]
  static constexpr int kGReg = kLPS * kSlotG > kSPS * kSlotS ? kLPS * kSlotG : kSPS * kSlotS;
  static constexpr int kWOff = kGReg, kNOff = kGReg + kLPS * kSlotW;
  static constexpr int kMat = kNOff + kMaxSlots * kSlotN;
  static constexpr int kE32 = NS * kG + kSmallK * kSmallN * kGs;  // floats per lane per tile
  static constexpr int kEW = NS * NQ3;                            // pairs per lane per tile
  static constexpr int kSL = NS + kSmallSlots;
  static constexpr size_t kHaloBytes = (size_t)2 * 4 * kHaloMax * sizeof(float2);
  // output stage of the Gauss-point pairs of one tile (float2 elements)
  static constexpr size_t kOut = TENO_STAGE_OUT_W ? out_stage_bytes<NQ3 * 4, float2>() : 0;
  static constexpr size_t kFixed = kHaloBytes + 2 * 4 * 8 + 16 + kOut;
  // blocks of 160 threads per SM (228 KB of shared memory, 1 KB reserved per
  // block): four with a 3-deep ring where that fits, else three (4-deep
  // ring if it fits)
  static constexpr bool kFour = kWBlocks != 3 &&
                                4 * ((size_t)3 * kMat + kFixed + 1024) <= (size_t)228 * 1024;
  static constexpr int kRingW =
      kFour ? 3 : (3 * ((size_t)4 * kMat + kFixed + 1024) <= (size_t)228 * 1024 ? 4 : 3);
  static constexpr int kBlocks = kFour ? 4 : 3;
  static constexpr size_t kOutOff = (size_t)kRingW * kMat + kHaloBytes + 2 * kRingW * 8 + 16;
  static constexpr size_t kSmem = kOutOff + kOut;
  static_assert(kSmallN % kSPS == 0, "directional stencil split");
  static_assert(kSlotG % 16 == 0 && kSlotW % 16 == 0 && kSlotS % 16 == 0 && kMat % 16 == 0,
                "bulk-copy sizes");
  // stage j: slots [slot0, slot0 + nslot) of stencil k (-1: large); byte
  // offsets / sizes of its FP32 block (og, bg) and W block (ow, bw) in the tile
  __device__ static void stage(int j, int& slot0, int& nslot, int& k, int& og, int& bg, int& ow,
                               int& bw) {
    if (j < kNL) {
      slot0 = j * kLPS;
      nslot = (NS - slot0) < kLPS ? (NS - slot0) : kLPS;
      k = -1;
      og = slot0 * kSlotG;
      bg = nslot * kSlotG;
      ow = slot0 * kSlotW;
      bw = nslot * kSlotW;
    } else {
      const int i = j - kNL;
      k = i / kPerSmall;
      const int s0 = (i % kPerSmall) * kSPS;
      slot0 = NS + k * kSmallN + s0;
      nslot = kSPS;
      og = NS * kSlotG + (k * kSmallN + s0) * kSlotS;
      bg = kSPS * kSlotS;
      ow = 0;
      bw = 0;
    }
  }
};

// Upper bound of |beta_fp32 - beta| relative to beta_fp32 + eps for m FP32
// coefficients a32_l from n-term FP32 dot products.  Coefficient l errs by at
// most e_l = (n + 7) u S_l with S_l = sum_s |G_ls| |d_s| (u = 2^-24; the
// stored matrix rounding and a difference conversion of up to 2u -- the FP64
// path truncates -- included), and sum_l S_l = e_abs = sum_s colsum_s |d_s|.
// With E = sum_l e_l, Cauchy-Schwarz gives
// |sum a32^2 - sum a^2| <= sum e_l (2 |a32_l| + e_l) <= 2 E sqrt(beta32) + E^2;
// the FP32 sum of squares adds (m + 2) u beta32.  Returns a value >= 1 when
// the bound is not informative.
__device__ __forceinline__ float beta_rel_bound(float beta32, float e_abs, int n, int m,
                                                float eps) {
  const float u = 5.9604645e-8f;
  const float E = (float)(n + 7) * u * e_abs * 1.0001f;
  const float eb = (float)(m + 2) * u * beta32 + E * (2.f * sqrtf(beta32) + E);
  const float t = beta32 + eps;
  if (!(eb < 0.5f * t)) return 1.f;
  return eb / (t - eb);
}

// FP64 -> FP32 by truncation of the significand, in integer instructions
// (the conversion instruction would take a slot of the FP64 pipe, which bounds
// the FP64 path's reconstruction).  Relative error below 2^-23 for results in
// the normal FP32 range; magnitudes below it give a signed zero (an absolute
// error under 1.2e-38), magnitudes above it, infinities and NaN give an
// infinity, which the cutoff screen sends to its FP64 fallback.
__device__ __forceinline__ float d2f_trunc(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

// pair difference U_s - U_0 of a halo cell (FP32 hi/lo splits of the states)
__device__ __forceinline__ DF halo_dif(const float2* st, int idx, float2 u0s) {
  const float2 q = st[idx];
  DF t = two_sum(q.x, -u0s.x);
  t.l += q.y - u0s.y;
  return two_sum(t.h, t.l);
}

// Rare paths of the W-form kernel, kept out of line so that their registers
// do not weigh on the main loop.  A: the cell's (hi, lo) matrices at its lane,
// nb: its halo positions, st: the tile's halo of its variable.
//
// Cutoff decision in FP64 from coefficients and beta in pairs.
template <int M, int NS>
__device__ __noinline__ uint8_t w_select_pairs(const float2* A, const uint16_t* nb,
                                               const float2* st, float2 u0s, int present,
                                               double ct, double eps) {
  DF al[M];
#pragma unroll
  for (int l = 0; l < M; ++l) al[l] = DF{0.f, 0.f};
  for (int s = 0; s < NS; ++s) {
    const DF d = halo_dif(st, nb[s * kTile] & kHaloPosMask, u0s);
#pragma unroll
    for (int l = 0; l < M; ++l) df_mac(al[l], __ldg(A + (int64_t)(s * M + l) * kTile), d);
  }
  double beta[kSmallK + 1];
  {
    DF bl = {0.f, 0.f};
#pragma unroll
    for (int l = 0; l < M; ++l) {
      const DF x = df_norm(al[l]);
      df_mac(bl, make_float2(x.h, x.l), x);
    }
    beta[kSmallK] = df_to_double(df_norm(bl));
  }
#pragma unroll
  for (int k = 0; k < kSmallK; ++k) {
    DF as[kSmallM];
#pragma unroll
    for (int l = 0; l < kSmallM; ++l) as[l] = DF{0.f, 0.f};
    if ((present >> k) & 1) {
      for (int s = 0; s < kSmallN; ++s) {
        const DF d = halo_dif(st, nb[(NS + k * kSmallN + s) * kTile] & kHaloPosMask, u0s);
        const float2* As = A + (int64_t)(M * NS + (k * kSmallN + s) * kSmallM) * kTile;
#pragma unroll
        for (int l = 0; l < kSmallM; ++l) df_mac(as[l], __ldg(As + l * kTile), d);
      }
    }
    DF q = {0.f, 0.f};
#pragma unroll
    for (int l = 0; l < kSmallM; ++l) {
      const DF x = df_norm(as[l]);
      df_mac(q, make_float2(x.h, x.l), x);
    }
    beta[k] = df_to_double(df_norm(q));
  }
  return select_fp64(beta, present, ct, eps);
}

// Gauss-point values of the equally weighted kept directional polynomials
// (step ii of the selection), in pairs; psi: the [point][kMaxM] table of
// Psi' as pairs.
template <int M, int NS, int NQ3, int NV>
__device__ __noinline__ void w_small_values(const float2* A, const uint16_t* nb, const float2* st,
                                            float2 u0s, uint8_t sel, const float2* psi,
                                            float2* out) {
  DF sum[kSmallM];
#pragma unroll
  for (int l = 0; l < kSmallM; ++l) sum[l] = DF{0.f, 0.f};
  for (int k = 0; k < kSmallK; ++k) {
    if (!((sel >> k) & 1)) continue;
    DF as[kSmallM];
#pragma unroll
    for (int l = 0; l < kSmallM; ++l) as[l] = DF{0.f, 0.f};
    for (int s = 0; s < kSmallN; ++s) {
      const DF d = halo_dif(st, nb[(NS + k * kSmallN + s) * kTile] & kHaloPosMask, u0s);
      const float2* As = A + (int64_t)(M * NS + (k * kSmallN + s) * kSmallM) * kTile;
#pragma unroll
      for (int l = 0; l < kSmallM; ++l) df_mac(as[l], __ldg(As + l * kTile), d);
    }
#pragma unroll
    for (int l = 0; l < kSmallM; ++l) {
      const DF x = df_norm(as[l]);
      DF q = two_sum(sum[l].h, x.h);
      q.l += sum[l].l + x.l;
      sum[l] = two_sum(q.h, q.l);
    }
  }
  // divide by the number of kept stencils (exact remainder correction)
  const int nd = (sel & 1) + ((sel >> 1) & 1) + ((sel >> 2) & 1);
  const float fn = (float)(nd ? nd : 1);
  DF cf[kSmallM];
#pragma unroll
  for (int l = 0; l < kSmallM; ++l) {
    const float qh = sum[l].h / fn;
    const float r = fmaf(-qh, fn, sum[l].h);
    cf[l] = nd ? two_sum(qh, (r + sum[l].l) / fn) : DF{0.f, 0.f};
  }
  const DF u0 = {u0s.x, u0s.y};
  for (int p = 0; p < NQ3; ++p) {
    DF sp = {0.f, 0.f};
#pragma unroll
    for (int l = 0; l < kSmallM; ++l) df_mac(sp, __ldg(psi + p * kMaxM + l), cf[l]);
    const DF r = u0 + df_norm(sp);
    out[p * NV] = make_float2(r.h, r.l);
  }
}

// The same two rare paths on the FP64 pipe (native FP64 W form): A is the
// cell's FP64 matrices at its lane, st the tile's halo of FP64 states.
template <int M, int NS>
__device__ __noinline__ uint8_t w_select_native(const double* A, const uint16_t* nb,
                                                const double* st, double u0, int present,
                                                double ct, double eps) {
  double al[M];
#pragma unroll
  for (int l = 0; l < M; ++l) al[l] = 0.0;
  for (int s = 0; s < NS; ++s) {
    const double d = st[nb[s * kTile] & kHaloPosMask] - u0;
#pragma unroll
    for (int l = 0; l < M; ++l) al[l] = fma(__ldg(A + (int64_t)(s * M + l) * kTile), d, al[l]);
  }
  double beta[kSmallK + 1];
  {
    double b = 0.0;
#pragma unroll
    for (int l = 0; l < M; ++l) b = fma(al[l], al[l], b);
    beta[kSmallK] = b;
  }
#pragma unroll
  for (int k = 0; k < kSmallK; ++k) {
    double as[kSmallM];
#pragma unroll
    for (int l = 0; l < kSmallM; ++l) as[l] = 0.0;
    if ((present >> k) & 1) {
      for (int s = 0; s < kSmallN; ++s) {
        const double d = st[nb[(NS + k * kSmallN + s) * kTile] & kHaloPosMask] - u0;
        const double* As = A + (int64_t)(M * NS + (k * kSmallN + s) * kSmallM) * kTile;
#pragma unroll
        for (int l = 0; l < kSmallM; ++l) as[l] = fma(__ldg(As + l * kTile), d, as[l]);
      }
    }
    double q = 0.0;
#pragma unroll
    for (int l = 0; l < kSmallM; ++l) q = fma(as[l], as[l], q);
    beta[k] = q;
  }
  return select_fp64(beta, present, ct, eps);
}

template <int M, int NS, int NQ3, int NV>
__device__ __noinline__ void w_small_native(const double* A, const uint16_t* nb, const double* st,
                                            double u0, uint8_t sel, const double* psi,
                                            double* out) {
  double sum[kSmallM];
#pragma unroll
  for (int l = 0; l < kSmallM; ++l) sum[l] = 0.0;
  for (int k = 0; k < kSmallK; ++k) {
    if (!((sel >> k) & 1)) continue;
    double as[kSmallM];
#pragma unroll
    for (int l = 0; l < kSmallM; ++l) as[l] = 0.0;
    for (int s = 0; s < kSmallN; ++s) {
      const double d = st[nb[(NS + k * kSmallN + s) * kTile] & kHaloPosMask] - u0;
      const double* As = A + (int64_t)(M * NS + (k * kSmallN + s) * kSmallM) * kTile;
#pragma unroll
      for (int l = 0; l < kSmallM; ++l) as[l] = fma(__ldg(As + l * kTile), d, as[l]);
    }
#pragma unroll
    for (int l = 0; l < kSmallM; ++l) sum[l] += as[l];
  }
  const int nd = (sel & 1) + ((sel >> 1) & 1) + ((sel >> 2) & 1);
  double cf[kSmallM];
#pragma unroll
  for (int l = 0; l < kSmallM; ++l) cf[l] = nd ? sum[l] / (double)nd : 0.0;
  for (int p = 0; p < NQ3; ++p) {
    double sp = 0.0;
#pragma unroll
    for (int l = 0; l < kSmallM; ++l) sp = fma(__ldg(psi + p * kMaxM + l), cf[l], sp);
    out[p * NV] = u0 + sp;
  }
}

// kN = false: the FP64 path in pairs (halo, W and Gauss values as (hi, lo)
// FP32 pairs); kN = true: the native FP64 path (FP64 halo, W and values, the
// multiply-adds on the FP64 pipe).  The FP32 cutoff screen is the same.
template <int M, int NS, int NQ, bool kN>
__global__ void __launch_bounds__(kTile * (kConsumers + 1), (WPlan<M, NS, 3 * NQ, 3, 4>::kBlocks))
    recon_tma_w_kernel(const ReconArgs a, const HaloArgs h, const void* __restrict__ psi_v,
                       const float* __restrict__ g32, const void* __restrict__ wq, int* err) {
  // 8-byte elements either way: halo states, W entries, Gauss-point values
  using HT = typename std::conditional<kN, double, float2>::type;
  using Acc = typename std::conditional<kN, double, DF>::type;
  constexpr int NQ3 = 3 * NQ;
  using P = WPlan<M, NS, NQ3, 3, 4>;
  constexpr int kR = P::kRingW;
  constexpr int NV = 4;
  constexpr int SL = NS + kSmallSlots;
  constexpr int E = M * NS + kSmallEntries;
  constexpr int kPer = NQ3 * NV;  // Gauss-point pairs per cell
  extern __shared__ __align__(128) unsigned char smem[];
  HT* halo = reinterpret_cast<HT*>(smem + (size_t)kR * P::kMat);  // [2][NV][kHaloMax]
  HT* ostg = reinterpret_cast<HT*>(smem + P::kOutOff);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)kR * P::kMat + P::kHaloBytes);
  uint64_t* empty = full + kR;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + kR);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n_tiles = (a.n_cell + kTile - 1) / kTile;
  if (threadIdx.x == 0) {
    *abort_flag = 0;
    for (int i = 0; i < kR; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kConsumers);
    }
    mbar_fence_init();
  }
  __syncthreads();
  if (warp == kConsumers) {
    // ---- producer lane: FP32 and W blocks of every tile
    if (lane == 0) {
      int64_t g = 0;
      for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const unsigned char* sg =
            reinterpret_cast<const unsigned char*>(g32) + tile * (int64_t)P::kE32 * kTile * 4;
        const unsigned char* sw =
            reinterpret_cast<const unsigned char*>(wq) + tile * (int64_t)P::kEW * kTile * 8;
        const unsigned char* sn =
            reinterpret_cast<const unsigned char*>(h.nbr_loc) + tile * (int64_t)P::kSL * P::kSlotN;
        for (int j = 0; j < P::kStages; ++j, ++g) {
          const int b = (int)(g % kR);
          if (g >= kR) {
            const int w = mbar_wait_or_abort(&empty[b], (uint32_t)((g / kR) - 1) & 1, abort_flag);
            if (w != 1) {
              if (w == 0) {
                atomicOr(err, 2);
                *abort_flag = 1;
              }
              for (int64_t i = g - kR; i < g; ++i) mbar_wait(&full[i % kR], (uint32_t)(i / kR) & 1);
              return;
            }
          }
          int slot0, nslot, k, og, bg, ow, bw;
          P::stage(j, slot0, nslot, k, og, bg, ow, bw);
          unsigned char* dst = smem + (size_t)b * P::kMat;
          const uint32_t bn = (uint32_t)(nslot * P::kSlotN);
          mbar_expect_tx(&full[b], (uint32_t)(bg + bw) + bn);
          bulk_g2s(dst, sg + og, (uint32_t)bg, &full[b]);
          if (bw) bulk_g2s(dst + P::kWOff, sw + ow, (uint32_t)bw, &full[b]);
          bulk_g2s(dst + P::kNOff, sn + slot0 * P::kSlotN, bn, &full[b]);
        }
      }
      // the block must not exit while a copy it issued is in flight
      for (int64_t i = g > kR ? g - kR : 0; i < g; ++i)
        mbar_wait(&full[i % kR], (uint32_t)(i / kR) & 1);
    }
    return;
  }
  // ---- consumers (the halo pipeline of recon_tma_kernel measured slower
  // here: this kernel is at its register limit)
  const int v = warp, tid = threadIdx.x;
  auto prefetch = [&](int64_t tile, int hb) {
    const int h0 = h.off[tile], H = h.off[tile + 1] - h0;
    for (int i = tid; i < H; i += kConsumers * kTile) {
      const int id = __ldg(h.ids + h0 + i);
#pragma unroll
      for (int w = 0; w < NV; ++w) {
        const void* src;
        if constexpr (kN)
          src = a.U + (int64_t)w * a.n_pad + id;
        else
          src = a.Us + (int64_t)w * a.n_pad + id;
        cp_async8(&halo[(hb * NV + w) * kHaloMax + i], src);
      }
    }
    cp_async_commit();
  };
  int64_t g = 0;
  int hb = 0;
  bool dead = false;  // a bounded wait of this block gave up: skip all work
  if ((int64_t)blockIdx.x < n_tiles) prefetch(blockIdx.x, 0);
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, hb ^= 1) {
    consumer_sync();  // every consumer is done with the other halo buffer
    const int64_t nxt = tile + gridDim.x;
    if (nxt < n_tiles)
      prefetch(nxt, hb ^ 1);
    else
      cp_async_commit();
    cp_async_wait<1>();
    consumer_sync();
    const HT* st = halo + (hb * NV + v) * kHaloMax;
    const uint16_t* nb = h.nbr_loc + tile * (int64_t)SL * kTile + lane;
    const int64_t c = tile * kTile + lane;  // may be a pad lane of the last tile
    HT u0s;
    if constexpr (kN)
      u0s = a.U[(int64_t)v * a.n_pad + (c < a.n_cell ? c : 0)];
    else
      u0s = a.Us[(int64_t)v * a.n_pad + (c < a.n_cell ? c : 0)];
    auto dif = [&](int idx) -> Acc {  // d_s = U_s - U_0 (pairs, or FP64)
      if constexpr (kN) {
        return st[idx] - u0s;
      } else {
        const float2 q = st[idx];
        DF t = two_sum(q.x, -u0s.x);
        t.l += q.y - u0s.y;
        return two_sum(t.h, t.l);
      }
    };
    float a32[M], s32[kSmallK][kSmallM], eL = 0.f, eS[kSmallK];
    Acc uq[NQ3];
#pragma unroll
    for (int l = 0; l < M; ++l) a32[l] = 0.f;
#pragma unroll
    for (int k = 0; k < kSmallK; ++k) {
      eS[k] = 0.f;
#pragma unroll
      for (int l = 0; l < kSmallM; ++l) s32[k][l] = 0.f;
    }
#pragma unroll
    for (int p = 0; p < NQ3; ++p) uq[p] = Acc{};
    // selection and Gauss-point values of cell c (after all stages of its tile)
    auto finish_cell = [&](int64_t tile, int64_t c) {
      const int present = a.smask[c];
      const HT* A = reinterpret_cast<const HT*>(a.ahat) + tile * (int64_t)E * kTile + lane;
      uint8_t sel;
      if (a.sel_in) {
        sel = a.sel_in[(int64_t)v * a.n_pad + c];
      } else if (a.linear) {
        sel = 8;
      } else {
        float t[kSmallK + 1];
        float rho = 0.f;
        {
          float bsum = 0.f;
#pragma unroll
          for (int l = 0; l < M; ++l) bsum = fmaf(a32[l], a32[l], bsum);
          t[kSmallK] = bsum + (float)a.eps;
          rho = beta_rel_bound(bsum, eL, NS, M, (float)a.eps);
#pragma unroll
          for (int k = 0; k < kSmallK; ++k) {
            float q = 0.f;
#pragma unroll
            for (int l = 0; l < kSmallM; ++l) q = fmaf(s32[k][l], s32[k][l], q);
            t[k] = q + (float)a.eps;
            if ((present >> k) & 1)
              rho = fmaxf(rho, beta_rel_bound(q, eS[k], kSmallN, kSmallM, (float)a.eps));
          }
        }
        // chi lies within the factor f of its FP32 value under the beta bounds
        bool near = a.force_near || !(rho < 0.25f);
        const float q = (1.f + rho) / (1.f - fminf(rho, 0.5f));
        const float q2 = q * q;
        const float f = q2 * q2 * q2 * 1.0001f;
        const float ct = (float)a.ct;
        if (chi_keep32_bound(t, kSmallK, present | 8, ct, f, &near)) {
          sel = 8;
        } else {
          sel = 0;
#pragma unroll
          for (int k = 0; k < kSmallK; ++k)
            if (((present >> k) & 1) && chi_keep32_bound(t, k, present & 7, ct, f, &near))
              sel |= (uint8_t)(1u << k);
        }
        if (near) {
          if constexpr (kN)
            sel = w_select_native<M, NS>(A, nb, st, u0s, present, a.ct, a.eps);
          else
            sel = w_select_pairs<M, NS>(A, nb, st, u0s, present, a.ct, a.eps);
        }
      }
      if (a.sel_out) a.sel_out[(int64_t)v * a.n_pad + c] = sel;
      // Gauss-point values ((hi, lo) pairs or FP64), to the output stage or to Uq
      HT* __restrict__ out = TENO_STAGE_OUT_W ? ostg + lane * (kPer + 1) + v
                                              : reinterpret_cast<HT*>(a.Uq) + c * kPer + v;
      if (sel & 8) {
        if constexpr (kN) {
#pragma unroll
          for (int p = 0; p < NQ3; ++p) out[p * NV] = u0s + uq[p];
        } else {
          const DF u0 = {u0s.x, u0s.y};
#pragma unroll
          for (int p = 0; p < NQ3; ++p) {
            const DF r = u0 + df_norm(uq[p]);
            out[p * NV] = make_float2(r.h, r.l);
          }
        }
      } else {
        if constexpr (kN)
          w_small_native<M, NS, NQ3, NV>(A, nb, st, u0s, sel,
                                         reinterpret_cast<const double*>(psi_v), out);
        else
          w_small_values<M, NS, NQ3, NV>(A, nb, st, u0s, sel,
                                         reinterpret_cast<const float2*>(psi_v), out);
      }
    };
    for (int j = 0; j < P::kStages; ++j, ++g) {
      const int b = (int)(g % kR);
      int slot0, nslot, k, og, bg, ow, bw;
      P::stage(j, slot0, nslot, k, og, bg, ow, bw);
      if (!dead) {
        const int w = mbar_wait_or_abort(&full[b], (uint32_t)(g / kR) & 1, abort_flag, a.wait_polls);
        if (w == 0) {
          atomicOr(err, 2);
          *abort_flag = 1;
        }
        dead = __any_sync(0xffffffffu, w != 1);
      }
      const unsigned char* buf = smem + (size_t)b * P::kMat;
      const uint16_t* nl = reinterpret_cast<const uint16_t*>(buf + P::kNOff) + lane;
      if (dead) {
        // skip the stage
      } else if (k < 0) {
        const float* gm = reinterpret_cast<const float*>(buf) + lane;
        const HT* wm = reinterpret_cast<const HT*>(buf + P::kWOff) + lane;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
          if (s < nslot) {
            const Acc d = dif(nl[s * kTile] & kHaloPosMask);
            float dh;
            if constexpr (kN)
              dh = d2f_trunc(d);
            else
              dh = d.h;
#pragma unroll
            for (int l = 0; l < M; ++l) a32[l] = fmaf(gm[(s * P::kG + l) * kTile], dh, a32[l]);
            eL = fmaf(gm[(s * P::kG + M) * kTile], fabsf(dh), eL);
#pragma unroll
            for (int p = 0; p < NQ3; ++p) {
              if constexpr (kN)
                uq[p] = fma(wm[(s * NQ3 + p) * kTile], d, uq[p]);
              else
                df_mac(uq[p], wm[(s * NQ3 + p) * kTile], d);
            }
          }
        }
      } else {
        const float* gm = reinterpret_cast<const float*>(buf) + lane;
#pragma unroll
        for (int kk = 0; kk < kSmallK; ++kk) {
          if (kk != k) continue;
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            const HT q = st[nl[s * kTile] & kHaloPosMask];
            float dh;
            if constexpr (kN)
              dh = d2f_trunc(q - u0s);
            else
              dh = (q.x - u0s.x) + (q.y - u0s.y);
#pragma unroll
            for (int l = 0; l < kSmallM; ++l)
              s32[kk][l] = fmaf(gm[(s * P::kGs + l) * kTile], dh, s32[kk][l]);
            eS[kk] = fmaf(gm[(s * P::kGs + kSmallM) * kTile], fabsf(dh), eS[kk]);
          }
        }
      }
      __syncwarp();
      if (lane == 0 && !dead) mbar_arrive(&empty[b]);
    }
    if (!dead && c < a.n_cell) finish_cell(tile, c);
    if constexpr (TENO_STAGE_OUT_W != 0) {
      consumer_sync();  // the tile's values are staged
      if (!dead)
        store_out_stage<kPer>(ostg, reinterpret_cast<HT*>(a.Uq) + tile * kTile * kPer,
                              (int)min((int64_t)kTile, a.n_cell - tile * kTile), tid);
    }
  }
  cp_async_wait<0>();
}

// ------------------------------------ characteristic variables (charvar)
// Characteristic reconstruction (Sec. 2.3 prefers characteristic variables):
// thread (cell, local edge e).  The coefficients of the four conservative
// variables are projected on the characteristic fields of the edge's outward
// normal at the cell-average state, L = L' T and R = T^T R' with T the
// rotation to the edge frame and L', R' the textbook eigenvectors of the 1D
// Euler flux Jacobian in that frame (fields u-c, entropy, shear, u+c).  Each
// field takes its own TENO selection (select_fp64), and the edge's Gauss-point
// values are U_0 + R (Psi' c~).  FP64 throughout; the values are stored in the
// path's Gauss-point type.
template <typename TQ>
__device__ __forceinline__ TQ from_d(double x) {
  if constexpr (std::is_same<TQ, DF>::value) {
    const float h = (float)x;
    return DF{h, (float)(x - (double)h)};
  } else {
    return (TQ)x;
  }
}

template <int M, int NQ, typename TQ>
__global__ void __launch_bounds__(128) char_finish_kernel(
    const double* __restrict__ coef, const double* __restrict__ U,
    const uint8_t* __restrict__ smask, const int32_t* __restrict__ c_faces,
    const double* __restrict__ f_geom, const EvalTable ev, TQ* __restrict__ Uq, int64_t n_cell,
    int64_t n_pad, double g, double ct, double eps, int linear) {
  constexpr int C = M + kSmallK * kSmallM;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_cell * 3) return;
  const int64_t c = idx / 3;
  const int e = (int)(idx % 3);
  const int cf = c_faces[3 * c + e];
  const int64_t f = cf >> 1;
  const double sg = (cf & 1) ? -1.0 : 1.0;  // the neighbour's normal is the opposite one
  const double nx = sg * f_geom[5 * f], ny = sg * f_geom[5 * f + 1];
  double W[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) W[v] = U[(int64_t)v * n_pad + c];
  // eigenvectors at the cell average
  const double r = W[0], un = (W[1] * nx + W[2] * ny) / r, ut = (W[2] * nx - W[1] * ny) / r;
  const double q2 = un * un + ut * ut, p = (g - 1.0) * (W[3] - 0.5 * r * q2);
  const double cs = sqrt(g * p / r), H = (W[3] + p) / r;
  const double b1 = (g - 1.0) / (cs * cs), b2 = 0.5 * b1 * q2;
  const double Lf[4][4] = {
      {0.5 * (b2 + un / cs), 0.5 * (-b1 * un - 1.0 / cs), -0.5 * b1 * ut, 0.5 * b1},
      {1.0 - b2, b1 * un, b1 * ut, -b1},
      {-ut, 0.0, 1.0, 0.0},
      {0.5 * (b2 - un / cs), 0.5 * (-b1 * un + 1.0 / cs), -0.5 * b1 * ut, 0.5 * b1}};
  const double Rf[4][4] = {{1.0, 1.0, 0.0, 1.0},
                           {un - cs, un, 0.0, un + cs},
                           {ut, ut, 1.0, ut},
                           {H - un * cs, 0.5 * q2, ut, H + un * cs}};
  // L = L' T, R = T^T R' with T = rotation (m_x, m_y) -> (m_n, m_t)
  double L[4][4], R[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    L[i][0] = Lf[i][0];
    L[i][1] = Lf[i][1] * nx - Lf[i][2] * ny;
    L[i][2] = Lf[i][1] * ny + Lf[i][2] * nx;
    L[i][3] = Lf[i][3];
    R[0][i] = Rf[0][i];
    R[1][i] = nx * Rf[1][i] - ny * Rf[2][i];
    R[2][i] = ny * Rf[1][i] + nx * Rf[2][i];
    R[3][i] = Rf[3][i];
  }
  const int present = smask[c];
  const double* cv = coef + c * 4 * C;
  // coefficient l of characteristic field i (recomputed where it is needed:
  // holding a field's C coefficients, and the full L and R, spilled)
  auto chc = [&](int i, int l) {
    return L[i][0] * cv[l] + L[i][1] * cv[C + l] + L[i][2] * cv[2 * C + l] + L[i][3] * cv[3 * C + l];
  };
  double corr[4][NQ];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int q = 0; q < NQ; ++q) corr[v][q] = 0.0;
#pragma unroll 1
  for (int i = 0; i < 4; ++i) {
    uint8_t sel = 8;
    if (!linear) {
      double beta[kSmallK + 1];
      double b = 0.0;
#pragma unroll 4
      for (int l = 0; l < M; ++l) {
        const double x = chc(i, l);
        b = fma(x, x, b);
      }
      beta[kSmallK] = b;
#pragma unroll
      for (int k = 0; k < kSmallK; ++k) {
        double bq = 0.0;
#pragma unroll
        for (int l = 0; l < kSmallM; ++l) {
          const double x = chc(i, M + k * kSmallM + l);
          bq = fma(x, x, bq);
        }
        beta[k] = bq;
      }
      sel = select_fp64(beta, present, ct, eps);
    }
    double gq[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) gq[q] = 0.0;
    if (sel & 8) {
#pragma unroll 4
      for (int l = 0; l < M; ++l) {
        const double x = chc(i, l);
#pragma unroll
        for (int q = 0; q < NQ; ++q) gq[q] = fma(x, ev.psi[(e * NQ + q) * kMaxM + l], gq[q]);
      }
    } else {
      // equal weights over the kept directional quadratics (kSmallM terms)
      const int nd = (sel & 1) + ((sel >> 1) & 1) + ((sel >> 2) & 1);
      const double w = nd ? 1.0 / nd : 0.0;
      double cfin[kSmallM];
#pragma unroll
      for (int l = 0; l < kSmallM; ++l) cfin[l] = 0.0;
#pragma unroll
      for (int k = 0; k < kSmallK; ++k) {
        if (!((sel >> k) & 1)) continue;
#pragma unroll
        for (int l = 0; l < kSmallM; ++l) cfin[l] = fma(w, chc(i, M + k * kSmallM + l), cfin[l]);
      }
#pragma unroll
      for (int l = 0; l < kSmallM; ++l)
#pragma unroll
        for (int q = 0; q < NQ; ++q) gq[q] = fma(cfin[l], ev.psi[(e * NQ + q) * kMaxM + l], gq[q]);
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
      for (int v = 0; v < 4; ++v) corr[v][q] = fma(R[v][i], gq[q], corr[v][q]);
  }
  TQ* out = Uq + ((int64_t)(c * 3 + e) * NQ) * 4;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int v = 0; v < 4; ++v) out[q * 4 + v] = from_d<TQ>(W[v] + corr[v][q]);
}

// The characteristic finish of the pair and mixed paths in pair arithmetic
// on the FP32 pipe (the FP64 version above is FP64-pipe bound): the same
// steps, from the (hi, lo) coefficients the reconstruction wrote.  The
// selection is screened in FP32 with the guard band of the pair path and
// decided in FP64 inside it; the Gauss values are written as pairs (pair
// path) or FP32 (mixed path).
template <int M, int NQ, typename TQ>
__global__ void __launch_bounds__(128) char_finish_df_kernel(
    const float2* __restrict__ coef, const double* __restrict__ U,
    const uint8_t* __restrict__ smask, const int32_t* __restrict__ c_faces,
    const double* __restrict__ f_geom, const DFTable ev, TQ* __restrict__ Uq, int64_t n_cell,
    int64_t n_pad, double g, double ct, double eps, int linear) {
  constexpr int C = M + kSmallK * kSmallM;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_cell * 3) return;
  const int64_t c = idx / 3;
  const int e = (int)(idx % 3);
  const int cf = c_faces[3 * c + e];
  const int64_t f = cf >> 1;
  const double sg = (cf & 1) ? -1.0 : 1.0;  // the neighbour's normal is the opposite one
  const DF nx = cst<DF>(sg * f_geom[5 * f]), ny = cst<DF>(sg * f_geom[5 * f + 1]);
  const DF one = {1.f, 0.f}, half = {0.5f, 0.f}, zero = {0.f, 0.f};
  const DF gm1 = cst<DF>(g - 1.0), gg = cst<DF>(g);
  DF W[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) W[v] = cst<DF>(U[(int64_t)v * n_pad + c]);
  // eigenvectors at the cell average, in the edge frame, then rotated
  const DF ir = one / W[0];
  const DF un = (W[1] * nx + W[2] * ny) * ir, ut = (W[2] * nx - W[1] * ny) * ir;
  const DF q2 = un * un + ut * ut;
  const DF p = gm1 * (W[3] - half * W[0] * q2);
  const DF cs = tsqrt(gg * p * ir), ics = one / cs, H = (W[3] + p) * ir;
  const DF b1 = gm1 * ics * ics, b2 = half * b1 * q2;
  const DF Lf[4][4] = {{half * (b2 + un * ics), half * (-(b1 * un) - ics), -(half * b1 * ut), half * b1},
                       {one - b2, b1 * un, b1 * ut, -b1},
                       {-ut, zero, one, zero},
                       {half * (b2 - un * ics), half * (-(b1 * un) + ics), -(half * b1 * ut), half * b1}};
  const DF Rf[4][4] = {{one, one, zero, one},
                       {un - cs, un, zero, un + cs},
                       {ut, ut, one, ut},
                       {H - un * cs, half * q2, ut, H + un * cs}};
  DF L[4][4], R[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    L[i][0] = Lf[i][0];
    L[i][1] = Lf[i][1] * nx - Lf[i][2] * ny;
    L[i][2] = Lf[i][1] * ny + Lf[i][2] * nx;
    L[i][3] = Lf[i][3];
    R[0][i] = Rf[0][i];
    R[1][i] = nx * Rf[1][i] - ny * Rf[2][i];
    R[2][i] = ny * Rf[1][i] + nx * Rf[2][i];
    R[3][i] = Rf[3][i];
  }
  const int present = smask[c];
  const float2* cv = coef + c * 4 * C;
  auto cp = [&](int j) { const float2 x = cv[j]; return DF{x.x, x.y}; };
  // coefficient l of characteristic field i (recomputed where it is needed)
  auto chc = [&](int i, int l) {
    return ((L[i][0] * cp(l) + L[i][1] * cp(C + l)) + L[i][2] * cp(2 * C + l)) +
           L[i][3] * cp(3 * C + l);
  };
  DF corr[4][NQ];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int q = 0; q < NQ; ++q) corr[v][q] = zero;
#pragma unroll 1
  for (int i = 0; i < 4; ++i) {
    uint8_t sel = 8;
    if (!linear) {
      DF bt[kSmallK + 1];
      {
        DF b = zero;
#pragma unroll 4
        for (int l = 0; l < M; ++l) {
          const DF x = chc(i, l);
          df_mac(b, make_float2(x.h, x.l), x);
        }
        bt[kSmallK] = df_norm(b);
#pragma unroll
        for (int k = 0; k < kSmallK; ++k) {
          DF q = zero;
#pragma unroll
          for (int l = 0; l < kSmallM; ++l) {
            const DF x = chc(i, M + k * kSmallM + l);
            df_mac(q, make_float2(x.h, x.l), x);
          }
          bt[k] = df_norm(q);
        }
      }
      float t[kSmallK + 1];
#pragma unroll
      for (int k = 0; k <= kSmallK; ++k) t[k] = bt[k].h + (float)eps;
      bool near = false;
      if (chi_keep32(t, kSmallK, present | 8, (float)ct, &near)) {
        sel = 8;
      } else {
        sel = 0;
#pragma unroll
        for (int k = 0; k < kSmallK; ++k)
          if (((present >> k) & 1) && chi_keep32(t, k, present & 7, (float)ct, &near))
            sel |= (uint8_t)(1u << k);
      }
      if (near) {
        double beta[kSmallK + 1];
#pragma unroll
        for (int k = 0; k <= kSmallK; ++k) beta[k] = df_to_double(bt[k]);
        sel = select_fp64(beta, present, ct, eps);
      }
    }
    DF gq[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) gq[q] = zero;
    if (sel & 8) {
#pragma unroll 4
      for (int l = 0; l < M; ++l) {
        const DF x = chc(i, l);
#pragma unroll
        for (int q = 0; q < NQ; ++q) df_mac(gq[q], ev.psi[(e * NQ + q) * kMaxM + l], x);
      }
    } else {
      // equal weights over the kept directional quadratics (kSmallM terms)
      const int nd = (sel & 1) + ((sel >> 1) & 1) + ((sel >> 2) & 1);
      const DF fn = {(float)(nd ? nd : 1), 0.f};
#pragma unroll
      for (int l = 0; l < kSmallM; ++l) {
        DF sum = zero;
#pragma unroll
        for (int k = 0; k < kSmallK; ++k)
          if ((sel >> k) & 1) sum = sum + chc(i, M + k * kSmallM + l);
        const DF x = nd ? sum / fn : zero;
#pragma unroll
        for (int q = 0; q < NQ; ++q) df_mac(gq[q], ev.psi[(e * NQ + q) * kMaxM + l], x);
      }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const DF gn = df_norm(gq[q]);
#pragma unroll
      for (int v = 0; v < 4; ++v) corr[v][q] = corr[v][q] + R[v][i] * gn;
    }
  }
  TQ* out = Uq + ((int64_t)(c * 3 + e) * NQ) * 4;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const DF r = W[v] + corr[v][q];
      if constexpr (std::is_same<TQ, DF>::value)
        out[q * 4 + v] = r;
      else
        out[q * 4 + v] = r.h;
    }
}

// FP32 hi/lo split of a state: hi = fl32(U), lo = fl32(U - hi)
// Positivity scaling of the reconstruction (Euler; an option, not in the
// paper, which reports its schemes robust on the Mach-10 shock case without
// stating a positivity treatment): Zhang and Shu's limiter.  Each cell's
// Gauss-point states U_q move towards the cell average, U_0 + theta (U_q -
// U_0), with the largest theta <= 1 that keeps the density, then the
// pressure, at least eps = min(1e-13, the average's value) at every face
// Gauss point of the cell.  The reconstruction is linear in its coefficients,
// so scaling the point values equals scaling the polynomial's deviation from
// its mean (the average is unchanged).  Density: theta = (rho_0 - eps) /
// (rho_0 - rho_q) where rho_q < eps; pressure (concave along the segment from
// the average): 60 bisection halvings of [0, 1].  FP64; one thread per cell.
__device__ __forceinline__ double pp_pressure(double g, const double* W) {
  return (g - 1.0) * (W[3] - 0.5 * (W[1] * W[1] + W[2] * W[2]) / W[0]);
}

template <int NQ, typename TQ>
__global__ void __launch_bounds__(128) positivity_kernel(const double* __restrict__ U,
                                                         TQ* __restrict__ Uq, int64_t n_cell,
                                                         int64_t n_pad, double g) {
  constexpr int NP = 3 * NQ;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cell) return;
  double U0[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) U0[v] = U[v * n_pad + c];
  const double er = fmin(1e-13, U0[0]), ep = fmin(1e-13, pp_pressure(g, U0));
  TQ* q0 = Uq + c * NP * 4;
  double W[NP][4];
#pragma unroll
  for (int q = 0; q < NP; ++q)
#pragma unroll
    for (int v = 0; v < 4; ++v) W[q][v] = to_d(q0[q * 4 + v]);
  bool scaled = false;
  // pass 0: density
  double th = 1.0;
#pragma unroll
  for (int q = 0; q < NP; ++q)
    if (W[q][0] < er) th = fmin(th, (U0[0] - er) / (U0[0] - W[q][0]));
  if (th < 1.0) {
    scaled = true;
#pragma unroll
    for (int q = 0; q < NP; ++q)
#pragma unroll
      for (int v = 0; v < 4; ++v) W[q][v] = U0[v] + th * (W[q][v] - U0[v]);
  }
  // pass 1: pressure
  th = 1.0;
  for (int q = 0; q < NP; ++q) {
    if (pp_pressure(g, W[q]) >= ep) continue;
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 60; ++it) {
      const double sm = 0.5 * (lo + hi);
      double X[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) X[v] = U0[v] + sm * (W[q][v] - U0[v]);
      if (X[0] > 0.0 && pp_pressure(g, X) >= ep)
        lo = sm;
      else
        hi = sm;
    }
    th = fmin(th, lo);
  }
  if (th < 1.0) {
    scaled = true;
#pragma unroll
    for (int q = 0; q < NP; ++q)
#pragma unroll
      for (int v = 0; v < 4; ++v) W[q][v] = U0[v] + th * (W[q][v] - U0[v]);
  }
  if (!scaled) return;
#pragma unroll
  for (int q = 0; q < NP; ++q)
#pragma unroll
    for (int v = 0; v < 4; ++v) q0[q * 4 + v] = from_d<TQ>(W[q][v]);
}

// The outflow layer (cells with a face on an outflow boundary) enters every
// face flux with its cell average: after the reconstruction, each Gauss slot
// of such a cell takes U_0 (in the Gauss-value type of the path).  One thread
// per (layer cell, slot).
template <int NV, int NQ3, typename TQ>
__global__ void layer_fill_kernel(const double* __restrict__ U, TQ* __restrict__ Uq,
                                  const int32_t* __restrict__ list, int64_t n, int64_t n_pad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * NQ3) return;
  const int64_t c = list[i / NQ3];
  const int p = (int)(i % NQ3);
  TQ* o = Uq + (c * NQ3 + p) * NV;
#pragma unroll
  for (int v = 0; v < NV; ++v) o[v] = from_d<TQ>(U[v * n_pad + c]);
}

// Adjoint of layer_fill_kernel: a layer cell's Gauss-slot cotangents (pairs
// on the pair path, FP64 otherwise) go to its cell average, summed per edge
// into ubd[cell][edge][var] (added to the cell's adjoint by the reverse
// gather), and the slots are cleared so that the reconstruction's adjoint
// sends nothing through the cell's polynomial.  One thread per (cell, edge).
template <int NV, int NQ, bool kPairs>
__global__ void layer_vjp_kernel(double* __restrict__ Uq_bar, double* __restrict__ ubd,
                                 const int32_t* __restrict__ list, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * 3) return;
  const int64_t c = list[i / 3];
  const int e = (int)(i % 3);
  double acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  const int64_t b = ((c * 3 + e) * NQ) * NV;
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int64_t j = b + q * NV + v;
      if constexpr (kPairs) {
        float2* u = reinterpret_cast<float2*>(Uq_bar) + j;
        acc[v] += (double)u->x + (double)u->y;
        *u = make_float2(0.f, 0.f);
      } else {
        acc[v] += Uq_bar[j];
        Uq_bar[j] = 0.0;
      }
    }
#pragma unroll
  for (int v = 0; v < NV; ++v) ubd[(c * 3 + e) * NV + v] = acc[v];
}

// Halo exchange of partitioned meshes (copy-based; each kernel touches only
// its own context's arrays).  pack: buf[v][i] = U[v][idx[i]]; unpack: the
// reverse, with the FP32 hi/lo split of the written states when Us is given;
// add = 1 adds instead (the adjoint's contributions returned to their owner).
__global__ void halo_pack_kernel(const double* __restrict__ U, int64_t ld,
                                 const int32_t* __restrict__ idx, int64_t n, int n_var,
                                 double* __restrict__ buf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t c = idx[i];
  for (int v = 0; v < n_var; ++v) buf[v * n + i] = U[v * ld + c];
}
__global__ void halo_unpack_kernel(double* __restrict__ U, int64_t ld,
                                   const int32_t* __restrict__ idx, int64_t n, int n_var,
                                   const double* __restrict__ buf, float2* __restrict__ Us,
                                   int add) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t c = idx[i];
  for (int v = 0; v < n_var; ++v) {
    const double x = add ? U[v * ld + c] + buf[v * n + i] : buf[v * n + i];
    U[v * ld + c] = x;
    if (Us) {
      const float hi = (float)x;
      Us[v * ld + c] = make_float2(hi, (float)(x - (double)hi));
    }
  }
}

__global__ void split_kernel(const double* __restrict__ U, float2* __restrict__ Us, int64_t n_cell,
                             int64_t n_pad, int n_var) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cell) return;
  for (int v = 0; v < n_var; ++v) {
    const double u = U[v * n_pad + c];
    const float hi = (float)u;
    Us[v * n_pad + c] = make_float2(hi, (float)(u - (double)hi));
  }
}

// ------------------------------------------------------------------ fluxes
struct FaceArgs {
  const int32_t* f_cells;
  const int8_t* f_edges;
  const double* f_geom;
  const float2* f_geom2;  // [n_face][3] nx, ny, |A| as (hi, lo) pairs
  int64_t n_pad;
  int64_t n_face;
  double gamma, adv_x, adv_y, time;
  int adv_field;
  double adv_cx, adv_cy, adv_omega, adv_r1, adv_r2;
  double gw[kMaxNq], gt[kMaxNq];
  float2 gw2[kMaxNq], g2, gm12;  // Gauss weights, gamma, gamma - 1 as pairs
};

// face constants in the flux scalar type: FP64 from the double geometry,
// pairs and floats from the copy split on the host (no FP64 conversions)
template <typename T>
__device__ __forceinline__ void face_k(const double* fg, const float2* fg2, int64_t f, double g,
                                       float2 g2, float2 gm12, RiemannK<T>& rk, T& tl) {
  if constexpr (std::is_same<T, double>::value) {
    rk = riemann_k<double>(fg[5 * f], fg[5 * f + 1], g);
    tl = fg[5 * f + 2];
  } else if constexpr (std::is_same<T, DF>::value) {
    const float2 nx = fg2[3 * f], ny = fg2[3 * f + 1], ln = fg2[3 * f + 2];
    rk = {DF{1.f, 0.f}, DF{0.5f, 0.f}, DF{gm12.x, gm12.y}, DF{g2.x, g2.y}, DF{nx.x, nx.y},
          DF{ny.x, ny.y}};
    tl = DF{ln.x, ln.y};
  } else {
    rk = {1.f, 0.5f, gm12.x, g2.x, fg2[3 * f].x, fg2[3 * f + 1].x};
    tl = fg2[3 * f + 2].x;
  }
}
template <typename T>
__device__ __forceinline__ T gauss_w(double w, float2 w2) {
  if constexpr (std::is_same<T, double>::value)
    return w;
  else if constexpr (std::is_same<T, DF>::value)
    return DF{w2.x, w2.y};
  else
    return w2.x;
}

// Gauss points of a face unrolled in the flux kernel: the pair-arithmetic
// solver is large enough that one copy of its code runs faster (fewer
// instruction-fetch stalls) than three; the FP32 and FP64 ones unroll
// Groups of NV = 4 values (the states at one Gauss point, the flux of one
// face) as 16-byte accesses; the arrays are cudaMalloc'd and indexed in whole
// groups, so every group starts on a 16-byte boundary.
template <int NV, typename T>
__device__ __forceinline__ void ld_group(const T* __restrict__ p, T (&x)[NV]) {
  if constexpr (NV == 4 && std::is_same<T, float>::value) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    x[0] = q.x, x[1] = q.y, x[2] = q.z, x[3] = q.w;
  } else if constexpr (NV == 4 && std::is_same<T, DF>::value) {
    const float4 q0 = __ldg(reinterpret_cast<const float4*>(p));
    const float4 q1 = __ldg(reinterpret_cast<const float4*>(p) + 1);
    x[0] = DF{q0.x, q0.y}, x[1] = DF{q0.z, q0.w}, x[2] = DF{q1.x, q1.y}, x[3] = DF{q1.z, q1.w};
  } else if constexpr (NV == 4 && std::is_same<T, double>::value) {
    const double2 q0 = __ldg(reinterpret_cast<const double2*>(p));
    const double2 q1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
    x[0] = q0.x, x[1] = q0.y, x[2] = q1.x, x[3] = q1.y;
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = p[v];
  }
}
template <int NV, typename T>
__device__ __forceinline__ void st_group(T* __restrict__ p, const T (&x)[NV]) {
  if constexpr (NV == 4 && std::is_same<T, float>::value) {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
  } else if constexpr (NV == 4 && std::is_same<T, DF>::value) {
    reinterpret_cast<float4*>(p)[0] = make_float4(x[0].h, x[0].l, x[1].h, x[1].l);
    reinterpret_cast<float4*>(p)[1] = make_float4(x[2].h, x[2].l, x[3].h, x[3].l);
  } else if constexpr (NV == 4 && std::is_same<T, double>::value) {
    reinterpret_cast<double2*>(p)[0] = make_double2(x[0], x[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(x[2], x[3]);
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) p[v] = x[v];
  }
}

#ifndef TENO_FLUX_UNROLL_PAIRS
#define TENO_FLUX_UNROLL_PAIRS 1
#endif
constexpr int kFluxUnrollPairs = TENO_FLUX_UNROLL_PAIRS;

template <int NV, int NQ, int FLUX, typename T>
__global__ void __launch_bounds__(256) face_flux_kernel(const FaceArgs a, const T* __restrict__ Uq,
                                                        T* __restrict__ K) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= a.n_face) return;
  const int o = a.f_cells[2 * f], n = a.f_cells[2 * f + 1];
  const int eo = a.f_edges[2 * f], en = a.f_edges[2 * f + 1];
  const double nx = a.f_geom[5 * f], ny = a.f_geom[5 * f + 1], len = a.f_geom[5 * f + 2];
  T acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = cst<T>(0.0);
  RiemannK<T> rk;
  T tl;
  face_k<T>(a.f_geom, a.f_geom2, f, a.gamma, a.g2, a.gm12, rk, tl);
  // (the Gauss values of an outflow-layer cell are its cell average, written
  // by layer_fill_kernel: at an outflow face both states are that average)
#pragma unroll (std::is_same<T, DF>::value ? kFluxUnrollPairs : 4)
  for (int k = 0; k < NQ; ++k) {
    T UL[NV], UR[NV], F[NV];
    ld_group<NV>(Uq + ((int64_t)(o * 3 + eo) * NQ + k) * NV, UL);
    if (n >= 0) {
      ld_group<NV>(Uq + ((int64_t)(n * 3 + en) * NQ + (NQ - 1 - k)) * NV, UR);
    } else if constexpr (NV == 4) {
      double x = a.f_geom[5 * f + 3] - ny * len * a.gt[k];
      ghost_state<T>(en, UL, nx, ny, x, a.time, a.gamma, UR);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) UR[v] = UL[v];
    }
    if constexpr (NV == 1) {
      const double xq = a.f_geom[5 * f + 3] - ny * len * a.gt[k];
      const double yq = a.f_geom[5 * f + 4] + nx * len * a.gt[k];
      const double an = adv_normal(a.adv_field, a.adv_x, a.adv_y, a.adv_cx, a.adv_cy,
                                   a.adv_omega, a.adv_r1, a.adv_r2, xq, yq, nx, ny);
      F[0] = cst<T>(an) * (an >= 0.0 ? UL[0] : UR[0]);
    } else {
      euler_riemann<T>(UL, UR, rk, FLUX == TENO_FLUX_HLLC, F);
    }
    const T wk = gauss_w<T>(a.gw[k], a.gw2[k]);
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = madd(wk, F[v], acc[v]);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = acc[v] * tl;
  st_group<NV>(K + f * NV, acc);
}

// ------------------------------------------------------------------ gather
struct GatherArgs {
  const int32_t* c_faces;
  const double* inv_area;
  int64_t n_cell, n_pad;
  double gamma;
};

template <int NV, typename TK>
__global__ void __launch_bounds__(256) gather_kernel(const GatherArgs a, const TK* __restrict__ K,
                                                     const double* __restrict__ Un,
                                                     const double* __restrict__ Us,
                                                     double* __restrict__ out, int mode, double cn,
                                                     double cs, double dt_fixed, double cfl,
                                                     const double* __restrict__ max_lam,
                                                     int* flag, float2* __restrict__ split) {
  // the step size once per block (one FP64 division)
  __shared__ double s_dt;
  if (mode != 0 && threadIdx.x == 0) s_dt = max_lam ? cfl / *max_lam : dt_fixed;
  if (mode != 0) __syncthreads();
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.n_cell) return;
  double acc[NV];
  if constexpr (std::is_same<TK, DF>::value || std::is_same<TK, float>::value) {
    // pair (or FP32) fluxes summed in pairs on the FP32 pipe, one conversion
    // per variable; three FP32 terms sum exactly in a pair
    DF sum[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) sum[v] = DF{0.f, 0.f};
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int cf = a.c_faces[3 * c + e];
      const int64_t f = cf >> 1;
      TK kf[NV];
      ld_group<NV>(K + f * NV, kf);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        DF k;
        if constexpr (std::is_same<TK, DF>::value)
          k = kf[v];
        else
          k = DF{kf[v], 0.f};
        sum[v] = (cf & 1) ? sum[v] - k : sum[v] + k;
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = to_d(sum[v]);
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int cf = a.c_faces[3 * c + e];
      const int64_t f = cf >> 1;
      const double s = (cf & 1) ? -1.0 : 1.0;
      TK kf[NV];
      ld_group<NV>(K + f * NV, kf);
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] = fma(s, to_d(kf[v]), acc[v]);
    }
  }
  const double ia = a.inv_area[c];
  if (mode == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v * a.n_pad + c] = -acc[v] * ia;
    return;
  }
  const double wr = cs * s_dt * ia;  // the stage's weight of the face-flux sum
  double u[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int64_t i = v * a.n_pad + c;
    u[v] = fma(-wr, acc[v], fma(cn, Un[i], cs * Us[i]));
    out[i] = u[v];
    if (split) {
      const float hi = (float)u[v];
      split[i] = make_float2(hi, (float)(u[v] - (double)hi));
    }
  }
  if constexpr (NV == 4) {
    // rho > 0 and p > 0, the latter as rho E - |m|^2 / 2 > 0 (no division)
    const double rho = u[0];
    const double pr = u[3] * rho - 0.5 * (u[1] * u[1] + u[2] * u[2]);
    if (!(rho > 0.0) || !(pr > 0.0)) atomicOr(flag, 1);
  } else {
    if (!(u[0] == u[0])) atomicOr(flag, 1);
  }
}

// --------------------------------------------------------------- CFL speed
template <int NV>
__global__ void __launch_bounds__(256) max_lambda_kernel(const double* __restrict__ U,
                                                         const double* __restrict__ cfl_len,
                                                         int64_t n_cell, int64_t n_pad,
                                                         double gamma, double adv_speed,
                                                         const double* __restrict__ cell_speed,
                                                         unsigned long long* out) {
  double lam = 0.0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cell;
       c += (int64_t)gridDim.x * blockDim.x) {
    double s;
    if constexpr (NV == 1) {
      s = cell_speed ? cell_speed[c] : adv_speed;
    } else {
      const double rho = U[c], u = U[n_pad + c] / rho, v = U[2 * n_pad + c] / rho;
      const double p = (gamma - 1.0) * (U[3 * n_pad + c] - 0.5 * rho * (u * u + v * v));
      s = sqrt(u * u + v * v) + sqrt(gamma * p / rho);
      // a non-physical cell (rho <= 0, p <= 0 or NaN) makes the maximum infinite, which
      // the host reports as TENO_ENONPHYS (fmax would drop a NaN speed)
      if (!(rho > 0.0) || !(p > 0.0)) s = __longlong_as_double(0x7ff0000000000000LL);
    }
    lam = fmax(lam, s / cfl_len[c]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
  __shared__ double red[32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = lam;
  __syncthreads();
  if (w == 0) {
    lam = l < (int)(blockDim.x >> 5) ? red[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
    // non-negative doubles order like their bit patterns
    if (l == 0) atomicMax(out, (unsigned long long)__double_as_longlong(lam));
  }
}

// The same maximum from the (hi, lo) split of the state that the FP64 and
// mixed paths keep for the reconstruction (Euler): lambda_c = (|u| + c) / L_c
// in pair arithmetic on the FP32 pipe (relative error ~1e-14, far below what
// a CFL step needs) with 1/L_c as host-split pairs; the maximum as FP64
// bits.  Non-physical cells (NaN speed) are skipped as fmax skips them.
__global__ void __launch_bounds__(256) max_lambda_split_kernel(const float2* __restrict__ Us,
                                                               const float2* __restrict__ ilen2,
                                                               int64_t n_cell, int64_t n_pad,
                                                               float2 g2, float2 gm12,
                                                               unsigned long long* out) {
  const DF one = {1.f, 0.f}, half = {0.5f, 0.f}, gg = {g2.x, g2.y}, gm1 = {gm12.x, gm12.y};
  DF lam = {0.f, 0.f};
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cell;
       c += (int64_t)gridDim.x * blockDim.x) {
    const float2 q0 = Us[c], q1 = Us[n_pad + c], q2 = Us[2 * n_pad + c], q3 = Us[3 * n_pad + c];
    const DF rho = {q0.x, q0.y}, mx = {q1.x, q1.y}, my = {q2.x, q2.y}, E = {q3.x, q3.y};
    const DF ir = one / rho;
    const DF u = mx * ir, v = my * ir;
    const DF q = u * u + v * v;
    const DF p = gm1 * (E - half * rho * q);
    const DF sp = tsqrt(q) + tsqrt(gg * p * ir);
    const float2 il = ilen2[c];
    const DF l = sp * DF{il.x, il.y};
    if (l.h == l.h) lam = vmax(lam, l);
  }
  double d = to_d(lam);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
  __shared__ double red[32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = d;
  __syncthreads();
  if (w == 0) {
    d = l < (int)(blockDim.x >> 5) ? red[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
    if (l == 0) atomicMax(out, (unsigned long long)__double_as_longlong(d));
  }
}

// -------------------------------------------------------------- utilities
__global__ void permute_kernel(const double* __restrict__ src, double* __restrict__ dst,
                               const int32_t* __restrict__ perm, int64_t n, int64_t ld_src,
                               int64_t ld_dst, int to_user) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (i >= n) return;
  const int64_t u = perm[i];
  if (to_user)
    dst[v * ld_dst + u] = src[v * ld_src + i];
  else
    dst[v * ld_dst + i] = src[v * ld_src + u];
}

__global__ void permute_u8_kernel(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst,
                                  const int32_t* __restrict__ perm, int64_t n, int64_t ld_src,
                                  int64_t ld_dst, int to_user) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (i >= n) return;
  const int64_t u = perm[i];
  if (to_user)
    dst[v * ld_dst + u] = src[v * ld_src + i];
  else
    dst[v * ld_dst + i] = src[v * ld_src + u];
}

__global__ void axpby_kernel(double* out, const double* a, double ca, const double* b, double cb,
                             int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = ca * a[i] + cb * b[i];
}

// ------------------------------------------------------------------ adjoint
struct VjpArgs {
  const int32_t* f_cells;
  const int8_t* f_edges;
  const double* f_geom;
  const float2* f_geom2;
  float2 g2, gm12;
  int adv_field;
  double adv_cx, adv_cy, adv_omega, adv_r1, adv_r2;
  const double* inv_area;
  int64_t n_face, n_pad;
  double gamma, adv_x, adv_y, time;
  double gw[kMaxNq], gt[kMaxNq];
  float2 gw2[kMaxNq];  // Gauss weights as (hi, lo) pairs
};

// Uq_bar[(c,edge,q)] = w_q |A| (dF/dU_side)^T Kbar with Kbar = dJ/dK_f
// (R_o has -K/|V_o|, R_n has +K/|V_n|); every Gauss slot of every cell is
// written by exactly one face.  Euler: the hand-written reverse sweep of the
// Riemann solver (euler_riemann_vjp, ghost_vjp).  Scalar advection, and Euler
// when built with TENO_VJP_REVERSE=0: Jacobian columns from forward-mode dual
// numbers over scalar S, ND seeded directions per pass (an interior face
// seeds the NV components of U_L, then those of U_R; a boundary face only U_L,
// the ghost state carrying dU_R/dU_L).
// Euler flux VJP by the hand-written reverse sweep (1) or by forward-mode
// dual numbers (0; kept as the cross-check of the reverse sweep)
#ifndef TENO_VJP_REVERSE
#define TENO_VJP_REVERSE 1
#endif
constexpr bool kVjpReverse = TENO_VJP_REVERSE != 0;

// Uq_bar entry i: (hi, lo) pairs on the pair path (S = DF; read as pairs by
// the reconstruction VJP, no FP64 conversion on either side), FP64 on the
// native path
template <typename S>
__device__ __forceinline__ void store_bar(double* base, int i, S x) {
  if constexpr (std::is_same<S, DF>::value)
    reinterpret_cast<float2*>(base)[i] = make_float2(x.h, x.l);
  else
    base[i] = to_d(x);
}

// minimum resident blocks of 128 threads per SM for the flux VJP (3: 168
// registers, measured 13 % faster than no cap; 0: no cap)
#ifndef TENO_VJP_MIN_BLOCKS
#define TENO_VJP_MIN_BLOCKS 3
#endif
template <int NV, int NQ, int FLUX, typename TQ, typename S, int ND>
__global__ void __launch_bounds__(128, TENO_VJP_MIN_BLOCKS > 0 ? TENO_VJP_MIN_BLOCKS : 1)
    face_flux_vjp_kernel(const VjpArgs a,
                                                            const TQ* __restrict__ Uq,
                                                            const double* __restrict__ w,
                                                            double* __restrict__ Uq_bar) {
  static_assert((2 * NV) % ND == 0, "directions per pass must divide 2 NV");
  using D = Dual<ND, S>;
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= a.n_face) return;
  const int o = a.f_cells[2 * f], n = a.f_cells[2 * f + 1];
  const int eo = a.f_edges[2 * f], en = a.f_edges[2 * f + 1];
  const double nx = a.f_geom[5 * f], ny = a.f_geom[5 * f + 1], len = a.f_geom[5 * f + 2];
  // Kbar in FP64 from the FP64 weights, once per face in the flux scalar type
  S Kb[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double kb = -w[v * a.n_pad + o] * a.inv_area[o];
    if (n >= 0) kb = fma(w[v * a.n_pad + n], a.inv_area[n], kb);
    Kb[v] = cst<S>(kb);
  }
  const int n_pass = ((n >= 0 ? 2 * NV : NV) + ND - 1) / ND;
  RiemannK<S> rks;
  S tl;  // |A| in the flux scalar type
  face_k<S>(a.f_geom, a.f_geom2, f, a.gamma, a.g2, a.gm12, rks, tl);
  const RiemannK<D> rk = riemann_k_dual<ND, S>(rks);
  for (int k = 0; k < NQ; ++k) {
    TQ ul[NV], ur[NV];
    ld_group<NV>(Uq + ((int64_t)(o * 3 + eo) * NQ + k) * NV, ul);
    if (n >= 0) ld_group<NV>(Uq + ((int64_t)(n * 3 + en) * NQ + (NQ - 1 - k)) * NV, ur);
    // x of the Gauss point (ghost states and the scalar field only)
    auto xq = [&]() { return a.f_geom[5 * f + 3] - ny * len * a.gt[k]; };
    const S wl = gauss_w<S>(a.gw[k], a.gw2[k]) * tl;
    S Kw[NV];  // w_k |A| Kbar in the flux scalar type
#pragma unroll
    for (int v = 0; v < NV; ++v) Kw[v] = wl * Kb[v];
    double* outL = Uq_bar + ((int64_t)(o * 3 + eo) * NQ + k) * NV;
    double* outR = n >= 0 ? Uq_bar + ((int64_t)(n * 3 + en) * NQ + (NQ - 1 - k)) * NV : outL;
    if constexpr (NV == 4 && kVjpReverse) {
      // reverse mode: one forward recomputation and its adjoint sweep
      S uL[NV], uR[NV], ULb[NV], URb[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        uL[v] = lift<S>(ul[v]);
        ULb[v] = cst<S>(0.0);
        URb[v] = cst<S>(0.0);
      }
      if (n >= 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) uR[v] = lift<S>(ur[v]);
      } else {
        ghost_state<S>(en, uL, nx, ny, xq(), a.time, a.gamma, uR);
      }
      euler_riemann_vjp<S>(uL, uR, rks, FLUX == TENO_FLUX_HLLC, Kw, ULb, URb);
      if (n < 0) ghost_vjp<S>(en, rks, URb, ULb);
      if constexpr (std::is_same<S, DF>::value) {
        st_group<NV>(reinterpret_cast<DF*>(outL), ULb);
        if (n >= 0) st_group<NV>(reinterpret_cast<DF*>(outR), URb);
      } else {
        st_group<NV>(outL, ULb);
        if (n >= 0) st_group<NV>(outR, URb);
      }
    } else {
      for (int pass = 0; pass < n_pass; ++pass) {
        const int dir0 = pass * ND;  // directions dir0 .. dir0+ND-1 of [U_L, U_R]
        D UL[NV], UR[NV], F[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          UL[v] = cst<D>(0.0);
          UL[v].v = lift<S>(ul[v]);
          if (v >= dir0 && v < dir0 + ND) UL[v].d[v - dir0] = cst<S>(1.0);
        }
        if (n >= 0) {
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            UR[v] = cst<D>(0.0);
            UR[v].v = lift<S>(ur[v]);
            if (NV + v >= dir0 && NV + v < dir0 + ND) UR[v].d[NV + v - dir0] = cst<S>(1.0);
          }
        } else if constexpr (NV == 4) {
          ghost_state<D>(en, UL, nx, ny, xq(), a.time, a.gamma, UR);  // carries dUR/dUL
        } else {
#pragma unroll
          for (int v = 0; v < NV; ++v) UR[v] = UL[v];
        }
        if constexpr (NV == 1) {
          const double yq = a.f_geom[5 * f + 4] + nx * len * a.gt[k];
          const double an = adv_normal(a.adv_field, a.adv_x, a.adv_y, a.adv_cx, a.adv_cy,
                                       a.adv_omega, a.adv_r1, a.adv_r2, xq(), yq, nx, ny);
          F[0] = an * (an >= 0.0 ? UL[0] : UR[0]);
        } else {
          euler_riemann<D>(UL, UR, rk, FLUX == TENO_FLUX_HLLC, F);
        }
#pragma unroll
        for (int j = 0; j < ND; ++j) {
          S sacc = cst<S>(0.0);
#pragma unroll
          for (int i = 0; i < NV; ++i) sacc = madd(F[i].d[j], Kw[i], sacc);
          const int g = dir0 + j;
          if (g < NV)
            store_bar<S>(outL, g, sacc);
          else if (n >= 0)
            store_bar<S>(outR, g - NV, sacc);
        }
      }
    }
  }
}

// stencil slots unrolled in the reconstruction VJP kernels (matrix loads in
// flight per thread)
#ifndef TENO_VJP_SLOT_UNROLL
#define TENO_VJP_SLOT_UNROLL 2
#endif
constexpr int kVjpSlotUnroll = TENO_VJP_SLOT_UNROLL;

// d_bar[tile][slot][v][32] = (A''^T abar)_slot with abar = w_k Psi'^T Uq_bar
// (selection frozen); u_self = sum_p Uq_bar - sum_slot d_bar (dU_0 terms).
template <int M, int NS, int NQ, int NV, typename TS>
__global__ void __launch_bounds__(128) recon_vjp_kernel(const TS* __restrict__ ahat,
                                                        const uint8_t* __restrict__ sel_in,
                                                        const double* __restrict__ Uq_bar,
                                                        double* __restrict__ d_bar,
                                                        double* __restrict__ u_self,
                                                        int64_t n_cell, int64_t n_pad,
                                                        const EvalTable ev) {
  const int lane = threadIdx.x, v = threadIdx.y;
  const int64_t tile = (int64_t)blockIdx.x * blockDim.z + threadIdx.z;
  const int64_t c = tile * kTile + lane;
  if (c >= n_cell) return;
  constexpr int E = M * NS + kSmallEntries;
  constexpr int SL = NS + kSmallSlots;
  const TS* A = ahat + tile * (int64_t)E * kTile + lane;
  // matrix entry as FP64 (pairs of the double-float storage are summed)
  auto ent = [](TS x) -> double {
    if constexpr (std::is_same<TS, float2>::value)
      return (double)x.x + (double)x.y;
    else
      return x;
  };
  double* db = d_bar + tile * (int64_t)SL * NV * kTile + lane * NV + v;
  double cb[M];
#pragma unroll
  for (int l = 0; l < M; ++l) cb[l] = 0.0;
  double u0b = 0.0;
  const double* ub = Uq_bar + c * (3 * NQ * NV) + v;
#pragma unroll
  for (int p = 0; p < 3 * NQ; ++p) {
    const double b = ub[p * NV];
    u0b += b;
#pragma unroll
    for (int l = 0; l < M; ++l) cb[l] = fma(b, ev.psi[p * kMaxM + l], cb[l]);
  }
  const uint8_t sel = sel_in[(int64_t)v * n_pad + c];
  double tot = 0.0;
  const bool large = sel & 8;
#pragma unroll (kVjpSlotUnroll)
  for (int s = 0; s < NS; ++s) {
    double t = 0.0;
    if (large) {
#pragma unroll
      for (int l = 0; l < M; ++l) t = fma(ent(A[(int64_t)(s * M + l) * kTile]), cb[l], t);
    }
    db[(int64_t)s * NV * kTile] = t;
    tot += t;
  }
  const int nd = (sel & 1) + ((sel >> 1) & 1) + ((sel >> 2) & 1);
  const double w = (!large && nd) ? 1.0 / nd : 0.0;
#pragma unroll
  for (int k = 0; k < kSmallK; ++k) {
    const double wk = ((sel >> k) & 1) ? w : 0.0;
    for (int s = 0; s < kSmallN; ++s) {
      double t = 0.0;
      if (wk != 0.0) {
        const TS* As = A + (int64_t)(M * NS + (k * kSmallN + s) * kSmallM) * kTile;
#pragma unroll
        for (int l = 0; l < kSmallM; ++l) t = fma(ent(As[l * kTile]), cb[l], t);
        t *= wk;
      }
      db[(int64_t)(NS + k * kSmallN + s) * NV * kTile] = t;
      tot += t;
    }
  }
  u_self[(int64_t)v * n_pad + c] = u0b - tot;
}

// Double-float version for the FP64 path (matrices stored as (hi, lo)
// pairs): the transposed matvecs run on the FP32 pipe; d_bar is written as
// pairs, u_self in FP64.
__device__ __forceinline__ DF d_to_df(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ DF df_div_small(DF a, int n) {  // a / n for n in 1..3
  const float fn = (float)n;
  const float qh = a.h / fn;
  const float r = fmaf(-qh, fn, a.h);  // exact remainder
  return two_sum(qh, (r + a.l) / fn);
}

template <int M, int NS, int NQ, int NV>
__global__ void __launch_bounds__(128) recon_vjp_df_kernel(const float2* __restrict__ ahat,
                                                           const uint8_t* __restrict__ sel_in,
                                                           const double* __restrict__ Uq_bar,
                                                           DF* __restrict__ d_bar,
                                                           double* __restrict__ u_self,
                                                           int64_t n_cell, int64_t n_pad,
                                                           const DFTable ev) {
  const int lane = threadIdx.x, v = threadIdx.y;
  const int64_t tile = (int64_t)blockIdx.x * blockDim.z + threadIdx.z;
  const int64_t c = tile * kTile + lane;
  if (c >= n_cell) return;
  constexpr int E = M * NS + kSmallEntries;
  constexpr int SL = NS + kSmallSlots;
  const float2* A = ahat + tile * (int64_t)E * kTile + lane;
  DF* db = d_bar + tile * (int64_t)SL * NV * kTile + lane * NV + v;
  DF cb[M];
#pragma unroll
  for (int l = 0; l < M; ++l) cb[l] = {0.f, 0.f};
  DF u0b = {0.f, 0.f};
  // Uq_bar as (hi, lo) pairs (written so by the pair-path flux VJP)
  const float2* ub = reinterpret_cast<const float2*>(Uq_bar) + c * (3 * NQ * NV) + v;
#pragma unroll
  for (int p = 0; p < 3 * NQ; ++p) {
    const DF b = {ub[p * NV].x, ub[p * NV].y};
    u0b = u0b + b;
#pragma unroll
    for (int l = 0; l < M; ++l) df_mac(cb[l], ev.psi[p * kMaxM + l], b);
  }
#pragma unroll
  for (int l = 0; l < M; ++l) cb[l] = df_norm(cb[l]);
  const uint8_t sel = sel_in[(int64_t)v * n_pad + c];
  DF tot = {0.f, 0.f};
  const bool large = sel & 8;
#pragma unroll (kVjpSlotUnroll)
  for (int s = 0; s < NS; ++s) {
    DF t = {0.f, 0.f};
    if (large) {
#pragma unroll
      for (int l = 0; l < M; ++l)
        df_mac(t, A[(int64_t)(s * M + l) * kTile], cb[l]);
      t = df_norm(t);
    }
    db[(int64_t)s * NV * kTile] = t;
    tot = tot + t;
  }
  const int nd = (sel & 1) + ((sel >> 1) & 1) + ((sel >> 2) & 1);
#pragma unroll
  for (int k = 0; k < kSmallK; ++k) {
    const bool on = !large && ((sel >> k) & 1);
    for (int s = 0; s < kSmallN; ++s) {
      DF t = {0.f, 0.f};
      if (on) {
        const float2* As = A + (int64_t)(M * NS + (k * kSmallN + s) * kSmallM) * kTile;
#pragma unroll
        for (int l = 0; l < kSmallM; ++l) df_mac(t, As[l * kTile], cb[l]);
        t = df_div_small(df_norm(t), nd);
      }
      db[(int64_t)(NS + k * kSmallN + s) * NV * kTile] = t;
      tot = tot + t;
    }
  }
  u_self[(int64_t)v * n_pad + c] = to_d(u0b - tot);
}

// Tiled reconstruction VJP (FP64 path, Euler, W form).  With the selection
// frozen, Uq_p = U_0 + sum_s W_ps d_s for the large polynomial (W = Psi' G,
// the per-cell pairs the forward W-form kernel uses), so d_bar_s =
// sum_p W_ps Uq_bar_p: NQ3 pair products per slot and no coefficient
// adjoint.  Directional stencils (cells whose large stencil is cut) take
// d_bar_s = (G_k^T Psi_k^T Uq_bar)_s / n_kept from their (hi, lo) matrices;
// their stages are streamed only for tiles where some (cell, variable) keeps
// a directional stencil, a predicate the producer and the consumers evaluate
// from the same selection bytes.  Each lane adds its d_bar_s to the tile's
// halo accumulator in shared memory at the slot's halo position (lanes with
// equal positions in lane order, by ranks the host stores next to the
// positions; slots in stencil order: deterministic sums).  The host assigns
// the large-stencil members to slots so that the lanes of a tile do not
// share a cell within a slot, and these slots take one round.  At the end of
// the tile the accumulator is written as one pair per (halo entry,
// variable), so the reverse gather reads the few halo entries that hold a
// cell instead of every stencil slot that holds it.  The tile's Uq_bar block is prefetched
// with cp.async one tile ahead.
constexpr int kRingV = 4;
constexpr int kUbStride = 38;  // doubles per cell in the Uq_bar stage (16-byte rows)
constexpr int kHaccStride = kHaloMax + 4;  // pairs per variable row (conflict-free transpose)

template <int M, int NS, int NQ3>
struct VjpPlan {
  static constexpr int kLPS = 4, kSPS = 4;
  static constexpr int kSlotW = NQ3 * kTile * 8;      // W pairs of one large slot
  static constexpr int kSlotS = kSmallM * kTile * 8;  // matrix pairs of one directional slot
  static constexpr int kSlotN = kTile * 2;            // halo positions (uint16) of one slot
  static constexpr int kNL = (NS + kLPS - 1) / kLPS;
  static constexpr int kPerSmall = kSmallN / kSPS;
  static constexpr int kStages = kNL + kSmallK * kPerSmall;
  static constexpr int kNOff = kLPS * kSlotW > kSPS * kSlotS ? kLPS * kSlotW : kSPS * kSlotS;
  static constexpr int kMat = kNOff + 4 * kSlotN;
  static constexpr int kSL = NS + kSmallSlots;
  static constexpr int64_t kTileW = (int64_t)NS * NQ3 * kTile * 8;
  static constexpr int64_t kTileA = (int64_t)(M * NS + kSmallEntries) * kTile * 8;
  static constexpr size_t kUbOff = (size_t)kRingV * kMat;
  static constexpr size_t kUbBytes = (size_t)2 * kTile * kUbStride * 8;
  static constexpr size_t kHaccOff = kUbOff + kUbBytes;
  static constexpr size_t kHaccBytes = (size_t)4 * kHaccStride * 8;
  static constexpr size_t kBarOff = kHaccOff + kHaccBytes;
  static constexpr size_t kSmem = kBarOff + 2 * kRingV * 8 + 16 + 16;
  static_assert(NQ3 * 4 <= kUbStride, "Uq_bar row");
  static_assert(kSmallN % kSPS == 0, "directional stencil split");
  static_assert(kMat % 16 == 0 && kUbOff % 16 == 0 && kHaccOff % 16 == 0 && kBarOff % 8 == 0,
                "alignment");
  // stage j: slots [slot0, slot0 + nslot) of stencil k (-1: large, from W;
  // else from the directional matrices), source byte offset in the tile's
  // W or matrix block
  __device__ static void stage(int j, int& slot0, int& nslot, int& k, int64_t& off, int& bytes) {
    if (j < kNL) {
      slot0 = j * kLPS;
      nslot = (NS - slot0) < kLPS ? (NS - slot0) : kLPS;
      k = -1;
      off = (int64_t)slot0 * kSlotW;
      bytes = nslot * kSlotW;
    } else {
      const int i = j - kNL;
      k = i / kPerSmall;
      const int s0 = (i % kPerSmall) * kSPS;
      slot0 = NS + k * kSmallN + s0;
      nslot = kSPS;
      off = (int64_t)(M * NS + (k * kSmallN + s0) * kSmallM) * kTile * 8;
      bytes = kSPS * kSlotS;
    }
  }
};

// the (cell, variable) of this selection byte keeps directional stencils:
// its large stencil is cut and at least one directional stencil is kept
__device__ __forceinline__ bool vjp_needs_small(uint8_t sel) {
  return !(sel & 8) && (sel & 7);
}

template <int M, int NS, int NQ>
__global__ void __launch_bounds__(kTile * (kConsumers + 1), 3)
    recon_vjp_tma_kernel(const float2* __restrict__ ahat, const float2* __restrict__ wq,
                         const HaloArgs h, const uint8_t* __restrict__ sel_in,
                         const double* __restrict__ Uq_bar, float2* __restrict__ part,
                         double* __restrict__ u_self, int64_t n_cell, int64_t n_pad,
                         const DFTable ev, int* err) {
  constexpr int NV = 4, NQ3 = 3 * NQ, kPer = NQ3 * NV;
  using VP = VjpPlan<M, NS, NQ3>;
  extern __shared__ __align__(128) unsigned char smem[];
  double* ubs = reinterpret_cast<double*>(smem + VP::kUbOff);     // [2][32][kUbStride]
  float2* hacc = reinterpret_cast<float2*>(smem + VP::kHaccOff);  // [NV][kHaccStride]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + VP::kBarOff);
  uint64_t* empty = full + kRingV;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + kRingV);
  int* need = const_cast<int*>(abort_flag) + 4;  // [NV] per-variable small-stencil flags
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n_tiles = (n_cell + kTile - 1) / kTile;
  if (threadIdx.x == 0) {
    *abort_flag = 0;
    for (int i = 0; i < kRingV; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kConsumers);
    }
    mbar_fence_init();
  }
  __syncthreads();
  if (warp == kConsumers) {
    // ---- producer lane: W blocks (and directional matrices where needed)
    if (lane == 0) {
      int64_t g = 0;
      for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const unsigned char* sw = reinterpret_cast<const unsigned char*>(wq) + tile * VP::kTileW;
        const unsigned char* sa = reinterpret_cast<const unsigned char*>(ahat) + tile * VP::kTileA;
        const unsigned char* sn =
            reinterpret_cast<const unsigned char*>(h.nbr_loc) + tile * (int64_t)VP::kSL * VP::kSlotN;
        // the tile's selection bytes: 2 x 16 per variable (rows of n_pad, a
        // multiple of 32), pad lanes masked
        const int nval = (int)min((int64_t)kTile, n_cell - tile * kTile);
        uint4 sw4[2 * NV];
#pragma unroll
        for (int w = 0; w < NV; ++w)
#pragma unroll
          for (int q = 0; q < 2; ++q)
            sw4[2 * w + q] =
                __ldg(reinterpret_cast<const uint4*>(sel_in + (int64_t)w * n_pad + tile * kTile) + q);
        bool small = false;
#pragma unroll
        for (int w = 0; w < NV; ++w)
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const uint32_t words[4] = {sw4[2 * w + q].x, sw4[2 * w + q].y, sw4[2 * w + q].z,
                                       sw4[2 * w + q].w};
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const uint8_t b = (uint8_t)(words[i >> 2] >> (8 * (i & 3)));
              small |= (16 * q + i < nval) && vjp_needs_small(b);
            }
          }
        const int n_stages = small ? VP::kStages : VP::kNL;
        for (int j = 0; j < n_stages; ++j, ++g) {
          const int b = (int)(g % kRingV);
          if (g >= kRingV) {
            const int w =
                mbar_wait_or_abort(&empty[b], (uint32_t)((g / kRingV) - 1) & 1, abort_flag);
            if (w != 1) {
              if (w == 0) {
                atomicOr(err, 2);
                *abort_flag = 1;
              }
              for (int64_t i = g - kRingV; i < g; ++i)
                mbar_wait(&full[i % kRingV], (uint32_t)(i / kRingV) & 1);
              return;
            }
          }
          int slot0, nslot, k, bytes;
          int64_t off;
          VP::stage(j, slot0, nslot, k, off, bytes);
          const uint32_t bn = (uint32_t)(nslot * VP::kSlotN);
          unsigned char* dst = smem + (size_t)b * VP::kMat;
          mbar_expect_tx(&full[b], (uint32_t)bytes + bn);
          bulk_g2s(dst, (k < 0 ? sw : sa) + off, (uint32_t)bytes, &full[b]);
          bulk_g2s(dst + VP::kNOff, sn + slot0 * VP::kSlotN, bn, &full[b]);
        }
      }
      // the block must not exit while a copy it issued is in flight
      for (int64_t i = g > kRingV ? g - kRingV : 0; i < g; ++i)
        mbar_wait(&full[i % kRingV], (uint32_t)(i / kRingV) & 1);
    }
    return;
  }
  // ---- consumers (warp v: variable v)
  const int v = warp, tid = threadIdx.x;
  // Uq_bar block of a tile (contiguous [cell][point][variable]) into stage hb
  auto prefetch = [&](int64_t tile, int hb) {
    const int nval = (int)min((int64_t)kTile, n_cell - tile * kTile);
    const double* src = Uq_bar + tile * kTile * kPer;
    double* dst = ubs + (size_t)hb * kTile * kUbStride;
    for (int e = tid; e < nval * (kPer / 2); e += kConsumers * kTile) {
      const int cl = e / (kPer / 2), w = e - cl * (kPer / 2);
      cp_async16(dst + cl * kUbStride + 2 * w, src + (int64_t)cl * kPer + 2 * w);
    }
    cp_async_commit();
  };
  float2* hrow = hacc + v * kHaccStride;
  // add t at the halo position of code (bits 0-7); lanes with equal
  // positions in the order of their precomputed ranks (bits 8-12)
  auto accumulate = [&](bool act, int code, DF t) {
    const int hp = code & kHaloPosMask;
    const unsigned rank = (unsigned)code >> 8;
    const unsigned rmax = __reduce_max_sync(0xffffffffu, act ? rank : 0u);
    for (unsigned r = 0; r <= rmax; ++r) {
      if (act && rank == r) {
        const float2 q = hrow[hp];
        const DF s = DF{q.x, q.y} + t;
        hrow[hp] = make_float2(s.h, s.l);
      }
      __syncwarp();
    }
  };
  int64_t g = 0;
  int hb = 0;
  bool dead = false;
  if ((int64_t)blockIdx.x < n_tiles) prefetch(blockIdx.x, 0);
  // the halo offsets and the selection byte of a tile, loaded a tile ahead
  auto pre = [&](int64_t tile, int& h0, int& H, uint8_t& sl) {
    h0 = 0, H = 0, sl = 0;
    if (tile < n_tiles) {
      h0 = h.off[tile];
      H = h.off[tile + 1] - h0;
      const int64_t cc = tile * kTile + lane;
      if (cc < n_cell) sl = sel_in[(int64_t)v * n_pad + cc];
    }
  };
  int h0n, Hn;
  uint8_t seln;
  pre(blockIdx.x, h0n, Hn, seln);
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, hb ^= 1) {
    consumer_sync();  // the previous tile's accumulator, flags and Uq_bar stage are released
    const int64_t nxt = tile + gridDim.x;
    if (nxt < n_tiles)
      prefetch(nxt, hb ^ 1);
    else
      cp_async_commit();
    const int h0 = h0n, H = Hn;
    const uint8_t sel = seln;
    pre(nxt, h0n, Hn, seln);
    for (int i = lane; i < H; i += kTile) hrow[i] = make_float2(0.f, 0.f);
    const int64_t c = tile * kTile + lane;
    const bool valid = c < n_cell;
    const bool vs = __any_sync(0xffffffffu, valid && vjp_needs_small(sel));
    if (lane == 0) need[v] = vs;
    cp_async_wait<1>();
    consumer_sync();  // the tile's Uq_bar has landed; the flags are set
    const bool small = need[0] | need[1] | need[2] | need[3];
    const int n_stages = small ? VP::kStages : VP::kNL;
    // Uq_bar of (c, v) at the Gauss points (stored as pairs); the dU_0 term
    DF ub[NQ3];
    DF u0b = {0.f, 0.f};
    {
      const float2* us = reinterpret_cast<const float2*>(ubs) +
                         (size_t)hb * kTile * kUbStride + lane * kUbStride + v;
#pragma unroll
      for (int p = 0; p < NQ3; ++p) {
        const float2 q = us[p * NV];
        ub[p] = valid ? DF{q.x, q.y} : DF{0.f, 0.f};
        u0b = u0b + ub[p];
      }
    }
    const bool large = valid && (sel & 8);
    const int nd = (sel & 1) + ((sel >> 1) & 1) + ((sel >> 2) & 1);
    // coefficient adjoints of the directional polynomials (first kSmallM
    // basis functions), only where some lane of the block needs them
    DF cbs[kSmallM];
#pragma unroll
    for (int l = 0; l < kSmallM; ++l) cbs[l] = {0.f, 0.f};
    if (small && valid && !large) {
#pragma unroll
      for (int p = 0; p < NQ3; ++p)
#pragma unroll
        for (int l = 0; l < kSmallM; ++l) df_mac(cbs[l], ev.psi[p * kMaxM + l], ub[p]);
#pragma unroll
      for (int l = 0; l < kSmallM; ++l) cbs[l] = df_norm(cbs[l]);
    }
    DF tot = {0.f, 0.f};
    for (int j = 0; j < n_stages; ++j, ++g) {
      const int b = (int)(g % kRingV);
      int slot0, nslot, k, bytes;
      int64_t off;
      VP::stage(j, slot0, nslot, k, off, bytes);
      if (!dead) {
        const int w = mbar_wait_or_abort(&full[b], (uint32_t)(g / kRingV) & 1, abort_flag);
        if (w == 0) {
          atomicOr(err, 2);
          *abort_flag = 1;
        }
        dead = __any_sync(0xffffffffu, w != 1);
      }
      const float2* mat = reinterpret_cast<const float2*>(smem + (size_t)b * VP::kMat) + lane;
      const uint16_t* nl =
          reinterpret_cast<const uint16_t*>(smem + (size_t)b * VP::kMat + VP::kNOff) + lane;
      if (dead) {
        // skip the stage
      } else if (k < 0) {
        if (__any_sync(0xffffffffu, large)) {
          // the stage's slot values first (independent chains), then their
          // accumulation slot by slot
          DF ts[VP::kLPS];
#pragma unroll
          for (int s = 0; s < VP::kLPS; ++s) {
            ts[s] = {0.f, 0.f};
            if (large && s < nslot) {
#pragma unroll
              for (int p = 0; p < NQ3; ++p) df_mac(ts[s], mat[(s * NQ3 + p) * kTile], ub[p]);
              ts[s] = df_norm(ts[s]);
            }
          }
#pragma unroll
          for (int s = 0; s < VP::kLPS; ++s) {
            if (s < nslot) {
              accumulate(large, nl[s * kTile], ts[s]);
              const DF q = two_sum(tot.h, ts[s].h);  // running sum, renormalised at the end
              tot.h = q.h;
              tot.l += q.l + ts[s].l;
            }
          }
        }
      } else {
        const bool on = valid && !large && ((sel >> k) & 1);
        if (__any_sync(0xffffffffu, on)) {
#pragma unroll
          for (int s = 0; s < VP::kSPS; ++s) {
            DF t = {0.f, 0.f};
            if (on) {
#pragma unroll
              for (int l = 0; l < kSmallM; ++l) df_mac(t, mat[(s * kSmallM + l) * kTile], cbs[l]);
              t = df_div_small(df_norm(t), nd);
            }
            accumulate(on, nl[s * kTile], t);
            const DF q = two_sum(tot.h, t.h);
            tot.h = q.h;
            tot.l += q.l + t.l;
          }
        }
      }
      __syncwarp();
      if (lane == 0 && !dead) mbar_arrive(&empty[b]);
    }
    if (valid && !dead) u_self[(int64_t)v * n_pad + c] = to_d(u0b - df_norm(tot));
    consumer_sync();  // every variable's accumulator is complete
    if (!dead) {
      float2* dst = part + (int64_t)h0 * NV;
      for (int e = tid; e < H * NV; e += kConsumers * kTile)
        dst[e] = hacc[(e & 3) * kHaccStride + (e >> 2)];
    }
  }
  cp_async_wait<0>();
}

#ifndef TENO_SCATTER_BATCH
#define TENO_SCATTER_BATCH 4
#endif
constexpr int kScatterBatch = TENO_SCATTER_BATCH;
// v[j] = u_self[j] + sum over the stencil slots that hold cell j.  d_bar is
// [tile][slot][lane][var]: the NV values of one slot entry are one 32-byte
// sector (NV = 4), read with vector loads; rev_idx holds entry numbers
// (tile * SL + slot) * 32 + lane.
template <int NV, typename TD>
__global__ void __launch_bounds__(256) scatter_gather_kernel(const int64_t* __restrict__ rev_off,
                                                             const int32_t* __restrict__ rev_idx,
                                                             const TD* __restrict__ d_bar,
                                                             const double* __restrict__ u_self0,
                                                             double* __restrict__ out,
                                                             int64_t n_cell, int64_t n_pad,
                                                             const double* __restrict__ ubd) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_cell) return;
  const int64_t r0 = rev_off[j], r1 = rev_off[j + 1];
  // the cell's own term, plus what its Gauss slots owe its average (outflow
  // layer cells, written by layer_vjp_kernel; zero elsewhere)
  double u_self[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    u_self[v] = u_self0[v * n_pad + j];
    if (ubd) u_self[v] += (ubd[(j * 3 + 0) * NV + v] + ubd[(j * 3 + 1) * NV + v]) +
                          ubd[(j * 3 + 2) * NV + v];
  }
  if constexpr (std::is_same<TD, DF>::value) {
    DF acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = d_to_df(u_self[v]);
    int64_t r = r0;
    if constexpr (NV == 4) {
      // kScatterBatch entries per round: every index, then every sector, is
      // requested before any is used (independent loads in flight)
      for (; r + kScatterBatch <= r1; r += kScatterBatch) {
        int id[kScatterBatch];
#pragma unroll
        for (int i = 0; i < kScatterBatch; ++i) id[i] = __ldg(rev_idx + r + i);
        float4 a[kScatterBatch], b[kScatterBatch];
#pragma unroll
        for (int i = 0; i < kScatterBatch; ++i) {
          const float4* e = reinterpret_cast<const float4*>(d_bar + (int64_t)id[i] * NV);
          a[i] = __ldg(e);
          b[i] = __ldg(e + 1);
        }
#pragma unroll
        for (int i = 0; i < kScatterBatch; ++i) {
          acc[0] = acc[0] + DF{a[i].x, a[i].y};
          acc[1] = acc[1] + DF{a[i].z, a[i].w};
          acc[2] = acc[2] + DF{b[i].x, b[i].y};
          acc[3] = acc[3] + DF{b[i].z, b[i].w};
        }
      }
    }
    for (; r < r1; ++r) {
      const TD* e = d_bar + (int64_t)rev_idx[r] * NV;
      if constexpr (NV == 4) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(e));
        const float4 b = __ldg(reinterpret_cast<const float4*>(e) + 1);
        acc[0] = acc[0] + DF{a.x, a.y};
        acc[1] = acc[1] + DF{a.z, a.w};
        acc[2] = acc[2] + DF{b.x, b.y};
        acc[3] = acc[3] + DF{b.z, b.w};
      } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = acc[v] + e[v];
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v * n_pad + j] = to_d(acc[v]);
  } else {
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = u_self[v];
    for (int64_t r = r0; r < r1; ++r) {
      const TD* e = d_bar + (int64_t)rev_idx[r] * NV;
      if constexpr (NV == 4) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(e));
        const double2 b = __ldg(reinterpret_cast<const double2*>(e) + 1);
        acc[0] += a.x;
        acc[1] += a.y;
        acc[2] += b.x;
        acc[3] += b.y;
      } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += e[v];
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v * n_pad + j] = acc[v];
  }
}

template <typename F>
cudaError_t dispatch_order(int order, F&& f) {
  switch (order) {
    case 3: return f(std::integral_constant<int, 5>{}, std::integral_constant<int, 12>{});
    case 4: return f(std::integral_constant<int, 9>{}, std::integral_constant<int, 20>{});
    case 5: return f(std::integral_constant<int, 14>{}, std::integral_constant<int, 30>{});
    case 6: return f(std::integral_constant<int, 20>{}, std::integral_constant<int, 42>{});
  }
  return cudaErrorInvalidValue;
}

}  // namespace

// ---------------------------------------------------------------- launchers
template <int M, int NS, int NQ, bool kDF, bool kExt>
cudaError_t launch_recon_tma(const ReconArgs& a, const DeviceMesh& dm, int* err, cudaStream_t st) {
  using TR = TmaTraits<kDF, M, NS, NQ>;
  using P = StagePlan<M, NS, (int)sizeof(typename TR::TE), TR::kLPS, TR::kSPS, TR::kRing>;
  auto kern = recon_tma_kernel<M, NS, NQ, kDF, kExt>;
  const int threads = kTile * (kConsumers + 1);
  constexpr bool kStage = TENO_STAGE_OUT && !kExt && !kDF;
  const size_t smem = P::kSmem + (kStage ? out_stage_bytes<3 * NQ * 4, float>() : 0);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem)) !=
      cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t tiles = (a.n_cell + kTile - 1) / kTile;
  const int64_t grid = std::min<int64_t>(tiles, (int64_t)per_sm * sms);
  kern<<<(unsigned)grid, threads, smem, st>>>(a, dm.halo, dm.eval_df, err);
  return cudaGetLastError();
}

template <int M, int NS, int NQ, bool kN>
cudaError_t launch_recon_tma_w(const ReconArgs& a, const DeviceMesh& dm, int* err,
                               cudaStream_t st) {
  using P = WPlan<M, NS, 3 * NQ, 3, 4>;
  auto kern = recon_tma_w_kernel<M, NS, NQ, kN>;
  const int threads = kTile * (kConsumers + 1);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)P::kSmem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, P::kSmem)) !=
      cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t tiles = (a.n_cell + kTile - 1) / kTile;
  const int64_t grid = std::min<int64_t>(tiles, (int64_t)per_sm * sms);
  const void* psi = kN ? (const void*)dm.psi_d : (const void*)dm.psi_df;
  kern<<<(unsigned)grid, threads, P::kSmem, st>>>(a, dm.halo, psi, dm.g32, dm.wq, err);
  return cudaGetLastError();
}

cudaError_t launch_char_finish(const DeviceMesh& dm, const double* U, void* Uq, cudaStream_t st) {
  if (!dm.coef_out || dm.n_var != 4) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)((dm.n_recon * 3 + 127) / 128);
  return dispatch_order(dm.order, [&](auto Mc, auto NSc) -> cudaError_t {
    constexpr int M = decltype(Mc)::value;
    (void)NSc;
    constexpr int NQ = (M <= 9) ? 2 : 3;
    if (dm.nq != NQ) return cudaErrorInvalidValue;
    auto go = [&](auto tq) -> cudaError_t {
      using TQ = typename decltype(tq)::type;
      if constexpr (std::is_same<TQ, double>::value)
        char_finish_kernel<M, NQ, TQ><<<grid, 128, 0, st>>>(
            dm.coef_out, U, dm.smask, dm.c_faces, dm.f_geom, dm.eval, (TQ*)Uq, dm.n_recon,
            dm.n_pad, dm.gamma, dm.ct, dm.eps, dm.linear);
      else
        char_finish_df_kernel<M, NQ, TQ><<<grid, 128, 0, st>>>(
            reinterpret_cast<const float2*>(dm.coef_out), U, dm.smask, dm.c_faces, dm.f_geom,
            dm.eval_df, (TQ*)Uq, dm.n_recon, dm.n_pad, dm.gamma, dm.ct, dm.eps, dm.linear);
      return cudaGetLastError();
    };
    if (dm.precision == TENO_FP64) return go(TypeTag<DF>{});
    if (dm.precision == TENO_FP32_MIXED) return go(TypeTag<float>{});
    return go(TypeTag<double>{});
  });
}

cudaError_t launch_recon(const DeviceMesh& dm, const double* U, const float2* Us, void* Uq,
                         uint8_t* sel_out, const uint8_t* sel_in, cudaStream_t st) {
  if (dm.precision != TENO_FP64_NATIVE && !Us) return cudaErrorInvalidValue;
  ReconArgs a;
  a.ahat = dm.ahat;
  a.nbr = dm.nbr;
  a.smask = dm.smask;
  a.U = U;
  a.Us = Us;
  a.Uq = Uq;
  a.sel_out = sel_out;
  a.sel_in = sel_in;
  a.n_cell = dm.n_recon;  // the cells reconstructed (all cells, or a partition's compute set)
  a.n_pad = dm.n_pad;
  a.ct = dm.ct;
  a.eps = dm.eps;
  a.linear = dm.linear;
  a.e_entries = dm.e_entries;
  a.scheme = dm.scheme;
  a.cw_dK = 1.0 - 1.0 / dm.cweno_dk;
  a.coef_out = dm.charvar ? dm.coef_out : nullptr;
  a.force_near = dm.debug & 1;
  a.wait_polls = (dm.debug & 2) ? 0u : kWaitLimit;
  const int64_t tiles = (a.n_cell + kTile - 1) / kTile;
  return dispatch_order(dm.order, [&](auto Mc, auto NSc) -> cudaError_t {
    constexpr int M = decltype(Mc)::value, NS = decltype(NSc)::value;
    auto go = [&](auto nqc, auto nvc) -> cudaError_t {
      constexpr int NQ = decltype(nqc)::value, NV = decltype(nvc)::value;
      // the TMA kernel covers Euler on the pair and mixed paths; variant 2
      // elsewhere takes the halo kernel. CWENO and the characteristic mode
      // take the TMA or the direct kernels: the halo kernel is compiled for
      // TENO in conservative variables only.
      const bool ext = dm.scheme != 0 || dm.charvar != 0;
      // the native FP64 path has the W-form kernel only (no pair TMA kernel)
      const bool wn = NV == 4 && dm.variant == 2 && dm.err_flag && dm.halo.off && !ext &&
                      dm.precision == TENO_FP64_NATIVE && dm.g32 && dm.wq && dm.psi_d;
      if constexpr (NV == 4) {
        if (wn) return launch_recon_tma_w<M, NS, NQ, true>(a, dm, dm.err_flag, st);
      }
      const bool tma = NV == 4 && dm.variant == 2 && dm.err_flag && dm.halo.off &&
                       dm.precision != TENO_FP64_NATIVE;
      if (!ext && (dm.variant == 0 || (dm.variant == 2 && !tma)) && dm.halo.off) {
        constexpr int TZh = 4 / NV;
        dim3 block(kTile, NV, TZh);
        dim3 grid((unsigned)((tiles + TZh - 1) / TZh));
        if (dm.precision == TENO_FP64)
          recon_halo_kernel<M, NS, NQ, NV, 0><<<grid, block, 0, st>>>(a, dm.halo, dm.eval_df);
        else if (dm.precision == TENO_FP32_MIXED)
          recon_halo_kernel<M, NS, NQ, NV, 1><<<grid, block, 0, st>>>(a, dm.halo, dm.eval_df);
        else
          recon_halo_kernel<M, NS, NQ, NV, 2><<<grid, block, 0, st>>>(a, dm.halo, dm.eval);
        return cudaGetLastError();
      }
      if constexpr (NV == 4) {
        if (tma) {
          if (dm.precision == TENO_FP64 && dm.scheme == 0 && dm.g32 && dm.wq && dm.psi_df)
            return launch_recon_tma_w<M, NS, NQ, false>(a, dm, dm.err_flag, st);
          if (ext) {
            if (dm.precision == TENO_FP64)
              return launch_recon_tma<M, NS, NQ, true, true>(a, dm, dm.err_flag, st);
            return launch_recon_tma<M, NS, NQ, false, true>(a, dm, dm.err_flag, st);
          }
          if (dm.precision == TENO_FP64)
            return launch_recon_tma<M, NS, NQ, true, false>(a, dm, dm.err_flag, st);
          return launch_recon_tma<M, NS, NQ, false, false>(a, dm, dm.err_flag, st);
        }
      }
      constexpr int TZ = 4 / NV;  // 128 threads per block
      dim3 block(kTile, NV, TZ);
      dim3 grid((unsigned)((tiles + TZ - 1) / TZ));
      if (dm.precision == TENO_FP64_NATIVE)
        recon_kernel<M, NS, NQ, NV, double, EvalTable><<<grid, block, 0, st>>>(a, dm.eval);
      else if (dm.precision == TENO_FP64)
        recon_df_kernel<M, NS, NQ, NV><<<grid, block, 0, st>>>(a, dm.eval_df);
      else
        recon_kernel<M, NS, NQ, NV, float, DFTable><<<grid, block, 0, st>>>(a, dm.eval_df);
      return cudaGetLastError();
    };
    constexpr int NQd = (M <= 9) ? 2 : 3;
    if (dm.nq != NQd) return cudaErrorInvalidValue;
    if (dm.n_var == 1) return go(std::integral_constant<int, NQd>{}, std::integral_constant<int, 1>{});
    return go(std::integral_constant<int, NQd>{}, std::integral_constant<int, 4>{});
  });
}

// (hi, lo) float pair of a double, on the host
static float2 split2(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

static FaceArgs face_args(const DeviceMesh& dm, double time) {
  FaceArgs a;
  a.f_cells = dm.f_cells;
  a.f_edges = dm.f_edges;
  a.f_geom = dm.f_geom;
  a.f_geom2 = dm.f_geom2;
  a.n_pad = dm.n_pad;
  a.n_face = dm.n_face;
  a.gamma = dm.gamma;
  a.adv_x = dm.adv_x;
  a.adv_y = dm.adv_y;
  a.adv_field = dm.adv_field;
  a.adv_cx = dm.adv_cx;
  a.adv_cy = dm.adv_cy;
  a.adv_omega = dm.adv_omega;
  a.adv_r1 = dm.adv_r1;
  a.adv_r2 = dm.adv_r2;
  a.time = time;
  for (int k = 0; k < kMaxNq; ++k) {
    a.gw[k] = dm.gw[k];
    a.gt[k] = dm.gt[k];
    a.gw2[k] = split2(dm.gw[k]);
  }
  a.g2 = split2(dm.gamma);
  a.gm12 = split2(dm.gamma - 1.0);
  return a;
}

cudaError_t launch_face_flux(const DeviceMesh& dm, const void* Uq, void* K, double time,
                             cudaStream_t st) {
  FaceArgs a = face_args(dm, time);
  const unsigned grid = (unsigned)((dm.n_face + 255) / 256);
  auto go = [&](auto nvc, auto nqc, auto flc) -> cudaError_t {
    constexpr int NV = decltype(nvc)::value, NQ = decltype(nqc)::value,
                  FL = decltype(flc)::value;
    if (dm.precision == TENO_FP64_NATIVE)
      face_flux_kernel<NV, NQ, FL, double><<<grid, 256, 0, st>>>(
          a, (const double*)Uq, (double*)K);
    else if (dm.precision == TENO_FP64)
      face_flux_kernel<NV, NQ, FL, DF><<<grid, 256, 0, st>>>(a, (const DF*)Uq, (DF*)K);
    else
      face_flux_kernel<NV, NQ, FL, float><<<grid, 256, 0, st>>>(a, (const float*)Uq, (float*)K);
    return cudaGetLastError();
  };
  using I1 = std::integral_constant<int, 1>;
  using I2 = std::integral_constant<int, 2>;
  using I3 = std::integral_constant<int, 3>;
  using I4 = std::integral_constant<int, 4>;
  using F0 = std::integral_constant<int, TENO_FLUX_UPWIND>;
  using F1 = std::integral_constant<int, TENO_FLUX_HLL>;
  using F2 = std::integral_constant<int, TENO_FLUX_HLLC>;
  if (dm.n_var == 1) return dm.nq == 2 ? go(I1{}, I2{}, F0{}) : go(I1{}, I3{}, F0{});
  if (dm.flux == TENO_FLUX_HLL) return dm.nq == 2 ? go(I4{}, I2{}, F1{}) : go(I4{}, I3{}, F1{});
  return dm.nq == 2 ? go(I4{}, I2{}, F2{}) : go(I4{}, I3{}, F2{});
}

cudaError_t launch_gather(const DeviceMesh& dm, const void* K, const double* Un, const double* Us,
                          double* out, int mode, double cn, double cs, double dt_fixed,
                          const double* max_lam, int* flag, float2* split, cudaStream_t st) {
  GatherArgs a{dm.c_faces, dm.inv_area, dm.n_update, dm.n_pad, dm.gamma};
  const unsigned grid = (unsigned)((dm.n_update + 255) / 256);
  auto go = [&](auto nvc, auto tkc) {
    constexpr int NV = decltype(nvc)::value;
    using TK = typename decltype(tkc)::type;
    gather_kernel<NV, TK><<<grid, 256, 0, st>>>(a, (const TK*)K, Un, Us, out, mode, cn, cs,
                                                dt_fixed, dm.cfl, max_lam, flag, split);
  };
  using I1 = std::integral_constant<int, 1>;
  using I4 = std::integral_constant<int, 4>;
  const bool one = dm.n_var == 1;
  if (dm.precision == TENO_FP64_NATIVE) {
    if (one) go(I1{}, TypeTag<double>{}); else go(I4{}, TypeTag<double>{});
  } else if (dm.precision == TENO_FP64) {
    if (one) go(I1{}, TypeTag<DF>{}); else go(I4{}, TypeTag<DF>{});
  } else {
    if (one) go(I1{}, TypeTag<float>{}); else go(I4{}, TypeTag<float>{});
  }
  return cudaGetLastError();
}

cudaError_t launch_layer_fill(const DeviceMesh& dm, const double* U, void* Uq, cudaStream_t st) {
  if (!dm.fo_n) return cudaSuccess;
  const int64_t nt = dm.fo_n * 3 * dm.nq;
  const unsigned grid = (unsigned)((nt + 255) / 256);
  auto go = [&](auto nvc, auto nqc) {
    constexpr int NV = decltype(nvc)::value, NQ3 = 3 * decltype(nqc)::value;
    if (dm.precision == TENO_FP64)
      layer_fill_kernel<NV, NQ3, DF><<<grid, 256, 0, st>>>(U, (DF*)Uq, dm.fo_list, dm.fo_n,
                                                            dm.n_pad);
    else if (dm.precision == TENO_FP32_MIXED)
      layer_fill_kernel<NV, NQ3, float><<<grid, 256, 0, st>>>(U, (float*)Uq, dm.fo_list,
                                                              dm.fo_n, dm.n_pad);
    else
      layer_fill_kernel<NV, NQ3, double><<<grid, 256, 0, st>>>(U, (double*)Uq, dm.fo_list,
                                                               dm.fo_n, dm.n_pad);
  };
  using I1 = std::integral_constant<int, 1>;
  using I4 = std::integral_constant<int, 4>;
  using Q2 = std::integral_constant<int, 2>;
  using Q3 = std::integral_constant<int, 3>;
  if (dm.n_var == 1) {
    if (dm.nq == 2) go(I1{}, Q2{}); else go(I1{}, Q3{});
  } else {
    if (dm.nq == 2) go(I4{}, Q2{}); else go(I4{}, Q3{});
  }
  return cudaGetLastError();
}

cudaError_t launch_layer_vjp(const DeviceMesh& dm, double* Uq_bar, double* ubd, cudaStream_t st) {
  if (!dm.fo_n) return cudaSuccess;
  const unsigned grid = (unsigned)((dm.fo_n * 3 + 255) / 256);
  const bool pairs = dm.precision == TENO_FP64;
  auto go = [&](auto nvc, auto nqc) {
    constexpr int NV = decltype(nvc)::value, NQ = decltype(nqc)::value;
    if (pairs)
      layer_vjp_kernel<NV, NQ, true><<<grid, 256, 0, st>>>(Uq_bar, ubd, dm.fo_list, dm.fo_n);
    else
      layer_vjp_kernel<NV, NQ, false><<<grid, 256, 0, st>>>(Uq_bar, ubd, dm.fo_list, dm.fo_n);
  };
  using I1 = std::integral_constant<int, 1>;
  using I4 = std::integral_constant<int, 4>;
  using Q2 = std::integral_constant<int, 2>;
  using Q3 = std::integral_constant<int, 3>;
  if (dm.n_var == 1) {
    if (dm.nq == 2) go(I1{}, Q2{}); else go(I1{}, Q3{});
  } else {
    if (dm.nq == 2) go(I4{}, Q2{}); else go(I4{}, Q3{});
  }
  return cudaGetLastError();
}

cudaError_t launch_positivity(const DeviceMesh& dm, const double* U, void* Uq,
                              cudaStream_t st) {
  if (dm.n_var != 4) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)((dm.n_recon + 127) / 128);
  auto go = [&](auto nq, auto tq) -> cudaError_t {
    constexpr int NQ = decltype(nq)::value;
    using TQ = typename decltype(tq)::type;
    positivity_kernel<NQ, TQ><<<grid, 128, 0, st>>>(U, (TQ*)Uq, dm.n_recon, dm.n_pad, dm.gamma);
    return cudaGetLastError();
  };
  auto by_type = [&](auto nq) -> cudaError_t {
    if (dm.precision == TENO_FP64) return go(nq, TypeTag<DF>{});
    if (dm.precision == TENO_FP32_MIXED) return go(nq, TypeTag<float>{});
    return go(nq, TypeTag<double>{});
  };
  if (dm.nq == 2) return by_type(std::integral_constant<int, 2>{});
  if (dm.nq == 3) return by_type(std::integral_constant<int, 3>{});
  return cudaErrorInvalidValue;
}

cudaError_t launch_halo_pack(const double* U, int64_t ld, const int32_t* idx, int64_t n,
                             int n_var, double* buf, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  halo_pack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(U, ld, idx, n, n_var, buf);
  return cudaGetLastError();
}
cudaError_t launch_halo_unpack(double* U, int64_t ld, const int32_t* idx, int64_t n, int n_var,
                               const double* buf, float2* Us, int add, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  halo_unpack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(U, ld, idx, n, n_var, buf, Us,
                                                                 add);
  return cudaGetLastError();
}

cudaError_t launch_split(const DeviceMesh& dm, const double* U, float2* Us, cudaStream_t st) {
  split_kernel<<<(unsigned)((dm.n_cell + 255) / 256), 256, 0, st>>>(U, Us, dm.n_cell, dm.n_pad,
                                                                    dm.n_var);
  return cudaGetLastError();
}

cudaError_t launch_max_lambda(const DeviceMesh& dm, const double* U, double* max_lam,
                              cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(max_lam, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  int64_t blocks = (dm.n_update + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  const double adv = sqrt(dm.adv_x * dm.adv_x + dm.adv_y * dm.adv_y);
  if (dm.n_var == 1)
    max_lambda_kernel<1><<<(unsigned)blocks, 256, 0, st>>>(
        U, dm.cfl_len, dm.n_update, dm.n_pad, dm.gamma, adv, dm.cell_speed,
        (unsigned long long*)max_lam);
  else
    max_lambda_kernel<4><<<(unsigned)blocks, 256, 0, st>>>(
        U, dm.cfl_len, dm.n_update, dm.n_pad, dm.gamma, adv, nullptr,
        (unsigned long long*)max_lam);
  return cudaGetLastError();
}

cudaError_t launch_max_lambda_split(const DeviceMesh& dm, const float2* Us, double* max_lam,
                                    cudaStream_t st) {
  if (dm.n_var != 4 || !dm.cfl_ilen2 || !Us) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(max_lam, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  int64_t blocks = (dm.n_update + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  max_lambda_split_kernel<<<(unsigned)blocks, 256, 0, st>>>(
      Us, dm.cfl_ilen2, dm.n_update, dm.n_pad, split2(dm.gamma), split2(dm.gamma - 1.0),
      (unsigned long long*)max_lam);
  return cudaGetLastError();
}

cudaError_t launch_permute(const double* src, double* dst, const int32_t* perm, int64_t n,
                           int64_t ld_src, int64_t ld_dst, int n_var, int to_user,
                           cudaStream_t st) {
  dim3 grid((unsigned)((n + 255) / 256), n_var);
  permute_kernel<<<grid, 256, 0, st>>>(src, dst, perm, n, ld_src, ld_dst, to_user);
  return cudaGetLastError();
}

cudaError_t launch_permute_u8(const uint8_t* src, uint8_t* dst, const int32_t* perm, int64_t n,
                              int64_t ld_src, int64_t ld_dst, int n_var, int to_user,
                              cudaStream_t st) {
  dim3 grid((unsigned)((n + 255) / 256), n_var);
  permute_u8_kernel<<<grid, 256, 0, st>>>(src, dst, perm, n, ld_src, ld_dst, to_user);
  return cudaGetLastError();
}

cudaError_t launch_axpby(double* out, const double* a, double ca, const double* b, double cb,
                         int64_t n, cudaStream_t st) {
  axpby_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, a, ca, b, cb, n);
  return cudaGetLastError();
}

#ifndef TENO_VJP_DIRS
#define TENO_VJP_DIRS 2
#endif
constexpr int kVjpDirs = TENO_VJP_DIRS;

cudaError_t launch_face_flux_vjp(const DeviceMesh& dm, const void* Uq, const double* w,
                                 double* Uq_bar, double time, cudaStream_t st) {
  VjpArgs a;
  a.f_cells = dm.f_cells;
  a.f_edges = dm.f_edges;
  a.f_geom = dm.f_geom;
  a.f_geom2 = dm.f_geom2;
  a.g2 = split2(dm.gamma);
  a.gm12 = split2(dm.gamma - 1.0);
  a.inv_area = dm.inv_area;
  a.n_face = dm.n_face;
  a.n_pad = dm.n_pad;
  a.gamma = dm.gamma;
  a.adv_x = dm.adv_x;
  a.adv_y = dm.adv_y;
  a.adv_field = dm.adv_field;
  a.adv_cx = dm.adv_cx;
  a.adv_cy = dm.adv_cy;
  a.adv_omega = dm.adv_omega;
  a.adv_r1 = dm.adv_r1;
  a.adv_r2 = dm.adv_r2;
  a.time = time;
  for (int k = 0; k < kMaxNq; ++k) {
    a.gw[k] = dm.gw[k];
    a.gt[k] = dm.gt[k];
    a.gw2[k] = split2(dm.gw[k]);
  }
  const unsigned grid = (unsigned)((dm.n_face + 127) / 128);
  auto go = [&](auto nvc, auto nqc, auto flc, auto tqc) {
    constexpr int NV = decltype(nvc)::value, NQ = decltype(nqc)::value,
                  FL = decltype(flc)::value;
    using TQ = typename decltype(tqc)::type;
    // pairs: FP32-pipe dual numbers, kVjpDirs directions per pass; FP64:
    // all 2 NV directions of an interior face in one pass
    if constexpr (std::is_same<TQ, DF>::value) {
      constexpr int ND = NV < kVjpDirs ? NV : kVjpDirs;
      face_flux_vjp_kernel<NV, NQ, FL, TQ, DF, ND><<<grid, 128, 0, st>>>(a, (const TQ*)Uq, w,
                                                                        Uq_bar);
    } else {
      face_flux_vjp_kernel<NV, NQ, FL, TQ, double, 2 * NV><<<grid, 128, 0, st>>>(
          a, (const TQ*)Uq, w, Uq_bar);
    }
  };
  using I1 = std::integral_constant<int, 1>;
  using I2 = std::integral_constant<int, 2>;
  using I3 = std::integral_constant<int, 3>;
  using I4 = std::integral_constant<int, 4>;
  using F0 = std::integral_constant<int, TENO_FLUX_UPWIND>;
  using F1 = std::integral_constant<int, TENO_FLUX_HLL>;
  using F2 = std::integral_constant<int, TENO_FLUX_HLLC>;
  auto pick = [&](auto tqc) {
    if (dm.n_var == 1) {
      if (dm.nq == 2) go(I1{}, I2{}, F0{}, tqc); else go(I1{}, I3{}, F0{}, tqc);
    } else if (dm.flux == TENO_FLUX_HLL) {
      if (dm.nq == 2) go(I4{}, I2{}, F1{}, tqc); else go(I4{}, I3{}, F1{}, tqc);
    } else {
      if (dm.nq == 2) go(I4{}, I2{}, F2{}, tqc); else go(I4{}, I3{}, F2{}, tqc);
    }
  };
  if (dm.precision == TENO_FP64)
    pick(TypeTag<DF>{});
  else
    pick(TypeTag<double>{});
  return cudaGetLastError();
}

cudaError_t launch_recon_vjp(const DeviceMesh& dm, const uint8_t* sel, const double* Uq_bar,
                             double* d_bar, double* u_self, cudaStream_t st) {
  const int64_t tiles = (dm.n_recon + kTile - 1) / kTile;
  return dispatch_order(dm.order, [&](auto Mc, auto NSc) -> cudaError_t {
    constexpr int M = decltype(Mc)::value, NS = decltype(NSc)::value;
    constexpr int NQ = (M <= 9) ? 2 : 3;
    if (dm.nq != NQ) return cudaErrorInvalidValue;
    auto go = [&](auto nvc, auto tsc) {
      constexpr int NV = decltype(nvc)::value;
      using TS = typename decltype(tsc)::type;
      constexpr int TZ = 4 / NV;
      dim3 block(kTile, NV, TZ);
      const unsigned grid = (unsigned)((tiles + TZ - 1) / TZ);
      if constexpr (std::is_same<TS, float2>::value)
        recon_vjp_df_kernel<M, NS, NQ, NV><<<grid, block, 0, st>>>(
            (const float2*)dm.ahat, sel, Uq_bar, (DF*)d_bar, u_self, dm.n_recon, dm.n_pad,
            dm.eval_df);
      else
        recon_vjp_kernel<M, NS, NQ, NV, TS><<<grid, block, 0, st>>>(
            (const TS*)dm.ahat, sel, Uq_bar, d_bar, u_self, dm.n_recon, dm.n_pad, dm.eval);
    };
    using I1 = std::integral_constant<int, 1>;
    using I4 = std::integral_constant<int, 4>;
    if (dm.precision == TENO_FP64) {
      if (dm.n_var == 1) go(I1{}, TypeTag<float2>{});
      else go(I4{}, TypeTag<float2>{});
    } else {
      if (dm.n_var == 1) go(I1{}, TypeTag<double>{});
      else go(I4{}, TypeTag<double>{});
    }
    return cudaGetLastError();
  });
}

template <int M, int NS, int NQ>
cudaError_t launch_recon_vjp_tma_t(const DeviceMesh& dm, const uint8_t* sel, const double* Uq_bar,
                                   float2* part, double* u_self, cudaStream_t st) {
  using VP = VjpPlan<M, NS, 3 * NQ>;
  auto kern = recon_vjp_tma_kernel<M, NS, NQ>;
  const int threads = kTile * (kConsumers + 1);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)VP::kSmem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, VP::kSmem)) !=
      cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t tiles = (dm.n_recon + kTile - 1) / kTile;
  const int64_t grid = std::min<int64_t>(tiles, (int64_t)per_sm * sms);
  kern<<<(unsigned)grid, threads, VP::kSmem, st>>>((const float2*)dm.ahat, dm.wq, dm.halo, sel,
                                                   Uq_bar, part, u_self, dm.n_recon, dm.n_pad,
                                                   dm.eval_df, dm.err_flag);
  return cudaGetLastError();
}

cudaError_t launch_recon_vjp_tma(const DeviceMesh& dm, const uint8_t* sel, const double* Uq_bar,
                                 double* part, double* u_self, cudaStream_t st) {
  if (dm.precision != TENO_FP64 || dm.n_var != 4 || !dm.halo.off || !dm.wq || !dm.err_flag)
    return cudaErrorInvalidValue;
  return dispatch_order(dm.order, [&](auto Mc, auto NSc) -> cudaError_t {
    constexpr int M = decltype(Mc)::value, NS = decltype(NSc)::value;
    constexpr int NQ = (M <= 9) ? 2 : 3;
    if (dm.nq != NQ) return cudaErrorInvalidValue;
    return launch_recon_vjp_tma_t<M, NS, NQ>(dm, sel, Uq_bar, reinterpret_cast<float2*>(part),
                                             u_self, st);
  });
}

cudaError_t launch_scatter_gather(const DeviceMesh& dm, const int64_t* rev_off,
                                  const int32_t* rev_idx, const double* d_bar,
                                  const double* u_self, double* v, const double* ubd,
                                  cudaStream_t st) {
  const unsigned grid = (unsigned)((dm.n_cell + 255) / 256);
  const bool pairs = dm.precision == TENO_FP64;  // d_bar holds (hi, lo) pairs
  if (dm.n_var == 1) {
    if (pairs)
      scatter_gather_kernel<1, DF><<<grid, 256, 0, st>>>(rev_off, rev_idx, (const DF*)d_bar,
                                                         u_self, v, dm.n_cell, dm.n_pad, ubd);
    else
      scatter_gather_kernel<1, double><<<grid, 256, 0, st>>>(rev_off, rev_idx, d_bar, u_self, v,
                                                             dm.n_cell, dm.n_pad, ubd);
  } else {
    if (pairs)
      scatter_gather_kernel<4, DF><<<grid, 256, 0, st>>>(rev_off, rev_idx, (const DF*)d_bar,
                                                         u_self, v, dm.n_cell, dm.n_pad, ubd);
    else
      scatter_gather_kernel<4, double><<<grid, 256, 0, st>>>(rev_off, rev_idx, d_bar, u_self, v,
                                                             dm.n_cell, dm.n_pad, ubd);
  }
  return cudaGetLastError();
}
}  // namespace teno
