// Device-side ideal-MHD building blocks (templated on the working precision).
//
// Method (arXiv 2211.12867, Sect. 2.1): ideal MHD solved in the frame
// co-rotating with the Sun with the TVDLF scheme and the Woodward limiter.
// The limiter is the monotonised-central slope applied to the primitive
// variables in index space; a face whose reconstructed density or pressure is
// not positive falls back to the cell values; the TVDLF flux is
// F = (F_L + F_R)/2 - c_max (U_R - U_L)/2 with c_max the larger |v_n| + c_f of
// the two face states; the normal magnetic flux is zero.
#pragma once
#include "icarus_internal.h"

template <typename real> struct RT;
template <> struct RT<double> {
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double abs_(double x) { return fabs(x); }
  static __device__ __forceinline__ double min_(double a, double b) { return fmin(a, b); }
  static __device__ __forceinline__ double max_(double a, double b) { return fmax(a, b); }
  static __device__ __forceinline__ double rcp_(double x) { return __drcp_rn(x); }
};
// FP32 mode: reciprocal and square root are the hardware approximations
// (PTX rcp.approx / sqrt.approx, relative error within about 1 ulp); the
// FP32 stencil is an approximation of the FP64 one at the 1e-6 level anyway
// and the correctly rounded forms cost several dependent instructions each.
template <> struct RT<float> {
  static __device__ __forceinline__ float sqrt_(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  }
  static __device__ __forceinline__ float abs_(float x) { return fabsf(x); }
  static __device__ __forceinline__ float min_(float a, float b) { return fminf(a, b); }
  static __device__ __forceinline__ float max_(float a, float b) { return fmaxf(a, b); }
  static __device__ __forceinline__ float rcp_(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  }
};

// Pressure from conserved variables.  In the mixed-precision mode the FP32
// result is replaced by an FP64 recomputation from the same (FP32-stored)
// conserved variables where the thermal energy is a small remainder of the
// total: p < pe * e or plasma beta = p / (B^2/2) < beta (settable; the
// library's defaults are pe = 0.002 and beta = 0.1).
struct Isl {
  float pe, beta;
};

template <typename real>
__device__ __forceinline__ real pressure_of(const real *u, real gamma, Isl) {
  real ir = RT<real>::rcp_(u[0]);
  real msq = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
  real me = real(0.5) * (u[5] * u[5] + u[6] * u[6] + u[7] * u[7]);
  real p = (gamma - real(1)) * (u[4] - real(0.5) * msq * ir - me);
  return p;
}

// FP64 pressure from FP32-stored variables.  The product of two floats is
// exact in double, so m.m and B.B carry no rounding beyond the double sums;
// 1/rho starts from the float reciprocal and one Newton step in double brings
// it to double accuracy (no FP64 division).
__device__ __forceinline__ float pressure_fp64_island(const float *u, float gamma) {
  const double r = u[0];
  double ri = (double)__frcp_rn(u[0]);
  ri = fma(ri, fma(-r, ri, 1.0), ri);
  const double m1 = u[1], m2 = u[2], m3 = u[3], b1 = u[5], b2 = u[6], b3 = u[7];
  const double ms = fma(m1, m1, fma(m2, m2, m3 * m3));
  const double bs = fma(b1, b1, fma(b2, b2, b3 * b3));
  const double h = fma(-0.5, bs, (double)u[4]);
  return (float)(((double)gamma - 1.0) * fma(-0.5 * ms, ri, h));
}

// float pressure without the island (accurate to ~1e-6 e; 1/rho is the
// approximate reciprocal, relative error below 2^-22, so the kinetic energy
// is off by at most ~3e-7 of e)
__device__ __forceinline__ float pressure_fp32(const float *u, float gamma) {
  const float ir = RT<float>::rcp_(u[0]);
  float msq = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
  float me = 0.5f * (u[5] * u[5] + u[6] * u[6] + u[7] * u[7]);
  return (gamma - 1.0f) * (u[4] - 0.5f * msq * ir - me);
}

template <>
__device__ __forceinline__ float pressure_of<float>(const float *u, float gamma, Isl isl) {
  float p = pressure_fp32(u, gamma);
  const float me = 0.5f * (u[5] * u[5] + u[6] * u[6] + u[7] * u[7]);
  if (p < isl.pe * u[4] || p < isl.beta * me) p = pressure_fp64_island(u, gamma);
  return p;
}

// pressure for the CFL wave speed: the float value suffices (relative error
// ~1e-6 e / p on a time-step bound taken with a 0.8 safety factor)
template <typename real>
__device__ __forceinline__ real pressure_for_speed(const real *u, real gamma) {
  return pressure_of<real>(u, gamma, Isl{0.f, 0.f});
}
template <>
__device__ __forceinline__ float pressure_for_speed<float>(const float *u, float gamma) {
  return pressure_fp32(u, gamma);
}

// U -> W with the pressure floor of the stage operator.
template <typename real>
__device__ __forceinline__ void cons2prim(const real *u, real *w, real gamma, real pfloor, Isl isl) {
  real ir = RT<real>::rcp_(u[0]);
  w[0] = u[0];
  w[1] = u[1] * ir;
  w[2] = u[2] * ir;
  w[3] = u[3] * ir;
  real p = pressure_of<real>(u, gamma, isl);
  w[4] = p < pfloor ? pfloor : p;
  w[5] = u[5];
  w[6] = u[6];
  w[7] = u[7];
}

// primitives for the CFL speed (no FP64 island in the FP32 mode)
template <typename real>
__device__ __forceinline__ void cons2prim_speed(const real *u, real *w, real gamma, real pfloor) {
  real ir = RT<real>::rcp_(u[0]);
  w[0] = u[0];
  w[1] = u[1] * ir;
  w[2] = u[2] * ir;
  w[3] = u[3] * ir;
  real p = pressure_for_speed<real>(u, gamma);
  w[4] = p < pfloor ? pfloor : p;
  w[5] = u[5];
  w[6] = u[6];
  w[7] = u[7];
}

template <typename real>
__device__ __forceinline__ void prim2cons(const real *w, real *u, real igm1) {
  real v2 = w[1] * w[1] + w[2] * w[2] + w[3] * w[3];
  real b2 = w[5] * w[5] + w[6] * w[6] + w[7] * w[7];
  u[0] = w[0];
  u[1] = w[0] * w[1];
  u[2] = w[0] * w[2];
  u[3] = w[0] * w[3];
  u[4] = w[4] * igm1 + real(0.5) * w[0] * v2 + real(0.5) * b2;
  u[5] = w[5];
  u[6] = w[6];
  u[7] = w[7];
}

// fast magnetosonic speed along direction D
template <typename real, int D>
__device__ __forceinline__ real fast_speed(const real *w, real gamma) {
  real ir = RT<real>::rcp_(w[0]);
  real a2 = gamma * w[4] * ir;
  real b2 = (w[5] * w[5] + w[6] * w[6] + w[7] * w[7]) * ir;
  real bn2 = w[5 + D] * w[5 + D] * ir;
  real s = a2 + b2;
  real disc = s * s - real(4) * a2 * bn2;
  disc = disc < real(0) ? real(0) : disc;
  return RT<real>::sqrt_(real(0.5) * (s + RT<real>::sqrt_(disc)));
}

// Half the monotonised-central slope: min(|dm|, |dm + dp| / 4, |dp|) with the
// common sign, 0 at an extremum.  Equal, bit for bit, to 0.5 * mc_slope (the
// factors are powers of two), with two multiplications fewer.
template <typename real>
__device__ __forceinline__ real mc_half_slope(real um, real u0, real up) {
  real dm = u0 - um, dp = up - u0;
  real s = dm + dp;
  real lim = RT<real>::min_(RT<real>::min_(RT<real>::abs_(dm), RT<real>::abs_(dp)), real(0.25) * RT<real>::abs_(s));
  lim = s > real(0) ? lim : -lim;
  return dm * dp > real(0) ? lim : real(0);
}

template <typename real>
__device__ __forceinline__ real mc_slope(real um, real u0, real up) {
  real dm = u0 - um, dp = up - u0;
  real dc = real(0.5) * (dm + dp);
  real lim = RT<real>::min_(real(2) * RT<real>::abs_(dm), real(2) * RT<real>::abs_(dp));
  lim = RT<real>::min_(lim, RT<real>::abs_(dc));
  real s = dc > real(0) ? lim : -lim;
  return dm * dp > real(0) ? s : real(0);
}

// physical flux along D from primitives (and the energy density e)
template <typename real, int D>
__device__ __forceinline__ void phys_flux(const real *w, real e, real *F) {
  real vn = w[1 + D], Bn = w[5 + D];
  real b2 = w[5] * w[5] + w[6] * w[6] + w[7] * w[7];
  real pt = w[4] + real(0.5) * b2;
  real vB = w[1] * w[5] + w[2] * w[6] + w[3] * w[7];
  real rvn = w[0] * vn;
  F[0] = rvn;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    F[1 + c] = rvn * w[1 + c] - w[5 + c] * Bn;
    F[5 + c] = vn * w[5 + c] - Bn * w[1 + c];
  }
  F[1 + D] += pt;
  F[5 + D] = real(0);
  F[4] = (e + pt) * vn - Bn * vB;
}

// Elementwise a + s * b over the 8 variables (s = +1 or -1).  FP32 mode uses
// the packed pair instructions of sm_100+ (two lanes per instruction, each
// rounded as the scalar operation would be).
template <typename real>
__device__ __forceinline__ void axpy8(const real *a, real s, const real *b, real *o) {
#pragma unroll
  for (int v = 0; v < NVAR; v++) o[v] = a[v] + s * b[v];
}
template <>
__device__ __forceinline__ void axpy8<float>(const float *a, float s, const float *b, float *o) {
  const float2 ss = make_float2(s, s);
#pragma unroll
  for (int v = 0; v < NVAR; v += 2) {
    const float2 r = __ffma2_rn(ss, make_float2(b[v], b[v + 1]), make_float2(a[v], a[v + 1]));
    o[v] = r.x;
    o[v + 1] = r.y;
  }
}

// Half MC slope from the one-sided differences dm, dp and their sum s, by
// sign arithmetic: with sigma the sign of s, the slope is
// sigma * max(0, min(sigma dm, sigma dp, |s| / 4)) -- zero unless dm and dp
// share s's sign, the same value as mc_half_slope (bar the sign of a zero).
__device__ __forceinline__ float half_mc_signed(float dm, float dp, float s) {
  const unsigned sg = __float_as_uint(s) & 0x80000000u;
  const float a = __uint_as_float(__float_as_uint(dm) ^ sg), b = __uint_as_float(__float_as_uint(dp) ^ sg);
  const float m = fmaxf(fminf(fminf(a, b), 0.25f * fabsf(s)), 0.f);
  return __uint_as_float(__float_as_uint(m) | sg);
}

// Half the monotonised-central slopes of the 8 variables at the middle of
// three cells (see mc_half_slope); the differences go in packed pairs in
// FP32 mode.
template <typename real>
__device__ __forceinline__ void mc_half_slopes8(const real *um, const real *u0, const real *up, real *out) {
#pragma unroll
  for (int v = 0; v < NVAR; v++) out[v] = mc_half_slope<real>(um[v], u0[v], up[v]);
}
template <>
__device__ __forceinline__ void mc_half_slopes8<float>(const float *um, const float *u0, const float *up,
                                                       float *out) {
#pragma unroll
  for (int v = 0; v < NVAR; v += 2) {
    const float2 c = make_float2(u0[v], u0[v + 1]);
    const float2 dm = __fadd2_rn(c, make_float2(-um[v], -um[v + 1]));
    const float2 dp = __fadd2_rn(make_float2(up[v], up[v + 1]), make_float2(-c.x, -c.y));
    const float2 sm = __fadd2_rn(dm, dp);
    out[v] = half_mc_signed(dm.x, dp.x, sm.x);
    out[v + 1] = half_mc_signed(dm.y, dp.y, sm.y);
  }
}

// Flux balance of CH variables of a cell: out[h] = -((Arp Fhi - Arm Flo) +
// (Atp Fth - Atm Ftl) + Ap (Fph - Fpl)) * iV, FP32 in packed pairs.
template <typename real, int CH>
__device__ __forceinline__ void flux_balance(const real *Fhi, const real *Flo, const real *fth, const real *ftl,
                                             const real *fph, const real *fpl, real Arp, real Arm, real Atp,
                                             real Atm, real Ap, real iV, real *out) {
#pragma unroll
  for (int h = 0; h < CH; h++) {
    const real div = (Arp * Fhi[h] - Arm * Flo[h]) + (Atp * fth[h] - Atm * ftl[h]) + Ap * (fph[h] - fpl[h]);
    out[h] = -div * iV;
  }
}
template <>
__device__ __forceinline__ void flux_balance<float, 4>(const float *Fhi, const float *Flo, const float *fth,
                                                       const float *ftl, const float *fph, const float *fpl,
                                                       float Arp, float Arm, float Atp, float Atm, float Ap,
                                                       float iV, float *out) {
  const float2 arp = make_float2(Arp, Arp), narm = make_float2(-Arm, -Arm), atp = make_float2(Atp, Atp),
               natm = make_float2(-Atm, -Atm), ap = make_float2(Ap, Ap), m1 = make_float2(-1.f, -1.f),
               niv = make_float2(-iV, -iV);
#pragma unroll
  for (int h = 0; h < 4; h += 2) {
    const float2 r = __ffma2_rn(narm, make_float2(Flo[h], Flo[h + 1]),
                                __fmul2_rn(arp, make_float2(Fhi[h], Fhi[h + 1])));
    const float2 t = __ffma2_rn(natm, make_float2(ftl[h], ftl[h + 1]),
                                __fmul2_rn(atp, make_float2(fth[h], fth[h + 1])));
    const float2 p = __ffma2_rn(m1, make_float2(fpl[h], fpl[h + 1]), make_float2(fph[h], fph[h + 1]));
    const float2 d = __ffma2_rn(ap, p, __fadd2_rn(r, t));
    const float2 o = __fmul2_rn(d, niv);
    out[h] = o.x;
    out[h + 1] = o.y;
  }
}

// fast magnetosonic speed along D from a face state, its 1/rho and |B|^2
template <typename real, int D>
__device__ __forceinline__ real fast_speed_pre(const real *w, real ir, real b2, real gamma) {
  const real a2 = gamma * w[4] * ir;
  const real bt2 = b2 * ir;
  const real bn2 = w[5 + D] * w[5 + D] * ir;
  const real s = a2 + bt2;
  real disc = s * s - real(4) * a2 * bn2;
  disc = disc < real(0) ? real(0) : disc;
  return RT<real>::sqrt_(real(0.5) * (s + RT<real>::sqrt_(disc)));
}

// One side's part of the TVDLF flux, G = F(W) + sc U(W) with sc = +c_max on
// the left and -c_max on the right, so that the flux is (G_L + G_R) / 2.
// Written out per component with w = v_n + sc:
//   mass rho w;  momentum m_k w - B_n B_k (+ p_T along n);
//   energy e w + p_T v_n - B_n (v.B);  induction B_k w - B_n v_k (k != n).
template <typename real, int D>
__device__ __forceinline__ void side_flux(const real *W, real b2, real igm1, real sc, real *G) {
  const real vn = W[1 + D], Bn = W[5 + D];
  const real w = vn + sc;
  const real m1 = W[0] * W[1], m2 = W[0] * W[2], m3 = W[0] * W[3];
  const real rv2 = m1 * W[1] + m2 * W[2] + m3 * W[3];
  const real pt = W[4] + real(0.5) * b2;
  const real e = W[4] * igm1 + real(0.5) * (rv2 + b2);
  const real vB = W[1] * W[5] + W[2] * W[6] + W[3] * W[7];
  G[0] = W[0] * w;
  G[1] = m1 * w - Bn * W[5];
  G[2] = m2 * w - Bn * W[6];
  G[3] = m3 * w - Bn * W[7];
  G[1 + D] += pt;
  G[4] = e * w + pt * vn - Bn * vB;
#pragma unroll
  for (int k = 0; k < 3; k++) G[5 + k] = k == D ? real(0) : W[5 + k] * w - Bn * W[1 + k];
}

// TVDLF flux from reconstructed face states WL | WR (primitive variables),
// F = (F_L + F_R)/2 - c_max (U_R - U_L)/2, c_max the larger |v_n| + c_f of
// the two states; b, c are the two cell values the face falls back to when a
// reconstructed density or pressure is not positive.  F2 receives TWICE the
// numerical flux (the caller folds the 1/2 into its face areas); the normal
// magnetic flux is zero.
template <typename real, int D>
__device__ __forceinline__ void tvdlf_states(real *WL, real *WR, const real *b, const real *c, real gamma,
                                             real igm1, real *F2) {
  if (!(WL[0] > real(0)) || !(WL[4] > real(0)) || !(WR[0] > real(0)) || !(WR[4] > real(0))) {
#pragma unroll
    for (int v = 0; v < NVAR; v++) {
      WL[v] = b[v];
      WR[v] = c[v];
    }
  }
  const real b2L = WL[5] * WL[5] + WL[6] * WL[6] + WL[7] * WL[7];
  const real b2R = WR[5] * WR[5] + WR[6] * WR[6] + WR[7] * WR[7];
  const real cl = RT<real>::abs_(WL[1 + D]) + fast_speed_pre<real, D>(WL, RT<real>::rcp_(WL[0]), b2L, gamma);
  const real cr = RT<real>::abs_(WR[1 + D]) + fast_speed_pre<real, D>(WR, RT<real>::rcp_(WR[0]), b2R, gamma);
  const real cm = cl > cr ? cl : cr;
  real GL[NVAR], GR[NVAR];
  side_flux<real, D>(WL, b2L, igm1, cm, GL);
  side_flux<real, D>(WR, b2R, igm1, -cm, GR);
  axpy8<real>(GL, real(1), GR, F2);
  F2[5 + D] = real(0);
}

// FP32 TVDLF flux (twice, see tvdlf_states) with the two face states in
// the two lanes of packed pairs (lane x the left state b + hb, lane y the
// right state c - hc; hb, hc the half slopes of cells b | c): the fast speed
// and the per-side flux G = F(W) +- c_max U(W) are computed once for both
// sides with the f32x2 instructions, each lane rounded as the scalar
// operation, and the lanes are added at the end.  A face whose reconstructed
// density or pressure is not positive takes the cell values.
template <int D>
__device__ __forceinline__ void tvdlf_pair(const float *b, const float *c, const float *hb, const float *hc,
                                           float gamma, float igm1, float *F2) {
  float2 W[NVAR];
#pragma unroll
  for (int v = 0; v < NVAR; v++) W[v] = make_float2(b[v] + hb[v], c[v] - hc[v]);
  if (!(W[0].x > 0.f) || !(W[4].x > 0.f) || !(W[0].y > 0.f) || !(W[4].y > 0.f)) {
#pragma unroll
    for (int v = 0; v < NVAR; v++) W[v] = make_float2(b[v], c[v]);
  }
  const float2 half = make_float2(0.5f, 0.5f);
  const float2 b2 = __ffma2_rn(W[7], W[7], __ffma2_rn(W[6], W[6], __fmul2_rn(W[5], W[5])));
  // fast magnetosonic speed along D of both states (fast_speed_pre)
  const float2 ir = make_float2(RT<float>::rcp_(W[0].x), RT<float>::rcp_(W[0].y));
  const float2 a2 = __fmul2_rn(__fmul2_rn(make_float2(gamma, gamma), W[4]), ir);
  const float2 bt2 = __fmul2_rn(b2, ir);
  const float2 bn2 = __fmul2_rn(__fmul2_rn(W[5 + D], W[5 + D]), ir);
  const float2 sum = __fadd2_rn(a2, bt2);
  float2 disc = __ffma2_rn(sum, sum, __fmul2_rn(__fmul2_rn(make_float2(-4.f, -4.f), a2), bn2));
  disc.x = fmaxf(disc.x, 0.f);
  disc.y = fmaxf(disc.y, 0.f);
  const float2 cf2 =
      __fmul2_rn(half, __fadd2_rn(sum, make_float2(RT<float>::sqrt_(disc.x), RT<float>::sqrt_(disc.y))));
  const float cm = fmaxf(fabsf(W[1 + D].x) + RT<float>::sqrt_(cf2.x), fabsf(W[1 + D].y) + RT<float>::sqrt_(cf2.y));
  // per-side flux with w = v_n + c_max on the left, v_n - c_max on the right
  const float2 vn = W[1 + D], nBn = __fmul2_rn(W[5 + D], make_float2(-1.f, -1.f));
  const float2 w = __fadd2_rn(vn, make_float2(cm, -cm));
  const float2 m1 = __fmul2_rn(W[0], W[1]), m2 = __fmul2_rn(W[0], W[2]), m3 = __fmul2_rn(W[0], W[3]);
  const float2 rv2 = __ffma2_rn(m3, W[3], __ffma2_rn(m2, W[2], __fmul2_rn(m1, W[1])));
  const float2 pt = __ffma2_rn(half, b2, W[4]);
  const float2 en = __ffma2_rn(W[4], make_float2(igm1, igm1), __fmul2_rn(half, __fadd2_rn(rv2, b2)));
  const float2 vB = __ffma2_rn(W[3], W[7], __ffma2_rn(W[2], W[6], __fmul2_rn(W[1], W[5])));
  float2 G[NVAR];
  G[0] = __fmul2_rn(W[0], w);
  G[1] = __ffma2_rn(m1, w, __fmul2_rn(nBn, W[5]));
  G[2] = __ffma2_rn(m2, w, __fmul2_rn(nBn, W[6]));
  G[3] = __ffma2_rn(m3, w, __fmul2_rn(nBn, W[7]));
  G[1 + D] = __fadd2_rn(G[1 + D], pt);
  G[4] = __ffma2_rn(en, w, __ffma2_rn(pt, vn, __fmul2_rn(nBn, vB)));
#pragma unroll
  for (int k = 0; k < 3; k++)
    if (k != D) G[5 + k] = __ffma2_rn(W[5 + k], w, __fmul2_rn(nBn, W[1 + k]));
#pragma unroll
  for (int v = 0; v < NVAR; v++) F2[v] = v == 5 + D ? 0.f : G[v].x + G[v].y;
}

// TVDLF face flux (twice, see tvdlf_states) from the four cells a, b | c, e
// around the face (primitive variables).  FP32: the difference c - b serves
// both half slopes, then tvdlf_pair.
template <typename real, int D>
__device__ __forceinline__ void tvdlf_face(const real *a, const real *b, const real *c, const real *e,
                                           real gamma, real igm1, real *F2) {
  if constexpr (sizeof(real) == 4) {
    float hb[NVAR], hc[NVAR];
#pragma unroll
    for (int v = 0; v < NVAR; v += 2) {
      const float2 B = make_float2(b[v], b[v + 1]), C = make_float2(c[v], c[v + 1]);
      const float2 d1 = __fadd2_rn(B, make_float2(-a[v], -a[v + 1]));
      const float2 d2 = __fadd2_rn(C, make_float2(-B.x, -B.y));
      const float2 d3 = __fadd2_rn(make_float2(e[v], e[v + 1]), make_float2(-C.x, -C.y));
      const float2 s1 = __fadd2_rn(d1, d2), s2 = __fadd2_rn(d2, d3);
      hb[v] = half_mc_signed(d1.x, d2.x, s1.x);
      hb[v + 1] = half_mc_signed(d1.y, d2.y, s1.y);
      hc[v] = half_mc_signed(d2.x, d3.x, s2.x);
      hc[v + 1] = half_mc_signed(d2.y, d3.y, s2.y);
    }
    tvdlf_pair<D>(b, c, hb, hc, gamma, igm1, F2);
    return;
  }
  real sb[NVAR], sc[NVAR], WL[NVAR], WR[NVAR];
  mc_half_slopes8<real>(a, b, c, sb);
  mc_half_slopes8<real>(b, c, e, sc);
  axpy8<real>(b, real(1), sb, WL);
  axpy8<real>(c, real(-1), sc, WR);
  tvdlf_states<real, D>(WL, WR, b, c, gamma, igm1, F2);
}

// asynchronous global -> shared copies of 8 or 16 bytes (cp.async)
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
  else if (BYTES == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
// wait until at most N of this thread's most recent copy groups are pending
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// floors on a freshly updated cell; returns the number of floor hits
template <typename real>
__device__ __forceinline__ int apply_floors(real *u, real gamma, real pfloor, real rfloor, Isl isl) {
  int hits = 0;
  if (u[0] < rfloor) {
    u[0] = rfloor;
    hits++;
  }
  // the plain-precision pressure is within ~1e-6 |e| of the exact one: only a
  // cell that might be below the floor pays for the precise recovery
  const real pq = pressure_for_speed<real>(u, gamma);
  const real margin = sizeof(real) == 4 ? real(1e-6) : real(0);
  if (pq > pfloor + margin * RT<real>::abs_(u[4])) return hits;
  real p = pressure_of<real>(u, gamma, isl);
  if (p < pfloor) {
    real ke = real(0.5) * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0];
    real me = real(0.5) * (u[5] * u[5] + u[6] * u[6] + u[7] * u[7]);
    u[4] = pfloor / (gamma - real(1)) + ke + me;
    hits++;
  }
  return hits;
}

// atomic max of a non-negative double through its bit pattern
__device__ __forceinline__ void atomic_max_pos(unsigned long long *addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}
