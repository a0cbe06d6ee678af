/*
 * Oracle, pointwise physics.  TEST INFRASTRUCTURE ONLY (see or_internal.h).
 *
 * Ideal MHD in normalised units (Sect. 2.1: ideal MHD solved in the frame
 * co-rotating with the Sun), TVDLF numerical flux with the Woodward
 * (monotonised-central) limiter (Sect. 2.1), the cone-CME geometry of
 * Eqs. 1-4 and the Loehner second-derivative refinement estimator.
 * Every routine is the plain definition, in FP64, in natural order.
 */
#include <math.h>
#include "or_internal.h"

/* W -> U: e = p/(gamma-1) + rho v^2/2 + B^2/2 (B carries sqrt(mu0)). */
void or_prim2cons(const double *W, double *U, double gamma) {
  double rho = W[RHO];
  double v2 = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
  double b2 = W[5] * W[5] + W[6] * W[6] + W[7] * W[7];
  U[RHO] = rho;
  U[MR] = rho * W[1];
  U[MT] = rho * W[2];
  U[MP] = rho * W[3];
  U[EN] = W[EN] / (gamma - 1.0) + 0.5 * rho * v2 + 0.5 * b2;
  U[BR] = W[5];
  U[BT] = W[6];
  U[BP] = W[7];
}

/* U -> W: p = (gamma-1)(e - m^2/(2 rho) - B^2/2). */
void or_cons2prim(const double *U, double *W, double gamma) {
  double rho = U[RHO];
  double vr = U[MR] / rho, vt = U[MT] / rho, vp = U[MP] / rho;
  double kin = 0.5 * rho * (vr * vr + vt * vt + vp * vp);
  double mag = 0.5 * (U[BR] * U[BR] + U[BT] * U[BT] + U[BP] * U[BP]);
  W[RHO] = rho;
  W[1] = vr;
  W[2] = vt;
  W[3] = vp;
  W[EN] = (gamma - 1.0) * (U[EN] - kin - mag);
  W[5] = U[BR];
  W[6] = U[BT];
  W[7] = U[BP];
}

/* Fast magnetosonic speed along direction d:
 * c_f^2 = (a^2 + b^2 + sqrt((a^2+b^2)^2 - 4 a^2 b_n^2)) / 2. */
double or_fast_speed(const double *W, int d, double gamma) {
  double rho = W[RHO];
  double a2 = gamma * W[EN] / rho;
  double b2 = (W[5] * W[5] + W[6] * W[6] + W[7] * W[7]) / rho;
  double bn2 = W[5 + d] * W[5 + d] / rho;
  double s = a2 + b2;
  double disc = s * s - 4.0 * a2 * bn2;
  if (disc < 0.0) disc = 0.0;
  return sqrt(0.5 * (s + sqrt(disc)));
}

/* Woodward (monotonised-central) limited slope in index space. */
double or_mc_slope(double um, double u0, double up) {
  double dm = u0 - um, dp = up - u0;
  if (dm * dp <= 0.0) return 0.0;
  double dc = 0.5 * (dm + dp);
  double lim = fmin(2.0 * fabs(dm), 2.0 * fabs(dp));
  lim = fmin(lim, fabs(dc));
  return dc > 0.0 ? lim : -lim;
}

/* Physical flux along d of the ideal-MHD conservation law, orthonormal
 * components.  The d-component of the induction flux is zero by definition. */
void or_phys_flux(const double *W, const double *U, int d, double *F) {
  double vn = W[1 + d], Bn = W[5 + d];
  double b2 = W[5] * W[5] + W[6] * W[6] + W[7] * W[7];
  double pt = W[EN] + 0.5 * b2;
  double vB = W[1] * W[5] + W[2] * W[6] + W[3] * W[7];
  F[RHO] = U[RHO] * vn;
  for (int c = 0; c < 3; c++) {
    F[1 + c] = U[1 + c] * vn - W[5 + c] * Bn;
    F[5 + c] = vn * W[5 + c] - Bn * W[1 + c];
  }
  F[1 + d] += pt;
  F[5 + d] = 0.0;
  F[EN] = (U[EN] + pt) * vn - Bn * vB;
}

/* TVDLF (local Lax-Friedrichs) face flux from reconstructed face states:
 * F = (F_L + F_R)/2 - c_max (U_R - U_L)/2, c_max the larger of |v_n| + c_f on
 * either side; the normal magnetic flux is exactly zero. */
void or_tvdlf(const double *WL, const double *WR, int d, double gamma, double *F) {
  double UL[NV], UR[NV], FL[NV], FR[NV];
  or_prim2cons(WL, UL, gamma);
  or_prim2cons(WR, UR, gamma);
  or_phys_flux(WL, UL, d, FL);
  or_phys_flux(WR, UR, d, FR);
  double cl = fabs(WL[1 + d]) + or_fast_speed(WL, d, gamma);
  double cr = fabs(WR[1 + d]) + or_fast_speed(WR, d, gamma);
  double cmax = cl > cr ? cl : cr;
  for (int v = 0; v < NV; v++) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * cmax * (UR[v] - UL[v]);
  F[5 + d] = 0.0;
}

/* Opening angle of the cone CME at the inner boundary radius R, Eqs. 1-3:
 * r_half = R sin(omega/2); R_c = t v + R - r_half;
 * theta = arccos((R_c^2 + R^2 - r_half^2) / (2 R_c R)).
 * Returns -1 when the sphere no longer intersects the shell (argument > 1) or
 * the injection window is closed. */
double or_cme_opening(const or_cme *c, double R, double t) {
  if (!c->active) return -1.0;
  double tau = t - c->t_start;
  if (tau < 0.0 || tau > c->t_max) return -1.0;
  double rh = R * sin(c->half_width);
  double Rc = tau * c->v + R - rh;
  double arg = (Rc * Rc + R * R - rh * rh) / (2.0 * Rc * R);
  if (arg > 1.0) return -1.0;
  return acos(arg);
}

/* Angular distance of a boundary point from the CME axis, Eq. 4 (colatitudes). */
double or_cme_distance(const or_cme *c, double colat, double lon) {
  double a = sin(colat) * sin(c->colat) * cos(lon - c->lon) + cos(colat) * cos(c->colat);
  if (a > 1.0) a = 1.0;
  if (a < -1.0) a = -1.0;
  return acos(a);
}

/* Loehner (1987) second-derivative estimator, diagonal-only form in index
 * space.  um/up: values at the -1/+1 neighbour in each of the 3 directions,
 * u0c: centre value (u0c[0]).  The operation order is fixed (the GPU
 * estimator follows the same order so flags agree bit for bit). */
double or_loehner(const double *um, const double *u0c, const double *up, double eps) {
  double u0 = u0c[0];
  double num = 0.0, den = 0.0;
  for (int d = 0; d < 3; d++) {
    double t1 = up[d] - u0;
    double t2 = u0 - um[d];
    double d2 = t1 - t2;
    double s = fabs(t1) + fabs(t2) + eps * ((fabs(up[d]) + 2.0 * fabs(u0)) + fabs(um[d]));
    num = num + d2 * d2;
    den = den + s * s;
  }
  if (den <= 0.0) return 0.0;
  return sqrt(num / den);
}

/* exported for the pins: c = {t_start, t_max, colat, lon, half_width, v};
 * out = {theta(t), d(colat, lon)} with R the inner boundary radius. */
void or_cme_eval(const double *c, double R, double t, double colat, double lon, double *out) {
  or_cme m = {c[0], c[1], c[2], c[3], c[4], c[5], 0.0, 0.0, 1};
  out[0] = or_cme_opening(&m, R, t);
  out[1] = or_cme_distance(&m, colat, lon);
}
