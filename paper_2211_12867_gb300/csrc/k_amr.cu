// State transfer, refinement estimator, regrid data movement, probe and
// conservation sums.
//
// Refinement estimator (arXiv 2211.12867, Sect. 3: refinement is triggered by
// criteria on the local solution; blocks coarsen again when the criterion
// fails): Loehner's second-derivative estimator of density and pressure in
// its diagonal index-space form, gated by a radial speed above the relaxed
// background.  It is evaluated in FP64 with explicitly rounded operations in a
// fixed order (no contraction), so the block flags agree bit for bit with any
// IEEE FP64 evaluation of the same formula on the same stored state.
#include "mhd_device.cuh"

namespace {

template <typename real>
__device__ __forceinline__ size_t cidx(const KParams &kp, int slot, int v, int p0, int p1, int p2) {
  return ((((size_t)slot * kp.nvs + v) * kp.P[0] + p0) * kp.P[1] + p1) * kp.P[2] + p2;
}

template <typename real>
__global__ void k_pack(const KParams kp, const real *U, int slot0, int nslots, double *out) {
  const size_t n = (size_t)nslots * NVAR * kp.icells;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % kp.icells);
    const int v = (int)((e / kp.icells) % NVAR);
    const int s = (int)(e / ((size_t)kp.icells * NVAR));
    const int k = c % kp.nb[2], j = (c / kp.nb[2]) % kp.nb[1], i = c / (kp.nb[2] * kp.nb[1]);
    out[e] = (double)U[cidx<real>(kp, slot0 + s, v, i + NGH, j + NGH, k + NGH)];
  }
}

template <typename real>
__global__ void k_unpack(const KParams kp, real *U, int slot0, int nslots, const double *in, int is_prim) {
  const size_t n = (size_t)nslots * kp.icells;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % kp.icells);
    const int s = (int)(e / kp.icells);
    const int k = c % kp.nb[2], j = (c / kp.nb[2]) % kp.nb[1], i = c / (kp.nb[2] * kp.nb[1]);
    double x[NVAR], u[NVAR];
#pragma unroll
    for (int v = 0; v < NVAR; v++) x[v] = in[((size_t)s * NVAR + v) * kp.icells + c];
    if (is_prim)
      prim2cons<double>(x, u, 1.0 / (kp.gamma - 1.0));
    else
#pragma unroll
      for (int v = 0; v < NVAR; v++) u[v] = x[v];
#pragma unroll
    for (int v = 0; v < NVAR; v++) U[cidx<real>(kp, slot0 + s, v, i + NGH, j + NGH, k + NGH)] = (real)u[v];
  }
}

// ---- estimator ----
__device__ __forceinline__ double est_pressure(const double *u, double gamma) {
  double msq = __dadd_rn(__dadd_rn(__dmul_rn(u[1], u[1]), __dmul_rn(u[2], u[2])), __dmul_rn(u[3], u[3]));
  double bsq = __dadd_rn(__dadd_rn(__dmul_rn(u[5], u[5]), __dmul_rn(u[6], u[6])), __dmul_rn(u[7], u[7]));
  double ke = __ddiv_rn(__dmul_rn(0.5, msq), u[0]);
  double me = __dmul_rn(0.5, bsq);
  return __dmul_rn(__dsub_rn(gamma, 1.0), __dsub_rn(__dsub_rn(u[4], ke), me));
}

__device__ __forceinline__ double loehner(const double *um, double u0, const double *up, double eps) {
  double num = 0.0, den = 0.0;
  for (int d = 0; d < 3; d++) {
    double t1 = __dsub_rn(up[d], u0);
    double t2 = __dsub_rn(u0, um[d]);
    double d2 = __dsub_rn(t1, t2);
    double w = __dadd_rn(__dadd_rn(fabs(up[d]), __dmul_rn(2.0, fabs(u0))), fabs(um[d]));
    double s = __dadd_rn(__dadd_rn(fabs(t1), fabs(t2)), __dmul_rn(eps, w));
    num = __dadd_rn(num, __dmul_rn(d2, d2));
    den = __dadd_rn(den, __dmul_rn(s, s));
  }
  if (den <= 0.0) return 0.0;
  return __dsqrt_rn(__ddiv_rn(num, den));
}

template <typename real>
__global__ void k_estimator(const KParams kp, const real *U, int slot0, double e_ref, double e_crs, double eps,
                            double dv, signed char *flags) {
  const int slot = slot0 + blockIdx.x;
  const DevBlock B = kp.blk[slot];
  const int L = B.level, sh = L - 1;
  const DevCme C = kp.cme[B.member];
  const bool has_bg = C.pad != 0;
  const size_t nbc = (size_t)kp.n_base_cells[0] * kp.n_base_cells[1] * kp.n_base_cells[2];
  const double *vbg = kp.vbg + (size_t)B.member * nbc;
  int refine = 0, keep = 0;
  // one refining cell settles the leaf's flag: the threads stop once any of
  // them has found one (s_refine), which leaves the flag unchanged
  __shared__ volatile int s_refine;
  if (threadIdx.x == 0) s_refine = 0;
  __syncthreads();
  // without a recorded background the gate is closed everywhere: no cell
  // counts and the block is flagged for coarsening
  for (int c = has_bg ? threadIdx.x : kp.icells; c < kp.icells && !s_refine; c += blockDim.x) {
    const int k = c % kp.nb[2], j = (c / kp.nb[2]) % kp.nb[1], i = c / (kp.nb[2] * kp.nb[1]);
    const int p0 = i + NGH, p1 = j + NGH, p2 = k + NGH;
    // the speed gate first: E only matters where it is open, and not at all
    // once this thread has found a refining cell (the flags are unchanged)
    const double r0 = (double)U[cidx<real>(kp, slot, 0, p0, p1, p2)];
    const double m0 = (double)U[cidx<real>(kp, slot, 1, p0, p1, p2)];
    {
      const int I = B.ix[0] * kp.nb[0] + i, J = B.ix[1] * kp.nb[1] + j, K = B.ix[2] * kp.nb[2] + k;
      const double vb = vbg[((size_t)(I >> sh) * kp.n_base_cells[1] + (J >> sh)) * kp.n_base_cells[2] + (K >> sh)];
      const double vr = __ddiv_rn(m0, r0);
      if (!(vr > __dadd_rn(vb, dv)) || refine) continue;
    }
    double u0[NVAR];
#pragma unroll
    for (int v = 0; v < NVAR; v++) u0[v] = (double)U[cidx<real>(kp, slot, v, p0, p1, p2)];
    double rm[3], rp[3], pm[3], pp[3];
    for (int d = 0; d < 3; d++) {
      int m[3] = {p0, p1, p2}, p[3] = {p0, p1, p2};
      m[d]--;
      p[d]++;
      double um[NVAR], up[NVAR];
#pragma unroll
      for (int v = 0; v < NVAR; v++) {
        um[v] = (double)U[cidx<real>(kp, slot, v, m[0], m[1], m[2])];
        up[v] = (double)U[cidx<real>(kp, slot, v, p[0], p[1], p[2])];
      }
      rm[d] = um[0];
      rp[d] = up[0];
      pm[d] = est_pressure(um, kp.gamma);
      pp[d] = est_pressure(up, kp.gamma);
    }
    const double er = loehner(rm, u0[0], rp, eps);
    const double ep = loehner(pm, est_pressure(u0, kp.gamma), pp, eps);
    const double E = er > ep ? er : ep;
    if (E > e_ref) {
      refine = 1;
      s_refine = 1;
    }
    if (E > e_crs) keep = 1;
  }
  refine = __syncthreads_or(refine);
  keep = __syncthreads_or(keep);
  if (threadIdx.x == 0) flags[blockIdx.x] = refine ? 1 : (keep ? 0 : -1);
}

// ---- shock criterion (Sect. 3.2) ----
// The paper refines where the velocity divergence is negative, inside
// windows around the Sun-Earth line and the CME's hemisphere, and coarsens
// once the criterion fails.  The divergence is the central difference at cell
// centres in spherical form; everything is FP64 with explicitly rounded
// operations in a fixed order, so the flags agree bit for bit with any IEEE
// FP64 evaluation of the same expression on the same stored state and
// geometry.
__device__ __forceinline__ double wrap_pi(double a) {
  const double pi = 3.14159265358979323846, tp = 2.0 * pi;
  return __dsub_rn(a, __dmul_rn(tp, floor(__ddiv_rn(__dadd_rn(a, pi), tp))));
}

template <typename real>
__device__ __forceinline__ double vel(const KParams &kp, const real *U, int slot, int v, int p0, int p1, int p2) {
  return __ddiv_rn((double)U[cidx<real>(kp, slot, v, p0, p1, p2)], (double)U[cidx<real>(kp, slot, 0, p0, p1, p2)]);
}

// which: 0 shock (div v < -div_thr), 1 tracer (X > x_thr), 2 combined
// (either), all inside the windows.  The tracer fraction X = (rho X) / rho is
// one correctly rounded division of the stored values.
template <typename real>
__global__ void k_shock_estimator(const KParams kp, const real *U, int slot0, double div_thr, double w_le,
                                  double w_ce, double w_lc, double x_thr, int which, signed char *flags) {
  const int slot = slot0 + blockIdx.x;
  const DevBlock B = kp.blk[slot];
  const LevelGeo<double> &G = kp.geo->d[B.level];
  const DevEarth E = kp.earth[B.member];
  const DevCme C = kp.cme[B.member];
  const double t = kp.t[B.member];
  const double lon_e = __dsub_rn(E.lon0, __dmul_rn(E.rate, __dsub_rn(t, E.t0)));
  const bool sph = kp.geometry == 0;
  int refine = 0;
  // one refining cell settles the leaf's flag (see k_estimator)
  __shared__ volatile int s_refine;
  if (threadIdx.x == 0) s_refine = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < kp.icells && !refine && !s_refine; c += blockDim.x) {
    const int k = c % kp.nb[2], j = (c / kp.nb[2]) % kp.nb[1], i = c / (kp.nb[2] * kp.nb[1]);
    const int I = B.ix[0] * kp.nb[0] + i + NGH, J = B.ix[1] * kp.nb[1] + j + NGH, K = B.ix[2] * kp.nb[2] + k + NGH;
    const double th = G.tc[J], ph = G.pc[K];
    bool in = true;
    if (w_le > 0.0) in = in && E.set && fabs(wrap_pi(__dsub_rn(ph, lon_e))) <= w_le;
    if (w_ce > 0.0) in = in && E.set && fabs(__dsub_rn(th, E.colat)) <= w_ce;
    if (w_lc > 0.0) in = in && C.active && fabs(wrap_pi(__dsub_rn(ph, C.lon))) <= w_lc;
    if (!in) continue;
    const int p0 = i + NGH, p1 = j + NGH, p2 = k + NGH;
    if (which >= 1 && vel(kp, U, slot, TRV, p0, p1, p2) > x_thr) {
      refine = 1;
      s_refine = 1;
      continue;
    }
    if (which == 1) continue;
    const double vrm = vel(kp, U, slot, 1, p0 - 1, p1, p2), vrp = vel(kp, U, slot, 1, p0 + 1, p1, p2);
    const double vtm = vel(kp, U, slot, 2, p0, p1 - 1, p2), vtp = vel(kp, U, slot, 2, p0, p1 + 1, p2);
    const double vpm = vel(kp, U, slot, 3, p0, p1, p2 - 1), vpp = vel(kp, U, slot, 3, p0, p1, p2 + 1);
    const double rm = G.rc[I - 1], r0 = G.rc[I], rp = G.rc[I + 1];
    const double tm = G.tc[J - 1], tp = G.tc[J + 1], qm = G.pc[K - 1], qp = G.pc[K + 1];
    double a, b, e;
    if (sph) {
      const double sm = G.sintc[J - 1], s0 = G.sintc[J], sp = G.sintc[J + 1];
      a = __ddiv_rn(__dsub_rn(__dmul_rn(__dmul_rn(rp, rp), vrp), __dmul_rn(__dmul_rn(rm, rm), vrm)),
                    __dmul_rn(__dmul_rn(r0, r0), __dsub_rn(rp, rm)));
      const double rs = __dmul_rn(r0, s0);
      b = __ddiv_rn(__dsub_rn(__dmul_rn(sp, vtp), __dmul_rn(sm, vtm)), __dmul_rn(rs, __dsub_rn(tp, tm)));
      e = __ddiv_rn(__dsub_rn(vpp, vpm), __dmul_rn(rs, __dsub_rn(qp, qm)));
    } else {
      a = __ddiv_rn(__dsub_rn(vrp, vrm), __dsub_rn(rp, rm));
      b = __ddiv_rn(__dsub_rn(vtp, vtm), __dsub_rn(tp, tm));
      e = __ddiv_rn(__dsub_rn(vpp, vpm), __dsub_rn(qp, qm));
    }
    const double div = __dadd_rn(__dadd_rn(a, b), e);
    if (div < -div_thr) {
      refine = 1;
      s_refine = 1;
    }
  }
  refine = __syncthreads_or(refine);
  if (threadIdx.x == 0) flags[blockIdx.x] = refine ? 1 : -1;
}

// ---- regrid data movement ----
template <typename real>
__device__ void prolong_child(const KParams &kp, const real *U, int cs, const int *Ic, int ch, real *out) {
  const DevBlock C = kp.blk[cs];
  const int Lc = C.level;
  const int nv = kp.nvs;   // the MHD variables and, when stored, the CME tracer
  int pc[3];
#pragma unroll
  for (int d = 0; d < 3; d++) pc[d] = Ic[d] - C.ix[d] * kp.nb[d] + NGH;
  real up[NVAR + 1], s[3][NVAR + 1];
#pragma unroll
  for (int v = 0; v < NVAR + 1; v++) {
    if (v >= nv) break;
    up[v] = U[cidx<real>(kp, cs, v, pc[0], pc[1], pc[2])];
    s[0][v] = mc_slope<real>(U[cidx<real>(kp, cs, v, pc[0] - 1, pc[1], pc[2])], up[v],
                             U[cidx<real>(kp, cs, v, pc[0] + 1, pc[1], pc[2])]);
    s[1][v] = mc_slope<real>(U[cidx<real>(kp, cs, v, pc[0], pc[1] - 1, pc[2])], up[v],
                             U[cidx<real>(kp, cs, v, pc[0], pc[1] + 1, pc[2])]);
    s[2][v] = mc_slope<real>(U[cidx<real>(kp, cs, v, pc[0], pc[1], pc[2] - 1)], up[v],
                             U[cidx<real>(kp, cs, v, pc[0], pc[1], pc[2] + 1)]);
  }
  const real *d0 = GeoSel<real>::dlt(kp.geo, Lc, 0), *d1 = GeoSel<real>::dlt(kp.geo, Lc, 1),
             *d2 = GeoSel<real>::dlt(kp.geo, Lc, 2);
  const real gamma = (real)kp.gamma;
  bool ok = true;
  for (int c = 0; c < 8; c++) {
    const real a = d0[2 * Ic[0] + ((c >> 2) & 1)], b = d1[2 * Ic[1] + ((c >> 1) & 1)], e = d2[2 * Ic[2] + (c & 1)];
    real u[NVAR + 1];
#pragma unroll
    for (int v = 0; v < NVAR + 1; v++)
      if (v < nv) u[v] = ((up[v] + s[0][v] * a) + s[1][v] * b) + s[2][v] * e;
    if (!(u[0] > real(0)) || !(pressure_of<real>(u, gamma, Isl{(float)kp.isl_pe, (float)kp.isl_beta}) > real(0))) ok = false;
    if (c == ch)
#pragma unroll
      for (int v = 0; v < NVAR + 1; v++)
        if (v < nv) out[v] = u[v];
  }
  if (!ok)
#pragma unroll
    for (int v = 0; v < NVAR + 1; v++)
      if (v < nv) out[v] = up[v];
}

template <typename real>
__global__ void k_regrid_move(const KParams kpo, const real *Uold, real *Unew, const DevBlock *nblk,
                              const MoveOp *ops) {
  const MoveOp op = ops[blockIdx.x];
  const int c = blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= kpo.icells) return;
  const int k = c % kpo.nb[2], j = (c / kpo.nb[2]) % kpo.nb[1], i = c / (kpo.nb[2] * kpo.nb[1]);
  const DevBlock N = nblk[op.dst];
  real val[NVAR + 1];
  const int nv = kpo.nvs;
  if (op.kind == 0) {
#pragma unroll
    for (int v = 0; v < NVAR + 1; v++)
      if (v < nv) val[v] = Uold[cidx<real>(kpo, op.src[0], v, i + NGH, j + NGH, k + NGH)];
  } else if (op.kind == 1) {
    const int F[3] = {N.ix[0] * kpo.nb[0] + i, N.ix[1] * kpo.nb[1] + j, N.ix[2] * kpo.nb[2] + k};
    const int Ic[3] = {F[0] >> 1, F[1] >> 1, F[2] >> 1};
    prolong_child<real>(kpo, Uold, op.src[0], Ic, ((F[0] & 1) << 2) | ((F[1] & 1) << 1) | (F[2] & 1), val);
  } else {
    const LevelGeo<real> &FG = GeoSel<real>::get(kpo.geo, N.level + 1);
    const int G[3] = {N.ix[0] * kpo.nb[0] + i, N.ix[1] * kpo.nb[1] + j, N.ix[2] * kpo.nb[2] + k};
    real sum[NVAR + 1];
#pragma unroll
    for (int v = 0; v < NVAR + 1; v++) sum[v] = real(0);
    real vs = real(0);
    for (int ch = 0; ch < 8; ch++) {
      const int f[3] = {2 * G[0] + ((ch >> 2) & 1), 2 * G[1] + ((ch >> 1) & 1), 2 * G[2] + (ch & 1)};
      int cb[3];
#pragma unroll
      for (int d = 0; d < 3; d++) cb[d] = f[d] / kpo.nb[d] - 2 * N.ix[d];
      const int os = op.src[(cb[0] << 2) | (cb[1] << 1) | cb[2]];
      const int q0 = f[0] - (2 * N.ix[0] + cb[0]) * kpo.nb[0] + NGH;
      const int q1 = f[1] - (2 * N.ix[1] + cb[1]) * kpo.nb[1] + NGH;
      const int q2 = f[2] - (2 * N.ix[2] + cb[2]) * kpo.nb[2] + NGH;
      const real V = FG.dr3[f[0] + NGH] * FG.dcos[f[1] + NGH] * FG.dphi;
#pragma unroll
      for (int v = 0; v < NVAR + 1; v++)
        if (v < nv) sum[v] += V * Uold[cidx<real>(kpo, os, v, q0, q1, q2)];
      vs += V;
    }
#pragma unroll
    for (int v = 0; v < NVAR + 1; v++) val[v] = sum[v] / vs;
  }
#pragma unroll
  for (int v = 0; v < NVAR + 1; v++)
    if (v < nv) Unew[cidx<real>(kpo, op.dst, v, i + NGH, j + NGH, k + NGH)] = val[v];
}

// ---- probe ----
__device__ int find_face(const double *f, int N, double x) {
  int lo = 0, hi = N;
  while (hi - lo > 1) {
    int m = (lo + hi) / 2;
    if (f[m + NGH] <= x) lo = m;
    else hi = m;
  }
  return lo;
}

template <typename real>
__global__ void k_probe(const KParams kp, const real *U, int member, int maxL, int npts, const double *pts,
                        double *out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= npts) return;
  double p[3] = {pts[3 * n], pts[3 * n + 1], pts[3 * n + 2]};
  if (kp.bc_lo[2] == 0) {
    const LevelGeo<double> &G1 = kp.geo->d[1];
    const double lo = G1.pf[NGH], hi = G1.pf[NGH + G1.n[2]], span = hi - lo;
    p[2] = lo + fmod(fmod(p[2] - lo, span) + span, span);
  }
  const LevelGeo<double> &GM = kp.geo->d[maxL];
  const double *faces[3] = {GM.rf, GM.tf, GM.pf};
  int I[3];
  bool bad = false;
  for (int d = 0; d < 3; d++) {
    const int N = GM.n[d];
    if (p[d] < faces[d][NGH] || p[d] >= faces[d][NGH + N]) bad = true;
    I[d] = find_face(faces[d], N, p[d]);
  }
  if (bad) {
    for (int v = 0; v < NVAR; v++) out[n * NVAR + v] = nan("");
    return;
  }
  int L = maxL, slot = -1;
  while (L >= 1) {
    const int o = (int)0;
    (void)o;
    const long long off = kp.lmap_off[member * (MAXLEV + 1) + L];
    const int s = L - 1;
    const int b0 = I[0] / kp.nb[0], b1 = I[1] / kp.nb[1], b2 = I[2] / kp.nb[2];
    const int n1 = kp.nbase[1] << s, n2 = kp.nbase[2] << s;
    const int v = kp.lmap[off + ((long long)b0 * n1 + b1) * n2 + b2];
    if (v >= 0) {
      slot = v;
      break;
    }
    for (int d = 0; d < 3; d++) I[d] >>= 1;
    L--;
  }
  if (slot < 0) {
    for (int v = 0; v < NVAR; v++) out[n * NVAR + v] = nan("");
    return;
  }
  const DevBlock B = kp.blk[slot];
  const LevelGeo<double> &G = kp.geo->d[B.level];
  const double *cen[3] = {G.rc, G.tc, G.pc};
  int q[3];
  double w[3];
  for (int d = 0; d < 3; d++) {
    const int P = kp.P[d], g0 = B.ix[d] * kp.nb[d] - NGH;
    int kk = 0;
    for (int s = 0; s < P - 1; s++)
      if (cen[d][g0 + s + NGH] <= p[d]) kk = s;
    if (kk > P - 2) kk = P - 2;
    const double c0 = cen[d][g0 + kk + NGH], c1 = cen[d][g0 + kk + 1 + NGH];
    q[d] = kk;
    w[d] = (p[d] - c0) / (c1 - c0);
  }
  double acc[NVAR];
  for (int v = 0; v < NVAR; v++) acc[v] = 0.0;
  for (int a = 0; a < 2; a++)
    for (int b = 0; b < 2; b++)
      for (int c = 0; c < 2; c++) {
        double u[NVAR];
        for (int v = 0; v < NVAR; v++) u[v] = (double)U[cidx<real>(kp, slot, v, q[0] + a, q[1] + b, q[2] + c)];
        const double ir = 1.0 / u[0];
        double W[NVAR];
        W[0] = u[0];
        W[1] = u[1] * ir;
        W[2] = u[2] * ir;
        W[3] = u[3] * ir;
        W[4] = (kp.gamma - 1.0) * (u[4] - 0.5 * u[0] * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]) -
                                   0.5 * (u[5] * u[5] + u[6] * u[6] + u[7] * u[7]));
        W[5] = u[5];
        W[6] = u[6];
        W[7] = u[7];
        const double wt = (a ? w[0] : 1.0 - w[0]) * (b ? w[1] : 1.0 - w[1]) * (c ? w[2] : 1.0 - w[2]);
        for (int v = 0; v < NVAR; v++) acc[v] += wt * W[v];
      }
  for (int v = 0; v < NVAR; v++) out[n * NVAR + v] = acc[v];
}

// ---- conservation sums: per-block partials in a fixed order ----
template <typename real>
__global__ void k_sums(const KParams kp, const real *U, int slot0, double *partial) {
  __shared__ double sh[NVAR][256];
  const int slot = slot0 + blockIdx.x;
  const DevBlock B = kp.blk[slot];
  const LevelGeo<real> &G = GeoSel<real>::get(kp.geo, B.level);
  const LevelGeo<double> &GD = kp.geo->d[B.level];
  double acc[NVAR];
  for (int v = 0; v < NVAR; v++) acc[v] = 0.0;
  (void)G;
  for (int c = threadIdx.x; c < kp.icells; c += blockDim.x) {
    const int k = c % kp.nb[2], j = (c / kp.nb[2]) % kp.nb[1], i = c / (kp.nb[2] * kp.nb[1]);
    const int I = B.ix[0] * kp.nb[0] + i + NGH, J = B.ix[1] * kp.nb[1] + j + NGH;
    const double V = GD.dr3[I] * GD.dcos[J] * GD.dphi;
    for (int v = 0; v < NVAR; v++) acc[v] += V * (double)U[cidx<real>(kp, slot, v, i + NGH, j + NGH, k + NGH)];
  }
  for (int v = 0; v < NVAR; v++) sh[v][threadIdx.x] = acc[v];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int v = 0; v < NVAR; v++) sh[v][threadIdx.x] += sh[v][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < NVAR) partial[(size_t)blockIdx.x * NVAR + threadIdx.x] = sh[threadIdx.x][0];
}

template <typename real>
__global__ void k_vbg(const KParams kp, const real *U, int member, int slot0, double *vbg) {
  const int slot = slot0 + blockIdx.x;
  const DevBlock B = kp.blk[slot];
  for (int c = blockIdx.y * blockDim.x + threadIdx.x; c < kp.icells; c += gridDim.y * blockDim.x) {
    const int k = c % kp.nb[2], j = (c / kp.nb[2]) % kp.nb[1], i = c / (kp.nb[2] * kp.nb[1]);
    const int I = B.ix[0] * kp.nb[0] + i, J = B.ix[1] * kp.nb[1] + j, K = B.ix[2] * kp.nb[2] + k;
    const double m = (double)U[cidx<real>(kp, slot, 1, i + NGH, j + NGH, k + NGH)];
    const double r = (double)U[cidx<real>(kp, slot, 0, i + NGH, j + NGH, k + NGH)];
    vbg[((size_t)I * kp.n_base_cells[1] + J) * kp.n_base_cells[2] + K] = m / r;
  }
  (void)member;
}

}  // namespace

void pack_state_launch(const KParams &kp, const void *U, int precision, int slot0, int nslots, double *out,
                       cudaStream_t s) {
  if (nslots <= 0) return;
  if (precision)
    k_pack<float><<<1024, 256, 0, s>>>(kp, (const float *)U, slot0, nslots, out);
  else
    k_pack<double><<<1024, 256, 0, s>>>(kp, (const double *)U, slot0, nslots, out);
}

void unpack_state_launch(const KParams &kp, void *U, int precision, int slot0, int nslots, const double *in,
                         int is_prim, cudaStream_t s) {
  if (nslots <= 0) return;
  if (precision)
    k_unpack<float><<<1024, 256, 0, s>>>(kp, (float *)U, slot0, nslots, in, is_prim);
  else
    k_unpack<double><<<1024, 256, 0, s>>>(kp, (double *)U, slot0, nslots, in, is_prim);
}

void estimator_launch(const KParams &kp, const void *U, int precision, int slot0, int nslots, double e_ref,
                      double e_crs, double eps, double dv, signed char *flags, cudaStream_t s) {
  if (nslots <= 0) return;
  if (precision)
    k_estimator<float><<<nslots, 256, 0, s>>>(kp, (const float *)U, slot0, e_ref, e_crs, eps, dv, flags);
  else
    k_estimator<double><<<nslots, 256, 0, s>>>(kp, (const double *)U, slot0, e_ref, e_crs, eps, dv, flags);
}

void shock_estimator_launch(const KParams &kp, const void *U, int precision, int slot0, int nslots,
                            const double *crit, signed char *flags, cudaStream_t s) {
  if (nslots <= 0) return;
  const int which = (int)crit[5];
  if (precision)
    k_shock_estimator<float><<<nslots, 256, 0, s>>>(kp, (const float *)U, slot0, crit[0], crit[1], crit[2], crit[3],
                                                     crit[4], which, flags);
  else
    k_shock_estimator<double><<<nslots, 256, 0, s>>>(kp, (const double *)U, slot0, crit[0], crit[1], crit[2],
                                                      crit[3], crit[4], which, flags);
}

void regrid_move_launch2(const KParams &kp_old, const void *Uold, void *Unew, const DevBlock *nblk, int precision,
                         const MoveOp *ops, int nops, cudaStream_t s) {
  if (nops <= 0) return;
  dim3 grid(nops, (kp_old.icells + 255) / 256);
  if (precision)
    k_regrid_move<float><<<grid, 256, 0, s>>>(kp_old, (const float *)Uold, (float *)Unew, nblk, ops);
  else
    k_regrid_move<double><<<grid, 256, 0, s>>>(kp_old, (const double *)Uold, (double *)Unew, nblk, ops);
}

void probe_launch2(const KParams &kp, const void *U, int precision, int member, int maxL, int npts, const double *pts,
                   double *out, cudaStream_t s) {
  if (npts <= 0) return;
  if (precision)
    k_probe<float><<<(npts + 127) / 128, 128, 0, s>>>(kp, (const float *)U, member, maxL, npts, pts, out);
  else
    k_probe<double><<<(npts + 127) / 128, 128, 0, s>>>(kp, (const double *)U, member, maxL, npts, pts, out);
}

void sums_launch(const KParams &kp, const void *U, int precision, int slot0, int nslots, double *partial,
                 cudaStream_t s) {
  if (nslots <= 0) return;
  if (precision)
    k_sums<float><<<nslots, 256, 0, s>>>(kp, (const float *)U, slot0, partial);
  else
    k_sums<double><<<nslots, 256, 0, s>>>(kp, (const double *)U, slot0, partial);
}

void vbg_launch(const KParams &kp, const void *U, int precision, int member, int slot0, int nslots, double *vbg,
                cudaStream_t s) {
  if (nslots <= 0) return;
  if (precision)
    k_vbg<float><<<dim3(nslots, (kp.icells + 4095) / 4096), 256, 0, s>>>(kp, (const float *)U, member, slot0, vbg);
  else
    k_vbg<double><<<dim3(nslots, (kp.icells + 4095) / 4096), 256, 0, s>>>(kp, (const double *)U, member, slot0, vbg);
}
