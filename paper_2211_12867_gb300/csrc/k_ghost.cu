// Ghost-cell fill, reflux and time-step kernels.
//
// Two ghost layers per block (arXiv 2211.12867, Sect. 2.1).  Ghosts are
// filled level by level, coarse to fine, so that a prolongation always reads
// a coarse block whose own ghosts are complete:
//   * same-level leaf      -> copy of its interior cell
//   * coarser leaf          -> conservative prolongation: parent value plus
//                             monotonised-central slopes of the conserved
//                             variables times the offset of the child's
//                             volume-weighted centre (falls back to the parent
//                             value when a child's pressure or density would
//                             not be positive)
//   * finer leaves          -> volume-weighted restriction of the 8 children
//   * outside the domain    -> physical boundary: fixed inner boundary map
//                             with the cone CME overlay (Eqs. 1-4),
//                             zero-gradient copy, or reflection; applied per
//                             direction r, theta, phi in that order over the
//                             whole padded slab.
// Reflux: a coarse leaf face next to finer leaves takes the sum of the fine
// area-weighted fluxes of the corrector stage (exact conservation across
// levels on the stretched spherical grid).
#include "mhd_device.cuh"

namespace {

__device__ __forceinline__ int wrap_dim(const KParams &kp, int L, int d, int G, bool &inside) {
  const int N = kp.n_base_cells[d] << (L - 1);
  if (kp.bc_lo[d] == 0) {  // periodic
    inside = true;
    G %= N;
    return G < 0 ? G + N : G;
  }
  inside = G >= 0 && G < N;
  return G;
}

// slot of the level-L leaf holding cell G (>=0), -1 coarser, -2 refined
__device__ __forceinline__ int lookup(const KParams &kp, int member, int L, const int *G) {
  const long long off = kp.lmap_off[member * (MAXLEV + 1) + L];
  const int s = L - 1;
  const int b0 = G[0] / kp.nb[0], b1 = G[1] / kp.nb[1], b2 = G[2] / kp.nb[2];
  const int n1 = kp.nbase[1] << s, n2 = kp.nbase[2] << s;
  return kp.lmap[off + ((long long)b0 * n1 + b1) * n2 + b2];
}

__device__ __forceinline__ size_t cell_index(const KParams &kp, int slot, int v, int p0, int p1, int p2) {
  return ((((size_t)slot * kp.nvs + v) * kp.P[0] + p0) * kp.P[1] + p1) * kp.P[2] + p2;
}

// Index of variable 0 at padded index (p0, p1, p2) of leaf `slot` (variable
// v lies v * P0 P1 P2 further on); with `direct`, a cell of the ghost layer
// that a same-level leaf holds is located in that leaf's interior (the ghost
// copy is not filled in the step's fills).
__device__ __forceinline__ size_t locate(const KParams &kp, int slot, int p0, int p1, int p2, bool direct) {
  if (direct) {
    const int s0 = p0 < NGH ? -1 : (p0 >= NGH + kp.nb[0] ? 1 : 0);
    const int s1 = p1 < NGH ? -1 : (p1 >= NGH + kp.nb[1] ? 1 : 0);
    const int s2 = p2 < NGH ? -1 : (p2 >= NGH + kp.nb[2] ? 1 : 0);
    if (s0 | s1 | s2) {
      const int o = kp.nb27[(size_t)slot * 27 + (s0 + 1) * 9 + (s1 + 1) * 3 + (s2 + 1)];
      if (o >= 0) return cell_index(kp, o, 0, p0 - s0 * kp.nb[0], p1 - s1 * kp.nb[1], p2 - s2 * kp.nb[2]);
    }
  }
  return cell_index(kp, slot, 0, p0, p1, p2);
}

// variable v at padded index (p0, p1, p2) of leaf `slot` (see locate)
template <typename real>
__device__ __forceinline__ real fetch(const KParams &kp, const real *U, int slot, int v, int p0, int p1, int p2,
                                      bool direct) {
  return U[locate(kp, slot, p0, p1, p2, direct) + (size_t)v * kp.P[0] * kp.P[1] * kp.P[2]];
}

// Conservative prolongation of coarse cell Ic (global at level Lc, held by
// leaf slot cs) into the 2 x 2 x 2 ghost cells of leaf `slot` starting at
// padded index p: child (i, j, k) = parent + MC slopes x offsets; if any
// child's density or pressure is not positive all eight take the parent
// value.  The seven stencil cells are located once (all their loads are
// independent); a first pass checks the eight children, a second writes them.
template <typename real>
__device__ __forceinline__ void prolong_into(const KParams &kp, real *U, int cs, int Lc, const int *Ic, int slot, const int *p,
                             bool direct) {
  const DevBlock C = kp.blk[cs];
  int pc[3];
#pragma unroll
  for (int d = 0; d < 3; d++) pc[d] = Ic[d] - C.ix[d] * kp.nb[d] + NGH;
  const size_t vs = (size_t)kp.P[0] * kp.P[1] * kp.P[2];
  const size_t i0 = cell_index(kp, cs, 0, pc[0], pc[1], pc[2]);
  const size_t im0 = locate(kp, cs, pc[0] - 1, pc[1], pc[2], direct), ip0 = locate(kp, cs, pc[0] + 1, pc[1], pc[2], direct);
  const size_t im1 = locate(kp, cs, pc[0], pc[1] - 1, pc[2], direct), ip1 = locate(kp, cs, pc[0], pc[1] + 1, pc[2], direct);
  const size_t im2 = locate(kp, cs, pc[0], pc[1], pc[2] - 1, direct), ip2 = locate(kp, cs, pc[0], pc[1], pc[2] + 1, direct);
  // the MHD variables and, when stored, the CME tracer (same slopes and
  // offsets; the positivity decision is the MHD variables')
  const int nv = kp.nvs;
  real up[NVAR + 1], s[3][NVAR + 1];
#pragma unroll
  for (int v = 0; v < NVAR + 1; v++) {
    if (v < nv) {
      const size_t o = v * vs;
      up[v] = U[i0 + o];
      s[0][v] = mc_slope<real>(U[im0 + o], up[v], U[ip0 + o]);
      s[1][v] = mc_slope<real>(U[im1 + o], up[v], U[ip1 + o]);
      s[2][v] = mc_slope<real>(U[im2 + o], up[v], U[ip2 + o]);
    }
  }
  const real *d0 = GeoSel<real>::dlt(kp.geo, Lc, 0), *d1 = GeoSel<real>::dlt(kp.geo, Lc, 1),
             *d2 = GeoSel<real>::dlt(kp.geo, Lc, 2);
  const real gamma = (real)kp.gamma;
  const real a0 = d0[2 * Ic[0]], a1 = d0[2 * Ic[0] + 1], b0 = d1[2 * Ic[1]], b1 = d1[2 * Ic[1] + 1],
             e0 = d2[2 * Ic[2]], e1 = d2[2 * Ic[2] + 1];
  bool ok = true;
  for (int c = 0; c < 8; c++) {
    const real a = (c & 4) ? a1 : a0, b = (c & 2) ? b1 : b0, e = (c & 1) ? e1 : e0;
    real u[NVAR];
#pragma unroll
    for (int v = 0; v < NVAR; v++) u[v] = ((up[v] + s[0][v] * a) + s[1][v] * b) + s[2][v] * e;
    if (!(u[0] > real(0)) || !(pressure_of<real>(u, gamma, Isl{(float)kp.isl_pe, (float)kp.isl_beta}) > real(0))) ok = false;
  }
  const size_t w0 = cell_index(kp, slot, 0, p[0], p[1], p[2]);
  const int P1 = kp.P[1], P2 = kp.P[2];
  for (int c = 0; c < 8; c++) {
    const real a = (c & 4) ? a1 : a0, b = (c & 2) ? b1 : b0, e = (c & 1) ? e1 : e0;
    const size_t wc = w0 + ((size_t)((c >> 2) & 1) * P1 + ((c >> 1) & 1)) * P2 + (c & 1);
#pragma unroll
    for (int v = 0; v < NVAR + 1; v++)
      if (v < nv) U[wc + v * vs] = ok ? ((up[v] + s[0][v] * a) + s[1][v] * b) + s[2][v] * e : up[v];
  }
}

// slot of the level-L leaf at block coordinates b (>= 0), -1 coarser, -2 refined
__device__ __forceinline__ int lookup_block(const KParams &kp, int member, int L, const int *b) {
  const long long off = kp.lmap_off[member * (MAXLEV + 1) + L];
  const int n1 = kp.nbase[1] << (L - 1), n2 = kp.nbase[2] << (L - 1);
  return kp.lmap[off + ((long long)b[0] * n1 + b[1]) * n2 + b[2]];
}

// volume-weighted mean of the 8 level-(L+1) cells under the level-L cell at
// padded index q of the level-L block b (global cell G); same arithmetic and
// order as the oracle's restriction.  Block sizes are even, so the eight
// children lie in one fine block: one lookup.
template <typename real>
__device__ __forceinline__ bool restrict_in_block(const KParams &kp, const real *U, int member, int L, const int *b, const int *q,
                                  const int *G, real *out) {
  const LevelGeo<real> &F = GeoSel<real>::get(kp.geo, L + 1);
  const int nv = kp.nvs;
  int fb[3], fq[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    const int l = 2 * (q[d] - NGH);   // first child, 0 .. 2 nb - 2 within the two fine blocks
    const int hi = l >= kp.nb[d] ? 1 : 0;
    fb[d] = 2 * b[d] + hi;
    fq[d] = l - hi * kp.nb[d] + NGH;
  }
  const int fs = lookup_block(kp, member, L + 1, fb);
  if (fs < 0) return false;
  const size_t vs = (size_t)kp.P[0] * kp.P[1] * kp.P[2];
  const size_t f0 = cell_index(kp, fs, 0, fq[0], fq[1], fq[2]);
  const int P1 = kp.P[1], P2 = kp.P[2];
  real sum[NVAR + 1];
#pragma unroll
  for (int v = 0; v < NVAR + 1; v++) sum[v] = real(0);
  real vsum = real(0);
  for (int c = 0; c < 8; c++) {
    const int c0 = (c >> 2) & 1, c1 = (c >> 1) & 1, c2 = c & 1;
    const real V = F.dr3[2 * G[0] + c0 + NGH] * F.dcos[2 * G[1] + c1 + NGH] * F.dphi;
    const size_t o = f0 + ((size_t)c0 * P1 + c1) * P2 + c2;
#pragma unroll
    for (int v = 0; v < NVAR + 1; v++)
      if (v < nv) sum[v] += V * U[o + v * vs];
    vsum += V;
  }
#pragma unroll
  for (int v = 0; v < NVAR + 1; v++) out[v] = sum[v] / vsum;
  return true;
}

// Same-level copy, prolongation or restriction into the ghost cells of the
// level-L leaves.  The shell list holds the padded (p0, p1, p2) of a block's
// ghost cells packed as p0 << 20 | p1 << 10 | p2; the neighbouring block and
// the cell's index inside it follow from which side of the interior the
// ghost lies on (no divisions).
template <typename real>
__global__ void __launch_bounds__(256, sizeof(real) == 4 ? 4 : 2) k_ghost_neighbour(const KParams kp, real *U, const int *list, const int *shell, int nshell,
                                  int L) {
  const int s = blockIdx.y * blockDim.x + threadIdx.x;
  if (s >= nshell) return;
  const int slot = list[blockIdx.x];
  const int member = kp.blk[slot].member;
  const int code = shell[s];
  const int p[3] = {code >> 20, (code >> 10) & 1023, code & 1023};
  int b[3], q[3], G[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    const int nb = kp.nb[d];
    const int side = p[d] < NGH ? -1 : (p[d] >= NGH + nb ? 1 : 0);
    const int nbl = kp.nbase[d] << (L - 1);
    int bd = kp.blk[slot].ix[d] + side;
    if (bd < 0 || bd >= nbl) {
      if (kp.bc_lo[d] != 0) return;  // physical boundary pass fills it
      bd += bd < 0 ? nbl : -nbl;     // periodic
    }
    b[d] = bd;
    q[d] = p[d] - side * nb;          // padded index inside block b
    G[d] = bd * nb + q[d] - NGH;      // global cell at level L
  }
  real val[NVAR + 1];
  const int nv = kp.nvs;
  const int o = lookup_block(kp, member, L, b);
  if (o >= 0) {
#pragma unroll
    for (int v = 0; v < NVAR + 1; v++)
      if (v < nv) val[v] = U[cell_index(kp, o, v, q[0], q[1], q[2])];
  } else if (o == -1) {
    // A coarse cell covers a 2 x 2 x 2 group of ghost cells (blocks start at
    // even global indices and there are two ghost layers): the group's
    // first cell computes the eight children once and writes all of them.
    if ((p[0] | p[1] | p[2]) & 1) return;
    int cb[3], Ic[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
      cb[d] = b[d] >> 1;
      Ic[d] = G[d] >> 1;
    }
    const int cs = lookup_block(kp, member, L - 1, cb);
    if (cs < 0) {
      atomicOr(kp.status, ST_TREE);
      return;
    }
    prolong_into<real>(kp, U, cs, L - 1, Ic, slot, p, false);
    return;
  } else {
    if (!restrict_in_block<real>(kp, U, member, L, b, q, G, val)) {
      atomicOr(kp.status, ST_TREE);
      return;
    }
  }
#pragma unroll
  for (int v = 0; v < NVAR + 1; v++)
    if (v < nv) U[cell_index(kp, slot, v, p[0], p[1], p[2])] = val[v];
}

// Ghost cells of one region of a level-L leaf (one of the 26 around it, r =
// 9 (sx + 1) + 3 (sy + 1) + sz + 1) that a coarser leaf holds (one lane per
// 2 x 2 x 2 group, prolongation) or finer leaves hold (one lane per cell,
// restriction).  A work item is up to 32 such tasks of one region, taken
// by one warp: item = (slot, r | finer << 8 | chunk << 9), tasks 32 chunk
// .. 32 chunk + 31 of the region-ordered shell list (group-first cells
// first) behind its table of (start, group-first cells, cells) per region.
// Same-level halo cells the prolongation's stencil reaches are read from
// the neighbouring leaf (the step's fills leave those ghost copies unfilled).
template <typename real>
__global__ void __launch_bounds__(256, sizeof(real) == 4 ? 3 : 2) k_ghost_regions(const KParams kp, real *U, const int2 *items, int nitems, const int *rshell, int L) {
  const int w = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (w >= nitems) return;
  const int2 e = items[w];
  const int slot = e.x, r = e.y & 255;
  const bool finer = ((e.y >> 8) & 1) != 0;
  const int t = ((e.y >> 9) << 5) + (threadIdx.x & 31);
  if (t >= (finer ? rshell[3 * r + 2] : rshell[3 * r + 1])) return;
  const int code = rshell[81 + rshell[3 * r] + t];
  const int p[3] = {code >> 20, (code >> 10) & 1023, code & 1023};
  const DevBlock B = kp.blk[slot];
  const int side[3] = {r / 9 - 1, (r / 3) % 3 - 1, r % 3 - 1};
  int b[3], q[3], G[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    // items exist only for neighbours inside the domain or across a
    // periodic direction
    const int nbl = kp.nbase[d] << (L - 1);
    int bd = B.ix[d] + side[d];
    if (bd < 0) bd += nbl;
    else if (bd >= nbl) bd -= nbl;
    b[d] = bd;
    q[d] = p[d] - side[d] * kp.nb[d];   // padded index inside block b
    G[d] = bd * kp.nb[d] + q[d] - NGH;
  }
  if (!finer) {
    int cb[3], Ic[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
      cb[d] = b[d] >> 1;
      Ic[d] = G[d] >> 1;
    }
    const int cs = lookup_block(kp, B.member, L - 1, cb);
    if (cs < 0) {
      atomicOr(kp.status, ST_TREE);
      return;
    }
    prolong_into<real>(kp, U, cs, L - 1, Ic, slot, p, true);
  } else {
    real val[NVAR + 1];
    if (!restrict_in_block<real>(kp, U, B.member, L, b, q, G, val)) {
      atomicOr(kp.status, ST_TREE);
      return;
    }
    const int nv = kp.nvs;
#pragma unroll
    for (int v = 0; v < NVAR + 1; v++)
      if (v < nv) U[cell_index(kp, slot, v, p[0], p[1], p[2])] = val[v];
  }
}

// inner boundary state (FP64): map of the containing base cell, cone CME
// overlay; u[TRV] = rho X with the CME tracer X = 1 in the CME plasma, else 0
__device__ void inner_state(const KParams &kp, int member, int L, int J, int K, double t, double *u) {
  double X = 0.0;
  const int n1 = kp.n_base_cells[1], n2 = kp.n_base_cells[2];
  const int jb = J >> (L - 1), kb = K >> (L - 1);
  const double *m = kp.bmap + (size_t)member * NVAR * n1 * n2;
  double w[NVAR];
#pragma unroll
  for (int v = 0; v < NVAR; v++) w[v] = m[((size_t)v * n1 + jb) * n2 + kb];
  const DevCme c = kp.cme[member];
  if (c.active) {
    const LevelGeo<double> &G = kp.geo->d[L];
    const double th = G.tc[J + NGH], ph = G.pc[K + NGH];
    const double R = G.rf[NGH];
    const double tau = t - c.t_start;
    if (tau >= 0.0 && tau <= c.t_max) {
      const double rh = R * sin(c.half_width);
      const double Rc = tau * c.v + R - rh;
      const double arg = (Rc * Rc + R * R - rh * rh) / (2.0 * Rc * R);
      if (!(arg > 1.0)) {
        const double open = acos(arg);
        double a = sin(th) * sin(c.colat) * cos(ph - c.lon) + cos(th) * cos(c.colat);
        a = a > 1.0 ? 1.0 : (a < -1.0 ? -1.0 : a);
        if (acos(a) <= open) {
          w[0] = c.rho;
          w[1] = c.v;
          w[2] = 0.0;
          w[3] = -kp.omega * R * sin(th);
          w[4] = c.p;
          w[5] = w[6] = w[7] = 0.0;
          X = 1.0;
        }
      }
    }
  }
  prim2cons<double>(w, u, 1.0 / (kp.gamma - 1.0));
  u[TRV] = w[0] * X;
}

// physical boundary of direction `dir`; sides[n] = (slot, side)
// faces: only the ghost cells inside the block in the two other directions
template <typename real>
__global__ void k_ghost_physical(const KParams kp, real *U, const int2 *sides, int dir, int L, double tfac,
                                 int faces, int skip_same) {
  const int2 sd = sides[blockIdx.x];
  const int slot = sd.x, side = sd.y;
  const int da = dir == 0 ? 1 : 0, db = dir == 2 ? 1 : 2;
  const int Pa = faces ? kp.nb[da] : kp.P[da], Pb = faces ? kp.nb[db] : kp.P[db], off = faces ? NGH : 0;
  const int idx = blockIdx.y * blockDim.x + threadIdx.x;
  if (idx >= NGH * Pa * Pb) return;
  const int gl = idx / (Pa * Pb), r = idx % (Pa * Pb), a = r / Pb + off, b = r % Pb + off;
  const int bc = side ? kp.bc_hi[dir] : kp.bc_lo[dir];
  const int nbd = kp.nb[dir];
  const int pg = side ? NGH + nbd + gl : NGH - 1 - gl;
  const int pn = side ? NGH + nbd - 1 : NGH;
  const int pm = side ? NGH + nbd - 1 - gl : NGH + gl;
  int q[3], s[3];
  q[dir] = pg;
  q[da] = a;
  q[db] = b;
  s[da] = a;
  s[db] = b;
  const DevBlock B = kp.blk[slot];
  if (bc == 3) {  // inner boundary (r low)
    bool in1, in2;
    const int J = wrap_dim(kp, L, 1, B.ix[1] * kp.nb[1] + q[1] - NGH, in1);
    const int K = wrap_dim(kp, L, 2, B.ix[2] * kp.nb[2] + q[2] - NGH, in2);
    if (!in1 || !in2) return;
    const double t = kp.t[B.member] + tfac * kp.dt_used[B.member];
    double u[NVAR + 1];
    inner_state(kp, B.member, L, J, K, t, u);
#pragma unroll
    for (int v = 0; v < NVAR + 1; v++)
      if (v < kp.nvs) U[cell_index(kp, slot, v, q[0], q[1], q[2])] = (real)u[v];
    return;
  }
  s[dir] = bc == 2 ? pm : pn;
#pragma unroll
  for (int v = 0; v < NVAR + 1; v++) {
    if (v >= kp.nvs) break;
    real x = fetch(kp, U, slot, v, s[0], s[1], s[2], skip_same != 0);
    if (bc == 2 && (v == 1 + dir || v == 5 + dir)) x = -x;
    U[cell_index(kp, slot, v, q[0], q[1], q[2])] = x;
  }
}

// reflux of coarse blocks with finer face neighbours; one CTA per block
template <typename real>
__global__ void k_reflux(const KParams kp, real *U, const real *flux, const int *list) {
  const int slot = list[blockIdx.x];
  const DevBlock B = kp.blk[slot];
  const double dtm = kp.dt_used[B.member];
  if (!(dtm > 0.0)) return;
  const real dt = (real)dtm;
  const int L = B.level;
  const int nb0 = kp.nb[0], nb1 = kp.nb[1], nb2 = kp.nb[2];
  const int fc[3] = {nb1 * nb2, nb0 * nb2, nb0 * nb1};
  const size_t fstride = (size_t)NVAR * 2 * (fc[0] + fc[1] + fc[2]);
  size_t foff[6];
  {
    size_t o = 0;
    for (int f = 0; f < 6; f++) {
      foff[f] = o;
      o += (size_t)NVAR * fc[f / 2];
    }
  }
  const LevelGeo<real> &G = GeoSel<real>::get(kp.geo, L);
  for (int f = 0; f < 6; f++) {
    if (B.nbr[f] != NB_FINER) continue;
    const int d = f / 2, hi = f % 2;
    const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
    for (int t = threadIdx.x; t < fc[d]; t += blockDim.x) {
      const int t1 = t / kp.nb[d2], t2 = t % kp.nb[d2];
      int Gc[3];
      Gc[d1] = B.ix[d1] * kp.nb[d1] + t1;
      Gc[d2] = B.ix[d2] * kp.nb[d2] + t2;
      Gc[d] = hi ? (B.ix[d] + 1) * kp.nb[d] : B.ix[d] * kp.nb[d] - 1;  // coarse cell across
      real fs[NVAR];
#pragma unroll
      for (int v = 0; v < NVAR; v++) fs[v] = real(0);
      for (int a = 0; a < 2; a++)
        for (int c = 0; c < 2; c++) {
          int F[3];
          F[d] = hi ? 2 * Gc[d] : 2 * Gc[d] + 1;
          F[d1] = 2 * Gc[d1] + a;
          F[d2] = 2 * Gc[d2] + c;
          bool in;
          for (int e = 0; e < 3; e++) F[e] = wrap_dim(kp, L + 1, e, F[e], in);
          const int fsl = lookup(kp, B.member, L + 1, F);
          if (fsl < 0) {
            atomicOr(kp.status, ST_TREE);
            continue;
          }
          const DevBlock FB = kp.blk[fsl];
          const int s1 = F[d1] - FB.ix[d1] * kp.nb[d1], s2 = F[d2] - FB.ix[d2] * kp.nb[d2];
          const real *src = flux + (size_t)fsl * fstride + foff[2 * d + (hi ? 0 : 1)];
#pragma unroll
          for (int v = 0; v < NVAR; v++) fs[v] += src[(size_t)v * fc[d] + s1 * kp.nb[d2] + s2];
        }
      int q[3];
      q[d] = hi ? NGH + kp.nb[d] - 1 : NGH;
      q[d1] = NGH + t1;
      q[d2] = NGH + t2;
      const int I = B.ix[0] * nb0 + q[0] - NGH, J = B.ix[1] * nb1 + q[1] - NGH;
      const real V = G.dr3[I + NGH] * G.dcos[J + NGH] * G.dphi;
      const real *own = flux + (size_t)slot * fstride + foff[f];
      const real sg = hi ? real(-1) : real(1);
#pragma unroll
      for (int v = 0; v < NVAR; v++) {
        const size_t ci = cell_index(kp, slot, v, q[0], q[1], q[2]);
        U[ci] += sg * dt / V * (fs[v] - own[(size_t)v * fc[d] + t]);
      }
    }
    __syncthreads();
  }
  // floors and CFL contribution of every corrected cell
  const real gamma = (real)kp.gamma, pfl = (real)kp.p_floor, rfl = (real)kp.rho_floor;
  double acc = 0.0;
  long long hits = 0;
  for (int f = 0; f < 6; f++) {
    if (B.nbr[f] != NB_FINER) continue;
    const int d = f / 2, hi = f % 2;
    const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
    for (int t = threadIdx.x; t < fc[d]; t += blockDim.x) {
      const int t1 = t / kp.nb[d2], t2 = t % kp.nb[d2];
      int q[3];
      q[d] = hi ? NGH + kp.nb[d] - 1 : NGH;
      q[d1] = NGH + t1;
      q[d2] = NGH + t2;
      real u[NVAR];
#pragma unroll
      for (int v = 0; v < NVAR; v++) u[v] = U[cell_index(kp, slot, v, q[0], q[1], q[2])];
      hits += apply_floors<real>(u, gamma, pfl, rfl, Isl{(float)kp.isl_pe, (float)kp.isl_beta});
#pragma unroll
      for (int v = 0; v < NVAR; v++) U[cell_index(kp, slot, v, q[0], q[1], q[2])] = u[v];
      real w[NVAR];
      cons2prim_speed<real>(u, w, gamma, pfl);
      const int I = B.ix[0] * nb0 + q[0] - NGH + NGH, J = B.ix[1] * nb1 + q[1] - NGH + NGH;
      real dx0 = G.dr[I], dx1 = G.dth[J], dx2 = G.dphi;
      if (kp.geometry == 0) {
        dx1 *= G.rc[I];
        dx2 *= G.rc[I] * G.sintc[J];
      }
      const real sp = (RT<real>::abs_(w[1]) + fast_speed<real, 0>(w, gamma)) / dx0 +
                      (RT<real>::abs_(w[2]) + fast_speed<real, 1>(w, gamma)) / dx1 +
                      (RT<real>::abs_(w[3]) + fast_speed<real, 2>(w, gamma)) / dx2;
      acc = fmax(acc, (double)sp);
    }
    __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc = fmax(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    hits += __shfl_xor_sync(0xffffffffu, hits, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (acc > 0.0) atomic_max_pos(&kp.inv_max[B.member], acc);
    if (hits) atomicAdd(kp.floor_hits, (unsigned long long)hits);
  }
}

__global__ void k_dt_begin(const KParams kp, const double *tstop) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= kp.n_members) return;
  double dt = fmin(kp.dt_cfl[m], tstop[m] - kp.t[m]);
  kp.dt_used[m] = dt > 0.0 ? dt : 0.0;
}

__global__ void k_dt_finalize(const KParams kp, double cfl) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m == 0) {
    // floor budget: the floors the step applied (both stages) against the
    // leaf cells it advanced
    const unsigned long long h = *kp.floor_hits, d = h - *kp.floor_prev;
    *kp.floor_prev = h;
    if (kp.floor_budget > 0.0 && d > 0) {
      double cells = 0.0;
      for (int q = 0; q < kp.n_members; q++)
        if (kp.dt_used[q] > 0.0) cells += kp.cells_m[q];
      if ((double)d > kp.floor_budget * cells) atomicOr(kp.status, ST_FLOOR);
    }
  }
  if (m >= kp.n_members) return;
  const double dt = kp.dt_used[m];
  if (dt > 0.0) {
    kp.t[m] += dt;
    kp.updates[m] += kp.cells_m[m];
    const double inv = __longlong_as_double((long long)kp.inv_max[m]);
    if (inv > 0.0) kp.dt_cfl[m] = cfl / inv;
  }
  kp.inv_max[m] = 0ull;
}

// CFL time step of the whole current state (after set_state / regrid / init)
template <typename real>
__global__ void k_dt_full(const KParams kp, const real *U) {
  const int slot = blockIdx.x;
  const DevBlock B = kp.blk[slot];
  const LevelGeo<real> &G = GeoSel<real>::get(kp.geo, B.level);
  const real gamma = (real)kp.gamma, pfl = (real)kp.p_floor;
  double acc = 0.0;
  for (int c = blockIdx.y * blockDim.x + threadIdx.x; c < kp.icells; c += gridDim.y * blockDim.x) {
    const int k = c % kp.nb[2], j = (c / kp.nb[2]) % kp.nb[1], i = c / (kp.nb[2] * kp.nb[1]);
    real u[NVAR], w[NVAR];
#pragma unroll
    for (int v = 0; v < NVAR; v++) u[v] = U[cell_index(kp, slot, v, i + NGH, j + NGH, k + NGH)];
    cons2prim_speed<real>(u, w, gamma, pfl);
    const int I = B.ix[0] * kp.nb[0] + i + NGH, J = B.ix[1] * kp.nb[1] + j + NGH;
    real dx0 = G.dr[I], dx1 = G.dth[J], dx2 = G.dphi;
    if (kp.geometry == 0) {
      dx1 *= G.rc[I];
      dx2 *= G.rc[I] * G.sintc[J];
    }
    const real sp = (RT<real>::abs_(w[1]) + fast_speed<real, 0>(w, gamma)) / dx0 +
                    (RT<real>::abs_(w[2]) + fast_speed<real, 1>(w, gamma)) / dx1 +
                    (RT<real>::abs_(w[3]) + fast_speed<real, 2>(w, gamma)) / dx2;
    acc = fmax(acc, (double)sp);
  }
  for (int o = 16; o > 0; o >>= 1) acc = fmax(acc, __shfl_xor_sync(0xffffffffu, acc, o));
  if ((threadIdx.x & 31) == 0 && acc > 0.0) atomic_max_pos(&kp.inv_max[B.member], acc);
}

__global__ void k_dt_from_max(const KParams kp, double cfl) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= kp.n_members) return;
  const double inv = __longlong_as_double((long long)kp.inv_max[m]);
  kp.dt_cfl[m] = inv > 0.0 ? cfl / inv : 0.0;
  kp.inv_max[m] = 0ull;
}

}  // namespace

void ghost_neighbour_launch(const KParams &kp, void *U, int precision, const int *list, int nlist, const int *shell,
                            int nshell, int level, cudaStream_t s) {
  if (nlist <= 0) return;
  dim3 grid(nlist, (nshell + 255) / 256);
  if (precision)
    k_ghost_neighbour<float><<<grid, 256, 0, s>>>(kp, (float *)U, list, shell, nshell, level);
  else
    k_ghost_neighbour<double><<<grid, 256, 0, s>>>(kp, (double *)U, list, shell, nshell, level);
}

void ghost_regions_launch(const KParams &kp, void *U, int precision, const int2 *items, int nitems,
                          const int *rshell, int level, cudaStream_t s) {
  if (nitems <= 0) return;
  const int grid = (nitems + 7) / 8;   // one warp per item
  if (precision)
    k_ghost_regions<float><<<grid, 256, 0, s>>>(kp, (float *)U, items, nitems, rshell, level);
  else
    k_ghost_regions<double><<<grid, 256, 0, s>>>(kp, (double *)U, items, nitems, rshell, level);
}

void ghost_physical_launch(const KParams &kp, void *U, int precision, const int2 *sides, int nsides, int dir,
                           int level, double tfac, bool faces_only, bool skip_same, cudaStream_t s) {
  if (nsides <= 0) return;
  const int da = dir == 0 ? 1 : 0, db = dir == 2 ? 1 : 2;
  const int n = faces_only ? NGH * kp.nb[da] * kp.nb[db] : NGH * kp.P[da] * kp.P[db];
  dim3 grid(nsides, (n + 127) / 128);
  if (precision)
    k_ghost_physical<float><<<grid, 128, 0, s>>>(kp, (float *)U, sides, dir, level, tfac, faces_only, skip_same);
  else
    k_ghost_physical<double><<<grid, 128, 0, s>>>(kp, (double *)U, sides, dir, level, tfac, faces_only, skip_same);
}

void reflux_launch(const KParams &kp, void *U, const void *flux, int precision, const int *list, int nlist,
                   cudaStream_t s) {
  if (nlist <= 0) return;
  if (precision)
    k_reflux<float><<<nlist, 256, 0, s>>>(kp, (float *)U, (const float *)flux, list);
  else
    k_reflux<double><<<nlist, 256, 0, s>>>(kp, (double *)U, (const double *)flux, list);
}

void dt_begin_launch(const KParams &kp, const double *tstop, cudaStream_t s) {
  k_dt_begin<<<(kp.n_members + 127) / 128, 128, 0, s>>>(kp, tstop);
}

void dt_finalize_launch(const KParams &kp, double cfl, cudaStream_t s) {
  k_dt_finalize<<<(kp.n_members + 127) / 128, 128, 0, s>>>(kp, cfl);
}

void dt_full_launch(const KParams &kp, const void *U, int precision, int nleaves, double cfl, cudaStream_t s) {
  if (nleaves > 0) {
    if (precision)
      k_dt_full<float><<<dim3(nleaves, (kp.icells + 4095) / 4096), 256, 0, s>>>(kp, (const float *)U);
    else
      k_dt_full<double><<<dim3(nleaves, (kp.icells + 4095) / 4096), 256, 0, s>>>(kp, (const double *)U);
  }
  k_dt_from_max<<<(kp.n_members + 127) / 128, 128, 0, s>>>(kp, cfl);
}
