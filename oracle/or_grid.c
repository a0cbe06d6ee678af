/*
 * Oracle, block-structured grid: geometry, tree, ghost fill, stage operator,
 * reflux, time step, refinement estimator, regrid, probe.
 * TEST INFRASTRUCTURE ONLY (see or_internal.h).
 *
 * Method (arXiv 2211.12867):
 *   Sect. 2.1  ideal MHD in the co-rotating frame, TVDLF + Woodward limiter,
 *              second order in space and time, parabolic div B cleaning,
 *              two ghost layers, fixed inner boundary, cone CME (Eqs. 1-4).
 *   Sect. 2.2  radial stretching: geometric radial faces (Eq. 5 gives N).
 *   Sect. 3    block AMR, factor 2 per level in every direction, neighbours
 *              differ by at most one level, blocks coarsen when the criterion
 *              no longer holds.
 * Where the paper is silent a reading is taken; each is stated at its use
 * below (tagged R2 ... R19).
 *
 * Everything is FP64 in natural loop order; no blocking, no fusion.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "or_internal.h"

/* ------------------------------------------------------------------ */
/* geometry                                                            */
/* ------------------------------------------------------------------ */
int or_ncells(const or_grid *g, int L, int d) { return g->p.n[d] << (L - 1); }
int or_pdim(const or_grid *g, int d) { return g->p.nb[d] + 2 * NG; }
size_t or_pcells(const or_grid *g) {
  return (size_t)or_pdim(g, 0) * or_pdim(g, 1) * or_pdim(g, 2);
}
double or_face(const or_grid *g, int L, int d, int I) { return g->xf[d][L][I + NG]; }
double or_centre(const or_grid *g, int L, int d, int I) {
  return 0.5 * (g->xf[d][L][I + NG] + g->xf[d][L][I + NG + 1]);
}

/* Faces of level L.  Radial stretching (Sect. 2.2, reading R8): r_I =
 * r_in (r_out/r_in)^(I/N_L); the exponent I/N_L is the same rational for a
 * coarse face and its fine twin, so every coarse face is a fine face. */
static void build_faces(or_grid *g) {
  for (int L = 1; L <= g->p.max_level; L++)
    for (int d = 0; d < 3; d++) {
      int N = or_ncells(g, L, d);
      double *f = malloc(sizeof(double) * (N + 2 * NG + 1));
      for (int I = -NG; I <= N + NG; I++) {
        double x = (double)I / (double)N;
        double v;
        if (d == 0 && g->p.geometry == 0 && g->p.stretch)
          v = g->p.xmin[0] * pow(g->p.xmax[0] / g->p.xmin[0], x);
        else
          v = g->p.xmin[d] + (g->p.xmax[d] - g->p.xmin[d]) * x;
        f[I + NG] = v;
      }
      g->xf[d][L] = f;
    }
}

/* Mean of the fractional index coordinate u in [0,1] over one fine cell
 * [a,b] along d, weighted by the volume element (r^2 dr, sin(theta) dtheta,
 * dphi; 1 in Cartesian mode).  Used by the conservative prolongation
 * (reading R9): child offset = weighted mean index of child - of parent. */
static double mean_frac(const or_grid *g, int d, double a, double b, double *w) {
  if (g->p.geometry == 1 || d == 2) {
    *w = b - a;
    return 0.5;
  }
  if (d == 0) {
    *w = (b * b * b - a * a * a) / 3.0;
    if (g->p.stretch) {
      double q = b / a, q3 = q * q * q;
      return q3 / (q3 - 1.0) - 1.0 / (3.0 * log(q));
    }
    double num = (b * b * b * b - a * a * a * a) / 4.0 - a * (b * b * b - a * a * a) / 3.0;
    return num / ((b - a) * (b * b * b - a * a * a) / 3.0);
  }
  /* theta, weight sin(theta) */
  *w = cos(a) - cos(b);
  double num = -(b - a) * cos(b) + sin(b) - sin(a);
  return num / ((b - a) * (cos(a) - cos(b)));
}

static void build_offsets(or_grid *g) {
  for (int L = 1; L < g->p.max_level; L++)
    for (int d = 0; d < 3; d++) {
      int N = or_ncells(g, L, d);
      double *t = malloc(sizeof(double) * 2 * N);
      for (int I = 0; I < N; I++) {
        double a = or_face(g, L + 1, d, 2 * I);
        double m = or_face(g, L + 1, d, 2 * I + 1);
        double b = or_face(g, L + 1, d, 2 * I + 2);
        double w0, w1;
        double x0 = -0.5 + 0.5 * mean_frac(g, d, a, m, &w0);
        double x1 = 0.0 + 0.5 * mean_frac(g, d, m, b, &w1);
        double xp = (w0 * x0 + w1 * x1) / (w0 + w1);
        t[2 * I] = x0 - xp;
        t[2 * I + 1] = x1 - xp;
      }
      g->dlt[d][L] = t;
    }
}

/* cell volume and face areas; spherical: V = (r+^3-r-^3)/3 (cos th- - cos th+) dphi */
static double cell_volume(const or_grid *g, int L, int I, int J, int K) {
  double r0 = or_face(g, L, 0, I), r1 = or_face(g, L, 0, I + 1);
  double t0 = or_face(g, L, 1, J), t1 = or_face(g, L, 1, J + 1);
  double p0 = or_face(g, L, 2, K), p1 = or_face(g, L, 2, K + 1);
  if (g->p.geometry == 1) return (r1 - r0) * (t1 - t0) * (p1 - p0);
  return (r1 * r1 * r1 - r0 * r0 * r0) / 3.0 * (cos(t0) - cos(t1)) * (p1 - p0);
}

/* area of the low face (index I,J,K) of direction d */
static double face_area(const or_grid *g, int L, int d, int I, int J, int K) {
  double r0 = or_face(g, L, 0, I), r1 = or_face(g, L, 0, I + 1);
  double t0 = or_face(g, L, 1, J), t1 = or_face(g, L, 1, J + 1);
  double p0 = or_face(g, L, 2, K), p1 = or_face(g, L, 2, K + 1);
  if (g->p.geometry == 1) {
    if (d == 0) return (t1 - t0) * (p1 - p0);
    if (d == 1) return (r1 - r0) * (p1 - p0);
    return (r1 - r0) * (t1 - t0);
  }
  if (d == 0) return r0 * r0 * (cos(t0) - cos(t1)) * (p1 - p0);
  if (d == 1) return sin(t0) * (r1 * r1 - r0 * r0) / 2.0 * (p1 - p0);
  return (r1 * r1 - r0 * r0) / 2.0 * (t1 - t0);
}

/* ------------------------------------------------------------------ */
/* block storage and tree                                              */
/* ------------------------------------------------------------------ */
static inline size_t pidx(const or_grid *g, int v, int i, int j, int k) {
  return (((size_t)v * or_pdim(g, 0) + i) * or_pdim(g, 1) + j) * or_pdim(g, 2) + k;
}

static int face_ncells(const or_grid *g, int d) {
  int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
  return g->p.nb[d1] * g->p.nb[d2];
}

static void alloc_block_data(or_grid *g, ob *b) {
  size_t n = or_pcells(g) * NVT;
  b->U = calloc(n, sizeof(double));
  b->Us = calloc(n, sizeof(double));
  for (int f = 0; f < 6; f++) b->fx[f] = calloc((size_t)face_ncells(g, f / 2) * NV, sizeof(double));
}

static void free_block_data(ob *b) {
  free(b->U);
  free(b->Us);
  b->U = b->Us = NULL;
  for (int f = 0; f < 6; f++) {
    free(b->fx[f]);
    b->fx[f] = NULL;
  }
}

static int nblocks_at(const or_grid *g, int L, int d) { return g->nbase[d] << (L - 1); }

/* Leaf covering global cell (L, I, J, K).  Periodic directions wrap; a cell
 * outside a non-periodic direction returns NULL.  *lev receives the level of
 * the returned block; a non-leaf at level L means "covered by finer leaves". */
static ob *find_cover(const or_grid *g, int L, int I, int J, int K, int *lev) {
  int c[3] = {I, J, K};
  for (int d = 0; d < 3; d++) {
    int N = or_ncells(g, L, d);
    if (g->p.bc_lo[d] == BC_PERIODIC) {
      c[d] %= N;
      if (c[d] < 0) c[d] += N;
    } else if (c[d] < 0 || c[d] >= N)
      return NULL;
  }
  int bx[3];
  for (int d = 0; d < 3; d++) bx[d] = (c[d] >> (L - 1)) / g->p.nb[d];
  ob *b = &g->base[(bx[0] * g->nbase[1] + bx[1]) * g->nbase[2] + bx[2]];
  while (!b->is_leaf && b->level < L) {
    int off[3];
    for (int d = 0; d < 3; d++) {
      int cb = (c[d] >> (L - b->level - 1)) / g->p.nb[d];
      off[d] = cb - 2 * b->ix[d];
    }
    b = b->child[(off[0] << 2) | (off[1] << 1) | off[2]];
  }
  *lev = b->level;
  return b;
}

static uint64_t morton(const or_grid *g, const ob *b) {
  uint64_t key = 0;
  int s = g->p.max_level - b->level;
  uint64_t x[3];
  for (int d = 0; d < 3; d++) x[d] = (uint64_t)b->ix[d] << s;
  for (int bit = 20; bit >= 0; bit--)
    for (int d = 0; d < 3; d++) key = (key << 1) | ((x[d] >> bit) & 1u);
  return key;
}

static const or_grid *sort_grid;
static int cmp_leaf(const void *a, const void *b) {
  uint64_t ka = morton(sort_grid, *(ob *const *)a), kb = morton(sort_grid, *(ob *const *)b);
  return ka < kb ? -1 : (ka > kb ? 1 : 0);
}

static void collect(or_grid *g, ob *b) {
  if (b->is_leaf) {
    if (g->nleaves == g->cap_leaves) {
      g->cap_leaves = g->cap_leaves ? 2 * g->cap_leaves : 256;
      g->leaves = realloc(g->leaves, sizeof(ob *) * g->cap_leaves);
    }
    g->leaves[g->nleaves++] = b;
    return;
  }
  for (int c = 0; c < 8; c++) collect(g, b->child[c]);
}

/* face-neighbour level of every leaf face (0 = physical boundary) */
static void face_levels(or_grid *g) {
  for (int n = 0; n < g->nleaves; n++) {
    ob *b = g->leaves[n];
    int L = b->level;
    for (int f = 0; f < 6; f++) {
      int d = f / 2, hi = f % 2;
      int c[3];
      for (int e = 0; e < 3; e++) c[e] = b->ix[e] * g->p.nb[e];
      c[d] = hi ? (b->ix[d] + 1) * g->p.nb[d] : b->ix[d] * g->p.nb[d] - 1;
      int lev;
      ob *o = find_cover(g, L, c[0], c[1], c[2], &lev);
      if (!o) b->nbr_level[f] = 0;
      else if (lev < L) b->nbr_level[f] = L - 1;
      else if (o->is_leaf) b->nbr_level[f] = L;
      else b->nbr_level[f] = L + 1;
    }
  }
}

static void rebuild_leaves(or_grid *g) {
  g->nleaves = 0;
  int nb = g->nbase[0] * g->nbase[1] * g->nbase[2];
  for (int i = 0; i < nb; i++) collect(g, &g->base[i]);
  sort_grid = g;
  qsort(g->leaves, g->nleaves, sizeof(ob *), cmp_leaf);
  face_levels(g);
}

/* ------------------------------------------------------------------ */
/* prolongation / restriction (reading R9)                             */
/* ------------------------------------------------------------------ */
static inline double *buf(ob *b, int which) { return which ? b->Us : b->U; }

/* The 8 children of coarse cell (padded pc) of leaf cb (level Lc, global Ic):
 * U_child = U_p + sum_d s_d delta_{child,d}, s_d the MC-limited index-space
 * slope of the conserved variables; if any child has p <= 0 or rho <= 0 all
 * children take U_p. */
static void prolong_children(const or_grid *g, ob *cb, int which, const int pc[3],
                             const int Ic[3], double out[8][NVT]) {
  double *A = buf(cb, which);
  int Lc = cb->level;
  double s[3][NVT], up[NVT];
  for (int v = 0; v < NVT; v++) {
    up[v] = A[pidx(g, v, pc[0], pc[1], pc[2])];
    for (int d = 0; d < 3; d++) {
      int m[3] = {pc[0], pc[1], pc[2]}, p[3] = {pc[0], pc[1], pc[2]};
      m[d]--;
      p[d]++;
      s[d][v] = or_mc_slope(A[pidx(g, v, m[0], m[1], m[2])], up[v], A[pidx(g, v, p[0], p[1], p[2])]);
    }
  }
  int ok = 1;
  for (int ch = 0; ch < 8; ch++) {
    int o[3] = {(ch >> 2) & 1, (ch >> 1) & 1, ch & 1};
    double dl[3];
    for (int d = 0; d < 3; d++) dl[d] = g->dlt[d][Lc][2 * Ic[d] + o[d]];
    for (int v = 0; v < NVT; v++)
      out[ch][v] = ((up[v] + s[0][v] * dl[0]) + s[1][v] * dl[1]) + s[2][v] * dl[2];
    double W[NV];
    or_cons2prim(out[ch], W, g->p.gamma);
    if (!(W[RHO] > 0.0) || !(W[EN] > 0.0)) ok = 0;
  }
  if (!ok)
    for (int ch = 0; ch < 8; ch++)
      for (int v = 0; v < NVT; v++) out[ch][v] = up[v];
}

/* prolonged value of fine cell (Lf, I, J, K) from coarse leaf cb */
static void prolong_cell(const or_grid *g, ob *cb, int which, int I, int J, int K, double *out) {
  int Ic[3] = {I >> 1, J >> 1, K >> 1};
  int pc[3];
  for (int d = 0; d < 3; d++) pc[d] = Ic[d] - cb->ix[d] * g->p.nb[d] + NG;
  double ch[8][NVT];
  prolong_children(g, cb, which, pc, Ic, ch);
  int c = ((I & 1) << 2) | ((J & 1) << 1) | (K & 1);
  memcpy(out, ch[c], sizeof(double) * NVT);
}

static int wrap(const or_grid *g, int L, int d, int I, int *inside);

/* volume-weighted mean of the 8 level-(L+1) cells under cell (L, I, J, K) */
static void restrict_cell(const or_grid *g, int which, int L, int I, int J, int K, double *out) {
  double sum[NVT] = {0}, vs = 0.0;
  for (int a = 0; a < 2; a++)
    for (int b = 0; b < 2; b++)
      for (int c = 0; c < 2; c++) {
        int fI = 2 * I + a, fJ = 2 * J + b, fK = 2 * K + c;
        int lev;
        ob *fb = find_cover(g, L + 1, fI, fJ, fK, &lev);
        if (!fb || lev != L + 1 || !fb->is_leaf) {
          fprintf(stderr, "oracle: restriction source is not a level-%d leaf\n", L + 1);
          abort();
        }
        int ins, cI = wrap(g, L + 1, 0, fI, &ins), cJ = wrap(g, L + 1, 1, fJ, &ins);
        int wK = wrap(g, L + 1, 2, fK, &ins);
        double V = cell_volume(g, L + 1, cI, cJ, wK);
        double *A = buf(fb, which);
        int p0 = cI - fb->ix[0] * g->p.nb[0] + NG;
        int p1 = cJ - fb->ix[1] * g->p.nb[1] + NG;
        int p2 = wK - fb->ix[2] * g->p.nb[2] + NG;
        for (int v = 0; v < NVT; v++) sum[v] += V * A[pidx(g, v, p0, p1, p2)];
        vs += V;
      }
  for (int v = 0; v < NVT; v++) out[v] = sum[v] / vs;
}

/* ------------------------------------------------------------------ */
/* ghost fill (level by level; reading R9/R13)                         */
/* ------------------------------------------------------------------ */
static int wrap(const or_grid *g, int L, int d, int I, int *inside) {
  int N = or_ncells(g, L, d);
  if (g->p.bc_lo[d] == BC_PERIODIC) {
    *inside = 1;
    return ((I % N) + N) % N;
  }
  *inside = (I >= 0 && I < N);
  return I;
}

static void fill_neighbour_ghosts(or_grid *g, ob *b, int which) {
  int L = b->level;
  double *A = buf(b, which);
  int P[3] = {or_pdim(g, 0), or_pdim(g, 1), or_pdim(g, 2)};
  for (int i = 0; i < P[0]; i++)
    for (int j = 0; j < P[1]; j++)
      for (int k = 0; k < P[2]; k++) {
        int p[3] = {i, j, k};
        int interior = 1;
        for (int d = 0; d < 3; d++)
          if (p[d] < NG || p[d] >= NG + g->p.nb[d]) interior = 0;
        if (interior) continue;
        int G[3], in = 1;
        for (int d = 0; d < 3; d++) {
          int ins;
          G[d] = wrap(g, L, d, b->ix[d] * g->p.nb[d] + p[d] - NG, &ins);
          if (!ins) in = 0;
        }
        if (!in) continue;
        int lev;
        ob *o = find_cover(g, L, G[0], G[1], G[2], &lev);
        double val[NVT];
        if (lev == L && o->is_leaf) {
          double *B = buf(o, which);
          int q[3];
          for (int d = 0; d < 3; d++) q[d] = G[d] - o->ix[d] * g->p.nb[d] + NG;
          for (int v = 0; v < NVT; v++) val[v] = B[pidx(g, v, q[0], q[1], q[2])];
        } else if (lev == L - 1) {
          prolong_cell(g, o, which, G[0], G[1], G[2], val);
        } else if (lev == L) {
          restrict_cell(g, which, L, G[0], G[1], G[2], val);
        } else {
          fprintf(stderr, "oracle: 2:1 balance violated in ghost fill\n");
          abort();
        }
        for (int v = 0; v < NVT; v++) A[pidx(g, v, i, j, k)] = val[v];
      }
}

/* inner-boundary ghost state: the boundary map of the containing base cell
 * (not rescaled in r, reading R13), overlaid by the cone CME where d <= theta(t)
 * (Eqs. 1-4).  CME plasma: v_r = v_CME, v_ph = -Omega r_in sin(theta), B = 0. */
static void inner_state(const or_grid *g, int L, int J, int K, double t, double *U) {
  double W[NV], X = 0.0;
  int jb = J >> (L - 1), kb = K >> (L - 1);
  int n1 = g->p.n[1], n2 = g->p.n[2];
  for (int v = 0; v < NV; v++) W[v] = g->map[((size_t)v * n1 + jb) * n2 + kb];
  double th = or_centre(g, L, 1, J), ph = or_centre(g, L, 2, K);
  double R = g->p.xmin[0];
  double open = or_cme_opening(&g->cme, R, t);
  if (open >= 0.0 && or_cme_distance(&g->cme, th, ph) <= open) {
    W[RHO] = g->cme.rho;
    W[1] = g->cme.v;
    W[2] = 0.0;
    W[3] = -g->p.omega * R * sin(th);
    W[EN] = g->cme.p;
    W[5] = W[6] = W[7] = 0.0;
    X = 1.0;   /* CME plasma carries the tracer (Sect. 3.1) */
  }
  or_prim2cons(W, U, g->p.gamma);
  U[TR] = W[RHO] * X;
}

static void fill_physical_ghosts(or_grid *g, ob *b, int which, double t) {
  int L = b->level;
  double *A = buf(b, which);
  int P[3] = {or_pdim(g, 0), or_pdim(g, 1), or_pdim(g, 2)};
  for (int d = 0; d < 3; d++) {
    for (int side = 0; side < 2; side++) {
      int bc = side ? g->p.bc_hi[d] : g->p.bc_lo[d];
      if (bc == BC_PERIODIC) continue;
      int last = nblocks_at(g, L, d) - 1;
      if (side == 0 && b->ix[d] != 0) continue;
      if (side == 1 && b->ix[d] != last) continue;
      int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
      for (int gl = 0; gl < NG; gl++) {
        int pg = side ? NG + g->p.nb[d] + gl : NG - 1 - gl;
        int pn = side ? NG + g->p.nb[d] - 1 : NG;
        int pm = side ? NG + g->p.nb[d] - 1 - gl : NG + gl;
        for (int a = 0; a < P[d1]; a++)
          for (int c = 0; c < P[d2]; c++) {
            int q[3], s[3];
            q[d] = pg;
            q[d1] = a;
            q[d2] = c;
            s[d1] = a;
            s[d2] = c;
            if (bc == BC_INNER) {
              int ins1, ins2;
              int J = wrap(g, L, 1, b->ix[1] * g->p.nb[1] + q[1] - NG, &ins1);
              int K = wrap(g, L, 2, b->ix[2] * g->p.nb[2] + q[2] - NG, &ins2);
              if (!ins1 || !ins2) continue;
              double U[NVT];
              inner_state(g, L, J, K, t, U);
              for (int v = 0; v < NVT; v++) A[pidx(g, v, q[0], q[1], q[2])] = U[v];
              continue;
            }
            s[d] = bc == BC_REFLECT ? pm : pn;
            for (int v = 0; v < NVT; v++) {
              double x = A[pidx(g, v, s[0], s[1], s[2])];
              if (bc == BC_REFLECT && (v == 1 + d || v == 5 + d)) x = -x;
              A[pidx(g, v, q[0], q[1], q[2])] = x;
            }
          }
      }
    }
  }
}

void or_ghost_fill(or_grid *g, int which, double t) {
  for (int L = 1; L <= g->p.max_level; L++) {
#pragma omp parallel for schedule(dynamic)
    for (int n = 0; n < g->nleaves; n++) {
      ob *b = g->leaves[n];
      if (b->level != L) continue;
      fill_neighbour_ghosts(g, b, which);
      fill_physical_ghosts(g, b, which, t);
    }
  }
}

/* ------------------------------------------------------------------ */
/* stage operator                                                      */
/* ------------------------------------------------------------------ */
static void stage_prim(const or_grid *g, const double *U, double *W) {
  or_cons2prim(U, W, g->p.gamma);
  if (W[EN] < g->p.p_floor) W[EN] = g->p.p_floor;
}

static long apply_floors(const or_grid *g, double *U) {
  long hits = 0;
  if (U[RHO] < g->p.rho_floor) {
    U[RHO] = g->p.rho_floor;
    hits++;
  }
  double W[NV];
  or_cons2prim(U, W, g->p.gamma);
  if (W[EN] < g->p.p_floor) {
    double ke = 0.5 * (U[MR] * U[MR] + U[MT] * U[MT] + U[MP] * U[MP]) / U[RHO];
    double me = 0.5 * (U[BR] * U[BR] + U[BT] * U[BT] + U[BP] * U[BP]);
    U[EN] = g->p.p_floor / (g->p.gamma - 1.0) + ke + me;
    hits++;
  }
  return hits;
}

/* Geometric source terms (reading R7) from the spherical divergence of the
 * momentum and induction tensors in orthonormal components, pressure parts in
 * area-difference form so that a uniform state is preserved:
 *   g_r = (A_r+ - A_r-)/V ~ 2/r,   g_t = (A_t+ - A_t-)/V ~ cot(theta)/r. */
static void geometric_source(const double *W, double gr, double gt, double *S) {
  double rho = W[RHO], vr = W[1], vt = W[2], vp = W[3];
  double Br = W[5], Bt = W[6], Bp = W[7];
  double pt = W[EN] + 0.5 * (Br * Br + Bt * Bt + Bp * Bp);
  double ir = 0.5 * gr;
  S[MR] += (rho * (vt * vt + vp * vp) - (Bt * Bt + Bp * Bp)) * ir + pt * gr;
  S[MT] += (-rho * vr * vt + Br * Bt) * ir + (rho * vp * vp - Bp * Bp) * gt + pt * gt;
  S[MP] += (-rho * vr * vp + Br * Bp) * ir - (rho * vt * vp - Bt * Bp) * gt;
  S[BT] += (vr * Bt - vt * Br) * ir;
  S[BP] += (vr * Bp - vp * Br) * ir + (vt * Bp - vp * Bt) * gt;
}

/* Coriolis -2 rho Omega x v and centrifugal -rho Omega x (Omega x r) with
 * Omega along the polar axis; the centrifugal force does work rho v.a_cf. */
static void rotation_source(const double *W, double Om, double rc, double th, double *S) {
  double rho = W[RHO], vr = W[1], vt = W[2], vp = W[3];
  double st = sin(th), ct = cos(th);
  S[MR] += rho * (2.0 * Om * vp * st + Om * Om * rc * st * st);
  S[MT] += rho * (2.0 * Om * vp * ct + Om * Om * rc * st * ct);
  S[MP] += -2.0 * Om * rho * (vr * st + vt * ct);
  S[EN] += rho * Om * Om * rc * st * (vr * st + vt * ct);
}

/* One stage on leaf b:  Uout = U0 + dtf * L(Uin)  (+ parabolic cleaning from
 * Uin when clean != 0).  Face fluxes times area are kept on block faces that
 * border a different level, for the reflux. */
static long stage_block(or_grid *g, ob *b, int in_which, double dtf, int clean, int store_flux) {
  const int *nb = g->p.nb;
  int L = b->level;
  int P[3] = {or_pdim(g, 0), or_pdim(g, 1), or_pdim(g, 2)};
  size_t pc = or_pcells(g);
  double *Uin = buf(b, in_which);
  double *U0 = b->U;
  double *W = malloc(sizeof(double) * pc * NV);
  /* primitives on the padded block */
  for (int i = 0; i < P[0]; i++)
    for (int j = 0; j < P[1]; j++)
      for (int k = 0; k < P[2]; k++) {
        double u[NV], w[NV];
        for (int v = 0; v < NV; v++) u[v] = Uin[pidx(g, v, i, j, k)];
        stage_prim(g, u, w);
        for (int v = 0; v < NV; v++) W[pidx(g, v, i, j, k)] = w[v];
      }
  int g0 = b->ix[0] * nb[0] - NG, g1 = b->ix[1] * nb[1] - NG, g2 = b->ix[2] * nb[2] - NG;
  /* area-weighted face fluxes per direction: faces f = 0..nb[d] */
  double *AF[3];
  for (int d = 0; d < 3; d++) {
    int n0 = nb[0] + (d == 0), n1 = nb[1] + (d == 1), n2 = nb[2] + (d == 2);
    AF[d] = malloc(sizeof(double) * n0 * n1 * n2 * NV);
    for (int a = 0; a < n0; a++)
      for (int c = 0; c < n1; c++)
        for (int e = 0; e < n2; e++) {
          int q[3] = {a + NG, c + NG, e + NG}; /* cell on the high side of the face */
          double w4[4][NV];
          for (int s = 0; s < 4; s++) {
            int r[3] = {q[0], q[1], q[2]};
            r[d] += s - 2;
            for (int v = 0; v < NV; v++) w4[s][v] = W[pidx(g, v, r[0], r[1], r[2])];
          }
          double WL[NV], WR[NV];
          for (int v = 0; v < NV; v++) {
            double sl = or_mc_slope(w4[0][v], w4[1][v], w4[2][v]);
            double sr = or_mc_slope(w4[1][v], w4[2][v], w4[3][v]);
            WL[v] = w4[1][v] + 0.5 * sl;
            WR[v] = w4[2][v] - 0.5 * sr;
          }
          if (!(WL[RHO] > 0.0) || !(WL[EN] > 0.0) || !(WR[RHO] > 0.0) || !(WR[EN] > 0.0))
            for (int v = 0; v < NV; v++) {
              WL[v] = w4[1][v];
              WR[v] = w4[2][v];
            }
          double F[NV];
          or_tvdlf(WL, WR, d, g->p.gamma, F);
          double A = face_area(g, L, d, g0 + q[0], g1 + q[1], g2 + q[2]);
          size_t o = (((size_t)a * n1 + c) * n2 + e) * NV;
          for (int v = 0; v < NV; v++) AF[d][o + v] = A * F[v];
        }
  }
  /* div B at cells within one layer of the interior (cleaning, reading R6) */
  double *D = NULL;
  if (clean) {
    D = calloc(pc, sizeof(double));
    for (int i = NG - 1; i <= NG + nb[0]; i++)
      for (int j = NG - 1; j <= NG + nb[1]; j++)
        for (int k = NG - 1; k <= NG + nb[2]; k++) {
          int I = g0 + i, J = g1 + j, K = g2 + k;
          double rm = or_centre(g, L, 0, I - 1), rc = or_centre(g, L, 0, I), rp = or_centre(g, L, 0, I + 1);
          double tm = or_centre(g, L, 1, J - 1), tc = or_centre(g, L, 1, J), tp = or_centre(g, L, 1, J + 1);
          double pm = or_centre(g, L, 2, K - 1), pp = or_centre(g, L, 2, K + 1);
          double brm = Uin[pidx(g, BR, i - 1, j, k)], brp = Uin[pidx(g, BR, i + 1, j, k)];
          double btm = Uin[pidx(g, BT, i, j - 1, k)], btp = Uin[pidx(g, BT, i, j + 1, k)];
          double bpm = Uin[pidx(g, BP, i, j, k - 1)], bpp = Uin[pidx(g, BP, i, j, k + 1)];
          double div;
          if (g->p.geometry == 1)
            div = (brp - brm) / (rp - rm) + (btp - btm) / (tp - tm) + (bpp - bpm) / (pp - pm);
          else
            div = (rp * rp * brp - rm * rm * brm) / (rc * rc * (rp - rm)) +
                  (sin(tp) * btp - sin(tm) * btm) / (rc * sin(tc) * (tp - tm)) +
                  (bpp - bpm) / (rc * sin(tc) * (pp - pm));
          D[(((size_t)i) * P[1] + j) * P[2] + k] = div;
        }
  }
  long hits = 0;
  for (int a = 0; a < nb[0]; a++)
    for (int c = 0; c < nb[1]; c++)
      for (int e = 0; e < nb[2]; e++) {
        int i = a + NG, j = c + NG, k = e + NG;
        int I = g0 + i, J = g1 + j, K = g2 + k;
        double V = cell_volume(g, L, I, J, K);
        double dU[NV];
        size_t o0lo = (((size_t)a * nb[1] + c) * nb[2] + e) * NV;
        size_t o0hi = (((size_t)(a + 1) * nb[1] + c) * nb[2] + e) * NV;
        size_t o1lo = (((size_t)a * (nb[1] + 1) + c) * nb[2] + e) * NV;
        size_t o1hi = (((size_t)a * (nb[1] + 1) + c + 1) * nb[2] + e) * NV;
        size_t o2lo = (((size_t)a * nb[1] + c) * (nb[2] + 1) + e) * NV;
        size_t o2hi = (((size_t)a * nb[1] + c) * (nb[2] + 1) + e + 1) * NV;
        for (int v = 0; v < NV; v++)
          dU[v] = -((AF[0][o0hi + v] - AF[0][o0lo + v]) + (AF[1][o1hi + v] - AF[1][o1lo + v]) +
                    (AF[2][o2hi + v] - AF[2][o2lo + v])) / V;
        double w[NV];
        for (int v = 0; v < NV; v++) w[v] = W[pidx(g, v, i, j, k)];
        if (g->p.geometry == 0) {
          double Arm = face_area(g, L, 0, I, J, K), Arp = face_area(g, L, 0, I + 1, J, K);
          double Atm = face_area(g, L, 1, I, J, K), Atp = face_area(g, L, 1, I, J + 1, K);
          double S[NV] = {0};
          geometric_source(w, (Arp - Arm) / V, (Atp - Atm) / V, S);
          rotation_source(w, g->p.omega, or_centre(g, L, 0, I), or_centre(g, L, 1, J), S);
          for (int v = 0; v < NV; v++) dU[v] += S[v];
        }
        double un[NV];
        for (int v = 0; v < NV; v++) un[v] = U0[pidx(g, v, i, j, k)] + dtf * dU[v];
        if (clean && g->p.divb_cd > 0.0) {
          double rm = or_centre(g, L, 0, I - 1), rc = or_centre(g, L, 0, I), rp = or_centre(g, L, 0, I + 1);
          double tm = or_centre(g, L, 1, J - 1), tc = or_centre(g, L, 1, J), tp = or_centre(g, L, 1, J + 1);
          double pm = or_centre(g, L, 2, K - 1), pp = or_centre(g, L, 2, K + 1);
          double dr = or_face(g, L, 0, I + 1) - or_face(g, L, 0, I);
          double dt_ = or_face(g, L, 1, J + 1) - or_face(g, L, 1, J);
          double dp = or_face(g, L, 2, K + 1) - or_face(g, L, 2, K);
#define DD(ii, jj, kk) D[(((size_t)(ii)) * P[1] + (jj)) * P[2] + (kk)]
          double gr, gt, gp, h2inv;
          if (g->p.geometry == 1) {
            gr = (DD(i + 1, j, k) - DD(i - 1, j, k)) / (rp - rm);
            gt = (DD(i, j + 1, k) - DD(i, j - 1, k)) / (tp - tm);
            gp = (DD(i, j, k + 1) - DD(i, j, k - 1)) / (pp - pm);
            h2inv = 1.0 / (dr * dr) + 1.0 / (dt_ * dt_) + 1.0 / (dp * dp);
          } else {
            double st = sin(tc);
            gr = (DD(i + 1, j, k) - DD(i - 1, j, k)) / (rp - rm);
            gt = (DD(i, j + 1, k) - DD(i, j - 1, k)) / (rc * (tp - tm));
            gp = (DD(i, j, k + 1) - DD(i, j, k - 1)) / (rc * st * (pp - pm));
            double xt = rc * dt_, xp = rc * st * dp;
            h2inv = 1.0 / (dr * dr) + 1.0 / (xt * xt) + 1.0 / (xp * xp);
          }
#undef DD
          double f = g->p.divb_cd / h2inv;
          double dB[3] = {f * gr, f * gt, f * gp};
          double bs[3] = {Uin[pidx(g, BR, i, j, k)], Uin[pidx(g, BT, i, j, k)], Uin[pidx(g, BP, i, j, k)]};
          for (int c3 = 0; c3 < 3; c3++) un[5 + c3] += dB[c3];
          un[EN] += bs[0] * dB[0] + bs[1] * dB[1] + bs[2] * dB[2];
        }
        hits += apply_floors(g, un);
        double *Out = in_which == 0 ? b->Us : b->U;
        for (int v = 0; v < NV; v++) Out[pidx(g, v, i, j, k)] = un[v];
        if (g->p.tracer) {
          /* CME tracer (Sect. 3.1; reading R19): rho X carried by the mass
           * flux of each face with X taken from the face's upwind cell */
          double fl[3][2];
          size_t oo[3][2] = {{o0lo, o0hi}, {o1lo, o1hi}, {o2lo, o2hi}};
          for (int d = 0; d < 3; d++)
            for (int h = 0; h < 2; h++) {
              int lo[3] = {i, j, k}, hi3[3] = {i, j, k};
              if (h) hi3[d]++;
              else lo[d]--;
              double F = AF[d][oo[d][h] + RHO];
              double Xl = Uin[pidx(g, TR, lo[0], lo[1], lo[2])] / Uin[pidx(g, RHO, lo[0], lo[1], lo[2])];
              double Xh = Uin[pidx(g, TR, hi3[0], hi3[1], hi3[2])] / Uin[pidx(g, RHO, hi3[0], hi3[1], hi3[2])];
              fl[d][h] = F * (F > 0.0 ? Xl : Xh);
            }
          double dT = -((fl[0][1] - fl[0][0]) + (fl[1][1] - fl[1][0]) + (fl[2][1] - fl[2][0])) / V;
          Out[pidx(g, TR, i, j, k)] = U0[pidx(g, TR, i, j, k)] + dtf * dT;
        }
      }
  if (store_flux) {
    for (int f = 0; f < 6; f++) {
      if (b->nbr_level[f] == 0 || b->nbr_level[f] == L) continue;
      int d = f / 2, hi = f % 2;
      int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
      int n1 = nb[1] + (d == 1), n2 = nb[2] + (d == 2);
      for (int t1 = 0; t1 < nb[d1]; t1++)
        for (int t2 = 0; t2 < nb[d2]; t2++) {
          int q[3];
          q[d] = hi ? nb[d] : 0;
          q[d1] = t1;
          q[d2] = t2;
          size_t o = (((size_t)q[0] * n1 + q[1]) * n2 + q[2]) * NV;
          for (int v = 0; v < NV; v++) b->fx[f][((size_t)t1 * nb[d2] + t2) * NV + v] = AF[d][o + v];
        }
    }
  }
  for (int d = 0; d < 3; d++) free(AF[d]);
  free(D);
  free(W);
  return hits;
}

/* Reflux (reading R10): a coarse leaf face that borders finer leaves takes the
 * sum of the fine area-weighted fluxes of the final stage. */
static long reflux(or_grid *g, double dt) {
  long hits = 0;
  const int *nb = g->p.nb;
  for (int n = 0; n < g->nleaves; n++) {
    ob *b = g->leaves[n];
    int L = b->level, any = 0;
    for (int f = 0; f < 6; f++) {
      if (b->nbr_level[f] != L + 1) continue;
      any = 1;
      int d = f / 2, hi = f % 2;
      int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
      for (int t1 = 0; t1 < nb[d1]; t1++)
        for (int t2 = 0; t2 < nb[d2]; t2++) {
          int G[3];
          G[d1] = b->ix[d1] * nb[d1] + t1;
          G[d2] = b->ix[d2] * nb[d2] + t2;
          G[d] = hi ? (b->ix[d] + 1) * nb[d] : b->ix[d] * nb[d] - 1; /* coarse cell across */
          double fs[NV] = {0};
          for (int a = 0; a < 2; a++)
            for (int c = 0; c < 2; c++) {
              int F[3];
              F[d] = hi ? 2 * G[d] : 2 * G[d] + 1;
              F[d1] = 2 * G[d1] + a;
              F[d2] = 2 * G[d2] + c;
              int lev;
              ob *fb = find_cover(g, L + 1, F[0], F[1], F[2], &lev);
              int ins;
              int w1 = wrap(g, L + 1, d1, F[d1], &ins), w2 = wrap(g, L + 1, d2, F[d2], &ins);
              int s1 = w1 - fb->ix[d1] * nb[d1], s2 = w2 - fb->ix[d2] * nb[d2];
              const double *src = fb->fx[2 * d + (hi ? 0 : 1)];
              for (int v = 0; v < NV; v++) fs[v] += src[((size_t)s1 * nb[d2] + s2) * NV + v];
            }
          int q[3];
          q[d] = hi ? NG + nb[d] - 1 : NG;
          q[d1] = NG + t1;
          q[d2] = NG + t2;
          int I = b->ix[0] * nb[0] + q[0] - NG, J = b->ix[1] * nb[1] + q[1] - NG, K = b->ix[2] * nb[2] + q[2] - NG;
          double V = cell_volume(g, L, I, J, K);
          const double *own = b->fx[f] + ((size_t)t1 * nb[d2] + t2) * NV;
          double sgn = hi ? -1.0 : 1.0;
          for (int v = 0; v < NV; v++) b->U[pidx(g, v, q[0], q[1], q[2])] += sgn * dt / V * (fs[v] - own[v]);
        }
    }
    if (!any) continue;
    /* floors on the corrected cells */
    for (int f = 0; f < 6; f++) {
      if (b->nbr_level[f] != L + 1) continue;
      int d = f / 2, hi = f % 2;
      int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
      for (int t1 = 0; t1 < nb[d1]; t1++)
        for (int t2 = 0; t2 < nb[d2]; t2++) {
          int q[3];
          q[d] = hi ? NG + nb[d] - 1 : NG;
          q[d1] = NG + t1;
          q[d2] = NG + t2;
          double u[NV];
          for (int v = 0; v < NV; v++) u[v] = b->U[pidx(g, v, q[0], q[1], q[2])];
          hits += apply_floors(g, u);
          for (int v = 0; v < NV; v++) b->U[pidx(g, v, q[0], q[1], q[2])] = u[v];
        }
    }
  }
  return hits;
}

/* CFL time step (reading R2): dt = C min over leaf cells of
 * 1 / sum_d (|v_d| + c_f,d) / dx_d;  dx = (dr, r_c dtheta, r_c sin(theta_c) dphi). */
double or_compute_dt(or_grid *g) {
  double mx = 0.0;
  const int *nb = g->p.nb;
  for (int n = 0; n < g->nleaves; n++) {
    ob *b = g->leaves[n];
    int L = b->level;
    for (int a = 0; a < nb[0]; a++)
      for (int c = 0; c < nb[1]; c++)
        for (int e = 0; e < nb[2]; e++) {
          int I = b->ix[0] * nb[0] + a, J = b->ix[1] * nb[1] + c, K = b->ix[2] * nb[2] + e;
          double u[NV], w[NV];
          for (int v = 0; v < NV; v++) u[v] = b->U[pidx(g, v, a + NG, c + NG, e + NG)];
          stage_prim(g, u, w);
          double dx[3];
          for (int d = 0; d < 3; d++) {
            int Id = d == 0 ? I : (d == 1 ? J : K);
            dx[d] = or_face(g, L, d, Id + 1) - or_face(g, L, d, Id);
          }
          if (g->p.geometry == 0) {
            double rc = or_centre(g, L, 0, I), tc = or_centre(g, L, 1, J);
            dx[1] = rc * dx[1];
            dx[2] = rc * sin(tc) * dx[2];
          }
          double s = 0.0;
          for (int d = 0; d < 3; d++) s += (fabs(w[1 + d]) + or_fast_speed(w, d, g->p.gamma)) / dx[d];
          if (s > mx) mx = s;
        }
  }
  return g->p.cfl / mx;
}

/* One step, midpoint predictor-corrector (reading R3):
 * U* = U^n + dt/2 L(U^n);  U^{n+1} = U^n + dt L(U*) + cleaning(U*); reflux. */
void or_step(or_grid *g, double dt) {
  long hits = 0;
  or_ghost_fill(g, 0, g->t);
#pragma omp parallel for schedule(dynamic) reduction(+ : hits)
  for (int n = 0; n < g->nleaves; n++) hits += stage_block(g, g->leaves[n], 0, 0.5 * dt, 0, 0);
  or_ghost_fill(g, 1, g->t + 0.5 * dt);
#pragma omp parallel for schedule(dynamic) reduction(+ : hits)
  for (int n = 0; n < g->nleaves; n++) hits += stage_block(g, g->leaves[n], 1, dt, 1, 1);
  hits += reflux(g, dt);
  g->floor_hits += hits;
  g->t += dt;
}

/* advance up to nsteps, dt clipped so that t does not pass t_stop */
int or_advance(or_grid *g, int nsteps, double t_stop) {
  int s;
  for (s = 0; s < nsteps; s++) {
    double dt = or_compute_dt(g);
    if (t_stop - g->t < dt) dt = t_stop - g->t;
    if (!(dt > 0.0)) break;
    or_step(g, dt);
  }
  return s;
}

/* ------------------------------------------------------------------ */
/* refinement estimator (reading R11) and regrid                       */
/* ------------------------------------------------------------------ */
static double est_pressure(const double *u, double gamma) {
  double msq = (u[MR] * u[MR] + u[MT] * u[MT]) + u[MP] * u[MP];
  double bsq = (u[BR] * u[BR] + u[BT] * u[BT]) + u[BP] * u[BP];
  double ke = (0.5 * msq) / u[RHO];
  double me = 0.5 * bsq;
  return (gamma - 1.0) * ((u[EN] - ke) - me);
}

/* crit = {e_refine, e_coarsen, eps, dv}; flags: +1 refine, 0 keep, -1 coarsen.
 * Needs ghost-filled U. */
void or_flag(or_grid *g, const double *crit, signed char *flags) {
  const int *nb = g->p.nb;
  for (int n = 0; n < g->nleaves; n++) {
    ob *b = g->leaves[n];
    int L = b->level;
    int refine = 0, keep = 0;
    for (int a = 0; a < nb[0]; a++)
      for (int c = 0; c < nb[1]; c++)
        for (int e = 0; e < nb[2]; e++) {
          int i = a + NG, j = c + NG, k = e + NG;
          double u0[NV], um[3][NV], up[3][NV];
          for (int v = 0; v < NV; v++) u0[v] = b->U[pidx(g, v, i, j, k)];
          for (int d = 0; d < 3; d++) {
            int m[3] = {i, j, k}, p[3] = {i, j, k};
            m[d]--;
            p[d]++;
            for (int v = 0; v < NV; v++) {
              um[d][v] = b->U[pidx(g, v, m[0], m[1], m[2])];
              up[d][v] = b->U[pidx(g, v, p[0], p[1], p[2])];
            }
          }
          double rm[3], rp[3], pm[3], pp[3], r0 = u0[RHO], p0 = est_pressure(u0, g->p.gamma);
          for (int d = 0; d < 3; d++) {
            rm[d] = um[d][RHO];
            rp[d] = up[d][RHO];
            pm[d] = est_pressure(um[d], g->p.gamma);
            pp[d] = est_pressure(up[d], g->p.gamma);
          }
          double er = or_loehner(rm, &r0, rp, crit[2]);
          double ep = or_loehner(pm, &p0, pp, crit[2]);
          double E = er > ep ? er : ep;
          int gate = 0;
          if (g->vbg) {
            int I = b->ix[0] * nb[0] + a, J = b->ix[1] * nb[1] + c, K = b->ix[2] * nb[2] + e;
            int s = L - 1;
            double vb = g->vbg[((size_t)(I >> s) * g->p.n[1] + (J >> s)) * g->p.n[2] + (K >> s)];
            double vr = u0[MR] / u0[RHO];
            gate = vr > vb + crit[3];
          }
          if (gate && E > crit[0]) refine = 1;
          if (gate && E > crit[1]) keep = 1;
        }
    flags[n] = refine ? 1 : (keep ? 0 : -1);
  }
}

/* ------------------------------------------------------------------ */
/* shock criterion (Sect. 3.2; reading R18)                            */
/* ------------------------------------------------------------------ */
/* e = {colat, lon0, t0, rate}: Earth at colatitude colat and longitude
 * lon0 - rate (t - t0) in the co-rotating frame */
void or_set_earth(or_grid *g, const double *e) {
  g->earth.colat = e[0];
  g->earth.lon0 = e[1];
  g->earth.t0 = e[2];
  g->earth.rate = e[3];
  g->earth.set = 1;
}

/* divergence of the velocity v = m / rho at interior cell (a, c, e) of leaf
 * b: central differences over the two neighbours in each direction, in the
 * spherical form (1/r^2) d(r^2 v_r)/dr + (1/(r sin)) d(sin v_th)/dth +
 * (1/(r sin)) dv_ph/dph with centre coordinates (Cartesian: plain central
 * differences).  Needs one ghost layer. */
static double divv_cell(or_grid *g, ob *b, int a, int c, int e) {
  const int L = b->level, *nb = g->p.nb;
  const int I = b->ix[0] * nb[0] + a, J = b->ix[1] * nb[1] + c, K = b->ix[2] * nb[2] + e;
  const int i = a + NG, j = c + NG, k = e + NG;
  const double *U = b->U;
  double vrm = U[pidx(g, MR, i - 1, j, k)] / U[pidx(g, RHO, i - 1, j, k)];
  double vrp = U[pidx(g, MR, i + 1, j, k)] / U[pidx(g, RHO, i + 1, j, k)];
  double vtm = U[pidx(g, MT, i, j - 1, k)] / U[pidx(g, RHO, i, j - 1, k)];
  double vtp = U[pidx(g, MT, i, j + 1, k)] / U[pidx(g, RHO, i, j + 1, k)];
  double vpm = U[pidx(g, MP, i, j, k - 1)] / U[pidx(g, RHO, i, j, k - 1)];
  double vpp = U[pidx(g, MP, i, j, k + 1)] / U[pidx(g, RHO, i, j, k + 1)];
  double xm[3], x0[3], xp[3];
  for (int d = 0; d < 3; d++) {
    int Id = d == 0 ? I : (d == 1 ? J : K);
    xm[d] = or_centre(g, L, d, Id - 1);
    x0[d] = or_centre(g, L, d, Id);
    xp[d] = or_centre(g, L, d, Id + 1);
  }
  double tr, tt, tp;
  if (g->p.geometry == 0) {
    double sm = sin(xm[1]), s0 = sin(x0[1]), sp = sin(xp[1]);
    tr = ((xp[0] * xp[0]) * vrp - (xm[0] * xm[0]) * vrm) / ((x0[0] * x0[0]) * (xp[0] - xm[0]));
    tt = (sp * vtp - sm * vtm) / ((x0[0] * s0) * (xp[1] - xm[1]));
    tp = (vpp - vpm) / ((x0[0] * s0) * (xp[2] - xm[2]));
  } else {
    tr = (vrp - vrm) / (xp[0] - xm[0]);
    tt = (vtp - vtm) / (xp[1] - xm[1]);
    tp = (vpp - vpm) / (xp[2] - xm[2]);
  }
  return (tr + tt) + tp;
}

/* the interior velocity divergence of leaf n, [i][j][k] (after a ghost fill) */
void or_divv(or_grid *g, int n, double *out) {
  ob *b = g->leaves[n];
  const int *nb = g->p.nb;
  for (int a = 0; a < nb[0]; a++)
    for (int c = 0; c < nb[1]; c++)
      for (int e = 0; e < nb[2]; e++) out[((size_t)a * nb[1] + c) * nb[2] + e] = divv_cell(g, b, a, c, e);
}

/* angle a in [-pi, pi) */
static double wrap_angle(double a) {
  const double pi = 3.14159265358979323846, tp = 2.0 * pi;
  return a - tp * floor((a + pi) / tp);
}

/* crit = {div_thr, dlon_earth, dcolat_earth, dlon_cme}: a cell counts where
 * div v < -div_thr and its centre lies within dlon_earth of Earth's
 * longitude, within dcolat_earth of Earth's colatitude and within dlon_cme of
 * the CME's longitude (a half width <= 0 switches its window off; the Earth
 * windows need or_set_earth, the CME window a CME).  A block is flagged +1
 * when some interior cell counts and -1 (coarsen) otherwise: the paper
 * refines where the criterion holds and coarsens once it no longer does.
 * Needs ghost-filled U. */
void or_flag_shock(or_grid *g, const double *crit, signed char *flags) {
  const int *nb = g->p.nb;
  const double lon_e = g->earth.lon0 - g->earth.rate * (g->t - g->earth.t0);
  for (int n = 0; n < g->nleaves; n++) {
    ob *b = g->leaves[n];
    int L = b->level, refine = 0;
    for (int a = 0; a < nb[0] && !refine; a++)
      for (int c = 0; c < nb[1] && !refine; c++)
        for (int e = 0; e < nb[2] && !refine; e++) {
          int J = b->ix[1] * nb[1] + c, K = b->ix[2] * nb[2] + e;
          double th = or_centre(g, L, 1, J), ph = or_centre(g, L, 2, K);
          int in = 1;
          if (crit[1] > 0.0) in = in && g->earth.set && fabs(wrap_angle(ph - lon_e)) <= crit[1];
          if (crit[2] > 0.0) in = in && g->earth.set && fabs(th - g->earth.colat) <= crit[2];
          if (crit[3] > 0.0) in = in && g->cme.active && fabs(wrap_angle(ph - g->cme.lon)) <= crit[3];
          if (!in) continue;
          if (divv_cell(g, b, a, c, e) < -crit[0]) refine = 1;
        }
    flags[n] = refine ? 1 : -1;
  }
}

/* ------------------------------------------------------------------ */
/* CME tracer (Sect. 3.1) and combined criterion (Sect. 3.3)           */
/* ------------------------------------------------------------------ */
/* rho X of every leaf's interior cells, [leaf][i][j][k] */
void or_get_tracer(or_grid *g, double *out) {
  const int *nb = g->p.nb;
  size_t bc = (size_t)nb[0] * nb[1] * nb[2];
  for (int n = 0; n < g->nleaves; n++)
    for (int a = 0; a < nb[0]; a++)
      for (int c = 0; c < nb[1]; c++)
        for (int e = 0; e < nb[2]; e++)
          out[n * bc + ((size_t)a * nb[1] + c) * nb[2] + e] = g->leaves[n]->U[pidx(g, TR, a + NG, c + NG, e + NG)];
}

void or_set_tracer(or_grid *g, const double *in) {
  const int *nb = g->p.nb;
  size_t bc = (size_t)nb[0] * nb[1] * nb[2];
  for (int n = 0; n < g->nleaves; n++)
    for (int a = 0; a < nb[0]; a++)
      for (int c = 0; c < nb[1]; c++)
        for (int e = 0; e < nb[2]; e++)
          g->leaves[n]->U[pidx(g, TR, a + NG, c + NG, e + NG)] = in[n * bc + ((size_t)a * nb[1] + c) * nb[2] + e];
}

/* crit = {x_thr, div_thr, dlon_earth, dcolat_earth, dlon_cme, combined}: a
 * cell counts where its tracer fraction X = rho X / rho exceeds x_thr (the
 * paper refines where X is non-zero: x_thr = 0), or, when combined != 0,
 * also where div v < -div_thr (Sect. 3.3); the windows are those of the
 * shock criterion (a half width <= 0 switches one off).  +1 where some
 * interior cell counts, -1 otherwise.  Needs ghost-filled U (for div v). */
void or_flag_tracer(or_grid *g, const double *crit, signed char *flags) {
  const int *nb = g->p.nb;
  const double lon_e = g->earth.lon0 - g->earth.rate * (g->t - g->earth.t0);
  for (int n = 0; n < g->nleaves; n++) {
    ob *b = g->leaves[n];
    int L = b->level, refine = 0;
    for (int a = 0; a < nb[0] && !refine; a++)
      for (int c = 0; c < nb[1] && !refine; c++)
        for (int e = 0; e < nb[2] && !refine; e++) {
          int J = b->ix[1] * nb[1] + c, K = b->ix[2] * nb[2] + e;
          double th = or_centre(g, L, 1, J), ph = or_centre(g, L, 2, K);
          int in = 1;
          if (crit[2] > 0.0) in = in && g->earth.set && fabs(wrap_angle(ph - lon_e)) <= crit[2];
          if (crit[3] > 0.0) in = in && g->earth.set && fabs(th - g->earth.colat) <= crit[3];
          if (crit[4] > 0.0) in = in && g->cme.active && fabs(wrap_angle(ph - g->cme.lon)) <= crit[4];
          if (!in) continue;
          int i = a + NG, j = c + NG, k = e + NG;
          double X = b->U[pidx(g, TR, i, j, k)] / b->U[pidx(g, RHO, i, j, k)];
          if (X > crit[0]) refine = 1;
          else if (crit[5] != 0.0 && divv_cell(g, b, a, c, e) < -crit[1]) refine = 1;
        }
    flags[n] = refine ? 1 : -1;
  }
}

/* every leaf sharing a face, edge or corner with leaf b (periodic aware) */
static int leaf_neighbours(or_grid *g, ob *b, ob **out, int cap) {
  int n = 0, L = b->level;
  int F = L + 1 <= g->p.max_level ? L + 1 : L; /* resolution of the probe shell */
  int s = F - L;
  int lo[3], hi[3];
  for (int d = 0; d < 3; d++) {
    lo[d] = ((b->ix[d] * g->p.nb[d]) << s) - 1;
    hi[d] = ((b->ix[d] + 1) * g->p.nb[d]) << s;
  }
  for (int I = lo[0]; I <= hi[0]; I++)
    for (int J = lo[1]; J <= hi[1]; J++)
      for (int K = lo[2]; K <= hi[2]; K++) {
        if (I != lo[0] && I != hi[0] && J != lo[1] && J != hi[1] && K != lo[2] && K != hi[2]) continue;
        int lev;
        ob *o = find_cover(g, F, I, J, K, &lev);
        if (!o || o == b || !o->is_leaf) continue;
        int dup = 0;
        for (int m = 0; m < n; m++)
          if (out[m] == o) dup = 1;
        if (!dup && n < cap) out[n++] = o;
      }
  return n;
}

static void refine_block(or_grid *g, ob *b) {
  const int *nb = g->p.nb;
  for (int c = 0; c < 8; c++) {
    ob *ch = calloc(1, sizeof(ob));
    ch->level = b->level + 1;
    ch->ix[0] = 2 * b->ix[0] + ((c >> 2) & 1);
    ch->ix[1] = 2 * b->ix[1] + ((c >> 1) & 1);
    ch->ix[2] = 2 * b->ix[2] + (c & 1);
    ch->parent = b;
    ch->is_leaf = 1;
    alloc_block_data(g, ch);
    b->child[c] = ch;
  }
  /* prolong the parent's interior into the children */
  for (int a = 0; a < nb[0]; a++)
    for (int c = 0; c < nb[1]; c++)
      for (int e = 0; e < nb[2]; e++) {
        int pc[3] = {a + NG, c + NG, e + NG};
        int Ic[3] = {b->ix[0] * nb[0] + a, b->ix[1] * nb[1] + c, b->ix[2] * nb[2] + e};
        double kids[8][NVT];
        prolong_children(g, b, 0, pc, Ic, kids);
        for (int ch = 0; ch < 8; ch++) {
          int o[3] = {(ch >> 2) & 1, (ch >> 1) & 1, ch & 1};
          int F[3];
          for (int d = 0; d < 3; d++) F[d] = 2 * Ic[d] + o[d];
          int cb[3];
          for (int d = 0; d < 3; d++) cb[d] = F[d] / nb[d] - 2 * b->ix[d];
          ob *kid = b->child[(cb[0] << 2) | (cb[1] << 1) | cb[2]];
          int q[3];
          for (int d = 0; d < 3; d++) q[d] = F[d] - kid->ix[d] * nb[d] + NG;
          for (int v = 0; v < NVT; v++) kid->U[pidx(g, v, q[0], q[1], q[2])] = kids[ch][v];
        }
      }
  free_block_data(b);
  b->is_leaf = 0;
}

static void coarsen_block(or_grid *g, ob *b) {
  const int *nb = g->p.nb;
  alloc_block_data(g, b);
  b->is_leaf = 1;
  /* children are still linked: restrict their interiors */
  for (int a = 0; a < nb[0]; a++)
    for (int c = 0; c < nb[1]; c++)
      for (int e = 0; e < nb[2]; e++) {
        int I = b->ix[0] * nb[0] + a, J = b->ix[1] * nb[1] + c, K = b->ix[2] * nb[2] + e;
        double sum[NVT] = {0}, vs = 0.0;
        for (int x = 0; x < 2; x++)
          for (int y = 0; y < 2; y++)
            for (int z = 0; z < 2; z++) {
              int F[3] = {2 * I + x, 2 * J + y, 2 * K + z};
              int cb[3];
              for (int d = 0; d < 3; d++) cb[d] = F[d] / nb[d] - 2 * b->ix[d];
              ob *kid = b->child[(cb[0] << 2) | (cb[1] << 1) | cb[2]];
              int q[3];
              for (int d = 0; d < 3; d++) q[d] = F[d] - kid->ix[d] * nb[d] + NG;
              double V = cell_volume(g, b->level + 1, F[0], F[1], F[2]);
              for (int v = 0; v < NVT; v++) sum[v] += V * kid->U[pidx(g, v, q[0], q[1], q[2])];
              vs += V;
            }
        for (int v = 0; v < NVT; v++) b->U[pidx(g, v, a + NG, c + NG, e + NG)] = sum[v] / vs;
      }
  for (int c = 0; c < 8; c++) {
    free_block_data(b->child[c]);
    free(b->child[c]);
    b->child[c] = NULL;
  }
}

/* Regrid (Sect. 3; reading R11): refine flagged leaves one level, coarsen
 * complete sibling families flagged -1, refinement wins, then enforce 2:1
 * balance over faces, edges and corners by iterating to the least fixed
 * point (coarsenings are cancelled first, then leaves are refined). */
void or_regrid(or_grid *g, const signed char *flags) {
  or_ghost_fill(g, 0, g->t);
  int n = g->nleaves;
  int *T = malloc(sizeof(int) * n);
  for (int i = 0; i < n; i++) {
    ob *b = g->leaves[i];
    b->flag = flags[i];
    T[i] = b->level;
    if (flags[i] > 0 && b->level < g->p.max_level) T[i] = b->level + 1;
  }
  /* index lookup */
  for (int i = 0; i < n; i++) g->leaves[i]->id = i;
  for (int i = 0; i < n; i++) {
    ob *b = g->leaves[i];
    if (flags[i] >= 0 || b->level == 1) continue;
    ob *par = b->parent;
    int all = 1;
    for (int c = 0; c < 8; c++) {
      ob *s = par->child[c];
      if (!s->is_leaf || s->flag >= 0) all = 0;
    }
    if (all) T[i] = b->level - 1;
  }
  int cap = 4096;
  ob **nbr = malloc(sizeof(ob *) * cap);
  int **lists = malloc(sizeof(int *) * n), *cnt = malloc(sizeof(int) * n);
  for (int i = 0; i < n; i++) {
    int m = leaf_neighbours(g, g->leaves[i], nbr, cap);
    lists[i] = malloc(sizeof(int) * (m > 0 ? m : 1));
    for (int k = 0; k < m; k++) lists[i][k] = nbr[k]->id;
    cnt[i] = m;
  }
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int i = 0; i < n; i++) {
      ob *b = g->leaves[i];
      for (int k = 0; k < cnt[i]; k++) {
        int j = lists[i][k];
        if (T[j] > T[i] + 1) {
          if (T[i] < b->level) {
            ob *par = b->parent;
            for (int c = 0; c < 8; c++) T[par->child[c]->id] = par->child[c]->level;
          } else {
            T[i] = b->level + 1;
          }
          changed = 1;
        }
      }
    }
  }
  /* apply: refinements, then coarsenings (disjoint sets of blocks) */
  ob **old = malloc(sizeof(ob *) * n);
  memcpy(old, g->leaves, sizeof(ob *) * n);
  for (int i = 0; i < n; i++)
    if (T[i] == old[i]->level + 1) refine_block(g, old[i]);
  for (int i = 0; i < n; i++) {
    if (T[i] != old[i]->level - 1) continue;
    ob *par = old[i]->parent;
    if (par->is_leaf) continue; /* family already coarsened */
    if (old[i] != par->child[0]) continue;
    coarsen_block(g, par);
  }
  for (int i = 0; i < n; i++) free(lists[i]);
  free(lists);
  free(cnt);
  free(nbr);
  free(old);
  free(T);
  rebuild_leaves(g);
}

/* ------------------------------------------------------------------ */
/* creation, state I/O, probe, sums                                    */
/* ------------------------------------------------------------------ */
or_grid *or_create(const or_params *p) {
  or_grid *g = calloc(1, sizeof(or_grid));
  g->p = *p;
  for (int d = 0; d < 3; d++) {
    if (p->n[d] % p->nb[d]) {
      free(g);
      return NULL;
    }
    g->nbase[d] = p->n[d] / p->nb[d];
  }
  build_faces(g);
  build_offsets(g);
  int nb = g->nbase[0] * g->nbase[1] * g->nbase[2];
  g->base = calloc(nb, sizeof(ob));
  for (int a = 0; a < g->nbase[0]; a++)
    for (int b = 0; b < g->nbase[1]; b++)
      for (int c = 0; c < g->nbase[2]; c++) {
        ob *o = &g->base[(a * g->nbase[1] + b) * g->nbase[2] + c];
        o->level = 1;
        o->ix[0] = a;
        o->ix[1] = b;
        o->ix[2] = c;
        o->is_leaf = 1;
        alloc_block_data(g, o);
      }
  g->map = calloc((size_t)NV * p->n[1] * p->n[2], sizeof(double));
  rebuild_leaves(g);
  return g;
}

static void free_tree(ob *b, int top) {
  if (!b->is_leaf)
    for (int c = 0; c < 8; c++)
      if (b->child[c]) free_tree(b->child[c], 0);
  free_block_data(b);
  if (!top) free(b);
}

void or_destroy(or_grid *g) {
  if (!g) return;
  int nb = g->nbase[0] * g->nbase[1] * g->nbase[2];
  for (int i = 0; i < nb; i++) free_tree(&g->base[i], 1);
  free(g->base);
  for (int d = 0; d < 3; d++)
    for (int L = 0; L <= OR_MAXL; L++) {
      free(g->xf[d][L]);
      free(g->dlt[d][L]);
    }
  free(g->map);
  free(g->vbg);
  free(g->leaves);
  free(g);
}

int or_nleaves(or_grid *g) { return g->nleaves; }
double or_time(or_grid *g) { return g->t; }
void or_set_time(or_grid *g, double t) { g->t = t; }
long or_floor_hits(or_grid *g) { return g->floor_hits; }
void or_set_threads(or_grid *g, int n) {
  g->nthreads = n;
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#endif
}
int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_get_tree(or_grid *g, int32_t *out) {
  for (int n = 0; n < g->nleaves; n++) {
    ob *b = g->leaves[n];
    out[4 * n] = b->level;
    out[4 * n + 1] = b->ix[0];
    out[4 * n + 2] = b->ix[1];
    out[4 * n + 3] = b->ix[2];
  }
}

size_t or_state_size(or_grid *g) {
  return (size_t)g->nleaves * NV * g->p.nb[0] * g->p.nb[1] * g->p.nb[2];
}

/* host layout [leaf (Morton)][v][i][j][k], interior cells only */
void or_set_state(or_grid *g, const double *in, int is_prim) {
  const int *nb = g->p.nb;
  size_t bc = (size_t)nb[0] * nb[1] * nb[2];
  for (int n = 0; n < g->nleaves; n++) {
    ob *b = g->leaves[n];
    const double *s = in + (size_t)n * NV * bc;
    for (int a = 0; a < nb[0]; a++)
      for (int c = 0; c < nb[1]; c++)
        for (int e = 0; e < nb[2]; e++) {
          size_t o = ((size_t)a * nb[1] + c) * nb[2] + e;
          double x[NV], u[NV];
          for (int v = 0; v < NV; v++) x[v] = s[v * bc + o];
          if (is_prim) or_prim2cons(x, u, g->p.gamma);
          else memcpy(u, x, sizeof(u));
          for (int v = 0; v < NV; v++) b->U[pidx(g, v, a + NG, c + NG, e + NG)] = u[v];
        }
  }
}

void or_get_state(or_grid *g, double *out) {
  const int *nb = g->p.nb;
  size_t bc = (size_t)nb[0] * nb[1] * nb[2];
  for (int n = 0; n < g->nleaves; n++) {
    ob *b = g->leaves[n];
    double *s = out + (size_t)n * NV * bc;
    for (int v = 0; v < NV; v++)
      for (int a = 0; a < nb[0]; a++)
        for (int c = 0; c < nb[1]; c++)
          for (int e = 0; e < nb[2]; e++)
            s[v * bc + ((size_t)a * nb[1] + c) * nb[2] + e] = b->U[pidx(g, v, a + NG, c + NG, e + NG)];
  }
}

/* padded block (with ghosts) of leaf n, buffer which, [v][i][j][k] */
void or_get_padded(or_grid *g, int n, int which, double *out) {
  memcpy(out, buf(g->leaves[n], which), sizeof(double) * or_pcells(g) * NV);
}

/* overwrite a leaf's padded block (ghost layers included) in buffer `which`;
 * lets a test run the estimator on data filled elsewhere */
void or_set_padded(or_grid *g, int n, int which, const double *in) {
  memcpy(buf(g->leaves[n], which), in, sizeof(double) * or_pcells(g) * NV);
}

void or_set_boundary_map(or_grid *g, const double *prim) {
  memcpy(g->map, prim, sizeof(double) * NV * g->p.n[1] * g->p.n[2]);
}

/* cme = {t_start, t_max, colat, lon, half_width, v, rho, p} */
void or_set_cme(or_grid *g, const double *c) {
  g->cme.t_start = c[0];
  g->cme.t_max = c[1];
  g->cme.colat = c[2];
  g->cme.lon = c[3];
  g->cme.half_width = c[4];
  g->cme.v = c[5];
  g->cme.rho = c[6];
  g->cme.p = c[7];
  g->cme.active = 1;
}

/* background radial speed per base cell, taken from the current state; all
 * leaves must be at the base level (nothing refines before the CME). */
int or_snapshot_vbg(or_grid *g) {
  const int *nb = g->p.nb;
  size_t n = (size_t)g->p.n[0] * g->p.n[1] * g->p.n[2];
  free(g->vbg);
  g->vbg = malloc(sizeof(double) * n);
  for (int l = 0; l < g->nleaves; l++) {
    ob *b = g->leaves[l];
    if (b->level != 1) return -1;
    for (int a = 0; a < nb[0]; a++)
      for (int c = 0; c < nb[1]; c++)
        for (int e = 0; e < nb[2]; e++) {
          int I = b->ix[0] * nb[0] + a, J = b->ix[1] * nb[1] + c, K = b->ix[2] * nb[2] + e;
          g->vbg[((size_t)I * g->p.n[1] + J) * g->p.n[2] + K] =
              b->U[pidx(g, MR, a + NG, c + NG, e + NG)] / b->U[pidx(g, RHO, a + NG, c + NG, e + NG)];
        }
  }
  return 0;
}

void or_set_vbg(or_grid *g, const double *v) {
  size_t n = (size_t)g->p.n[0] * g->p.n[1] * g->p.n[2];
  free(g->vbg);
  g->vbg = malloc(sizeof(double) * n);
  memcpy(g->vbg, v, sizeof(double) * n);
}

/* Probe (reading R15): trilinear interpolation of the primitives between the
 * cell centres of the finest leaf containing the point. */
void or_probe(or_grid *g, int npts, const double *x, double *out) {
  or_ghost_fill(g, 0, g->t);
  int L = g->p.max_level;
  for (int n = 0; n < npts; n++) {
    double p[3] = {x[3 * n], x[3 * n + 1], x[3 * n + 2]};
    if (g->p.bc_lo[2] == BC_PERIODIC) {
      double span = g->p.xmax[2] - g->p.xmin[2];
      p[2] = g->p.xmin[2] + fmod(fmod(p[2] - g->p.xmin[2], span) + span, span);
    }
    int I[3], bad = 0;
    for (int d = 0; d < 3; d++) {
      int N = or_ncells(g, L, d);
      if (p[d] < or_face(g, L, d, 0) || p[d] >= or_face(g, L, d, N)) bad = 1;
      int lo = 0, hi = N;
      while (hi - lo > 1) {
        int m = (lo + hi) / 2;
        if (or_face(g, L, d, m) <= p[d]) lo = m;
        else hi = m;
      }
      I[d] = lo;
    }
    if (bad) {
      for (int v = 0; v < NV; v++) out[n * NV + v] = NAN;
      continue;
    }
    int lev;
    ob *b = find_cover(g, L, I[0], I[1], I[2], &lev);
    int q[3];
    double w[3];
    for (int d = 0; d < 3; d++) {
      int P = or_pdim(g, d), g0 = b->ix[d] * g->p.nb[d] - NG;
      int k = 0;
      for (int s = 0; s < P - 1; s++)
        if (or_centre(g, lev, d, g0 + s) <= p[d]) k = s;
      if (k > P - 2) k = P - 2;
      double c0 = or_centre(g, lev, d, g0 + k), c1 = or_centre(g, lev, d, g0 + k + 1);
      q[d] = k;
      w[d] = (p[d] - c0) / (c1 - c0);
    }
    double acc[NV] = {0};
    for (int a = 0; a < 2; a++)
      for (int c = 0; c < 2; c++)
        for (int e = 0; e < 2; e++) {
          double u[NV], W[NV];
          for (int v = 0; v < NV; v++) u[v] = b->U[pidx(g, v, q[0] + a, q[1] + c, q[2] + e)];
          or_cons2prim(u, W, g->p.gamma);
          double wt = (a ? w[0] : 1.0 - w[0]) * (c ? w[1] : 1.0 - w[1]) * (e ? w[2] : 1.0 - w[2]);
          for (int v = 0; v < NV; v++) acc[v] += wt * W[v];
        }
    for (int v = 0; v < NV; v++) out[n * NV + v] = acc[v];
  }
}

/* conservation sums sum_cells V U over all leaves */
void or_sums(or_grid *g, double *out) {
  const int *nb = g->p.nb;
  for (int v = 0; v < NV; v++) out[v] = 0.0;
  for (int n = 0; n < g->nleaves; n++) {
    ob *b = g->leaves[n];
    for (int a = 0; a < nb[0]; a++)
      for (int c = 0; c < nb[1]; c++)
        for (int e = 0; e < nb[2]; e++) {
          int I = b->ix[0] * nb[0] + a, J = b->ix[1] * nb[1] + c, K = b->ix[2] * nb[2] + e;
          double V = cell_volume(g, b->level, I, J, K);
          for (int v = 0; v < NV; v++) out[v] += V * b->U[pidx(g, v, a + NG, c + NG, e + NG)];
        }
  }
}

/* total volume of the leaves (a geometry check) */
double or_total_volume(or_grid *g) {
  const int *nb = g->p.nb;
  double s = 0.0;
  for (int n = 0; n < g->nleaves; n++) {
    ob *b = g->leaves[n];
    for (int a = 0; a < nb[0]; a++)
      for (int c = 0; c < nb[1]; c++)
        for (int e = 0; e < nb[2]; e++)
          s += cell_volume(g, b->level, b->ix[0] * nb[0] + a, b->ix[1] * nb[1] + c, b->ix[2] * nb[2] + e);
  }
  return s;
}

/* faces of level L along d, N+1 values */
void or_get_faces(or_grid *g, int L, int d, double *out) {
  int N = or_ncells(g, L, d);
  for (int I = 0; I <= N; I++) out[I] = or_face(g, L, d, I);
}

/* prolongation offsets of level L along d: [N][2] */
void or_get_offsets(or_grid *g, int L, int d, double *out) {
  int N = or_ncells(g, L, d);
  memcpy(out, g->dlt[d][L], sizeof(double) * 2 * N);
}

/* one isolated stage on every leaf, for unit checks: which=0 computes
 * Us = U + dtf L(U) after ghost fill at time t. */
void or_stage_only(or_grid *g, double dtf, double t) {
  or_ghost_fill(g, 0, t);
  for (int n = 0; n < g->nleaves; n++) stage_block(g, g->leaves[n], 0, dtf, 0, 0);
}

void or_get_stage_state(or_grid *g, double *out) {
  const int *nb = g->p.nb;
  size_t bc = (size_t)nb[0] * nb[1] * nb[2];
  for (int n = 0; n < g->nleaves; n++) {
    ob *b = g->leaves[n];
    double *s = out + (size_t)n * NV * bc;
    for (int v = 0; v < NV; v++)
      for (int a = 0; a < nb[0]; a++)
        for (int c = 0; c < nb[1]; c++)
          for (int e = 0; e < nb[2]; e++)
            s[v * bc + ((size_t)a * nb[1] + c) * nb[2] + e] = b->Us[pidx(g, v, a + NG, c + NG, e + NG)];
  }
}

/* check of the 2:1 rule over faces, edges and corners: returns the number of
 * offending leaf pairs (brute force over the neighbour shell). */
int or_balance_violations(or_grid *g) {
  int bad = 0, cap = 4096;
  ob **nbr = malloc(sizeof(ob *) * cap);
  for (int n = 0; n < g->nleaves; n++) {
    int m = leaf_neighbours(g, g->leaves[n], nbr, cap);
    for (int k = 0; k < m; k++) {
      int dl = nbr[k]->level - g->leaves[n]->level;
      if (dl > 1 || dl < -1) bad++;
    }
  }
  free(nbr);
  return bad;
}
