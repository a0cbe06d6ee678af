// libicarus host runtime: the C ABI of include/icarus.h.
//
// Owns the small host-side bookkeeping of a context: the layout of the
// caller's device arena, the per-level geometry tables (stretched radial
// faces, Sect. 2.2 of arXiv 2211.12867), the leaf lists of every ensemble
// member (block AMR of Sect. 3: factor 2 per level, neighbours within one
// level), the regrid decision (2:1 balance over faces, edges and corners as
// the least balanced refinement), the per-step launch sequence and its CUDA
// graph.  All arithmetic on the state happens in the kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/icarus.h"
#include "icarus_internal.h"

namespace {

constexpr size_t ALIGN = 256;
constexpr int MLP_CAP = 65536;   // training samples held on the device
constexpr int MLP_BMAX = 4096;   // largest batch

struct Leaf {
  int level;
  int ix[3];
};

struct Member {
  int max_level = 1;
  std::vector<Leaf> leaves;            // Morton order
  std::vector<std::vector<int>> map;   // per level: leaf index, -1 none/coarser, -2 refined
  DevCme cme{};
};

struct Region {
  size_t off = 0, bytes = 0;
};

struct Layout {
  size_t total = 0;
  Region geo, tables, blk, blk_alt, nb27, U, Us, Ualt, flux, lmap, lmap_off, bmap, cme, earth, vbg, scal, flags, lists,
      rent, sides, rlist, ops, shell, rshell, staging, partial, probe_in, probe_out, mlp_par, mlp_feat, mlp_X, mlp_T, mlp_idx,
      mlp_act, mlp_xin;
  size_t staging_doubles = 0, table_doubles = 0;
  int max_blocks = 0, nshell = 0;   // nshell: ghost cells of a padded block
  long long lmap_ints = 0;
  Region add(size_t b) {
    Region r;
    r.off = total;
    r.bytes = b;
    total += (b + ALIGN - 1) / ALIGN * ALIGN;
    return r;
  }
};

int nbase_total(const icarus_grid_desc *d) {
  return (d->n_cells[0] / d->block[0]) * (d->n_cells[1] / d->block[1]) * (d->n_cells[2] / d->block[2]);
}

long long blocks_at_level(const icarus_grid_desc *d, int L) {
  return (long long)nbase_total(d) << (3 * (L - 1));
}

// per level: r faces (N+2G+1) + 5 r cell tables (N+2G) + theta faces + 6
// theta cell tables + phi faces + phi centres; then prolongation offsets
size_t table_count(const icarus_grid_desc *d) {
  size_t n = 0;
  for (int L = 1; L <= d->max_level; L++) {
    const size_t N0 = (size_t)d->n_cells[0] << (L - 1), N1 = (size_t)d->n_cells[1] << (L - 1),
                 N2 = (size_t)d->n_cells[2] << (L - 1);
    n += 2 * (N0 + 2 * NGH + 1) + 4 * (N0 + 2 * NGH);  // rf, r2f | dr3, dr2, rc, dr
    n += 2 * (N1 + 2 * NGH + 1) + 5 * (N1 + 2 * NGH);  // tf, sinf | dcos, tc, sintc, costc, dth
    n += (N2 + 2 * NGH + 1) + (N2 + 2 * NGH);          // pf | pc
    if (L < d->max_level) n += 2 * (N0 + N1 + N2);     // offsets
  }
  return n;
}

// ghost-fill work items a leaf can need at most: 32-task chunks of the ghost
// cells of its 26 regions (all of them held by finer leaves)
int items_per_block(const icarus_grid_desc *d) {
  const int n0 = d->block[0], n1 = d->block[1], n2 = d->block[2];
  auto chunks = [](int cells) { return (cells + 31) / 32; };
  return 2 * (chunks(NGH * n1 * n2) + chunks(NGH * n0 * n2) + chunks(NGH * n0 * n1)) +
         4 * (chunks(NGH * NGH * n0) + chunks(NGH * NGH * n1) + chunks(NGH * NGH * n2)) + 8 * chunks(NGH * NGH * NGH);
}

int shell_count(const icarus_grid_desc *d) {
  const int P = (d->block[0] + 2 * NGH) * (d->block[1] + 2 * NGH) * (d->block[2] + 2 * NGH);
  return P - d->block[0] * d->block[1] * d->block[2];
}

icarus_status validate(const icarus_grid_desc *d) {
  if (!d) return ICARUS_ERR_ARG;
  if (d->max_level < 1 || d->max_level > MAXLEV) return ICARUS_ERR_ARG;
  if (d->n_members < 1 || d->n_members > 4096) return ICARUS_ERR_ARG;
  if (d->precision != ICARUS_FP64 && d->precision != ICARUS_FP32_MIXED) return ICARUS_ERR_ARG;
  if (d->tracer != 0 && d->tracer != 1) return ICARUS_ERR_ARG;
  if (d->geometry != ICARUS_SPHERICAL && d->geometry != ICARUS_CARTESIAN) return ICARUS_ERR_ARG;
  for (int k = 0; k < 3; k++) {
    if (d->block[k] < 4 || d->block[k] % 2 || d->block[k] + 2 * NGH > 1024) return ICARUS_ERR_ARG;
    if (d->n_cells[k] < d->block[k] || d->n_cells[k] % d->block[k]) return ICARUS_ERR_ARG;
    if (!(d->x_max[k] > d->x_min[k])) return ICARUS_ERR_ARG;
    if ((d->bc_lo[k] == ICARUS_BC_PERIODIC) != (d->bc_hi[k] == ICARUS_BC_PERIODIC)) return ICARUS_ERR_ARG;
    if (d->bc_lo[k] < 0 || d->bc_lo[k] > 3 || d->bc_hi[k] < 0 || d->bc_hi[k] > 3) return ICARUS_ERR_ARG;
    if (k > 0 && d->bc_lo[k] == ICARUS_BC_INNER) return ICARUS_ERR_ARG;
    if (d->bc_hi[k] == ICARUS_BC_INNER) return ICARUS_ERR_ARG;
    if (((long long)d->n_cells[k] << (d->max_level - 1)) > (1 << 20)) return ICARUS_ERR_ARG;
  }
  if (d->radial_stretch && !(d->x_min[0] > 0.0)) return ICARUS_ERR_ARG;
  if (d->geometry == ICARUS_SPHERICAL && !(d->x_min[1] > 0.0 && d->x_max[1] < M_PI)) return ICARUS_ERR_ARG;
  if (!(d->gamma > 1.0) || !(d->cfl > 0.0) || d->divb_cd < 0.0) return ICARUS_ERR_ARG;
  if (d->max_blocks < 0) return ICARUS_ERR_ARG;
  return ICARUS_OK;
}

Layout make_layout(const icarus_grid_desc *d) {
  Layout L;
  const int nm = d->n_members;
  const int base = nbase_total(d) * nm;
  L.max_blocks = d->max_blocks > 0 ? std::max(d->max_blocks, base) : base;
  const size_t mb = L.max_blocks;
  const size_t rs = d->precision == ICARUS_FP64 ? 8 : 4;
  const size_t pc = (size_t)(d->block[0] + 2 * NGH) * (d->block[1] + 2 * NGH) * (d->block[2] + 2 * NGH);
  const size_t ic = (size_t)d->block[0] * d->block[1] * d->block[2];
  const bool amr = d->max_level > 1;
  L.table_doubles = table_count(d);
  L.geo = L.add(sizeof(Geometry));
  L.tables = L.add(L.table_doubles * (8 + 4));
  L.blk = L.add(mb * sizeof(DevBlock));
  L.blk_alt = L.add(amr ? mb * sizeof(DevBlock) : 0);
  L.nb27 = L.add(mb * 27 * sizeof(int));
  const size_t nvs = NVAR + (d->tracer ? 1 : 0);   // variables stored per cell
  L.U = L.add(mb * nvs * pc * rs);
  L.Us = L.add(mb * nvs * pc * rs);
  L.Ualt = L.add(amr ? mb * nvs * pc * rs : 0);
  const size_t fcells = 2 * ((size_t)d->block[1] * d->block[2] + (size_t)d->block[0] * d->block[2] +
                             (size_t)d->block[0] * d->block[1]);
  L.flux = L.add(amr ? mb * NVAR * fcells * rs : 0);
  long long li = 0;
  for (int Lv = 1; Lv <= d->max_level; Lv++) li += blocks_at_level(d, Lv);
  L.lmap_ints = li * nm;
  L.lmap = L.add((size_t)L.lmap_ints * sizeof(int));
  L.lmap_off = L.add((size_t)nm * (MAXLEV + 1) * sizeof(long long));
  L.bmap = L.add((size_t)nm * NVAR * d->n_cells[1] * d->n_cells[2] * sizeof(double));
  L.cme = L.add((size_t)nm * sizeof(DevCme));
  L.earth = L.add((size_t)nm * sizeof(DevEarth));
  L.vbg = L.add((size_t)nm * d->n_cells[0] * d->n_cells[1] * d->n_cells[2] * sizeof(double));
  L.scal = L.add((size_t)nm * 7 * sizeof(double) + 64);
  L.flags = L.add(mb);
  L.lists = L.add(2 * mb * sizeof(int));        // all-leaf list + per-level lists
  L.rent = L.add((size_t)items_per_block(d) * mb * sizeof(int2));   // per level: ghost-fill work items
  L.sides = L.add(6 * mb * sizeof(int2));       // (slot, side) per level, per direction
  L.rlist = L.add(mb * sizeof(int));
  L.ops = L.add(amr ? mb * sizeof(MoveOp) : 0);
  L.nshell = shell_count(d);
  L.shell = L.add((size_t)L.nshell * sizeof(int));
  L.rshell = L.add((size_t)(81 + L.nshell) * sizeof(int));   // region table, then the shell cells by region
  const size_t per_block = NVAR * ic;
  size_t chunk = std::max<size_t>(1, (size_t)(64u << 20) / (per_block * 8));
  chunk = std::min(chunk, mb);
  L.staging_doubles = chunk * per_block;
  L.staging = L.add(L.staging_doubles * sizeof(double));
  L.partial = L.add(mb * NVAR * sizeof(double));
  L.probe_in = L.add(4096 * 3 * sizeof(double));
  L.probe_out = L.add(4096 * NVAR * sizeof(double));
  // learned pre-flagger: parameters, gradient and Adam moments (4 x n), leaf
  // features and probabilities, training set, batch activations
  L.mlp_par = L.add((size_t)4 * mlp_n_params() * sizeof(float) + 64);
  L.mlp_feat = L.add(mb * (64 + 1) * sizeof(float));
  L.mlp_X = L.add((size_t)MLP_CAP * 64 * sizeof(float));
  L.mlp_T = L.add((size_t)MLP_CAP * sizeof(float));
  L.mlp_idx = L.add((size_t)MLP_CAP * sizeof(int));
  L.mlp_act = L.add((size_t)MLP_BMAX * (4 * 128 + 2) * sizeof(float));
  L.mlp_xin = L.add((size_t)MLP_BMAX * 65 * sizeof(float));
  return L;
}

// 8-point Gauss-Legendre rule on [-1, 1] (Newton iteration on P_8)
void gauss_legendre(double *x, double *w) {
  const int n = 8;
  for (int i = 0; i < n; i++) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; it++) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; k++) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; k++) {
      double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

}  // namespace

struct icarus_ctx {
  icarus_grid_desc d{};
  int nbd[MAXLEV + 2][3] = {};   // blocks per direction at each level (tree logic looks these up)
  Layout lay;
  int prec = 0;
  size_t rsize = 8;
  cudaStream_t stream = nullptr;
  char *arena = nullptr;
  int nsm = 1;
  int dev = 0;   // CUDA device current when the context was created
  // device pointers
  Geometry *geo = nullptr;
  DevBlock *blk = nullptr, *blk_alt = nullptr;
  int *nb27 = nullptr;
  void *U = nullptr, *Us = nullptr, *Ualt = nullptr, *flux = nullptr;
  int *lmap = nullptr;
  long long *lmap_off = nullptr;
  double *bmap = nullptr, *vbg = nullptr, *staging = nullptr, *partial = nullptr, *probe_in = nullptr,
         *probe_out = nullptr;
  DevCme *cme = nullptr;
  DevEarth *earth = nullptr;
  double *t = nullptr, *dt_used = nullptr, *dt_cfl = nullptr, *tstop = nullptr, *updates = nullptr,
         *cells_m = nullptr;
  unsigned long long *inv_max = nullptr, *floor_hits = nullptr, *floor_prev = nullptr;
  unsigned int *status = nullptr;
  signed char *flags = nullptr;
  int *all_list = nullptr, *lvl_list = nullptr, *rlist = nullptr, *shell = nullptr;
  int2 *rent = nullptr;     // per level: (slot, region | finer << 8 | chunk << 9), up to 32 ghost tasks of a region held by coarser / finer leaves
  int *rshell = nullptr;    // per region (start, group-first cells, cells), then the shell cells ordered by region
  int2 *sides = nullptr;
  MoveOp *ops = nullptr;
  // host mirrors
  std::vector<Member> mem;
  int nleaves = 0;
  std::vector<int> mem_off;                 // first slot of each member
  std::vector<DevBlock> hblk;
  int lvl_count[MAXLEV + 1] = {0}, lvl_start[MAXLEV + 1] = {0};
  int rent_start[MAXLEV + 1] = {0}, rent_face[MAXLEV + 1] = {0}, rent_count[MAXLEV + 1] = {0};
  int reg_tab[27][3] = {};  // per region: start in the region-ordered shell, group-first cells, cells
  int side_count[MAXLEV + 1][3] = {{0}}, side_start[MAXLEV + 1][3] = {{0}};
  int nrlist = 0, max_level_present = 1;
  std::vector<signed char> hflags;
  bool flags_valid = false;
  KParams kp{};
  // launch configuration
  int tile_j = 0, tile_k = 0, seg_len = 0, occ = 1;
  double isl_pe = 0.002, isl_beta = 0.1;  // FP64 pressure islands: p < 0.002 e or beta < 0.1
  double floor_budget = ICARUS_DEFAULT_FLOOR_BUDGET;
  // status word read back without a synchronisation after steps that return
  // no times (pinned host word, event of its copy)
  unsigned int *h_status = nullptr;
  cudaEvent_t status_ev = nullptr;
  bool status_pending = false;
  bool use_graph = true;
  cudaGraphExec_t graph = nullptr;
  bool graph_valid = false;
  bool poisoned = false;
  bool ghosts_fresh = false;   // ghosts of U filled for the current state and time
  int nshell_face = 0;         // ghost cells outside the block in one direction (first in the shell list)
  bool direct_halo = true;     // stage kernels read same-level halos from the neighbours themselves
  std::vector<double> h_tstop;
  int kernels_per_step = 0;
  // learned pre-flagger
  float *mlp_theta = nullptr, *mlp_grad = nullptr, *mlp_m = nullptr, *mlp_v = nullptr, *mlp_loss = nullptr;
  float *mlp_feat = nullptr, *mlp_prob = nullptr, *mlp_X = nullptr, *mlp_T = nullptr, *mlp_h1 = nullptr,
        *mlp_h2 = nullptr, *mlp_dh2 = nullptr, *mlp_dh1 = nullptr, *mlp_y = nullptr, *mlp_dz = nullptr,
        *mlp_xin = nullptr, *mlp_tin = nullptr;
  int *mlp_idx = nullptr;
  int mlp_n = 0, mlp_step = 0;
  bool mlp_ready = false;
  // per-launch profiling
  bool prof_on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_kind;   // kind of each event pair
  size_t ev_used = 0;         // events recorded since the last read
};

namespace {

#define CK(x)                                                                     \
  do {                                                                            \
    cudaError_t e_ = (x);                                                         \
    if (e_ != cudaSuccess) {                                                      \
      fprintf(stderr, "libicarus: %s failed: %s\n", #x, cudaGetErrorString(e_)); \
      return ICARUS_ERR_CUDA;                                                     \
    }                                                                             \
  } while (0)

template <typename T>
T *at(icarus_ctx *c, const Region &r) {
  return reinterpret_cast<T *>(c->arena + r.off);
}

uint64_t morton_key(const Leaf &l, int shift_to) {
  uint64_t key = 0;
  const int s = shift_to - l.level;
  uint64_t x[3];
  for (int d = 0; d < 3; d++) x[d] = (uint64_t)l.ix[d] << s;
  for (int bit = 20; bit >= 0; bit--)
    for (int d = 0; d < 3; d++) key = (key << 1) | ((x[d] >> bit) & 1u);
  return key;
}

int nblk_dim(const icarus_ctx *c, int L, int d) { return c->nbd[L][d]; }

long long map_index(const icarus_ctx *c, int L, const int *b) {
  return ((long long)b[0] * nblk_dim(c, L, 1) + b[1]) * nblk_dim(c, L, 2) + b[2];
}

// wrap a block index of level L; false if outside a non-periodic direction
bool wrap_block(const icarus_ctx *c, int L, int *b) {
  for (int d = 0; d < 3; d++) {
    const int n = nblk_dim(c, L, d);
    if (c->d.bc_lo[d] == ICARUS_BC_PERIODIC) {
      if (b[d] < 0) b[d] += n;
      else if (b[d] >= n) b[d] -= n;
      if (b[d] < 0 || b[d] >= n) b[d] = ((b[d] % n) + n) % n;
    } else if (b[d] < 0 || b[d] >= n) {
      return false;
    }
  }
  return true;
}

// Level maps of a member: leaf index, -2 (refined) or -1 (covered by a
// coarser leaf).  Returns false if two leaves overlap (a leaf lies inside
// another one or appears twice); the maps are then incomplete.
bool build_member_map(icarus_ctx *c, Member &m) {
  m.map.assign(c->d.max_level + 1, std::vector<int>());
  for (int L = 1; L <= c->d.max_level; L++) m.map[L].assign((size_t)blocks_at_level(&c->d, L), -1);
  bool ok = true;
  for (size_t n = 0; n < m.leaves.size(); n++) {
    const Leaf &l = m.leaves[n];
    int &own = m.map[l.level][map_index(c, l.level, l.ix)];
    if (own != -1) ok = false;   // a duplicate, or an ancestor of a finer leaf
    own = (int)n;
    int b[3] = {l.ix[0], l.ix[1], l.ix[2]};
    for (int L = l.level - 1; L >= 1; L--) {
      for (int d = 0; d < 3; d++) b[d] >>= 1;
      int &e = m.map[L][map_index(c, L, b)];
      if (e >= 0) ok = false;    // inside a coarser leaf
      e = -2;
    }
  }
  return ok;
}

// relation of the region (level L, block index b) to the leaves: the leaf
// index, -2 refined, -1 covered by a coarser leaf
int region_state(const icarus_ctx *c, const Member &m, int L, const int *b) { return m.map[L][map_index(c, L, b)]; }

// adjacent leaves of a leaf at most: 4 finer leaves per face, 2 per edge, 1
// per corner
constexpr int NB_MAX = 6 * 4 + 12 * 2 + 8;

// adjacent leaves of leaf n (faces, edges, corners)
void neighbours(const icarus_ctx *c, const Member &m, int n, std::vector<int> &out) {
  out.clear();
  const Leaf &l = m.leaves[n];
  const int L = l.level;
  for (int dx = -1; dx <= 1; dx++)
    for (int dy = -1; dy <= 1; dy++)
      for (int dz = -1; dz <= 1; dz++) {
        if (!dx && !dy && !dz) continue;
        const int dir[3] = {dx, dy, dz};
        int b[3] = {l.ix[0] + dx, l.ix[1] + dy, l.ix[2] + dz};
        if (!wrap_block(c, L, b)) continue;
        const int s = region_state(c, m, L, b);
        if (s >= 0) {
          out.push_back(s);
        } else if (s == -2) {
          if (L + 1 > c->d.max_level) continue;
          for (int ch = 0; ch < 8; ch++) {
            const int o[3] = {(ch >> 2) & 1, (ch >> 1) & 1, ch & 1};
            bool touch = true;
            for (int d = 0; d < 3; d++) {
              if (dir[d] == 1 && o[d] != 0) touch = false;
              if (dir[d] == -1 && o[d] != 1) touch = false;
            }
            if (!touch) continue;
            int cb[3];
            for (int d = 0; d < 3; d++) cb[d] = 2 * b[d] + o[d];
            const int cs = region_state(c, m, L + 1, cb);
            if (cs >= 0) out.push_back(cs);
          }
        } else {
          int pb[3] = {b[0] >> 1, b[1] >> 1, b[2] >> 1};
          if (L > 1) {
            const int ps = region_state(c, m, L - 1, pb);
            if (ps >= 0) out.push_back(ps);
          }
        }
      }
  std::sort(out.begin(), out.end());
  out.erase(std::unique(out.begin(), out.end()), out.end());
}

// A leaf list read from outside (a checkpoint) must be a tree this library
// could have built: leaves in strictly increasing Morton order, no overlap,
// the whole domain covered, and adjacent leaves (faces, edges, corners) at
// most one level apart.
bool tree_is_valid(icarus_ctx *c, Member &m) {
  const int top = c->d.max_level;
  const long long nl = (long long)m.leaves.size();
  std::vector<uint64_t> key(nl);
#pragma omp parallel for schedule(static)
  for (long long n = 0; n < nl; n++) key[n] = morton_key(m.leaves[n], top);
  for (long long n = 1; n < nl; n++)
    if (!(key[n - 1] < key[n])) return false;
  if (!build_member_map(c, m)) return false;
  // coverage, counted in blocks of the finest level
  unsigned long long vol = 0;
  for (const Leaf &l : m.leaves) vol += 1ull << (3 * (top - l.level));
  if (vol != (unsigned long long)blocks_at_level(&c->d, top)) return false;
  // 2:1 balance: no neighbour region two levels coarser or finer (leaves
  // checked in parallel; the maps are only read)
  auto balanced = [&](const Leaf &l) {
    const int L = l.level;
    for (int dx = -1; dx <= 1; dx++)
      for (int dy = -1; dy <= 1; dy++)
        for (int dz = -1; dz <= 1; dz++) {
          if (!dx && !dy && !dz) continue;
          int b[3] = {l.ix[0] + dx, l.ix[1] + dy, l.ix[2] + dz};
          if (!wrap_block(c, L, b)) continue;
          const int s = region_state(c, m, L, b);
          if (s == -1) {   // covered by a coarser leaf: it must be the parent level's
            if (L < 2) return false;
            int pb[3] = {b[0] >> 1, b[1] >> 1, b[2] >> 1};
            if (region_state(c, m, L - 1, pb) < 0) return false;
          } else if (s == -2) {   // refined: the children touching leaf l must be leaves
            const int dir[3] = {dx, dy, dz};
            for (int ch = 0; ch < 8; ch++) {
              const int o[3] = {(ch >> 2) & 1, (ch >> 1) & 1, ch & 1};
              bool touch = true;
              for (int d = 0; d < 3; d++) {
                if (dir[d] == 1 && o[d] != 0) touch = false;
                if (dir[d] == -1 && o[d] != 1) touch = false;
              }
              if (!touch || L + 1 > top) continue;
              int cb[3];
              for (int d = 0; d < 3; d++) cb[d] = 2 * b[d] + o[d];
              if (region_state(c, m, L + 1, cb) < 0) return false;
            }
          }
        }
    return true;
  };
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (long long n = 0; n < nl; n++)
    if (!balanced(m.leaves[n])) bad = 1;
  return bad == 0;
}

// device tables that depend on the leaf lists
icarus_status upload_tree(icarus_ctx *c, DevBlock *blk_dst) {
  const icarus_grid_desc &d = c->d;
  c->nleaves = 0;
  c->mem_off.assign(d.n_members, 0);
  for (int m = 0; m < d.n_members; m++) {
    c->mem_off[m] = c->nleaves;
    c->nleaves += (int)c->mem[m].leaves.size();
  }
  if (c->nleaves > c->lay.max_blocks) return ICARUS_ERR_CAPACITY;
  c->hblk.assign(c->nleaves, DevBlock{});
  std::vector<int> nb27((size_t)c->nleaves * 27, -1);
  std::vector<int> all(c->nleaves);
  std::vector<std::vector<int>> per_level(MAXLEV + 1);
  std::vector<std::vector<int2>> ent_face(MAXLEV + 1), ent_rest(MAXLEV + 1);
  std::vector<std::vector<int2>> sd[3];
  for (int k = 0; k < 3; k++) sd[k].assign(MAXLEV + 1, std::vector<int2>());
  std::vector<int> rl;
  c->max_level_present = 1;
  // the relation of each leaf to the 27 regions around it (0 outside a
  // non-periodic direction, 1 same-level leaf, 2 coarser, 3 finer) and the
  // same-level neighbours, found in parallel (the maps are only read)
  std::vector<unsigned char> rel((size_t)c->nleaves * 27, 0);
  for (int m = 0; m < d.n_members; m++) {
    const Member &M = c->mem[m];
    const long long nl = (long long)M.leaves.size();
#pragma omp parallel for schedule(static)
    for (long long n = 0; n < nl; n++) {
      const Leaf &l = M.leaves[n];
      const size_t slot = (size_t)c->mem_off[m] + n;
      for (int r = 0; r < 27; r++) {
        int b[3] = {l.ix[0] + r / 9 - 1, l.ix[1] + (r / 3) % 3 - 1, l.ix[2] + r % 3 - 1};
        if (!wrap_block(c, l.level, b)) continue;
        const int s = region_state(c, M, l.level, b);
        rel[slot * 27 + r] = s >= 0 ? 1 : (s == -2 ? 3 : 2);
        if (s >= 0) nb27[slot * 27 + r] = c->mem_off[m] + s;
      }
    }
  }
  for (int m = 0; m < d.n_members; m++) {
    const Member &M = c->mem[m];
    for (size_t n = 0; n < M.leaves.size(); n++) {
      const Leaf &l = M.leaves[n];
      const int slot = c->mem_off[m] + (int)n;
      const unsigned char *rs = rel.data() + (size_t)slot * 27;
      DevBlock &B = c->hblk[slot];
      B.member = m;
      B.level = l.level;
      B.lmax = M.max_level;
      for (int k = 0; k < 3; k++) B.ix[k] = l.ix[k];
      B.phys = 0;
      bool finer = false;
      for (int f = 0; f < 6; f++) {
        const int dd = f / 2, hi = f % 2;
        const int r = 13 + (hi ? 1 : -1) * (dd == 0 ? 9 : (dd == 1 ? 3 : 1));
        if (rs[r] == 0) {
          B.nbr[f] = NB_PHYS;
          B.phys |= 1 << f;
          sd[dd][l.level].push_back(make_int2(slot, hi));
          continue;
        }
        B.nbr[f] = rs[r] == 1 ? NB_SAME : (rs[r] == 3 ? NB_FINER : NB_COARSER);
        if (rs[r] == 3) finer = true;
      }
      if (finer) rl.push_back(slot);
      // the regions held by coarser or finer leaves go to the ghost fill's
      // work items of up to 32 tasks (2x2x2 groups under a coarser leaf,
      // cells next to finer ones), face regions first
      for (int r = 0; r < 27; r++) {
        if (rs[r] < 2) continue;
        const int dx = r / 9 - 1, dy = (r / 3) % 3 - 1, dz = r % 3 - 1;
        const bool face = (dx != 0) + (dy != 0) + (dz != 0) == 1, fin = rs[r] == 3;
        const int tasks = fin ? c->reg_tab[r][2] : c->reg_tab[r][1];
        for (int ch = 0; 32 * ch < tasks; ch++)
          (face ? ent_face : ent_rest)[l.level].push_back(make_int2(slot, r | (fin ? 256 : 0) | ch << 9));
      }
      all[slot] = slot;
      per_level[l.level].push_back(slot);
      c->max_level_present = std::max(c->max_level_present, l.level);
    }
  }
  // level maps (slot numbers)
  std::vector<int> lm((size_t)c->lay.lmap_ints, -1);
  std::vector<long long> off((size_t)d.n_members * (MAXLEV + 1), 0);
  long long o = 0;
  for (int m = 0; m < d.n_members; m++)
    for (int L = 1; L <= d.max_level; L++) {
      off[(size_t)m * (MAXLEV + 1) + L] = o;
      const std::vector<int> &mp = c->mem[m].map[L];
      for (size_t q = 0; q < mp.size(); q++) lm[o + q] = mp[q] >= 0 ? mp[q] + c->mem_off[m] : mp[q];
      o += (long long)mp.size();
    }
  std::vector<int> lv;
  std::vector<int2> ent;
  for (int L = 1; L <= MAXLEV; L++) {
    c->lvl_start[L] = (int)lv.size();
    c->lvl_count[L] = (int)per_level[L].size();
    lv.insert(lv.end(), per_level[L].begin(), per_level[L].end());
    c->rent_start[L] = (int)ent.size();
    c->rent_face[L] = (int)ent_face[L].size();
    c->rent_count[L] = (int)(ent_face[L].size() + ent_rest[L].size());
    ent.insert(ent.end(), ent_face[L].begin(), ent_face[L].end());
    ent.insert(ent.end(), ent_rest[L].begin(), ent_rest[L].end());
  }
  if (ent.size() > (size_t)items_per_block(&c->d) * c->lay.max_blocks) return ICARUS_ERR_CAPACITY;
  std::vector<int2> sv;
  for (int L = 1; L <= MAXLEV; L++)
    for (int k = 0; k < 3; k++) {
      c->side_start[L][k] = (int)sv.size();
      c->side_count[L][k] = (int)sd[k][L].size();
      sv.insert(sv.end(), sd[k][L].begin(), sd[k][L].end());
    }
  c->nrlist = (int)rl.size();
  {
    std::vector<double> cm(d.n_members);
    for (int m = 0; m < d.n_members; m++)
      cm[m] = (double)c->mem[m].leaves.size() * d.block[0] * d.block[1] * d.block[2];
    CK(cudaMemcpyAsync(c->cells_m, cm.data(), sizeof(double) * cm.size(), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  cudaStream_t s = c->stream;
  CK(cudaMemcpyAsync(blk_dst, c->hblk.data(), sizeof(DevBlock) * c->nleaves, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->nb27, nb27.data(), sizeof(int) * nb27.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->lmap, lm.data(), sizeof(int) * lm.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->lmap_off, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->all_list, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->lvl_list, lv.data(), sizeof(int) * lv.size(), cudaMemcpyHostToDevice, s));
  if (!ent.empty()) CK(cudaMemcpyAsync(c->rent, ent.data(), sizeof(int2) * ent.size(), cudaMemcpyHostToDevice, s));
  if (!sv.empty()) CK(cudaMemcpyAsync(c->sides, sv.data(), sizeof(int2) * sv.size(), cudaMemcpyHostToDevice, s));
  if (!rl.empty()) CK(cudaMemcpyAsync(c->rlist, rl.data(), sizeof(int) * rl.size(), cudaMemcpyHostToDevice, s));
  // host buffers above are freed on return: wait for the copies
  CK(cudaStreamSynchronize(s));
  c->graph_valid = false;
  c->flags_valid = false;
  return ICARUS_OK;
}

void fill_kp(icarus_ctx *c) {
  KParams &k = c->kp;
  const icarus_grid_desc &d = c->d;
  k.nvs = NVAR + (d.tracer ? 1 : 0);
  for (int i = 0; i < 3; i++) {
    k.nb[i] = d.block[i];
    k.P[i] = d.block[i] + 2 * NGH;
    k.nbase[i] = d.n_cells[i] / d.block[i];
    k.bc_lo[i] = d.bc_lo[i];
    k.bc_hi[i] = d.bc_hi[i];
    k.n_base_cells[i] = d.n_cells[i];
  }
  k.pcells = k.P[0] * k.P[1] * k.P[2];
  k.icells = k.nb[0] * k.nb[1] * k.nb[2];
  k.n_members = d.n_members;
  k.geometry = d.geometry;
  k.gamma = d.gamma;
  k.omega = d.omega;
  k.cd = d.divb_cd;
  k.p_floor = d.p_floor;
  k.rho_floor = d.rho_floor;
  k.isl_pe = c->isl_pe;
  k.isl_beta = c->isl_beta;
  k.geo = c->geo;
  k.blk = c->blk;
  k.nb27 = c->nb27;
  k.lmap = c->lmap;
  k.lmap_off = c->lmap_off;
  k.bmap = c->bmap;
  k.cme = c->cme;
  k.earth = c->earth;
  k.vbg = c->vbg;
  k.t = c->t;
  k.dt_used = c->dt_used;
  k.dt_cfl = c->dt_cfl;
  k.updates = c->updates;
  k.cells_m = c->cells_m;
  k.inv_max = c->inv_max;
  k.status = c->status;
  k.floor_hits = c->floor_hits;
  k.floor_prev = c->floor_prev;
  k.floor_budget = c->floor_budget;
}

// geometry tables of every level, FP64 and FP32 copies
icarus_status build_geometry(icarus_ctx *c) {
  const icarus_grid_desc &d = c->d;
  std::vector<double> hd;
  hd.reserve(c->lay.table_doubles);
  Geometry hg;
  memset(&hg, 0, sizeof(hg));
  double *dbase = at<double>(c, c->lay.tables);
  float *fbase = reinterpret_cast<float *>(dbase + c->lay.table_doubles);
  struct Rec {
    size_t off;
    int lev, which, dir;
  };
  std::vector<Rec> recs;
  auto push = [&](const std::vector<double> &v) {
    size_t o = hd.size();
    hd.insert(hd.end(), v.begin(), v.end());
    return o;
  };
  const bool sph = d.geometry == ICARUS_SPHERICAL;
  auto face = [&](int L, int dd, int I) {
    const int N = d.n_cells[dd] << (L - 1);
    const double x = (double)I / (double)N;
    if (dd == 0 && sph && d.radial_stretch) return d.x_min[0] * std::pow(d.x_max[0] / d.x_min[0], x);
    return d.x_min[dd] + (d.x_max[dd] - d.x_min[dd]) * x;
  };
  std::vector<size_t> offs[MAXLEV + 1];
  for (int L = 1; L <= d.max_level; L++) {
    const int N0 = d.n_cells[0] << (L - 1), N1 = d.n_cells[1] << (L - 1), N2 = d.n_cells[2] << (L - 1);
    std::vector<double> rf(N0 + 2 * NGH + 1), r2f(rf.size()), dr3(N0 + 2 * NGH), dr2(dr3.size()), rc(dr3.size()),
        dr(dr3.size());
    for (int I = -NGH; I <= N0 + NGH; I++) {
      rf[I + NGH] = face(L, 0, I);
      r2f[I + NGH] = sph ? rf[I + NGH] * rf[I + NGH] : 1.0;
    }
    for (int I = -NGH; I < N0 + NGH; I++) {
      const double a = rf[I + NGH], b = rf[I + NGH + 1];
      dr3[I + NGH] = sph ? (b * b * b - a * a * a) / 3.0 : b - a;
      dr2[I + NGH] = sph ? (b * b - a * a) / 2.0 : b - a;
      rc[I + NGH] = 0.5 * (a + b);
      dr[I + NGH] = b - a;
    }
    std::vector<double> tf(N1 + 2 * NGH + 1), sinf(tf.size()), dcos(N1 + 2 * NGH), tc(dcos.size()), sintc(dcos.size()),
        costc(dcos.size()), dth(dcos.size());
    for (int J = -NGH; J <= N1 + NGH; J++) {
      tf[J + NGH] = face(L, 1, J);
      sinf[J + NGH] = sph ? std::sin(tf[J + NGH]) : 1.0;
    }
    for (int J = -NGH; J < N1 + NGH; J++) {
      const double a = tf[J + NGH], b = tf[J + NGH + 1];
      dcos[J + NGH] = sph ? std::cos(a) - std::cos(b) : b - a;
      tc[J + NGH] = 0.5 * (a + b);
      sintc[J + NGH] = sph ? std::sin(tc[J + NGH]) : 1.0;
      costc[J + NGH] = sph ? std::cos(tc[J + NGH]) : 0.0;
      dth[J + NGH] = b - a;
    }
    std::vector<double> pf(N2 + 2 * NGH + 1), pcv(N2 + 2 * NGH);
    for (int K = -NGH; K <= N2 + NGH; K++) pf[K + NGH] = face(L, 2, K);
    for (int K = -NGH; K < N2 + NGH; K++) pcv[K + NGH] = 0.5 * (pf[K + NGH] + pf[K + NGH + 1]);
    const double dphi = (d.x_max[2] - d.x_min[2]) / N2;
    std::vector<size_t> &o = offs[L];
    o.push_back(push(rf));
    o.push_back(push(r2f));
    o.push_back(push(dr3));
    o.push_back(push(dr2));
    o.push_back(push(rc));
    o.push_back(push(dr));
    o.push_back(push(tf));
    o.push_back(push(sinf));
    o.push_back(push(dcos));
    o.push_back(push(tc));
    o.push_back(push(sintc));
    o.push_back(push(costc));
    o.push_back(push(dth));
    o.push_back(push(pf));
    o.push_back(push(pcv));
    hg.d[L].dphi = dphi;
    hg.f[L].dphi = (float)dphi;
    hg.d[L].n[0] = hg.f[L].n[0] = N0;
    hg.d[L].n[1] = hg.f[L].n[1] = N1;
    hg.d[L].n[2] = hg.f[L].n[2] = N2;
  }
  // prolongation offsets: child centroid minus parent centroid in the
  // parent's index coordinate, volume weighted (8-point Gauss-Legendre on
  // each child; exact for the polynomial weights)
  double gx[8], gw[8];
  gauss_legendre(gx, gw);
  for (int L = 1; L < d.max_level; L++) {
    for (int dd = 0; dd < 3; dd++) {
      const int N = d.n_cells[dd] << (L - 1);
      std::vector<double> t(2 * (size_t)N);
      const bool logr = sph && dd == 0 && d.radial_stretch;
      for (int I = 0; I < N; I++) {
        const double a = face(L, dd, I), b = face(L, dd, I + 1), m = face(L + 1, dd, 2 * I + 1);
        auto weight = [&](double x) {
          if (!sph || dd == 2) return 1.0;
          return dd == 0 ? x * x : std::sin(x);
        };
        auto xi = [&](double x) { return logr ? std::log(x / a) / std::log(b / a) - 0.5 : (x - a) / (b - a) - 0.5; };
        double M0[2], M1[2];
        for (int ch = 0; ch < 2; ch++) {
          const double lo = ch ? m : a, hi = ch ? b : m, h = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
          M0[ch] = M1[ch] = 0.0;
          for (int q = 0; q < 8; q++) {
            const double x = mid + h * gx[q];
            const double wv = gw[q] * h * weight(x);
            M0[ch] += wv;
            M1[ch] += wv * xi(x);
          }
        }
        const double xp = (M1[0] + M1[1]) / (M0[0] + M0[1]);
        t[2 * I] = M1[0] / M0[0] - xp;
        t[2 * I + 1] = M1[1] / M0[1] - xp;
      }
      offs[L].push_back(push(t));
    }
  }
  if (hd.size() != c->lay.table_doubles) {
    fprintf(stderr, "libicarus: geometry table size mismatch\n");
    return ICARUS_ERR_ARG;
  }
  std::vector<float> hf(hd.size());
  for (size_t i = 0; i < hd.size(); i++) hf[i] = (float)hd[i];
  for (int L = 1; L <= d.max_level; L++) {
    const std::vector<size_t> &o = offs[L];
    const double *b = dbase;
    const float *f = fbase;
    LevelGeo<double> &G = hg.d[L];
    LevelGeo<float> &F = hg.f[L];
    G.rf = b + o[0]; F.rf = f + o[0];
    G.r2f = b + o[1]; F.r2f = f + o[1];
    G.dr3 = b + o[2]; F.dr3 = f + o[2];
    G.dr2 = b + o[3]; F.dr2 = f + o[3];
    G.rc = b + o[4]; F.rc = f + o[4];
    G.dr = b + o[5]; F.dr = f + o[5];
    G.tf = b + o[6]; F.tf = f + o[6];
    G.sinf = b + o[7]; F.sinf = f + o[7];
    G.dcos = b + o[8]; F.dcos = f + o[8];
    G.tc = b + o[9]; F.tc = f + o[9];
    G.sintc = b + o[10]; F.sintc = f + o[10];
    G.costc = b + o[11]; F.costc = f + o[11];
    G.dth = b + o[12]; F.dth = f + o[12];
    G.pf = b + o[13]; F.pf = f + o[13];
    G.pc = b + o[14]; F.pc = f + o[14];
    if (L < d.max_level)
      for (int dd = 0; dd < 3; dd++) {
        hg.dlt[L][dd] = b + o[15 + dd];
        hg.dltf[L][dd] = f + o[15 + dd];
      }
  }
  CK(cudaMemcpyAsync(dbase, hd.data(), sizeof(double) * hd.size(), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(fbase, hf.data(), sizeof(float) * hf.size(), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->geo, &hg, sizeof(Geometry), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return ICARUS_OK;
}

// ---- launch sequence ----
void prof_mark(icarus_ctx *c, int kind, int end) {
  if (c->ev_used >= c->ev.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    c->ev.push_back(e);
  }
  if (!end) {
    if (c->ev_used / 2 >= c->ev_kind.size()) c->ev_kind.resize(c->ev_used / 2 + 1);
    c->ev_kind[c->ev_used / 2] = kind;
  }
  cudaEventRecord(c->ev[c->ev_used], c->stream);
  c->ev_used++;
}
void default_tiles(icarus_ctx *c) {
  const int n1 = c->d.block[1], n2 = c->d.block[2];
  const int trc = c->d.tracer;
  if (c->tile_j && c->tile_k) {
    c->occ = stage_max_ctas_per_sm(c->prec, c->tile_j, c->tile_k, trc);
    return;
  }
  if (c->prec && n1 >= 12 && n2 >= 20) {
    c->tile_j = 12;
    c->tile_k = 20;
  } else if (n2 >= 32) {
    c->tile_j = c->prec ? 8 : 4;
    c->tile_k = 32;
  } else if (n1 >= 12 && n2 >= 12) {
    c->tile_j = 12;
    c->tile_k = 12;
  } else {
    c->tile_j = 8;
    c->tile_k = 8;
  }
  if (!stage_tile_supported(c->prec, c->tile_j, c->tile_k, trc)) {
    c->tile_j = 8;
    c->tile_k = 8;
  }
  c->occ = stage_max_ctas_per_sm(c->prec, c->tile_j, c->tile_k, trc);
}

StageLaunch stage_cfg(icarus_ctx *c, int stage2) {
  StageLaunch sl{};
  sl.tile_j = c->tile_j;
  sl.tile_k = c->tile_k;
  sl.tiles_j = (c->d.block[1] + sl.tile_j - 1) / sl.tile_j;
  sl.tiles_k = (c->d.block[2] + sl.tile_k - 1) / sl.tile_k;
  const int slots = c->nsm * c->occ;
  int seg = c->seg_len;
  if (seg <= 0) {
    // enough work items for ~4 waves of the persistent grid, segments >= 8 planes
    const long long base = (long long)c->nleaves * sl.tiles_j * sl.tiles_k;
    long long segs = (4LL * slots + base - 1) / std::max(1LL, base);
    segs = std::max(1LL, std::min<long long>(segs, c->d.block[0] / 8 > 0 ? c->d.block[0] / 8 : 1));
    seg = (c->d.block[0] + (int)segs - 1) / (int)segs;
  }
  seg = std::max(1, std::min(std::min(seg, c->d.block[0]), STAGE_SEG_MAX));
  sl.seg_len = seg;
  sl.segs = (c->d.block[0] + seg - 1) / seg;
  sl.list = c->all_list;
  sl.nlist = c->nleaves;
  const long long nwork = (long long)sl.nlist * sl.tiles_j * sl.tiles_k * sl.segs;
  sl.grid = (int)std::max(1LL, std::min<long long>(nwork, slots));
  sl.stage2 = stage2;
  sl.dtfac = stage2 ? 1.0 : 0.5;
  return sl;
}

// optional event pair around a launch (profiling mode only)
struct ProfScope {
  icarus_ctx *c;
  int kind;
  ProfScope(icarus_ctx *c_, int k) : c(c_), kind(k) {
    if (c->prof_on) prof_mark(c, kind, 0);
  }
  ~ProfScope() {
    if (c->prof_on) prof_mark(c, kind, 1);
  }
};

// Ghost fill of buf at the member times (+ tfac dt).  faces_only: only the
// ghost cells outside the block in exactly one direction -- enough for the
// predictor stage, whose stencils are crosses and whose face fluxes take no
// transverse halo; the corrector's cleaning takes div B on the ring around
// the tile, which reaches edge ghosts, and the probe, the estimators and the
// regrid get every ghost cell too.
int enqueue_ghost(icarus_ctx *c, void *buf, double tfac, bool faces_only = false, bool skip_same = false) {
  int n = 0;
  for (int L = 1; L <= c->max_level_present; L++) {
    if (c->lvl_count[L] == 0) continue;
    if (skip_same) {
      // the ghost cells same-level leaves hold are read by the stage kernels
      // from those leaves: only the regions held by coarser or finer leaves
      const int ne = faces_only ? c->rent_face[L] : c->rent_count[L];
      if (ne > 0) {
        ProfScope p(c, 1);
        ghost_regions_launch(c->kp, buf, c->prec, c->rent + c->rent_start[L], ne, c->rshell, L, c->stream);
        n++;
      }
    } else {
      ProfScope p(c, 1);
      ghost_neighbour_launch(c->kp, buf, c->prec, c->lvl_list + c->lvl_start[L], c->lvl_count[L], c->shell,
                             faces_only ? c->nshell_face : c->lay.nshell, L, c->stream);
      n++;
    }
    for (int dd = 0; dd < 3; dd++) {
      if (c->side_count[L][dd] == 0) continue;
      ProfScope p(c, 2);
      ghost_physical_launch(c->kp, buf, c->prec, c->sides + c->side_start[L][dd], c->side_count[L][dd], dd, L, tfac,
                            faces_only, skip_same, c->stream);
      n++;
    }
  }
  return n;
}

int enqueue_step(icarus_ctx *c) {
  int n = 0;
  {
    ProfScope p(c, 0);
    dt_begin_launch(c->kp, c->tstop, c->stream);
  }
  n++;
  // the step's fills leave the ghost cells that same-level leaves hold to the
  // stage kernels, which read them from those leaves
  n += enqueue_ghost(c, c->U, 0.0, true, c->direct_halo);
  StageLaunch s1 = stage_cfg(c, 0);
  s1.direct = c->direct_halo;
  s1.Uin = c->U;
  s1.U0 = c->U;
  s1.Uout = c->Us;
  s1.flux = nullptr;
  {
    ProfScope p(c, 3);
    stage_launch(c->kp, s1, c->prec, c->stream);
  }
  n++;
  n += enqueue_ghost(c, c->Us, 0.5, false, c->direct_halo);
  StageLaunch s2 = stage_cfg(c, 1);
  s2.direct = c->direct_halo;
  s2.Uin = c->Us;
  s2.U0 = c->U;
  s2.Uout = c->U;
  s2.flux = c->d.max_level > 1 ? c->flux : nullptr;
  {
    ProfScope p(c, 4);
    stage_launch(c->kp, s2, c->prec, c->stream);
  }
  n++;
  if (c->nrlist > 0) {
    ProfScope p(c, 5);
    reflux_launch(c->kp, c->U, c->flux, c->prec, c->rlist, c->nrlist, c->stream);
    n++;
  }
  {
    ProfScope p(c, 6);
    dt_finalize_launch(c->kp, c->d.cfl, c->stream);
  }
  n++;
  return n;
}

// ghost fill, features and predicted refinement probability of every leaf
void mlp_leaf_probabilities(icarus_ctx *c) {
  enqueue_ghost(c, c->U, 0.0);
  mlp_features_launch(c->kp, c->U, c->prec, 0, c->nleaves, c->mlp_feat, c->stream);
  for (int b0 = 0; b0 < c->nleaves; b0 += MLP_BMAX) {
    const int B = std::min(MLP_BMAX, c->nleaves - b0);
    mlp_forward_launch(c->mlp_theta, c->mlp_feat + (size_t)b0 * 64, nullptr, B, c->mlp_h1, c->mlp_h2,
                       c->mlp_prob + b0, c->stream);
  }
}

// seeded permutation (splitmix64 + Fisher-Yates)
void permutation(std::vector<int> &p, int n, uint64_t &state) {
  p.resize(n);
  for (int i = 0; i < n; i++) p[i] = i;
  for (int i = n - 1; i > 0; i--) {
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const int j = (int)(z % (uint64_t)(i + 1));
    std::swap(p[i], p[j]);
  }
}

// status of a status word read back from the device; poisons the context
icarus_status status_of_word(icarus_ctx *c, unsigned int w) {
  if (w & (ST_NAN | ST_FLOOR | ST_TREE)) {
    c->poisoned = true;
    return ICARUS_ERR_NONPHYSICAL;
  }
  if (w & ST_TIMEOUT) {
    c->poisoned = true;
    return ICARUS_ERR_TIMEOUT;
  }
  return ICARUS_OK;
}

icarus_status check_status(icarus_ctx *c) {
  unsigned int w = 0;
  CK(cudaMemcpyAsync(&w, c->status, sizeof(w), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->status_pending = false;
  return status_of_word(c, w);
}

// the status word copied after an earlier step, if its copy has landed
// (no synchronisation)
icarus_status poll_status(icarus_ctx *c) {
  if (!c->status_pending) return ICARUS_OK;
  const cudaError_t q = cudaEventQuery(c->status_ev);
  if (q == cudaErrorNotReady) return ICARUS_OK;
  c->status_pending = false;
  if (q != cudaSuccess) return ICARUS_ERR_CUDA;
  return status_of_word(c, *c->h_status);
}

icarus_status recompute_dt(icarus_ctx *c) {
  CK(cudaMemsetAsync(c->inv_max, 0, sizeof(unsigned long long) * c->d.n_members, c->stream));
  ProfScope p(c, 9);
  dt_full_launch(c->kp, c->U, c->prec, c->nleaves, c->d.cfl, c->stream);
  CK(cudaPeekAtLastError());
  return ICARUS_OK;
}

bool member_ok(icarus_ctx *c, int m) { return c && m >= 0 && m < c->d.n_members; }

}  // namespace

// ======================================================================
extern "C" {

const char *icarus_status_string(icarus_status s) {
  switch (s) {
    case ICARUS_OK: return "ok";
    case ICARUS_ERR_ARG: return "invalid argument";
    case ICARUS_ERR_ARENA: return "arena too small or misaligned";
    case ICARUS_ERR_CUDA: return "CUDA runtime error";
    case ICARUS_ERR_NONPHYSICAL: return "non-physical state on the device";
    case ICARUS_ERR_TIMEOUT: return "bounded device wait gave up";
    case ICARUS_ERR_STATE: return "call out of order or context poisoned";
    case ICARUS_ERR_CAPACITY: return "block pool capacity exceeded";
  }
  return "unknown status";
}

icarus_status icarus_arena_bytes(const icarus_grid_desc *desc, size_t *bytes) {
  if (!bytes) return ICARUS_ERR_ARG;
  icarus_status st = validate(desc);
  if (st != ICARUS_OK) return st;
  *bytes = make_layout(desc).total;
  return ICARUS_OK;
}

icarus_status icarus_init_grid(const icarus_grid_desc *desc, icarus_ctx **out) {
  if (!out) return ICARUS_ERR_ARG;
  *out = nullptr;
  icarus_status st = validate(desc);
  if (st != ICARUS_OK) return st;
  Layout lay = make_layout(desc);
  if (!desc->arena || desc->arena_bytes < lay.total) return ICARUS_ERR_ARENA;
  if ((uintptr_t)desc->arena % ALIGN) return ICARUS_ERR_ARENA;
  icarus_ctx *c = new (std::nothrow) icarus_ctx();
  if (!c) return ICARUS_ERR_ARG;
  c->d = *desc;
  for (int L = 1; L <= MAXLEV + 1; L++)
    for (int d = 0; d < 3; d++) c->nbd[L][d] = (desc->n_cells[d] / desc->block[d]) << (L - 1);
  c->lay = lay;
  c->prec = desc->precision == ICARUS_FP32_MIXED ? 1 : 0;
  c->rsize = c->prec ? 4 : 8;
  c->stream = (cudaStream_t)desc->stream;
  c->arena = (char *)desc->arena;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete c;
    return ICARUS_ERR_CUDA;
  }
  c->dev = dev;
  if (cudaHostAlloc((void **)&c->h_status, sizeof(unsigned int), cudaHostAllocDefault) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->status_ev, cudaEventDisableTiming) != cudaSuccess) {
    if (c->h_status) cudaFreeHost(c->h_status);
    delete c;
    return ICARUS_ERR_CUDA;
  }
  // the allocation-free sums' scratch is put in place now, while the caller
  // can still give up device memory for it
  if (static_sums_prepare(dev) != 0) {
    cudaEventDestroy(c->status_ev);
    cudaFreeHost(c->h_status);
    delete c;
    return ICARUS_ERR_CUDA;
  }
  c->geo = at<Geometry>(c, lay.geo);
  c->blk = at<DevBlock>(c, lay.blk);
  c->blk_alt = lay.blk_alt.bytes ? at<DevBlock>(c, lay.blk_alt) : nullptr;
  c->nb27 = at<int>(c, lay.nb27);
  c->U = c->arena + lay.U.off;
  c->Us = c->arena + lay.Us.off;
  c->Ualt = lay.Ualt.bytes ? c->arena + lay.Ualt.off : nullptr;
  c->flux = lay.flux.bytes ? c->arena + lay.flux.off : nullptr;
  c->lmap = at<int>(c, lay.lmap);
  c->lmap_off = at<long long>(c, lay.lmap_off);
  c->bmap = at<double>(c, lay.bmap);
  c->cme = at<DevCme>(c, lay.cme);
  c->earth = at<DevEarth>(c, lay.earth);
  c->vbg = at<double>(c, lay.vbg);
  double *sc = at<double>(c, lay.scal);
  const int nm = desc->n_members;
  c->t = sc;
  c->dt_used = sc + nm;
  c->dt_cfl = sc + 2 * nm;
  c->tstop = sc + 3 * nm;
  c->inv_max = reinterpret_cast<unsigned long long *>(sc + 4 * nm);
  c->status = reinterpret_cast<unsigned int *>(sc + 5 * nm);
  c->floor_hits = reinterpret_cast<unsigned long long *>(sc + 5 * nm + 1);
  c->updates = sc + 5 * nm + 2;
  c->cells_m = sc + 6 * nm + 2;
  c->floor_prev = reinterpret_cast<unsigned long long *>(sc + 7 * nm + 2);
  c->flags = at<signed char>(c, lay.flags);
  c->all_list = at<int>(c, lay.lists);
  c->lvl_list = c->all_list + lay.max_blocks;
  c->rent = at<int2>(c, lay.rent);
  c->sides = at<int2>(c, lay.sides);
  c->rlist = at<int>(c, lay.rlist);
  c->ops = lay.ops.bytes ? at<MoveOp>(c, lay.ops) : nullptr;
  c->shell = at<int>(c, lay.shell);
  c->rshell = at<int>(c, lay.rshell);
  c->staging = at<double>(c, lay.staging);
  c->partial = at<double>(c, lay.partial);
  c->probe_in = at<double>(c, lay.probe_in);
  c->probe_out = at<double>(c, lay.probe_out);
  {
    float *par = at<float>(c, lay.mlp_par);
    const int np = mlp_n_params();
    c->mlp_theta = par;
    c->mlp_grad = par + np;
    c->mlp_m = par + 2 * (size_t)np;
    c->mlp_v = par + 3 * (size_t)np;
    c->mlp_loss = par + 4 * (size_t)np;
    c->mlp_feat = at<float>(c, lay.mlp_feat);
    c->mlp_prob = c->mlp_feat + (size_t)lay.max_blocks * 64;
    c->mlp_X = at<float>(c, lay.mlp_X);
    c->mlp_T = at<float>(c, lay.mlp_T);
    c->mlp_idx = at<int>(c, lay.mlp_idx);
    float *act = at<float>(c, lay.mlp_act);
    c->mlp_h1 = act;
    c->mlp_h2 = act + (size_t)MLP_BMAX * 128;
    c->mlp_dh2 = act + (size_t)2 * MLP_BMAX * 128;
    c->mlp_dh1 = act + (size_t)3 * MLP_BMAX * 128;
    c->mlp_y = act + (size_t)4 * MLP_BMAX * 128;
    c->mlp_dz = c->mlp_y + MLP_BMAX;
    c->mlp_xin = at<float>(c, lay.mlp_xin);
    c->mlp_tin = c->mlp_xin + (size_t)MLP_BMAX * 64;
  }
  auto fail = [&](icarus_status s) {
    cudaEventDestroy(c->status_ev);
    cudaFreeHost(c->h_status);
    delete c;
    return s;
  };
  // zero the small per-member and status words; the state pools are zeroed too
  if (cudaMemsetAsync(c->arena + lay.scal.off, 0, lay.scal.bytes, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->arena + lay.cme.off, 0, lay.cme.bytes, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->arena + lay.earth.off, 0, lay.earth.bytes, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->arena + lay.bmap.off, 0, lay.bmap.bytes, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->arena + lay.U.off, 0, lay.U.bytes, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->arena + lay.Us.off, 0, lay.Us.bytes, c->stream) != cudaSuccess)
    return fail(ICARUS_ERR_CUDA);
  if ((st = build_geometry(c)) != ICARUS_OK) return fail(st);
  // shell (ghost) cells of a padded block: face ghosts first, then edges and
  // corners; within each part the cells with even (p0, p1, p2) -- the first
  // cells of the 2 x 2 x 2 groups a coarse neighbour's prolongation fills --
  // come first, so that those threads share warps; memory order otherwise
  {
    std::vector<int> sh;
    const int P0 = desc->block[0] + 2 * NGH, P1 = desc->block[1] + 2 * NGH, P2 = desc->block[2] + 2 * NGH;
    auto add = [&](bool faces, bool leaders) {
      for (int i = 0; i < P0; i++)
        for (int j = 0; j < P1; j++)
          for (int k = 0; k < P2; k++) {
            const int out = (i < NGH || i >= NGH + desc->block[0]) + (j < NGH || j >= NGH + desc->block[1]) +
                            (k < NGH || k >= NGH + desc->block[2]);
            const bool lead = ((i | j | k) & 1) == 0;
            if ((faces ? out == 1 : out > 1) && lead == leaders) sh.push_back((i << 20) | (j << 10) | k);
          }
    };
    add(true, true);
    add(true, false);
    c->nshell_face = (int)sh.size();
    add(false, true);
    add(false, false);
    // the same cells ordered by region (r = 9 (sx + 1) + 3 (sy + 1) + sz + 1
    // with s the side of each coordinate: -1 low ghost, 0 interior, +1 high
    // ghost), group-first cells first within a region; a table of (start,
    // group-first cells, cells) per region ahead of them
    std::vector<int> rs(81, 0);
    auto side = [&](int p, int d) { return p < NGH ? -1 : (p >= NGH + desc->block[d] ? 1 : 0); };
    for (int r = 0; r < 27; r++) {
      const int want[3] = {r / 9 - 1, (r / 3) % 3 - 1, r % 3 - 1};
      const int start = (int)rs.size() - 81;
      int lead_n = 0;
      for (int pass = 0; pass < 2 && r != 13; pass++)
        for (int i = 0; i < P0; i++)
          for (int j = 0; j < P1; j++)
            for (int k = 0; k < P2; k++) {
              if (side(i, 0) != want[0] || side(j, 1) != want[1] || side(k, 2) != want[2]) continue;
              const bool lead = ((i | j | k) & 1) == 0;
              if (lead != (pass == 0)) continue;
              rs.push_back((i << 20) | (j << 10) | k);
              if (lead) lead_n++;
            }
      rs[3 * r] = start;
      rs[3 * r + 1] = lead_n;
      rs[3 * r + 2] = (int)rs.size() - 81 - start;
      for (int q = 0; q < 3; q++) c->reg_tab[r][q] = rs[3 * r + q];
    }
    if (cudaMemcpyAsync(c->shell, sh.data(), sizeof(int) * sh.size(), cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(c->rshell, rs.data(), sizeof(int) * rs.size(), cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return fail(ICARUS_ERR_CUDA);
  }
  // base blocks of every member, Morton order
  c->mem.assign(nm, Member());
  const int nb0 = desc->n_cells[0] / desc->block[0], nb1 = desc->n_cells[1] / desc->block[1],
            nb2 = desc->n_cells[2] / desc->block[2];
  for (int m = 0; m < nm; m++) {
    Member &M = c->mem[m];
    M.max_level = desc->max_level;
    for (int a = 0; a < nb0; a++)
      for (int b = 0; b < nb1; b++)
        for (int e = 0; e < nb2; e++) M.leaves.push_back(Leaf{1, {a, b, e}});
    std::sort(M.leaves.begin(), M.leaves.end(), [&](const Leaf &x, const Leaf &y) {
      return morton_key(x, desc->max_level) < morton_key(y, desc->max_level);
    });
    build_member_map(c, M);
  }
  fill_kp(c);
  if ((st = upload_tree(c, c->blk)) != ICARUS_OK) return fail(st);
  default_tiles(c);
  c->h_tstop.assign(nm, 0.0);
  // the uniform zero state has no time step: mark dt as unknown (0) until a state is set
  *out = c;
  return ICARUS_OK;
}

void icarus_destroy(icarus_ctx *c) {
  if (!c) return;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->status_ev) {
    cudaEventSynchronize(c->status_ev);
    cudaEventDestroy(c->status_ev);
  }
  if (c->h_status) cudaFreeHost(c->h_status);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  delete c;
}

icarus_status icarus_set_inner_boundary(icarus_ctx *c, int member, const double *prim) {
  if (!member_ok(c, member) || !prim) return ICARUS_ERR_ARG;
  c->ghosts_fresh = false;
  if (c->poisoned) return ICARUS_ERR_STATE;
  const size_t n = (size_t)NVAR * c->d.n_cells[1] * c->d.n_cells[2];
  CK(cudaMemcpyAsync(c->bmap + member * n, prim, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->graph_valid = false;
  return ICARUS_OK;
}

icarus_status icarus_inject_cone_cme(icarus_ctx *c, int member, const icarus_cone *p) {
  if (!member_ok(c, member) || !p) return ICARUS_ERR_ARG;
  c->ghosts_fresh = false;
  if (c->poisoned) return ICARUS_ERR_STATE;
  if (!(p->v > 0.0) || !(p->half_width > 0.0) || !(p->half_width < M_PI / 2) || !(p->rho > 0.0) || !(p->p > 0.0))
    return ICARUS_ERR_ARG;
  Member &M = c->mem[member];
  for (const Leaf &l : M.leaves)
    if (l.level != 1) return ICARUS_ERR_STATE;
  DevCme dc{};
  dc.t_start = p->t_start;
  dc.t_max = p->t_max;
  dc.colat = p->colat;
  dc.lon = p->lon;
  dc.half_width = p->half_width;
  dc.v = p->v;
  dc.rho = p->rho;
  dc.p = p->p;
  dc.active = 1;
  dc.pad = 1;  // background speed recorded below
  M.cme = dc;
  CK(cudaMemcpyAsync(c->cme + member, &M.cme, sizeof(DevCme), cudaMemcpyHostToDevice, c->stream));
  const size_t nbc = (size_t)c->d.n_cells[0] * c->d.n_cells[1] * c->d.n_cells[2];
  vbg_launch(c->kp, c->U, c->prec, member, c->mem_off[member], (int)M.leaves.size(), c->vbg + member * nbc,
             c->stream);
  CK(cudaPeekAtLastError());
  CK(cudaStreamSynchronize(c->stream));
  return ICARUS_OK;
}

icarus_status icarus_set_time(icarus_ctx *c, int member, double t) {
  if (!member_ok(c, member)) return ICARUS_ERR_ARG;
  c->ghosts_fresh = false;
  CK(cudaMemcpyAsync(c->t + member, &t, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return ICARUS_OK;
}

icarus_status icarus_set_earth(icarus_ctx *c, int member, double colat, double lon0, double t0, double rate) {
  if (!member_ok(c, member) || !std::isfinite(colat) || !std::isfinite(lon0) || !std::isfinite(t0) ||
      !std::isfinite(rate))
    return ICARUS_ERR_ARG;
  const DevEarth e{colat, lon0, t0, rate, 1, 0};
  CK(cudaMemcpyAsync(c->earth + member, &e, sizeof(DevEarth), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return ICARUS_OK;
}

icarus_status icarus_set_member_max_level(icarus_ctx *c, int member, int L) {
  if (!member_ok(c, member) || L < 1 || L > c->d.max_level) return ICARUS_ERR_ARG;
  c->mem[member].max_level = L;
  // the block table carries each block's finest level (learned pre-flags)
  const int off = c->mem_off[member], n = (int)c->mem[member].leaves.size();
  if (n > 0 && (int)c->hblk.size() >= off + n) {
    for (int s = off; s < off + n; s++) c->hblk[s].lmax = L;
    CK(cudaMemcpyAsync(c->blk + off, c->hblk.data() + off, sizeof(DevBlock) * n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return ICARUS_OK;
}

icarus_status icarus_set_tile(icarus_ctx *c, int tj, int tk, int seg) {
  if (!c) return ICARUS_ERR_ARG;
  if (tj || tk) {
    if (!stage_tile_supported(c->prec, tj, tk, c->d.tracer)) return ICARUS_ERR_ARG;
    c->tile_j = tj;
    c->tile_k = tk;
    default_tiles(c);
  } else {
    c->tile_j = c->tile_k = 0;
    default_tiles(c);
  }
  c->seg_len = seg > 0 ? seg : 0;
  c->graph_valid = false;
  return ICARUS_OK;
}

icarus_status icarus_set_direct_halo(icarus_ctx *c, int enable) {
  if (!c) return ICARUS_ERR_ARG;
  c->direct_halo = enable != 0;
  c->graph_valid = false;
  return ICARUS_OK;
}

icarus_status icarus_use_graph(icarus_ctx *c, int enable) {
  if (!c) return ICARUS_ERR_ARG;
  c->use_graph = enable != 0;
  return ICARUS_OK;
}

icarus_status icarus_kernels_per_step(icarus_ctx *c, int *n) {
  if (!c || !n) return ICARUS_ERR_ARG;
  int k = 4 + (c->nrlist > 0 ? 1 : 0);  // dt begin, two stages, dt finalize, reflux
  for (int L = 1; L <= c->max_level_present; L++) {
    if (!c->lvl_count[L]) continue;
    // neighbour ghost pass of both fills (with direct halo reads only over
    // the regions held by coarser or finer leaves: faces in the first fill)
    if (c->direct_halo) k += (c->rent_face[L] > 0) + (c->rent_count[L] > 0);
    else k += 2;
    for (int d = 0; d < 3; d++)
      if (c->side_count[L][d]) k += 2;   // physical ghost pass, both fills
  }
  *n = k;
  return ICARUS_OK;
}

icarus_status icarus_step(icarus_ctx *c, int n_steps, const double *t_stop, double *t_out) {
  if (!c || n_steps < 0 || !t_stop) return ICARUS_ERR_ARG;
  if (n_steps > 0) c->ghosts_fresh = false;
  if (c->poisoned) return ICARUS_ERR_STATE;
  {
    // a non-physical state left by an earlier call that returned no times
    const icarus_status st = poll_status(c);
    if (st != ICARUS_OK) return st;
  }
  const int nm = c->d.n_members;
  c->h_tstop.assign(t_stop, t_stop + nm);
  CK(cudaMemcpyAsync(c->tstop, c->h_tstop.data(), sizeof(double) * nm, cudaMemcpyHostToDevice, c->stream));
  if (n_steps > 0) {
    if (c->use_graph && !c->prof_on && c->stream != nullptr) {
      if (!c->graph_valid) {
        if (c->graph) {
          cudaGraphExecDestroy(c->graph);
          c->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        c->kernels_per_step = enqueue_step(c);
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (e != cudaSuccess) {
          fprintf(stderr, "libicarus: graph capture failed: %s\n", cudaGetErrorString(e));
          return ICARUS_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&c->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
          fprintf(stderr, "libicarus: graph instantiate failed: %s\n", cudaGetErrorString(e));
          return ICARUS_ERR_CUDA;
        }
        c->graph_valid = true;
      }
    }
    // When every member has a finite stop time, the members' times are read
    // back every STEP_CHUNK steps and the call returns once all have landed
    // (the remaining steps would launch work for nobody).
    bool bounded = true;
    for (int m = 0; m < nm; m++) bounded = bounded && std::isfinite(c->h_tstop[m]);
    constexpr int STEP_CHUNK = 8;
    std::vector<double> th(nm);
    for (int s0 = 0; s0 < n_steps; s0 += STEP_CHUNK) {
      const int ns = std::min(STEP_CHUNK, n_steps - s0);
      if (c->graph_valid && c->use_graph && !c->prof_on && c->stream != nullptr) {
        for (int s = 0; s < ns; s++) CK(cudaGraphLaunch(c->graph, c->stream));
      } else {
        for (int s = 0; s < ns; s++) c->kernels_per_step = enqueue_step(c);
        CK(cudaPeekAtLastError());
      }
      if (bounded && s0 + ns < n_steps) {
        unsigned int w = 0;
        CK(cudaMemcpyAsync(th.data(), c->t, sizeof(double) * nm, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(&w, c->status, sizeof(w), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        const icarus_status st = status_of_word(c, w);
        if (st != ICARUS_OK) return st;
        bool done = true;
        for (int m = 0; m < nm; m++) done = done && th[m] >= c->h_tstop[m];
        if (done) break;
      }
    }
  }
  // the host copy of t_stop stays alive in the context until the next call
  if (t_out) {
    CK(cudaMemcpyAsync(t_out, c->t, sizeof(double) * nm, cudaMemcpyDeviceToHost, c->stream));
    icarus_status st = check_status(c);
    if (st != ICARUS_OK) return st;
  } else if (n_steps > 0) {
    // no synchronisation: the status word follows the steps into pinned host
    // memory and is looked at by the next call
    CK(cudaMemcpyAsync(c->h_status, c->status, sizeof(unsigned int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaEventRecord(c->status_ev, c->stream));
    c->status_pending = true;
  }
  return ICARUS_OK;
}

icarus_status icarus_ghost_fill(icarus_ctx *c) {
  if (!c) return ICARUS_ERR_ARG;
  if (c->poisoned) return ICARUS_ERR_STATE;
  enqueue_ghost(c, c->U, 0.0);
  CK(cudaPeekAtLastError());
  c->ghosts_fresh = true;
  return ICARUS_OK;
}

icarus_status icarus_n_leaves(icarus_ctx *c, int member, int *n) {
  if (!c || !n) return ICARUS_ERR_ARG;
  if (member < 0) {
    *n = c->nleaves;
    return ICARUS_OK;
  }
  if (!member_ok(c, member)) return ICARUS_ERR_ARG;
  *n = (int)c->mem[member].leaves.size();
  return ICARUS_OK;
}

icarus_status icarus_get_tree(icarus_ctx *c, int member, int32_t *rows, int capacity, int *n) {
  if (!member_ok(c, member) || !n) return ICARUS_ERR_ARG;
  const Member &M = c->mem[member];
  *n = (int)M.leaves.size();
  if (!rows) return ICARUS_OK;
  if (capacity < *n) return ICARUS_ERR_ARG;
  for (int i = 0; i < *n; i++) {
    rows[4 * i] = M.leaves[i].level;
    for (int d = 0; d < 3; d++) rows[4 * i + 1 + d] = M.leaves[i].ix[d];
  }
  return ICARUS_OK;
}

icarus_status icarus_set_state(icarus_ctx *c, int member, const double *host, size_t n, int is_prim) {
  if (!member_ok(c, member) || !host) return ICARUS_ERR_ARG;
  c->ghosts_fresh = false;
  if (c->poisoned) return ICARUS_ERR_STATE;
  const size_t per = (size_t)NVAR * c->kp.icells;
  const int nl = (int)c->mem[member].leaves.size();
  if (n != per * nl) return ICARUS_ERR_ARG;
  const int chunk = (int)(c->lay.staging_doubles / per);
  for (int s0 = 0; s0 < nl; s0 += chunk) {
    const int ns = std::min(chunk, nl - s0);
    CK(cudaMemcpyAsync(c->staging, host + (size_t)s0 * per, sizeof(double) * per * ns, cudaMemcpyHostToDevice,
                       c->stream));
    unpack_state_launch(c->kp, c->U, c->prec, c->mem_off[member] + s0, ns, c->staging, is_prim, c->stream);
    CK(cudaPeekAtLastError());
    CK(cudaStreamSynchronize(c->stream));
  }
  icarus_status st = recompute_dt(c);
  if (st != ICARUS_OK) return st;
  CK(cudaStreamSynchronize(c->stream));
  return ICARUS_OK;
}

icarus_status icarus_get_state(icarus_ctx *c, int member, double *host, size_t n) {
  if (!member_ok(c, member) || !host) return ICARUS_ERR_ARG;
  const size_t per = (size_t)NVAR * c->kp.icells;
  const int nl = (int)c->mem[member].leaves.size();
  if (n != per * nl) return ICARUS_ERR_ARG;
  const int chunk = (int)(c->lay.staging_doubles / per);
  for (int s0 = 0; s0 < nl; s0 += chunk) {
    const int ns = std::min(chunk, nl - s0);
    pack_state_launch(c->kp, c->U, c->prec, c->mem_off[member] + s0, ns, c->staging, c->stream);
    CK(cudaPeekAtLastError());
    CK(cudaMemcpyAsync(host + (size_t)s0 * per, c->staging, sizeof(double) * per * ns, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return ICARUS_OK;
}

icarus_status icarus_get_padded(icarus_ctx *c, int member, int leaf, double *host, size_t n) {
  if (!member_ok(c, member) || !host) return ICARUS_ERR_ARG;
  const int nl = (int)c->mem[member].leaves.size();
  if (leaf < 0 || leaf >= nl || n != (size_t)NVAR * c->kp.pcells) return ICARUS_ERR_ARG;
  const size_t slot = (size_t)c->mem_off[member] + leaf;
  std::vector<unsigned char> raw(n * c->rsize);
  const size_t stride = (size_t)c->kp.nvs * c->kp.pcells * c->rsize;   // bytes per slot
  CK(cudaMemcpyAsync(raw.data(), static_cast<const char *>(c->U) + slot * stride, raw.size(),
                     cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (c->prec) {
    const float *f = reinterpret_cast<const float *>(raw.data());
    for (size_t q = 0; q < n; q++) host[q] = (double)f[q];
  } else {
    memcpy(host, raw.data(), raw.size());
  }
  return ICARUS_OK;
}

}  // extern "C"

namespace {

// the tracer plane (padded) of every leaf of a member into / out of host
// memory: one strided copy
icarus_status tracer_planes(icarus_ctx *c, int member, std::vector<unsigned char> &raw, bool to_host) {
  const size_t nl = c->mem[member].leaves.size();
  const size_t plane = (size_t)c->kp.pcells * c->rsize, stride = (size_t)c->kp.nvs * plane;
  char *base = static_cast<char *>(c->U) + (size_t)c->mem_off[member] * stride + (size_t)TRV * plane;
  if (to_host) {
    raw.resize(nl * plane);
    CK(cudaMemcpy2DAsync(raw.data(), plane, base, stride, plane, nl, cudaMemcpyDeviceToHost, c->stream));
  } else {
    CK(cudaMemcpy2DAsync(base, stride, raw.data(), plane, plane, nl, cudaMemcpyHostToDevice, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return ICARUS_OK;
}

template <typename F>
void for_interior(const icarus_ctx *c, F f) {
  const int *nb = c->d.block;
  const int P1 = nb[1] + 2 * NGH, P2 = nb[2] + 2 * NGH;
  size_t q = 0;
  for (int i = 0; i < nb[0]; i++)
    for (int j = 0; j < nb[1]; j++)
      for (int k = 0; k < nb[2]; k++, q++) f(q, ((size_t)(i + NGH) * P1 + j + NGH) * P2 + k + NGH);
}

}  // namespace

extern "C" {

icarus_status icarus_get_tracer(icarus_ctx *c, int member, double *host, size_t n) {
  if (!member_ok(c, member) || !host) return ICARUS_ERR_ARG;
  if (!c->d.tracer) return ICARUS_ERR_STATE;
  const size_t nl = c->mem[member].leaves.size(), ic = (size_t)c->kp.icells, pc = (size_t)c->kp.pcells;
  if (n != nl * ic) return ICARUS_ERR_ARG;
  std::vector<unsigned char> raw;
  icarus_status st = tracer_planes(c, member, raw, true);
  if (st != ICARUS_OK) return st;
  for (size_t b = 0; b < nl; b++)
    for_interior(c, [&](size_t q, size_t pidx) {
      host[b * ic + q] = c->prec ? (double)reinterpret_cast<const float *>(raw.data())[b * pc + pidx]
                                 : reinterpret_cast<const double *>(raw.data())[b * pc + pidx];
    });
  return ICARUS_OK;
}

icarus_status icarus_set_tracer(icarus_ctx *c, int member, const double *host, size_t n) {
  if (!member_ok(c, member) || !host) return ICARUS_ERR_ARG;
  if (!c->d.tracer) return ICARUS_ERR_STATE;
  if (c->poisoned) return ICARUS_ERR_STATE;
  const size_t nl = c->mem[member].leaves.size(), ic = (size_t)c->kp.icells, pc = (size_t)c->kp.pcells;
  if (n != nl * ic) return ICARUS_ERR_ARG;
  c->ghosts_fresh = false;
  std::vector<unsigned char> raw;
  icarus_status st = tracer_planes(c, member, raw, true);   // keep the ghost layers
  if (st != ICARUS_OK) return st;
  for (size_t b = 0; b < nl; b++)
    for_interior(c, [&](size_t q, size_t pidx) {
      if (c->prec) reinterpret_cast<float *>(raw.data())[b * pc + pidx] = (float)host[b * ic + q];
      else reinterpret_cast<double *>(raw.data())[b * pc + pidx] = host[b * ic + q];
    });
  return tracer_planes(c, member, raw, false);
}

icarus_status icarus_get_dt(icarus_ctx *c, double *dt) {
  if (!c || !dt) return ICARUS_ERR_ARG;
  CK(cudaMemcpyAsync(dt, c->dt_cfl, sizeof(double) * c->d.n_members, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return ICARUS_OK;
}

icarus_status icarus_cell_updates(icarus_ctx *c, double *out) {
  if (!c || !out) return ICARUS_ERR_ARG;
  CK(cudaMemcpyAsync(out, c->updates, sizeof(double) * c->d.n_members, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return ICARUS_OK;
}

icarus_status icarus_status_word(icarus_ctx *c, uint32_t *word, uint64_t *floor_hits) {
  if (!c) return ICARUS_ERR_ARG;
  unsigned int w = 0;
  unsigned long long f = 0;
  CK(cudaMemcpyAsync(&w, c->status, sizeof(w), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&f, c->floor_hits, sizeof(f), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (word) *word = w;
  if (floor_hits) *floor_hits = f;
  return ICARUS_OK;
}

icarus_status icarus_conservation_sums(icarus_ctx *c, int member, double *out8) {
  if (!member_ok(c, member) || !out8) return ICARUS_ERR_ARG;
  const int nl = (int)c->mem[member].leaves.size();
  sums_launch(c->kp, c->U, c->prec, c->mem_off[member], nl, c->partial, c->stream);
  CK(cudaPeekAtLastError());
  std::vector<double> h((size_t)nl * NVAR);
  CK(cudaMemcpyAsync(h.data(), c->partial, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int v = 0; v < NVAR; v++) out8[v] = 0.0;
  for (int b = 0; b < nl; b++)
    for (int v = 0; v < NVAR; v++) out8[v] += h[(size_t)b * NVAR + v];
  return ICARUS_OK;
}

icarus_status icarus_probe(icarus_ctx *c, int member, int n_pts, const double *rtp, double *prim_out) {
  if (!member_ok(c, member) || n_pts < 0 || n_pts > 4096 || (n_pts && (!rtp || !prim_out))) return ICARUS_ERR_ARG;
  if (c->poisoned) return ICARUS_ERR_STATE;
  if (!n_pts) return ICARUS_OK;
  // probes of several members at one time share one ghost fill
  if (!c->ghosts_fresh) {
    enqueue_ghost(c, c->U, 0.0);
    c->ghosts_fresh = true;
  }
  CK(cudaMemcpyAsync(c->probe_in, rtp, sizeof(double) * 3 * n_pts, cudaMemcpyHostToDevice, c->stream));
  probe_launch2(c->kp, c->U, c->prec, member, c->d.max_level, n_pts, c->probe_in, c->probe_out, c->stream);
  CK(cudaPeekAtLastError());
  CK(cudaMemcpyAsync(prim_out, c->probe_out, sizeof(double) * NVAR * n_pts, cudaMemcpyDeviceToHost, c->stream));
  return check_status(c);
}

icarus_status icarus_flag_refine(icarus_ctx *c, const icarus_refine *crit, int8_t *flags_out) {
  if (!c || !crit) return ICARUS_ERR_ARG;
  if (crit->mode < ICARUS_FLAG_PLAIN || crit->mode > ICARUS_FLAG_COMBINED) return ICARUS_ERR_ARG;
  if ((crit->mode == ICARUS_FLAG_TRACER || crit->mode == ICARUS_FLAG_COMBINED) && !c->d.tracer)
    return ICARUS_ERR_STATE;
  if (c->poisoned) return ICARUS_ERR_STATE;
  if (!c->ghosts_fresh) {
    enqueue_ghost(c, c->U, 0.0);
    c->ghosts_fresh = true;
  }
  if (crit->mode >= ICARUS_FLAG_SHOCK) {
    // shock (0), tracer (1) or combined (2) criterion
    const int which = crit->mode - ICARUS_FLAG_SHOCK;
    const double w[6] = {crit->div_thr, crit->dlon_earth, crit->dcolat_earth, crit->dlon_cme, crit->x_thr,
                         (double)which};
    if (!(w[0] >= 0.0) || !(w[1] < M_PI) || !(w[2] < M_PI) || !(w[3] < M_PI) || !(w[4] >= 0.0))
      return ICARUS_ERR_ARG;
    ProfScope p(c, 7);
    shock_estimator_launch(c->kp, c->U, c->prec, 0, c->nleaves, w, c->flags, c->stream);
  } else {
    ProfScope p(c, 7);
    estimator_launch(c->kp, c->U, c->prec, 0, c->nleaves, crit->e_refine, crit->e_coarsen, crit->eps, crit->dv,
                     c->flags, c->stream);
  }
  if (crit->mode == ICARUS_FLAG_LEARNED) {
    if (!c->mlp_ready) return ICARUS_ERR_STATE;
    for (int k = 0; k < 3; k++)
      if (c->d.block[k] % 4) return ICARUS_ERR_ARG;   // the features' sub-cubes
    mlp_leaf_probabilities(c);
    mlp_combine_launch(c->mlp_prob, c->blk, c->flags, c->nleaves, c->stream);
  }
  CK(cudaPeekAtLastError());
  c->hflags.assign(c->nleaves, 0);
  CK(cudaMemcpyAsync(c->hflags.data(), c->flags, c->nleaves, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (flags_out) memcpy(flags_out, c->hflags.data(), c->nleaves);
  c->flags_valid = true;
  return ICARUS_OK;
}

icarus_status icarus_set_flags(icarus_ctx *c, const int8_t *flags) {
  if (!c || !flags) return ICARUS_ERR_ARG;
  c->hflags.assign((const signed char *)flags, (const signed char *)flags + c->nleaves);
  c->flags_valid = true;
  return ICARUS_OK;
}

icarus_status icarus_regrid(icarus_ctx *c) {
  if (!c) return ICARUS_ERR_ARG;
  const bool fresh = c->ghosts_fresh;   // e.g. filled by the flagging just before
  c->ghosts_fresh = false;
  if (c->poisoned) return ICARUS_ERR_STATE;
  if (!c->flags_valid) return ICARUS_ERR_STATE;
  if (c->d.max_level == 1) {
    c->flags_valid = false;
    return ICARUS_OK;
  }
  // ghosts of the current state: prolongation reads the parents' halos
  if (!fresh) enqueue_ghost(c, c->U, 0.0);
  CK(cudaPeekAtLastError());
  std::vector<MoveOp> ops;
  std::vector<Member> next(c->d.n_members);
  int slot = 0;
  for (int m = 0; m < c->d.n_members; m++) {
    const Member &M = c->mem[m];
    const int n = (int)M.leaves.size();
    const signed char *fl = c->hflags.data() + c->mem_off[m];
    std::vector<int> T(n);
    for (int i = 0; i < n; i++) {
      T[i] = M.leaves[i].level;
      if (fl[i] > 0 && M.leaves[i].level < M.max_level) T[i]++;
    }
    // complete sibling families flagged -1 coarsen (a family is contiguous in
    // Morton order and starts at child 0)
    for (int i = 0; i + 7 < n; i++) {
      const Leaf &l = M.leaves[i];
      if (l.level == 1 || (l.ix[0] & 1) || (l.ix[1] & 1) || (l.ix[2] & 1)) continue;
      bool fam = true;
      for (int q = 0; q < 8 && fam; q++) {
        const Leaf &s = M.leaves[i + q];
        const int o[3] = {(q >> 2) & 1, (q >> 1) & 1, q & 1};
        if (s.level != l.level || fl[i + q] >= 0) fam = false;
        for (int d = 0; d < 3; d++)
          if (s.ix[d] != l.ix[d] + o[d]) fam = false;
      }
      if (fam)
        for (int q = 0; q < 8; q++) T[i + q] = l.level - 1;
    }
    // 2:1 balance, least fixed point
    // neighbour lists in one flat array, NB_MAX per leaf (found in parallel:
    // the lookups only read the member's maps)
    std::vector<int> nb_cnt(n), nb_all((size_t)n * NB_MAX);
#pragma omp parallel
    {
      std::vector<int> tmp;
      tmp.reserve(NB_MAX);
#pragma omp for schedule(static)
      for (int i = 0; i < n; i++) {
        neighbours(c, M, i, tmp);
        const int k = std::min<int>((int)tmp.size(), NB_MAX);
        std::copy(tmp.begin(), tmp.begin() + k, nb_all.begin() + (size_t)i * NB_MAX);
        nb_cnt[i] = k;
      }
    }
    bool changed = true;
    while (changed) {
      changed = false;
      for (int i = 0; i < n; i++) {
        for (int e = i * NB_MAX; e < i * NB_MAX + nb_cnt[i]; e++) {
          const int j = nb_all[e];
          if (T[j] > T[i] + 1) {
            if (T[i] < M.leaves[i].level) {
              // cancel the family's coarsening: find child 0 of the family
              const Leaf &l = M.leaves[i];
              int b[3] = {l.ix[0] & ~1, l.ix[1] & ~1, l.ix[2] & ~1};
              const int first = M.map[l.level][map_index(c, l.level, b)];
              for (int q = 0; q < 8; q++) T[first + q] = l.level;
            } else {
              T[i] = M.leaves[i].level + 1;
            }
            changed = true;
          }
        }
      }
    }
    // new leaf list (Morton order preserved) and data movement
    Member &N = next[m];
    N.max_level = M.max_level;
    N.cme = M.cme;
    for (int i = 0; i < n;) {
      const Leaf &l = M.leaves[i];
      const int old_slot = c->mem_off[m] + i;
      if (T[i] == l.level + 1) {
        for (int ch = 0; ch < 8; ch++) {
          Leaf k{l.level + 1, {2 * l.ix[0] + ((ch >> 2) & 1), 2 * l.ix[1] + ((ch >> 1) & 1), 2 * l.ix[2] + (ch & 1)}};
          N.leaves.push_back(k);
          MoveOp op{};
          op.kind = 1;
          op.dst = slot++;
          op.src[0] = old_slot;
          ops.push_back(op);
        }
        i++;
      } else if (T[i] == l.level - 1) {
        Leaf p{l.level - 1, {l.ix[0] >> 1, l.ix[1] >> 1, l.ix[2] >> 1}};
        N.leaves.push_back(p);
        MoveOp op{};
        op.kind = 2;
        op.dst = slot++;
        for (int q = 0; q < 8; q++) op.src[q] = old_slot + q;
        ops.push_back(op);
        i += 8;
      } else {
        N.leaves.push_back(l);
        MoveOp op{};
        op.kind = 0;
        op.dst = slot++;
        op.src[0] = old_slot;
        ops.push_back(op);
        i++;
      }
    }
  }
  if (slot > c->lay.max_blocks) return ICARUS_ERR_CAPACITY;
  // old tables stay valid for the movement kernel: build the new ones in the
  // alternate block table
  KParams kp_old = c->kp;
  std::vector<Member> old = std::move(c->mem);
  c->mem = std::move(next);
  // the new level maps are built by the tree check after the move
  // upload the new block table into blk_alt first (the move kernel needs the
  // new block coordinates and the old table at the same time)
  icarus_status st;
  {
    // compute the new host block table without touching device level maps yet
    std::vector<DevBlock> nb;
    int s2 = 0;
    for (int m = 0; m < c->d.n_members; m++)
      for (const Leaf &l : c->mem[m].leaves) {
        DevBlock B{};
        B.member = m;
        B.level = l.level;
        for (int d = 0; d < 3; d++) B.ix[d] = l.ix[d];
        nb.push_back(B);
        s2++;
      }
    CK(cudaMemcpyAsync(c->blk_alt, nb.data(), sizeof(DevBlock) * nb.size(), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->ops, ops.data(), sizeof(MoveOp) * ops.size(), cudaMemcpyHostToDevice, c->stream));
    {
      ProfScope p(c, 8);
      regrid_move_launch2(kp_old, c->U, c->Ualt, c->blk_alt, c->prec, c->ops, (int)ops.size(), c->stream);
    }
    CK(cudaPeekAtLastError());
    CK(cudaStreamSynchronize(c->stream));
  }
  std::swap(c->U, c->Ualt);
  // the new trees must be balanced and cover the domain (a failure here is a
  // defect of the balance step, reported rather than stepped through)
  for (int m = 0; m < c->d.n_members; m++)
    if (!tree_is_valid(c, c->mem[m])) {
      fprintf(stderr, "libicarus: regrid produced an invalid tree for member %d\n", m);
      c->poisoned = true;
      return ICARUS_ERR_STATE;
    }
  if ((st = upload_tree(c, c->blk)) != ICARUS_OK) return st;
  fill_kp(c);
  st = recompute_dt(c);
  if (st != ICARUS_OK) return st;
  CK(cudaStreamSynchronize(c->stream));
  c->flags_valid = false;
  return ICARUS_OK;
}

icarus_status icarus_set_fp64_islands(icarus_ctx *c, double p_over_e, double beta) {
  if (!c || !(p_over_e >= 0.0) || !(beta >= 0.0)) return ICARUS_ERR_ARG;
  c->ghosts_fresh = false;
  c->isl_pe = p_over_e;
  c->isl_beta = beta;
  fill_kp(c);
  c->graph_valid = false;
  return ICARUS_OK;
}

icarus_status icarus_set_floor_budget(icarus_ctx *c, double max_fraction) {
  if (!c || !(max_fraction >= 0.0)) return ICARUS_ERR_ARG;
  c->floor_budget = max_fraction;
  fill_kp(c);
  c->graph_valid = false;
  return ICARUS_OK;
}

icarus_status icarus_profile(icarus_ctx *c, int enable) {
  if (!c) return ICARUS_ERR_ARG;
  c->prof_on = enable != 0;
  c->ev_used = 0;
  return ICARUS_OK;
}

icarus_status icarus_profile_read(icarus_ctx *c, double *ms, int *count, int nkinds) {
  if (!c || !ms || !count || nkinds < 1 || nkinds > 10) return ICARUS_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < nkinds; k++) {
    ms[k] = 0.0;
    count[k] = 0;
  }
  for (size_t p = 0; p + 1 < c->ev_used; p += 2) {
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, c->ev[p], c->ev[p + 1]));
    const int k = c->ev_kind[p / 2];
    if (k < nkinds) {
      ms[k] += t;
      count[k]++;
    }
  }
  c->ev_used = 0;
  return ICARUS_OK;
}

}  // extern "C"

// Read-only view of one member's leaves for kernels that live outside this
// file (no state is changed).
int ctx_device(const icarus_ctx *c) { return c ? c->dev : -1; }

int ctx_member_view(icarus_ctx *c, int member, KParams *kp, const void **U, int *precision, int *slot0, int *nleaves,
                    cudaStream_t *stream) {
  if (!c || member < 0 || member >= c->d.n_members) return -1;
  *kp = c->kp;
  *U = c->U;
  *precision = c->prec;
  *slot0 = c->mem_off[member];
  *nleaves = (int)c->mem[member].leaves.size();
  *stream = c->stream;
  return 0;
}

extern "C" {

// ---- learned pre-flagger ----
icarus_status icarus_mlp_set_params(icarus_ctx *c, const float *host, size_t n) {
  if (!c || !host || n != (size_t)mlp_n_params()) return ICARUS_ERR_ARG;
  const size_t bytes = n * sizeof(float);
  CK(cudaMemcpyAsync(c->mlp_theta, host, bytes, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(c->mlp_m, 0, bytes, c->stream));
  CK(cudaMemsetAsync(c->mlp_v, 0, bytes, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->mlp_step = 0;
  c->mlp_ready = true;
  return ICARUS_OK;
}

icarus_status icarus_mlp_get_params(icarus_ctx *c, float *host, size_t n) {
  if (!c || !host || n != (size_t)mlp_n_params()) return ICARUS_ERR_ARG;
  CK(cudaMemcpyAsync(host, c->mlp_theta, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return ICARUS_OK;
}

icarus_status icarus_mlp_features(icarus_ctx *c, float *host_out) {
  if (!c) return ICARUS_ERR_ARG;
  for (int k = 0; k < 3; k++)
    if (c->d.block[k] % 4) return ICARUS_ERR_ARG;
  enqueue_ghost(c, c->U, 0.0);
  mlp_features_launch(c->kp, c->U, c->prec, 0, c->nleaves, c->mlp_feat, c->stream);
  CK(cudaPeekAtLastError());
  if (host_out)
    CK(cudaMemcpyAsync(host_out, c->mlp_feat, sizeof(float) * 64 * c->nleaves, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return ICARUS_OK;
}

icarus_status icarus_mlp_predict_leaves(icarus_ctx *c, float *prob_host) {
  if (!c || !prob_host) return ICARUS_ERR_ARG;
  if (!c->mlp_ready) return ICARUS_ERR_STATE;
  for (int k = 0; k < 3; k++)
    if (c->d.block[k] % 4) return ICARUS_ERR_ARG;
  mlp_leaf_probabilities(c);
  CK(cudaPeekAtLastError());
  CK(cudaMemcpyAsync(prob_host, c->mlp_prob, sizeof(float) * c->nleaves, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return ICARUS_OK;
}

icarus_status icarus_mlp_predict(icarus_ctx *c, const float *x_host, int n, float *y_host) {
  if (!c || !x_host || !y_host || n < 0 || n > MLP_BMAX) return ICARUS_ERR_ARG;
  if (!c->mlp_ready) return ICARUS_ERR_STATE;
  CK(cudaMemcpyAsync(c->mlp_xin, x_host, sizeof(float) * 64 * n, cudaMemcpyHostToDevice, c->stream));
  mlp_forward_launch(c->mlp_theta, c->mlp_xin, nullptr, n, c->mlp_h1, c->mlp_h2, c->mlp_y, c->stream);
  CK(cudaPeekAtLastError());
  CK(cudaMemcpyAsync(y_host, c->mlp_y, sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return ICARUS_OK;
}

icarus_status icarus_mlp_grad(icarus_ctx *c, const float *x_host, const float *t_host, int n, float *grad_host,
                              float *loss_out) {
  if (!c || !x_host || !t_host || !grad_host || n < 1 || n > MLP_BMAX) return ICARUS_ERR_ARG;
  if (!c->mlp_ready) return ICARUS_ERR_STATE;
  CK(cudaMemcpyAsync(c->mlp_xin, x_host, sizeof(float) * 64 * n, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->mlp_tin, t_host, sizeof(float) * n, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(c->mlp_loss, 0, sizeof(float), c->stream));
  mlp_forward_launch(c->mlp_theta, c->mlp_xin, nullptr, n, c->mlp_h1, c->mlp_h2, c->mlp_y, c->stream);
  mlp_backward_launch(c->mlp_theta, c->mlp_xin, c->mlp_tin, nullptr, n, c->mlp_h1, c->mlp_h2, c->mlp_y, c->mlp_dz,
                      c->mlp_dh2, c->mlp_dh1, c->mlp_grad, c->mlp_loss, c->stream);
  CK(cudaPeekAtLastError());
  CK(cudaMemcpyAsync(grad_host, c->mlp_grad, sizeof(float) * mlp_n_params(), cudaMemcpyDeviceToHost, c->stream));
  float l = 0.f;
  CK(cudaMemcpyAsync(&l, c->mlp_loss, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (loss_out) *loss_out = l / (float)n;
  return ICARUS_OK;
}

icarus_status icarus_mlp_dataset_clear(icarus_ctx *c) {
  if (!c) return ICARUS_ERR_ARG;
  c->mlp_n = 0;
  return ICARUS_OK;
}

icarus_status icarus_mlp_dataset_add(icarus_ctx *c, const float *x_host, const float *t_host, int n, int *total) {
  if (!c || n < 0 || (n && (!x_host || !t_host))) return ICARUS_ERR_ARG;
  if (c->mlp_n + n > MLP_CAP) return ICARUS_ERR_CAPACITY;
  if (n) {
    CK(cudaMemcpyAsync(c->mlp_X + (size_t)c->mlp_n * 64, x_host, sizeof(float) * 64 * n, cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(c->mlp_T + c->mlp_n, t_host, sizeof(float) * n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  c->mlp_n += n;
  if (total) *total = c->mlp_n;
  return ICARUS_OK;
}

icarus_status icarus_mlp_train(icarus_ctx *c, int n_train, int epochs, int batch, double lr, uint64_t seed,
                               float *loss_per_epoch) {
  if (!c || n_train < 1 || n_train > c->mlp_n || epochs < 0 || batch < 1 || batch > MLP_BMAX || !(lr > 0.0))
    return ICARUS_ERR_ARG;
  if (!c->mlp_ready) return ICARUS_ERR_STATE;
  std::vector<int> perm;
  uint64_t st = seed;
  for (int e = 0; e < epochs; e++) {
    permutation(perm, n_train, st);
    CK(cudaMemcpyAsync(c->mlp_idx, perm.data(), sizeof(int) * n_train, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->mlp_loss, 0, sizeof(float), c->stream));
    for (int b0 = 0; b0 < n_train; b0 += batch) {
      const int B = std::min(batch, n_train - b0);
      const int *idx = c->mlp_idx + b0;
      mlp_forward_launch(c->mlp_theta, c->mlp_X, idx, B, c->mlp_h1, c->mlp_h2, c->mlp_y, c->stream);
      mlp_backward_launch(c->mlp_theta, c->mlp_X, c->mlp_T, idx, B, c->mlp_h1, c->mlp_h2, c->mlp_y, c->mlp_dz,
                          c->mlp_dh2, c->mlp_dh1, c->mlp_grad, c->mlp_loss, c->stream);
      mlp_adam_launch(c->mlp_theta, c->mlp_grad, c->mlp_m, c->mlp_v, (float)lr, ++c->mlp_step, c->stream);
    }
    CK(cudaPeekAtLastError());
    float l = 0.f;
    CK(cudaMemcpyAsync(&l, c->mlp_loss, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (loss_per_epoch) loss_per_epoch[e] = l;
  }
  return ICARUS_OK;
}

}  // extern "C"


// ======================================================================
// Checkpoint / resume.  A checkpoint holds everything a step reads: the
// descriptor fields that fix the grid and the physics (checked on load), per
// member its finest level, cone CME, leaf tree, time, CFL time step and
// cell-update count, the inner-boundary maps and background speeds, the
// leaves' state in the working precision (with ghosts), the FP64-island
// thresholds, the floor-hit count and, if set, the pre-flagger's parameters.
namespace {

const char CK_MAGIC[8] = {'I', 'C', 'A', 'R', 'U', 'S', 'C', 'K'};
const uint32_t CK_VERSION = 1;

// the descriptor fields a checkpoint must agree on, in a fixed order
std::vector<double> ck_fingerprint(const icarus_grid_desc &d) {
  std::vector<double> f;
  for (int k = 0; k < 3; k++) f.push_back(d.n_cells[k]);
  for (int k = 0; k < 3; k++) f.push_back(d.block[k]);
  f.push_back(d.max_level);
  f.push_back(d.radial_stretch);
  f.push_back(d.geometry);
  for (int k = 0; k < 3; k++) f.push_back(d.x_min[k]);
  for (int k = 0; k < 3; k++) f.push_back(d.x_max[k]);
  f.push_back(d.gamma);
  f.push_back(d.omega);
  f.push_back(d.cfl);
  f.push_back(d.divb_cd);
  f.push_back(d.p_floor);
  f.push_back(d.rho_floor);
  f.push_back(d.precision);
  f.push_back(d.n_members);
  for (int k = 0; k < 3; k++) f.push_back(d.bc_lo[k]);
  for (int k = 0; k < 3; k++) f.push_back(d.bc_hi[k]);
  f.push_back(d.tracer);
  return f;
}

struct CkFile {
  FILE *f = nullptr;
  bool ok = true;
  ~CkFile() {
    if (f) fclose(f);
  }
  void put(const void *p, size_t n) {
    if (ok && n && fwrite(p, 1, n, f) != n) ok = false;
  }
  void get(void *p, size_t n) {
    if (ok && n && fread(p, 1, n, f) != n) ok = false;
  }
};

size_t slot_bytes(const icarus_ctx *c) { return (size_t)c->kp.nvs * c->kp.pcells * c->rsize; }

}  // namespace

extern "C" {

icarus_status icarus_save(icarus_ctx *c, const char *path) {
  if (!c || !path) return ICARUS_ERR_ARG;
  const int nm = c->d.n_members;
  const size_t nbc = (size_t)c->d.n_cells[0] * c->d.n_cells[1] * c->d.n_cells[2];
  const size_t nbm = (size_t)NVAR * c->d.n_cells[1] * c->d.n_cells[2];
  std::vector<double> t(nm), dtc(nm), upd(nm), bmap(nm * nbm), vbg(nm * nbc);
  unsigned long long hits = 0;
  std::vector<unsigned char> U(slot_bytes(c) * c->nleaves);
  std::vector<float> theta(c->mlp_ready ? mlp_n_params() : 0);
  cudaStream_t s = c->stream;
  CK(cudaMemcpyAsync(t.data(), c->t, sizeof(double) * nm, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(dtc.data(), c->dt_cfl, sizeof(double) * nm, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(upd.data(), c->updates, sizeof(double) * nm, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(bmap.data(), c->bmap, sizeof(double) * bmap.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(vbg.data(), c->vbg, sizeof(double) * vbg.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&hits, c->floor_hits, sizeof(hits), cudaMemcpyDeviceToHost, s));
  if (!U.empty()) CK(cudaMemcpyAsync(U.data(), c->U, U.size(), cudaMemcpyDeviceToHost, s));
  if (!theta.empty())
    CK(cudaMemcpyAsync(theta.data(), c->mlp_theta, sizeof(float) * theta.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CkFile F;
  F.f = fopen(path, "wb");
  if (!F.f) return ICARUS_ERR_ARG;
  F.put(CK_MAGIC, 8);
  F.put(&CK_VERSION, sizeof(CK_VERSION));
  const std::vector<double> fp = ck_fingerprint(c->d);
  const uint32_t nfp = (uint32_t)fp.size();
  F.put(&nfp, sizeof(nfp));
  F.put(fp.data(), sizeof(double) * fp.size());
  for (int m = 0; m < nm; m++) {
    const Member &M = c->mem[m];
    const int32_t hdr[2] = {M.max_level, (int32_t)M.leaves.size()};
    F.put(hdr, sizeof(hdr));
    F.put(&M.cme, sizeof(DevCme));
    for (const Leaf &l : M.leaves) {
      const int32_t row[4] = {l.level, l.ix[0], l.ix[1], l.ix[2]};
      F.put(row, sizeof(row));
    }
  }
  F.put(t.data(), sizeof(double) * nm);
  F.put(dtc.data(), sizeof(double) * nm);
  F.put(upd.data(), sizeof(double) * nm);
  F.put(bmap.data(), sizeof(double) * bmap.size());
  F.put(vbg.data(), sizeof(double) * vbg.size());
  F.put(&hits, sizeof(hits));
  const double isl[2] = {c->isl_pe, c->isl_beta};
  F.put(isl, sizeof(isl));
  F.put(U.data(), U.size());
  const int32_t nth = (int32_t)theta.size();
  F.put(&nth, sizeof(nth));
  F.put(theta.data(), sizeof(float) * theta.size());
  return F.ok ? ICARUS_OK : ICARUS_ERR_ARG;
}

icarus_status icarus_load(icarus_ctx *c, const char *path) {
  if (!c || !path) return ICARUS_ERR_ARG;
  c->ghosts_fresh = false;
  const int nm = c->d.n_members;
  const size_t nbc = (size_t)c->d.n_cells[0] * c->d.n_cells[1] * c->d.n_cells[2];
  const size_t nbm = (size_t)NVAR * c->d.n_cells[1] * c->d.n_cells[2];
  CkFile F;
  F.f = fopen(path, "rb");
  if (!F.f) return ICARUS_ERR_ARG;
  char magic[8];
  uint32_t ver = 0, nfp = 0;
  F.get(magic, 8);
  F.get(&ver, sizeof(ver));
  F.get(&nfp, sizeof(nfp));
  const std::vector<double> fp = ck_fingerprint(c->d);
  if (!F.ok || memcmp(magic, CK_MAGIC, 8) != 0 || ver != CK_VERSION || nfp != fp.size()) return ICARUS_ERR_ARG;
  std::vector<double> fq(nfp);
  F.get(fq.data(), sizeof(double) * nfp);
  if (!F.ok || memcmp(fq.data(), fp.data(), sizeof(double) * nfp) != 0) return ICARUS_ERR_ARG;
  std::vector<Member> next(nm);
  size_t total = 0;
  for (int m = 0; m < nm; m++) {
    int32_t hdr[2] = {0, 0};
    F.get(hdr, sizeof(hdr));
    if (!F.ok || hdr[0] < 1 || hdr[0] > c->d.max_level || hdr[1] < 1) return ICARUS_ERR_ARG;
    // a corrupt count must not reach the allocation below
    if ((size_t)hdr[1] > (size_t)c->lay.max_blocks - total) return ICARUS_ERR_CAPACITY;
    next[m].max_level = hdr[0];
    F.get(&next[m].cme, sizeof(DevCme));
    next[m].leaves.resize(hdr[1]);
    for (Leaf &l : next[m].leaves) {
      int32_t row[4];
      F.get(row, sizeof(row));
      if (!F.ok || row[0] < 1 || row[0] > c->d.max_level) return ICARUS_ERR_ARG;
      l.level = row[0];
      for (int d = 0; d < 3; d++) {
        l.ix[d] = row[1 + d];
        if (l.ix[d] < 0 || l.ix[d] >= nblk_dim(c, l.level, d)) return ICARUS_ERR_ARG;
      }
    }
    if (!tree_is_valid(c, next[m])) return ICARUS_ERR_ARG;
    total += next[m].leaves.size();
  }
  std::vector<double> t(nm), dtc(nm), upd(nm), bmap(nm * nbm), vbg(nm * nbc);
  unsigned long long hits = 0;
  double isl[2];
  F.get(t.data(), sizeof(double) * nm);
  F.get(dtc.data(), sizeof(double) * nm);
  F.get(upd.data(), sizeof(double) * nm);
  F.get(bmap.data(), sizeof(double) * bmap.size());
  F.get(vbg.data(), sizeof(double) * vbg.size());
  F.get(&hits, sizeof(hits));
  F.get(isl, sizeof(isl));
  std::vector<unsigned char> U(slot_bytes(c) * total);
  F.get(U.data(), U.size());
  int32_t nth = 0;
  F.get(&nth, sizeof(nth));
  if (!F.ok || (nth != 0 && nth != mlp_n_params())) return ICARUS_ERR_ARG;
  std::vector<float> theta(nth);
  F.get(theta.data(), sizeof(float) * nth);
  if (!F.ok) return ICARUS_ERR_ARG;
  // everything read: replace the context's state
  c->mem = std::move(next);
  for (Member &M : c->mem) build_member_map(c, M);
  icarus_status st = upload_tree(c, c->blk);
  if (st != ICARUS_OK) return st;
  c->isl_pe = isl[0];
  c->isl_beta = isl[1];
  fill_kp(c);
  cudaStream_t s = c->stream;
  for (int m = 0; m < nm; m++) CK(cudaMemcpyAsync(c->cme + m, &c->mem[m].cme, sizeof(DevCme), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->t, t.data(), sizeof(double) * nm, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->dt_cfl, dtc.data(), sizeof(double) * nm, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->updates, upd.data(), sizeof(double) * nm, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->bmap, bmap.data(), sizeof(double) * bmap.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->vbg, vbg.data(), sizeof(double) * vbg.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->floor_hits, &hits, sizeof(hits), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->floor_prev, &hits, sizeof(hits), cudaMemcpyHostToDevice, s));   // the budget counts from here
  CK(cudaMemsetAsync(c->status, 0, sizeof(unsigned int), s));
  c->status_pending = false;
  if (!U.empty()) CK(cudaMemcpyAsync(c->U, U.data(), U.size(), cudaMemcpyHostToDevice, s));
  if (nth) {
    CK(cudaMemcpyAsync(c->mlp_theta, theta.data(), sizeof(float) * nth, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(c->mlp_m, 0, sizeof(float) * nth, s));
    CK(cudaMemsetAsync(c->mlp_v, 0, sizeof(float) * nth, s));
    c->mlp_step = 0;
    c->mlp_ready = true;
  } else {
    c->mlp_ready = false;   // the saved context had no pre-flagger parameters
  }
  CK(cudaStreamSynchronize(s));
  c->poisoned = false;
  c->flags_valid = false;
  c->graph_valid = false;
  return ICARUS_OK;
}

}  // extern "C"
