// Internal types of libicarus shared by the host runtime and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define NVAR 8
#define TRV 8          // index of the CME tracer rho X in a slot (when stored)
#define NGH 2
#define MAXLEV 8

// status bits of the sticky device word
#define ST_NAN 1u
#define ST_FLOOR 2u
#define ST_TIMEOUT 4u
#define ST_TREE 8u       // a ghost cell's neighbour was not where the tree says (2:1 balance broken)

// face-neighbour relation of a leaf face
enum { NB_PHYS = 0, NB_SAME = 1, NB_COARSER = 2, NB_FINER = 3 };

// per-slot block record (slot == global leaf index)
struct DevBlock {
  int member, level;
  int ix[3];
  int nbr[6];      // NB_* per face (dir*2 + side)
  int phys;        // bit (2*d+side): block touches a non-periodic boundary there
  int lmax;        // finest level of the block's member
};

// 1D geometry tables of one level, indexed with an offset of NGH so that the
// ghost range is addressable.  Faces: f[I + NGH], I in [-NGH, N + NGH];
// cells: c[I + NGH], I in [-NGH, N + NGH).
template <typename real>
struct LevelGeo {
  const real *rf;    // radial faces
  const real *r2f;   // r_f^2 (Cartesian: 1)
  const real *dr3;   // (r+^3 - r-^3)/3 (Cartesian: dx)
  const real *dr2;   // (r+^2 - r-^2)/2 (Cartesian: dx)
  const real *rc;    // cell centre (arithmetic mid-point of the faces)
  const real *dr;    // r+ - r-
  const real *tf;    // colatitude faces
  const real *sinf;  // sin(theta_f) (Cartesian: 1)
  const real *dcos;  // cos(theta-) - cos(theta+) (Cartesian: dy)
  const real *tc;    // centre
  const real *sintc, *costc;
  const real *dth;   // theta+ - theta-
  const real *pf;    // phi faces
  const real *pc;    // phi centres
  real dphi;         // uniform phi width (Cartesian: dz)
  int n[3];
};

struct Geometry {
  LevelGeo<double> d[MAXLEV + 1];
  LevelGeo<float> f[MAXLEV + 1];
  // prolongation offsets of coarse level L, direction d: [2*Ic + child]
  const double *dlt[MAXLEV + 1][3];
  const float *dltf[MAXLEV + 1][3];
  // fine cell volume factors for restriction come from the fine level tables
};

template <typename real> struct GeoSel;
template <> struct GeoSel<double> {
  static __host__ __device__ const LevelGeo<double> &get(const Geometry *g, int L) { return g->d[L]; }
  static __host__ __device__ const double *dlt(const Geometry *g, int L, int d) { return g->dlt[L][d]; }
};
template <> struct GeoSel<float> {
  static __host__ __device__ const LevelGeo<float> &get(const Geometry *g, int L) { return g->f[L]; }
  static __host__ __device__ const float *dlt(const Geometry *g, int L, int d) { return g->dltf[L][d]; }
};

struct DevCme {
  double t_start, t_max, colat, lon, half_width, v, rho, p;
  int active, pad;
};

// Earth's direction for the windows of the shock criterion: colatitude and
// longitude lon0 - rate (t - t0) in the co-rotating frame
struct DevEarth {
  double colat, lon0, t0, rate;
  int set, pad;
};

// everything a kernel needs to know about the grid (passed by value)
struct KParams {
  int nb[3], P[3];
  int nvs;                     // variables stored per cell: NVAR, or NVAR + 1 with the CME tracer rho X
  int pad_nvs;
  int pcells, icells;
  int nbase[3];
  int n_members;
  int geometry;
  int bc_lo[3], bc_hi[3];
  double gamma, omega, cd, p_floor, rho_floor;
  const Geometry *geo;
  const DevBlock *blk;
  const int *nb27;             // [slot][27]: slot of the same-level leaf at block offset (dr, dth, dph) in
                               // {-1,0,1}^3, index (dr+1)*9 + (dth+1)*3 + (dph+1); -1 if none (coarser,
                               // finer or outside a non-periodic boundary)
  const int *lmap;             // level maps, concatenated
  const long long *lmap_off;   // [member * (MAXLEV+1) + L]
  const double *bmap;          // [member][8][n1][n2] inner boundary primitives
  const DevCme *cme;           // [member]
  const DevEarth *earth;       // [member]
  const double *vbg;           // [member][n0][n1][n2] background v_r
  double *t;                   // [member]
  double *dt_used;             // [member]
  double *dt_cfl;              // [member]
  double *updates;             // [member] cumulative leaf-cell updates
  const double *cells_m;       // [member] leaf cells of the member
  unsigned long long *inv_max; // [member] bit pattern of a positive double
  unsigned int *status;
  unsigned long long *floor_hits;
  unsigned long long *floor_prev;  // floor counter at the end of the previous step
  double floor_budget;         // floor hits per cell-update of a step that set ST_FLOOR (0: no budget)
  int n_base_cells[3];
  double isl_pe, isl_beta;     // FP64 pressure-island thresholds (FP32 mode)
};

// ---- launch wrappers (defined in the kernel translation units) ----
struct StageLaunch {
  const void *Uin;    // stage input (padded)
  const void *U0;     // base state U^n (padded)
  void *Uout;         // output (padded interior written)
  void *flux;         // reflux face buffer or nullptr
  const int *list;    // slots to update
  int nlist;
  int tiles_j, tiles_k, segs, seg_len;
  double dtfac;       // 0.5 (predictor) or 1 (corrector)
  int stage2;         // 1: cleaning, dt accumulation, reflux fluxes
  int direct;         // 1: halo cells held by a same-level leaf are read from its interior
  int tile_j, tile_k; // tile shape
  int grid;           // CTAs (persistent loop)
};
int stage_launch(const KParams &kp, const StageLaunch &sl, int precision, cudaStream_t s);
// longest radial segment a stage work item marches (its geometry is staged
// in shared memory)
constexpr int STAGE_SEG_MAX = 64;
// tracer: the CME tracer is stored and advected (one more shared ring)
size_t stage_smem_bytes(int precision, int tj, int tk, int tracer);
int stage_tile_supported(int precision, int tj, int tk, int tracer);
int stage_max_ctas_per_sm(int precision, int tj, int tk, int tracer);

// ghost fill
// ghost_neighbour: every ghost cell of the listed leaves (copy, prolongation
// or restriction); ghost_regions: work items of up to 32 cells (or 2x2x2
// groups) of the regions around a leaf held by a coarser or finer leaf, while the ghost cells same-level leaves
// hold are left unfilled (the stage kernels read them from those leaves, and
// prolongation and the physical-boundary copies with skip_same read such
// cells from the neighbour as well)
void ghost_neighbour_launch(const KParams &kp, void *U, int precision, const int *list, int nlist,
                            const int *shell, int nshell, int level, cudaStream_t s);
void ghost_regions_launch(const KParams &kp, void *U, int precision, const int2 *items, int nitems,
                          const int *rshell, int level, cudaStream_t s);
void ghost_physical_launch(const KParams &kp, void *U, int precision, const int2 *sides, int nsides,
                           int dir, int level, double tshift_fac, bool faces_only, bool skip_same, cudaStream_t s);
void reflux_launch(const KParams &kp, void *U, const void *flux, int precision, const int *list, int nlist,
                   cudaStream_t s);
void dt_begin_launch(const KParams &kp, const double *tstop, cudaStream_t s);
void dt_finalize_launch(const KParams &kp, double cfl, cudaStream_t s);
void dt_full_launch(const KParams &kp, const void *U, int precision, int nleaves, double cfl, cudaStream_t s);

// state and AMR support
void pack_state_launch(const KParams &kp, const void *U, int precision, int slot0, int nslots, double *out,
                       cudaStream_t s);
void unpack_state_launch(const KParams &kp, void *U, int precision, int slot0, int nslots, const double *in,
                         int is_prim, cudaStream_t s);
void estimator_launch(const KParams &kp, const void *U, int precision, int slot0, int nslots, double e_ref,
                      double e_crs, double eps, double dv, signed char *flags, cudaStream_t s);
// shock / tracer / combined criterion: crit = {div_thr, dlon_earth,
// dcolat_earth, dlon_cme, x_thr, which (0 shock, 1 tracer, 2 combined)}
void shock_estimator_launch(const KParams &kp, const void *U, int precision, int slot0, int nslots,
                            const double *crit, signed char *flags, cudaStream_t s);
struct MoveOp {       // one new leaf of a regrid
  int kind;           // 0 copy, 1 prolong from the old parent, 2 restrict from 8 old children
  int dst;            // new slot
  int src[8];         // old slots (copy/prolong: src[0]; restrict: children by child id)
};
void regrid_move_launch2(const KParams &kp_old, const void *Uold, void *Unew, const DevBlock *nblk, int precision,
                         const MoveOp *ops, int nops, cudaStream_t s);
void probe_launch2(const KParams &kp, const void *U, int precision, int member, int maxL, int npts,
                   const double *pts, double *out, cudaStream_t s);
void sums_launch(const KParams &kp, const void *U, int precision, int slot0, int nslots, double *partial,
                 cudaStream_t s);
void vbg_launch(const KParams &kp, const void *U, int precision, int member, int slot0, int nslots, double *vbg,
                cudaStream_t s);

// learned pre-flagger (k_mlp.cu)
int mlp_n_params();
void mlp_features_launch(const KParams &kp, const void *U, int precision, int slot0, int nslots, float *out,
                         cudaStream_t s);
void mlp_forward_launch(const float *theta, const float *X, const int *idx, int B, float *h1, float *h2, float *y,
                        cudaStream_t s);
void mlp_backward_launch(const float *theta, const float *X, const float *T, const int *idx, int B,
                         const float *h1, const float *h2, const float *y, float *dz, float *dh2, float *dh1,
                         float *grad, float *loss, cudaStream_t s);
void mlp_adam_launch(float *theta, const float *g, float *m, float *v, float lr, int step, cudaStream_t s);
void mlp_combine_launch(const float *prob, const DevBlock *blk, signed char *flags, int n, cudaStream_t s);

struct icarus_ctx;
int ctx_member_view(icarus_ctx *c, int member, KParams *kp, const void **U, int *precision, int *slot0,
                    int *nleaves, cudaStream_t *stream);
// CUDA device the context was created on
int ctx_device(const icarus_ctx *c);
// scratch of the allocation-free sums on device dev (k_sums_static.cu)
int static_sums_prepare(int dev);
