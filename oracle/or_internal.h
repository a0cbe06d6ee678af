/*
 * Plain FP64 CPU oracle for the Icarus finite-volume MHD update
 * (arXiv 2211.12867, Sect. 2.1-2.2 and 3).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists so that the CUDA library can be
 * checked against an independent, slow, obviously-correct implementation.  It
 * shares no code, header, table or constant with the CUDA library; only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may load it.
 *
 * Conventions (shared by every oracle source file):
 *   variables  U = (rho, m_r, m_th, m_ph, e, B_r, B_th, B_ph)   index 0..7
 *              W = (rho, v_r, v_th, v_ph, p, B_r, B_th, B_ph)
 *   units      length 1 AU, speed 100 km/s, density m_p cm^-3, B with mu0
 *              absorbed (normalised units of the grid descriptor).
 *   direction  0 = r (index i), 1 = theta (j), 2 = phi (k); Cartesian mode
 *              uses the same slots for x, y, z.
 *   blocks     padded with NG = 2 ghost layers; storage [v][i][j][k] with
 *              v = 0..7 the MHD variables and v = TR the CME tracer rho X
 *              (zero unless the tracer is on).
 */
#ifndef OR_INTERNAL_H
#define OR_INTERNAL_H
#include <stddef.h>
#include <stdint.h>

#define NV 8
#define NVT 9   /* storage per cell: the 8 MHD variables and the CME tracer rho X */
#define TR 8    /* index of the tracer in a block's storage */
#define NG 2
#define OR_MAXL 8

enum { RHO = 0, MR = 1, MT = 2, MP = 3, EN = 4, BR = 5, BT = 6, BP = 7 };
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_REFLECT = 2, BC_INNER = 3 };

typedef struct {
  int geometry;            /* 0 spherical, 1 cartesian */
  int n[3];                /* base-level cells per direction */
  int nb[3];               /* interior cells per block */
  int max_level;           /* 1 = single level */
  int stretch;             /* 1 = geometric radial faces (Sect. 2.2) */
  double xmin[3], xmax[3]; /* r [AU], colatitude [rad], longitude [rad] */
  double gamma, omega, cfl, divb_cd;
  int bc_lo[3], bc_hi[3];
  double p_floor, rho_floor;
  int tracer;              /* 1: advect the CME density tracer (Sect. 3.1) */
} or_params;

typedef struct {           /* cone CME, Eqs. 1-4; normalised units */
  double t_start, t_max, colat, lon, half_width, v, rho, p;
  int active;
} or_cme;

typedef struct {           /* Earth's direction for the shock windows (Sect. 3.2) */
  double colat, lon0, t0, rate;   /* longitude lon0 - rate (t - t0), co-rotating */
  int set;
} or_earth;

typedef struct ob ob;
struct ob {
  int level;               /* 1 = base */
  int ix[3];               /* block index at its own level */
  ob *parent;
  ob *child[8];            /* child c = (a<<2)|(b<<1)|c3 for offsets a,b,c3 */
  int is_leaf;
  double *U, *Us;          /* padded state and stage state, NVT variables */
  double *fx[6];           /* area x flux on faces (lo/hi per dir), [cell][v] */
  int nbr_level[6];        /* level of face-neighbour region owner (0 = boundary) */
  signed char flag;
  int id;                  /* position in the leaf list during regrid */
};

typedef struct {
  or_params p;
  int nbase[3];
  ob *base;                /* nbase[0]*nbase[1]*nbase[2] */
  ob **leaves;
  int nleaves, cap_leaves;
  double *xf[3][OR_MAXL + 1];     /* faces per direction and level, offset NG */
  double *dlt[3][OR_MAXL + 1];    /* prolongation offsets [coarse cell][2] */
  double *map;             /* inner boundary primitives [8][n1][n2] */
  double *vbg;             /* background v_r per base cell, or NULL */
  or_cme cme;
  or_earth earth;
  double t;
  long floor_hits;
  int nthreads;
} or_grid;

/* pointwise physics (or_physics.c) */
void or_prim2cons(const double *W, double *U, double gamma);
void or_cons2prim(const double *U, double *W, double gamma);
double or_fast_speed(const double *W, int d, double gamma);
double or_mc_slope(double um, double u0, double up);
void or_phys_flux(const double *W, const double *U, int d, double *F);
void or_tvdlf(const double *WL, const double *WR, int d, double gamma, double *F);
double or_cme_opening(const or_cme *c, double R, double t);
double or_cme_distance(const or_cme *c, double colat, double lon);
double or_loehner(const double *um, const double *u0c, const double *up, double eps);

/* grid helpers (or_grid.c) */
int or_pdim(const or_grid *g, int d);
size_t or_pcells(const or_grid *g);
double or_face(const or_grid *g, int L, int d, int I);
double or_centre(const or_grid *g, int L, int d, int I);
int or_ncells(const or_grid *g, int L, int d);

#endif
