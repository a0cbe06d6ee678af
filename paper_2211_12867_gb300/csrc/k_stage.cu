// Stage operator of the midpoint predictor-corrector on every leaf block.
//
//   predictor  U*      = U^n + dt/2 L(U^n)
//   corrector  U^{n+1} = U^n + dt   L(U*) + cleaning(U*)
//
// L(U) = -(1/V) sum_faces A F_TVDLF + S_geometric + S_rotation (arXiv
// 2211.12867, Sect. 2.1: TVDLF with the Woodward limiter, second order in space
// and time, ideal MHD in the co-rotating frame, parabolic div B cleaning).
// Geometric sources come from the spherical divergence of the momentum and
// induction tensors with the pressure parts in face-area-difference form (a
// uniform state is preserved to round-off); rotation sources are the Coriolis
// and centrifugal forces with the centrifugal work.  Cleaning is the
// diffusive (parabolic) form dB = C_d h^2 grad(div B*), de = B*.dB, with
// central differences and h^-2 = sum_d dx_d^-2.
//
// GPU design: one CTA owns a (theta x phi) tile of one block and marches along
// r.  Primitives of five consecutive r-planes live in a shared-memory ring
// (each cell of the tile plus its 2-cell halo is loaded and converted once per
// CTA); the r-face flux is carried in registers from one plane to the next;
// theta and phi face fluxes are computed once per face into shared memory and
// read by the two cells that share the face; div B of the corrector lives in a
// 4-plane ring.  The corrector also accumulates the CFL time step of the new
// state (FP64 max of the inverse time step per member) and stores the
// area-weighted face fluxes of block faces that border a different level for
// the reflux.  The grid is persistent: CTAs stride over (block, tile,
// r-segment) work items of all levels and all ensemble members.
#include <cstdio>

#include "mhd_device.cuh"

namespace {

template <typename real>
struct StageSmem {
  // tracer: a 5-plane ring of the CME tracer fraction X follows the rest
  static constexpr size_t bytes(int tj, int tk, bool tracer = false) {
    return sizeof(real) * (size_t)(5 * NVAR * (tj + 4) * (tk + 4) + 2 * NVAR * (tj + 1) * tk +
                                   2 * NVAR * tj * (tk + 1) + 4 * (tj + 2) * (tk + 2) +
                                   NVAR * ((tj * tk + 31) / 32 * 32) + geo(tj, tk) +
                                   (tracer ? 5 * (tj + 4) * (tk + 4) : 0));
  }
  // geometry of one work item: 6 plane arrays and the faces in r, 6 row
  // arrays and the faces in theta, 1 column array
  static constexpr int geo(int tj, int tk) {
    return 6 * (STAGE_SEG_MAX + 4) + (STAGE_SEG_MAX + 5) + 6 * (tj + 4) + (tj + 5) + (tk + 4);
  }
};

// The inverse time step is accumulated in the working precision (a maximum is
// exact in any precision) and enters the FP64 reduction once per warp.
template <typename real>
__device__ __forceinline__ void flush_acc(const KParams &kp, real &acc, int member, long long &hits) {
  // warp max of the inverse time step, one atomic per warp
  for (int o = 16; o > 0; o >>= 1) acc = RT<real>::max_(acc, __shfl_xor_sync(0xffffffffu, acc, o));
  long long h = hits;
  for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
  if ((threadIdx.x & 31) == 0 && member >= 0) {
    if (acc > real(0)) atomic_max_pos(&kp.inv_max[member], (double)acc);
    if (h) atomicAdd(kp.floor_hits, (unsigned long long)h);
  }
  acc = real(0);
  hits = 0;
}

// Shared arrays of 8-variable cells (the primitive ring, the face fluxes) are
// stored as [NVAR / CH][cell][CH] with CH = 16 bytes / sizeof(real): a cell's
// variables come in NVAR / CH 16-byte loads and consecutive cells are
// consecutive vectors (no bank conflicts between neighbouring threads).
template <typename real> struct Vec16;
template <> struct Vec16<float> {
  using T = float4;
  static constexpr int CH = 4;
  static __device__ __forceinline__ void put(T x, float *w) { w[0] = x.x; w[1] = x.y; w[2] = x.z; w[3] = x.w; }
  static __device__ __forceinline__ T get(const float *w) { return make_float4(w[0], w[1], w[2], w[3]); }
};
template <> struct Vec16<double> {
  using T = double2;
  static constexpr int CH = 2;
  static __device__ __forceinline__ void put(T x, double *w) { w[0] = x.x; w[1] = x.y; }
  static __device__ __forceinline__ T get(const double *w) { return make_double2(w[0], w[1]); }
};
template <typename real, int N>
__device__ __forceinline__ void ld8(const real *a, int q, real *w) {
  using V = Vec16<real>;
#pragma unroll
  for (int c = 0; c < NVAR / V::CH; c++)
    V::put(*reinterpret_cast<const typename V::T *>(a + (c * N + q) * V::CH), w + c * V::CH);
}
template <typename real, int N>
__device__ __forceinline__ void st8(real *a, int q, const real *w) {
  using V = Vec16<real>;
#pragma unroll
  for (int c = 0; c < NVAR / V::CH; c++)
    *reinterpret_cast<typename V::T *>(a + (c * N + q) * V::CH) = V::get(w + c * V::CH);
}
// one variable of a cell in that layout
template <typename real, int N>
__device__ __forceinline__ real &el(real *a, int v, int q) {
  constexpr int CH = Vec16<real>::CH;
  return a[((v / CH) * N + q) * CH + v % CH];
}
template <typename real, int N>
__device__ __forceinline__ real el(const real *a, int v, int q) {
  constexpr int CH = Vec16<real>::CH;
  return a[((v / CH) * N + q) * CH + v % CH];
}

// threads per CTA: the tile's cells rounded up to whole warps (the extra
// threads own no cell but share the loads and the face fluxes)
constexpr int stage_threads(int tj, int tk) { return (tj * tk + 31) / 32 * 32; }
constexpr int cmin(int a, int b) { return a < b ? a : b; }
constexpr int cmax(int a, int b) { return a > b ? a : b; }
// resident CTAs per SM the register budget is sized for (FP32): as many as
// the shared memory of an SM (228 KB, 1 KB reserved per CTA) holds, and no
// more than leave 128 registers a thread; at least 2.  FP64: 1.
constexpr int stage_min_ctas(int real_bytes, int tj, int tk) {
  return real_bytes != 4 ? 1
                         : cmax(2, cmin(65536 / (stage_threads(tj, tk) * 128),
                                        (int)(233472 / (StageSmem<float>::bytes(tj, tk) + 1024))));
}

template <typename real, int TJ, int TK, bool S2>
__global__ void __launch_bounds__(stage_threads(TJ, TK), stage_min_ctas(sizeof(real), TJ, TK))
    k_stage(const KParams kp, const StageLaunch sl) {
  constexpr int NT = stage_threads(TJ, TK), RJ = TJ + 4, RK = TK + 4, RP = RJ * RK;
  constexpr int DJ = TJ + 2, DK = TK + 2, DP = DJ * DK;
  constexpr int NTH = (TJ + 1) * TK, NPH = TJ * (TK + 1);   // theta / phi faces of a plane
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real *ring = reinterpret_cast<real *>(smem_raw);
  real *fth = ring + 5 * NVAR * RP;     // two buffers of theta-face fluxes
  real *fph = fth + 2 * NVAR * NTH;     // two buffers of phi-face fluxes
  real *dring = fph + 2 * NVAR * NPH;
  real *u0s = dring + 4 * DP;           // U^n of the thread's own cell, next plane
  // geometry of the work item (plane arrays from plane ib-2, row arrays from
  // row -2 of the tile, phi centres from column -2)
  constexpr int NRP = STAGE_SEG_MAX + 4, NJ = TJ + 4;
  real *s_rc = u0s + NVAR * NT, *s_dr2 = s_rc + NRP, *s_dr3 = s_dr2 + NRP;
  real *s_r2f = s_dr3 + NRP;                                  // STAGE_SEG_MAX + 5 faces
  // reciprocal centre spacings over two cells (theta rows, phi columns, r
  // planes), reciprocal widths and radii: the divergence and the cleaning
  // gradient take these per row, column or plane
  real *s_itc2 = s_r2f + NRP + 1, *s_st = s_itc2 + NJ, *s_ct = s_st + NJ, *s_dcos = s_ct + NJ, *s_dth = s_dcos + NJ;
  real *s_sinf = s_dth + NJ;                                  // TJ + 5 faces
  real *s_ipc2 = s_sinf + NJ + 1;                             // TK + 4
  real *s_ird2 = s_ipc2 + TK + 4, *s_idr = s_ird2 + NRP, *s_irc = s_idr + NRP, *s_idth = s_irc + NRP;
  real *xring = s_idth + NJ;                                  // tracer X, 5 planes (if stored)
  const bool trc = kp.nvs > NVAR;

  const int tid = threadIdx.x, jl = tid / TK, kl = tid % TK;
  const real gamma = (real)kp.gamma, pfl = (real)kp.p_floor, rfl = (real)kp.rho_floor;
  const int nb0 = kp.nb[0], nb1 = kp.nb[1], nb2 = kp.nb[2];
  const int P1 = kp.P[1], P2 = kp.P[2];
  const size_t plane = (size_t)P1 * P2, vstride = (size_t)kp.P[0] * plane, bstride = kp.nvs * vstride;
  const int per_block = sl.tiles_j * sl.tiles_k * sl.segs;
  const int nwork = sl.nlist * per_block;
  const bool spherical = kp.geometry == 0;
  const real Om = (real)kp.omega, Cd = (real)kp.cd;
  const Isl isl{(float)kp.isl_pe, (float)kp.isl_beta};
  const real igm1 = real(1) / (gamma - real(1));

  // reflux face buffer layout (per slot): faces in order r-lo, r-hi, th-lo,
  // th-hi, ph-lo, ph-hi; each [v][t1][t2]
  const int fc0 = nb1 * nb2, fc1 = nb0 * nb2, fc2 = nb0 * nb1;
  const size_t fstride = (size_t)NVAR * 2 * (fc0 + fc1 + fc2);

  real inv_acc = real(0);
  long long hits = 0;
  int cur_member = -1;

  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    int li = w / per_block, rem = w - li * per_block;
    const int seg = rem % sl.segs;
    rem /= sl.segs;
    const int tk = rem % sl.tiles_k, tj = rem / sl.tiles_k;
    const int slot = sl.list[li];
    const DevBlock B = kp.blk[slot];
    const double dtm = kp.dt_used[B.member];
    if (!(dtm > 0.0)) continue;  // member has reached its stop time (uniform)
    if (S2 && B.member != cur_member) {
      flush_acc(kp, inv_acc, cur_member, hits);
      cur_member = B.member;
    }
    const real dt = (real)(dtm * sl.dtfac);
    const LevelGeo<real> &G = GeoSel<real>::get(kp.geo, B.level);
    const int j0 = tj * TJ, k0 = tk * TK;
    const int nvj = min(TJ, nb1 - j0), nvk = min(TK, nb2 - k0);
    const int ib = seg * sl.seg_len, ie = min(nb0, ib + sl.seg_len);
    const int I0 = B.ix[0] * nb0, J0 = B.ix[1] * nb1 + j0, K0 = B.ix[2] * nb2 + k0;
    const real *Uin = reinterpret_cast<const real *>(sl.Uin) + (size_t)slot * bstride;
    const real *U0 = reinterpret_cast<const real *>(sl.U0) + (size_t)slot * bstride;
    real *Uout = reinterpret_cast<real *>(sl.Uout) + (size_t)slot * bstride;
    const bool valid = tid < TJ * TK && jl < nvj && kl < nvk;
    const int j = j0 + jl, k = k0 + kl;           // interior indices in the block

    // Planes of U_in are copied asynchronously (cp.async, 4 bytes per copy)
    // straight into their ring slot and converted to primitives in place one
    // iteration later, by the thread that copied them (no barrier between
    // copy and conversion).  A unit is two cells half a plane apart, so the
    // threads of a warp write consecutive cells.  Units go to the highest
    // thread indices, which own no second div B position.
    constexpr int NU = RP / 2;
    auto slotp = [&](int p) -> real * { return ring + ((p + 5) % 5) * NVAR * RP; };
    auto xslot = [&](int p) -> real * { return xring + ((p + 5) % 5) * RP; };
    // Cells of the plane outside the block that a same-level leaf holds come
    // straight from that leaf's interior (sl.direct: the step's ghost fills
    // leave such ghost copies unfilled); the others from this block's ghost
    // layer (coarser or finer neighbours, physical boundaries).
    const int *nb27 = kp.nb27 + (size_t)slot * 27;
    const real *Uall = reinterpret_cast<const real *>(sl.Uin);
    auto issue_plane = [&](int p) {
      real *dst = slotp(p);
      const int sr = p < 0 ? -1 : (p >= nb0 ? 1 : 0);
      for (int u = NT - 1 - tid; u < NU; u += NT) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const int q = u + h * NU, jj = q / RK, kk = q - (q / RK) * RK;
          const int pj = j0 + jj, pk = k0 + kk;
          if (pj < P1 && pk < P2) {
            const real *src = Uin + (size_t)(p + NGH) * plane + (size_t)pj * P2 + pk;
            if (sl.direct) {
              const int sj = pj < NGH ? -1 : (pj >= NGH + nb1 ? 1 : 0);
              const int sk = pk < NGH ? -1 : (pk >= NGH + nb2 ? 1 : 0);
              if (sr | sj | sk) {
                const int o = nb27[(sr + 1) * 9 + (sj + 1) * 3 + (sk + 1)];
                if (o >= 0)
                  src = Uall + (size_t)o * bstride + (size_t)(p - sr * nb0 + NGH) * plane +
                        (size_t)(pj - sj * nb1) * P2 + (pk - sk * nb2);
              }
            }
#pragma unroll
            for (int v = 0; v < NVAR; v++) cp_async<sizeof(real)>(&el<real, RP>(dst, v, q), src + v * vstride);
            if (trc) cp_async<sizeof(real)>(xslot(p) + q, src + TRV * vstride);
          }
        }
      }
      cp_async_commit();
    };
    auto convert_plane = [&](int p) {
      real *pl = slotp(p);
      for (int u = NT - 1 - tid; u < NU; u += NT) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const int q = u + h * NU, jj = q / RK, kk = q - (q / RK) * RK;
          if (j0 + jj < P1 && k0 + kk < P2) {
            real uu[NVAR], wv[NVAR];
            ld8<real, RP>(pl, q, uu);
            cons2prim<real>(uu, wv, gamma, pfl, isl);
            st8<real, RP>(pl, q, wv);
            if (trc) xslot(p)[q] *= RT<real>::rcp_(uu[0]);   // rho X -> X
          }
        }
      }
    };
    // U^n of the thread's own cell at plane p, copied asynchronously one
    // plane ahead (only this thread reads it: no barrier); always commits a
    // group so that the group counts stay uniform
    auto issue_u0 = [&](int p) {
      if (valid && p < ie) {
        const real *src = U0 + (size_t)(p + NGH) * plane + (size_t)(j + NGH) * P2 + (k + NGH);
#pragma unroll
        for (int v = 0; v < NVAR; v++) cp_async<sizeof(real)>(u0s + v * NT + tid, src + v * vstride);
      }
      cp_async_commit();
    };
    auto ringp = [&](int p) -> const real * { return ring + ((p + 5) % 5) * NVAR * RP; };
    auto gather = [&](const real *pl, int jj, int kk, real *w) { ld8<real, RP>(pl, jj * RK + kk, w); };
    // half the limited radial slope at plane p of the thread's column
    auto rslope = [&](int p, real *sl_) {
      const real *pm = ringp(p - 1), *pc = ringp(p), *pp = ringp(p + 1);
      const int o = (jl + 2) * RK + kl + 2;
      real a[NVAR], b[NVAR], c[NVAR];
      ld8<real, RP>(pm, o, a);
      ld8<real, RP>(pc, o, b);
      ld8<real, RP>(pp, o, c);
      mc_half_slopes8<real>(a, b, c, sl_);
    };
    // radial face between planes p-1 and p from the slopes at both planes
    auto rflux = [&](int p, const real *sm, const real *sp, real *F) {
      real b[NVAR], c[NVAR];
      gather(ringp(p - 1), jl + 2, kl + 2, b);
      gather(ringp(p), jl + 2, kl + 2, c);
      if constexpr (sizeof(real) == 4) {
        tvdlf_pair<0>(b, c, sm, sp, gamma, igm1, F);
      } else {
        real WL[NVAR], WR[NVAR];
        axpy8<real>(b, real(1), sm, WL);
        axpy8<real>(c, real(-1), sp, WR);
        tvdlf_states<real, 0>(WL, WR, b, c, gamma, igm1, F);
      }
    };
    // div B at plane p on the (TJ+2) x (TK+2) positions around the tile
    auto divb_plane = [&](int p) {
      real *dst = dring + (p & 3) * DP;
      const real *pm = ringp(p - 1), *pc = ringp(p), *pp = ringp(p + 1);
      const int pr = p - ib + 2;   // plane index in the staged arrays
      const real rcm = s_rc[pr - 1], rcc = s_rc[pr], rcp = s_rc[pr + 1];
      // plane-uniform radial factors
      const real wm = spherical ? rcm * rcm : real(1), wp = spherical ? rcp * rcp : real(1);
      const real fr = RT<real>::rcp_((spherical ? rcc * rcc : real(1)) * (rcp - rcm));
      for (int q = tid; q < DP; q += NT) {
        const int dj = q / DK - 1, dk = q - (q / DK) * DK - 1;
        if (dj > nvj || dk > nvk) continue;
        const int jj = dj + 2, kk = dk + 2;
        const int o = jj * RK + kk;
        const real brm = el<real, RP>(pm, 5, o), brp = el<real, RP>(pp, 5, o);
        const real btm = el<real, RP>(pc, 6, o - RK), btp = el<real, RP>(pc, 6, o + RK);
        const real bpm = el<real, RP>(pc, 7, o - 1), bpp = el<real, RP>(pc, 7, o + 1);
        const real itc2 = s_itc2[dj + 2], ipc2 = s_ipc2[dk + 2];
        real div;
        if (spherical) {
          const real stc = s_st[dj + 2];
          const real sm = s_st[dj + 1], sp = s_st[dj + 3];
          const real irs = RT<real>::rcp_(rcc * stc);
          div = (wp * brp - wm * brm) * fr + (sp * btp - sm * btm) * irs * itc2 + (bpp - bpm) * irs * ipc2;
        } else {
          div = (brp - brm) * fr + (btp - btm) * itc2 + (bpp - bpm) * ipc2;
        }
        dst[q] = div;
      }
    };

    // ---- geometry of the work item into shared memory (read after the
    // prologue's first barrier); rows / columns past the block's edge are
    // never read and not loaded ----
    {
      const int npl = ie - ib + 4, ir0 = I0 + ib - 2 + NGH;
      for (int q = tid; q < npl; q += NT) {
        s_rc[q] = G.rc[ir0 + q];
        s_dr2[q] = G.dr2[ir0 + q];
        s_dr3[q] = G.dr3[ir0 + q];
        s_idr[q] = RT<real>::rcp_(G.dr[ir0 + q]);
        s_irc[q] = RT<real>::rcp_(G.rc[ir0 + q]);
        if (q >= 1 && q + 1 < npl) s_ird2[q] = RT<real>::rcp_(G.rc[ir0 + q + 1] - G.rc[ir0 + q - 1]);
      }
      for (int q = tid; q <= npl; q += NT) s_r2f[q] = G.r2f[ir0 + q];
      const int jr0 = J0 - 2 + NGH;
      for (int q = tid; q < nvj + 4; q += NT) {
        if (q >= 1 && q + 1 < nvj + 4) s_itc2[q] = RT<real>::rcp_(G.tc[jr0 + q + 1] - G.tc[jr0 + q - 1]);
        s_st[q] = G.sintc[jr0 + q];
        s_ct[q] = G.costc[jr0 + q];
        s_dcos[q] = G.dcos[jr0 + q];
        s_dth[q] = G.dth[jr0 + q];
        s_idth[q] = RT<real>::rcp_(G.dth[jr0 + q]);
      }
      for (int q = tid; q <= nvj + 4; q += NT) s_sinf[q] = G.sinf[jr0 + q];
      const int kr0 = K0 - 2 + NGH;
      for (int q = 1 + tid; q + 1 < nvk + 4; q += NT) s_ipc2[q] = RT<real>::rcp_(G.pc[kr0 + q + 1] - G.pc[kr0 + q - 1]);
    }
    const real dphi = G.dphi, idphi = RT<real>::rcp_(dphi);

    // ---- prologue: planes ib-2 .. ib+2 converted, r flux at face ib ----
    for (int p = ib - 2; p <= ib + 2; p++) issue_plane(p);
    cp_async_wait_all();
    for (int p = ib - 2; p <= ib + 2; p++) convert_plane(p);
    __syncthreads();
    if (S2) {
      divb_plane(ib - 1);
      divb_plane(ib);
    }
    real Flo[NVAR], sc[NVAR];
    real xprev = real(0);   // tracer X of this column at the previous plane
    if (valid) {
      real s0[NVAR];
      rslope(ib - 1, s0);
      rslope(ib, sc);
      rflux(ib, s0, sc, Flo);
      if (trc) xprev = xslot(ib - 1)[(jl + 2) * RK + kl + 2];
    }
    __syncthreads();   // plane ib-2 is read no more: its slot takes plane ib+3
    if (ib + 3 <= ie + 1) issue_plane(ib + 3);
    else cp_async_commit();
    issue_u0(ib);

    // One barrier per plane.  Phase A (before it): theta and phi face fluxes
    // of plane i into face buffer i&1, div B of plane i+1, conversion of plane
    // i+3.  Phase B (after it): r flux at face i+1 and the update of the
    // thread's cell of plane i, then the copies of plane i+4 (into the slot of
    // plane i-1, which neither phase reads any more) and of U^n at plane i+1.
    // A thread in phase A of plane i+1 can overlap others still in phase B of
    // plane i: they use the other face buffer, another div B slot and
    // disjoint ring slots.
    for (int i = ib; i < ie; i++) {
      real *fthb = fth + (i & 1) * NVAR * NTH, *fphb = fph + (i & 1) * NVAR * NPH;
      {
        const real *pl = ringp(i);
        for (int f = tid; f < NTH + NPH; f += NT) {
          real a[NVAR], b[NVAR], c[NVAR], e[NVAR], F[NVAR];
          if (f < NTH) {
            const int row = f / TK, col = f - (f / TK) * TK;
            if (row <= nvj && col < nvk) {
              gather(pl, row, col + 2, a);
              gather(pl, row + 1, col + 2, b);
              gather(pl, row + 2, col + 2, c);
              gather(pl, row + 3, col + 2, e);
              tvdlf_face<real, 1>(a, b, c, e, gamma, igm1, F);
              st8<real, NTH>(fthb, row * TK + col, F);
            }
          } else {
            // phi faces: the first TJ * TK in rows of TK (a warp's quarters stay
            // in one row when TK is a multiple of 8), then the last column
            const int g = f - NTH;
            const int row = g < TJ * TK ? g / TK : g - TJ * TK;
            const int col = g < TJ * TK ? g - (g / TK) * TK : TK;
            if (row < nvj && col <= nvk) {
              gather(pl, row + 2, col, a);
              gather(pl, row + 2, col + 1, b);
              gather(pl, row + 2, col + 2, c);
              gather(pl, row + 2, col + 3, e);
              tvdlf_face<real, 2>(a, b, c, e, gamma, igm1, F);
              st8<real, NPH>(fphb, row * (TK + 1) + col, F);
            }
          }
        }
      }
      if (S2) divb_plane(i + 1);
      if (i + 3 <= ie + 1) {
        cp_async_wait_group<1>();   // plane i+3 landed (U^n of plane i may not have)
        convert_plane(i + 3);
      }
      __syncthreads();
      real Fhi[NVAR];
      if (valid) {
        real sn[NVAR];
        rslope(i + 1, sn);
        rflux(i + 1, sc, sn, Fhi);
#pragma unroll
        for (int v = 0; v < NVAR; v++) sc[v] = sn[v];
      }
      if (valid) {
        const int pr = i - ib + 2, jr = jl + 2;   // indices in the staged arrays
        const real dcos = s_dcos[jr], dr2 = s_dr2[pr];
        // face areas; the fluxes carry a factor 2 (tvdlf_states), which the
        // half areas hArm ... hAp take back
        const real Arm = s_r2f[pr] * dcos * dphi, Arp = s_r2f[pr + 1] * dcos * dphi;
        const real Atm = s_sinf[jr] * dr2 * dphi, Atp = s_sinf[jr + 1] * dr2 * dphi;
        const real Ap = dr2 * s_dth[jr];
        const real hArm = real(0.5) * Arm, hArp = real(0.5) * Arp, hAtm = real(0.5) * Atm, hAtp = real(0.5) * Atp,
                   hAp = real(0.5) * Ap;
        const real V = s_dr3[pr] * dcos * dphi;
        const real iV = RT<real>::rcp_(V);
        real w[NVAR];
        gather(ringp(i), jl + 2, kl + 2, w);
        real un[NVAR];
        const size_t cidx = (size_t)(i + NGH) * plane + (size_t)(j + NGH) * P2 + (k + NGH);
        {
          constexpr int CH = Vec16<real>::CH;
          const int qt = jl * TK + kl, qp = jl * (TK + 1) + kl;
#pragma unroll
          for (int c = 0; c < NVAR / CH; c++) {
            real ftl[CH], fth_[CH], fpl[CH], fph_[CH];
            using V = Vec16<real>;
            V::put(*reinterpret_cast<const typename V::T *>(fthb + (c * NTH + qt) * CH), ftl);
            V::put(*reinterpret_cast<const typename V::T *>(fthb + (c * NTH + qt + TK) * CH), fth_);
            V::put(*reinterpret_cast<const typename V::T *>(fphb + (c * NPH + qp) * CH), fpl);
            V::put(*reinterpret_cast<const typename V::T *>(fphb + (c * NPH + qp + 1) * CH), fph_);
            flux_balance<real, CH>(Fhi + c * CH, Flo + c * CH, fth_, ftl, fph_, fpl, hArp, hArm, hAtp, hAtm, hAp,
                                   iV, un + c * CH);
          }
        }
        if (spherical) {
          const real gr = (Arp - Arm) * iV, gt = (Atp - Atm) * iV, ir = real(0.5) * gr;
          const real rho = w[0], vr = w[1], vt = w[2], vp = w[3], Br = w[5], Bt = w[6], Bp = w[7];
          const real pt = w[4] + real(0.5) * (Br * Br + Bt * Bt + Bp * Bp);
          un[1] += (rho * (vt * vt + vp * vp) - (Bt * Bt + Bp * Bp)) * ir + pt * gr;
          un[2] += (-rho * vr * vt + Br * Bt) * ir + (rho * vp * vp - Bp * Bp) * gt + pt * gt;
          un[3] += (-rho * vr * vp + Br * Bp) * ir - (rho * vt * vp - Bt * Bp) * gt;
          un[6] += (vr * Bt - vt * Br) * ir;
          un[7] += (vr * Bp - vp * Br) * ir + (vt * Bp - vp * Bt) * gt;
          const real rc = s_rc[pr], st = s_st[jr], ct = s_ct[jr];
          const real vs = vr * st + vt * ct;
          un[1] += rho * (real(2) * Om * vp * st + Om * Om * rc * st * st);
          un[2] += rho * (real(2) * Om * vp * ct + Om * Om * rc * st * ct);
          un[3] += real(-2) * Om * rho * vs;
          un[4] += rho * Om * Om * rc * st * vs;
        }
        cp_async_wait_group<0>();   // this thread's U^n copy of plane i
        {
          real u0[NVAR];
#pragma unroll
          for (int v = 0; v < NVAR; v++) u0[v] = u0s[v * NT + tid];
          axpy8<real>(u0, dt, un, un);
        }
        if (S2 && Cd > real(0)) {
          const real *dm = dring + ((i - 1) & 3) * DP, *dc = dring + (i & 3) * DP, *dp = dring + ((i + 1) & 3) * DP;
          const int q = (jl + 1) * DK + (kl + 1);
          const real ird2 = s_ird2[pr], itc2 = s_itc2[jr], ipc2 = s_ipc2[kl + 2];
          const real idr = s_idr[pr], idth = s_idth[jr];
          real gr_, gt_, gp_, h2inv;
          if (spherical) {
            const real irc = s_irc[pr], irs = RT<real>::rcp_(s_rc[pr] * s_st[jr]);
            gr_ = (dp[q] - dm[q]) * ird2;
            gt_ = (dc[q + DK] - dc[q - DK]) * irc * itc2;
            gp_ = (dc[q + 1] - dc[q - 1]) * irs * ipc2;
            const real ixt = irc * idth, ixp = irs * idphi;
            h2inv = idr * idr + ixt * ixt + ixp * ixp;
          } else {
            gr_ = (dp[q] - dm[q]) * ird2;
            gt_ = (dc[q + DK] - dc[q - DK]) * itc2;
            gp_ = (dc[q + 1] - dc[q - 1]) * ipc2;
            h2inv = idr * idr + idth * idth + idphi * idphi;
          }
          const real f = Cd * RT<real>::rcp_(h2inv);
          const real dB0 = f * gr_, dB1 = f * gt_, dB2 = f * gp_;
          un[5] += dB0;
          un[6] += dB1;
          un[7] += dB2;
          un[4] += w[5] * dB0 + w[6] * dB1 + w[7] * dB2;
        }
        if (trc) {
          // CME tracer (Sect. 3.1): rho X carried by each face's mass flux
          // with X from the face's upwind cell
          // X at plane i-1 of this column is carried from the previous plane:
          // that ring slot already receives the copy of plane i+4
          const int o = (jl + 2) * RK + kl + 2;
          const real *xc = xslot(i), *xp = xslot(i + 1);
          const real X0 = xc[o];
          const real ftl0 = el<real, NTH>(fthb, 0, jl * TK + kl), fth0 = el<real, NTH>(fthb, 0, (jl + 1) * TK + kl);
          const real fpl0 = el<real, NPH>(fphb, 0, jl * (TK + 1) + kl), fph0 = el<real, NPH>(fphb, 0, jl * (TK + 1) + kl + 1);
          const real arm = hArm * Flo[0] * (Flo[0] > real(0) ? xprev : X0);
          const real arp = hArp * Fhi[0] * (Fhi[0] > real(0) ? X0 : xp[o]);
          const real atm = hAtm * ftl0 * (ftl0 > real(0) ? xc[o - RK] : X0);
          const real atp = hAtp * fth0 * (fth0 > real(0) ? X0 : xc[o + RK]);
          const real apm = hAp * fpl0 * (fpl0 > real(0) ? xc[o - 1] : X0);
          const real app = hAp * fph0 * (fph0 > real(0) ? X0 : xc[o + 1]);
          const real dT = -((arp - arm) + (atp - atm) + (app - apm)) * iV;
          Uout[TRV * vstride + cidx] = U0[TRV * vstride + cidx] + dt * dT;
          xprev = X0;
        }
        hits += apply_floors<real>(un, gamma, pfl, rfl, isl);
        if (!(un[0] == un[0]) || !(un[4] == un[4])) atomicOr(kp.status, ST_NAN);
#pragma unroll
        for (int v = 0; v < NVAR; v++) Uout[v * vstride + cidx] = un[v];
        if (S2) {
          // CFL contribution of the new state (cells next to a finer face are
          // left to the reflux, which changes them once more)
          const bool skip = (i == 0 && B.nbr[0] == NB_FINER) || (i == nb0 - 1 && B.nbr[1] == NB_FINER) ||
                            (j == 0 && B.nbr[2] == NB_FINER) || (j == nb1 - 1 && B.nbr[3] == NB_FINER) ||
                            (k == 0 && B.nbr[4] == NB_FINER) || (k == nb2 - 1 && B.nbr[5] == NB_FINER);
          if (!skip) {
            real wn[NVAR];
            cons2prim_speed<real>(un, wn, gamma, pfl);
            real dx1 = s_dth[jr], dx2 = dphi;
            if (spherical) {
              dx1 *= s_rc[pr];
              dx2 *= s_rc[pr] * s_st[jr];
            }
            const real s = (RT<real>::abs_(wn[1]) + fast_speed<real, 0>(wn, gamma)) * s_idr[pr] +
                           (RT<real>::abs_(wn[2]) + fast_speed<real, 1>(wn, gamma)) * RT<real>::rcp_(dx1) +
                           (RT<real>::abs_(wn[3]) + fast_speed<real, 2>(wn, gamma)) * RT<real>::rcp_(dx2);
            inv_acc = RT<real>::max_(inv_acc, s);
          }
          if (sl.flux) {
            real *fb = reinterpret_cast<real *>(sl.flux) + (size_t)slot * fstride;
            // r faces
            if (i == 0 && (B.nbr[0] == NB_COARSER || B.nbr[0] == NB_FINER))
#pragma unroll
              for (int v = 0; v < NVAR; v++) fb[(size_t)v * fc0 + j * nb2 + k] = hArm * Flo[v];
            if (i == nb0 - 1 && (B.nbr[1] == NB_COARSER || B.nbr[1] == NB_FINER))
#pragma unroll
              for (int v = 0; v < NVAR; v++) fb[(size_t)NVAR * fc0 + (size_t)v * fc0 + j * nb2 + k] = hArp * Fhi[v];
            const size_t o2 = (size_t)2 * NVAR * fc0, o4 = o2 + (size_t)2 * NVAR * fc1;
            if (j == 0 && (B.nbr[2] == NB_COARSER || B.nbr[2] == NB_FINER))
#pragma unroll
              for (int v = 0; v < NVAR; v++)
                fb[o2 + (size_t)v * fc1 + i * nb2 + k] = hAtm * el<real, NTH>(fthb, v, jl * TK + kl);
            if (j == nb1 - 1 && (B.nbr[3] == NB_COARSER || B.nbr[3] == NB_FINER))
#pragma unroll
              for (int v = 0; v < NVAR; v++)
                fb[o2 + (size_t)NVAR * fc1 + (size_t)v * fc1 + i * nb2 + k] = hAtp * el<real, NTH>(fthb, v, (jl + 1) * TK + kl);
            if (k == 0 && (B.nbr[4] == NB_COARSER || B.nbr[4] == NB_FINER))
#pragma unroll
              for (int v = 0; v < NVAR; v++)
                fb[o4 + (size_t)v * fc2 + i * nb1 + j] = hAp * el<real, NPH>(fphb, v, jl * (TK + 1) + kl);
            if (k == nb2 - 1 && (B.nbr[5] == NB_COARSER || B.nbr[5] == NB_FINER))
#pragma unroll
              for (int v = 0; v < NVAR; v++)
                fb[o4 + (size_t)NVAR * fc2 + (size_t)v * fc2 + i * nb1 + j] = hAp * el<real, NPH>(fphb, v, jl * (TK + 1) + kl + 1);
          }
        }
#pragma unroll
        for (int v = 0; v < NVAR; v++) Flo[v] = Fhi[v];
      }
      if (i + 4 <= ie + 1) issue_plane(i + 4);
      else cp_async_commit();
      issue_u0(i + 1);
    }
    cp_async_wait_all();
    __syncthreads();  // shared memory is reused by the next work item
  }
  if (S2) flush_acc(kp, inv_acc, cur_member, hits);
  else {
    long long h = hits;
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    if ((threadIdx.x & 31) == 0 && h) atomicAdd(kp.floor_hits, (unsigned long long)h);
  }
}

// dynamic shared memory limit of both instances of a tile, raised (never
// lowered) to what a launch needs
template <typename real, int TJ, int TK>
void ensure_smem(size_t smem) {
  static size_t configured = 0;
  if (smem > configured) {
    cudaFuncSetAttribute(k_stage<real, TJ, TK, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_stage<real, TJ, TK, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = smem;
  }
}

template <typename real, int TJ, int TK>
int launch_t(const KParams &kp, const StageLaunch &sl, cudaStream_t s) {
  const size_t smem = StageSmem<real>::bytes(TJ, TK, kp.nvs > NVAR);
  ensure_smem<real, TJ, TK>(smem);
  if (sl.stage2)
    k_stage<real, TJ, TK, true><<<sl.grid, stage_threads(TJ, TK), smem, s>>>(kp, sl);
  else
    k_stage<real, TJ, TK, false><<<sl.grid, stage_threads(TJ, TK), smem, s>>>(kp, sl);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template <typename real>
int dispatch(const KParams &kp, const StageLaunch &sl, cudaStream_t s) {
  if (sl.tile_j == 8 && sl.tile_k == 8) return launch_t<real, 8, 8>(kp, sl, s);
  if (sl.tile_j == 12 && sl.tile_k == 12) return launch_t<real, 12, 12>(kp, sl, s);
  if (sl.tile_j == 8 && sl.tile_k == 32) return launch_t<real, 8, 32>(kp, sl, s);
  if (sl.tile_j == 4 && sl.tile_k == 32) return launch_t<real, 4, 32>(kp, sl, s);
  if (sl.tile_j == 12 && sl.tile_k == 20) return launch_t<real, 12, 20>(kp, sl, s);
  if (sl.tile_j == 6 && sl.tile_k == 36) return launch_t<real, 6, 36>(kp, sl, s);
  if (sl.tile_j == 10 && sl.tile_k == 24) return launch_t<real, 10, 24>(kp, sl, s);
  if (sl.tile_j == 8 && sl.tile_k == 24) return launch_t<real, 8, 24>(kp, sl, s);
  return -2;
}

template <typename real, int TJ, int TK>
int occupancy_t(bool tracer) {
  int n = 0;
  const size_t smem = StageSmem<real>::bytes(TJ, TK, tracer);
  ensure_smem<real, TJ, TK>(smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stage<real, TJ, TK, true>, stage_threads(TJ, TK), smem) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

template <typename real>
int occupancy(int tj, int tk, bool tracer) {
  if (tj == 8 && tk == 8) return occupancy_t<real, 8, 8>(tracer);
  if (tj == 12 && tk == 12) return occupancy_t<real, 12, 12>(tracer);
  if (tj == 8 && tk == 32) return occupancy_t<real, 8, 32>(tracer);
  if (tj == 4 && tk == 32) return occupancy_t<real, 4, 32>(tracer);
  if (tj == 12 && tk == 20) return occupancy_t<real, 12, 20>(tracer);
  if (tj == 6 && tk == 36) return occupancy_t<real, 6, 36>(tracer);
  if (tj == 10 && tk == 24) return occupancy_t<real, 10, 24>(tracer);
  if (tj == 8 && tk == 24) return occupancy_t<real, 8, 24>(tracer);
  return 1;
}

}  // namespace

size_t stage_smem_bytes(int precision, int tj, int tk, int tracer) {
  return precision ? StageSmem<float>::bytes(tj, tk, tracer) : StageSmem<double>::bytes(tj, tk, tracer);
}

// an instantiated tile whose shared memory fits one CTA on this device
int stage_tile_supported(int precision, int tj, int tk, int tracer) {
  const bool known = (tj == 8 && tk == 8) || (tj == 12 && tk == 12) || (tj == 8 && tk == 32) ||
                     (tj == 4 && tk == 32) || (tj == 12 && tk == 20) || (tj == 6 && tk == 36) ||
                     (tj == 10 && tk == 24) || (tj == 8 && tk == 24);
  if (!known) return 0;
  int dev = 0, lim = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  return stage_smem_bytes(precision, tj, tk, tracer) <= (size_t)lim;
}

int stage_max_ctas_per_sm(int precision, int tj, int tk, int tracer) {
  return precision ? occupancy<float>(tj, tk, tracer) : occupancy<double>(tj, tk, tracer);
}

int stage_launch(const KParams &kp, const StageLaunch &sl, int precision, cudaStream_t s) {
  if (sl.nlist <= 0) return 0;
  return precision ? dispatch<float>(kp, sl, s) : dispatch<double>(kp, sl, s);
}
