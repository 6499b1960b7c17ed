// Discrete adjoint of the coupled step (reverse mode, hand-written).
//
// The step maps the post-collision state s^{n-1} to s^n cell by cell:
// s^n(x) = C_x(P_x(s^{n-1}), theta_x), where P_x pulls the 24 populations
// (plain links from neighbours, boundary links from the cell itself, the
// virtual cells of the outlet and of the pressure inlet, the inlet velocity)
// and C_x relaxes them (Eq. 1,
// 8, 10) with the catalyst terms (Eq. 12-17).  Every plain link (y, q) of
// s^{n-1} has exactly one consumer, the fluid cell y + e_q, so the transpose
// of the pull is a push: the consumer writes the adjoint of what it pulled
// straight into lambda^{n-1}(y, q).  C_x is linear in the pulled values
// once the velocity is known, so the reverse needs from the forward step
// only its reverse records (RecPtrs, written by the step kernel's REC
// instantiation): per cell the Eq. 8 auxiliary velocity, the scalar sums
// and the O2 flux moments; per edge cell its pulled values; per edge or
// catalyst cell its own sums.  Two kernels per step, run concurrently
// (they write disjoint links):
//   k_adj_interior (one thread per cell; cells without edge bits): back-
//     propagates lambda^n(x) through C_x from the cell record, pushes the 24
//     link adjoints to the source cells and accumulates the parameter
//     adjoints of x.  Catalyst cells of the volumetric mode also read their
//     own state (through their own record); that adjoint goes to O(x).
//     Solid cells zero their own lambda^{n-1}.
//   k_adj_edge (one warp per listed edge cell): the same for cells with
//     boundary links, from their pulled values; the adjoint of values taken
//     from the cell's own state goes to O(x, q), a virtual column's uses of
//     the cells above and below to V.
// At a cell that uses its own state, lambda^{n-1}(y, q) is therefore split:
// the pushed value (only if y + e_q is a fluid consumer) + O(y, q) + the
// virtual-column terms.  The next reverse step adds the parts when it reads lambda
// (O and V are double-buffered for that); k_adj_fix adds them in place once,
// after the last step, for a caller that reads lambda itself.
// Storage is the domain's storage type S; arithmetic is R.
#pragma once
#include "lbm_core.cuh"

namespace pemlbm {

// The link tables of the core packed into single constants (2 bits per link for the
// direction + 1, 4 bits for the opposite link), so that a link index known
// only at run time costs a shift and a mask instead of a local-memory
// table.  The D2Q5 links of Eq. 9 are the first five D2Q9 links.
namespace dirbits {
constexpr int ex[9] = EX9_TAB, ey[9] = EY9_TAB, op[9] = OP9_TAB;
constexpr unsigned long long pack(const int (&t)[9], int bits, int bias) {
  unsigned long long r = 0;
  for (int i = 0; i < 9; ++i) r |= (unsigned long long)(t[i] + bias) << (bits * i);
  return r;
}
constexpr unsigned kEX = (unsigned)pack(ex, 2, 1), kEY = (unsigned)pack(ey, 2, 1);
constexpr unsigned long long kOP = pack(op, 4, 0);
}  // namespace dirbits
__host__ __device__ __forceinline__ constexpr int ex9(int i) {
  return (int)((dirbits::kEX >> (2 * i)) & 3u) - 1;
}
__host__ __device__ __forceinline__ constexpr int ey9(int i) {
  return (int)((dirbits::kEY >> (2 * i)) & 3u) - 1;
}
__host__ __device__ __forceinline__ constexpr int op9(int i) {
  return (int)((dirbits::kOP >> (4 * i)) & 15ull);
}
// Direction of population plane q (0..8 flow, 9..23 three D2Q5 scalars).
__host__ __device__ __forceinline__ constexpr int plane_link(int q) {
  return q < 9 ? q : (q - 9) % 5;
}
static_assert(ex9(5) == 1 && ey9(5) == 1 && ex9(7) == -1 && ey9(8) == -1 && op9(5) == 7 &&
                  op9(8) == 6 && op9(3) == 1,
              "packed link tables");


// Per-step adjoint workspace (device pointers).
template <typename R> struct AdjBufs {
  const R *lam;      // lambda^n, [24][plane] (deviation coordinates = full coordinates);
                     // at own-use cells only the pushed links are valid, the
                     // rest of lambda^n is O_in / V_in
  R *O;              // own-use adjoints of this step [24][plane] (own-use cells only)
  R *V;              // virtual columns of this step: [side][2][10][ny], side 0 the outlet,
                     // 1 the pressure inlet (down: from y+1 to y, up: from y-1 to y)
  const R *O_in;     // the same two left by the previous reverse step
  const R *V_in;
  R *gphi, *gK, *gD;        // per-cell parameter gradients of the current segment [plane]
  double *gU;               // d objective / d u_in_avg (velocity inlet) or d dp_in (pressure)
  R *lam_out;        // lambda^{n-1} [24][plane] (pushed links)
  const uint32_t *pushed;   // per edge cell: bit q set if link q has a fluid consumer
};

// Adjoint of the D2Q5 collision of scalar s (collide_scalar).  Given the
// output adjoints lo[5], accumulates into ld[5] (pulled values), lux, luy,
// and the adjoints of the source, b, w1 and q1.  The collision is linear in
// the populations, so its reverse needs of them only the deviation sum
// Cdev and the flux moments n1, n2 (the latter for the q1 adjoint).
template <typename R>
__device__ __forceinline__ void collide_scalar_rev(const KArgsT<R> &a, const MatCoef<R> &mc, int s,
                                                   R ux, R uy, R Cdev, R n1, R n2, R srcv,
                                                   const R lo[5], R ld[5], R &lux, R &luy,
                                                   R &lsrc, R &lb, R &lw1, R &lq1) {
  const R Q1 = mc.q1[s], Q3 = R(a.Q3), b = mc.b[s], w1 = mc.w1[s], w0 = R(1) - R(4) * w1;
  const R C = Cdev + R(a.Cref[s]), Ca = Cdev + R(a.adv_off[s]);
  // outputs: o0 = 0.2 (n0 - n3') + w0 src; o1,3 = ev +- 0.25 n4' ... (see forward)
  const R lex = lo[1] + lo[3], ley = lo[2] + lo[4];
  const R ln1p = R(0.5) * (lo[1] - lo[3]), ln2p = R(0.5) * (lo[2] - lo[4]);
  const R lev = lex + ley, ln4p = R(0.25) * (lex - ley);
  R ln0 = R(0.2) * lev + R(0.2) * lo[0];
  const R ln3p = R(0.05) * lev - R(0.2) * lo[0];
  lw1 += srcv * lev - R(4) * srcv * lo[0];
  lsrc += w1 * lev + w0 * lo[0];
  const R ln4 = (R(1) - Q3) * ln4p;
  const R ln3 = (R(1) - Q3) * ln3p;
  lb += Q3 * C * ln3p;
  R lC = Q3 * b * ln3p;
  const R ln1 = (R(1) - Q1) * ln1p, ln2 = (R(1) - Q1) * ln2p;
  lux += Q1 * Ca * ln1p;
  luy += Q1 * Ca * ln2p;
  lC += Q1 * ux * ln1p + Q1 * uy * ln2p;
  lq1 += (ux * Ca - n1) * ln1p + (uy * Ca - n2) * ln2p;
  const R lCdev = lC + ln0;
  const R le13 = ln3 + ln4, le24 = ln3 - ln4;
  ld[0] += R(-4) * ln3 + lCdev;
  ld[1] += ln1 + le13 + lCdev;
  ld[3] += -ln1 + le13 + lCdev;
  ld[2] += ln2 + le24 + lCdev;
  ld[4] += -ln2 + le24 + lCdev;
}

// Adjoint of collide_flow + the flow part of macros (Eq. 1, 3-8).  Given the
// output adjoints lo[9] and the adjoints lux, luy of the velocity coming
// from the scalar collisions, accumulates ld[9] and the adjoints of phi
// (direct), darcy, forch, l0, l1 and 1/phi.  The collision is linear in the
// populations once u is known, so the reverse needs of them only the
// auxiliary velocity (vx, vy) of Eq. 8 (body-force half-step included).
template <typename R>
__device__ __forceinline__ void flow_rev(const KArgsT<R> &a, const MatCoef<R> &mc, R vx, R vy,
                                         const R lo[9], R lux_in, R luy_in, R ld[9], R &lphi,
                                         R &ldarcy, R &lforch, R &ll0, R &ll1, R &lip) {
  const R sn = R(a.s_nu), sq = R(a.s_q), g = R(a.body_g), ip = mc.inv_phi;
  // ---- the macroscopic values of the forward step (macros)
  // (the forward step's own operations, so that u is the forward value)
  const R vn = vsqrt(vx * vx + vy * vy);
  const R rr = vsqrt(mc.l0 * mc.l0 + mc.l1 * vn);
  const R den = mc.l0 + rr, inv_den = vrcp(den);
  const R ux = vx * inv_den, uy = vy * inv_den;
  const R u2 = ux * ux + uy * uy, un = vn * inv_den;
  const R Fx = -mc.darcy * ux - mc.forch * un * ux + mc.phi * g;
  const R Fy = -mc.darcy * uy - mc.forch * un * uy;
  const R uF = ux * Fx + uy * Fy;
  const R hn = R(1) - R(0.5) * sn, hq = R(1) - R(0.5) * sq;
  // ---- back through f* = M^T diag(1/n) m*
  R la[9];
  la[0] = lo[0] + lo[1] + lo[2] + lo[3] + lo[4] + lo[5] + lo[6] + lo[7] + lo[8];
  la[1] = R(-4) * lo[0] - (lo[1] + lo[2] + lo[3] + lo[4]) + R(2) * (lo[5] + lo[6] + lo[7] + lo[8]);
  la[2] = R(4) * lo[0] - R(2) * (lo[1] + lo[2] + lo[3] + lo[4]) + (lo[5] + lo[6] + lo[7] + lo[8]);
  la[3] = lo[1] - lo[3] + lo[5] - lo[6] - lo[7] + lo[8];
  la[4] = R(-2) * (lo[1] - lo[3]) + lo[5] - lo[6] - lo[7] + lo[8];
  la[5] = lo[2] - lo[4] + lo[5] + lo[6] - lo[7] - lo[8];
  la[6] = R(-2) * (lo[2] - lo[4]) + lo[5] + lo[6] - lo[7] - lo[8];
  la[7] = lo[1] - lo[2] + lo[3] - lo[4];
  la[8] = lo[5] - lo[6] + lo[7] - lo[8];
  const R lm0p = la[0] * R(1.0 / 9), lm1p = la[1] * R(1.0 / 36), lm2p = la[2] * R(1.0 / 36);
  const R lm3p = la[3] * R(1.0 / 6), lm4p = la[4] * R(1.0 / 12), lm5p = la[5] * R(1.0 / 6);
  const R lm6p = la[6] * R(1.0 / 12), lm7p = la[7] * R(0.25), lm8p = la[8] * R(0.25);
  // ---- back through m* = m - S (m - m_eq) + (1 - S/2) G
  R lm[9];
  lm[0] = (R(1) - sn) * lm0p;
  lm[1] = (R(1) - sn) * lm1p;
  lm[2] = (R(1) - sn) * lm2p;
  lm[3] = lm3p;
  lm[4] = (R(1) - sq) * lm4p;
  lm[5] = lm5p;
  lm[6] = (R(1) - sq) * lm6p;
  lm[7] = (R(1) - sn) * lm7p;
  lm[8] = (R(1) - sn) * lm8p;
  R lP = R(6) * sn * lm1p - R(9) * sn * lm2p;
  R lu2 = R(3) * sn * ip * lm1p - R(3) * sn * ip * lm2p;
  R luF = R(6) * hn * ip * lm1p - R(6) * hn * ip * lm2p;
  lip += R(3) * sn * u2 * lm1p + R(6) * hn * uF * lm1p - R(3) * sn * u2 * lm2p -
         R(6) * hn * uF * lm2p;
  R lFx = lm3p - hq * lm4p, lFy = lm5p - hq * lm6p;
  R lux = lux_in - sq * lm4p, luy = luy_in - sq * lm6p;
  // m7: E = (ux^2 - uy^2) ip, H = 2 (ux Fx - uy Fy) ip
  lux += sn * R(2) * ux * ip * lm7p + hn * R(2) * Fx * ip * lm7p;
  luy += -sn * R(2) * uy * ip * lm7p - hn * R(2) * Fy * ip * lm7p;
  lFx += hn * R(2) * ux * ip * lm7p;
  lFy += -hn * R(2) * uy * ip * lm7p;
  lip += sn * (ux * ux - uy * uy) * lm7p + hn * R(2) * (ux * Fx - uy * Fy) * lm7p;
  // m8: E = ux uy ip, H = (ux Fy + uy Fx) ip
  lux += sn * uy * ip * lm8p + hn * Fy * ip * lm8p;
  luy += sn * ux * ip * lm8p + hn * Fx * ip * lm8p;
  lFy += hn * ux * ip * lm8p;
  lFx += hn * uy * ip * lm8p;
  lip += sn * ux * uy * lm8p + hn * (ux * Fy + uy * Fx) * lm8p;
  // uF = ux Fx + uy Fy
  lux += Fx * luF;
  luy += Fy * luF;
  lFx += ux * luF;
  lFy += uy * luF;
  // u2 in the energy equilibria
  lux += R(2) * ux * lu2;
  luy += R(2) * uy * lu2;
  // F = -darcy u - forch |u| u + phi g x
  const R lFu = ux * lFx + uy * lFy;
  lux += (-mc.darcy - mc.forch * un) * lFx;
  luy += (-mc.darcy - mc.forch * un) * lFy;
  const R lun = -mc.forch * lFu;
  ldarcy += -lFu;
  lforch += -un * lFu;
  lphi += g * lFx;
  if (un > R(0)) {
    lux += ux / un * lun;
    luy += uy / un * lun;
  }
  // P = 0.6 s18 - 0.4 |u|^2 ip
  const R ls18 = R(0.6) * lP;
  lux += R(-0.8) * ux * ip * lP;
  luy += R(-0.8) * uy * ip * lP;
  lip += R(-0.4) * u2 * lP;
  // u = v / (l0 + sqrt(l0^2 + l1 |v|))
  const R lden = -(ux * lux + uy * luy) / den;
  R lvx = lux / den, lvy = luy / den;
  if (vn > R(0)) {
    const R dr = mc.l1 / (R(2) * rr) * lden;   // d den / d vn = l1 / (2 rr)
    lvx += dr * vx / vn;
    lvy += dr * vy / vn;
  }
  ll0 += lden * (R(1) + mc.l0 / rr);
  ll1 += lden * vn / (R(2) * rr);
  lphi += R(0.5) * g * lvx;
  // moments and velocity back to the pulled populations
  const int EX[9] = EX9_TAB, EY[9] = EY9_TAB;
  const R M1[9] = {-4, -1, -1, -1, -1, 2, 2, 2, 2};
  const R M2[9] = {4, -2, -2, -2, -2, 1, 1, 1, 1};
  const R M4[9] = {0, -2, 0, 2, 0, 1, -1, -1, 1};
  const R M6[9] = {0, 0, -2, 0, 2, 1, 1, -1, -1};
  const R M7[9] = {0, 1, -1, 1, -1, 0, 0, 0, 0};
  const R M8[9] = {0, 0, 0, 0, 0, 1, -1, 1, -1};
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    ld[i] += lm[0] + M1[i] * lm[1] + M2[i] * lm[2] + R(EX[i]) * (lm[3] + lvx) + M4[i] * lm[4] +
             R(EY[i]) * (lm[5] + lvy) + M6[i] * lm[6] + M7[i] * lm[7] + M8[i] * lm[8] +
             (i > 0 ? ls18 : R(0));
  }
}

// d k / d theta of the rate k = A exp(e_in - c1 theta / (T T_in)): -c1 k / T^2.
template <typename R> __device__ __forceinline__ R drate_dtheta(const KArgsT<R> &a, R k, R theta) {
  const R T = R(a.T_in) + theta;
  return -R(a.k_c1) * k / (T * T);
}
// The same for the Butler-Volmer anodic rate k_a (constant c1_a; 0 when k_a = 0).
template <typename R>
__device__ __forceinline__ R drate_anodic_dtheta(const KArgsT<R> &a, R ka, R theta) {
  const R T = R(a.T_in) + theta;
  return -R(a.k_c1_a) * ka / (T * T);
}

// Parameter chain of one cell: adjoints of the derived coefficients to the
// caller's fields phi, K and D_O2 (Eq. 7, 8, 10), in the arithmetic type,
// accumulated per checkpoint segment (k_adj_fold adds each segment into the
// FP64 totals).
template <typename R>
__device__ __forceinline__ void param_rev(const KArgsT<R> &a, const MatCoef<R> &mc, int fickian,
                                          R lphi, R ldarcy, R lforch, R ll0, R ll1, R lip,
                                          R lbO2, R lw1O2, R lq1O2, R *gphi, R *gK, R *gD) {
  ldarcy += R(0.25) * ll0;
  lforch += R(0.5) * ll1;
  const R ip = mc.inv_phi;
  // darcy = phi nu / K, forch = 0.143 phi^-1/2 K^-1/2
  const R ddf = ldarcy * mc.darcy + R(0.5) * lforch * mc.forch;
  const R dphi = lphi - lip * ip * ip + (ldarcy * mc.darcy - R(0.5) * lforch * mc.forch) * ip;
  const R sqrt3 = R(1.7320508075688772);
  R dD;
  if (fickian) {
    const R q1 = mc.q1[1];
    dD = lq1O2 * (-q1 * q1 * R(10) / (R(4) + mc.b[1]));
  } else {
    dD = lbO2 * R(20) * sqrt3 + lw1O2 * sqrt3;
  }
  *gphi += dphi;
  if (mc.darcy > R(0)) {
    const R nu = (R(1) / R(a.s_nu) - R(0.5)) / R(3);
    const R inv_K = mc.darcy * ip / nu;
    *gK += -ddf * inv_K;
  }
  *gD += dD;
}

}  // namespace pemlbm

namespace pemlbm {

// Inlet parabola derivative: d u_in(yh) / d u_in_avg.
template <typename R> __device__ __forceinline__ R dinlet_du(const KArgsT<R> &a, R yh) {
  R s = (yh - R(a.y_ch0) + R(0.5)) / R(a.h_ch);
  return (s <= R(0) || s >= R(1)) ? R(0) : R(6) * s * (R(1) - s);
}

// Accumulation into the per-cell sums of the edge kernel, where each lane
// of a warp reverses one link of the same cell (shared memory).
template <typename R> __device__ __forceinline__ void acc_shared(R *p, R v) { atomicAdd(p, v); }

// Cross-row adjoints of the virtual columns (has_vcol) live in B.V as
// [side][down, up][10][ny], side 0 the outlet and 1 the inlet (vcol_side
// gives the offset of the side in units of ny).
template <typename R>
__device__ __forceinline__ int vcol_side(const KArgsT<R> &a, int x) {
  return x == a.nx - 1 ? 0 : 20;
}

// Reverse of the pull of one flow link i at edge cell (x, y).  lam is the
// adjoint of the pulled value; it is pushed to lambda^{n-1} of the source
// (plain link, `out`), or goes to Oacc (own populations), the virtual
// cells' adjoints (outlet, pressure inlet) or the inlet drive.  Oacc, Vdn, Vup and lip_own
// are shared by the lanes of the cell; lU is the lane's own.
template <typename R>
__device__ __forceinline__ void pull_flow_rev(const RecPtrs<R> &rp, const KArgsT<R> &a,
                                              const uint8_t *__restrict__ mask,
                                              const uint16_t *__restrict__ mid,
                                              const MatCoef<R> *__restrict__ pal, int i, int x,
                                              int y, uint8_t m, R lam, R *__restrict__ out,
                                              R *Oacc, R *Vdn, R *Vup, R *lip_own, R &lU) {
  const int opi = op9(i);
  int sx = x - ex9(i), sy = y - ey9(i);
  if (sy < 0 || sy >= a.ny) {
    acc_shared(&Oacc[opi], lam);
    return;
  }
  if (sx < 0 || sx >= a.nx) {
    if (a.periodic) {
      sx = sx < 0 ? sx + a.nx : sx - a.nx;
    } else {
      const bool in = sx < 0;
      if (in && !(a.inlet_pressure && (m & M_INLET))) {   // velocity inlet, or a wall
        acc_shared(&Oacc[opi], lam);
        if (m & M_INLET)
          lU += lam * R(6) * w9<R>(i) * R(ex9(i)) * dinlet_du<R>(a, R(y) - R(0.5) * R(ey9(i)));
        return;
      }
      // outlet, or the pressure inlet: the virtual column repeats column vx
      // at the source row with its pressure moved (by dp_in at the inlet)
      const int vx = in ? 0 : a.nx - 1;
      const long long vc = (long long)sy * a.nxp + vx;
      if (in && !(mask[vc] & M_INLET)) {               // the GDL's end wall
        acc_shared(&Oacc[opi], lam);
        return;
      }
      // the momentum of the source cell's own flow populations (its own
      // record; a solid cell keeps the rest state, zero deviations)
      const int sv = rp.slot[vc];
      const R jx = sv >= 0 ? rp.own[4LL * sv + 2] : R(0);
      const R jy = sv >= 0 ? rp.own[4LL * sv + 3] : R(0);
      const R ipv = pal[mid[vc]].inv_phi;
      const R ldP = lam9<R>(i) * lam;
      if (in) lU += ldP;                               // d value / d dp_in
      R lv[10];
#pragma unroll
      for (int k = 0; k < 9; ++k)
        lv[k] = ldP * ((k > 0 ? R(-0.6) : R(0)) + R(0.8) * ipv * (jx * R(ex9(k)) + jy * R(ey9(k))));
      lv[i] += lam;
      lv[9] = ldP * R(0.4) * (jx * jx + jy * jy);   // adjoint of the virtual cell's 1/phi
      R *dst = sy == y ? nullptr : (sy < y ? Vdn : Vup);
      if (!dst) {
#pragma unroll
        for (int k = 0; k < 9; ++k) acc_shared(&Oacc[k], lv[k]);
        acc_shared(lip_own, lv[9]);
      } else {
#pragma unroll
        for (int k = 0; k < 10; ++k) acc_shared(&dst[k], lv[k]);
      }
      return;
    }
  }
  // plain link (possibly across the periodic seam) unless the source is solid
  const long long sc = (long long)sy * a.nxp + sx;
  if ((m & M_NEAR_SOLID) && (mask[sc] & REG_MASK) == REG_SOLID) {
    acc_shared(&Oacc[opi], lam);
    return;
  }
#ifdef PEMLBM_BOUNDS_CHECK
  if (!in_bounds((long long)i * a.plane + sc, 24 * a.plane, 33)) return;
#endif
  out[(long long)i * a.plane + sc] = lam;
}

// Reverse of the pull of link i of scalar s at edge cell (x, y); Oacc and
// lw1 are shared by the lanes of the cell.
template <typename R>
__device__ __forceinline__ void pull_scalar_rev(const KArgsT<R> &a, const uint8_t *__restrict__ mask,
                                                const MatCoef<R> &mc, int s, int i, int x, int y,
                                                uint8_t m, R lam, R *__restrict__ out, R *Oacc,
                                                R *lw1) {
  const int q = 9 + 5 * s, opi = op9(i);
  int sx = x - ex9(i), sy = y - ey9(i);
  if (sy < 0) {
    acc_shared(&Oacc[q + opi], lam);
    return;
  }
  if (sy >= a.ny) {
    if (a.top_dirichlet) {
      acc_shared(&Oacc[q + opi], -lam);
      acc_shared(lw1, R(2) * R(a.Ctop[s]) * lam);
    } else {
      acc_shared(&Oacc[q + opi], lam);
    }
    return;
  }
  if (sx < 0 || sx >= a.nx) {
    if (a.periodic) {
      sx = sx < 0 ? sx + a.nx : sx - a.nx;
    } else if (sx < 0) {
      if (m & M_INLET) {
        acc_shared(&Oacc[q + opi], -lam);
        acc_shared(lw1, R(2) * R(a.Cin[s]) * lam);
      } else {
        acc_shared(&Oacc[q + opi], lam);
      }
      return;
    } else {
      acc_shared(&Oacc[q + i], lam);   // fully developed: the cell's own population of link i
      return;
    }
  }
  const long long sc = (long long)sy * a.nxp + sx;
  if ((m & M_NEAR_SOLID) && (mask[sc] & REG_MASK) == REG_SOLID) {
    acc_shared(&Oacc[q + opi], lam);
    return;
  }
#ifdef PEMLBM_BOUNDS_CHECK
  if (!in_bounds((long long)(q + i) * a.plane + sc, 24 * a.plane, 34)) return;
#endif
  out[(long long)(q + i) * a.plane + sc] = lam;
}

// Loads the 8-value cell record of cell c (two 4-value groups).
template <typename R> struct CellRec { R v[8]; };
__device__ __forceinline__ CellRec<float> ld_cell_rec(const float *r) {
  const float4 a = __ldg(reinterpret_cast<const float4 *>(r));
  const float4 b = __ldg(reinterpret_cast<const float4 *>(r) + 1);
  return CellRec<float>{{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w}};
}
__device__ __forceinline__ CellRec<double> ld_cell_rec(const double *r) {
  CellRec<double> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double2 t = __ldg(reinterpret_cast<const double2 *>(r) + k);
    o.v[2 * k] = t.x;
    o.v[2 * k + 1] = t.y;
  }
  return o;
}

// Reverse of the update of one fluid interior cell (no edge bits; see the
// file comment) from its cell record.  Catalyst cells of the volumetric
// mode also read their own state (the sink, from their own record) and
// leave that adjoint in O.
template <typename R>
__device__ __forceinline__ void adj_interior_cell(const RecPtrs<R> &rp,
                                                  const uint16_t *__restrict__ mid,
                                                  const MatCoef<R> *__restrict__ pal,
                                                  const KArgsT<R> &a, int fickian,
                                                  const AdjBufs<R> &B, long long c, uint8_t m) {
  const long long P = a.plane, W = a.nxp;
  const MatCoef<R> mc = pal[mid[c]];
  // this cell's segment gradients, read before any store of the thread so
  // that their latency overlaps the record loads (no other thread of the
  // launch touches them)
  R gacc[3] = {B.gphi[c], B.gK[c], B.gD[c]};
  const CellRec<R> rec = in_bounds(8 * c + 7, 8 * P, 32) ? ld_cell_rec(rp.cell + 8 * c)
                                                         : CellRec<R>{};
  const R vx = rec.v[0], vy = rec.v[1], n1 = rec.v[5], n2 = rec.v[6];
  const bool vol = a.mode == 1 && (m & REG_MASK) == REG_CATALYST;
  // lambda^n of link q: every link of an interior cell is pushed; a
  // catalyst cell adds the own-use adjoint the previous step left in O_in
  auto lam_at = [&](int q) -> R {
    if (!in_bounds(q * P + c, 24 * P, 30)) return R(0);
    R v = ld_r(B.lam + q * P + c);
    if (vol && q >= 9 && q < 19) v += ld_r(B.O_in + q * P + c);
    return v;
  };
  // pushes into lambda^{n-1} (the bounds-checked build skips one outside it)
  auto push = [&](long long k, R v) {
    if (in_bounds(k, 24 * P, 31)) B.lam_out[k] = v;
  };
  // forward reaction terms (kept for the reverse)
  R theta = 0, k = 0, ka = 0, Cv = 0, S_vol = 0;
  if (vol) {
    const R *ow = rp.own + 4LL * rp.slot[c];
    theta = ow[0];
    Cv = ow[1];
    k = rate<R>(a, R(a.kA_vol), theta);
    ka = rate_anodic<R>(a, R(a.kA_vol_a), theta);
    S_vol = (ka - k * Cv) / (R(1) + k);
  }
  // ---- reverse of the collisions; every link is plain, so each link's
  // adjoint is pushed to its source as soon as it is known
  R lcf[9], lcg[5];
#pragma unroll
  for (int i = 0; i < 9; ++i) lcf[i] = R(0);
  R lphi = 0, ldarcy = 0, lforch = 0, ll0 = 0, ll1 = 0, lip = 0;
  R lb[3] = {0, 0, 0}, lw1[3] = {0, 0, 0}, lq1[3] = {0, 0, 0}, lsrc[3] = {0, 0, 0};
  {
    const R vn = vsqrt(vx * vx + vy * vy);
    const R inv_den = vrcp(mc.l0 + vsqrt(mc.l0 * mc.l0 + mc.l1 * vn));
    const R ux = vx * inv_den, uy = vy * inv_den;
    const R srcv[3] = {-S_vol * R(a.hpo) * mc.inv_sigma, S_vol, R(-2) * S_vol};
    R lux = 0, luy = 0;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      R lo[5];
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        lo[i] = lam_at(9 + 5 * s + i);
        lcg[i] = R(0);
      }
      collide_scalar_rev<R>(a, mc, s, ux, uy, rec.v[2 + s], s == 1 ? n1 : R(0),
                            s == 1 ? n2 : R(0), srcv[s], lo, lcg, lux, luy, lsrc[s], lb[s], lw1[s],
                            lq1[s]);
#pragma unroll
      for (int i = 0; i < 5; ++i) push((9 + 5 * s + i) * P + c - ey9(i) * W - ex9(i), lcg[i]);
    }
    R lo[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) lo[i] = lam_at(i);
    flow_rev<R>(a, mc, vx, vy, lo, lux, luy, lcf, lphi, ldarcy, lforch, ll0, ll1, lip);
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) push(i * P + c - ey9(i) * W - ex9(i), lcf[i]);
  // volumetric sources (-S h / sigma, S, -2 S): own-use adjoints of theta, C_O2
  if (vol) {
    const R lS = -R(a.hpo) * mc.inv_sigma * lsrc[0] + lsrc[1] - R(2) * lsrc[2];
    // S = (k_a - k C)/(1 + k): dS/dC, dS/dk and dS/dk_a, with k and k_a of theta
    const R lC_own = lS * (-k / (R(1) + k));
    const R lth_own = lS * (-(Cv + ka) / ((R(1) + k) * (R(1) + k))) * drate_dtheta<R>(a, k, theta) +
                      lS / (R(1) + k) * drate_anodic_dtheta<R>(a, ka, theta);
#pragma unroll
    for (int q = 0; q < 24; ++q)
      B.O[q * P + c] = q >= 9 && q < 14 ? lth_own : (q >= 14 && q < 19 ? lC_own : R(0));
  }
  // ---- parameters of this cell
  param_rev<R>(a, mc, fickian, lphi, ldarcy, lforch, ll0, ll1, lip, lb[1], lw1[1], lq1[1],
               &gacc[0], &gacc[1], &gacc[2]);
  B.gphi[c] = gacc[0];
  B.gK[c] = gacc[1];
  B.gD[c] = gacc[2];
}

// Cells without edge bits, one thread per cell (grid over the lattice);
// solid cells zero their own lambda^{n-1} (nothing is ever pushed there).
template <typename R>
__global__ void __launch_bounds__(128, 8)
k_adj_interior(RecPtrs<R> rp, const uint8_t *__restrict__ mask, const uint16_t *__restrict__ mid,
               const MatCoef<R> *__restrict__ pal, KArgsT<R> a, int fickian, AdjBufs<R> B) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  const long long c = (long long)y * a.nxp + x;
  const uint8_t m = mask[c];
  if ((m & REG_MASK) == REG_SOLID) {
#pragma unroll
    for (int q = 0; q < 24; ++q) B.lam_out[q * a.plane + c] = R(0);
    return;
  }
  if (m & M_EDGE) return;
  adj_interior_cell<R>(rp, mid, pal, a, fickian, B, c, m);
}

// Fluid cells with edge bits, one warp per entry of `cells` (linear cell
// indices y * nxp + x), four cells per block.  An edge cell's boundary
// pulls and their reverses are independent per link, so lane q < 24 takes
// link q (in parallel instead of one long serial chain per cell); lane 0
// runs the cell's collision reverse in between.  lam_complete: lambda^n
// holds every link in full (the seed, or the caller's), O_in and V_in are
// zero.  seed_cell >= 0: the "CL temperature" seed on a zero lambda^n.
constexpr int kEdgeWarps = 4, kEdgeMinBlocks = 1;
// Launch order of a reverse step: the edge kernel before (true) or after
// the interior kernel; the first one's blocks are dispatched first.
constexpr bool kAdjEdgeFirst = true;
template <typename R>
__global__ void __launch_bounds__(32 * kEdgeWarps, kEdgeMinBlocks)
k_adj_edge(RecPtrs<R> rp, const uint8_t *__restrict__ mask, const uint16_t *__restrict__ mid,
           const MatCoef<R> *__restrict__ pal, KArgsT<R> a, int fickian, AdjBufs<R> B,
           const long long *__restrict__ cells, int ncells, long long seed_cell,
           int lam_complete) {
  struct Shared {
    R pulled[24];   // post-stream values of the cell
    R lin[24];      // lambda^n of the cell
    R lpull[24];    // adjoints of the pulled values
    R O[24];        // own-use adjoints
    R V[20];        // virtual column: 10 down (to y - 1's use), 10 up
    R lip, lw1[3];
  };
  __shared__ Shared sh_all[kEdgeWarps];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * kEdgeWarps + w;
  if (t >= ncells) return;   // whole warps leave
  Shared &sh = sh_all[w];
  const long long c = cells[t], P = a.plane, W = a.nxp;
#ifdef PEMLBM_BOUNDS_CHECK
  // every lambda, own-use, gradient and virtual-column access of the cell is
  // c + q P (q < 24), c itself or indexed by its row: bounded by c < P
  if (!in_bounds(c, P, 35)) return;   // (the whole warp: one cell)
#endif
  const int y = (int)(c / a.nxp), x = (int)(c - (long long)y * a.nxp);
  const uint8_t m = mask[c];
  const MatCoef<R> mc = pal[mid[c]];
  const bool vcol = has_vcol(a, x);
  const int vs = vcol_side(a, x);
  // ---- phase 1 (lane q): the pulled value of link q (the cell's record;
  // its slot is its index t in the list), lambda^n of link q
  if (lane < 24) {
    const int q = lane;
    sh.pulled[q] = rp.pulled[24LL * t + q];
    const uint32_t pbits = lam_complete ? 0xffffffffu : B.pushed[t];
    R lv = ((pbits >> q) & 1u) ? ld_r(B.lam + q * P + c) : R(0);
    lv += ld_r(B.O_in + q * P + c);
    if (vcol && q < 9) {
      if (y + 1 < a.ny) lv += ld_r(B.V_in + (vs + 0 * 10 + q) * a.ny + (y + 1));
      if (y - 1 >= 0) lv += ld_r(B.V_in + (vs + 1 * 10 + q) * a.ny + (y - 1));
    }
    sh.lin[q] = lv;
    sh.O[q] = R(0);
  }
  if (lane < 20) sh.V[lane] = R(0);
  if (lane == 0) sh.lip = sh.lw1[0] = sh.lw1[1] = sh.lw1[2] = R(0);
  __syncwarp();
  // ---- phase 2 (lane 0): reaction and collision reverse of the cell
  R lphi = 0, ldarcy = 0, lforch = 0, ll0 = 0, ll1 = 0, lip = 0;
  R lb1 = 0, lq1_1 = 0, lw1[3] = {0, 0, 0};
  R gacc[3] = {0, 0, 0};
  if (lane == 0) {
    gacc[0] = B.gphi[c];
    gacc[1] = B.gK[c];
    gacc[2] = B.gD[c];
    Cell<R> cell;
#pragma unroll
    for (int i = 0; i < 9; ++i) cell.f[i] = sh.pulled[i];
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
      for (int i = 0; i < 5; ++i) cell.g[s][i] = sh.pulled[9 + 5 * s + i];
    const bool surf = a.mode == 0 && (m & M_YLO);
    const bool vol = a.mode == 1 && (m & REG_MASK) == REG_CATALYST;
    R theta = 0, k = 0, ka = 0, kappa = 0, gd = 0, Cv = 0, S_vol = 0;
    if (surf || vol) theta = rp.own[4LL * t];
    if (surf) {
      k = rate<R>(a, R(a.kA_surf), theta);
      ka = rate_anodic<R>(a, R(a.kA_surf_a), theta);
      kappa = k / (R(2) * mc.w1[1]);
      gd = cell.g[1][2] + R(a.wr1[1]) * R(a.Cref[1]);
      const R Jv = (gd * (R(2) * kappa) - ka) / (R(1) + kappa);
      cell.g[1][2] -= Jv;
      cell.g[0][2] += R(a.hpo) * mc.inv_sigma * Jv;
      cell.g[2][2] += R(2) * Jv;
    }
    if (vol) {
      Cv = rp.own[4LL * t + 1];
      k = rate<R>(a, R(a.kA_vol), theta);
      ka = rate_anodic<R>(a, R(a.kA_vol_a), theta);
      S_vol = (ka - k * Cv) / (R(1) + k);
    }
    R lcf[9], lcg[3][5];
#pragma unroll
    for (int i = 0; i < 9; ++i) lcf[i] = R(0);
    R lb[3] = {0, 0, 0}, lq1[3] = {0, 0, 0}, lsrc[3] = {0, 0, 0};
    {
      const Macro<R> u = macros<R>(a, mc, cell);
      const R srcv[3] = {-S_vol * R(a.hpo) * mc.inv_sigma, S_vol, R(-2) * S_vol};
      R lux = 0, luy = 0;
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        R lo[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
          lo[i] = sh.lin[9 + 5 * s + i];
          lcg[s][i] = R(0);
        }
        collide_scalar_rev<R>(a, mc, s, u.ux, u.uy, u.C[s], cell.g[s][1] - cell.g[s][3],
                              cell.g[s][2] - cell.g[s][4], srcv[s], lo, lcg[s], lux, luy,
                              lsrc[s], lb[s], lw1[s], lq1[s]);
      }
      R lo[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) lo[i] = sh.lin[i];
      flow_rev<R>(a, mc, u.vx, u.vy, lo, lux, luy, lcf, lphi, ldarcy, lforch, ll0, ll1, lip);
    }
    if (vol) {   // volumetric sources (-S h / sigma, S, -2 S)
      const R lS = -R(a.hpo) * mc.inv_sigma * lsrc[0] + lsrc[1] - R(2) * lsrc[2];
      const R lC_own = lS * (-k / (R(1) + k));
      const R lth_own =
          lS * (-(Cv + ka) / ((R(1) + k) * (R(1) + k))) * drate_dtheta<R>(a, k, theta) +
          lS / (R(1) + k) * drate_anodic_dtheta<R>(a, ka, theta);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        sh.O[9 + q] += lth_own;
        sh.O[14 + q] += lC_own;
      }
    }
    if (c == seed_cell) {
#pragma unroll
      for (int i = 0; i < 5; ++i) lcg[0][i] += R(1);
    }
    if (surf) {   // reverse of the surface reaction (post -> pre link values)
      const R lJ = -lcg[1][2] + R(a.hpo) * mc.inv_sigma * lcg[0][2] + R(2) * lcg[2][2];
      // J = (2 kappa g_d - k_a)/(1 + kappa)
      const R lgd = lJ * R(2) * kappa / (R(1) + kappa);
      const R lkap = lJ * (R(2) * gd + ka) / ((R(1) + kappa) * (R(1) + kappa));
      const R lk = lkap / (R(2) * mc.w1[1]);
      lw1[1] += -lkap * k / (R(2) * mc.w1[1] * mc.w1[1]);
      const R lth = lk * drate_dtheta<R>(a, k, theta) +
                    (-lJ / (R(1) + kappa)) * drate_anodic_dtheta<R>(a, ka, theta);
#pragma unroll
      for (int q = 0; q < 5; ++q) sh.O[9 + q] += lth;
      lcg[1][2] += lgd;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) sh.lpull[i] = lcf[i];
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
      for (int i = 0; i < 5; ++i) sh.lpull[9 + 5 * s + i] = lcg[s][i];
    lb1 = lb[1];
    lq1_1 = lq1[1];
  }
  __syncwarp();
  // ---- phase 3 (lane q): reverse of the pull of link q
  R lU = 0;
  if (lane < 24) {
    const int q = lane;
    if (q < 9) {
      pull_flow_rev<R>(rp, a, mask, mid, pal, q, x, y, m, sh.lpull[q], B.lam_out, sh.O, sh.V,
                       sh.V + 10, &sh.lip, lU);
    } else {
      const int s = (q - 9) / 5;
      pull_scalar_rev<R>(a, mask, mc, s, q - 9 - 5 * s, x, y, m, sh.lpull[q], B.lam_out, sh.O,
                         &sh.lw1[s]);
    }
  }
  __syncwarp();
  // ---- phase 4: own-use and virtual-column adjoints out; parameters (lane 0)
  if (lane < 24) B.O[lane * P + c] = sh.O[lane];
  if (vcol && lane < 10) {
    B.V[(vs + 0 * 10 + lane) * a.ny + y] = sh.V[lane];
    B.V[(vs + 1 * 10 + lane) * a.ny + y] = sh.V[10 + lane];
  }
  if (lane == 0) {
    lip += sh.lip;
#pragma unroll
    for (int s = 0; s < 3; ++s) lw1[s] += sh.lw1[s];
    if (vcol) {   // the virtual column's use of this cell's 1/phi in the previous step
      R vsum_ip = 0;
      if (y + 1 < a.ny) vsum_ip += ld_r(B.V_in + (vs + 0 * 10 + 9) * a.ny + (y + 1));
      if (y - 1 >= 0) vsum_ip += ld_r(B.V_in + (vs + 1 * 10 + 9) * a.ny + (y - 1));
      gacc[0] += -vsum_ip * mc.inv_phi * mc.inv_phi;
    }
    param_rev<R>(a, mc, fickian, lphi, ldarcy, lforch, ll0, ll1, lip, lb1, lw1[1], lq1_1,
                 &gacc[0], &gacc[1], &gacc[2]);
    B.gphi[c] = gacc[0];
    B.gK[c] = gacc[1];
    B.gD[c] = gacc[2];
  }
  // inlet drive (velocity, or dp_in): warp sum, one FP64 atomic per warp that has inlet links
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) lU += __shfl_down_sync(0xffffffffu, lU, off);
  if (lane == 0 && lU != R(0)) atomicAdd(B.gU, (double)lU);
}

// Completes lambda in place after the last reverse step, at the own-use
// cells (edge cells, then catalyst cells of the volumetric mode), one thread
// per (link q, entry of `cells`), q-major so that neighbouring threads touch
// neighbouring cells: lambda(y, q) = pushed value (if y + e_q is a fluid
// consumer) + O(y, q) + the virtual columns' uses of y (B.lam_out, B.O, B.V:
// the buffers of that step); their 1/phi terms go to gphi.
template <typename R>
__global__ void __launch_bounds__(256)
k_adj_fix(const uint8_t *__restrict__ mask, const uint16_t *__restrict__ mid,
          const MatCoef<R> *__restrict__ pal, KArgsT<R> a, AdjBufs<R> B,
          const long long *__restrict__ cells, int ncells) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 24LL * ncells) return;
  const int q = (int)(t / ncells);
  const long long c = cells[t - (long long)q * ncells], P = a.plane;
#ifdef PEMLBM_BOUNDS_CHECK
  if (!in_bounds(c, P, 36)) return;
#endif
  const int y = (int)(c / a.nxp), x = (int)(c - (long long)y * a.nxp);
  const bool vcol = has_vcol(a, x);
  const int vs = vcol_side(a, x);
  const int ex = ex9(plane_link(q)), ey = ey9(plane_link(q));
  int cx = x + ex;
  const int cy = y + ey;
  bool pushed = false;
  if (cy >= 0 && cy < a.ny) {
    if (a.periodic) cx = cx < 0 ? cx + a.nx : (cx >= a.nx ? cx - a.nx : cx);
    if (cx >= 0 && cx < a.nx) pushed = (mask[(long long)cy * a.nxp + cx] & REG_MASK) != REG_SOLID;
  }
  R l = pushed ? B.lam_out[q * P + c] : R(0);
  l += B.O[q * P + c];
  if (vcol && q < 9) {
    if (y + 1 < a.ny) l += B.V[(vs + 0 * 10 + q) * a.ny + (y + 1)];
    if (y - 1 >= 0) l += B.V[(vs + 1 * 10 + q) * a.ny + (y - 1)];
  }
  B.lam_out[q * P + c] = l;
  if (vcol && q == 0) {
    R vsum_ip = 0;
    if (y + 1 < a.ny) vsum_ip += B.V[(vs + 0 * 10 + 9) * a.ny + (y + 1)];
    if (y - 1 >= 0) vsum_ip += B.V[(vs + 1 * 10 + 9) * a.ny + (y - 1)];
    const R ip = pal[mid[c]].inv_phi;
    B.gphi[c] += -vsum_ip * ip * ip;
  }
}

// Seed of the "mean current density" objective: lambda^{N-1} = d i_avg /
// d s^{N-1} (own populations of the catalyst cells) and the objective's
// direct parameter dependence.  weight = i_scale / nx.
template <typename S>
__global__ void __launch_bounds__(128)
k_adj_seed_current(const S *__restrict__ src_p, const uint8_t *__restrict__ mask,
                   const uint16_t *__restrict__ mid,
                   const MatCoef<typename Real<S>::type> *__restrict__ pal,
                   KArgsT<typename Real<S>::type> a, int fickian,
                   double weight, AdjBufs<typename Real<S>::type> B) {
  using R = typename Real<S>::type;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  const long long c = (long long)y * a.nxp + x, P = a.plane;
  const uint8_t m = mask[c];
  R l[24];
#pragma unroll
  for (int q = 0; q < 24; ++q) l[q] = R(0);
  if ((m & REG_MASK) != REG_SOLID) {
    const Pops<S> src{src_p, a.plane, a.nxp};
    const MatCoef<R> mc = pal[mid[c]];
    const R w = R(weight);
    if (a.mode == 0 && (m & M_YLO)) {
      const R theta = own_sum<S, R>(src, 0, x, y) + a.theta0;
      const R k = rate<R>(a, R(a.kA_surf), theta);
      const R ka = rate_anodic<R>(a, R(a.kA_surf_a), theta);
      const R kappa = k / (R(2) * mc.w1[1]);
      const R gd = R(src.at(9 + 5 + 4, x, y)) + R(a.wr1[1]) * R(a.Cref[1]);
      const R lkap = w * (R(2) * gd + ka) / ((R(1) + kappa) * (R(1) + kappa));
      const R lth = lkap / (R(2) * mc.w1[1]) * drate_dtheta<R>(a, k, theta) +
                    (-w / (R(1) + kappa)) * drate_anodic_dtheta<R>(a, ka, theta);
#pragma unroll
      for (int q = 0; q < 5; ++q) l[9 + q] += lth;
      l[18] += w * R(2) * kappa / (R(1) + kappa);
      if (!fickian) {
        const R lw1 = -lkap * k / (R(2) * mc.w1[1] * mc.w1[1]);
        B.gD[c] += lw1 * R(1.7320508075688772);
      }
    } else if (a.mode == 1 && (m & REG_MASK) == REG_CATALYST) {
      const R theta = own_sum<S, R>(src, 0, x, y) + a.theta0;
      const R Cv = own_sum<S, R>(src, 1, x, y) + R(a.Cref[1]);
      const R k = rate<R>(a, R(a.kA_vol), theta);
      const R ka = rate_anodic<R>(a, R(a.kA_vol_a), theta);
      const R lS = -w;   // i_avg = sum(-S) weight
      const R lC = lS * (-k / (R(1) + k));
      const R lth = lS * (-(Cv + ka) / ((R(1) + k) * (R(1) + k))) * drate_dtheta<R>(a, k, theta) +
                    lS / (R(1) + k) * drate_anodic_dtheta<R>(a, ka, theta);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        l[9 + q] += lth;
        l[14 + q] += lC;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 24; ++q) B.lam_out[q * P + c] = l[q];
}

// Adds a segment's gradients (arithmetic type) into the FP64 totals and
// clears them: n values per array, three arrays.
template <typename R>
__global__ void k_adj_fold(R *__restrict__ g0, R *__restrict__ g1, R *__restrict__ g2,
                           double *__restrict__ t0, double *__restrict__ t1,
                           double *__restrict__ t2, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    t0[i] += (double)g0[i];
    t1[i] += (double)g1[i];
    t2[i] += (double)g2[i];
    g0[i] = R(0);
    g1[i] = R(0);
    g2[i] = R(0);
  }
}

}  // namespace pemlbm
