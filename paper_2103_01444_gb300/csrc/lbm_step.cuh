// The coupled step kernel (one cell per thread, pull scheme) and its
// launcher, templated on the population storage type S.  Kept apart from
// the read-out, batch and adjoint kernels so that its sources can be
// identified on their own.
#pragma once
#include "lbm_core.cuh"
#include "lbm_launch.h"

namespace pemlbm {

// Own-state and pulled records of a listed cell (see RecPtrs): the values
// the reverse of its reaction and of its boundary links needs.  `cell`
// holds the post-stream values before the surface reaction.
template <typename S, typename R, bool CG>
__device__ __forceinline__ void write_listed_records(const Pops<S, CG> &src, const KArgsT<R> &a,
                                                     const RecPtrs<R> &rp, uint8_t m, long long c,
                                                     int x, int y, const Cell<R> &cell) {
  const bool cat = a.mode == 1 && (m & REG_MASK) == REG_CATALYST;
  if (!(m & M_EDGE) && !cat) return;
  const long long sl = rp.slot[c];
  R th = 0, cv = 0, jx = 0, jy = 0;
  if ((a.mode == 0 && (m & M_YLO)) || cat) th = own_sum<S, R, CG>(src, 0, x, y) + a.theta0;
  if (cat) cv = own_sum<S, R, CG>(src, 1, x, y) + R(a.Cref[1]);
  if (has_vcol(a, x)) {
    R d[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) d[k] = R(src.at(k, x, y));
    jx = d[1] - d[3] + d[5] - d[6] - d[7] + d[8];
    jy = d[2] - d[4] + d[5] + d[6] - d[7] - d[8];
  }
  stq(rp.own + 4 * sl, th, cv, jx, jy);
  if (m & M_EDGE) {
    R *p = rp.pulled + 24 * sl;
#pragma unroll
    for (int i = 0; i < 9; ++i) p[i] = cell.f[i];
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
      for (int i = 0; i < 5; ++i) p[9 + 5 * s + i] = cell.g[s][i];
  }
}

// ------------------------------------------------------------- step (K1)
// One coupled update of cell (x, y): src -> dst.  Shared by the single-
// domain step and the batched steps.  X: closed ends, fixed wall values and
// buoyancy compiled in (see pull_flow_edge).  REC: the step also writes
// its reverse records (RecPtrs) for the discrete adjoint.
template <typename S, bool CG = false, bool SR = false, bool X = false, bool REC = false>
__device__ __forceinline__ void cell_update(const S *__restrict__ src_p, S *__restrict__ dst,
                                            const uint8_t *__restrict__ mask,
                                            const uint16_t *__restrict__ mid,
                                            const MatCoef<typename Real<S>::type> *__restrict__ pal,
                                            const KArgsT<typename Real<S>::type> &a, int x,
                                            int y,
                                            const RecPtrs<typename Real<S>::type> &rp = {}) {
  using R = typename Real<S>::type;
  const long long c = (long long)y * a.nxp + x;
  const Pops<S, CG> src{src_p, a.plane, a.nxp};
  const uint8_t m = ld_mask(mask, c, a, 20);
  Cell<R> cell;
  load_interior<S, R, CG>(src, a, x, y, cell);
  // solid cells run the same arithmetic on their (unused) values and only
  // skip the stores, so no branch stands between the mask and the loads
  const bool live = (m & REG_MASK) != REG_SOLID;
  const MatCoef<R> mc = pal[ld_mid(mid, c, a, 21)];
  if (m & M_EDGE) {
    // next to grains but away from the lattice's edges: bounce-back only
    if ((m & M_EDGE) == M_NEAR_SOLID)
      bounce_solid<S, R, CG>(src, x, y, ld_mask(mask, a.plane + c, a, 23), cell);
    else fix_edges<S, R, CG, X>(src, a, mask, mid, pal, mc, x, y, m, cell);
  }
  if constexpr (REC)
    if (live) write_listed_records<S, R, CG>(src, a, rp, m, c, x, y, cell);
  if (a.mode == 0 && (m & M_YLO)) surface_reaction<S, R, CG>(src, a, mc, x, cell);
  R S_vol = 0;
  if (a.mode == 1 && (m & REG_MASK) == REG_CATALYST) S_vol = volume_sink<S, R, CG>(src, a, x, y);
  const Macro<R> u = macros<R, X>(a, mc, cell);
  if constexpr (REC) {
    if (live) {
      R *r = rp.cell + 8 * c;
      stq(r, u.vx, u.vy, u.C[0], u.C[1]);
      stq(r + 4, u.C[2], cell.g[1][1] - cell.g[1][3], cell.g[1][2] - cell.g[1][4], R(0));
    }
  }
  R o[9];
  collide_flow<R, X>(a, mc, u, cell.f, o);
  // 16-bit storage with stochastic rounding: a random stream per cell and
  // step (hash of the cell and the device step counter), twelve 32-bit
  // xorshift draws; population q (0-8 flow, 9 + 5 s + i scalar s) takes half
  // q & 1 of draw q >> 1.  Each draw's two halves thus round populations of
  // one lattice (the pair f_8, T_0 aside): giving both halves of a draw to
  // f_i and T_i of the same link correlated the rounding of u and of T, and
  // the mean of their product then biased the advected heat (at 50 k steps
  // on the 8192 x 2048 grain cathode the BF16 current was off by 271%
  // against 2% with this assignment).
  unsigned rnd[12] = {};
  if constexpr (SR) {
    unsigned rs = hash32((unsigned)c * 0x9e3779b9u ^ hash32(__ldg(a.seed_ctr) + 0x632be5abu)) | 1u;
#pragma unroll
    for (int j = 0; j < 12; ++j) rnd[j] = xorshift32(rs);
  }
  auto r16 = [&](int q) { return (q & 1) ? rnd[q >> 1] >> 16 : rnd[q >> 1] & 0xffffu; };
  const long long P = a.plane;
  // (the bounds-checked build skips a store outside the 24 planes)
  auto st_ok = [&](long long k, int width) { return in_bounds(k, 24 * P, 24) && in_bounds(k + width - 1, 24 * P, 24); };
  if (live) {   // the diagonal flow links
    if constexpr (SR) {
#pragma unroll
      for (int i = 5; i < 9; ++i)
        if (st_ok(pop_index(i, c, P), 1)) st_sr(dst + pop_index(i, c, P), o[i], r16(i));
    } else {
#pragma unroll
      for (int i = 5; i < 9; ++i)
        if (st_ok(pop_index(i, c, P), 1)) st_r(dst + pop_index(i, c, P), o[i]);
    }
  }
  const R srcv[3] = {-S_vol * R(a.hpo) * mc.inv_sigma, S_vol, R(-2) * S_vol};
  R g[3][5];
#pragma unroll
  for (int s = 0; s < 3; ++s)
    collide_scalar<R>(a, mc, s, u.ux, u.uy, u.C[s], cell.g[s], srcv[s], g[s]);
  if (live) {   // links 0-4 of the flow and the three scalars, one group each
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      if (!st_ok(pop_index(i, c, P), 4)) continue;
      if constexpr (SR) {
        stq_sr(dst + pop_index(i, c, P), o[i], g[0][i], g[1][i], g[2][i], r16(i), r16(9 + i),
               r16(14 + i), r16(19 + i));
      } else {
        stq(dst + pop_index(i, c, P), o[i], g[0][i], g[1][i], g[2][i]);
      }
    }
  }
}

// SR: 16-bit stores with stochastic rounding (a separate instantiation, so
// the round-to-nearest kernel carries none of its code); X as cell_update.
template <typename S, int BX, int BY, int MINB, bool SR = false, bool X = false>
__global__ void __launch_bounds__(BX * BY, MINB)
k_step(const S *__restrict__ src_p, S *__restrict__ dst, const uint8_t *__restrict__ mask,
       const uint16_t *__restrict__ mid, const MatCoef<typename Real<S>::type> *__restrict__ pal,
       KArgsT<typename Real<S>::type> a) {
  const int x = blockIdx.x * BX + (threadIdx.x % BX);
  const int y = blockIdx.y * BY + (threadIdx.x / BX);
  if (x >= a.nx || y >= a.ny) return;
  cell_update<S, false, SR, X>(src_p, dst, mask, mid, pal, a, x, y);
}

// The step with its reverse records (plain cathode set-ups, round-to-
// nearest storage: what the adjoint covers).
template <typename S, int BX, int BY, int MINB>
__global__ void __launch_bounds__(BX * BY, MINB)
k_step_rec(const S *__restrict__ src_p, S *__restrict__ dst, const uint8_t *__restrict__ mask,
           const uint16_t *__restrict__ mid, const MatCoef<typename Real<S>::type> *__restrict__ pal,
           KArgsT<typename Real<S>::type> a, RecPtrs<typename Real<S>::type> rp) {
  const int x = blockIdx.x * BX + (threadIdx.x % BX);
  const int y = blockIdx.y * BY + (threadIdx.x / BX);
  if (x >= a.nx || y >= a.ny) return;
  cell_update<S, false, false, false, true>(src_p, dst, mask, mid, pal, a, x, y, rp);
}

// ------------------------------------------------------ launcher
template <typename S, int V>
void launch_step_v(const void *src, void *dst, const DevGeom &g, const KArgs &a, cudaStream_t st) {
  constexpr StepShape sh = kStepShapes[V];
  dim3 grid((a.nx + sh.bx - 1) / sh.bx, (a.ny + sh.by - 1) / sh.by);
  using R = typename Real<S>::type;
  if (needs_extended(a)) {
    // two shapes of the extended step: 128 x 2 at 80 registers (variants
    // 0-2) and 64 x 2 at 64 registers (the rest); the tuner picks one
    constexpr StepShape sx = kStepShapes[V <= 2 ? 1 : 7];
    dim3 gx((a.nx + sx.bx - 1) / sx.bx, (a.ny + sx.by - 1) / sx.by);
    k_step<S, sx.bx, sx.by, sx.minb, false, true><<<gx, sx.bx * sx.by, 0, st>>>(
        (const S *)src, (S *)dst, g.mask, g.mid, (const MatCoef<R> *)g.pal, narrow_args<R>(a));
    return;
  }
  if constexpr (sizeof(S) == 2) {
    if (a.stochastic) {
      k_step<S, sh.bx, sh.by, sh.minb, true><<<grid, sh.bx * sh.by, 0, st>>>(
          (const S *)src, (S *)dst, g.mask, g.mid, (const MatCoef<R> *)g.pal, narrow_args<R>(a));
      return;
    }
  }
  k_step<S, sh.bx, sh.by, sh.minb><<<grid, sh.bx * sh.by, 0, st>>>(
      (const S *)src, (S *)dst, g.mask, g.mid, (const MatCoef<R> *)g.pal, narrow_args<R>(a));
}

constexpr StepShape kRecShape = {64, 2, 6};
template <typename S>
void launch_step_rec(const void *src, void *dst, const DevGeom &g, const KArgs &a,
                     const RecBufs &r, cudaStream_t st) {
  using R = typename Real<S>::type;
  dim3 grid((a.nx + kRecShape.bx - 1) / kRecShape.bx, (a.ny + kRecShape.by - 1) / kRecShape.by);
  const RecPtrs<R> rp{(R *)r.cell, (R *)r.own, (R *)r.pulled, r.slot};
  k_step_rec<S, kRecShape.bx, kRecShape.by, kRecShape.minb><<<grid, kRecShape.bx * kRecShape.by,
                                                              0, st>>>(
      (const S *)src, (S *)dst, g.mask, g.mid, (const MatCoef<R> *)g.pal, narrow_args<R>(a), rp);
}

template <typename S>
void launch_step(const void *src, void *dst, const DevGeom &g, const KArgs &a, int variant,
                 cudaStream_t st) {
  switch (variant) {
    case 1: launch_step_v<S, 1>(src, dst, g, a, st); break;
    case 2: launch_step_v<S, 2>(src, dst, g, a, st); break;
    case 3: launch_step_v<S, 3>(src, dst, g, a, st); break;
    case 4: launch_step_v<S, 4>(src, dst, g, a, st); break;
    case 5: launch_step_v<S, 5>(src, dst, g, a, st); break;
    case 6: launch_step_v<S, 6>(src, dst, g, a, st); break;
    case 7: launch_step_v<S, 7>(src, dst, g, a, st); break;
    default: launch_step_v<S, 0>(src, dst, g, a, st); break;
  }
}

}  // namespace pemlbm
