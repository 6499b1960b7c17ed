// The coupled step kernel (one cell per thread, pull scheme) and its
// launcher, templated on the population storage type S.  Kept apart from
// the read-out, batch and adjoint kernels so that its sources can be
// identified on their own.
#pragma once
#include "lbm_core.cuh"
#include "lbm_launch.h"

namespace pemlbm {

// ------------------------------------------------------------- step (K1)
// One coupled update of cell (x, y): src -> dst.  Shared by the single-
// domain step and the batched steps.
template <typename S, bool CG = false>
__device__ __forceinline__ void cell_update(const S *__restrict__ src_p, S *__restrict__ dst,
                                            const uint8_t *__restrict__ mask,
                                            const uint16_t *__restrict__ mid,
                                            const MatCoef<typename Real<S>::type> *__restrict__ pal,
                                            const KArgsT<typename Real<S>::type> &a, int x,
                                            int y) {
  using R = typename Real<S>::type;
  const long long c = (long long)y * a.nxp + x;
  const Pops<S, CG> src{src_p, a.plane, a.nxp};
  const uint8_t m = mask[c];
  Cell<R> cell;
  load_interior<S, R, CG>(src, a, x, y, cell);
  // solid cells run the same arithmetic on their (unused) values and only
  // skip the stores, so no branch stands between the mask and the loads
  const bool live = (m & REG_MASK) != REG_SOLID;
  const MatCoef<R> mc = pal[mid[c]];
  if (m & M_EDGE) {
    // next to grains but away from the lattice's edges: bounce-back only
    if ((m & M_EDGE) == M_NEAR_SOLID) bounce_solid<S, R, CG>(src, x, y, mask[a.plane + c], cell);
    else fix_edges<S, R, CG>(src, a, mask, mid, pal, mc, x, y, m, cell);
  }
  if (a.mode == 0 && (m & M_YLO)) surface_reaction<S, R, CG>(src, a, mc, x, cell);
  R S_vol = 0;
  if (a.mode == 1 && (m & REG_MASK) == REG_CATALYST) S_vol = volume_sink<S, R, CG>(src, a, x, y);
  const Macro<R> u = macros<R>(a, mc, cell);
  R o[9];
  collide_flow<R>(a, mc, u, cell.f, o);
  S *out = dst + c;
  if (live) {
#pragma unroll
    for (int i = 0; i < 9; ++i) st_r(out + (long long)i * a.plane, o[i]);
  }
  const R srcv[3] = {-S_vol * R(a.hpo) * mc.inv_sigma, S_vol, R(-2) * S_vol};
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    R g[5];
    collide_scalar<R>(a, mc, s, u.ux, u.uy, u.C[s], cell.g[s], srcv[s], g);
    if (live) {
#pragma unroll
      for (int i = 0; i < 5; ++i) st_r(out + (long long)(9 + 5 * s + i) * a.plane, g[i]);
    }
  }
}

template <typename S, int BX, int BY, int MINB>
__global__ void __launch_bounds__(BX * BY, MINB)
k_step(const S *__restrict__ src_p, S *__restrict__ dst, const uint8_t *__restrict__ mask,
       const uint16_t *__restrict__ mid, const MatCoef<typename Real<S>::type> *__restrict__ pal,
       KArgsT<typename Real<S>::type> a) {
  const int x = blockIdx.x * BX + (threadIdx.x % BX);
  const int y = blockIdx.y * BY + (threadIdx.x / BX);
  if (x >= a.nx || y >= a.ny) return;
  cell_update<S>(src_p, dst, mask, mid, pal, a, x, y);
}

// ------------------------------------------------------ launcher
template <typename S, int V>
void launch_step_v(const void *src, void *dst, const DevGeom &g, const KArgs &a, cudaStream_t st) {
  constexpr StepShape sh = kStepShapes[V];
  dim3 grid((a.nx + sh.bx - 1) / sh.bx, (a.ny + sh.by - 1) / sh.by);
  k_step<S, sh.bx, sh.by, sh.minb><<<grid, sh.bx * sh.by, 0, st>>>(
      (const S *)src, (S *)dst, g.mask, g.mid,
      (const MatCoef<typename Real<S>::type> *)g.pal, narrow_args<typename Real<S>::type>(a));
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
