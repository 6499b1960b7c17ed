// Kernels of the coupled cathode step and its read-outs, templated on the
// population storage type S (double, float, bf16, fp16).  Arithmetic runs in
// R = Real<S>::type (FP64 for double storage, FP32 otherwise); reductions
// accumulate in FP64.
#pragma once
#include "lbm_adjoint.cuh"
#include "lbm_core.cuh"
#include "lbm_launch.h"
#include "lbm_step.cuh"

namespace pemlbm {

// ---------------------------------------------------- batched steps (K6)
// Many cases of uneven size advance together.  The tiles of all cases (BX x
// BY cells each) are numbered case after case; tile_start[c] is the first
// tile of case c.  A block finds its case by binary search and stages that
// case's arguments in shared memory.
__device__ __forceinline__ int batch_case_of(const int *__restrict__ tile_start, int ncases, int t) {
  int lo = 0, hi = ncases - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(tile_start + mid) <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename R>
__device__ __forceinline__ void stage_args(const BatchCaseT<R> *__restrict__ cases, int c,
                                           KArgsT<R> *sa) {
  const int *srcw = reinterpret_cast<const int *>(&cases[c].a);
  int *dstw = reinterpret_cast<int *>(sa);
  for (int k = threadIdx.x; k < (int)(sizeof(KArgsT<R>) / sizeof(int)); k += blockDim.x)
    dstw[k] = __ldg(srcw + k);
}

template <typename S, int BX, int BY, bool CG>
__device__ __forceinline__ void batch_tile(const BatchCaseT<typename Real<S>::type> *__restrict__ cases,
                                           const int *__restrict__ tile_start, int ncases, int t,
                                           int parity, KArgsT<typename Real<S>::type> *sa,
                                           int *sc) {
  using R = typename Real<S>::type;
  if (threadIdx.x == 0) *sc = batch_case_of(tile_start, ncases, t);
  __syncthreads();
  const int c = *sc;
  stage_args(cases, c, sa);
  __syncthreads();
  const BatchCaseT<R> &bc = cases[c];
  const int tile = t - __ldg(tile_start + c);
  const int tx = tile % bc.tiles_x, ty = tile / bc.tiles_x;
  const int x = tx * BX + (threadIdx.x % BX);
  const int cur = bc.cur0 ^ parity;
  const S *src = (const S *)bc.pop[cur];
  S *dst = (S *)bc.pop[cur ^ 1];
  for (int r = 0; r < kBatchRows; ++r) {
    const int y = (ty * kBatchRows + r) * BY + (threadIdx.x / BX);
    if (x < sa->nx && y < sa->ny)
      cell_update<S, CG>(src, dst, bc.mask, bc.mid, (const MatCoef<R> *)bc.pal, *sa, x, y);
  }
  __syncthreads();   // the staged arguments are reused by the next tile
}

// One launch per step: one block per tile.
template <typename S, int BX, int BY, int MINB>
__global__ void __launch_bounds__(BX * BY, MINB)
k_batch_step(const BatchCaseT<typename Real<S>::type> *__restrict__ cases,
             const int *__restrict__ tile_start, int ncases, int parity) {
  __shared__ KArgsT<typename Real<S>::type> sa;
  __shared__ int sc;
  batch_tile<S, BX, BY, false>(cases, tile_start, ncases, blockIdx.x, parity, &sa, &sc);
}

// Grid-wide barrier of a cooperative launch.  Every wait is bounded: after
// spin_limit polls the block raises *status and returns false, and so does
// every block that later finds *status raised.
__device__ __forceinline__ bool grid_barrier(unsigned *count, unsigned *gen, unsigned nblocks,
                                             int *status, long long spin_limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *vgen = gen;
    const unsigned g = *vgen;
    __threadfence();
    if (atomicAdd(count, 1u) == nblocks - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      long long spins = 0;
      while (*vgen == g) {
        if (++spins > spin_limit) {
          atomicExch(status, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *((volatile int *)status) == 0;
}

// Persistent: nsteps steps in one cooperative launch of co-resident blocks,
// each looping over tiles, a grid barrier between steps.  Population loads
// bypass L1 (other SMs wrote them in the previous step).
template <typename S, int BX, int BY, int MINB>
__global__ void __launch_bounds__(BX * BY, MINB)
k_batch_persistent(const BatchCaseT<typename Real<S>::type> *__restrict__ cases,
                   const int *__restrict__ tile_start, int ncases, int total_tiles, int nsteps,
                   unsigned *bar, int *status, long long spin_limit) {
  __shared__ KArgsT<typename Real<S>::type> sa;
  __shared__ int sc;
  for (int step = 0; step < nsteps; ++step) {
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x)
      batch_tile<S, BX, BY, true>(cases, tile_start, ncases, t, step & 1, &sa, &sc);
    if (!grid_barrier(bar, bar + 1, gridDim.x, status, spin_limit)) return;
  }
}

// ------------------------------------------------ fields of the last step
// out [6][ny][nx] doubles: u_x, u_y, p, T, C_O2, C_H2O from stream(src).
template <typename S>
__global__ void k_fields(const S *__restrict__ src_p, const uint8_t *__restrict__ mask,
                         const uint16_t *__restrict__ mid,
                         const MatCoef<typename Real<S>::type> *__restrict__ pal,
                         KArgsT<typename Real<S>::type> a, double *__restrict__ out) {
  using R = typename Real<S>::type;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  const long long c = (long long)y * a.nxp + x, n = (long long)a.nx * a.ny,
                  o = (long long)y * a.nx + x;
  const uint8_t m = mask[c];
  if ((m & REG_MASK) == REG_SOLID) {
    for (int k = 0; k < 6; ++k) out[k * n + o] = 0.0;
    return;
  }
  const Pops<S> src{src_p, a.plane, a.nxp};
  const MatCoef<R> mc = pal[mid[c]];
  Cell<R> cell;
  pull_cell<S, R, false, true>(src, a, mask, mid, pal, mc, x, y, m, cell);
  if (a.mode == 0 && (m & M_YLO)) surface_reaction<S, R>(src, a, mc, x, cell);
  const Macro<R> u = macros<R, true>(a, mc, cell);
  out[0 * n + o] = (double)u.ux;
  out[1 * n + o] = (double)u.uy;
  out[2 * n + o] = ((double)u.Pdev + 1.0 / 3.0) / (double)mc.phi;
  for (int s = 0; s < 3; ++s) out[(3 + s) * n + o] = (double)u.C[s] + a.Cref[s];
}

// ---------------------------------------------- FP64 block reduction
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double *smem /* N * 32 */) {
#pragma unroll
  for (int k = 0; k < N; ++k)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0)
    for (int k = 0; k < N; ++k) smem[k * 32 + warp] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      double t = lane < nw ? smem[k * 32 + lane] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
      v[k] = t;
    }
  }
}

// ------------------------------------- inlet / outlet balances (K3b)
// Net inflow of mass and of the three scalars through the inlet column and
// through the outlet column during the last step, recomputed from the state
// before it (src) with the step's own boundary pulls.  Each incoming
// boundary link counts its pulled value, each population that leaves the
// lattice through the column counts negatively; opposite links carry equal
// weights, so the deviation references cancel.  One block; rows in a fixed
// order per thread, then a fixed-order block sum (deterministic).
// out: in_mass, in_T, in_O2, in_H2O, out_mass, out_T, out_O2, out_H2O.
template <typename S>
__global__ void __launch_bounds__(kReduceThreads)
k_balances(const S *__restrict__ src_p, const uint8_t *__restrict__ mask,
           const uint16_t *__restrict__ mid, const MatCoef<typename Real<S>::type> *__restrict__ pal,
           KArgsT<typename Real<S>::type> a, double *__restrict__ out) {
  using R = typename Real<S>::type;
  __shared__ double sm[8 * 32];
  const Pops<S> src{src_p, a.plane, a.nxp};
  const int EX[9] = EX9_TAB, EY[9] = EY9_TAB, OP[9] = OP9_TAB;
  double acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = 0.0;
  if (!a.periodic) {
    for (int y = threadIdx.x; y < a.ny; y += blockDim.x) {
      for (int side = 0; side < 2; ++side) {
        if (side ? a.halo_hi : a.halo_lo) continue;   // a slab side: no flow out of the lattice
        const int x = side ? a.nx - 1 : 0;
        const long long c = (long long)y * a.nxp + x;
        const uint8_t m = mask[c];
        if ((m & REG_MASK) == REG_SOLID) continue;
        const MatCoef<R> mc = pal[mid[c]];
        const int dir = side ? -1 : 1;             // e_x of the links entering through this side
        double *o = acc + 4 * side;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
          const int sy = y - EY[i];
          if (EX[i] == dir) {                       // enters through the column
            if (sy < 0 || sy >= a.ny) continue;     // a wall link
            const R v = pull_flow_edge<S, R, false, true>(src, a, mask, mid, pal, i, x, y, m, R(0));
            // inlet: the pulled value replaces the bounced one (the moving-wall
            // or virtual-column excess); outlet: the whole pulled value
            o[0] += side ? (double)v : (double)v - (double)R(src.at(OP[i], x, y));
          } else if (side && EX[i] == -dir) {       // leaves through the outlet
            const int ty = y + EY[i];
            if (ty >= 0 && ty < a.ny) o[0] -= (double)R(src.at(i, x, y));
          }
        }
#pragma unroll
        for (int s = 0; s < 3; ++s) {
          const int q = 9 + 5 * s;
          const int lin = side ? 3 : 1;              // D2Q5 link entering through the column
          const R v = pull_scalar_edge<S, R, false, true>(src, a, mask, mc, s, lin, x, y, m, R(0));
          if (side) {
            o[1 + s] += (double)v - (double)R(src.at(q + 1, x, y));   // in via 3, out via 1
          } else if ((m & M_INLET) || ((a.wall_dir >> s) & 1)) {
            o[1 + s] += (double)v - (double)R(src.at(q + 3, x, y));   // Dirichlet excess
          }
        }
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], off);
  }
  if (lane == 0)
    for (int k = 0; k < 8; ++k) sm[k * 32 + warp] = acc[k];
  __syncthreads();
  if (threadIdx.x < 8) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += sm[threadIdx.x * 32 + w];
    out[threadIdx.x] = t;
  }
}

// --------------------------------------------- catalyst reduction (K3)
// Recomputes the reaction applied in the last step from the state before it
// (src).  Blocks of kCatalystBX columns x kCatalystBY row-threads: each
// column's O2 consumption J(x) (the surface link of the thin film, or the
// sum of the volumetric sinks over the catalyst rows) is reduced in shared
// memory in a fixed order and written, with its heat h J(x), to colsum
// [2][nx] (FP64); profile[x] = J(x) i_scale (A/cm^2) when not NULL.
template <typename S>
__global__ void __launch_bounds__(kCatalystBX * kCatalystBY)
k_catalyst(const S *__restrict__ src_p, const uint8_t *__restrict__ mask,
           const uint16_t *__restrict__ mid, const MatCoef<typename Real<S>::type> *__restrict__ pal,
           KArgsT<typename Real<S>::type> a, double i_scale, float *__restrict__ profile,
           double *__restrict__ colsum) {
  using R = typename Real<S>::type;
  __shared__ double sm[kCatalystBY][kCatalystBX];
  const Pops<S> src{src_p, a.plane, a.nxp};
  const int tx = threadIdx.x % kCatalystBX, ty = threadIdx.x / kCatalystBX;
  const int x = blockIdx.x * kCatalystBX + tx;
  double J = 0.0;
  if (x < a.nx) {
    if (a.mode == 0) {
      if (ty == 0 && (mask[x] & REG_MASK) != REG_SOLID) {
        const MatCoef<R> mc = pal[mid[x]];
        Cell<R> cell;  // only the upward links matter: the bounced g*_4 of each scalar
        cell.g[1][2] = R(src.at(9 + 5 * 1 + 4, x, 0));
        cell.g[0][2] = 0;
        cell.g[2][2] = 0;
        J = (double)surface_reaction<S, R>(src, a, mc, x, cell);
      }
    } else {
      for (int y = ty; y < a.ny_cl; y += kCatalystBY)
        if ((mask[(long long)y * a.nxp + x] & REG_MASK) == REG_CATALYST)
          J -= (double)volume_sink<S, R>(src, a, x, y);
    }
  }
  sm[ty][tx] = J;
  __syncthreads();
  if (ty == 0 && x < a.nx) {
    double t = 0.0;
    for (int k = 0; k < kCatalystBY; ++k) t += sm[k][tx];
    colsum[x] = t;
    colsum[a.nx + x] = t * a.hpo;
    if (profile) profile[x] = (float)(t * i_scale);
  }
}

// Sums the per-column J and heat in a fixed order: out[0], out[1].
__global__ void k_sum_columns(const double *__restrict__ colsum, int nx, double *__restrict__ out);

// ------------------------------------------------- residual (K4)
// Moments of the post-collision state: X = (j_x, j_y, T - T_in, C_O2, C_H2O).
// One thread per cell: the change since the snapshot and the value are
// squared, summed over the warp by shuffles, then over the block in FP64
// (10 partial sums per block).  The values are compared with snap_in and
// written to snap_out (arithmetic precision R).  The two may be one buffer
// (updated in place), but distinct buffers are much faster: reading and then
// writing the same addresses in one launch took about 4x the kernel's time at
// 4096 x 1024.  Non-finite values raise *bad.
template <typename S>
__global__ void __launch_bounds__(kResidualBX * kResidualBY)
k_residual(const S *__restrict__ src_p, const uint8_t *__restrict__ mask,
           KArgsT<typename Real<S>::type> a, const typename Real<S>::type *snap_in,
           typename Real<S>::type *snap_out, double *__restrict__ partial,
           int *__restrict__ bad) {
  using R = typename Real<S>::type;
  __shared__ R sm[10 * 32];
  const Pops<S> src{src_p, a.plane, a.nxp};
  const int x = blockIdx.x * kResidualBX + (threadIdx.x % kResidualBX);
  const int y = blockIdx.y * kResidualBY + (threadIdx.x / kResidualBX);
  R v[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) v[k] = R(0);
  if (x < a.nx && y < a.ny) {
    const long long n = (long long)a.nx * a.ny, o = (long long)y * a.nx + x;
    // the cell's values are loaded without waiting for its mask
    Cell<R> own;
    load_own<S, R>(src, x, y, own);
    const bool live = (mask[(long long)y * a.nxp + x] & REG_MASK) != REG_SOLID;
    const R *d = own.f;
    R X[5];
    X[0] = d[1] - d[3] + d[5] - d[6] - d[7] + d[8];
    X[1] = d[2] - d[4] + d[5] + d[6] - d[7] - d[8];
    X[2] = d2q5_sum<R>(own.g[0][0], own.g[0][1], own.g[0][2], own.g[0][3], own.g[0][4]) + a.theta0;
    X[3] = d2q5_sum<R>(own.g[1][0], own.g[1][1], own.g[1][2], own.g[1][3], own.g[1][4]) + R(a.Cref[1]);
    X[4] = d2q5_sum<R>(own.g[2][0], own.g[2][1], own.g[2][2], own.g[2][3], own.g[2][4]) + R(a.Cref[2]);
    // all five snapshot values are read before any is written, so the loads
    // overlap (and an in-place update reads the old values)
    R prev[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) prev[k] = snap_in[k * n + o];
    if (live) {
      bool ok = true;
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        ok = ok && isfinite(X[k]);
        const R dv = X[k] - prev[k];
        v[k] = dv * dv;
        v[5 + k] = X[k] * X[k];
      }
#pragma unroll
      for (int k = 0; k < 5; ++k) snap_out[k * n + o] = X[k];
      if (!ok) *bad = 1;
    }
  }
#pragma unroll
  for (int k = 0; k < 10; ++k) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
  }
  // lane 0 holds the warp sums; only they are widened (the FP64 pipe is
  // narrow), and the block sum of the warp sums is FP64
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0)
    for (int k = 0; k < 10; ++k) sm[k * 32 + warp] = v[k];
  __syncthreads();
  if (threadIdx.x < 10) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += (double)sm[threadIdx.x * 32 + w];
    partial[((long long)blockIdx.y * gridDim.x + blockIdx.x) * 10 + threadIdx.x] = t;
  }
}

// Sums nblocks x 10 partials in a fixed order; 10 blocks, block k sums
// quantity k into out[k].
__global__ void k_sum_partials(const double *__restrict__ partial, int nblocks,
                               double *__restrict__ out);

// ----------------------------------------------------------- init (C2)
template <typename S>
__global__ void k_init(S *__restrict__ pop, const uint8_t *__restrict__ mask,
                       const uint16_t *__restrict__ mid,
                       const MatCoef<typename Real<S>::type> *__restrict__ pal,
                       KArgsT<typename Real<S>::type> a) {
  using R = typename Real<S>::type;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= a.nxp || y >= a.ny) return;
  const long long c = (long long)y * a.nxp + x;
  const bool live = x < a.nx && (mask[c] & REG_MASK) != REG_SOLID;
  R d0[3], d1[3];
  for (int s = 0; s < 3; ++s) {
    R w1 = live ? pal[mid[c]].w1[s] : R(a.wr1[s]);
    R w0 = R(1) - R(4) * w1;
    // equilibrium of C_in at rest with the cell's own b, minus the reference
    d0[s] = w0 * R(a.Cin[s]) - R(a.wr0[s]) * R(a.Cref[s]);
    d1[s] = w1 * R(a.Cin[s]) - R(a.wr1[s]) * R(a.Cref[s]);
    if (!live) d0[s] = d1[s] = R(0);
  }
  // flow deviations zero; links 0-4 by groups, then the diagonal flow links
  stq(pop + pop_index(0, c, a.plane), R(0), d0[0], d0[1], d0[2]);
  for (int i = 1; i < 5; ++i) stq(pop + pop_index(i, c, a.plane), R(0), d1[0], d1[1], d1[2]);
  for (int i = 5; i < 9; ++i) st_r(pop + pop_index(i, c, a.plane), R(0));
}

// ------------------------------------------- full-value state in/out
template <typename S>
__global__ void k_get_state(const S *__restrict__ pop, const uint8_t *__restrict__ mask,
                            KArgsT<typename Real<S>::type> a, double *__restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  const long long c = (long long)y * a.nxp + x, n = (long long)a.nx * a.ny,
                  o = (long long)y * a.nx + x;
  const bool solid = (mask[c] & REG_MASK) == REG_SOLID;
  const double W9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
  for (int q = 0; q < 24; ++q) {
    double ref;
    if (q < 9) ref = W9[q];
    else {
      const int s = (q - 9) / 5, i = (q - 9) % 5;
      ref = (double)(i == 0 ? a.wr0[s] : a.wr1[s]) * (double)a.Cref[s];
    }
    out[q * n + o] = solid ? 0.0 : (double)ld_r(pop + pop_index(q, c, a.plane)) + ref;
  }
}

template <typename S>
__global__ void k_set_state(S *__restrict__ pop, const uint8_t *__restrict__ mask,
                            KArgsT<typename Real<S>::type> a, const double *__restrict__ in) {
  using R = typename Real<S>::type;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  const long long c = (long long)y * a.nxp + x, n = (long long)a.nx * a.ny,
                  o = (long long)y * a.nx + x;
  const bool solid = (mask[c] & REG_MASK) == REG_SOLID;
  const double W9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
  for (int q = 0; q < 24; ++q) {
    double ref;
    if (q < 9) ref = W9[q];
    else {
      const int s = (q - 9) / 5, i = (q - 9) % 5;
      ref = (double)(i == 0 ? a.wr0[s] : a.wr1[s]) * (double)a.Cref[s];
    }
    st_r(pop + pop_index(q, c, a.plane), solid ? R(0) : R(in[q * n + o] - ref));
  }
}

// ------------------------------------------------------ launchers
template <typename S, int V>
void launch_batch_v(const BatchCase *cases, const int *tile_start, int ncases, int total_tiles,
                    int parity, cudaStream_t st) {
  constexpr StepShape sh = kStepShapes[V];
  k_batch_step<S, sh.bx, sh.by, sh.minb><<<total_tiles, sh.bx * sh.by, 0, st>>>(
      (const BatchCaseT<typename Real<S>::type> *)cases, tile_start, ncases, parity);
}

template <typename S>
void launch_batch_step(const BatchCase *cases, const int *tile_start, int ncases, int total_tiles,
                       int variant, int parity, cudaStream_t st) {
  switch (variant) {
    case 1: launch_batch_v<S, 1>(cases, tile_start, ncases, total_tiles, parity, st); break;
    case 2: launch_batch_v<S, 2>(cases, tile_start, ncases, total_tiles, parity, st); break;
    case 3: launch_batch_v<S, 3>(cases, tile_start, ncases, total_tiles, parity, st); break;
    case 4: launch_batch_v<S, 4>(cases, tile_start, ncases, total_tiles, parity, st); break;
    case 5: launch_batch_v<S, 5>(cases, tile_start, ncases, total_tiles, parity, st); break;
    case 6: launch_batch_v<S, 6>(cases, tile_start, ncases, total_tiles, parity, st); break;
    case 7: launch_batch_v<S, 7>(cases, tile_start, ncases, total_tiles, parity, st); break;
    default: launch_batch_v<S, 0>(cases, tile_start, ncases, total_tiles, parity, st); break;
  }
}


template <typename S>
cudaError_t launch_batch_persistent(const BatchCase *cases, const int *tile_start, int ncases,
                                    int total_tiles, int nsteps, unsigned *bar, int *status,
                                    long long spin_limit, cudaStream_t st) {
  auto kern = k_batch_persistent<S, kPersistBX, kPersistBY, kPersistMinB>;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPersistBX * kPersistBY, 0);
  if (e != cudaSuccess) return e;
  int grid = sms * per_sm;
  if (grid > total_tiles) grid = total_tiles;
  if (grid < 1) return cudaErrorInvalidConfiguration;
  const BatchCaseT<typename Real<S>::type> *rc = (const BatchCaseT<typename Real<S>::type> *)cases;
  void *args[] = {(void *)&rc, (void *)&tile_start, (void *)&ncases, (void *)&total_tiles,
                  (void *)&nsteps, (void *)&bar, (void *)&status, (void *)&spin_limit};
  return cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(kPersistBX * kPersistBY),
                                     args, 0, st);
}

template <typename R> AdjBufs<R> adj_bufs(const AdjPtrs &b) {
  return AdjBufs<R>{(const R *)b.lam, (R *)b.O, (R *)b.V, (const R *)b.O_in, (const R *)b.V_in,
                    (R *)b.gphi, (R *)b.gK, (R *)b.gD, b.gU, (R *)b.lam_out, b.pushed};
}

template <typename S>
void launch_adj_fold(const DevGeom &g, const KArgs &a, const AdjPtrs &b, cudaStream_t st) {
  using R = typename Real<S>::type;
  (void)g;
  k_adj_fold<R><<<4 * 152, 256, 0, st>>>((R *)b.gphi, (R *)b.gK, (R *)b.gD, b.tphi, b.tK, b.tD,
                                         a.plane);
}

// One reverse step.  The edge cells (a short list whose threads each run a
// long boundary path) go first on the side stream, concurrently with the
// interior cells on `st`; both push into lambda^{n-1}.  The fork and join
// are events, so the step can be captured into a graph (two parallel
// branches).
template <typename S>
void launch_adj_step(const RecBufs &r, const DevGeom &g, const KArgs &a, int fickian,
                     const AdjPtrs &b, long long seed_cell, int lam_complete, cudaStream_t st,
                     cudaStream_t side, cudaEvent_t fork, cudaEvent_t join) {
  using R = typename Real<S>::type;
  const KArgsT<R> an = narrow_args<R>(a);
  const AdjBufs<R> B = adj_bufs<R>(b);
  const MatCoef<R> *pal = (const MatCoef<R> *)g.pal;
  const RecPtrs<R> rp{(R *)r.cell, (R *)r.own, (R *)r.pulled, r.slot};
  auto edge = [&] {
    if (b.n_edge <= 0) return;
    cudaStreamWaitEvent(side, fork, 0);
    k_adj_edge<R><<<(b.n_edge + kEdgeWarps - 1) / kEdgeWarps, 32 * kEdgeWarps, 0, side>>>(
        rp, g.mask, g.mid, pal, an, fickian, B, b.cells, b.n_edge, seed_cell, lam_complete);
    cudaEventRecord(join, side);
  };
  if (b.n_edge > 0) cudaEventRecord(fork, st);
  if (kAdjEdgeFirst) edge();
  k_adj_interior<R><<<dim3((a.nx + 127) / 128, a.ny), 128, 0, st>>>(rp, g.mask, g.mid, pal, an,
                                                                    fickian, B);
  if (!kAdjEdgeFirst) edge();
  if (b.n_edge > 0) cudaStreamWaitEvent(st, join, 0);
}

// Completes lambda in place at the own-use cells after the last step
// (b.lam_out, b.O and b.V are that step's buffers).
template <typename S>
void launch_adj_finish(const DevGeom &g, const KArgs &a, const AdjPtrs &b, cudaStream_t st) {
  using R = typename Real<S>::type;
  if (b.n_own <= 0) return;
  const long long n = 24LL * b.n_own;
  k_adj_fix<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      g.mask, g.mid, (const MatCoef<R> *)g.pal, narrow_args<R>(a), adj_bufs<R>(b), b.cells,
      b.n_own);
}

template <typename S>
void launch_adj_seed_current(const void *src, const DevGeom &g, const KArgs &a, int fickian,
                             double weight, const AdjPtrs &b, cudaStream_t st) {
  using R = typename Real<S>::type;
  dim3 grid((a.nx + 127) / 128, a.ny);
  k_adj_seed_current<S><<<grid, 128, 0, st>>>((const S *)src, g.mask, g.mid,
                                              (const MatCoef<R> *)g.pal, narrow_args<R>(a),
                                              fickian, weight, adj_bufs<R>(b));
}

// Narrows a host table of batched cases into `staging` (pinned) and copies
// it to the device table.
template <typename S>
void batch_upload(const BatchCase *host, int n, void *staging, void *dev, cudaStream_t st) {
  using R = typename Real<S>::type;
  BatchCaseT<R> *out = (BatchCaseT<R> *)staging;
  for (int c = 0; c < n; ++c) {
    out[c].a = narrow_args<R>(host[c].a);
    out[c].pop[0] = host[c].pop[0];
    out[c].pop[1] = host[c].pop[1];
    out[c].mask = host[c].mask;
    out[c].mid = host[c].mid;
    out[c].pal = host[c].pal;
    out[c].cur0 = host[c].cur0;
    out[c].tiles_x = host[c].tiles_x;
  }
  cudaMemcpyAsync(dev, staging, sizeof(BatchCaseT<R>) * n, cudaMemcpyHostToDevice, st);
}

template <typename S>
void launch_fields(const void *src, const DevGeom &g, const KArgs &a, double *out, cudaStream_t st) {
  dim3 grid((a.nx + 127) / 128, a.ny);
  k_fields<S><<<grid, 128, 0, st>>>((const S *)src, g.mask, g.mid,
                                    (const MatCoef<typename Real<S>::type> *)g.pal,
                                    narrow_args<typename Real<S>::type>(a), out);
}

template <typename S>
void launch_balances(const void *src, const DevGeom &g, const KArgs &a, double *out,
                     cudaStream_t st) {
  using R = typename Real<S>::type;
  k_balances<S><<<1, kReduceThreads, 0, st>>>((const S *)src, g.mask, g.mid,
                                              (const MatCoef<R> *)g.pal, narrow_args<R>(a), out);
}

template <typename S>
void launch_catalyst(const void *src, const DevGeom &g, const KArgs &a, double i_scale,
                     float *profile, double *colsum, double *out, cudaStream_t st) {
  const int nb = (a.nx + kCatalystBX - 1) / kCatalystBX;
  k_catalyst<S><<<nb, kCatalystBX * kCatalystBY, 0, st>>>(
      (const S *)src, g.mask, g.mid, (const MatCoef<typename Real<S>::type> *)g.pal,
      narrow_args<typename Real<S>::type>(a), i_scale, profile, colsum);
  k_sum_columns<<<1, kReduceThreads, 0, st>>>(colsum, a.nx, out);
}

template <typename S>
void launch_residual(const void *src, const DevGeom &g, const KArgs &a, const void *snap_in,
                     void *snap_out, double *partial, int *bad, double *out, cudaStream_t st) {
  dim3 grid((a.nx + kResidualBX - 1) / kResidualBX, (a.ny + kResidualBY - 1) / kResidualBY);
  k_residual<S><<<grid, kResidualBX * kResidualBY, 0, st>>>(
      (const S *)src, g.mask, narrow_args<typename Real<S>::type>(a),
      (const typename Real<S>::type *)snap_in, (typename Real<S>::type *)snap_out, partial, bad);
  k_sum_partials<<<10, kReduceThreads, 0, st>>>(partial, grid.x * grid.y, out);
}

template <typename S>
void launch_init(void *pop, const DevGeom &g, const KArgs &a, cudaStream_t st) {
  dim3 grid((a.nxp + 127) / 128, a.ny);
  k_init<S><<<grid, 128, 0, st>>>((S *)pop, g.mask, g.mid,
                                  (const MatCoef<typename Real<S>::type> *)g.pal,
                                  narrow_args<typename Real<S>::type>(a));
}

template <typename S>
void launch_get_state(const void *pop, const DevGeom &g, const KArgs &a, double *out, cudaStream_t st) {
  dim3 grid((a.nx + 127) / 128, a.ny);
  k_get_state<S><<<grid, 128, 0, st>>>((const S *)pop, g.mask,
                                        narrow_args<typename Real<S>::type>(a), out);
}

template <typename S>
void launch_set_state(void *pop, const DevGeom &g, const KArgs &a, const double *in, cudaStream_t st) {
  dim3 grid((a.nx + 127) / 128, a.ny);
  k_set_state<S><<<grid, 128, 0, st>>>((S *)pop, g.mask, narrow_args<typename Real<S>::type>(a),
                                        in);
}

template <typename S> unsigned long long bounds_first_bad() {
#ifdef PEMLBM_BOUNDS_CHECK
  unsigned long long v = 0, zero = 0;
  cudaMemcpyFromSymbol(&v, g_bounds_first_bad, sizeof v);
  cudaMemcpyToSymbol(g_bounds_first_bad, &zero, sizeof zero);
  return v;
#else
  return 0;
#endif
}

#define PEMLBM_INSTANTIATE(S)                                                                   \
  template unsigned long long bounds_first_bad<S>();                                           \
  template void launch_step<S>(const void *, void *, const DevGeom &, const KArgs &, int,       \
                               cudaStream_t);                                                   \
  template void launch_fields<S>(const void *, const DevGeom &, const KArgs &, double *,        \
                                 cudaStream_t);                                                 \
  template void launch_balances<S>(const void *, const DevGeom &, const KArgs &, double *,      \
                                   cudaStream_t);                                                \
  template void launch_catalyst<S>(const void *, const DevGeom &, const KArgs &, double,        \
                                   float *, double *, double *, cudaStream_t);                  \
  template void launch_residual<S>(const void *, const DevGeom &, const KArgs &, const void *,  \
                                   void *, double *, int *, double *, cudaStream_t);            \
  template void launch_init<S>(void *, const DevGeom &, const KArgs &, cudaStream_t);           \
  template void launch_get_state<S>(const void *, const DevGeom &, const KArgs &, double *,     \
                                    cudaStream_t);                                              \
  template void launch_set_state<S>(void *, const DevGeom &, const KArgs &, const double *,     \
                                    cudaStream_t);                                              \
  template void launch_batch_step<S>(const BatchCase *, const int *, int, int, int, int,        \
                                     cudaStream_t);                                             \
  template cudaError_t launch_batch_persistent<S>(const BatchCase *, const int *, int, int, int, \
                                                  unsigned *, int *, long long, cudaStream_t);  \
  template void batch_upload<S>(const BatchCase *, int, void *, void *, cudaStream_t);         \
  template void launch_step_rec<S>(const void *, void *, const DevGeom &, const KArgs &,         \
                                   const RecBufs &, cudaStream_t);                               \
  template void launch_adj_step<S>(const RecBufs &, const DevGeom &, const KArgs &, int,          \
                                   const AdjPtrs &, long long, int, cudaStream_t, cudaStream_t,    \
                                   cudaEvent_t, cudaEvent_t);                                      \
  template void launch_adj_finish<S>(const DevGeom &, const KArgs &, const AdjPtrs &,            \
                                     cudaStream_t);                                              \
  template void launch_adj_fold<S>(const DevGeom &, const KArgs &, const AdjPtrs &,              \
                                   cudaStream_t);                                               \
  template void launch_adj_seed_current<S>(const void *, const DevGeom &, const KArgs &, int,    \
                                           double, const AdjPtrs &, cudaStream_t);

}  // namespace pemlbm
