// Kernels of the coupled cathode step and its read-outs, templated on the
// population storage type S (double, float, bf16, fp16).  Arithmetic runs in
// R = Real<S>::type (FP64 for double storage, FP32 otherwise); reductions
// accumulate in FP64.
#pragma once
#include "lbm_core.cuh"
#include "lbm_launch.h"

namespace pemlbm {

// ------------------------------------------------------------- step (K1)
template <typename S>
__global__ void __launch_bounds__(kStepThreads)
k_step(const S *__restrict__ src_p, S *__restrict__ dst, const uint8_t *__restrict__ mask,
       const uint16_t *__restrict__ mid, const MatCoef<typename Real<S>::type> *__restrict__ pal,
       KArgs a) {
  using R = typename Real<S>::type;
  const int x = blockIdx.x * kStepBX + (threadIdx.x % kStepBX);
  const int y = blockIdx.y * kStepBY + (threadIdx.x / kStepBX);
  if (x >= a.nx || y >= a.ny) return;
  const long long c = (long long)y * a.nxp + x;
  const uint8_t m = mask[c];
  if ((m & REG_MASK) == REG_SOLID) return;
  const Pops<S> src{src_p, a.plane, a.nxp};
  const MatCoef<R> mc = pal[mid[c]];
  Cell<R> cell;
  pull_cell<S, R>(src, a, mask, mid, pal, mc, x, y, m, cell);
  if (a.mode == 0 && (m & M_YLO)) surface_reaction<S, R>(src, a, mc, x, cell);
  R S_vol = 0;
  if (a.mode == 1 && (m & REG_MASK) == REG_CATALYST) S_vol = volume_sink<S, R>(src, a, x, y);
  const Macro<R> u = macros<R>(a, mc, cell);
  R o[9];
  collide_flow<R>(a, mc, u, cell.f, o);
  S *out = dst + c;
#pragma unroll
  for (int i = 0; i < 9; ++i) st_r(out + (long long)i * a.plane, o[i]);
  const R srcv[3] = {-S_vol * R(a.hpo), S_vol, R(-2) * S_vol};
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    R g[5];
    collide_scalar<R>(a, mc, s, u.ux, u.uy, u.C[s], cell.g[s], srcv[s], g);
#pragma unroll
    for (int i = 0; i < 5; ++i) st_r(out + (long long)(9 + 5 * s + i) * a.plane, g[i]);
  }
}

// ------------------------------------------------ fields of the last step
// out [6][ny][nx] doubles: u_x, u_y, p, T, C_O2, C_H2O from stream(src).
template <typename S>
__global__ void k_fields(const S *__restrict__ src_p, const uint8_t *__restrict__ mask,
                         const uint16_t *__restrict__ mid,
                         const MatCoef<typename Real<S>::type> *__restrict__ pal, KArgs a,
                         double *__restrict__ out) {
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
  pull_cell<S, R>(src, a, mask, mid, pal, mc, x, y, m, cell);
  if (a.mode == 0 && (m & M_YLO)) surface_reaction<S, R>(src, a, mc, x, cell);
  const Macro<R> u = macros<R>(a, mc, cell);
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

// --------------------------------------------- catalyst reduction (K3)
// Recomputes the reaction applied in the last step from the state before it
// (src): per column the O2 consumed J(x) and the heat q(x).  One block of
// kReduceThreads threads; out[0] = sum J, out[1] = sum q (FP64, lattice
// units); profile[x] = J(x) * i_scale (A/cm^2) if not NULL.
template <typename S>
__global__ void __launch_bounds__(kReduceThreads)
k_catalyst(const S *__restrict__ src_p, const uint8_t *__restrict__ mask,
           const uint16_t *__restrict__ mid, const MatCoef<typename Real<S>::type> *__restrict__ pal,
           KArgs a, double i_scale, float *__restrict__ profile, double *__restrict__ out) {
  using R = typename Real<S>::type;
  __shared__ double sm[2 * 32];
  const Pops<S> src{src_p, a.plane, a.nxp};
  double acc[2] = {0.0, 0.0};
  for (int x = threadIdx.x; x < a.nx; x += blockDim.x) {
    double J = 0.0;
    if (a.mode == 0) {
      const uint8_t m = mask[x];
      if ((m & REG_MASK) != REG_SOLID) {
        const MatCoef<R> mc = pal[mid[x]];
        Cell<R> cell;  // only the upward O2 link is needed: it is the bounced g*_4
        cell.g[1][2] = R(src.at(9 + 5 * 1 + 4, x, 0));
        cell.g[0][2] = 0;
        cell.g[2][2] = 0;
        J = (double)surface_reaction<S, R>(src, a, mc, x, cell);
      }
    } else {
      for (int y = 0; y < a.ny_cl; ++y) {
        const uint8_t m = mask[(long long)y * a.nxp + x];
        if ((m & REG_MASK) == REG_CATALYST) J -= (double)volume_sink<S, R>(src, a, x, y);
      }
    }
    acc[0] += J;
    acc[1] += J * a.hpo;
    if (profile) profile[x] = (float)(J * i_scale);
  }
  block_sum<2>(acc, sm);
  if (threadIdx.x == 0) {
    out[0] = acc[0];
    out[1] = acc[1];
  }
}

// ------------------------------------------------- residual (K4)
// Moments of the post-collision state: X = (j_x, j_y, T - T_in, C_O2, C_H2O).
// Accumulates per block sum (X - X_prev)^2 and sum X^2 (10 doubles), then
// overwrites the snapshot; flags non-finite values.
template <typename S>
__global__ void __launch_bounds__(kReduceThreads)
k_residual(const S *__restrict__ src_p, const uint8_t *__restrict__ mask, KArgs a,
           double *__restrict__ snap, double *__restrict__ partial, int *__restrict__ bad) {
  using R = typename Real<S>::type;
  __shared__ double sm[10 * 32];
  const Pops<S> src{src_p, a.plane, a.nxp};
  double acc[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) acc[k] = 0.0;
  const long long n = (long long)a.nx * a.ny;
  for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < n;
       o += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(o / a.nx), x = (int)(o % a.nx);
    if ((mask[(long long)y * a.nxp + x] & REG_MASK) == REG_SOLID) continue;
    R d[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) d[k] = R(src.at(k, x, y));
    double X[5];
    X[0] = (double)(d[1] - d[3] + d[5] - d[6] - d[7] + d[8]);
    X[1] = (double)(d[2] - d[4] + d[5] + d[6] - d[7] - d[8]);
    X[2] = (double)own_sum<S, R>(src, 0, x, y) + (a.Cref[0] - a.T_in);
    X[3] = (double)own_sum<S, R>(src, 1, x, y) + a.Cref[1];
    X[4] = (double)own_sum<S, R>(src, 2, x, y) + a.Cref[2];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      if (!isfinite(X[k])) *bad = 1;
      const double dv = X[k] - snap[k * n + o];
      acc[k] += dv * dv;
      acc[5 + k] += X[k] * X[k];
      snap[k * n + o] = X[k];
    }
  }
  block_sum<10>(acc, sm);
  if (threadIdx.x == 0)
    for (int k = 0; k < 10; ++k) partial[(long long)blockIdx.x * 10 + k] = acc[k];
}

// Sums nblocks x 10 partials in a fixed order.
__global__ void k_sum_partials(const double *__restrict__ partial, int nblocks,
                               double *__restrict__ out);

// ----------------------------------------------------------- init (C2)
template <typename S>
__global__ void k_init(S *__restrict__ pop, const uint8_t *__restrict__ mask,
                       const uint16_t *__restrict__ mid,
                       const MatCoef<typename Real<S>::type> *__restrict__ pal, KArgs a) {
  using R = typename Real<S>::type;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= a.nxp || y >= a.ny) return;
  const long long c = (long long)y * a.nxp + x;
  const bool live = x < a.nx && (mask[c] & REG_MASK) != REG_SOLID;
  for (int i = 0; i < 9; ++i) st_r(pop + i * a.plane + c, R(0));
  for (int s = 0; s < 3; ++s) {
    R w1 = live ? pal[mid[c]].w1[s] : R(a.wr1[s]);
    R w0 = R(1) - R(4) * w1;
    // equilibrium of C_in at rest with the cell's own b, minus the reference
    R d0 = w0 * R(a.Cin[s]) - R(a.wr0[s]) * R(a.Cref[s]);
    R d1 = w1 * R(a.Cin[s]) - R(a.wr1[s]) * R(a.Cref[s]);
    if (!live) d0 = d1 = R(0);
    st_r(pop + (9 + 5 * s) * a.plane + c, d0);
    for (int i = 1; i < 5; ++i) st_r(pop + (9 + 5 * s + i) * a.plane + c, d1);
  }
}

// ------------------------------------------- full-value state in/out
template <typename S>
__global__ void k_get_state(const S *__restrict__ pop, const uint8_t *__restrict__ mask, KArgs a,
                            double *__restrict__ out) {
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
      ref = (i == 0 ? a.wr0[s] : a.wr1[s]) * a.Cref[s];
    }
    out[q * n + o] = solid ? 0.0 : (double)ld_r(pop + q * a.plane + c) + ref;
  }
}

template <typename S>
__global__ void k_set_state(S *__restrict__ pop, const uint8_t *__restrict__ mask, KArgs a,
                            const double *__restrict__ in) {
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
      ref = (i == 0 ? a.wr0[s] : a.wr1[s]) * a.Cref[s];
    }
    st_r(pop + q * a.plane + c, solid ? R(0) : R(in[q * n + o] - ref));
  }
}

// ------------------------------------------------------ launchers
template <typename S>
void launch_step(const void *src, void *dst, const DevGeom &g, const KArgs &a, cudaStream_t st) {
  dim3 grid((a.nx + kStepBX - 1) / kStepBX, (a.ny + kStepBY - 1) / kStepBY);
  k_step<S><<<grid, kStepThreads, 0, st>>>(
      (const S *)src, (S *)dst, g.mask, g.mid,
      (const MatCoef<typename Real<S>::type> *)g.pal, a);
}

template <typename S>
void launch_fields(const void *src, const DevGeom &g, const KArgs &a, double *out, cudaStream_t st) {
  dim3 grid((a.nx + 127) / 128, a.ny);
  k_fields<S><<<grid, 128, 0, st>>>((const S *)src, g.mask, g.mid,
                                    (const MatCoef<typename Real<S>::type> *)g.pal, a, out);
}

template <typename S>
void launch_catalyst(const void *src, const DevGeom &g, const KArgs &a, double i_scale,
                     float *profile, double *out, cudaStream_t st) {
  k_catalyst<S><<<1, kReduceThreads, 0, st>>>((const S *)src, g.mask, g.mid,
                                              (const MatCoef<typename Real<S>::type> *)g.pal, a,
                                              i_scale, profile, out);
}

template <typename S>
void launch_residual(const void *src, const DevGeom &g, const KArgs &a, double *snap,
                     double *partial, int nblocks, int *bad, double *out, cudaStream_t st) {
  k_residual<S><<<nblocks, kReduceThreads, 0, st>>>((const S *)src, g.mask, a, snap, partial, bad);
  k_sum_partials<<<1, kReduceThreads, 0, st>>>(partial, nblocks, out);
}

template <typename S>
void launch_init(void *pop, const DevGeom &g, const KArgs &a, cudaStream_t st) {
  dim3 grid((a.nxp + 127) / 128, a.ny);
  k_init<S><<<grid, 128, 0, st>>>((S *)pop, g.mask, g.mid,
                                  (const MatCoef<typename Real<S>::type> *)g.pal, a);
}

template <typename S>
void launch_get_state(const void *pop, const DevGeom &g, const KArgs &a, double *out, cudaStream_t st) {
  dim3 grid((a.nx + 127) / 128, a.ny);
  k_get_state<S><<<grid, 128, 0, st>>>((const S *)pop, g.mask, a, out);
}

template <typename S>
void launch_set_state(void *pop, const DevGeom &g, const KArgs &a, const double *in, cudaStream_t st) {
  dim3 grid((a.nx + 127) / 128, a.ny);
  k_set_state<S><<<grid, 128, 0, st>>>((S *)pop, g.mask, a, in);
}

#define PEMLBM_INSTANTIATE(S)                                                                   \
  template void launch_step<S>(const void *, void *, const DevGeom &, const KArgs &, cudaStream_t); \
  template void launch_fields<S>(const void *, const DevGeom &, const KArgs &, double *,        \
                                 cudaStream_t);                                                 \
  template void launch_catalyst<S>(const void *, const DevGeom &, const KArgs &, double,        \
                                   float *, double *, cudaStream_t);                            \
  template void launch_residual<S>(const void *, const DevGeom &, const KArgs &, double *,      \
                                   double *, int, int *, double *, cudaStream_t);               \
  template void launch_init<S>(void *, const DevGeom &, const KArgs &, cudaStream_t);           \
  template void launch_get_state<S>(const void *, const DevGeom &, const KArgs &, double *,     \
                                    cudaStream_t);                                              \
  template void launch_set_state<S>(void *, const DevGeom &, const KArgs &, const double *,     \
                                    cudaStream_t);

}  // namespace pemlbm
