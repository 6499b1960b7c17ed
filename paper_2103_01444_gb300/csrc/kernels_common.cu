// Type-independent kernels: node mask, material palette, partial sums.
#include "lbm_kernels.cuh"

namespace pemlbm {

// Node mask (Sec. 4 geometry): region by rows, boundary bits by position,
// explicit solids, and a flag for cells with a solid D2Q9 neighbour; a
// second plane of the same size says which neighbours are solid.  The
// domain may be the x-slab [x0, x0 + nx) of a lattice nxg wide: positions,
// boundary bits and solid neighbours are those of the whole lattice (solid
// is [ny][nxg]), and a slab side inside the lattice gets no x bits.
__global__ void k_build_mask(uint8_t *__restrict__ mask, const uint8_t *__restrict__ solid, int nx,
                             int ny, int nxp, int ny_cl, int ny_gdl, int mode, int periodic,
                             int closed, int x0, int nxg) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= nxp || y >= ny) return;
  const long long c = (long long)y * nxp + x;
  const long long plane = (long long)nxp * ny;
  if (x >= nx) {
    mask[c] = REG_SOLID;   // padding and ghost columns: never updated
    mask[plane + c] = 0;
    return;
  }
  const int gx = x0 + x;
  auto is_solid = [&](int xx, int yy) { return solid && solid[(long long)yy * nxg + xx]; };
  uint8_t reg;
  if (is_solid(gx, y)) reg = REG_SOLID;
  else if (mode == 1 && y < ny_cl) reg = REG_CATALYST;
  else if (y < ny_cl + ny_gdl) reg = REG_POROUS;
  else reg = REG_CLEAR;
  uint8_t m = reg;
  if (gx == 0) m |= M_XLO;
  if (gx == nxg - 1) m |= M_XHI;
  if (y == ny - 1) m |= M_YHI;
  if (y == 0) m |= M_YLO;
  if (reg == REG_CLEAR && gx == 0 && !periodic && !closed) m |= M_INLET;
  // second plane: bit i - 1 set when the source x - e_i of flow link i
  // (i = 1..8, Eq. 2 order) is a solid cell inside the lattice
  uint8_t nb = 0;
  if (reg != REG_SOLID && solid) {
    const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    for (int i = 1; i < 9; ++i) {
      int sx = gx - ex[i];
      const int sy = y - ey[i];
      if (sy < 0 || sy >= ny) continue;
      if (periodic) sx = (sx + nxg) % nxg;
      if (sx < 0 || sx >= nxg) continue;
      if (is_solid(sx, sy)) nb |= (uint8_t)(1u << (i - 1));
    }
    if (nb) m |= M_NEAR_SOLID;
  }
  mask[c] = m;
  mask[plane + c] = nb;
}

// Ghost columns of x-slabs.  Six populations cross a slab side: those
// moving +x (f1, f5, f8 and the D2Q5 link-1 planes of T, O2, H2O) leave
// through the high side into the right neighbour's low ghost column, those
// moving -x (f3, f6, f7 and the link-3 planes) through the low side into
// the left neighbour's high ghost column.  Population q's ghost of row y is
// cell y nxp - 1 (low side) or cell y nxp + nx (high side), inside the row
// padding; row 0's low ghost is cell -1, which pop_index places in the last
// padding cell of the plane (or group plane) stored before.
// One copy moves one direction's six planes for every row: from column col
// of a lattice buffer (or a packed [6][ny] array) to offset off of a lattice
// buffer (or a packed array).
template <typename S>
__global__ void k_halo_copy(const S *__restrict__ src, long long src_plane, int src_nxp,
                            long long src_off, int src_packed, S *__restrict__ dst,
                            long long dst_plane, int dst_nxp, long long dst_off, int dst_packed,
                            int ny, int plus) {
  const int y = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
  if (y >= ny || k >= 6) return;
  const int mv_plus[6] = {1, 5, 8, 10, 15, 20}, mv_minus[6] = {3, 6, 7, 12, 17, 22};
  const long long q = plus ? mv_plus[k] : mv_minus[k];
  const long long si = src_packed ? (long long)k * ny + y
                                  : pop_index(q, (long long)y * src_nxp + src_off, src_plane);
  const long long di = dst_packed ? (long long)k * ny + y
                                  : pop_index(q, (long long)y * dst_nxp + dst_off, dst_plane);
  dst[di] = src[si];
}

__global__ void k_seed_advance(unsigned *ctr) { *ctr += 1u; }

void launch_seed_advance(unsigned *ctr, cudaStream_t st) { k_seed_advance<<<1, 1, 0, st>>>(ctr); }

void launch_build_mask(uint8_t *mask, const uint8_t *solid, int nx, int ny, int nxp, int ny_cl,
                       int ny_gdl, int mode, int periodic, int closed, int x0, int nxg,
                       cudaStream_t st) {
  dim3 grid((nxp + 127) / 128, ny);
  k_build_mask<<<grid, 128, 0, st>>>(mask, solid, nx, ny, nxp, ny_cl, ny_gdl, mode, periodic,
                                     closed, x0, nxg);
}

void launch_halo_copy(const HaloSide &src, const HaloSide &dst, int ny, int plus, int esize,
                      cudaStream_t st) {
  dim3 grid((ny + 127) / 128, 6);
#define PEMLBM_HALO(T)                                                                         \
  k_halo_copy<T><<<grid, 128, 0, st>>>((const T *)src.p, src.plane, src.nxp, src.off,          \
                                       src.packed, (T *)dst.p, dst.plane, dst.nxp, dst.off,   \
                                       dst.packed, ny, plus)
  if (esize == 8) PEMLBM_HALO(double);
  else if (esize == 4) PEMLBM_HALO(float);
  else PEMLBM_HALO(uint16_t);
#undef PEMLBM_HALO
}

// Per-material coefficients: Darcy and Forchheimer terms of Eq. 7, the l0,
// l1 of Eq. 8 (dt = 1), and per scalar the b of Eq. 10 with the flux-moment
// rate.  As printed, b = 20 sqrt(3) alpha - 4 with the fixed rate
// 6/(3 + sqrt 3); in the Fickian mode b is that of the scalar's largest
// diffusivity and alpha = c_s^2 (1/q1 - 1/2) sets q1, c_s^2 = (4 + b)/10.
template <typename R>
__global__ void k_prep_palette(MatCoef<R> *__restrict__ pal, const MatRaw *__restrict__ raw,
                               int npal, double nu, int forchheimer, ScalarMode mode) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npal) return;
  const MatRaw r = raw[k];
  MatCoef<R> c;
  const double phi = r.phi;
  double darcy = 0.0, forch = 0.0;
  if (!isinf(r.K)) {
    darcy = phi * nu / r.K;
    if (forchheimer) forch = phi * (0.143 * pow(phi, -1.5)) / sqrt(r.K);
  }
  c.phi = R(phi);
  c.inv_phi = R(1.0 / phi);
  c.darcy = R(darcy);
  c.forch = R(forch);
  c.l0 = R(0.5 + 0.25 * darcy);
  c.l1 = R(0.5 * forch);
  const double sqrt3 = sqrt(3.0);
  for (int s = 0; s < 3; ++s) {
    double b, q1;
    if (mode.fickian) {
      b = 20.0 * sqrt3 * mode.alpha_max[s] - 4.0;
      q1 = 1.0 / (r.alpha[s] * 10.0 / (4.0 + b) + 0.5);
    } else {
      b = 20.0 * sqrt3 * r.alpha[s] - 4.0;
      q1 = 6.0 / (3.0 + sqrt3);
    }
    c.b[s] = R(b);
    c.w1[s] = R((4.0 + b) / 20.0);
    c.q1[s] = R(q1);
  }
  c.inv_sigma = R(1.0 / r.sigma);
  pal[k] = c;
}

void launch_prep_palette(void *pal, const MatRaw *raw, int npal, double nu, int forchheimer,
                         const ScalarMode &mode, bool fp64, cudaStream_t st) {
  const int nb = (npal + 127) / 128;
  if (fp64)
    k_prep_palette<double><<<nb, 128, 0, st>>>((MatCoef<double> *)pal, raw, npal, nu, forchheimer,
                                                mode);
  else
    k_prep_palette<float><<<nb, 128, 0, st>>>((MatCoef<float> *)pal, raw, npal, nu, forchheimer,
                                               mode);
}

// Block k sums quantity k over the nblocks partials (rows of 10): each
// thread adds its blocks in increasing order, then a fixed-order block sum.
__global__ void __launch_bounds__(kReduceThreads)
k_sum_partials(const double *__restrict__ partial, int nblocks, double *__restrict__ out) {
  __shared__ double sm[32];
  const int k = blockIdx.x;
  double acc[1] = {0.0};
#pragma unroll 4
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) acc[0] += partial[(long long)b * 10 + k];
  block_sum<1>(acc, sm);
  if (threadIdx.x == 0) out[k] = acc[0];
}

__global__ void __launch_bounds__(kReduceThreads)
k_sum_columns(const double *__restrict__ colsum, int nx, double *__restrict__ out) {
  __shared__ double sm[2 * 32];
  double acc[2] = {0.0, 0.0};
  for (int x = threadIdx.x; x < nx; x += blockDim.x) {
    acc[0] += colsum[x];
    acc[1] += colsum[nx + x];
  }
  block_sum<2>(acc, sm);
  if (threadIdx.x == 0) {
    out[0] = acc[0];
    out[1] = acc[1];
  }
}

}  // namespace pemlbm
