// Host-visible declarations of the kernel launchers (implemented per storage
// type in kernels_*.cu and shared helpers in kernels_common.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pemlbm {

struct KArgs;
struct MatRaw;

// Launch shape of the coupled step: kStepBX consecutive cells along x per
// row, kStepBY rows per block.
constexpr int kStepBX = 128;
constexpr int kStepBY = 2;
constexpr int kStepThreads = kStepBX * kStepBY;
constexpr int kReduceThreads = 512;

// Device-resident geometry shared by all kernels of a domain.
struct DevGeom {
  const uint8_t *mask;   // [ny][nxp] node bits
  const uint16_t *mid;   // [ny][nxp] palette index
  const void *pal;       // MatCoef<R>[npal]
};

template <typename S> void launch_step(const void *src, void *dst, const DevGeom &g, const KArgs &a, cudaStream_t st);
template <typename S> void launch_fields(const void *src, const DevGeom &g, const KArgs &a, double *out, cudaStream_t st);
template <typename S> void launch_catalyst(const void *src, const DevGeom &g, const KArgs &a, double i_scale, float *profile, double *out, cudaStream_t st);
template <typename S> void launch_residual(const void *src, const DevGeom &g, const KArgs &a, double *snap, double *partial, int nblocks, int *bad, double *out, cudaStream_t st);
template <typename S> void launch_init(void *pop, const DevGeom &g, const KArgs &a, cudaStream_t st);
template <typename S> void launch_get_state(const void *pop, const DevGeom &g, const KArgs &a, double *out, cudaStream_t st);
template <typename S> void launch_set_state(void *pop, const DevGeom &g, const KArgs &a, const double *in, cudaStream_t st);

// Node mask from the geometry (solid may be NULL).
void launch_build_mask(uint8_t *mask, const uint8_t *solid, int nx, int ny, int nxp, int ny_cl,
                       int ny_gdl, int mode, int periodic, cudaStream_t st);
// Derived material coefficients of a palette (Eq. 7, 8, 10): R = double if
// fp64 else float.
void launch_prep_palette(void *pal, const MatRaw *raw, int npal, double nu, int forchheimer,
                         bool fp64, cudaStream_t st);

}  // namespace pemlbm
