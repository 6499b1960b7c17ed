// Host-visible declarations of the kernel launchers (implemented per storage
// type in kernels_*.cu and shared helpers in kernels_common.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pemlbm {

template <typename F> struct KArgsT;
using KArgs = KArgsT<double>;
struct MatRaw;
struct ScalarMode;

// Launch shapes of the coupled step: BX consecutive cells along x per row,
// BY rows per block, and the minimum resident blocks per SM asked of the
// register allocator.  lbm_tune times them and keeps the fastest.
struct StepShape { int bx, by, minb; };
constexpr int kStepVariants = 8;
constexpr StepShape kStepShapes[kStepVariants] = {
    {128, 2, 1}, {128, 2, 3}, {128, 2, 4}, {64, 4, 4},
    {256, 1, 4}, {32, 8, 4}, {128, 1, 8}, {64, 2, 8}};
constexpr int kReduceThreads = 512;
// Persistent batched step: 128 x 1 cells per block, 8 blocks per SM asked of
// the register allocator; the grid is the number of co-resident blocks.
constexpr int kPersistBX = 128, kPersistBY = 1, kPersistMinB = 8;
// A batched tile is BX x (BY * kBatchRows) cells: each thread updates
// kBatchRows cells, so the case lookup and argument staging are amortised.
constexpr int kBatchRows = 8;
constexpr int kResidualBX = 128, kResidualBY = 2;      // residual blocks
constexpr int kCatalystBX = 32, kCatalystBY = 8;       // catalyst reduction blocks

// One case of a batched step: its arguments, buffers and geometry.
template <typename F> struct BatchCaseT;
using BatchCase = BatchCaseT<double>;
template <typename F> struct KArgsT;

// Device-resident geometry shared by all kernels of a domain.
struct DevGeom {
  const uint8_t *mask;   // [ny][nxp] node bits, then [ny][nxp] solid-neighbour bits
  const uint16_t *mid;   // [ny][nxp] palette index
  const void *pal;       // MatCoef<R>[npal]
};

template <typename S> void launch_step(const void *src, void *dst, const DevGeom &g, const KArgs &a, int variant, cudaStream_t st);
// Reverse records of one step (device pointers, the arithmetic type of the
// domain; layout as RecPtrs in lbm_core.cuh).
struct RecBufs {
  void *cell, *own, *pulled;
  const int *slot;
};
// One step src -> dst that also writes its reverse records.
template <typename S> void launch_step_rec(const void *src, void *dst, const DevGeom &g, const KArgs &a, const RecBufs &r, cudaStream_t st);
template <typename S> void launch_fields(const void *src, const DevGeom &g, const KArgs &a, double *out, cudaStream_t st);
template <typename S> void launch_balances(const void *src, const DevGeom &g, const KArgs &a, double *out, cudaStream_t st);
template <typename S> void launch_catalyst(const void *src, const DevGeom &g, const KArgs &a, double i_scale, float *profile, double *colsum, double *out, cudaStream_t st);
// Residual of state src against snap_in, writing the new snapshot to snap_out
// (the same buffer for an in-place update).
template <typename S> void launch_residual(const void *src, const DevGeom &g, const KArgs &a, const void *snap_in, void *snap_out, double *partial, int *bad, double *out, cudaStream_t st);
// Blocks of the residual kernel (= rows of its partial-sum buffer).
inline int residual_blocks(int nx, int ny) {
  return ((nx + kResidualBX - 1) / kResidualBX) * ((ny + kResidualBY - 1) / kResidualBY);
}
template <typename S> void launch_init(void *pop, const DevGeom &g, const KArgs &a, cudaStream_t st);
template <typename S> void launch_get_state(const void *pop, const DevGeom &g, const KArgs &a, double *out, cudaStream_t st);
template <typename S> void launch_set_state(void *pop, const DevGeom &g, const KArgs &a, const double *in, cudaStream_t st);

template <typename S> void batch_upload(const BatchCase *host, int n, void *staging, void *dev, cudaStream_t st);
template <typename S> void launch_batch_step(const BatchCase *cases, const int *tile_start, int ncases, int total_tiles, int variant, int parity, cudaStream_t st);
template <typename S> cudaError_t launch_batch_persistent(const BatchCase *cases, const int *tile_start, int ncases, int total_tiles, int nsteps, unsigned *bar, int *status, long long spin_limit, cudaStream_t st);

// Buffers of one reverse step (types follow the domain's arithmetic).
struct AdjPtrs {
  const void *lam;
  void *O, *V;               // own-use / outlet adjoints written by this step
  const void *O_in, *V_in;   // those of the previous step
  void *gphi, *gK, *gD;      // segment gradients (arithmetic type)
  double *gU;
  void *lam_out;
  double *tphi, *tK, *tD;    // FP64 totals
  const long long *cells;    // fluid edge cells, then volumetric catalyst cells
  const uint32_t *pushed;    // per edge cell: links that have a fluid consumer
  int n_edge, n_own;         // edge cells; all own-use cells
};
template <typename S> void launch_adj_step(const RecBufs &r, const DevGeom &g, const KArgs &a, int fickian, const AdjPtrs &b, long long seed_cell, int lam_complete, cudaStream_t st, cudaStream_t side, cudaEvent_t fork, cudaEvent_t join);
template <typename S> void launch_adj_finish(const DevGeom &g, const KArgs &a, const AdjPtrs &b, cudaStream_t st);
template <typename S> void launch_adj_fold(const DevGeom &g, const KArgs &a, const AdjPtrs &b, cudaStream_t st);
template <typename S> void launch_adj_seed_current(const void *src, const DevGeom &g, const KArgs &a, int fickian, double weight, const AdjPtrs &b, cudaStream_t st);

// The first out-of-range access that this storage type's kernels recorded
// (the bounds-checked build; site << 48 | index, 0 for none, and always 0 in
// the plain build), cleared when read.
template <typename S> unsigned long long bounds_first_bad();

// Advances the step counter that seeds stochastic 16-bit rounding.
void launch_seed_advance(unsigned *ctr, cudaStream_t st);

// Material palette built on the device from per-cell fields in device
// memory ([ny][nx] doubles; sigma may be NULL = 1): the distinct tuples in
// row-major order of first occurrence into raw (at most max_pal), and every
// fluid cell's entry into mid ([ny][nxp]; other cells 0).  The outcome is
// left in *st (device memory): flags (kPal*), the smallest invalid cell
// (row-major index) and the palette size.  scratch: palette_scratch_bytes.
struct PalFields { const double *phi, *K, *aT, *DO2, *DH2O, *sigma; };
struct PalStatus { int flags, bad_cell, claimed, npal; };
enum { kPalInvalid = 1, kPalTooMany = 2, kPalCollision = 4 };
constexpr int kPalTable = 1 << 18;   // hash slots: 4 x the largest palette
size_t palette_scratch_bytes(int nx, int ny);
cudaError_t launch_device_palette(const PalFields &f, const uint8_t *mask, int nx, int ny, int nxp,
                                  uint16_t *mid, MatRaw *raw, int max_pal, void *scratch,
                                  PalStatus *st, cudaStream_t s);

// Node mask from the geometry (solid may be NULL): the domain is the x-slab
// [x0, x0 + nx) of a lattice nxg wide, solid is [ny][nxg].
void launch_build_mask(uint8_t *mask, const uint8_t *solid, int nx, int ny, int nxp, int ny_cl,
                       int ny_gdl, int mode, int periodic, int closed, int x0, int nxg,
                       cudaStream_t st);
// One end of a halo copy: a lattice buffer (plane stride, row pitch, offset
// of the column within a row: nx - 1 or 0 to read an edge column, -1 or nx
// to write a ghost column) or a packed [6][ny] array (packed = 1).
struct HaloSide { void *p; long long plane; int nxp; long long off; int packed; };
// Copies the six populations that move +x (plus = 1) or -x (plus = 0) across
// a slab side, for every row; element size esize (2, 4, 8).
void launch_halo_copy(const HaloSide &src, const HaloSide &dst, int ny, int plus, int esize,
                      cudaStream_t st);
// Derived material coefficients of a palette (Eq. 7, 8, 10): R = double if
// fp64 else float.
void launch_prep_palette(void *pal, const MatRaw *raw, int npal, double nu, int forchheimer,
                         const ScalarMode &mode, bool fp64, cudaStream_t st);

}  // namespace pemlbm
