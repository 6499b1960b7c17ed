// Material palette built on the device from per-cell fields that are
// already in device memory (lbm_set_fields with on_device = 1).
//
// The palette holds the distinct material tuples (phi, K, alpha_T, D_O2,
// D_H2O, rho_cp_ratio) of the fluid cells in order of first occurrence in
// row-major order, and every fluid cell's index into it: the same palette,
// entry for entry, as the host build of the same fields.  Steps:
//   1. insert: every fluid cell validates its tuple and hashes it into an
//      open-addressing table (64-bit keys claimed with atomicCAS, linear
//      probing; the lanes of a warp with one tuple insert it once), and each
//      slot records the smallest cell index of its tuple;
//   2. count / scan: the cells that are their slot's smallest index are the
//      first occurrences; a block count, one scan over the blocks and a
//      rank within the block number them in row-major order;
//   3. assign: first occurrences write their tuple to the palette and their
//      number to their slot; every cell then reads its slot's number and
//      compares its tuple with the palette entry (a 64-bit hash collision
//      between two different tuples is reported, never merged).
// Probing stops once more slots are claimed than the palette may hold, so
// the table (4 x the largest palette) never fills.
#include "lbm_kernels.cuh"

namespace pemlbm {

namespace {

constexpr int kPalThreads = 256;

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

struct Tuple { double v[6]; };

__device__ __forceinline__ Tuple load_tuple(const PalFields &f, long long o) {
  Tuple t;
  t.v[0] = f.phi[o];
  t.v[1] = f.K[o];
  t.v[2] = f.aT[o];
  t.v[3] = f.DO2[o];
  t.v[4] = f.DH2O[o];
  t.v[5] = f.sigma ? f.sigma[o] : 1.0;
  return t;
}

// Validity of a tuple: the ranges lbm_set_fields accepts.
__device__ __forceinline__ bool valid_tuple(const Tuple &t) {
  const double amax = 5.0 / (20.0 * 1.7320508075688772);
  bool ok = t.v[0] > 0.0 && t.v[0] <= 1.0 && t.v[1] > 0.0 && t.v[5] >= 1e-6 && !isinf(t.v[5]);
  for (int s = 2; s < 5; ++s) ok = ok && t.v[s] > 0.0 && t.v[s] <= amax;
  return ok;
}

__device__ __forceinline__ unsigned long long hash_tuple(const Tuple &t) {
  unsigned long long h = 0x9e3779b97f4a7c15ull;
  for (int k = 0; k < 6; ++k) h = mix64(h ^ (unsigned long long)__double_as_longlong(t.v[k]));
  return h ? h : 1ull;   // 0 marks an empty slot
}

__device__ __forceinline__ bool fluid(const uint8_t *mask, int nxp, int x, int y) {
  return (mask[(long long)y * nxp + x] & REG_MASK) != REG_SOLID;
}

__global__ void k_pal_clear(unsigned long long *keys, int *rep, int *slot_id, int ts, PalStatus *st) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ts) {
    keys[i] = 0ull;
    rep[i] = 0x7fffffff;
    slot_id[i] = -1;
  }
  if (i == 0) {
    st->flags = 0;
    st->bad_cell = 0x7fffffff;
    st->claimed = 0;
    st->npal = 0;
  }
}

// Lanes of a warp that hold the same tuple insert it once: the lowest of
// them (the smallest cell index, since cells follow the lanes) probes the
// table for the group and broadcasts the slot.  Every lane of the warp takes
// part (a launch of whole warps), those without a valid fluid cell with key 0.
__global__ void __launch_bounds__(kPalThreads)
k_pal_insert(PalFields f, const uint8_t *__restrict__ mask, int nx, int ny, int nxp,
             unsigned long long *keys, int *rep, int *cellslot, int ts, int max_pal,
             PalStatus *st) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long h = 0ull;   // 0: nothing to insert
  if (c < (long long)nx * ny) {
    const int x = (int)(c % nx), y = (int)(c / nx);
    if (fluid(mask, nxp, x, y)) {
      const Tuple t = load_tuple(f, c);
      if (valid_tuple(t)) {
        h = hash_tuple(t);
      } else {
        atomicOr(&st->flags, kPalInvalid);
        atomicMin(&st->bad_cell, (int)c);
      }
    }
  }
  const unsigned peers = __match_any_sync(0xffffffffu, h);
  const int leader = __ffs(peers) - 1;
  int slot = -1;
  if (h != 0ull && (int)(threadIdx.x & 31) == leader) {
    if (*((volatile int *)&st->claimed) > max_pal) {        // too many materials already
      atomicOr(&st->flags, kPalTooMany);
    } else {
      unsigned s = (unsigned)(h & (unsigned long long)(ts - 1));
      for (int probe = 0; probe < ts; ++probe) {
        const unsigned long long old = atomicCAS(&keys[s], 0ull, h);
        if (old == h) {
          slot = (int)s;
          break;
        }
        if (old == 0ull) {
          if (atomicAdd(&st->claimed, 1) >= max_pal) atomicOr(&st->flags, kPalTooMany);
          slot = (int)s;
          break;
        }
        if (*((volatile int *)&st->claimed) > max_pal) {    // too many materials: stop probing
          atomicOr(&st->flags, kPalTooMany);
          break;
        }
        s = (s + 1) & (unsigned)(ts - 1);
      }
      if (slot >= 0) atomicMin(&rep[slot], (int)c);
    }
  }
  slot = __shfl_sync(0xffffffffu, slot, leader);
  if (h != 0ull && slot >= 0) cellslot[c] = slot;
}

// Whether cell c is its tuple's first occurrence (valid, fluid cells only).
__device__ __forceinline__ bool first_occurrence(const uint8_t *mask, int nx, int nxp, long long c,
                                                 long long n, const int *cellslot, const int *rep) {
  if (c >= n) return false;
  const int x = (int)(c % nx), y = (int)(c / nx);
  if (!fluid(mask, nxp, x, y)) return false;
  return rep[cellslot[c]] == (int)c;
}

__device__ __forceinline__ int block_rank(bool flag, int *warp_tot, int &block_total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned b = __ballot_sync(0xffffffffu, flag);
  const int in_warp = __popc(b & ((1u << lane) - 1u));
  if (lane == 0) warp_tot[warp] = __popc(b);
  __syncthreads();
  int before = 0;
  block_total = 0;
  for (int w = 0; w < nw; ++w) {
    if (w < warp) before += warp_tot[w];
    block_total += warp_tot[w];
  }
  return before + in_warp;
}

__global__ void __launch_bounds__(kPalThreads)
k_pal_count(const uint8_t *__restrict__ mask, int nx, int ny, int nxp, const int *cellslot,
            const int *rep, int *block_cnt) {
  __shared__ int warp_tot[kPalThreads / 32];
  const long long n = (long long)nx * ny;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int total;
  block_rank(first_occurrence(mask, nx, nxp, c, n, cellslot, rep), warp_tot, total);
  if (threadIdx.x == 0) block_cnt[blockIdx.x] = total;
}

// Exclusive scan of the block counts in one block; the total is the palette size.
__global__ void k_pal_scan(int *block_cnt, int nblocks, PalStatus *st) {
  __shared__ int carry;
  __shared__ int warp_tot[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nblocks; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = i < nblocks ? block_cnt[i] : 0;
    // inclusive scan within the warp, then across warps
    int s = v;
    for (int off = 1; off < 32; off <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, s, off);
      if ((threadIdx.x & 31) >= off) s += u;
    }
    if ((threadIdx.x & 31) == 31) warp_tot[threadIdx.x >> 5] = s;
    __syncthreads();
    int before = 0, chunk = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      if (w < (int)(threadIdx.x >> 5)) before += warp_tot[w];
      chunk += warp_tot[w];
    }
    if (i < nblocks) block_cnt[i] = carry + before + s - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += chunk;
    __syncthreads();
  }
  if (threadIdx.x == 0) st->npal = carry;
}

__global__ void __launch_bounds__(kPalThreads)
k_pal_assign(PalFields f, const uint8_t *__restrict__ mask, int nx, int ny, int nxp,
             const int *cellslot, const int *rep, const int *block_off, int *slot_id,
             MatRaw *raw, int max_pal) {
  __shared__ int warp_tot[kPalThreads / 32];
  const long long n = (long long)nx * ny;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool first = first_occurrence(mask, nx, nxp, c, n, cellslot, rep);
  int total;
  const int r = block_rank(first, warp_tot, total);
  if (!first) return;
  const int id = block_off[blockIdx.x] + r;
  slot_id[cellslot[c]] = id;
  if (id >= 0 && id < max_pal) {
    const Tuple t = load_tuple(f, c);
    MatRaw m;
    m.phi = t.v[0];
    m.K = t.v[1];
    m.alpha[0] = t.v[2];
    m.alpha[1] = t.v[3];
    m.alpha[2] = t.v[4];
    m.sigma = t.v[5];
    raw[id] = m;
  }
}

__global__ void __launch_bounds__(kPalThreads)
k_pal_index(PalFields f, const uint8_t *__restrict__ mask, int nx, int ny, int nxp,
            const int *cellslot, const int *slot_id, const MatRaw *raw, uint16_t *mid,
            int max_pal, PalStatus *st) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= (long long)nx * ny) return;
  const int x = (int)(c % nx), y = (int)(c / nx);
  if (!fluid(mask, nxp, x, y)) return;
  const int id = slot_id[cellslot[c]];
  if (id < 0 || id >= max_pal) {      // a cell left out by an invalid or oversized set
    atomicOr(&st->flags, kPalTooMany);
    return;
  }
  mid[(long long)y * nxp + x] = (uint16_t)id;
  const Tuple t = load_tuple(f, c);
  const MatRaw m = raw[id];
  if (!(m.phi == t.v[0] && m.K == t.v[1] && m.alpha[0] == t.v[2] && m.alpha[1] == t.v[3] &&
        m.alpha[2] == t.v[4] && m.sigma == t.v[5]))
    atomicOr(&st->flags, kPalCollision);
}

}  // namespace

// Scratch layout: hash keys, smallest cell per slot, palette number per
// slot (kPalTable each), the slot of every cell, the block counts.
size_t palette_scratch_bytes(int nx, int ny) {
  const long long n = (long long)nx * ny;
  const long long nb = (n + kPalThreads - 1) / kPalThreads;
  return (size_t)kPalTable * (8 + 4 + 4) + (size_t)n * 4 + (size_t)nb * 4;
}

cudaError_t launch_device_palette(const PalFields &f, const uint8_t *mask, int nx, int ny, int nxp,
                                  uint16_t *mid, MatRaw *raw, int max_pal, void *scratch,
                                  PalStatus *st, cudaStream_t s) {
  const long long n = (long long)nx * ny;
  const int nb = (int)((n + kPalThreads - 1) / kPalThreads);
  char *p = (char *)scratch;
  auto *keys = (unsigned long long *)p;
  p += (size_t)kPalTable * 8;
  int *rep = (int *)p;
  p += (size_t)kPalTable * 4;
  int *slot_id = (int *)p;
  p += (size_t)kPalTable * 4;
  int *cellslot = (int *)p;
  p += (size_t)n * 4;
  int *block_cnt = (int *)p;
  cudaError_t e = cudaMemsetAsync(mid, 0, sizeof(uint16_t) * (size_t)nxp * ny, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cellslot, 0, sizeof(int) * (size_t)n, s);
  if (e != cudaSuccess) return e;
  k_pal_clear<<<(kPalTable + 255) / 256, 256, 0, s>>>(keys, rep, slot_id, kPalTable, st);
  k_pal_insert<<<nb, kPalThreads, 0, s>>>(f, mask, nx, ny, nxp, keys, rep, cellslot, kPalTable,
                                          max_pal, st);
  k_pal_count<<<nb, kPalThreads, 0, s>>>(mask, nx, ny, nxp, cellslot, rep, block_cnt);
  k_pal_scan<<<1, 1024, 0, s>>>(block_cnt, nb, st);
  k_pal_assign<<<nb, kPalThreads, 0, s>>>(f, mask, nx, ny, nxp, cellslot, rep, block_cnt, slot_id,
                                          raw, max_pal);
  k_pal_index<<<nb, kPalThreads, 0, s>>>(f, mask, nx, ny, nxp, cellslot, slot_id, raw, mid,
                                         max_pal, st);
  return cudaGetLastError();
}

}  // namespace pemlbm
