// Device core of the coupled cathode lattice-Boltzmann step (sm_103a).
//
// One thread updates one cell: it pulls the 24 populations that stream into
// the cell (9 D2Q9 flow + 3 x 5 D2Q5 scalar populations, Eq. 1 and 10 left-
// hand sides), applies the boundary links of Sec. 4 where the source lies
// outside the fluid, forms the macroscopic values (Eq. 8, 11), relaxes in
// moment space (Eq. 1, 3-7 for the flow; Eq. 10 for T, O2, H2O), adds the
// catalyst sources (Eq. 12-17) and writes the 24 post-collision values to
// the other buffer.
//
// Storage: a buffer of 24 planes' worth of values, each plane ny rows x nxp
// (padded) columns, x fastest.  Links 0-4 of the flow (Eq. 2) and of the
// three scalars (Eq. 9) point the same way, so the four values of link i of a
// cell (f_i, g_T,i, g_O2,i, g_H2O,i) are kept side by side: five planes of
// 4-value groups, then the diagonal flow links 5-8 as plain planes
// (pop_index).  An interior pull of links 0-4 is then one vector load from
// the source cell, and the store of the cell's links 0-4 one vector store.
// Every value is a DEVIATION from a fixed per-direction reference:
// f_i - w_i rho0 for the flow and g_i - wref_{s,i} Cref_s for scalar s,
// where wref are the D2Q5 equilibrium weights of one reference b per scalar.
// The references do not depend on the cell, so a pull never needs the
// source cell's material, and all arithmetic runs on small numbers (the
// collision is written directly in deviation moments).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pemlbm {

// ------------------------------------------------------------ bounds checks
// A build with -DPEMLBM_BOUNDS_CHECK (the checked library of build.py) tests
// the index of every population, mask, material-index and palette access of
// the step's device code, and of the adjoint's lambda accesses, against the
// extent of its buffer.  An access outside it is skipped (a load gives 0, a
// mask load a solid cell) and the first one of each translation unit is
// recorded as site << 48 | (index & (2^48 - 1)) for lbm_bounds_check.
// Nothing traps.  Without the flag every check is the constant true.
#ifdef PEMLBM_BOUNDS_CHECK
static __device__ unsigned long long g_bounds_first_bad = 0;
__device__ __forceinline__ bool in_bounds(long long i, long long n, unsigned site) {
  if (i >= 0 && i < n) return true;
  atomicCAS(&g_bounds_first_bad, 0ull,
            ((unsigned long long)site << 48) | ((unsigned long long)i & 0xffffffffffffull));
  return false;
}
#else
__device__ __forceinline__ constexpr bool in_bounds(long long, long long, unsigned) { return true; }
#endif
// Elements of a population buffer: 24 planes and the guard that keeps the
// unconditional pulls of the top row inside the allocation.
__host__ __device__ __forceinline__ constexpr long long pop_extent(long long plane, int nxp) {
  return 24 * plane + nxp + 64;
}

// Element offset of population q (0-8 flow, 9 + 5 s + i link i of scalar s)
// of cell c in a buffer whose planes hold P cells each.
__host__ __device__ __forceinline__ constexpr long long pop_index(int q, long long c, long long P) {
  return q < 5 ? 4 * (q * P + c)
       : q < 9 ? (15 + q) * P + c
               : 4 * (((q - 9) % 5) * P + c) + 1 + (q - 9) / 5;
}

// ------------------------------------------------------------------ mask
enum : uint8_t {
  REG_MASK = 3, REG_CLEAR = 0, REG_POROUS = 1, REG_CATALYST = 2, REG_SOLID = 3,
  M_XLO = 1 << 2, M_XHI = 1 << 3, M_YHI = 1 << 4, M_YLO = 1 << 5,
  M_INLET = 1 << 6, M_NEAR_SOLID = 1 << 7,
  M_EDGE = M_XLO | M_XHI | M_YHI | M_YLO | M_NEAR_SOLID
};

// --------------------------------------------------------------- storage
template <typename S> struct Real { using type = float; };
template <> struct Real<double> { using type = double; };

__device__ __forceinline__ float ld_r(const float *p) { return __ldg(p); }
__device__ __forceinline__ double ld_r(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ld_r(const __nv_bfloat16 *p) {
  return __uint_as_float((unsigned)__ldg(reinterpret_cast<const unsigned short *>(p)) << 16);
}
__device__ __forceinline__ float ld_r(const __half *p) {
  return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short *>(p))));
}

// Loads that bypass L1 (L2 only).  Within one launch L1 is not coherent
// across SMs, so a kernel that reads, across a grid barrier, what other SMs
// wrote must use these.
__device__ __forceinline__ float ld_cg(const float *p) { return __ldcg(p); }
__device__ __forceinline__ double ld_cg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg(const __nv_bfloat16 *p) {
  const unsigned short b = __ldcg(reinterpret_cast<const unsigned short *>(p));
  return __bfloat162float(__ushort_as_bfloat16(b));
}
__device__ __forceinline__ float ld_cg(const __half *p) {
  const unsigned short b = __ldcg(reinterpret_cast<const unsigned short *>(p));
  return __half2float(__ushort_as_half(b));
}
template <bool CG, typename S> __device__ __forceinline__ auto ldp(const S *p) {
  if constexpr (CG) return ld_cg(p);
  else return ld_r(p);
}

// Stochastic rounding of a step's 16-bit stores: unbiased, E[stored] = v,
// so increments far below half an ulp of a stored value still accumulate.
// r16 holds 16 uniform random bits.  Both formats add a uniform fraction of
// the 16-bit spacing to the magnitude and round toward zero, which rounds
// the magnitude up with probability equal to the dropped fraction.  BF16
// keeps the top 16 bits of the FP32 pattern, so the fraction is added to
// the 16 bits below them.  FP16's spacing at |v| is 2^(E - 10) for an FP32
// exponent E of a normal FP16 value and 2^-24 below 2^-14; the FP32 sum
// v + sign(v) u spacing rounds at 2^-13 of that spacing or finer, a bias
// below 1e-4 of one rounding step.
// sr_bits returns the 16-bit pattern; the pointer only selects the format.
__device__ __forceinline__ unsigned short sr_bits(const __nv_bfloat16 *, float v, unsigned r16) {
  return (unsigned short)((__float_as_uint(v) + r16) >> 16);
}
__device__ __forceinline__ unsigned short sr_bits(const __half *, float v, unsigned r16) {
  const unsigned e = __float_as_uint(v) & 0x7f800000u;
  const float spacing = __uint_as_float(max(e, 113u << 23) - (10u << 23));
  const float a = fmaf(copysignf(spacing, v), (float)r16 * (1.0f / 65536.0f), v);
  return __half_as_ushort(__float2half_rz(a));
}
template <typename S> __device__ __forceinline__ void st_sr(S *p, float v, unsigned r16) {
  *reinterpret_cast<unsigned short *>(p) = sr_bits(p, v, r16);
}
// Random bits for cell c of a step: a 32-bit integer hash of (c, seed), and
// a xorshift stream from it for the cell's 24 stores.
__device__ __forceinline__ unsigned hash32(unsigned x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}
__device__ __forceinline__ unsigned xorshift32(unsigned &s) {
  s ^= s << 13;
  s ^= s >> 17;
  s ^= s << 5;
  return s;
}

// One group of four values (links i of the flow and of the three scalars).
template <typename R> struct Quad { R v[4]; };
template <bool CG>
__device__ __forceinline__ Quad<float> ldq(const float *p) {
  const float4 *q = reinterpret_cast<const float4 *>(p);
  const float4 t = CG ? __ldcg(q) : __ldg(q);
  return Quad<float>{{t.x, t.y, t.z, t.w}};
}
template <bool CG>
__device__ __forceinline__ Quad<double> ldq(const double *p) {
  const double2 *q = reinterpret_cast<const double2 *>(p);
  const double2 t0 = CG ? __ldcg(q) : __ldg(q), t1 = CG ? __ldcg(q + 1) : __ldg(q + 1);
  return Quad<double>{{t0.x, t0.y, t1.x, t1.y}};
}
// 16-bit groups: one 8-byte load, the first value in the low half of the
// first word; each conversion is exact (as __bfloat162float, __half2float)
template <bool CG>
__device__ __forceinline__ Quad<float> ldq(const __nv_bfloat16 *p) {
  const uint2 *q = reinterpret_cast<const uint2 *>(p);
  const uint2 t = CG ? __ldcg(q) : __ldg(q);
  return Quad<float>{{__uint_as_float(t.x << 16), __uint_as_float(t.x & 0xffff0000u),
                      __uint_as_float(t.y << 16), __uint_as_float(t.y & 0xffff0000u)}};
}
template <bool CG>
__device__ __forceinline__ Quad<float> ldq(const __half *p) {
  const uint2 *q = reinterpret_cast<const uint2 *>(p);
  const uint2 t = CG ? __ldcg(q) : __ldg(q);
  const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&t.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&t.y));
  return Quad<float>{{a.x, a.y, b.x, b.y}};
}

__device__ __forceinline__ void st_r(float *p, float v) { *p = v; }
__device__ __forceinline__ void st_r(double *p, double v) { *p = v; }
__device__ __forceinline__ void st_r(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void st_r(__half *p, float v) { *p = __float2half_rn(v); }

// Group stores (round to nearest even, as st_r).
__device__ __forceinline__ void stq(float *p, float a, float b, float c, float d) {
  *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void stq(double *p, double a, double b, double c, double d) {
  reinterpret_cast<double2 *>(p)[0] = make_double2(a, b);
  reinterpret_cast<double2 *>(p)[1] = make_double2(c, d);
}
__device__ __forceinline__ uint2 pack4(unsigned short a, unsigned short b, unsigned short c,
                                       unsigned short d) {
  return make_uint2((unsigned)a | ((unsigned)b << 16), (unsigned)c | ((unsigned)d << 16));
}
// (paired conversions: each half rounds as __float2bfloat16_rn / __float2half_rn)
__device__ __forceinline__ void stq(__nv_bfloat16 *p, float a, float b, float c, float d) {
  const __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
  *reinterpret_cast<uint2 *>(p) = make_uint2(*reinterpret_cast<const unsigned *>(&lo),
                                             *reinterpret_cast<const unsigned *>(&hi));
}
__device__ __forceinline__ void stq(__half *p, float a, float b, float c, float d) {
  const __half2 lo = __floats2half2_rn(a, b), hi = __floats2half2_rn(c, d);
  *reinterpret_cast<uint2 *>(p) = make_uint2(*reinterpret_cast<const unsigned *>(&lo),
                                             *reinterpret_cast<const unsigned *>(&hi));
}
// Group stores with stochastic rounding; ra..rd are the 16 random bits of
// each value.
template <typename S>
__device__ __forceinline__ void stq_sr(S *p, float a, float b, float c, float d, unsigned ra,
                                       unsigned rb, unsigned rc, unsigned rd) {
  *reinterpret_cast<uint2 *>(p) =
      pack4(sr_bits(p, a, ra), sr_bits(p, b, rb), sr_bits(p, c, rc), sr_bits(p, d, rd));
}

// Material coefficients of one palette entry, derived from (phi, K, alpha)
// by k_prep_palette: 16 values so an entry is 4 x 16-byte vectors in FP32.
template <typename R> struct alignas(16 * sizeof(R) >= 64 ? 64 : 16) MatCoef {
  R phi, inv_phi;   // porosity and 1/phi
  R darcy, forch;   // phi nu / K and phi F_phi / sqrt(K) of Eq. 7
  R l0, l1;         // Eq. 8
  R b[3];           // b of Eq. 10 for T, O2, H2O
  R w1[3];          // (4 + b)/20: D2Q5 equilibrium weight of the moving links
  R q1[3];          // relaxation rate of the D2Q5 flux moments
  R inv_sigma;      // (rho c_p)_f / (rho c_p)_eff: scales the reaction heat
};

// Raw material tuple as given by the caller (lattice units).
struct MatRaw { double phi, K, alpha[3], sigma; };

// How each scalar's diffusivity enters Eq. 10 (see lbm_params.interface_mode).
struct ScalarMode { int fickian; double alpha_max[3]; };

// Launch-invariant arguments (passed by value: constant bank).  The host
// fills them in FP64 (KArgs) and narrows them to the kernels' arithmetic
// type once per launch, so no kernel converts per cell.
template <typename F> struct KArgsT {
  int nx, ny, nxp, periodic;
  long long plane;          // elements per population plane
  int mode;                 // 0 thin film, 1 volumetric catalyst rows
  int ny_cl, y_ch0;         // catalyst rows; first channel row
  int top_dirichlet;
  F s_nu, s_q;              // 1/tau and the q-moment rate of Sec. 2.1
  F body_g;                 // body force per unit mass along x
  F u_in_avg, h_ch;         // inlet parabola
  int inlet_pressure;       // 1: pressure inlet (virtual column -1 at phi p = 1/3 + dp_in)
  F dp_in;
  F Q3;                     // Eq. 10 rate of the energy moments
  F Cref[3], wr0[3], wr1[3], bref[3];  // deviation references
  F adv_off[3];             // advected value of scalar s = deviation sum + adv_off[s]:
                            // Cref (u C, Eq. 10 as printed) or Cref - C_in (u (C - C_in))
  F Cin[3], Ctop[3];
  // kinetics: k(T) = A exp(e_in - c1 (T - T_in)/(T T_in)), Eq. 13, 14, 16, 17
  F kA_surf, kA_vol, k_ein, k_c1, T_in;
  // Butler-Volmer anodic branch, same form (all zero for Tafel kinetics)
  F kA_surf_a, kA_vol_a, k_ein_a, k_c1_a;
  F theta0;                 // Cref_T - T_in
  int stochastic;           // 16-bit step stores: 1 stochastic rounding, 0 nearest even
  const unsigned *seed_ctr; // device step counter seeding the stochastic rounding
  F hpo;                    // temperature per unit O2 consumed (Eq. 15, 16)
  // Boussinesq buoyancy: force per unit mass (gam_x, gam_y) (T - T_buoy),
  // with T - T_buoy = C_T + buoy_off (C_T the deviation sum of the T lattice)
  F gam_x, gam_y, buoy_off;
  int closed_x;             // 1: both x ends are no-slip walls
  int halo_lo, halo_hi;     // x-slab sides that border a neighbour slab: pulls across
                            // them read the ghost column (x = -1 or nx) the exchange fills
  int wall_dir;             // bit 3 k + s: scalar s fixed to Cwall[k][s] on wall k
  F Cwall[3][3];            // k: 0 the x = 0 end, 1 the x = nx - 1 end, 2 the bottom
  int npal;                 // palette entries (the bounds-checked build tests indices)
};
using KArgs = KArgsT<double>;

// Whether a set-up uses what only the X instantiations of the step carry.
template <typename F> __host__ __device__ inline bool needs_extended(const KArgsT<F> &a) {
  return a.closed_x || a.wall_dir || a.gam_x != F(0) || a.gam_y != F(0);
}

template <typename F> __host__ __device__ inline KArgsT<F> narrow_args(const KArgs &a) {
  KArgsT<F> r;
  r.nx = a.nx; r.ny = a.ny; r.nxp = a.nxp; r.periodic = a.periodic; r.plane = a.plane;
  r.mode = a.mode; r.ny_cl = a.ny_cl; r.y_ch0 = a.y_ch0; r.top_dirichlet = a.top_dirichlet;
  r.s_nu = F(a.s_nu); r.s_q = F(a.s_q); r.body_g = F(a.body_g); r.u_in_avg = F(a.u_in_avg);
  r.h_ch = F(a.h_ch); r.Q3 = F(a.Q3);
  r.inlet_pressure = a.inlet_pressure; r.dp_in = F(a.dp_in);
  r.gam_x = F(a.gam_x); r.gam_y = F(a.gam_y); r.buoy_off = F(a.buoy_off);
  r.closed_x = a.closed_x; r.wall_dir = a.wall_dir; r.npal = a.npal;
  r.halo_lo = a.halo_lo; r.halo_hi = a.halo_hi;
  for (int k = 0; k < 3; ++k)
    for (int s = 0; s < 3; ++s) r.Cwall[k][s] = F(a.Cwall[k][s]);
  for (int s = 0; s < 3; ++s) {
    r.Cref[s] = F(a.Cref[s]); r.wr0[s] = F(a.wr0[s]); r.wr1[s] = F(a.wr1[s]);
    r.bref[s] = F(a.bref[s]); r.Cin[s] = F(a.Cin[s]); r.Ctop[s] = F(a.Ctop[s]);
    r.adv_off[s] = F(a.adv_off[s]);
  }
  r.kA_surf = F(a.kA_surf); r.kA_vol = F(a.kA_vol); r.k_ein = F(a.k_ein); r.k_c1 = F(a.k_c1);
  r.T_in = F(a.T_in); r.theta0 = F(a.theta0); r.hpo = F(a.hpo);
  r.stochastic = a.stochastic; r.seed_ctr = a.seed_ctr;
  r.kA_surf_a = F(a.kA_surf_a); r.kA_vol_a = F(a.kA_vol_a);
  r.k_ein_a = F(a.k_ein_a); r.k_c1_a = F(a.k_c1_a);
  return r;
}

// Mask, material-index and palette loads of the step (checked in the
// bounds-checked build; the mask has two planes).
template <typename F>
__device__ __forceinline__ uint8_t ld_mask(const uint8_t *__restrict__ mask, long long i,
                                           const KArgsT<F> &a, unsigned site) {
#ifdef PEMLBM_BOUNDS_CHECK
  if (!in_bounds(i, 2 * a.plane, site)) return uint8_t(REG_SOLID);
#endif
  return mask[i];
}
template <typename F>
__device__ __forceinline__ uint16_t ld_mid(const uint16_t *__restrict__ mid, long long i,
                                           const KArgsT<F> &a, unsigned site) {
#ifdef PEMLBM_BOUNDS_CHECK
  if (!in_bounds(i, a.plane, site)) return uint16_t(0);
  const uint16_t k = mid[i];
  return in_bounds(k, a.npal, site + 1) ? k : uint16_t(0);
#else
  return mid[i];
#endif
}

// One case of a batched step (device table entry).
template <typename F> struct BatchCaseT {
  KArgsT<F> a;
  const void *pop[2];       // the case's two population buffers
  const uint8_t *mask;
  const uint16_t *mid;
  const void *pal;
  int cur0;                 // buffer holding the state when the batched run starts
  int tiles_x;              // tiles along x
};
using BatchCase = BatchCaseT<double>;

// Reverse records of one forward step: what the transpose of the step
// (the discrete adjoint) needs from the state the step started from, so
// that a reverse sweep reads these instead of stepping forward again.
//   cell[8 c + 0..7]: per cell, the Eq. 8 auxiliary velocity (vx, vy), the
//     three deviation sums of the post-stream scalars (T, O2, H2O) and the
//     O2 flux moments n1, n2 of Eq. 10 (after the surface reaction), then
//     one unused value: two 4-value groups;
//   own[4 s + 0..3]: per listed cell s (fluid cells with edge bits, then
//     catalyst cells of the volumetric mode): T - T_in and C_O2 of the
//     cell's own state (the reaction's arguments, Eq. 13-17) and the
//     momentum (jx, jy) of its own flow populations (what a virtual column
//     of the outlet or of the pressure inlet takes from it);
//   pulled[24 s + q]: per edge cell s, its 24 post-stream values before the
//     surface reaction (population order of pop_index);
//   slot[c]: the listed index of cell c, -1 for other cells.
template <typename R> struct RecPtrs {
  R *cell, *own, *pulled;
  const int *slot;
};

// Columns whose cells feed a virtual column: the outlet (x = nx - 1) and,
// with the pressure inlet, x = 0.
template <typename R>
__host__ __device__ __forceinline__ bool has_vcol(const KArgsT<R> &a, int x) {
  return !a.periodic && (x == a.nx - 1 || (x == 0 && a.inlet_pressure));
}

// Velocity sets, Eq. 2 and Eq. 9 orders (folded by the compiler once the
// loops over links are unrolled).
#define EX9_TAB {0, 1, 0, -1, 0, 1, -1, -1, 1}
#define EY9_TAB {0, 0, 1, 0, -1, 1, 1, -1, -1}
#define OP9_TAB {0, 3, 4, 1, 2, 7, 8, 5, 6}

template <typename R> __device__ __forceinline__ R w9(int i) {
  return i == 0 ? R(4.0 / 9.0) : (i < 5 ? R(1.0 / 9.0) : R(1.0 / 36.0));
}
// d f_i^eq / d(phi p) of the Eq. 5 equilibrium: 1/3 (axis), 1/12 (diagonal).
template <typename R> __device__ __forceinline__ R lam9(int i) {
  return i == 0 ? R(-5.0 / 3.0) : (i < 5 ? R(1.0 / 3.0) : R(1.0 / 12.0));
}

// Population planes of one buffer; CG selects L2-only loads.
template <typename S, bool CG = false> struct Pops {
  const S *__restrict__ p;
  long long plane;
  int nxp;
  __device__ __forceinline__ auto at(int q, int x, int y) const {
#ifdef PEMLBM_BOUNDS_CHECK
    const long long i = pop_index(q, (long long)y * nxp + x, plane);
    using V = decltype(ldp<CG>(p));
    if (!in_bounds(i, pop_extent(plane, nxp), 1)) return V(0);
#endif
    return ldp<CG>(p + pop_index(q, (long long)y * nxp + x, plane));
  }
};

// Inlet parabola at height yh (cell centres at integer y).
template <typename R> __device__ __forceinline__ R inlet_u(const KArgsT<R> &a, R yh) {
  R s = (yh - R(a.y_ch0) + R(0.5)) / R(a.h_ch);
  return (s <= R(0) || s >= R(1)) ? R(0) : R(6) * R(a.u_in_avg) * s * (R(1) - s);
}

// ------------------------------------------------------------------ pull
// Every cell first loads its 24 interior pulls unconditionally (the
// allocation carries a guard after the last plane, so the addresses of
// edge cells stay inside it); links whose source lies outside the plain
// fluid are then replaced below.  Issuing the loads before the node mask
// arrives keeps one DRAM latency off the critical path.

// Flow link i into cell (x, y) whose source may lie outside the fluid;
// `v` is the interior pull already loaded for this link.  X: the extended
// set-ups (closed x ends, fixed wall values, buoyancy) are compiled in; the
// cathode's own step kernels are built without them.
template <typename S, typename R, bool CG = false, bool X = false>
__device__ R pull_flow_edge(const Pops<S, CG> &src, const KArgsT<R> &a, const uint8_t *__restrict__ mask,
                            const uint16_t *__restrict__ mid, const MatCoef<R> *__restrict__ pal,
                            int i, int x, int y, uint8_t m, R v) {
  const int EX[9] = EX9_TAB, EY[9] = EY9_TAB, OP[9] = OP9_TAB;
  int sx = x - EX[i], sy = y - EY[i];
  if (sy < 0 || sy >= a.ny) return R(src.at(OP[i], x, y));            // wall
  if ((sx < 0 && a.halo_lo) || (sx >= a.nx && a.halo_hi)) {
    // the neighbour slab's ghost, unless that cell is solid (second mask plane)
    if ((m & M_NEAR_SOLID) && ((ld_mask(mask, a.plane + (long long)y * a.nxp + x, a, 10) >> (i - 1)) & 1u))
      return R(src.at(OP[i], x, y));
    return v;
  }
  if (sx < 0 || sx >= a.nx) {
    if (a.periodic) {
      sx = sx < 0 ? sx + a.nx : sx - a.nx;
    } else {
      const bool in = sx < 0;
      if constexpr (X)
        if (!in && a.closed_x) return R(src.at(OP[i], x, y));       // closed end: wall
      if (in && !(a.inlet_pressure && (m & M_INLET))) {             // velocity inlet / wall
        R w = R(src.at(OP[i], x, y));
        if (m & M_INLET) w += R(6) * w9<R>(i) * R(EX[i]) * inlet_u<R>(a, R(y) - R(0.5) * R(EY[i]));
        return w;
      }
      // outlet, or the pressure inlet: a virtual column (nx, or -1) repeats
      // the lattice's last (or first) column at the source row, with its
      // equilibrium pressure part moved to phi p = 1/3 (+ dp_in at the
      // inlet); at the inlet a source row outside the channel is the GDL's
      // end wall
      const int vx = in ? 0 : a.nx - 1;
      const long long vc = (long long)sy * a.nxp + vx;
      if (in && !(ld_mask(mask, vc, a, 11) & M_INLET)) return R(src.at(OP[i], x, y));
      R d[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) d[k] = R(src.at(k, vx, sy));
      R jx = d[1] - d[3] + d[5] - d[6] - d[7] + d[8];
      R jy = d[2] - d[4] + d[5] + d[6] - d[7] - d[8];
      R s18 = ((d[1] + d[3]) + (d[2] + d[4])) + ((d[5] + d[7]) + (d[6] + d[8]));
      R inv_phi = pal[ld_mid(mid, vc, a, 12)].inv_phi;
      R dP = (in ? R(a.dp_in) : R(0)) + (R(-0.6) * s18 + R(0.4) * (jx * jx + jy * jy) * inv_phi);
      return d[i] + lam9<R>(i) * dP;
    }
    if ((m & M_NEAR_SOLID) && (ld_mask(mask, (long long)sy * a.nxp + sx, a, 14) & REG_MASK) == REG_SOLID)
      return R(src.at(OP[i], x, y));
    return R(src.at(i, sx, sy));                                      // periodic wrap
  }
  if ((m & M_NEAR_SOLID) && (ld_mask(mask, (long long)sy * a.nxp + sx, a, 14) & REG_MASK) == REG_SOLID)
    return R(src.at(OP[i], x, y));                                    // solid grain
  return v;
}

// Anti-bounce-back of a wall link of scalar s held at value Cw (the
// halfway wall's value) given the bounced deviation w: in full values
// g_in = -g_out + 2 w1 Cw, i.e. in deviations -w + 2 w1 Cw - 2 wr1 Cref,
// evaluated as 2 w1 (Cw - Cref) + 2 (w1 - wr1) Cref so that a wall at the
// reference value adds no rounding of the two large products.
template <typename R>
__device__ __forceinline__ R wall_value(const KArgsT<R> &a, const MatCoef<R> &mc, int s, R w, R Cw) {
  const R w1 = mc.w1[s], Cref = R(a.Cref[s]);
  return -w + R(2) * w1 * (Cw - Cref) + R(2) * (w1 - R(a.wr1[s])) * Cref;
}

// Scalar link i of scalar s into cell (x, y); the bottom wall returns the
// insulated (or, with X, fixed) value and the reaction is applied afterwards.
template <typename S, typename R, bool CG = false, bool X = false>
__device__ R pull_scalar_edge(const Pops<S, CG> &src, const KArgsT<R> &a, const uint8_t *__restrict__ mask,
                              const MatCoef<R> &mc, int s, int i, int x, int y, uint8_t m, R v) {
  const int EX[5] = {0, 1, 0, -1, 0}, EY[5] = {0, 0, 1, 0, -1}, OP[5] = {0, 3, 4, 1, 2};
  const int q = 9 + 5 * s;
  int sx = x - EX[i], sy = y - EY[i];
  if (sy < 0) {
    R w = R(src.at(q + OP[i], x, y));
    if constexpr (X)
      if ((a.wall_dir >> (6 + s)) & 1) w = wall_value<R>(a, mc, s, w, R(a.Cwall[2][s]));
    return w;
  }
  if (sy >= a.ny) {
    R w = R(src.at(q + OP[i], x, y));
    if (a.top_dirichlet)
      w = wall_value<R>(a, mc, s, w, R(a.Ctop[s]));
    return w;
  }
  if ((sx < 0 && a.halo_lo) || (sx >= a.nx && a.halo_hi)) {
    // the neighbour slab's ghost, unless that cell is solid (second mask plane)
    if ((m & M_NEAR_SOLID) && ((ld_mask(mask, a.plane + (long long)y * a.nxp + x, a, 15) >> (i - 1)) & 1u))
      return R(src.at(q + OP[i], x, y));
    return v;
  }
  if (sx < 0 || sx >= a.nx) {
    if (a.periodic) {
      sx = sx < 0 ? sx + a.nx : sx - a.nx;
    } else if (sx < 0) {
      R w = R(src.at(q + OP[i], x, y));
      if (m & M_INLET) {
        w = wall_value<R>(a, mc, s, w, R(a.Cin[s]));
      } else if constexpr (X) {
        if ((a.wall_dir >> s) & 1) w = wall_value<R>(a, mc, s, w, R(a.Cwall[0][s]));
      }
      return w;
    } else if (X && a.closed_x) {
      R w = R(src.at(q + OP[i], x, y));
      if ((a.wall_dir >> (3 + s)) & 1) w = wall_value<R>(a, mc, s, w, R(a.Cwall[1][s]));
      return w;
    } else {
      return R(src.at(q + i, a.nx - 1, y));                           // fully developed
    }
    if ((m & M_NEAR_SOLID) && (ld_mask(mask, (long long)sy * a.nxp + sx, a, 14) & REG_MASK) == REG_SOLID)
      return R(src.at(q + OP[i], x, y));
    return R(src.at(q + i, sx, sy));
  }
  if ((m & M_NEAR_SOLID) && (ld_mask(mask, (long long)sy * a.nxp + sx, a, 14) & REG_MASK) == REG_SOLID)
    return R(src.at(q + OP[i], x, y));
  return v;
}

// The 24 post-stream deviations of one cell.
template <typename R> struct Cell {
  R f[9];
  R g[3][5];
};

// Rate constant of the catalyst at temperature deviation theta = T - T_in:
// A exp(e_in - c1 theta / (T T_in)) with T = T_in + theta.
template <typename R> __device__ __forceinline__ R rate(const KArgsT<R> &a, R A, R theta) {
  R T = R(a.T_in) + theta;
  return A * exp(R(a.k_ein) - R(a.k_c1) * theta / (T * R(a.T_in)));
}
// Butler-Volmer anodic branch: O2 produced per step (link or cell); 0 for
// Tafel kinetics (A = 0), without evaluating the exponential.
template <typename R> __device__ __forceinline__ R rate_anodic(const KArgsT<R> &a, R A, R theta) {
  if (A == R(0)) return R(0);
  R T = R(a.T_in) + theta;
  return A * exp(R(a.k_ein_a) - R(a.k_c1_a) * theta / (T * R(a.T_in)));
}

// Sum of the cell's own post-collision deviations of scalar s.
// Opposite links are summed first: their large advective parts cancel
// exactly in FP32 (Sterbenz), so the small sum keeps full precision.
template <typename R>
__device__ __forceinline__ R d2q5_sum(R d0, R d1, R d2, R d3, R d4) {
  return d0 + ((d1 + d3) + (d2 + d4));
}

template <typename S, typename R, bool CG = false>
__device__ __forceinline__ R own_sum(const Pops<S, CG> &src, int s, int x, int y) {
  const int q = 9 + 5 * s;
  return d2q5_sum<R>(R(src.at(q, x, y)), R(src.at(q + 1, x, y)), R(src.at(q + 2, x, y)),
                     R(src.at(q + 3, x, y)), R(src.at(q + 4, x, y)));
}

// Surface reaction of the thin film at a bottom cell (Sec. 4): the implicit
// Tafel link.  Returns the O2 consumed J (lattice units) and modifies the
// three upward links.  theta_n = T^n - T_in from the cell's own state.
template <typename S, typename R, bool CG = false>
__device__ __forceinline__ R surface_reaction(const Pops<S, CG> &src, const KArgsT<R> &a,
                                              const MatCoef<R> &mc, int x, Cell<R> &c) {
  R theta = own_sum<S, R, CG>(src, 0, x, 0) + a.theta0;
  R k = rate<R>(a, R(a.kA_surf), theta);
  R kappa = k / (R(2) * mc.w1[1]);
  R gdown = c.g[1][2] + R(a.wr1[1]) * R(a.Cref[1]);   // full g*_4 of O2 (bounced)
  // J = k C_w - k_a with C_w = (g_down + g_up)/(2 w1), solved for g_up
  R ka = rate_anodic<R>(a, R(a.kA_surf_a), theta);
  R J = (gdown * (R(2) * kappa) - ka) / (R(1) + kappa);
  c.g[1][2] -= J;
  c.g[0][2] += R(a.hpo) * mc.inv_sigma * J;
  c.g[2][2] += R(2) * J;
  return J;
}

// Volumetric catalyst sink of a catalyst cell (backward Euler in C).
template <typename S, typename R, bool CG = false>
__device__ __forceinline__ R volume_sink(const Pops<S, CG> &src, const KArgsT<R> &a, int x, int y) {
  R theta = own_sum<S, R, CG>(src, 0, x, y) + a.theta0;
  R C = own_sum<S, R, CG>(src, 1, x, y) + R(a.Cref[1]);
  R k = rate<R>(a, R(a.kA_vol), theta);
  R ka = rate_anodic<R>(a, R(a.kA_vol_a), theta);
  return (ka - k * C) / (R(1) + k);   // backward Euler of dC/dt = k_a - k C
}

// The 24 interior pulls of cell (x, y), issued without looking at the mask.
template <typename S, typename R, bool CG = false>
__device__ __forceinline__ void load_interior(const Pops<S, CG> &src, const KArgsT<R> &a, int x, int y,
                                              Cell<R> &c) {
  const long long c0 = (long long)y * a.nxp + x, P = a.plane, W = a.nxp;
  // links 0-4: one group load from the source cell x - e_i; the offsets are
  // pop_index's, written from two base addresses (fewer live registers)
  const long long from[5] = {0, -1, -W, 1, W};
#pragma unroll
  for (int i = 0; i < 5; ++i) {
#ifdef PEMLBM_BOUNDS_CHECK
    const long long k = 4 * (i * P + c0 + from[i]), n = pop_extent(P, a.nxp);
    if (!in_bounds(k, n, 2) || !in_bounds(k + 3, n, 2)) {
      c.f[i] = c.g[0][i] = c.g[1][i] = c.g[2][i] = R(0);
      continue;
    }
#endif
    const auto v = ldq<CG>(src.p + 4 * (i * P + c0 + from[i]));
    c.f[i] = v.v[0];
    c.g[0][i] = v.v[1];
    c.g[1][i] = v.v[2];
    c.g[2][i] = v.v[3];
  }
  const S *d = src.p + 20 * P + c0;
#ifdef PEMLBM_BOUNDS_CHECK
  const long long n = pop_extent(P, a.nxp), dk[4] = {20 * P + c0 - W - 1, 21 * P + c0 - W + 1,
                                                     22 * P + c0 + W + 1, 23 * P + c0 + W - 1};
  if (!in_bounds(dk[0], n, 3) || !in_bounds(dk[1], n, 3) || !in_bounds(dk[2], n, 3) ||
      !in_bounds(dk[3], n, 3)) {
    c.f[5] = c.f[6] = c.f[7] = c.f[8] = R(0);
    return;
  }
#endif
  c.f[5] = ldp<CG>(d - W - 1);
  c.f[6] = ldp<CG>(d + P - W + 1);
  c.f[7] = ldp<CG>(d + 2 * P + W + 1);
  c.f[8] = ldp<CG>(d + 3 * P + W - 1);
}

// The cell's own 24 stored values (no streaming), by groups.
template <typename S, typename R, bool CG = false>
__device__ __forceinline__ void load_own(const Pops<S, CG> &src, int x, int y, Cell<R> &c) {
  const long long c0 = (long long)y * src.nxp + x, P = src.plane;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
#ifdef PEMLBM_BOUNDS_CHECK
    const long long k = pop_index(i, c0, P), n = pop_extent(P, src.nxp);
    if (!in_bounds(k, n, 4) || !in_bounds(k + 3, n, 4)) {
      c.f[i] = c.g[0][i] = c.g[1][i] = c.g[2][i] = R(0);
      continue;
    }
#endif
    const auto v = ldq<CG>(src.p + pop_index(i, c0, P));
    c.f[i] = v.v[0];
    c.g[0][i] = v.v[1];
    c.g[1][i] = v.v[2];
    c.g[2][i] = v.v[3];
  }
#pragma unroll
  for (int i = 5; i < 9; ++i) {
#ifdef PEMLBM_BOUNDS_CHECK
    if (!in_bounds(pop_index(i, c0, P), pop_extent(P, src.nxp), 4)) {
      c.f[i] = R(0);
      continue;
    }
#endif
    c.f[i] = ldp<CG>(src.p + pop_index(i, c0, P));
  }
}

// Replaces the pulls of links that cross a wall, the inlet, the outlet, a
// periodic seam or a solid grain (cells with any edge bit only).
template <typename S, typename R, bool CG = false, bool X = false>
__device__ __forceinline__ void fix_edges(const Pops<S, CG> &src, const KArgsT<R> &a,
                                          const uint8_t *__restrict__ mask,
                                          const uint16_t *__restrict__ mid,
                                          const MatCoef<R> *__restrict__ pal,
                                          const MatCoef<R> &mc, int x, int y, uint8_t m,
                                          Cell<R> &c) {
#pragma unroll
  for (int i = 1; i < 9; ++i)
    c.f[i] = pull_flow_edge<S, R, CG, X>(src, a, mask, mid, pal, i, x, y, m, c.f[i]);
#pragma unroll
  for (int s = 0; s < 3; ++s)
#pragma unroll
    for (int i = 1; i < 5; ++i)
      c.g[s][i] = pull_scalar_edge<S, R, CG, X>(src, a, mask, mc, s, i, x, y, m, c.g[s][i]);
}

// Cells whose only edge bit is M_NEAR_SOLID: a link whose source is a solid
// grain takes the cell's own population of the opposite link (bounce-back,
// as pull_flow_edge and pull_scalar_edge do); nb holds the solid sources
// (bit i - 1 for link i of Eq. 2; the D2Q5 links are the first four).
template <typename S, typename R, bool CG = false>
__device__ __forceinline__ void bounce_solid(const Pops<S, CG> &src, int x, int y, uint32_t nb,
                                             Cell<R> &c) {
  const int OP[9] = OP9_TAB;
#pragma unroll
  for (int i = 1; i < 9; ++i)
    if (nb & (1u << (i - 1))) c.f[i] = R(src.at(OP[i], x, y));
#pragma unroll
  for (int s = 0; s < 3; ++s)
#pragma unroll
    for (int i = 1; i < 5; ++i)
      if (nb & (1u << (i - 1))) c.g[s][i] = R(src.at(9 + 5 * s + OP[i], x, y));
}

// Pull all 24 populations of a non-solid cell (x, y).
template <typename S, typename R, bool CG = false, bool X = false>
__device__ __forceinline__ void pull_cell(const Pops<S, CG> &src, const KArgsT<R> &a,
                                          const uint8_t *__restrict__ mask,
                                          const uint16_t *__restrict__ mid,
                                          const MatCoef<R> *__restrict__ pal,
                                          const MatCoef<R> &mc, int x, int y, uint8_t m,
                                          Cell<R> &c) {
  load_interior<S, R, CG>(src, a, x, y, c);
  if (m & M_EDGE) fix_edges<S, R, CG, X>(src, a, mask, mid, pal, mc, x, y, m, c);
}

// Square root and reciprocal of the Eq. 8 velocity in the FP32 arithmetic
// path: the hardware approximations (PTX sqrt.approx.f32, rcp.approx.ftz.f32,
// a few instructions each instead of the correctly rounded sequences, which
// made up a large part of the 16-bit step's instruction-bound time).  Their
// error is of the order of FP32 rounding itself, well below what storing the
// populations in FP32 adds at every step; the argument of the reciprocal is
// at least l0 >= 1/2, never subnormal.  FP64 keeps the correctly rounded
// operations.
__device__ __forceinline__ float vsqrt(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double vsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float vrcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double vrcp(double x) { return 1.0 / x; }

// Macroscopic values of a post-stream cell (Eq. 8, 11).
template <typename R> struct Macro {
  R ux, uy, un;     // velocity and its magnitude
  R Pdev;           // phi p - rho0/3
  R C[3];           // deviation sums (value - Cref)
  R vx, vy;         // auxiliary velocity of Eq. 8 (the reverse records keep it)
};

// Body force per unit mass at a cell whose T deviation sum is CT: the
// uniform force along x, plus the Boussinesq buoyancy with X.
template <typename R, bool X>
__device__ __forceinline__ void body_force(const KArgsT<R> &a, R CT, R &Gx, R &Gy) {
  Gx = R(a.body_g);
  Gy = R(0);
  if constexpr (X) {
    const R tb = CT + R(a.buoy_off);   // T - T_buoy
    Gx += R(a.gam_x) * tb;
    Gy = R(a.gam_y) * tb;
  }
}

template <typename R, bool X = false>
__device__ __forceinline__ Macro<R> macros(const KArgsT<R> &a, const MatCoef<R> &mc, const Cell<R> &c) {
  Macro<R> r;
  const R *d = c.f;
  R Gx, Gy;
  body_force<R, X>(a, d2q5_sum<R>(c.g[0][0], c.g[0][1], c.g[0][2], c.g[0][3], c.g[0][4]), Gx, Gy);
  R vx = d[1] - d[3] + d[5] - d[6] - d[7] + d[8] + R(0.5) * mc.phi * Gx;
  R vy = d[2] - d[4] + d[5] + d[6] - d[7] - d[8];
  if constexpr (X) vy += R(0.5) * mc.phi * Gy;
  // u = v / den with one reciprocal of den; |u| = |v| / den, so u's
  // magnitude needs no square root of its own
  R vn = vsqrt(vx * vx + vy * vy);
  R inv_den = vrcp(mc.l0 + vsqrt(mc.l0 * mc.l0 + mc.l1 * vn));
  r.vx = vx;
  r.vy = vy;
  r.ux = vx * inv_den;
  r.uy = vy * inv_den;
  r.un = vn * inv_den;
  R s18 = ((d[1] + d[3]) + (d[2] + d[4])) + ((d[5] + d[7]) + (d[6] + d[8]));
  r.Pdev = R(0.6) * s18 - R(0.4) * (r.ux * r.ux + r.uy * r.uy) * mc.inv_phi;
#pragma unroll
  for (int s = 0; s < 3; ++s)
    r.C[s] = d2q5_sum<R>(c.g[s][0], c.g[s][1], c.g[s][2], c.g[s][3], c.g[s][4]);
  return r;
}

// D2Q9 MRT collision with the porous force, in deviation moments (Eq. 1, 3-7).
template <typename R, bool X = false>
__device__ __forceinline__ void collide_flow(const KArgsT<R> &a, const MatCoef<R> &mc, const Macro<R> &u,
                                             const R d[9], R o[9]) {
  const R sn = R(a.s_nu), sq = R(a.s_q);
  R ux = u.ux, uy = u.uy, u2 = ux * ux + uy * uy, un = u.un, ip = mc.inv_phi;
  R Gx, Gy;
  body_force<R, X>(a, u.C[0], Gx, Gy);
  R Fx = -mc.darcy * ux - mc.forch * un * ux + mc.phi * Gx;
  R Fy = -mc.darcy * uy - mc.forch * un * uy;
  if constexpr (X) Fy += mc.phi * Gy;
  R ax = (d[1] + d[3]) + (d[2] + d[4]), dg = (d[5] + d[7]) + (d[6] + d[8]);
  R m0 = d[0] + ax + dg;
  R m1 = R(-4) * d[0] - ax + R(2) * dg;
  R m2 = R(4) * d[0] - R(2) * ax + dg;
  R m3 = d[1] - d[3] + d[5] - d[6] - d[7] + d[8];
  R m4 = R(-2) * (d[1] - d[3]) + d[5] - d[6] - d[7] + d[8];
  R m5 = d[2] - d[4] + d[5] + d[6] - d[7] - d[8];
  R m6 = R(-2) * (d[2] - d[4]) + d[5] + d[6] - d[7] - d[8];
  R m7 = d[1] - d[2] + d[3] - d[4];
  R m8 = d[5] - d[6] + d[7] - d[8];
  R uF = ux * Fx + uy * Fy;
  // m* = m - S (m - m_eq) + (1 - S/2) G, equilibria relative to the rest state
  R half_n = R(1) - R(0.5) * sn, half_q = R(1) - R(0.5) * sq;
  m0 = m0 - sn * m0;
  m1 = m1 - sn * (m1 - (R(6) * u.Pdev + R(3) * u2 * ip)) + half_n * (R(6) * uF * ip);
  m2 = m2 - sn * (m2 - (R(-9) * u.Pdev - R(3) * u2 * ip)) + half_n * (R(-6) * uF * ip);
  m3 = m3 + Fx;
  m4 = m4 - sq * (m4 + ux) + half_q * (-Fx);
  m5 = m5 + Fy;
  m6 = m6 - sq * (m6 + uy) + half_q * (-Fy);
  m7 = m7 - sn * (m7 - (ux * ux - uy * uy) * ip) + half_n * (R(2) * (ux * Fx - uy * Fy) * ip);
  m8 = m8 - sn * (m8 - ux * uy * ip) + half_n * ((ux * Fy + uy * Fx) * ip);
  // f* = M^-1 m*, M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)
  R a0 = m0 * R(1.0 / 9), a1 = m1 * R(1.0 / 36), a2 = m2 * R(1.0 / 36);
  R a3 = m3 * R(1.0 / 6), a4 = m4 * R(1.0 / 12), a5 = m5 * R(1.0 / 6), a6 = m6 * R(1.0 / 12);
  R a7 = m7 * R(0.25), a8 = m8 * R(0.25);
  // The conserved moments are closed by remainders: 1/6 and 1/9 are not
  // binary fractions, so 6 * (m3 / 6) != m3 in floating point, and a collision
  // built only from the scaled moments would multiply the momentum (and the
  // mass) by the same constant factor at every cell and step, a coherent
  // source.  Instead the axis pairs carry what the diagonals leave of m3 and
  // m5, and the rest population what the others leave of m0 (identical in
  // exact arithmetic; rounding then stays local and unbiased).
  R axs = a0 - a1 - R(2) * a2, dgs = a0 + R(2) * a1 + a2;
  o[5] = dgs + a3 + a4 + a5 + a6 + a8;
  o[6] = dgs - a3 - a4 + a5 + a6 - a8;
  o[7] = dgs - a3 - a4 - a5 - a6 + a8;
  o[8] = dgs + a3 + a4 - a5 - a6 - a8;
  const R hx = R(0.5) * (m3 - ((o[5] - o[7]) + (o[8] - o[6])));
  const R hy = R(0.5) * (m5 - ((o[5] - o[7]) + (o[6] - o[8])));
  o[1] = (axs + a7) + hx;
  o[3] = (axs + a7) - hx;
  o[2] = (axs - a7) + hy;
  o[4] = (axs - a7) - hy;
  o[0] = m0 - (((o[1] + o[3]) + (o[2] + o[4])) + ((o[5] + o[7]) + (o[6] + o[8])));
}

// D2Q5 MRT collision of scalar s in deviation moments (Eq. 10), plus a
// volumetric source src added with the cell's equilibrium weights.
template <typename R>
__device__ __forceinline__ void collide_scalar(const KArgsT<R> &a, const MatCoef<R> &mc, int s,
                                               R ux, R uy, R Cdev, const R d[5], R srcv, R o[5]) {
  const R Q1 = mc.q1[s], Q3 = R(a.Q3);
  // the advected value: C, or its excess over the inlet value (then about
  // zero in the deviation storage, so the flux populations stay small)
  R Ca = Cdev + R(a.adv_off[s]);
  R n0 = Cdev;
  R n1 = d[1] - d[3], n2 = d[2] - d[4];
  R e13 = d[1] + d[3], e24 = d[2] + d[4];
  R n3 = R(-4) * d[0] + (e13 + e24);
  R n4 = e13 - e24;
  R b = mc.b[s];
  n1 -= Q1 * (n1 - ux * Ca);
  n2 -= Q1 * (n2 - uy * Ca);
  n3 -= Q3 * (n3 - (b * Cdev + (b - R(a.bref[s])) * R(a.Cref[s])));
  n4 -= Q3 * n4;
  R w1 = mc.w1[s];
  // even parts first, the large odd (advective) part added last; the rest
  // population takes what the moving ones leave of n0 + src, so that the
  // collision conserves C up to one local rounding (5 * 0.2 != 1 in binary:
  // the scaled form would multiply every cell's C by the same factor at
  // every step)
  R ev = n0 * R(0.2) + n3 * R(0.05) + w1 * srcv;
  R ex = ev + R(0.25) * n4, ey = ev - R(0.25) * n4;
  o[1] = ex + R(0.5) * n1;
  o[3] = ex - R(0.5) * n1;
  o[2] = ey + R(0.5) * n2;
  o[4] = ey - R(0.5) * n2;
  o[0] = (n0 + srcv) - ((o[1] + o[3]) + (o[2] + o[4]));
}

}  // namespace pemlbm
