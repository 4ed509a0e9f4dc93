// Lattice-Boltzmann kernels: the fused pull stream-collide over the whole lattice (Eqs. 9-10
// with Guo forcing and half-way bounce-back), the velocity gather at the active interface
// tiles (the velocity step of Sec. III), and the read-back / initialisation helpers.
//
// Populations are stored as deviations f_i - w_i rho0 ("shifted"), structure of arrays
// [19][nz][ny][nx] with x fastest. The state array holds post-collision populations of
// the previous step; a pull reads f_i(x - c_i) from it, which is the streaming step.
// Right after initialisation the state holds post-streaming populations ("fresh") and the
// first collision reads them in place. The storage type S may be narrower than the
// arithmetic type `real` (FP16 / BF16 storage with FP32 arithmetic), see Storage below.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <string.h>

#include "iblb_internal.cuh"

namespace iblb {
namespace {

template <typename real>
struct LatParams {
  int nx, ny, nz, has_walls;
  int ntx, nty;
  size_t ncell;
  real omega;        // 1/tau
  real guo;          // 1 - 1/(2 tau)
  real rho0;
  real g[3];         // uniform body force
  real wb[19];       // 6 w_i rho0 (c_i . u_bottom): moving-wall term, bottom wall
  real wt[19];       // same for the top wall
};

template <typename real>
LatParams<real> lat_params(const Ctx &c) {
  LatParams<real> p;
  p.nx = c.nx; p.ny = c.ny; p.nz = c.nz; p.has_walls = c.has_walls;
  p.ntx = c.ntx; p.nty = c.nty;
  p.ncell = c.ncell;
  p.omega = (real)(1.0 / c.tau);
  p.guo = (real)(1.0 - 0.5 / c.tau);
  p.rho0 = (real)c.rho0;
  for (int k = 0; k < 3; k++) p.g[k] = (real)c.g[k];
  for (int i = 0; i < Q; i++) {
    double cb = cx(i) * c.ub[0] + cy(i) * c.ub[1] + cz(i) * c.ub[2];
    double ct = cx(i) * c.ut[0] + cy(i) * c.ut[1] + cz(i) * c.ut[2];
    p.wb[i] = (real)(6.0 * wgt(i) * c.rho0 * cb);
    p.wt[i] = (real)(6.0 * wgt(i) * c.rho0 * ct);
  }
  return p;
}

// Storage of the shifted populations. Population i is stored as g_i = (f_i - w_i rho0) k_i
// in type S and used as f_i - w_i rho0 in type `real`. For float and double k_i = 1. For the
// 16-bit types (arithmetic stays FP32) k_i = K / w_i: the deviations of the 19 directions
// then share one scale, about |drho| + 3 |c.u|, and with K = 1024 the FP16 values sit well
// inside its normal range (6.1e-5 .. 65504), so each keeps FP16's 11-bit significand. BF16
// has FP32's exponent range and needs no shift (K = 1).
template <typename S>
struct Storage;
template <>
struct Storage<double> {
  using V2 = double2;
  static constexpr double K = 0.0;  // 0: stored unscaled
};
template <>
struct Storage<float> {
  using V2 = float2;
  static constexpr double K = 0.0;
};
template <>
struct Storage<__half> {
  using V2 = __half2;
  static constexpr double K = 1024.0;
};
template <>
struct Storage<__nv_bfloat16> {
  using V2 = __nv_bfloat162;
  static constexpr double K = 1.0;
};

// k_i and 1 / k_i
template <typename S>
__host__ __device__ constexpr double kscale(int i) {
  return Storage<S>::K == 0.0 ? 1.0 : Storage<S>::K / wgt(i);
}
template <typename S>
__host__ __device__ constexpr double kinv(int i) {
  return Storage<S>::K == 0.0 ? 1.0 : wgt(i) / Storage<S>::K;
}

__device__ __forceinline__ float widen(float v) { return v; }
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ float widen(__half v) { return __half2float(v); }
__device__ __forceinline__ float widen(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ void widen2(float2 v, float &a, float &b) { a = v.x; b = v.y; }
__device__ __forceinline__ void widen2(double2 v, double &a, double &b) { a = v.x; b = v.y; }
__device__ __forceinline__ void widen2(__half2 v, float &a, float &b) {
  a = __low2float(v);
  b = __high2float(v);
}
__device__ __forceinline__ void widen2(__nv_bfloat162 v, float &a, float &b) {
  a = __low2float(v);
  b = __high2float(v);
}

// Rounding of `real` values to the storage type (round to nearest even).
template <typename S>
struct Narrow;
template <>
struct Narrow<float> {
  __device__ static float one(float v) { return v; }
  __device__ static float2 two(float a, float b) { return make_float2(a, b); }
};
template <>
struct Narrow<double> {
  __device__ static double one(double v) { return v; }
  __device__ static double2 two(double a, double b) { return make_double2(a, b); }
};
template <>
struct Narrow<__half> {
  __device__ static __half one(float v) { return __float2half_rn(v); }
  __device__ static __half2 two(float a, float b) { return __floats2half2_rn(a, b); }
};
template <>
struct Narrow<__nv_bfloat16> {
  __device__ static __nv_bfloat16 one(float v) { return __float2bfloat16_rn(v); }
  __device__ static __nv_bfloat162 two(float a, float b) { return __floats2bfloat162_rn(a, b); }
};

// The deviation f_i - w_i rho0 stored at element `idx` of array p (population i).
template <typename real, typename S>
__device__ __forceinline__ real dev(const S *__restrict__ p, int i, size_t idx) {
  return real(widen(p[idx])) * real(kinv<S>(i));
}

// Loads of the shell-velocity pass, whose pulled rows are scattered over the lattice: the
// prefetch-size qualifier bounds each L2 fill from DRAM to 64 bytes (a plain load brings a
// whole 128-byte line for a 4-byte access). The pass runs beside the full-lattice pass, which
// gets the DRAM bandwidth saved (256^3: 23.6 MB against 37.4 MB per launch).
#define IBLB_SCATTER_LD "ld.global.L2::64B"
__device__ __forceinline__ float ld_scattered(const float *p) {
  float v;
  asm(IBLB_SCATTER_LD ".f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double ld_scattered(const double *p) {
  double v;
  asm(IBLB_SCATTER_LD ".f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ __half ld_scattered(const __half *p) {
  unsigned short v;
  asm(IBLB_SCATTER_LD ".b16 %0, [%1];" : "=h"(v) : "l"(p));
  return __ushort_as_half(v);
}
__device__ __forceinline__ __nv_bfloat16 ld_scattered(const __nv_bfloat16 *p) {
  unsigned short v;
  asm(IBLB_SCATTER_LD ".b16 %0, [%1];" : "=h"(v) : "l"(p));
  return __ushort_as_bfloat16(v);
}
__device__ __forceinline__ float2 ld_scattered(const float2 *p) {
  float2 v;
  asm(IBLB_SCATTER_LD ".v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ double2 ld_scattered(const double2 *p) {
  double2 v;
  asm(IBLB_SCATTER_LD ".v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ __half2 ld_scattered(const __half2 *p) {
  unsigned v;
  asm(IBLB_SCATTER_LD ".b32 %0, [%1];" : "=r"(v) : "l"(p));
  __half2 h;
  memcpy(&h, &v, sizeof(v));
  return h;
}
__device__ __forceinline__ __nv_bfloat162 ld_scattered(const __nv_bfloat162 *p) {
  unsigned v;
  asm(IBLB_SCATTER_LD ".b32 %0, [%1];" : "=r"(v) : "l"(p));
  __nv_bfloat162 h;
  memcpy(&h, &v, sizeof(v));
  return h;
}

// dev() through ld_scattered
template <typename real, typename S>
__device__ __forceinline__ real dev_scattered(const S *__restrict__ p, int i, size_t idx) {
  return real(widen(ld_scattered(p + idx))) * real(kinv<S>(i));
}

// Pull the 19 post-streaming populations of fluid node (x, y, z) from post-collision array
// `fp`. A link whose source is a wall node is bounced back: the opposite post-collision
// population of the same node plus the moving-wall term.
template <typename real, typename S, bool SCATTERED = false>
__device__ __forceinline__ void pull(const S *__restrict__ fp, const LatParams<real> &P, int x,
                                     int y, int z, real f[Q]) {
  const int xm = x == 0 ? P.nx - 1 : x - 1, xp = x == P.nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? P.ny - 1 : y - 1, yp = y == P.ny - 1 ? 0 : y + 1;
  int zm = z - 1, zp = z + 1;
  if (!P.has_walls) {
    zm = z == 0 ? P.nz - 1 : zm;
    zp = z == P.nz - 1 ? 0 : zp;
  }
  const bool wall_below = P.has_walls && zm == 0;
  const bool wall_above = P.has_walls && zp == P.nz - 1;
  const size_t plane = (size_t)P.nx * P.ny;
  // source offsets along each axis, indexed by 1 - c (c = +1 -> minus side, c = -1 -> plus side)
  const size_t zo[3] = {(size_t)zm * plane, (size_t)z * plane, (size_t)zp * plane};
  const size_t yo[3] = {(size_t)ym * P.nx, (size_t)y * P.nx, (size_t)yp * P.nx};
  const int xo[3] = {xm, x, xp};
  const size_t n = zo[1] + yo[1] + x;
#pragma unroll
  for (int i = 0; i < Q; i++) {
    // (opposite directions have the same weight, so population i's scale serves both)
    const bool bounce = (cz(i) > 0 && wall_below) || (cz(i) < 0 && wall_above);
    const size_t idx = bounce ? (size_t)opp(i) * P.ncell + n
                              : (size_t)i * P.ncell + zo[1 - cz(i)] + yo[1 - cy(i)] + xo[1 - cx(i)];
    f[i] = SCATTERED ? dev_scattered<real>(fp, i, idx) : dev<real>(fp, i, idx);
    if (bounce) f[i] += cz(i) > 0 ? P.wb[i] : P.wt[i];
  }
}

// Interface force density of node (x, y, z) from the active-tile table (0 if inactive).
template <typename real>
__device__ __forceinline__ void tile_force(const int *__restrict__ tile_slot,
                                           const Vec4<real> *__restrict__ Fslot,
                                           const LatParams<real> &P, int x, int y, int z,
                                           real F[3]) {
  F[0] = P.g[0];
  F[1] = P.g[1];
  F[2] = P.g[2];
  if (tile_slot == nullptr) return;
  const int t = ((z >> 2) * P.nty + (y >> 2)) * P.ntx + (x >> 2);
  const int s = tile_slot[t];
  if (s >= 0) {
    const int cell = (x & 3) + 4 * (y & 3) + 16 * (z & 3);
    const Vec4<real> Fs = Fslot[(size_t)s * TILE_CELLS + cell];
    F[0] += Fs.x;
    F[1] += Fs.y;
    F[2] += Fs.z;
  }
}

__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }

// n / (hi + lo) for |lo| << |hi| and r1 ~ 1/hi: q0 = n r1, then the residual
// n - q0 hi - q0 lo (the first product exactly, by a fused multiply-add) corrects it once.
template <typename real>
__device__ __forceinline__ real quotient(real n, real hi, real lo, real r1) {
  const real q0 = n * r1;
  real e = fma_(-q0, hi, n);
  e = fma_(-q0, lo, e);
  return fma_(e, r1, q0);
}

// BGK collision with Guo forcing (Eqs. 9-10) of one node's shifted populations f, storing
// the post-collision populations at node n of fout. Opposite directions i, i+1 (i odd) share
// c.u and c.F up to sign, so each pair is computed from its symmetric and antisymmetric parts:
//   f^eq - w rho0 = w [drho + rho (4.5 (c.u)^2 - 1.5 u^2)] +- w rho 3 (c.u)      (Eq. 10)
//   S = w (1 - 1/2tau) [9 (c.F)(c.u) - 3 u.F] +- w (1 - 1/2tau) 3 (c.F)          (Eq. 9)
// With FORCE false the force is zero and the Guo terms vanish.
template <typename real, bool FORCE>
__device__ __forceinline__ void collide(real f[Q], const real F[3], const LatParams<real> &P) {
  // moments: rho = rho0 + sum f~, j = sum c f~ (the rest-state part carries no momentum)
  real drho = f[0], jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    drho += f[i] + f[i + 1];
    const real d = f[i] - f[i + 1];
    if (cx(i)) jx += cx(i) > 0 ? d : -d;
    if (cy(i)) jy += cy(i) > 0 ? d : -d;
    if (cz(i)) jz += cz(i) > 0 ? d : -d;
  }
  // rho = rho0 + drho is never rounded as a whole: rho_lo carries the rounding remainder of
  // the sum (Fast2Sum, |rho0| >= |drho|), and rho X is expanded as rho0 X + drho X
  const real rho_hi = P.rho0 + drho;
  const real rho_lo = (P.rho0 - rho_hi) + drho;
  const real r1 = real(1) / rho_hi;
  real ux = jx, uy = jy, uz = jz;
  if (FORCE) {
    ux += real(0.5) * F[0];
    uy += real(0.5) * F[1];
    uz += real(0.5) * F[2];
  }
  // u = j'/(rho_hi + rho_lo): a first quotient and one residual correction by fused
  // multiply-adds, which keeps u within about an ulp of the exact quotient. The float
  // rounding of u is what the FP32 path's drift from the FP64 solution grows from (the other
  // roundings of the collision, the storage and the interface part matter two to three
  // orders of magnitude less), so it is worth the six extra multiply-adds.
  ux = quotient(ux, rho_hi, rho_lo, r1);
  uy = quotient(uy, rho_hi, rho_lo, r1);
  uz = quotient(uz, rho_hi, rho_lo, r1);
  const real uu15 = real(1.5) * (ux * ux + uy * uy + uz * uz);
  const real om = P.omega;
  real uF3 = 0;
  if (FORCE) uF3 = real(3) * (ux * F[0] + uy * F[1] + uz * F[2]);
  {  // rest population
    const real w = (real)wgt(0);
    const real feq = w * (drho - P.rho0 * uu15 - drho * uu15);
    real out = f[0] + om * (feq - f[0]);
    if (FORCE) out -= w * P.guo * uF3;
    f[0] = out;
  }
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const real w = (real)wgt(i);
    const real cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
    const real xs = real(4.5) * cu * cu - uu15;
    const real xa = real(3) * cu;
    const real sym = w * (drho + P.rho0 * xs + drho * xs);
    const real asym = w * (P.rho0 * xa + drho * xa);
    real a = f[i] + om * (sym + asym - f[i]);
    real b = f[i + 1] + om * (sym - asym - f[i + 1]);
    if (FORCE) {
      const real cF = cx(i) * F[0] + cy(i) * F[1] + cz(i) * F[2];
      const real ssym = w * P.guo * (real(9) * cF * cu - uF3);
      const real sasym = w * P.guo * real(3) * cF;
      a += ssym + sasym;
      b += ssym - sasym;
    }
    f[i] = a;
    f[i + 1] = b;
  }
}

// Post-streaming populations a (node x0) and b (node x0 + 1) of two fluid nodes, x0 even,
// from post-collision array `fin` (FIRST: `fin` already holds post-streaming populations,
// read in place). Populations that do not move along x are one aligned 2-wide load; a link
// whose source is a wall node is bounced back (opposite population of the same node plus the
// moving-wall term).
template <typename real, typename S, bool FIRST>
__device__ __forceinline__ void load_pair(const S *__restrict__ fin, const LatParams<real> &P,
                                          int x0, int y, int z, real a[Q], real b[Q]) {
  using V2 = typename Storage<S>::V2;
  const size_t plane = (size_t)P.nx * P.ny;
  const size_t n = (size_t)z * plane + (size_t)y * P.nx + x0;
  if (FIRST) {
#pragma unroll
    for (int i = 0; i < Q; i++) {
      widen2(*reinterpret_cast<const V2 *>(fin + (size_t)i * P.ncell + n), a[i], b[i]);
      a[i] *= real(kinv<S>(i));
      b[i] *= real(kinv<S>(i));
    }
    return;
  }
  const int xm = x0 == 0 ? P.nx - 1 : x0 - 1;   // source of node x0 for c_x = +1
  const int xp = x0 + 2 == P.nx ? 0 : x0 + 2;   // source of node x0 + 1 for c_x = -1
  const int ym = y == 0 ? P.ny - 1 : y - 1, yp = y == P.ny - 1 ? 0 : y + 1;
  int zm = z - 1, zp = z + 1;
  if (!P.has_walls) {
    zm = z == 0 ? P.nz - 1 : zm;
    zp = z == P.nz - 1 ? 0 : zp;
  }
  const bool wall_below = P.has_walls && zm == 0;
  const bool wall_above = P.has_walls && zp == P.nz - 1;
  const size_t zo[3] = {(size_t)zm * plane, (size_t)z * plane, (size_t)zp * plane};
  const size_t yo[3] = {(size_t)ym * P.nx, (size_t)y * P.nx, (size_t)yp * P.nx};
#pragma unroll
  for (int i = 0; i < Q; i++) {
    if ((cz(i) > 0 && wall_below) || (cz(i) < 0 && wall_above)) {
      widen2(*reinterpret_cast<const V2 *>(fin + (size_t)opp(i) * P.ncell + n), a[i], b[i]);
      const real wall = cz(i) > 0 ? P.wb[i] : P.wt[i];
      a[i] = a[i] * real(kinv<S>(opp(i))) + wall;
      b[i] = b[i] * real(kinv<S>(opp(i))) + wall;
      continue;
    }
    const S *row = fin + (size_t)i * P.ncell + zo[1 - cz(i)] + yo[1 - cy(i)];
    if (cx(i) == 0) {
      widen2(*reinterpret_cast<const V2 *>(row + x0), a[i], b[i]);
    } else if (cx(i) > 0) {
      a[i] = widen(row[xm]);
      b[i] = widen(row[x0]);
    } else {
      a[i] = widen(row[x0 + 1]);
      b[i] = widen(row[xp]);
    }
    a[i] *= real(kinv<S>(i));
    b[i] *= real(kinv<S>(i));
  }
}

template <typename real, typename S>
__device__ __forceinline__ void store_pair(S *__restrict__ fout, const LatParams<real> &P,
                                           size_t n, const real a[Q], const real b[Q]) {
  using V2 = typename Storage<S>::V2;
#pragma unroll
  for (int i = 0; i < Q; i++)
    *reinterpret_cast<V2 *>(fout + (size_t)i * P.ncell + n) =
        Narrow<S>::two(a[i] * real(kscale<S>(i)), b[i] * real(kscale<S>(i)));
}

// K1: fused stream-collide of every fluid node with the uniform body force only (FORCE: the
// body force is non-zero). The nodes of active interface tiles are collided again by K1t with
// their interface force, so this pass does not wait for the interface chain of the step.
// Each thread owns the two nodes (x0, x0 + 1), x0 even: populations that do not move along x
// and every store are one aligned 2-wide access, and the address arithmetic is shared.
// With ROWS each block covers blockDim.y lattice rows (small lattices); without, one row
// (kept as its own instance: the row arithmetic costs the single-row kernel registers).
template <typename real, typename S, bool FIRST, bool FORCE, bool ROWS>
__global__ void __launch_bounds__(128) stream_collide_kernel(const S *__restrict__ fin,
                                                             S *__restrict__ fout,
                                                             const LatParams<real> P, int z0) {
  const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = ROWS ? blockIdx.y * blockDim.y + threadIdx.y : blockIdx.y;
  const int z = blockIdx.z + z0;
  if (x0 >= P.nx) return;
  real a[Q], b[Q];  // populations of nodes x0 and x0 + 1
  load_pair<real, S, FIRST>(fin, P, x0, y, z, a, b);
  const real F[3] = {P.g[0], P.g[1], P.g[2]};
  collide<real, FORCE>(a, F, P);
  collide<real, FORCE>(b, F, P);
  store_pair(fout, P, (size_t)z * P.nx * P.ny + (size_t)y * P.nx + x0, a, b);
}

// Two-wide FP32 arithmetic (one packed instruction per operation on sm_100 and later):
// lane x belongs to the first node of a pair, lane y to the second.
__device__ __forceinline__ float2 dup(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, dup(-1.0f), a); }

// BGK collision with Guo forcing (Eqs. 9-10) of a node pair held in the scaled storage units
// of a 16-bit type, g_i = (f_i - w_i rho0) K / w_i. The moments weigh g_i by w_i / K, and the
// update is the one of `collide` multiplied through by k_i = K / w_i, where the weights cancel:
//   g*_i = g_i + omega (K [drho + rho (4.5 (c.u)^2 - 1.5 u^2) +- 3 rho (c.u)] - g_i)
//          + K (1 - 1/2tau) [9 (c.F)(c.u) - 3 u.F +- 3 (c.F)]
// (F uniform over the pair). rho is rounded once here: the storage rounding of the 16-bit
// types is four orders of magnitude above it.
template <bool FORCE>
__device__ __forceinline__ void collide_pair_scaled(float2 g[Q], const float F[3],
                                                    const LatParams<float> &P, float K) {
  const float iK = 1.0f / K;
  float2 drho = mul2(g[0], dup(float(wgt(0)) * iK));
  float2 jx = dup(0.0f), jy = dup(0.0f), jz = dup(0.0f);
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const float2 w = dup(float(wgt(i)) * iK);
    drho = fma2(add2(g[i], g[i + 1]), w, drho);
    const float2 d = mul2(sub2(g[i], g[i + 1]), w);
    if (cx(i)) jx = cx(i) > 0 ? add2(jx, d) : sub2(jx, d);
    if (cy(i)) jy = cy(i) > 0 ? add2(jy, d) : sub2(jy, d);
    if (cz(i)) jz = cz(i) > 0 ? add2(jz, d) : sub2(jz, d);
  }
  const float2 rho = add2(dup(P.rho0), drho);
  const float2 inv_rho = make_float2(__frcp_rn(rho.x), __frcp_rn(rho.y));
  float2 ux = jx, uy = jy, uz = jz;
  if (FORCE) {
    ux = fma2(dup(0.5f), dup(F[0]), ux);
    uy = fma2(dup(0.5f), dup(F[1]), uy);
    uz = fma2(dup(0.5f), dup(F[2]), uz);
  }
  ux = mul2(ux, inv_rho);
  uy = mul2(uy, inv_rho);
  uz = mul2(uz, inv_rho);
  const float2 uu15 = mul2(dup(1.5f), fma2(ux, ux, fma2(uy, uy, mul2(uz, uz))));
  const float2 om = dup(P.omega), omc = dup(1.0f - P.omega);
  const float2 Kdrho = mul2(dup(K), drho), Krho = mul2(dup(K), rho);
  const float2 Krho3 = mul2(dup(3.0f), Krho);
  float2 KuF3 = dup(0.0f);
  const float Kguo = K * P.guo;
  if (FORCE)
    KuF3 = mul2(dup(3.0f * Kguo),
                fma2(ux, dup(F[0]), fma2(uy, dup(F[1]), mul2(uz, dup(F[2])))));
  {  // rest population: g*_0 = (1 - omega) g_0 + omega K (drho - rho 1.5 u^2) - K guo 3 u.F
    const float2 feq = sub2(Kdrho, mul2(Krho, uu15));
    float2 out = fma2(omc, g[0], mul2(om, feq));
    if (FORCE) out = sub2(out, KuF3);
    g[0] = out;
  }
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    float2 cu = dup(0.0f);
    if (cx(i)) cu = cx(i) > 0 ? add2(cu, ux) : sub2(cu, ux);
    if (cy(i)) cu = cy(i) > 0 ? add2(cu, uy) : sub2(cu, uy);
    if (cz(i)) cu = cz(i) > 0 ? add2(cu, uz) : sub2(cu, uz);
    const float2 xs = fma2(mul2(dup(4.5f), cu), cu, mul2(dup(-1.0f), uu15));
    const float2 sym = fma2(Krho, xs, Kdrho);
    const float2 asym = mul2(Krho3, cu);
    float2 a = fma2(omc, g[i], mul2(om, add2(sym, asym)));
    float2 b = fma2(omc, g[i + 1], mul2(om, sub2(sym, asym)));
    if (FORCE) {
      const float cF = cx(i) * F[0] + cy(i) * F[1] + cz(i) * F[2];
      const float2 ssym = sub2(mul2(dup(9.0f * Kguo * cF), cu), KuF3);
      const float2 sasym = dup(3.0f * Kguo * cF);
      a = add2(a, add2(ssym, sasym));
      b = add2(b, sub2(ssym, sasym));
    }
    g[i] = a;
    g[i + 1] = b;
  }
}

template <typename V2>
__device__ __forceinline__ float2 widen_pair(V2 v);
template <>
__device__ __forceinline__ float2 widen_pair(__half2 v) { return __half22float2(v); }
template <>
__device__ __forceinline__ float2 widen_pair(__nv_bfloat162 v) { return __bfloat1622float2(v); }
template <typename V2>
__device__ __forceinline__ V2 narrow_pair(float2 v);
template <>
__device__ __forceinline__ __half2 narrow_pair(float2 v) { return __float22half2_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat162 narrow_pair(float2 v) { return __float22bfloat162_rn(v); }

// Reinterpret 32 bits as a pair of 16-bit storage values, and back.
template <typename V2>
__device__ __forceinline__ V2 as_pair(unsigned int u) {
  V2 v;
  memcpy(&v, &u, sizeof(v));
  return v;
}
template <typename V2>
__device__ __forceinline__ unsigned int as_bits(V2 v) {
  unsigned int u;
  memcpy(&u, &v, sizeof(u));
  return u;
}

// K1 for 16-bit storage: each thread owns four nodes x0 .. x0 + 3 (x0 a multiple of 4), so
// every population row is one aligned 8-byte load (plus one 2-byte load of the neighbouring
// node for the directions that move along x) and every store one 8-byte store: half the
// memory instructions of the two-node form and twice the bytes in flight per thread, which a
// 2-byte type needs to keep HBM busy. The loaded rows stay packed in registers (`lo` holds
// nodes x0, x0 + 1, `hi` nodes x0 + 2, x0 + 3) and are widened one node pair at a time for
// the collision; the results are packed back in place.
template <typename S, bool FIRST, bool FORCE>
__device__ __forceinline__ void quad_nodes(const S *__restrict__ fin, S *__restrict__ fout,
                                           const LatParams<float> &P, int x0, int y, int z) {
  using V2 = typename Storage<S>::V2;
  const size_t plane = (size_t)P.nx * P.ny;
  const size_t n = (size_t)z * plane + (size_t)y * P.nx + x0;
  unsigned int lo[Q], hi[Q];  // packed pairs (x0, x0 + 1) and (x0 + 2, x0 + 3)
  bool bounced[Q];            // population i comes from the wall: add the wall term
  if (FIRST) {
#pragma unroll
    for (int i = 0; i < Q; i++) {
      const uint2 v = *reinterpret_cast<const uint2 *>(fin + (size_t)i * P.ncell + n);
      lo[i] = v.x;
      hi[i] = v.y;
      bounced[i] = false;
    }
  } else {
    const int xm = x0 == 0 ? P.nx - 1 : x0 - 1;   // source of node x0 for c_x = +1
    const int xp = x0 + 4 == P.nx ? 0 : x0 + 4;   // source of node x0 + 3 for c_x = -1
    const int ym = y == 0 ? P.ny - 1 : y - 1, yp = y == P.ny - 1 ? 0 : y + 1;
    int zm = z - 1, zp = z + 1;
    if (!P.has_walls) {
      zm = z == 0 ? P.nz - 1 : zm;
      zp = z == P.nz - 1 ? 0 : zp;
    }
    const bool wall_below = P.has_walls && zm == 0;
    const bool wall_above = P.has_walls && zp == P.nz - 1;
    const size_t zo[3] = {(size_t)zm * plane, (size_t)z * plane, (size_t)zp * plane};
    const size_t yo[3] = {(size_t)ym * P.nx, (size_t)y * P.nx, (size_t)yp * P.nx};
#pragma unroll
    for (int i = 0; i < Q; i++) {
      bounced[i] = (cz(i) > 0 && wall_below) || (cz(i) < 0 && wall_above);
      if (bounced[i]) {
        const uint2 v = *reinterpret_cast<const uint2 *>(fin + (size_t)opp(i) * P.ncell + n);
        lo[i] = v.x;
        hi[i] = v.y;
        continue;
      }
      const S *row = fin + (size_t)i * P.ncell + zo[1 - cz(i)] + yo[1 - cy(i)];
      const uint2 v = *reinterpret_cast<const uint2 *>(row + x0);  // nodes x0 .. x0 + 3
      if (cx(i) == 0) {
        lo[i] = v.x;
        hi[i] = v.y;
      } else if (cx(i) > 0) {  // sources x0 - 1 .. x0 + 2
        const unsigned int e = *reinterpret_cast<const unsigned short *>(row + xm);
        lo[i] = __byte_perm(e, v.x, 0x5410);
        hi[i] = __byte_perm(v.x, v.y, 0x5432);
      } else {  // sources x0 + 1 .. x0 + 4
        const unsigned int e = *reinterpret_cast<const unsigned short *>(row + xp);
        lo[i] = __byte_perm(v.x, v.y, 0x5432);
        hi[i] = __byte_perm(v.y, e, 0x5432);
      }
    }
  }
  const float F[3] = {P.g[0], P.g[1], P.g[2]};
#pragma unroll
  for (int h = 0; h < 2; h++) {  // node pairs (x0, x0 + 1), (x0 + 2, x0 + 3)
    unsigned int *pk = h ? hi : lo;
    float2 g[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
      g[i] = widen_pair(as_pair<V2>(pk[i]));
      if (bounced[i]) {  // stored units: the wall term times k_i
        const float wall = (cz(i) > 0 ? P.wb[i] : P.wt[i]) * float(kscale<S>(i));
        g[i] = add2(g[i], dup(wall));
      }
    }
    collide_pair_scaled<FORCE>(g, F, P, float(Storage<S>::K));
#pragma unroll
    for (int i = 0; i < Q; i++) pk[i] = as_bits(narrow_pair<V2>(g[i]));
  }
#pragma unroll
  for (int i = 0; i < Q; i++)
    *reinterpret_cast<uint2 *>(fout + (size_t)i * P.ncell + n) = make_uint2(lo[i], hi[i]);
}

template <typename S, bool FIRST, bool FORCE>
__global__ void __launch_bounds__(128) stream_collide_quad_kernel(const S *__restrict__ fin,
                                                                  S *__restrict__ fout,
                                                                  const LatParams<float> P,
                                                                  int z0) {
  const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;  // blockDim.y rows per block
  const int z = blockIdx.z + z0;
  if (x0 >= P.nx) return;
  quad_nodes<S, FIRST, FORCE>(fin, fout, P, x0, y, z);
}

// --- K1s: stream-collide with the pulled rows staged in shared memory by bulk copies ----------
//
// A unit of work is R lattice rows (y0 .. y0 + R - 1 at one z). The pulled populations of a
// unit are whole x-rows of the population array: population i of row (y, z) streams from row
// (y - c_iy, z - c_iz), or, for a link from a wall node, is population opp(i) of row (y, z)
// itself. A producer warp copies those 19 R rows into a shared-memory stage with cp.async.bulk,
// their completion counted in bytes on the stage's `full` mbarrier; NC compute warps read the
// nodes from the stage (the periodic x wrap is an index into the row), collide them and store
// the results straight to global memory, then release the stage on its `empty` mbarrier. D
// stages rotate, so the bytes in flight per SM are set by shared memory, not by registers.
// Every wait is bounded: a wait that gives up records H_TIMEOUT in the health word and the
// block returns once the producer has waited (again bounded) for its own copies in flight.

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Non-blocking test for the completion of the phase of parity `parity`.
__device__ __forceinline__ bool mbar_test_wait(unsigned long long *bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
constexpr unsigned long long kDrainWaitNs = 1000000000ull;  // the wait for copies in flight
constexpr int kStageWaitPolls = 1 << 26;                     // polls before any wait gives up
// Wait for the completion of the phase of parity `parity`; false if the wait gave up (after
// limit_ns nanoseconds of the global timer) or another warp of the block raised `abort_flag`
// meanwhile. limit_ns = 0: one non-blocking test.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity,
                                          const volatile int *abort_flag,
                                          unsigned long long limit_ns) {
  if (limit_ns == 0) return mbar_test_wait(bar, parity);
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (int k = 0; k < kStageWaitPolls; k++) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag || global_ns() - t0 > limit_ns) return false;
  }
  return false;
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from global to
// shared memory, completing `bytes` transactions on mbarrier `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Shape of the staged pass: units of R rows, D stages of R * 19 rows of nx values each.
struct StageGeom {
  int z0;            // first fluid layer
  int units_per_z;   // ny / R
  int nunits;        // units_per_z * fluid layers
  int R, D;
  int stage_elems;   // R * 19 * nx
  unsigned long long wait_ns;  // limit of a wait for a stage or for a free stage
};

// Bytes ahead of the first stage: the 2 D mbarriers and the abort flag.
constexpr int kStageHeader = 256;

// Row (z, wall flags) of a unit. Links from a wall exist only on the first and last fluid
// layer, and they are the same for every row of the unit.
struct UnitRows {
  int z, y0, zm, zp;
  bool wall_below, wall_above;
};
template <typename real>
__device__ __forceinline__ UnitRows unit_rows(int unit, const LatParams<real> &P,
                                              const StageGeom &G) {
  UnitRows u;
  u.z = G.z0 + unit / G.units_per_z;
  u.y0 = (unit % G.units_per_z) * G.R;
  u.zm = u.z - 1;
  u.zp = u.z + 1;
  if (!P.has_walls) {
    u.zm = u.z == 0 ? P.nz - 1 : u.zm;
    u.zp = u.z == P.nz - 1 ? 0 : u.zp;
  }
  u.wall_below = P.has_walls && u.zm == 0;
  u.wall_above = P.has_walls && u.zp == P.nz - 1;
  return u;
}

// Signs of c_iy and c_iz as bit masks over i, for run-time direction indices.
__host__ __device__ constexpr unsigned dir_mask(int axis, int sign) {
  unsigned m = 0;
  for (int i = 0; i < Q; i++) {
    const int c = axis == 1 ? cy(i) : cz(i);
    if (c == sign) m |= 1u << i;
  }
  return m;
}
constexpr unsigned kYPos = dir_mask(1, 1), kYNeg = dir_mask(1, -1);
constexpr unsigned kZPos = dir_mask(2, 1), kZNeg = dir_mask(2, -1);
__device__ __forceinline__ int dir_c(unsigned pos, unsigned neg, int i) {
  return (int)((pos >> i) & 1u) - (int)((neg >> i) & 1u);
}

// Producer lanes: queue the copies of `unit` into `stage` (lane 0 has armed `full` with the
// byte count). The stage holds [19][R][nx] values: block i is population i of lattice rows
// y0 .. y0 + R - 1 as pulled, or population opp(i) of those rows for a link from the wall. The
// R source rows of a population are consecutive rows of one plane, so one copy brings them,
// or two where they wrap around y.
template <typename S>
__device__ __forceinline__ void stage_issue(const S *__restrict__ fin, S *stage,
                                            unsigned long long *full, const UnitRows &u,
                                            const LatParams<float> &P, const StageGeom &G,
                                            int lane) {
  if (lane >= Q) return;
  const int i = lane;
  const unsigned row_bytes = (unsigned)(P.nx * sizeof(S));
  const size_t plane = (size_t)P.nx * P.ny;
  const int ciy = dir_c(kYPos, kYNeg, i);
  const int ciz = dir_c(kZPos, kZNeg, i);
  S *dst = stage + (size_t)i * G.R * P.nx;
  if ((ciz > 0 && u.wall_below) || (ciz < 0 && u.wall_above)) {
    const size_t src = (size_t)opp(i) * P.ncell + (size_t)u.z * plane + (size_t)u.y0 * P.nx;
    bulk_g2s(dst, fin + src, G.R * row_bytes, full);
    return;
  }
  const int zs = ciz > 0 ? u.zm : (ciz < 0 ? u.zp : u.z);
  const S *pop = fin + (size_t)i * P.ncell + (size_t)zs * plane;
  const int ys = u.y0 - ciy;  // source of row y0; rows ys .. ys + R - 1 follow (mod ny)
  if (ys < 0) {               // row y0 = 0 pulls from row ny - 1
    bulk_g2s(dst, pop + (size_t)(P.ny - 1) * P.nx, row_bytes, full);
    if (G.R > 1) bulk_g2s(dst + P.nx, pop, (G.R - 1) * row_bytes, full);
  } else if (ys + G.R > P.ny) {  // the last row of the unit pulls from row 0
    if (G.R > 1) bulk_g2s(dst, pop + (size_t)ys * P.nx, (G.R - 1) * row_bytes, full);
    bulk_g2s(dst + (size_t)(G.R - 1) * P.nx, pop, row_bytes, full);
  } else {
    bulk_g2s(dst, pop + (size_t)ys * P.nx, G.R * row_bytes, full);
  }
}

// Compute lanes, FP32 storage: the node pair (x0, x0 + 1) of one lattice row, whose pulled
// population i is the stage row rows + i * stride, collided and stored at node n of fout.
template <bool FORCE>
__device__ __forceinline__ void staged_pair(const float *rows, int stride, int x0,
                                            const UnitRows &u, const LatParams<float> &P,
                                            float *__restrict__ fout, size_t n) {
  const int xm = x0 == 0 ? P.nx - 1 : x0 - 1;  // source of node x0 for c_x = +1
  const int xp = x0 + 2 == P.nx ? 0 : x0 + 2;  // source of node x0 + 1 for c_x = -1
  float a[Q], b[Q];
#pragma unroll
  for (int i = 0; i < Q; i++) {
    const float *row = rows + i * stride;
    if ((cz(i) > 0 && u.wall_below) || (cz(i) < 0 && u.wall_above)) {
      const float2 v = *reinterpret_cast<const float2 *>(row + x0);
      const float wall = cz(i) > 0 ? P.wb[i] : P.wt[i];
      a[i] = v.x + wall;
      b[i] = v.y + wall;
    } else if (cx(i) == 0) {
      const float2 v = *reinterpret_cast<const float2 *>(row + x0);
      a[i] = v.x;
      b[i] = v.y;
    } else if (cx(i) > 0) {
      a[i] = row[xm];
      b[i] = row[x0];
    } else {
      a[i] = row[x0 + 1];
      b[i] = row[xp];
    }
  }
  const float F[3] = {P.g[0], P.g[1], P.g[2]};
  collide<float, FORCE>(a, F, P);
  collide<float, FORCE>(b, F, P);
  store_pair(fout, P, n, a, b);
}

// Compute lanes, 16-bit storage: the four nodes x0 .. x0 + 3 (as in K1's 16-bit form, with
// the rows read from the stage).
template <typename S, bool FORCE>
__device__ __forceinline__ void staged_quad(const S *rows, int stride, int x0, const UnitRows &u,
                                            const LatParams<float> &P, S *__restrict__ fout,
                                            size_t n) {
  using V2 = typename Storage<S>::V2;
  const int xm = x0 == 0 ? P.nx - 1 : x0 - 1;  // source of node x0 for c_x = +1
  const int xp = x0 + 4 == P.nx ? 0 : x0 + 4;  // source of node x0 + 3 for c_x = -1
  unsigned int lo[Q], hi[Q];
#pragma unroll
  for (int i = 0; i < Q; i++) {
    const S *row = rows + i * stride;
    const uint2 v = *reinterpret_cast<const uint2 *>(row + x0);
    const bool bounced = (cz(i) > 0 && u.wall_below) || (cz(i) < 0 && u.wall_above);
    if (bounced || cx(i) == 0) {
      lo[i] = v.x;
      hi[i] = v.y;
    } else if (cx(i) > 0) {  // sources x0 - 1 .. x0 + 2
      const unsigned int e = *reinterpret_cast<const unsigned short *>(row + xm);
      lo[i] = __byte_perm(e, v.x, 0x5410);
      hi[i] = __byte_perm(v.x, v.y, 0x5432);
    } else {  // sources x0 + 1 .. x0 + 4
      const unsigned int e = *reinterpret_cast<const unsigned short *>(row + xp);
      lo[i] = __byte_perm(v.x, v.y, 0x5432);
      hi[i] = __byte_perm(v.y, e, 0x5432);
    }
  }
  const float F[3] = {P.g[0], P.g[1], P.g[2]};
#pragma unroll
  for (int h = 0; h < 2; h++) {  // node pairs (x0, x0 + 1), (x0 + 2, x0 + 3)
    unsigned int *pk = h ? hi : lo;
    float2 g[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
      g[i] = widen_pair(as_pair<V2>(pk[i]));
      if ((cz(i) > 0 && u.wall_below) || (cz(i) < 0 && u.wall_above)) {
        const float wall = (cz(i) > 0 ? P.wb[i] : P.wt[i]) * float(kscale<S>(i));
        g[i] = add2(g[i], dup(wall));
      }
    }
    collide_pair_scaled<FORCE>(g, F, P, float(Storage<S>::K));
#pragma unroll
    for (int i = 0; i < Q; i++) pk[i] = as_bits(narrow_pair<V2>(g[i]));
  }
#pragma unroll
  for (int i = 0; i < Q; i++)
    *reinterpret_cast<uint2 *>(fout + (size_t)i * P.ncell + n) = make_uint2(lo[i], hi[i]);
}

// Compute lanes, 16-bit storage, two nodes x0, x0 + 1 (x0 even): one 4-byte word per row,
// plus the neighbouring 2-byte value for the directions that move along x; the node pair is
// collided exactly as each pair of the four-node form.
template <typename S, bool FORCE>
__device__ __forceinline__ void staged_pair16(const S *rows, int stride, int x0, const UnitRows &u,
                                              const LatParams<float> &P, S *__restrict__ fout,
                                              size_t n) {
  using V2 = typename Storage<S>::V2;
  const int xm = x0 == 0 ? P.nx - 1 : x0 - 1;  // source of node x0 for c_x = +1
  const int xp = x0 + 2 == P.nx ? 0 : x0 + 2;  // source of node x0 + 1 for c_x = -1
  float2 g[Q];
#pragma unroll
  for (int i = 0; i < Q; i++) {
    const S *row = rows + i * stride;
    const unsigned int w = *reinterpret_cast<const unsigned int *>(row + x0);
    const bool bounced = (cz(i) > 0 && u.wall_below) || (cz(i) < 0 && u.wall_above);
    unsigned int pr;
    if (bounced || cx(i) == 0) {
      pr = w;
    } else if (cx(i) > 0) {  // sources x0 - 1, x0
      const unsigned int e = *reinterpret_cast<const unsigned short *>(row + xm);
      pr = __byte_perm(e, w, 0x5410);
    } else {  // sources x0 + 1, x0 + 2
      const unsigned int e = *reinterpret_cast<const unsigned short *>(row + xp);
      pr = __byte_perm(w, e, 0x5432);
    }
    g[i] = widen_pair(as_pair<V2>(pr));
    if (bounced) {  // stored units: the wall term times k_i
      const float wall = (cz(i) > 0 ? P.wb[i] : P.wt[i]) * float(kscale<S>(i));
      g[i] = add2(g[i], dup(wall));
    }
  }
  const float F[3] = {P.g[0], P.g[1], P.g[2]};
  collide_pair_scaled<FORCE>(g, F, P, float(Storage<S>::K));
#pragma unroll
  for (int i = 0; i < Q; i++)
    *reinterpret_cast<unsigned int *>(fout + (size_t)i * P.ncell + n) = as_bits(narrow_pair<V2>(g[i]));
}

// Launch bound of the staged kernel: 8 compute warps and the copying warp with four nodes per
// lane (the four-node form needs ~170 registers), 16 + 1 warps with two.
__host__ __device__ constexpr int staged_threads(int npt) { return npt == 4 ? 288 : 544; }

// K1s: persistent staged stream-collide (not the first step of a run). blockDim.x = 32 (NC + 1)
// (NC <= 8 with NPT = 4, <= 16 with NPT = 2): warps 0 .. NC-1 compute, warp NC produces. Block
// b takes units b, b + gridDim.x, ... NPT nodes per compute lane: 2 for FP32, 2 or 4 for 16-bit
// storage.
template <typename S, bool FORCE, int NPT>
__global__ void __launch_bounds__(staged_threads(NPT), 1) stream_collide_staged_kernel(
    const S *__restrict__ fin, S *__restrict__ fout, const LatParams<float> P,
    const StageGeom G, int *__restrict__ health) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned long long *full = reinterpret_cast<unsigned long long *>(smem);
  unsigned long long *empty = full + G.D;
  volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + G.D);
  S *stages = reinterpret_cast<S *>(smem + kStageHeader);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int NC = (blockDim.x >> 5) - 1;
  if (threadIdx.x == 0) {
    for (int s = 0; s < G.D; s++) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, NC);
    }
    *abort_flag = 0;
    fence_barrier_init();
  }
  __syncthreads();
  const int my_units = G.nunits > (int)blockIdx.x
                           ? (G.nunits - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x
                           : 0;
  if (warp == NC) {  // producer
    int issued = 0;
    for (int k = 0; k < my_units; k++) {
      const int s = k % G.D;
      if (k >= G.D) {  // stage s is free once every compute warp released unit k - D
        bool ok = true;
        if (lane == 0) ok = mbar_wait(empty + s, ((k / G.D) - 1) & 1, abort_flag, G.wait_ns);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          if (lane == 0) {
            *abort_flag = 1;
            atomicOr(health, H_TIMEOUT);
          }
          break;
        }
      }
      const UnitRows u = unit_rows(blockIdx.x + k * gridDim.x, P, G);
      S *stage = stages + (size_t)s * G.stage_elems;
      if (lane == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(full + s, (unsigned)(G.R * Q * P.nx * sizeof(S)));
      }
      __syncwarp();
      stage_issue(fin, stage, full + s, u, P, G, lane);
      issued = k + 1;
    }
    // copies still in flight land before the block exits: those of the last D units issued
    // (a unit before them was waited for by every compute warp before its stage was reused)
    if (lane == 0) {
      const int no_abort = 0;
      for (int k = issued - G.D < 0 ? 0 : issued - G.D; k < issued; k++)
        if (!mbar_wait(full + k % G.D, (k / G.D) & 1, &no_abort, kDrainWaitNs))
          atomicOr(health, H_TIMEOUT);
    }
    return;
  }
  // compute warps
  const int per_row = P.nx / NPT;
  const size_t plane = (size_t)P.nx * P.ny;
  for (int k = 0; k < my_units; k++) {
    const int s = k % G.D;
    if (!__all_sync(0xffffffffu, mbar_wait(full + s, (k / G.D) & 1, abort_flag, G.wait_ns))) {
      if (lane == 0) {
        *abort_flag = 1;
        atomicOr(health, H_TIMEOUT);
      }
      return;
    }
    const UnitRows u = unit_rows(blockIdx.x + k * gridDim.x, P, G);
    const S *stage = stages + (size_t)s * G.stage_elems;
    for (int w = warp * 32 + lane; w < G.R * per_row; w += NC * 32) {
      const int r = w / per_row, x0 = NPT * (w - r * per_row);
      const size_t n = (size_t)u.z * plane + (size_t)(u.y0 + r) * P.nx + x0;
      if constexpr (sizeof(S) == 2 && NPT == 4)
        staged_quad<S, FORCE>(stage + (size_t)r * P.nx, G.R * P.nx, x0, u, P, fout, n);
      else if constexpr (sizeof(S) == 2)
        staged_pair16<S, FORCE>(stage + (size_t)r * P.nx, G.R * P.nx, x0, u, P, fout, n);
      else
        staged_pair<FORCE>(stage + (size_t)r * P.nx, G.R * P.nx, x0, u, P, fout, n);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(empty + s);
  }
}

// K1 over many contexts in one launch (the batched ensemble; never the first, in-place step):
// each thread takes one node group in memory order, a pair (x0, x0 + 1) or, with 16-bit
// storage, four nodes x0 .. x0 + 3, and runs the very code of the single-context kernels on it,
// so each context's populations come out bit for bit as from those.
template <typename real, typename S>
struct StreamArgs {
  const S *fin;
  S *fout;
  LatParams<real> P;
  int z0;       // first fluid layer
  int per_row;  // node groups per lattice row
  int ngroups;  // node groups of the context
  int force;    // the body force is non-zero
};

// Blocks per SM the batched pass is compiled for: 6 (80 registers) for FP32, where it keeps
// the occupancy it has without the velocity correction (93 registers otherwise); no bound for
// the others, which would spill under it.
// Blocks per SM of the batched pass, run as a persistent grid over its blocks (0: one launch
// block per 128 node groups). A pass that does not fill the SMs leaves room for the interface
// kernels of the other stream, which then run beside it instead of after it (96 wetting
// boxes: 1.317 ms per step with 4, 1.322 with 3, 1.402 with 6, 1.425 with 2, against 1.342
// ms with a block per 128 node groups).
constexpr int kK1MultiPerSM = 4;

template <typename real, typename S>
struct MultiMinBlocks {
  static constexpr int value =
      sizeof(real) == 4 && sizeof(S) == 4 ? (kK1MultiPerSM > 0 ? kK1MultiPerSM : 6) : 1;
};

template <typename real, typename S>
__global__ void __launch_bounds__(128, MultiMinBlocks<real, S>::value) stream_collide_kernel_multi(
    const StreamArgs<real, S> *__restrict__ all, const int *__restrict__ start, int n) {
  __shared__ int s_start[kMultiMax + 1];
  for (int k = threadIdx.x; k <= n; k += blockDim.x) s_start[k] = start[k];
  __syncthreads();
  const int total = s_start[n];
  for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
  const MultiBlock m = multi_block_of(s_start, n, vb);
  const StreamArgs<real, S> &A = all[m.inst];
  const int g = m.block * blockDim.x + threadIdx.x;
  if (g >= A.ngroups) continue;
  const int row = g / A.per_row;
  const int y = row % A.P.ny, z = A.z0 + row / A.P.ny;
  if constexpr (sizeof(S) == 2) {
    const int x0 = 4 * (g - row * A.per_row);
    if (A.force) quad_nodes<S, false, true>(A.fin, A.fout, A.P, x0, y, z);
    else quad_nodes<S, false, false>(A.fin, A.fout, A.P, x0, y, z);
  } else {
    const int x0 = 2 * (g - row * A.per_row);
    real a[Q], b[Q];
    load_pair<real, S, false>(A.fin, A.P, x0, y, z, a, b);
    const real F[3] = {A.P.g[0], A.P.g[1], A.P.g[2]};
    if (A.force) {
      collide<real, true>(a, F, A.P);
      collide<real, true>(b, F, A.P);
    } else {
      collide<real, false>(a, F, A.P);
      collide<real, false>(b, F, A.P);
    }
    store_pair(A.fout, A.P, (size_t)z * A.P.nx * A.P.ny + (size_t)y * A.P.nx + x0, a, b);
  }
  }
}

// K1t: the fluid nodes of the active tiles with body + interface force. Runs after K1 of the
// same step and corrects K1's result there in place. The collision (BGK with Guo forcing,
// Eqs. 9-10) keeps rho and turns the momentum j into j + Ft (Ft the total force), so K1's
// output f0 at a node (the collision with the body force g alone) gives rho = rho0 + sum f0
// and u0 = (sum c f0 - g/2)/rho without the pre-collision populations; with the interface
// force F the post-collision populations are f0 + D,
//   D_i = omega (f^eq_i(rho, uF) - f^eq_i(rho, u0)) + S_i(uF, g + F) - S_i(u0, g),
//   uF = u0 + F/(2 rho).
// K1t therefore reads and writes only each node's own populations, no pulled neighbours.
// Its work list is the node pairs (x0, x0 + 1), x0 even, that hold a node of some vertex's
// stencil, appended by the spreading's gather pass (K4b) as slot * 32 + pair; one thread per
// listed pair. Pairs without force keep K1's result, which is already final.
template <typename real, typename S>
struct TilesArgs {
  S *fout;
  const int *slot_tile, *pair_list, *npairs_ptr;
  const Vec4<real> *Fslot;
  LatParams<real> P;
  int max_pairs;
};

// f (deviations, after the collision with the body force g alone) becomes the collision
// with g + F; see K1t above. D is a quadratic form in the lattice vector: for a direction i
// and its opposite,
//   D_i = w_i (c_i^T M c_i + q0 + c_i . v),   D_opp(i) = w_i (c_i^T M c_i + q0 - c_i . v),
//   M = 9/4 omega rho (dl s^T + s dl^T) + 9/2 gamma (Ft uF^T + uF Ft^T - g u0^T - u0 g^T),
//   v = 3 (omega rho dl + gamma F),  dl = uF - u0,  s = uF + u0,  Ft = g + F,
// so a node needs ten numbers (M's diagonal, twice its off-diagonal, q0, v) once its
// moments are known, and each direction a few adds.
template <typename real>
struct Correction {
  real dx, dy, dz;     // M_aa
  real oxy, oxz, oyz;  // 2 M_ab
  real q0;             // -1.5 omega rho (uF^2 - u0^2) - 3 gamma (uF.Ft - u0.g)
  real vx, vy, vz;
};

// Moments of K1's output at one node: drho = sum f, J = sum c f (deviations).
template <typename real>
struct Moments {
  real drho = 0, Jx = 0, Jy = 0, Jz = 0;
  __device__ __forceinline__ void add(int i, real f) {
    drho += f;
    if (cx(i)) Jx += cx(i) > 0 ? f : -f;
    if (cy(i)) Jy += cy(i) > 0 ? f : -f;
    if (cz(i)) Jz += cz(i) > 0 ? f : -f;
  }
};

template <typename real>
__device__ __forceinline__ Correction<real> correction_of(const Moments<real> &m, const real F[3],
                                                         const LatParams<real> &P) {
  const real drho = m.drho, Jx = m.Jx, Jy = m.Jy, Jz = m.Jz;
  const real rho = P.rho0 + drho;
  const real ir = real(1) / rho;
  const real u0[3] = {(Jx - real(0.5) * P.g[0]) * ir, (Jy - real(0.5) * P.g[1]) * ir,
                      (Jz - real(0.5) * P.g[2]) * ir};
  const real dl[3] = {real(0.5) * F[0] * ir, real(0.5) * F[1] * ir, real(0.5) * F[2] * ir};
  const real uF[3] = {u0[0] + dl[0], u0[1] + dl[1], u0[2] + dl[2]};
  const real sm[3] = {uF[0] + u0[0], uF[1] + u0[1], uF[2] + u0[2]};
  const real Ft[3] = {P.g[0] + F[0], P.g[1] + F[1], P.g[2] + F[2]};
  const real a = real(4.5) * P.omega * rho, b = real(9) * P.guo;
  Correction<real> k;
  k.q0 = real(-1.5) * P.omega * rho * (dl[0] * sm[0] + dl[1] * sm[1] + dl[2] * sm[2]) -
         real(3) * P.guo *
             ((uF[0] * Ft[0] + uF[1] * Ft[1] + uF[2] * Ft[2]) -
              (u0[0] * P.g[0] + u0[1] * P.g[1] + u0[2] * P.g[2]));
  k.dx = a * dl[0] * sm[0] + b * (Ft[0] * uF[0] - P.g[0] * u0[0]);
  k.dy = a * dl[1] * sm[1] + b * (Ft[1] * uF[1] - P.g[1] * u0[1]);
  k.dz = a * dl[2] * sm[2] + b * (Ft[2] * uF[2] - P.g[2] * u0[2]);
  k.oxy = a * (dl[0] * sm[1] + dl[1] * sm[0]) +
          b * (Ft[0] * uF[1] + Ft[1] * uF[0] - P.g[0] * u0[1] - P.g[1] * u0[0]);
  k.oxz = a * (dl[0] * sm[2] + dl[2] * sm[0]) +
          b * (Ft[0] * uF[2] + Ft[2] * uF[0] - P.g[0] * u0[2] - P.g[2] * u0[0]);
  k.oyz = a * (dl[1] * sm[2] + dl[2] * sm[1]) +
          b * (Ft[1] * uF[2] + Ft[2] * uF[1] - P.g[1] * u0[2] - P.g[2] * u0[1]);
  const real oa = P.omega * rho;
  k.vx = real(3) * (oa * dl[0] + P.guo * F[0]);
  k.vy = real(3) * (oa * dl[1] + P.guo * F[1]);
  k.vz = real(3) * (oa * dl[2] + P.guo * F[2]);
  return k;
}

// D_i of one node (i and its opposite share M and v; c_opp = -c_i flips only c_i . v).
template <typename real>
__device__ __forceinline__ real correction_delta(int i, const Correction<real> &k) {
  real quad = k.q0, lin = 0;
  if (cx(i)) { quad += k.dx; lin += cx(i) > 0 ? k.vx : -k.vx; }
  if (cy(i)) { quad += k.dy; lin += cy(i) > 0 ? k.vy : -k.vy; }
  if (cz(i)) { quad += k.dz; lin += cz(i) > 0 ? k.vz : -k.vz; }
  if (cx(i) && cy(i)) quad += cx(i) * cy(i) > 0 ? k.oxy : -k.oxy;
  if (cx(i) && cz(i)) quad += cx(i) * cz(i) > 0 ? k.oxz : -k.oxz;
  if (cy(i) && cz(i)) quad += cy(i) * cz(i) > 0 ? k.oyz : -k.oyz;
  return real(wgt(i)) * (quad + lin);
}

template <typename real, typename S>
__device__ __forceinline__ void tiles_body(const TilesArgs<real, S> &A, int bid, int nb) {
  using V2 = typename Storage<S>::V2;
  S *__restrict__ fout = A.fout;
  const int *__restrict__ slot_tile = A.slot_tile;
  const int *__restrict__ pair_list = A.pair_list;
  const Vec4<real> *__restrict__ Fslot = A.Fslot;
  const LatParams<real> P = A.P;  // held in registers: the loop below is latency-bound
  const int npairs = min(*A.npairs_ptr, A.max_pairs);
  for (int k = bid * blockDim.x + threadIdx.x; k < npairs; k += nb * blockDim.x) {
    const int e = pair_list[k];
    const int s = e >> 5, cell = 2 * (e & 31);  // slot, and the pair's first node in the tile
    const Vec4<real> Fa = Fslot[(size_t)s * TILE_CELLS + cell];
    const Vec4<real> Fb = Fslot[(size_t)s * TILE_CELLS + cell + 1];
    if (Fa.x == real(0) && Fa.y == real(0) && Fa.z == real(0) && Fb.x == real(0) &&
        Fb.y == real(0) && Fb.z == real(0))
      continue;
    const int t = slot_tile[s];
    const int tx = t % P.ntx, ty = (t / P.ntx) % P.nty, tz = t / (P.ntx * P.nty);
    const int x0 = tx * TILE + (cell & 3), y = ty * TILE + ((cell >> 2) & 3);
    const int z = tz * TILE + (cell >> 4);
    if (z >= P.nz || (P.has_walls && (z == 0 || z == P.nz - 1))) continue;
    const size_t n = (size_t)z * P.nx * P.ny + (size_t)y * P.nx + x0;
    real a[Q], b[Q];
    Moments<real> ma, mb;
#pragma unroll
    for (int i = 0; i < Q; i++) {
      widen2(*reinterpret_cast<const V2 *>(fout + (size_t)i * P.ncell + n), a[i], b[i]);
      a[i] *= real(kinv<S>(i));
      b[i] *= real(kinv<S>(i));
      ma.add(i, a[i]);
      mb.add(i, b[i]);
    }
    const real FA[3] = {Fa.x, Fa.y, Fa.z};
    const real FB[3] = {Fb.x, Fb.y, Fb.z};
    const Correction<real> ka = correction_of<real>(ma, FA, P);
    const Correction<real> kb = correction_of<real>(mb, FB, P);
#pragma unroll
    for (int i = 0; i < Q; i++) {
      a[i] += correction_delta<real>(i, ka);
      b[i] += correction_delta<real>(i, kb);
    }
    store_pair(fout, P, n, a, b);
  }
}

template <typename real, typename S>
__global__ void __launch_bounds__(128) stream_collide_tiles_kernel(const TilesArgs<real, S> A) {
  tiles_body<real, S>(A, blockIdx.x, gridDim.x);
}

// the batched form reads its argument record as well: held to 128 registers (4 blocks per SM,
// as the single-context kernel) for float arithmetic
template <typename real>
struct TilesMultiMinBlocks { static constexpr int value = sizeof(real) == 4 ? 4 : 1; };

template <typename real, typename S>
__global__ void __launch_bounds__(128, TilesMultiMinBlocks<real>::value) stream_collide_tiles_kernel_multi(
    const TilesArgs<real, S> *__restrict__ all, const int *__restrict__ start, int n) {
  const MultiBlock m = multi_block(start, n);
  tiles_body<real, S>(all[m.inst], m.block, m.nblocks);
}

// K1b: velocity after streaming at the nodes the interpolation reads: the nodes of the pairs
// that K4b listed (every fluid node of a vertex's stencil, and its pair partner); one thread
// per node of a listed pair. u = (j + (g + F)/2)/rho, the velocity of the forced collision
// (Eq. 10 with Guo's forcing). The wall layers, which the interpolation takes from the wall
// velocities, are never listed.
template <typename real, typename S>
struct ShellArgs {
  const S *fpost;
  const int *slot_tile, *pair_list, *npairs_ptr;
  const Vec4<real> *Fslot;
  Vec4<real> *Uslot;
  LatParams<real> P;
  int max_pairs;
};

template <typename real, typename S>
__device__ __forceinline__ void shell_body(const ShellArgs<real, S> &A, int bid, int nb) {
  const S *__restrict__ fpost = A.fpost;
  const int *__restrict__ slot_tile = A.slot_tile;
  const int *__restrict__ pair_list = A.pair_list;
  const Vec4<real> *__restrict__ Fslot = A.Fslot;
  Vec4<real> *__restrict__ Uslot = A.Uslot;
  const LatParams<real> P = A.P;
  const int nodes = 2 * min(*A.npairs_ptr, A.max_pairs);
  for (int k = bid * blockDim.x + threadIdx.x; k < nodes; k += nb * blockDim.x) {
    const int e = pair_list[k >> 1];
    const int s = e >> 5, cell = 2 * (e & 31) + (k & 1);
    const int t = slot_tile[s];
    const int tx = t % P.ntx, ty = (t / P.ntx) % P.nty, tz = t / (P.ntx * P.nty);
    const int x = tx * TILE + (cell & 3), y = ty * TILE + ((cell >> 2) & 3),
              z = tz * TILE + (cell >> 4);
    if (z >= P.nz || (P.has_walls && (z == 0 || z == P.nz - 1))) continue;
    real f[Q];
    pull<real, S, true>(fpost, P, x, y, z, f);
    real drho = 0, j[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < Q; i++) {
      drho += f[i];
      j[0] += cx(i) * f[i];
      j[1] += cy(i) * f[i];
      j[2] += cz(i) * f[i];
    }
    const Vec4<real> Fs = Fslot[(size_t)s * TILE_CELLS + cell];
    const real Fk[3] = {Fs.x, Fs.y, Fs.z};
    const real rho_hi = P.rho0 + drho;
    const real rho_lo = (P.rho0 - rho_hi) + drho;
    const real r1 = real(1) / rho_hi;
    const real inv_rho = r1 * (real(1) - rho_lo * r1);
    Vec4<real> uv;
    uv.x = (j[0] + real(0.5) * (P.g[0] + Fk[0])) * inv_rho;
    uv.y = (j[1] + real(0.5) * (P.g[1] + Fk[1])) * inv_rho;
    uv.z = (j[2] + real(0.5) * (P.g[2] + Fk[2])) * inv_rho;
    uv.w = real(0);
    Uslot[(size_t)s * TILE_CELLS + cell] = uv;
  }
}

template <typename real, typename S>
__global__ void __launch_bounds__(128) shell_velocity_kernel(const ShellArgs<real, S> A) {
  shell_body<real, S>(A, blockIdx.x, gridDim.x);
}

template <typename real, typename S>
__global__ void __launch_bounds__(128) shell_velocity_kernel_multi(
    const ShellArgs<real, S> *__restrict__ all, const int *__restrict__ start, int n) {
  const MultiBlock m = multi_block(start, n);
  shell_body<real, S>(all[m.inst], m.block, m.nblocks);
}

// rho and u of every node of the current post-streaming state (read-back, not on the step).
template <typename real, typename S>
__global__ void fields_kernel(const S *__restrict__ fstate, int fresh,
                              const int *__restrict__ tile_slot,
                              const Vec4<real> *__restrict__ Fslot,
                              const LatParams<real> P, double3 ub, double3 ut, double rho0,
                              double *__restrict__ rho_out, double *__restrict__ u_out) {
  const size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (n >= P.ncell) return;
  const int x = (int)(n % P.nx), y = (int)((n / P.nx) % P.ny), z = (int)(n / ((size_t)P.nx * P.ny));
  if (P.has_walls && (z == 0 || z == P.nz - 1)) {
    const double3 w = z == 0 ? ub : ut;
    rho_out[n] = rho0;
    u_out[3 * n] = w.x; u_out[3 * n + 1] = w.y; u_out[3 * n + 2] = w.z;
    return;
  }
  real f[Q];
  if (fresh) {
    for (int i = 0; i < Q; i++) f[i] = dev<real>(fstate, i, (size_t)i * P.ncell + n);
  } else {
    pull(fstate, P, x, y, z, f);
  }
  double drho = 0, j[3] = {0, 0, 0};
  for (int i = 0; i < Q; i++) {
    drho += (double)f[i];
    j[0] += cx(i) * (double)f[i];
    j[1] += cy(i) * (double)f[i];
    j[2] += cz(i) * (double)f[i];
  }
  real F[3];
  tile_force(tile_slot, Fslot, P, x, y, z, F);
  const double rho = rho0 + drho;
  rho_out[n] = rho;
  for (int k = 0; k < 3; k++) u_out[3 * n + k] = (j[k] + 0.5 * (double)F[k]) / rho;
}

template <typename real, typename S>
__global__ void populations_kernel(const S *__restrict__ fstate, int fresh,
                                   const LatParams<real> P, double rho0,
                                   double *__restrict__ f_out) {
  const size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (n >= P.ncell) return;
  const int x = (int)(n % P.nx), y = (int)((n / P.nx) % P.ny), z = (int)(n / ((size_t)P.nx * P.ny));
  if (P.has_walls && (z == 0 || z == P.nz - 1)) {
    for (int i = 0; i < Q; i++) f_out[(size_t)i * P.ncell + n] = 0.0;
    return;
  }
  real f[Q];
  if (fresh) {
    for (int i = 0; i < Q; i++) f[i] = dev<real>(fstate, i, (size_t)i * P.ncell + n);
  } else {
    pull(fstate, P, x, y, z, f);
  }
  for (int i = 0; i < Q; i++) f_out[(size_t)i * P.ncell + n] = wgt(i) * rho0 + (double)f[i];
}

template <typename real, typename S>
__global__ void init_equilibrium_kernel(S *__restrict__ fstate, const LatParams<real> P,
                                        double rho0, const double *__restrict__ rho_in,
                                        const double *__restrict__ u_in) {
  const size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (n >= P.ncell) return;
  const int z = (int)(n / ((size_t)P.nx * P.ny));
  const bool wall = P.has_walls && (z == 0 || z == P.nz - 1);
  const double rho = rho_in[n];
  const double ux = u_in[3 * n], uy = u_in[3 * n + 1], uz = u_in[3 * n + 2];
  const double uu = ux * ux + uy * uy + uz * uz;
  for (int i = 0; i < Q; i++) {
    const double cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
    const double v = wgt(i) * ((rho - rho0) + rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
    fstate[(size_t)i * P.ncell + n] = Narrow<S>::one(wall ? real(0) : (real)(v * kscale<S>(i)));
  }
}

template <typename S>
cudaError_t stream_collide_quad_t(Ctx &c, int first, cudaStream_t st) {
  const LatParams<float> P = lat_params<float>(c);
  const int z0 = c.has_walls ? 1 : 0;
  const int nzf = c.has_walls ? c.nz - 2 : c.nz;
  const int quads = c.nx / 4;  // four nodes per thread along x
  const int bx = quads < 128 ? quads : 128;
  const int rows = k1_block_rows(c);
  const dim3 grid((quads + bx - 1) / bx, c.ny / rows, nzf), block(bx, rows);
  const S *fin = (const S *)c.f[c.cur];
  S *fout = (S *)c.f[c.cur ^ 1];
  const bool force = c.g[0] != 0.0 || c.g[1] != 0.0 || c.g[2] != 0.0;
  if (first) {
    if (force) stream_collide_quad_kernel<S, true, true><<<grid, block, 0, st>>>(fin, fout, P, z0);
    else stream_collide_quad_kernel<S, true, false><<<grid, block, 0, st>>>(fin, fout, P, z0);
  } else {
    if (force) stream_collide_quad_kernel<S, false, true><<<grid, block, 0, st>>>(fin, fout, P, z0);
    else stream_collide_quad_kernel<S, false, false><<<grid, block, 0, st>>>(fin, fout, P, z0);
  }
  return cudaGetLastError();
}

// Nodes per compute lane of the staged pass: 2 for FP32; for 16-bit storage k1_nodes, by
// default kStageNodes16.
template <typename S>
int staged_nodes(const Ctx &c) {
  if (sizeof(S) != 2) return 2;
  return c.k1_nodes > 0 ? c.k1_nodes : kStageNodes16;
}

// Shape of the staged pass on context c (false where it does not apply: a row of the storage
// type that is not a whole number of 16-byte blocks, or too little shared memory for two
// stages). R lattice rows per unit (`rows`, or by default as many as keep one population's
// copy within kStageCopyBytes): the copies are few and large, which the copy engine needs.
template <typename S>
bool stage_geom(const Ctx &c, int stages, int rows, StageGeom &G, size_t &smem) {
  const int NPT = staged_nodes<S>(c);
  const size_t row_bytes = (size_t)c.nx * sizeof(S);
  if (row_bytes % 16 != 0 || c.nx % NPT != 0) return false;
  auto fits = [&](int r, int d) { return kStageHeader + (size_t)d * r * Q * row_bytes <= (size_t)c.smem_optin; };
  int R = rows;
  if (R <= 0) {
    R = 1;
    while (R < 16 && c.ny % (2 * R) == 0 && 2 * R * row_bytes <= kStageCopyBytes && fits(2 * R, 2))
      R *= 2;
  }
  if (c.ny % R != 0 || !fits(R, 2)) return false;
  const size_t stage_bytes = (size_t)R * Q * row_bytes;
  int D = stages;
  while (D > 2 && !fits(R, D)) D--;
  G.z0 = c.has_walls ? 1 : 0;
  G.units_per_z = c.ny / R;
  G.nunits = G.units_per_z * (c.has_walls ? c.nz - 2 : c.nz);
  G.R = R;
  G.D = D;
  G.stage_elems = R * Q * c.nx;
  G.wait_ns = c.stage_wait_ns;
  smem = kStageHeader + D * stage_bytes;
  return true;
}

template <typename S, bool FORCE, int NPT>
cudaError_t launch_staged(Ctx &c, const StageGeom &G, size_t smem, int nc, cudaStream_t st) {
  auto kern = stream_collide_staged_kernel<S, FORCE, NPT>;
  if (32 * (nc + 1) > staged_threads(NPT)) nc = staged_threads(NPT) / 32 - 1;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // one block per SM of the lattice partition, each working through its share of the units
  const int sms = c.green[0] ? c.lat_sms : c.sm_count;
  const int grid = G.nunits < sms ? G.nunits : sms;
  kern<<<grid, 32 * (nc + 1), smem, st>>>((const S *)c.f[c.cur], (S *)c.f[c.cur ^ 1],
                                          lat_params<float>(c), G, c.counters + 3);
  return cudaGetLastError();
}

// The kind of stream-collide kernel asked for, resolved for storage type S: AUTO takes the
// staged kernel for 16-bit storage, where it is the faster one (for FP32 the direct kernel
// already runs at the copy bandwidth).
template <typename S>
bool staged_kind(const Ctx &c) {
  if (sizeof(S) == 8 || c.k1_kind == IBLB_STREAM_COLLIDE_DIRECT) return false;
  return c.k1_kind == IBLB_STREAM_COLLIDE_STAGED || sizeof(S) == 2;
}

template <typename real, typename S>
bool uses_staged_t(const Ctx &c) {
  StageGeom G;
  size_t smem = 0;
  return staged_kind<S>(c) &&
         stage_geom<S>(c, c.k1_stages > 0 ? c.k1_stages : kStages, c.k1_unit_rows, G, smem);
}

// K1 through the staged kernel where it applies; *used tells whether it did.
template <typename real, typename S>
cudaError_t stream_collide_staged_t(Ctx &c, cudaStream_t st, bool *used) {
  *used = false;
  if constexpr (sizeof(S) == 8) {
    return cudaSuccess;
  } else {
    const int nc = c.k1_warps > 0 ? c.k1_warps : kStageWarps;
    const int stages = c.k1_stages > 0 ? c.k1_stages : kStages;
    StageGeom G;
    size_t smem = 0;
    if (!staged_kind<S>(c) || !stage_geom<S>(c, stages, c.k1_unit_rows, G, smem))
      return cudaSuccess;
    *used = true;
    const bool force = c.g[0] != 0.0 || c.g[1] != 0.0 || c.g[2] != 0.0;
    if constexpr (sizeof(S) == 2)
      if (staged_nodes<S>(c) == 4)
        return force ? launch_staged<S, true, 4>(c, G, smem, nc, st)
                     : launch_staged<S, false, 4>(c, G, smem, nc, st);
    return force ? launch_staged<S, true, 2>(c, G, smem, nc, st)
                 : launch_staged<S, false, 2>(c, G, smem, nc, st);
  }
}

template <typename real, typename S>
cudaError_t stream_collide_t(Ctx &c, int first, cudaStream_t st) {
  if (!first) {
    bool used = false;
    const cudaError_t e = stream_collide_staged_t<real, S>(c, st, &used);
    if (used) return e;
  }
  if constexpr (sizeof(S) == 2) return stream_collide_quad_t<S>(c, first, st);
  const LatParams<real> P = lat_params<real>(c);
  const int z0 = c.has_walls ? 1 : 0;
  const int nzf = c.has_walls ? c.nz - 2 : c.nz;
  const int half = c.nx / 2;  // two nodes per thread along x
  const int bx = half < 128 ? half : 128;
  const int rows = k1_block_rows(c);
  const dim3 grid((half + bx - 1) / bx, c.ny / rows, nzf), block(bx, rows);
  const S *fin = (const S *)c.f[c.cur];
  S *fout = (S *)c.f[c.cur ^ 1];
  const bool force = c.g[0] != 0.0 || c.g[1] != 0.0 || c.g[2] != 0.0;
  if (rows > 1) {
    if (first) {
      if (force) stream_collide_kernel<real, S, true, true, true><<<grid, block, 0, st>>>(fin, fout, P, z0);
      else stream_collide_kernel<real, S, true, false, true><<<grid, block, 0, st>>>(fin, fout, P, z0);
    } else {
      if (force) stream_collide_kernel<real, S, false, true, true><<<grid, block, 0, st>>>(fin, fout, P, z0);
      else stream_collide_kernel<real, S, false, false, true><<<grid, block, 0, st>>>(fin, fout, P, z0);
    }
  } else {
    if (first) {
      if (force) stream_collide_kernel<real, S, true, true, false><<<grid, block, 0, st>>>(fin, fout, P, z0);
      else stream_collide_kernel<real, S, true, false, false><<<grid, block, 0, st>>>(fin, fout, P, z0);
    } else {
      if (force) stream_collide_kernel<real, S, false, true, false><<<grid, block, 0, st>>>(fin, fout, P, z0);
      else stream_collide_kernel<real, S, false, false, false><<<grid, block, 0, st>>>(fin, fout, P, z0);
    }
  }
  return cudaGetLastError();
}

// Argument records of K1t and K1b for the step that starts from c's current state (K1t pulls
// from f[cur] into f[cur ^ 1]; K1b reads the array that step writes, `fpost`).
template <typename real, typename S>
TilesArgs<real, S> tiles_args(const Ctx &c) {
  TilesArgs<real, S> a;
  a.fout = (S *)c.f[c.cur ^ 1];
  a.slot_tile = c.slot_tile[c.map];
  a.pair_list = c.pair_list;
  a.npairs_ptr = c.counters + 5;
  a.Fslot = (const Vec4<real> *)c.Fslot[c.map];
  a.P = lat_params<real>(c);
  a.max_pairs = 32 * c.max_slots;
  return a;
}
// a thread per listed pair; single context: four 128-thread blocks per SM (about 78k pairs
// in one pass); in a batch a block per eight of the context's expected active tiles
int tiles_blocks(const Ctx &c, bool batched) {
  int grid = batched ? (c.tile_estimate + 7) / 8 : c.sm_count * 4;
  if (grid > c.max_slots) grid = c.max_slots;
  return grid < 1 ? 1 : grid;
}

template <typename real, typename S>
ShellArgs<real, S> shell_args(const Ctx &c, const void *fpost) {
  ShellArgs<real, S> a;
  a.fpost = (const S *)fpost;
  a.slot_tile = c.slot_tile[c.map];
  a.pair_list = c.pair_list;
  a.npairs_ptr = c.counters + 5;
  a.Fslot = (const Vec4<real> *)c.Fslot[c.map];
  a.Uslot = (Vec4<real> *)c.Uslot;
  a.P = lat_params<real>(c);
  a.max_pairs = 32 * c.max_slots;
  return a;
}
// a thread per node of a listed pair, 128 per block; single context: sixteen blocks per SM of
// the partition it runs on; in a batch a block per two of the context's expected active tiles
int shell_blocks(const Ctx &c, bool batched) {
  const int sms = c.ib_sms > 0 ? c.ib_sms : c.sm_count;
  int grid = batched ? (c.tile_estimate + 1) / 2 : sms * 16;
  if (grid > c.max_slots) grid = c.max_slots;
  return grid < 1 ? 1 : grid;
}

template <typename real, typename S>
StreamArgs<real, S> stream_args(const Ctx &c) {
  StreamArgs<real, S> a;
  a.fin = (const S *)c.f[c.cur];
  a.fout = (S *)c.f[c.cur ^ 1];
  a.P = lat_params<real>(c);
  a.z0 = c.has_walls ? 1 : 0;
  a.per_row = sizeof(S) == 2 ? c.nx / 4 : c.nx / 2;
  a.ngroups = a.per_row * c.ny * (c.has_walls ? c.nz - 2 : c.nz);
  a.force = c.g[0] != 0.0 || c.g[1] != 0.0 || c.g[2] != 0.0;
  return a;
}

template <typename real, typename S>
cudaError_t stream_collide_tiles_t(Ctx &c, int first, cudaStream_t st) {
  const int grid = tiles_blocks(c, false);
  (void)first;  // K1t corrects K1's output in place, whatever K1 read
  stream_collide_tiles_kernel<real, S><<<grid, 128, 0, st>>>(tiles_args<real, S>(c));
  return cudaGetLastError();
}

template <typename real, typename S>
cudaError_t shell_velocity_t(Ctx &c, cudaStream_t st) {
  shell_velocity_kernel<real, S><<<shell_blocks(c, false), 128, 0, st>>>(
      shell_args<real, S>(c, c.f[c.cur]));
  return cudaGetLastError();
}

template <typename T>
void append_record(std::vector<unsigned char> &bytes, const T &rec) {
  const size_t off = bytes.size();
  bytes.resize(off + sizeof(T));
  memcpy(bytes.data() + off, &rec, sizeof(T));
}

template <typename real, typename S>
int lattice_multi_record_t(const Ctx &c, MultiKernel k, std::vector<unsigned char> &bytes) {
  switch (k) {
    case MK_STREAM_COLLIDE: {
      const StreamArgs<real, S> a = stream_args<real, S>(c);
      append_record(bytes, a);
      const int b = (a.ngroups + 127) / 128;
      return b < 1 ? 1 : b;
    }
    case MK_TILES: append_record(bytes, tiles_args<real, S>(c)); return tiles_blocks(c, true);
    case MK_SHELL:
      append_record(bytes, shell_args<real, S>(c, c.f[c.cur ^ 1]));
      return shell_blocks(c, true);
    default: return -1;
  }
}

template <typename real, typename S>
cudaError_t lattice_launch_multi_t(MultiKernel k, const MultiLaunch &m, cudaStream_t s) {
  switch (k) {
    case MK_STREAM_COLLIDE: {
      static int sms = 0;
      if (!sms && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess)
        sms = 0;
      const int cap = kK1MultiPerSM * sms;
      const int grid = cap > 0 && m.blocks > cap ? cap : m.blocks;
      stream_collide_kernel_multi<real, S><<<grid, 128, 0, s>>>(
          (const StreamArgs<real, S> *)m.args, m.start, m.n);
      break;
    }
    case MK_TILES:
      stream_collide_tiles_kernel_multi<real, S><<<m.blocks, 128, 0, s>>>(
          (const TilesArgs<real, S> *)m.args, m.start, m.n);
      break;
    case MK_SHELL:
      shell_velocity_kernel_multi<real, S><<<m.blocks, 128, 0, s>>>(
          (const ShellArgs<real, S> *)m.args, m.start, m.n);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename real, typename S>
size_t lattice_record_align_t(MultiKernel k) {
  switch (k) {
    case MK_STREAM_COLLIDE: return alignof(StreamArgs<real, S>);
    case MK_TILES: return alignof(TilesArgs<real, S>);
    case MK_SHELL: return alignof(ShellArgs<real, S>);
    default: return 0;
  }
}

template <typename real, typename S>
cudaError_t fields_t(Ctx &c, double *rho_dev, double *u_dev) {
  const int blocks = (int)((c.ncell + 255) / 256);
  const double3 ub = make_double3(c.ub[0], c.ub[1], c.ub[2]);
  const double3 ut = make_double3(c.ut[0], c.ut[1], c.ut[2]);
  // the force of the last spreading step lives in the map that step used
  const int *ts = (c.nv && c.have_force) ? c.tile_slot[c.map ^ 1] : nullptr;
  fields_kernel<real, S><<<blocks, 256, 0, c.stream>>>(
      (const S *)c.f[c.cur], c.fresh, ts, (const Vec4<real> *)c.Fslot[c.map ^ 1],
      lat_params<real>(c), ub, ut, c.rho0, rho_dev, u_dev);
  return cudaGetLastError();
}

template <typename real, typename S>
cudaError_t populations_t(Ctx &c, double *f_dev) {
  const int blocks = (int)((c.ncell + 255) / 256);
  populations_kernel<real, S><<<blocks, 256, 0, c.stream>>>(
      (const S *)c.f[c.cur], c.fresh, lat_params<real>(c), c.rho0, f_dev);
  return cudaGetLastError();
}

template <typename real, typename S>
cudaError_t init_equilibrium_t(Ctx &c, const double *rho_dev, const double *u_dev) {
  const int blocks = (int)((c.ncell + 255) / 256);
  init_equilibrium_kernel<real, S><<<blocks, 256, 0, c.stream>>>(
      (S *)c.f[c.cur], lat_params<real>(c), c.rho0, rho_dev, u_dev);
  return cudaGetLastError();
}

}  // namespace

int k1_block_rows(const Ctx &c) {
  // a block is at most 128 threads (the kernels' launch bound); ny is a multiple of 4, so
  // every row count 1, 2, 4 divides it
  const int per_row = c.pop_size == 2 ? c.nx / 4 : c.nx / 2;
  const int bx = per_row < 128 ? per_row : 128;
  int rows = c.k1_rows > 0 ? c.k1_rows : 1;
  while (rows > 1 && bx * rows > 128) rows /= 2;
  return rows;
}

// Dispatch on the context's precision: (arithmetic, storage) = (double, double) for FP64,
// (float, float) for FP32, (float, half) for FP16 and (float, bfloat16) for BF16.
#define IBLB_DISPATCH(c, FN, ...)                                         \
  switch ((c).precision) {                                                \
    case IBLB_FP64: return FN<double, double>(__VA_ARGS__);               \
    case IBLB_FP16: return FN<float, __half>(__VA_ARGS__);                \
    case IBLB_BF16: return FN<float, __nv_bfloat16>(__VA_ARGS__);         \
    default: return FN<float, float>(__VA_ARGS__);                        \
  }

bool stream_collide_staged(const Ctx &c) { IBLB_DISPATCH(c, uses_staged_t, c) }

int lattice_multi_record(const Ctx &c, MultiKernel k, std::vector<unsigned char> &bytes) {
  IBLB_DISPATCH(c, lattice_multi_record_t, c, k, bytes)
}

cudaError_t lattice_launch_multi(int precision, MultiKernel k, const MultiLaunch &m,
                                 cudaStream_t s) {
  switch (precision) {
    case IBLB_FP64: return lattice_launch_multi_t<double, double>(k, m, s);
    case IBLB_FP16: return lattice_launch_multi_t<float, __half>(k, m, s);
    case IBLB_BF16: return lattice_launch_multi_t<float, __nv_bfloat16>(k, m, s);
    default: return lattice_launch_multi_t<float, float>(k, m, s);
  }
}

size_t lattice_multi_record_align(int precision, MultiKernel k) {
  switch (precision) {
    case IBLB_FP64: return lattice_record_align_t<double, double>(k);
    case IBLB_FP16: return lattice_record_align_t<float, __half>(k);
    case IBLB_BF16: return lattice_record_align_t<float, __nv_bfloat16>(k);
    default: return lattice_record_align_t<float, float>(k);
  }
}

cudaError_t launch_stream_collide(Ctx &c, int first, cudaStream_t s) {
  IBLB_DISPATCH(c, stream_collide_t, c, first, s)
}

cudaError_t launch_stream_collide_tiles(Ctx &c, int first, cudaStream_t s) {
  IBLB_DISPATCH(c, stream_collide_tiles_t, c, first, s)
}

cudaError_t launch_shell_velocity(Ctx &c, cudaStream_t s) { IBLB_DISPATCH(c, shell_velocity_t, c, s) }

cudaError_t launch_fields(Ctx &c, double *rho_dev, double *u_dev) {
  IBLB_DISPATCH(c, fields_t, c, rho_dev, u_dev)
}

cudaError_t launch_populations(Ctx &c, double *f_dev) { IBLB_DISPATCH(c, populations_t, c, f_dev) }

cudaError_t launch_init_equilibrium(Ctx &c, const double *rho_dev, const double *u_dev) {
  IBLB_DISPATCH(c, init_equilibrium_t, c, rho_dev, u_dev)
}

}  // namespace iblb
