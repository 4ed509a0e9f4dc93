// Lattice-Boltzmann kernels: the fused pull stream-collide over the whole lattice (Eqs. 9-10
// with Guo forcing and half-way bounce-back), the velocity gather at the active interface
// tiles (the velocity step of Sec. III), and the read-back / initialisation helpers.
//
// Populations are stored as deviations f_i - w_i rho0 ("shifted"), structure of arrays
// [19][nz][ny][nx] with x fastest. The state array holds post-collision populations of
// the previous step; a pull reads f_i(x - c_i) from it, which is the streaming step.
// Right after initialisation the state holds post-streaming populations ("fresh") and the
// first collision reads them in place.
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

// Pull the 19 post-streaming populations of fluid node (x, y, z) from post-collision array
// `fp`. A link whose source is a wall node is bounced back: the opposite post-collision
// population of the same node plus the moving-wall term.
template <typename real>
__device__ __forceinline__ void pull(const real *__restrict__ fp, const LatParams<real> &P, int x,
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
    const real *fi = fp + (size_t)i * P.ncell;
    if (cz(i) > 0 && wall_below) {
      f[i] = fp[(size_t)opp(i) * P.ncell + n] + P.wb[i];
    } else if (cz(i) < 0 && wall_above) {
      f[i] = fp[(size_t)opp(i) * P.ncell + n] + P.wt[i];
    } else {
      f[i] = fi[zo[1 - cz(i)] + yo[1 - cy(i)] + xo[1 - cx(i)]];
    }
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
  // rho = rho0 + drho is never rounded as a whole: 1/rho carries the rounding remainder of
  // the sum (Fast2Sum, |rho0| >= |drho|), and rho X is expanded as rho0 X + drho X
  const real rho_hi = P.rho0 + drho;
  const real rho_lo = (P.rho0 - rho_hi) + drho;
  const real r1 = real(1) / rho_hi;
  const real inv_rho = r1 * (real(1) - rho_lo * r1);
  real ux = jx, uy = jy, uz = jz;
  if (FORCE) {
    ux += real(0.5) * F[0];
    uy += real(0.5) * F[1];
    uz += real(0.5) * F[2];
  }
  ux *= inv_rho;
  uy *= inv_rho;
  uz *= inv_rho;
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

template <typename real>
struct Vec2;
template <>
struct Vec2<float> {
  using T = float2;
};
template <>
struct Vec2<double> {
  using T = double2;
};

// Post-streaming populations a (node x0) and b (node x0 + 1) of two fluid nodes, x0 even,
// from post-collision array `fin` (FIRST: `fin` already holds post-streaming populations,
// read in place). Populations that do not move along x are one aligned 2-wide load; a link
// whose source is a wall node is bounced back (opposite population of the same node plus the
// moving-wall term).
template <typename real, bool FIRST>
__device__ __forceinline__ void load_pair(const real *__restrict__ fin, const LatParams<real> &P,
                                          int x0, int y, int z, real a[Q], real b[Q]) {
  using V2 = typename Vec2<real>::T;
  const size_t plane = (size_t)P.nx * P.ny;
  const size_t n = (size_t)z * plane + (size_t)y * P.nx + x0;
  if (FIRST) {
#pragma unroll
    for (int i = 0; i < Q; i++) {
      const V2 v = *reinterpret_cast<const V2 *>(fin + (size_t)i * P.ncell + n);
      a[i] = v.x;
      b[i] = v.y;
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
      const V2 v = *reinterpret_cast<const V2 *>(fin + (size_t)opp(i) * P.ncell + n);
      const real wall = cz(i) > 0 ? P.wb[i] : P.wt[i];
      a[i] = v.x + wall;
      b[i] = v.y + wall;
      continue;
    }
    const real *row = fin + (size_t)i * P.ncell + zo[1 - cz(i)] + yo[1 - cy(i)];
    if (cx(i) == 0) {
      const V2 v = *reinterpret_cast<const V2 *>(row + x0);
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
}

template <typename real>
__device__ __forceinline__ void store_pair(real *__restrict__ fout, const LatParams<real> &P,
                                           size_t n, const real a[Q], const real b[Q]) {
  using V2 = typename Vec2<real>::T;
#pragma unroll
  for (int i = 0; i < Q; i++) {
    V2 v;
    v.x = a[i];
    v.y = b[i];
    *reinterpret_cast<V2 *>(fout + (size_t)i * P.ncell + n) = v;
  }
}

// K1: fused stream-collide of every fluid node with the uniform body force only (FORCE: the
// body force is non-zero). The nodes of active interface tiles are collided again by K1t with
// their interface force, so this pass does not wait for the interface chain of the step.
// Each thread owns the two nodes (x0, x0 + 1), x0 even: populations that do not move along x
// and every store are one aligned 2-wide access, and the address arithmetic is shared.
template <typename real, bool FIRST, bool FORCE>
__global__ void __launch_bounds__(128) stream_collide_kernel(const real *__restrict__ fin,
                                                             real *__restrict__ fout,
                                                             const LatParams<real> P, int z0) {
  const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y;
  const int z = blockIdx.z + z0;
  if (x0 >= P.nx) return;
  real a[Q], b[Q];  // populations of nodes x0 and x0 + 1
  load_pair<real, FIRST>(fin, P, x0, y, z, a, b);
  const real F[3] = {P.g[0], P.g[1], P.g[2]};
  collide<real, FORCE>(a, F, P);
  collide<real, FORCE>(b, F, P);
  store_pair(fout, P, (size_t)z * P.nx * P.ny + (size_t)y * P.nx + x0, a, b);
}

// K1t: stream-collide of the fluid nodes of the active tiles with body + interface force,
// one warp per tile (grid-stride), each thread the node pair (x0, x0 + 1) of a tile row as in
// K1. Runs after K1 of the same step and overwrites those nodes. Pairs whose interface force
// is zero keep K1's result, which is already the post-collision state with the body force
// alone.
template <typename real, bool FIRST>
__global__ void __launch_bounds__(128) stream_collide_tiles_kernel(
    const real *__restrict__ fin, real *__restrict__ fout, const int *__restrict__ slot_tile,
    const int *__restrict__ nslots_ptr, const Vec4<real> *__restrict__ Fslot,
    const LatParams<real> P, int max_slots) {
  const int nslots = min(*nslots_ptr, max_slots);
  const int lane = threadIdx.x & 31;
  const int px = lane & 1, ly = (lane >> 1) & 3, lz = lane >> 3;
  const int cell = 16 * lz + 4 * ly + 2 * px;
  const int warps = blockDim.x >> 5;
  for (int s = blockIdx.x * warps + (threadIdx.x >> 5); s < nslots; s += gridDim.x * warps) {
    const Vec4<real> Fa = Fslot[(size_t)s * TILE_CELLS + cell];
    const Vec4<real> Fb = Fslot[(size_t)s * TILE_CELLS + cell + 1];
    const int t = slot_tile[s];
    const int tx = t % P.ntx, ty = (t / P.ntx) % P.nty, tz = t / (P.ntx * P.nty);
    const int x0 = tx * TILE + 2 * px, y = ty * TILE + ly, z = tz * TILE + lz;
    if (z >= P.nz || (P.has_walls && (z == 0 || z == P.nz - 1))) continue;
    if (Fa.x == real(0) && Fa.y == real(0) && Fa.z == real(0) && Fb.x == real(0) &&
        Fb.y == real(0) && Fb.z == real(0))
      continue;
    real a[Q], b[Q];
    load_pair<real, FIRST>(fin, P, x0, y, z, a, b);
    const real FA[3] = {P.g[0] + Fa.x, P.g[1] + Fa.y, P.g[2] + Fa.z};
    const real FB[3] = {P.g[0] + Fb.x, P.g[1] + Fb.y, P.g[2] + Fb.z};
    collide<real, true>(a, FA, P);
    collide<real, true>(b, FB, P);
    store_pair(fout, P, (size_t)z * P.nx * P.ny + (size_t)y * P.nx + x0, a, b);
  }
}

// K1b: velocity after streaming at every node of the active interface tiles.
// One 64-thread block per active tile (grid-stride over the device-side tile count).
template <typename real>
__global__ void __launch_bounds__(64) shell_velocity_kernel(const real *__restrict__ fpost,
                                                            const int *__restrict__ slot_tile,
                                                            const int *__restrict__ nslots_ptr,
                                                            const Vec4<real> *__restrict__ Fslot,
                                                            Vec4<real> *__restrict__ Uslot,
                                                            const LatParams<real> P, real ubx,
                                                            real uby, real ubz, real utx,
                                                            real uty, real utz, int max_slots) {
  const int nslots = min(*nslots_ptr, max_slots);
  const int cell = threadIdx.x;
  for (int s = blockIdx.x; s < nslots; s += gridDim.x) {
    const int t = slot_tile[s];
    const int tx = t % P.ntx, ty = (t / P.ntx) % P.nty, tz = t / (P.ntx * P.nty);
    const int x = tx * TILE + (cell & 3), y = ty * TILE + ((cell >> 2) & 3),
              z = tz * TILE + (cell >> 4);
    real u[3] = {0, 0, 0};
    if (z < P.nz) {
      if (P.has_walls && z == 0) {
        u[0] = ubx; u[1] = uby; u[2] = ubz;
      } else if (P.has_walls && z == P.nz - 1) {
        u[0] = utx; u[1] = uty; u[2] = utz;
      } else {
        real f[Q];
        pull(fpost, P, x, y, z, f);
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
        for (int k = 0; k < 3; k++)
          u[k] = (j[k] + real(0.5) * (P.g[k] + Fk[k])) * inv_rho;
      }
    }
    Vec4<real> uv;
    uv.x = u[0];
    uv.y = u[1];
    uv.z = u[2];
    uv.w = real(0);
    Uslot[(size_t)s * TILE_CELLS + cell] = uv;
  }
}

// rho and u of every node of the current post-streaming state (read-back, not on the step).
template <typename real>
__global__ void fields_kernel(const real *__restrict__ fstate, int fresh,
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
    for (int i = 0; i < Q; i++) f[i] = fstate[(size_t)i * P.ncell + n];
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

template <typename real>
__global__ void populations_kernel(const real *__restrict__ fstate, int fresh,
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
    for (int i = 0; i < Q; i++) f[i] = fstate[(size_t)i * P.ncell + n];
  } else {
    pull(fstate, P, x, y, z, f);
  }
  for (int i = 0; i < Q; i++) f_out[(size_t)i * P.ncell + n] = wgt(i) * rho0 + (double)f[i];
}

template <typename real>
__global__ void init_equilibrium_kernel(real *__restrict__ fstate, const LatParams<real> P,
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
    fstate[(size_t)i * P.ncell + n] = wall ? real(0) : (real)v;
  }
}

template <typename real>
cudaError_t stream_collide_t(Ctx &c, int first, cudaStream_t st) {
  const LatParams<real> P = lat_params<real>(c);
  const int z0 = c.has_walls ? 1 : 0;
  const int nzf = c.has_walls ? c.nz - 2 : c.nz;
  const int half = c.nx / 2;  // two nodes per thread along x
  const int bx = half < 128 ? half : 128;
  dim3 grid((half + bx - 1) / bx, c.ny, nzf);
  const real *fin = (const real *)c.f[c.cur];
  real *fout = (real *)c.f[c.cur ^ 1];
  const bool force = c.g[0] != 0.0 || c.g[1] != 0.0 || c.g[2] != 0.0;
  if (first) {
    if (force) stream_collide_kernel<real, true, true><<<grid, bx, 0, st>>>(fin, fout, P, z0);
    else stream_collide_kernel<real, true, false><<<grid, bx, 0, st>>>(fin, fout, P, z0);
  } else {
    if (force) stream_collide_kernel<real, false, true><<<grid, bx, 0, st>>>(fin, fout, P, z0);
    else stream_collide_kernel<real, false, false><<<grid, bx, 0, st>>>(fin, fout, P, z0);
  }
  return cudaGetLastError();
}

template <typename real>
cudaError_t stream_collide_tiles_t(Ctx &c, int first, cudaStream_t st) {
  const LatParams<real> P = lat_params<real>(c);
  int grid = c.sm_count * 8;  // 4 tiles per block: up to ~4900 active tiles in one pass
  if (4 * grid > c.max_slots) grid = (c.max_slots + 3) / 4;
  if (grid < 1) grid = 1;
  const real *fin = (const real *)c.f[c.cur];
  real *fout = (real *)c.f[c.cur ^ 1];
  if (first)
    stream_collide_tiles_kernel<real, true><<<grid, 128, 0, st>>>(
        fin, fout, c.slot_tile[c.map], c.counters + c.map, (const Vec4<real> *)c.Fslot[c.map], P,
        c.max_slots);
  else
    stream_collide_tiles_kernel<real, false><<<grid, 128, 0, st>>>(
        fin, fout, c.slot_tile[c.map], c.counters + c.map, (const Vec4<real> *)c.Fslot[c.map], P,
        c.max_slots);
  return cudaGetLastError();
}

template <typename real>
cudaError_t shell_velocity_t(Ctx &c, cudaStream_t st) {
  const LatParams<real> P = lat_params<real>(c);
  int grid = c.sm_count * 32;
  if (grid > c.max_slots) grid = c.max_slots;
  if (grid < 1) grid = 1;
  shell_velocity_kernel<real><<<grid, TILE_CELLS, 0, st>>>(
      (const real *)c.f[c.cur], c.slot_tile[c.map], c.counters + c.map,
      (const Vec4<real> *)c.Fslot[c.map], (Vec4<real> *)c.Uslot, P, (real)c.ub[0], (real)c.ub[1], (real)c.ub[2], (real)c.ut[0],
      (real)c.ut[1], (real)c.ut[2], c.max_slots);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_stream_collide(Ctx &c, int first, cudaStream_t s) {
  return c.precision == IBLB_FP64 ? stream_collide_t<double>(c, first, s)
                                  : stream_collide_t<float>(c, first, s);
}

cudaError_t launch_stream_collide_tiles(Ctx &c, int first, cudaStream_t s) {
  return c.precision == IBLB_FP64 ? stream_collide_tiles_t<double>(c, first, s)
                                  : stream_collide_tiles_t<float>(c, first, s);
}

cudaError_t launch_shell_velocity(Ctx &c, cudaStream_t s) {
  return c.precision == IBLB_FP64 ? shell_velocity_t<double>(c, s) : shell_velocity_t<float>(c, s);
}

cudaError_t launch_fields(Ctx &c, double *rho_dev, double *u_dev) {
  const int blocks = (int)((c.ncell + 255) / 256);
  const double3 ub = make_double3(c.ub[0], c.ub[1], c.ub[2]);
  const double3 ut = make_double3(c.ut[0], c.ut[1], c.ut[2]);
  // the force of the last spreading step lives in the map that step used
  const int *ts = (c.nv && c.have_force) ? c.tile_slot[c.map ^ 1] : nullptr;
  if (c.precision == IBLB_FP64) {
    fields_kernel<double><<<blocks, 256, 0, c.stream>>>(
        (const double *)c.f[c.cur], c.fresh, ts, (const Vec4<double> *)c.Fslot[c.map ^ 1], lat_params<double>(c),
        ub, ut, c.rho0, rho_dev, u_dev);
  } else {
    fields_kernel<float><<<blocks, 256, 0, c.stream>>>(
        (const float *)c.f[c.cur], c.fresh, ts, (const Vec4<float> *)c.Fslot[c.map ^ 1], lat_params<float>(c), ub,
        ut, c.rho0, rho_dev, u_dev);
  }
  return cudaGetLastError();
}

cudaError_t launch_populations(Ctx &c, double *f_dev) {
  const int blocks = (int)((c.ncell + 255) / 256);
  if (c.precision == IBLB_FP64)
    populations_kernel<double><<<blocks, 256, 0, c.stream>>>(
        (const double *)c.f[c.cur], c.fresh, lat_params<double>(c), c.rho0, f_dev);
  else
    populations_kernel<float><<<blocks, 256, 0, c.stream>>>(
        (const float *)c.f[c.cur], c.fresh, lat_params<float>(c), c.rho0, f_dev);
  return cudaGetLastError();
}

cudaError_t launch_init_equilibrium(Ctx &c, const double *rho_dev, const double *u_dev) {
  const int blocks = (int)((c.ncell + 255) / 256);
  if (c.precision == IBLB_FP64)
    init_equilibrium_kernel<double><<<blocks, 256, 0, c.stream>>>(
        (double *)c.f[c.cur], lat_params<double>(c), c.rho0, rho_dev, u_dev);
  else
    init_equilibrium_kernel<float><<<blocks, 256, 0, c.stream>>>(
        (float *)c.f[c.cur], lat_params<float>(c), c.rho0, rho_dev, u_dev);
  return cudaGetLastError();
}

}  // namespace iblb
