// Discrete adjoint of the coupled IB-LB step (Sec. III), in double precision: gradients of an
// observable of the final vertex positions with respect to the interface parameters
// theta = (alpha1, alpha2, alpha3, eps) of Eqs. 2 and 19. The forward run is that of the
// context, FP64 or FP32; with FP32 the reverse pass linearises the double-precision step about
// the recomputed FP32 trajectory.
//
// One forward step n maps (P_n, q_n) to (P_{n+1}, q_{n+1}), P being the post-collision
// populations the pull scheme keeps between steps:
//   phi   = phi(q_n; theta)                          nodal forces, Eqs. 16-19
//   F(x)  = sum_v phi_v W(x - q_v)                   spreading on the fluid nodes, Eqs. 13-15
//   P'(x) = C(pull(P_n)(x), g + F(x))                BGK + Guo collision of the streamed state
//   u(x)  = (sum_i c_i pull(P')(x)_i + (g+F)/2)/rho  velocity after streaming
//   q_{n+1,v} = q_{n,v} + sum_x u(x) W(x - q_v)      interpolation and Euler update, Eqs. 11-12
// The reverse step applies the transposed Jacobians in the opposite order:
//   interpolation^T (including the derivative of the Peskin weights in q), the velocity
//   moments^T, the collision^T with the streaming^T (a permutation of (node, direction)
//   pairs: every adjoint population is written exactly once, no atomics), spreading^T, and
//   the transposed force Jacobian dphi/dq, which is symmetric (phi = -grad E) and is applied
//   as a forward-mode (dual number) derivative of the face forces along the adjoint force.
//   The forces are linear in alpha and eps, so dphi/dtheta is the force with one parameter
//   set to 1 and the others to 0.
// The trajectory is recorded as checkpoints every K steps; the reverse pass recomputes each
// segment forward from its checkpoint with the ordinary step, so the recomputed states are
// the recorded ones bit for bit.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "iblb_internal.cuh"

namespace iblb {
namespace {

// --- device helpers --------------------------------------------------------------------

struct Dual {
  double v, d;
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator*(double s, Dual a) { return {s * a.v, s * a.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double r = 1.0 / b.v;
  return {a.v * r, (a.d - a.v * r * b.d) * r};
}
__device__ __forceinline__ Dual operator/(Dual a, double s) { return {a.v / s, a.d / s}; }
__device__ __forceinline__ Dual operator/(double s, Dual b) {
  const double r = 1.0 / b.v;
  return {s * r, -s * r * r * b.d};
}
__device__ __forceinline__ Dual operator+(double s, Dual a) { return {a.v + s, a.d}; }
__device__ __forceinline__ Dual operator-(Dual a, double s) { return {a.v - s, a.d}; }
__device__ __forceinline__ Dual dlog(Dual a) { return {log(a.v), a.d / a.v}; }
__device__ __forceinline__ double dlog(double a) { return log(a); }
__device__ __forceinline__ Dual dabs(Dual a) { return a.v < 0 ? -a : a; }
__device__ __forceinline__ double dabs(double a) { return fabs(a); }
template <typename T>
__device__ __forceinline__ T make(double v, double d);
template <>
__device__ __forceinline__ double make<double>(double v, double) { return v; }
template <>
__device__ __forceinline__ Dual make<Dual>(double v, double d) { return {v, d}; }

// Forces of one face on its three corners (out[3 c + k]): the strain part, the negative
// gradient of A0 w_S of Eq. 2 with the Skalak invariants of the face (readings R4, R5),
// and the Lennard-Jones wall part of Eq. 19 (thirds of the centroid force, readings R6-R8).
template <typename T>
__device__ void face_forces(const T x[3][3], double H11, double H12, double H22, double A0,
                            double a1, double a2, double a3, double eps, double xi, bool lj,
                            double zb, double zt, T out[9]) {
  T a[3], b[3];
  for (int k = 0; k < 3; k++) {
    a[k] = x[1][k] - x[0][k];
    b[k] = x[2][k] - x[0][k];
  }
  const T g11 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
  const T g12 = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
  const T g22 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  const T detG = g11 * g22 - g12 * g12;
  const double detG0 = 4.0 * A0 * A0;
  const T L = dlog(detG / detG0);  // ln(I2 + 1)
  const double dE_dI1 = A0 * 0.5 * a3;
  const T dE_dL = A0 * (0.5 * (a1 - a3) + 0.25 * (a1 + a2) * L);
  for (int k = 0; k < 3; k++) {
    const T dI1_da = 2.0 * (H11 * a[k] + H12 * b[k]);
    const T dI1_db = 2.0 * (H12 * a[k] + H22 * b[k]);
    const T dL_da = (2.0 * (a[k] * g22) - 2.0 * (g12 * b[k])) / detG;
    const T dL_db = (2.0 * (b[k] * g11) - 2.0 * (g12 * a[k])) / detG;
    const T dE_da = dE_dI1 * dI1_da + dE_dL * dL_da;
    const T dE_db = dE_dI1 * dI1_db + dE_dL * dL_db;
    out[3 + k] = -dE_da;
    out[6 + k] = -dE_db;
    out[k] = dE_da + dE_db;
  }
  if (lj) {
    const T gz = (x[0][2] + x[1][2] + x[2][2]) / 3.0;
    T fz = make<T>(0.0, 0.0);
    for (int w = 0; w < 2; w++) {
      const T dz = gz - (w == 0 ? zb : zt);
      const T d = dabs(dz);
      const T r = xi / d;
      const T r2 = r * r;
      const T s6 = r2 * r2 * r2;
      fz = fz + (48.0 * eps) * ((s6 * s6 - 0.5 * s6) * dz / (d * d));
    }
    for (int c = 0; c < 3; c++) out[3 * c + 2] = out[3 * c + 2] + fz / 3.0;
  }
}

struct FaceArgs {
  int nf;
  const int *faces;
  const double *fref;  // [nf][4]: H11, H12, H22, A0
  double centre[3];
  double alpha[3], eps, xi;
  int lj;  // wall force on and the lattice has walls
  double zb, zt;
};

// Forward pass over faces at positions q: corner forces fc [nf][9], volume gradient share
// (a x b)/6 per corner fn [nf][3] and the face's share of V, fV [nf].
__global__ void adj_face_value_kernel(FaceArgs A, const double *__restrict__ q,
                                      double *__restrict__ fc, double *__restrict__ fn,
                                      double *__restrict__ fV) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= A.nf) return;
  double x[3][3];
  for (int c = 0; c < 3; c++)
    for (int k = 0; k < 3; k++) x[c][k] = q[3 * A.faces[3 * j + c] + k];
  const double *H = A.fref + 4 * j;
  double out[9];
  face_forces<double>(x, H[0], H[1], H[2], H[3], A.alpha[0], A.alpha[1], A.alpha[2], A.eps,
                      A.xi, A.lj, A.zb, A.zt, out);
  for (int k = 0; k < 9; k++) fc[9 * j + k] = out[k];
  double a[3], b[3], r[3][3];
  for (int k = 0; k < 3; k++) {
    a[k] = x[1][k] - x[0][k];
    b[k] = x[2][k] - x[0][k];
    for (int c = 0; c < 3; c++) r[c][k] = x[c][k] - A.centre[k];
  }
  fn[3 * j] = (a[1] * b[2] - a[2] * b[1]) / 6.0;
  fn[3 * j + 1] = (a[2] * b[0] - a[0] * b[2]) / 6.0;
  fn[3 * j + 2] = (a[0] * b[1] - a[1] * b[0]) / 6.0;
  fV[j] = (r[0][0] * (r[1][1] * r[2][2] - r[1][2] * r[2][1]) +
           r[0][1] * (r[1][2] * r[2][0] - r[1][0] * r[2][2]) +
           r[0][2] * (r[1][0] * r[2][1] - r[1][1] * r[2][0])) / 6.0;
}

// Derivative pass over faces along the tangent t (the adjoint force lambda_phi):
// d(corner forces) fj [nf][9], d((a x b)/6) dn [nf][3], ((a x b)/6) . (t0 + t1 + t2) fdot [nf]
// (a share of grad V . t), and t . dphi/dtheta_k per face, fpar [nf][4].
__global__ void adj_face_tangent_kernel(FaceArgs A, const double *__restrict__ q,
                                        const double *__restrict__ t, double *__restrict__ fj,
                                        double *__restrict__ dn, double *__restrict__ fdot,
                                        double *__restrict__ fpar) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= A.nf) return;
  Dual x[3][3];
  double xv[3][3], tv[3][3];
  for (int c = 0; c < 3; c++)
    for (int k = 0; k < 3; k++) {
      const int v = A.faces[3 * j + c];
      xv[c][k] = q[3 * v + k];
      tv[c][k] = t[3 * v + k];
      x[c][k] = {xv[c][k], tv[c][k]};
    }
  const double *H = A.fref + 4 * j;
  Dual out[9];
  face_forces<Dual>(x, H[0], H[1], H[2], H[3], A.alpha[0], A.alpha[1], A.alpha[2], A.eps, A.xi,
                    A.lj, A.zb, A.zt, out);
  for (int k = 0; k < 9; k++) fj[9 * j + k] = out[k].d;
  Dual a[3], b[3];
  for (int k = 0; k < 3; k++) {
    a[k] = x[1][k] - x[0][k];
    b[k] = x[2][k] - x[0][k];
  }
  const Dual n0 = (a[1] * b[2] - a[2] * b[1]) / 6.0;
  const Dual n1 = (a[2] * b[0] - a[0] * b[2]) / 6.0;
  const Dual n2 = (a[0] * b[1] - a[1] * b[0]) / 6.0;
  dn[3 * j] = n0.d;
  dn[3 * j + 1] = n1.d;
  dn[3 * j + 2] = n2.d;
  double ts[3];
  for (int k = 0; k < 3; k++) ts[k] = tv[0][k] + tv[1][k] + tv[2][k];
  fdot[j] = n0.v * ts[0] + n1.v * ts[1] + n2.v * ts[2];
  // the forces are linear in each parameter: dphi/dtheta_k is the force with theta = e_k
  for (int p = 0; p < 4; p++) {
    double o[9];
    const double e1 = p == 0, e2 = p == 1, e3 = p == 2, ee = p == 3;
    face_forces<double>(xv, H[0], H[1], H[2], H[3], e1, e2, e3, ee, A.xi, p == 3 && A.lj, A.zb,
                        A.zt, o);
    double s = 0.0;
    for (int c = 0; c < 3; c++)
      for (int k = 0; k < 3; k++) s += o[3 * c + k] * tv[c][k];
    fpar[4 * j + p] = s;
  }
}

// Fixed-order sums over faces (one block of 1024 threads): out[0] = sum a, out[1..m] = sums of
// b's columns; with grad, the b sums (the parameter derivatives of the step) are also added to
// grad[0..m-1]. Strided per-thread sums, then warp shuffles, then one warp over the warps.
constexpr int kSumThreads = 1024;
__global__ void __launch_bounds__(kSumThreads) adj_face_sums_kernel(
    int nf, const double *__restrict__ a, const double *__restrict__ b, int m,
    double *__restrict__ out, double *__restrict__ grad) {
  __shared__ double sh[kSumThreads / 32][5];
  const int t = threadIdx.x, lane = t & 31, wq = t >> 5;
  double acc[5] = {0, 0, 0, 0, 0};
  for (int j = t; j < nf; j += kSumThreads) {
    acc[0] += a[j];
    for (int k = 0; k < m; k++) acc[1 + k] += b[(size_t)m * j + k];
  }
  for (int k = 0; k <= m; k++) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wq][k] = v;
  }
  __syncthreads();
  if (wq == 0) {
    for (int k = 0; k <= m; k++) {
      double v = sh[lane][k];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) {
        out[k] = v;
        if (grad && k > 0) grad[k - 1] += v;
      }
    }
  }
}

struct VolArgs {
  int on;
  double kV, V0;
};

// phi_v = sum over the faces at v of the corner forces - kV (V - V0)/V0 dV/dq_v (forward), or
// lam_q_v += the tangent of that along lambda_phi (derivative pass, `tangent`):
//   d(corner forces) - kV/V0 [(V - V0) d(dV/dq_v) + (grad V . t) dV/dq_v].
__global__ void adj_vertex_kernel(int nv, const int *__restrict__ vf_start,
                                  const int *__restrict__ vf_list, const double *__restrict__ corner,
                                  const double *__restrict__ fn, const double *__restrict__ dn,
                                  const double *__restrict__ sums,
                                  const double *__restrict__ sums_t, VolArgs va, int tangent,
                                  double *__restrict__ out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  double f[3] = {0, 0, 0}, g[3] = {0, 0, 0}, dg[3] = {0, 0, 0};
  for (int e = vf_start[v]; e < vf_start[v + 1]; e++) {
    const int j = vf_list[e] / 3, c = vf_list[e] % 3;
    for (int k = 0; k < 3; k++) {
      f[k] += corner[9 * j + 3 * c + k];
      g[k] += fn[3 * j + k];
      if (tangent) dg[k] += dn[3 * j + k];
    }
  }
  if (!tangent) {
    const double coef = va.on ? va.kV * (sums[0] - va.V0) / va.V0 : 0.0;
    for (int k = 0; k < 3; k++) out[3 * v + k] = f[k] - coef * g[k];
  } else {
    // sums[0] = V (value pass), sums_t[0] = grad V . t (derivative pass)
    const double coef = va.on ? va.kV * (sums[0] - va.V0) / va.V0 : 0.0;
    const double coef2 = va.on ? va.kV / va.V0 * sums_t[0] : 0.0;
    for (int k = 0; k < 3; k++) out[3 * v + k] += f[k] - coef * dg[k] - coef2 * g[k];
  }
}

// --- immersed-boundary transposes ------------------------------------------------------

struct LatArgs {
  int nx, ny, nz, walls;
  size_t ncell;
  double rho0, omega, gamma;  // 1/tau, 1 - 1/(2 tau)
  double g[3];
  double ub[3], ut[3];        // wall velocities
  double wb[19], wt[19];      // moving-wall terms of the bounce-back (deviation units)
};

// Peskin's 4-point function (Eq. 15, reading R2) and its derivative, sharing the root.
__device__ __forceinline__ void peskin_wdw(double r, double &w, double &dwdr) {
  const double a = fabs(r), sg = r < 0 ? -1.0 : 1.0;
  if (a <= 1.0) {
    const double s = sqrt(1.0 + 4.0 * a - 4.0 * a * a);
    w = 0.125 * (3.0 - 2.0 * a + s);
    dwdr = sg * 0.125 * (-2.0 + (2.0 - 4.0 * a) / s);
  } else if (a <= 2.0) {
    const double s = sqrt(-7.0 + 12.0 * a - 4.0 * a * a);
    w = 0.125 * (5.0 - 2.0 * a - s);
    dwdr = sg * 0.125 * (-2.0 - (6.0 - 4.0 * a) / s);
  } else {
    w = 0.0;
    dwdr = 0.0;
  }
}

// Stencil of a vertex position: base node floor(p) - 1 per axis, the 1D weights w and their
// derivatives dw with respect to p (= -d peskin(x - p)/dx). Computed once per vertex and
// reverse step, then read by the three per-vertex passes (double square roots and divisions
// are costly here: FP64 runs at 1/64 of the FP32 rate).
struct Stencil {
  int base[3];
  int pad;
  double w[3][4], dw[3][4];
};

// one thread per (vertex, axis)
__global__ void adj_stencil_kernel(int nv, const double *__restrict__ q, Stencil *__restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * nv) return;
  const int v = t / 3, k = t - 3 * v;
  const double p = q[t];
  const int base = (int)floor(p) - 1;
  Stencil &s = out[v];
  s.base[k] = base;
  if (k == 0) s.pad = 0;
  for (int d = 0; d < 4; d++) {
    double w, dwdr;
    peskin_wdw((double)(base + d) - p, w, dwdr);
    s.w[k][d] = w;
    s.dw[k][d] = -dwdr;
  }
}

// z kind of a node: 0 fluid, 1 bottom wall, 2 top wall, -1 beyond the array (reading R9).
__device__ __forceinline__ int zkind(int z, const LatArgs &L) {
  if (!L.walls) return 0;
  if (z < 0 || z >= L.nz) return -1;
  if (z == 0) return 1;
  if (z == L.nz - 1) return 2;
  return 0;
}
__device__ __forceinline__ int wrapi(int a, int n) {
  const int r = a % n;
  return r < 0 ? r + n : r;
}
__device__ __forceinline__ size_t node_of(int x, int y, int z, const LatArgs &L) {
  return ((size_t)wrapi(z, L.nz) * L.ny + wrapi(y, L.ny)) * L.nx + wrapi(x, L.nx);
}

// Source of the pulled population i at fluid node (x, y, z): element index into P (i-th
// array) and whether the link bounces back from a wall (then: population opp(i) at the same
// node, plus the wall term).
__device__ __forceinline__ size_t pull_source(int x, int y, int z, int i, const LatArgs &L,
                                              bool &bounced) {
  const int sz = z - cz(i);
  bounced = L.walls && (sz == 0 || sz == L.nz - 1);
  if (bounced) return (size_t)opp(i) * L.ncell + node_of(x, y, z, L);
  return (size_t)i * L.ncell + node_of(x - cx(i), y - cy(i), sz, L);
}

// Post-streaming populations (deviations) at fluid node (x, y, z) from the post-collision
// populations P as stored, in the arithmetic type A of the forward state: double for FP64
// contexts; float for FP32 contexts, whose forward step ran in float (the reverse pass
// linearises the double-precision step about that trajectory; its rho and u are formed in
// float, like the forward step's, and the adjoint arithmetic itself stays double).
template <typename A, typename T>
__device__ __forceinline__ void pull_dev(const T *__restrict__ P, int x, int y, int z,
                                         const LatArgs &L, A f[Q]) {
#pragma unroll
  for (int i = 0; i < Q; i++) {
    bool bb;
    const size_t s = pull_source(x, y, z, i, L, bb);
    f[i] = (A)P[s] + (bb ? (A)(cz(i) > 0 ? L.wb[i] : L.wt[i]) : A(0));
  }
}

// Velocity (Guo shift with the total force g + F) of deviations f; returns rho. Opposite
// directions are summed in pairs.
template <typename A>
__device__ __forceinline__ A velocity(const A f[Q], const A Ft[3], A rho0, A u[3]) {
  A drho = f[0], j[3] = {0, 0, 0};
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    drho += f[i] + f[i + 1];
    const A d = f[i] - f[i + 1];
    if (cx(i)) j[0] += cx(i) > 0 ? d : -d;
    if (cy(i)) j[1] += cy(i) > 0 ? d : -d;
    if (cz(i)) j[2] += cz(i) > 0 ? d : -d;
  }
  const A rho = rho0 + drho;
  const A ir = A(1) / rho;
  for (int k = 0; k < 3; k++) u[k] = (j[k] + A(0.5) * Ft[k]) * ir;
  return rho;
}

// Velocity and density after streaming at a node.
struct alignas(32) NodeU {
  double x, y, z, rho;
};

__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// The per-vertex passes run one warp per vertex: lane l handles the stencil nodes
// (dx, dy, dz) = (l & 3, (l >> 2) & 3, (l >> 4) + 2 h) for h = 0, 1.

// Spreading at q_n onto the fluid nodes (Eq. 13): F += W phi. F is zero on entry at every
// stencil node: the spreading transpose of the previous reverse step cleared it.
__global__ void adj_spread_kernel(int nv, const Stencil *__restrict__ st,
                                  const double *__restrict__ phi, LatArgs L,
                                  double *__restrict__ F) {
  const int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (v >= nv) return;
  const Stencil &s = st[v];
  const double ph[3] = {phi[3 * v], phi[3 * v + 1], phi[3 * v + 2]};
  const int dx = lane & 3, dy = (lane >> 2) & 3;
  for (int h = 0; h < 2; h++) {
    const int dz = (lane >> 4) + 2 * h;
    const int z = s.base[2] + dz;
    if (zkind(z, L) != 0) continue;  // wall layer: force dropped; beyond: skipped
    const double w = s.w[0][dx] * s.w[1][dy] * s.w[2][dz];
    const size_t n = node_of(s.base[0] + dx, s.base[1] + dy, z, L);
    for (int k = 0; k < 3; k++) atomicAdd(&F[3 * n + k], w * ph[k]);
  }
}

// Velocity and density after streaming at every fluid node, U = (u, rho), from the
// post-collision populations P_{n+1} and the step's total force g + F.
template <typename T>
__global__ void adj_moments_kernel(const T *__restrict__ P, const double *__restrict__ F,
                                   LatArgs L, NodeU *__restrict__ U) {
  const size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (n >= L.ncell) return;
  const int x = (int)(n % L.nx), y = (int)((n / L.nx) % L.ny), z = (int)(n / ((size_t)L.nx * L.ny));
  if (zkind(z, L) != 0) return;
  using A = T;  // the forward state's arithmetic type
  A f[Q], u[3];
  pull_dev<A>(P, x, y, z, L, f);
  const A Ft[3] = {(A)(L.g[0] + F[3 * n]), (A)(L.g[1] + F[3 * n + 1]), (A)(L.g[2] + F[3 * n + 2])};
  const A rho = velocity<A>(f, Ft, (A)L.rho0, u);
  U[n] = NodeU{(double)u[0], (double)u[1], (double)u[2], (double)rho};
}

// Interpolation^T: lam_qn_v = lam_v + sum_x (u(x) . lam_v) dW/dq_v, and lam_u(x) += W lam_v
// on the fluid nodes, with u(x) the velocity of the step (the wall velocity on wall layers).
__global__ void adj_interp_t_kernel(int nv, const Stencil *__restrict__ st,
                                    const double *__restrict__ lam, const NodeU *__restrict__ U,
                                    LatArgs L, double *__restrict__ lam_qn,
                                    double *__restrict__ lam_u) {
  const int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (v >= nv) return;
  const Stencil &s = st[v];
  const double l[3] = {lam[3 * v], lam[3 * v + 1], lam[3 * v + 2]};
  const int dx = lane & 3, dy = (lane >> 2) & 3;
  double acc[3] = {0, 0, 0};
  for (int h = 0; h < 2; h++) {
    const int dz = (lane >> 4) + 2 * h;
    const int z = s.base[2] + dz;
    const int kind = zkind(z, L);
    if (kind < 0) continue;
    const double wx = s.w[0][dx], wy = s.w[1][dy], wz = s.w[2][dz];
    double u[3];
    if (kind == 1) {
      for (int k = 0; k < 3; k++) u[k] = L.ub[k];
    } else if (kind == 2) {
      for (int k = 0; k < 3; k++) u[k] = L.ut[k];
    } else {
      const size_t n = node_of(s.base[0] + dx, s.base[1] + dy, z, L);
      const NodeU un = U[n];
      u[0] = un.x;
      u[1] = un.y;
      u[2] = un.z;
      const double w = wx * wy * wz;
      for (int k = 0; k < 3; k++) atomicAdd(&lam_u[3 * n + k], w * l[k]);
    }
    const double ul = u[0] * l[0] + u[1] * l[1] + u[2] * l[2];
    acc[0] += ul * s.dw[0][dx] * wy * wz;
    acc[1] += ul * wx * s.dw[1][dy] * wz;
    acc[2] += ul * wx * wy * s.dw[2][dz];
  }
  for (int k = 0; k < 3; k++) acc[k] = warp_sum(acc[k]);
  if (lane == 0)
    for (int k = 0; k < 3; k++) lam_qn[3 * v + k] = l[k] + acc[k];
}

// Velocity moments^T at the fluid nodes with lam_u != 0: the adjoint of each pulled
// population, (c_i - u) . lam_u / rho, added to its source in lam_P (its force part,
// lam_u / (2 rho), is added by the collision transpose, which also clears lam_u).
__global__ void adj_velocity_t_kernel(const double *__restrict__ lam_u,
                                      const NodeU *__restrict__ U, LatArgs L,
                                      double *__restrict__ lam_P) {
  const size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (n >= L.ncell) return;
  const int x = (int)(n % L.nx), y = (int)((n / L.nx) % L.ny), z = (int)(n / ((size_t)L.nx * L.ny));
  if (zkind(z, L) != 0) return;
  const double lu[3] = {lam_u[3 * n], lam_u[3 * n + 1], lam_u[3 * n + 2]};
  if (lu[0] == 0.0 && lu[1] == 0.0 && lu[2] == 0.0) return;
  const NodeU un = U[n];
  const double ir = 1.0 / un.rho;
  const double ulu = (un.x * lu[0] + un.y * lu[1] + un.z * lu[2]) * ir;
  const double l[3] = {lu[0] * ir, lu[1] * ir, lu[2] * ir};
#pragma unroll
  for (int i = 0; i < Q; i++) {
    double a = -ulu;
    if (cx(i)) a += cx(i) > 0 ? l[0] : -l[0];
    if (cy(i)) a += cy(i) > 0 ? l[1] : -l[1];
    if (cz(i)) a += cz(i) > 0 ? l[2] : -l[2];
    bool bb;
    lam_P[pull_source(x, y, z, i, L, bb)] += a;  // each (source, direction) has one puller
  }
}

// Collision^T and streaming^T at every fluid node. mu = lam_P1 at the node is the adjoint of
// the post-collision populations out_i = f_i - omega (f_i - feq_i(rho, u)) + S_i(u, F) of the
// pulled pre-collision f (BGK with Guo forcing). With the moments of mu,
//   m0 = sum w_i mu_i, m1 = sum w_i mu_i c_i, M2 = sum w_i mu_i c_i c_i^T,
// the vector-Jacobian product is
//   lam_f_j = (1 - omega) mu_j + A + B . (c_j - u) / rho,
//   A = omega (m0 + 3 u.m1 + 4.5 u.M2 u - 1.5 u.u m0)                      (d/d rho)
//   B = omega rho (3 m1 + 9 M2 u - 3 m0 u) + gamma (9 M2 Ft - 3 m0 Ft)     (d/d u)
//   lam_F = B / (2 rho) + gamma (3 m1 - 3 m0 u + 9 M2 u)                     (d/d F)
// (u depends on f through (sum c f + Ft/2)/rho; Ft = g + F). lam_f_j goes to the source of
// the pulled population (a permutation: written once). The velocity-moment transpose of step
// n+1 adds lam_u / (2 rho_{n+1}) to lam_F here, and lam_u is cleared for the next step.
template <typename T>
__global__ void adj_collide_t_kernel(const double *__restrict__ lam_P1, const T *__restrict__ Pn,
                                     const double *__restrict__ F, const NodeU *__restrict__ U1,
                                     double *__restrict__ lam_u, LatArgs L, int fresh,
                                     double *__restrict__ lam_P0, double *__restrict__ lam_F) {
  const size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (n >= L.ncell) return;
  const int x = (int)(n % L.nx), y = (int)((n / L.nx) % L.ny), z = (int)(n / ((size_t)L.nx * L.ny));
  if (zkind(z, L) != 0) return;
  using A = T;  // the forward state's arithmetic type
  A f[Q], ua[3];
  if (fresh) {
#pragma unroll
    for (int i = 0; i < Q; i++) f[i] = (A)Pn[(size_t)i * L.ncell + n];
  } else {
    pull_dev<A>(Pn, x, y, z, L, f);
  }
  const double Ft[3] = {L.g[0] + F[3 * n], L.g[1] + F[3 * n + 1], L.g[2] + F[3 * n + 2]};
  const A Fta[3] = {(A)Ft[0], (A)Ft[1], (A)Ft[2]};
  const double rho = (double)velocity<A>(f, Fta, (A)L.rho0, ua);
  const double u[3] = {(double)ua[0], (double)ua[1], (double)ua[2]};
  const double ir = 1.0 / rho;
  double mu[Q];
#pragma unroll
  for (int i = 0; i < Q; i++) mu[i] = lam_P1[(size_t)i * L.ncell + n];
  // moments of mu from opposite pairs: c c^T is the same for both, c changes sign
  double m0 = wgt(0) * mu[0], m1[3] = {0, 0, 0}, mxx = 0, myy = 0, mzz = 0, mxy = 0, mxz = 0,
         myz = 0;
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const double ws = wgt(i) * (mu[i] + mu[i + 1]);
    const double wd = wgt(i) * (mu[i] - mu[i + 1]);
    m0 += ws;
    if (cx(i)) { m1[0] += cx(i) > 0 ? wd : -wd; mxx += ws; }
    if (cy(i)) { m1[1] += cy(i) > 0 ? wd : -wd; myy += ws; }
    if (cz(i)) { m1[2] += cz(i) > 0 ? wd : -wd; mzz += ws; }
    if (cx(i) && cy(i)) mxy += cx(i) * cy(i) > 0 ? ws : -ws;
    if (cx(i) && cz(i)) mxz += cx(i) * cz(i) > 0 ? ws : -ws;
    if (cy(i) && cz(i)) myz += cy(i) * cz(i) > 0 ? ws : -ws;
  }
  const double M2u[3] = {mxx * u[0] + mxy * u[1] + mxz * u[2], mxy * u[0] + myy * u[1] + myz * u[2],
                         mxz * u[0] + myz * u[1] + mzz * u[2]};
  const double M2F[3] = {mxx * Ft[0] + mxy * Ft[1] + mxz * Ft[2],
                         mxy * Ft[0] + myy * Ft[1] + myz * Ft[2],
                         mxz * Ft[0] + myz * Ft[1] + mzz * Ft[2]};
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const double um1 = u[0] * m1[0] + u[1] * m1[1] + u[2] * m1[2];
  const double uM2u = u[0] * M2u[0] + u[1] * M2u[1] + u[2] * M2u[2];
  const double Arho = L.omega * (m0 + 3.0 * um1 + 4.5 * uM2u - 1.5 * uu * m0);
  double B[3], lf[3];
  for (int k = 0; k < 3; k++) {
    B[k] = L.omega * rho * (3.0 * m1[k] + 9.0 * M2u[k] - 3.0 * m0 * u[k]) +
           L.gamma * (9.0 * M2F[k] - 3.0 * m0 * Ft[k]);
    lf[k] = 0.5 * B[k] * ir + L.gamma * (3.0 * m1[k] - 3.0 * m0 * u[k] + 9.0 * M2u[k]);
  }
  const double lu[3] = {lam_u[3 * n], lam_u[3 * n + 1], lam_u[3 * n + 2]};
  if (lu[0] != 0.0 || lu[1] != 0.0 || lu[2] != 0.0) {
    const double h = 0.5 / U1[n].rho;
    for (int k = 0; k < 3; k++) {
      lf[k] += lu[k] * h;
      lam_u[3 * n + k] = 0.0;
    }
  }
  for (int k = 0; k < 3; k++) lam_F[3 * n + k] = lf[k];
  const double b[3] = {B[0] * ir, B[1] * ir, B[2] * ir};
  const double s0 = Arho - (u[0] * b[0] + u[1] * b[1] + u[2] * b[2]);
  const double om1 = 1.0 - L.omega;
  double lam[Q];
  lam[0] = om1 * mu[0] + s0;
#pragma unroll
  for (int i = 1; i < Q; i += 2) {  // c.b changes sign between opposite directions
    double cb = 0.0;
    if (cx(i)) cb += cx(i) > 0 ? b[0] : -b[0];
    if (cy(i)) cb += cy(i) > 0 ? b[1] : -b[1];
    if (cz(i)) cb += cz(i) > 0 ? b[2] : -b[2];
    lam[i] = om1 * mu[i] + s0 + cb;
    lam[i + 1] = om1 * mu[i + 1] + s0 - cb;
  }
#pragma unroll
  for (int i = 0; i < Q; i++) {
    if (fresh) {
      lam_P0[(size_t)i * L.ncell + n] = lam[i];
    } else {
      bool bb;
      lam_P0[pull_source(x, y, z, i, L, bb)] = lam[i];  // a permutation: written once
    }
  }
}

// Spreading^T: lam_phi_v = sum_x W lam_F(x) over the fluid nodes, and
// lam_qn_v += sum_x (phi_v . lam_F(x)) dW/dq_v. The step's force field F is no longer
// needed afterwards: its stencil nodes are cleared here, which leaves F zero for the next
// reverse step's spreading.
__global__ void adj_spread_t_kernel(int nv, const Stencil *__restrict__ st,
                                    const double *__restrict__ phi, const double *__restrict__ lam_F,
                                    LatArgs L, double *__restrict__ lam_phi,
                                    double *__restrict__ lam_qn, double *__restrict__ F) {
  const int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (v >= nv) return;
  const Stencil &s = st[v];
  const double ph[3] = {phi[3 * v], phi[3 * v + 1], phi[3 * v + 2]};
  const int dx = lane & 3, dy = (lane >> 2) & 3;
  double lp[3] = {0, 0, 0}, acc[3] = {0, 0, 0};
  for (int h = 0; h < 2; h++) {
    const int dz = (lane >> 4) + 2 * h;
    const int z = s.base[2] + dz;
    if (zkind(z, L) != 0) continue;
    const size_t n = node_of(s.base[0] + dx, s.base[1] + dy, z, L);
    const double lf[3] = {lam_F[3 * n], lam_F[3 * n + 1], lam_F[3 * n + 2]};
    const double wx = s.w[0][dx], wy = s.w[1][dy], wz = s.w[2][dz];
    const double w = wx * wy * wz;
    for (int k = 0; k < 3; k++) {
      lp[k] += w * lf[k];
      F[3 * n + k] = 0.0;
    }
    const double pl = ph[0] * lf[0] + ph[1] * lf[1] + ph[2] * lf[2];
    acc[0] += pl * s.dw[0][dx] * wy * wz;
    acc[1] += pl * wx * s.dw[1][dy] * wz;
    acc[2] += pl * wx * wy * s.dw[2][dz];
  }
  for (int k = 0; k < 3; k++) {
    lp[k] = warp_sum(lp[k]);
    acc[k] = warp_sum(acc[k]);
  }
  if (lane == 0)
    for (int k = 0; k < 3; k++) {
      lam_phi[3 * v + k] = lp[k];
      lam_qn[3 * v + k] += acc[k];
    }
}

// --- host side ---------------------------------------------------------------------------

struct Adjoint {
  int nsteps = 0, every = 0, first_fresh = 0;
  std::vector<void *> ck_P;           // populations at steps 0, K, 2K, ..., nsteps (storage type)
  std::vector<double *> ck_q;         // positions at the same steps
  std::vector<void *> seg_P;          // states of the segment being reversed (storage type)
  std::vector<double *> seg_q;
  double *lam_P[2] = {nullptr, nullptr};
  double *lam_q = nullptr, *lam_qn = nullptr, *lam_phi = nullptr, *lam_F = nullptr,
         *lam_u = nullptr, *F = nullptr, *phi = nullptr;
  double *fc = nullptr, *fn = nullptr, *fV = nullptr, *fj = nullptr, *dn = nullptr,
         *fdot = nullptr, *fpar = nullptr, *sums = nullptr, *sums_t = nullptr, *grad = nullptr;
  NodeU *U = nullptr;       // [ncell] velocity and density after streaming of the step
  Stencil *st = nullptr;    // [nv] stencils of the step's positions
};

void free_all(Adjoint *a) {
  auto f = [](void *p) {
    if (p) cudaFree(p);
  };
  for (void *p : a->ck_P) f(p);
  for (double *p : a->ck_q) f(p);
  for (void *p : a->seg_P) f(p);
  for (double *p : a->seg_q) f(p);
  f(a->lam_P[0]); f(a->lam_P[1]); f(a->lam_q); f(a->lam_qn); f(a->lam_phi); f(a->lam_F);
  f(a->lam_u); f(a->F); f(a->phi); f(a->fc); f(a->fn); f(a->fV); f(a->fj); f(a->dn); f(a->fdot);
  f(a->fpar); f(a->sums); f(a->sums_t); f(a->grad); f(a->U); f(a->st);
  delete a;
}

int afail(Ctx &c, int code, const std::string &m) {
  c.err = m;
  return code;
}

#define ADJ_TRY(c, expr)                                                                   \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return iblb::afail((c), e_ == cudaErrorMemoryAllocation ? IBLB_ENOMEM : IBLB_ECUDA,   \
                   std::string(#expr) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

cudaError_t dmalloc(double **p, size_t n) {
  *p = nullptr;
  return cudaMalloc((void **)p, (n ? n : 1) * sizeof(double));
}

FaceArgs face_args(const Ctx &c) {
  FaceArgs A;
  A.nf = c.nf;
  A.faces = c.faces;
  A.fref = c.fref;
  for (int k = 0; k < 3; k++) {
    A.centre[k] = c.centre[k];
    A.alpha[k] = c.iface.alpha[k];
  }
  A.eps = c.iface.eps;
  A.xi = c.iface.xi;
  A.lj = c.iface.wall_force_on && c.has_walls;
  A.zb = 0.5;
  A.zt = c.nz - 1.5;
  return A;
}

LatArgs lat_args(const Ctx &c) {
  LatArgs L;
  L.nx = c.nx; L.ny = c.ny; L.nz = c.nz; L.walls = c.has_walls;
  L.ncell = c.ncell;
  L.rho0 = c.rho0;
  L.omega = 1.0 / c.tau;
  L.gamma = 1.0 - 0.5 / c.tau;
  for (int k = 0; k < 3; k++) {
    L.g[k] = c.g[k];
    L.ub[k] = c.ub[k];
    L.ut[k] = c.ut[k];
  }
  for (int i = 0; i < Q; i++) {
    const double cb = cx(i) * c.ub[0] + cy(i) * c.ub[1] + cz(i) * c.ub[2];
    const double ct = cx(i) * c.ut[0] + cy(i) * c.ut[1] + cz(i) * c.ut[2];
    L.wb[i] = 6.0 * wgt(i) * c.rho0 * cb;
    L.wt[i] = 6.0 * wgt(i) * c.rho0 * ct;
  }
  return L;
}

// A checkpoint: the populations as stored (so that restoring them continues bit for bit) and
// the positions.
int snapshot_raw(Ctx &c, void *P, double *q) {
  ADJ_TRY(c, cudaMemcpyAsync(P, c.f[c.cur], (size_t)Q * c.ncell * c.pop_size,
                             cudaMemcpyDeviceToDevice, c.stream));
  ADJ_TRY(c, cudaMemcpyAsync(q, c.q, (size_t)3 * c.nv * sizeof(double), cudaMemcpyDeviceToDevice,
                             c.stream));
  return 0;
}

// n steps queued with the health check of iblb_step at their end
int run_steps(Ctx &c, int n) {
  ADJ_TRY(c, cudaMemsetAsync(c.counters + 3, 0, sizeof(int), c.stream));
  if (int rc = enqueue_steps(c, n)) return rc;
  int hw = 0;
  ADJ_TRY(c, cudaMemcpyAsync(&hw, c.counters + 3, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  ADJ_TRY(c, cudaStreamSynchronize(c.stream));
  return health_status(c, hw);
}

// Recompute a segment: from the restored state, `len` steps, the state after each one copied
// (as stored) to seg_P[m], seg_q[m]; everything queued, one health check at the end.
int recompute_segment(Ctx &c, Adjoint *a, int len) {
  ADJ_TRY(c, cudaMemsetAsync(c.counters + 3, 0, sizeof(int), c.stream));
  if (int rc = snapshot_raw(c, a->seg_P[0], a->seg_q[0])) return rc;
  for (int m = 1; m <= len; m++) {
    if (int rc = enqueue_steps(c, 1)) return rc;
    if (int rc = snapshot_raw(c, a->seg_P[m], a->seg_q[m])) return rc;
  }
  int hw = 0;
  ADJ_TRY(c, cudaMemcpyAsync(&hw, c.counters + 3, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  ADJ_TRY(c, cudaStreamSynchronize(c.stream));
  return health_status(c, hw);
}

// Reverse step n: a->lam_q (of q_{n+1}) and a->lam_P[1] (of P_{n+1}) become those of q_n, P_n
// in a->lam_qn and a->lam_P[0] (swapped by the caller). Pn, Pn1 are stored populations (T).
// No scratch field needs clearing: F and lam_u are zero between steps (cleared by their last
// readers), lam_F and lam_P0 are overwritten at every fluid node.
template <typename T>
int reverse_step(Ctx &c, Adjoint *a, const T *Pn, const double *qn, const T *Pn1, int fresh) {
  const FaceArgs FA = face_args(c);
  const LatArgs L = lat_args(c);
  const VolArgs va{c.iface.volume_force_on, c.iface.kV, c.V0};
  // small blocks for the per-face and per-vertex passes: a few thousand threads spread over
  // all SMs (their double arithmetic, not memory, sets their time)
  const int tb = 32, tw = 128;
  const unsigned gf = (unsigned)((c.nf + tb - 1) / tb), gv = (unsigned)((c.nv + tb - 1) / tb);
  const unsigned gs = (unsigned)((3 * c.nv + tb - 1) / tb);     // a thread per (vertex, axis)
  const unsigned gw = (unsigned)((32L * c.nv + tw - 1) / tw);   // a warp per vertex
  const unsigned gn = (unsigned)((c.ncell + 255) / 256);
  cudaStream_t st = c.stream;
  // forward pieces at q_n: forces, volume, stencils, the spread force field, the moments
  adj_face_value_kernel<<<gf, tb, 0, st>>>(FA, qn, a->fc, a->fn, a->fV);
  adj_face_sums_kernel<<<1, kSumThreads, 0, st>>>(c.nf, a->fV, nullptr, 0, a->sums, nullptr);
  adj_vertex_kernel<<<gv, tb, 0, st>>>(c.nv, c.vf_start, c.vf_list, a->fc, a->fn, nullptr, a->sums,
                                       nullptr, va, 0, a->phi);
  adj_stencil_kernel<<<gs, tb, 0, st>>>(c.nv, qn, a->st);
  adj_spread_kernel<<<gw, tw, 0, st>>>(c.nv, a->st, a->phi, L, a->F);
  adj_moments_kernel<T><<<gn, 256, 0, st>>>(Pn1, a->F, L, a->U);
  // interpolation^T, velocity^T, collision^T and streaming^T, spreading^T
  adj_interp_t_kernel<<<gw, tw, 0, st>>>(c.nv, a->st, a->lam_q, a->U, L, a->lam_qn, a->lam_u);
  adj_velocity_t_kernel<<<gn, 256, 0, st>>>(a->lam_u, a->U, L, a->lam_P[1]);
  adj_collide_t_kernel<T><<<gn, 256, 0, st>>>(a->lam_P[1], Pn, a->F, a->U, a->lam_u, L, fresh,
                                              a->lam_P[0], a->lam_F);
  adj_spread_t_kernel<<<gw, tw, 0, st>>>(c.nv, a->st, a->phi, a->lam_F, L, a->lam_phi, a->lam_qn,
                                         a->F);
  // force Jacobian^T along lam_phi, and the parameter derivatives (added to grad)
  adj_face_tangent_kernel<<<gf, tb, 0, st>>>(FA, qn, a->lam_phi, a->fj, a->dn, a->fdot, a->fpar);
  adj_face_sums_kernel<<<1, kSumThreads, 0, st>>>(c.nf, a->fdot, a->fpar, 4, a->sums_t, a->grad);
  adj_vertex_kernel<<<gv, tb, 0, st>>>(c.nv, c.vf_start, c.vf_list, a->fj, a->fn, a->dn, a->sums,
                                       a->sums_t, va, 1, a->lam_qn);
  ADJ_TRY(c, cudaGetLastError());
  return 0;
}

}  // namespace

void adjoint_free(Ctx &c) {
  if (c.adj) free_all((Adjoint *)c.adj);
  c.adj = nullptr;
}

}  // namespace iblb

using iblb::Ctx;

extern "C" {

int iblb_adjoint_record(iblb_ctx *h, int32_t nsteps, int32_t every) {
  if (!h) return IBLB_EINVAL;
  Ctx &c = h->c;
  if (c.precision != IBLB_FP64 && c.precision != IBLB_FP32)
    return iblb::afail(c, IBLB_EINVAL, "the adjoint needs an IBLB_FP64 or IBLB_FP32 context");
  if (c.nv == 0) return iblb::afail(c, IBLB_EINVAL, "no mesh has been added");
  if (nsteps < 1 || every < 1) return iblb::afail(c, IBLB_EINVAL, "nsteps and every must be >= 1");
  if (int rc = iblb::settle_health(c)) return rc;  // a failure of earlier iblb_step_async steps
  iblb::adjoint_free(c);
  auto *a = new iblb::Adjoint();
  c.adj = a;
  a->nsteps = nsteps;
  a->every = every < nsteps ? every : nsteps;
  a->first_fresh = c.fresh;
  const size_t pn = (size_t)iblb::Q * c.ncell, qn = (size_t)3 * c.nv;
  const int nck = (nsteps + a->every - 1) / a->every + 1;
  for (int k = 0; k < nck; k++) {
    void *P = nullptr;
    double *q = nullptr;
    ADJ_TRY(c, cudaMalloc(&P, pn * c.pop_size));
    a->ck_P.push_back(P);
    ADJ_TRY(c, iblb::dmalloc(&q, qn));
    a->ck_q.push_back(q);
  }
  ADJ_TRY(c, cudaStreamSynchronize(c.stream));
  if (int rc = iblb::snapshot_raw(c, a->ck_P[0], a->ck_q[0])) return rc;
  int done = 0;
  for (int k = 1; k < nck; k++) {
    const int n = nsteps - done < a->every ? nsteps - done : a->every;
    if (int rc = iblb::run_steps(c, n)) return rc;
    done += n;
    if (int rc = iblb::snapshot_raw(c, a->ck_P[k], a->ck_q[k])) return rc;
  }
  ADJ_TRY(c, cudaStreamSynchronize(c.stream));
  return IBLB_OK;
}

int iblb_adjoint_gradient(iblb_ctx *h, const double *dJdq, double *dJdtheta) {
  if (!h || !dJdq || !dJdtheta) return IBLB_EINVAL;
  Ctx &c = h->c;
  auto *a = (iblb::Adjoint *)c.adj;
  if (!a) return iblb::afail(c, IBLB_EINVAL, "no trajectory recorded (iblb_adjoint_record)");
  if (int rc = iblb::settle_health(c)) return rc;
  const size_t pn = (size_t)iblb::Q * c.ncell, qn = (size_t)3 * c.nv;
  // work arrays (kept for later calls)
  if (!a->lam_q) {
    ADJ_TRY(c, iblb::dmalloc(&a->lam_P[0], pn));
    ADJ_TRY(c, iblb::dmalloc(&a->lam_P[1], pn));
    ADJ_TRY(c, iblb::dmalloc(&a->lam_q, qn));
    ADJ_TRY(c, iblb::dmalloc(&a->lam_qn, qn));
    ADJ_TRY(c, iblb::dmalloc(&a->lam_phi, qn));
    ADJ_TRY(c, iblb::dmalloc(&a->phi, qn));
    ADJ_TRY(c, iblb::dmalloc(&a->lam_F, 3 * c.ncell));
    ADJ_TRY(c, iblb::dmalloc(&a->lam_u, 3 * c.ncell));
    ADJ_TRY(c, iblb::dmalloc(&a->F, 3 * c.ncell));
    ADJ_TRY(c, iblb::dmalloc(&a->fc, (size_t)9 * c.nf));
    ADJ_TRY(c, iblb::dmalloc(&a->fj, (size_t)9 * c.nf));
    ADJ_TRY(c, iblb::dmalloc(&a->fn, (size_t)3 * c.nf));
    ADJ_TRY(c, iblb::dmalloc(&a->dn, (size_t)3 * c.nf));
    ADJ_TRY(c, iblb::dmalloc(&a->fV, (size_t)c.nf));
    ADJ_TRY(c, iblb::dmalloc(&a->fdot, (size_t)c.nf));
    ADJ_TRY(c, iblb::dmalloc(&a->fpar, (size_t)4 * c.nf));
    ADJ_TRY(c, iblb::dmalloc(&a->sums, 8));
    ADJ_TRY(c, iblb::dmalloc(&a->sums_t, 8));
    ADJ_TRY(c, iblb::dmalloc(&a->grad, 4));
    ADJ_TRY(c, cudaMalloc((void **)&a->U, c.ncell * sizeof(iblb::NodeU)));
    ADJ_TRY(c, cudaMalloc((void **)&a->st, (size_t)c.nv * sizeof(iblb::Stencil)));
    for (int m = 0; m <= a->every; m++) {
      void *P = nullptr;
      double *q = nullptr;
      ADJ_TRY(c, cudaMalloc(&P, pn * c.pop_size));
      a->seg_P.push_back(P);
      ADJ_TRY(c, iblb::dmalloc(&q, qn));
      a->seg_q.push_back(q);
    }
  }
  ADJ_TRY(c, cudaMemcpyAsync(a->lam_q, dJdq, qn * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  ADJ_TRY(c, cudaMemsetAsync(a->lam_P[0], 0, pn * sizeof(double), c.stream));
  ADJ_TRY(c, cudaMemsetAsync(a->lam_P[1], 0, pn * sizeof(double), c.stream));
  // zero between reverse steps (each step leaves them so)
  ADJ_TRY(c, cudaMemsetAsync(a->F, 0, 3 * c.ncell * sizeof(double), c.stream));
  ADJ_TRY(c, cudaMemsetAsync(a->lam_u, 0, 3 * c.ncell * sizeof(double), c.stream));
  ADJ_TRY(c, cudaMemsetAsync(a->grad, 0, 4 * sizeof(double), c.stream));
  const int nseg = (int)a->ck_P.size() - 1;
  int rc = 0;
  for (int s = nseg - 1; s >= 0 && rc == 0; s--) {
    const int first = s * a->every;
    const int len = (a->nsteps - first) < a->every ? a->nsteps - first : a->every;
    const int fresh0 = s == 0 ? a->first_fresh : 0;
    rc = iblb::restore_state(c, a->ck_P[s], a->ck_q[s], fresh0);
    if (rc == 0) rc = iblb::recompute_segment(c, a, len);
    for (int m = len - 1; m >= 0 && rc == 0; m--) {
      const int fresh = s == 0 && m == 0 && a->first_fresh;
      if (c.pop_size == sizeof(double))
        rc = iblb::reverse_step<double>(c, a, (const double *)a->seg_P[m], a->seg_q[m],
                                        (const double *)a->seg_P[m + 1], fresh);
      else
        rc = iblb::reverse_step<float>(c, a, (const float *)a->seg_P[m], a->seg_q[m],
                                       (const float *)a->seg_P[m + 1], fresh);
      std::swap(a->lam_q, a->lam_qn);
      std::swap(a->lam_P[0], a->lam_P[1]);
    }
  }
  // back to the end of the recorded run
  if (rc == 0) rc = iblb::restore_state(c, a->ck_P[nseg], a->ck_q[nseg], 0);
  if (rc) return rc;
  ADJ_TRY(c, cudaMemcpyAsync(dJdtheta, a->grad, 4 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  ADJ_TRY(c, cudaStreamSynchronize(c.stream));
  return IBLB_OK;
}

int iblb_adjoint_release(iblb_ctx *h) {
  if (!h) return IBLB_EINVAL;
  cudaStreamSynchronize(h->c.stream);
  iblb::adjoint_free(h->c);
  return IBLB_OK;
}

}  // extern "C"
