// Interface kernels: per-face forces (Eqs. 2, 17-19) with the double-precision volume sum,
// per-vertex gathering into nodal forces (Eq. 16) and binning by 4x4x4 source tile,
// spreading by owner-computes gather over the binned vertices (Eq. 13), interpolation and
// the Euler update (Eqs. 11-12), and the marking of active tiles for the next step.
//
// Arithmetic runs in the population type `real` (float or double); vertex positions, the
// enclosed volume V and V - V0 are always double.
#include <math.h>
#include <string.h>

#include "iblb_internal.cuh"

namespace iblb {
namespace {

struct Dims {
  int nx, ny, nz, has_walls, ntx, nty, ntz, max_slots;
  double zb, zt;              // wall planes
  double inx, iny, inz;       // 1/nx, 1/ny, 1/nz
};

Dims dims_of(const Ctx &c) {
  Dims d;
  d.nx = c.nx; d.ny = c.ny; d.nz = c.nz; d.has_walls = c.has_walls;
  d.ntx = c.ntx; d.nty = c.nty; d.ntz = c.ntz; d.max_slots = c.max_slots;
  d.zb = 0.5;
  d.zt = c.nz - 1.5;
  d.inx = 1.0 / c.nx;
  d.iny = 1.0 / c.ny;
  d.inz = 1.0 / c.nz;
  return d;
}

__device__ __forceinline__ int floor_div4(int a) { return a >> 2; }  // arithmetic shift floors

// p reduced to [0, n) for a periodic axis (positions are stored unwrapped); inv_n = 1/n, so
// no double division is issued (slow on this part). Rounding may leave p at -tiny or n.
__device__ __forceinline__ double wrap_pos(double p, int n, double inv_n) {
  return p - n * floor(p * inv_n);
}

__device__ __forceinline__ float log_(float v) { return logf(v); }
__device__ __forceinline__ double log_(double v) { return log(v); }
__device__ __forceinline__ float sqrt_(float v) { return sqrtf(v); }
__device__ __forceinline__ double sqrt_(double v) { return sqrt(v); }

// Lennard-Jones force along z on a centroid at signed height dz above a wall plane (Eq. 19;
// d points from the wall foot point to the centroid).
template <typename real>
__device__ __forceinline__ real lj_fz(real dz, real eps48, real xi) {
  const real inv_d2 = real(1) / (dz * dz);
  const real s2 = xi * xi * inv_d2;
  const real s6 = s2 * s2 * s2;
  return eps48 * (s6 * s6 - real(0.5) * s6) * dz * inv_d2;
}

// Per-face reference data in the population type, stored by component ([FGEO][nf]): A, B
// (edges), X0 - c, the reference centroid height above the bottom and the top wall plane, a
// pad, and the reference metric inverse H11, H12, H22 with the reference area A0 (rounded
// once on the host).
constexpr int FGEO = 16;

// Interface parameters of the face kernel, rounded once to the population type on the host
// (FP64 issues at 1/64 of the FP32 rate on this GPU: no per-face conversions).
template <typename real>
struct FaceParams {
  real a3;        // alpha3
  real cL0, cL1;  // 0.5 (alpha1 - alpha3), 0.25 (alpha1 + alpha2)
  real eps48, xi;
  int wall_on;
};

// K3a: one thread per face, in the population type. Writes the strain + wall force of each
// corner, the face's contribution (a x b)/6 to the volume gradient of each of its corners,
// and one partial sum per block of V_j - V0_j, the change of the face's share of the volume.
// With reset != 0 it also clears the tile map that the previous step used.
//
// V_j = (x0 - c) . (a x b) / 6 for a fixed point c. Written with the displacements
// u_k = x_k - X_k from the reference shape (da = u1 - u0, db = u2 - u0, reference edges A, B)
// the change is
//   6 (V_j - V0_j) = u0 . (a x b) + (X0 - c) . (da x b + A x db),
// a sum of terms proportional to the displacement, so float arithmetic loses nothing to the
// cancellation between V and V0 (the per-block partials are summed in double).
template <typename real>
struct FaceArgs {
  int nf;
  const int *faces;
  const Vec4<real> *disp;
  const real *fgeo;
  real *fcontrib, *fnorm;
  double *vol_partial;
  FaceParams<real> fp;
  Dims D;
  int *other_tile_slot;
  const int *other_slot_tile, *other_nslots;
  int reset;
  int *ovf_count;
  unsigned *spill_bits;  // [spill_words] cleared here, before the vertex kernel bins
  int spill_words;
};

// K3a for block `bid` of `nb` (the single-context kernel and the batched one share it).
template <typename real>
__device__ __forceinline__ void face_body(const FaceArgs<real> &A, int bid, int nb) {
  const int nf = A.nf;
  const int *__restrict__ faces = A.faces;
  const Vec4<real> *__restrict__ disp = A.disp;
  const real *__restrict__ fgeo = A.fgeo;
  real *__restrict__ fcontrib = A.fcontrib;
  real *__restrict__ fnorm = A.fnorm;
  double *__restrict__ vol_partial = A.vol_partial;
  const FaceParams<real> fp = A.fp;
  const Dims D = A.D;
  __shared__ double warp_sum[8];
  const int j = bid * blockDim.x + threadIdx.x;
  real dvj = 0;
  if (j < nf) {
    const int iv[3] = {faces[3 * j], faces[3 * j + 1], faces[3 * j + 2]};
    real u[3][3];
    for (int c = 0; c < 3; c++) {
      const Vec4<real> d = disp[iv[c]];
      u[c][0] = d.x;
      u[c][1] = d.y;
      u[c][2] = d.z;
    }
    // A, B, X0 - c, centroid heights above the walls, pad, H11 H12 H22 A0; stored by
    // component ([FGEO][nf]), so that each load of a warp reads one contiguous row
    real geo[FGEO];
#pragma unroll
    for (int k = 0; k < FGEO; k++) geo[k] = k == 11 ? real(0) : fgeo[(size_t)k * nf + j];
    real A[3], B[3], X0c[3], da[3], db[3], a[3], b[3];
    for (int k = 0; k < 3; k++) {
      A[k] = geo[k];
      B[k] = geo[3 + k];
      X0c[k] = geo[6 + k];
      da[k] = u[1][k] - u[0][k];
      db[k] = u[2][k] - u[0][k];
      a[k] = A[k] + da[k];
      b[k] = B[k] + db[k];
    }
    const real H11 = geo[12], H12 = geo[13], H22 = geo[14], A0 = geo[15];
    const real G11 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    const real G12 = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    const real G22 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    const real detG = G11 * G22 - G12 * G12;
    const real L = log_(detG / (real(4) * A0 * A0));  // log(I2 + 1), det G0 = 4 A0^2
    const real dE_dI1 = real(0.5) * fp.a3 * A0;
    const real dE_dL = A0 * (fp.cL0 + fp.cL1 * L);
    const real inv_detG = real(1) / detG;
    real f0[3], f1[3], f2[3];
    for (int k = 0; k < 3; k++) {
      // dE/da and dE/db with I1 = H11 G11 + 2 H12 G12 + H22 G22 - 2, L = log det G + const
      const real ga = dE_dI1 * real(2) * (H11 * a[k] + H12 * b[k]) +
                      dE_dL * real(2) * (a[k] * G22 - G12 * b[k]) * inv_detG;
      const real gb = dE_dI1 * real(2) * (H12 * a[k] + H22 * b[k]) +
                      dE_dL * real(2) * (b[k] * G11 - G12 * a[k]) * inv_detG;
      f1[k] = -ga;
      f2[k] = -gb;
      f0[k] = ga + gb;
    }
    if (fp.wall_on && D.has_walls) {
      // centroid height above each wall plane: reference height (from the set-up, in double)
      // plus the mean displacement
      const real uz = (u[0][2] + u[1][2] + u[2][2]) * real(1.0 / 3.0);
      const real third = (lj_fz<real>(geo[9] + uz, fp.eps48, fp.xi) +
                          lj_fz<real>(geo[10] + uz, fp.eps48, fp.xi)) *
                         real(1.0 / 3.0);
      f0[2] += third;
      f1[2] += third;
      f2[2] += third;
    }
    real *fc = fcontrib + 9 * (size_t)j;
    for (int k = 0; k < 3; k++) {
      fc[k] = f0[k];
      fc[3 + k] = f1[k];
      fc[6 + k] = f2[k];
    }
    // For a closed surface the gradient of V at vertex i does not depend on the point about
    // which the tetrahedra are taken; with that point at x_i every face around i contributes
    // (a x b)/6, the same edge cross product for all three corners.
    const real n[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2],
                       a[0] * b[1] - a[1] * b[0]};
    const real m[3] = {da[1] * b[2] - da[2] * b[1] + A[1] * db[2] - A[2] * db[1],
                       da[2] * b[0] - da[0] * b[2] + A[2] * db[0] - A[0] * db[2],
                       da[0] * b[1] - da[1] * b[0] + A[0] * db[1] - A[1] * db[0]};
    const real sixth = real(1.0 / 6.0);
    real *fn = fnorm + 3 * (size_t)j;
    fn[0] = n[0] * sixth;
    fn[1] = n[1] * sixth;
    fn[2] = n[2] * sixth;
    dvj = (u[0][0] * n[0] + u[0][1] * n[1] + u[0][2] * n[2] + X0c[0] * m[0] + X0c[1] * m[1] +
           X0c[2] * m[2]) * sixth;
  }
  // block sum of V_j - V0_j, fixed shuffle tree (within a warp in the population type)
  real dw = (real)dvj;
  for (int o = 16; o > 0; o >>= 1) dw += __shfl_down_sync(0xffffffffu, dw, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = (double)dw;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? warp_sum[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) vol_partial[bid] = v;
  }
  if (bid == 0 && threadIdx.x == 0) {
    A.ovf_count[0] = 0;  // vertices beyond their bucket (a count only)
    A.ovf_count[2] = 0;  // number of source tiles (counters[4])
    A.ovf_count[3] = 0;  // listed force pairs (counters[5]), appended by K4b
  }
  for (int w = bid * blockDim.x + threadIdx.x; w < A.spill_words; w += nb * blockDim.x)
    A.spill_bits[w] = 0u;
  if (A.reset) {
    const int n_other = min(*A.other_nslots, D.max_slots);
    for (int s = bid * blockDim.x + threadIdx.x; s < n_other; s += nb * blockDim.x)
      A.other_tile_slot[A.other_slot_tile[s]] = -1;
  }
}

template <typename real>
__global__ void __launch_bounds__(256) face_kernel(const FaceArgs<real> A) {
  face_body(A, blockIdx.x, gridDim.x);
}

template <typename real>
__global__ void __launch_bounds__(256) face_kernel_multi(const FaceArgs<real> *__restrict__ all,
                                                         const int *__restrict__ start, int n) {
  const MultiBlock m = multi_block(start, n);
  face_body(all[m.inst], m.block, m.nblocks);
}

// kV (V - V0)/V0 from the per-block partial sums of V - V0, by one warp in a fixed order;
// also returns V.
__device__ __forceinline__ double volume_coef(const double *__restrict__ part, int n, double V0,
                                              double kV, int volume_on, double *V_out) {
  double dv = 0.0;
  for (int k = threadIdx.x & 31; k < n; k += 32) dv += part[k];
  for (int o = 16; o > 0; o >>= 1) dv += __shfl_down_sync(0xffffffffu, dv, o);
  dv = __shfl_sync(0xffffffffu, dv, 0);
  if (V_out) *V_out = V0 + dv;
  return volume_on ? kV * dv / V0 : 0.0;
}

// One-dimensional Peskin weights of the four nodes floor(p)-1 .. floor(p)+2 (Eq. 15).
// With r = p - floor(p) and s = sqrt(1 + 4r - 4r^2) the four branches reduce to
// (3-2r-s)/8, (3-2r+s)/8, (1+2r+s)/8, (1+2r-s)/8, which sum to one.
template <typename real>
__device__ __forceinline__ void peskin_weights(double p, int &base, real w[4]) {
  const double fl = floor(p);
  base = (int)fl - 1;
  const real r = (real)(p - fl);
  const real s = sqrt_(real(1) + real(4) * r - real(4) * r * r);
  w[0] = (real(3) - real(2) * r - s) * real(0.125);
  w[1] = (real(3) - real(2) * r + s) * real(0.125);
  w[2] = (real(1) + real(2) * r + s) * real(0.125);
  w[3] = (real(1) + real(2) * r - s) * real(0.125);
}

// Faces around a vertex gathered with all loads in flight (icosphere valences are 5 and 6).
constexpr int GATHER_UNROLL = 8;

// K3b: one thread per vertex. Gathers, in face order, the strain + wall force of the vertex's
// corners (phi, Eq. 16 without the volume term) and its volume gradient g = dV/dq_i; the
// volume term -kV (V - V0)/V0 g is added where the force is used (spreading, read-back),
// after V is complete. Then the delta stencil of the vertex and its binning into the source
// tile (the tile that holds its base node).
struct VolumeParams {
  double V0, kV;
  int volume_on, vol_blocks;
};

template <typename real>
struct VertexArgs {
  int nv;
  const int *vf_start, *vf_list;
  const real *fcontrib, *fnorm;
  const double *q;
  Vec4<real> *phi, *gvol;
  StencilRec<real> *stencil;
  int bin;
  const int *tile_slot;
  int *slot_count, *bucket, *ovf_count, *src_index, *nsources, *health, *zero_counter;
  unsigned *spill_bits;  // bit i: vertex i did not fit in its tile's bucket
  const double *vol_partial;  // per-block V_j - V0_j partials of the face kernel
  VolumeParams vp;
  real *vcoef;                // out: kV (V - V0)/V0 for the spreading pass
  Dims D;
};

template <typename real>
__device__ __forceinline__ void vertex_body(const VertexArgs<real> &A, int bid) {
  const int nv = A.nv;
  const int *__restrict__ vf_start = A.vf_start;
  const int *__restrict__ vf_list = A.vf_list;
  const real *__restrict__ fcontrib = A.fcontrib;
  const real *__restrict__ fnorm = A.fnorm;
  const double *__restrict__ q = A.q;
  const int bin = A.bin;
  const Dims D = A.D;
  const int i = bid * blockDim.x + threadIdx.x;
  if (bid == 0 && threadIdx.x == 0 && A.zero_counter) *A.zero_counter = 0;
  if (bid == 0 && threadIdx.x < 32) {
    // the volume-force coefficient of the step, once (the spreading pass reads it), and the
    // volume health check
    double V;
    const real coef = (real)volume_coef(A.vol_partial, A.vp.vol_blocks, A.vp.V0, A.vp.kV,
                                        A.vp.volume_on, &V);
    if (threadIdx.x == 0) {
      *A.vcoef = coef;
      if (!(fabs(V / A.vp.V0 - 1.0) <= 0.05)) atomicOr(A.health, H_VOLUME);
    }
  }
  if (i >= nv) return;
  const int e0 = vf_start[i], e1 = vf_start[i + 1];
  real F[3] = {0, 0, 0}, g[3] = {0, 0, 0};
  for (int eb = e0; eb < e1; eb += GATHER_UNROLL) {
    int fcs[GATHER_UNROLL];
#pragma unroll
    for (int u = 0; u < GATHER_UNROLL; u++) fcs[u] = eb + u < e1 ? vf_list[eb + u] : -1;
#pragma unroll
    for (int u = 0; u < GATHER_UNROLL; u++) {
      if (fcs[u] < 0) continue;
      const int fc = fcs[u];  // face * 3 + corner
      const int f = fc / 3;
      for (int k = 0; k < 3; k++) {
        F[k] += fcontrib[3 * (size_t)fc + k];
        g[k] += fnorm[3 * (size_t)f + k];
      }
    }
  }
  Vec4<real> pv, gv;
  pv.x = F[0]; pv.y = F[1]; pv.z = F[2]; pv.w = real(0);
  gv.x = g[0]; gv.y = g[1]; gv.z = g[2]; gv.w = real(0);
  A.phi[i] = pv;
  A.gvol[i] = gv;
  if (!bin) return;
  StencilRec<real> rec;
  peskin_weights<real>(wrap_pos(q[3 * (size_t)i], D.nx, D.inx), rec.base[0], rec.w[0]);
  peskin_weights<real>(wrap_pos(q[3 * (size_t)i + 1], D.ny, D.iny), rec.base[1], rec.w[1]);
  const double pz = q[3 * (size_t)i + 2];
  peskin_weights<real>(D.has_walls ? pz : wrap_pos(pz, D.nz, D.inz), rec.base[2], rec.w[2]);
  // base in [-2, n - 1] on the periodic axes (rounding of the wrap): bring it into [0, n)
  if (rec.base[0] < 0) rec.base[0] += D.nx;
  if (rec.base[1] < 0) rec.base[1] += D.ny;
  if (!D.has_walls && rec.base[2] < 0) rec.base[2] += D.nz;
  rec.pad = 0;
  A.stencil[i] = rec;
  const int bz = min(max(rec.base[2], 0), D.nz - 1);
  const int t = ((bz >> 2) * D.nty + (rec.base[1] >> 2)) * D.ntx + (rec.base[0] >> 2);
  const int s = A.tile_slot[t];
  if (s < 0) {
    atomicOr(A.health, H_CAPACITY);
    return;
  }
  const int rank = atomicAdd(&A.slot_count[s], 1);
  if (rank == 0) A.src_index[s] = atomicAdd(A.nsources, 1);  // first vertex: the tile gets a region
  if (rank < BUCKET_CAP) {
    A.bucket[(size_t)s * BUCKET_CAP + rank] = i;
  } else {
    // which vertices end up in the bucket depends on the order of the atomics; the spread
    // pass therefore adds every vertex of a tile that spilled in vertex-index order
    atomicAdd(A.ovf_count, 1);
    atomicOr(&A.spill_bits[i >> 5], 1u << (i & 31));
  }
}

template <typename real>
__global__ void __launch_bounds__(256) vertex_kernel(const VertexArgs<real> A) {
  vertex_body(A, blockIdx.x);
}

template <typename real>
__global__ void __launch_bounds__(256) vertex_kernel_multi(
    const VertexArgs<real> *__restrict__ all, const int *__restrict__ start, int n) {
  const MultiBlock m = multi_block(start, n);
  vertex_body(all[m.inst], m.block);
}

// Spreading works on regions: the stencils of the vertices binned in a source tile S (base
// node in S) cover the 7x7x7 nodes S_lo .. S_lo + 6.
constexpr int REGION = 7;
constexpr int REGION_NODES = REGION * REGION * REGION;
// Source tiles per block of K4a (shared memory per warp: the region and the staged records).
template <typename real>
struct SrcWarps {
  static constexpr int value = sizeof(real) == 4 ? 4 : 2;
};

// w[d] for a run-time d in 0..3 without indexing a local array.
template <typename real>
__device__ __forceinline__ real pick4(const real w[4], int d) {
  return d == 0 ? w[0] : d == 1 ? w[1] : d == 2 ? w[2] : w[3];
}

// K4a: spreading, first pass (Eq. 13). One warp per source tile S: its bucket is sorted by
// vertex index (rank by comparison, at most 64 entries), the vertices' stencil records and
// forces (completed with the volume term -kV (V - V0)/V0 dV/dq) are staged in shared memory,
// and the vertices are then added one after another into the 7x7x7 region of S, each lane
// adding two of the 64 stencil nodes of a vertex (distinct nodes, so no atomics). The region
// is written out and its index pushed to the (up to 8) tiles T = S + {0,1}^3 it overlaps.
// A tile with more than 64 vertices (its bucket holds 64 of them, chosen by the order of the
// binning atomics) marks its bucket's vertices in the spill bitmap, which already holds its
// spilled ones, and adds all of its vertices in increasing vertex index instead, found by a
// scan of the bitmap. Either way the order of summation depends only on the vertex set.
template <typename real>
struct SourceArgs {
  const int *tile_slot, *slot_tile, *nslots_ptr, *slot_count, *src_index, *bucket;
  unsigned *spill_bits;
  int spill_words;
  const StencilRec<real> *stencil;
  const Vec4<real> *phi, *gvol;
  const real *vcoef;  // kV (V - V0)/V0, written by the vertex kernel of the step
  Vec4<real> *Rslot;
  int *out_src;
  Dims D;
};

template <typename real>
__device__ __forceinline__ void spread_source_body(const SourceArgs<real> &A, int bid, int nb) {
  const int *__restrict__ tile_slot = A.tile_slot;
  const int *__restrict__ slot_tile = A.slot_tile;
  const int *__restrict__ slot_count = A.slot_count;
  const int *__restrict__ src_index = A.src_index;
  const int *__restrict__ bucket = A.bucket;
  unsigned *spill_bits = A.spill_bits;
  const StencilRec<real> *__restrict__ stencil = A.stencil;
  const Vec4<real> *__restrict__ phi = A.phi;
  const Vec4<real> *__restrict__ gvol = A.gvol;
  int *__restrict__ out_src = A.out_src;
  const Dims D = A.D;
  constexpr int W = SrcWarps<real>::value;
  __shared__ Vec4<real> s_region[W][REGION_NODES];
  __shared__ real s_w[W][BUCKET_CAP][12];
  __shared__ Vec4<real> s_f[W][BUCKET_CAP];
  __shared__ int s_b[W][BUCKET_CAP][3];
  const int nslots = min(*A.nslots_ptr, D.max_slots);
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const real coef = *A.vcoef;
  Vec4<real> *region = s_region[wq];
  // the two stencil nodes of this lane
  const int dxa = lane & 3, dya = (lane >> 2) & 3, dza = lane >> 4;  // node lane; node lane + 32
  for (int s = bid * W + wq; s < nslots; s += nb * W) {
    const int cnt = slot_count[s];
    if (cnt == 0) continue;  // no vertex has its base node here: no region
    const int n = min(cnt, BUCKET_CAP);
    const int t = slot_tile[s];
    const int tsx = t % D.ntx, tsy = (t / D.ntx) % D.nty, tsz = t / (D.ntx * D.nty);
    const int Sx = tsx * TILE, Sy = tsy * TILE, Sz = tsz * TILE;
    const int reg = src_index[s];
    // push the region to the tiles it overlaps: T = S + e, seen from T as source e
    if (lane < 8) {
      int ux = tsx + (lane & 1), uy = tsy + ((lane >> 1) & 1), uz = tsz + (lane >> 2);
      ux = ux >= D.ntx ? ux - D.ntx : ux;
      uy = uy >= D.nty ? uy - D.nty : uy;
      bool ok = true;
      if (uz >= D.ntz) {
        if (D.has_walls) ok = false;
        uz -= D.ntz;
      }
      if (ok) {
        const int slot_t = tile_slot[(uz * D.nty + uy) * D.ntx + ux];
        if (slot_t >= 0) out_src[8 * (size_t)slot_t + lane] = reg;
      }
    }
    const int *bk = bucket + (size_t)s * BUCKET_CAP;
    if (cnt <= BUCKET_CAP) {
      // sort the bucket by vertex index and stage the records in that order
      const int v0 = lane < n ? bk[lane] : 0x7fffffff;
      const int v1 = lane + 32 < n ? bk[lane + 32] : 0x7fffffff;
      int r0 = 0, r1 = 0;
      for (int m = 0; m < n; m++) {
        const int vm = __shfl_sync(0xffffffffu, m < 32 ? v0 : v1, m & 31);
        r0 += vm < v0;
        r1 += vm < v1;
      }
      for (int h = 0; h < 2; h++) {
        const int v = h ? v1 : v0;
        const int r = h ? r1 : r0;
        if ((h ? lane + 32 : lane) >= n) continue;
        const StencilRec<real> rec = stencil[v];
        const Vec4<real> pv = phi[v], gv = gvol[v];
        for (int k = 0; k < 4; k++) {
          s_w[wq][r][k] = rec.w[0][k];
          s_w[wq][r][4 + k] = rec.w[1][k];
          s_w[wq][r][8 + k] = rec.w[2][k];
        }
        s_f[wq][r] = Vec4<real>{pv.x - coef * gv.x, pv.y - coef * gv.y, pv.z - coef * gv.z, real(0)};
        // base relative to S_lo (x, y wrapped into [0, n) by the vertex kernel)
        s_b[wq][r][0] = rec.base[0] - Sx;
        s_b[wq][r][1] = rec.base[1] - Sy;
        s_b[wq][r][2] = rec.base[2] - Sz;
      }
      for (int k = lane; k < REGION_NODES; k += 32) region[k] = Vec4<real>{0, 0, 0, 0};
      __syncwarp();
      for (int c = 0; c < n; c++) {
        const int bx = s_b[wq][c][0], by = s_b[wq][c][1], bz = s_b[wq][c][2];
        const Vec4<real> f = s_f[wq][c];
        const real wxy = s_w[wq][c][dxa] * s_w[wq][c][4 + dya];
        for (int h = 0; h < 2; h++) {
          const int dz = dza + 2 * h;  // node lane + 32 h has the same dx, dy and dz + 2
          const int rz = bz + dz;
          if (rz < 0 || rz >= REGION) continue;  // beyond the lattice in z
          const real w = wxy * s_w[wq][c][8 + dz];
          Vec4<real> &o = region[(rz * REGION + by + dya) * REGION + bx + dxa];
          o.x += w * f.x;
          o.y += w * f.y;
          o.z += w * f.z;
          o.w = real(1);  // a stencil node of some vertex (the interpolation reads it)
        }
        __syncwarp();
      }
    } else {
      // the tile spilled: mark its bucket's vertices too, then add every vertex of the tile in
      // increasing index (bitmap words read through L2, where the atomics are performed)
      atomicOr(&spill_bits[bk[lane] >> 5], 1u << (bk[lane] & 31));
      atomicOr(&spill_bits[bk[lane + 32] >> 5], 1u << (bk[lane + 32] & 31));
      for (int k = lane; k < REGION_NODES; k += 32) region[k] = Vec4<real>{0, 0, 0, 0};
      __syncwarp();
      for (int wb = 0; wb < A.spill_words; wb += 32) {
        const unsigned word_l = wb + lane < A.spill_words ? __ldcg(&spill_bits[wb + lane]) : 0u;
        unsigned nonzero = __ballot_sync(0xffffffffu, word_l != 0u);
        while (nonzero) {
          const int l = __ffs(nonzero) - 1;
          nonzero &= nonzero - 1;
          const unsigned word = __shfl_sync(0xffffffffu, word_l, l);
          const int vl = (wb + l) * 32 + lane;  // this lane's vertex of the word
          bool mine = false;
          if ((word >> lane) & 1u) {
            const StencilRec<real> rl = stencil[vl];
            const int bzc = min(max(rl.base[2], 0), D.nz - 1);
            mine = (rl.base[0] >> 2) == tsx && (rl.base[1] >> 2) == tsy && (bzc >> 2) == tsz;
          }
          unsigned members = __ballot_sync(0xffffffffu, mine);
          while (members) {  // the tile's vertices of this word, in index order
            const int b = __ffs(members) - 1;
            members &= members - 1;
            const int v = (wb + l) * 32 + b;
            const StencilRec<real> rec = stencil[v];
            const int bx = rec.base[0] - Sx, by = rec.base[1] - Sy, bz = rec.base[2] - Sz;
            const Vec4<real> pv = phi[v], gv = gvol[v];
            const real fx = pv.x - coef * gv.x, fy = pv.y - coef * gv.y, fz = pv.z - coef * gv.z;
            const real wxy = pick4(rec.w[0], dxa) * pick4(rec.w[1], dya);
            for (int h = 0; h < 2; h++) {
              const int dz = dza + 2 * h;
              const int rz = bz + dz;
              if (rz < 0 || rz >= REGION) continue;
              const real w = wxy * pick4(rec.w[2], dz);
              Vec4<real> &o = region[(rz * REGION + by + dya) * REGION + bx + dxa];
              o.x += w * fx;
              o.y += w * fy;
              o.z += w * fz;
              o.w = real(1);
            }
            __syncwarp();
          }
        }
      }
    }
    Vec4<real> *out = A.Rslot + (size_t)reg * REGION_NODES;
    for (int k = lane; k < REGION_NODES; k += 32) out[k] = region[k];
    __syncwarp();
  }
}

template <typename real>
__global__ void __launch_bounds__(32 * SrcWarps<real>::value) spread_source_kernel(
    const SourceArgs<real> A) {
  spread_source_body(A, blockIdx.x, gridDim.x);
}

template <typename real>
__global__ void __launch_bounds__(32 * SrcWarps<real>::value) spread_source_kernel_multi(
    const SourceArgs<real> *__restrict__ all, const int *__restrict__ start, int n) {
  const MultiBlock m = multi_block(start, n);
  spread_source_body(all[m.inst], m.block, m.nblocks);
}

// K4b: spreading, second pass. One 64-thread block per active tile T (grid-stride), thread =
// node (lx, ly, lz): the force is the sum, in the fixed order e = 0..7, of the regions of the
// source tiles S = T - e pushed by K4a; the node sits at (l + 4 e) in S's region. On a
// periodic axis only 4 nodes long S - e and S coincide and the two terms are the node's two
// images in the region. Force landing on a wall layer is dropped. K4a marks each region
// node that lies in a vertex's stencil (w = 1); K4b lists the node pairs holding such a node,
// the work of the active-tile correction (K1t) and of the shell velocity (K1b).
template <typename real>
struct GatherArgs {
  const int *slot_tile, *nslots_ptr, *out_src;
  const Vec4<real> *Rslot;
  Vec4<real> *Fslot;
  int *pair_list, *npairs;  // node pairs (x even, x + 1) in some vertex's stencil, for K1t, K1b
  Dims D;
};

template <typename real>
__device__ __forceinline__ void spread_gather_body(const GatherArgs<real> &A, int bid, int nb) {
  const int *__restrict__ slot_tile = A.slot_tile;
  const int *__restrict__ out_src = A.out_src;
  const Vec4<real> *__restrict__ Rslot = A.Rslot;
  Vec4<real> *__restrict__ Fslot = A.Fslot;
  const Dims D = A.D;
  const int nslots = min(*A.nslots_ptr, D.max_slots);
  const int tid = threadIdx.x;
  const int lx = tid & 3, ly = (tid >> 2) & 3, lz = tid >> 4;
  for (int b = bid; b < nslots; b += nb) {
    const int *src = out_src + 8 * (size_t)b;
    real f[3] = {0, 0, 0};
    bool stencil_node = false;
    for (int e = 0; e < 8; e++) {
      const int reg = src[e];
      const int rx = lx + 4 * (e & 1), ry = ly + 4 * ((e >> 1) & 1), rz = lz + 4 * (e >> 2);
      if (reg < 0 || rx >= REGION || ry >= REGION || rz >= REGION) continue;
      const Vec4<real> r = Rslot[(size_t)reg * REGION_NODES + (rz * REGION + ry) * REGION + rx];
      f[0] += r.x;
      f[1] += r.y;
      f[2] += r.z;
      stencil_node |= r.w != real(0);
    }
    const int Z = (slot_tile[b] / (D.ntx * D.nty)) * TILE + lz;
    const bool drop = D.has_walls && (Z == 0 || Z >= D.nz - 1);
    Vec4<real> o;
    o.x = drop ? real(0) : f[0];
    o.y = drop ? real(0) : f[1];
    o.z = drop ? real(0) : f[2];
    o.w = real(0);
    Fslot[(size_t)b * TILE_CELLS + tid] = o;
    // list the pairs (tid even, tid + 1) of this warp of which either node is a fluid node of
    // some vertex's stencil (every node that can carry a force, and every node the
    // interpolation reads off the wall layers): one atomic per warp, entries in pair order
    // within the warp
    const unsigned m = __ballot_sync(0xffffffffu, stencil_node && !drop);
    const unsigned pm = (m | (m >> 1)) & 0x55555555u;  // bit 2k: pair k is listed
    const int lane = tid & 31;
    int base = 0;
    if (lane == 0 && pm) base = atomicAdd(A.npairs, __popc(pm));
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((pm >> lane) & 1u)
      A.pair_list[base + __popc(pm & ((1u << lane) - 1u))] = 32 * b + (tid >> 1);
  }
}

template <typename real>
__global__ void __launch_bounds__(64) spread_gather_kernel(const GatherArgs<real> A) {
  spread_gather_body(A, blockIdx.x, gridDim.x);
}

template <typename real>
__global__ void __launch_bounds__(64) spread_gather_kernel_multi(
    const GatherArgs<real> *__restrict__ all, const int *__restrict__ start, int n) {
  const MultiBlock m = multi_block(start, n);
  spread_gather_body(all[m.inst], m.block, m.nblocks);
}

// Claim tile t in map (tile_slot, slot_tile, nslots): the first claimant takes a new slot.
// A plain read first keeps the many vertices of an already-claimed tile off the atomic.
__device__ __forceinline__ void claim_tile(int t, int *tile_slot, int *slot_tile, int *nslots,
                                           int *slot_count, int *out_src, int *health,
                                           int max_slots) {
  if (*(volatile int *)&tile_slot[t] != -1) return;
  if (atomicCAS(&tile_slot[t], -1, -2) == -1) {
    const int s = atomicAdd(nslots, 1);
    if (s < max_slots) {
      slot_tile[s] = t;
      slot_count[s] = 0;
      for (int e = 0; e < 8; e++) out_src[8 * (size_t)s + e] = -1;
      atomicExch(&tile_slot[t], s);
    } else {
      atomicOr(health, H_CAPACITY);
    }
  }
}

// Tiles covered along one axis by the stencil of coordinate p: t0 (lower) and t1 (upper,
// equal to t0 when the four nodes fall in one tile); `ok1` tells whether t1 is a distinct
// tile that exists. Periodic axes wrap; along a walled z axis tiles beyond the lattice are
// skipped (valid flags).
struct AxisTiles {
  int t0, t1;
  bool ok0, ok1;
};

__device__ __forceinline__ AxisTiles axis_tiles(double p, int nt, double inv_n, bool periodic) {
  AxisTiles a;
  if (periodic) p = wrap_pos(p, 4 * nt, inv_n);
  const int b = (int)floor(p) - 1;
  int t0 = floor_div4(b), t1 = floor_div4(b + 3);
  a.ok1 = t1 != t0;
  if (periodic) {  // b in [-2, 4 nt - 1]: t0 in [-1, nt - 1], t1 in [0, nt]
    t0 = t0 < 0 ? t0 + nt : t0;
    t1 = t1 >= nt ? t1 - nt : t1;
    a.ok0 = true;
    a.ok1 = a.ok1 && t1 != t0;  // a short periodic axis may wrap onto the same tile
  } else {
    a.ok0 = t0 >= 0 && t0 < nt;
    a.ok1 = a.ok1 && t1 >= 0 && t1 < nt;
  }
  a.t0 = t0;
  a.t1 = t1;
  return a;
}

// Claim, in map (tile_slot, slot_tile, nslots), tile e (bit k picks the upper tile along
// axis k) of the stencil described by ax.
__device__ __forceinline__ void mark_tile(const AxisTiles ax[3], int e, const Dims &D,
                                          int *tile_slot, int *slot_tile, int *nslots,
                                          int *slot_count, int *out_src, int *health) {
  int t[3];
  for (int k = 0; k < 3; k++) {
    const bool up = (e >> k) & 1;
    if (up ? !ax[k].ok1 : !ax[k].ok0) return;
    t[k] = up ? ax[k].t1 : ax[k].t0;
  }
  claim_tile((t[2] * D.nty + t[1]) * D.ntx + t[0], tile_slot, slot_tile, nslots, slot_count,
             out_src, health, D.max_slots);
}

// K2: interpolation (Eq. 11) and the Euler update (Eq. 12); 4 lanes per vertex, lane dz
// sums the 16 nodes of its z-plane of the stencil, the 4 planes are summed by shuffles and
// the update is added to the double position by lane 0, which also finds the tiles of the new
// stencil; each lane then marks two of those (up to 8) tiles in the other map.
// The delta-weight accumulation of a vertex is carried at double precision in every
// precision (VertexSum): each stencil row's four products w_x u (one x row of a tile, in the
// arithmetic type) is added to the vertex's sum with its weight w_y w_z, and the four planes'
// sums are added across the lanes, without rounding the sum back to float.
template <typename real>
struct VertexSum;

// FP64 contexts: a plain double sum.
template <>
struct VertexSum<double> {
  double s[3] = {0.0, 0.0, 0.0};
  __device__ __forceinline__ void add_prod(int k, double a, double b) { s[k] += a * b; }
  __device__ __forceinline__ void set(int k, double x) { s[k] = x; }
  __device__ __forceinline__ void add_lanes(int o) {
    for (int k = 0; k < 3; k++) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
  }
  __device__ __forceinline__ double value(int k) const { return s[k]; }
};

// Float contexts: the sum is a pair of floats hi + lo (double-float arithmetic), kept exact
// up to rounding at about 2^-44 of the sum with the error-free transformations of Dekker
// (the product a b = p + e, e by a fused multiply-add) and Knuth (TwoSum: s + err = x + y).
// This is as accurate as a double sum of the same float products; on GB300 double arithmetic
// runs at 1/64 of the float rate, and the double form lengthened the 16-bit step. The _rn
// intrinsics keep the compiler from fusing the steps the transformations rely on.
template <>
struct VertexSum<float> {
  float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f};
  __device__ __forceinline__ void add(int k, float x, float xerr) {
    const float s = __fadd_rn(hi[k], x);
    const float bp = __fsub_rn(s, hi[k]);
    const float err = __fadd_rn(__fsub_rn(hi[k], __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi[k] = s;
    lo[k] = __fadd_rn(lo[k], __fadd_rn(err, xerr));
  }
  __device__ __forceinline__ void add_prod(int k, float a, float b) {
    const float p = __fmul_rn(a, b);
    add(k, p, __fmaf_rn(a, b, -p));
  }
  __device__ __forceinline__ void set(int k, double x) {
    hi[k] = __double2float_rn(x);
    lo[k] = __double2float_rn(x - (double)hi[k]);
  }
  // the same result in every lane of the butterfly: the addition is commutative and TwoSum's
  // error term is exact
  __device__ __forceinline__ void add_lanes(int o) {
    for (int k = 0; k < 3; k++) {
      const float h = __shfl_xor_sync(0xffffffffu, hi[k], o);
      const float l = __shfl_xor_sync(0xffffffffu, lo[k], o);
      lo[k] = __fadd_rn(lo[k], l);
      add(k, h, 0.f);
    }
  }
  __device__ __forceinline__ double value(int k) const { return (double)hi[k] + (double)lo[k]; }
};

template <typename real>
struct InterpArgs {
  int nv;
  const StencilRec<real> *stencil;
  const int *tile_slot;
  const Vec4<real> *Uslot;
  double *q, *qdot;
  const double *xref;
  Vec4<real> *disp;
  double3 ub, ut;
  Dims D;
  int *next_tile_slot, *next_slot_tile, *next_nslots, *slot_count, *out_src, *health;
};

template <typename real>
__device__ __forceinline__ void interp_body(const InterpArgs<real> &A, int bid) {
  const int nv = A.nv;
  const StencilRec<real> *__restrict__ stencil = A.stencil;
  const int *__restrict__ tile_slot = A.tile_slot;
  const Vec4<real> *__restrict__ Uslot = A.Uslot;
  double *__restrict__ q = A.q;
  double *__restrict__ qdot = A.qdot;
  const double *__restrict__ xref = A.xref;
  Vec4<real> *__restrict__ disp = A.disp;
  const double3 ub = A.ub, ut = A.ut;
  const Dims D = A.D;
  int *next_tile_slot = A.next_tile_slot;
  int *__restrict__ health = A.health;
  const int gid = bid * blockDim.x + threadIdx.x;
  const int v = gid >> 2;
  const int dz = gid & 3;
  const bool valid = v < nv;
  VertexSum<real> acc;
  if (valid) {
    const StencilRec<real> rec = stencil[v];
    int Z = rec.base[2] + dz;
    if (!D.has_walls) Z = Z >= D.nz ? Z - D.nz : Z;
    if (Z >= 0 && Z < D.nz) {
      const real wz = pick4(rec.w[2], dz);
      if (D.has_walls && (Z == 0 || Z == D.nz - 1)) {
        const double3 w = Z == 0 ? ub : ut;
        const double sxy =
            ((double)rec.w[0][0] + (double)rec.w[0][1] + (double)rec.w[0][2] + (double)rec.w[0][3]) *
            ((double)rec.w[1][0] + (double)rec.w[1][1] + (double)rec.w[1][2] + (double)rec.w[1][3]) *
            (double)wz;
        acc.set(0, sxy * w.x);
        acc.set(1, sxy * w.y);
        acc.set(2, sxy * w.z);
      } else {
        // the 4 stencil nodes along x (and along y) fall in at most two tiles: look up the
        // (up to) four tile slots of this z-plane once
        int X[4], Y[4];
        for (int d = 0; d < 4; d++) {
          const int xx = rec.base[0] + d, yy = rec.base[1] + d;
          X[d] = xx >= D.nx ? xx - D.nx : xx;
          Y[d] = yy >= D.ny ? yy - D.ny : yy;
        }
        const int tzrow = (Z >> 2) * D.nty;
        int sl[2][2];
        for (int iy = 0; iy < 2; iy++)
          for (int ix = 0; ix < 2; ix++)
            sl[iy][ix] = tile_slot[(tzrow + (Y[3 * iy] >> 2)) * D.ntx + (X[3 * ix] >> 2)];
        for (int dy = 0; dy < 4; dy++) {
          const int iy = (Y[dy] >> 2) != (Y[0] >> 2);
          const int crow = 4 * (Y[dy] & 3) + 16 * (Z & 3);
          real r3[3] = {0, 0, 0};
          for (int dx = 0; dx < 4; dx++) {
            const int sidx = sl[iy][(X[dx] >> 2) != (X[0] >> 2)];
            if (sidx < 0) {  // unmarked tile: only after a capacity failure, flagged there
              atomicOr(health, H_CAPACITY);
              continue;
            }
            const Vec4<real> u = Uslot[(size_t)sidx * TILE_CELLS + (X[dx] & 3) + crow];
            const real w = rec.w[0][dx];
            r3[0] += w * u.x;
            r3[1] += w * u.y;
            r3[2] += w * u.z;
          }
          const real wyz = rec.w[1][dy] * wz;
          acc.add_prod(0, wyz, r3[0]);
          acc.add_prod(1, wyz, r3[1]);
          acc.add_prod(2, wyz, r3[2]);
        }
      }
    }
  }
  // sum of the 4 planes (fixed butterfly order)
  for (int o = 2; o > 0; o >>= 1) acc.add_lanes(o);
  // lane dz == 0 updates the vertex in double and finds the tiles of its new stencil; the
  // other three lanes take the tiles from it (FP64 issues at 1/64 of the FP32 rate on this
  // GPU, so that work is done once per vertex)
  int tq[6] = {0, 0, 0, 0, 0, 0};  // t0, t1 of each axis
  int flags = 0;                   // bit 2k / 2k + 1: ok0 / ok1 of axis k; bit 6: mark
  if (valid && dz == 0) {
    double pn[3], qd[3];
    int h = 0;
    for (int k = 0; k < 3; k++) {
      qd[k] = acc.value(k);
      pn[k] = q[3 * (size_t)v + k] + qd[k];
      qdot[3 * (size_t)v + k] = qd[k];
      q[3 * (size_t)v + k] = pn[k];
      if (!(fabs(qd[k]) < 0.1)) h |= (qd[k] == qd[k]) ? H_FAST : H_NAN;
    }
    if (D.has_walls && (pn[2] - D.zb < 0.05 || D.zt - pn[2] < 0.05)) h |= H_WALL;
    if (h) atomicOr(health, h);
    Vec4<real> d;
    d.x = (real)(pn[0] - xref[3 * (size_t)v]);
    d.y = (real)(pn[1] - xref[3 * (size_t)v + 1]);
    d.z = (real)(pn[2] - xref[3 * (size_t)v + 2]);
    d.w = real(0);
    disp[v] = d;
    if (next_tile_slot != nullptr && pn[0] == pn[0] && pn[1] == pn[1] && pn[2] == pn[2]) {
      const AxisTiles ax[3] = {axis_tiles(pn[0], D.ntx, D.inx, true),
                               axis_tiles(pn[1], D.nty, D.iny, true),
                               axis_tiles(pn[2], D.ntz, D.inz, !D.has_walls)};
      for (int k = 0; k < 3; k++) {
        tq[2 * k] = ax[k].t0;
        tq[2 * k + 1] = ax[k].t1;
        flags |= (ax[k].ok0 ? 1 : 0) << (2 * k) | (ax[k].ok1 ? 1 : 0) << (2 * k + 1);
      }
      flags |= 64;
    }
  }
  for (int k = 0; k < 6; k++) tq[k] = __shfl_sync(0xffffffffu, tq[k], 0, 4);
  flags = __shfl_sync(0xffffffffu, flags, 0, 4);
  if (valid && (flags & 64)) {  // each lane claims two of the (up to 8) tiles
    AxisTiles ax[3];
    for (int k = 0; k < 3; k++) {
      ax[k].t0 = tq[2 * k];
      ax[k].t1 = tq[2 * k + 1];
      ax[k].ok0 = (flags >> (2 * k)) & 1;
      ax[k].ok1 = (flags >> (2 * k + 1)) & 1;
    }
    mark_tile(ax, dz, D, next_tile_slot, A.next_slot_tile, A.next_nslots, A.slot_count,
              A.out_src, health);
    mark_tile(ax, dz + 4, D, next_tile_slot, A.next_slot_tile, A.next_nslots, A.slot_count,
              A.out_src, health);
  }
}

template <typename real>
__global__ void __launch_bounds__(256) interp_kernel(const InterpArgs<real> A) {
  interp_body(A, blockIdx.x);
}

template <typename real>
__global__ void __launch_bounds__(256) interp_kernel_multi(
    const InterpArgs<real> *__restrict__ all, const int *__restrict__ start, int n) {
  const MultiBlock m = multi_block(start, n);
  interp_body(all[m.inst], m.block);
}

// Standalone marking of the current positions (after setting vertices); also refreshes the
// float displacement from the reference shape.
template <typename real>
__global__ void mark_kernel(int nv, const double *__restrict__ q, const double *__restrict__ xref,
                            Vec4<real> *__restrict__ disp, Dims D, int *tile_slot,
                            int *slot_tile, int *nslots, int *slot_count, int *out_src,
                            int *health) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = gid >> 3, e = gid & 7;
  if (v >= nv) return;
  const double p[3] = {q[3 * (size_t)v], q[3 * (size_t)v + 1], q[3 * (size_t)v + 2]};
  if (e == 0) {
    Vec4<real> d;
    d.x = (real)(p[0] - xref[3 * (size_t)v]);
    d.y = (real)(p[1] - xref[3 * (size_t)v + 1]);
    d.z = (real)(p[2] - xref[3 * (size_t)v + 2]);
    d.w = real(0);
    disp[v] = d;
  }
  if (p[0] == p[0] && p[1] == p[1] && p[2] == p[2]) {
    AxisTiles ax[3];
    ax[0] = axis_tiles(p[0], D.ntx, D.inx, true);
    ax[1] = axis_tiles(p[1], D.nty, D.iny, true);
    ax[2] = axis_tiles(p[2], D.ntz, D.inz, !D.has_walls);
    mark_tile(ax, e, D, tile_slot, slot_tile, nslots, slot_count, out_src, health);
  }
}

__global__ void clear_counts_kernel(const int *__restrict__ nslots, int *__restrict__ slot_count,
                                    int *__restrict__ ovf_count, int max_slots) {
  const int n = min(*nslots, max_slots);
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
    slot_count[s] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ovf_count[0] = 0;
    ovf_count[2] = 0;
    ovf_count[3] = 0;
  }
}

template <typename real>
__global__ void expand_force_kernel(const int *__restrict__ slot_tile, const int *__restrict__ nslots,
                                    const Vec4<real> *__restrict__ Fslot, Dims D,
                                    double *__restrict__ F) {
  const int n = min(*nslots, D.max_slots);
  for (int b = blockIdx.x; b < n; b += gridDim.x) {
    const int t = slot_tile[b];
    const int tx = t % D.ntx, ty = (t / D.ntx) % D.nty, tz = t / (D.ntx * D.nty);
    const int c = threadIdx.x;
    const int X = tx * TILE + (c & 3), Y = ty * TILE + ((c >> 2) & 3), Z = tz * TILE + (c >> 4);
    if (Z >= D.nz) continue;
    const size_t node = ((size_t)Z * D.ny + Y) * D.nx + X;
    const Vec4<real> f = Fslot[(size_t)b * TILE_CELLS + c];
    F[3 * node] = (double)f.x;
    F[3 * node + 1] = (double)f.y;
    F[3 * node + 2] = (double)f.z;
  }
}

// Nodal force of Eq. 16, phi - kV (V - V0)/V0 dV/dq, in double for read-back.
template <typename real>
__global__ void combine_forces_kernel(int nv, const Vec4<real> *__restrict__ phi,
                                      const Vec4<real> *__restrict__ gvol,
                                      const double *__restrict__ vol_partial, VolumeParams vp,
                                      double *__restrict__ out) {
  __shared__ double s_coef;
  if (threadIdx.x < 32) {
    const double coef = volume_coef(vol_partial, vp.vol_blocks, vp.V0, vp.kV, vp.volume_on, nullptr);
    if (threadIdx.x == 0) s_coef = coef;
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  const real coef = (real)s_coef;
  const Vec4<real> p = phi[i], g = gvol[i];
  out[3 * (size_t)i] = (double)(p.x - coef * g.x);
  out[3 * (size_t)i + 1] = (double)(p.y - coef * g.y);
  out[3 * (size_t)i + 2] = (double)(p.z - coef * g.z);
}

__global__ void volume_sum_kernel(const double *__restrict__ part, int n, double V0,
                                  double *__restrict__ out) {
  double V;
  volume_coef(part, n, V0, 0.0, 0, &V);
  if (threadIdx.x == 0) *out = V;
}

VolumeParams volume_params(const Ctx &c) {
  VolumeParams vp;
  vp.V0 = c.V0;
  vp.kV = c.iface.kV;
  vp.volume_on = c.iface.volume_force_on;
  vp.vol_blocks = c.vol_blocks;
  return vp;
}

// Argument records of the step kernels for context c as it is now (its cur and map), shared by
// the single-context launches and the batched ones.
template <typename real>
FaceArgs<real> face_args(const Ctx &c, int reset) {
  FaceArgs<real> a;
  const double *al = c.iface.alpha;
  a.fp.a3 = (real)al[2];
  a.fp.cL0 = (real)(0.5 * (al[0] - al[2]));
  a.fp.cL1 = (real)(0.25 * (al[0] + al[1]));
  a.fp.eps48 = (real)(48.0 * c.iface.eps);
  a.fp.xi = (real)c.iface.xi;
  a.fp.wall_on = c.iface.wall_force_on;
  const int other = c.map ^ 1;
  a.nf = c.nf;
  a.faces = c.faces;
  a.disp = (const Vec4<real> *)c.disp;
  a.fgeo = (const real *)c.fgeo;
  a.fcontrib = (real *)c.fcontrib;
  a.fnorm = (real *)c.fnorm;
  a.vol_partial = c.vol_partial;
  a.D = dims_of(c);
  a.other_tile_slot = c.tile_slot[other];
  a.other_slot_tile = c.slot_tile[other];
  a.other_nslots = c.counters + other;
  a.reset = reset;
  a.ovf_count = c.counters + 2;
  a.spill_bits = c.spill_bits;
  a.spill_words = c.spill_words;
  return a;
}
int face_blocks(const Ctx &c) { return c.vol_blocks; }

template <typename real>
VertexArgs<real> vertex_args(const Ctx &c, int bin) {
  VertexArgs<real> a;
  a.nv = c.nv;
  a.vf_start = c.vf_start;
  a.vf_list = c.vf_list;
  a.fcontrib = (const real *)c.fcontrib;
  a.fnorm = (const real *)c.fnorm;
  a.q = c.q;
  a.phi = (Vec4<real> *)c.phi;
  a.gvol = (Vec4<real> *)c.gvol;
  a.stencil = (StencilRec<real> *)c.stencil;
  a.bin = bin;
  a.tile_slot = c.tile_slot[c.map];
  a.slot_count = c.slot_count;
  a.bucket = c.bucket;
  a.ovf_count = c.counters + 2;
  a.spill_bits = c.spill_bits;
  a.src_index = c.src_index;
  a.nsources = c.counters + 4;
  a.health = c.counters + 3;
  a.zero_counter = bin == 2 ? c.counters + (c.map ^ 1) : nullptr;
  a.vol_partial = c.vol_partial;
  a.vp = volume_params(c);
  a.vcoef = (real *)c.vcoef;
  a.D = dims_of(c);
  return a;
}
int vertex_blocks(const Ctx &c) { return (c.nv + 255) / 256; }

template <typename real>
SourceArgs<real> source_args(const Ctx &c) {
  SourceArgs<real> a;
  a.tile_slot = c.tile_slot[c.map];
  a.slot_tile = c.slot_tile[c.map];
  a.nslots_ptr = c.counters + c.map;
  a.slot_count = c.slot_count;
  a.src_index = c.src_index;
  a.bucket = c.bucket;
  a.spill_bits = c.spill_bits;
  a.spill_words = c.spill_words;
  a.stencil = (const StencilRec<real> *)c.stencil;
  a.phi = (const Vec4<real> *)c.phi;
  a.gvol = (const Vec4<real> *)c.gvol;
  a.vcoef = (const real *)c.vcoef;
  a.Rslot = (Vec4<real> *)c.Rslot;
  a.out_src = c.out_src[c.map];
  a.D = dims_of(c);
  return a;
}
// persistent grids sized to the SMs the interface chain runs on; in a batch (no partition,
// many contexts side by side) to the context's expected active tiles instead: one warp per
// two (source) tiles
template <typename real>
int source_blocks(const Ctx &c, bool batched) {
  constexpr int W = SrcWarps<real>::value;
  const int sms = c.ib_sms > 0 ? c.ib_sms : c.sm_count;
  int g = batched ? (c.tile_estimate + 2 * W - 1) / (2 * W) : sms * 8;
  if (g * W > c.max_slots) g = (c.max_slots + W - 1) / W;
  return g < 1 ? 1 : g;
}

template <typename real>
GatherArgs<real> gather_args(const Ctx &c) {
  GatherArgs<real> a;
  a.slot_tile = c.slot_tile[c.map];
  a.nslots_ptr = c.counters + c.map;
  a.out_src = c.out_src[c.map];
  a.Rslot = (const Vec4<real> *)c.Rslot;
  a.Fslot = (Vec4<real> *)c.Fslot[c.map];
  a.pair_list = c.pair_list;
  a.npairs = c.counters + 5;
  a.D = dims_of(c);
  return a;
}
int gather_blocks(const Ctx &c, bool batched) {
  const int sms = c.ib_sms > 0 ? c.ib_sms : c.sm_count;
  int g = batched ? (c.tile_estimate + 1) / 2 : sms * 16;  // batched: a block per two tiles
  if (g > c.max_slots) g = c.max_slots;
  return g < 1 ? 1 : g;
}

template <typename real>
InterpArgs<real> interp_args(const Ctx &c) {
  const int other = c.map ^ 1;
  InterpArgs<real> a;
  a.nv = c.nv;
  a.stencil = (const StencilRec<real> *)c.stencil;
  a.tile_slot = c.tile_slot[c.map];
  a.Uslot = (const Vec4<real> *)c.Uslot;
  a.q = c.q;
  a.qdot = c.qdot;
  a.xref = c.xref;
  a.disp = (Vec4<real> *)c.disp;
  a.ub = make_double3(c.ub[0], c.ub[1], c.ub[2]);
  a.ut = make_double3(c.ut[0], c.ut[1], c.ut[2]);
  a.D = dims_of(c);
  a.next_tile_slot = c.tile_slot[other];
  a.next_slot_tile = c.slot_tile[other];
  a.next_nslots = c.counters + other;
  a.slot_count = c.slot_count;
  a.out_src = c.out_src[other];
  a.health = c.counters + 3;
  return a;
}
int interp_blocks(const Ctx &c) { return (int)((4L * c.nv + 255) / 256); }

template <typename real>
cudaError_t face_forces_t(Ctx &c, int reset, cudaStream_t st) {
  face_kernel<real><<<face_blocks(c), 256, 0, st>>>(face_args<real>(c, reset));
  return cudaGetLastError();
}

template <typename real>
cudaError_t vertex_forces_t(Ctx &c, int bin, cudaStream_t st) {
  vertex_kernel<real><<<vertex_blocks(c), 256, 0, st>>>(vertex_args<real>(c, bin));
  return cudaGetLastError();
}

template <typename real>
cudaError_t spread_t(Ctx &c, cudaStream_t st) {
  constexpr int W = SrcWarps<real>::value;
  spread_source_kernel<real><<<source_blocks<real>(c, false), 32 * W, 0, st>>>(source_args<real>(c));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  spread_gather_kernel<real><<<gather_blocks(c, false), TILE_CELLS, 0, st>>>(gather_args<real>(c));
  return cudaGetLastError();
}

template <typename real>
cudaError_t interp_t(Ctx &c, cudaStream_t st) {
  interp_kernel<real><<<interp_blocks(c), 256, 0, st>>>(interp_args<real>(c));
  return cudaGetLastError();
}

template <typename T>
void append_record(std::vector<unsigned char> &bytes, const T &rec) {
  const size_t off = bytes.size();
  bytes.resize(off + sizeof(T));
  memcpy(bytes.data() + off, &rec, sizeof(T));
}

template <typename real>
int ib_multi_record_t(const Ctx &c, MultiKernel k, std::vector<unsigned char> &bytes) {
  switch (k) {
    case MK_FACE: append_record(bytes, face_args<real>(c, 1)); return face_blocks(c);
    case MK_VERTEX: append_record(bytes, vertex_args<real>(c, 2)); return vertex_blocks(c);
    case MK_SOURCE: append_record(bytes, source_args<real>(c)); return source_blocks<real>(c, true);
    case MK_GATHER: append_record(bytes, gather_args<real>(c)); return gather_blocks(c, true);
    case MK_INTERP: append_record(bytes, interp_args<real>(c)); return interp_blocks(c);
    default: return -1;
  }
}

template <typename real>
cudaError_t ib_launch_multi_t(MultiKernel k, const MultiLaunch &m, cudaStream_t s) {
  constexpr int W = SrcWarps<real>::value;
  switch (k) {
    case MK_FACE:
      face_kernel_multi<real><<<m.blocks, 256, 0, s>>>((const FaceArgs<real> *)m.args, m.start, m.n);
      break;
    case MK_VERTEX:
      vertex_kernel_multi<real><<<m.blocks, 256, 0, s>>>((const VertexArgs<real> *)m.args, m.start,
                                                          m.n);
      break;
    case MK_SOURCE:
      spread_source_kernel_multi<real><<<m.blocks, 32 * W, 0, s>>>(
          (const SourceArgs<real> *)m.args, m.start, m.n);
      break;
    case MK_GATHER:
      spread_gather_kernel_multi<real><<<m.blocks, TILE_CELLS, 0, s>>>(
          (const GatherArgs<real> *)m.args, m.start, m.n);
      break;
    case MK_INTERP:
      interp_kernel_multi<real><<<m.blocks, 256, 0, s>>>((const InterpArgs<real> *)m.args, m.start,
                                                          m.n);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename real>
size_t ib_record_align(MultiKernel k) {
  switch (k) {
    case MK_FACE: return alignof(FaceArgs<real>);
    case MK_VERTEX: return alignof(VertexArgs<real>);
    case MK_SOURCE: return alignof(SourceArgs<real>);
    case MK_GATHER: return alignof(GatherArgs<real>);
    case MK_INTERP: return alignof(InterpArgs<real>);
    default: return 0;
  }
}

}  // namespace

int ib_multi_record(const Ctx &c, MultiKernel k, std::vector<unsigned char> &bytes) {
  return c.precision == IBLB_FP64 ? ib_multi_record_t<double>(c, k, bytes)
                                  : ib_multi_record_t<float>(c, k, bytes);
}

cudaError_t ib_launch_multi(int precision, MultiKernel k, const MultiLaunch &m, cudaStream_t s) {
  return precision == IBLB_FP64 ? ib_launch_multi_t<double>(k, m, s)
                                : ib_launch_multi_t<float>(k, m, s);
}

size_t ib_multi_record_align(int precision, MultiKernel k) {
  return precision == IBLB_FP64 ? ib_record_align<double>(k) : ib_record_align<float>(k);
}

size_t stencil_record_bytes(const Ctx &c) {
  return c.precision == IBLB_FP64 ? sizeof(StencilRec<double>) : sizeof(StencilRec<float>);
}

cudaError_t launch_face_forces(Ctx &c, int reset_other_map, cudaStream_t s) {
  return c.precision == IBLB_FP64 ? face_forces_t<double>(c, reset_other_map, s)
                                  : face_forces_t<float>(c, reset_other_map, s);
}

// bin: 0 forces only; 1 forces + stencil + binning; 2 as 1 and also zero the other map's
// tile counter (inside a step, after that map was cleared by the face kernel).
cudaError_t launch_vertex_forces(Ctx &c, int bin, cudaStream_t s) {
  return c.precision == IBLB_FP64 ? vertex_forces_t<double>(c, bin, s)
                                  : vertex_forces_t<float>(c, bin, s);
}

cudaError_t launch_spread(Ctx &c, cudaStream_t s) {
  return c.precision == IBLB_FP64 ? spread_t<double>(c, s) : spread_t<float>(c, s);
}

cudaError_t launch_interpolate_advect(Ctx &c, cudaStream_t s) {
  return c.precision == IBLB_FP64 ? interp_t<double>(c, s) : interp_t<float>(c, s);
}

cudaError_t launch_mark(Ctx &c) {
  const long threads = 8L * c.nv;
  const unsigned blocks = (unsigned)((threads + 255) / 256);
  if (c.precision == IBLB_FP64)
    mark_kernel<double><<<blocks, 256, 0, c.stream>>>(
        c.nv, c.q, c.xref, (Vec4<double> *)c.disp, dims_of(c), c.tile_slot[c.map],
        c.slot_tile[c.map], c.counters + c.map, c.slot_count, c.out_src[c.map], c.counters + 3);
  else
    mark_kernel<float><<<blocks, 256, 0, c.stream>>>(
        c.nv, c.q, c.xref, (Vec4<float> *)c.disp, dims_of(c), c.tile_slot[c.map],
        c.slot_tile[c.map], c.counters + c.map, c.slot_count, c.out_src[c.map], c.counters + 3);
  return cudaGetLastError();
}

cudaError_t launch_clear_counts(Ctx &c) {
  int grid = (c.max_slots + 255) / 256;
  if (grid > 1024) grid = 1024;
  clear_counts_kernel<<<grid, 256, 0, c.stream>>>(c.counters + c.map, c.slot_count, c.counters + 2,
                                                  c.max_slots);
  return cudaGetLastError();
}

cudaError_t launch_expand_force(Ctx &c, double *F_dev) {
  int grid = c.sm_count * 8;
  if (grid > c.max_slots) grid = c.max_slots;
  if (grid < 1) grid = 1;
  if (c.precision == IBLB_FP64)
    expand_force_kernel<double><<<grid, TILE_CELLS, 0, c.stream>>>(
        c.slot_tile[c.map], c.counters + c.map, (const Vec4<double> *)c.Fslot[c.map], dims_of(c), F_dev);
  else
    expand_force_kernel<float><<<grid, TILE_CELLS, 0, c.stream>>>(
        c.slot_tile[c.map], c.counters + c.map, (const Vec4<float> *)c.Fslot[c.map], dims_of(c), F_dev);
  return cudaGetLastError();
}

cudaError_t launch_phi_to_double(Ctx &c, double *phi_dev) {
  const int blocks = (c.nv + 255) / 256;
  if (c.precision == IBLB_FP64)
    combine_forces_kernel<double><<<blocks, 256, 0, c.stream>>>(
        c.nv, (const Vec4<double> *)c.phi, (const Vec4<double> *)c.gvol, c.vol_partial,
        volume_params(c), phi_dev);
  else
    combine_forces_kernel<float><<<blocks, 256, 0, c.stream>>>(
        c.nv, (const Vec4<float> *)c.phi, (const Vec4<float> *)c.gvol, c.vol_partial,
        volume_params(c), phi_dev);
  return cudaGetLastError();
}

cudaError_t launch_volume(Ctx &c, double *V_dev) {
  volume_sum_kernel<<<1, 32, 0, c.stream>>>(c.vol_partial, c.vol_blocks, c.V0, V_dev);
  return cudaGetLastError();
}

}  // namespace iblb
