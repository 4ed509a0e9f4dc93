// Internal declarations of the IB-LB CUDA library: the context, device constants of the
// D3Q19 lattice and the launchers each translation unit provides.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/iblb.h"

namespace iblb {

// ---------------------------------------------------------------------------------------
// D3Q19 (Sec. III): 0 rest, 1..6 axis, 7..18 edge diagonals; opposite pairs (2k-1, 2k).
// ---------------------------------------------------------------------------------------
constexpr int Q = 19;
__host__ __device__ constexpr int cx(int i) {
  constexpr int t[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
  return t[i];
}
__host__ __device__ constexpr int cy(int i) {
  constexpr int t[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
  return t[i];
}
__host__ __device__ constexpr int cz(int i) {
  constexpr int t[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
  return t[i];
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
// weights 1/3, 1/18, 1/36 (Sec. III footnote)
__host__ __device__ constexpr double wgt(int i) {
  return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Interface tiles: the lattice is cut into 4x4x4 tiles; only tiles touched by a vertex's
// 4x4x4 delta stencil ("active" tiles) carry force and velocity buffers.
constexpr int TILE = 4;
constexpr int TILE_CELLS = TILE * TILE * TILE;
// vertices per source-tile bucket; the rest of a fuller tile is marked in a spill bitmap
constexpr int BUCKET_CAP = 64;

// Health word bits (read back by iblb_step).
constexpr int H_NAN = 1, H_FAST = 2, H_WALL = 4, H_VOLUME = 8, H_CAPACITY = 16;
// a bounded wait of the staged stream-collide pipeline gave up (the kernel returned early)
constexpr int H_TIMEOUT = 32;

// Default shape of the staged stream-collide pass: stages per block, compute warps per block.
constexpr int kStages = 4, kStageWarps = 8;
// Nodes per compute lane of the staged pass with 16-bit storage (2 or 4).
constexpr int kStageNodes16 = 4;
// Default size of one population's copy in the staged pass (bytes): rows per unit follow.
constexpr size_t kStageCopyBytes = 4096;

// Batched launches: one grid over the blocks of many contexts. Instance i of a launch owns the
// grid's blocks start[i] .. start[i + 1] - 1 (start[0] = 0, start[n] = the grid size).
constexpr int kMultiMax = 256;  // instances per batched launch

struct MultiBlock {
  int inst;     // instance of this block
  int block;    // block index within the instance's share
  int nblocks;  // blocks of the instance
};

// Instance and local block of this block (every thread of the block must call it).
// Instance and block of virtual block b, from the block offsets staged in shared memory.
__device__ __forceinline__ MultiBlock multi_block_of(const int *s_start, int n, int b) {
  int lo = 0, hi = n;  // the largest lo with start[lo] <= b
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (s_start[mid] <= b) lo = mid;
    else hi = mid;
  }
  MultiBlock m;
  m.inst = lo;
  m.block = b - s_start[lo];
  m.nblocks = s_start[lo + 1] - s_start[lo];
  return m;
}

__device__ __forceinline__ MultiBlock multi_block(const int *__restrict__ start, int n) {
  __shared__ int s_start[kMultiMax + 1];
  for (int k = threadIdx.x; k <= n; k += blockDim.x) s_start[k] = start[k];
  __syncthreads();
  const int b = blockIdx.x;
  int lo = 0, hi = n;  // the largest lo with start[lo] <= b
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (s_start[mid] <= b) lo = mid;
    else hi = mid;
  }
  MultiBlock m;
  m.inst = lo;
  m.block = b - s_start[lo];
  m.nblocks = s_start[lo + 1] - s_start[lo];
  return m;
}

// Force and velocity blocks of the active tiles are [slot][64 nodes] of these: x, y, z and one
// pad, so that each node is one aligned vector access.
template <typename real>
struct alignas(4 * sizeof(real)) Vec4 {
  real x, y, z, w;
};

// Per-vertex stencil record written by the vertex kernel and read by spreading and
// interpolation: base node (floor(q) - 1, x/y wrapped), the 3x4 one-dimensional weights.
template <typename real>
struct StencilRec {
  int base[3];
  int pad;
  real w[3][4];
};

struct Ctx {
  // lattice
  int nx = 0, ny = 0, nz = 0, precision = 0, has_walls = 1;
  double tau = 1.0, rho0 = 1.0, ub[3] = {0, 0, 0}, ut[3] = {0, 0, 0}, g[3] = {0, 0, 0};
  size_t ncell = 0;
  size_t real_size = 4;  // interface arithmetic type (force, velocity, stencil buffers)
  size_t pop_size = 4;   // population storage type
  void *f[2] = {nullptr, nullptr};  // populations f_i - w_i rho0, [19][nz][ny][nx]
  int cur = 0;                      // f[cur] holds the state
  int fresh = 1;                    // state is post-streaming (no collision done yet)
  int have_force = 0;               // a spread field exists (for read_fields)
  cudaStream_t stream = nullptr;   // caller's stream: transfers and read-back kernels
  cudaStream_t ls = nullptr;       // stream of the stream-collide passes of iblb_step
  cudaStream_t ib = nullptr;       // library stream: the interface chain of each step
  void *green[2] = {nullptr, nullptr};  // SM partitions (CUgreenCtx): [0] interface, [1] lattice
  int ib_sms = 0;                  // SMs of the interface partition (0: no partition)
  int lat_sms = 0;                 // SMs of the lattice partition (with a partition)
  cudaEvent_t ev_force = nullptr;  // spread force of the step is ready (recorded on ib)
  cudaEvent_t ev_coll = nullptr;   // post-collision populations of the step are complete
  cudaEvent_t ev_sync = nullptr;   // general cross-stream join
  // tiles
  int ntx = 0, nty = 0, ntz = 0;
  size_t ntiles = 0;
  int max_slots = 0;
  int tile_estimate = 0;  // active tiles expected for the mesh (sizes the batched grids)
  int *tile_slot[2] = {nullptr, nullptr};  // [ntiles] slot or -1
  int *slot_tile[2] = {nullptr, nullptr};  // [max_slots] tile id of each active slot
  int *counters = nullptr;  // [0..1] nslots per map, [2] spilled vertices, [3] health, [4] sources,
                            // [5] listed force pairs
  int *src_index = nullptr;                // [max_slots] region of a source tile (slot)
  void *Rslot = nullptr;                   // [max_sources][343] Vec4 spreading regions
  int *out_src[2] = {nullptr, nullptr};    // per map: [max_slots][8] region of source T - e
  int max_sources = 0;
  int *slot_count = nullptr;               // [max_slots] vertices in each source bucket
  int *bucket = nullptr;                   // [max_slots][BUCKET_CAP]
  unsigned *spill_bits = nullptr;          // [spill_words] bit v: vertex v did not fit in its
                                           //   tile's bucket (cleared by every face pass)
  int spill_words = 0;                     // (nv + 31) / 32
  void *Fslot[2] = {nullptr, nullptr};     // per map: [max_slots][64] Vec4 force density
  void *Uslot = nullptr;                   // [max_slots][64] Vec4 velocity
  int *pair_list = nullptr;                // [32 max_slots] slot * 32 + pair: the node pairs with
                                           //   a non-zero force (K4b appends, K1t reads)
  int map = 0;                             // tile map of the current vertex positions
  // mesh
  int nv = 0, nf = 0;
  double *q = nullptr;       // [nv][3] positions (double in every precision)
  double *qdot = nullptr;    // [nv][3]
  int *faces = nullptr;      // [nf][3]
  double *fref = nullptr;    // [nf][4] reference metric inverse (H11, H12, H22) and A0
  double *xref = nullptr;    // [nv][3] reference vertex positions
  void *disp = nullptr;      // [nv] Vec4: q - xref in the population type (kept by K2)
  void *fgeo = nullptr;      // [16][nf] reference edges A, B, X0 - c, heights above the walls,
                             //   (pad), metric inverse H11 H12 H22 and A0, by component
  void *vcoef = nullptr;     // kV (V - V0)/V0 of the step, in the population type (K3b writes it)
  int *vf_start = nullptr;   // [nv+1] CSR vertex -> (face*3 + corner)
  int *vf_list = nullptr;    // [3 nf]
  void *fcontrib = nullptr;  // [nf][3 corners][3]: strain + wall force per corner
  void *fnorm = nullptr;     // [nf][3]: (a x b)/6, the face's volume gradient at each corner
  double *vol_partial = nullptr;  // [vol_blocks] partial sums of V - V0 (one per face block)
  int vol_blocks = 0;
  void *phi = nullptr;       // [nv] Vec4: strain + wall part of the nodal force (Eq. 16 without
                             //   the volume term, which is applied where the force is used)
  void *gvol = nullptr;      // [nv] Vec4: dV/dq of each vertex
  void *stencil = nullptr;   // [nv] StencilRec
  double V0 = 0.0, centre[3] = {0, 0, 0};
  iblb_iface_params iface{};
  // bookkeeping
  int64_t steps_done = 0;
  int profiling = 0;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  int64_t k1_launches = 0, kernel_launches = 0;
  std::vector<cudaEvent_t> ev_near;  // events around the active-tile collision (profiling)
  size_t ev_near_used = 0;
  double *dscratch = nullptr;  // host-transfer staging buffer (doubles)
  void *adj = nullptr;         // recorded trajectory and work arrays of the adjoint (adjoint.cu)
  size_t dscratch_len = 0;
  int sm_count = 0;
  int k1_rows = 0;          // lattice rows per block of the stream-collide pass (0: 1)
  int k1_kind = 0;          // IBLB_STREAM_COLLIDE_AUTO, _STAGED or _DIRECT
  int k1_stages = 0;        // stages of the staged pass (0: kStages)
  int k1_warps = 0;         // compute warps per block of the staged pass (0: kStageWarps)
  int k1_unit_rows = 0;     // lattice rows per unit of the staged pass (0: by copy size)
  int k1_nodes = 0;         // nodes per compute lane of the staged pass, 16-bit (0: default)
  unsigned long long stage_wait_ns = 1000000000ull;  // limit of a staged pass's waits (ns)
  int smem_optin = 0;       // shared memory a block may opt in to (bytes)
  int health_every = 1000;  // iblb_step reads the health word every this many steps (0: at its end)
  int health_pending = 0;   // steps queued by iblb_step_async whose health word is unread
  int *health_host = nullptr;  // pinned: the health word read with a call's own transfers
  uint64_t config_gen = 0;  // bumped by every call that changes what a queued step launches
  std::string err;
};

// Split the device's SMs into an interface partition of about `want` SMs and a lattice
// partition with the rest (green contexts), setting c.green, c.ib (interface stream, priority
// prio_hi), c.ls, c.ib_sms and c.lat_sms; false (nothing created) where the device or driver
// cannot partition. release_sms undoes it.
bool split_sms(Ctx &c, int want, int prio_hi);
void release_sms(Ctx &c);
// Queue nsteps coupled steps on the context's streams: no synchronisation, no health read
// (iblb_step adds those). Returns 0 or an IBLB_E* code (message in c.err).
int enqueue_steps(Ctx &c, int nsteps);
// IBLB_OK for a clear health word, else the matching error code (message in c.err).
int health_status(Ctx &c, int health_word);
// Replace the state by populations P (the storage layout of f[cur]) and positions q (device
// arrays), with the given fresh flag, and mark the tiles of q: the next step continues from
// there exactly as from the state that P and q were copied from.
int restore_state(Ctx &c, const void *P, const double *q, int fresh);
// A failure of steps queued by iblb_step_async: read with a synchronisation (settle_health), or
// queued before a read call's own synchronisation (queue_health) and taken after it
// (pending_health). Each returns IBLB_OK or the failure, and clears the pending mark.
int settle_health(Ctx &c);
int queue_health(Ctx &c);
int pending_health(Ctx &c);
// Release the adjoint's memory (no-op without one).
void adjoint_free(Ctx &c);
// Lattice rows per block of the stream-collide pass (k1_rows within the launch bound).
int k1_block_rows(const Ctx &c);
// Whether the stream-collide steps after the first take the staged kernel.
bool stream_collide_staged(const Ctx &c);

// Launchers (each returns cudaGetLastError() of its launch) on stream `s`.
// Stream-collide of every fluid node with the body force only (no interface force).
cudaError_t launch_stream_collide(Ctx &c, int first, cudaStream_t s);
// Stream-collide again of the nodes of the active tiles, with the interface force.
cudaError_t launch_stream_collide_tiles(Ctx &c, int first, cudaStream_t s);
cudaError_t launch_shell_velocity(Ctx &c, cudaStream_t s);
cudaError_t launch_fields(Ctx &c, double *rho_dev, double *u_dev);
cudaError_t launch_populations(Ctx &c, double *f_dev);
cudaError_t launch_init_equilibrium(Ctx &c, const double *rho_dev, const double *u_dev);

cudaError_t launch_face_forces(Ctx &c, int reset_other_map, cudaStream_t s);
// Device bytes of one stencil record in the context's precision.
size_t stencil_record_bytes(const Ctx &c);
cudaError_t launch_vertex_forces(Ctx &c, int bin, cudaStream_t s);
cudaError_t launch_spread(Ctx &c, cudaStream_t s);
cudaError_t launch_interpolate_advect(Ctx &c, cudaStream_t s);
cudaError_t launch_mark(Ctx &c);
cudaError_t launch_clear_counts(Ctx &c);
cudaError_t launch_expand_force(Ctx &c, double *F_dev);
cudaError_t launch_phi_to_double(Ctx &c, double *phi_dev);
cudaError_t launch_volume(Ctx &c, double *V_dev);

// Batched step kernels: each covers a group of contexts of one precision in one launch (the
// batched ensemble). A record is the argument block one context's kernel would be launched
// with, for the context's current buffer indices (cur, map).
enum MultiKernel {
  MK_FACE,            // K3a
  MK_VERTEX,          // K3b
  MK_SOURCE,          // K4a
  MK_GATHER,          // K4b
  MK_STREAM_COLLIDE,  // K1 (not the first, in-place step)
  MK_TILES,           // K1t
  MK_SHELL,           // K1b
  MK_INTERP,          // K2
};
struct MultiLaunch {
  const void *args = nullptr;  // device: the n records, one per context
  const int *start = nullptr;  // device: n + 1 block offsets
  int n = 0, blocks = 0;
};
// Append context c's record for kernel k to `bytes` and return its number of blocks (at least
// 1), or -1 where k does not belong to this file.
int ib_multi_record(const Ctx &c, MultiKernel k, std::vector<unsigned char> &bytes);
int lattice_multi_record(const Ctx &c, MultiKernel k, std::vector<unsigned char> &bytes);
// Alignment of the records of kernel k for this precision (records are packed at their size);
// 0 where k does not belong to the file.
size_t ib_multi_record_align(int precision, MultiKernel k);
size_t lattice_multi_record_align(int precision, MultiKernel k);
// Launch kernel k over the records of m (contexts of precision `precision`) on stream s.
cudaError_t ib_launch_multi(int precision, MultiKernel k, const MultiLaunch &m, cudaStream_t s);
cudaError_t lattice_launch_multi(int precision, MultiKernel k, const MultiLaunch &m,
                                 cudaStream_t s);

}  // namespace iblb

// The opaque handle of the C ABI.
struct iblb_ctx {
  iblb::Ctx c;
};
