// C ABI of the IB-LB library (declared in include/iblb.h): context management, mesh set-up
// (reference metric, vertex->face lists), the step driver in the order of Sec. III, and the
// read-back, checkpoint and profiling calls.
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <unordered_map>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "iblb_internal.cuh"

using iblb::Ctx;

namespace {

int fail(Ctx &c, int code, const std::string &msg) {
  c.err = msg;
  return code;
}

#define CUDA_TRY(c, expr)                                                               \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail((c), e_ == cudaErrorMemoryAllocation ? IBLB_ENOMEM : IBLB_ECUDA,       \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));                  \
  } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void **)p, count * sizeof(T));
}

cudaError_t dalloc_bytes(void **p, size_t bytes) {
  *p = nullptr;
  return cudaMalloc(p, bytes ? bytes : 1);
}

void dfree(void *p) {
  if (p) cudaFree(p);
}

int staging(Ctx &c, size_t n_doubles) {
  if (c.dscratch_len >= n_doubles) return 0;
  dfree(c.dscratch);
  c.dscratch = nullptr;
  c.dscratch_len = 0;
  CUDA_TRY(c, dalloc(&c.dscratch, n_doubles));
  c.dscratch_len = n_doubles;
  return 0;
}

int check_mesh_id(Ctx &c, int mesh_id) {
  if (c.nv == 0) return fail(c, IBLB_EINVAL, "no mesh has been added");
  if (mesh_id != 0) return fail(c, IBLB_EINVAL, "unknown mesh id");
  return 0;
}

// Clear a tile map and mark it for the current vertex positions.
int remark(Ctx &c, int which) {
  CUDA_TRY(c, cudaMemsetAsync(c.tile_slot[which], 0xff, c.ntiles * sizeof(int), c.stream));
  CUDA_TRY(c, cudaMemsetAsync(c.counters + which, 0, sizeof(int), c.stream));
  const int saved = c.map;
  c.map = which;
  cudaError_t e = iblb::launch_mark(c);
  c.map = saved;
  CUDA_TRY(c, e);
  return 0;
}

int read_health(Ctx &c, int *h) {
  CUDA_TRY(c, cudaMemcpyAsync(h, c.counters + 3, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  CUDA_TRY(c, cudaStreamSynchronize(c.stream));
  return 0;
}

// An unstable run reports that first: its garbage positions can also leave tiles unmarked.
int health_error(Ctx &c, int h) {
  if (h & iblb::H_TIMEOUT)
    return fail(c, IBLB_ETIMEOUT, "stream-collide pipeline: a bounded wait for staged data gave up");
  const int unstable = iblb::H_NAN | iblb::H_FAST | iblb::H_WALL | iblb::H_VOLUME;
  if (!(h & unstable))
    return fail(c, IBLB_ECAPACITY, "active-tile table capacity exceeded");
  std::string m = "health check failed:";
  if (h & iblb::H_NAN) m += " NaN in vertex velocity;";
  if (h & iblb::H_FAST) m += " |qdot| >= 0.1;";
  if (h & iblb::H_WALL) m += " vertex within 0.05 of a wall plane;";
  if (h & iblb::H_VOLUME) m += " |V/V0 - 1| > 0.05;";
  if (h & iblb::H_CAPACITY) m += " (active-tile table capacity also exceeded);";
  return fail(c, IBLB_EUNSTABLE, m);
}

cudaEvent_t pooled_event(Ctx &c) {
  if (c.ev_used == c.ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c.ev_pool.push_back(e);
  }
  return c.ev_pool[c.ev_used++];
}

// Driver entry points for SM partitions (green contexts), looked up at run time so that the
// library loads without the driver library present.
struct GreenApi {
  PFN_cuDeviceGet_v2000 device_get = nullptr;
  PFN_cuDeviceGetDevResource_v12040 get_resource = nullptr;
  PFN_cuDevSmResourceSplitByCount_v12040 split = nullptr;
  PFN_cuDevResourceGenerateDesc_v12040 make_desc = nullptr;
  PFN_cuGreenCtxCreate_v12040 create = nullptr;
  PFN_cuGreenCtxDestroy_v12040 destroy = nullptr;
  PFN_cuGreenCtxStreamCreate_v12050 stream_create = nullptr;
  PFN_cuStreamDestroy_v4000 stream_destroy = nullptr;
};

bool green_api(GreenApi &g) {
  struct Entry {
    const char *name;
    void **fn;
    unsigned version;
  } entries[] = {{"cuDeviceGet", (void **)&g.device_get, 2000},
                 {"cuDeviceGetDevResource", (void **)&g.get_resource, 12040},
                 {"cuDevSmResourceSplitByCount", (void **)&g.split, 12040},
                 {"cuDevResourceGenerateDesc", (void **)&g.make_desc, 12040},
                 {"cuGreenCtxCreate", (void **)&g.create, 12040},
                 {"cuGreenCtxDestroy", (void **)&g.destroy, 12040},
                 {"cuGreenCtxStreamCreate", (void **)&g.stream_create, 12050},
                 {"cuStreamDestroy", (void **)&g.stream_destroy, 4000}};
  for (auto &e : entries) {
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(e.name, e.fn, e.version, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || *e.fn == nullptr)
      return false;
  }
  return true;
}

// Split the device's SMs into an interface partition of about `want` SMs and a lattice
// partition with the rest, each with its own stream. Returns false (and leaves nothing
// behind) when the device or driver cannot partition.
bool make_partitions(Ctx &c, int want, int prio_hi) {
  GreenApi g;
  if (!green_api(g)) return false;
  int ord = 0;
  CUdevice dev;
  if (cudaGetDevice(&ord) != cudaSuccess || g.device_get(&dev, ord) != CUDA_SUCCESS) return false;
  CUdevResource all, part, rest;
  unsigned int groups = 1;
  if (g.get_resource(dev, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS) return false;
  if (g.split(&part, &groups, &all, &rest, 0, (unsigned)want) != CUDA_SUCCESS || groups != 1 ||
      rest.sm.smCount < part.sm.smCount)
    return false;
  CUdevResourceDesc d_ib, d_lat;
  if (g.make_desc(&d_ib, &part, 1) != CUDA_SUCCESS || g.make_desc(&d_lat, &rest, 1) != CUDA_SUCCESS)
    return false;
  CUgreenCtx gi = nullptr, gl = nullptr;
  CUstream si = nullptr, sl = nullptr;
  bool ok = g.create(&gi, d_ib, dev, CU_GREEN_CTX_DEFAULT_STREAM) == CUDA_SUCCESS &&
            g.create(&gl, d_lat, dev, CU_GREEN_CTX_DEFAULT_STREAM) == CUDA_SUCCESS &&
            g.stream_create(&si, gi, CU_STREAM_NON_BLOCKING, prio_hi) == CUDA_SUCCESS &&
            g.stream_create(&sl, gl, CU_STREAM_NON_BLOCKING, 0) == CUDA_SUCCESS;
  if (!ok) {
    if (si) g.stream_destroy(si);
    if (sl) g.stream_destroy(sl);
    if (gi) g.destroy(gi);
    if (gl) g.destroy(gl);
    return false;
  }
  c.green[0] = gi;
  c.green[1] = gl;
  c.ib = (cudaStream_t)si;
  c.ls = (cudaStream_t)sl;
  c.ib_sms = (int)part.sm.smCount;
  c.lat_sms = (int)rest.sm.smCount;
  return true;
}

void free_partitions(Ctx &c) {
  GreenApi g;
  if (!c.green[0] || !green_api(g)) return;
  if (c.ib) g.stream_destroy((CUstream)c.ib);
  if (c.ls) g.stream_destroy((CUstream)c.ls);
  g.destroy((CUgreenCtx)c.green[0]);
  g.destroy((CUgreenCtx)c.green[1]);
  c.ib = c.ls = nullptr;
  c.green[0] = c.green[1] = nullptr;
}

// Reference shape of a mesh: centre (mean vertex), per-face inverse metric and area, the
// reference edges A, B, X0 - centre and the centroid heights above the wall planes zb, zt of
// each face, and the enclosed volume V0.
bool reference_shape(const double *verts, int nv, const int32_t *faces, int nf, double zb,
                     double zt, std::vector<double> &fref, std::vector<double> &fgeo,
                     double centre[3], double *V0_out) {
  fref.assign((size_t)4 * nf, 0.0);
  fgeo.assign((size_t)16 * nf, 0.0);
  for (int k = 0; k < 3; k++) centre[k] = 0.0;
  for (int i = 0; i < nv; i++)
    for (int k = 0; k < 3; k++) centre[k] += verts[3 * i + k] / nv;
  double V0 = 0.0;
  for (int j = 0; j < nf; j++) {
    const double *X0 = verts + 3 * faces[3 * j], *X1 = verts + 3 * faces[3 * j + 1],
                 *X2 = verts + 3 * faces[3 * j + 2];
    double a[3], b[3], r0[3], r1[3], r2[3];
    for (int k = 0; k < 3; k++) {
      a[k] = X1[k] - X0[k];
      b[k] = X2[k] - X0[k];
      r0[k] = X0[k] - centre[k];
      r1[k] = X1[k] - centre[k];
      r2[k] = X2[k] - centre[k];
    }
    const double g11 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    const double g12 = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    const double g22 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    const double det = g11 * g22 - g12 * g12;
    if (!(det > 0)) return false;
    fref[4 * j] = g22 / det;
    fref[4 * j + 1] = -g12 / det;
    fref[4 * j + 2] = g11 / det;
    fref[4 * j + 3] = 0.5 * std::sqrt(det);
    for (int k = 0; k < 3; k++) {
      fgeo[16 * j + k] = a[k];
      fgeo[16 * j + 3 + k] = b[k];
      fgeo[16 * j + 6 + k] = r0[k];
    }
    const double gz = (X0[2] + X1[2] + X2[2]) / 3.0;
    fgeo[16 * j + 9] = gz - zb;
    fgeo[16 * j + 10] = gz - zt;
    for (int k = 0; k < 4; k++) fgeo[16 * j + 12 + k] = fref[4 * j + k];  // in the face kernel's type
    V0 += (r0[0] * (r1[1] * r2[2] - r1[2] * r2[1]) + r0[1] * (r1[2] * r2[0] - r1[0] * r2[2]) +
           r0[2] * (r1[0] * r2[1] - r1[1] * r2[0])) / 6.0;
  }
  *V0_out = V0;
  return V0 > 0;
}

// Upload the reference shape (positions X, per-face data) of the context's mesh.
int upload_reference(Ctx &c, const double *X, const std::vector<double> &fref,
                     const std::vector<double> &fgeo) {
  // expected active tiles, for sizing the batched step's grids: the stencils cover a band about
  // two tiles thick around the surface, A / 8 tiles; twice that allows for the shape changing
  double area = 0.0;
  for (size_t j = 3; j < fref.size(); j += 4) area += fref[j];
  long est = (long)(area / 4.0) + 64;
  c.tile_estimate = (int)(est < c.max_slots ? est : c.max_slots);
  CUDA_TRY(c, cudaMemcpyAsync(c.fref, fref.data(), fref.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  CUDA_TRY(c, cudaMemcpyAsync(c.xref, X, (size_t)3 * c.nv * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  // the face kernel reads the per-face data by component: [16][nf]
  const size_t nf = fgeo.size() / 16;
  std::vector<double> soa(fgeo.size());
  for (size_t j = 0; j < nf; j++)
    for (size_t k = 0; k < 16; k++) soa[k * nf + j] = fgeo[16 * j + k];
  if (c.precision == IBLB_FP64) {
    CUDA_TRY(c, cudaMemcpyAsync(c.fgeo, soa.data(), soa.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    CUDA_TRY(c, cudaStreamSynchronize(c.stream));  // the host buffers are the caller's locals
  } else {
    std::vector<float> g32(soa.begin(), soa.end());
    CUDA_TRY(c, cudaMemcpyAsync(c.fgeo, g32.data(), g32.size() * sizeof(float), cudaMemcpyHostToDevice, c.stream));
    CUDA_TRY(c, cudaStreamSynchronize(c.stream));
  }
  return 0;
}

}  // namespace

extern "C" {

int iblb_create(const iblb_lattice_desc *d, void *cuda_stream, iblb_ctx **out) {
  if (!out) return IBLB_EINVAL;
  *out = nullptr;
  if (!d) return IBLB_EINVAL;
  const int periodic = d->z_periodic ? 1 : 0;
  if (d->nx < 4 || d->ny < 4 || d->nx % 4 || d->ny % 4 || d->nz < (periodic ? 4 : 3) ||
      (periodic && d->nz % 4) || !(d->tau > 0.5) || !(d->rho0 > 0) ||
      (d->precision != IBLB_FP32 && d->precision != IBLB_FP64 && d->precision != IBLB_FP16 &&
       d->precision != IBLB_BF16))
    return IBLB_EINVAL;
  if (!periodic && (d->wall_u_bottom[2] != 0.0 || d->wall_u_top[2] != 0.0)) return IBLB_EINVAL;
  iblb_ctx *h = new iblb_ctx();
  Ctx &c = h->c;
  c.nx = d->nx; c.ny = d->ny; c.nz = d->nz;
  c.precision = d->precision;
  c.has_walls = !periodic;
  c.tau = d->tau;
  c.rho0 = d->rho0;
  for (int k = 0; k < 3; k++) {
    c.ub[k] = d->wall_u_bottom[k];
    c.ut[k] = d->wall_u_top[k];
    c.g[k] = d->body_force[k];
  }
  c.stream = (cudaStream_t)cuda_stream;
  c.ncell = (size_t)c.nx * c.ny * c.nz;
  c.real_size = c.precision == IBLB_FP64 ? 8 : 4;
  c.pop_size = c.precision == IBLB_FP64 ? 8 : (c.precision == IBLB_FP32 ? 4 : 2);
  c.ntx = c.nx / 4;
  c.nty = c.ny / 4;
  c.ntz = (c.nz + 3) / 4;
  c.ntiles = (size_t)c.ntx * c.nty * c.ntz;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c.sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&c.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  for (int b = 0; b < 2 && e == cudaSuccess; b++) e = dalloc_bytes(&c.f[b], (size_t)iblb::Q * c.ncell * c.pop_size);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.f[0], 0, (size_t)iblb::Q * c.ncell * c.pop_size, c.stream);
  // The interface chain runs on its own partition of SMs (default 32) so that the concurrent
  // full-lattice pass keeps the rest undisturbed; without partitions both share the GPU and
  // the interface stream gets the highest priority, so that its small kernels are scheduled
  // between the blocks of the full-lattice pass instead of after it.
  int prio_lo = 0, prio_hi = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  // Default split, from sweeps of the interface SMs. A full-lattice pass of at least 1 GiB
  // hides the interface chain on 24 SMs (256^3 FP32, 2.5 GB: 40.3k MLUPS against 39.3k on 32,
  // 31.5k on 16 and 34.8k unpartitioned); 16-bit storage halves the pass, so the chain takes
  // 40 (256^3 FP16: 66.0k against 59.0k on 32). A shorter pass leaves the chain as the
  // critical path, which then takes 64 SMs (128x128x96 FP32 wetting, 1.5 M nodes: 0.090 ms
  // against 0.115 ms on 32 SMs; 32^3 FP64 shear: 0.136 ms against 0.138 ms on 32 and
  // 0.149 ms unpartitioned). An FP64 pass that long is bound by the FP64 units (1/64 of the
  // FP32 rate), not by memory, and the interface chain is short beside it: no partition
  // (256^3 FP64: 7.05 ms per step against 7.30 on 8 interface SMs and 8.20 on 24).
  const size_t pass_bytes = (size_t)2 * iblb::Q * c.ncell * c.pop_size;
  const int want = d->ib_sms != 0 ? d->ib_sms
                   : pass_bytes < ((size_t)1 << 30) ? 64
                   : c.pop_size == 2 ? 40
                   : c.pop_size == 8 ? -1
                   : 24;
  if (e == cudaSuccess && !(want > 0 && make_partitions(c, want, prio_hi))) {
    e = cudaStreamCreateWithPriority(&c.ib, cudaStreamNonBlocking, prio_hi);
    c.ls = c.stream;
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ev_force, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ev_coll, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ev_sync, cudaEventDisableTiming);
  if (e == cudaSuccess) e = dalloc(&c.counters, 8);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&c.health_host, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(c.counters, 0, 8 * sizeof(int), c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) {
    iblb_destroy(h);
    return e == cudaErrorMemoryAllocation ? IBLB_ENOMEM : IBLB_ECUDA;
  }
  *out = h;
  return IBLB_OK;
}

void iblb_destroy(iblb_ctx *h) {
  if (!h) return;
  Ctx &c = h->c;
  cudaStreamSynchronize(c.stream);
  if (c.ib) cudaStreamSynchronize(c.ib);
  if (c.ls) cudaStreamSynchronize(c.ls);
  for (int b = 0; b < 2; b++) {
    dfree(c.f[b]);
    dfree(c.tile_slot[b]);
    dfree(c.slot_tile[b]);
    dfree(c.out_src[b]);
    dfree(c.Fslot[b]);
  }
  dfree(c.counters); dfree(c.slot_count); dfree(c.src_index); dfree(c.Rslot); dfree(c.bucket); dfree(c.spill_bits); dfree(c.Uslot); dfree(c.pair_list);
  dfree(c.q); dfree(c.qdot); dfree(c.faces); dfree(c.fref); dfree(c.xref); dfree(c.fgeo); dfree(c.vcoef); dfree(c.disp); dfree(c.vf_start); dfree(c.vf_list);
  dfree(c.fcontrib); dfree(c.fnorm); dfree(c.vol_partial); dfree(c.phi); dfree(c.gvol); dfree(c.stencil);
  dfree(c.dscratch);
  if (c.health_host) cudaFreeHost(c.health_host);
  iblb::adjoint_free(c);
  for (cudaEvent_t ev : c.ev_pool) cudaEventDestroy(ev);
  for (cudaEvent_t ev : c.ev_near) cudaEventDestroy(ev);
  if (c.ev_force) cudaEventDestroy(c.ev_force);
  if (c.ev_coll) cudaEventDestroy(c.ev_coll);
  if (c.ev_sync) cudaEventDestroy(c.ev_sync);
  if (c.green[0]) free_partitions(c);
  else if (c.ib) cudaStreamDestroy(c.ib);
  delete h;
}

const char *iblb_last_error(const iblb_ctx *h) { return h ? h->c.err.c_str() : "null context"; }

int iblb_add_mesh(iblb_ctx *h, const double *verts, int32_t nv, const int32_t *faces, int32_t nf,
                  int32_t *mesh_id) {
  if (!h) return IBLB_EINVAL;
  Ctx &c = h->c;
  if (c.nv) return fail(c, IBLB_EINVAL, "one mesh per context");
  if (!verts || !faces || nv < 4 || nf != 2 * nv - 4)
    return fail(c, IBLB_EINVAL, "mesh must be closed: nf == 2 nv - 4, nv >= 4");
  // closedness and orientation: each directed edge once, its reverse once
  std::unordered_map<uint64_t, int> edges;
  edges.reserve((size_t)3 * nf * 2);
  for (int j = 0; j < nf; j++) {
    for (int k = 0; k < 3; k++) {
      const int a = faces[3 * j + k], b = faces[3 * j + (k + 1) % 3];
      if (a < 0 || a >= nv || b < 0 || b >= nv || a == b)
        return fail(c, IBLB_EINVAL, "face index out of range or degenerate face");
      const uint64_t key = ((uint64_t)(uint32_t)a << 32) | (uint32_t)b;
      if (edges.count(key)) return fail(c, IBLB_EINVAL, "directed edge used twice: inconsistent orientation");
      edges[key] = j;
    }
  }
  for (const auto &kv : edges) {
    const uint64_t rev = (kv.first << 32) | (kv.first >> 32);
    if (!edges.count(rev)) return fail(c, IBLB_EINVAL, "open mesh: an edge has one face");
  }
  for (int i = 0; i < 3 * nv; i++)
    if (!std::isfinite(verts[i])) return fail(c, IBLB_EINVAL, "non-finite vertex coordinate");
  std::vector<double> fref, fgeo;
  double centre[3], V0;
  if (!reference_shape(verts, nv, faces, nf, 0.5, c.nz - 1.5, fref, fgeo, centre, &V0))
    return fail(c, IBLB_EINVAL, "degenerate reference face or mesh not oriented outward");
  // vertex -> (face, corner) lists in face order
  std::vector<int> vf_start(nv + 1, 0), vf_list((size_t)3 * nf);
  for (int j = 0; j < 3 * nf; j++) vf_start[faces[j] + 1]++;
  for (int i = 0; i < nv; i++) vf_start[i + 1] += vf_start[i];
  {
    std::vector<int> fill(vf_start.begin(), vf_start.end() - 1);
    for (int j = 0; j < nf; j++)
      for (int k = 0; k < 3; k++) vf_list[fill[faces[3 * j + k]]++] = 3 * j + k;
  }
  // the force-pair list indexes slot * 32 + pair in an int: at most 2^26 tile slots
  if ((long)(8L * nv < (long)c.ntiles ? 8L * nv : (long)c.ntiles) > (1L << 26))
    return fail(c, IBLB_ECAPACITY, "mesh too large: more than 2^26 interface tile slots");
  c.nv = nv;
  c.nf = nf;
  c.V0 = V0;
  for (int k = 0; k < 3; k++) c.centre[k] = centre[k];
  c.vol_blocks = (nf + 255) / 256;  // one partial volume change per face block
  const size_t rs = c.real_size;
  long ms = 8L * nv;
  if ((size_t)ms > c.ntiles) ms = (long)c.ntiles;
  c.max_slots = (int)ms;
  // iface defaults
  c.iface.alpha[0] = c.iface.alpha[1] = c.iface.alpha[2] = 0.0;
  c.iface.kV = 1.0;
  c.iface.eps = 0.0;
  c.iface.xi = 0.5;
  c.iface.wall_force_on = 0;
  c.iface.volume_force_on = 1;
  CUDA_TRY(c, dalloc(&c.q, (size_t)3 * nv));
  CUDA_TRY(c, dalloc(&c.qdot, (size_t)3 * nv));
  CUDA_TRY(c, dalloc(&c.faces, (size_t)3 * nf));
  CUDA_TRY(c, dalloc(&c.fref, (size_t)4 * nf));
  CUDA_TRY(c, dalloc(&c.xref, (size_t)3 * nv));
  CUDA_TRY(c, dalloc_bytes(&c.fgeo, (size_t)16 * nf * rs));
  CUDA_TRY(c, dalloc_bytes(&c.vcoef, sizeof(double)));
  CUDA_TRY(c, dalloc_bytes(&c.disp, (size_t)4 * nv * rs));
  CUDA_TRY(c, dalloc(&c.vf_start, (size_t)nv + 1));
  CUDA_TRY(c, dalloc(&c.vf_list, (size_t)3 * nf));
  CUDA_TRY(c, dalloc_bytes(&c.fcontrib, (size_t)9 * nf * rs));
  CUDA_TRY(c, dalloc_bytes(&c.fnorm, (size_t)3 * nf * rs));
  CUDA_TRY(c, dalloc(&c.vol_partial, (size_t)c.vol_blocks));
  CUDA_TRY(c, dalloc_bytes(&c.phi, (size_t)4 * nv * rs));
  CUDA_TRY(c, dalloc_bytes(&c.gvol, (size_t)4 * nv * rs));
  CUDA_TRY(c, dalloc_bytes(&c.stencil, (size_t)nv * iblb::stencil_record_bytes(c)));
  for (int b = 0; b < 2; b++) {
    CUDA_TRY(c, dalloc(&c.tile_slot[b], c.ntiles));
    CUDA_TRY(c, dalloc(&c.slot_tile[b], (size_t)c.max_slots));
    CUDA_TRY(c, dalloc(&c.out_src[b], (size_t)8 * c.max_slots));
    CUDA_TRY(c, dalloc_bytes(&c.Fslot[b], (size_t)c.max_slots * 4 * iblb::TILE_CELLS * rs));
    CUDA_TRY(c, cudaMemsetAsync(c.tile_slot[b], 0xff, c.ntiles * sizeof(int), c.stream));
  }
  CUDA_TRY(c, dalloc(&c.slot_count, (size_t)c.max_slots));
  CUDA_TRY(c, dalloc(&c.pair_list, (size_t)32 * c.max_slots));
  CUDA_TRY(c, dalloc(&c.src_index, (size_t)c.max_slots));
  c.max_sources = nv < c.max_slots ? nv : c.max_slots;  // a source tile holds >= 1 vertex base
  CUDA_TRY(c, dalloc_bytes(&c.Rslot, (size_t)c.max_sources * 343 * 4 * rs));
  CUDA_TRY(c, dalloc(&c.bucket, (size_t)c.max_slots * iblb::BUCKET_CAP));
  c.spill_words = (nv + 31) / 32;
  CUDA_TRY(c, dalloc(&c.spill_bits, (size_t)c.spill_words));
  CUDA_TRY(c, cudaMemsetAsync(c.spill_bits, 0, (size_t)c.spill_words * sizeof(unsigned), c.stream));
  CUDA_TRY(c, dalloc_bytes(&c.Uslot, (size_t)c.max_slots * 4 * iblb::TILE_CELLS * rs));
  // only the listed (stencil) nodes are written each step, and only they are read
  CUDA_TRY(c, cudaMemsetAsync(c.Uslot, 0, (size_t)c.max_slots * 4 * iblb::TILE_CELLS * rs, c.stream));
  CUDA_TRY(c, cudaMemsetAsync(c.counters, 0, 8 * sizeof(int), c.stream));
  CUDA_TRY(c, cudaMemsetAsync(c.qdot, 0, (size_t)3 * nv * sizeof(double), c.stream));
  CUDA_TRY(c, cudaMemcpyAsync(c.q, verts, (size_t)3 * nv * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  CUDA_TRY(c, cudaMemcpyAsync(c.faces, faces, (size_t)3 * nf * sizeof(int), cudaMemcpyHostToDevice, c.stream));
  CUDA_TRY(c, cudaMemcpyAsync(c.vf_start, vf_start.data(), (size_t)(nv + 1) * sizeof(int), cudaMemcpyHostToDevice, c.stream));
  CUDA_TRY(c, cudaMemcpyAsync(c.vf_list, vf_list.data(), (size_t)3 * nf * sizeof(int), cudaMemcpyHostToDevice, c.stream));
  if (int rc = upload_reference(c, verts, fref, fgeo)) return rc;
  c.map = 0;
  c.config_gen++;
  c.have_force = 0;
  int rc = remark(c, 0);
  if (rc) return rc;
  CUDA_TRY(c, cudaStreamSynchronize(c.stream));
  if (mesh_id) *mesh_id = 0;
  return IBLB_OK;
}

int iblb_set_interface(iblb_ctx *h, int32_t mesh_id, const iblb_iface_params *p) {
  if (!h || !p) return IBLB_EINVAL;
  Ctx &c = h->c;
  if (int rc = check_mesh_id(c, mesh_id)) return rc;
  for (int k = 0; k < 3; k++)
    if (!std::isfinite(p->alpha[k])) return fail(c, IBLB_EINVAL, "non-finite alpha");
  if (!std::isfinite(p->kV) || !std::isfinite(p->eps) || !(p->xi > 0))
    return fail(c, IBLB_EINVAL, "invalid kV, eps or xi");
  c.iface = *p;
  c.config_gen++;
  return IBLB_OK;
}

int iblb_set_vertices(iblb_ctx *h, int32_t mesh_id, const double *q) {
  if (!h || !q) return IBLB_EINVAL;
  Ctx &c = h->c;
  if (int rc = check_mesh_id(c, mesh_id)) return rc;
  CUDA_TRY(c, cudaMemcpyAsync(c.q, q, (size_t)3 * c.nv * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  // the map of the last spreading step (map ^ 1) stays: read_fields still uses its force
  return remark(c, c.map);
}

int iblb_init_equilibrium(iblb_ctx *h, const double *rho, const double *u) {
  if (!h || !rho || !u) return IBLB_EINVAL;
  Ctx &c = h->c;
  if (int rc = staging(c, 4 * c.ncell)) return rc;
  CUDA_TRY(c, cudaMemcpyAsync(c.dscratch, rho, c.ncell * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  CUDA_TRY(c, cudaMemcpyAsync(c.dscratch + c.ncell, u, 3 * c.ncell * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  CUDA_TRY(c, iblb::launch_init_equilibrium(c, c.dscratch, c.dscratch + c.ncell));
  CUDA_TRY(c, cudaStreamSynchronize(c.stream));
  c.fresh = 1;
  c.have_force = 0;
  c.health_pending = 0;  // the state those steps left is gone
  c.config_gen++;
  return IBLB_OK;
}

// One step in the order of Sec. III on two streams. The interface chain (forces, spreading;
// after the collision: velocity gather, interpolation, update, marking) runs on the library
// stream `ib`. The stream-collide of every node with the body force only runs on the
// caller's stream without waiting for it, so it overlaps the interface chain of the same
// step and the tail of the previous one; then the nodes of the active tiles are collided
// again once the spread force is ready.
int iblb_step(iblb_ctx *h, int32_t nsteps) {
  if (!h) return IBLB_EINVAL;
  Ctx &c = h->c;
  if (nsteps < 0) return fail(c, IBLB_EINVAL, "nsteps < 0");
  if (nsteps == 0) return IBLB_OK;
  if (int rc = iblb::settle_health(c)) return rc;  // a failure of earlier iblb_step_async steps
  CUDA_TRY(c, cudaMemsetAsync(c.counters + 3, 0, sizeof(int), c.stream));
  // the health word is read every health_every steps (and at the end), so that a run that goes
  // unstable stops near where it did
  for (int done = 0; done < nsteps;) {
    const int n = c.health_every > 0 && c.health_every < nsteps - done ? c.health_every
                                                                        : nsteps - done;
    if (int rc = iblb::enqueue_steps(c, n)) return rc;
    done += n;
    int hw = 0;
    if (int rc = read_health(c, &hw)) return rc;
    if (hw) return health_error(c, hw);
  }
  return IBLB_OK;
}

int iblb_step_async(iblb_ctx *h, int32_t nsteps) {
  if (!h) return IBLB_EINVAL;
  Ctx &c = h->c;
  if (nsteps < 0) return fail(c, IBLB_EINVAL, "nsteps < 0");
  if (nsteps == 0) return IBLB_OK;
  // a failure still unread stays in the health word; otherwise it starts clear
  if (!c.health_pending) CUDA_TRY(c, cudaMemsetAsync(c.counters + 3, 0, sizeof(int), c.stream));
  if (int rc = iblb::enqueue_steps(c, nsteps)) return rc;
  c.health_pending = 1;
  return IBLB_OK;
}

int iblb_check_health(iblb_ctx *h) {
  if (!h) return IBLB_EINVAL;
  return iblb::settle_health(h->c);
}

int iblb_set_health_interval(iblb_ctx *h, int32_t every) {
  if (!h) return IBLB_EINVAL;
  if (every < 0) return fail(h->c, IBLB_EINVAL, "the health interval must be >= 0");
  h->c.health_every = every;
  return IBLB_OK;
}

}  // extern "C"

namespace iblb {

bool split_sms(Ctx &c, int want, int prio_hi) { return make_partitions(c, want, prio_hi); }
void release_sms(Ctx &c) { free_partitions(c); }

int enqueue_steps(Ctx &c, int nsteps) {
  // the library streams start after everything queued so far on the context's stream
  CUDA_TRY(c, cudaEventRecord(c.ev_sync, c.stream));
  CUDA_TRY(c, cudaStreamWaitEvent(c.ib, c.ev_sync, 0));
  if (c.ls != c.stream) CUDA_TRY(c, cudaStreamWaitEvent(c.ls, c.ev_sync, 0));
  for (int s = 0; s < nsteps; s++) {
    if (c.nv) {
      CUDA_TRY(c, iblb::launch_face_forces(c, 1, c.ib));
      CUDA_TRY(c, iblb::launch_vertex_forces(c, 2, c.ib));
      CUDA_TRY(c, iblb::launch_spread(c, c.ib));
      CUDA_TRY(c, cudaEventRecord(c.ev_force, c.ib));
      c.kernel_launches += 4;  // face, vertex and the two spreading passes
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c.profiling) {
      e0 = pooled_event(c);
      e1 = pooled_event(c);
      if (!e0 || !e1) return fail(c, IBLB_ECUDA, "cudaEventCreate failed");
      CUDA_TRY(c, cudaEventRecord(e0, c.ls));
    }
    CUDA_TRY(c, iblb::launch_stream_collide(c, c.fresh, c.ls));
    if (c.profiling) CUDA_TRY(c, cudaEventRecord(e1, c.ls));
    c.k1_launches += 1;
    c.kernel_launches += 1;
    if (c.nv) {
      CUDA_TRY(c, cudaStreamWaitEvent(c.ls, c.ev_force, 0));
      CUDA_TRY(c, iblb::launch_stream_collide_tiles(c, c.fresh, c.ls));
      CUDA_TRY(c, cudaEventRecord(c.ev_coll, c.ls));
      c.kernel_launches += 1;
    }
    c.cur ^= 1;
    c.fresh = 0;
    if (c.nv) {
      // the shell velocity and the interpolation of the call's last step have no next lattice
      // pass to hide under: with partitions they run on the caller's stream, on all SMs
      cudaStream_t tail = c.ib;
      if (s == nsteps - 1 && c.green[0]) {
        tail = c.stream;
        CUDA_TRY(c, cudaStreamWaitEvent(c.stream, c.ev_force, 0));
      }
      CUDA_TRY(c, cudaStreamWaitEvent(tail, c.ev_coll, 0));
      CUDA_TRY(c, iblb::launch_shell_velocity(c, tail));
      CUDA_TRY(c, iblb::launch_interpolate_advect(c, tail));
      c.kernel_launches += 2;
      c.map ^= 1;
      c.have_force = 1;
    }
    c.steps_done++;
  }
  // the context's stream continues after the last step on both library streams
  CUDA_TRY(c, cudaEventRecord(c.ev_sync, c.ib));
  CUDA_TRY(c, cudaStreamWaitEvent(c.stream, c.ev_sync, 0));
  if (c.ls != c.stream) {
    CUDA_TRY(c, cudaEventRecord(c.ev_coll, c.ls));
    CUDA_TRY(c, cudaStreamWaitEvent(c.stream, c.ev_coll, 0));
  }
  return 0;
}

int health_status(Ctx &c, int hw) { return hw ? health_error(c, hw) : IBLB_OK; }

int settle_health(Ctx &c) {
  if (!c.health_pending) return IBLB_OK;
  c.health_pending = 0;
  int hw = 0;
  if (int rc = read_health(c, &hw)) return rc;
  return health_status(c, hw);
}

int queue_health(Ctx &c) {
  if (c.health_pending)
    CUDA_TRY(c, cudaMemcpyAsync(c.health_host, c.counters + 3, sizeof(int), cudaMemcpyDeviceToHost,
                                c.stream));
  return IBLB_OK;
}

int pending_health(Ctx &c) {
  if (!c.health_pending) return IBLB_OK;
  c.health_pending = 0;
  return health_status(c, *c.health_host);
}

int restore_state(Ctx &c, const void *P, const double *q, int fresh) {
  CUDA_TRY(c, cudaMemcpyAsync(c.f[c.cur], P, (size_t)Q * c.ncell * c.pop_size,
                              cudaMemcpyDeviceToDevice, c.stream));
  CUDA_TRY(c, cudaMemcpyAsync(c.q, q, (size_t)3 * c.nv * sizeof(double), cudaMemcpyDeviceToDevice,
                              c.stream));
  c.fresh = fresh;
  return remark(c, c.map);
}

}  // namespace iblb

extern "C" {

int iblb_read_fields(iblb_ctx *h, double *rho, double *u) {
  if (!h || !rho || !u) return IBLB_EINVAL;
  Ctx &c = h->c;
  if (int rc = staging(c, 4 * c.ncell)) return rc;
  if (int rc = iblb::queue_health(c)) return rc;
  CUDA_TRY(c, iblb::launch_fields(c, c.dscratch, c.dscratch + c.ncell));
  CUDA_TRY(c, cudaMemcpyAsync(rho, c.dscratch, c.ncell * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  CUDA_TRY(c, cudaMemcpyAsync(u, c.dscratch + c.ncell, 3 * c.ncell * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  CUDA_TRY(c, cudaStreamSynchronize(c.stream));
  return iblb::pending_health(c);
}

int iblb_read_fields_device(iblb_ctx *h, double *rho_dev, double *u_dev) {
  if (!h || !rho_dev || !u_dev) return IBLB_EINVAL;
  Ctx &c = h->c;
  CUDA_TRY(c, iblb::launch_fields(c, rho_dev, u_dev));
  return IBLB_OK;
}

int iblb_read_populations(iblb_ctx *h, double *f) {
  if (!h || !f) return IBLB_EINVAL;
  Ctx &c = h->c;
  if (int rc = staging(c, (size_t)iblb::Q * c.ncell)) return rc;
  CUDA_TRY(c, iblb::launch_populations(c, c.dscratch));
  CUDA_TRY(c, cudaMemcpyAsync(f, c.dscratch, (size_t)iblb::Q * c.ncell * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  CUDA_TRY(c, cudaStreamSynchronize(c.stream));
  return IBLB_OK;
}

int iblb_read_vertices(iblb_ctx *h, int32_t mesh_id, double *q) {
  if (!h || !q) return IBLB_EINVAL;
  Ctx &c = h->c;
  if (int rc = check_mesh_id(c, mesh_id)) return rc;
  if (int rc = iblb::queue_health(c)) return rc;
  CUDA_TRY(c, cudaMemcpyAsync(q, c.q, (size_t)3 * c.nv * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  CUDA_TRY(c, cudaStreamSynchronize(c.stream));
  return iblb::pending_health(c);
}

int iblb_read_vertices_device(iblb_ctx *h, int32_t mesh_id, double *q_dev) {
  if (!h || !q_dev) return IBLB_EINVAL;
  Ctx &c = h->c;
  if (int rc = check_mesh_id(c, mesh_id)) return rc;
  CUDA_TRY(c, cudaMemcpyAsync(q_dev, c.q, (size_t)3 * c.nv * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
  return IBLB_OK;
}

int iblb_read_vertex_velocities(iblb_ctx *h, int32_t mesh_id, double *qdot) {
  if (!h || !qdot) return IBLB_EINVAL;
  Ctx &c = h->c;
  if (int rc = check_mesh_id(c, mesh_id)) return rc;
  if (int rc = iblb::queue_health(c)) return rc;
  CUDA_TRY(c, cudaMemcpyAsync(qdot, c.qdot, (size_t)3 * c.nv * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  CUDA_TRY(c, cudaStreamSynchronize(c.stream));
  return iblb::pending_health(c);
}

int iblb_read_forces(iblb_ctx *h, int32_t mesh_id, double *phi) {
  if (!h || !phi) return IBLB_EINVAL;
  Ctx &c = h->c;
  if (int rc = check_mesh_id(c, mesh_id)) return rc;
  if (int rc = staging(c, (size_t)3 * c.nv)) return rc;
  if (int rc = iblb::queue_health(c)) return rc;
  CUDA_TRY(c, iblb::launch_face_forces(c, 0, c.stream));
  CUDA_TRY(c, iblb::launch_vertex_forces(c, 0, c.stream));
  CUDA_TRY(c, iblb::launch_phi_to_double(c, c.dscratch));
  CUDA_TRY(c, cudaMemcpyAsync(phi, c.dscratch, (size_t)3 * c.nv * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  CUDA_TRY(c, cudaStreamSynchronize(c.stream));
  return iblb::pending_health(c);
}

int iblb_read_force_field(iblb_ctx *h, double *F) {
  if (!h || !F) return IBLB_EINVAL;
  Ctx &c = h->c;
  if (int rc = staging(c, 3 * c.ncell)) return rc;
  if (int rc = iblb::settle_health(c)) return rc;  // the health word is reused below
  CUDA_TRY(c, cudaMemsetAsync(c.dscratch, 0, 3 * c.ncell * sizeof(double), c.stream));
  if (c.nv) {
    CUDA_TRY(c, cudaMemsetAsync(c.counters + 3, 0, sizeof(int), c.stream));
    CUDA_TRY(c, iblb::launch_face_forces(c, 0, c.stream));
    CUDA_TRY(c, iblb::launch_vertex_forces(c, 1, c.stream));
    CUDA_TRY(c, iblb::launch_spread(c, c.stream));
    CUDA_TRY(c, iblb::launch_expand_force(c, c.dscratch));
    CUDA_TRY(c, iblb::launch_clear_counts(c));
  }
  CUDA_TRY(c, cudaMemcpyAsync(F, c.dscratch, 3 * c.ncell * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  CUDA_TRY(c, cudaStreamSynchronize(c.stream));
  if (c.nv) {
    int hw = 0;
    if (int rc = read_health(c, &hw)) return rc;
    if (hw & iblb::H_CAPACITY) return health_error(c, iblb::H_CAPACITY);
  }
  return IBLB_OK;
}

int iblb_read_volume(iblb_ctx *h, int32_t mesh_id, double *V, double *V0) {
  if (!h || !V || !V0) return IBLB_EINVAL;
  Ctx &c = h->c;
  if (int rc = check_mesh_id(c, mesh_id)) return rc;
  if (int rc = staging(c, 1)) return rc;
  if (int rc = iblb::queue_health(c)) return rc;
  CUDA_TRY(c, iblb::launch_face_forces(c, 0, c.stream));
  CUDA_TRY(c, iblb::launch_volume(c, c.dscratch));
  CUDA_TRY(c, cudaMemcpyAsync(V, c.dscratch, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  CUDA_TRY(c, cudaStreamSynchronize(c.stream));
  *V0 = c.V0;
  return iblb::pending_health(c);
}

// ---------------------------------------------------------------------------------------
// Checkpoint: header + populations (as stored) + mesh state.
// ---------------------------------------------------------------------------------------
namespace {
struct StateHeader {
  char magic[8];
  int32_t nx, ny, nz, precision, has_walls, nv, nf, fresh;
  int64_t steps_done;
  double tau, rho0, ub[3], ut[3], g[3], V0, centre[3];
  iblb_iface_params iface;
};
}  // namespace

int iblb_save_state(iblb_ctx *h, const char *path) {
  if (!h || !path) return IBLB_EINVAL;
  Ctx &c = h->c;
  StateHeader hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, "IBLBST02", 8);
  hd.nx = c.nx; hd.ny = c.ny; hd.nz = c.nz; hd.precision = c.precision; hd.has_walls = c.has_walls;
  hd.nv = c.nv; hd.nf = c.nf; hd.fresh = c.fresh; hd.steps_done = c.steps_done;
  hd.tau = c.tau; hd.rho0 = c.rho0; hd.V0 = c.V0;
  for (int k = 0; k < 3; k++) {
    hd.ub[k] = c.ub[k]; hd.ut[k] = c.ut[k]; hd.g[k] = c.g[k]; hd.centre[k] = c.centre[k];
  }
  hd.iface = c.iface;
  const size_t fbytes = (size_t)iblb::Q * c.ncell * c.pop_size;
  std::vector<char> fbuf(fbytes);
  std::vector<double> qbuf((size_t)3 * c.nv), qdbuf((size_t)3 * c.nv);
  std::vector<double> refbuf((size_t)3 * c.nv);
  std::vector<int> fcs((size_t)3 * c.nf);
  CUDA_TRY(c, cudaMemcpyAsync(fbuf.data(), c.f[c.cur], fbytes, cudaMemcpyDeviceToHost, c.stream));
  if (c.nv) {
    CUDA_TRY(c, cudaMemcpyAsync(qbuf.data(), c.q, qbuf.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    CUDA_TRY(c, cudaMemcpyAsync(qdbuf.data(), c.qdot, qdbuf.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    CUDA_TRY(c, cudaMemcpyAsync(refbuf.data(), c.xref, refbuf.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    CUDA_TRY(c, cudaMemcpyAsync(fcs.data(), c.faces, fcs.size() * sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  }
  CUDA_TRY(c, cudaStreamSynchronize(c.stream));
  FILE *fp = fopen(path, "wb");
  if (!fp) return fail(c, IBLB_EINVAL, std::string("cannot open for writing: ") + path);
  bool ok = fwrite(&hd, sizeof(hd), 1, fp) == 1 && fwrite(fbuf.data(), 1, fbytes, fp) == fbytes;
  if (c.nv) {
    ok = ok && fwrite(qbuf.data(), sizeof(double), qbuf.size(), fp) == qbuf.size();
    ok = ok && fwrite(qdbuf.data(), sizeof(double), qdbuf.size(), fp) == qdbuf.size();
    ok = ok && fwrite(refbuf.data(), sizeof(double), refbuf.size(), fp) == refbuf.size();
    ok = ok && fwrite(fcs.data(), sizeof(int), fcs.size(), fp) == fcs.size();
  }
  ok = (fclose(fp) == 0) && ok;
  if (!ok) return fail(c, IBLB_EINVAL, std::string("write failed: ") + path);
  return IBLB_OK;
}

int iblb_load_state(iblb_ctx *h, const char *path) {
  if (!h || !path) return IBLB_EINVAL;
  Ctx &c = h->c;
  FILE *fp = fopen(path, "rb");
  if (!fp) return fail(c, IBLB_EINVAL, std::string("cannot open: ") + path);
  StateHeader hd;
  bool ok = fread(&hd, sizeof(hd), 1, fp) == 1 && memcmp(hd.magic, "IBLBST02", 8) == 0;
  if (!ok || hd.nx != c.nx || hd.ny != c.ny || hd.nz != c.nz || hd.precision != c.precision ||
      hd.has_walls != c.has_walls || hd.nv != c.nv || hd.nf != c.nf) {
    fclose(fp);
    return fail(c, IBLB_EINVAL, "state file does not match this context");
  }
  const size_t fbytes = (size_t)iblb::Q * c.ncell * c.pop_size;
  std::vector<char> fbuf(fbytes);
  std::vector<double> qbuf((size_t)3 * c.nv), qdbuf((size_t)3 * c.nv);
  std::vector<double> refbuf((size_t)3 * c.nv);
  std::vector<int> fcs((size_t)3 * c.nf);
  ok = fread(fbuf.data(), 1, fbytes, fp) == fbytes;
  if (c.nv) {
    ok = ok && fread(qbuf.data(), sizeof(double), qbuf.size(), fp) == qbuf.size();
    ok = ok && fread(qdbuf.data(), sizeof(double), qdbuf.size(), fp) == qdbuf.size();
    ok = ok && fread(refbuf.data(), sizeof(double), refbuf.size(), fp) == refbuf.size();
    ok = ok && fread(fcs.data(), sizeof(int), fcs.size(), fp) == fcs.size();
  }
  fclose(fp);
  if (!ok) return fail(c, IBLB_EINVAL, "truncated state file");
  if (c.nv) {
    std::vector<int> mine((size_t)3 * c.nf);
    CUDA_TRY(c, cudaMemcpy(mine.data(), c.faces, mine.size() * sizeof(int), cudaMemcpyDeviceToHost));
    if (mine != fcs) return fail(c, IBLB_EINVAL, "state file has a different face list");
  }
  c.tau = hd.tau; c.rho0 = hd.rho0;
  for (int k = 0; k < 3; k++) { c.ub[k] = hd.ub[k]; c.ut[k] = hd.ut[k]; c.g[k] = hd.g[k]; }
  c.fresh = hd.fresh;
  c.steps_done = hd.steps_done;
  c.health_pending = 0;  // the state of any unread iblb_step_async steps is replaced
  CUDA_TRY(c, cudaMemcpyAsync(c.f[c.cur], fbuf.data(), fbytes, cudaMemcpyHostToDevice, c.stream));
  if (c.nv) {
    std::vector<double> fref, fgeo;
    double centre[3], V0;
    if (!reference_shape(refbuf.data(), c.nv, fcs.data(), c.nf, 0.5, c.nz - 1.5, fref, fgeo,
                         centre, &V0))
      return fail(c, IBLB_EINVAL, "state file has a degenerate reference shape");
    if (int rc = upload_reference(c, refbuf.data(), fref, fgeo)) return rc;
    c.V0 = V0;
    for (int k = 0; k < 3; k++) c.centre[k] = centre[k];
    c.iface = hd.iface;
    CUDA_TRY(c, cudaMemcpyAsync(c.q, qbuf.data(), qbuf.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    CUDA_TRY(c, cudaMemcpyAsync(c.qdot, qdbuf.data(), qdbuf.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    c.have_force = 0;
    if (int rc = remark(c, c.map)) return rc;
    c.config_gen++;
  }
  CUDA_TRY(c, cudaStreamSynchronize(c.stream));
  return IBLB_OK;
}

int64_t iblb_steps_done(const iblb_ctx *h) { return h ? h->c.steps_done : -1; }

int iblb_set_profiling(iblb_ctx *h, int32_t on) {
  if (!h) return IBLB_EINVAL;
  Ctx &c = h->c;
  CUDA_TRY(c, cudaStreamSynchronize(c.stream));
  c.profiling = on ? 1 : 0;
  c.ev_used = 0;
  c.k1_launches = 0;
  c.kernel_launches = 0;
  return IBLB_OK;
}

int iblb_profile(iblb_ctx *h, double *k1_ms, int64_t *k1_launches, int64_t *kernel_launches) {
  if (!h || !k1_ms || !k1_launches || !kernel_launches) return IBLB_EINVAL;
  Ctx &c = h->c;
  CUDA_TRY(c, cudaStreamSynchronize(c.stream));
  double total = 0.0;
  for (size_t k = 0; k + 1 < c.ev_used; k += 2) {
    float ms = 0.f;
    CUDA_TRY(c, cudaEventElapsedTime(&ms, c.ev_pool[k], c.ev_pool[k + 1]));
    total += ms;
  }
  *k1_ms = total;
  *k1_launches = c.k1_launches;
  *kernel_launches = c.kernel_launches;
  return IBLB_OK;
}

int iblb_set_stream_collide(iblb_ctx *h, int32_t kind, int32_t stages, int32_t warps,
                            int32_t rows, int32_t nodes) {
  if (!h) return IBLB_EINVAL;
  Ctx &c = h->c;
  if (kind != IBLB_STREAM_COLLIDE_AUTO && kind != IBLB_STREAM_COLLIDE_STAGED &&
      kind != IBLB_STREAM_COLLIDE_DIRECT)
    return fail(c, IBLB_EINVAL, "stream-collide kind must be AUTO (0), STAGED (1) or DIRECT (2)");
  if (stages != 0 && (stages < 2 || stages > 8))
    return fail(c, IBLB_EINVAL, "stages must be 0 or 2..8");
  if (nodes != 0 && nodes != 2 && nodes != 4) return fail(c, IBLB_EINVAL, "nodes must be 0, 2 or 4");
  if (warps < 0 || warps > 16) return fail(c, IBLB_EINVAL, "warps must be 0 or 1..16");
  if (rows < 0 || rows > 16 || (rows & (rows - 1)) || (rows && c.ny % rows))
    return fail(c, IBLB_EINVAL, "rows must be 0 or a power of two up to 16 that divides ny");
  c.k1_kind = kind;
  c.k1_stages = stages;
  c.k1_warps = warps;
  c.k1_unit_rows = rows;
  c.k1_nodes = nodes;
  c.config_gen++;
  return IBLB_OK;
}

int iblb_set_stage_wait_limit(iblb_ctx *h, int64_t ns) {
  if (!h) return IBLB_EINVAL;
  if (ns < 0 || ns > 60000000000ll) return fail(h->c, IBLB_EINVAL, "wait limit must be 0 .. 60 s");
  h->c.stage_wait_ns = (unsigned long long)ns;
  h->c.config_gen++;
  return IBLB_OK;
}

int32_t iblb_stream_collide_staged(const iblb_ctx *h) {
  return h ? (iblb::stream_collide_staged(h->c) ? 1 : 0) : -1;
}

int32_t iblb_interface_sms(const iblb_ctx *h) { return h ? h->c.ib_sms : -1; }

int64_t iblb_bytes_per_cell(const iblb_ctx *h) {
  return h ? (int64_t)(2 * iblb::Q * h->c.pop_size) : -1;
}

}  // extern "C"
