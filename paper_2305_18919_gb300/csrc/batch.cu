// Batched ensemble: many independent IB-LB contexts (lattices and meshes of any sizes)
// advanced together. Each kernel of the coupled step (face forces, vertex gather, the two
// spreading passes, stream-collide, the active-tile recollision, the shell velocity,
// interpolation) is one launch over all contexts of a precision: its blocks find their context
// in a block table and read that context's argument record (the arguments of the context's own
// launch), then run the same device code as the single-context kernels, so every context ends
// bit for bit as when stepped alone. The records are built for both parities of a pair of steps
// (a pair returns the double-buffer indices of populations and tile maps to where they were)
// and rebuilt when a context changes. The interface chain and the stream-collide passes are
// queued on two streams joined by events as in a single context's step. The paper advances one
// box at a time; this is the ensemble form of its parameter sweeps (Sec. V).
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "iblb_internal.cuh"

using iblb::Ctx;

namespace {

// Instances of one precision, stepped by the same batched launches (at most kMultiMax).
struct Group {
  int precision = 0;
  std::vector<int> members;
};

// Host image of one batched launch: the records of its instances and its block table.
struct Table {
  std::vector<unsigned char> bytes;
  std::vector<int> start{0};
  size_t args_off = 0, start_off = 0;
};

using iblb::MultiKernel;
constexpr MultiKernel kKernels[] = {iblb::MK_FACE,   iblb::MK_VERTEX,          iblb::MK_SOURCE,
                                    iblb::MK_GATHER, iblb::MK_STREAM_COLLIDE, iblb::MK_TILES,
                                    iblb::MK_SHELL,  iblb::MK_INTERP};
constexpr int kNumKernels = sizeof(kKernels) / sizeof(kKernels[0]);
constexpr int kPairSteps = 2;  // records are built for both parities of a pair of steps

bool lattice_kernel(MultiKernel k) {
  return k == iblb::MK_STREAM_COLLIDE || k == iblb::MK_TILES || k == iblb::MK_SHELL;
}

}  // namespace

struct iblb_batch {
  std::vector<iblb_ctx *> inst;
  std::vector<cudaStream_t> streams;  // one per instance (the instance's own stream)
  std::vector<cudaEvent_t> joins;     // one per instance
  cudaStream_t stream = nullptr;      // caller's stream
  iblb::Ctx part;                     // the batch's SM partitions and their streams (ib, ls)
  cudaEvent_t ev_force = nullptr, ev_coll = nullptr, ev_join = nullptr;
  std::vector<Group> groups;
  std::vector<Table> tabs;     // [parity][group][kernel]
  void *arena = nullptr;       // device: every table's records and block offsets
  bool tables = false;         // tabs/arena hold records of the instances' current state
  std::vector<uint64_t> gens;  // config_gen, cur, map of every instance when recorded
  std::vector<int> curs, maps;
  std::vector<int> status;     // per-instance result of the last iblb_batch_step
  int *health = nullptr;       // pinned, one word per instance
  std::string err;
};

namespace {

int bfail(iblb_batch *b, int code, const std::string &msg) {
  b->err = msg;
  return code;
}

#define BATCH_TRY(b, expr)                                                                  \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return bfail((b), e_ == cudaErrorMemoryAllocation ? IBLB_ENOMEM : IBLB_ECUDA,          \
                   std::string(#expr) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

int inst_fail(iblb_batch *b, int i, int rc) {
  return bfail(b, rc, "instance " + std::to_string(i) + ": " + b->inst[i]->c.err);
}

// `to` waits for everything queued so far on `from`.
cudaError_t follow(cudaStream_t to, cudaStream_t from, cudaEvent_t ev) {
  cudaError_t e = cudaEventRecord(ev, from);
  return e == cudaSuccess ? cudaStreamWaitEvent(to, ev, 0) : e;
}

bool tables_current(const iblb_batch *b) {
  if (!b->tables) return false;
  for (size_t i = 0; i < b->inst.size(); i++) {
    const Ctx &c = b->inst[i]->c;
    if (b->gens[i] != c.config_gen || b->curs[i] != c.cur || b->maps[i] != c.map) return false;
  }
  return true;
}

std::vector<Group> make_groups(const iblb_batch *b) {
  std::map<int, std::vector<int>> by_precision;
  for (size_t i = 0; i < b->inst.size(); i++)
    by_precision[b->inst[i]->c.precision].push_back((int)i);
  std::vector<Group> groups;
  for (const auto &kv : by_precision)
    for (size_t o = 0; o < kv.second.size(); o += iblb::kMultiMax) {
      Group g;
      g.precision = kv.first;
      const size_t e = std::min(kv.second.size(), o + (size_t)iblb::kMultiMax);
      g.members.assign(kv.second.begin() + o, kv.second.begin() + e);
      groups.push_back(g);
    }
  return groups;
}

// Build the argument records and block tables of every batched launch, for both parities of a
// pair of steps from the instances' current state, into one device arena.
int build_tables(iblb_batch *b) {
  if (b->arena) {
    BATCH_TRY(b, cudaStreamSynchronize(b->stream));  // the last steps that read it are done
    cudaFree(b->arena);
    b->arena = nullptr;
  }
  b->tables = false;
  b->groups = make_groups(b);
  const size_t G = b->groups.size(), n = b->inst.size();
  b->tabs.assign(kPairSteps * G * kNumKernels, Table());
  std::vector<int> cur0(n), map0(n);
  for (size_t i = 0; i < n; i++) {
    cur0[i] = b->inst[i]->c.cur;
    map0[i] = b->inst[i]->c.map;
  }
  int rc = 0;
  for (int p = 0; p < kPairSteps && rc == 0; p++) {
    for (size_t i = 0; i < n; i++) {  // the state a step of this parity starts from
      Ctx &c = b->inst[i]->c;
      c.cur = cur0[i] ^ p;
      c.map = map0[i] ^ (c.nv ? p : 0);
    }
    for (size_t g = 0; g < G && rc == 0; g++)
      for (int ki = 0; ki < kNumKernels && rc == 0; ki++) {
        Table &t = b->tabs[(p * G + g) * kNumKernels + ki];
        const MultiKernel k = kKernels[ki];
        for (int i : b->groups[g].members) {
          const Ctx &c = b->inst[i]->c;
          if (k != iblb::MK_STREAM_COLLIDE && c.nv == 0) continue;  // no mesh: lattice only
          const int blocks = lattice_kernel(k) ? iblb::lattice_multi_record(c, k, t.bytes)
                                               : iblb::ib_multi_record(c, k, t.bytes);
          if (blocks < 1) {
            rc = bfail(b, IBLB_ECUDA, "batched launch without a record");
            break;
          }
          t.start.push_back(t.start.back() + blocks);
        }
      }
  }
  for (size_t i = 0; i < n; i++) {
    b->inst[i]->c.cur = cur0[i];
    b->inst[i]->c.map = map0[i];
  }
  if (rc) return rc;
  // each table's records, then its block offsets, each 256-byte aligned (a multiple of every
  // record's alignment)
  size_t total = 0;
  for (Table &t : b->tabs) {
    t.args_off = total;
    total = (total + t.bytes.size() + 255) / 256 * 256;
    t.start_off = total;
    total = (total + t.start.size() * sizeof(int) + 255) / 256 * 256;
  }
  std::vector<unsigned char> image(total, 0);
  for (const Table &t : b->tabs) {
    if (!t.bytes.empty()) memcpy(image.data() + t.args_off, t.bytes.data(), t.bytes.size());
    memcpy(image.data() + t.start_off, t.start.data(), t.start.size() * sizeof(int));
  }
  BATCH_TRY(b, cudaMalloc(&b->arena, total));
  BATCH_TRY(b, cudaMemcpy(b->arena, image.data(), total, cudaMemcpyHostToDevice));
  for (size_t i = 0; i < n; i++) {
    const Ctx &c = b->inst[i]->c;
    b->gens[i] = c.config_gen;
    b->curs[i] = c.cur;
    b->maps[i] = c.map;
  }
  b->tables = true;
  return 0;
}

// Queue kernel ki of every group (records of step parity p) on stream s.
int launch_kernel(iblb_batch *b, int p, int ki, cudaStream_t s) {
  const size_t G = b->groups.size();
  for (size_t g = 0; g < G; g++) {
    const Table &t = b->tabs[(p * G + g) * kNumKernels + ki];
    iblb::MultiLaunch m;
    m.n = (int)t.start.size() - 1;
    if (m.n == 0) continue;
    m.blocks = t.start.back();
    m.args = (const unsigned char *)b->arena + t.args_off;
    m.start = (const int *)((const unsigned char *)b->arena + t.start_off);
    const MultiKernel k = kKernels[ki];
    const cudaError_t e = lattice_kernel(k) ? iblb::lattice_launch_multi(b->groups[g].precision, k, m, s)
                                            : iblb::ib_launch_multi(b->groups[g].precision, k, m, s);
    if (e != cudaSuccess)
      return bfail(b, IBLB_ECUDA, std::string("batched launch: ") + cudaGetErrorString(e));
  }
  return 0;
}

// Queue one coupled step of every instance (records of parity p): the interface chain on the
// interface stream, the stream-collide passes on the lattice stream, joined by events as in
// iblb_step.
int enqueue_batched_step(iblb_batch *b, int p) {
  cudaStream_t ifc = b->part.ib, lat = b->part.ls;
  for (int ki = 0; ki < 4; ki++)  // K3a, K3b, K4a, K4b
    if (int rc = launch_kernel(b, p, ki, ifc)) return rc;
  BATCH_TRY(b, cudaEventRecord(b->ev_force, ifc));
  if (int rc = launch_kernel(b, p, 4, lat)) return rc;  // K1
  BATCH_TRY(b, cudaStreamWaitEvent(lat, b->ev_force, 0));
  if (int rc = launch_kernel(b, p, 5, lat)) return rc;  // K1t
  BATCH_TRY(b, cudaEventRecord(b->ev_coll, lat));
  BATCH_TRY(b, cudaStreamWaitEvent(ifc, b->ev_coll, 0));
  for (int ki = 6; ki < 8; ki++)  // K1b, K2
    if (int rc = launch_kernel(b, p, ki, ifc)) return rc;
  return 0;
}

}  // namespace

extern "C" {

int iblb_batch_create(const iblb_lattice_desc *descs, int32_t n, void *cuda_stream,
                      iblb_batch **out) {
  if (!out) return IBLB_EINVAL;
  *out = nullptr;
  if (!descs || n < 1) return IBLB_EINVAL;
  iblb_batch *b = new iblb_batch();
  b->stream = (cudaStream_t)cuda_stream;
  int rc = 0;
  // two streams, the interface chain's and the lattice passes'; with descs[0].ib_sms > 0 they
  // run on SM partitions as a single context's. The default is no partition: the interface
  // work of many meshes needs more SMs than the lattice pass can leave it (96 wetting boxes:
  // 14.1k MLUPS with 32 interface SMs, 19.0k with 48, 23.0k with 64 or with no partition)
  int prio_lo = 0, prio_hi = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  const int want = descs[0].ib_sms;
  if (e == cudaSuccess && !(want > 0 && iblb::split_sms(b->part, want, prio_hi))) {
    e = cudaStreamCreateWithFlags(&b->part.ib, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->part.ls, cudaStreamNonBlocking);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_force, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_coll, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->health, sizeof(int) * n);
  for (int i = 0; i < n && e == cudaSuccess && rc == 0; i++) {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) break;
    b->streams.push_back(s);
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) break;
    b->joins.push_back(ev);
    iblb_lattice_desc d = descs[i];
    d.ib_sms = -1;  // no SM partition: the instances share the GPU
    iblb_ctx *h = nullptr;
    rc = iblb_create(&d, s, &h);
    if (rc == 0) b->inst.push_back(h);
  }
  if (e != cudaSuccess || rc != 0) {
    iblb_batch_destroy(b);
    if (rc) return rc;
    return e == cudaErrorMemoryAllocation ? IBLB_ENOMEM : IBLB_ECUDA;
  }
  b->gens.assign(n, 0);
  b->curs.assign(n, 0);
  b->maps.assign(n, 0);
  b->status.assign(n, IBLB_OK);
  *out = b;
  return IBLB_OK;
}

void iblb_batch_destroy(iblb_batch *b) {
  if (!b) return;
  for (cudaStream_t s : b->streams) cudaStreamSynchronize(s);
  cudaStreamSynchronize(b->stream);
  if (b->part.ib) cudaStreamSynchronize(b->part.ib);
  if (b->part.ls) cudaStreamSynchronize(b->part.ls);
  if (b->arena) cudaFree(b->arena);
  for (iblb_ctx *h : b->inst) iblb_destroy(h);
  for (cudaEvent_t ev : b->joins) cudaEventDestroy(ev);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t ev : {b->ev_force, b->ev_coll, b->ev_join})
    if (ev) cudaEventDestroy(ev);
  if (b->part.green[0]) {
    iblb::release_sms(b->part);
  } else {
    if (b->part.ib) cudaStreamDestroy(b->part.ib);
    if (b->part.ls) cudaStreamDestroy(b->part.ls);
  }
  if (b->health) cudaFreeHost(b->health);
  delete b;
}

const char *iblb_batch_last_error(const iblb_batch *b) { return b ? b->err.c_str() : "null batch"; }

int32_t iblb_batch_size(const iblb_batch *b) { return b ? (int32_t)b->inst.size() : -1; }

iblb_ctx *iblb_batch_context(iblb_batch *b, int32_t i) {
  if (!b || i < 0 || i >= (int32_t)b->inst.size()) return nullptr;
  return b->inst[i];
}

int iblb_batch_tune(iblb_batch *b, int32_t trials) {
  if (!b || trials < 1) return IBLB_EINVAL;
  // one choice per lattice shape and precision: the rows per block of the stream-collide
  // pass (1, 2 or 4 lattice rows within the 128-thread launch bound), timed on the
  // instance's own stream without advancing it (the pass writes only the array that the
  // next step overwrites)
  std::map<std::tuple<int, int, int, int>, int> best_rows;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BATCH_TRY(b, cudaEventCreate(&e0));
  BATCH_TRY(b, cudaEventCreate(&e1));
  int rc = 0;
  for (size_t i = 0; i < b->inst.size() && rc == 0; i++) {
    Ctx &c = b->inst[i]->c;
    const auto key = std::make_tuple(c.nx, c.ny, c.nz, c.precision);
    auto it = best_rows.find(key);
    if (it == best_rows.end()) {
      float best = 1e30f;
      int pick = 1;
      for (int rows : {1, 2, 4}) {
        c.k1_rows = rows;
        if (iblb::k1_block_rows(c) != rows) continue;  // beyond the launch bound
        float total = 0.f;
        for (int t = 0; t <= trials && rc == 0; t++) {  // launch 0 warms up
          cudaError_t e = cudaEventRecord(e0, c.stream);
          if (e == cudaSuccess) e = iblb::launch_stream_collide(c, c.fresh, c.stream);
          if (e == cudaSuccess) e = cudaEventRecord(e1, c.stream);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          float ms = 0.f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          if (e != cudaSuccess) rc = bfail(b, IBLB_ECUDA, std::string("tuning: ") + cudaGetErrorString(e));
          if (t > 0) total += ms;
        }
        if (rc == 0 && total < best) {
          best = total;
          pick = rows;
        }
      }
      it = best_rows.emplace(key, pick).first;
    }
    c.k1_rows = it->second;
    c.config_gen++;  // the launch shape changed: the batched records are stale
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

int32_t iblb_batch_k1_rows(const iblb_batch *b, int32_t i) {
  if (!b || i < 0 || i >= (int32_t)b->inst.size()) return -1;
  return iblb::k1_block_rows(b->inst[i]->c);
}

int iblb_batch_step(iblb_batch *b, int32_t nsteps) {
  if (!b) return IBLB_EINVAL;
  if (nsteps < 0) return bfail(b, IBLB_EINVAL, "nsteps < 0");
  const size_t n = b->inst.size();
  std::fill(b->status.begin(), b->status.end(), IBLB_OK);
  if (nsteps == 0) return IBLB_OK;
  // every instance starts after the caller's stream; its health word is cleared
  for (size_t i = 0; i < n; i++) {
    Ctx &c = b->inst[i]->c;
    BATCH_TRY(b, follow(c.stream, b->stream, b->joins[i]));
    // a failure of the instance's own iblb_step_async steps, still unread, stays in the word
    if (!c.health_pending) BATCH_TRY(b, cudaMemsetAsync(c.counters + 3, 0, sizeof(int), c.stream));
  }
  int done = 0;
  // a freshly initialised state is collided in place by its first step, which the batched
  // kernels do not do: every instance takes that step through the single-context kernels
  bool any_fresh = false;
  for (size_t i = 0; i < n; i++) any_fresh = any_fresh || b->inst[i]->c.fresh;
  if (any_fresh) {
    for (size_t i = 0; i < n; i++)
      if (int rc = iblb::enqueue_steps(b->inst[i]->c, 1)) return inst_fail(b, (int)i, rc);
    done = 1;
  }
  if (nsteps - done >= kPairSteps) {
    if (!tables_current(b))
      if (int rc = build_tables(b)) return rc;
    // the partition streams start after everything queued on the instances' streams
    for (size_t i = 0; i < n; i++) BATCH_TRY(b, follow(b->stream, b->inst[i]->c.stream, b->joins[i]));
    BATCH_TRY(b, follow(b->part.ib, b->stream, b->ev_join));
    BATCH_TRY(b, follow(b->part.ls, b->stream, b->ev_join));
    for (; nsteps - done >= kPairSteps; done += kPairSteps) {
      for (int p = 0; p < kPairSteps; p++)
        if (int rc = enqueue_batched_step(b, p)) return rc;
      for (size_t i = 0; i < n; i++) {
        Ctx &c = b->inst[i]->c;
        c.steps_done += kPairSteps;
        if (c.nv) c.have_force = 1;
        c.fresh = 0;
      }
    }
    BATCH_TRY(b, follow(b->stream, b->part.ib, b->ev_join));
    BATCH_TRY(b, follow(b->stream, b->part.ls, b->ev_join));
    for (size_t i = 0; i < n; i++) BATCH_TRY(b, follow(b->inst[i]->c.stream, b->stream, b->joins[i]));
  }
  if (nsteps > done)
    for (size_t i = 0; i < n; i++)
      if (int rc = iblb::enqueue_steps(b->inst[i]->c, nsteps - done)) return inst_fail(b, (int)i, rc);
  // the caller's stream continues after every instance; then the health words are read
  for (size_t i = 0; i < n; i++) {
    Ctx &c = b->inst[i]->c;
    BATCH_TRY(b, follow(b->stream, c.stream, b->joins[i]));
    BATCH_TRY(b, cudaMemcpyAsync(b->health + i, c.counters + 3, sizeof(int), cudaMemcpyDeviceToHost,
                                 b->stream));
  }
  BATCH_TRY(b, cudaStreamSynchronize(b->stream));
  int first = IBLB_OK;
  for (size_t i = 0; i < n; i++) {
    b->inst[i]->c.health_pending = 0;
    b->status[i] = iblb::health_status(b->inst[i]->c, b->health[i]);
    if (b->status[i] != IBLB_OK && first == IBLB_OK) {
      first = b->status[i];
      b->err = "instance " + std::to_string(i) + ": " + b->inst[i]->c.err;
    }
  }
  return first;
}

int iblb_batch_status(const iblb_batch *b, int32_t *status) {
  if (!b || !status) return IBLB_EINVAL;
  for (size_t i = 0; i < b->inst.size(); i++) status[i] = b->status[i];
  return IBLB_OK;
}

}  // extern "C"
