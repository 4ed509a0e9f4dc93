// Batched ensemble: many independent IB-LB contexts (lattices and meshes of any sizes)
// advanced together. Each context runs the same step as iblb_step, on its own stream and
// without an SM partition; the batch captures two steps of every context into one CUDA graph
// and replays it, so the instances' small kernels run side by side from one graph launch per
// two steps instead of one host launch each. Two steps return every context's
// double-buffer indices (populations, tile maps) to where they started, which is what lets
// the same graph be replayed. The paper advances one box at a time; this is the ensemble form
// of its parameter sweeps (Sec. V).
#include <algorithm>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "iblb_internal.cuh"

using iblb::Ctx;

struct iblb_batch {
  std::vector<iblb_ctx *> inst;
  std::vector<cudaStream_t> streams;  // one per instance (the instance's own stream)
  std::vector<cudaEvent_t> joins;     // one per instance
  cudaStream_t stream = nullptr;      // caller's stream
  cudaStream_t cap = nullptr;         // origin stream of the graph capture
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<uint64_t> gens;  // config_gen, cur, map of every instance when captured
  std::vector<int> curs, maps;
  std::vector<int> status;     // per-instance result of the last iblb_batch_step
  int *health = nullptr;       // pinned, one word per instance
  std::string err;
};

namespace {

constexpr int kGraphSteps = 2;  // even: the double buffers are back in place after a replay

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

bool graph_current(const iblb_batch *b) {
  if (!b->exec) return false;
  for (size_t i = 0; i < b->inst.size(); i++) {
    const Ctx &c = b->inst[i]->c;
    if (b->gens[i] != c.config_gen || b->curs[i] != c.cur || b->maps[i] != c.map) return false;
  }
  return true;
}

// Capture kGraphSteps steps of every instance into b->exec. Queuing a step advances the host
// copy of a context's state (buffer indices, counters), so that state is put back afterwards:
// the graph has been recorded, nothing has run.
int capture(iblb_batch *b) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  BATCH_TRY(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  int rc = 0;
  if (cudaEventRecord(b->fork, b->cap) != cudaSuccess) rc = bfail(b, IBLB_ECUDA, "capture fork");
  for (size_t i = 0; i < b->inst.size() && rc == 0; i++) {
    Ctx &c = b->inst[i]->c;
    const int cur = c.cur, map = c.map, fresh = c.fresh, have_force = c.have_force;
    const int64_t steps = c.steps_done, k1l = c.k1_launches, kl = c.kernel_launches;
    if (cudaStreamWaitEvent(c.stream, b->fork, 0) != cudaSuccess) rc = IBLB_ECUDA;
    if (rc == 0) rc = iblb::enqueue_steps(c, kGraphSteps);
    if (rc == 0 && cudaEventRecord(b->joins[i], c.stream) != cudaSuccess) rc = IBLB_ECUDA;
    if (rc == 0 && cudaStreamWaitEvent(b->cap, b->joins[i], 0) != cudaSuccess) rc = IBLB_ECUDA;
    c.cur = cur;
    c.map = map;
    c.fresh = fresh;
    c.have_force = have_force;
    c.steps_done = steps;
    c.k1_launches = k1l;
    c.kernel_launches = kl;
    if (rc) rc = inst_fail(b, (int)i, rc);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return bfail(b, IBLB_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  const cudaError_t e2 = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) {
    b->exec = nullptr;
    return bfail(b, IBLB_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2));
  }
  for (size_t i = 0; i < b->inst.size(); i++) {
    const Ctx &c = b->inst[i]->c;
    b->gens[i] = c.config_gen;
    b->curs[i] = c.cur;
    b->maps[i] = c.map;
  }
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
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
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
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (iblb_ctx *h : b->inst) iblb_destroy(h);
  for (cudaEvent_t ev : b->joins) cudaEventDestroy(ev);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
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
    c.config_gen++;  // the launch shape changed: a captured graph is stale
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
    BATCH_TRY(b, cudaMemsetAsync(c.counters + 3, 0, sizeof(int), c.stream));
  }
  int done = 0;
  // a freshly initialised state is collided in place by its first step, which the graph
  // does not hold: every instance takes that step directly
  bool any_fresh = false;
  for (size_t i = 0; i < n; i++) any_fresh = any_fresh || b->inst[i]->c.fresh;
  if (any_fresh) {
    for (size_t i = 0; i < n; i++)
      if (int rc = iblb::enqueue_steps(b->inst[i]->c, 1)) return inst_fail(b, (int)i, rc);
    done = 1;
  }
  if (nsteps - done >= kGraphSteps) {
    if (!graph_current(b))
      if (int rc = capture(b)) return rc;
    for (size_t i = 0; i < n; i++) BATCH_TRY(b, follow(b->stream, b->inst[i]->c.stream, b->joins[i]));
    for (; nsteps - done >= kGraphSteps; done += kGraphSteps) {
      BATCH_TRY(b, cudaGraphLaunch(b->exec, b->stream));
      for (size_t i = 0; i < n; i++) {
        Ctx &c = b->inst[i]->c;
        c.steps_done += kGraphSteps;
        if (c.nv) c.have_force = 1;
        c.fresh = 0;
      }
    }
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
