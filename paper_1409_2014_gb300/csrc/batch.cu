// batch.cu -- many densities (of possibly different grids) per launch sequence.
//
// Members that share a plan are solved together: every kernel of the pipeline
// runs once for the whole group, its persistent CTAs iterating over
// (member, work item) pairs.  The groups (one per distinct plan) are scheduled
// in one of two ways:
//   * one launch per pipeline stage for all groups (batch_ragged.cu), each
//     group on its own range of the stage's CTAs -- eight launches per batch
//     whatever the number of grid sizes (mixed-precision plans of 256^2 ..
//     2048^2 with the DS multiplier);
//   * one launch sequence per group on forked streams, so that different grid
//     sizes overlap (any plans).
// DSNU_BATCH_AUTO takes the forked streams: on GB300 they solve the 64-member
// batch of grids 256^2 .. 2048^2 in 3.26 ms against 3.43 ms for the stage
// launches, since the hardware interleaves the concurrent groups' stages
// while a stage launch ends for all groups at once.  Either launch sequence
// can be captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace {

struct Group {
  dsnu_plan plan;
  std::vector<int> members;        // indices into the batch
  std::vector<dsnu::Member> host;  // bound pointers
  dsnu::Member* dev = nullptr;     // device copy of `host`
  cudaStream_t stream = nullptr;   // fork target
  cudaEvent_t done = nullptr;
};

dsnu_status bfail(dsnu_status s, const std::string& m) {
  dsnu::set_last_error(m);
  return s;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

struct dsnu_batch_s {
  int count = 0;
  std::vector<dsnu_plan> plans;
  std::vector<size_t> ws_off;  // per member, bytes into the batch workspace
  size_t ws_total = 0;
  std::vector<Group> groups;
  cudaEvent_t fork = nullptr;
  bool bound = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int schedule = DSNU_BATCH_AUTO;  // requested
  dsnu::Ragged* ragged = nullptr;   // the one-launch-per-stage tables, when in use
};

static void drop_graph(dsnu_batch_s* B) {
  if (B->exec) {
    cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
  }
  if (B->graph) {
    cudaGraphDestroy(B->graph);
    B->graph = nullptr;
  }
}

// (Re)build the one-launch-per-stage tables for the bound members when the
// schedule asks for them.
static dsnu_status setup_schedule(dsnu_batch_s* B) {
  dsnu::ragged_destroy(B->ragged);
  B->ragged = nullptr;
  if (!B->bound || B->schedule != DSNU_BATCH_STAGE_LAUNCHES) return DSNU_OK;
  std::vector<dsnu_plan> plans;
  for (const Group& g : B->groups) plans.push_back(g.plan);
  std::string why;
  if (!dsnu::ragged_eligible(plans.data(), int(plans.size()), &why))
    return bfail(DSNU_EUNSUPPORTED, "one launch per stage: " + why);
  std::vector<dsnu::RaggedGroupIn> in;
  for (const Group& g : B->groups)
    in.push_back(dsnu::RaggedGroupIn{g.plan, g.dev, g.host[0], int(g.members.size())});
  return dsnu::ragged_create(in.data(), int(in.size()), &B->ragged);
}

static dsnu_status enqueue(dsnu_batch_s* B, cudaStream_t st) {
  if (B->ragged) return dsnu::ragged_enqueue(B->ragged, st);
  if (cudaEventRecord(B->fork, st) != cudaSuccess) return bfail(DSNU_ECUDA, "event record failed");
  for (Group& g : B->groups) {
    if (cudaStreamWaitEvent(g.stream, B->fork, 0) != cudaSuccess) return bfail(DSNU_ECUDA, "stream wait failed");
    dsnu::Members m;
    m.dev = g.dev;
    m.count = int(g.members.size());
    m.one = g.host[0];
    const dsnu_plan p = g.plan;
    const dsnu_status s = (p->geom.precision == DSNU_MIXED)
                              ? dsnu::run_pipeline_f32(p->geom, p->tab, p->ws_layout, m, g.stream, 0, nullptr)
                              : dsnu::run_pipeline_f64(p->geom, p->tab, p->ws_layout, m, g.stream, 0, nullptr);
    if (s != DSNU_OK) return s;
    if (cudaEventRecord(g.done, g.stream) != cudaSuccess) return bfail(DSNU_ECUDA, "event record failed");
    if (cudaStreamWaitEvent(st, g.done, 0) != cudaSuccess) return bfail(DSNU_ECUDA, "stream wait failed");
  }
  return DSNU_OK;
}

static void release(dsnu_batch_s* B) {
  drop_graph(B);
  dsnu::ragged_destroy(B->ragged);  // (the caller has no solve of the batch in flight)
  for (Group& g : B->groups) {
    if (g.stream) cudaStreamSynchronize(g.stream);
    if (g.dev) cudaFree(g.dev);
    if (g.done) cudaEventDestroy(g.done);
    if (g.stream) cudaStreamDestroy(g.stream);
  }
  if (B->fork) cudaEventDestroy(B->fork);
}

extern "C" {

dsnu_status dsnu_batch_create(int32_t count, const dsnu_plan* plans, dsnu_batch* out) {
  if (count < 1 || !plans || !out) return bfail(DSNU_EINVAL, "count >= 1, plans and out required");
  dsnu_batch_s* B = new (std::nothrow) dsnu_batch_s();
  if (!B) return bfail(DSNU_ENOMEM, "host allocation failed");
  B->count = count;
  B->plans.assign(plans, plans + count);
  B->ws_off.resize(count);
  for (int i = 0; i < count; ++i) {
    if (!plans[i]) {
      delete B;
      return bfail(DSNU_EINVAL, "NULL plan in batch");
    }
    B->ws_off[i] = B->ws_total;
    B->ws_total += align256(plans[i]->ws_layout.total);
    Group* g = nullptr;
    for (Group& x : B->groups)
      if (x.plan == plans[i]) g = &x;
    if (!g) {
      B->groups.emplace_back();
      g = &B->groups.back();
      g->plan = plans[i];
    }
    g->members.push_back(i);
  }
  cudaError_t e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
  for (Group& g : B->groups) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&g.dev, g.members.size() * sizeof(dsnu::Member));
  }
  if (e != cudaSuccess) {
    release(B);
    delete B;
    return bfail(DSNU_ECUDA, std::string("batch set-up: ") + cudaGetErrorString(e));
  }
  *out = B;
  return DSNU_OK;
}

size_t dsnu_batch_workspace_bytes(dsnu_batch b) { return b ? b->ws_total : 0; }

dsnu_status dsnu_batch_bind(dsnu_batch b, const double* const* rho_dev, double* const* phi_dev,
                            void* workspace_dev, size_t bytes, void* stream) {
  if (!b || !rho_dev || !phi_dev || !workspace_dev) return bfail(DSNU_EINVAL, "NULL argument");
  if (bytes < b->ws_total) return bfail(DSNU_EINVAL, "batch workspace too small");
  if (reinterpret_cast<uintptr_t>(workspace_dev) & 255) return bfail(DSNU_EINVAL, "workspace must be 256-byte aligned");
  for (int i = 0; i < b->count; ++i)
    if (!rho_dev[i] || !phi_dev[i]) return bfail(DSNU_EINVAL, "NULL member pointer");
  for (int i = 0; i < b->count; ++i)
    if ((reinterpret_cast<uintptr_t>(rho_dev[i]) | reinterpret_cast<uintptr_t>(phi_dev[i])) & 15)
      return bfail(DSNU_EINVAL, "member buffers must be 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace_dev);
  cudaError_t e = cudaSuccess;
  for (Group& g : b->groups) {
    g.host.clear();
    for (int i : g.members) g.host.push_back(dsnu::Member{rho_dev[i], phi_dev[i], ws + b->ws_off[i]});
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g.dev, g.host.data(), g.host.size() * sizeof(dsnu::Member), cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return bfail(DSNU_ECUDA, std::string("member table upload: ") + cudaGetErrorString(e));
  drop_graph(b);
  b->bound = true;
  return setup_schedule(b);
}

dsnu_status dsnu_batch_set_schedule(dsnu_batch b, int32_t schedule) {
  if (!b) return bfail(DSNU_EINVAL, "NULL batch");
  if (schedule != DSNU_BATCH_AUTO && schedule != DSNU_BATCH_STAGE_LAUNCHES && schedule != DSNU_BATCH_FORKED_STREAMS)
    return bfail(DSNU_EINVAL, "unknown batch schedule");
  const int old = b->schedule;
  b->schedule = schedule;
  drop_graph(b);
  const dsnu_status s = setup_schedule(b);
  if (s != DSNU_OK) {
    b->schedule = old;
    setup_schedule(b);
  }
  return s;
}

int32_t dsnu_batch_schedule(dsnu_batch b) {
  if (!b || !b->bound) return -1;
  return b->ragged ? DSNU_BATCH_STAGE_LAUNCHES : DSNU_BATCH_FORKED_STREAMS;
}

int32_t dsnu_batch_launches(dsnu_batch b) {
  if (!b || !b->bound) return -1;
  if (b->ragged) return dsnu::ragged_launches(b->ragged);
  int n = 0;
  for (const Group& g : b->groups) n += g.plan->geom.standard ? 3 : dsnu::kStages;
  return n;
}

dsnu_status dsnu_batch_capture_graph(dsnu_batch b, void* stream) {
  if (!b || !b->bound) return bfail(DSNU_EINVAL, "batch not bound (dsnu_batch_bind)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bfail(DSNU_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
  const dsnu_status s = enqueue(b, st);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(st, &graph);
  if (s != DSNU_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return bfail(DSNU_ECUDA, std::string("end capture: ") + cudaGetErrorString(e));
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return bfail(DSNU_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->graph = graph;
  b->exec = exec;
  return DSNU_OK;
}

dsnu_status dsnu_batch_solve(dsnu_batch b, void* stream) {
  if (!b || !b->bound) return bfail(DSNU_EINVAL, "batch not bound (dsnu_batch_bind)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (b->exec) {
    const cudaError_t e = cudaGraphLaunch(b->exec, st);
    return e == cudaSuccess ? DSNU_OK : bfail(DSNU_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  }
  return enqueue(b, st);
}

dsnu_status dsnu_batch_destroy(dsnu_batch b) {
  if (!b) return DSNU_OK;
  release(b);
  delete b;
  return DSNU_OK;
}

}  // extern "C"
