// Host side of the batched launch: the plan (job and state tables plus a
// workspace for many networks), rac_plan_* entry points, and the
// multi-network path of rac_enforce_batch.
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "rac_internal.h"

namespace rac {
rac_status launch_batch(const BatchParams &P, cudaStream_t stream);
}

using namespace rac;

struct rac_plan {
  int device = 0;
  int32_t n_items = 0, n_jobs = 0, total_states = 0, total_slabs = 0;
  int64_t chg_slot_words = 0, u_slot_words = 0, bufB_words = 0;
  size_t rel_bytes = 0;  // relation stores of the jobs
  bool any_packed = false;  // some network's relation rows are packed
  // device tables
  BatchJob *jobs = nullptr;
  int64_t *state_off = nullptr, *scratch_off = nullptr, *chg_off = nullptr;
  int32_t *res_idx = nullptr, *state_job = nullptr;
  int32_t *chg_state = nullptr;  // state of each word of a chg slot
  // device workspace (clean between launches)
  uint32_t *bufB = nullptr, *any = nullptr, *wipe = nullptr, *chg = nullptr, *chgU = nullptr;
  uint32_t *st_info = nullptr, *job_alive = nullptr;
  BatchSync *sync = nullptr;
  bool stream_ordered = false;  // allocated with cudaMallocAsync (temporary plans)
  cudaStream_t alloc_stream = nullptr;
};

namespace {

struct PlanHost {
  std::vector<BatchJob> jobs;
  std::vector<int64_t> state_off, scratch_off, chg_off;
  std::vector<int32_t> res_idx, state_job, chg_state;
  int32_t total_slabs = 0;
  int64_t chg_slot_words = 0, u_slot_words = 0, bufB_words = 0;
  size_t rel_bytes = 0;
  bool any_packed = false;
};

rac_status build_host_plan(const rac_network *const *nets, int32_t n_nets, int32_t n_items,
                           const int32_t *item_net, const int64_t *item_dom_off, PlanHost &H) {
  std::vector<std::vector<int32_t>> groups(size_t(std::max(n_nets, 1)));
  for (int32_t i = 0; i < n_items; ++i) {
    const int32_t k = item_net[i];
    if (k < 0 || k >= n_nets || !nets[k]) {
      set_error("item " + std::to_string(i) + " names a bad network");
      return RAC_EINVAL;
    }
    if (item_dom_off[i] < 0) {
      set_error("item " + std::to_string(i) + " has a negative offset");
      return RAC_EINVAL;
    }
    groups[size_t(k)].push_back(i);
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_error("cudaGetDevice failed");
    return RAC_ECUDA;
  }
  for (int32_t k = 0; k < n_nets; ++k) {
    const std::vector<int32_t> &g = groups[size_t(k)];
    if (g.empty()) continue;
    const rac_network *net = nets[k];
    if (net->device != dev) {
      set_error("the current CUDA device is not the device of network " + std::to_string(k));
      return RAC_EINVAL;
    }
    BatchJob J = {};
    J.rel = static_cast<const uint4 *>(net->d_rel);
    J.slabs = net->d_slabs;
    J.n = net->n;
    J.d = net->d;
    J.q = net->q;
    J.lcode = net->q + (net->packed ? 16 : 0);
    J.nb = net->nb;
    J.n_slabs = int32_t(net->n_slabs);
    J.slab_base = H.total_slabs;
    J.n_states = int32_t(g.size());
    J.state_base = int32_t(H.state_off.size());
    J.u_off = H.u_slot_words;
    H.u_slot_words += net->nb;
    H.total_slabs += J.n_slabs;
    H.rel_bytes += net->rel_bytes;
    H.any_packed = H.any_packed || net->packed != 0;
    const int32_t job = int32_t(H.jobs.size());
    for (int32_t item : g) {
      H.state_off.push_back(item_dom_off[item]);
      H.scratch_off.push_back(H.bufB_words);
      H.bufB_words += (int64_t(net->n) + 31) / 32 * 32;
      H.chg_off.push_back(H.chg_slot_words);
      H.chg_slot_words += net->nb;
      H.chg_state.insert(H.chg_state.end(), size_t(net->nb), int32_t(H.state_job.size()));
      H.res_idx.push_back(item);
      H.state_job.push_back(job);
    }
    H.jobs.push_back(J);
  }
  return RAC_OK;
}

template <typename T>
cudaError_t dev_alloc(rac_plan *p, T **ptr, size_t count) {
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  if (p->stream_ordered) return cudaMallocAsync(reinterpret_cast<void **>(ptr), bytes, p->alloc_stream);
  return cudaMalloc(reinterpret_cast<void **>(ptr), bytes);
}

void plan_free(rac_plan *p) {
  if (!p) return;
  void *ptrs[] = {p->jobs, p->state_off, p->scratch_off, p->chg_off, p->res_idx, p->state_job,
                  p->chg_state,
                  p->bufB, p->any, p->wipe, p->chg, p->chgU, p->st_info, p->job_alive, p->sync};
  for (void *q : ptrs) {
    if (!q) continue;
    if (p->stream_ordered)
      cudaFreeAsync(q, p->alloc_stream);
    else
      cudaFree(q);
  }
  delete p;
}

// Allocate and fill the device side of a plan.  The copies and memsets are
// enqueued on `s` (pageable sources: staged before the calls return).
rac_status plan_upload(rac_plan *p, const PlanHost &H, cudaStream_t s) {
  const int64_t T = int64_t(H.state_off.size());
  const int64_t J = int64_t(H.jobs.size());
  bool ok = dev_alloc(p, &p->jobs, size_t(J)) == cudaSuccess &&
            dev_alloc(p, &p->state_off, size_t(T)) == cudaSuccess &&
            dev_alloc(p, &p->scratch_off, size_t(T)) == cudaSuccess &&
            dev_alloc(p, &p->chg_off, size_t(T)) == cudaSuccess &&
            dev_alloc(p, &p->res_idx, size_t(T)) == cudaSuccess &&
            dev_alloc(p, &p->state_job, size_t(T)) == cudaSuccess &&
            dev_alloc(p, &p->chg_state, size_t(H.chg_slot_words)) == cudaSuccess &&
            dev_alloc(p, &p->bufB, size_t(H.bufB_words)) == cudaSuccess &&
            dev_alloc(p, &p->any, size_t(3 * T)) == cudaSuccess &&
            dev_alloc(p, &p->wipe, size_t(3 * T)) == cudaSuccess &&
            dev_alloc(p, &p->chg, size_t(3 * H.chg_slot_words)) == cudaSuccess &&
            dev_alloc(p, &p->chgU, size_t(3 * H.u_slot_words)) == cudaSuccess &&
            dev_alloc(p, &p->st_info, size_t(T)) == cudaSuccess &&
            dev_alloc(p, &p->job_alive, size_t(3 * J)) == cudaSuccess &&
            dev_alloc(p, &p->sync, 1) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    set_error("device allocation of the batch plan failed");
    return RAC_ENOMEM;
  }
  cudaError_t e = cudaSuccess;
  auto cp = [&](void *dst, const void *src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
  };
  auto zero = [&](void *dst, int v, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemsetAsync(dst, v, bytes, s);
  };
  cp(p->jobs, H.jobs.data(), H.jobs.size() * sizeof(BatchJob));
  cp(p->state_off, H.state_off.data(), H.state_off.size() * 8);
  cp(p->scratch_off, H.scratch_off.data(), H.scratch_off.size() * 8);
  cp(p->chg_off, H.chg_off.data(), H.chg_off.size() * 8);
  cp(p->res_idx, H.res_idx.data(), H.res_idx.size() * 4);
  cp(p->state_job, H.state_job.data(), H.state_job.size() * 4);
  cp(p->chg_state, H.chg_state.data(), H.chg_state.size() * 4);
  // the state every launch expects: scratch domains all ones, the rest zero
  zero(p->bufB, 0xFF, size_t(H.bufB_words) * 4);
  zero(p->any, 0, size_t(3 * T) * 4);
  zero(p->wipe, 0, size_t(3 * T) * 4);
  zero(p->chg, 0, size_t(3 * H.chg_slot_words) * 4);
  zero(p->chgU, 0, size_t(3 * H.u_slot_words) * 4);
  zero(p->st_info, 0, size_t(T) * 4);
  zero(p->job_alive, 0, size_t(3 * J) * 4);
  zero(p->sync, 0, sizeof(BatchSync));
  if (e != cudaSuccess) return cuda_fail(e, "upload of the batch plan");
  p->n_jobs = int32_t(J);
  p->total_states = int32_t(T);
  p->total_slabs = H.total_slabs;
  p->chg_slot_words = H.chg_slot_words;
  p->u_slot_words = H.u_slot_words;
  p->bufB_words = H.bufB_words;
  p->rel_bytes = H.rel_bytes;
  p->any_packed = H.any_packed;
  return RAC_OK;
}

rac_status plan_launch(const rac_plan *p, const uint32_t *dom_in, uint32_t *dom_out,
                       int32_t *iterations, int32_t *status, int32_t max_sweeps, uint32_t flags,
                       cudaStream_t s) {
  if (p->total_states == 0) return RAC_OK;
  BatchParams P = {};
  P.jobs = p->jobs;
  P.n_jobs = p->n_jobs;
  P.total_slabs = p->total_slabs;
  P.total_states = p->total_states;
  P.state_off = p->state_off;
  P.scratch_off = p->scratch_off;
  P.chg_off = p->chg_off;
  P.res_idx = p->res_idx;
  P.dom_in = dom_in;
  P.dom_out = dom_out;
  P.bufB = p->bufB;
  P.iterations = iterations;
  P.status = status;
  P.any = p->any;
  P.wipe = p->wipe;
  P.chg = p->chg;
  P.chgU = p->chgU;
  P.st_info = p->st_info;
  P.job_alive = p->job_alive;
  P.state_job = p->state_job;
  P.chg_state = p->chg_state;
  P.chg_slot_words = p->chg_slot_words;
  P.u_slot_words = p->u_slot_words;
  P.sync = p->sync;
  P.max_sweeps = max_sweeps;
  P.flags = flags;
  P.wait_limit_ns = wait_limit_for(flags);
  P.rel_evict_first = p->rel_bytes > kEvictFirstBytes ? 1u : 0u;
  P.any_packed = p->any_packed ? 1u : 0u;
  return launch_batch(P, s);
}

constexpr uint32_t kPlanFlags = RAC_STOP_ON_WIPEOUT | RAC_INCREMENTAL | RAC_TEST_WITHHOLD_ARRIVAL;  // no tensor kernel

}  // namespace

namespace rac {
// The multi-network path of rac_enforce_batch: a temporary plan whose device
// memory is allocated and freed in stream order around one launch.
rac_status enforce_batch_multi(const rac_network *const *nets, int32_t n_nets, int32_t n_items,
                               const int32_t *item_net, const int64_t *item_dom_off,
                               const uint32_t *dom_in, uint32_t *dom_out, int32_t *iterations,
                               int32_t *status, int32_t max_sweeps, uint32_t flags,
                               cudaStream_t s) {
  PlanHost H;
  rac_status rc = build_host_plan(nets, n_nets, n_items, item_net, item_dom_off, H);
  if (rc != RAC_OK) return rc;
  rac_plan *p = new (std::nothrow) rac_plan();
  if (!p) {
    set_error("out of host memory");
    return RAC_ENOMEM;
  }
  p->stream_ordered = true;
  p->alloc_stream = s;
  cudaGetDevice(&p->device);
  p->n_items = n_items;
  rc = plan_upload(p, H, s);
  if (rc == RAC_OK) rc = plan_launch(p, dom_in, dom_out, iterations, status, max_sweeps, flags, s);
  plan_free(p);  // stream-ordered frees after the launch
  return rc;
}
}  // namespace rac

extern "C" {

rac_status rac_plan_create(const rac_network *const *nets, int32_t n_nets, int32_t n_items,
                           const int32_t *item_net, const int64_t *item_dom_off, rac_plan **out) try {
  set_error("");
  if (!out) {
    set_error("out is NULL");
    return RAC_EINVAL;
  }
  *out = nullptr;
  if (n_items < 0 || n_nets < 0 || (n_items > 0 && (!nets || !item_net || !item_dom_off))) {
    set_error("bad counts or NULL tables");
    return RAC_EINVAL;
  }
  PlanHost H;
  rac_status rc = build_host_plan(nets, n_nets, n_items, item_net, item_dom_off, H);
  if (rc != RAC_OK) return rc;
  rac_plan *p = new (std::nothrow) rac_plan();
  if (!p) {
    set_error("out of host memory");
    return RAC_ENOMEM;
  }
  cudaGetDevice(&p->device);
  p->n_items = n_items;
  rc = plan_upload(p, H, nullptr);
  if (rc == RAC_OK) {
    cudaError_t e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize after the plan upload");
  }
  if (rc != RAC_OK) {
    plan_free(p);
    return rc;
  }
  *out = p;
  return RAC_OK;
} RAC_CATCH_STATUS

rac_status rac_plan_enforce(rac_plan *plan, const uint32_t *dom_in, uint32_t *dom_out,
                            int32_t *iterations, int32_t *status, int32_t max_sweeps,
                            uint32_t flags, rac_stream_t stream) try {
  set_error("");
  if (!plan || (plan->total_states > 0 && (!dom_in || !dom_out || !iterations || !status))) {
    set_error("NULL argument");
    return RAC_EINVAL;
  }
  if (flags & ~kPlanFlags) {
    set_error("unknown flag");
    return RAC_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device) {
    set_error("the current CUDA device is not the plan's device");
    return RAC_EINVAL;
  }
  return plan_launch(plan, dom_in, dom_out, iterations, status, max_sweeps, flags,
                     reinterpret_cast<cudaStream_t>(stream));
} RAC_CATCH_STATUS

void rac_plan_destroy(rac_plan *plan) { plan_free(plan); }

}  // extern "C"
