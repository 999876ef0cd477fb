// Serving form: a request loop over many completion jobs on one GPU.
//
// mc_submit copies a job (its observed entries and SVT parameters) and
// queues it; worker threads admit queued jobs in arrival order whenever a
// slot is free and the job's device-memory footprint fits the server's
// budget, so jobs that arrive while others run start as soon as slots and
// memory free up (continuous batching).  An admitted job gets its own handle
// and CUDA stream: its sparse iterate, recycled subspace and factors stay
// resident on the device, and the kernels of different jobs overlap on the
// GPU.  A finished job's factors are copied to host memory, its device
// memory is released at once and the next queued job is admitted.  Every
// kernel is deterministic, so a job's result does not depend on what else
// runs beside it.
//
// With simulate != 0 the workers do not touch the GPU: a job "runs" for
// params.i_max microseconds and returns an empty result, which lets the
// admission, ordering and cancellation logic be exercised on any host.
#include "mc_common.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

enum JobState { QUEUED = 0, ACTIVE = 1, DONE = 2, CANCELLED = 3, FAILED = 4 };

struct Job {
  uint64_t id = 0;
  int64_t m = 0, n = 0;
  std::vector<int64_t> row_ptr;
  std::vector<int32_t> col;
  std::vector<float> val;
  mc_params prm{};
  size_t footprint = 0;
  size_t dev_now = 0, dev_peak = 0;  // device bytes held through the job's allocator
  cudaMemPool_t pool = nullptr;
  JobState state = QUEUED;
  std::atomic<bool> cancel{false};
  mc_status status = MC_PENDING;
  std::string error;
  // result
  int iters = 0, r = 0, converged = 0;
  double err = 0;
  std::vector<float> Us, V, sigma;
  Clock::time_point t_submit, t_start, t_end;
};

}  // namespace

struct mc_server_s {
  size_t budget = 0, in_use = 0, peak_in_use = 0;
  int max_active = 1, device = 0, simulate = 0;
  int active = 0, peak_active = 0;
  int64_t completed = 0;
  uint64_t next_id = 1;
  cudaMemPool_t pool = nullptr;  // the server's own stream-ordered pool
  bool stopping = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::map<uint64_t, std::unique_ptr<Job>> jobs;
  std::vector<std::thread> workers;
  std::vector<uint64_t> admit_order;
};

namespace {

// Device bytes a job may need (an upper bound used for admission): the CSR
// and CSC arrays with their segment plans, and the panels and small matrices
// at the widest block K_t its parameters allow.
size_t job_footprint(int64_t m, int64_t n, int64_t nnz, const mc_params &p) {
  const int64_t mn = std::min(m, n);
  const int64_t kcap = p.k_max > 0 ? std::min<int64_t>(p.k_max, mn) : mn;
  const int64_t kt = std::max<int64_t>(
      1, std::min<int64_t>({1024, mn, (kcap + std::max(p.s, 0)) * (std::max(p.p_max, p.p0) + 1)}));
  const size_t sparse = 28u * (size_t)nnz + 8u * (size_t)(m + n + 2) + 16u * (size_t)(m + n + nnz / 128 + 2);
  const size_t panels = 4u * 6u * (size_t)(m + n) * (size_t)kt;
  const size_t small = 4u * 8u * (size_t)kt * (size_t)kt + 4u * mc::gemm_tn_scratch_floats(std::max(m, n), (int)kt, (int)kt) +
                       mc::eig_work_bytes((int)kt, (int)kt);
  return sparse + panels + small + (size_t(8) << 20);
}

void *job_alloc(void *ctx, size_t bytes, void *stream) {
  Job *J = static_cast<Job *>(ctx);
  void *p = nullptr;
  if (cudaMallocFromPoolAsync(&p, bytes, J->pool, static_cast<cudaStream_t>(stream)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  J->dev_now += bytes;
  J->dev_peak = std::max(J->dev_peak, J->dev_now);
  return p;
}

void job_free(void *ctx, void *ptr, size_t bytes, void *stream) {
  Job *J = static_cast<Job *>(ctx);
  cudaFreeAsync(ptr, static_cast<cudaStream_t>(stream));
  J->dev_now -= std::min(J->dev_now, bytes);
}

void run_job(mc_server_s *S, Job *J) {
  if (S->simulate) {
    std::this_thread::sleep_for(std::chrono::microseconds(std::max(0, J->prm.i_max)));
    J->iters = J->prm.i_max;
    J->status = J->cancel.load() ? MC_ECANCELLED : MC_OK;
    return;
  }
  cudaSetDevice(S->device);
  J->pool = S->pool;
  mc_allocator hook{J, job_alloc, job_free};
  mc_handle h = nullptr;
  mc_status st = mc_create(&h, J->m, J->n, (int64_t)J->col.size(), J->row_ptr.data(), J->col.data(), J->val.data(),
                           nullptr, &hook);
  if (st != MC_OK) {
    J->status = st;
    J->error = mc_last_error();
    return;
  }
  mc::handle_single_stream(h);  // many jobs share the GPU's work queues
  mc_iter_info info{};
  mc_status last = MC_OK;
  int it = 0;
  for (; it < J->prm.i_max; ++it) {
    if (J->cancel.load()) {
      last = MC_ECANCELLED;
      break;
    }
    last = mc_svt_step(h, &J->prm, &info);
    if (last != MC_OK || info.converged) break;
  }
  if (last == MC_OK || last == MC_ECANCELLED) {
    int r = 0;
    if (mc_svt_factors(h, 0, nullptr, nullptr, nullptr, &r) == MC_OK && last == MC_OK) {
      J->Us.resize((size_t)J->m * r);
      J->V.resize((size_t)J->n * r);
      J->sigma.resize(r);
      mc_svt_factors(h, r, J->Us.data(), J->V.data(), J->sigma.data(), &r);
    }
    J->r = r;
  } else {
    J->error = mc_last_error();
  }
  J->iters = info.i;
  J->err = info.err;
  J->converged = info.converged;
  J->status = last == MC_OK ? (info.converged ? MC_OK : MC_ENOTCONVERGED) : last;
  mc_destroy(h);
}

void worker_loop(mc_server_s *S) {
  if (!S->simulate) cudaSetDevice(S->device);
  for (;;) {
    Job *J = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stopping) return;
        // admit the head of the queue when its footprint fits (arrival order)
        while (!S->queue.empty()) {
          auto it = S->jobs.find(S->queue.front());
          if (it == S->jobs.end() || it->second->state != QUEUED) {
            S->queue.pop_front();
            continue;
          }
          break;
        }
        if (!S->queue.empty()) {
          Job *cand = S->jobs[S->queue.front()].get();
          if (S->in_use + cand->footprint <= S->budget || S->active == 0) {
            S->queue.pop_front();
            J = cand;
            J->state = ACTIVE;
            J->t_start = Clock::now();
            S->in_use += J->footprint;
            S->peak_in_use = std::max(S->peak_in_use, S->in_use);
            S->active += 1;
            S->peak_active = std::max(S->peak_active, S->active);
            S->admit_order.push_back(J->id);
            break;
          }
        }
        S->cv_work.wait(lk);
      }
    }
    try {
      run_job(S, J);
    } catch (...) {
      J->status = MC_EINTERNAL;
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      J->t_end = Clock::now();
      J->state = J->status == MC_ECANCELLED ? CANCELLED : (J->status == MC_OK || J->status == MC_ENOTCONVERGED ? DONE : FAILED);
      S->in_use -= J->footprint;
      S->active -= 1;
      S->completed += 1;
      // the job's input copies are no longer needed
      std::vector<int64_t>().swap(J->row_ptr);
      std::vector<int32_t>().swap(J->col);
      std::vector<float>().swap(J->val);
    }
    S->cv_work.notify_all();
    S->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

mc_status mc_server_create(mc_server *out, size_t budget_bytes, int max_active, int device, int simulate) {
  if (!out || max_active < 1 || max_active > 256) return MC_EINVAL;
  *out = nullptr;
  auto *S = new (std::nothrow) mc_server_s();
  if (!S) return MC_ENOMEM;
  S->budget = budget_bytes;
  S->max_active = max_active;
  S->device = device;
  S->simulate = simulate;
  if (!simulate) {
    size_t free_b = 0, total_b = 0;
    if (cudaSetDevice(device) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      delete S;
      return MC_ECUDA;
    }
    if (budget_bytes == 0) S->budget = free_b / 2;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&S->pool, &props) != cudaSuccess) {
      cudaGetLastError();
      delete S;
      return MC_ECUDA;
    }
    // keep freed blocks for the next job instead of returning them at every synchronisation
    uint64_t keep = S->budget;
    cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  try {
    for (int i = 0; i < max_active; ++i) S->workers.emplace_back(worker_loop, S);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stopping = true;
    }
    S->cv_work.notify_all();
    for (auto &t : S->workers) t.join();
    if (S->pool) cudaMemPoolDestroy(S->pool);
    delete S;
    return MC_EINTERNAL;
  }
  *out = S;
  return MC_OK;
}

void mc_server_destroy(mc_server S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto &kv : S->jobs) kv.second->cancel.store(true);
    S->stopping = true;
  }
  S->cv_work.notify_all();
  for (auto &t : S->workers) t.join();
  if (S->pool) cudaMemPoolDestroy(S->pool);
  delete S;
}

mc_status mc_submit(mc_server S, const mc_job_desc *d, uint64_t *job_id) {
  if (!S || !d || !job_id) return MC_EINVAL;
  if (d->m < 1 || d->n < 1 || d->nnz < 0 || !d->row_ptr || (d->nnz > 0 && (!d->col || !d->val))) return MC_EINVAL;
  std::unique_ptr<Job> J(new (std::nothrow) Job());
  if (!J) return MC_ENOMEM;
  try {
    J->m = d->m;
    J->n = d->n;
    J->row_ptr.assign(d->row_ptr, d->row_ptr + d->m + 1);
    J->col.assign(d->col, d->col + d->nnz);
    J->val.assign(d->val, d->val + d->nnz);
  } catch (...) {
    return MC_ENOMEM;
  }
  J->prm = d->params;
  J->footprint = job_footprint(d->m, d->n, d->nnz, d->params);
  J->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) return MC_EBUSY;
    J->id = S->next_id++;
    *job_id = J->id;
    S->queue.push_back(J->id);
    S->jobs[J->id] = std::move(J);
  }
  S->cv_work.notify_all();
  return MC_OK;
}

mc_status mc_cancel(mc_server S, uint64_t job_id) {
  if (!S) return MC_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(job_id);
  if (it == S->jobs.end()) return MC_EINVAL;
  Job *J = it->second.get();
  J->cancel.store(true);
  if (J->state == QUEUED) {
    J->state = CANCELLED;
    J->status = MC_ECANCELLED;
    J->t_start = J->t_end = Clock::now();
  }
  return MC_OK;
}

mc_status mc_poll(mc_server S, uint64_t job_id, mc_result *out) {
  if (!S || !out) return MC_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(job_id);
  if (it == S->jobs.end()) return MC_EINVAL;
  Job *J = it->second.get();
  if (J->state == QUEUED || J->state == ACTIVE) return MC_PENDING;
  std::memset(out, 0, sizeof(*out));
  out->status = J->status;
  out->iters = J->iters;
  out->r = J->r;
  out->converged = J->converged;
  out->err = J->err;
  out->m = J->m;
  out->n = J->n;
  out->Us = J->Us.empty() ? nullptr : J->Us.data();
  out->V = J->V.empty() ? nullptr : J->V.data();
  out->sigma = J->sigma.empty() ? nullptr : J->sigma.data();
  out->queue_s = std::chrono::duration<double>(J->t_start - J->t_submit).count();
  out->latency_s = std::chrono::duration<double>(J->t_end - J->t_submit).count();
  out->footprint_bytes = J->footprint;
  out->device_bytes_peak = J->dev_peak;
  out->message = J->error.c_str();
  return J->status == MC_ECANCELLED ? MC_ECANCELLED : MC_OK;
}

mc_status mc_wait(mc_server S, uint64_t job_id, double timeout_s) {
  if (!S) return MC_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto done = [&] {
    auto it = S->jobs.find(job_id);
    return it == S->jobs.end() || (it->second->state != QUEUED && it->second->state != ACTIVE);
  };
  if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) return MC_ETIMEOUT;
  return S->jobs.count(job_id) ? MC_OK : MC_EINVAL;
}

mc_status mc_result_release(mc_server S, uint64_t job_id) {
  if (!S) return MC_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(job_id);
  if (it == S->jobs.end()) return MC_EINVAL;
  if (it->second->state == QUEUED || it->second->state == ACTIVE) return MC_EBUSY;
  S->jobs.erase(it);
  return MC_OK;
}

mc_status mc_server_stats(mc_server S, mc_server_info *out) {
  if (!S || !out) return MC_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(out, 0, sizeof(*out));
  out->budget_bytes = S->budget;
  out->in_use_bytes = S->in_use;
  out->peak_in_use_bytes = S->peak_in_use;
  out->active = S->active;
  out->peak_active = S->peak_active;
  out->queued = 0;
  for (uint64_t id : S->queue) {
    auto it = S->jobs.find(id);
    if (it != S->jobs.end() && it->second->state == QUEUED) out->queued += 1;
  }
  out->admitted = (int64_t)S->admit_order.size();
  out->completed = S->completed;
  out->slots = S->max_active;
  return MC_OK;
}

int64_t mc_server_admit_order(mc_server S, uint64_t *ids, int64_t cap) {
  if (!S) return -1;
  std::lock_guard<std::mutex> lk(S->mu);
  const int64_t n = (int64_t)S->admit_order.size();
  for (int64_t i = 0; i < std::min(n, cap); ++i) ids[i] = S->admit_order[i];
  return n;
}

}  // extern "C"
