// Serving runtime: continuous batching of encode requests and decode queries
// of uneven sizes on one GPU.
//
// Requests arrive from any host thread.  Admission is first come, first
// served against a device-memory budget: a request reserves its transient
// buffers plus, for an encode, the resident model it creates, and waits in
// the queue while the budget is short.  Worker threads each own a library
// handle and a CUDA stream; a free worker takes every admitted request of one
// kind and runs it as one job, so jobs of several workers overlap on the
// device and requests that arrive while others run join the next job.
//   encode job: the requests' data are copied into one device buffer and
//               fitted as one batch of independent fits (one launch sequence
//               for all of them); the fitted models stay resident.
//   decode job: the queries' points are copied to the device, every batch
//               they read is decoded in one launch, the values go back.
// A resident model lives until mfa_server_release; a batch is freed (by the
// worker that owns its memory) when its last model is released and no decode
// reads it.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mfa_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct BatchRef {
  mfa_batch* b = nullptr;
  int owner = 0;       // worker whose handle allocated it
  int live = 0;        // models not yet released
  int readers = 0;     // decode jobs in flight on it
  long long keep = 0;  // bytes of budget its resident models hold
};

struct Resident {
  std::shared_ptr<BatchRef> batch;
  int index = 0;
  int dim = 1;
  bool released = false;
};

struct Req {
  int64_t id = 0;
  int kind = 0;  // 0 encode, 1 decode
  mfa_instance inst{};
  const void* q = nullptr;
  int precision = MFA_PREC_MIXED;
  long long q_bytes = 0;
  int64_t model = 0;
  int64_t npts = 0;
  const double* pts = nullptr;
  double* out = nullptr;
  long long need = 0;  // reserved at admission
  long long keep = 0;  // kept after completion (resident model)
  std::shared_ptr<BatchRef> batch;  // decode: the batch read, pinned when the job is taken
  int index = 0;                           // decode: instance within it
  bool admitted = false, done = false;
  int status = MFA_OK;
  double t_submit = 0, t_admit = 0, t_start = 0, t_done = 0;
};

}  // namespace

struct mfa_server {
  int device = 0;
  long long budget = 0, used = 0, peak = 0;
  int max_batch = 64;
  long long max_decode_pts = 1LL << 26;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> queue;                 // submitted, not admitted (FIFO)
  std::deque<Req*> ready_enc, ready_dec;  // admitted, not started
  std::unordered_map<int64_t, std::unique_ptr<Req>> reqs;
  std::unordered_map<int64_t, Resident> models;
  std::vector<std::vector<std::shared_ptr<BatchRef>>> to_free;  // per worker
  std::vector<mfa_handle*> handles;
  std::vector<cudaStream_t> streams;
  std::vector<std::thread> workers;
  mfa_handle* ctl = nullptr;  // API-side queries (control points)
  cudaStream_t ctl_stream = nullptr;
  std::mutex ctl_mu;
  int64_t next_id = 1;
  bool stop = false;
  long long jobs_enc = 0, jobs_dec = 0;
};

namespace {

double now_s(const mfa_server* s) { return std::chrono::duration<double>(Clock::now() - s->t0).count(); }

// Budget of one encode: staged data, the batch's scratch (two float-float
// stages of at most the data size each) and its resident part.
void encode_bytes(const mfa_instance& in, long long q_bytes, int precision, long long* need, long long* keep) {
  (void)precision;
  const long long es = 8;  // FP64 or float-float control points
  long long ncp = 1, tables = 0;
  for (int a = 0; a < in.dim; ++a) {
    ncp *= in.nspans[a] + in.degree;
    tables += in.npts[a] * (long long)(in.degree + 1) * 24 + (in.nspans[a] + in.degree) * 96LL;
  }
  *keep = ncp * es + tables + 4096;
  *need = q_bytes + 2 * (q_bytes / 4 + 1) * es + *keep + (1LL << 20);
}

void admit_locked(mfa_server* s) {
  while (!s->queue.empty()) {
    Req* r = s->queue.front();
    if (s->used + r->need > s->budget) break;  // first come, first served: the head waits
    s->queue.pop_front();
    s->used += r->need;
    s->peak = std::max(s->peak, s->used);
    r->admitted = true;
    r->t_admit = now_s(s);
    (r->kind == 0 ? s->ready_enc : s->ready_dec).push_back(r);
  }
}

bool model_ready_locked(mfa_server* s, int64_t model) {
  auto it = s->models.find(model);
  return it != s->models.end() && !it->second.released;
}

// A decode can run once its model is resident, or must be reported as
// failed once its model is gone (released, or its encode failed); it waits
// while the encode is still queued or running.
bool decode_takeable_locked(mfa_server* s, const Req* r) {
  if (model_ready_locked(s, r->model)) return true;
  auto it = s->reqs.find(r->model);
  return it == s->reqs.end() || it->second->done;
}

void release_batch_locked(mfa_server* s, const std::shared_ptr<BatchRef>& br) {
  if (br->live == 0 && br->readers == 0 && br->b) {
    s->used -= br->keep;
    br->keep = 0;
    s->to_free[br->owner].push_back(br);
  }
}

struct Job {
  int kind = -1;
  std::vector<Req*> reqs;
};

// The oldest admitted work: encodes of one precision, or decodes whose model
// is resident (queries of models still being fitted wait in the list).
Job take_job_locked(mfa_server* s) {
  Job j;
  Req* oldest_dec = nullptr;
  for (Req* r : s->ready_dec)
    if (decode_takeable_locked(s, r)) {
      oldest_dec = r;
      break;
    }
  Req* oldest_enc = s->ready_enc.empty() ? nullptr : s->ready_enc.front();
  if (oldest_enc && (!oldest_dec || oldest_enc->t_admit <= oldest_dec->t_admit)) {
    const int prec = oldest_enc->precision;
    j.kind = 0;
    for (auto it = s->ready_enc.begin(); it != s->ready_enc.end() && (int)j.reqs.size() < s->max_batch;) {
      if ((*it)->precision == prec) {
        j.reqs.push_back(*it);
        it = s->ready_enc.erase(it);
      } else {
        ++it;
      }
    }
  } else if (oldest_dec) {
    j.kind = 1;
    long long pts = 0;
    for (auto it = s->ready_dec.begin(); it != s->ready_dec.end();) {
      Req* r = *it;
      if (decode_takeable_locked(s, r) && (j.reqs.empty() || pts + r->npts <= s->max_decode_pts)) {
        pts += r->npts;
        j.reqs.push_back(r);
        it = s->ready_dec.erase(it);
      } else {
        ++it;
      }
    }
    for (Req* r : j.reqs) {
      auto m = s->models.find(r->model);
      if (m != s->models.end() && !m->second.released) {
        r->batch = m->second.batch;
        r->index = m->second.index;
        r->batch->readers++;
      }
    }
  }
  return j;
}

void finish_locked(mfa_server* s, Req* r, int status) {
  r->status = status;
  r->done = true;
  r->t_done = now_s(s);
  s->used -= r->need - (status == MFA_OK ? r->keep : 0);
}

void run_encode_job(mfa_server* s, int w, Job& j) {
  mfa_handle* h = s->handles[w];
  cudaStream_t st = s->streams[w];
  std::vector<mfa_instance> inst;
  long long total = 0;
  for (Req* r : j.reqs) {
    mfa_instance in = r->inst;
    in.q_offset = total / 4;
    total += r->q_bytes;
    inst.push_back(in);
  }
  void* dq = nullptr;
  cudaError_t e = cudaMallocAsync(&dq, (size_t)total, st);
  long long off = 0;
  for (size_t k = 0; k < j.reqs.size() && e == cudaSuccess; ++k) {
    e = cudaMemcpyAsync((char*)dq + off, j.reqs[k]->q, (size_t)j.reqs[k]->q_bytes, cudaMemcpyDefault, st);
    off += j.reqs[k]->q_bytes;
  }
  mfa_batch* b = nullptr;
  int rc = e == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
  if (rc == MFA_OK)
    rc = mfa_encode_batch(h, (int)inst.size(), inst.data(), dq, MFA_F32, 1, j.reqs[0]->precision, &b);
  if (dq) cudaFreeAsync(dq, st);
  cudaStreamSynchronize(st);
  std::lock_guard<std::mutex> lk(s->mu);
  if (rc == MFA_OK) {
    auto br = std::make_shared<BatchRef>();
    br->b = b;
    br->owner = w;
    br->live = (int)j.reqs.size();
    for (size_t k = 0; k < j.reqs.size(); ++k) {
      Req* r = j.reqs[k];
      br->keep += r->keep;
      s->models[r->id] = Resident{br, (int)k, r->inst.dim, false};
      finish_locked(s, r, MFA_OK);
    }
  } else {
    for (Req* r : j.reqs) finish_locked(s, r, rc);
  }
  s->jobs_enc++;
}

void run_decode_job(mfa_server* s, int w, Job& j) {
  mfa_handle* h = s->handles[w];
  cudaStream_t st = s->streams[w];
  // group the queries by the batch they read
  std::vector<std::pair<std::shared_ptr<BatchRef>, std::vector<std::pair<Req*, int>>>> groups;
  std::vector<Req*> missing;
  for (Req* r : j.reqs) {  // the batches were pinned when the job was taken
    if (!r->batch) {
      missing.push_back(r);
      continue;
    }
    size_t g = 0;
    while (g < groups.size() && groups[g].first != r->batch) ++g;
    if (g == groups.size()) groups.push_back({r->batch, {}});
    groups[g].second.push_back({r, r->index});
  }
  std::vector<std::pair<Req*, int>> results;
  for (auto& g : groups) {
    const int nq = (int)g.second.size();
    std::vector<int64_t> off(nq + 1, 0);
    std::vector<int32_t> qi(nq);
    for (int k = 0; k < nq; ++k) {
      off[k + 1] = off[k] + g.second[k].first->npts;
      qi[k] = g.second[k].second;
    }
    const long long np = off[nq];
    const size_t bytes = (size_t)(nq + 1) * 8 + (size_t)nq * 4 + (size_t)np * 32 + 64;
    void* d = nullptr;
    cudaError_t e = cudaMallocAsync(&d, bytes, st);
    long long* doff = (long long*)d;
    double* dpts = (double*)(doff + nq + 1);
    double* dout = dpts + 3 * np;
    int32_t* dqi = (int32_t*)(dout + np);
    if (e == cudaSuccess) e = cudaMemcpyAsync(doff, off.data(), (nq + 1) * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dqi, qi.data(), nq * 4, cudaMemcpyHostToDevice, st);
    for (int k = 0; k < nq && e == cudaSuccess; ++k)
      if (g.second[k].first->npts)
        e = cudaMemcpyAsync(dpts + 3 * off[k], g.second[k].first->pts, (size_t)g.second[k].first->npts * 24,
                            cudaMemcpyDefault, st);
    int rc = e == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
    if (rc == MFA_OK && np > 0)
      rc = mfa::batch_decode_points_impl(h, g.first->b, nq, dqi, (const int64_t*)doff, dpts, dout, 1);
    for (int k = 0; k < nq && rc == MFA_OK; ++k)
      if (g.second[k].first->npts &&
          cudaMemcpyAsync(g.second[k].first->out, dout + off[k], (size_t)g.second[k].first->npts * 8,
                          cudaMemcpyDefault, st) != cudaSuccess)
        rc = MFA_ERR_CUDA;
    if (d) cudaFreeAsync(d, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == MFA_OK) rc = MFA_ERR_CUDA;
    for (auto& q : g.second) results.push_back({q.first, rc});
  }
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto& g : groups) {
    g.first->readers -= (int)g.second.size();
    release_batch_locked(s, g.first);
    for (auto& q : g.second) q.first->batch.reset();
  }
  for (auto& r : results) finish_locked(s, r.first, r.second);
  for (Req* r : missing) finish_locked(s, r, MFA_ERR_ARG);
  s->jobs_dec++;
}

void worker_loop(mfa_server* s, int w) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    if (!s->to_free[w].empty()) {
      std::vector<std::shared_ptr<BatchRef>> fr;
      fr.swap(s->to_free[w]);
      lk.unlock();
      for (auto& br : fr) {
        mfa_batch_free(br->b);
        br->b = nullptr;
      }
      cudaStreamSynchronize(s->streams[w]);
      lk.lock();
      continue;
    }
    admit_locked(s);
    Job j = take_job_locked(s);
    if (j.kind < 0) {
      if (s->stop && s->queue.empty() && s->ready_enc.empty() && s->ready_dec.empty()) break;
      s->cv.wait(lk);
      continue;
    }
    const double t = now_s(s);
    for (Req* r : j.reqs) r->t_start = t;
    lk.unlock();
    if (j.kind == 0)
      run_encode_job(s, w, j);
    else
      run_decode_job(s, w, j);
    lk.lock();
    s->cv.notify_all();
  }
}

}  // namespace

int mfa_server_create(int device, int32_t workers, int64_t mem_budget, int32_t max_batch, mfa_server** out) {
  if (!out || workers < 1 || workers > 64 || mem_budget <= 0) return MFA_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return MFA_ERR_ARG;
  }
  cudaSetDevice(device);
  mfa_server* s = new (std::nothrow) mfa_server();
  if (!s) return MFA_ERR_OOM;
  s->device = device;
  s->budget = mem_budget;
  s->max_batch = max_batch > 0 ? max_batch : 64;
  s->t0 = Clock::now();
  s->to_free.resize(workers);
  for (int w = 0; w < workers; ++w) {
    cudaStream_t st = nullptr;
    mfa_handle* h = nullptr;
    int rc = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
    if (rc == MFA_OK) rc = mfa_create(device, st, &h);
    if (rc != MFA_OK) {
      if (st) cudaStreamDestroy(st);
      mfa_server_destroy(s);
      return rc;
    }
    s->streams.push_back(st);
    s->handles.push_back(h);
  }
  if (cudaStreamCreateWithFlags(&s->ctl_stream, cudaStreamNonBlocking) != cudaSuccess ||
      mfa_create(device, s->ctl_stream, &s->ctl) != MFA_OK) {
    mfa_server_destroy(s);
    return MFA_ERR_CUDA;
  }
  for (int w = 0; w < workers; ++w) s->workers.emplace_back(worker_loop, s, w);
  *out = s;
  return MFA_OK;
}

int64_t mfa_server_encode(mfa_server* s, const mfa_instance* inst, const void* host_q, int precision) {
  if (!s || !inst || !host_q) return MFA_ERR_ARG;
  if (precision != MFA_PREC_FP64 && precision != MFA_PREC_MIXED && precision != MFA_PREC_FP32) return MFA_ERR_ARG;
  if (inst->dim < 1 || inst->dim > MFA_MAX_DIM || inst->degree < 1 || inst->degree > MFA_MAX_DEGREE) return MFA_ERR_ARG;
  auto r = std::make_unique<Req>();
  r->kind = 0;
  r->inst = *inst;
  r->inst.q_offset = 0;
  long long n = 1;
  for (int a = 0; a < inst->dim; ++a) {
    if (inst->npts[a] < 1 || inst->nspans[a] < 1) return MFA_ERR_ARG;
    n *= inst->npts[a];
  }
  r->q = host_q;
  r->precision = precision;
  r->q_bytes = n * 4;
  encode_bytes(r->inst, r->q_bytes, precision, &r->need, &r->keep);
  std::lock_guard<std::mutex> lk(s->mu);
  if (r->need > s->budget) return MFA_ERR_OOM;
  r->id = s->next_id++;
  r->t_submit = now_s(s);
  Req* p = r.get();
  s->reqs[r->id] = std::move(r);
  s->queue.push_back(p);
  s->cv.notify_all();
  return p->id;
}

int64_t mfa_server_decode(mfa_server* s, int64_t model, int64_t npts, const double* host_pts, double* host_out) {
  if (!s || npts < 0 || (npts > 0 && (!host_pts || !host_out))) return MFA_ERR_ARG;
  auto r = std::make_unique<Req>();
  r->kind = 1;
  r->model = model;
  r->npts = npts;
  r->pts = host_pts;
  r->out = host_out;
  r->need = npts * 32 + 4096;
  std::lock_guard<std::mutex> lk(s->mu);
  if (r->need > s->budget) return MFA_ERR_OOM;
  auto it = s->reqs.find(model);
  const bool known = (it != s->reqs.end() && it->second->kind == 0) || s->models.count(model);
  if (!known) return MFA_ERR_ARG;
  r->id = s->next_id++;
  r->t_submit = now_s(s);
  Req* p = r.get();
  s->reqs[r->id] = std::move(r);
  s->queue.push_back(p);
  s->cv.notify_all();
  return p->id;
}

int mfa_server_wait(mfa_server* s, int64_t id, double timeout_s, mfa_request_info* info) {
  if (!s) return MFA_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return MFA_ERR_ARG;
  Req* r = it->second.get();
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(
                                            timeout_s > 0 ? timeout_s : 1e9));
  while (!r->done) {
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout && !r->done) return MFA_ERR_TIMEOUT;
  }
  if (info) {
    info->status = r->status;
    info->kind = r->kind;
    info->t_submit = r->t_submit;
    info->t_admit = r->t_admit;
    info->t_start = r->t_start;
    info->t_done = r->t_done;
  }
  const int st = r->status;
  // an encode stays known as a model; other finished requests are forgotten
  if (r->kind == 1 || st != MFA_OK) s->reqs.erase(it);
  return st;
}

int mfa_server_release(mfa_server* s, int64_t model) {
  if (!s) return MFA_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->models.find(model);
  if (it == s->models.end() || it->second.released) return MFA_ERR_ARG;
  it->second.released = true;
  std::shared_ptr<BatchRef> br = it->second.batch;
  s->models.erase(it);
  s->reqs.erase(model);
  br->live--;
  release_batch_locked(s, br);
  s->cv.notify_all();
  return MFA_OK;
}

int64_t mfa_server_num_ctrl(mfa_server* s, int64_t model) {
  if (!s) return MFA_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->models.find(model);
  if (it == s->models.end()) return MFA_ERR_ARG;
  return mfa::batch_instance_num_ctrl(it->second.batch->b, it->second.index);
}

int mfa_server_get_ctrl(mfa_server* s, int64_t model, double* host_out, int64_t cap) {
  if (!s || !host_out) return MFA_ERR_ARG;
  std::shared_ptr<BatchRef> br;
  int index = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->models.find(model);
    if (it == s->models.end()) return MFA_ERR_ARG;
    br = it->second.batch;
    index = it->second.index;
    br->readers++;
  }
  int rc;
  {
    std::lock_guard<std::mutex> lc(s->ctl_mu);
    rc = mfa::batch_instance_ctrl(s->ctl, br->b, index, host_out, cap);
  }
  std::lock_guard<std::mutex> lk(s->mu);
  br->readers--;
  release_batch_locked(s, br);
  s->cv.notify_all();
  return rc;
}

int mfa_server_stats(mfa_server* s, mfa_server_stats_t* st) {
  if (!s || !st) return MFA_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  st->budget = s->budget;
  st->reserved = s->used;
  st->peak_reserved = s->peak;
  st->queued = (int64_t)s->queue.size();
  st->resident_models = (int64_t)s->models.size();
  st->encode_jobs = s->jobs_enc;
  st->decode_jobs = s->jobs_dec;
  return MFA_OK;
}

int mfa_server_destroy(mfa_server* s) {
  if (!s) return MFA_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    // release every resident model so its batch is freed by its owner
    for (auto& m : s->models) {
      m.second.released = true;
      m.second.batch->live--;
      release_batch_locked(s, m.second.batch);
    }
    s->models.clear();
    s->cv.notify_all();
  }
  for (auto& t : s->workers) t.join();
  // batches queued for freeing after the workers stopped
  for (size_t w = 0; w < s->to_free.size(); ++w)
    for (auto& br : s->to_free[w])
      if (br->b) mfa_batch_free(br->b);
  for (mfa_handle* h : s->handles) mfa_destroy(h);
  if (s->ctl) mfa_destroy(s->ctl);
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  if (s->ctl_stream) cudaStreamDestroy(s->ctl_stream);
  delete s;
  return MFA_OK;
}
