// Request server (include/helm.h, "request server"): continuous batching of
// independent Helmholtz solves on one GPU.
//
// Threads:
//   submit (caller)  -> pending FIFO -> admission (memory budget, slot count)
//   setup thread     : stream + helm_setup + load vector upload + solve start
//   stepping thread  : advances every active solve without blocking
//   finish thread    : solution download, handle destruction, budget release
// Admission runs under the server mutex whenever a request arrives or one
// finishes, so requests that arrive while others are on the GPU enter as soon
// as memory and a slot are free.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "runtime.h"

using namespace helm;

namespace {

struct Req {
  int64_t ticket = 0;
  helm_request r{};
  std::vector<double2> F;   // host copy of the load vector
  void* x_host = nullptr;
  int64_t N = 0;
  helm_ticket_info info{};
  bool done = false;
  cudaStream_t stream = nullptr;
  helm_t h = nullptr;
  double2* Fd = nullptr;
  double2* xd = nullptr;
  Task* task = nullptr;
};

int64_t num_dofs(const helm_request& r) {
  const int n = (int)std::lround(1.0 / r.h);
  int64_t side = (int64_t)r.order * n + 1, N = 1;
  for (int d = 0; d < r.opts.dim; ++d) N *= side;
  return N;
}

}  // namespace

struct helm_server {
  size_t budget = 0;
  int max_active = 1;
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;        // wakes the worker threads
  std::condition_variable cv_done;   // wakes waiters
  std::deque<Req*> pending, to_setup, to_finish;
  std::vector<Req*> incoming;        // set up, waiting to be picked up by the stepper
  std::unordered_map<int64_t, Req*> all;
  size_t reserved = 0;
  int inflight = 0;
  int64_t next = 1;
  int64_t unfinished = 0;
  bool stop = false;
  std::thread setup_thr, step_thr, finish_thr;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  // FIFO admission under the lock: the head waits until it fits
  void admit() {
    while (!pending.empty() && inflight < max_active) {
      Req* q = pending.front();
      if (reserved + q->info.bytes > budget) break;
      pending.pop_front();
      reserved += q->info.bytes;
      ++inflight;
      q->info.t_admit = now();
      to_setup.push_back(q);
    }
    cv.notify_all();
  }
  void finish_locked(Req* q) {   // caller holds mu
    q->done = true;
    --unfinished;
    cv_done.notify_all();
  }
  void release(Req* q) {
    std::lock_guard<std::mutex> lk(mu);
    reserved -= q->info.bytes;
    --inflight;
    finish_locked(q);
    admit();
  }

  void setup_loop() {
    cudaSetDevice(device);
    for (;;) {
      Req* q;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return stop || !to_setup.empty(); });
        if (to_setup.empty()) return;
        q = to_setup.front();
        to_setup.pop_front();
      }
      int rc = cudaStreamCreateWithFlags(&q->stream, cudaStreamNonBlocking) == cudaSuccess ? HELM_OK : HELM_ECUDA;
      helm_opts o = q->r.opts;
      o.stream = q->stream;
      if (rc == HELM_OK) rc = helm_setup(q->r.k, q->r.h, q->r.order, q->r.shift, &o, &q->h);
      if (rc == HELM_OK) {
        helm_setup_info(q->h, &q->info.setup_ms, nullptr);
        const size_t bytes = sizeof(double2) * (size_t)q->N;
        if (cudaMallocAsync((void**)&q->Fd, bytes, q->stream) != cudaSuccess ||
            cudaMallocAsync((void**)&q->xd, bytes, q->stream) != cudaSuccess) {
          rc = HELM_ENOMEM;
        } else if (cudaMemcpyAsync(q->Fd, q->F.data(), bytes, cudaMemcpyHostToDevice, q->stream) != cudaSuccess) {
          rc = HELM_ECUDA;
        }
      }
      if (rc == HELM_OK) rc = task_create(q->h, q->Fd, q->xd, &q->task);
      std::lock_guard<std::mutex> lk(mu);
      if (rc != HELM_OK) {
        q->info.rc = rc;
        to_finish.push_back(q);
      } else {
        q->info.t_start = now();
        incoming.push_back(q);
      }
      cv.notify_all();
    }
  }

  void step_loop() {
    cudaSetDevice(device);
    std::vector<Req*> act;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu);
        if (act.empty()) cv.wait(lk, [&] { return stop || !incoming.empty(); });
        if (stop && act.empty() && incoming.empty()) return;
        act.insert(act.end(), incoming.begin(), incoming.end());
        incoming.clear();
      }
      bool progress = false;
      for (size_t i = 0; i < act.size();) {
        Req* q = act[i];
        int rc = HELM_OK;
        if (task_step(q->task, false, &q->info.res, &rc)) {
          q->info.rc = rc;
          act[i] = act.back();
          act.pop_back();
          std::lock_guard<std::mutex> lk(mu);
          to_finish.push_back(q);
          cv.notify_all();
          progress = true;
        } else {
          ++i;
        }
      }
      if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }

  void finish_loop() {
    cudaSetDevice(device);
    for (;;) {
      Req* q;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return stop || !to_finish.empty(); });
        if (to_finish.empty()) return;
        q = to_finish.front();
        to_finish.pop_front();
      }
      if (q->info.rc == HELM_OK && q->x_host && q->xd) {
        if (cudaMemcpyAsync(q->x_host, q->xd, sizeof(double2) * (size_t)q->N, cudaMemcpyDeviceToHost, q->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(q->stream) != cudaSuccess)
          q->info.rc = HELM_ECUDA;
      }
      if (q->task) task_destroy(q->task);
      if (q->Fd) cudaFreeAsync(q->Fd, q->stream);
      if (q->xd) cudaFreeAsync(q->xd, q->stream);
      if (q->h) helm_destroy(q->h);   // synchronises the stream
      if (q->stream) {
        cudaStreamSynchronize(q->stream);
        cudaStreamDestroy(q->stream);
      }
      q->task = nullptr;
      q->Fd = q->xd = nullptr;
      q->h = nullptr;
      q->stream = nullptr;
      q->F.clear();
      q->F.shrink_to_fit();
      q->info.t_done = now();
      release(q);
    }
  }
};

extern "C" {

int helm_request_bytes(const helm_request* r, size_t* bytes) {
  if (!r || !bytes) return HELM_EINVAL;
  if (!(r->h > 0)) return HELM_EINVAL;
  const int n = (int)std::lround(1.0 / r->h);
  if (n < 4 || n % 2 || !(r->order == 1 || r->order == 2) || !(r->opts.dim == 2 || r->opts.dim == 3) ||
      r->opts.restart < 1)
    return HELM_EINVAL;
  *bytes = estimate_bytes(r->opts.dim, r->order, n, r->opts.precision, r->opts.restart) +
           2 * sizeof(double2) * (size_t)num_dofs(*r);   // the server's load and solution vectors
  return HELM_OK;
}

int helm_device_bytes(helm_t h, size_t* bytes) {
  if (!h || !bytes) return HELM_EINVAL;
  *bytes = handle_bytes(h);
  return HELM_OK;
}

int helm_server_create(size_t budget_bytes, int max_active, helm_server_t* out) {
  if (!out || budget_bytes == 0 || max_active < 1) return HELM_EINVAL;
  *out = nullptr;
  helm_server* s = new (std::nothrow) helm_server();
  if (!s) return HELM_ENOMEM;
  s->budget = budget_bytes;
  s->max_active = max_active;
  s->t0 = std::chrono::steady_clock::now();
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return HELM_ECUDA;
  }
  try {
    s->setup_thr = std::thread(&helm_server::setup_loop, s);
    s->step_thr = std::thread(&helm_server::step_loop, s);
    s->finish_thr = std::thread(&helm_server::finish_loop, s);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
      s->cv.notify_all();
    }
    if (s->setup_thr.joinable()) s->setup_thr.join();
    if (s->step_thr.joinable()) s->step_thr.join();
    if (s->finish_thr.joinable()) s->finish_thr.join();
    delete s;
    return HELM_ENOMEM;
  }
  *out = s;
  return HELM_OK;
}

int helm_server_submit(helm_server_t s, const helm_request* r, const void* F_host, void* x_host, int64_t* ticket) {
  if (!s || !r || !F_host || !ticket) return HELM_EINVAL;
  size_t bytes = 0;
  int rc = helm_request_bytes(r, &bytes);
  if (rc) return rc;
  Req* q = new (std::nothrow) Req();
  if (!q) return HELM_ENOMEM;
  q->r = *r;
  q->N = num_dofs(*r);
  q->x_host = x_host;
  q->info.bytes = bytes;
  try {
    q->F.assign((const double2*)F_host, (const double2*)F_host + q->N);
  } catch (...) {
    delete q;
    return HELM_ENOMEM;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  q->ticket = s->next++;
  q->info.t_submit = s->now();
  s->all[q->ticket] = q;
  ++s->unfinished;
  if (bytes > s->budget) {   // can never fit: fail the ticket at once
    q->info.rc = HELM_ENOMEM;
    q->info.t_admit = q->info.t_start = q->info.t_done = q->info.t_submit;
    s->finish_locked(q);
  } else {
    s->pending.push_back(q);
    s->admit();
  }
  *ticket = q->ticket;
  return HELM_OK;
}

int helm_server_poll(helm_server_t s, int64_t ticket, int* done, helm_ticket_info* info) {
  if (!s || !done) return HELM_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return HELM_EINVAL;
  *done = it->second->done ? 1 : 0;
  if (*done && info) *info = it->second->info;
  return HELM_OK;
}

int helm_server_wait(helm_server_t s, int64_t ticket, helm_ticket_info* info) {
  if (!s) return HELM_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return HELM_EINVAL;
  Req* q = it->second;
  s->cv_done.wait(lk, [&] { return q->done; });
  if (info) *info = q->info;
  return HELM_OK;
}

int helm_server_drain(helm_server_t s) {
  if (!s) return HELM_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_done.wait(lk, [&] { return s->unfinished == 0; });
  return HELM_OK;
}

void helm_server_destroy(helm_server_t s) {
  if (!s) return;
  helm_server_drain(s);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  s->setup_thr.join();
  s->step_thr.join();
  s->finish_thr.join();
  for (auto& kv : s->all) delete kv.second;
  delete s;
}

}  // extern "C"
