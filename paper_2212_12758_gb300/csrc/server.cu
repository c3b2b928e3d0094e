// Serving runtime of libfab: continuous admission of f(A)b requests onto a set
// of worker slots. Each slot is a host thread with its own CUDA stream and its
// own grow-only device workspace (a clone that points at the request's matrix),
// so solves of different sizes, matrices and functions run concurrently on the
// device and their bases and sketches stay resident between requests. A request
// leaves the queue (in order) as soon as a slot is free and its workspace fits
// both the server's device-memory budget and the memory the device reports free;
// a blocked slot first releases its own cached workspace. Latency is measured
// from submission to completion.
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "handle.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  fab_handle* h = nullptr;
  fab_params p{};
  std::vector<double> b, x;
  size_t need = 0;  // estimated workspace bytes
  int rc = FAB_OK;
  char err[256] = "";  // fab_last_error() of the slot thread when rc == FAB_ECUDA
  fab_stats st{};
  Clock::time_point t_submit, t_done;
  bool done = false;
};

struct Slot {
  std::thread th;
  cudaStream_t stream = nullptr;
  fab_handle* ws = nullptr;  // workspace clone (null until first use)
  size_t held = 0;           // device bytes held by ws
  bool busy = false;
  double* pin = nullptr;     // pinned staging of b and x (grow-only, 2 pin_n doubles)
  size_t pin_n = 0;
};

}  // namespace

struct fab_server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> reqs;
  std::vector<Slot> slots;
  size_t budget = 0;
  uint64_t next_id = 1;
  int device = 0;
  bool stop = false;
  int64_t submitted = 0, completed = 0;
};

namespace {

constexpr size_t kFreeMargin = (size_t)256 << 20;  // device memory kept free beyond a request's need

size_t held_by_others(const fab_server* s, int self) {
  size_t t = 0;
  for (int i = 0; i < (int)s->slots.size(); ++i)
    if (i != self) t += s->slots[i].held;
  return t;
}

// Would the head request fit if slot `self` took it (reusing its workspace)?
bool admissible(const fab_server* s, int self, const Request* r) {
  const Slot& sl = s->slots[self];
  const size_t after = sl.held > r->need ? sl.held : r->need;
  if (held_by_others(s, self) + after > s->budget) return false;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const size_t grow = after - sl.held;
  return grow + kFreeMargin <= free_b;
}

void worker(fab_server* s, int self) {
  cudaSetDevice(s->device);
  fab::use_blocking_waits(true);
  struct Release {
    ~Release() { fab::use_blocking_waits(false); }
  } release;
  Slot& sl = s->slots[self];
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stop) return;
        if (!s->queue.empty()) {
          Request* head = s->queue.front();
          if (admissible(s, self, head)) {
            r = head;
            s->queue.pop_front();
            sl.busy = true;
            // reserve the workspace now: other slots' admission must see it
            // while this solve grows it
            if (sl.held < r->need) sl.held = r->need;
            break;
          }
          if (sl.held > 0) {  // blocked: give back this slot's cached workspace and retry
            fab_destroy(sl.ws);
            sl.ws = nullptr;
            sl.held = 0;
            continue;
          }
        }
        s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
      }
    }
    // solve outside the lock on this slot's stream and workspace; a host allocation
    // that fails here is the request's error, not the worker's end
    try {
      if (!sl.ws) sl.ws = fab::clone_for_workspace(r->h);
      else fab::point_to_matrix(sl.ws, r->h);
      fab_params p = r->p;
      p.stream = sl.stream;
      const size_t n = r->b.size();
      r->x.assign(n, 0.0);
      if (sl.pin_n < n) {  // pinned staging: the copies run asynchronously on the slot's stream
        if (sl.pin) cudaFreeHost(sl.pin);
        sl.pin = nullptr;
        sl.pin_n = 0;
        if (cudaHostAlloc(&sl.pin, 2 * n * sizeof(double), cudaHostAllocDefault) == cudaSuccess) sl.pin_n = n;
        else cudaGetLastError();
      }
      if (sl.pin) {
        memcpy(sl.pin, r->b.data(), n * sizeof(double));
        r->rc = fab_apply(sl.ws, &p, sl.pin, sl.pin + n, 0, &r->st);
        memcpy(r->x.data(), sl.pin + n, n * sizeof(double));
      } else {
        r->rc = fab_apply(sl.ws, &p, r->b.data(), r->x.data(), 0, &r->st);
      }
      if (r->rc == FAB_ECUDA) snprintf(r->err, sizeof(r->err), "%s", fab_last_error());
    } catch (...) {
      r->rc = fab::abi_error_code();
      r->x.clear();
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      sl.held = sl.ws ? fab::handle_ws_bytes(sl.ws) : 0;
      sl.busy = false;
      r->t_done = Clock::now();
      r->done = true;
      s->completed += 1;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace

extern "C" int fab_server_create(fab_server** out, size_t hbm_budget_bytes, int slots) try {
  if (!out || slots < 1 || slots > 64) return FAB_EINVAL;
  *out = nullptr;
  fab_server* s = new fab_server();
  // Releases whatever was set up (streams, workers already started) on every early
  // return and on an exception (a thread that cannot start, a host allocation).
  struct Owner {
    fab_server* s;
    ~Owner() {
      if (s) fab_server_destroy(s);
    }
  } owner{s};
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    cudaGetLastError();
    return FAB_ECUDA;
  }
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return FAB_ECUDA;
  }
  s->budget = hbm_budget_bytes ? hbm_budget_bytes : (free_b / 10) * 9;
  s->slots.resize(slots);
  for (int i = 0; i < slots; ++i) {
    if (cudaStreamCreateWithFlags(&s->slots[i].stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      s->slots[i].stream = nullptr;
      return FAB_ECUDA;
    }
  }
  for (int i = 0; i < slots; ++i) s->slots[i].th = std::thread(worker, s, i);
  owner.s = nullptr;
  *out = s;
  return FAB_OK;
} catch (...) {
  return fab::abi_error_code();
}

extern "C" int fab_server_submit(fab_server* s, fab_handle* h, const fab_params* p, const double* b,
                                 uint64_t* ticket) try {
  if (!s || !h || !p || !b || !ticket || p->f == FAB_F_SIGN) return FAB_EINVAL;
  Request* r = new Request();
  r->h = h;
  r->p = *p;
  r->p.stream = nullptr;
  r->b.assign(b, b + h->n);
  r->need = fab::estimate_ws_bytes(h, p);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop || r->need > s->budget) {
      delete r;
      return s->stop ? FAB_EINVAL : FAB_ENOMEM;
    }
    if (p->precision == FAB_MIXED) {  // the shared FP32 matrix copy is made once, here
      const int rc = fab::ensure_vals32(h, nullptr);
      if (rc != FAB_OK) {
        delete r;
        return rc;
      }
    }
    r->id = s->next_id++;
    r->t_submit = Clock::now();
    s->reqs[r->id] = r;
    s->queue.push_back(r);
    s->submitted += 1;
    *ticket = r->id;
  }
  s->cv_work.notify_all();
  return FAB_OK;
} catch (...) {
  return fab::abi_error_code();
}

extern "C" int fab_server_poll(fab_server* s, uint64_t ticket, double* x, fab_stats* st, double* latency_ms,
                               int timeout_ms) try {
  if (!s) return FAB_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return FAB_EINVAL;
  Request* r = it->second;
  const auto until = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
  while (!r->done) {
    if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout && !r->done) return FAB_ETIMEOUT;
  }
  if (x) memcpy(x, r->x.data(), r->x.size() * sizeof(double));
  if (st) *st = r->st;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  const int rc = r->rc;
  if (rc == FAB_ECUDA) fab::set_last_error(r->err);
  s->reqs.erase(it);
  delete r;
  return rc;
} catch (...) {
  return fab::abi_error_code();
}

extern "C" int fab_server_stats_get(fab_server* s, fab_server_stats* out) try {
  if (!s || !out) return FAB_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->queued = (int64_t)s->queue.size();
  for (const Slot& sl : s->slots) {
    out->in_flight += sl.busy ? 1 : 0;
    out->bytes_in_use += (double)sl.held;
  }
  out->bytes_budget = (double)s->budget;
  return FAB_OK;
} catch (...) {
  return fab::abi_error_code();
}

extern "C" void fab_server_destroy(fab_server* s) try {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (Slot& sl : s->slots)
    if (sl.th.joinable()) sl.th.join();  // a slot finishes the solve it is running, then exits
  for (Slot& sl : s->slots) {
    if (sl.ws) fab_destroy(sl.ws);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.pin) cudaFreeHost(sl.pin);
  }
  for (auto& kv : s->reqs) delete kv.second;
  cudaGetLastError();
  delete s;
} catch (...) {
}
