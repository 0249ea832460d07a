// Serving runtime: continuous batching of cell-batch solve requests into one
// resident persistent kernel per mechanism.
//
// The paper's solver is called once per CFD time step for all cells of a
// domain (Sec. 2.4: a cell leaves the workload when it reaches t_f and the
// freed slot takes the next cell).  Here requests from several concurrent CFD
// steps (independent batches, each with its own t_f) arrive over time.  A
// worker thread owns every CUDA call of the server:
//
//   admission   strict FIFO over submitted requests; a request is admitted
//               when its device bytes fit in the arena (a fixed device
//               allocation of the memory budget, first-fit, nothing is
//               allocated while serving) and its mechanism has a free slot;
//   publication its inputs are copied to the arena, then its slot, then the
//               kernel's pub_seq and published words, all on one copy stream
//               so that the kernel never sees an id before its data;
//   solving     each mechanism's kernel runs on its own stream and share of
//               the SMs, claims ids below `published` as its lanes free up
//               (the same refill as a single solve), and leaves on its own
//               after a bounded idle time; the worker relaunches it when work
//               is waiting and it is not running;
//   completion  the last cell of a request writes the request's slot key
//               to a host-mapped mailbox; the worker then copies the
//               results out on a second copy stream and, when that copy has
//               finished, reports the request and frees its arena range.
//
// Slots are retired in sequence order, which the kernel's slot search relies
// on (see serve_find_slot).  All waits are bounded.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "stev_internal.h"

using stev::BatchDesc;
using stev::ServeCtl;
using stev::ServeSlot;
using stev::host::fail;

namespace {

using Clock = std::chrono::steady_clock;

constexpr long long kIdleNs = 20 * 1000 * 1000;  // a serving kernel leaves after 20 ms idle
constexpr int kDefaultQueue = 1024;

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t request_bytes(long n, int S) {
  return 2 * align256((size_t)n * 8) + align256((size_t)n * S * 8) + align256((size_t)n * 4) +
         align256((size_t)n);
}

// First-fit allocator over the arena [0, size).
class Arena {
 public:
  void init(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
  }
  bool alloc(size_t bytes, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t o = it->first, rest = it->second - bytes;
      free_.erase(it);
      if (rest) free_[o + bytes] = rest;
      *off = o;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<size_t, size_t> free_;  // offset -> bytes
};

enum ReqState { kQueued, kRunning, kCopying, kDone };

struct Request {
  long long id = 0;
  int lane = 0;
  long n = 0;
  double dt = 0;
  const double *T = nullptr, *P = nullptr, *Y = nullptr;
  double *T_out = nullptr, *Y_out = nullptr;
  int* iters = nullptr;
  unsigned char* status = nullptr;
  size_t off = 0, bytes = 0;
  long long seq = -1;
  int slot = -1;
  long long key = -1;  // slot key; the mailbox holds it once the last cell is done
  ReqState state = kQueued;
  double t_submit = 0, t_admit = 0, t_done = 0;
  cudaEvent_t ev = nullptr;  // results copied out
  double *dT = nullptr, *dP = nullptr, *dY = nullptr;
  int* dit = nullptr;
  unsigned char* dst = nullptr;
};

struct Lane {
  stev_mechanism* m = nullptr;
  stev::host::ServeConfig cfg{};
  int grid = 0;
  cudaStream_t ks = nullptr;  // kernel stream
  cudaEvent_t kev = nullptr;  // recorded after each launch
  bool running = false;
  ServeCtl* d_ctl = nullptr;
  ServeSlot* d_slots = nullptr;
  ServeSlot* h_slots = nullptr;     // pinned staging, one per slot
  long long* h_pub = nullptr;       // pinned staging [q][2]: pub_seq, published
  long long* h_mail = nullptr;      // host-mapped mailbox [q] + error word
  long long* d_mail = nullptr;      // its device address
  int* h_stop = nullptr;            // pinned staging of ctl.stop
  long long next_seq = 0, retire_seq = 0;
  unsigned long long next_off = 0;
  std::vector<Request*> slot_req;
  long long launches = 0;
};

}  // namespace

struct stev_server {
  int device = 0;
  int q = kDefaultQueue;
  std::vector<Lane> lanes;
  unsigned char* d_arena = nullptr;
  size_t budget = 0;
  Arena arena;
  size_t resident = 0, peak = 0;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  Clock::time_point t0;
  std::thread worker;
  std::vector<cudaEvent_t> ev_pool;
  // worker-owned
  std::deque<Request*> pending;
  std::vector<Request*> inflight;
  // shared, under mu
  std::mutex mu;
  std::mutex join_mu;  // one joiner of the worker at a time
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> incoming;
  std::deque<stev_request_info> done;
  bool quit = false, stopped = false;
  double stop_timeout = 30.0;
  stev_status err = STEV_OK;
  std::string err_msg;
  long long next_id = 0;
  std::vector<unsigned long long> lane_cells;  // cells submitted per mechanism
  stev_server_stats stats{};
};

namespace {

double now_s(const stev_server* s) {
  return std::chrono::duration<double>(Clock::now() - s->t0).count();
}

// CUDA_TRY for the worker: records the failure in the thread's last error.
#define SRV_TRY(expr)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(e_ == cudaErrorMemoryAllocation ? STEV_ENOMEM : STEV_ECUDA,           \
                  "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

void report(stev_server* s, Request* r, int status, long cells_done) {
  stev_request_info info{};
  info.id = r->id;
  info.mechanism = r->lane;
  info.status = status;
  info.n_cells = r->n;
  info.cells_done = cells_done;
  info.t_submit = r->t_submit;
  info.t_admit = r->t_admit;
  info.t_done = r->t_done;
  std::lock_guard<std::mutex> lk(s->mu);
  s->done.push_back(info);
  if (status == STEV_OK) s->stats.completed++;
  else s->stats.cancelled++;
  s->stats.cells_completed += cells_done;
  s->cv_done.notify_all();
}

stev_status get_event(stev_server* s, cudaEvent_t* ev) {
  if (!s->ev_pool.empty()) {
    *ev = s->ev_pool.back();
    s->ev_pool.pop_back();
    return STEV_OK;
  }
  SRV_TRY(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
  return STEV_OK;
}

stev_status admit(stev_server* s, Request* r, size_t off) {
  Lane& ln = s->lanes[r->lane];
  const int S = ln.cfg.S;
  const size_t n = (size_t)r->n;
  unsigned char* base = s->d_arena + off;
  r->off = off;
  r->dT = reinterpret_cast<double*>(base);
  r->dP = reinterpret_cast<double*>(base + align256(n * 8));
  r->dY = reinterpret_cast<double*>(base + 2 * align256(n * 8));
  r->dit = reinterpret_cast<int*>(base + 2 * align256(n * 8) + align256(n * S * 8));
  r->dst = base + 2 * align256(n * 8) + align256(n * S * 8) + align256(n * 4);
  SRV_TRY(cudaMemcpyAsync(r->dT, r->T, n * 8, cudaMemcpyHostToDevice, s->h2d));
  SRV_TRY(cudaMemcpyAsync(r->dP, r->P, n * 8, cudaMemcpyHostToDevice, s->h2d));
  SRV_TRY(cudaMemcpyAsync(r->dY, r->Y, n * S * 8, cudaMemcpyHostToDevice, s->h2d));
  r->seq = ln.next_seq++;
  r->slot = (int)(r->seq % s->q);
  ServeSlot& hs = ln.h_slots[r->slot];
  hs.d = BatchDesc{r->dT, r->dP, r->dY, r->dT, r->dY, r->dit, r->dst, r->dt, (long long)n};
  hs.key = (ln.next_off << stev::kServeSeqBits) | ((unsigned long long)r->seq & stev::kServeSeqMask);
  hs.done = 0;
  r->key = (long long)hs.key;
  ln.next_off += n;
  long long* pub = ln.h_pub + 2 * r->slot;
  pub[0] = r->seq;
  pub[1] = (long long)ln.next_off;
  // slot, then pub_seq, then published: in stream order
  SRV_TRY(cudaMemcpyAsync(ln.d_slots + r->slot, &hs, sizeof(ServeSlot), cudaMemcpyHostToDevice, s->h2d));
  SRV_TRY(cudaMemcpyAsync(&ln.d_ctl->pub_seq, pub, 8, cudaMemcpyHostToDevice, s->h2d));
  SRV_TRY(cudaMemcpyAsync(&ln.d_ctl->published, pub + 1, 8, cudaMemcpyHostToDevice, s->h2d));
  ln.slot_req[r->slot] = r;
  r->state = kRunning;
  r->t_admit = now_s(s);
  s->inflight.push_back(r);
  s->resident += r->bytes;
  s->peak = std::max(s->peak, s->resident);
  std::lock_guard<std::mutex> lk(s->mu);
  s->stats.admitted++;
  s->stats.resident_bytes = s->resident;
  s->stats.peak_resident_bytes = s->peak;
  return STEV_OK;
}

stev_status launch_lane(stev_server* s, Lane& ln) {
  stev_status st = stev::host::serve_launch(ln.m, ln.d_ctl, ln.d_slots, ln.d_mail, s->q, kIdleNs,
                                            ln.grid, ln.ks);
  if (st != STEV_OK) return st;
  SRV_TRY(cudaEventRecord(ln.kev, ln.ks));
  ln.running = true;
  ln.launches++;
  std::lock_guard<std::mutex> lk(s->mu);
  s->stats.kernel_launches++;
  return STEV_OK;
}

stev_status copy_out(stev_server* s, Request* r) {
  const int S = s->lanes[r->lane].cfg.S;
  const size_t n = (size_t)r->n;
  SRV_TRY(cudaMemcpyAsync(r->T_out, r->dT, n * 8, cudaMemcpyDeviceToHost, s->d2h));
  SRV_TRY(cudaMemcpyAsync(r->Y_out, r->dY, n * S * 8, cudaMemcpyDeviceToHost, s->d2h));
  SRV_TRY(cudaMemcpyAsync(r->iters, r->dit, n * 4, cudaMemcpyDeviceToHost, s->d2h));
  SRV_TRY(cudaMemcpyAsync(r->status, r->dst, n, cudaMemcpyDeviceToHost, s->d2h));
  stev_status st = get_event(s, &r->ev);
  if (st != STEV_OK) return st;
  SRV_TRY(cudaEventRecord(r->ev, s->d2h));
  r->state = kCopying;
  return STEV_OK;
}

void retire(stev_server* s) {
  for (Lane& ln : s->lanes) {
    while (ln.retire_seq < ln.next_seq) {
      const int slot = (int)(ln.retire_seq % s->q);
      Request* x = ln.slot_req[slot];
      if (x && x->state != kDone) break;
      if (x) {
        if (x->ev) s->ev_pool.push_back(x->ev);
        delete x;
        ln.slot_req[slot] = nullptr;
      }
      ln.retire_seq++;
    }
  }
}

// One pass of the worker; *busy tells whether work is in flight.
stev_status progress(stev_server* s, bool* busy) {
  // admission, strict FIFO
  while (!s->pending.empty()) {
    Request* r = s->pending.front();
    if (r->n == 0) {
      s->pending.pop_front();
      r->t_admit = r->t_done = now_s(s);
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stats.admitted++;
      }
      report(s, r, STEV_OK, 0);
      delete r;
      continue;
    }
    Lane& ln = s->lanes[r->lane];
    if (ln.next_seq - ln.retire_seq >= s->q) break;
    size_t off = 0;
    if (!s->arena.alloc(r->bytes, &off)) break;
    s->pending.pop_front();
    stev_status st = admit(s, r, off);
    if (st != STEV_OK) return st;
  }
  // kernels: note exits, relaunch where work waits
  for (Lane& ln : s->lanes) {
    if (((volatile long long*)ln.h_mail)[s->q] != -1)
      return fail(STEV_ECUDA, "serving kernel dropped a cell whose slot lookup fell outside its request");
    if (ln.running) {
      const cudaError_t e = cudaEventQuery(ln.kev);
      if (e == cudaSuccess) ln.running = false;
      else if (e != cudaErrorNotReady) SRV_TRY(e);
    }
  }
  for (Request* r : s->inflight) {
    if (r->state != kRunning) continue;
    Lane& ln = s->lanes[r->lane];
    if (!ln.running) {
      stev_status st = launch_lane(s, ln);
      if (st != STEV_OK) return st;
    }
  }
  // completions
  for (Request* r : s->inflight) {
    if (r->state != kRunning) continue;
    const volatile long long* mail = s->lanes[r->lane].h_mail;
    if (mail[r->slot] == r->key) {
      stev_status st = copy_out(s, r);
      if (st != STEV_OK) return st;
    }
  }
  std::vector<Request*> keep;
  keep.reserve(s->inflight.size());
  for (Request* r : s->inflight) {
    if (r->state == kCopying) {
      const cudaError_t e = cudaEventQuery(r->ev);
      if (e == cudaSuccess) {
        r->state = kDone;
        r->t_done = now_s(s);
        s->arena.release(r->off, r->bytes);
        s->resident -= r->bytes;
        {
          std::lock_guard<std::mutex> lk(s->mu);
          s->stats.resident_bytes = s->resident;
        }
        report(s, r, STEV_OK, r->n);
        continue;
      }
      if (e != cudaErrorNotReady) SRV_TRY(e);
    }
    keep.push_back(r);
  }
  s->inflight.swap(keep);
  retire(s);
  *busy = !s->inflight.empty() || !s->pending.empty();
  return STEV_OK;
}

// Stops the kernels (they finish the cells they hold, claim nothing new and
// leave), reports finished requests and cancels the rest.  Bounded by
// s->stop_timeout; returns STEV_ETIMEOUT if a kernel did not leave in time.
stev_status shutdown(stev_server* s) {
  stev_status first = STEV_OK;
  for (Lane& ln : s->lanes) {
    *ln.h_stop = 1;
    const cudaError_t e = cudaMemcpyAsync(&ln.d_ctl->stop, ln.h_stop, 4, cudaMemcpyHostToDevice, s->h2d);
    if (e != cudaSuccess && first == STEV_OK)
      first = fail(STEV_ECUDA, "stopping a serving kernel: %s", cudaGetErrorString(e));
  }
  const auto deadline = Clock::now() + std::chrono::duration<double>(s->stop_timeout);
  bool left = false;
  while (!left) {
    left = true;
    for (Lane& ln : s->lanes) {
      if (!ln.running) continue;
      const cudaError_t e = cudaEventQuery(ln.kev);
      if (e == cudaErrorNotReady) left = false;
      else ln.running = false;
    }
    if (left) break;
    if (Clock::now() > deadline) {
      return fail(STEV_ETIMEOUT, "serving kernels did not stop within %.1f s", s->stop_timeout);
    }
    std::this_thread::sleep_for(std::chrono::milliseconds(1));
  }
  // finished requests still get their results; the rest are cancelled
  for (Request* r : s->inflight) {
    if (r->state == kRunning && ((volatile long long*)s->lanes[r->lane].h_mail)[r->slot] == r->key) {
      stev_status st = copy_out(s, r);
      if (st != STEV_OK && first == STEV_OK) first = st;
    }
  }
  if (cudaStreamSynchronize(s->d2h) != cudaSuccess && first == STEV_OK)
    first = fail(STEV_ECUDA, "copying results out at shutdown");
  for (Request* r : s->inflight) {
    r->t_done = now_s(s);
    if (r->state == kCopying) {
      report(s, r, STEV_OK, r->n);
    } else {
      unsigned long long done = 0;  // the kernels have left: the count is final
      if (cudaMemcpy(&done, &s->lanes[r->lane].d_slots[r->slot].done, sizeof done,
                     cudaMemcpyDeviceToHost) != cudaSuccess && first == STEV_OK)
        first = fail(STEV_ECUDA, "reading a cancelled request's progress");
      report(s, r, STEV_EINCOMPLETE, (long)std::min<unsigned long long>(done, (unsigned long long)r->n));
    }
    r->state = kDone;
  }
  s->inflight.clear();
  for (Request* r : s->pending) {
    r->t_done = now_s(s);
    report(s, r, STEV_EINCOMPLETE, 0);
    delete r;
  }
  s->pending.clear();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (Request* r : s->incoming) {
      stev_request_info info{};
      info.id = r->id;
      info.mechanism = r->lane;
      info.status = STEV_EINCOMPLETE;
      info.n_cells = r->n;
      info.t_submit = r->t_submit;
      s->done.push_back(info);
      s->stats.cancelled++;
      delete r;
    }
    s->incoming.clear();
  }
  retire(s);
  return first;
}

void worker_main(stev_server* s) {
  cudaSetDevice(s->device);
  stev_status st = STEV_OK;
  bool busy = false;
  while (true) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (!s->quit && s->incoming.empty())
        s->cv_work.wait_for(lk, busy ? std::chrono::microseconds(20) : std::chrono::microseconds(1000));
      while (!s->incoming.empty()) {
        s->pending.push_back(s->incoming.front());
        s->incoming.pop_front();
      }
      if (s->quit) break;
    }
    st = progress(s, &busy);
    if (st != STEV_OK) break;
  }
  std::string msg = st != STEV_OK ? std::string(stev_last_error()) : std::string();
  stev_status st2 = shutdown(s);
  std::lock_guard<std::mutex> lk(s->mu);
  if (st != STEV_OK && s->err == STEV_OK) {
    s->err = st;
    s->err_msg = msg;
  }
  if (st2 != STEV_OK && s->err == STEV_OK) {
    s->err = st2;
    s->err_msg = stev_last_error();
  }
  s->stopped = true;
  s->cv_done.notify_all();
}

void free_server(stev_server* s, bool device_ok) {
  for (Lane& ln : s->lanes) {
    for (Request*& r : ln.slot_req) {
      delete r;
      r = nullptr;
    }
    if (device_ok) {
      if (ln.d_ctl) cudaFree(ln.d_ctl);
      if (ln.d_slots) cudaFree(ln.d_slots);
      if (ln.h_mail) cudaFreeHost(ln.h_mail);
    }
    if (ln.h_slots) cudaFreeHost(ln.h_slots);
    if (ln.h_pub) cudaFreeHost(ln.h_pub);
    if (ln.h_stop) cudaFreeHost(ln.h_stop);
    if (ln.ks) cudaStreamDestroy(ln.ks);
    if (ln.kev) cudaEventDestroy(ln.kev);
  }
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  if (device_ok && s->d_arena) cudaFree(s->d_arena);
  if (s->h2d) cudaStreamDestroy(s->h2d);
  if (s->d2h) cudaStreamDestroy(s->d2h);
  delete s;
}

#define CREATE_TRY(expr)                                                              \
  do {                                                                                \
    cudaError_t e_ = (expr);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      free_server(s, true);                                                           \
      return fail(e_ == cudaErrorMemoryAllocation ? STEV_ENOMEM : STEV_ECUDA,         \
                  "%s: %s", #expr, cudaGetErrorString(e_));                           \
    }                                                                                 \
  } while (0)

}  // namespace

extern "C" stev_status stev_server_create(stev_mechanism* const* mechs, int n_mechs,
                                          const int* sm_share, size_t mem_budget,
                                          int queue_len, stev_server** out) {
  stev::host::clear_error();
  if (!out) return fail(STEV_EINVAL, "out is NULL");
  *out = nullptr;
  if (!mechs || n_mechs < 1) return fail(STEV_EINVAL, "need at least one mechanism");
  if (queue_len < 0 || queue_len > (1 << 20)) return fail(STEV_EINVAL, "queue_len must be in [0, 2^20]");
  if (mem_budget == 0) return fail(STEV_EINVAL, "mem_budget is 0");
  std::vector<stev::host::ServeConfig> cfg(n_mechs);
  for (int i = 0; i < n_mechs; ++i) {
    stev_status st = stev::host::serve_config(mechs[i], &cfg[i]);
    if (st != STEV_OK) return st;
    if (cfg[i].device != cfg[0].device) return fail(STEV_EINVAL, "mechanisms live on different devices");
  }
  const int sms = cfg[0].sms;
  std::vector<int> share(n_mechs);
  int total = 0;
  for (int i = 0; i < n_mechs; ++i) {
    share[i] = sm_share ? sm_share[i] : sms / n_mechs;
    if (share[i] < 1) return fail(STEV_EINVAL, "sm_share[%d] must be >= 1", i);
    total += share[i];
  }
  if (total > sms) return fail(STEV_EINVAL, "sm_share adds up to %d SMs; the device has %d", total, sms);
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != cfg[0].device)
    return fail(STEV_EINVAL, "mechanisms live on device %d, current is %d", cfg[0].device, dev);

  stev_server* s = new stev_server();
  s->device = cfg[0].device;
  s->q = queue_len ? queue_len : kDefaultQueue;
  s->budget = mem_budget;
  s->t0 = Clock::now();
  s->lanes.resize(n_mechs);
  s->lane_cells.assign(n_mechs, 0);
  CREATE_TRY(cudaMalloc(&s->d_arena, mem_budget));
  s->arena.init(mem_budget);
  CREATE_TRY(cudaStreamCreateWithFlags(&s->h2d, cudaStreamNonBlocking));
  CREATE_TRY(cudaStreamCreateWithFlags(&s->d2h, cudaStreamNonBlocking));
  for (int i = 0; i < n_mechs; ++i) {
    Lane& ln = s->lanes[i];
    ln.m = mechs[i];
    ln.cfg = cfg[i];
    // one CTA per SM of the share: the partition between mechanisms is exact
    ln.grid = share[i];
    ln.slot_req.assign(s->q, nullptr);
    CREATE_TRY(cudaStreamCreateWithFlags(&ln.ks, cudaStreamNonBlocking));
    CREATE_TRY(cudaEventCreateWithFlags(&ln.kev, cudaEventDisableTiming));
    CREATE_TRY(cudaMalloc(&ln.d_ctl, sizeof(ServeCtl)));
    CREATE_TRY(cudaMemset(ln.d_ctl, 0, sizeof(ServeCtl)));
    CREATE_TRY(cudaMalloc(&ln.d_slots, sizeof(ServeSlot) * s->q));
    CREATE_TRY(cudaMemset(ln.d_slots, 0xff, sizeof(ServeSlot) * s->q));  // key = all ones: no request
    CREATE_TRY(cudaHostAlloc(&ln.h_slots, sizeof(ServeSlot) * s->q, cudaHostAllocDefault));
    CREATE_TRY(cudaHostAlloc(&ln.h_pub, 16 * (size_t)s->q, cudaHostAllocDefault));
    CREATE_TRY(cudaHostAlloc(&ln.h_stop, sizeof(int), cudaHostAllocDefault));
    CREATE_TRY(cudaHostAlloc(&ln.h_mail, 8 * ((size_t)s->q + 1), cudaHostAllocMapped));
    for (int k = 0; k <= s->q; ++k) ln.h_mail[k] = -1;
    CREATE_TRY(cudaHostGetDevicePointer((void**)&ln.d_mail, ln.h_mail, 0));
  }
  s->stats.budget_bytes = mem_budget;
  CREATE_TRY(cudaDeviceSynchronize());
  s->worker = std::thread(worker_main, s);
  *out = s;
  return STEV_OK;
}

extern "C" stev_status stev_server_submit(stev_server* s, int mech, long n, double dt,
                                          const double* T, const double* P, const double* Y,
                                          double* T_out, double* Y_out, int* iters,
                                          unsigned char* cell_status, long long* request_id) {
  stev::host::clear_error();
  if (!s) return fail(STEV_EINVAL, "server is NULL");
  if (mech < 0 || mech >= (int)s->lanes.size()) return fail(STEV_EINVAL, "mechanism index %d out of range", mech);
  if (n < 0) return fail(STEV_EINVAL, "n_cells < 0");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(STEV_EINVAL, "dt_cfd must be finite and > 0");
  if (n > 0 && (!T || !P || !Y || !T_out || !Y_out || !iters || !cell_status))
    return fail(STEV_EINVAL, "NULL array");
  const size_t bytes = request_bytes(n, s->lanes[mech].cfg.S);
  if (bytes > s->budget)
    return fail(STEV_EINVAL, "request needs %zu device bytes; the budget is %zu", bytes, s->budget);
  Request* r = new Request();
  r->lane = mech;
  r->n = n;
  r->dt = dt;
  r->T = T; r->P = P; r->Y = Y;
  r->T_out = T_out; r->Y_out = Y_out; r->iters = iters; r->status = cell_status;
  r->bytes = bytes;
  r->t_submit = now_s(s);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->err != STEV_OK) {
    delete r;
    return fail(s->err, "server failed: %s", s->err_msg.c_str());
  }
  if (s->quit || s->stopped) {
    delete r;
    return fail(STEV_EINVAL, "server is stopped");
  }
  if (s->lane_cells[mech] + (unsigned long long)n >= stev::kServeMaxIds) {
    delete r;
    return fail(STEV_EINVAL, "this server has used up its cell id space; create a new one");
  }
  s->lane_cells[mech] += (unsigned long long)n;
  r->id = s->next_id++;
  if (request_id) *request_id = r->id;
  s->incoming.push_back(r);
  s->stats.submitted++;
  s->cv_work.notify_one();
  return STEV_OK;
}

extern "C" stev_status stev_server_poll(stev_server* s, stev_request_info* out, int max_out,
                                        int* n_out, double timeout_s) {
  stev::host::clear_error();
  if (!s || !n_out || (max_out > 0 && !out)) return fail(STEV_EINVAL, "NULL argument");
  *n_out = 0;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && timeout_s > 0 && !s->stopped) {
    s->cv_done.wait_for(lk, std::chrono::duration<double>(std::min(timeout_s, 3600.0)),
                        [s] { return !s->done.empty() || s->stopped; });
  }
  int k = 0;
  while (k < max_out && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  *n_out = k;
  if (s->err != STEV_OK) return fail(s->err, "server failed: %s", s->err_msg.c_str());
  return STEV_OK;
}

extern "C" stev_status stev_server_get_stats(stev_server* s, stev_server_stats* out) {
  stev::host::clear_error();
  if (!s || !out) return fail(STEV_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  return STEV_OK;
}

extern "C" double stev_server_clock(const stev_server* s) { return s ? now_s(s) : 0.0; }

extern "C" stev_status stev_server_stop(stev_server* s, double timeout_s) {
  stev::host::clear_error();
  if (!s) return fail(STEV_EINVAL, "server is NULL");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->quit) s->stop_timeout = timeout_s > 0 ? std::min(timeout_s, 3600.0) : 30.0;
    s->quit = true;
    s->cv_work.notify_all();
  }
  {
    std::lock_guard<std::mutex> lk(s->join_mu);
    if (s->worker.joinable()) s->worker.join();
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->err != STEV_OK) return fail(s->err, "%s", s->err_msg.c_str());
  return STEV_OK;
}

extern "C" stev_status stev_server_destroy(stev_server* s, double timeout_s) {
  stev::host::clear_error();
  if (!s) return STEV_OK;
  stev_server_stop(s, timeout_s);
  stev_status st;
  std::string msg;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    st = s->err;
    msg = s->err_msg;
  }
  // a kernel that did not stop may still use the device buffers: keep them
  const bool device_ok = st != STEV_ETIMEOUT;
  free_server(s, device_ok);
  if (st != STEV_OK) return fail(st, "%s", msg.c_str());
  return STEV_OK;
}
