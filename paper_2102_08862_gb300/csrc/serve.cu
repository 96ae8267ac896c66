// serve.cu -- the serving runtime (tpc_server_*): a request loop that admits time
// frames of differing length by free device memory, keeps the trackers' state
// resident on the GPU, runs several frames at once on separate streams, and
// records per-request timestamps for latency percentiles.
//
// The paper replays recorded time frames through its processing chain from
// memory (Sec. 1); it has no serving interface.  This one is built from the
// library's own entry points:
//  - a slot is a tracker handle (its arena sized for a cluster capacity) with its
//    own CUDA stream and one worker thread, which runs tpc_track_timeframe_host
//    for the requests it is given (copies in, tracks, copies out, synchronises
//    its stream); slots run concurrently, so a frame's copies and kernels overlap
//    with other frames' (continuous batching: a request is admitted as soon as a
//    slot and memory free up, while others are on the GPU);
//  - the scheduler thread admits requests in arrival order (FIFO, no overtaking,
//    so no request starves): a free slot whose capacity fits, else a new slot if
//    the slot count and the memory budget allow it, else a free but too small
//    slot replaced by a larger one if the budget allows, else the request waits
//    (tpc_server_admit holds that policy and is exported for tests); when no slot
//    is busy and the request still cannot be placed, the idle slots too small for
//    it are retired so that their memory can hold a larger one.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/tpcca.h"
#include "tpc_internal.h"

using tpc::report;

extern "C" int tpc_server_admit(uint32_t n, const uint32_t *slot_cap, const uint64_t *slot_bytes,
                                const uint8_t *slot_busy, int n_slots, int max_slots, uint64_t budget,
                                uint64_t new_bytes, int *action) {
  if (!action) return -1;
  *action = TPC_ADMIT_WAIT;
  if (n_slots < 0 || (n_slots > 0 && (!slot_cap || !slot_bytes || !slot_busy))) return -1;
  uint64_t used = 0;
  for (int i = 0; i < n_slots; ++i) used += slot_bytes[i];
  // 1. the free slot of smallest sufficient capacity
  int best = -1;
  for (int i = 0; i < n_slots; ++i)
    if (!slot_busy[i] && slot_cap[i] >= n && (best < 0 || slot_cap[i] < slot_cap[best])) best = i;
  if (best >= 0) {
    *action = TPC_ADMIT_RUN;
    return best;
  }
  // 2. a new slot
  if (n_slots < max_slots && used + new_bytes <= budget) {
    *action = TPC_ADMIT_CREATE;
    return n_slots;
  }
  // 3. replace the largest free slot that is too small
  int rep = -1;
  for (int i = 0; i < n_slots; ++i)
    if (!slot_busy[i] && (rep < 0 || slot_bytes[i] > slot_bytes[rep])) rep = i;
  if (rep >= 0 && used - slot_bytes[rep] + new_bytes <= budget) {
    *action = TPC_ADMIT_REPLACE;
    return rep;
  }
  return -1;
}

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id;
  tpc_clusters cl;   // host arrays (caller owned until the result is returned)
  tpc_tracks out;    // host arrays
  double t_submit = 0, t_start = 0, t_done = 0;
  int slot = -1;
  int status = TPC_OK;
  uint32_t n_tracks = 0;
};

struct Slot {
  tpc_tf *tf = nullptr;
  cudaStream_t stream = nullptr;
  uint32_t cap = 0;
  uint64_t bytes = 0;
  bool busy = false;
  bool retire = false;
  Request *job = nullptr;
  std::thread worker;
  std::condition_variable cv;
};

}  // namespace

struct tpc_server {
  tpc_server_config cfg;
  std::vector<unsigned char> blob;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<Request *> queue;
  std::deque<Request *> done;
  std::vector<Slot *> slots;
  std::thread scheduler;
  bool stop = false;
  uint64_t next_id = 1;
  std::string create_error;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

uint32_t round_capacity(uint32_t n) {
  const uint64_t c = ((uint64_t)n * 5 / 4 + (1u << 20) - 1) & ~(uint64_t)((1u << 20) - 1);  // +25 %, whole Mi
  return (uint32_t)(c > (1u << 30) ? (1u << 30) : c);
}

uint64_t slot_bytes_for(const tpc_server *s, uint32_t cap) {
  tpc_tf_config c = s->cfg.tf;
  c.max_clusters = cap;
  size_t b = 0;
  if (tpc_tf_arena_bytes(&c, &b) != TPC_OK) return ~0ull;
  return b;
}

void worker_loop(tpc_server *s, Slot *sl) {
  cudaSetDevice(s->cfg.device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    sl->cv.wait(lk, [&] { return sl->job != nullptr || sl->retire || s->stop; });
    if (!sl->job) return;  // retired or stopping with nothing to do
    Request *r = sl->job;
    lk.unlock();
    r->t_start = s->now();
    uint32_t nt = 0;
    tpc_tracks out = r->out;
    out.n_tracks_host = &nt;
    out.n_tracks = nullptr;
    const int rc = tpc_track_timeframe_host(sl->tf, &r->cl, &out, sl->stream);
    r->status = rc;
    r->n_tracks = nt;
    r->t_done = s->now();
    lk.lock();
    sl->job = nullptr;
    sl->busy = false;
    s->done.push_back(r);
    s->cv_done.notify_all();
    s->cv_sched.notify_all();
    if (sl->retire || s->stop) return;
  }
}

// create (or re-create) slot k with capacity cap; called by the scheduler with the lock released
int make_slot(tpc_server *s, Slot *sl, uint32_t cap) {
  tpc_tf_config c = s->cfg.tf;
  c.max_clusters = cap;
  c.device = s->cfg.device;
  c.profile_stages = 0;
  tpc_tf *tf = nullptr;
  int rc = tpc_tf_create(&c, &tf);
  if (rc != TPC_OK) return rc;
  if (c.mode == TPC_MODE_PRUNED) {
    rc = tpc_mlp_load(tf, s->blob.data(), s->blob.size());
    if (rc != TPC_OK) {
      tpc_tf_destroy(tf);
      return rc;
    }
  }
  if (!sl->stream && cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess) {
    tpc_tf_destroy(tf);
    return report(TPC_ERR_CUDA, "tpc_server: stream creation failed");
  }
  sl->tf = tf;
  sl->cap = cap;
  sl->bytes = slot_bytes_for(s, cap);
  return TPC_OK;
}

void scheduler_loop(tpc_server *s) {
  cudaSetDevice(s->cfg.device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv_sched.wait(lk, [&] { return s->stop || !s->queue.empty(); });
    if (s->stop) return;
    Request *r = s->queue.front();
    const int ns = (int)s->slots.size();
    std::vector<uint32_t> cap(ns);
    std::vector<uint64_t> bytes(ns);
    std::vector<uint8_t> busy(ns);
    for (int i = 0; i < ns; ++i) {
      cap[i] = s->slots[i]->cap;
      bytes[i] = s->slots[i]->bytes;
      busy[i] = s->slots[i]->busy;
    }
    const uint32_t want = round_capacity(r->cl.n ? r->cl.n : 1);
    const uint64_t new_bytes = slot_bytes_for(s, want);
    int action = TPC_ADMIT_WAIT;
    const int k = tpc_server_admit(r->cl.n, cap.data(), bytes.data(), busy.data(), ns, s->cfg.max_slots,
                                   s->cfg.hbm_budget_bytes, new_bytes, &action);
    if (action == TPC_ADMIT_WAIT) {
      bool fits_later = new_bytes <= s->cfg.hbm_budget_bytes;
      for (int i = 0; i < ns; ++i) fits_later = fits_later || cap[i] >= r->cl.n;
      if (!fits_later) {  // no slot is large enough and none fits the budget: fail the request
        s->queue.pop_front();
        r->status = TPC_ERR_CAPACITY;
        r->t_start = r->t_done = s->now();
        s->done.push_back(r);
        s->cv_done.notify_all();
        continue;
      }
      bool any_busy = false;
      for (int i = 0; i < ns; ++i) any_busy = any_busy || busy[i];
      if (!any_busy) {
        // nothing will free up by itself: retire the idle slots too small for this
        // request (their memory blocks a new slot), then decide again
        std::vector<Slot *> gone;
        for (auto it = s->slots.begin(); it != s->slots.end();) {
          if ((*it)->cap < r->cl.n) {
            (*it)->retire = true;
            (*it)->cv.notify_all();
            gone.push_back(*it);
            it = s->slots.erase(it);
          } else {
            ++it;
          }
        }
        lk.unlock();
        for (auto *sl : gone) {
          if (sl->worker.joinable()) sl->worker.join();
          if (sl->tf) tpc_tf_destroy(sl->tf);
          if (sl->stream) cudaStreamDestroy(sl->stream);
          delete sl;
        }
        lk.lock();
        if (!gone.empty()) continue;
      }
      s->cv_sched.wait(lk);  // a slot frees up, or a new request / stop arrives
      continue;
    }
    s->queue.pop_front();
    Slot *sl = nullptr;
    int rc = TPC_OK;
    if (action == TPC_ADMIT_RUN) {
      sl = s->slots[k];
    } else if (action == TPC_ADMIT_CREATE) {
      sl = new Slot();
      sl->busy = true;  // reserved while it is built
      s->slots.push_back(sl);
      lk.unlock();
      rc = make_slot(s, sl, want);
      lk.lock();
      if (rc == TPC_OK) {
        sl->worker = std::thread(worker_loop, s, sl);
      } else {  // drop the slot again
        s->slots.erase(std::find(s->slots.begin(), s->slots.end(), sl));
        if (sl->stream) cudaStreamDestroy(sl->stream);
        delete sl;
        sl = nullptr;
      }
    } else {  // replace: the old handle is free (no job), destroy and rebuild with the larger capacity
      sl = s->slots[k];
      sl->busy = true;
      tpc_tf *old = sl->tf;
      sl->tf = nullptr;
      sl->bytes = 0;
      lk.unlock();
      tpc_tf_destroy(old);
      rc = make_slot(s, sl, want);
      lk.lock();
    }
    if (rc != TPC_OK) {
      if (sl) {
        sl->busy = false;
        if (!sl->tf) sl->cap = 0;
      }
      r->status = rc;
      r->t_start = r->t_done = s->now();
      s->done.push_back(r);
      s->cv_done.notify_all();
      continue;
    }
    sl->busy = true;
    r->slot = (int)(std::find(s->slots.begin(), s->slots.end(), sl) - s->slots.begin());
    sl->job = r;
    sl->cv.notify_one();
  }
}

}  // namespace

extern "C" void tpc_server_default_config(tpc_server_config *c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->hbm_budget_bytes = 180ull << 30;
  c->max_slots = 4;
  c->device = 0;
  tpc_default_config(&c->tf);
}

extern "C" int tpc_server_create(const tpc_server_config *cfg, tpc_server **out) {
  report(TPC_OK, "");
  if (!cfg || !out) return report(TPC_ERR_ARG, "tpc_server_create: null argument");
  *out = nullptr;
  if (cfg->max_slots < 1 || cfg->max_slots > 64) return report(TPC_ERR_ARG, "tpc_server_create: max_slots in [1, 64]");
  if (cfg->hbm_budget_bytes == 0) return report(TPC_ERR_ARG, "tpc_server_create: zero memory budget");
  if (cfg->tf.mode == TPC_MODE_PRUNED && (!cfg->mlp_blob || cfg->mlp_bytes < tpc_mlp_blob_bytes()))
    return report(TPC_ERR_ARG, "tpc_server_create: TPC_MODE_PRUNED needs the classifier weights");
  tpc_tf_config probe = cfg->tf;
  probe.max_clusters = 1;
  size_t b = 0;
  const int rc = tpc_tf_arena_bytes(&probe, &b);
  if (rc != TPC_OK) return rc;
  tpc_server *s = new tpc_server();
  s->cfg = *cfg;
  if (cfg->mlp_blob)
    s->blob.assign(static_cast<const unsigned char *>(cfg->mlp_blob),
                   static_cast<const unsigned char *>(cfg->mlp_blob) + cfg->mlp_bytes);
  s->t0 = Clock::now();
  s->scheduler = std::thread(scheduler_loop, s);
  *out = s;
  return TPC_OK;
}

extern "C" int tpc_server_submit(tpc_server *s, const tpc_clusters *cl, const tpc_tracks *out, uint64_t *id) {
  report(TPC_OK, "");
  if (!s || !cl || !out || !id) return report(TPC_ERR_ARG, "tpc_server_submit: null argument");
  if (cl->n > 0 && (!cl->sector || !cl->row || !cl->pad || !cl->time || !out->cluster_track))
    return report(TPC_ERR_ARG, "tpc_server_submit: null array");
  Request *r = new Request();
  r->cl = *cl;
  r->out = *out;
  std::lock_guard<std::mutex> lk(s->mu);
  r->id = s->next_id++;
  r->t_submit = s->now();
  *id = r->id;
  s->queue.push_back(r);
  s->cv_sched.notify_all();
  return TPC_OK;
}

extern "C" int tpc_server_poll(tpc_server *s, tpc_server_result *res, int max, int wait_ms) {
  report(TPC_OK, "");
  if (!s || !res || max < 1) return report(TPC_ERR_ARG, "tpc_server_poll: bad argument");
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && wait_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
  int k = 0;
  while (k < max && !s->done.empty()) {
    Request *r = s->done.front();
    s->done.pop_front();
    res[k].id = r->id;
    res[k].status = r->status;
    res[k].n_clusters = r->cl.n;
    res[k].n_tracks = r->n_tracks;
    res[k].slot = r->slot;
    res[k].t_submit = r->t_submit;
    res[k].t_start = r->t_start;
    res[k].t_done = r->t_done;
    delete r;
    ++k;
  }
  return k;
}

extern "C" int tpc_server_stats(tpc_server *s, int *n_slots, uint64_t *bytes_in_use, int *queued) {
  report(TPC_OK, "");
  if (!s) return report(TPC_ERR_ARG, "tpc_server_stats: null server");
  std::lock_guard<std::mutex> lk(s->mu);
  uint64_t b = 0;
  for (auto *sl : s->slots) b += sl->bytes;
  if (n_slots) *n_slots = (int)s->slots.size();
  if (bytes_in_use) *bytes_in_use = b;
  if (queued) *queued = (int)s->queue.size();
  return TPC_OK;
}

extern "C" void tpc_server_destroy(tpc_server *s) {
  if (!s) return;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    // finish what is queued or running
    s->cv_done.wait(lk, [&] {
      if (!s->queue.empty()) return false;
      for (auto *sl : s->slots)
        if (sl->busy) return false;
      return true;
    });
    s->stop = true;
    s->cv_sched.notify_all();
    for (auto *sl : s->slots) sl->cv.notify_all();
  }
  if (s->scheduler.joinable()) s->scheduler.join();
  for (auto *sl : s->slots) {
    if (sl->worker.joinable()) sl->worker.join();
    if (sl->tf) tpc_tf_destroy(sl->tf);
    if (sl->stream) cudaStreamDestroy(sl->stream);
    delete sl;
  }
  for (auto *r : s->done) delete r;
  delete s;
}
