// Continuous-batching request loop (serving form of the foveation path).
//
// Requests carry one frame in host memory. A worker thread
//   1. admits pending requests in arrival order while their input and output
//      buffers fit in a fixed device arena (admission by device memory) and
//      fewer than max_inflight requests are admitted;
//   2. copies each admitted input to the device on a copy stream;
//   3. whenever no batch is rendering, renders up to max_batch admitted
//      requests, one batch per (format, channel count) (fovea_render_batch:
//      sigma table, cost-ordered work list, persistent kernel) on a compute
//      stream that waits on the device for their input copies; requests
//      admitted while a batch renders gather into the next one;
//   4. copies each result back to its caller's host buffer on a third stream
//      and, once that copy is seen complete, frees the arena space.
// The paper's per-frame loop (Algorithm 1: pinned host -> device, kernel,
// device -> pinned host) is the special case max_batch = 1.
#if defined(__linux__)
#include <sys/prctl.h>
#endif
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "arena.h"
#include "fovea.h"
#include "fovea_host.h"

namespace {

double now_us() {
  using namespace std::chrono;
  return (double)duration_cast<nanoseconds>(steady_clock::now().time_since_epoch()).count() * 1e-3;
}

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

enum State { PENDING, ADMITTED, LAUNCHED, DONE };

struct Request {
  long long id = 0;
  fovea_frame f{};
  size_t bytes = 0;
  size_t off = 0;          // arena offset of [input | output]
  fovea_request_times t{};
  State state = PENDING;
  int status = 0;          // render status of its batch
  int fault_slot = -1;     // pinned word that receives its batch's device fault word
  cudaEvent_t ev_in = nullptr, ev_done = nullptr;
};

}  // namespace

struct fovea_server {
  fovea_server_config cfg{};
  int device = 0;
  char* arena_base = nullptr;
  fovea::Arena arena;
  fovea_ctx* ctx = nullptr;
  cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
  std::vector<cudaEvent_t> event_pool;
  std::deque<cudaEvent_t> batch_events;  // renders queued on s_comp
  std::mutex mu;
  std::condition_variable cv_done, cv_work;
  std::deque<Request*> pending;
  std::vector<Request*> admitted;  // state ADMITTED
  std::vector<Request*> launched;  // state LAUNCHED
  std::unordered_map<long long, Request*> all;
  long long next_id = 0;
  bool stop = false;
  std::thread worker;
  // Device fault words of the batches: after each batch the context's word
  // is copied into a pinned slot (and cleared) on the compute stream; the
  // batch's requests read it once their output copy is complete. A slot is
  // free again when every request of its batch has finished (at most
  // max_inflight batches hold requests, so max_inflight + 1 slots suffice).
  unsigned int* fault_words = nullptr;  // pinned, one per slot
  std::vector<int> fault_refs;          // unfinished requests per slot
  std::vector<int> fault_free;          // free slots
  unsigned int* fault_dev = nullptr;    // the batch context's device fault word

  cudaEvent_t get_event() {
    if (!event_pool.empty()) {
      cudaEvent_t e = event_pool.back();
      event_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
  }

  void finish(Request* r, int status) {
    r->t.done_us = now_us();
    if (r->fault_slot >= 0) {  // the output copy is complete, so the batch's fault word has landed
      const unsigned int w = fault_words[r->fault_slot];
      if (status == FOVEA_OK && w) status = fovea::fault_status(w);
      if (--fault_refs[(size_t)r->fault_slot] == 0) fault_free.push_back(r->fault_slot);
      r->fault_slot = -1;
    }
    r->t.status = status;
    if (r->state == ADMITTED || r->state == LAUNCHED) arena.release(r->off, 2 * align_up(r->bytes));
    r->state = DONE;
    if (r->ev_in) event_pool.push_back(r->ev_in);
    if (r->ev_done) event_pool.push_back(r->ev_done);
    r->ev_in = r->ev_done = nullptr;
  }

  void run();
};

void fovea_server::run() {
  cudaSetDevice(device);
#if defined(__linux__)
  prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);  // 1 us: short polling sleeps stay short
#endif
  std::vector<Request*> fresh, ready;
  std::vector<fovea_frame> frames;
  for (;;) {
    bool progressed = false;
    fresh.clear();
    {
      std::unique_lock<std::mutex> lk(mu);
      if (stop && pending.empty() && admitted.empty() && launched.empty()) break;
      while (!pending.empty() && (int)(admitted.size() + launched.size()) < cfg.max_inflight) {
        Request* r = pending.front();
        size_t off = 0;
        if (!arena.alloc(2 * align_up(r->bytes), &off)) break;  // wait for memory to free up
        pending.pop_front();
        r->off = off;
        r->state = ADMITTED;
        r->t.admit_us = now_us();
        r->ev_in = get_event();
        r->ev_done = get_event();
        admitted.push_back(r);
        fresh.push_back(r);
      }
    }
    for (Request* r : fresh) {  // input copies on the copy stream
      if (cudaMemcpyAsync(arena_base + r->off, r->f.in, r->bytes, cudaMemcpyHostToDevice, s_in) != cudaSuccess ||
          cudaEventRecord(r->ev_in, s_in) != cudaSuccess) {
        const int st = fovea::record_cuda_failure((int)cudaGetLastError());
        std::lock_guard<std::mutex> lk(mu);
        admitted.erase(std::find(admitted.begin(), admitted.end(), r));
        finish(r, st);
        cv_done.notify_all();
      }
      progressed = true;
    }
    // Retire finished renders. One batch at a time on the compute stream:
    // requests that become ready while it runs form the next batch (an idle
    // GPU takes a request at once, a busy one collects them).
    while (!batch_events.empty() && cudaEventQuery(batch_events.front()) == cudaSuccess) {
      std::lock_guard<std::mutex> lk(mu);
      event_pool.push_back(batch_events.front());
      batch_events.pop_front();
    }
    if (batch_events.empty()) {
      ready.clear();
      {
        // Every admitted request joins the batch, whether or not its input
        // copy has landed: the compute stream waits for the copies on the
        // device, so the launch overlaps them and no host poll sits between
        // a copy finishing and its render starting.
        std::lock_guard<std::mutex> lk(mu);
        const size_t take = std::min(admitted.size(), (size_t)cfg.max_batch);
        ready.assign(admitted.begin(), admitted.begin() + (long)take);
        admitted.erase(admitted.begin(), admitted.begin() + (long)take);
      }
      int wait_status = FOVEA_OK;
      for (Request* r : ready) {
        if (cudaEventQuery(r->ev_in) != cudaSuccess && cudaStreamWaitEvent(s_comp, r->ev_in, 0) != cudaSuccess)
          wait_status = fovea::record_cuda_failure((int)cudaGetLastError());
      }
      if (!ready.empty()) {
        // One batch per (format, channel count): a request is rendered by the
        // same kernel whatever else arrived with it, so its result does not
        // depend on the mix.
        std::stable_sort(ready.begin(), ready.end(), [](const Request* a, const Request* b) {
          return a->f.format != b->f.format ? a->f.format < b->f.format : a->f.channels < b->f.channels;
        });
        fovea::TraceRange trace("server batch");
        const double t0 = now_us();
        bool failed = false;
        for (size_t g0 = 0; g0 < ready.size();) {
          size_t g1 = g0 + 1;
          while (g1 < ready.size() && ready[g1]->f.format == ready[g0]->f.format &&
                 ready[g1]->f.channels == ready[g0]->f.channels)
            ++g1;
          frames.resize(g1 - g0);
          for (size_t i = g0; i < g1; ++i) {
            fovea_frame f = ready[i]->f;
            f.in = arena_base + ready[i]->off;
            f.out = arena_base + ready[i]->off + align_up(ready[i]->bytes);
            frames[i - g0] = f;
          }
          const int st = wait_status != FOVEA_OK ? wait_status
                                                 : fovea_render_batch(ctx, frames.data(), (int)frames.size(), s_comp);
          for (size_t i = g0; i < g1; ++i) {
            ready[i]->status = st;
            ready[i]->t.batch_size = (int)(g1 - g0);
          }
          failed |= st != FOVEA_OK;
          g0 = g1;
        }
        cudaEvent_t eb = nullptr;
        int slot = -1;
        {
          std::lock_guard<std::mutex> lk(mu);
          eb = get_event();
          if (!fault_free.empty()) {
            slot = fault_free.back();
            fault_free.pop_back();
          }
        }
        // the batch's fault word goes to the slot and is cleared for the next batch
        int tail_status = FOVEA_OK;
        if (slot < 0 ||
            cudaMemcpyAsync(fault_words + slot, fault_dev, sizeof(unsigned int), cudaMemcpyDeviceToHost, s_comp) !=
                cudaSuccess ||
            cudaMemsetAsync(fault_dev, 0, sizeof(unsigned int), s_comp) != cudaSuccess ||
            !eb || cudaEventRecord(eb, s_comp) != cudaSuccess || cudaStreamWaitEvent(s_out, eb, 0) != cudaSuccess)
          tail_status = slot < 0 ? FOVEA_ECUDA : fovea::record_cuda_failure((int)cudaGetLastError());
        if (eb) batch_events.push_back(eb);
        std::lock_guard<std::mutex> lk(mu);
        int refs = 0;
        for (Request* r : ready) {
          r->t.start_us = t0;
          if (r->status == FOVEA_OK) r->status = tail_status;
          if (r->status == FOVEA_OK &&
              (cudaMemcpyAsync(r->f.out, arena_base + r->off + align_up(r->bytes), r->bytes, cudaMemcpyDeviceToHost,
                               s_out) != cudaSuccess ||
               cudaEventRecord(r->ev_done, s_out) != cudaSuccess))
            r->status = fovea::record_cuda_failure((int)cudaGetLastError());
          if (r->status != FOVEA_OK) {
            finish(r, r->status);
            failed = true;
            continue;
          }
          r->fault_slot = slot;
          ++refs;
          r->state = LAUNCHED;
          launched.push_back(r);
        }
        if (slot >= 0) {
          fault_refs[(size_t)slot] = refs;
          if (refs == 0) fault_free.push_back(slot);
        }
        if (failed) cv_done.notify_all();
        progressed = true;
      }
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      bool any = false;
      for (size_t i = 0; i < launched.size();) {
        Request* r = launched[i];
        if (cudaEventQuery(r->ev_done) == cudaSuccess) {
          finish(r, FOVEA_OK);
          launched.erase(launched.begin() + (long)i);
          any = true;
        } else {
          ++i;
        }
      }
      if (any) {
        cv_done.notify_all();
        progressed = true;
      }
    }
    if (!progressed) {
      std::unique_lock<std::mutex> lk(mu);
      if (pending.empty() && admitted.empty() && launched.empty() && !stop) {
        cv_work.wait_for(lk, std::chrono::milliseconds(5));
      } else {
        // Work is in flight: poll again after 10 us (the worker runs with a
        // 1 us timer slack, so the sleep stays short, yet the submitting
        // threads still get the lock between polls).
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(10));
      }
    }
  }
}

extern "C" {

double fovea_server_now_us(void) { return now_us(); }

int fovea_server_create(const fovea_server_config* cfg, fovea_server** out) {
  if (!cfg || !out) return FOVEA_EINVAL;
  *out = nullptr;
  if (cfg->device_budget_bytes < 2 * kAlign || cfg->max_batch <= 0 || cfg->max_inflight <= 0 || cfg->block <= 0)
    return FOVEA_EINVAL;
  fovea_server* s = new (std::nothrow) fovea_server();
  if (!s) return FOVEA_ENOMEM;
  s->cfg = *cfg;
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaMalloc(&s->arena_base, cfg->device_budget_bytes) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->s_in, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->s_comp, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->s_out, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    fovea_server_destroy(s);
    return FOVEA_ENOMEM;
  }
  s->arena.reset(cfg->device_budget_bytes);
  const int nslots = cfg->max_inflight + 1;
  if (cudaHostAlloc(&s->fault_words, (size_t)nslots * sizeof(unsigned int), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    s->fault_words = nullptr;
    fovea_server_destroy(s);
    return FOVEA_ENOMEM;
  }
  s->fault_refs.assign((size_t)nslots, 0);
  for (int i = nslots - 1; i >= 0; --i) s->fault_free.push_back(i);
  fovea_sigma_law law{FOVEA_LAW_LINEAR, 0.5, 0.02, 0.0, nullptr, 0.0, FOVEA_GRID_ANCHORED};
  int st = fovea_create(0, 0, 3, cfg->block, &law, FOVEA_U8_HWC, &s->ctx);
  if (st == FOVEA_OK) st = fovea::ctx_fault_word(s->ctx, &s->fault_dev);
  // Every batch runs one fixed configuration (not one the batch autotuner
  // chose for batches of its kind), so a request's result does not depend on
  // what it is batched with.
  if (st == FOVEA_OK) {
    const fovea_config fixed{256, 0, 32, 1};
    st = fovea_set_config(s->ctx, &fixed);
  }
  // Size the batch buffers for the largest batch the arena can hold, so that
  // no batch grows them (a growth recaptures the batch graphs on this
  // thread, and the backlog that makes a batch large is when that hurts
  // most). A batch's frames are all resident in the arena, input and output,
  // so they hold at most budget / 2 pixels; a frame of W x H pixels has at
  // most (W / B + 1) (H / B + 1) items, at most 4 W H / B^2 when both sides
  // are at least B. Smaller frames are covered by 16 items a frame; beyond
  // the cap the buffers still grow on demand.
  if (st == FOVEA_OK) {
    const long long bb = (long long)cfg->block * cfg->block;
    const long long items = std::min<long long>(
        2 * (long long)(cfg->device_budget_bytes / (size_t)bb) + 16ll * cfg->max_batch, 1ll << 22);
    st = fovea_reserve(s->ctx, std::min(cfg->max_batch, 1 << 24), items);
  }
  if (st != FOVEA_OK) {
    fovea_server_destroy(s);
    return st;
  }
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return FOVEA_OK;
}

long long fovea_server_submit(fovea_server* s, const fovea_frame* f, double arrival_us) {
  if (!s || !f || !f->in || !f->out) return FOVEA_EINVAL;
  fovea::FrameLaw law;
  law.sigma0 = f->sigma0; law.k = f->k; law.smap = f->sigma_map; law.smap_max = f->sigma_map_max;
  law.grid = f->grid;
  const int st = fovea::check_frame(f->width, f->height, f->channels, f->format, s->cfg.block, law, f->fix_x,
                                    f->fix_y);
  if (st != FOVEA_OK) return st;
  const size_t bytes = fovea::frame_bytes(f->width, f->height, f->channels, f->format);
  if (2 * align_up(bytes) > s->cfg.device_budget_bytes) return FOVEA_EBUSY;
  Request* r = new (std::nothrow) Request();
  if (!r) return FOVEA_ENOMEM;
  r->f = *f;
  r->bytes = bytes;
  r->t.arrival_us = arrival_us;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    delete r;
    return FOVEA_EINVAL;
  }
  r->id = s->next_id++;
  s->all[r->id] = r;
  s->pending.push_back(r);
  s->cv_work.notify_one();
  return r->id;
}

int fovea_server_wait(fovea_server* s, long long id, int timeout_ms, fovea_request_times* times) {
  if (!s) return FOVEA_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return FOVEA_EINVAL;
  Request* r = it->second;
  if (r->state != DONE) {
    if (timeout_ms <= 0) return FOVEA_ETIMEOUT;
    s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [r] { return r->state == DONE; });
    if (r->state != DONE) return FOVEA_ETIMEOUT;
  }
  if (times) *times = r->t;
  s->all.erase(it);
  delete r;
  return FOVEA_OK;
}

void fovea_server_destroy(fovea_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->s_in) cudaStreamSynchronize(s->s_in);
  if (s->s_comp) cudaStreamSynchronize(s->s_comp);
  if (s->s_out) cudaStreamSynchronize(s->s_out);
  for (auto& kv : s->all) {
    Request* r = kv.second;
    if (r->ev_in) cudaEventDestroy(r->ev_in);
    if (r->ev_done) cudaEventDestroy(r->ev_done);
    delete r;
  }
  for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : s->batch_events) cudaEventDestroy(e);
  if (s->ctx) fovea_destroy(s->ctx);
  if (s->s_in) cudaStreamDestroy(s->s_in);
  if (s->s_comp) cudaStreamDestroy(s->s_comp);
  if (s->s_out) cudaStreamDestroy(s->s_out);
  cudaFree(s->arena_base);
  if (s->fault_words) cudaFreeHost(s->fault_words);
  delete s;
}

}  // extern "C"
