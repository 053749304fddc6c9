// Served path: continuous batching of group-finding requests.
//
// cso_submit queues a request and returns at once.  A fixed set of worker
// slots (each a full pipeline context: its own CUDA streams, workspace and
// pinned buffers, driven by its own host thread) takes requests in
// submission order as soon as a slot is free and the device memory the
// request needs fits the context's budget next to the requests already
// running.  Admitted requests run concurrently, so their kernels overlap on
// the GPU; every request is computed exactly as cso_find_groups computes it
// alone.  cso_poll waits for a ticket.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "cells.cuh"
#include "pipeline.cuh"
#include "stream.cuh"

struct ServedState {
  std::mutex mu;
  std::condition_variable cv_work;  // workers wait for admissible requests
  std::condition_variable cv_done;  // pollers wait for completions
  std::deque<ServedRequest*> queue;
  std::unordered_map<uint64_t, ServedRequest*> tickets;
  std::vector<cso_ctx*> slots;
  std::unordered_map<uint64_t, StreamState*> streams;  // slab streams by request_id
  std::vector<std::thread> workers;
  size_t in_use = 0;  // device bytes reserved by running requests
  bool stop = false;
};

static double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// device workspace one request needs (what ctx_reserve will ask for)
static size_t request_bytes(const cso_input* in, const cso_params* p, const cso_output* out, int* rc) {
  cso_params q = *p;
  *rc = cso_params_derive(&q);
  if (*rc != CSO_OK) return 0;
  int nc = 0;
  *rc = cells_choose(q.b2, &nc);
  if (*rc != CSO_OK) return 0;
  if (in->x_hi > 0) {
    // a slab: its window holds the slab, its ghosts and the open groups
    // behind it; budget three slabs' worth of particles over the slab's
    // columns and a margin
    const long long cols = (long long)(in->x_hi - in->x_lo) * nc / CSO_BOX + 8;
    return workspace_bytes(3 * in->n + 4096, (cols < nc ? cols : nc) * nc * nc, false);
  }
  *rc = cells_check_dense(nc);
  if (*rc != CSO_OK) return 0;
  return workspace_bytes(in->n, (long long)nc * nc * nc, !in->on_device || !out->on_device) +
         (size_t)(in->n / 16 + 1024) * 2 * sizeof(cso_halo);
}

static bool is_slab(const ServedRequest* r) { return r->in.x_hi > 0; }

// First admissible request in submission order: a whole box whose workspace
// fits the budget next to the running ones (none may overtake a whole box that
// does not fit yet), or a slab whose stream is not being worked on.
static std::deque<ServedRequest*>::iterator pick(ServedState& S, size_t budget) {
  for (auto it = S.queue.begin(); it != S.queue.end(); ++it) {
    ServedRequest* r = *it;
    const bool fits = budget == 0 || S.in_use + r->need <= budget;
    if (!is_slab(r)) {
      if (fits) return it;
      return S.queue.end();
    }
    auto st = S.streams.find(r->in.request_id);
    const bool busy = st != S.streams.end() && st->second->busy;
    if (!busy && fits) return it;
  }
  return S.queue.end();
}

static void finish(ServedRequest* r, int rc, double t) {
  r->status = rc;
  r->t_done = t;
  r->done = true;
}

static void run_slab(cso_ctx* slot, ServedState& S, ServedRequest* r) {
  StreamState* ss = nullptr;
  {
    std::lock_guard<std::mutex> lock(S.mu);
    auto it = S.streams.find(r->in.request_id);
    if (it != S.streams.end()) ss = it->second;
  }
  int rc = CSO_OK;
  if (!ss) {
    cso_set_error("a slab stream must start at x = 0");
    rc = CSO_ERR_STATE;
  }
  if (rc == CSO_OK && ss->failed) {
    cso_set_error("an earlier slab of this stream failed");
    rc = CSO_ERR_STATE;
  }
  if (rc == CSO_OK) {
    CSO_CUDA_VOID(cudaSetDevice(slot->device));
    rc = stream_step(slot, *ss, &r->in, r->out, r);
    if (rc != CSO_OK) ss->failed = true;
  }
  std::lock_guard<std::mutex> lock(S.mu);
  const double t = now_s();
  if (rc != CSO_OK) {
    finish(r, rc, t);
    if (ss) {  // every pending slab of a failed stream fails with it
      for (auto& sl : ss->slabs)
        if (!sl.completed && sl.req && !sl.req->done) finish(sl.req, CSO_ERR_STATE, t);
    }
  } else {
    bool all = true;
    for (auto& sl : ss->slabs) {
      if (sl.newly_completed) {
        sl.newly_completed = false;
        sl.req->out->n_halos = sl.n_halos;
        finish(sl.req, sl.n_halos > sl.out.halo_cap ? CSO_ERR_CAPACITY : CSO_OK, t);
      }
      all = all && sl.completed;
    }
    if (all && ss->x_received == CSO_BOX) {  // the stream is over
      S.streams.erase(ss->id);
      stream_release(ss);
      ss = nullptr;
    }
  }
  if (ss) ss->busy = false;
}

static void worker_loop(cso_ctx* parent, int k) {
  ServedState& S = *parent->served;
  cso_ctx* slot = S.slots[k];
  for (;;) {
    ServedRequest* r = nullptr;
    {
      std::unique_lock<std::mutex> lock(S.mu);
      S.cv_work.wait(lock, [&] { return S.stop || pick(S, parent->budget) != S.queue.end(); });
      if (S.stop) return;
      auto it = pick(S, parent->budget);
      r = *it;
      S.queue.erase(it);
      S.in_use += r->need;
      r->t_start = now_s();
      if (is_slab(r)) {
        auto st = S.streams.find(r->in.request_id);
        if (st != S.streams.end()) {
          st->second->busy = true;
        } else if (r->in.x_lo == 0) {  // the first slab opens the stream
          StreamState* ss = nullptr;
          if (stream_begin(&ss, r->in.request_id, &r->p) == CSO_OK) {
            ss->busy = true;
            S.streams[r->in.request_id] = ss;
          }
        }
      }
    }
    if (is_slab(r)) {
      run_slab(slot, S, r);
      std::lock_guard<std::mutex> lock(S.mu);
      S.in_use -= r->need;
    } else {
      // idle slots keep their workspace for the next request; the budget
      // counts what running requests reserve
      int rc = cso_find_groups(slot, &r->in, &r->p, r->out);
      std::lock_guard<std::mutex> lock(S.mu);
      finish(r, rc, now_s());
      S.in_use -= r->need;
    }
    S.cv_done.notify_all();
    S.cv_work.notify_all();
  }
}

static int served_start(cso_ctx* c) {
  if (c->served) return CSO_OK;
  ServedState* S = new ServedState();
  c->served = S;
  const int nslots = c->served_slots > 0 ? c->served_slots : 4;
  for (int k = 0; k < nslots; ++k) {
    cso_ctx* s = nullptr;
    int rc = cso_init(&s, c->device, 0, c->flags);
    if (rc != CSO_OK) return rc;
    S->slots.push_back(s);
  }
  for (int k = 0; k < nslots; ++k) S->workers.emplace_back(worker_loop, c, k);
  return CSO_OK;
}

void served_stop(cso_ctx* c) {
  ServedState* S = c->served;
  if (!S) return;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto* s : S->slots) cso_free(s);
  for (auto& kv : S->streams) stream_release(kv.second);
  for (auto& kv : S->tickets) delete kv.second;
  for (auto* r : S->queue) (void)r;  // owned through the ticket table
  delete S;
  c->served = nullptr;
}

extern "C" int cso_submit(cso_ctx* c, const cso_input* in, const cso_params* p, cso_output* out, uint64_t* ticket) {
  if (!c || !ticket) return CSO_ERR_ARG;
  CSO_TRY(check_io(in, p, out));
  int rc = CSO_OK;
  const size_t need = request_bytes(in, p, out, &rc);
  if (rc != CSO_OK) return rc;
  if (c->budget && need > c->budget) {
    cso_set_error("request needs %zu bytes of device memory, the budget is %zu", need, c->budget);
    return CSO_ERR_BUDGET;
  }
  CSO_TRY(served_start(c));
  ServedRequest* r = new ServedRequest();
  r->in = *in;
  r->p = *p;
  r->out = out;
  r->need = need;
  r->t_submit = now_s();
  ServedState& S = *c->served;
  bool admitted_now;
  {
    std::lock_guard<std::mutex> lock(S.mu);
    r->ticket = ++c->next_ticket;
    S.tickets[r->ticket] = r;
    admitted_now = S.queue.empty() && (c->budget == 0 || S.in_use + need <= c->budget);
    S.queue.push_back(r);
  }
  S.cv_work.notify_all();
  *ticket = r->ticket;
  return admitted_now ? CSO_OK : CSO_EAGAIN;
}

extern "C" int cso_poll(cso_ctx* c, uint64_t ticket, int32_t* done, int32_t timeout_us) {
  if (!c || !done) return CSO_ERR_ARG;
  *done = 0;
  if (!c->served) {
    cso_set_error("unknown ticket %llu", (unsigned long long)ticket);
    return CSO_ERR_STATE;
  }
  ServedState& S = *c->served;
  std::unique_lock<std::mutex> lock(S.mu);
  auto it = S.tickets.find(ticket);
  if (it == S.tickets.end()) {
    cso_set_error("unknown ticket %llu", (unsigned long long)ticket);
    return CSO_ERR_STATE;
  }
  ServedRequest* r = it->second;
  if (!r->done && timeout_us != 0) {
    auto pred = [&] { return r->done; };
    if (timeout_us < 0) S.cv_done.wait(lock, pred);
    else S.cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), pred);
  }
  if (!r->done) {
    if (timeout_us > 0) {
      cso_set_error("ticket %llu not done after %d us", (unsigned long long)ticket, (int)timeout_us);
      return CSO_ERR_TIMEOUT;
    }
    return CSO_OK;
  }
  *done = 1;
  return r->status;
}

extern "C" int cso_ticket_times(cso_ctx* c, uint64_t ticket, double* t_submit, double* t_start, double* t_done) {
  if (!c || !c->served) return CSO_ERR_STATE;
  ServedState& S = *c->served;
  std::lock_guard<std::mutex> lock(S.mu);
  auto it = S.tickets.find(ticket);
  if (it == S.tickets.end() || !it->second->done) return CSO_ERR_STATE;
  if (t_submit) *t_submit = it->second->t_submit;
  if (t_start) *t_start = it->second->t_start;
  if (t_done) *t_done = it->second->t_done;
  return CSO_OK;
}

extern "C" double cso_clock(void) { return now_s(); }
