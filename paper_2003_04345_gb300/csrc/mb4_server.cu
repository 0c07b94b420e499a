// libmb4 serving loop: continuous batching of MB4 simulation requests.
//
// One batch per shape class (nx, ny, tx, ty, onsite, h), each on its own CUDA
// stream, inside an HBM budget.  The classes run independently in time: the loop
// polls each class's last chunk with an event and, as soon as THAT class is idle,
//   1. books the chunk's steps and retires the requests that reached their step
//      count (final energy, final state), freeing their slots,
//   2. admits every arrived request of that class into a free slot (creating the
//      class's batch when the budget allows, releasing idle batches when it does
//      not), queues the observables of the new requests (their start energy, read
//      back asynchronously) and
//   3. enqueues the class's next chunk of steps (at most 32, never past its earliest
//      finishing request) and records its event.
// A small class therefore keeps admitting, stepping and retiring while a large class
// is in the middle of a long chunk; the kernels of different classes overlap on the
// GPU, and smaller classes run on higher-priority streams.  States stay on the GPU from
// admission to completion.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <new>
#include <thread>
#include <vector>

#include "mb4_internal.h"

namespace {

constexpr long long kMaxChunk = 32;   // steps per pass: bounds the wait before new admissions

struct ServerReq {
  mb4_grid grid{};
  double h = 0, chi = 0, arrival = 0;
  int nsteps = 0;
  std::vector<double> v, re, im;
  mb4_result res{};
  int cls = -1, slot = -1;
  long long remaining = 0;
  bool queued = true;
  std::vector<double> out_re, out_im;
};

struct ClassBatch {
  mb4_grid grid{};
  double h = 0;
  mb4_batch* b = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;        // recorded after the class's last enqueued chunk
  bool in_flight = false;            // a chunk is queued or running on the class's stream
  double* obs = nullptr;             // page-locked, slots x 6: observables read back asynchronously
  std::vector<int> start_pending;    // slots whose start energy is in obs once the chunk is done
  int slots = 0;
  long long bytes = 0;
  std::vector<long long> slot_req;   // request in each slot, -1 = free
  int running = 0;
  long long chunk = 0;
};

bool same_class(const ClassBatch& c, const mb4_grid& g, double h) {
  return c.grid.nx == g.nx && c.grid.ny == g.ny && c.grid.tx == g.tx && c.grid.ty == g.ty &&
         c.grid.onsite == g.onsite && c.h == h;
}

}  // namespace

struct mb4_server {
  long long budget = 0;
  int max_slots = 1;
  int keep = 0;
  mb4_options opt{};
  std::vector<ServerReq> reqs;
  std::deque<long long> queue;
  std::vector<ClassBatch*> classes;
  long long used = 0;
  long long n_done = 0;
  std::chrono::steady_clock::time_point t0;
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

void free_class(ClassBatch* c) {
  if (c->b) mb4_batch_destroy(c->b);
  if (c->done) cudaEventDestroy(c->done);
  if (c->obs) cudaFreeHost(c->obs);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

void release_class(mb4_server* s, size_t idx) {
  ClassBatch* c = s->classes[idx];
  s->used -= c->bytes;
  free_class(c);
  s->classes.erase(s->classes.begin() + idx);
}

// A batch for (grid, h) with as many slots as the budget allows (at most max_slots),
// releasing idle batches first if needed.  Returns nullptr if not even one slot fits now.
ClassBatch* create_class(mb4_server* s, const mb4_grid& g, double h, int want) {
  const long long one = mb4_batch_bytes(g.nx, g.ny, 1, &s->opt);
  if (one <= 0) return nullptr;
  if (s->used + one > s->budget) {
    for (size_t i = 0; i < s->classes.size();) {
      if (s->classes[i]->running == 0 && !s->classes[i]->in_flight) release_class(s, i);
      else ++i;
      if (s->used + one <= s->budget) break;
    }
  }
  if (s->used + one > s->budget) return nullptr;
  int slots = std::max(1, std::min(s->max_slots, want));
  while (slots > 1 && s->used + mb4_batch_bytes(g.nx, g.ny, slots, &s->opt) > s->budget) slots /= 2;
  ClassBatch* c = new (std::nothrow) ClassBatch();
  if (!c) return nullptr;
  c->grid = g;
  c->h = h;
  c->slots = slots;
  c->bytes = mb4_batch_bytes(g.nx, g.ny, slots, &s->opt);
  // Smaller classes get higher stream priority: when SMs free up, the block scheduler
  // serves their short kernels before the pending blocks of a large class, so a small
  // request is not stretched to the pace of a large class running beside it.
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  const long long sites = (long long)g.nx * g.ny;
  const int prio = (sites <= 128LL * 128) ? greatest : (sites <= 512LL * 512) ? (least + greatest) / 2 : least;
  if (cudaStreamCreateWithPriority(&c->stream, cudaStreamNonBlocking, prio) != cudaSuccess) {
    delete c;
    return nullptr;
  }
  mb4_options o = s->opt;
  o.stream = c->stream;
  // no launch-shape timing at admission: its launches would queue behind the kernels of
  // the classes already running (a delay for the new request) and time their load rather
  // than the class's own kernels; the classes keep the default shape
  o.autotune = 0;
  const size_t S = (size_t)g.nx * g.ny;
  std::vector<double> V(S * slots, 0.0), chi(slots, 0.0);
  mb4_potential pot{V.data(), 0};
  if (cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost((void**)&c->obs, (size_t)slots * 6 * sizeof(double)) != cudaSuccess ||
      mb4_batch_create(&g, slots, &pot, chi.data(), h, &o, &c->b) != MB4_OK ||
      mb4_batch_enable(c->b, -1, 0) != MB4_OK) {
    free_class(c);
    return nullptr;
  }
  c->slot_req.assign(slots, -1);
  s->used += c->bytes;
  s->classes.push_back(c);
  return c;
}

void complete(mb4_server* s, ClassBatch* c, int slot, int status, double energy_end) {
  const long long id = c->slot_req[slot];
  ServerReq& r = s->reqs[id];
  r.res.status = status;
  r.res.done = 1;
  r.res.completed = s->now();
  r.res.energy_end = energy_end;
  if (s->keep) {
    const size_t S = (size_t)r.grid.nx * r.grid.ny;
    r.out_re.resize(S);
    r.out_im.resize(S);
    mb4_batch_get_state(c->b, slot, r.out_re.data(), r.out_im.data(), 0);
  }
  mb4_batch_enable(c->b, slot, 0);
  c->slot_req[slot] = -1;
  c->running -= 1;
  s->n_done += 1;
}

// Books the finished chunk of an idle class: steps, start energies of the requests admitted
// before it, retirement of the requests that are done.  Returns MB4_OK or a call failure.
int harvest_class(mb4_server* s, ClassBatch* c, std::vector<mb4_stats>& stats, std::vector<int>& codes,
                  std::vector<double>& obs) {
  for (int sl : c->start_pending)                // queued before the chunk, so complete now
    if (c->slot_req[sl] >= 0) s->reqs[c->slot_req[sl]].res.energy_start = c->obs[(size_t)sl * 6];
  c->start_pending.clear();
  stats.resize(c->slots);
  codes.resize(c->slots);
  const int wrc = mb4_batch_wait(c->b, stats.data(), codes.data());   // the stream is idle
  if (wrc != MB4_OK && wrc != MB4_ERR_NEWTON_NOT_CONVERGED && wrc != MB4_ERR_NONFINITE && wrc != MB4_ERR_TIMEOUT)
    return wrc;                                  // the call itself failed
  bool finished = false;
  for (int sl = 0; sl < c->slots; ++sl) {
    const long long id = c->slot_req[sl];
    if (id < 0) continue;
    ServerReq& r = s->reqs[id];
    r.res.steps_done += stats[sl].steps_done;
    r.res.newton_iters_total += stats[sl].newton_iters_total;
    r.remaining -= stats[sl].steps_done;
    if (codes[sl] != MB4_OK || r.remaining <= 0) finished = true;
  }
  if (!finished) return MB4_OK;
  obs.resize((size_t)c->slots * 6);
  const int orc = mb4_batch_observables(c->b, obs.data());   // final energies (idle stream)
  if (orc != MB4_OK) return orc;
  for (int sl = 0; sl < c->slots; ++sl) {
    const long long id = c->slot_req[sl];
    if (id < 0) continue;
    if (codes[sl] != MB4_OK || s->reqs[id].remaining <= 0) complete(s, c, sl, codes[sl], obs[(size_t)sl * 6]);
  }
  if (std::any_of(codes.begin(), codes.end(), [](int x) { return x != MB4_OK; })) mb4_batch_clear_errors(c->b);
  return MB4_OK;
}

}  // namespace

extern "C" {

int mb4_server_create(long long budget, int max_slots, int keep_states, const mb4_options* opt,
                      mb4_server** out) {
  if (!out || budget <= 0 || max_slots < 1) return MB4_ERR_INVALID_ARG;
  *out = nullptr;
  mb4_server* s = new (std::nothrow) mb4_server();
  if (!s) return MB4_ERR_OUT_OF_MEMORY;
  if (opt) s->opt = *opt;
  else mb4_default_options(&s->opt);
  if (mb4_batch_bytes(8, 8, 1, &s->opt) <= 0) {
    delete s;
    return MB4_ERR_INVALID_ARG;
  }
  s->budget = budget;
  s->max_slots = max_slots;
  s->keep = keep_states ? 1 : 0;
  s->t0 = std::chrono::steady_clock::now();
  *out = s;
  return MB4_OK;
}

void mb4_server_destroy(mb4_server* s) {
  if (!s) return;
  while (!s->classes.empty()) release_class(s, s->classes.size() - 1);
  delete s;
}

double mb4_server_clock(const mb4_server* s) { return s ? s->now() : 0.0; }

int mb4_server_submit(mb4_server* s, const mb4_request* q, long long* id) {
  if (!s || !q || !q->v || !q->re || !q->im || q->nsteps < 1) return MB4_ERR_INVALID_ARG;
  const mb4_grid& g = q->grid;
  if (g.nx < 3 || g.ny < 3 || (long long)g.nx * g.ny > (1LL << 30)) return MB4_ERR_INVALID_ARG;
  if (!std::isfinite(q->h) || q->h == 0.0 || !std::isfinite(q->chi) || !std::isfinite(q->arrival))
    return MB4_ERR_INVALID_ARG;
  const long long one = mb4_batch_bytes(g.nx, g.ny, 1, &s->opt);
  if (one <= 0) return MB4_ERR_INVALID_ARG;
  if (one > s->budget) return MB4_ERR_ADMISSION_REJECTED;
  ServerReq r;
  r.grid = g;
  r.h = q->h;
  r.chi = q->chi;
  r.nsteps = q->nsteps;
  r.arrival = q->arrival;
  const size_t S = (size_t)g.nx * g.ny;
  for (size_t k = 0; k < S; ++k)
    if (!std::isfinite(q->v[k]) || !std::isfinite(q->re[k]) || !std::isfinite(q->im[k])) return MB4_ERR_INVALID_ARG;
  r.v.assign(q->v, q->v + S);
  r.re.assign(q->re, q->re + S);
  r.im.assign(q->im, q->im + S);
  r.res.arrival = q->arrival;
  s->reqs.push_back(std::move(r));
  const long long k = (long long)s->reqs.size() - 1;
  s->queue.push_back(k);
  if (id) *id = k;
  return MB4_OK;
}

int mb4_server_run(mb4_server* s, double until, long long* n_done) {
  if (!s) return MB4_ERR_INVALID_ARG;
  std::vector<mb4_stats> stats;
  std::vector<int> codes;
  std::vector<double> obs;
  for (;;) {
    const double t = s->now();
    if (t >= until) break;
    bool progress = false;
    // 1. classes whose chunk has finished: book it, retire finished requests
    for (ClassBatch* c : s->classes) {
      if (!c->in_flight) continue;
      const cudaError_t q = cudaEventQuery(c->done);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) return MB4_ERR_CUDA;
      c->in_flight = false;
      progress = true;
      const int rc = harvest_class(s, c, stats, codes, obs);
      if (rc != MB4_OK) return rc;
    }
    // 2. admission (first come, first served among the requests that have arrived), into
    //    classes that are idle; a request whose class is mid-chunk waits for that chunk only
    for (auto it = s->queue.begin(); it != s->queue.end();) {
      ServerReq& r = s->reqs[*it];
      if (r.arrival > t) {
        ++it;
        continue;
      }
      ClassBatch* c = nullptr;
      bool busy_class = false;                   // a batch of this class is mid-chunk with room
      for (ClassBatch* cb : s->classes)
        if (same_class(*cb, r.grid, r.h) && cb->running < cb->slots) {
          if (cb->in_flight) {
            busy_class = true;
            continue;
          }
          c = cb;
          break;
        }
      if (!c && !busy_class) {
        int want = 0;   // requests of this class that have arrived and wait
        for (long long q : s->queue)
          if (s->reqs[q].arrival <= t && s->reqs[q].grid.nx == r.grid.nx && s->reqs[q].grid.ny == r.grid.ny &&
              s->reqs[q].h == r.h)
            ++want;
        c = create_class(s, r.grid, r.h, want);
      }
      if (!c) {
        ++it;
        continue;
      }
      int slot = -1;
      for (int k = 0; k < c->slots; ++k)
        if (c->slot_req[k] < 0) {
          slot = k;
          break;
        }
      if (slot < 0) {
        ++it;
        continue;
      }
      int rc = mb4_batch_load(c->b, slot, r.v.data(), r.chi, r.re.data(), r.im.data(), 0);
      if (rc == MB4_ERR_INVALID_ARG) {           // this request's inputs do not fit its class: it fails alone
        r.res.status = rc;
        r.res.done = 1;
        r.res.admitted = r.res.completed = s->now();
        r.queued = false;
        s->n_done += 1;
        it = s->queue.erase(it);
        continue;
      }
      if (rc != MB4_OK) return rc;
      c->slot_req[slot] = *it;
      c->running += 1;
      c->start_pending.push_back(slot);
      r.cls = 0;
      r.slot = slot;
      r.remaining = r.nsteps;
      r.queued = false;
      r.res.admitted = s->now();
      std::vector<double>().swap(r.v);
      std::vector<double>().swap(r.re);
      std::vector<double>().swap(r.im);
      progress = true;
      it = s->queue.erase(it);
    }
    // 3. every idle class with running requests: the start energies of its new requests
    //    (read back when the chunk is done), then its next chunk and its event
    for (ClassBatch* c : s->classes) {
      if (c->in_flight || c->running == 0) continue;
      if (!c->start_pending.empty()) {
        const int rc = mb4::batch_observables_async(c->b, c->obs);
        if (rc != MB4_OK) return rc;
      }
      long long k = kMaxChunk;
      for (int sl = 0; sl < c->slots; ++sl)
        if (c->slot_req[sl] >= 0) k = std::min(k, s->reqs[c->slot_req[sl]].remaining);
      int rc = mb4_batch_step_async(c->b, (int)k);
      if (rc != MB4_OK) return rc;
      if (cudaEventRecord(c->done, c->stream) != cudaSuccess) return MB4_ERR_CUDA;
      c->chunk = k;
      c->in_flight = true;
      progress = true;
    }
    bool any_flight = false;
    for (ClassBatch* c : s->classes) any_flight |= c->in_flight;
    if (!any_flight && s->queue.empty()) break;
    if (progress) continue;
    // 4. nothing to do until a chunk finishes or a request arrives
    double next = 1e300;
    for (long long q : s->queue) next = std::min(next, s->reqs[q].arrival);
    if (!any_flight) {
      if (next <= s->now()) {
        if (s->classes.empty()) return MB4_ERR_ADMISSION_REJECTED;   // arrived, nothing creatable
      }
      const double dt = std::min(next - s->now(), until - s->now());
      if (dt > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(dt, 0.01)));
    } else {
      std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
  }
  if (n_done) *n_done = s->n_done;
  return MB4_OK;
}

int mb4_server_result(const mb4_server* s, long long id, mb4_result* out, double* re, double* im) {
  if (!s || id < 0 || id >= (long long)s->reqs.size() || !out) return MB4_ERR_INVALID_ARG;
  const ServerReq& r = s->reqs[id];
  *out = r.res;
  if ((re || im) && r.res.done) {
    if (!s->keep || r.out_re.empty()) return MB4_ERR_INVALID_ARG;
    if (re) std::memcpy(re, r.out_re.data(), r.out_re.size() * sizeof(double));
    if (im) std::memcpy(im, r.out_im.data(), r.out_im.size() * sizeof(double));
  }
  return MB4_OK;
}

}  // extern "C"
