// Serving runtime: continuous admission of reciprocal evaluations (and gradients) for
// metasurfaces of different sizes and angular distributions on one GPU.
//
// Many evaluations are what the method is for (the inverse-design loops of Sec. 5.1 and
// the many-angle averages it replaces, Sec. 1).  Here requests arrive one by one and are
// served by `slots` workers, each a host thread with its own CUDA stream, so evaluations
// of different requests overlap on the device.  Device memory comes from one arena
// allocated when the server starts; a request is admitted when a slot is free and its
// grid (footprint from the descriptor) can be carved out of the arena, after evicting
// resident factorisations that no request is using, least recently used first.  A request
// that does not fit waits at the head of the queue until memory is released; free slots
// may start up to `lookahead` later requests that do fit ahead of it, and a head request
// passed over that many times blocks further overtaking.  Requests that carry a
// design_key leave their factorised grid resident (up to cache_bytes) so a later request
// with the same key, geometry and widths skips assembly and factorisation.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "arena.h"
#include "common.cuh"

rci_status rci_grid_alloc_with(const rci_grid_desc* desc, cudaStream_t stream, const DevMem* mem,
                               int with_grad, rci_grid** out);
rci_status rci_grid_init(rci_grid* g);
void rci_grid_rebind_stream(rci_grid* g, cudaStream_t s);
void rci_grid_destroy_idle(rci_grid* g);

namespace {

constexpr int MAX_SLOTS = 64;
constexpr int MAX_BYPASS = 16;

struct Request {
  uint64_t ticket = 0;
  rci_grid_desc desc{};
  std::vector<double> widths;
  rci_objective obj{};
  std::vector<double> w_row;   // USER_ROW objective (copied)
  rci_light light{};
  std::vector<double> lags;    // USER_LAGS light (copied)
  std::vector<double> tab;     // TABULATED light: angles then densities (copied)
  int want_grad = 0;
  uint64_t key = 0;
  double* grad_out = nullptr;
  double t_submit = 0.0;
  size_t footprint = 0;
  int bypassed = 0;
};

struct Resident {
  rci_grid* g = nullptr;
  uint64_t key = 0;
  rci_grid_desc desc{};
  std::vector<double> widths;
  size_t bytes = 0;
  uint64_t last_use = 0;
  bool pinned = false;
};

bool same_desc(const rci_grid_desc& a, const rci_grid_desc& b) {
  return std::memcmp(&a, &b, sizeof(rci_grid_desc)) == 0;
}

}  // namespace

struct rci_server {
  int device = 0, slots = 1, lookahead = 0;
  size_t cache_cap = 0;
  void* base = nullptr;
  Arena arena;
  std::mutex amu;  // arena
  std::mutex mu;   // everything below
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, rci_result> done;
  std::unordered_map<uint64_t, int> outstanding;  // submitted, not yet collected
  std::list<Resident> cache;                       // front = most recently used
  size_t cache_bytes = 0;
  int in_flight = 0;   // admitted, not yet finished
  int running = 0;     // holding (or allocating) a grid
  bool stop = false;
  uint64_t next_ticket = 1, use_clock = 0;
  rci_server_stats st{};
  std::vector<cudaStream_t> streams;
  std::vector<std::thread> workers;
  std::chrono::steady_clock::time_point t0;
  DevMem mem;

  double now_us() const {
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

cudaError_t arena_alloc(void* ctx, void** p, size_t bytes) {
  auto* s = static_cast<rci_server*>(ctx);
  std::lock_guard<std::mutex> lk(s->amu);
  size_t off = 0;
  if (!s->arena.alloc(bytes, &off)) return cudaErrorMemoryAllocation;
  *p = static_cast<char*>(s->base) + off;
  return cudaSuccess;
}

void arena_free(void* ctx, void* p) {
  auto* s = static_cast<rci_server*>(ctx);
  std::lock_guard<std::mutex> lk(s->amu);
  s->arena.release((size_t)(static_cast<char*>(p) - static_cast<char*>(s->base)));
}

size_t arena_largest_free(rci_server* s) {
  std::lock_guard<std::mutex> lk(s->amu);
  return s->arena.largest_free();
}

// Drop the least recently used resident grid nobody is using (caller holds s->mu).
// A resident grid has no device work pending (its worker drained the slot's stream before
// retiring it), so its memory returns to the arena at once, without waiting on the stream
// it last ran on, which another slot's request may be using by now.
bool evict_one(rci_server* s) {
  for (auto it = s->cache.end(); it != s->cache.begin();) {
    --it;
    if (it->pinned) continue;
    rci_grid_destroy_idle(it->g);
    s->cache_bytes -= it->bytes;
    s->cache.erase(it);
    s->st.cache_evictions++;
    return true;
  }
  return false;
}

// A resident grid for this request (pinned), or nullptr (caller holds s->mu).
rci_grid* cache_take(rci_server* s, const Request* r) {
  if (!r->key) return nullptr;
  for (auto it = s->cache.begin(); it != s->cache.end(); ++it) {
    if (it->pinned || it->key != r->key || !same_desc(it->desc, r->desc) ||
        it->widths != r->widths)
      continue;
    it->pinned = true;
    it->last_use = ++s->use_clock;
    s->cache.splice(s->cache.begin(), s->cache, it);
    return it->g;
  }
  return nullptr;
}

// An idle resident grid that a request would reuse (caller holds s->mu).
bool cache_match(const rci_server* s, const Request* r) {
  if (!r->key) return false;
  for (const auto& e : s->cache)
    if (!e.pinned && e.key == r->key && same_desc(e.desc, r->desc) && e.widths == r->widths)
      return true;
  return false;
}

bool evictable(const rci_server* s) {
  for (const auto& e : s->cache)
    if (!e.pinned) return true;
  return false;
}

// Next request for a free worker (removed from the queue), or nullptr when it should wait
// for memory.  The head is taken when it reuses a resident grid, when its footprint fits in
// the largest free block (then every one of its allocations fits: first fit leaves that
// block whole for whatever the earlier blocks cannot hold), when idle resident grids can be
// evicted for it, or when nothing else holds memory (it then fits or fails with ENOMEM).  Otherwise one
// of the next `lookahead` requests that fits may start first, unless the head has been
// passed over MAX_BYPASS times.  Caller holds s->mu.
Request* pick(rci_server* s) {
  Request* head = s->queue.front();
  if (s->running == 0 || cache_match(s, head) || evictable(s)) {
    s->queue.pop_front();
    return head;
  }
  const size_t largest = arena_largest_free(s);
  if (head->footprint <= largest) {
    s->queue.pop_front();
    return head;
  }
  if (s->lookahead > 0 && head->bypassed < MAX_BYPASS) {
    const int n = std::min<int>((int)s->queue.size(), s->lookahead + 1);
    for (int k = 1; k < n; ++k) {
      Request* r = s->queue[k];
      if (r->footprint <= largest || cache_match(s, r)) {
        head->bypassed++;
        s->st.bypasses++;
        s->queue.erase(s->queue.begin() + k);
        return r;
      }
    }
  }
  return nullptr;
}

void finish(rci_server* s, Request* r, const rci_result& res) {
  std::lock_guard<std::mutex> lk(s->mu);
  s->done[r->ticket] = res;
  s->in_flight--;
  s->st.completed++;
  if (res.status != RCI_OK && res.status != RCI_ENOCONV) s->st.failed++;
  s->cv_done.notify_all();
  s->cv_work.notify_all();
}

void run_request(Request* r, rci_grid* g, bool hit, rci_result* res) {
  rci_info info{};
  rci_status st = RCI_OK;
  if (!hit) {
    st = rci_set_design(g, r->widths.data(), (int64_t)r->widths.size(), 0);
    if (st == RCI_OK) st = rci_factor(g);
  }
  double F = 0.0;
  if (st == RCI_OK) {
    if (r->want_grad)
      st = rci_avg_intensity_grad(g, &r->obj, &r->light, &F, r->grad_out, &info);
    else
      st = rci_avg_intensity(g, &r->obj, &r->light, &F, &info);
  }
  res->status = st;
  res->value = F;
  res->refine_iters = info.refine_iters;
  res->fp64_fallback = info.fallback;
  res->simt_refactor = info.simt_refactor;
  res->rel_residual = info.rel_residual;
}

void worker(rci_server* s, int slot) {
  cudaSetDevice(s->device);
  cudaStream_t stream = s->streams[slot];
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
    if (s->queue.empty()) return;  // stopping and drained
    Request* r = pick(s);
    if (!r) {  // the head waits for memory: sleep until a request finishes or arrives
      s->st.admission_waits++;
      s->cv_done.wait(lk);
      continue;
    }
    rci_grid* g = cache_take(s, r);
    const bool hit = g != nullptr;
    rci_result res{};
    res.t_submit_us = r->t_submit;
    res.footprint = r->footprint;
    // ---- admission (under s->mu, so decisions see every allocation): carve the grid out
    // of the arena, evicting idle resident grids; if it still does not fit while other
    // requests hold memory, back to the front of the queue to wait; if nothing else holds
    // memory it never fits
    bool requeued = false;
    while (!g) {
      rci_status cs = rci_grid_alloc_with(&r->desc, stream, &s->mem, 1, &g);
      if (cs == RCI_OK) break;
      g = nullptr;
      if (cs != RCI_ENOMEM) {
        res.status = cs;
        break;
      }
      if (evict_one(s)) continue;
      if (s->running > 0) {
        s->queue.push_front(r);
        requeued = true;
        break;
      }
      res.status = RCI_ENOMEM;
      break;
    }
    if (requeued) {
      s->st.admission_waits++;
      s->cv_done.wait(lk);
      continue;
    }
    s->in_flight++;
    if (hit) s->st.cache_hits++;
    if (!g) {
      lk.unlock();
      res.t_start_us = res.t_end_us = s->now_us();
      finish(s, r, res);
      delete r;
      lk.lock();
      continue;
    }
    s->running++;
    lk.unlock();
    if (!hit) {
      rci_status is = rci_grid_init(g);
      if (is != RCI_OK) {
        res.status = is;
        lk.lock();
        rci_destroy_grid(g);
        s->running--;
        lk.unlock();
        res.t_start_us = res.t_end_us = s->now_us();
        finish(s, r, res);
        delete r;
        lk.lock();
        continue;
      }
    }
    rci_grid_rebind_stream(g, stream);
    res.t_start_us = s->now_us();
    res.cache_hit = hit ? 1 : 0;
    run_request(r, g, hit, &res);
    // nothing of this request stays queued on the slot's stream once it is retired (an
    // evaluation that failed part-way may have left work behind)
    cudaStreamSynchronize(stream);
    res.t_end_us = s->now_us();
    lk.lock();
    // ---- retire: keep the factorisation resident for a keyed request, or release it
    const bool keep =
        r->key && s->cache_cap > 0 && (res.status == RCI_OK || res.status == RCI_ENOCONV);
    if (hit) {
      for (auto& e : s->cache)
        if (e.g == g) e.pinned = false;
    } else if (keep) {
      Resident e;
      e.g = g;
      e.key = r->key;
      e.desc = r->desc;
      e.widths = r->widths;
      size_t by = 0;
      rci_grid_query(g, nullptr, nullptr, nullptr, &by);
      e.bytes = by;
      e.last_use = ++s->use_clock;
      s->cache.push_front(e);
      s->cache_bytes += by;
      while (s->cache_bytes > s->cache_cap && evict_one(s)) {
      }
    } else {
      rci_destroy_grid(g);
    }
    s->running--;
    lk.unlock();
    finish(s, r, res);
    delete r;
    lk.lock();
  }
}

rci_status copy_request(rci_server* s, const rci_request* q, Request* r) {
  r->desc = q->grid;
  r->desc.device = s->device;
  if (q->grid.n_cells < 1 || !q->widths) return RCI_EINVAL;
  r->widths.assign(q->widths, q->widths + q->grid.n_cells);
  r->obj = q->obj;
  r->light = q->light;
  if (rci_grid_footprint(&r->desc, 1, &r->footprint) != RCI_OK) return RCI_EINVAL;
  const int64_t n_src = (int64_t)q->grid.n_cells * q->grid.cell_px;
  if (q->obj.kind == RCI_OBJ_USER_ROW) {
    if (!q->obj.w_row) return RCI_EINVAL;
    r->w_row.assign(q->obj.w_row, q->obj.w_row + 2 * n_src);
    r->obj.w_row = r->w_row.data();
  }
  if (q->light.kind == RCI_LIGHT_USER_LAGS) {
    if (!q->light.lags) return RCI_EINVAL;
    r->lags.assign(q->light.lags, q->light.lags + n_src);
    r->light.lags = r->lags.data();
  }
  if (q->light.kind == RCI_LIGHT_TABULATED) {
    const int64_t nt = q->light.n_tab;
    if (!q->light.tab_theta || !q->light.tab_rho || nt < 2 || nt > 65536) return RCI_EINVAL;
    r->tab.assign(q->light.tab_theta, q->light.tab_theta + nt);
    r->tab.insert(r->tab.end(), q->light.tab_rho, q->light.tab_rho + nt);
    r->light.tab_theta = r->tab.data();
    r->light.tab_rho = r->tab.data() + nt;
  }
  r->want_grad = q->want_grad != 0;
  if (r->want_grad && !q->grad_out) return RCI_EINVAL;
  r->grad_out = q->grad_out;
  r->key = q->design_key;
  return RCI_OK;
}

}  // namespace

extern "C" {

rci_status rci_server_create(const rci_server_desc* d, rci_server** out) {
  if (!d || !out) return RCI_EINVAL;
  *out = nullptr;
  if (d->slots < 1 || d->slots > MAX_SLOTS || d->lookahead < 0) return RCI_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || d->device < 0 || d->device >= ndev)
    return RCI_ECUDA;
  if (cudaSetDevice(d->device) != cudaSuccess) return RCI_ECUDA;
  size_t bytes = d->arena_bytes;
  if (bytes == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return RCI_ECUDA;
    bytes = fr / 10 * 9;
  }
  rci_server* s = new (std::nothrow) rci_server();
  if (!s) return RCI_ENOMEM;
  s->device = d->device;
  s->slots = d->slots;
  s->lookahead = d->lookahead;
  s->cache_cap = d->cache_bytes;
  if (cudaMalloc(&s->base, bytes) != cudaSuccess) {
    delete s;
    return RCI_ENOMEM;
  }
  s->arena.reset(bytes, 256);
  s->mem.ctx = s;
  s->mem.alloc_fn = arena_alloc;
  s->mem.free_fn = arena_free;
  s->t0 = std::chrono::steady_clock::now();
  s->streams.resize(d->slots);
  for (auto& st : s->streams) {
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      st = nullptr;
      rci_server_destroy(s);
      return RCI_ECUDA;
    }
  }
  for (int k = 0; k < d->slots; ++k) s->workers.emplace_back(worker, s, k);
  *out = s;
  return RCI_OK;
}

rci_status rci_server_submit(rci_server* s, const rci_request* q, uint64_t* ticket) {
  if (!s || !q || !ticket) return RCI_EINVAL;
  Request* r = new (std::nothrow) Request();
  if (!r) return RCI_ENOMEM;
  rci_status st = copy_request(s, q, r);
  if (st != RCI_OK) {
    delete r;
    return st;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    delete r;
    return RCI_ESTATE;
  }
  r->ticket = s->next_ticket++;
  r->t_submit = s->now_us();
  s->outstanding[r->ticket] = 1;
  s->queue.push_back(r);
  s->st.submitted++;
  *ticket = r->ticket;
  s->cv_work.notify_one();
  // workers whose head request waits for memory sleep until a request finishes; a new
  // request may be one the look-ahead can start now, so they look at the queue again
  s->cv_done.notify_all();
  return RCI_OK;
}

rci_status rci_server_wait(rci_server* s, uint64_t ticket, double timeout_s, rci_result* out) {
  if (!s || !out) return RCI_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  if (!s->outstanding.count(ticket)) return RCI_EINVAL;
  auto ready = [&] { return s->done.count(ticket) > 0; };
  if (timeout_s < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
    return RCI_ETIMEOUT;
  }
  *out = s->done[ticket];
  s->done.erase(ticket);
  s->outstanding.erase(ticket);
  return RCI_OK;
}

rci_status rci_server_stats_read(rci_server* s, rci_server_stats* out) {
  if (!s || !out) return RCI_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->in_flight = s->in_flight;
  out->queued = (int32_t)s->queue.size();
  out->resident = (int32_t)s->cache.size();
  out->cache_bytes = s->cache_bytes;
  std::lock_guard<std::mutex> la(s->amu);
  out->arena_bytes = s->arena.capacity();
  out->arena_used = s->arena.used();
  out->arena_peak = s->arena.peak();
  return RCI_OK;
}

rci_status rci_server_destroy(rci_server* s) {
  if (!s) return RCI_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  cudaSetDevice(s->device);
  for (auto& e : s->cache) rci_destroy_grid(e.g);
  s->cache.clear();
  for (Request* r : s->queue) delete r;
  for (auto st : s->streams)
    if (st) cudaStreamDestroy(st);
  if (s->base) cudaFree(s->base);
  delete s;
  return RCI_OK;
}

}  // extern "C"
