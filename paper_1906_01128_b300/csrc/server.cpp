// server.cpp — a request loop for deep-copy-and-update requests (dc_server_*).
//
// The server owns a device pool (the HBM budget, a caller-owned buffer) and a
// mapped pinned host pool, both sub-allocated first-fit.  `nslots` worker
// threads, each with its own CUDA stream, take requests as they arrive and as
// slots and memory free up (continuous batching: the work of requests on
// different slots overlaps on the device).  A served tree stays resident (its
// plan, arena and pinned staging) until memory is needed, then the least
// recently used idle tree is evicted.  Requests on one key keep their order.
// A re-touch of a resident tree skips the deep copy: the copy back leaves the
// host and device copies identical, so only the update and the copy back run.
// With DC_SERVER_SEQUENTIAL the same requests are handled one at a time in
// arrival order with nothing kept resident (the plain per-structure path).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "internal.hpp"

using namespace dc;
using clk = std::chrono::steady_clock;

namespace {

// First-fit allocator over [0, cap) in 256-byte units.
class RangeAlloc {
 public:
  void reset(uint64_t cap) {
    free_.clear();
    if (cap) free_[0] = cap;
  }
  bool alloc(uint64_t bytes, uint64_t* off) {
    bytes = round_up(std::max<uint64_t>(bytes, 1), 256);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const uint64_t rest = it->second - bytes, at = it->first + bytes;
      free_.erase(it);
      if (rest) free_[at] = rest;
      return true;
    }
    return false;
  }
  void release(uint64_t off, uint64_t bytes) {
    bytes = round_up(std::max<uint64_t>(bytes, 1), 256);
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
  std::map<uint64_t, uint64_t> free_;
};

struct Resident {
  dc_plan_s* plan = nullptr;
  uint64_t dev_off = 0, dev_len = 0, pin_off = 0, pin_len = 0;
  uint64_t last_use = 0;
  bool busy = false;
};

}  // namespace

struct dc_server_s {
  std::vector<dc_type> types;
  std::vector<std::vector<dc_field>> fields;
  dc_schema schema{};
  uint8_t* dev = nullptr;
  uint64_t dev_bytes = 0;
  uint8_t* pin = nullptr;
  uint8_t* pin_dev = nullptr;
  uint64_t pin_bytes = 0;
  RangeAlloc dalloc, palloc;
  uint32_t nslots = 1, flags = 0;
  std::vector<cudaStream_t> streams;
  std::unordered_map<uint64_t, Resident> cache;
  uint64_t tick = 0, resident_bytes = 0;
  std::mutex m;
  std::condition_variable cv;
  dc_server_stats stats{};
  dc_status first_status = DC_OK;
  std::string first_error;
};

namespace {

// Free memory for `dev_len` + `pin_len` bytes by evicting idle residents, least
// recently used first.  Called with the lock held.
bool make_room(dc_server_s* S, uint64_t dev_len, uint64_t pin_len, uint64_t* doff, uint64_t* poff) {
  for (;;) {
    uint64_t d, q;
    if (S->dalloc.alloc(dev_len, &d)) {
      if (S->palloc.alloc(pin_len, &q)) {
        *doff = d;
        *poff = q;
        return true;
      }
      S->dalloc.release(d, dev_len);
    }
    uint64_t victim = 0, oldest = ~0ull;
    bool found = false;
    for (auto& kv : S->cache)
      if (!kv.second.busy && kv.second.plan && kv.second.last_use < oldest) {
        oldest = kv.second.last_use;
        victim = kv.first;
        found = true;
      }
    if (!found) return false;
    Resident& r = S->cache[victim];
    dc_plan_destroy(r.plan);
    S->dalloc.release(r.dev_off, r.dev_len);
    S->palloc.release(r.pin_off, r.pin_len);
    S->resident_bytes -= r.dev_len;
    S->cache.erase(victim);
    S->stats.evictions++;
  }
}

void note_error(dc_server_s* S, dc_status st) {
  if (S->first_status == DC_OK) {
    S->first_status = st;
    S->first_error = last_error();
  }
  S->stats.failed++;
}

}  // namespace

extern "C" {

dc_status dc_server_create(const dc_schema* schema, void* dev_pool, uint64_t dev_bytes, uint64_t pinned_bytes,
                           uint32_t nslots, uint32_t flags, dc_server_t* out) {
  if (!out) return fail(DC_EINVAL, "out is NULL");
  *out = nullptr;
  SchemaCopy check;
  dc_status st = copy_schema(schema, &check);
  if (st) return st;
  if (!dev_pool || (uintptr_t)dev_pool % 256) return fail(DC_EINVAL, "device pool must be 256-byte aligned");
  if (nslots == 0 || nslots > 64) return fail(DC_EINVAL, "slots must be in [1, 64]");
  dc_server_s* S = new (std::nothrow) dc_server_s;
  if (!S) return fail(DC_ENOMEM, "out of host memory");
  S->types.assign(schema->types, schema->types + schema->ntypes);
  S->fields.resize(schema->ntypes);
  for (uint32_t t = 0; t < schema->ntypes; t++) {
    S->fields[t].assign(schema->types[t].fields, schema->types[t].fields + schema->types[t].nfields);
    S->types[t].fields = S->fields[t].data();
  }
  S->schema = dc_schema{schema->ntypes, schema->root_type, S->types.data()};
  S->dev = static_cast<uint8_t*>(dev_pool);
  S->dev_bytes = dev_bytes / 256 * 256;
  S->pin_bytes = round_up(std::max<uint64_t>(pinned_bytes, 256), 256);
  S->flags = flags;
  S->nslots = (flags & DC_SERVER_SEQUENTIAL) ? 1 : nslots;
  cudaError_t e = host_alloc((void**)&S->pin, S->pin_bytes, cudaHostAllocMapped);
  if (e != cudaSuccess) {
    delete S;
    return fail(DC_ENOMEM, "pinned pool of %llu bytes: %s", (unsigned long long)pinned_bytes, cudaGetErrorString(e));
  }
  if ((e = cudaHostGetDevicePointer((void**)&S->pin_dev, S->pin, 0)) != cudaSuccess) {
    cudaFreeHost(S->pin);
    delete S;
    return cuda_fail(e, "cudaHostGetDevicePointer");
  }
  S->dalloc.reset(S->dev_bytes);
  S->palloc.reset(S->pin_bytes);
  S->streams.resize(S->nslots);
  for (auto& st2 : S->streams)
    if ((e = cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking)) != cudaSuccess) {
      dc_server_destroy(S);
      return cuda_fail(e, "cudaStreamCreateWithFlags");
    }
  *out = S;
  return DC_OK;
}

dc_status dc_server_run(dc_server_t S, const dc_request* reqs, uint64_t n, const dc_op* op, double* latency_ms) {
  if (!S || (n && (!reqs || !op))) return fail(DC_EINVAL, "NULL argument");
  std::deque<uint64_t> pending;  // arrived, not taken; arrival order
  uint64_t arrived = 0, finished = 0;
  bool stop = false;
  const auto start = clk::now();
  auto at = [&](uint64_t i) {
    return start + std::chrono::duration_cast<clk::duration>(std::chrono::duration<double>(reqs[i].arrival_s));
  };

  auto worker = [&](uint32_t slot) {
    cudaStream_t cs = S->streams[slot];
    std::unique_lock<std::mutex> lk(S->m);
    for (;;) {
      // the first pending request whose key is idle (earlier requests of a busy key stay first)
      uint64_t pick = ~0ull;
      std::unordered_set<uint64_t> blocked;
      for (auto it = pending.begin(); it != pending.end(); ++it) {
        const uint64_t k = reqs[*it].key;
        if (blocked.count(k)) continue;
        auto c = S->cache.find(k);
        if (c != S->cache.end() && c->second.busy) {
          blocked.insert(k);
          continue;
        }
        pick = *it;
        pending.erase(it);
        break;
      }
      if (pick == ~0ull) {
        if (stop) return;
        S->cv.wait(lk);
        continue;
      }
      const dc_request& rq = reqs[pick];
      Resident& r = S->cache[rq.key];
      const bool resident = r.plan != nullptr;
      r.busy = true;
      lk.unlock();
      dc_status st = DC_OK;
      bool admitted = resident;
      if (!resident) {  // plan outside the lock, then admit by memory
        dc_plan_s* p = nullptr;
        st = dc_plan(&S->schema, rq.host_root, &p);
        if (!st) {
          const uint64_t dl = p->L.total, pl = pinned_need(p);
          lk.lock();
          uint64_t doff = 0, poff = 0;
          for (;;) {
            if (make_room(S, dl, pl, &doff, &poff)) {
              admitted = true;
              break;
            }
            bool others_busy = false;
            for (auto& kv : S->cache)
              if (kv.second.busy && kv.first != rq.key && kv.second.plan) others_busy = true;
            if (!others_busy) break;  // nothing held elsewhere will be freed: larger than the budget
            S->cv.wait(lk);          // wait for another slot to finish
          }
          Resident& rr = S->cache[rq.key];
          if (admitted) {
            rr.plan = p;
            rr.dev_off = doff;
            rr.dev_len = dl;
            rr.pin_off = poff;
            rr.pin_len = pl;
            S->resident_bytes += dl;
            S->stats.peak_resident_bytes = std::max(S->stats.peak_resident_bytes, S->resident_bytes);
          }
          lk.unlock();
          if (admitted) {
            st = bind_borrowed(p, S->dev + doff, dl, S->pin + poff, S->pin_dev + poff, cs);
          } else {
            dc_plan_destroy(p);
            st = fail(DC_EBUDGET, "request %llu needs %llu device bytes: more than the budget",
                      (unsigned long long)pick, (unsigned long long)dl);
          }
        }
      }
      lk.lock();
      Resident& rr = S->cache[rq.key];
      dc_plan_s* p = rr.plan;
      lk.unlock();
      uint64_t h2d = 0, d2h = 0;
      if (!st && p) {
        if (resident && rq.retouch) {  // the device copy equals the host tree: update and copy back only
          st = dc_update_leaves(p, op, cs);
          if (!st) st = dc_copy_back(p, 0, cs);
        } else {
          st = dc_roundtrip(p, op, cs);
          h2d = p->payload;
        }
        if (!st)
          for (uint32_t b : *p->written) d2h += p->blocks[b].bytes;
      }
      const double lat = std::chrono::duration<double, std::milli>(clk::now() - at(pick)).count();
      lk.lock();
      if (latency_ms) latency_ms[pick] = st ? -1.0 : lat;
      if (st) {
        note_error(S, st);
      } else {
        S->stats.served++;
        S->stats.h2d_bytes += h2d;
        S->stats.d2h_bytes += d2h;
        if (resident) S->stats.resident_hits++;
      }
      Resident& done = S->cache[rq.key];
      done.busy = false;
      done.last_use = ++S->tick;
      if ((st || (S->flags & DC_SERVER_SEQUENTIAL)) && done.plan) {  // nothing kept resident
        dc_plan_destroy(done.plan);
        S->dalloc.release(done.dev_off, done.dev_len);
        S->palloc.release(done.pin_off, done.pin_len);
        S->resident_bytes -= done.dev_len;
        done.plan = nullptr;
      }
      if (!done.plan) S->cache.erase(rq.key);
      finished++;
      S->cv.notify_all();
    }
  };

  std::vector<std::thread> ws;
  for (uint32_t i = 0; i < S->nslots; i++) ws.emplace_back(worker, i);
  {  // inject the requests at their arrival times
    std::unique_lock<std::mutex> lk(S->m);
    while (arrived < n) {
      const auto now = clk::now();
      while (arrived < n && at(arrived) <= now) {
        pending.push_back(arrived++);
        S->cv.notify_all();
      }
      if (arrived < n) S->cv.wait_until(lk, at(arrived));
    }
    while (finished < n) S->cv.wait(lk);
    stop = true;
    S->cv.notify_all();
  }
  for (auto& w : ws) w.join();
  S->stats.wall_s += std::chrono::duration<double>(clk::now() - start).count();
  if (S->first_status) return fail(S->first_status, "%s", S->first_error.c_str());
  return DC_OK;
}

dc_status dc_server_stats_get(dc_server_t S, dc_server_stats* out) {
  if (!S || !out) return fail(DC_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> g(S->m);
  *out = S->stats;
  out->resident_bytes = S->resident_bytes;
  return DC_OK;
}

dc_status dc_server_destroy(dc_server_t S) {
  if (!S) return DC_OK;
  for (auto& kv : S->cache)
    if (kv.second.plan) dc_plan_destroy(kv.second.plan);
  for (auto st : S->streams)
    if (st) cudaStreamDestroy(st);
  if (S->pin) cudaFreeHost(S->pin);
  delete S;
  return DC_OK;
}

}  // extern "C"
