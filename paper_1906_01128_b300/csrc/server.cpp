// server.cpp — a request loop for deep-copy-and-update requests (dc_server_*).
//
// The server owns a device pool (the HBM budget, a caller-owned buffer) and a
// mapped pinned host pool, both sub-allocated first-fit.  `nslots` worker
// threads, each with its own CUDA stream, take requests as they arrive and as
// slots and memory free up (continuous batching: the work of requests on
// different slots overlaps on the device).  A served tree stays resident (its
// plan and its device arena) until device memory is needed, then the least
// recently used idle tree is evicted.  Pinned staging is held only while a
// request runs: a request borrows it from the pinned pool for its transfers and
// returns it when it completes, so resident trees never hold host memory and
// the device budget alone decides what stays.  Requests on one key keep their
// order.
// A re-touch of a resident tree skips the deep copy: the copy back leaves the
// host and device copies identical, so only the update and the copy back run.
// With DC_SERVER_SEQUENTIAL the same requests are handled one at a time in
// arrival order with nothing kept resident (the plain per-structure path).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
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

// Best-fit allocator over [0, cap) in 256-byte units: free ranges by offset
// (for merging neighbours) and by size (for the smallest range that fits).
class RangeAlloc {
 public:
  static uint64_t extent(uint64_t bytes) { return round_up(std::max<uint64_t>(bytes, 1), 256); }
  void reset(uint64_t cap) {
    free_.clear();
    by_size_.clear();
    if (cap) add(0, cap);
  }
  bool alloc(uint64_t bytes, uint64_t* off) {
    bytes = extent(bytes);
    auto it = by_size_.lower_bound(bytes);
    if (it == by_size_.end()) return false;
    const uint64_t at = it->second, len = it->first;
    remove(at, len);
    if (len > bytes) add(at + bytes, len - bytes);
    *off = at;
    return true;
  }
  void release(uint64_t off, uint64_t bytes) {
    uint64_t lo = off, hi = off + extent(bytes);
    auto nx = free_.lower_bound(hi);
    if (nx != free_.end() && nx->first == hi) {
      hi += nx->second;
      remove(nx->first, nx->second);
    }
    auto pv = free_.lower_bound(lo);
    if (pv != free_.begin()) {
      --pv;
      if (pv->first + pv->second == lo) {
        lo = pv->first;
        remove(pv->first, pv->second);
      }
    }
    add(lo, hi - lo);
  }
  // the free range that starts at `at`, or ends at `at` (0 if none)
  uint64_t free_from(uint64_t at) const {
    auto it = free_.find(at);
    return it == free_.end() ? 0 : it->second;
  }
  uint64_t free_until(uint64_t at) const {
    auto it = free_.lower_bound(at);
    if (it == free_.begin()) return 0;
    --it;
    return it->first + it->second == at ? it->second : 0;
  }

 private:
  void add(uint64_t at, uint64_t len) {
    free_[at] = len;
    by_size_.emplace(len, at);
  }
  void remove(uint64_t at, uint64_t len) {
    free_.erase(at);
    auto r = by_size_.equal_range(len);
    for (auto it = r.first; it != r.second; ++it)
      if (it->second == at) {
        by_size_.erase(it);
        break;
      }
  }
  std::map<uint64_t, uint64_t> free_;          // offset -> length
  std::multimap<uint64_t, uint64_t> by_size_;  // length -> offset
};

struct Resident {
  dc_plan_s* plan = nullptr;
  uint64_t dev_off = 0, dev_len = 0;
  uint64_t last_use = 0;
  bool busy = false;
  bool idle_listed = false;
  std::list<uint64_t>::iterator idle_it;  // its place in the idle list (when idle_listed)
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
  std::list<uint64_t> idle;               // resident idle keys, least recently used first
  std::map<uint64_t, uint64_t> by_addr;   // device offset -> key, every resident
  uint64_t tick = 0, resident_bytes = 0;
  uint32_t pin_holders = 0;  // requests holding pinned staging
  std::mutex m;
  std::condition_variable cv;
  dc_server_stats stats{};
  dc_status first_status = DC_OK;
  std::string first_error;
};

namespace {

void unlist_idle(dc_server_s* S, Resident& r) {
  if (r.idle_listed) {
    S->idle.erase(r.idle_it);
    r.idle_listed = false;
  }
}

void list_idle(dc_server_s* S, uint64_t key, Resident& r) {
  unlist_idle(S, r);
  r.idle_it = S->idle.insert(S->idle.end(), key);
  r.idle_listed = true;
}

// Drop a resident: its device range back to the pool, its plan to `victims`.
void evict(dc_server_s* S, uint64_t key, std::vector<dc_plan_s*>* victims) {
  Resident& r = S->cache[key];
  unlist_idle(S, r);
  victims->push_back(r.plan);
  S->dalloc.release(r.dev_off, r.dev_len);
  S->by_addr.erase(r.dev_off);
  S->resident_bytes -= r.dev_len;
  S->cache.erase(key);
  S->stats.evictions++;
}

// Device memory for `dev_len` bytes.  If no free range fits, the hole is made
// around an idle resident, least recently used first: the window grows over
// the free ranges and idle residents next to it (in address order) until it
// holds dev_len bytes, and exactly the residents inside it are evicted; a seed
// whose window is closed off by busy residents before that is passed over.
// The evicted plans go to `victims`, to be destroyed once the lock is released
// (nothing of theirs is in flight: an idle resident's requests have completed).
// Called with the lock held.
bool make_room(dc_server_s* S, uint64_t dev_len, uint64_t* doff, std::vector<dc_plan_s*>* victims) {
  if (S->dalloc.alloc(dev_len, doff)) return true;
  const uint64_t need = RangeAlloc::extent(dev_len);
  auto idle_at = [&](uint64_t off, uint64_t* key, uint64_t* len) {
    auto it = S->by_addr.find(off);
    if (it == S->by_addr.end()) return false;
    const Resident& r = S->cache[it->second];
    if (r.busy) return false;
    *key = it->second;
    *len = RangeAlloc::extent(r.dev_len);
    return true;
  };
  for (uint64_t seed : S->idle) {
    const Resident& r = S->cache[seed];
    uint64_t lo = r.dev_off, hi = lo + RangeAlloc::extent(r.dev_len);
    std::vector<uint64_t> take{seed};
    bool open_hi = true, open_lo = true;
    while (hi - lo < need && (open_hi || open_lo)) {
      if (open_hi) {  // grow up: a free range, else an idle resident, starting at hi
        uint64_t k, len = S->dalloc.free_from(hi);
        if (len) {
          hi += len;
        } else if (hi < S->dev_bytes && idle_at(hi, &k, &len)) {
          take.push_back(k);
          hi += len;
        } else {
          open_hi = false;
        }
        continue;
      }
      uint64_t len = S->dalloc.free_until(lo);  // grow down: a free range, else an idle resident, ending at lo
      if (len) {
        lo -= len;
        continue;
      }
      auto it = S->by_addr.lower_bound(lo);
      if (it != S->by_addr.begin()) {
        --it;
        uint64_t k;
        if (idle_at(it->first, &k, &len) && it->first + len == lo) {
          take.push_back(k);
          lo = it->first;
          continue;
        }
      }
      open_lo = false;
    }
    if (hi - lo < need) continue;
    for (uint64_t k : take) evict(S, k, victims);
    return S->dalloc.alloc(dev_len, doff);
  }
  return false;
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
      unlist_idle(S, r);  // a busy resident is never evicted
      dc_plan_s* p = r.plan;  // read under the lock: other slots may grow the map
      uint64_t dev_off = r.dev_off, dev_len = r.dev_len;
      lk.unlock();
      dc_status st = DC_OK;
      std::vector<dc_plan_s*> victims;
      if (!resident) {  // plan outside the lock, then admit by device memory
        st = dc_plan(&S->schema, rq.host_root, &p);
        if (!st) {
          const uint64_t dl = p->L.total;
          uint64_t doff = 0;
          bool admitted = false;
          lk.lock();
          for (;;) {
            if (make_room(S, dl, &doff, &victims)) {
              admitted = true;
              break;
            }
            bool others_busy = false;
            for (auto& kv : S->cache)
              if (kv.second.busy && kv.first != rq.key && kv.second.plan) others_busy = true;
            if (!others_busy) break;  // nothing held elsewhere will be freed: larger than the budget
            S->cv.wait(lk);          // wait for another slot to finish
          }
          if (admitted) {
            Resident& rr = S->cache[rq.key];
            rr.plan = p;
            rr.dev_off = dev_off = doff;
            rr.dev_len = dev_len = dl;
            S->by_addr[doff] = rq.key;
            S->resident_bytes += dl;
            S->stats.peak_resident_bytes = std::max(S->stats.peak_resident_bytes, S->resident_bytes);
          }
          lk.unlock();
          if (!admitted) {
            dc_plan_destroy(p);
            p = nullptr;
            st = fail(DC_EBUDGET, "request %llu needs %llu device bytes: more than the budget",
                      (unsigned long long)pick, (unsigned long long)dl);
          }
        }
      }
      for (dc_plan_s* v : victims) dc_plan_destroy(v);
      // pinned staging for this request's transfers, returned when it completes
      uint64_t poff = 0, plen = 0;
      if (!st && p) {
        const uint64_t need = pinned_need(p);
        bool got = false;
        lk.lock();
        for (;;) {
          if (S->palloc.alloc(need, &poff)) {
            got = true;
            S->pin_holders++;
            break;
          }
          if (!S->pin_holders) break;  // nothing will be returned: larger than the pinned pool
          S->cv.wait(lk);              // another request returns its staging when it completes
        }
        lk.unlock();
        if (got)
          plen = need;
        else
          st = fail(DC_EBUDGET, "request %llu needs %llu bytes of pinned staging: more than the pool",
                    (unsigned long long)pick, (unsigned long long)need);
      }
      uint64_t h2d = 0, d2h = 0;
      if (!st && p) {
        if (!resident) {
          st = bind_borrowed(p, S->dev + dev_off, dev_len, S->pin + poff, S->pin_dev + poff, cs);
        } else {
          st = lend_pinned(p, S->pin + poff, S->pin_dev + poff);
        }
      }
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
      if (plen) {  // the request's transfers are complete
        S->palloc.release(poff, plen);
        S->pin_holders--;
      }
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
      dc_plan_s* drop = nullptr;
      if ((st || (S->flags & DC_SERVER_SEQUENTIAL)) && done.plan) {  // nothing kept resident
        drop = done.plan;
        S->dalloc.release(done.dev_off, done.dev_len);
        S->by_addr.erase(done.dev_off);
        S->resident_bytes -= done.dev_len;
        done.plan = nullptr;
      }
      if (done.plan)
        list_idle(S, rq.key, done);
      else
        S->cache.erase(rq.key);
      finished++;
      S->cv.notify_all();
      if (drop) {
        lk.unlock();
        dc_plan_destroy(drop);
        lk.lock();
      }
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
