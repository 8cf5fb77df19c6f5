// partition.cpp — assigning independent trees to GPUs by bytes (dc_partition_by_bytes).
//
// The batched and served forms shard by tree with no exchange between GPUs,
// so the only multi-GPU decision is which trees each rank takes.  Greedy
// LPT (longest processing time first): trees in decreasing size, each to
// the part with the fewest bytes so far, so that no part exceeds the mean by
// more than one tree.  Ties go to the lower index, which makes the result a
// function of the input alone: every rank computes the same assignment.
#include <algorithm>
#include <numeric>
#include <queue>
#include <vector>

#include "internal.hpp"

using namespace dc;

extern "C" dc_status dc_partition_by_bytes(const uint64_t* bytes, uint64_t n, uint32_t nparts, uint32_t* part_of,
                                           uint64_t* part_bytes) {
  if (nparts == 0) return fail(DC_EINVAL, "nparts must be at least 1");
  if (n && (!bytes || !part_of)) return fail(DC_EINVAL, "NULL argument");
  std::vector<uint64_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](uint64_t a, uint64_t b) { return bytes[a] > bytes[b]; });
  // min-heap of (load, part): the least-loaded part first, the lower index on ties
  using Load = std::pair<uint64_t, uint32_t>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
  for (uint32_t k = 0; k < nparts; k++) heap.push({0, k});
  std::vector<uint64_t> load(nparts, 0);
  for (uint64_t i : order) {
    Load l = heap.top();
    heap.pop();
    if (UINT64_MAX - l.first < bytes[i]) return fail(DC_EINVAL, "byte total overflows");
    part_of[i] = l.second;
    l.first += bytes[i];
    load[l.second] = l.first;
    heap.push(l);
  }
  if (part_bytes) std::copy(load.begin(), load.end(), part_bytes);
  return DC_OK;
}
