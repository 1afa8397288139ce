// pgvimp_pool.h -- first-fit range allocator of the server's device and
// pinned-host pools (internal; host code only, no CUDA).
#pragma once
#include <stddef.h>

#include <algorithm>
#include <iterator>
#include <map>

namespace pgv {

constexpr size_t kGranule = 256;

inline size_t round_up(size_t v) { return (v + kGranule - 1) & ~(kGranule - 1); }

// First-fit range allocator over [0, total) with coalescing of free ranges.
class RangeAllocator {
 public:
  void reset(size_t total) {
    free_.clear();
    free_[0] = total;
    total_ = total;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = round_up(std::max<size_t>(bytes, 1));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes, next = it->first + bytes;
      free_.erase(it);
      if (rest) free_[next] = rest;
      used_ += bytes;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = round_up(std::max<size_t>(bytes, 1));
    used_ -= bytes;
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
  size_t total() const { return total_; }
  size_t used() const { return used_; }
  size_t free_ranges() const { return free_.size(); }
  size_t largest_free() const {
    size_t m = 0;
    for (const auto& kv : free_) m = std::max(m, kv.second);
    return m;
  }

 private:
  std::map<size_t, size_t> free_;
  size_t total_ = 0, used_ = 0;
};

}  // namespace pgv
