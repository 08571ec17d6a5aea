// Offset allocator for one contiguous range of device memory (host-side bookkeeping only).
//
// The serving runtime takes one large device allocation when it starts and carves every
// grid out of it with this class, so that admitting and retiring requests never calls
// cudaMalloc / cudaFree (cudaFree synchronises the whole device and would stall the
// evaluations running on the other streams).
//
// First fit over a free list ordered by offset; blocks are rounded up to `align` bytes;
// a freed block merges with free neighbours.  Not thread-safe: callers serialise.
#pragma once

#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>
#include <unordered_map>

class Arena {
 public:
  explicit Arena(size_t capacity = 0, size_t align = 256) { reset(capacity, align); }

  void reset(size_t capacity, size_t align = 256) {
    align_ = align ? align : 1;
    cap_ = capacity / align_ * align_;
    free_.clear();
    live_.clear();
    if (cap_) free_[0] = cap_;
    used_ = peak_ = 0;
  }

  // Lowest-offset free block that holds `bytes` (rounded up); false if none does.
  bool alloc(size_t bytes, size_t* off) {
    const size_t b = round(bytes ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < b) continue;
      const size_t o = it->first, rest = it->second - b;
      free_.erase(it);
      if (rest) free_[o + b] = rest;
      live_[o] = b;
      used_ += b;
      if (used_ > peak_) peak_ = used_;
      *off = o;
      return true;
    }
    return false;
  }

  // Release a block returned by alloc; false (and no change) for an unknown offset.
  bool release(size_t off) {
    auto lv = live_.find(off);
    if (lv == live_.end()) return false;
    size_t o = off, b = lv->second;
    live_.erase(lv);
    used_ -= b;
    auto next = free_.lower_bound(o);
    if (next != free_.end() && o + b == next->first) {
      b += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == o) {
        prev->second += b;
        return true;
      }
    }
    free_[o] = b;
    return true;
  }

  size_t round(size_t b) const { return (b + align_ - 1) / align_ * align_; }
  size_t capacity() const { return cap_; }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }
  size_t live_blocks() const { return live_.size(); }
  size_t free_blocks() const { return free_.size(); }
  size_t largest_free() const {
    size_t m = 0;
    for (const auto& f : free_) m = f.second > m ? f.second : m;
    return m;
  }

 private:
  size_t align_ = 256, cap_ = 0, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;            // offset -> bytes, disjoint, non-adjacent
  std::unordered_map<size_t, size_t> live_;  // offset -> bytes
};
