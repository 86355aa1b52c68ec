// First-fit range allocator used by the serving engine for its device pool.
// Host-only C++ (no CUDA), so that it can be tested on its own.
#pragma once

#include <stdint.h>

#include <iterator>
#include <map>

namespace velo {

// Hands out [offset, offset + n) ranges of a pool of `size` bytes: the
// lowest-addressed free range that fits (first fit).  A released range merges
// with free neighbours, so the free list never holds two adjacent ranges.
class Pool {
 public:
  void init(uint64_t size) {
    free_.clear();
    if (size) free_[0] = size;
    size_ = size;
    used_ = peak_ = 0;
  }
  bool alloc(uint64_t n, uint64_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      *off = it->first;
      const uint64_t rest = it->second - n;
      const uint64_t at = it->first + n;
      free_.erase(it);
      if (rest) free_[at] = rest;
      used_ += n;
      if (used_ > peak_) peak_ = used_;
      return true;
    }
    return false;
  }
  void release(uint64_t off, uint64_t n) {
    used_ -= n;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + n == next->first) {
      n += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += n;
        return;
      }
    }
    free_[off] = n;
  }
  uint64_t size() const { return size_; }
  uint64_t used() const { return used_; }
  uint64_t peak() const { return peak_; }
  template <class F>
  void for_each_free(F f) const {
    for (const auto& r : free_) f(r.first, r.second);
  }
  uint64_t largest_free() const {
    uint64_t m = 0;
    for (const auto& f : free_) m = f.second > m ? f.second : m;
    return m;
  }

 private:
  std::map<uint64_t, uint64_t> free_;
  uint64_t size_ = 0, used_ = 0, peak_ = 0;
};

}  // namespace velo
