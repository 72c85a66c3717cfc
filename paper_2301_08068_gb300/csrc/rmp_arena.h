// rmp_arena.h -- host-side first-fit allocator of offsets in one device memory region (the
// request server's memory budget).  Pure host code, no CUDA: blocks are multiples of 256
// bytes, free ranges are kept sorted by offset and coalesced on release.
#pragma once

#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>

namespace rmp {

class Arena {
 public:
  static constexpr size_t kAlign = 256;
  static constexpr size_t kFail = ~(size_t)0;

  explicit Arena(size_t size) : size_(size / kAlign * kAlign) {
    if (size_) free_[0] = size_;
  }

  static size_t round(size_t bytes) { return (bytes + kAlign - 1) / kAlign * kAlign; }

  // Offset of a block of at least `bytes` (first fit), or kFail.
  size_t alloc(size_t bytes) {
    bytes = round(bytes ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, rest = it->second - bytes;
      free_.erase(it);
      if (rest) free_[off + bytes] = rest;
      used_ += bytes;
      if (used_ > high_) high_ = used_;
      return off;
    }
    return kFail;
  }

  // Return a block obtained from alloc(bytes).
  void release(size_t off, size_t bytes) {
    bytes = round(bytes ? bytes : 1);
    used_ -= bytes;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + bytes == next->first) {   // merge with the next range
      bytes += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {                  // merge with the previous one
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }

  // Largest block alloc() could return now.
  size_t largest_free() const {
    size_t m = 0;
    for (const auto& f : free_) m = f.second > m ? f.second : m;
    return m;
  }

  size_t size() const { return size_; }
  size_t used() const { return used_; }
  size_t high_water() const { return high_; }
  size_t free_ranges() const { return free_.size(); }

 private:
  size_t size_;
  size_t used_ = 0, high_ = 0;
  std::map<size_t, size_t> free_;   // offset -> length
};

}  // namespace rmp
