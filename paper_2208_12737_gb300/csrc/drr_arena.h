// Offset arena: a thread-safe first-fit allocator over [0, capacity) with
// alignment and coalescing of freed neighbours.  The serving loop carves every
// admitted request's device and pinned-host buffers out of two fixed regions
// with it, so admission is decided by free bytes in the region (the budget),
// never by the driver's free memory.  Pure host code: no CUDA calls.
#pragma once

#include <cstddef>
#include <cstdint>
#include <map>
#include <mutex>

namespace drr {

class OffsetArena {
 public:
  OffsetArena(size_t capacity, size_t align) : capacity_(capacity), align_(align ? align : 1) {
    if (capacity_ > 0) free_[0] = capacity_;
  }

  // Returns true and the block offset, or false if no free run is large enough.
  bool alloc(size_t bytes, size_t* offset) {
    std::lock_guard<std::mutex> lk(mu_);
    const size_t need = round_up(bytes ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < need) continue;
      const size_t off = it->first, len = it->second;
      free_.erase(it);
      if (len > need) free_[off + need] = len - need;
      used_[off] = need;
      in_use_ += need;
      *offset = off;
      return true;
    }
    return false;
  }

  // Frees a block returned by alloc(); returns false for an unknown offset.
  bool release(size_t offset) {
    std::lock_guard<std::mutex> lk(mu_);
    auto u = used_.find(offset);
    if (u == used_.end()) return false;
    size_t off = u->first, len = u->second;
    used_.erase(u);
    in_use_ -= len;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + len == next->first) {
      len += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += len;
        return true;
      }
    }
    free_[off] = len;
    return true;
  }

  size_t capacity() const { return capacity_; }
  size_t in_use() {
    std::lock_guard<std::mutex> lk(mu_);
    return in_use_;
  }
  size_t largest_free() {
    std::lock_guard<std::mutex> lk(mu_);
    size_t m = 0;
    for (auto& kv : free_) m = kv.second > m ? kv.second : m;
    return m;
  }
  size_t rounded(size_t bytes) const { return round_up(bytes ? bytes : 1); }

 private:
  size_t round_up(size_t b) const { return (b + align_ - 1) / align_ * align_; }
  size_t capacity_, align_;
  size_t in_use_ = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  std::map<size_t, size_t> used_;  // offset -> length
  std::mutex mu_;
};

}  // namespace drr
