// First-fit sub-allocator of the served loop's device pool: offsets into
// [0, size), every block rounded up to kPoolAlign bytes, free blocks kept
// sorted by offset and merged with their neighbours on release. Plain C++
// (no CUDA), so the host tests compile it on its own.
#pragma once
#include <cstddef>
#include <iterator>
#include <map>

namespace stp {

constexpr size_t kPoolAlign = 256;

inline size_t pool_align_up(size_t x) { return (x + kPoolAlign - 1) & ~(kPoolAlign - 1); }

// alloc: the lowest-offset free block that fits; release: insert and merge.
class Pool {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    used_ = 0;
  }
  bool alloc(size_t n, size_t* off) {
    n = pool_align_up(n);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n;
        const size_t start = it->first + n;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += n;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = pool_align_up(n);
    used_ -= n;
    auto it = free_.emplace(off, n).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

}  // namespace stp
