// First-fit allocator over a fixed range of offsets (the serving loop's
// device arena; it hands out offsets only and touches no memory). Free space
// is a map from offset to length with no two ranges adjacent: a release
// merges with its neighbours, so freeing everything restores one range.
#pragma once

#include <cstddef>
#include <iterator>
#include <map>

namespace fovea {

class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
  }
  // Lowest-offset free range of at least n: its first n units.
  bool alloc(size_t n, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n, start = it->first + n;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
  }
  // Return [off, off + n), which must have come from alloc and not been
  // released since.
  void release(size_t off, size_t n) {
    auto it = free_.emplace(off, n).first;
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
  const std::map<size_t, size_t>& free_ranges() const { return free_; }

 private:
  std::map<size_t, size_t> free_;
};

}  // namespace fovea
