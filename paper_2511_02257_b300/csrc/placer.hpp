// Offline placement of a plan's tensors in one device (or pinned host)
// arena: best-fit with coalescing, growing the high-water mark on demand.
// Every free range remembers, per stream, the last instruction that touched
// its bytes, so that a tensor placed there can wait for exactly that work.
#pragma once

#include <cstdint>
#include <iterator>
#include <map>
#include <set>
#include <utility>

namespace lqc {

struct Seg {
  int64_t size;
  int32_t dep[3];     // last instruction per stream that touched the bytes
};

// alloc() takes the smallest free range that holds the (256-byte rounded)
// size, the lowest address among equal sizes; with none, it extends the top
// (merging a free range that ends there).  A (size, offset) index finds the
// range in O(log n).  release() coalesces with free neighbours, keeping the
// later instruction of each stream.
struct Placer {
  std::map<int64_t, Seg> free_;                  // offset -> free range
  std::set<std::pair<int64_t, int64_t>> by_size;  // (size, offset) of free_
  int64_t top = 0;

  static int64_t rounded(int64_t size) { return (size + 255) & ~int64_t(255); }
  static int32_t mx(int32_t a, int32_t b) { return a > b ? a : b; }

  void put(int64_t off, const Seg& s) {
    free_[off] = s;
    by_size.insert({s.size, off});
  }
  void take(std::map<int64_t, Seg>::iterator it) {
    by_size.erase({it->second.size, it->first});
    free_.erase(it);
  }

  int64_t alloc(int64_t size, int32_t dep[3]) {
    size = rounded(size);
    auto bs = by_size.lower_bound({size, INT64_MIN});
    if (bs == by_size.end()) {
      int64_t off = top;
      dep[0] = dep[1] = dep[2] = -1;
      if (!free_.empty()) {
        auto last = std::prev(free_.end());
        if (last->first + last->second.size == top) {
          off = last->first;
          for (int s = 0; s < 3; ++s) dep[s] = last->second.dep[s];
          take(last);
        }
      }
      top = off + size;
      return off;
    }
    auto it = free_.find(bs->second);
    const int64_t off = it->first;
    const Seg sg = it->second;
    take(it);
    for (int s = 0; s < 3; ++s) dep[s] = sg.dep[s];
    if (sg.size > size) put(off + size, Seg{sg.size - size, {sg.dep[0], sg.dep[1], sg.dep[2]}});
    return off;
  }

  void release(int64_t off, int64_t size, const int32_t dep[3]) {
    size = rounded(size);
    Seg s{size, {dep[0], dep[1], dep[2]}};
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && off + size == nx->first) {
      s.size += nx->second.size;
      for (int k = 0; k < 3; ++k) s.dep[k] = mx(s.dep[k], nx->second.dep[k]);
      take(nx);
    }
    auto it = free_.lower_bound(off);
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second.size == off) {
        Seg merged = pv->second;
        merged.size += s.size;
        for (int k = 0; k < 3; ++k) merged.dep[k] = mx(merged.dep[k], s.dep[k]);
        const int64_t poff = pv->first;
        take(pv);
        put(poff, merged);
        return;
      }
    }
    put(off, s);
  }
};

}  // namespace lqc
