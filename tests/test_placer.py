"""The executor's arena placement (csrc/placer.hpp), on the host: against
the plain best-fit definition -- take the smallest free range that holds
the 256-byte rounded size, the lowest address among equal sizes, else grow
the top (merging a free range that ends there); on release merge with free
neighbours, keeping per stream the later instruction -- over random
allocation/release sequences, every returned offset, inherited dependency,
the top and the whole free list must agree after every step."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DRIVER = r"""
#include <cstdio>
#include <random>
#include <vector>
#include "placer.hpp"

struct R { long long off, size; int dep[3]; };
struct Ref {                        // the definition, over a list sorted by address
  std::vector<R> fr;
  long long top = 0;
  static long long rnd(long long s) { return (s + 255) / 256 * 256; }
  long long alloc(long long size, int dep[3]) {
    size = rnd(size);
    int best = -1;
    for (int i = 0; i < (int)fr.size(); ++i)
      if (fr[i].size >= size && (best < 0 || fr[i].size < fr[best].size)) best = i;
    if (best < 0) {
      long long off = top;
      dep[0] = dep[1] = dep[2] = -1;
      if (!fr.empty() && fr.back().off + fr.back().size == top) {
        off = fr.back().off;
        for (int s = 0; s < 3; ++s) dep[s] = fr.back().dep[s];
        fr.pop_back();
      }
      top = off + size;
      return off;
    }
    R b = fr[best];
    fr.erase(fr.begin() + best);
    for (int s = 0; s < 3; ++s) dep[s] = b.dep[s];
    if (b.size > size) {
      R rest{b.off + size, b.size - size, {b.dep[0], b.dep[1], b.dep[2]}};
      fr.insert(fr.begin() + best, rest);
    }
    return b.off;
  }
  void release(long long off, long long size, const int dep[3]) {
    size = rnd(size);
    R s{off, size, {dep[0], dep[1], dep[2]}};
    int i = 0;
    while (i < (int)fr.size() && fr[i].off < off) ++i;
    if (i < (int)fr.size() && off + size == fr[i].off) {
      s.size += fr[i].size;
      for (int k = 0; k < 3; ++k) s.dep[k] = std::max(s.dep[k], fr[i].dep[k]);
      fr.erase(fr.begin() + i);
    }
    if (i > 0 && fr[i - 1].off + fr[i - 1].size == off) {
      fr[i - 1].size += s.size;
      for (int k = 0; k < 3; ++k) fr[i - 1].dep[k] = std::max(fr[i - 1].dep[k], s.dep[k]);
      return;
    }
    fr.insert(fr.begin() + i, s);
  }
};

int main() {
  for (int seed = 0; seed < 20; ++seed) {
    std::mt19937_64 rng(seed);
    lqc::Placer p;
    Ref r;
    struct Live { long long off, size; };
    std::vector<Live> live;
    int clock[3] = {0, 0, 0};
    for (int step = 0; step < 10000; ++step) {
      const bool grow = live.empty() || rng() % 100 < 55;
      if (grow) {
        const long long choice[5] = {256, 4096, 65536, 1 << 20, 3 << 20};
        long long size = choice[rng() % 5] - (long long)(rng() % 300);
        if (size < 1) size = 1;
        int d1[3], d2[3];
        const long long o1 = p.alloc(size, d1), o2 = r.alloc(size, d2);
        if (o1 != o2 || d1[0] != d2[0] || d1[1] != d2[1] || d1[2] != d2[2]) {
          printf("alloc mismatch seed %d step %d: %lld vs %lld\n", seed, step, o1, o2);
          return 1;
        }
        live.push_back({o1, size});
      } else {
        const size_t k = rng() % live.size();
        int dep[3];
        for (int s = 0; s < 3; ++s) dep[s] = (rng() % 2) ? ++clock[s] : -1;
        p.release(live[k].off, live[k].size, dep);
        r.release(live[k].off, live[k].size, dep);
        live.erase(live.begin() + k);
      }
      if (p.top != r.top || p.free_.size() != r.fr.size() || p.by_size.size() != r.fr.size()) {
        printf("state mismatch seed %d step %d\n", seed, step);
        return 1;
      }
      size_t i = 0;
      for (auto& kv : p.free_) {
        const R& q = r.fr[i++];
        if (kv.first != q.off || kv.second.size != q.size || kv.second.dep[0] != q.dep[0] ||
            kv.second.dep[1] != q.dep[1] || kv.second.dep[2] != q.dep[2] ||
            !p.by_size.count({kv.second.size, kv.first})) {
          printf("free list mismatch seed %d step %d\n", seed, step);
          return 1;
        }
      }
    }
  }
  printf("ok\n");
  return 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="no C++ compiler")
def test_placer_matches_best_fit_definition(tmp_path):
    src = tmp_path / "placer_test.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "placer_test"
    r = subprocess.run(["g++", "-std=c++17", "-O2", "-I",
                        os.path.join(ROOT, "paper_2511_02257_b300", "csrc"), str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
