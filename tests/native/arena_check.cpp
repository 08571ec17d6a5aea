// Randomised check of the serving arena (first-fit, coalescing offset allocator) against a
// byte-ownership model: no two live blocks overlap, every block lies inside the capacity,
// first fit returns the lowest offset that can hold the request, and freeing everything
// leaves one free block of the whole capacity.  Prints "arena ok" on success.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <vector>

#include "../../paper_2207_10701_gb300/csrc/arena.h"

static int fail(const char* what, long a, long b) {
  std::printf("arena FAIL: %s (%ld, %ld)\n", what, a, b);
  return 1;
}

int main() {
  const size_t align = 256, cap = 1 << 20;
  for (int seed = 0; seed < 20; ++seed) {
    std::mt19937_64 rng(seed);
    Arena a(cap, align);
    std::vector<int> owner(cap / align, -1);  // model: which block owns each granule
    std::map<size_t, size_t> live;             // offset -> rounded bytes
    int next_id = 0;
    std::map<size_t, int> id_of;
    for (int step = 0; step < 4000; ++step) {
      const bool do_alloc = live.empty() || (rng() % 100) < 55;
      if (do_alloc) {
        const size_t want = 1 + rng() % (cap / 16);
        const size_t b = (want + align - 1) / align * align, g = b / align;
        // model first fit: lowest granule run of length g that is free
        long expect = -1;
        for (size_t s = 0, run = 0; s < owner.size(); ++s) {
          run = owner[s] < 0 ? run + 1 : 0;
          if (run == g) { expect = (long)(s + 1 - g); break; }
        }
        size_t off = 0;
        const bool ok = a.alloc(want, &off);
        if (ok != (expect >= 0)) return fail("alloc success differs from model", ok, expect);
        if (!ok) continue;
        if ((long)(off / align) != expect) return fail("not first fit", (long)off, expect * (long)align);
        if (off % align || off + b > cap) return fail("block outside capacity", (long)off, (long)b);
        for (size_t k = off / align; k < off / align + g; ++k) {
          if (owner[k] >= 0) return fail("overlap", (long)k, owner[k]);
          owner[k] = next_id;
        }
        live[off] = b;
        id_of[off] = next_id++;
      } else {
        auto it = live.begin();
        std::advance(it, rng() % live.size());
        if (!a.release(it->first)) return fail("release of a live block refused", (long)it->first, 0);
        for (size_t k = it->first / align; k < (it->first + it->second) / align; ++k) owner[k] = -1;
        id_of.erase(it->first);
        live.erase(it);
      }
      size_t used = 0;
      for (auto& l : live) used += l.second;
      if (used != a.used()) return fail("used bytes differ", (long)used, (long)a.used());
    }
    if (a.release(cap + 7)) return fail("release of an unknown offset accepted", 0, 0);
    for (auto& l : live) a.release(l.first);
    if (a.used() != 0 || a.free_blocks() != 1 || a.largest_free() != cap)
      return fail("free list not coalesced after releasing everything", (long)a.free_blocks(),
                  (long)a.largest_free());
  }
  std::printf("arena ok\n");
  return 0;
}
