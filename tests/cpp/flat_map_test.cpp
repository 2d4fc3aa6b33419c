// Randomised check of the factorization's host block map (csrc/flat_map.h)
// against std::unordered_map: inserts, overwrites, erases, lookups, growth,
// iteration and swap.  Prints "ok" and exits 0 when every operation agrees.
#include <cstdio>
#include <random>
#include <unordered_map>

#include "../../paper_1611_03189_gb300/csrc/flat_map.h"

int main() {
  std::mt19937_64 rng(7);
  for (int trial = 0; trial < 40; ++trial) {
    hs::FlatMap<long long> f;
    std::unordered_map<unsigned long long, long long> u;
    const int keys = 1 + (int)(rng() % 3000);
    if (trial % 3 == 0) f.reserve((size_t)keys);
    for (int op = 0; op < 30000; ++op) {
      const unsigned long long k = ((rng() % keys) << 32) | (rng() % 5);
      const int r = (int)(rng() % 10);
      if (r < 4) {
        const long long v = (long long)(rng() >> 1);
        f[k] = v;
        u[k] = v;
      } else if (r < 5) {
        auto ins = f.try_emplace(k);
        const bool fresh = u.find(k) == u.end();
        if (ins.second != fresh) return std::printf("try_emplace: inserted flag\n"), 1;
        if (fresh) {
          *ins.first = 42;
          u[k] = 42;
        } else if (*ins.first != u[k]) {
          return std::printf("try_emplace: value\n"), 1;
        }
      } else if (r < 7) {
        f.erase(k);
        u.erase(k);
      } else if (r < 9) {
        auto it = f.find(k);
        auto jt = u.find(k);
        if ((it == f.end()) != (jt == u.end())) return std::printf("find: presence\n"), 1;
        if (it != f.end() && (it->first != k || it->second != jt->second)) return std::printf("find: value\n"), 1;
      } else if (f.count(k) != u.count(k)) {
        return std::printf("count\n"), 1;
      }
    }
    if (f.size() != u.size()) return std::printf("size\n"), 1;
    size_t n = 0;
    for (auto &kv : f) {
      ++n;
      auto jt = u.find(kv.first);
      if (jt == u.end() || jt->second != kv.second) return std::printf("iteration\n"), 1;
    }
    if (n != u.size()) return std::printf("iteration count\n"), 1;
    hs::FlatMap<long long> g;
    g.swap(f);
    if (g.size() != u.size() || f.size() != 0) return std::printf("swap\n"), 1;
    g.clear();
    if (g.size() != 0 || g.begin() != g.end()) return std::printf("clear\n"), 1;
  }
  std::printf("ok\n");
  return 0;
}
