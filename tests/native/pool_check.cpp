// Drives the serving pool allocator (velo_pool.hpp) from a script on stdin:
//   init <size> | alloc <n> | release <off> <n> | dump
// and prints one line per command: the offset of an allocation (or "fail"),
// "ok" for init / release, and for dump the used / peak bytes followed by the
// free list as offset:size pairs.
#include <stdio.h>
#include <string.h>

#include "velo_pool.hpp"

int main() {
  velo::Pool pool;
  char cmd[32];
  while (scanf("%31s", cmd) == 1) {
    unsigned long long a = 0, b = 0;
    if (!strcmp(cmd, "init")) {
      if (scanf("%llu", &a) != 1) return 2;
      pool.init(a);
      printf("ok\n");
    } else if (!strcmp(cmd, "alloc")) {
      if (scanf("%llu", &a) != 1) return 2;
      uint64_t off = 0;
      if (pool.alloc(a, &off)) printf("%llu\n", (unsigned long long)off);
      else printf("fail\n");
    } else if (!strcmp(cmd, "release")) {
      if (scanf("%llu %llu", &a, &b) != 2) return 2;
      pool.release(a, b);
      printf("ok\n");
    } else if (!strcmp(cmd, "dump")) {
      printf("%llu %llu %llu", (unsigned long long)pool.used(), (unsigned long long)pool.peak(),
             (unsigned long long)pool.largest_free());
      pool.for_each_free([](uint64_t off, uint64_t n) { printf(" %llu:%llu", (unsigned long long)off, (unsigned long long)n); });
      printf("\n");
    } else {
      return 2;
    }
  }
  return 0;
}
