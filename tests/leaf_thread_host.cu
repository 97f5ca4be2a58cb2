// Host build of the thread-granular leaf insert and delete (leaf_thread.cuh)
// for the CPU tests.  The leaf is copied next to an inaccessible page (before it or
// after it), so any access outside the leaf's LB bytes faults the test.
#include <sys/mman.h>
#include <unistd.h>

#include "../paper_2305_05055_gb300/csrc/leaf_thread.cuh"

extern "C" int lt_insert(uint8_t* leaf, uint32_t LB, uint32_t uold, uint32_t m,
                         const uint64_t* keys, uint32_t s, uint32_t* out, int guard_after,
                         int del) {
  const size_t pg = (size_t)sysconf(_SC_PAGESIZE);
  const size_t span = ((LB + pg - 1) / pg + 2) * pg;
  uint8_t* base = (uint8_t*)mmap(nullptr, span, PROT_READ | PROT_WRITE,
                                 MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
  if (base == MAP_FAILED) return -1;
  uint8_t* lp;
  if (guard_after) {
    mprotect(base + span - pg, pg, PROT_NONE);
    lp = base + span - pg - LB;
  } else {
    mprotect(base, pg, PROT_NONE);
    lp = base + pg;
  }
  memcpy(lp, leaf, LB);
  uint64_t y[leafthr::kKeys] = {0, 0, 0, 0};
  for (uint32_t i = 0; i < s && i < leafthr::kKeys; i++) y[i] = keys[i];
  uint32_t rpos[leafthr::kKeys], rcode[leafthr::kKeys], epos[leafthr::kKeys],
      ekey[leafthr::kKeys];
  uint64_t rval[leafthr::kKeys];
  int32_t esa[leafthr::kKeys];
  const leafthr::Scratch S{rpos, rval, rcode, epos, esa, ekey, 1};
  leafthr::Result R{};
  const uint32_t st = del ? leafthr::delete_leaf(lp, LB, uold, m, y, s, S, R)
                          : leafthr::insert_leaf(lp, LB, uold, m, y, s, S, R);
  memcpy(leaf, lp, LB);
  munmap(base, span);
  out[0] = R.nb;
  out[1] = R.newc;
  out[2] = R.added;
  out[3] = R.wlo;
  out[4] = R.whi;
  out[5] = (uint32_t)R.newhead;
  out[6] = (uint32_t)(R.newhead >> 32);
  return (int)st;
}
