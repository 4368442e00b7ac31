// Grid-wide barrier of a cooperative launch, shared by the fused sweep (sweep.cu) and the
// grid-parallel factorisation of the coarsest level (setup.cu).
#pragma once

#include "internal.cuh"

namespace cav {

// Grid-wide barrier of a cooperative launch (every CTA resident), called by one thread per
// CTA between CTA-level barriers.  Arrivals go to GB_GROUPS counters (CTA b to counter b mod
// GB_GROUPS, each on its own 128-byte line), so at most G / GB_GROUPS atomics queue on one
// address; the last CTA of each group resets its counter and adds one to the top counter, and
// the last group's CTA resets that and advances the generation, which releases everyone.  The
// state returns to its start at every barrier, so it serves launch after launch.  Each wait
// is bounded: it gives up after about a second, recording DEV_TIMEOUT.
__device__ inline unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ inline void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ inline unsigned atom_add_acq_rel_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
constexpr int GB_GROUPS = 8, GB_STRIDE = 32;  // arrival counters of the grid barrier
constexpr int GB_WORDS = (GB_GROUPS + 2) * GB_STRIDE;
static_assert(GB_WORDS <= CAV_GBAR_WORDS, "the hierarchy's barrier state");
constexpr long long GRID_WAIT_LIMIT = 1LL << 31;  // clock cycles
__device__ inline void grid_barrier(unsigned* bar, int* status) {
  const unsigned G = gridDim.x, g = blockIdx.x % GB_GROUPS;
  const unsigned ngroups = G < (unsigned)GB_GROUPS ? G : (unsigned)GB_GROUPS;
  const unsigned gsize = (G - g + GB_GROUPS - 1) / GB_GROUPS;  // CTAs b < G with b mod GB_GROUPS = g
  unsigned* top = bar + GB_GROUPS * GB_STRIDE;
  unsigned* gen_p = top + GB_STRIDE;
  // acquire-release atomics carry the CTA's writes (ordered before the caller's bar.sync) to
  // the last arriver, whose release of the generation carries everything to the waiters'
  // acquire loads; the plain resets are ordered by the atomics and the release after them
  const unsigned gen = ld_acquire_u32(gen_p);
  if (atom_add_acq_rel_u32(&bar[g * GB_STRIDE], 1u) + 1 == gsize) {  // the last of its group
    bar[g * GB_STRIDE] = 0u;
    if (atom_add_acq_rel_u32(top, 1u) + 1 == ngroups) {  // the last group: release everyone
      *top = 0u;
      st_release_u32(gen_p, gen + 1);
      return;
    }
  }
  const long long t0 = clock64();
  while (ld_acquire_u32(gen_p) == gen) {
    if (clock64() - t0 > GRID_WAIT_LIMIT) {
      atomicExch(status, DEV_TIMEOUT);
      return;
    }
  }
}

}  // namespace cav
