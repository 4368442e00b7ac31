// One weighted additive CAV sweep (Eq. additive_cav_saddle) and the V-cycle of Sec. 4.
//
// A sweep on level l with iterate w and right-hand side b:
//   1. r = b - K_E w                                   (stencil kernel + E_E rows)
//   2. delta_p = diag(s_c) X_p diag(s_r) r|_p for every enlarged patch p
//      (batched variable-size GEMV; the inverses, the only large operand, are streamed
//      from HBM through shared memory by TMA bulk copies in a persistent kernel)
//   3. w_k += alpha / count_k * (sum of the corrections at k of every patch holding k):
//      unknowns held only by standard 5-unknown Vanka patches in a stencil kernel (their
//      shared 5x5 inverse is applied on the fly), the others one warp per unknown over the
//      slots of the enlarged patches holding it (fixed order, no atomics)
//   4. remove the mean pressure (Sec. 3.3).
#include <algorithm>
#include <map>
#include <mutex>
#include <queue>
#include <set>
#include <tuple>
#include <string>
#include <utility>

#include "internal.cuh"
#include "device_util.cuh"
#include "level_math.cuh"
#include "sweep_parts.cuh"
#include "grid_sync.cuh"
#include "tma_util.cuh"

namespace cav {

// ------------------------------------------------------------------ 2. patch apply

// Fallback for patches too large for the pipelined kernel: one CTA per patch, the scaled
// residual in shared memory, the column-major inverse (ld = round8(n)) read straight from
// global memory, each thread owning V consecutive rows.
template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS)
k_patch_apply(const int* __restrict__ order, const int64_t* __restrict__ off, const int* __restrict__ dofs,
              const int64_t* __restrict__ inv_off, const T* __restrict__ inv, const double* __restrict__ s_r,
              const double* __restrict__ s_c, const double* __restrict__ r, double* __restrict__ delta) {
  pdl_wait();
  pdl_trigger();
  typedef VecLoad<T> VL;
  typedef typename VL::acc_t acc_t;
  constexpr int V = VL::V;
  extern __shared__ unsigned char smem_raw[];
  acc_t* y = reinterpret_cast<acc_t*>(smem_raw);
  const int p = order[blockIdx.x];
  const int64_t d0 = off[p];
  const int n = (int)(off[p + 1] - d0);
  const int ld = (n + 7) & ~7;
  for (int b = threadIdx.x; b < n; b += THREADS) y[b] = (acc_t)(s_r[d0 + b] * r[dofs[d0 + b]]);
  __syncthreads();
  const T* X = inv + inv_off[p];
  for (int a0 = threadIdx.x * V; a0 < n; a0 += THREADS * V) {
    acc_t acc[V];
#pragma unroll
    for (int q = 0; q < V; ++q) acc[q] = 0;
    const T* col = X + a0;
    for (int b = 0; b < n; ++b) {
      acc_t x0[V];
      VL::load(col + (int64_t)b * ld, x0);
      const acc_t yb = y[b];
#pragma unroll
      for (int q = 0; q < V; ++q) acc[q] = mad(x0[q], yb, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < V; ++q)
      if (a0 + q < n) delta[d0 + a0 + q] = s_c[d0 + a0 + q] * (double)acc[q];
  }
}

constexpr int TMA_CONSUMER_WARPS = 4;
constexpr int TMA_THREADS = 32 * (TMA_CONSUMER_WARPS + 2);  // producer, gatherer, consumers
constexpr int TMA_MAXPASS = 2;          // row passes per consumer thread
constexpr int Y_SLOTS = 2;
constexpr int GATHER_UNROLL = 8;  // slots per lane in one round of the gatherer's loads
constexpr int FUSED_CONSUMER_WARPS = 6;
constexpr int FUSED_THREADS = 32 * (FUSED_CONSUMER_WARPS + 2);  // = UPD_THREADS

template <typename T, int CW>
__host__ __device__ constexpr int tma_max_rows() {
  return TMA_MAXPASS * 32 * CW * VecLoad<T>::V;
}

// The q-th patch a persistent CTA takes (q = round * G + CTA): rounds alternate direction over
// the size-descending order, so every CTA gets a large and a small patch in each pair of
// rounds and their loads stay balanced.
__device__ inline int zigzag(int q, int G, int n) {
  const int r = q / G, c = q - r * G;
  const int len = min(G, n - r * G);
  return (r & 1) ? r * G + (len - 1 - c) : q;
}

// Arguments of the batched patch apply (the enlarged patches of one level).
template <typename T>
struct ApplyArgs {
  int n_big;
  const int* order;
  const int64_t* off;
  const int* dofs;
  const int64_t* inv_off;
  const T* inv;
  const double* s_r;
  const double* s_c;
  const double* r;
  double* delta;
  int max_n;
  int* status;
  const int* s_off;   // nullable: CTA b takes the patches s_list[s_off[b] .. s_off[b + 1]) (in order);
  const int* s_list;  // null: the zigzag over the size-descending order
};

// Patches of this CTA, and its t-th one.
template <typename T>
__device__ inline int apply_count(const ApplyArgs<T>& a) {
  if (a.s_off) return a.s_off[blockIdx.x + 1] - a.s_off[blockIdx.x];
  return (a.n_big > (int)blockIdx.x) ? (a.n_big - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
}
template <typename T>
__device__ inline int apply_patch(const ApplyArgs<T>& a, int t) {
  if (a.s_off) return a.s_list[a.s_off[blockIdx.x] + t];
  return a.order[zigzag((int)blockIdx.x + t * (int)gridDim.x, gridDim.x, a.n_big)];
}

// The shared-memory ring of the persistent patch apply: TMA_STAGES stages of TMA_CHUNK bytes,
// Y_SLOTS gathered vectors, their mbarriers and the CTA's abort flag.
template <typename T, int TMA_STAGES, int TMA_CHUNK>
struct ApplyRing {
  typedef typename VecLoad<T>::acc_t acc_t;
  unsigned char* stage_buf;
  acc_t* ybuf;
  size_t yslot;  // elements per gathered vector
  uint64_t *full, *empty, *yfull, *yempty;
  int* abort_flag;
  __device__ ApplyRing(unsigned char* smem, int max_n) {
    const size_t ybytes = ((size_t)max_n * sizeof(acc_t) + 127) & ~(size_t)127;
    stage_buf = smem;
    ybuf = reinterpret_cast<acc_t*>(smem + TMA_STAGES * TMA_CHUNK);
    yslot = ybytes / sizeof(acc_t);
    full = reinterpret_cast<uint64_t*>(smem + TMA_STAGES * TMA_CHUNK + Y_SLOTS * ybytes);
    empty = full + TMA_STAGES;
    yfull = empty + TMA_STAGES;
    yempty = yfull + Y_SLOTS;
    abort_flag = reinterpret_cast<int*>(yempty + Y_SLOTS);
  }
  static size_t bytes(int max_n) {
    const size_t ybytes = ((size_t)max_n * sizeof(acc_t) + 127) & ~(size_t)127;
    return (size_t)TMA_STAGES * TMA_CHUNK + Y_SLOTS * ybytes + (2 * TMA_STAGES + 2 * Y_SLOTS) * sizeof(uint64_t) +
           16;  // the CTA's abort flag
  }
  // one thread: the barriers for CW consumer warps
  __device__ void init(int cw) {
    *abort_flag = 0;
    for (int s = 0; s < TMA_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], cw);
    }
    for (int s = 0; s < Y_SLOTS; ++s) {
      mbar_init(&yfull[s], 32);
      mbar_init(&yempty[s], cw);
    }
    mbar_fence_init();
  }
};

// Persistent batched patch apply.  CTA c takes the patches zigzag(c), zigzag(c + G), ... of
// the size-descending order, with three roles:
//  * one lane (producer): streams each patch's column-major inverse -- a contiguous block of
//    n * ld elements -- into a ring of TMA_STAGES shared-memory stages of at most TMA_CHUNK
//    bytes (whole columns) with cp.async.bulk; "full" mbarriers carry the transaction bytes,
//    "empty" mbarriers take one arrival per consumer warp;
//  * one warp (gatherer): writes y = s_r * r|_p of the coming patches into a double-buffered
//    shared ring ("yfull": 32 lane arrivals, "yempty": one arrival per consumer warp), so the
//    dependent index -> residual loads of patch t+1 overlap the streaming of patch t;
//  * CW consumer warps: acc[rows] += X[rows, b] y[b] stage by stage, each thread owning V
//    consecutive rows (up to TMA_MAXPASS row blocks), then delta = s_c * acc.
// Every wait is bounded.  A wait that runs out records DEV_TIMEOUT and raises the CTA's abort
// flag; every role then stops (no further copies, arrivals or writes; the delta of the
// remaining patches is left unwritten and the host reports IB_ERR_TIMEOUT), and the producer
// waits for the copies it has in flight to land before it returns.  A warp's give-up
// decision is taken by all its lanes together.
template <typename T, int TMA_STAGES, int TMA_CHUNK>
__device__ inline void apply_producer(const ApplyArgs<T>& a, ApplyRing<T, TMA_STAGES, TMA_CHUNK>& R) {
  volatile int* ab = R.abort_flag;
  int stage = 0;
  uint32_t phase = 0;
  uint32_t used = 0, last_par = 0;  // per stage: a copy was issued; parity of its last phase
  bool ok = true;
  const int count = apply_count(a);
  for (int t = 0; ok && t < count; ++t) {
    const int p = apply_patch(a, t);
    const int n = (int)(a.off[p + 1] - a.off[p]);
    const uint32_t col_bytes = (uint32_t)(((n + 7) & ~7) * sizeof(T));
    const int cpc = TMA_CHUNK / (int)col_bytes;
    const unsigned char* src = reinterpret_cast<const unsigned char*>(a.inv + a.inv_off[p]);
    for (int b0 = 0; b0 < n; b0 += cpc) {
      const int nc = min(cpc, n - b0);
      if (!mbar_wait(&R.empty[stage], phase ^ 1u, a.status, ab, false)) {
        ok = false;
        break;
      }
      const uint32_t bytes = (uint32_t)nc * col_bytes;
      mbar_arrive_expect_tx(&R.full[stage], bytes);
      bulk_copy_g2s(R.stage_buf + (size_t)stage * TMA_CHUNK, src + (size_t)b0 * col_bytes, bytes, &R.full[stage]);
      used |= 1u << stage;
      last_par = phase ? (last_par | (1u << stage)) : (last_par & ~(1u << stage));
      if (++stage == TMA_STAGES) {
        stage = 0;
        phase ^= 1u;
      }
    }
  }
  // every issued copy lands before the role ends (immediate when the consumers saw them all)
  for (int s = 0; s < TMA_STAGES; ++s)
    if ((used >> s) & 1u) mbar_drain(&R.full[s], (last_par >> s) & 1u, a.status);
}

template <typename T, int TMA_STAGES, int TMA_CHUNK>
__device__ inline void apply_gatherer(const ApplyArgs<T>& a, ApplyRing<T, TMA_STAGES, TMA_CHUNK>& R) {
  typedef typename VecLoad<T>::acc_t acc_t;
  volatile int* ab = R.abort_flag;
  const int lane = threadIdx.x & 31;
  const int count = apply_count(a);
  for (int t = 0; t < count; ++t) {
    const int slot = t & 1;
    const uint32_t par = (uint32_t)((t >> 1) & 1);
    const bool got = mbar_wait(&R.yempty[slot], par ^ 1u, a.status, ab, false);
    if (!__all_sync(0xffffffffu, got)) break;
    const int p = apply_patch(a, t);
    const int64_t d0 = a.off[p];
    const int n = (int)(a.off[p + 1] - d0);
    acc_t* y = R.ybuf + (size_t)slot * R.yslot;
    // GATHER_UNROLL slots per lane per round: every index load of the round is issued, then
    // every residual load, so a patch costs two dependent load latencies per round instead
    // of two per 32 slots
    for (int b0 = lane; b0 < n; b0 += 32 * GATHER_UNROLL) {
      int idx[GATHER_UNROLL];
      double sr[GATHER_UNROLL], rv[GATHER_UNROLL];
#pragma unroll
      for (int u = 0; u < GATHER_UNROLL; ++u) {
        const int b = b0 + 32 * u;
        idx[u] = (b < n) ? a.dofs[d0 + b] : -1;
        sr[u] = (b < n) ? a.s_r[d0 + b] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < GATHER_UNROLL; ++u) rv[u] = (idx[u] >= 0) ? a.r[idx[u]] : 0.0;
#pragma unroll
      for (int u = 0; u < GATHER_UNROLL; ++u) {
        const int b = b0 + 32 * u;
        if (b < n) y[b] = (acc_t)(sr[u] * rv[u]);
      }
    }
    mbar_arrive(&R.yfull[slot]);
  }
}

// ct: the thread's index among the CW consumer warps' threads
template <typename T, int TMA_STAGES, int TMA_CHUNK, int CW>
__device__ inline void apply_consumer(const ApplyArgs<T>& a, ApplyRing<T, TMA_STAGES, TMA_CHUNK>& R, int ct,
                                      bool stall) {
  typedef VecLoad<T> VL;
  typedef typename VL::acc_t acc_t;
  constexpr int V = VL::V;
  constexpr int CT = 32 * CW;
  volatile int* ab = R.abort_flag;
  const int lane = threadIdx.x & 31;
  int stage = 0;
  uint32_t phase = 0;
  const int count = apply_count(a);
  for (int t = 0; t < count; ++t) {
    const int p = apply_patch(a, t);
    const int64_t d0 = a.off[p];
    const int n = (int)(a.off[p + 1] - d0);
    const int ld = (n + 7) & ~7;
    const int cpc = TMA_CHUNK / (int)(ld * sizeof(T));
    const int slot = t & 1;
    if (!__all_sync(0xffffffffu, mbar_wait(&R.yfull[slot], (uint32_t)((t >> 1) & 1), a.status, ab, stall))) break;
    const acc_t* y = R.ybuf + (size_t)slot * R.yslot;
    acc_t acc[TMA_MAXPASS][V];
#pragma unroll
    for (int ps = 0; ps < TMA_MAXPASS; ++ps)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[ps][v] = 0;
    bool dead = false;
    for (int b0 = 0; b0 < n; b0 += cpc) {
      const int nc = min(cpc, n - b0);
      if (!__all_sync(0xffffffffu, mbar_wait(&R.full[stage], phase, a.status, ab, stall))) {
        dead = true;
        break;
      }
      const T* X = reinterpret_cast<const T*>(R.stage_buf + (size_t)stage * TMA_CHUNK);
#pragma unroll
      for (int ps = 0; ps < TMA_MAXPASS; ++ps) {
        const int a0 = (ps * CT + ct) * V;
        if (a0 < n) {
#pragma unroll 4
          for (int c = 0; c < nc; ++c) {
            acc_t x0[V];
            VL::load_shared(X + (size_t)c * ld + a0, x0);
            const acc_t y0 = y[b0 + c];
#pragma unroll
            for (int v = 0; v < V; ++v) acc[ps][v] = mad(x0[v], y0, acc[ps][v]);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&R.empty[stage]);
      if (++stage == TMA_STAGES) {
        stage = 0;
        phase ^= 1u;
      }
    }
    if (dead) break;
    __syncwarp();
    if (lane == 0) mbar_arrive(&R.yempty[slot]);
#pragma unroll
    for (int ps = 0; ps < TMA_MAXPASS; ++ps) {
      const int a0 = (ps * CT + ct) * V;
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (a0 + v < n) a.delta[d0 + a0 + v] = a.s_c[d0 + a0 + v] * (double)acc[ps][v];
    }
  }
}

template <typename T, int TMA_STAGES, int TMA_CHUNK>
__global__ void __launch_bounds__(TMA_THREADS) k_patch_apply_tma(ApplyArgs<T> a) {
  extern __shared__ __align__(128) unsigned char smem[];
  ApplyRing<T, TMA_STAGES, TMA_CHUNK> R(smem, a.max_n);
  const bool stall = wait_stall_enabled();
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) R.init(TMA_CONSUMER_WARPS);
  __syncthreads();
  // Under a programmatic launch the residual kernel ahead may still be running.  Only the
  // gatherer reads what it writes (r), so only the gatherer waits for it; the producer streams
  // the inverses (never written during a sweep) from the start, and the consumers write delta
  // only after the gatherer's first handoff, when every earlier kernel (the previous sweep's
  // scatter, which reads delta) has finished.  (Measured: launching the finest level's apply
  // this way made its sweep slower, 86 -> 103 us, the early bulk traffic delaying the
  // latency-bound residual kernel; the launchers do not request it.)
  pdl_trigger();
  if (warp == 0) {
    if ((threadIdx.x & 31) == 0) apply_producer(a, R);
    return;
  }
  if (warp == 1) {
    pdl_wait();
    apply_gatherer(a, R);
    return;
  }
  apply_consumer<T, TMA_STAGES, TMA_CHUNK, TMA_CONSUMER_WARPS>(a, R, (int)threadIdx.x - 64, stall);
}

// ------------------------------------------------------------------ the fused sweep

// bar.sync on a named barrier for the nthreads threads of warps 1.. (the producer warp apart)
__device__ inline void group_sync(int nthreads) { asm volatile("bar.sync 2, %0;" ::"r"(nthreads) : "memory"); }

// One whole sweep of an additive level in one persistent cooperative launch (the four parts
// of Eq. additive_cav_saddle plus, optionally, the mean removal of Sec. 3.3), each part the
// same block-level work as its separate kernel:
//   R  r = b - K_E w (skipped for w = 0: r = b), on warps 1-7 as 224-thread blocks, while the
//      producer lane of warp 0 already streams the first inverse stages;
//   -- grid barrier (r complete) --
//   A  the patch apply: warp 0 producer, warp 1 gatherer, warps 2-7 consumers;
//   -- grid barrier (delta complete) --
//   U  the scatter / update as 256-thread blocks, each writing its pressure partial;
//   -- grid barrier (partials complete), only with remove_mean --
//   M  p -= mean(p).
// The kernel boundaries it replaces cost a launch gap and a tail each, and the pipeline's
// first stages no longer start cold after the residual.
template <typename T, int TMA_STAGES, int TMA_CHUNK>
__global__ void __launch_bounds__(FUSED_THREADS)
k_sweep_fused(ResArgs ra, int nb_res, ApplyArgs<T> a, UpdArgs ua, int nb_upd, int remove_mean, int n_partial,
              double* wpart, unsigned* bar) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double sm[8];
  ApplyRing<T, TMA_STAGES, TMA_CHUNK> R(smem, a.max_n);
  const bool stall = wait_stall_enabled();
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) R.init(FUSED_CONSUMER_WARPS);
  __syncthreads();
  if (warp == 0) {
    if ((threadIdx.x & 31) == 0) apply_producer(a, R);
  } else {
    if (nb_res > 0) {
      for (int vb = blockIdx.x; vb < nb_res; vb += gridDim.x) residual_block<7>(ra, vb, (int)threadIdx.x - 32);
      group_sync(FUSED_THREADS - 32);
      if (threadIdx.x == 32) grid_barrier(bar, a.status);
      group_sync(FUSED_THREADS - 32);
    }
    if (warp == 1) apply_gatherer(a, R);
    else apply_consumer<T, TMA_STAGES, TMA_CHUNK, FUSED_CONSUMER_WARPS>(a, R, (int)threadIdx.x - 64, stall);
  }
  __syncthreads();
  if (threadIdx.x == 0) grid_barrier(bar, a.status);
  __syncthreads();
  // the scatter's (block, warp) units spread over every warp of the grid; each unit's sum of
  // new pressures goes to wpart, and the block partials are formed from them in warp order
  // after the next barrier (the separate kernel's order)
  const int lane = threadIdx.x & 31;
  for (int u = blockIdx.x * (FUSED_THREADS / 32) + warp; u < nb_upd * 8; u += gridDim.x * (FUSED_THREADS / 32)) {
    const double pn = update_warp(ua, u >> 3, u & 7);
    if (lane == 0) wpart[u] = pn;
  }
  __syncthreads();
  if (threadIdx.x == 0) grid_barrier(bar, a.status);
  __syncthreads();
  for (int vb = blockIdx.x * FUSED_THREADS + threadIdx.x; vb < nb_upd; vb += gridDim.x * FUSED_THREADS) {
    double tot = 0.0;
    for (int q = 0; q < 8; ++q) tot += wpart[vb * 8 + q];
    ua.partial[vb] = tot;
  }
  if (remove_mean) {
    __syncthreads();
    if (threadIdx.x == 0) grid_barrier(bar, a.status);
    __syncthreads();
    remove_mean_block(ua.N, n_partial, ua.partial, ua.w + 2 * ua.N * ua.N, (int)blockIdx.x, (int)gridDim.x, sm);
  }
}

// ------------------------------------------------------------------ 3. scatter / update

// Scatter / update in one launch with two block roles (update_block: cell tiles, then the
// unknowns held by enlarged patches), each block writing its partial sum of new pressures.
__global__ void __launch_bounds__(UPD_THREADS) k_update(UpdArgs a) {
  pdl_wait();  // programmatic launch: the patch apply (delta) and residual (r) have finished
  pdl_trigger();
  __shared__ double sm[8];
  update_block(a, (int)blockIdx.x, sm);
}

// 4. p -= mean(p): every block reduces the partials in the same order, then subtracts.
__global__ void k_remove_mean(int N, int n_partial, const double* __restrict__ partial, double* __restrict__ p) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sm[8];
  remove_mean_block(N, n_partial, partial, p, (int)blockIdx.x, (int)gridDim.x, sm);
}

void launch_remove_mean(int N, int n_partial, const double* partial, double* p, cudaStream_t st) {
  const int nblk = div_up(N * N, 256) < 296 ? div_up(N * N, 256) : 296;
  launch_k(k_remove_mean, dim3(nblk), dim3(256), 0, st, false, N, n_partial, partial, p);
}

// Coarsest level: z = (dense inverse) [r; 0], one warp per row, row-major with leading
// dimension ld (n + 1 for the bordered periodic system, n on the channel).
__global__ void k_coarse_apply(int n, int ld, const double* __restrict__ inv, const double* __restrict__ r,
                               double* __restrict__ z) {
  pdl_wait();
  pdl_trigger();
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* a = inv + (int64_t)row * ld;
  double s = 0.0;
  for (int b = lane; b < n; b += 32) s += a[b] * r[b];
  s = warp_sum(s);
  if (lane == 0) z[row] = s;
}

// ------------------------------------------------------------------ host drivers

static LevelOps ops_of(const Level& lv) {
  LevelOps o;
  o.N = lv.N;
  o.h = lv.h;
  o.rho_dt = lv.rho_dt;
  o.mu = lv.mu;
  o.dt = lv.dt;
  o.ee = &lv.ee;
  o.channel = lv.channel;
  return o;
}

// Whether prof_begin / prof_end record events (event-record nodes in a captured V-cycle).
bool prof_records(const cav_hierarchy* H, int level) {
  if (level != 0 || H->no_events) return false;
  return H->capturing || (H->prof_on && (size_t)(2 * H->prof_used + 1) < H->prof_ev.size());
}

void prof_begin(const cav_hierarchy* H, int level, cudaStream_t st) {
  cav_hierarchy* h = const_cast<cav_hierarchy*>(H);
  if (level != 0 || h->no_events) return;
  if (h->capturing) {
    std::vector<cudaEvent_t>& ev = h->vc_ev[h->capturing - 1];
    const size_t q = ev.size();
    ev.resize(q + 2);
    CAV_CHECK_CUDA(cudaEventCreate(&ev[q]));
    CAV_CHECK_CUDA(cudaEventCreate(&ev[q + 1]));
    // External: becomes an event-record node of the graph, recorded on every replay
    CAV_CHECK_CUDA(cudaEventRecordWithFlags(ev[q], st, cudaEventRecordExternal));
    return;
  }
  if (!h->prof_on || (size_t)(2 * h->prof_used + 1) >= h->prof_ev.size()) return;
  CAV_CHECK_CUDA(cudaEventRecord(h->prof_ev[2 * h->prof_used], st));
}
void prof_end(const cav_hierarchy* H, int level, cudaStream_t st) {
  cav_hierarchy* h = const_cast<cav_hierarchy*>(H);
  if (level != 0 || h->no_events) return;
  if (h->capturing) {
    CAV_CHECK_CUDA(cudaEventRecordWithFlags(h->vc_ev[h->capturing - 1].back(), st, cudaEventRecordExternal));
    return;
  }
  if (!h->prof_on || (size_t)(2 * h->prof_used + 1) >= h->prof_ev.size()) return;
  CAV_CHECK_CUDA(cudaEventRecord(h->prof_ev[2 * h->prof_used + 1], st));
  h->prof_pending.emplace_back(h->prof_ev[2 * h->prof_used], h->prof_ev[2 * h->prof_used + 1]);
  ++h->prof_pushed;
  ++h->prof_used;
}

// Read the recorded pairs in issue order, up to push count `upto` (all when negative);
// waits for each pair's stop event.
void prof_collect(cav_hierarchy* H, long long upto) {
  if (upto < 0) upto = H->prof_pushed;
  size_t q = 0;
  while (H->prof_popped < upto && q < H->prof_pending.size()) {
    float ms = 0.f;
    CAV_CHECK_CUDA(cudaEventSynchronize(H->prof_pending[q].second));
    CAV_CHECK_CUDA(cudaEventElapsedTime(&ms, H->prof_pending[q].first, H->prof_pending[q].second));
    H->prof_acc_ms += ms;
    H->prof_acc_n += 1;
    ++q;
    ++H->prof_popped;
  }
  H->prof_pending.erase(H->prof_pending.begin(), H->prof_pending.begin() + q);
  if (H->prof_pending.empty()) H->prof_used = 0;
}

// Multiprocessor count of the current device (cached per device).
static int sm_count() {
  static std::mutex m;
  static int count[64] = {};
  int dev = 0;
  CAV_CHECK_CUDA(cudaGetDevice(&dev));
  CAV_REQUIRE(dev >= 0 && dev < 64, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(m);
  if (count[dev] == 0) CAV_CHECK_CUDA(cudaDeviceGetAttribute(&count[dev], cudaDevAttrMultiProcessorCount, dev));
  return count[dev];
}

// Raise a kernel's dynamic shared memory limit on the current device, once per (kernel,
// device): the attribute is per device, so a process using several GPUs sets it on each.
static void allow_dynamic_smem(const void* kernel, int bytes) {
  static std::mutex m;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  CAV_CHECK_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(m);
  if (done.count({kernel, dev})) return;
  CAV_CHECK_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.insert({kernel, dev});
}

// Patch-apply variants the autotuner chooses among (per level, timed at set-up):
//   0: TMA, 4 stages x 16 KiB, 3 CTAs/SM     1: TMA, 4 x 16 KiB, 2 CTAs/SM
//   2: TMA, 8 stages x 8 KiB, 3 CTAs/SM      3: TMA, 4 x 8 KiB, 4 CTAs/SM
//   4: one CTA per patch, no staging
// All variants accumulate each row over the columns in ascending order with fused
// multiply-adds, so they produce identical bits.
struct ApplyVariant {
  int stages, chunk, ctas_per_sm;
};
static const ApplyVariant kVariants[NUM_APPLY_VARIANTS] = {
    {4, 16384, 3}, {4, 16384, 2}, {8, 8192, 3}, {4, 8192, 4}, {0, 0, 0}};

// The scatter's arguments and block count on level lv (its 32 x 8 cell tiles, then the
// unknowns held by enlarged patches, four per warp).
// r32 (nullable): the residual r in FP32 (FP32 / BF16 levels, sweeps that formed a residual);
// the standard patches are then applied in FP32.
static UpdArgs update_args(const cav_hierarchy* H, const Level& lv, const double* delta, const double* r, double* w,
                           bool w_is_zero, double* partial, const float* r32 = nullptr) {
  UpdArgs a;
  a.N = lv.N;
  a.alpha = H->desc.alpha;
  for (int k = 0; k < 3; ++k)
    for (int q = 0; q < 25; ++q) {
      a.S.m[k][q] = lv.std_inv[k][q];
      a.S32.m[k][q] = (float)lv.std_inv[k][q];
    }
  a.r32 = r32;
  a.gx = div_up(lv.N, 32);
  a.nb_std = a.gx * div_up(lv.N, 8);
  a.inc_off = lv.inc_off;
  a.n_touched = lv.n_touched;
  a.touched = lv.touched;
  a.cell_big = lv.cell_big;
  a.inc_slot = lv.inc_slot;
  a.delta = delta;
  a.r = r;
  a.w = w;
  a.w_is_zero = w_is_zero ? 1 : 0;
  a.partial = partial;
  a.channel = lv.channel;
  a.theta_t = lv.touch_theta;
  return a;
}
__global__ void k_touch_theta(UpdArgs a, double* __restrict__ theta) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.n_touched) return;
  const int k = a.touched[t];
  const StdHolders hs = std_holders(a.N, a.cell_big, a.channel, k);
  theta[t] = 1.0 / (double)((int)(a.inc_off[k + 1] - a.inc_off[k]) + hs.n);
}

void build_touch_theta(cav_hierarchy* H, Level& lv, cudaStream_t st) {
  lv.touch_theta = H->arena.alloc<double>(std::max(lv.n_touched, 1));
  if (lv.n_touched == 0) return;
  UpdArgs a = update_args(H, lv, nullptr, nullptr, nullptr, false, nullptr);
  k_touch_theta<<<div_up(lv.n_touched, 256), 256, 0, st>>>(a, lv.touch_theta);
  CAV_CHECK_LAUNCH();
}

static int update_blocks(const Level& lv) {
  return div_up(lv.N, 32) * div_up(lv.N, 8) + div_up(lv.n_touched, SCATTER_TOUCHED_PER_BLOCK);
}

template <typename T>
static ApplyArgs<T> apply_args(const cav_hierarchy* H, const Level& lv, const T* inv, const double* r,
                               double* delta) {
  ApplyArgs<T> a;
  a.n_big = lv.n_big;
  a.order = lv.order;
  a.off = lv.big_off;
  a.dofs = lv.big_dofs;
  a.inv_off = lv.inv_off;
  a.inv = inv;
  a.s_r = lv.s_r;
  a.s_c = lv.s_c;
  a.r = r;
  a.delta = delta;
  a.max_n = lv.big_max_n;
  a.status = H->status;
  a.s_off = nullptr;
  a.s_list = nullptr;
  return a;
}

// The level's balanced schedule for a grid of G CTAs, if set-up built one (else the zigzag).
template <typename T>
static void use_schedule(ApplyArgs<T>& a, const Level& lv, int G) {
  for (size_t q = 0; q < lv.sched_G.size(); ++q)
    if (lv.sched_G[q] == G) {
      a.s_off = lv.sched_off[q];
      a.s_list = lv.sched_list[q];
    }
}

// Balanced schedules of a level's enlarged patches for every grid size the patch apply and
// the fused sweep launch with (1-4 CTAs per SM, capped at the patch count): longest
// processing time first -- in the size-descending order, each patch goes to the CTA with the
// fewest inverse bytes so far (ties: the lowest CTA) -- so every CTA streams nearly the same
// bytes and the launch ends with no long tail.  Each CTA takes its patches largest first.
void build_schedules(cav_hierarchy* H, Level& lv, cudaStream_t st) {
  lv.sched_G.clear();
  lv.sched_off.clear();
  lv.sched_list.clear();
  if (lv.n_big == 0) return;
  std::vector<int> order(lv.n_big);
  CAV_CHECK_CUDA(cudaMemcpyAsync(order.data(), lv.order, sizeof(int) * lv.n_big, cudaMemcpyDeviceToHost, st));
  CAV_CHECK_CUDA(cudaStreamSynchronize(st));
  const int sms = sm_count();
  std::vector<int> grids;
  for (int c = 1; c <= 4; ++c) {
    grids.push_back(c * sms);
    grids.push_back(std::min(lv.n_big, c * sms));
  }
  std::sort(grids.begin(), grids.end());
  grids.erase(std::unique(grids.begin(), grids.end()), grids.end());
  for (const int G : grids) {
    std::vector<std::vector<int>> lists(G);
    typedef std::pair<int64_t, int> Load;  // (bytes so far, CTA)
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int b = 0; b < G; ++b) heap.push(Load(0, b));
    for (const int p : order) {
      Load l = heap.top();
      heap.pop();
      const int n = lv.host_sizes[p];
      lists[l.second].push_back(p);
      l.first += (int64_t)n * round8(n);
      heap.push(l);
    }
    std::vector<int> off(G + 1, 0), flat;
    flat.reserve(lv.n_big);
    for (int b = 0; b < G; ++b) {
      off[b + 1] = off[b] + (int)lists[b].size();
      flat.insert(flat.end(), lists[b].begin(), lists[b].end());
    }
    int* d_off = H->arena.alloc<int>(G + 1);
    int* d_list = H->arena.alloc<int>(lv.n_big);
    CAV_CHECK_CUDA(cudaMemcpyAsync(d_off, off.data(), sizeof(int) * (G + 1), cudaMemcpyHostToDevice, st));
    CAV_CHECK_CUDA(cudaMemcpyAsync(d_list, flat.data(), sizeof(int) * lv.n_big, cudaMemcpyHostToDevice, st));
    lv.sched_G.push_back(G);
    lv.sched_off.push_back(d_off);
    lv.sched_list.push_back(d_list);
  }
  CAV_CHECK_CUDA(cudaStreamSynchronize(st));
}

template <typename T, int STAGES, int CHUNK>
static void launch_tma(const cav_hierarchy* H, const Level& lv, const T* inv, const double* r, double* delta,
                       int ctas_per_sm, cudaStream_t st, bool pdl) {
  const size_t smem = ApplyRing<T, STAGES, CHUNK>::bytes(lv.big_max_n);
  allow_dynamic_smem(reinterpret_cast<const void*>(k_patch_apply_tma<T, STAGES, CHUNK>), 200 * 1024);
  const int grid = std::min(lv.n_big, ctas_per_sm * sm_count());
  ApplyArgs<T> aa = apply_args<T>(H, lv, inv, r, delta);
  use_schedule(aa, lv, grid);
  launch_k(k_patch_apply_tma<T, STAGES, CHUNK>, dim3(grid), dim3(TMA_THREADS), smem, st, pdl, aa);
}

// Can variant v run this level?  (rows per consumer thread and one whole column per stage)
template <typename T>
static bool variant_fits(const Level& lv, int v) {
  if (kVariants[v].stages == 0) return true;
  return lv.big_max_n <= tma_max_rows<T, TMA_CONSUMER_WARPS>() &&
         (size_t)round8(lv.big_max_n) * sizeof(T) <= (size_t)kVariants[v].chunk;
}

// Resident CTAs per SM of a kernel at a given dynamic shared memory size (cached per device).
static int resident_ctas(const void* kernel, int threads, size_t smem) {
  static std::mutex m;
  static std::map<std::tuple<const void*, size_t, int>, int> cache;
  int dev = 0;
  CAV_CHECK_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(m);
  const auto key = std::make_tuple(kernel, smem, dev);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int n = 0;
  CAV_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem));
  cache[key] = n;
  return n;
}

// The whole sweep of an additive level as one cooperative launch of k_sweep_fused with the
// staging shape of apply variant v (its stages, chunk and CTAs per SM, capped by residency).
// Returns false (nothing launched) when the level cannot take it.
template <typename T, int STAGES, int CHUNK>
static bool launch_fused(const cav_hierarchy* H, const Level& lv, const T* inv, const double* b, double* w,
                         bool w_is_zero, double* r_buf, float* r32, double* delta, double* partial,
                         bool remove_mean, int ctas_per_sm, cudaStream_t st) {
  if (lv.big_max_n > tma_max_rows<T, FUSED_CONSUMER_WARPS>() || (size_t)round8(lv.big_max_n) * sizeof(T) > CHUNK)
    return false;
  const void* kern = reinterpret_cast<const void*>(k_sweep_fused<T, STAGES, CHUNK>);
  const size_t smem = ApplyRing<T, STAGES, CHUNK>::bytes(lv.big_max_n);
  allow_dynamic_smem(kern, 200 * 1024);
  const int per_sm = std::min(ctas_per_sm, resident_ctas(kern, FUSED_THREADS, smem));
  if (per_sm < 1) return false;
  const int grid = per_sm * sm_count();
  const double* r = w_is_zero ? b : r_buf;
  ResArgs ra = residual_args(ops_of(lv), w, b, r_buf, 0, FUSED_THREADS / 32 - 1);
  ra.out32 = w_is_zero ? nullptr : r32;
  const int nb_res = w_is_zero ? 0 : residual_blocks(ra, FUSED_THREADS / 32 - 1);
  ApplyArgs<T> aa = apply_args<T>(H, lv, inv, r, delta);
  use_schedule(aa, lv, grid);
  const UpdArgs ua = update_args(H, lv, delta, r, w, w_is_zero, partial, ra.out32);
  const int nb_upd = update_blocks(lv);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(FUSED_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: the grid barriers need it
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CAV_CHECK_CUDA(cudaLaunchKernelEx(&cfg, k_sweep_fused<T, STAGES, CHUNK>, ra, nb_res, aa, ua, nb_upd,
                                    (remove_mean && !lv.channel) ? 1 : 0, lv.n_partial, lv.wpart, H->gbar));
  CAV_CHECK_LAUNCH();
  return true;
}

template <typename T>
static bool launch_fused_variant(const cav_hierarchy* H, const Level& lv, const T* inv, const double* b, double* w,
                                 bool w_is_zero, double* r_buf, float* r32, double* delta, double* partial,
                                 bool remove_mean, int v, cudaStream_t st) {
  switch (v) {
    case 0: return launch_fused<T, 4, 16384>(H, lv, inv, b, w, w_is_zero, r_buf, r32, delta, partial, remove_mean, 3, st);
    case 1: return launch_fused<T, 4, 16384>(H, lv, inv, b, w, w_is_zero, r_buf, r32, delta, partial, remove_mean, 2, st);
    case 2: return launch_fused<T, 8, 8192>(H, lv, inv, b, w, w_is_zero, r_buf, r32, delta, partial, remove_mean, 3, st);
    case 3: return launch_fused<T, 4, 8192>(H, lv, inv, b, w, w_is_zero, r_buf, r32, delta, partial, remove_mean, 4, st);
    default: return false;
  }
}

// r32: FP32 copy of the residual on FP32 / BF16 levels (null on FP64 levels)
static bool launch_fused_any(const cav_hierarchy* H, const Level& lv, const double* b, double* w, bool w_is_zero,
                             double* r_buf, float* r32, double* delta, double* partial, bool remove_mean, int v,
                             cudaStream_t st) {
  if (lv.n_big == 0 || !H->gbar || !lv.wpart) return false;
  if (lv.precision == CAV_PREC_FP32)
    return launch_fused_variant<float>(H, lv, lv.inv32, b, w, w_is_zero, r_buf, r32, delta, partial, remove_mean, v,
                                       st);
  if (lv.precision == CAV_PREC_BF16)
    return launch_fused_variant<__nv_bfloat16>(H, lv, lv.inv16, b, w, w_is_zero, r_buf, r32, delta, partial,
                                               remove_mean, v, st);
  return launch_fused_variant<double>(H, lv, lv.inv64, b, w, w_is_zero, r_buf, nullptr, delta, partial, remove_mean,
                                      v, st);
}

template <typename T>
static void launch_patch_apply_variant(const cav_hierarchy* H, const Level& lv, const T* inv, const double* r,
                                       double* delta, int v, cudaStream_t st, bool pdl) {
  typedef typename VecLoad<T>::acc_t acc_t;
  if (!variant_fits<T>(lv, v)) v = NUM_APPLY_VARIANTS - 1;
  switch (v) {
    case 0: launch_tma<T, 4, 16384>(H, lv, inv, r, delta, 3, st, pdl); break;
    case 1: launch_tma<T, 4, 16384>(H, lv, inv, r, delta, 2, st, pdl); break;
    case 2: launch_tma<T, 8, 8192>(H, lv, inv, r, delta, 3, st, pdl); break;
    case 3: launch_tma<T, 4, 8192>(H, lv, inv, r, delta, 4, st, pdl); break;
    default: {
      const size_t smem = sizeof(acc_t) * (size_t)lv.big_max_n;
      launch_k(k_patch_apply<T, 128>, dim3(lv.n_big), dim3(128), smem, st, pdl, lv.order, lv.big_off, lv.big_dofs,
               lv.inv_off, inv, lv.s_r, lv.s_c, r, delta);
    }
  }
}

static void launch_patch_apply_any(const cav_hierarchy* H, const Level& lv, const double* r, double* delta, int v,
                                   cudaStream_t st, bool pdl = false) {
  if (lv.precision == CAV_PREC_FP32) launch_patch_apply_variant<float>(H, lv, lv.inv32, r, delta, v, st, pdl);
  else if (lv.precision == CAV_PREC_BF16)
    launch_patch_apply_variant<__nv_bfloat16>(H, lv, lv.inv16, r, delta, v, st, pdl);
  else launch_patch_apply_variant<double>(H, lv, lv.inv64, r, delta, v, st, pdl);
}

// Autotuner: time every variant on this level's own patches (two warm-up and five timed
// launches each, CUDA events on the set-up stream) and keep the fastest.
void autotune_level(cav_hierarchy* H, Level& lv, cudaStream_t st) {
  lv.apply_variant = 0;
  if (lv.n_big == 0) return;
  cudaEvent_t e0, e1;
  CAV_CHECK_CUDA(cudaEventCreate(&e0));
  CAV_CHECK_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int v = 0; v < NUM_APPLY_VARIANTS; ++v) {
    for (int w = 0; w < 2; ++w) launch_patch_apply_any(H, lv, lv.r, lv.delta, v, st);
    CAV_CHECK_CUDA(cudaEventRecord(e0, st));
    for (int w = 0; w < 5; ++w) launch_patch_apply_any(H, lv, lv.r, lv.delta, v, st);
    CAV_CHECK_CUDA(cudaEventRecord(e1, st));
    CAV_CHECK_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    CAV_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    lv.apply_us[v] = 1e3f * ms / 5.f;
    if (ms < best) {
      best = ms;
      lv.apply_variant = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

// The four steps of one sweep with explicit scratch (residual r_buf and, on FP32 / BF16
// levels, its FP32 copy r32_buf; packed corrections delta_buf, partial sums partial_buf);
// shared by cav_sweep and cav_sweep_noalloc.
// pdl_first: the operation ahead of the sweep's first kernel on st is one of this library's
// kernels, so it may be a programmatic launch (the kernels after it are, except around the
// finest level's profiling events, whose record nodes sit between the kernels).
// The first sweep from w = 0 forms no residual (r = b) and applies the standard patches in
// FP64 on every level.
static void sweep_impl(const cav_hierarchy* H, int l, const double* b, double* w, bool w_is_zero, double* r_buf,
                       float* r32_buf, double* delta_buf, double* partial_buf, bool profile, cudaStream_t st,
                       bool remove_mean = true, bool pdl_first = false, bool allow_fused = true) {
  const Level& lv = H->levels[l];
  const double* r = b;
  float* r32 = (lv.precision != CAV_PREC_FP64 && !w_is_zero) ? r32_buf : nullptr;
  const bool events = profile && prof_records(H, l);
  if (lv.fused && allow_fused) {  // one cooperative launch (the profiling record then spans the whole sweep)
    if (events) prof_begin(H, l, st);
    const bool ok = launch_fused_any(H, lv, b, w, w_is_zero, r_buf, r32, delta_buf, partial_buf, remove_mean,
                                     lv.apply_variant, st);
    if (events) prof_end(H, l, st);
    CAV_REQUIRE(ok, "sweep: the level's fused sweep cannot be launched");
    return;
  }
  bool pdl = pdl_first;
  if (!w_is_zero) {
    launch_apply(ops_of(lv), w, b, r_buf, 0, st, pdl, r32);
    r = r_buf;
    pdl = true;
  }
  if (lv.n_big > 0) {
    if (events) prof_begin(H, l, st);
    launch_patch_apply_any(H, lv, r, delta_buf, lv.apply_variant, st, false);
    if (events) prof_end(H, l, st);
    // measured: a programmatic launch of the scatter after the persistent apply slows the
    // sweep (its blocks sit resident beside the apply's), so it is a plain launch
    pdl = false;
  }
  const UpdArgs ua = update_args(H, lv, delta_buf, r, w, w_is_zero, partial_buf, r32);
  launch_k(k_update, dim3(update_blocks(lv)), dim3(UPD_THREADS), 0, st, pdl, ua);
  if (remove_mean && !lv.channel) {  // the channel's pressure is determined: no mean to remove
    const int nblk = div_up(lv.N * lv.N, 256) < 296 ? div_up(lv.N * lv.N, 256) : 296;
    launch_k(k_remove_mean, dim3(nblk), dim3(256), 0, st, true, lv.N, lv.n_partial, (const double*)partial_buf,
             w + 2 * lv.N * lv.N);
  }
}

// Set-up: one sweep of an additive level in the V-cycle's form (w nonzero, no mean removal)
// timed as separate kernels and as the fused cooperative kernel (two warm-up and five timed
// sweeps each, CUDA events), keeping the faster; both forms give the same bits.  force: 1 use
// the fused kernel wherever it can run, -1 never, 0 time both.
void choose_sweep_form(cav_hierarchy* H, Level& lv, int force, cudaStream_t st) {
  lv.fused = 0;
  lv.sweep_us[0] = lv.sweep_us[1] = 0.f;
  if (lv.n_big == 0 || lv.coloured || lv.coarsest || force < 0) return;
  const int l = (int)(&lv - &H->levels[0]);
  const size_t n3 = 3 * (size_t)lv.N * lv.N;
  CAV_CHECK_CUDA(cudaMemsetAsync(lv.x, 0, sizeof(double) * n3, st));
  CAV_CHECK_CUDA(cudaMemsetAsync(lv.b, 0, sizeof(double) * n3, st));
  if (!launch_fused_any(H, lv, lv.b, lv.x, false, lv.r, lv.r32, lv.delta, lv.partial, false, lv.apply_variant, st))
    return;
  if (force > 0) {
    lv.fused = 1;
    return;
  }
  cudaEvent_t e0, e1;
  CAV_CHECK_CUDA(cudaEventCreate(&e0));
  CAV_CHECK_CUDA(cudaEventCreate(&e1));
  for (int f = 0; f < 2; ++f) {
    lv.fused = f;
    for (int w = 0; w < 2; ++w) sweep_impl(H, l, lv.b, lv.x, false, lv.r, lv.r32, lv.delta, lv.partial, false, st, false);
    CAV_CHECK_CUDA(cudaEventRecord(e0, st));
    for (int w = 0; w < 5; ++w) sweep_impl(H, l, lv.b, lv.x, false, lv.r, lv.r32, lv.delta, lv.partial, false, st, false);
    CAV_CHECK_CUDA(cudaEventRecord(e1, st));
    CAV_CHECK_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    CAV_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    lv.sweep_us[f] = 1e3f * ms / 5.f;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  lv.fused = (lv.sweep_us[1] < lv.sweep_us[0]) ? 1 : 0;
}

void sweep_set_wait_stall(int enable) {
  CAV_CHECK_CUDA(cudaMemcpyToSymbol(g_wait_stall, &enable, sizeof(int)));
}

void level_sweep(const cav_hierarchy* H, int l, const double* b, double* w, bool w_is_zero, cudaStream_t st) {
  const Level& lv = H->levels[l];
  if (lv.coloured) {
    coloured_sweep(H, l, b, w, w_is_zero, lv.partial, true, true, st);
    return;
  }
  sweep_impl(H, l, b, w, w_is_zero, lv.r, lv.r32, lv.delta, lv.partial, true, st);
}

// Inside the V-cycle a constant pressure never changes a residual (G 1 = 0) or a patch
// correction (which depends on the residual only), and prolongation maps constants to
// constants, so removing the mean after every sweep (Sec. 3.3) and removing it once from the
// V-cycle's output give the same iterate up to rounding.  The cycle removes it once, using
// the partial sums the finest level's last sweep already produced.
static void cycle_sweep(const cav_hierarchy* H, int l, const double* b, double* w, bool w_is_zero,
                        cudaStream_t st, bool pdl_first) {
  const Level& lv = H->levels[l];
  if (lv.coloured) {
    coloured_sweep(H, l, b, w, w_is_zero, lv.partial, false, true, st);
    return;
  }
  sweep_impl(H, l, b, w, w_is_zero, lv.r, lv.r32, lv.delta, lv.partial, true, st, false, pdl_first);
}

void coarse_solve(const cav_hierarchy* H, const double* r, double* z, cudaStream_t st, bool pdl) {
  const Level& lv = H->levels.back();
  const int n = 3 * lv.N * lv.N;
  launch_k(k_coarse_apply, dim3(div_up(n, 8)), dim3(256), 0, st, pdl, n, lv.coarse_m,
           (const double*)lv.coarse_inv, r, z);
}

// One level of the V-cycle.  Every kernel after the first of the cycle follows another of its
// kernels on the stream (the coloured sweep's zeroing memset is followed by its first class
// step, launched without the attribute), so they are programmatic launches: each launch's
// latency hides under the kernel ahead of it.
static void vcycle_level(const cav_hierarchy* H, int l, const double* b, double* x, cudaStream_t st) {
  const Level& lv = H->levels[l];
  const bool pdl_in = l > 0;  // the finest level's first kernel is the cycle's first
  if (lv.coarsest) {
    coarse_solve(H, b, x, st, pdl_in);
    return;
  }
  const int NN = lv.N * lv.N;
  const int nu_pre = lv.nu_pre, nu_post = lv.nu_post;
  if (nu_pre == 0) CAV_CHECK_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * 3 * NN, st));
  for (int s = 0; s < nu_pre; ++s) cycle_sweep(H, l, b, x, s == 0, st, s > 0 || pdl_in);
  // after a coloured sweep of the finest level an event-record node may precede the residual
  const bool after_events = lv.coloured && prof_records(H, l);
  launch_apply(ops_of(lv), x, b, lv.r, 0, st, (nu_pre > 0 || pdl_in) && !after_events);
  const Level& lc = H->levels[l + 1];
  launch_restrict(lc.N, lv.r, lc.b, lv.channel, st, true);
  vcycle_level(H, l + 1, lc.b, lc.x, st);
  launch_prolong_add(lc.N, lc.x, x, lv.channel, st, true);
  for (int s = 0; s < nu_post; ++s) cycle_sweep(H, l, b, x, false, st, true);
  if (l == 0 && !lv.channel) {
    if (nu_post > 0 && lv.coloured) {
      pressure_mean_remove(lv.N, lv.partial, x + 2 * NN, st);
    } else if (nu_post > 0) {
      const int nblk = div_up(NN, 256) < 296 ? div_up(NN, 256) : 296;
      launch_k(k_remove_mean, dim3(nblk), dim3(256), 0, st, true, lv.N, lv.n_partial, (const double*)lv.partial,
               x + 2 * NN);
    } else {
      // nu_post = 0: the prolonged correction carries the coarse levels' pressure mean (they
      // skip the removal, which K_E cannot see); take the mean of x's pressure itself
      pressure_mean_remove(lv.N, lv.partial, x + 2 * NN, st);
    }
  }
}

// Capture the whole V-cycle (input levels[0].b, output levels[0].x) as CUDA graph instance g.
static bool vcycle_capture(cav_hierarchy* H, int g) {
  if (H->vc_exec[g]) return true;
  if (H->graph_failed) return false;
  if (!H->capture_stream) CAV_CHECK_CUDA(cudaStreamCreateWithFlags(&H->capture_stream, cudaStreamNonBlocking));
  const Level& l0 = H->levels[0];
  cudaGraph_t graph = nullptr;
  CAV_CHECK_CUDA(cudaStreamBeginCapture(H->capture_stream, cudaStreamCaptureModeThreadLocal));
  H->capturing = 1 + g;
  bool ok = true;
  const int64_t c0 = launch_count();
  try {
    vcycle_level(H, 0, l0.b, l0.x, H->capture_stream);
  } catch (...) {
    ok = false;
  }
  H->capturing = 0;
  H->vc_kernels[g] = (int)(launch_count() - c0);
  note_launches(-(long long)H->vc_kernels[g]);  // recorded, not run
  const cudaError_t e = cudaStreamEndCapture(H->capture_stream, &graph);
  if (!ok || e != cudaSuccess || !graph) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    H->graph_failed = 1;
    return false;
  }
  const cudaError_t e2 = cudaGraphInstantiate(&H->vc_exec[g], graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) {
    cudaGetLastError();
    H->vc_exec[g] = nullptr;
    H->graph_failed = 1;
    return false;
  }
  return true;
}

void vcycle(const cav_hierarchy* Hc, const double* r, double* z, cudaStream_t st) {
  cav_hierarchy* H = const_cast<cav_hierarchy*>(Hc);
  const int g = H->vc_next;
  if (!vcycle_capture(H, g)) {
    vcycle_level(H, 0, r, z, st);
    return;
  }
  H->vc_next ^= 1;
  const Level& l0 = H->levels[0];
  const size_t bytes = sizeof(double) * 3 * (size_t)l0.N * l0.N;
  CAV_CHECK_CUDA(cudaMemcpyAsync(l0.b, r, bytes, cudaMemcpyDeviceToDevice, st));
  CAV_CHECK_CUDA(cudaGraphLaunch(H->vc_exec[g], st));
  note_launches(H->vc_kernels[g]);
  CAV_CHECK_CUDA(cudaMemcpyAsync(z, l0.x, bytes, cudaMemcpyDeviceToDevice, st));
  if (H->prof_on) {
    const std::vector<cudaEvent_t>& ev = H->vc_ev[g];
    for (size_t q = 0; q + 1 < ev.size(); q += 2) {
      H->prof_pending.emplace_back(ev[q], ev[q + 1]);
      ++H->prof_pushed;
    }
  }
}

void vcycle_inline(const cav_hierarchy* H, cudaStream_t st) {
  const Level& l0 = H->levels[0];
  vcycle_level(H, 0, l0.b, l0.x, st);
}

void vcycle_prepare(cav_hierarchy* H) {
  vcycle_capture(H, 0);
  vcycle_capture(H, 1);
}

void vcycle_release(cav_hierarchy* H) {
  for (int g = 0; g < 2; ++g) {
    if (H->vc_exec[g]) cudaGraphExecDestroy(H->vc_exec[g]);
    H->vc_exec[g] = nullptr;
    for (auto& e : H->vc_ev[g]) cudaEventDestroy(e);
    H->vc_ev[g].clear();
  }
  if (H->capture_stream) cudaStreamDestroy(H->capture_stream);
  H->capture_stream = nullptr;
}

}  // namespace cav

// ------------------------------------------------------------------ allocation-free sweep
//
// cav_sweep keeps its scratch (the residual, the packed patch corrections and the partial
// sums of the pressure mean) in buffers that cav_setup allocated.  cav_sweep_noalloc runs
// the same kernels with that scratch taken from the fixed array below instead, so a caller
// can run a sweep without the library reserving per-hierarchy scratch for it.  The array is
// a file-scope device variable: every GPU that loads this library holds its 8 MiB until the
// process exits.  Host code cannot use the array's name as a device address; the address is
// looked up once per device with cudaGetSymbolAddress.

namespace cav {

static __device__ __align__(256) double g_noalloc_scratch[CAV_NOALLOC_SCRATCH_DOUBLES];
static std::mutex g_noalloc_mutex;
static double* g_noalloc_address[64] = {};

// Device address of the scratch array on the current device (looked up on first use).
static double* noalloc_scratch(int device) {
  CAV_REQUIRE(device >= 0 && device < 64, "cav_sweep_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_address[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_error(std::string("cav_sweep_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      throw Fail{IB_ERR_CUDA};
    }
    g_noalloc_address[device] = static_cast<double*>(p);
  }
  return g_noalloc_address[device];
}

static inline size_t round_up32(size_t n) { return (n + 31) & ~(size_t)31; }

// Rejects a level whose scratch would not fit in the fixed array, naming both sizes.
static void noalloc_require(int level, size_t need, const char* what) {
  if (need <= (size_t)CAV_NOALLOC_SCRATCH_DOUBLES) return;
  set_error("cav_sweep_noalloc: level " + std::to_string(level) + " needs " + std::to_string(need) +
            " doubles of scratch (" + what + "); the static array holds " +
            std::to_string((size_t)CAV_NOALLOC_SCRATCH_DOUBLES));
  throw Fail{IB_ERR_INVALID};
}

}  // namespace cav

extern "C" ib_status cav_sweep_noalloc(const cav_hierarchy* h, int32_t level, const double* b, double* w,
                                       cudaStream_t st) {
  using namespace cav;
  try {
    CAV_REQUIRE(h && b && w, "cav_sweep_noalloc: NULL argument");
    CAV_REQUIRE(level >= 0 && level < (int32_t)h->levels.size(), "cav_sweep_noalloc: level out of range");
    const Level& lv = h->levels[level];
    CAV_REQUIRE(!lv.coarsest, "cav_sweep_noalloc: no smoother on the coarsest level");
    int device = -1;
    CAV_CHECK_CUDA(cudaGetDevice(&device));
    CAV_REQUIRE(device == h->sys->device, "cav_sweep_noalloc: the current device is not the hierarchy's device");
    if (lv.coloured) {
      // the class-by-class sweep needs scratch only for the pressure mean's partial sums
      const size_t n_pc = round_up32((size_t)div_up((int64_t)lv.N * lv.N, 256));
      noalloc_require(level, n_pc, "partial sums of the pressure mean, rounded to 32");
      coloured_sweep(h, level, b, w, false, noalloc_scratch(device), true, false, st);
      return take_status(h->status, st, "cav_sweep_noalloc");
    }
    const size_t n_r = round_up32((size_t)3 * lv.N * lv.N);
    // FP32 / BF16 levels: the residual's FP32 copy, 3 N^2 floats in ceil(3 N^2 / 2) doubles
    const size_t n_r32 = lv.precision != CAV_PREC_FP64 ? round_up32((size_t)div_up(3LL * lv.N * lv.N, 2)) : 0;
    const size_t n_d = round_up32((size_t)lv.big_sum_n);
    const size_t n_p = round_up32((size_t)lv.n_partial);
    noalloc_require(level, n_r + n_r32 + n_d + n_p,
                    "3 N^2 + (FP32 and BF16 levels) 3 N^2 / 2 + enlarged-patch unknowns + partial sums, each "
                    "rounded to 32");
    double* base = noalloc_scratch(device);
    double* r = base;               // written in full by the residual kernel before any read
    float* r32 = n_r32 ? reinterpret_cast<float*>(base + n_r) : nullptr;  // likewise
    double* delta = base + n_r + n_r32;  // written in full by the patch-apply kernel before any read
                                         // (not read at all on a level without enlarged patches)
    double* partial = delta + n_d;  // written in full by the update kernels before any read
    // separate kernels: the fused one keeps per-level scratch of the hierarchy (its warp sums)
    sweep_impl(h, level, b, w, false, r, r32, delta, partial, false, st, true, false, false);
    return take_status(h->status, st, "cav_sweep_noalloc");
  } catch (const Fail& f) {
    return f.st;
  } catch (...) {
    set_error("cav_sweep_noalloc: internal error");
    return IB_ERR_INTERNAL;
  }
}
