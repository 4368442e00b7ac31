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
#include <mutex>
#include <set>
#include <string>
#include <utility>

#include "internal.cuh"
#include "device_util.cuh"
#include "level_math.cuh"
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

__device__ inline void consumer_sync(int nthreads) { asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory"); }

constexpr int TMA_CONSUMER_WARPS = 4;
constexpr int TMA_THREADS = 32 * (TMA_CONSUMER_WARPS + 2);  // producer, gatherer, consumers
constexpr int TMA_MAXPASS = 2;          // row passes per consumer thread
constexpr int Y_SLOTS = 2;

template <typename T>
__host__ __device__ constexpr int tma_max_rows() {
  return TMA_MAXPASS * 32 * TMA_CONSUMER_WARPS * VecLoad<T>::V;
}

// The q-th patch a persistent CTA takes (q = round * G + CTA): rounds alternate direction over
// the size-descending order, so every CTA gets a large and a small patch in each pair of
// rounds and their loads stay balanced.
__device__ inline int zigzag(int q, int G, int n) {
  const int r = q / G, c = q - r * G;
  const int len = min(G, n - r * G);
  return (r & 1) ? r * G + (len - 1 - c) : q;
}

// Persistent batched patch apply.  CTA c takes the patches zigzag(c), zigzag(c + G), ... of
// the size-descending order, with three roles:
//  * warp 0, one lane (producer): streams each patch's column-major inverse -- a contiguous
//    block of n * ld elements -- into a ring of TMA_STAGES shared-memory stages of at most
//    TMA_CHUNK bytes (whole columns) with cp.async.bulk; "full" mbarriers carry the
//    transaction bytes, "empty" mbarriers take one arrival per consumer warp;
//  * warp 1 (gatherer): writes y = s_r * r|_p of the coming patches into a double-buffered
//    shared ring ("yfull": 32 lane arrivals, "yempty": one arrival per consumer warp), so the
//    dependent index -> residual loads of patch t+1 overlap the streaming of patch t;
//  * warps 2..5 (consumers): acc[rows] += X[rows, b] y[b] stage by stage, each thread
//    owning V consecutive rows (up to TMA_MAXPASS row blocks), then delta = s_c * acc.
// Every wait is bounded.  A wait that runs out records DEV_TIMEOUT and raises the CTA's abort
// flag; every role then stops (no further copies, arrivals or writes; the delta of the
// remaining patches is left unwritten and the host reports IB_ERR_TIMEOUT), and the producer
// waits for the copies it has in flight to land before the CTA exits.  A warp's give-up
// decision is taken by all its lanes together.
template <typename T, int TMA_STAGES, int TMA_CHUNK>
__global__ void __launch_bounds__(TMA_THREADS)
k_patch_apply_tma(int n_big, const int* __restrict__ order, const int64_t* __restrict__ off,
                  const int* __restrict__ dofs, const int64_t* __restrict__ inv_off, const T* __restrict__ inv,
                  const double* __restrict__ s_r, const double* __restrict__ s_c, const double* __restrict__ r,
                  double* __restrict__ delta, int max_n, int* status) {
  typedef VecLoad<T> VL;
  typedef typename VL::acc_t acc_t;
  constexpr int V = VL::V;
  constexpr int CT = 32 * TMA_CONSUMER_WARPS;
  static_assert(TMA_STAGES <= 32, "stage bit masks");
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* stage_buf = smem;
  const size_t ybytes = ((size_t)max_n * sizeof(acc_t) + 127) & ~(size_t)127;
  acc_t* ybuf = reinterpret_cast<acc_t*>(smem + TMA_STAGES * TMA_CHUNK);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + TMA_STAGES * TMA_CHUNK + Y_SLOTS * ybytes);
  uint64_t* empty = full + TMA_STAGES;
  uint64_t* yfull = empty + TMA_STAGES;
  uint64_t* yempty = yfull + Y_SLOTS;
  int* abort_flag = reinterpret_cast<int*>(yempty + Y_SLOTS);
  volatile int* ab = abort_flag;
  const bool stall = wait_stall_enabled();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    *abort_flag = 0;
    for (int s = 0; s < TMA_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], TMA_CONSUMER_WARPS);
    }
    for (int s = 0; s < Y_SLOTS; ++s) {
      mbar_init(&yfull[s], 32);
      mbar_init(&yempty[s], TMA_CONSUMER_WARPS);
    }
    mbar_fence_init();
  }
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
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t used = 0, last_par = 0;  // per stage: a copy was issued; parity of its last phase
      bool ok = true;
      for (int q = blockIdx.x; ok && q < n_big; q += gridDim.x) {
        const int p = order[zigzag(q, gridDim.x, n_big)];
        const int n = (int)(off[p + 1] - off[p]);
        const uint32_t col_bytes = (uint32_t)(((n + 7) & ~7) * sizeof(T));
        const int cpc = TMA_CHUNK / (int)col_bytes;
        const unsigned char* src = reinterpret_cast<const unsigned char*>(inv + inv_off[p]);
        for (int b0 = 0; b0 < n; b0 += cpc) {
          const int nc = min(cpc, n - b0);
          if (!mbar_wait(&empty[stage], phase ^ 1u, status, ab, false)) {
            ok = false;
            break;
          }
          const uint32_t bytes = (uint32_t)nc * col_bytes;
          mbar_arrive_expect_tx(&full[stage], bytes);
          bulk_copy_g2s(stage_buf + (size_t)stage * TMA_CHUNK, src + (size_t)b0 * col_bytes, bytes, &full[stage]);
          used |= 1u << stage;
          last_par = phase ? (last_par | (1u << stage)) : (last_par & ~(1u << stage));
          if (++stage == TMA_STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // every issued copy lands before the CTA exits (immediate when the consumers saw them all)
      for (int s = 0; s < TMA_STAGES; ++s)
        if ((used >> s) & 1u) mbar_drain(&full[s], (last_par >> s) & 1u, status);
    }
    return;
  }

  if (warp == 1) {
    pdl_wait();
    int t = 0;
    for (int q = blockIdx.x; q < n_big; q += gridDim.x, ++t) {
      const int slot = t & 1;
      const uint32_t par = (uint32_t)((t >> 1) & 1);
      const bool got = mbar_wait(&yempty[slot], par ^ 1u, status, ab, false);
      if (!__all_sync(0xffffffffu, got)) break;
      const int p = order[zigzag(q, gridDim.x, n_big)];
      const int64_t d0 = off[p];
      const int n = (int)(off[p + 1] - d0);
      acc_t* y = ybuf + (size_t)slot * (ybytes / sizeof(acc_t));
      for (int b = lane; b < n; b += 32) y[b] = (acc_t)(s_r[d0 + b] * r[dofs[d0 + b]]);
      mbar_arrive(&yfull[slot]);
    }
    return;
  }

  const int ct = threadIdx.x - 64;
  int stage = 0;
  uint32_t phase = 0;
  int t = 0;
  for (int q = blockIdx.x; q < n_big; q += gridDim.x, ++t) {
    const int p = order[zigzag(q, gridDim.x, n_big)];
    const int64_t d0 = off[p];
    const int n = (int)(off[p + 1] - d0);
    const int ld = (n + 7) & ~7;
    const int cpc = TMA_CHUNK / (int)(ld * sizeof(T));
    const int slot = t & 1;
    if (!__all_sync(0xffffffffu, mbar_wait(&yfull[slot], (uint32_t)((t >> 1) & 1), status, ab, stall))) break;
    const acc_t* y = ybuf + (size_t)slot * (ybytes / sizeof(acc_t));
    acc_t acc[TMA_MAXPASS][V];
#pragma unroll
    for (int ps = 0; ps < TMA_MAXPASS; ++ps)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[ps][v] = 0;
    bool dead = false;
    for (int b0 = 0; b0 < n; b0 += cpc) {
      const int nc = min(cpc, n - b0);
      if (!__all_sync(0xffffffffu, mbar_wait(&full[stage], phase, status, ab, stall))) {
        dead = true;
        break;
      }
      const T* X = reinterpret_cast<const T*>(stage_buf + (size_t)stage * TMA_CHUNK);
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
      if (lane == 0) mbar_arrive(&empty[stage]);
      if (++stage == TMA_STAGES) {
        stage = 0;
        phase ^= 1u;
      }
    }
    if (dead) break;
    __syncwarp();
    if (lane == 0) mbar_arrive(&yempty[slot]);
#pragma unroll
    for (int ps = 0; ps < TMA_MAXPASS; ++ps) {
      const int a0 = (ps * CT + ct) * V;
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (a0 + v < n) delta[d0 + a0 + v] = s_c[d0 + a0 + v] * (double)acc[ps][v];
    }
  }
}

// ------------------------------------------------------------------ 3. scatter / update

constexpr int TOUCH_WARPS = 8;

// Scatter / update in one launch with two block roles.
//  * Blocks [0, nb_std): a 32 x 8 tile of cells, one thread per cell.  For each unknown of the
//    cell that no enlarged patch holds, both incident cells (one for a pressure) keep their
//    standard patch, so count_k is 2 (1) and the correction is the stencil of the shared 5x5
//    inverse applied to r.
//  * The remaining blocks: eight lanes per unknown held by at least one enlarged patch (four
//    unknowns per warp).  The lanes sum the enlarged patches' corrections at the unknown (fixed
//    lane-strided order, fixed shuffle tree); the group's first lane adds the standard patches
//    of its incident cells that kept their Vanka patch and divides by the total patch count.
// On the channel a v face of the outflow row has one incident cell (the one above it), and
// the standard patches of the outflow and inflow rows have their own inverses.
// Each block writes the partial sum of the new pressures it produced (fixed order); the
// stencil blocks' partials come first, then the touched blocks'.
__global__ void __launch_bounds__(256)
k_update(int N, double alpha, StdInv S, int nb_std, int gx, const int64_t* __restrict__ inc_off,
         int n_touched, const int* __restrict__ touched, const uint8_t* __restrict__ cell_big,
         const int* __restrict__ inc_slot, const double* __restrict__ delta, const double* __restrict__ r,
         double* __restrict__ w, int w_is_zero, double* __restrict__ partial, bool channel) {
  pdl_wait();  // programmatic launch: the patch apply (delta) and residual (r) have finished
  pdl_trigger();
  __shared__ double sm[8];
  const int NN = N * N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double pnew = 0.0;
  if ((int)blockIdx.x < nb_std) {
    const int i = (blockIdx.x % gx) * 32 + lane;
    const int j = (blockIdx.x / gx) * 8 + warp;
    if (i < N && j < N) {
      const int c = j * N + i;
      const int im = (i == 0) ? N - 1 : i - 1, jm = (j == 0) ? N - 1 : j - 1;
      if (inc_off[c + 1] == inc_off[c]) {
        const double s = std_row(S, 1, r, N, im, j, channel) + std_row(S, 0, r, N, i, j, channel);
        w[c] = (w_is_zero ? 0.0 : w[c]) + alpha * (s / 2.0);
      }
      if (inc_off[NN + c + 1] == inc_off[NN + c]) {
        if (channel && j == 0) {  // the outflow row's v face: one incident cell
          const double s = std_row(S, 2, r, N, i, j, channel);
          w[NN + c] = (w_is_zero ? 0.0 : w[NN + c]) + alpha * s;
        } else {
          const double s = std_row(S, 3, r, N, i, jm, channel) + std_row(S, 2, r, N, i, j, channel);
          w[NN + c] = (w_is_zero ? 0.0 : w[NN + c]) + alpha * (s / 2.0);
        }
      }
      if (inc_off[2 * NN + c + 1] == inc_off[2 * NN + c]) {
        const double s = std_row(S, 4, r, N, i, j, channel);
        pnew = (w_is_zero ? 0.0 : w[2 * NN + c]) + alpha * s;
        w[2 * NN + c] = pnew;
      }
    }
    pnew = warp_sum(pnew);
  } else {
    const int sub = lane / TOUCH_LANES, sl = lane % TOUCH_LANES;
    const int t = (((int)blockIdx.x - nb_std) * TOUCH_WARPS + warp) * TOUCH_PER_WARP + sub;
    double s = 0.0;
    int k = -1;
    int64_t q0 = 0, q1 = 0;
    if (t < n_touched) {
      k = touched[t];
      q0 = inc_off[k];
      q1 = inc_off[k + 1];
      for (int64_t q = q0 + sl; q < q1; q += TOUCH_LANES) s += delta[inc_slot[q]];
    }
#pragma unroll
    for (int o = TOUCH_LANES / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (k >= 0) {
      if (sl == 0) {
        const int comp = k / NN, c = k % NN, i = c % N, j = c / N;
        const int im = (i == 0) ? N - 1 : i - 1, jm = (j == 0) ? N - 1 : j - 1;
        int cnt = (int)(q1 - q0);
        double st = 0.0;
        if (comp == 0) {
          if (!cell_big[j * N + im]) { st += std_row(S, 1, r, N, im, j, channel); ++cnt; }
          if (!cell_big[c]) { st += std_row(S, 0, r, N, i, j, channel); ++cnt; }
        } else if (comp == 1) {
          if (!(channel && j == 0) && !cell_big[jm * N + i]) { st += std_row(S, 3, r, N, i, jm, channel); ++cnt; }
          if (!cell_big[c]) { st += std_row(S, 2, r, N, i, j, channel); ++cnt; }
        } else {
          if (!cell_big[c]) { st += std_row(S, 4, r, N, i, j, channel); ++cnt; }
        }
        const double nw = (w_is_zero ? 0.0 : w[k]) + alpha * ((st + s) / (double)cnt);
        w[k] = nw;
        if (comp == 2) pnew = nw;
      }
    }
    // the warp's new pressures: group leaders' values in fixed order
    double wp = 0.0;
#pragma unroll
    for (int g = 0; g < TOUCH_PER_WARP; ++g) wp += __shfl_sync(0xffffffffu, pnew, g * TOUCH_LANES);
    pnew = wp;
  }
  if (lane == 0) sm[warp] = pnew;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int q = 0; q < 8; ++q) tot += sm[q];
    partial[blockIdx.x] = tot;
  }
}

// 4. p -= mean(p): every block reduces the partials in the same order, then subtracts.
__global__ void k_remove_mean(int N, int n_partial, const double* __restrict__ partial, double* __restrict__ p) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sm[8];
  double t = 0.0;
  for (int q = threadIdx.x; q < n_partial; q += blockDim.x) t += partial[q];
  t = block_sum(t, sm);
  const double mean = t / ((double)N * (double)N);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N * N; c += gridDim.x * blockDim.x) p[c] -= mean;
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
  if (level != 0) return false;
  return H->capturing || (H->prof_on && (size_t)(2 * H->prof_used + 1) < H->prof_ev.size());
}

void prof_begin(const cav_hierarchy* H, int level, cudaStream_t st) {
  cav_hierarchy* h = const_cast<cav_hierarchy*>(H);
  if (level != 0) return;
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
  if (level != 0) return;
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

template <typename T, int STAGES, int CHUNK>
static void launch_tma(const cav_hierarchy* H, const Level& lv, const T* inv, const double* r, double* delta,
                       int ctas_per_sm, cudaStream_t st, bool pdl) {
  typedef typename VecLoad<T>::acc_t acc_t;
  const size_t ybytes = ((size_t)lv.big_max_n * sizeof(acc_t) + 127) & ~(size_t)127;
  const size_t smem = (size_t)STAGES * CHUNK + Y_SLOTS * ybytes + (2 * STAGES + 2 * Y_SLOTS) * sizeof(uint64_t) +
                      16;  // the CTA's abort flag
  allow_dynamic_smem(reinterpret_cast<const void*>(k_patch_apply_tma<T, STAGES, CHUNK>), 200 * 1024);
  const int grid = std::min(lv.n_big, ctas_per_sm * sm_count());
  launch_k(k_patch_apply_tma<T, STAGES, CHUNK>, dim3(grid), dim3(TMA_THREADS), smem, st, pdl, lv.n_big, lv.order,
           lv.big_off, lv.big_dofs, lv.inv_off, inv, lv.s_r, lv.s_c, r, delta, lv.big_max_n, H->status);
}

// Can variant v run this level?  (rows per consumer thread and one whole column per stage)
template <typename T>
static bool variant_fits(const Level& lv, int v) {
  if (kVariants[v].stages == 0) return true;
  return lv.big_max_n <= tma_max_rows<T>() && (size_t)round8(lv.big_max_n) * sizeof(T) <= (size_t)kVariants[v].chunk;
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

// The four steps of one sweep with explicit scratch (residual r_buf, packed corrections
// delta_buf, partial sums partial_buf); shared by cav_sweep and cav_sweep_noalloc.
// pdl_first: the operation ahead of the sweep's first kernel on st is one of this library's
// kernels, so it may be a programmatic launch (the kernels after it are, except around the
// finest level's profiling events, whose record nodes sit between the kernels).
static void sweep_impl(const cav_hierarchy* H, int l, const double* b, double* w, bool w_is_zero, double* r_buf,
                       double* delta_buf, double* partial_buf, bool profile, cudaStream_t st,
                       bool remove_mean = true, bool pdl_first = false) {
  const Level& lv = H->levels[l];
  const double* r = b;
  const bool events = profile && prof_records(H, l);
  bool pdl = pdl_first;
  if (!w_is_zero) {
    launch_apply(ops_of(lv), w, b, r_buf, 0, st, pdl);
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
  StdInv S;
  for (int k = 0; k < 3; ++k)
    for (int q = 0; q < 25; ++q) S.m[k][q] = lv.std_inv[k][q];
  const int gx = div_up(lv.N, 32), gy = div_up(lv.N, 8);
  const int nb_std = gx * gy;
  const int nb_touch = div_up(lv.n_touched, TOUCH_WARPS * TOUCH_PER_WARP);
  launch_k(k_update, dim3(nb_std + nb_touch), dim3(256), 0, st, pdl, lv.N, H->desc.alpha, S, nb_std, gx, lv.inc_off,
           lv.n_touched, lv.touched, lv.cell_big, lv.inc_slot, delta_buf, r, w, w_is_zero ? 1 : 0, partial_buf,
           lv.channel);
  if (remove_mean && !lv.channel) {  // the channel's pressure is determined: no mean to remove
    const int nblk = div_up(lv.N * lv.N, 256) < 296 ? div_up(lv.N * lv.N, 256) : 296;
    launch_k(k_remove_mean, dim3(nblk), dim3(256), 0, st, true, lv.N, lv.n_partial, (const double*)partial_buf,
             w + 2 * lv.N * lv.N);
  }
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
  sweep_impl(H, l, b, w, w_is_zero, lv.r, lv.delta, lv.partial, true, st);
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
  sweep_impl(H, l, b, w, w_is_zero, lv.r, lv.delta, lv.partial, true, st, false, pdl_first);
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
      level_sweep(H, l, b, x, false, st);  // nu_post = 0: one more full sweep to fix the gauge
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
  try {
    vcycle_level(H, 0, l0.b, l0.x, H->capture_stream);
  } catch (...) {
    ok = false;
  }
  H->capturing = 0;
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
  note_launch();
  CAV_CHECK_CUDA(cudaMemcpyAsync(z, l0.x, bytes, cudaMemcpyDeviceToDevice, st));
  if (H->prof_on) {
    const std::vector<cudaEvent_t>& ev = H->vc_ev[g];
    for (size_t q = 0; q + 1 < ev.size(); q += 2) {
      H->prof_pending.emplace_back(ev[q], ev[q + 1]);
      ++H->prof_pushed;
    }
  }
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
    const size_t n_d = round_up32((size_t)lv.big_sum_n);
    const size_t n_p = round_up32((size_t)lv.n_partial);
    noalloc_require(level, n_r + n_d + n_p,
                    "3 N^2 + enlarged-patch unknowns + partial sums, each rounded to 32");
    double* base = noalloc_scratch(device);
    double* r = base;               // written in full by the residual kernel before any read
    double* delta = base + n_r;     // written in full by the patch-apply kernel before any read
                                    // (not read at all on a level without enlarged patches)
    double* partial = delta + n_d;  // written in full by the update kernels before any read
    sweep_impl(h, level, b, w, false, r, delta, partial, false, st);
    return take_status(h->status, st, "cav_sweep_noalloc");
  } catch (const Fail& f) {
    return f.st;
  } catch (...) {
    set_error("cav_sweep_noalloc: internal error");
    return IB_ERR_INTERNAL;
  }
}
