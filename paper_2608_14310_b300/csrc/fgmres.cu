// Right-preconditioned flexible GMRES (Sec. 5) on the device.
//
// Arnoldi uses classical Gram-Schmidt applied twice (CGS2): each pass computes all k+1
// inner products in one launch and subtracts them in one launch, so an iteration costs a
// fixed handful of kernels instead of 2k.  Every reduction is two-stage with a fixed
// partition and order, so results are bitwise reproducible.  The Hessenberg column, the
// Givens rotations and the residual estimate live on the device; the host reads one small
// record per iteration to test convergence.
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "device_util.cuh"

namespace cav {

static constexpr int FG_THREADS = 256;

// The Arnoldi kernels are bound by the FP64 pipe as much as by HBM (on this part one FP64
// FMA per 8-byte element already asks for more FP64 issue than the SMs have at full memory
// bandwidth), so they keep FP64 work other than the products to a minimum.  A block owns a
// chunk of the vectors; a thread owns the elements tid, tid + 256, ... of that chunk
// (coalesced).

// Inner products: 4 elements per thread, 8 vectors per block.
constexpr int DOT_PER_THREAD = 4, DOT_CHUNK = FG_THREADS * DOT_PER_THREAD, DOT_GROUP = 8;
// Combinations: 2 elements per thread (more blocks, more loads in flight per SM).
constexpr int CMB_PER_THREAD = 2, CMB_CHUNK = FG_THREADS * CMB_PER_THREAD;

static int dot_blocks(int64_t n) { return (int)((n + DOT_CHUNK - 1) / DOT_CHUNK); }
static int cmb_blocks(int64_t n) { return (int)((n + CMB_CHUNK - 1) / CMB_CHUNK); }

// Warp reduction of 8 values per lane in 9 additions (not 8 x 5): three exchange steps halve
// the number of values a lane carries, two plain steps finish.  Lane L with L % 4 == 0 ends
// holding the warp sum of value L / 4.  The pattern is fixed, so the result is reproducible.
__device__ inline double warp_sum8_transposed(double* v) {
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double send = b4 ? v[q] : v[q + 4], keep = b4 ? v[q + 4] : v[q];
    v[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double send = b3 ? v[q] : v[q + 2], keep = b3 ? v[q + 2] : v[q];
    v[q] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const double send = b2 ? v[0] : v[1], keep = b2 ? v[1] : v[0];
  double t = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  t += __shfl_xor_sync(0xffffffffu, t, 2);
  t += __shfl_xor_sync(0xffffffffu, t, 1);
  return t;
}

// partial[i * gridDim.x + bx] = chunk bx's share of <V_i, w> for i < kcount.  Block (bx, g)
// takes vectors 8g .. 8g+7, so w is read once per eight vectors; per vector the chunk's sum
// is a fixed per-warp tree, then the eight warp sums in warp order.  kdev (nullable): kcount
// = *kdev + 1, the iteration index read from device memory (a graph's fixed grid covers
// every iteration; blocks past kcount exit).
__global__ void __launch_bounds__(FG_THREADS)
k_multi_dot(const double* __restrict__ V, int64_t n, int kcount, const double* __restrict__ w,
            double* __restrict__ partial, const int* __restrict__ kdev) {
  pdl_wait();  // programmatic launch: the kernel ahead (which writes w or V) has finished
  pdl_trigger();
  if (kdev) kcount = *kdev + 1;
  if ((int)blockIdx.y * DOT_GROUP >= kcount) return;
  __shared__ double sm[DOT_GROUP][FG_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * DOT_CHUNK + threadIdx.x;
  double wr[DOT_PER_THREAD];
#pragma unroll
  for (int j = 0; j < DOT_PER_THREAD; ++j) {
    const int64_t e = base + j * FG_THREADS;
    wr[j] = (e < n) ? w[e] : 0.0;
  }
  const int i0 = blockIdx.y * DOT_GROUP;
  double s[DOT_GROUP];
  if (i0 + DOT_GROUP <= kcount && base + (DOT_PER_THREAD - 1) * FG_THREADS < n) {
#pragma unroll
    for (int v = 0; v < DOT_GROUP; ++v) {
      const double* vi = V + (int64_t)(i0 + v) * n + base;
      double a = 0.0;
#pragma unroll
      for (int j = 0; j < DOT_PER_THREAD; ++j) a += vi[j * FG_THREADS] * wr[j];
      s[v] = a;
    }
  } else {
#pragma unroll
    for (int v = 0; v < DOT_GROUP; ++v) {
      s[v] = 0.0;
      if (i0 + v < kcount) {
        const double* vi = V + (int64_t)(i0 + v) * n;
#pragma unroll
        for (int j = 0; j < DOT_PER_THREAD; ++j) {
          const int64_t e = base + j * FG_THREADS;
          if (e < n) s[v] += vi[e] * wr[j];
        }
      }
    }
  }
  const double t = warp_sum8_transposed(s);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if ((lane & 3) == 0) sm[lane >> 2][warp] = t;
  __syncthreads();
  if (threadIdx.x < DOT_GROUP && i0 + (int)threadIdx.x < kcount) {
    double u = 0.0;
#pragma unroll
    for (int q = 0; q < FG_THREADS / 32; ++q) u += sm[threadIdx.x][q];
    partial[(int64_t)(i0 + threadIdx.x) * gridDim.x + blockIdx.x] = u;
  }
}

// out[i] = sum_b partial[i * nb + b] (fixed order); add_to (nullable) += out.  kdev
// (nullable): only blocks i <= *kdev run, and add_to is offset by *kdev * add_stride.
__global__ void k_finalize(const double* __restrict__ partial, int nb, double* out, double* add_to,
                           const int* __restrict__ kdev, int64_t add_stride) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sm[FG_THREADS / 32];
  const int i = blockIdx.x;
  if (kdev) {
    const int k = *kdev;
    if (i > k) return;
    if (add_to) add_to += (int64_t)k * add_stride;
  }
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partial[(int64_t)i * nb + b];
  s = block_sum(s, sm);
  if (threadIdx.x == 0) {
    out[i] = s;
    if (add_to) add_to[i] += s;
  }
}

// SIGN = -1: w -= sum_{i < kcount} c[i] V_i;  SIGN = +1: w += sum_{i < kcount} c[i] V_i.
// Per element the sum runs over i in ascending order.  sq_partial (nullable) receives the
// chunk's share of ||w_new||^2 (block_sum order).
// kdev (nullable): kcount = *kdev + kadd.
template <int SIGN>
__global__ void __launch_bounds__(FG_THREADS)
k_combine(const double* __restrict__ V, int64_t n, int kcount, const double* __restrict__ c,
          double* __restrict__ w, double* __restrict__ sq_partial, const int* __restrict__ kdev, int kadd) {
  pdl_wait();
  pdl_trigger();
  if (kdev) kcount = *kdev + kadd;
  __shared__ double sm[FG_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * CMB_CHUNK + threadIdx.x;
  double acc[CMB_PER_THREAD];
#pragma unroll
  for (int j = 0; j < CMB_PER_THREAD; ++j) acc[j] = 0.0;
  if (base + (CMB_PER_THREAD - 1) * FG_THREADS < n) {
#pragma unroll 4
    for (int i = 0; i < kcount; ++i) {
      const double ci = c[i];
      const double* vi = V + (int64_t)i * n + base;
#pragma unroll
      for (int j = 0; j < CMB_PER_THREAD; ++j) acc[j] += ci * vi[j * FG_THREADS];
    }
  } else {
    for (int i = 0; i < kcount; ++i) {
      const double ci = c[i];
      const double* vi = V + (int64_t)i * n;
#pragma unroll
      for (int j = 0; j < CMB_PER_THREAD; ++j) {
        const int64_t e = base + j * FG_THREADS;
        if (e < n) acc[j] += ci * vi[e];
      }
    }
  }
  double sq = 0.0;
#pragma unroll
  for (int j = 0; j < CMB_PER_THREAD; ++j) {
    const int64_t e = base + j * FG_THREADS;
    if (e < n) {
      const double wn = (SIGN < 0) ? w[e] - acc[j] : w[e] + acc[j];
      w[e] = wn;
      sq += wn * wn;
    }
  }
  if (sq_partial) {
    sq = block_sum(sq, sm);
    if (threadIdx.x == 0) sq_partial[blockIdx.x] = sq;
  }
}

// v = w * scale[0]
__global__ void k_scale(const double* __restrict__ w, int64_t n, const double* __restrict__ scale,
                        double* __restrict__ v) {
  pdl_wait();
  pdl_trigger();
  const double s = scale[0];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    v[e] = w[e] * s;
}

// Scalars layout (doubles): H[(maxit+1) * maxit] column-major, cs[maxit], sn[maxit],
// g[maxit+1], y[maxit], h[maxit+1] (CGS pass), misc[16].
struct FgLayout {
  int maxit;
  int64_t H, cs, sn, g, y, h, misc, total;
  explicit FgLayout(int m) : maxit(m) {
    H = 0;
    cs = H + (int64_t)(m + 1) * m;
    sn = cs + m;
    g = sn + m;
    y = g + m + 1;
    h = y + m;
    misc = h + m + 1;
    total = misc + 16;
  }
};
// misc: [0] ||b||^2, [1] ||r0||^2, [2] ||w||^2, [3] 1/beta, [4] |g_{k+1}|, [5] 1/h_{k+1,k}

__global__ void k_init_beta(double* S, FgLayout L) {
  double* misc = S + L.misc;
  const double beta = sqrt(misc[1]);
  misc[3] = (beta > 0.0) ? 1.0 / beta : 0.0;
  S[L.g] = beta;
}

// Hessenberg column k: apply the k earlier rotations, form rotation k, update g (Sec. 5).
// The rotations are a serial chain; the column and the rotation pairs are staged in shared
// memory first (all threads), so the chain runs on shared-memory latency, not L2 latency.
constexpr int GIVENS_SMEM_MAX = 1024;
__global__ void k_givens(double* S, FgLayout L, int k, const int* __restrict__ kdev) {
  pdl_wait();
  pdl_trigger();
  if (kdev) k = *kdev;
  __shared__ double sh[3 * GIVENS_SMEM_MAX];
  double* Hg = S + L.H + (int64_t)k * (L.maxit + 1);
  double* csg = S + L.cs;
  double* sng = S + L.sn;
  double* g = S + L.g;
  double* misc = S + L.misc;
  const bool staged = k + 2 <= GIVENS_SMEM_MAX;
  double* Hk = staged ? sh : Hg;
  double* cs = staged ? sh + GIVENS_SMEM_MAX : csg;
  double* sn = staged ? sh + 2 * GIVENS_SMEM_MAX : sng;
  if (staged) {
    for (int i = threadIdx.x; i <= k; i += blockDim.x) {
      Hk[i] = Hg[i];
      if (i < k) {
        cs[i] = csg[i];
        sn[i] = sng[i];
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double vnorm = sqrt(misc[2]);
    Hk[k + 1] = vnorm;
    for (int i = 0; i < k; ++i) {
      const double t = cs[i] * Hk[i] + sn[i] * Hk[i + 1];
      Hk[i + 1] = -sn[i] * Hk[i] + cs[i] * Hk[i + 1];
      Hk[i] = t;
    }
    const double d = hypot(Hk[k], Hk[k + 1]);
    const double c = (d != 0.0) ? Hk[k] / d : 1.0;
    const double sk = (d != 0.0) ? Hk[k + 1] / d : 0.0;
    csg[k] = c;
    sng[k] = sk;
    Hk[k] = d;
    Hk[k + 1] = 0.0;
    g[k + 1] = -sk * g[k];
    g[k] = c * g[k];
    misc[4] = fabs(g[k + 1]);
    misc[5] = (vnorm > 0.0) ? 1.0 / vnorm : 0.0;
  }
  __syncthreads();
  if (staged)
    for (int i = threadIdx.x; i <= k + 1; i += blockDim.x) Hg[i] = Hk[i];
}

__global__ void k_trisolve(double* S, FgLayout L, int k, const int* __restrict__ kdev) {
  pdl_wait();
  pdl_trigger();
  if (kdev) k = *kdev;
  const double* H = S + L.H;
  const double* g = S + L.g;
  double* y = S + L.y;
  const int ld = L.maxit + 1;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int j = i + 1; j < k; ++j) s -= H[(int64_t)j * ld + i] * y[j];
    y[i] = s / H[(int64_t)i * ld + i];
  }
}

static int vec_blocks(int64_t n) {
  int nb = div_up(n, FG_THREADS * 4);
  return nb < 1 ? 1 : (nb > 1184 ? 1184 : nb);
}

static void ensure_workspace(cav_hierarchy* H, int maxit, int64_t n) {
  if (H->ws_maxit >= maxit) return;
  if (H->host_b) cudaFreeHost(H->host_b);
  H->host_b = nullptr;
  if (H->dl_host) cudaFreeHost(H->dl_host);
  H->dl_host = nullptr;
  dl_plan_free(H->dl_plan);  // its graph refers to the buffers released below
  H->dl_plan = nullptr;
  H->ws_arena.release();
  H->V = H->ws_arena.alloc<double>((size_t)(maxit + 1) * n);
  H->Z = H->ws_arena.alloc<double>((size_t)maxit * n);
  FgLayout L(maxit);
  H->dev_scalars = H->ws_arena.alloc<double>(L.total);
  int nbmax = reduce_blocks(n);
  if (dot_blocks(n) > nbmax) nbmax = dot_blocks(n);
  if (cmb_blocks(n) > nbmax) nbmax = cmb_blocks(n);
  H->red_partial = H->ws_arena.alloc<double>((size_t)(maxit + 2) * nbmax);
  H->io_b = H->ws_arena.alloc<double>(n);
  H->io_x = H->ws_arena.alloc<double>(n);
  H->dl_w = H->ws_arena.alloc<double>(n);
  H->dl_kc = H->ws_arena.alloc<int>(8);
  H->dl_hist = H->ws_arena.alloc<double>((size_t)maxit + 1);
  CAV_CHECK_CUDA(cudaMallocHost(&H->dl_host, sizeof(double) * (32 + (size_t)maxit + 1)));
  if (!H->fg_ev[0]) {
    CAV_CHECK_CUDA(cudaEventCreateWithFlags(&H->fg_ev[0], cudaEventDisableTiming));
    CAV_CHECK_CUDA(cudaEventCreateWithFlags(&H->fg_ev[1], cudaEventDisableTiming));
  }
  CAV_CHECK_CUDA(cudaMallocHost(&H->host_b, sizeof(double) * 16));
  H->ws_maxit = maxit;
}

void krylov_reserve(cav_hierarchy* H, int maxit, int64_t n) { ensure_workspace(H, maxit, n); }

static void dot_to(const cav_hierarchy* H, const double* a, const double* b, int64_t n, double* out,
                   cudaStream_t st) {
  const int nb = dot_blocks(n);
  k_multi_dot<<<dim3(nb, 1), FG_THREADS, 0, st>>>(a, n, 1, b, H->red_partial, nullptr);
  CAV_CHECK_LAUNCH();
  k_finalize<<<1, FG_THREADS, 0, st>>>(H->red_partial, nb, out, nullptr, nullptr, 0);
  CAV_CHECK_LAUNCH();
}

// One system's solve as a sequence of host steps, so that a batched call can advance many
// systems in lockstep, each on its own stream:
//   fg_start        r0 = b - K x, ||b||^2, ||r0||^2 (queued)
//   fg_begin        read the norms (after a sync), set V_0 = r0 / beta
//   fg_issue(k)     iteration k: V-cycle, K z, CGS2, ||w||, Givens, scale, record
//   fg_check(k)     wait for iteration k's record and test convergence
//   fg_finish       y = H^-1 g, x += Z y, true residual (queued); fg_result after a sync
struct FgState {
  const ib_system* sys = nullptr;
  cav_hierarchy* H = nullptr;
  const fgmres_desc* d = nullptr;
  fgmres_info* info = nullptr;
  double* history = nullptr;
  cudaStream_t st = nullptr;
  const double* b_user = nullptr;
  double* x_user = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  int64_t n = 0;
  FgLayout L{1};
  LevelOps op{};
  int nb = 0, cb = 0, nbmax = 0, vb = 0;
  double ref = 0, beta = 0, est = 0;
  int k_done = 0, pending = -1;
  bool converged = false, active = false;
  int nonfinite = -1;  // iteration whose residual estimate was not finite (-1: none)
  long long prof_mark[2] = {0, 0};
};

static void fg_start(FgState& s) {
  cav_hierarchy* H = s.H;
  const Level& l0 = H->levels[0];
  s.n = 3LL * l0.N * l0.N;
  ensure_workspace(H, s.d->maxit, s.n);
  s.L = FgLayout(s.d->maxit);
  s.b = s.b_user;
  s.x = s.x_user;
  if (s.d->host_io) {
    CAV_CHECK_CUDA(cudaMemcpyAsync(H->io_b, s.b_user, sizeof(double) * s.n, cudaMemcpyHostToDevice, s.st));
    CAV_CHECK_CUDA(cudaMemcpyAsync(H->io_x, s.x_user, sizeof(double) * s.n, cudaMemcpyHostToDevice, s.st));
    s.b = H->io_b;
    s.x = H->io_x;
  }
  double* S = H->dev_scalars;
  CAV_CHECK_CUDA(cudaMemsetAsync(S, 0, sizeof(double) * s.L.total, s.st));
  // the Krylov operator is the system's current K_E; the hierarchy only preconditions (it may
  // have been built from an earlier configuration of the same system)
  s.op = LevelOps{l0.N, l0.h, l0.rho_dt, l0.mu, l0.dt, &s.sys->ee, l0.channel};
  s.nb = dot_blocks(s.n);
  s.cb = cmb_blocks(s.n);
  s.nbmax = s.nb > s.cb ? s.nb : s.cb;
  if (reduce_blocks(s.n) > s.nbmax) s.nbmax = reduce_blocks(s.n);
  s.vb = vec_blocks(s.n);
  double* misc = S + s.L.misc;
  launch_apply(s.op, s.x, s.b, H->V, 0, s.st);  // r0 -> V_0
  dot_to(H, s.b, s.b, s.n, misc + 0, s.st);
  dot_to(H, H->V, H->V, s.n, misc + 1, s.st);
  k_init_beta<<<1, 1, 0, s.st>>>(S, s.L);
  CAV_CHECK_LAUNCH();
  CAV_CHECK_CUDA(cudaMemcpyAsync(H->host_b, misc, sizeof(double) * 2, cudaMemcpyDeviceToHost, s.st));
}

// after the stream has been synchronised
static void fg_begin(FgState& s) {
  cav_hierarchy* H = s.H;
  const double bnorm = std::sqrt(H->host_b[0]);
  s.beta = std::sqrt(H->host_b[1]);
  s.ref = (s.d->rel_to == 1) ? s.beta : bnorm;
  s.est = (s.ref > 0) ? s.beta / s.ref : 0.0;
  if (s.history) s.history[0] = s.est;
  s.k_done = 0;
  s.pending = -1;
  if (!(s.ref > 0.0) || s.beta <= s.d->rtol * s.ref) {
    s.converged = true;
    s.active = false;
    return;
  }
  s.active = true;
  k_scale<<<s.vb, FG_THREADS, 0, s.st>>>(H->V, s.n, H->dev_scalars + s.L.misc + 3, H->V);
  CAV_CHECK_LAUNCH();
}

static void fg_issue(FgState& s, int k) {
  cav_hierarchy* H = s.H;
  const int64_t n = s.n;
  const int maxit = s.d->maxit;
  double* S = H->dev_scalars;
  double* misc = S + s.L.misc;
  double* vk = H->V + (int64_t)k * n;
  double* zk = H->Z + (int64_t)k * n;
  double* w = H->V + (int64_t)(k + 1) * n;
  vcycle(H, vk, zk, s.st);
  launch_apply(s.op, zk, nullptr, w, 1, s.st);
  // the second pass's update also yields the chunk sums of ||w||^2 (after the dot partials);
  // every kernel below follows another of these kernels: programmatic launches
  double* sq_partial = H->red_partial + (int64_t)(maxit + 1) * s.nbmax;
  const double* Vc = H->V;
  for (int pass = 0; pass < 2; ++pass) {
    launch_k(k_multi_dot, dim3(s.nb, div_up(k + 1, DOT_GROUP)), dim3(FG_THREADS), 0, s.st, true, Vc, n, k + 1,
             (const double*)w, H->red_partial, (const int*)nullptr);
    launch_k(k_finalize, dim3(k + 1), dim3(FG_THREADS), 0, s.st, true, (const double*)H->red_partial, s.nb,
             S + s.L.h, S + s.L.H + (int64_t)k * (maxit + 1), (const int*)nullptr, (int64_t)0);
    launch_k(k_combine<-1>, dim3(s.cb), dim3(FG_THREADS), 0, s.st, true, Vc, n, k + 1, (const double*)(S + s.L.h),
             w, pass == 1 ? sq_partial : nullptr, (const int*)nullptr, 0);
  }
  launch_k(k_finalize, dim3(1), dim3(FG_THREADS), 0, s.st, true, (const double*)sq_partial, s.cb, misc + 2,
           (double*)nullptr, (const int*)nullptr, (int64_t)0);
  launch_k(k_givens, dim3(1), dim3(128), 0, s.st, true, S, s.L, k, (const int*)nullptr);
  launch_k(k_scale, dim3(s.vb), dim3(FG_THREADS), 0, s.st, true, (const double*)w, n, (const double*)(misc + 5), w);
  CAV_CHECK_CUDA(cudaMemcpyAsync(H->host_b + 8 + (k & 1), misc + 4, sizeof(double), cudaMemcpyDeviceToHost, s.st));
  CAV_CHECK_CUDA(cudaEventRecord(H->fg_ev[k & 1], s.st));
  s.prof_mark[k & 1] = H->prof_pushed;
}

static bool fg_check(FgState& s, int kk) {
  cav_hierarchy* H = s.H;
  CAV_CHECK_CUDA(cudaEventSynchronize(H->fg_ev[kk & 1]));
  if (H->prof_on) prof_collect(H, s.prof_mark[kk & 1]);
  if (!std::isfinite(H->host_b[8 + (kk & 1)])) {
    // the preconditioned vector of iteration kk was not finite: stop, keeping the iterate
    // of the kk iterations before it (their Hessenberg columns are finite)
    s.nonfinite = kk;
    s.k_done = kk;
    return false;
  }
  s.k_done = kk + 1;
  s.est = H->host_b[8 + (kk & 1)] / s.ref;
  if (s.history) s.history[kk + 1] = s.est;
  return H->host_b[8 + (kk & 1)] <= s.d->rtol * s.ref;
}

// Advance one system by one iteration in the lockstep: issue iteration k, then read the
// previous iteration's convergence record while iteration k is queued (if iteration k - 1
// converged, iteration k's work is discarded -- it writes only Hessenberg column k, Givens
// pair k, g[k..k+1], V_{k+1} and Z_k, none of which the solution uses).
static void fg_step(FgState& s, int k) {
  if (!s.active) return;
  fg_issue(s, k);
  if (s.pending >= 0) {
    const bool conv = fg_check(s, s.pending);
    if (conv || s.nonfinite >= 0) {
      s.converged = conv;
      s.active = false;
      s.pending = -1;
      return;
    }
  }
  s.pending = k;
}

static void fg_drain(FgState& s) {
  if (s.pending >= 0) {
    if (fg_check(s, s.pending)) s.converged = true;
    s.pending = -1;
  }
  s.active = false;
}

static void fg_finish(FgState& s) {
  cav_hierarchy* H = s.H;
  double* S = H->dev_scalars;
  double* misc = S + s.L.misc;
  if (s.k_done > 0) {
    k_trisolve<<<1, 1, 0, s.st>>>(S, s.L, s.k_done, nullptr);
    CAV_CHECK_LAUNCH();
    k_combine<1><<<s.cb, FG_THREADS, 0, s.st>>>(H->Z, s.n, s.k_done, S + s.L.y, s.x, nullptr, nullptr, 0);
    CAV_CHECK_LAUNCH();
  }
  const Level& l0 = H->levels[0];
  launch_apply(s.op, s.x, s.b, l0.r, 0, s.st);  // true residual at exit
  dot_to(H, l0.r, l0.r, s.n, misc + 6, s.st);
  CAV_CHECK_CUDA(cudaMemcpyAsync(H->host_b + 6, misc + 6, sizeof(double), cudaMemcpyDeviceToHost, s.st));
  if (s.d->host_io)
    CAV_CHECK_CUDA(cudaMemcpyAsync(s.x_user, s.x, sizeof(double) * s.n, cudaMemcpyDeviceToHost, s.st));
  // the hierarchy's device status word (a bounded wait that ran out in any V-cycle)
  CAV_CHECK_CUDA(cudaMemcpyAsync(reinterpret_cast<int*>(H->host_b + 15), H->status, sizeof(int),
                                 cudaMemcpyDeviceToHost, s.st));
}

// after the stream has been synchronised
static ib_status fg_result(FgState& s) {
  s.info->iters = s.k_done;
  s.info->converged = s.converged ? 1 : 0;
  s.info->relres_est = s.est;
  if (s.nonfinite >= 0)
    set_error("fgmres_solve: the preconditioned vector of iteration " + std::to_string(s.nonfinite) +
              " is not finite (the V-cycle diverged; with the coloured smoother this happens when "
              "rounded FP32 inverses of very ill-conditioned patches make the undamped sweep "
              "diverge: use FP64 inverses); x holds the iterate before it");
  s.info->relres_true = (s.ref > 0) ? std::sqrt(s.H->host_b[6]) / s.ref : 0.0;
  const int code = *reinterpret_cast<const int*>(s.H->host_b + 15);
  if (code != DEV_OK) {
    CAV_CHECK_CUDA(cudaMemsetAsync(s.H->status, 0, sizeof(int), s.st));
    CAV_CHECK_CUDA(cudaStreamSynchronize(s.st));
    set_error("fgmres_solve: " + status_message(code));
    return status_of(code);
  }
  return s.converged ? IB_OK : IB_ERR_NOCONV;
}

ib_status fgmres_run(const ib_system* sys, cav_hierarchy* H, const double* b_in, double* x_in,
                     const fgmres_desc* d, fgmres_info* info, double* history, cudaStream_t st) {
  FgState s;
  s.sys = sys;
  s.H = H;
  s.d = d;
  s.info = info;
  s.history = history;
  s.st = st;
  s.b_user = b_in;
  s.x_user = x_in;
  fg_start(s);
  CAV_CHECK_CUDA(cudaStreamSynchronize(st));
  fg_begin(s);
  for (int k = 0; k < d->maxit && s.active; ++k) fg_step(s, k);
  fg_drain(s);
  fg_finish(s);
  CAV_CHECK_CUDA(cudaStreamSynchronize(st));
  return fg_result(s);
}

// Many independent systems in lockstep, each on its own stream (created once per
// hierarchy): their V-cycle graphs, products and Arnoldi kernels overlap on the device.
// Returns IB_OK if every system converged, IB_ERR_NOCONV otherwise (infos hold each result).
ib_status fgmres_run_batched(int count, const ib_system* const* sys, cav_hierarchy* const* H,
                             const double* const* b, double* const* x, const fgmres_desc* d,
                             fgmres_info* infos, cudaStream_t st) {
  std::vector<FgState> S(count);
  cudaEvent_t start_ev = nullptr;
  CAV_CHECK_CUDA(cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming));
  CAV_CHECK_CUDA(cudaEventRecord(start_ev, st));
  for (int i = 0; i < count; ++i) {
    if (!H[i]->solve_stream) CAV_CHECK_CUDA(cudaStreamCreateWithFlags(&H[i]->solve_stream, cudaStreamNonBlocking));
    CAV_CHECK_CUDA(cudaStreamWaitEvent(H[i]->solve_stream, start_ev, 0));
    S[i].sys = sys[i];
    S[i].H = H[i];
    S[i].d = d;
    S[i].info = &infos[i];
    S[i].st = H[i]->solve_stream;
    S[i].b_user = b[i];
    S[i].x_user = x[i];
    fg_start(S[i]);
  }
  for (int i = 0; i < count; ++i) CAV_CHECK_CUDA(cudaStreamSynchronize(S[i].st));
  for (int i = 0; i < count; ++i) fg_begin(S[i]);
  for (int k = 0; k < d->maxit; ++k) {
    bool any = false;
    for (int i = 0; i < count; ++i) {
      fg_step(S[i], k);
      any = any || S[i].active;
    }
    if (!any) break;
  }
  for (int i = 0; i < count; ++i) fg_drain(S[i]);
  for (int i = 0; i < count; ++i) fg_finish(S[i]);
  bool all = true;
  ib_status failure = IB_OK;
  for (int i = 0; i < count; ++i) {
    CAV_CHECK_CUDA(cudaStreamSynchronize(S[i].st));
    const ib_status r = fg_result(S[i]);
    if (r != IB_OK && r != IB_ERR_NOCONV && failure == IB_OK) failure = r;
    all = (r == IB_OK) && all;
  }
  cudaEventDestroy(start_ev);
  if (failure != IB_OK) return failure;
  return all ? IB_OK : IB_ERR_NOCONV;
}

// ------------------------------------------------------------------ device-driven iterations
//
// fgmres_desc.loop = 1: a whole solve is one CUDA graph: the prologue (r_0, the norms, V_0),
// a conditional while node whose body is one FGMRES iteration (copy V_k in, the V-cycle, K_E
// z_k, CGS2, ||w||, Givens, V_{k+1} and Z_k stored, the convergence test), and the epilogue
// (y = H^-1 g, x += Z y, the true residual, the records copied to pinned host memory).  The
// body's kernels read the iteration index k from device memory; the test kernel ends the loop
// through cudaGraphSetConditional, so no host round trip separates two iterations.  A batch
// of systems is one graph whose branches are the systems' solves: every system runs its own
// loop and stops at its own convergence.  The arithmetic is the host-driven loop's, kernel for
// kernel, so the results are bitwise the same.

// kc (ints): [0] body executions so far = the iteration index k, [1] iterations kept (k_done),
// [2] converged, [3] iteration whose residual estimate was not finite (-1: none).
// misc (doubles): [7] ||ref||, [8] the last relative residual estimate.

__global__ void k_dl_init(double* S, FgLayout L, int rel_to, double rtol, int* kc, double* hist,
                          cudaGraphConditionalHandle cond) {
  pdl_wait();
  pdl_trigger();
  double* misc = S + L.misc;
  const double bnorm = sqrt(misc[0]), beta = sqrt(misc[1]);
  const double ref = (rel_to == 1) ? beta : bnorm;
  misc[3] = (beta > 0.0) ? 1.0 / beta : 0.0;
  S[L.g] = beta;
  misc[7] = ref;
  const double est = (ref > 0.0) ? beta / ref : 0.0;
  misc[8] = est;
  hist[0] = est;
  const bool done = !(ref > 0.0) || beta <= rtol * ref;
  kc[0] = 0;
  kc[1] = 0;
  kc[2] = done ? 1 : 0;
  kc[3] = -1;
  cudaGraphSetConditional(cond, done ? 0u : 1u);
}

// dst = V_k
__global__ void k_dl_copy_in(const double* __restrict__ V, int64_t n, const int* __restrict__ kc,
                             double* __restrict__ dst) {
  pdl_wait();
  pdl_trigger();
  const double* src = V + (int64_t)kc[0] * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

// V_{k+1} = w * scale[0] and Z_k = z
__global__ void k_dl_store(const double* __restrict__ w, int64_t n, const double* __restrict__ scale,
                           double* __restrict__ V, const double* __restrict__ z, double* __restrict__ Z,
                           const int* __restrict__ kc) {
  pdl_wait();
  pdl_trigger();
  const int64_t k = kc[0];
  const double s = scale[0];
  double* v = V + (k + 1) * n;
  double* zk = Z + k * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    v[e] = w[e] * s;
    zk[e] = z[e];
  }
}

// the convergence test of iteration k, as fg_check makes it
__global__ void k_dl_check(double* S, FgLayout L, double rtol, int maxit, int* kc, double* hist,
                           cudaGraphConditionalHandle cond) {
  pdl_wait();
  pdl_trigger();
  double* misc = S + L.misc;
  const int k = kc[0];
  const double gk = misc[4], ref = misc[7];
  bool stop;
  if (!isfinite(gk)) {
    kc[3] = k;  // keep the k iterations before it
    kc[1] = k;
    stop = true;
  } else {
    kc[1] = k + 1;
    const double est = gk / ref;
    misc[8] = est;
    hist[k + 1] = est;
    const bool conv = gk <= rtol * ref;
    kc[2] = conv ? 1 : 0;
    stop = conv || k + 1 >= maxit;
  }
  kc[0] = k + 1;
  cudaGraphSetConditional(cond, stop ? 0u : 1u);
}

struct DlPlan {
  cudaGraphExec_t exec = nullptr;
  std::vector<uint64_t> key;
  std::vector<cudaEvent_t> events;   // fork / join of a batch's branches (capture only)
  // kernels per system: prologue + epilogue, and per body execution (launch accounting)
  std::vector<int> k_fixed, k_body;
};

void dl_plan_free(DlPlan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  for (auto& e : p->events) cudaEventDestroy(e);
  delete p;
}

static void dl_key_add(std::vector<uint64_t>& key, const FgState& s) {
  key.push_back(s.H->uid);
  key.push_back(s.H->epoch);
  key.push_back(s.sys->uid);
  key.push_back(s.sys->epoch);
  key.push_back((uint64_t)(uintptr_t)s.b_user);
  key.push_back((uint64_t)(uintptr_t)s.x_user);
  key.push_back((uint64_t)(uintptr_t)s.H->V);
}

static std::vector<uint64_t> dl_key(const std::vector<FgState>& S, const fgmres_desc* d) {
  std::vector<uint64_t> key;
  uint64_t rt = 0;
  std::memcpy(&rt, &d->rtol, sizeof(rt));
  key.push_back(rt);
  key.push_back((uint64_t)d->maxit);
  key.push_back((uint64_t)d->rel_to);
  key.push_back(S.size());
  for (const FgState& s : S) dl_key_add(key, s);
  return key;
}

// One system's solve captured on cs (already capturing); the loop body is captured into the
// conditional node's body graph on bs.  Returns the kernels of the prologue and epilogue and
// those of one body execution.
static void dl_capture_system(FgState& s, cudaStream_t cs, cudaStream_t bs, int& k_fixed, int& k_body) {
  cav_hierarchy* H = s.H;
  const Level& l0 = H->levels[0];
  s.n = 3LL * l0.N * l0.N;
  s.L = FgLayout(s.d->maxit);
  s.b = s.b_user;
  s.x = s.x_user;
  s.op = LevelOps{l0.N, l0.h, l0.rho_dt, l0.mu, l0.dt, &s.sys->ee, l0.channel};
  s.nb = dot_blocks(s.n);
  s.cb = cmb_blocks(s.n);
  s.nbmax = s.nb > s.cb ? s.nb : s.cb;
  if (reduce_blocks(s.n) > s.nbmax) s.nbmax = reduce_blocks(s.n);
  s.vb = vec_blocks(s.n);
  const int64_t n = s.n;
  const int maxit = s.d->maxit;
  double* S = H->dev_scalars;
  double* misc = S + s.L.misc;
  int* kc = H->dl_kc;

  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edata = nullptr;
  size_t ndeps = 0;
  CAV_CHECK_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, nullptr, nullptr, nullptr));
  CAV_REQUIRE(cst == cudaStreamCaptureStatusActive && g, "fgmres: device loop capture is not active");
  cudaGraphConditionalHandle cond;
  CAV_CHECK_CUDA(cudaGraphConditionalHandleCreate(&cond, g, 0, 0));

  const int64_t c0 = launch_count();
  // prologue (fg_start and fg_begin)
  CAV_CHECK_CUDA(cudaMemsetAsync(S, 0, sizeof(double) * s.L.total, cs));
  launch_apply(s.op, s.x, s.b, H->V, 0, cs);  // r0 -> V_0
  dot_to(H, s.b, s.b, n, misc + 0, cs);
  dot_to(H, H->V, H->V, n, misc + 1, cs);
  launch_k(k_dl_init, dim3(1), dim3(1), 0, cs, true, S, s.L, s.d->rel_to, s.d->rtol, kc, H->dl_hist, cond);
  launch_k(k_scale, dim3(s.vb), dim3(FG_THREADS), 0, cs, true, (const double*)H->V, n, (const double*)(misc + 3),
           H->V);

  // the loop
  CAV_CHECK_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, &edata, &ndeps));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode = nullptr;
  CAV_CHECK_CUDA(cudaGraphAddNode(&cnode, g, deps, edata, ndeps, &cp));
  CAV_CHECK_CUDA(cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaGraph_t body = cp.conditional.phGraph_out[0];

  const int64_t c1 = launch_count();
  CAV_CHECK_CUDA(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  bool body_ok = true;
  try {
    double* w = H->dl_w;
    double* sq_partial = H->red_partial + (int64_t)(maxit + 1) * s.nbmax;
    launch_k(k_dl_copy_in, dim3(s.vb), dim3(FG_THREADS), 0, bs, false, (const double*)H->V, n, (const int*)kc, l0.b);
    H->no_events = 1;
    vcycle_inline(H, bs);
    H->no_events = 0;
    launch_apply(s.op, l0.x, nullptr, w, 1, bs, true);
    const double* Vc = H->V;
    const int gy = div_up(maxit, DOT_GROUP);  // k + 1 <= maxit vectors
    for (int pass = 0; pass < 2; ++pass) {
      launch_k(k_multi_dot, dim3(s.nb, gy), dim3(FG_THREADS), 0, bs, true, Vc, n, 0, (const double*)w,
               H->red_partial, (const int*)kc);
      launch_k(k_finalize, dim3(maxit), dim3(FG_THREADS), 0, bs, true, (const double*)H->red_partial, s.nb,
               S + s.L.h, S + s.L.H, (const int*)kc, (int64_t)(maxit + 1));
      launch_k(k_combine<-1>, dim3(s.cb), dim3(FG_THREADS), 0, bs, true, Vc, n, 0, (const double*)(S + s.L.h), w,
               pass == 1 ? sq_partial : nullptr, (const int*)kc, 1);
    }
    launch_k(k_finalize, dim3(1), dim3(FG_THREADS), 0, bs, true, (const double*)sq_partial, s.cb, misc + 2,
             (double*)nullptr, (const int*)nullptr, (int64_t)0);
    launch_k(k_givens, dim3(1), dim3(128), 0, bs, true, S, s.L, 0, (const int*)kc);
    launch_k(k_dl_store, dim3(s.vb), dim3(FG_THREADS), 0, bs, true, (const double*)w, n, (const double*)(misc + 5),
             H->V, (const double*)l0.x, H->Z, (const int*)kc);
    launch_k(k_dl_check, dim3(1), dim3(1), 0, bs, true, S, s.L, s.d->rtol, maxit, kc, H->dl_hist, cond);
  } catch (...) {
    body_ok = false;
  }
  H->no_events = 0;
  cudaGraph_t body_out = nullptr;
  const cudaError_t be = cudaStreamEndCapture(bs, &body_out);
  if (!body_ok) throw Fail{IB_ERR_CUDA};
  if (be != cudaSuccess) {
    set_error(std::string("fgmres: capturing the loop body: ") + cudaGetErrorString(be));
    throw Fail{IB_ERR_CUDA};
  }
  const int64_t c2 = launch_count();

  // epilogue (fg_finish)
  launch_k(k_trisolve, dim3(1), dim3(1), 0, cs, false, S, s.L, 0, (const int*)(kc + 1));
  launch_k(k_combine<1>, dim3(s.cb), dim3(FG_THREADS), 0, cs, true, (const double*)H->Z, n, 0,
           (const double*)(S + s.L.y), s.x, (double*)nullptr, (const int*)(kc + 1), 0);
  launch_apply(s.op, s.x, s.b, l0.r, 0, cs, true);  // true residual at exit
  dot_to(H, l0.r, l0.r, n, misc + 6, cs);
  double* hb = H->dl_host;
  CAV_CHECK_CUDA(cudaMemcpyAsync(hb, misc, sizeof(double) * 16, cudaMemcpyDeviceToHost, cs));
  CAV_CHECK_CUDA(cudaMemcpyAsync(hb + 16, kc, sizeof(int) * 8, cudaMemcpyDeviceToHost, cs));
  CAV_CHECK_CUDA(cudaMemcpyAsync(hb + 20, H->status, sizeof(int), cudaMemcpyDeviceToHost, cs));
  CAV_CHECK_CUDA(cudaMemcpyAsync(hb + 32, H->dl_hist, sizeof(double) * (maxit + 1), cudaMemcpyDeviceToHost, cs));
  const int64_t c3 = launch_count();
  k_fixed = (int)((c1 - c0) + (c3 - c2));
  k_body = (int)(c2 - c1);
  note_launches(-(long long)(c3 - c0));  // recorded, not run
}

// After the graph ran: the results as fg_result reports them.
static ib_status dl_result(FgState& s) {
  const double* hb = s.H->dl_host;
  const int* kc = reinterpret_cast<const int*>(hb + 16);
  const double* misc = hb;
  s.k_done = kc[1];
  s.converged = kc[2] != 0;
  s.nonfinite = kc[3];
  s.est = misc[8];
  const double ref = misc[7];
  s.info->iters = s.k_done;
  s.info->converged = s.converged ? 1 : 0;
  s.info->relres_est = s.est;
  s.info->relres_true = (ref > 0) ? std::sqrt(misc[6]) / ref : 0.0;
  if (s.history)
    for (int i = 0; i <= s.k_done; ++i) s.history[i] = hb[32 + i];
  if (s.nonfinite >= 0)
    set_error("fgmres_solve: the preconditioned vector of iteration " + std::to_string(s.nonfinite) +
              " is not finite (the V-cycle diverged; with the coloured smoother this happens when "
              "rounded FP32 inverses of very ill-conditioned patches make the undamped sweep "
              "diverge: use FP64 inverses); x holds the iterate before it");
  const int code = *reinterpret_cast<const int*>(hb + 20);
  if (code != DEV_OK) {
    CAV_CHECK_CUDA(cudaMemsetAsync(s.H->status, 0, sizeof(int), s.st));
    CAV_CHECK_CUDA(cudaStreamSynchronize(s.st));
    set_error("fgmres_solve: " + status_message(code));
    return status_of(code);
  }
  return s.converged ? IB_OK : IB_ERR_NOCONV;
}

// Ends whatever capture is still open on the plan's streams after a failure.
static void dl_abort_capture(cudaStream_t origin, cudaStream_t bs, const std::vector<cudaStream_t>& branches) {
  cudaStreamCaptureStatus cst;
  if (cudaStreamIsCapturing(bs, &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(bs, &g);
  }
  if (cudaStreamIsCapturing(origin, &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(origin, &g);
    if (g) cudaGraphDestroy(g);
  }
  for (cudaStream_t b : branches) {
    if (cudaStreamIsCapturing(b, &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(b, &g);
      if (g) cudaGraphDestroy(g);
    }
  }
  cudaGetLastError();
}

// Capture and instantiate the solves of S (one branch each) as one graph.
static DlPlan* dl_build(std::vector<FgState>& S, cudaStream_t origin, cudaStream_t bs, bool pdl) {
  DlPlan* plan = new DlPlan();
  const int count = (int)S.size();
  plan->k_fixed.assign(count, 0);
  plan->k_body.assign(count, 0);
  std::vector<cudaStream_t> branches;
  const bool old_off = pdl_off();
  pdl_off() = !pdl;
  cudaGraph_t graph = nullptr;
  try {
    if (count > 1) {  // streams and events exist before the capture starts
      plan->events.resize(count + 1, nullptr);
      for (auto& e : plan->events) CAV_CHECK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      for (int i = 0; i < count; ++i) {
        cav_hierarchy* H = S[i].H;
        if (!H->solve_stream) CAV_CHECK_CUDA(cudaStreamCreateWithFlags(&H->solve_stream, cudaStreamNonBlocking));
      }
    }
    CAV_CHECK_CUDA(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
    if (count == 1) {
      dl_capture_system(S[0], origin, bs, plan->k_fixed[0], plan->k_body[0]);
    } else {
      CAV_CHECK_CUDA(cudaEventRecord(plan->events[0], origin));
      for (int i = 0; i < count; ++i) {
        cav_hierarchy* H = S[i].H;
        branches.push_back(H->solve_stream);
        CAV_CHECK_CUDA(cudaStreamWaitEvent(H->solve_stream, plan->events[0], 0));
        dl_capture_system(S[i], H->solve_stream, bs, plan->k_fixed[i], plan->k_body[i]);
        CAV_CHECK_CUDA(cudaEventRecord(plan->events[i + 1], H->solve_stream));
        CAV_CHECK_CUDA(cudaStreamWaitEvent(origin, plan->events[i + 1], 0));
      }
    }
    CAV_CHECK_CUDA(cudaStreamEndCapture(origin, &graph));
    CAV_CHECK_CUDA(cudaGraphInstantiate(&plan->exec, graph, 0));
    cudaGraphDestroy(graph);
  } catch (...) {
    pdl_off() = old_off;
    if (graph) cudaGraphDestroy(graph);
    dl_abort_capture(origin, bs, branches);
    dl_plan_free(plan);
    throw;
  }
  pdl_off() = old_off;
  return plan;
}

// Run the solves of S as one graph launch on st (built on first use, then cached in the first
// system's hierarchy while the key -- systems, hierarchies, buffers, tolerances -- holds).
static void dl_run(std::vector<FgState>& S, const fgmres_desc* d, cudaStream_t st) {
  cav_hierarchy* H0 = S[0].H;
  for (FgState& s : S) {
    const Level& l0 = s.H->levels[0];
    ensure_workspace(s.H, d->maxit, 3LL * l0.N * l0.N);
  }
  std::vector<uint64_t> key = dl_key(S, d);
  if (!H0->dl_plan || H0->dl_plan->key != key) {
    dl_plan_free(H0->dl_plan);
    H0->dl_plan = nullptr;
    if (!H0->dl_stream) CAV_CHECK_CUDA(cudaStreamCreateWithFlags(&H0->dl_stream, cudaStreamNonBlocking));
    if (!H0->dl_body_stream) CAV_CHECK_CUDA(cudaStreamCreateWithFlags(&H0->dl_body_stream, cudaStreamNonBlocking));
    DlPlan* plan = nullptr;
    try {
      plan = dl_build(S, H0->dl_stream, H0->dl_body_stream, true);
    } catch (const Fail&) {
      // programmatic edges inside a conditional body may be refused: build without them
      plan = dl_build(S, H0->dl_stream, H0->dl_body_stream, false);
    }
    plan->key = key;
    H0->dl_plan = plan;
  }
  DlPlan* plan = H0->dl_plan;
  CAV_CHECK_CUDA(cudaGraphLaunch(plan->exec, st));
  CAV_CHECK_CUDA(cudaStreamSynchronize(st));
  long long kernels = 0;
  for (size_t i = 0; i < S.size(); ++i) {
    const int* kc = reinterpret_cast<const int*>(S[i].H->dl_host + 16);
    kernels += plan->k_fixed[i] + (long long)kc[0] * plan->k_body[i];
  }
  note_launches(kernels);
}

ib_status fgmres_run_device(const ib_system* sys, cav_hierarchy* H, const double* b, double* x,
                            const fgmres_desc* d, fgmres_info* info, double* history, cudaStream_t st) {
  std::vector<FgState> S(1);
  S[0].sys = sys;
  S[0].H = H;
  S[0].d = d;
  S[0].info = info;
  S[0].history = history;
  S[0].st = st;
  S[0].b_user = b;
  S[0].x_user = x;
  dl_run(S, d, st);
  return dl_result(S[0]);
}

ib_status fgmres_run_batched_device(int count, const ib_system* const* sys, cav_hierarchy* const* H,
                                    const double* const* b, double* const* x, const fgmres_desc* d,
                                    fgmres_info* infos, cudaStream_t st) {
  std::vector<FgState> S(count);
  for (int i = 0; i < count; ++i) {
    S[i].sys = sys[i];
    S[i].H = H[i];
    S[i].d = d;
    S[i].info = &infos[i];
    S[i].st = st;
    S[i].b_user = b[i];
    S[i].x_user = x[i];
  }
  dl_run(S, d, st);
  bool all = true;
  ib_status failure = IB_OK;
  for (int i = 0; i < count; ++i) {
    const ib_status r = dl_result(S[i]);
    if (r != IB_OK && r != IB_ERR_NOCONV && failure == IB_OK) failure = r;
    all = (r == IB_OK) && all;
  }
  if (failure != IB_OK) return failure;
  return all ? IB_OK : IB_ERR_NOCONV;
}

}  // namespace cav
