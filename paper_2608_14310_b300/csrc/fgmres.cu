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

// partial[i * nb + bx] = block bx's share of <V_i, w> for i < kcount
__global__ void k_multi_dot(const double* __restrict__ V, int64_t n, int kcount, const double* __restrict__ w,
                            double* partial) {
  __shared__ double sm[FG_THREADS / 32];
  const int i = blockIdx.y;
  const double* v = V + (int64_t)i * n;
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    s += v[e] * w[e];
  s = block_sum(s, sm);
  if (threadIdx.x == 0) partial[(int64_t)i * gridDim.x + blockIdx.x] = s;
}

// out[i] = sum_b partial[i * nb + b] (fixed order); add_to (nullable) += out
__global__ void k_finalize(const double* __restrict__ partial, int nb, double* out, double* add_to) {
  __shared__ double sm[FG_THREADS / 32];
  const int i = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partial[(int64_t)i * nb + b];
  s = block_sum(s, sm);
  if (threadIdx.x == 0) {
    out[i] = s;
    if (add_to) add_to[i] += s;
  }
}

// w -= sum_{i < kcount} h[i] V_i
__global__ void k_sub_multi(const double* __restrict__ V, int64_t n, int kcount, const double* __restrict__ h,
                            double* __restrict__ w) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < kcount; ++i) s += h[i] * V[(int64_t)i * n + e];
    w[e] -= s;
  }
}

// x += sum_{i < kcount} y[i] Z_i
__global__ void k_add_multi(const double* __restrict__ Z, int64_t n, int kcount, const double* __restrict__ y,
                            double* __restrict__ x) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < kcount; ++i) s += y[i] * Z[(int64_t)i * n + e];
    x[e] += s;
  }
}

// v = w * scale[0]
__global__ void k_scale(const double* __restrict__ w, int64_t n, const double* __restrict__ scale,
                        double* __restrict__ v) {
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

__global__ void k_givens(double* S, FgLayout L, int k) {
  double* Hk = S + L.H + (int64_t)k * (L.maxit + 1);
  double* cs = S + L.cs;
  double* sn = S + L.sn;
  double* g = S + L.g;
  double* misc = S + L.misc;
  const double vnorm = sqrt(misc[2]);
  Hk[k + 1] = vnorm;
  for (int i = 0; i < k; ++i) {
    const double t = cs[i] * Hk[i] + sn[i] * Hk[i + 1];
    Hk[i + 1] = -sn[i] * Hk[i] + cs[i] * Hk[i + 1];
    Hk[i] = t;
  }
  const double d = hypot(Hk[k], Hk[k + 1]);
  cs[k] = (d != 0.0) ? Hk[k] / d : 1.0;
  sn[k] = (d != 0.0) ? Hk[k + 1] / d : 0.0;
  Hk[k] = d;
  Hk[k + 1] = 0.0;
  g[k + 1] = -sn[k] * g[k];
  g[k] = cs[k] * g[k];
  misc[4] = fabs(g[k + 1]);
  misc[5] = (vnorm > 0.0) ? 1.0 / vnorm : 0.0;
}

__global__ void k_trisolve(double* S, FgLayout L, int k) {
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
  H->ws_arena.release();
  H->V = H->ws_arena.alloc<double>((size_t)(maxit + 1) * n);
  H->Z = H->ws_arena.alloc<double>((size_t)maxit * n);
  FgLayout L(maxit);
  H->dev_scalars = H->ws_arena.alloc<double>(L.total);
  H->red_partial = H->ws_arena.alloc<double>((size_t)(maxit + 2) * reduce_blocks(n));
  H->io_b = H->ws_arena.alloc<double>(n);
  H->io_x = H->ws_arena.alloc<double>(n);
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
  const int nb = reduce_blocks(n);
  k_multi_dot<<<dim3(nb, 1), FG_THREADS, 0, st>>>(a, n, 1, b, H->red_partial);
  CAV_CHECK_LAUNCH();
  k_finalize<<<1, FG_THREADS, 0, st>>>(H->red_partial, nb, out, nullptr);
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
  int nb = 0, vb = 0;
  double ref = 0, beta = 0, est = 0;
  int k_done = 0, pending = -1;
  bool converged = false, active = false;
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
  s.op = LevelOps{l0.N, l0.h, l0.rho_dt, l0.mu, l0.dt, &l0.ee};
  s.nb = reduce_blocks(s.n);
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
  for (int pass = 0; pass < 2; ++pass) {
    k_multi_dot<<<dim3(s.nb, k + 1), FG_THREADS, 0, s.st>>>(H->V, n, k + 1, w, H->red_partial);
    CAV_CHECK_LAUNCH();
    k_finalize<<<k + 1, FG_THREADS, 0, s.st>>>(H->red_partial, s.nb, S + s.L.h, S + s.L.H + (int64_t)k * (maxit + 1));
    CAV_CHECK_LAUNCH();
    k_sub_multi<<<s.vb, FG_THREADS, 0, s.st>>>(H->V, n, k + 1, S + s.L.h, w);
    CAV_CHECK_LAUNCH();
  }
  dot_to(H, w, w, n, misc + 2, s.st);
  k_givens<<<1, 1, 0, s.st>>>(S, s.L, k);
  CAV_CHECK_LAUNCH();
  k_scale<<<s.vb, FG_THREADS, 0, s.st>>>(w, n, misc + 5, w);
  CAV_CHECK_LAUNCH();
  CAV_CHECK_CUDA(cudaMemcpyAsync(H->host_b + 8 + (k & 1), misc + 4, sizeof(double), cudaMemcpyDeviceToHost, s.st));
  CAV_CHECK_CUDA(cudaEventRecord(H->fg_ev[k & 1], s.st));
  s.prof_mark[k & 1] = H->prof_pushed;
}

static bool fg_check(FgState& s, int kk) {
  cav_hierarchy* H = s.H;
  CAV_CHECK_CUDA(cudaEventSynchronize(H->fg_ev[kk & 1]));
  if (H->prof_on) prof_collect(H, s.prof_mark[kk & 1]);
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
  if (s.pending >= 0 && fg_check(s, s.pending)) {
    s.converged = true;
    s.active = false;
    s.pending = -1;
    return;
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
    k_trisolve<<<1, 1, 0, s.st>>>(S, s.L, s.k_done);
    CAV_CHECK_LAUNCH();
    k_add_multi<<<s.vb, FG_THREADS, 0, s.st>>>(H->Z, s.n, s.k_done, S + s.L.y, s.x);
    CAV_CHECK_LAUNCH();
  }
  const Level& l0 = H->levels[0];
  launch_apply(s.op, s.x, s.b, l0.r, 0, s.st);  // true residual at exit
  dot_to(H, l0.r, l0.r, s.n, misc + 6, s.st);
  CAV_CHECK_CUDA(cudaMemcpyAsync(H->host_b + 6, misc + 6, sizeof(double), cudaMemcpyDeviceToHost, s.st));
  if (s.d->host_io)
    CAV_CHECK_CUDA(cudaMemcpyAsync(s.x_user, s.x, sizeof(double) * s.n, cudaMemcpyDeviceToHost, s.st));
}

// after the stream has been synchronised
static ib_status fg_result(FgState& s) {
  s.info->iters = s.k_done;
  s.info->converged = s.converged ? 1 : 0;
  s.info->relres_est = s.est;
  s.info->relres_true = (s.ref > 0) ? std::sqrt(s.H->host_b[6]) / s.ref : 0.0;
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
  for (int i = 0; i < count; ++i) {
    CAV_CHECK_CUDA(cudaStreamSynchronize(S[i].st));
    all = (fg_result(S[i]) == IB_OK) && all;
  }
  cudaEventDestroy(start_ev);
  return all ? IB_OK : IB_ERR_NOCONV;
}

}  // namespace cav
