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

static void dot_to(const cav_hierarchy* H, const double* a, const double* b, int64_t n, double* out,
                   cudaStream_t st) {
  const int nb = reduce_blocks(n);
  k_multi_dot<<<dim3(nb, 1), FG_THREADS, 0, st>>>(a, n, 1, b, H->red_partial);
  CAV_CHECK_LAUNCH();
  k_finalize<<<1, FG_THREADS, 0, st>>>(H->red_partial, nb, out, nullptr);
  CAV_CHECK_LAUNCH();
}

ib_status fgmres_run(const ib_system* sys, cav_hierarchy* H, const double* b_in, double* x_in,
                     const fgmres_desc* d, fgmres_info* info, double* history, cudaStream_t st) {
  const Level& l0 = H->levels[0];
  const int64_t n = 3LL * l0.N * l0.N;
  const int maxit = d->maxit;
  ensure_workspace(H, maxit, n);
  FgLayout L(maxit);
  double* S = H->dev_scalars;
  double* misc = S + L.misc;
  double* hbuf = H->host_b;  // pinned, 16 doubles
  const double* b = b_in;
  double* x = x_in;
  if (d->host_io) {
    double* bd = H->io_b;
    double* xd = H->io_x;
    CAV_CHECK_CUDA(cudaMemcpyAsync(bd, b_in, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    CAV_CHECK_CUDA(cudaMemcpyAsync(xd, x_in, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    b = bd;
    x = xd;
  }
  CAV_CHECK_CUDA(cudaMemsetAsync(S, 0, sizeof(double) * L.total, st));
  LevelOps op{l0.N, l0.h, l0.rho_dt, l0.mu, l0.dt, &l0.ee};
  const int nb = reduce_blocks(n);
  const int vb = vec_blocks(n);
  double* V = H->V;
  double* Z = H->Z;
  // r0 = b - K x  -> V_0
  launch_apply(op, x, b, V, 0, st);
  dot_to(H, b, b, n, misc + 0, st);
  dot_to(H, V, V, n, misc + 1, st);
  k_init_beta<<<1, 1, 0, st>>>(S, L);
  CAV_CHECK_LAUNCH();
  CAV_CHECK_CUDA(cudaMemcpyAsync(hbuf, misc, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
  CAV_CHECK_CUDA(cudaStreamSynchronize(st));
  const double bnorm = std::sqrt(hbuf[0]), beta = std::sqrt(hbuf[1]);
  const double ref = (d->rel_to == 1) ? beta : bnorm;
  int k_done = 0;
  bool converged = false;
  double est = (ref > 0) ? beta / ref : 0.0;
  if (history) history[0] = est;
  if (!(ref > 0.0) || beta <= d->rtol * ref) {
    converged = true;
  } else {
    k_scale<<<vb, FG_THREADS, 0, st>>>(V, n, misc + 3, V);
    CAV_CHECK_LAUNCH();
    // The convergence test of iteration k is read on the host while iteration k + 1 is
    // already queued: the host never waits on an idle device.  If iteration k converged,
    // iteration k + 1's work is discarded -- it writes only Hessenberg column k + 1, Givens
    // pair k + 1, g[k+1..k+2] and V_{k+2}, Z_{k+1}, none of which the solution uses.
    int pending = -1;
    long long prof_mark[2] = {0, 0};  // profiling records issued up to the end of iteration k
    auto check = [&](int kk) -> bool {
      CAV_CHECK_CUDA(cudaEventSynchronize(H->fg_ev[kk & 1]));
      if (H->prof_on) prof_collect(H, prof_mark[kk & 1]);
      k_done = kk + 1;
      est = hbuf[8 + (kk & 1)] / ref;
      if (history) history[kk + 1] = est;
      return hbuf[8 + (kk & 1)] <= d->rtol * ref;
    };
    for (int k = 0; k < maxit; ++k) {
      double* vk = V + (int64_t)k * n;
      double* zk = Z + (int64_t)k * n;
      double* w = V + (int64_t)(k + 1) * n;
      vcycle(H, vk, zk, st);
      launch_apply(op, zk, nullptr, w, 1, st);
      for (int pass = 0; pass < 2; ++pass) {
        k_multi_dot<<<dim3(nb, k + 1), FG_THREADS, 0, st>>>(V, n, k + 1, w, H->red_partial);
        CAV_CHECK_LAUNCH();
        k_finalize<<<k + 1, FG_THREADS, 0, st>>>(H->red_partial, nb, S + L.h, S + L.H + (int64_t)k * (maxit + 1));
        CAV_CHECK_LAUNCH();
        k_sub_multi<<<vb, FG_THREADS, 0, st>>>(V, n, k + 1, S + L.h, w);
        CAV_CHECK_LAUNCH();
      }
      dot_to(H, w, w, n, misc + 2, st);
      k_givens<<<1, 1, 0, st>>>(S, L, k);
      CAV_CHECK_LAUNCH();
      k_scale<<<vb, FG_THREADS, 0, st>>>(w, n, misc + 5, w);
      CAV_CHECK_LAUNCH();
      CAV_CHECK_CUDA(cudaMemcpyAsync(hbuf + 8 + (k & 1), misc + 4, sizeof(double), cudaMemcpyDeviceToHost, st));
      CAV_CHECK_CUDA(cudaEventRecord(H->fg_ev[k & 1], st));
      prof_mark[k & 1] = H->prof_pushed;
      if (pending >= 0 && check(pending)) {
        converged = true;
        pending = -1;
        break;
      }
      pending = k;
    }
    if (pending >= 0 && check(pending)) converged = true;
    CAV_CHECK_CUDA(cudaStreamSynchronize(st));
    k_trisolve<<<1, 1, 0, st>>>(S, L, k_done);
    CAV_CHECK_LAUNCH();
    k_add_multi<<<vb, FG_THREADS, 0, st>>>(Z, n, k_done, S + L.y, x);
    CAV_CHECK_LAUNCH();
  }
  // true residual at exit
  launch_apply(op, x, b, l0.r, 0, st);
  dot_to(H, l0.r, l0.r, n, misc + 6, st);
  CAV_CHECK_CUDA(cudaMemcpyAsync(hbuf + 6, misc + 6, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (d->host_io) CAV_CHECK_CUDA(cudaMemcpyAsync(x_in, x, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  CAV_CHECK_CUDA(cudaStreamSynchronize(st));
  info->iters = k_done;
  info->converged = converged ? 1 : 0;
  info->relres_est = est;
  info->relres_true = (ref > 0) ? std::sqrt(hbuf[6]) / ref : 0.0;
  return converged ? IB_OK : IB_ERR_NOCONV;
}

}  // namespace cav
