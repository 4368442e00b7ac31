// One weighted additive CAV sweep (Eq. additive_cav_saddle) and the V-cycle of Sec. 4.
//
// A sweep on level l with iterate w and right-hand side b:
//   1. r = b - K_E w                                   (stencil kernel + E_E rows)
//   2. delta_p = diag(s_c) X_p diag(s_r) r|_p for every enlarged patch p
//      (batched variable-size GEMV, one CTA per patch, inverses streamed from HBM)
//   3. w_k += alpha / count_k * (sum over standard patches holding k of their 5x5 solve
//      + sum over enlarged patches holding k of delta_p at k's slot)
//      (owner computes: one thread per cell, fixed summation order, no atomics)
//   4. remove the mean pressure (Sec. 3.3).
#include "internal.cuh"
#include "device_util.cuh"

namespace cav {

// ------------------------------------------------------------------ 2. patch apply

template <typename T>
struct VecLoad;
template <>
struct VecLoad<double> {
  static constexpr int V = 2;
  typedef double acc_t;
  __device__ static void load(const double* p, acc_t* out) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    out[0] = v.x;
    out[1] = v.y;
  }
};
template <>
struct VecLoad<float> {
  static constexpr int V = 4;
  typedef float acc_t;
  __device__ static void load(const float* p, acc_t* out) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    out[0] = v.x;
    out[1] = v.y;
    out[2] = v.z;
    out[3] = v.w;
  }
};
template <>
struct VecLoad<__nv_bfloat16> {
  static constexpr int V = 8;
  typedef float acc_t;
  __device__ static void load(const __nv_bfloat16* p, acc_t* out) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 f = __bfloat1622float2(h[q]);
      out[2 * q] = f.x;
      out[2 * q + 1] = f.y;
    }
  }
};

// One CTA per enlarged patch (in descending-size order).  The scaled residual
// y = s_r * r|_p is staged in shared memory; the inverse is column-major with ld = round8(n)
// so each thread owns V consecutive rows and streams one 16-byte vector per column.
template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS)
k_patch_apply(const int* __restrict__ order, const int64_t* __restrict__ off, const int* __restrict__ dofs,
              const int64_t* __restrict__ inv_off, const T* __restrict__ inv, const double* __restrict__ s_r,
              const double* __restrict__ s_c, const double* __restrict__ r, double* __restrict__ delta) {
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
    int b = 0;
    for (; b + 4 <= n; b += 4) {
      acc_t x0[V], x1[V], x2[V], x3[V];
      VL::load(col + (int64_t)(b + 0) * ld, x0);
      VL::load(col + (int64_t)(b + 1) * ld, x1);
      VL::load(col + (int64_t)(b + 2) * ld, x2);
      VL::load(col + (int64_t)(b + 3) * ld, x3);
      const acc_t y0 = y[b], y1 = y[b + 1], y2 = y[b + 2], y3 = y[b + 3];
#pragma unroll
      for (int q = 0; q < V; ++q) acc[q] += x0[q] * y0 + x1[q] * y1 + x2[q] * y2 + x3[q] * y3;
    }
    for (; b < n; ++b) {
      acc_t x0[V];
      VL::load(col + (int64_t)b * ld, x0);
      const acc_t yb = y[b];
#pragma unroll
      for (int q = 0; q < V; ++q) acc[q] += x0[q] * yb;
    }
#pragma unroll
    for (int q = 0; q < V; ++q)
      if (a0 + q < n) delta[d0 + a0 + q] = s_c[d0 + a0 + q] * (double)acc[q];
  }
}

// ------------------------------------------------------------------ 3. scatter / update

struct StdInv {
  double m[25];
};

// canonical slots of cell (i, j)'s standard patch: u_ij, u_i+1j, v_ij, v_ij+1, p_ij
__device__ inline double std_row(const StdInv& S, int row, const double* __restrict__ r, int N, int i, int j) {
  const int NN = N * N;
  const int ip = (i + 1 == N) ? 0 : i + 1, jp = (j + 1 == N) ? 0 : j + 1;
  const double y0 = r[j * N + i], y1 = r[j * N + ip], y2 = r[NN + j * N + i], y3 = r[NN + jp * N + i],
               y4 = r[2 * NN + j * N + i];
  const double* m = S.m + 5 * row;
  return m[0] * y0 + m[1] * y1 + m[2] * y2 + m[3] * y3 + m[4] * y4;
}

template <int BX, int BY>
__global__ void __launch_bounds__(BX* BY)
k_update(int N, double alpha, StdInv S, const uint8_t* __restrict__ cell_big, const int64_t* __restrict__ inc_off,
         const int* __restrict__ inc_slot, const double* __restrict__ delta, const double* __restrict__ r,
         double* __restrict__ w, int w_is_zero, double* __restrict__ partial) {
  __shared__ double sm[BX * BY / 32];
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int NN = N * N;
  double pnew = 0.0;
  if (i < N && j < N) {
    const int c = j * N + i;
    const int im = (i == 0) ? N - 1 : i - 1, jm = (j == 0) ? N - 1 : j - 1;
    const bool big_c = cell_big[c] != 0;
    const bool big_l = cell_big[j * N + im] != 0, big_d = cell_big[jm * N + i] != 0;
    // u_ij: standard patches of cells (i-1, j) [slot 1] and (i, j) [slot 0]
    {
      double s = 0.0;
      int cnt = 0;
      if (!big_l) { s += std_row(S, 1, r, N, im, j); ++cnt; }
      if (!big_c) { s += std_row(S, 0, r, N, i, j); ++cnt; }
      const int k = c;
      for (int64_t q = inc_off[k]; q < inc_off[k + 1]; ++q) { s += delta[inc_slot[q]]; ++cnt; }
      const double old = w_is_zero ? 0.0 : w[k];
      w[k] = old + alpha * (s / (double)cnt);
    }
    // v_ij: standard patches of cells (i, j-1) [slot 3] and (i, j) [slot 2]
    {
      double s = 0.0;
      int cnt = 0;
      if (!big_d) { s += std_row(S, 3, r, N, i, jm); ++cnt; }
      if (!big_c) { s += std_row(S, 2, r, N, i, j); ++cnt; }
      const int k = NN + c;
      for (int64_t q = inc_off[k]; q < inc_off[k + 1]; ++q) { s += delta[inc_slot[q]]; ++cnt; }
      const double old = w_is_zero ? 0.0 : w[k];
      w[k] = old + alpha * (s / (double)cnt);
    }
    // p_ij: the standard patch of cell (i, j) [slot 4]
    {
      double s = 0.0;
      int cnt = 0;
      if (!big_c) { s += std_row(S, 4, r, N, i, j); ++cnt; }
      const int k = 2 * NN + c;
      for (int64_t q = inc_off[k]; q < inc_off[k + 1]; ++q) { s += delta[inc_slot[q]]; ++cnt; }
      const double old = w_is_zero ? 0.0 : w[k];
      pnew = old + alpha * (s / (double)cnt);
      w[k] = pnew;
    }
  }
  // partial sums of the new pressure for the mean (fixed order)
  const int tid = threadIdx.y * BX + threadIdx.x;
  double v = warp_sum(pnew);
  if ((tid & 31) == 0) sm[tid >> 5] = v;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < BX * BY / 32; ++q) t += sm[q];
    partial[blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// 4. p -= mean(p): every block reduces the partials in the same order, then subtracts.
__global__ void k_remove_mean(int N, int n_partial, const double* __restrict__ partial, double* __restrict__ p) {
  __shared__ double sm[8];
  double t = 0.0;
  for (int q = threadIdx.x; q < n_partial; q += blockDim.x) t += partial[q];
  t = block_sum(t, sm);
  const double mean = t / ((double)N * (double)N);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N * N; c += gridDim.x * blockDim.x) p[c] -= mean;
}

// Coarsest level: z = (dense bordered inverse) [r; 0], one warp per row, row-major.
__global__ void k_coarse_apply(int n, const double* __restrict__ inv, const double* __restrict__ r,
                               double* __restrict__ z) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* a = inv + (int64_t)row * (n + 1);
  double s = 0.0;
  for (int b = lane; b < n; b += 32) s += a[b] * r[b];
  s = warp_sum(s);
  if (lane == 0) z[row] = s;
}

// ------------------------------------------------------------------ host drivers

static constexpr int APPLY_THREADS = 128;
static constexpr int UBX = 32, UBY = 8;

static LevelOps ops_of(const Level& lv) {
  LevelOps o;
  o.N = lv.N;
  o.h = lv.h;
  o.rho_dt = lv.rho_dt;
  o.mu = lv.mu;
  o.dt = lv.dt;
  o.ee = &lv.ee;
  return o;
}

void prof_begin(const cav_hierarchy* H, int level, cudaStream_t st) {
  cav_hierarchy* h = const_cast<cav_hierarchy*>(H);
  if (!h->prof_on || level != 0) return;
  if ((size_t)(2 * h->prof_used + 1) >= h->prof_ev.size()) return;
  CAV_CHECK_CUDA(cudaEventRecord(h->prof_ev[2 * h->prof_used], st));
}
void prof_end(const cav_hierarchy* H, int level, cudaStream_t st) {
  cav_hierarchy* h = const_cast<cav_hierarchy*>(H);
  if (!h->prof_on || level != 0) return;
  if ((size_t)(2 * h->prof_used + 1) >= h->prof_ev.size()) return;
  CAV_CHECK_CUDA(cudaEventRecord(h->prof_ev[2 * h->prof_used + 1], st));
  ++h->prof_used;
}

template <typename T>
static void launch_patch_apply(const Level& lv, const T* inv, const double* r, cudaStream_t st) {
  typedef typename VecLoad<T>::acc_t acc_t;
  const size_t smem = sizeof(acc_t) * (size_t)lv.big_max_n;
  k_patch_apply<T, APPLY_THREADS><<<lv.n_big, APPLY_THREADS, smem, st>>>(
      lv.order, lv.big_off, lv.big_dofs, lv.inv_off, inv, lv.s_r, lv.s_c, r, lv.delta);
  CAV_CHECK_LAUNCH();
}

void level_sweep(const cav_hierarchy* H, int l, const double* b, double* w, bool w_is_zero, cudaStream_t st) {
  const Level& lv = H->levels[l];
  const double* r = b;
  if (!w_is_zero) {
    launch_apply(ops_of(lv), w, b, lv.r, 0, st);
    r = lv.r;
  }
  if (lv.n_big > 0) {
    prof_begin(H, l, st);
    if (lv.precision == CAV_PREC_FP32) launch_patch_apply<float>(lv, lv.inv32, r, st);
    else if (lv.precision == CAV_PREC_BF16) launch_patch_apply<__nv_bfloat16>(lv, lv.inv16, r, st);
    else launch_patch_apply<double>(lv, lv.inv64, r, st);
    prof_end(H, l, st);
  }
  StdInv S;
  for (int q = 0; q < 25; ++q) S.m[q] = lv.std_inv[q];
  dim3 blk(UBX, UBY), grd(div_up(lv.N, UBX), div_up(lv.N, UBY));
  k_update<UBX, UBY><<<grd, blk, 0, st>>>(lv.N, H->desc.alpha, S, lv.cell_big, lv.inc_off, lv.inc_slot,
                                          lv.delta, r, w, w_is_zero ? 1 : 0, lv.partial);
  CAV_CHECK_LAUNCH();
  const int npart = grd.x * grd.y;
  k_remove_mean<<<div_up(lv.N * lv.N, 256) < 296 ? div_up(lv.N * lv.N, 256) : 296, 256, 0, st>>>(
      lv.N, npart, lv.partial, w + 2 * lv.N * lv.N);
  CAV_CHECK_LAUNCH();
}

void coarse_solve(const cav_hierarchy* H, const double* r, double* z, cudaStream_t st) {
  const Level& lv = H->levels.back();
  const int n = 3 * lv.N * lv.N;
  k_coarse_apply<<<div_up(n, 8), 256, 0, st>>>(n, lv.coarse_inv, r, z);
  CAV_CHECK_LAUNCH();
}

static void vcycle_level(const cav_hierarchy* H, int l, const double* b, double* x, cudaStream_t st) {
  const Level& lv = H->levels[l];
  if (lv.coarsest) {
    coarse_solve(H, b, x, st);
    return;
  }
  const int NN = lv.N * lv.N;
  const int nu_pre = H->desc.nu_pre, nu_post = H->desc.nu_post;
  if (nu_pre == 0) CAV_CHECK_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * 3 * NN, st));
  for (int s = 0; s < nu_pre; ++s) level_sweep(H, l, b, x, s == 0, st);
  launch_apply(ops_of(lv), x, b, lv.r, 0, st);
  const Level& lc = H->levels[l + 1];
  launch_restrict(lc.N, lv.r, lc.b, st);
  vcycle_level(H, l + 1, lc.b, lc.x, st);
  launch_prolong_add(lc.N, lc.x, x, st);
  for (int s = 0; s < nu_post; ++s) level_sweep(H, l, b, x, false, st);
}

void vcycle(const cav_hierarchy* H, const double* r, double* z, cudaStream_t st) {
  vcycle_level(H, 0, r, z, st);
}

}  // namespace cav
