// The multiplicative CAV sweep of Sec. 3.3 in a parallel order: the patches are split into
// colour classes whose members share no unknown and are not coupled by any entry of K_E, and
// the classes are visited in turn.  Every patch p of a class then solves
//     w_p <- w_p + D_c X_p D_r (b - K_E w)_p
// from the current iterate, and since no patch of the class reads what another writes, one
// launch per class gives the sequential multiplicative sweep in class-by-class order.
//
// Set-up (host): first-fit greedy colouring, the enlarged patches in cell order first, then
// the standard ones, over the structural coupling of K_E (Stokes stencils plus E_E's pattern).
//
// One class step (one launch, programmatic dependent launch between consecutive classes):
//  * each enlarged patch is one thread-block cluster of C CTAs; its slots are dealt to the
//    CTAs round-robin.  Before waiting for the previous class, a CTA loads its job and slot
//    records, copies its slots' E_E rows into shared memory and issues TMA bulk copies of the
//    matching columns of the column-major inverse.  After the wait it evaluates its slots'
//    residual rows from the current iterate (E_E sums four lanes per slot, Stokes rows one per
//    lane), forms the partial product X[:, mine] y[mine], pushes each row's partial into the
//    shared memory of the CTA owning that row, and after one cluster barrier sums its rows'
//    partials in a fixed order and writes w.
//  * standard cells take five lanes each (one Stokes row per lane, the shared 5 x 5 inverse
//    applied after a shuffle).
//
// The box smoother B(b,o) (Sec. 3.1, 3.3) runs on the same machinery: one enlarged patch per
// block, blocks in lexicographic order of their lower-left cells, and a per-slot mask that
// writes only the unexpanded block's unknowns (restricted injection).  The conflict relation
// still reads the whole (expanded) patch, so a class's solves stay independent.
#include <cooperative_groups.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "internal.cuh"
#include "device_util.cuh"
#include "level_math.cuh"
#include "tma_util.cuh"

namespace cg = cooperative_groups;

namespace cav {

// ------------------------------------------------------------------ set-up: colour classes

// Per packed slot of the enlarged patches: start and length of its row in E_E's compact CSR
// (length 0 for a pressure or a velocity without an E_E row).
__global__ void k_slot_rows(int64_t n_slots, const int* __restrict__ dofs, int NN, const int* __restrict__ row_of,
                            const int64_t* __restrict__ rowptr, int2* __restrict__ out) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_slots) return;
  const int k = dofs[s];
  int2 e = make_int2(0, 0);
  if (k < 2 * NN && row_of) {
    const int r = row_of[k];
    if (r >= 0) e = make_int2((int)rowptr[r], (int)(rowptr[r + 1] - rowptr[r]));
  }
  out[s] = e;
}

// E_E values rounded to FP32 for the FP32 local residuals of FP32-inverse levels.
__global__ void k_round_f32(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) out[q] = (float)in[q];
}

// The iterate's FP32 copy at the start of a coloured sweep (FP32-inverse levels).
__global__ void k_to_f32(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) out[q] = (float)in[q];
}

template <typename T>
struct ColourStep;
template <typename T>
__global__ void k_colour_step(const ColourStep<T> a, const double* __restrict__ b, double* w);

static void colour_step_attributes();

void colour_fetch(const Level& lv, ColourPlan& P, cudaStream_t st) {
  const int NN = lv.N * lv.N;
  CAV_REQUIRE(lv.ee.nnz < (int64_t)1 << 31, "coloured smoother: E_E too large for 32-bit row offsets");
  CAV_REQUIRE(lv.big_sum_n < (int64_t)1 << 31, "coloured smoother: too many patch slots for 32-bit offsets");
  P.big.assign(NN, 0);
  P.off.assign(lv.n_big + 1, 0);
  P.inv_off.assign(lv.n_big + 1, 0);
  P.bd.assign(lv.big_sum_n, 0);
  P.row_of.assign(2 * NN, -1);
  P.rowptr.assign(lv.ee.n_rows + 1, 0);
  P.cols.assign(lv.ee.nnz, 0);
  CAV_CHECK_CUDA(cudaMemcpyAsync(P.big.data(), lv.cell_big, NN, cudaMemcpyDeviceToHost, st));
  if (lv.n_big) {
    CAV_CHECK_CUDA(cudaMemcpyAsync(P.off.data(), lv.big_off, sizeof(int64_t) * (lv.n_big + 1), cudaMemcpyDeviceToHost, st));
    CAV_CHECK_CUDA(cudaMemcpyAsync(P.inv_off.data(), lv.inv_off, sizeof(int64_t) * (lv.n_big + 1),
                                   cudaMemcpyDeviceToHost, st));
    CAV_CHECK_CUDA(cudaMemcpyAsync(P.bd.data(), lv.big_dofs, sizeof(int) * lv.big_sum_n, cudaMemcpyDeviceToHost, st));
  }
  if (lv.ee.n_rows) {
    CAV_CHECK_CUDA(cudaMemcpyAsync(P.row_of.data(), lv.ee.row_of, sizeof(int) * 2 * NN, cudaMemcpyDeviceToHost, st));
    CAV_CHECK_CUDA(cudaMemcpyAsync(P.rowptr.data(), lv.ee.rowptr, sizeof(int64_t) * (lv.ee.n_rows + 1),
                                   cudaMemcpyDeviceToHost, st));
    CAV_CHECK_CUDA(cudaMemcpyAsync(P.cols.data(), lv.ee.cols, sizeof(int) * lv.ee.nnz, cudaMemcpyDeviceToHost, st));
  }
  CAV_CHECK_CUDA(cudaStreamSynchronize(st));
}

void colour_plan(Level& lv, ColourPlan& P) {
  const int N = lv.N, NN = N * N, n = 3 * NN;
  const std::vector<uint8_t>& big = P.big;
  const std::vector<int64_t>& off = P.off;
  const std::vector<int>& bd = P.bd;
  const std::vector<int>& row_of = P.row_of;
  const std::vector<int64_t>& rowptr = P.rowptr;
  const std::vector<int>& cols = P.cols;
  // units: the cells (CAV / Vanka patches), or the blocks (box patches, all enlarged)
  const bool box = lv.box;
  const int nunits = box ? lv.n_big : NN;
  // enlarged-patch index of each unit; unknowns of a unit's patch
  std::vector<int> pidx(nunits, -1);
  if (box) std::iota(pidx.begin(), pidx.end(), 0);
  else
    for (int c = 0, q = 0; c < NN; ++c)
      if (big[c]) pidx[c] = q++;
  auto is_big = [&](int c) { return box || big[c] != 0; };
  const bool ch = lv.channel;
  int stdbuf[5];
  auto patch = [&](int c, const int*& ptr, int& len) {
    if (is_big(c)) {
      const int q = pidx[c];
      ptr = bd.data() + off[q];
      len = (int)(off[q + 1] - off[q]);
    } else {
      const int i = c % N, j = c / N;
      len = 0;
      stdbuf[len++] = c;
      stdbuf[len++] = j * N + (i + 1) % N;
      stdbuf[len++] = NN + c;
      if (!(ch && j + 1 == N)) stdbuf[len++] = NN + ((j + 1) % N) * N + i;  // the channel's inflow row: no v_{i,N}
      stdbuf[len++] = 2 * NN + c;
      ptr = stdbuf;
    }
  };
  // holders: for every unknown, the units whose patch holds it (ascending)
  std::vector<int> hoff(n + 1, 0);
  for (int c = 0; c < nunits; ++c) {
    const int* ptr;
    int len;
    patch(c, ptr, len);
    for (int t = 0; t < len; ++t) ++hoff[ptr[t] + 1];
  }
  for (int k = 0; k < n; ++k) hoff[k + 1] += hoff[k];
  std::vector<int> hold(hoff[n]);
  {
    std::vector<int> cur(hoff.begin(), hoff.end() - 1);
    for (int c = 0; c < nunits; ++c) {
      const int* ptr;
      int len;
      patch(c, ptr, len);
      for (int t = 0; t < len; ++t) hold[cur[ptr[t]]++] = c;
    }
  }
  // first fit in visit order: enlarged patches (more than the five unknowns of V_ij) in unit
  // order, then the others; a Vanka patch stored with its own inverse (its unknowns have E_E
  // rows) is still visited with the standard ones
  auto enlarged = [&](int c) {
    if (box) return true;
    if (!is_big(c)) return false;
    const int q = pidx[c];
    return off[q + 1] - off[q] > 5;
  };
  std::vector<int> order;
  order.reserve(nunits);
  for (int c = 0; c < nunits; ++c)
    if (enlarged(c)) order.push_back(c);
  for (int c = 0; c < nunits; ++c)
    if (!enlarged(c)) order.push_back(c);
  std::vector<int> colour(nunits, -1), dstamp(n, -1), cstamp;
  std::vector<int> reach;
  reach.reserve(8192);
  auto wrap = [N](int a) { return a < 0 ? a + N : (a >= N ? a - N : a); };
  for (const int c : order) {
    reach.clear();
    auto add = [&](int k) {
      if (dstamp[k] != c) {
        dstamp[k] = c;
        reach.push_back(k);
      }
    };
    const int* ptr;
    int len;
    patch(c, ptr, len);
    for (int t = 0; t < len; ++t) {
      const int k = ptr[t];
      const int comp = k / NN, cc = k % NN, i = cc % N, j = cc / N;
      add(k);
      // channel: no wrap in y; the outflow row's ghosts reach the v faces of the row (u row)
      // and the u faces of the row (v row), the inflow row loses the prescribed v_{i,N}
      const bool bot = ch && j == 0, top = ch && j + 1 == N;
      if (comp == 0) {  // u row: A0 stencil in u, G to the two adjacent cells
        add(j * N + wrap(i + 1));
        add(j * N + wrap(i - 1));
        if (!top) add(wrap(j + 1) * N + i);
        if (!bot) {
          add(wrap(j - 1) * N + i);
        } else {
          add(NN + j * N + i);
          add(NN + j * N + wrap(i - 1));
        }
        add(2 * NN + j * N + i);
        add(2 * NN + j * N + wrap(i - 1));
      } else if (comp == 1) {
        add(NN + j * N + wrap(i + 1));
        add(NN + j * N + wrap(i - 1));
        if (!top) add(NN + wrap(j + 1) * N + i);
        if (!bot) {
          add(NN + wrap(j - 1) * N + i);
          add(2 * NN + wrap(j - 1) * N + i);
        } else {
          add(j * N + wrap(i + 1));
          add(j * N + i);
        }
        add(2 * NN + j * N + i);
      } else {  // p row: -D
        add(j * N + i);
        add(j * N + wrap(i + 1));
        add(NN + j * N + i);
        if (!top) add(NN + wrap(j + 1) * N + i);
      }
      if (comp < 2 && row_of[k] >= 0) {
        const int r = row_of[k];
        for (int64_t q = rowptr[r]; q < rowptr[r + 1]; ++q) add(cols[q]);
      }
    }
    for (const int k : reach)
      for (int h = hoff[k]; h < hoff[k + 1]; ++h) {
        const int col = colour[hold[h]];
        if (col >= 0) cstamp[col] = c;
      }
    int col = 0;
    while (col < (int)cstamp.size() && cstamp[col] == c) ++col;
    if (col == (int)cstamp.size()) cstamp.push_back(-1);
    colour[c] = col;
  }
  const int nc = (int)cstamp.size();
  lv.n_colours = nc;
  lv.ee_row_max = 0;
  for (int r = 0; r < lv.ee.n_rows; ++r) lv.ee_row_max = std::max(lv.ee_row_max, (int)(rowptr[r + 1] - rowptr[r]));
  check_colour_step(lv);
  lv.colour_of_cell = colour;
  lv.col_big_start.assign(nc + 1, 0);
  lv.col_std_start.assign(nc + 1, 0);
  for (int c = 0; c < nunits; ++c) ++(is_big(c) ? lv.col_big_start : lv.col_std_start)[colour[c] + 1];
  for (int k = 0; k < nc; ++k) {
    lv.col_big_start[k + 1] += lv.col_big_start[k];
    lv.col_std_start[k + 1] += lv.col_std_start[k];
  }
  const int nstd = nunits - lv.n_big;
  std::vector<int> hb(lv.n_big);
  P.hs.assign(nstd, 0);
  {
    std::vector<int> cb(lv.col_big_start.begin(), lv.col_big_start.end() - 1);
    std::vector<int> cs(lv.col_std_start.begin(), lv.col_std_start.end() - 1);
    for (int c = 0; c < nunits; ++c) {
      if (is_big(c)) hb[cb[colour[c]]++] = pidx[c];
      else P.hs[cs[colour[c]]++] = c;
    }
  }
  // job records of the enlarged patches, class by class: (p, n, slot offset) and inverse offset
  P.jobs.resize(lv.n_big);
  P.jinv.resize(lv.n_big);
  for (int t = 0; t < lv.n_big; ++t) {
    const int q = hb[t];
    P.jobs[t] = make_int4(q, (int)(off[q + 1] - off[q]), (int)off[q], 0);
    P.jinv[t] = P.inv_off[q];
  }
}

void colour_upload(cav_hierarchy* H, Level& lv, const ColourPlan& P, cudaStream_t st) {
  Arena& A = H->arena;
  const int NN = lv.N * lv.N;
  const int nstd = (int)P.hs.size();
  lv.col_job = A.alloc<int4>(std::max(lv.n_big, 1));
  lv.col_inv = A.alloc<int64_t>(std::max(lv.n_big, 1));
  if (lv.n_big) {
    CAV_CHECK_CUDA(cudaMemcpyAsync(lv.col_job, P.jobs.data(), sizeof(int4) * lv.n_big, cudaMemcpyHostToDevice, st));
    CAV_CHECK_CUDA(cudaMemcpyAsync(lv.col_inv, P.jinv.data(), sizeof(int64_t) * lv.n_big, cudaMemcpyHostToDevice, st));
  }
  lv.col_std = A.alloc<int>(std::max(nstd, 1));
  if (nstd)
    CAV_CHECK_CUDA(cudaMemcpyAsync(lv.col_std, P.hs.data(), sizeof(int) * nstd, cudaMemcpyHostToDevice, st));
  // the class step's shared memory can exceed the 48 KB default (set here, outside any capture)
  colour_step_attributes();
  if (lv.precision == CAV_PREC_FP32) {
    lv.w32 = A.alloc<float>(3 * (size_t)NN);
    lv.ee_vals32 = A.alloc<float>(std::max<int64_t>(lv.ee.nnz, 1));
    if (lv.ee.nnz) {
      k_round_f32<<<div_up(lv.ee.nnz, 256), 256, 0, st>>>(lv.ee.nnz, lv.ee.vals, lv.ee_vals32);
      CAV_CHECK_LAUNCH();
    }
  }
  lv.slot_ee = A.alloc<int2>(std::max<int64_t>(lv.big_sum_n, 1));
  if (lv.big_sum_n) {
    k_slot_rows<<<div_up(lv.big_sum_n, 256), 256, 0, st>>>(lv.big_sum_n, lv.big_dofs, NN,
                                                           lv.ee.n_rows ? lv.ee.row_of : nullptr, lv.ee.rowptr,
                                                           lv.slot_ee);
    CAV_CHECK_LAUNCH();
  }
  CAV_CHECK_CUDA(cudaStreamSynchronize(st));
}

// ------------------------------------------------------------------ one class step
//
// B300 executes an FP64 instruction of a warp in about 64 cycles whatever the number of
// active lanes, and an SM sustains roughly one FP64 warp instruction per 19 cycles.  The
// residual rows are therefore laid out lane-dense: E_E sums with four lanes per slot on
// warps 0-3, Stokes rows one per lane on warps 4-7, standard cells one row per lane.

constexpr int CS_THREADS = 256;
constexpr int CS_EE_LANES = 4;                   // lanes per slot for the E_E row sums
constexpr int CS_EE_SLOTS = 128 / CS_EE_LANES;   // slots per pass of warps 0-3
constexpr int CS_MAXPASS = 4;                    // row passes of the slice product
constexpr int CS_EE_BATCH = 8;                   // E_E entries gathered per lane before the FMAs
constexpr int CS_CLUSTER = 8;                    // CTAs per enlarged patch
constexpr int CS_SLICE_CAP = 160 * 1024;         // shared-memory bytes for a staged slice
constexpr int CS_STD_WARPS = 4;                  // warps per block on standard cells
constexpr int CS_STD_PER_WARP = 6;               // standard cells per warp (five lanes each)
constexpr int CS_STD_CELLS = CS_STD_WARPS * CS_STD_PER_WARP;

template <typename T>
struct ColourStep {
  int N;
  double ih;        // 1 / h
  double cdiag;     // rho/dt + 4 mu / h^2: the diagonal of A0
  double cnb;       // -mu / h^2: A0's neighbour coefficient
  double dt;
  const int* dofs;
  const double* s_r;
  const double* s_c;
  const T* inv;
  const int2* slot_ee;
  const int* row_of;
  const int64_t* rowptr;
  const int* cols;
  const double* vals;
  const float* vals32;   // E_E values rounded to FP32 (FP32-inverse levels)
  float* w32;            // FP32-inverse levels: (float) of the iterate, kept beside it; null on FP64 levels
  const uint8_t* inject; // box patches: 1 where a slot receives its correction; null: every slot
  const int4* jobs;      // this class's enlarged patches
  const int64_t* job_inv;
  int nbig;
  const int* std_list;   // this class's standard cells
  int nstd;
  int ee_row_max;        // longest E_E row on the level (the per-slot stride of the staged rows)
  int slice_cap;         // bytes of the shared-memory slice buffer (at least one column)
  int chunk_max;         // slots per slice, upper bound over the level
  int ld_max;
  int* status;
  bool channel;          // the channel's boundary rows and standard patches (Sec. 5.3)
  StdInv S;
};

// Slots (columns, and rows of the result) of cluster rank `rank` of C for a patch of n
// slots: rank, rank + C, rank + 2C, ...  Dealing them round-robin balances the E_E rows,
// which sit on the velocity slots only, over the cluster's CTAs.
__device__ inline int slots_of(int n, int rank, int C) { return (n > rank) ? (n - rank + C - 1) / C : 0; }

__device__ inline void cluster_arrive_relaxed() { asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory"); }
__device__ inline void cluster_arrive_release() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ inline void cluster_wait_acquire() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// Precision of a class step's local residual rows: FP64 with FP64 inverses; with FP32
// inverses the whole local solve is an FP32 preconditioner step, so the residual rows are
// evaluated in FP32 from the FP64 iterate (converted on load), which B300 executes about 60
// times faster than FP64.  The iterate update stays FP64.
template <typename T>
struct ResidualType {
  typedef float type;
};
template <>
struct ResidualType<double> {
  typedef double type;
};

// the iterate read from L2 (ld.global.cg): earlier class steps wrote it while this kernel ran.
// FP32 residual rows read the iterate's FP32 copy, which holds exactly (float) of every FP64
// value: the same numbers without a conversion per load (on B300 an FP64-to-FP32 conversion
// holds its SM sub-partition like any FP64 instruction).
template <typename R>
__device__ inline R ldw(const double* p) {
  return (R)__ldcg(p);
}
template <typename R>
__device__ inline R ldw(const float* p) {
  return (R)__ldcg(p);
}
// the iterate the residual rows of precision R read: the FP32 copy or the FP64 iterate
__device__ inline const float* iter_src(const float*, const float* w32, const double*) { return w32; }
__device__ inline const double* iter_src(const double*, const float*, const double* w) { return w; }

// A boundary row (j = 0 or N - 1) of the channel's Stokes part of K_E w, from the ghost rules
// of the level's operator (homogeneous boundary data), with a = rho/dt and m = mu/h^2 written
// as cdiag = a + 4m, cnb = -m:
//   outflow u:  (a + 3m) u - m (u_E + u_W + u_N + v_ij) + m v_{i-1,j} + (p_ij - p_{i-1,j}) / h
//   outflow v:  (a + 3m) v - 3m v_N + m (u_{i+1,j} - u_ij) + 2 p_ij / h
//   inflow u:   (a + 5m) u - m (u_E + u_W + u_S) + (p_ij - p_{i-1,j}) / h
//   inflow v:   (a + 4m) v - m (v_E + v_W + v_S) + (p_ij - p_{i,j-1}) / h
//   inflow p:   -((u_{i+1,j} - u_ij) - v_ij) / h;  the outflow p row is the periodic one.
template <typename R, typename T, typename W>
__device__ inline R channel_row_l2(const ColourStep<T>& a, const W* w, int comp, int i, int j) {
  const int N = a.N, NN = N * N;
  const int ip = (i + 1 == N) ? 0 : i + 1, im = (i == 0) ? N - 1 : i - 1;
  const W* u = w;
  const W* v = w + NN;
  const W* p = w + 2 * NN;
  const int c = j * N + i;
  const R ih = (R)a.ih, m = (R)(-a.cnb), cdiag = (R)a.cdiag;
  if (j == 0) {
    if (comp == 0)
      return (cdiag - m) * ldw<R>(u + c) -
             m * ((ldw<R>(u + j * N + ip) + ldw<R>(u + j * N + im)) + (ldw<R>(u + N + i) + ldw<R>(v + c))) +
             m * ldw<R>(v + j * N + im) + ih * (ldw<R>(p + c) - ldw<R>(p + j * N + im));
    if (comp == 1)
      return (cdiag - m) * ldw<R>(v + c) - (R)3 * m * ldw<R>(v + N + i) +
             m * (ldw<R>(u + j * N + ip) - ldw<R>(u + c)) + (R)2 * ih * ldw<R>(p + c);
    return -((ldw<R>(u + j * N + ip) - ldw<R>(u + c)) + (ldw<R>(v + N + i) - ldw<R>(v + c))) * ih;
  }
  if (comp == 0)
    return (cdiag + m) * ldw<R>(u + c) -
           m * ((ldw<R>(u + j * N + ip) + ldw<R>(u + j * N + im)) + ldw<R>(u + (j - 1) * N + i)) +
           ih * (ldw<R>(p + c) - ldw<R>(p + j * N + im));
  if (comp == 1)
    return cdiag * ldw<R>(v + c) -
           m * ((ldw<R>(v + j * N + ip) + ldw<R>(v + j * N + im)) + ldw<R>(v + (j - 1) * N + i)) +
           ih * (ldw<R>(p + c) - ldw<R>(p + (j - 1) * N + i));
  return -((ldw<R>(u + j * N + ip) - ldw<R>(u + c)) - ldw<R>(v + c)) * ih;
}

// Stokes row of unknown (comp, i, j) of K_E w (Eq. intro_saddle: A0 u + G p, or -D u), in the
// form cdiag u_c + cnb (sum of the four neighbours) + (p_c - p_w) / h, seven operations in R.
template <typename R, typename T, typename W>
__device__ inline R stokes_row_l2(const ColourStep<T>& a, const W* w, int comp, int i, int j) {
  const int N = a.N, NN = N * N;
  if (a.channel && (j == 0 || j + 1 == N)) return channel_row_l2<R>(a, w, comp, i, j);
  const int ip = (i + 1 == N) ? 0 : i + 1, im = (i == 0) ? N - 1 : i - 1;
  const int jp = (j + 1 == N) ? 0 : j + 1, jm = (j == 0) ? N - 1 : j - 1;
  const int c = j * N + i;
  const W* p = w + 2 * NN;
  const R ih = (R)a.ih, cnb = (R)a.cnb, cdiag = (R)a.cdiag;
  if (comp < 2) {
    const W* u = w + comp * NN;
    const int cw = (comp == 0) ? j * N + im : jm * N + i;  // the other cell of the face's gradient
    const R nb = (ldw<R>(u + j * N + ip) + ldw<R>(u + j * N + im)) + (ldw<R>(u + jp * N + i) + ldw<R>(u + jm * N + i));
    return mad(ih, ldw<R>(p + c) - ldw<R>(p + cw), mad(cnb, nb, cdiag * ldw<R>(u + c)));
  }
  const W* u = w;
  const W* v = w + NN;
  return -((ldw<R>(u + j * N + ip) - ldw<R>(u + c)) + (ldw<R>(v + jp * N + i) - ldw<R>(v + c))) * ih;
}

// One class step.  Blocks [0, C nbig) are the clusters of the enlarged patches, the rest take
// the standard cells.  Everything that does not depend on the iterate (job records, slot
// records, b, the E_E entries' L1 prefetch, the TMA copy of the inverse slice) happens before
// pdl_wait(), overlapping the previous class step.
// Column groups of the slice product: FP32 partials are cheap to sum, so the columns are split
// over four groups of 64 threads; FP64 additions cost a 64-cycle warp slot each, so the FP64
// product keeps one group.
template <typename T>
struct ProductShape {
  static constexpr int CG = (sizeof(typename VecLoad<T>::acc_t) == 4) ? 4 : 1;
  static constexpr int RT = CS_THREADS / CG;  // row threads per group
};

template <typename T>
__global__ void __launch_bounds__(CS_THREADS)
k_colour_step(const ColourStep<T> a, const double* __restrict__ b, double* w) {
  typedef VecLoad<T> VL;
  typedef typename VL::acc_t acc_t;
  constexpr int V = VL::V;
  constexpr int C = CS_CLUSTER;
  constexpr int CG = ProductShape<T>::CG, RT = ProductShape<T>::RT;
  typedef typename ResidualType<T>::type res_t;
  const int NN = a.N * a.N;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int big_blocks = a.nbig * C;

  if ((int)blockIdx.x >= big_blocks) {
    pdl_trigger();
    // ---- standard cells: five lanes per cell, one Stokes row each; the shared 5 x 5 inverse
    // is applied after a shuffle of the cell's five residuals
    if (warp >= CS_STD_WARPS) return;
    const int slot = lane / 5, q = lane % 5;
    const int t = ((int)blockIdx.x - big_blocks) * CS_STD_CELLS + warp * CS_STD_PER_WARP + slot;
    const bool act = slot < CS_STD_PER_WARP && t < a.nstd;
    int k = 0, ci = 0, cj = 0, comp = 0, ro = -1, kind = 0;
    double bk = 0.0;
    bool slot_act = act;
    if (act) {
      const int c = a.std_list[t];
      const int i = c % a.N, j = c / a.N;
      const int ip = (i + 1 == a.N) ? 0 : i + 1, jp = (j + 1 == a.N) ? 0 : j + 1;
      kind = std_kind(a.N, j, a.channel);
      // canonical slots: u_ij, u_i+1j, v_ij, v_ij+1, p_ij (the channel's inflow row has no v_ij+1)
      comp = (q < 2) ? 0 : (q < 4 ? 1 : 2);
      ci = (q == 1) ? ip : i;
      cj = (q == 3) ? jp : j;
      k = comp * NN + cj * a.N + ci;
      slot_act = !(kind == 2 && q == 3);
      if (slot_act) {
        bk = b[k];
        if (comp < 2 && a.row_of) ro = a.row_of[k];
      }
    }
    pdl_wait();
    double r = 0.0, old = 0.0;
    if (slot_act) {
      old = __ldcg(w + k);
      double kr = stokes_row_l2<double>(a, w, comp, ci, cj);
      if (ro >= 0) {
        double s = 0.0;
        for (int64_t e = a.rowptr[ro]; e < a.rowptr[ro + 1]; ++e) s += a.vals[e] * __ldcg(w + a.cols[e]);
        kr -= a.dt * s;
      }
      r = bk - kr;
    }
    const int base = (lane / 5) * 5;
    double rr[5];
#pragma unroll
    for (int c2 = 0; c2 < 5; ++c2) rr[c2] = __shfl_sync(0xffffffffu, r, min(base + c2, 31));
    if (slot_act) {
      const double* m = a.S.m[kind] + 5 * q;
      const double nw = old + (m[0] * rr[0] + m[1] * rr[1] + m[2] * rr[2] + m[3] * rr[3] + m[4] * rr[4]);
      w[k] = nw;
      if (a.w32) a.w32[k] = (float)nw;
    }
    return;
  }

  // ---- one CTA of an enlarged patch's cluster
  cluster_arrive_relaxed();  // every CTA of the cluster is running once this phase completes
  const int rank = (int)(blockIdx.x % C);
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  T* xs = reinterpret_cast<T*>(smem + 128);
  const int cm4 = (a.chunk_max + 3) & ~3;
  acc_t* y = reinterpret_cast<acc_t*>(smem + 128 + a.slice_cap);  // [cm4]
  acc_t* recv = y + cm4;                                          // [C][CG][cm4] partials of my rows
  double* sold = reinterpret_cast<double*>(recv + C * CG * cm4);  // [cm4] iterate before the step
  double* ssc = sold + cm4;                                       // [cm4] column scales
  res_t* sb = reinterpret_cast<res_t*>(ssc + cm4);                // [cm4] b at my slots
  res_t* ssr = sb + cm4;                                          // [cm4] row scales (powers of two)
  res_t* see = ssr + cm4;                                         // [cm4] E_E row sums
  res_t* sst = see + cm4;                                         // [cm4] Stokes rows
  int* sk = reinterpret_cast<int*>(sst + cm4);                    // [cm4] unknowns
  int2* se = reinterpret_cast<int2*>(sk + cm4);                   // [cm4] E_E rows
  const int R = a.ee_row_max;
  int* ecol = reinterpret_cast<int*>(se + cm4);                    // [cm4][R] my slots' E_E columns
  res_t* evl = reinterpret_cast<res_t*>(ecol + cm4 * R);          // [cm4][R] and values
  const int4 job = a.jobs[blockIdx.x / C];
  const int64_t ioff = a.job_inv[blockIdx.x / C];
  const int n = job.y;
  const int d0 = job.z;
  const int ld = (n + 7) & ~7;
  const int m = slots_of(n, rank, C);  // this CTA's slots: g = rank + C s, s < m
  const int col_bytes = ld * (int)sizeof(T);
  const int pc = max(1, a.slice_cap / col_bytes);  // columns per staged piece
  const T* X = a.inv + ioff;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0 && m > 0) {
    const int nc = min(pc, m);
    mbar_arrive_expect_tx(bar, (uint32_t)(nc * col_bytes));
    for (int cl = 0; cl < nc; ++cl)
      bulk_copy_g2s(xs + (size_t)cl * ld, X + (int64_t)(rank + C * cl) * ld, (uint32_t)col_bytes, bar);
  }
  // slot records of the slice (independent of the iterate)
  for (int s = tid; s < m; s += CS_THREADS) {
    const int g = d0 + rank + C * s;
    const int k = a.dofs[g];
    sk[s] = k;
    se[s] = a.slot_ee[g];
    ssr[s] = (res_t)a.s_r[g];
    ssc[s] = a.s_c[g];
    sb[s] = (res_t)b[k];
  }
  __syncthreads();
  // the slots' E_E rows (columns and values never change) staged in shared memory, so that
  // after the wait only the iterate is gathered from L2
  const int eg = tid / CS_EE_LANES, el = tid % CS_EE_LANES;  // E_E groups (warps 0-3)
  if (tid < 128)
    for (int s = eg; s < m; s += CS_EE_SLOTS) {
      const int2 e = se[s];
      for (int q = el; q < e.y; q += CS_EE_LANES) {
        ecol[s * R + q] = a.cols[e.x + q];
        evl[s * R + q] = (sizeof(res_t) == 4) ? (res_t)a.vals32[e.x + q] : (res_t)a.vals[e.x + q];
      }
    }
  pdl_wait();
  // Let the next class step launch now: its prologue (job and slot records, staged E_E rows,
  // TMA copies of its inverse slices) overlaps this step's work, and it cannot run further
  // ahead because its own trigger follows its wait for this step.  Triggering at entry
  // instead let several later classes queue their copies ahead of this step's residual reads.
  pdl_trigger();
  // residual rows of the slice: E_E sums on warps 0-3, Stokes rows on warps 4-7, from the
  // iterate's FP32 copy when they are evaluated in FP32
  const auto* wr = iter_src(static_cast<const res_t*>(nullptr), a.w32, w);
  if (tid < 128) {
    for (int t0 = 0; t0 < m; t0 += CS_EE_SLOTS) {
      const int s = t0 + eg;
      int2 e = make_int2(0, 0);
      if (s < m) e = se[s];
      // this lane's entries q = e.x + el + CS_EE_LANES t, t < cnt: in batches, every load of a
      // batch is issued before its FMAs (batch counts are warp-uniform, so no FMA slot is spent
      // on lanes that have run out)
      const int cnt = (e.y > el) ? (e.y - el + CS_EE_LANES - 1) / CS_EE_LANES : 0;
      const int wmax = __reduce_max_sync(0xffffffffu, cnt);
      res_t acc = 0;
      for (int t0 = 0; t0 < wmax; t0 += CS_EE_BATCH) {
        res_t vv[CS_EE_BATCH], wv[CS_EE_BATCH];
#pragma unroll
        for (int t = 0; t < CS_EE_BATCH; ++t) {
          const int q = s * R + el + (t0 + t) * CS_EE_LANES;
          const bool ok = t0 + t < cnt;
          vv[t] = ok ? evl[q] : (res_t)0;
          wv[t] = ok ? ldw<res_t>(wr + ecol[q]) : (res_t)0;
        }
        static_assert(CS_EE_BATCH == 8, "the tail below is written for batches of eight");
        switch (min(wmax - t0, CS_EE_BATCH)) {  // warp-uniform: only the needed FMAs issue
          case 8: acc = mad(vv[7], wv[7], acc);  // fall through
          case 7: acc = mad(vv[6], wv[6], acc);  // fall through
          case 6: acc = mad(vv[5], wv[5], acc);  // fall through
          case 5: acc = mad(vv[4], wv[4], acc);  // fall through
          case 4: acc = mad(vv[3], wv[3], acc);  // fall through
          case 3: acc = mad(vv[2], wv[2], acc);  // fall through
          case 2: acc = mad(vv[1], wv[1], acc);  // fall through
          default: acc = mad(vv[0], wv[0], acc);
        }
      }
#pragma unroll
      for (int o = CS_EE_LANES / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (s < m && el == 0) see[s] = acc;
    }
  } else {
    for (int s = tid - 128; s < m; s += 128) {
      const int k = sk[s];
      const int comp = k / NN, cc = k % NN;
      sold[s] = __ldcg(w + k);
      sst[s] = stokes_row_l2<res_t>(a, wr, comp, cc % a.N, cc / a.N);
    }
  }
  __syncthreads();
  // y = D_r (b - K_E w), K_E w = Stokes - dt E_E w (E_E rows only on velocities that have one)
  for (int s = tid; s < m; s += CS_THREADS) {
    const res_t kr = (se[s].y > 0) ? sst[s] - (res_t)a.dt * see[s] : sst[s];
    y[s] = (acc_t)(ssr[s] * (sb[s] - kr));
  }
  __syncthreads();
  // partial product X[:, slice] y[slice]: column group cgp takes the slice's columns
  // cgp, cgp + CG, ...; each of its RT threads owns V consecutive rows per pass
  const int cgp = tid / RT, rt = tid % RT;
  acc_t accv[CS_MAXPASS][V];
#pragma unroll
  for (int ps = 0; ps < CS_MAXPASS; ++ps)
#pragma unroll
    for (int v = 0; v < V; ++v) accv[ps][v] = 0;
  // A bounded wait that runs out records DEV_TIMEOUT; the CTA then stops staging (the host
  // reports IB_ERR_TIMEOUT), after waiting for the copy in flight to land.
  bool alive = true;
  const bool stall = wait_stall_enabled();
  uint32_t phase = 0;
  for (int b0 = 0; b0 < m; b0 += pc) {
    const int nc = min(pc, m - b0);
    const bool got = mbar_wait(bar, phase, a.status, nullptr, stall);
    if (got) {
#pragma unroll
      for (int ps = 0; ps < CS_MAXPASS; ++ps) {
        const int r0 = (ps * RT + rt) * V;
        if (r0 < n) {
#pragma unroll 4
          for (int cl = cgp; cl < nc; cl += CG) {
            acc_t x[V];
            VL::load_shared(xs + (size_t)cl * ld + r0, x);
            const acc_t yc = y[b0 + cl];
#pragma unroll
            for (int v = 0; v < V; ++v) accv[ps][v] = mad(x[v], yc, accv[ps][v]);
          }
        }
      }
    }
    alive = __syncthreads_and(got ? 1 : 0) != 0;  // one decision for the whole CTA
    if (!alive) {
      if (tid == 0) mbar_drain(bar, phase, a.status);
      __syncthreads();
      break;
    }
    if (tid == 0 && b0 + pc < m) {
      const int nn = min(pc, m - b0 - pc);
      mbar_arrive_expect_tx(bar, (uint32_t)(nn * col_bytes));
      for (int cl = 0; cl < nn; ++cl)
        bulk_copy_g2s(xs + (size_t)cl * ld, X + (int64_t)(rank + C * (b0 + pc + cl)) * ld, (uint32_t)col_bytes,
                      bar);
    }
    phase ^= 1u;
  }
  // push each row's partial to the CTA owning that row (distributed shared memory)
  cg::cluster_group cluster = cg::this_cluster();
  cluster_wait_acquire();  // the start-up phase: every CTA of the cluster is running
#pragma unroll
  for (int ps = 0; ps < CS_MAXPASS; ++ps) {
    const int r0 = (ps * RT + rt) * V;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int row = r0 + v;
      if (row < n) {
        acc_t* dst = cluster.map_shared_rank(recv, row % C);
        dst[(rank * CG + cgp) * cm4 + row / C] = accv[ps][v];
      }
    }
  }
  cluster_arrive_release();
  cluster_wait_acquire();
  // my rows: sum the C partials in rank order, scale, add to the iterate
  for (int s = tid; s < m; s += CS_THREADS) {
    acc_t sum = 0;
#pragma unroll
    for (int q = 0; q < C * CG; ++q) sum += recv[q * cm4 + s];
    // restricted injection (box patches): only the unexpanded block's unknowns are written
    if (a.inject == nullptr || a.inject[d0 + rank + C * s]) {
      const double nw = sold[s] + ssc[s] * (double)sum;
      w[sk[s]] = nw;
      if (a.w32) a.w32[sk[s]] = (float)nw;
    }
  }
}

// Kernel attributes of the class step, set once per set-up outside any capture: dynamic shared
// memory above the 48 KB default, and clusters above the portable size of 8 when configured.
static void colour_step_attributes() {
  CAV_CHECK_CUDA(cudaFuncSetAttribute(k_colour_step<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  CAV_CHECK_CUDA(cudaFuncSetAttribute(k_colour_step<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  if (CS_CLUSTER > 8) {
    CAV_CHECK_CUDA(cudaFuncSetAttribute(k_colour_step<double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    CAV_CHECK_CUDA(cudaFuncSetAttribute(k_colour_step<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  }
}

// The FP32 copy of E_E's values on an FP32-inverse coloured level, after E_E's values changed
// (cav_refactor); the other class-step records depend on the structure only.
void colour_refresh_values(Level& lv, cudaStream_t st) {
  if (lv.precision == CAV_PREC_FP32 && lv.ee.nnz) {
    k_round_f32<<<div_up(lv.ee.nnz, 256), 256, 0, st>>>(lv.ee.nnz, lv.ee.vals, lv.ee_vals32);
    CAV_CHECK_LAUNCH();
  }
}

void colour_set_wait_stall(int enable) {
  CAV_CHECK_CUDA(cudaMemcpyToSymbol(g_wait_stall, &enable, sizeof(int)));
}

// Sums of the pressure block over tiles of 256 cells (fixed order), for the mean removal.
__global__ void k_pressure_partials(int NN, const double* __restrict__ p, double* __restrict__ partial) {
  __shared__ double sm[8];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const double v = (c < NN) ? p[c] : 0.0;
  const double t = block_sum(v, sm);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

template <typename T>
static size_t step_smem(int chunk_max, int slice_cap, int ee_row_max) {
  typedef typename VecLoad<T>::acc_t acc_t;
  typedef typename ResidualType<T>::type res_t;
  const int cm4 = (chunk_max + 3) & ~3;
  return 128 + (size_t)slice_cap + sizeof(acc_t) * (size_t)(cm4 * (1 + CS_CLUSTER * ProductShape<T>::CG)) +
         (size_t)cm4 * (2 * sizeof(double) + 4 * sizeof(res_t) + sizeof(int) + sizeof(int2)) +
         (size_t)cm4 * ee_row_max * (sizeof(int) + sizeof(res_t));
}

// Slice layout of a level's class steps: padded column length, slots per CTA, bytes of the
// staged inverse slice, and the dynamic shared memory that follows from them.
struct StepShape {
  int ld_max, chunk_max, slice_cap;
  size_t smem;
};
template <typename T>
static StepShape step_shape(const Level& lv) {
  StepShape sh;
  const int max_n = std::max(lv.big_max_n, 1);
  sh.ld_max = round8(max_n);
  sh.chunk_max = (max_n + CS_CLUSTER - 1) / CS_CLUSTER;
  const int col_bytes = sh.ld_max * (int)sizeof(T);
  sh.slice_cap = std::min(sh.chunk_max * col_bytes, std::max(col_bytes, (CS_SLICE_CAP / col_bytes) * col_bytes));
  sh.smem = step_smem<T>(sh.chunk_max, sh.slice_cap, lv.ee_row_max);
  return sh;
}

void check_colour_step(const Level& lv) {
  const bool f32 = lv.precision == CAV_PREC_FP32;
  const int max_n = f32 ? CS_MAXPASS * ProductShape<float>::RT * VecLoad<float>::V
                        : CS_MAXPASS * ProductShape<double>::RT * VecLoad<double>::V;
  CAV_REQUIRE(lv.big_max_n <= max_n, "coloured smoother: patch too large");
  const size_t smem = f32 ? step_shape<float>(lv).smem : step_shape<double>(lv).smem;
  CAV_REQUIRE(smem <= 200 * 1024, "coloured smoother: class step needs too much shared memory "
                                  "(patches too large, or E_E rows too long)");
}

template <typename T>
static void launch_step(const cav_hierarchy* H, const Level& lv, const T* inv, int k, const double* b, double* w,
                        bool programmatic, cudaStream_t st) {
  ColourStep<T> a;
  a.N = lv.N;
  a.ih = 1.0 / lv.h;
  const double ih2 = 1.0 / (lv.h * lv.h);
  a.cdiag = lv.rho_dt + 4.0 * lv.mu * ih2;
  a.cnb = -lv.mu * ih2;
  a.dt = lv.dt;
  a.dofs = lv.big_dofs;
  a.s_r = lv.s_r;
  a.s_c = lv.s_c;
  a.inv = inv;
  a.slot_ee = lv.slot_ee;
  const bool has_ee = lv.ee.n_rows > 0;
  a.row_of = has_ee ? lv.ee.row_of : nullptr;
  a.rowptr = lv.ee.rowptr;
  a.cols = lv.ee.cols;
  a.vals = lv.ee.vals;
  a.vals32 = lv.ee_vals32;
  a.w32 = lv.w32;
  a.inject = lv.inject;
  a.jobs = lv.col_job + lv.col_big_start[k];
  a.job_inv = lv.col_inv + lv.col_big_start[k];
  a.nbig = lv.col_big_start[k + 1] - lv.col_big_start[k];
  a.std_list = lv.col_std + lv.col_std_start[k];
  a.nstd = lv.col_std_start[k + 1] - lv.col_std_start[k];
  const StepShape sh = step_shape<T>(lv);
  a.ld_max = sh.ld_max;
  a.chunk_max = sh.chunk_max;
  a.slice_cap = sh.slice_cap;
  a.status = H->status;
  for (int kd = 0; kd < 3; ++kd)
    for (int q = 0; q < 25; ++q) a.S.m[kd][q] = lv.std_inv[kd][q];
  a.channel = lv.channel;
  a.ee_row_max = lv.ee_row_max;
  const size_t smem = sh.smem;
  CAV_REQUIRE(smem <= 200 * 1024, "coloured smoother: class step needs too much shared memory");
  const int std_blocks = div_up(a.nstd, CS_STD_CELLS);
  int grid = a.nbig * CS_CLUSTER + std_blocks;
  grid = div_up(grid, CS_CLUSTER) * CS_CLUSTER;
  if (grid == 0) return;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(CS_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS_CLUSTER;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = programmatic ? 2 : 1;
  CAV_CHECK_CUDA(cudaLaunchKernelEx(&cfg, k_colour_step<T>, a, b, w));
  CAV_CHECK_LAUNCH();
}

// Largest patch the class step handles: CS_MAXPASS row passes per thread.
template <typename T>
static int colour_max_n() {
  return CS_MAXPASS * ProductShape<T>::RT * VecLoad<T>::V;
}

void coloured_sweep(const cav_hierarchy* H, int l, const double* b, double* w, bool w_is_zero, double* partial,
                    bool remove_mean, bool profile, cudaStream_t st) {
  const Level& lv = H->levels[l];
  const int NN = lv.N * lv.N;
  CAV_REQUIRE(lv.precision != CAV_PREC_BF16,
              "coloured smoother: BF16 patch inverses make the undamped multiplicative sweep diverge; "
              "use FP32 or FP64");
  if (w_is_zero) CAV_CHECK_CUDA(cudaMemsetAsync(w, 0, sizeof(double) * 3 * (size_t)NN, st));
  if (lv.w32) {  // the FP32 copy the class steps' residual rows read, equal to (float) w
    if (w_is_zero) {
      CAV_CHECK_CUDA(cudaMemsetAsync(lv.w32, 0, sizeof(float) * 3 * (size_t)NN, st));
    } else {
      k_to_f32<<<div_up(3 * (int64_t)NN, 256), 256, 0, st>>>(3 * (int64_t)NN, w, lv.w32);
      CAV_CHECK_LAUNCH();
    }
  }
  if (profile) prof_begin(H, l, st);
  for (int k = 0; k < lv.n_colours; ++k) {
    // class steps after the first overlap their prologue with the step before them
    const bool programmatic = k > 0;
    if (lv.precision == CAV_PREC_FP32) {
      CAV_REQUIRE(lv.big_max_n <= colour_max_n<float>(), "coloured smoother: patch too large");
      launch_step<float>(H, lv, lv.inv32, k, b, w, programmatic, st);
    } else {
      CAV_REQUIRE(lv.big_max_n <= colour_max_n<double>(), "coloured smoother: patch too large");
      launch_step<double>(H, lv, lv.inv64, k, b, w, programmatic, st);
    }
  }
  if (profile) prof_end(H, l, st);
  // the channel's pressure is determined (traction outflow): no mean to remove
  if (remove_mean && !lv.channel) pressure_mean_remove(lv.N, partial, w + 2 * (size_t)NN, st);
}

void pressure_mean_remove(int N, double* partial, double* p, cudaStream_t st) {
  const int nblk = div_up(N * N, 256);
  k_pressure_partials<<<nblk, 256, 0, st>>>(N * N, p, partial);
  CAV_CHECK_LAUNCH();
  launch_remove_mean(N, nblk, partial, p, st);
}

}  // namespace cav
