// The pieces of one weighted additive sweep (Eq. additive_cav_saddle) that its separate
// kernels (k_residual, k_update, k_remove_mean) and the fused persistent sweep kernel share.
// Each function is the work of one (virtual) block, so both forms do the same arithmetic in
// the same order and produce the same bits.
#pragma once

#include "device_util.cuh"
#include "internal.cuh"
#include "level_math.cuh"

namespace cav {

constexpr int ROWS_PER_WARP = 32 / ROW_LANES;  // E_E rows per warp: 8 lanes each

struct ResArgs {
  int N;
  double h, rho_dt, mu, dt;
  StokesCoef sc;       // the Stokes rows' coefficients (1 / h, 1 / h^2, 2 mu / h from the host)
  const double* w;
  const double* b;     // nullable (= 0)
  double* out;
  float* out32;        // nullable: out rounded to FP32 as well (the sweeps of FP32 / BF16 levels)
  int mode;            // 0: out = b - K_E w;  1: out = K_E w
  int gx;              // cell tiles along x (32 cells wide)
  int nb_cells;        // cell tiles
  const int* row_of;   // nullable: E_E row index of each velocity unknown (-1: none)
  int n_rows;
  const int* rows;
  const int64_t* rowptr;
  const int* cols;
  const double* vals;
  bool channel;
};

// One block of the residual with WARPS warps (tid < 32 WARPS).  Blocks [0, nb_cells) take a
// 32 x WARPS tile of cells, one thread per cell, and write every row there except the
// velocity rows E_E touches; the remaining blocks take those rows eight lanes each (four rows
// per warp) and write the Stokes part plus -dt sum_l E_E[row, l] w[l] (fixed lane-strided
// order, fixed shuffle tree).  Every row's value is independent of WARPS.
template <int WARPS>
__device__ inline void residual_block(const ResArgs& a, int vb, int tid) {
  const int N = a.N, NN = N * N;
  if (vb < a.nb_cells) {
    const int i = (vb % a.gx) * 32 + (tid % 32);
    const int j = (vb / a.gx) * WARPS + (tid / 32);
    if (i >= N || j >= N) return;
    const int c = j * N + i;
    const StokesRows k = stokes_rows(N, a.sc, a.w, i, j, a.channel);
    const bool eu = a.row_of && a.row_of[c] >= 0, ev = a.row_of && a.row_of[NN + c] >= 0;
    const double* b = a.b;
    double ou = k.ku, ov = k.kv, op = k.kp;
    if (a.mode == 0) {
      ou = (b ? b[c] : 0.0) - k.ku;
      ov = (b ? b[NN + c] : 0.0) - k.kv;
      op = (b ? b[2 * NN + c] : 0.0) - k.kp;
    }
    if (!eu) a.out[c] = ou;
    if (!ev) a.out[NN + c] = ov;
    a.out[2 * NN + c] = op;
    if (a.out32) {
      if (!eu) a.out32[c] = (float)ou;
      if (!ev) a.out32[NN + c] = (float)ov;
      a.out32[2 * NN + c] = (float)op;
    }
    return;
  }
  const int warp = tid >> 5, lane = tid & 31;
  const int sub = lane / ROW_LANES, sl = lane % ROW_LANES;
  const int r = ((vb - a.nb_cells) * WARPS + warp) * ROWS_PER_WARP + sub;
  double s = (r < a.n_rows) ? ee_row_lane_sum(a.rowptr, a.cols, a.vals, a.w, r, sl) : 0.0;
  s = row_group_reduce(s);
  if (r < a.n_rows && sl == 0) {
    const int row = a.rows[r];
    const int comp = row / NN, c = row % NN;
    // only this row's Stokes part (the active rows are sorted, u rows first, so a warp's rows
    // are nearly always of one component and one branch runs)
    double kst;
    if (comp == 0) kst = stokes_u_row(N, a.sc, a.w, c % N, c / N, a.channel);
    else kst = stokes_v_row(N, a.sc, a.w, c % N, c / N, a.channel);
    const double kr = kst - a.dt * s;
    const double o = (a.mode == 0) ? ((a.b ? a.b[row] : 0.0) - kr) : kr;
    a.out[row] = o;
    if (a.out32) a.out32[row] = (float)o;
  }
}

constexpr int UPD_THREADS = 256;
constexpr int TOUCH_WARPS = UPD_THREADS / 32;

struct UpdArgs {
  int N;
  double alpha;
  StdInv S;
  int nb_std, gx;
  const int64_t* inc_off;
  int n_touched;
  const int* touched;
  const uint8_t* cell_big;
  const int* inc_slot;
  const double* delta;
  const double* r;
  const float* r32;       // nullable: r in FP32; the standard patches are then applied in FP32 (S32)
  StdInv32 S32;
  double* w;
  int w_is_zero;
  double* partial;
  bool channel;
  const double* theta_t;  // [n_touched] 1 / (patches holding the unknown): Theta of Eq. additive_cav_saddle
};
static_assert(TOUCH_WARPS * TOUCH_PER_WARP == SCATTER_TOUCHED_PER_BLOCK, "the scatter's block shape");

// Correction of row `row` of the standard patch of cell (i, j): FP64 from r, or FP32 from r32.
__device__ inline double std_corr(const UpdArgs& a, int row, int i, int j) {
  return a.r32 ? (double)std_row32(a.S32, row, a.r32, a.N, i, j, a.channel)
               : std_row(a.S, row, a.r, a.N, i, j, a.channel);
}
// The sum of rows r1 of cell (i1, j1) and r2 of cell (i2, j2) (formed in FP32 on FP32 levels).
__device__ inline double std_corr2(const UpdArgs& a, int r1, int i1, int j1, int r2, int i2, int j2) {
  if (a.r32)
    return (double)(std_row32(a.S32, r1, a.r32, a.N, i1, j1, a.channel) +
                    std_row32(a.S32, r2, a.r32, a.N, i2, j2, a.channel));
  return std_row(a.S, r1, a.r, a.N, i1, j1, a.channel) + std_row(a.S, r2, a.r, a.N, i2, j2, a.channel);
}

// One 256-thread block of the scatter / update.
//  * Blocks [0, nb_std): a 32 x 8 tile of cells, one thread per cell.  For each unknown of the
//    cell that no enlarged patch holds, both incident cells (one for a pressure) keep their
//    standard patch, so count_k is 2 (1) and the correction is the stencil of the shared 5x5
//    inverse applied to r.
//  * The remaining blocks: four lanes per unknown held by at least one enlarged patch (eight
//    unknowns per warp).  The lanes sum the enlarged patches' corrections at the unknown (fixed
//    lane-strided order, fixed shuffle tree); the group's first lane adds the standard patches
//    of its incident cells that kept their Vanka patch and multiplies by Theta_k, the
//    reciprocal of the total patch count (formed once at set-up: an FP64 division per unknown
//    and sweep costs B300 more than the rest of the unknown's update).
// On the channel a v face of the outflow row has one incident cell (the one above it), and
// the standard patches of the outflow and inflow rows have their own inverses.
// Each block writes the partial sum of the new pressures it produced (fixed order) to
// partial[vb]; the stencil blocks' partials come first, then the touched blocks'.
//
// update_warp is warp `warp` of block vb: every lane of the calling warp takes part, and every
// lane returns the warp's sum of new pressures (fixed order).  Warps of one block are
// independent, so any warp may do any block's share.
__device__ inline double update_warp(const UpdArgs& a, int vb, int warp) {
  const int N = a.N, NN = N * N;
  const int lane = threadIdx.x & 31;
  double* w = a.w;
  const bool channel = a.channel;
  double pnew = 0.0;
  if (vb < a.nb_std) {
    const int i = (vb % a.gx) * 32 + lane;
    const int j = (vb / a.gx) * 8 + warp;
    if (i < N && j < N) {
      const int c = j * N + i;
      const int im = (i == 0) ? N - 1 : i - 1, jm = (j == 0) ? N - 1 : j - 1;
      if (a.inc_off[c + 1] == a.inc_off[c]) {
        const double s = std_corr2(a, 1, im, j, 0, i, j);
        w[c] = (a.w_is_zero ? 0.0 : w[c]) + a.alpha * (s / 2.0);
      }
      if (a.inc_off[NN + c + 1] == a.inc_off[NN + c]) {
        if (channel && j == 0) {  // the outflow row's v face: one incident cell
          const double s = std_corr(a, 2, i, j);
          w[NN + c] = (a.w_is_zero ? 0.0 : w[NN + c]) + a.alpha * s;
        } else {
          const double s = std_corr2(a, 3, i, jm, 2, i, j);
          w[NN + c] = (a.w_is_zero ? 0.0 : w[NN + c]) + a.alpha * (s / 2.0);
        }
      }
      if (a.inc_off[2 * NN + c + 1] == a.inc_off[2 * NN + c]) {
        const double s = std_corr(a, 4, i, j);
        pnew = (a.w_is_zero ? 0.0 : w[2 * NN + c]) + a.alpha * s;
        w[2 * NN + c] = pnew;
      }
    }
    pnew = warp_sum(pnew);
  } else {
    const int sub = lane / TOUCH_LANES, sl = lane % TOUCH_LANES;
    const int t = ((vb - a.nb_std) * TOUCH_WARPS + warp) * TOUCH_PER_WARP + sub;
    double s = 0.0;
    int k = -1;
    int64_t q0 = 0, q1 = 0;
    if (t < a.n_touched) {
      k = a.touched[t];
      q0 = a.inc_off[k];
      q1 = a.inc_off[k + 1];
      s = touched_lane_sum(a.inc_slot, a.delta, q0, q1, sl);
    }
#pragma unroll
    for (int o = TOUCH_LANES / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (k >= 0) {
      if (sl == 0) {
        const StdHolders hs = std_holders(N, a.cell_big, channel, k);
        double st = 0.0;
        if (hs.n > 0) st += std_corr(a, hs.row0, hs.i0, hs.j0);
        if (hs.n > 1) st += std_corr(a, hs.row1, hs.i1, hs.j1);
        const double nw = (a.w_is_zero ? 0.0 : w[k]) + a.alpha * ((st + s) * a.theta_t[t]);
        w[k] = nw;
        if (k >= 2 * NN) pnew = nw;
      }
    }
    // the warp's new pressures: group leaders' values in fixed order
    double wp = 0.0;
#pragma unroll
    for (int g = 0; g < TOUCH_PER_WARP; ++g) wp += __shfl_sync(0xffffffffu, pnew, g * TOUCH_LANES);
    pnew = wp;
  }
  return pnew;
}

// One whole block (every thread calls this): its warps' sums in warp order into partial[vb].
// sm: 8 doubles of shared memory.
__device__ inline void update_block(const UpdArgs& a, int vb, double* sm) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double pnew = update_warp(a, vb, warp);
  if (lane == 0) sm[warp] = pnew;
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0;
    for (int q = 0; q < 8; ++q) tot += sm[q];
    a.partial[vb] = tot;
  }
  __syncthreads();  // sm is reused by the caller's next block
}

// p -= mean(p) as block vb of nvb 256-thread blocks: every block reduces the partials in the
// same order, then subtracts on its cells.  sm: 8 doubles of shared memory.
__device__ inline void remove_mean_block(int N, int n_partial, const double* partial, double* p, int vb, int nvb,
                                         double* sm) {
  double t = 0.0;
  for (int q = threadIdx.x; q < n_partial; q += UPD_THREADS) t += partial[q];
  t = block_sum(t, sm);
  const double mean = t / ((double)N * (double)N);
  for (int c = vb * UPD_THREADS + threadIdx.x; c < N * N; c += nvb * UPD_THREADS) p[c] -= mean;
}

// host side (stencil.cu): the residual's arguments for blocks of `warps` warps, and its block count
ResArgs residual_args(const LevelOps& op, const double* w, const double* b, double* out, int mode, int warps);
int residual_blocks(const ResArgs& a, int warps);

}  // namespace cav
