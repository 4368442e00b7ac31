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
  const double* w;
  const double* b;     // nullable (= 0)
  double* out;
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
    const StokesRows k = stokes_rows(N, a.h, a.rho_dt, a.mu, a.w, i, j, a.channel);
    const bool eu = a.row_of && a.row_of[c] >= 0, ev = a.row_of && a.row_of[NN + c] >= 0;
    const double* b = a.b;
    if (a.mode == 0) {
      if (!eu) a.out[c] = (b ? b[c] : 0.0) - k.ku;
      if (!ev) a.out[NN + c] = (b ? b[NN + c] : 0.0) - k.kv;
      a.out[2 * NN + c] = (b ? b[2 * NN + c] : 0.0) - k.kp;
    } else {
      if (!eu) a.out[c] = k.ku;
      if (!ev) a.out[NN + c] = k.kv;
      a.out[2 * NN + c] = k.kp;
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
    const StokesRows k = stokes_rows(N, a.h, a.rho_dt, a.mu, a.w, c % N, c / N, a.channel);
    const double kr = ((comp == 0) ? k.ku : k.kv) - a.dt * s;
    a.out[row] = (a.mode == 0) ? ((a.b ? a.b[row] : 0.0) - kr) : kr;
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
  double* w;
  int w_is_zero;
  double* partial;
  bool channel;
};

// One 256-thread block of the scatter / update.
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
// Each block writes the partial sum of the new pressures it produced (fixed order) to
// partial[vb]; the stencil blocks' partials come first, then the touched blocks'.
//
// update_warp is warp `warp` of block vb: every lane of the calling warp takes part, and every
// lane returns the warp's sum of new pressures (fixed order).  Warps of one block are
// independent, so any warp may do any block's share.
__device__ inline double update_warp(const UpdArgs& a, int vb, int warp) {
  const int N = a.N, NN = N * N;
  const int lane = threadIdx.x & 31;
  const StdInv& S = a.S;
  const double* r = a.r;
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
        const double s = std_row(S, 1, r, N, im, j, channel) + std_row(S, 0, r, N, i, j, channel);
        w[c] = (a.w_is_zero ? 0.0 : w[c]) + a.alpha * (s / 2.0);
      }
      if (a.inc_off[NN + c + 1] == a.inc_off[NN + c]) {
        if (channel && j == 0) {  // the outflow row's v face: one incident cell
          const double s = std_row(S, 2, r, N, i, j, channel);
          w[NN + c] = (a.w_is_zero ? 0.0 : w[NN + c]) + a.alpha * s;
        } else {
          const double s = std_row(S, 3, r, N, i, jm, channel) + std_row(S, 2, r, N, i, j, channel);
          w[NN + c] = (a.w_is_zero ? 0.0 : w[NN + c]) + a.alpha * (s / 2.0);
        }
      }
      if (a.inc_off[2 * NN + c + 1] == a.inc_off[2 * NN + c]) {
        const double s = std_row(S, 4, r, N, i, j, channel);
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
      for (int64_t q = q0 + sl; q < q1; q += TOUCH_LANES) s += a.delta[a.inc_slot[q]];
    }
#pragma unroll
    for (int o = TOUCH_LANES / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (k >= 0) {
      if (sl == 0) {
        const int comp = k / NN, c = k % NN, i = c % N, j = c / N;
        const int im = (i == 0) ? N - 1 : i - 1, jm = (j == 0) ? N - 1 : j - 1;
        int cnt = (int)(q1 - q0);
        double st = 0.0;
        const uint8_t* cell_big = a.cell_big;
        if (comp == 0) {
          if (!cell_big[j * N + im]) { st += std_row(S, 1, r, N, im, j, channel); ++cnt; }
          if (!cell_big[c]) { st += std_row(S, 0, r, N, i, j, channel); ++cnt; }
        } else if (comp == 1) {
          if (!(channel && j == 0) && !cell_big[jm * N + i]) { st += std_row(S, 3, r, N, i, jm, channel); ++cnt; }
          if (!cell_big[c]) { st += std_row(S, 2, r, N, i, j, channel); ++cnt; }
        } else {
          if (!cell_big[c]) { st += std_row(S, 4, r, N, i, j, channel); ++cnt; }
        }
        const double nw = (a.w_is_zero ? 0.0 : w[k]) + a.alpha * ((st + s) / (double)cnt);
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
