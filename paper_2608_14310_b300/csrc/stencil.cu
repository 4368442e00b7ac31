// Stokes stencils of K_E, the E_E product, and the grid transfers of Sec. 4.
#include "internal.cuh"
#include "device_util.cuh"
#include "level_math.cuh"

namespace cav {

constexpr int RES_BX = 32, RES_BY = 8, RES_WARPS = RES_BX * RES_BY / 32;
constexpr int ROWS_PER_WARP = 32 / ROW_LANES;  // E_E rows: 8 lanes each

// Residual (mode 0: out = b - K_E w, b may be null) or product (mode 1: out = K_E w) in one
// launch with two block roles.  Blocks [0, nb_cells) take a 32 x 8 tile of cells, one thread
// per cell, and write every row there except the velocity rows E_E touches; the remaining
// blocks take those rows eight lanes each (four rows per warp) and write the Stokes part plus
// -dt sum_l E_E[row, l] w[l] (fixed lane-strided order, fixed shuffle tree).
__global__ void __launch_bounds__(RES_BX* RES_BY)
k_residual(int N, double h, double rho_dt, double mu, double dt, const double* __restrict__ w,
           const double* __restrict__ b, double* __restrict__ out, int mode, int nb_cells, int gx,
           const int* __restrict__ row_of, int n_rows, const int* __restrict__ rows,
           const int64_t* __restrict__ rowptr, const int* __restrict__ cols, const double* __restrict__ vals,
           bool channel) {
  pdl_wait();  // programmatic launch: the kernel ahead (which writes w or b) has finished
  pdl_trigger();
  const int NN = N * N;
  if ((int)blockIdx.x < nb_cells) {
    const int i = (blockIdx.x % gx) * RES_BX + (threadIdx.x % RES_BX);
    const int j = (blockIdx.x / gx) * RES_BY + (threadIdx.x / RES_BX);
    if (i >= N || j >= N) return;
    const int c = j * N + i;
    const StokesRows k = stokes_rows(N, h, rho_dt, mu, w, i, j, channel);
    const bool eu = row_of && row_of[c] >= 0, ev = row_of && row_of[NN + c] >= 0;
    if (mode == 0) {
      if (!eu) out[c] = (b ? b[c] : 0.0) - k.ku;
      if (!ev) out[NN + c] = (b ? b[NN + c] : 0.0) - k.kv;
      out[2 * NN + c] = (b ? b[2 * NN + c] : 0.0) - k.kp;
    } else {
      if (!eu) out[c] = k.ku;
      if (!ev) out[NN + c] = k.kv;
      out[2 * NN + c] = k.kp;
    }
    return;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / ROW_LANES, sl = lane % ROW_LANES;
  const int r = (((int)blockIdx.x - nb_cells) * RES_WARPS + warp) * ROWS_PER_WARP + sub;
  double s = (r < n_rows) ? ee_row_lane_sum(rowptr, cols, vals, w, r, sl) : 0.0;
  s = row_group_reduce(s);
  if (r < n_rows && sl == 0) {
    const int row = rows[r];
    const int comp = row / NN, c = row % NN;
    const StokesRows k = stokes_rows(N, h, rho_dt, mu, w, c % N, c / N, channel);
    const double kr = ((comp == 0) ? k.ku : k.kv) - dt * s;
    out[row] = (mode == 0) ? ((b ? b[row] : 0.0) - kr) : kr;
  }
}

void launch_apply(const LevelOps& op, const double* w, const double* b, double* out, int mode,
                  cudaStream_t st, bool pdl) {
  const int gx = div_up(op.N, RES_BX), gy = div_up(op.N, RES_BY);
  const int nb_cells = gx * gy;
  const bool has_ee = op.ee && op.ee->n_rows > 0;
  const int nb_rows = has_ee ? div_up(op.ee->n_rows, RES_WARPS * ROWS_PER_WARP) : 0;
  launch_k(k_residual, dim3(nb_cells + nb_rows), dim3(RES_BX * RES_BY), 0, st, pdl, op.N, op.h, op.rho_dt, op.mu,
           op.dt, w, b, out, mode, nb_cells, gx, has_ee ? op.ee->row_of : nullptr, has_ee ? op.ee->n_rows : 0,
           has_ee ? op.ee->rows : nullptr, has_ee ? op.ee->rowptr : nullptr, has_ee ? op.ee->cols : nullptr,
           has_ee ? op.ee->vals : nullptr, op.channel);
}

// Restriction (Sec. 4), one thread per coarse cell (I, J).
__global__ void k_restrict(int Nc, const double* __restrict__ rf, double* __restrict__ bc, bool channel) {
  pdl_wait();
  pdl_trigger();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= Nc || J >= Nc) return;
  restrict_cell(Nc, rf, bc, I, J, channel);
}

// w_f += P x_c (Sec. 4), one thread per fine cell (i, j).
__global__ void k_prolong_add(int Nc, const double* __restrict__ xc, double* __restrict__ wf, bool channel) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= 2 * Nc || j >= 2 * Nc) return;
  prolong_cell(Nc, xc, wf, i, j, channel);
}

void launch_restrict(int Nc, const double* r_f, double* b_c, bool channel, cudaStream_t st, bool pdl) {
  launch_k(k_restrict, dim3(div_up(Nc, 32), div_up(Nc, 8)), dim3(32, 8), 0, st, pdl, Nc, r_f, b_c, channel);
}

void launch_prolong_add(int Nc, const double* x_c, double* w_f, bool channel, cudaStream_t st, bool pdl) {
  launch_k(k_prolong_add, dim3(div_up(2 * Nc, 32), div_up(2 * Nc, 8)), dim3(32, 8), 0, st, pdl, Nc, x_c, w_f,
           channel);
}

}  // namespace cav
