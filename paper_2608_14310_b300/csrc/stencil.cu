// Stokes stencils of K_E, the E_E product, and the grid transfers of Sec. 4.
#include "internal.cuh"
#include "device_util.cuh"
#include "level_math.cuh"
#include "sweep_parts.cuh"

namespace cav {

constexpr int RES_BX = 32, RES_BY = 8, RES_WARPS = RES_BX * RES_BY / 32;

// Residual (mode 0: out = b - K_E w, b may be null) or product (mode 1: out = K_E w) in one
// launch with two block roles (residual_block: cell tiles, then E_E rows).
__global__ void __launch_bounds__(RES_BX* RES_BY) k_residual(ResArgs a) {
  pdl_wait();  // programmatic launch: the kernel ahead (which writes w or b) has finished
  pdl_trigger();
  residual_block<RES_WARPS>(a, (int)blockIdx.x, (int)threadIdx.x);
}

ResArgs residual_args(const LevelOps& op, const double* w, const double* b, double* out, int mode, int warps) {
  ResArgs a;
  a.N = op.N;
  a.h = op.h;
  a.rho_dt = op.rho_dt;
  a.mu = op.mu;
  a.dt = op.dt;
  a.sc.ih = 1.0 / op.h;
  a.sc.ih2 = 1.0 / (op.h * op.h);
  a.sc.tmu_h = 2.0 * op.mu / op.h;
  a.sc.cdiag = op.rho_dt + 4.0 * op.mu * a.sc.ih2;
  a.sc.cnb = -op.mu * a.sc.ih2;
  a.w = w;
  a.b = b;
  a.out = out;
  a.out32 = nullptr;
  a.mode = mode;
  a.gx = div_up(op.N, 32);
  a.nb_cells = a.gx * div_up(op.N, warps);
  const bool has_ee = op.ee && op.ee->n_rows > 0;
  a.row_of = has_ee ? op.ee->row_of : nullptr;
  a.n_rows = has_ee ? op.ee->n_rows : 0;
  a.rows = has_ee ? op.ee->rows : nullptr;
  a.rowptr = has_ee ? op.ee->rowptr : nullptr;
  a.cols = has_ee ? op.ee->cols : nullptr;
  a.vals = has_ee ? op.ee->vals : nullptr;
  a.channel = op.channel;
  return a;
}

int residual_blocks(const ResArgs& a, int warps) { return a.nb_cells + div_up(a.n_rows, warps * ROWS_PER_WARP); }

void launch_apply(const LevelOps& op, const double* w, const double* b, double* out, int mode,
                  cudaStream_t st, bool pdl, float* out32) {
  ResArgs a = residual_args(op, w, b, out, mode, RES_WARPS);
  a.out32 = out32;
  launch_k(k_residual, dim3(residual_blocks(a, RES_WARPS)), dim3(RES_BX * RES_BY), 0, st, pdl, a);
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
