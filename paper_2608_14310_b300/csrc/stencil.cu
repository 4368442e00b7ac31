// Stokes stencils of K_E, the E_E product, and the grid transfers of Sec. 4.
#include "internal.cuh"
#include "device_util.cuh"

namespace cav {

// Rows of the Stokes part of K_E w (Eq. Eul_schur) at cell (i, j):
//   u: (rho/dt) u - mu L u + (p_ij - p_i-1j)/h,  v: likewise,  p: -(D u)_ij.
struct StokesRows {
  double ku, kv, kp;
};
__device__ inline StokesRows stokes_rows(int N, double h, double rho_dt, double mu, const double* __restrict__ w,
                                         int i, int j) {
  const int NN = N * N;
  const int ip = (i + 1 == N) ? 0 : i + 1, im = (i == 0) ? N - 1 : i - 1;
  const int jp = (j + 1 == N) ? 0 : j + 1, jm = (j == 0) ? N - 1 : j - 1;
  const double* u = w;
  const double* v = w + NN;
  const double* p = w + 2 * NN;
  const int c = j * N + i;
  const double ih = 1.0 / h, ih2 = 1.0 / (h * h);
  const double uc = u[c], vc = v[c], pc = p[c];
  const double lu = (u[j * N + ip] + u[j * N + im] + u[jp * N + i] + u[jm * N + i] - 4.0 * uc) * ih2;
  const double lv = (v[j * N + ip] + v[j * N + im] + v[jp * N + i] + v[jm * N + i] - 4.0 * vc) * ih2;
  StokesRows o;
  o.ku = rho_dt * uc - mu * lu + (pc - p[j * N + im]) * ih;
  o.kv = rho_dt * vc - mu * lv + (pc - p[jm * N + i]) * ih;
  o.kp = -((u[j * N + ip] - uc) + (v[jp * N + i] - vc)) * ih;
  return o;
}

constexpr int RES_BX = 32, RES_BY = 8, RES_WARPS = RES_BX * RES_BY / 32;

// Residual (mode 0: out = b - K_E w, b may be null) or product (mode 1: out = K_E w) in one
// launch with two block roles.  Blocks [0, nb_cells) take a 32 x 8 tile of cells, one thread
// per cell, and write every row there except the velocity rows E_E touches; the remaining
// blocks take those rows one warp each and write the Stokes part plus
// -dt sum_l E_E[row, l] w[l] (fixed lane-strided order, fixed shuffle tree).
__global__ void __launch_bounds__(RES_BX* RES_BY)
k_residual(int N, double h, double rho_dt, double mu, double dt, const double* __restrict__ w,
           const double* __restrict__ b, double* __restrict__ out, int mode, int nb_cells, int gx,
           const int* __restrict__ row_of, int n_rows, const int* __restrict__ rows,
           const int64_t* __restrict__ rowptr, const int* __restrict__ cols, const double* __restrict__ vals) {
  const int NN = N * N;
  if ((int)blockIdx.x < nb_cells) {
    const int i = (blockIdx.x % gx) * RES_BX + (threadIdx.x % RES_BX);
    const int j = (blockIdx.x / gx) * RES_BY + (threadIdx.x / RES_BX);
    if (i >= N || j >= N) return;
    const int c = j * N + i;
    const StokesRows k = stokes_rows(N, h, rho_dt, mu, w, i, j);
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
  const int r = ((int)blockIdx.x - nb_cells) * RES_WARPS + warp;
  if (r >= n_rows) return;
  double s = 0.0;
  for (int64_t q = rowptr[r] + lane; q < rowptr[r + 1]; q += 32) s += vals[q] * w[cols[q]];
  s = warp_sum(s);
  if (lane == 0) {
    const int row = rows[r];
    const int comp = row / NN, c = row % NN;
    const StokesRows k = stokes_rows(N, h, rho_dt, mu, w, c % N, c / N);
    const double kr = ((comp == 0) ? k.ku : k.kv) - dt * s;
    out[row] = (mode == 0) ? ((b ? b[row] : 0.0) - kr) : kr;
  }
}

void launch_apply(const LevelOps& op, const double* w, const double* b, double* out, int mode,
                  cudaStream_t st) {
  const int gx = div_up(op.N, RES_BX), gy = div_up(op.N, RES_BY);
  const int nb_cells = gx * gy;
  const bool has_ee = op.ee && op.ee->n_rows > 0;
  const int nb_rows = has_ee ? div_up(op.ee->n_rows, RES_WARPS) : 0;
  k_residual<<<nb_cells + nb_rows, RES_BX * RES_BY, 0, st>>>(
      op.N, op.h, op.rho_dt, op.mu, op.dt, w, b, out, mode, nb_cells, gx, has_ee ? op.ee->row_of : nullptr,
      has_ee ? op.ee->n_rows : 0, has_ee ? op.ee->rows : nullptr, has_ee ? op.ee->rowptr : nullptr,
      has_ee ? op.ee->cols : nullptr, has_ee ? op.ee->vals : nullptr);
  CAV_CHECK_LAUNCH();
}

// Restriction (Sec. 4), one thread per coarse cell (I, J):
//   velocity R = (1/4) P^T of RT0 prolongation, pressure = mean of the four fine cells.
__global__ void k_restrict(int Nc, const double* __restrict__ rf, double* __restrict__ bc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= Nc || J >= Nc) return;
  const int Nf = 2 * Nc, NNf = Nf * Nf, NNc = Nc * Nc;
  const double* u = rf;
  const double* v = rf + NNf;
  const double* p = rf + 2 * NNf;
  const int i0 = 2 * I, j0 = 2 * J;
  const int im = (i0 == 0) ? Nf - 1 : i0 - 1, jm = (j0 == 0) ? Nf - 1 : j0 - 1;
  const int i1 = i0 + 1, j1 = j0 + 1;
  // u faces: coincident (i0, j0), (i0, j1) weight 1; midline (i0 +- 1, j0/j1) weight 1/2
  const double ru = u[j0 * Nf + i0] + u[j1 * Nf + i0] +
                    0.5 * (u[j0 * Nf + i1] + u[j1 * Nf + i1]) + 0.5 * (u[j0 * Nf + im] + u[j1 * Nf + im]);
  const double rv = v[j0 * Nf + i0] + v[j0 * Nf + i1] +
                    0.5 * (v[j1 * Nf + i0] + v[j1 * Nf + i1]) + 0.5 * (v[jm * Nf + i0] + v[jm * Nf + i1]);
  const double rp = p[j0 * Nf + i0] + p[j0 * Nf + i1] + p[j1 * Nf + i0] + p[j1 * Nf + i1];
  const int c = J * Nc + I;
  bc[c] = 0.25 * ru;
  bc[NNc + c] = 0.25 * rv;
  bc[2 * NNc + c] = 0.25 * rp;
}

// w_f += P x_c (Sec. 4), one thread per fine cell (i, j): RT0 velocity interpolation and
// bilinear pressure interpolation between cell centres (9/16, 3/16, 3/16, 1/16).
__global__ void k_prolong_add(int Nc, const double* __restrict__ xc, double* __restrict__ wf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int Nf = 2 * Nc;
  if (i >= Nf || j >= Nf) return;
  const int NNf = Nf * Nf, NNc = Nc * Nc;
  const double* U = xc;
  const double* V = xc + NNc;
  const double* P = xc + 2 * NNc;
  const int I = i >> 1, J = j >> 1;
  const int Ip = (I + 1 == Nc) ? 0 : I + 1, Jp = (J + 1 == Nc) ? 0 : J + 1;
  const int Im = (I == 0) ? Nc - 1 : I - 1, Jm = (J == 0) ? Nc - 1 : J - 1;
  double du, dv;
  if ((i & 1) == 0) du = U[J * Nc + I];
  else du = 0.5 * (U[J * Nc + I] + U[J * Nc + Ip]);
  if ((j & 1) == 0) dv = V[J * Nc + I];
  else dv = 0.5 * (V[J * Nc + I] + V[Jp * Nc + I]);
  const int Is = (i & 1) ? Ip : Im, Js = (j & 1) ? Jp : Jm;
  const double dp = (9.0 / 16.0) * P[J * Nc + I] + (3.0 / 16.0) * P[J * Nc + Is] +
                    (3.0 / 16.0) * P[Js * Nc + I] + (1.0 / 16.0) * P[Js * Nc + Is];
  const int c = j * Nf + i;
  wf[c] += du;
  wf[NNf + c] += dv;
  wf[2 * NNf + c] += dp;
}

void launch_restrict(int Nc, const double* r_f, double* b_c, cudaStream_t st) {
  dim3 blk(32, 8), grd(div_up(Nc, 32), div_up(Nc, 8));
  k_restrict<<<grd, blk, 0, st>>>(Nc, r_f, b_c);
  CAV_CHECK_LAUNCH();
}

void launch_prolong_add(int Nc, const double* x_c, double* w_f, cudaStream_t st) {
  dim3 blk(32, 8), grd(div_up(2 * Nc, 32), div_up(2 * Nc, 8));
  k_prolong_add<<<grd, blk, 0, st>>>(Nc, x_c, w_f);
  CAV_CHECK_LAUNCH();
}

}  // namespace cav
