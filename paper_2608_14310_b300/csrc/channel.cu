// The channel time step of the flow-past-a-fiber benchmark (Sec. 5.3), the pieces that are
// not the linear solve:
//
//   * the step's base right-hand side  b = [ (rho/dt) u^n - rho N[u^n] ; 0 ] + g,
//     N[u] = (u . grad) u the explicit convective term (centred differences, each velocity
//     component averaged from its four neighbours onto the other's faces), g the boundary
//     vector of the inflow v = -U(t^{n+1}) on the top wall and of the traction outflow, whose
//     backflow term (rho/2) min(u.n, 0) u is taken at u^n (n = (0, -1));
//   * the right-hand side of one Newton system at the iterate w_k (Eqs. im_disc_mom,
//     im_disc_advec, Eul_schur, with the force at X_k = X^n + dt J^n u_k):
//         rhs_k = b + [ S^n F(X_k) - dt E_E(X_k) u_k ; 0 ],
//     E_E(X_k) = S^n E(X_k) J^n the system's E_E set up with X_lin = X_k; the linear system is
//     K_E(X_k) w = rhs_k, and K_E(X_k) w_k - rhs_k is the Newton residual at w_k;
//   * the 2-norm of a residual, for the Newton loop's stopping test.
//
// Ghost values (the same rules as the operator's, now with the boundary data):
//   u_{i,N} = 2 u_top - u_{i,N-1} (u_top = 0),  v_{i,N} = v_top,
//   u_{i,-1} = u_{i,0} + (v_{i,0} - v_{i-1,0}) + h t_x,i / mu,
//   v_{i,-1} = v_{i,0} + (u_{i+1,-1} - u_{i,-1}),
//   p_{i,-1} = 2 t_y,i + (2 mu / h)(v_{i,1} - v_{i,-1}) - p_{i,0},
// with t_x at the points (i h, 0) and t_y at ((i + 1/2) h, 0).  The constant parts of the
// rows they enter form g (moved to the right-hand side with the opposite sign):
//   u row (i, 0):      + t_x,i / h
//   v row (i, 0):      + (2 t_y,i - (t_x,i+1 - t_x,i)) / h
//   v row (i, N - 1):  + mu v_top / h^2
//   p row (i, N - 1):  + v_top / h
#include <cmath>
#include <string>

#include "internal.cuh"
#include "device_util.cuh"
#include "level_math.cuh"

namespace cav {

// Backflow traction at u^n: the boundary u extrapolated as (3 u_0 - u_1) / 2, v at (i h, 0)
// the mean of its two neighbours:  t_x,i = (rho/2) min(-vb, 0) ub,  t_y,i = (rho/2) min(-v_i0, 0) v_i0.
__device__ inline double backflow_tx(int N, double rho, const double* u, const double* v, int i) {
  const int im = (i == 0) ? N - 1 : i - 1;
  const double ub = 0.5 * (3.0 * u[i] - u[N + i]);
  const double vb = 0.5 * (v[i] + v[im]);
  return 0.5 * rho * fmin(-vb, 0.0) * ub;
}
__device__ inline double backflow_ty(double rho, const double* v, int i) {
  return 0.5 * rho * fmin(-v[i], 0.0) * v[i];
}

// One thread per cell (i, j): the rows u_ij, v_ij, p_ij of b.
__global__ void k_channel_rhs(int N, double h, double rho, double mu, double dt, double v_top_next,
                              double v_top_prev, const double* __restrict__ w, double* __restrict__ b) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int NN = N * N;
  if (c >= NN) return;
  const int i = c % N, j = c / N;
  const int ip = (i + 1 == N) ? 0 : i + 1, im = (i == 0) ? N - 1 : i - 1;
  const double* u = w;
  const double* v = w + NN;
  const double ih = 1.0 / h, i2h = 0.5 / h;
  const double tx_i = backflow_tx(N, rho, u, v, i), tx_ip = backflow_tx(N, rho, u, v, ip);
  // ghost rows of u^n for the convective term (u_top = 0, v_top = the previous step's inflow);
  // the row below the outflow is read at x = i and x = i + 1 only
  auto U = [&](int x, int y) -> double {
    if (y == N) return -u[(N - 1) * N + x];
    if (y == -1) {
      const int xm = (x == 0) ? N - 1 : x - 1;
      const double tx = (x == i) ? tx_i : tx_ip;
      return u[x] + (v[x] - v[xm]) + h * tx / mu;
    }
    return u[y * N + x];
  };
  auto Vv = [&](int x, int y) -> double {
    if (y == N) return v_top_prev;
    if (y == -1) {
      const int xp = (x + 1 == N) ? 0 : x + 1;
      return v[x] + (U(xp, -1) - U(x, -1));
    }
    return v[y * N + x];
  };
  // u face (i, j): N_u = u du/dx + vbar du/dy
  const double uc = u[c], vc = v[c];
  const double dudx = (u[j * N + ip] - u[j * N + im]) * i2h;
  const double dudy = (U(i, j + 1) - U(i, j - 1)) * i2h;
  const double vbar = 0.25 * (Vv(i, j) + Vv(im, j) + Vv(i, j + 1) + Vv(im, j + 1));
  const double Nu = uc * dudx + vbar * dudy;
  // v face (i, j): N_v = ubar dv/dx + v dv/dy
  const double dvdx = (v[j * N + ip] - v[j * N + im]) * i2h;
  const double dvdy = (Vv(i, j + 1) - Vv(i, j - 1)) * i2h;
  const double ubar = 0.25 * (U(i, j) + U(ip, j) + U(i, j - 1) + U(ip, j - 1));
  const double Nv = ubar * dvdx + vc * dvdy;
  double bu = rho / dt * uc - rho * Nu;
  double bv = rho / dt * vc - rho * Nv;
  double bp = 0.0;
  // boundary vector of this step (inflow v_top_next, traction with the backflow term)
  if (j == 0) {
    bu += tx_i * ih;
    bv += (2.0 * backflow_ty(rho, v, i) - (tx_ip - tx_i)) * ih;
  }
  if (j + 1 == N) {
    bv += mu * v_top_next * ih * ih;
    bp += v_top_next * ih;
  }
  b[c] = bu;
  b[NN + c] = bv;
  b[2 * NN + c] = bp;
}

// rhs = b_base + [S F - dt E_E w ; 0]: spread force already in f (velocity rows); one thread
// per velocity row adds b_base and, on E_E's rows, -dt sum_l E_E[row, l] w_l (fixed order);
// the pressure rows copy b_base.
// (f and rhs may be the same buffer: each thread reads f[k] before writing rhs[k])
__global__ void k_newton_rhs(int N, double dt, const double* __restrict__ b_base, const double* __restrict__ w,
                             const double* f, const int* __restrict__ row_of,
                             const int64_t* __restrict__ rowptr, const int* __restrict__ cols,
                             const double* __restrict__ vals, double* rhs) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int NN = N * N;
  if (k >= 3 * NN) return;
  if (k >= 2 * NN) {
    rhs[k] = b_base[k];
    return;
  }
  double s = 0.0;
  const int r = row_of ? row_of[k] : -1;
  if (r >= 0)
    for (int64_t q = rowptr[r]; q < rowptr[r + 1]; ++q) s += vals[q] * w[cols[q]];
  rhs[k] = (b_base[k] + f[k]) - dt * s;
}

}  // namespace cav

using namespace cav;

extern "C" {

ib_status ib_channel_rhs(const ib_system* s, const double* w_n, double U_next, double U_prev, double* b,
                         cudaStream_t st) {
  try {
    CAV_REQUIRE(s && w_n && b, "ib_channel_rhs: NULL argument");
    CAV_REQUIRE(s->bc == IB_BC_CHANNEL, "ib_channel_rhs: the system is not a channel (IB_BC_CHANNEL)");
    CAV_REQUIRE(w_n != b, "ib_channel_rhs: w_n and b must not alias");
    const int NN = s->N * s->N;
    k_channel_rhs<<<div_up(NN, 256), 256, 0, st>>>(s->N, s->h, s->rho, s->mu, s->dt, -U_next, -U_prev, w_n, b);
    CAV_CHECK_LAUNCH();
    return IB_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

ib_status ib_newton_rhs(const ib_system* s, const double* b_base, const double* w, double* rhs, cudaStream_t st) {
  try {
    CAV_REQUIRE(s && b_base && w && rhs, "ib_newton_rhs: NULL argument");
    CAV_REQUIRE(rhs != b_base && rhs != w, "ib_newton_rhs: rhs must not alias b_base or w");
    const int NN = s->N * s->N;
    // rhs = S F(X_lin) on the velocity rows (the spread leaves the pressure rows alone; the
    // kernel below writes them)
    ib_force_launch(s, s->F, st);
    ib_spread_launch(s, s->F, rhs, 0, nullptr, nullptr, st);
    const bool has_ee = s->ee.n_rows > 0;
    k_newton_rhs<<<div_up(3 * NN, 256), 256, 0, st>>>(s->N, s->dt, b_base, w, rhs, has_ee ? s->ee.row_of : nullptr,
                                                     s->ee.rowptr, s->ee.cols, s->ee.vals, rhs);
    CAV_CHECK_LAUNCH();
    return IB_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

ib_status ib_residual_norm(const ib_system* s, const double* b, const double* x, double* r, double* norm,
                           cudaStream_t st) {
  try {
    CAV_REQUIRE(s && b && x && r && norm, "ib_residual_norm: NULL argument");
    const int64_t n = 3LL * s->N * s->N;
    LevelOps o{s->N, s->h, s->rho / s->dt, s->mu, s->dt, &s->ee, s->bc == IB_BC_CHANNEL};
    launch_apply(o, x, b, r, 0, st);
    *norm = std::sqrt(device_dot(r, r, n, s->partial, st));
    return IB_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

}  // extern "C"
