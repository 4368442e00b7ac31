// Per-cell and per-row arithmetic of one multigrid level (the Stokes rows of K_E, the E_E
// row sums, the grid transfers, the standard Vanka patch and the patch-inverse loads), kept
// in one place so that every kernel evaluating them does so with the same expressions.

#pragma once
#include <cuda_bf16.h>

namespace cav {

// ------------------------------------------------------------------ Stokes rows of K_E

// Rows of the Stokes part of K_E w (Eq. Eul_schur) at cell (i, j):
//   u: (rho/dt) u - mu L u + (p_ij - p_i-1j)/h,  v: likewise,  p: -(D u)_ij.
struct StokesRows {
  double ku, kv, kp;
};
__device__ inline StokesRows stokes_rows(int N, double h, double rho_dt, double mu, const double* w, int i, int j) {
  const int NN = N * N;
  const int ip = (i + 1 == N) ? 0 : i + 1, im = (i == 0) ? N - 1 : i - 1;
  const int jp = (j + 1 == N) ? 0 : j + 1, jm = (j == 0) ? N - 1 : j - 1;
  const double* u = w;
  const double* v = w + NN;
  const double* p = w + 2 * NN;
  const int c = j * N + i;
  const double ih = 1.0 / h, ih2 = 1.0 / (h * h);
  const double uc = u[c], vc = v[c], pc = p[c];
  const double uip = u[j * N + ip], vjp = v[jp * N + i];
  const double lu = (uip + u[j * N + im] + u[jp * N + i] + u[jm * N + i] - 4.0 * uc) * ih2;
  const double lv = (v[j * N + ip] + v[j * N + im] + vjp + v[jm * N + i] - 4.0 * vc) * ih2;
  StokesRows o;
  o.ku = rho_dt * uc - mu * lu + (pc - p[j * N + im]) * ih;
  o.kv = rho_dt * vc - mu * lv + (pc - p[jm * N + i]) * ih;
  o.kp = -((uip - uc) + (vjp - vc)) * ih;
  return o;
}

// E_E rows: 8 lanes per row, lane-strided over the row's entries, then a fixed xor tree.
constexpr int ROW_LANES = 8;
__device__ inline double ee_row_lane_sum(const int64_t* __restrict__ rowptr, const int* __restrict__ cols,
                                         const double* __restrict__ vals, const double* w, int r, int sl) {
  double s = 0.0;
  for (int64_t q = rowptr[r] + sl; q < rowptr[r + 1]; q += ROW_LANES) s += vals[q] * w[cols[q]];
  return s;
}
// all 32 lanes must call this
__device__ inline double row_group_reduce(double s) {
#pragma unroll
  for (int o = ROW_LANES / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// ------------------------------------------------------------------ grid transfers (Sec. 4)

// Restriction at coarse cell (I, J): velocity R = (1/4) P^T of RT0 prolongation, pressure
// the mean of the four fine cells.
__device__ inline void restrict_cell(int Nc, const double* rf, double* bc, int I, int J) {
  const int Nf = 2 * Nc, NNf = Nf * Nf, NNc = Nc * Nc;
  const double* u = rf;
  const double* v = rf + NNf;
  const double* p = rf + 2 * NNf;
  const int i0 = 2 * I, j0 = 2 * J;
  const int im = (i0 == 0) ? Nf - 1 : i0 - 1, jm = (j0 == 0) ? Nf - 1 : j0 - 1;
  const int i1 = i0 + 1, j1 = j0 + 1;
  // u faces: coincident (i0, j0), (i0, j1) weight 1; midline (i0 +- 1, j0/j1) weight 1/2
  const double ru = u[j0 * Nf + i0] + u[j1 * Nf + i0] +
                    0.5 * (u[j0 * Nf + i1] + u[j1 * Nf + i1]) +
                    0.5 * (u[j0 * Nf + im] + u[j1 * Nf + im]);
  const double rv = v[j0 * Nf + i0] + v[j0 * Nf + i1] +
                    0.5 * (v[j1 * Nf + i0] + v[j1 * Nf + i1]) +
                    0.5 * (v[jm * Nf + i0] + v[jm * Nf + i1]);
  const double rp = p[j0 * Nf + i0] + p[j0 * Nf + i1] + p[j1 * Nf + i0] +
                    p[j1 * Nf + i1];
  const int c = J * Nc + I;
  bc[c] = 0.25 * ru;
  bc[NNc + c] = 0.25 * rv;
  bc[2 * NNc + c] = 0.25 * rp;
}

// w_f += P x_c at fine cell (i, j): RT0 velocity interpolation and bilinear pressure
// interpolation between cell centres (9/16, 3/16, 3/16, 1/16).
__device__ inline void prolong_cell(int Nc, const double* xc, double* wf, int i, int j) {
  const int Nf = 2 * Nc;
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
  wf[c] = wf[c] + du;
  wf[NNf + c] = wf[NNf + c] + dv;
  wf[2 * NNf + c] = wf[2 * NNf + c] + dp;
}

// ------------------------------------------------------------------ patch inverses

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
  __device__ static void load_shared(const double* p, acc_t* out) {
    const double2 v = *reinterpret_cast<const double2*>(p);
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
  __device__ static void load_shared(const float* p, acc_t* out) {
    const float4 v = *reinterpret_cast<const float4*>(p);
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
  __device__ static void unpack(const uint4& v, acc_t* out) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 f = __bfloat1622float2(h[q]);
      out[2 * q] = f.x;
      out[2 * q + 1] = f.y;
    }
  }
  __device__ static void load(const __nv_bfloat16* p, acc_t* out) {
    unpack(__ldg(reinterpret_cast<const uint4*>(p)), out);
  }
  __device__ static void load_shared(const __nv_bfloat16* p, acc_t* out) {
    unpack(*reinterpret_cast<const uint4*>(p), out);
  }
};

// acc + x * y as one fused multiply-add, so every kernel variant accumulates a patch's
// columns in the same order with the same rounding (the autotuner's choice cannot change
// a result bit).
__device__ inline double mad(double x, double y, double acc) { return fma(x, y, acc); }
__device__ inline float mad(float x, float y, float acc) { return fmaf(x, y, acc); }

// ------------------------------------------------------------------ standard Vanka patch

struct StdInv {
  double m[25];
};

// canonical slots of cell (i, j)'s standard patch: u_ij, u_i+1j, v_ij, v_ij+1, p_ij
__device__ inline double std_row(const StdInv& S, int row, const double* r, int N, int i, int j) {
  const int NN = N * N;
  const int ip = (i + 1 == N) ? 0 : i + 1, jp = (j + 1 == N) ? 0 : j + 1;
  const double y0 = r[j * N + i], y1 = r[j * N + ip], y2 = r[NN + j * N + i],
               y3 = r[NN + jp * N + i], y4 = r[2 * NN + j * N + i];
  const double* m = S.m + 5 * row;
  return m[0] * y0 + m[1] * y1 + m[2] * y2 + m[3] * y3 + m[4] * y4;
}

constexpr int TOUCH_LANES = 8;                    // lanes per touched unknown
constexpr int TOUCH_PER_WARP = 32 / TOUCH_LANES;  // touched unknowns per warp

}  // namespace cav
