// Per-cell and per-row arithmetic of one multigrid level (the Stokes rows of K_E, the E_E
// row sums, the grid transfers, the standard Vanka patch and the patch-inverse loads), kept
// in one place so that every kernel evaluating them does so with the same expressions.

#pragma once
#include <cuda_bf16.h>

namespace cav {

// ------------------------------------------------------------------ Stokes rows of K_E

// Rows of the Stokes part of K_E w (Eq. Eul_schur) at cell (i, j):
//   u: (rho/dt) u - mu L u + (p_ij - p_i-1j)/h,  v: likewise,  p: -(D u)_ij.
// Periodic grid: every index wraps.  Channel (Sec. 5.3; periodic in x, prescribed inflow on
// the top wall y = L, traction outflow on y = 0): the same rows with homogeneous boundary
// data, values outside the unknowns taken from ghost values (the boundary data of a time
// step enter its right-hand side instead):
//   above the top row   u_{i,N} = -u_{i,N-1} (the wall value is the mean), v_{i,N} = 0;
//   below the bottom row, from the tangential traction, continuity in the ghost cell and the
//   normal traction:  u_{i,-1} = u_{i,0} + (v_{i,0} - v_{i-1,0}),
//                     v_{i,-1} = v_{i,0} + (u_{i+1,-1} - u_{i,-1}),
//                     p_{i,-1} = (2 mu / h)(v_{i,1} - v_{i,-1}) - p_{i,0}.
struct StokesRows {
  double ku, kv, kp;
};
// The coefficients of a level's Stokes rows, formed once on the host: on B300 every FP64 warp
// instruction holds its SM sub-partition for tens of cycles, and a division is a long sequence
// of them.  ih = 1 / h, ih2 = 1 / (h h), tmu_h = 2 mu / h; cdiag = rho/dt + 4 mu / h^2 and
// cnb = -mu / h^2, so a velocity row is cdiag u + cnb (its four neighbours' sum) + the pressure
// difference / h.
struct StokesCoef {
  double ih, ih2, tmu_h, cdiag, cnb;
};
// Each row alone (stokes_rows is the three together, with the same bits): the u row at face
// (i, j), the v row, and the p row.  A velocity row is evaluated in seven operations,
// cdiag u_c + cnb (sum of the four neighbours) + (p_c - p_w) / h, as the class step does.
__device__ inline double stokes_u_row(int N, const StokesCoef& sc, const double* w, int i, int j,
                                      bool channel = false) {
  const int NN = N * N;
  const int ip = (i + 1 == N) ? 0 : i + 1, im = (i == 0) ? N - 1 : i - 1;
  const int jp = (j + 1 == N) ? 0 : j + 1, jm = (j == 0) ? N - 1 : j - 1;
  const bool bot = channel && j == 0, top = channel && j + 1 == N;
  const double* u = w;
  const double* v = w + NN;
  const double* p = w + 2 * NN;
  const int c = j * N + i;
  const double uc = u[c], pc = p[c];
  const double uip = u[j * N + ip];
  const double u_up = top ? -uc : u[jp * N + i];
  const double u_dn = bot ? uc + (v[c] - v[j * N + im]) : u[jm * N + i];  // u_{i,-1} on the channel
  const double nb = (uip + u[j * N + im]) + (u_up + u_dn);
  return fma(sc.ih, pc - p[j * N + im], fma(sc.cnb, nb, sc.cdiag * uc));
}
__device__ inline double stokes_v_row(int N, const StokesCoef& sc, const double* w, int i, int j,
                                      bool channel = false) {
  const int NN = N * N;
  const int ip = (i + 1 == N) ? 0 : i + 1, im = (i == 0) ? N - 1 : i - 1;
  const int jp = (j + 1 == N) ? 0 : j + 1, jm = (j == 0) ? N - 1 : j - 1;
  const bool bot = channel && j == 0, top = channel && j + 1 == N;
  const double* u = w;
  const double* v = w + NN;
  const double* p = w + 2 * NN;
  const int c = j * N + i;
  const double vc = v[c], pc = p[c];
  const double vjp = top ? 0.0 : v[jp * N + i];
  double v_dn, p_dn;
  if (bot) {
    const double uc = u[c], uip = u[j * N + ip];
    const double gu = uc + (vc - v[j * N + im]);              // u_{i,-1}
    const double gu_ip = uip + (v[j * N + ip] - vc);          // u_{i+1,-1}
    v_dn = vc + (gu_ip - gu);                                 // v_{i,-1}
    p_dn = sc.tmu_h * (v[jp * N + i] - v_dn) - pc;            // p_{i,-1}
  } else {
    v_dn = v[jm * N + i];
    p_dn = p[jm * N + i];
  }
  const double nb = (v[j * N + ip] + v[j * N + im]) + (vjp + v_dn);
  return fma(sc.ih, pc - p_dn, fma(sc.cnb, nb, sc.cdiag * vc));
}
__device__ inline double stokes_p_row(int N, const StokesCoef& sc, const double* w, int i, int j,
                                      bool channel = false) {
  const int NN = N * N;
  const int ip = (i + 1 == N) ? 0 : i + 1, jp = (j + 1 == N) ? 0 : j + 1;
  const bool top = channel && j + 1 == N;
  const double* u = w;
  const double* v = w + NN;
  const int c = j * N + i;
  const double uc = u[c], vc = v[c];
  const double uip = u[j * N + ip];
  const double vjp = top ? 0.0 : v[jp * N + i];
  return -((uip - uc) + (vjp - vc)) * sc.ih;
}
__device__ inline StokesRows stokes_rows(int N, const StokesCoef& sc, const double* w, int i, int j,
                                         bool channel = false) {
  StokesRows o;
  o.ku = stokes_u_row(N, sc, w, i, j, channel);
  o.kv = stokes_v_row(N, sc, w, i, j, channel);
  o.kp = stokes_p_row(N, sc, w, i, j, channel);
  return o;
}

// E_E rows: 8 lanes per row, lane-strided over the row's entries, then a fixed xor tree.  A
// lane takes its entries in batches of LOAD_BATCH: every column index of the batch is loaded,
// then every iterate value, then the multiply-adds in entry order, so a row costs two
// dependent load latencies per batch instead of two per entry.
constexpr int ROW_LANES = 8;
constexpr int LOAD_BATCH = 8;
__device__ inline double ee_row_lane_sum(const int64_t* __restrict__ rowptr, const int* __restrict__ cols,
                                         const double* __restrict__ vals, const double* w, int r, int sl) {
  const int64_t q1 = rowptr[r + 1];
  double s = 0.0;
  for (int64_t qb = rowptr[r] + sl; qb < q1; qb += ROW_LANES * LOAD_BATCH) {
    int c[LOAD_BATCH];
    double v[LOAD_BATCH], x[LOAD_BATCH];
#pragma unroll
    for (int u = 0; u < LOAD_BATCH; ++u) {
      const int64_t q = qb + (int64_t)u * ROW_LANES;
      c[u] = (q < q1) ? cols[q] : -1;
      v[u] = (q < q1) ? vals[q] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < LOAD_BATCH; ++u) x[u] = (c[u] >= 0) ? w[c[u]] : 0.0;
#pragma unroll
    for (int u = 0; u < LOAD_BATCH; ++u)
      if (c[u] >= 0) s = fma(v[u], x[u], s);
  }
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
// Channel: the fine v faces below coarse row J = 0 do not exist (the transpose of the
// channel prolongation below).
__device__ inline void restrict_cell(int Nc, const double* rf, double* bc, int I, int J, bool channel = false) {
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
                    ((channel && J == 0) ? 0.0 : 0.5 * (v[jm * Nf + i0] + v[jm * Nf + i1]));
  const double rp = p[j0 * Nf + i0] + p[j0 * Nf + i1] + p[j1 * Nf + i0] +
                    p[j1 * Nf + i1];
  const int c = J * Nc + I;
  bc[c] = 0.25 * ru;
  bc[NNc + c] = 0.25 * rv;
  bc[2 * NNc + c] = 0.25 * rp;
}

// w_f += P x_c at fine cell (i, j): RT0 velocity interpolation and bilinear pressure
// interpolation between cell centres (9/16, 3/16, 3/16, 1/16).  Channel: a fine v face on
// the midline of a top-row coarse cell takes half the coarse face below it (the prescribed
// top faces carry no correction), and the pressure stencil is clamped to the boundary cells
// in y.
__device__ inline void prolong_cell(int Nc, const double* xc, double* wf, int i, int j, bool channel = false) {
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
  else if (channel && J + 1 == Nc) dv = 0.5 * V[J * Nc + I];
  else dv = 0.5 * (V[J * Nc + I] + V[Jp * Nc + I]);
  int Js = (j & 1) ? Jp : Jm;
  if (channel) Js = (j & 1) ? min(J + 1, Nc - 1) : max(J - 1, 0);
  const int Is = (i & 1) ? Ip : Im;
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

// Inverse(s) of the standard Vanka patch in canonical slot order (u_ij, u_i+1j, v_ij,
// v_ij+1, p_ij), scalings folded in.  Periodic grid: one matrix (all cells alike).  Channel:
// kind 0 interior rows, kind 1 the outflow row j = 0, kind 2 the inflow row j = N - 1, whose
// patch has no v_{i,N} (slot 3: zero row and column).
struct StdInv {
  double m[3][25];
};
__device__ inline int std_kind(int N, int j, bool channel) {
  return !channel ? 0 : (j == 0 ? 1 : (j + 1 == N ? 2 : 0));
}

__device__ inline double std_row(const StdInv& S, int row, const double* r, int N, int i, int j,
                                 bool channel = false) {
  const int NN = N * N;
  const int ip = (i + 1 == N) ? 0 : i + 1, jp = (j + 1 == N) ? 0 : j + 1;
  const int kind = std_kind(N, j, channel);
  const double y0 = r[j * N + i], y1 = r[j * N + ip], y2 = r[NN + j * N + i],
               y3 = (kind == 2) ? 0.0 : r[NN + jp * N + i], y4 = r[2 * NN + j * N + i];
  const double* m = S.m[kind] + 5 * row;
  return m[0] * y0 + m[1] * y1 + m[2] * y2 + m[3] * y3 + m[4] * y4;
}

// The same inverse rounded to FP32, applied to the FP32 copy of the residual on levels whose
// patch inverses are stored in FP32 or BF16 (there every patch inverse is applied in FP32).
struct StdInv32 {
  float m[3][25];
};
__device__ inline float std_row32(const StdInv32& S, int row, const float* r, int N, int i, int j,
                                  bool channel = false) {
  const int NN = N * N;
  const int ip = (i + 1 == N) ? 0 : i + 1, jp = (j + 1 == N) ? 0 : j + 1;
  const int kind = std_kind(N, j, channel);
  const float y0 = r[j * N + i], y1 = r[j * N + ip], y2 = r[NN + j * N + i],
              y3 = (kind == 2) ? 0.f : r[NN + jp * N + i], y4 = r[2 * NN + j * N + i];
  const float* m = S.m[kind] + 5 * row;
  return m[0] * y0 + m[1] * y1 + m[2] * y2 + m[3] * y3 + m[4] * y4;
}

constexpr int TOUCH_LANES = 4;                    // lanes per touched unknown
constexpr int TOUCH_PER_WARP = 32 / TOUCH_LANES;  // touched unknowns per warp

// The standard patches (cells that kept their Vanka patch) holding unknown k, in the order
// the scatter adds their corrections: cell (i0, j0), then (i1, j1), and the row of the shared
// 5 x 5 inverse that gives each one's correction at k.  On the channel a v face of the
// outflow row has only the cell above it.  (Scalar fields: an array here would be indexed at
// run time and live in local memory.)
struct StdHolders {
  int n;
  int i0, j0, row0, i1, j1, row1;
};
__device__ inline StdHolders std_holders(int N, const uint8_t* cell_big, bool channel, int k) {
  const int NN = N * N;
  const int comp = k / NN, c = k % NN, i = c % N, j = c / N;
  const int im = (i == 0) ? N - 1 : i - 1, jm = (j == 0) ? N - 1 : j - 1;
  StdHolders h;
  h.n = 0;
  h.i0 = h.j0 = h.row0 = h.i1 = h.j1 = h.row1 = 0;
  auto add = [&](int ci, int cj, int row) {
    if (h.n == 0) {
      h.i0 = ci;
      h.j0 = cj;
      h.row0 = row;
    } else {
      h.i1 = ci;
      h.j1 = cj;
      h.row1 = row;
    }
    ++h.n;
  };
  if (comp == 0) {
    if (!cell_big[j * N + im]) add(im, j, 1);
    if (!cell_big[c]) add(i, j, 0);
  } else if (comp == 1) {
    if (!(channel && j == 0) && !cell_big[jm * N + i]) add(i, jm, 3);
    if (!cell_big[c]) add(i, j, 2);
  } else {
    if (!cell_big[c]) add(i, j, 4);
  }
  return h;
}

// One lane's share of the corrections at a touched unknown: delta[inc_slot[q]] for q = q0 + sl,
// q0 + sl + TOUCH_LANES, ... below q1, summed in that order, the slot indices and then the
// corrections of each batch of LOAD_BATCH loaded before the additions.
__device__ inline double touched_lane_sum(const int* __restrict__ inc_slot, const double* delta, int64_t q0,
                                          int64_t q1, int sl) {
  double s = 0.0;
  for (int64_t qb = q0 + sl; qb < q1; qb += TOUCH_LANES * LOAD_BATCH) {
    int id[LOAD_BATCH];
    double d[LOAD_BATCH];
#pragma unroll
    for (int u = 0; u < LOAD_BATCH; ++u) {
      const int64_t q = qb + (int64_t)u * TOUCH_LANES;
      id[u] = (q < q1) ? inc_slot[q] : -1;
    }
#pragma unroll
    for (int u = 0; u < LOAD_BATCH; ++u) d[u] = (id[u] >= 0) ? delta[id[u]] : 0.0;
#pragma unroll
    for (int u = 0; u < LOAD_BATCH; ++u)
      if (id[u] >= 0) s += d[u];
  }
  return s;
}

}  // namespace cav
