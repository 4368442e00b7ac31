// Hierarchy set-up (Sec. 3.2, 3.3, 4): Galerkin E_E on coarse levels, CAV (or box) patch
// sets, extraction of local matrices, one-pass equilibration, inverses, and the transpose
// incidence used by the scatter of the additive sweep.
#include <algorithm>
#include <cstdlib>
#include <numeric>

#include <cooperative_groups.h>

#include "internal.cuh"
#include "device_util.cuh"
#include "grid_sync.cuh"

namespace cav {

// ------------------------------------------------------------------ Galerkin E_E

// Fine faces k with P[k, K] != 0 for coarse face K = (c, I, J) and their weights
// (RT0: coincident faces weight 1, faces on the coarse cell's midlines weight 1/2); returns
// their count.  Channel: a coarse v face of the outflow row J = 0 has no fine faces below it.
__device__ inline int pcol(int c, int I, int J, int Nf, int* fi, int* fj, double* wt, bool channel = false) {
  if (c == 0) {
    const int i0 = 2 * I, j0 = 2 * J;
    fi[0] = i0; fj[0] = j0; wt[0] = 1.0;
    fi[1] = i0; fj[1] = j0 + 1; wt[1] = 1.0;
    fi[2] = i0 - 1; fj[2] = j0; wt[2] = 0.5;
    fi[3] = i0 - 1; fj[3] = j0 + 1; wt[3] = 0.5;
    fi[4] = i0 + 1; fj[4] = j0; wt[4] = 0.5;
    fi[5] = i0 + 1; fj[5] = j0 + 1; wt[5] = 0.5;
  } else {
    const int i0 = 2 * I, j0 = 2 * J;
    fi[0] = i0; fj[0] = j0; wt[0] = 1.0;
    fi[1] = i0 + 1; fj[1] = j0; wt[1] = 1.0;
    fi[2] = i0; fj[2] = j0 - 1; wt[2] = 0.5;
    fi[3] = i0 + 1; fj[3] = j0 - 1; wt[3] = 0.5;
    fi[4] = i0; fj[4] = j0 + 1; wt[4] = 0.5;
    fi[5] = i0 + 1; fj[5] = j0 + 1; wt[5] = 0.5;
  }
  int n = 6;
  if (channel && c == 1 && J == 0) {  // drop entries 2 and 3 (fine row -1)
    fi[2] = fi[4]; fj[2] = fj[4]; wt[2] = wt[4];
    fi[3] = fi[5]; fj[3] = fj[5]; wt[3] = wt[5];
    n = 4;
  }
  for (int t = 0; t < n; ++t) {
    fi[t] = pmod(fi[t], Nf);
    fj[t] = pmod(fj[t], Nf);
  }
  return n;
}

__global__ void k_coarse_active(int Nc, const int* __restrict__ row_of_f, int* flag, bool channel) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  const int NNc = Nc * Nc;
  if (K >= 2 * NNc) return;
  const int c = K / NNc, rem = K % NNc, I = rem % Nc, J = rem / Nc;
  const int Nf = 2 * Nc;
  int fi[6], fj[6];
  double wt[6];
  const int nt = pcol(c, I, J, Nf, fi, fj, wt, channel);
  int f = 0;
  for (int t = 0; t < nt; ++t) f |= (row_of_f[c * Nf * Nf + fj[t] * Nf + fi[t]] >= 0);
  flag[K] = f;
}

__device__ inline int find_col(const int* cols, int64_t b, int64_t e, int key) {
  // binary search in the sorted column list [b, e); returns position or -1
  int64_t lo = b, hi = e;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    const int v = cols[mid];
    if (v < key) lo = mid + 1;
    else hi = mid;
  }
  return (lo < e && cols[lo] == key) ? (int)(lo - b) : -1;
}

// One warp per active coarse row K; lanes walk the window of coarse columns L (same
// component; with CROSS, the u plane and then the v plane, for an E_E whose rows reach the
// other component) in ascending global order and evaluate
//   E_c[K, L] = sum_{k in Pcol(K)} sum_{l in Pcol(L)} (1/4) P[k,K] E_f[k,l] P[l,L]
// in a fixed order; (K, L) is structurally nonzero iff some (k, l) is in E_f's pattern.
template <bool CROSS>
__global__ void k_galerkin(int Nc, int Wc, int n_rows, const int* __restrict__ rows,
                           const int* __restrict__ row_of_f, const int64_t* __restrict__ rowptr_f,
                           const int* __restrict__ cols_f, const double* __restrict__ vals_f,
                           int* row_count, const int64_t* __restrict__ rowptr, int* cols, double* vals,
                           int pass, bool channel) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= n_rows) return;
  const int NNc = Nc * Nc, Nf = 2 * Nc, NNf = Nf * Nf;
  const int K = rows[r];
  const int c = K / NNc, rem = K % NNc, I = rem % Nc, J = rem / Nc;
  int ki[6], kj[6];
  double kw[6];
  const int nk = pcol(c, I, J, Nf, ki, kj, kw, channel);
  int krow[6];
  for (int t = 0; t < 6; ++t) krow[t] = (t < nk) ? row_of_f[c * NNf + kj[t] * Nf + ki[t]] : -1;
  const Win wx = make_win(I, Wc, Nc), wy = make_win(J, Wc, Nc);
  const int ncell = wx.len * wy.len;
  int64_t outpos = (pass == 1) ? rowptr[r] : 0;
  int total = 0;
  for (int pl = 0; pl < (CROSS ? 2 : 1); ++pl) {
    const int cl = CROSS ? pl : c;  // component of the columns
    for (int base = 0; base < ncell; base += 32) {
      const int tp = base + lane;
      bool f = false;
      double val = 0.0;
      int L = 0;
      if (tp < ncell) {
        const int typ = tp / wx.len, txp = tp % wx.len;
        const int gy = win_glob(wy, win_asc(wy, typ), Nc), gx = win_glob(wx, win_asc(wx, txp), Nc);
        L = cl * NNc + gy * Nc + gx;
        int li[6], lj[6];
        double lw[6];
        const int nl = pcol(cl, gx, gy, Nf, li, lj, lw, channel);
        for (int t = 0; t < 6; ++t) {
          if (krow[t] < 0) continue;
          const int64_t b = rowptr_f[krow[t]], e = rowptr_f[krow[t] + 1];
          double s = 0.0;
          for (int u = 0; u < nl; ++u) {
            const int l = cl * NNf + lj[u] * Nf + li[u];
            const int pos = find_col(cols_f, b, e, l);
            if (pos >= 0) {
              f = true;
              s += vals_f[b + pos] * lw[u];
            }
          }
          val += 0.25 * kw[t] * s;
        }
      }
      const unsigned bal = __ballot_sync(0xffffffffu, f);
      if (pass == 1 && f) {
        const int rank = __popc(bal & ((1u << lane) - 1u));
        cols[outpos + total + rank] = L;
        vals[outpos + total + rank] = val;
      }
      total += __popc(bal);
    }
  }
  if (pass == 0 && lane == 0) row_count[r] = total;
}

__global__ void k_compact_rows2(int n, const int* flag, const int64_t* pos, int* rows, int* row_of) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n) return;
  if (flag[f]) {
    rows[pos[f]] = f;
    row_of[f] = (int)pos[f];
  } else {
    row_of[f] = -1;
  }
}

static void galerkin_level(const EECsr& fine, int Nc, EECsr& out, Arena& A, int* d_scratch, bool channel,
                           cudaStream_t st) {
  Arena scratch;
  const int NNc = Nc * Nc;
  int* flag = scratch.alloc<int>(2 * NNc);
  int64_t* pos = scratch.alloc<int64_t>(2 * NNc + 1);
  out.row_of = A.alloc<int>(2 * NNc);
  k_coarse_active<<<div_up(2 * NNc, 256), 256, 0, st>>>(Nc, fine.row_of, flag, channel);
  CAV_CHECK_LAUNCH();
  exclusive_scan(flag, pos, 2 * NNc, st, &scratch);
  int64_t nrows = 0;
  CAV_CHECK_CUDA(cudaMemcpyAsync(&nrows, pos + 2 * NNc, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CAV_CHECK_CUDA(cudaStreamSynchronize(st));
  out.n_rows = (int)nrows;
  out.rows = A.alloc<int>(nrows);
  k_compact_rows2<<<div_up(2 * NNc, 256), 256, 0, st>>>(2 * NNc, flag, pos, out.rows, out.row_of);
  CAV_CHECK_LAUNCH();
  // coarse window: fine offsets up to W_f plus one fine face on either side of each transfer
  const int Wc = fine.W / 2 + 2;
  int* row_count = scratch.alloc<int>(nrows + 1);
  out.rowptr = A.alloc<int64_t>(nrows + 1);
  const int grid = div_up(nrows, 8);
  out.cross = fine.cross;
  auto galerkin = [&](const int64_t* rowptr, int* cols, double* vals, int pass) {
    if (nrows == 0) return;
    if (out.cross)
      k_galerkin<true><<<grid, 256, 0, st>>>(Nc, Wc, (int)nrows, out.rows, fine.row_of, fine.rowptr, fine.cols,
                                             fine.vals, row_count, rowptr, cols, vals, pass, channel);
    else
      k_galerkin<false><<<grid, 256, 0, st>>>(Nc, Wc, (int)nrows, out.rows, fine.row_of, fine.rowptr, fine.cols,
                                              fine.vals, row_count, rowptr, cols, vals, pass, channel);
    CAV_CHECK_LAUNCH();
  };
  galerkin(nullptr, nullptr, nullptr, 0);
  exclusive_scan(row_count, out.rowptr, nrows, st, &scratch);
  int64_t nnz = 0;
  CAV_CHECK_CUDA(cudaMemcpyAsync(&nnz, out.rowptr + nrows, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CAV_CHECK_CUDA(cudaStreamSynchronize(st));
  out.nnz = nnz;
  out.cols = A.alloc<int>(nnz);
  out.vals = A.alloc<double>(nnz);
  galerkin(out.rowptr, out.cols, out.vals, 1);
  ee_compute_window(out, Nc, d_scratch, st);
  scratch.release();
}

// The coarse E_E's values for an unchanged structural pattern (cav_refactor): the fill pass of
// the same kernel into the level's existing arrays (the columns it writes are the ones
// already there).
static void galerkin_values(const EECsr& fine, int Nc, EECsr& out, bool channel, cudaStream_t st) {
  if (out.n_rows == 0) return;
  const int Wc = fine.W / 2 + 2;
  const int grid = div_up(out.n_rows, 8);
  if (out.cross)
    k_galerkin<true><<<grid, 256, 0, st>>>(Nc, Wc, out.n_rows, out.rows, fine.row_of, fine.rowptr, fine.cols,
                                           fine.vals, nullptr, out.rowptr, out.cols, out.vals, 1, channel);
  else
    k_galerkin<false><<<grid, 256, 0, st>>>(Nc, Wc, out.n_rows, out.rows, fine.row_of, fine.rowptr, fine.cols,
                                            fine.vals, nullptr, out.rowptr, out.cols, out.vals, 1, channel);
  CAV_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ CAV patch sets

// Velocity unknowns U_ij of cell (i, j)'s Vanka patch: u_ij, u_i+1j, v_ij, v_ij+1; on the
// channel's inflow row the top face is prescribed, so U_ij has three (U[3] = -1).
__device__ inline int cell_velocities(int N, int i, int j, bool channel, int* U) {
  const int NN = N * N;
  U[0] = j * N + i;
  U[1] = j * N + (i + 1) % N;
  U[2] = NN + j * N + i;
  U[3] = (channel && j + 1 == N) ? -1 : NN + ((j + 1) % N) * N + i;
  return U[3] < 0 ? 3 : 4;
}

// CAV: cell c = (i, j) keeps its standard Vanka patch iff no velocity of U_ij couples through
// E_E to a velocity outside U_ij (Eq. cav_patch_set; E_E's pattern is symmetric).  Vanka
// (B(1,0)): every patch is V_ij, but one whose velocities have E_E rows has E_E entries in its
// local matrix K_{E,p} = R_p K_E R_p^T, so it cannot share the E_E-free standard inverse: it
// is flagged for an inverse of its own (its set stays V_ij).  Flagged cells are "big": their
// patch is stored explicitly and factorised on its own.
__global__ void k_cell_flags(int N, int cav, const int* __restrict__ row_of, const int64_t* __restrict__ rowptr,
                             const int* __restrict__ cols, uint8_t* big, int* flag, bool channel) {
  const int cidx = blockIdx.x * blockDim.x + threadIdx.x;
  const int NN = N * N;
  if (cidx >= NN) return;
  const int i = cidx % N, j = cidx / N;
  int U4[4];
  const int nu = cell_velocities(N, i, j, channel, U4);
  int enl = 0;
  if (!cav) {
    for (int t = 0; t < nu; ++t) enl |= (row_of[U4[t]] >= 0);
  } else {
    for (int t = 0; t < nu && !enl; ++t) {
      const int r = row_of[U4[t]];
      if (r < 0) continue;
      for (int64_t q = rowptr[r]; q < rowptr[r + 1]; ++q) {
        const int k = cols[q];
        if (k != U4[0] && k != U4[1] && k != U4[2] && k != U4[3]) {
          enl = 1;
          break;
        }
      }
    }
  }
  big[cidx] = (uint8_t)enl;
  flag[cidx] = enl;
}

__global__ void k_flag_nonempty_off(int n, const int64_t* off, int* flag) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < n) flag[f] = (off[f + 1] > off[f]) ? 1 : 0;
}

__global__ void k_compact_cells(int n, const int* flag, const int64_t* pos, int* out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < n && flag[f]) out[pos[f]] = f;
}

__device__ inline void mark_cell(uint8_t* cm, const Win& wx, const Win& wy, int N, int ci, int cj,
                                 int* status) {
  const int ox = win_off(wx, pmod(ci, N), N), oy = win_off(wy, pmod(cj, N), N);
  if (ox < 0 || oy < 0) atomicExch(status, DEV_WINDOW);
  else cm[oy * wx.len + ox] = 1;
}
// The cells incident to velocity face k: a u face's left and right cells, a v face's cells
// below and above (on the channel's outflow row only the one above).
__device__ inline void mark_face_cells(uint8_t* cm, const Win& wx, const Win& wy, int N, int k,
                                       int* status, bool channel) {
  const int NN = N * N;
  const int c = k / NN, rem = k % NN, i = rem % N, j = rem / N;
  if (c == 0) mark_cell(cm, wx, wy, N, i - 1, j, status);
  else if (!(channel && j == 0)) mark_cell(cm, wx, wy, N, i, j - 1, status);
  mark_cell(cm, wx, wy, N, i, j, status);
}
__device__ inline void mark_dof(uint8_t* dm, const Win& wx, const Win& wy, int N, int comp, int gi,
                                int gj, int* status) {
  const int ox = win_off(wx, pmod(gi, N), N), oy = win_off(wy, pmod(gj, N), N);
  if (ox < 0 || oy < 0) atomicExch(status, DEV_WINDOW);
  else dm[(comp * wy.len + oy) * wx.len + ox] = 1;
}

// One warp per enlarged cell: Uhat = U_ij u (E_E neighbours of U_ij), cells C(Uhat), and the
// union V(C) of their Vanka patches, enumerated in ascending global order (u, v, p blocks;
// y then x).  pass 0 counts, pass 1 writes.
__global__ void k_cav_sets(int N, int W, int n_big, const int* __restrict__ big_cell,
                           const int* __restrict__ row_of, const int64_t* __restrict__ rowptr,
                           const int* __restrict__ cols, int* sizes, const int64_t* __restrict__ off,
                           int* dofs, int pass, int* status, bool channel, bool cav) {
  extern __shared__ unsigned char smem[];
  const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.x * warps + warp;
  const int Wc = W + 2, Wd = W + 3;
  const int lenC = (2 * Wc + 1 >= N) ? N : 2 * Wc + 1;
  const int lenD = (2 * Wd + 1 >= N) ? N : 2 * Wd + 1;
  const int per_warp = lenC * lenC + 3 * lenD * lenD;
  uint8_t* cm = smem + (size_t)warp * per_warp;
  uint8_t* dm = cm + lenC * lenC;
  if (p >= n_big) return;
  const int NN = N * N;
  const int cell = big_cell[p];
  const int i = cell % N, j = cell / N;
  const Win cx = make_win(i, Wc, N), cy = make_win(j, Wc, N);
  const Win dx = make_win(i, Wd, N), dy = make_win(j, Wd, N);
  for (int t = lane; t < per_warp; t += 32) cm[t] = 0;
  __syncwarp();
  int U4[4];
  const int nu = cell_velocities(N, i, j, channel, U4);
  if (!cav) {
    // Vanka: the flagged cell's own patch V_ij
    if (lane == 0) mark_cell(cm, cx, cy, N, i, j, status);
  }
  for (int t = 0; cav && t < nu; ++t) {
    if (lane == 0) mark_face_cells(cm, cx, cy, N, U4[t], status, channel);
    const int r = row_of[U4[t]];
    if (r < 0) continue;
    for (int64_t q = rowptr[r] + lane; q < rowptr[r + 1]; q += 32)
      mark_face_cells(cm, cx, cy, N, cols[q], status, channel);
  }
  __syncwarp();
  for (int t = lane; t < lenC * lenC; t += 32) {
    if (!cm[t]) continue;
    const int oy = t / lenC, ox = t % lenC;
    const int a = win_glob(cx, ox, N), b = win_glob(cy, oy, N);
    mark_dof(dm, dx, dy, N, 0, a, b, status);
    mark_dof(dm, dx, dy, N, 0, a + 1, b, status);
    mark_dof(dm, dx, dy, N, 1, a, b, status);
    if (!(channel && b + 1 == N)) mark_dof(dm, dx, dy, N, 1, a, b + 1, status);
    mark_dof(dm, dx, dy, N, 2, a, b, status);
  }
  __syncwarp();
  int64_t outpos = (pass == 1) ? off[p] : 0;
  int total = 0;
  for (int comp = 0; comp < 3; ++comp) {
    for (int typ = 0; typ < dy.len; ++typ) {
      const int ty = win_asc(dy, typ);
      const int gy = win_glob(dy, ty, N);
      for (int base = 0; base < dx.len; base += 32) {
        const int txp = base + lane;
        bool f = false;
        int gx = 0;
        if (txp < dx.len) {
          const int tx = win_asc(dx, txp);
          gx = win_glob(dx, tx, N);
          f = dm[(comp * dy.len + ty) * dx.len + tx] != 0;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (pass == 1 && f) {
          const int rank = __popc(bal & ((1u << lane) - 1u));
          dofs[outpos + total + rank] = comp * NN + gy * N + gx;
        }
        total += __popc(bal);
      }
    }
  }
  if (pass == 0 && lane == 0) sizes[p] = total;
}

// ------------------------------------------------------------------ local factorisation

struct LevelK {
  int N;
  double h, rho_dt, mu, dt;
  // formed once on the host, so the extraction of every patch matrix does no FP64 division
  // (the values the device would compute: IEEE division is correctly rounded on both):
  // 1 / h, 1 / (h h), rho/dt - mu (-4 / (h h)) (a velocity diagonal), mu / (h h)
  double ih, ih2, vdiag, mh2;
  bool channel;
  const int* row_of;
  const int64_t* rowptr;
  const int* cols;
  const double* vals;
};

// The Stokes entries of a boundary row (j = 0 or N - 1) of the channel's K_E: the rows of the
// ghost rules (homogeneous data), written out term by term.  With a = rho/dt, m = mu/h^2:
//   outflow row  u_{i,0}:  a + 3m at u_{i,0}; -m at u_{i+-1,0}, u_{i,1}, v_{i,0}; +m at v_{i-1,0};
//                          +-1/h at p_{i,0}, p_{i-1,0}
//                v_{i,0}:  a + 3m at v_{i,0}; -3m at v_{i,1}; +m at u_{i+1,0}; -m at u_{i,0};
//                          2/h at p_{i,0}; v_{i+-1,0} cancel (structural zeros)
//                p_{i,0}:  -(D u)_{i,0} as on the periodic grid
//   inflow row   u_{i,N-1}: a + 5m on the diagonal, the rest as on the periodic grid without
//                the wrap to row 0; v_{i,N-1} and p_{i,N-1}: the periodic rows without the
//                prescribed v_{i,N}.
// Returns the number of entries written to col / val (at most 8).
__device__ inline int channel_row(const LevelK& L, int comp, int i, int j, int* col, double* val) {
  const int N = L.N, NN = N * N;
  const int ip = (i + 1 == N) ? 0 : i + 1, im = (i == 0) ? N - 1 : i - 1;
  const double a = L.rho_dt, m = L.mh2, ih = L.ih;
  auto U = [&](int x, int y) { return y * N + x; };
  auto Vf = [&](int x, int y) { return NN + y * N + x; };
  auto Pc = [&](int x, int y) { return 2 * NN + y * N + x; };
  int n = 0;
  auto put = [&](int g, double v) {
    col[n] = g;
    val[n] = v;
    ++n;
  };
  if (j == 0) {
    if (comp == 0) {
      put(U(i, 0), a + 3.0 * m); put(U(ip, 0), -m); put(U(im, 0), -m); put(U(i, 1), -m);
      put(Vf(i, 0), -m); put(Vf(im, 0), m); put(Pc(i, 0), ih); put(Pc(im, 0), -ih);
    } else if (comp == 1) {
      put(Vf(i, 0), a + 3.0 * m); put(Vf(ip, 0), 0.0); put(Vf(im, 0), 0.0); put(Vf(i, 1), -3.0 * m);
      put(U(ip, 0), m); put(U(i, 0), -m); put(Pc(i, 0), 2.0 * ih);
    } else {
      put(U(ip, 0), -ih); put(U(i, 0), ih); put(Vf(i, 1), -ih); put(Vf(i, 0), ih);
    }
  } else {
    if (comp == 0) {
      put(U(i, j), a + 5.0 * m); put(U(ip, j), -m); put(U(im, j), -m); put(U(i, j - 1), -m);
      put(Pc(i, j), ih); put(Pc(im, j), -ih);
    } else if (comp == 1) {
      put(Vf(i, j), a + 4.0 * m); put(Vf(ip, j), -m); put(Vf(im, j), -m); put(Vf(i, j - 1), -m);
      put(Pc(i, j), ih); put(Pc(i, j - 1), -ih);
    } else {
      put(U(ip, j), -ih); put(U(i, j), ih); put(Vf(i, j), ih);
    }
  }
  return n;
}

// Entry (ga, gb) of K_E on one level (Eq. Eul_schur), with or without the E_E term.
__device__ double ke_entry(const LevelK& L, int ga, int gb, bool use_ee) {
  const int N = L.N, NN = N * N;
  const int ca = ga / NN, ra = ga % NN, ia = ra % N, ja = ra / N;
  const int cb = gb / NN, rb = gb % NN, ib = rb % N, jb = rb / N;
  if (L.channel && (ja == 0 || ja == N - 1)) {
    int col[8];
    double val[8];
    const int n = channel_row(L, ca, ia, ja, col, val);
    double v = 0.0;
    for (int t = 0; t < n; ++t)
      if (col[t] == gb) v += val[t];
    if (use_ee && ca < 2 && cb < 2 && L.row_of[ga] >= 0) {
      const int r = L.row_of[ga];
      const int pos = find_col(L.cols, L.rowptr[r], L.rowptr[r + 1], gb);
      if (pos >= 0) v = v - L.dt * L.vals[L.rowptr[r] + pos];
    }
    return v;
  }
  if (ca < 2 && cb < 2) {
    if (ca != cb) {
      double v = 0.0;
      if (use_ee && L.row_of[ga] >= 0) {
        const int r = L.row_of[ga];
        const int pos = find_col(L.cols, L.rowptr[r], L.rowptr[r + 1], gb);
        if (pos >= 0) v = 0.0 - L.dt * L.vals[L.rowptr[r] + pos];
      }
      return v;
    }
    const double ih2 = L.ih2;
    double v = 0.0;
    if (ga == gb) {
      v = L.vdiag;
    } else {
      const int dxp = pmod(ia - ib, N), dyp = pmod(ja - jb, N);
      int nb = 0;
      if (ja == jb && (dxp == 1 || dxp == N - 1)) nb += (N == 2) ? 2 : 1;
      if (ia == ib && (dyp == 1 || dyp == N - 1)) nb += (N == 2) ? 2 : 1;
      if (nb) v = -L.mu * (nb * ih2);
    }
    if (use_ee && L.row_of[ga] >= 0) {
      const int r = L.row_of[ga];
      const int pos = find_col(L.cols, L.rowptr[r], L.rowptr[r + 1], gb);
      if (pos >= 0) v = v - L.dt * L.vals[L.rowptr[r] + pos];
    }
    return v;
  }
  if (ca == 2 && cb == 2) return 0.0;
  // G (velocity row, pressure column) and -D = G^T (pressure row, velocity column)
  int cv, iv, jv, ip, jp;
  if (ca < 2) { cv = ca; iv = ia; jv = ja; ip = ib; jp = jb; }
  else { cv = cb; iv = ib; jv = jb; ip = ia; jp = ja; }
  const double ih = L.ih;
  if (ip == iv && jp == jv) return ih;
  if (cv == 0 && jp == jv && ip == pmod(iv - 1, N)) return -ih;
  if (cv == 1 && ip == iv && jp == pmod(jv - 1, N)) return -ih;
  return 0.0;
}

struct FactorJob {
  const int* jobs;          // nullable: block b factorises patch jobs[b] (else patch b)
  const int64_t* dof_off;   // per patch offsets into dofs (n_jobs + 1)
  const int* dofs;
  const int64_t* mat_off;   // per patch element offset into A (ld * (n + border))
  double* A;                // column-major, ld = round8(n + border)
  double* s_r;              // per patch (n + border) scales; offsets dof_off[p] + p * border
  double* s_c;
  int* mdim;                // out: per patch matrix order m = n + border
  int border_all_pressure;  // 1: add the pressure-mean border when a patch holds every pressure
  int use_ee;
};

// One block per patch: extract K_{E,p} (column-major, ld = round8(m)), one pass of row then
// column max-norm equilibration with power-of-two scales (Sec. 3.3), then in-place
// Gauss-Jordan inversion with partial pivoting (first maximal row on ties).  The result is
// the inverse of diag(s_r) K diag(s_c); a zero pivot raises DEV_SINGULAR.
__global__ void k_factor(LevelK L, FactorJob J, int bordered_job, int* status) {
  extern __shared__ double sh[];
  const int p = J.jobs ? J.jobs[blockIdx.x] : (int)blockIdx.x;
  const int64_t d0 = J.dof_off[p];
  const int n = (int)(J.dof_off[p + 1] - d0);
  const int NN = L.N * L.N;
  __shared__ int s_border;
  __shared__ int s_piv;
  __shared__ double s_pmax[32];
  __shared__ int s_pidx[32];
  if (threadIdx.x == 0) {
    int border = 0;
    if (bordered_job) border = 1;
    else if (J.border_all_pressure) {
      int np = 0;
      for (int a = 0; a < n; ++a) np += (J.dofs[d0 + a] >= 2 * NN);
      border = (np == NN);
    }
    s_border = border;
    J.mdim[p] = n + border;
  }
  __syncthreads();
  const int m = n + s_border;
  const int ld = (m + 7) & ~7;
  double* A = J.A + J.mat_off[p];
  const int64_t so = d0 + p;  // one spare scale slot per patch for a border
  double* sr = J.s_r + so;
  double* sc = J.s_c + so;
  double* rowk = sh;
  double* colk = sh + m;
  const int* dofs = J.dofs + d0;
  // extraction
  for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
    const int b = (int)(e / m), a = (int)(e % m);
    double v;
    if (a < n && b < n) v = ke_entry(L, dofs[a], dofs[b], J.use_ee != 0);
    else if (a == n && b == n) v = 0.0;
    else {
      const int g = (a == n) ? dofs[b] : dofs[a];
      v = (g >= 2 * NN) ? 1.0 : 0.0;
    }
    A[(int64_t)b * ld + a] = v;
  }
  __syncthreads();
  // row scales
  for (int a = threadIdx.x; a < m; a += blockDim.x) {
    double mx = 0.0;
    for (int b = 0; b < m; ++b) mx = fmax(mx, fabs(A[(int64_t)b * ld + a]));
    sr[a] = (mx > 0.0) ? pow2_recip(mx) : 1.0;
    if (mx == 0.0) atomicExch(status, DEV_SINGULAR);
  }
  __syncthreads();
  // column scales of diag(s_r) K
  for (int b = threadIdx.x; b < m; b += blockDim.x) {
    double mx = 0.0;
    for (int a = 0; a < m; ++a) mx = fmax(mx, fabs(sr[a] * A[(int64_t)b * ld + a]));
    sc[b] = (mx > 0.0) ? pow2_recip(mx) : 1.0;
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
    const int b = (int)(e / m), a = (int)(e % m);
    A[(int64_t)b * ld + a] = sr[a] * A[(int64_t)b * ld + a] * sc[b];
  }
  __syncthreads();
  // Gauss-Jordan with row pivoting; the column permutation is undone at the end
  int* perm = reinterpret_cast<int*>(sh + 2 * m);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < m; ++k) {
    // pivot: first row of maximal modulus in column k, rows k..m-1
    double best = -1.0;
    int bi = m;
    for (int a = k + threadIdx.x; a < m; a += blockDim.x) {
      const double v = fabs(A[(int64_t)k * ld + a]);
      if (v > best) { best = v; bi = a; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { s_pmax[warp] = best; s_pidx[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double bb = -1.0;
      int ii = m;
      for (int w = 0; w < nw; ++w)
        if (s_pmax[w] > bb || (s_pmax[w] == bb && s_pidx[w] < ii)) { bb = s_pmax[w]; ii = s_pidx[w]; }
      s_piv = ii;
      perm[k] = ii;
      if (!(bb > 0.0)) atomicExch(status, DEV_SINGULAR);
    }
    __syncthreads();
    const int pr = s_piv;
    if (pr != k && pr < m) {
      for (int b = threadIdx.x; b < m; b += blockDim.x) {
        const double t = A[(int64_t)b * ld + k];
        A[(int64_t)b * ld + k] = A[(int64_t)b * ld + pr];
        A[(int64_t)b * ld + pr] = t;
      }
    }
    __syncthreads();
    const double piv = A[(int64_t)k * ld + k];
    const double ipiv = (piv != 0.0) ? 1.0 / piv : 0.0;
    for (int b = threadIdx.x; b < m; b += blockDim.x) {
      rowk[b] = (b == k) ? ipiv : A[(int64_t)b * ld + k] * ipiv;
    }
    for (int a = threadIdx.x; a < m; a += blockDim.x) colk[a] = A[(int64_t)k * ld + a];
    __syncthreads();
    // rank-one update, warps over columns and lanes over rows (coalesced, no index division)
    for (int b = warp; b < m; b += nw) {
      double* colp = A + (int64_t)b * ld;
      const double rb = rowk[b];
      if (b == k) {
        for (int a = lane; a < m; a += 32) colp[a] = (a == k) ? rb : -colk[a] * ipiv;
      } else {
        for (int a = lane; a < m; a += 32) colp[a] = (a == k) ? rb : colp[a] - colk[a] * rb;
      }
    }
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, last first
  for (int k = m - 1; k >= 0; --k) {
    const int pr = perm[k];
    if (pr != k && pr < m) {
      for (int a = threadIdx.x; a < m; a += blockDim.x) {
        const double t = A[(int64_t)k * ld + a];
        A[(int64_t)k * ld + a] = A[(int64_t)pr * ld + a];
        A[(int64_t)pr * ld + a] = t;
      }
    }
    __syncthreads();
  }
}

// The coarsest level's factorisation on the whole GPU: the steps of k_factor (extraction,
// power-of-two row then column equilibration, Gauss-Jordan with the first maximal pivot, the
// row interchanges undone as column interchanges at the end) in one cooperative launch, CTA
// `rank` owning the columns rank, rank + G, ... and a grid barrier between elimination steps.
// Every value comes from the same expressions in the same order as in k_factor, so the
// inverse is the same bit for bit.  One barrier per step.  Lookahead: in step k the owner of
// column k + 1 updates that column first; FG_PIV_WARPS of its warps then find the next pivot
// and publish column k + 1 with the pivot row interchanged (pub_col, pub_piv: double-buffered
// by the step's parity) while the other warps update the remaining columns.  A CTA's first
// sc_cols columns stay in shared memory for the whole elimination (the rest are streamed from
// L2 every step).  perm: m ints.  A barrier that runs out records DEV_TIMEOUT; every CTA then
// stops at its next barrier (one decision per CTA: thread 0 reads the status word and shares
// it through s_ok).
constexpr int FG_THREADS = 512;  // threads per CTA of k_factor_grid
constexpr int FG_ROWS = 6;       // register rows per thread of its update (the rest in a plain loop)
constexpr int FG_PIV_WARPS = 4;  // warps of the next column's owner that search its pivot
__device__ inline bool factor_grid_sync(unsigned* bar, int* status, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    grid_barrier(bar, status);
    *s_ok = *reinterpret_cast<volatile int*>(status) != DEV_TIMEOUT;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Warps 0 .. FG_PIV_WARPS - 1 of the owner of column k (its values at col): the pivot (the first
// row of maximal modulus among rows k..m-1, as in k_factor; the moduli are compared as their
// bit patterns, which order non-negative doubles as the values do), published with the
// interchanged column.  Synchronises those warps only (named barrier 1).
__device__ inline void factor_grid_pivot(const double* col, int ld, int m, int k, double* pub_col, int* pub_piv,
                                         int* perm, int* status, unsigned long long* s_pkey, int* s_pidx,
                                         int* s_piv) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  constexpr int NT = FG_PIV_WARPS * 32;
  unsigned long long best = 0;
  int bi = m;
  for (int a = k + t; a < m; a += NT) {
    const unsigned long long v = (unsigned long long)__double_as_longlong(col[a]) & 0x7fffffffffffffffull;
    if (bi == m || v > best) { best = v; bi = a; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (oi < m && (bi == m || ob > best || (ob == best && oi < bi))) { best = ob; bi = oi; }
  }
  if (lane == 0) { s_pkey[warp] = best; s_pidx[warp] = bi; }
  asm volatile("bar.sync 1, %0;" ::"r"(NT) : "memory");
  if (t == 0) {
    unsigned long long bb = 0;
    int ii = m;
    for (int w = 0; w < FG_PIV_WARPS; ++w)
      if (s_pidx[w] < m && (ii == m || s_pkey[w] > bb || (s_pkey[w] == bb && s_pidx[w] < ii))) {
        bb = s_pkey[w];
        ii = s_pidx[w];
      }
    *s_piv = ii;
    perm[k] = ii;
    pub_piv[k & 1] = ii;
    if (!(__longlong_as_double((long long)bb) > 0.0)) atomicExch(status, DEV_SINGULAR);
  }
  asm volatile("bar.sync 1, %0;" ::"r"(NT) : "memory");
  const int pr = *s_piv;
  double* out = pub_col + (int64_t)(k & 1) * ld;
  for (int a = t; a < m; a += NT) {
    double v = col[a];
    if (pr != k && pr < m) {
      if (a == k) v = col[pr];
      else if (a == pr) v = col[k];
    }
    out[a] = v;
  }
}

// The steps before the elimination, on the whole grid: the coarsest matrix (bordered by the
// pressure-mean row and column when `bordered`) extracted into J.A, then power-of-two row and
// column equilibration (the scales into J.s_r, J.s_c), as in k_factor.  False if a barrier
// ran out.
__device__ bool factor_grid_prepare(const LevelK& L, const FactorJob& J, int bordered, int* status, unsigned* bar,
                                    int* s_ok) {
  const int G = gridDim.x, rank = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int64_t gt = (int64_t)rank * nt + tid, GT = (int64_t)G * nt;
  const int64_t d0 = J.dof_off[0];
  const int n = (int)(J.dof_off[1] - d0);
  const int NN = L.N * L.N;
  const int m = n + bordered;
  if (gt == 0) J.mdim[0] = m;
  const int ld = (m + 7) & ~7;
  double* A = J.A + J.mat_off[0];
  double* sr = J.s_r + d0;
  double* sc = J.s_c + d0;
  const int* dofs = J.dofs + d0;
  for (int64_t e = gt; e < (int64_t)m * m; e += GT) {
    const int b = (int)(e / m), a = (int)(e % m);
    double v;
    if (a < n && b < n) v = ke_entry(L, dofs[a], dofs[b], J.use_ee != 0);
    else if (a == n && b == n) v = 0.0;
    else {
      const int g = (a == n) ? dofs[b] : dofs[a];
      v = (g >= 2 * NN) ? 1.0 : 0.0;
    }
    A[(int64_t)b * ld + a] = v;
  }
  if (!factor_grid_sync(bar, status, s_ok)) return false;
  for (int64_t a = gt; a < m; a += GT) {
    double mx = 0.0;
    for (int b = 0; b < m; ++b) mx = fmax(mx, fabs(A[(int64_t)b * ld + a]));
    sr[a] = (mx > 0.0) ? pow2_recip(mx) : 1.0;
    if (mx == 0.0) atomicExch(status, DEV_SINGULAR);
  }
  if (!factor_grid_sync(bar, status, s_ok)) return false;
  for (int64_t b = gt; b < m; b += GT) {
    double mx = 0.0;
    for (int a = 0; a < m; ++a) mx = fmax(mx, fabs(sr[a] * A[(int64_t)b * ld + a]));
    sc[b] = (mx > 0.0) ? pow2_recip(mx) : 1.0;
  }
  if (!factor_grid_sync(bar, status, s_ok)) return false;
  for (int64_t e = gt; e < (int64_t)m * m; e += GT) {
    const int b = (int)(e / m), a = (int)(e % m);
    A[(int64_t)b * ld + a] = sr[a] * A[(int64_t)b * ld + a] * sc[b];
  }
  if (!factor_grid_sync(bar, status, s_ok)) return false;
  return true;
}

// The row interchanges undone as column interchanges, last first (each row on its own).
__device__ void factor_grid_unscramble(double* A, int ld, int m, const int* perm) {
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, GT = (int64_t)gridDim.x * blockDim.x;
  for (int64_t a = gt; a < m; a += GT) {
    for (int k = m - 1; k >= 0; --k) {
      const int pr = perm[k];
      if (pr != k && pr < m) {
        const double t = A[(int64_t)k * ld + a];
        A[(int64_t)k * ld + a] = A[(int64_t)pr * ld + a];
        A[(int64_t)pr * ld + a] = t;
      }
    }
  }
}

__global__ void __launch_bounds__(FG_THREADS) k_factor_grid(LevelK L, FactorJob J, int bordered, int* status, unsigned* bar,
                                                      double* pub_col, int* pub_piv, int* perm, int sc_cols) {
  // shared memory: per own column rb, then the value moving to the pivot row; then the first
  // sc_cols own columns
  extern __shared__ double sh[];
  __shared__ unsigned long long s_pkey[FG_PIV_WARPS];
  __shared__ int s_pidx[FG_PIV_WARPS];
  __shared__ int s_piv, s_ok;
  const int G = gridDim.x, rank = blockIdx.x, tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5;
  const int m = (int)(J.dof_off[1] - J.dof_off[0]) + bordered;
  const int ld = (m + 7) & ~7;
  double* A = J.A + J.mat_off[0];
  const int ncol_max = (m + G - 1) / G;
  double* cs = sh + 2 * ncol_max;  // [sc_cols][ld]
  if (!factor_grid_prepare(L, J, bordered, status, bar, &s_ok)) return;
  const int ncol = (m > rank) ? (m - rank + G - 1) / G : 0;  // own columns rank + j G, j < ncol
  const int nsc = min(sc_cols, ncol);
  // own column j: in shared memory for j < nsc, else in the matrix
  auto col = [&](int j) -> double* {
    return (j < nsc) ? cs + (int64_t)j * ld : A + (int64_t)(rank + j * G) * ld;
  };
  for (int j = 0; j < nsc; ++j)
    for (int a = tid; a < m; a += nt) cs[(int64_t)j * ld + a] = A[(int64_t)(rank + j * G) * ld + a];
  __syncthreads();
  if (rank == 0 && warp < FG_PIV_WARPS)
    factor_grid_pivot(col(0), ld, m, 0, pub_col, pub_piv, perm, status, s_pkey, s_pidx, &s_piv);
  if (!factor_grid_sync(bar, status, &s_ok)) return;
  for (int k = 0; k < m; ++k) {
    const int pr = pub_piv[k & 1];
    const double* colk = pub_col + (int64_t)(k & 1) * ld;
    const bool swap = pr != k && pr < m;
    const int jn = (k + 1 < m && (k + 1) % G == rank) ? (k + 1) / G : -1;  // own index of column k + 1
    // this thread's register rows a = tid + q nt of the pivot column
    double ck[FG_ROWS];
#pragma unroll
    for (int q = 0; q < FG_ROWS; ++q) {
      const int a = tid + q * nt;
      ck[q] = (a < m) ? colk[a] : 0.0;
    }
    const double piv = colk[k];
    const double ipiv = (piv != 0.0) ? 1.0 / piv : 0.0;
    // rowk of k_factor for the own columns (after the interchange), and the entry that moves
    // from row k to row pr
    for (int j = tid; j < ncol; j += nt) {
      const int b = rank + j * G;
      const double* c = col(j);
      const double ak = c[k];
      const double ap = swap ? c[pr] : ak;
      sh[j] = (b == k) ? ipiv : ap * ipiv;
      sh[ncol + j] = ak;
    }
    __syncthreads();
    // the next column's owner: that column first, then its pivot on FG_PIV_WARPS warps
    if (jn >= 0) {
      double* colp = col(jn);
      const double rb = sh[jn], moved = sh[ncol + jn];
      for (int a = tid; a < m; a += nt) {
        const double c = (swap && a == pr) ? moved : colp[a];
        colp[a] = (a == k) ? rb : c - colk[a] * rb;
      }
      __syncthreads();
      if (warp < FG_PIV_WARPS)
        factor_grid_pivot(colp, ld, m, k + 1, pub_col, pub_piv, perm, status, s_pkey, s_pidx, &s_piv);
    }
    // the other own columns on the register rows, two at a time: the next pair's entries are
    // loaded before the current pair is updated
    double cur[2][FG_ROWS], nxt[2][FG_ROWS];
    auto load_pair = [&](int j0, double (&v)[2][FG_ROWS]) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int j = j0 + u;
        const bool live = j < ncol && j != jn;
        const double* c = col(live ? j : 0);
#pragma unroll
        for (int q = 0; q < FG_ROWS; ++q) {
          const int a = tid + q * nt;
          v[u][q] = (live && a < m) ? c[a] : 0.0;
        }
      }
    };
    load_pair(0, cur);
    for (int j0 = 0; j0 < ncol; j0 += 2) {
      if (j0 + 2 < ncol) load_pair(j0 + 2, nxt);
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int j = j0 + u;
        if (j >= ncol || j == jn) continue;
        const int b = rank + j * G;
        double* colp = col(j);
        const double rb = sh[j], moved = sh[ncol + j];
#pragma unroll
        for (int q = 0; q < FG_ROWS; ++q) {
          const int a = tid + q * nt;
          if (a >= m) continue;
          if (b == k) {
            colp[a] = (a == k) ? rb : -ck[q] * ipiv;
          } else {
            const double c = (swap && a == pr) ? moved : cur[u][q];
            colp[a] = (a == k) ? rb : c - ck[q] * rb;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int q = 0; q < FG_ROWS; ++q) cur[u][q] = nxt[u][q];
    }
    // rows beyond the register rows
    for (int a = FG_ROWS * nt + tid; a < m; a += nt) {
      const double cka = colk[a];
      for (int j = 0; j < ncol; ++j) {
        if (j == jn) continue;
        const int b = rank + j * G;
        double* colp = col(j);
        const double rb = sh[j];
        if (b == k) {
          colp[a] = (a == k) ? rb : -cka * ipiv;
        } else {
          const double c = (swap && a == pr) ? sh[ncol + j] : colp[a];
          colp[a] = (a == k) ? rb : c - cka * rb;
        }
      }
    }
    if (!factor_grid_sync(bar, status, &s_ok)) return;
  }
  // the shared-memory columns back into the matrix
  for (int j = 0; j < nsc; ++j)
    for (int a = tid; a < m; a += nt) A[(int64_t)(rank + j * G) * ld + a] = cs[(int64_t)j * ld + a];
  if (!factor_grid_sync(bar, status, &s_ok)) return;
  factor_grid_unscramble(A, ld, m, perm);
}

// The same factorisation blocked in panels of GP_PB columns, with one grid barrier per panel
// instead of one per elimination step.  CTA 0 factorises the panels: in the interval of panel
// p it loads panel p + 1's columns into shared memory, applies panel p's steps to them, then
// eliminates within the panel (pivot search, interchange, update of the panel's columns) and
// publishes, per step k, the pivot row and the pivot column as the other columns use it (cpan,
// ppiv: double-buffered by the panel's parity).  The other CTAs own the columns cyclically and
// apply panel p's steps to every own column outside panels p and p + 1, GP_C columns at a
// time held in registers (rows tid + q GP_THREADS), the two entries a step needs from a
// column (rows k and p_k) passed through shared memory.  A column goes through the steps
// k = 0, 1, ... in order with the expressions of k_factor, so the inverse is the same bit for
// bit.  Needs m <= R GP_THREADS and (GP_PB + 1) round8(m) doubles of shared memory.
constexpr int GP_THREADS = 512;
constexpr int GP_PB = 8;  // panel width
constexpr int GP_C = 4;   // columns per register chunk

template <int R>
__global__ void __launch_bounds__(GP_THREADS) k_factor_panels(LevelK L, FactorJob J, int bordered, int* status,
                                                              unsigned* bar, double* cpan, int* ppiv, int* perm) {
  // panel CTA: [GP_PB][ld] the panel's columns, then [ld] the current pivot column;
  // the others: [GP_PB][ld] the published pivot columns of the panel being applied
  extern __shared__ double gsh[];
  __shared__ double s_ak[2][GP_C], s_ap[2][GP_C];
  __shared__ double s_rb[GP_PB], s_mv[GP_PB], s_ipiv[GP_PB];
  __shared__ int s_pr[GP_PB];
  __shared__ unsigned long long s_key[GP_THREADS / 32];
  __shared__ int s_idx[GP_THREADS / 32];
  __shared__ int s_piv, s_ok;
  const int G = gridDim.x, rank = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = (int)(J.dof_off[1] - J.dof_off[0]) + bordered;
  const int ld = (m + 7) & ~7;
  double* A = J.A + J.mat_off[0];
  const int npan = (m + GP_PB - 1) / GP_PB;
  const int U = G - 1;  // column j belongs to CTA 1 + j % U
  if (!factor_grid_prepare(L, J, bordered, status, bar, &s_ok)) return;
  double* colbuf = gsh + (int64_t)GP_PB * ld;

  // --- the panel CTA's parts
  auto panel_width = [&](int q) { return min(GP_PB, m - q * GP_PB); };
  auto panel_load = [&](int q) {
    const int nb = panel_width(q);
    for (int i = 0; i < nb; ++i)
      for (int a = tid; a < m; a += GP_THREADS) gsh[(int64_t)i * ld + a] = A[(int64_t)(q * GP_PB + i) * ld + a];
    __syncthreads();
  };
  auto panel_store = [&](int q) {
    const int nb = panel_width(q);
    for (int i = 0; i < nb; ++i)
      for (int a = tid; a < m; a += GP_THREADS) A[(int64_t)(q * GP_PB + i) * ld + a] = gsh[(int64_t)i * ld + a];
  };
  // panel p's published steps applied to panel p + 1's columns in shared memory; each step's
  // pivot-column rows of this thread are loaded one step ahead
  auto panel_apply = [&](int p) {
    const int nbp = panel_width(p), nb = panel_width(p + 1);
    double ckn[R];
    auto load_ck = [&](int i, double (&v)[R]) {
      const double* ck = cpan + (int64_t)((p & 1) * GP_PB + i) * ld;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int a = tid + q * GP_THREADS;
        v[q] = (a < m) ? ck[a] : 0.0;
      }
    };
    load_ck(0, ckn);
    for (int i = 0; i < nbp; ++i) {
      double ckc[R];
#pragma unroll
      for (int q = 0; q < R; ++q) ckc[q] = ckn[q];
      if (i + 1 < nbp) load_ck(i + 1, ckn);
      const int k = p * GP_PB + i;
      const int pr = ppiv[(p & 1) * GP_PB + i];
      const bool swap = pr != k && pr < m;
      const double piv = cpan[(int64_t)((p & 1) * GP_PB + i) * ld + k];
      const double ipiv = (piv != 0.0) ? 1.0 / piv : 0.0;
      if (tid < nb) {
        const double* c = gsh + (int64_t)tid * ld;
        const double ak = c[k];
        const double ap = swap ? c[pr] : ak;
        s_rb[tid] = ap * ipiv;
        s_mv[tid] = ak;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int a = tid + q * GP_THREADS;
        if (a >= m) continue;
        for (int i2 = 0; i2 < nb; ++i2) {
          double* colp = gsh + (int64_t)i2 * ld;
          const double rb = s_rb[i2];
          const double c = (swap && a == pr) ? s_mv[i2] : colp[a];
          colp[a] = (a == k) ? rb : c - ckc[q] * rb;
        }
      }
      __syncthreads();
    }
  };
  // elimination within panel q (its columns in shared memory, already through panel q - 1)
  auto panel_factor = [&](int q) {
    const int nb = panel_width(q);
    for (int i = 0; i < nb; ++i) {
      const int k = q * GP_PB + i;
      const double* ci = gsh + (int64_t)i * ld;
      unsigned long long best = 0;
      int bi = m;
      for (int a = k + tid; a < m; a += GP_THREADS) {
        const unsigned long long v = (unsigned long long)__double_as_longlong(ci[a]) & 0x7fffffffffffffffull;
        if (bi == m || v > best) { best = v; bi = a; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi < m && (bi == m || ob > best || (ob == best && oi < bi))) { best = ob; bi = oi; }
      }
      if (lane == 0) { s_key[warp] = best; s_idx[warp] = bi; }
      __syncthreads();
      if (tid == 0) {
        unsigned long long bb = 0;
        int ii = m;
        for (int w = 0; w < GP_THREADS / 32; ++w)
          if (s_idx[w] < m && (ii == m || s_key[w] > bb || (s_key[w] == bb && s_idx[w] < ii))) {
            bb = s_key[w];
            ii = s_idx[w];
          }
        if (!(__longlong_as_double((long long)bb) > 0.0)) atomicExch(status, DEV_SINGULAR);
        s_piv = ii;
        perm[k] = ii;
        ppiv[(q & 1) * GP_PB + i] = ii;
      }
      __syncthreads();
      const int pr = s_piv;
      const bool swap = pr != k && pr < m;
      // the pivot column with rows k and pr interchanged, kept and published; the columns'
      // rb and moved entries in the same pass (all read the columns before the update)
      const double piv = swap ? ci[pr] : ci[k];
      const double ipiv = (piv != 0.0) ? 1.0 / piv : 0.0;
      double* pub = cpan + (int64_t)((q & 1) * GP_PB + i) * ld;
      for (int a = tid; a < m; a += GP_THREADS) {
        double v = ci[a];
        if (swap) {
          if (a == k) v = ci[pr];
          else if (a == pr) v = ci[k];
        }
        colbuf[a] = v;
        pub[a] = v;
      }
      if (tid < nb) {
        const double* c = gsh + (int64_t)tid * ld;
        const double ak = c[k];
        const double ap = swap ? c[pr] : ak;
        s_rb[tid] = (tid == i) ? ipiv : ap * ipiv;
        s_mv[tid] = ak;
      }
      __syncthreads();
      for (int a = tid; a < m; a += GP_THREADS) {
        const double cka = colbuf[a];
        for (int i2 = 0; i2 < nb; ++i2) {
          double* colp = gsh + (int64_t)i2 * ld;
          const double rb = s_rb[i2];
          if (i2 == i) {
            colp[a] = (a == k) ? rb : -cka * ipiv;
          } else {
            const double c = (swap && a == pr) ? s_mv[i2] : colp[a];
            colp[a] = (a == k) ? rb : c - cka * rb;
          }
        }
      }
      __syncthreads();
    }
  };

  // --- the other CTAs: panel p's steps on their own columns outside panels p and p + 1
  const int ncol = (rank >= 1 && m > rank - 1) ? (m - (rank - 1) + U - 1) / U : 0;  // own j = rank - 1 + t U
  unsigned slot_ctr = 0;
  auto update_apply = [&](int p) {
    const int nbp = panel_width(p);
    for (int i = 0; i < nbp; ++i)
      for (int a = tid; a < m; a += GP_THREADS)
        gsh[(int64_t)i * ld + a] = cpan[(int64_t)((p & 1) * GP_PB + i) * ld + a];
    if (tid < nbp) {
      const int k = p * GP_PB + tid;
      s_pr[tid] = ppiv[(p & 1) * GP_PB + tid];
      const double piv = cpan[(int64_t)((p & 1) * GP_PB + tid) * ld + k];
      s_ipiv[tid] = (piv != 0.0) ? 1.0 / piv : 0.0;
    }
    __syncthreads();
    auto live = [&](int t) {
      if (t >= ncol) return false;
      const int pj = (rank - 1 + t * U) / GP_PB;
      return pj != p && pj != p + 1;
    };
    double cur[GP_C][R];
    auto load_chunk = [&](int t0, double (&v)[GP_C][R]) {
#pragma unroll
      for (int c = 0; c < GP_C; ++c) {
        const int t = t0 + c;
        const bool lv = live(t);
        const double* col = A + (int64_t)(rank - 1 + (lv ? t : 0) * U) * ld;
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const int a = tid + q * GP_THREADS;
          v[c][q] = (lv && a < m) ? col[a] : 0.0;
        }
      }
    };
    for (int t0 = 0; t0 < ncol; t0 += GP_C) {
      load_chunk(t0, cur);
      bool lv[GP_C];
      bool any = false;
#pragma unroll
      for (int c = 0; c < GP_C; ++c) {
        lv[c] = live(t0 + c);
        any = any || lv[c];
      }
      if (any) {
        for (int i = 0; i < nbp; ++i) {
          const int k = p * GP_PB + i;
          const int pr = s_pr[i];
          const bool swap = pr != k && pr < m;
          const double ipiv = s_ipiv[i];
          const int sl = slot_ctr & 1;
          ++slot_ctr;
#pragma unroll
          for (int q = 0; q < R; ++q) {
            const int a = tid + q * GP_THREADS;
            if (a == k) {
#pragma unroll
              for (int c = 0; c < GP_C; ++c) s_ak[sl][c] = cur[c][q];
            }
            if (a == pr) {
#pragma unroll
              for (int c = 0; c < GP_C; ++c) s_ap[sl][c] = cur[c][q];
            }
          }
          __syncthreads();
          const double* ck = gsh + (int64_t)i * ld;
#pragma unroll
          for (int c = 0; c < GP_C; ++c) {
            if (!lv[c]) continue;
            const double ak = s_ak[sl][c];
            const double ap = swap ? s_ap[sl][c] : ak;
            const double rb = ap * ipiv, moved = ak;
#pragma unroll
            for (int q = 0; q < R; ++q) {
              const int a = tid + q * GP_THREADS;
              if (a >= m) continue;
              const double cc = (swap && a == pr) ? moved : cur[c][q];
              cur[c][q] = (a == k) ? rb : cc - ck[a] * rb;
            }
          }
        }
#pragma unroll
        for (int c = 0; c < GP_C; ++c) {
          if (!lv[c]) continue;
          double* col = A + (int64_t)(rank - 1 + (t0 + c) * U) * ld;
#pragma unroll
          for (int q = 0; q < R; ++q) {
            const int a = tid + q * GP_THREADS;
            if (a < m) col[a] = cur[c][q];
          }
        }
      }
    }
    __syncthreads();  // gsh is refilled by the next panel
  };

  if (rank == 0) {
    panel_load(0);
    panel_factor(0);
    panel_store(0);
  }
  if (!factor_grid_sync(bar, status, &s_ok)) return;
  for (int p = 0; p < npan; ++p) {
    if (rank == 0) {
      if (p + 1 < npan) {
        panel_load(p + 1);
        panel_apply(p);
        panel_factor(p + 1);
        panel_store(p + 1);
      }
    } else {
      update_apply(p);
    }
    if (!factor_grid_sync(bar, status, &s_ok)) return;
  }
  factor_grid_unscramble(A, ld, m, perm);
}

// The same factorisation for one patch on a pair of CTAs (a cluster of two), the matrix held
// in shared memory: CTA r keeps the columns b = r, r + 2, ... of the m x m matrix (about 200 KB each for m = 224), so a patch of up to FP_MMAX unknowns never leaves the SMs.
// Every value is computed by the same expressions in the same order as in k_factor, and
// the pivot is the same (the first row of maximal modulus), so the inverse is bitwise the
// same.  Per elimination step the column's owner finds the pivot and publishes the pivot row
// index and the column (before the interchange) to both CTAs through distributed shared
// memory, one cluster barrier later both interchange rows and update their own columns; the
// published column is double-buffered, so one barrier per step suffices.  The column
// interchanges that undo the pivoting are folded into the final store.
constexpr int FP_THREADS = 512;
constexpr int FP_MMAX = 224;
// below this size the per-step cluster barrier outweighs the global-memory traffic it saves
// (measured: the fiber channel at N = 64, patches under 100 unknowns, set up in 21.7 ms with
// the one-CTA kernel and 25.4 ms with pairs; the N = 256 membrane, 128-218, 80 -> 75 ms)
constexpr int FP_MMIN = 128;

static size_t factor_pair_smem(int m) {
  const int ld = (m + 7) & ~7, mc = (m + 1) / 2;
  return (size_t)mc * ld * sizeof(double)          // my columns
         + (size_t)4 * m * sizeof(double)            // published columns (2), row maxima (2)
         + (size_t)mc * sizeof(double)              // the pivot row on my columns
         + (size_t)3 * m * sizeof(int) + 64;        // pivots, column map, its inverse
}

constexpr int FP_ROWS_PER_LANE = (FP_MMAX + 31) / 32;

// One warp of the owner of column k (local index k >> 1): the first row a >= k of maximal
// modulus (compared as the magnitudes' bit patterns, which order non-negative doubles as the
// values do), written to perm[k] in both CTAs, and the column before the interchange into
// pub[k & 1] of both.
__device__ void pair_pivot_publish(cooperative_groups::cluster_group& cluster, const double* A, int ld, int m,
                                   int k, double* pub, int* perm, int* status) {
  const int lane = threadIdx.x & 31;
  const int r = (int)cluster.block_rank();
  const double* ak = A + (int64_t)(k >> 1) * ld;
  unsigned long long best = 0;
  int bi = m;
  for (int a = k + lane; a < m; a += 32) {
    const unsigned long long v = (unsigned long long)__double_as_longlong(ak[a]) & 0x7fffffffffffffffull;
    if (bi == m || v > best) { best = v; bi = a; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (oi < m && (bi == m || ob > best || (ob == best && oi < bi))) { best = ob; bi = oi; }
  }
  if (lane == 0) {
    if (!(__longlong_as_double((long long)best) > 0.0)) atomicExch(status, DEV_SINGULAR);
    perm[k] = bi;
    *cluster.map_shared_rank(perm + k, r ^ 1) = bi;
  }
  double* colk = pub + (k & 1) * m;
  double* peer = cluster.map_shared_rank(colk, r ^ 1);
  for (int a = lane; a < m; a += 32) {
    const double v = ak[a];
    colk[a] = v;
    peer[a] = v;
  }
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(FP_THREADS, 2)
k_factor_pair(LevelK L, FactorJob J, const int* __restrict__ jobs, int* status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) double shp[];
  const int r = (int)cluster.block_rank();
  const int p = jobs[blockIdx.x >> 1];
  const int64_t d0 = J.dof_off[p];
  const int n = (int)(J.dof_off[p + 1] - d0);
  const int NN = L.N * L.N;
  __shared__ int s_border;
  if (threadIdx.x == 0) {
    int border = 0;
    if (J.border_all_pressure) {
      int np = 0;
      for (int a = 0; a < n; ++a) np += (J.dofs[d0 + a] >= 2 * NN);
      border = (np == NN);
    }
    s_border = border;
    if (r == 0) J.mdim[p] = n + border;
  }
  __syncthreads();
  const int m = n + s_border;
  const int ld = (m + 7) & ~7;
  const int mc = (m - r + 1) / 2;  // my columns
  double* A = shp;                                   // [mc][ld]
  double* pub = A + (size_t)((m + 1) / 2) * ld;      // [2][m] published columns
  double* rmax = pub + 2 * m;                        // [2][m] row maxima of each CTA
  double* rowk = rmax + 2 * m;                       // [(m + 1) / 2]
  int* perm = reinterpret_cast<int*>(rowk + (m + 1) / 2);
  int* src = perm + m;
  int* dst = src + m;
  const int64_t so = d0 + p;
  double* sr = J.s_r + so;
  double* sc = J.s_c + so;
  const int* dofs = J.dofs + d0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = FP_THREADS / 32;
  // extraction of my columns
  for (int64_t e = tid; e < (int64_t)mc * m; e += FP_THREADS) {
    const int q = (int)(e / m), a = (int)(e % m);
    const int b = 2 * q + r;
    double v;
    if (a < n && b < n) v = ke_entry(L, dofs[a], dofs[b], J.use_ee != 0);
    else if (a == n && b == n) v = 0.0;
    else {
      const int g = (a == n) ? dofs[b] : dofs[a];
      v = (g >= 2 * NN) ? 1.0 : 0.0;
    }
    A[(int64_t)q * ld + a] = v;
  }
  __syncthreads();
  // row scales: the maximum over my columns, exchanged, then over both
  {
    double* peer = cluster.map_shared_rank(rmax, r ^ 1);
    for (int a = tid; a < m; a += FP_THREADS) {
      double mx = 0.0;
      for (int q = 0; q < mc; ++q) mx = fmax(mx, fabs(A[(int64_t)q * ld + a]));
      rmax[r * m + a] = mx;
      peer[r * m + a] = mx;
    }
  }
  cluster.sync();
  double* srl = pub;  // the row scales, kept in the (not yet used) published-column buffer
  for (int a = tid; a < m; a += FP_THREADS) {
    const double mx = fmax(rmax[a], rmax[m + a]);
    srl[a] = (mx > 0.0) ? pow2_recip(mx) : 1.0;
    if (r == 0) {
      sr[a] = srl[a];
      if (mx == 0.0) atomicExch(status, DEV_SINGULAR);
    }
  }
  __syncthreads();
  // column scales of diag(s_r) K on my columns, then the scaled matrix
  double* scl = rmax;  // my columns' scales (the row maxima are no longer needed)
  for (int q = tid; q < mc; q += FP_THREADS) {
    double mx = 0.0;
    for (int a = 0; a < m; ++a) mx = fmax(mx, fabs(srl[a] * A[(int64_t)q * ld + a]));
    scl[q] = (mx > 0.0) ? pow2_recip(mx) : 1.0;
    sc[2 * q + r] = scl[q];
  }
  __syncthreads();
  for (int64_t e = tid; e < (int64_t)mc * m; e += FP_THREADS) {
    const int q = (int)(e / m), a = (int)(e % m);
    A[(int64_t)q * ld + a] = srl[a] * A[(int64_t)q * ld + a] * scl[q];
  }
  // both CTAs are done with the scales before the first column is published into pub
  cluster.sync();
  // column 0's pivot and the column itself, published by its owner (CTA 0)
  if (r == 0 && warp == 0) pair_pivot_publish(cluster, A, ld, m, 0, pub, perm, status);
  cluster.sync();
  for (int k = 0; k < m; ++k) {
    double* colk = pub + (k & 1) * m;
    const int pr = perm[k];
    // row interchange k <-> pr on my columns and in the published column
    if (pr != k && pr < m) {
      for (int q = tid; q < mc; q += FP_THREADS) {
        double* c = A + (int64_t)q * ld;
        const double t = c[k];
        c[k] = c[pr];
        c[pr] = t;
      }
      if (tid == 0) {
        const double t = colk[k];
        colk[k] = colk[pr];
        colk[pr] = t;
      }
    }
    __syncthreads();
    const double piv = colk[k];
    const double ipiv = (piv != 0.0) ? 1.0 / piv : 0.0;
    for (int q = tid; q < mc; q += FP_THREADS) {
      const int b = 2 * q + r;
      rowk[q] = (b == k) ? ipiv : A[(int64_t)q * ld + k] * ipiv;
    }
    __syncthreads();
    // lookahead: the owner of column k + 1 updates it first; warp 0 then finds its pivot and
    // publishes it while the other warps update the remaining columns
    const int kn = k + 1;
    const bool own_next = kn < m && (kn & 1) == r;
    const int qn = kn >> 1;
    if (own_next) {
      double* colp = A + (int64_t)qn * ld;
      const double rb = rowk[qn];
      for (int a = tid; a < m; a += FP_THREADS) colp[a] = (a == k) ? rb : colp[a] - colk[a] * rb;
      __syncthreads();
    }
    if (own_next && warp == 0) {
      pair_pivot_publish(cluster, A, ld, m, kn, pub, perm, status);
    } else {
      // rank-one update of my other columns: warps over columns, lanes over rows, the pivot
      // column's entries of this lane's rows held in registers
      double ck[FP_ROWS_PER_LANE];
#pragma unroll
      for (int i = 0; i < FP_ROWS_PER_LANE; ++i) {
        const int a = lane + 32 * i;
        ck[i] = (a < m) ? colk[a] : 0.0;
      }
      const int w0 = own_next ? warp - 1 : warp, nwu = own_next ? nw - 1 : nw;
      for (int q = w0; q < mc; q += nwu) {
        if (own_next && q == qn) continue;
        double* colp = A + (int64_t)q * ld;
        const double rb = rowk[q];
        if (2 * q + r == k) {
#pragma unroll
          for (int i = 0; i < FP_ROWS_PER_LANE; ++i) {
            const int a = lane + 32 * i;
            if (a < m) colp[a] = (a == k) ? rb : -ck[i] * ipiv;
          }
        } else {
#pragma unroll
          for (int i = 0; i < FP_ROWS_PER_LANE; ++i) {
            const int a = lane + 32 * i;
            if (a < m) colp[a] = (a == k) ? rb : colp[a] - ck[i] * rb;
          }
        }
      }
    }
    cluster.sync();  // the next pivot and column are published; this step's reads are done
  }
  // undo the row interchanges as column interchanges (last first): the column at position c
  // of the result is my column src[c] when src[c] is one of mine
  if (tid == 0) {
    for (int c = 0; c < m; ++c) src[c] = c;
    for (int k = m - 1; k >= 0; --k) {
      const int pr = perm[k];
      if (pr != k && pr < m) {
        const int t = src[k];
        src[k] = src[pr];
        src[pr] = t;
      }
    }
    for (int c = 0; c < m; ++c) dst[src[c]] = c;
  }
  __syncthreads();
  double* out = J.A + J.mat_off[p];
  for (int q = warp; q < mc; q += nw) {
    const int c = dst[2 * q + r];
    const double* colp = A + (int64_t)q * ld;
    for (int a = lane; a < m; a += 32) out[(int64_t)c * ld + a] = colp[a];
  }
  cluster.sync();  // no CTA exits while its peer may still write into its shared memory
}

// Fold the scalings: out[a][b] = s_c[a] X[a][b] s_r[b], row-major (m x m).
__global__ void k_fold_rowmajor(int m, const double* X, const double* s_r, const double* s_c, double* out) {
  const int ld = (m + 7) & ~7;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    const int a = e / m, b = e % m;
    out[e] = s_c[a] * X[(int64_t)b * ld + a] * s_r[b];
  }
}

template <typename T>
__global__ void k_downcast(int64_t n, const double* in, T* out);
template <>
__global__ void k_downcast<float>(int64_t n, const double* in, float* out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (float)in[e];
}
template <>
__global__ void k_downcast<__nv_bfloat16>(int64_t n, const double* in, __nv_bfloat16* out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = __double2bfloat16(in[e]);
}

// transpose incidence: slots of each unknown (pass 0 counts, pass 1 fills)
__global__ void k_incidence(int64_t n_slots, const int* dofs, int* count, const int64_t* off, int* cursor,
                            int* slot, int pass) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_slots) return;
  const int d = dofs[s];
  if (pass == 0) atomicAdd(&count[d], 1);
  else slot[off[d] + atomicAdd(&cursor[d], 1)] = (int)s;
}

__global__ void k_sort_lists2(int n, const int64_t* off, int* list) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n) return;
  const int64_t b = off[f], e = off[f + 1];
  for (int64_t i = b + 1; i < e; ++i) {
    const int v = list[i];
    int64_t j = i - 1;
    while (j >= b && list[j] > v) {
      list[j + 1] = list[j];
      --j;
    }
    list[j + 1] = v;
  }
}

// Copy each factorised patch's leading n x n block (ld = round8(n)) and first n scales into
// the packed storage used by the sweep.
__global__ void k_pack(const int64_t* off, const int64_t* mat_off, const int* mdim, const int64_t* inv_off,
                       const double* work, const double* wsr, const double* wsc, double* inv, double* s_r,
                       double* s_c) {
  const int p = blockIdx.x;
  const int64_t d0 = off[p];
  const int n = (int)(off[p + 1] - d0);
  const int m = mdim[p];
  const int lds = (m + 7) & ~7, ldd = (n + 7) & ~7;
  const double* src = work + mat_off[p];
  double* dst = inv + inv_off[p];
  for (int64_t e = threadIdx.x; e < (int64_t)n * ldd; e += blockDim.x) {
    const int b = (int)(e / ldd), a = (int)(e % ldd);
    dst[e] = (a < n) ? src[(int64_t)b * lds + a] : 0.0;
  }
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    s_r[d0 + a] = wsr[d0 + p + a];
    s_c[d0 + a] = wsc[d0 + p + a];
  }
}

// ------------------------------------------------------------------ driver

static LevelK level_k(const Level& lv) {
  LevelK k;
  k.N = lv.N;
  k.h = lv.h;
  k.rho_dt = lv.rho_dt;
  k.mu = lv.mu;
  k.dt = lv.dt;
  k.ih = 1.0 / lv.h;
  k.ih2 = 1.0 / (lv.h * lv.h);
  k.vdiag = lv.rho_dt - lv.mu * (-4.0 / (lv.h * lv.h));
  k.mh2 = lv.mu / (lv.h * lv.h);
  k.channel = lv.channel;
  k.row_of = lv.ee.row_of;
  k.rowptr = lv.ee.rowptr;
  k.cols = lv.ee.cols;
  k.vals = lv.ee.vals;
  return k;
}

static size_t factor_smem(int m) { return (size_t)(2 * m) * sizeof(double) + (size_t)m * sizeof(int) + 16; }

static void check_status(cav_hierarchy* H, cudaStream_t st, const char* where) {
  const int s = read_status(H->status, st);
  if (s != DEV_OK) {
    set_error(std::string(where) + ": " + status_message(s));
    throw Fail{status_of(s)};
  }
}

// ------------------------------------------------------------------ box patch sets

// B(b,o) patches (Sec. 3.1): the blocks in lexicographic order of their lower-left cells
// (I, J), i fastest; a block's patch holds every unknown of the cells (I + r, J + s),
// -o <= r, s <= b + o - 1 (periodic), ascending; inject marks the unknowns of the unexpanded
// block's cells (restricted injection, Sec. 3.3).  With b + 2 o < N no unknown repeats.
// Index arithmetic only, on the host.
static void box_sets(int N, int b, int o, std::vector<int>& cells, std::vector<int>& sizes, std::vector<int>& dofs,
                     std::vector<uint8_t>& inject) {
  const int NN = N * N;
  std::vector<std::pair<int, uint8_t>> buf;
  for (int J = 0; J < N; J += b)
    for (int I = 0; I < N; I += b) {
      buf.clear();
      // u faces (i, j) sit between cells (i - 1, j) and (i, j): columns -o .. b + o
      for (int s = -o; s < b + o; ++s)
        for (int r = -o; r <= b + o; ++r)
          buf.push_back({pmod(J + s, N) * N + pmod(I + r, N), (uint8_t)(r >= 0 && r <= b && s >= 0 && s < b)});
      // v faces (i, j) sit between cells (i, j - 1) and (i, j): rows -o .. b + o
      for (int s = -o; s <= b + o; ++s)
        for (int r = -o; r < b + o; ++r)
          buf.push_back({NN + pmod(J + s, N) * N + pmod(I + r, N), (uint8_t)(r >= 0 && r < b && s >= 0 && s <= b)});
      for (int s = -o; s < b + o; ++s)
        for (int r = -o; r < b + o; ++r)
          buf.push_back({2 * NN + pmod(J + s, N) * N + pmod(I + r, N), (uint8_t)(r >= 0 && r < b && s >= 0 && s < b)});
      std::sort(buf.begin(), buf.end());
      cells.push_back(J * N + I);
      sizes.push_back((int)buf.size());
      for (const auto& q : buf) {
        dofs.push_back(q.first);
        inject.push_back(q.second);
      }
    }
}

// The standard Vanka patches appended to a level's stored sets for factorisation, in
// canonical slot order (u_ij, u_i+1j, v_ij, v_ij+1, p_ij): one for a periodic level (cell
// (0, 0)), three for the channel (interior rows, the outflow row, the inflow row without
// v_{i,N}).
static void standard_patch_dofs(const Level& lv, std::vector<int>& std_dofs, std::vector<int>& std_len) {
  const int N = lv.N, NN = N * N;
  {
    auto cell = [&](int i, int j) {
      int ds[5] = {j * N + i, j * N + (i + 1) % N, NN + j * N + i, NN + ((j + 1) % N) * N + i, 2 * NN + j * N + i};
      const bool top = lv.channel && j + 1 == N;
      int len = 0;
      for (int t = 0; t < 5; ++t)
        if (!(top && t == 3)) std_dofs.push_back(ds[t]), ++len;
      std_len.push_back(len);
    };
    if (lv.channel) {
      cell(0, 1);      // interior rows
      cell(0, 0);      // outflow row
      cell(0, N - 1);  // inflow row (no v_{i,N})
    } else {
      cell(0, 0);
    }
  }
}

// The numerical part of a smoothing level's set-up: extract every stored patch's local matrix
// from the level's current K_E, equilibrate, invert (batched Gauss-Jordan, FP64), pack, and
// store in the level's precision; with `standard`, also the standard patches' shared
// inverses (E_E-free, so they do not change when only E_E's values do).  The structure (sets,
// offsets, incidence, classes) must already be in place; buffers are allocated on the first
// call and reused by later ones (cav_refactor), so graphs captured on them stay valid.
static void factor_patches(cav_hierarchy* H, Level& lv, bool standard, cudaStream_t st) {
  Arena& A = H->arena;
  Arena scratch;
  const int64_t nbig = lv.n_big;
  const std::vector<int>& hsizes = lv.host_sizes;
  const int64_t sum_n = lv.big_sum_n, inv_elems = lv.inv_elems;
  const int max_n = lv.big_max_n;
  const LevelK LK = level_k(lv);
  std::vector<int> std_dofs, std_len;
  standard_patch_dofs(lv, std_dofs, std_len);
  // 3. factorise the enlarged patches, then the standard Vanka patch(es) (jobs nbig ..) in
  //    canonical slot order (u_ij, u_i+1j, v_ij, v_ij+1, p_ij; the inflow row without v_ij+1)
  //    without E_E.
  CAV_CHECK_CUDA(cudaMemcpyAsync(lv.big_dofs + sum_n, std_dofs.data(), sizeof(int) * std_dofs.size(),
                                 cudaMemcpyHostToDevice, st));
  const int n_std = standard ? (int)std_len.size() : 0;
  const int njobs = (int)nbig + n_std;
  std::vector<int64_t> hoff_ext(njobs + 1);
  hoff_ext[0] = 0;
  for (int p = 0; p < njobs; ++p) hoff_ext[p + 1] = hoff_ext[p] + (p < nbig ? hsizes[p] : std_len[p - nbig]);
  std::vector<int64_t> hmat_off(njobs + 1, 0);
  for (int p = 0; p < njobs; ++p) {
    const int m = (p < nbig) ? hsizes[p] : std_len[p - nbig];
    // a patch holding every pressure of a periodic level gets one border row and column
    hmat_off[p + 1] = hmat_off[p] + (int64_t)round8(m + 1) * (m + 1);
  }
  int64_t* d_off_ext = scratch.alloc<int64_t>(njobs + 1);
  int64_t* d_mat_off = scratch.alloc<int64_t>(njobs + 1);
  CAV_CHECK_CUDA(cudaMemcpyAsync(d_off_ext, hoff_ext.data(), sizeof(int64_t) * (njobs + 1), cudaMemcpyHostToDevice, st));
  CAV_CHECK_CUDA(cudaMemcpyAsync(d_mat_off, hmat_off.data(), sizeof(int64_t) * (njobs + 1), cudaMemcpyHostToDevice, st));
  double* work = scratch.alloc<double>(hmat_off[njobs]);
  double* wsr = scratch.alloc<double>(hoff_ext[njobs] + njobs + 8);
  double* wsc = scratch.alloc<double>(hoff_ext[njobs] + njobs + 8);
  int* mdim = scratch.alloc<int>(njobs + 1);
  FactorJob J;
  J.jobs = nullptr;
  J.mdim = mdim;
  J.dof_off = d_off_ext;
  J.dofs = lv.big_dofs;
  J.mat_off = d_mat_off;
  J.A = work;
  J.s_r = wsr;
  J.s_c = wsc;
  J.border_all_pressure = lv.channel ? 0 : 1;  // the channel's pressure is determined
  J.use_ee = 1;
  const int mmax = std::max(max_n, 5) + 1;
  const size_t fsm = factor_smem(mmax);
  if (fsm > 48 * 1024)
    CAV_CHECK_CUDA(cudaFuncSetAttribute(k_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm));
  if (nbig > 0) {
    // patches of FP_MMIN .. FP_MMAX unknowns (with a possible border) on CTA pairs with the
    // matrix in shared memory; the others one CTA each in global memory.  CAV_FACTOR_GLOBAL=1 sends
    // every patch to the global-memory kernel (a test hook: both give the same bits).
    const char* force_global = std::getenv("CAV_FACTOR_GLOBAL");
    const bool pairs_on = !(force_global && force_global[0] == '1');
    std::vector<int> pair_jobs, glob_jobs;
    int pair_mmax = 0;
    for (int p = 0; p < (int)nbig; ++p) {
      if (pairs_on && hsizes[p] >= FP_MMIN && hsizes[p] + 1 <= FP_MMAX) {
        pair_jobs.push_back(p);
        pair_mmax = std::max(pair_mmax, hsizes[p] + 1);
      } else {
        glob_jobs.push_back(p);
      }
    }
    if (!pair_jobs.empty()) {
      // largest first (the block scheduler issues CTAs in order); the patches whose matrices
      // leave room for two CTAs per SM (m <= m2) in a launch of their own
      std::stable_sort(pair_jobs.begin(), pair_jobs.end(), [&](int a, int b) { return hsizes[a] > hsizes[b]; });
      int dev = 0, smem_sm = 0;
      CAV_CHECK_CUDA(cudaGetDevice(&dev));
      CAV_CHECK_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
      int m2 = pair_mmax;
      while (m2 > FP_MMIN && 2 * (factor_pair_smem(m2) + 2048) > (size_t)smem_sm) --m2;
      const int nl = (int)(std::find_if(pair_jobs.begin(), pair_jobs.end(),
                                        [&](int p) { return hsizes[p] + 1 <= m2; }) - pair_jobs.begin());
      int* d_jobs = scratch.alloc<int>(pair_jobs.size());
      CAV_CHECK_CUDA(cudaMemcpyAsync(d_jobs, pair_jobs.data(), sizeof(int) * pair_jobs.size(), cudaMemcpyHostToDevice,
                                     st));
      const size_t psm = factor_pair_smem(pair_mmax);
      CAV_CHECK_CUDA(cudaFuncSetAttribute(k_factor_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
      if (nl > 0) {
        k_factor_pair<<<2 * nl, FP_THREADS, psm, st>>>(LK, J, d_jobs, H->status);
        CAV_CHECK_LAUNCH();
      }
      if (nl < (int)pair_jobs.size()) {
        k_factor_pair<<<2 * ((int)pair_jobs.size() - nl), FP_THREADS, factor_pair_smem(m2), st>>>(LK, J, d_jobs + nl,
                                                                                                   H->status);
        CAV_CHECK_LAUNCH();
      }
    }
    if (!glob_jobs.empty()) {
      FactorJob Jg = J;
      if ((int)glob_jobs.size() < (int)nbig) {
        int* d_jobs = scratch.alloc<int>(glob_jobs.size());
        CAV_CHECK_CUDA(cudaMemcpyAsync(d_jobs, glob_jobs.data(), sizeof(int) * glob_jobs.size(),
                                       cudaMemcpyHostToDevice, st));
        Jg.jobs = d_jobs;
      }
      k_factor<<<(int)glob_jobs.size(), 256, fsm, st>>>(LK, Jg, 0, H->status);
      CAV_CHECK_LAUNCH();
    }
  }
  // the standard patches: same kernel, one block each, no E_E
  if (standard) {
    FactorJob Js = J;
    Js.dof_off = d_off_ext + nbig;
    Js.mat_off = d_mat_off + nbig;
    Js.mdim = mdim + nbig;
    Js.s_r = wsr + nbig;  // scale slots of job p start at dof_off[p] + p
    Js.s_c = wsc + nbig;
    Js.use_ee = 0;
    Js.border_all_pressure = 0;
    k_factor<<<n_std, 64, factor_smem(6), st>>>(LK, Js, 0, H->status);
    CAV_CHECK_LAUNCH();
    double* d_std = scratch.alloc<double>(25 * n_std);
    for (int q = 0; q < n_std; ++q) {
      const int p = (int)nbig + q;
      k_fold_rowmajor<<<1, 32, 0, st>>>(std_len[q], work + hmat_off[p], wsr + hoff_ext[p] + p, wsc + hoff_ext[p] + p,
                                        d_std + 25 * q);
      CAV_CHECK_LAUNCH();
    }
    std::vector<double> hstd(25 * n_std);
    CAV_CHECK_CUDA(cudaMemcpyAsync(hstd.data(), d_std, sizeof(double) * 25 * n_std, cudaMemcpyDeviceToHost, st));
    CAV_CHECK_CUDA(cudaStreamSynchronize(st));
    // kind 0 interior (or every periodic cell), 1 outflow row, 2 inflow row: the inflow row's
    // 4 x 4 inverse goes to slots (0, 1, 2, 4) with slot 3 (v_ij+1) left zero
    for (int k = 0; k < 3; ++k)
      for (int q = 0; q < 25; ++q) lv.std_inv[k][q] = 0.0;
    for (int q = 0; q < n_std; ++q) {
      const int m = std_len[q];
      int slot[5] = {0, 1, 2, 3, 4};
      if (m == 4) slot[3] = 4;
      for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) lv.std_inv[q][slot[a] * 5 + slot[b]] = hstd[25 * q + a * m + b];
    }
    if (n_std == 1)
      for (int k = 1; k < 3; ++k)
        for (int q = 0; q < 25; ++q) lv.std_inv[k][q] = lv.std_inv[0][q];
  }
  check_status(H, st, "patch factorisation");
  // 4. pack the inverses (ld = round8(n), column-major) and scales; bordered patches are
  //    applied with their border slot's residual entry equal to zero, so only the leading
  //    n x n block and the first n scales are needed.
  if (!lv.s_r) {
    lv.s_r = A.alloc<double>(sum_n);
    lv.s_c = A.alloc<double>(sum_n);
    lv.inv64 = A.alloc<double>(std::max<int64_t>(inv_elems, 1));
  }
  if (nbig > 0) {
    k_pack<<<(int)nbig, 256, 0, st>>>(lv.big_off, d_mat_off, mdim, lv.inv_off, work, wsr, wsc, lv.inv64,
                                      lv.s_r, lv.s_c);
    CAV_CHECK_LAUNCH();
  }
  lv.precision = H->desc.precision;
  if (lv.precision == CAV_PREC_FP32) {
    if (!lv.inv32) lv.inv32 = A.alloc<float>(std::max<int64_t>(inv_elems, 1));
    k_downcast<float><<<1184, 256, 0, st>>>(inv_elems, lv.inv64, lv.inv32);
    CAV_CHECK_LAUNCH();
  } else if (lv.precision == CAV_PREC_BF16) {
    if (!lv.inv16) lv.inv16 = A.alloc<__nv_bfloat16>(std::max<int64_t>(inv_elems, 1));
    k_downcast<__nv_bfloat16><<<1184, 256, 0, st>>>(inv_elems, lv.inv64, lv.inv16);
    CAV_CHECK_LAUNCH();
  }
  CAV_CHECK_CUDA(cudaStreamSynchronize(st));
  scratch.release();
}

static void build_smoother(cav_hierarchy* H, Level& lv, cudaStream_t st) {
  Arena& A = H->arena;
  Arena scratch;
  const int N = lv.N, NN = N * N;
  const LevelK LK = level_k(lv);
  lv.cell_big = A.alloc<uint8_t>(NN);
  int64_t nbig = 0;
  std::vector<int> hsizes;
  std::vector<int> box_dofs;
  int cav_set_warps = 1;
  size_t cav_set_smem = 0;
  if (lv.box) {
    // 1-2. box patches: every one is enlarged, no cell keeps a standard patch
    std::vector<int> cells;
    std::vector<uint8_t> inj;
    box_sets(N, H->desc.box_b, H->desc.box_o, cells, hsizes, box_dofs, inj);
    nbig = (int64_t)cells.size();
    lv.n_big = (int)nbig;
    std::vector<int64_t> off(nbig + 1, 0);
    for (int64_t p = 0; p < nbig; ++p) off[p + 1] = off[p] + hsizes[p];
    lv.big_cell = A.alloc<int>(nbig);
    lv.big_off = A.alloc<int64_t>(nbig + 1);
    lv.inject = A.alloc<uint8_t>(box_dofs.size());
    CAV_CHECK_CUDA(cudaMemsetAsync(lv.cell_big, 0, NN, st));
    CAV_CHECK_CUDA(cudaMemcpyAsync(lv.big_cell, cells.data(), sizeof(int) * nbig, cudaMemcpyHostToDevice, st));
    CAV_CHECK_CUDA(cudaMemcpyAsync(lv.big_off, off.data(), sizeof(int64_t) * (nbig + 1), cudaMemcpyHostToDevice, st));
    CAV_CHECK_CUDA(cudaMemcpyAsync(lv.inject, inj.data(), inj.size(), cudaMemcpyHostToDevice, st));
    CAV_CHECK_CUDA(cudaStreamSynchronize(st));
  } else {
    // 1. enlarged cells
    int* flag = scratch.alloc<int>(NN);
    int64_t* pos = scratch.alloc<int64_t>(NN + 1);
    k_cell_flags<<<div_up(NN, 256), 256, 0, st>>>(N, H->desc.kind == CAV_PATCH_CAV ? 1 : 0, lv.ee.row_of,
                                                 lv.ee.rowptr, lv.ee.cols, lv.cell_big, flag, lv.channel);
    CAV_CHECK_LAUNCH();
    exclusive_scan(flag, pos, NN, st, &scratch);
    CAV_CHECK_CUDA(cudaMemcpyAsync(&nbig, pos + NN, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CAV_CHECK_CUDA(cudaStreamSynchronize(st));
    lv.n_big = (int)nbig;
    lv.big_cell = A.alloc<int>(nbig);
    k_compact_cells<<<div_up(NN, 256), 256, 0, st>>>(NN, flag, pos, lv.big_cell);
    CAV_CHECK_LAUNCH();
    // 2. CAV patch sets (count, scan; the write follows below)
    const int W = lv.ee.W;
    const int Wc = W + 2, Wd = W + 3;
    const int lenC = (2 * Wc + 1 >= N) ? N : 2 * Wc + 1;
    const int lenD = (2 * Wd + 1 >= N) ? N : 2 * Wd + 1;
    const int per_warp = lenC * lenC + 3 * lenD * lenD;
    int warps = 8;
    while (warps > 1 && (size_t)warps * per_warp > 96 * 1024) warps >>= 1;
    const size_t smem = (size_t)warps * per_warp;
    CAV_REQUIRE(smem <= 200 * 1024, "CAV patch window too large");
    if (smem > 48 * 1024)
      CAV_CHECK_CUDA(cudaFuncSetAttribute(k_cav_sets, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cav_set_warps = warps;
    cav_set_smem = smem;
    int* sizes = scratch.alloc<int>(nbig + 1);
    lv.big_off = A.alloc<int64_t>(nbig + 1);
    if (nbig > 0) {
      k_cav_sets<<<div_up(nbig, warps), warps * 32, smem, st>>>(N, W, (int)nbig, lv.big_cell, lv.ee.row_of,
                                                                lv.ee.rowptr, lv.ee.cols, sizes, nullptr,
                                                                nullptr, 0, H->status, lv.channel,
                                                                H->desc.kind == CAV_PATCH_CAV);
      CAV_CHECK_LAUNCH();
    }
    exclusive_scan(sizes, lv.big_off, nbig, st, &scratch);
    hsizes.resize(nbig);
    if (nbig > 0)
      CAV_CHECK_CUDA(cudaMemcpyAsync(hsizes.data(), sizes, sizeof(int) * nbig, cudaMemcpyDeviceToHost, st));
    CAV_CHECK_CUDA(cudaStreamSynchronize(st));
  }
  int64_t sum_n = 0, sum_n2 = 0;
  int max_n = 0;
  std::vector<int64_t> hinv_off(nbig + 1, 0);
  for (int64_t p = 0; p < nbig; ++p) {
    const int n = hsizes[p];
    sum_n += n;
    sum_n2 += (int64_t)n * n;
    max_n = std::max(max_n, n);
    hinv_off[p + 1] = hinv_off[p] + (int64_t)round8(n) * n;
  }
  lv.big_sum_n = sum_n;
  lv.big_sum_n2 = sum_n2;
  lv.n_big_small = 0;
  for (int64_t p = 0; p < nbig; ++p) lv.n_big_small += (hsizes[p] <= 5 && !lv.box) ? 1 : 0;
  lv.big_max_n = max_n;
  lv.inv_elems = hinv_off[nbig];
  // the standard patches are appended to the stored sets for factorisation
  std::vector<int> std_dofs, std_len;
  standard_patch_dofs(lv, std_dofs, std_len);
  const int n_std = (int)std_len.size();
  lv.big_dofs = A.alloc<int>(sum_n + (int64_t)std_dofs.size());
  if (lv.box) {
    if (sum_n > 0)
      CAV_CHECK_CUDA(cudaMemcpyAsync(lv.big_dofs, box_dofs.data(), sizeof(int) * sum_n, cudaMemcpyHostToDevice, st));
  } else if (nbig > 0) {
    k_cav_sets<<<div_up(nbig, cav_set_warps), cav_set_warps * 32, cav_set_smem, st>>>(
        N, lv.ee.W, (int)nbig, lv.big_cell, lv.ee.row_of, lv.ee.rowptr, lv.ee.cols, nullptr, lv.big_off,
        lv.big_dofs, 1, H->status, lv.channel, H->desc.kind == CAV_PATCH_CAV);
    CAV_CHECK_LAUNCH();
  }
  check_status(H, st, "patch sets");
  // launch order: descending size
  std::vector<int> order(nbig);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hsizes[a] > hsizes[b]; });
  lv.order = A.alloc<int>(nbig);
  lv.inv_off = A.alloc<int64_t>(nbig + 1);
  if (nbig > 0) {
    CAV_CHECK_CUDA(cudaMemcpyAsync(lv.order, order.data(), sizeof(int) * nbig, cudaMemcpyHostToDevice, st));
  }
  CAV_CHECK_CUDA(cudaMemcpyAsync(lv.inv_off, hinv_off.data(), sizeof(int64_t) * (nbig + 1),
                                 cudaMemcpyHostToDevice, st));
  // 3-4. factorise and store the inverses (also the standard patches')
  lv.host_sizes = hsizes;
  build_schedules(H, lv, st);
  factor_patches(H, lv, true, st);
  // 5. transpose incidence of the packed slots
  int* cnt = scratch.alloc<int>(3 * NN);
  int* cur = scratch.alloc<int>(3 * NN);
  CAV_CHECK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * 3 * NN, st));
  CAV_CHECK_CUDA(cudaMemsetAsync(cur, 0, sizeof(int) * 3 * NN, st));
  lv.inc_off = A.alloc<int64_t>(3 * NN + 1);
  lv.inc_slot = A.alloc<int>(sum_n);
  if (sum_n > 0) {
    k_incidence<<<div_up(sum_n, 256), 256, 0, st>>>(sum_n, lv.big_dofs, cnt, nullptr, nullptr, nullptr, 0);
    CAV_CHECK_LAUNCH();
  }
  exclusive_scan(cnt, lv.inc_off, 3 * NN, st, &scratch);
  if (sum_n > 0) {
    k_incidence<<<div_up(sum_n, 256), 256, 0, st>>>(sum_n, lv.big_dofs, cnt, lv.inc_off, cur, lv.inc_slot, 1);
    CAV_CHECK_LAUNCH();
    k_sort_lists2<<<div_up(3 * NN, 256), 256, 0, st>>>(3 * NN, lv.inc_off, lv.inc_slot);
    CAV_CHECK_LAUNCH();
  }
  // unknowns held by at least one enlarged patch (ascending), for the warp-per-unknown scatter
  {
    int* tflag = scratch.alloc<int>(3 * NN);
    int64_t* tpos = scratch.alloc<int64_t>(3 * NN + 1);
    k_flag_nonempty_off<<<div_up(3 * NN, 256), 256, 0, st>>>(3 * NN, lv.inc_off, tflag);
    CAV_CHECK_LAUNCH();
    exclusive_scan(tflag, tpos, 3 * NN, st, &scratch);
    int64_t nt = 0;
    CAV_CHECK_CUDA(cudaMemcpyAsync(&nt, tpos + 3 * NN, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CAV_CHECK_CUDA(cudaStreamSynchronize(st));
    lv.n_touched = (int)nt;
    lv.touched = A.alloc<int>(nt);
    k_compact_cells<<<div_up(3 * NN, 256), 256, 0, st>>>(3 * NN, tflag, tpos, lv.touched);
    CAV_CHECK_LAUNCH();
  }
  build_touch_theta(H, lv, st);
  if (lv.channel && !lv.box) {  // standard patches of the inflow row have four unknowns
    std::vector<uint8_t> top(N);
    CAV_CHECK_CUDA(cudaMemcpyAsync(top.data(), lv.cell_big + (size_t)(N - 1) * N, N, cudaMemcpyDeviceToHost, st));
    CAV_CHECK_CUDA(cudaStreamSynchronize(st));
    lv.n_std4 = 0;
    for (int i = 0; i < N; ++i) lv.n_std4 += top[i] ? 0 : 1;
  }
  lv.n_partial_std = div_up(N, 32) * div_up(N, 8);
  lv.n_partial = lv.n_partial_std + div_up(lv.n_touched, SCATTER_TOUCHED_PER_BLOCK);  // then the touched blocks
  lv.partial = A.alloc<double>(lv.n_partial);
  lv.wpart = A.alloc<double>(8 * (size_t)lv.n_partial);
  lv.delta = A.alloc<double>(std::max<int64_t>(sum_n, 1));
  CAV_CHECK_CUDA(cudaStreamSynchronize(st));
  scratch.release();
}

// coarsest systems above this order are factorised by the grid-parallel kernel
constexpr int COARSEST_GRID_M = 256;

// Enqueues the coarsest system's factorisation on st (no sync): its buffers come from scratch,
// which the caller releases after checking the status.
static void build_coarsest(cav_hierarchy* H, Level& lv, cudaStream_t st, Arena& scratch) {
  Arena& A = H->arena;
  // periodic: bordered by the pressure-mean constraint; channel: the plain operator
  const int N = lv.N, NN = N * N, n = 3 * NN, m = lv.channel ? n : n + 1;
  const LevelK LK = level_k(lv);
  std::vector<int> all(n);
  std::iota(all.begin(), all.end(), 0);
  int* d_dofs = scratch.alloc<int>(n);
  CAV_CHECK_CUDA(cudaMemcpyAsync(d_dofs, all.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  int64_t hoff[2] = {0, n};
  int64_t hmo[2] = {0, (int64_t)round8(m) * m};
  int64_t* d_off = scratch.alloc<int64_t>(2);
  int64_t* d_mo = scratch.alloc<int64_t>(2);
  CAV_CHECK_CUDA(cudaMemcpyAsync(d_off, hoff, sizeof(hoff), cudaMemcpyHostToDevice, st));
  CAV_CHECK_CUDA(cudaMemcpyAsync(d_mo, hmo, sizeof(hmo), cudaMemcpyHostToDevice, st));
  double* work = scratch.alloc<double>(hmo[1]);
  double* wsr = scratch.alloc<double>(m);
  double* wsc = scratch.alloc<double>(m);
  int* mdim = scratch.alloc<int>(1);
  FactorJob J;
  J.jobs = nullptr;
  J.mdim = mdim;
  J.dof_off = d_off;
  J.dofs = d_dofs;
  J.mat_off = d_mo;
  J.A = work;
  J.s_r = wsr;
  J.s_c = wsc;
  J.border_all_pressure = 0;
  J.use_ee = 1;
  if (m > COARSEST_GRID_M && !std::getenv("CAV_COARSEST_ONE_CTA")) {
    // a larger coarsest level: the factorisation on every SM, blocked in panels where the panel
    // fits in shared memory, else column by column (both give the one-CTA kernel's bits; the
    // test hooks CAV_COARSEST_ONE_CTA and CAV_COARSEST_COLUMNS select the other forms)
    int sms = 0, dev = 0, per_sm = 0, optin = 0;
    CAV_CHECK_CUDA(cudaGetDevice(&dev));
    CAV_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CAV_CHECK_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int bordered = lv.channel ? 0 : 1;
    const size_t col_bytes = sizeof(double) * (size_t)round8(m);
    int* perm = scratch.alloc<int>(m);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(sms);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: the grid barriers need it
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    constexpr int GP_R = 7;  // register rows per thread of the panel kernel
    cudaFuncAttributes pa;
    CAV_CHECK_CUDA(cudaFuncGetAttributes(&pa, k_factor_panels<GP_R>));
    const size_t psm = (GP_PB + 1) * col_bytes;
    const bool panels = !std::getenv("CAV_COARSEST_COLUMNS") && m <= GP_R * GP_THREADS && sms >= 2 &&
                        psm + pa.sharedSizeBytes <= (size_t)optin;
    if (panels) {
      CAV_CHECK_CUDA(cudaFuncSetAttribute(k_factor_panels<GP_R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
      CAV_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_factor_panels<GP_R>, GP_THREADS, psm));
      CAV_REQUIRE(per_sm >= 1, "coarsest factorisation: the panel kernel cannot be resident");
      double* cpan = scratch.alloc<double>(2 * (size_t)GP_PB * round8(m));
      int* ppiv = scratch.alloc<int>(2 * GP_PB);
      cfg.blockDim = dim3(GP_THREADS);
      cfg.dynamicSmemBytes = psm;
      CAV_CHECK_CUDA(cudaLaunchKernelEx(&cfg, k_factor_panels<GP_R>, LK, J, bordered, H->status, H->gbar, cpan, ppiv,
                                        perm));
      CAV_CHECK_LAUNCH();
    } else {
      // rb and the moved entries per own column, then as many whole own columns as fit
      cudaFuncAttributes fa;
      CAV_CHECK_CUDA(cudaFuncGetAttributes(&fa, k_factor_grid));
      const int ncol_max = (m + sms - 1) / sms;
      const size_t base = 2 * sizeof(double) * (size_t)ncol_max;
      const size_t room = (size_t)optin - fa.sharedSizeBytes;
      const int sc_cols = room > base ? (int)std::min<size_t>((room - base) / col_bytes, (size_t)ncol_max) : 0;
      const size_t gsm = base + (size_t)sc_cols * col_bytes;
      CAV_CHECK_CUDA(cudaFuncSetAttribute(k_factor_grid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm));
      CAV_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_factor_grid, FG_THREADS, gsm));
      CAV_REQUIRE(per_sm >= 1, "coarsest factorisation: the grid kernel cannot be resident");
      double* pub_col = scratch.alloc<double>(2 * (size_t)round8(m));
      int* pub_piv = scratch.alloc<int>(2);
      cfg.blockDim = dim3(FG_THREADS);
      cfg.dynamicSmemBytes = gsm;
      CAV_CHECK_CUDA(cudaLaunchKernelEx(&cfg, k_factor_grid, LK, J, bordered, H->status, H->gbar, pub_col, pub_piv,
                                        perm, sc_cols));
      CAV_CHECK_LAUNCH();
    }
  } else {
    const size_t fsm = factor_smem(m);
    if (fsm > 48 * 1024)
      CAV_CHECK_CUDA(cudaFuncSetAttribute(k_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm));
    k_factor<<<1, 1024, fsm, st>>>(LK, J, lv.channel ? 0 : 1, H->status);
    CAV_CHECK_LAUNCH();
  }
  lv.coarse_m = m;
  if (!lv.coarse_inv) lv.coarse_inv = A.alloc<double>((size_t)m * m);  // reused by cav_refactor
  k_fold_rowmajor<<<64, 256, 0, st>>>(m, work, wsr, wsc, lv.coarse_inv);
  CAV_CHECK_LAUNCH();
}

void build_levels(cav_hierarchy* H, cudaStream_t st) {
  const ib_system* s = H->sys;
  Arena& A = H->arena;
  std::vector<int> sizes{s->N};
  while (sizes.back() / 2 >= H->desc.coarsest_N && sizes.back() % 2 == 0) sizes.push_back(sizes.back() / 2);
  CAV_REQUIRE(sizes.size() >= 2, "the grid cannot be coarsened to coarsest_N (need N >= 2 coarsest_N)");
  H->levels.resize(sizes.size());
  int* d_scr = A.alloc<int>(1);
  for (size_t l = 0; l < sizes.size(); ++l) {
    Level& lv = H->levels[l];
    lv.N = sizes[l];
    lv.h = s->L / lv.N;
    lv.rho_dt = s->rho / s->dt;
    lv.mu = s->mu;
    lv.dt = s->dt;
    lv.channel = s->bc == IB_BC_CHANNEL;
    lv.coarsest = (l + 1 == sizes.size());
    const cav_desc& d = H->desc;
    lv.coloured = !lv.coarsest && d.smoother == CAV_SMOOTH_COLOURED &&
                  (d.coloured_levels <= 0 || (int)l < d.coloured_levels);
    lv.box = !lv.coarsest && d.kind == CAV_PATCH_BOX;
    if (lv.box)
      CAV_REQUIRE(lv.N % d.box_b == 0 && d.box_b + 2 * d.box_o < lv.N,
                  "cav_setup: box patches B(b,o) need every smoothing level's N divisible by b and b + 2 o < N");
    const bool nu_add = d.smoother == CAV_SMOOTH_COLOURED && !lv.coloured && d.nu_additive > 0;
    lv.nu_pre = nu_add ? d.nu_additive : d.nu_pre;
    lv.nu_post = nu_add ? d.nu_additive : d.nu_post;
    if (l == 0) {
      // the hierarchy's own copy: ib_update_structure may replace the system's E_E later
      lv.ee = s->ee;
      lv.ee.rows = A.alloc<int>(std::max(s->ee.n_rows, 1));
      lv.ee.rowptr = A.alloc<int64_t>(s->ee.n_rows + 1);
      lv.ee.cols = A.alloc<int>(std::max<int64_t>(s->ee.nnz, 1));
      lv.ee.vals = A.alloc<double>(std::max<int64_t>(s->ee.nnz, 1));
      lv.ee.row_of = A.alloc<int>(2 * (size_t)lv.N * lv.N);
      if (s->ee.n_rows) {
        CAV_CHECK_CUDA(cudaMemcpyAsync(lv.ee.rows, s->ee.rows, sizeof(int) * s->ee.n_rows, cudaMemcpyDeviceToDevice, st));
        CAV_CHECK_CUDA(cudaMemcpyAsync(lv.ee.cols, s->ee.cols, sizeof(int) * s->ee.nnz, cudaMemcpyDeviceToDevice, st));
        CAV_CHECK_CUDA(cudaMemcpyAsync(lv.ee.vals, s->ee.vals, sizeof(double) * s->ee.nnz, cudaMemcpyDeviceToDevice, st));
      }
      CAV_CHECK_CUDA(cudaMemcpyAsync(lv.ee.rowptr, s->ee.rowptr, sizeof(int64_t) * (s->ee.n_rows + 1),
                                     cudaMemcpyDeviceToDevice, st));
      CAV_CHECK_CUDA(cudaMemcpyAsync(lv.ee.row_of, s->ee.row_of, sizeof(int) * 2 * (size_t)lv.N * lv.N,
                                     cudaMemcpyDeviceToDevice, st));
    } else {
      galerkin_level(H->levels[l - 1].ee, lv.N, lv.ee, A, d_scr, lv.channel, st);
    }
    const int NN = lv.N * lv.N;
    lv.r = A.alloc<double>(3 * NN);
    if (!lv.coarsest && d.precision != CAV_PREC_FP64) lv.r32 = A.alloc<float>(3 * NN);
    lv.x = A.alloc<double>(3 * NN);
    lv.b = A.alloc<double>(3 * NN);
  }
  {
    // the coarsest factorisation is enqueued before the host computes the coloured levels'
    // classes, so the two overlap; its scratch is released once the stream has passed it
    std::vector<ColourPlan> plans(sizes.size());
    Arena coarse_scratch;
    try {
      for (size_t l = 0; l < sizes.size(); ++l) {
        Level& lv = H->levels[l];
        if (lv.coarsest) continue;
        build_smoother(H, lv, st);
        if (lv.coloured) colour_fetch(lv, plans[l], st);
      }
      build_coarsest(H, H->levels.back(), st, coarse_scratch);
      for (size_t l = 0; l < sizes.size(); ++l)
        if (H->levels[l].coloured) colour_plan(H->levels[l], plans[l]);
      check_status(H, st, "coarsest factorisation");
      coarse_scratch.release();
    } catch (...) {
      cudaStreamSynchronize(st);
      coarse_scratch.release();
      throw;
    }
    for (size_t l = 0; l < sizes.size(); ++l)
      if (H->levels[l].coloured) colour_upload(H, H->levels[l], plans[l], st);
  }
  if (H->desc.autotune)
    for (auto& lv : H->levels)
      if (!lv.coarsest && !lv.coloured) autotune_level(H, lv, st);
  // the sweep's form: timed with the autotuner, else separate kernels; CAV_SWEEP_FORM=fused
  // or =separate (a test hook) forces one form (both give the same bits)
  const char* form = std::getenv("CAV_SWEEP_FORM");
  const int force = (form && std::string(form) == "fused") ? 1
                    : (form && std::string(form) == "separate") ? -1 : (H->desc.autotune ? 0 : -1);
  for (auto& lv : H->levels)
    if (!lv.coarsest && !lv.coloured) choose_sweep_form(H, lv, force, st);
  CAV_CHECK_CUDA(cudaStreamSynchronize(st));
  check_status(H, st, "autotune");
  // capture both V-cycle graph instances now, so no solve pays for it
  vcycle_prepare(H);
  if (H->desc.krylov_capacity > 0)
    krylov_reserve(H, H->desc.krylov_capacity, 3LL * H->levels[0].N * H->levels[0].N);
}

// ------------------------------------------------------------------ refactorisation

// 1 in *flag if a[0..n) and b[0..n) differ anywhere
__global__ void k_differ32(int64_t n, const int* __restrict__ a, const int* __restrict__ b, int* flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (a[i] != b[i]) atomicExch(flag, 1);
}
__global__ void k_differ64(int64_t n, const int64_t* __restrict__ a, const int64_t* __restrict__ b, int* flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (a[i] != b[i]) atomicExch(flag, 1);
}

bool same_ee_pattern(const EECsr& a, const EECsr& b, int* d_flag, cudaStream_t st) {
  if (a.n_rows != b.n_rows || a.nnz != b.nnz || a.cross != b.cross) return false;
  if (a.n_rows == 0) return true;
  CAV_CHECK_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), st));
  k_differ32<<<div_up(a.n_rows, 256) < 1184 ? div_up(a.n_rows, 256) : 1184, 256, 0, st>>>(a.n_rows, a.rows, b.rows,
                                                                                         d_flag);
  CAV_CHECK_LAUNCH();
  k_differ64<<<div_up(a.n_rows + 1, 256) < 1184 ? div_up(a.n_rows + 1, 256) : 1184, 256, 0, st>>>(
      a.n_rows + 1, a.rowptr, b.rowptr, d_flag);
  CAV_CHECK_LAUNCH();
  if (a.nnz) {
    k_differ32<<<div_up(a.nnz, 256) < 1184 ? div_up(a.nnz, 256) : 1184, 256, 0, st>>>(a.nnz, a.cols, b.cols, d_flag);
    CAV_CHECK_LAUNCH();
  }
  return read_status(d_flag, st) == 0;
}

void refactor_levels(cav_hierarchy* H, const ib_system* s, cudaStream_t st) {
  Level& l0 = H->levels[0];
  if (s->ee.nnz)
    CAV_CHECK_CUDA(cudaMemcpyAsync(l0.ee.vals, s->ee.vals, sizeof(double) * s->ee.nnz, cudaMemcpyDeviceToDevice, st));
  for (size_t l = 1; l < H->levels.size(); ++l)
    galerkin_values(H->levels[l - 1].ee, H->levels[l].N, H->levels[l].ee, H->levels[l].channel, st);
  Arena coarse_scratch;
  try {
    for (auto& lv : H->levels) {
      if (lv.coarsest) {
        build_coarsest(H, lv, st, coarse_scratch);
        continue;
      }
      factor_patches(H, lv, false, st);
      if (lv.coloured) colour_refresh_values(lv, st);
    }
    CAV_CHECK_CUDA(cudaStreamSynchronize(st));
    check_status(H, st, "refactorisation");
  } catch (...) {
    cudaStreamSynchronize(st);
    coarse_scratch.release();
    throw;
  }
  coarse_scratch.release();
  H->sys = s;
}

}  // namespace cav
