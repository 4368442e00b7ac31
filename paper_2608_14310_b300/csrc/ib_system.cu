// Lagrangian markers, the four-point kernel supports of S and J, the force matrix E, and the
// assembly of the Eulerian elasticity matrix E_E = S E J (Sec. 2, Eq. intro_saddle).
#include <algorithm>
#include <cmath>

#include "internal.cuh"
#include "device_util.cuh"

namespace cav {

// Per (component c, marker a): support of the four-point kernel along x and y.
// Face positions: u at (i h, (j+1/2) h), v at ((i+1/2) h, j h).  Along one axis with
// offset o (0 or 1/2) the marker couples to index f - 1 + s (s = 0..3) iff |r_s| < 2 with
//   q = X/h, t = q - o, f = floor(t), a = t - f, r_s = (a + 1) - s,
// and the 1-D weight is phi(r_s).  The support decides E_E's structural pattern.
__global__ void k_marker_support(int M, double h, const double* __restrict__ X,
                                 int* sup_i0, int* sup_j0, double* wx, double* wy,
                                 uint8_t* mask) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= 2 * M) return;
  const int c = id / M, a = id % M;
  const double ox = (c == 0) ? 0.0 : 0.5;
  const double oy = (c == 0) ? 0.5 : 0.0;
  uint8_t m = 0;
  for (int axis = 0; axis < 2; ++axis) {
    const double q = X[axis * M + a] / h;
    const double t = q - (axis == 0 ? ox : oy);
    const double f = floor(t);
    const double fr = t - f;
    double* w = (axis == 0 ? wx : wy) + 4 * id;
    for (int s = 0; s < 4; ++s) {
      const double r = (fr + 1.0) - (double)s;
      const bool in = fabs(r) < 2.0;
      w[s] = in ? phi4(r) : 0.0;
      if (in) m |= (uint8_t)(1u << (s + 4 * axis));
    }
    if (axis == 0) sup_i0[id] = (int)f - 1;
    else sup_j0[id] = (int)f - 1;
  }
  mask[id] = m;
}

// E coefficient of (a, a + d), identical on both components (Eq. disc_force_law, Sec. 5.2).
__global__ void k_force_band(int M, int bw, int law, double ds, double k_target,
                             double k_stretch, double k_bend, double* band) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= M) return;
  for (int d = -bw; d <= bw; ++d) {
    double e = 0.0;
    if (law == IB_FORCE_TARGET) {
      e = -k_target;
    } else {
      if (d == 0 && k_target != 0.0) e += -k_target;  // tethers to targets (Sec. 5.2) on any law
      if (k_stretch != 0.0) {
        const double c2 = k_stretch / (ds * ds);
        if (d == 0) e += c2 * -2.0;
        else if (d == 1 || d == -1) e += c2 * 1.0;
      }
      if (law == IB_FORCE_BEAM && k_bend != 0.0) {
        const double c4 = -k_bend / (ds * ds * ds * ds);
        const double st[5] = {1.0, -4.0, 6.0, -4.0, 1.0};
        e += c4 * st[d + 2];
      }
    }
    band[a * (2 * bw + 1) + (d + bw)] = e;
  }
}

__device__ inline int support_face(int N, int c, int i0, int j0, int sx, int sy) {
  return c * N * N + pmod(j0 + sy, N) * N + pmod(i0 + sx, N);
}

// pass 0: count markers per face; pass 1: write marker ids (order fixed afterwards by a sort)
__global__ void k_face_markers(int N, int M, const int* sup_i0, const int* sup_j0,
                               const uint8_t* mask, int* count, const int64_t* off, int* cursor,
                               int* list, int pass) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= 2 * M) return;
  const int c = id / M, a = id % M;
  const uint8_t m = mask[id];
  for (int sy = 0; sy < 4; ++sy) {
    if (!(m & (1u << (sy + 4)))) continue;
    for (int sx = 0; sx < 4; ++sx) {
      if (!(m & (1u << sx))) continue;
      const int f = support_face(N, c, sup_i0[id], sup_j0[id], sx, sy);
      if (pass == 0) {
        atomicAdd(&count[f], 1);
      } else {
        const int pos = atomicAdd(&cursor[f], 1);
        list[off[f] + pos] = a;
      }
    }
  }
}

// Sort each short list ascending (insertion sort), one thread per list.
__global__ void k_sort_lists(int n, const int64_t* off, int* list) {
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

__global__ void k_flag_nonempty(int n, const int64_t* off, int* flag) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < n) flag[f] = (off[f + 1] > off[f]) ? 1 : 0;
}

// rows[] and row_of[] from a 0/1 flag array and its exclusive scan.
__global__ void k_compact_rows(int n, const int* flag, const int64_t* pos, int* rows, int* row_of) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n) return;
  if (flag[f]) {
    rows[pos[f]] = f;
    row_of[f] = (int)pos[f];
  } else {
    row_of[f] = -1;
  }
}

// One warp per active row k of E_E = S E J on the finest grid.  Contributions are gathered
// into a shared-memory window of column faces (same component as k) around k: for every
// marker a whose support holds k (ascending) and every b in E's band of a, the 16 lanes add
// S[k,a] E[a,b] J[b,l] for the <= 16 faces l of b's support -- distinct cells, so no two
// lanes touch the same entry and the summation order is fixed.  pass 0 counts the
// structural nonzeros of the row; pass 1 writes them in ascending column order.
__global__ void k_ee_assemble(int N, int M, int bw, int closed, double h, int W,
                              const double* __restrict__ omega, const double* __restrict__ band,
                              const int* __restrict__ sup_i0, const int* __restrict__ sup_j0,
                              const double* __restrict__ wx, const double* __restrict__ wy,
                              const uint8_t* __restrict__ mask, const int64_t* __restrict__ fm_off,
                              const int* __restrict__ fm_list, int n_rows, const int* __restrict__ rows,
                              int* row_count, const int64_t* __restrict__ rowptr, int* cols,
                              double* vals, int pass, int* status) {
  extern __shared__ unsigned char smem[];
  const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * warps + warp;
  const int lenmax = (2 * W + 1 >= N) ? N : 2 * W + 1;
  const int cells = lenmax * lenmax;
  double* acc = reinterpret_cast<double*>(smem) + (size_t)warp * cells;
  uint8_t* flg = reinterpret_cast<uint8_t*>(reinterpret_cast<double*>(smem) + (size_t)warps * cells) +
                 (size_t)warp * cells;
  if (row >= n_rows) return;
  const int k = rows[row];
  const int NN = N * N;
  const int c = k / NN, rem = k % NN, ik = rem % N, jk = rem / N;
  const Win wxn = make_win(ik, W, N), wyn = make_win(jk, W, N);
  for (int t = lane; t < cells; t += 32) {
    acc[t] = 0.0;
    flg[t] = 0;
  }
  __syncwarp();
  const double inv_h2 = 1.0 / (h * h);
  for (int64_t q = fm_off[k]; q < fm_off[k + 1]; ++q) {
    const int a = fm_list[q];
    const int ida = c * M + a;
    const int si = pmod(ik - sup_i0[ida], N), sj = pmod(jk - sup_j0[ida], N);
    const double s_ka = wx[4 * ida + si] * wy[4 * ida + sj] * (omega[a] * inv_h2);
    for (int d = -bw; d <= bw; ++d) {
      int b = a + d;
      if (closed) b = pmod(b, M);
      else if (b < 0 || b >= M) continue;
      const double coef = s_ka * band[a * (2 * bw + 1) + (d + bw)];
      const int idb = c * M + b;
      if (lane < 16) {
        const int sx = lane & 3, sy = lane >> 2;
        const uint8_t mb = mask[idb];
        if ((mb & (1u << sx)) && (mb & (1u << (sy + 4)))) {
          const int gi = pmod(sup_i0[idb] + sx, N), gj = pmod(sup_j0[idb] + sy, N);
          const int ox = win_off(wxn, gi, N), oy = win_off(wyn, gj, N);
          if (ox < 0 || oy < 0) {
            atomicExch(status, DEV_WINDOW);
          } else {
            const int cell = oy * wxn.len + ox;
            acc[cell] += coef * (wx[4 * idb + sx] * wy[4 * idb + sy]);
            flg[cell] = 1;
          }
        }
      }
      __syncwarp();
    }
  }
  __syncwarp();
  // ascending global column order: rows of the window (y) ascending, then x ascending
  int64_t outpos = (pass == 1) ? rowptr[row] : 0;
  int total = 0;
  for (int typ = 0; typ < wyn.len; ++typ) {
    const int ty = win_asc(wyn, typ);
    const int gy = win_glob(wyn, ty, N);
    for (int base = 0; base < wxn.len; base += 32) {
      const int txp = base + lane;
      int tx = 0, gx = 0;
      bool f = false;
      if (txp < wxn.len) {
        tx = win_asc(wxn, txp);
        gx = win_glob(wxn, tx, N);
        f = flg[ty * wxn.len + tx] != 0;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, f);
      if (pass == 1 && f) {
        const int rank = __popc(bal & ((1u << lane) - 1u));
        cols[outpos + total + rank] = c * NN + gy * N + gx;
        vals[outpos + total + rank] = acc[ty * wxn.len + tx];
      }
      total += __popc(bal);
    }
  }
  if (pass == 0 && lane == 0) row_count[row] = total;
}

// ------------------------------------------------------------------ fiber law (Sec. 5.3)

// Gradient g (component-major, 2M) and Hessian of the fiber's energy on an open chain at X
// (interleaved), the Hessian as a block band H[p][q - p + 2][c][c2] = d2E / dX_{c,p} dX_{c2,q}.
//   bending     EI/(2 ds^5) sum_k c_k^2,  c_k = D_k x D_{k+1} = a0 b1 - a1 b0,
//               a = D_k = X_{k+1} - X_k, b = D_{k+1} = X_{k+2} - X_{k+1}
//   stretching  K_s/(2 ds) sum_k (|D_k| - ds)^2
//   clamp       K_p/2 |X_m - X_c|^2 + K_t/2 |(X_{m+1} - X_{m-1})/(2 ds) - e_x|^2
// Host arithmetic in FP64; the chain is short (tens to hundreds of markers).
static void fiber_derivatives(const ib_system* s, const double* X, std::vector<double>& g, std::vector<double>& H) {
  const int M = s->M;
  const double ds = s->ds;
  g.assign(2 * (size_t)M, 0.0);
  H.assign((size_t)M * 5 * 4, 0.0);
  auto P = [&](int k, int c) { return X[2 * k + c]; };
  auto addg = [&](int k, int c, double v) { g[(size_t)c * M + k] += v; };
  auto addh = [&](int p, int c, int q, int c2, double v) { H[(((size_t)p * 5 + (q - p + 2)) * 2 + c) * 2 + c2] += v; };
  // bending: variables z = (a0, a1, b0, b1); dz/dX: a = X_{k+1} - X_k, b = X_{k+2} - X_{k+1}
  const double cb = s->k_bend / std::pow(ds, 5);
  for (int k = 0; k + 2 < M; ++k) {
    const double a[2] = {P(k + 1, 0) - P(k, 0), P(k + 1, 1) - P(k, 1)};
    const double b[2] = {P(k + 2, 0) - P(k + 1, 0), P(k + 2, 1) - P(k + 1, 1)};
    const double c = a[0] * b[1] - a[1] * b[0];
    const double dz[4] = {b[1], -b[0], -a[1], a[0]};  // dc/dz
    // d2c/dz2: +1 at (a0, b1), -1 at (a1, b0), symmetric
    double hz[4][4];
    for (int u = 0; u < 4; ++u)
      for (int v = 0; v < 4; ++v) hz[u][v] = cb * dz[u] * dz[v];
    hz[0][3] += cb * c;
    hz[3][0] += cb * c;
    hz[1][2] -= cb * c;
    hz[2][1] -= cb * c;
    // marker and sign of each z-component's dependence: z in a -> (k: -1, k+1: +1); in b -> (k+1: -1, k+2: +1)
    const int mk[2][2] = {{k, k + 1}, {k + 1, k + 2}};
    for (int u = 0; u < 4; ++u) {
      const int vu = u / 2, cu = u % 2;
      addg(mk[vu][0], cu, -cb * c * dz[u]);
      addg(mk[vu][1], cu, cb * c * dz[u]);
      for (int v = 0; v < 4; ++v) {
        const int vv = v / 2, cv = v % 2;
        for (int su = 0; su < 2; ++su)
          for (int sv = 0; sv < 2; ++sv)
            addh(mk[vu][su], cu, mk[vv][sv], cv, (su ? 1.0 : -1.0) * (sv ? 1.0 : -1.0) * hz[u][v]);
      }
    }
  }
  // stretching: per link, grad (|d| - ds) d/|d| and Hessian u u^T + (|d| - ds)/|d| (I - u u^T)
  const double cs = s->k_stretch / ds;
  for (int k = 0; k + 1 < M; ++k) {
    const double d[2] = {P(k + 1, 0) - P(k, 0), P(k + 1, 1) - P(k, 1)};
    const double L = std::sqrt(d[0] * d[0] + d[1] * d[1]);
    const double u[2] = {d[0] / L, d[1] / L};
    const double r = (L - ds) / L;
    for (int c = 0; c < 2; ++c) {
      addg(k, c, -cs * (L - ds) * u[c]);
      addg(k + 1, c, cs * (L - ds) * u[c]);
      for (int c2 = 0; c2 < 2; ++c2) {
        const double h = cs * (u[c] * u[c2] + r * ((c == c2 ? 1.0 : 0.0) - u[c] * u[c2]));
        addh(k, c, k, c2, h);
        addh(k + 1, c, k + 1, c2, h);
        addh(k, c, k + 1, c2, -h);
        addh(k + 1, c, k, c2, -h);
      }
    }
  }
  // midpoint clamp
  const int m = M / 2;
  const double xc[2] = {s->clamp_x, s->clamp_y};
  const double ex[2] = {1.0, 0.0};
  const double ct = s->k_tan / (2.0 * ds);
  for (int c = 0; c < 2; ++c) {
    addg(m, c, s->k_pos * (P(m, c) - xc[c]));
    addh(m, c, m, c, s->k_pos);
    const double tv = (P(m + 1, c) - P(m - 1, c)) / (2.0 * ds) - ex[c];
    addg(m + 1, c, ct * tv);
    addg(m - 1, c, -ct * tv);
    const double h = s->k_tan / (4.0 * ds * ds);
    addh(m + 1, c, m + 1, c, h);
    addh(m - 1, c, m - 1, c, h);
    addh(m + 1, c, m - 1, c, -h);
    addh(m - 1, c, m + 1, c, -h);
  }
}

// E_E = S E J for a law whose E couples the two components (the fiber's tangent): one warp
// per active row k (component c); the window holds the column faces of both components (two
// planes of the same x / y extent).  For every marker a whose c-support holds k (ascending),
// every b in E's band of a and each component c2, the 16 lanes add
// S[k,(c,a)] E[(c,a),(c2,b)] J[(c2,b),l] over the faces l of (c2, b)'s support -- distinct
// faces, so no two lanes touch the same entry and the order is fixed.  Columns are written
// u plane first, then v, each in ascending order.  pass 0 counts, pass 1 writes.
__global__ void k_ee_assemble_x(int N, int M, int bw, double h, int W, const double* __restrict__ omega,
                                const double* __restrict__ eblk, const int* __restrict__ sup_i0,
                                const int* __restrict__ sup_j0, const double* __restrict__ wx,
                                const double* __restrict__ wy, const uint8_t* __restrict__ mask,
                                const int64_t* __restrict__ fm_off, const int* __restrict__ fm_list, int n_rows,
                                const int* __restrict__ rows, int* row_count, const int64_t* __restrict__ rowptr,
                                int* cols, double* vals, int pass, int* status) {
  extern __shared__ unsigned char smem[];
  const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * warps + warp;
  const int lenmax = (2 * W + 1 >= N) ? N : 2 * W + 1;
  const int cells = lenmax * lenmax;
  double* acc = reinterpret_cast<double*>(smem) + (size_t)warp * 2 * cells;
  uint8_t* flg = reinterpret_cast<uint8_t*>(reinterpret_cast<double*>(smem) + (size_t)warps * 2 * cells) +
                 (size_t)warp * 2 * cells;
  if (row >= n_rows) return;
  const int k = rows[row];
  const int NN = N * N;
  const int c = k / NN, rem = k % NN, ik = rem % N, jk = rem / N;
  const Win wxn = make_win(ik, W, N), wyn = make_win(jk, W, N);
  const int plane = wxn.len * wyn.len;
  for (int t = lane; t < 2 * cells; t += 32) {
    acc[t] = 0.0;
    flg[t] = 0;
  }
  __syncwarp();
  const double inv_h2 = 1.0 / (h * h);
  for (int64_t q = fm_off[k]; q < fm_off[k + 1]; ++q) {
    const int a = fm_list[q];
    const int ida = c * M + a;
    const int si = pmod(ik - sup_i0[ida], N), sj = pmod(jk - sup_j0[ida], N);
    const double s_ka = wx[4 * ida + si] * wy[4 * ida + sj] * (omega[a] * inv_h2);
    for (int d = -bw; d <= bw; ++d) {
      const int b = a + d;
      if (b < 0 || b >= M) continue;
      for (int c2 = 0; c2 < 2; ++c2) {
        const double coef = s_ka * eblk[(((size_t)a * (2 * bw + 1) + (d + bw)) * 2 + c) * 2 + c2];
        const int idb = c2 * M + b;
        if (lane < 16) {
          const int sx = lane & 3, sy = lane >> 2;
          const uint8_t mb = mask[idb];
          if ((mb & (1u << sx)) && (mb & (1u << (sy + 4)))) {
            const int gi = pmod(sup_i0[idb] + sx, N), gj = pmod(sup_j0[idb] + sy, N);
            const int ox = win_off(wxn, gi, N), oy = win_off(wyn, gj, N);
            if (ox < 0 || oy < 0) {
              atomicExch(status, DEV_WINDOW);
            } else {
              const int cell = c2 * plane + oy * wxn.len + ox;
              acc[cell] += coef * (wx[4 * idb + sx] * wy[4 * idb + sy]);
              flg[cell] = 1;
            }
          }
        }
        __syncwarp();
      }
    }
  }
  __syncwarp();
  int64_t outpos = (pass == 1) ? rowptr[row] : 0;
  int total = 0;
  for (int c2 = 0; c2 < 2; ++c2)
    for (int typ = 0; typ < wyn.len; ++typ) {
      const int ty = win_asc(wyn, typ);
      const int gy = win_glob(wyn, ty, N);
      for (int base = 0; base < wxn.len; base += 32) {
        const int txp = base + lane;
        int tx = 0, gx = 0;
        bool f = false;
        if (txp < wxn.len) {
          tx = win_asc(wxn, txp);
          gx = win_glob(wxn, tx, N);
          f = flg[c2 * plane + ty * wxn.len + tx] != 0;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (pass == 1 && f) {
          const int rank = __popc(bal & ((1u << lane) - 1u));
          cols[outpos + total + rank] = c2 * NN + gy * N + gx;
          vals[outpos + total + rank] = acc[c2 * plane + ty * wxn.len + tx];
        }
        total += __popc(bal);
      }
    }
  if (pass == 0 && lane == 0) row_count[row] = total;
}

// Max per-axis periodic offset between an E_E row face and its column faces.
__global__ void k_ee_window(int N, int n_rows, const int* rows, const int64_t* rowptr,
                            const int* cols, int* out) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= n_rows) return;
  const int NN = N * N;
  const int k = rows[r] % NN;
  const int ik = k % N, jk = k / N;
  int m = 0;
  for (int64_t q = rowptr[r] + lane; q < rowptr[r + 1]; q += 32) {
    const int l = cols[q] % NN;
    int dx = abs((l % N) - ik), dy = abs((l / N) - jk);
    dx = min(dx, N - dx);
    dy = min(dy, N - dy);
    m = max(m, max(dx, dy));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) atomicMax(out, m);
}

void ee_compute_window(EECsr& ee, int N, int* d_scratch, cudaStream_t st) {
  CAV_CHECK_CUDA(cudaMemsetAsync(d_scratch, 0, sizeof(int), st));
  if (ee.n_rows > 0) {
    k_ee_window<<<div_up(ee.n_rows, 8), 256, 0, st>>>(N, ee.n_rows, ee.rows, ee.rowptr, ee.cols,
                                                      d_scratch);
    CAV_CHECK_LAUNCH();
  }
  int w = 0;
  CAV_CHECK_CUDA(cudaMemcpyAsync(&w, d_scratch, sizeof(int), cudaMemcpyDeviceToHost, st));
  CAV_CHECK_CUDA(cudaStreamSynchronize(st));
  ee.W = w;
}

// F = E X^n + k_target X_target (component-major, both components), the Lagrangian force
// of the linear laws at the current configuration (Eq. disc_force_law, Sec. 5.2).
__global__ void k_force(int M, int bw, int closed, const double* __restrict__ band, const double* __restrict__ X,
                        double k_target, const double* __restrict__ Xt, double* __restrict__ F) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= 2 * M) return;
  const int c = id / M, a = id % M;
  double f = 0.0;
  for (int d = -bw; d <= bw; ++d) {
    int b = a + d;
    if (closed) b = pmod(b, M);
    else if (b < 0 || b >= M) continue;
    f += band[a * (2 * bw + 1) + (d + bw)] * X[c * M + b];
  }
  if (Xt) f += k_target * Xt[id];
  F[id] = f;
}

// f = S F on every velocity face (Sec. 2): the face's markers in ascending order,
// S[face, a] = omega_a / h^2 * phi phi.  One thread per face, no atomics.  With rhs != 0
// the face value also takes rho_dt * u_prev + f_body (right-hand side of Eq. Eul_schur)
// and the pressure rows are zeroed.
__global__ void k_spread(int N, int M, double h, const double* __restrict__ omega, const int* __restrict__ sup_i0,
                         const int* __restrict__ sup_j0, const double* __restrict__ wx, const double* __restrict__ wy,
                         const int64_t* __restrict__ fm_off, const int* __restrict__ fm_list,
                         const double* __restrict__ F, double* __restrict__ f, int rhs, double rho_dt,
                         const double* __restrict__ u_prev, const double* __restrict__ f_body) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int NN = N * N;
  if (k >= 3 * NN) return;
  if (k >= 2 * NN) {
    if (rhs) f[k] = 0.0;
    return;
  }
  const int c = k / NN, rem = k % NN, ik = rem % N, jk = rem / N;
  const double inv_h2 = 1.0 / (h * h);
  double s = 0.0;
  if (fm_off)
    for (int64_t q = fm_off[k]; q < fm_off[k + 1]; ++q) {
      const int a = fm_list[q];
      const int ida = c * M + a;
      const int si = pmod(ik - sup_i0[ida], N), sj = pmod(jk - sup_j0[ida], N);
      s += wx[4 * ida + si] * wy[4 * ida + sj] * (omega[a] * inv_h2) * F[ida];
    }
  if (rhs) {
    double v = s;
    if (u_prev) v += rho_dt * u_prev[k];
    if (f_body) v += f_body[k];
    f[k] = v;
  } else {
    f[k] = s;
  }
}

// U = J u (Sec. 2): U_a = sum over the marker's 4 x 4 support of phi phi u_face.  With
// dt != 0, instead X_out = X + dt U (Eq. im_disc_advec).
__global__ void k_interp(int N, int M, const int* __restrict__ sup_i0, const int* __restrict__ sup_j0,
                         const double* __restrict__ wx, const double* __restrict__ wy, const uint8_t* __restrict__ mask,
                         const double* __restrict__ u, double* __restrict__ U, double dt, const double* __restrict__ X) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= 2 * M) return;
  const int c = id / M;
  const uint8_t m = mask[id];
  double s = 0.0;
  for (int sy = 0; sy < 4; ++sy) {
    if (!(m & (1u << (sy + 4)))) continue;
    for (int sx = 0; sx < 4; ++sx) {
      if (!(m & (1u << sx))) continue;
      const int face = c * N * N + pmod(sup_j0[id] + sy, N) * N + pmod(sup_i0[id] + sx, N);
      s += wx[4 * id + sx] * wy[4 * id + sy] * u[face];
    }
  }
  U[id] = (dt != 0.0) ? X[id] + dt * s : s;
}

void ib_force_launch(const ib_system* s, double* F, cudaStream_t st) {
  if (s->M == 0) return;
  if (s->law == IB_FORCE_FIBER) {  // evaluated at set-up, at the linearisation point
    CAV_CHECK_CUDA(cudaMemcpyAsync(F, s->Ffib, sizeof(double) * 2 * s->M, cudaMemcpyDeviceToDevice, st));
    return;
  }
  k_force<<<div_up(2 * s->M, 128), 128, 0, st>>>(s->M, s->bw, s->closed, s->Eband, s->X, s->k_target, s->Xt, F);
  CAV_CHECK_LAUNCH();
}
void ib_spread_launch(const ib_system* s, const double* F, double* f, int rhs, const double* u_prev,
                      const double* f_body, cudaStream_t st) {
  const int NN = s->N * s->N;
  k_spread<<<div_up(3 * NN, 256), 256, 0, st>>>(s->N, s->M, s->h, s->omega, s->sup_i0, s->sup_j0, s->sup_wx,
                                               s->sup_wy, s->M ? s->fm_off : nullptr, s->fm_list, F, f, rhs,
                                               s->rho / s->dt, u_prev, f_body);
  CAV_CHECK_LAUNCH();
}
void ib_interp_launch(const ib_system* s, const double* u, double* U, double dt, cudaStream_t st) {
  if (s->M == 0) return;
  k_interp<<<div_up(2 * s->M, 128), 128, 0, st>>>(s->N, s->M, s->sup_i0, s->sup_j0, s->sup_wx, s->sup_wy,
                                                 s->sup_mask, u, U, dt, s->X);
  CAV_CHECK_LAUNCH();
}

static size_t ee_smem_per_warp(int W, int N) {
  const int len = (2 * W + 1 >= N) ? N : 2 * W + 1;
  return (size_t)len * len * (sizeof(double) + 1);
}

void build_markers_and_ee(ib_system* s, const double* X_il, const double* X_lin_il, const double* omega_host,
                          cudaStream_t st) {
  const int N = s->N, M = s->M, NN = N * N;
  Arena& A = s->arena;
  Arena scratch;
  try {
    s->ee.row_of = A.alloc<int>(2 * NN);
    if (M == 0) {
      CAV_CHECK_CUDA(cudaMemsetAsync(s->ee.row_of, 0xff, sizeof(int) * 2 * NN, st));
      s->ee.rowptr = A.alloc<int64_t>(1);
      CAV_CHECK_CUDA(cudaMemsetAsync(s->ee.rowptr, 0, sizeof(int64_t), st));
      s->ee.n_rows = 0;
      s->ee.nnz = 0;
      s->ee.W = 0;
      CAV_CHECK_CUDA(cudaStreamSynchronize(st));
      return;
    }
    // markers to component-major device arrays
    std::vector<double> Xcm(2 * (size_t)M);
    for (int a = 0; a < M; ++a) {
      Xcm[a] = X_il[2 * a];
      Xcm[M + a] = X_il[2 * a + 1];
    }
    s->X = A.alloc<double>(2 * M);
    s->omega = A.alloc<double>(M);
    s->F = A.alloc<double>(2 * M);
    s->U = A.alloc<double>(2 * M);
    CAV_CHECK_CUDA(cudaMemcpyAsync(s->X, Xcm.data(), sizeof(double) * 2 * M, cudaMemcpyHostToDevice, st));
    CAV_CHECK_CUDA(cudaMemcpyAsync(s->omega, omega_host, sizeof(double) * M, cudaMemcpyHostToDevice, st));
    s->sup_i0 = A.alloc<int>(2 * M);
    s->sup_j0 = A.alloc<int>(2 * M);
    s->sup_wx = A.alloc<double>(8 * M);
    s->sup_wy = A.alloc<double>(8 * M);
    s->sup_mask = A.alloc<uint8_t>(2 * M);
    k_marker_support<<<div_up(2 * M, 128), 128, 0, st>>>(M, s->h, s->X, s->sup_i0, s->sup_j0,
                                                        s->sup_wx, s->sup_wy, s->sup_mask);
    CAV_CHECK_LAUNCH();
    const bool fib = s->law == IB_FORCE_FIBER;
    if (fib) {
      // the fiber's force and tangent at the linearisation point: F = -g/ds, E = -H/ds
      std::vector<double> g, H;
      fiber_derivatives(s, X_lin_il, g, H);
      for (double& v : g) v = -v / s->ds;
      for (double& v : H) v = -v / s->ds;
      s->Eblock = A.alloc<double>(H.size());
      s->Ffib = A.alloc<double>(g.size());
      CAV_CHECK_CUDA(cudaMemcpyAsync(s->Eblock, H.data(), sizeof(double) * H.size(), cudaMemcpyHostToDevice, st));
      CAV_CHECK_CUDA(cudaMemcpyAsync(s->Ffib, g.data(), sizeof(double) * g.size(), cudaMemcpyHostToDevice, st));
      CAV_CHECK_CUDA(cudaStreamSynchronize(st));
    } else {
      s->Eband = A.alloc<double>((size_t)M * (2 * s->bw + 1));
      k_force_band<<<div_up(M, 128), 128, 0, st>>>(M, s->bw, s->law, s->ds, s->k_target, s->k_stretch,
                                                  s->k_bend, s->Eband);
      CAV_CHECK_LAUNCH();
    }
    // face -> markers incidence
    int* count = scratch.alloc<int>(2 * NN);
    int* cursor = scratch.alloc<int>(2 * NN);
    CAV_CHECK_CUDA(cudaMemsetAsync(count, 0, sizeof(int) * 2 * NN, st));
    CAV_CHECK_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int) * 2 * NN, st));
    k_face_markers<<<div_up(2 * M, 128), 128, 0, st>>>(N, M, s->sup_i0, s->sup_j0, s->sup_mask,
                                                      count, nullptr, nullptr, nullptr, 0);
    CAV_CHECK_LAUNCH();
    s->fm_off = A.alloc<int64_t>(2 * NN + 1);
    exclusive_scan(count, s->fm_off, 2 * NN, st, &scratch);
    int64_t total = 0;
    CAV_CHECK_CUDA(cudaMemcpyAsync(&total, s->fm_off + 2 * NN, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CAV_CHECK_CUDA(cudaStreamSynchronize(st));
    s->fm_list = A.alloc<int>(total);
    k_face_markers<<<div_up(2 * M, 128), 128, 0, st>>>(N, M, s->sup_i0, s->sup_j0, s->sup_mask,
                                                      count, s->fm_off, cursor, s->fm_list, 1);
    CAV_CHECK_LAUNCH();
    k_sort_lists<<<div_up(2 * NN, 256), 256, 0, st>>>(2 * NN, s->fm_off, s->fm_list);
    CAV_CHECK_LAUNCH();
    // active rows
    int* flag = scratch.alloc<int>(2 * NN);
    int64_t* pos = scratch.alloc<int64_t>(2 * NN + 1);
    k_flag_nonempty<<<div_up(2 * NN, 256), 256, 0, st>>>(2 * NN, s->fm_off, flag);
    CAV_CHECK_LAUNCH();
    exclusive_scan(flag, pos, 2 * NN, st, &scratch);
    int64_t nrows = 0;
    CAV_CHECK_CUDA(cudaMemcpyAsync(&nrows, pos + 2 * NN, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CAV_CHECK_CUDA(cudaStreamSynchronize(st));
    EECsr& ee = s->ee;
    ee.n_rows = (int)nrows;
    ee.rows = A.alloc<int>(nrows);
    k_compact_rows<<<div_up(2 * NN, 256), 256, 0, st>>>(2 * NN, flag, pos, ee.rows, ee.row_of);
    CAV_CHECK_LAUNCH();
    // window half-width: two kernel reaches plus the largest marker separation within E's band
    double D = 0.0;
    for (int a = 0; a < M; ++a) {
      for (int d = -s->bw; d <= s->bw; ++d) {
        int b = a + d;
        if (s->closed) b = ((b % M) + M) % M;
        else if (b < 0 || b >= M) continue;
        for (int ax = 0; ax < 2; ++ax) {
          double dd = std::fabs(X_il[2 * a + ax] - X_il[2 * b + ax]);
          dd = std::fmod(dd, s->L);
          dd = std::min(dd, s->L - dd);
          D = std::max(D, dd / s->h);
        }
      }
    }
    const int W = (int)std::ceil(D) + 5;
    const int warps = 4;
    // the cross-component assembly keeps two window planes per warp
    const size_t smem = warps * ee_smem_per_warp(W, N) * (fib ? 2 : 1);
    CAV_REQUIRE(smem <= 200 * 1024, "E_E stencil window too large (markers too far apart in E's band)");
    if (smem > 48 * 1024) {
      if (fib)
        CAV_CHECK_CUDA(cudaFuncSetAttribute(k_ee_assemble_x, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      else
        CAV_CHECK_CUDA(cudaFuncSetAttribute(k_ee_assemble, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    ee.cross = fib ? 1 : 0;
    int* row_count = scratch.alloc<int>(nrows + 1);
    const int grid = div_up(nrows, warps);
    ee.rowptr = A.alloc<int64_t>(nrows + 1);
    auto assemble = [&](const int64_t* rowptr, int* cols, double* vals, int pass) {
      if (nrows == 0) return;
      if (fib)
        k_ee_assemble_x<<<grid, warps * 32, smem, st>>>(N, M, s->bw, s->h, W, s->omega, s->Eblock, s->sup_i0,
                                                        s->sup_j0, s->sup_wx, s->sup_wy, s->sup_mask, s->fm_off,
                                                        s->fm_list, (int)nrows, ee.rows, row_count, rowptr, cols,
                                                        vals, pass, s->status);
      else
        k_ee_assemble<<<grid, warps * 32, smem, st>>>(N, M, s->bw, s->closed, s->h, W, s->omega, s->Eband,
                                                      s->sup_i0, s->sup_j0, s->sup_wx, s->sup_wy, s->sup_mask,
                                                      s->fm_off, s->fm_list, (int)nrows, ee.rows, row_count,
                                                      rowptr, cols, vals, pass, s->status);
      CAV_CHECK_LAUNCH();
    };
    assemble(nullptr, nullptr, nullptr, 0);
    exclusive_scan(row_count, ee.rowptr, nrows, st, &scratch);
    int64_t nnz = 0;
    CAV_CHECK_CUDA(cudaMemcpyAsync(&nnz, ee.rowptr + nrows, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CAV_CHECK_CUDA(cudaStreamSynchronize(st));
    ee.nnz = nnz;
    ee.cols = A.alloc<int>(nnz);
    ee.vals = A.alloc<double>(nnz);
    assemble(ee.rowptr, ee.cols, ee.vals, 1);
    ee_compute_window(ee, N, scratch.alloc<int>(1), st);
    scratch.release();
  } catch (...) {
    cudaStreamSynchronize(st);
    scratch.release();
    throw;
  }
}

}  // namespace cav
