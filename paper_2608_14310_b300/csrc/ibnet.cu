// Small convolutional network that predicts the initial guess of each time step's solve from
// the previous steps' fields (velocity, pressure, spread Lagrangian force), with its own
// forward, backward and Adam kernels (FP32).  Periodic (circular) padding matches the
// periodic MAC grid.  Architecture: conv3x3(in -> hidden) GELU, (n_hidden - 1) x
// [conv3x3(hidden -> hidden) GELU], conv3x3(hidden -> out).  Tensors are [batch][channel][N][N].
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"
#include "device_util.cuh"

namespace cav {

constexpr int CT = 16;       // pixel tile edge
constexpr int CO_TILE = 32;  // output channels per block

// out[b, co, y, x] = bias[co] + sum_ci sum_ky,kx W[co, ci, ky, kx] in[b, ci, y+ky-1, x+kx-1]
// (indices mod N).  Block: a 16 x 16 pixel tile of one sample and up to 32 output channels;
// the input channel's 18 x 18 halo tile and its 32 x 9 weights are staged in shared memory.
// The sum over (ci, ky, kx) runs in a fixed order.  With wflip != 0 the kernel computes the
// transposed convolution used by the backward pass: weights read as W[ci, co, 2-ky, 2-kx]
// from a [Cin_fwd = Cout][Cout_fwd = Cin] layout (see k_conv_bwd_data).
__global__ void __launch_bounds__(CT* CT)
k_conv_fwd(const float* __restrict__ in, const float* __restrict__ W, const float* __restrict__ bias,
           float* __restrict__ out, int Cin, int Cout, int N, int tiles_x, int wflip) {
  __shared__ float tile[CT + 2][CT + 2];
  __shared__ float wsh[CO_TILE][9];
  const int tx = threadIdx.x % CT, ty = threadIdx.x / CT;
  const int tile_id = blockIdx.x;
  const int x0 = (tile_id % tiles_x) * CT, y0 = (tile_id / tiles_x) * CT;
  const int co0 = blockIdx.y * CO_TILE;
  const int b = blockIdx.z;
  const int x = x0 + tx, y = y0 + ty;
  float acc[CO_TILE];
#pragma unroll
  for (int q = 0; q < CO_TILE; ++q) acc[q] = 0.f;
  const size_t NN = (size_t)N * N;
  for (int ci = 0; ci < Cin; ++ci) {
    __syncthreads();
    const float* src = in + ((size_t)b * Cin + ci) * NN;
    for (int t = threadIdx.x; t < (CT + 2) * (CT + 2); t += CT * CT) {
      const int hy = t / (CT + 2), hx = t % (CT + 2);
      const int gy = pmod(y0 + hy - 1, N), gx = pmod(x0 + hx - 1, N);
      tile[hy][hx] = src[(size_t)gy * N + gx];
    }
    for (int t = threadIdx.x; t < CO_TILE * 9; t += CT * CT) {
      const int q = t / 9, k = t % 9;
      const int co = co0 + q;
      float wv = 0.f;
      if (co < Cout) {
        if (!wflip) wv = W[((size_t)co * Cin + ci) * 9 + k];
        else wv = W[((size_t)ci * Cout + co) * 9 + (8 - k)];
      }
      wsh[q][k] = wv;
    }
    __syncthreads();
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const float v = tile[ty + ky][tx + kx];
#pragma unroll
        for (int q = 0; q < CO_TILE; ++q) acc[q] = fmaf(wsh[q][ky * 3 + kx], v, acc[q]);
      }
  }
  if (x < N && y < N) {
#pragma unroll
    for (int q = 0; q < CO_TILE; ++q) {
      const int co = co0 + q;
      if (co < Cout) out[((size_t)b * Cout + co) * NN + (size_t)y * N + x] = acc[q] + (bias ? bias[co] : 0.f);
    }
  }
}

// gW[co, ci, ky, kx] = sum_{b, y, x} g[b, co, y, x] in[b, ci, y+ky-1, x+kx-1]; one block per
// (co, ci), threads over (b, pixel) in a fixed stride, fixed block reduction.
__global__ void k_conv_bwd_weight(const float* __restrict__ in, const float* __restrict__ g, float* __restrict__ gW,
                                  int B, int Cin, int Cout, int N) {
  __shared__ float red[9][8];
  const int co = blockIdx.x, ci = blockIdx.y;
  const size_t NN = (size_t)N * N;
  float acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = 0.f;
  const size_t total = (size_t)B * NN;
  for (size_t e = threadIdx.x; e < total; e += blockDim.x) {
    const int b = (int)(e / NN);
    const int pix = (int)(e % NN);
    const int y = pix / N, x = pix % N;
    const float gv = g[((size_t)b * Cout + co) * NN + pix];
    const float* src = in + ((size_t)b * Cin + ci) * NN;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const int gy = pmod(y + ky - 1, N);
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) acc[ky * 3 + kx] = fmaf(gv, src[(size_t)gy * N + pmod(x + kx - 1, N)], acc[ky * 3 + kx]);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const float v = warp_sumf(acc[k]);
    if (lane == 0) red[k][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
    gW[((size_t)co * Cin + ci) * 9 + threadIdx.x] = t;
  }
}

// gb[co] = sum_{b, pixel} g[b, co, pixel]
__global__ void k_conv_bwd_bias(const float* __restrict__ g, float* __restrict__ gb, int B, int Cout, int N) {
  __shared__ float red[8];
  const int co = blockIdx.x;
  const size_t NN = (size_t)N * N;
  float s = 0.f;
  for (size_t e = threadIdx.x; e < (size_t)B * NN; e += blockDim.x) {
    const int b = (int)(e / NN);
    s += g[((size_t)b * Cout + co) * NN + (e % NN)];
  }
  s = warp_sumf(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    gb[co] = t;
  }
}

// GELU(z) = z Phi(z), Phi the standard normal distribution function (via erff).
__global__ void k_gelu(const float* __restrict__ z, float* __restrict__ a, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float v = z[i];
    a[i] = 0.5f * v * (1.f + erff(v * 0.70710678118654752f));
  }
}
// g_z = g_a * (Phi(z) + z phi(z))
__global__ void k_gelu_bwd(const float* __restrict__ z, const float* __restrict__ ga, float* __restrict__ gz, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float v = z[i];
    const float Phi = 0.5f * (1.f + erff(v * 0.70710678118654752f));
    const float phi = 0.39894228040143268f * expf(-0.5f * v * v);
    gz[i] = ga[i] * (Phi + v * phi);
  }
}

// MSE: g = 2 (out - target) / n and per-block partial sums of (out - target)^2.
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ tgt, float* __restrict__ g, size_t n,
                      float* __restrict__ partial) {
  __shared__ float red[8];
  float s = 0.f;
  const float sc = 2.f / (float)n;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float d = out[i] - tgt[i];
    g[i] = sc * d;
    s = fmaf(d, d, s);
  }
  s = warp_sumf(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}
// <a, b> with FP64 products and sums: per-block partials in a fixed order, then their sum in
// block order (reproducible).
constexpr int IN_BLOCKS = 296;
__global__ void k_inner(const float* __restrict__ a, const float* __restrict__ b, size_t n, double* __restrict__ partial) {
  __shared__ double red[8];
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s = fma((double)a[i], (double)b[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}
__global__ void k_inner_sum(const double* __restrict__ partial, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < n; ++i) t += partial[i];
    *out = t;
  }
}

__global__ void k_sum_partials(const float* __restrict__ partial, int n, float scale, float* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < n; ++i) t += partial[i];
    out[0] = t * scale;
  }
}

// Adam (Kingma and Ba, 2015) with bias correction; step t >= 1.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       size_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// Network input from the solver's last three steps x_0, x_1, x_2 (oldest first) and spread
// forces f_0, f_1, f_2: channel groups of five (u, v, p, f_u, f_v) holding the increments
// x_1 - x_0 and f_1 - f_0, then x_2 - x_1 and f_2 - f_1, then the current x_2 and f_2, each
// divided by its scale.  Increments are formed in FP64 before rounding to FP32.
struct PackPtrs {
  const double* x[3];
  const double* f[3];
  float inv_scale[15];
};
__global__ void k_pack_input(PackPtrs P, int N, float* __restrict__ out) {
  const size_t NN = (size_t)N * N;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < 15 * NN; e += (size_t)gridDim.x * blockDim.x) {
    const int ch = (int)(e / NN);
    const size_t pix = e % NN;
    const int t = ch / 5, k = ch % 5;
    const size_t off = (k < 3) ? k * NN + pix : (k - 3) * NN + pix;
    const double* const* src = (k < 3) ? P.x : P.f;
    double v;
    if (t < 2) v = src[t + 1][off] - src[t][off];
    else v = src[2][off];
    out[e] = (float)(v * (double)P.inv_scale[ch]);
  }
}
// The history in difference form: K steps (oldest first), channel groups for the differences
// of order d = K - 1, ..., 1, 0 in time at the newest step of (u, v, p, f_u, f_v), d = 0 being
// the newest fields themselves; each channel divided by its scale.
struct HistPtrs {
  const double* x[4];
  const double* f[4];
  float inv_scale[20];
  int K;
};
__global__ void k_pack_history(HistPtrs P, int N, float* __restrict__ out) {
  const size_t NN = (size_t)N * N;
  const int K = P.K;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < 5 * (size_t)K * NN;
       e += (size_t)gridDim.x * blockDim.x) {
    const int ch = (int)(e / NN);
    const size_t pix = e % NN;
    const int d = K - 1 - ch / 5, k = ch % 5;
    const size_t off = (k < 3) ? k * NN + pix : (k - 3) * NN + pix;
    const double* const* src = (k < 3) ? P.x : P.f;
    // the d-th backward difference: sum_m (-1)^m binom(d, m) value at step K - 1 - m
    double v = 0.0, c = 1.0;
    for (int m = 0; m <= d; ++m) {
      v += c * src[K - 1 - m][off];
      c = -c * (double)(d - m) / (double)(m + 1);
    }
    out[e] = (float)(v * (double)P.inv_scale[ch]);
  }
}

// target = (x_new - base) / scale per field (u, v, p), base = x_prev, or the linear
// extrapolation 2 x_prev - x_prev2 when x_prev2 is given
// The extrapolation base of a prediction from the last one, two or three steps: x_prev;
// 2 x_prev - x_prev2 (linear); 3 x_prev - 3 x_prev2 + x_prev3 (quadratic).
__device__ inline double extrapolation_base(const double* xp, const double* xp2, const double* xp3, size_t e) {
  if (xp3) return xp3[e] + 3.0 * (xp[e] - xp2[e]);
  if (xp2) return xp[e] + (xp[e] - xp2[e]);
  return xp[e];
}

__global__ void k_pack_target(const double* __restrict__ xn, const double* __restrict__ xp,
                              const double* __restrict__ xp2, const double* __restrict__ xp3, float s0, float s1,
                              float s2, int N, float* __restrict__ out) {
  const size_t NN = (size_t)N * N;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < 3 * NN; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / NN);
    const double inv = 1.0 / (double)(k == 0 ? s0 : (k == 1 ? s1 : s2));
    out[e] = (float)((xn[e] - extrapolation_base(xp, xp2, xp3, e)) * inv);
  }
}
// x_out = base + scale * delta per field, base as in k_pack_target
__global__ void k_apply_delta(const double* __restrict__ xp, const double* __restrict__ xp2,
                              const double* __restrict__ xp3, const float* __restrict__ d, float s0, float s1,
                              float s2, int N, double* __restrict__ xo) {
  const size_t NN = (size_t)N * N;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < 3 * NN; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / NN);
    const float s = (k == 0 ? s0 : (k == 1 ? s1 : s2));
    xo[e] = extrapolation_base(xp, xp2, xp3, e) + (d ? (double)s * (double)d[e] : 0.0);
  }
}

static int grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)(b > 2368 ? 2368 : (b < 1 ? 1 : b));
}

}  // namespace cav

using namespace cav;

struct ibnet {
  ibnet_desc d{};
  int L = 0;                          // conv layers
  std::vector<int> cin, cout;         // per layer
  std::vector<size_t> woff, boff;     // offsets of W_l and b_l in the flat parameter vector
  size_t n_params = 0;
  Arena arena;
  float* p = nullptr;                 // parameters
  float* g = nullptr;                 // gradients
  float* m = nullptr;                 // Adam moments
  float* v = nullptr;
  float* wflip = nullptr;             // scratch (unused: the flipped read is done in the kernel)
  long long t = 0;                    // Adam step count
  // activation workspace for (batch, N)
  int ws_b = 0, ws_n = 0;
  Arena ws;
  std::vector<float*> a;              // a[l]: input of conv l (a[0] = network input, copied)
  std::vector<float*> z;              // z[l]: output of conv l (pre-activation)
  float* gbuf[2] = {nullptr, nullptr};
  float* partial = nullptr;
  float* loss_dev = nullptr;
  double* inner_partial = nullptr;    // [IN_BLOCKS + 1] (ibnet_inner), allocated on first use
};

static void net_workspace(ibnet* net, int B, int N) {
  if (net->ws_b >= B && net->ws_n == N) return;
  net->ws.release();
  net->a.assign(net->L, nullptr);
  net->z.assign(net->L, nullptr);
  const size_t NN = (size_t)N * N;
  int cmax = 0;
  for (int l = 0; l < net->L; ++l) {
    net->a[l] = net->ws.alloc<float>((size_t)B * net->cin[l] * NN);
    net->z[l] = net->ws.alloc<float>((size_t)B * net->cout[l] * NN);
    cmax = std::max(cmax, std::max(net->cin[l], net->cout[l]));
  }
  net->gbuf[0] = net->ws.alloc<float>((size_t)B * cmax * NN);
  net->gbuf[1] = net->ws.alloc<float>((size_t)B * cmax * NN);
  net->partial = net->ws.alloc<float>(2368);
  net->loss_dev = net->ws.alloc<float>(1);
  net->ws_b = B;
  net->ws_n = N;
}

static void conv_launch(const float* in, const float* W, const float* b, float* out, int B, int Cin, int Cout, int N,
                        int flip, cudaStream_t st) {
  const int tiles = div_up(N, CT);
  dim3 grid(tiles * tiles, div_up(Cout, CO_TILE), B);
  k_conv_fwd<<<grid, CT * CT, 0, st>>>(in, W, b, out, Cin, Cout, N, tiles, flip);
  CAV_CHECK_LAUNCH();
}

// Forward pass: in (B x in_ch x N x N) -> out (B x out_ch x N x N); keeps activations.
static void net_forward(ibnet* net, const float* in, float* out, int B, int N, cudaStream_t st) {
  net_workspace(net, B, N);
  const size_t NN = (size_t)N * N;
  CAV_CHECK_CUDA(cudaMemcpyAsync(net->a[0], in, sizeof(float) * B * net->cin[0] * NN, cudaMemcpyDeviceToDevice, st));
  for (int l = 0; l < net->L; ++l) {
    conv_launch(net->a[l], net->p + net->woff[l], net->p + net->boff[l], net->z[l], B, net->cin[l], net->cout[l], N,
                0, st);
    if (l + 1 < net->L) {
      const size_t n = (size_t)B * net->cout[l] * NN;
      k_gelu<<<grid_for(n), 256, 0, st>>>(net->z[l], net->a[l + 1], n);
      CAV_CHECK_LAUNCH();
    }
  }
  if (out)
    CAV_CHECK_CUDA(cudaMemcpyAsync(out, net->z[net->L - 1], sizeof(float) * B * net->cout[net->L - 1] * NN,
                                   cudaMemcpyDeviceToDevice, st));
}

// Loss and gradients (into net->g) for the last forward pass against `target`.
static void net_backward(ibnet* net, const float* target, int B, int N, cudaStream_t st) {
  const size_t NN = (size_t)N * N;
  const int Lm = net->L - 1;
  const size_t nout = (size_t)B * net->cout[Lm] * NN;
  float* g = net->gbuf[0];
  const int nb = grid_for(nout);
  k_mse<<<nb, 256, 0, st>>>(net->z[Lm], target, g, nout, net->partial);
  CAV_CHECK_LAUNCH();
  k_sum_partials<<<1, 32, 0, st>>>(net->partial, nb, 1.f / (float)nout, net->loss_dev);
  CAV_CHECK_LAUNCH();
  for (int l = Lm; l >= 0; --l) {
    // g holds dLoss/dz_l
    k_conv_bwd_weight<<<dim3(net->cout[l], net->cin[l]), 256, 0, st>>>(net->a[l], g, net->g + net->woff[l], B,
                                                                       net->cin[l], net->cout[l], N);
    CAV_CHECK_LAUNCH();
    k_conv_bwd_bias<<<net->cout[l], 256, 0, st>>>(g, net->g + net->boff[l], B, net->cout[l], N);
    CAV_CHECK_LAUNCH();
    if (l == 0) break;
    // dLoss/da_l = conv^T(g); then through GELU of layer l-1
    float* ga = net->gbuf[1];
    conv_launch(g, net->p + net->woff[l], nullptr, ga, B, net->cout[l], net->cin[l], N, 1, st);
    const size_t n = (size_t)B * net->cin[l] * NN;
    k_gelu_bwd<<<grid_for(n), 256, 0, st>>>(net->z[l - 1], ga, g, n);
    CAV_CHECK_LAUNCH();
  }
}

static uint64_t splitmix(uint64_t& s) {
  s += 0x9E3779B97F4A7C15ULL;
  uint64_t z = s;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

extern "C" {

ib_status ibnet_create(const ibnet_desc* d, ibnet** out) {
  if (!out) {
    set_error("ibnet_create: out is NULL");
    return IB_ERR_INVALID;
  }
  *out = nullptr;
  ibnet* net = nullptr;
  try {
    CAV_REQUIRE(d && d->in_ch >= 1 && d->hidden >= 1 && d->n_hidden >= 1 && d->out_ch >= 1, "ibnet_create: bad desc");
    CAV_REQUIRE(d->hidden <= 256 && d->in_ch <= 256 && d->out_ch <= 256, "ibnet_create: too many channels");
    net = new ibnet();
    net->d = *d;
    net->L = d->n_hidden + 1;
    for (int l = 0; l < net->L; ++l) {
      net->cin.push_back(l == 0 ? d->in_ch : d->hidden);
      net->cout.push_back(l + 1 == net->L ? d->out_ch : d->hidden);
    }
    size_t off = 0;
    for (int l = 0; l < net->L; ++l) {
      net->woff.push_back(off);
      off += (size_t)net->cout[l] * net->cin[l] * 9;
      net->boff.push_back(off);
      off += net->cout[l];
    }
    net->n_params = off;
    // uniform(-a, a) with a = sqrt(6 / fan_in) for weights (GELU-friendly scale), zero bias;
    // the last layer is scaled by 0.1 so the initial prediction is a small correction
    std::vector<float> h(off, 0.f);
    uint64_t s = d->seed;
    for (int l = 0; l < net->L; ++l) {
      const double a = std::sqrt(6.0 / (net->cin[l] * 9.0)) * (l + 1 == net->L ? 0.1 : 1.0);
      for (size_t i = 0; i < (size_t)net->cout[l] * net->cin[l] * 9; ++i) {
        const double u = (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
        h[net->woff[l] + i] = (float)((2.0 * u - 1.0) * a);
      }
    }
    net->p = net->arena.alloc<float>(off);
    net->g = net->arena.alloc<float>(off);
    net->m = net->arena.alloc<float>(off);
    net->v = net->arena.alloc<float>(off);
    CAV_CHECK_CUDA(cudaMemcpy(net->p, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice));
    CAV_CHECK_CUDA(cudaMemset(net->m, 0, sizeof(float) * off));
    CAV_CHECK_CUDA(cudaMemset(net->v, 0, sizeof(float) * off));
    CAV_CHECK_CUDA(cudaMemset(net->g, 0, sizeof(float) * off));
    *out = net;
    return IB_OK;
  } catch (const Fail& f) {
    if (net) {
      net->arena.release();
      delete net;
    }
    return f.st;
  } catch (...) {
    if (net) {
      net->arena.release();
      delete net;
    }
    set_error("ibnet_create: internal error");
    return IB_ERR_INTERNAL;
  }
}

void ibnet_destroy(ibnet* net) {
  if (!net) return;
  cudaDeviceSynchronize();
  net->ws.release();
  net->arena.release();
  if (net->inner_partial) cudaFree(net->inner_partial);
  delete net;
}

int64_t ibnet_num_params(const ibnet* net) { return net ? (int64_t)net->n_params : 0; }

ib_status ibnet_get_params(const ibnet* net, float* host) {
  try {
    CAV_REQUIRE(net && host, "ibnet_get_params: NULL argument");
    CAV_CHECK_CUDA(cudaMemcpy(host, net->p, sizeof(float) * net->n_params, cudaMemcpyDeviceToHost));
    return IB_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

ib_status ibnet_set_params(ibnet* net, const float* host) {
  try {
    CAV_REQUIRE(net && host, "ibnet_set_params: NULL argument");
    CAV_CHECK_CUDA(cudaMemcpy(net->p, host, sizeof(float) * net->n_params, cudaMemcpyHostToDevice));
    CAV_CHECK_CUDA(cudaMemset(net->m, 0, sizeof(float) * net->n_params));
    CAV_CHECK_CUDA(cudaMemset(net->v, 0, sizeof(float) * net->n_params));
    net->t = 0;
    return IB_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

ib_status ibnet_forward(ibnet* net, const float* in, float* out, int32_t batch, int32_t N, cudaStream_t st) {
  try {
    CAV_REQUIRE(net && in && out && batch >= 1 && N >= 1, "ibnet_forward: bad argument");
    net_forward(net, in, out, batch, N, st);
    return IB_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

ib_status ibnet_inner(ibnet* net, int64_t n, const float* a, const float* b, double* out, cudaStream_t st) {
  try {
    CAV_REQUIRE(net && a && b && out && n >= 0, "ibnet_inner: bad argument");
    if (!net->inner_partial) CAV_CHECK_CUDA(cudaMalloc(&net->inner_partial, sizeof(double) * (IN_BLOCKS + 1)));
    k_inner<<<IN_BLOCKS, 256, 0, st>>>(a, b, (size_t)n, net->inner_partial);
    CAV_CHECK_LAUNCH();
    k_inner_sum<<<1, 32, 0, st>>>(net->inner_partial, IN_BLOCKS, net->inner_partial + IN_BLOCKS);
    CAV_CHECK_LAUNCH();
    CAV_CHECK_CUDA(cudaMemcpyAsync(out, net->inner_partial + IN_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, st));
    CAV_CHECK_CUDA(cudaStreamSynchronize(st));
    return IB_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

ib_status ibnet_gradients(ibnet* net, const float* in, const float* target, int32_t batch, int32_t N,
                          float* loss_host, float* grads_host, cudaStream_t st) {
  try {
    CAV_REQUIRE(net && in && target && batch >= 1 && N >= 1, "ibnet_gradients: bad argument");
    net_forward(net, in, nullptr, batch, N, st);
    net_backward(net, target, batch, N, st);
    if (loss_host) CAV_CHECK_CUDA(cudaMemcpyAsync(loss_host, net->loss_dev, sizeof(float), cudaMemcpyDeviceToHost, st));
    if (grads_host)
      CAV_CHECK_CUDA(cudaMemcpyAsync(grads_host, net->g, sizeof(float) * net->n_params, cudaMemcpyDeviceToHost, st));
    CAV_CHECK_CUDA(cudaStreamSynchronize(st));
    return IB_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

ib_status ibnet_train_step(ibnet* net, const float* in, const float* target, int32_t batch, int32_t N, float lr,
                           float* loss_host, cudaStream_t st) {
  try {
    CAV_REQUIRE(net && in && target && batch >= 1 && N >= 1 && lr > 0, "ibnet_train_step: bad argument");
    net_forward(net, in, nullptr, batch, N, st);
    net_backward(net, target, batch, N, st);
    net->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - (float)std::pow(b1, (double)net->t), c2 = 1.f - (float)std::pow(b2, (double)net->t);
    k_adam<<<grid_for(net->n_params), 256, 0, st>>>(net->p, net->g, net->m, net->v, net->n_params, lr, b1, b2, 1e-8f,
                                                     c1, c2);
    CAV_CHECK_LAUNCH();
    if (loss_host) {
      CAV_CHECK_CUDA(cudaMemcpyAsync(loss_host, net->loss_dev, sizeof(float), cudaMemcpyDeviceToHost, st));
      CAV_CHECK_CUDA(cudaStreamSynchronize(st));
    }
    return IB_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

ib_status ibnet_pack_input(int32_t N, const double* const* hist_x, const double* const* hist_f,
                           const float* in_scale, float* out, cudaStream_t st) {
  try {
    CAV_REQUIRE(N >= 1 && hist_x && hist_f && in_scale && out, "ibnet_pack_input: NULL argument");
    PackPtrs P;
    for (int t = 0; t < 3; ++t) {
      CAV_REQUIRE(hist_x[t] && hist_f[t], "ibnet_pack_input: NULL history entry");
      P.x[t] = hist_x[t];
      P.f[t] = hist_f[t];
    }
    for (int c = 0; c < 15; ++c) {
      CAV_REQUIRE(in_scale[c] > 0.f, "ibnet_pack_input: scales must be positive");
      P.inv_scale[c] = 1.f / in_scale[c];
    }
    const size_t n = 15ull * N * N;
    k_pack_input<<<grid_for(n), 256, 0, st>>>(P, N, out);
    CAV_CHECK_LAUNCH();
    return IB_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

ib_status ibnet_pack_history(int32_t N, int32_t K, const double* const* hist_x, const double* const* hist_f,
                             const float* in_scale, float* out, cudaStream_t st) {
  try {
    CAV_REQUIRE(N >= 1 && hist_x && hist_f && in_scale && out, "ibnet_pack_history: NULL argument");
    CAV_REQUIRE(K >= 1 && K <= 4, "ibnet_pack_history: K must be in [1, 4]");
    HistPtrs P{};
    P.K = K;
    for (int t = 0; t < K; ++t) {
      CAV_REQUIRE(hist_x[t] && hist_f[t], "ibnet_pack_history: NULL history entry");
      P.x[t] = hist_x[t];
      P.f[t] = hist_f[t];
    }
    for (int c = 0; c < 5 * K; ++c) {
      CAV_REQUIRE(in_scale[c] > 0.f, "ibnet_pack_history: scales must be positive");
      P.inv_scale[c] = 1.f / in_scale[c];
    }
    const size_t n = 5ull * K * N * N;
    k_pack_history<<<grid_for(n), 256, 0, st>>>(P, N, out);
    CAV_CHECK_LAUNCH();
    return IB_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

ib_status ibnet_pack_target(int32_t N, const double* x_new, const double* x_prev, const double* x_prev2,
                            const double* x_prev3, const float* out_scale, float* out, cudaStream_t st) {
  try {
    CAV_REQUIRE(N >= 1 && x_new && x_prev && out_scale && out, "ibnet_pack_target: NULL argument");
    CAV_REQUIRE(!x_prev3 || x_prev2, "ibnet_pack_target: x_prev3 needs x_prev2");
    const size_t n = 3ull * N * N;
    k_pack_target<<<grid_for(n), 256, 0, st>>>(x_new, x_prev, x_prev2, x_prev3, out_scale[0], out_scale[1],
                                               out_scale[2], N, out);
    CAV_CHECK_LAUNCH();
    return IB_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

ib_status ibnet_apply_delta(int32_t N, const double* x_prev, const double* x_prev2, const double* x_prev3,
                            const float* delta, const float* out_scale, double* x_out, cudaStream_t st) {
  try {
    CAV_REQUIRE(N >= 1 && x_prev && out_scale && x_out, "ibnet_apply_delta: NULL argument");
    CAV_REQUIRE(!x_prev3 || x_prev2, "ibnet_apply_delta: x_prev3 needs x_prev2");
    const size_t n = 3ull * N * N;
    k_apply_delta<<<grid_for(n), 256, 0, st>>>(x_prev, x_prev2, x_prev3, delta, out_scale[0], out_scale[1],
                                               out_scale[2], N, x_out);
    CAV_CHECK_LAUNCH();
    return IB_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

}  // extern "C"
