// Device-side helpers: periodic indexing, stencil windows, warp reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cav {

// Programmatic dependent launch.  A kernel launched with programmatic stream serialization
// may start before the kernel ahead of it in the stream has finished: pdl_trigger() lets the
// next kernel launch, pdl_wait() blocks until the kernel ahead has completed and its writes are
// visible.  A kernel launched that way calls pdl_wait() in each CTA before reading data an
// earlier kernel wrote or writing data it reads.  Without a programmatic launch both are no-ops.
__device__ inline void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ inline void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__host__ __device__ inline int pmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// A window of one periodic axis: global coordinates base, base+1, ..., base+len-1 (mod N).
// When 2W+1 >= N the window is the whole axis (base 0, len N).  Walking t' = 0..len-1 with
// t = (t0 + t') % len visits the window's global coordinates in ascending order.
struct Win {
  int base, len, t0;
};

__device__ inline Win make_win(int c, int W, int N) {
  Win w;
  if (2 * W + 1 >= N) {
    w.base = 0;
    w.len = N;
    w.t0 = 0;
  } else {
    w.base = pmod(c - W, N);
    w.len = 2 * W + 1;
    w.t0 = (w.base + w.len > N) ? (N - w.base) : 0;
  }
  return w;
}
// window offset of global coordinate g, or -1 if outside
__device__ inline int win_off(const Win& w, int g, int N) {
  int o = pmod(g - w.base, N);
  return o < w.len ? o : -1;
}
__device__ inline int win_glob(const Win& w, int t, int N) { return (w.base + t) % N; }
__device__ inline int win_asc(const Win& w, int tp) { return (w.t0 + tp) % w.len; }

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block sum (deterministic for a fixed blockDim); every thread gets the total.
// smem must hold blockDim.x / 32 doubles.
__device__ inline double block_sum(double v, double* smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += smem[i];
  return t;
}

// Peskin's four-point kernel (the kernel named in Sec. 2 of the paper).
__device__ inline double phi4(double r) {
  r = fabs(r);
  if (r <= 1.0) return (3.0 - 2.0 * r + sqrt(1.0 + 4.0 * r - 4.0 * r * r)) / 8.0;
  if (r < 2.0) return (5.0 - 2.0 * r - sqrt(-7.0 + 12.0 * r - 4.0 * r * r)) / 8.0;
  return 0.0;
}

// Reciprocal power of two of a positive max-norm m: 2^-e with m = f 2^e, f in [1/2, 1).
__device__ inline double pow2_recip(double m) {
  int e;
  frexp(m, &e);
  return ldexp(1.0, -e);
}

}  // namespace cav
