// Deterministic reductions and scans used by set-up and by the Krylov solver.
#include <string>

#include "internal.cuh"
#include "device_util.cuh"

namespace cav {

static constexpr int SCAN_BLOCK = 1024;

// In-place exclusive scan of one 1024-element chunk per block; block totals to `sums`.
__global__ void k_scan_chunk(int64_t* data, int64_t n, int64_t* sums) {
  __shared__ int64_t warp_tot[32];
  const int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
  int64_t v = (i < n) ? data[i] : 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t t = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;  // inclusive over warps
  }
  __syncthreads();
  const int64_t before = (warp > 0 ? warp_tot[warp - 1] : 0) + x - v;
  if (i < n) data[i] = before;
  if (threadIdx.x == SCAN_BLOCK - 1) sums[blockIdx.x] = warp_tot[31];
}

__global__ void k_scan_add(int64_t* data, int64_t n, const int64_t* offs) {
  const int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
  if (i < n) data[i] += offs[blockIdx.x];
}

__global__ void k_widen(const int* in, int64_t* out, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i];
  if (i == n) out[n] = 0;
}

__global__ void k_set_total(int64_t* out, int64_t n, const int* counts) {
  // out[n] = out[n-1] + counts[n-1]
  out[n] = (n > 0) ? out[n - 1] + counts[n - 1] : 0;
}

static void scan_inplace(int64_t* data, int64_t n, cudaStream_t st, Arena* scratch) {
  if (n <= 0) return;
  const int nb = div_up(n, SCAN_BLOCK);
  int64_t* sums = scratch->alloc<int64_t>(nb);
  k_scan_chunk<<<nb, SCAN_BLOCK, 0, st>>>(data, n, sums);
  CAV_CHECK_LAUNCH();
  if (nb > 1) {
    scan_inplace(sums, nb, st, scratch);
    k_scan_add<<<nb, SCAN_BLOCK, 0, st>>>(data, n, sums);
    CAV_CHECK_LAUNCH();
  }
}

void exclusive_scan(const int* counts, int64_t* out, int64_t n, cudaStream_t st, Arena* scratch) {
  k_widen<<<div_up(n + 1, 256), 256, 0, st>>>(counts, out, n);
  CAV_CHECK_LAUNCH();
  scan_inplace(out, n, st, scratch);
  k_set_total<<<1, 1, 0, st>>>(out, n, counts);
  CAV_CHECK_LAUNCH();
}

int reduce_blocks(int64_t n) {
  int nb = div_up(n, 2048);
  if (nb < 1) nb = 1;
  if (nb > 512) nb = 512;
  return nb;
}

static constexpr int RED_THREADS = 256;

// partial[b] = sum over the b-th strided share of a[i] * b[i] (fixed order)
__global__ void k_dot_partials(const double* __restrict__ a, const double* __restrict__ b,
                               int64_t n, double* partial) {
  __shared__ double sm[RED_THREADS / 32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  s = block_sum(s, sm);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

void launch_dot_partials(const double* a, const double* b, int64_t n, double* partial,
                         cudaStream_t st) {
  k_dot_partials<<<reduce_blocks(n), RED_THREADS, 0, st>>>(a, b, n, partial);
  CAV_CHECK_LAUNCH();
}

// out[0] = sum of partial[0 .. nb) in a fixed order (one block)
__global__ void k_sum_partials(const double* __restrict__ partial, int nb, double* out) {
  __shared__ double sm[RED_THREADS / 32];
  double s = 0.0;
  for (int q = threadIdx.x; q < nb; q += blockDim.x) s += partial[q];
  s = block_sum(s, sm);
  if (threadIdx.x == 0) out[0] = s;
}

double device_dot(const double* a, const double* b, int64_t n, double* partial, cudaStream_t st) {
  const int nb = reduce_blocks(n);
  k_dot_partials<<<nb, RED_THREADS, 0, st>>>(a, b, n, partial);
  CAV_CHECK_LAUNCH();
  k_sum_partials<<<1, RED_THREADS, 0, st>>>(partial, nb, partial + nb);
  CAV_CHECK_LAUNCH();
  double h = 0.0;
  CAV_CHECK_CUDA(cudaMemcpyAsync(&h, partial + nb, sizeof(double), cudaMemcpyDeviceToHost, st));
  CAV_CHECK_CUDA(cudaStreamSynchronize(st));
  return h;
}

int read_status(int* d_status, cudaStream_t st) {
  int h = 0;
  CAV_CHECK_CUDA(cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CAV_CHECK_CUDA(cudaStreamSynchronize(st));
  return h;
}

std::string status_message(int code) {
  switch (code) {
    case DEV_TIMEOUT:
      return "a bounded device-side wait ran out (a TMA copy or a pipeline stage did not arrive in time); "
             "the call's output is not valid";
    case DEV_WINDOW: return "a stencil window overflowed";
    case DEV_SINGULAR: return "zero pivot in a local patch matrix";
    case DEV_CAPACITY: return "a device-side capacity was exceeded";
    default: return "device status code " + std::to_string(code);
  }
}

ib_status status_of(int code) {
  if (code == DEV_OK) return IB_OK;
  if (code == DEV_TIMEOUT) return IB_ERR_TIMEOUT;
  if (code == DEV_SINGULAR) return IB_ERR_SINGULAR;
  return IB_ERR_INTERNAL;
}

ib_status take_status(int* d_status, cudaStream_t st, const char* who) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CAV_CHECK_CUDA(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return IB_OK;
  const int code = read_status(d_status, st);
  if (code == DEV_OK) return IB_OK;
  CAV_CHECK_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), st));
  CAV_CHECK_CUDA(cudaStreamSynchronize(st));
  set_error(std::string(who) + ": " + status_message(code));
  return status_of(code);
}

}  // namespace cav
