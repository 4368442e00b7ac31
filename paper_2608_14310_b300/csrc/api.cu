// C ABI entry points (include/ib_cav.h).  Every call catches library failures and turns
// them into an ib_status with a thread-local message.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

#include <atomic>

namespace cav {
static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};
void set_error(const std::string& msg) { g_last_error = msg; }
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(); }
static std::atomic<uint64_t> g_uid{0};
uint64_t next_uid() { return g_uid.fetch_add(1, std::memory_order_relaxed) + 1; }
ib_status fgmres_run(const ib_system* sys, cav_hierarchy* H, const double* b, double* x, const fgmres_desc* d,
                     fgmres_info* info, double* history, cudaStream_t st);
ib_status fgmres_run_device(const ib_system* sys, cav_hierarchy* H, const double* b, double* x,
                            const fgmres_desc* d, fgmres_info* info, double* history, cudaStream_t st);
ib_status fgmres_run_batched_device(int count, const ib_system* const* sys, cav_hierarchy* const* H,
                                    const double* const* b, double* const* x, const fgmres_desc* d,
                                    fgmres_info* infos, cudaStream_t st);
ib_status fgmres_run_batched(int count, const ib_system* const* sys, cav_hierarchy* const* H,
                             const double* const* b, double* const* x, const fgmres_desc* d,
                             fgmres_info* infos, cudaStream_t st);
}  // namespace cav

using namespace cav;

#define CAV_API_BEGIN try {
#define CAV_API_END                                   \
  }                                                   \
  catch (const Fail& f) {                             \
    return f.st;                                      \
  }                                                   \
  catch (const std::exception& e) {                   \
    set_error(std::string("internal: ") + e.what());  \
    return IB_ERR_INTERNAL;                           \
  }                                                   \
  catch (...) {                                       \
    set_error("internal: unknown exception");         \
    return IB_ERR_INTERNAL;                           \
  }

extern "C" {

const char* ib_last_error(void) { return g_last_error.c_str(); }
int ib_abi_version(void) { return 5; }
int64_t ib_launch_count(void) { return g_launches.load(); }

ib_status ib_setup(const ib_grid_desc* grid, const ib_structure_desc* sd, cudaStream_t st, ib_system** out) {
  if (!out) { set_error("ib_setup: out is NULL"); return IB_ERR_INVALID; }
  *out = nullptr;
  ib_system* s = nullptr;
  CAV_API_BEGIN
  CAV_REQUIRE(grid && sd, "ib_setup: NULL descriptor");
  CAV_REQUIRE(grid->N >= 8 && grid->N <= 16384, "ib_setup: N must be in [8, 16384]");
  CAV_REQUIRE(grid->L > 0 && grid->rho > 0 && grid->mu >= 0 && grid->dt > 0,
              "ib_setup: L, rho, dt must be positive and mu non-negative");
  CAV_REQUIRE(grid->bc == IB_BC_PERIODIC || grid->bc == IB_BC_CHANNEL, "ib_setup: unknown boundary condition");
  if (grid->bc == IB_BC_CHANNEL && sd->M > 0 && sd->X) {
    // E_E, S and J are assembled as on the periodic grid: the markers' four-point supports
    // must stay clear of the top and bottom walls (no wrap in y)
    const double h = grid->L / grid->N;
    for (int a = 0; a < sd->M; ++a) {
      const double y = sd->X[2 * a + 1];
      CAV_REQUIRE(y >= 2.5 * h && y <= grid->L - 2.5 * h,
                  "ib_setup: on the channel every marker must lie at least 2.5 h from the top and bottom "
                  "walls (its kernel support may not reach them)");
    }
  }
  CAV_REQUIRE(sd->M >= 0, "ib_setup: M must be non-negative");
  CAV_REQUIRE(sd->M == 0 || (sd->X && sd->omega), "ib_setup: X and omega are required when M > 0");
  CAV_REQUIRE(sd->law >= IB_FORCE_TARGET && sd->law <= IB_FORCE_FIBER, "ib_setup: unknown force law");
  s = new ib_system();
  s->uid = next_uid();
  s->N = grid->N;
  s->L = grid->L;
  s->h = grid->L / grid->N;
  s->rho = grid->rho;
  s->mu = grid->mu;
  s->dt = grid->dt;
  s->bc = grid->bc;
  s->law = sd->law;
  s->closed = sd->closed ? 1 : 0;
  s->ds = sd->ds;
  s->k_target = sd->k_target;
  s->k_stretch = sd->k_stretch;
  s->k_bend = sd->k_bend;
  s->k_pos = sd->k_pos;
  s->k_tan = sd->k_tan;
  s->clamp_x = sd->clamp_x;
  s->clamp_y = sd->clamp_y;
  CAV_CHECK_CUDA(cudaGetDevice(&s->device));
  // structural band of E: target -> diagonal; membrane -> +-1 when k_stretch != 0;
  // beam -> +-2 when k_bend != 0, else +-1 when k_stretch != 0; otherwise no structure
  int M = sd->M, bw = 0;
  if (sd->law == IB_FORCE_TARGET) bw = 0;
  else if (sd->law == IB_FORCE_FIBER) {
    // bending couples markers two links apart; the tangent couples x and y
    if (M > 0) {
      CAV_REQUIRE(!sd->closed, "ib_setup: the fiber law needs an open marker chain");
      CAV_REQUIRE(M >= 3 && M % 2 == 1, "ib_setup: the fiber law needs an odd number of markers, at least 3");
      CAV_REQUIRE(sd->ds > 0, "ib_setup: ds must be positive");
      CAV_REQUIRE(sd->k_target == 0.0, "ib_setup: the fiber law takes no tethers (k_target must be 0)");
      bw = 2;
    }
  } else if (sd->law == IB_FORCE_MEMBRANE) {
    if (sd->k_stretch != 0.0) bw = 1;
    else if (sd->k_target != 0.0) bw = 0;
    else M = 0;
  } else {
    if (sd->k_bend != 0.0) bw = 2;
    else if (sd->k_stretch != 0.0) bw = 1;
    else if (sd->k_target != 0.0) bw = 0;
    else M = 0;
  }
  if (M > 0 && bw > 0 && sd->law != IB_FORCE_FIBER) {
    CAV_REQUIRE(sd->closed, "ib_setup: membrane and beam laws need a closed marker chain");
    CAV_REQUIRE(M >= 2 * bw + 1, "ib_setup: too few markers for the force stencil");
    CAV_REQUIRE(sd->ds > 0, "ib_setup: ds must be positive");
  }
  s->M = M;
  s->bw = bw;
  s->status = s->arena.alloc<int>(1);
  s->partial = s->arena.alloc<double>(reduce_blocks(3LL * s->N * s->N) + 1);
  CAV_CHECK_CUDA(cudaMemsetAsync(s->status, 0, sizeof(int), st));
  build_markers_and_ee(s, sd->X, sd->X_lin ? sd->X_lin : sd->X, sd->omega, st);
  if (M > 0) {
    s->X_host.assign(sd->X, sd->X + 2 * (size_t)M);
    if (sd->X_target) {
      std::vector<double> cm(2 * (size_t)M);
      for (int a = 0; a < M; ++a) {
        cm[a] = sd->X_target[2 * a];
        cm[M + a] = sd->X_target[2 * a + 1];
      }
      s->Xt = s->arena.alloc<double>(2 * M);
      CAV_CHECK_CUDA(cudaMemcpyAsync(s->Xt, cm.data(), sizeof(double) * 2 * M, cudaMemcpyHostToDevice, st));
      CAV_CHECK_CUDA(cudaStreamSynchronize(st));
    }
  }
  const int code = read_status(s->status, st);
  if (code != DEV_OK) {
    set_error("ib_setup: E_E assembly window overflow");
    throw Fail{IB_ERR_INTERNAL};
  }
  *out = s;
  return IB_OK;
  }
  catch (const Fail& f) {
    if (s) { s->arena.release(); delete s; }
    return f.st;
  }
  catch (...) {
    if (s) { s->arena.release(); delete s; }
    set_error("ib_setup: internal error");
    return IB_ERR_INTERNAL;
  }
}

ib_status ib_update_structure(ib_system* s, const ib_structure_desc* sd, cudaStream_t st) {
  CAV_API_BEGIN
  CAV_REQUIRE(s && sd, "ib_update_structure: NULL argument");
  int device = -1;
  CAV_CHECK_CUDA(cudaGetDevice(&device));
  CAV_REQUIRE(device == s->device, "ib_update_structure: the current device is not the system's device");
  ib_grid_desc g;
  g.N = s->N;
  g.L = s->L;
  g.rho = s->rho;
  g.mu = s->mu;
  g.dt = s->dt;
  g.bc = s->bc;
  ib_system* fresh = nullptr;
  const ib_status r = ib_setup(&g, sd, st, &fresh);
  if (r != IB_OK) return r;  // the handle keeps its previous configuration
  const uint64_t uid = s->uid, epoch = s->epoch;
  std::swap(*s, *fresh);
  s->uid = uid;  // the same handle, new buffers: solve graphs built with it are rebuilt
  s->epoch = epoch + 1;
  ib_destroy(fresh);  // now holds the previous configuration's device memory
  return IB_OK;
  CAV_API_END
}

static LevelOps sys_ops(const ib_system* s) {
  LevelOps o{s->N, s->h, s->rho / s->dt, s->mu, s->dt, &s->ee, s->bc == IB_BC_CHANNEL};
  return o;
}

ib_status ib_apply(const ib_system* s, const double* x, double* y, cudaStream_t st) {
  CAV_API_BEGIN
  CAV_REQUIRE(s && x && y, "ib_apply: NULL argument");
  launch_apply(sys_ops(s), x, nullptr, y, 1, st);
  return IB_OK;
  CAV_API_END
}

ib_status ib_residual(const ib_system* s, const double* b, const double* x, double* r, cudaStream_t st) {
  CAV_API_BEGIN
  CAV_REQUIRE(s && b && x && r, "ib_residual: NULL argument");
  launch_apply(sys_ops(s), x, b, r, 0, st);
  return IB_OK;
  CAV_API_END
}

ib_status ib_force(const ib_system* s, double* F, cudaStream_t st) {
  CAV_API_BEGIN
  CAV_REQUIRE(s && F, "ib_force: NULL argument");
  ib_force_launch(s, F, st);
  return IB_OK;
  CAV_API_END
}

ib_status ib_spread(const ib_system* s, const double* F, double* f, cudaStream_t st) {
  CAV_API_BEGIN
  CAV_REQUIRE(s && f && (F || s->M == 0), "ib_spread: NULL argument");
  ib_spread_launch(s, F, f, 0, nullptr, nullptr, st);
  return IB_OK;
  CAV_API_END
}

ib_status ib_interp(const ib_system* s, const double* u, double* U, cudaStream_t st) {
  CAV_API_BEGIN
  CAV_REQUIRE(s && u && (U || s->M == 0), "ib_interp: NULL argument");
  ib_interp_launch(s, u, U, 0.0, st);
  return IB_OK;
  CAV_API_END
}

ib_status ib_step_rhs(const ib_system* s, const double* u_prev, const double* f_body, double* b, cudaStream_t st) {
  CAV_API_BEGIN
  CAV_REQUIRE(s && b, "ib_step_rhs: NULL argument");
  ib_force_launch(s, s->F, st);
  ib_spread_launch(s, s->F, b, 1, u_prev, f_body, st);
  return IB_OK;
  CAV_API_END
}

ib_status ib_advect(const ib_system* s, const double* u, double* X_next, cudaStream_t st) {
  CAV_API_BEGIN
  CAV_REQUIRE(s && u && X_next, "ib_advect: NULL argument");
  const int M = s->M;
  if (M == 0) return IB_OK;
  ib_interp_launch(s, u, s->U, s->dt, st);
  std::vector<double> cm(2 * (size_t)M);
  CAV_CHECK_CUDA(cudaMemcpyAsync(cm.data(), s->U, sizeof(double) * 2 * M, cudaMemcpyDeviceToHost, st));
  CAV_CHECK_CUDA(cudaStreamSynchronize(st));
  for (int a = 0; a < M; ++a) {
    X_next[2 * a] = cm[a];
    X_next[2 * a + 1] = cm[M + a];
  }
  return IB_OK;
  CAV_API_END
}

void ib_destroy(ib_system* s) {
  if (!s) return;
  cudaDeviceSynchronize();
  s->arena.release();
  delete s;
}

ib_status cav_setup(const ib_system* s, const cav_desc* d, cudaStream_t st, cav_hierarchy** out) {
  if (!out) { set_error("cav_setup: out is NULL"); return IB_ERR_INVALID; }
  *out = nullptr;
  cav_hierarchy* H = nullptr;
  try {
    CAV_REQUIRE(s && d, "cav_setup: NULL argument");
    CAV_REQUIRE(d->kind == CAV_PATCH_CAV || d->kind == CAV_PATCH_VANKA || d->kind == CAV_PATCH_BOX,
                "cav_setup: unknown patch kind");
    if (d->kind == CAV_PATCH_BOX) {
      CAV_REQUIRE(d->smoother == CAV_SMOOTH_COLOURED && d->coloured_levels == 0,
                  "cav_setup: box patches use the multiplicative (coloured) smoother on every level");
      CAV_REQUIRE(d->box_b >= 1 && d->box_o >= 0 && d->box_b + 2 * d->box_o <= 16,
                  "cav_setup: box patches need b >= 1, o >= 0 and b + 2 o <= 16");
    }
    CAV_REQUIRE(d->coarsest_N >= 2, "cav_setup: coarsest_N must be >= 2");
    CAV_REQUIRE(d->nu_pre >= 0 && d->nu_post >= 0 && d->nu_pre + d->nu_post >= 1,
                "cav_setup: need at least one sweep per level");
    CAV_REQUIRE(d->precision >= CAV_PREC_FP64 && d->precision <= CAV_PREC_BF16, "cav_setup: unknown precision");
    CAV_REQUIRE(std::isfinite(d->alpha) && d->alpha > 0, "cav_setup: alpha must be positive");
    CAV_REQUIRE(d->krylov_capacity >= 0 && d->krylov_capacity <= 4096, "cav_setup: bad krylov_capacity");
    CAV_REQUIRE(d->smoother == CAV_SMOOTH_ADDITIVE || d->smoother == CAV_SMOOTH_COLOURED,
                "cav_setup: unknown smoother");
    CAV_REQUIRE(d->coloured_levels >= 0 && d->nu_additive >= 0, "cav_setup: negative coloured_levels or nu_additive");
    CAV_REQUIRE(!(d->smoother == CAV_SMOOTH_COLOURED && d->precision == CAV_PREC_BF16),
                "cav_setup: the coloured (multiplicative) smoother needs FP32 or FP64 patch inverses: with "
                "BF16-rounded inverses the undamped sweep diverges");
    H = new cav_hierarchy();
    H->uid = next_uid();
    H->sys = s;
    H->desc = *d;
    H->grid_N = s->N;
    H->grid_bc = s->bc;
    H->grid_L = s->L;
    H->grid_rho = s->rho;
    H->grid_mu = s->mu;
    H->grid_dt = s->dt;
    H->status = H->arena.alloc<int>(1);
    H->flag = H->arena.alloc<int>(1);
    H->gbar = H->arena.alloc<unsigned>(CAV_GBAR_WORDS);
    CAV_CHECK_CUDA(cudaMemsetAsync(H->status, 0, sizeof(int), st));
    CAV_CHECK_CUDA(cudaMemsetAsync(H->gbar, 0, CAV_GBAR_WORDS * sizeof(unsigned), st));
    build_levels(H, st);
    *out = H;
    return IB_OK;
  } catch (const Fail& f) {
    if (H) { cudaDeviceSynchronize(); H->arena.release(); delete H; }
    return f.st;
  } catch (...) {
    if (H) { cudaDeviceSynchronize(); H->arena.release(); delete H; }
    set_error("cav_setup: internal error");
    return IB_ERR_INTERNAL;
  }
}

ib_status cav_refactor(cav_hierarchy* h, const ib_system* s, cudaStream_t st) {
  CAV_API_BEGIN
  CAV_REQUIRE(h && s, "cav_refactor: NULL argument");
  CAV_REQUIRE(h->grid_N == s->N && h->grid_L == s->L && h->grid_rho == s->rho && h->grid_mu == s->mu &&
                  h->grid_dt == s->dt && h->grid_bc == s->bc,
              "cav_refactor: the system's grid or parameters differ from the hierarchy's");
  int device = -1;
  CAV_CHECK_CUDA(cudaGetDevice(&device));
  CAV_REQUIRE(device == s->device, "cav_refactor: the current device is not the system's device");
  if (!same_ee_pattern(s->ee, h->levels[0].ee, h->flag, st)) {
    set_error("cav_refactor: E_E's structural pattern changed (markers moved across faces): use cav_setup");
    return IB_ERR_INVALID;
  }
  refactor_levels(h, s, st);
  ++h->epoch;  // a cached solve graph may hold the previous values (e.g. kernel arguments)
  return IB_OK;
  CAV_API_END
}

ib_status cav_num_levels(const cav_hierarchy* h, int32_t* levels) {
  CAV_API_BEGIN
  CAV_REQUIRE(h && levels, "cav_num_levels: NULL argument");
  *levels = (int32_t)h->levels.size();
  return IB_OK;
  CAV_API_END
}

static const Level& level_of(const cav_hierarchy* h, int32_t level) {
  CAV_REQUIRE(h, "NULL hierarchy");
  CAV_REQUIRE(level >= 0 && level < (int32_t)h->levels.size(), "level out of range");
  return h->levels[level];
}

ib_status cav_get_level_info(const cav_hierarchy* h, int32_t level, cav_level_info* info) {
  CAV_API_BEGIN
  CAV_REQUIRE(info, "cav_get_level_info: NULL info");
  const Level& lv = level_of(h, level);
  std::memset(info, 0, sizeof(*info));
  const int64_t NN = (int64_t)lv.N * lv.N;
  info->N = lv.N;
  info->is_coarsest = lv.coarsest ? 1 : 0;
  info->ee_nnz = lv.ee.nnz;
  info->ee_rows = lv.ee.n_rows;
  info->ee_window = lv.ee.W;
  if (lv.coarsest) {
    info->n_patches = 1;
    info->max_n = (int32_t)(3 * NN);
    info->sum_n = 3 * NN;
    info->sum_n2 = 9 * NN * NN;
  } else {
    const int64_t nstd = lv.box ? 0 : NN - lv.n_big;  // n_std4 of them have four unknowns
    info->n_patches = (int32_t)(lv.box ? lv.n_big : NN);
    info->n_enlarged = lv.n_big - lv.n_big_small;
    info->max_n = lv.box ? lv.big_max_n : std::max(lv.big_max_n, nstd > lv.n_std4 ? 5 : 4);
    info->sum_n = lv.big_sum_n + 5 * nstd - lv.n_std4;
    info->sum_n2 = lv.big_sum_n2 + 25 * nstd - 9 * (int64_t)lv.n_std4;
    info->enlarged_sum_n = lv.big_sum_n;
    info->enlarged_sum_n2 = lv.big_sum_n2;
    const int bytes = (lv.precision == CAV_PREC_FP64) ? 8 : (lv.precision == CAV_PREC_FP32 ? 4 : 2);
    info->inverse_bytes = lv.inv_elems * bytes;
    info->apply_variant = lv.apply_variant;
    for (int v = 0; v < 5; ++v) info->apply_us[v] = lv.apply_us[v];
    info->n_colours = lv.n_colours;
    info->sweep_form = lv.fused;
    info->sweep_us[0] = lv.sweep_us[0];
    info->sweep_us[1] = lv.sweep_us[1];
  }
  return IB_OK;
  CAV_API_END
}

ib_status cav_patch_export(const cav_hierarchy* h, int32_t level, int64_t* offsets, int32_t* dofs,
                           int32_t* n_patches, int64_t* sum_n) {
  CAV_API_BEGIN
  const Level& lv = level_of(h, level);
  CAV_REQUIRE(!lv.coarsest, "cav_patch_export: the coarsest level has no patches");
  const int N = lv.N, NN = N * N;
  const int64_t total = lv.big_sum_n + (lv.box ? 0 : 5LL * (NN - lv.n_big) - lv.n_std4);
  if (n_patches) *n_patches = lv.box ? lv.n_big : NN;
  if (sum_n) *sum_n = total;
  if (!offsets || !dofs) return IB_OK;
  if (lv.box) {  // one patch per block, every one stored explicitly
    std::vector<int64_t> off(lv.n_big + 1);
    CAV_CHECK_CUDA(cudaMemcpy(off.data(), lv.big_off, sizeof(int64_t) * (lv.n_big + 1), cudaMemcpyDeviceToHost));
    for (int p = 0; p <= lv.n_big; ++p) offsets[p] = off[p];
    if (lv.big_sum_n)
      CAV_CHECK_CUDA(cudaMemcpy(dofs, lv.big_dofs, sizeof(int) * lv.big_sum_n, cudaMemcpyDeviceToHost));
    return IB_OK;
  }
  std::vector<uint8_t> big(NN);
  std::vector<int> cells(lv.n_big);
  std::vector<int64_t> off(lv.n_big + 1);
  std::vector<int> bd(lv.big_sum_n);
  CAV_CHECK_CUDA(cudaMemcpy(big.data(), lv.cell_big, NN, cudaMemcpyDeviceToHost));
  if (lv.n_big) {
    CAV_CHECK_CUDA(cudaMemcpy(cells.data(), lv.big_cell, sizeof(int) * lv.n_big, cudaMemcpyDeviceToHost));
    CAV_CHECK_CUDA(cudaMemcpy(off.data(), lv.big_off, sizeof(int64_t) * (lv.n_big + 1), cudaMemcpyDeviceToHost));
    CAV_CHECK_CUDA(cudaMemcpy(bd.data(), lv.big_dofs, sizeof(int) * lv.big_sum_n, cudaMemcpyDeviceToHost));
  }
  int64_t pos = 0;
  int q = 0;
  for (int c = 0; c < NN; ++c) {
    offsets[c] = pos;
    if (big[c]) {
      for (int64_t t = off[q]; t < off[q + 1]; ++t) dofs[pos++] = bd[t];
      ++q;
    } else {
      const int i = c % N, j = c / N;
      int v[5] = {j * N + i, j * N + (i + 1) % N, NN + j * N + i, NN + ((j + 1) % N) * N + i, 2 * NN + j * N + i};
      int len = 5;
      if (lv.channel && j + 1 == N) {  // the inflow row: no v_{i,N}
        v[3] = v[4];
        len = 4;
      }
      std::sort(v, v + len);
      for (int t = 0; t < len; ++t) dofs[pos++] = v[t];
    }
  }
  offsets[NN] = pos;
  return IB_OK;
  CAV_API_END
}

ib_status cav_colour_export(const cav_hierarchy* h, int32_t level, int32_t* colour_of_cell, int32_t* n_colours) {
  CAV_API_BEGIN
  const Level& lv = level_of(h, level);
  CAV_REQUIRE(!lv.coarsest, "cav_colour_export: the coarsest level has no patches");
  CAV_REQUIRE(lv.coloured, "cav_colour_export: this level's smoother is additive");
  if (n_colours) *n_colours = lv.n_colours;
  if (colour_of_cell)
    for (size_t c = 0; c < lv.colour_of_cell.size(); ++c) colour_of_cell[c] = lv.colour_of_cell[c];
  return IB_OK;
  CAV_API_END
}

ib_status cav_ee_export(const cav_hierarchy* h, int32_t level, int64_t* rowptr, int32_t* cols, double* vals,
                        int64_t* nnz) {
  CAV_API_BEGIN
  const Level& lv = level_of(h, level);
  const int NN = lv.N * lv.N;
  if (nnz) *nnz = lv.ee.nnz;
  if (!rowptr || !cols || !vals) return IB_OK;
  std::vector<int> rows(lv.ee.n_rows);
  std::vector<int64_t> rp(lv.ee.n_rows + 1, 0);
  std::vector<int> c(lv.ee.nnz);
  std::vector<double> v(lv.ee.nnz);
  if (lv.ee.n_rows) {
    CAV_CHECK_CUDA(cudaMemcpy(rows.data(), lv.ee.rows, sizeof(int) * lv.ee.n_rows, cudaMemcpyDeviceToHost));
    CAV_CHECK_CUDA(cudaMemcpy(rp.data(), lv.ee.rowptr, sizeof(int64_t) * (lv.ee.n_rows + 1), cudaMemcpyDeviceToHost));
    CAV_CHECK_CUDA(cudaMemcpy(c.data(), lv.ee.cols, sizeof(int) * lv.ee.nnz, cudaMemcpyDeviceToHost));
    CAV_CHECK_CUDA(cudaMemcpy(v.data(), lv.ee.vals, sizeof(double) * lv.ee.nnz, cudaMemcpyDeviceToHost));
  }
  int64_t pos = 0;
  int q = 0;
  for (int r = 0; r < 2 * NN; ++r) {
    rowptr[r] = pos;
    if (q < lv.ee.n_rows && rows[q] == r) {
      for (int64_t t = rp[q]; t < rp[q + 1]; ++t) {
        cols[pos] = c[t];
        vals[pos] = v[t];
        ++pos;
      }
      ++q;
    }
  }
  rowptr[2 * NN] = pos;
  return IB_OK;
  CAV_API_END
}

ib_status cav_sweep(const cav_hierarchy* h, int32_t level, const double* b, double* w, cudaStream_t st) {
  CAV_API_BEGIN
  const Level& lv = level_of(h, level);
  CAV_REQUIRE(!lv.coarsest, "cav_sweep: no smoother on the coarsest level");
  CAV_REQUIRE(b && w, "cav_sweep: NULL vector");
  level_sweep(h, level, b, w, false, st);
  return take_status(h->status, st, "cav_sweep");
  CAV_API_END
}

ib_status cav_residual(const cav_hierarchy* h, int32_t level, const double* b, const double* w, double* r,
                       cudaStream_t st) {
  CAV_API_BEGIN
  const Level& lv = level_of(h, level);
  CAV_REQUIRE(b && w && r, "cav_residual: NULL vector");
  LevelOps o{lv.N, lv.h, lv.rho_dt, lv.mu, lv.dt, &lv.ee, lv.channel};
  launch_apply(o, w, b, r, 0, st);
  return IB_OK;
  CAV_API_END
}

ib_status cav_restrict(const cav_hierarchy* h, int32_t level, const double* r, double* bc, cudaStream_t st) {
  CAV_API_BEGIN
  const Level& lv = level_of(h, level);
  CAV_REQUIRE(!lv.coarsest && r && bc, "cav_restrict: bad level or NULL vector");
  launch_restrict(lv.N / 2, r, bc, lv.channel, st);
  return IB_OK;
  CAV_API_END
}

ib_status cav_prolong_add(const cav_hierarchy* h, int32_t level, const double* xc, double* w, cudaStream_t st) {
  CAV_API_BEGIN
  const Level& lv = level_of(h, level);
  CAV_REQUIRE(!lv.coarsest && xc && w, "cav_prolong_add: bad level or NULL vector");
  launch_prolong_add(lv.N / 2, xc, w, lv.channel, st);
  return IB_OK;
  CAV_API_END
}

ib_status cav_coarse_solve(const cav_hierarchy* h, const double* r, double* z, cudaStream_t st) {
  CAV_API_BEGIN
  CAV_REQUIRE(h && r && z, "cav_coarse_solve: NULL argument");
  coarse_solve(h, r, z, st);
  return IB_OK;
  CAV_API_END
}

ib_status vcycle_apply(const cav_hierarchy* h, const double* r, double* z, cudaStream_t st) {
  CAV_API_BEGIN
  CAV_REQUIRE(h && r && z, "vcycle_apply: NULL argument");
  CAV_REQUIRE(r != z, "vcycle_apply: r and z must not alias");
  vcycle(h, r, z, st);
  return take_status(h->status, st, "vcycle_apply");
  CAV_API_END
}

ib_status ib_test_wait_stall(int32_t enable) {
  CAV_API_BEGIN
  sweep_set_wait_stall(enable ? 1 : 0);
  colour_set_wait_stall(enable ? 1 : 0);
  return IB_OK;
  CAV_API_END
}

ib_status cav_profile(cav_hierarchy* h, int32_t enable) {
  CAV_API_BEGIN
  CAV_REQUIRE(h, "cav_profile: NULL hierarchy");
  if (enable && h->prof_ev.empty()) {
    h->prof_ev.resize(2 * 8192);
    for (auto& e : h->prof_ev) CAV_CHECK_CUDA(cudaEventCreate(&e));
  }
  h->prof_on = enable ? 1 : 0;
  h->prof_used = 0;
  h->prof_pending.clear();
  h->prof_pushed = h->prof_popped = 0;
  h->prof_acc_ms = 0.0;
  h->prof_acc_n = 0;
  return IB_OK;
  CAV_API_END
}

ib_status cav_profile_read(cav_hierarchy* h, int32_t* launches, double* total_ms) {
  CAV_API_BEGIN
  CAV_REQUIRE(h && launches && total_ms, "cav_profile_read: NULL argument");
  prof_collect(h, -1);
  *launches = h->prof_acc_n;
  *total_ms = h->prof_acc_ms;
  h->prof_acc_n = 0;
  h->prof_acc_ms = 0.0;
  return IB_OK;
  CAV_API_END
}

void cav_destroy(cav_hierarchy* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  vcycle_release(h);
  dl_plan_free(h->dl_plan);
  if (h->dl_stream) cudaStreamDestroy(h->dl_stream);
  if (h->dl_body_stream) cudaStreamDestroy(h->dl_body_stream);
  if (h->dl_host) cudaFreeHost(h->dl_host);
  for (auto& e : h->fg_ev)
    if (e) cudaEventDestroy(e);
  if (h->solve_stream) cudaStreamDestroy(h->solve_stream);
  for (auto& e : h->prof_ev) cudaEventDestroy(e);
  h->arena.release();
  h->ws_arena.release();
  if (h->host_b) cudaFreeHost(h->host_b);
  delete h;
}

ib_status fgmres_solve(const ib_system* s, const cav_hierarchy* h, const double* b, double* x,
                       const fgmres_desc* d, fgmres_info* info, double* history, cudaStream_t st) {
  CAV_API_BEGIN
  CAV_REQUIRE(s && h && b && x && d && info, "fgmres_solve: NULL argument");
  CAV_REQUIRE(h->sys == s, "fgmres_solve: hierarchy was built for another system");
  CAV_REQUIRE(d->maxit >= 1 && d->maxit <= 4096, "fgmres_solve: maxit must be in [1, 4096]");
  CAV_REQUIRE(d->rtol >= 0 && std::isfinite(d->rtol), "fgmres_solve: bad rtol");
  CAV_REQUIRE(d->loop == 0 || d->loop == 1, "fgmres_solve: loop must be 0 or 1");
  CAV_REQUIRE(!(d->loop == 1 && d->host_io), "fgmres_solve: the device-driven loop takes device buffers only");
  std::memset(info, 0, sizeof(*info));
  ib_status r = d->loop ? fgmres_run_device(s, const_cast<cav_hierarchy*>(h), b, x, d, info, history, st)
                        : fgmres_run(s, const_cast<cav_hierarchy*>(h), b, x, d, info, history, st);
  // a stop before maxit (a non-finite preconditioned vector) already left its own message
  if (r == IB_ERR_NOCONV && info->iters >= d->maxit) set_error("fgmres_solve: maxit reached above tolerance");
  return r;
  CAV_API_END
}

ib_status fgmres_solve_batched(int32_t count, const ib_system* const* systems,
                               const cav_hierarchy* const* hierarchies, const double* const* b, double* const* x,
                               const fgmres_desc* d, fgmres_info* infos, cudaStream_t st) {
  CAV_API_BEGIN
  CAV_REQUIRE(count >= 1 && systems && hierarchies && b && x && d && infos, "fgmres_solve_batched: bad argument");
  CAV_REQUIRE(d->maxit >= 1 && d->maxit <= 4096, "fgmres_solve_batched: maxit must be in [1, 4096]");
  CAV_REQUIRE(d->rtol >= 0 && std::isfinite(d->rtol), "fgmres_solve_batched: bad rtol");
  CAV_REQUIRE(!d->host_io, "fgmres_solve_batched: device buffers only");
  CAV_REQUIRE(d->loop == 0 || d->loop == 1, "fgmres_solve_batched: loop must be 0 or 1");
  std::vector<cav_hierarchy*> H(count);
  for (int i = 0; i < count; ++i) {
    CAV_REQUIRE(systems[i] && hierarchies[i] && b[i] && x[i], "fgmres_solve_batched: NULL entry");
    CAV_REQUIRE(hierarchies[i]->sys == systems[i], "fgmres_solve_batched: hierarchy/system mismatch");
    for (int j = 0; j < i; ++j)
      CAV_REQUIRE(hierarchies[j] != hierarchies[i], "fgmres_solve_batched: a hierarchy appears twice");
    H[i] = const_cast<cav_hierarchy*>(hierarchies[i]);
    std::memset(&infos[i], 0, sizeof(fgmres_info));
  }
  ib_status r = d->loop ? fgmres_run_batched_device(count, systems, H.data(), b, x, d, infos, st)
                        : fgmres_run_batched(count, systems, H.data(), b, x, d, infos, st);
  if (r == IB_ERR_NOCONV) set_error("fgmres_solve_batched: some systems stopped above tolerance");
  return r;
  CAV_API_END
}

}  // extern "C"
