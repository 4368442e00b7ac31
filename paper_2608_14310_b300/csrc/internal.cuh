// Internal declarations of the CAV multigrid library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ib_cav.h"

namespace cav {

// ------------------------------------------------------------------ errors

void set_error(const std::string& msg);
struct Fail {
  ib_status st;
};
#define CAV_CHECK_CUDA(call)                                                        \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      ::cav::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));       \
      throw ::cav::Fail{e_ == cudaErrorMemoryAllocation ? IB_ERR_OOM : IB_ERR_CUDA}; \
    }                                                                               \
  } while (0)
// counts every kernel launch of the library (host side), for launch accounting
void note_launch();
// adds n (may be negative) to the count: kernels replayed inside graphs, or a capture's
// launches taken back (a capture records kernels, it does not run them)
void note_launches(long long n);
int64_t launch_count();
// a process-wide unique id for a handle (systems, hierarchies)
uint64_t next_uid();
#define CAV_CHECK_LAUNCH()                  \
  do {                                      \
    ::cav::note_launch();                   \
    CAV_CHECK_CUDA(cudaGetLastError());     \
  } while (0)
#define CAV_REQUIRE(cond, msg)                                                      \
  do {                                                                              \
    if (!(cond)) {                                                                  \
      ::cav::set_error(msg);                                                        \
      throw ::cav::Fail{IB_ERR_INVALID};                                            \
    }                                                                               \
  } while (0)

constexpr int NUM_APPLY_VARIANTS = 5;
// unknowns held by enlarged patches that one 256-thread block of the scatter updates
constexpr int SCATTER_TOUCHED_PER_BLOCK = 64;

// Device status word codes (written by kernels, read by the host after set-up or a solve).
enum : int { DEV_OK = 0, DEV_WINDOW = 1, DEV_SINGULAR = 2, DEV_CAPACITY = 3, DEV_TIMEOUT = 4 };

// ------------------------------------------------------------------ device memory

// Owns a list of device allocations; freed together with the owning handle.
struct Arena {
  std::vector<void*> ptrs;
  template <typename T>
  T* alloc(size_t count) {
    void* p = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    CAV_CHECK_CUDA(cudaMalloc(&p, bytes));
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
};

// ------------------------------------------------------------------ E_E on one level

struct DlPlan;  // a solve captured as a graph (fgmres.cu)

// words of a hierarchy's grid-barrier state (the fused sweep, sweep.cu)
constexpr int CAV_GBAR_WORDS = 320;

// E_E restricted to its structurally nonzero velocity rows, each row's columns sorted.
struct EECsr {
  int n_rows = 0;            // active rows
  int64_t nnz = 0;
  int W = 0;                 // per-axis |offset| bound between a row face and its columns
  int* rows = nullptr;       // [n_rows] global velocity index of each active row
  int64_t* rowptr = nullptr; // [n_rows + 1]
  int* cols = nullptr;       // [nnz]
  double* vals = nullptr;    // [nnz]
  int* row_of = nullptr;     // [2 N^2] active row index or -1
  int cross = 0;             // 1: rows may have columns in the other velocity component
};

// ------------------------------------------------------------------ one grid level

struct Level {
  int N = 0;
  double h = 0, rho_dt = 0, mu = 0, dt = 0;
  bool channel = false;          // the channel's boundary rows, transfers and patches (Sec. 5.3)
  bool coarsest = false;
  bool coloured = false;         // this level smooths with the class-by-class multiplicative sweep
  bool box = false;              // box patches B(b,o): one per block, all enlarged, restricted injection
  int nu_pre = 0, nu_post = 0;   // sweeps per side in the V-cycle
  EECsr ee;

  // patches (smoothing levels): one per cell; enlarged ones are stored explicitly
  int n_big = 0;                 // enlarged patches
  int n_std4 = 0;                // standard patches with four unknowns (the channel's inflow row)
  std::vector<int> host_sizes;   // [n_big] stored patch sizes (host copy, for refactorisation)
  int n_big_small = 0;           // stored patches with at most five unknowns (Vanka patches whose
                                 // unknowns have E_E rows)
  int64_t big_sum_n = 0, big_sum_n2 = 0, inv_elems = 0;
  int big_max_n = 0;
  uint8_t* cell_big = nullptr;   // [N^2] 1 if the cell's patch is enlarged
  int* big_cell = nullptr;       // [n_big] cell index of each enlarged patch (ascending)
  int64_t* big_off = nullptr;    // [n_big + 1] offsets into big_dofs / packed delta
  int* big_dofs = nullptr;       // [big_sum_n] sorted global indices
  int64_t* inv_off = nullptr;    // [n_big + 1] element offsets of each inverse (ld * n)
  int* order = nullptr;          // [n_big] patches by descending size (launch order)
  uint8_t* inject = nullptr;     // [big_sum_n] box patches: 1 where the slot receives its
                                 // correction (the unexpanded block); null otherwise
  double* s_r = nullptr;         // [big_sum_n] row scales (power of two)
  double* s_c = nullptr;         // [big_sum_n] column scales
  double* inv64 = nullptr;       // [inv_elems] equilibrated inverses, column-major, ld = round8(n)
  float* inv32 = nullptr;
  __nv_bfloat16* inv16 = nullptr;
  int precision = CAV_PREC_FP64;
  int apply_variant = 0;         // patch-apply kernel variant (autotuned when requested)
  float apply_us[8] = {0};       // the autotuner's timing of each variant (us per launch)
  std::vector<int> sched_G;        // balanced patch schedules of the persistent apply, per grid
  std::vector<int*> sched_off;     // size: [G + 1] offsets into sched_list, per CTA
  std::vector<int*> sched_list;    // [n_big] patch indices, CTA by CTA
  int fused = 0;                 // 1: the additive sweep runs as one cooperative kernel
  float sweep_us[2] = {0, 0};    // the autotuner's timing of one sweep: separate kernels, fused
  int64_t* inc_off = nullptr;    // [3 N^2 + 1] transpose incidence: slots of each unknown
  int* inc_slot = nullptr;       // [big_sum_n] packed-delta slots, ascending per unknown
  int n_touched = 0;             // unknowns held by at least one enlarged patch
  int* touched = nullptr;        // [n_touched] ascending
  double* touch_theta = nullptr; // [n_touched] 1 / (patches holding each one)
  double std_inv[3][25];         // inverse of the standard Vanka patch, canonical order
                                 // (u_ij, u_i+1j, v_ij, v_ij+1, p_ij), scalings folded in:
                                 // [0] every cell of a periodic level, or the channel's
                                 // interior rows; [1] the channel's outflow row, [2] its
                                 // inflow row (slot 3 absent: zero row and column)

  // colour classes for the multiplicative sweep (smoother CAV_SMOOTH_COLOURED): patches of
  // one class share no unknown and no entry of K_E couples them, so a class is solved at once
  int n_colours = 0;
  std::vector<int> colour_of_cell;   // [N^2, or n_big for box patches] host copy, for export
  std::vector<int> col_big_start;    // [n_colours + 1] offsets into col_job / col_inv
  std::vector<int> col_std_start;    // [n_colours + 1] offsets into col_std
  int4* col_job = nullptr;           // [n_big] enlarged patches class by class: (p, n, slot offset, 0)
  int64_t* col_inv = nullptr;        // [n_big] element offset of each one's inverse, same order
  int* col_std = nullptr;            // [N^2 - n_big] standard cells, class by class
  int2* slot_ee = nullptr;           // [big_sum_n] per packed slot: (start, length) of its E_E row
  float* ee_vals32 = nullptr;        // [ee.nnz] E_E values in FP32 (FP32-inverse coloured levels)
  float* w32 = nullptr;              // [3 N^2] (float) of the iterate during a coloured sweep (FP32 levels)
  int ee_row_max = 0;                // longest E_E row on this level

  // coarsest level: dense inverse, row-major m x m: the bordered system (m = n + 1) on a
  // periodic level, the plain one (m = n) on the channel, whose pressure is determined
  double* coarse_inv = nullptr;
  int coarse_m = 0;

  // work vectors of this level
  double* r = nullptr;           // [3 N^2] residual
  float* r32 = nullptr;          // [3 N^2] the residual in FP32 (FP32 / BF16 additive levels): the
                                 // standard patches' inverse is applied in FP32 there
  double* x = nullptr;           // [3 N^2] V-cycle iterate
  double* b = nullptr;           // [3 N^2] V-cycle right-hand side (levels > 0)
  double* delta = nullptr;       // [big_sum_n] packed patch corrections
  double* wpart = nullptr;       // [8 n_partial] the fused sweep's per-warp pressure sums
  double* partial = nullptr;     // partial sums for the pressure mean: stencil part, then
  int n_partial = 0;             // the part of the unknowns touched by enlarged patches
  int n_partial_std = 0;
};

}  // namespace cav

// ------------------------------------------------------------------ handles

struct ib_system {
  int N = 0;
  int bc = IB_BC_PERIODIC;       // ib_bc
  double L = 1, h = 0, rho = 0, mu = 0, dt = 0;
  int M = 0, law = 0, closed = 0, bw = 0;
  double ds = 0, k_target = 0, k_stretch = 0, k_bend = 0;
  double k_pos = 0, k_tan = 0, clamp_x = 0, clamp_y = 0;  // fiber law's midpoint clamp
  int device = 0;
  cav::Arena arena;
  // markers (component-major x[0..M), y[M..2M))
  double* X = nullptr;
  double* omega = nullptr;
  double* Eband = nullptr;       // [M * (2 bw + 1)] E coefficient of (a, a + d)
  double* Eblock = nullptr;      // fiber law: [M][2 bw + 1][2][2] E entry ((c, a), (c2, a + d))
  double* Ffib = nullptr;        // fiber law: [2M] F at the linearisation point
  double* Xt = nullptr;          // [2M] target positions (component-major) or null
  double* F = nullptr;           // [2M] Lagrangian force scratch
  double* U = nullptr;           // [2M] marker velocity / next positions scratch
  std::vector<double> X_host;    // interleaved copy of X^n (for the advection output)
  // kernel support per (component c, marker a): index c * M + a
  int* sup_i0 = nullptr;         // first face index along x (may be negative / >= N)
  int* sup_j0 = nullptr;
  double* sup_wx = nullptr;      // [2M * 4]
  double* sup_wy = nullptr;
  uint8_t* sup_mask = nullptr;   // [2M] bits 0-3: x support, bits 4-7: y support
  int64_t* fm_off = nullptr;     // [2 N^2 + 1] face -> markers whose support holds it
  int* fm_list = nullptr;        // ascending marker ids
  cav::EECsr ee;                 // finest-level E_E
  uint64_t uid = 0;              // identity of the handle (kept by ib_update_structure)
  uint64_t epoch = 0;            // bumped whenever ib_update_structure replaces the buffers
  int* status = nullptr;         // device status word
  double* partial = nullptr;     // [reduce_blocks(3 N^2) + 1] reduction scratch
};

struct cav_hierarchy {
  const ib_system* sys = nullptr;
  cav_desc desc{};
  std::vector<cav::Level> levels;
  cav::Arena arena;
  int* status = nullptr;
  int* flag = nullptr;           // device scratch word (pattern comparison)
  uint64_t uid = 0;              // identity of the handle
  uint64_t epoch = 0;            // bumped by cav_refactor (cached solve graphs are rebuilt)
  // the grid the hierarchy was built for (cav_refactor accepts only systems on the same grid;
  // the system it was built from may have been destroyed by then)
  int grid_N = 0, grid_bc = 0;
  double grid_L = 0, grid_rho = 0, grid_mu = 0, grid_dt = 0;
  // FGMRES workspace (grown on demand)
  int ws_maxit = 0;
  double* V = nullptr;   // (maxit + 1) x n
  double* Z = nullptr;   // maxit x n
  double* dev_scalars = nullptr;  // Hessenberg, Givens, g and small temporaries
  double* red_partial = nullptr;  // partial sums for multi-dot reductions
  double* host_b = nullptr;       // pinned scalars read back per iteration
  cudaEvent_t fg_ev[2] = {nullptr, nullptr};  // per-iteration convergence records
  cudaStream_t solve_stream = nullptr;         // this system's stream in batched solves
  double* io_b = nullptr;         // device staging for host_io
  double* io_x = nullptr;
  cav::Arena ws_arena;
  // live timing of the finest level's patch-apply launches
  int prof_on = 0;
  int prof_used = 0;
  std::vector<cudaEvent_t> prof_ev;  // pairs (start, stop) for launches outside graphs
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pending;  // recorded, not yet read, in issue order
  long long prof_pushed = 0, prof_popped = 0;
  double prof_acc_ms = 0.0;
  int prof_acc_n = 0;
  // The V-cycle captured as a CUDA graph (input lv0.b, output lv0.x), two instances used
  // alternately so that a replay's event records are read before the instance replays again
  cudaGraphExec_t vc_exec[2] = {nullptr, nullptr};
  int vc_next = 0;
  cudaStream_t capture_stream = nullptr;
  std::vector<cudaEvent_t> vc_ev[2];  // event pairs around the finest-level applies
  int capturing = 0;                  // 0: not capturing, 1 + instance: capturing that instance
  int graph_failed = 0;
  int vc_kernels[2] = {0, 0};         // kernels in each V-cycle graph (launch accounting)
  unsigned* gbar = nullptr;           // grid-barrier state of the fused sweep (counters, generation)
  int no_events = 0;                  // 1 while a solve graph is captured: no event records
  // device-driven solves (fgmres_desc.loop = 1): scratch and the cached executable graph
  double* dl_w = nullptr;             // [n] the new Krylov vector before normalisation
  int* dl_kc = nullptr;               // [8] iteration counters
  double* dl_hist = nullptr;          // [maxit + 1] residual estimates
  double* dl_host = nullptr;          // pinned: [32] records + [maxit + 1] history
  cav::DlPlan* dl_plan = nullptr;     // the last solve graph built with this hierarchy first
  cudaStream_t dl_stream = nullptr, dl_body_stream = nullptr;
};

namespace cav {

// a solve (or a batch of solves) captured as one executable graph (fgmres.cu)
void dl_plan_free(DlPlan* p);

// ------------------------------------------------------------------ kernels' host wrappers

// While set on the calling thread, launch_k launches without the programmatic attribute
// (a graph whose programmatic edges could not be instantiated is rebuilt this way).
inline bool& pdl_off() {
  static thread_local bool off = false;
  return off;
}

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Launch kernel k on st.  pdl: as a programmatic dependent launch, so the kernel's blocks may
// be scheduled before the kernel ahead of it on st has finished (the launch latency hides under
// that kernel).  The kernel must call pdl_wait() before touching memory an earlier kernel reads
// or writes; pdl is only set when the operation ahead of the launch on st is one of this
// library's kernels.
template <typename... KArgs, typename... Args>
inline void launch_k(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
                     Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (pdl && !pdl_off()) ? 1 : 0;
  CAV_CHECK_CUDA(cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...));
  CAV_CHECK_LAUNCH();
}

inline int round8(int n) { return (n + 7) & ~7; }

// ib_system.cu
// X_lin_interleaved: where the fiber law's force and tangent are taken (X for the others)
void build_markers_and_ee(ib_system* s, const double* X_interleaved, const double* X_lin_interleaved,
                          const double* omega_host, cudaStream_t st);
void ib_force_launch(const ib_system* s, double* F, cudaStream_t st);
void ib_spread_launch(const ib_system* s, const double* F, double* f, int rhs, const double* u_prev,
                      const double* f_body, cudaStream_t st);
void ib_interp_launch(const ib_system* s, const double* u, double* U, double dt, cudaStream_t st);
void ee_compute_window(EECsr& ee, int N, int* d_scratch, cudaStream_t st);

// stencil.cu: operators of one level (finest level uses the system's E_E)
struct LevelOps {
  int N;
  double h, rho_dt, mu, dt;
  const EECsr* ee;
  bool channel = false;
};
// mode 0: out = b - K w  (b may be null = 0);  mode 1: out = K w.  pdl: see launch_k.
// out32 (nullable): out rounded to FP32 as well.
void launch_apply(const LevelOps& op, const double* w, const double* b, double* out, int mode,
                  cudaStream_t st, bool pdl = false, float* out32 = nullptr);
void launch_restrict(int Nc, const double* r_f, double* b_c, bool channel, cudaStream_t st, bool pdl = false);
void launch_prolong_add(int Nc, const double* x_c, double* w_f, bool channel, cudaStream_t st, bool pdl = false);

// setup.cu
void build_levels(cav_hierarchy* H, cudaStream_t st);
// true if the two E_E share their structural pattern (rows, row pointers, columns); syncs
bool same_ee_pattern(const EECsr& a, const EECsr& b, int* d_flag, cudaStream_t st);
// new values of the system's finest E_E on an unchanged pattern: Galerkin values, patch and
// coarsest inverses recomputed into the hierarchy's existing buffers; binds H to s
void refactor_levels(cav_hierarchy* H, const ib_system* s, cudaStream_t st);

// colour.cu: colour classes (set-up) and the class-by-class multiplicative sweep
// The set-up of a coloured level in three parts: colour_fetch copies the level's patch sets
// and E_E pattern to the host (syncs st); colour_plan computes the first-fit classes and the
// class-ordered job tables on the host alone (no CUDA call, so a host thread can run it while
// the device works; it writes only lv's class fields and P); colour_upload stores the tables on
// the device (syncs st).
struct ColourPlan {
  std::vector<uint8_t> big;
  std::vector<int64_t> off, inv_off, rowptr;
  std::vector<int> bd, row_of, cols;
  std::vector<int4> jobs;      // class-ordered enlarged patches: (patch, size, slot offset, 0)
  std::vector<int64_t> jinv;   // their inverses' offsets
  std::vector<int> hs;         // class-ordered standard cells
};
void colour_fetch(const Level& lv, ColourPlan& P, cudaStream_t st);
void colour_plan(Level& lv, ColourPlan& P);
void colour_upload(cav_hierarchy* H, Level& lv, const ColourPlan& P, cudaStream_t st);
void colour_refresh_values(Level& lv, cudaStream_t st);
// fails (IB_ERR_INVALID) when the level's class steps would not fit in shared memory
void check_colour_step(const Level& lv);
void coloured_sweep(const cav_hierarchy* H, int l, const double* b, double* w, bool w_is_zero,
                    double* partial, bool remove_mean, bool profile, cudaStream_t st);
// p -= mean(p) over the N^2 cells, partial holding at least ceil(N^2 / 256) doubles
void pressure_mean_remove(int N, double* partial, double* p, cudaStream_t st);

// sweep.cu
void launch_remove_mean(int N, int n_partial, const double* partial, double* p, cudaStream_t st);
void level_sweep(const cav_hierarchy* H, int l, const double* b, double* w, bool w_is_zero,
                 cudaStream_t st);
void coarse_solve(const cav_hierarchy* H, const double* r, double* z, cudaStream_t st, bool pdl = false);
bool prof_records(const cav_hierarchy* H, int level);
void prof_begin(const cav_hierarchy* H, int level, cudaStream_t st);
void prof_end(const cav_hierarchy* H, int level, cudaStream_t st);
void prof_collect(cav_hierarchy* H, long long upto = -1);
void vcycle_release(cav_hierarchy* H);
void autotune_level(cav_hierarchy* H, Level& lv, cudaStream_t st);
// balanced patch schedules of a level's persistent apply for its launch grids (set-up)
void build_schedules(cav_hierarchy* H, Level& lv, cudaStream_t st);
// Theta of every touched unknown: 1 / (enlarged patches holding it + standard patches of its
// incident cells) (set-up, after the incidence, the touched list and cell_big)
void build_touch_theta(cav_hierarchy* H, Level& lv, cudaStream_t st);
// the additive sweep's form on level lv: separate kernels or one fused cooperative kernel
// (force 1: fused where possible, -1: separate, 0: the faster by timing)
void choose_sweep_form(cav_hierarchy* H, Level& lv, int force, cudaStream_t st);
void vcycle_prepare(cav_hierarchy* H);
void krylov_reserve(cav_hierarchy* H, int maxit, int64_t n);
void vcycle(const cav_hierarchy* H, const double* r, double* z, cudaStream_t st);
// the V-cycle's kernels launched directly on st (input levels[0].b, output levels[0].x), for
// capture into a solve graph
void vcycle_inline(const cav_hierarchy* H, cudaStream_t st);

// reductions (reduce.cu)
int reduce_blocks(int64_t n);
void launch_dot_partials(const double* a, const double* b, int64_t n, double* partial,
                         cudaStream_t st);
// <a, b> on the device (fixed order), returned to the host after a stream synchronisation;
// partial holds at least reduce_blocks(n) + 1 doubles
double device_dot(const double* a, const double* b, int64_t n, double* partial, cudaStream_t st);
// exclusive scan of int counts into int64 offsets (out has n + 1 entries)
void exclusive_scan(const int* counts, int64_t* out, int64_t n, cudaStream_t st, Arena* scratch);

int read_status(int* d_status, cudaStream_t st);
// The message and the ABI status for a device status code.
std::string status_message(int code);
ib_status status_of(int code);
// After the work queued on `st`: reads the device status word, clears it and turns a
// recorded failure into a status with a message (IB_ERR_TIMEOUT for a bounded wait that ran
// out).  Synchronises `st`; while `st` is being captured into a graph it reads nothing and
// returns IB_OK.
ib_status take_status(int* d_status, cudaStream_t st, const char* who);
// Test hook: make every stallable bounded wait run out (each translation unit with waits).
void sweep_set_wait_stall(int enable);
void colour_set_wait_stall(int enable);

}  // namespace cav
