// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <vector>

#include "sphgb.h"

#define SPH_MAX_BOX 1024
#define SPH_NDIR 13
#define SPH_SELF_DIR 0  // self interactions sweep along sort direction 0 (the z axis)
#define SPH_PART_STRIDE 8  // floats per (work unit, particle) partial: the sums and a count

// ---------------------------------------------------------------------------
// error handling: every CUDA call is checked and mapped to SPH_ERR_CUDA
// ---------------------------------------------------------------------------
#define SPH_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      fprintf(stderr, "sphgb: %s failed at %s:%d: %s\n", #call, __FILE__, __LINE__,     \
              cudaGetErrorString(e_));                                                   \
      return e_ == cudaErrorMemoryAllocation ? SPH_ERR_OOM : SPH_ERR_CUDA;               \
    }                                                                                    \
  } while (0)

#define SPH_TRY(expr)        \
  do {                       \
    int r_ = (expr);         \
    if (r_ != SPH_OK) return r_; \
  } while (0)

// device status word bits
enum : int {
  ST_CELL_LIMIT = 1,
  ST_NOT_CONVERGED = 2,
  ST_CAPACITY = 4,
  ST_BAD_INDEX = 8,
  ST_TIMEOUT = 16,
  ST_BAD_INPUT = 32,  // a non-finite position or a non-positive h guess
};

// ---------------------------------------------------------------------------
// device buffers owned by the context
// ---------------------------------------------------------------------------
struct DBuf {
  void* p = nullptr;
  size_t cap = 0;
  template <class T>
  T* as() const { return reinterpret_cast<T*>(p); }
};
int dbuf_ensure(DBuf& b, size_t bytes);
void dbuf_free(DBuf& b);

// ---------------------------------------------------------------------------
// primitives (prims.cu)
// ---------------------------------------------------------------------------
// exclusive scans; `total` (device, nullable) receives the sum
int scan_exclusive_i32(const int* in, int* out, int n, int* total, DBuf& tmp, cudaStream_t s);
int scan_exclusive_i64(const long long* in, long long* out, int n, long long* total, DBuf& tmp,
                       cudaStream_t s);
// stable LSD radix sort of (key, value) on bits [0, nbits) of the keys.
// Sorted data ends in keys/vals; keys_alt/vals_alt are scratch of size n.
int radix_sort_u64(unsigned long long* keys, int* vals, unsigned long long* keys_alt, int* vals_alt,
                   int n, int nbits, DBuf& tmp, cudaStream_t s);

// ---------------------------------------------------------------------------
// the context
// ---------------------------------------------------------------------------
struct sph_ctx {
  sph_params prm;
  // problem
  int64_t n = 0;
  int nbox = 0;
  int kbits = 16;  // morton bits per axis
  std::vector<long long> box_off;  // nbox+1
  std::vector<double> box_L;       // nbox
  std::vector<int> box_t;          // log2 top cells per axis
  std::vector<int> top_base;       // first top-cell node per box (nbox+1)
  bool built = false;
  long long state_gen = 0;  // bumped by every call that replaces the forward state
  // positions moved since the build without rebuilding (velocity-Verlet
  // steps): twice the largest displacement, added to the sweeps' axial and
  // box margins and taken off the cell limits of the h solve
  float reuse_pad = 0.f;
  bool vv_ready = false;    // vv_h holds the smoothing lengths of the last step
  DBuf vv_acc, vv_du, vv_dt, vv_vp, vv_up, vv_h, vv_tmp, vv_red;
  bool have_density = false;
  bool have_force = false;
  int have_d2 = 0;

  // box tables (device)
  DBuf d_box_off, d_box_L, d_box_t, d_top_base;

  // particles in Morton (cell) order
  DBuf keys, keys_alt, perm, perm_alt;
  DBuf xs;        // double, 3 per particle (wrapped absolute positions)
  DBuf pos4;      // float4 (x_rel, y_rel, z_rel, m)
  DBuf h;         // float current smoothing length
  DBuf hguess;    // float build-time h
  DBuf hlim;      // float per-particle cell limit
  DBuf pnode;     // int leaf node of each particle
  DBuf p_et;      // float top-cell edge of each particle's box
  DBuf nleaf_dev; // int leaves of the last build

  // octree nodes
  int ncell = 0, ntop = 0, max_depth = 0;
  std::vector<int> gen_start;  // node id where each generation starts (+ end)
  DBuf n_first, n_count, n_parent, n_child0, n_top, n_flags, n_need;
  DBuf n_ijk;     // int4 (ix, iy, iz, level)
  DBuf n_box;     // int
  DBuf n_hmax;    // float max h of the particles in the node (current h)
  DBuf n_hbuild;  // float max h at build time
  DBuf n_hlim;    // float
  DBuf n_sbase;   // long long: base of the node's 13 sorted lists (-1 none)
  DBuf n_nblk, n_blk0;  // leaves: number of particle blocks and the first block
  DBuf n_lo, n_hi;      // float4 particle bounding box of the node (top-cell frame)
  DBuf n_listed, n_ex;  // int: node has sorted lists; interaction entries a reference expands to

  // tasks
  int nself = 0, npair = 0;
  DBuf t_cur, t_next;        // int4 work tasks per generation
  DBuf t_final_pair;         // int4 {ci, cj, packed offset/periodic, 0}
  DBuf t_final_self;         // int
  DBuf t_cnt, t_cnt2, t_off, t_off2;
  DBuf task_ctl;             // int: tasks of the current generation, final self and pair counts
  DBuf tree_ctl;             // int: generation bounds, overflow flag, generation starts
  size_t node_cap = 0;       // octree node capacity (kept from build to build)
  void* tree_host = nullptr; // pinned: per-generation split counts read back while enqueueing

  // blocks
  int nblock = 0, nleaf = 0;
  int64_t ndt = 0;
  DBuf b_first, b_count, b_leaf, b_dtoff, b_order, b_cost, b_hmax;
  DBuf b_lo, b_hi;  // float4 particle bounding box of the block
  // work units: slices of the blocks' interaction lists (b_order holds the
  // units in LPT order); partial sums of blocks cut into several units
  int nunits = 0;
  DBuf b_nseg, u_off, b_part, u_block, u_seg, u_e0, u_e1, u_key, part, blk_done;
  long long part_cols = 0;  // (slice, particle) columns of the blocks cut into slices
  DBuf sl_list;             // unsigned: the slices' pair lists, pair_list_cap per column
  DBuf plan_max;     // unsigned long long: largest estimated block cost of the last estimate
  DBuf u_act;        // int: units of the active blocks in LPT order (masked sweeps)
  DBuf dt_cj;      // int
  DBuf dt_code;    // int: dir | (sgn+1) << 8
  DBuf dt_shift;   // float4 (sx, sy, sz, 0)
  DBuf adj_off, adj_list;  // per-node CSR of final pair tasks

  // sorted lists
  int64_t sorted_entries = 0;
  DBuf s_key, s_idx;

  // physics state (cell order)
  DBuf rho, drho, nngb, dnngb, d2rho, omega, Avec, fdat;  // fdat: float4 per particle for force
  DBuf d2nngb;    // float d^2 N / dh^2 (h iteration)
  DBuf visc4;     // float4 (c, rho, Balsara f, div v) for the viscous force
  DBuf dt_s;      // float time step (Eq. dt)
  float visc_alpha = 0.f, visc_cfl = 0.25f;
  DBuf vel4;      // float4 (vx, vy, vz, hinv)
  DBuf u_s;       // float
  DBuf acc4;      // float4 (ax, ay, az, dudt)
  DBuf cnt_i;     // int per-particle counts
  // h solver
  DBuf h_lo, h_hi;   // double bracket
  DBuf h_dx;         // float previous |step| in ln h
  DBuf h_gb;         // float4 g = ln(N/n_ngb) and dg/dln h at the bracket ends
  DBuf h_flag;       // int: bit0 active, bit1 hi evaluated, bit2 cell limit
  DBuf blk_active;   // int per block
  // adjoint state
  DBuf adj4, adj4b;  // adjoint per-particle j data (cell order)
  DBuf g_A, g_rho_s, g_drho_s, g_h_s, g_u_s, g_x4;
  // force pair lists: per particle (cell order), the j of every pair
  // r < max(h_i, h_j) with its top-cell image code, recorded by the force
  // sweep; later phases over the same pair set read them instead of sweeping
  DBuf fl_list;      // unsigned, groups of 32 particles x fl_K entries x 32 lanes
  DBuf fl_cnt;       // int entries per particle, -1 when the list overflowed
  DBuf fl_flag;      // int bit 0: list overflowed (swept instead)
  DBuf fl_blk;       // int per block: holds an overflowed particle
  DBuf fl_over;      // int number of overflowed particles
  int fl_K = 0;
  bool fl_valid = false;

  // misc
  DBuf status;       // int device status word + counters
  DBuf counters;     // long long[8]
  DBuf queue;        // int work counters
  DBuf scan_tmp, sort_tmp, tmp_a, tmp_b, tmp_c;
  int* dump_pi = nullptr;
  int* dump_pj = nullptr;
  long long dump_cap = 0;

  sph_stats stats{};
  int sweep_grid = 0;
  int sweep_cap = 128;  // buffered j-particles per warp in the sweeps
  bool dir_table_set = false;
  // device-side h iteration graph
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t g_graph = nullptr;
  cudaGraphExec_t g_exec = nullptr;
  long long build_gen = 0, g_gen = -1, g_body_kernels = 0;
  DBuf solve_ctl;
  int sweep_threads = 0;
  // profiling: (phase, start, stop) events recorded around sweep launches
  bool profile = false;
  int cur_phase = 0;
  struct Ev { int phase; cudaEvent_t a, b; };
  std::vector<Ev> ev_pending;
  std::vector<cudaEvent_t> ev_pool;
  DBuf prof_units;  // 4 unsigned long long per pending profiled launch
  unsigned long long prof_units_acc[8] = {0};
  unsigned long long prof_cand_acc[8] = {0};
  unsigned long long prof_gath_acc[8] = {0};
  double prof_ms[8] = {0};
  int prof_n[8] = {0};
  double prof_build_ms[8] = {0};
  int prof_builds = 0;
  double prof_t = 0;  // host time (ms) of the last build-stage boundary
};
// profiling: synchronise the stream and charge the host time since the
// previous boundary to build stage k (k < 0 only starts the clock)
int build_mark(sph_ctx* c, cudaStream_t s, int k);
cudaEvent_t ev_get(sph_ctx* c);
int prof_resolve(sph_ctx* c);

// ---------------------------------------------------------------------------
// stages (build.cu, sweep.cu)
// ---------------------------------------------------------------------------
int build_decomposition(sph_ctx* c, const double* pos, const float* h_guess, cudaStream_t s);
// rebuild cells, tasks, blocks and sorted lists from the h in c->hguess
// (Morton order and positions unchanged)
int build_from_guess(sph_ctx* c, cudaStream_t s);
int run_sweep(sph_ctx* c, int phase, int only_active, int counting, cudaStream_t s);
int set_dir_table(sph_ctx* c);  // the 13 sort directions into constant memory (once)
int compute_node_hmax(sph_ctx* c, cudaStream_t s);
// re-plan the work units from block costs estimated with the current h
// (only_active: the particles still iterating in the h solve) when the
// present plan would leave one unit well above the balanced share of the
// resident warps; *changed tells whether it did
int replan_units(sph_ctx* c, int only_active, bool* changed, cudaStream_t s);

// sweep phases
enum : int {
  PH_DENSITY = 0,      // rho, drho/dh, N, dN/dh (+count)
  PH_DENSITY_D2 = 1,   // d^2 rho/dh^2 only
  PH_FORCE = 2,        // acc, du/dt (+count)
  PH_FORCE_ADJ = 3,    // force adjoint gather
  PH_DENSITY_ADJ = 4,  // density adjoint gather
  PH_VELDERIV = 5,     // div v, curl v and the Balsara switch (viscosity)
  PH_FORCE_VISC = 6,   // force with artificial viscosity and the time-step signal speed
  PH_DUMP_DENSITY = 8,
  PH_DUMP_FORCE = 9,
};

inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

// running count of kernel launches issued by this library (all contexts)
void note_launch();
void note_launch_n(long long k);  // adjust by k (graph-executed launches)
long long launch_count();
