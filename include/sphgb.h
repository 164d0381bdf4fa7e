/*
 * sphgb.h — C ABI of the GB300 SPH neighbour-interaction library.
 *
 * Computes the two SPH loops of Gonnet, "Efficient and Scalable Algorithms
 * for Smoothed Particle Hydrodynamics on Hybrid Shared/Distributed-Memory
 * Architectures" (arXiv 1404.2303):
 *   - density, Eq. (rho), with each particle's smoothing length h_i solved
 *     so that the weighted neighbour number of Eq. (nneigh) equals N_ngb;
 *   - the ghost quantities P_i and Omega_i (text after Eq. (dudt));
 *   - the force loop, Eq. (dvdt) and Eq. (dudt);
 * over the hierarchical cell decomposition of Section 3.2 (top grid of
 * edge >= h_max, recursive octree split, self and pair interactions split
 * as in Fig. SplitCell / SplitPair) with the sorted cell-pair interactions
 * of Section 3.3 (13 stored sort directions, axial cutoff, hierarchical
 * merge of sub-cell sorts).  It also provides the reverse-mode adjoints of
 * both loops (the paper has none): gradients with respect to positions,
 * masses and internal energies, with h differentiated implicitly.
 *
 * Conventions for every entry point:
 *   - All array arguments are DEVICE pointers owned by the caller; the
 *     library never frees them.  Arrays are in the caller's particle order.
 *     Positions are AoS float64 (n x 3, x y z per particle); velocities,
 *     accelerations and position gradients are AoS float32 (n x 3); every
 *     per-particle scalar is a float32 array of length n unless stated.
 *   - `stream` is a cudaStream_t passed as void*; all work is enqueued on it.
 *   - The context owns the decomposition (cells, tasks, sorted lists,
 *     particle copies in cell order) and all scratch memory; it allocates
 *     during sph_create / sph_build / sph_build_batch only.
 *   - Return value: SPH_OK (0) or a negative sph_status.  Calls that must
 *     read a device result (sph_build*, sph_density, and any call that
 *     reports an interaction count) synchronise `stream`; the others are
 *     asynchronous and report device-side failures through the next
 *     synchronising call or sph_sync_status.  No device code traps or
 *     asserts: failures set a status word read by the host.
 *   - A context is not thread-safe; use one per host thread.
 *
 * Precision: pair arithmetic is FP32 on cell-relative coordinates; absolute
 * positions, cell origins and the smoothing-length bracket are FP64.  With
 * positions that are multiples of L*2^-24 in a box of side L = 2^k, every
 * coordinate difference is exact in FP32 and the neighbour predicate
 * fma(dz,dz,fma(dy,dy,dx*dx)) < fl(h*h) is bit-reproducible.
 */
#ifndef SPHGB_H
#define SPHGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sph_ctx sph_ctx;

enum sph_status {
  SPH_OK = 0,
  SPH_ERR_INVALID_ARG = -1,     /* bad size, null pointer, box too small for h (n_top < 4) */
  SPH_ERR_CUDA = -2,            /* a CUDA runtime call failed */
  SPH_ERR_OOM = -3,             /* device allocation failed */
  SPH_ERR_H_NOT_CONVERGED = -4, /* Newton/bisection hit max_newton */
  SPH_ERR_CELL_LIMIT = -5,      /* a solved h exceeds what the decomposition covers after max_rebuild rebuilds */
  SPH_ERR_NOT_BUILT = -6,       /* call needs sph_build / sph_density first */
  SPH_ERR_TIMEOUT = -7,         /* a bounded device wait gave up */
  SPH_ERR_CAPACITY = -8         /* an output buffer was too small (sph_pairs_dump) */
};

/* Parameters.  Physical constants follow Section 4.2 of the paper
 * (N_ngb = 48, gamma = 5/3, split above 300 particles when more than 87.5 %
 * have h < edge/2). */
typedef struct sph_params {
  float n_ngb;          /* target weighted neighbour number, Eq. (nneigh); 48 */
  float gamma;          /* adiabatic index, P = (gamma-1) rho u; 5/3 */
  int32_t split_count;  /* split a cell holding more than this many particles ... ; 300 */
  float split_frac;     /* ... when more than this fraction have h <= edge/2; 0.875 */
  int32_t block_max;    /* largest particle block (sort unit; a warp sweeps it in chunks of 32) (32..256); 64 */
  int32_t max_newton;   /* h iterations per solve; 64 */
  int32_t max_rebuild;  /* decomposition rebuilds when a solved h outgrows its cell; 4 */
  int32_t kahan;        /* 1: compensated (Neumaier) sums across interaction tasks; 0: plain FP32 */
  int32_t morton_bits;  /* octree depth limit below the box, bits per axis (8..20); 16 */
  float h_tol;          /* converged when |N - n_ngb| <= h_tol * n_ngb; 2^-19 */
  int32_t warps_per_cta;/* sweep kernels: warps per CTA (1..8); 8 */
  int32_t ctas_per_sm;  /* sweep kernels: resident CTAs per SM used to size the persistent grid; 0 = occupancy */
  int32_t h_est_mode;   /* h estimate when no guess is given: 0 density of the leaf's parent,
                           1 the lower of leaf and parent densities; 1 */
  float h_est_factor;   /* the cells are built for the estimate times this margin (fewer
                           rebuilds); the solve starts from the estimate itself; 1.5 */
  int32_t sweep_cap;    /* sweep kernels: j-particles a warp buffers in shared memory between
                           compute passes (multiple of 32, 32..1024); 128 */
  int32_t use_graph;    /* 1: each h-iteration round runs as one CUDA graph with a device-side
                           while loop (no host round trip per iteration); 0: host loop.
                           Profiling (sph_profile) always uses the host loop; 1 */
  int32_t sweep_lists;  /* sweep kernels, bit k for phase k (0 density, 1 d2rho/dh2, 2 force,
                           3 force adjoint, 4 density adjoint): each lane first tests every
                           buffered candidate with the phase's exact FP32 predicate and keeps
                           a list of the accepted ones, then evaluates only those (otherwise
                           every lane evaluates every candidate); needs sweep_cap <= 256; 0x08 */
  int32_t pair_list_cap;/* force pair lists: the force sweep records, per particle, every j with
                           r < max(h_i, h_j) (up to this many; 0 disables), and the phases over
                           that pair set afterwards (d2rho/dh2, force adjoint, density adjoint)
                           read the lists instead of sweeping; a particle with more pairs is
                           swept.  Costs 4 * n * pair_list_cap bytes of device memory; needs
                           sweep_cap <= 256 and n < 2^27; 256 */
  int32_t list_cap;     /* cells of at most this many particles (0..4096) get their 13 sorted
                           lists, merged from their children's; a pair task naming a larger
                           cell walks its listed descendants (or the blocks of a larger leaf)
                           instead; 4096 */
  int32_t sorted_sweep; /* 1: sorted cell-pair sweeps (Section 3.3: axial windows in the
                           sorted lists, candidates filtered by the chunk's box); 0: the
                           naive cell-pair loop over the same tasks, every particle of every
                           target a candidate (ablation of the sorting; same results); 1 */
} sph_params;

/* Statistics of the last build and sweeps (host copy). */
typedef struct sph_stats {
  int64_t n;                 /* particles */
  int32_t nbox;              /* independent boxes */
  int32_t ncell;             /* cells (all levels, including empty children) */
  int32_t nleaf;             /* non-empty leaf cells */
  int32_t nblock;            /* particle blocks (sweep work units) */
  int32_t nself;             /* final self-interaction tasks */
  int32_t npair;             /* final pair-interaction tasks */
  int64_t ndt;               /* directed block<-cell interaction records */
  int32_t max_depth;         /* deepest octree level reached */
  int32_t top_level[8];      /* log2 of top cells per axis for the first 8 boxes */
  int32_t newton_iters;      /* h iterations of the last sph_density */
  int32_t rebuilds;          /* rebuilds triggered by the last sph_density */
  int64_t density_interactions; /* directed (i<-j, r<h_i, self included) of the last counted density pass */
  int64_t force_pairs;       /* unordered pairs r<max(h_i,h_j) of the last counted force pass */
  int64_t sorted_entries;    /* (key, index) entries held in sorted lists */
  /* sweep-kernel device time per phase while profiling is on (sph_profile):
   * 0 density, 1 d2rho/dh2, 2 force, 3 force adjoint, 4 density adjoint */
  double sweep_ms[8];
  int32_t sweep_launches[8];
  int64_t sweep_units[8];    /* pairs accepted by those launches: directed (i<-j) for
                                phases 0 and 1, ordered i != j pairs for 2..4 */
  int64_t sweep_candidates[8]; /* (i, j) candidates those launches evaluated */
  int32_t newton_active[32]; /* particles still iterating after each of the first 32 h iterations
                                of the last sph_density, rounds after a rebuild included (0 afterwards) */
  int32_t unconverged;       /* particles left unconverged by the last sph_density */
  int32_t sweep_grid;        /* CTAs of the last sweep launch */
  int32_t sweep_threads;     /* threads per CTA of the sweep launches */
  /* build wall time per stage while profiling is on (the stream is synchronised at each
   * stage boundary): 0 Morton order, 1 h estimate, 2 octree, 3 pair tasks, 4 blocks and
   * block sorts, 5 hierarchical merge, 6 interaction lists, 7 node h maxima */
  double build_ms[8];
  int32_t builds;            /* decompositions built while profiling (rebuilds included) */
  int64_t sweep_gathered[8]; /* j entries the sweeps' axial windows held, per phase (before the
                                chunk's box test; one per chunk, not per lane) */
  int32_t pairs_unlisted;    /* particles the last force sweep recorded no pair list for (swept
                                again by the phases over the force pairs) ... */
  int32_t pairs_unlisted_cut; /* ... of which in blocks cut into several work units */
} sph_stats;

/* Fill *p with the defaults listed above. */
void sph_default_params(sph_params* p);

/* Create a context.  Returns SPH_ERR_INVALID_ARG for out-of-range params. */
int sph_create(const sph_params* p, sph_ctx** out);

/* Free the context and every device buffer it owns.  NULL is ignored. */
void sph_destroy(sph_ctx* ctx);

/* Build the decomposition of Section 3.2 for one periodic cube [0, box)^3:
 * Morton order, top grid of edge >= max h (a power of two cells per axis,
 * at least 4), octree split of Section 3.2 / 4.2, self and pair tasks
 * split per Fig. SplitCell / SplitPair, and the 13-direction sorted lists
 * of Section 3.3 (leaf blocks sorted, parents merged from their children).
 *   pos      n x 3 float64 positions (wrapped into the box here)
 *   h_guess  n float32 initial smoothing lengths; NULL = estimate from the
 *            local particle density of a count-only octree
 * Synchronises `stream`.  INVALID_ARG if n <= 0, box <= 0 or max h > box/4. */
int sph_build(sph_ctx* ctx, int64_t n, const double* pos, double box,
              const float* h_guess, void* stream);

/* As sph_build for `nbox` independent boxes stored back to back:
 *   offsets  HOST array of nbox+1 particle offsets (offsets[0] = 0)
 *   boxes    HOST array of nbox box sizes
 * All boxes share one decomposition table, one task list and one
 * persistent sweep launch per phase. */
int sph_build_batch(sph_ctx* ctx, int32_t nbox, const int64_t* offsets, const double* boxes,
                    const double* pos, const float* h_guess, void* stream);

/* Density at GIVEN smoothing lengths, Eq. (rho) and Eq. (nneigh):
 *   m        masses
 *   h        smoothing lengths (each must not exceed what the built
 *            decomposition covers: CELL_LIMIT otherwise)
 *   rho      out: rho_i = sum_{r_ij<h_i} m_j W(r_ij, h_i), self included
 *   drho_dh  out (nullable): d rho_i / d h_i at fixed positions
 *   nngb     out (nullable): (4/3) pi h_i^3 sum_j W(r_ij, h_i)
 *   dnngb_dh out (nullable): d nngb_i / d h_i
 *   count    out (nullable, int32): directed neighbours r_ij < h_i (FP32
 *            predicate), self included; when given the call synchronises
 *            and records the total in sph_stats.density_interactions
 * The result becomes the context's density state for sph_force. */
int sph_density_fixed_h(sph_ctx* ctx, const float* m, const float* h, float* rho,
                        float* drho_dh, float* nngb, float* dnngb_dh, int32_t* count,
                        void* stream);

/* Density with the smoothing-length solve of Eq. (nneigh): Newton steps on
 * N_i(h) - n_ngb kept inside an FP64 bisection bracket, re-sweeping only
 * blocks that still hold unconverged particles; when a root lies beyond a
 * particle's cell limit the decomposition is rebuilt (max_rebuild times)
 * from the current h.  Starts from the build's h guesses.
 *   m      masses
 *   h      out (nullable): solved smoothing lengths
 *   rho    out (nullable): densities at the solved h
 *   omega  out (nullable): Omega_i = 1 + h_i/(3 rho_i) d rho_i/d h_i
 *   iters  out (nullable, HOST int32): Newton iterations used
 * Synchronises `stream`. */
int sph_density(sph_ctx* ctx, const float* m, float* h, float* rho, float* omega,
                int32_t* iters, void* stream);

/* Ghost step and force loop, Eq. (dvdt) and Eq. (dudt), over all pairs
 * r_ij < max(h_i, h_j), using the density state of the last sph_density /
 * sph_density_fixed_h (masses, h, rho, d rho/dh):
 *   u      internal energies (P_i = (gamma-1) rho_i u_i)
 *   vel    n x 3 float32 velocities (NULL = all zero)
 *   acc    out: n x 3 float32 dv_i/dt
 *   dudt   out (nullable): du_i/dt
 *   count  out (nullable, int32): partners j != i with r_ij < max(h_i,h_j)
 *          (FP32 predicate); when given the call synchronises and records
 *          the number of unordered pairs in sph_stats.force_pairs
 * With pair_list_cap > 0 the sweep also records every particle's pairs
 * (context-owned, 4 n pair_list_cap bytes) for the adjoint calls that
 * follow. */
int sph_force(sph_ctx* ctx, const float* u, const float* vel, float* acc, float* dudt,
              int32_t* count, void* stream);

/* Force with the Monaghan-Balsara artificial viscosity and the time step
 * (Section 4.1: the viscous terms added to Eq. (dvdt) and Eq. (dudt); Eq. (dt)),
 * at the h and densities of the last sph_density:
 *   a_i  = Eq. (dvdt) - 1/4 sum_j m_j Pi_ij (f_i + f_j) (grad W(r,h_i) + grad W(r,h_j)),
 *   du_i = Eq. (dudt) + 1/8 sum_j m_j Pi_ij (f_i + f_j) v_ij.(grad W(r,h_i) + grad W(r,h_j)),
 *   Pi_ij = -alpha (c_i + c_j - 3 w_ij) w_ij / (rho_i + rho_j), w_ij = min(0, v_ij.r_ij/r_ij),
 *   f_i = |div v_i| / (|div v_i| + |curl v_i| + 1e-4 c_i/h_i) (Balsara's switch, with div v
 *   and curl v summed over r < h_i), c = sqrt(gamma (gamma - 1) u),
 *   dt_i = c_cfl 2 h_i / max_j (c_i + c_j + max(0, -3 w_ij)),
 * sums and maximum over r_ij < max(h_i, h_j).
 *   u        [n] internal energies (caller order, device)
 *   vel      [3n] velocities, AoS (device; required)
 *   alpha    viscosity parameter (>= 0; the paper's runs use 0.8)
 *   c_cfl    CFL constant (> 0; the paper's runs use 1/4)
 *   acc      [3n] out, accelerations (AoS);  dudt [n] out (nullable);  dt [n] out
 *   balsara  [n] out, f_i (nullable)
 * Returns SPH_ERR_NOT_BUILT without a density, SPH_ERR_INVALID_ARG for bad
 * arguments.  The adjoints do not cover the viscous terms: after this call
 * sph_force_adjoint and the force part of sph_adjoint need a new sph_force. */
int sph_force_viscous(sph_ctx* ctx, const float* u, const float* vel, float alpha, float c_cfl,
                      float* acc, float* dudt, float* dt, float* balsara, void* stream);

/* One velocity-Verlet time step (Section 4.1: kick-drift-kick with one
 * global step) of the SPH equations with the artificial viscosity, for ONE
 * periodic cube [0, box)^3, advancing the caller's state in place:
 *   a0, du0 = forces at (pos, vel, u)                 (h solved afresh)
 *   vh = vel + dt/2 a0,  uh = u + dt/2 du0,  pos += dt vh (wrapped)
 *   a1, du1 = forces at (pos, vh + dt/2 a0, uh + dt/2 du0)
 *   vel = vh + dt/2 a1,  u = uh + dt/2 du1
 * where "forces" are Eq. (dvdt) and Eq. (dudt) with the Monaghan-Balsara
 * terms (sph_force_viscous; alpha = 0 gives the inviscid equations).  The
 * decomposition is kept from step to step (the pseudo-Verlet reuse of
 * Section 4.1): a decomposition built for h (1 + slack) serves while twice
 * the largest displacement since the build stays below the smallest margin
 * between a particle's cell limit and its h; the sweeps then widen their
 * axial cutoff and box tests by that amount.  Otherwise, or when a solved h
 * outgrows the reduced limit, the decomposition is rebuilt from the current
 * positions.  The first call builds it (h from the density estimate).
 * Between steps the context keeps the moved positions on that
 * decomposition: sph_density / sph_force / sph_force_viscous then run on it,
 * and report SPH_ERR_CELL_LIMIT (instead of rebuilding in place) when a
 * solved h outgrows it; sph_build starts afresh.
 *   n        particles (fixed across the steps of one context)
 *   pos      n x 3 float64 positions, in/out (device)
 *   vel      n x 3 float32 velocities, in/out;  u  n float32 energies, in/out
 *   m        n float32 masses
 *   dt       the step;  alpha, c_cfl  as for sph_force_viscous
 *   slack    extra cell margin as a fraction of h (0 < slack <= 1; 0.25 is usual)
 *   dt_min   out (HOST, nullable): the smallest time step of Eq. (dt) at the
 *            end of the step (evaluated with the predicted velocities)
 *   rebuilt  out (HOST, nullable): decompositions built during the step
 * Synchronises `stream`.  The adjoint calls do not cover this step. */
int sph_verlet_step(sph_ctx* ctx, int64_t n, double* pos, float* vel, float* u, const float* m,
                    double box, double dt, float alpha, float c_cfl, float slack, float* dt_min,
                    int32_t* rebuilt, void* stream);

/* Reverse mode of the ghost step and the force loop for a scalar L with
 * upstream gradients g_acc = dL/d acc (n x 3) and g_dudt = dL/d dudt
 * (nullable = 0), at the state of the last sph_force:
 *   g_pos  out: n x 3 float32, the force loop's part of dL/dx
 *   g_m    out: its part of dL/dm
 *   g_u    out: dL/du (complete: u enters only through P)
 *   g_rho  out: dL/d rho_i through P_i, Omega_i and A_i
 *   g_drho out: dL/d (d rho_i/d h_i) through Omega_i
 *   g_h    out: explicit dL/d h_i (kernel h-dependence of the force terms
 *          and of Omega_i), before the implicit h step */
int sph_force_adjoint(sph_ctx* ctx, const float* g_acc, const float* g_dudt, float* g_pos,
                      float* g_m, float* g_u, float* g_rho, float* g_drho, float* g_h,
                      void* stream);

/* Reverse mode of the density loop and of the implicit smoothing-length
 * solve: with total upstream g_rho, g_drho (nullable) and explicit g_h
 * (nullable), ADDS to g_pos (n x 3) and g_m the density loop's
 * contributions, including x-bar -= lambda_i dN_i/dx with
 * lambda_i = g_h_i / (dN_i/dh_i) (h solves N_i(h_i, x) = n_ngb). */
int sph_density_adjoint(sph_ctx* ctx, const float* g_rho, const float* g_drho,
                        const float* g_h, float* g_pos, float* g_m, void* stream);

/* Both adjoints in sequence for upstream (g_rho, g_acc, g_dudt); writes
 * g_pos (n x 3), g_m and g_u.  g_rho / g_acc / g_dudt may be NULL (= 0). */
int sph_adjoint(sph_ctx* ctx, const float* g_rho, const float* g_acc, const float* g_dudt,
                float* g_pos, float* g_m, float* g_u, void* stream);

/* Test hook: the accepted pair set of one sweep, in caller indices.
 *   phase 0: density at the current h (directed i<-j, r<h_i, self included)
 *   phase 1: force (ordered i != j, r < max(h_i, h_j))
 *   pi, pj  out: int32 device arrays of capacity `cap`
 *   n_out   out (HOST): number of pairs found (CAPACITY if > cap)
 * Synchronises `stream`. */
int sph_pairs_dump(sph_ctx* ctx, int32_t phase, int64_t cap, int32_t* pi, int32_t* pj,
                   int64_t* n_out, void* stream);

/* Enable (1) or disable (0) per-launch timing of the sweep kernels with
 * CUDA events recorded on the launch stream (no synchronisation is added),
 * counting variants of the sweeps (accepted pairs and candidates), the h
 * iteration as a host loop, and timing of the build stages (there the
 * stream is synchronised at each stage boundary); either call resets the
 * accumulated values.  sph_get_stats synchronises on the recorded events
 * and reports per-phase totals. */
int sph_profile(sph_ctx* ctx, int32_t enable);

/* Change the sweep launch shape of a built context (the decomposition is
 * kept): warps per CTA (1..8), shared-memory j buffer per warp (multiple of
 * 32, 32..1024) and resident CTAs per SM for the persistent grid (0 =
 * occupancy).  Results do not depend on these; speed does (the autotuner
 * in the Python package searches them). */
int sph_set_sweep_config(sph_ctx* ctx, int32_t warps_per_cta, int32_t sweep_cap,
                         int32_t ctas_per_sm);

/* Copy the statistics of the last calls into *out. */
int sph_get_stats(sph_ctx* ctx, sph_stats* out);

/* ---------------------------------------------------------------------------
 * Allocation-free entry point.  The paper has no counterpart: this exists
 * for callers that cannot call cudaMalloc, e.g. code that runs inside a
 * framework owning all device memory (a custom-call or plugin interface
 * that only hands in preplanned buffers), code on a real-time path where an
 * allocation may block or fail, or applications that must not grow their
 * device footprint after start-up.
 *
 * Density with the smoothing-length solve for ONE small periodic box
 * [0, box)^3: each h_i is moved by Newton steps inside an FP64 bracket until
 * the weighted neighbour number (32/3) sum_j w(r_ij/h_i) equals n_ngb, with
 * every sum taken by direct summation over all particle pairs (no cell
 * decomposition, no context), allocating nothing.  The per-particle
 * solver scratch (FP64 bracket, flags, sums) lives in a file-scope device
 * array sized for SPH_NOALLOC_MAX_N particles (about 0.6 MB) that every
 * GPU loading this library holds until the process exits.
 *   n        particles, 1..SPH_NOALLOC_MAX_N (larger n: SPH_ERR_INVALID_ARG
 *            and a message on stderr)
 *   pos      n x 3 float64 positions (device)
 *   m        n float32 masses (device)
 *   h_guess  n float32 initial h (device, nullable: the h holding n_ngb
 *            particles at the mean density)
 *   n_ngb    target weighted neighbour number (> 32/3; 48 is usual)
 *   max_iter Newton/bisection iterations at most
 *   h_out, rho_out  n float32 outputs (device; either may be NULL); rho_out
 *            is always the density at the h written to h_out
 *   iters    out (HOST, nullable): iterations used
 * Returns SPH_ERR_CELL_LIMIT if some h would exceed box/2 and
 * SPH_ERR_H_NOT_CONVERGED after max_iter.  Synchronises `stream`.
 * Every call looks up the scratch array's device address on the current
 * device (cudaGetSymbolAddress); the first call on a device also loads the
 * library's device code there, so make that first call before any stream
 * capture.  Every call on a device shares the one array,
 * which keeps the last call's contents: calls that overlap on the GPU
 * (different streams or host threads) race and must be serialised by the
 * caller. */
#define SPH_NOALLOC_MAX_N 16384
int sph_density_small_noalloc(int32_t n, const double* pos, double box, const float* m,
                              const float* h_guess, float n_ngb, int32_t max_iter, float* h_out,
                              float* rho_out, int32_t* iters, void* stream);

/* Number of kernel launches this library has issued since it was loaded
 * (all contexts). */
int64_t sph_launch_count(void);

/* A counter that changes with every call that replaces the context's
 * forward state (sph_build*, sph_density*, sph_force*); the adjoint calls
 * always differentiate the state of the latest such calls, so a caller that
 * holds on to a forward (an autograd graph) compares the counter before
 * asking for its adjoint.  -1 for NULL.  (Bookkeeping; no counterpart in
 * the paper.) */
int64_t sph_state_generation(const sph_ctx* ctx);

/* Synchronise `stream` and return (then clear) the device status word. */
int sph_sync_status(sph_ctx* ctx, void* stream);

/* Static description of a status code. */
const char* sph_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* SPHGB_H */
