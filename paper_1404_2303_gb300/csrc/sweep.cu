// Interaction sweeps: the sorted cell-pair interactions of Section 3.3 run
// as persistent warps.  A warp takes one particle block (a leaf cell or a
// slice of a large leaf) from an LPT-ordered queue and walks the block's
// directed interaction list: its own leaf (the self interaction, swept in
// a two-sided window along sort axis 0) and every cell it shares a final
// pair task with (the pair interaction, swept from the interface along the
// pair's sort axis, one of 13, up to the axial cutoff of the paper's sorted
// loop).  Each particle's sums stay in the registers of the lane that owns
// it, so no atomics touch the accumulators; each pair is evaluated from
// both sides instead of being updated symmetrically under the task
// conflicts of Section 3.4.
//
// Per chunk of 32 block particles (one per lane, consecutive in Morton
// order, so spatially compact) the warp first gathers: for every task it
// projects its particles on the task's sort axis, takes the chunk's axial
// window, and appends the j-particles inside it (shifted into the block's
// frame) to a shared-memory buffer.  When the buffer is full the warp
// computes: every lane evaluates every buffered j branch-free (the cubic
// spline's clamps zero everything beyond the support), then folds the
// buffer's partial sums into its running sums with a compensated
// (Neumaier) addition.
#include <algorithm>
#include <cfloat>

#include "geom.cuh"
#include "internal.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr float SIGMA = 2.546479089470325f;  // 8/pi

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
  return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(FULL, v, o));
  return v;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__constant__ float c_dir[SPH_NDIR][3];

// a pair-list entry: j (27 bits) and the top-cell image of j seen from i,
// one of (-1, 0, 1)^3 (5 bits): the shift is that vector times the box's
// top-cell edge, exactly the float shift of the pair task
constexpr unsigned TAG_J = (1u << 27) - 1u;
__device__ __forceinline__ int img_of(float s) { return s > 0.f ? 2 : (s < 0.f ? 0 : 1); }
__device__ __forceinline__ unsigned make_tag(int j, float sx, float sy, float sz) {
  return (unsigned)j | ((unsigned)(img_of(sx) * 9 + img_of(sy) * 3 + img_of(sz)) << 27);
}

struct SweepArgs {
  int nblock;
  int nunits;           // work units (slices of the blocks' interaction lists)
  const int* nunits_dev;  // non-null: the unit count of a compacted order, on the device
  int cap;  // buffered j-particles per warp between two compute passes
  const int* order;     // units in LPT order
  const int* u_block;   // unit -> block, slice index and entry range
  const int* u_seg;
  const long long* u_e0;
  const long long* u_e1;
  const int* b_nseg;    // slices per block
  const long long* b_part;  // partial-sum base of a block cut into slices (floats)
  float* part;
  int* blk_done;        // slices of the block finished in this launch
  const int* b_first;
  const int* b_count;
  const long long* b_dtoff;
  const int* dt_cj;
  const int* dt_code;
  const float4* dt_shift;
  const int* n_count;
  const long long* n_sbase;
  const int* n_child0;  // first child of a cell (-1: leaf)
  const float* n_hmax;
  const float* b_hmax;
  const float4* n_lo;   // particle bounding boxes of cells and blocks
  const float4* n_hi;
  const float4* b_lo;
  const float4* b_hi;
  const float* s_key;
  const int* s_idx;
  const float4* pos4;   // x_rel, y_rel, z_rel, m
  const float* h;
  const float4* vel4;   // vx, vy, vz, 1/h
  const float4* fdat;   // force: (D = 6 sigma m A / h^4, h^2, C = 6 sigma A / h^4, A)
  const float4* adj4;   // adjoint j data
  const float4* adj4b;
  const int* blk_active;
  int* queue;
  int* status;
  float delta;
  float gamma;          // viscosity: adiabatic index, alpha, C_CFL
  float alpha;
  float c_cfl;
  const float* rho_in;  // viscosity: rho and u (cell order), (c, rho, f, div v) per particle
  const float* u_in;
  const float4* visc4;
  int kahan;
  int naive;            // ablation: whole targets, no axial window, no box filter
  int bmax;             // largest block (particles)
  const int* pflag;     // h iteration: per-particle flags (bit 0: still iterating)
  // outputs (cell order)
  float* o0;
  float* o1;
  float* o2;
  float* o3;
  float* o6;
  float4* o4;
  float4* o5;
  int* ocnt;
  unsigned long long* units;  // profiling: accepted pairs, lane candidates, window entries
  // force pair lists (written by the force sweep, read by k_listeval)
  unsigned* fl_list;
  unsigned* sl_list;    // pair lists of the slices of blocks cut into work units
  int* fl_cnt;
  int* fl_flag;
  int* fl_blk;
  int* fl_over;
  int fl_K;
  const float* p_et;
  long long n;
  const int* run_if;    // non-null: the launch does nothing when *run_if == 0
  // pair dump
  const int* perm;
  int* dump_i;
  int* dump_j;
  unsigned long long* dump_n;
  long long dump_cap;
};

// ---------------------------------------------------------------------------
// density, Eq. (rho) and Eq. (nneigh): per directed interaction (i <- j),
// with w = 2 (a^3 - 4 b^3), w' = 6 (4 b^2 - a^2), w'' = 12 (a - 4 b),
// a = (1-q)+, b = (1/2-q)+, accumulate  m w/2,  m (w/2 + q w'/6),  w/2,
// q w'/6  and  q (q w''/12 + w'/6)  (the last for d^2 N/dh^2, which the h
// iteration's Halley step uses)
// ---------------------------------------------------------------------------
struct PDensity {
  static constexpr int NACC = 5;
  static constexpr int MINB = 4;  // resident CTAs per SM the register budget is set for
  static constexpr int NMAX = 0;  // trailing accumulators that take a maximum
  static constexpr int JW = 1;
  static constexpr bool WRITES = false;
  static constexpr bool USES_HJ = false;
  struct I {
    float x, y, z, h, hinv, h2;
  };
  __device__ static void load_i(const SweepArgs& a, int p, I& i) {
    float4 q = a.pos4[p];
    float h = a.h[p];
    i.x = q.x; i.y = q.y; i.z = q.z;
    i.h = h;
    i.hinv = 1.0f / h;
    i.h2 = __fmul_rn(h, h);
  }
  __device__ static void null_i(I& i) {
    i.x = i.y = i.z = 0.f;
    i.h = 0.f; i.hinv = 0.f; i.h2 = 0.f;
  }
  __device__ static float cut_h(float h, float) { return h; }
  __device__ static void stage(const SweepArgs& a, int j, unsigned tag, float4 pj, float4* tile, int lane,
                                int cap) {
    tile[lane] = pj;
  }
  // the directed-interaction predicate r < h_i in FP32
  __device__ static bool test(const I& i, const float4* tile, int t, int cap) {
    float4 p = tile[t];
    float dx = __fsub_rn(i.x, p.x), dy = __fsub_rn(i.y, p.y), dz = __fsub_rn(i.z, p.z);
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))) < i.h2;
  }
  template <bool COUNT>
  __device__ static void interact(const I& i, const float4* tile, int t, float* acc, int& cnt, int cap) {
    float4 p = tile[t];
    float dx = __fsub_rn(i.x, p.x), dy = __fsub_rn(i.y, p.y), dz = __fsub_rn(i.z, p.z);
    float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    float q = sqrt_approx(r2) * i.hinv;
    float aa = fmaxf(1.f - q, 0.f), bb = fmaxf(0.5f - q, 0.f);
    float a2 = aa * aa, b2 = bb * bb;
    float wh = fmaf(-4.f * b2, bb, a2 * aa);  // w/2
    float d6 = fmaf(4.f, b2, -a2);            // w'/6
    float qd = q * d6;
    acc[0] = fmaf(p.w, wh, acc[0]);
    acc[1] = fmaf(p.w, wh + qd, acc[1]);
    acc[2] += wh;
    acc[3] += qd;
    acc[4] = fmaf(q, fmaf(q, fmaf(-4.f, bb, aa), d6), acc[4]);
    if (COUNT) cnt += r2 < i.h2 ? 1 : 0;
  }
  // rho = sigma/h^3 * 2 S0; drho/dh = -sigma/h^4 * 6 S1; N = 64/3 S2; dN/dh = -64/h S3;
  // d^2N/dh^2 = 128/h^2 S4
  __device__ static void finalize(const SweepArgs& a, int p, const float* s) {
    float h = a.h[p];
    float hi = 1.0f / h;
    float hi3 = hi * hi * hi;
    a.o0[p] = 2.f * SIGMA * hi3 * s[0];
    if (a.o1) a.o1[p] = -6.f * SIGMA * hi3 * hi * s[1];
    if (a.o2) a.o2[p] = (64.f / 3.f) * s[2];
    if (a.o3) a.o3[p] = -64.f * hi * s[3];
    if (a.o6) a.o6[p] = 128.f * hi * hi * s[4];
  }
};

// d^2 rho / dh^2 = sigma/h^5 sum m (12 w + 8 q w' + q^2 w''), w'' = 12 (a - 4b)
struct PDensityD2 {
  static constexpr int NACC = 1;
  static constexpr int MINB = 3;  // resident CTAs per SM the register budget is set for
  static constexpr int NMAX = 0;  // trailing accumulators that take a maximum
  static constexpr int JW = 1;
  static constexpr bool WRITES = false;
  static constexpr bool USES_HJ = false;
  using I = PDensity::I;
  __device__ static void load_i(const SweepArgs& a, int p, I& i) { PDensity::load_i(a, p, i); }
  __device__ static void null_i(I& i) { PDensity::null_i(i); }
  __device__ static float cut_h(float h, float) { return h; }
  __device__ static void stage(const SweepArgs& a, int j, unsigned tag, float4 pj, float4* tile, int lane,
                                int cap) {
    PDensity::stage(a, j, tag, pj, tile, lane, cap);
  }
  __device__ static bool test(const I& i, const float4* tile, int t, int cap) {
    return PDensity::test(i, tile, t, cap);
  }
  template <bool COUNT>
  __device__ static void interact(const I& i, const float4* tile, int t, float* acc, int& cnt, int cap) {
    float4 p = tile[t];
    float dx = __fsub_rn(i.x, p.x), dy = __fsub_rn(i.y, p.y), dz = __fsub_rn(i.z, p.z);
    float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    float q = sqrt_approx(r2) * i.hinv;
    float aa = fmaxf(1.f - q, 0.f), bb = fmaxf(0.5f - q, 0.f);
    float a2 = aa * aa, b2 = bb * bb;
    float w = 2.f * fmaf(-4.f * b2, bb, a2 * aa);
    float dw = 6.f * fmaf(4.f, b2, -a2);
    float d2w = 12.f * (aa - 4.f * bb);
    acc[0] = fmaf(p.w, fmaf(12.f, w, q * fmaf(8.f, dw, q * d2w)), acc[0]);
    if (COUNT) cnt += r2 < i.h2 ? 1 : 0;
  }
  __device__ static void finalize(const SweepArgs& a, int p, const float* s) {
    float hi = 1.0f / a.h[p];
    float hi2 = hi * hi;
    a.o0[p] = SIGMA * hi2 * hi2 * hi * s[0];
  }
};

// ---------------------------------------------------------------------------
// force, Eq. (dvdt) and (dudt), gathered from i's side over r < max(h_i, h_j):
//   a_i  = -sum_j (m_j C_i w'_i/6 + D_j w'_j/6) (x_i - x_j)/r
//   du_i = C_i sum_j m_j (w'_i/6) (v_i - v_j).(x_i - x_j)/r
// with C = 6 sigma A / h^4, D = m C, A = P/(Omega rho^2)
// ---------------------------------------------------------------------------
struct PForce {
  static constexpr int NACC = 4;
  static constexpr int MINB = 2;  // resident CTAs per SM the register budget is set for
  static constexpr int NMAX = 0;  // trailing accumulators that take a maximum
  static constexpr int JW = 3;
  static constexpr bool WRITES = true;  // records the pair lists
  static constexpr bool USES_HJ = true;
  struct I {
    float x, y, z, vx, vy, vz, h, hinv, h2, C;
    int p;
  };
  __device__ static void load_i(const SweepArgs& a, int p, I& i) {
    float4 q = a.pos4[p];
    float4 v = a.vel4[p];
    float4 f = a.fdat[p];
    i.p = p;
    i.x = q.x; i.y = q.y; i.z = q.z;
    i.vx = v.x; i.vy = v.y; i.vz = v.z;
    i.hinv = v.w;
    i.h = a.h[p];
    i.h2 = f.y;
    i.C = f.z;
  }
  __device__ static void null_i(I& i) {
    i.x = i.y = i.z = i.vx = i.vy = i.vz = 0.f;
    i.h = i.hinv = i.h2 = i.C = 0.f;
    i.p = -1;
  }
  __device__ static float cut_h(float h, float hj) { return fmaxf(h, hj); }
  __device__ static void stage(const SweepArgs& a, int j, unsigned tag, float4 pj, float4* tile, int lane,
                                int cap) {
    tile[lane] = pj;
    tile[cap + lane] = a.vel4[j];
    float4 f = a.fdat[j];
    tile[2 * cap + lane] = make_float4(f.x, f.y, f.z, __uint_as_float(tag));
  }
  // the force-pair predicate r < max(h_i, h_j) in FP32
  __device__ static bool test(const I& i, const float4* tile, int t, int cap) {
    float4 p = tile[t];
    float dx = __fsub_rn(i.x, p.x), dy = __fsub_rn(i.y, p.y), dz = __fsub_rn(i.z, p.z);
    float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    return r2 < fmaxf(i.h2, tile[2 * cap + t].y);
  }
  template <bool COUNT>
  __device__ static void interact(const I& i, const float4* tile, int t, float* acc, int& cnt, int cap) {
    float4 p = tile[t];
    float4 v = tile[cap + t];
    float4 f = tile[2 * cap + t];
    float dx = __fsub_rn(i.x, p.x), dy = __fsub_rn(i.y, p.y), dz = __fsub_rn(i.z, p.z);
    float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    float rinv = r2 > 0.f ? rsqrt_approx(r2) : 0.f;
    float r = r2 * rinv;
    float qi = r * i.hinv, qj = r * v.w;
    float ai = fmaxf(1.f - qi, 0.f), bi = fmaxf(0.5f - qi, 0.f);
    float aj = fmaxf(1.f - qj, 0.f), bj = fmaxf(0.5f - qj, 0.f);
    float di = fmaf(4.f * bi, bi, -ai * ai);
    float dj = fmaf(4.f * bj, bj, -aj * aj);
    float tm = p.w * di;
    float coef = fmaf(tm, i.C, f.x * dj) * rinv;
    acc[0] = fmaf(coef, dx, acc[0]);
    acc[1] = fmaf(coef, dy, acc[1]);
    acc[2] = fmaf(coef, dz, acc[2]);
    float vd = fmaf(i.vz - v.z, dz, fmaf(i.vy - v.y, dy, (i.vx - v.x) * dx));
    acc[3] = fmaf(tm * rinv, vd, acc[3]);
    if (COUNT) cnt += (r2 < fmaxf(i.h2, f.y) && (int)(__float_as_uint(f.w) & TAG_J) != i.p) ? 1 : 0;
  }
  __device__ static void finalize(const SweepArgs& a, int p, const float* s) {
    float C = a.fdat[p].z;
    a.o4[p] = make_float4(-s[0], -s[1], -s[2], C * s[3]);
  }
};

// ---------------------------------------------------------------------------
// force adjoint: reverse mode of Eq. (dvdt)/(dudt) gathered from i's side.
// With xh = (x_i - x_j)/r, G = dW/dr = 6 sigma/h^4 d6, G' = 12 sigma/h^5 e,
// dG/dh = -sigma/h^5 (24 d6 + 12 q e)  (d6 = w'/6, e = w''/12), and
// upstream abar (acc) and ubar (du/dt):
//   gA_i += G_i [ -m_j abar_i.xh + m_i abar_j.xh + ubar_i m_j t ]
//   gh_i += dG/dh_i [ same bracket ]              (times A_i at the end)
//   gm_i += Phi abar_j.xh + ubar_j A_j G_j t
//   gx_i += (c1 - c2 beta - c3 t) xh + c2 b + c3 v_ij
// where t = v_ij.xh, Phi = A_i G_i + A_j G_j, b = m_i abar_j - m_j abar_i,
// beta = b.xh, c1 = Phi' beta + (E G'_i + F G'_j) t, c2 = Phi/r,
// c3 = (E G_i + F G_j)/r, E = ubar_i A_i m_j, F = ubar_j A_j m_i.
// ---------------------------------------------------------------------------
struct PForceAdj {
  static constexpr int NACC = 6;  // gx, gy, gz, gm, gA, gh
  static constexpr int MINB = 2;  // resident CTAs per SM the register budget is set for
  static constexpr int NMAX = 0;  // trailing accumulators that take a maximum
  static constexpr int JW = 4;
  static constexpr bool WRITES = false;
  static constexpr bool USES_HJ = true;
  struct I {
    float x, y, z, m, vx, vy, vz, h, hinv, h2, A, ax, ay, az, ub;
  };
  __device__ static void load_i(const SweepArgs& a, int p, I& i) {
    float4 q = a.pos4[p], v = a.vel4[p], g = a.adj4[p], f = a.fdat[p];
    i.x = q.x; i.y = q.y; i.z = q.z; i.m = q.w;
    i.vx = v.x; i.vy = v.y; i.vz = v.z; i.hinv = v.w;
    i.h = a.h[p];
    i.h2 = f.y;
    i.A = f.w;
    i.ax = g.x; i.ay = g.y; i.az = g.z; i.ub = g.w;
  }
  __device__ static void null_i(I& i) {
    i.x = i.y = i.z = i.m = i.vx = i.vy = i.vz = i.h = i.hinv = i.h2 = i.A = 0.f;
    i.ax = i.ay = i.az = i.ub = 0.f;
  }
  __device__ static float cut_h(float h, float hj) { return fmaxf(h, hj); }
  __device__ static void stage(const SweepArgs& a, int j, unsigned tag, float4 pj, float4* tile, int lane,
                                int cap) {
    tile[lane] = pj;
    tile[cap + lane] = a.vel4[j];
    tile[2 * cap + lane] = a.adj4[j];
    const float4 f = a.fdat[j];
    tile[3 * cap + lane] = make_float4(f.w, f.y, 0.f, 0.f);
  }
  __device__ static bool test(const I& i, const float4* tile, int t, int cap) {
    float4 p = tile[t];
    float dx = __fsub_rn(i.x, p.x), dy = __fsub_rn(i.y, p.y), dz = __fsub_rn(i.z, p.z);
    float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    return r2 < fmaxf(i.h2, tile[3 * cap + t].y);
  }
  template <bool COUNT>
  __device__ static void interact(const I& i, const float4* tile, int t, float* acc, int& cnt, int cap) {
    float4 p = tile[t], v = tile[cap + t], g = tile[2 * cap + t];
    float Aj = tile[3 * cap + t].x;
    float dx = __fsub_rn(i.x, p.x), dy = __fsub_rn(i.y, p.y), dz = __fsub_rn(i.z, p.z);
    float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    float rinv = r2 > 0.f ? rsqrt_approx(r2) : 0.f;
    float r = r2 * rinv;
    float xx = dx * rinv, xy = dy * rinv, xz = dz * rinv;
    float qi = r * i.hinv, qj = r * v.w;
    float ai = fmaxf(1.f - qi, 0.f), bi = fmaxf(0.5f - qi, 0.f);
    float aj = fmaxf(1.f - qj, 0.f), bj = fmaxf(0.5f - qj, 0.f);
    float d6i = fmaf(4.f * bi, bi, -ai * ai), d6j = fmaf(4.f * bj, bj, -aj * aj);
    float ei = fmaf(-4.f, bi, ai), ej = fmaf(-4.f, bj, aj);
    float hi2 = i.hinv * i.hinv, hj2 = v.w * v.w;
    float hi4 = hi2 * hi2, hj4 = hj2 * hj2;
    float Gi = 6.f * SIGMA * hi4 * d6i, Gj = 6.f * SIGMA * hj4 * d6j;
    float Gpi = 12.f * SIGMA * hi4 * i.hinv * ei, Gpj = 12.f * SIGMA * hj4 * v.w * ej;
    float Ghi = -SIGMA * hi4 * i.hinv * fmaf(24.f, d6i, 12.f * qi * ei);
    float vx = i.vx - v.x, vy = i.vy - v.y, vz = i.vz - v.z;
    float tt = fmaf(vz, xz, fmaf(vy, xy, vx * xx));
    float sai = fmaf(i.az, xz, fmaf(i.ay, xy, i.ax * xx));
    float saj = fmaf(g.z, xz, fmaf(g.y, xy, g.x * xx));
    float br = fmaf(i.ub * p.w, tt, fmaf(i.m, saj, -p.w * sai));
    acc[4] = fmaf(Gi, br, acc[4]);
    acc[5] = fmaf(Ghi, br, acc[5]);
    float Phi = fmaf(i.A, Gi, Aj * Gj);
    float dPhi = fmaf(i.A, Gpi, Aj * Gpj);
    float E = i.ub * i.A * p.w, F = g.w * Aj * i.m;
    acc[3] = fmaf(Phi, saj, fmaf(g.w * Aj * Gj, tt, acc[3]));
    float bx = fmaf(i.m, g.x, -p.w * i.ax), by = fmaf(i.m, g.y, -p.w * i.ay),
          bz = fmaf(i.m, g.z, -p.w * i.az);
    float beta = fmaf(i.m, saj, -p.w * sai);
    float c1 = fmaf(dPhi, beta, fmaf(E, Gpi, F * Gpj) * tt);
    float c2 = Phi * rinv;
    float c3 = fmaf(E, Gi, F * Gj) * rinv;
    float cx = c1 - c2 * beta - c3 * tt;
    acc[0] = fmaf(cx, xx, fmaf(c2, bx, fmaf(c3, vx, acc[0])));
    acc[1] = fmaf(cx, xy, fmaf(c2, by, fmaf(c3, vy, acc[1])));
    acc[2] = fmaf(cx, xz, fmaf(c2, bz, fmaf(c3, vz, acc[2])));
    if (COUNT) cnt += (r2 > 0.f && (qi < 1.f || qj < 1.f)) ? 1 : 0;
  }
  __device__ static void finalize(const SweepArgs& a, int p, const float* s) {
    a.o4[p] = make_float4(s[0], s[1], s[2], s[3]);
    a.o0[p] = s[4];
    a.o1[p] = s[5];
  }
};

// ---------------------------------------------------------------------------
// density adjoint: reverse mode of Eq. (rho), of d rho/dh and of the
// implicit h of Eq. (nneigh), gathered from i's side over r < max(h_i, h_j).
// Per particle k (precomputed): P_k = 2 sigma/h^3 rbar_k,
// Q_k = 6 sigma/h^4 rbar'_k, R_k = 6 sigma/h^4 rbar_k, S_k = sigma/h^5 rbar'_k,
// L_k = 64 lambda_k / h_k  (rbar = dL/drho, rbar' = dL/d(drho/dh),
// lambda_k = hbar_k / (dN_k/dh_k)).  With wh = w/2, d6 = w'/6, e = w''/12:
//   gm_i += P_j wh_j - Q_j (wh_j + q_j d6_j)          (r < h_j, self included)
//   T_k   = m_other [R_k d6_k - S_k (24 d6_k + 12 q_k e_k)] - L_k d6_k
//   gx_i += (T_i + T_j) (x_i - x_j)/r
// ---------------------------------------------------------------------------
struct PDensityAdj {
  static constexpr int NACC = 4;  // gx, gy, gz, gm
  static constexpr int MINB = 3;  // resident CTAs per SM the register budget is set for
  static constexpr int NMAX = 0;  // trailing accumulators that take a maximum
  static constexpr int JW = 3;
  static constexpr bool WRITES = false;
  static constexpr bool USES_HJ = true;
  struct I {
    float x, y, z, m, h, hinv, h2, R, S, L;
  };
  __device__ static void load_i(const SweepArgs& a, int p, I& i) {
    float4 q = a.pos4[p], u = a.adj4[p], w = a.adj4b[p];
    i.x = q.x; i.y = q.y; i.z = q.z; i.m = q.w;
    i.h = a.h[p];
    i.hinv = u.x;
    i.h2 = w.z;
    i.R = u.w; i.S = w.x; i.L = w.y;
  }
  __device__ static void null_i(I& i) {
    i.x = i.y = i.z = i.m = i.h = i.hinv = i.h2 = i.R = i.S = i.L = 0.f;
  }
  __device__ static float cut_h(float h, float hj) { return fmaxf(h, hj); }
  __device__ static void stage(const SweepArgs& a, int j, unsigned tag, float4 pj, float4* tile, int lane,
                                int cap) {
    tile[lane] = pj;
    tile[cap + lane] = a.adj4[j];
    tile[2 * cap + lane] = a.adj4b[j];
  }
  // r < max(h_i, h_j); the self term (r = 0) is included
  __device__ static bool test(const I& i, const float4* tile, int t, int cap) {
    float4 p = tile[t];
    float dx = __fsub_rn(i.x, p.x), dy = __fsub_rn(i.y, p.y), dz = __fsub_rn(i.z, p.z);
    float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    return r2 < fmaxf(i.h2, tile[2 * cap + t].z);
  }
  template <bool COUNT>
  __device__ static void interact(const I& i, const float4* tile, int t, float* acc, int& cnt, int cap) {
    float4 p = tile[t], u = tile[cap + t], w = tile[2 * cap + t];
    float dx = __fsub_rn(i.x, p.x), dy = __fsub_rn(i.y, p.y), dz = __fsub_rn(i.z, p.z);
    float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    float rinv = r2 > 0.f ? rsqrt_approx(r2) : 0.f;
    float r = r2 * rinv;
    float qi = r * i.hinv, qj = r * u.x;
    float ai = fmaxf(1.f - qi, 0.f), bi = fmaxf(0.5f - qi, 0.f);
    float aj = fmaxf(1.f - qj, 0.f), bj = fmaxf(0.5f - qj, 0.f);
    float ai2 = ai * ai, bi2 = bi * bi, aj2 = aj * aj, bj2 = bj * bj;
    float d6i = fmaf(4.f, bi2, -ai2), d6j = fmaf(4.f, bj2, -aj2);
    float ei = fmaf(-4.f, bi, ai), ej = fmaf(-4.f, bj, aj);
    float whj = fmaf(-4.f * bj2, bj, aj2 * aj);
    acc[3] = fmaf(u.y, whj, fmaf(-u.z, fmaf(qj, d6j, whj), acc[3]));
    float Ti = fmaf(p.w, fmaf(i.R, d6i, -i.S * fmaf(24.f, d6i, 12.f * qi * ei)), -i.L * d6i);
    float Tj = fmaf(i.m, fmaf(u.w, d6j, -w.x * fmaf(24.f, d6j, 12.f * qj * ej)), -w.y * d6j);
    float c = (Ti + Tj) * rinv;
    acc[0] = fmaf(c, dx, acc[0]);
    acc[1] = fmaf(c, dy, acc[1]);
    acc[2] = fmaf(c, dz, acc[2]);
    if (COUNT) cnt += (r2 > 0.f && (qi < 1.f || qj < 1.f)) ? 1 : 0;
  }
  __device__ static void finalize(const SweepArgs& a, int p, const float* s) {
    float4 o = a.o4[p];
    a.o4[p] = make_float4(o.x + s[0], o.y + s[1], o.z + s[2], o.w + s[3]);
  }
};

// ---------------------------------------------------------------------------
// velocity divergence and curl (Section 4.1) over r < h_i, with
// gW = grad W(r, h_i) = (6 sigma/h_i^4)(w'/6)(x_i - x_j)/r:
//   S_div = sum_j m_j (v_j - v_i) . gW,  S_curl = sum_j m_j (v_j - v_i) x gW,
// div v_i = S_div/rho_i, curl v_i = -S_curl/rho_i, and the Balsara switch
// f_i = |div v_i| / (|div v_i| + |curl v_i| + 1e-4 c_i/h_i), c = sqrt(g(g-1)u)
// ---------------------------------------------------------------------------
struct PVelDeriv {
  static constexpr int NACC = 4;  // div, curl x, y, z
  static constexpr int MINB = 2;  // resident CTAs per SM the register budget is set for
  static constexpr int NMAX = 0;
  static constexpr int JW = 2;
  static constexpr bool USES_HJ = false;
  static constexpr bool WRITES = false;
  struct I {
    float x, y, z, vx, vy, vz, h, h2, hinv, G0;
  };
  __device__ static void load_i(const SweepArgs& a, int p, I& i) {
    float4 q = a.pos4[p], v = a.vel4[p];
    float h = a.h[p];
    i.x = q.x; i.y = q.y; i.z = q.z;
    i.vx = v.x; i.vy = v.y; i.vz = v.z;
    i.hinv = v.w;
    i.h = h;
    i.h2 = __fmul_rn(h, h);
    float hi2 = v.w * v.w;
    i.G0 = 6.f * SIGMA * hi2 * hi2;
  }
  __device__ static void null_i(I& i) {
    i.x = i.y = i.z = i.vx = i.vy = i.vz = i.h = i.h2 = i.hinv = i.G0 = 0.f;
  }
  __device__ static float cut_h(float h, float) { return h; }
  __device__ static void stage(const SweepArgs& a, int j, unsigned tag, float4 pj, float4* tile, int lane,
                                int cap) {
    tile[lane] = pj;
    tile[cap + lane] = a.vel4[j];
  }
  __device__ static bool test(const I& i, const float4* tile, int t, int cap) {
    float4 p = tile[t];
    float dx = __fsub_rn(i.x, p.x), dy = __fsub_rn(i.y, p.y), dz = __fsub_rn(i.z, p.z);
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))) < i.h2;
  }
  template <bool COUNT>
  __device__ static void interact(const I& i, const float4* tile, int t, float* acc, int& cnt, int cap) {
    float4 p = tile[t], v = tile[cap + t];
    float dx = __fsub_rn(i.x, p.x), dy = __fsub_rn(i.y, p.y), dz = __fsub_rn(i.z, p.z);
    float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    float rinv = r2 > 0.f ? rsqrt_approx(r2) : 0.f;
    float q = r2 * rinv * i.hinv;
    float aa = fmaxf(1.f - q, 0.f), bb = fmaxf(0.5f - q, 0.f);
    float g = p.w * i.G0 * fmaf(4.f * bb, bb, -aa * aa) * rinv;  // m_j |gW| / r
    float ux = v.x - i.vx, uy = v.y - i.vy, uz = v.z - i.vz;   // v_j - v_i
    acc[0] = fmaf(g, fmaf(uz, dz, fmaf(uy, dy, ux * dx)), acc[0]);
    acc[1] = fmaf(g, fmaf(uy, dz, -uz * dy), acc[1]);
    acc[2] = fmaf(g, fmaf(uz, dx, -ux * dz), acc[2]);
    acc[3] = fmaf(g, fmaf(ux, dy, -uy * dx), acc[3]);
    if (COUNT) cnt += r2 < i.h2 ? 1 : 0;
  }
  __device__ static void finalize(const SweepArgs& a, int p, const float* s) {
    const float rho = a.rho_in[p];
    const float div = s[0] / rho;
    const float cx = -s[1] / rho, cy = -s[2] / rho, cz = -s[3] / rho;
    const float c = sqrtf(a.gamma * (a.gamma - 1.f) * a.u_in[p]);
    const float ad = fabsf(div), ac = sqrtf(fmaf(cz, cz, fmaf(cy, cy, cx * cx)));
    const float f = ad / (ad + ac + 1e-4f * c / a.h[p]);
    a.o5[p] = make_float4(c, rho, f, div);
  }
};

// ---------------------------------------------------------------------------
// force with the Monaghan-Balsara viscosity of Section 4.1 and the signal
// speed of Eq. (dt), over r < max(h_i, h_j).  On top of PForce's terms:
//   a_i  -= 1/4 m_j Pi_ij (f_i + f_j) (G_i + G_j) (x_i - x_j)/r
//   du_i += 1/8 m_j Pi_ij (f_i + f_j) (G_i + G_j) v_ij.(x_i - x_j)/r
//   Pi_ij = -alpha (c_i + c_j - 3 w_ij) w_ij / (rho_i + rho_j),
//   w_ij = min(0, v_ij.(x_i - x_j)/r), G = dW/dr = (6 sigma/h^4)(w'/6),
// and the largest c_i + c_j + max(0, -3 w_ij) over the pairs with r > 0
// ---------------------------------------------------------------------------
struct PForceVisc {
  static constexpr int NACC = 6;  // a (3), du pressure, du viscous, max signal speed
  static constexpr int MINB = 2;  // resident CTAs per SM the register budget is set for
  static constexpr int NMAX = 1;
  static constexpr int JW = 4;
  static constexpr bool USES_HJ = true;
  static constexpr bool WRITES = false;
  struct I {
    float x, y, z, vx, vy, vz, h, hinv, h2, C, G0, c, rho, f, alpha;
    int p;
  };
  __device__ static void load_i(const SweepArgs& a, int p, I& i) {
    float4 q = a.pos4[p], v = a.vel4[p], f = a.fdat[p], w = a.visc4[p];
    i.p = p;
    i.h = a.h[p];
    i.x = q.x; i.y = q.y; i.z = q.z;
    i.vx = v.x; i.vy = v.y; i.vz = v.z;
    i.hinv = v.w;
    i.h2 = f.y;
    i.C = f.z;
    float hi2 = v.w * v.w;
    i.G0 = 6.f * SIGMA * hi2 * hi2;
    i.c = w.x; i.rho = w.y; i.f = w.z;
    i.alpha = a.alpha;
  }
  __device__ static void null_i(I& i) {
    i.x = i.y = i.z = i.vx = i.vy = i.vz = i.h = i.hinv = i.h2 = i.C = i.G0 = 0.f;
    i.c = 0.f; i.rho = 1.f; i.f = 0.f; i.alpha = 0.f;
    i.p = -1;
  }
  __device__ static float cut_h(float h, float hj) { return fmaxf(h, hj); }
  __device__ static void stage(const SweepArgs& a, int j, unsigned tag, float4 pj, float4* tile, int lane,
                                int cap) {
    tile[lane] = pj;
    tile[cap + lane] = a.vel4[j];
    float4 f = a.fdat[j];
    tile[2 * cap + lane] = make_float4(f.x, f.y, f.z, __int_as_float(j));
    tile[3 * cap + lane] = a.visc4[j];
  }
  __device__ static bool test(const I& i, const float4* tile, int t, int cap) {
    float4 p = tile[t];
    float dx = __fsub_rn(i.x, p.x), dy = __fsub_rn(i.y, p.y), dz = __fsub_rn(i.z, p.z);
    float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    return r2 < fmaxf(i.h2, tile[2 * cap + t].y);
  }
  template <bool COUNT>
  __device__ static void interact(const I& i, const float4* tile, int t, float* acc, int& cnt, int cap) {
    float4 p = tile[t], v = tile[cap + t], f = tile[2 * cap + t], w = tile[3 * cap + t];
    float dx = __fsub_rn(i.x, p.x), dy = __fsub_rn(i.y, p.y), dz = __fsub_rn(i.z, p.z);
    float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    float rinv = r2 > 0.f ? rsqrt_approx(r2) : 0.f;
    float r = r2 * rinv;
    float qi = r * i.hinv, qj = r * v.w;
    float ai = fmaxf(1.f - qi, 0.f), bi = fmaxf(0.5f - qi, 0.f);
    float aj = fmaxf(1.f - qj, 0.f), bj = fmaxf(0.5f - qj, 0.f);
    float di = fmaf(4.f * bi, bi, -ai * ai);
    float dj = fmaf(4.f * bj, bj, -aj * aj);
    // pressure (as PForce)
    float tm = p.w * di;
    float coef = fmaf(tm, i.C, f.x * dj) * rinv;
    float vx = i.vx - v.x, vy = i.vy - v.y, vz = i.vz - v.z;
    float vd = fmaf(vz, dz, fmaf(vy, dy, vx * dx));   // v_ij . (x_i - x_j)
    acc[3] = fmaf(tm * rinv, vd, acc[3]);
    // viscosity
    float wv = fminf(0.f, vd * rinv);
    float Pi = -i.alpha * (i.c + w.x - 3.f * wv) * wv / (i.rho + w.y);
    float hj2 = v.w * v.w;
    float gs = fmaf(i.G0, di, 6.f * SIGMA * hj2 * hj2 * dj) * rinv;  // (G_i + G_j)/r
    float kv = p.w * Pi * (i.f + w.z) * gs;
    float ct = fmaf(0.25f, kv, coef);
    acc[0] = fmaf(ct, dx, acc[0]);
    acc[1] = fmaf(ct, dy, acc[1]);
    acc[2] = fmaf(ct, dz, acc[2]);
    acc[4] = fmaf(0.125f * kv, vd, acc[4]);
    // signal speed of Eq. (dt) over the force pairs (r > 0)
    const bool pair = r2 > 0.f && r2 < fmaxf(i.h2, f.y);
    acc[5] = fmaxf(acc[5], pair ? i.c + w.x + fmaxf(0.f, -3.f * vd * rinv) : 0.f);
    if (COUNT) cnt += (r2 < fmaxf(i.h2, f.y) && __float_as_int(f.w) != i.p) ? 1 : 0;
  }
  __device__ static void finalize(const SweepArgs& a, int p, const float* s) {
    const float C = a.fdat[p].z;
    a.o4[p] = make_float4(-s[0], -s[1], -s[2], fmaf(C, s[3], s[4]));
    const float c = a.visc4[p].x;
    const float sig = s[5] > 0.f ? s[5] : 2.f * c;
    a.o0[p] = a.c_cfl * 2.f * a.h[p] / sig;
  }
};

// ---------------------------------------------------------------------------
// pair dump (test hook): records accepted pairs in caller indices
// ---------------------------------------------------------------------------
template <int FORCE>
struct PDump {
  static constexpr int NACC = 1;
  static constexpr int MINB = 3;  // resident CTAs per SM the register budget is set for
  static constexpr int NMAX = 0;  // trailing accumulators that take a maximum
  static constexpr int JW = 2;
  static constexpr bool WRITES = false;
  static constexpr bool USES_HJ = FORCE != 0;
  struct I {
    float x, y, z, h, h2;
    int p;
    const SweepArgs* a;
  };
  __device__ static void load_i(const SweepArgs& a, int p, I& i) {
    float4 q = a.pos4[p];
    float h = a.h[p];
    i.x = q.x; i.y = q.y; i.z = q.z;
    i.h = h;
    i.h2 = __fmul_rn(h, h);
    i.p = p;
    i.a = &a;
  }
  __device__ static void null_i(I& i) {
    i.x = i.y = i.z = 0.f;
    i.h = 0.f; i.h2 = -1.f;
    i.p = -1;
    i.a = nullptr;
  }
  __device__ static float cut_h(float h, float hj) { return FORCE ? fmaxf(h, hj) : h; }
  __device__ static void stage(const SweepArgs& a, int j, unsigned tag, float4 pj, float4* tile, int lane,
                                int cap) {
    float h = a.h[j];
    tile[lane] = pj;
    tile[cap + lane] = make_float4(__fmul_rn(h, h), __int_as_float(j), 0.f, 0.f);
  }
  __device__ static bool test(const I&, const float4*, int, int) { return true; }
  template <bool COUNT>
  __device__ static void interact(const I& i, const float4* tile, int t, float* acc, int& cnt, int cap) {
    if (i.p < 0) return;
    float4 p = tile[t];
    float4 e = tile[cap + t];
    float dx = __fsub_rn(i.x, p.x), dy = __fsub_rn(i.y, p.y), dz = __fsub_rn(i.z, p.z);
    float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    int j = __float_as_int(e.y);
    bool ok = FORCE ? (r2 < fmaxf(i.h2, e.x) && j != i.p) : (r2 < i.h2);
    if (ok) {
      const SweepArgs& a = *i.a;
      unsigned long long k = atomicAdd(a.dump_n, 1ull);
      if ((long long)k < a.dump_cap) {
        a.dump_i[k] = a.perm[i.p];
        a.dump_j[k] = a.perm[j];
      }
    }
    (void)acc;
    (void)cnt;
  }
  __device__ static void finalize(const SweepArgs&, int, const float*) {}
};

// ---------------------------------------------------------------------------
// the generic persistent sweep
// ---------------------------------------------------------------------------
template <class P>
__device__ __forceinline__ void fold(float* acc, float* cmp, float* part, int kahan) {
#pragma unroll
  for (int k = 0; k < P::NACC; ++k) {
    float x = part[k];
    if (k >= P::NACC - P::NMAX) {  // a running maximum (partials start at 0)
      acc[k] = fmaxf(acc[k], x);
    } else if (kahan) {
      float S = acc[k];
      float T = S + x;
      cmp[k] += fabsf(S) >= fabsf(x) ? (S - T) + x : (x - T) + S;
      acc[k] = T;
    } else {
      acc[k] += x;
    }
    part[k] = 0.f;
  }
}

// One compute pass over the buffered j-particles.  A lane evaluates the
// candidates t = sub, sub + G, sub + 2G, ... for the particle it serves: G = 1
// (one particle per lane, every candidate) unless the chunk holds few
// particles, when G lanes share one particle (see k_sweep).  Without lists
// the evaluation is branch-free (the spline's clamps zero the pairs beyond
// the support), so a lane pays the full interaction for each candidate.
// With lists each lane first applies the exact FP32 predicate of its phase
// to its candidates and records the accepted slots in its own column of a
// byte list (lane-private, so no synchronisation between the two loops),
// then evaluates only those: the warp runs as long as its longest list
// instead of the whole buffer.
// A phase that records pair lists (WRITES) appends the tag of every
// accepted pair to its particle's list column wl (entry k at wl[32 k]):
// the G lanes of a particle write at their exclusive prefix within the
// group after the group's running total wtot, which keeps counting past the
// capacity wcap to flag the overflow.
template <class P, bool COUNT, bool LIST>
__device__ __forceinline__ void compute_pass(const typename P::I& I, bool vi, const float4* buf,
                                             unsigned char* lst, int staged, int cap, float* part,
                                             int& cnt, unsigned* wl, int& wtot, int wcap, int sub,
                                             int G) {
  __syncwarp();
  if (LIST) {
    const int lane = threadIdx.x & 31;
    int nl = 0;
    if (vi) {
#pragma unroll 4
      for (int t = sub; t < staged; t += G) {
        if (P::test(I, buf, t, cap)) {
          lst[nl * 32 + lane] = (unsigned char)t;
          ++nl;
        }
      }
    }
    int pre = 0, gtot = nl;
    if (P::WRITES && G > 1) {  // exclusive prefix of the accepted counts within the group
      int x = nl;
      for (int o = 1; o < G; o <<= 1) {
        const int y = __shfl_up_sync(FULL, x, o);
        if ((lane & (G - 1)) >= o) x += y;
      }
      pre = x - nl;
      gtot = __shfl_sync(FULL, x, (lane | (G - 1)));
    }
    const int nmax = __reduce_max_sync(FULL, nl);
    for (int k = 0; k < nmax; ++k) {
      if (k < nl) {
        const int t = lst[k * 32 + lane];
        P::template interact<COUNT>(I, buf, t, part, cnt, cap);
        if (P::WRITES && wl) {
          const int e = wtot + pre + k;
          if (e < wcap) wl[(size_t)e * 32] = __float_as_uint(buf[2 * cap + t].w);
        }
      }
    }
    if (P::WRITES) wtot += gtot;
  } else {
#pragma unroll 2
    for (int t = sub; t < staged; t += G) P::template interact<COUNT>(I, buf, t, part, cnt, cap);
  }
  __syncwarp();
}

// first index in [0, n) whose predicate flips from true to false, for a
// predicate true on a prefix (binary search, one lane)
#define SPH_PARTITION(n, pred_of_mid, out)       \
  do {                                           \
    int lo_ = 0, hi_ = (n);                      \
    while (lo_ < hi_) {                          \
      int mid = (lo_ + hi_) >> 1;                \
      if (pred_of_mid) lo_ = mid + 1; else hi_ = mid; \
    }                                            \
    (out) = lo_;                                 \
  } while (0)

// a listed target of at least DESC_MIN particles of which the chunk's reach
// covers less than DESC_FRAC of the box is swept through its children
constexpr int DESC_MIN = 64;
constexpr float DESC_FRAC = 0.5f;

// fraction of [lo, hi] inside [a, b] (a point: 1 inside, 0 outside)
__device__ __forceinline__ float overlap_frac(float lo, float hi, float a, float b) {
  const float w = hi - lo;
  const float o = fminf(hi, b) - fmaxf(lo, a);
  return w > 0.f ? fminf(fmaxf(o / w, 0.f), 1.f) : (lo >= a && lo <= b ? 1.f : 0.f);
}

// band of a particle's h above the block's smallest h, HCLASS bands per
// factor 2 (0..15 HCLASS); 31 for particles that need no sweep (converged
// during the h iteration, or with a recorded pair list in a masked sweep)
constexpr int HCLASS = 1;
__device__ __forceinline__ int h_class(const SweepArgs& a, int p, float hmin) {
  if (a.pflag && !(a.pflag[p] & 1)) return 31;
  const float r = a.h[p] / hmin;
  const int c = r < 1.f ? 0 : (int)((float)HCLASS * __log2f(r));
  return c > 15 * HCLASS ? 15 * HCLASS : c;
}

// shared memory of one warp, in float4: j buffer, chunk positions, the
// block's particle order, and (list mode) the per-lane byte lists
template <class P, bool LIST>
__host__ __device__ __forceinline__ int warp_smem_f4(int cap, int bmax) {
  return cap * P::JW + 32 + bmax / 4 + (LIST ? cap * 2 : 0);
}

// The slice of a block cut into several work units that finishes last adds
// the partial sums of all slices in slice order (deterministic whatever the
// finishing order) and finalises; its counter returns to zero for the next
// launch.  No unit waits for another.  (Kept out of line: it runs once per
// sliced block and would otherwise add registers to the whole sweep.)
template <class P, bool COUNT, bool LIST>
__device__ __noinline__ void combine_slices(const SweepArgs& a, int b, int bf, int bn, int nseg) {
  const int lane = threadIdx.x & 31;
  __threadfence();
  __syncwarp();
  int last = 0;
  if (lane == 0) last = atomicAdd(a.blk_done + b, 1) == nseg - 1;
  last = __shfl_sync(FULL, last, 0);
  if (!last) return;
  __threadfence();
  for (int k = lane; k < bn; k += 32) {
    const int p = bf + k;
    if (a.pflag && !(a.pflag[p] & 1)) continue;  // not swept in this launch
    float v[P::NACC];
    int cg = 0;
    for (int sg = 0; sg < nseg; ++sg) {
      const float* pp = a.part + a.b_part[b] + ((size_t)sg * bn + k) * SPH_PART_STRIDE;
#pragma unroll
      for (int kk = 0; kk < P::NACC; ++kk) {
        const float x = __ldcg(pp + kk);
        v[kk] = sg == 0 ? x : (kk >= P::NACC - P::NMAX ? fmaxf(v[kk], x) : v[kk] + x);
      }
      cg += __float_as_int(__ldcg(pp + P::NACC));
    }
    P::finalize(a, p, v);
    if (COUNT && a.ocnt) a.ocnt[p] = cg;
    if (P::WRITES && LIST && a.fl_list) {
      // the particle's list: its slices' lists in slice order, unless one
      // of them overflowed or they do not fit together (then it is swept
      // by the phases that follow)
      static_assert(!P::WRITES || P::NACC + 2 <= SPH_PART_STRIDE, "slice list count slot");
      int tot = 0;
      bool ok = a.sl_list != nullptr;
      for (int sg = 0; sg < nseg && ok; ++sg) {
        const int ci = __float_as_int(
            __ldcg(a.part + a.b_part[b] + ((size_t)sg * bn + k) * SPH_PART_STRIDE + P::NACC + 1));
        ok = ci >= 0;
        tot += ci;
      }
      ok = ok && tot <= a.fl_K;
      if (ok) {
        unsigned* dst = a.fl_list + ((size_t)(p >> 5) * a.fl_K) * 32 + (p & 31);
        int e = 0;
        for (int sg = 0; sg < nseg; ++sg) {
          const long long col = a.b_part[b] / SPH_PART_STRIDE + (long long)sg * bn + k;
          const unsigned* src = a.sl_list + ((size_t)(col >> 5) * a.fl_K) * 32 + (col & 31);
          const int ci = __float_as_int(
              __ldcg(a.part + a.b_part[b] + ((size_t)sg * bn + k) * SPH_PART_STRIDE + P::NACC + 1));
          for (int q = 0; q < ci; ++q, ++e) dst[(size_t)e * 32] = __ldcg(src + (size_t)q * 32);
        }
        a.fl_cnt[p] = tot;
        a.fl_flag[p] = 0;
      } else {
        a.fl_cnt[p] = -1;
        a.fl_flag[p] = 1;
        atomicAdd(a.fl_over, 1);
        atomicAdd(a.fl_over + 1, 1);
        a.fl_blk[b] = 1;
      }
    }
  }
  __syncwarp();
  if (lane == 0) a.blk_done[b] = 0;
}

template <class P, bool COUNT, bool LIST>
__global__ void __launch_bounds__(256, P::MINB) k_sweep(SweepArgs a) {
  extern __shared__ float4 smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cap = a.cap;
  float4* buf = smem + (size_t)warp * warp_smem_f4<P, LIST>(cap, a.bmax);
  float4* cpos = buf + cap * P::JW;  // the chunk's particles (x, y, z, h)
  int* ord = reinterpret_cast<int*>(cpos + 32);  // the block's particles grouped by h class
  unsigned char* lst = reinterpret_cast<unsigned char*>(cpos + 32 + a.bmax / 4);
  const unsigned lt = (1u << lane) - 1u;
  if (a.run_if && *a.run_if == 0) return;
  const int nun = a.nunits_dev ? *a.nunits_dev : a.nunits;
  for (;;) {
    int q = 0;
    if (lane == 0) q = atomicAdd(a.queue, 1);
    q = __shfl_sync(FULL, q, 0);
    if (q >= nun) break;
    const int un = a.order[q];
    const int b = a.u_block[un];
    if (a.blk_active && a.blk_active[b] == 0) continue;
    const int bf = a.b_first[b], bn = a.b_count[b];
    // this unit's slice of the block's interaction list; a block cut into
    // several slices leaves partial sums for the last slice to finish
    const int seg = a.u_seg[un], nseg = a.b_nseg[b];
    const long long e0 = a.u_e0[un], e1 = a.u_e1[un];
    // The block's particles are swept grouped by h class (factor-2 bands
    // above the block's smallest h, Morton order inside a band): chunks share
    // one window per task, set by their largest h, so a few large-h particles
    // must not widen the windows of many small-h ones (a leaf at the edge of
    // a dense clump can hold h values three decades apart).  During the h
    // iteration only particles still iterating are swept.
    float hmin = FLT_MAX;
    for (int k = lane; k < bn; k += 32) hmin = fminf(hmin, a.h[bf + k]);
    hmin = warp_min(hmin);
    unsigned present = 0;
    for (int k = lane; k < bn; k += 32) present |= 1u << h_class(a, bf + k, hmin);
    present = __reduce_or_sync(FULL, present) & 0x7fffffffu;  // class 31: not swept
    while (present) {
      const int cls = __ffs(present) - 1;
      present &= present - 1;
      int ncls = 0;
      for (int k0 = 0; k0 < bn; k0 += 32) {
        const int k = k0 + lane;
        const bool in = k < bn && h_class(a, bf + k, hmin) == cls;
        const unsigned mk = __ballot_sync(FULL, in);
        if (in) ord[ncls + __popc(mk & lt)] = k;
        ncls += __popc(mk);
      }
      __syncwarp();
    for (int c0 = 0; c0 < ncls; c0 += 32) {
      const int nc = min(32, ncls - c0);
      // chunk geometry (positions, bounding box, largest h) with lane k
      // holding chunk particle k
      {
        const int po = bf + ord[c0 + (lane < nc ? lane : 0)];
        const float4 q = a.pos4[po];
        float4 me = make_float4(q.x, q.y, q.z, lane < nc ? a.h[po] : 0.f);
        cpos[lane] = me;
      }
      const float bx0 = warp_min(cpos[lane].x), bx1 = warp_max(cpos[lane].x);
      const float by0 = warp_min(cpos[lane].y), by1 = warp_max(cpos[lane].y);
      const float bz0 = warp_min(cpos[lane].z), bz1 = warp_max(cpos[lane].z);
      const float hmx = warp_max(cpos[lane].w);
      __syncwarp();
      // A chunk of few particles (the last of a block, or a sparse h band:
      // the large-h particles next to a clump, each with 10^4 - 10^5
      // candidates) would leave most lanes idle; there G = 32 / nc lanes
      // (rounded to a power of two) serve each particle, lane l taking chunk
      // particle l / G and every G-th candidate from l % G, and the G partial
      // sums are added at the end.
      const int G = nc > 16 ? 1 : nc > 8 ? 2 : nc > 4 ? 4 : nc > 2 ? 8 : nc > 1 ? 16 : 32;
      const int slot = lane / G, sub = lane & (G - 1);
      const bool vi = slot < nc;
      const int pi = bf + ord[c0 + (vi ? slot : 0)];
      typename P::I I;
      if (vi) P::load_i(a, pi, I); else P::null_i(I);
      float acc[P::NACC], cmp[P::NACC], part[P::NACC];
#pragma unroll
      for (int k = 0; k < P::NACC; ++k) acc[k] = cmp[k] = part[k] = 0.f;
      int cnt = 0, ncand = 0, staged = 0, wtot = 0;
      long long ngath = 0;
      // pair-list column: the particle's own, or for a block cut into
      // slices this slice's column (the last slice concatenates them)
      unsigned* wl = nullptr;
      if (P::WRITES && LIST && a.fl_list && vi) {
        if (nseg == 1) {
          wl = a.fl_list + ((size_t)(pi >> 5) * a.fl_K) * 32 + (pi & 31);
        } else if (a.sl_list) {
          const long long col = a.b_part[b] / SPH_PART_STRIDE + (long long)seg * bn + (pi - bf);
          wl = a.sl_list + ((size_t)(col >> 5) * a.fl_K) * 32 + (col & 31);
        }
      }
      // window of the chunk in one target's sorted list of direction dir
      // (the axial cutoff of the sorted sweep): [js, js + jn) of its ncj
      // entries; hj is the target's largest h (phases over max(h_i, h_j))
      auto window = [&](const float* K, int ncj, int dir, int sgn, float ksh, float hj, int& js,
                        int& jn) {
        const float ux = c_dir[dir][0], uy = c_dir[dir][1], uz = c_dir[dir][2];
        float U = -FLT_MAX, L = FLT_MAX;
        for (int p = 0; p < nc; ++p) {
          const float4 c = cpos[p];
          const float k = sort_key(c.x, c.y, c.z, ux, uy, uz);
          const float ct = P::cut_h(c.w, hj) + a.delta;
          const float sk = sgn < 0 ? -k : k;
          U = fmaxf(U, sk + ct);
          L = fminf(L, k - ct);
        }
        js = 0;
        jn = 0;
        if (ncj <= 0) return;
        if (sgn > 0) {
          SPH_PARTITION(ncj, K[mid] + ksh <= U, jn);
        } else if (sgn < 0) {
          SPH_PARTITION(ncj, -(K[mid] + ksh) > U, js);
          jn = ncj - js;
        } else {
          int je;
          SPH_PARTITION(ncj, K[mid] < L, js);
          SPH_PARTITION(ncj, K[mid] <= U, je);
          jn = max(je - js, 0);
        }
      };
      // flat gather over the 32 lanes' windows (lane l: entries [js, js + jn)
      // of the list at jb, shifted by sh), filtered by the chunk's box, into
      // the shared buffer (a compute pass whenever it fills)
      auto gather = [&](long long jb, int js, int jn, float4 sh, float C2) {
        int incl = jn;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          int y = __shfl_up_sync(FULL, incl, o);
          if (lane >= o) incl += y;
        }
        const int excl = incl - jn;
        const int total = __shfl_sync(FULL, incl, 31);
        if (COUNT && a.units) ngath += total;
        // UNR entries per lane per step, their chains of dependent loads
        // (index, then position) in flight together; the force-like phases,
        // at their register limit, take one
        constexpr int UNR = P::USES_HJ ? 1 : 2;
        for (int f0 = 0; f0 < total; f0 += 32 * UNR) {
          int jx[UNR];
          float4 pv[UNR];
          bool tk[UNR];
          float shx[UNR], shy[UNR], shz[UNR], ck2[UNR];
#pragma unroll
          for (int u = 0; u < UNR; ++u) {
            const int f = f0 + 32 * u + lane;
            int k = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
              int v = __shfl_sync(FULL, excl, k + step);
              if (v <= f) k += step;
            }
            const long long jbk = __shfl_sync(FULL, jb, k);
            const int jsk = __shfl_sync(FULL, js, k);
            const int exk = __shfl_sync(FULL, excl, k);
            shx[u] = __shfl_sync(FULL, sh.x, k);
            shy[u] = __shfl_sync(FULL, sh.y, k);
            shz[u] = __shfl_sync(FULL, sh.z, k);
            ck2[u] = __shfl_sync(FULL, C2, k);
            jx[u] = f < total ? a.s_idx[jbk + jsk + (f - exk)] : -1;
          }
#pragma unroll
          for (int u = 0; u < UNR; ++u) {
            tk[u] = false;
            pv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (jx[u] >= 0) {
              const float4 q = a.pos4[jx[u]];
              pv[u] = make_float4(__fadd_rn(q.x, shx[u]), __fadd_rn(q.y, shy[u]),
                                  __fadd_rn(q.z, shz[u]), q.w);
            }
          }
#pragma unroll
          for (int u = 0; u < UNR; ++u) {
            if (jx[u] >= 0) {
              const float4 pj = pv[u];
              const float dx = fmaxf(fmaxf(bx0 - pj.x, pj.x - bx1), 0.f);
              const float dy = fmaxf(fmaxf(by0 - pj.y, pj.y - by1), 0.f);
              const float dz = fmaxf(fmaxf(bz0 - pj.z, pj.z - bz1), 0.f);
              float lim2 = ck2[u];
              if (P::USES_HJ) {
                const float cj = fmaxf(hmx, a.h[jx[u]]) + a.delta;
                lim2 = cj * cj;
              }
              tk[u] = a.naive || fmaf(dz, dz, fmaf(dy, dy, dx * dx)) <= lim2;
            }
          }
#pragma unroll
          for (int u = 0; u < UNR; ++u) {
            const unsigned mt = __ballot_sync(FULL, tk[u]);
            const int nt = __popc(mt);
            if (staged + nt > cap) {
              compute_pass<P, COUNT, LIST>(I, vi, buf, lst, staged, cap, part, cnt, wl, wtot,
                                           a.fl_K, sub, G);
              if (COUNT && vi && sub < staged) ncand += (staged - sub + G - 1) / G;
              fold<P>(acc, cmp, part, a.kahan);
              staged = 0;
            }
            if (tk[u])
              P::stage(a, jx[u], P::WRITES ? make_tag(jx[u], shx[u], shy[u], shz[u]) : 0u, pv[u],
                       buf, staged + __popc(mt & lt), cap);
            staged += nt;
          }
        }
      };
      // fraction of a target box (shifted) inside the chunk's box grown by C
      auto reach_frac = [&](float4 tlo, float4 thi, float4 sh, float C) {
        return overlap_frac(__fadd_rn(tlo.x, sh.x), __fadd_rn(thi.x, sh.x), bx0 - C, bx1 + C) *
               overlap_frac(__fadd_rn(tlo.y, sh.y), __fadd_rn(thi.y, sh.y), by0 - C, by1 + C) *
               overlap_frac(__fadd_rn(tlo.z, sh.z), __fadd_rn(thi.z, sh.z), bz0 - C, bz1 + C);
      };
      for (long long g = e0; g < e1; g += 32) {
        // ---- one lane per interaction task
        const long long e = g + lane;
        const bool ve = e < e1;
        int cj = 0, code = 1 << 8, ncj = 0;
        float4 sh = make_float4(0.f, 0.f, 0.f, 0.f);
        long long jb = 0;
        float hj = 0.f;
        bool desc = false;
        if (ve) {
          cj = a.dt_cj[e];
          code = a.dt_code[e];
          sh = a.dt_shift[e];
          float4 tlo, thi;
          if (cj >= 0) {  // a cell with sorted lists
            ncj = a.n_count[cj];
            jb = a.n_sbase[cj];
            if (P::USES_HJ) hj = a.n_hmax[cj];
            tlo = a.n_lo[cj];
            thi = a.n_hi[cj];
          } else {        // a block of a cell without them
            const int bj = -1 - cj;
            ncj = a.b_count[bj];
            jb = 13ll * a.b_first[bj];
            if (P::USES_HJ) hj = a.b_hmax[bj];
            tlo = a.b_lo[bj];
            thi = a.b_hi[bj];
          }
          // a target whose box lies beyond the reach of the whole chunk has
          // no candidate (the margin delta covers the rounding of the shift)
          const float gx = fmaxf(fmaxf(__fadd_rn(tlo.x, sh.x) - bx1, bx0 - __fadd_rn(thi.x, sh.x)), 0.f);
          const float gy = fmaxf(fmaxf(__fadd_rn(tlo.y, sh.y) - by1, by0 - __fadd_rn(thi.y, sh.y)), 0.f);
          const float gz = fmaxf(fmaxf(__fadd_rn(tlo.z, sh.z) - bz1, bz0 - __fadd_rn(thi.z, sh.z)), 0.f);
          const float Ct = (P::USES_HJ ? fmaxf(hmx, hj) : hmx) + a.delta;
          if (!a.naive && fmaf(gz, gz, fmaf(gy, gy, gx * gx)) > Ct * Ct) ncj = 0;
          // in a phase over r < max(h_i, h_j), a large target of which the
          // chunk reaches a small part is swept through its children's lists
          // (each with its own box and largest h, where the target's largest
          // h would widen every window), which prunes the far children and
          // narrows the windows
          desc = P::USES_HJ && !a.naive && cj >= 0 && ncj >= DESC_MIN && a.n_child0[cj] >= 0 &&
                 reach_frac(tlo, thi, sh, Ct) < DESC_FRAC;
        }
        const int dir = code & 255, sgn = (code >> 8) - 1;
        jb += (long long)dir * ncj;
        const float ksh = sgn != 0 ? sort_key(sh.x, sh.y, sh.z, c_dir[dir][0], c_dir[dir][1],
                                              c_dir[dir][2])
                                   : 0.f;
        int js = 0, jn = 0;
        if (a.naive) {
          jn = ve ? ncj : 0;  // every particle of the target is a candidate
        } else if (ve && !desc) {
          window(a.s_key + jb, ncj, dir, sgn, ksh, hj, js, jn);
        }
        const float C = (P::USES_HJ ? fmaxf(hmx, hj) : hmx) + a.delta;
        gather(jb, js, jn, sh, C * C);
        // ---- the descended targets, one at a time: lane l < 8 takes child l
        unsigned dm = __ballot_sync(FULL, desc);
        while (dm) {
          const int t = __ffs(dm) - 1;
          dm &= dm - 1;
          const int cjt = __shfl_sync(FULL, cj, t), codet = __shfl_sync(FULL, code, t);
          const float4 sht = make_float4(__shfl_sync(FULL, sh.x, t), __shfl_sync(FULL, sh.y, t),
                                         __shfl_sync(FULL, sh.z, t), 0.f);
          const float kst = __shfl_sync(FULL, ksh, t);
          const int dirt = codet & 255, sgnt = (codet >> 8) - 1;
          int nch = 0, jsc = 0, jnc = 0;
          long long jbc = 0;
          float hjc = 0.f;
          if (lane < 8) {
            const int ch = a.n_child0[cjt] + lane;
            nch = a.n_count[ch];
            if (nch > 0) {
              if (P::USES_HJ) hjc = a.n_hmax[ch];
              const float4 clo = a.n_lo[ch], chi = a.n_hi[ch];
              const float Cc = (P::USES_HJ ? fmaxf(hmx, hjc) : hmx) + a.delta;
              const float gx = fmaxf(fmaxf(__fadd_rn(clo.x, sht.x) - bx1, bx0 - __fadd_rn(chi.x, sht.x)), 0.f);
              const float gy = fmaxf(fmaxf(__fadd_rn(clo.y, sht.y) - by1, by0 - __fadd_rn(chi.y, sht.y)), 0.f);
              const float gz = fmaxf(fmaxf(__fadd_rn(clo.z, sht.z) - bz1, bz0 - __fadd_rn(chi.z, sht.z)), 0.f);
              if (fmaf(gz, gz, fmaf(gy, gy, gx * gx)) > Cc * Cc) nch = 0;  // beyond reach
              jbc = a.n_sbase[ch] + (long long)dirt * a.n_count[ch];
            }
          }
          if (nch > 0) window(a.s_key + jbc, nch, dirt, sgnt, kst, hjc, jsc, jnc);
          const float Cc = (P::USES_HJ ? fmaxf(hmx, hjc) : hmx) + a.delta;
          gather(jbc, jsc, jnc, sht, Cc * Cc);
        }
      }
      compute_pass<P, COUNT, LIST>(I, vi, buf, lst, staged, cap, part, cnt, wl, wtot, a.fl_K, sub,
                                   G);
      if (COUNT && vi && sub < staged) ncand += (staged - sub + G - 1) / G;
      fold<P>(acc, cmp, part, a.kahan);
      float v[P::NACC];
#pragma unroll
      for (int k = 0; k < P::NACC; ++k) v[k] = acc[k] + cmp[k];
      int cg = cnt;
      if (G > 1) {  // the G partial sums of a particle, in a fixed order
        for (int o = G >> 1; o > 0; o >>= 1) {
#pragma unroll
          for (int k = 0; k < P::NACC; ++k) {
            const float y = __shfl_xor_sync(FULL, v[k], o);
            v[k] = k >= P::NACC - P::NMAX ? fmaxf(v[k], y) : v[k] + y;
          }
          cg += __shfl_xor_sync(FULL, cg, o);
        }
      }
      if (nseg > 1) {
        if (vi && sub == 0) {
          float* pp = a.part + a.b_part[b] + ((size_t)seg * bn + (pi - bf)) * SPH_PART_STRIDE;
#pragma unroll
          for (int k = 0; k < P::NACC; ++k) pp[k] = v[k];
          pp[P::NACC] = __int_as_float(cg);
          if (P::WRITES) pp[P::NACC + 1] = __int_as_float(wl ? (wtot > a.fl_K ? -1 : wtot) : -1);
        }
      } else if (vi && sub == 0) {
        P::finalize(a, pi, v);
        if (COUNT && a.ocnt) a.ocnt[pi] = cg;
        if (wl) {
          const bool over = wtot > a.fl_K;
          a.fl_cnt[pi] = over ? -1 : wtot;
          a.fl_flag[pi] = over ? 1 : 0;
          if (over) {
            atomicAdd(a.fl_over, 1);
            a.fl_blk[b] = 1;
          }
        }
      }
      if (COUNT && a.units) {
        int ct = vi ? cnt : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          ct += __shfl_xor_sync(FULL, ct, o);
          ncand += __shfl_xor_sync(FULL, ncand, o);
        }
        if (lane == 0) {
          atomicAdd(a.units, (unsigned long long)ct);
          atomicAdd(a.units + 1, (unsigned long long)ncand);
          atomicAdd(a.units + 2, (unsigned long long)ngath);
        }
      }
      __syncwarp();
    }
    }
    if (nseg > 1) combine_slices<P, COUNT, LIST>(a, b, bf, bn, nseg);
  }
}

// Masked sweeps (the h iteration's later rounds, the overflow sweeps after
// the pair lists) touch few blocks; rather than have every warp claim and
// skip hundreds of thousands of idle units through one atomic counter, the
// units of the active blocks are compacted first, in LPT order: per tile of
// UC_TILE units a count, then each tile adds the counts before it and
// scatters its active units (a ballot scan per warp, the warps in order).
constexpr int UC_TILE = 1024;
constexpr int UC_THREADS = 256;

__device__ __forceinline__ bool unit_on(const SweepArgs& a, int q) {
  return a.blk_active[a.u_block[a.order[q]]] != 0;
}

__global__ void __launch_bounds__(UC_THREADS) k_unit_count(SweepArgs a, int* tcnt) {
  int on = 0;
  const bool run = !a.run_if || *a.run_if != 0;
  for (int k = 0; k < UC_TILE / UC_THREADS; ++k) {
    const int q = blockIdx.x * UC_TILE + k * UC_THREADS + threadIdx.x;
    if (run && q < a.nunits) on += unit_on(a, q) ? 1 : 0;
  }
  on = __reduce_add_sync(FULL, on);
  __shared__ int ws[UC_THREADS / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = on;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < UC_THREADS / 32; ++w) t += ws[w];
    tcnt[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(UC_THREADS) k_unit_compact(SweepArgs a, const int* tcnt,
                                                            int ntiles, int* nact, int* out) {
  __shared__ int ws[UC_THREADS / 32];
  __shared__ int base;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int pre = 0;
  for (int t = threadIdx.x; t < (int)blockIdx.x; t += UC_THREADS) pre += tcnt[t];
  pre = __reduce_add_sync(FULL, pre);
  if (lane == 0) ws[w] = pre;
  __syncthreads();
  if (threadIdx.x == 0) {
    int b = 0;
    for (int k = 0; k < UC_THREADS / 32; ++k) b += ws[k];
    base = b;
  }
  const bool run = !a.run_if || *a.run_if != 0;
  for (int k = 0; k < UC_TILE / UC_THREADS; ++k) {
    __syncthreads();  // base and ws are settled; ws may be overwritten
    const int q = blockIdx.x * UC_TILE + k * UC_THREADS + threadIdx.x;
    const bool on = run && q < a.nunits && unit_on(a, q);
    const unsigned m = __ballot_sync(FULL, on);
    if (lane == 0) ws[w] = __popc(m);
    __syncthreads();
    int off = base;
    for (int v = 0; v < w; ++v) off += ws[v];
    if (on) out[off + __popc(m & ((1u << lane) - 1u))] = a.order[q];
    __syncthreads();  // every thread has read base and ws
    if (threadIdx.x == 0) {
      int t = 0;
      for (int v = 0; v < UC_THREADS / 32; ++v) t += ws[v];
      base += t;
    }
  }
  __syncthreads();
  if (blockIdx.x == ntiles - 1 && threadIdx.x == 0) *nact = base;
}

// replaces the unit order of a masked sweep by the compacted one
int compact_units(sph_ctx* c, SweepArgs& a, cudaStream_t s) {
  if (!a.blk_active || a.nunits == 0) return SPH_OK;
  const int ntiles = div_up(a.nunits, UC_TILE);
  int* tcnt = c->u_act.as<int>();
  int* nact = tcnt + ntiles;
  int* out = nact + 1;
  { k_unit_count<<<ntiles, UC_THREADS, 0, s>>>(a, tcnt); note_launch(); }
  { k_unit_compact<<<ntiles, UC_THREADS, 0, s>>>(a, tcnt, ntiles, nact, out); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  a.order = out;
  a.nunits_dev = nact;
  return SPH_OK;
}

template <class P, bool COUNT, bool LIST>
int launch_shape(sph_ctx* c, SweepArgs& a, cudaStream_t s) {
  const int warps = c->prm.warps_per_cta;
  size_t smem = (size_t)warps * warp_smem_f4<P, LIST>(a.cap, a.bmax) * sizeof(float4);
  auto kern = k_sweep<P, COUNT, LIST>;
  if (smem > 48 * 1024)
    SPH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, nsm = 0, per_sm = c->prm.ctas_per_sm;
  SPH_CUDA(cudaGetDevice(&dev));
  SPH_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (per_sm <= 0) {
    SPH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps, smem));
    if (per_sm <= 0) per_sm = 1;
  }
  int grid = nsm * per_sm;
  int maxgrid = div_up(a.nunits, warps);
  if (grid > maxgrid) grid = maxgrid > 0 ? maxgrid : 1;
  c->sweep_grid = grid;
  c->sweep_threads = 32 * warps;
  SPH_TRY(compact_units(c, a, s));
  SPH_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(int), s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->profile) {
    if (c->ev_pending.size() >= 2048) SPH_TRY(prof_resolve(c));
    a.units = c->prof_units.as<unsigned long long>() + 4 * c->ev_pending.size();
    SPH_CUDA(cudaMemsetAsync(a.units, 0, 4 * sizeof(unsigned long long), s));
    e0 = ev_get(c);
    e1 = ev_get(c);
    SPH_CUDA(cudaEventRecord(e0, s));
  }
  { kern<<<grid, 32 * warps, smem, s>>>(a); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  if (c->profile) {
    SPH_CUDA(cudaEventRecord(e1, s));
    c->ev_pending.push_back({c->cur_phase, e0, e1});
  }
  return SPH_OK;
}

// ---------------------------------------------------------------------------
// a phase over the force pairs (or a subset of them) from the recorded pair
// lists: one lane per particle, 32 consecutive particles per warp, each
// lane walks its own list (coalesced: entry k of the warp's 32 particles is
// one 128-byte row), gathers its j data into registers and applies the
// phase's predicate and interaction; particles whose list overflowed are
// left to a masked sweep
// ---------------------------------------------------------------------------
constexpr int LE_WARPS = 8;

template <class P, bool COUNT>
__global__ void __launch_bounds__(LE_WARPS * 32) k_listeval(SweepArgs a) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long ngrp = (a.n + 31) >> 5;
  for (long long g = (long long)blockIdx.x * LE_WARPS + warp; g < ngrp;
       g += (long long)gridDim.x * LE_WARPS) {
    const long long p = g * 32 + lane;
    const int np = p < a.n ? a.fl_cnt[p] : -1;
    const bool vi = np >= 0;
    typename P::I I;
    if (vi) P::load_i(a, (int)p, I); else P::null_i(I);
    const float et = vi ? a.p_et[p] : 0.f;
    float acc[P::NACC], cmp[P::NACC], part[P::NACC];
#pragma unroll
    for (int k = 0; k < P::NACC; ++k) acc[k] = cmp[k] = part[k] = 0.f;
    int cnt = 0;
    const int nmax = __reduce_max_sync(FULL, vi ? np : 0);
    const unsigned* wl = a.fl_list + ((size_t)g * a.fl_K) * 32 + lane;
    // UNR entries per step, their loads issued before any arithmetic; the j
    // data of an entry sit in registers (a one-slot tile)
    constexpr int UNR = P::JW >= 3 ? 2 : 4;
    constexpr unsigned NONE = 0xffffffffu;  // image code 31: no entry
    for (int k0 = 0; k0 < nmax; k0 += 32) {
      const int k1 = min(nmax, k0 + 32);
      for (int k = k0; k < k1; k += UNR) {
        unsigned e[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) e[u] = k + u < np ? wl[(size_t)(k + u) * 32] : NONE;
        float4 tl[UNR][P::JW];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          if (e[u] != NONE) {
            const int j = (int)(e[u] & TAG_J);
            const int im = (int)(e[u] >> 27);
            const float4 q = a.pos4[j];
            const float4 pj = make_float4(__fadd_rn(q.x, (float)(im / 9 - 1) * et),
                                          __fadd_rn(q.y, (float)((im / 3) % 3 - 1) * et),
                                          __fadd_rn(q.z, (float)(im % 3 - 1) * et), q.w);
            P::stage(a, j, e[u], pj, tl[u], 0, 1);
          }
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u)
          if (e[u] != NONE && P::test(I, tl[u], 0, 1))
            P::template interact<COUNT>(I, tl[u], 0, part, cnt, 1);
      }
      fold<P>(acc, cmp, part, a.kahan);
    }
    if (vi) {
      float v[P::NACC];
#pragma unroll
      for (int k = 0; k < P::NACC; ++k) v[k] = acc[k] + cmp[k];
      P::finalize(a, (int)p, v);
      if (COUNT && a.ocnt) a.ocnt[p] = cnt;
    }
    if (COUNT && a.units) {
      int ct = vi ? cnt : 0, nc = vi ? np : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ct += __shfl_xor_sync(FULL, ct, o);
        nc += __shfl_xor_sync(FULL, nc, o);
      }
      if (lane == 0) {
        atomicAdd(a.units, (unsigned long long)ct);
        atomicAdd(a.units + 1, (unsigned long long)nc);
      }
    }
  }
}

template <class P, bool COUNT>
int launch_listeval(sph_ctx* c, SweepArgs& a, cudaStream_t s) {
  auto kern = k_listeval<P, COUNT>;
  int dev = 0, nsm = 0, per_sm = 0;
  SPH_CUDA(cudaGetDevice(&dev));
  SPH_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  SPH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, LE_WARPS * 32, 0));
  if (per_sm <= 0) per_sm = 1;
  const long long ngrp = (a.n + 31) >> 5;
  int grid = (int)std::min<long long>((long long)nsm * per_sm, div_up(ngrp, LE_WARPS));
  if (grid < 1) grid = 1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->profile) {
    if (c->ev_pending.size() >= 2048) SPH_TRY(prof_resolve(c));
    a.units = c->prof_units.as<unsigned long long>() + 4 * c->ev_pending.size();
    SPH_CUDA(cudaMemsetAsync(a.units, 0, 4 * sizeof(unsigned long long), s));
    e0 = ev_get(c);
    e1 = ev_get(c);
    SPH_CUDA(cudaEventRecord(e0, s));
  }
  { kern<<<grid, LE_WARPS * 32, 0, s>>>(a); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  if (c->profile) {
    SPH_CUDA(cudaEventRecord(e1, s));
    c->ev_pending.push_back({c->cur_phase, e0, e1});
  }
  return SPH_OK;
}

// list mode per phase (bit k of sweep_lists for phase k); byte lists hold
// slots below 256
template <class P, bool COUNT>
int launch(sph_ctx* c, SweepArgs& a, cudaStream_t s) {
  a.cap = c->sweep_cap;
  a.bmax = c->prm.block_max;
  const bool list = a.cap <= 256 && (a.fl_list != nullptr || c->cur_phase == PH_FORCE_VISC ||
                                     (c->cur_phase <= PH_DENSITY_ADJ &&
                                      ((c->prm.sweep_lists >> c->cur_phase) & 1)));
  return list ? launch_shape<P, COUNT, true>(c, a, s) : launch_shape<P, COUNT, false>(c, a, s);
}

// a phase over (a subset of) the force pairs: from the pair lists when the
// force sweep recorded them for the current h, plus a masked sweep of the
// particles whose list overflowed (it returns at once when none did);
// otherwise a plain sweep
template <class P, bool COUNT>
int launch_pairs(sph_ctx* c, SweepArgs& a, cudaStream_t s) {
  if (!c->fl_valid) return launch<P, COUNT>(c, a, s);
  a.fl_list = c->fl_list.as<unsigned>();
  a.fl_cnt = c->fl_cnt.as<int>();
  a.fl_K = c->fl_K;
  a.p_et = c->p_et.as<float>();
  a.n = c->n;
  {
    const int r = launch_listeval<P, COUNT>(c, a, s);
    if (r != SPH_OK) return r;
  }
  SweepArgs f = a;
  f.fl_list = nullptr;
  f.pflag = c->fl_flag.as<int>();
  f.blk_active = c->fl_blk.as<int>();
  f.run_if = c->fl_over.as<int>();
  return launch<P, COUNT>(c, f, s);
}

}  // namespace

cudaEvent_t ev_get(sph_ctx* c) {
  if (c->ev_pool.empty()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  cudaEvent_t e = c->ev_pool.back();
  c->ev_pool.pop_back();
  return e;
}

int prof_resolve(sph_ctx* c) {
  std::vector<unsigned long long> units(4 * c->ev_pending.size());
  if (!units.empty())
    SPH_CUDA(cudaMemcpy(units.data(), c->prof_units.p, units.size() * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost));
  size_t k = 0;
  for (auto& e : c->ev_pending) {
    SPH_CUDA(cudaEventSynchronize(e.b));
    float ms = 0.f;
    SPH_CUDA(cudaEventElapsedTime(&ms, e.a, e.b));
    if (e.phase >= 0 && e.phase < 8) {
      c->prof_ms[e.phase] += ms;
      c->prof_n[e.phase] += 1;
      c->prof_units_acc[e.phase] += units[4 * k];
      c->prof_cand_acc[e.phase] += units[4 * k + 1];
      c->prof_gath_acc[e.phase] += units[4 * k + 2];
    }
    ++k;
    c->ev_pool.push_back(e.a);
    c->ev_pool.push_back(e.b);
  }
  c->ev_pending.clear();
  return SPH_OK;
}

int set_dir_table(sph_ctx* c) {
  if (c->dir_table_set) return SPH_OK;
  float t[SPH_NDIR][3];
  for (int d = 0; d < SPH_NDIR; ++d) dir_unit(d, t[d][0], t[d][1], t[d][2]);
  SPH_CUDA(cudaMemcpyToSymbol(c_dir, t, sizeof(t)));
  c->dir_table_set = true;
  return SPH_OK;
}

int run_sweep(sph_ctx* c, int phase, int only_active, int counting, cudaStream_t s) {
  if (c->nblock == 0) return SPH_OK;
  c->cur_phase = phase;
  if (c->profile && phase != PH_DUMP_DENSITY && phase != PH_DUMP_FORCE) counting = 1;
  SPH_TRY(set_dir_table(c));
  SweepArgs a{};
  a.nblock = c->nblock;
  a.nunits = c->nunits;
  a.order = c->b_order.as<int>();
  a.u_block = c->u_block.as<int>();
  a.u_seg = c->u_seg.as<int>();
  a.u_e0 = c->u_e0.as<long long>();
  a.u_e1 = c->u_e1.as<long long>();
  a.b_nseg = c->b_nseg.as<int>();
  a.b_part = c->b_part.as<long long>();
  a.part = c->part.as<float>();
  a.blk_done = c->blk_done.as<int>();
  a.b_first = c->b_first.as<int>();
  a.b_count = c->b_count.as<int>();
  a.b_dtoff = c->b_dtoff.as<long long>();
  a.dt_cj = c->dt_cj.as<int>();
  a.dt_code = c->dt_code.as<int>();
  a.dt_shift = c->dt_shift.as<float4>();
  a.n_count = c->n_count.as<int>();
  a.n_sbase = c->n_sbase.as<long long>();
  a.n_child0 = c->n_child0.as<int>();
  a.n_hmax = c->n_hmax.as<float>();
  a.b_hmax = c->b_hmax.as<float>();
  a.n_lo = c->n_lo.as<float4>();
  a.n_hi = c->n_hi.as<float4>();
  a.b_lo = c->b_lo.as<float4>();
  a.b_hi = c->b_hi.as<float4>();
  a.s_key = c->s_key.as<float>();
  a.s_idx = c->s_idx.as<int>();
  a.pos4 = c->pos4.as<float4>();
  a.h = c->h.as<float>();
  a.vel4 = c->vel4.as<float4>();
  a.fdat = c->fdat.as<float4>();
  a.blk_active = only_active ? c->blk_active.as<int>() : nullptr;
  a.pflag = only_active ? c->h_flag.as<int>() : nullptr;
  a.queue = c->queue.as<int>();
  a.status = c->status.as<int>();
  double emax = 0;
  for (int b = 0; b < c->nbox; ++b) emax = std::max(emax, c->box_L[b] / (double)(1 << c->box_t[b]));
  // margin of the axial cutoff and the box tests: the rounding of the FP32
  // keys and shifts, plus twice the largest displacement since the build
  // when positions were moved without rebuilding (stale keys and boxes)
  a.delta = (float)(emax * (1.0 / 65536.0)) + c->reuse_pad;
  a.kahan = c->prm.kahan ? 1 : 0;
  a.naive = c->prm.sorted_sweep ? 0 : 1;
  a.ocnt = counting ? c->cnt_i.as<int>() : nullptr;
  switch (phase) {
    case PH_DENSITY:
      a.o0 = c->rho.as<float>();
      a.o1 = c->drho.as<float>();
      a.o2 = c->nngb.as<float>();
      a.o3 = c->dnngb.as<float>();
      a.o6 = c->d2nngb.as<float>();
      return counting ? launch<PDensity, true>(c, a, s) : launch<PDensity, false>(c, a, s);
    case PH_DENSITY_D2:
      a.o0 = c->d2rho.as<float>();
      return counting ? launch_pairs<PDensityD2, true>(c, a, s)
                      : launch_pairs<PDensityD2, false>(c, a, s);
    case PH_FORCE:
      a.o4 = c->acc4.as<float4>();
      c->fl_valid = false;
      if (c->prm.pair_list_cap > 0 && c->sweep_cap <= 256 && c->n < (1ll << 27)) {
        const long long ng = (c->n + 31) >> 5;
        SPH_TRY(dbuf_ensure(c->fl_list, sizeof(unsigned) * (size_t)ng * 32 * c->prm.pair_list_cap));
        SPH_TRY(dbuf_ensure(c->fl_cnt, sizeof(int) * (size_t)c->n));
        SPH_TRY(dbuf_ensure(c->fl_flag, sizeof(int) * (size_t)c->n));
        SPH_TRY(dbuf_ensure(c->fl_blk, sizeof(int) * (size_t)c->nblock));
        SPH_TRY(dbuf_ensure(c->fl_over, 64));
        SPH_CUDA(cudaMemsetAsync(c->fl_blk.p, 0, sizeof(int) * (size_t)c->nblock, s));
        SPH_CUDA(cudaMemsetAsync(c->fl_over.p, 0, 2 * sizeof(int), s));
        c->fl_K = c->prm.pair_list_cap;
        a.sl_list = nullptr;
        if (c->part_cols > 0) {  // lists of the slices of blocks cut into work units
          const size_t cols = (size_t)((c->part_cols + 31) / 32) * 32;
          SPH_TRY(dbuf_ensure(c->sl_list, sizeof(unsigned) * cols * c->prm.pair_list_cap));
          a.sl_list = c->sl_list.as<unsigned>();
        }
        a.fl_list = c->fl_list.as<unsigned>();
        a.fl_cnt = c->fl_cnt.as<int>();
        a.fl_flag = c->fl_flag.as<int>();
        a.fl_blk = c->fl_blk.as<int>();
        a.fl_over = c->fl_over.as<int>();
        a.fl_K = c->fl_K;
        const int r = counting ? launch<PForce, true>(c, a, s) : launch<PForce, false>(c, a, s);
        if (r != SPH_OK) return r;
        c->fl_valid = true;
        return SPH_OK;
      }
      return counting ? launch<PForce, true>(c, a, s) : launch<PForce, false>(c, a, s);
    case PH_FORCE_ADJ:
      a.adj4 = c->adj4.as<float4>();
      a.o4 = c->g_x4.as<float4>();
      a.o0 = c->g_A.as<float>();
      a.o1 = c->g_h_s.as<float>();
      return counting ? launch_pairs<PForceAdj, true>(c, a, s)
                      : launch_pairs<PForceAdj, false>(c, a, s);
    case PH_DENSITY_ADJ:
      a.adj4 = c->adj4.as<float4>();
      a.adj4b = c->adj4b.as<float4>();
      a.o4 = c->g_x4.as<float4>();
      return counting ? launch_pairs<PDensityAdj, true>(c, a, s)
                      : launch_pairs<PDensityAdj, false>(c, a, s);
    case PH_VELDERIV:
      a.rho_in = c->rho.as<float>();
      a.u_in = c->u_s.as<float>();
      a.gamma = c->prm.gamma;
      a.o5 = c->visc4.as<float4>();
      return counting ? launch<PVelDeriv, true>(c, a, s) : launch<PVelDeriv, false>(c, a, s);
    case PH_FORCE_VISC:
      a.visc4 = c->visc4.as<float4>();
      a.alpha = c->visc_alpha;
      a.c_cfl = c->visc_cfl;
      a.o4 = c->acc4.as<float4>();
      a.o0 = c->dt_s.as<float>();
      return counting ? launch<PForceVisc, true>(c, a, s) : launch<PForceVisc, false>(c, a, s);
    case PH_DUMP_DENSITY:
    case PH_DUMP_FORCE:
      a.perm = c->perm.as<int>();
      a.dump_i = c->dump_pi;
      a.dump_j = c->dump_pj;
      a.dump_n = c->counters.as<unsigned long long>();
      a.dump_cap = c->dump_cap;
      a.kahan = 0;
      a.cap = c->sweep_cap;
      a.bmax = c->prm.block_max;
      return phase == PH_DUMP_DENSITY ? launch_shape<PDump<0>, false, false>(c, a, s)
                                      : launch_shape<PDump<1>, false, false>(c, a, s);
    default:
      return SPH_ERR_INVALID_ARG;
  }
}
